// The succinct lookup table that Section 7 proposes for the tetrahedral map:
// the layer starts T3(k) = k(k+1)(k+2)/6 for every k whose start lies below
// 2^32 (2953 words, 11.8 KB), fixed at build time in constant memory.  A
// block finds its layer as the largest k < m with T3(k) <= omega by binary
// search: every thread of a block searches the same omega, so each step is
// one broadcast read of the constant cache instead of the cube and square
// roots of the closed form.  The table has O(T_n^(1/3)) entries, o(T_n).
#pragma once

#include <cstdint>

namespace tri {

constexpr uint32_t TET_TABLE_LAYERS = 2953;  // k = 0 .. 2952: T3(2952) < 2^32 <= T3(2953)

struct TetStarts {
    uint32_t v[TET_TABLE_LAYERS];
};

constexpr TetStarts make_tet_starts()
{
    TetStarts t{};
    for (uint32_t k = 0; k < TET_TABLE_LAYERS; ++k) {
        t.v[k] = (uint32_t)((uint64_t)k * (k + 1) * (k + 2) / 6);
    }
    return t;
}

static __constant__ TetStarts c_tet_starts = make_tet_starts();

// Layer of block omega among m <= TET_TABLE_LAYERS layers (omega < T3(m)).
__device__ __forceinline__ uint32_t tet_layer_table(uint32_t w, uint32_t m)
{
    uint32_t lo = 0, hi = m;  // T3(lo) <= w < T3(hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (c_tet_starts.v[mid] <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void tet_block_table(uint32_t w, uint32_t m, uint32_t &L, uint32_t &R, uint32_t &C)
{
    L = tet_layer_table(w, m);
    lambda_diag<TRI_SQRT_R>((uint32_t)(w - c_tet_starts.v[L]), R, C);
}

}  // namespace tri
