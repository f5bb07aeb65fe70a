// Block- and thread-space maps onto triangular and tetrahedral domains.
//
// lambda(omega) (Section 3.1, Eq. eq_gmap and Eq. eq_theorem_nodiag), the
// square-root estimates of Section 4.1, the comparison maps of Section 4.2
// (BB, RB, REC, UTM) and the tetrahedral map of Section 6.  Every map that
// takes a floating-point root is followed by an exact integer correction
// against the row (or layer) starts, so its result is the exact one for every
// input in range; the estimates differ only in cost.
#pragma once

#include <cstdint>
#include <type_traits>

#include "../../include/tri.h"

namespace tri {

// T(i) = i(i+1)/2: first block number of row i in the enumeration matrix
// (Eq. eq_matrix_indexing).
__host__ __device__ __forceinline__ uint64_t T2(uint64_t i) { return (i * (i + 1)) >> 1; }

// T3(k) = k(k+1)(k+2)/6: first block number of layer k of the tetrahedron
// (Section 6).
__host__ __device__ __forceinline__ uint64_t T3(uint64_t k) { return k * (k + 1) * (k + 2) / 6; }

// ---------------------------------------------------------------- sqrt ----
// Estimate of sqrt(x) for x >= 0.25 by the three strategies of Section 4.1.
template <int SQ>
__device__ __forceinline__ float sqrt_estimate(float x)
{
    if constexpr (SQ == TRI_SQRT_X) {
        return sqrtf(x);
    } else if constexpr (SQ == TRI_SQRT_R) {
        return x * rsqrtf(x);
    } else {
        // Fast inverse square root (C. Lomont, "Fast inverse square root",
        // 2003): halve the exponent by an integer shift subtracted from the
        // magic constant, then refine y ~ 1/sqrt(x) with Newton's iteration
        // y <- y (3/2 - x/2 y^2), three times.
        const float h = 0.5f * x;
        float y = __int_as_float(0x5f3759df - (__float_as_int(x) >> 1));
        y = y * (1.5f - h * y * y);
        y = y * (1.5f - h * y * y);
        y = y * (1.5f - h * y * y);
        return x * y;
    }
}

// -------------------------------------------------------------- lambda ----
// Eq. eq_gmap: omega -> (i, j), i = floor(sqrt(1/4 + 2 omega) - 1/2),
// j = omega - i(i+1)/2, for every omega < 2^32.  The FP32 estimate of i is
// within one row of the true one over that whole range (checked exhaustively
// by tri_lambda_verify), so one integer step fixes it.
template <int SQ>
__device__ __forceinline__ void lambda_diag(uint32_t w, uint32_t &i, uint32_t &j)
{
    const float est = sqrt_estimate<SQ>(fmaf(2.0f, (float)w, 0.25f)) - 0.5f;
    uint32_t r = __float2uint_rz(est);  // floor; negative estimates saturate to 0
    long long c = (long long)w - (long long)T2(r);
    if (c < 0) {
        --r;
        c += r + 1;
    } else if (c > (long long)r) {
        c -= r + 1;
        ++r;
    }
    i = r;
    j = (uint32_t)c;
}

// Eq. eq_theorem_nodiag: strict triangle j < i.  Row i holds i blocks and
// starts at i(i-1)/2 (the printed j = omega - i(i+1)/2 is negative at omega
// = 0; the row start that makes the enumeration consistent is i(i-1)/2).
template <int SQ>
__device__ __forceinline__ void lambda_nodiag(uint32_t w, uint32_t &i, uint32_t &j)
{
    const float est = sqrt_estimate<SQ>(fmaf(2.0f, (float)w, 0.25f)) + 0.5f;
    uint32_t r = __float2uint_rz(est);
    if (r == 0) r = 1;
    long long c = (long long)w - (long long)T2(r - 1);
    if (c < 0) {
        --r;
        c += r;
    } else if (c >= (long long)r) {
        c -= r;
        ++r;
    }
    i = r;
    j = (uint32_t)c;
}

// ---------------------------------------------------------- block maps ----
// A block map turns blockIdx into a block (bi, bj) of the with-diagonal
// triangle of m block rows, or reports that the block has no work.
struct BlockMap {
    uint64_t nblocks;  // lambda: one past the last block number (m(m+1)/2 for the whole triangle)
    uint32_t m;        // block rows of the triangle
    uint32_t level;    // REC: 0 = diagonal pass, l >= 1 = squares of side 2^(l-1)
    uint64_t w0;       // lambda: the block number of grid position 0 (a band of block rows
                       // [R0, R1) is the range [T(R0), T(R1)) of lambda's numbering)
};

enum : int {
    MAP_LAMBDA = TRI_MAP_LAMBDA,
    MAP_BB = TRI_MAP_BB,
    MAP_RB = TRI_MAP_RB,
    MAP_REC = TRI_MAP_REC,
    MAP_UTM = TRI_MAP_UTM,
    MAP_LAMBDA_PD = TRI_MAP_LAMBDA_PDELTA,
    MAP_TET_TABLE = TRI_MAP_TET_TABLE,
    MAP_LAMBDA_ND = 100  // strict lambda (Eq. eq_theorem_nodiag), shifted by one row
};

// The block of grid position (bx, by) in a grid of gx columns: map_block
// for the running block, and for any other position of the same launch (a
// kernel may prefetch for the block that will run a given number of
// positions later).
template <int MAP, int SQ = TRI_SQRT_R>
__device__ __forceinline__ bool map_block_at(const BlockMap &a, uint32_t bx, uint32_t by, uint32_t gx, uint32_t &bi,
                                             uint32_t &bj)
{
    if constexpr (MAP == MAP_LAMBDA || MAP == MAP_LAMBDA_PD || MAP == MAP_LAMBDA_ND) {
        // omega from the (1-D, 2-D or P_Delta) grid, row-major over the grid
        const uint64_t w = a.w0 + (uint64_t)by * gx + bx;
        if (w >= a.nblocks) return false;
        if constexpr (MAP == MAP_LAMBDA_ND) {
            uint32_t I;
            lambda_nodiag<SQ>((uint32_t)w, I, bj);
            bi = I - 1;  // strict row I >= 1 covers with-diagonal row I - 1
        } else {
            lambda_diag<SQ>((uint32_t)w, bi, bj);
        }
        return true;
    } else if constexpr (MAP == MAP_BB) {
        // Section 4.2: the m x m box; blocks above the diagonal leave at once
        bi = by;
        bj = bx;
        return bj <= bi;
    } else if constexpr (MAP == MAP_RB) {
        // Section 4.2, rectangular box: the part of the box right of the
        // diagonal is rotated under it.  Grid: m columns x h rows, h =
        // (m+1)/2 for odd m, m/2 + 1 for even m (whose last row is half used).
        const uint32_t tx = bx, ty = by, m = a.m;
        if (tx < ty) {
            bi = ty - 1;
            bj = tx;
        } else {
            if ((m & 1u) == 0 && ty == m / 2) return false;
            bi = m - ty - 1;
            bj = m - tx - 1;
        }
        return true;
    } else if constexpr (MAP == MAP_REC) {
        // Recursive partition (Ries et al.), bottom-up over m = 2^k block
        // rows: level 0 is the diagonal pass; level l holds 2^(k-l) squares of
        // side s = 2^(l-1) blocks, square q covering block rows
        // [q 2^l + s, (q+1) 2^l) and block columns [q 2^l, q 2^l + s).
        if (a.level == 0) {
            bi = bj = bx;
        } else {
            const uint32_t s = 1u << (a.level - 1);
            const uint32_t q = by >> (a.level - 1), r = by & (s - 1);
            bi = (q << a.level) + s + r;
            bj = (q << a.level) + bx;
        }
        return true;
    } else {
        return false;
    }
}

template <int MAP, int SQ = TRI_SQRT_R>
__device__ __forceinline__ bool map_block(const BlockMap &a, uint32_t &bi, uint32_t &bj)
{
    return map_block_at<MAP, SQ>(a, blockIdx.x, blockIdx.y, gridDim.x, bi, bj);
}

// The block `ahead` grid positions after the running one (row-major over the
// grid), if that position exists and maps to a block.
template <int MAP, int SQ = TRI_SQRT_R>
__device__ __forceinline__ bool map_block_ahead(const BlockMap &a, uint32_t ahead, uint32_t &bi, uint32_t &bj)
{
    const uint64_t lin = (uint64_t)blockIdx.y * gridDim.x + blockIdx.x + ahead;
    const uint64_t y = lin / gridDim.x;
    if (y >= gridDim.y) return false;
    return map_block_at<MAP, SQ>(a, (uint32_t)(lin - y * gridDim.x), (uint32_t)y, gridDim.x, bi, bj);
}

// --------------------------------------------------------------- UTM ----
// Upper-triangular map of Avril et al. (Section 4.2), thread space, 1-indexed:
// thread k of N(N-1)/2 -> (a, b), 1 <= a < b <= N, row a starting at
// S(a) = (a-1)(2N-a)/2:  a = floor(((2N+1) - sqrt((2N-1)^2 - 8k)) / 2),
// b = a + 1 + k - S(a).  The discriminant is formed in 64-bit integers and
// only its root is taken in FP32, followed by an exact correction of a.
__device__ __forceinline__ void utm_pair(uint64_t k, uint64_t N, uint32_t &a_out, uint32_t &b_out)
{
    const uint64_t disc = (2 * N - 1) * (2 * N - 1) - 8 * k;
    const float est = 0.5f * ((float)(2 * N + 1) - sqrtf((float)disc));
    long long a = (long long)est;
    if (a < 1) a = 1;
    auto S = [N](long long t) { return (uint64_t)((t - 1) * (long long)(2 * N - t) / 2); };
    while (a > 1 && S(a) > k) --a;
    while (S(a + 1) <= k) ++a;
    a_out = (uint32_t)a;
    b_out = (uint32_t)((uint64_t)a + 1 + k - S(a));
}

// ---------------------------------------------------------- tetrahedron ----
// Section 6: omega -> layer k = floor(x), x the real root of
// x^3 + 3x^2 + 2x - 6 omega = 0, by the closed form printed there (Cardano),
// evaluated in FP32 and corrected exactly against T3; omega = 0 (where the
// closed form takes the root of a negative number) is layer 0.  Then the 2-D
// lambda of omega - T3(k) gives (row, col).
__device__ __forceinline__ uint32_t tet_layer(uint32_t w)
{
    uint32_t k = 0;
    if (w != 0) {
        const float fw = (float)w;
        const float s = cbrtf(sqrtf(fmaf(729.0f * fw, fw, -3.0f)) + 27.0f * fw);
        // 3^(-2/3) and 3^(-1/3)
        const float x = s * 0.48074985f + 0.69336127f / s - 1.0f;
        k = __float2uint_rz(fmaxf(x, 0.0f));
    }
    while (k > 0 && T3(k) > w) --k;
    while (T3(k + 1) <= w) ++k;
    return k;
}

__device__ __forceinline__ void tet_block(uint32_t w, uint32_t &L, uint32_t &R, uint32_t &C)
{
    L = tet_layer(w);
    lambda_diag<TRI_SQRT_R>((uint32_t)(w - T3(L)), R, C);
}

}  // namespace tri

// ------------------------------------------------------------------ host ----
namespace trihost {

inline bool rho_ok(uint32_t rho) { return rho == 8 || rho == 16 || rho == 32; }

inline bool is_pow2(uint32_t v) { return v && !(v & (v - 1)); }

inline uint32_t ilog2(uint32_t v)
{
    uint32_t r = 0;
    while (v >>= 1) ++r;
    return r;
}

// 1-D grid for nb blocks when it fits gridDim.x, else a 2-D grid whose
// row-major numbering covers nb with fewer than gy spare blocks.
inline dim3 linear_grid(uint64_t nb)
{
    const uint64_t maxx = 0x7FFFFFFFull;
    if (nb <= maxx) return dim3((unsigned)nb, 1, 1);
    const uint64_t gy = (nb + maxx - 1) / maxx;
    return dim3((unsigned)((nb + gy - 1) / gy), (unsigned)gy, 1);
}

// ceil(sqrt(v)) for v < 2^64 by integer search
inline uint64_t isqrt_ceil(uint64_t v)
{
    uint64_t r = 0;
    for (int b = 31; b >= 0; --b) {
        const uint64_t t = r | (1ull << b);
        if (t * t <= v) r = t;
    }
    return r * r == v ? r : r + 1;
}

// Whether a 2-D block map can cover m block rows with CUDA's grid limits:
// TRI_OK, TRI_ERANGE (too many blocks; REC with m not a power of two) or
// TRI_EINVAL (not a 2-D block map).  m is taken in 64 bits so that a block
// count computed from n near 2^32 cannot wrap.
inline int map_range(int map, uint64_t m)
{
    switch (map) {
    case TRI_MAP_LAMBDA: return m <= 0xFFFFFFFFull && tri::T2(m) <= 0xFFFFFFFFull ? TRI_OK : TRI_ERANGE;
    case TRI_MAP_LAMBDA_PDELTA:
        return m <= 0xFFFFFFFFull && tri::T2(m) <= 0xFFFFFFFFull && isqrt_ceil(tri::T2(m)) <= 65535 ? TRI_OK
                                                                                                    : TRI_ERANGE;
    case TRI_MAP_BB: return m <= 65535 ? TRI_OK : TRI_ERANGE;
    case TRI_MAP_RB: return ((m & 1u) ? (m + 1) / 2 : m / 2 + 1) <= 65535 && m <= 65535 * 2 ? TRI_OK : TRI_ERANGE;
    case TRI_MAP_REC:
        return m <= 0xFFFFFFFFull && is_pow2((uint32_t)m) && (m < 2 || m / 2 <= 65535) ? TRI_OK : TRI_ERANGE;
    default: return TRI_EINVAL;
    }
}

// The launches of a 2-D block map over m block rows: go(tag, grid, bm) is
// called once per launch (REC: once per level) with tag an
// std::integral_constant holding the kernel's MAP; returns a tri_status.
template <class Go>
int map_launches(int map, uint32_t m, Go &&go)
{
    using tri::BlockMap;
    BlockMap bm{};
    bm.m = m;
    bm.nblocks = tri::T2(m);
    cudaError_t e = cudaSuccess;
    switch (map) {
    case TRI_MAP_LAMBDA:
        if (bm.nblocks > 0xFFFFFFFFull) return TRI_ERANGE;
        e = go(std::integral_constant<int, tri::MAP_LAMBDA>{}, linear_grid(bm.nblocks), bm);
        break;
    case TRI_MAP_LAMBDA_PDELTA: {
        if (bm.nblocks > 0xFFFFFFFFull) return TRI_ERANGE;
        const uint64_t mp = isqrt_ceil(bm.nblocks);
        if (mp > 65535) return TRI_ERANGE;
        e = go(std::integral_constant<int, tri::MAP_LAMBDA_PD>{}, dim3((unsigned)mp, (unsigned)mp), bm);
        break;
    }
    case TRI_MAP_BB:
        if (m > 65535) return TRI_ERANGE;
        e = go(std::integral_constant<int, tri::MAP_BB>{}, dim3(m, m), bm);
        break;
    case TRI_MAP_RB: {
        const uint32_t h = (m & 1u) ? (m + 1) / 2 : m / 2 + 1;
        if (h > 65535) return TRI_ERANGE;
        e = go(std::integral_constant<int, tri::MAP_RB>{}, dim3(m, h), bm);
        break;
    }
    case TRI_MAP_REC: {
        if (!is_pow2(m)) return TRI_ERANGE;
        const uint32_t k = ilog2(m);
        if (k > 0 && m / 2 > 65535) return TRI_ERANGE;
        for (uint32_t l = 0; l <= k && e == cudaSuccess; ++l) {
            bm.level = l;
            const dim3 g = l == 0 ? dim3(m) : dim3(1u << (l - 1), m / 2);
            e = go(std::integral_constant<int, tri::MAP_REC>{}, g, bm);
        }
        break;
    }
    default:
        return TRI_EINVAL;
    }
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

}  // namespace trihost
