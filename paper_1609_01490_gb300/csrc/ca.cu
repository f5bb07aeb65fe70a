// One synchronous step of an outer-totalistic cellular automaton on the
// triangular domain {0 <= j <= i < n}, shared-memory halo tiles placed by a
// block map (Section 5's shared-memory scenario, applied to the cellular
// automaton that Section 1 lists among the TD problems).
#include <cuda_runtime.h>

#include "tri_maps.cuh"

using namespace tri;

namespace {

// Tile: S x S cells, S = 4*RHO.  Thread (ty, tx) owns the 4-cell word tx of
// the four consecutive tile rows 4ty .. 4ty+3.  The halo tile holds S+2 rows
// of RHO+2 words (one word either side), cell bytes normalised to 0/1 and
// zeroed outside the domain.
// LIFE: the rule is Conway's (birth on 3, survival on 2 or 3), evaluated with
// two SIMD byte compares on the 3 x 3 sum including the cell itself (alive
// next iff the sum is 3, or 4 with the cell alive); otherwise the general
// outer-totalistic rule is looked up per byte in `table`.
template <int MAP, int RHO, bool LIFE>
__global__ void __launch_bounds__(RHO *RHO) ca_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                                      uint32_t n, size_t ld, uint32_t table, BlockMap bm)
{
    constexpr int S = 4 * RHO, W = RHO + 2, H = S + 2;
    __shared__ uint32_t halo[H][W];
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RHO + tx;
    const long long row0 = (long long)bi * S - 1;    // global row of halo row 0
    const long long wc0 = (long long)bj * RHO - 1;   // global word column of halo word 0

    for (int t = tid; t < H * W; t += RHO * RHO) {
        const int y = t / W, w = t - y * W;
        const long long a = row0 + y, wc = wc0 + w;
        uint32_t v = 0;
        if (a >= 0 && a < (long long)n && wc >= 0 && 4 * wc <= a) {
            v = *reinterpret_cast<const uint32_t *>(in + (size_t)a * ld + 4 * wc);
            v = __vcmpne4(v, 0u) & 0x01010101u;            // alive -> 1
            const long long over = 4 * wc + 3 - a;         // bytes past the diagonal
            if (over > 0) v &= 0xFFFFFFFFu >> (8 * over);  // cells j > a are outside
        }
        halo[y][w] = v;
    }
    __syncthreads();

    // horizontal 3-sums of halo rows 4ty .. 4ty+5
    uint32_t hs[6], ctr[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int y = 4 * ty + q;
        const uint32_t L = halo[y][tx], C = halo[y][tx + 1], R = halo[y][tx + 2];
        hs[q] = __funnelshift_l(L, C, 8) + C + __funnelshift_r(C, R, 8);
        ctr[q] = C;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long a = row0 + 1 + 4 * ty + q;
        if (a >= (long long)n) break;
        const long long wc = wc0 + 1 + tx;
        if (4 * wc > a) continue;
        const uint32_t alive = ctr[q + 1];
        const uint32_t sum = hs[q] + hs[q + 1] + hs[q + 2];  // 3 x 3 sum, 0..9 per byte
        uint32_t nxt = 0;
        if constexpr (LIFE) {
            nxt = (__vcmpeq4(sum, 0x03030303u) | (__vcmpeq4(sum, 0x04040404u) & (alive * 0xFFu))) & 0x01010101u;
        } else {
            const uint32_t idx = sum + (alive << 3);  // count + 9*alive = sum - alive + 9*alive
#pragma unroll
            for (int b = 0; b < 4; ++b) nxt |= ((table >> ((idx >> (8 * b)) & 0xFFu)) & 1u) << (8 * b);
        }
        uint8_t *dst = out + (size_t)a * ld + 4 * wc;
        if (4 * wc + 3 <= a) {
            *reinterpret_cast<uint32_t *>(dst) = nxt;
        } else {
            for (int b = 0; 4 * wc + b <= a; ++b) dst[b] = (uint8_t)(nxt >> (8 * b));
        }
    }
}

template <int MAP, bool LIFE>
void launch_rule(uint32_t rho, dim3 g, cudaStream_t s, const uint8_t *in, uint8_t *out, uint32_t n, size_t ld,
                 uint32_t table, BlockMap bm)
{
    switch (rho) {
    case 8: ca_kernel<MAP, 8, LIFE><<<g, dim3(8, 8), 0, s>>>(in, out, n, ld, table, bm); break;
    case 16: ca_kernel<MAP, 16, LIFE><<<g, dim3(16, 16), 0, s>>>(in, out, n, ld, table, bm); break;
    default: ca_kernel<MAP, 32, LIFE><<<g, dim3(32, 32), 0, s>>>(in, out, n, ld, table, bm); break;
    }
}

// Conway's rule as a table: birth on 3 (bit 3), survival on 2 or 3 (bits 9 + 2, 9 + 3).
constexpr uint32_t LIFE_TABLE = (1u << 3) | (1u << (9 + 2)) | (1u << (9 + 3));

template <int MAP>
cudaError_t launch_rho(uint32_t rho, dim3 g, cudaStream_t s, const uint8_t *in, uint8_t *out, uint32_t n, size_t ld,
                       uint32_t table, BlockMap bm)
{
    if (table == LIFE_TABLE) launch_rule<MAP, true>(rho, g, s, in, out, n, ld, table, bm);
    else launch_rule<MAP, false>(rho, g, s, in, out, n, ld, table, bm);
    return cudaGetLastError();
}

}  // namespace

extern "C" int tri_ca_step(const uint8_t *in, uint8_t *out, uint32_t n, size_t ld, uint32_t birth_mask,
                           uint32_t survive_mask, int map, uint32_t rho, void *stream)
{
    if (!in || !out || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (ld < n || (ld & 15) || ((uintptr_t)in & 3) || ((uintptr_t)out & 3)) return TRI_EINVAL;
    // no aliasing: the two buffers of n rows must not overlap
    const size_t span = (size_t)(n - 1) * ld + n;
    if ((in < out + span) && (out < in + span)) return TRI_EINVAL;
    if ((birth_mask | survive_mask) >> 9) return TRI_EINVAL;
    const uint32_t table = birth_mask | (survive_mask << 9);  // bit count + 9*alive
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t S = 4 * rho, m = (n + S - 1) / S;
    BlockMap bm{};
    bm.m = m;
    bm.nblocks = T2(m);
    cudaError_t e = cudaSuccess;
    switch (map) {
    case TRI_MAP_LAMBDA:
        e = launch_rho<MAP_LAMBDA>(rho, trihost::linear_grid(bm.nblocks), s, in, out, n, ld, table, bm);
        break;
    case TRI_MAP_LAMBDA_PDELTA: {
        const uint64_t mp = trihost::isqrt_ceil(bm.nblocks);
        e = launch_rho<MAP_LAMBDA_PD>(rho, dim3((unsigned)mp, (unsigned)mp), s, in, out, n, ld, table, bm);
        break;
    }
    case TRI_MAP_BB:
        e = launch_rho<MAP_BB>(rho, dim3(m, m), s, in, out, n, ld, table, bm);
        break;
    case TRI_MAP_RB: {
        const uint32_t h = (m & 1u) ? (m + 1) / 2 : m / 2 + 1;
        e = launch_rho<MAP_RB>(rho, dim3(m, h), s, in, out, n, ld, table, bm);
        break;
    }
    case TRI_MAP_REC: {
        if (!trihost::is_pow2(m)) return TRI_ERANGE;
        const uint32_t k = trihost::ilog2(m);
        for (uint32_t l = 0; l <= k && e == cudaSuccess; ++l) {
            bm.level = l;
            const dim3 g = l == 0 ? dim3(m) : dim3(1u << (l - 1), m / 2);
            e = launch_rho<MAP_REC>(rho, g, s, in, out, n, ld, table, bm);
        }
        break;
    }
    default:
        return TRI_EINVAL;
    }
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}
