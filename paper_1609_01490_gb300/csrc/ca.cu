// One synchronous step of an outer-totalistic cellular automaton on the
// triangular domain {0 <= j <= i < n}, shared-memory halo tiles placed by a
// block map (Section 5's shared-memory scenario, applied to the cellular
// automaton that Section 1 lists among the TD problems).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "tri_maps.cuh"

using namespace tri;

namespace {

// Tile: S x S cells, S = 4*RHO, in S/16 strips of 16 cells.  The block has S
// threads: thread t takes strip c = t % NS (NS = S/16 strips) of the tile rows
// [Hr g, Hr g + Hr), g = t / NS, Hr = S/16, and keeps its Hr + 2 input rows (one
// above, one below) in registers as four 4-cell words each, loaded with one
// 16-byte load per row.  The cell left (right) of the strip comes from the
// neighbouring lane by shuffle, or, for the tile's first (last) strip, from a
// 4-byte load beyond the tile.  Cell bytes are normalised to 0/1 and zeroed
// outside the domain (j > i, rows outside [0, n)); the neighbour counts are
// byte-SIMD sums.
// LIFE: the rule is Conway's (birth on 3, survival on 2 or 3), evaluated with
// two SIMD byte compares on the 3 x 3 sum including the cell itself (alive
// next iff the sum is 3, or 4 with the cell alive); otherwise the general
// outer-totalistic rule is looked up per byte in `table`.
template <int MAP, int RHO, bool LIFE>
__global__ void __launch_bounds__(4 * RHO) ca_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                                     uint32_t n, size_t ld, uint32_t table, BlockMap bm)
{
    constexpr int S = 4 * RHO, NS = S / 16, HR = S / 16;
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    const int t = threadIdx.x, c = t % NS, g = t / NS;
    const long long cc = (long long)bj * S + 16 * c;         // first cell (byte) column of the strip
    const long long a0 = (long long)bi * S + HR * g - 1;     // global row of the first register row
    // keep the domain part of the word at byte column col of row a (col a multiple of 4)
    auto clip = [](uint32_t w, long long col, long long a) {
        w = __vcmpne4(w, 0u) & 0x01010101u;  // alive -> 1
        const long long over = col + 3 - a;  // bytes past the diagonal
        return over <= 0 ? w : (over >= 4 ? 0u : w & (0xFFFFFFFFu >> (8 * over)));
    };
    uint32_t w[HR + 2][4], lw[HR + 2], rw[HR + 2];
#pragma unroll
    for (int q = 0; q < HR + 2; ++q) {
        const long long a = a0 + q;
        const bool rok = a >= 0 && a < (long long)n;
        const uint8_t *row = in + (rok ? (size_t)a * ld : 0);
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (rok && cc <= a) v = __ldg(reinterpret_cast<const uint4 *>(row + cc));
        lw[q] = (c == 0 && rok && cc >= 4 && cc - 4 <= a) ? __ldg(reinterpret_cast<const uint32_t *>(row + cc - 4)) : 0u;
        rw[q] = (c == NS - 1 && rok && cc + 16 <= a) ? __ldg(reinterpret_cast<const uint32_t *>(row + cc + 16)) : 0u;
        w[q][0] = v.x;
        w[q][1] = v.y;
        w[q][2] = v.z;
        w[q][3] = v.w;
    }
    // normalise, clip at the diagonal, fetch the neighbours' edge words, horizontal 3-sums
    uint32_t hs[HR + 2][4], ctr[HR + 2][4];
#pragma unroll
    for (int q = 0; q < HR + 2; ++q) {
        const long long a = a0 + q;
#pragma unroll
        for (int k = 0; k < 4; ++k) w[q][k] = clip(w[q][k], cc + 4 * k, a);
        const uint32_t lc = clip(lw[q], cc - 4, a), rc = clip(rw[q], cc + 16, a);
        const uint32_t up = __shfl_up_sync(0xffffffffu, w[q][3], 1, NS);    // strip c - 1, last word
        const uint32_t dn = __shfl_down_sync(0xffffffffu, w[q][0], 1, NS);  // strip c + 1, first word
        const uint32_t L = c == 0 ? lc : up, R = c == NS - 1 ? rc : dn;
        const uint32_t W0 = w[q][0], W1 = w[q][1], W2 = w[q][2], W3 = w[q][3];
        hs[q][0] = __funnelshift_l(L, W0, 8) + W0 + __funnelshift_r(W0, W1, 8);
        hs[q][1] = __funnelshift_l(W0, W1, 8) + W1 + __funnelshift_r(W1, W2, 8);
        hs[q][2] = __funnelshift_l(W1, W2, 8) + W2 + __funnelshift_r(W2, W3, 8);
        hs[q][3] = __funnelshift_l(W2, W3, 8) + W3 + __funnelshift_r(W3, R, 8);
#pragma unroll
        for (int k = 0; k < 4; ++k) ctr[q][k] = w[q][k];
    }
#pragma unroll
    for (int q = 1; q <= HR; ++q) {
        const long long a = a0 + q;
        if (a >= (long long)n) break;
        if (cc > a) continue;  // the strip is past the diagonal in this row
        uint32_t nxt[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t alive = ctr[q][k];
            const uint32_t sum = hs[q - 1][k] + hs[q][k] + hs[q + 1][k];  // 3 x 3 sum, 0..9 per byte
            uint32_t r = 0;
            if constexpr (LIFE) {
                r = (__vcmpeq4(sum, 0x03030303u) | (__vcmpeq4(sum, 0x04040404u) & (alive * 0xFFu))) & 0x01010101u;
            } else {
                const uint32_t idx = sum + (alive << 3);  // count + 9*alive = sum - alive + 9*alive
#pragma unroll
                for (int b = 0; b < 4; ++b) r |= ((table >> ((idx >> (8 * b)) & 0xFFu)) & 1u) << (8 * b);
            }
            nxt[k] = r;
        }
        uint8_t *dst = out + (size_t)a * ld + cc;
        if (cc + 15 <= a) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(nxt[0], nxt[1], nxt[2], nxt[3]);
        } else {
            for (int b = 0; cc + b <= a; ++b) dst[b] = (uint8_t)(nxt[b >> 2] >> (8 * (b & 3)));
        }
    }
}

// Conway's rule bit-sliced: one bit per cell, 32 cells per word.  Tile S x S,
// S = 4*RHO, with NS (S / HR) threads: thread t takes the 32-cell strip c =
// t % NS (NS = S/32) of the tile rows [HR g, HR g + HR), g = t / NS, HR =
// min(S/16, 4), and reads its HR + 2 input rows (one above, one below) as two
// 16-byte loads each, all issued before any is used.  (At S = 128 four rows
// per thread in 128-thread blocks took 0.0633 ms per step at n = 16384
// against 0.0657 ms for eight rows in 64-thread blocks; the bounding box gave
// 0.0764 and 0.0612 ms.)  Each row's 32 bytes become one word (bit b = byte b non-zero,
// cleared past the diagonal and outside rows [0, n)); the cells left and
// right of the strip come from the neighbouring lanes' words by shuffle, or,
// at the tile's edges, from a 4-byte load beyond it.  Per row, the three
// horizontal neighbours give a parity word s and a majority word c (the count
// of the three is s + 2c); over three rows the 3 x 3 sum is
// ones + 2 (k + x + 2y) with ones, k the parity and majority of the three s,
// and x, y those of the three c.  The cell lives on iff the sum (itself
// included) is 3, or 4 with the cell alive.
__device__ __forceinline__ uint32_t alive_nibble(uint32_t w)  // bit b: byte b of w non-zero
{
    const uint32_t h = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;  // bit 7 of each non-zero byte
    return (h * 0x00204081u) >> 28;  // bits 7, 15, 23, 31 -> 28, 29, 30, 31
}

__device__ __forceinline__ uint32_t nibble_bytes(uint32_t nib)  // bit b -> byte b (0 or 1)
{
    return (nib * 0x00204081u) & 0x01010101u;
}

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c) { return (a & b) | (a & c) | (b & c); }

// rows per thread and threads per block of the bit-sliced step
template <int RHO>
__host__ __device__ constexpr int life_rows() { return (4 * RHO) / 16 < 4 ? (4 * RHO) / 16 : 4; }
template <int RHO>
__host__ __device__ constexpr int life_threads() { return (4 * RHO / 32) * (4 * RHO / life_rows<RHO>()); }

// The step is bound by the latency of its loads.  With 128 x 128-cell tiles
// (rho = 32) each block therefore first asks L2 to prefetch the input rows of
// the tile whose block starts `ahead` grid positions later (half the blocks
// resident at once): by the time that block runs, its rows are on their way
// from DRAM or in L2.  At n = 16384 this took lambda from 0.0624 to 0.0555 ms
// per step and the bounding box from 0.0754 to 0.0650 ms (a fixed 512
// positions: 0.0548; 1024: 0.0602; 2048: 0.0746).  With 64 x 64-cell tiles
// (one-warp blocks) the prefetches cost more than they save (0.0739 ->
// 0.0829 ms), so ahead = 0 there.
template <int MAP, int RHO>
__global__ void __launch_bounds__(life_threads<RHO>()) ca_life_bits_kernel(const uint8_t *__restrict__ in,
                                                                            uint8_t *__restrict__ out, uint32_t n,
                                                                            size_t ld, BlockMap bm, uint32_t ahead)
{
    constexpr int S = 4 * RHO, NS = S / 32, HR = life_rows<RHO>(), NT = NS * (S / HR);
    if (ahead) {
        uint32_t pi, pj;
        if (map_block_ahead<MAP>(bm, ahead, pi, pj)) {
            // two 128-byte lines per input row of that tile (rows outside the
            // grid or wholly above the diagonal are skipped; the second line
            // only when it lies inside the row)
            const long long c0 = (long long)pj * S;
            for (int r = threadIdx.x; r < S + 2; r += NT) {
                const long long a = (long long)pi * S + r - 1;
                if (a >= 0 && a < (long long)n && c0 <= a) {
                    const uint8_t *q = in + (size_t)a * ld + (size_t)c0;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
                    if ((size_t)c0 + 127 < ld) asm volatile("prefetch.global.L2 [%0];" ::"l"(q + 127));
                }
            }
        }
    }
    constexpr unsigned FULL = NT >= 32 ? 0xffffffffu : ((1u << NT) - 1u);
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    const int t = threadIdx.x, c = t % NS, g = t / NS;
    const long long cc = (long long)bj * S + 32 * c;      // first cell (byte) column of the strip
    const long long a0 = (long long)bi * S + HR * g - 1;  // global row of the first register row
    uint32_t B[HR + 2], sH[HR + 2], cH[HR + 2];
    // all of the strip's loads first (2 x 16 bytes per row and the edge
    // words), so that they are in flight together; then the bit packing
    uint4 v0[HR + 2], v1[HR + 2];
    uint32_t le[HR + 2], re[HR + 2];
#pragma unroll
    for (int q = 0; q < HR + 2; ++q) {
        const long long a = a0 + q;
        const bool rok = a >= 0 && a < (long long)n;
        const uint8_t *row = in + (rok ? (size_t)a * ld : 0);
        v0[q] = v1[q] = make_uint4(0u, 0u, 0u, 0u);
        if (rok && cc <= a) v0[q] = __ldg(reinterpret_cast<const uint4 *>(row + cc));
        if (rok && cc + 16 <= a) v1[q] = __ldg(reinterpret_cast<const uint4 *>(row + cc + 16));
        le[q] = (c == 0 && rok && cc >= 4 && cc - 1 <= a) ? __ldg(reinterpret_cast<const uint32_t *>(row + cc - 4)) : 0u;
        re[q] = (c == NS - 1 && rok && cc + 32 <= a) ? __ldg(reinterpret_cast<const uint32_t *>(row + cc + 32)) : 0u;
    }
#pragma unroll
    for (int q = 0; q < HR + 2; ++q) {
        const long long a = a0 + q;
        const bool rok = a >= 0 && a < (long long)n;
        uint32_t b = alive_nibble(v0[q].x) | (alive_nibble(v0[q].y) << 4) | (alive_nibble(v0[q].z) << 8) |
                     (alive_nibble(v0[q].w) << 12) | (alive_nibble(v1[q].x) << 16) | (alive_nibble(v1[q].y) << 20) |
                     (alive_nibble(v1[q].z) << 24) | (alive_nibble(v1[q].w) << 28);
        const long long inside = a - cc;  // columns cc .. cc + inside lie in the domain
        b = !rok || inside < 0 ? 0u : (inside >= 31 ? b : b & ((2u << inside) - 1u));
        B[q] = b;
        // the cells beyond the strip's ends
        uint32_t lb = le[q] >> 24 ? 1u : 0u, rb = re[q] & 0xFFu ? 1u : 0u;
        const uint32_t up = __shfl_up_sync(FULL, b, 1, NS);    // strip c - 1
        const uint32_t dn = __shfl_down_sync(FULL, b, 1, NS);  // strip c + 1
        if (c > 0) lb = up >> 31;
        if (c < NS - 1) rb = dn & 1u;
        const uint32_t L = (b << 1) | lb, R = (b >> 1) | (rb << 31);  // left and right neighbour of each cell
        sH[q] = L ^ b ^ R;
        cH[q] = maj3(L, b, R);
    }
#pragma unroll
    for (int q = 1; q <= HR; ++q) {
        const long long a = a0 + q;
        if (a >= (long long)n) break;
        if (cc > a) continue;  // the strip is past the diagonal in this row
        const uint32_t ones = sH[q - 1] ^ sH[q] ^ sH[q + 1], k = maj3(sH[q - 1], sH[q], sH[q + 1]);
        const uint32_t x = cH[q - 1] ^ cH[q] ^ cH[q + 1], y = maj3(cH[q - 1], cH[q], cH[q + 1]);
        const uint32_t three = ones & (x ^ k) & ~y;                             // sum 3
        const uint32_t four = ~ones & ((y & ~x & ~k) | (~y & x & k));           // sum 4
        const uint32_t nx = three | (four & B[q]);
        uint8_t *dst = out + (size_t)a * ld + cc;
        const uint4 o0 = make_uint4(nibble_bytes(nx & 0xFu), nibble_bytes((nx >> 4) & 0xFu),
                                    nibble_bytes((nx >> 8) & 0xFu), nibble_bytes((nx >> 12) & 0xFu));
        const uint4 o1 = make_uint4(nibble_bytes((nx >> 16) & 0xFu), nibble_bytes((nx >> 20) & 0xFu),
                                    nibble_bytes((nx >> 24) & 0xFu), nibble_bytes(nx >> 28));
        if (cc + 31 <= a) {
            *reinterpret_cast<uint4 *>(dst) = o0;
            *reinterpret_cast<uint4 *>(dst + 16) = o1;
        } else {
            for (int b = 0; cc + b <= a; ++b) dst[b] = (uint8_t)((nx >> b) & 1u);
        }
    }
}

// Half the blocks of this kernel that fit on the GPU at once (the L2
// prefetch distance of the Life step), looked up once per device.
template <int MAP, int RHO>
uint32_t life_ahead()
{
    static std::mutex mu;
    static int cached_dev = -1;
    static uint32_t cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (dev != cached_dev) {
        int per = 0, nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ca_life_bits_kernel<MAP, RHO>, life_threads<RHO>(), 0) !=
            cudaSuccess)
            per = 0;
        cached = (uint32_t)(nsm > 0 && per > 0 ? nsm * per / 2 : 0);
        cached_dev = dev;
    }
    return cached;
}

template <int MAP, bool LIFE>
void launch_rule(uint32_t rho, dim3 g, cudaStream_t s, const uint8_t *in, uint8_t *out, uint32_t n, size_t ld,
                 uint32_t table, BlockMap bm)
{
    if constexpr (LIFE) {
        switch (rho) {
        case 8: ca_life_bits_kernel<MAP, 8><<<g, life_threads<8>(), 0, s>>>(in, out, n, ld, bm, 0u); return;
        case 16: ca_life_bits_kernel<MAP, 16><<<g, life_threads<16>(), 0, s>>>(in, out, n, ld, bm, 0u); return;
        default:
            ca_life_bits_kernel<MAP, 32><<<g, life_threads<32>(), 0, s>>>(in, out, n, ld, bm, life_ahead<MAP, 32>());
            return;
        }
    }
    switch (rho) {
    case 8: ca_kernel<MAP, 8, LIFE><<<g, 32, 0, s>>>(in, out, n, ld, table, bm); break;
    case 16: ca_kernel<MAP, 16, LIFE><<<g, 64, 0, s>>>(in, out, n, ld, table, bm); break;
    default: ca_kernel<MAP, 32, LIFE><<<g, 128, 0, s>>>(in, out, n, ld, table, bm); break;
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

// The checks every step call makes: buffers, alignment, no aliasing, masks.
static int ca_args_ok(const uint8_t *in, const uint8_t *out, uint32_t n, size_t ld, uint32_t birth_mask,
                      uint32_t survive_mask, uint32_t rho)
{
    if (!in || !out || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (ld < n || (ld & 15) || ((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return TRI_EINVAL;
    // no aliasing: the two buffers of n rows must not overlap
    const size_t span = (size_t)(n - 1) * ld + n;
    if ((in < out + span) && (out < in + span)) return TRI_EINVAL;
    if ((birth_mask | survive_mask) >> 9) return TRI_EINVAL;
    return TRI_OK;
}

extern "C" int tri_ca_step(const uint8_t *in, uint8_t *out, uint32_t n, size_t ld, uint32_t birth_mask,
                           uint32_t survive_mask, int map, uint32_t rho, void *stream)
{
    const int ok = ca_args_ok(in, out, n, ld, birth_mask, survive_mask, rho);
    if (ok != TRI_OK) return ok;
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

// Row bands of one grid for several GPUs: band k holds the block rows from
// the first whose lambda number T(R) reaches k / ranks of the T(m) tiles, so
// the bands hold equal tile counts to within one block row.
extern "C" int tri_ca_partition(uint32_t n, uint32_t rho, uint32_t ranks, uint32_t rank, uint32_t *row_begin,
                                uint32_t *row_end)
{
    if (!row_begin || !row_end || ranks == 0 || rank >= ranks || !trihost::rho_ok(rho)) return TRI_EINVAL;
    const uint32_t S = 4 * rho, m = (uint32_t)(((uint64_t)n + S - 1) / S);
    const uint64_t total = T2(m);
    auto edge = [&](uint32_t k) -> uint32_t {
        if (k >= ranks) return m;
        const long double target = (long double)total * k / ranks;
        uint32_t lo = 0, hi = m;  // smallest R in [0, m] with T(R) >= target
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if ((long double)T2(mid) >= target) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    };
    *row_begin = (uint32_t)std::min<uint64_t>(n, (uint64_t)S * edge(rank));
    *row_end = (uint32_t)std::min<uint64_t>(n, (uint64_t)S * edge(rank + 1));
    return TRI_OK;
}

// One step of rows [row_begin, row_end) only: the lambda blocks of those
// block rows, numbers [T(R0), T(R1)), read rows row_begin - 1 .. row_end of
// `in` (those inside the grid) and write the band's domain cells of `out`.
extern "C" int tri_ca_step_rows(const uint8_t *in, uint8_t *out, uint32_t n, size_t ld, uint32_t birth_mask,
                                uint32_t survive_mask, uint32_t rho, uint32_t row_begin, uint32_t row_end,
                                void *stream)
{
    const int ok = ca_args_ok(in, out, n, ld, birth_mask, survive_mask, rho);
    if (ok != TRI_OK) return ok;
    const uint32_t S = 4 * rho;
    if (row_begin > row_end || row_end > n) return TRI_EINVAL;
    if (row_begin == row_end) return TRI_OK;  // an empty band (also one at row n) does nothing
    if (row_begin % S != 0 || (row_end % S != 0 && row_end != n)) return TRI_EINVAL;
    const uint32_t table = birth_mask | (survive_mask << 9);
    const uint32_t m = (n + S - 1) / S, R0 = row_begin / S, R1 = (row_end + S - 1) / S;
    BlockMap bm{};
    bm.m = m;
    bm.w0 = T2(R0);
    bm.nblocks = T2(R1);
    const cudaError_t e = launch_rho<MAP_LAMBDA>(rho, trihost::linear_grid(bm.nblocks - bm.w0),
                                                 (cudaStream_t)stream, in, out, n, ld, table, bm);
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}
