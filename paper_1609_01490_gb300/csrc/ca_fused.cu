// Several steps of Conway's rule per pass through memory (temporal blocking)
// on the triangular domain {0 <= j <= i < n}.  Each block owns a 128 x 128
// cell tile placed by a block map (Section 3; the triangular-domain automaton
// of Section 1).  One warp reads the tile with a halo of 16 cells on every
// side, once, packs it to bits (32 cells per word) and keeps it in registers:
// lane l holds region rows 5 l .. 5 l + 4, five words each.  It takes up to
// 16 steps there and writes the tile's domain cells back as bytes.  A cell of
// the region is exact after s steps when it lies at least s cells inside the
// region, so after 16 steps the tile itself is; the halo cells are computed
// only to get it there.  After every step the cells outside the domain
// (j > i, i >= n, j < 0) are cleared, as the rule counts them dead.
#include <cuda_runtime.h>

#include <algorithm>

#include "tri_internal.h"
#include "tri_maps.cuh"

using namespace tri;

namespace {

constexpr uint32_t TS = 128;                 // tile side in cells (the rho = 32 tile of tri_ca_step)
constexpr int KH = 16;                       // halo in cells on each side, and steps per pass
constexpr uint32_t WPR = 5;                  // words per region row: columns j0 - 16 .. j0 + 143
constexpr uint32_t ROWS = TS + 2 * KH;       // region rows: i0 - 16 .. i0 + 143
constexpr uint32_t RPL = ROWS / 32;          // region rows per lane
static_assert(RPL * 32 == ROWS, "one warp holds the region");
static_assert(KH <= 16, "the halo must fit the 16-cell margins of the region's words");

// Four bytes -> four bits at 0 .. 3 (byte k non-zero -> bit k).  Bit 7 of
// each byte of t marks a non-zero byte: its low seven bits plus 0x7F carry
// into bit 7 unless all zero, and a byte >= 0x80 has it already.  Times
// 2^21 + 2^14 + 2^7 + 1, bits 7, 15, 23, 31 land at 28, 29, 30, 31; every
// other product bit lands below 28 or past 31, each at its own position, so
// nothing carries into the top four.
__device__ __forceinline__ uint32_t nib_of(uint32_t x)
{
    const uint32_t t = (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
    return (t * 0x00204081u) >> 28;
}

// 16 bytes -> 16 bits
__device__ __forceinline__ uint32_t pack16(const uint4 q)
{
    return nib_of(q.x) + 16u * (nib_of(q.y) + 16u * (nib_of(q.z) + 16u * nib_of(q.w)));
}

// bit k of a nibble -> byte k = 0 or 1: the multiply puts copies of bit k at
// k, k + 7, k + 14, k + 21, and only the copy at 8k falls on a byte's bit 0.
__device__ __forceinline__ uint32_t bits4_to_bytes(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// bits lo .. hi of a word (empty when hi < lo), for any ints
__device__ __forceinline__ uint32_t span_bits(int lo, int hi)
{
    lo = lo > 0 ? lo : 0;
    hi = hi < 31 ? hi : 31;
    if (hi < lo) return 0u;
    return (0xFFFFFFFFu >> (31 - hi)) & (0xFFFFFFFFu << lo);
}

__device__ __forceinline__ int clamp_small(int64_t v) { return (int)(v < -4096 ? -4096 : (v > 4096 ? 4096 : v)); }

// The domain within the region as small ints: region rows g in [ilo, ihi]
// are cell rows 0 .. n - 1, and row g holds the domain's region columns lo ..
// min(dd + g, lastrel) (dd = i0 - j0; lastrel = n - 1 - (j0 - 16); lo = 16
// in the first block column, where cell column 0 is region column 16).
// Values beyond +-4096 are clamped: only -1 .. 160 matter.
struct RegionDomain {
    int lo, dd, lastrel, ilo, ihi;
    __device__ __forceinline__ uint32_t mask(int g, int w) const
    {
        if (g < ilo || g > ihi) return 0u;
        const int hi = min(dd + g, lastrel);
        return span_bits(lo - 32 * w, hi - 32 * w);
    }
    // every cell of the region lies in the domain
    __device__ __forceinline__ bool full() const
    {
        return lo == 0 && ilo == 0 && ihi >= (int)ROWS - 1 && dd >= (int)ROWS - 1 && lastrel >= (int)ROWS - 1;
    }
};

// For each word of a row: the sum of the cell and its two side neighbours as
// (s3 + 2 c3), and of the two side neighbours alone as (s2 + 2 c2), from the
// row's west and east planes (bit b of a word is region column 32 w + b).
__device__ __forceinline__ void row_sums(const uint32_t (&row)[WPR], uint32_t (&s3)[WPR], uint32_t (&c3)[WPR],
                                         uint32_t (&s2)[WPR], uint32_t (&c2)[WPR])
{
#pragma unroll
    for (uint32_t w = 0; w < WPR; ++w) {
        const uint32_t l = w ? row[w - 1] : 0u, r = w + 1 < WPR ? row[w + 1] : 0u;
        const uint32_t W = __funnelshift_l(l, row[w], 1), E = __funnelshift_r(row[w], r, 1);
        s2[w] = W ^ E;
        c2[w] = W & E;
        s3[w] = s2[w] ^ row[w];
        c3[w] = c2[w] | (row[w] & s2[w]);
    }
}

// `steps` steps of the region held by the warp.  Each row's sums are formed
// once, by the lane that holds it, and used by the rows above and below it;
// a lane gets the 3-sums of the row above its first and below its last from
// its neighbours by shuffle.  The region's first and last rows are stepped
// from whatever their shuffles return: like every cell that lacks neighbours
// in the region, they are wrong after the first step, and the wrong rim grows
// one cell per step.
template <bool MASKED>
__device__ __forceinline__ void run_steps(uint32_t (&c)[RPL][WPR], uint32_t lane, uint32_t steps,
                                          const RegionDomain &dom)
{
    for (uint32_t s = 0; s < steps; ++s) {
        // sums of the lane's first and last rows, formed once: their 3-sums go
        // to the neighbouring lanes by shuffle (as the sums of the row above
        // or below theirs) and all four are used here
        uint32_t fs3[WPR], fc3[WPR], fs2[WPR], fc2[WPR], ls3[WPR], lc3[WPR], ls2[WPR], lc2[WPR];
        row_sums(c[0], fs3, fc3, fs2, fc2);
        row_sums(c[RPL - 1], ls3, lc3, ls2, lc2);
        uint32_t ps3[WPR], pc3[WPR], ds3[WPR], dc3[WPR];
#pragma unroll
        for (uint32_t w = 0; w < WPR; ++w) {
            ps3[w] = __shfl_up_sync(0xFFFFFFFFu, ls3[w], 1);
            pc3[w] = __shfl_up_sync(0xFFFFFFFFu, lc3[w], 1);
            ds3[w] = __shfl_down_sync(0xFFFFFFFFu, fs3[w], 1);
            dc3[w] = __shfl_down_sync(0xFFFFFFFFu, fc3[w], 1);
        }
        uint32_t cs3[WPR], cc3[WPR], cs2[WPR], cc2[WPR];
#pragma unroll
        for (uint32_t w = 0; w < WPR; ++w) {
            cs3[w] = fs3[w];
            cc3[w] = fc3[w];
            cs2[w] = fs2[w];
            cc2[w] = fc2[w];
        }
#pragma unroll
        for (uint32_t r = 0; r < RPL; ++r) {
            uint32_t ns3[WPR], nc3[WPR], ns2[WPR], nc2[WPR];
            if (r + 2 < RPL) {
                row_sums(c[r + 1], ns3, nc3, ns2, nc2);
            } else if (r + 2 == RPL) {
#pragma unroll
                for (uint32_t w = 0; w < WPR; ++w) {
                    ns3[w] = ls3[w];
                    nc3[w] = lc3[w];
                    ns2[w] = ls2[w];
                    nc2[w] = lc2[w];
                }
            } else {  // the row below the lane's last: its 3-sums from the next lane
#pragma unroll
                for (uint32_t w = 0; w < WPR; ++w) {
                    ns3[w] = ds3[w];
                    nc3[w] = dc3[w];
                    ns2[w] = 0u;
                    nc2[w] = 0u;
                }
            }
#pragma unroll
            for (uint32_t w = 0; w < WPR; ++w) {
                // the 8 neighbours: (ps3 + 2 pc3) + (ns3 + 2 nc3) + (cs2 + 2 cc2)
                // = x1 + 2 (x2 + y1) + 4 y2
                const uint32_t x1 = ps3[w] ^ ns3[w] ^ cs2[w];
                const uint32_t x2 = (ps3[w] & ns3[w]) | (cs2[w] & (ps3[w] ^ ns3[w]));
                const uint32_t y1 = pc3[w] ^ nc3[w] ^ cc2[w];
                const uint32_t y2 = (pc3[w] & nc3[w]) | (cc2[w] & (pc3[w] ^ nc3[w]));
                // alive next: count 3, or count 2 and alive now (>= 4 when x2 & y1 or y2)
                uint32_t v = (x2 ^ y1) & ~((x2 & y1) | y2) & (x1 | c[r][w]);
                if constexpr (MASKED) v &= dom.mask((int)(lane * RPL + r), (int)w);
                c[r][w] = v;
            }
#pragma unroll
            for (uint32_t w = 0; w < WPR; ++w) {
                ps3[w] = cs3[w];
                pc3[w] = cc3[w];
                cs3[w] = ns3[w];
                cc3[w] = nc3[w];
                cs2[w] = ns2[w];
                cc2[w] = nc2[w];
            }
        }
    }
}

// 128 registers a thread (16 warps per SM; a few spill in the masked form):
// the ALU pipe, not occupancy, bounds the steps
template <int MAP>
__global__ void __launch_bounds__(32, 16) ca_life_run_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                                             uint32_t n, size_t ld, BlockMap bm, uint32_t steps)
{
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    __shared__ uint32_t s_rows[ROWS * WPR];  // region row g, word w at g * WPR + w
    const uint32_t lane = threadIdx.x;
    const int64_t i0 = (int64_t)bi * TS, j0 = (int64_t)bj * TS;
    const int64_t ibase = i0 - KH, jbase = j0 - 16, last = (int64_t)n - 1;
    RegionDomain dom;
    dom.lo = bj == 0 ? 16 : 0;
    dom.dd = clamp_small(i0 - j0);
    dom.lastrel = clamp_small(last - jbase);
    dom.ilo = clamp_small(ibase < 0 ? -ibase : 0);
    dom.ihi = clamp_small(last - ibase);
    const bool full = dom.full();

    // load: region word e = g * WPR + w, five words a lane at a time, every
    // load of a batch issued before any is used; a tile whose region lies
    // inside the domain needs no masks
#pragma unroll 1
    for (uint32_t b = 0; b < ROWS * WPR / 32; b += 5) {
        uint4 v[5][2];
        uint32_t mk[5];
#pragma unroll
        for (uint32_t k = 0; k < 5; ++k) {
            const uint32_t e = (b + k) * 32 + lane, g = e / WPR, w = e - g * WPR;
            if (full) {
                const uint8_t *src = in + (size_t)(ibase + g) * ld + (size_t)(jbase + 32 * (int64_t)w);
                mk[k] = 0xFFFFFFFFu;
                v[k][0] = *reinterpret_cast<const uint4 *>(src);
                v[k][1] = *reinterpret_cast<const uint4 *>(src + 16);
            } else {
                mk[k] = dom.mask((int)g, (int)w);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // a half word with a domain column starts at a column in [0, n - 1]:
                    // its 16-byte chunk lies inside the row (ld >= n, both multiples of 16)
                    v[k][h] = make_uint4(0, 0, 0, 0);
                    if ((mk[k] >> (16 * h)) & 0xFFFFu)
                        v[k][h] = *reinterpret_cast<const uint4 *>(in + (size_t)(ibase + g) * ld +
                                                                   (size_t)(jbase + 32 * (int64_t)w + 16 * h));
                }
            }
        }
#pragma unroll
        for (uint32_t k = 0; k < 5; ++k)
            s_rows[(b + k) * 32 + lane] = (pack16(v[k][0]) + 65536u * pack16(v[k][1])) & mk[k];
    }
    __syncwarp();
    // lane l takes region rows 5 l .. 5 l + 4 (a stride of 25 words: no bank conflicts)
    uint32_t c[RPL][WPR];
#pragma unroll
    for (uint32_t r = 0; r < RPL; ++r)
#pragma unroll
        for (uint32_t w = 0; w < WPR; ++w) c[r][w] = s_rows[(lane * RPL + r) * WPR + w];
    if (full)
        run_steps<false>(c, lane, steps, dom);
    else
        run_steps<true>(c, lane, steps, dom);
    __syncwarp();
#pragma unroll
    for (uint32_t r = 0; r < RPL; ++r)
#pragma unroll
        for (uint32_t w = 0; w < WPR; ++w) s_rows[(lane * RPL + r) * WPR + w] = c[r][w];
    __syncwarp();

    // the tile's domain cells: 128 rows x 8 chunks of 16 cells; chunk ch of
    // tile row rr is bits 16 + 16 ch .. + 15 of region row KH + rr (all of
    // them for a tile inside the domain)
#pragma unroll 4
    for (uint32_t e = lane; e < TS * 8; e += 32) {
        const uint32_t rr = e >> 3, ch = e & 7;
        const int64_t i = i0 + rr, col = j0 + 16 * (int64_t)ch;
        const uint32_t off = 16 + 16 * ch;
        const uint32_t b16 = s_rows[(KH + rr) * WPR + (off >> 5)] >> (off & 31);
        const uint4 q = make_uint4(bits4_to_bytes(b16 & 15u), bits4_to_bytes((b16 >> 4) & 15u),
                                   bits4_to_bytes((b16 >> 8) & 15u), bits4_to_bytes((b16 >> 12) & 15u));
        if (full) {
            *reinterpret_cast<uint4 *>(out + (size_t)i * ld + (size_t)col) = q;
            continue;
        }
        if (i > last || col > i) continue;
        uint8_t *dst = out + (size_t)i * ld + (size_t)col;
        const int64_t lastc = i < last ? i : last;  // the row's last domain column
        if (col + 15 <= lastc) {
            *reinterpret_cast<uint4 *>(dst) = q;
        } else {
            for (int64_t k = 0; k <= lastc - col; ++k) dst[k] = (uint8_t)((b16 >> k) & 1u);
        }
    }
}

int launch_run_pass(int map, const uint8_t *in, uint8_t *out, uint32_t n, size_t ld, uint32_t steps, cudaStream_t s)
{
    const uint32_t m = (n + TS - 1) / TS;
    return trihost::map_launches(map, m, [&](auto tag, dim3 g, const BlockMap &bm) -> cudaError_t {
        constexpr int MAP = decltype(tag)::value;
        ca_life_run_kernel<MAP><<<g, 32, 0, s>>>(in, out, n, ld, bm, steps);
        return cudaGetLastError();
    });
}

constexpr uint32_t LIFE_BIRTH_MASK = 1u << 3, LIFE_SURVIVE_MASK = (1u << 2) | (1u << 3);

bool overlap(const uint8_t *a, const uint8_t *b, size_t span) { return a < b + span && b < a + span; }

}  // namespace

extern "C" int tri_ca_run(const uint8_t *in, uint8_t *out, uint8_t *scratch, uint32_t n, size_t ld,
                          uint32_t birth_mask, uint32_t survive_mask, int map, uint32_t rho, uint32_t steps,
                          void *stream)
{
    if (!in || !out || n == 0 || steps == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (ld < n || (ld & 15) || ((uintptr_t)in & 15) || ((uintptr_t)out & 15) || ((uintptr_t)scratch & 15))
        return TRI_EINVAL;
    if ((birth_mask | survive_mask) >> 9) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_LAMBDA_PDELTA && map != TRI_MAP_BB && map != TRI_MAP_RB &&
        map != TRI_MAP_REC)
        return TRI_EINVAL;
    const bool fused = birth_mask == LIFE_BIRTH_MASK && survive_mask == LIFE_SURVIVE_MASK && rho == 32;
    const uint32_t per = fused ? (uint32_t)KH : 1u;
    const uint32_t passes = (steps + per - 1) / per;
    const size_t span = (size_t)(n - 1) * ld + n;
    if (overlap(in, out, span)) return TRI_EINVAL;
    if (passes > 1) {
        if (!scratch || overlap(scratch, in, span) || overlap(scratch, out, span)) return TRI_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // pass p writes `out` when passes - 1 - p is even, `scratch` otherwise,
    // so the last pass writes `out` and `in` is only read
    const uint8_t *src = in;
    for (uint32_t p = 0; p < passes; ++p) {
        uint8_t *dst = ((passes - 1 - p) % 2 == 0) ? out : scratch;
        const uint32_t k = std::min(per, steps - p * per);
        int r;
        if (fused)
            r = launch_run_pass(map, src, dst, n, ld, k, s);
        else
            r = tri_ca_step(src, dst, n, ld, birth_mask, survive_mask, map, rho, stream);
        if (r != TRI_OK) return r;
        src = dst;
    }
    return TRI_OK;
}
