// Several steps of Conway's rule per pass through memory (temporal blocking)
// on the triangular domain {0 <= j <= i < n}.  Each block owns a 128 x 128
// cell tile placed by a block map (Section 3; the triangular-domain automaton
// of Section 1).  It reads the tile with a halo of K cells on every side,
// once, as bits (32 cells per word) in shared memory, runs up to K steps
// there, and writes the tile's domain cells back as bytes.  A cell of the
// region is exact after s steps when it lies at least s cells inside the
// region, so after K steps the tile itself is; the halo cells are computed
// only to get it there.  After every step the cells outside the domain
// (j > i, i >= n, j < 0) are cleared, as the rule counts them dead.
#include <cuda_runtime.h>

#include <algorithm>

#include "tri_internal.h"
#include "tri_maps.cuh"

using namespace tri;

namespace {

constexpr uint32_t TS = 128;  // tile side in cells (the rho = 32 tile of tri_ca_step)
constexpr uint32_t WPR = 5;   // words per region row: columns j0 - 16 .. j0 + 143 (halo <= 16)
constexpr uint32_t PITCH = WPR + 2;  // a zero word on each side of a row in shared memory
constexpr uint32_t GROUPS = 48;      // row groups: thread (w, g) steps word w of rows [g R, (g + 1) R)
constexpr int RUN_THREADS = WPR * GROUPS;

// byte k of x non-zero -> bit k (k < 4): bit 7 of each byte marks a non-zero
// byte (its low seven bits plus 0x7F carry into bit 7 unless all zero); one
// multiply then moves the four marks, 8 bits apart, to bits 24 .. 27.
__device__ __forceinline__ uint32_t bytes4_to_bits(uint32_t x)
{
    const uint32_t t = (((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x) & 0x80808080u;
    return ((t >> 7) * 0x01020408u) >> 24;
}

// bit k of a nibble -> byte k = 0 or 1: the multiply puts copies of bit k at
// k, k + 7, k + 14, k + 21, and only the copy at 8k falls on a byte's bit 0.
__device__ __forceinline__ uint32_t bits4_to_bytes(uint32_t nib) { return (nib * 0x00204081u) & 0x01010101u; }

// One row's three neighbour planes of word w: west (column b - 1), the word
// itself and east (column b + 1), from the words left (l) and right (r) of it.
struct Planes {
    uint32_t w, c, e;
};
__device__ __forceinline__ Planes planes(uint32_t l, uint32_t c, uint32_t r)
{
    return {__funnelshift_l(l, c, 1), c, __funnelshift_r(c, r, 1)};
}

// One step of Conway's rule for 32 cells from the planes of the row above
// (u), the row itself (m) and the row below (d).
__device__ __forceinline__ uint32_t life_word(const Planes &u, const Planes &m, const Planes &d)
{
    // row sums as (ones, twos): three cells above, three below, two beside
    const uint32_t sa = u.w ^ u.c ^ u.e, ca = (u.w & u.c) | (u.e & (u.w ^ u.c));
    const uint32_t sb = d.w ^ d.c ^ d.e, cb = (d.w & d.c) | (d.e & (d.w ^ d.c));
    const uint32_t sm = m.w ^ m.e, cm = m.w & m.e;
    // count = x1 + 2 (x2 + y1) + 4 y2 = x1 + 2 z1 + 4 (z2 + y2)
    const uint32_t x1 = sa ^ sb ^ sm, x2 = (sa & sb) | (sm & (sa ^ sb));
    const uint32_t y1 = ca ^ cb ^ cm, y2 = (ca & cb) | (cm & (ca ^ cb));
    const uint32_t z1 = x2 ^ y1, z2 = x2 & y1;
    // alive next: count 3, or count 2 and alive now (count >= 4 when z2 | y2)
    return z1 & ~(z2 | y2) & (x1 | m.c);
}

template <int MAP, int K>
__global__ void __launch_bounds__(RUN_THREADS) ca_life_run_kernel(const uint8_t *__restrict__ in,
                                                                   uint8_t *__restrict__ out, uint32_t n, size_t ld,
                                                                   BlockMap bm, uint32_t steps)
{
    static_assert(K >= 1 && K <= 16, "the halo must fit the 16-cell margins of the region's words");
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    constexpr uint32_t ROWS = TS + 2 * K, RPT = (ROWS + GROUPS - 1) / GROUPS;
    // the state (two buffers, rows of PITCH words: a zero, words 0 .. 4, a
    // zero) and the domain mask; region row r = cell row i0 - K + r, bit b of
    // word w = column j0 - 16 + 32 w + b
    __shared__ uint32_t s_a[ROWS * PITCH], s_b[ROWS * PITCH], s_mask[ROWS * WPR];
    const uint32_t tid = threadIdx.y * WPR + threadIdx.x;
    const int64_t i0 = (int64_t)bi * TS, j0 = (int64_t)bj * TS;
    const int64_t ibase = i0 - K, jbase = j0 - 16, last = (int64_t)n - 1;

    for (uint32_t e = tid; e < ROWS * WPR; e += RUN_THREADS) {
        const uint32_t r = e / WPR, w = e - r * WPR;
        const int64_t i = ibase + r, c0 = jbase + 32 * (int64_t)w;
        // domain columns of the word: 0 <= c0 + b <= min(i, n - 1), for 0 <= i < n
        uint32_t mask = 0;
        if (i >= 0 && i <= last) {
            const int64_t lo = -c0 > 0 ? -c0 : 0;
            const int64_t top = (i < last ? i : last) - c0, hi = top < 31 ? top : 31;
            if (hi >= lo) mask = (hi - lo == 31) ? 0xFFFFFFFFu : (((1u << (hi - lo + 1)) - 1u) << lo);
        }
        uint32_t bits = 0;
        // a half word with a domain column starts at a column in [0, n - 1]:
        // its 16-byte chunk lies inside the row (ld >= n, both multiples of 16)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if ((mask >> (16 * h)) & 0xFFFFu) {
                const uint4 v = *reinterpret_cast<const uint4 *>(in + (size_t)i * ld + (size_t)(c0 + 16 * h));
                const uint32_t b16 = bytes4_to_bits(v.x) | (bytes4_to_bits(v.y) << 4) |
                                     (bytes4_to_bits(v.z) << 8) | (bytes4_to_bits(v.w) << 12);
                bits |= b16 << (16 * h);
            }
        }
        s_a[r * PITCH + 1 + w] = bits & mask;
        // the first and last region rows are never stepped: both buffers keep them
        if (r == 0 || r == ROWS - 1) s_b[r * PITCH + 1 + w] = bits & mask;
        s_mask[e] = mask;
    }
    for (uint32_t r = tid; r < ROWS; r += RUN_THREADS) {
        s_a[r * PITCH] = s_a[r * PITCH + PITCH - 1] = 0u;
        s_b[r * PITCH] = s_b[r * PITCH + PITCH - 1] = 0u;
    }
    __syncthreads();

    // thread (w, g) steps word w of rows r0 .. r1 - 1, sliding a window of
    // three rows down them; the first and last region rows have no row
    // beyond them and keep their first values, which reach at most K - 1
    // rows inward in K steps
    const uint32_t w = threadIdx.x;
    const uint32_t r0 = max(1u, threadIdx.y * RPT), r1 = min(ROWS - 1, (threadIdx.y + 1) * RPT);
    uint32_t *cur = s_a, *nxt = s_b;
    for (uint32_t s = 0; s < steps; ++s) {
        if (r0 < r1) {
            const uint32_t *p = cur + (r0 - 1) * PITCH + w;  // words w - 1 .. w + 1 at p[0 .. 2]
            Planes up = planes(p[0], p[1], p[2]);
            Planes mid = planes(p[PITCH], p[PITCH + 1], p[PITCH + 2]);
            for (uint32_t r = r0; r < r1; ++r) {
                const uint32_t *q = cur + (r + 1) * PITCH + w;
                const Planes dn = planes(q[0], q[1], q[2]);
                nxt[r * PITCH + 1 + w] = life_word(up, mid, dn) & s_mask[r * WPR + w];
                up = mid;
                mid = dn;
            }
        }
        __syncthreads();
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
    }

    // the tile's domain cells: 128 rows x 8 chunks of 16 cells; chunk ch is
    // region bits 16 + 16 ch .. +15, inside one word (shift 0 or 16)
    for (uint32_t e = tid; e < TS * 8; e += RUN_THREADS) {
        const uint32_t rr = e >> 3, ch = e & 7;
        const int64_t i = i0 + rr, c = j0 + 16 * (int64_t)ch;
        if (i > last || c > i) continue;
        const uint32_t off = 16 + 16 * ch;
        const uint32_t b16 = (cur[(K + rr) * PITCH + 1 + (off >> 5)] >> (off & 31)) & 0xFFFFu;
        uint8_t *dst = out + (size_t)i * ld + (size_t)c;
        const int64_t lastc = i < last ? i : last;  // the row's last domain column
        if (c + 15 <= lastc) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(bits4_to_bytes(b16 & 15u), bits4_to_bytes((b16 >> 4) & 15u),
                                                         bits4_to_bytes((b16 >> 8) & 15u), bits4_to_bytes(b16 >> 12));
        } else {
            for (int64_t k = 0; k <= lastc - c; ++k) dst[k] = (uint8_t)((b16 >> k) & 1u);
        }
    }
}

template <int K>
int launch_run_pass(int map, const uint8_t *in, uint8_t *out, uint32_t n, size_t ld, uint32_t steps, cudaStream_t s)
{
    const uint32_t m = (n + TS - 1) / TS;
    return trihost::map_launches(map, m, [&](auto tag, dim3 g, const BlockMap &bm) -> cudaError_t {
        constexpr int MAP = decltype(tag)::value;
        ca_life_run_kernel<MAP, K><<<g, dim3(WPR, GROUPS), 0, s>>>(in, out, n, ld, bm, steps);
        return cudaGetLastError();
    });
}

constexpr uint32_t LIFE_BIRTH_MASK = 1u << 3, LIFE_SURVIVE_MASK = (1u << 2) | (1u << 3);
constexpr uint32_t RUN_K = 8;  // steps per pass

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
    const uint32_t per = fused ? RUN_K : 1u;
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
            r = launch_run_pass<RUN_K>(map, src, dst, n, ld, k, s);
        else
            r = tri_ca_step(src, dst, n, ld, birth_mask, survive_mask, map, rho, stream);
        if (r != TRI_OK) return r;
        src = dst;
    }
    return TRI_OK;
}
