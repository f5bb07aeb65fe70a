// Collision detection of N spheres with random radii (Section 5, test 3), the
// paper's shared-memory workload: every block of a 2-D block map stages the
// spheres of its row and column tiles in shared memory and tests its pairs
// from registers.  UTM, a thread-space map, tests one pair per thread from
// global memory instead (the paper notes it cannot use the 2-D shared tile).
//
// The test of a pair i > j is s <= (r_i + r_j)^2 with
// s = (c_i0 - c_j0)^2 + (c_i1 - c_j1)^2 + ..., each step a separate FP32
// operation rounded to nearest (no fused multiply-add), so the decisions are
// exactly those of any other implementation that takes the same steps.
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "tri_maps.cuh"

using namespace tri;

namespace {

struct CollideOut {
    uint32_t *count;               // per-sphere counts, or null
    uint32_t *pairs;               // (i, j) list, or null
    uint64_t cap;                  // entries of the list
    unsigned long long *n_pairs;   // colliding pairs found
};

// The exact test in scalar FP32: the reference order of operations.
template <int DIM>
__device__ __forceinline__ bool hit_scalar(const float *a, const float *b)
{
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float dk = __fsub_rn(a[k], b[k]);
        const float sq = __fmul_rn(dk, dk);
        s = k == 0 ? sq : __fadd_rn(s, sq);
    }
    const float rr = __fadd_rn(a[DIM], b[DIM]);
    return s <= __fmul_rn(rr, rr);
}

// A colliding pair: one slot of the list, one count for each sphere.
__device__ __forceinline__ void record(const CollideOut &o, uint32_t i, uint32_t j)
{
    const unsigned long long q = atomicAdd(o.n_pairs, 1ull);
    if (q < o.cap) {
        o.pairs[2 * q] = i;
        o.pairs[2 * q + 1] = j;
    }
    if (o.count) {
        atomicAdd(o.count + i, 1u);
        atomicAdd(o.count + j, 1u);
    }
}

// One S x S pair tile, S = RHO*R: rows i0 = bi S + [0, S), columns
// j0 = bj S + [0, S).  The 2 S spheres are staged transposed ([coordinate or
// radius][sphere]), the rows with each value duplicated into both halves of
// an 8-byte word.  Thread (ty, tx) owns rows ty + u RHO (u < R) and, for
// R >= 2, the column pairs 2 tx + 2 RHO v + {0, 1} (v < R/2), tested two at a
// time with f32x2 instructions, whose lanes round exactly as the scalar
// operations of the reference order do.  The fast pass keeps one word: the
// AND of the bits of q - s over all the thread's pairs; since q - s rounds to
// a value >= 0 exactly when q >= s, a clear sign bit means some pair may hit
// (or some input is NaN).  Only such threads (a few per contact, plus the
// diagonal, where a sphere meets itself) repeat the packed pass, compare s
// and q lane by lane and record the valid pairs (i < n, j < i).
// Padding spheres past n sit at +inf (rows) and -inf (columns), so their
// tests give s = inf and never flag.  For R = 1 each thread takes the scalar
// test of its one pair.  Not inlined: every block map calls the same body.
template <int RHO, int R, int DIM>
__device__ __noinline__ void collide_tile(const float *__restrict__ c, const float *__restrict__ rad, uint32_t n,
                                          uint32_t bi, uint32_t bj, CollideOut o)
{
    constexpr int S = RHO * R;
    constexpr int RC = R == 1 ? 1 : R / 2;
    __shared__ f2 si[DIM + 1][S];                       // rows, duplicated
    __shared__ __align__(8) float sj[DIM + 1][S + 2];   // columns
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RHO + tx;
    const uint64_t i0 = (uint64_t)bi * S, j0 = (uint64_t)bj * S;
    const float inf = __int_as_float(0x7f800000);
    // coalesced staging of S consecutive spheres: centres (S DIM floats), then radii
    for (int t = tid; t < S * DIM; t += RHO * RHO) {
        const int r = t / DIM, k = t - r * DIM;
        const float a = i0 + r < n ? c[i0 * DIM + t] : inf;
        si[k][r] = f2_pack(a, a);
        sj[k][r] = j0 + r < n ? c[j0 * DIM + t] : -inf;
    }
    for (int t = tid; t < S; t += RHO * RHO) {
        const float a = i0 + t < n ? rad[i0 + t] : 0.0f;
        si[DIM][t] = f2_pack(a, a);
        sj[DIM][t] = j0 + t < n ? rad[j0 + t] : 0.0f;
    }
    __syncthreads();

    if constexpr (R == 1) {
        float a[DIM + 1], b[DIM + 1], dummy;
#pragma unroll
        for (int k = 0; k <= DIM; ++k) {
            f2_unpack(si[k][ty], a[k], dummy);
            b[k] = sj[k][tx];
        }
        const uint64_t i = i0 + ty, j = j0 + tx;
        if (hit_scalar<DIM>(a, b) && i < n && j < i) record(o, (uint32_t)i, (uint32_t)j);
        return;
    } else {
        f2 b2[RC][DIM + 1];
#pragma unroll
        for (int v = 0; v < RC; ++v)
#pragma unroll
            for (int k = 0; k <= DIM; ++k) b2[v][k] = *reinterpret_cast<const f2 *>(&sj[k][2 * tx + 2 * RHO * v]);
        // s and q of the column pair v for row values a2, in the reference order
        auto test = [&](const f2 *a2, int v, f2 &s, f2 &q) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const f2 dk = f2_sub(a2[k], b2[v][k]);
                s = k == 0 ? f2_mul(dk, dk) : f2_add(s, f2_mul(dk, dk));
            }
            const f2 rr = f2_add(a2[DIM], b2[v][DIM]);
            q = f2_mul(rr, rr);
        };
        uint32_t acc = 0xFFFFFFFFu;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            f2 a2[DIM + 1];
#pragma unroll
            for (int k = 0; k <= DIM; ++k) a2[k] = si[k][ty + u * RHO];
#pragma unroll
            for (int v = 0; v < RC; ++v) {
                f2 s, q;
                test(a2, v, s, q);
                const f2 d = f2_sub(q, s);
                acc &= (uint32_t)d & (uint32_t)(d >> 32);
            }
        }
        if ((int)acc < 0) return;
        // some pair may hit: the same tests again, decided lane by lane
#pragma unroll 1
        for (int u = 0; u < R; ++u) {
            const uint64_t i = i0 + ty + u * RHO;
            if (i >= n) break;
            f2 a2[DIM + 1];
#pragma unroll
            for (int k = 0; k <= DIM; ++k) a2[k] = si[k][ty + u * RHO];
#pragma unroll
            for (int v = 0; v < RC; ++v) {
                f2 s, q;
                test(a2, v, s, q);
                float s0, s1, q0, q1;
                f2_unpack(s, s0, s1);
                f2_unpack(q, q0, q1);
                const uint64_t j = j0 + 2 * tx + 2 * RHO * v;
                if (s0 <= q0 && j < i) record(o, (uint32_t)i, (uint32_t)j);
                if (s1 <= q1 && j + 1 < i) record(o, (uint32_t)i, (uint32_t)(j + 1));
            }
        }
    }
}

// 8 x 8 pairs per thread on 16 x 16 threads: registers capped at 64 so that
// four blocks share an SM (uncapped the tile takes over 100 and three fit,
// which leaves too few warps to cover the staging loads).
template <int MAP, int RHO, int R, int DIM>
__global__ void __launch_bounds__(RHO *RHO, (RHO == 16 && R == 8) ? 4 : 1)
    collide_kernel(const float *__restrict__ c, const float *__restrict__ rad, uint32_t n, CollideOut o, BlockMap bm)
{
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    collide_tile<RHO, R, DIM>(c, rad, n, bi, bj, o);
}

// UTM (Section 4.2): thread k of the (n+1) n / 2 pairs j <= i, one test each,
// operands from global memory; the diagonal threads (j = i) do nothing.
template <int DIM>
__global__ void collide_utm_kernel(const float *__restrict__ c, const float *__restrict__ rad, uint32_t n,
                                   CollideOut o)
{
    const uint64_t N = (uint64_t)n + 1;
    const uint64_t total = N * n / 2;
    const uint64_t k = ((uint64_t)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                       threadIdx.y * blockDim.x + threadIdx.x;
    if (k >= total) return;
    uint32_t a, b;
    utm_pair(k, N, a, b);
    const uint32_t i = b - 2, j = a - 1;
    if (j >= i) return;
    float pa[DIM + 1], pb[DIM + 1];
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
        pa[t] = c[(uint64_t)i * DIM + t];
        pb[t] = c[(uint64_t)j * DIM + t];
    }
    pa[DIM] = rad[i];
    pb[DIM] = rad[j];
    if (hit_scalar<DIM>(pa, pb)) record(o, i, j);
}

template <int DIM>
int launch_dim(const float *c, const float *rad, uint32_t n, int map, uint32_t rho, uint32_t reg, CollideOut o,
               cudaStream_t s)
{
    if (map == TRI_MAP_UTM) {
        const uint64_t N = (uint64_t)n + 1, total = N * n / 2, tpb = (uint64_t)rho * rho;
        if (total > 0xFFFFFFFFull) return TRI_ERANGE;
        collide_utm_kernel<DIM><<<trihost::linear_grid((total + tpb - 1) / tpb), dim3(rho, rho), 0, s>>>(c, rad,
                                                                                                         n, o);
        return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
    }
    const uint32_t S = rho * reg, m = (n + S - 1) / S;
    return trihost::map_launches(map, m, [&](auto tag, dim3 g, const BlockMap &bm) -> cudaError_t {
        constexpr int MAP = decltype(tag)::value;
#define TRI_C(RH, RG)                                                                                          \
    if (rho == RH && reg == RG) {                                                                              \
        collide_kernel<MAP, RH, RG, DIM><<<g, dim3(RH, RH), 0, s>>>(c, rad, n, o, bm);                         \
        return cudaGetLastError();                                                                             \
    }
        TRI_C(8, 1) TRI_C(8, 4) TRI_C(8, 8) TRI_C(16, 1) TRI_C(16, 4) TRI_C(16, 8) TRI_C(32, 1) TRI_C(32, 4)
#undef TRI_C
        return cudaErrorInvalidValue;
    });
}

}  // namespace

extern "C" int tri_collide(const float *centres, const float *radii, uint32_t n, uint32_t dim, int map,
                           uint32_t rho, uint32_t reg, uint32_t *count, uint32_t *pairs, uint64_t pair_cap,
                           unsigned long long *n_pairs, void *stream)
{
    if ((n && (!centres || !radii)) || !n_pairs || (!pairs && pair_cap > 0)) return TRI_EINVAL;
    if (dim < 1 || dim > 3 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (reg == 0) reg = rho <= 16 ? 8 : 4;
    if ((reg != 1 && reg != 4 && reg != 8) || (reg == 8 && rho > 16)) return TRI_EINVAL;
    if (map < TRI_MAP_LAMBDA || map > TRI_MAP_LAMBDA_PDELTA) return TRI_EINVAL;
    if (n > 0) {  // every range check before the first call that touches the device
        const int st = map == TRI_MAP_UTM
                           ? ((uint64_t)n + 1) * n / 2 <= 0xFFFFFFFFull ? TRI_OK : TRI_ERANGE
                           : trihost::map_range(map, ((uint64_t)n + rho * reg - 1) / (rho * reg));
        if (st != TRI_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(n_pairs, 0, sizeof(*n_pairs), s) != cudaSuccess) return TRI_ECUDA;
    if (count && n && cudaMemsetAsync(count, 0, sizeof(uint32_t) * n, s) != cudaSuccess) return TRI_ECUDA;
    if (n == 0) return TRI_OK;
    const CollideOut o{count, pairs, pairs ? pair_cap : 0, n_pairs};
    switch (dim) {
    case 1: return launch_dim<1>(centres, radii, n, map, rho, reg, o, s);
    case 2: return launch_dim<2>(centres, radii, n, map, rho, reg, o, s);
    default: return launch_dim<3>(centres, radii, n, map, rho, reg, o, s);
    }
}
