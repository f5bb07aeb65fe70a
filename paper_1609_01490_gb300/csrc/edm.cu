// Euclidean distance matrix on CUDA cores in FP32 by direct differences
// (Section 5, test 2), single triangles under any map, and many uneven
// triangles in one persistent launch.
#include <cuda_runtime.h>

#include <type_traits>

#include "f32x2.cuh"
#include "tri_internal.h"
#include "tri_maps.cuh"

using namespace tri;

namespace {

constexpr int KC = 32;  // features staged per shared-memory pass

// Shared memory of a tile pass: the block's row points [k][r] (pitch S + 1,
// odd, so that the transposed writes of a warp hit distinct banks) and
// column points [k][c] (pitch S + 2, even, so that a thread's two adjacent
// columns load as one 8-byte word).  The pipelined form keeps two passes of
// KC features in dynamic shared memory, one computed while the next is
// copied in.
template <int RHO, int R>
struct TileSmem {
    static constexpr int S = RHO * R;
    static constexpr int LI = S + 1, LJ = S + 2;
    static constexpr int PASS = KC * (LI + LJ);  // floats (even: the column part stays 8-byte aligned)
    static constexpr size_t PIPE_BYTES = sizeof(float) * 2 * PASS;
};

// Asynchronous 4-byte global -> shared copy (zero-filled when !valid, which
// then reads nothing).
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

template <int R>
struct TileAcc {
    static constexpr int RC = R == 1 ? 1 : R / 2;  // column groups per thread
    // a[u][v]: packed partial sums of row u with columns c(v) and c(v) + 1
    // (R >= 2); for R = 1 the low half holds the single pair
    unsigned long long a[R][RC];
};

// Features [0, kc) of one staged pass added into the thread's pairs.
template <int RHO, int R>
__device__ __forceinline__ void tile_pass(const float *si, const float *sj, uint32_t kc, int tx, int ty,
                                          TileAcc<R> &acc)
{
    using L = TileSmem<RHO, R>;
    constexpr int RC = TileAcc<R>::RC;
    if constexpr (R == 1) {
        float a = __uint_as_float((uint32_t)acc.a[0][0]);
#pragma unroll 4
        for (uint32_t k = 0; k < kc; ++k) {
            const float df = si[k * L::LI + ty] - sj[k * L::LJ + tx];
            a = fmaf(df, df, a);
        }
        acc.a[0][0] = __float_as_uint(a);
    } else {
#pragma unroll 4
        for (uint32_t k = 0; k < kc; ++k) {
            unsigned long long b2[RC];
#pragma unroll
            for (int v = 0; v < RC; ++v)
                b2[v] = *reinterpret_cast<const unsigned long long *>(sj + k * L::LJ + 2 * tx + 2 * RHO * v);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                const float a = si[k * L::LI + ty + u * RHO];
                const unsigned long long a2 = f2_pack(a, a);
#pragma unroll
                for (int v = 0; v < RC; ++v) {
                    const unsigned long long df = f2_sub(a2, b2[v]);
                    acc.a[u][v] = f2_fma(df, df, acc.a[u][v]);
                }
            }
        }
    }
}

// The square roots of the thread's pairs with j <= i < n, to the packed rows.
template <int RHO, int R>
__device__ __forceinline__ void tile_store(const TileAcc<R> &acc, float *__restrict__ out, uint32_t n, uint64_t i0,
                                           uint64_t j0, int tx, int ty)
{
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const uint64_t i = i0 + ty + u * RHO;
        if (i >= n) continue;
        float *row = out + T2(i);
        if constexpr (R == 1) {
            const uint64_t j = j0 + tx;
            if (j <= i) row[j] = sqrtf(__uint_as_float((uint32_t)acc.a[0][0]));
        } else {
#pragma unroll
            for (int v = 0; v < TileAcc<R>::RC; ++v) {
                const uint64_t j = j0 + 2 * tx + 2 * RHO * v;
                float lo, hi;
                f2_unpack(acc.a[u][v], lo, hi);
                if (j <= i) row[j] = sqrtf(lo);
                if (j + 1 <= i) row[j + 1] = sqrtf(hi);
            }
        }
    }
}

// The pipelined tile's pass buffers: the start of the kernel's dynamic shared memory.
extern __shared__ __align__(16) float tile_smem[];

// One (RHO R) x (RHO R) tile.  Thread (ty, tx) owns rows ty + u RHO and, for
// R = 1, column tx; for R >= 2, the column pairs 2 tx + 2 RHO v + {0, 1}
// (v < R / 2), updated two at a time with f32x2 instructions, so that a
// warp's 16 threads of a row cover 32 consecutive columns.  The features are
// taken KC at a time.  PIPE = false (d <= KC: one pass, nothing to overlap)
// stages with plain loads and stores into static shared memory; PIPE = true
// copies the next pass in asynchronously while the current one is computed
// (TileSmem::PIPE_BYTES of dynamic shared memory) and ends without a block
// barrier: a caller that runs another tile in the same block synchronises
// the block first.
// Not inlined: every block map calls the same compiled tile body, so the maps
// differ only in how a block finds its (bi, bj).
template <int RHO, int R, bool PIPE>
__device__ __noinline__ void edm_tile(const float *__restrict__ x, uint32_t n, uint32_t d,
                                      float *__restrict__ out, uint32_t bi, uint32_t bj)
{
    using L = TileSmem<RHO, R>;
    constexpr int S = L::S;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * RHO + tx;
    const uint64_t i0 = (uint64_t)bi * S, j0 = (uint64_t)bj * S;
    TileAcc<R> acc;
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < TileAcc<R>::RC; ++v) acc.a[u][v] = 0ull;

    if constexpr (!PIPE) {
        __shared__ float si[KC][L::LI];
        __shared__ __align__(8) float sj[KC][L::LJ];
        for (uint32_t k0 = 0; k0 < d; k0 += KC) {
            const uint32_t kc = min((uint32_t)KC, d - k0);
            // stage x[i0 + r][k0 + k] and x[j0 + r][k0 + k], transposed to [k][r]
            for (uint32_t t = tid; t < (uint32_t)S * kc; t += RHO * RHO) {
                const uint32_t r = t / kc, k = t - r * kc;
                const uint64_t gi = i0 + r, gj = j0 + r;
                si[k][r] = gi < n ? x[gi * d + k0 + k] : 0.0f;
                sj[k][r] = gj < n ? x[gj * d + k0 + k] : 0.0f;
            }
            __syncthreads();
            tile_pass<RHO, R>(&si[0][0], &sj[0][0], kc, tx, ty, acc);
            __syncthreads();
        }
    } else {
        // copy features [k0, k0 + KC) of the block's rows and columns,
        // transposed to [k][r], into pass buffer b (a warp reads 32
        // consecutive features of one point: one 128-byte line)
        auto stage = [&](int b, uint32_t k0) {
            float *si = tile_smem + b * L::PASS, *sj = si + KC * L::LI;
            const uint32_t kc = min((uint32_t)KC, d - k0);
            auto one = [&](uint32_t r, uint32_t k) {
                const uint64_t gi = i0 + r, gj = j0 + r;
                cp_async4(si + k * L::LI + r, gi < n ? x + gi * d + k0 + k : x, gi < n);
                cp_async4(sj + k * L::LJ + r, gj < n ? x + gj * d + k0 + k : x, gj < n);
            };
            if (kc == KC) {
                for (uint32_t e = tid; e < (uint32_t)S * KC; e += RHO * RHO) one(e / KC, e % KC);
            } else {
                for (uint32_t e = tid; e < (uint32_t)S * kc; e += RHO * RHO) {
                    const uint32_t r = e / kc;
                    one(r, e - r * kc);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        const uint32_t passes = (d + KC - 1) / KC;
        stage(0, 0);
        for (uint32_t c = 0; c < passes; ++c) {
            if (c + 1 < passes) {
                stage((c + 1) & 1, (c + 1) * KC);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            const float *si = tile_smem + (c & 1) * L::PASS;
            tile_pass<RHO, R>(si, si + KC * L::LI, min((uint32_t)KC, d - c * KC), tx, ty, acc);
            if (c + 2 < passes) __syncthreads();  // this buffer is refilled for pass c + 2
        }
    }
    tile_store<RHO, R>(acc, out, n, i0, j0, tx, ty);
}

template <int MAP, int RHO, int R, bool PIPE>
__global__ void __launch_bounds__(RHO *RHO) edm_kernel(const float *__restrict__ x, uint32_t n, uint32_t d,
                                                       float *__restrict__ out, BlockMap bm)
{
    uint32_t bi, bj;
    if (!map_block<MAP>(bm, bi, bj)) return;
    edm_tile<RHO, R, PIPE>(x, n, d, out, bi, bj);
}

// UTM is a thread-space map: one thread per pair, no tile to stage.
__global__ void edm_utm_kernel(const float *__restrict__ x, uint32_t n, uint32_t d, float *__restrict__ out)
{
    const uint64_t N = (uint64_t)n + 1;
    const uint64_t total = N * n / 2;
    const uint64_t k = ((uint64_t)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                       threadIdx.y * blockDim.x + threadIdx.x;
    if (k >= total) return;
    uint32_t a, b;
    utm_pair(k, N, a, b);
    const uint64_t i = b - 2, j = a - 1;
    const float *xi = x + i * d, *xj = x + j * d;
    float acc = 0.0f;
    for (uint32_t t = 0; t < d; ++t) {
        const float df = xi[t] - xj[t];
        acc = fmaf(df, df, acc);
    }
    out[T2(i) + j] = sqrtf(acc);
}

template <int MAP, int RHO, int R>
cudaError_t launch_one(dim3 g, cudaStream_t s, const float *x, uint32_t n, uint32_t d, float *out, BlockMap bm)
{
    if (d <= (uint32_t)KC) {
        edm_kernel<MAP, RHO, R, false><<<g, dim3(RHO, RHO), 0, s>>>(x, n, d, out, bm);
        return cudaGetLastError();
    }
    constexpr size_t smem = TileSmem<RHO, R>::PIPE_BYTES;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(edm_kernel<MAP, RHO, R, true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    edm_kernel<MAP, RHO, R, true><<<g, dim3(RHO, RHO), smem, s>>>(x, n, d, out, bm);
    return cudaGetLastError();
}

template <int MAP>
cudaError_t launch_rr(uint32_t rho, uint32_t reg, dim3 g, cudaStream_t s, const float *x, uint32_t n, uint32_t d,
                      float *out, BlockMap bm)
{
#define TRI_E(RH, RG)                                                                                          \
    if (rho == RH && reg == RG) return launch_one<MAP, RH, RG>(g, s, x, n, d, out, bm);
    TRI_E(8, 1) TRI_E(8, 2) TRI_E(8, 4) TRI_E(8, 8) TRI_E(16, 1) TRI_E(16, 2) TRI_E(16, 4) TRI_E(16, 8)
    TRI_E(32, 1) TRI_E(32, 2) TRI_E(32, 4)
#undef TRI_E
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ batched ----
// Exclusive prefix sum of the per-instance block counts m_k(m_k+1)/2 into
// off[0..count], in one block with a fixed order (no inter-block waiting).
__global__ void batched_scan_kernel(const uint32_t *__restrict__ n_k, uint32_t count, uint32_t S,
                                    uint64_t *__restrict__ off, int *__restrict__ status)
{
    __shared__ uint64_t part[1024];
    const uint32_t t = threadIdx.x, nt = blockDim.x;
    const uint32_t per = (count + nt - 1) / nt;
    const uint32_t b0 = min(count, t * per), b1 = min(count, b0 + per);
    uint64_t s = 0;
    for (uint32_t k = b0; k < b1; ++k) {
        const uint64_t m = (n_k[k] + (uint64_t)S - 1) / S;
        const uint64_t nb = T2(m);
        if (nb <= 0xFFFFFFFFull) s += nb;
    }
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        uint64_t run = 0;
        for (uint32_t q = 0; q < nt; ++q) {
            const uint64_t v = part[q];
            part[q] = run;
            run += v;
        }
    }
    __syncthreads();
    uint64_t run = part[t];
    for (uint32_t k = b0; k < b1; ++k) {
        off[k] = run;
        const uint64_t m = (n_k[k] + (uint64_t)S - 1) / S;
        const uint64_t nb = T2(m);
        if (nb <= 0xFFFFFFFFull) {
            run += nb;
        } else {
            atomicExch(status, (int)TRI_ERANGE);  // instance skipped: lambda needs omega < 2^32
        }
    }
    if (t == nt - 1) off[count] = run;
}

// Persistent CTAs walk the global block numbers omega_g with a grid stride;
// each finds its instance by binary search over the block offsets (staged in
// shared memory when they fit) and maps the local number with lambda.
template <int RHO, int R, bool PIPE>
__global__ void __launch_bounds__(RHO *RHO)
    edm_batched_kernel(const float *__restrict__ x_cat, const uint64_t *__restrict__ pt_off,
                       const uint32_t *__restrict__ n_k, uint32_t count, uint32_t d, float *__restrict__ out_cat,
                       const uint64_t *__restrict__ out_off, const uint64_t *__restrict__ boff, uint32_t smem_cnt)
{
    // dynamic shared memory: the tile's pass buffers, then the block offsets
    uint64_t *soff = reinterpret_cast<uint64_t *>(tile_smem + (PIPE ? 2 * TileSmem<RHO, R>::PASS : 0));
    const bool in_smem = smem_cnt >= count + 1;
    if (in_smem)
        for (uint32_t t = threadIdx.y * RHO + threadIdx.x; t <= count; t += RHO * RHO) soff[t] = boff[t];
    __syncthreads();
    const uint64_t *off = in_smem ? soff : boff;
    const uint64_t total = off[count];
    for (uint64_t wg = blockIdx.x; wg < total; wg += gridDim.x) {
        // largest k with off[k] <= wg (instances with no blocks are skipped)
        uint32_t lo = 0, hi = count;  // off[lo] <= wg < off[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= wg) lo = mid;
            else hi = mid;
        }
        uint32_t bi, bj;
        lambda_diag<TRI_SQRT_R>((uint32_t)(wg - off[lo]), bi, bj);
        // a pipelined tile ends without a barrier: the block's previous
        // tile has read its last pass before this tile's first copies land
        if (PIPE) __syncthreads();
        edm_tile<RHO, R, PIPE>(x_cat + pt_off[lo] * d, n_k[lo], d, out_cat + out_off[lo], bi, bj);
    }
}

template <int RHO, int R, bool PIPE>
cudaError_t launch_batched_pipe(cudaStream_t s, const float *x_cat, const uint64_t *pt_off, const uint32_t *n_k,
                                uint32_t count, uint32_t d, float *out_cat, const uint64_t *out_off,
                                const uint64_t *boff)
{
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    uint32_t smem_cnt = count + 1;
    if (smem_cnt > 4096) smem_cnt = 0;  // large batches search the offsets in global memory
    const size_t dyn = (PIPE ? TileSmem<RHO, R>::PIPE_BYTES : 0) + (size_t)smem_cnt * sizeof(uint64_t);
    if (cudaFuncSetAttribute(edm_batched_kernel<RHO, R, PIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn) != cudaSuccess)
        return cudaErrorInvalidValue;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, edm_batched_kernel<RHO, R, PIPE>, RHO * RHO, dyn);
    if (per < 1) per = 1;
    edm_batched_kernel<RHO, R, PIPE><<<nsm * per, dim3(RHO, RHO), dyn, s>>>(x_cat, pt_off, n_k, count, d, out_cat,
                                                                             out_off, boff, smem_cnt);
    return cudaGetLastError();
}

template <int RHO, int R>
cudaError_t launch_batched_one(cudaStream_t s, const float *x_cat, const uint64_t *pt_off, const uint32_t *n_k,
                               uint32_t count, uint32_t d, float *out_cat, const uint64_t *out_off,
                               const uint64_t *boff)
{
    if (d <= (uint32_t)KC)
        return launch_batched_pipe<RHO, R, false>(s, x_cat, pt_off, n_k, count, d, out_cat, out_off, boff);
    return launch_batched_pipe<RHO, R, true>(s, x_cat, pt_off, n_k, count, d, out_cat, out_off, boff);
}

}  // namespace

int trihost::edm_fp32(const float *x, uint32_t n, uint32_t d, float *out, int map, uint32_t rho, uint32_t reg,
                      cudaStream_t s)
{
    if (reg == 0) reg = 4;  // 4 x 4 pairs per thread: fastest at every d measured (3, 64, 128)
    // 8 x 8 pairs per thread only with rho <= 16 (registers and static shared memory)
    if ((reg != 1 && reg != 2 && reg != 4 && reg != 8) || (reg == 8 && rho > 16)) return TRI_EINVAL;
    if (map == TRI_MAP_UTM) {
        const uint64_t N = (uint64_t)n + 1, total = N * n / 2, tpb = (uint64_t)rho * rho;
        if (total > 0xFFFFFFFFull) return TRI_ERANGE;
        edm_utm_kernel<<<trihost::linear_grid((total + tpb - 1) / tpb), dim3(rho, rho), 0, s>>>(x, n, d, out);
        return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
    }
    const uint32_t S = rho * reg;
    const uint32_t m = (n + S - 1) / S;
    BlockMap bm{};
    bm.m = m;
    bm.nblocks = T2(m);
    cudaError_t e = cudaSuccess;
    switch (map) {
    case TRI_MAP_LAMBDA:
        if (bm.nblocks > 0xFFFFFFFFull) return TRI_ERANGE;
        e = launch_rr<MAP_LAMBDA>(rho, reg, trihost::linear_grid(bm.nblocks), s, x, n, d, out, bm);
        break;
    case TRI_MAP_LAMBDA_PDELTA: {
        if (bm.nblocks > 0xFFFFFFFFull) return TRI_ERANGE;
        const uint64_t mp = trihost::isqrt_ceil(bm.nblocks);
        if (mp > 65535) return TRI_ERANGE;
        e = launch_rr<MAP_LAMBDA_PD>(rho, reg, dim3((unsigned)mp, (unsigned)mp), s, x, n, d, out, bm);
        break;
    }
    case TRI_MAP_BB:
        if (m > 65535) return TRI_ERANGE;
        e = launch_rr<MAP_BB>(rho, reg, dim3(m, m), s, x, n, d, out, bm);
        break;
    case TRI_MAP_RB: {
        const uint32_t h = (m & 1u) ? (m + 1) / 2 : m / 2 + 1;
        if (h > 65535) return TRI_ERANGE;
        e = launch_rr<MAP_RB>(rho, reg, dim3(m, h), s, x, n, d, out, bm);
        break;
    }
    case TRI_MAP_REC: {
        if (!trihost::is_pow2(m)) return TRI_ERANGE;
        const uint32_t k = trihost::ilog2(m);
        if (k > 0 && m / 2 > 65535) return TRI_ERANGE;
        for (uint32_t l = 0; l <= k && e == cudaSuccess; ++l) {
            bm.level = l;
            const dim3 g = l == 0 ? dim3(m) : dim3(1u << (l - 1), m / 2);
            e = launch_rr<MAP_REC>(rho, reg, g, s, x, n, d, out, bm);
        }
        break;
    }
    default:
        return TRI_EINVAL;
    }
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tri_edm_batched_workspace_size(uint32_t count, size_t *bytes)
{
    if (!bytes) return TRI_EINVAL;
    *bytes = 16 + sizeof(uint64_t) * ((size_t)count + 1);
    return TRI_OK;
}

extern "C" int tri_edm_batched(const float *x_cat, const uint64_t *pt_off, const uint32_t *n_k, uint32_t count,
                               uint32_t d, float *out_cat, const uint64_t *out_off, uint32_t rho, uint32_t reg,
                               void *workspace, size_t ws_bytes, void *stream)
{
    if (!x_cat || !pt_off || !n_k || !out_cat || !out_off || !workspace || d == 0 || count == 0)
        return TRI_EINVAL;
    if (!trihost::rho_ok(rho)) return TRI_EINVAL;
    if (reg == 0) reg = 4;  // 4 x 4 pairs per thread: fastest at every d measured (3, 64, 128)
    // 8 x 8 pairs per thread only with rho <= 16 (registers and static shared memory)
    if ((reg != 1 && reg != 2 && reg != 4 && reg != 8) || (reg == 8 && rho > 16)) return TRI_EINVAL;
    size_t need = 0;
    tri_edm_batched_workspace_size(count, &need);
    if (ws_bytes < need || ((uintptr_t)workspace & 15)) return TRI_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int *status = (int *)workspace;
    uint64_t *boff = (uint64_t *)((char *)workspace + 16);
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return TRI_ECUDA;
    batched_scan_kernel<<<1, 1024, 0, s>>>(n_k, count, rho * reg, boff, status);
    if (cudaGetLastError() != cudaSuccess) return TRI_ECUDA;
    cudaError_t e = cudaErrorInvalidValue;
#define TRI_B(RH, RG)                                                                                          \
    if (rho == RH && reg == RG)                                                                                \
        e = launch_batched_one<RH, RG>(s, x_cat, pt_off, n_k, count, d, out_cat, out_off, boff);
    TRI_B(8, 1) TRI_B(8, 2) TRI_B(8, 4) TRI_B(8, 8) TRI_B(16, 1) TRI_B(16, 2) TRI_B(16, 4) TRI_B(16, 8)
    TRI_B(32, 1) TRI_B(32, 2) TRI_B(32, 4)
#undef TRI_B
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}
