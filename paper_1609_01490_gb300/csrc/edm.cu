// Euclidean distance matrix on CUDA cores in FP32 by direct differences
// (Section 5, test 2): one triangle under any block map.  The tile itself is
// in edm_tile.cuh; many uneven triangles in one launch are in edm_batched.cu.
#include <cuda_runtime.h>

#include "edm_tile.cuh"
#include "tri_internal.h"

using namespace tri;
using namespace tri::tile;

namespace {

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
        edm_kernel<MAP, RHO, R, false><<<g, dim3(RHO, RHO), TileSmem<RHO, R>::bytes(false), s>>>(x, n, d, out, bm);
        return cudaGetLastError();
    }
    constexpr size_t smem = TileSmem<RHO, R>::bytes(true);
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

}  // namespace

int trihost::edm_fp32(const float *x, uint32_t n, uint32_t d, float *out, int map, uint32_t rho, uint32_t reg,
                      cudaStream_t s)
{
    if (reg == 0) reg = 4;  // 4 x 4 pairs per thread: fastest at every d measured (3, 64, 128)
    // 8 x 8 pairs per thread only with rho <= 16 (registers and shared memory)
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
