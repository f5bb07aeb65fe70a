// Arithmetic peak probes for the ALU rooflines: long chains of independent
// fused multiply-adds per thread, timed by the caller.  FP32 scalar, FP32 in
// two-lane f32x2 form and FP64; each counts 2 flop per lane per FMA.
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "tri_maps.cuh"

using namespace tri;

namespace {

constexpr int CHAINS = 8;  // independent accumulators per thread (covers the FMA latency)

template <int KIND>
__global__ void __launch_bounds__(256) fma_probe_kernel(uint32_t iters, float seed, float *sink)
{
    const float b = 0.999999f, c = 1e-7f * seed;
    if constexpr (KIND == 0) {
        float a[CHAINS];
#pragma unroll
        for (int q = 0; q < CHAINS; ++q) a[q] = seed + q + threadIdx.x;
        for (uint32_t t = 0; t < iters; ++t)
#pragma unroll
            for (int q = 0; q < CHAINS; ++q) a[q] = fmaf(a[q], b, c);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < CHAINS; ++q) s += a[q];
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else if constexpr (KIND == 1) {
        f2 a[CHAINS];
        const f2 B = f2_pack(b, b), C = f2_pack(c, c);
#pragma unroll
        for (int q = 0; q < CHAINS; ++q) a[q] = f2_pack(seed + q, seed - q + threadIdx.x);
        for (uint32_t t = 0; t < iters; ++t)
#pragma unroll
            for (int q = 0; q < CHAINS; ++q) a[q] = f2_fma(a[q], B, C);
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < CHAINS; ++q) {
            float lo, hi;
            f2_unpack(a[q], lo, hi);
            s += lo + hi;
        }
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else {
        double a[CHAINS];
        const double bd = b, cd = c;
#pragma unroll
        for (int q = 0; q < CHAINS; ++q) a[q] = (double)seed + q + threadIdx.x;
        for (uint32_t t = 0; t < iters; ++t)
#pragma unroll
            for (int q = 0; q < CHAINS; ++q) a[q] = fma(a[q], bd, cd);
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < CHAINS; ++q) s += a[q];
        sink[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
    }
}

}  // namespace

extern "C" int tri_peak_probe(int kind, uint32_t blocks, uint32_t iters, float *sink, double *flop, void *stream)
{
    if (!sink || !flop || blocks == 0 || (kind < 0 || kind > 2)) return TRI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0) fma_probe_kernel<0><<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
    else if (kind == 1) fma_probe_kernel<1><<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
    else fma_probe_kernel<2><<<blocks, 256, 0, s>>>(iters, 1.0f, sink);
    const double lanes = kind == 1 ? 2.0 : 1.0;
    *flop = 2.0 * lanes * CHAINS * (double)iters * blocks * 256.0;
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}
