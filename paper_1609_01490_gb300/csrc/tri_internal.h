// Entry points shared between the library's translation units (not exported).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace trihost {

// FP32 direct-difference EDM under any block map (edm.cu).
int edm_fp32(const float *x, uint32_t n, uint32_t d, float *out, int map, uint32_t rho, uint32_t reg,
             cudaStream_t s);

// Tensor-core Gram EDM with split-BF16 operands and FP64 recompute (edm_tc.cu).
size_t edm_tc_workspace(uint32_t n, uint32_t d, int prec);
int edm_tc(const float *x, uint32_t n, uint32_t d, float *out, int map, int prec, void *ws, size_t ws_bytes,
           unsigned long long *n_flagged, cudaStream_t s);

}  // namespace trihost
