// Entry points that dispatch between kernels, and library metadata.
#include <cuda_runtime.h>

#include "tri_internal.h"
#include "tri_maps.cuh"

extern "C" const char *tri_status_string(int status)
{
    switch (status) {
    case TRI_OK: return "TRI_OK";
    case TRI_EINVAL: return "TRI_EINVAL: invalid argument";
    case TRI_ERANGE: return "TRI_ERANGE: size out of the map's range";
    case TRI_ECUDA: return "TRI_ECUDA: CUDA runtime or launch error";
    case TRI_EOVERFLOW: return "TRI_EOVERFLOW: device list overflow";
    case TRI_ETIMEOUT: return "TRI_ETIMEOUT: bounded device wait gave up";
    case TRI_ENOSPACE: return "TRI_ENOSPACE: workspace too small or misaligned";
    default: return "unknown tri_status";
    }
}

extern "C" int tri_version(void) { return 10000; }

extern "C" int tri_edm_workspace_size(uint32_t n, uint32_t d, int prec, size_t *bytes)
{
    if (!bytes) return TRI_EINVAL;
    if (prec == TRI_FP32) {
        *bytes = 0;
        return TRI_OK;
    }
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    *bytes = trihost::edm_tc_workspace(n, d, prec);
    return TRI_OK;
}

extern "C" int tri_edm(const float *x, uint32_t n, uint32_t d, float *out, int map, uint32_t rho, uint32_t reg,
                       int prec, void *workspace, size_t ws_bytes, unsigned long long *n_flagged, void *stream)
{
    if (!x || !out || n == 0 || d == 0) return TRI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == TRI_FP32) {
        if (!trihost::rho_ok(rho)) return TRI_EINVAL;
        if (n_flagged && cudaMemsetAsync(n_flagged, 0, sizeof(*n_flagged), s) != cudaSuccess) return TRI_ECUDA;
        return trihost::edm_fp32(x, n, d, out, map, rho, reg, s);
    }
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_BB) return TRI_EINVAL;
    return trihost::edm_tc(x, n, d, out, map, prec, workspace, ws_bytes, n_flagged, s);
}
