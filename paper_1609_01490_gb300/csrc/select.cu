// Map and rho selection from a learned cost model (not in the paper): the
// candidates of a (kernel, n, d) configuration, their features, and the
// model's argmin over them on the GPU; plus the read of device status words.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "tri_maps.cuh"

namespace {

constexpr int NF = TRI_SELECT_FEATURES;
constexpr uint32_t RHOS[3] = {8, 16, 32};
// map one-hot order of the features
constexpr int MAP_ORDER[6] = {TRI_MAP_LAMBDA, TRI_MAP_LAMBDA_PDELTA, TRI_MAP_BB, TRI_MAP_RB, TRI_MAP_REC, TRI_MAP_UTM};

// The candidate maps of each kernel (the autotuner's sets).
int kernel_maps(int kernel, int *maps)
{
    if (kernel == TRI_KERNEL_EDM) {
        for (int k = 0; k < 6; ++k) maps[k] = MAP_ORDER[k];
        return 6;
    }
    if (kernel == TRI_KERNEL_CA) {
        for (int k = 0; k < 5; ++k) maps[k] = MAP_ORDER[k];
        return 5;
    }
    maps[0] = TRI_MAP_LAMBDA;
    maps[1] = TRI_MAP_BB;
    return 2;
}

// Tile side in elements: the EDM default of 4 x 4 pairs per thread, the Life
// step's 4 rho cells, the triplet kernel's rho points.
uint64_t tile_side(int kernel, uint32_t rho) { return kernel == TRI_KERNEL_AT ? rho : 4ull * rho; }

// Blocks the map launches (the bounding box counts its discarded blocks).
double launched_blocks(int kernel, uint32_t n, int map, uint32_t rho)
{
    const double m = (double)((n + tile_side(kernel, rho) - 1) / tile_side(kernel, rho));
    if (kernel == TRI_KERNEL_AT) return map == TRI_MAP_BB ? m * m * m : m * (m + 1) * (m + 2) / 6.0;
    if (map == TRI_MAP_BB) return m * m;
    if (map == TRI_MAP_RB) {
        const uint64_t mi = (uint64_t)m;
        return m * (double)((mi & 1) ? (mi + 1) / 2 : mi / 2 + 1);
    }
    if (map == TRI_MAP_UTM) return (double)(n + 1) * n / 2.0 / ((double)rho * rho);
    return m * (m + 1) / 2.0;
}

// Candidates (maps outer, rho inner) and their features in FP64.
int features(int kernel, uint32_t n, uint32_t d, double *X, int *maps, uint32_t *rhos, uint32_t *count)
{
    if (!X || !maps || !rhos || !count || n == 0) return TRI_EINVAL;
    if (kernel != TRI_KERNEL_EDM && kernel != TRI_KERNEL_CA && kernel != TRI_KERNEL_AT) return TRI_EINVAL;
    int kmaps[6];
    const int nm = kernel_maps(kernel, kmaps);
    uint32_t c = 0;
    for (int a = 0; a < nm; ++a)
        for (uint32_t r : RHOS) {
            if (kmaps[a] == TRI_MAP_REC) {  // REC needs a power-of-two number of block rows
                const uint64_t side = tile_side(kernel, r), m = (n + side - 1) / side;
                if (m & (m - 1)) continue;
            }
            double *f = X + (size_t)c * NF;
            for (int q = 0; q < NF; ++q) f[q] = 0.0;
            const double blocks = launched_blocks(kernel, n, kmaps[a], r);
            f[0] = std::log2((double)n);
            f[1] = std::log2((double)(d > 1 ? d : 1));
            f[2] = std::log2((double)r);
            f[3] = std::log2(blocks > 1.0 ? blocks : 1.0);
            f[4 + kernel] = 1.0;
            for (int q = 0; q < 6; ++q)
                if (MAP_ORDER[q] == kmaps[a]) f[7 + q] = 1.0;
            f[13] = std::log2((double)tile_side(kernel, r));
            maps[c] = kmaps[a];
            rhos[c] = r;
            ++c;
        }
    *count = c;
    return TRI_OK;
}

}  // namespace

extern "C" int tri_select_features(int kernel, uint32_t n, uint32_t d, float *X, int *maps, uint32_t *rhos,
                                   uint32_t *count)
{
    if (!X) return TRI_EINVAL;
    double F[TRI_SELECT_MAX_CANDIDATES * NF];
    const int st = features(kernel, n, d, F, maps, rhos, count);
    if (st != TRI_OK) return st;
    for (uint32_t q = 0; q < *count * NF; ++q) X[q] = (float)F[q];
    return TRI_OK;
}

extern "C" int tri_select_workspace_size(uint32_t h1, uint32_t h2, size_t *bytes)
{
    if (!bytes) return TRI_EINVAL;
    size_t mlp = 0;
    const int st = tri_mlp_workspace_size(TRI_SELECT_MAX_CANDIDATES, h1, h2, &mlp);
    if (st != TRI_OK) return st;
    *bytes = 1024 + 256 + mlp;  // standardised features, argmin index, MLP activations
    return TRI_OK;
}

extern "C" int tri_select(const tri_cost_model *model, int kernel, uint32_t n, uint32_t d, int *map, uint32_t *rho,
                          void *workspace, size_t ws_bytes, void *stream)
{
    if (!map || !rho || n == 0) return TRI_EINVAL;
    if (kernel != TRI_KERNEL_EDM && kernel != TRI_KERNEL_CA && kernel != TRI_KERNEL_AT) return TRI_EINVAL;
    if (!model || !model->theta) {  // no model: the library default
        *map = TRI_MAP_LAMBDA;
        *rho = 16;
        return TRI_OK;
    }
    if (!model->mu || !model->sd) return TRI_EINVAL;
    size_t need = 0;
    int st = tri_select_workspace_size(model->h1, model->h2, &need);
    if (st != TRI_OK) return st;
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 255)) return TRI_ENOSPACE;
    double F[TRI_SELECT_MAX_CANDIDATES * NF];
    float X[TRI_SELECT_MAX_CANDIDATES * NF];
    int maps[TRI_SELECT_MAX_CANDIDATES];
    uint32_t rhos[TRI_SELECT_MAX_CANDIDATES], count = 0;
    if ((st = features(kernel, n, d, F, maps, rhos, &count)) != TRI_OK) return st;
    // standardised in FP64, rounded to FP32 once (as the trainer does)
    for (uint32_t c = 0; c < count; ++c)
        for (int q = 0; q < NF; ++q) {
            const double sd = model->sd[q] != 0.0 ? model->sd[q] : 1.0;
            X[c * NF + q] = (float)((F[c * NF + q] - model->mu[q]) / sd);
        }
    char *ws = (char *)workspace;
    float *Xd = (float *)ws;
    uint32_t *best = (uint32_t *)(ws + 1024);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(Xd, X, sizeof(float) * count * NF, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TRI_ECUDA;
    size_t mlp = 0;
    tri_mlp_workspace_size(TRI_SELECT_MAX_CANDIDATES, model->h1, model->h2, &mlp);
    if ((st = tri_mlp_argmin(model->theta, Xd, count, NF, model->h1, model->h2, best, ws + 1280, mlp, stream)) !=
        TRI_OK)
        return st;
    uint32_t b = 0;
    if (cudaMemcpyAsync(&b, best, sizeof(b), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TRI_ECUDA;
    if (b >= count) return TRI_ECUDA;
    *map = maps[b];
    *rho = rhos[b];
    return TRI_OK;
}

extern "C" int tri_sync_status(const int *status, int *value, void *stream)
{
    if (!status || !value) return TRI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int v = 0;
    if (cudaMemcpyAsync(&v, status, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TRI_ECUDA;
    *value = v;
    return TRI_OK;
}
