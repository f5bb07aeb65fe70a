// Many uneven Euclidean distance triangles (Section 5, test 2) in one
// persistent launch: every instance's blocks are numbered in one global
// sequence, each CTA finds the instance of a number by binary search over the
// per-instance block offsets and maps the local number with lambda (Eq. 4).
#include <cuda_runtime.h>

#include "edm_tile.cuh"
#include "tri_internal.h"

using namespace tri;
using namespace tri::tile;

namespace {

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

// The tile variant for a block: UA live row groups, the smallest compiled
// count >= ua (counts step by R / 4 at R = 8, by 1 below), and the diagonal
// form on the instance's diagonal blocks (R >= 4; at R <= 2 a thread has one
// column group, which the diagonal form keeps).  Where instances span only a
// few tiles a side, their last row blocks and diagonal blocks are a sizeable
// share of all tiles, and these forms skip the accumulators past n or above
// the diagonal.
template <int RHO, int R, bool PIPE, int UA = R>
__device__ __forceinline__ void batched_tile(int ua, bool diag, const float *x, uint32_t n, uint32_t d, float *out,
                                             uint32_t bi, uint32_t bj)
{
    constexpr int STEP = R >= 8 ? R / 4 : 1;
    if constexpr (UA > STEP) {
        if (ua <= UA - STEP) {
            batched_tile<RHO, R, PIPE, UA - STEP>(ua, diag, x, n, d, out, bi, bj);
            return;
        }
    }
    if constexpr (R >= 4) {
        if (diag) {
            edm_tile_body<RHO, R, PIPE, UA, true>(x, n, d, out, bi, bj);
            return;
        }
    }
    edm_tile_body<RHO, R, PIPE, UA, false>(x, n, d, out, bi, bj);
}

// Persistent CTAs take the global block numbers omega_g in turn: the first
// is the CTA's index, each later one the next value of a device counter plus
// the grid size, claimed with one atomic at the start of a tile and read at
// its end, so that the claim's latency hides behind the tile and CTAs that
// run faster take more tiles.  Each CTA finds the instance of its number by
// binary search over the block offsets (staged in shared memory when they
// fit) and maps the local number with lambda.
template <int RHO, int R, bool PIPE>
__global__ void __launch_bounds__(RHO *RHO)
    edm_batched_kernel(const float *__restrict__ x_cat, const uint64_t *__restrict__ pt_off,
                       const uint32_t *__restrict__ n_k, uint32_t count, uint32_t d, float *__restrict__ out_cat,
                       const uint64_t *__restrict__ out_off, const uint64_t *__restrict__ boff, uint32_t smem_cnt,
                       unsigned long long *__restrict__ claims)
{
    constexpr uint32_t S = RHO * R;
    const uint32_t tid = threadIdx.y * RHO + threadIdx.x;
    // dynamic shared memory: the tile's pass buffers (an even number of
    // floats), then the block offsets
    uint64_t *soff = reinterpret_cast<uint64_t *>(tile_smem + (PIPE ? 2 : 1) * TileSmem<RHO, R>::PASS);
    __shared__ uint64_t s_next[2];  // the next block number, alternating between tiles
    const bool in_smem = smem_cnt >= count + 1;
    if (in_smem)
        for (uint32_t t = tid; t <= count; t += RHO * RHO) soff[t] = boff[t];
    __syncthreads();
    const uint64_t *off = in_smem ? soff : boff;
    const uint64_t total = off[count];
    uint64_t wg = blockIdx.x;
    for (uint32_t it = 0; wg < total; ++it) {
        unsigned long long claim = 0;
        if (tid == 0) claim = atomicAdd(claims, 1ull);
        // largest k with off[k] <= wg (instances with no blocks are skipped)
        uint32_t lo = 0, hi = count;  // off[lo] <= wg < off[hi]
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= wg) lo = mid;
            else hi = mid;
        }
        uint32_t bi, bj;
        lambda_diag<TRI_SQRT_R>((uint32_t)(wg - off[lo]), bi, bj);
        const uint32_t n = n_k[lo];
        // rows of the instance from the block's first row on: bi < ceil(n / S)
        const uint32_t left = n - bi * S;
        const int ua = left >= S ? R : (int)((left + RHO - 1) / RHO);
        batched_tile<RHO, R, PIPE>(ua, bi == bj, x_cat + pt_off[lo] * d, n, d, out_cat + out_off[lo], bi, bj);
        if (tid == 0) s_next[it & 1] = gridDim.x + claim;
        // the barrier publishes the next number and ends the tile: a
        // pipelined tile returns without one, and the next tile's first
        // copies must not land before every warp has read the last pass
        __syncthreads();
        wg = s_next[it & 1];
    }
}

template <int RHO, int R, bool PIPE>
cudaError_t launch_batched_pipe(cudaStream_t s, const float *x_cat, const uint64_t *pt_off, const uint32_t *n_k,
                                uint32_t count, uint32_t d, float *out_cat, const uint64_t *out_off,
                                const uint64_t *boff, unsigned long long *claims)
{
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    uint32_t smem_cnt = count + 1;
    if (smem_cnt > 4096) smem_cnt = 0;  // large batches search the offsets in global memory
    const size_t dyn = TileSmem<RHO, R>::bytes(PIPE) + (size_t)smem_cnt * sizeof(uint64_t);
    if (cudaFuncSetAttribute(edm_batched_kernel<RHO, R, PIPE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn) != cudaSuccess)
        return cudaErrorInvalidValue;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, edm_batched_kernel<RHO, R, PIPE>, RHO * RHO, dyn);
    if (per < 1) per = 1;
    edm_batched_kernel<RHO, R, PIPE><<<nsm * per, dim3(RHO, RHO), dyn, s>>>(x_cat, pt_off, n_k, count, d, out_cat,
                                                                             out_off, boff, smem_cnt, claims);
    return cudaGetLastError();
}

template <int RHO, int R>
cudaError_t launch_batched_one(cudaStream_t s, const float *x_cat, const uint64_t *pt_off, const uint32_t *n_k,
                               uint32_t count, uint32_t d, float *out_cat, const uint64_t *out_off,
                               const uint64_t *boff, unsigned long long *claims)
{
    if (d <= (uint32_t)KC)
        return launch_batched_pipe<RHO, R, false>(s, x_cat, pt_off, n_k, count, d, out_cat, out_off, boff, claims);
    return launch_batched_pipe<RHO, R, true>(s, x_cat, pt_off, n_k, count, d, out_cat, out_off, boff, claims);
}

}  // namespace

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
    // 8 x 8 pairs per thread only with rho <= 16 (registers and shared memory)
    if ((reg != 1 && reg != 2 && reg != 4 && reg != 8) || (reg == 8 && rho > 16)) return TRI_EINVAL;
    size_t need = 0;
    tri_edm_batched_workspace_size(count, &need);
    if (ws_bytes < need || ((uintptr_t)workspace & 15)) return TRI_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    // workspace: the status word at byte 0, the tile-claim counter at byte 8,
    // the block offsets from byte 16
    int *status = (int *)workspace;
    unsigned long long *claims = (unsigned long long *)((char *)workspace + 8);
    uint64_t *boff = (uint64_t *)((char *)workspace + 16);
    if (cudaMemsetAsync(workspace, 0, 16, s) != cudaSuccess) return TRI_ECUDA;
    batched_scan_kernel<<<1, 1024, 0, s>>>(n_k, count, rho * reg, boff, status);
    if (cudaGetLastError() != cudaSuccess) return TRI_ECUDA;
    cudaError_t e = cudaErrorInvalidValue;
#define TRI_B(RH, RG)                                                                                          \
    if (rho == RH && reg == RG)                                                                                \
        e = launch_batched_one<RH, RG>(s, x_cat, pt_off, n_k, count, d, out_cat, out_off, boff, claims);
    TRI_B(8, 1) TRI_B(8, 2) TRI_B(8, 4) TRI_B(8, 8) TRI_B(16, 1) TRI_B(16, 2) TRI_B(16, 4) TRI_B(16, 8)
    TRI_B(32, 1) TRI_B(32, 2) TRI_B(32, 4)
#undef TRI_B
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

// Instances of one batch for several GPUs: with B_k = T(ceil(n_k / S)) the
// block count of instance k (S = rho reg) and P_k = B_0 + ... + B_{k-1}, rank
// r takes the instances k whose P_k lies in [r / ranks, (r + 1) / ranks) of
// the total, each whole: its own slices of pt_off, n_k and out_off, no shared
// output.
extern "C" int tri_edm_batched_partition(const uint32_t *n_k, uint32_t count, uint32_t rho, uint32_t reg,
                                         uint32_t ranks, uint32_t rank, uint32_t *k_begin, uint32_t *k_end)
{
    if ((!n_k && count > 0) || !k_begin || !k_end || ranks == 0 || rank >= ranks) return TRI_EINVAL;
    if (!trihost::rho_ok(rho) || (reg != 1 && reg != 2 && reg != 4 && reg != 8) || (reg == 8 && rho > 16))
        return TRI_EINVAL;
    const uint64_t S = (uint64_t)rho * reg;
    uint64_t total = 0;
    for (uint32_t k = 0; k < count; ++k) total += T2((n_k[k] + S - 1) / S);
    // first instance whose prefix reaches share r of the total (count if none)
    auto edge = [&](uint32_t r) -> uint32_t {
        if (r == 0) return 0;
        if (r >= ranks) return count;
        const long double target = (long double)total * r / ranks;
        uint64_t run = 0;
        for (uint32_t k = 0; k < count; ++k) {
            if ((long double)run >= target) return k;
            run += T2((n_k[k] + S - 1) / S);
        }
        return count;
    };
    *k_begin = edge(rank);
    *k_end = edge(rank + 1);
    return TRI_OK;
}
