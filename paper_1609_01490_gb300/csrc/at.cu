// Axilrod-Teller triple-dipole energy over the strict triplets i > j > k:
// a triplet-interaction n-body sum on the tetrahedral domain of Section 6,
// with blocks placed by the tetrahedral lambda or by an m^3 bounding box.
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "tri_maps.cuh"
#include "tet_table.cuh"

using namespace tri;

namespace {

// Block (L, R, C), L >= R >= C, of rho x (rho / AT_ROWS) threads: thread
// (ty, tx) takes j = R*rho + tx and the AT_ROWS rows i = L*rho + ty + u*(rho /
// AT_ROWS), and loops k over block C (k < j), each b(j, k) read once for all
// its rows.  With squared sides a = |ij|^2, b = |jk|^2, c = |ki|^2 the law of
// cosines gives cos g_i cos g_j cos g_k = (a+c-b)(a+b-c)(b+c-a) / (8abc) and
// (r_ij r_jk r_ki)^3 = (abc)^(3/2).  Terms are formed and summed per thread in
// FP32 (two k at a time with f32x2 instructions, into two running sums per
// row), summed over each warp in FP32 and over the warps in FP64 into
// partial[T3(L)+T2(R)+C].  (Two rows per thread halve the per-triplet share
// of the block's setup: the map, the pair quantities and the sums.)
constexpr int AT_ROWS = 2;

template <int MAP>
__global__ void at_kernel(const float *__restrict__ p, uint32_t n, double nu, uint32_t m, uint64_t w0,
                          uint64_t nblocks, double *__restrict__ partial)
{
    uint32_t L, R, C;
    if constexpr (MAP == MAP_LAMBDA || MAP == MAP_TET_TABLE) {
        // blocks [w0, nblocks) of the tetrahedral numbering, one per grid position
        const uint64_t w = w0 + (uint64_t)blockIdx.y * gridDim.x + blockIdx.x;
        if (w >= nblocks) return;
        if constexpr (MAP == MAP_TET_TABLE) tet_block_table((uint32_t)w, m, L, R, C);
        else tet_block((uint32_t)w, L, R, C);
    } else {
        C = blockIdx.x;
        R = blockIdx.y;
        L = blockIdx.z;
        if (R > L || C > R) return;
    }
    // The block's pair quantities, once each: b(j, k) = |p_j - p_k|^2 for j in
    // block R and c(i, k) = |p_k - p_i|^2 for i in block L, k in block C, with
    // the same operations as the per-triplet form (so the same bits); rows
    // padded by two floats so that a warp's 8-byte loads of (k, k + 1) fall on
    // distinct banks.
    __shared__ __align__(8) float sb[32][34], sc[32][34];
    __shared__ double wsum[16];
    const uint32_t rho = blockDim.x, rows = blockDim.y;  // rows = rho / AT_ROWS
    const uint32_t tid = threadIdx.y * rho + threadIdx.x;
    const uint32_t kk = C * rho + threadIdx.x;
#pragma unroll
    for (int u = 0; u < AT_ROWS; ++u) {
        const uint32_t r = threadIdx.y + u * rows;
        const uint32_t jj = R * rho + r, ii = L * rho + r;
        float bv = 0.0f, cv = 0.0f;
        if (kk < n) {
            const float xk = p[3 * kk], yk = p[3 * kk + 1], zk = p[3 * kk + 2];
            if (jj < n) {
                const float ex = p[3 * jj] - xk, ey = p[3 * jj + 1] - yk, ez = p[3 * jj + 2] - zk;
                bv = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            }
            if (ii < n) {
                const float fx = xk - p[3 * ii], fy = yk - p[3 * ii + 1], fz = zk - p[3 * ii + 2];
                cv = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
            }
        }
        sb[r][threadIdx.x] = bv;
        sc[r][threadIdx.x] = cv;
    }
    __syncthreads();
    const uint32_t j = R * rho + threadIdx.x;
    float s = 0.0f;
    if (j < n) {
        const float xj = p[3 * j], yj = p[3 * j + 1], zj = p[3 * j + 2];
        // row u takes part iff j < i_u < n; a row that does not is computed
        // on a dummy side (a = 1) and left out of the sum
        bool act[AT_ROWS];
        f2 A[AT_ROWS], S[AT_ROWS];
        float a1[AT_ROWS];
        const float *crow[AT_ROWS];
#pragma unroll
        for (int u = 0; u < AT_ROWS; ++u) {
            const uint32_t r = threadIdx.y + u * rows, i = L * rho + r;
            act[u] = i < n && j < i;
            float a = 1.0f;
            if (act[u]) {
                const float dx = p[3 * i] - xj, dy = p[3 * i + 1] - yj, dz = p[3 * i + 2] - zj;
                a = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            }
            a1[u] = a;
            A[u] = f2_pack(a, a);
            S[u] = f2_pack(0.0f, 0.0f);
            crow[u] = sc[r];
        }
        const uint32_t kend = min(j, (C + 1) * rho) - C * rho;  // k < j
        const float *brow = sb[threadIdx.x];
        const f2 K = f2_pack(0.375f, 0.375f), ONE = f2_pack(1.0f, 1.0f), M2 = f2_pack(-2.0f, -2.0f);
        uint32_t t = 0;
        for (; t + 1 < kend; t += 2) {
            const f2 b = *reinterpret_cast<const f2 *>(&brow[t]);
#pragma unroll
            for (int u = 0; u < AT_ROWS; ++u) {
                const f2 c = *reinterpret_cast<const f2 *>(&crow[u][t]);
                const f2 q = f2_mul(f2_mul(A[u], b), c);
                // P = (b + c - a)(c + a - b)(a + b - c) = (s - 2a)(s - 2b)(s - 2c), s = a + b + c
                const f2 sum = f2_add(f2_add(A[u], b), c);
                const f2 P = f2_mul(f2_mul(f2_fma(M2, A[u], sum), f2_fma(M2, b, sum)), f2_fma(M2, c, sum));
                float q0, q1;
                f2_unpack(q, q0, q1);
                const f2 rs = f2_pack(rsqrtf(q0), rsqrtf(q1));
                const f2 inv = f2_mul(rs, rs);
                // term = (1 + 3 P / (8 q)) / q^(3/2), accumulated by one fused multiply-add
                S[u] = f2_fma(f2_mul(f2_fma(f2_mul(K, P), inv, ONE), inv), rs, S[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < AT_ROWS; ++u) {
            float s0, s1;
            f2_unpack(S[u], s0, s1);
            float su = s0 + s1;
            if (t < kend) {  // an odd last k
                const float a = a1[u], b = brow[t], c = crow[u][t];
                const float q = a * b * c;
                const float sum = a + b + c;
                const float P = fmaf(-2.0f, a, sum) * fmaf(-2.0f, b, sum) * fmaf(-2.0f, c, sum);
                const float rs = rsqrtf(q);
                const float inv = rs * rs;
                su = fmaf(fmaf(0.375f * P, inv, 1.0f) * inv, rs, su);
            }
            if (act[u]) s += su;
        }
    }
    // warp sums in FP32 (5 more roundings of at most 2^-24 of the magnitude
    // sum each; FP64 arithmetic is scarce on this part), warp totals in FP64
    float v = s;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const uint32_t nthreads = rho * rows, lane = tid & 31, warp = tid >> 5;
    if (lane == 0) wsum[warp] = (double)v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (uint32_t q = 0; q < (nthreads + 31) / 32; ++q) t += wsum[q];
        partial[T3(L) + T2(R) + C - w0] = nu * t;
    }
}

// Fixed-order sum of the partials: thread t adds a contiguous run, then
// thread 0 adds the run totals in order.
__global__ void at_reduce_kernel(const double *__restrict__ partial, uint64_t count, double *__restrict__ energy)
{
    __shared__ double part[1024];
    const uint32_t t = threadIdx.x, nt = blockDim.x;
    const uint64_t per = (count + nt - 1) / nt;
    const uint64_t b0 = min(count, (uint64_t)t * per), b1 = min(count, b0 + per);
    double s = 0.0;
    for (uint64_t q = b0; q < b1; ++q) s += partial[q];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        double e = 0.0;
        for (uint32_t q = 0; q < nt; ++q) e += part[q];
        *energy = e;
    }
}

}  // namespace

extern "C" int tet_at_workspace_size(uint32_t n, uint32_t rho, int map, size_t *bytes)
{
    if (!bytes || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_TET_TABLE && map != TRI_MAP_BB) return TRI_EINVAL;
    const uint64_t m = ((uint64_t)n + rho - 1) / rho;
    *bytes = (size_t)(T3(m) * sizeof(double));
    return TRI_OK;
}

// Launches the partial-sum kernel over blocks [w0, w1) of the tetrahedral
// numbering (all T3(m) blocks for the box) into `partial` (at least w1 - w0
// doubles, block w at w - w0) and the fixed-order reduction into *energy.
static int at_energy_launch(const float *xyz, uint32_t n, double nu, double *energy, int map, uint32_t rho,
                            uint64_t w0, uint64_t w1, double *partial, cudaStream_t s)
{
    const uint64_t m = ((uint64_t)n + rho - 1) / rho;
    const uint64_t nb = w1 - w0;
    const dim3 blk(rho, rho / AT_ROWS);
    if (map == TRI_MAP_LAMBDA || map == TRI_MAP_TET_TABLE) {
        if (w1 > 0xFFFFFFFFull) return TRI_ERANGE;
        if (nb > 0) {
            if (map == TRI_MAP_LAMBDA)
                at_kernel<MAP_LAMBDA><<<trihost::linear_grid(nb), blk, 0, s>>>(xyz, n, nu, (uint32_t)m, w0, w1,
                                                                                partial);
            else
                at_kernel<MAP_TET_TABLE><<<trihost::linear_grid(nb), blk, 0, s>>>(xyz, n, nu, (uint32_t)m, w0, w1,
                                                                                   partial);
        }
    } else {
        if (m > 65535) return TRI_ERANGE;
        at_kernel<MAP_BB><<<dim3((unsigned)m, (unsigned)m, (unsigned)m), blk, 0, s>>>(xyz, n, nu, (uint32_t)m, 0,
                                                                                        nb, partial);
    }
    if (cudaGetLastError() != cudaSuccess) return TRI_ECUDA;
    at_reduce_kernel<<<1, 1024, 0, s>>>(partial, nb, energy);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tet_at_energy(const float *xyz, uint32_t n, double nu, double *energy, int map, uint32_t rho,
                             void *workspace, size_t ws_bytes, void *stream)
{
    if (!xyz || !energy || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_TET_TABLE && map != TRI_MAP_BB) return TRI_EINVAL;
    size_t need = 0;
    tet_at_workspace_size(n, rho, map, &need);
    if (!workspace || ws_bytes < need || ((uintptr_t)workspace & 7)) return TRI_ENOSPACE;
    const uint64_t m = ((uint64_t)n + rho - 1) / rho;
    return at_energy_launch(xyz, n, nu, energy, map, rho, 0, T3(m), (double *)workspace, (cudaStream_t)stream);
}

// The tetrahedral block range of one of several GPUs: [floor(T k / ranks),
// floor(T (k + 1) / ranks)) of the T = T3(m) blocks, in lambda's numbering.
extern "C" int tet_at_partition(uint32_t n, uint32_t rho, uint32_t ranks, uint32_t rank, uint64_t *omega_begin,
                                uint64_t *omega_end)
{
    if (!omega_begin || !omega_end || ranks == 0 || rank >= ranks || !trihost::rho_ok(rho)) return TRI_EINVAL;
    const uint64_t m = ((uint64_t)n + rho - 1) / rho, T = T3(m);
    if (T > 0xFFFFFFFFull) return TRI_ERANGE;
    // floor(T k / ranks) without overflow: T = q ranks + r
    const uint64_t q = T / ranks, r = T % ranks;
    auto edge = [&](uint64_t k) { return q * k + r * k / ranks; };
    *omega_begin = edge(rank);
    *omega_end = edge(rank + 1);
    return TRI_OK;
}

extern "C" int tet_at_energy_range(const float *xyz, uint32_t n, double nu, double *energy, int map, uint32_t rho,
                                   uint64_t omega_begin, uint64_t omega_end, void *workspace, size_t ws_bytes,
                                   void *stream)
{
    if (!xyz || !energy || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_TET_TABLE) return TRI_EINVAL;
    const uint64_t m = ((uint64_t)n + rho - 1) / rho;
    if (omega_begin > omega_end || omega_end > T3(m)) return TRI_EINVAL;
    if (!workspace || ws_bytes < (omega_end - omega_begin) * sizeof(double) || ((uintptr_t)workspace & 7))
        return TRI_ENOSPACE;
    return at_energy_launch(xyz, n, nu, energy, map, rho, omega_begin, omega_end, (double *)workspace,
                            (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// tet_at_energy_noalloc: the same energy with no workspace argument.
//
// Some callers cannot call cudaMalloc when they need this energy: code whose
// device memory is all handed out by another allocator (a framework's caching
// pool or a fixed arena sized at start-up), and code that must not trigger the
// device-wide synchronisation that cudaMalloc and cudaFree can imply.  For
// them the block partials live in an array compiled into the library
// (AT_STATIC_PARTIALS doubles, 2 MiB), which every GPU that loads the library
// holds until the process exits.  The caller still owns the points and the
// result.
#include <mutex>

namespace {

constexpr size_t AT_STATIC_PARTIALS = size_t(1) << 18;  // 262,144 doubles = 2 MiB
static __device__ __align__(256) double g_at_partials[AT_STATIC_PARTIALS];

constexpr int AT_MAX_DEVICES = 64;
std::mutex g_at_mu;
double *g_at_ptr[AT_MAX_DEVICES] = {};

// Device address of g_at_partials on the current device, looked up once per
// device with that device current (host code cannot use the symbol itself).
int at_static_partials(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= AT_MAX_DEVICES) return TRI_ECUDA;
    std::lock_guard<std::mutex> lock(g_at_mu);
    if (!g_at_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_at_partials) != cudaSuccess || !p) return TRI_ECUDA;
        g_at_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_at_ptr[dev];
    return TRI_OK;
}

}  // namespace

extern "C" int tet_at_energy_noalloc(const float *xyz, uint32_t n, double nu, double *energy, int map, uint32_t rho,
                                     void *stream)
{
    if (!xyz || !energy || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_TET_TABLE && map != TRI_MAP_BB) return TRI_EINVAL;
    size_t need = 0;
    tet_at_workspace_size(n, rho, map, &need);
    if (need > sizeof(double) * AT_STATIC_PARTIALS) return TRI_ENOSPACE;  // more blocks than the array holds
    double *partial = nullptr;
    const int st = at_static_partials(&partial);
    if (st != TRI_OK) return st;
    // Every partial the reduction reads is written by this call's first
    // kernel, so nothing in the array needs clearing between calls.
    const uint64_t m = ((uint64_t)n + rho - 1) / rho;
    return at_energy_launch(xyz, n, nu, energy, map, rho, 0, T3(m), partial, (cudaStream_t)stream);
}
