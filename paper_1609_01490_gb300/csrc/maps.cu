// tri_map_launch, tri_lambda_verify, tet_map: the maps on their own
// (Section 4.1's dummy kernel and coverage/exactness checks of every map).
#include <cuda_runtime.h>

#include "tri_maps.cuh"
#include "tet_table.cuh"

using namespace tri;

namespace {

// One mapped element (i, j) of the triangle; `strict` selects the index of the
// strict triangle i(i-1)/2 + j.
template <int BODY>
__device__ __forceinline__ void body2(uint32_t i, uint32_t j, int strict, uint32_t *out)
{
    if constexpr (BODY == TRI_BODY_DUMMY) {
        *(volatile uint32_t *)out = i + j;
    } else if constexpr (BODY == TRI_BODY_SENTINEL) {
        if (i + j == 0xFFFFFFFFu) *(volatile uint32_t *)out = i + j;
    } else {
        const uint64_t idx = strict ? T2((uint64_t)i - 1) + j : T2(i) + j;
        atomicAdd(out + idx, 1u);
    }
}

// Block maps: block (bi, bj) of the with-diagonal triangle of block rows,
// thread (ty, tx) -> row r = bi*rho + ty, column j = bj*rho + tx, r >= j.  The
// strict domain j < i < n is the with-diagonal one of n-1 rows shifted down
// by one: element row i = r + strict.
template <int MAP, int SQ, int BODY>
__global__ void map_kernel(BlockMap bm, uint32_t n, int strict, uint32_t *out)
{
    uint32_t bi, bj;
    if (!map_block<MAP, SQ>(bm, bi, bj)) return;
    const uint32_t r = bi * blockDim.y + threadIdx.y;
    const uint32_t j = bj * blockDim.x + threadIdx.x;
    const uint32_t i = r + strict;
    if (i >= n || j > r) return;
    body2<BODY>(i, j, strict, out);
}

// UTM: thread k -> (a, b) over N items, then (i, j) = (b-2, a-1) for the
// with-diagonal domain (N = n+1) or (b-1, a-1) for the strict one (N = n).
template <int BODY>
__global__ void utm_kernel(uint64_t total, uint64_t N, int strict, uint32_t *out)
{
    const uint64_t k = ((uint64_t)blockIdx.y * gridDim.x + blockIdx.x) * (blockDim.x * blockDim.y) +
                       threadIdx.y * blockDim.x + threadIdx.x;
    if (k >= total) return;
    uint32_t a, b;
    utm_pair(k, N, a, b);
    const uint32_t i = strict ? b - 1 : b - 2, j = a - 1;
    body2<BODY>(i, j, strict, out);
}

template <int MAP, int BODY>
cudaError_t launch_map_sq(int sq, dim3 g, dim3 blk, cudaStream_t s, BlockMap bm, uint32_t n, int strict,
                          uint32_t *out)
{
    switch (sq) {
    case TRI_SQRT_X: map_kernel<MAP, TRI_SQRT_X, BODY><<<g, blk, 0, s>>>(bm, n, strict, out); break;
    case TRI_SQRT_R: map_kernel<MAP, TRI_SQRT_R, BODY><<<g, blk, 0, s>>>(bm, n, strict, out); break;
    default: map_kernel<MAP, TRI_SQRT_N, BODY><<<g, blk, 0, s>>>(bm, n, strict, out); break;
    }
    return cudaGetLastError();
}

template <int BODY>
int map_launch_body(int map, int sq, uint32_t n, uint32_t rho, int with_diag, uint32_t *out, cudaStream_t s)
{
    const int strict = with_diag ? 0 : 1;
    const uint64_t ne = (uint64_t)n - strict;  // rows of the with-diagonal domain
    if (ne == 0) return TRI_OK;                // strict domain of one element is empty
    const uint32_t m = (uint32_t)((ne + rho - 1) / rho);
    const dim3 blk(rho, rho);
    BlockMap bm{};
    bm.m = m;
    bm.nblocks = T2(m);
    cudaError_t e = cudaSuccess;
    switch (map) {
    case TRI_MAP_LAMBDA:
    case TRI_MAP_LAMBDA_PDELTA: {
        if (bm.nblocks > 0xFFFFFFFFull) return TRI_ERANGE;
        dim3 g;
        if (map == TRI_MAP_LAMBDA) {
            g = trihost::linear_grid(bm.nblocks);
        } else {
            const uint64_t mp = trihost::isqrt_ceil(bm.nblocks);
            if (mp > 65535) return TRI_ERANGE;
            g = dim3((unsigned)mp, (unsigned)mp);
        }
        if (strict)
            e = launch_map_sq<MAP_LAMBDA_ND, BODY>(sq, g, blk, s, bm, n, strict, out);
        else if (map == TRI_MAP_LAMBDA)
            e = launch_map_sq<MAP_LAMBDA, BODY>(sq, g, blk, s, bm, n, strict, out);
        else
            e = launch_map_sq<MAP_LAMBDA_PD, BODY>(sq, g, blk, s, bm, n, strict, out);
        break;
    }
    case TRI_MAP_BB:
        if (m > 65535) return TRI_ERANGE;
        map_kernel<MAP_BB, TRI_SQRT_R, BODY><<<dim3(m, m), blk, 0, s>>>(bm, n, strict, out);
        e = cudaGetLastError();
        break;
    case TRI_MAP_RB: {
        const uint32_t h = (m & 1u) ? (m + 1) / 2 : m / 2 + 1;
        if (h > 65535) return TRI_ERANGE;
        map_kernel<MAP_RB, TRI_SQRT_R, BODY><<<dim3(m, h), blk, 0, s>>>(bm, n, strict, out);
        e = cudaGetLastError();
        break;
    }
    case TRI_MAP_REC: {
        if (!trihost::is_pow2(m)) return TRI_ERANGE;
        const uint32_t k = trihost::ilog2(m);
        if (m / 2 > 65535 && k > 0) return TRI_ERANGE;
        for (uint32_t l = 0; l <= k && e == cudaSuccess; ++l) {
            bm.level = l;
            const dim3 g = l == 0 ? dim3(m) : dim3(1u << (l - 1), m / 2);
            map_kernel<MAP_REC, TRI_SQRT_R, BODY><<<g, blk, 0, s>>>(bm, n, strict, out);
            e = cudaGetLastError();
        }
        break;
    }
    case TRI_MAP_UTM: {
        const uint64_t N = strict ? n : (uint64_t)n + 1;
        const uint64_t total = N * (N - 1) / 2;
        const uint64_t tpb = (uint64_t)rho * rho;
        const uint64_t nb = (total + tpb - 1) / tpb;
        if (total > 0xFFFFFFFFull) return TRI_ERANGE;
        utm_kernel<BODY><<<trihost::linear_grid(nb), blk, 0, s>>>(total, N, strict, out);
        e = cudaGetLastError();
        break;
    }
    default:
        return TRI_EINVAL;
    }
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

// Exhaustive check of lambda: one thread per omega.
template <int SQ, int STRICT>
__global__ void lambda_verify_kernel(uint64_t w0, uint64_t w1, unsigned long long *res)
{
    const uint64_t w = w0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long bad = 0, si = 0, sj = 0, sii = 0, sjj = 0, sij = 0;
    if (w < w1) {
        uint32_t i, j;
        bool ok;
        if constexpr (STRICT) {
            lambda_nodiag<SQ>((uint32_t)w, i, j);
            ok = i >= 1 && j < i && T2((uint64_t)i - 1) <= w && w < T2(i) && T2((uint64_t)i - 1) + j == w;
        } else {
            lambda_diag<SQ>((uint32_t)w, i, j);
            ok = j <= i && T2(i) <= w && w < T2((uint64_t)i + 1) && T2(i) + j == w;
        }
        bad = ok ? 0 : 1;
        si = i;
        sj = j;
        sii = (unsigned long long)i * i;
        sjj = (unsigned long long)j * j;
        sij = (unsigned long long)i * j;
    }
    // warp sums, one atomic per warp and quantity
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_down_sync(0xffffffffu, bad, o);
        si += __shfl_down_sync(0xffffffffu, si, o);
        sj += __shfl_down_sync(0xffffffffu, sj, o);
        sii += __shfl_down_sync(0xffffffffu, sii, o);
        sjj += __shfl_down_sync(0xffffffffu, sjj, o);
        sij += __shfl_down_sync(0xffffffffu, sij, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(res + 0, bad);
        atomicAdd(res + 1, si);
        atomicAdd(res + 2, sj);
        atomicAdd(res + 3, sii);
        atomicAdd(res + 4, sjj);
        atomicAdd(res + 5, sij);
    }
}

// Tetrahedral blocks: block omega -> (L, R, C), L >= R >= C, by the closed
// form (MAP_LAMBDA) or the layer table (MAP_TET_TABLE), or the m^3 box
// (MAP_BB, blocks outside the tetrahedron leave at once); thread (ty, tx)
// takes i in block L, j in block R, and loops k over block C.
template <int MAP, int BODY>
__global__ void tet_kernel(uint64_t nblocks, uint32_t m, uint32_t n, uint32_t *out)
{
    uint32_t L, R, C;
    if constexpr (MAP == MAP_BB) {
        C = blockIdx.x;
        R = blockIdx.y;
        L = blockIdx.z;
        if (R > L || C > R) return;
    } else {
        const uint64_t w = (uint64_t)blockIdx.y * gridDim.x + blockIdx.x;
        if (w >= nblocks) return;
        if constexpr (MAP == MAP_TET_TABLE) tet_block_table((uint32_t)w, m, L, R, C);
        else tet_block((uint32_t)w, L, R, C);
    }
    const uint32_t rho = blockDim.x;
    const uint32_t i = L * rho + threadIdx.y, j = R * rho + threadIdx.x;
    if (i >= n || j >= i) return;
    const uint32_t kend = min(j, (C + 1) * rho);
    for (uint32_t k = C * rho; k < kend; ++k) {
        if constexpr (BODY == TRI_BODY_DUMMY) {
            *(volatile uint32_t *)out = i + j + k;
        } else if constexpr (BODY == TRI_BODY_SENTINEL) {
            if (i + j + k == 0xFFFFFFFFu) *(volatile uint32_t *)out = i + j + k;
        } else {
            const uint64_t I = i, J = j;
            const uint64_t idx = I * (I - 1) * (I - 2) / 6 + J * (J - 1) / 2 + k;
            atomicAdd(out + idx, 1u);
        }
    }
}

// ------------------------------------------------ the printed formulas ----
// Section 4.1 as printed: the row of omega is the FP32 estimate of
// sqrt(2 omega + 1/4) - 1/2 (plus eps = 1e-4 for lambda_N and lambda_R),
// floored, with no integer correction.
template <int SQ>
__device__ __forceinline__ uint32_t lambda_row_printed(uint32_t w)
{
    const float eps = SQ == TRI_SQRT_X ? 0.0f : 1e-4f;
    const float est = sqrt_estimate<SQ>(fmaf(2.0f, (float)w, 0.25f)) + eps - 0.5f;
    return __float2uint_rz(est);
}

// Section 4.2 as printed (Avril et al.): thread k of n items,
// a = floor((-(2n + 1) + sqrt(4n^2 - 4n - 8k + 1)) / -2), b = (a + 1) + k -
// (a - 1)(2n - a)/2, with the square root's argument and a in FP32.
__device__ __forceinline__ void utm_pair_printed(uint64_t k, uint64_t n, uint64_t &a, uint64_t &b)
{
    const float fn = (float)n, fk = (float)k;
    const float disc = 4.0f * fn * fn - 4.0f * fn - 8.0f * fk + 1.0f;
    const float af = floorf((-(2.0f * fn + 1.0f) + sqrtf(disc)) / -2.0f);
    const long long ai = af < 0.0f ? 0 : (long long)af;
    a = (uint64_t)ai;
    b = (uint64_t)((long long)a + 1 + (long long)k - ((long long)a - 1) * (2 * (long long)n - (long long)a) / 2);
}

// Lowers *first_bad to the smallest index in [i0, i1) where the printed
// formula disagrees with the exact map (one index per thread).
template <int MAPK, int SQ>
__global__ void first_error_kernel(uint64_t n_items, uint64_t i0, uint64_t i1, unsigned long long *first_bad)
{
    const uint64_t x = i0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (x < i1) {
        if constexpr (MAPK == MAP_UTM) {
            uint32_t ea, eb;
            utm_pair(x, n_items, ea, eb);
            uint64_t a, b;
            utm_pair_printed(x, n_items, a, b);
            bad = a != ea || b != eb;
        } else {
            uint32_t ei, ej;
            lambda_diag<TRI_SQRT_R>((uint32_t)x, ei, ej);
            bad = lambda_row_printed<SQ>((uint32_t)x) != ei;
        }
    }
    const unsigned any = __ballot_sync(0xffffffffu, bad);
    if (any && (threadIdx.x & 31) == (unsigned)(__ffs(any) - 1)) atomicMin(first_bad, (unsigned long long)x);
}

}  // namespace

extern "C" int tri_map_first_error(int map, int sqrt_kind, uint64_t n_items, uint64_t begin, uint64_t end,
                                   unsigned long long *first_bad, void *stream)
{
    if (!first_bad || begin > end) return TRI_EINVAL;
    if (sqrt_kind < TRI_SQRT_X || sqrt_kind > TRI_SQRT_N) return TRI_EINVAL;
    if (map == TRI_MAP_LAMBDA) {
        if (end > (1ull << 32)) return TRI_ERANGE;
    } else if (map == TRI_MAP_UTM) {
        if (n_items < 2 || n_items > (1ull << 31) || end > n_items * (n_items - 1) / 2) return TRI_ERANGE;
    } else {
        return TRI_EINVAL;
    }
    if (begin == end) return TRI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned tpb = 256;
    const dim3 g = trihost::linear_grid((end - begin + tpb - 1) / tpb);
    if (g.y > 1) return TRI_ERANGE;  // one launch covers at most 2^31 - 1 blocks of 256
    if (map == TRI_MAP_UTM) {
        first_error_kernel<MAP_UTM, TRI_SQRT_X><<<g, tpb, 0, s>>>(n_items, begin, end, first_bad);
    } else if (sqrt_kind == TRI_SQRT_X) {
        first_error_kernel<MAP_LAMBDA, TRI_SQRT_X><<<g, tpb, 0, s>>>(n_items, begin, end, first_bad);
    } else if (sqrt_kind == TRI_SQRT_R) {
        first_error_kernel<MAP_LAMBDA, TRI_SQRT_R><<<g, tpb, 0, s>>>(n_items, begin, end, first_bad);
    } else {
        first_error_kernel<MAP_LAMBDA, TRI_SQRT_N><<<g, tpb, 0, s>>>(n_items, begin, end, first_bad);
    }
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tri_map_launch(int map, int sqrt_kind, uint32_t n, uint32_t rho, int with_diag, int body,
                              uint32_t *out, void *stream)
{
    if (!out || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (sqrt_kind < TRI_SQRT_X || sqrt_kind > TRI_SQRT_N) return TRI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    switch (body) {
    case TRI_BODY_DUMMY: return map_launch_body<TRI_BODY_DUMMY>(map, sqrt_kind, n, rho, with_diag, out, s);
    case TRI_BODY_SENTINEL:
        return map_launch_body<TRI_BODY_SENTINEL>(map, sqrt_kind, n, rho, with_diag, out, s);
    case TRI_BODY_COUNT: return map_launch_body<TRI_BODY_COUNT>(map, sqrt_kind, n, rho, with_diag, out, s);
    default: return TRI_EINVAL;
    }
}

extern "C" int tri_lambda_verify(int sqrt_kind, int with_diag, uint64_t w_begin, uint64_t w_end,
                                 unsigned long long *result, void *stream)
{
    if (!result) return TRI_EINVAL;
    if (sqrt_kind < TRI_SQRT_X || sqrt_kind > TRI_SQRT_N) return TRI_EINVAL;
    if (w_end > (1ull << 32) || w_begin > w_end) return TRI_ERANGE;
    if (w_begin == w_end) return TRI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t cnt = w_end - w_begin;
    const unsigned tpb = 256;
    const dim3 g((unsigned)((cnt + tpb - 1) / tpb));
#define TRI_LV(SQ, ST) lambda_verify_kernel<SQ, ST><<<g, tpb, 0, s>>>(w_begin, w_end, result)
    if (with_diag) {
        if (sqrt_kind == TRI_SQRT_X) TRI_LV(TRI_SQRT_X, 0);
        else if (sqrt_kind == TRI_SQRT_R) TRI_LV(TRI_SQRT_R, 0);
        else TRI_LV(TRI_SQRT_N, 0);
    } else {
        if (sqrt_kind == TRI_SQRT_X) TRI_LV(TRI_SQRT_X, 1);
        else if (sqrt_kind == TRI_SQRT_R) TRI_LV(TRI_SQRT_R, 1);
        else TRI_LV(TRI_SQRT_N, 1);
    }
#undef TRI_LV
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tet_map_ex(int map, uint32_t n, uint32_t rho, int body, uint32_t *out, void *stream)
{
    if (!out || n == 0 || !trihost::rho_ok(rho)) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_TET_TABLE && map != TRI_MAP_BB) return TRI_EINVAL;
    if (body != TRI_BODY_DUMMY && body != TRI_BODY_SENTINEL && body != TRI_BODY_COUNT) return TRI_EINVAL;
    if (n < 3) return TRI_OK;
    const uint64_t m = (n + rho - 1) / rho;
    const uint64_t nb = T3(m);
    if (nb > 0xFFFFFFFFull) return TRI_ERANGE;
    if (map == TRI_MAP_BB && m > 65535) return TRI_ERANGE;
    cudaStream_t s = (cudaStream_t)stream;
    const dim3 g = map == TRI_MAP_BB ? dim3((unsigned)m, (unsigned)m, (unsigned)m) : trihost::linear_grid(nb);
    const dim3 blk(rho, rho);
#define TRI_T(MP, BD) tet_kernel<MP, BD><<<g, blk, 0, s>>>(nb, (uint32_t)m, n, out)
#define TRI_TB(MP)                                                                                             \
    if (body == TRI_BODY_DUMMY) TRI_T(MP, TRI_BODY_DUMMY);                                                     \
    else if (body == TRI_BODY_SENTINEL) TRI_T(MP, TRI_BODY_SENTINEL);                                          \
    else TRI_T(MP, TRI_BODY_COUNT);
    if (map == TRI_MAP_LAMBDA) {
        TRI_TB(MAP_LAMBDA)
    } else if (map == TRI_MAP_TET_TABLE) {
        TRI_TB(MAP_TET_TABLE)
    } else {
        TRI_TB(MAP_BB)
    }
#undef TRI_TB
#undef TRI_T
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tet_map(uint32_t n, uint32_t rho, int body, uint32_t *out, void *stream)
{
    return tet_map_ex(TRI_MAP_LAMBDA, n, rho, body, out, stream);
}
