// One block's tile of the FP32 direct-difference Euclidean distance map
// (Section 5, test 2): a (RHO R) x (RHO R) square of pairs d(i, j) with
// j <= i written to the packed lower triangle.  Shared by the single-triangle
// kernels (every block map) and the batched persistent kernel, each of which
// compiles its own copy.
#pragma once

#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "tri_maps.cuh"

namespace tri {
namespace tile {

constexpr int KC = 32;  // features staged per shared-memory pass

// Shared memory of a tile pass: the block's row points [k][r] (pitch S + 1,
// odd, so that the transposed writes of a warp hit distinct banks) and
// column points [k][c] (pitch S + 2, even, so that a thread's two adjacent
// columns load as one 8-byte word).  The pipelined form keeps two passes of
// KC features, one computed while the next is copied in; the plain form
// keeps one.  Both sit at the start of the kernel's dynamic shared memory, so
// that a kernel calling several tile variants holds one copy of the buffers.
template <int RHO, int R>
struct TileSmem {
    static constexpr int S = RHO * R;
    static constexpr int LI = S + 1, LJ = S + 2;
    static constexpr int PASS = KC * (LI + LJ);  // floats (even: the column part stays 8-byte aligned)
    // dynamic shared memory of a tile: one pass buffer, or two when pipelined
    static constexpr size_t bytes(bool pipe) { return sizeof(float) * (pipe ? 2 : 1) * PASS; }
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

// Which of a thread's (row u, column group v) accumulators a tile computes.
// Thread (ty, tx) owns rows ty + u RHO and columns 2 tx + 2 RHO v + {0, 1}.
//  - Rows u >= UA lie past the instance's last point: a tile of the last row
//    block computes only UA = ceil(rows left / RHO) row groups, for every
//    thread alike.
//  - On a diagonal tile (i0 = j0) a group with v > u / 2 starts at column
//    offset 2 RHO v >= RHO (u + 1), past the largest row offset of group u,
//    RHO - 1 + u RHO: every pair in it has j > i for every thread, so the
//    diagonal tile skips those groups (20 of 32 kept at R = 8, 6 of 8 at R = 4).
// Both tests are compile-time constants once the loops are unrolled.
template <int R, int UA, bool DIAG>
__device__ __forceinline__ constexpr bool tile_live(int u, int v)
{
    return u < UA && (!DIAG || v <= u / 2);
}

// Features [0, kc) of one staged pass added into the thread's live pairs.
template <int RHO, int R, int UA, bool DIAG>
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
                if (tile_live<R, UA, DIAG>(UA - 1, v))
                    b2[v] = *reinterpret_cast<const unsigned long long *>(sj + k * L::LJ + 2 * tx + 2 * RHO * v);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                if (!tile_live<R, UA, DIAG>(u, 0)) continue;
                const float a = si[k * L::LI + ty + u * RHO];
                const unsigned long long a2 = f2_pack(a, a);
#pragma unroll
                for (int v = 0; v < RC; ++v) {
                    if (!tile_live<R, UA, DIAG>(u, v)) continue;
                    const unsigned long long df = f2_sub(a2, b2[v]);
                    acc.a[u][v] = f2_fma(df, df, acc.a[u][v]);
                }
            }
        }
    }
}

// The square roots of the thread's live pairs with j <= i < n, to the packed rows.
template <int RHO, int R, int UA, bool DIAG>
__device__ __forceinline__ void tile_store(const TileAcc<R> &acc, float *__restrict__ out, uint32_t n, uint64_t i0,
                                           uint64_t j0, int tx, int ty)
{
#pragma unroll
    for (int u = 0; u < R; ++u) {
        if (!tile_live<R, UA, DIAG>(u, 0)) continue;
        const uint64_t i = i0 + ty + u * RHO;
        if (i >= n) continue;
        float *row = out + T2(i);
        if constexpr (R == 1) {
            const uint64_t j = j0 + tx;
            if (j <= i) row[j] = sqrtf(__uint_as_float((uint32_t)acc.a[0][0]));
        } else {
#pragma unroll
            for (int v = 0; v < TileAcc<R>::RC; ++v) {
                if (!tile_live<R, UA, DIAG>(u, v)) continue;
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
// stages with plain loads and stores into one pass buffer; PIPE = true
// copies the next pass in asynchronously while the current one is computed
// (two pass buffers) and ends without a block barrier: a caller that runs
// another tile in the same block synchronises the block first.  UA and DIAG
// select the live accumulators (tile_live); the caller guarantees that rows
// from i0 + UA RHO on are past n and, for DIAG, that i0 = j0.
template <int RHO, int R, bool PIPE, int UA = R, bool DIAG = false>
__device__ __forceinline__ void edm_tile_body(const float *__restrict__ x, uint32_t n, uint32_t d,
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
        float *si = tile_smem, *sj = si + KC * L::LI;
        for (uint32_t k0 = 0; k0 < d; k0 += KC) {
            const uint32_t kc = min((uint32_t)KC, d - k0);
            // stage x[i0 + r][k0 + k] and x[j0 + r][k0 + k], transposed to [k][r]
            for (uint32_t t = tid; t < (uint32_t)S * kc; t += RHO * RHO) {
                const uint32_t r = t / kc, k = t - r * kc;
                const uint64_t gi = i0 + r, gj = j0 + r;
                si[k * L::LI + r] = gi < n ? x[gi * d + k0 + k] : 0.0f;
                sj[k * L::LJ + r] = gj < n ? x[gj * d + k0 + k] : 0.0f;
            }
            __syncthreads();
            tile_pass<RHO, R, UA, DIAG>(si, sj, kc, tx, ty, acc);
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
            tile_pass<RHO, R, UA, DIAG>(si, si + KC * L::LI, min((uint32_t)KC, d - c * KC), tx, ty, acc);
            if (c + 2 < passes) __syncthreads();  // this buffer is refilled for pass c + 2
        }
    }
    tile_store<RHO, R, UA, DIAG>(acc, out, n, i0, j0, tx, ty);
}

// The tile as a function of its own: every block map calls the same compiled
// body, so the maps differ only in how a block finds its (bi, bj).
template <int RHO, int R, bool PIPE>
__device__ __noinline__ void edm_tile(const float *__restrict__ x, uint32_t n, uint32_t d,
                                      float *__restrict__ out, uint32_t bi, uint32_t bj)
{
    edm_tile_body<RHO, R, PIPE>(x, n, d, out, bi, bj);
}

}  // namespace tile
}  // namespace tri
