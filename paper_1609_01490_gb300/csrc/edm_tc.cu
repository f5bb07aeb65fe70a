// Euclidean distance matrix on tcgen05 tensor cores (not in the paper, which
// evaluates distances directly): d_ij^2 = |x_i|^2 + |x_j|^2 - 2 x_i.x_j with the
// Gram term x_i.x_j from BF16 products accumulated in FP32 in tensor memory.
//
// Precision.  Each FP32 input is split into BF16 planes, x = hi + lo (+ mid):
//   hi = bf16(x), r = x - hi (exact), mid = bf16(r), lo = bf16(r - mid).
// Three planes represent x exactly (3 x 8 significant bits = FP32's 24);
// the Gram term keeps the products hi.hi', hi.mid', mid.hi', hi.lo', lo.hi',
// mid.mid' (BF16X6) and drops those below 2^-24 |x||y|; the two-plane form
// (BF16X3) keeps hi.hi', hi.lo', lo.hi'.  Every BF16 x BF16 product is exact
// in FP32.  A pair whose estimate falls below tau (|x_i|^2 + |x_j|^2) has lost
// too many digits to cancellation and is flagged; a second kernel recomputes
// flagged pairs in FP64 by direct differences (the paper's definition).
//
// Kernels.  prepare: FP64 row norms (stored as FP32) and the BF16 planes,
// K padded to a multiple of 64.  gram: persistent, one CTA per SM, 128 x 128
// pair tiles taken in lambda order (Eq. eq_gmap): first one contiguous run of
// tile numbers per CTA, then short runs taken from a global counter by
// whichever CTA is free (SMs do not all store at the same rate), so
// consecutive tiles mostly share their row block and the CTA keeps that row
// block's planes (A) resident in shared memory while TMA streams the column
// blocks (B) through a ring of 16 KB stages, one plane of one 64-wide K chunk each.
// Warp 0 takes the tiles and passes them to the other roles through a small
// queue in shared memory, and issues TMA,
// warp 1 issues tcgen05.mma into a double-buffered TMEM accumulator (with the
// column block as the M operand, so TMEM lanes are output columns), warps
// 2-17 read TMEM back, form the distances, flag cancellations and store the
// packed row segments (P = 2: whole segments through shared memory; P = 3:
// one coalesced 128-byte store per warp and row).  fixup: FP64
// recompute of the flagged pairs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "tri_internal.h"
#include "tri_maps.cuh"

using namespace tri;

namespace {

constexpr int TILE = 128;                  // pair tile side (UMMA M = N = 128)
constexpr int KCH = 64;                    // K per chunk: one 128-byte swizzle row of BF16
constexpr int CHUNK_BYTES = TILE * KCH * 2;  // 16 KB: 128 rows x 64 BF16
constexpr int NEPI = 16;                   // epilogue warps: 4 TMEM lane quarters x 4 row groups
constexpr int NTHREADS = 64 + 32 * NEPI;   // TMA warp, MMA warp, epilogue warps
constexpr int EPI_ROWS = 16;               // output rows per TMEM load in the epilogue
constexpr int NORM_FLOATS = 2 * 32;       // per epilogue warp: norms of its 32 rows of the tile (double buffered)
constexpr int STG_ROWS = 8;                // rows staged at a time by a row group
constexpr int STG_LD = TILE + 4;           // staging row: 128 distances shifted by the row's 16-byte phase
constexpr int STG_FLOATS = STG_ROWS * STG_LD;  // one staging buffer
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // a bounded wait gives up after 2 s
constexpr int TQ = 8;                      // tile queue slots (producer -> MMA and epilogue)
constexpr unsigned long long TQ_END = ~0ull;  // queue entry after the last tile
constexpr uint32_t STATIC_PCT = 80;        // share of the tiles assigned up front, in contiguous runs
constexpr uint32_t DYN_CHUNK = 8;          // tiles per grab from the global counter afterwards
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int MAX_STAGES = 12;             // B ring depth cap (16 KB stages)

constexpr float TAU_X6 = 0.3125f;  // flag threshold for hi/mid/lo (derived bound)
constexpr float TAU_X3 = 0.0625f;  // flag threshold for hi/lo (empirical)

struct WsLayout {
    size_t hdr, norms, planes, flags, total;
    unsigned long long cap;
};

// Workspace: [header 256 B: flag counter (u64 at 0), status (int at 8), tile
// counter (u64 at 16)][norms n FP32][planes
// P x n x dp BF16][flag list cap x u64], each part 256-byte aligned.
WsLayout ws_layout(uint32_t n, uint32_t d, int prec)
{
    const int P = prec == TRI_BF16X6 ? 3 : 2;
    const size_t dp = ((size_t)d + KCH - 1) / KCH * KCH;
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    WsLayout L;
    L.hdr = 0;
    L.norms = 256;
    L.planes = al(L.norms + sizeof(float) * n);
    L.cap = (unsigned long long)std::max<size_t>(1u << 20, 4 * (size_t)n);
    L.flags = al(L.planes + (size_t)P * n * dp * 2);
    L.total = al(L.flags + L.cap * sizeof(unsigned long long));
    return L;
}

// --------------------------------------------------------------- PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete.  Gives up after
// WAIT_LIMIT_NS, or early when another role has already given up (unless
// abort_flag is null: the drain waits at exit must not cut short a copy or
// MMA that is still writing).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t start = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 15) == 0) {
            if (abort_flag && *abort_flag) return false;
            if (global_ns() - start > WAIT_LIMIT_NS) return false;
            __nanosleep(64);
        }
    }
}

// mbar_wait by lane 0 with the result broadcast, so the whole warp leaves
// together and agrees on it.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    int r = 0;
    if ((threadIdx.x & 31) == 0) r = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
    return __shfl_sync(0xffffffffu, r, 0) != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y,
                                            int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 128 (bits 17-22 hold N/8), M = 128 (bits 24-28 hold M/16).
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TILE >> 3) << 17) |
                           ((uint32_t)(TILE >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 TMEM lanes x 16 columns: thread t receives lane (base + t), 16 columns.
// The load is asynchronous: tmem_wait16 must run before the registers are read.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Completes the outstanding TMEM loads.  The registers pass through the asm
// as read-write operands, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])::"memory");
}

// ------------------------------------------------------------ prepare ----
// One warp per row: FP64 norm (rounded to FP32) and the BF16 planes.
template <int P>
__global__ void prepare_kernel(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t dp,
                               float *__restrict__ norms, __nv_bfloat16 *__restrict__ planes)
{
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float *row = x + (size_t)warp * d;
    double s = 0.0;
    for (uint32_t k = lane; k < dp; k += 32) {
        const float v = k < d ? row[k] : 0.0f;
        s += (double)v * (double)v;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(hi);
        const size_t o = (size_t)warp * dp + k;
        planes[o] = hi;
        if constexpr (P == 2) {
            planes[(size_t)n * dp + o] = __float2bfloat16_rn(r1);
        } else {
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(mid);
            planes[(size_t)n * dp + o] = mid;
            planes[2 * (size_t)n * dp + o] = __float2bfloat16_rn(r2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) norms[warp] = (float)s;
}

// --------------------------------------------------------------- gram ----
struct GramArgs {
    uint32_t n, nkc;           // points, 64-wide K chunks
    uint32_t m;                // tile rows of the triangle
    uint64_t ntiles;           // tile numbers walked: m(m+1)/2 (lambda) or m*m (BB)
    uint64_t static_per;       // tile numbers per CTA in its up-front run
    uint64_t dyn_start;        // first tile number handed out by the counter
    uint32_t chunk;            // tile numbers per grab from the counter
    uint32_t stages;           // B ring depth
    float tau;
    const float *norms;
    float *out;
    unsigned long long *flag_count, *flag_list, flag_cap;
    unsigned long long *tile_counter;  // zero at launch
    int *status;
};

template <int MAP>
__device__ __forceinline__ bool tile_of(uint64_t t, uint32_t m, uint32_t &bi, uint32_t &bj)
{
    if constexpr (MAP == MAP_LAMBDA) {
        lambda_diag<TRI_SQRT_R>((uint32_t)t, bi, bj);
        return true;
    } else {
        bi = (uint32_t)(t / m);
        bj = (uint32_t)(t - (uint64_t)bi * m);
        return bj <= bi;  // bounding box: tiles above the diagonal are skipped
    }
}

// The split keeps the products of row plane pa and column plane pb with
// pa + pb <= P - 1: hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid for P = 3
// and hi.hi, hi.lo, lo.hi for P = 2.

// Offset of packed row i0 + k within 16 bytes, T2(i0 + k) mod 4, for i0 a
// multiple of 16 (then it equals T2(k) mod 4).
__host__ __device__ constexpr uint32_t row_phase(uint32_t k) { return ((k * (k + 1)) >> 1) & 3u; }

// Barrier among the `count` threads of one epilogue row group (ids 1..).
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// 1/sqrt by the MUFU unit (flush-to-zero approximation; relative error a few
// 2^-23, far inside the 1e-5 the distances are held to).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Shared-memory matrix descriptor of a K-major operand with 128-byte swizzle:
// start address (bits 0-13) and leading byte offset (bits 16-29, unused for
// swizzled K-major) in 16-byte units form the low word; the high word holds
// the stride byte offset (8 rows x 128 B = 1024 B between 8-row groups), the
// descriptor version for tcgen05 and the swizzle mode, all constant here.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t addr) { return (addr >> 4) | (1u << 16); }
constexpr uint32_t kDescHi = (1024u >> 4) | (1u << 14) | (2u << 29);  // SBO, version, 128-byte swizzle


template <int MAP, int P>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_kernel(const __grid_constant__ CUtensorMap tmap, const GramArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand area
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t a_bytes = (uint32_t)P * g.nkc * CHUNK_BYTES;
    constexpr uint32_t stage_bytes = CHUNK_BYTES;            // one plane of one K chunk
    constexpr uint32_t stg_floats = P == 2 ? (NEPI / 4) * 2 * STG_FLOATS : 0;  // two staging buffers per row group
    const uint32_t sA = base;                                  // [kc][p] chunks
    const uint32_t sB = base + a_bytes;                        // [stage] chunks of one plane
    float *epi = reinterpret_cast<float *>(gbase + a_bytes + g.stages * stage_bytes);
    float *stage_base = epi + NEPI * NORM_FLOATS;  // one staging area per row group
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage_base + stg_floats);
    // barriers: fullA, freeA, done, tmem_full[2], tmem_empty[2], fullB[stages], emptyB[stages]
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t b_fullA = bar0, b_freeA = bar0 + 8, b_done = bar0 + 16;
    const uint32_t b_tfull = bar0 + 24, b_tempty = bar0 + 40;
    const uint32_t b_fullB = bar0 + 56, b_emptyB = bar0 + 56 + 8 * g.stages;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    // tile queue: entry (bi << 32 | bj), or TQ_END; full: one arrival by the
    // producer, empty: one by the MMA thread and one per epilogue warp
    __shared__ volatile unsigned long long s_tq[TQ];
    __shared__ __align__(8) uint64_t s_tqbar[2 * TQ];
    const uint32_t b_tqfull = smem_u32(s_tqbar), b_tqempty = b_tqfull + 8 * TQ;

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(b_fullA, 1);
        mbar_init(b_freeA, 1);
        mbar_init(b_done, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_tfull + 8 * i, 1);
            mbar_init(b_tempty + 8 * i, NEPI);  // one arrival per epilogue warp
        }
        for (uint32_t s = 0; s < g.stages; ++s) {
            mbar_init(b_fullB + 8 * s, 1);
            mbar_init(b_emptyB + 8 * s, 1);
        }
        for (int s = 0; s < TQ; ++s) {
            mbar_init(b_tqfull + 8 * s, 1);
            mbar_init(b_tqempty + 8 * s, 1 + NEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // Queue entry k sits in slot k % TQ; its fill is phase k / TQ of the slot's barriers.
    auto tq_push = [&](uint32_t k, unsigned long long v) {
        const uint32_t slot = k % TQ;
        if (!mbar_wait(b_tqempty + 8 * slot, ((k / TQ) & 1) ^ 1, &s_abort)) return false;
        s_tq[slot] = v;
        mbar_arrive(b_tqfull + 8 * slot);
        return true;
    };
    // by one thread (the MMA issuer)
    auto tq_pop = [&](uint32_t k, unsigned long long &v) {
        const uint32_t slot = k % TQ;
        if (!mbar_wait(b_tqfull + 8 * slot, (k / TQ) & 1, &s_abort)) return false;
        v = s_tq[slot];
        mbar_arrive(b_tqempty + 8 * slot);
        return true;
    };
    // by a whole epilogue warp: lane 0 waits, reads and releases the slot, then
    // broadcasts the entry
    auto tq_pop_warp = [&](uint32_t k, unsigned long long &v) {
        unsigned long long r = 0;
        int ok = 0;
        if ((threadIdx.x & 31) == 0) {
            const uint32_t slot = k % TQ;
            ok = mbar_wait(b_tqfull + 8 * slot, (k / TQ) & 1, &s_abort) ? 1 : 0;
            if (ok) {
                r = s_tq[slot];
                mbar_arrive(b_tqempty + 8 * slot);
            }
        }
        v = __shfl_sync(0xffffffffu, r, 0);
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    // The TMA and MMA roles run on lane 0 of their warps.  Between two MMAs
    // the issuing thread does nothing but add descriptor offsets: a
    // 128x128x16 MMA takes about 68 cycles, and any longer gap in the issue
    // stream leaves the tensor pipe idle.  Each stage holds one plane of one
    // 64-wide K chunk of the column block: the MMA thread waits once per
    // 4 (P - pb) MMAs for column plane pb.
    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap) : "memory");
            uint32_t a_row = 0xFFFFFFFFu, a_loads = 0, stage = 0, b_phase = 0, loads = 0, k = 0;
            bool ok = true;
            // this CTA's up-front run of tile numbers, then runs from the counter
            uint64_t t = (uint64_t)blockIdx.x * g.static_per, tend = t + g.static_per;
            while (ok) {
                if (t >= tend) {
                    t = g.dyn_start + atomicAdd(g.tile_counter, (unsigned long long)g.chunk);
                    if (t >= g.ntiles) break;
                    tend = t + g.chunk < g.ntiles ? t + g.chunk : g.ntiles;
                }
                uint32_t bi, bj;
                if (!tile_of<MAP>(t++, g.m, bi, bj)) continue;
                if (!tq_push(k++, ((unsigned long long)bi << 32) | bj)) {
                    ok = false;
                    break;
                }
                if (bi != a_row) {
                    if (a_loads > 0 && !mbar_wait(b_freeA, (a_loads - 1) & 1, &s_abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(b_fullA, a_bytes);
                    for (uint32_t kc = 0; kc < g.nkc; ++kc)
                        for (int p = 0; p < P; ++p)
                            tma_load_3d(sA + (kc * P + p) * CHUNK_BYTES, &tmap, b_fullA, kc * KCH, bi * TILE, p);
                    ++a_loads;
                    a_row = bi;
                }
                for (uint32_t kc = 0; kc < g.nkc && ok; ++kc) {
                    for (int p = 0; p < P; ++p) {
                        if (!mbar_wait(b_emptyB + 8 * stage, b_phase ^ 1, &s_abort)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(b_fullB + 8 * stage, stage_bytes);
                        tma_load_3d(sB + stage * CHUNK_BYTES, &tmap, b_fullB + 8 * stage, kc * KCH, bj * TILE, p);
                        ++loads;
                        if (++stage == g.stages) {
                            stage = 0;
                            b_phase ^= 1;
                        }
                    }
                }
            }
            if (ok) ok = tq_push(k, TQ_END);
            if (!ok) {
                s_abort = 1;
                atomicExch(g.status, (int)TRI_ETIMEOUT);
            }
            // never leave a copy in flight: wait for the last load into every
            // stage (load k went to stage k % stages, in phase k / stages)
            for (uint32_t st = 0; st < g.stages && st < loads; ++st) {
                const uint32_t last = loads - 1 - ((loads - 1 - st) % g.stages);
                mbar_wait(b_fullB + 8 * st, (last / g.stages) & 1, nullptr);
            }
            if (a_loads) mbar_wait(b_fullA, (a_loads - 1) & 1, nullptr);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t a_row = 0xFFFFFFFFu, a_loads = 0, stage = 0, b_phase = 0, acc = 0, acc_phase = 0;
            bool ok = true;
            const uint64_t a_desc0 = ((uint64_t)kDescHi << 32) | sdesc_lo(sA);
            const uint64_t b_desc0 = ((uint64_t)kDescHi << 32) | sdesc_lo(sB);
            constexpr uint32_t CH16 = CHUNK_BYTES >> 4;  // one 16 KB chunk in descriptor units
            for (uint32_t k = 0;; ++k) {
                unsigned long long v;
                if (!tq_pop(k, v)) {
                    ok = false;
                    break;
                }
                if (v == TQ_END) break;
                const uint32_t bi = (uint32_t)(v >> 32);
                if (bi != a_row) {
                    if (a_loads > 0) umma_commit(b_freeA);  // old A is free once issued MMAs finish
                    if (!mbar_wait(b_fullA, a_loads & 1, &s_abort)) {
                        ok = false;
                        break;
                    }
                    ++a_loads;
                    a_row = bi;
                }
                if (!mbar_wait(b_tempty + 8 * acc, acc_phase ^ 1, &s_abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + acc * TILE;
                for (uint32_t kc = 0; kc < g.nkc && ok; ++kc) {
                    const uint64_t a_desc = a_desc0 + kc * P * CH16;
#pragma unroll
                    for (int pb = 0; pb < P; ++pb) {
                        if (!mbar_wait(b_fullB + 8 * stage, b_phase, &s_abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t b_desc = b_desc0 + stage * CH16;
#pragma unroll
                        for (int pa = 0; pa + pb < P; ++pa)
#pragma unroll
                            for (int kk = 0; kk < KCH / 16; ++kk)
                                // the column tile is the M operand: TMEM lane = output column;
                                // +2 per 16-element K step (32 bytes in 16-byte units)
                                umma_bf16(d_tmem, b_desc + 2 * kk, a_desc + pa * CH16 + 2 * kk,
                                          (kc | pb | pa | kk) ? 1u : 0u);
                        umma_commit(b_emptyB + 8 * stage);  // stage free when these MMAs finish
                        if (++stage == g.stages) {
                            stage = 0;
                            b_phase ^= 1;
                        }
                    }
                }
                if (!ok) break;
                umma_commit(b_tfull + 8 * acc);  // accumulator ready for the epilogue
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicExch(g.status, (int)TRI_ETIMEOUT);
            }
            // all issued MMAs complete before TMEM is released
            umma_commit(b_done);
            mbar_wait(b_done, 0, nullptr);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..17)
        // The accumulator holds the tile transposed: TMEM lane = output column
        // j, TMEM column = output row i.  Warp e = warp - 2 reads lane quarter
        // q = warp % 4 (the quarter a warp may access), so each thread owns one
        // column j, and takes the 16-row chunks c = grp + NG u (grp = e / 4,
        // NG = NEPI / 4 warps per quarter) of the tile's 8.  For every row the warp's 32 lanes hold 32
        // consecutive entries of that packed row: one coalesced 128-byte
        // store per row, straight from registers.  The next chunk's TMEM load
        // is in flight while the current one is processed; the next tile's
        // norms are fetched while the current tile is stored.
        constexpr int NG = NEPI / 4;                // warps per TMEM lane quarter
        constexpr int NCH = TILE / EPI_ROWS / NG;   // 16-row chunks per warp and tile
        const uint32_t e = warp - 2, q = warp & 3, grp = e >> 2;
        float *snorm = epi + e * NORM_FLOATS;     // norms of this warp's rows, two buffers
        float *stg = stage_base + grp * 2 * STG_FLOATS;  // this row group's two staging buffers
        uint32_t hc = 0;                                   // halves staged so far (selects the buffer)
        const float tau = g.tau;
        // next tile's norms: lane l holds the norms of row l % 16 of chunks
        // u = 2v + l / 16 (16 rows each) and of its own column
        float pfr[NCH / 2], pfj = 0.0f;
        auto prefetch = [&](unsigned long long tv) {
            const uint32_t a = (uint32_t)(tv >> 32), b = (uint32_t)tv;
#pragma unroll
            for (int v = 0; v < NCH / 2; ++v) {
                const uint32_t u = 2 * v + (lane >> 4);
                const uint32_t ii = a * TILE + (grp + NG * u) * EPI_ROWS + (lane & 15);
                pfr[v] = ii < g.n ? __ldg(g.norms + ii) : 0.0f;
            }
            const uint32_t jj = b * TILE + q * 32 + lane;
            pfj = jj < g.n ? __ldg(g.norms + jj) : 0.0f;
        };
        uint32_t acc = 0, acc_phase = 0, nbuf = 0, k = 0;
        auto fail = [&]() {
            if (lane == 0) {
                s_abort = 1;
                atomicExch(g.status, (int)TRI_ETIMEOUT);
            }
        };
        unsigned long long cur;
        if (!tq_pop_warp(k++, cur)) {
            fail();
            cur = TQ_END;
        }
        if (cur != TQ_END) prefetch(cur);
        while (cur != TQ_END) {
            const uint32_t bi = (uint32_t)(cur >> 32), bj = (uint32_t)cur;
            float *rn = snorm + nbuf * 32;  // this tile's row norms: [chunk u][16]
#pragma unroll
            for (int v = 0; v < NCH / 2; ++v) rn[32 * v + lane] = pfr[v];
            const float nj = pfj;
            __syncwarp();
            unsigned long long nxt;
            if (!tq_pop_warp(k++, nxt)) {
                fail();
                break;
            }
            if (nxt != TQ_END) prefetch(nxt);
            if (!warp_wait(b_tfull + 8 * acc, acc_phase, &s_abort)) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicExch(g.status, (int)TRI_ETIMEOUT);
                }
                break;
            }
            tc_fence_after();
            const uint32_t j = bj * TILE + q * 32 + lane;  // this thread's column
            const uint32_t taddr = tmem + ((q * 32) << 16) + acc * TILE;
            uint32_t raw[2][EPI_ROWS];
            tmem_ld16(taddr + grp * EPI_ROWS, raw[0]);
#pragma unroll
            for (int u = 0; u < NCH; ++u) {
                uint32_t(&cur)[EPI_ROWS] = raw[u & 1];
                tmem_wait16(cur);
                if (u + 1 < NCH) tmem_ld16(taddr + (grp + NG * (u + 1)) * EPI_ROWS, raw[(u + 1) & 1]);
                const uint32_t i0 = bi * TILE + (grp + NG * u) * EPI_ROWS;  // first row of the chunk
                float ni[EPI_ROWS];
#pragma unroll
                for (int k = 0; k < EPI_ROWS; k += 4) {
                    const float4 v4 = *reinterpret_cast<const float4 *>(rn + u * EPI_ROWS + k);
                    ni[k] = v4.x;
                    ni[k + 1] = v4.y;
                    ni[k + 2] = v4.z;
                    ni[k + 3] = v4.w;
                }
                // fast path: d = d2 * rsqrt(d2); one test per chunk for a pair
                // with d2 <= tau (|x_i|^2 + |x_j|^2) (cancellation, the
                // diagonal, or padding)
                float dv[EPI_ROWS], d2v[EPI_ROWS];
                float worst = 1.0f;
#pragma unroll
                for (int k = 0; k < EPI_ROWS; ++k) {
                    const float s = ni[k] + nj;
                    const float d2 = fmaf(-2.0f, __uint_as_float(cur[k]), s);
                    d2v[k] = d2;
                    worst = fminf(worst, fmaf(-tau, s, d2));
                    dv[k] = d2 * rsqrt_approx(d2);
                }
                if (worst <= 0.0f) {
#pragma unroll
                    for (int k = 0; k < EPI_ROWS; ++k) {
                        const float d2 = d2v[k];
                        if (d2 <= tau * (ni[k] + nj)) {
                            const uint32_t i = i0 + k;
                            if (i < g.n && j < i) {
                                const unsigned long long slot = atomicAdd(g.flag_count, 1ull);
                                if (slot < g.flag_cap) g.flag_list[slot] = ((unsigned long long)i << 32) | j;
                            }
                            // provisional value (flagged pairs are recomputed; the diagonal is exact 0)
                            dv[k] = (i == j || d2 <= 0.0f) ? 0.0f : d2 * rsqrt_approx(d2);
                        }
                    }
                }
                if constexpr (P == 2) {
                // Store through shared memory in two halves of 8 rows: the row
                // group's four warps (one per 32-column quarter) write their
                // columns of each row into a staging row shifted by the row's
                // 16-byte phase (T2(i0 + k) mod 4, which depends on k only since
                // i0 is a multiple of 16); then each warp writes two whole row
                // segments, the aligned middle with one float4 per lane and the
                // ends with scalar stores, so every 128-byte line of a segment's
                // middle is written by one instruction.  The two staging buffers
                // alternate: the barrier before a half's stores also tells each
                // warp that the group has finished reading the buffer it will
                // fill next, so one barrier per half suffices.
#pragma unroll
                for (int half = 0; half < EPI_ROWS / STG_ROWS; ++half) {
                    float *sb = stg + (hc & 1) * STG_FLOATS;
                    ++hc;
#pragma unroll
                    for (int kk = 0; kk < STG_ROWS; ++kk) {
                        const int k = half * STG_ROWS + kk;
                        sb[kk * STG_LD + row_phase(k) + q * 32 + lane] = dv[k];
                    }
                    named_sync(1 + grp, 128);
#pragma unroll
                    for (int r2 = 0; r2 < STG_ROWS / 4; ++r2) {
                        const uint32_t kk = q * (STG_ROWS / 4) + r2, k = half * STG_ROWS + kk, i = i0 + k;
                        if (i < g.n) {
                            const uint32_t len = bi == bj ? i - bj * TILE + 1 : TILE;  // columns of row i here
                            float *seg = g.out + T2(i) + bj * TILE;
                            const uint32_t ph = row_phase(k), head = (4 - ph) & 3;
                            const float *src = sb + kk * STG_LD + ph;
                            const uint32_t h = head < len ? head : len;
                            const uint32_t nv = (len - h) >> 2;
                            if (lane < nv)
                                __stcs(reinterpret_cast<float4 *>(seg + h) + lane,
                                       *reinterpret_cast<const float4 *>(src + h + 4 * lane));
                            const uint32_t t0 = h + 4 * nv, tail = len - t0;  // h <= 3, tail <= 3
                            if (lane < h) __stcs(seg + lane, src[lane]);
                            if (lane >= 4 && lane - 4 < tail) __stcs(seg + t0 + lane - 4, src[t0 + lane - 4]);
                        }
                    }
                }
                } else {
                    // Direct stores: for each row the warp's 32 lanes hold 32
                    // consecutive packed entries, written by one 128-byte store.
                    // For P = 3 the tensor core's operand reads already take most
                    // of the shared-memory bandwidth, and staging (which also
                    // costs two operand stages) measured slower.
                    float *row = g.out + T2(i0) + j;  // row i0, column j
                    if (bi != bj && (bi + 1) * TILE <= g.n) {
#pragma unroll
                        for (int k = 0; k < EPI_ROWS; ++k) {
                            __stcs(row, dv[k]);
                            row += i0 + k + 1;  // T2(i + 1) - T2(i)
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < EPI_ROWS; ++k) {
                            const uint32_t i = i0 + k;
                            if (i < g.n && j <= i) __stcs(row, dv[k]);
                            row += i + 1;
                        }
                    }
                }
            }
            tc_fence_before();
            if (lane == 0) mbar_arrive(b_tempty + 8 * acc);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1;
            }
            nbuf ^= 1;
            cur = nxt;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// -------------------------------------------------------------- fixup ----
// FP64 direct-difference recompute of the flagged pairs.  If the list
// overflowed, every pair whose stored distance passes a slightly wider
// version of the flag test is recomputed instead.
__global__ void fixup_kernel(const float *__restrict__ x, uint32_t n, uint32_t d, float *__restrict__ out,
                             const float *__restrict__ norms, const unsigned long long *__restrict__ count,
                             const unsigned long long *__restrict__ list, unsigned long long cap, float tau,
                             unsigned long long *n_flagged)
{
    const unsigned long long cnt = *count;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (uint64_t)gridDim.x * blockDim.x;
    if (tid == 0 && n_flagged) *n_flagged = cnt;
    auto recompute = [&](uint32_t i, uint32_t j) {
        const float *xi = x + (size_t)i * d, *xj = x + (size_t)j * d;
        double s = 0.0;
        for (uint32_t k = 0; k < d; ++k) {
            const double df = (double)xi[k] - (double)xj[k];
            s = fma(df, df, s);
        }
        out[T2(i) + j] = (float)sqrt(s);
    };
    if (cnt <= cap) {
        for (uint64_t e = tid; e < cnt; e += nth) {
            const unsigned long long v = list[e];
            recompute((uint32_t)(v >> 32), (uint32_t)(v & 0xFFFFFFFFu));
        }
    } else {
        const uint64_t total = T2(n);
        const float wide = 1.0625f * tau;
        for (uint64_t p = tid; p < total; p += nth) {
            uint32_t i, j;
            lambda_diag<TRI_SQRT_X>((uint32_t)p, i, j);
            if (i == j) continue;
            const float v = out[p];
            if (v * v < wide * (norms[i] + norms[j])) recompute(i, j);
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

uint32_t num_sms()
{
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? (uint32_t)nsm : 1;
}

}  // namespace

size_t trihost::edm_tc_workspace(uint32_t n, uint32_t d, int prec) { return ws_layout(n, d, prec).total; }

namespace {

struct TcPlan {
    int P;
    uint32_t dp, nkc, stages;
    size_t smem;
};

bool plan(uint32_t d, int prec, TcPlan &p)
{
    p.P = prec == TRI_BF16X6 ? 3 : 2;
    p.dp = (d + KCH - 1) / KCH * KCH;
    p.nkc = p.dp / KCH;
    const size_t stg = p.P == 2 ? (size_t)(NEPI / 4) * 2 * STG_FLOATS : 0;  // P = 2 stages its stores
    const size_t fixed = 1024 /*align*/ + (NEPI * NORM_FLOATS + stg) * 4 + 8 * (7 + 2 * MAX_STAGES);
    const size_t a = (size_t)p.P * p.nkc * CHUNK_BYTES, st = CHUNK_BYTES;
    if (fixed + a + 2 * st > (size_t)SMEM_LIMIT) return false;
    p.stages = (uint32_t)std::min<size_t>(MAX_STAGES, (SMEM_LIMIT - fixed - a) / st);
    p.smem = fixed + a + p.stages * st;
    return true;
}

}  // namespace

// Largest n whose packed triangle n(n+1)/2 stays below 2^32 entries (the
// recompute pass walks it with 32-bit lambda).
constexpr uint32_t TC_MAX_N = 92681;

extern "C" int tri_edm_prepare(const float *x, uint32_t n, uint32_t d, int prec, void *workspace, size_t ws_bytes,
                               void *stream)
{
    if (!x || n == 0 || d == 0) return TRI_EINVAL;
    if (n > TC_MAX_N) return TRI_ERANGE;
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    TcPlan pl;
    if (!plan(d, prec, pl)) return TRI_ERANGE;
    const WsLayout L = ws_layout(n, d, prec);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 255)) return TRI_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) return TRI_ECUDA;
    const unsigned blocks = (unsigned)(((uint64_t)n * 32 + 255) / 256);
    if (pl.P == 3)
        prepare_kernel<3><<<blocks, 256, 0, s>>>(x, n, d, pl.dp, (float *)(ws + L.norms),
                                                 (__nv_bfloat16 *)(ws + L.planes));
    else
        prepare_kernel<2><<<blocks, 256, 0, s>>>(x, n, d, pl.dp, (float *)(ws + L.norms),
                                                 (__nv_bfloat16 *)(ws + L.planes));
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tri_edm_gram(uint32_t n, uint32_t d, float *out, int map, int prec, void *workspace, size_t ws_bytes,
                            void *stream)
{
    if (!out || n == 0 || d == 0) return TRI_EINVAL;
    if (n > TC_MAX_N) return TRI_ERANGE;
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_BB) return TRI_EINVAL;
    if ((uintptr_t)out & 15) return TRI_EINVAL;  // row segments are written with 16-byte stores
    TcPlan pl;
    if (!plan(d, prec, pl)) return TRI_ERANGE;
    const WsLayout L = ws_layout(n, d, prec);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 255)) return TRI_ENOSPACE;
    const uint32_t m = (n + TILE - 1) / TILE;
    const uint64_t ntiles = map == TRI_MAP_LAMBDA ? T2(m) : (uint64_t)m * m;
    if (ntiles > 0xFFFFFFFFull) return TRI_ERANGE;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return TRI_ECUDA;
    char *ws = (char *)workspace;
    CUtensorMap tmap;
    const cuuint64_t gdim[3] = {pl.dp, n, (cuuint64_t)pl.P};
    const cuuint64_t gstride[2] = {(cuuint64_t)pl.dp * 2, (cuuint64_t)n * pl.dp * 2};
    const cuuint32_t box[3] = {KCH, TILE, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ws + L.planes, gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return TRI_ECUDA;
    GramArgs g{};
    g.n = n;
    g.nkc = pl.nkc;
    g.m = m;
    g.ntiles = ntiles;
    g.stages = pl.stages;
    g.tau = pl.P == 3 ? TAU_X6 : TAU_X3;
    g.norms = (const float *)(ws + L.norms);
    g.out = out;
    g.flag_count = (unsigned long long *)(ws + L.hdr);
    g.status = (int *)(ws + L.hdr + 8);
    g.tile_counter = (unsigned long long *)(ws + L.hdr + 16);
    g.flag_list = (unsigned long long *)(ws + L.flags);
    g.flag_cap = L.cap;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(num_sms(), ntiles);
    g.static_per = ntiles * STATIC_PCT / 100 / grid;
    g.dyn_start = g.static_per * grid;
    g.chunk = DYN_CHUNK;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(g.tile_counter, 0, sizeof(unsigned long long), s) != cudaSuccess) return TRI_ECUDA;
    cudaError_t e;
#define TRI_G(MP, PP)                                                                                          \
    e = cudaFuncSetAttribute(gram_kernel<MP, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);  \
    if (e == cudaSuccess) gram_kernel<MP, PP><<<grid, NTHREADS, pl.smem, s>>>(tmap, g);
    if (map == TRI_MAP_LAMBDA) {
        if (pl.P == 3) {
            TRI_G(MAP_LAMBDA, 3)
        } else {
            TRI_G(MAP_LAMBDA, 2)
        }
    } else {
        if (pl.P == 3) {
            TRI_G(MAP_BB, 3)
        } else {
            TRI_G(MAP_BB, 2)
        }
    }
#undef TRI_G
    if (e != cudaSuccess) return TRI_ECUDA;
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

extern "C" int tri_edm_fixup(const float *x, uint32_t n, uint32_t d, float *out, int prec, void *workspace,
                             size_t ws_bytes, unsigned long long *n_flagged, void *stream)
{
    if (!x || !out || n == 0 || d == 0) return TRI_EINVAL;
    if (n > TC_MAX_N) return TRI_ERANGE;
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    const WsLayout L = ws_layout(n, d, prec);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 255)) return TRI_ENOSPACE;
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream;
    fixup_kernel<<<num_sms() * 4, 256, 0, s>>>(x, n, d, out, (const float *)(ws + L.norms),
                                               (const unsigned long long *)(ws + L.hdr),
                                               (const unsigned long long *)(ws + L.flags), L.cap,
                                               prec == TRI_BF16X6 ? TAU_X6 : TAU_X3, n_flagged);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

int trihost::edm_tc(const float *x, uint32_t n, uint32_t d, float *out, int map, int prec, void *ws,
                    size_t ws_bytes, unsigned long long *n_flagged, cudaStream_t s)
{
    int st = tri_edm_prepare(x, n, d, prec, ws, ws_bytes, s);
    if (st == TRI_OK) st = tri_edm_gram(n, d, out, map, prec, ws, ws_bytes, s);
    if (st == TRI_OK) st = tri_edm_fixup(x, n, d, out, prec, ws, ws_bytes, n_flagged, s);
    return st;
}
