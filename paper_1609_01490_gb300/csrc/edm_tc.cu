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
// Kernels.  prepare: row norms (FP32 pairs, stored as FP32) and the BF16 planes,
// K padded to a multiple of 64.  gram: persistent clusters of two CTAs on two
// SMs (a CTA pair), one pair per two SMs.  A unit of work is a 2 x 2 block of
// 128 x 128 pair tiles (row blocks 2R, 2R + 1, column blocks 2C, 2C + 1),
// taken in lambda order over the triangle of units (Eq. eq_gmap): first one
// contiguous run of units per pair, then short runs from a global counter by
// whichever pair is free.  CTA r keeps row block 2R + r resident in shared
// memory (the planes of A, reloaded when R changes) and streams column block
// 2C + r through a ring of 16 KB TMA stages, one plane of one 64-wide K chunk
// each.  One thread of the even CTA issues tcgen05.mma.cta_group::2 with M =
// 256 (the two column blocks), N = 256 (the two row blocks), K = 16, so each
// instruction does 128 x 256 x 16 on each SM; each CTA's TMEM receives its
// column block x both row blocks, double buffered (2 x 256 columns).  Warp 0
// of the even CTA takes the units and passes them to both CTAs' roles through
// a small queue in shared memory (written across the pair); warp 0 of each CTA
// issues its TMA; warps 2-17 of each CTA read TMEM back (lanes = output
// columns), form the distances, flag cancellations and store the packed rows
// (one coalesced 128-byte store per warp and row; the four warps that hold the
// four 32-column quarters of the same rows store them together).  fixup: FP64
// recompute of the flagged pairs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>

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
// Each epilogue warp holds TILE / (NEPI / 4) rows of a tile: the norm buffers
// and the prefetch pattern are sized for 32 (16 epilogue warps).
static_assert(TILE / (NEPI / 4) == 32, "epilogue norm buffers assume 32 rows per warp and tile");
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // a bounded wait gives up after 2 s
constexpr int TQ = 8;                      // unit queue slots (producer -> MMA and epilogues, both CTAs)
constexpr unsigned long long TQ_END = ~0ull;  // queue entry after the last unit
constexpr uint32_t STATIC_PCT = 80;        // share of the units assigned up front, in contiguous runs per pair
constexpr uint32_t DYN_CHUNK = 2;          // units per grab from the global counter afterwards
constexpr int SMEM_LIMIT = 227 * 1024;
constexpr int MAX_STAGES = 12;             // B ring depth cap (16 KB stages)

constexpr float TAU_X3 = 0.0625f;  // flag threshold for hi/lo (empirical)

// Flag threshold for hi/mid/lo with nkc 64-wide K chunks.  The Gram term's
// error is at most 2^-23 (dropped products) plus 2^-23 per FP32 accumulation
// step (24 MMAs of K = 16 per chunk: 6 plane products x 4) of
// sum_k |x_ik x_jk| <= (|x_i|^2 + |x_j|^2) / 2; with the norms' and the final
// combination's roundings, |error of d^2| <= (2 + 24 nkc) 2^-23 (|x_i|^2 +
// |x_j|^2).  The relative error of d is about half that of d^2, and the
// square root adds up to ~1.5e-7, so a pair with d^2 > tau (|x_i|^2 + |x_j|^2)
// stays within 1e-5 when tau = (2 + 24 nkc) 2^-23 / (2 (1e-5 - 2e-7)).
// tau = 0.158 (d <= 64), 0.304 (d <= 128), 0.450 (d <= 192).
float tau_x6(uint32_t nkc) { return (float)((2.0 + 24.0 * nkc) * std::ldexp(1.0, -23) / (2.0 * (1e-5 - 2e-7))); }

float flag_tau(int prec, uint32_t d)
{
    return prec == TRI_BF16X6 ? tau_x6((d + KCH - 1) / KCH) : TAU_X3;
}

struct WsLayout {
    size_t hdr, norms, planes, flags, total;
    unsigned long long cap;
};

// Workspace: [header 256 B: flag counter (u64 at 0), status (int at 8), tile
// counter (u64 at 16), tri_edm_host's two list-start slots (u64 at 24, 32),
// the wait limit of the Gram kernel's waits between roles in ns (u64 at 40,
// 0: WAIT_LIMIT_NS)][norms n FP32][planes P x n x dp BF16][flag list cap x
// u64], each part 256-byte aligned.  tri_edm_prepare clears the header.
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

// As mbar_try, with acquire at cluster scope: for barriers that the other CTA
// of the pair arrives on with release at cluster scope.
__device__ __forceinline__ bool mbar_try_cl(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
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
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns = WAIT_LIMIT_NS)
{
    auto test = [&]() { return CL ? mbar_try_cl(bar, parity) : mbar_try(bar, parity); };
    if (test()) return true;
    const uint64_t start = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (test()) return true;
        if ((it & 15) == 0) {
            if (abort_flag && *abort_flag) return false;
            if (global_ns() - start > limit_ns) return false;
            __nanosleep(64);
        }
    }
}

// mbar_wait by lane 0 with the result broadcast, so the whole warp leaves
// together and agrees on it.
template <bool CL = false>
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, uint64_t limit_ns)
{
    int r = 0;
    if ((threadIdx.x & 31) == 0) r = mbar_wait<CL>(bar, parity, abort_flag, limit_ns) ? 1 : 0;
    return __shfl_sync(0xffffffffu, r, 0) != 0;
}

// ------------------------------------------------------- CTA pair ----
// The Gram kernel runs as clusters of two CTAs on two SMs (a CTA pair).
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// All threads of both CTAs; orders earlier shared-memory writes (and barrier
// initialisation) before later accesses by the other CTA.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Arrive on a barrier given by its cluster address (own or the other CTA's),
// with release at CTA scope: it orders nothing of this thread's other memory
// traffic for the other CTA, and so does not wait for this thread's pending
// global stores (a cluster-scope release would).  Used where the waiting side
// needs no data from this thread (tcgen05 fences order the TMEM reads).
__device__ __forceinline__ void mbar_arrive_cl(uint32_t cl_bar)
{
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cl_bar) : "memory");
}

// Arrive with release at cluster scope: orders this thread's earlier stores
// into the other CTA's shared memory before the arrival.
__device__ __forceinline__ void mbar_arrive_cl_release(uint32_t cl_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Cancels bytes that a phase was told to expect (copies that never started).
__device__ __forceinline__ void mbar_complete_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void st_cl_u32(uint32_t cl_addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cl_addr), "r"(v) : "memory");
}

__device__ __forceinline__ void st_cl_u64(uint32_t cl_addr, unsigned long long v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(cl_addr), "l"(v) : "memory");
}

__device__ __forceinline__ void st_cl_s32(uint32_t cl_addr, int v)
{
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(cl_addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_cl_u32(uint32_t cl_addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(cl_addr) : "memory");
    return v;
}

// TMA tile load into this CTA's shared memory whose completion (bytes) is
// counted on a barrier of either CTA of the pair (cl_bar: cluster address).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, uint32_t cl_bar, int x, int y,
                                                 int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(cl_bar)
        : "memory");
}

// Instruction descriptor, kind::f16 across the CTA pair: FP32 accumulator,
// BF16 A and B, both K-major, N = 256 (bits 17-22 hold N/8), M = 256 (bits
// 24-28 hold M/16).  Rows 0-127 of M (and of N) come from the even CTA,
// 128-255 from the odd one; each CTA's TMEM receives its own 128 rows of M
// across all 256 columns of N.
constexpr uint32_t IDESC2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * TILE) >> 3) << 17) |
                            ((uint32_t)((2 * TILE) >> 4) << 24);

// One MMA over the pair: A (M side) and B (N side) are read at the same
// shared-memory offsets in both CTAs; each CTA holds half of A's M rows and
// half of B's N rows.
__device__ __forceinline__ void umma2_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC2), "r"(accumulate)
        : "memory");
}

// Arrive on the barrier at this offset in both CTAs once the issued MMAs finish.
__device__ __forceinline__ void umma2_commit_both(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"((uint16_t)3)
        : "memory");
}

// Arrive on the issuing CTA's barrier once the issued MMAs finish.
__device__ __forceinline__ void umma2_commit_own(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
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
// Error-free transformations on FP32 pairs (Knuth's TwoSum; the product error
// from one FMA): a + b = s + e and a * a = p + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// One warp per row: the BF16 planes and the row norm |x|^2, summed as an
// unevaluated pair hi + lo of FP32 numbers (products split exactly by FMA,
// sums by TwoSum; about 48 significant bits, FP64 being scarce on this part),
// rounded to FP32 once at the end.
template <int P>
__global__ void prepare_kernel(const float *__restrict__ x, uint32_t n, uint32_t d, uint32_t dp,
                               float *__restrict__ norms, __nv_bfloat16 *__restrict__ planes)
{
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float *row = x + (size_t)warp * d;
    float hi = 0.0f, lo = 0.0f;
    for (uint32_t k = lane; k < dp; k += 32) {
        const float v = k < d ? row[k] : 0.0f;
        const float p = v * v, pe = fmaf(v, v, -p);  // v^2 = p + pe
        float t, te;
        two_sum(hi, p, t, te);
        hi = t;
        lo += te + pe;
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
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, o), ol = __shfl_down_sync(0xffffffffu, lo, o);
        float t, te;
        two_sum(hi, oh, t, te);
        hi = t;
        lo += ol + te;
    }
    if (lane == 0) norms[warp] = hi + lo;
}

// --------------------------------------------------------------- gram ----
// A unit is a 2 x 2 block of tiles: row blocks 2R, 2R + 1 and column blocks
// 2C, 2C + 1.  CTA r of the pair holds row block 2R + r (half of the MMA's N
// side) and streams column block 2C + r (half of its M side); its accumulator
// covers the tiles (2R, 2C + r) and (2R + 1, 2C + r).
struct GramArgs {
    uint32_t n, nkc;           // points, 64-wide K chunks
    uint32_t m;                // tile rows of the triangle
    uint32_t mb;               // unit rows: ceil(m / 2)
    uint64_t u0, nunits;       // units walked: [u0, nunits) of lambda over the mb-row triangle or the mb x mb box
    uint64_t static_per;       // units per CTA pair in its up-front run
    uint64_t dyn_start;        // first unit handed out by the counter
    uint32_t chunk;            // units per grab from the counter
    uint32_t stages;           // B ring depth
    float tau;
    const float *norms;
    float *out;
    unsigned long long *flag_count, *flag_list, flag_cap;
    unsigned long long *tile_counter;  // zero at launch
    int *status;
    const unsigned long long *wait_limit;  // ns a wait between roles may take; 0: WAIT_LIMIT_NS
};

// Unit number u -> (R, C): lambda over the triangle of units (Eq. eq_gmap),
// or row-major over the mb x mb box with units above the diagonal skipped.
template <int MAP>
__device__ __forceinline__ bool unit_of(uint64_t u, uint32_t mb, uint32_t &R, uint32_t &C)
{
    if constexpr (MAP == MAP_LAMBDA) {
        lambda_diag<TRI_SQRT_R>((uint32_t)u, R, C);
        return true;
    } else {
        R = (uint32_t)(u / mb);
        C = (uint32_t)(u - (uint64_t)R * mb);
        return C <= R;
    }
}

// The split keeps the products of row plane pa and column plane pb with
// pa + pb <= P - 1: hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid for P = 3
// and hi.hi, hi.lo, lo.hi for P = 2.


// Barrier among the `count` threads of one epilogue row group (ids 1..).
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// The same barrier with a vote: true iff `ok` holds in every thread of the
// group.  A named barrier cannot give up, so the row group takes a unit (and
// the barriers inside it) only when all four of its warps have one; after a
// failed wait in any of them, all four stop together.
__device__ __forceinline__ bool named_sync_all(uint32_t id, uint32_t count, bool ok)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(id), "r"(count)
        : "memory");
    return r != 0;
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
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    gram_kernel(const __grid_constant__ CUtensorMap tmap, const GramArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand area, at the same offsets in both CTAs
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t a_bytes = (uint32_t)P * g.nkc * CHUNK_BYTES;  // this CTA's row block
    constexpr uint32_t stage_bytes = CHUNK_BYTES;               // one plane of one K chunk
    const uint32_t sA = base;                                   // [kc][p] chunks
    const uint32_t sB = base + a_bytes;                         // [stage] chunks of one plane
    float *epi = reinterpret_cast<float *>(gbase + a_bytes + g.stages * stage_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(epi + NEPI * NORM_FLOATS);
    // barriers: fullA, freeA, done, tmem_full[2], tmem_empty[2], fullB[stages], emptyB[stages]
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t b_fullA = bar0, b_freeA = bar0 + 8, b_done = bar0 + 16;
    const uint32_t b_tfull = bar0 + 24, b_tempty = bar0 + 40;
    const uint32_t b_fullB = bar0 + 56, b_emptyB = bar0 + 56 + 8 * g.stages;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    // unit queue: entry (R << 32 | C), or TQ_END, written by the even CTA's
    // producer into both CTAs
    __shared__ volatile unsigned long long s_tq[TQ];
    __shared__ __align__(8) uint64_t s_tqbar[2 * TQ];
    // the odd CTA's copy counts (B stages, A row blocks), reported to the even
    // CTA's producer at the end so that it can wait for every copy in flight
    __shared__ uint32_t s_odd_loads[2];
    __shared__ __align__(8) uint64_t s_odd_done;
    const uint32_t b_tqfull = smem_u32(s_tqbar), b_tqempty = b_tqfull + 8 * TQ;

    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank(), other = rank ^ 1u;
    const bool leader = rank == 0;  // the even CTA issues the pair's MMAs
    // Barriers that count work of both CTAs live in the even CTA: fullA and
    // fullB (one expect_tx arrival by the even CTA for both CTAs' bytes: the
    // odd CTA's copies may land before it, which only takes the transaction
    // count below zero until the arrival), tmem_empty
    // (every epilogue warp of both) and the queue's empty barriers (the even
    // CTA's MMA thread and epilogue warps, the odd CTA's producer and epilogue
    // warps).  freeA, emptyB and tmem_full receive one multicast commit in each CTA.
    if (threadIdx.x == 0) {
        s_abort = 0;
        mbar_init(b_fullA, 1);
        mbar_init(b_freeA, 1);
        mbar_init(b_done, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_tfull + 8 * i, 1);
            mbar_init(b_tempty + 8 * i, 2 * NEPI);
        }
        for (uint32_t s = 0; s < g.stages; ++s) {
            mbar_init(b_fullB + 8 * s, 1);
            mbar_init(b_emptyB + 8 * s, 1);
        }
        for (int s = 0; s < TQ; ++s) {
            mbar_init(b_tqfull + 8 * s, 1);
            mbar_init(b_tqempty + 8 * s, 2 + 2 * NEPI);
        }
        mbar_init(smem_u32(&s_odd_done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // one warp in each CTA of the pair allocates (the pair's accumulators
        // sit at the same TMEM address in both)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    // The MMAs address both CTAs' accumulators with the even CTA's address:
    // run only if the two allocations agree.
    const bool run = ld_cl_u32(mapa(smem_u32(&s_tmem), other)) == tmem;
    if (!run && threadIdx.x == 0) atomicExch(g.status, (int)TRI_ECUDA);
    // limit of the waits between roles (the waits that drain copies and MMAs
    // before exit always keep WAIT_LIMIT_NS)
    const uint64_t wl = *g.wait_limit ? (uint64_t)*g.wait_limit : WAIT_LIMIT_NS;

    // cluster addresses of the even CTA's shared barriers and of the other CTA's queue
    const uint32_t L_fullA = mapa(b_fullA, 0), L_fullB = mapa(b_fullB, 0), L_tempty = mapa(b_tempty, 0);
    const uint32_t L_tqempty = mapa(b_tqempty, 0);
    const uint32_t O_tqfull = mapa(b_tqfull, other), O_tq = mapa(smem_u32((const void *)s_tq), other);
    const uint32_t O_abort = mapa(smem_u32((const void *)&s_abort), other);
    // a failed wait stops both CTAs of the pair
    auto give_up = [&]() {
        s_abort = 1;
        st_cl_s32(O_abort, 1);
        atomicExch(g.status, (int)TRI_ETIMEOUT);
    };

    // Queue entry k sits in slot k % TQ; its fill is phase k / TQ of the slot's barriers.
    // Pushed by the even CTA's producer into both CTAs.
    auto tq_push = [&](uint32_t k, unsigned long long v) {
        const uint32_t slot = k % TQ;
        if (!mbar_wait(b_tqempty + 8 * slot, ((k / TQ) & 1) ^ 1, &s_abort, wl)) return false;
        s_tq[slot] = v;
        mbar_arrive(b_tqfull + 8 * slot);
        st_cl_u64(O_tq + 8 * slot, v);
        mbar_arrive_cl_release(O_tqfull + 8 * slot);
        return true;
    };
    // by one thread (the even CTA's MMA issuer, the odd CTA's producer)
    auto tq_pop = [&](uint32_t k, unsigned long long &v) {
        const uint32_t slot = k % TQ;
        if (!mbar_wait<true>(b_tqfull + 8 * slot, (k / TQ) & 1, &s_abort, wl)) return false;
        v = s_tq[slot];
        mbar_arrive_cl(L_tqempty + 8 * slot);  // release (CTA scope) orders the read before the arrival
        return true;
    };
    // by a whole epilogue warp: lane 0 waits, reads and releases the slot, then
    // broadcasts the entry
    auto tq_pop_warp = [&](uint32_t k, unsigned long long &v) {
        unsigned long long r = 0;
        int ok = 0;
        if ((threadIdx.x & 31) == 0) {
            const uint32_t slot = k % TQ;
            ok = mbar_wait<true>(b_tqfull + 8 * slot, (k / TQ) & 1, &s_abort, wl) ? 1 : 0;
            if (ok) {
                r = s_tq[slot];
                mbar_arrive_cl(L_tqempty + 8 * slot);  // release (CTA scope) orders the read before the arrival
            }
        }
        v = __shfl_sync(0xffffffffu, r, 0);
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    // The TMA and MMA roles run on lane 0 of their warps.  Between two MMAs
    // the issuing thread does nothing but add descriptor offsets: a
    // 256x256x16 pair MMA takes about 136 cycles on each SM, and any longer
    // gap in the issue stream leaves the tensor pipes idle.  Each stage holds
    // one plane of one 64-wide K chunk of a CTA's column block: the MMA thread
    // waits once per 4 (P - pb) MMAs for column plane pb.
    if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0 && run) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap) : "memory");
            uint32_t a_row = 0xFFFFFFFFu, a_loads = 0, stage = 0, b_phase = 0, loads = 0, k = 0;
            bool ok = true;
            // the pair's up-front run of units, then runs from the counter
            uint64_t u = g.u0 + (uint64_t)(blockIdx.x >> 1) * g.static_per, uend = u + g.static_per;
            for (;;) {
                uint32_t R, C;
                if (leader) {
                    bool have = false;
                    while (!have) {
                        if (u >= uend) {
                            u = g.dyn_start + atomicAdd(g.tile_counter, (unsigned long long)g.chunk);
                            if (u >= g.nunits) break;
                            uend = u + g.chunk < g.nunits ? u + g.chunk : g.nunits;
                        }
                        have = unit_of<MAP>(u++, g.mb, R, C);
                    }
                    if (!have) break;
                    if (!tq_push(k++, ((unsigned long long)R << 32) | C)) {
                        ok = false;
                        break;
                    }
                } else {
                    unsigned long long v;
                    if (!tq_pop(k++, v)) {
                        ok = false;
                        break;
                    }
                    if (v == TQ_END) break;
                    R = (uint32_t)(v >> 32);
                    C = (uint32_t)v;
                }
                const uint32_t rb = 2 * R + rank, cb = 2 * C + rank;  // this CTA's row and column blocks
                if (R != a_row) {
                    if (a_loads > 0 && !mbar_wait(b_freeA, (a_loads - 1) & 1, &s_abort, wl)) {
                        ok = false;
                        break;
                    }
                    if (leader) mbar_expect_tx(b_fullA, 2 * a_bytes);
                    for (uint32_t kc = 0; kc < g.nkc; ++kc)
                        for (int pl = 0; pl < P; ++pl)
                            tma_load_3d_pair(sA + (kc * P + pl) * CHUNK_BYTES, &tmap, L_fullA, kc * KCH, rb * TILE, pl);
                    ++a_loads;
                    a_row = R;
                }
                for (uint32_t kc = 0; kc < g.nkc && ok; ++kc) {
                    for (int pl = 0; pl < P; ++pl) {
                        if (!mbar_wait(b_emptyB + 8 * stage, b_phase ^ 1, &s_abort, wl)) {
                            ok = false;
                            break;
                        }
                        if (leader) mbar_expect_tx(b_fullB + 8 * stage, 2 * stage_bytes);
                        tma_load_3d_pair(sB + stage * CHUNK_BYTES, &tmap, L_fullB + 8 * stage, kc * KCH, cb * TILE, pl);
                        ++loads;
                        if (++stage == g.stages) {
                            stage = 0;
                            b_phase ^= 1;
                        }
                    }
                }
                if (!ok) break;
            }
            if (leader && ok) ok = tq_push(k, TQ_END);
            if (!ok) give_up();
            // Never leave a copy in flight.  Both CTAs' copies complete on the
            // even CTA's barriers, whose phases need the even CTA's expect_tx
            // arrival and both CTAs' bytes.  After a give-up the two producers
            // may have started different numbers of copies (the odd one up to
            // a ring ahead of the even one, or behind it; A row blocks at most
            // one apart), so the odd CTA reports its counts and the even one
            // arrives with the byte count of each copy only the odd CTA
            // started, and cancels the expected bytes of each copy it alone
            // started.  Then every phase up to the last copy completes once its
            // bytes land, and the even CTA waits for them all: load k went to
            // stage k % stages, phase k / stages.  The final cluster barrier
            // holds the odd CTA until then.
            if (!leader) {
                st_cl_u32(mapa(smem_u32(&s_odd_loads[0]), 0), loads);
                st_cl_u32(mapa(smem_u32(&s_odd_loads[1]), 0), a_loads);
                mbar_arrive_cl_release(mapa(smem_u32(&s_odd_done), 0));
            } else {
                uint32_t lo = loads, ao = a_loads;
                if (mbar_wait<true>(smem_u32(&s_odd_done), 0, nullptr)) {
                    lo = *(volatile uint32_t *)&s_odd_loads[0];
                    ao = *(volatile uint32_t *)&s_odd_loads[1];
                }
                for (uint32_t c = lo; c < loads; ++c) mbar_complete_tx(b_fullB + 8 * (c % g.stages), stage_bytes);
                for (uint32_t c = loads; c < lo; ++c) mbar_expect_tx(b_fullB + 8 * (c % g.stages), stage_bytes);
                if (ao < a_loads) mbar_complete_tx(b_fullA, a_bytes);
                if (ao > a_loads) mbar_expect_tx(b_fullA, a_bytes);
                const uint32_t nb = loads > lo ? loads : lo, na = a_loads > ao ? a_loads : ao;
                for (uint32_t st = 0; st < g.stages && st < nb; ++st) {
                    const uint32_t last = nb - 1 - ((nb - 1 - st) % g.stages);
                    mbar_wait(b_fullB + 8 * st, (last / g.stages) & 1, nullptr);
                }
                if (na) mbar_wait(b_fullA, (na - 1) & 1, nullptr);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (even CTA)
        if (lane == 0 && leader && run) {
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
                const uint32_t R = (uint32_t)(v >> 32);
                if (R != a_row) {
                    if (a_loads > 0) umma2_commit_both(b_freeA);  // old A is free once issued MMAs finish
                    if (!mbar_wait(b_fullA, a_loads & 1, &s_abort, wl)) {
                        ok = false;
                        break;
                    }
                    ++a_loads;
                    a_row = R;
                }
                if (!mbar_wait(b_tempty + 8 * acc, acc_phase ^ 1, &s_abort, wl)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem + acc * (2 * TILE);  // 256 columns per accumulator
                for (uint32_t kc = 0; kc < g.nkc && ok; ++kc) {
                    const uint64_t a_desc = a_desc0 + kc * P * CH16;
#pragma unroll
                    for (int pb = 0; pb < P; ++pb) {
                        if (!mbar_wait(b_fullB + 8 * stage, b_phase, &s_abort, wl)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t b_desc = b_desc0 + stage * CH16;
#pragma unroll
                        for (int pa = 0; pa + pb < P; ++pa)
#pragma unroll
                            for (int kk = 0; kk < KCH / 16; ++kk)
                                // the column blocks are the M operand: TMEM lane = output
                                // column; +2 per 16-element K step (32 bytes in 16-byte units)
                                umma2_bf16(d_tmem, b_desc + 2 * kk, a_desc + pa * CH16 + 2 * kk,
                                           (kc | pb | pa | kk) ? 1u : 0u);
                        umma2_commit_both(b_emptyB + 8 * stage);  // stage free (both CTAs) when these MMAs finish
                        if (++stage == g.stages) {
                            stage = 0;
                            b_phase ^= 1;
                        }
                    }
                }
                if (!ok) break;
                umma2_commit_both(b_tfull + 8 * acc);  // accumulators ready for both epilogues
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            }
            if (!ok) give_up();
            // all issued MMAs complete before TMEM is released
            umma2_commit_own(b_done);
            mbar_wait(b_done, 0, nullptr);
        }
    } else if (run) {
        // ------------------------------------------------ epilogue (warps 2..17, both CTAs)
        // The accumulator holds this CTA's two tiles (2R + t, 2C + rank),
        // t = 0, 1, transposed: TMEM lane = output column j, TMEM column t *
        // 128 + (row i within the tile).  Warp e = warp - 2 reads lane quarter
        // q = warp % 4 (the quarter a warp may access), so each thread owns
        // one column j, and takes the 16-row chunks c = grp + NG u (grp = e /
        // 4, NG = NEPI / 4 warps per quarter) of each tile's 8.  The next
        // chunk's TMEM load is in flight while the current one is processed;
        // the next tile's norms are fetched while the current tile is stored.
        // A tile above the diagonal (the odd CTA's upper tile of a diagonal
        // unit) or below the last row block is computed but not read.
        constexpr int NG = NEPI / 4;                // warps per TMEM lane quarter
        constexpr int NCH = TILE / EPI_ROWS / NG;   // 16-row chunks per warp and tile
        const uint32_t e = warp - 2, q = warp & 3, grp = e >> 2;
        float *snorm = epi + e * NORM_FLOATS;     // norms of this warp's rows, two buffers
        const float tau = g.tau;
        // next tile's norms: lane l holds the norms of row l % 16 of chunks
        // u = 2v + l / 16 (16 rows each) and of its own column
        float pfr[NCH / 2], pfj = 0.0f;
        auto prefetch = [&](uint32_t a, uint32_t b) {  // row block a, column block b
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
            if (lane == 0) give_up();
        };
        unsigned long long cur;
        if (!tq_pop_warp(k++, cur)) {
            fail();
            cur = TQ_END;
        }
        if (cur != TQ_END) prefetch(2 * (uint32_t)(cur >> 32), 2 * (uint32_t)cur + rank);
        for (;;) {
            // this unit's accumulators; the row group goes on only if each of
            // its warps has the unit and its accumulators (after the last
            // unit, or after a failed wait anywhere, all four stop together)
            const bool have = cur != TQ_END;
            const bool got = have && warp_wait<true>(b_tfull + 8 * acc, acc_phase, &s_abort, wl);
            if (have && !got) fail();
            if (!named_sync_all(1 + grp, 128, got)) break;
            const uint32_t R = (uint32_t)(cur >> 32), bj = 2 * (uint32_t)cur + rank;
            unsigned long long nxt = TQ_END;
            tc_fence_after();
#pragma unroll 1
            for (uint32_t t = 0; t < 2; ++t) {
                const uint32_t bi = 2 * R + t;
                const bool valid = bj <= bi && bi < g.m;
                float *rn = snorm + nbuf * 32;  // this tile's row norms: [chunk u][16]
#pragma unroll
                for (int v = 0; v < NCH / 2; ++v) rn[32 * v + lane] = pfr[v];
                const float nj = pfj;
                __syncwarp();
                if (t == 0) {
                    prefetch(bi + 1, bj);
                } else if (!tq_pop_warp(k++, nxt)) {
                    fail();  // the group stops at the next unit's vote
                    nxt = TQ_END;
                } else if (nxt != TQ_END) {
                    prefetch(2 * (uint32_t)(nxt >> 32), 2 * (uint32_t)nxt + rank);
                }
                if (valid) {
                    const uint32_t j = bj * TILE + q * 32 + lane;  // this thread's column
                    const uint32_t taddr = tmem + ((q * 32) << 16) + acc * (2 * TILE) + t * TILE;
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
                        // Direct stores: for each row the warp's 32 lanes hold 32
                        // consecutive packed entries, written by one 128-byte store.
                        // The row group's four warps hold the four quarters of the
                        // same 16 rows; a barrier before their stores keeps them
                        // writing the same rows at the same time, so the partly
                        // written 32-byte sectors at the quarters' edges meet in L2
                        // soon after each other (BF16X6, N = 65536, d = 128: 2.24 ms
                        // with one barrier per unit, 2.19 per tile, 2.09 per 16
                        // rows, 2.09 per 8, 2.14 per 4).  Staging whole row segments
                        // through shared memory competes with the tensor core's
                        // operand reads: BF16X6 2.51 ms, BF16X3 2.42 ms against
                        // 1.95 ms direct; assembling only the 32-byte sectors that
                        // straddle two quarters of a row, 2.63 ms.
                        named_sync(1 + grp, 128);
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
                nbuf ^= 1;
            }
            tc_fence_before();
            if (lane == 0) mbar_arrive_cl(L_tempty + 8 * acc);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1;
            }
            cur = nxt;
        }
    }
    // neither CTA releases its TMEM or exits while the other (or the even
    // CTA's MMAs and copies) may still use its shared memory or accumulators
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// -------------------------------------------------------------- fixup ----
// FP64 direct-difference recompute of the flagged pairs appended since the
// previous call (list entries [*start, count); all of them when start is
// null).  If the list overflowed, every pair of the packed range [p_begin,
// p_end) whose stored distance passes a slightly wider version of the flag
// test is recomputed instead.  next_start (if not null) receives the count,
// for the next call.
__global__ void fixup_kernel(const float *__restrict__ x, uint32_t d, float *__restrict__ out,
                             const float *__restrict__ norms, const unsigned long long *__restrict__ count,
                             const unsigned long long *__restrict__ list, unsigned long long cap, float tau,
                             unsigned long long *n_flagged, const unsigned long long *start,
                             unsigned long long *next_start, uint64_t p_begin, uint64_t p_end)
{
    const unsigned long long cnt = *count, first = start ? *start : 0ull;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (uint64_t)gridDim.x * blockDim.x;
    if (tid == 0 && n_flagged) *n_flagged = cnt;
    if (tid == 0 && next_start) *next_start = cnt;
    // by one thread: four independent partial sums, so the loads of
    // consecutive features overlap
    auto recompute = [&](uint32_t i, uint32_t j) {
        const float *xi = x + (size_t)i * d, *xj = x + (size_t)j * d;
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        uint32_t k = 0;
        for (; k + 4 <= d; k += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double df = (double)xi[k + u] - (double)xj[k + u];
                s[u] = fma(df, df, s[u]);
            }
        for (; k < d; ++k) {
            const double df = (double)xi[k] - (double)xj[k];
            s[0] = fma(df, df, s[0]);
        }
        out[T2(i) + j] = (float)sqrt((s[0] + s[1]) + (s[2] + s[3]));
    };
    if (cnt <= cap) {
        // one warp per listed pair: lanes take strided features, then a fixed-order tree sum
        const uint32_t lane = threadIdx.x & 31;
        for (uint64_t e = first + (tid >> 5); e < cnt; e += nth >> 5) {
            const unsigned long long v = list[e];
            const uint32_t i = (uint32_t)(v >> 32), j = (uint32_t)(v & 0xFFFFFFFFu);
            const float *xi = x + (size_t)i * d, *xj = x + (size_t)j * d;
            double s = 0.0;
            for (uint32_t k = lane; k < d; k += 32) {
                const double df = (double)xi[k] - (double)xj[k];
                s = fma(df, df, s);
            }
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) out[T2(i) + j] = (float)sqrt(s);
        }
    } else {
        const float wide = 1.0625f * tau;
        for (uint64_t p = p_begin + tid; p < p_end; p += nth) {
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
    const size_t fixed = 1024 /*align*/ + NEPI * NORM_FLOATS * 4 + 8 * (7 + 2 * MAX_STAGES);
    const size_t a = (size_t)p.P * p.nkc * CHUNK_BYTES, st = CHUNK_BYTES;  // one row block per CTA
    if (fixed + a + 2 * st > (size_t)SMEM_LIMIT) return false;
    p.stages = (uint32_t)std::min<size_t>(MAX_STAGES, (SMEM_LIMIT - fixed - a) / st);
    p.smem = fixed + a + p.stages * st;
    return true;
}

// Launches the pair kernel on as many CTA pairs as can be resident at once
// (cached per instantiation and shared-memory size), splitting the units into
// an up-front run per pair and counter-driven runs.
template <int MP, int PP>
cudaError_t launch_gram(const CUtensorMap &tmap, GramArgs g, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(gram_kernel<MP, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static int cached_dev = -1, cached_pairs = 0;
    static size_t cached_smem = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    std::unique_lock<std::mutex> lock(mu);
    if (cached_dev != dev || cached_smem != smem) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (num_sms() / 2));
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, gram_kernel<MP, PP>, &cfg) != cudaSuccess || ncl < 1) {
            (void)cudaGetLastError();
            ncl = (int)(num_sms() / 2);
        }
        cached_dev = dev;
        cached_smem = smem;
        cached_pairs = ncl;
    }
    const int npairs = cached_pairs;
    lock.unlock();
    const uint64_t units = g.nunits - g.u0;
    const uint64_t pairs = std::min<uint64_t>((uint64_t)(npairs > 0 ? npairs : 1), units);
    g.static_per = units * STATIC_PCT / 100 / pairs;
    g.dyn_start = g.u0 + g.static_per * pairs;
    g.chunk = DYN_CHUNK;
    gram_kernel<MP, PP><<<(unsigned)(2 * pairs), NTHREADS, smem, s>>>(tmap, g);
    return cudaGetLastError();
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

namespace {

// Unit rows [R0, R1) of the Gram kernel, whose output is the packed rows
// [256 R0, min(n, 256 R1)).
int gram_range(uint32_t n, uint32_t d, float *out, int map, int prec, void *workspace, size_t ws_bytes, uint32_t R0,
               uint32_t R1, cudaStream_t s)
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
    const uint32_t m = (n + TILE - 1) / TILE, mb = (m + 1) / 2;
    if (R1 > mb) R1 = mb;
    if (R0 >= R1) return TRI_OK;
    // units: 2 x 2 tile blocks, lambda over the mb-row triangle or the mb x mb box
    const uint64_t u0 = map == TRI_MAP_LAMBDA ? T2(R0) : (uint64_t)R0 * mb;
    const uint64_t nunits = map == TRI_MAP_LAMBDA ? T2(R1) : (uint64_t)R1 * mb;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return TRI_ECUDA;
    char *ws = (char *)workspace;
    // 128-row blocks of the planes (row blocks and column blocks alike)
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
    g.mb = mb;
    g.u0 = u0;
    g.nunits = nunits;
    g.stages = pl.stages;
    g.tau = flag_tau(prec, d);
    g.norms = (const float *)(ws + L.norms);
    g.out = out;
    g.flag_count = (unsigned long long *)(ws + L.hdr);
    g.status = (int *)(ws + L.hdr + 8);
    g.tile_counter = (unsigned long long *)(ws + L.hdr + 16);
    g.wait_limit = (const unsigned long long *)(ws + L.hdr + 40);
    g.flag_list = (unsigned long long *)(ws + L.flags);
    g.flag_cap = L.cap;
    if (cudaMemsetAsync(g.tile_counter, 0, sizeof(unsigned long long), s) != cudaSuccess) return TRI_ECUDA;
    cudaError_t e;
    if (map == TRI_MAP_LAMBDA)
        e = pl.P == 3 ? launch_gram<MAP_LAMBDA, 3>(tmap, g, pl.smem, s) : launch_gram<MAP_LAMBDA, 2>(tmap, g, pl.smem, s);
    else
        e = pl.P == 3 ? launch_gram<MAP_BB, 3>(tmap, g, pl.smem, s) : launch_gram<MAP_BB, 2>(tmap, g, pl.smem, s);
    return e == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

}  // namespace

extern "C" int tri_edm_gram(uint32_t n, uint32_t d, float *out, int map, int prec, void *workspace, size_t ws_bytes,
                            void *stream)
{
    if (n == 0) return TRI_EINVAL;
    const uint32_t mb = ((n + TILE - 1) / TILE + 1) / 2;
    return gram_range(n, d, out, map, prec, workspace, ws_bytes, 0, mb, (cudaStream_t)stream);
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
    fixup_kernel<<<num_sms() * 4, 256, 0, s>>>(x, d, out, (const float *)(ws + L.norms),
                                               (const unsigned long long *)(ws + L.hdr),
                                               (const unsigned long long *)(ws + L.flags), L.cap,
                                               flag_tau(prec, d), n_flagged, nullptr, nullptr, 0,
                                               T2(n));
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

// ------------------------------------------------------ split over ranks ----
// One triangle split across processes (one per GPU): rank r computes a band
// of whole unit rows (256 rows each, the Gram kernel's unit) whose packed
// entries form one contiguous range of the output, so the ranks need no
// exchange while they compute.  Band edges are placed at equal shares of the
// n(n+1)/2 pairs: rank r's band starts at the first unit row whose packed
// offset reaches r/ranks of the total.

extern "C" int tri_edm_partition(uint32_t n, uint32_t ranks, uint32_t rank, uint32_t *row_begin, uint32_t *row_end,
                                 uint64_t *pair_begin, uint64_t *pair_end)
{
    if (!row_begin || !row_end || !pair_begin || !pair_end || ranks == 0 || rank >= ranks) return TRI_EINVAL;
    if (n > TC_MAX_N) return TRI_ERANGE;
    const uint32_t unit = 2 * TILE, mb = (n + unit - 1) / unit;
    const uint64_t total = T2(n);
    // first unit row R whose start T2(min(n, 256 R)) is at least share k of the pairs
    auto edge = [&](uint32_t k) -> uint32_t {
        if (k >= ranks) return mb;
        const long double target = (long double)total * k / ranks;
        uint32_t lo = 0, hi = mb;  // smallest R in [0, mb] with T2(min(n, unit R)) >= target
        while (lo < hi) {
            const uint32_t mid = (lo + hi) / 2;
            if ((long double)T2(std::min<uint64_t>(n, (uint64_t)unit * mid)) >= target) hi = mid;
            else lo = mid + 1;
        }
        return lo;
    };
    const uint32_t R0 = edge(rank), R1 = edge(rank + 1);
    *row_begin = (uint32_t)std::min<uint64_t>(n, (uint64_t)unit * R0);
    *row_end = (uint32_t)std::min<uint64_t>(n, (uint64_t)unit * R1);
    *pair_begin = T2(*row_begin);
    *pair_end = T2(*row_end);
    return TRI_OK;
}

extern "C" int tri_edm_rows(const float *x, uint32_t n, uint32_t d, uint32_t row_begin, uint32_t row_end,
                            float *out_band, int map, int prec, void *workspace, size_t ws_bytes,
                            unsigned long long *n_flagged, void *stream)
{
    if (!x || !out_band || n == 0 || d == 0) return TRI_EINVAL;
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_BB) return TRI_EINVAL;
    if (n > TC_MAX_N) return TRI_ERANGE;
    const uint32_t unit = 2 * TILE;
    if (row_begin > row_end || row_end > n) return TRI_EINVAL;
    if (row_begin < row_end && (row_begin % unit != 0 || (row_end % unit != 0 && row_end != n))) return TRI_EINVAL;
    if ((uintptr_t)out_band & 15) return TRI_EINVAL;
    TcPlan pl;
    if (!plan(d, prec, pl)) return TRI_ERANGE;
    const WsLayout L = ws_layout(n, d, prec);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 255)) return TRI_ENOSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int r = tri_edm_prepare(x, n, d, prec, workspace, ws_bytes, s);
    if (r != TRI_OK || row_begin == row_end) return r;
    // The kernels index the whole packed triangle; the band's first entry,
    // T2(row_begin) = 128 R0 (256 R0 + 1), is a multiple of 128, so the
    // shifted base keeps out_band's 16-byte alignment.
    const uint64_t p0 = T2(row_begin), p1 = T2(row_end);
    float *base = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(out_band) - p0 * sizeof(float));
    if ((r = gram_range(n, d, base, map, prec, workspace, ws_bytes, row_begin / unit,
                        (row_end + unit - 1) / unit, s)) != TRI_OK)
        return r;
    char *ws = (char *)workspace;
    fixup_kernel<<<num_sms() * 4, 256, 0, s>>>(x, d, base, (const float *)(ws + L.norms),
                                               (const unsigned long long *)(ws + L.hdr),
                                               (const unsigned long long *)(ws + L.flags), L.cap, flag_tau(prec, d),
                                               n_flagged, nullptr, nullptr, p0, p1);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ECUDA;
}

// ---------------------------------------------------------------- host ----
namespace {

// One non-blocking copy stream per device for tri_edm_host's device-to-host copies.
cudaStream_t copy_stream()
{
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

}  // namespace

extern "C" int tri_edm_host(const float *x_host, uint32_t n, uint32_t d, float *out_host, int map, int prec,
                            uint32_t bands, float *x_dev, float *out_dev, void *workspace, size_t ws_bytes,
                            unsigned long long *n_flagged, void *stream)
{
    if (!x_host || !out_host || !x_dev || !out_dev || n == 0 || d == 0) return TRI_EINVAL;
    if (prec != TRI_BF16X3 && prec != TRI_BF16X6) return TRI_EINVAL;
    if (map != TRI_MAP_LAMBDA && map != TRI_MAP_BB) return TRI_EINVAL;
    if (n > TC_MAX_N) return TRI_ERANGE;
    TcPlan pl;
    if (!plan(d, prec, pl)) return TRI_ERANGE;
    const WsLayout L = ws_layout(n, d, prec);
    if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 255)) return TRI_ENOSPACE;
    if ((uintptr_t)out_dev & 15) return TRI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream, cs = copy_stream();
    if (!cs) return TRI_ECUDA;
    const uint32_t m = (n + TILE - 1) / TILE, mb = (m + 1) / 2;
    const uint64_t total = T2(n);
    // bands of about 512 MB of output each (equal areas: unit-row edges ~ mb sqrt(k / B))
    if (bands == 0) bands = (uint32_t)std::min<uint64_t>(16, std::max<uint64_t>(1, total * 4 / (512ull << 20)));
    bands = std::min(bands, mb);
    char *ws = (char *)workspace;
    unsigned long long *slot = (unsigned long long *)(ws + L.hdr + 24);  // two list-start slots
    if (cudaMemcpyAsync(x_dev, x_host, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TRI_ECUDA;
    int r = tri_edm_prepare(x_dev, n, d, prec, workspace, ws_bytes, s);  // also zeroes both slots
    if (r != TRI_OK) return r;
    bool queued = false;  // a copy is on the copy stream: the caller's stream must wait for it, error or not
    uint32_t R0 = 0;
    for (uint32_t b = 0; b < bands && r == TRI_OK; ++b) {
        uint32_t R1 = b + 1 == bands ? mb : (uint32_t)std::ceil(mb * std::sqrt((double)(b + 1) / bands));
        R1 = std::min(std::max(R1, R0 + 1), mb);
        if (R0 >= mb) break;
        if ((r = gram_range(n, d, out_dev, map, prec, workspace, ws_bytes, R0, R1, s)) != TRI_OK) break;
        const uint64_t p0 = T2(std::min<uint64_t>(n, 2ull * TILE * R0)), p1 = T2(std::min<uint64_t>(n, 2ull * TILE * R1));
        fixup_kernel<<<num_sms() * 4, 256, 0, s>>>(x_dev, d, out_dev, (const float *)(ws + L.norms),
                                                   (const unsigned long long *)(ws + L.hdr),
                                                   (const unsigned long long *)(ws + L.flags), L.cap,
                                                   flag_tau(prec, d), n_flagged, slot + (b & 1),
                                                   slot + ((b + 1) & 1), p0, p1);
        if (cudaGetLastError() != cudaSuccess) {
            r = TRI_ECUDA;
            break;
        }
        // the band's rows are final: copy them while the next band computes
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            r = TRI_ECUDA;
            break;
        }
        cudaError_t e = cudaEventRecord(ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
        cudaEventDestroy(ev);
        if (e == cudaSuccess && p1 > p0) {
            e = cudaMemcpyAsync(out_host + p0, out_dev + p0, (p1 - p0) * sizeof(float), cudaMemcpyDeviceToHost, cs);
            queued = queued || e == cudaSuccess;
        }
        if (e != cudaSuccess) r = TRI_ECUDA;
        R0 = R1;
    }
    if (!queued) return r;
    // the caller's stream completes only after the last copy (also after an
    // error, so that the caller may free or reuse the buffers once it has
    // synchronised its stream)
    cudaEvent_t done;
    cudaError_t e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        e = cudaEventRecord(done, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, done, 0);
        cudaEventDestroy(done);
    }
    if (e != cudaSuccess) {
        // cannot order the streams: wait for the copies here instead
        cudaStreamSynchronize(cs);
        if (r == TRI_OK) r = TRI_ECUDA;
    }
    return r;
}
