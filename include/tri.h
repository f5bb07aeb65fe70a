/*
 * tri.h -- C ABI of libtri.so: GPU kernels on triangular and tetrahedral
 * domains whose grids are mapped onto the domain by the block-space map
 * lambda(omega) of Navarro, Bustos and Hitschfeld, "A Non-linear GPU Thread
 * Map for Triangular Domains" (arXiv 1609.01490), with the bounding-box,
 * rectangular-box, recursive-partition and upper-triangular maps of its
 * Section 4.2 as comparison kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named as device pointers must point to memory of the current
 *    CUDA device; the caller owns all of it.  No entry point allocates device
 *    memory.  Those that need scratch take a caller-provided `workspace` of at
 *    least the size the matching *_workspace_size call reports.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every launch is asynchronous on it; results are ready when the
 *    stream is synchronised.
 *  - The return value is a tri_status.  It reports argument errors (checked
 *    on the host before anything is launched) and launch errors.  Errors the
 *    kernels detect on the device are written to device status words named in
 *    the individual calls.
 *  - Packed triangles are row-major lower triangles with the diagonal:
 *    element (i, j), 0 <= j <= i < n, lives at offset i(i+1)/2 + j
 *    (Eq. eq_matrix_indexing of Section 3.1 applied to elements), 64-bit.
 *  - rho is the number of threads per block side (Section 3.1: blocks of
 *    rho x rho threads); accepted values are 8, 16 and 32.
 */
#ifndef TRI_H
#define TRI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TRI_API __attribute__((visibility("default")))
#else
#define TRI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TRI_OK = 0,
    TRI_EINVAL = 1,    /* null pointer, unsupported rho/tile/enum value, zero size */
    TRI_ERANGE = 2,    /* domain too large for the map (e.g. more than 2^32 blocks),
                          or a size the map cannot cover (REC with a block count that
                          is not a power of two) */
    TRI_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    TRI_EOVERFLOW = 4, /* a bounded device list overflowed (reported through the
                          device status of the call) */
    TRI_ETIMEOUT = 5,  /* a bounded device wait gave up */
    TRI_ENOSPACE = 6   /* workspace smaller than the size query reports */
} tri_status;

/* Block-space and thread-space maps (Sections 3 and 4.2). */
typedef enum {
    TRI_MAP_LAMBDA = 0,        /* lambda(omega), Eq. eq_gmap, 1-D (or 2-D beyond
                                  2^31 - 1 blocks) grid of exactly m(m+1)/2 blocks */
    TRI_MAP_BB = 1,            /* bounding box: m x m blocks, blocks above the
                                  diagonal discarded (Section 4.2) */
    TRI_MAP_RB = 2,            /* rectangular box: upper part folded under the
                                  diagonal, ceil((m+1)/2) x m blocks (Section 4.2) */
    TRI_MAP_REC = 3,           /* recursive partition: one diagonal pass plus one
                                  launch per level; m must be a power of two */
    TRI_MAP_UTM = 4,           /* upper-triangular map of Avril et al., thread space
                                  (Section 4.2) */
    TRI_MAP_LAMBDA_PDELTA = 5, /* lambda(omega) on the balanced m' x m' grid P_Delta,
                                  m' = ceil(sqrt(m(m+1)/2)) (Section 3.1) */
    TRI_MAP_TET_TABLE = 6      /* tetrahedral calls only: lambda with the layer
                                  found in a table of layer starts (Section 7) */
} tri_map;

/* Square-root estimate inside lambda (Section 4.1).  Every variant is followed
 * by an exact integer correction, so all three give identical maps. */
typedef enum {
    TRI_SQRT_X = 0, /* sqrtf(x)                                   (lambda_X) */
    TRI_SQRT_R = 1, /* x * rsqrtf(x)                              (lambda_R) */
    TRI_SQRT_N = 2  /* x * y, y = 1/sqrt(x) by three Newton steps from the
                       0x5f3759df seed (Lomont)                   (lambda_N) */
} tri_sqrt;

typedef enum {
    TRI_FP32 = 0,   /* direct differences in FP32 on CUDA cores */
    TRI_BF16X3 = 1, /* Gram form on tcgen05 tensor cores: hi/lo BF16 split,
                       3 products, FP32 accumulation, FP64 recompute of flagged pairs */
    TRI_BF16X6 = 2  /* Gram form on tcgen05: hi/mid/lo BF16 split, 6 products,
                       FP32 accumulation, FP64 recompute of flagged pairs */
} tri_prec;

typedef enum {
    TRI_BODY_DUMMY = 0,    /* every mapped thread stores i+j to out[0] (Section 4.1's
                              dummy kernel) */
    TRI_BODY_SENTINEL = 1, /* stores only if i+j == 0xFFFFFFFF (never), so the time
                              is the map alone */
    TRI_BODY_COUNT = 2     /* atomically increments out[index(i,j)]: a coverage test */
} tri_body;

/* Human-readable name of a tri_status value (static storage). */
TRI_API const char *tri_status_string(int status);

/* Library version, major*10000 + minor*100 + patch. */
TRI_API int tri_version(void);

/*
 * tri_map_launch -- run one map over the element domain of size n.
 *   Section 3.1 (lambda, Eq. eq_gmap / eq_theorem_nodiag), Section 4.1 (dummy
 *   kernel, square-root variants), Section 4.2 (BB, RB, REC, UTM).
 *   with_diag = 1: domain {0 <= j <= i < n}; with_diag = 0: {0 <= j < i < n}
 *   (lambda then uses the strict form, Eq. eq_theorem_nodiag).
 *   out (device, uint32): DUMMY/SENTINEL one word; COUNT n(n+1)/2 (with_diag)
 *   or n(n-1)/2 counters, index i(i+1)/2 + j or i(i-1)/2 + j; the caller zeroes
 *   them first.  sqrt_kind is used by the lambda maps only.
 *   Errors: TRI_EINVAL (null out, bad enum, rho not 8/16/32, n = 0),
 *   TRI_ERANGE (more than 2^32 - 1 blocks or threads; REC with ceil(n/rho) not
 *   a power of two), TRI_ECUDA.
 */
TRI_API int tri_map_launch(int map, int sqrt_kind, uint32_t n, uint32_t rho, int with_diag,
                   int body, uint32_t *out, void *stream);

/*
 * tri_lambda_verify -- evaluate lambda (Eq. eq_gmap, or Eq. eq_theorem_nodiag
 * when with_diag = 0) for every omega in [w_begin, w_end), w_end <= 2^32,
 * one thread per omega, and check each result against the exact row
 * invariant T(i) <= omega < T(i+1), 0 <= j <= i (strict form: T(i-1) <= omega
 * < T(i), 0 <= j < i), with T(i) = i(i+1)/2 in 64-bit integers.
 *   result (device, 6 x uint64, zeroed by the caller) accumulates, modulo
 *   2^64: [0] violations, [1] sum i, [2] sum j, [3] sum i*i, [4] sum j*j,
 *   [5] sum i*j.
 *   Errors: TRI_EINVAL, TRI_ERANGE (w_end > 2^32 or w_begin > w_end), TRI_ECUDA.
 */
TRI_API int tri_lambda_verify(int sqrt_kind, int with_diag, uint64_t w_begin, uint64_t w_end,
                      unsigned long long *result, void *stream);

/*
 * tri_peak_probe -- arithmetic peak probe for the ALU rooflines (not in the
 * paper): `blocks` blocks of 256 threads, each thread running 8 independent
 * chains of `iters` fused multiply-adds: kind 0 FP32 (fma.rn.f32), 1 FP32 in
 * two-lane form (fma.rn.f32x2, two results per instruction), 2 FP64.  The
 * caller times the launch on its stream; *flop (host) receives the floating-
 * point operations launched (2 per result).  sink (device FP32, blocks x 256)
 * receives one value per thread so that the chains are kept.
 *   Errors: TRI_EINVAL, TRI_ECUDA.
 */
TRI_API int tri_peak_probe(int kind, uint32_t blocks, uint32_t iters, float *sink, double *flop, void *stream);

/*
 * tri_map_first_error -- where the printed formulas, taken without the exact
 * integer correction this library applies, first give a wrong result:
 *   map = TRI_MAP_LAMBDA: for every omega in [begin, end) (end <= 2^32), the
 *     row floor(e + eps - 1/2), e the FP32 estimate sqrt_kind of
 *     sqrt(2 omega + 1/4), eps = 1e-4 for TRI_SQRT_N and TRI_SQRT_R and 0 for
 *     TRI_SQRT_X (Section 4.1), against the exact row (n_items unused);
 *   map = TRI_MAP_UTM: for every thread k in [begin, end) of n_items items
 *     (2 <= n_items <= 2^31, end <= n_items (n_items - 1) / 2), the pair (a, b)
 *     of the formula of Section 4.2 with its square root argument and a in
 *     FP32, against the exact pair (sqrt_kind unused but checked).
 *   first_bad (device uint64, set by the caller, e.g. to UINT64_MAX): lowered
 *   atomically to the smallest failing omega or k in the range.
 *   Errors: TRI_EINVAL (null first_bad, begin > end, bad map or sqrt_kind),
 *   TRI_ERANGE (range limits above, or more than 2^31 - 1 blocks of 256
 *   threads in one call), TRI_ECUDA.
 */
TRI_API int tri_map_first_error(int map, int sqrt_kind, uint64_t n_items, uint64_t begin, uint64_t end,
                                unsigned long long *first_bad, void *stream);

/*
 * tri_edm -- Euclidean distance matrix over i >= j (Section 5, test 2):
 *   out[i(i+1)/2 + j] = sqrt(sum_k (x[i][k] - x[j][k])^2), the diagonal 0.
 *   x (device, FP32) row-major [n][d]; out (device, FP32) n(n+1)/2 entries.
 *   prec = TRI_FP32: blocks of rho x rho threads, each thread reg x reg pairs
 *   (reg in {1, 2, 4, 8}, 8 only with rho <= 16; 0 picks 4); each block covers
 *   an S x S pair tile, S = rho*reg, placed by `map` (any tri_map).  For reg
 *   >= 2 a thread updates two adjacent columns per f32x2 instruction.  No
 *   workspace.
 *   prec = TRI_BF16X3 / TRI_BF16X6: 2 x 2 blocks of 128 x 128 pair tiles per
 *   CTA pair on tcgen05 tensor cores (cta_group::2), placed by
 *   TRI_MAP_LAMBDA or TRI_MAP_BB; rho and reg are ignored;
 *   needs `workspace` of tri_edm_workspace_size bytes (256-byte aligned).
 *   Pairs whose Gram estimate of d^2 falls below tau*(|x_i|^2 + |x_j|^2) are
 *   recomputed in FP64 by direct differences (BF16X6: tau = (2 + 24 c)
 *   2^-23 / 1.96e-5 for c = ceil(d / 64) K chunks, which bounds every other
 *   distance's relative error by 1e-5; BF16X3: tau = 0.0625, no bound); n_flagged (device uint64,
 *   may be NULL) receives how many were flagged.  If more were flagged than
 *   the workspace list holds, the recompute pass scans the whole triangle
 *   instead (slower, same result).
 *   Errors: TRI_EINVAL (null pointers, d = 0, bad enum/rho/reg, n = 0),
 *   TRI_ERANGE (too many blocks for the map), TRI_ENOSPACE, TRI_ECUDA.
 */
TRI_API int tri_edm(const float *x, uint32_t n, uint32_t d, float *out, int map, uint32_t rho,
            uint32_t reg, int prec, void *workspace, size_t ws_bytes,
            unsigned long long *n_flagged, void *stream);

/* Workspace bytes tri_edm needs for (n, d, prec); 0 for TRI_FP32. */
TRI_API int tri_edm_workspace_size(uint32_t n, uint32_t d, int prec, size_t *bytes);

/*
 * The three phases of tri_edm for prec = TRI_BF16X3 / TRI_BF16X6, callable on
 * their own (same stream, in this order) to time them or to reuse prepared
 * operands.  workspace: tri_edm_workspace_size bytes, 256-byte aligned.
 * Tensor-core limits: n <= 92681 (packed triangle below 2^32 entries),
 * d <= 192 for BF16X6 and d <= 320 for BF16X3 (the split planes of one row
 * block stay resident in shared memory beside at least two 16 KB operand
 * stages); larger sizes give TRI_ERANGE.
 *
 *   tri_edm_prepare: clears the workspace header, then writes the FP32 row
 *     norms |x_i|^2 (summed to ~48 bits as FP32 pairs) and the BF16 split
 *     planes (hi, lo or hi, mid, lo; K zero-padded to a multiple of 64).
 *   tri_edm_gram: tensor-core Gram term, d^2 = |x_i|^2 + |x_j|^2 - 2 x_i.x_j,
 *     clamped at 0, square root stored to out (packed, FP32); pairs with
 *     d^2 < tau (|x_i|^2 + |x_j|^2) appended to the workspace's flag list.
 *     map: TRI_MAP_LAMBDA (2 x 2 blocks of tiles in lambda order) or
 *     TRI_MAP_BB.  Runs as clusters of two CTAs (tcgen05 cta_group::2).  A
 *     device wait that exceeds 2 s sets the workspace status word (int at
 *     byte 8) to TRI_ETIMEOUT; both CTAs of the pair then stop, wait for
 *     their copies and MMAs in flight, free their tensor memory and return.
 *     The workspace's uint64 at byte 40 (cleared by tri_edm_prepare) sets a
 *     shorter limit, in ns, for the waits between the kernel's roles; it
 *     exists so that tests can make those waits run out.  If the two CTAs of
 *     a pair cannot share their tensor-memory address the word becomes
 *     TRI_ECUDA and the pair does no work.
 *   tri_edm_fixup: recomputes the flagged pairs in FP64 by direct differences
 *     (or, when the list overflowed, every pair whose stored distance passes a
 *     slightly wider flag test) and writes the flag count to *n_flagged
 *     (device uint64, may be NULL).
 */
TRI_API int tri_edm_prepare(const float *x, uint32_t n, uint32_t d, int prec, void *workspace,
                            size_t ws_bytes, void *stream);
TRI_API int tri_edm_gram(uint32_t n, uint32_t d, float *out, int map, int prec, void *workspace,
                         size_t ws_bytes, void *stream);
TRI_API int tri_edm_fixup(const float *x, uint32_t n, uint32_t d, float *out, int prec, void *workspace,
                          size_t ws_bytes, unsigned long long *n_flagged, void *stream);

/*
 * End-to-end EDM from and to host memory (not in the paper, which starts
 * from device-resident points): copies x_host (n x d FP32, row-major) to
 * x_dev, runs tri_edm_prepare, then computes the packed triangle in `bands`
 * row bands (Gram term + FP64 recompute of the band's flagged pairs) and
 * copies each finished band from out_dev to out_host on a library-owned
 * copy stream while the next band computes, so the device-to-host copy (the
 * bound of this call on a host attached through NVLink-C2C) overlaps the
 * compute.  bands = 0 picks about 512 MB of output per band (1 to 16).
 * prec: TRI_BF16X3 or TRI_BF16X6; map: TRI_MAP_LAMBDA or TRI_MAP_BB.
 * x_dev (n*d floats), out_dev (n(n+1)/2 floats, 16-byte aligned) and the
 * workspace (tri_edm_workspace_size bytes, 256-byte aligned) are device
 * buffers owned by the caller.  Host buffers should be pinned for the copies
 * to run asynchronously.  The call enqueues the work and returns: `stream`
 * completes after the last copy, so synchronise it before reading out_host.
 * out_host and out_dev hold the same triangle as tri_edm's out.
 * Errors: TRI_EINVAL (null pointer, zero size, bad map or prec, unaligned
 * out_dev), TRI_ERANGE / TRI_ENOSPACE as tri_edm, TRI_ECUDA.  After an error
 * in a later band, `stream` still completes only after the copies already
 * queued, so the buffers may be reused once the stream is synchronised.
 */
TRI_API int tri_edm_host(const float *x_host, uint32_t n, uint32_t d, float *out_host, int map, int prec,
                         uint32_t bands, float *x_dev, float *out_dev, void *workspace, size_t ws_bytes,
                         unsigned long long *n_flagged, void *stream);

/*
 * One EDM split across processes, one per GPU (the row order of Section 3's
 * enumeration matrix makes each band of rows one contiguous range of the
 * packed output, so the ranks compute without exchanging anything).
 *
 *   tri_edm_partition: host only, no device work.  The rows [*row_begin,
 *     *row_end) and the packed entries [*pair_begin, *pair_end) =
 *     [T(row_begin), T(row_end)), T(i) = i(i+1)/2, that rank `rank` of
 *     `ranks` computes: bands of whole 256-row unit rows (the tensor-core
 *     kernel's unit of work), the band of rank r starting at the first unit
 *     row whose packed offset reaches r/ranks of the n(n+1)/2 pairs.  The
 *     bands are disjoint and cover the triangle in rank order; a rank may
 *     get an empty band when n is small.  Errors: TRI_EINVAL (null pointer,
 *     ranks = 0, rank >= ranks), TRI_ERANGE (n > 92681).
 *   tri_edm_rows: the tensor-core EDM (prec TRI_BF16X3 or TRI_BF16X6, map
 *     TRI_MAP_LAMBDA or TRI_MAP_BB) of the rows [row_begin, row_end) only,
 *     with row_begin a multiple of 256 and row_end a multiple of 256 or n:
 *     x (device) holds all n points (every row pairs with all columns j <= i);
 *     out_band (device, 16-byte aligned, T(row_end) - T(row_begin) floats)
 *     receives the packed entries T(row_begin) .. T(row_end) - 1 from its
 *     first element on, the same values as tri_edm writes there.  Runs
 *     tri_edm_prepare, the Gram kernel over the band's units and the FP64
 *     recompute of the band's flagged pairs; workspace and n_flagged as
 *     tri_edm.  Errors as tri_edm; TRI_EINVAL also for a band not on unit
 *     rows.
 */
TRI_API int tri_edm_partition(uint32_t n, uint32_t ranks, uint32_t rank, uint32_t *row_begin, uint32_t *row_end,
                              uint64_t *pair_begin, uint64_t *pair_end);
TRI_API int tri_edm_rows(const float *x, uint32_t n, uint32_t d, uint32_t row_begin, uint32_t row_end,
                         float *out_band, int map, int prec, void *workspace, size_t ws_bytes,
                         unsigned long long *n_flagged, void *stream);

/*
 * tri_edm_batched -- many EDM triangles of uneven size in one persistent
 * launch (lambda applied to each instance's own block numbers, found from
 * an exclusive prefix sum of the per-instance block counts m_k(m_k+1)/2).
 *   x_cat (device FP32): the instances' points, row-major, concatenated;
 *   pt_off (device uint64 [count]): first row of instance k in x_cat;
 *   n_k (device uint32 [count]): points in instance k (0 allowed);
 *   out_cat (device FP32) / out_off (device uint64 [count]): instance k's
 *   packed triangle starts at out_cat + out_off[k].
 *   rho in {8,16,32}, reg in {1,2,4,8} as in tri_edm (FP32 direct differences).
 *   workspace: tri_edm_batched_workspace_size bytes, 16-byte aligned (a
 *   status word, a tile counter and the block offsets; the call clears the
 *   first 16 bytes itself).  Issues a 16-byte memset and two kernels and no
 *   host synchronisation, so it can be captured in a CUDA graph.
 *   Errors: TRI_EINVAL, TRI_ENOSPACE, TRI_ECUDA; an instance whose block count
 *   overflows 32 bits sets device status word ws[0] to TRI_ERANGE and is skipped.
 */
TRI_API int tri_edm_batched(const float *x_cat, const uint64_t *pt_off, const uint32_t *n_k,
                    uint32_t count, uint32_t d, float *out_cat, const uint64_t *out_off,
                    uint32_t rho, uint32_t reg, void *workspace, size_t ws_bytes,
                    void *stream);
TRI_API int tri_edm_batched_workspace_size(uint32_t count, size_t *bytes);

/*
 * tri_edm_batched_partition -- host only, no device work: the instances
 * [*k_begin, *k_end) of a batch that rank `rank` of `ranks` computes, one
 * process per GPU.  With B_k = T(ceil(n_k / (rho reg))) the block count of
 * instance k and P_k = B_0 + ... + B_{k-1}, rank r takes the instances whose
 * P_k lies in [r / ranks, (r + 1) / ranks) of the total: whole instances,
 * contiguous, disjoint and in rank order, the ranges covering [0, count); a
 * rank may get none.  The rank then calls tri_edm_batched on its slices of
 * pt_off, n_k and out_off (count = *k_end - *k_begin); the instances' outputs
 * are disjoint, so nothing is exchanged.
 *   n_k (HOST uint32 [count]); rho, reg as in tri_edm_batched.
 *   Errors: TRI_EINVAL (null pointer, ranks = 0, rank >= ranks, bad rho or reg).
 */
TRI_API int tri_edm_batched_partition(const uint32_t *n_k, uint32_t count, uint32_t rho, uint32_t reg,
                                      uint32_t ranks, uint32_t rank, uint32_t *k_begin, uint32_t *k_end);

/*
 * tri_ca_step -- one synchronous step of an outer-totalistic cellular
 * automaton (Game of Life: birth_mask = 1<<3, survive_mask = 1<<2 | 1<<3) on
 * the triangular domain {0 <= j <= i < n} (Section 1 lists cellular automata
 * on triangular domains among the TD problems; Section 5 motivates the
 * tiled form).  A cell is alive when its byte is non-zero; neighbours
 * outside the domain count as dead.  Each thread streams its strip's rows
 * through registers (neighbouring strips exchange edge cells by warp
 * shuffle); only domain cells of `out` are written (0 or 1).
 *   in, out (device uint8, 16-byte aligned) row-major with leading dimension
 *   ld (bytes); ld >= n and ld a multiple of 16; in != out (no aliasing).
 *   map: LAMBDA, LAMBDA_PDELTA, BB, RB or REC.  rho in {8,16,32}: each block
 *   covers a (4 rho) x (4 rho) cell tile.  Conway's rule runs bit-sliced with
 *   2 rho threads, each a 32-cell strip of rho/4 consecutive rows held as one
 *   bit per cell (two 16-byte loads per row); other rules run with 4 rho
 *   threads, each a 16-cell strip of byte counters (one 16-byte load per row).
 *   Errors: TRI_EINVAL (null, aliasing, bad ld/rho/map), TRI_ERANGE, TRI_ECUDA.
 */
TRI_API int tri_ca_step(const uint8_t *in, uint8_t *out, uint32_t n, size_t ld,
                uint32_t birth_mask, uint32_t survive_mask, int map, uint32_t rho,
                void *stream);

/*
 * tri_ca_run -- `steps` synchronous steps of the automaton of tri_ca_step,
 * the result in `out`.  Conway's rule at rho = 32 (128 x 128-cell tiles) runs
 * up to 16 steps per pass through memory: one warp per tile reads the tile
 * with a 16-cell halo once, holds it as bits in registers (five region rows
 * per lane, vertical neighbours by warp shuffle), takes the steps there
 * (clearing the cells outside the domain after each) and writes the tile's
 * domain cells once.  Other rules and rho take one tri_ca_step per step.  The
 * result is the same bit for bit as `steps` calls of tri_ca_step.
 *   in (read only), out and scratch (device uint8, 16-byte aligned, row-major
 *   with leading dimension ld as in tri_ca_step): pairwise disjoint.  scratch
 *   holds intermediate states when more than one pass is needed (steps > 16
 *   for the fused form, steps > 1 otherwise) and may be NULL otherwise.  Only
 *   domain cells of out and scratch are written.
 *   map: LAMBDA, LAMBDA_PDELTA, BB, RB or REC; rho in {8,16,32}; steps >= 1.
 *   Issues one launch per pass (REC: one per level and pass) and no host
 *   synchronisation.
 *   Errors: TRI_EINVAL (null, aliasing, bad ld/rho/map/masks, steps = 0,
 *   missing scratch), TRI_ERANGE (REC with a block count that is not a power
 *   of two), TRI_ECUDA.
 */
TRI_API int tri_ca_run(const uint8_t *in, uint8_t *out, uint8_t *scratch, uint32_t n, size_t ld,
                       uint32_t birth_mask, uint32_t survive_mask, int map, uint32_t rho,
                       uint32_t steps, void *stream);

/*
 * One cellular-automaton grid split across processes, one per GPU, in row
 * bands.  lambda numbers the tiles row by row (Section 3.1), so the tiles of
 * block rows [R0, R1) are the numbers [T(R0), T(R1)), T(R) = R(R+1)/2.  Each
 * step a band needs one row beyond each of its edges from the neighbouring
 * bands (the halo), and nothing else.
 *
 *   tri_ca_partition: host only, no device work.  The rows [*row_begin,
 *     *row_end) of rank `rank` of `ranks`: whole block rows of 4 rho cells,
 *     the band of rank r starting at the first block row R with T(R) >= r /
 *     ranks of the T(m) tiles, m = ceil(n / (4 rho)).  Bands are disjoint,
 *     cover [0, n) in rank order and hold equal tile counts to within one
 *     block row; a rank may get an empty band when n is small.
 *     Errors: TRI_EINVAL (null pointer, ranks = 0, rank >= ranks, bad rho).
 *
 *   tri_ca_step_rows: tri_ca_step (map lambda) restricted to rows [row_begin,
 *     row_end): only those rows' domain cells of `out` are written, and only
 *     rows row_begin - 1 .. row_end of `in` (those inside [0, n)) are read,
 *     so a rank's buffers need hold only its band and the two halo rows.
 *     row_begin must be a multiple of 4 rho, row_end one too or n.  An empty
 *     band (row_begin = row_end, n included) does nothing.  Buffers, rule, rho and errors as tri_ca_step, and
 *     TRI_EINVAL for a band that is not whole block rows or not inside [0, n].
 */
TRI_API int tri_ca_partition(uint32_t n, uint32_t rho, uint32_t ranks, uint32_t rank,
                             uint32_t *row_begin, uint32_t *row_end);
TRI_API int tri_ca_step_rows(const uint8_t *in, uint8_t *out, uint32_t n, size_t ld,
                             uint32_t birth_mask, uint32_t survive_mask, uint32_t rho,
                             uint32_t row_begin, uint32_t row_end, void *stream);

/*
 * tri_collide -- collision detection of N spheres (Section 5, test 3): every
 * pair i > j whose centres lie at most r_i + r_j apart (touching counts).
 * The test is taken on squares, s = sum_k (c[i][k] - c[j][k])^2 added in
 * increasing k, collide <=> s <= (r_i + r_j)^2, each step one FP32 operation
 * rounded to nearest (no fused multiply-add), so any implementation that
 * takes the same steps reaches the same decisions bit for bit.
 *   centres (device, FP32) row-major [n][dim], dim in {1, 2, 3}; radii
 *   (device, FP32) [n].
 *   map: any tri_map.  rho in {8, 16, 32}; reg in {1, 4, 8} (0 picks 8 for
 *   rho <= 16 and 4 for rho = 32; 8 only with rho <= 16): blocks of rho x rho threads, each thread reg x reg
 *   pairs of an S x S tile, S = rho*reg, whose 2 S spheres are staged in
 *   shared memory (the paper's shared-memory test).  UTM (a thread-space map)
 *   runs one pair per thread from global memory instead; reg is ignored there.
 *   count (device uint32 [n], may be NULL): zeroed by the call, then
 *   count[i] = the number of spheres sphere i collides with.
 *   n_pairs (device uint64, required): zeroed by the call, then the number of
 *   colliding pairs.
 *   pairs (device uint32 [pair_cap][2], may be NULL when pair_cap = 0): the
 *   first min(n_pairs, pair_cap) colliding pairs found, as (i, j) with i > j,
 *   in no particular order; the caller compares n_pairs with pair_cap to see
 *   whether the list is complete.
 *   Errors: TRI_EINVAL (null n_pairs, null centres/radii with n > 0, pairs NULL with pair_cap >
 *   0, dim or rho or reg or map out of range), TRI_ERANGE (too many blocks
 *   for the map; REC with a block count that is not a power of two),
 *   TRI_ECUDA.  n = 0 only zeroes n_pairs.
 */
TRI_API int tri_collide(const float *centres, const float *radii, uint32_t n, uint32_t dim, int map,
                        uint32_t rho, uint32_t reg, uint32_t *count, uint32_t *pairs, uint64_t pair_cap,
                        unsigned long long *n_pairs, void *stream);

/*
 * tet_map -- map blocks onto the discrete tetrahedron (Section 6): block
 * omega -> (layer, row, col), layer >= row >= col, with the layer taken from
 * the real root of x^3 + 3x^2 + 2x - 6 omega = 0 (an FP32 estimate plus an
 * exact integer correction against T_k = k(k+1)(k+2)/6) and (row, col) from
 * the 2-D lambda of omega - T_layer.  Blocks hold rho x rho threads, each
 * looping over the rho elements of the third block index; the element
 * domain is the strict triplets n > i > j > k >= 0.
 *   out as in tri_map_launch; COUNT index C(i,3) + C(j,2) + k, C(n,3) counters.
 *   Errors: TRI_EINVAL, TRI_ERANGE (more than 2^32 - 1 blocks), TRI_ECUDA.
 */
TRI_API int tet_map(uint32_t n, uint32_t rho, int body, uint32_t *out, void *stream);

/*
 * tet_map_ex -- tet_map under a chosen map:
 *   TRI_MAP_LAMBDA: as tet_map (the closed-form cubic root);
 *   TRI_MAP_TET_TABLE: the succinct lookup table that Section 7 proposes: the
 *     layer starts T_k for every T_k < 2^32 (2953 words, o(T_n), fixed at build
 *     time in constant memory); a block finds its layer by binary search over
 *     the first m entries (one broadcast read per step) and its (row, col) by
 *     the 2-D lambda, so no cube root is taken;
 *   TRI_MAP_BB: the m^3 bounding box of blocks, those outside the tetrahedron
 *     leaving at once (Section 6 puts its waste at up to 6x).
 *   Other arguments, results and errors as tet_map; TRI_EINVAL for other maps,
 *   TRI_ERANGE for BB with m > 65535.
 */
TRI_API int tet_map_ex(int map, uint32_t n, uint32_t rho, int body, uint32_t *out, void *stream);

/*
 * tet_at_energy -- Axilrod-Teller triple-dipole energy of n points, a
 * triplet-interaction n-body sum over the tetrahedral domain (Section 6):
 *   E = sum_{i>j>k} nu (1 + 3 cos g_i cos g_j cos g_k) / (r_ij r_jk r_ki)^3.
 *   xyz (device FP32 [n][3]); energy (device, one double).  Terms in FP32,
 *   block partials in FP64 written to the workspace, then summed in a fixed
 *   order by a second kernel, so the result is deterministic.
 *   map: TRI_MAP_LAMBDA (tetrahedral lambda), TRI_MAP_TET_TABLE (the same
 *   blocks with the layer from the table of tet_map_ex; bit-identical
 *   result) or TRI_MAP_BB (m^3 box with
 *   discard).  rho in {8,16,32}.
 *   Errors: TRI_EINVAL, TRI_ERANGE, TRI_ENOSPACE, TRI_ECUDA.
 */
TRI_API int tet_at_energy(const float *xyz, uint32_t n, double nu, double *energy, int map,
                  uint32_t rho, void *workspace, size_t ws_bytes, void *stream);
TRI_API int tet_at_workspace_size(uint32_t n, uint32_t rho, int map, size_t *bytes);

/*
 * One Axilrod-Teller energy split across processes, one per GPU: each rank
 * sums the triplets of a contiguous range of the tetrahedral block numbers
 * (Section 6: block w = T3(L) + T(R) + C, T3(L) = L(L+1)(L+2)/6, with m =
 * ceil(n / rho) layers), and the ranks add their partial energies (one FP64
 * all-reduce).
 *
 *   tet_at_partition: host only, no device work.  The blocks
 *     [*omega_begin, *omega_end) = [floor(T k / ranks), floor(T (k+1) /
 *     ranks)) of the T = T3(m) blocks for k = rank: disjoint, covering [0, T)
 *     in rank order.  Errors: TRI_EINVAL (null pointer, ranks = 0, rank >=
 *     ranks, bad rho), TRI_ERANGE (T >= 2^32).
 *
 *   tet_at_energy_range: the energy of the strict triplets in blocks
 *     [omega_begin, omega_end), written to *energy (device, one double): block
 *     partials in FP64, then a fixed-order sum, as tet_at_energy.  An empty
 *     range gives 0.  The ranges of any partition of [0, T) add up to
 *     tet_at_energy's result up to the order of the FP64 additions.
 *     map: TRI_MAP_LAMBDA or TRI_MAP_TET_TABLE.  workspace: device, 8-byte
 *     aligned, at least (omega_end - omega_begin) doubles.
 *     Errors: TRI_EINVAL (null pointer, n = 0, bad rho or map, omega_begin >
 *     omega_end or omega_end > T), TRI_ENOSPACE, TRI_ERANGE (T >= 2^32),
 *     TRI_ECUDA.
 */
TRI_API int tet_at_partition(uint32_t n, uint32_t rho, uint32_t ranks, uint32_t rank,
                             uint64_t *omega_begin, uint64_t *omega_end);
TRI_API int tet_at_energy_range(const float *xyz, uint32_t n, double nu, double *energy, int map,
                                uint32_t rho, uint64_t omega_begin, uint64_t omega_end,
                                void *workspace, size_t ws_bytes, void *stream);

/*
 * tet_at_energy_noalloc -- tet_at_energy without a workspace, for callers
 * that cannot call cudaMalloc: code whose device memory is all handed out by
 * another allocator (a framework's caching pool, an arena fixed at start-up)
 * and code that must not trigger the device-wide synchronisation cudaMalloc
 * and cudaFree can imply.  The paper has no counterpart; this is a property
 * of the library, not of the method.
 *   The block partials live in a 2 MiB array (262,144 doubles) compiled into
 *   libtri.so, which every GPU that loads the library holds until the process
 *   exits.  Sizes whose partial count T_m, m = ceil(n/rho), exceeds it are
 *   rejected with TRI_ENOSPACE (n <= 920 at rho = 8, 1840 at rho = 16, 3680
 *   at rho = 32).  Allocates nothing: no cudaMalloc, cudaFree or allocating
 *   library call.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   All calls share the one array: calls whose kernels may overlap on the GPU
 *   (different streams, or host threads without ordering between them) race
 *   on it and must be serialised by the caller.  Nothing in it has to start
 *   at zero: each call writes every partial it reads.
 *   Arguments, result and other errors as in tet_at_energy.
 */
TRI_API int tet_at_energy_noalloc(const float *xyz, uint32_t n, double nu, double *energy, int map,
                                  uint32_t rho, void *stream);

/*
 * MLP cost model y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (one output), used
 * to predict the log run time of a (kernel, n, d, map, rho) configuration.
 * Not in the paper.  theta (device FP32) holds W1 [H1][F], b1 [H1],
 * W2 [H2][H1], b2 [H2], W3 [H2], b3 [1] contiguously, row-major.
 * X (device FP32 [B][F]), y (device FP32 [B]).  H1, H2 <= 128, F <= 64.
 * workspace: tri_mlp_workspace_size bytes (activations of the batch).
 *
 *   tri_mlp_forward: pred[b] for every row of X.
 *   tri_mlp_grad:    loss = mean_b (pred[b] - y[b])^2 into *loss (device float)
 *                    and its gradient w.r.t. theta into grad (device, overwritten).
 *   tri_mlp_adam:    one Adam step (t counts from 1) on theta with moments m, v.
 *   tri_mlp_argmin:  forward over B candidate rows and write the index of the
 *                    smallest prediction to *best (device uint32).
 */
TRI_API int tri_mlp_workspace_size(uint32_t B, uint32_t H1, uint32_t H2, size_t *bytes);
TRI_API int tri_mlp_forward(const float *theta, const float *X, uint32_t B, uint32_t F, uint32_t H1,
                    uint32_t H2, float *pred, void *workspace, size_t ws_bytes, void *stream);
TRI_API int tri_mlp_grad(const float *theta, const float *X, const float *y, uint32_t B, uint32_t F,
                 uint32_t H1, uint32_t H2, float *loss, float *grad, void *workspace,
                 size_t ws_bytes, void *stream);
TRI_API int tri_mlp_adam(float *theta, const float *grad, float *m, float *v, uint32_t nparams,
                 uint32_t t, float lr, float beta1, float beta2, float eps, void *stream);
TRI_API int tri_mlp_argmin(const float *theta, const float *X, uint32_t B, uint32_t F, uint32_t H1,
                   uint32_t H2, uint32_t *best, void *workspace, size_t ws_bytes,
                   void *stream);

/*
 * Map and rho selection from the learned cost model (not in the paper).
 * Candidates of a (kernel, n, d) configuration are the autotuner's: for EDM
 * the maps LAMBDA, LAMBDA_PDELTA, BB, RB, REC, UTM, for the Life step the
 * same without UTM, for the triplet energy LAMBDA and BB; each with rho in
 * {8, 16, 32}; REC only where the block rows are a power of two.  Their
 * TRI_SELECT_FEATURES features: log2 n, log2 d, log2 rho, log2 of the blocks
 * the map launches, kernel one-hot (EDM, CA, AT), map one-hot (LAMBDA,
 * LAMBDA_PDELTA, BB, RB, REC, UTM), log2 of the tile side (4 rho for EDM
 * and CA, rho for AT).
 *
 *   tri_select_features: host only.  Writes the candidates (maps outer, rho
 *     inner) to maps[] / rhos[] and their raw features to X [count][F]
 *     (FP32), count <= TRI_SELECT_MAX_CANDIDATES.
 *   tri_select: standardises the features with the model's mu and sd (host
 *     FP64), evaluates the MLP on the device (tri_mlp_argmin, theta on the
 *     device in tri_mlp layout with F = TRI_SELECT_FEATURES) and writes the
 *     candidate of smallest predicted log time (relative to the default
 *     candidate) to *map and *rho.  Synchronises `stream`.  A NULL model or
 *     theta gives the library default (TRI_MAP_LAMBDA, rho 16) with no device
 *     work.  workspace: tri_select_workspace_size bytes, 256-byte aligned.
 *   tri_sync_status: synchronises `stream` and reads one device status word
 *     (the tensor-core workspace's int at byte 8, the batched EDM's ws[0])
 *     into *value.
 *   Errors: TRI_EINVAL (null pointers, n = 0, unknown kernel), TRI_ENOSPACE,
 *   TRI_ECUDA.
 */
#define TRI_SELECT_FEATURES 14
#define TRI_SELECT_MAX_CANDIDATES 18
typedef enum { TRI_KERNEL_EDM = 0, TRI_KERNEL_CA = 1, TRI_KERNEL_AT = 2 } tri_kernel;
typedef struct {
    const float *theta;     /* device, tri_mlp parameter layout */
    uint32_t h1, h2;        /* hidden widths */
    const double *mu, *sd;  /* host, TRI_SELECT_FEATURES each */
} tri_cost_model;
TRI_API int tri_select_features(int kernel, uint32_t n, uint32_t d, float *X, int *maps, uint32_t *rhos,
                                uint32_t *count);
TRI_API int tri_select_workspace_size(uint32_t h1, uint32_t h2, size_t *bytes);
TRI_API int tri_select(const tri_cost_model *model, int kernel, uint32_t n, uint32_t d, int *map, uint32_t *rho,
                       void *workspace, size_t ws_bytes, void *stream);
TRI_API int tri_sync_status(const int *status, int *value, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TRI_H */
