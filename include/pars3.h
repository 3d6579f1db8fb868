/*
 * pars3.h -- C ABI of the GB300 skew-symmetric SpMV library.
 *
 * The library applies y = (alpha I + S) x for a sparse skew-symmetric S
 * (S = -S^T, Sec. 1, Eq. 1) stored as its strict lower triangle only (the
 * half storage of Sec. 3), after the preprocessing of Sec. 3.1.2: a
 * reverse Cuthill-McKee reordering squeezes S towards a band and the band is
 * split three ways -- the diagonal (here alpha I, S has a zero diagonal), a
 * middle part within a bandwidth W of the diagonal and an outer part beyond
 * it.  Every stored middle entry l_ij is read once and used twice
 * (y_i += l_ij x_j and y_j -= l_ij x_i, Eqs. 2-6); the conflicting
 * (cross-tile) mirrored products go through a halo buffer that a fixed-order
 * pass folds in, so no atomics are used and results are bitwise
 * reproducible from run to run.  On top of the operator sits the minimal
 * residual (MRS) Krylov solver for shifted skew systems named in Sec. 1.
 *
 * Conventions
 *  - Every function returns an int status: PARS3_OK (0) or a negative code.
 *    Nothing throws across the ABI.  pars3_strerror() names a code.
 *  - Host input arrays belong to the caller and are copied; the caller may
 *    free them after the call returns.
 *  - A handle (pars3_handle) owns its host metadata and, after
 *    pars3_upload(), its device buffers; pars3_free() releases both.
 *  - Device vectors (x, y, X, Y, b) are caller-allocated device pointers in
 *    the handle's REORDERED numbering: x'[k] = x[perm[k]].
 *    pars3_permute()/pars3_unpermute() convert on the device.  Device
 *    vectors must be 16-byte aligned.
 *  - stream arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream).  Calls that launch kernels are asynchronous
 *    with respect to the host unless stated otherwise.
 *  - Integer indices are int32 (n < 2^31, stored nonzeros < 2^31).
 *  - Threads: different handles may be used from different host threads at
 *    once; one handle must not be used by two host threads at the same time
 *    (it grows scratch and caches graphs on first use).  A handle stays on
 *    the device that was current at pars3_upload(); calls on it must run
 *    with that device current.
 *  - With PARS3_SPLIT_SYMMETRIC the same calls apply S = L + L^T (the
 *    symmetric case the paper's method also covers, abstract and Sec. 5).
 */
#ifndef PARS3_H
#define PARS3_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define PARS3_OK 0
#define PARS3_EINVAL (-1)       /* bad argument (size, null pointer, alignment, parameter range) */
#define PARS3_ENOTSKEW (-2)     /* input is not a valid strict lower triangle: an entry on or above
                                   the diagonal, an unsorted or duplicate column, a bad row pointer */
#define PARS3_ENOMEM (-3)       /* host or device allocation failed */
#define PARS3_ECUDA (-4)        /* a CUDA runtime call failed */
#define PARS3_ENOCONV (-5)      /* MRS reached its iteration limit before the tolerance */
#define PARS3_ETIMEOUT (-6)     /* a bounded device-side wait gave up (error word set by a kernel) */
#define PARS3_EUNSUPPORTED (-7) /* valid request this build does not support (e.g. precision not packed) */
#define PARS3_ESTATE (-8)       /* handle in the wrong state (e.g. not uploaded) */
#define PARS3_ENONFINITE (-9)   /* a NaN or Inf value in the input */

/* ------------------------------------------------------------ precisions */
#define PARS3_F64 0   /* values fp64, vectors fp64, accumulation fp64 */
#define PARS3_F32 1   /* values fp32, vectors fp32, accumulation fp32 */
#define PARS3_BF16 2  /* values bf16 (round-to-nearest-even of the fp32 rounding of the
                         fp64 input), vectors fp32, accumulation fp32 */
#define PARS3_DTYPE_BIT(d) (1 << (d))

/* ---------------------------------------------------------------- flags */
#define PARS3_RCM_GUARD 1 /* pars3_reorder: return the identity when RCM would widen the band */
#define PARS3_RCM_PERIPHERAL 2 /* pars3_reorder: start each component at a George-Liu pseudo-peripheral
                                  vertex (from the (degree, index) candidate, move to the smallest
                                  (degree, index) vertex of the last BFS level while that strictly
                                  increases the eccentricity) */
#define PARS3_RCM_LOCAL 4 /* pars3_reorder: order by the RCM of the local edges only -- those on a
                             triangle or a 4-cycle, plus those between two vertices whose degree
                             product exceeds 4096 -- so that the random long-range "shortcut" edges
                             of a small-world pattern do not steer it (they stay in the matrix) */
#define PARS3_SPLIT_SYMMETRIC 1 /* pars3_split_params.flags: S = L + L^T (the symmetric variant the
                                   paper's method also covers, abstract and Sec. 5) instead of the
                                   skew-symmetric S = L - L^T */

#define PARS3_VARIANT_LOOKAHEAD 1 /* pars3_split_params.variant, see there */

typedef struct pars3_handle pars3_handle;

/* Split parameters (Sec. 3.1.2, Fig. 8: the middle/outer boundary is a
 * user-given bandwidth).  T and W are powers of two with 32 <= W <= T <=
 * 32768; 0 selects the default rule (W = smallest power of two >= the
 * reordered bandwidth, clamped to [32, w_cap]; T = max(W, 1024)), where
 * w_cap = 1024 when PARS3_F64 is packed and 2048 otherwise (two tile stages
 * must fit in shared memory). */
typedef struct {
    int32_t T;          /* row tile: rows [tT, tT+T) are owned by one thread block */
    int32_t W;          /* middle bandwidth: stored (i, j) with i - j <= W are middle entries */
    int32_t dtypes;     /* bit mask of PARS3_DTYPE_BIT(d) value precisions to pack (0 = F64 only) */
    int32_t long_row;   /* full-storage row length above which a row is cut into pieces that are
                           summed separately and added in order by the fold (0 = default 128, at most 128) */
    int32_t flags;      /* 0 (skew-symmetric) or PARS3_SPLIT_SYMMETRIC */
    int32_t piece;      /* entries per piece of a long row (0 = default 192; 8 <= piece <= 255) */
    int32_t long_slices;/* 32-piece slices of long rows per thread block (0 = default 32; at most 1024) */
    int32_t lane_bytes; /* pars3_spmm: bytes of X a lane holds per row, 4/8 (one element), 16 or 32
                           (0 = rule: 32 when k >= 16 allows it, else 16 when k allows it, else one element) */
    int32_t variant;    /* tile kernel: 0 = default; PARS3_VARIANT_LOOKAHEAD = fp32 / bf16 tiles load the next
                           slice's columns ahead at two blocks per SM (fp64 tiles always do) */
    int32_t reserved[3];
} pars3_split_params;

/* Read-only view of a handle's canonical split (host memory owned by the
 * handle, valid until pars3_free).  It is the bit-exact contract with the
 * oracle: values are moved or negated, never computed. */
typedef struct {
    int32_t n, T, W, ntiles;
    int64_t nnz;                 /* stored strict-lower entries */
    int64_t counts[3];           /* middle-local, middle-halo, outer */
    const int32_t *perm;         /* [n] new -> old */
    const int32_t *rowptr;       /* [n+1] strict-lower CSR of P S P^T */
    const int32_t *col;          /* [nnz] */
    const double *val;           /* [nnz] (skew: an entry whose orientation flipped carries the flipped sign) */
    const uint8_t *cls;          /* [nnz] 0 middle-local, 1 middle-halo, 2 outer */
    const int32_t *tile_ptr;     /* [ntiles+1] */
    const int32_t *tile_list;    /* [counts0+counts1] middle entries of each tile, (column, row) order */
    const int32_t *outer_csr;    /* [counts2] outer entries, (row, column) order */
    const int32_t *outer_csc;    /* [counts2] outer entries, (column, row) order */
} pars3_canonical;

/* Sizes of the device layout (for reports and tests). */
typedef struct {
    int32_t n, T, W, ntiles, dtypes;
    int64_t nnz;
    int64_t half_entries;        /* entries on the half-storage tile path (read once, used twice) */
    int64_t full_entries;        /* full-storage entries on the row path (outer entries twice) */
    int64_t long_entries;        /* full-storage entries of long rows (summed in pieces) */
    int32_t long_rows, long_pieces;
    int64_t halo_targets;        /* distinct rows that receive a cross-tile mirrored sum */
    int32_t max_tile_half;       /* largest number of half-path entries of one tile */
    int32_t smem_bytes[3];       /* dynamic shared memory of pars3_spmv's tile kernel per precision (0 = not
                                    packed, or nothing staged) */
    int64_t device_bytes;        /* device memory held by the handle after upload */
    int64_t bytes_per_spmv[3];   /* modelled DRAM bytes of one pars3_spmv per precision */
    int64_t bandwidth;           /* max i - j of the reordered lower triangle */
    int32_t symmetric;           /* 1 for a PARS3_SPLIT_SYMMETRIC handle */
    int32_t reserved;
} pars3_info;

/* MRS options (Sec. 1: minimal residual method for shifted skew systems,
 * one product and one inner product per iteration). */
typedef struct {
    double rtol;         /* target ||b - A x||_2 / ||b||_2 (true residual, fp64) */
    int32_t max_iter;    /* total inner iterations over all refinement cycles */
    int32_t inner;       /* PARS3_F64: plain fp64 MRS; PARS3_F32 / PARS3_BF16: inner MRS in that
                            precision inside fp64 iterative refinement */
    double inner_rtol;   /* relative reduction asked of each inner solve (refinement only) */
    int32_t max_outer;   /* refinement cycles */
    int32_t check_every; /* iterations between device-side convergence checks of the recursion */
    int32_t reserved[4];
} pars3_mrs_opts;

typedef struct {
    int32_t iters;       /* inner iterations performed */
    int32_t outer;       /* refinement cycles (1 for plain fp64) */
    double true_relres;  /* final ||b - A x|| / ||b|| computed in fp64 on the device */
    double est_relres;   /* last recursive residual estimate */
    int32_t status;      /* PARS3_OK or PARS3_ENOCONV */
    int32_t reserved[3];
} pars3_mrs_result;

/* ------------------------------------------------------------- functions */

/* Name of a status code (static string). */
const char *pars3_strerror(int code);

/* Library version and the CUDA architecture it was built for (e.g. 103). */
int pars3_version(int32_t *major, int32_t *minor, int32_t *cuda_arch);

/* pars3_reorder -- Sec. 1 and Sec. 3.1.2: reverse Cuthill-McKee ordering of
 * the symmetric pattern of S, on the host.  rowptr[n+1]/col[nnz] is the
 * strict lower pattern (sorted unique columns < row).  Each connected
 * component is searched breadth-first from its unvisited vertex of least
 * (degree, index); a dequeued vertex appends its unvisited neighbours in
 * (degree, index) order; the whole visit order is reversed.  perm_out[n]
 * (caller-allocated) receives new -> old.  With PARS3_RCM_GUARD the identity
 * is returned when the RCM bandwidth would exceed the original (Sec. 4.1:
 * already banded matrices gain nothing).  PARS3_RCM_PERIPHERAL and
 * PARS3_RCM_LOCAL select the variants described at the flags (both may be
 * combined with the guard; bandwidths and the guard always count every
 * stored entry).  bw_before/bw_after may be NULL.  Errors: EINVAL (n < 0,
 * null pointer, unknown flag), ENOTSKEW (pattern not strict lower), ENOMEM. */
int pars3_reorder(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t flags,
                  int32_t *perm_out, int64_t *bw_before, int64_t *bw_after);

/* pars3_reorder_device -- the ordering of pars3_reorder, computed on the GPU
 * (Sec. 1 and Sec. 3.1.2; the paper leaves preprocessing out of its timings,
 * Sec. 4, but a batch of matrices pays it every time).  rowptr[n+1] and
 * col[nnz] are DEVICE arrays holding the strict lower pattern, perm_out[n]
 * a caller-allocated DEVICE array that receives new -> old.  The result is
 * identical, element for element, to pars3_reorder with the same flags:
 * components are placed in the order of their (degree, index)-smallest
 * vertex, searched level by level with every vertex appended by the first
 * vertex of the previous level adjacent to it, in (degree, index) order.
 * Flags: PARS3_RCM_GUARD, PARS3_RCM_PERIPHERAL and PARS3_RCM_LOCAL, as for
 * pars3_reorder.  bw_before/bw_after (host, may be NULL) as for
 * pars3_reorder.  Runs on `stream` and returns after the result is
 * complete (it synchronizes the stream a few times to size its work).
 * Allocates device scratch of about 52 bytes per stored entry plus 130 per
 * vertex, freed before returning.  Requires nnz < 2^30.
 * Errors: EINVAL (n < 0, null pointer, unknown flag), ENOTSKEW (pattern
 * not strict lower; checked on the device before any other use of it),
 * ENOMEM, EUNSUPPORTED, ECUDA, ETIMEOUT (the bounded union-find retries ran
 * out; not expected). */
int pars3_reorder_device(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t flags,
                         int32_t *perm_out, int64_t *bw_before, int64_t *bw_after, void *stream);

/* pars3_reorder_device_batched -- pars3_reorder_device for `count` matrices
 * in one call, searched together (the work is the block-diagonal union of
 * the patterns, so the number of sequential level steps is that of the
 * deepest matrix, not the sum over matrices).  n[count], rowptr[count],
 * col[count], perm_out[count] are HOST arrays; rowptr[m], col[m] and
 * perm_out[m] are DEVICE arrays of matrix m as for pars3_reorder_device
 * (col[m] and perm_out[m] may be NULL when matrix m has no entries or no
 * vertices).  bw_before/bw_after are host arrays of count values, or NULL.
 * Every perm_out[m] equals pars3_reorder of matrix m alone with the same
 * flags.  The union must have fewer than 2^31 vertices and 2^30 entries.
 * Errors as for pars3_reorder_device; ENOTSKEW when any matrix fails the
 * check (then no perm_out is written). */
int pars3_reorder_device_batched(int32_t count, const int32_t *n, const int32_t *const *rowptr,
                                 const int32_t *const *col, int32_t flags, int32_t *const *perm_out,
                                 int64_t *bw_before, int64_t *bw_after, void *stream);

/* pars3_split -- Sec. 3.1.2 and Figs. 7-8: reorder S by perm (new -> old;
 * NULL = identity), re-triangularize (an entry landing above the diagonal is
 * stored mirrored with its sign flipped, Eq. 2), classify every stored entry
 * as middle-local / middle-halo / outer for tile T and bandwidth W, and build
 * the device layout for the precisions in p->dtypes.  val[nnz] are fp64 host
 * values.  On success *out is a new handle (free with pars3_free).
 * Errors: EINVAL (bad T/W/dtypes/perm), ENOTSKEW, ENONFINITE, ENOMEM. */
int pars3_split(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                const int32_t *perm, const pars3_split_params *p, pars3_handle **out);

/* pars3_split_device -- pars3_split with the canonical split computed on
 * the GPU (Sec. 3.1.2, Eq. 2, Figs. 7-8): rowptr[n+1], col[nnz], val[nnz]
 * (fp64) and perm[n] (new -> old, NULL = identity) are DEVICE arrays.  On
 * the device the pattern, values and permutation are checked, the entries
 * are permuted and re-triangularized (sign flip, Eq. 2), sorted by
 * (row, col), classified for (T, W) and listed per tile and in CSR / CSC
 * order, and the device layout is built from them (the decisions over rows
 * and tiles by the host builder's own rules); the new handle holds host
 * copies of all of it, as a pars3_split handle does.  The result -- every
 * array pars3_split_export shows, and the layout (pars3_layout_digest) --
 * is identical to pars3_split with the same inputs and parameters.  Runs on
 * `stream` and returns after the handle is complete.  Allocates temporary
 * device memory (about 100 bytes per stored entry).  Errors as for
 * pars3_split, plus ECUDA. */
int pars3_split_device(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                       const int32_t *perm, const pars3_split_params *p, pars3_handle **out, void *stream);

/* Canonical split of a handle (host view; see pars3_canonical). */
int pars3_split_export(const pars3_handle *h, pars3_canonical *out);

/* pars3_layout_digest -- a 64-bit FNV-1a digest of the handle's device
 * layout (every array with its length, and the scalars the kernels read),
 * for checking that two handles hold the same layout (e.g. one from
 * pars3_split and one from pars3_split_device).  Host only.
 * Errors: EINVAL (null pointer). */
int pars3_layout_digest(const pars3_handle *h, uint64_t *digest);

/* Device-layout sizes of a handle. */
int pars3_info_get(const pars3_handle *h, pars3_info *out);

/* Host-only consistency check of the device layout against the canonical
 * split: every middle entry appears once on the half path, every other
 * entry twice on the full/long paths with mirrored sign.  Returns PARS3_OK
 * or PARS3_EINVAL. */
int pars3_layout_check(const pars3_handle *h);

/* pars3_upload -- allocate the handle's device buffers on the current
 * device and copy the layout (cudaMemcpyAsync on stream, then the stream is
 * synchronized).  Idempotent.  Errors: ENOMEM, ECUDA. */
int pars3_upload(pars3_handle *h, void *stream);

/* pars3_spmv -- y = (alpha I + P S P^T) x for x, y of n entries in the
 * handle's numbering: fp64 vectors for PARS3_F64, fp32 for PARS3_F32 and
 * PARS3_BF16.  Two kernels: the tile kernel (blocks that sum the pieces of
 * long rows, then one block per row tile: TMA staging of the x window
 * [tT-W, tT+T) and of the half-storage middle entries with their in-tile
 * mirrored sums in shared memory, the full-storage outer rows) and the fold
 * kernel (cross-tile halo sums and long-row piece sums, fixed order).  x and
 * y must not overlap.  The call only enqueues work: a failure inside a
 * kernel shows in pars3_check.  Errors: EINVAL, ESTATE (not uploaded),
 * EUNSUPPORTED (precision not packed), ECUDA. */
int pars3_spmv(const pars3_handle *h, int32_t dtype, double alpha, const void *x, void *y,
               void *stream);

/* pars3_spmm -- Y = (alpha I + P S P^T) X for k right-hand sides stored
 * row-major (X[i*k + c]), 1 <= k <= 32.  Same precisions and errors as
 * pars3_spmv. */
int pars3_spmm(const pars3_handle *h, int32_t dtype, double alpha, int32_t k, const void *X,
               void *Y, void *stream);

/* pars3_spmm_batched -- count independent products Y_m = (alpha_m I + S_m) X_m
 * (uneven sizes, same dtype and k) in ONE persistent kernel launch over a
 * fixed-order list of (matrix, tile) work items, followed by one fold
 * launch; with capture != 0 the pair is recorded once in a CUDA graph kept
 * by the first handle and replayed on later calls with the same arguments.
 * hs[count], alpha[count] (host), X[count], Y[count] (device pointers, host
 * array).  One SpMM lane width serves the whole batch: the handles'
 * lane_bytes when all of them carry the same value, else the rule (see
 * pars3_split_params).  Errors: as pars3_spmm. */
int pars3_spmm_batched(pars3_handle *const *hs, int32_t count, int32_t dtype, const double *alpha,
                       int32_t k, const void *const *X, void *const *Y, int32_t capture,
                       void *stream);

/* pars3_mrs -- solve (alpha I + P S P^T) x = b (Sec. 1: MRS, one product
 * and one inner product per iteration) on the device.  b[n], x[n] are fp64
 * device vectors in the handle's numbering; x holds x0 on entry and the
 * solution on exit.  opts->inner selects plain fp64 MRS or an fp32 / bf16
 * inner MRS inside fp64 iterative refinement (true residual, inner products
 * and norms in fp64).  The inner loop runs as a CUDA graph with a
 * device-side while-condition; the host only syncs once per refinement
 * cycle.  alpha must be nonzero.  res may be NULL.  Errors: EINVAL, ESTATE,
 * EUNSUPPORTED (also for a PARS3_SPLIT_SYMMETRIC handle: the recurrence
 * needs a skew-symmetric S), ENOCONV (limit reached; x holds the best
 * iterate), ECUDA, ETIMEOUT. */
int pars3_mrs(const pars3_handle *h, double alpha, const double *b, double *x,
              const pars3_mrs_opts *opts, pars3_mrs_result *res, void *stream);

/* pars3_permute / pars3_unpermute -- dst[k] = src[perm[k]] and
 * dst[perm[k]] = src[k] for n*k_cols elements of the given precision's vector
 * type (row-major blocks of k_cols columns). */
int pars3_permute(const pars3_handle *h, int32_t dtype, int32_t k_cols, const void *src, void *dst,
                  void *stream);
int pars3_unpermute(const pars3_handle *h, int32_t dtype, int32_t k_cols, const void *src, void *dst,
                    void *stream);

/* pars3_spmv_host -- end-to-end product on HOST vectors in the ORIGINAL
 * numbering: copies x (n entries of the precision's vector type) to the
 * device, permutes, applies the operator, un-permutes and copies y back,
 * all on stream, then synchronizes the stream.  Staging buffers are owned
 * by the handle (allocated on first use).  Errors: as pars3_spmv. */
int pars3_spmv_host(pars3_handle *h, int32_t dtype, double alpha, const void *x_host, void *y_host,
                    void *stream);

/* pars3_spmv_noalloc -- the same product as pars3_spmv, for callers that
 * cannot have the library allocate device memory for its scratch (all
 * device memory handed to another allocator or pool, or a fixed memory
 * budget).  The paper has no counterpart: this is a deployment variant.
 * The scratch (cross-tile halo sums and long-row partial sums) lives in one
 * library-wide device array of 4 MiB that every GPU loading the library
 * holds until the process exits; the call allocates nothing.  The array's
 * device address is looked up on the first call with a given device
 * current.  CUDA loads a library's device code lazily by default, so that
 * first call may also load the code that holds the array, which reserves
 * its 4 MiB on that device then: make the first call on each device before
 * any stream capture and before any memory budget takes effect.
 * Every call shares the array (its contents are overwritten before they
 * are read), so calls that overlap on the GPU race.  Returns
 * PARS3_EUNSUPPORTED when the handle needs more scratch than the array
 * holds (halo targets plus long-row slots times the accumulator size: 8
 * bytes for PARS3_F64, 4 otherwise); other errors as pars3_spmv. */
int pars3_spmv_noalloc(const pars3_handle *h, int32_t dtype, double alpha, const void *x, void *y,
                       void *stream);

/* Reads and clears the handle's device error word (synchronizes the
 * stream).  Returns PARS3_OK, PARS3_ETIMEOUT or PARS3_ECUDA.  PARS3_ETIMEOUT
 * means a bounded device-side wait for a staged copy gave up (about a
 * second) in some call since the last check: the outputs of the tiles
 * concerned were written as NaN and the results of those calls are invalid
 * (a copy still in flight may also have landed in a later block's shared
 * memory, so treat every result since the last PARS3_OK as invalid). */
int pars3_check(const pars3_handle *h, void *stream);

/* pars3_autotune -- times pars3_spmm (k right-hand sides) on the current
 * device and returns the fastest split parameters in *best (fields not
 * searched are copied from *base): the cut points (T, W) (coordinate search
 * over powers of two), then, for matrices with long rows, the long-row
 * threshold, piece length and long slices per block, then the tile kernel
 * variant (fp32 / bf16, k = 1) or the lane width of the multi-vector
 * product (k > 1).  The matrix arguments are those of pars3_split (host
 * arrays); they are copied to the device, reordered there once, and every
 * candidate is split on the GPU as pars3_split_device splits it.  Leaves no
 * device state behind.  Errors: as pars3_split_device and pars3_upload. */
int pars3_autotune(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                   const int32_t *perm, const pars3_split_params *base, int32_t dtype, int32_t k,
                   pars3_split_params *best, double *best_us);

/* pars3_fp64_fma_rate -- measurement helper (the paper has no counterpart):
 * the current device's fp64 fused multiply-add rate in FMAs per second, from
 * a kernel of independent FMA chains on every SM (best of three timed runs
 * after a warm-up, CUDA events on stream; synchronizes the stream).  The
 * fp64 products read one value and do one FMA per stored entry, so on a part
 * with a narrow fp64 unit this rate bounds them beside HBM bandwidth.
 * Allocates and frees 8 bytes of device memory.  Errors: EINVAL (null
 * pointer), ECUDA, ENOMEM. */
int pars3_fp64_fma_rate(double *fma_per_s, void *stream);

/* Release a handle (host and device memory).  NULL is ignored. */
void pars3_free(pars3_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* PARS3_H */
