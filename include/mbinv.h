/*
 * mbinv - memory-bounded block recursive inverse on one GB300 (sm_103a).
 *
 * Block Recursive Inversion (BRI) of Cosme, Fernandes, de Carvalho and
 * Xavier-de-Souza, "Memory-Usage Advantageous Block Recursive Matrix Inverse"
 * (arXiv:1612.00001).  For an n x n matrix M viewed as a k x k grid of b x b
 * blocks (b = n / k, Sec. 2 Eq. blockmatricesnxn), the library returns one
 * block N_ij of M^-1 at a time (Sec. 3, Eq. blockmatrix_NxN), all k^2 blocks
 * by k^2 independent runs (Sec. 5), or many independent problems at once.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major with an explicit leading dimension in elements.
 *   - Block indices are 0-based; the paper counts from 1.
 *   - A pointer may refer to host or device memory; the library asks the CUDA
 *     runtime which (cudaPointerGetAttributes).  Host buffers are copied
 *     through the library's own pinned staging.
 *   - Every call returns an mbinv_status; nothing is thrown across the ABI.
 *   - A context is used by one host thread at a time.  Calls are synchronous:
 *     when a call returns, its outputs are written (work runs on the stream
 *     given in the options).
 *   - The library never reads or writes past the sizes it is given.  Inputs
 *     are borrowed (never freed); outputs are owned by the caller.
 *   - Errors: MBINV_EINVAL for bad arguments (nothing is launched),
 *     MBINV_ENOMEM_CAP when the plan cannot fit device_cap_bytes (decided
 *     before any launch), MBINV_ESINGULAR when a b x b pivot the recursion
 *     must invert is singular to working precision (the paper assumes all of
 *     them are nonsingular, Sec. 1 and Sec. 3), MBINV_ECUDA for a CUDA error.
 */
#ifndef MBINV_H
#define MBINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBINV_OK = 0,
    MBINV_EINVAL = 1,
    MBINV_ENOMEM_CAP = 2,
    MBINV_ESINGULAR = 3,
    MBINV_ENOTCONV = 4,
    MBINV_ETIMEOUT = 5,
    MBINV_ECUDA = 6,
    MBINV_ENOTSUP = 7,
    MBINV_ECALLBACK = 8         /* a block producer (mbinv_block_fn) failed */
} mbinv_status;

/* Element type of M, of the outputs and of G / dM. */
typedef enum { MBINV_DTYPE_F64 = 0, MBINV_DTYPE_F32 = 1 } mbinv_dtype;

/* Arithmetic of the Schur-complement sweep.
 *   MBINV_FP64        every product and every b x b inverse in FP64.
 *   MBINV_FP32        every product and every inverse in FP32.
 *   MBINV_MIXED_BF16  Schur products on the tensor cores (tcgen05) with BF16
 *                     operand slices and FP32 accumulation, frame values kept
 *                     in FP32, every b x b pivot inverted in FP64; with
 *                     refine_steps = 1 the block is corrected by an FP64
 *                     block-row residual (see mbinv_block).
 *   MBINV_FP64_TC     frame values and b x b inverses in FP64 as MBINV_FP64;
 *                     the Schur products run on the BF16 tensor cores as
 *                     exact digit products: every row of the left operand
 *                     and every column of the right one is scaled by a power
 *                     of two, rounded to a 56-bit integer and split into 8
 *                     balanced base-128 digits; the 36 digit pairs whose
 *                     weights reach 2^-56 are summed exactly in FP32 and
 *                     recombined in integer arithmetic.  Each product then
 *                     carries an error below K 2^-53 max|row| max|column|
 *                     (the paper computes in plain FP64; this is a way to
 *                     run its FP64 products on the tensor pipe). */
typedef enum { MBINV_FP64 = 0, MBINV_FP32 = 1, MBINV_MIXED_BF16 = 2, MBINV_FP64_TC = 3 } mbinv_precision;

/* Order of evaluation (Sec. 5-6: the method's point is a bounded memory
 * footprint; its cost is recomputation or, here, traffic to host memory).
 *   MBINV_SCHEDULE_AUTO     level by level when that fits device_cap_bytes,
 *                           else MBINV_SCHEDULE_BOUNDED; M stays in host
 *                           memory when it is there and its device copy
 *                           alone would not fit the cap.
 *   MBINV_SCHEDULE_LEVELS   level by level, every frame of an order in the
 *                           same grouped launches; MBINV_ENOMEM_CAP when the
 *                           smallest chunking does not fit.
 *   MBINV_SCHEDULE_BOUNDED  depth first, one operation per launch sequence,
 *                           in as many b x b device slots as the cap leaves;
 *                           values needed again later wait in pinned host
 *                           memory (the one needed last goes first), and a
 *                           host M is read block by block as it is needed.
 *                           Not with MBINV_MIXED_BF16 or k not dividing n
 *                           (MBINV_ENOTSUP). */
typedef enum { MBINV_SCHEDULE_AUTO = 0, MBINV_SCHEDULE_LEVELS = 1, MBINV_SCHEDULE_BOUNDED = 2 } mbinv_schedule;

/* The method.
 *   MBINV_VARIANT_PAPER      the paper's recursion (Sec. 3): frames of non-
 *                            principal submatrices reduced by their roles'
 *                            Schur complements, memoized and merged.
 *   MBINV_VARIANT_PRINCIPAL  the reformulation around the Schur complement
 *                            M/A of Eq. SchurofA that the paper names as
 *                            future work (Sec. 8): the blocks other than i
 *                            and j are eliminated in ascending order with
 *                            principal pivots S[c][c] (S the running Schur
 *                            complement), then N_ii = S_ii^-1, or for i != j
 *                            N_ij = -S_ii^-1 S_ij (S_jj - S_ji S_ii^-1 S_ij)^-1.
 *                            Principal pivots keep the stability of block
 *                            elimination (and exist wherever the principal
 *                            minors do); the work is about (2/3) k^3 b^3 per
 *                            block.  M on the device, k dividing n, no
 *                            MBINV_MIXED_BF16, blocks returned in the working
 *                            type; else MBINV_ENOTSUP. */
typedef enum { MBINV_VARIANT_PAPER = 0, MBINV_VARIANT_PRINCIPAL = 1 } mbinv_variant;

typedef struct {
    size_t struct_size;         /* sizeof(mbinv_options) */
    mbinv_precision precision;
    size_t device_cap_bytes;    /* bound on the library's device memory
                                   (workspace plus its own copy of M);
                                   0 = no bound */
    int refine_steps;           /* 0 or 1: one two-sided refinement step
                                   (see mbinv_block), any precision */
    int bf16_slices;            /* MIXED_BF16 only: operands split into
                                   1, 2 or 3 BF16 slices (1, 3 or 6
                                   products) */
    void *cuda_stream;          /* cudaStream_t; NULL = default stream */
    uint64_t pad_seed;          /* seed of the coupling block used when k
                                   does not divide n */
    int profile;                /* 1: time every launch with CUDA events and
                                   report device seconds per kernel family */
    int schedule;               /* an mbinv_schedule: how the frames are
                                   ordered and where M lives */
    int out_dtype;              /* type of the returned blocks: 0 = M's
                                   type, 1 = FP64, 2 = FP32 (an FP32 M whose
                                   blocks are computed in FP64 can return
                                   them in FP64) */
    double sing_tol;            /* a pivot is singular when its largest
                                   candidate is at most sing_tol times the
                                   matrix's largest magnitude; 0 = b times
                                   the unit roundoff of the working type */
    int variant;                /* an mbinv_variant: the paper's recursion
                                   or the principal-Schur variant */
    int pivot_cond;             /* 1: estimate ||P||_1 ||P^-1||_1 of every
                                   inverted pivot (reported as
                                   max_pivot_cond; about 2% of a step) */
    int no_graphs;              /* 1: never replay a CUDA graph.  0: a call
                                   whose launch sequence equals the previous
                                   call's on this context (same blocks,
                                   buffers and schedule; not profiled; no
                                   host copies) is captured into a graph
                                   the second time and replayed after */
    int reserved;
    const char *tune_cache_path; /* file written by mbinv_autotune (may be
                                   NULL): its tuned panel-cluster settings are
                                   loaded when the context is created */
} mbinv_options;

typedef struct {
    double gemm_flops;          /* algorithmic flops of the Schur products
                                   (2 m n k each) */
    double inv_flops;           /* 2 b^3 per b x b inverse */
    double seconds;             /* wall time of the call */
    double rel_residual;        /* refined path: ||E_i^T - X_i M||_F / sqrt(b) */
    size_t peak_device_bytes;   /* high-water mark of the library's device
                                   memory during the call: the bytes it held
                                   allocated (its copy of M included),
                                   counted at every allocation and free */
    size_t frames;              /* frames evaluated: frames that compute the
                                   same value are evaluated once for all the
                                   requests of a call (see request_frames) */
    size_t inversions;          /* b x b inverses performed */
    size_t launches;            /* kernel launches issued */
    int64_t failed_pivot;       /* on MBINV_ESINGULAR: index of the failing
                                   inverse in launch order, else -1 */
    double gemm_device_seconds; /* profile = 1: device time of the Schur
                                   product launches */
    double inv_device_seconds;  /* profile = 1: device time of the inverse
                                   launches */
    size_t gemm_launches;       /* Schur product launches */
    double pack_device_seconds; /* profile = 1: device time of operand
                                   packing (FP64_TC digits, MIXED_BF16
                                   slices) */
    double inv_panel_device_seconds; /* profile = 1: the part of
                                   inv_device_seconds spent in the panel
                                   factorisations */
    double inv_panel_flops;     /* algorithmic flops of the panel
                                   factorisations: 2 b w^2 per panel of
                                   width w */
    double inv_update_flops;    /* algorithmic flops of the trailing
                                   updates: 2 b w (b - w) per panel (with
                                   inv_panel_flops, 2 b^3 per inverse) */
    size_t inv_panel_launches;  /* profile = 1: panel factorisation launches
                                   timed in inv_panel_device_seconds */
    size_t request_frames;      /* frames the requests would evaluate run
                                   one by one (each request's own distinct
                                   frames, summed); frames <= request_frames */
    size_t planned_device_bytes; /* the planner's reckoning of the same
                                   high-water mark, made before any launch */
    double pack_bytes;          /* algorithmic bytes of operand packing:
                                   FP64_TC 8 B read and 16 B of digits
                                   written per operand entry, 4 B per row */
    double host_in_bytes;       /* bounded schedule: bytes copied host ->
                                   device (blocks of a host M, values
                                   brought back) */
    double host_out_bytes;      /* bounded schedule: bytes of values spilled
                                   to host memory */
    size_t host_spill_bytes;    /* bounded schedule: pinned host memory the
                                   spilled values took at once */
    size_t graph_replays;       /* launch sequences replayed from a CUDA
                                   graph during the call */
    double max_pivot_cond;      /* pivot_cond = 1: largest 1-norm condition
                                   estimate ||P||_1 ||P^-1||_1 over the
                                   inverted pivots (0 when not computed) */
} mbinv_report;

typedef struct mbinv_ctx mbinv_ctx;

/* Producer of M for a context that does not store it (Sec. 5: a matrix that
 * can be computed element by element need not be stored, as in LS-SVM
 * training).  Writes M[r0 : r0 + rows, c0 : c0 + cols] (element offsets,
 * 0-based) into dst - device memory, row-major, leading dimension ldd, of
 * type dtype (an mbinv_dtype) - with its work ordered on the CUDA stream
 * `stream`, which it must not synchronise with other streams' work on dst.
 * Returns 0, or nonzero to fail the call with MBINV_ECALLBACK. */
typedef int (*mbinv_block_fn)(int64_t r0, int64_t c0, int64_t rows, int64_t cols, void *dst, int64_t ldd,
                              int dtype, void *stream, void *user);

/* The LS-SVM matrix of Sec. 7, Eq. A, as a producer: with n points x_1..x_n
 * of dimension dim,
 *     A_gamma = [[0, 1^T], [1, K + I / gamma]],  K_pq = exp(-|x_p - x_q|^2 / (2 sigma^2)),
 * of order n + 1 (row and column 0 are the border).  Pass mbinv_rbf_block as
 * the producer and a mbinv_rbf* as user; x is device memory, n x dim
 * row-major FP64, and must stay valid while the context is used.  Entries
 * are computed in FP64 on the GPU (and rounded to dtype). */
typedef struct {
    const double *x;
    int64_t n, dim;
    double sigma, gamma;
} mbinv_rbf;
int mbinv_rbf_block(int64_t r0, int64_t c0, int64_t rows, int64_t cols, void *dst, int64_t ldd, int dtype,
                    void *stream, void *user);

/* Called after each finished block by mbinv_all_blocks. */
typedef void (*mbinv_block_done_cb)(int64_t i, int64_t j, void *user);

/* One independent problem of mbinv_batched_blocks. */
typedef struct {
    int64_t n, k;               /* order of M and blocks per side */
    int64_t i, j;               /* requested block, 0-based */
    const void *M;              /* row-major, leading dimension ld, dtype of
                                   the batch; host or device */
    int64_t ld;
    void *out;                  /* b_i x b_j result, leading dimension ldo */
    int64_t ldo;
    int status;                 /* written: mbinv_status of this problem */
} mbinv_problem;

/* Fills *opt with defaults: FP64, no cap, no refinement, 3 slices, default
 * stream, pad_seed 0. */
void mbinv_default_options(mbinv_options *opt);

/* Creates a context for an n x n matrix split into k x k blocks
 * (Sec. 2, Eq. blockmatricesnxn).  When k does not divide n the matrix is
 * bordered to order k * ceil(n/k) (Sec. 3, Eq. M_augmented; see mbinv_block
 * for the border used).  M is borrowed.  Device memory: it must stay valid
 * and unchanged until mbinv_destroy.  Host memory: it is copied to the device
 * during this call, unless the bounded schedule keeps it in host memory
 * (schedule MBINV_SCHEDULE_BOUNDED, or MBINV_SCHEDULE_AUTO with a cap that
 * the device copy plus 16 b x b value slots would exceed; k must divide n
 * and k >= 2): then it is read block by block during the calls and must stay
 * valid and unchanged until mbinv_destroy, pinned host memory being the
 * fastest.  dtype is an mbinv_dtype.  opt may be NULL. */
mbinv_status mbinv_create(mbinv_ctx **out, int64_t n, int64_t k, int dtype, const void *M, int64_t ld,
                          const mbinv_options *opt);

/* Re-reads M after the caller changed its contents (same buffer, shape and
 * dtype as given to mbinv_create): the next problem of a stream of matrices
 * of one shape, without a new context (its plans, workspace and captured
 * launch graphs stay).  A context that copied M to the device (host M; device
 * M that is padded or converted) copies it again on the context's stream and
 * returns when the copy is complete; a context that reads the caller's
 * buffer in place (device M of the sweep's type, host-resident M of the
 * bounded schedule) or produces M has nothing to refresh and returns
 * MBINV_OK.  The caller's buffer must be valid for the call; with host
 * memory it is free to change again once the call returns. */
mbinv_status mbinv_reload(mbinv_ctx *ctx);

/* A context whose M (n x n, type dtype) is produced on demand by fn and
 * never stored: every block the recursion reads is written by fn into a
 * device value slot just before its use, under the bounded schedule (depth
 * first; with a cap, values needed later wait in pinned host memory).  k
 * must divide n and be at least 2 (else MBINV_ENOTSUP), and MBINV_MIXED_BF16
 * and refine_steps = 1 are not supported (the refinement residual reads all
 * of M).  fn and user must stay valid until mbinv_destroy. */
mbinv_status mbinv_create_from_fn(mbinv_ctx **out, int64_t n, int64_t k, int dtype, mbinv_block_fn fn, void *user,
                                  const mbinv_options *opt);

/* N_ij, the b x b block (i, j) of M^-1 (Sec. 3.1-3.2, Eq. blockmatrix_NxN;
 * any block through a permutation of block rows and columns, Sec. 3.2 last
 * paragraph).  out is b_i x b_j with leading dimension ldo, in M's dtype,
 * host or device; b_i = b except for the last block when k does not divide n.
 * When k does not divide n, the border is [[M, 0], [0, I]] for requests that
 * do not touch the padded block or sit on the diagonal, [[M, B'], [0, I]] for
 * (i, k-1), [[M, 0], [C', I]] for (k-1, j), B' and C'^T uniform in [-1, 1)
 * drawn by SplitMix64 from pad_seed; the top-left n x n block of each
 * bordered inverse is M^-1.  report may be NULL.
 * With refine_steps = 1 the call also computes block row i (X_i) and block
 * column j (Y_j) of the inverse with the same sweep (kept in FP32 on the
 * FP32-valued paths, FP64 on FP64 and FP64_TC) and returns
 * X_i E_j + (E_i^T - X_i M) Y_j, the residual and the correction taken in
 * FP64: the result's error is -dX M dY, the product of the sweep's errors
 * (the method is not in the paper).  MBINV_ENOTCONV when the residual's
 * scaled norm is not below 1. */
mbinv_status mbinv_block(mbinv_ctx *ctx, int64_t i, int64_t j, void *out, int64_t ldo, mbinv_report *report);

/* Several blocks of M^-1, each by its own run of the recursion (Sec. 3.1-3.2,
 * the k^2-runs reading of Sec. 5), the runs executed together.  Their frames
 * are merged by what they compute - a frame that several runs (or several
 * branches of one run) compute from the same operand frames is evaluated
 * once, the reuse across branches that Sec. 8 proposes - and every level of
 * the merged recursion goes out in grouped launches.  A merged frame rounds
 * exactly as in each run alone, so every block equals, bit for bit, the block
 * its run alone returns.  ij holds count pairs (i, j); outs[t] (host or
 * device, M's dtype) receives block (ij[2t], ij[2t+1]) with leading dimension
 * ldos[t].  width bounds how many runs are merged (0 = 8), and the cap may
 * lower it.  With refine_steps = 1 every block is refined as in mbinv_block,
 * each needed block row and column computed once (their runs merged width at
 * a time). */
mbinv_status mbinv_blocks(mbinv_ctx *ctx, int64_t count, const int64_t *ij, void *const *outs, const int64_t *ldos,
                          int width, mbinv_report *report);

/* All blocks of M^-1 by k^2 runs (Sec. 5).  Without a cap all runs are
 * merged as in mbinv_blocks (k = 8: 6116 distinct frames instead of 64 x 270);
 * under a cap one block row at a time, split further if the cap asks.  out is
 * n x n with leading dimension ldo (host or device).  done (may be NULL) is a
 * k*k row-major bitmap of blocks to skip; cb (may be NULL) is called for each
 * finished block once its chunk (all blocks, or its block row under a cap) is
 * written, so a caller can checkpoint and resume: blocks computed in a resumed
 * call are bit for bit those of an uninterrupted one. */
mbinv_status mbinv_all_blocks(mbinv_ctx *ctx, void *out, int64_t ldo, const uint8_t *done, mbinv_block_done_cb cb,
                              void *user, mbinv_report *report);

/* Block row i of M^-1 (b_i x n, leading dimension ldo): k runs of the
 * recursion, one per block, executed together. */
mbinv_status mbinv_block_row(mbinv_ctx *ctx, int64_t i, void *out, int64_t ldo, mbinv_report *report);

/* Block column j of M^-1 (n x b_j, leading dimension ldo). */
mbinv_status mbinv_block_col(mbinv_ctx *ctx, int64_t j, void *out, int64_t ldo, mbinv_report *report);

/* Adjoint of L = sum(G .* N_ij) with respect to M:
 *   dM += -(X_i)^T G (Y_j)^T,  X_i = block row i, Y_j = block column j of M^-1,
 * both recomputed block by block with the recursion.  G is b_i x b_j
 * (leading dimension ldg), dM is n x n (leading dimension ldd) and is
 * accumulated into, both in M's dtype, host or device.  On MBINV_FP64 and
 * MBINV_FP64_TC the rows, columns and products are FP64 (digit products on
 * the tensor cores on FP64_TC), and with refine_steps = 1 every block of
 * M^-1 is first computed (runs merged) and that whole approximate inverse
 * N~ is improved by Newton-Schulz steps N~ <- N~ + N~ (I - M N~), each of
 * which squares ||I - M N~|| (converging when it is below 1), until that
 * residual stops falling (at most 12; the best N~ is kept and its residual
 * reported in rel_residual), X_i and Y_j then being its block row and
 * column (3 n^2 doubles of device memory; M on the device, k dividing n,
 * else MBINV_ENOTSUP).  The paper has no gradient; this is the derivative of
 * its output. */
mbinv_status mbinv_backward(mbinv_ctx *ctx, int64_t i, int64_t j, const void *G, int64_t ldg, void *dM, int64_t ldd,
                            mbinv_report *report);

/* Many independent problems (the paper's blocks are embarrassingly parallel,
 * Sec. 8), all in dtype with the options opt (may be NULL).  Each problem's
 * status field is written; the return value is MBINV_OK when every problem
 * succeeded, else the first failing status.  The problems' runs are executed
 * together, level by level, in grouped launches that mix orders b (in waves
 * whose summed workspace fits device_cap_bytes); MIXED_BF16 with
 * refine_steps = 1 is not supported here (MBINV_ENOTSUP). */
mbinv_status mbinv_batched_blocks(int64_t count, mbinv_problem *probs, int dtype, const mbinv_options *opt,
                                  mbinv_report *report);

void mbinv_destroy(mbinv_ctx *ctx);

/* Autotuner of the pivot inverses' panel factorisation (the leaf and level
 * inverses of the recursion, Sec. 5 and 7): for count matrices of order b
 * inverted together in `precision`, times the batched inversion of count
 * synthetic matrices (uniform[-1, 1) + b I) with the panel's thread-block
 * clusters scaled by 2^bias, bias = -2..2 around the built-in rule, keeps the
 * fastest (it applies to every later batch of that order and size in the
 * process) and appends "b count precision bias seconds" to cache_path (may be
 * NULL), which a context reads back through tune_cache_path.  The cluster
 * size changes where rows are eliminated, not how: results are bit for bit
 * the same.  *best_bias and *best_seconds (either may be NULL) receive the
 * choice and its device time per batch.  Allocates and frees its own
 * scratch (count x b x b doubles and the inverses' workspace). */
mbinv_status mbinv_autotune(int64_t b, int64_t count, int precision, const char *cache_path, int *best_bias,
                            double *best_seconds);

/* Largest order accepted by mbinv_invert_noalloc. */
#define MBINV_NOALLOC_MAX_B 512

/* X = A^-1 for one b x b matrix, by the same pivoted Gauss-Jordan kernels the
 * recursion uses for its pivots (FP64 arithmetic), for callers that cannot
 * allocate device memory when they call: for instance code running while a
 * framework's caching allocator holds nearly all of the GPU's memory, or code
 * that must not pay the device-wide synchronisation of cudaFree.  The paper
 * has no counterpart; this is an entry point of the library only.
 *   A, X:   device pointers, row-major, leading dimensions lda, ldx >= b,
 *           dtype MBINV_DTYPE_F64 or MBINV_DTYPE_F32 (both the same).
 *   b:      1 <= b <= MBINV_NOALLOC_MAX_B; anything else returns
 *           MBINV_EINVAL before any launch.
 *   stream: cudaStream_t (NULL = default stream); the call returns once the
 *           result is written.
 * Returns MBINV_ESINGULAR when a pivot is singular to working precision.
 * All scratch (about 2.2 MB) is one fixed device array per GPU, held from the
 * library's load until the process exits; no cudaMalloc, cudaFree or other
 * allocating routine is called.  Every call on a device shares that array and
 * overwrites what it uses, so calls whose GPU work overlaps (two threads or
 * two streams) race: serialise them.  Each call waits on the host for its
 * own result (it reads its status word back before returning).  The first
 * call on a device also looks up the array's device address with that device
 * current; that first call should come before any stream capture. */
mbinv_status mbinv_invert_noalloc(const void *A, int64_t lda, void *X, int64_t ldx, int64_t b, int dtype,
                                  void *stream);

const char *mbinv_status_string(mbinv_status s);

/* Library version string. */
const char *mbinv_version(void);

/* Text of the last CUDA error seen by this thread (after MBINV_ECUDA). */
const char *mbinv_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MBINV_H */
