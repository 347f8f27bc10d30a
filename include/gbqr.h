/*
 * gbqr.h - C ABI of a GB300 (sm_103a) library for recursive Householder QR
 * and least squares, after Ballard, Demmel, Grigori, Jacquelin, Knight,
 * "A 3D Parallel Algorithm for QR Decomposition" (arXiv 1805.05278).
 *
 * Method: the Elmroth-Gustavson recursion QR-EG (Algorithm 2, Section 2.4)
 * in Householder (compact-WY) representation (Section 2.3), whose base case
 * is TSQR over row blocks (Section 5, Appendix C) - the paper's 1D-CAQR-EG
 * (Section 6) restated for the SMs of one GPU.
 *
 * Conventions shared by every call:
 *   - Real FP64, column-major: element (i, j) of a matrix X with leading
 *     dimension ldx is X[i + j*ldx].  m >= n >= 0 (Section 2.1), except
 *     that gbqr_factor also takes wide matrices (m < n).
 *   - Matrix pointers are device pointers unless a call says otherwise.  The
 *     caller owns every matrix; the library only borrows the pointers for the
 *     duration of the stream-ordered work it enqueues.
 *   - Calls are asynchronous on the context's stream.  A returned status
 *     reports argument errors and launch failures; device-side conditions
 *     (non-finite input) are collected in a device-side record that
 *     gbqr_sync() reads.
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - Every int64_t size must be >= 0; leading dimensions must be >= max(1, rows).
 *
 * Householder representation returned by gbqr_factor (Section 2.3):
 *   Q = I - V T V^T, V unit lower trapezoidal (m x n, unit diagonal implied),
 *   T upper triangular, R upper triangular (n x n).  V's strict lower
 *   trapezoid and R's upper triangle overwrite A in place.  Reflector j is
 *   H_j = I - tau_j v_j v_j^T with beta_j = -sgn(alpha_j) ||column||,
 *   sgn(0) = +1 and no exception for an already-reduced column (tau_j = 2
 *   there) - the convention that the TSQR reconstruction of Appendix C.2
 *   produces, so that V, T and R are identical (up to rounding) to those of
 *   unblocked Householder QR.
 */
#ifndef GBQR_H
#define GBQR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GBQR_API __attribute__((visibility("default")))
#else
#define GBQR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbqr_ctx gbqr_ctx;

typedef enum {
    GBQR_OK = 0,
    GBQR_EINVAL = 1,       /* invalid argument (size, leading dimension, null pointer) */
    GBQR_ENOMEM = 2,       /* workspace too small or device allocation failed */
    GBQR_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    GBQR_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    GBQR_ENONFINITE = 5,   /* input held NaN or Inf (reported by gbqr_sync) */
    GBQR_ERANKDEF = 6,     /* least squares: R has an exactly zero diagonal entry */
    GBQR_EBUSY = 7,        /* context busy (e.g. workspace in use by queued work) */
    GBQR_EUNSUPPORTED = 8, /* valid request outside what this build implements */
    GBQR_ENOCONV = 9       /* least squares: mixed-precision refinement did not converge */
} gbqr_status;

/* Storage of the kernel T. */
typedef enum {
    /* n x n upper triangular T of the whole Q = I - V T V^T, as returned by
     * Algorithm 2 (pure QR-EG recursion, T assembled at every level). */
    GBQR_T_FULL = 0,
    /* nb x n: the n/nb diagonal blocks of T, block k (width w_k = min(nb,
     * n - k*nb)) at T[0:w_k, k*nb : k*nb + w_k].  Produced by a right-looking
     * top level over panels of width nb, each panel factored by QR-EG, so
     * the superdiagonal blocks of T are never formed (Section 8.4).
     * Q = Q_0 Q_1 ... with Q_k = I - V_k T_k V_k^T. */
    GBQR_T_PANEL = 1
} gbqr_t_layout;

typedef enum {
    GBQR_FP64 = 0,          /* every step in FP64 */
    GBQR_MIXED_BF16 = 1,    /* reserved: tensor-core update GEMMs + refinement */
    GBQR_MIXED_SPLITBF16 = 2,
    GBQR_FP32 = 3,
    GBQR_PREC_AUTO = 4      /* serving: mixed for large problems (n >= 256, m n^2 >= 1e9),
                               FP64 otherwise, FP64 again when refinement fails */
} gbqr_prec;

/* FP64 GEMM engine (gbqr_opts.fp64_gemm). */
#define GBQR_GEMM_DMMA 1
#define GBQR_GEMM_DFMA 2

/* Algorithm parameters.  Zero selects the library's tuned default. */
typedef struct {
    int32_t cutoff_b;   /* QR-EG base-case threshold b: base case when n <= b
                           (Algorithm 2); 1 <= b <= 64 */
    int32_t panel_nb;   /* GBQR_T_PANEL: top-level panel width nb (>= 1) */
    int32_t leaf_rows;  /* TSQR leaf height target m_p (>= b; Section 5 needs m_p >= n);
                           0 = about one leaf per SM, at least 128 rows, and up to
                           256 where that leaves one merge level instead of two */
    int32_t fanout;     /* TSQR reduction-tree fan-out k (2..16; the paper's
                           binomial tree is k = 2, Appendix C.1; 0 = the
                           fewest merge levels with k <= 16, k >= 8) */
    int32_t lookahead;  /* GBQR_T_PANEL: 0 or 1 = factor panel k+1 on a
                           high-priority internal stream while the rest of
                           panel k's trailing update runs (default); -1 = off */
    int32_t update_prec;/* GBQR_T_PANEL trailing-update products: GBQR_FP64
                           (default), GBQR_MIXED_BF16 (one BF16 slice) or
                           GBQR_MIXED_SPLITBF16 (three slices, FP32-level) on
                           the tensor cores.  Reflector generation, the TSQR
                           R-merges and the in-panel products stay FP64. */
    int32_t batch_streams; /* gbqr_factor_batched: streams to spread over (1..128) */
    int32_t fp64_gemm;  /* FP64 GEMM tiles of 64 x 64 outputs: 0 or GBQR_GEMM_DFMA
                           = CUDA-core FMA (default, measured faster);
                           GBQR_GEMM_DMMA = FP64 tensor cores (mma.sync
                           m8n8k4).  Both are deterministic and differ by
                           rounding only. */
} gbqr_opts;

/* Device-side record of one or more calls since the last gbqr_sync(). */
typedef struct {
    int64_t nonfinite;     /* non-zero if a NaN/Inf input was seen */
    int64_t zero_pivots;   /* reflectors whose column was exactly zero */
    int64_t rankdef_col;   /* least squares: first j with R(j,j) == 0, else -1 */
    int64_t refine_iters;  /* least squares, mixed precision: refinement steps taken */
    double refine_last;    /* ... and ||dx|| / ||x|| of the last step */
    int64_t gmres_steps;   /* least squares, mixed: Arnoldi steps of GMRES refinement */
    double backward_err;   /* least squares: ||A^T s|| / (||A||_F ||s|| + ||A||_F^2 ||x||), s = b - A x */
    int64_t reserved[1];
} gbqr_info;

/* Per-kernel-family totals of traced launches (see gbqr_trace_enable). */
typedef struct {
    char name[24];         /* "gemm", "tc_gemm", "tsqr_up", "tsqr_down", "trsv", "gemv", "other" */
    int64_t launches;
    double ms;             /* summed device time between launch-bracketing events */
    double flops;          /* summed algorithmic FP64 flops of those launches */
    double bytes;          /* summed algorithmic bytes (operands read + written once) */
} gbqr_trace_rec;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Allocates nothing on the device until a call needs workspace.
 * Errors: EINVAL (out NULL, bad device), ECUDA. */
GBQR_API gbqr_status gbqr_create(gbqr_ctx **out, int device, void *cuda_stream);

/* Synchronise the context's stream and release everything it owns. */
GBQR_API gbqr_status gbqr_destroy(gbqr_ctx *ctx);

/* Re-bind the context to another stream (work already queued stays where it is). */
GBQR_API gbqr_status gbqr_set_stream(gbqr_ctx *ctx, void *cuda_stream);

/* Caller-owned device workspace of `bytes` bytes (16-byte aligned), used
 * instead of library allocations.  It must stay valid until the work using
 * it completes.  ptr NULL returns to library-owned workspace (grown on demand
 * by cudaMalloc, outside any stream capture). */
GBQR_API gbqr_status gbqr_set_workspace(gbqr_ctx *ctx, void *ptr, size_t bytes);

/* Workspace bytes that gbqr_factor / gbqr_apply_* / gbqr_form_q /
 * gbqr_ls_solve need for an m x n problem with the given layout and options
 * (opts NULL = defaults).  Returns 0 for invalid sizes. */
GBQR_API size_t gbqr_workspace_bytes(int64_t m, int64_t n, int t_layout, const gbqr_opts *opts);

/* Wait for the context's stream, then copy out (and clear) the device-side
 * info record.  info may be NULL.  Returns ENONFINITE if non-finite input
 * was seen, else OK (or ECUDA for an asynchronous CUDA error). */
GBQR_API gbqr_status gbqr_sync(gbqr_ctx *ctx, gbqr_info *info);

/* ---- factorization (Algorithm 2 with TSQR base case) -------------------- */

/* QR-factor the m x n matrix A in place.
 *   A   (m x n, lda):  in: A.  out: V's strict lower trapezoid and R's upper
 *                      triangle (Householder representation, Section 2.3).
 *                      m >= n except for the wide case below.
 *   T   (ldt x n):     out: the kernel T in `t_layout` (GBQR_T_FULL: n x n,
 *                      ldt >= n, zeros written below the diagonal;
 *                      GBQR_T_PANEL: nb x n, ldt >= nb, nb = opts->panel_nb or
 *                      the default that gbqr_default_panel_nb reports).
 * Inductive case: n1 = floor(n/2); M1 = V_L^T A_R; M2 = T_L^T M1;
 * A_R -= V_L M2; recursion on the trailing block; T12 = -T_L (V_L^T [0; V_R]) T_R
 * (Algorithm 2).  Base case (n <= b): TSQR with leaf QR per CTA, a fan-out-k
 * tree of structured R merges, the downsweep that forms the leading columns
 * W of Q, and the Householder reconstruction X + S = LU, T = U S L^{-T},
 * R = -S R_tree, V = W U^{-1} (Appendix C).
 * A and T may instead both be HOST pointers (pageable or pinned): the call
 * then stages them through device workspace, copies the results back and
 * returns after the stream has synchronised.  With page-locked buffers and
 * the PANEL layout with look-ahead, the copies overlap the factorization:
 * panels 0 and 1 arrive first and the rest behind them on a copy stream,
 * and each panel's columns and T block are copied back as soon as that
 * panel is factored.
 * Wide A (m < n, Section 2.1): the leading m x m block is factored as above
 * and the m reflectors are applied to the remaining n - m columns, giving
 * R = [R1, Q^T A2] (upper trapezoidal) over A; T then holds the min(m, n) = m
 * reflectors' kernel (FULL: m x m; PANEL: nb x m), and apply_qt / apply_q /
 * form_q take n = m.  Device pointers only for wide A (host: EUNSUPPORTED).
 * Errors: EINVAL (lda < m, ldt too small, bad opts), ENOMEM, ECUDA,
 * EUNSUPPORTED. */
GBQR_API gbqr_status gbqr_factor(gbqr_ctx *ctx, int64_t m, int64_t n, double *A, int64_t lda,
                        double *T, int64_t ldt, int t_layout, const gbqr_opts *opts);

/* gbqr_factor in FP32: A (m x n, m >= n) and T are float DEVICE arrays and
 * every step computes in FP32 with the float instantiations of the same
 * kernels (TSQR, tiled GEMM); same layouts, options and look-ahead.
 * opts->update_prec must be GBQR_FP64 / 0 (no tensor-core updates); the
 * autotuner's cache is not used.  Errors: EINVAL (m < n, lda, ldt, opts),
 * EUNSUPPORTED (host pointers), ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_factor_f32(gbqr_ctx *ctx, int64_t m, int64_t n, float *A, int64_t lda,
                                     float *T, int64_t ldt, int t_layout, const gbqr_opts *opts);

/* Default top-level panel width for GBQR_T_PANEL on an m x n problem. */
GBQR_API int64_t gbqr_default_panel_nb(int64_t m, int64_t n);

/* ---- batched factorization and graph capture ---------------------------- */

/* count independent QR factorizations (the 1D-CAQR-EG instance of Section 6
 * for each matrix): A[i] (m[i] x n[i], lda[i], device) is factored in place
 * exactly as gbqr_factor does with GBQR_T_PANEL, T[i] (ldt[i] x n[i]) receives
 * its panel kernels.  m, n, A, lda, T, ldt are HOST arrays of count entries.
 * The matrices are spread over opts->batch_streams (default 128) internal streams (largest first, to
 * the least loaded stream), forked from and joined back to the context's
 * stream by events, so a capture of the context's stream (gbqr_graph_begin /
 * gbqr_graph_end) turns the whole batch into one graph launch.  Each stream
 * has its own workspace slice (gbqr_batched_workspace_bytes in total); the
 * first call creates the streams and grows library-owned workspace, so make
 * it before any capture.  opts apply to every matrix (panel_nb per matrix is
 * min(opts->panel_nb or 128, n[i]); the cutoff b defaults to 16 here).
 * Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_factor_batched(gbqr_ctx *ctx, int count, const int64_t *m, const int64_t *n,
                                         double *const *A, const int64_t *lda, double *const *T,
                                         const int64_t *ldt, const gbqr_opts *opts);

/* The same batch in FP32: A[i], T[i] are float, and every step - the TSQR
 * leaves, merges, reconstruction and the QR-EG update and T-assembly products
 * - computes in FP32 with the same kernels instantiated for float (this part
 * issues FP32 at 64x its FP64 rate, and the TSQR reflector chains shorten
 * accordingly).  Same layout, scheduling, streams, workspace and graph
 * capture rules as gbqr_factor_batched; opts->update_prec must be GBQR_FP64
 * (meaning: no tensor-core updates) or zero; the autotuner's cache is not
 * used.  Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_factor_batched_f32(gbqr_ctx *ctx, int count, const int64_t *m, const int64_t *n,
                                             float *const *A, const int64_t *lda, float *const *T,
                                             const int64_t *ldt, const gbqr_opts *opts);

/* Workspace bytes gbqr_factor_batched needs for these shapes (0 if invalid). */
GBQR_API size_t gbqr_batched_workspace_bytes(int count, const int64_t *m, const int64_t *n, const gbqr_opts *opts);

typedef struct gbqr_graph gbqr_graph;

/* Begin capturing the context's stream into a CUDA graph (relaxed capture
 * mode).  Every library call until gbqr_graph_end is recorded, not run; the
 * calls must not need new workspace or streams (make one uncaptured call
 * first).  Tracing must be off.  Errors: EINVAL, EBUSY, ECUDA. */
GBQR_API gbqr_status gbqr_graph_begin(gbqr_ctx *ctx);
/* End the capture and instantiate it; *out receives the graph. */
GBQR_API gbqr_status gbqr_graph_end(gbqr_ctx *ctx, gbqr_graph **out);
/* Launch a captured graph on the context's stream (asynchronous). */
GBQR_API gbqr_status gbqr_graph_launch(gbqr_ctx *ctx, gbqr_graph *g);
GBQR_API gbqr_status gbqr_graph_destroy(gbqr_graph *g);

/* ---- applying Q (basis-kernel update equation, Section 2.3) ------------ */

/* B <- Q^T B for the m x nrhs matrix B, with Q = I - V T V^T given by the
 * packed V\R (from gbqr_factor, lda) and T in `t_layout` (nb = panel width
 * for GBQR_T_PANEL, ignored for GBQR_T_FULL).
 * Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_apply_qt(gbqr_ctx *ctx, int64_t m, int64_t n, const double *VR, int64_t lda,
                          const double *T, int64_t ldt, int t_layout, int64_t nb,
                          int64_t nrhs, double *B, int64_t ldb);

/* B <- Q B (same arguments as gbqr_apply_qt). */
GBQR_API gbqr_status gbqr_apply_q(gbqr_ctx *ctx, int64_t m, int64_t n, const double *VR, int64_t lda,
                         const double *T, int64_t ldt, int t_layout, int64_t nb,
                         int64_t nrhs, double *B, int64_t ldb);

/* Thin Q: Q (m x n, ldq) <- Q [I_n; 0].  Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_form_q(gbqr_ctx *ctx, int64_t m, int64_t n, const double *VR, int64_t lda,
                        const double *T, int64_t ldt, int t_layout, int64_t nb,
                        double *Q, int64_t ldq);

/* ---- least squares (Section 2.1 problem, solved through the QR) -------- */

/* x = argmin ||A x - b||_2 for m x n A of full column rank (m >= n)
 * (Section 2.1), through the QR of a workspace copy of A (A itself is not
 * modified): c = Q^T b, x = R^{-1} c(0:n) by blocked back substitution.
 *   prec GBQR_FP64: every step in FP64 (the backward-stable solution).
 *   prec GBQR_MIXED_SPLITBF16 / GBQR_MIXED_BF16: the trailing-update
 *     products of the factorization run on the tensor cores (3 or 1 BF16
 *     slices, FP32 accumulation; reflectors and R-merges stay FP64), then
 *     the solution is refined on the augmented system [I A; A^T 0][r; x] =
 *     [b; 0] with FP64 residuals: each correction is GMRES on Bjorck's
 *     scaled system [aI A; A^T 0] (a ~ sigma_min / sqrt 2) preconditioned by
 *     the mixed factors (up to 8 corrections of at most 100 Arnoldi steps;
 *     GMRES-IR of Carson, Higham and Pranesh).  Unlike classical refinement
 *     it does not need kappa(A) u_f < 1 (u_f ~ 2^-22 for three slices).
 * Success means the normwise backward error
 *   eta = ||A^T s|| / (||A||_F ||s|| + ||A||_F^2 ||x||),  s = b - A x,
 * computed in FP64, is at most 4 u (1 + sqrt(m) ||s|| / (||s|| + ||A||_F ||x||))
 * (u = 2^-53: the level that rounding in forming s and A^T s leaves even for
 * the exact solution); the FP64 path always reports success (eta is
 * reported only).
 * b has m entries, x receives n (device pointers).  info (may be NULL)
 * receives rankdef_col, backward_err and, for the mixed path, refine_iters
 * (corrections applied), refine_last, gmres_steps.
 * Synchronous: returns after x is written.
 * Errors: EINVAL, ENOMEM, ECUDA, ERANKDEF (an exactly zero R(j,j)),
 * ENOCONV (mixed: backward error above target after refinement),
 * EUNSUPPORTED. */
GBQR_API gbqr_status gbqr_ls_solve(gbqr_ctx *ctx, int64_t m, int64_t n, const double *A, int64_t lda,
                          const double *b, double *x, int prec, gbqr_info *info);

/* ---- tensor-core GEMM (mixed precision building block) ----------------- */

/* C = alpha * op(A) * B + beta * C for FP64 column-major matrices, computed
 * on the tcgen05 tensor cores: each operand is split into nsplit (1..3) BF16
 * slices x = x_1 + ... (x_1 = bf16(x), x_2 = bf16(x - x_1), ...) and the
 * slice products x_i y_j with i + j <= nsplit + 1 are accumulated in FP32
 * (1, 3 or 6 products).  op(A) = A^T (A stored K x M) when transa != 0, else
 * A (stored M x K); B is stored K x N; C is M x N.  This is the product the
 * mixed-precision path uses for the update M1 = V^T A_R, A_R -= V M2 of
 * Algorithm 2 / the right-looking update (Section 8.4) in place of FP64.
 * Accuracy: about 2^-8, 2^-16, 2^-23 relative to |A||B| for nsplit 1, 2, 3
 * (FP32 accumulation over K adds ~K 2^-24).  Operand magnitudes must stay
 * within BF16's exponent range (|x| < 3e38; slices below ~1e-38 flush).
 * Asynchronous; needs workspace for the slices (grown automatically).
 * Errors: EINVAL, ENOMEM, ECUDA; a device-side timeout shows at gbqr_sync. */
GBQR_API gbqr_status gbqr_gemm_split_bf16(gbqr_ctx *ctx, int transa, int64_t M, int64_t N, int64_t K,
                                          double alpha, const double *A, int64_t lda, const double *B,
                                          int64_t ldb, double beta, double *C, int64_t ldc, int nsplit);

/* ---- autotuner ------------------------------------------------------------ */

/* The paper chooses its block sizes (the cutoff b of Algorithm 2, the TSQR
 * tree of Section 5 / Appendix C, the panel width of Section 8.4's
 * right-looking top level) from a cost model of a distributed machine.  Here
 * they are measured: coordinate descent from the library defaults over
 * cutoff_b {8,16,32,64}, fanout {adaptive,2,4,8,16}, leaf_rows {default,128,...,1024},
 * and for PANEL panel_nb {64,...,256} and lookahead, and for FP64 the GEMM
 * engine; each candidate is gbqr_factor on a synthetic m x n matrix, timed
 * with CUDA events on the context's stream (best of 2-5 runs after a
 * warm-up); a candidate must win by 1%.  Trials stop when the next would
 * overrun budget_ms of wall clock (the first measurement always runs).
 *
 * The winner is written to *best (every field explicit), its time to
 * *best_ms (may be NULL), and cached in the context for the power-of-two
 * class of (m, n), t_layout and update_prec.  Later calls of gbqr_factor and
 * gbqr_ls_solve on this context take the cached values for every option
 * field the caller leaves zero — except panel_nb: in gbqr_factor it fixes
 * the caller's T layout (pass best->panel_nb explicitly, with ldt >= it), and
 * gbqr_ls_solve keeps its default (the tuner times the factorization; the
 * solve's refinement applies Q panel by panel).
 * Synchronous; allocates m*n + 256*n doubles for the duration.
 * Errors: EINVAL (m < n, n < 1, bad layout/precision, FULL with mixed),
 * ENOMEM, ECUDA. */
#define GBQR_TUNE_FACTOR 0
#define GBQR_TUNE_BATCHED 1
GBQR_API gbqr_status gbqr_autotune(gbqr_ctx *ctx, int64_t m, int64_t n, int t_layout, int update_prec,
                                   double budget_ms, gbqr_opts *best, double *best_ms);

/* The same for gbqr_factor_batched on `count` matrices of shapes (m[i], n[i])
 * (synthetic contents, one buffer): batch_streams {16,...,128}, cutoff_b
 * {8,16,32}, fanout {adaptive,2,4,8,16}, leaf_rows {default,256,512}.  Each candidate
 * is captured into a CUDA graph on a private stream and its graph launches
 * are timed (the way a batch is meant to run; eager enqueueing of thousands
 * of launches is host-bound).  EBUSY while tracing is on.  Cached per
 * update_prec; gbqr_factor_batched then uses it for zero fields.  The cached
 * batch_streams changes the workspace gbqr_factor_batched needs: query
 * gbqr_batched_workspace_bytes with *best.  Allocates sum(m_i n_i + n_i^2)
 * doubles for the duration.  Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_autotune_batched(gbqr_ctx *ctx, int count, const int64_t *m, const int64_t *n,
                                           int update_prec, double budget_ms, gbqr_opts *best, double *best_ms);

/* The cached result for kind GBQR_TUNE_FACTOR (shape class of m, n; layout;
 * precision) or GBQR_TUNE_BATCHED (precision only).  EINVAL when none. */
GBQR_API gbqr_status gbqr_tuned_lookup(const gbqr_ctx *ctx, int kind, int64_t m, int64_t n, int t_layout,
                                       int update_prec, gbqr_opts *out);

/* ---- serving: least squares with continuous batching -------------------- */

typedef enum { GBQR_REQ_QUEUED = 0, GBQR_REQ_RUNNING = 1, GBQR_REQ_DONE = 2 } gbqr_req_state;

typedef struct {
    int64_t m, n;          /* problem size, m >= n >= 1 */
    const double *A;       /* device, m x n column-major (lda >= m), not modified */
    int64_t lda;
    const double *b;       /* device, m entries */
    double *x;             /* device, n entries: the solution */
    int32_t prec;          /* GBQR_FP64, GBQR_MIXED_*, or GBQR_PREC_AUTO */
    int32_t pad;
    uint64_t tag;          /* caller's label, echoed in the result */
} gbqr_request;

typedef struct {
    int32_t state;         /* gbqr_req_state */
    int32_t status;        /* gbqr_status of the solve (when done) */
    int32_t prec_used;     /* the precision that produced x */
    int32_t fell_back;     /* 1: GBQR_PREC_AUTO ran mixed, missed the target, re-ran FP64 */
    int64_t refine_iters;
    double queue_ms;       /* submit -> admitted */
    double run_ms;         /* admitted -> done */
    double latency_ms;     /* submit -> done */
    int64_t footprint_bytes; /* workspace + the request's A, b, x bytes, held against the cap */
    uint64_t tag;
    int32_t bypassed;      /* later requests admitted while this one waited (<= 8) */
    int32_t pad2;
} gbqr_result;

/* Start a serving loop on `device` attached to ctx: `workers` host threads,
 * each with a private context and stream, so admitted requests overlap on
 * the device; at most mem_cap_bytes of request footprint in flight.  A
 * request's footprint is its workspace (gbqr_workspace_bytes of its shape
 * and precision, + 1 MiB) plus its own A, b and x.  A queued request is
 * admitted (first fit, in arrival order) when a worker is free and its
 * footprint fits under the cap beside the running ones; at most 8 later
 * requests may be admitted ahead of a waiting one, after which it blocks the
 * queue until it fits (at the latest when nothing else runs).  Its workspace
 * comes from the stream-ordered allocator and returns on completion.  Each request runs
 * gbqr_ls_solve (Section 2.1 least squares through the QR); the kernels are
 * deterministic, so a result does not depend on what else is in flight.
 * Errors: EINVAL, EBUSY (already started), ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_server_start(gbqr_ctx *ctx, int device, int workers, size_t mem_cap_bytes);
/* Queue a request; *id receives its handle.  The request's buffers must stay
 * valid until it is done.  Errors: EINVAL, ENOMEM (footprint above the cap),
 * EBUSY (stopping). */
GBQR_API gbqr_status gbqr_submit(gbqr_ctx *ctx, const gbqr_request *req, uint64_t *id);
/* State of request id; wait != 0 blocks until it is done.  A done result is
 * returned once and then forgotten.  Errors: EINVAL (unknown id). */
GBQR_API gbqr_status gbqr_poll(gbqr_ctx *ctx, uint64_t id, int wait, gbqr_result *out);
/* Serve what is queued, then stop the workers. */
GBQR_API gbqr_status gbqr_server_stop(gbqr_ctx *ctx);

/* ---- tracing ------------------------------------------------------------ */

/* Turn launch tracing on (non-zero) or off.  While on, every kernel launch is
 * bracketed by CUDA events on the context's stream and its algorithmic
 * flops/bytes are counted. */
GBQR_API gbqr_status gbqr_trace_enable(gbqr_ctx *ctx, int on);

/* Synchronise, then write up to `max` per-family totals to out[] and their
 * number to *count; clears the trace. */
GBQR_API gbqr_status gbqr_trace_read(gbqr_ctx *ctx, gbqr_trace_rec *out, int max, int *count);

/* Number of kernel launches the context has issued since creation. */
GBQR_API int64_t gbqr_launch_count(const gbqr_ctx *ctx);

/* ---- allocation-free tall-skinny QR ------------------------------------ */

/* QR of a tall-skinny m x n matrix (n <= 32, m >= n) with no device
 * allocation and no context: the same TSQR kernels as the base case of
 * gbqr_factor (leaf QR, merge tree, downsweep, reconstruction), with the
 * tree's scratch in a fixed 16 MiB static device array instead of a
 * workspace.  The paper has no counterpart to this entry point.
 *
 * For callers that cannot call cudaMalloc: code that must not synchronise
 * the device (cudaMalloc/cudaFree can serialise with every stream), code
 * whose allocator owns the device memory budget and must see every byte,
 * and deployments that fix their device footprint at load time.  The caller
 * passes its input and outputs only.
 *   A (m x n, lda >= m): in: A; out: V (strict lower, unit diagonal implied)
 *                        and R (upper triangle), as gbqr_factor.
 *   T (n x n, ldt >= n): out: the n x n upper triangular kernel, zeros below.
 *   cuda_stream:         the cudaStream_t to enqueue on (asynchronous).
 * Every GPU that loads this library holds the 16 MiB array until the
 * process exits.  Under lazy module loading (CUDA_MODULE_LOADING=LAZY, the
 * default) the array comes into being on a device at the first call there,
 * which may therefore allocate and synchronise; under EAGER loading it exists
 * from context creation.  Make that first call at initialisation, and before
 * any stream capture: it also looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  All calls share the
 * array and it keeps the last call's contents; each call clears the tree's
 * arrival counters itself.  Calls that overlap on the GPU (other streams,
 * other host threads) race on the array: serialise them.  The tree is the one
 * gbqr_factor plans for an m x n base case (default leaf height, adaptive
 * fan-out).  Leaves are at most about 600 rows tall (shared memory) at
 * n = 32, so the array holds the tree of m up to about 400,000 rows there.
 * Larger m, n > 32, m < n or too small leading dimensions return EINVAL
 * before any CUDA call.
 * Errors: EINVAL, ECUDA, EUNSUPPORTED (device index >= 64). */
GBQR_API gbqr_status gbqr_tsqr_static(int64_t m, int64_t n, double *A, int64_t lda,
                                      double *T, int64_t ldt, void *cuda_stream);

/* ---- diagnostics -------------------------------------------------------- */

/* Measure the FP64 FMA throughput of CUDA device `device`: kind 0 = DFMA on
 * the CUDA cores, kind 1 = DMMA (mma.sync m8n8k4 f64 on the tensor cores).
 * Runs `iters` iterations of 8 independent chains per thread on 8 CTAs of
 * 256 threads per SM, best of 3 timed launches; *tflops receives TFLOP/s.
 * The paper has no counterpart: this is the denominator of the roofline
 * that the FP64 kernels are reported against.  Synchronous; allocates 8
 * bytes.  Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_fp64_peak(int device, int kind, int iters, double *tflops);

/* Failure-detection self-test: one CTA runs the bounded mbarrier wait of the
 * tensor-core GEMM (about 2 s by %globaltimer) on a barrier that nothing
 * arrives at.  Expected result: GBQR_ETIMEOUT with *completed = 0, and the
 * device still usable afterwards (the kernel returns instead of hanging).
 * The paper has no counterpart.  Synchronous (about 2 s); allocates 8 bytes.
 * Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_selftest_wait_timeout(int device, int *completed);

/* Failure-detection self-test of the persistent batched kernel: one CTA is
 * given a task whose dependency never completes, so its bounded wait (wait_ms,
 * 1..10000) must run out, raise the kernel's abort and timeout flags and
 * return.  Expected: GBQR_ETIMEOUT with *completed = 0, and the device still
 * usable.  The paper has no counterpart.  Synchronous; allocates 1 KB.
 * Errors: EINVAL, ENOMEM, ECUDA. */
GBQR_API gbqr_status gbqr_selftest_batched_wait(int device, int wait_ms, int *completed);

/* Failure-detection self-test of the persistent triangular-solve chain (and,
 * by the same wait, of the one-vector Q application): one CTA is handed the
 * second block of a two-block solve, so the block it waits for is never
 * solved and its bounded wait (wait_ms, 1..10000) must run out, raise the
 * abort and timeout flags, and return with the launch's counters reset.
 * Expected: GBQR_ETIMEOUT with *completed = 0 (no block solved), and the
 * device still usable.  The paper has no counterpart.  Synchronous;
 * allocates about 200 KB.  Errors: EINVAL, ENOMEM, ECUDA (also when the
 * counters were not left zero). */
GBQR_API gbqr_status gbqr_selftest_chain_wait(int device, int wait_ms, int *completed);

/* Human-readable name of a status. */
GBQR_API const char *gbqr_strerror(gbqr_status s);

#ifdef __cplusplus
}
#endif

#endif /* GBQR_H */
