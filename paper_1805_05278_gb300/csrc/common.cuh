// Internal declarations shared by the library's translation units.
// Not part of the C ABI (see include/gbqr.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gbqr.h"

namespace gbqr {

constexpr int kThreads = 256;   // threads per CTA for every kernel family
constexpr int kMaxPanel = 64;   // largest TSQR panel width w (= cutoff b)
constexpr int kMaxBatchB = 32;  // largest panel width of the persistent batched kernel

// ---------------------------------------------------------------- tracing
enum Family { FAM_GEMM = 0, FAM_TC_GEMM, FAM_TSQR_UP, FAM_TSQR_DOWN, FAM_TRSV, FAM_GEMV, FAM_OTHER, FAM_BATCHED, FAM_COUNT };

struct Tracer {
    virtual void begin(cudaStream_t s, Family f) = 0;
    virtual void end(cudaStream_t s, Family f, double flops, double bytes) = 0;
    virtual ~Tracer() {}
};

// Everything a launcher needs besides its operands.
struct Exec {
    cudaStream_t stream = nullptr;
    Tracer *tracer = nullptr;   // null = tracing off
    int64_t *launches = nullptr;
    int num_sms = 152;
    int device = 0;
    bool dmma = false;          // 64 x 64 FP64 GEMM tiles on the FP64 tensor cores (else DFMA)
};

inline void trace_begin(const Exec &ex, Family f) {
    if (ex.tracer) ex.tracer->begin(ex.stream, f);
}
inline gbqr_status trace_end(const Exec &ex, Family f, double flops, double bytes) {
    if (ex.launches) ++*ex.launches;
    if (ex.tracer) ex.tracer->end(ex.stream, f, flops, bytes);
    return cudaPeekAtLastError() == cudaSuccess ? GBQR_OK : GBQR_ECUDA;
}

// ------------------------------------------------------------------ GEMM
// Structural masks on a STORED operand (row r, column c of the array as laid
// out in memory, before any transpose).
enum Mask {
    MASK_NONE = 0,
    MASK_UNIT_LOWER = 1,  // r < c -> 0, r == c -> 1, r > c -> stored value (a V basis)
    MASK_UPPER = 2        // r > c -> 0 (a T kernel or an R factor)
};

// C (M x N) = alpha * op(A) * op(B) + beta * C.
//   ta == false: A stored M x K;  ta == true: A stored K x M, op(A) = A^T.
//   B is stored K x N (no transpose needed by any caller).
template <class Real>
struct GemmOpT {
    int64_t M = 0, N = 0, K = 0;
    const Real *A = nullptr; int64_t lda = 1; bool ta = false; int maskA = MASK_NONE;
    const Real *B = nullptr; int64_t ldb = 1; int maskB = MASK_NONE;
    Real *C = nullptr; int64_t ldc = 1;
    Real alpha = Real(1), beta = Real(0);
};
using GemmOp = GemmOpT<double>;

// Scratch for split-K: partial tiles and self-resetting per-tile counters
// (must be zero before the first use; every launch leaves them zero).
template <class Real>
struct GemmScratchT {
    Real *partial = nullptr; size_t partial_elems = 0;
    unsigned *counters = nullptr; size_t ncounters = 0;
};
using GemmScratch = GemmScratchT<double>;

size_t gemm_partial_elems_max(int num_sms);   // the most split-K scratch the planner can use
size_t gemm_partial_elems_min(int num_sms);   // enough for 4 split CTAs per SM
size_t gemm_counters_max(int num_sms);
// Real = double (FP64 path) or float (FP32 batched path)
template <class Real>
gbqr_status gemm(const Exec &ex, const GemmOpT<Real> &op, const GemmScratchT<Real> &sc);
// Algorithmic flops of op (structural zeros of masked operands excluded).
template <class Real>
double gemm_algorithmic_flops(const GemmOpT<Real> &op);

#define TRY_ST(x) do { gbqr_status _s = (x); if (_s != GBQR_OK) return _s; } while (0)

// ------------------------------------------------------ tensor-core GEMM
// C (FP64, M x N) = alpha * op(A) * B + beta * C with op(A) = A^T when ta
// (A stored K x M) or A (stored M x K), B stored K x N, on tcgen05 tensor
// cores as the sum of BF16 slice products (nsplit slices per operand, FP32
// accumulation).  Masks as for gemm().
struct TcGemmOp {
    int64_t M = 0, N = 0, K = 0;
    const double *A = nullptr; int64_t lda = 1; bool ta = false; int maskA = MASK_NONE;
    const double *B = nullptr; int64_t ldb = 1; int maskB = MASK_NONE;
    double *C = nullptr; int64_t ldc = 1;
    double alpha = 1.0, beta = 0.0;
    int nsplit = 3;
};
struct TcScratch {
    void *base = nullptr; size_t bytes = 0;   // slices + split-K partials
    int *err = nullptr;                       // device flag raised on a timed-out wait
};
size_t tc_gemm_scratch_bytes(int64_t M, int64_t N, int64_t K, int num_sms);
// The driver's cuTensorMapEncodeTiled (as a PFN_cuTensorMapEncodeTiled_v12000),
// or null when the driver does not provide it.
void *tensor_map_encoder();
gbqr_status tc_gemm(const Exec &ex, const TcGemmOp &op, const TcScratch &sc);

// ------------------------------------------------------------------ TSQR
// Base case of Algorithm 2: TSQR of an mp x w panel (Section 5, Appendix C).
struct TsqrPlan {
    int64_t mp = 0; int w = 0;
    int P = 1;          // leaves (CTAs of the leaf stage)
    int k = 2;          // tree fan-out
    int L = 0;          // tree levels above the leaves
    int hmax = 0;       // tallest leaf
    int ldS = 0;        // up kernel shared-memory leading dimension (>= hmax, >= k*w)
    int ldW = 0;        // down kernel shared-memory leading dimension (>= hmax)
    int64_t nodes = 0;  // leaves + internal nodes
    size_t smem_up = 0, smem_down = 0;
    // workspace element counts
    size_t nR = 0, nT = 0, nY = 0, nX = 0, ncount = 0;
};

template <class Real>
struct TsqrWorkT {
    Real *R = nullptr, *T = nullptr, *Y = nullptr, *X = nullptr;
    unsigned *counters = nullptr;   // zero before first use; left zero
};
using TsqrWork = TsqrWorkT<double>;

// Plan for an mp x w panel.  leaf_rows = target leaf height (0 = default),
// fanout in [2, 16], or 0: the fewest merge levels a fan-out k <= 16 gives
// (the smallest such k >= 8).  Returns false if the panel cannot be planned.
bool tsqr_plan(int64_t mp, int w, int leaf_rows, int fanout, int num_sms, TsqrPlan *plan);
// Worst-case plan sizes over panels of height <= mp and width <= w.
TsqrPlan tsqr_plan_bound(int64_t mp, int w, int leaf_rows, int fanout, int num_sms);
// Real = double (FP64 path) or float (FP32 batched path); the plan's shared
// memory sizes are the FP64 ones (enough for either).
template <class Real>
gbqr_status tsqr_run(const Exec &ex, const TsqrPlan &plan, Real *A, int64_t lda,
                     Real *Tout, int64_t ldt, const TsqrWorkT<Real> &work);

// ---------------------------------------------------- persistent batched QR
// Many independent QRs in one launch (batched.cu): a plan (task list in
// list-schedule order, workspace layout) is cached per set of shapes; each
// call uploads the matrix table and the task list and launches one
// persistent kernel.  T layout: panel kernels of width b (PANEL, nb = b).
struct BatchPlan;
void batch_plan_free(BatchPlan *pl);
double batch_plan_estimate_ms(const BatchPlan *pl);
size_t batched_plan_bytes(const BatchPlan *pl);
// Validates the shapes and returns the cached plan, building it when it is
// missing and may_build (else EBUSY).
template <class Real>
gbqr_status batched_plan(BatchPlan **cache, int device, int num_sms, int count, const int64_t *m,
                         const int64_t *n, const int64_t *lda, const int64_t *ldt, int b, bool may_build,
                         BatchPlan **out);
// Enqueues the table upload, the counter reset and the launch on ex.stream.
// capturing: the table is staged in page-locked memory returned in *owned,
// which the captured graph must keep alive.
template <class Real>
gbqr_status batched_enqueue(const Exec &ex, BatchPlan *pl, Real *const *A, Real *const *T, const int64_t *m,
                            const int64_t *n, const int64_t *lda, const int64_t *ldt, char *ws, size_t ws_bytes,
                            int *timeout_flag, unsigned long long *nonfinite, bool capturing, void **owned);

// ------------------------------------------------------------ small kernels
gbqr_status fill_identity(const Exec &ex, int64_t m, int64_t n, double *Q, int64_t ldq);
gbqr_status zero_strict_lower(const Exec &ex, int64_t n, double *T, int64_t ldt);
gbqr_status copy_matrix(const Exec &ex, int64_t m, int64_t n, const double *src, int64_t lds,
                        double *dst, int64_t ldd);
template <class Real>
gbqr_status scan_nonfinite(const Exec &ex, int64_t m, int64_t n, const Real *A, int64_t lda,
                           unsigned long long *flag);
// x (n) <- R^{-1} x, R upper triangular n x n (ldr); records the first zero
// diagonal index (or leaves *rankdef untouched) via atomicMin.
// Dinv (optional): inverses of R's 64 x 64 diagonal blocks from
// trsv_block_inverses; each block step is then a small matrix-vector product
// instead of a substitution chain (the mixed path's repeated solves).
gbqr_status trsv_upper(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *x,
                       long long *rankdef, const double *Dinv = nullptr);
gbqr_status trsv_block_inverses(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *Dinv,
                                long long *rankdef);
constexpr int kTrsvBlockSize = 64;

// x (n) <- R^{-T} x (forward substitution with the lower triangle R^T).
gbqr_status trsv_upper_t(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *x, long long *rankdef,
                         const double *Dinv = nullptr);
// y = alpha A x + beta y (A m x n); partial: >= m * chunks doubles of scratch.
// mask MASK_UNIT_LOWER treats A as a unit lower trapezoidal basis.
gbqr_status gemv_n(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, const double *x, double alpha,
                   double beta, double *y, double *partial, size_t partial_elems, int mask = MASK_NONE);
// g = alpha A^T r + beta g
gbqr_status gemv_t(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, const double *r, double alpha,
                   double beta, double *g, int mask = MASK_NONE);
// out[0] = ||x||^2, out[1] = ||y||^2 (n entries each)
gbqr_status norms2(const Exec &ex, int64_t n, const double *x, const double *y, double *out);
// y = op(T) w for k x k upper triangular T (k <= 256)
gbqr_status trmv_upper(const Exec &ex, int k, const double *T, int64_t ldt, bool trans, const double *w, double *y);
// out[0] = ||A||_F^2 (m x n); colsq: n doubles of scratch.  Fixed order.
gbqr_status frob2(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, double *colsq, double *out);
// y = a x + b y
gbqr_status axpby(const Exec &ex, int64_t n, double a, const double *x, double b, double *y);
// R x = c (trans: R^T x = c) for one vector with the inverses of R's 64 x 64
// diagonal blocks in Dinv (trsv_block_inverses): one persistent launch, the
// blocks solved in order and published through counters (4, zero on entry,
// left zero); timeout: the context's device flag for a bounded wait.
gbqr_status trsv_chain(const Exec &ex, bool trans, int64_t n, const double *R, int64_t ldr, double *x,
                       const double *Dinv, unsigned *counters, size_t ncounters, int *timeout);
constexpr int kApplyVecMaxW = 256;   // widest panel apply_vec takes
// x <- Q^T x (trans) or Q x for one vector x (m), Q from the packed V of
// VR (lda) and the panel kernels of T (ldt; tfull: T is the full n x n
// kernel and its diagonal pb x pb blocks are used), panels of width pb: one
// persistent launch.  y2: 2 pb doubles; partial: >= ceil(m / rows per
// item) pb doubles; counters: 5, zero on entry, left zero; timeout: the
// context's device flag, raised if a bounded wait runs out.
gbqr_status apply_vec(const Exec &ex, bool trans, int64_t m, int64_t n, const double *VR, int64_t lda,
                      const double *T, int64_t ldt, bool tfull, int64_t pb, double *x, double *y2, size_t ny,
                      double *partial, size_t partial_elems, unsigned *counters, size_t ncounters, int *timeout);

// ------------------------------------------------------------ tuner cache
// Context accessors for the tuner (the context's layout lives in api.cu).
// Keys: kind (GBQR_TUNE_FACTOR / GBQR_TUNE_BATCHED), the power-of-two classes
// of m and n, the T layout and the update precision.
uint64_t tune_key(int kind, int64_t m, int64_t n, int t_layout, int update_prec);
cudaStream_t ctx_stream(const gbqr_ctx *cx);
int ctx_device(const gbqr_ctx *cx);
bool ctx_tracing(const gbqr_ctx *cx);
void ctx_store_tuned(gbqr_ctx *cx, uint64_t key, const gbqr_opts &o);
bool ctx_lookup_tuned(const gbqr_ctx *cx, uint64_t key, gbqr_opts *o);
void ctx_copy_tuned(const gbqr_ctx *from, gbqr_ctx *to);
// frees the page-locked tables recorded by a capture (after its graph is gone)
void ctx_free_capture_owned(gbqr_ctx *cx);
// gbqr_factor / gbqr_factor_batched without the tuner cache (the tuner's own
// measurements must see exactly the options it passes)
gbqr_status factor_untuned(gbqr_ctx *cx, int64_t m, int64_t n, double *A, int64_t lda, double *T, int64_t ldt,
                           int t_layout, const gbqr_opts *opts);
// prepare_only: validate, create the lane streams and size the workspace,
// enqueue nothing (what a graph capture of the same call needs beforehand).
template <class Real>
gbqr_status factor_batched_untuned(gbqr_ctx *cx, int count, const int64_t *m, const int64_t *n, Real *const *A,
                                   const int64_t *lda, Real *const *T, const int64_t *ldt, const gbqr_opts *opts,
                                   bool prepare_only = false);

}  // namespace gbqr
