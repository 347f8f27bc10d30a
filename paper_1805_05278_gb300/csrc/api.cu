// C ABI of the library (include/gbqr.h) and the host-side drivers:
//   - the QR-EG recursion of Algorithm 2 (GBQR_T_FULL),
//   - a right-looking top level over panels of width nb whose panels are
//     factored by QR-EG, never forming superdiagonal blocks of T
//     (Section 8.4; GBQR_T_PANEL),
//   - applying Q / Q^T and forming the thin Q (basis-kernel update,
//     Section 2.3), and the least-squares solve built on them.
// All device work is enqueued on the context's stream; nothing here computes
// on the host.
#include "common.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <type_traits>
#include <vector>

using namespace gbqr;

namespace {

constexpr int kDefaultCutoff = 16;   // measured best of 8, 16, 32 (FP64 and mixed)
constexpr int kDefaultFanout = 0;   // 0: the TSQR planner chooses
constexpr int64_t kDefaultPanel = 128;
constexpr int kBatchLanes = 128;      // streams a batched factorization spreads over (measured best of 16..128)
constexpr int kBatchCutoff = 16;      // batched default cutoff b (measured best of 16, 32)
constexpr int kKrylov = 100;          // GMRES refinement: Arnoldi steps per correction
constexpr int kInPanelTcMinCols = 32;  // mixed path: in-panel updates on the tensor cores from n1 >= 32 (16 measured slower) ...
constexpr int64_t kInPanelTcMinRows = 2048;   // ... and m >= 2048
constexpr int kMaxBatchLanes = 128;

struct DeviceInfo {
    unsigned long long nonfinite;
    long long rankdef;
    int timeout;       // a bounded device-side wait ran out
    int pad;
};

// ------------------------------------------------------------ event tracer
struct EventTracer final : Tracer {
    struct Rec { Family f; size_t e0, e1; double flops, bytes; };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    size_t used = 0, open = 0;
    bool failed = false;

    size_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { failed = true; return SIZE_MAX; }
            pool.push_back(e);
        }
        return used++;
    }
    void begin(cudaStream_t s, Family) override {
        open = next();
        if (open != SIZE_MAX) cudaEventRecord(pool[open], s);
    }
    void end(cudaStream_t s, Family f, double flops, double bytes) override {
        size_t e = next();
        if (e == SIZE_MAX || open == SIZE_MAX) return;
        cudaEventRecord(pool[e], s);
        recs.push_back({f, open, e, flops, bytes});
    }
    ~EventTracer() override {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

const char *kFamilyNames[FAM_COUNT] = {"gemm", "tc_gemm", "tsqr_up", "tsqr_down", "trsv", "gemv", "other", "batched"};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Params {
    int b = kDefaultCutoff;
    int64_t nb = kDefaultPanel;
    int leaf_rows = 0;
    int fanout = kDefaultFanout;
    bool lookahead = true;
    int nsplit = 0;        // 0: FP64 updates; 1..3: split-BF16 tensor-core updates
    bool dmma = false;     // FP64 GEMM engine of 64 x 64 tiles: DFMA (0.94 vs 0.83 TFLOP/s on 8192^2)
};

bool resolve(const gbqr_opts *o, int64_t m, int64_t n, Params *p) {
    Params r;
    r.nb = gbqr_default_panel_nb(m, n);
    if (o) {
        if (o->cutoff_b < 0 || o->cutoff_b > kMaxPanel) return false;
        if (o->panel_nb < 0 || o->leaf_rows < 0) return false;
        if (o->fanout != 0 && (o->fanout < 2 || o->fanout > 16)) return false;
        if (o->cutoff_b) r.b = o->cutoff_b;
        if (o->panel_nb) r.nb = o->panel_nb;
        if (o->leaf_rows) r.leaf_rows = o->leaf_rows;
        if (o->fanout) r.fanout = o->fanout;
        if (o->lookahead < -1 || o->lookahead > 1) return false;
        if (o->batch_streams < 0) return false;
        if (o->lookahead == -1) r.lookahead = false;
        if (o->update_prec == GBQR_MIXED_BF16) r.nsplit = 1;
        else if (o->update_prec == GBQR_MIXED_SPLITBF16) r.nsplit = 3;
        else if (o->update_prec != GBQR_FP64) return false;
        if (o->fp64_gemm == GBQR_GEMM_DMMA) r.dmma = true;
        else if (o->fp64_gemm != 0 && o->fp64_gemm != GBQR_GEMM_DFMA) return false;
    }
    r.nb = std::max<int64_t>(1, r.nb);
    *p = r;
    return true;
}

// Workspace regions (bytes, 256-aligned) for an m x n problem.
struct Layout {
    size_t partial = 0, gcount = 0, tR = 0, tT = 0, tY = 0, tX = 0, tcount = 0;
    size_t M1 = 0, M2 = 0, bigA = 0, bigT = 0, vec = 0;
    size_t partial2 = 0, gcount2 = 0, M1b = 0, M2b = 0;   // second lane (look-ahead panel stream)
    size_t tc = 0, n_tc = 0;                              // tensor-core slices (mixed updates)
    size_t tc2 = 0, n_tc2 = 0;                            // ... of the look-ahead lane's in-panel updates
    size_t kry = 0, n_kry = 0;                            // least squares, mixed: Krylov basis of the refinement
    size_t dinv = 0, n_dinv = 0;                          // ... and inverses of R's diagonal blocks
    size_t total = 0;
    size_t n_partial = 0, n_gcount = 0, n_M = 0, n_Mb = 0, n_bigA = 0, n_bigT = 0, counter_bytes = 0;
    TsqrPlan tsqr;
};

Layout make_layout(int64_t m, int64_t n, int t_layout, const Params &pr, int num_sms, bool staging = true,
                   size_t min_M = 0) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 16), 256); return o; };
    // split-K scratch grows with the problem (a quarter of m n elements per
    // lane) between what 4 and 16 split CTAs per SM need: the planner splits
    // only as far as the buffer allows
    L.n_partial = std::min(gemm_partial_elems_max(num_sms),
                           std::max(gemm_partial_elems_min(num_sms),
                                    (size_t)std::max<int64_t>(m, 1) * (size_t)std::max<int64_t>(n, 1) / 4));
    L.n_gcount = gemm_counters_max(num_sms);
    const int w = (int)std::max<int64_t>(1, std::min<int64_t>(pr.b, n));
    L.tsqr = tsqr_plan_bound(std::max<int64_t>(m, 1), w, pr.leaf_rows, pr.fanout, num_sms);
    const int64_t nb = std::min<int64_t>(pr.nb, std::max<int64_t>(n, 1));
    // temporaries of the update / T-assembly products and of applying Q
    size_t nM = (size_t)((n + 1) / 2) * (size_t)(n / 2 + 1);
    nM = std::max(nM, (size_t)nb * (size_t)std::max<int64_t>(n, 1));
    if (t_layout == GBQR_T_FULL) nM = std::max(nM, (size_t)std::max<int64_t>(n, 1) * (size_t)std::max<int64_t>(n, 1));
    nM = std::max(nM, min_M);   // e.g. Q^T A2 of a wide matrix
    L.n_M = nM;
    L.n_bigA = staging ? (size_t)std::max<int64_t>(m, 1) * (size_t)std::max<int64_t>(n, 1) : 1;
    L.n_bigT = staging ? (size_t)std::max<int64_t>(n, 1) * (size_t)std::max<int64_t>(n, 1) : 1;
    L.partial = take(L.n_partial * 8);
    L.counter_bytes = align_up(L.n_gcount * 4, 16) + L.tsqr.ncount * 4;
    L.gcount = take(L.counter_bytes);
    L.tcount = L.gcount + align_up(L.n_gcount * 4, 16);
    L.tR = take(L.tsqr.nR * 8);
    L.tT = take(L.tsqr.nT * 8);
    L.tY = take(L.tsqr.nY * 8);
    L.tX = take(L.tsqr.nX * 8);
    L.M1 = take(nM * 8);
    L.M2 = take(nM * 8);
    // second lane: panel factorizations of width <= nb run there
    L.n_Mb = std::max<size_t>((size_t)nb * (size_t)nb, 16);
    L.partial2 = take(pr.lookahead ? L.n_partial * 8 : 16);
    L.gcount2 = take(align_up(L.n_gcount * 4, 16));
    L.M1b = take(L.n_Mb * 8);
    L.M2b = take(L.n_Mb * 8);
    if (pr.nsplit > 0) {
        // W1 = V^T C (M = nb, N <= n, K <= m) and C -= V W2 (M <= m, N <= n, K = nb)
        L.n_tc = std::max(tc_gemm_scratch_bytes(nb, std::max<int64_t>(n, 1), std::max<int64_t>(m, 1), num_sms),
                          tc_gemm_scratch_bytes(std::max<int64_t>(m, 1), std::max<int64_t>(n, 1), nb, num_sms));
        L.tc = take(L.n_tc);
        // in-panel updates (M, N <= nb/2, K <= m) on the look-ahead lane
        const int64_t h = std::max<int64_t>(nb / 2, 1);
        L.n_tc2 = pr.lookahead ? tc_gemm_scratch_bytes(h, h, std::max<int64_t>(m, 1), num_sms) : 0;
        if (L.n_tc2) L.tc2 = take(L.n_tc2);
    }
    L.bigA = take(L.n_bigA * 8);
    L.bigT = take(L.n_bigT * 8);
    // least squares: vectors f, r (m) and x, dx, g (n) of the refinement
    L.vec = take(staging ? ((size_t)3 * std::max<int64_t>(m, 1) + 4 * (size_t)std::max<int64_t>(n, 1) + 16) * 8 : 16);
    // GMRES refinement (mixed least squares): kKrylov + 2 vectors of m + n,
    // and the projections and norms read back each Arnoldi step
    if (staging && pr.nsplit > 0) {
        L.n_kry = (size_t)(kKrylov + 2) * (size_t)(std::max<int64_t>(m, 1) + std::max<int64_t>(n, 1)) + 4 * (kKrylov + 2) + 16;
        L.kry = take(L.n_kry * 8);
        L.n_dinv = (size_t)((std::max<int64_t>(n, 1) + kTrsvBlockSize - 1) / kTrsvBlockSize) * kTrsvBlockSize * kTrsvBlockSize;
        L.dinv = take(L.n_dinv * 8);
    }
    L.total = off;
    return L;
}

}  // namespace

struct gbqr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 152;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = true;
    DeviceInfo *dinfo = nullptr;
    int64_t launches = 0;
    EventTracer *tracer = nullptr;
    bool tracing = false;
    cudaStream_t side = nullptr;          // high-priority stream for look-ahead panels
    cudaEvent_t ev_panel = nullptr, ev_ready = nullptr, ev_fork = nullptr;
    cudaStream_t copy = nullptr;          // host <-> device copies of the staged path
    cudaEvent_t ev_in0 = nullptr, ev_in1 = nullptr, ev_in = nullptr;   // staged input: panel 0, panel 1, the rest
    std::vector<cudaStream_t> lanes;      // batched factorization: one stream per lane
    std::vector<cudaEvent_t> lane_done;
    mutable std::mutex tuned_mu;           // autotuner results (gbqr_autotune*)
    std::unordered_map<uint64_t, gbqr_opts> tuned;
    gbqr::BatchPlan *bplan[2] = {nullptr, nullptr};   // persistent batched engine: FP64, FP32 plans
    std::vector<void *> capture_owned;    // page-locked tables a capture in progress refers to

    Exec exec() {
        Exec e;
        e.stream = stream;
        e.tracer = tracing ? tracer : nullptr;
        e.launches = &launches;
        e.num_sms = num_sms;
        e.device = device;
        return e;
    }
};

namespace gbqr {

static int ilog2_ceil(int64_t v) {
    int r = 0;
    while (((int64_t)1 << r) < v && r < 62) ++r;
    return r;
}

uint64_t tune_key(int kind, int64_t m, int64_t n, int t_layout, int update_prec) {
    return ((uint64_t)(kind & 0xff) << 40) | ((uint64_t)ilog2_ceil(std::max<int64_t>(m, 1)) << 32) |
           ((uint64_t)ilog2_ceil(std::max<int64_t>(n, 1)) << 24) | ((uint64_t)(t_layout & 0xff) << 8) |
           (uint64_t)(update_prec & 0xff);
}
cudaStream_t ctx_stream(const gbqr_ctx *cx) { return cx->stream; }
int ctx_device(const gbqr_ctx *cx) { return cx->device; }
bool ctx_tracing(const gbqr_ctx *cx) { return cx->tracing; }
void ctx_store_tuned(gbqr_ctx *cx, uint64_t key, const gbqr_opts &o) {
    std::lock_guard<std::mutex> lk(cx->tuned_mu);
    cx->tuned[key] = o;
}
bool ctx_lookup_tuned(const gbqr_ctx *cx, uint64_t key, gbqr_opts *o) {
    std::lock_guard<std::mutex> lk(cx->tuned_mu);
    auto it = cx->tuned.find(key);
    if (it == cx->tuned.end()) return false;
    *o = it->second;
    return true;
}
void ctx_free_capture_owned(gbqr_ctx *cx) {
    for (void *h : cx->capture_owned) cudaFreeHost(h);
    cx->capture_owned.clear();
}
void ctx_copy_tuned(const gbqr_ctx *from, gbqr_ctx *to) {
    std::unordered_map<uint64_t, gbqr_opts> copy;
    {
        std::lock_guard<std::mutex> lk(from->tuned_mu);
        copy = from->tuned;
    }
    std::lock_guard<std::mutex> lk(to->tuned_mu);
    to->tuned = std::move(copy);
}

}  // namespace gbqr

namespace {

// Tuned parameters for a call: the cached autotuner result for this shape
// class, with every non-zero field of the caller's options taking precedence.
// The panel width changes the PANEL T layout the caller allocated and later
// passes to apply_q, so it is only taken where the call owns T (allow_nb).
const gbqr_opts *with_tuned(const gbqr_ctx *cx, int kind, int64_t m, int64_t n, int t_layout,
                            const gbqr_opts *o, gbqr_opts *eff, bool allow_nb) {
    const int prec = o ? o->update_prec : GBQR_FP64;
    gbqr_opts t;
    if (!ctx_lookup_tuned(cx, tune_key(kind, m, n, t_layout, prec), &t)) return o;
    if (o) {
        if (o->cutoff_b) t.cutoff_b = o->cutoff_b;
        if (o->panel_nb) t.panel_nb = o->panel_nb;
        if (o->leaf_rows) t.leaf_rows = o->leaf_rows;
        if (o->fanout) t.fanout = o->fanout;
        if (o->lookahead) t.lookahead = o->lookahead;
        if (o->batch_streams) t.batch_streams = o->batch_streams;
        if (o->fp64_gemm) t.fp64_gemm = o->fp64_gemm;
    }
    if (!allow_nb) t.panel_nb = o ? o->panel_nb : 0;
    t.update_prec = prec;
    *eff = t;
    return eff;
}

// Per-call view of the carved workspace.
struct Work {
    gbqr_ctx *cx;
    Exec ex;
    Layout L;
    Params pr;
    GemmScratch gs;
    TsqrWork tw;
    double *M1, *M2, *bigA, *bigT, *vec, *kry, *dinv;
    size_t n_M;                      // capacity of M1 / M2 of this lane
    TcScratch tcs;                   // tensor-core scratch (main lane, mixed updates)
    TcScratch tcs2;                  // ... of the look-ahead lane
    GemmScratch gs2;
    double *M1b, *M2b;

    // Typed views of the workspace (regions are sized for FP64; an FP32 call
    // uses the same bytes).
    template <class Real> Real *m1() const { return reinterpret_cast<Real *>(M1); }
    template <class Real> Real *m2() const { return reinterpret_cast<Real *>(M2); }
    template <class Real> GemmScratchT<Real> gsr() const {
        GemmScratchT<Real> g;
        g.partial = reinterpret_cast<Real *>(gs.partial);
        g.partial_elems = gs.partial_elems * (sizeof(double) / sizeof(Real));
        g.counters = gs.counters;
        g.ncounters = gs.ncounters;
        return g;
    }
    template <class Real> TsqrWorkT<Real> twr() const {
        TsqrWorkT<Real> t;
        t.R = reinterpret_cast<Real *>(tw.R);
        t.T = reinterpret_cast<Real *>(tw.T);
        t.Y = reinterpret_cast<Real *>(tw.Y);
        t.X = reinterpret_cast<Real *>(tw.X);
        t.counters = tw.counters;
        return t;
    }

    // The second lane: same TSQR workspace, its own GEMM scratch and
    // temporaries, enqueued on the context's side stream.
    Work lane2() const {
        Work o = *this;
        o.ex.stream = cx->side;
        o.gs = gs2;
        o.M1 = M1b;
        o.M2 = M2b;
        o.n_M = L.n_Mb;
        o.tcs = tcs2;
        return o;
    }
};

gbqr_status ensure_workspace(gbqr_ctx *cx, size_t bytes) {
    if (bytes <= cx->ws_bytes) return GBQR_OK;
    if (!cx->ws_owned) return GBQR_ENOMEM;
    if (cx->ws) {
        cudaStreamSynchronize(cx->stream);
        if (cx->side) cudaStreamSynchronize(cx->side);
        if (cx->copy) cudaStreamSynchronize(cx->copy);
        for (auto st : cx->lanes) cudaStreamSynchronize(st);
        cudaFree(cx->ws);
        cx->ws = nullptr;
        cx->ws_bytes = 0;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
    cx->ws = (char *)p;
    cx->ws_bytes = bytes;
    return GBQR_OK;
}

// Point w's buffers into the workspace region at `base` laid out as L.
void carve_work(gbqr_ctx *cx, char *base, const Layout &L, const Params &pr, const Exec &ex, Work *w) {
    w->cx = cx;
    w->pr = pr;
    w->L = L;
    w->ex = ex;
    w->ex.dmma = pr.dmma;
    w->gs.partial = (double *)(base + w->L.partial);
    w->gs.partial_elems = w->L.n_partial;
    w->gs.counters = (unsigned *)(base + w->L.gcount);
    w->gs.ncounters = w->L.n_gcount;
    w->tw.R = (double *)(base + w->L.tR);
    w->tw.T = (double *)(base + w->L.tT);
    w->tw.Y = (double *)(base + w->L.tY);
    w->tw.X = (double *)(base + w->L.tX);
    w->tw.counters = (unsigned *)(base + w->L.tcount);
    w->M1 = (double *)(base + w->L.M1);
    w->M2 = (double *)(base + w->L.M2);
    w->bigA = (double *)(base + w->L.bigA);
    w->bigT = (double *)(base + w->L.bigT);
    w->vec = (double *)(base + w->L.vec);
    w->kry = w->L.n_kry ? (double *)(base + w->L.kry) : nullptr;
    w->dinv = w->L.n_dinv ? (double *)(base + w->L.dinv) : nullptr;
    w->n_M = w->L.n_M;
    w->gs2.partial = (double *)(base + w->L.partial2);
    w->gs2.partial_elems = pr.lookahead ? w->L.n_partial : 0;
    w->gs2.counters = (unsigned *)(base + w->L.gcount2);
    w->gs2.ncounters = w->L.n_gcount;
    w->M1b = (double *)(base + w->L.M1b);
    w->M2b = (double *)(base + w->L.M2b);
    w->tcs.base = w->L.n_tc ? (void *)(base + w->L.tc) : nullptr;
    w->tcs.bytes = w->L.n_tc;
    w->tcs.err = &cx->dinfo->timeout;
    w->tcs2.base = w->L.n_tc2 ? (void *)(base + w->L.tc2) : nullptr;
    w->tcs2.bytes = w->L.n_tc2;
    w->tcs2.err = &cx->dinfo->timeout;
}

// Arrival counters start at zero (every kernel leaves them zero again).
gbqr_status zero_counters(const Work &w, cudaStream_t s) {
    char *base = (char *)w.gs.partial - w.L.partial;
    if (cudaMemsetAsync(base + w.L.gcount, 0, w.L.counter_bytes, s) != cudaSuccess) return GBQR_ECUDA;
    if (cudaMemsetAsync(base + w.L.gcount2, 0, align_up(w.L.n_gcount * 4, 16), s) != cudaSuccess) return GBQR_ECUDA;
    return GBQR_OK;
}

gbqr_status begin_work(gbqr_ctx *cx, int64_t m, int64_t n, int t_layout, const Params &pr, Work *w,
                       size_t min_M = 0) {
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    const Layout L = make_layout(m, n, t_layout, pr, cx->num_sms, true, min_M);
    gbqr_status st = ensure_workspace(cx, L.total);
    if (st != GBQR_OK) return st;
    carve_work(cx, cx->ws, L, pr, cx->exec(), w);
    return zero_counters(*w, cx->stream);
}

#define TRY(x) do { gbqr_status _s = (x); if (_s != GBQR_OK) return _s; } while (0)

// C (mr x nc) <- (I - V op(T) V^T) C; op(T) = T^T when trans.  V is the unit
// lower trapezoidal mr x kv basis, T the kv x kv upper triangular kernel.
template <class Real>
gbqr_status apply_block(Work &w, bool trans, int64_t mr, int64_t nc, int64_t kv,
                        const Real *V, int64_t ldv, const Real *T, int64_t ldt, Real *C, int64_t ldc,
                        int nsplit = 0) {
    if (mr <= 0 || nc <= 0 || kv <= 0) return GBQR_OK;
    if ((size_t)kv * (size_t)nc > w.n_M) return GBQR_ENOMEM;
    constexpr bool fp64 = std::is_same<Real, double>::value;
    if constexpr (fp64) {
    if (nc == 1) {
        // one vector: matrix-vector products instead of 1-column GEMM tiles
        TRY(gemv_t(w.ex, mr, kv, V, ldv, C, 1.0, 0.0, w.M1, MASK_UNIT_LOWER));
        if (kv > 0x7fffffff) return GBQR_EUNSUPPORTED;
        TRY(trmv_upper(w.ex, (int)kv, T, ldt, trans, w.M1, w.M2));
        return gemv_n(w.ex, mr, kv, V, ldv, w.M2, -1.0, 1.0, C, w.gs.partial, w.gs.partial_elems, MASK_UNIT_LOWER);
    }
    if (nsplit > 0 && w.tcs.base) {
        // mixed precision: the two large products on the tensor cores
        // (split-BF16, FP32 accumulation), the small T product in FP64
        TcGemmOp g;
        g.M = kv; g.N = nc; g.K = mr;
        g.A = V; g.lda = ldv; g.ta = true; g.maskA = MASK_UNIT_LOWER;
        g.B = C; g.ldb = ldc; g.C = w.M1; g.ldc = kv; g.nsplit = nsplit;
        TRY(tc_gemm(w.ex, g, w.tcs));
        GemmOp h;
        h.M = kv; h.N = nc; h.K = kv;
        h.A = T; h.lda = ldt; h.ta = trans; h.maskA = MASK_UPPER;
        h.B = w.M1; h.ldb = kv; h.C = w.M2; h.ldc = kv;
        TRY(gemm(w.ex, h, w.gs));
        TcGemmOp u;
        u.M = mr; u.N = nc; u.K = kv;
        u.A = V; u.lda = ldv; u.ta = false; u.maskA = MASK_UNIT_LOWER;
        u.B = w.M2; u.ldb = kv; u.C = C; u.ldc = ldc; u.alpha = -1.0; u.beta = 1.0; u.nsplit = nsplit;
        return tc_gemm(w.ex, u, w.tcs);
    }
    }
    Real *M1 = w.m1<Real>(), *M2 = w.m2<Real>();
    const GemmScratchT<Real> gsr = w.gsr<Real>();
    GemmOpT<Real> g;
    g.M = kv; g.N = nc; g.K = mr;
    g.A = V; g.lda = ldv; g.ta = true; g.maskA = MASK_UNIT_LOWER;
    g.B = C; g.ldb = ldc; g.C = M1; g.ldc = kv;
    TRY(gemm(w.ex, g, gsr));
    GemmOpT<Real> h;
    h.M = kv; h.N = nc; h.K = kv;
    h.A = T; h.lda = ldt; h.ta = trans; h.maskA = MASK_UPPER;
    h.B = M1; h.ldb = kv; h.C = M2; h.ldc = kv;
    TRY(gemm(w.ex, h, gsr));
    GemmOpT<Real> u;
    u.M = mr; u.N = nc; u.K = kv;
    u.A = V; u.lda = ldv; u.ta = false; u.maskA = MASK_UNIT_LOWER;
    u.B = M2; u.ldb = kv; u.C = C; u.ldc = ldc; u.alpha = Real(-1); u.beta = Real(1);
    return gemm(w.ex, u, gsr);
}

// Base case: TSQR of the m x n panel (n <= b).
template <class Real>
gbqr_status base_qr(Work &w, int64_t m, int64_t n, Real *A, int64_t lda, Real *T, int64_t ldt) {
    TsqrPlan pl;
    if (!tsqr_plan(m, (int)n, w.pr.leaf_rows, w.pr.fanout, w.ex.num_sms, &pl)) return GBQR_EINVAL;
    if (pl.nR > w.L.tsqr.nR || pl.nT > w.L.tsqr.nT || pl.nY > w.L.tsqr.nY || pl.ncount > w.L.tsqr.ncount)
        return GBQR_ENOMEM;
    return tsqr_run(w.ex, pl, A, lda, T, ldt, w.twr<Real>());
}

// Algorithm 2: (V, T, R) = QR-EG(A, b), V\R in place over A, T (n x n) at T.
template <class Real>
gbqr_status qr_eg(Work &w, int64_t m, int64_t n, Real *A, int64_t lda, Real *T, int64_t ldt) {
    if (n <= 0) return GBQR_OK;
    if (n <= w.pr.b) return base_qr(w, m, n, A, lda, T, ldt);
    const int64_t n1 = n / 2, n2 = n - n1;
    Real *AR = A + n1 * lda;
    Real *M1 = w.m1<Real>(), *M2 = w.m2<Real>();
    const GemmScratchT<Real> gsr = w.gsr<Real>();
    TRY(qr_eg(w, m, n1, A, lda, T, ldt));                  // left recursion
    // M1 = V_L^T A_R ; M2 = T_L^T M1 ; A_R -= V_L M2.  On the mixed path the
    // two tall products go to the tensor cores once they are large enough to
    // beat the FP64 kernel's latency (the T-assembly below stays FP64, so T
    // stays consistent with V and Q = I - V T V^T orthogonal to FP64 accuracy).
    const int nsplit_in = (w.pr.nsplit > 0 && n1 >= kInPanelTcMinCols && m >= kInPanelTcMinRows) ? w.pr.nsplit : 0;
    TRY(apply_block(w, true, m, n2, n1, A, lda, T, ldt, AR, lda, nsplit_in));
    // right recursion on B22
    Real *TR = T + n1 + n1 * ldt;
    TRY(qr_eg(w, m - n1, n2, A + n1 + n1 * lda, lda, TR, ldt));
    // M3 = V_L(n1:m, :)^T V_R ; M4 = M3 T_R ; T12 = -T_L M4
    if ((size_t)n1 * (size_t)n2 > w.n_M) return GBQR_ENOMEM;
    GemmOpT<Real> g3;
    g3.M = n1; g3.N = n2; g3.K = m - n1;
    g3.A = A + n1; g3.lda = lda; g3.ta = true; g3.maskA = MASK_NONE;
    g3.B = A + n1 + n1 * lda; g3.ldb = lda; g3.maskB = MASK_UNIT_LOWER;
    g3.C = M1; g3.ldc = n1;
    TRY(gemm(w.ex, g3, gsr));
    GemmOpT<Real> g4;
    g4.M = n1; g4.N = n2; g4.K = n2;
    g4.A = M1; g4.lda = n1; g4.ta = false;
    g4.B = TR; g4.ldb = ldt; g4.maskB = MASK_UPPER;
    g4.C = M2; g4.ldc = n1;
    TRY(gemm(w.ex, g4, gsr));
    GemmOpT<Real> g5;
    g5.M = n1; g5.N = n2; g5.K = n1;
    g5.A = T; g5.lda = ldt; g5.ta = false; g5.maskA = MASK_UPPER;
    g5.B = M2; g5.ldb = n1;
    g5.C = T + n1 * ldt; g5.ldc = ldt; g5.alpha = Real(-1); g5.beta = Real(0);
    return gemm(w.ex, g5, gsr);
}

// Zero T(i, j) for i > (j mod nb) (the strict lower part of every block).
template <class Real>
__global__ void zero_below_blocks_kernel(int64_t rows, int64_t n, int64_t nb, Real *T, int64_t ldt) {
    const int64_t total = rows * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows, j = e / rows;
        if (i > j % nb) T[i + j * ldt] = Real(0);
    }
}

template <class Real>
gbqr_status zero_below_blocks(Work &w, int64_t rows, int64_t n, int64_t nb, Real *T, int64_t ldt) {
    if (rows <= 1 || n <= 0) return GBQR_OK;
    trace_begin(w.ex, FAM_OTHER);
    const int64_t total = rows * n;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)w.ex.num_sms * 8));
    zero_below_blocks_kernel<Real><<<grid, 256, 0, w.ex.stream>>>(rows, n, nb, T, ldt);
    return trace_end(w.ex, FAM_OTHER, 0.0, (double)sizeof(Real) / 2.0 * (double)total);
}

// Host buffers of a staged factorization (PANEL layout with look-ahead):
// their panels travel on the context's copy stream, overlapped with the
// factorization of the others.
struct HostIO {
    double *A; int64_t lda;   // m x n
    double *T; int64_t ldt;   // trows x n
};

// Column blocks [c0, c0 + nc) of the m-row host matrix to the device, each
// scanned for non-finite entries on arrival; `done` marks the last one.
gbqr_status stage_in(Work &w, const HostIO &io, double *A, int64_t lda, int64_t m, int64_t c0, int64_t nc,
                     cudaEvent_t done) {
    gbqr_ctx *cx = w.cx;
    if (nc > 0) {
        if (cudaMemcpy2DAsync(A + c0 * lda, lda * 8, io.A + c0 * io.lda, io.lda * 8, m * 8, nc,
                              cudaMemcpyHostToDevice, cx->copy) != cudaSuccess)
            return GBQR_ECUDA;
        Exec ce = w.ex;
        ce.stream = cx->copy;
        TRY(scan_nonfinite(ce, m, nc, A + c0 * lda, lda, &cx->dinfo->nonfinite));
    }
    return cudaEventRecord(done, cx->copy) == cudaSuccess ? GBQR_OK : GBQR_ECUDA;
}

// Panel [j0, j0 + wd) is final once its factorization (ev_panel, just
// recorded) is done: its columns and T block go back while later panels run.
gbqr_status stage_out(Work &w, const HostIO &io, const double *A, int64_t lda, const double *T, int64_t ldt,
                      int64_t m, int64_t trows, int64_t j0, int64_t wd) {
    gbqr_ctx *cx = w.cx;
    if (cudaStreamWaitEvent(cx->copy, cx->ev_panel, 0) != cudaSuccess ||
        cudaMemcpy2DAsync(io.A + j0 * io.lda, io.lda * 8, A + j0 * lda, lda * 8, m * 8, wd, cudaMemcpyDeviceToHost,
                          cx->copy) != cudaSuccess ||
        cudaMemcpy2DAsync(io.T + j0 * io.ldt, io.ldt * 8, T + j0 * ldt, ldt * 8, trows * 8, wd,
                          cudaMemcpyDeviceToHost, cx->copy) != cudaSuccess)
        return GBQR_ECUDA;
    return GBQR_OK;
}

template <class Real>
gbqr_status factor_device(Work &w, int64_t m, int64_t n, Real *A, int64_t lda, Real *T, int64_t ldt, int layout,
                          const HostIO *io = nullptr) {
    DeviceInfo *di = w.cx->dinfo;
    if (!io) TRY(scan_nonfinite(w.ex, m, n, A, lda, &di->nonfinite));
    if (layout == GBQR_T_FULL) {
        TRY(zero_below_blocks(w, n, n, std::max<int64_t>(n, 1), T, ldt));
        return qr_eg(w, m, n, A, lda, T, ldt);
    }
    const int64_t nb = std::min<int64_t>(w.pr.nb, n);
    TRY(zero_below_blocks(w, nb, n, nb, T, ldt));
    const int64_t npan = (n + nb - 1) / nb;
    gbqr_ctx *cx = w.cx;
    if (!w.pr.lookahead || npan == 1 || !cx->side) {
        for (int64_t j0 = 0; j0 < n; j0 += nb) {
            const int64_t wd = std::min<int64_t>(nb, n - j0);
            Real *Ap = A + j0 + j0 * lda;
            Real *Tk = T + j0 * ldt;
            TRY(qr_eg(w, m - j0, wd, Ap, lda, Tk, ldt));
            if (j0 + wd < n)
                TRY(apply_block(w, true, m - j0, n - j0 - wd, wd, Ap, lda, Tk, ldt, A + j0 + (j0 + wd) * lda, lda,
                                w.pr.nsplit));
        }
        return GBQR_OK;
    }
    // Look-ahead (depth 1): panel k+1 is factored on the high-priority side
    // stream while the rest of panel k's trailing update runs on the main
    // stream.  Event fork/join only, so the sequence is graph-capturable.
    Work wp = w.lane2();
    const cudaStream_t ms = w.ex.stream, ss = cx->side;
    if (io) {
        // staged: the copy stream starts after the work already on the main
        // stream (the staging buffer may still be in use), then brings in
        // panel 0, panel 1 and the rest, in that order
        if constexpr (!std::is_same<Real, double>::value) return GBQR_EINVAL;
        else {
            const int64_t b0 = nb, b1 = std::min<int64_t>(nb, n - b0);
            if (cudaEventRecord(cx->ev_in0, ms) != cudaSuccess || cudaStreamWaitEvent(cx->copy, cx->ev_in0, 0) != cudaSuccess)
                return GBQR_ECUDA;
            TRY(stage_in(w, *io, A, lda, m, 0, b0, cx->ev_in0));
            TRY(stage_in(w, *io, A, lda, m, b0, b1, cx->ev_in1));
            TRY(stage_in(w, *io, A, lda, m, b0 + b1, n - b0 - b1, cx->ev_in));
            if (cudaStreamWaitEvent(ms, cx->ev_in0, 0) != cudaSuccess) return GBQR_ECUDA;
        }
    }
    auto panel_out = [&](int64_t j0, int64_t wd) -> gbqr_status {
        if constexpr (std::is_same<Real, double>::value)
            if (io) return stage_out(w, *io, A, lda, T, ldt, m, ldt, j0, wd);
        return GBQR_OK;
    };
    if (cudaEventRecord(cx->ev_fork, ms) != cudaSuccess || cudaStreamWaitEvent(ss, cx->ev_fork, 0) != cudaSuccess)
        return GBQR_ECUDA;
    TRY(qr_eg(wp, m, std::min<int64_t>(nb, n), A, lda, T, ldt));
    if (cudaEventRecord(cx->ev_panel, ss) != cudaSuccess) return GBQR_ECUDA;
    TRY(panel_out(0, std::min<int64_t>(nb, n)));
    for (int64_t k = 0; k < npan; ++k) {
        const int64_t j0 = k * nb, wd = std::min<int64_t>(nb, n - j0);
        if (cudaStreamWaitEvent(ms, cx->ev_panel, 0) != cudaSuccess) return GBQR_ECUDA;   // panel k done
        if (k + 1 == npan) break;
        const int64_t j1 = j0 + wd, w1 = std::min<int64_t>(nb, n - j1);
        const Real *Vk = A + j0 + j0 * lda;
        const Real *Tk = T + j0 * ldt;
        if (io && k == 0 && cudaStreamWaitEvent(ms, cx->ev_in1, 0) != cudaSuccess) return GBQR_ECUDA;
        // panel k+1's columns first ...
        TRY(apply_block(w, true, m - j0, w1, wd, Vk, lda, Tk, ldt, A + j0 + j1 * lda, lda, w.pr.nsplit));
        if (cudaEventRecord(cx->ev_ready, ms) != cudaSuccess || cudaStreamWaitEvent(ss, cx->ev_ready, 0) != cudaSuccess)
            return GBQR_ECUDA;
        // ... then panel k+1 on the side stream, concurrently with the rest of the update
        TRY(qr_eg(wp, m - j1, w1, A + j1 + j1 * lda, lda, T + j1 * ldt, ldt));
        if (cudaEventRecord(cx->ev_panel, ss) != cudaSuccess) return GBQR_ECUDA;
        TRY(panel_out(j1, w1));
        if (io && k == 0 && cudaStreamWaitEvent(ms, cx->ev_in, 0) != cudaSuccess) return GBQR_ECUDA;
        if (j1 + w1 < n)
            TRY(apply_block(w, true, m - j0, n - j1 - w1, wd, Vk, lda, Tk, ldt, A + j0 + (j1 + w1) * lda, lda,
                            w.pr.nsplit));
    }
    return GBQR_OK;
}

// B <- Q^T B (trans) or Q B, for either T layout.  col0 > 0 restricts the
// update of panel k to columns >= its first column (used by form_q, where
// the columns to the left are still unit vectors that Q_k leaves alone).
gbqr_status apply_q_any(Work &w, bool trans, int64_t m, int64_t n, const double *VR, int64_t lda,
                        const double *T, int64_t ldt, int layout, int64_t nb, int64_t nrhs,
                        double *B, int64_t ldb, bool form_q_structure) {
    if (n <= 0 || nrhs <= 0) return GBQR_OK;
    if (layout == GBQR_T_FULL && !form_q_structure)
        return apply_block(w, trans, m, nrhs, n, VR, lda, T, ldt, B, ldb);
    // blocked over panels of width nb; for GBQR_T_FULL the panel kernels are
    // the diagonal blocks of T (those of consecutive reflectors).
    const int64_t pb = (layout == GBQR_T_FULL) ? std::min<int64_t>(kDefaultPanel, n) : nb;
    const int64_t npan = (n + pb - 1) / pb;
    if (nrhs == 1 && !form_q_structure && pb <= kApplyVecMaxW && (size_t)(2 * pb) <= w.n_M && w.tcs.err)
        // one vector: every panel in one persistent launch
        return apply_vec(w.ex, trans, m, n, VR, lda, T, ldt, layout == GBQR_T_FULL, pb, B, w.M1, w.n_M,
                         w.gs.partial, w.gs.partial_elems, w.gs.counters, w.gs.ncounters, w.tcs.err);
    for (int64_t q = 0; q < npan; ++q) {
        const int64_t k = trans ? q : npan - 1 - q;
        const int64_t j0 = k * pb, wd = std::min<int64_t>(pb, n - j0);
        const double *Tk = (layout == GBQR_T_FULL) ? T + j0 + j0 * ldt : T + j0 * ldt;
        const int64_t c0 = form_q_structure ? j0 : 0;
        TRY(apply_block(w, trans, m - j0, nrhs - c0, wd, VR + j0 + j0 * lda, lda, Tk, ldt, B + j0 + c0 * ldb, ldb));
    }
    return GBQR_OK;
}

// gbqr_factor_batched runs as one persistent kernel unless the caller asks
// for panels wider than the cutoff, a cutoff above the persistent kernel's
// limit or tensor-core updates: then the per-matrix panel path, spread over
// internal streams.
bool persistent_batch(const gbqr_opts *o) {
    if (!o) return true;
    const int b = o->cutoff_b ? o->cutoff_b : kBatchCutoff;
    return b <= kMaxBatchB && (o->panel_nb == 0 || o->panel_nb == b) && o->update_prec == GBQR_FP64;
}

bool is_host_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return true; }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// Page-locked host memory: asynchronous copies from and to it do not block
// the calling thread.
bool is_pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeHost;
}

gbqr_status check_layout_args(int64_t m, int64_t n, int64_t lda, int64_t ldt, int layout, int64_t nb) {
    if (m < 0 || n < 0 || m < n) return GBQR_EINVAL;
    if (lda < std::max<int64_t>(1, m)) return GBQR_EINVAL;
    if (layout == GBQR_T_FULL) {
        if (ldt < std::max<int64_t>(1, n)) return GBQR_EINVAL;
    } else if (layout == GBQR_T_PANEL) {
        if (nb < 1 || ldt < std::max<int64_t>(1, std::min(nb, n))) return GBQR_EINVAL;
    } else {
        return GBQR_EINVAL;
    }
    return GBQR_OK;
}

}  // namespace

extern "C" {

int64_t gbqr_default_panel_nb(int64_t m, int64_t n) {
    (void)m;
    return std::max<int64_t>(1, std::min<int64_t>(kDefaultPanel, n));
}

const char *gbqr_strerror(gbqr_status s) {
    switch (s) {
        case GBQR_OK: return "ok";
        case GBQR_EINVAL: return "invalid argument";
        case GBQR_ENOMEM: return "out of workspace or device memory";
        case GBQR_ECUDA: return "CUDA error";
        case GBQR_ETIMEOUT: return "device-side wait timed out";
        case GBQR_ENONFINITE: return "non-finite input";
        case GBQR_ERANKDEF: return "rank deficient (zero diagonal in R)";
        case GBQR_EBUSY: return "context busy";
        case GBQR_EUNSUPPORTED: return "unsupported in this build";
        case GBQR_ENOCONV: return "iterative refinement did not converge";
    }
    return "unknown status";
}

gbqr_status gbqr_create(gbqr_ctx **out, int device, void *cuda_stream) {
    if (!out) return GBQR_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return GBQR_ECUDA; }
    if (device < 0 || device >= ndev) return GBQR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    gbqr_ctx *cx = new (std::nothrow) gbqr_ctx();
    if (!cx) return GBQR_ENOMEM;
    cx->device = device;
    cx->stream = (cudaStream_t)cuda_stream;
    if (cudaDeviceGetAttribute(&cx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete cx;
        return GBQR_ECUDA;
    }
    if (cudaMalloc((void **)&cx->dinfo, sizeof(DeviceInfo)) != cudaSuccess) { delete cx; return GBQR_ENOMEM; }
    DeviceInfo zero{0ull, LLONG_MAX, 0, 0};
    if (cudaMemcpy(cx->dinfo, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(cx->dinfo);
        delete cx;
        return GBQR_ECUDA;
    }
    cx->tracer = new (std::nothrow) EventTracer();
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&cx->side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&cx->ev_panel, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cx->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cx->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&cx->ev_in0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cx->ev_in1, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&cx->ev_in, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        gbqr_destroy(cx);
        return GBQR_ECUDA;
    }
    *out = cx;
    return GBQR_OK;
}

gbqr_status gbqr_destroy(gbqr_ctx *cx) {
    if (!cx) return GBQR_EINVAL;
    gbqr_server_stop(cx);   // a serving loop attached to this context, if any
    cudaSetDevice(cx->device);
    cudaStreamSynchronize(cx->stream);
    if (cx->side) cudaStreamSynchronize(cx->side);
    if (cx->copy) cudaStreamSynchronize(cx->copy);
    if (cx->ws_owned && cx->ws) cudaFree(cx->ws);
    cx->ws = nullptr;
    if (cx->dinfo) cudaFree(cx->dinfo);
    if (cx->ev_panel) cudaEventDestroy(cx->ev_panel);
    if (cx->ev_ready) cudaEventDestroy(cx->ev_ready);
    if (cx->ev_fork) cudaEventDestroy(cx->ev_fork);
    if (cx->side) cudaStreamDestroy(cx->side);
    if (cx->ev_in0) cudaEventDestroy(cx->ev_in0);
    if (cx->ev_in1) cudaEventDestroy(cx->ev_in1);
    if (cx->ev_in) cudaEventDestroy(cx->ev_in);
    if (cx->copy) cudaStreamDestroy(cx->copy);
    for (auto st : cx->lanes) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (auto ev : cx->lane_done) cudaEventDestroy(ev);
    for (auto pl : cx->bplan) gbqr::batch_plan_free(pl);
    gbqr::ctx_free_capture_owned(cx);
    delete cx->tracer;
    delete cx;
    return GBQR_OK;
}

gbqr_status gbqr_set_stream(gbqr_ctx *cx, void *cuda_stream) {
    if (!cx) return GBQR_EINVAL;
    cx->stream = (cudaStream_t)cuda_stream;
    return GBQR_OK;
}

gbqr_status gbqr_set_workspace(gbqr_ctx *cx, void *ptr, size_t bytes) {
    if (!cx) return GBQR_EINVAL;
    if (ptr && ((uintptr_t)ptr % 16) != 0) return GBQR_EINVAL;
    if (cx->ws_owned && cx->ws) {
        cudaStreamSynchronize(cx->stream);
        if (cx->side) cudaStreamSynchronize(cx->side);
        if (cx->copy) cudaStreamSynchronize(cx->copy);
        cudaFree(cx->ws);
    }
    cx->ws = (char *)ptr;
    cx->ws_bytes = ptr ? bytes : 0;
    cx->ws_owned = (ptr == nullptr);
    return GBQR_OK;
}

size_t gbqr_workspace_bytes(int64_t m, int64_t n, int t_layout, const gbqr_opts *opts) {
    if (m < 0 || n < 0) return 0;
    if (t_layout != GBQR_T_FULL && t_layout != GBQR_T_PANEL) return 0;
    Params pr;
    if (!resolve(opts, m, n, &pr)) return 0;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { cudaGetLastError(); sms = 152; }
    } else {
        cudaGetLastError();
    }
    if (n > m) {   // wide: the leading m x m block, then Q^T A2
        const int64_t nbp = std::min<int64_t>(pr.nb, std::max<int64_t>(m, 1));
        return make_layout(m, m, t_layout, pr, sms, true,
                           (size_t)(t_layout == GBQR_T_FULL ? m : nbp) * (size_t)(n - m)).total;
    }
    return make_layout(m, n, t_layout, pr, sms).total;
}

gbqr_status gbqr_sync(gbqr_ctx *cx, gbqr_info *info) {
    if (!cx) return GBQR_EINVAL;
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    if (cudaStreamSynchronize(cx->stream) != cudaSuccess) return GBQR_ECUDA;
    DeviceInfo h{0ull, LLONG_MAX, 0, 0};
    if (cudaMemcpy(&h, cx->dinfo, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return GBQR_ECUDA;
    DeviceInfo zero{0ull, LLONG_MAX, 0, 0};
    if (cudaMemcpy(cx->dinfo, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) return GBQR_ECUDA;
    if (info) {
        memset(info, 0, sizeof *info);
        info->nonfinite = (int64_t)h.nonfinite;
        info->rankdef_col = h.rankdef == LLONG_MAX ? -1 : (int64_t)h.rankdef;
    }
    if (h.timeout) return GBQR_ETIMEOUT;
    return h.nonfinite ? GBQR_ENONFINITE : GBQR_OK;
}

gbqr_status gbqr_factor(gbqr_ctx *cx, int64_t m, int64_t n, double *A, int64_t lda,
                        double *T, int64_t ldt, int t_layout, const gbqr_opts *opts) {
    if (!cx) return GBQR_EINVAL;
    gbqr_opts eff;
    return gbqr::factor_untuned(cx, m, n, A, lda, T, ldt, t_layout,
                                with_tuned(cx, GBQR_TUNE_FACTOR, m, n, t_layout, opts, &eff, false));
}

}  // extern "C"

gbqr_status gbqr::factor_untuned(gbqr_ctx *cx, int64_t m, int64_t n, double *A, int64_t lda,
                                 double *T, int64_t ldt, int t_layout, const gbqr_opts *opts) {
    if (!cx) return GBQR_EINVAL;
    Params pr;
    if (!resolve(opts, m, n, &pr)) return GBQR_EINVAL;
    if (m >= 0 && n > m) {
        // Wide matrix (Section 2.1): A = [A1 A2] with square A1 = Q R1 by
        // QR-EG, then R = [R1, Q^T A2] by applying the m reflectors to A2.
        const int64_t k = m, nr = n - m;
        TRY(check_layout_args(m, k, lda, ldt, t_layout, pr.nb));
        if (k == 0) return GBQR_OK;
        if (!A || !T) return GBQR_EINVAL;
        if (is_host_pointer(A) || is_host_pointer(T)) return GBQR_EUNSUPPORTED;
        const int64_t nbp = std::min<int64_t>(pr.nb, k);
        Work w;
        TRY(begin_work(cx, m, k, t_layout, pr, &w, (size_t)(t_layout == GBQR_T_FULL ? k : nbp) * (size_t)nr));
        TRY(factor_device(w, m, k, A, lda, T, ldt, t_layout));
        return apply_q_any(w, true, m, k, A, lda, T, ldt, t_layout, nbp, nr, A + (size_t)k * lda, lda, false);
    }
    TRY(check_layout_args(m, n, lda, ldt, t_layout, pr.nb));
    if (n == 0) return GBQR_OK;
    if (!A || !T) return GBQR_EINVAL;
    Work w;
    TRY(begin_work(cx, m, n, t_layout, pr, &w));
    const bool hostA = is_host_pointer(A), hostT = is_host_pointer(T);
    if (hostA != hostT) return GBQR_EINVAL;
    if (!hostA) return factor_device(w, m, n, A, lda, T, ldt, t_layout);
    // host buffers: stage through the workspace, factor, copy back, synchronise
    const int64_t trows = (t_layout == GBQR_T_FULL) ? n : std::min<int64_t>(pr.nb, n);
    if ((size_t)trows * (size_t)n > w.L.n_bigT) return GBQR_ENOMEM;
    if (t_layout == GBQR_T_PANEL && pr.lookahead && cx->side && cx->copy && n > trows && is_pinned_host(A) &&
        is_pinned_host(T)) {
        // PANEL with look-ahead and page-locked buffers: panels in and out on
        // the copy stream, overlapped with the factorization (factor_device)
        const HostIO io{A, lda, T, ldt};
        const gbqr_status st = factor_device(w, m, n, w.bigA, m, w.bigT, trows, t_layout, &io);
        // drain all three streams even after an error: copies already queued
        // still write into the caller's buffers
        const cudaError_t e_copy = cudaStreamSynchronize(cx->copy);
        const cudaError_t e_side = cudaStreamSynchronize(cx->side);
        const cudaError_t e_main = cudaStreamSynchronize(cx->stream);
        const bool ok = e_copy == cudaSuccess && e_side == cudaSuccess && e_main == cudaSuccess;
        if (st != GBQR_OK) return st;
        return ok ? GBQR_OK : GBQR_ECUDA;
    }
    if (cudaMemcpy2DAsync(w.bigA, m * 8, A, lda * 8, m * 8, n, cudaMemcpyHostToDevice, cx->stream) != cudaSuccess)
        return GBQR_ECUDA;
    TRY(factor_device(w, m, n, w.bigA, m, w.bigT, trows, t_layout));
    if (cudaMemcpy2DAsync(A, lda * 8, w.bigA, m * 8, m * 8, n, cudaMemcpyDeviceToHost, cx->stream) != cudaSuccess)
        return GBQR_ECUDA;
    if (cudaMemcpy2DAsync(T, ldt * 8, w.bigT, trows * 8, trows * 8, n, cudaMemcpyDeviceToHost, cx->stream) != cudaSuccess)
        return GBQR_ECUDA;
    return cudaStreamSynchronize(cx->stream) == cudaSuccess ? GBQR_OK : GBQR_ECUDA;
}

extern "C" {

gbqr_status gbqr_factor_f32(gbqr_ctx *cx, int64_t m, int64_t n, float *A, int64_t lda, float *T, int64_t ldt,
                            int t_layout, const gbqr_opts *opts) {
    if (!cx) return GBQR_EINVAL;
    Params pr;
    if (!resolve(opts, m, n, &pr) || pr.nsplit != 0) return GBQR_EINVAL;
    TRY(check_layout_args(m, n, lda, ldt, t_layout, pr.nb));
    if (n == 0) return GBQR_OK;
    if (!A || !T) return GBQR_EINVAL;
    if (is_host_pointer(A) || is_host_pointer(T)) return GBQR_EUNSUPPORTED;
    Work w;
    TRY(begin_work(cx, m, n, t_layout, pr, &w));
    return factor_device(w, m, n, A, lda, T, ldt, t_layout);
}

static gbqr_status apply_entry(gbqr_ctx *cx, bool trans, int64_t m, int64_t n, const double *VR, int64_t lda,
                               const double *T, int64_t ldt, int layout, int64_t nb, int64_t nrhs,
                               double *B, int64_t ldb) {
    if (!cx) return GBQR_EINVAL;
    if (layout == GBQR_T_FULL) nb = std::max<int64_t>(n, 1);
    TRY(check_layout_args(m, n, lda, ldt, layout, nb));
    if (nrhs < 0 || ldb < std::max<int64_t>(1, m)) return GBQR_EINVAL;
    if (n == 0 || nrhs == 0) return GBQR_OK;
    if (!VR || !T || !B) return GBQR_EINVAL;
    Params pr;
    resolve(nullptr, m, n, &pr);
    if (layout == GBQR_T_PANEL) pr.nb = nb;
    Work w;
    TRY(begin_work(cx, m, std::max(n, nrhs), layout, pr, &w));
    if (layout == GBQR_T_FULL && (size_t)n * (size_t)nrhs > w.L.n_M) return GBQR_ENOMEM;
    return apply_q_any(w, trans, m, n, VR, lda, T, ldt, layout, nb, nrhs, B, ldb, false);
}

gbqr_status gbqr_apply_qt(gbqr_ctx *cx, int64_t m, int64_t n, const double *VR, int64_t lda,
                          const double *T, int64_t ldt, int t_layout, int64_t nb,
                          int64_t nrhs, double *B, int64_t ldb) {
    return apply_entry(cx, true, m, n, VR, lda, T, ldt, t_layout, nb, nrhs, B, ldb);
}

gbqr_status gbqr_apply_q(gbqr_ctx *cx, int64_t m, int64_t n, const double *VR, int64_t lda,
                         const double *T, int64_t ldt, int t_layout, int64_t nb,
                         int64_t nrhs, double *B, int64_t ldb) {
    return apply_entry(cx, false, m, n, VR, lda, T, ldt, t_layout, nb, nrhs, B, ldb);
}

gbqr_status gbqr_form_q(gbqr_ctx *cx, int64_t m, int64_t n, const double *VR, int64_t lda,
                        const double *T, int64_t ldt, int t_layout, int64_t nb,
                        double *Q, int64_t ldq) {
    if (!cx) return GBQR_EINVAL;
    if (t_layout == GBQR_T_FULL) nb = std::max<int64_t>(n, 1);
    TRY(check_layout_args(m, n, lda, ldt, t_layout, nb));
    if (ldq < std::max<int64_t>(1, m)) return GBQR_EINVAL;
    if (n == 0) return GBQR_OK;
    if (!VR || !T || !Q) return GBQR_EINVAL;
    Params pr;
    resolve(nullptr, m, n, &pr);
    if (t_layout == GBQR_T_PANEL) pr.nb = nb;
    Work w;
    TRY(begin_work(cx, m, n, t_layout, pr, &w));
    TRY(fill_identity(w.ex, m, n, Q, ldq));
    return apply_q_any(w, false, m, n, VR, lda, T, ldt, t_layout, nb, n, Q, ldq, true);
}

gbqr_status gbqr_ls_solve(gbqr_ctx *cx, int64_t m, int64_t n, const double *A, int64_t lda,
                          const double *b, double *x, int prec, gbqr_info *info) {
    if (!cx) return GBQR_EINVAL;
    if (prec != GBQR_FP64 && prec != GBQR_MIXED_BF16 && prec != GBQR_MIXED_SPLITBF16) return GBQR_EUNSUPPORTED;
    if (m < n || n < 0 || lda < std::max<int64_t>(1, m)) return GBQR_EINVAL;
    if (info) memset(info, 0, sizeof *info);
    if (info) info->rankdef_col = -1;
    if (n == 0) return GBQR_OK;
    if (!A || !b || !x) return GBQR_EINVAL;
    Params pr;
    gbqr_opts o;
    memset(&o, 0, sizeof o);
    o.update_prec = prec;
    gbqr_opts eff;
    // tuned cutoff / fan-out / leaf height / engine, but not the tuned panel
    // width: the tuner times the factorization alone, while every refinement
    // step applies Q and Q^T panel by panel (nb = 64 instead of 128 measured
    // 13 % slower for the mixed 32768 x 2048 solve)
    if (!resolve(with_tuned(cx, GBQR_TUNE_FACTOR, m, n, GBQR_T_PANEL, &o, &eff, false), m, n, &pr)) return GBQR_EINVAL;
    Work w;
    TRY(begin_work(cx, m, n, GBQR_T_PANEL, pr, &w));
    const int64_t nb = std::min<int64_t>(pr.nb, n);
    DeviceInfo *di = cx->dinfo;
    static const long long kNone = LLONG_MAX;
    if (cudaMemcpyAsync(&di->rankdef, &kNone, sizeof kNone, cudaMemcpyHostToDevice, cx->stream) != cudaSuccess)
        return GBQR_ECUDA;
    double *f = w.vec, *r = f + m, *nrm = r + m;          // nrm: 2 doubles (+ padding)
    double *dx = nrm + 16, *g = dx + n;
    // factor a copy of A; c = Q^T b; x = R^{-1} c(0:n)
    TRY(copy_matrix(w.ex, m, n, A, lda, w.bigA, m));
    TRY(factor_device(w, m, n, w.bigA, m, w.bigT, nb, GBQR_T_PANEL));
    TRY(copy_matrix(w.ex, m, 1, b, m, f, m));
    TRY(apply_q_any(w, true, m, n, w.bigA, m, w.bigT, nb, GBQR_T_PANEL, nb, 1, f, m, false));
    TRY(copy_matrix(w.ex, n, 1, f, n, x, n));
    // the mixed path solves with R a dozen times: invert its diagonal blocks
    // once, and every block step becomes a small matrix-vector product
    const double *dinv = (prec != GBQR_FP64) ? w.dinv : nullptr;
    if (dinv) TRY(trsv_block_inverses(w.ex, n, w.bigA, m, w.dinv, &di->rankdef));
    // with the block inverses, each solve is one launch of the block chain
    auto solve_r = [&](bool trans, double *v) -> gbqr_status {
        if (dinv) return trsv_chain(w.ex, trans, n, w.bigA, m, v, dinv, w.gs.counters, w.gs.ncounters, &di->timeout);
        return trans ? trsv_upper_t(w.ex, n, w.bigA, m, v, &di->rankdef, dinv)
                     : trsv_upper(w.ex, n, w.bigA, m, v, &di->rankdef, dinv);
    };
    TRY(solve_r(false, x));
    // Refinement on the augmented system K [r; x] = [b; 0], K = [I A; A^T 0],
    // with FP64 residuals.  The mixed QR solves K approximately (M^{-1}):
    //   h = R^{-T} g,  d = Q^T f,  dx = R^{-1} (d(0:n) - h),  dr = Q [h; d(n:m)].
    // Corrections are computed by GMRES on M^{-1} K with the mixed factors as
    // preconditioner until the backward error reaches its target (the
    // three-precision GMRES-IR for least squares of Carson, Higham and
    // Pranesh, here with FP64 residuals and working precision and
    // split-BF16 factors).
    double *dr = g + n, *tmp = dr + m;                     // m and n doubles
    auto read = [&](const double *dev, double *host, int count) -> gbqr_status {
        if (cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, cx->stream) != cudaSuccess ||
            cudaStreamSynchronize(cx->stream) != cudaSuccess)
            return GBQR_ECUDA;
        return GBQR_OK;
    };
    // normwise backward error of the LS solution, s = b - A x (FP64):
    //   eta = ||A^T s|| / (||A||_F ||s|| + ||A||_F^2 ||x||),
    // and the target it is held to: the level that rounding in forming s and
    // A^T s in FP64 leaves even for the exact solution, about
    //   u (1 + sqrt(m) ||s|| / (||s|| + ||A||_F ||x||))   (u = 2^-53),
    // times 4.  Small-residual problems must reach a few u; large-residual
    // ones are allowed the sqrt(m) u floor of the A^T s product.
    TRY(frob2(w.ex, m, n, A, lda, tmp, nrm + 4));
    double eta_tol = 0.0;
    auto backward_error = [&](double *eta) -> gbqr_status {
        TRY(copy_matrix(w.ex, m, 1, b, m, dr, m));
        TRY(gemv_n(w.ex, m, n, A, lda, x, -1.0, 1.0, dr, w.gs.partial, w.gs.partial_elems));
        TRY(gemv_t(w.ex, m, n, A, lda, dr, 1.0, 0.0, tmp));
        TRY(norms2(w.ex, n, tmp, x, nrm));
        TRY(norms2(w.ex, m, dr, dr, nrm + 2));
        double h[5];
        TRY(read(nrm, h, 5));
        const double an = std::sqrt(h[4]), sn = std::sqrt(h[2]), axn = an * std::sqrt(h[1]);
        const double den = an * sn + an * axn;
        *eta = den > 0.0 ? std::sqrt(h[0]) / den : (h[0] > 0.0 ? INFINITY : 0.0);
        const double wres = (sn + axn) > 0.0 ? sn / (sn + axn) : 1.0;
        eta_tol = 4.0 * 0x1.0p-53 * (1.0 + std::sqrt((double)m) * wres);
        return GBQR_OK;
    };
    int iters = 0;
    int64_t gmres_steps = 0;
    double last = 0.0, eta = 0.0;
    if (prec != GBQR_FP64) {
        auto precond = [&](double *fv, double *gv, double *dxv) -> gbqr_status {
            // in (fv, gv); out: dr in fv, dx in dxv; gv is overwritten (h)
            TRY(solve_r(true, gv));
            TRY(apply_q_any(w, true, m, n, w.bigA, m, w.bigT, nb, GBQR_T_PANEL, nb, 1, fv, m, false));
            TRY(copy_matrix(w.ex, n, 1, fv, n, dxv, n));
            TRY(axpby(w.ex, n, -1.0, gv, 1.0, dxv));
            TRY(solve_r(false, dxv));
            TRY(copy_matrix(w.ex, n, 1, gv, n, fv, n));
            return apply_q_any(w, false, m, n, w.bigA, m, w.bigT, nb, GBQR_T_PANEL, nb, 1, fv, m, false);
        };
        auto residual = [&]() -> gbqr_status {          // f = b - r - A x, g = -A^T r
            TRY(copy_matrix(w.ex, m, 1, b, m, f, m));
            TRY(axpby(w.ex, m, -1.0, r, 1.0, f));
            TRY(gemv_n(w.ex, m, n, A, lda, x, -1.0, 1.0, f, w.gs.partial, w.gs.partial_elems));
            return gemv_t(w.ex, m, n, A, lda, r, -1.0, 0.0, g);
        };
        auto step_ratio = [&](const double *dxv, double *ratio) -> gbqr_status {   // ||dx|| / ||x||
            TRY(norms2(w.ex, n, dxv, x, nrm));
            double hn[2];
            TRY(read(nrm, hn, 2));
            *ratio = hn[1] > 0.0 ? std::sqrt(hn[0] / hn[1]) : (hn[0] > 0.0 ? INFINITY : 0.0);
            return GBQR_OK;
        };
        TRY(copy_matrix(w.ex, m, 1, b, m, r, m));
        TRY(gemv_n(w.ex, m, n, A, lda, x, -1.0, 1.0, r, w.gs.partial, w.gs.partial_elems));
        TRY(backward_error(&eta));
        // GMRES-IR: each correction solves the augmented system by GMRES
        // preconditioned with the mixed factors.  The Krylov space of M^{-1} K
        // holds the iterates of classical refinement, so GMRES never needs
        // more operator applications than it, and it keeps converging where
        // kappa(A) u_f > 1 makes classical refinement diverge.  GMRES works on
        // Bjorck's scaled system K_a [r / a; x] = [b; 0], K_a = [aI A; A^T 0]
        // with a = sigma_min(A) / sqrt(2) (estimated by min |R(j,j)|): kappa(K_1)
        // grows like kappa(A)^2, kappa(K_a) only like 2 kappa(A).  With
        // D = diag(a I_m, I_n), K_a = D K_1 D in the variables D^{-1}[r; x],
        // so the preconditioned operator is D^{-1} (M^{-1} K_1) D and the
        // unscaled solves are reused.
        if (eta > eta_tol && w.kry) {
            const int64_t N = m + n;
            std::vector<double> diag(n);
            if (cudaMemcpy2DAsync(diag.data(), sizeof(double), w.bigA, (size_t)(m + 1) * sizeof(double),
                                  sizeof(double), n, cudaMemcpyDeviceToHost, cx->stream) != cudaSuccess ||
                cudaStreamSynchronize(cx->stream) != cudaSuccess)
                return GBQR_ECUDA;
            double rmin = INFINITY;
            for (double v : diag) rmin = std::min(rmin, std::fabs(v));
            const double alpha = (rmin > 0.0 && std::isfinite(rmin)) ? rmin / std::sqrt(2.0) : 1.0;
            double *V = w.kry;                                  // Arnoldi basis, kKrylov + 1 columns of N
            double *dvec = V + (size_t)(kKrylov + 1) * N;       // the correction [dr; dx]
            double *hd = dvec + N;                              // projections (2 x (kKrylov + 1)) and a norm
            const int hstride = kKrylov + 1;
            std::vector<double> H((size_t)(kKrylov + 1) * kKrylov, 0.0), cs(kKrylov), sn(kKrylov),
                e(kKrylov + 1), hb(2 * hstride + 2), y(kKrylov);
            for (int outer = 0; outer < 8 && eta > eta_tol; ++outer) {
                TRY(residual());
                TRY(copy_matrix(w.ex, m, 1, f, m, V, m));
                TRY(copy_matrix(w.ex, n, 1, g, n, tmp, n));
                TRY(precond(V, tmp, V + m));                    // v0 = D^{-1} M^{-1} [f; g]
                TRY(axpby(w.ex, m, 1.0 / alpha, V, 0.0, V));
                TRY(norms2(w.ex, N, V, V, nrm));
                double h0[1];
                TRY(read(nrm, h0, 1));
                const double beta = std::sqrt(h0[0]);
                if (!(beta > 0.0) || !std::isfinite(beta)) break;
                TRY(axpby(w.ex, N, 1.0 / beta, V, 0.0, V));
                std::fill(e.begin(), e.end(), 0.0);
                e[0] = beta;
                int k = 0;
                for (int j = 0; j < kKrylov; ++j) {
                    double *vj = V + (size_t)j * N, *wv = V + (size_t)(j + 1) * N;
                    // w = D^{-1} M^{-1} K D v_j with K [t; u] = [t + A u; A^T t], t = a v_r
                    TRY(axpby(w.ex, m, alpha, vj, 0.0, wv));
                    TRY(gemv_t(w.ex, m, n, A, lda, wv, 1.0, 0.0, tmp));
                    TRY(gemv_n(w.ex, m, n, A, lda, vj + m, 1.0, 1.0, wv, w.gs.partial, w.gs.partial_elems));
                    TRY(precond(wv, tmp, wv + m));
                    TRY(axpby(w.ex, m, 1.0 / alpha, wv, 0.0, wv));
                    // classical Gram-Schmidt, twice
                    TRY(gemv_t(w.ex, N, j + 1, V, N, wv, 1.0, 0.0, hd));
                    TRY(gemv_n(w.ex, N, j + 1, V, N, hd, -1.0, 1.0, wv, w.gs.partial, w.gs.partial_elems));
                    TRY(gemv_t(w.ex, N, j + 1, V, N, wv, 1.0, 0.0, hd + hstride));
                    TRY(gemv_n(w.ex, N, j + 1, V, N, hd + hstride, -1.0, 1.0, wv, w.gs.partial, w.gs.partial_elems));
                    TRY(norms2(w.ex, N, wv, wv, hd + 2 * hstride));
                    TRY(read(hd, hb.data(), 2 * hstride + 1));
                    double *Hj = H.data() + (size_t)j * (kKrylov + 1);
                    for (int i = 0; i <= j; ++i) Hj[i] = hb[i] + hb[hstride + i];
                    const double hnext = std::sqrt(hb[2 * hstride]);
                    Hj[j + 1] = hnext;
                    for (int i = 0; i < j; ++i) {                  // previous Givens rotations
                        const double t = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
                        Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
                        Hj[i] = t;
                    }
                    const double rho = std::hypot(Hj[j], Hj[j + 1]);
                    cs[j] = rho > 0.0 ? Hj[j] / rho : 1.0;
                    sn[j] = rho > 0.0 ? Hj[j + 1] / rho : 0.0;
                    Hj[j] = rho;
                    Hj[j + 1] = 0.0;
                    e[j + 1] = -sn[j] * e[j];
                    e[j] = cs[j] * e[j];
                    k = j + 1;
                    if (!(hnext > 0.0) || std::fabs(e[j + 1]) <= 1e-10 * beta) break;
                    TRY(axpby(w.ex, N, 1.0 / hnext, wv, 0.0, wv));
                }
                // y = H(0:k, 0:k)^{-1} e(0:k); correction = V(:, 0:k) y
                for (int i = k - 1; i >= 0; --i) {
                    double t = e[i];
                    for (int l = i + 1; l < k; ++l) t -= H[(size_t)l * (kKrylov + 1) + i] * y[l];
                    const double d = H[(size_t)i * (kKrylov + 1) + i];
                    y[i] = d != 0.0 ? t / d : 0.0;
                }
                if (cudaMemcpyAsync(hd, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, cx->stream) != cudaSuccess)
                    return GBQR_ECUDA;
                TRY(gemv_n(w.ex, N, k, V, N, hd, 1.0, 0.0, dvec, w.gs.partial, w.gs.partial_elems));
                double ratio = 0.0;
                TRY(step_ratio(dvec + m, &ratio));
                if (!(ratio == ratio)) break;
                TRY(axpby(w.ex, n, 1.0, dvec + m, 1.0, x));
                TRY(axpby(w.ex, m, alpha, dvec, 1.0, r));        // back to r = a (r / a)
                ++iters;
                gmres_steps += k;
                last = ratio;
                TRY(backward_error(&eta));
                if (ratio <= 1e-16) break;
            }
        }
    } else {
        TRY(backward_error(&eta));
    }
    const bool converged = (prec == GBQR_FP64) || eta <= eta_tol;   // FP64: eta is reported only
    long long rk = -1;
    if (cudaMemcpyAsync(&rk, &di->rankdef, sizeof rk, cudaMemcpyDeviceToHost, cx->stream) != cudaSuccess)
        return GBQR_ECUDA;
    if (cudaStreamSynchronize(cx->stream) != cudaSuccess) return GBQR_ECUDA;
    if (rk == LLONG_MAX) rk = -1;
    if (info) {
        info->rankdef_col = rk;
        info->refine_iters = iters;
        info->refine_last = last;
        info->gmres_steps = gmres_steps;
        info->backward_err = eta;
    }
    if (rk >= 0) return GBQR_ERANKDEF;
    return converged ? GBQR_OK : GBQR_ENOCONV;
}

gbqr_status gbqr_factor_batched(gbqr_ctx *cx, int count, const int64_t *m, const int64_t *n, double *const *A,
                                const int64_t *lda, double *const *T, const int64_t *ldt, const gbqr_opts *opts) {
    if (!cx) return GBQR_EINVAL;
    gbqr_opts eff;
    return gbqr::factor_batched_untuned(cx, count, m, n, A, lda, T, ldt,
                                        with_tuned(cx, GBQR_TUNE_BATCHED, 0, 0, GBQR_T_PANEL, opts, &eff, false));
}

gbqr_status gbqr_factor_batched_f32(gbqr_ctx *cx, int count, const int64_t *m, const int64_t *n, float *const *A,
                                    const int64_t *lda, float *const *T, const int64_t *ldt, const gbqr_opts *opts) {
    if (!cx) return GBQR_EINVAL;
    if (opts && opts->update_prec != GBQR_FP64) return GBQR_EINVAL;   // FP32 throughout
    return gbqr::factor_batched_untuned(cx, count, m, n, A, lda, T, ldt, opts);
}

}  // extern "C"

template <class Real>
gbqr_status gbqr::factor_batched_untuned(gbqr_ctx *cx, int count, const int64_t *m, const int64_t *n, Real *const *A,
                                         const int64_t *lda, Real *const *T, const int64_t *ldt, const gbqr_opts *opts,
                                         bool prepare_only) {
    if (!cx || count < 0) return GBQR_EINVAL;
    if (count == 0) return GBQR_OK;
    if (!m || !n || !A || !lda || !T || !ldt) return GBQR_EINVAL;
    if (persistent_batch(opts)) {
        // one persistent launch (batched.cu); T in panels of width b
        if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
        const int b = opts && opts->cutoff_b ? opts->cutoff_b : kBatchCutoff;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(cx->stream, &cs) != cudaSuccess) return GBQR_ECUDA;
        const bool capturing = cs != cudaStreamCaptureStatusNone;
        BatchPlan *pl = nullptr;
        TRY(batched_plan<Real>(&cx->bplan[sizeof(Real) == 8 ? 0 : 1], cx->device, cx->num_sms, count, m, n, lda, ldt,
                               b, !capturing, &pl));
        if (capturing && cx->ws_bytes < batched_plan_bytes(pl)) return GBQR_EBUSY;
        TRY(ensure_workspace(cx, batched_plan_bytes(pl)));
        if (prepare_only) return GBQR_OK;
        void *owned = nullptr;
        const gbqr_status st = batched_enqueue<Real>(cx->exec(), pl, A, T, m, n, lda, ldt, cx->ws, cx->ws_bytes,
                                                     &cx->dinfo->timeout, &cx->dinfo->nonfinite, capturing, &owned);
        if (owned) cx->capture_owned.push_back(owned);
        return st;
    }
    int64_t mmax = 1, nmax = 1;
    std::vector<double> cost(count);
    for (int i = 0; i < count; ++i) {
        Params pi;
        if (!resolve(opts, m[i], n[i], &pi)) return GBQR_EINVAL;
        TRY(check_layout_args(m[i], n[i], lda[i], ldt[i], GBQR_T_PANEL, pi.nb));
        if (n[i] > 0 && (!A[i] || !T[i])) return GBQR_EINVAL;
        mmax = std::max(mmax, m[i]);
        nmax = std::max(nmax, n[i]);
        cost[i] = 2.0 * m[i] * (double)n[i] * n[i] - 2.0 * (double)n[i] * n[i] * n[i] / 3.0 + 1e5 * n[i];
    }
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    Params pr;
    if (!resolve(opts, mmax, nmax, &pr)) return GBQR_EINVAL;
    pr.lookahead = false;                       // one stream per lane
    if (!opts || opts->cutoff_b == 0) pr.b = kBatchCutoff;
    const int S = std::min(count, opts && opts->batch_streams > 0 ? std::min(opts->batch_streams, kMaxBatchLanes) : kBatchLanes);
    const int lane_sms = std::max(8, (2 * cx->num_sms + S - 1) / S);
    const Layout L = make_layout(mmax, nmax, GBQR_T_PANEL, pr, lane_sms, /*staging=*/false);
    const size_t lane_bytes = align_up(L.total, 256);
    TRY(ensure_workspace(cx, lane_bytes * S));
    // lane streams and their completion events (created on first use: make
    // the first batched call before any stream capture)
    while ((int)cx->lanes.size() < S) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return GBQR_ECUDA;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) { cudaStreamDestroy(st); return GBQR_ECUDA; }
        cx->lanes.push_back(st);
        cx->lane_done.push_back(ev);
    }
    if (prepare_only) return GBQR_OK;
    // largest problems first, each to the least loaded lane
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int>> work(S);
    std::vector<double> load(S, 0.0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        work[l].push_back(i);
        load[l] += cost[i];
    }
    // fork from the context stream, one lane per stream, join back
    if (cudaEventRecord(cx->ev_fork, cx->stream) != cudaSuccess) return GBQR_ECUDA;
    for (int l = 0; l < S; ++l) {
        if (cudaStreamWaitEvent(cx->lanes[l], cx->ev_fork, 0) != cudaSuccess) return GBQR_ECUDA;
        Exec ex = cx->exec();
        ex.stream = cx->lanes[l];
        ex.num_sms = lane_sms;
        Work w;
        carve_work(cx, cx->ws + lane_bytes * l, L, pr, ex, &w);
        TRY(zero_counters(w, ex.stream));
        for (int i : work[l]) {
            if (n[i] == 0) continue;
            Params pi;
            resolve(opts, m[i], n[i], &pi);
            w.pr.nb = pi.nb;   // the cutoff stays the batch's (pr.b)
            TRY(factor_device(w, m[i], n[i], A[i], lda[i], T[i], ldt[i], GBQR_T_PANEL));
        }
        if (cudaEventRecord(cx->lane_done[l], ex.stream) != cudaSuccess) return GBQR_ECUDA;
        if (cudaStreamWaitEvent(cx->stream, cx->lane_done[l], 0) != cudaSuccess) return GBQR_ECUDA;
    }
    return GBQR_OK;
}

template gbqr_status gbqr::factor_batched_untuned<double>(gbqr_ctx *, int, const int64_t *, const int64_t *,
                                                          double *const *, const int64_t *, double *const *,
                                                          const int64_t *, const gbqr_opts *, bool);
template gbqr_status gbqr::factor_batched_untuned<float>(gbqr_ctx *, int, const int64_t *, const int64_t *,
                                                         float *const *, const int64_t *, float *const *,
                                                         const int64_t *, const gbqr_opts *, bool);

extern "C" {

size_t gbqr_batched_workspace_bytes(int count, const int64_t *m, const int64_t *n, const gbqr_opts *opts) {
    if (count <= 0 || !m || !n) return 0;
    if (persistent_batch(opts)) {
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const int b = opts && opts->cutoff_b ? opts->cutoff_b : kBatchCutoff;
        std::vector<int64_t> ld(count), ldt(count);
        for (int i = 0; i < count; ++i) {
            ld[i] = std::max<int64_t>(1, m[i]);
            ldt[i] = std::max<int64_t>(1, std::min<int64_t>(b, n[i]));
        }
        gbqr::BatchPlan *cache = nullptr, *pl = nullptr;
        const gbqr_status st = gbqr::batched_plan<double>(&cache, dev, sms, count, m, n, ld.data(), ldt.data(), b,
                                                          true, &pl);
        const size_t bytes = st == GBQR_OK ? gbqr::batched_plan_bytes(pl) : 0;
        gbqr::batch_plan_free(cache);
        return bytes;
    }
    int64_t mmax = 1, nmax = 1;
    for (int i = 0; i < count; ++i) {
        if (m[i] < n[i] || n[i] < 0) return 0;
        mmax = std::max(mmax, m[i]);
        nmax = std::max(nmax, n[i]);
    }
    Params pr;
    if (!resolve(opts, mmax, nmax, &pr)) return 0;
    pr.lookahead = false;
    if (!opts || opts->cutoff_b == 0) pr.b = kBatchCutoff;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 152;
    }
    const int S = std::min(count, opts && opts->batch_streams > 0 ? std::min(opts->batch_streams, kMaxBatchLanes) : kBatchLanes);
    const int lane_sms = std::max(8, (2 * sms + S - 1) / S);
    return align_up(make_layout(mmax, nmax, GBQR_T_PANEL, pr, lane_sms, false).total, 256) * S;
}

struct gbqr_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void *> owned;   // page-locked tables its memcpy nodes read at every launch
};

gbqr_status gbqr_graph_begin(gbqr_ctx *cx) {
    if (!cx) return GBQR_EINVAL;
    if (cx->tracing) return GBQR_EBUSY;
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    gbqr::ctx_free_capture_owned(cx);   // left by a capture that was not ended
    return cudaStreamBeginCapture(cx->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess ? GBQR_OK : GBQR_ECUDA;
}

gbqr_status gbqr_graph_end(gbqr_ctx *cx, gbqr_graph **out) {
    if (!cx || !out) return GBQR_EINVAL;
    *out = nullptr;
    gbqr_graph *g = new (std::nothrow) gbqr_graph();
    if (!g) return GBQR_ENOMEM;
    if (cudaStreamEndCapture(cx->stream, &g->graph) != cudaSuccess ||
        cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        if (g->graph) cudaGraphDestroy(g->graph);
        gbqr::ctx_free_capture_owned(cx);
        delete g;
        return GBQR_ECUDA;
    }
    g->owned.swap(cx->capture_owned);
    *out = g;
    return GBQR_OK;
}

gbqr_status gbqr_graph_launch(gbqr_ctx *cx, gbqr_graph *g) {
    if (!cx || !g) return GBQR_EINVAL;
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    return cudaGraphLaunch(g->exec, cx->stream) == cudaSuccess ? GBQR_OK : GBQR_ECUDA;
}

gbqr_status gbqr_graph_destroy(gbqr_graph *g) {
    if (!g) return GBQR_EINVAL;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (void *h : g->owned) cudaFreeHost(h);
    delete g;
    return GBQR_OK;
}

gbqr_status gbqr_trace_enable(gbqr_ctx *cx, int on) {
    if (!cx || !cx->tracer) return GBQR_EINVAL;
    cx->tracing = on != 0;
    return GBQR_OK;
}

gbqr_status gbqr_trace_read(gbqr_ctx *cx, gbqr_trace_rec *out, int max, int *count) {
    if (!cx || !cx->tracer || (max > 0 && !out)) return GBQR_EINVAL;
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    if (cudaStreamSynchronize(cx->stream) != cudaSuccess) return GBQR_ECUDA;
    gbqr_trace_rec agg[FAM_COUNT];
    memset(agg, 0, sizeof agg);
    for (int f = 0; f < FAM_COUNT; ++f) strncpy(agg[f].name, kFamilyNames[f], sizeof agg[f].name - 1);
    EventTracer *t = cx->tracer;
    for (auto &r : t->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t->pool[r.e0], t->pool[r.e1]) != cudaSuccess) return GBQR_ECUDA;
        agg[r.f].launches += 1;
        agg[r.f].ms += ms;
        agg[r.f].flops += r.flops;
        agg[r.f].bytes += r.bytes;
    }
    t->recs.clear();
    t->used = 0;
    int c = 0;
    for (int f = 0; f < FAM_COUNT && c < max; ++f)
        if (agg[f].launches) out[c++] = agg[f];
    if (count) *count = c;
    return t->failed ? GBQR_ECUDA : GBQR_OK;
}

int64_t gbqr_launch_count(const gbqr_ctx *cx) { return cx ? cx->launches : 0; }

gbqr_status gbqr_gemm_split_bf16(gbqr_ctx *cx, int transa, int64_t M, int64_t N, int64_t K, double alpha,
                                 const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                                 double *C, int64_t ldc, int nsplit) {
    if (!cx) return GBQR_EINVAL;
    if (M < 0 || N < 0 || K < 0 || nsplit < 1 || nsplit > 3) return GBQR_EINVAL;
    if (lda < std::max<int64_t>(1, transa ? K : M) || ldb < std::max<int64_t>(1, K) || ldc < std::max<int64_t>(1, M))
        return GBQR_EINVAL;
    if (M == 0 || N == 0) return GBQR_OK;
    if (!A || !B || !C) return GBQR_EINVAL;
    if (cudaSetDevice(cx->device) != cudaSuccess) return GBQR_ECUDA;
    const size_t need = tc_gemm_scratch_bytes(M, N, std::max<int64_t>(K, 1), cx->num_sms);
    TRY(ensure_workspace(cx, need));
    Exec ex = cx->exec();
    TcGemmOp op;
    op.M = M; op.N = N; op.K = K;
    op.A = A; op.lda = lda; op.ta = transa != 0;
    op.B = B; op.ldb = ldb;
    op.C = C; op.ldc = ldc; op.alpha = alpha; op.beta = beta;
    op.nsplit = nsplit;
    TcScratch sc;
    sc.base = cx->ws;
    sc.bytes = cx->ws_bytes;
    sc.err = &cx->dinfo->timeout;
    if (K == 0) {
        // C = beta * C: one FP64 GEMM launch with an empty K range does exactly that
        GemmOp g;
        g.M = M; g.N = N; g.K = 0; g.A = A; g.lda = lda; g.B = B; g.ldb = 1; g.C = C; g.ldc = ldc;
        g.alpha = alpha; g.beta = beta;
        GemmScratch gs;
        return gemm(ex, g, gs);
    }
    return tc_gemm(ex, op, sc);
}

}  // extern "C"
