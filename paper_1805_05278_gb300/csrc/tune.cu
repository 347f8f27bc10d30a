// Autotuner for the algorithm's free parameters.
//
// The paper trades latency against bandwidth and flops through the block
// sizes of its distributed schedules (the cutoff b of Algorithm 2, the
// reduction-tree shape of TSQR in Section 5 and Appendix C, the panel width of
// a right-looking top level in Section 8.4) and picks them from an alpha-beta-
// gamma cost model.  On one GPU the same trade-off reappears as
//   b        QR-EG cutoff: narrower base cases mean more, smaller GEMMs but
//            shorter serial reflector chains in the TSQR leaves;
//   k        TSQR tree fan-out: fewer levels (serial merges) vs. bigger ones;
//   m_p      TSQR leaf height: more CTAs vs. more work per leaf;
//   nb       top-level panel width (PANEL layout);
//   look-ahead on/off and the FP64 GEMM engine,
// and no closed-form model predicts the FP64 issue-bound kernels well, so the
// tuner measures: coordinate descent from the library defaults, one parameter
// at a time, each candidate timed with CUDA events on the context's stream
// (best of a few runs after one warm-up) on a synthetic matrix of the
// requested shape.  A candidate replaces the incumbent only when it is at
// least 1% faster.  The search stops early when the wall-clock budget would
// be exceeded.  The winner is cached in the context, keyed by the shape's
// power-of-two class, precision and layout, and later calls with zero
// (default) fields pick it up.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

namespace gbqr {
namespace {

// Uniform [-1, 1) from the splitmix64 finaliser of (seed + i * golden gamma)
// (Steele, Lea, Flood 2014): timing inputs only; the values do not matter.
__global__ void __launch_bounds__(kThreads) fill_uniform_kernel(int64_t count, uint64_t seed, double *x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (double)(z >> 11) * 0x1.0p-52 - 1.0;
    }
}

cudaError_t fill_uniform(cudaStream_t st, int num_sms, int64_t count, uint64_t seed, double *x) {
    if (count <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((count + kThreads - 1) / kThreads, (int64_t)num_sms * 8);
    fill_uniform_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(count, seed, x);
    return cudaPeekAtLastError();
}

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// One measured configuration: best of `reps` timed runs after one warm-up.
// `run` enqueues the work on `st` (after `prep`, which is not timed).
template <class Prep, class Run>
gbqr_status time_best(cudaStream_t st, int reps, Prep prep, Run run, double *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return GBQR_ECUDA;
    }
    double best = 1e300;
    gbqr_status st_out = GBQR_OK;
    for (int r = 0; r <= reps && st_out == GBQR_OK; ++r) {
        if (prep() != cudaSuccess) { st_out = GBQR_ECUDA; break; }
        if (cudaEventRecord(e0, st) != cudaSuccess) { st_out = GBQR_ECUDA; break; }
        st_out = run();
        if (st_out != GBQR_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st_out = GBQR_ECUDA; break; }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) best = std::min(best, (double)t);      // r == 0 is the warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return st_out;
}

// Coordinate descent over `axes` (each a field of gbqr_opts and its candidate
// values), starting from `start`.  `measure(opts, &ms)` times one candidate.
struct Axis {
    int32_t gbqr_opts::*field;
    std::vector<int32_t> values;
};

template <class Measure>
gbqr_status descend(const gbqr_opts &start, const std::vector<Axis> &axes, double budget_ms, Measure measure,
                    gbqr_opts *best, double *best_ms, int *trials) {
    const auto t0 = Clock::now();
    gbqr_opts cur = start;
    double cur_ms = 0.0;
    TRY_ST(measure(cur, &cur_ms));
    int n_trials = 1;
    for (const Axis &ax : axes) {
        for (int32_t v : ax.values) {
            if (cur.*(ax.field) == v) continue;
            // stop when one more trial (about 3 runs of the incumbent) would overrun
            if (ms_since(t0) + 3.5 * cur_ms > budget_ms) goto done;
            gbqr_opts cand = cur;
            cand.*(ax.field) = v;
            double ms = 0.0;
            const gbqr_status s = measure(cand, &ms);
            ++n_trials;
            if (s == GBQR_ENOMEM || s == GBQR_EINVAL) continue;   // candidate not feasible here
            if (s != GBQR_OK) return s;
            if (ms < 0.99 * cur_ms) { cur = cand; cur_ms = ms; }
        }
    }
done:
    *best = cur;
    *best_ms = cur_ms;
    if (trials) *trials = n_trials;
    return GBQR_OK;
}

int reps_for(double ms) { return ms < 5.0 ? 5 : (ms < 50.0 ? 3 : 2); }

}  // namespace
}  // namespace gbqr

using namespace gbqr;

extern "C" {

GBQR_API gbqr_status gbqr_autotune(gbqr_ctx *ctx, int64_t m, int64_t n, int t_layout, int update_prec,
                                   double budget_ms, gbqr_opts *best, double *best_ms) {
    if (!ctx || !best || m < n || n < 1 || budget_ms < 0.0) return GBQR_EINVAL;
    if (t_layout != GBQR_T_FULL && t_layout != GBQR_T_PANEL) return GBQR_EINVAL;
    if (update_prec != GBQR_FP64 && update_prec != GBQR_MIXED_BF16 && update_prec != GBQR_MIXED_SPLITBF16)
        return GBQR_EINVAL;
    if (t_layout == GBQR_T_FULL && update_prec != GBQR_FP64) return GBQR_EINVAL;
    const int dev = ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) return GBQR_ECUDA;
    cudaStream_t st = ctx_stream(ctx);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    constexpr int64_t kMaxNb = 256;
    const int64_t ldt = (t_layout == GBQR_T_FULL) ? n : std::min<int64_t>(kMaxNb, n);
    double *A = nullptr, *T = nullptr;
    if (cudaMalloc(&A, (size_t)m * n * 8) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
    if (cudaMalloc(&T, (size_t)ldt * n * 8) != cudaSuccess) { cudaGetLastError(); cudaFree(A); return GBQR_ENOMEM; }

    gbqr_opts start;
    memset(&start, 0, sizeof start);
    start.update_prec = update_prec;
    start.cutoff_b = 16;
    start.fanout = 0;   // the planner's adaptive fan-out
    start.lookahead = 1;
    start.fp64_gemm = GBQR_GEMM_DFMA;
    if (t_layout == GBQR_T_PANEL) start.panel_nb = (int32_t)gbqr_default_panel_nb(m, n);

    std::vector<Axis> axes;
    axes.push_back({&gbqr_opts::cutoff_b, {8, 16, 32, 64}});
    axes.push_back({&gbqr_opts::fanout, {0, 2, 4, 8, 16}});
    axes.push_back({&gbqr_opts::leaf_rows, {0, 128, 256, 512, 1024}});
    if (t_layout == GBQR_T_PANEL) {
        std::vector<int32_t> nbs;
        for (int32_t v : {64, 128, 192, 256})
            if (v <= ldt) nbs.push_back(v);
        axes.push_back({&gbqr_opts::panel_nb, nbs});
        axes.push_back({&gbqr_opts::lookahead, {1, -1}});
    }
    if (update_prec == GBQR_FP64) axes.push_back({&gbqr_opts::fp64_gemm, {GBQR_GEMM_DFMA, GBQR_GEMM_DMMA}});

    uint64_t seed = 0x5EEDull;
    int reps = 0;
    auto measure = [&](const gbqr_opts &o, double *ms) -> gbqr_status {
        auto prep = [&]() { return fill_uniform(st, sms, m * n, seed, A); };
        auto run = [&]() { return factor_untuned(ctx, m, n, A, m, T, ldt, t_layout, &o); };
        if (reps == 0) {   // size the repetitions from one untimed run of the start point
            double probe = 0.0;
            TRY_ST(time_best(st, 1, prep, run, &probe));
            reps = reps_for(probe);
        }
        return time_best(st, reps, prep, run, ms);
    };
    double ms = 0.0;
    const gbqr_status s = descend(start, axes, budget_ms, measure, best, &ms, nullptr);
    cudaStreamSynchronize(st);
    cudaFree(A);
    cudaFree(T);
    if (s != GBQR_OK) return s;
    if (best_ms) *best_ms = ms;
    ctx_store_tuned(ctx, tune_key(GBQR_TUNE_FACTOR, m, n, t_layout, update_prec), *best);
    return GBQR_OK;
}

GBQR_API gbqr_status gbqr_autotune_batched(gbqr_ctx *ctx, int count, const int64_t *m, const int64_t *n,
                                           int update_prec, double budget_ms, gbqr_opts *best, double *best_ms) {
    if (!ctx || !best || count < 1 || !m || !n || budget_ms < 0.0) return GBQR_EINVAL;
    if (update_prec != GBQR_FP64 && update_prec != GBQR_MIXED_BF16 && update_prec != GBQR_MIXED_SPLITBF16)
        return GBQR_EINVAL;
    std::vector<int64_t> offA(count + 1, 0), offT(count + 1, 0), ld(count), ldt(count);
    for (int i = 0; i < count; ++i) {
        if (m[i] < n[i] || n[i] < 0) return GBQR_EINVAL;
        ld[i] = std::max<int64_t>(1, m[i]);
        ldt[i] = std::max<int64_t>(1, n[i]);        // holds any panel width <= n
        offA[i + 1] = offA[i] + ld[i] * n[i];
        offT[i + 1] = offT[i] + ldt[i] * n[i];
    }
    const int dev = ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) return GBQR_ECUDA;
    cudaStream_t st = ctx_stream(ctx);
    if (cudaStreamSynchronize(st) != cudaSuccess) return GBQR_ECUDA;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *A = nullptr, *T = nullptr;
    if (cudaMalloc(&A, (size_t)std::max<int64_t>(offA[count], 1) * 8) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
    if (cudaMalloc(&T, (size_t)std::max<int64_t>(offT[count], 1) * 8) != cudaSuccess) { cudaGetLastError(); cudaFree(A); return GBQR_ENOMEM; }
    std::vector<double *> pa(count), pt(count);
    for (int i = 0; i < count; ++i) { pa[i] = A + offA[i]; pt[i] = T + offT[i]; }

    gbqr_opts start;
    memset(&start, 0, sizeof start);
    start.update_prec = update_prec;
    start.cutoff_b = 16;
    // the persistent batched kernel (panel width = cutoff b): b is its only
    // parameter; its row-block height follows from b and shared memory
    std::vector<Axis> axes;
    axes.push_back({&gbqr_opts::cutoff_b, {8, 16, 24, 32}});

    // A batch is meant to be replayed as one captured graph (gbqr_graph_*):
    // eager calls are bound by the host enqueueing thousands of launches, so
    // each candidate is captured on a private stream and its graph launches
    // are timed.  One eager call first creates the lanes and sizes the
    // workspace (neither may happen during a capture): prepare_only does
    // both without enqueueing the batch.
    cudaStream_t priv = nullptr;
    if (cudaStreamCreateWithFlags(&priv, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(A);
        cudaFree(T);
        return GBQR_ECUDA;
    }
    gbqr_set_stream(ctx, priv);
    int reps = 0;
    auto measure = [&](const gbqr_opts &o, double *ms) -> gbqr_status {
        auto call = [&](bool prepare_only) {
            return factor_batched_untuned(ctx, count, m, n, pa.data(), ld.data(), pt.data(), ldt.data(), &o,
                                          prepare_only);
        };
        auto prep = [&]() { return fill_uniform(priv, sms, offA[count], 0xBA7Cull, A); };
        TRY_ST(call(true));
        if (cudaStreamSynchronize(priv) != cudaSuccess) return GBQR_ECUDA;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(priv, cudaStreamCaptureModeRelaxed) != cudaSuccess) return GBQR_ECUDA;
        const gbqr_status cs = call(false);
        const cudaError_t ce = cudaStreamEndCapture(priv, &g);
        if (cs != GBQR_OK || ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            ctx_free_capture_owned(ctx);
            return cs != GBQR_OK ? cs : GBQR_ECUDA;
        }
        auto run = [&]() { return cudaGraphLaunch(ge, priv) == cudaSuccess ? GBQR_OK : GBQR_ECUDA; };
        if (reps == 0) {
            double probe = 0.0;
            gbqr_status s0 = time_best(priv, 1, prep, run, &probe);
            if (s0 != GBQR_OK) { cudaGraphExecDestroy(ge); cudaGraphDestroy(g); ctx_free_capture_owned(ctx); return s0; }
            reps = reps_for(probe);
        }
        const gbqr_status s = time_best(priv, reps, prep, run, ms);
        cudaGraphExecDestroy(ge);
        cudaGraphDestroy(g);
        ctx_free_capture_owned(ctx);   // the graph's page-locked tables
        return s;
    };
    double ms = 0.0;
    const gbqr_status s = ctx_tracing(ctx) ? GBQR_EBUSY : descend(start, axes, budget_ms, measure, best, &ms, nullptr);
    cudaStreamSynchronize(priv);
    gbqr_set_stream(ctx, st);
    cudaStreamDestroy(priv);
    cudaFree(A);
    cudaFree(T);
    if (s != GBQR_OK) return s;
    if (best_ms) *best_ms = ms;
    ctx_store_tuned(ctx, tune_key(GBQR_TUNE_BATCHED, 0, 0, GBQR_T_PANEL, update_prec), *best);
    return GBQR_OK;
}

GBQR_API gbqr_status gbqr_tuned_lookup(const gbqr_ctx *ctx, int kind, int64_t m, int64_t n, int t_layout,
                                       int update_prec, gbqr_opts *out) {
    if (!ctx || !out || (kind != GBQR_TUNE_FACTOR && kind != GBQR_TUNE_BATCHED)) return GBQR_EINVAL;
    const uint64_t key = (kind == GBQR_TUNE_BATCHED) ? tune_key(GBQR_TUNE_BATCHED, 0, 0, GBQR_T_PANEL, update_prec)
                                                : tune_key(GBQR_TUNE_FACTOR, m, n, t_layout, update_prec);
    return ctx_lookup_tuned(ctx, key, out) ? GBQR_OK : GBQR_EINVAL;
}

}  // extern "C"
