// Least-squares serving loop with continuous batching (host side).
//
// Requests are queued by gbqr_submit and served by W worker threads, each
// owning a private context (its own CUDA stream), so the device overlaps the
// work of every admitted request.  Admission is by HBM footprint: a request
// starts when a worker is idle and its footprint (its workspace,
// gbqr_workspace_bytes for its shape and precision, plus its own A, b and x)
// fits under the byte cap together with the requests already running; the queue is scanned first-fit, so a small
// request can start while a large one waits for memory - but at most
// kMaxBypass later requests may start ahead of a waiting one: after that it
// blocks the queue until it fits (at the latest when nothing else runs), so
// no request waits indefinitely behind a stream of small ones.  Each request's
// workspace comes from the stream-ordered allocator and is returned when it
// completes, so memory freed by one request admits the next.
//
// GBQR_PREC_AUTO requests run the mixed path (tensor-core updates + FP64
// refinement) when the update GEMMs dominate their cost, FP64 otherwise, and
// fall back to FP64 when the refinement stalls (condition number beyond
// what FP32-level updates can refine).
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

// Later requests that may be admitted ahead of a waiting one.
constexpr int kMaxBypass = 8;

struct Record {
    gbqr_request req;
    size_t footprint = 0;
    int bypassed = 0;      // later requests admitted while this one waited
    int state = GBQR_REQ_QUEUED;
    gbqr_status status = GBQR_OK;
    int prec_used = GBQR_FP64;
    bool fell_back = false;
    int64_t iters = 0;
    Clock::time_point t_submit, t_start, t_done;
};

// GBQR_PREC_AUTO: the tensor-core updates only pay off where the update
// GEMMs dominate the solve.  Measured single-solve speed-ups of the mixed
// path over FP64 (graded columns, kappa ~ 1e4, two GMRES steps each):
// 3.19x at 65536 x 1024, 1.96x at 65536 x 512, 1.88x at 16384 x 1024,
// 1.36x at 16384 x 512, 1.32x at 65536 x 256, 1.12x at 8192 x 512, 1.08x
// at 16384 x 256, 1.01x at 2048 x 1024 (all m n^2 >= 1e9); slower below
// (0.96x at 8192 x 256, 0.93x at 2048 x 512) and at n <= 128 (0.63-0.94x):
// there the FP64 panel chain dominates and the refinement adds its steps.
int auto_precision(int64_t m, int64_t n) {
    return (n >= 256 && (double)m * n * n >= 1e9) ? GBQR_MIXED_SPLITBF16 : GBQR_FP64;
}

// The request's own device operands: A (lda x n), b (m) and x (n), FP64.
size_t operand_bytes(const gbqr_request &r) {
    return sizeof(double) * ((size_t)r.lda * (size_t)r.n + (size_t)r.m + (size_t)r.n);
}

// HBM a request holds while it runs: the workspace of gbqr_ls_solve for its
// shape and precision (with the serving context's autotuned parameters where
// it has some - the workers carry a copy of that cache, so they size their
// work the same way), plus its own A (lda x n), b (m) and x (n).
size_t footprint_of(const gbqr_ctx *cx, const gbqr_request &r, int prec) {
    gbqr_opts o;
    memset(&o, 0, sizeof o);
    if (gbqr::ctx_lookup_tuned(cx, gbqr::tune_key(GBQR_TUNE_FACTOR, r.m, r.n, GBQR_T_PANEL, prec), &o)) {
        o.batch_streams = 0;
    }
    o.update_prec = prec;
    return gbqr_workspace_bytes(r.m, r.n, GBQR_T_PANEL, &o) + ((size_t)1 << 20) + operand_bytes(r);
}

}  // namespace

struct gbqr_server {
    int device = 0;
    size_t cap = 0, in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Record> recs;
    uint64_t next_id = 1;
    bool stopping = false;
    int running = 0;
    std::vector<std::thread> workers;
    std::vector<gbqr_ctx *> ctxs;
    std::vector<cudaStream_t> streams;
};

namespace {

void worker_loop(gbqr_server *sv, int wi) {
    cudaSetDevice(sv->device);
    gbqr_ctx *cx = sv->ctxs[wi];
    cudaStream_t st = sv->streams[wi];
    for (;;) {
        uint64_t id = 0;
        Record *rec = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stopping && sv->queue.empty()) return;
                // first request (in arrival order) whose footprint fits; a
                // request already passed kMaxBypass times stops the scan, so
                // nothing behind it starts before it does
                auto it = sv->queue.begin();
                for (; it != sv->queue.end(); ++it) {
                    Record &r = sv->recs[*it];
                    if (sv->in_use + r.footprint <= sv->cap || sv->running == 0) break;
                    if (r.bypassed >= kMaxBypass) { it = sv->queue.end(); break; }
                }
                if (it != sv->queue.end()) {
                    for (auto jt = sv->queue.begin(); jt != it; ++jt) ++sv->recs[*jt].bypassed;
                    id = *it;
                    sv->queue.erase(it);
                    rec = &sv->recs[id];
                    sv->in_use += rec->footprint;
                    ++sv->running;
                    rec->state = GBQR_REQ_RUNNING;
                    rec->t_start = Clock::now();
                    break;
                }
                sv->cv_work.wait(lk);
            }
        }
        // run outside the lock; the record stays put (unordered_map nodes are stable)
        const gbqr_request r = rec->req;
        gbqr_status status = GBQR_OK;
        int64_t iters = 0;
        int used = r.prec;
        bool fell_back = false;
        void *ws = nullptr;
        const size_t ws_bytes = rec->footprint - operand_bytes(r);   // the rest is the caller's A, b, x
        if (cudaMallocAsync(&ws, ws_bytes, st) != cudaSuccess) {
            cudaGetLastError();
            status = GBQR_ENOMEM;
        } else {
            gbqr_set_workspace(cx, ws, ws_bytes);
            gbqr_info info;
            const int first = (r.prec == GBQR_PREC_AUTO) ? auto_precision(r.m, r.n) : r.prec;
            used = first;
            status = gbqr_ls_solve(cx, r.m, r.n, r.A, r.lda, r.b, r.x, first, &info);
            iters = info.refine_iters;
            if (r.prec == GBQR_PREC_AUTO && status == GBQR_ENOCONV) {
                used = GBQR_FP64;
                fell_back = true;
                status = gbqr_ls_solve(cx, r.m, r.n, r.A, r.lda, r.b, r.x, GBQR_FP64, &info);
            }
            gbqr_set_workspace(cx, nullptr, 0);
            cudaFreeAsync(ws, st);
            cudaStreamSynchronize(st);
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            rec->status = status;
            rec->iters = iters;
            rec->prec_used = used;
            rec->fell_back = fell_back;
            rec->t_done = Clock::now();
            rec->state = GBQR_REQ_DONE;
            sv->in_use -= rec->footprint;
            --sv->running;
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

// The server hangs off the context through a side table (the context layout
// lives in api.cu).
namespace {
std::mutex g_servers_mu;
std::unordered_map<const gbqr_ctx *, gbqr_server *> g_servers;

gbqr_server *server_of(const gbqr_ctx *cx) {
    std::lock_guard<std::mutex> lk(g_servers_mu);
    auto it = g_servers.find(cx);
    return it == g_servers.end() ? nullptr : it->second;
}
}  // namespace

extern "C" {

GBQR_API gbqr_status gbqr_server_start(gbqr_ctx *ctx, int device, int workers, size_t mem_cap_bytes) {
    if (!ctx || workers < 1 || workers > 256 || mem_cap_bytes == 0) return GBQR_EINVAL;
    if (server_of(ctx)) return GBQR_EBUSY;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    gbqr_server *sv = new (std::nothrow) gbqr_server();
    if (!sv) return GBQR_ENOMEM;
    sv->device = device;
    sv->cap = mem_cap_bytes;
    // keep freed request workspace cached in this process's pool (up to the cap)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = mem_cap_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    for (int i = 0; i < workers; ++i) {
        cudaStream_t st;
        gbqr_ctx *wc = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
        if (gbqr_create(&wc, device, st) != GBQR_OK) { cudaStreamDestroy(st); break; }
        gbqr::ctx_copy_tuned(ctx, wc);
        sv->streams.push_back(st);
        sv->ctxs.push_back(wc);
    }
    if ((int)sv->ctxs.size() != workers) {
        for (auto c : sv->ctxs) gbqr_destroy(c);
        for (auto st : sv->streams) cudaStreamDestroy(st);
        delete sv;
        return GBQR_ECUDA;
    }
    for (int i = 0; i < workers; ++i) sv->workers.emplace_back(worker_loop, sv, i);
    std::lock_guard<std::mutex> lk(g_servers_mu);
    g_servers[ctx] = sv;
    return GBQR_OK;
}

GBQR_API gbqr_status gbqr_submit(gbqr_ctx *ctx, const gbqr_request *req, uint64_t *id) {
    gbqr_server *sv = server_of(ctx);
    if (!sv || !req || !id) return GBQR_EINVAL;
    const gbqr_request &r = *req;
    if (r.m < r.n || r.n < 1 || r.lda < r.m || !r.A || !r.b || !r.x) return GBQR_EINVAL;
    if (r.prec != GBQR_FP64 && r.prec != GBQR_MIXED_BF16 && r.prec != GBQR_MIXED_SPLITBF16 && r.prec != GBQR_PREC_AUTO)
        return GBQR_EINVAL;
    Record rec;
    rec.req = r;
    // AUTO may fall back to FP64 inside the same workspace: size for both
    rec.footprint = (r.prec == GBQR_PREC_AUTO)
                        ? std::max(footprint_of(ctx, r, auto_precision(r.m, r.n)), footprint_of(ctx, r, GBQR_FP64))
                        : footprint_of(ctx, r, r.prec);
    if (rec.footprint > sv->cap) return GBQR_ENOMEM;
    rec.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) return GBQR_EBUSY;
        *id = sv->next_id++;
        sv->recs.emplace(*id, rec);
        sv->queue.push_back(*id);
    }
    sv->cv_work.notify_one();
    return GBQR_OK;
}

GBQR_API gbqr_status gbqr_poll(gbqr_ctx *ctx, uint64_t id, int wait, gbqr_result *out) {
    gbqr_server *sv = server_of(ctx);
    if (!sv || !out) return GBQR_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->recs.find(id);
    if (it == sv->recs.end()) return GBQR_EINVAL;
    if (wait) sv->cv_done.wait(lk, [&] { return it->second.state == GBQR_REQ_DONE; });
    const Record &r = it->second;
    memset(out, 0, sizeof *out);
    out->state = r.state;
    out->tag = r.req.tag;
    if (r.state == GBQR_REQ_DONE) {
        out->status = r.status;
        out->prec_used = r.prec_used;
        out->fell_back = r.fell_back ? 1 : 0;
        out->refine_iters = r.iters;
        out->queue_ms = ms_between(r.t_submit, r.t_start);
        out->run_ms = ms_between(r.t_start, r.t_done);
        out->latency_ms = ms_between(r.t_submit, r.t_done);
        out->footprint_bytes = (int64_t)r.footprint;
        out->bypassed = r.bypassed;
        sv->recs.erase(it);   // results are read once
    }
    return GBQR_OK;
}

GBQR_API gbqr_status gbqr_server_stop(gbqr_ctx *ctx) {
    gbqr_server *sv = server_of(ctx);
    if (!sv) return GBQR_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    for (auto c : sv->ctxs) gbqr_destroy(c);
    for (auto st : sv->streams) cudaStreamDestroy(st);
    {
        std::lock_guard<std::mutex> lk(g_servers_mu);
        g_servers.erase(ctx);
    }
    delete sv;
    return GBQR_OK;
}

}  // extern "C"
