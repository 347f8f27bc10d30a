// Q^T x or Q x for ONE vector x, Q = Q_0 Q_1 ... Q_{p-1} from the panels of
// a factorization, Q_k = I - V_k T_k V_k^T (the basis-kernel form of Section
// 2.3, applied panel by panel as in the PANEL layout of Section 8.4) - the
// vector products of every least-squares solve and of each refinement step.
//
// One persistent launch does every panel.  Work items are (stage s, row block
// b): stage s finishes x -= V_{s-1} y_{s-1} for the panel applied before it
// (phase A) and forms this block's share of w_s = V_s^T x for the next panel
// (phase B); stage p does phase A only.  CTAs take items in ticket order from
// a counter.  The last item of a stage to arrive sums the blocks' shares in
// a fixed order, forms y_s = op(T_s) w_s and publishes it with a release
// store; items of stage s+1 wait (acquire) for that.  An item waits only for
// items with smaller tickets, which CTAs already running have taken, so the
// launch makes progress whether or not all of its CTAs are resident at once;
// the waits are still bounded by %globaltimer and raise the context's
// timeout flag when they run out.
//
// Row chunks of 64 (two rows per lane); warp g owns the g-th eighth of each
// panel's columns, so every V load is a coalesced 256-byte column segment,
// and a chunk issues all its loads (V_s, x, V_{s-1}) before its first
// barrier.  Chunks wholly below both panels' unit triangles take a path
// without masks.  Sums are in a fixed order: results do not depend on which
// CTA ran which item.
#include "common.cuh"

#include <algorithm>

namespace gbqr {
namespace {

constexpr int kChunk = 64;                     // rows per chunk (two per lane)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxW = kApplyVecMaxW;
constexpr int kTiles = kMaxW / 32;             // 32-wide blocks of T
static_assert(kMaxW % (32 * kWarps) == 0 && kMaxW <= kThreads, "one column of w per thread");
static_assert(kWarps * kChunk <= kTiles * kMaxW, "phase A partials fit the T-product buffer");

enum { kTicket = 0, kArrive = 1, kReady = 2, kDone = 3, kAbort = 4, kNumCounters = 5 };

struct ApplyVec {
    int64_t m, lda, ldt, R;    // R: rows per item (a multiple of kChunk)
    int n, pb, npan, nblk;     // panel width, panels, row blocks
    int trans, tfull;          // Q^T (else Q); T is the full n x n kernel (else nb x n panel kernels)
    const double *VR, *T;
    double *x;
    double *y;                 // 2 pb: y of the stage before, ping-pong
    double *partial;           // nblk pb: the blocks' shares of w
    unsigned *ctr;             // kNumCounters: zero on entry, left zero
    int *timeout;
    long long wait_ns;
};

struct Stage {
    int64_t jp, jk, lo;        // first column of the previous / current panel, first row touched
    int wp, wk;                // widths (0: absent)
    int b0, S;                 // first row block, number of items
};

__device__ __forceinline__ Stage stage_of(const ApplyVec &p, int s) {
    Stage st;
    st.jp = st.jk = p.m;
    st.wp = st.wk = 0;
    if (s > 0) {
        const int k = p.trans ? s - 1 : p.npan - s;
        st.jp = (int64_t)k * p.pb;
        st.wp = (int)min((int64_t)p.pb, (int64_t)p.n - st.jp);
    }
    if (s < p.npan) {
        const int k = p.trans ? s : p.npan - 1 - s;
        st.jk = (int64_t)k * p.pb;
        st.wk = (int)min((int64_t)p.pb, (int64_t)p.n - st.jk);
    }
    st.lo = min(st.jp, st.jk);
    st.b0 = (int)(st.lo / p.R);
    st.S = p.nblk - st.b0;
    return st;
}

__device__ __forceinline__ const double *panel_T(const ApplyVec &p, int64_t j) {
    return p.tfull ? p.T + j + j * p.ldt : p.T + j * p.ldt;
}

__device__ __forceinline__ int ld_acquire(const unsigned *q) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *q, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(q), "r"(v) : "memory");
}
// Arrival on a counter with acquire-release semantics at GPU scope: after
// a CTA barrier, thread 0's release publishes the whole CTA's earlier
// writes, and the last arriver's acquire (followed by a barrier) makes every
// arrived CTA's writes visible to its threads - no separate fences.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *q, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(q), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void prefetch_l2(const double *q) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Entry (r, c) of a unit lower trapezoidal panel whose diagonal starts at
// row top, given v = the stored value at (r, c): zero above the diagonal, one
// on it, v below it; zero where in is false (a row outside the item or a
// column the thread does not own).  Callers load v unconditionally from a
// clamped, always valid address, so that a chunk's loads are all in flight
// at once instead of each waiting behind its guard.
__device__ __forceinline__ double vsel(double v, int64_t rr, int c, bool in) {
    return (!in || rr < c) ? 0.0 : (rr == c ? 1.0 : v);
}

// Thread 0: wait until `want` stages are published.  False when the launch
// is aborting (a wait ran out here or elsewhere).
__device__ bool wait_ready(const ApplyVec &p, int want) {
    if (ld_acquire(p.ctr + kReady) >= want) return true;
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while (ld_acquire(p.ctr + kReady) < want) {
        if (*(volatile unsigned *)(p.ctr + kAbort)) return false;
        if (global_ns() - t0 > (unsigned long long)p.wait_ns) {
            atomicExch(p.ctr + kAbort, 1u);
            atomicExch(p.timeout, 1);
            return false;
        }
        __nanosleep(ns);
        if (ns < 256) ns *= 2;
    }
    return true;
}

struct Smem {
    double ys[kMaxW];                  // this stage's w (last arriver)
    double yw[kWarps * 32];            // warp g's slice of y_{s-1}, zero past its columns
    double part[kTiles * kMaxW];       // phase A partials (8 x 64), then share sums and T-tile partials
    double xs[kChunk];
    int flag;
    int ticket;
};

// Phase A and B of one item over rows [r0, r1): x -= V_{s-1} y_{s-1} on
// those rows, acc[j] += V_s(:, ck0 + j)^T x.
template <int CW>
__device__ void item_rows(const ApplyVec &p, const Stage &st, Smem &sm, int64_t r0, int64_t r1, double (&acc)[CW]) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int cwp = (st.wp + kWarps - 1) / kWarps, cwk = (st.wk + kWarps - 1) / kWarps;
    const int cp0 = g * cwp, ck0 = g * cwk, ck1 = min(st.wk, ck0 + cwk);
    const double *Vp = st.wp ? p.VR + st.jp * p.lda : nullptr;
    const double *Vk = st.wk ? p.VR + st.jk * p.lda : nullptr;
    const double *ywg = sm.yw + g * 32;
    for (int64_t s0 = r0; s0 < r1; s0 += kChunk) {
        const int64_t ra = s0 + lane, rb = ra + 32, rx = s0 + tid;
        if (s0 + kChunk < r1) {
            // the next chunk's column segments into L2 (four 128-byte lines
            // of a column per group of four lanes, eight columns per pass)
            const int64_t rn = min(s0 + kChunk + (lane & 3) * 16, r1 - 1);
            for (int j = lane >> 2; j < CW; j += 8) {
                if (Vk) prefetch_l2(Vk + (int64_t)min(ck0 + j, st.wk - 1) * p.lda + rn);
                if (Vp) prefetch_l2(Vp + (int64_t)min(cp0 + j, st.wp - 1) * p.lda + rn);
            }
        }
        const bool fast = s0 + kChunk <= r1 && (!Vk || s0 >= st.jk + st.wk) && (!Vp || s0 >= st.jp + st.wp);
        const bool ina = ra < r1, inb = rb < r1;
        const int64_t la = min(ra, r1 - 1), lb = min(rb, r1 - 1);    // clamped rows: valid addresses
        double vb0[CW], vb1[CW];
        if (Vk) {
            if (fast) {
                // columns past the warp's own load a valid duplicate; their
                // accumulators are never written out
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const double *q = Vk + (int64_t)min(ck0 + j, st.wk - 1) * p.lda + ra;
                    vb0[j] = __ldg(q);
                    vb1[j] = __ldg(q + 32);
                }
            } else {
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const int c = ck0 + j;
                    const int64_t off = (int64_t)min(c, st.wk - 1) * p.lda;
                    vb0[j] = vsel(__ldg(Vk + off + la), ra - st.jk, c, ina && c < ck1);
                    vb1[j] = vsel(__ldg(Vk + off + lb), rb - st.jk, c, inb && c < ck1);
                }
            }
        }
        double xv = 0.0;
        if (tid < kChunk && rx < r1) xv = __ldcg(p.x + rx);   // written by other CTAs' earlier items
        if (Vp) {
            double a0 = 0.0, a1 = 0.0;
            if (fast) {
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const double *q = Vp + (int64_t)min(cp0 + j, st.wp - 1) * p.lda + ra;
                    const double yc = ywg[j];
                    a0 = fma(__ldg(q), yc, a0);
                    a1 = fma(__ldg(q + 32), yc, a1);
                }
            } else {
#pragma unroll
                for (int j = 0; j < CW; ++j) {
                    const int c = cp0 + j;
                    const int64_t off = (int64_t)min(c, st.wp - 1) * p.lda;
                    const double yc = ywg[j];
                    a0 = fma(vsel(__ldg(Vp + off + la), ra - st.jp, c, ina), yc, a0);
                    a1 = fma(vsel(__ldg(Vp + off + lb), rb - st.jp, c, inb), yc, a1);
                }
            }
            sm.part[g * kChunk + lane] = a0;
            sm.part[g * kChunk + lane + 32] = a1;
        }
        __syncthreads();
        if (tid < kChunk) {
            if (Vp) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < kWarps; ++q) s += sm.part[q * kChunk + tid];
                xv -= s;
                if (rx < r1) __stcg(p.x + rx, xv);
            }
            sm.xs[tid] = xv;
        }
        __syncthreads();
        if (Vk) {
            const double xa = sm.xs[lane], xb = sm.xs[lane + 32];
#pragma unroll
            for (int j = 0; j < CW; ++j) acc[j] = fma(vb1[j], xb, fma(vb0[j], xa, acc[j]));
        }
    }
}

// Last arriver of stage s: w = sum of the S shares (fixed order, two halves
// for panels up to 128 wide), then y_s = op(T_s) w over the 32 x 32 tiles of
// T's triangle (one warp per tile, lane = output row, the tile's 32 loads
// independent).
__device__ void finish_stage(const ApplyVec &p, const Stage &st, Smem &sm, int s) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int wk = st.wk, S = st.S;
    const int halves = (wk <= kThreads / 2) ? 2 : 1;
    const int c = tid % (kThreads / halves), h = tid / (kThreads / halves);
    const int qa = h * ((S + halves - 1) / halves), qb = min(S, qa + (S + halves - 1) / halves);
    if (c < wk) {
        const double *src = p.partial + c;
        double acc = 0.0;
        for (int q0 = qa; q0 < qb; q0 += 32) {
            double v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = __ldcg(src + (int64_t)min(q0 + q, qb - 1) * wk);
#pragma unroll
            for (int q = 0; q < 32; ++q) acc += (q0 + q < qb) ? v[q] : 0.0;
        }
        sm.part[h * kMaxW + c] = acc;
    }
    __syncthreads();
    if (tid < wk) sm.ys[tid] = (halves == 2) ? sm.part[tid] + sm.part[kMaxW + tid] : sm.part[tid];
    __syncthreads();
    const double *Tk = panel_T(p, st.jk);
    const int nbk = (wk + 31) / 32;
    for (int t = g; t < nbk * nbk; t += kWarps) {
        const int I = t % nbk, L = t / nbk;
        if (p.trans ? (L > I) : (L < I)) continue;     // tile outside the triangle
        const int i = I * 32 + lane, ic = min(i, wk - 1);
        double tv[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int lc = min(L * 32 + q, wk - 1);
            tv[q] = __ldg(p.trans ? Tk + lc + (int64_t)ic * p.ldt : Tk + ic + (int64_t)lc * p.ldt);
        }
        double a = 0.0;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int l = L * 32 + q;
            // trans: y_i = sum_{l <= i} T(l, i) w_l;  else y_i = sum_{l >= i} T(i, l) w_l
            const bool ok = i < wk && l < wk && (p.trans ? l <= i : l >= i);
            a = ok ? fma(tv[q], sm.ys[min(l, kMaxW - 1)], a) : a;
        }
        if (i < wk) sm.part[L * kMaxW + i] = a;
    }
    __syncthreads();
    if (tid < wk) {
        const int I = tid / 32;
        const int lb = p.trans ? 0 : I, le = p.trans ? I : nbk - 1;
        double y = 0.0;
        for (int L = lb; L <= le; ++L) y += sm.part[L * kMaxW + tid];
        __stcg(p.y + (s & 1) * p.pb + tid, y);
    }
    __syncthreads();
    if (tid == 0) st_release(p.ctr + kReady, s + 1);   // publishes y_s (and the reset arrival count)
}

template <int CW>
__global__ void __launch_bounds__(kThreads, 1) apply_vec_kernel(ApplyVec p) {
    __shared__ Smem sm;
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    int s = 0;
    long long base = 0;                                  // items of the stages before s
    Stage st = stage_of(p, 0);
    for (;;) {
        __syncthreads();                                 // the previous item is done with shared memory
        if (tid == 0) sm.ticket = (int)atomicAdd(p.ctr + kTicket, 1u);
        __syncthreads();
        const long long t = sm.ticket;
        while (s <= p.npan && t >= base + st.S) {
            base += st.S;
            ++s;
            if (s <= p.npan) st = stage_of(p, s);
        }
        if (s > p.npan) break;
        const int b = st.b0 + (int)(t - base);
        if (tid == 0) sm.flag = wait_ready(p, s) ? 1 : 0;
        __syncthreads();
        if (!sm.flag) break;
        // y_{s-1}, split into the warps' column slices
        const int cwp = (st.wp + kWarps - 1) / kWarps;
        for (int i = tid; i < kWarps * 32; i += kThreads) {
            const int gg = i / 32, jj = i % 32, c = gg * cwp + jj;
            sm.yw[i] = (jj < cwp && c < st.wp) ? __ldcg(p.y + ((s - 1) & 1) * p.pb + c) : 0.0;
        }
        // this stage's T into L2 for whichever item arrives last: item i
        // takes columns i, i + S, ... (one 128-byte line per lane)
        if (st.wk && g == kWarps - 1)
            for (int c = b - st.b0; c < st.wk; c += st.S)
                if (lane * 16 < st.wk) prefetch_l2(panel_T(p, st.jk) + (int64_t)c * p.ldt + lane * 16);
        __syncthreads();
        double acc[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[j] = 0.0;
        const int64_t r0 = max((int64_t)b * p.R, st.lo), r1 = min((int64_t)(b + 1) * p.R, p.m);
        item_rows<CW>(p, st, sm, r0, r1, acc);
        if (st.wk == 0) continue;                        // the last stage: phase A only
        // this item's share of w: each owned column summed over the lanes
        const int cwk = (st.wk + kWarps - 1) / kWarps, ck0 = g * cwk, ck1 = min(st.wk, ck0 + cwk);
#pragma unroll
        for (int j = 0; j < CW; ++j) {
            double v = acc[j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0 && ck0 + j < ck1) sm.ys[ck0 + j] = v;
        }
        __syncthreads();
        if (tid < st.wk) __stcg(p.partial + (int64_t)(b - st.b0) * st.wk + tid, sm.ys[tid]);
        __syncthreads();
        if (tid == 0) {
            const bool last = atom_add_acq_rel(p.ctr + kArrive, 1u) == (unsigned)(st.S - 1);
            if (last) p.ctr[kArrive] = 0u;                // ordered before the release of y_s
            sm.flag = last ? 1 : 0;
        }
        __syncthreads();
        if (sm.flag) finish_stage(p, st, sm, s);
    }
    // the last CTA out resets the counters for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(p.ctr + kDone, 1u) == gridDim.x - 1) {
            p.ctr[kTicket] = 0u;
            p.ctr[kArrive] = 0u;
            p.ctr[kReady] = 0u;
            p.ctr[kAbort] = 0u;
            __threadfence();
            p.ctr[kDone] = 0u;
        }
    }
}

}  // namespace

gbqr_status apply_vec(const Exec &ex, bool trans, int64_t m, int64_t n, const double *VR, int64_t lda,
                      const double *T, int64_t ldt, bool tfull, int64_t pb, double *x, double *y2, size_t ny,
                      double *partial, size_t partial_elems, unsigned *counters, size_t ncounters, int *timeout) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    if (pb < 1 || pb > kMaxW || n > m || !timeout) return GBQR_EINVAL;
    const int64_t npan = (n + pb - 1) / pb;
    if (npan > 0x3fffffff) return GBQR_EUNSUPPORTED;
    // rows per item: whole chunks, about one item per SM for the longest stage
    const int64_t per = (m + ex.num_sms - 1) / ex.num_sms;
    const int64_t R = (per + kChunk - 1) / kChunk * kChunk;
    const int64_t nblk = (m + R - 1) / R;
    if ((size_t)(2 * pb) > ny || (size_t)(nblk * pb) > partial_elems || ncounters < kNumCounters) return GBQR_ENOMEM;
    ApplyVec p;
    p.m = m; p.lda = lda; p.ldt = ldt; p.R = R;
    p.n = (int)n; p.pb = (int)pb; p.npan = (int)npan; p.nblk = (int)nblk;
    p.trans = trans ? 1 : 0; p.tfull = tfull ? 1 : 0;
    p.VR = VR; p.T = T; p.x = x; p.y = y2; p.partial = partial; p.ctr = counters; p.timeout = timeout;
    p.wait_ns = 5000000000ll;   // 5 s: far beyond any stage's critical path
    const unsigned grid = (unsigned)std::min<int64_t>(nblk, ex.num_sms);
    // algorithmic traffic: each panel's V read twice (phases A and B), x in and out per stage
    double bytes = 0.0, flops = 0.0;
    for (int64_t k = 0; k < npan; ++k) {
        const int64_t j = k * pb, w = std::min<int64_t>(pb, n - j);
        bytes += 2.0 * 8.0 * (double)(m - j) * w + 8.0 * (double)w * w / 2 + 16.0 * (double)(m - j);
        flops += 4.0 * (double)(m - j) * w + (double)w * w;
    }
    trace_begin(ex, FAM_GEMV);
    if (pb <= 16 * kWarps)
        apply_vec_kernel<16><<<grid, kThreads, 0, ex.stream>>>(p);
    else
        apply_vec_kernel<32><<<grid, kThreads, 0, ex.stream>>>(p);
    return trace_end(ex, FAM_GEMV, flops, bytes);
}

}  // namespace gbqr
