// Q^T x or Q x for ONE vector x, Q = Q_0 Q_1 ... Q_{p-1} from the panels of
// a factorization, Q_k = I - V_k T_k V_k^T (the basis-kernel form of Section
// 2.3, applied panel by panel as in the PANEL layout of Section 8.4) - the
// vector products of every least-squares solve and of each refinement step.
//
// One persistent launch does every panel.  Work items are (stage s, row block
// b): stage s finishes x -= V_{s-1} y_{s-1} for the panel applied before it
// (phase A) and forms this block's share of w_s = V_s^T x for the next panel
// (phase B); stage p does phase A only.  CTAs take items in ticket order from
// a counter.  The shares are summed by a fixed two-level tree: the last item
// of each group of 16 to arrive sums its group, and the last group to arrive
// sums the group sums, forms y_s = op(T_s) w_s and publishes it with a
// release store; items of stage s+1 wait (acquire) for that.  An item waits
// only for items with smaller tickets, which CTAs already running have
// taken, so the launch makes progress whether or not all of its CTAs are
// resident at once; the waits are still bounded by %globaltimer and raise
// the context's timeout flag when they run out.  Sums are in a fixed order:
// results do not depend on which CTA ran which item.
//
// Rows stream through shared memory by TMA when the layout allows (panels up
// to 128 wide, even lda, 16-byte aligned V): per 32-row chunk one tensor box
// of each panel, a ring of stages completed by mbarriers, the next chunk's
// box issued as soon as a slot frees and an item's first boxes issued before
// its dependency wait.  On this part per-lane loads reach about 4 TB/s of
// reads, bulk tensor copies about 7.4.  Otherwise per-lane loads in 64-row
// chunks (two rows per lane).  Warp g owns the g-th eighth of each panel's
// columns; lane = row.  The stage's T is copied into shared memory column by
// column (its upper triangle only) by bulk copies when aligned, else read
// by per-lane loads.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

namespace gbqr {
namespace {

constexpr int kChunkL = 64;                    // per-lane-load path: rows per chunk (two per lane)
constexpr int kChunkT = 32;                    // TMA path: rows per chunk (one per lane), the box height
constexpr int kWarps = kThreads / 32;
constexpr int kMaxW = kApplyVecMaxW;
constexpr int kTmaMaxW = 128;                  // widest panel of the TMA path
constexpr int kTiles = kMaxW / 32;             // 32-wide blocks of T
constexpr int kGroup = 16;                     // items per group of the share tree
constexpr int kMaxGroups = 16;                 // groups per stage
constexpr int kRingBytes = 192 * 1024;         // TMA ring, and staged T, in dynamic shared memory
constexpr int kMaxStages = 4;
static_assert(kMaxW % (32 * kWarps) == 0 && kMaxW <= kThreads, "one column of w per thread");
static_assert(kWarps * kChunkL <= kTiles * kMaxW, "phase A partials fit the T-product buffer");
static_assert(kTmaMaxW * (kTmaMaxW + 2) * 8 <= kRingBytes, "staged T fits the ring");
static_assert(kTmaMaxW <= 32 * (kWarps - 1), "the warp staging T is not one of those reading the group sums");

enum { kTicket = 0, kArrive = 1, kReady = 2, kDone = 3, kAbort = 4, kGroupCtr = 5, kNumCounters = kGroupCtr + kMaxGroups };

struct ApplyVec {
    int64_t m, lda, ldt, R;    // R: rows per item (a multiple of kChunkT on the TMA path, else of kChunkL)
    int n, pb, npan, nblk;     // panel width, panels, row blocks
    int trans, tfull;          // Q^T (else Q); T is the full n x n kernel (else nb x n panel kernels)
    int tsm, stages, tstride;  // T staged by bulk copies; TMA ring depth; staged T's column stride
    const double *VR, *T;
    double *x;
    double *y;                 // 2 pb: y of the stage before, ping-pong
    double *partial;           // nblk pb: the items' shares of w
    double *gsum;              // kMaxGroups pb: the groups' sums
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
__device__ __forceinline__ uint32_t smem_u32(const void *q) { return (uint32_t)__cvta_generic_to_shared(q); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Wait for the mbarrier phase of the given parity (every thread of the CTA
// calls it).  Bounded: gives up after the launch's wait limit, and then
// raises the flags.  With stop_on_abort it also gives up as soon as another
// CTA has raised the abort flag; waits for this CTA's own copies in flight
// (before it reuses or leaves its shared memory) pass false.
__device__ bool mbar_wait(const ApplyVec &p, uint32_t a, uint32_t parity, bool stop_on_abort = true) {
    if (mbar_try(a, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (stop_on_abort && *(volatile unsigned *)(p.ctr + kAbort)) return false;
        if (global_ns() - t0 > (unsigned long long)p.wait_ns) {
            atomicExch(p.ctr + kAbort, 1u);
            atomicExch(p.timeout, 1);
            return false;
        }
    }
}

// Entry (r, c) of a unit lower trapezoidal panel whose diagonal starts at
// row top, given v = the stored value at (r, c): zero above the diagonal, one
// on it, v below it; zero where in is false (a row outside the item or a
// column the thread does not own).  The per-lane-load path loads v
// unconditionally from a clamped, always valid address, so that a chunk's
// loads are all in flight at once instead of each waiting behind its guard.
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
    double ys[kMaxW];                  // the item's share of w, then the stage's w
    double yw[kWarps * 32];            // warp g's slice of y_{s-1}, zero past its columns
    double part[kTiles * kMaxW];       // phase A partials, then T-tile partials
    double xs[kChunkL];
    alignas(8) unsigned long long full[kMaxStages];   // TMA ring slots: box bytes landed
    alignas(8) unsigned long long tbar;               // staged T landed
    unsigned tpar;                                    // parity of tbar's next phase
    int flag;
    int ticket;
};

// Phase A and B of one item over rows [r0, r1) with per-lane loads (any
// lda): x -= V_{s-1} y_{s-1} on those rows, acc[j] += V_s(:, ck0 + j)^T x.
template <int CW>
__device__ void item_rows_lsu(const ApplyVec &p, const Stage &st, Smem &sm, int64_t r0, int64_t r1, double (&acc)[CW]) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int cwp = (st.wp + kWarps - 1) / kWarps, cwk = (st.wk + kWarps - 1) / kWarps;
    const int cp0 = g * cwp, ck0 = g * cwk, ck1 = min(st.wk, ck0 + cwk);
    const double *Vp = st.wp ? p.VR + st.jp * p.lda : nullptr;
    const double *Vk = st.wk ? p.VR + st.jk * p.lda : nullptr;
    const double *ywg = sm.yw + g * 32;
    for (int64_t s0 = r0; s0 < r1; s0 += kChunkL) {
        const int64_t ra = s0 + lane, rb = ra + 32, rx = s0 + tid;
        if (s0 + kChunkL < r1) {
            // the next chunk's column segments into L2 (four 128-byte lines
            // of a column per group of four lanes, eight columns per pass)
            const int64_t rn = min(s0 + kChunkL + (lane & 3) * 16, r1 - 1);
            for (int j = lane >> 2; j < CW; j += 8) {
                if (Vk) prefetch_l2(Vk + (int64_t)min(ck0 + j, st.wk - 1) * p.lda + rn);
                if (Vp) prefetch_l2(Vp + (int64_t)min(cp0 + j, st.wp - 1) * p.lda + rn);
            }
        }
        const bool fast = s0 + kChunkL <= r1 && (!Vk || s0 >= st.jk + st.wk) && (!Vp || s0 >= st.jp + st.wp);
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
        if (tid < kChunkL && rx < r1) xv = __ldcg(p.x + rx);   // written by other CTAs' earlier items
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
            sm.part[g * kChunkL + lane] = a0;
            sm.part[g * kChunkL + lane + 32] = a1;
        }
        __syncthreads();
        if (tid < kChunkL) {
            if (Vp) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < kWarps; ++q) s += sm.part[q * kChunkL + tid];
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

// The TMA ring of one item: chunk i (32 rows from c0 + 32 i) lands in slot
// i % stages: the box of V_s (32 x pb, column-major) and after it the box of
// V_{s-1}.  Thread 0 issues; every thread waits on the slot's mbarrier.
struct Ring {
    double *base;
    int64_t c0;        // first chunk row (even: TMA's row coordinate times 8 bytes must be 16-byte aligned)
    int nch;           // chunks of the item
    int issued, used;  // chunks issued / consumed
    unsigned ph;       // parity bit per slot
};

__device__ __forceinline__ void ring_issue(const CUtensorMap *map, const ApplyVec &p, const Stage &st, Smem &sm,
                                           Ring &rg) {
    const int i = rg.issued++;
    const int slot = i % p.stages;
    double *dst = rg.base + (size_t)slot * 2 * kChunkT * p.pb;
    const uint32_t bar = smem_u32(&sm.full[slot]);
    const uint32_t bytes = (uint32_t)((st.wk ? 1 : 0) + (st.wp ? 1 : 0)) * kChunkT * p.pb * 8;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads of the slot came before
    mbar_expect_tx(bar, bytes);
    const int x = (int)(rg.c0 + (int64_t)kChunkT * i);
    if (st.wk) tma_load_2d(smem_u32(dst), map, x, (int)st.jk, bar);
    if (st.wp) tma_load_2d(smem_u32(dst + kChunkT * p.pb), map, x, (int)st.jp, bar);
}

// Every thread: wait for the chunks issued but not consumed (bounded), so
// that no copy into shared memory is in flight when the CTA leaves.
__device__ void ring_drain(const ApplyVec &p, Smem &sm, Ring &rg) {
    while (rg.used < rg.issued) {
        const int slot = rg.used % p.stages;
        mbar_wait(p, smem_u32(&sm.full[slot]), (rg.ph >> slot) & 1u, false);
        rg.ph ^= 1u << slot;
        ++rg.used;
    }
}

// Phase A and B of one item over rows [r0, r1) from the TMA ring (chunk 0
// .. stages-1 already issued).  False if a wait ran out (the caller drains).
template <int CW>
__device__ bool item_rows_tma(const CUtensorMap *map, const ApplyVec &p, const Stage &st, Smem &sm, Ring &rg,
                              int64_t r0, int64_t r1, double (&acc)[CW]) {
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    const int cwp = (st.wp + kWarps - 1) / kWarps, cwk = (st.wk + kWarps - 1) / kWarps;
    const int cp0 = g * cwp, ck0 = g * cwk, ck1 = min(st.wk, ck0 + cwk);
    const double *ywg = sm.yw + g * 32;
    for (int i = 0; i < rg.nch; ++i) {
        const int64_t s0 = rg.c0 + (int64_t)kChunkT * i, r = s0 + lane;
        const bool in = r >= r0 && r < r1;
        double xv = 0.0;
        if (g == 0 && in) xv = __ldcg(p.x + r);          // written by other CTAs' earlier items
        const int slot = rg.used % p.stages;
        const bool ok = mbar_wait(p, smem_u32(&sm.full[slot]), (rg.ph >> slot) & 1u);
        rg.ph ^= 1u << slot;
        ++rg.used;
        const double *Vc = rg.base + (size_t)slot * 2 * kChunkT * p.pb;   // V_s box: column c at Vc + 32 c
        const double *Vq = Vc + kChunkT * p.pb;                           // V_{s-1} box
        const bool fast = s0 >= r0 && s0 + kChunkT <= r1 && (!st.wk || s0 >= st.jk + st.wk) &&
                          (!st.wp || s0 >= st.jp + st.wp);
        if (st.wp) {
            double a = 0.0;
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const int c = cp0 + j;
                const double v = Vq[min(c, p.pb - 1) * kChunkT + lane];   // zero weight past the warp's columns
                a = fma(fast ? v : vsel(v, r - st.jp, c, in), ywg[j], a);
            }
            sm.part[g * 32 + lane] = a;
        }
        if (__syncthreads_or(!ok)) {                     // a wait ran out: the whole CTA stops,
            rg.ph ^= 1u << slot;                         // and this chunk counts as still in
            --rg.used;                                   // flight for the caller's drain
            return false;
        }
        // the slot of chunk i - 1 is free: every warp finished it before this
        // barrier (all threads count the issue, thread 0 makes it)
        if (i >= 1 && rg.issued < rg.nch) {
            if (tid == 0) ring_issue(map, p, st, sm, rg);
            else ++rg.issued;
        }
        if (g == 0) {
            if (st.wp) {
                double sum = 0.0;
#pragma unroll
                for (int q = 0; q < kWarps; ++q) sum += sm.part[q * 32 + lane];
                xv -= sum;
                if (in) __stcg(p.x + r, xv);
            }
            sm.xs[lane] = xv;
        }
        __syncthreads();
        if (st.wk) {
            const double xr = sm.xs[lane];
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const int c = ck0 + j;
                const double v = Vc[min(c, p.pb - 1) * kChunkT + lane];
                acc[j] = fma(fast ? v : vsel(v, r - st.jk, c, in && c < ck1), xr, acc[j]);
            }
        }
    }
    return true;
}

// y_s = op(T_s) w (w in sm.ys), T_s upper triangular (wk x wk), element
// (r, c) at Tsrc[r + c ld] (shared memory when staged, else global).  FP64
// instructions are the cost here (a warp's FMA occupies the SM's FP64 pipe
// for tens of cycles), so the wk (wk + 1) / 2 products are spread evenly:
// outputs i and wk - 1 - i form a pair with wk + 1 terms together, and each
// pair's terms are split into P parts, one per thread; then each output
// sums its P part sums in order.  T^T w puts a pair's parts on adjacent
// lanes (they read along a column of T), T w puts adjacent pairs there
// (they read along a row).
template <bool SMEM>
__device__ void t_product(const ApplyVec &p, const Stage &st, Smem &sm, const double *Tsrc, int64_t ld, double *y) {
    const int tid = threadIdx.x, wk = st.wk;
    const int np = (wk + 1) / 2;                           // pairs; the middle output alone if wk is odd
    const int P = min(kTiles, kThreads / np);              // parts per pair
    const int pair = p.trans ? tid / P : tid % np, h = p.trans ? tid % P : tid / np;
    if (pair < np && h < P) {
        const int i = pair, i2 = wk - 1 - pair;
        // terms of output o: T w: l = o .. wk - 1 (T(o, l));  T^T w: l = 0 .. o (T(l, o))
        const int nA = p.trans ? i + 1 : wk - i;
        const int total = (i == i2) ? nA : wk + 1;
        const int L = (wk + 1 + P - 1) / P;
        double aA = 0.0, aB = 0.0;
        for (int v = h * L; v < min(total, (h + 1) * L); ++v) {
            const bool sideA = v < nA;
            const int o = sideA ? i : i2, u = sideA ? v : v - nA;
            const int l = p.trans ? u : o + u;
            const int64_t idx = p.trans ? (int64_t)l + (int64_t)o * ld : (int64_t)o + (int64_t)l * ld;
            const double t = SMEM ? Tsrc[idx] : __ldg(Tsrc + idx);
            const double r = fma(t, sm.ys[l], sideA ? aA : aB);
            if (sideA) aA = r; else aB = r;
        }
        sm.part[h * kMaxW + i] = aA;
        if (i2 != i) sm.part[h * kMaxW + i2] = aB;
    }
    __syncthreads();
    if (tid < wk) {
        double a = sm.part[tid];
        for (int q = 1; q < P; ++q) a += sm.part[q * kMaxW + tid];
        __stcg(y + tid, a);
    }
}

// Copy T_s's upper triangle into shared memory: column c (rows 0..c) at
// Ts + c tstride, one bulk copy per column of its 16-byte pairs, the odd last
// entry of a column by a plain load.  One warp issues; completes on sm.tbar.
__device__ void t_stage_issue(const ApplyVec &p, const Stage &st, Smem &sm, double *Ts) {
    const int lane = threadIdx.x & 31, wk = st.wk;
    const double *Tk = panel_T(p, st.jk);
    const uint32_t bar = smem_u32(&sm.tbar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic reads of the ring came before
    // sum over columns of floor((c + 1) / 2) pairs = floor(wk^2 / 4)
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(wk * wk / 4) * 16);
    __syncwarp();
    for (int c = lane; c < wk; c += 32) {
        const uint32_t pairs = (uint32_t)(c + 1) / 2;
        if (pairs) bulk_g2s(smem_u32(Ts + (size_t)c * p.tstride), Tk + (int64_t)c * p.ldt, pairs * 16, bar);
        if ((c + 1) & 1) Ts[(size_t)c * p.tstride + c] = __ldg(Tk + (int64_t)c * p.ldt + c);
    }
}

// After an item of stage s (its share of w in sm.ys): store the share and
// arrive at its group; the group's last arriver sums the group's shares and
// arrives at the stage; the stage's last arriver forms w and y_s and
// releases stage s + 1.  Ts: shared memory for the staged T (TMA path).
__device__ void arrive_item(const ApplyVec &p, const Stage &st, Smem &sm, int s, int b, double *Ts) {
    const int tid = threadIdx.x, wk = st.wk;
    const int item = b - st.b0, G = item / kGroup, cnt = min(kGroup, st.S - G * kGroup);
    const int ng = (st.S + kGroup - 1) / kGroup;
    if (tid < wk) __stcg(p.partial + (int64_t)item * wk + tid, sm.ys[tid]);
    __syncthreads();
    if (tid == 0) {
        const bool last = atom_add_acq_rel(p.ctr + kGroupCtr + G, 1u) == (unsigned)(cnt - 1);
        if (last) p.ctr[kGroupCtr + G] = 0u;             // ordered before the release of y_s
        sm.flag = last ? 1 : 0;
    }
    __syncthreads();
    if (!sm.flag) return;
    if (tid < wk) {
        const double *src = p.partial + (int64_t)G * kGroup * wk + tid;
        double v[kGroup];
#pragma unroll
        for (int q = 0; q < kGroup; ++q) v[q] = __ldcg(src + (int64_t)min(q, cnt - 1) * wk);
        double a = v[0];
#pragma unroll
        for (int q = 1; q < kGroup; ++q)
            if (q < cnt) a += v[q];
        __stcg(p.gsum + (int64_t)G * wk + tid, a);
    }
    __syncthreads();
    if (tid == 0) {
        const bool last = atom_add_acq_rel(p.ctr + kArrive, 1u) == (unsigned)(ng - 1);
        if (last) p.ctr[kArrive] = 0u;
        sm.flag = last ? 1 : 0;
    }
    __syncthreads();
    if (!sm.flag) return;
    // the stage's last arriver: T on its way (the last warp issues) while
    // warps 0-3 read the group sums
    const bool staged = p.tsm && Ts;
    if (staged && (tid >> 5) == kWarps - 1) t_stage_issue(p, st, sm, Ts);
    if (tid < wk) {
        const double *src = p.gsum + tid;
        double v[kMaxGroups];
#pragma unroll
        for (int q = 0; q < kMaxGroups; ++q) v[q] = __ldcg(src + (int64_t)min(q, ng - 1) * wk);
        double a = v[0];
#pragma unroll
        for (int q = 1; q < kMaxGroups; ++q)
            if (q < ng) a += v[q];
        sm.ys[tid] = a;
    }
    double *y = p.y + (s & 1) * p.pb;
    if (staged) {
        const bool ok = __syncthreads_and(mbar_wait(p, smem_u32(&sm.tbar), sm.tpar, false));
        if (ok) t_product<true>(p, st, sm, Ts, p.tstride, y);   // else the launch is aborting
        __syncthreads();
        if (tid == 0) sm.tpar ^= 1u;
    } else {
        __syncthreads();
        t_product<false>(p, st, sm, panel_T(p, st.jk), p.ldt, y);
    }
    __syncthreads();
    if (tid == 0) st_release(p.ctr + kReady, s + 1);   // publishes y_s and the reset counters
}

template <int CW, bool TMA>
__global__ void __launch_bounds__(kThreads, 1) apply_vec_kernel(const __grid_constant__ CUtensorMap map, ApplyVec p) {
    __shared__ Smem sm;
    extern __shared__ __align__(128) unsigned char dyn[];           // TMA ring, or the share buffer alone
    double *ring = TMA ? reinterpret_cast<double *>(dyn) : nullptr;
    const int tid = threadIdx.x, lane = tid & 31, g = tid >> 5;
    if (TMA && tid == 0) {
        for (int i = 0; i < kMaxStages; ++i) mbar_init(smem_u32(&sm.full[i]), 1);
        mbar_init(smem_u32(&sm.tbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.tpar = 0u;
    }
    Ring rg;
    rg.base = ring; rg.c0 = 0; rg.nch = 0; rg.issued = rg.used = 0; rg.ph = 0u;
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
        const int64_t r0 = max((int64_t)b * p.R, st.lo), r1 = min((int64_t)(b + 1) * p.R, p.m);
        if (TMA) {
            // V does not depend on earlier stages: its first boxes go out before the wait
            rg.c0 = r0 & ~(int64_t)1;
            rg.nch = (int)((r1 - rg.c0 + kChunkT - 1) / kChunkT);
            rg.issued = rg.used = 0;
            if (tid == 0)
                for (int i = 0; i < min(rg.nch, p.stages); ++i) ring_issue(&map, p, st, sm, rg);
            else
                rg.issued = min(rg.nch, p.stages);
        }
        // this stage's T into L2 for whichever item arrives last: item i
        // takes columns i, i + S, ... (one 128-byte line per lane)
        if (st.wk && g == kWarps - 1)
            for (int c = b - st.b0; c < st.wk; c += st.S)
                if (lane * 16 < st.wk) prefetch_l2(panel_T(p, st.jk) + (int64_t)c * p.ldt + lane * 16);
        if (tid == 0) sm.flag = wait_ready(p, s) ? 1 : 0;
        __syncthreads();
        if (!sm.flag) {
            if (TMA) ring_drain(p, sm, rg);
            break;
        }
        // y_{s-1}, split into the warps' column slices
        const int cwp = (st.wp + kWarps - 1) / kWarps;
        for (int i = tid; i < kWarps * 32; i += kThreads) {
            const int gg = i / 32, jj = i % 32, c = gg * cwp + jj;
            sm.yw[i] = (jj < cwp && c < st.wp) ? __ldcg(p.y + ((s - 1) & 1) * p.pb + c) : 0.0;
        }
        __syncthreads();
        double acc[CW];
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[j] = 0.0;
        if constexpr (TMA) {
            if (!item_rows_tma<CW>(&map, p, st, sm, rg, r0, r1, acc)) {
                ring_drain(p, sm, rg);
                break;
            }
        } else {
            item_rows_lsu<CW>(p, st, sm, r0, r1, acc);
        }
        if (st.wk == 0) continue;                        // the last stage: phase A only
        // this item's share of w: the lanes' accumulators through shared
        // memory (lane-major rows of odd length), then per column a sum over
        // the lanes in two halves - a fraction of the FP64 additions of a
        // shuffle tree per column
        {
            double *red = reinterpret_cast<double *>(dyn);
            constexpr int RL = kWarps * CW + 1;
            __syncthreads();                             // the buffer overlays the ring slot the last chunk read
#pragma unroll
            for (int j = 0; j < CW; ++j) red[lane * RL + g * CW + j] = acc[j];
            __syncthreads();
            const int cwk = (st.wk + kWarps - 1) / kWarps;
            const int half = (st.wk <= kThreads / 2) ? kThreads / 2 : kThreads;
            const int c = tid % half, hh = tid / half, lanes = 32 * half / kThreads;
            if (c < st.wk) {
                const int pos = (c / cwk) * CW + c % cwk;
                const double *col = red + hh * lanes * RL + pos;
                double a = col[0];
                for (int l = 1; l < lanes; ++l) a += col[l * RL];
                sm.part[hh * kMaxW + c] = a;
            }
            __syncthreads();
            if (tid < st.wk) sm.ys[tid] = (half < kThreads) ? sm.part[tid] + sm.part[kMaxW + tid] : sm.part[tid];
            // the buffer is part of the TMA ring: order these generic writes before later bulk copies into it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        arrive_item(p, st, sm, s, b, ring);
    }
    // the last CTA out resets the counters for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(p.ctr + kDone, 1u) == gridDim.x - 1) {
            for (int i = 0; i < kNumCounters; ++i)
                if (i != kDone) p.ctr[i] = 0u;
            __threadfence();
            p.ctr[kDone] = 0u;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(tensor_map_encoder());
}

}  // namespace

gbqr_status apply_vec(const Exec &ex, bool trans, int64_t m, int64_t n, const double *VR, int64_t lda,
                      const double *T, int64_t ldt, bool tfull, int64_t pb, double *x, double *y2, size_t ny,
                      double *partial, size_t partial_elems, unsigned *counters, size_t ncounters, int *timeout) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    if (pb < 1 || pb > kMaxW || n > m || !timeout) return GBQR_EINVAL;
    const int64_t npan = (n + pb - 1) / pb;
    if (npan > 0x3fffffff) return GBQR_EUNSUPPORTED;
    // rows per item: whole chunks, about one item per SM for the longest
    // stage, at most kGroup * kMaxGroups items
    const int64_t per = (m + std::min(ex.num_sms, kGroup * kMaxGroups) - 1) / std::min(ex.num_sms, kGroup * kMaxGroups);
    const bool tma_shape = pb <= kTmaMaxW && lda % 2 == 0 && ((uintptr_t)VR % 16) == 0;
    const int64_t gran = tma_shape ? kChunkT : kChunkL;
    const int64_t R = (per + gran - 1) / gran * gran;
    const int64_t nblk = (m + R - 1) / R;
    if ((size_t)(2 * pb) > ny || (size_t)((nblk + kMaxGroups) * pb) > partial_elems || ncounters < kNumCounters)
        return GBQR_ENOMEM;
    ApplyVec p;
    p.m = m; p.lda = lda; p.ldt = ldt; p.R = R;
    p.n = (int)n; p.pb = (int)pb; p.npan = (int)npan; p.nblk = (int)nblk;
    p.trans = trans ? 1 : 0; p.tfull = tfull ? 1 : 0;
    p.VR = VR; p.T = T; p.x = x; p.y = y2; p.partial = partial; p.gsum = partial + nblk * pb;
    p.ctr = counters; p.timeout = timeout;
    p.wait_ns = 5000000000ll;   // 5 s: far beyond any stage's critical path
    // the TMA path: a 2-D tensor map over VR (rows x columns, box 32 x pb)
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    bool tma = tma_shape && m < 0x7fffffff && n < 0x7fffffff && encoder() != nullptr;
    if (tma) {
        cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
        cuuint64_t strides[1] = {(cuuint64_t)lda * 8};
        cuuint32_t box[2] = {(cuuint32_t)kChunkT, (cuuint32_t)pb};
        cuuint32_t estr[2] = {1, 1};
        tma = encoder()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(VR), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    p.stages = tma ? (int)std::min<int64_t>(kMaxStages, kRingBytes / (2 * kChunkT * pb * 8)) : 0;
    p.tstride = (int)((pb + 1) / 2 * 2);
    p.tsm = tma && ldt % 2 == 0 && ((uintptr_t)T % 16) == 0 && (!tfull || pb % 2 == 0) ? 1 : 0;
    const unsigned grid = (unsigned)std::min<int64_t>(nblk, ex.num_sms);
    // dynamic shared memory: the TMA ring, which also holds the lanes'
    // accumulators at the end of an item (32 rows of 8 CW + 1 doubles)
    const bool wide = pb > 16 * kWarps;
    const size_t red_bytes = (size_t)32 * (kWarps * (wide ? 32 : 16) + 1) * 8;
    const size_t dyn = tma ? (size_t)kRingBytes : red_bytes;
    {
        static std::atomic<bool> attr_done[64];
        if (!(ex.device >= 0 && ex.device < 64) || !attr_done[ex.device].load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(apply_vec_kernel<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kRingBytes) != cudaSuccess ||
                cudaFuncSetAttribute(apply_vec_kernel<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)32 * (kWarps * 16 + 1) * 8)) != cudaSuccess ||
                cudaFuncSetAttribute(apply_vec_kernel<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((size_t)32 * (kWarps * 32 + 1) * 8)) != cudaSuccess)
                return GBQR_ECUDA;
            if (ex.device >= 0 && ex.device < 64) attr_done[ex.device].store(true, std::memory_order_release);
        }
    }
    // algorithmic traffic: each panel's V read twice (phases A and B), x in and out per stage
    double bytes = 0.0, flops = 0.0;
    for (int64_t k = 0; k < npan; ++k) {
        const int64_t j = k * pb, w = std::min<int64_t>(pb, n - j);
        bytes += 2.0 * 8.0 * (double)(m - j) * w + 8.0 * (double)w * w / 2 + 16.0 * (double)(m - j);
        flops += 4.0 * (double)(m - j) * w + (double)w * w;
    }
    trace_begin(ex, FAM_GEMV);
    if (tma)
        apply_vec_kernel<16, true><<<grid, kThreads, dyn, ex.stream>>>(map, p);
    else if (!wide)
        apply_vec_kernel<16, false><<<grid, kThreads, dyn, ex.stream>>>(map, p);
    else
        apply_vec_kernel<32, false><<<grid, kThreads, dyn, ex.stream>>>(map, p);
    return trace_end(ex, FAM_GEMV, flops, bytes);
}

}  // namespace gbqr
