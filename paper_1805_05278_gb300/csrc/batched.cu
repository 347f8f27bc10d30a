// Persistent batched QR: thousands of independent, uneven QR factorizations
// in ONE kernel launch (the 1D-CAQR-EG instance of Section 6 for each
// matrix: a right-looking top level over panels of width b, Section 8.4,
// each panel factored by TSQR, Section 5 / Appendix C).
//
// Work decomposition.  Matrix i (m_i x n_i) is cut into column blocks of
// width b.  Its tasks are
//   panel(i, k)            the QR of block k's rows k*b .. m_i-1 (once the
//                          k earlier panels have been applied to it): V_k,
//                          T_k and R_k in place, T_k into the caller's T;
//   update(i, k, c0..c1)   C <- (I - V_k T_k V_k^T)^T C for the column blocks
//                          c0 .. c1-1 (the basis-kernel update of Section
//                          2.3: W = V^T C, W = T^T W, C -= V W).
// A per-(matrix, block) counter records how many panels have been applied to
// the block (+1 once the block itself is factored); a task's dependencies
// are conditions on those counters.  The host orders all tasks by a list
// schedule of estimated durations (critical path first), which is a
// topological order; the CTAs of the persistent grid take tasks in that
// order from an atomic dispenser and wait for the task's counters before
// running it.  Every dependency of a task comes earlier in the order and is
// held by a CTA that is already running, so the waits always end; each is
// nevertheless bounded by %globaltimer, and a wait that runs out raises an
// abort flag that every CTA checks (the host then reports GBQR_ETIMEOUT).
//
// A panel task is TSQR with a flat tree inside one CTA (the reduction tree
// of Appendix C.1 with fan-out P, reduced sequentially): row block 0 is
// factored as a leaf, then each further block is stacked under the running
// R and the structured [R; A_q] is factored (V = [I; Y_q]).  The Householder
// vectors are then reconstructed (Appendix C.2): the top w x w block X of
// W = Q [I; 0] comes from the chain B_P = I, B_q = (I - T_q) B_{q+1} and
// leaf 0's Q-factor; X + S = L U with S_jj = sgn(X^_jj); T = U S L^{-T},
// R = -S R_tree, V_top = L.  The rows below follow the shortcut noted at the
// end of Appendix C, starting the chain from B = U^{-1}: V_q = -Y_q T_q B_{q+1}.
// So V, T and R equal those of unblocked Householder QR up to rounding.
#include "tsqr_dev.cuh"

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

namespace gbqr {
namespace {

constexpr int kUpdCols = 64;    // columns of an update task (the look-ahead block excepted)

constexpr size_t kSmemBudget = 110 * 1024;   // two CTAs per SM

template <class Real>
struct BMat {
    Real *A;        // m x n, column-major, lda
    Real *T;        // b x n panel kernels, ldt
    int64_t lda, ldt;
    int m, n;
    int state0;     // its first column-block counter
    int pad;
};

template <class Real>
struct BParams {
    const BMat<Real> *mats;
    const int4 *tasks;      // (matrix, k, c0, c1): a panel task when c0 == c1 (== k)
    int ntasks;
    int b, hblk, ldS, hup;    // panel width, panel row-block height, its shared ld, update chunk rows
    int *state;             // per (matrix, column block): panels applied, +1 once factored
    unsigned *next;         // task dispenser
    int *abort;             // raised by a wait that ran out; every CTA then stops
    int *timeout;           // the context's device-side timeout record
    unsigned long long *nonfinite;
    Real *tscr;             // per CTA: T of each row block of the panel being factored
    size_t tscr_stride;     // elements per CTA
    int tscr_blocks;
    long long wait_ns;
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool non_finite(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff;
}
__device__ __forceinline__ bool non_finite(float x) { return ((__float_as_int(x) >> 23) & 0xff) == 0xff; }

template <class Real>
__device__ int scan_block(const Real *S, int ldS, int h, int w) {
    int bad = 0;
    for (int idx = threadIdx.x; idx < h * w; idx += blockDim.x) {
        const int r = idx % h, c = idx / h;
        bad |= non_finite(S[r + (size_t)c * ldS]) ? 1 : 0;
    }
    return bad;
}

// Thread 0: wait until the task's column-block counters allow it to run.
// Returns false (after raising the abort flag on a timeout) when it must not.
template <class Real>
__device__ bool wait_deps(const BParams<Real> &p, const int *st, int k, int c0, int c1) {
    auto ready = [&]() {
        if (c0 == c1) return ld_acquire(st + k) >= k;              // panel k: k panels applied to block k
        if (ld_acquire(st + k) < k + 1) return false;              // update: panel k factored ...
        for (int c = c0; c < c1; ++c)
            if (ld_acquire(st + c) < k) return false;              // ... and panels 0..k-1 applied to c
        return true;
    };
    const unsigned long long t0 = global_ns();
    unsigned ns = 64;
    while (!ready()) {
        if (*(volatile int *)p.abort) return false;
        if (global_ns() - t0 > (unsigned long long)p.wait_ns) {
            atomicExch(p.abort, 1);
            atomicExch(p.timeout, 1);
            return false;
        }
        __nanosleep(ns);
        if (ns < 2048) ns *= 2;
    }
    return true;
}

// Asynchronous global -> shared copies (cp.async, one element each: the
// column segments of a chunk need not be 16-byte aligned).  The waits on a
// task's counters end with an acquire at GPU scope, which orders these
// copies after the writes that other CTAs released.
template <class Real>
__device__ __forceinline__ void cp_async(Real *dst_smem, const Real *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    if constexpr (sizeof(Real) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// dst(r, c) = src(r, c) for an h x w block, the whole CTA, asynchronously.
template <class Real>
__device__ __forceinline__ void async_block(Real *dst, int ldd, const Real *src, int64_t lds, int h, int w) {
    for (int idx = threadIdx.x; idx < h * w; idx += blockDim.x) {
        const int c = idx / h, r = idx - c * h;
        cp_async(dst + r + c * ldd, src + r + (int64_t)c * lds);
    }
}

// M <- T (V1^T B) for w <= kMaxBatchB (the leaf_z of the TSQR downsweep with
// fewer registers): V1 unit lower (column-major, ld w, strict lower part
// read), T upper in M on entry, B upper; C is w x w scratch.
template <class Real>
__device__ void leaf_z_small(const Real *V1, const Real *B, Real *C, Real *M, int w) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < w * w; idx += nthr) {          // C = V1^T B (upper)
        const int i = idx % w, c = idx / w;
        Real s = Real(0);
        if (i <= c) {
            s = B[i + c * w];
            for (int l = i + 1; l <= c; ++l) s = rfma(V1[l + i * w], B[l + c * w], s);
        }
        C[idx] = s;
    }
    __syncthreads();
    constexpr int kPer = (kMaxBatchB * kMaxBatchB + kThreads - 1) / kThreads;
    Real z[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {                         // Z = T C, then over M
        const int idx = tid + q * nthr;
        if (idx < w * w) {
            const int i = idx % w, c = idx / w;
            Real s = Real(0);
            for (int l = i; l <= c; ++l) s = rfma(M[i + l * w], C[l + c * w], s);
            z[q] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int idx = tid + q * nthr;
        if (idx < w * w) M[idx] = z[q];
    }
    __syncthreads();
}

// V rows of one row block: out(r, c) = -sum_{i <= c} Y(r, i) Z(i, c) for
// rows r0 .. r0 + h - 1 of S (ld ldS) and Z upper w x w (ld w), written to
// the panel at out (ld lda).  Each thread takes whole rows with Y(r, :) in
// registers, so the w column sums are independent chains.
template <int MaxB, class Real>
__device__ __forceinline__ void v_rows(const Real *S, int ldS, int r0, int h, const Real *Z, int w, Real *out,
                                       int64_t lda) {
    for (int r = r0 + (int)threadIdx.x; r < r0 + h; r += blockDim.x) {
        Real y[MaxB];
#pragma unroll
        for (int i = 0; i < MaxB; ++i) y[i] = (i < w) ? S[r + (size_t)i * ldS] : Real(0);
#pragma unroll
        for (int c = 0; c < MaxB; ++c) {
            if (c < w) {
                Real s = Real(0);
#pragma unroll
                for (int i = 0; i <= c; ++i) s = rfma(y[i], Z[i + c * w], s);
                out[r + (int64_t)c * lda] = -s;
            }
        }
    }
}

// Panel task (flat-tree TSQR in one CTA, then the Householder
// reconstruction); returns non-zero if the panel held a NaN or Inf.
// Shared memory: S (ldS x b), then Tt, G, Mx, Bm, Cm, X, Li, Ui (b x b each,
// used with leading dimension w), then 8 b reflector scalars and signs.
template <int MaxB, class Real>
__device__ int panel_task(const BParams<Real> &p, const BMat<Real> &M, int k, Real *sm, Real *tscr) {
    const int b = p.b, tid = threadIdx.x, nthr = blockDim.x;
    const int j0 = k * b;
    const int w = min(b, M.n - j0);
    const int mr = M.m - j0;
    const int64_t lda = M.lda;
    Real *A = M.A + j0 + (int64_t)j0 * lda;
    const int ldS = p.ldS, bb = b * b, ww = w * w;
    Real *S = sm;
    Real *Tt = S + (size_t)ldS * b;
    Real *G = Tt + bb, *Mx = G + bb, *Bm = Mx + bb, *Cm = Bm + bb, *X = Cm + bb, *Li = X + bb, *Ui = Li + bb;
    Real *aux = Ui + bb;
    const Refl<Real> rf{aux, aux + w, aux + 2 * w, aux + 3 * w, aux + 4 * w, aux + 7 * b};
    Real *Sg = aux + 5 * b, *rU = Sg + b;
    const int P = (mr + p.hblk - 1) / p.hblk;
    auto rb = [&](int q) { return (int)((int64_t)q * mr / P); };
    int bad = 0;
    if (P > p.tscr_blocks) return 1;   // cannot happen: the host sizes tscr for the tallest panel

    // ---- upsweep: block 0 as a leaf, then each block stacked under R
    const int h0 = rb(1);
    async_block(S, ldS, A, lda, h0, w);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    bad |= scan_block(S, ldS, h0, w);
    householder_block(S, ldS, w, LeafRows{h0}, rf, G);
    finish_block(S, ldS, w, rf, G);
    // leaf 0's normalised V into its rows of the panel (read again below)
    for (int idx = tid; idx < h0 * w; idx += nthr) {
        const int r = idx % h0, c = idx / h0;
        if (r > c) A[r + (int64_t)c * lda] = S[r + (size_t)c * ldS] * rf.sc[c];
    }
    build_t(Tt, G, rf.tau, Mx, w);
    for (int idx = tid; idx < ww; idx += nthr) tscr[idx] = Tt[idx];
    for (int idx = tid; idx < ww; idx += nthr) {          // R_0: clear the strict lower part
        const int i = idx % w, c = idx / w;
        if (i > c) S[i + (size_t)c * ldS] = Real(0);
    }
    __syncthreads();
    for (int q = 1; q < P; ++q) {
        const int r0 = rb(q), hq = rb(q + 1) - r0;
        async_block(S + w, ldS, A + r0, lda, hq, w);
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        bad |= scan_block(S + w, ldS, hq, w);
        householder_block(S, ldS, w, StackRows{w, hq}, rf, G);
        finish_block(S, ldS, w, rf, G);
        for (int idx = tid; idx < hq * w; idx += nthr) {   // Y_q (normalised) over the block's rows
            const int r = idx % hq, c = idx / hq;
            A[r0 + r + (int64_t)c * lda] = S[w + r + (size_t)c * ldS] * rf.sc[c];
        }
        build_t(Tt, G, rf.tau, Mx, w);
        for (int idx = tid; idx < ww; idx += nthr) tscr[(size_t)q * bb + idx] = Tt[idx];
        __syncthreads();
    }
    // R_tree is S's top w x w upper triangle

    // ---- top block X of W = Q [I; 0]: B_P = I, B_q = B_{q+1} - T_q B_{q+1}
    for (int idx = tid; idx < ww; idx += nthr) Bm[idx] = (idx % w == idx / w) ? Real(1) : Real(0);
    __syncthreads();
    for (int q = P - 1; q >= 1; --q) {
        for (int idx = tid; idx < ww; idx += nthr) Mx[idx] = tscr[(size_t)q * bb + idx];
        __syncthreads();
        upper_upper(Mx, Bm, Cm, w, Real(1));
        __syncthreads();
        for (int idx = tid; idx < ww; idx += nthr) Bm[idx] -= Cm[idx];
        __syncthreads();
    }
    // X = B_1 - V0top Z0, Z0 = T_0 (V0top^T B_1)
    for (int idx = tid; idx < ww; idx += nthr) {
        const int i = idx % w, c = idx / w;
        Li[idx] = (i > c) ? __ldcg(A + i + (int64_t)c * lda) : Real(0);
        Mx[idx] = tscr[idx];
    }
    __syncthreads();
    leaf_z_small(Li, Bm, Cm, Mx, w);
    for (int idx = tid; idx < ww; idx += nthr) {
        const int r = idx % w, c = idx / w;
        Real s = (r <= c) ? Mx[r + c * w] : Real(0);
        for (int i = 0; i < min(r, c + 1); ++i) s = rfma(Li[i * w + r], Mx[i + c * w], s);
        X[idx] = Bm[idx] - s;
    }
    __syncthreads();
    // X + S = L U, S_jj = sgn(X^_jj) added to the pivot before column j is
    // eliminated; the multipliers go to Cm
    for (int j = 0; j < w; ++j) {
        if (tid == 0) {
            const Real sg = X[j + j * w] < Real(0) ? -Real(1) : Real(1);
            Sg[j] = sg;
            const Real piv = X[j + j * w] + sg;
            X[j + j * w] = piv;
            rU[j] = real_rcp(piv);
        }
        __syncthreads();
        const Real rp = rU[j];
        const int rem = w - j - 1;
        for (int idx = tid; idx < rem * (rem + 1); idx += nthr) {
            const int i = j + 1 + idx % rem, c = j + idx / rem;
            const Real l = X[i + j * w] * rp;
            if (c == j) Cm[i + j * w] = l;
            else X[i + c * w] = rfma(-l, X[j + c * w], X[i + c * w]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < ww; idx += nthr) {
        const int i = idx % w, c = idx / w;
        if (i > c) X[idx] = Cm[idx];
    }
    __syncthreads();
    build_t(Ui, X, rU, Cm, w);                 // U^{-1}: strict upper of X, diagonal 1 / rU
    unit_lower_inverse(X, Li, Cm, w);          // L^{-1}
    {
        // T = U S L^{-T}; a last panel narrower than b gets zeros in rows
        // w .. nb-1 of its block (nb = min(b, n) rows: the panel layout)
        Real *Tout = M.T + (int64_t)j0 * M.ldt;
        const int nbr = min(b, M.n);
        for (int idx = tid; idx < nbr * w; idx += nthr) {
            const int i = idx % nbr, c = idx / nbr;
            Real t = Real(0);
            if (i < w)
                for (int l = i; l <= c; ++l) t = rfma(X[i + l * w] * Sg[l], (l == c) ? Real(1) : Li[c + l * w], t);
            Tout[i + (int64_t)c * M.ldt] = t;
        }
    }
    // keep R_tree (S is reused below) and start the chain from U^{-1}
    for (int idx = tid; idx < ww; idx += nthr) {
        const int i = idx % w, c = idx / w;
        Bm[idx] = Ui[idx];
        Ui[idx] = (i <= c) ? S[i + (size_t)c * ldS] : Real(0);
    }
    __syncthreads();

    // ---- V rows: V_q = -Y_q Z_q, Z_q = T_q B_{q+1}, B_q = B_{q+1} - Z_q
    for (int q = P - 1; q >= 1; --q) {
        const int r0 = rb(q), hq = rb(q + 1) - r0;
        for (int idx = tid; idx < ww; idx += nthr) Mx[idx] = tscr[(size_t)q * bb + idx];
        async_block(S, ldS, A + r0, lda, hq, w);
        cp_commit();
        upper_upper(Mx, Bm, Cm, w, Real(1));
        cp_wait<0>();
        __syncthreads();
        v_rows<MaxB>(S, ldS, 0, hq, Cm, w, A + r0, lda);
        for (int idx = tid; idx < ww; idx += nthr) Bm[idx] -= Cm[idx];
        __syncthreads();
    }
    // block 0 below its top w rows: -V_0(r, :) Z0, Z0 = T_0 (V0top^T B_1)
    for (int idx = tid; idx < ww; idx += nthr) {
        const int i = idx % w, c = idx / w;
        Li[idx] = (i > c) ? __ldcg(A + i + (int64_t)c * lda) : Real(0);
        Mx[idx] = tscr[idx];
    }
    async_block(S, ldS, A, lda, h0, w);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    leaf_z_small(Li, Bm, Cm, Mx, w);
    v_rows<MaxB>(S, ldS, w, h0 - w, Mx, w, A, lda);
    // top rows: L strictly below the diagonal, R = -S R_tree on and above
    for (int idx = tid; idx < ww; idx += nthr) {
        const int i = idx % w, c = idx / w;
        A[i + (int64_t)c * lda] = (i <= c) ? -Sg[i] * Ui[idx] : X[idx];
    }
    return bad;
}

// Update task: C <- (I - V T V^T)^T C for columns [c0 b, min(c1 b, n)) and
// rows k b .. m-1, V = panel k's reflectors (unit lower; R above them is
// masked), T = its kernel.  Two passes over the rows in chunks of H rows,
// each chunk copied asynchronously into one of two stages while the other
// stage is computed on: W = V^T C (each thread accumulates its W entries
// over every row), then W = T^T W, then C -= V W.  In FP64 the FMAs bound
// the task; in FP32 (64x the FMA rate) shared-memory reads would, so there
// each thread of pass 1 accumulates a 2 x (kMaxOut/2) block of W (one
// shared load per FMA instead of two), and in pass 2 each thread keeps its
// row of V in registers and reads W by broadcast.
template <int MaxB, class Real>
__device__ void update_task(const BParams<Real> &p, const BMat<Real> &M, int k, int c0, int c1, Real *sm) {
    constexpr int kMaxOut = (MaxB * kUpdCols + kThreads - 1) / kThreads;   // W entries per thread
    const int b = p.b, tid = threadIdx.x, nthr = blockDim.x;
    const int j0 = k * b, w = min(b, M.n - j0), mr = M.m - j0;
    const int col0 = c0 * b, cw = min(c1 * b, M.n) - col0;
    const int64_t lda = M.lda;
    const Real *V = M.A + j0 + (int64_t)j0 * lda;
    Real *C = M.A + j0 + (int64_t)col0 * lda;
    const Real *Tg = M.T + (int64_t)j0 * M.ldt;
    const int H = p.hup, ldc = p.hup + 1;             // odd stride: no bank conflicts across j
    const int vst = ldc * b, cst = ldc * kUpdCols;    // stage sizes
    Real *Vs = sm;                     // 2 stages of H x w
    Real *Cs = Vs + 2 * vst;           // 2 stages of H x cw
    Real *Ws = Cs + 2 * cst;           // w x cw, ld b
    Real *Ts = Ws + b * kUpdCols;      // w x w, ld b
    const int nch = (mr + H - 1) / H;
    auto issue = [&](int ch, bool with_c) {
        const int r0 = ch * H, hc = min(H, mr - r0), st = ch & 1;
        async_block(Vs + st * vst, ldc, V + r0, lda, hc, w);
        if (with_c) async_block(Cs + st * cst, ldc, C + r0, lda, hc, cw);
        cp_commit();
    };
    // V's top: 1 on the diagonal, 0 above it (R lives there); H >= b, so
    // only chunk 0 holds those rows
    auto mask_top = [&](Real *Vc, int hc) {
        for (int idx = tid; idx < min(hc, w) * w; idx += nthr) {
            const int r = idx % w, j = idx / w;
            if (r <= j) Vc[r + j * ldc] = (r == j) ? Real(1) : Real(0);
        }
    };
    issue(0, true);
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int i = idx % w, j = idx / w;
        Ts[i + j * b] = (i <= j) ? __ldcg(Tg + i + (int64_t)j * M.ldt) : Real(0);
    }
    const int nout = w * cw;
    Real acc[kMaxOut];
#pragma unroll
    for (int q = 0; q < kMaxOut; ++q) acc[q] = Real(0);
    // FP32 pass-1 blocking: MaxB / 2 pairs of V columns x kUpdCols / kCr
    // groups of C columns = kThreads blocks
    constexpr bool kFp32 = sizeof(Real) == 4;
    constexpr int kCr = kMaxOut / 2;
    static_assert(!kFp32 || (MaxB / 2) * (kUpdCols / kCr) == kThreads, "FP32 pass-1 blocking");
    const int jb = tid % (MaxB / 2), cb = tid / (MaxB / 2);
    Real acc2[2][kCr];
#pragma unroll
    for (int q = 0; q < kCr; ++q) { acc2[0][q] = Real(0); acc2[1][q] = Real(0); }
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) { issue(ch + 1, true); cp_wait<1>(); }
        else cp_wait<0>();
        __syncthreads();
        const int hc = min(H, mr - ch * H), st = ch & 1;
        Real *Vc = Vs + st * vst, *Cc = Cs + st * cst;
        if (ch == 0) { mask_top(Vc, hc); __syncthreads(); }
        if constexpr (kFp32) {
            // columns j of this thread: 2 jb, 2 jb + 1; columns c: kCr cb + q
            const Real *v0 = Vc + (2 * jb) * ldc, *v1 = v0 + ldc, *cp = Cc + (kCr * cb) * ldc;
            for (int r = 0; r < hc; ++r) {
                const Real a0 = v0[r], a1 = v1[r];
#pragma unroll
                for (int q = 0; q < kCr; ++q) {
                    const Real x = cp[r + q * ldc];
                    acc2[0][q] = rfma(a0, x, acc2[0][q]);
                    acc2[1][q] = rfma(a1, x, acc2[1][q]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < kMaxOut; ++q) {
                const int o = tid + q * kThreads;
                if (o < nout) {
                    const int j = o % w, c = o / w;
                    const Real *vp = Vc + j * ldc, *cp = Cc + c * ldc;
                    Real a = acc[q];
                    for (int r = 0; r < hc; ++r) a = rfma(vp[r], cp[r], a);
                    acc[q] = a;
                }
            }
        }
        __syncthreads();                 // the stage is reloaded two chunks on
    }
    issue(0, true);                      // pass 2's first chunk, under the T^T W product
    if constexpr (kFp32) {
#pragma unroll
        for (int jj = 0; jj < 2; ++jj)
#pragma unroll
            for (int q = 0; q < kCr; ++q) {
                const int j = 2 * jb + jj, c = kCr * cb + q;
                if (j < w && c < cw) Ws[j + c * b] = acc2[jj][q];
            }
    } else {
#pragma unroll
        for (int q = 0; q < kMaxOut; ++q) {
            const int o = tid + q * kThreads;
            if (o < nout) Ws[o % w + (o / w) * b] = acc[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxOut; ++q) {             // W <- T^T W
        const int o = tid + q * kThreads;
        if (o < nout) {
            const int j = o % w, c = o / w;
            Real s = Real(0);
            for (int i = 0; i <= j; ++i) s = rfma(Ts[i + j * b], Ws[i + c * b], s);
            acc[q] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxOut; ++q) {
        const int o = tid + q * kThreads;
        if (o < nout) Ws[o % w + (o / w) * b] = acc[q];
    }
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) { issue(ch + 1, true); cp_wait<1>(); }
        else cp_wait<0>();
        __syncthreads();
        const int r0 = ch * H, hc = min(H, mr - r0), st = ch & 1;
        Real *Vc = Vs + st * vst, *Cc = Cs + st * cst;
        if (ch == 0) { mask_top(Vc, hc); __syncthreads(); }
        if constexpr (kFp32) {
            // thread: row r (consecutive across lanes: coalesced C), every
            // groups-th column from g; V(r, :) in registers, W by broadcast
            const int nr = min(H, nthr), groups = nthr / nr;
            for (int r = tid % nr; r < hc; r += nr) {
                Real vr[MaxB];
#pragma unroll
                for (int j = 0; j < MaxB; ++j) vr[j] = (j < w) ? Vc[r + j * ldc] : Real(0);
                for (int c = tid / nr; c < cw; c += groups) {
                    const Real *wc = Ws + c * b;
                    Real s = Real(0);
#pragma unroll
                    for (int j = 0; j < MaxB; ++j) s = rfma(vr[j], (j < w) ? wc[j] : Real(0), s);
                    C[r0 + r + (int64_t)c * lda] = Cc[r + c * ldc] - s;
                }
            }
        } else {
            for (int e = tid; e < hc * cw; e += nthr) {
                const int c = e / hc, r = e - c * hc;
                Real s = Real(0);
                for (int j = 0; j < w; ++j) s = rfma(Vc[r + j * ldc], Ws[j + c * b], s);
                C[r0 + r + (int64_t)c * lda] = Cc[r + c * ldc] - s;
            }
        }
        __syncthreads();
    }
}

// MaxB: the largest panel width b this instantiation runs (16 or 32).
template <int MaxB, class Real>
__global__ void __launch_bounds__(kThreads, 2) batched_qr_kernel(BParams<Real> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *sm = reinterpret_cast<Real *>(smem_raw);
    __shared__ int s_task[4];
    __shared__ int s_go;
    Real *tscr = p.tscr + (size_t)blockIdx.x * p.tscr_stride;
    for (;;) {
        if (threadIdx.x == 0) {
            int go = 0;
            if (!*(volatile int *)p.abort) {
                const unsigned t = atomicAdd(p.next, 1u);
                if (t < (unsigned)p.ntasks) {
                    const int4 tk = p.tasks[t];
                    s_task[0] = tk.x; s_task[1] = tk.y; s_task[2] = tk.z; s_task[3] = tk.w;
                    go = wait_deps(p, p.state + p.mats[tk.x].state0, tk.y, tk.z, tk.w) ? 1 : 0;
                }
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) return;
        const int mi = s_task[0], k = s_task[1], c0 = s_task[2], c1 = s_task[3];
        const BMat<Real> M = p.mats[mi];
        int bad = 0;
        if (c0 == c1) bad = panel_task<MaxB>(p, M, k, sm, tscr);
        else update_task<MaxB>(p, M, k, c0, c1, sm);
        bad = __syncthreads_or(bad);
        if (threadIdx.x == 0) {
            if (bad) atomicOr(p.nonfinite, 1ull);
            __threadfence();
            int *st = p.state + M.state0;
            if (c0 == c1) st_release(st + k, k + 1);
            else
                for (int c = c0; c < c1; ++c) st_release(st + c, k + 1);
        }
    }
}

// The instantiation that runs panel width b.
template <class Real>
const void *kernel_for(int b) {
    return b <= 16 ? (const void *)batched_qr_kernel<16, Real> : (const void *)batched_qr_kernel<kMaxBatchB, Real>;
}

size_t panel_smem(int b, int hblk, size_t real) {
    return real * ((size_t)(hblk + b) * b + 8 * (size_t)b * b + 8 * (size_t)b);
}
size_t update_smem(int b, int hup, size_t real) {
    return real * (2 * (size_t)(hup + 1) * (b + kUpdCols) + (size_t)b * kUpdCols + (size_t)b * b);
}

// Rows per update chunk: the most (a multiple of 16, at most 128) whose two
// stages fit the shared-memory budget.
int update_rows(int b, size_t real) {
    int h = 128;
    while (h > 16 && update_smem(b, h, real) > kSmemBudget) h -= 16;
    return h;
}

// Tallest row block a panel task's shared memory holds (a multiple of 32).
int block_rows(int b, size_t real) {
    const size_t fixed = panel_smem(b, 0, real);
    if (fixed >= kSmemBudget) return 0;
    int h = (int)((kSmemBudget - fixed) / (real * (size_t)b)) / 32 * 32;
    return std::max(h, 0);
}

uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

}  // namespace

struct BatchPlan {
    uint64_t key = 0;            // shapes, leading dimensions, b, scalar size, device
    size_t real = 8;
    int b = 16, hblk = 0, hup = 64, ldS = 0, grid = 0, ntasks = 0, nstate = 0, tscr_blocks = 0, count = 0;
    size_t smem = 0;
    size_t off_tasks = 0, off_state = 0, off_tscr = 0, total = 0, table_bytes = 0, state_bytes = 0;
    size_t tscr_stride = 0;
    std::vector<int4> order;     // the task list, in list-schedule order
    std::vector<int> state0;     // each matrix's first column-block counter
    std::vector<unsigned char> stage;   // pageable staging of the table for uncaptured calls
    double est_ms = 0.0;         // the list schedule's estimated makespan
};

void batch_plan_free(BatchPlan *pl) { delete pl; }

double batch_plan_estimate_ms(const BatchPlan *pl) { return pl ? pl->est_ms : 0.0; }
size_t batched_plan_bytes(const BatchPlan *pl) { return pl ? pl->total : 0; }

namespace {

// Task list of the batch in list-schedule order: tasks are started on G
// simulated workers as workers free up, highest bottom level (longest path
// to the end of its matrix, in estimated cycles) first.
struct SimTask {
    int mat, k, c0, c1;
    double dur, bl = 0.0;
    int npred = 0;
    std::vector<int> succ;
};

bool build_plan(BatchPlan *pl, int count, const int64_t *m, const int64_t *n, int b, int grid, size_t real,
                size_t mat_bytes) {
    std::vector<SimTask> tk;
    pl->state0.assign(count, 0);
    int nstate = 0, maxP = 1;
    const int ublk = std::max(1, kUpdCols / b);
    std::vector<int> prev_grp, cur_grp;
    for (int i = 0; i < count; ++i) {
        pl->state0[i] = nstate;
        if (n[i] == 0) continue;
        const int nbk = (int)((n[i] + b - 1) / b);
        nstate += nbk;
        prev_grp.assign(nbk, -1);
        for (int k = 0; k < nbk; ++k) {
            const int w = (int)std::min<int64_t>(b, n[i] - (int64_t)k * b);
            const double mr = (double)(m[i] - (int64_t)k * b);
            const int P = (int)((m[i] - (int64_t)k * b + pl->hblk - 1) / pl->hblk);
            maxP = std::max(maxP, P);
            // estimated cycles of one CTA sharing its SM's FP64 pipe with another
            SimTask pt{i, k, k, k, 2.0 * mr * w * w + 4000.0 * w * P + 2e4};
            const int pid = (int)tk.size();
            tk.push_back(pt);
            if (k > 0) { tk[prev_grp[k]].succ.push_back(pid); tk[pid].npred++; }
            cur_grp.assign(nbk, -1);
            int c = k + 1;
            while (c < nbk) {
                const int c1 = (c == k + 1) ? c + 1 : std::min(nbk, c + ublk);
                const double cw = (double)(std::min<int64_t>((int64_t)c1 * b, n[i]) - (int64_t)c * b);
                SimTask ut{i, k, c, c1, 2.2 * mr * w * cw + 1e4};
                const int uid = (int)tk.size();
                tk.push_back(ut);
                tk[pid].succ.push_back(uid);
                tk[uid].npred++;
                if (k > 0) {
                    int last = -1;
                    for (int cc = c; cc < c1; ++cc)
                        if (prev_grp[cc] != last) {
                            last = prev_grp[cc];
                            tk[last].succ.push_back(uid);
                            tk[uid].npred++;
                        }
                }
                for (int cc = c; cc < c1; ++cc) cur_grp[cc] = uid;
                c = c1;
            }
            prev_grp.swap(cur_grp);
        }
    }
    if (tk.size() > (size_t)(INT32_MAX / 2)) return false;
    // bottom levels (creation order is topological)
    for (int t = (int)tk.size() - 1; t >= 0; --t) {
        double best = 0.0;
        for (int s2 : tk[t].succ) best = std::max(best, tk[s2].bl);
        tk[t].bl = tk[t].dur + best;
    }
    // list schedule on `grid` workers
    auto cmp = [&](int a, int c) { return tk[a].bl < tk[c].bl || (tk[a].bl == tk[c].bl && a > c); };
    std::priority_queue<int, std::vector<int>, decltype(cmp)> ready(cmp);
    for (int t = 0; t < (int)tk.size(); ++t)
        if (tk[t].npred == 0) ready.push(t);
    typedef std::pair<double, int> Ev;
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
    pl->order.clear();
    pl->order.reserve(tk.size());
    double now = 0.0;
    int free_w = grid;
    while (!ready.empty() || !running.empty()) {
        while (free_w > 0 && !ready.empty()) {
            const int t = ready.top();
            ready.pop();
            pl->order.push_back(make_int4(tk[t].mat, tk[t].k, tk[t].c0, tk[t].c1));
            running.push(Ev(now + tk[t].dur, t));
            --free_w;
        }
        if (running.empty()) break;
        const Ev e = running.top();
        running.pop();
        now = e.first;
        ++free_w;
        for (int s2 : tk[e.second].succ)
            if (--tk[s2].npred == 0) ready.push(s2);
    }
    if (pl->order.size() != tk.size()) return false;
    pl->est_ms = now / 2.07e6;
    pl->ntasks = (int)pl->order.size();
    pl->nstate = nstate;
    pl->tscr_blocks = maxP;
    pl->count = count;
    // device layout: [matrix table | task list] (uploaded each call)
    // [counters, dispenser, abort flag] [per-CTA T scratch]
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    pl->off_tasks = al(mat_bytes * (size_t)count);
    pl->table_bytes = pl->off_tasks + sizeof(int4) * pl->order.size();
    pl->off_state = al(pl->table_bytes);
    pl->state_bytes = sizeof(int) * ((size_t)nstate + 2);
    pl->off_tscr = al(pl->off_state + pl->state_bytes);
    pl->tscr_stride = (size_t)maxP * b * b;
    pl->total = al(pl->off_tscr + real * pl->tscr_stride * (size_t)grid);
    return true;
}

}  // namespace

template <class Real>
gbqr_status batched_plan(BatchPlan **cache, int device, int num_sms, int count, const int64_t *m,
                         const int64_t *n, const int64_t *lda, const int64_t *ldt, int b, bool may_build,
                         BatchPlan **out) {
    *out = nullptr;
    if (b < 1 || b > kMaxBatchB) return GBQR_EINVAL;
    const int hblk = block_rows(b, sizeof(Real));
    if (hblk < 2 * b) return GBQR_EINVAL;
    for (int i = 0; i < count; ++i)
        if (m[i] < n[i] || n[i] < 0 || m[i] > INT32_MAX / 2 || lda[i] < std::max<int64_t>(1, m[i]) ||
            ldt[i] < std::max<int64_t>(1, std::min<int64_t>(b, n[i])))
            return GBQR_EINVAL;
    uint64_t key = 1469598103934665603ull;
    const int sz = (int)sizeof(Real);
    key = fnv(key, &count, sizeof count);
    key = fnv(key, &b, sizeof b);
    key = fnv(key, &sz, sizeof sz);
    key = fnv(key, &device, sizeof device);
    key = fnv(key, m, sizeof(int64_t) * count);
    key = fnv(key, n, sizeof(int64_t) * count);
    key = fnv(key, lda, sizeof(int64_t) * count);
    key = fnv(key, ldt, sizeof(int64_t) * count);
    BatchPlan *pl = *cache;
    if (pl && pl->key == key) { *out = pl; return GBQR_OK; }
    if (!may_build) return GBQR_EBUSY;
    const int hup = update_rows(b, sizeof(Real));
    const size_t smem = std::max(panel_smem(b, hblk, sizeof(Real)), update_smem(b, hup, sizeof(Real)));
    const void *kern = kernel_for<Real>(b);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return GBQR_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess || per_sm < 1)
        return GBQR_ECUDA;
    if (!pl) {
        pl = new (std::nothrow) BatchPlan();
        if (!pl) return GBQR_ENOMEM;
        *cache = pl;
    }
    pl->key = 0;
    pl->real = sizeof(Real);
    pl->b = b;
    pl->hblk = hblk;
    pl->hup = hup;
    pl->ldS = hblk + b;
    pl->smem = smem;
    pl->grid = per_sm * num_sms;
    if (!build_plan(pl, count, m, n, b, pl->grid, sizeof(Real), sizeof(BMat<Real>))) return GBQR_ENOMEM;
    pl->key = key;
    *out = pl;
    return GBQR_OK;
}

template <class Real>
gbqr_status batched_enqueue(const Exec &ex, BatchPlan *pl, Real *const *A, Real *const *T, const int64_t *m,
                            const int64_t *n, const int64_t *lda, const int64_t *ldt, char *ws, size_t ws_bytes,
                            int *timeout_flag, unsigned long long *nonfinite, bool capturing, void **owned) {
    *owned = nullptr;
    if (!pl || pl->real != sizeof(Real) || ws_bytes < pl->total) return GBQR_EINVAL;
    if (pl->ntasks == 0) return GBQR_OK;
    for (int i = 0; i < pl->count; ++i)
        if (n[i] > 0 && (!A[i] || !T[i])) return GBQR_EINVAL;
    // the matrix table and the task list, uploaded on the stream: from
    // pageable staging when running now (the copy is staged before the call
    // returns), from page-locked memory that the captured graph keeps when
    // capturing
    unsigned char *host = nullptr;
    if (capturing) {
        if (cudaMallocHost((void **)&host, pl->table_bytes) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
        *owned = host;
    } else {
        pl->stage.resize(pl->table_bytes);
        host = pl->stage.data();
    }
    BMat<Real> *mats = reinterpret_cast<BMat<Real> *>(host);
    for (int i = 0; i < pl->count; ++i) {
        BMat<Real> bm;
        bm.A = A[i]; bm.T = T[i]; bm.lda = lda[i]; bm.ldt = ldt[i];
        bm.m = (int)m[i]; bm.n = (int)n[i]; bm.state0 = pl->state0[i]; bm.pad = 0;
        memcpy(mats + i, &bm, sizeof bm);
    }
    memcpy(host + pl->off_tasks, pl->order.data(), sizeof(int4) * pl->order.size());
    if (cudaMemcpyAsync(ws, host, pl->table_bytes, cudaMemcpyHostToDevice, ex.stream) != cudaSuccess ||
        cudaMemsetAsync(ws + pl->off_state, 0, pl->state_bytes, ex.stream) != cudaSuccess)
        return GBQR_ECUDA;
    BParams<Real> p;
    p.mats = reinterpret_cast<const BMat<Real> *>(ws);
    p.tasks = reinterpret_cast<const int4 *>(ws + pl->off_tasks);
    p.ntasks = pl->ntasks;
    p.b = pl->b;
    p.hblk = pl->hblk;
    p.hup = pl->hup;
    p.ldS = pl->ldS;
    p.state = reinterpret_cast<int *>(ws + pl->off_state);
    p.next = reinterpret_cast<unsigned *>(p.state + pl->nstate);
    p.abort = p.state + pl->nstate + 1;
    p.timeout = timeout_flag;
    p.nonfinite = nonfinite;
    p.tscr = reinterpret_cast<Real *>(ws + pl->off_tscr);
    p.tscr_stride = pl->tscr_stride;
    p.tscr_blocks = pl->tscr_blocks;
    p.wait_ns = 5000000000ll;   // 5 s: far beyond any one matrix's critical path
    trace_begin(ex, FAM_BATCHED);
    if (pl->b <= 16) batched_qr_kernel<16, Real><<<pl->grid, kThreads, pl->smem, ex.stream>>>(p);
    else batched_qr_kernel<kMaxBatchB, Real><<<pl->grid, kThreads, pl->smem, ex.stream>>>(p);
    return trace_end(ex, FAM_BATCHED, 0.0, 0.0);
}

template gbqr_status batched_plan<double>(BatchPlan **, int, int, int, const int64_t *, const int64_t *,
                                          const int64_t *, const int64_t *, int, bool, BatchPlan **);
template gbqr_status batched_plan<float>(BatchPlan **, int, int, int, const int64_t *, const int64_t *,
                                         const int64_t *, const int64_t *, int, bool, BatchPlan **);
template gbqr_status batched_enqueue<double>(const Exec &, BatchPlan *, double *const *, double *const *,
                                             const int64_t *, const int64_t *, const int64_t *, const int64_t *,
                                             char *, size_t, int *, unsigned long long *, bool, void **);
template gbqr_status batched_enqueue<float>(const Exec &, BatchPlan *, float *const *, float *const *,
                                            const int64_t *, const int64_t *, const int64_t *, const int64_t *,
                                            char *, size_t, int *, unsigned long long *, bool, void **);

}  // namespace gbqr

// Failure-detection self-test of the dependency wait: one CTA of the FP64
// kernel gets a task list holding only update(0, 0, 1, 2), whose panel
// (block 0 factored) never runs, so its wait must give up after wait_ms,
// raise the abort and timeout flags and return.  completed: block 1's
// counter afterwards (0: the update did not run).
extern "C" GBQR_API gbqr_status gbqr_selftest_batched_wait(int device, int wait_ms, int *completed) {
    using namespace gbqr;
    if (!completed || wait_ms < 1 || wait_ms > 10000) return GBQR_EINVAL;
    *completed = -1;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    // [mats | tasks | state (2) + dispenser + abort | timeout flag] in one allocation
    const size_t off_tasks = 256, off_state = 512, off_flag = 768, bytes = 1024;
    char *d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
    gbqr_status st = GBQR_OK;
    BMat<double> bm;
    bm.A = reinterpret_cast<double *>(d); bm.T = reinterpret_cast<double *>(d);   // never dereferenced
    bm.lda = 64; bm.ldt = 16; bm.m = 64; bm.n = 32; bm.state0 = 0; bm.pad = 0;
    const int4 task = make_int4(0, 0, 1, 2);
    if (cudaMemset(d, 0, bytes) != cudaSuccess || cudaMemcpy(d, &bm, sizeof bm, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + off_tasks, &task, sizeof task, cudaMemcpyHostToDevice) != cudaSuccess)
        st = GBQR_ECUDA;
    const size_t smem = std::max(panel_smem(16, 64, 8), update_smem(16, 16, 8));
    if (st == GBQR_OK &&
        cudaFuncSetAttribute(batched_qr_kernel<16, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        st = GBQR_ECUDA;
    int h[2] = {0, 0};
    if (st == GBQR_OK) {
        BParams<double> p;
        p.mats = reinterpret_cast<const BMat<double> *>(d);
        p.tasks = reinterpret_cast<const int4 *>(d + off_tasks);
        p.ntasks = 1;
        p.b = 16; p.hblk = 64; p.ldS = 80; p.hup = 16;
        p.state = reinterpret_cast<int *>(d + off_state);
        p.next = reinterpret_cast<unsigned *>(p.state + 2);
        p.abort = p.state + 3;
        p.timeout = reinterpret_cast<int *>(d + off_flag);
        p.nonfinite = reinterpret_cast<unsigned long long *>(d + off_flag + 8);
        p.tscr = reinterpret_cast<double *>(d);
        p.tscr_stride = 0;
        p.tscr_blocks = 0;
        p.wait_ns = (long long)wait_ms * 1000000ll;
        batched_qr_kernel<16, double><<<1, kThreads, smem>>>(p);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h[0], d + off_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&h[1], d + off_state + sizeof(int), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = GBQR_ECUDA;
    }
    cudaFree(d);
    if (st != GBQR_OK) return st;
    *completed = h[1];
    return h[0] ? GBQR_ETIMEOUT : GBQR_OK;
}
