// Device building blocks of the TSQR base case (Section 5, Appendix C),
// shared by the single-panel TSQR kernels (tsqr.cu) and the persistent
// batched QR kernel (batched.cu): warp reductions, coalesced block loads,
// the Householder QR of a block held in shared memory (its rows described
// by a Rows policy), the kernel T by the closed form of Section 2.3, and the
// small triangular products of the downsweep and reconstruction.
#pragma once

#include "common.cuh"

namespace gbqr {
namespace {

__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double real_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float real_sqrt(float x) { return sqrtf(x); }
// 1/x rounded to nearest: the same value as the IEEE division 1/x, through
// the reciprocal intrinsic, which takes about 60 % of the division's FP64
// issue slots on this part
__device__ __forceinline__ double real_rcp(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float real_rcp(float x) { return __frcp_rn(x); }

constexpr unsigned kFull = 0xffffffffu;

template <class Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Warp sums of N <= 4 per-lane values; every lane receives all N sums.  For
// N > 1 a butterfly reduce-scatter (halve the set at offsets 16 and 8, then
// three full stages) costs 6 FP64 adds instead of 5 per value.
template <int N, class Real>
__device__ __forceinline__ void warp_sum_n(Real (&v)[4]) {
    if (N == 1) { v[0] = warp_sum(v[0]); return; }
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    Real k0 = h16 ? v[2] : v[0], k1 = h16 ? v[3] : v[1];
    const Real s0 = h16 ? v[0] : v[2], s1 = h16 ? v[1] : v[3];
    k0 += __shfl_xor_sync(kFull, s0, 16);
    k1 += __shfl_xor_sync(kFull, s1, 16);
    Real k = h8 ? k1 : k0;
    const Real s = h8 ? k0 : k1;
    k += __shfl_xor_sync(kFull, s, 8);
    k += __shfl_xor_sync(kFull, k, 4);
    k += __shfl_xor_sync(kFull, k, 2);
    k += __shfl_xor_sync(kFull, k, 1);
    // lane L now holds sum number 2*bit4(L) + bit3(L)
    v[0] = __shfl_sync(kFull, k, 0);
    v[1] = __shfl_sync(kFull, k, 8);
    v[2] = __shfl_sync(kFull, k, 16);
    v[3] = __shfl_sync(kFull, k, 24);
}

// dst(r, c) = src(r, c) for an h x w column-major block (dst ld ldd, src ld
// lds), the whole CTA: every thread issues up to 8 loads before its first
// store, so a block read from L2 or HBM costs about one memory latency
// instead of one per column.
template <class Real>
__device__ __forceinline__ void load_block(Real *dst, int64_t ldd, const Real *src, int64_t lds, int h, int w) {
    constexpr int kBatch = 8;
    const int tid = threadIdx.x, nthr = blockDim.x, total = h * w;
    for (int base = tid; base < total; base += kBatch * nthr) {
        Real v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int idx = base + k * nthr;
            if (idx < total) {
                const int c = idx / h, r = idx - c * h;
                v[k] = __ldcg(src + r + (int64_t)c * lds);
            }
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int idx = base + k * nthr;
            if (idx < total) {
                const int c = idx / h, r = idx - c * h;
                dst[r + (int64_t)c * ldd] = v[k];
            }
        }
    }
}

// Rows of column j below its pivot in a leaf block: j+1 .. h-1.
struct LeafRows {
    int h;
    static constexpr bool kNextPivotInB = true;   // step j touches row j+1
    template <class F>
    __device__ __forceinline__ void each(int j, int lane, F &&f) const {
        for (int r = j + 1 + lane; r < h; r += 32) f(r);
    }
    // Of the rows step j touches, those below the pivot of column j+1; no
    // row of column j+1 below its pivot is outside step j's rows.
    __device__ __forceinline__ bool below_next(int j, int r) const { return r > j + 1; }
    template <class F>
    __device__ __forceinline__ void each_untouched(int, int, F &&) const {}
    // pivot row j first (f(r, true)), then rows(j): one pass, no separate
    // pivot-row term
    template <class F>
    __device__ __forceinline__ void each_with_pivot(int j, int lane, F &&f) const {
        for (int r = j + lane; r < h; r += 32) f(r, r == j);
    }
};

// Rows of column j below its pivot in cnt stacked w x w upper triangles:
// rows 0..j of every triangle after the first.  The (cnt-1)(j+1) entries are
// spread over the lanes as one flat list, so a lane touches about
// (cnt-1)(j+1)/32 of them instead of cnt-1.  Entry e = b d + r (d = j+1) is
// row r of triangle b+1; a lane steps e by 32 = q d + s, so (b, r) advances
// by (q, s) with at most one carry and only the first entry needs a division.
struct MergeRows {
    int w, cnt;
    static constexpr bool kNextPivotInB = false;
    // Of the rows step j touches, those below the pivot of column j+1 (every
    // triangle after the first); row j+1 of those triangles is below that
    // pivot too but outside step j's rows.
    __device__ __forceinline__ bool below_next(int, int r) const { return r >= w; }
    template <class F>
    __device__ __forceinline__ void each_untouched(int j, int lane, F &&f) const {
        for (int i = 1 + lane; i < cnt; i += 32) f(i * w + j + 1);
    }
    template <class F>
    __device__ __forceinline__ void walk(int d, int e, F &&f) const {
        const int n = (cnt - 1) * d;
        if (e >= n) return;
        const int q = 32 / d, s = 32 - q * d;
        int b = e / d, r = e - b * d;
        for (; e < n; e += 32) {
            f((b + 1) * w + r);
            b += q;
            r += s;
            if (r >= d) { r -= d; ++b; }
        }
    }
    template <class F>
    __device__ __forceinline__ void each(int j, int lane, F &&f) const {
        walk(j + 1, lane, f);
    }
    // entry 0 of the flat list is the pivot; entry i > 0 is e = i - 1 above
    template <class F>
    __device__ __forceinline__ void each_with_pivot(int j, int lane, F &&f) const {
        if (lane == 0) f(j, true);
        walk(j + 1, lane == 0 ? 31 : lane - 1, [&](int r) { f(r, false); });
    }
};

// Rows of column j below its pivot in a w x w upper triangle R stacked on a
// dense block of h rows, [R; A] (rows 0..w-1, then w..w+h-1): the h dense
// rows.  R's rows below a pivot are zero and stay zero, so the stacked
// Householder vectors are [e_j; y_j] and V = [I; Y].
struct StackRows {
    int w, h;
    static constexpr bool kNextPivotInB = false;
    template <class F>
    __device__ __forceinline__ void each(int, int lane, F &&f) const {
        for (int r = w + lane; r < w + h; r += 32) f(r);
    }
    __device__ __forceinline__ bool below_next(int, int r) const { return r >= w; }
    template <class F>
    __device__ __forceinline__ void each_untouched(int, int, F &&) const {}
    // entry 0 of the list is the pivot, entry e > 0 dense row w + e - 1
    template <class F>
    __device__ __forceinline__ void each_with_pivot(int j, int lane, F &&f) const {
        for (int e = lane; e <= h; e += 32) f(e == 0 ? j : w + e - 1, e == 0);
    }
};

// Reflectors are kept unnormalised while a block is factored.  With
// beta = -sgn(alpha) ||column|| (sgn(0) = +1), d = alpha - beta (no
// cancellation) and x the column below its pivot, the normalised vector is
// v = [1; x/d] and tau = (beta - alpha)/beta; with vh = [d; x] and
// q = 1/(beta d) the same reflector is H = I - tau v v^T = I + q vh vh^T.
// So the pivot warp only publishes beta (on the pivot), d, beta*d and the
// squared norm below the pivot: the reciprocal q is taken by another warp
// during the next step, and the scaling of x by 1/d, tau and the Gram entries
// are settled once per block (finish_block).  A zero column (beta = 0) is
// stored as d = 1, beta*d = 0, and q_of maps it to q = -2: H = I - 2 e e^T,
// tau = 2.
template <class Real>
struct Refl {
    Real *tau;   // tau[c], from finish_block on
    Real *d;     // d[c]
    Real *bd;    // beta[c] * d[c]  (0 for a zero column)
    Real *q;     // q[c] = 1/(beta d), published in step c
    Real *sc;    // 1/d[c], from finish_block on
    Real *sg;    // squared norm of column c below its pivot, published with it
};

template <class Real>
__device__ __forceinline__ Real q_of(Real bd) { return bd == Real(0) ? Real(-2) : real_rcp(bd); }

// q_j goes from the warp that computes it (the pivot warp's sub-partition
// partner, bar.arrive on both) to the six warps that update other columns
// through named barrier 1 (7 warps) and to the pivot warp through named
// barrier 2 (2 warps), so that neither waits for the other.  Every step the
// partner arrives once at each, and each of the other seven warps syncs
// exactly once at its own.
constexpr int kQBarrier = 1;
constexpr int kQThreads = 7 * 32;
constexpr int kQPivotBarrier = 2;
constexpr int kQPivotThreads = 2 * 32;
// (barrier.* without .aligned: correct even where a warp is not converged)
__device__ __forceinline__ void q_arrive() {
    __syncwarp();
    asm volatile("barrier.arrive %0, %1;" ::"n"(kQBarrier), "n"(kQThreads) : "memory");
    asm volatile("barrier.arrive %0, %1;" ::"n"(kQPivotBarrier), "n"(kQPivotThreads) : "memory");
}
__device__ __forceinline__ void q_sync() {
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"n"(kQBarrier), "n"(kQThreads) : "memory");
}
__device__ __forceinline__ void q_sync_pivot() {
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"n"(kQPivotBarrier), "n"(kQPivotThreads) : "memory");
}

// One warp turns column c (pivot entry alpha, squared norm below the pivot
// sig2) into an unnormalised reflector: beta on the pivot; d, beta*d and
// sig2 published.
template <class Real>
__device__ __forceinline__ void publish_pivot(Real *S, int ldS, int c, const Refl<Real> &rf, Real alpha, Real sig2) {
    const int lane = threadIdx.x & 31;
    Real *col = S + (size_t)c * ldS;
    const Real nrm = real_sqrt(rfma(alpha, alpha, sig2));
    const Real beta = alpha < Real(0) ? nrm : -nrm;
    const Real d = beta != Real(0) ? alpha - beta : Real(1);
    __syncwarp();
    if (lane == 0) { col[c] = beta; rf.d[c] = d; rf.bd[c] = beta * d; rf.sg[c] = sig2; }
    __syncwarp();
}

template <class Real, class Rows>
__device__ void warp_pivot(Real *S, int ldS, int c, const Rows &rows, const Refl<Real> &rf) {
    const int lane = threadIdx.x & 31;
    const Real *col = S + (size_t)c * ldS;
    Real part = Real(0);
    rows.each(c, lane, [&](int r) { const Real x = col[r]; part = rfma(x, x, part); });
    publish_pivot(S, ldS, c, rf, col[c], warp_sum(part));
}

// The pivot warp's share of step j: reflector j applied to column c = j+1,
// then column c published as the next reflector.  With x = column c before
// the step, v = vh_j and f = q_j vh_j^T x, the rows B below pivot j are
// updated to x + f v, so the squared norm of column c below its own pivot is
//     S2 + f (2 S3 + f s4)   (minus the new pivot entry's square where B
//                             holds it, as in a leaf block),
// with S2 = sum of x^2 over B and over the rows below pivot c outside B,
// S3 = sum of v x over B and s4 = sum of v^2 over B, which is column j's
// published norm.  So one pass over the rows and one warp reduction (of S2
// and S3) come before the square root, instead of a pass, a reduction, a
// second pass and a second reduction.  Where the three terms cancel (the result is below half their
// magnitude, so it would carry more than a few rounding errors of them),
// the norm is summed directly from the updated rows instead.
template <class Real, class Rows>
__device__ void pivot_step(Real *S, int ldS, int j, int w, const Rows &rows, const Refl<Real> &rf) {
    const int lane = threadIdx.x & 31, c = j + 1;
    if (c >= w) { q_sync_pivot(); return; }        // last step: q_j is only stored
    const Real dj = rf.d[j];
    const Real *vj = S + (size_t)j * ldS;
    Real *col = S + (size_t)c * ldS;
    const Real xj = col[j];                        // row j of column c, before the step
    const Real xc = col[c], vc = vj[c];            // the next pivot row
    Real s3 = Real(0), s2 = Real(0);
    rows.each(j, lane, [&](int r) {
        const Real x = col[r];
        s3 = rfma(vj[r], x, s3);
        s2 = rfma(x, x, s2);
    });
    rows.each_untouched(j, lane, [&](int r) { const Real x = col[r]; s2 = rfma(x, x, s2); });
    Real sums[4] = {s3, s2, Real(0), Real(0)};
    warp_sum_n<2>(sums);
    const Real S3 = sums[0], S2 = sums[1], s4 = rf.sg[j];
    q_sync_pivot();                                // q_j from the partner warp
    const Real f = rf.q[j] * rfma(dj, xj, S3);
    const Real sumB = rfma(f, rfma(f, s4, Real(2) * S3), S2);
    Real alpha = xc, sig2 = sumB;
    if (Rows::kNextPivotInB) {
        alpha = rfma(f, vc, xc);
        sig2 = rfma(-alpha, alpha, sumB);
    }
    const bool direct = !(sig2 >= Real(0.5) * rfma(f * f, s4, S2));
    if (!direct) {
        rows.each_with_pivot(j, lane, [&](int r, bool piv) { col[r] = rfma(f, piv ? dj : vj[r], col[r]); });
    } else {
        Real part = Real(0);
        rows.each_with_pivot(j, lane, [&](int r, bool piv) {
            const Real x = rfma(f, piv ? dj : vj[r], col[r]);
            col[r] = x;
            if (rows.below_next(j, r)) part = rfma(x, x, part);
        });
        rows.each_untouched(j, lane, [&](int r) { const Real x = col[r]; part = rfma(x, x, part); });
        sig2 = warp_sum(part);
    }
    publish_pivot(S, ldS, c, rf, alpha, sig2);
}

// One warp applies reflector j to N columns (c > j: A(:,c) += q_j vh_j
// (vh_j^T A(:,c))) or, for c < j, records the unscaled Gram entry
// vh_c^T vh_j (scaled to v_c^T v_j by finish_block).  q_j is taken from the
// partner warp through the named barrier, once per step (*synced).
template <int N, class Real, class Rows>
__device__ __forceinline__ void warp_apply(Real *S, int ldS, int j, const Rows &rows, const int (&cols)[4],
                                           const Refl<Real> &rf, Real *G, int w, bool *synced, Real *qj) {
    const int lane = threadIdx.x & 31;
    const Real *vj = S + (size_t)j * ldS;
    const Real dj = rf.d[j];
    Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
    rows.each_with_pivot(j, lane, [&](int r, bool piv) {
        const Real v = piv ? dj : vj[r];
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = rfma(v, S[r + (size_t)cols[q] * ldS], acc[q]);
    });
    warp_sum_n<N>(acc);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const int c = cols[q];
        if (c > j) {
            if (!*synced) { q_sync(); *synced = true; *qj = rf.q[j]; }
            const Real f = *qj * acc[q];
            Real *colc = S + (size_t)c * ldS;
            rows.each_with_pivot(j, lane, [&](int r, bool piv) {
                colc[r] = rfma(f, piv ? dj : vj[r], colc[r]);
            });
        } else if (lane == 0) {
            G[c + j * w] = acc[q];
        }
    }
}

// Householder QR of the w columns held in shared memory S (column-major,
// leading dimension ldS); column j acts on its pivot row j and the rows that
// `rows` lists.  During step j one warp (j % 8) updates column j+1 and turns
// it into the next reflector while six others share every remaining column
// round robin, so each step needs one CTA barrier (and the q_j hand-over).
// On GB300 a warp issues at most one FP64 instruction per ~64 cycles and an
// SM sub-partition one per ~76, and a dependent FP64 result takes ~125
// cycles, so the step time is the longer of the pivot warp's dependency
// chain and the FP64 instruction count of the busiest sub-partition: the
// pivot warp (square root, one warp reduction) carries nothing else, and the
// warp that shares its sub-partition (warp i runs on sub-partition i % 4)
// only takes the reciprocal q_j off the pivot warp's chain.  Leaves the
// reflectors unnormalised (vh_c below the pivots, d, beta*d, q); finish_block
// settles them.
template <class Real, class Rows>
__device__ void householder_block(Real *S, int ldS, int w, const Rows &rows, const Refl<Real> &rf, Real *G) {
    static_assert(kThreads == 256, "the q_j hand-over is laid out for 8 warps");
    constexpr int nw = kThreads / 32;
    const int wid = threadIdx.x >> 5;
    if (wid == 0) warp_pivot(S, ldS, 0, rows, rf);
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        const int nxt = j + 1;
        const int pw = j % nw;                         // pivot warp of this step
        const int partner = (pw + 4) % nw;
        if (wid == pw) {
            pivot_step(S, ldS, j, w, rows, rf);
        } else if (wid == partner) {
            if ((threadIdx.x & 31) == 0) rf.q[j] = q_of(rf.bd[j]);
            __syncwarp();
            __threadfence_block();
            q_arrive();
        } else {
            const int nexcl = (nxt < w) ? 2 : 1;
            const int ncols = w - nexcl;
            constexpr int nwork = nw - 2;
            int me = (wid - pw - 1 + nw) % nw;        // 0 .. nw-2
            if (me > (partner - pw - 1 + nw) % nw) --me;   // skip the partner's slot
            bool synced = false;
            Real qj = Real(0);
            int cols[4] = {0, 0, 0, 0};
            int g = 0;
            for (int t = me; t < ncols; t += nwork) {
                cols[g++] = (t < j) ? t : t + nexcl;
                if (g == 4) { warp_apply<4>(S, ldS, j, rows, cols, rf, G, w, &synced, &qj); g = 0; }
            }
            if (g == 1) warp_apply<1>(S, ldS, j, rows, cols, rf, G, w, &synced, &qj);
            else if (g == 2) warp_apply<2>(S, ldS, j, rows, cols, rf, G, w, &synced, &qj);
            else if (g == 3) warp_apply<3>(S, ldS, j, rows, cols, rf, G, w, &synced, &qj);
            if (!synced) q_sync();                     // exactly one sync per step
        }
        __syncthreads();
    }
}

// After householder_block: tau[c] = -d^2 q, sc[c] = 1/d (= beta q, 1 for a
// zero column) and the Gram entries G(c, j) = v_c^T v_j = sc_c sc_j
// vh_c^T vh_j (strict upper, ld w).  The caller scales x by sc when it writes
// V out.  Ends with a CTA barrier.
template <class Real>
__device__ void finish_block(const Real *S, int ldS, int w, const Refl<Real> &rf, Real *G) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int c = tid; c < w; c += nthr) {
        const Real q = rf.q[c], d = rf.d[c], bd = rf.bd[c];
        rf.tau[c] = -(d * d) * q;
        rf.sc[c] = bd == Real(0) ? Real(1) : S[c + (size_t)c * ldS] * q;
    }
    __syncthreads();
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int c = idx % w, j = idx / w;
        if (c < j) G[idx] *= rf.sc[c] * rf.sc[j];
    }
    __syncthreads();
}

// The kernel T of Q = I - V T V^T from tau and the strict upper Gram matrix
// G = striu(V^T V): T^{-1} = striu(G) + diag(1/tau) (the closed form of
// Section 2.3).  Built bottom-up over block sizes s = 1, 2, 4, ...: for each
// pair of adjacent diagonal blocks T12 = -T11 G12 T22 (the T assembly of
// Algorithm 2), so the dependency depth is log2(w) small products instead of
// a w-step recurrence.  M is w x w scratch.  T, G, M: ld w, shared memory.
template <class Real>
__device__ void build_t(Real *T, const Real *G, const Real *tau, Real *M, int w) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int i = idx % w, c = idx / w;
        T[idx] = (i == c) ? tau[i] : Real(0);
    }
    __syncthreads();
    for (int s = 1; s < w; s *= 2) {
        const int s2 = 2 * s;
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int row = idx % w, col = idx / w;
            const int b1 = (row & ~(s2 - 1)) + s;
            if (row >= b1 || col < b1 || col >= b1 + s) continue;
            Real acc = Real(0);   // (G12 T22)(row, col)
            for (int l = b1; l <= col; ++l) acc = rfma(G[row + l * w], T[l + col * w], acc);
            M[idx] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int row = idx % w, col = idx / w;
            const int b1 = (row & ~(s2 - 1)) + s;
            if (row >= b1 || col < b1 || col >= b1 + s) continue;
            Real acc = Real(0);   // (T11 M)(row, col)
            for (int l = row; l < b1; ++l) acc = rfma(T[row + l * w], M[l + col * w], acc);
            T[idx] = -acc;
        }
        __syncthreads();
    }
}

// C = sign * A * B for upper triangular w x w A, B (ld w): C is upper
// triangular, its strict lower part is written as zero.
template <class Real>
__device__ void upper_upper(const Real *A, const Real *B, Real *C, int w, Real sign) {
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int i = idx % w, c = idx / w;
        Real s = Real(0);
        for (int l = i; l <= c; ++l) s = rfma(A[i + l * w], B[l + c * w], s);
        C[idx] = sign * s;
    }
}

// Inverse of the unit lower triangular L (ld w) into Li (ld w), blocked
// bottom-up like build_t: Li21 = -Li22 L21 Li11 for each pair of blocks.
template <class Real>
__device__ void unit_lower_inverse(const Real *L, Real *Li, Real *M, int w) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int i = idx % w, c = idx / w;
        Li[idx] = (i == c) ? Real(1) : Real(0);
    }
    __syncthreads();
    for (int s = 1; s < w; s *= 2) {
        const int s2 = 2 * s;
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int row = idx % w, col = idx / w;
            const int b1 = (col & ~(s2 - 1)) + s;   // pair (b0 = b1 - s, b1), col in block 0, row in block 1
            if (col >= b1 || row < b1 || row >= b1 + s) continue;
            Real acc = Real(0);   // (L21 Li11)(row, col)
            for (int l = col; l < b1; ++l) acc = rfma(L[row + l * w], Li[l + col * w], acc);
            M[idx] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int row = idx % w, col = idx / w;
            const int b1 = (col & ~(s2 - 1)) + s;
            if (col >= b1 || row < b1 || row >= b1 + s) continue;
            Real acc = M[idx];   // Li22(row,row) = 1
            for (int l = b1; l < row; ++l) acc = rfma(Li[row + l * w], M[l + col * w], acc);
            Li[idx] = -acc;
        }
        __syncthreads();
    }
}

// Z (over M) = T (V1^T B) for a leaf: V1 = the unit lower top w x w block of
// the leaf's V (entry (l, i), l > i, at V1[l * ld1v + i * ldv]), T upper (in
// M on entry), B upper; C is w x w scratch.  Z is upper triangular.
template <class Real>
__device__ void leaf_z(const Real *V1, int64_t ldv, const Real *B, Real *C, Real *M, int w) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < w * w; idx += nthr) {          // C = V1^T B (upper)
        const int i = idx % w, c = idx / w;
        Real s = Real(0);
        if (i <= c) {
            s = B[i + c * w];
            for (int l = i + 1; l <= c; ++l) s = rfma(V1[(size_t)i * ldv + l], B[l + c * w], s);
        }
        C[idx] = s;
    }
    __syncthreads();
    Real z2[(kMaxPanel * kMaxPanel + kThreads - 1) / kThreads];   // Z = T C, then over M
    int q = 0;
    for (int idx = tid; idx < w * w; idx += nthr, ++q) {
        const int i = idx % w, c = idx / w;
        Real s = Real(0);
        for (int l = i; l <= c; ++l) s = rfma(M[i + l * w], C[l + c * w], s);
        z2[q] = s;
    }
    __syncthreads();
    q = 0;
    for (int idx = tid; idx < w * w; idx += nthr, ++q) M[idx] = z2[q];
    __syncthreads();
}

}  // namespace
}  // namespace gbqr
