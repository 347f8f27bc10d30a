// TSQR base case of QR-EG (Algorithm 2, base case), restated for the SMs of
// one GPU (Section 5 and Appendix C).  Each CTA plays one of the paper's
// processors: it owns a contiguous block of the panel's rows.
//
//   tsqr_up_kernel     (Appendix C.1, upsweep): every CTA factors its m_p x w
//                      row block with Householder reflectors in shared memory
//                      (local-QR), keeps (V_p, T_p) and passes R_p up a
//                      fan-out-k tree.  The tree "Reduce" is fused into the
//                      same launch: the last CTA to arrive at a node (atomic
//                      arrival counter) factors the stacked upper triangles
//                      of its children; no CTA ever waits on another.
//   tsqr_down_kernel   (Appendix C.2, downsweep and reconstruction, one
//                      launch): every CTA walks from the root to leaf 0 and
//                      forms the top w x w block X of W = Q [I; 0] (from the
//                      copy of leaf 0's top V block the upsweep kept), factors
//                      X + S = LU with S_jj = sgn(X^_jj) added before
//                      eliminating column j, and inverts U.  It then walks to
//                      its own leaf applying the node Q-factors to
//                      B^(L) = U^{-1} instead of I - the shortcut noted at the
//                      end of Appendix C - so its rows of Q [U^{-1}; 0] are
//                      V_p = W_p U^{-1} directly, with no per-row triangular
//                      solve.  CTA 0 writes T = U S L^{-T}, V_top = L and
//                      R = -S R^(L).  The small LU and the walk to leaf 0 are
//                      repeated by every CTA instead of being broadcast, so
//                      the launch needs no inter-CTA waiting.
//
// Merged nodes exploit the structure of stacked triangles: the Householder
// vector of column j has a 1 in row j of the first triangle and non-zeros
// only in rows 0..j of the others, so V = [I; Y_1; ...] with each Y_i upper
// triangular and V^T [B; 0] = B in the downsweep.
#include "tsqr_dev.cuh"

#include <algorithm>
#include <atomic>

namespace gbqr {
namespace {

template <class Real>
struct TsqrParamsT {
    Real *A; int64_t lda;     // panel top-left, mp x w
    int64_t mp; int w;
    int P, k, L, ldS, ldW;
    Real *wsR, *wsT, *wsY, *wsX;
    unsigned *counters;
    Real *Tout; int64_t ldt;
};

// The cnt consecutive w x w slots at src (slot i, entry (row, col) at
// i w^2 + row + col w) stacked into S: slot i's entry goes to S(i w + row,
// col).  Up to 8 loads in flight per thread, as in load_block.
template <class Real>
__device__ __forceinline__ void load_stack(Real *S, int64_t ldS, const Real *src, int cnt, int w) {
    constexpr int kBatch = 8;
    const int tid = threadIdx.x, nthr = blockDim.x, ww = w * w, total = cnt * ww;
    for (int base = tid; base < total; base += kBatch * nthr) {
        Real v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int e = base + k * nthr;
            if (e < total) v[k] = __ldcg(src + e);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int e = base + k * nthr;
            if (e < total) {
                const int i = e / ww, rem = e - i * ww, col = rem / w, row = rem - col * w;
                S[(i * w + row) + (int64_t)col * ldS] = v[k];
            }
        }
    }
}

__device__ __forceinline__ int64_t leaf_begin(int64_t mp, int P, int p) { return (int64_t)p * mp / P; }

// Up kernel shared memory: S (ldS x w), then T, G (w x w each), then the
// per-column reflector data (Refl: tau, d, beta*d, q, 1/d, norm; w each).
template <class Real>
__global__ void __launch_bounds__(kThreads) tsqr_up_kernel(TsqrParamsT<Real> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *smem = reinterpret_cast<Real *>(smem_raw);
    const int w = p.w, ldS = p.ldS, tid = threadIdx.x, nthr = blockDim.x;
    Real *S = smem;
    Real *T = S + (size_t)ldS * w;
    Real *G = T + w * w;
    Real *aux = G + w * w;
    const Refl<Real> rf{aux, aux + w, aux + 2 * w, aux + 3 * w, aux + 4 * w, aux + 5 * w};
    __shared__ int s_last;

    const int leaf = blockIdx.x;
    const int64_t r0 = leaf_begin(p.mp, p.P, leaf), r1 = leaf_begin(p.mp, p.P, leaf + 1);
    const int h = (int)(r1 - r0);
    const size_t ww = (size_t)w * w;

    load_block(S, ldS, p.A + r0, p.lda, h, w);
    __syncthreads();
    householder_block(S, ldS, w, LeafRows{h}, rf, G);
    finish_block(S, ldS, w, rf, G);

    // V_p (strict lower, normalised here) and R_p (upper) back to the panel
    // rows, R_p to the tree; then T_p, with the leaf block's shared memory as
    // scratch.  Leaf 0 also keeps a copy of its top w x w block of V: every
    // CTA of the downsweep reads it to form X while CTA 0 overwrites those
    // rows of the panel.
    for (int c = 0; c < w; ++c) {
        const Real sc = rf.sc[c];
        for (int r = tid; r < h; r += nthr) {
            const Real x = S[(size_t)c * ldS + r];
            p.A[(r0 + r) + c * p.lda] = (r > c) ? x * sc : x;
        }
    }
    if (leaf == 0)
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            p.wsX[idx] = (i > c) ? S[(size_t)c * ldS + i] * rf.sc[c] : Real(0);
        }
    {
        Real *Rn = p.wsR + (size_t)leaf * ww;
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            Rn[idx] = (i <= c) ? S[(size_t)c * ldS + i] : Real(0);
        }
    }
    __syncthreads();
    build_t(T, G, rf.tau, S, w);
    {
        Real *Tn = p.wsT + (size_t)leaf * ww;
        for (int idx = tid; idx < w * w; idx += nthr) Tn[idx] = T[idx];
    }

    // Climb: the last of a node's children to arrive merges them.
    int node = leaf, Nl = p.P;
    int64_t off = 0, off_next = p.P;
    while (Nl > 1) {
        const int parent = node / p.k, first = parent * p.k;
        const int cnt = min(p.k, Nl - first);
        const int Nnext = (Nl + p.k - 1) / p.k;
        const int64_t pidx = off_next + parent;
        __threadfence();
        __syncthreads();
        if (cnt > 1) {
            if (tid == 0) {
                const unsigned prev = atomicAdd(&p.counters[pidx - p.P], 1u);
                s_last = (prev == (unsigned)(cnt - 1));
            }
            __syncthreads();
            if (!s_last) return;
            __threadfence();
            if (tid == 0) p.counters[pidx - p.P] = 0u;
            load_stack(S, ldS, p.wsR + (size_t)(off + first) * ww, cnt, w);   // the children's R, stacked
            __syncthreads();
            householder_block(S, ldS, w, MergeRows{w, cnt}, rf, G);
            finish_block(S, ldS, w, rf, G);
            Real *Rn = p.wsR + (size_t)pidx * ww, *Tn = p.wsT + (size_t)pidx * ww;
            Real *Yn = p.wsY + (size_t)(pidx - p.P) * (p.k - 1) * ww;
            for (int idx = tid; idx < w * w; idx += nthr) {
                const int i = idx % w, c = idx / w;
                Rn[idx] = (i <= c) ? S[(size_t)c * ldS + i] : Real(0);
            }
            for (int b = 1; b < cnt; ++b)
                for (int idx = tid; idx < w * w; idx += nthr) {
                    const int i = idx % w, c = idx / w;
                    Yn[(size_t)(b - 1) * ww + idx] = (i <= c) ? S[(size_t)c * ldS + b * w + i] * rf.sc[c] : Real(0);
                }
            __syncthreads();
            build_t(T, G, rf.tau, S, w);
            for (int idx = tid; idx < w * w; idx += nthr) Tn[idx] = T[idx];
        } else {
            // single child: the node is the identity, its R passes through
            const Real *Rc = p.wsR + (size_t)(off + node) * ww;
            Real *Rn = p.wsR + (size_t)pidx * ww;
            for (int idx = tid; idx < w * w; idx += nthr) Rn[idx] = Rc[idx];
        }
        node = parent;
        off = off_next;
        off_next += Nnext;
        Nl = Nnext;
    }
}

// B <- (the node Q-factors along the root-to-`target` path) applied to
// B = I at the root, or to the upper triangular Binit (Appendix C.2,
// downsweep): each node on the path gives its child [B_0; B_1; ...] =
// (I - V T V^T)[B; 0] = [B - T B; -Y_1 T B; ...].  T, Y and B are upper
// triangular, so B stays upper triangular and each product costs about
// w^3/6 multiply-adds.  C, M: w x w scratch.
template <class Real>
__device__ void walk_path(const TsqrParamsT<Real> &p, int target, Real *B, Real *C, Real *M, Real *Yb,
                          const Real *Binit = nullptr) {
    const int w = p.w, tid = threadIdx.x, nthr = blockDim.x;
    const int ww = w * w;
    constexpr int kPer = (kMaxPanel * kMaxPanel + kThreads - 1) / kThreads;   // entries per thread
    int anc[41], Nlev[41];
    int64_t offl[41];
    anc[0] = target; Nlev[0] = p.P; offl[0] = 0;
    for (int lv = 0; lv < p.L; ++lv) {
        anc[lv + 1] = anc[lv] / p.k;
        Nlev[lv + 1] = (Nlev[lv] + p.k - 1) / p.k;
        offl[lv + 1] = offl[lv] + Nlev[lv];
    }
    // the node above level lv merges cnt children; a single child passes through
    auto count = [&](int lv) { return min(p.k, Nlev[lv] - anc[lv + 1] * p.k); };
    auto next_merge = [&](int lv) {
        while (lv >= 0 && count(lv) == 1) --lv;
        return lv;
    };
    // the node's T and (for a child after the first) its Y block, staged in
    // registers so that the next level's loads overlap this level's products
    Real tn[kPer], yn[kPer];
    auto fetch = [&](int lv) {
        const int parent = anc[lv + 1], pos = anc[lv] - parent * p.k;
        const int64_t pidx = offl[lv + 1] + parent;
        const Real *Tn = p.wsT + (size_t)pidx * ww;
        const Real *Yn = p.wsY + ((size_t)(pidx - p.P) * (p.k - 1) + (pos > 0 ? pos - 1 : 0)) * ww;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int idx = tid + q * nthr;
            if (idx < ww) {
                tn[q] = __ldcg(Tn + idx);
                if (pos > 0) yn[q] = __ldcg(Yn + idx);
            }
        }
    };
    for (int idx = tid; idx < ww; idx += nthr) B[idx] = Binit ? Binit[idx] : ((idx % w == idx / w) ? Real(1) : Real(0));
    int cur = next_merge(p.L - 1);
    if (cur >= 0) fetch(cur);
    __syncthreads();
    while (cur >= 0) {
        const int pos = anc[cur] - anc[cur + 1] * p.k;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int idx = tid + q * nthr;
            if (idx < ww) {
                M[idx] = tn[q];
                if (pos > 0) Yb[idx] = yn[q];
            }
        }
        __syncthreads();
        const int nxt = next_merge(cur - 1);
        if (nxt >= 0) fetch(nxt);
        upper_upper(M, B, C, w, Real(1));          // C = T_node B
        __syncthreads();
        if (pos == 0) {
            for (int idx = tid; idx < ww; idx += nthr) B[idx] -= C[idx];
        } else {
            upper_upper(Yb, C, B, w, -Real(1));    // B = -Y_pos C
        }
        __syncthreads();
        cur = nxt;
    }
}

// Downsweep and reconstruction in one launch (Appendix C.2).  W = Q [I; 0]
// row block p is W_p = (I - V_p T_p V_p^T)[B_p; 0] with B_p from the path
// root -> leaf p.  The top block X of W (leaf 0's top rows) is formed by every
// CTA from leaf 0's path and the copy of leaf 0's top V block that the
// upsweep kept, so no CTA waits for another; then, in every CTA:
//   X + S = L U with S_jj = sgn(X^_jj) added before column j is eliminated;
//   V rows = W rows U^{-1} for this leaf's rows below the top w;
// and CTA 0 writes T = U S L^{-T}, V_top = L and R = -S R^(L) (R^(L) at the root).
template <class Real>
__global__ void __launch_bounds__(kThreads) tsqr_down_kernel(TsqrParamsT<Real> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *smem = reinterpret_cast<Real *>(smem_raw);
    const int w = p.w, ldS = p.ldW, tid = threadIdx.x, nthr = blockDim.x;
    const size_t ww = (size_t)w * w;
    Real *B = smem;          // w x w: B of the path walked
    Real *C = B + ww;        // w x w scratch
    Real *M = C + ww;        // w x w: T, then Z, then U^{-1}, then T_p and Z_p
    Real *X = M + ww;        // w x w: X, then L (strict lower) and U
    Real *Li = X + ww;       // w x w: leaf 0's top V block, then L^{-1}
    Real *Sg = Li + ww;      // w signs
    Real *rU = Sg + w;       // w reciprocals of diag(U)
    Real *Vs = rU + w;       // ldS x w: this leaf's rows of V, then of W and V

    const int leaf = blockIdx.x;
    // X = [B_0; 0] top rows - V0 Z0, V0 = leaf 0's unit lower top block
    walk_path(p, 0, B, C, M, X);                          // X is free until formed below
    for (int idx = tid; idx < w * w; idx += nthr) {
        Li[idx] = __ldcg(p.wsX + idx);
        M[idx] = __ldcg(p.wsT + idx);                        // T of leaf 0
    }
    __syncthreads();
    leaf_z(Li, w, B, C, M, w);
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int r = idx % w, c = idx / w;
        Real s = (r <= c) ? M[r + c * w] : Real(0);
        for (int i = 0; i < min(r, c + 1); ++i) s = rfma(Li[i * w + r], M[i + c * w], s);
        X[idx] = B[idx] - s;
    }
    __syncthreads();
    // X + S = L U.  Per step one thread adds the sign to the pivot and takes
    // its reciprocal; then every entry of the trailing block forms its own
    // multiplier l_i = X(i, j) / pivot and is updated in the same pass, the
    // multipliers going to C, so X's column j and row j are only read during
    // the step (two barriers per step).  C is free here.
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
            if (c == j) C[i + j * w] = l;
            else X[i + c * w] = rfma(-l, X[j + c * w], X[i + c * w]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int i = idx % w, c = idx / w;
        if (i > c) X[idx] = C[idx];                           // L below the diagonal
    }
    __syncthreads();
    // U^{-1} into M (Z of leaf 0 is no longer needed): the inverse of the
    // upper triangular matrix with strict upper part U and diagonal 1/rU,
    // which is what build_t computes from (G, tau)
    Real *Ui = M;
    build_t(Ui, X, rU, C, w);
    if (leaf == 0) {
        // T = U S L^{-T}: T(i, c) = sum_{l=i}^{c} U(i, l) S_l Li(c, l)
        unit_lower_inverse(X, Li, C, w);
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            Real t = Real(0);
            for (int l = i; l <= c; ++l) t = rfma(X[i + l * w] * Sg[l], (l == c) ? Real(1) : Li[c + l * w], t);
            p.Tout[i + c * p.ldt] = t;
        }
        __syncthreads();
        upper_upper(B, Ui, C, w, Real(1));                    // leaf 0: B_0 U^{-1}
        __syncthreads();
        for (int idx = tid; idx < w * w; idx += nthr) B[idx] = C[idx];
    } else {
        // from B^(L) = U^{-1}: the walk copies Ui into B before it first
        // stages a node's T in M; Li is free here
        walk_path(p, leaf, B, C, M, Li, Ui);
    }
    __syncthreads();

    // this leaf: V_p = (I - V_p T_p V_p^T)[B_p; 0] with B_p from B^(L) = U^{-1}
    const int64_t r0 = leaf_begin(p.mp, p.P, leaf), r1 = leaf_begin(p.mp, p.P, leaf + 1);
    const int h = (int)(r1 - r0);
    load_block(Vs, ldS, p.A + r0, p.lda, h, w);
    {
        const Real *Tp = p.wsT + (size_t)leaf * ww;
        for (int idx = tid; idx < w * w; idx += nthr) M[idx] = Tp[idx];
    }
    __syncthreads();
    leaf_z(Vs, ldS, B, C, M, w);
    for (int r = tid; r < h; r += nthr) {
        if (r0 + r < w) continue;                           // leaf 0's top block: L \ R below
        // V(r, c) = [B; 0](r, c) - sum_{i <= min(r, c)} Vhat(r, i) Z(i, c), in place, c descending
        for (int c = w - 1; c >= 0; --c) {
            Real s = (r <= c) ? M[r + c * w] : Real(0);
            const int iend = min(r, c + 1);
            for (int i = 0; i < iend; ++i) s = rfma(Vs[(size_t)i * ldS + r], M[i + c * w], s);
            Vs[(size_t)c * ldS + r] = ((r < w) ? B[r + c * w] : Real(0)) - s;
        }
    }
    __syncthreads();
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < h; r += nthr)
            if (r0 + r >= w) p.A[(r0 + r) + c * p.lda] = Vs[(size_t)c * ldS + r];
    if (leaf == 0) {
        // top block: L strictly below the diagonal, R = -S R^(L) on and above;
        // R^(L) sits in the last node slot (the root)
        int64_t nodes = p.P, Nl = p.P;
        while (Nl > 1) { Nl = (Nl + p.k - 1) / p.k; nodes += Nl; }
        const Real *RL = p.wsR + (size_t)(nodes - 1) * ww;
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            p.A[i + c * p.lda] = (i <= c) ? -Sg[i] * __ldcg(RL + idx) : X[i + c * w];
        }
    }
}

size_t up_smem(int ldS, int w) { return sizeof(double) * ((size_t)ldS * w + 2 * (size_t)w * w + 6 * (size_t)w); }
size_t down_smem(int ldS, int w) { return sizeof(double) * ((size_t)ldS * w + 5 * (size_t)w * w + 2 * w); }

constexpr size_t kSmemCap = 200 * 1024;
constexpr int kDefaultFanout = 8;
constexpr int kMaxFanout = 16;

}  // namespace

bool tsqr_plan(int64_t mp, int w, int leaf_rows, int fanout, int num_sms, TsqrPlan *plan) {
    if (w < 1 || w > kMaxPanel || mp < w) return false;
    TsqrPlan pl;
    pl.mp = mp; pl.w = w;
    // tallest leaf that every kernel's shared memory can hold
    const size_t cap_el = kSmemCap / sizeof(double);
    int64_t hcap = (int64_t)((cap_el - (2 * (size_t)w * w + 6 * (size_t)w)) / w);          // up
    hcap = std::min<int64_t>(hcap, (int64_t)((cap_el - 5 * (size_t)w * w - 2 * w) / w));   // down + recon
    if (hcap < w) return false;
    // default: about one leaf per SM (the leaf phase is the only one that
    // uses the whole GPU), but at least 128 rows - shorter panels then get
    // fewer leaves and one merge level less, which measured faster - and
    // never shorter than the panel is wide
    const int sms = num_sms > 0 ? num_sms : 152;
    int64_t target = leaf_rows > 0 ? leaf_rows : std::max<int64_t>({(int64_t)w, (int64_t)128, (mp + sms - 1) / sms});
    // ... and up to 256 rows where that saves a whole merge level (17 to 32
    // leaves of 128 rows become 16 of at most 256: one merge instead of two)
    if (leaf_rows <= 0 && target == 128 && (mp + 127) / 128 > kMaxFanout && (mp + kMaxFanout - 1) / kMaxFanout <= 256)
        target = (mp + kMaxFanout - 1) / kMaxFanout;
    target = std::max<int64_t>(target, w);
    int64_t P = (mp + target - 1) / target;
    P = std::max<int64_t>(P, (mp + hcap - 1) / hcap);   // leaves no taller than hcap
    P = std::min<int64_t>(P, mp / w);                    // every leaf keeps >= w rows
    P = std::max<int64_t>(P, 1);
    if (P > (1 << 24)) return false;
    pl.P = (int)P;
    pl.hmax = (int)((mp + P - 1) / P);
    if (pl.hmax > hcap) return false;
    // fan-out: as requested (2 .. 16), else the fewest serial merge levels a
    // fan-out of at most 16 gives, with the smallest such k >= 8: a level
    // costs a fixed chain of w Householder steps, while a merge grows only
    // with the k - 1 stacked triangles below its pivots.  The merge of k
    // stacked triangles (k*w rows) must fit the up kernel's shared memory.
    auto levels = [&](int kk) { int64_t n = P; int l = 0; while (n > 1) { n = (n + kk - 1) / kk; ++l; } return l; };
    int k = kDefaultFanout;
    if (fanout > 0) {
        k = std::min(kMaxFanout, std::max(2, fanout));
    } else {
        for (int c = kDefaultFanout + 1; c <= kMaxFanout; ++c)
            if (levels(c) < levels(k)) k = c;
    }
    while (k > 2 && up_smem(k * w, w) > kSmemCap) --k;
    pl.k = k;
    pl.ldS = std::max(pl.hmax, pl.k * w);   // up kernel (leaf block or k stacked triangles)
    pl.ldW = pl.hmax;                        // down kernel (leaf block only)
    int64_t nodes = P, Nl = P, L = 0, internal = 0;
    while (Nl > 1) { Nl = (Nl + pl.k - 1) / pl.k; nodes += Nl; internal += Nl; ++L; }
    if (L > 40) return false;
    pl.L = (int)L;
    pl.nodes = nodes;
    const size_t ww = (size_t)w * w;
    pl.nR = (size_t)nodes * ww;
    pl.nT = (size_t)nodes * ww;
    pl.nY = (size_t)std::max<int64_t>(internal, 1) * (pl.k - 1) * ww;
    pl.nX = ww;
    pl.ncount = (size_t)std::max<int64_t>(internal, 1);
    pl.smem_up = up_smem(pl.ldS, w);
    pl.smem_down = down_smem(pl.ldW, w);
    if (pl.smem_up > kSmemCap || pl.smem_down > kSmemCap) return false;
    *plan = pl;
    return true;
}

TsqrPlan tsqr_plan_bound(int64_t mp, int w, int leaf_rows, int fanout, int num_sms) {
    // Workspace grows with the number of leaves P.  For panels of height
    // <= mp and width ww <= w: with an explicit leaf height P grows with the
    // height; with the default (about one leaf per SM) a shorter panel can
    // round to more leaves, but never to more than the SM count.  Take the
    // larger of the two counts, then the node counts of a tree that size.
    TsqrPlan best;
    const int sms = num_sms > 0 ? num_sms : 152;
    for (int ww = 1; ww <= w; ++ww) {
        TsqrPlan pl;
        if (mp < ww || !tsqr_plan(mp, ww, leaf_rows, fanout, num_sms, &pl)) continue;
        int64_t P = pl.P;
        if (leaf_rows <= 0) P = std::max<int64_t>(P, std::min<int64_t>(sms, mp / ww));
        // a shorter panel may get another fan-out: bound over all of them
        const size_t w2 = (size_t)ww * ww;
        for (int k = 2; k <= kMaxFanout; ++k) {
            int64_t nodes = P, Nl = P, internal = 0;
            while (Nl > 1) { Nl = (Nl + k - 1) / k; nodes += Nl; internal += Nl; }
            best.nR = std::max(best.nR, (size_t)nodes * w2);
            best.nT = std::max(best.nT, (size_t)nodes * w2);
            best.nY = std::max(best.nY, (size_t)std::max<int64_t>(internal, 1) * (k - 1) * w2);
            best.ncount = std::max(best.ncount, (size_t)std::max<int64_t>(internal, 1));
        }
        best.nX = std::max(best.nX, w2);
    }
    return best;
}

template <class Real>
gbqr_status tsqr_run(const Exec &ex, const TsqrPlan &pl, Real *A, int64_t lda,
                     Real *Tout, int64_t ldt, const TsqrWorkT<Real> &work) {
    TsqrParamsT<Real> p;
    p.A = A; p.lda = lda; p.mp = pl.mp; p.w = pl.w;
    p.P = pl.P; p.k = pl.k; p.L = pl.L; p.ldS = pl.ldS; p.ldW = pl.ldW;
    p.wsR = work.R; p.wsT = work.T; p.wsY = work.Y; p.wsX = work.X;
    p.counters = work.counters;
    p.Tout = Tout; p.ldt = ldt;

    // per device and scalar type, once (server workers launch from several threads)
    static std::atomic<bool> attr_done[64];
    if (!(ex.device >= 0 && ex.device < 64) || !attr_done[ex.device].load(std::memory_order_acquire)) {
        const int cap = (int)kSmemCap;
        if (cudaFuncSetAttribute(tsqr_up_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
            cudaFuncSetAttribute(tsqr_down_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess)
            return GBQR_ECUDA;
        if (ex.device >= 0 && ex.device < 64) attr_done[ex.device].store(true, std::memory_order_release);
    }
    const double w = pl.w, mp = (double)pl.mp;
    const double ww = w * w;
    gbqr_status st;

    trace_begin(ex, FAM_TSQR_UP);
    tsqr_up_kernel<Real><<<pl.P, kThreads, pl.smem_up, ex.stream>>>(p);
    // leaf Householder ~2 m w^2 + T ~ m w^2; merges ~ (nodes) * w^3
    st = trace_end(ex, FAM_TSQR_UP, 3.0 * mp * ww + (double)(pl.nodes - pl.P) * 1.5 * ww * w,
                   (double)sizeof(Real) * (2.0 * mp * w + 3.0 * (double)pl.nodes * ww));
    if (st != GBQR_OK) return st;

    trace_begin(ex, FAM_TSQR_DOWN);
    tsqr_down_kernel<Real><<<pl.P, kThreads, pl.smem_down, ex.stream>>>(p);
    // per leaf: two path walks (~2 L products of w^3/6 each), X, its LU and
    // U^{-1} (~2 w^3/3), and the leaf's rows of Q [U^{-1}; 0] (~m_p w^2)
    st = trace_end(ex, FAM_TSQR_DOWN,
                   2.0 * mp * ww + (double)pl.P * ((4.0 * pl.L + 4.0) * ww * w / 3.0),
                   (double)sizeof(Real) * (2.0 * mp * w + 2.0 * (double)pl.nodes * ww));
    return st;
}

template gbqr_status tsqr_run<double>(const Exec &, const TsqrPlan &, double *, int64_t, double *, int64_t,
                                     const TsqrWorkT<double> &);
template gbqr_status tsqr_run<float>(const Exec &, const TsqrPlan &, float *, int64_t, float *, int64_t,
                                    const TsqrWorkT<float> &);

}  // namespace gbqr
