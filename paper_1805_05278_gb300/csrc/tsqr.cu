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
//   tsqr_down_kernel   (Appendix C.2, downsweep): every CTA walks from the
//                      root to its leaf applying the node Q-factors to
//                      B^(L) = I, then forms its rows W_p of the leading w
//                      columns of Q.
//   tsqr_recon_kernel  (Appendix C.2, reconstruction): X + S = LU of the top
//                      w x w block of W with S_jj = sgn(X^_jj) added before
//                      eliminating column j; T = U S L^{-T}, R = -S R^(L),
//                      V_top = L, and V_p = W_p U^{-1} for every other row.
//                      The small LU is repeated by every CTA instead of being
//                      broadcast, so the launch needs no inter-CTA waiting.
//
// Merged nodes exploit the structure of stacked triangles: the Householder
// vector of column j has a 1 in row j of the first triangle and non-zeros
// only in rows 0..j of the others, so V = [I; Y_1; ...] with each Y_i upper
// triangular and V^T [B; 0] = B in the downsweep.
#include "common.cuh"

#include <algorithm>

namespace gbqr {
namespace {

struct TsqrParams {
    double *A; int64_t lda;     // panel top-left, mp x w
    int64_t mp; int w;
    int P, k, L, ldS, ldW;
    double *wsR, *wsT, *wsY, *wsX;
    unsigned *counters;
    double *Tout; int64_t ldt;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; every thread receives the same value (fixed order).
__device__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__device__ __forceinline__ int64_t leaf_begin(int64_t mp, int P, int p) { return (int64_t)p * mp / P; }

// Rows of column j below its pivot in a leaf block: j+1 .. h-1.
struct LeafRows {
    int h;
    __device__ int count(int j) const { return h - j - 1; }
    __device__ int row(int j, int idx) const { return j + 1 + idx; }
};

// Rows of column j below its pivot in cnt stacked w x w upper triangles:
// rows 0..j of every triangle after the first.
struct MergeRows {
    int w, cnt;
    __device__ int count(int j) const { return (cnt - 1) * (j + 1); }
    __device__ int row(int j, int idx) const {
        const int i = idx / (j + 1);
        return (i + 1) * w + (idx - i * (j + 1));
    }
};

// Householder QR of the w columns held in shared memory S (column-major,
// leading dimension ldS), column j acting on its pivot row j and the rows
// that `rows` lists.  On return: R on and above the pivots, the vectors'
// entries below them (unit pivot implied), tau[0:w], and T (w x w, ld w,
// zero below the diagonal) by the forward recurrence
// T(0:j, j) = -tau_j T(0:j, 0:j) (V(:, 0:j)^T v_j).  The inner products
// v_c^T v_j for c < j come from the same pass that updates columns c > j.
// Sign convention: beta = -sgn(alpha) * ||column||, sgn(0) = +1; a zero
// column gives v = e_j, tau = 2.
template <class Rows>
__device__ void householder_block(double *S, int ldS, int w, Rows rows, double *tau, double *T,
                                  double *red, double *z) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nthr = blockDim.x, nw = nthr >> 5;
    for (int i = tid; i < w * w; i += nthr) T[i] = 0.0;
    for (int j = 0; j < w; ++j) {
        const int cnt = rows.count(j);
        double *colj = S + (size_t)j * ldS;
        double part = 0.0;
        for (int idx = tid; idx < cnt; idx += nthr) {
            const double x = colj[rows.row(j, idx)];
            part = fma(x, x, part);
        }
        const double sig2 = block_sum(part, red);   // ends with __syncthreads
        const double alpha = colj[j];
        const double nrm = sqrt(fma(alpha, alpha, sig2));
        const double beta = alpha < 0.0 ? nrm : -nrm;
        double tj, scal;
        if (beta == 0.0) { tj = 2.0; scal = 0.0; }
        else { tj = (beta - alpha) / beta; scal = 1.0 / (alpha - beta); }
        __syncthreads();   // every thread has read alpha
        if (tid == 0) { colj[j] = beta; tau[j] = tj; }
        if (beta != 0.0)
            for (int idx = tid; idx < cnt; idx += nthr) colj[rows.row(j, idx)] *= scal;
        __syncthreads();
        // one warp per other column: s_c = A(j,c) + sum_r v_j(r) A(r,c)
        for (int c = wid; c < w; c += nw) {
            if (c == j) continue;
            double *colc = S + (size_t)c * ldS;
            double d = 0.0;
            for (int idx = lane; idx < cnt; idx += 32) {
                const int r = rows.row(j, idx);
                d = fma(colj[r], colc[r], d);
            }
            d = warp_sum(d) + colc[j];
            __syncwarp();
            if (c > j) {
                const double f = tj * d;
                if (lane == 0) colc[j] -= f;
                for (int idx = lane; idx < cnt; idx += 32) {
                    const int r = rows.row(j, idx);
                    colc[r] = fma(-f, colj[r], colc[r]);
                }
            } else if (lane == 0) {
                z[c] = d;
            }
        }
        __syncthreads();
        for (int i = tid; i <= j; i += nthr) {
            double tv = tj;
            if (i < j) {
                double s = 0.0;
                for (int l = i; l < j; ++l) s = fma(T[i + l * w], z[l], s);
                tv = -tj * s;
            }
            T[i + j * w] = tv;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) tsqr_up_kernel(TsqrParams p) {
    extern __shared__ double smem[];
    const int w = p.w, ldS = p.ldS, tid = threadIdx.x, nthr = blockDim.x;
    double *S = smem;
    double *T = S + (size_t)ldS * w;
    double *tau = T + w * w;
    double *z = tau + w;
    double *red = z + w;
    __shared__ int s_last;

    const int leaf = blockIdx.x;
    const int64_t r0 = leaf_begin(p.mp, p.P, leaf), r1 = leaf_begin(p.mp, p.P, leaf + 1);
    const int h = (int)(r1 - r0);
    const size_t ww = (size_t)w * w;

    for (int c = 0; c < w; ++c)
        for (int r = tid; r < h; r += nthr) S[(size_t)c * ldS + r] = p.A[(r0 + r) + c * p.lda];
    __syncthreads();
    householder_block(S, ldS, w, LeafRows{h}, tau, T, red, z);

    // V_p (strict lower) and R_p (upper) back to the panel rows; T_p, R_p to the tree.
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < h; r += nthr) p.A[(r0 + r) + c * p.lda] = S[(size_t)c * ldS + r];
    {
        double *Rn = p.wsR + (size_t)leaf * ww, *Tn = p.wsT + (size_t)leaf * ww;
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            Rn[idx] = (i <= c) ? S[(size_t)c * ldS + i] : 0.0;
            Tn[idx] = T[idx];
        }
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
            for (int i = 0; i < cnt; ++i) {
                const double *Rc = p.wsR + (size_t)(off + first + i) * ww;
                for (int idx = tid; idx < w * w; idx += nthr)
                    S[(size_t)(idx / w) * ldS + i * w + (idx % w)] = __ldcg(Rc + idx);
            }
            __syncthreads();
            householder_block(S, ldS, w, MergeRows{w, cnt}, tau, T, red, z);
            double *Rn = p.wsR + (size_t)pidx * ww, *Tn = p.wsT + (size_t)pidx * ww;
            double *Yn = p.wsY + (size_t)(pidx - p.P) * (p.k - 1) * ww;
            for (int idx = tid; idx < w * w; idx += nthr) {
                const int i = idx % w, c = idx / w;
                Rn[idx] = (i <= c) ? S[(size_t)c * ldS + i] : 0.0;
                Tn[idx] = T[idx];
            }
            for (int b = 1; b < cnt; ++b)
                for (int idx = tid; idx < w * w; idx += nthr) {
                    const int i = idx % w, c = idx / w;
                    Yn[(size_t)(b - 1) * ww + idx] = (i <= c) ? S[(size_t)c * ldS + b * w + i] : 0.0;
                }
        } else {
            // single child: the node is the identity, its R passes through
            const double *Rc = p.wsR + (size_t)(off + node) * ww;
            double *Rn = p.wsR + (size_t)pidx * ww;
            for (int idx = tid; idx < w * w; idx += nthr) Rn[idx] = Rc[idx];
        }
        node = parent;
        off = off_next;
        off_next += Nnext;
        Nl = Nnext;
    }
}

// C = Tri * B for w x w matrices in shared memory (ld w); Tri upper triangular.
__device__ void upper_times(const double *Tri, const double *B, double *C, int w, double sign) {
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
        const int i = idx % w, c = idx / w;
        double s = 0.0;
        for (int l = i; l < w; ++l) s = fma(Tri[i + l * w], B[l + c * w], s);
        C[idx] = sign * s;
    }
}

__global__ void __launch_bounds__(kThreads) tsqr_down_kernel(TsqrParams p) {
    extern __shared__ double smem[];
    const int w = p.w, ldS = p.ldW, tid = threadIdx.x, nthr = blockDim.x;
    const size_t ww = (size_t)w * w;
    double *B = smem;
    double *C = B + ww;
    double *M = C + ww;      // node T, then node Y / leaf T_p
    double *Vs = M + ww;     // leaf block, ldS x w

    const int leaf = blockIdx.x;
    const int64_t r0 = leaf_begin(p.mp, p.P, leaf), r1 = leaf_begin(p.mp, p.P, leaf + 1);
    const int h = (int)(r1 - r0);

    // ancestors and level sizes (L <= 40)
    int anc[41], Nlev[41];
    int64_t offl[41];
    anc[0] = leaf; Nlev[0] = p.P; offl[0] = 0;
    for (int lv = 0; lv < p.L; ++lv) {
        anc[lv + 1] = anc[lv] / p.k;
        Nlev[lv + 1] = (Nlev[lv] + p.k - 1) / p.k;
        offl[lv + 1] = offl[lv] + Nlev[lv];
    }
    for (int idx = tid; idx < w * w; idx += nthr) B[idx] = (idx % w == idx / w) ? 1.0 : 0.0;
    __syncthreads();
    for (int lv = p.L - 1; lv >= 0; --lv) {
        const int parent = anc[lv + 1], first = parent * p.k;
        const int cnt = min(p.k, Nlev[lv] - first);
        if (cnt == 1) continue;
        const int pos = anc[lv] - first;
        const int64_t pidx = offl[lv + 1] + parent;
        const double *Tn = p.wsT + (size_t)pidx * ww;
        for (int idx = tid; idx < w * w; idx += nthr) M[idx] = Tn[idx];
        __syncthreads();
        upper_times(M, B, C, w, 1.0);          // C = T_node B
        __syncthreads();
        if (pos == 0) {
            for (int idx = tid; idx < w * w; idx += nthr) B[idx] -= C[idx];
        } else {
            const double *Yn = p.wsY + ((size_t)(pidx - p.P) * (p.k - 1) + (pos - 1)) * ww;
            for (int idx = tid; idx < w * w; idx += nthr) M[idx] = Yn[idx];
            __syncthreads();
            upper_times(M, C, B, w, -1.0);     // B = -Y_pos C
        }
        __syncthreads();
    }

    // leaf: W_p = (I - V_p T_p V_p^T) [B; 0]
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < h; r += nthr) Vs[(size_t)c * ldS + r] = p.A[(r0 + r) + c * p.lda];
    {
        const double *Tp = p.wsT + (size_t)leaf * ww;
        for (int idx = tid; idx < w * w; idx += nthr) M[idx] = Tp[idx];
    }
    __syncthreads();
    // C = V1^T B, V1 = unit lower top w x w of the leaf block
    for (int idx = tid; idx < w * w; idx += nthr) {
        const int i = idx % w, c = idx / w;
        double s = B[i + c * w];
        for (int l = i + 1; l < w; ++l) s = fma(Vs[(size_t)i * ldS + l], B[l + c * w], s);
        C[idx] = s;
    }
    __syncthreads();
    // B stays; reuse M <- T_p C  (need a temp: write into Vs? no - use C2 in place of T)
    {
        // compute Z2 = T_p * C into registers then overwrite M after a barrier
        double z2[(kMaxPanel * kMaxPanel + kThreads - 1) / kThreads];
        int q = 0;
        for (int idx = tid; idx < w * w; idx += nthr, ++q) {
            const int i = idx % w, c = idx / w;
            double s = 0.0;
            for (int l = i; l < w; ++l) s = fma(M[i + l * w], C[l + c * w], s);
            z2[q] = s;
        }
        __syncthreads();
        q = 0;
        for (int idx = tid; idx < w * w; idx += nthr, ++q) M[idx] = z2[q];
    }
    __syncthreads();
    // W(r, c) = [B; 0](r, c) - sum_{i <= min(r, w-1)} Vhat(r, i) Z2(i, c)
    for (int idx = tid; idx < h * w; idx += nthr) {
        const int r = idx % h, c = idx / h;
        double s = 0.0;
        const int imax = min(r, w - 1);
        for (int i = 0; i < imax; ++i) s = fma(Vs[(size_t)i * ldS + r], M[i + c * w], s);
        // i == imax: unit diagonal if r < w, stored entry otherwise
        s += (r < w ? 1.0 : Vs[(size_t)imax * ldS + r]) * M[imax + c * w];
        const double bw = (r < w) ? B[r + c * w] : 0.0;
        const double wv = bw - s;
        p.A[(r0 + r) + c * p.lda] = wv;
        if (leaf == 0 && r < w) p.wsX[r + c * w] = wv;
    }
}

__global__ void __launch_bounds__(kThreads) tsqr_recon_kernel(TsqrParams p) {
    extern __shared__ double smem[];
    const int w = p.w, ldS = p.ldW, tid = threadIdx.x, nthr = blockDim.x;
    const size_t ww = (size_t)w * w;
    double *X = smem;            // w x w: L (strict lower) and U (upper)
    double *Tm = X + ww;         // w x w
    double *Sg = Tm + ww;        // w signs
    double *rU = Sg + w;         // w reciprocals of diag(U)
    double *Wb = rU + w;         // ldS x w

    for (int idx = tid; idx < w * w; idx += nthr) X[idx] = __ldcg(p.wsX + idx);
    __syncthreads();
    // X + S = L U, S_jj = sgn(X^_jj) added before column j is eliminated.
    for (int j = 0; j < w; ++j) {
        if (tid == 0) {
            const double s = X[j + j * w] < 0.0 ? -1.0 : 1.0;
            Sg[j] = s;
            X[j + j * w] += s;
        }
        __syncthreads();
        const double piv = X[j + j * w];
        for (int i = j + 1 + tid; i < w; i += nthr) X[i + j * w] /= piv;
        __syncthreads();
        const int rem = w - j - 1;
        for (int idx = tid; idx < rem * rem; idx += nthr) {
            const int i = j + 1 + idx % rem, c = j + 1 + idx / rem;
            X[i + c * w] = fma(-X[i + j * w], X[j + c * w], X[i + c * w]);
        }
        __syncthreads();
    }
    for (int j = tid; j < w; j += nthr) rU[j] = 1.0 / X[j + j * w];

    const int leaf = blockIdx.x;
    if (leaf == 0) {
        // T = U S L^{-T}:  T(:, j) = U(:, j) S_j - sum_{l<j} L(j, l) T(:, l); thread i owns row i.
        for (int i = tid; i < w; i += nthr) {
            for (int j = 0; j < w; ++j) {
                double t = 0.0;
                if (i <= j) {
                    t = X[i + j * w] * Sg[j];
                    for (int l = i; l < j; ++l) t = fma(-X[j + l * w], Tm[i + l * w], t);
                }
                Tm[i + j * w] = t;
            }
        }
        __syncthreads();
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            p.Tout[i + c * p.ldt] = Tm[idx];
        }
        // top block of the panel: L strictly below the diagonal, R = -S R^(L)
        // on and above it; R^(L) sits in the last node slot (the root).
        int64_t nodes = p.P, Nl = p.P;
        while (Nl > 1) { Nl = (Nl + p.k - 1) / p.k; nodes += Nl; }
        const double *RL = p.wsR + (size_t)(nodes - 1) * ww;
        for (int idx = tid; idx < w * w; idx += nthr) {
            const int i = idx % w, c = idx / w;
            p.A[i + c * p.lda] = (i <= c) ? -Sg[i] * __ldcg(RL + idx) : X[i + c * w];
        }
    }
    __syncthreads();

    // V rows: V(r, :) = W(r, :) U^{-1} for the rows of this leaf below the top w.
    const int64_t r0 = leaf_begin(p.mp, p.P, leaf), r1 = leaf_begin(p.mp, p.P, leaf + 1);
    const int64_t rs = max(r0, (int64_t)w);
    const int h = (int)max((int64_t)0, r1 - rs);
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < h; r += nthr) Wb[(size_t)c * ldS + r] = p.A[(rs + r) + c * p.lda];
    __syncthreads();
    for (int r = tid; r < h; r += nthr) {
        for (int j = 0; j < w; ++j) {
            double v = Wb[(size_t)j * ldS + r];
            for (int l = 0; l < j; ++l) v = fma(-Wb[(size_t)l * ldS + r], X[l + j * w], v);
            Wb[(size_t)j * ldS + r] = v * rU[j];
        }
    }
    __syncthreads();
    for (int c = 0; c < w; ++c)
        for (int r = tid; r < h; r += nthr) p.A[(rs + r) + c * p.lda] = Wb[(size_t)c * ldS + r];
}

size_t up_smem(int ldS, int w) { return sizeof(double) * ((size_t)ldS * w + (size_t)w * w + 2 * w + 32); }
size_t down_smem(int ldS, int w) { return sizeof(double) * ((size_t)ldS * w + 3 * (size_t)w * w); }
size_t recon_smem(int ldS, int w) { return sizeof(double) * ((size_t)ldS * w + 2 * (size_t)w * w + 2 * w); }

constexpr size_t kSmemCap = 200 * 1024;

}  // namespace

bool tsqr_plan(int64_t mp, int w, int leaf_rows, int fanout, int num_sms, TsqrPlan *plan) {
    (void)num_sms;
    if (w < 1 || w > kMaxPanel || mp < w) return false;
    TsqrPlan pl;
    pl.mp = mp; pl.w = w;
    // fan-out: as requested, but the merge of k stacked triangles (k*w rows)
    // must fit the up kernel's shared memory
    int k = std::min(8, std::max(2, fanout > 0 ? fanout : 2));
    while (k > 2 && up_smem(k * w, w) > kSmemCap) --k;
    pl.k = k;
    // tallest leaf that every kernel's shared memory can hold
    const size_t cap_el = kSmemCap / sizeof(double);
    int64_t hcap = (int64_t)((cap_el - ((size_t)w * w + 2 * w + 32)) / w);                 // up
    hcap = std::min<int64_t>(hcap, (int64_t)((cap_el - 3 * (size_t)w * w) / w));           // down
    hcap = std::min<int64_t>(hcap, (int64_t)((cap_el - 2 * (size_t)w * w - 2 * w) / w));   // recon
    if (hcap < w) return false;
    int64_t target = leaf_rows > 0 ? leaf_rows : std::max<int64_t>(2 * w, 64);
    target = std::max<int64_t>(target, w);
    int64_t P = (mp + target - 1) / target;
    P = std::max<int64_t>(P, (mp + hcap - 1) / hcap);   // leaves no taller than hcap
    P = std::min<int64_t>(P, mp / w);                    // every leaf keeps >= w rows
    P = std::max<int64_t>(P, 1);
    if (P > (1 << 24)) return false;
    pl.P = (int)P;
    pl.hmax = (int)((mp + P - 1) / P);
    if (pl.hmax > hcap) return false;
    pl.ldS = std::max(pl.hmax, pl.k * w);   // up kernel (leaf block or k stacked triangles)
    pl.ldW = pl.hmax;                        // down / recon kernels (leaf block only)
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
    pl.smem_recon = recon_smem(pl.ldW, w);
    if (pl.smem_up > kSmemCap || pl.smem_down > kSmemCap || pl.smem_recon > kSmemCap) return false;
    *plan = pl;
    return true;
}

TsqrPlan tsqr_plan_bound(int64_t mp, int w, int leaf_rows, int fanout, int num_sms) {
    // Workspace grows with the number of leaves, which grows with mp and
    // shrinks with w: take the element-wise maximum over widths 1..w at mp.
    TsqrPlan best;
    for (int ww = 1; ww <= w; ++ww) {
        TsqrPlan pl;
        if (mp < ww || !tsqr_plan(mp, ww, leaf_rows, fanout, num_sms, &pl)) continue;
        best.nR = std::max(best.nR, pl.nR);
        best.nT = std::max(best.nT, pl.nT);
        best.nY = std::max(best.nY, pl.nY);
        best.nX = std::max(best.nX, pl.nX);
        best.ncount = std::max(best.ncount, pl.ncount);
    }
    return best;
}

gbqr_status tsqr_run(const Exec &ex, const TsqrPlan &pl, double *A, int64_t lda,
                     double *Tout, int64_t ldt, const TsqrWork &work) {
    TsqrParams p;
    p.A = A; p.lda = lda; p.mp = pl.mp; p.w = pl.w;
    p.P = pl.P; p.k = pl.k; p.L = pl.L; p.ldS = pl.ldS; p.ldW = pl.ldW;
    p.wsR = work.R; p.wsT = work.T; p.wsY = work.Y; p.wsX = work.X;
    p.counters = work.counters;
    p.Tout = Tout; p.ldt = ldt;

    static bool attr_done[64] = {false};
    if (ex.device >= 0 && ex.device < 64 && !attr_done[ex.device]) {
        const int cap = (int)kSmemCap;
        if (cudaFuncSetAttribute(tsqr_up_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
            cudaFuncSetAttribute(tsqr_down_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess ||
            cudaFuncSetAttribute(tsqr_recon_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess)
            return GBQR_ECUDA;
        attr_done[ex.device] = true;
    }
    const double w = pl.w, mp = (double)pl.mp;
    const double ww = w * w;
    gbqr_status st;

    trace_begin(ex, FAM_TSQR_UP);
    tsqr_up_kernel<<<pl.P, kThreads, pl.smem_up, ex.stream>>>(p);
    // leaf Householder ~2 m w^2 + T ~ m w^2; merges ~ (nodes) * w^3
    st = trace_end(ex, FAM_TSQR_UP, 3.0 * mp * ww + (double)(pl.nodes - pl.P) * 1.5 * ww * w,
                   8.0 * (2.0 * mp * w + 3.0 * (double)pl.nodes * ww));
    if (st != GBQR_OK) return st;

    trace_begin(ex, FAM_TSQR_DOWN);
    tsqr_down_kernel<<<pl.P, kThreads, pl.smem_down, ex.stream>>>(p);
    st = trace_end(ex, FAM_TSQR_DOWN, 2.0 * mp * ww + (double)pl.P * (2.0 * pl.L + 2.0) * ww * w,
                   8.0 * (2.0 * mp * w + 2.0 * (double)pl.nodes * ww));
    if (st != GBQR_OK) return st;

    trace_begin(ex, FAM_TSQR_RECON);
    tsqr_recon_kernel<<<pl.P, kThreads, pl.smem_recon, ex.stream>>>(p);
    st = trace_end(ex, FAM_TSQR_RECON, mp * ww + (double)pl.P * ww * w * 2.0 / 3.0,
                   8.0 * (2.0 * mp * w + 2.0 * ww));
    return st;
}

}  // namespace gbqr
