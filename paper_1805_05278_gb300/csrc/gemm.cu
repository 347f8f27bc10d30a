// FP64 GEMM for the update and T-assembly products of QR-EG (Algorithm 2):
//   M1 = V_L^T A_R,  M2 = T_L^T M1,  A_R -= V_L M2          (update)
//   M3 = V_L^T [0; V_R],  M4 = M3 T_R,  T12 = -T_L M4        (T assembly)
// and the same three-product update for the right-looking top level
// (Section 8.4) and for applying Q (basis-kernel update, Section 2.3).
//
// The operands carry structure that the paper's analysis deliberately
// ignores (Section 2.3) but that costs real FP64 cycles here: V is unit lower
// trapezoidal and T upper triangular.  The kernel masks them while staging
// tiles and trims each tile's K range to the rows/columns that can be
// non-zero, so triangular products cost about half of a dense one.
//
// Tall inner products (K = m, small M x N output) are split over K across
// CTAs - the in-GPU form of the paper's K-split 1DMM followed by a Reduce
// (Section 4, Lemma 3).  The partial tiles are summed by a fixed-shape tree
// of "last CTA to arrive" reductions (fan-in 8): no CTA ever waits on
// another, and the summation order is fixed, so results are deterministic.
#include "common.cuh"

#include <algorithm>
#include <type_traits>

namespace gbqr {
namespace {

constexpr int BK = 16;
constexpr int kGroup = 8;   // fan-in of the split-K reduction tree

template <class Real>
struct GemmParamsT {
    int64_t M, N, K;
    const Real *A; int64_t lda; int maskA;
    const Real *B; int64_t ldb; int maskB;
    Real *C; int64_t ldc;
    Real alpha, beta;
    Real *partial;            // per tile: slots_per_tile * BM*BN elements
    unsigned *counters;       // per tile: counters_per_tile
    int slots_per_tile, counters_per_tile;
};
using GemmParams = GemmParamsT<double>;

__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }

template <class Real>
__device__ __forceinline__ Real masked(const Real *X, int64_t ld, int64_t r, int64_t c, int mask) {
    if (mask == MASK_UNIT_LOWER) {
        if (r < c) return Real(0);
        if (r == c) return Real(1);
    } else if (mask == MASK_UPPER) {
        if (r > c) return Real(0);
    }
    return X[r + c * ld];
}

// K range [kb, ke) outside which op(A)(i, k) or op(B)(k, j) is structurally
// zero for every i in [m0, m0+BM) and j in [n0, n0+BN).
template <class P>
__device__ __forceinline__ void k_range(const P &p, bool ta, int64_t m0, int64_t n0,
                                        int BM, int BN, int64_t &kb, int64_t &ke) {
    kb = 0; ke = p.K;
    if (p.maskA == MASK_UNIT_LOWER) {
        if (!ta) ke = min(ke, m0 + BM);   // A(i,k) != 0 needs k <= i
        else kb = max(kb, m0);            // A(k,i) != 0 needs k >= i
    } else if (p.maskA == MASK_UPPER) {
        if (!ta) kb = max(kb, m0);        // A(i,k) != 0 needs k >= i
        else ke = min(ke, m0 + BM);       // A(k,i) != 0 needs k <= i
    }
    if (p.maskB == MASK_UNIT_LOWER) kb = max(kb, n0);       // B(k,j) != 0 needs k >= j
    else if (p.maskB == MASK_UPPER) ke = min(ke, n0 + BN);  // B(k,j) != 0 needs k <= j
}

template <class Real, int BM, int BN, bool TA>
__global__ void __launch_bounds__(kThreads) dgemm_kernel(GemmParamsT<Real> p) {
    constexpr int RM = BM / 16, RN = BN / 16;
    __shared__ Real As[BK][BM + 1];
    __shared__ Real Bs[BK][BN + 1];
    __shared__ int s_last;

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    const int S = gridDim.z, z = blockIdx.z;

    int64_t kb, ke;
    k_range(p, TA, m0, n0, BM, BN, kb, ke);
    int64_t k_lo = kb, k_hi = kb;
    if (ke > kb) {
        int64_t chunk = (ke - kb + S - 1) / S;
        chunk = (chunk + BK - 1) / BK * BK;
        k_lo = kb + (int64_t)z * chunk;
        k_hi = min(ke, k_lo + chunk);
    }

    Real acc[RM][RN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < RN; ++c) acc[r][c] = Real(0);

    for (int64_t k0 = k_lo; k0 < k_hi; k0 += BK) {
        // op(A) tile: rows m0.., k0..
#pragma unroll
        for (int idx = tid; idx < BM * BK; idx += kThreads) {
            int i, kk;
            if (!TA) { i = idx % BM; kk = idx / BM; }   // coalesced along rows of stored A
            else     { kk = idx % BK; i = idx / BK; }   // coalesced along rows of stored A (= k)
            const int64_t gi = m0 + i, gk = k0 + kk;
            Real v = Real(0);
            if (gi < p.M && gk < k_hi) v = TA ? masked(p.A, p.lda, gk, gi, p.maskA)
                                              : masked(p.A, p.lda, gi, gk, p.maskA);
            As[kk][i] = v;
        }
        // B tile: stored K x N, coalesced along k
#pragma unroll
        for (int idx = tid; idx < BK * BN; idx += kThreads) {
            const int kk = idx % BK, j = idx / BK;
            const int64_t gk = k0 + kk, gj = n0 + j;
            Real v = Real(0);
            if (gj < p.N && gk < k_hi) v = masked(p.B, p.ldb, gk, gj, p.maskB);
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Real a[RM], b[RN];
#pragma unroll
            for (int r = 0; r < RM; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < RN; ++c) b[c] = Bs[kk][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < RN; ++c) acc[r][c] = rfma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }

    if (S > 1) {
        // Split-K: deterministic tree of last-arriver reductions.
        const int64_t tile = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
        Real *tp = p.partial + (size_t)tile * p.slots_per_tile * (BM * BN);
        unsigned *tc = p.counters + (size_t)tile * p.counters_per_tile;
        int slot = z, Sl = S, base = 0, cbase = 0;
        for (;;) {
            Real *dst = tp + (size_t)(base + slot) * (BM * BN);
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < RN; ++c) dst[(tx + 16 * r) + (ty + 16 * c) * BM] = acc[r][c];
            const int group = slot / kGroup, first = group * kGroup;
            const int cnt = min(kGroup, Sl - first);
            const int Snext = (Sl + kGroup - 1) / kGroup;
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                unsigned prev = atomicAdd(&tc[cbase + group], 1u);
                s_last = (prev == (unsigned)(cnt - 1));
            }
            __syncthreads();
            if (!s_last) return;
            __threadfence();
            if (tid == 0) tc[cbase + group] = 0u;   // leave the counter zero for the next launch
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < RN; ++c) {
                    Real s = Real(0);
                    for (int q = 0; q < cnt; ++q)
                        s += __ldcg(tp + (size_t)(base + first + q) * (BM * BN) + (tx + 16 * r) + (ty + 16 * c) * BM);
                    acc[r][c] = s;
                }
            if (Snext == 1) break;
            base += Sl;
            cbase += Snext;
            slot = group;
            Sl = Snext;
        }
    }

#pragma unroll
    for (int c = 0; c < RN; ++c) {
        const int64_t gj = n0 + ty + 16 * c;
        if (gj >= p.N) continue;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const int64_t gi = m0 + tx + 16 * r;
            if (gi >= p.M) continue;
            Real *cp = p.C + gi + gj * p.ldc;
            Real v = p.alpha * acc[r][c];
            if (p.beta != Real(0)) v = rfma(p.beta, *cp, v);
            *cp = v;
        }
    }
}

// 64 x 64 tiles on the FP64 tensor cores: mma.sync m8n8k4 (DMMA).  Same
// staging, masks, K-range trimming and split-K tree as dgemm_kernel; 8 warps
// as 2 (M) x 4 (N), each owning a 32 x 16 block = 4 x 2 MMA tiles.  Fragment
// layouts of m8n8k4.f64: A (8x4, row) lane -> (lane/4, lane%4); B (4x8, col)
// lane -> (lane%4, lane/4); C/D (8x8) lane -> (lane/4, 2*(lane%4) + i).
__device__ __forceinline__ void dmma_8x8x4(double &d0, double &d1, double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

template <bool TA>
__global__ void __launch_bounds__(kThreads) dgemm_dmma_kernel(GemmParams p) {
    constexpr int BM = 64, BN = 64;
    // Row stride 68 = 4 (mod 16) doubles: the fragment loads (4 k-rows x 8
    // consecutive columns per warp) then touch 16 distinct bank pairs per half-warp.
    __shared__ double As[BK][BM + 4];
    __shared__ double Bs[BK][BN + 4];
    __shared__ int s_last;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    const int S = gridDim.z, z = blockIdx.z;

    int64_t kb, ke;
    k_range(p, TA, m0, n0, BM, BN, kb, ke);
    int64_t k_lo = kb, k_hi = kb;
    if (ke > kb) {
        int64_t chunk = (ke - kb + S - 1) / S;
        chunk = (chunk + BK - 1) / BK * BK;
        k_lo = kb + (int64_t)z * chunk;
        k_hi = min(ke, k_lo + chunk);
    }

    double acc[4][2][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) { acc[a][b][0] = 0.0; acc[a][b][1] = 0.0; }

    for (int64_t k0 = k_lo; k0 < k_hi; k0 += BK) {
#pragma unroll
        for (int idx = tid; idx < BM * BK; idx += kThreads) {
            int i, kk;
            if (!TA) { i = idx % BM; kk = idx / BM; }
            else     { kk = idx % BK; i = idx / BK; }
            const int64_t gi = m0 + i, gk = k0 + kk;
            double v = 0.0;
            if (gi < p.M && gk < k_hi) v = TA ? masked(p.A, p.lda, gk, gi, p.maskA)
                                              : masked(p.A, p.lda, gi, gk, p.maskA);
            As[kk][i] = v;
        }
#pragma unroll
        for (int idx = tid; idx < BK * BN; idx += kThreads) {
            const int kk = idx % BK, j = idx / BK;
            const int64_t gk = k0 + kk, gj = n0 + j;
            double v = 0.0;
            if (gj < p.N && gk < k_hi) v = masked(p.B, p.ldb, gk, gj, p.maskB);
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kq = 0; kq < BK; kq += 4) {
            double a[4], b[2];
#pragma unroll
            for (int ms = 0; ms < 4; ++ms) a[ms] = As[kq + (lane & 3)][wm * 32 + ms * 8 + (lane >> 2)];
#pragma unroll
            for (int ns = 0; ns < 2; ++ns) b[ns] = Bs[kq + (lane & 3)][wn * 16 + ns * 8 + (lane >> 2)];
#pragma unroll
            for (int ms = 0; ms < 4; ++ms)
#pragma unroll
                for (int ns = 0; ns < 2; ++ns) dmma_8x8x4(acc[ms][ns][0], acc[ms][ns][1], a[ms], b[ns]);
        }
        __syncthreads();
    }

    // element q = (ms, ns, i) of this thread sits at tile row/col:
    auto row_of = [&](int ms) { return wm * 32 + ms * 8 + (lane >> 2); };
    auto col_of = [&](int ns, int i) { return wn * 16 + ns * 8 + 2 * (lane & 3) + i; };

    if (S > 1) {
        const int64_t tile = blockIdx.x + (int64_t)blockIdx.y * gridDim.x;
        double *tp = p.partial + (size_t)tile * p.slots_per_tile * (BM * BN);
        unsigned *tc = p.counters + (size_t)tile * p.counters_per_tile;
        int slot = z, Sl = S, base = 0, cbase = 0;
        for (;;) {
            double *dst = tp + (size_t)(base + slot) * (BM * BN);
#pragma unroll
            for (int ms = 0; ms < 4; ++ms)
#pragma unroll
                for (int ns = 0; ns < 2; ++ns)
#pragma unroll
                    for (int i = 0; i < 2; ++i) dst[row_of(ms) + col_of(ns, i) * BM] = acc[ms][ns][i];
            const int group = slot / kGroup, first = group * kGroup;
            const int cnt = min(kGroup, Sl - first);
            const int Snext = (Sl + kGroup - 1) / kGroup;
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                unsigned prev = atomicAdd(&tc[cbase + group], 1u);
                s_last = (prev == (unsigned)(cnt - 1));
            }
            __syncthreads();
            if (!s_last) return;
            __threadfence();
            if (tid == 0) tc[cbase + group] = 0u;
#pragma unroll
            for (int ms = 0; ms < 4; ++ms)
#pragma unroll
                for (int ns = 0; ns < 2; ++ns)
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        double s = 0.0;
                        for (int q = 0; q < cnt; ++q)
                            s += __ldcg(tp + (size_t)(base + first + q) * (BM * BN) + row_of(ms) + col_of(ns, i) * BM);
                        acc[ms][ns][i] = s;
                    }
            if (Snext == 1) break;
            base += Sl;
            cbase += Snext;
            slot = group;
            Sl = Snext;
        }
    }

#pragma unroll
    for (int ms = 0; ms < 4; ++ms)
#pragma unroll
        for (int ns = 0; ns < 2; ++ns)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int64_t gi = m0 + row_of(ms), gj = n0 + col_of(ns, i);
                if (gi >= p.M || gj >= p.N) continue;
                double *cp = p.C + gi + gj * p.ldc;
                double v = p.alpha * acc[ms][ns][i];
                if (p.beta != 0.0) v = fma(p.beta, *cp, v);
                *cp = v;
            }
}

int tile_for(int64_t d) { return d <= 16 ? 16 : (d <= 32 ? 32 : 64); }

// Slots and counters per tile of the reduction tree for S splits.
void tree_shape(int S, int *slots, int *counters) {
    int s = 0, c = 0, Sl = S;
    while (Sl > 1) {
        s += Sl;
        Sl = (Sl + kGroup - 1) / kGroup;
        c += Sl;
    }
    *slots = std::max(s, 1);
    *counters = std::max(c, 1);
}

template <class Real, int BM, int BN>
cudaError_t launch_bm_bn(const GemmParamsT<Real> &p, bool ta, dim3 grid, cudaStream_t st) {
    if (ta) dgemm_kernel<Real, BM, BN, true><<<grid, kThreads, 0, st>>>(p);
    else dgemm_kernel<Real, BM, BN, false><<<grid, kThreads, 0, st>>>(p);
    return cudaPeekAtLastError();
}

template <class Real, int BM>
cudaError_t launch_bm(int BN, const GemmParamsT<Real> &p, bool ta, dim3 grid, cudaStream_t st) {
    switch (BN) {
        case 16: return launch_bm_bn<Real, BM, 16>(p, ta, grid, st);
        case 32: return launch_bm_bn<Real, BM, 32>(p, ta, grid, st);
        default: return launch_bm_bn<Real, BM, 64>(p, ta, grid, st);
    }
}

// At most this many split CTAs per SM.  The split count also stops where the
// partial tiles would not fit the caller's scratch, so a smaller buffer only
// limits the splitting.  (A 128 x 7936 product of graded 8192^2 - 252 tiles
// over K = 8192 - split 2 at 4 CTAs per SM left 48 SMs with 4 CTAs and 104
// with 3, 1.06 TFLOP/s; split 3 or more, 1.20.)
constexpr int kMaxSplitCtasPerSm = 16;
constexpr int kBaseSplitCtasPerSm = 4;

size_t partial_elems_for(int ctas_per_sm, int num_sms) {
    // the reduction tree adds at most a quarter more slots, plus a few per tile
    const size_t ctas = (size_t)ctas_per_sm * num_sms;
    return (ctas + ctas / 4 + 64) * 64 * 64;
}

}  // namespace

size_t gemm_partial_elems_max(int num_sms) { return partial_elems_for(kMaxSplitCtasPerSm, num_sms); }
size_t gemm_partial_elems_min(int num_sms) { return partial_elems_for(kBaseSplitCtasPerSm, num_sms); }

size_t gemm_counters_max(int num_sms) { return (size_t)kMaxSplitCtasPerSm * num_sms * 2 + 64; }

template <class Real>
double gemm_algorithmic_flops(const GemmOpT<Real> &op) {
    // 2*M*N*K for a dense product; a masked triangular operand halves its
    // square part.  (Exact for the shapes used: the triangle is the leading
    // square of the masked operand.)
    double M = (double)op.M, N = (double)op.N, K = (double)op.K;
    double f = 2.0 * M * N * K;
    auto tri = [](double rows, double cols) {  // non-zero entries of a unit-lower/upper rows x cols
        double s = std::min(rows, cols);
        return rows * cols - s * (s - 1) / 2.0;
    };
    if (op.maskA != MASK_NONE) f = 2.0 * N * tri(op.ta ? K : M, op.ta ? M : K);
    else if (op.maskB != MASK_NONE) f = 2.0 * M * tri(K, N);
    return f;
}

template <class Real>
gbqr_status gemm(const Exec &ex, const GemmOpT<Real> &op, const GemmScratchT<Real> &sc) {
    if (op.M <= 0 || op.N <= 0) return GBQR_OK;
    if (op.K <= 0) {
        if (op.beta == Real(1)) return GBQR_OK;
    }
    // A small output (the T products of Algorithm 2 are 64 x 64 x 64 at the
    // panel's top node) on 64 x 64 tiles would run on a handful of SMs at one
    // SM's FP64 rate (2 FMA/clock: ~60 us for 64^3): shrink the tiles until
    // the output spans the SMs, then split K.
    // (FP64 only: FP32 runs 64x faster per SM on this part, and the extra
    // splits measured slower for the FP32 batch.)
    constexpr bool fp64 = std::is_same<Real, double>::value;
    int BM = tile_for(op.M), BN = tile_for(op.N);
    auto count_tiles = [&](int bm, int bn) { return ((op.M + bm - 1) / bm) * ((op.N + bn - 1) / bn); };
    while (fp64 && count_tiles(BM, BN) < ex.num_sms && (BM > 16 || BN > 16)) {
        if (BM >= BN && BM > 16) BM /= 2;
        else BN /= 2;
    }
    const int64_t tm = (op.M + BM - 1) / BM, tn = (op.N + BN - 1) / BN;
    if (tm > 0x7fffffff || tn > 65535) return GBQR_EUNSUPPORTED;
    const int64_t tiles = tm * tn;
    const int64_t ktiles = (std::max<int64_t>(op.K, 0) + BK - 1) / BK;

    // Split K when the output alone cannot fill the GPU: at least 4 K-tiles
    // per split where K allows, one where it is short; pick the split count
    // whose CTA total wastes the least of the last wave.
    int S = 1;
    const int64_t fill = 2LL * ex.num_sms;
    if (tiles < fill && ktiles >= (fp64 ? 2 : 8)) {
        const int64_t per = (ktiles >= 32 || !fp64) ? 4 : 1;
        const int64_t smax = std::min<int64_t>({ktiles / per, (int64_t)kMaxSplitCtasPerSm * ex.num_sms / tiles, 512});
        double best = -1.0;
        for (int64_t s = 1; s <= smax; ++s) {
            if (s > 1) {   // the split's partial tiles and counters must fit the scratch
                int sl = 1, ct = 1;
                tree_shape((int)s, &sl, &ct);
                if (!sc.partial || !sc.counters || (size_t)tiles * sl * BM * BN > sc.partial_elems ||
                    (size_t)tiles * ct > sc.ncounters)
                    continue;
            }
            const double ctas = (double)(tiles * s);
            const double waves = std::ceil(ctas / ex.num_sms);
            // useful fraction of the occupied SM-waves, lightly favouring more parallelism
            const double eff = ctas / (waves * ex.num_sms) * std::min(1.0, ctas / (double)fill);
            if (eff > best + 1e-9) { best = eff; S = (int)s; }
        }
    }
    GemmParamsT<Real> p;
    p.M = op.M; p.N = op.N; p.K = std::max<int64_t>(op.K, 0);
    p.A = op.A; p.lda = op.lda; p.maskA = op.maskA;
    p.B = op.B; p.ldb = op.ldb; p.maskB = op.maskB;
    p.C = op.C; p.ldc = op.ldc; p.alpha = op.alpha; p.beta = op.beta;
    p.partial = sc.partial; p.counters = sc.counters;
    p.slots_per_tile = 1; p.counters_per_tile = 1;
    if (S > 1) {
        tree_shape(S, &p.slots_per_tile, &p.counters_per_tile);
        size_t need_p = (size_t)tiles * p.slots_per_tile * BM * BN;
        size_t need_c = (size_t)tiles * p.counters_per_tile;
        if (need_p > sc.partial_elems || need_c > sc.ncounters || !sc.partial || !sc.counters) return GBQR_ENOMEM;
    }
    dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)S);
    trace_begin(ex, FAM_GEMM);
    cudaError_t e;
    bool launched = false;
    if constexpr (std::is_same<Real, double>::value) {
        if (BM == 64 && BN == 64 && ex.dmma) {
            if (op.ta) dgemm_dmma_kernel<true><<<grid, kThreads, 0, ex.stream>>>(p);
            else dgemm_dmma_kernel<false><<<grid, kThreads, 0, ex.stream>>>(p);
            e = cudaPeekAtLastError();
            launched = true;
        }
    }
    if (!launched) {
        switch (BM) {
            case 16: e = launch_bm<Real, 16>(BN, p, op.ta, grid, ex.stream); break;
            case 32: e = launch_bm<Real, 32>(BN, p, op.ta, grid, ex.stream); break;
            default: e = launch_bm<Real, 64>(BN, p, op.ta, grid, ex.stream); break;
        }
    }
    if (e != cudaSuccess) return GBQR_ECUDA;
    const double bytes = (double)sizeof(Real) *
                         ((double)op.M * op.K + (double)op.K * op.N + (op.beta != Real(0) ? 2.0 : 1.0) * op.M * op.N);
    return trace_end(ex, FAM_GEMM, gemm_algorithmic_flops(op), bytes);
}

template gbqr_status gemm<double>(const Exec &, const GemmOpT<double> &, const GemmScratchT<double> &);
template gbqr_status gemm<float>(const Exec &, const GemmOpT<float> &, const GemmScratchT<float> &);
template double gemm_algorithmic_flops<double>(const GemmOpT<double> &);
template double gemm_algorithmic_flops<float>(const GemmOpT<float> &);

}  // namespace gbqr
