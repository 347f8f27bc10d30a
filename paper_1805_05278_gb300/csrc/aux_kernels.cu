// Small kernels around the factorization: forming [I; 0] for the thin Q,
// zeroing the lower triangle of T, copies, the non-finite input scan, the
// blocked triangular solves with R and R^T, and the FP64 matrix-vector
// products, norms and vector updates of the least-squares refinement.
#include "common.cuh"

#include <algorithm>

namespace gbqr {
namespace {

// Grid-stride over an m x n column-major matrix, one thread per element,
// consecutive threads on consecutive rows (coalesced).
// Elementwise kernels over an m x n column-major matrix: a 2-D grid, x
// striding rows and y striding columns (no 64-bit division per entry).
#define FOR_EACH_ENTRY(m, n, body)                                                                      \
    for (int64_t j = blockIdx.y; j < (n); j += gridDim.y)                                               \
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (m); i += (int64_t)gridDim.x * blockDim.x) \
            body

__global__ void __launch_bounds__(kThreads) fill_identity_kernel(int64_t m, int64_t n, double *Q, int64_t ldq) {
    FOR_EACH_ENTRY(m, n, { Q[i + j * ldq] = (i == j) ? 1.0 : 0.0; })
}

__global__ void __launch_bounds__(kThreads) zero_strict_lower_kernel(int64_t n, double *T, int64_t ldt) {
    FOR_EACH_ENTRY(n, n, { if (i > j) T[i + j * ldt] = 0.0; })
}

__global__ void __launch_bounds__(kThreads) copy_kernel(int64_t m, int64_t n, const double *src, int64_t lds,
                                                      double *dst, int64_t ldd) {
    FOR_EACH_ENTRY(m, n, { dst[i + j * ldd] = src[i + j * lds]; })
}

template <class Real>
__global__ void __launch_bounds__(kThreads) nonfinite_kernel(int64_t m, int64_t n, const Real *A, int64_t lda,
                                                           unsigned long long *flag) {
    int bad = 0;
    FOR_EACH_ENTRY(m, n, { bad |= !isfinite(A[i + j * lda]); })
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1ull);
}

constexpr int kTrsvBlock = 64;





// y(m) = alpha * A(m x n) x + beta * y, split over column chunks with FP64
// partials P[chunk][m], then summed in a fixed order (deterministic).
// mask MASK_UNIT_LOWER: A(i, j) = 0 for i < j and 1 for i == j (a V basis).
__global__ void __launch_bounds__(kThreads) gemv_n_partial_kernel(int64_t m, int64_t n, int64_t chunk,
                                                                 const double *A, int64_t lda, const double *x,
                                                                 double *P, int mask) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.y * chunk;
    int64_t c1 = min(n, c0 + chunk);
    if (i >= m) return;
    double acc = 0.0;
    if (mask == MASK_UNIT_LOWER) {
        if (i >= c0 && i < c1) acc = x[i];
        c1 = min(c1, i);
    }
    // four independent chains: a dependent FP64 FMA costs ~100 cycles here
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t j = c0;
    for (; j + 3 < c1; j += 4) {
        acc = fma(A[i + j * lda], x[j], acc);
        a1 = fma(A[i + (j + 1) * lda], x[j + 1], a1);
        a2 = fma(A[i + (j + 2) * lda], x[j + 2], a2);
        a3 = fma(A[i + (j + 3) * lda], x[j + 3], a3);
    }
    for (; j < c1; ++j) acc = fma(A[i + j * lda], x[j], acc);
    P[(int64_t)blockIdx.y * m + i] = (acc + a1) + (a2 + a3);
}

__global__ void __launch_bounds__(kThreads) gemv_n_reduce_kernel(int64_t m, int nchunks, const double *P, double alpha,
                                                                double beta, double *y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += P[(int64_t)c * m + i];
    y[i] = (beta == 0.0) ? alpha * s : fma(beta, y[i], alpha * s);
}

// g(n) = alpha * A^T r + beta * g: one CTA per column, every thread on rows
// strided by the block size in four independent chains (a single warp per
// column ran an m/32-long dependent FMA chain at ~100 cycles a link).
__global__ void __launch_bounds__(kThreads) gemv_t_kernel(int64_t m, int64_t n, const double *A, int64_t lda,
                                                         const double *r, double alpha, double beta, double *g,
                                                         int mask) {
    __shared__ double red[kThreads / 32];
    const int64_t j = blockIdx.x;
    if (j >= n) return;
    const double *a = A + j * lda;
    double acc = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t i0 = 0;
    if (mask == MASK_UNIT_LOWER) {
        if (threadIdx.x == 0 && j < m) acc = r[j];
        i0 = j + 1;
    }
    const int64_t step = blockDim.x;
    int64_t i = i0 + threadIdx.x;
    for (; i + 3 * step < m; i += 4 * step) {
        acc = fma(a[i], r[i], acc);
        a1 = fma(a[i + step], r[i + step], a1);
        a2 = fma(a[i + 2 * step], r[i + 2 * step], a2);
        a3 = fma(a[i + 3 * step], r[i + 3 * step], a3);
    }
    for (; i < m; i += step) acc = fma(a[i], r[i], acc);
    acc = (acc + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        g[j] = (beta == 0.0) ? alpha * s : fma(beta, g[j], alpha * s);
    }
}

// out[0] = sum x^2, out[1] = sum y^2 (one CTA, fixed order).
__global__ void __launch_bounds__(kThreads) norms2_kernel(int64_t n, const double *x, const double *y, double *out) {
    __shared__ double red[2][kThreads / 32];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        a = fma(x[i], x[i], a);
        b = fma(y[i], y[i], b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += red[0][w]; s1 += red[1][w]; }
        out[0] = s0;
        out[1] = s1;
    }
}

// colsq[j] = sum_i A(i, j)^2: one warp per column.
__global__ void __launch_bounds__(kThreads) colsq_kernel(int64_t m, int64_t n, const double *A, int64_t lda,
                                                        double *colsq) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    double acc = 0.0;
    for (int64_t i = lane; i < m; i += 32) acc = fma(A[i + j * lda], A[i + j * lda], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) colsq[j] = acc;
}

// out[0] = sum x (one CTA, fixed order)
__global__ void __launch_bounds__(kThreads) sum_kernel(int64_t n, const double *x, double *out) {
    __shared__ double red[kThreads / 32];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        out[0] = s;
    }
}

// y = a * x + b * y (elementwise)
__global__ void __launch_bounds__(kThreads) axpby_kernel(int64_t n, double a, const double *x, double b, double *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

// One warp solves the s x s diagonal block of R whose rows/columns start at
// jb, with the right-hand side in xs[0:s] (shared memory): back substitution
// (transpose = false, R upper) or forward substitution with R^T.  The block
// is staged in shared memory by the whole CTA first; pivots are used through
// their reciprocals so that each step is one multiply, one shuffle and one
// FMA on the critical path.
__device__ void warp_block_solve(int64_t jb, int s, const double *R, int64_t ldr, double *xs, double *Rs,
                                 bool transpose, long long *rankdef) {
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
        const int i = idx % s, c = idx / s;
        Rs[i + c * kTrsvBlock] = R[(jb + i) + (jb + c) * ldr];
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double c0 = (lane < s) ? xs[lane] : 0.0, c1 = (lane + 32 < s) ? xs[lane + 32] : 0.0;
        double r0 = 0.0, r1 = 0.0;
        if (lane < s) {
            const double d = Rs[lane + lane * kTrsvBlock];
            if (d == 0.0) atomicMin(rankdef, (long long)(jb + lane));
            r0 = 1.0 / d;
        }
        if (lane + 32 < s) {
            const double d = Rs[(lane + 32) + (lane + 32) * kTrsvBlock];
            if (d == 0.0) atomicMin(rankdef, (long long)(jb + lane + 32));
            r1 = 1.0 / d;
        }
        for (int t = 0; t < s; ++t) {
            const int j = transpose ? t : s - 1 - t;
            const bool hi = j >= 32;
            const double mine = hi ? c1 * r1 : c0 * r0;
            const double xj = __shfl_sync(0xffffffffu, mine, j & 31);
            if ((j & 31) == lane) { if (hi) c1 = xj; else c0 = xj; }
            // remaining rows: i < j (back substitution) or i > j (forward, R^T)
            const int i0 = lane, i1 = lane + 32;
            if (!transpose) {
                if (i0 < j) c0 = fma(-Rs[i0 + j * kTrsvBlock], xj, c0);
                if (i1 < j) c1 = fma(-Rs[i1 + j * kTrsvBlock], xj, c1);
            } else {
                if (i0 > j && i0 < s) c0 = fma(-Rs[j + i0 * kTrsvBlock], xj, c0);
                if (i1 > j && i1 < s) c1 = fma(-Rs[j + i1 * kTrsvBlock], xj, c1);
            }
        }
        if (lane < s) xs[lane] = c0;
        if (lane + 32 < s) xs[lane + 32] = c1;
    }
    __syncthreads();
}

// Inverses of the diagonal blocks of R (kTrsvBlock x kTrsvBlock, upper
// triangular), one CTA per block, for the refinement's repeated solves with
// the same R.  Bottom-up over block sizes 1, 2, 4, ...: for each pair of
// adjacent diagonal blocks Ri12 = -Ri11 R12 Ri22, so the dependency depth is
// log2 of the block size (a substitution would chain the whole block).
__global__ void __launch_bounds__(kThreads) trsv_block_inverse_kernel(int64_t n, const double *R, int64_t ldr,
                                                                    double *Dinv, long long *rankdef) {
    constexpr int B = kTrsvBlock;
    __shared__ double Rs[B * B], Ri[B * B], M[B * B];
    const int64_t jb = (int64_t)blockIdx.x * B;
    const int s = (int)((n - jb) < (int64_t)B ? (n - jb) : (int64_t)B);
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int idx = tid; idx < B * B; idx += nthr) {
        const int i = idx % B, c = idx / B;
        Rs[idx] = (i < s && c < s && i <= c) ? R[(jb + i) + (jb + c) * ldr] : 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < B * B; idx += nthr) {
        const int i = idx % B, c = idx / B;
        double v = 0.0;
        if (i == c && i < s) {
            const double d = Rs[idx];
            if (d == 0.0) atomicMin(rankdef, (long long)(jb + i));
            v = 1.0 / d;
        }
        Ri[idx] = v;
    }
    __syncthreads();
    for (int h = 1; h < B; h *= 2) {
        const int h2 = 2 * h;
        for (int idx = tid; idx < B * B; idx += nthr) {     // M = R12 Ri22
            const int row = idx % B, col = idx / B;
            const int b1 = (row / h2) * h2 + h;
            if (row >= b1 || col < b1 || col >= b1 + h) continue;
            double acc = 0.0;
            for (int l = b1; l <= col; ++l) acc = fma(Rs[row + l * B], Ri[l + col * B], acc);
            M[idx] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < B * B; idx += nthr) {     // Ri12 = -Ri11 M
            const int row = idx % B, col = idx / B;
            const int b1 = (row / h2) * h2 + h;
            if (row >= b1 || col < b1 || col >= b1 + h) continue;
            double acc = 0.0;
            for (int l = row; l < b1; ++l) acc = fma(Ri[row + l * B], M[l + col * B], acc);
            Ri[idx] = -acc;
        }
        __syncthreads();
    }
    double *D = Dinv + (size_t)blockIdx.x * B * B;
    for (int idx = tid; idx < B * B; idx += nthr) D[idx] = Ri[idx];
}

// x(jb : jb+s) <- op(Di) x(jb : jb+s) for a block inverse Di (upper, ld B;
// op = transpose for R^T): four threads per row, shuffles across the four.
__device__ void block_inverse_apply(int64_t jb, int s, const double *Di, double *x, double *xs, bool transpose) {
    constexpr int B = kTrsvBlock;
    if (threadIdx.x < s) xs[threadIdx.x] = x[jb + threadIdx.x];
    __syncthreads();
    const int i = threadIdx.x >> 2, part = threadIdx.x & 3;
    double acc = 0.0;
    if (i < s) {
        if (!transpose)
            for (int c = i + part; c < s; c += 4) acc = fma(Di[i + c * B], xs[c], acc);
        else
            for (int c = part; c <= i; c += 4) acc = fma(Di[c + i * B], xs[c], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (i < s && part == 0) x[jb + i] = acc;
}

// Back substitution R x = c, one launch per block (from the bottom): apply
// the just-solved block x(j0:j0+s) to rows [0, j0) - each CTA owns 64 rows,
// its four warp pairs splitting the block's columns in quarters (a warp reads
// 32 consecutive rows of a column), combined in a fixed order - then the CTA
// owning the block just above, rows [jn, j0), solves it.
__global__ void __launch_bounds__(kThreads) trsv_step_kernel(int64_t j0, int s, int64_t jn, int sn, const double *R,
                                                           int64_t ldr, double *x, long long *rankdef,
                                                           const double *Dinv) {
    constexpr int kRows = 64;
    __shared__ double xb[kTrsvBlock];
    __shared__ double xs[kTrsvBlock];
    __shared__ double Rs[kTrsvBlock * kTrsvBlock];
    __shared__ double part[4][kRows];
    if (threadIdx.x < s) xb[threadIdx.x] = x[j0 + threadIdx.x];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    if (s > 0) {
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int q = wid >> 1, rl = (wid & 1) * 32 + lane;
        const int64_t i = r0 + rl;
        const int qw = (s + 3) / 4, c0 = q * qw, c1 = min(s, c0 + qw);
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (i < j0) {
            const double *Ri = R + i + j0 * ldr;
            int l = c0;
            for (; l + 3 < c1; l += 4) {
                a0 = fma(Ri[l * ldr], xb[l], a0);
                a1 = fma(Ri[(l + 1) * ldr], xb[l + 1], a1);
                a2 = fma(Ri[(l + 2) * ldr], xb[l + 2], a2);
                a3 = fma(Ri[(l + 3) * ldr], xb[l + 3], a3);
            }
            for (; l < c1; ++l) a0 = fma(Ri[l * ldr], xb[l], a0);
        }
        part[q][rl] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        if (threadIdx.x < kRows && r0 + threadIdx.x < j0)
            x[r0 + threadIdx.x] -= (part[0][threadIdx.x] + part[1][threadIdx.x]) +
                                   (part[2][threadIdx.x] + part[3][threadIdx.x]);
    }
    if (sn > 0 && jn >= r0 && jn < r0 + kRows) {
        __syncthreads();                 // this CTA's rows [jn, j0) are final
        __threadfence_block();
        if (Dinv) {
            block_inverse_apply(jn, sn, Dinv + (size_t)(jn / kTrsvBlock) * kTrsvBlock * kTrsvBlock, x, xs, false);
            return;
        }
        if (threadIdx.x < sn) xs[threadIdx.x] = x[jn + threadIdx.x];
        __syncthreads();
        warp_block_solve(jn, sn, R, ldr, xs, Rs, false, rankdef);
        if (threadIdx.x < sn) x[jn + threadIdx.x] = xs[threadIdx.x];
    }
}

// Forward substitution R^T h = g, one launch per block (from the top): apply
// the just-solved block h(jp:jp+sp) to entries [jp+sp, n) - each CTA owns 64
// entries, one warp per entry - then the CTA owning the next block solves it.
__global__ void __launch_bounds__(kThreads) trsv_t_step_kernel(int64_t n, int64_t jp, int sp, int sn,
                                                             const double *R, int64_t ldr, double *x,
                                                             long long *rankdef, const double *Dinv) {
    __shared__ double xb[kTrsvBlock];
    __shared__ double xs[kTrsvBlock];
    __shared__ double Rs[kTrsvBlock * kTrsvBlock];
    if (threadIdx.x < sp) xb[threadIdx.x] = x[jp + threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t e0 = jp + sp + (int64_t)blockIdx.x * kTrsvBlock;   // first entry of this CTA
    if (sp > 0) {
        for (int q = wid; q < kTrsvBlock; q += kThreads / 32) {
            const int64_t i = e0 + q;
            if (i >= n) break;
            double acc = 0.0;
            for (int l = lane; l < sp; l += 32) acc = fma(R[(jp + l) + i * ldr], xb[l], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) x[i] -= acc;
        }
    }
    if (blockIdx.x == 0 && sn > 0) {
        __syncthreads();
        __threadfence_block();
        if (Dinv) {
            block_inverse_apply(e0, sn, Dinv + (size_t)(e0 / kTrsvBlock) * kTrsvBlock * kTrsvBlock, x, xs, true);
            return;
        }
        if (threadIdx.x < sn) xs[threadIdx.x] = x[e0 + threadIdx.x];
        __syncthreads();
        warp_block_solve(e0, sn, R, ldr, xs, Rs, true, rankdef);
        if (threadIdx.x < sn) x[e0 + threadIdx.x] = xs[threadIdx.x];
    }
}

// y = op(T) w for a k x k upper triangular T: one warp per output entry
// (lanes split the row's dot product; a thread per row ran a k-long
// dependent FMA chain).
__global__ void __launch_bounds__(kThreads) trmv_kernel(int k, const double *T, int64_t ldt, bool trans,
                                                      const double *w, double *y) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (i >= k) return;
    double acc = 0.0;
    if (!trans)
        for (int l = i + lane; l < k; l += 32) acc = fma(T[i + (int64_t)l * ldt], w[l], acc);
    else
        for (int l = lane; l <= i; l += 32) acc = fma(T[l + (int64_t)i * ldt], w[l], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[i] = acc;
}

// Grid of the elementwise kernels: enough row blocks to cover a column, and
// columns until about 32 CTAs per SM.
dim3 grid2d(int64_t m, int64_t n, int num_sms) {
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>((m + kThreads - 1) / kThreads, (int64_t)num_sms * 8));
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>({n, (int64_t)65535, (int64_t)num_sms * 32 / gx + 1}));
    return dim3((unsigned)gx, (unsigned)gy);
}

unsigned grid_for(int64_t elems, int num_sms) {
    const int64_t want = (elems + kThreads - 1) / kThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
}

}  // namespace

gbqr_status fill_identity(const Exec &ex, int64_t m, int64_t n, double *Q, int64_t ldq) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    fill_identity_kernel<<<grid2d(m, n, ex.num_sms), kThreads, 0, ex.stream>>>(m, n, Q, ldq);
    return trace_end(ex, FAM_OTHER, 0.0, 8.0 * m * n);
}

gbqr_status zero_strict_lower(const Exec &ex, int64_t n, double *T, int64_t ldt) {
    if (n <= 1) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    zero_strict_lower_kernel<<<grid2d(n, n, ex.num_sms), kThreads, 0, ex.stream>>>(n, T, ldt);
    return trace_end(ex, FAM_OTHER, 0.0, 4.0 * n * n);
}

gbqr_status copy_matrix(const Exec &ex, int64_t m, int64_t n, const double *src, int64_t lds,
                        double *dst, int64_t ldd) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    copy_kernel<<<grid2d(m, n, ex.num_sms), kThreads, 0, ex.stream>>>(m, n, src, lds, dst, ldd);
    return trace_end(ex, FAM_OTHER, 0.0, 16.0 * m * n);
}

template <class Real>
gbqr_status scan_nonfinite(const Exec &ex, int64_t m, int64_t n, const Real *A, int64_t lda,
                           unsigned long long *flag) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    nonfinite_kernel<Real><<<grid2d(m, n, ex.num_sms), kThreads, 0, ex.stream>>>(m, n, A, lda, flag);
    return trace_end(ex, FAM_OTHER, 0.0, (double)sizeof(Real) * m * n);
}
template gbqr_status scan_nonfinite<double>(const Exec &, int64_t, int64_t, const double *, int64_t,
                                            unsigned long long *);
template gbqr_status scan_nonfinite<float>(const Exec &, int64_t, int64_t, const float *, int64_t,
                                           unsigned long long *);

gbqr_status trsv_block_inverses(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *Dinv,
                                long long *rankdef) {
    if (n <= 0) return GBQR_OK;
    const int64_t nblk = (n + kTrsvBlock - 1) / kTrsvBlock;
    trace_begin(ex, FAM_TRSV);
    trsv_block_inverse_kernel<<<(unsigned)nblk, kThreads, 0, ex.stream>>>(n, R, ldr, Dinv, rankdef);
    return trace_end(ex, FAM_TRSV, (double)nblk * kTrsvBlock * kTrsvBlock * kTrsvBlock / 3.0,
                     8.0 * nblk * kTrsvBlock * kTrsvBlock * 2.0);
}

gbqr_status trsv_upper(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *x, long long *rankdef,
                       const double *Dinv) {
    if (n <= 0) return GBQR_OK;
    const int64_t nblk = (n + kTrsvBlock - 1) / kTrsvBlock;
    // launch k applies block k (solved) and solves block k-1; the first
    // launch applies nothing and solves the last block
    for (int64_t k = nblk; k >= 1; --k) {
        const int64_t j0 = (k == nblk) ? n : k * kTrsvBlock;
        const int s = (k == nblk) ? 0 : (int)std::min<int64_t>(kTrsvBlock, n - j0);
        const int64_t jn = (k - 1) * kTrsvBlock;
        const int sn = (int)std::min<int64_t>(kTrsvBlock, n - jn);
        const unsigned grid = (unsigned)std::max<int64_t>(1, (j0 + 63) / 64);   // 64 rows per CTA
        trace_begin(ex, FAM_TRSV);
        trsv_step_kernel<<<grid, kThreads, 0, ex.stream>>>(j0, s, jn, sn, R, ldr, x, rankdef, Dinv);
        TRY_ST(trace_end(ex, FAM_TRSV, 2.0 * j0 * s + (double)sn * sn, 8.0 * j0 * s));
    }
    return GBQR_OK;
}

gbqr_status trsv_upper_t(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *x, long long *rankdef,
                         const double *Dinv) {
    if (n <= 0) return GBQR_OK;
    const int64_t nblk = (n + kTrsvBlock - 1) / kTrsvBlock;
    // launch k applies block k-1 (solved) and solves block k; the first
    // launch applies nothing and solves block 0
    for (int64_t k = 0; k < nblk; ++k) {
        const int64_t jp = (k == 0) ? 0 : (k - 1) * kTrsvBlock;
        const int sp = (k == 0) ? 0 : kTrsvBlock;
        const int64_t jk = k * kTrsvBlock;
        const int sn = (int)std::min<int64_t>(kTrsvBlock, n - jk);
        const int64_t rest = n - (jp + sp);
        const unsigned grid = (unsigned)std::max<int64_t>(1, (rest + kTrsvBlock - 1) / kTrsvBlock);
        trace_begin(ex, FAM_TRSV);
        trsv_t_step_kernel<<<grid, kThreads, 0, ex.stream>>>(n, jp, sp, sn, R, ldr, x, rankdef, Dinv);
        TRY_ST(trace_end(ex, FAM_TRSV, 2.0 * rest * sp + (double)sn * sn, 8.0 * rest * sp));
    }
    return GBQR_OK;
}

gbqr_status trmv_upper(const Exec &ex, int k, const double *T, int64_t ldt, bool trans, const double *w, double *y) {
    if (k <= 0) return GBQR_OK;
    trace_begin(ex, FAM_GEMV);
    trmv_kernel<<<(unsigned)((k + kThreads / 32 - 1) / (kThreads / 32)), kThreads, 0, ex.stream>>>(k, T, ldt, trans, w, y);
    return trace_end(ex, FAM_GEMV, (double)k * k, 4.0 * k * k);
}

gbqr_status gemv_n(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, const double *x, double alpha,
                   double beta, double *y, double *partial, size_t partial_elems, int mask) {
    if (m <= 0) return GBQR_OK;
    const int64_t rowblocks = (m + kThreads - 1) / kThreads;
    int64_t nchunks = std::max<int64_t>(1, std::min<int64_t>((4LL * ex.num_sms + rowblocks - 1) / rowblocks, std::max<int64_t>(n / 32, 1)));
    while (nchunks > 1 && (size_t)(nchunks * m) > partial_elems) --nchunks;
    if ((size_t)m > partial_elems) return GBQR_ENOMEM;
    const int64_t chunk = (std::max<int64_t>(n, 1) + nchunks - 1) / nchunks;
    nchunks = (std::max<int64_t>(n, 1) + chunk - 1) / chunk;
    trace_begin(ex, FAM_GEMV);
    gemv_n_partial_kernel<<<dim3((unsigned)rowblocks, (unsigned)nchunks), kThreads, 0, ex.stream>>>(m, n, chunk, A, lda, x, partial, mask);
    TRY_ST(trace_end(ex, FAM_GEMV, 2.0 * m * n, 8.0 * m * n));
    trace_begin(ex, FAM_GEMV);
    gemv_n_reduce_kernel<<<(unsigned)rowblocks, kThreads, 0, ex.stream>>>(m, (int)nchunks, partial, alpha, beta, y);
    return trace_end(ex, FAM_GEMV, (double)nchunks * m, 8.0 * (nchunks + 2) * m);
}

gbqr_status gemv_t(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, const double *r, double alpha,
                   double beta, double *g, int mask) {
    if (n <= 0) return GBQR_OK;
    if (n > 0x7fffffff) return GBQR_EUNSUPPORTED;
    trace_begin(ex, FAM_GEMV);
    gemv_t_kernel<<<(unsigned)n, kThreads, 0, ex.stream>>>(m, n, A, lda, r, alpha, beta, g, mask);
    return trace_end(ex, FAM_GEMV, 2.0 * m * n, 8.0 * m * n);
}

gbqr_status norms2(const Exec &ex, int64_t n, const double *x, const double *y, double *out) {
    trace_begin(ex, FAM_OTHER);
    norms2_kernel<<<1, kThreads, 0, ex.stream>>>(n, x, y, out);
    return trace_end(ex, FAM_OTHER, 4.0 * n, 16.0 * n);
}

gbqr_status frob2(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, double *colsq, double *out) {
    if (n <= 0) return GBQR_OK;
    const int per = kThreads / 32;
    trace_begin(ex, FAM_OTHER);
    colsq_kernel<<<(unsigned)((n + per - 1) / per), kThreads, 0, ex.stream>>>(m, n, A, lda, colsq);
    TRY_ST(trace_end(ex, FAM_OTHER, 2.0 * m * n, 8.0 * m * n));
    trace_begin(ex, FAM_OTHER);
    sum_kernel<<<1, kThreads, 0, ex.stream>>>(n, colsq, out);
    return trace_end(ex, FAM_OTHER, (double)n, 8.0 * n);
}

gbqr_status axpby(const Exec &ex, int64_t n, double a, const double *x, double b, double *y) {
    if (n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    axpby_kernel<<<grid_for(n, ex.num_sms), kThreads, 0, ex.stream>>>(n, a, x, b, y);
    return trace_end(ex, FAM_OTHER, 3.0 * n, 24.0 * n);
}

}  // namespace gbqr
