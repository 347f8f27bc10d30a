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
__global__ void __launch_bounds__(kThreads) fill_identity_kernel(int64_t m, int64_t n, double *Q, int64_t ldq) {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m, j = e / m;
        Q[i + j * ldq] = (i == j) ? 1.0 : 0.0;
    }
}

__global__ void __launch_bounds__(kThreads) zero_strict_lower_kernel(int64_t n, double *T, int64_t ldt) {
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        if (i > j) T[i + j * ldt] = 0.0;
    }
}

__global__ void __launch_bounds__(kThreads) copy_kernel(int64_t m, int64_t n, const double *src, int64_t lds,
                                                      double *dst, int64_t ldd) {
    const int64_t total = m * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m, j = e / m;
        dst[i + j * ldd] = src[i + j * lds];
    }
}

__global__ void __launch_bounds__(kThreads) nonfinite_kernel(int64_t m, int64_t n, const double *A, int64_t lda,
                                                           unsigned long long *flag) {
    const int64_t total = m * n;
    int bad = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % m, j = e / m;
        bad |= !isfinite(A[i + j * lda]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1ull);
}

constexpr int kTrsvBlock = 64;

// Solve the diagonal block R(j0:j0+s, j0:j0+s) x = x(j0:j0+s) in place
// (column-oriented back substitution, one CTA of kTrsvBlock threads).
__global__ void __launch_bounds__(kTrsvBlock) trsv_diag_kernel(int64_t j0, int s, const double *R, int64_t ldr,
                                                              double *x, long long *rankdef) {
    __shared__ double xs[kTrsvBlock];
    const int t = threadIdx.x;
    if (t < s) xs[t] = x[j0 + t];
    __syncthreads();
    for (int j = s - 1; j >= 0; --j) {
        const double d = R[(j0 + j) + (j0 + j) * ldr];
        if (t == 0) {
            if (d == 0.0) atomicMin(rankdef, (long long)(j0 + j));
            xs[j] = xs[j] / d;
        }
        __syncthreads();
        if (t < j) xs[t] = fma(-R[(j0 + t) + (j0 + j) * ldr], xs[j], xs[t]);
        __syncthreads();
    }
    if (t < s) x[j0 + t] = xs[t];
}

// x(0:j0) -= R(0:j0, j0:j0+s) x(j0:j0+s), one thread per row.
__global__ void __launch_bounds__(kThreads) trsv_update_kernel(int64_t j0, int s, const double *R, int64_t ldr,
                                                             double *x) {
    __shared__ double xb[kTrsvBlock];
    if (threadIdx.x < s) xb[threadIdx.x] = x[j0 + threadIdx.x];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= j0) return;
    double acc = 0.0;
    for (int l = 0; l < s; ++l) acc = fma(R[i + (j0 + l) * ldr], xb[l], acc);
    x[i] -= acc;
}

// x(j0+s:n) -= R(j0:j0+s, j0+s:n)^T x(j0:j0+s): one warp per later column.
__global__ void __launch_bounds__(kThreads) trsv_t_update_kernel(int64_t n, int64_t j0, int s, const double *R,
                                                               int64_t ldr, double *x) {
    __shared__ double xb[kTrsvBlock];
    if (threadIdx.x < s) xb[threadIdx.x] = x[j0 + threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t i = j0 + s + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    double acc = 0.0;
    for (int l = lane; l < s; l += 32) acc = fma(R[(j0 + l) + i * ldr], xb[l], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[i] -= acc;
}

// Solve R(j0:j0+s, j0:j0+s)^T y = x(j0:j0+s) in place (forward substitution).
__global__ void __launch_bounds__(kTrsvBlock) trsv_t_diag_kernel(int64_t j0, int s, const double *R, int64_t ldr,
                                                                double *x, long long *rankdef) {
    __shared__ double xs[kTrsvBlock];
    const int t = threadIdx.x;
    if (t < s) xs[t] = x[j0 + t];
    __syncthreads();
    for (int j = 0; j < s; ++j) {
        const double d = R[(j0 + j) + (j0 + j) * ldr];
        if (t == 0) {
            if (d == 0.0) atomicMin(rankdef, (long long)(j0 + j));
            xs[j] = xs[j] / d;
        }
        __syncthreads();
        if (t > j && t < s) xs[t] = fma(-R[(j0 + j) + (j0 + t) * ldr], xs[j], xs[t]);
        __syncthreads();
    }
    if (t < s) x[j0 + t] = xs[t];
}

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
    for (int64_t j = c0; j < c1; ++j) acc = fma(A[i + j * lda], x[j], acc);
    P[(int64_t)blockIdx.y * m + i] = acc;
}

__global__ void __launch_bounds__(kThreads) gemv_n_reduce_kernel(int64_t m, int nchunks, const double *P, double alpha,
                                                                double beta, double *y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += P[(int64_t)c * m + i];
    y[i] = (beta == 0.0) ? alpha * s : fma(beta, y[i], alpha * s);
}

// g(n) = alpha * A^T r + beta * g: one warp per column.
__global__ void __launch_bounds__(kThreads) gemv_t_kernel(int64_t m, int64_t n, const double *A, int64_t lda,
                                                         const double *r, double alpha, double beta, double *g,
                                                         int mask) {
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= n) return;
    double acc = 0.0;
    int64_t i0 = 0;
    if (mask == MASK_UNIT_LOWER) {
        if (lane == 0 && j < m) acc = r[j];
        i0 = j + 1;
    }
    for (int64_t i = i0 + lane; i < m; i += 32) acc = fma(A[i + j * lda], r[i], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) g[j] = (beta == 0.0) ? alpha * acc : fma(beta, g[j], alpha * acc);
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

// y = a * x + b * y (elementwise)
__global__ void __launch_bounds__(kThreads) axpby_kernel(int64_t n, double a, const double *x, double b, double *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (b == 0.0) ? a * x[i] : fma(a, x[i], b * y[i]);
}

unsigned grid_for(int64_t elems, int num_sms) {
    const int64_t want = (elems + kThreads - 1) / kThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
}

}  // namespace

gbqr_status fill_identity(const Exec &ex, int64_t m, int64_t n, double *Q, int64_t ldq) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    fill_identity_kernel<<<grid_for(m * n, ex.num_sms), kThreads, 0, ex.stream>>>(m, n, Q, ldq);
    return trace_end(ex, FAM_OTHER, 0.0, 8.0 * m * n);
}

gbqr_status zero_strict_lower(const Exec &ex, int64_t n, double *T, int64_t ldt) {
    if (n <= 1) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    zero_strict_lower_kernel<<<grid_for(n * n, ex.num_sms), kThreads, 0, ex.stream>>>(n, T, ldt);
    return trace_end(ex, FAM_OTHER, 0.0, 4.0 * n * n);
}

gbqr_status copy_matrix(const Exec &ex, int64_t m, int64_t n, const double *src, int64_t lds,
                        double *dst, int64_t ldd) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    copy_kernel<<<grid_for(m * n, ex.num_sms), kThreads, 0, ex.stream>>>(m, n, src, lds, dst, ldd);
    return trace_end(ex, FAM_OTHER, 0.0, 16.0 * m * n);
}

gbqr_status scan_nonfinite(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda,
                           unsigned long long *flag) {
    if (m <= 0 || n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    nonfinite_kernel<<<grid_for(m * n, ex.num_sms), kThreads, 0, ex.stream>>>(m, n, A, lda, flag);
    return trace_end(ex, FAM_OTHER, 0.0, 8.0 * m * n);
}

gbqr_status trsv_upper(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *x, long long *rankdef) {
    for (int64_t j0 = ((n - 1) / kTrsvBlock) * kTrsvBlock; j0 >= 0 && n > 0; j0 -= kTrsvBlock) {
        const int s = (int)std::min<int64_t>(kTrsvBlock, n - j0);
        trace_begin(ex, FAM_OTHER);
        trsv_diag_kernel<<<1, kTrsvBlock, 0, ex.stream>>>(j0, s, R, ldr, x, rankdef);
        gbqr_status st = trace_end(ex, FAM_OTHER, (double)s * s, 8.0 * s * s / 2);
        if (st != GBQR_OK) return st;
        if (j0 > 0) {
            trace_begin(ex, FAM_OTHER);
            trsv_update_kernel<<<(unsigned)((j0 + kThreads - 1) / kThreads), kThreads, 0, ex.stream>>>(j0, s, R, ldr, x);
            st = trace_end(ex, FAM_OTHER, 2.0 * j0 * s, 8.0 * j0 * s);
            if (st != GBQR_OK) return st;
        }
    }
    return GBQR_OK;
}

gbqr_status trsv_upper_t(const Exec &ex, int64_t n, const double *R, int64_t ldr, double *x, long long *rankdef) {
    for (int64_t j0 = 0; j0 < n; j0 += kTrsvBlock) {
        const int s = (int)std::min<int64_t>(kTrsvBlock, n - j0);
        trace_begin(ex, FAM_OTHER);
        trsv_t_diag_kernel<<<1, kTrsvBlock, 0, ex.stream>>>(j0, s, R, ldr, x, rankdef);
        gbqr_status st = trace_end(ex, FAM_OTHER, (double)s * s, 8.0 * s * s / 2);
        if (st != GBQR_OK) return st;
        const int64_t rest = n - j0 - s;
        if (rest > 0) {
            trace_begin(ex, FAM_OTHER);
            const int per = kThreads / 32;
            trsv_t_update_kernel<<<(unsigned)((rest + per - 1) / per), kThreads, 0, ex.stream>>>(n, j0, s, R, ldr, x);
            st = trace_end(ex, FAM_OTHER, 2.0 * rest * s, 8.0 * rest * s);
            if (st != GBQR_OK) return st;
        }
    }
    return GBQR_OK;
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
    trace_begin(ex, FAM_OTHER);
    gemv_n_partial_kernel<<<dim3((unsigned)rowblocks, (unsigned)nchunks), kThreads, 0, ex.stream>>>(m, n, chunk, A, lda, x, partial, mask);
    TRY_ST(trace_end(ex, FAM_OTHER, 2.0 * m * n, 8.0 * m * n));
    trace_begin(ex, FAM_OTHER);
    gemv_n_reduce_kernel<<<(unsigned)rowblocks, kThreads, 0, ex.stream>>>(m, (int)nchunks, partial, alpha, beta, y);
    return trace_end(ex, FAM_OTHER, (double)nchunks * m, 8.0 * (nchunks + 2) * m);
}

gbqr_status gemv_t(const Exec &ex, int64_t m, int64_t n, const double *A, int64_t lda, const double *r, double alpha,
                   double beta, double *g, int mask) {
    if (n <= 0) return GBQR_OK;
    const int per = kThreads / 32;
    trace_begin(ex, FAM_OTHER);
    gemv_t_kernel<<<(unsigned)((n + per - 1) / per), kThreads, 0, ex.stream>>>(m, n, A, lda, r, alpha, beta, g, mask);
    return trace_end(ex, FAM_OTHER, 2.0 * m * n, 8.0 * m * n);
}

gbqr_status norms2(const Exec &ex, int64_t n, const double *x, const double *y, double *out) {
    trace_begin(ex, FAM_OTHER);
    norms2_kernel<<<1, kThreads, 0, ex.stream>>>(n, x, y, out);
    return trace_end(ex, FAM_OTHER, 4.0 * n, 16.0 * n);
}

gbqr_status axpby(const Exec &ex, int64_t n, double a, const double *x, double b, double *y) {
    if (n <= 0) return GBQR_OK;
    trace_begin(ex, FAM_OTHER);
    axpby_kernel<<<grid_for(n, ex.num_sms), kThreads, 0, ex.stream>>>(n, a, x, b, y);
    return trace_end(ex, FAM_OTHER, 3.0 * n, 24.0 * n);
}

}  // namespace gbqr
