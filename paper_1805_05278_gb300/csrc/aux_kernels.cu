// Small HBM-bound kernels around the factorization: forming [I; 0] for the
// thin Q, zeroing the lower triangle of T, copies, the non-finite input scan,
// and the blocked back substitution R x = c of the least-squares solve.
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

}  // namespace gbqr
