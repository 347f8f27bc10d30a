// R x = c or R^T x = c for one vector, R upper triangular (n x n), with the
// inverses of R's 64 x 64 diagonal blocks precomputed (the mixed
// least-squares solve of Sections 2.1 and 2.3 uses them for its dozen
// triangular solves): one persistent launch instead of one launch per block.
//
// Blocks are solved in order (from the last for R, from the first for R^T).
// CTAs take blocks in that order from a ticket counter.  A CTA holding block
// i accumulates sum_j R_ij x_j over the blocks j solved before it as each is
// published (an acquire on a counter of solved blocks), with the next R block
// already loaded into registers while it waits; then x_i = Dinv_i (c_i - sum)
// and a release store publishes it.  So the chain from one block to the next
// is one 64 x 64 product with the block just solved, one with the inverse,
// and a release/acquire - the other updates run ahead, off the chain.  A CTA
// waits only for blocks with smaller tickets, which CTAs already running
// hold; every wait is bounded by %globaltimer and raises the context's
// timeout flag when it runs out.  Sums are in a fixed order, so the result
// does not depend on which CTA solved which block.
#include "common.cuh"

#include <algorithm>

namespace gbqr {
namespace {

constexpr int B = 64;                          // block size (the diagonal inverses' size)
static_assert(kThreads == 256, "4 quarter-columns x 64 rows, or 8 warps x 8 rows");

enum { kTicket = 0, kSolved = 1, kDone = 2, kAbort = 3, kNumCounters = 4 };

struct Chain {
    int64_t n, ldr;
    const double *R, *Dinv;
    double *x;
    int nblk, trans;
    unsigned *ctr;
    int *timeout;
    long long wait_ns;
};

__device__ __forceinline__ int ld_acquire(const unsigned *q) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(q) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *q, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(q), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every thread: wait until `want` blocks are solved (each thread acquires
// for itself; a warp's polls coalesce).  False when the launch is aborting.
__device__ bool wait_solved(const Chain &p, int want) {
    if (ld_acquire(p.ctr + kSolved) >= want) return true;
    const unsigned long long t0 = global_ns();
    unsigned ns = 32;
    while (ld_acquire(p.ctr + kSolved) < want) {
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

// Block order t -> block index.
__device__ __forceinline__ int block_of(const Chain &p, int t) { return p.trans ? t : p.nblk - 1 - t; }

// The 16 entries of the product block (rows of block i, columns of block j)
// a thread uses, clamped to valid addresses (rows or columns past n load a
// valid duplicate that meets a zero x or is never stored).
//   R:   thread (q = warp / 2, row rl = 32 (warp % 2) + lane), entries
//        R(64 i + rl, 64 j + 16 q + k), k < 16;
//   R^T: thread (warp w, lane l), entries R(64 j + l + 32 h, 64 i + 8 w + k'),
//        h < 2, k' < 8 (index 2 k' + h), read down R's columns.
__device__ __forceinline__ void load_block(const Chain &p, int i, int j, double (&v)[16]) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t last = p.n - 1;
    if (!p.trans) {
        const int64_t r = min((int64_t)B * i + 32 * (w & 1) + lane, last);
        const int64_t c0 = (int64_t)B * j + 16 * (w >> 1);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = __ldg(p.R + r + min(c0 + k, last) * p.ldr);
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t col = min((int64_t)B * i + 8 * w + k, last);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                v[2 * k + h] = __ldg(p.R + min((int64_t)B * j + lane + 32 * h, last) + col * p.ldr);
        }
    }
}

// acc += block (i, j) times x_j (x_j past n counts as zero).
__device__ __forceinline__ void fma_block(const Chain &p, int j, const double (&v)[16], double (&acc)[8]) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t base = (int64_t)B * j;
    if (!p.trans) {
        // one row, 16 columns: acc[0] carries the sum (two chains for latency)
        const int64_t c0 = base + 16 * (w >> 1);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const double xc = (c0 + k < p.n) ? __ldcg(p.x + c0 + k) : 0.0;
            acc[k & 1] = fma(v[k], xc, acc[k & 1]);
        }
    } else {
        // 8 columns of R, two rows each
        const double x0 = (base + lane < p.n) ? __ldcg(p.x + base + lane) : 0.0;
        const double x1 = (base + lane + 32 < p.n) ? __ldcg(p.x + base + lane + 32) : 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fma(v[2 * k + 1], x1, fma(v[2 * k], x0, acc[k]));
    }
}

__global__ void __launch_bounds__(kThreads, 1) trsv_chain_kernel(Chain p) {
    __shared__ double red[B * 33];       // R^T: per row the 32 lanes' partials (padded); R: 4 quarters x 64
    __shared__ double rhs[B];
    __shared__ int s_ticket;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_ticket = (int)atomicAdd(p.ctr + kTicket, 1u);
        __syncthreads();
        const int t = s_ticket;
        if (t >= p.nblk) break;
        const int i = block_of(p, t);
        const int64_t r0 = (int64_t)B * i;
        const int s = (int)min((int64_t)B, p.n - r0);
        const double *Di = p.Dinv + (size_t)i * B * B;
        // the inverse's entries this thread multiplies, loaded up front:
        //   R:   Dinv(rl, 16 q + k);   R^T: Dinv(l + 32 h, 8 w + k') (column 8w + k')
        double dv[16];
        if (!p.trans) {
#pragma unroll
            for (int k = 0; k < 16; ++k) dv[k] = __ldg(Di + (32 * (w & 1) + lane) + (16 * (w >> 1) + k) * B);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int h = 0; h < 2; ++h) dv[2 * k + h] = __ldg(Di + (lane + 32 * h) + (8 * w + k) * B);
        }
        double acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.0;
        bool ok = true;
        if (t > 0) {
            double v[16];
            load_block(p, i, block_of(p, 0), v);
            for (int u = 0; u < t && ok; ++u) {
                ok = wait_solved(p, u + 1);
                if (!ok) break;
                fma_block(p, block_of(p, u), v, acc);
                if (u + 1 < t) load_block(p, i, block_of(p, u + 1), v);   // in flight during the next wait
            }
        }
        if (__syncthreads_or(!ok)) break;                  // a wait ran out: every thread stops
        // rhs = c_i - sum, summed in a fixed order
        if (!p.trans) {
            red[(w >> 1) * B + 32 * (w & 1) + lane] = acc[0] + acc[1];
            __syncthreads();
            if (tid < B) {
                const double sum = (red[tid] + red[B + tid]) + (red[2 * B + tid] + red[3 * B + tid]);
                rhs[tid] = (tid < s) ? __ldcg(p.x + r0 + tid) - sum : 0.0;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) red[(8 * w + k) * 33 + lane] = acc[k];
            __syncthreads();
            if (tid < B) {
                const double *row = red + tid * 33;
                double a = row[0], b = row[16];
#pragma unroll
                for (int l = 1; l < 16; ++l) {
                    a += row[l];
                    b += row[16 + l];
                }
                rhs[tid] = (tid < s) ? __ldcg(p.x + r0 + tid) - (a + b) : 0.0;
            }
        }
        __syncthreads();
        // x_i = Dinv_i rhs (Dinv upper triangular; zero below its diagonal)
        if (!p.trans) {
            double a0 = 0.0, a1 = 0.0;
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                a0 = fma(dv[k], rhs[16 * (w >> 1) + k], a0);
                a1 = fma(dv[k + 1], rhs[16 * (w >> 1) + k + 1], a1);
            }
            red[(w >> 1) * B + 32 * (w & 1) + lane] = a0 + a1;
            __syncthreads();
            if (tid < s) p.x[r0 + tid] = (red[tid] + red[B + tid]) + (red[2 * B + tid] + red[3 * B + tid]);
        } else {
            // x_r = sum_c Dinv(c, r) rhs_c: this thread's columns 8w + k', rows l, l + 32
            const double r0v = rhs[lane], r1v = rhs[lane + 32];
#pragma unroll
            for (int k = 0; k < 8; ++k) red[(8 * w + k) * 33 + lane] = fma(dv[2 * k + 1], r1v, dv[2 * k] * r0v);
            __syncthreads();
            if (tid < B) {
                const double *row = red + tid * 33;
                double a = row[0], b = row[16];
#pragma unroll
                for (int l = 1; l < 16; ++l) {
                    a += row[l];
                    b += row[16 + l];
                }
                if (tid < s) p.x[r0 + tid] = a + b;
            }
        }
        __syncthreads();
        if (tid == 0) st_release(p.ctr + kSolved, t + 1);   // publishes x_i (the CTA's stores came before the barrier)
    }
    // the last CTA out resets the counters for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(p.ctr + kDone, 1u) == gridDim.x - 1) {
            p.ctr[kTicket] = 0u;
            p.ctr[kSolved] = 0u;
            p.ctr[kAbort] = 0u;
            __threadfence();
            p.ctr[kDone] = 0u;
        }
    }
}

}  // namespace

gbqr_status trsv_chain(const Exec &ex, bool trans, int64_t n, const double *R, int64_t ldr, double *x,
                       const double *Dinv, unsigned *counters, size_t ncounters, int *timeout) {
    if (n <= 0) return GBQR_OK;
    if (!R || !x || !Dinv || !timeout || ldr < n) return GBQR_EINVAL;
    if (ncounters < kNumCounters) return GBQR_ENOMEM;
    const int64_t nblk = (n + B - 1) / B;
    if (nblk > 0x3fffffff) return GBQR_EUNSUPPORTED;
    Chain p;
    p.n = n; p.ldr = ldr; p.R = R; p.Dinv = Dinv; p.x = x;
    p.nblk = (int)nblk; p.trans = trans ? 1 : 0;
    p.ctr = counters; p.timeout = timeout;
    p.wait_ns = 5000000000ll;   // 5 s: far beyond the whole chain
    const unsigned grid = (unsigned)std::min<int64_t>(nblk, ex.num_sms);
    trace_begin(ex, FAM_TRSV);
    trsv_chain_kernel<<<grid, kThreads, 0, ex.stream>>>(p);
    return trace_end(ex, FAM_TRSV, (double)n * n + 2.0 * nblk * B * B, 4.0 * (double)n * n + 8.0 * nblk * B * B);
}

}  // namespace gbqr

// Failure-detection self-test: one CTA is handed the second block of a
// two-block solve (the ticket counter starts at 1), so the first block is
// never solved and its bounded wait must run out.
extern "C" GBQR_API gbqr_status gbqr_selftest_chain_wait(int device, int wait_ms, int *completed) {
    using namespace gbqr;
    if (!completed || wait_ms < 1 || wait_ms > 10000) return GBQR_EINVAL;
    *completed = -1;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    const int64_t n = 2 * B;
    // [R (n x n) | Dinv (2 blocks) | x (n) | counters (4) + timeout flag]
    const size_t nR = (size_t)n * n, nD = 2 * (size_t)B * B;
    const size_t bytes = 8 * (nR + nD + n) + 64;
    char *d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
    double *R = reinterpret_cast<double *>(d), *Dv = R + nR, *x = Dv + nD;
    unsigned *ctr = reinterpret_cast<unsigned *>(x + n);
    int *flag = reinterpret_cast<int *>(ctr + kNumCounters);
    gbqr_status st = GBQR_OK;
    double xh[2 * B];
    for (int i = 0; i < n; ++i) xh[i] = 1.0;
    const unsigned one = 1u;
    if (cudaMemset(d, 0, bytes) != cudaSuccess || cudaMemcpy(x, xh, sizeof xh, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctr + kTicket, &one, sizeof one, cudaMemcpyHostToDevice) != cudaSuccess)
        st = GBQR_ECUDA;
    int h = 0;
    unsigned left[kNumCounters] = {1u, 1u, 1u, 1u};
    if (st == GBQR_OK) {
        Chain p;
        p.n = n; p.ldr = n; p.R = R; p.Dinv = Dv; p.x = x;
        p.nblk = 2; p.trans = 0;
        p.ctr = ctr; p.timeout = flag;
        p.wait_ns = (long long)wait_ms * 1000000ll;
        trsv_chain_kernel<<<1, kThreads>>>(p);
        if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&h, flag, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(xh, x, sizeof xh, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(left, ctr, sizeof left, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = GBQR_ECUDA;
    }
    cudaFree(d);
    if (st != GBQR_OK) return st;
    // blocks solved: the waiting block (rows 0..63) would have been overwritten
    int solved = 0;
    for (int i = 0; i < B; ++i) solved |= (xh[i] != 1.0) ? 1 : 0;
    *completed = solved;
    for (int i = 0; i < kNumCounters; ++i)
        if (left[i] != 0u) return GBQR_ECUDA;   // the counters must be left zero for the next launch
    return h ? GBQR_ETIMEOUT : GBQR_OK;
}
