// FP64 throughput probe: the roofline denominator of the FP64 path.
// Not a step of the QR method; it measures what this GPU's FP64 units
// deliver, on the CUDA cores (DFMA) and on the tensor cores through the
// legacy double-precision mma.sync (DMMA), so that kernels can be reported
// as a fraction of a measured peak.
#include "common.cuh"

namespace gbqr {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) dfma_probe_kernel(int iters, double seed, double *out) {
    double acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed * (threadIdx.x + c + 1);
    const double a = 1.0 + 1e-12 * seed, b = 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == 12345.678) out[0] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(kThreads) dmma_probe_kernel(int iters, double seed, double *out) {
    double d[kChains / 2][2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) { d[c][0] = seed * (threadIdx.x + c); d[c][1] = seed; }
    const double a = 1.0 + 1e-12 * seed, b = 1e-9 * (threadIdx.x & 3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) {
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(d[c][0]), "+d"(d[c][1])
                         : "d"(a), "d"(b));
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += d[c][0] + d[c][1];
    if (s == 12345.678) out[0] = s;
}

// One CTA of `warps` warps, each running a chain of dependent FP64
// operations; clock64 per warp.  op 0: DFMA, 1: sqrt, 2: reciprocal.
constexpr int kLatIters = 256;

__global__ void latency_probe_kernel(int op, double *out, long long *cyc) {
    double x = 1.0 + threadIdx.x * 1e-9;
    const double a = 0.9999999, b = 1e-7;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < kLatIters; ++i) {
        if (op == 0) x = fma(x, a, b);
        else if (op == 1) x = sqrt(x + b);
        else x = 1.0 / (x + b);
    }
    const long long t1 = clock64();
    out[threadIdx.x] = x;
    if ((threadIdx.x & 31) == 0) cyc[threadIdx.x >> 5] = t1 - t0;
}

}  // namespace
}  // namespace gbqr

struct gbqr_ctx;

extern "C" GBQR_API gbqr_status gbqr_fp64_issue_cycles(int device, int op, int warps, double *cycles) {
    using namespace gbqr;
    if (!cycles || op < 0 || op > 2 || warps < 1 || warps > 32) return GBQR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    double *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&out, 1024 * sizeof(double)) != cudaSuccess) return GBQR_ENOMEM;
    if (cudaMalloc(&cyc, 32 * sizeof(long long)) != cudaSuccess) { cudaFree(out); return GBQR_ENOMEM; }
    long long h[32] = {0};
    gbqr_status st = GBQR_OK;
    for (int rep = 0; rep < 2 && st == GBQR_OK; ++rep) {
        latency_probe_kernel<<<1, warps * 32>>>(op, out, cyc);
        if (cudaDeviceSynchronize() != cudaSuccess) st = GBQR_ECUDA;
    }
    if (st == GBQR_OK && cudaMemcpy(h, cyc, warps * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = GBQR_ECUDA;
    long long mx = 0;
    for (int i = 0; i < warps; ++i) mx = h[i] > mx ? h[i] : mx;
    *cycles = (double)mx / kLatIters;
    cudaFree(out);
    cudaFree(cyc);
    return st;
}

extern "C" GBQR_API gbqr_status gbqr_fp64_peak(int device, int kind, int iters, double *tflops) {
    using namespace gbqr;
    if (!tflops || (kind != 0 && kind != 1) || iters < 1) return GBQR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return GBQR_ECUDA;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return GBQR_ENOMEM;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { cudaFree(out); return GBQR_ECUDA; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * 8;
    double best_ms = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0, s);
        if (kind == 0) dfma_probe_kernel<<<blocks, kThreads, 0, s>>>(iters, 1.0 + rep, out);
        else dmma_probe_kernel<<<blocks, kThreads, 0, s>>>(iters, 1.0 + rep, out);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best_ms) best_ms = ms;   // first launch is a warm-up
    }
    gbqr_status st = cudaGetLastError() == cudaSuccess ? GBQR_OK : GBQR_ECUDA;
    const double threads = (double)blocks * kThreads;
    // DFMA: kChains FMAs per iteration per thread; DMMA: kChains/2 m8n8k4
    // products (256 FMAs per warp each) per iteration per warp.
    const double flops = (kind == 0) ? 2.0 * kChains * (double)iters * threads
                                     : 2.0 * 256.0 * (kChains / 2) * (double)iters * (threads / 32.0);
    *tflops = (st == GBQR_OK) ? flops / (best_ms * 1e-3) / 1e12 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(out);
    return st;
}
