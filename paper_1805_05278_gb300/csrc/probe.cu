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

}  // namespace
}  // namespace gbqr

struct gbqr_ctx;

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
