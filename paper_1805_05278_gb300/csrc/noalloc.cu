// Allocation-free tall-skinny QR: the TSQR kernels of the base case, with
// their reduction-tree scratch in a fixed static device array instead of a
// workspace, and no context.
//
// Who needs it: callers that cannot call cudaMalloc.  cudaMalloc/cudaFree can
// synchronise the whole device, which a latency-critical pipeline running
// other streams cannot afford; a framework whose caching allocator owns the
// device memory budget must not see memory appear behind its back; and some
// deployments must fix their device footprint when the library is loaded.
// Such a caller passes its input and outputs and nothing else.
//
// The array below is part of the module image: every GPU that loads this
// library holds kStaticScratchBytes of device memory for it until the
// process exits.  With lazy module loading (CUDA's default) the module, and
// with it the array, is loaded on a device by the first call there, which may
// then allocate and synchronise; callers that must avoid that make one call
// at initialisation.  All calls share it and it keeps the last call's contents,
// so each call clears the part that must start at zero (the tree's arrival
// counters).  Calls that overlap on the GPU (different streams, or different
// host threads) race on the array.
#include "common.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;   // 16 MiB per device
constexpr int kStaticMaxCols = 32;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_tsqr_scratch[kStaticScratchBytes];

struct DeviceScratch {
    std::once_flag once;
    void *ptr = nullptr;                 // device address of g_tsqr_scratch
    cudaError_t err = cudaErrorNotReady;
};
DeviceScratch g_scratch[kMaxDevices];

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Bytes of the static array that plan `pl` uses, in the carving order below.
size_t scratch_bytes(const gbqr::TsqrPlan &pl) {
    return align256(pl.nR * 8) + align256(pl.nT * 8) + align256(pl.nY * 8) + align256(pl.nX * 8) +
           align256(pl.ncount * 4);
}

// The base case's own plan: default leaf height and the adaptive fan-out of
// gbqr_factor.  No other plan needs less scratch: the default already takes
// the fewest leaves the kernels' shared memory allows once a panel needs more
// than one leaf per SM (leaf height is capped at about 600 rows at n = 32),
// and fewer leaves means fewer tree nodes.  With n = 32 the 16 MiB hold
// about 650 leaves, so m up to about 400,000 rows.
bool plan_that_fits(int64_t m, int n, gbqr::TsqrPlan *out) {
    gbqr::TsqrPlan pl;
    if (!gbqr::tsqr_plan(m, n, 0, 0, 0, &pl)) return false;
    if (scratch_bytes(pl) > kStaticScratchBytes) return false;
    *out = pl;
    return true;
}

}  // namespace

extern "C" GBQR_API gbqr_status gbqr_tsqr_static(int64_t m, int64_t n, double *A, int64_t lda,
                                                 double *T, int64_t ldt, void *cuda_stream) {
    using namespace gbqr;
    // size checks first: they need no device and reject before any CUDA call
    if (m < 0 || n < 0 || m < n) return GBQR_EINVAL;
    if (n > kStaticMaxCols) return GBQR_EINVAL;
    if (lda < std::max<int64_t>(1, m) || ldt < std::max<int64_t>(1, n)) return GBQR_EINVAL;
    if (n == 0) return GBQR_OK;
    if (!A || !T) return GBQR_EINVAL;
    TsqrPlan pl;
    if (!plan_that_fits(m, (int)n, &pl)) return GBQR_EINVAL;   // tree exceeds the static scratch

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GBQR_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return GBQR_EUNSUPPORTED;
    // Set-up, once per device, with that device current: the host-side name
    // of a __device__ array is not a device address, so ask the runtime.
    DeviceScratch &ds = g_scratch[dev];
    std::call_once(ds.once, [&ds] { ds.err = cudaGetSymbolAddress(&ds.ptr, g_tsqr_scratch); });
    if (ds.err != cudaSuccess || !ds.ptr) return GBQR_ECUDA;

    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GBQR_ECUDA;
    char *base = (char *)ds.ptr;
    TsqrWork work;
    size_t off = 0;
    work.R = (double *)(base + off); off += align256(pl.nR * 8);
    work.T = (double *)(base + off); off += align256(pl.nT * 8);
    work.Y = (double *)(base + off); off += align256(pl.nY * 8);
    work.X = (double *)(base + off); off += align256(pl.nX * 8);
    work.counters = (unsigned *)(base + off);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(work.counters, 0, pl.ncount * sizeof(unsigned), stream) != cudaSuccess) return GBQR_ECUDA;
    Exec ex;
    ex.stream = stream;
    ex.num_sms = sms;
    ex.device = dev;
    return tsqr_run(ex, pl, A, lda, T, ldt, work);
}
