// Split-BF16 GEMM on the 5th-generation tensor cores (tcgen05), for the
// mixed-precision form of the update products of QR (Algorithm 2 and the
// right-looking update of Section 8.4):
//
//   C (FP64, M x N) = alpha * op(A) * B + beta * C,   op(A) = A or A^T,
//
// with each FP64 operand split into s <= 3 BF16 slices x = x_1 + x_2 + x_3
// (x_1 = bf16(x), x_2 = bf16(x - x_1), ...), and the products x_i y_j with
// i + j <= s + 1 (6 products for s = 3) accumulated in FP32 in tensor memory:
// FP32-level accuracy from BF16 tensor cores.
//
// Kernel structure (one CTA per 128 x BN output tile, 6 warps):
//   warp 0      TMA producer: 3-D tensor loads (K x rows x slices) of BF16
//               tiles, 128-byte swizzle, into a ring of stages guarded by
//               mbarriers (full: bytes landed; empty: MMAs done reading).
//               Long K (at least 4 K tiles per CTA): K-major - per K step one
//               load of every slice of the 128 x 64 A tile and one of every
//               slice of the BN x 64 B tile, so each slice tile is read once
//               (2-4 stages).  Short K: product-major - per product and K
//               step one A slice tile and one B slice tile (4 stages): the
//               first MMA waits for one small stage, and re-reads of the few
//               tiles come from L2.
//   warp 1      allocates TMEM; one thread issues tcgen05.mma kind::f16
//               (M = 128, N = BN, K = 16 per instruction) for every product
//               of every stage, then tcgen05.commit.  The leading product
//               x_1 y_1 accumulates in one TMEM accumulator and the smaller
//               ones in a second, so their low-order bits are not rounded
//               away against the leading product's running sum at every K
//               step; the epilogue adds the two once.
//   warps 2-5   epilogue: tcgen05.ld the FP32 accumulators (warp w reads TMEM
//               lanes 32*(w%4) .. +31), combine into C in FP64 (or write FP32
//               split-K partials).  Each FP64 instruction takes a warp about
//               64 cycles here, so the epilogue spends as few as it can: the
//               C -= update is one conversion and one subtraction per entry.
// Every mbarrier wait is bounded (about 2 s by %globaltimer); on timeout the
// kernel raises an error flag, stops issuing work, drains what it issued and
// frees its TMEM.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

namespace gbqr {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;          // one 128-byte swizzle row of BF16
constexpr int TC_MAX_STAGES = 4;
constexpr size_t TC_SMEM_LIMIT = 225 * 1024;   // dynamic shared memory a CTA may take
constexpr int TC_THREADS = 192;
constexpr uint32_t A_TILE_BYTES = TC_BM * TC_BK * 2;

struct TcParams {
    int M, N, K;
    int ktiles_per_split;
    int nsplit;              // slices per operand
    int kmajor;              // 1: every slice per K step (box depth nsplit); 0: one product per stage
    int stages;              // ring depth
    int npairs;
    int pair_a[6], pair_b[6];
    double *C; int64_t ldc;
    double alpha, beta;
    float *partial;          // split-K partials: [z][M x N] column-major
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity; give up after ~2 s or as soon as
// another thread of the grid has raised the error flag.
__device__ bool mbar_wait(uint32_t a, uint32_t parity, int *err) {
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (*(volatile int *)err) return false;
        if (global_ns() - t0 > 2000000000ull) {
            atomicExch(err, 1);
            return false;
        }
    }
}

// The bounded wait above on a barrier nothing ever arrives at: it must give
// up after its time limit, raise the error flag and let the kernel return.
__global__ void wait_selftest_kernel(int *err, int *completed) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) *completed = mbar_wait(a, 0u, err) ? 1 : 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major BF16 tile written by TMA with
// 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);   // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams p) {
    constexpr uint32_t B_TILE_BYTES = BN * TC_BK * 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NS = p.stages;
    const int depth = p.kmajor ? p.nsplit : 1;   // slice tiles per operand in a stage
    const uint32_t a_stage = (uint32_t)depth * A_TILE_BYTES, b_stage = (uint32_t)depth * B_TILE_BYTES;
    uint8_t *sA = smem;
    uint8_t *sB = sA + NS * a_stage;
    uint64_t *bars = (uint64_t *)(sB + NS * b_stage);   // full[S], empty[S], done
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * NS + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN, z = blockIdx.z;
    const int ktiles = (p.K + TC_BK - 1) / TC_BK;
    const int kt0 = z * p.ktiles_per_split;
    const int nk = max(0, min(ktiles, kt0 + p.ktiles_per_split) - kt0);
    const int total = p.kmajor ? nk : nk * p.npairs;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + NS), done = smem_u32(bars + 2 * NS);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // two accumulators (leading product, the others) when there are several products
    const uint32_t tcols = p.npairs > 1 ? 2 * BN : BN;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int it = 0; it < total; ++it) {
                const int s = it % NS, r = it / NS;
                if (!mbar_wait(empty0 + 8 * s, (uint32_t)((r & 1) ^ 1), p.err)) break;
                const int pair = p.kmajor ? 0 : it / nk, kt = kt0 + (p.kmajor ? it : it % nk);
                mbar_expect_tx(full0 + 8 * s, a_stage + b_stage);
                tma_load_3d(smem_u32(sA + s * a_stage), &tmA, kt * TC_BK, m0, p.kmajor ? 0 : p.pair_a[pair],
                            full0 + 8 * s);
                tma_load_3d(smem_u32(sB + s * b_stage), &tmB, kt * TC_BK, n0, p.kmajor ? 0 : p.pair_b[pair],
                            full0 + 8 * s);
                issued = it + 1;
            }
            // after an abort, let the loads already issued land before the CTA exits
            if (issued < total)
                for (int it = max(0, issued - NS); it < issued; ++it)
                    mbar_wait(full0 + 8 * (it % NS), (uint32_t)((it / NS) & 1), p.err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_BM, BN);
            for (int it = 0; it < total; ++it) {
                const int s = it % NS, r = it / NS;
                if (!mbar_wait(full0 + 8 * s, (uint32_t)(r & 1), p.err)) break;
                tc_fence_after();
                // the products of this stage: the smaller ones into the second
                // accumulator, the leading one (last in the list) into the first
                const int q0 = p.kmajor ? 0 : it / nk, q1 = p.kmajor ? p.npairs : q0 + 1;
                const int kstep = p.kmajor ? it : it % nk;
                for (int q = q0; q < q1; ++q) {
                    const int ai = p.kmajor ? p.pair_a[q] : 0, bi = p.kmajor ? p.pair_b[q] : 0;
                    const uint64_t ad = sw128_desc(smem_u32(sA + s * a_stage + ai * A_TILE_BYTES));
                    const uint64_t bd = sw128_desc(smem_u32(sB + s * b_stage + bi * B_TILE_BYTES));
                    const bool lead = q == p.npairs - 1;
                    const uint32_t acc_addr = lead ? tmem : tmem + (uint32_t)BN;
                    // the first MMA into each accumulator overwrites it
                    const bool first = kstep == 0 && (lead || q == 0);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk)
                        mma_bf16(acc_addr, ad + 2 * kk, bd + 2 * kk, idesc, (!first || kk > 0) ? 1u : 0u);
                }
                mma_commit(empty0 + 8 * s);
            }
            mma_commit(done);   // arrives once every MMA issued above has completed
        }
    } else {
        const int q = warp & 3;             // TMEM lane quadrant of this warp
        const int row = q * 32 + lane;
        const bool ok = mbar_wait(done, 0u, p.err);
        tc_fence_after();
        const int m = m0 + row;
        // Each thread owns one row of the tile: per 32-column chunk, all 32 C
        // loads are issued before any store, so a warp keeps 32 coalesced
        // 256-byte loads in flight (one at a time, the FP64 read-modify-write
        // of C is latency-bound at a few GB/s per SM).
#pragma unroll 1
        for (int chunk = 0; chunk < BN / 32; ++chunk) {
            uint32_t v[32], v2[32];
            if (total > 0) tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(chunk * 32), v);
            if (total > 0 && p.npairs > 1)
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(BN + chunk * 32), v2);
            if (!ok || m >= p.M) continue;
            const int nbase = n0 + chunk * 32;
            const int cnt = min(32, p.N - nbase);
            if (cnt <= 0) continue;
            if (p.partial) {
                float *pp = p.partial + (size_t)z * p.M * p.N + m + (size_t)nbase * p.M;
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < cnt)
                        pp[(size_t)c * p.M] = (total > 0) ? __uint_as_float(v[c]) +
                                                                (p.npairs > 1 ? __uint_as_float(v2[c]) : 0.0f)
                                                          : 0.0f;
            } else {
                double *cp = p.C + m + (size_t)nbase * p.ldc;
                double cv[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) cv[c] = (p.beta != 0.0 && c < cnt) ? cp[(size_t)c * p.ldc] : 0.0;
                const bool sub = p.beta == 1.0 && p.alpha == -1.0, plain = p.beta == 0.0 && p.alpha == 1.0;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    if (c < cnt) {
                        const float f = (total > 0) ? __uint_as_float(v[c]) + (p.npairs > 1 ? __uint_as_float(v2[c]) : 0.0f)
                                                    : 0.0f;
                        const double d = (double)f;
                        double out;
                        if (sub) out = cv[c] - d;
                        else if (plain) out = d;
                        else if (p.beta == 0.0) out = p.alpha * d;
                        else out = fma(p.beta, cv[c], p.alpha * d);
                        cp[(size_t)c * p.ldc] = out;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
    }
}

// C = beta * C + alpha * sum_z P[z] (FP64 accumulation of FP32 partials).
// 2-D grid: x over rows m, y over columns n (no 64-bit division per entry).
__global__ void __launch_bounds__(kThreads) tc_reduce_kernel(int M, int N, int S, const float *P, double *C,
                                                           int64_t ldc, double alpha, double beta) {
    const int64_t total = (int64_t)M * N;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    for (int n = blockIdx.y; n < N; n += gridDim.y) {
        const int64_t e = m + (int64_t)n * M;
        double s = 0.0;
        for (int z = 0; z < S; ++z) s += (double)P[(size_t)z * total + e];
        double *cp = C + m + (int64_t)n * ldc;
        double out;
        if (beta == 0.0) out = (alpha == 1.0) ? s : alpha * s;
        else if (beta == 1.0 && alpha == -1.0) out = *cp - s;
        else out = fma(beta, *cp, alpha * s);
        *cp = out;
    }
}

__device__ __forceinline__ double masked_at(const double *X, int64_t ld, int64_t r, int64_t c, int mask) {
    if (mask == MASK_UNIT_LOWER) {
        if (r < c) return 0.0;
        if (r == c) return 1.0;
    } else if (mask == MASK_UPPER) {
        if (r > c) return 0.0;
    }
    return X[r + c * ld];
}

// Slices of x: the s <= 3 BF16 pieces carry 24 significant bits between
// them, which FP32 holds, so the recurrence r -= bf16(r) runs in FP32 (exact
// subtractions; this part issues FP32 at 64x its FP64 rate) after one
// rounding of x to FP32.
__device__ __forceinline__ void split_slices(double x, int ns, __nv_bfloat16 (&h)[3]) {
    float r = (float)x;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        h[s] = __float2bfloat16_rn(r);
        r -= __bfloat162float(h[s]);
        if (s + 1 >= ns) break;
    }
}

__device__ __forceinline__ void split_store(double x, int ns, __nv_bfloat16 *dst, size_t slice_stride) {
    __nv_bfloat16 h[3];
    split_slices(x, ns, h);
    for (int s = 0; s < ns; ++s) dst[s * slice_stride] = h[s];
}

// BF16 slices of an FP64 operand, K-major for the MMA: operand row i holds
// K contiguous values at dst[i * ldd + k] (ldd a multiple of 8).
//   !transpose: operand (i, k) = stored (k, i)   (stored K x R, column-major)
//    transpose: operand (i, k) = stored (i, k)   (stored R x K, column-major)
// Entries k in [K, ldd) are zero.  mask applies to the stored coordinates.
// 2-D grid: x over K in chunks of 4 consecutive entries per thread (one
// 8-byte store of four BF16 per slice; ldd is a multiple of 8), y over rows.
__global__ void __launch_bounds__(kThreads) split_plain_kernel(int64_t K, int64_t R, const double *src, int64_t lds,
                                                             int mask, int ns, __nv_bfloat16 *dst, int64_t ldd,
                                                             size_t slice_stride) {
    const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (k0 >= ldd) return;
    for (int64_t i = blockIdx.y; i < R; i += gridDim.y) {
        __nv_bfloat16 h[4][3];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t k = k0 + q;
            const double x = (k < K) ? masked_at(src, lds, k, i, mask) : 0.0;
            split_slices(x, ns, h[q]);
        }
        for (int s = 0; s < ns; ++s) {
            __nv_bfloat162 lo = __halves2bfloat162(h[0][s], h[1][s]);
            __nv_bfloat162 hi = __halves2bfloat162(h[2][s], h[3][s]);
            uint2 v;
            v.x = *reinterpret_cast<uint32_t *>(&lo);
            v.y = *reinterpret_cast<uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(dst + s * slice_stride + i * ldd + k0) = v;
        }
    }
}

__global__ void __launch_bounds__(kThreads) split_transpose_kernel(int64_t K, int64_t R, const double *src,
                                                                 int64_t lds, int mask, int ns,
                                                                 __nv_bfloat16 *dst, int64_t ldd,
                                                                 size_t slice_stride) {
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int y = ty; y < 32; y += 8) {
        const int64_t i = i0 + tx, k = k0 + y;                 // read along i (contiguous in stored column k)
        tile[y][tx] = (i < R && k < K) ? masked_at(src, lds, i, k, mask) : 0.0;
    }
    __syncthreads();
    for (int y = ty; y < 32; y += 8) {
        const int64_t i = i0 + y, k = k0 + tx;                 // write along k (contiguous in dst row i)
        if (i < R && k < ldd) split_store(tile[tx][y], ns, dst + i * ldd + k, slice_stride);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D map over BF16 slices: dims (K, rows, slices), row stride ldd elements;
// one box holds box_slices slices of a 64 x box_rows tile.
bool make_map(CUtensorMap *map, const void *base, int64_t K, int64_t rows, int slices, int64_t ldd, int box_rows,
              int box_slices) {
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)ldd * 2, (cuuint64_t)ldd * (cuuint64_t)rows * 2};
    cuuint32_t box[3] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows, (cuuint32_t)box_slices};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// depth: slice tiles per operand in a stage (nsplit when K-major, else 1)
size_t tc_stage_bytes(int BN, int depth) { return (size_t)depth * (A_TILE_BYTES + (size_t)BN * TC_BK * 2); }
// Deepest ring (at most TC_MAX_STAGES) that fits the shared-memory limit.
int tc_stages(int BN, int depth) {
    const size_t fixed = 1024 + 256;
    return (int)std::min<size_t>(TC_MAX_STAGES, (TC_SMEM_LIMIT - fixed) / tc_stage_bytes(BN, depth));
}
size_t tc_smem_bytes(int BN, int depth) { return 1024 + tc_stages(BN, depth) * tc_stage_bytes(BN, depth) + 256; }

int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }

}  // namespace

void *tensor_map_encoder() { return (void *)encode_fn(); }

size_t tc_gemm_scratch_bytes(int64_t M, int64_t N, int64_t K, int num_sms) {
    const int64_t ldk = pad8(std::max<int64_t>(K, 1));
    size_t b = 0;
    b += (size_t)3 * std::max<int64_t>(M, 1) * ldk * 2 + 256;     // A slices
    b += (size_t)3 * std::max<int64_t>(N, 1) * ldk * 2 + 256;     // B slices
    b += (size_t)4 * num_sms * TC_BM * 128 * 4 + 256;            // split-K partials (bounded below)
    return b;
}

gbqr_status tc_gemm(const Exec &ex, const TcGemmOp &op, const TcScratch &sc) {
    if (op.M <= 0 || op.N <= 0) return GBQR_OK;
    if (op.nsplit < 1 || op.nsplit > 3) return GBQR_EINVAL;
    if (op.M > (1 << 30) || op.N > (1 << 30) || op.K > (1 << 30)) return GBQR_EUNSUPPORTED;
    const int64_t K = std::max<int64_t>(op.K, 1), ldk = pad8(K);
    const size_t sa = (size_t)op.M * ldk, sb = (size_t)op.N * ldk;
    const size_t need = ((size_t)3 * sa * 2 + 255) / 256 * 256 + ((size_t)3 * sb * 2 + 255) / 256 * 256;
    if (!sc.base || need > sc.bytes) return GBQR_ENOMEM;
    __nv_bfloat16 *As = (__nv_bfloat16 *)sc.base;
    __nv_bfloat16 *Bs = (__nv_bfloat16 *)((char *)sc.base + ((size_t)3 * sa * 2 + 255) / 256 * 256);
    float *partial = (float *)((char *)Bs + ((size_t)3 * sb * 2 + 255) / 256 * 256);
    const size_t partial_cap = (sc.bytes - need) / 4;

    // slices of op(A) (rows M) and of B (rows N), K-major
    trace_begin(ex, FAM_OTHER);
    auto plain_grid = [&](int64_t rows) {
        return dim3((unsigned)((ldk / 4 + kThreads - 1) / kThreads), (unsigned)std::min<int64_t>(std::max<int64_t>(rows, 1), 65535));
    };
    if (op.ta) {
        split_plain_kernel<<<plain_grid(op.M), kThreads, 0, ex.stream>>>(op.K, op.M, op.A, op.lda, op.maskA, op.nsplit,
                                                                          As, ldk, sa);
    } else {
        dim3 g((unsigned)((ldk + 31) / 32), (unsigned)((op.M + 31) / 32));
        split_transpose_kernel<<<g, kThreads, 0, ex.stream>>>(op.K, op.M, op.A, op.lda, op.maskA, op.nsplit, As, ldk, sa);
    }
    TRY_ST(trace_end(ex, FAM_OTHER, 0.0, (8.0 + 2.0 * op.nsplit) * op.M * K));
    trace_begin(ex, FAM_OTHER);
    split_plain_kernel<<<plain_grid(op.N), kThreads, 0, ex.stream>>>(op.K, op.N, op.B, op.ldb, op.maskB, op.nsplit,
                                                                      Bs, ldk, sb);
    TRY_ST(trace_end(ex, FAM_OTHER, 0.0, (8.0 + 2.0 * op.nsplit) * op.N * K));

    // tile shape and split-K
    const int BN = (((op.M + TC_BM - 1) / TC_BM) * ((op.N + 127) / 128) >= ex.num_sms) ? 128 : 64;
    const int64_t tm = (op.M + TC_BM - 1) / TC_BM, tn = (op.N + BN - 1) / BN;
    const int ktiles = (int)((K + TC_BK - 1) / TC_BK);
    int S = 1;
    // split K until the grid covers the SMs (the partials are summed in a
    // fixed order by tc_reduce_kernel, so the result does not depend on timing)
    if (tm * tn < ex.num_sms) S = (int)std::min<int64_t>({(ex.num_sms + tm * tn - 1) / (tm * tn), (int64_t)ktiles, 64});
    while (S > 1 && (size_t)S * op.M * op.N > partial_cap) --S;
    const int per = (ktiles + S - 1) / S;
    S = (ktiles + per - 1) / per;   // every split gets at least one K tile

    TcParams p;
    p.M = (int)op.M; p.N = (int)op.N; p.K = (int)K;
    p.ktiles_per_split = per;
    p.nsplit = op.nsplit;
    p.kmajor = (op.nsplit > 1 && per >= 4) ? 1 : 0;
    const int depth = p.kmajor ? op.nsplit : 1;
    p.stages = tc_stages(BN, depth);
    static const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
    p.npairs = op.nsplit == 1 ? 1 : (op.nsplit == 2 ? 3 : 6);
    // smaller products first, the leading one last
    for (int q = 0; q < p.npairs; ++q) {
        p.pair_a[q] = pa[p.npairs - 1 - q];
        p.pair_b[q] = pb[p.npairs - 1 - q];
    }
    p.C = op.C; p.ldc = op.ldc; p.alpha = op.alpha; p.beta = op.beta;
    p.partial = (S > 1) ? partial : nullptr;
    p.err = sc.err;

    CUtensorMap mA, mB;
    if (!make_map(&mA, As, K, op.M, op.nsplit, ldk, TC_BM, depth) || !make_map(&mB, Bs, K, op.N, op.nsplit, ldk, BN, depth))
        return GBQR_ECUDA;
    const size_t smem = tc_smem_bytes(BN, depth);
    // per device and tile width, once (server workers launch from several
    // threads): allow the limit, each launch asks for what its ring needs
    static std::atomic<bool> attr[64][2];
    const int bi = BN == 128 ? 1 : 0;
    const bool cached = ex.device >= 0 && ex.device < 64;
    if (!cached || !attr[ex.device][bi].load(std::memory_order_acquire)) {
        const int lim = (int)TC_SMEM_LIMIT;
        cudaError_t e = (BN == 128) ? cudaFuncSetAttribute(tc_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
                                    : cudaFuncSetAttribute(tc_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return GBQR_ECUDA;
        if (cached) attr[ex.device][bi].store(true, std::memory_order_release);
    }
    dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)S);
    trace_begin(ex, FAM_TC_GEMM);
    if (BN == 128) tc_gemm_kernel<128><<<grid, TC_THREADS, smem, ex.stream>>>(mA, mB, p);
    else tc_gemm_kernel<64><<<grid, TC_THREADS, smem, ex.stream>>>(mA, mB, p);
    const double pairs_flops = 2.0 * (double)op.M * op.N * K * p.npairs;
    TRY_ST(trace_end(ex, FAM_TC_GEMM, pairs_flops, 2.0 * op.nsplit * ((double)op.M + op.N) * K));   // each slice once
    if (S > 1) {
        trace_begin(ex, FAM_OTHER);
        const int64_t total = op.M * op.N;
        const dim3 g((unsigned)((op.M + kThreads - 1) / kThreads), (unsigned)std::min<int64_t>(op.N, 65535));
        tc_reduce_kernel<<<g, kThreads, 0, ex.stream>>>((int)op.M, (int)op.N, S, partial, op.C, op.ldc, op.alpha, op.beta);
        TRY_ST(trace_end(ex, FAM_OTHER, (double)S * total, 4.0 * S * total + 16.0 * total));
    }
    return GBQR_OK;
}

}  // namespace gbqr

extern "C" GBQR_API gbqr_status gbqr_selftest_wait_timeout(int device, int *completed) {
    if (!completed) return GBQR_EINVAL;
    *completed = -1;
    if (cudaSetDevice(device) != cudaSuccess) return GBQR_ECUDA;
    int *d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return GBQR_ENOMEM; }
    int h[2] = {0, 0};
    gbqr_status st = GBQR_OK;
    if (cudaMemset(d, 0, 2 * sizeof(int)) != cudaSuccess) st = GBQR_ECUDA;
    if (st == GBQR_OK) {
        gbqr::wait_selftest_kernel<<<1, 32>>>(d, d + 1);
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = GBQR_ECUDA;
    }
    cudaFree(d);
    if (st != GBQR_OK) return st;
    *completed = h[1];
    return h[0] ? GBQR_ETIMEOUT : GBQR_OK;
}
