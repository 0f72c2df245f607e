// Dense tensor-core rate of the matcher's MMA shape (the roofline of the
// BF16 and FP8 brute-force forms), kept apart from the matcher's sources.
#include <cuda_runtime.h>

#include <algorithm>

#include "mrf_internal.h"
#include "tc.cuh"

namespace {
constexpr int BM = 128;                   // rows of A (as the matcher's voxel tile)
constexpr int BN = 256;                   // rows of B (as the matcher's dictionary tile)
constexpr int kTileA = BM * 128;          // 128-byte rows
constexpr int kTileB = BN * 128;
constexpr uint64_t kWaitLimitNs = 4000000000ull;
}  // namespace

// ---------------------------------------------------------------------------
// Dense tensor-core rate of the matcher's MMA shape (M = 128, N = 256,
// cta_group::1, operands in 128-byte-swizzled shared memory, FP32 accumulate
// in TMEM): one CTA per SM, one thread issuing back-to-back MMAs into two
// accumulators, no loads in the loop. The roofline of the BF16 and FP8 forms.

namespace {

constexpr int kRateIters = 20000;

template <int MODE>
__global__ void __launch_bounds__(128, 1) mma_rate_kernel(int iters, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *tA = smem, *tB = smem + kTileA;   // 128 and 256 rows of 128 bytes
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kTileA + kTileB) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor-core reads
    if (threadIdx.x == 0) { mbar_init(&done_bar, 1); fence_mbar_init(); }
    if (warp == 1) { tmem_alloc(&tmem_slot, 2 * BN); tmem_relinquish(); }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_slot;
    if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = MODE == MRF_FP8E4M3 ? make_idesc(0, 0, BM, BN) : make_idesc(1, 1, BM, BN);
        const uint64_t a0 = smem_desc_sw128(tA), b0 = smem_desc_sw128(tB);
        for (int it = 0; it < iters; ++it) {
            const uint32_t d = tmem_base + (uint32_t)((it & 1) * BN);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                const uint32_t accum = (it > 1 || kk > 0) ? 1u : 0u;
                if (MODE == MRF_FP8E4M3) mma_f8(d, a0 + adv, b0 + adv, idesc, accum);
                else mma_f16(d, a0 + adv, b0 + adv, idesc, accum);
            }
        }
        mma_commit(&done_bar);
        const uint64_t t0 = global_timer_ns();
        while (!mbar_try_wait(&done_bar, 0)) {
            if (global_timer_ns() - t0 > kWaitLimitNs) { atomicExch(err, 1); break; }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 2 * BN);
    }
}

}  // namespace

extern "C" int mrf_mma_rate(mrf_ctx *ctx, int32_t precision, double *tflops)
{
    if (!ctx || !tflops) return set_error(MRF_E_INVALID, "NULL argument");
    if (precision != MRF_BF16 && precision != MRF_FP8E4M3)
        return set_error(MRF_E_INVALID, "mma rate: precision must be MRF_BF16 or MRF_FP8E4M3");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    // more than half an SM's shared memory, so that no SM holds two CTAs (each takes all 512 TMEM columns)
    const size_t smem = std::max<size_t>(kTileA + kTileB + 1024, 120 * 1024);
    auto kern = precision == MRF_FP8E4M3 ? mma_rate_kernel<MRF_FP8E4M3> : mma_rate_kernel<MRF_BF16>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "mma rate shared-memory attribute");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(t0, ctx->aux);
        kern<<<ctx->sm_count, 128, smem, ctx->aux>>>(kRateIters, ctx->err_flag);
        cudaEventRecord(t1, ctx->aux);
        e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms > 0.f &&
            (best == 0.f || ms < best))
            best = ms;   // the first launch only warms up
        count_launch(ctx);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e != cudaSuccess) return cuda_fail(e, "mma rate kernel");
    const double k_per_instr = precision == MRF_FP8E4M3 ? 32.0 : 16.0;
    const double flops = (double)ctx->sm_count * kRateIters * 4 * 2.0 * BM * BN * k_per_instr;
    *tflops = best > 0.f ? flops / (best * 1e-3) / 1e12 : 0.0;
    return MRF_OK;
}
