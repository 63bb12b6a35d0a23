// Measurement hook: the issue rate of the FP8 tensor-core instruction the
// direct route uses (tcgen05.mma kind::f8f6f4, M = 128, N = 256, K = 32),
// back to back from shared memory on every SM, without copies or waits.  It
// is the tensor pipe's FP8 peak on this GPU at its present clock, the
// denominator beside the GEMM-derived one in the route's roofline.
#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

constexpr int kPeakOperandBytes = 128 * 128 + 256 * 128;   // A (128 rows) + B (256 rows) of 128 B
constexpr int kPeakSmem = 120 * 1024;                       // one CTA per SM (tensor memory per CTA)

__global__ void __launch_bounds__(64, 1) k_tc_peak(int iters, unsigned int* err) {
    extern __shared__ uint8_t raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t done;
    __shared__ uint32_t tbase;
    for (int i = threadIdx.x; i < kPeakOperandBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(base)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&done), 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tmem_alloc(smem_u32(&tbase), kDirectN);
        tmem_relinquish();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the zeros, seen by the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 32) {
        const uint64_t ad = umma_desc_sw128(smem_u32(base));
        const uint64_t bd = umma_desc_sw128(smem_u32(base + 128 * 128));
        const uint32_t idesc = idesc_e4m3_f32(kDirectM, kDirectN);
        for (int i = 0; i < iters; ++i)
            for (int ks = 0; ks < 4; ++ks) tc_mma_f8(tbase, ad + 2ull * ks, bd + 2ull * ks, idesc, (i | ks) != 0);
        tc_commit(smem_u32(&done));
        mbar_wait_drain(smem_u32(&done), 0);
        if (!mbar_try_wait(smem_u32(&done), 0)) atomicOr(err, MORPH_DEVERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(tbase, kDirectN);
    }
}

}  // namespace morph

using namespace morph;

extern "C" int morph_tc_fp8_peak(morph_ctx* ctx, double* tflops) {
    if (!ctx || !tflops) return MORPH_E_INVAL;
    MORPH_CUDA_TRY(cudaSetDevice(ctx->device));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_tc_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem));
    cudaStream_t st = nullptr;
    MORPH_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MORPH_CUDA_TRY(cudaEventCreate(&e0));
    MORPH_CUDA_TRY(cudaEventCreate(&e1));
    const int iters = 4096;   // 16384 MMAs per SM: about 1 ms at full rate
    k_tc_peak<<<ctx->num_sms, 64, kPeakSmem, st>>>(iters / 8, ctx->d_err);   // warm-up
    MORPH_CUDA_TRY(cudaEventRecord(e0, st));
    k_tc_peak<<<ctx->num_sms, 64, kPeakSmem, st>>>(iters, ctx->d_err);
    MORPH_CUDA_TRY(cudaEventRecord(e1, st));
    MORPH_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    MORPH_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    MORPH_CUDA_TRY(cudaGetLastError());
    const double flop = static_cast<double>(ctx->num_sms) * iters * 4.0 * 2.0 * kDirectM * kDirectN * 32.0;
    *tflops = ms > 0.f ? flop / (static_cast<double>(ms) * 1e-3) / 1e12 : 0.0;
    return MORPH_OK;
}
