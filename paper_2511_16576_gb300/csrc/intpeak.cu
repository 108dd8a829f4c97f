// intpeak.cu -- integer-ALU throughput probe (roofline denominator of A1).
//
// The MinHash walk is bound by 32-bit integer instructions (64-bit multiplies,
// shifts and xors of the point generator, compares of the bbox test).  This
// probe issues the same instruction classes -- integer multiply-add, add,
// xor, shift -- in 8 independent dependency chains per thread (enough ILP to
// hide latency) on every SM, and reports thread-level integer instructions
// per second.  Inline PTX keeps the compiler from folding the chains.
#include <chrono>

#include "pmh_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kOpsPerChainIter = 4;  // mad.lo, add, xor, shl

__global__ void __launch_bounds__(256) int_peak_kernel(uint32_t* out, int iters, uint32_t seed)
{
    uint32_t x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = seed + threadIdx.x * 7u + c;
        y[c] = seed ^ (blockIdx.x * 13u + c);
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            asm volatile(
                "mad.lo.u32 %0, %0, 0x9E3779B9, %1;\n\t"
                "add.u32 %1, %1, %0;\n\t"
                "xor.b32 %0, %0, %1;\n\t"
                "shl.b32 %1, %1, 3;\n\t"
                : "+r"(x[c]), "+r"(y[c]));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c] + y[c];
    if (acc == 0x12345678u) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" int pmh_probe_int_peak(pmh_ctx ctx, double* h_ops, double* h_seconds)
{
    PMH_TRY(pmh_check_device(ctx));
    if (!h_ops) return pmh_set_error(PMH_ERR_ARG, "null output");
    int per_sm = 0;
    PMH_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_peak_kernel, 256, 0));
    int blocks = ctx->sm_count * (per_sm > 0 ? per_sm : 1);
    uint32_t* out = nullptr;
    PMH_TRY(pmh_scratch(ctx, SCR_MISC, sizeof(uint32_t) * (size_t)blocks * 256, (void**)&out));
    cudaEvent_t e0, e1;
    PMH_CUDA_TRY(cudaEventCreate(&e0));
    PMH_CUDA_TRY(cudaEventCreate(&e1));
    const int iters = 20000;
    // warm-up
    int_peak_kernel<<<blocks, 256>>>(out, iters / 10, 1u);
    PMH_LAUNCHED("int_peak_kernel");
    PMH_CUDA_TRY(cudaDeviceSynchronize());
    float best_ms = 1e30f;
    for (int r = 0; r < 3; ++r) {
        PMH_CUDA_TRY(cudaEventRecord(e0));
        int_peak_kernel<<<blocks, 256>>>(out, iters, 2u + r);
        PMH_LAUNCHED("int_peak_kernel");
        PMH_CUDA_TRY(cudaEventRecord(e1));
        PMH_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        PMH_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double ops = (double)blocks * 256.0 * iters * kChains * kOpsPerChainIter;
    *h_ops = ops / (best_ms * 1e-3);
    if (h_seconds) *h_seconds = best_ms * 1e-3;
    return PMH_OK;
}
