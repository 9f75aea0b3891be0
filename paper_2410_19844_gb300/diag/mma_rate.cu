// Diagnostic: raw tcgen05.mma issue rate.  One CTA per SM issues 80,000
// M=128 (N=256 or 128), K=16 BF16 MMAs on a fixed shared-memory tile, with no
// loads, in several accumulator patterns, and with a tcgen05.commit (mode 8)
// or a commit plus an mbarrier poll (mode 9) after every four MMAs.  It is the
// measurement behind the two-atom stages of the CTA-pair mainloop.  Build and
// run from the repository root on a GB300:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        paper_2410_19844_gb300/diag/mma_rate.cu -o mma_rate && ./mma_rate
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "../csrc/tc_ptx.cuh"
using namespace sos::tc;
__global__ void __launch_bounds__(128, 1) probe(int iters, unsigned long long* out_ns, int* status, int mode) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* base = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);
    uint8_t* sA = base; uint8_t* sB = base + 16384;
    uint64_t* bar = reinterpret_cast<uint64_t*>(base + 16384 + 32768);
    uint64_t* bar2 = bar + 1;                // committed to every 4 MMAs (modes 8, 9)
    uint64_t* bar3 = bar + 2;                // already complete, polled every 4 MMAs (mode 9)
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 3);
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int i = threadIdx.x; i < (16384 + 32768) / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sA)[i] = 0x3f803f80u;
    if (threadIdx.x == 0) { mbar_init(bar, 1); mbar_init(bar2, 1); mbar_init(bar3, 1); mbar_arrive(bar3); fence_mbar_init(); }
    if (warp == 0) { tmem_alloc(slot, 512); tmem_relinquish(); }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before(); __syncthreads(); tc_fence_after();
    uint32_t tb = *slot;
    if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16_f32(128, 256, 0, 0);
        uint64_t t0 = global_timer_ns();
        for (int it = 0; it < iters; ++it) {
            for (int kk = 0; kk < 4; ++kk) {
                uint64_t ad = smem_desc_sw128(smem_u32(sA) + kk * 32, 16, 1024);
                uint64_t bd = smem_desc_sw128(smem_u32(sB) + kk * 32, 16, 1024);
                const uint32_t acc = (it > 1 || kk) ? 1u : 0u;
                if (mode == 0) {            // two accumulators, switching every 4 MMAs
                    umma_bf16(tb + (it & 1) * 256, ad, bd, idesc, acc);
                } else if (mode == 1) {     // one accumulator chain, N = 256
                    umma_bf16(tb, ad, bd, idesc, (it > 0 || kk) ? 1u : 0u);
                } else if (mode == 2) {     // two N = 128 halves, interleaved every MMA
                    constexpr uint32_t id128 = idesc_bf16_f32(128, 128, 0, 0);
                    uint64_t bd2 = smem_desc_sw128(smem_u32(sB) + 128 * 128 + kk * 32, 16, 1024);
                    umma_bf16(tb, ad, bd, id128, (it > 0 || kk) ? 1u : 0u);
                    umma_bf16(tb + 128, ad, bd2, id128, (it > 0 || kk) ? 1u : 0u);
                } else if (mode == 3) {     // two accumulators, switching every MMA
                    umma_bf16(tb + (kk & 1) * 256, ad, bd, idesc, (it > 0 || kk > 1) ? 1u : 0u);
                } else if (mode == 4) {     // two accumulators, switching every 2 MMAs
                    umma_bf16(tb + ((kk >> 1) & 1) * 256, ad, bd, idesc, (it > 0 || (kk & 1)) ? 1u : 0u);
                } else if (mode == 5) {     // two accumulators, switching every 8 MMAs
                    umma_bf16(tb + ((it >> 1) & 1) * 256, ad, bd, idesc, (it > 3 || kk || (it & 1)) ? 1u : 0u);
                } else if (mode == 6) {     // four N = 128 accumulators, 4 MMAs each in turn
                    constexpr uint32_t id128 = idesc_bf16_f32(128, 128, 0, 0);
                    umma_bf16(tb + (it & 3) * 128, ad, bd, id128, (it > 3 || kk) ? 1u : 0u);
                } else if (mode == 7) {     // one N = 128 chain
                    constexpr uint32_t id128 = idesc_bf16_f32(128, 128, 0, 0);
                    umma_bf16(tb, ad, bd, id128, (it > 0 || kk) ? 1u : 0u);
                } else {                    // modes 8, 9: one N = 256 chain with bookkeeping
                    umma_bf16(tb, ad, bd, idesc, (it > 0 || kk) ? 1u : 0u);
                }
            }
            if (mode >= 8) umma_commit(bar2);
            if (mode == 9) {
                if (!mbar_wait(bar3, 0, 1000000000ull)) atomicExch(status, -4);
                tc_fence_after();
            }
        }
        umma_commit(bar);
        if (!mbar_wait(bar, 0, 2000000000ull)) atomicExch(status, -4);
        uint64_t t1 = global_timer_ns();
        if (blockIdx.x == 0) *out_ns = t1 - t0;
    }
    tc_fence_before(); __syncthreads();
    if (warp == 0) { __syncwarp(); tc_fence_after(); tmem_dealloc(tb, 512); }
}
int main() {
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    unsigned long long* d_ns; int* d_st; cudaMalloc(&d_ns, 8); cudaMalloc(&d_st, 4); cudaMemset(d_st, 0, 4);
    int smem = 120 * 1024;   // one CTA per SM (TMEM: 512 columns each)
    cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int modes[] = {1, 0, 5, 3, 8, 9, 7, 1, 0, 5, 3, 8, 9, 7};
    for (int rep = 0; rep < 14; ++rep) {
        int iters = 20000, mode = modes[rep];
        cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
        cudaEventRecord(a); probe<<<sms, 128, smem>>>(iters, d_ns, d_st, mode); cudaEventRecord(b);
        cudaError_t e = cudaEventSynchronize(b);
        float ms; cudaEventElapsedTime(&ms, a, b);
        unsigned long long ns; cudaMemcpy(&ns, d_ns, 8, cudaMemcpyDeviceToHost); int st; cudaMemcpy(&st, d_st, 4, cudaMemcpyDeviceToHost);
        const double per = (mode == 6 || mode == 7) ? 0.5 : 1.0;   // N = 128 instructions
        double flops = 2.0 * 128 * 256 * 16 * 4.0 * iters * sms * per;
        printf("mode %d err=%s status=%d event %.3f ms -> %.0f TF/s ; in-kernel CTA0 %.3f ms -> per-SM %.0f flop/ns\n",
               mode, cudaGetErrorString(e), st, ms, flops / ms / 1e9, ns / 1e6, flops / sms / ns);
    }
    return 0;
}
