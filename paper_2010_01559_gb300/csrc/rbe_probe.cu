// rbe_probe.cu -- measured unit throughput for rooflines (rbe_probe_peaks).
//
// Two saturating kernels, four resident blocks per SM: eight independent
// chains per thread of __sincosf (the special-function unit's sin and cos, as
// the structure-factor and force passes issue them) or of FP32 FMA.  Each
// block records its duration in SM cycles and in global-timer nanoseconds; the
// per-SM rate is the work of an SM's blocks over their longest duration in
// cycles, and the clock is cycles over nanoseconds.
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "rbe.h"

namespace rbe_probe {

constexpr int kThreads = 256, kBlocksPerSm = 4, kChains = 8, kIters = 2048;

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <bool SFU>
__global__ void __launch_bounds__(kThreads) k_probe(float* sink, long long* cyc,
                                                     unsigned long long* ns) {
    float v[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = 0.25f + 0.01f * (float)(threadIdx.x + j);
    __syncthreads();
    const long long c0 = clock64();
    const unsigned long long t0 = gtime();
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if (SFU) {
                float s, c;
                __sincosf(v[j], &s, &c);
                v[j] = s + c * 0.5f;       // stays in [-1.2, 1.2]: no range reduction
            } else {
                v[j] = fmaf(v[j], 0.999f, 0.001f);
            }
        }
    }
    __syncthreads();
    const long long c1 = clock64();
    const unsigned long long t1 = gtime();
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc += v[j];
    sink[blockIdx.x * kThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0) {
        cyc[blockIdx.x] = c1 - c0;
        ns[blockIdx.x] = t1 - t0;
    }
}

}  // namespace rbe_probe

extern "C" rbe_status rbe_probe_peaks(rbe_peaks* out) {
    using namespace rbe_probe;
    if (!out) return RBE_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RBE_ERR_CUDA;
    const int blocks = sms * kBlocksPerSm;
    float* sink = nullptr;
    long long* cyc = nullptr;
    unsigned long long* ns = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * blocks * kThreads) != cudaSuccess) return RBE_ERR_CUDA;
    if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess ||
        cudaMalloc(&ns, sizeof(unsigned long long) * blocks) != cudaSuccess) {
        cudaFree(sink);
        cudaFree(cyc);
        return RBE_ERR_CUDA;
    }
    std::vector<long long> hc(blocks);
    std::vector<unsigned long long> hn(blocks);
    double rate[2] = {0.0, 0.0}, mhz = 0.0;
    bool ok = true;
    for (int pass = 0; pass < 2 && ok; ++pass) {
        for (int rep = 0; rep < 2 && ok; ++rep) {   // the first launch warms up clocks and caches
            if (pass == 0) k_probe<true><<<blocks, kThreads>>>(sink, cyc, ns);
            else k_probe<false><<<blocks, kThreads>>>(sink, cyc, ns);
            ok = cudaDeviceSynchronize() == cudaSuccess &&
                 cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) ==
                     cudaSuccess &&
                 cudaMemcpy(hn.data(), ns, sizeof(unsigned long long) * blocks,
                            cudaMemcpyDeviceToHost) == cudaSuccess;
        }
        if (!ok) break;
        long long cmax = 1;
        unsigned long long nmax = 1;
        for (int b = 0; b < blocks; ++b) {
            if (hc[b] > cmax) cmax = hc[b];
            if (hn[b] > nmax) nmax = hn[b];
        }
        // work of one SM's blocks: sin and cos count one result each
        const double per_sm = (double)kBlocksPerSm * kThreads * kIters * kChains * (pass == 0 ? 2.0 : 1.0);
        rate[pass] = per_sm / (double)cmax;
        mhz = (double)cmax / (double)nmax * 1e3;
    }
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(ns);
    if (!ok) return RBE_ERR_CUDA;
    out->sfu_per_clk_sm = rate[0];
    out->ffma_per_clk_sm = rate[1];
    out->sm_clock_mhz = mhz;
    out->sms = sms;
    return RBE_OK;
}
