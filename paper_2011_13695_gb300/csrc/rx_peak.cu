// Measured FP32 FMA throughput of the current GPU (no paper counterpart).
//
// The chain's CUDA-core stages are bound by FP32 arithmetic, not by HBM; their
// roofline needs the FMA pipes' real rate on this part at the clock it runs,
// not a unit count times a nominal clock. One launch fills every SM with CTAs
// whose threads run independent FMA chains (eight per thread, enough to cover
// the FMA latency at full occupancy); the entry point times it with CUDA
// events after a warm-up launch and returns flops per second (an FMA is two).
// The packed form issues fma.rn.f32x2 (two lanes' worth of FMAs per
// instruction), which sm_100-class parts execute; both forms are measured.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rx.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ float g_sink;   // written only when a chain's result is NaN, which keeps the chains live

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) k_fma_rate(int iters, float s, float c) {
    const float t = (float)(threadIdx.x + blockIdx.x) * 1e-7f;
    float acc = 0.0f;
    if constexpr (PACKED) {
        float2 v[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) v[j] = make_float2(t + j, t - j);
        const float2 ss = make_float2(s, s), cc = make_float2(c, c);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) v[j] = __ffma2_rn(v[j], ss, cc);
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc += v[j].x + v[j].y;
    } else {
        float v[kChains];
#pragma unroll
        for (int j = 0; j < kChains; ++j) v[j] = t + j;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) v[j] = fmaf(v[j], s, c);
        }
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc += v[j];
    }
    if (acc != acc) g_sink = acc;
}

}  // namespace

extern "C" rx_status rx_fp32_fma_rate(int32_t packed, int32_t iters, double* flops_per_s, double* ms,
                                      rx_stream_t stream_) {
    if (!flops_per_s || iters < 1) return RX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream_;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RX_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RX_ECUDA;
    const void* fn = packed ? (const void*)k_fma_rate<true> : (const void*)k_fma_rate<false>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1)
        return RX_ECUDA;
    const int grid = sms * per_sm;
    auto launch = [&](int it) {
        if (packed) k_fma_rate<true><<<grid, kThreads, 0, s>>>(it, 0.9999999f, 1e-7f);
        else k_fma_rate<false><<<grid, kThreads, 0, s>>>(it, 0.9999999f, 1e-7f);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return RX_ECUDA;
    launch(iters / 8 > 0 ? iters / 8 : 1);   // warm-up: module load, clocks up
    cudaEventRecord(e0, s);
    launch(iters);
    cudaEventRecord(e1, s);
    float t = 0.0f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess &&
                    cudaGetLastError() == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || t <= 0.0f) return RX_ECUDA;
    const double flops = (double)grid * kThreads * (double)iters * kChains * 2.0 * (packed ? 2.0 : 1.0);
    *flops_per_s = flops / (t * 1e-3);
    if (ms) *ms = t;
    return RX_OK;
}
