// peaks.cu -- issue-rate microbenchmarks for the roofline denominators.
//
// The hot path is bound by plain arithmetic issue (the tree walk: float32
// FMA-pipe work plus three special-function operations per interaction) and,
// in a few short kernels, by the float64 pipe.  These kernels measure what
// this GPU sustains for each: every thread runs kChains independent chains
// (no dependency stalls), enough warps per SM to fill every scheduler, and
// the result is kept live through a conditional store.
#include "hts_internal.cuh"

namespace hts {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// kind 0: float32 FMA (2 flop each); 1: special-function rsqrt (1 op each);
// 2: float64 FMA (2 flop each)
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(int iters, float seed, float *sink)
{
    if (KIND == 2) {
        double a[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = (double)seed + 1e-3 * (threadIdx.x + u);
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int u = 0; u < kChains; ++u) a[u] = fma(a[u], 0.9999999999, 1e-10);
        }
        double t = 0.0;
#pragma unroll
        for (int u = 0; u < kChains; ++u) t += a[u];
        if (t == 1234.5678) sink[0] = (float)t;
    } else {
        float a[kChains];
#pragma unroll
        for (int u = 0; u < kChains; ++u) a[u] = seed + 1e-3f * (float)(threadIdx.x + u);
        for (int k = 0; k < iters; ++k) {
#pragma unroll
            for (int u = 0; u < kChains; ++u) a[u] = KIND == 0 ? fmaf(a[u], 0.9999999f, 1e-7f) : rsqrtf(a[u]);
        }
        float t = 0.f;
#pragma unroll
        for (int u = 0; u < kChains; ++u) t += a[u];
        if (t == 1234.5678f) sink[0] = t;
    }
}

template <int KIND>
double time_peak(int blocks, int iters, float *sink, cudaEvent_t a, cudaEvent_t b, float *ms)
{
    peak_kernel<KIND><<<blocks, kPeakThreads>>>(iters / 16, 1.0f, sink);  // warm-up
    cudaEventRecord(a);
    peak_kernel<KIND><<<blocks, kPeakThreads>>>(iters, 1.0f, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
    const double ops = (double)blocks * kPeakThreads * kChains * (double)iters * (KIND == 1 ? 1.0 : 2.0);
    return *ms > 0.f ? ops / (*ms * 1e-3) / 1e12 : 0.0;
}

}  // namespace
}  // namespace hts

extern "C" HTS_API int hts_measure_peaks(int device, double *out3)
{
    if (!out3 || device < 0) return HTS_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return HTS_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return HTS_ECUDA;
    const int blocks = prop.multiProcessorCount * 8;  // 64 warps per SM
    float *sink = nullptr;
    if (cudaMalloc((void **)&sink, sizeof(float)) != cudaSuccess) return HTS_EOOM;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.f;
    out3[0] = hts::time_peak<0>(blocks, 1 << 17, sink, a, b, &ms);  // float32 FMA, TFLOP/s
    out3[1] = hts::time_peak<1>(blocks, 1 << 13, sink, a, b, &ms);  // rsqrt, Tops/s
    out3[2] = hts::time_peak<2>(blocks, 1 << 11, sink, a, b, &ms);  // float64 FMA, TFLOP/s
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e == cudaSuccess ? HTS_OK : HTS_ECUDA;
}
