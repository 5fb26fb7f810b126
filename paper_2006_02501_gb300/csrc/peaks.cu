// Measured arithmetic peaks of the current device: the denominators behind the
// evaluation kernels' rooflines (FP64 fused multiply-add, FP32 fused
// multiply-add scalar and packed FP32x2, single-precision reciprocal square
// root of the special-function unit).  Each kernel runs kChains independent
// dependency chains per thread on every SM (enough warps and independent work
// to keep the pipe busy), times the launch with CUDA events and counts two
// flops per multiply-add and one operation per reciprocal square root.
#include <cuda_runtime.h>

#include "common.cuh"
#include "pair_math.cuh"

namespace mh {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int k = 0; k < iters; ++k)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-12345.0) out[0] = s;          // keeps the chains alive
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(float *out, int iters, float a, float b)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int k = 0; k < iters; ++k)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -12345.0f) out[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_rsqrt(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0f + threadIdx.x * 1e-3f + c;
    for (int k = 0; k < iters; ++k)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = rsqrt_mufu(x[c]) + 1.0f;
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -12345.0f) out[0] = s;
}

template <typename Launch>
int time_launch(Launch &&launch, cudaStream_t st, float *ms)
{
    cudaEvent_t e0, e1;
    MH_CUDA(cudaEventCreate(&e0));
    MH_CUDA(cudaEventCreate(&e1));
    launch();                                    // warm-up
    MH_CUDA(cudaEventRecord(e0, st));
    launch();
    MH_CUDA(cudaEventRecord(e1, st));
    MH_CUDA(cudaEventSynchronize(e1));
    MH_LAUNCHED("peak kernel");
    MH_CUDA(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return MH_OK;
}

}  // namespace

}  // namespace mh

using namespace mh;

extern "C" int mh_measure_peaks(double *out4)
{
    if (!out4) {
        set_error("mh_measure_peaks: out4 is NULL");
        return MH_EINVAL;
    }
    int dev = 0, n_sm = 0;
    MH_CUDA(cudaGetDevice(&dev));
    MH_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    float *sink = nullptr;                       // 8 bytes: also the FP64 kernel's (never taken) store
    MH_CUDA(cudaMalloc((void **)&sink, sizeof(double)));
    const unsigned grid = (unsigned)n_sm * 8;
    const double threads = (double)grid * kPeakThreads;
    cudaStream_t st = 0;
    float ms = 0.0f;
    int rc = MH_OK;
    // 20-40 ms per launch at 2.07 GHz (FP64 has 2 lanes per SM, FP32 128): long
    // against the event resolution and the launch latency
    const int it64 = 8192, it32 = 131072, itr = 65536;
    if (!rc) rc = time_launch([&] { k_peak_fma<double><<<grid, kPeakThreads, 0, st>>>((double *)sink, it64, 0.999999, 1e-7); }, st, &ms);
    if (!rc) out4[0] = 2.0 * kChains * it64 * threads / (ms * 1e-3) / 1e12;
    if (!rc) rc = time_launch([&] { k_peak_fma<float><<<grid, kPeakThreads, 0, st>>>(sink, it32, 0.999999f, 1e-7f); }, st, &ms);
    if (!rc) out4[1] = 2.0 * kChains * it32 * threads / (ms * 1e-3) / 1e12;
    if (!rc) rc = time_launch([&] { k_peak_ffma2<<<grid, kPeakThreads, 0, st>>>(sink, it32 / 2, 0.999999f, 1e-7f); }, st, &ms);
    if (!rc) out4[2] = 4.0 * kChains * (it32 / 2) * threads / (ms * 1e-3) / 1e12;
    if (!rc) rc = time_launch([&] { k_peak_rsqrt<<<grid, kPeakThreads, 0, st>>>(sink, itr); }, st, &ms);
    if (!rc) out4[3] = (double)kChains * itr * threads / (ms * 1e-3) / 1e12;
    cudaFree(sink);
    return rc;
}
