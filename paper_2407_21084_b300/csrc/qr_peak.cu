// qr_peak.cu -- measured FMA throughput of this GPU's FP32 and FP64 pipes.
//
// The path-and-series kernel is bound by FP32 fused multiply-adds (FP64 in
// the plain form), so its roofline denominator is the rate at which the SMs
// of this device retire them. This file measures that rate instead of
// deriving it from a lane count and a clock: every thread of a grid that
// fills every SM runs kChains independent FMA chains (enough independent
// work per warp that the pipe, not the chain latency, is the limit), and the
// launches are timed with CUDA events on the caller's stream. Nothing is
// changed on the device (no clock or power setting); the clock the SMs ran
// at is whatever the driver chose, which the caller samples alongside.
#include <cuda_runtime.h>

#include <algorithm>

#include "qr_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ T fma_step(T x, T a, T b)
{
    return fma(x, a, b);
}

__device__ __forceinline__ float2 fma_step(float2 x, float2 a, float2 b)
{
    return __ffma2_rn(x, a, b);
}

template <typename T>
__device__ __forceinline__ T seed_val(int t, int c);
template <>
__device__ __forceinline__ float seed_val<float>(int t, int c)
{
    return 1.0f + 1e-7f * (float)((t * kChains + c) & 1023);
}
template <>
__device__ __forceinline__ double seed_val<double>(int t, int c)
{
    return 1.0 + 1e-13 * (double)((t * kChains + c) & 1023);
}
template <>
__device__ __forceinline__ float2 seed_val<float2>(int t, int c)
{
    return make_float2(seed_val<float>(t, c), seed_val<float>(t, c + 1));
}

__device__ __forceinline__ float lane_sum(float v) { return v; }
__device__ __forceinline__ double lane_sum(double v) { return v; }
__device__ __forceinline__ float lane_sum(float2 v) { return v.x + v.y; }

// x <- x a + b on kChains independent chains, iters x kUnroll times; a is
// just below 1 and b small so that the values stay finite and normal. The
// chain sums are written out so that no chain can be removed.
template <typename T, typename S>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, long long iters, S* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = seed_val<T>(t, c);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma_step(x[c], a, b);
    }
    S s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += lane_sum(x[c]);
    out[t] = s;
}

// half of the chains scalar, half packed two-lane, interleaved: both FP32
// forms in flight at once (3 FMA per lane per chain step pair)
__global__ void __launch_bounds__(kThreads) k_fma_mixed(float a, float b, long long iters, float* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int H = kChains / 2;
    float xs[H];
    float2 xp[H];
#pragma unroll
    for (int c = 0; c < H; ++c) {
        xs[c] = seed_val<float>(t, c);
        xp[c] = seed_val<float2>(t, c + H);
    }
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < H; ++c) {
                xs[c] = fmaf(xs[c], a, b);
                xp[c] = __ffma2_rn(xp[c], a2, b2);
            }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < H; ++c) s += xs[c] + lane_sum(xp[c]);
    out[t] = s;
}

template <typename T, typename S>
qr_status run_peak(T a, T b, int lanes, double target_ms, cudaStream_t st, double* tflops, double* ms_out,
                   int* sms_out, void (*kern)(T, T, long long, S*) = k_fma_chains<T, S>)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QR_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QR_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0) != cudaSuccess) return QR_ECUDA;
    per_sm = std::max(per_sm, 1);
    const int blocks = sms * per_sm;
    const long long threads = (long long)blocks * kThreads;
    S* out = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&out), (size_t)threads * sizeof(S), st) != cudaSuccess)
        return QR_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    qr_status rc = QR_OK;
    auto timed = [&](long long iters, int launches, float* ms) -> bool {
        if (cudaEventRecord(e0, st) != cudaSuccess) return false;
        for (int r = 0; r < launches; ++r) kern<<<blocks, kThreads, 0, st>>>(a, b, iters, out);
        if (cudaGetLastError() != cudaSuccess) return false;
        if (cudaEventRecord(e1, st) != cudaSuccess) return false;
        if (cudaEventSynchronize(e1) != cudaSuccess) return false;
        return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
    };
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = QR_ECUDA;
            break;
        }
        // calibrate: one launch of 256 iterations (after a warm-up launch),
        // then size launches of about 20 ms and repeat them for target_ms
        float ms = 0.f;
        long long iters = 256;
        if (!timed(iters, 1, &ms) || !timed(iters, 1, &ms)) {
            rc = QR_ECUDA;
            break;
        }
        const double per_iter = std::max((double)ms, 1e-3) / (double)iters;
        iters = std::max(16LL, (long long)(20.0 / per_iter));
        const int launches = std::max(1, (int)(target_ms / 20.0 + 0.5));
        if (!timed(iters, launches, &ms)) {
            rc = QR_ECUDA;
            break;
        }
        // lanes: twice the FMA per chain step, averaged over the chains (2, 4,
        // or 3 for the mixed form)
        const double fma = (double)threads * (double)iters * kUnroll * kChains * (lanes / 2.0) * launches;
        if (tflops) *tflops = 2.0 * fma / ((double)ms * 1e-3) / 1e12;
        if (ms_out) *ms_out = ms;
        if (sms_out) *sms_out = sms;
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (rc == QR_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = QR_ECUDA;
    return rc;
}

}  // namespace

extern "C" qr_status qr_fma_peak(int kind, double ms, void* stream, double* tflops_out, double* ms_out,
                                 int* sm_count_out)
{
    if (!(ms > 0.0) || ms > 60000.0) return QR_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (kind) {
    case QR_PEAK_FP32:
        return run_peak<float, float>(0.9999999f, 1e-7f, 2, ms, st, tflops_out, ms_out, sm_count_out);
    case QR_PEAK_FP32X2:
        return run_peak<float2, float>(make_float2(0.9999999f, 0.9999998f), make_float2(1e-7f, 2e-7f), 4, ms, st,
                                       tflops_out, ms_out, sm_count_out);
    case QR_PEAK_FP32MIX:
        return run_peak<float, float>(0.9999999f, 1e-7f, 3, ms, st, tflops_out, ms_out, sm_count_out, k_fma_mixed);
    case QR_PEAK_FP64:
        return run_peak<double, double>(0.9999999999999, 1e-13, 2, ms, st, tflops_out, ms_out, sm_count_out);
    default:
        return QR_EINVAL;
    }
}
