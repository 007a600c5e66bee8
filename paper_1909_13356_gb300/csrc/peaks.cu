// peaks.cu -- throughput of the arithmetic pipes the pair kernels run on
// (lsm_measure_peaks).
//
// The pair kernels are bound by plain ALU work, not by HBM or the tensor
// cores: FP32 fused multiply-adds (scalar and packed f32x2), FP64 FMAs, and
// the special-function unit's reciprocal square root and exp2.  Each probe
// kernel runs eight independent dependency chains per thread of one
// instruction kind, on every SM at full occupancy, and is timed with CUDA
// events on the caller's stream; the best of three launches after a warm-up
// is kept.  The values are the denominators of the kernels' roofline
// fractions.
#include <algorithm>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(int iters, float b, float c, float* sink)
{
    float a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += a[k];
    if (s == 1.2345e-30f) sink[0] = s;   // never true; keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(int iters, float b, float c, float* sink)
{
    float2 a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = make_float2((float)(threadIdx.x + k), (float)k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += a[k].x + a[k].y;
    if (s == 1.2345e-30f) sink[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(int iters, double b, double c, float* sink)
{
    double a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += a[k];
    if (s == 1.2345e-300) sink[0] = (float)s;
}

// kind 0: rsqrt.approx.f32, kind 1: ex2.approx.ftz.f32 of the negated value
// (bounded in (0, 1]); one special-function op per chain step
template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) k_peak_mufu(int iters, float* sink)
{
    float a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = 1.0f + 0.01f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) {
            float r;
            if (KIND == 0) {
                asm volatile("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            } else {
                const float t = -a[k];
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
            }
            a[k] = r;
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += a[k];
    if (s == 1.2345e-30f) sink[0] = s;
}

}  // namespace
}  // namespace lsm

using namespace lsm;

extern "C" int lsm_measure_peaks(lsm_ctx* c, lsm_peaks* out, void* stream)
{
    if (!c || !out) return LSM_E_INVALID_ARG;
    Ctx* ctx = &c->c;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        ctx->err = "measure_peaks: cudaSetDevice failed";
        return LSM_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = LSM_OK;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak_ffma, kPeakThreads, 0);
    const int blocks = ctx->num_sms * std::max(1, per_sm);
    const double threads = (double)blocks * kPeakThreads;
    // iterations sized for roughly 5-20 ms per launch on GB300
    const int it_f = 1 << 16, it_d = 1 << 10, it_m = 1 << 13;
    double best[5] = {1e30, 1e30, 1e30, 1e30, 1e30};
    do {
        if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
            cudaEventCreate(&e1) != cudaSuccess) {
            ctx->err = "measure_peaks: allocation of the probe's events failed";
            rc = LSM_E_CUDA;
            break;
        }
        for (int kind = 0; kind < 5 && rc == LSM_OK; kind++) {
            for (int rep = 0; rep < 4; rep++) {
                if (cudaEventRecord(e0, st) != cudaSuccess) {
                    ctx->err = "measure_peaks: cudaEventRecord failed";
                    rc = LSM_E_CUDA;
                    break;
                }
                switch (kind) {
                    case 0: k_peak_ffma<<<blocks, kPeakThreads, 0, st>>>(it_f, 0.999f, 1e-3f, sink); break;
                    case 1: k_peak_ffma2<<<blocks, kPeakThreads, 0, st>>>(it_f, 0.999f, 1e-3f, sink); break;
                    case 2: k_peak_dfma<<<blocks, kPeakThreads, 0, st>>>(it_d, 0.999, 1e-3, sink); break;
                    case 3: k_peak_mufu<0><<<blocks, kPeakThreads, 0, st>>>(it_m, sink); break;
                    default: k_peak_mufu<1><<<blocks, kPeakThreads, 0, st>>>(it_m, sink); break;
                }
                ctx->launches++;
                if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                    cudaEventSynchronize(e1) != cudaSuccess) {
                    ctx->err = "measure_peaks: probe launch failed";
                    rc = LSM_E_CUDA;
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) best[kind] = std::min(best[kind], (double)ms);   // rep 0 warms up
            }
        }
    } while (false);
    if (rc == LSM_OK) {
        const double ch = kPeakChains;
        out->ffma_tflops = threads * it_f * ch * 2.0 / (best[0] * 1e-3) / 1e12;
        out->ffma2_tflops = threads * it_f * ch * 4.0 / (best[1] * 1e-3) / 1e12;
        out->dfma_tflops = threads * it_d * ch * 2.0 / (best[2] * 1e-3) / 1e12;
        out->rsqrt_gops = threads * it_m * ch / (best[3] * 1e-3) / 1e9;
        out->ex2_gops = threads * it_m * ch / (best[4] * 1e-3) / 1e9;
        for (int k = 0; k < 5; k++) out->ms[k] = best[k];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    return rc;
}
