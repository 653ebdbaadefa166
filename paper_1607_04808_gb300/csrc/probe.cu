// Measured arithmetic rates of the current device: the denominators of the
// roofline fractions of the kernels that are bound by arithmetic rather than
// by memory (the real-space pair sum, spreading, and the FP64 path).  The
// paper has no counterpart; it reports CPU times only.
//
// Each rate comes from a register-only kernel: every thread runs CH
// independent chains of fused multiply-adds (v = v a + b, |a| < 1 so the
// values stay bounded), one block per 256 threads, 8 blocks per SM, so every
// scheduler has many warps and every warp CH independent instructions in
// flight.  The result of each chain is written out, so nothing is folded away.
// The time is the best of several launches timed with CUDA events; the
// iteration count is first calibrated so that one launch takes about 20 ms.
#include "se_internal.cuh"

#include <algorithm>

namespace se {

namespace {

constexpr int CH = 8;       // independent chains per thread
constexpr int UNROLL = 16;  // FMAs per chain per loop iteration

__global__ void __launch_bounds__(256) k_rate_fma32(int iters, float a, float b, float *out) {
    float v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = 1e-3f * (float)(threadIdx.x + i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < UNROLL; k++)
#pragma unroll
            for (int i = 0; i < CH; i++) v[i] = fmaf(v[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; i++) s += v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_rate_ffma2(int iters, float a, float b, float *out) {
    float2 v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = make_float2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)i);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < UNROLL; k++)
#pragma unroll
            for (int i = 0; i < CH; i++) v[i] = __ffma2_rn(v[i], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CH; i++) s += v[i].x + v[i].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_rate_fma64(int iters, double a, double b, float *out) {
    double v[CH];
#pragma unroll
    for (int i = 0; i < CH; i++) v[i] = 1e-3 * (double)(threadIdx.x + i);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < UNROLL; k++)
#pragma unroll
            for (int i = 0; i < CH; i++) v[i] = fma(v[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < CH; i++) s += v[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// which = 0: FP32 fmaf, 1: FP32 paired, 2: FP64.  Returns TFLOP/s (2 flops per
// FMA, 4 per paired FMA) or a negative value on a CUDA error.
double measure(int which, int nblk, float *out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1.0;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1.0;
    }
    auto launch = [&](int iters) {
        if (which == 0) k_rate_fma32<<<nblk, 256>>>(iters, 0.999999f, 1e-7f, out);
        else if (which == 1) k_rate_ffma2<<<nblk, 256>>>(iters, 0.999999f, 1e-7f, out);
        else k_rate_fma64<<<nblk, 256>>>(iters, 0.999999999, 1e-12, out);
    };
    auto timed = [&](int iters) -> float {
        cudaEventRecord(e0);
        launch(iters);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    double best = -1.0;
    int iters = 64;
    float ms = timed(iters);  // warm-up and first calibration
    for (int k = 0; k < 6 && ms >= 0.f && ms < 5.f; k++) {
        iters *= 4;
        ms = timed(iters);
    }
    if (ms > 0.f) {
        iters = (int)std::min(1e9, std::max(1.0, iters * (20.0 / ms)));
        for (int rep = 0; rep < 3; rep++) {
            ms = timed(iters);
            if (ms <= 0.f) break;
            const double fma = (double)nblk * 256.0 * iters * UNROLL * CH * (which == 1 ? 2.0 : 1.0);
            best = std::max(best, 2.0 * fma / (ms * 1e-3) / 1e12);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return best;
}

}  // namespace

}  // namespace se

extern "C" se_status_t se_measure_peaks(se_peaks_t *out) {
    using namespace se;
    if (!out) return fail(SE_ERR_INVALID_ARG, "se_measure_peaks: out is NULL");
    int dev = 0, sms = 0;
    SE_CUDA_TRY(cudaGetDevice(&dev));
    SE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int nblk = 8 * sms;
    float *buf = nullptr;
    SE_CUDA_TRY(cudaMalloc(&buf, (size_t)nblk * 256 * sizeof(float)));
    const double r32 = measure(0, nblk, buf);
    const double r32p = measure(1, nblk, buf);
    const double r64 = measure(2, nblk, buf);
    cudaFree(buf);
    if (r32 <= 0.0 || r32p <= 0.0 || r64 <= 0.0)
        return fail(SE_ERR_CUDA, "se_measure_peaks: a probe launch failed");
    out->fp32_fma_tflops = r32;
    out->fp32_ffma2_tflops = r32p;
    out->fp64_fma_tflops = r64;
    out->sm_count = sms;
    return SE_OK;
}
