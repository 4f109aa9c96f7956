// conegs_measure_fp32_peak: the device's FP32 fused multiply-add throughput,
// measured, as the denominator of the rasteriser's roofline (the rasteriser
// runs on the FP32 FMA pipe: the pair response has no dense contraction).
//
// Every thread of a grid that fills every SM runs eight independent FMA
// chains (enough to cover the pipe's latency), each FMA counted as 2 flops;
// the packed f32x2 form is measured too and the larger rate is reported.
#include <cstdio>

#include "../../include/conegs.h"
#include "common.cuh"

namespace conegs {
void set_error_message(const char *msg);
}  // namespace conegs

namespace {

constexpr int PEAK_THREADS = 512;
constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(PEAK_THREADS) fma_chain_kernel(float *out, int iters, float m, float c) {
    float a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;   // keeps the chains alive; never true in practice
}

__global__ void __launch_bounds__(PEAK_THREADS) fma2_chain_kernel(float *out, int iters, float m, float c) {
    float2 a[PEAK_CHAINS / 2];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS / 2; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS / 2; ++k) a[k] = __ffma2_rn(a[k], m2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS / 2; ++k) s += a[k].x + a[k].y;
    if (s == 12345.678f) out[blockIdx.x] = s;
}

conegs_status fail_peak(const char *what, cudaError_t e) {
    char msg[200];
    snprintf(msg, sizeof msg, "measure_fp32_peak: %s: %s", what, cudaGetErrorString(e));
    conegs::set_error_message(msg);
    return CONEGS_ERR_CUDA;
}

}  // namespace

extern "C" conegs_status conegs_measure_fp32_peak(int device, double *tflops, double *ms) {
    if (!tflops) {
        conegs::set_error_message("measure_fp32_peak: NULL output");
        return CONEGS_ERR_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail_peak("cudaSetDevice", e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel, PEAK_THREADS, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 2;
    const int grid = conegs::num_sms() * per_sm;
    const int iters = 1 << 16;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best = 0.0, best_ms = 0.0;
    conegs_status st = CONEGS_OK;
    if ((e = cudaMalloc(&out, sizeof(float) * grid)) != cudaSuccess) st = fail_peak("cudaMalloc", e);
    if (st == CONEGS_OK && ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess))
        st = fail_peak("cudaEventCreate", e);
    for (int variant = 0; st == CONEGS_OK && variant < 2; ++variant) {
        for (int rep = 0; rep < 4 && st == CONEGS_OK; ++rep) {      // first repetition warms up
            cudaEventRecord(e0, 0);
            if (variant == 0)
                fma_chain_kernel<<<grid, PEAK_THREADS>>>(out, iters, 0.99999994f, 1e-7f);
            else
                fma2_chain_kernel<<<grid, PEAK_THREADS>>>(out, iters, 0.99999994f, 1e-7f);
            cudaEventRecord(e1, 0);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                st = fail_peak("kernel", e);
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            const double flops = 2.0 * PEAK_CHAINS * (double)iters * PEAK_THREADS * grid;
            const double r = flops / (t * 1e-3) / 1e12;
            if (rep > 0 && r > best) {
                best = r;
                best_ms = t;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    cudaSetDevice(prev);
    if (st != CONEGS_OK) return st;
    *tflops = best;
    if (ms) *ms = best_ms;
    return CONEGS_OK;
}
