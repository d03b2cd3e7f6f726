// CUDA-core arithmetic peaks of the device, measured (ot_alu_peaks): the
// denominators of the FP64 and FP32 rooflines of the interaction kernels,
// which are bound by the FP64 and FP32 pipes, not by HBM or tensor cores.
//
// Each kernel runs CH independent FMA chains per thread over `iters`
// iterations on 8 CTAs of 256 threads per SM, so every SM sub-partition has
// enough independent FMAs in flight to cover the pipe latency; the chains
// converge (x <- a x + b with |a| < 1), so no value overflows.  The result is
// stored so that no FMA is dead code.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/octofmm.h"

namespace otfmm {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_f64(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 1e-3 * threadIdx.x + c;
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_f32(double* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 1e-3f * threadIdx.x + c;
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Paired FP32 FMA: two FMAs (one per half of a float2) per instruction.
__global__ void __launch_bounds__(256) k_peak_f32x2(double* out, int iters, float a, float b) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = make_float2(1e-3f * threadIdx.x + c, 2e-3f * threadIdx.x - c);
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace otfmm

using namespace otfmm;

extern "C" int ot_alu_peaks(int device, int reps, double* fp64_tflops, double* fp32_tflops,
                            double* fp32x2_tflops) {
    if (reps < 1) reps = 1;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return OT_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = 8 * std::max(1, sms), threads = 256;
    double* buf = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = OT_OK;
    if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = OT_ERR_CUDA;
    // iterations per launch: about 10-20 ms of each pipe at GB300 rates
    const int it64 = 256, it32 = 8192;
    auto best_of = [&](auto launch, double flops) -> double {
        float best = 1e30f;
        for (int r = 0; r <= reps && rc == OT_OK; r++) {  // the first launch warms up
            cudaEventRecord(e0, s);
            launch();
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = OT_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, ms);
        }
        return rc == OT_OK ? flops / (best * 1e-3) / 1e12 : 0.0;
    };
    const double per_thread = 16.0 * kChains * 2.0;  // FMAs per iteration x 2 flops
    const double n = (double)blocks * threads;
    double v64 = 0.0, v32 = 0.0, v32x2 = 0.0;
    if (rc == OT_OK)
        v64 = best_of([&] { k_peak_f64<<<blocks, threads, 0, s>>>(buf, it64, 0.999999, 1e-6); },
                      n * it64 * per_thread);
    if (rc == OT_OK)
        v32 = best_of([&] { k_peak_f32<<<blocks, threads, 0, s>>>(buf, it32, 0.9999f, 1e-4f); },
                      n * it32 * per_thread);
    if (rc == OT_OK)
        v32x2 = best_of([&] { k_peak_f32x2<<<blocks, threads, 0, s>>>(buf, it32, 0.9999f, 1e-4f); },
                        n * it32 * per_thread * 2.0);
    if (rc == OT_OK && cudaGetLastError() != cudaSuccess) rc = OT_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (buf) cudaFree(buf);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    if (rc != OT_OK) return rc;
    if (fp64_tflops) *fp64_tflops = v64;
    if (fp32_tflops) *fp32_tflops = v32;
    if (fp32x2_tflops) *fp32x2_tflops = v32x2;
    return OT_OK;
}
