// Error of the library's FP32 reciprocal square root (hardware seed plus one
// Newton-Raphson step) against 1/sqrt computed in FP64 and rounded to FP32,
// in units in the last place, over 2^24 arguments spread log-uniformly over
// [2^-20, 2^40] plus every power of two in that range.  Prints the largest
// error of the refined and of the unrefined seed.
#include <cmath>
#include <cstdio>
#include <cuda_runtime.h>
#include "../paper_2412_15518_gb300/csrc/pair_formula.cuh"

__device__ float ulp_err(float v, float a) {
    const float ref = (float)(1.0 / sqrt((double)a));
    const double ulp = (double)nextafterf(ref, INFINITY) - (double)ref;
    return (float)(fabs((double)v - (double)ref) / ulp);
}

__global__ void k_check(int n, float* err_refined, float* err_seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = (i < 61) ? ldexpf(1.0f, i - 20) : exp2f(-20.0f + 60.0f * (float)(i - 61) / (float)(n - 61));
    err_refined[i] = ulp_err(otfmm::rsqrt_(a), a);
    err_seed[i] = ulp_err(rsqrtf(a), a);
}

int main() {
    const int n = 1 << 24;
    float *e1, *e2;
    if (cudaMalloc(&e1, n * sizeof(float)) != cudaSuccess || cudaMalloc(&e2, n * sizeof(float)) != cudaSuccess) return 2;
    k_check<<<(n + 255) / 256, 256>>>(n, e1, e2);
    float* h1 = new float[n];
    float* h2 = new float[n];
    if (cudaMemcpy(h1, e1, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(h2, e2, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    float m1 = 0.f, m2 = 0.f;
    for (int i = 0; i < n; i++) {
        m1 = h1[i] > m1 ? h1[i] : m1;
        m2 = h2[i] > m2 ? h2[i] : m2;
    }
    printf("%.4f %.4f\n", m1, m2);
    return 0;
}
