// Microbenchmark of the plain arithmetic pipes, for the roofline denominators of the element
// kernels (no counterpart in the paper): every thread runs 8 independent chains of fused
// multiply-adds, enough to keep each SM's pipe issuing every cycle, on a grid of 8 blocks of 256
// threads per SM.  kind 0: FP32 FFMA; 1: packed FP32x2 FFMA2 (two FMAs per instruction, the form of
// the packed dual numbers of the interior kernel); 2: FP64 DFMA.

#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "imga_internal.h"

namespace imga {

namespace {

template <class T>
__global__ void __launch_bounds__(256) fma_chains(int iters, T b, T c, T* __restrict__ out) {
    T a[8];
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == T(12345.678)) out[threadIdx.x] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(256) fma2_chains(int iters, float b, float c, float* __restrict__ out) {
    float2 a[8];
    for (int k = 0; k < 8; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x + 2 * k));
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
    float s = 0.f;
    for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
    if (s == 12345.678f) out[threadIdx.x] = s;
}

}  // namespace

int peak_flops(int device, int kind, double* tflops, std::string& err) {
    if (cudaSetDevice(device) != cudaSuccess) { err = "cudaSetDevice failed"; return 1; }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = 8 * std::max(1, sms);
    const int iters = kind == 2 ? 64 : 2048;   // 16 x 8 FMAs per iteration and thread
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, 256 * sizeof(double)) != cudaSuccess) { err = "cudaMalloc failed"; return 1; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up
        cudaEventRecord(e0);
        if (kind == 0) fma_chains<float><<<grid, 256>>>(iters, 0.999999f, 1e-7f, (float*)buf);
        else if (kind == 1) fma2_chains<<<grid, 256>>>(iters, 0.999999f, 1e-7f, (float*)buf);
        else fma_chains<double><<<grid, 256>>>(iters, 0.999999, 1e-7, buf);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (cudaGetLastError() != cudaSuccess) { err = "microbenchmark launch failed"; return 1; }
    const double fmas = (double)grid * 256 * iters * 16 * 8 * (kind == 1 ? 2 : 1);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return 0;
}

}  // namespace imga
