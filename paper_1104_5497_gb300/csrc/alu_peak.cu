// alu_peak.cu -- the FP32 and FP64 FMA throughput of this GPU, measured: the
// denominators of the trackers' ALU roofline (the method has no counterpart; this is
// measurement support, built into its own small library).
//
// Every thread runs CHAINS independent FMA chains a = a * m + c (0 < m < 1: the values
// approach c / (1 - m) and stay finite) for `iters` rounds; the grid is blocks_per_sm blocks of 256
// threads per SM, enough independent work per scheduler to cover the FMA latency.  One
// FMA is two flops.  The result is written (to a small device array) only when it equals
// a value it cannot reach, so the compiler keeps every FMA.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;

__device__ float g_sink32[256];
__device__ double g_sink64[256];
template <class T>
__device__ __forceinline__ T *sink();
template <>
__device__ __forceinline__ float *sink<float>() { return g_sink32; }
template <>
__device__ __forceinline__ double *sink<double>() { return g_sink64; }

template <class T>
__global__ void __launch_bounds__(256) fma_kernel(T seed, T mul, T add, int iters) {
    T a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) a[c] = seed + T(threadIdx.x + c) * T(1e-7);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < UNROLL; u++)
#pragma unroll
            for (int c = 0; c < CHAINS; c++) a[c] = fma(a[c], mul, add);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += a[c];
    if (s == T(-12345.0)) sink<T>()[threadIdx.x] = s;   // never: every a[c] stays positive
}

template <class T>
int run(int blocks_per_sm, int iters, double *tflops, float *ms) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int grid = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 1;
    const T mul = T(0.999), add = T(1e-3);
    fma_kernel<T><<<grid, 256>>>(T(1), mul, add, iters / 8 > 0 ? iters / 8 : 1);   // warm-up
    cudaEventRecord(e0);
    fma_kernel<T><<<grid, 256>>>(T(1), mul, add, iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || t <= 0.f) return 1;
    const double fmas = (double)grid * 256.0 * iters * UNROLL * CHAINS;
    *tflops = 2.0 * fmas / (t * 1e-3) / 1e12;
    *ms = t;
    return 0;
}

}  // namespace

extern "C" {

// Measured FMA throughput in TFLOP/s on the current device: precision 32 or 64,
// blocks_per_sm resident blocks of 256 threads per SM, iters rounds of 128 FMAs per
// thread.  Writes *tflops and the kernel's *ms; returns 0, or 1 on a CUDA error or bad
// argument.
int nphc_alu_peak(int precision, int blocks_per_sm, int iters, double *tflops, float *ms) {
    if (!tflops || !ms || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1) return 1;
    if (precision == 32) return run<float>(blocks_per_sm, iters, tflops, ms);
    if (precision == 64) return run<double>(blocks_per_sm, iters, tflops, ms);
    return 1;
}

}  // extern "C"
