// FMA-throughput probe: the ALU roofline denominators of the float64 and
// float32 kernels, measured on the device the library runs on.  Each thread
// runs 8 independent fused multiply-add chains (enough independent work to
// fill the pipes), the grid fills every SM several times over.
#include "tc_internal.h"

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T a, T b) {
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-1.2345) out[blockIdx.x] = s;   // keeps the chains alive
}

template <typename T>
static cudaError_t probe(double* tflops) {
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    T* out = nullptr;
    const int blocks = sms * 8, threads = 256;
    if ((e = cudaMalloc(&out, blocks * sizeof(T))) != cudaSuccess) return e;
    const int iters = sizeof(T) == 8 ? 4096 : 65536;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    k_fma_probe<T><<<blocks, threads>>>(out, iters / 16, (T)0.999999, (T)1e-7);   // warm-up
    cudaEventRecord(t0);
    k_fma_probe<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(t1);
    e = cudaEventSynchronize(t1);
    float ms = 0;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return cudaGetLastError();
}

cudaError_t tc_probe_fma(double* fp64_tflops, double* fp32_tflops) {
    cudaError_t e = probe<double>(fp64_tflops);
    if (e != cudaSuccess) return e;
    return probe<float>(fp32_tflops);
}
