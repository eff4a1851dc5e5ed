// Compute-peak microbenchmark used by the benchmark for its ALU rooflines:
// independent FMA chains on every SM in FP32 and FP64, timed with CUDA
// events.  Built into its own library (libpeaks_gb300.so); not part of the
// solver's C ABI.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;   // independent dependency chains per thread
constexpr int kThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma(R* out, int iters, R b, R c) {
    R a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = R(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    R s = R(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename R>
double run(int iters, int blocks_per_sm) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1.0;
    const int blocks = sms * blocks_per_sm;
    R* out = nullptr;
    if (cudaMalloc(&out, sizeof(R) * (size_t)blocks * kThreads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b close to 1 and c small keep the chains finite for any iteration count
    const R b = R(0.999999), c = R(1e-3);
    k_fma<R><<<blocks, kThreads>>>(out, iters / 10 + 1, b, c);  // warm-up
    cudaEventRecord(e0);
    k_fma<R><<<blocks, kThreads>>>(out, iters, b, c);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || ms <= 0.f) return -1.0;
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
    return flops / (ms * 1e-3) / 1e12;
}

}  // namespace

// Measured FMA throughput in TFLOP/s (2 flops per FMA) of the current device;
// negative on a CUDA error.
extern "C" double peaks_fp32_tflops(int iters) { return run<float>(iters, 8); }
extern "C" double peaks_fp64_tflops(int iters) { return run<double>(iters, 8); }
