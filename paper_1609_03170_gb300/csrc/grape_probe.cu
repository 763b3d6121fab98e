// grape_probe.cu - measured FMA throughput of the device (FP32 and FP64), the
// denominators of the propagation kernels' ALU roofline: the double-float
// kernels run on the FP32 pipes, the native ones on the FP64 pipe.
//
// Every thread runs kChains independent multiply-add chains
// x <- x * a + b with |a| < 1 (they settle at b / (1 - a): no overflow and
// no subnormals), kUnroll rounds per loop iteration, so the pipes always
// have independent work; one store per thread keeps the chains live.
#include "grape.h"
#include "grape_internal.h"

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T *out, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x & 7) * T(0.125) + T(c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t probe(int blocks_per_sm, int iters, double *tflops, double *ms_out) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const int blocks = sms * blocks_per_sm;
    T *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-6);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first run warms up
        cudaEventRecord(e0, s);
        fma_probe_kernel<T><<<blocks, threads, 0, s>>>(out, iters, a, b);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) {
        const double fmas = (double)blocks * threads * iters * kUnroll * kChains;
        *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
        *ms_out = best;
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    return e;
}

}  // namespace

// precision: GRAPE_PREC_DF64 measures the FP32 pipes, GRAPE_PREC_FP64 the
// FP64 pipe; about 50 ms per run at the nominal rates (80 TFLOP/s FP32,
// 1.2 TFLOP/s FP64), best of three after one warm-up run
cudaError_t grape_probe_fma(int precision, double *tflops, double *ms) {
    return precision == GRAPE_PREC_FP64 ? probe<double>(4, 6000, tflops, ms)
                                        : probe<float>(8, 100000, tflops, ms);
}
