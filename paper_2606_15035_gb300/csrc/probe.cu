// pic_probe_fma_rates: measured FMA throughput of this GPU in FP64 and FP32 (sm_103a).
//
// The FP64 particle kernels of this library are bound by the FP64 pipe, not by HBM, so
// their roofline divides by an arithmetic peak.  The derived peak (SM count x FMA per clock
// per SM x clock) is backed by this probe: every thread runs independent FMA chains
// x <- x * b + c (8 per thread, so that the pipe, not the dependency latency, sets the rate)
// over a grid that fills every SM, timed with CUDA events on the given stream.
#include "pic_internal.h"

namespace {

constexpr int CHAINS = 8;
constexpr int PROBE_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_chains(int iters, T b, T c, T* __restrict__ out) {
    T x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = T(1) + T(k) * T(1e-3) + T(threadIdx.x) * T(1e-6);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s == T(-12345)) out[0] = s;   // never true: keeps the chains live
}

template <typename T>
double rate(cudaStream_t st, int blocks, int iters, T* out) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // b slightly below 1 and c small keep every chain bounded and normal
    k_fma_chains<T><<<blocks, PROBE_THREADS, 0, st>>>(iters, T(0.9999999), T(1e-7), out);   // warm-up
    cudaEventRecord(a, st);
    k_fma_chains<T><<<blocks, PROBE_THREADS, 0, st>>>(iters, T(0.9999999), T(1e-7), out);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double flops = 2.0 * CHAINS * (double)iters * blocks * PROBE_THREADS;
    return ms > 0.0f ? flops / (ms * 1e-3) : 0.0;
}

}  // namespace

extern "C" pic_status pic_probe_fma_rates(void* stream, double* fp64_flops, double* fp32_flops) {
    if (!fp64_flops || !fp32_flops) return PIC_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    void* out = nullptr;
    // the probe's only output slot (never written in practice) lives in the library's stream-ordered
    // scratch: one 8-byte allocation for the duration of the call
    if (cudaMallocAsync(&out, sizeof(double), st) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_OOM;
    }
    const int blocks = sms * 16;
    *fp64_flops = rate<double>(st, blocks, 4096, static_cast<double*>(out));
    *fp32_flops = rate<float>(st, blocks, 65536, static_cast<float*>(out));
    cudaFreeAsync(out, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    return PIC_OK;
}
