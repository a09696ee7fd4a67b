// Measured arithmetic peaks of the GPU for the roofline of the ALU-bound
// stage kernels: a kernel of independent fused multiply-add chains in FP32
// or FP64, timed with CUDA events.  Diagnostics only; no step uses it.
#include <cuda_runtime.h>

#include "../../include/cgks.h"

namespace {

// CH independent chains per thread, each an FMA recurrence x = x * a + b
// whose values stay bounded (|a| < 1); the result is written so that the
// compiler keeps every chain.
template <typename T, int CH>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b)
{
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int nsm, double* tflops, float* ms_out)
{
    constexpr int CH = 8;
    const int threads = 256, per_sm = 8;
    const int blocks = nsm * per_sm;
    const int iters = sizeof(T) == 4 ? 4096 : 256;
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return CGKS_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = CGKS_OK;
    float best = 1e30f;
    for (int rep = 0; rep < 5 && rc == CGKS_OK; ++rep) {
        cudaEventRecord(e0);
        k_fma<T, CH><<<blocks, threads>>>(out, iters, (T)0.999, (T)1e-4);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = CGKS_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // the first launch warms up
    }
    if (cudaGetLastError() != cudaSuccess) rc = CGKS_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (rc) return rc;
    double flops = 2.0 * 16.0 * CH * (double)iters * threads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return CGKS_OK;
}

} // namespace

extern "C" int cgks_fma_peak(int precision, double* tflops, float* ms)
{
    if (!tflops || (precision != CGKS_FP64 && precision != CGKS_FP32_BULK)) return CGKS_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CGKS_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CGKS_ECUDA;
    return precision == CGKS_FP64 ? run<double>(nsm, tflops, ms) : run<float>(nsm, tflops, ms);
}
