// Arithmetic-pipe throughput probes for the roofline of the plain FP64 form.
//
// GB300's FP64 pipe is narrow, so the FP64 form of the sifting kernels is bound by FP64
// arithmetic rather than by memory. Its roofline needs the measured FP64 rate of this GPU,
// which these kernels provide: every thread runs kChains independent chains of fused
// multiply-adds (2 flops each) in registers, enough warps per SM to fill the pipe, no
// memory traffic besides one store per thread. The probes change no GPU setting.
#include <cuda_runtime.h>

#include <string>

#include "semd_runtime.h"

namespace semd {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static semd_status fma_rate(int iters, double *gflops, cudaStream_t s, std::string &err)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        err = "no CUDA device";
        return SEMD_ECUDA;
    }
    const int blocks = sms * 8, threads = 256;
    T *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&out, (size_t)blocks * threads * sizeof(T), s);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_fma_probe<T><<<blocks, threads, 0, s>>>(out, iters / 10 + 1, T(0.999), T(1e-3));
        cudaEventRecord(e0, s);
        k_fma_probe<T><<<blocks, threads, 0, s>>>(out, iters, T(0.999), T(1e-3));
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, e0, e1);
    if (out)
        cudaFreeAsync(out, s);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        err = std::string("probe: ") + cudaGetErrorString(e);
        return SEMD_ECUDA;
    }
    const double flops = 2.0 * kChains * (double)iters * blocks * threads;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return SEMD_OK;
}

} // namespace semd

extern "C" semd_status serial_emd_fma_rate(int precision, int iters, double *gflops, void *stream)
{
    std::string err;
    if (!gflops || iters < 1 || (precision != SEMD_FP64 && precision != SEMD_FP32_MIXED))
        return SEMD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == SEMD_FP64 ? semd::fma_rate<double>(iters, gflops, s, err)
                                  : semd::fma_rate<float>(iters, gflops, s, err);
}
