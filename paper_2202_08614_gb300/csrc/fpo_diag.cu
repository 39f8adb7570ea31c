// Diagnostics: the FP32 FMA throughput of the device, the denominator of the
// FP32 roofline for the library's SIMT arithmetic kernels (the latent
// decoder's FP32 decode and gradient, the per-visit IDFT), measured on the
// GPU itself rather than taken from a data sheet.
#include <cuda_runtime.h>

#include <cstdint>

#include "fpo.h"
#include "fpo_internal.h"

namespace fpo {
namespace {

constexpr int FMA_CHAINS = 16;  // independent dependency chains per thread

// Every thread runs FMA_CHAINS independent chains a = a * b + c for `iters`
// steps (2 flop each); b and c arrive at run time, so nothing folds.  One
// value per thread is stored, so nothing is eliminated.
__global__ void __launch_bounds__(1024) fma_peak_kernel(float *sink, uint32_t iters, float b, float c)
{
    float a[FMA_CHAINS];
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < FMA_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) s += a[k];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace fpo

extern "C" int fpo_fma_peak(uint32_t blocks, uint32_t threads, uint32_t iters, float *sink, double *flops,
                            void *cuda_stream)
{
    using namespace fpo;
    if (blocks == 0 || threads == 0 || threads > 1024 || (threads & 31) != 0)
        return set_last_error(FPO_ERR_INVALID_ARG, "blocks > 0, threads a multiple of 32 in [32, 1024]");
    if (!sink) return set_last_error(FPO_ERR_INVALID_ARG, "sink is NULL");
    fma_peak_kernel<<<blocks, threads, 0, (cudaStream_t)cuda_stream>>>(sink, iters, 0.999999f, 1e-6f);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_last_error(FPO_ERR_CUDA, cudaGetErrorString(e));
    if (flops) *flops = 2.0 * FMA_CHAINS * (double)iters * (double)blocks * (double)threads;
    return FPO_OK;
}
