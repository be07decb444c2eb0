// gea_probe.cu -- arithmetic peak probe (gea_probe_fma in include/gea.h).
//
// The time step's stencil and solver kernels are bound by the FP64 issue
// rate of GB300 (two FP64 FMA lanes per SM), not by HBM. Their roofline needs
// that peak as a measured number on the same GPU and clocks: this kernel runs
// eight independent FMA chains per thread, long enough that the pipe is
// saturated and the launch overhead is negligible, and the caller times it
// with CUDA events. The paper has no counterpart.
#include "../../include/gea.h"

#include <cuda_runtime.h>

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <class R>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(int iters, R a, R b, R *out)
{
    R x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (R)(threadIdx.x + 1) * (R)1e-3 + (R)j;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], a, b);
    }
    R s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    // every chain feeds the stored value, so none can be removed
    out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int gea_probe_fma(int32_t bits, int32_t blocks, int32_t iters, void *out, void *stream)
{
    if ((bits != 64 && bits != 32) || blocks < 1 || iters < 1 || !out) return GEA_ERR_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // a slightly contracting map keeps the chains bounded: x -> a x + b
    // converges to b / (1 - a)
    if (bits == 64)
        k_fma_chains<double><<<blocks, kProbeThreads, 0, st>>>(iters, 0.999999, 1e-6, static_cast<double *>(out));
    else
        k_fma_chains<float><<<blocks, kProbeThreads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float *>(out));
    return cudaGetLastError() == cudaSuccess ? GEA_OK : GEA_ERR_CUDA;
}
