// gea_probe.cu -- arithmetic peak probe (gea_probe_fma in include/gea.h)
// and grid-barrier latency probe (gea_probe_barrier).
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

// Words of the barrier probe's scratch: the arrival counter, a status word
// (read after every barrier when asked, as the persistent step kernels do),
// and the give-up flag.
struct BarScratch {
    unsigned count;
    int status;
    int gave_up;
};

constexpr unsigned long long kBarPolls = 1ull << 22;

// `iters` grid barriers of the persistent step kernels' protocol: thread 0
// of each block arrives with one acquire-release add on a monotone counter
// and polls it with acquire loads until it reaches k x blocks; the block's
// threads meet at __syncthreads on both sides. A poll limit bounds every
// wait: a block that gives up sets the flag, and every block leaves at its
// next barrier once the flag is set.
__global__ void __launch_bounds__(kProbeThreads) k_grid_barriers(BarScratch *w, int iters, int read_status)
{
    __shared__ int s_stop;
    const unsigned nb = gridDim.x;
    for (int it = 0; it < iters; ++it) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned target = (unsigned)(it + 1) * nb;
            unsigned c;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(c) : "l"(&w->count) : "memory");
            c += 1u;
            unsigned long long polls = 0;
            while ((int)(c - target) < 0) {
                if (polls++ >= kBarPolls) {
                    atomicExch(&w->gave_up, 1);
                    break;
                }
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(&w->count) : "memory");
            }
            int st = 0;
            if (read_status) asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(st) : "l"(&w->status) : "memory");
            s_stop = st | *(volatile int *)&w->gave_up;
        }
        __syncthreads();
        if (s_stop) break;
    }
}

}  // namespace

extern "C" int gea_probe_barrier(int32_t blocks, int32_t iters, int32_t read_status, void *scratch, void *stream)
{
    if (blocks < 1 || iters < 1 || !scratch) return GEA_ERR_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_barriers, kProbeThreads, 0) != cudaSuccess)
        return GEA_ERR_CUDA;
    // every block must be resident at once (the cooperative launch checks it too)
    if ((long long)blocks > (long long)sms * per_sm) return GEA_ERR_INVAL;
    BarScratch *w = static_cast<BarScratch *>(scratch);
    if (cudaMemsetAsync(w, 0, sizeof(BarScratch), st) != cudaSuccess) return GEA_ERR_CUDA;
    int rs = read_status ? 1 : 0;
    void *args[] = {&w, &iters, &rs};
    if (cudaLaunchCooperativeKernel((const void *)k_grid_barriers, dim3(blocks), dim3(kProbeThreads), args, 0, st) !=
        cudaSuccess)
        return GEA_ERR_CUDA;
    return GEA_OK;
}

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
