// gea_noalloc.cu -- total mass and total energy of a caller-owned state with
// no device allocation (gea_mass_energy_noalloc in include/gea.h).
//
// Some callers cannot allocate device memory: their device memory is owned by
// a framework's caching allocator or a fixed arena, or they run in a loop
// that must not call cudaMalloc (it can synchronise the device or fail at
// run time). This entry point needs no context and allocates nothing: the
// per-block partial sums and the arrival counter of its reduction live in a
// fixed file-scope device array, resident on every device that loads the
// library until the process exits.
//
// In host code, g_scratch names a host-side stand-in, not a device address;
// the device address is looked up once per device with cudaGetSymbolAddress
// (with that device current) and passed to the kernel.
#include "../../include/gea.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int kThreads = 256;
// blocks of the largest accepted launch, ceil(GEA_NOALLOC_MAX_CELLS / kThreads):
// every block of a launch has a partial slot
constexpr int kMaxBlocks = (GEA_NOALLOC_MAX_CELLS + kThreads - 1) / kThreads;
static_assert((long long)kMaxBlocks * kThreads >= GEA_NOALLOC_MAX_CELLS, "a partial slot per block");
constexpr int kMaxDevices = 64;

// [0, kMaxBlocks): mass partials, [kMaxBlocks, 2 kMaxBlocks): energy partials,
// then the arrival counter (its own 256-byte slot).
static __device__ __align__(256) double g_scratch[2 * kMaxBlocks + 32];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One thread per cell of a dense nz x nx state: m = rho V, e = rho (cv T + K +
// g z) V; block sums into scratch, the last block adds them in a fixed order.
__global__ void k_mass_energy_fixed(int nx, int nz, double dx, double dz, double cv, double g,
                                    const double *__restrict__ rho, const double *__restrict__ u,
                                    const double *__restrict__ w, const double *__restrict__ T,
                                    double *__restrict__ out, double *scratch)
{
    __shared__ double sm[kThreads / 32], se[kThreads / 32];
    __shared__ int am_last;
    const long long n = (long long)nx * nz;
    const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int nb = gridDim.x;
    double m = 0.0, e = 0.0;
    if (t < n) {
        const int k = (int)(t / nx);
        const double V = dx * dz, z = (k + 0.5) * dz;
        const double K = 0.5 * (u[t] * u[t] + w[t] * w[t]);
        m = rho[t] * V;
        e = rho[t] * (cv * T[t] + K + g * z) * V;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    m = warp_sum(m);
    e = warp_sum(e);
    if (lane == 0) { sm[wid] = m; se[wid] = e; }
    __syncthreads();
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + 2 * kMaxBlocks);
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) { a += sm[q]; b += se[q]; }
        scratch[blockIdx.x] = a;
        scratch[kMaxBlocks + blockIdx.x] = b;
        __threadfence();
        am_last = atomicAdd(counter, 1u) == (unsigned)nb - 1u;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nb; q += kThreads) {
        a += __ldcg(&scratch[q]);
        b += __ldcg(&scratch[kMaxBlocks + q]);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    __syncthreads();
    if (lane == 0) { sm[wid] = a; se[wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) { ta += sm[q]; tb += se[q]; }
        out[0] = ta;
        out[1] = tb;
        *counter = 0u;
    }
}

// Device address of g_scratch on the current device, looked up once per
// device and kept for the life of the process (a cudaDeviceReset unloads the
// module, after which the kept address is stale: the header says so).
cudaError_t scratch_address(double **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *ptr = static_cast<double *>(g_addr[dev]);
    return cudaSuccess;
}

}  // namespace

extern "C" int gea_mass_energy_noalloc(int32_t nx, int32_t nz, double lx, double lz, double cp,
                                       double R, double g, const double *rho, const double *u,
                                       const double *w, const double *T, double *out, void *stream)
{
    if (nx < 1 || nz < 1 || !(lx > 0) || !(lz > 0) || !rho || !u || !w || !T || !out)
        return GEA_ERR_INVAL;
    const long long n = (long long)nx * nz;
    if (n > GEA_NOALLOC_MAX_CELLS) return GEA_ERR_INVAL;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return GEA_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero
    if (cudaMemsetAsync(scratch + 2 * kMaxBlocks, 0, sizeof(unsigned), st) != cudaSuccess)
        return GEA_ERR_CUDA;
    const int blocks = (int)((n + kThreads - 1) / kThreads);
    k_mass_energy_fixed<<<blocks, kThreads, 0, st>>>(nx, nz, lx / nx, lz / nz, cp - R, g, rho, u, w,
                                                      T, out, scratch);
    return cudaGetLastError() == cudaSuccess ? GEA_OK : GEA_ERR_CUDA;
}
