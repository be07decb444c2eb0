// gea_debug.cu -- pad poisoning and checking for GEA_FLAG_DEBUG_PADS
// contexts (include/gea.h, "Pad checking"), a stand-in for a device memory
// checker: the pads of every pitched array (row padding, the array's unused
// tail and the guard band behind it) hold a NaN pattern, and a check counts
// the pads that no longer hold it.
#include "gea_internal.cuh"
#include "gea_debug.cuh"
#include "../../include/gea.h"

namespace gea {

namespace {

constexpr int kPadThreads = 256;
constexpr int kPadBlocksPerRegion = 16;

__device__ __forceinline__ bool is_pad(const PadRegionDev &r, long long e)
{
    const long long row = e / r.pitch;
    const long long col = e - row * r.pitch;
    return row >= r.rows || col >= r.cols;
}

// blockIdx.y: region; the blocks of a region stride over its elements
__global__ void k_pad_poison(const PadRegionDev *R)
{
    const PadRegionDev r = R[blockIdx.y];
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < r.span; e += step) {
        if (!is_pad(r, e)) continue;
        if (r.esize == 8) reinterpret_cast<unsigned long long *>(r.ptr)[e] = GEA_PAD_POISON64;
        else reinterpret_cast<unsigned *>(r.ptr)[e] = GEA_PAD_POISON32;
    }
}

// Counts the changed pads into res->bad. The first changed element is
// recorded as key = region << 40 | element, for the lowest `ordinal` that
// found one (res->first: checks run in launch order, so a later check that
// finds the same changed pads does not displace the first launch's key).
__global__ void k_pad_check(const PadRegionDev *R, PadResult *res, int ordinal)
{
    const int reg = blockIdx.y;
    const PadRegionDev r = R[reg];
    const long long step = (long long)gridDim.x * blockDim.x;
    unsigned long long nbad = 0, key = ~0ull;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < r.span; e += step) {
        if (!is_pad(r, e)) continue;
        const bool ok = r.esize == 8 ? reinterpret_cast<const unsigned long long *>(r.ptr)[e] == GEA_PAD_POISON64
                                     : reinterpret_cast<const unsigned *>(r.ptr)[e] == GEA_PAD_POISON32;
        if (!ok) {
            ++nbad;
            const unsigned long long k = ((unsigned long long)reg << 40) | (unsigned long long)e;
            key = k < key ? k : key;
        }
    }
    if (nbad) {
        atomicAdd(&res->bad, nbad);
        if (atomicMin(&res->first, ordinal) >= ordinal) atomicMin(&res->key, key);
    }
}

}  // namespace

cudaError_t launch_pad_poison(const PadRegionDev *R, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_pad_poison<<<dim3(kPadBlocksPerRegion, n), kPadThreads, 0, st>>>(R);
    return cudaGetLastError();
}

cudaError_t launch_pad_check(const PadRegionDev *R, int n, PadResult *res, int ordinal, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_pad_check<<<dim3(kPadBlocksPerRegion, n), kPadThreads, 0, st>>>(R, res, ordinal);
    return cudaGetLastError();
}

}  // namespace gea
