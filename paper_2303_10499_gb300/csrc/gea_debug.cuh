// gea_debug.cuh -- pad checking of GEA_FLAG_DEBUG_PADS contexts
// (gea_debug.cu; used by the context code in gea_capi.cu).
#pragma once
#include <cuda_runtime.h>

namespace gea {

constexpr int kMaxPadRegions = 512;   // arrays of one context, at most
// One pitched array: rows x cols elements in use, row pitch `pitch`, `span`
// elements up to the next array (tail and guard band included).
struct PadRegionDev {
    char *ptr;
    long long span;
    int esize, pitch, rows, cols;
};
// first: lowest check ordinal that found a changed pad (INT_MAX: none); key:
// region << 40 | element of the lowest changed pad that check found
struct PadResult {
    unsigned long long bad;
    unsigned long long key;
    int first;
    int pad_;
};
cudaError_t launch_pad_poison(const PadRegionDev *R, int n, cudaStream_t st);
cudaError_t launch_pad_check(const PadRegionDev *R, int n, PadResult *res, int ordinal, cudaStream_t st);

}  // namespace gea
