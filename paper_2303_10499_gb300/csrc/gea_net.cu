// gea_net.cu -- the learned pressure-correction network: a convolutional
// multigrid-style U-Net (4 levels, 16 base channels) with its forward pass,
// energy loss, backward pass and Adam update, all on the GPU.
//
// The 3x3 layers with 16-64 channels run on the tensor cores (gea_conv.cu):
// forward, and the data gradient as the same correlation with the taps
// mirrored and the channel roles swapped. The first layer (one input
// channel), the 1x1 output layer, the weight gradients (a reduction over all
// pixels into at most 64 x 64 x 9 values per layer, which does not fill a
// 128-row MMA tile) and the elementwise parts run on the CUDA cores in FP32.
// Every reduction is deterministic: per-block partial sums added in a fixed
// order.
#include "../../include/gea.h"
#include "../../include/gea_net.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

cudaError_t gea_conv3x3_launch(int n, int h, int w, int cin, int cout, int mode, int flags, const uint16_t *x0,
                               const uint16_t *x1, const uint16_t *wt, const float *bias, void *y, int *status,
                               cudaStream_t st);

namespace gea_net_impl {

enum { SRC_X = 0, SRC_PREV = 1, SRC_POOL = 2, SRC_UPADD = 3 };

// cin, cout, kernel size, activation, input kind, input layer a (the layer
// read, averaged or prolonged), skip layer b (UPADD), level
struct LayerDef {
    int cin, cout, k, act, kind, a, b, level;
};

constexpr int L = GEA_NET_LAYERS;
constexpr LayerDef kL[L] = {
    {1, 16, 3, 1, SRC_X, -1, -1, 0},     // e0a
    {16, 16, 3, 1, SRC_PREV, 0, -1, 0},  // e0b
    {16, 32, 3, 1, SRC_POOL, 1, -1, 1},  // e1a
    {32, 32, 3, 1, SRC_PREV, 2, -1, 1},  // e1b
    {32, 64, 3, 1, SRC_POOL, 3, -1, 2},  // e2a
    {64, 64, 3, 1, SRC_PREV, 4, -1, 2},  // e2b
    {64, 64, 3, 1, SRC_POOL, 5, -1, 3},  // e3a
    {64, 64, 3, 1, SRC_PREV, 6, -1, 3},  // e3b
    {64, 64, 3, 1, SRC_UPADD, 7, 5, 2},  // d2a
    {64, 32, 3, 1, SRC_PREV, 8, -1, 2},  // d2b
    {32, 32, 3, 1, SRC_UPADD, 9, 3, 1},  // d1a
    {32, 16, 3, 1, SRC_PREV, 10, -1, 1}, // d1b
    {16, 16, 3, 1, SRC_UPADD, 11, 1, 0}, // d0a
    {16, 16, 3, 1, SRC_PREV, 12, -1, 0}, // d0b
    {16, 1, 1, 0, SRC_PREV, 13, -1, 0},  // out
};
constexpr int kOut = L - 1;
constexpr int kThreads = 256;
constexpr int kWgThreads = 128;
constexpr int kWgTile = 128;     // pixels per weight-gradient tile (one row segment)
constexpr int kMaxSlices = 96;   // weight-gradient CTAs per tap

__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
__device__ __forceinline__ uint16_t f2bf(float f)
{
    __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ float round_bf(float f) { return bf2f(f2bf(f)); }

// ---- per-sample sums (deterministic: block partials, then a fixed-order sum) ----

// part[b * gridDim.x + blk] = sum over the block's share of sample b of v^2
// (sq) or v. A thread takes four consecutive values at a time (per is a
// multiple of 64) into four FP64 sums, which it adds in a fixed order, with
// one 16-byte load when x is 16-byte aligned (vec); v^2 of an FP32 value is
// exact in FP64, so fma(v, v, s) adds it with the one rounding of the sum.
__global__ void k_sample_partials(const float *x, long long per, int sq, int vec, double *part)
{
    __shared__ double red[kThreads];
    const int b = blockIdx.y;
    const float *xs = x + (size_t)b * per;
    const long long n4 = per / 4;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n4; i += (long long)gridDim.x * kThreads) {
        float4 v;
        if (vec) {
            v = __ldg(reinterpret_cast<const float4 *>(xs) + i);
        } else {
            v.x = __ldg(&xs[4 * i]); v.y = __ldg(&xs[4 * i + 1]);
            v.z = __ldg(&xs[4 * i + 2]); v.w = __ldg(&xs[4 * i + 3]);
        }
        if (sq) {
            s0 = fma((double)v.x, (double)v.x, s0);
            s1 = fma((double)v.y, (double)v.y, s1);
            s2 = fma((double)v.z, (double)v.z, s2);
            s3 = fma((double)v.w, (double)v.w, s3);
        } else {
            s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
        }
    }
    red[threadIdx.x] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = red[0];
}

// out[b] = scale(sum of the nblk partials of sample b); mode 0: sqrt(s / per)
// (rms), 1: s / per (mean). One block per sample: thread t adds partials
// t, t + kThreads, ..., then a fixed-order tree.
__global__ void k_sample_finish(const double *part, int nblk, long long per, int mode, float *out)
{
    __shared__ double red[kThreads];
    const int b = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) s += part[(size_t)b * nblk + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = mode == 0 ? (float)sqrt(red[0] / (double)per) : (float)(red[0] / (double)per);
}

// x = r / rms per sample (0 if rms = 0), FP32 and bfloat16
__global__ void k_prep(const float *r, const float *rms, long long per, long long total, float *xh, uint16_t *xb)
{
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (i >= total) return;
    const float s = rms[i / per];
    const float v = s > 0.0f ? r[i] / s : 0.0f;
    xh[i] = v;
    xb[i] = f2bf(v);
}

// ---- first layer (1 input channel) and output layer (1x1) on the CUDA cores ----

// Pixels of one row per thread in the first layer (w is a multiple of 8):
// each weight read from shared memory serves kFirstPix multiply-adds.
constexpr int kFirstPix = 4;

__global__ void __launch_bounds__(kThreads) k_conv_first(int n, int h, int w, const uint16_t *x, const float *wt,
                                                         const float *bias, int relu, uint16_t *y)
{
    __shared__ float sw[16 * 9], sb[16];
    for (int e = threadIdx.x; e < 16 * 9; e += kThreads) sw[e] = round_bf(wt[e]);
    if (threadIdx.x < 16) sb[threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    const long long p0 = (blockIdx.x * (long long)kThreads + threadIdx.x) * kFirstPix;
    if (p0 >= (long long)n * h * w) return;
    const int j0 = (int)(p0 % w);
    const int i = (int)((p0 / w) % h);
    const long long base = p0 - ((long long)i * w + j0);
    // input rows i-1..i+1, columns j0-1..j0+kFirstPix (zero outside the image)
    float xv[3][kFirstPix + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int ii = i + r - 1;
#pragma unroll
        for (int c = 0; c < kFirstPix + 2; ++c) {
            const int jj = j0 + c - 1;
            xv[r][c] = (ii >= 0 && ii < h && jj >= 0 && jj < w) ? bf2f(x[base + (long long)ii * w + jj]) : 0.0f;
        }
    }
    // per output: the bias, then the taps in row-major order, one FMA each
    uint32_t u[kFirstPix][8];
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
        float o[2][kFirstPix];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int px = 0; px < kFirstPix; ++px) o[k][px] = sb[c + k];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float wv = sw[(c + k) * 9 + t];
#pragma unroll
                for (int px = 0; px < kFirstPix; ++px) o[k][px] = fmaf(wv, xv[t / 3][px + t % 3], o[k][px]);
            }
#pragma unroll
            for (int px = 0; px < kFirstPix; ++px)
                if (relu) o[k][px] = fmaxf(o[k][px], 0.0f);
        }
#pragma unroll
        for (int px = 0; px < kFirstPix; ++px)
            u[px][c / 2] = (uint32_t)f2bf(o[0][px]) | ((uint32_t)f2bf(o[1][px]) << 16);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(y + p0 * 16);
#pragma unroll
    for (int px = 0; px < kFirstPix; ++px) {
        dst[2 * px] = make_uint4(u[px][0], u[px][1], u[px][2], u[px][3]);
        dst[2 * px + 1] = make_uint4(u[px][4], u[px][5], u[px][6], u[px][7]);
    }
}

__global__ void k_conv_out(long long npix, const uint16_t *x, const float *wt, const float *bias, float *y)
{
    const long long p = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (p >= npix) return;
    const uint4 *src = reinterpret_cast<const uint4 *>(x + p * 16);
    const uint4 a = src[0], b = src[1];
    const uint32_t u[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    float s = bias[0];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        s = fmaf(round_bf(wt[2 * c]), bf2f((uint16_t)(u[c] & 0xFFFFu)), s);
        s = fmaf(round_bf(wt[2 * c + 1]), bf2f((uint16_t)(u[c] >> 16)), s);
    }
    y[p] = s;
}

// Output layer backward: g13[p][c] = dy[p] w[c]; block partials of
// dW[c] = sum dy x[p][c] and db = sum dy (17 per block).
__global__ void k_out_backward(long long npix, const float *dy, const uint16_t *x, const float *wt, float *g13,
                               float *part)
{
    __shared__ float red[17][kThreads];
    const long long p = blockIdx.x * (long long)kThreads + threadIdx.x;
    float v[17];
#pragma unroll
    for (int c = 0; c < 17; ++c) v[c] = 0.0f;
    if (p < npix) {
        const float d = dy[p];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            g13[p * 16 + c] = d * round_bf(wt[c]);
            v[c] = d * bf2f(x[p * 16 + c]);
        }
        v[16] = d;
    }
#pragma unroll
    for (int c = 0; c < 17; ++c) red[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < 17; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 17) part[(size_t)blockIdx.x * 17 + threadIdx.x] = red[threadIdx.x][0];
}

// out[j] = sum over s < ns of part[s * stride + j], j < nout
__global__ void k_sum_partials(const float *part, int ns, int stride, int nout, float *out)
{
    const int j = blockIdx.x * kThreads + threadIdx.x;
    if (j >= nout) return;
    float s = 0.0f;
    for (int i = 0; i < ns; ++i) s += part[(size_t)i * stride + j];
    out[j] = s;
}

// ---- backward elementwise parts ----

// g *= (act > 0) when relu; gb = bfloat16(g)
__global__ void k_mask(long long cnt, float *g, const uint16_t *act, int relu, uint16_t *gb)
{
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (i >= cnt) return;
    float v = g[i];
    if (relu && !(bf2f(act[i]) > 0.0f)) v = 0.0f;
    g[i] = v;
    if (gb) gb[i] = f2bf(v);
}

__global__ void k_add(long long cnt, float *dst, const float *src)
{
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (i < cnt) dst[i] += src[i];
}

// the gradient of a 2x2 average: dst (n x 2h x 2w x c) += gin(n x h x w x c) / 4
__global__ void k_pool_backward(int n, int h, int w, int c, float *dst, const float *gin)
{
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    const long long tot = (long long)n * 4 * h * w * c;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long pix = i / c;
    const int W2 = 2 * w, H2 = 2 * h;
    const int x = (int)(pix % W2), y = (int)((pix / W2) % H2);
    const long long b = pix / ((long long)W2 * H2);
    dst[i] += 0.25f * gin[(((size_t)b * h + y / 2) * w + x / 2) * c + ch];
}

// the gradient of a nearest-neighbour prolongation: dst (n x h/2 x w/2 x c)
// += sum of the 2x2 children in gin (n x h x w x c)
__global__ void k_up_backward(int n, int h, int w, int c, float *dst, const float *gin)
{
    const int hc = h / 2, wc = w / 2;
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    const long long tot = (long long)n * hc * wc * c;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long pix = i / c;
    const int x = (int)(pix % wc), y = (int)((pix / wc) % hc);
    const long long b = pix / ((long long)wc * hc);
    const float *g = gin + (((size_t)b * h + 2 * y) * w + 2 * x) * c + ch;
    dst[i] += (g[0] + g[c]) + (g[(size_t)w * c] + g[(size_t)w * c + c]);
}

// ---- weight gradients (FP32, CUDA cores) ----

struct WgArgs {
    int n, h, w;            // the layer's (output) size; POOL sources are 2h x 2w
    const uint16_t *x0, *x1;
    const float *g;         // masked output gradient, n x h x w x cout
    float *part;            // [slice][tap][cout * cin]
    float *partb;           // [slice][cout]
    int ntiles, tiles_per_row, nslices;
};

// The input value of the layer (fused as the forward pass forms it) at
// pixel (b, yy, xx), channel c; zero outside the image.
template <int CIN, int MODE>
__device__ __forceinline__ float wg_input(const WgArgs &a, int b, int yy, int xx, int c)
{
    if (yy < 0 || yy >= a.h || xx < 0 || xx >= a.w) return 0.0f;
    if (MODE == GEA_CONV_PLAIN) return bf2f(a.x0[(((size_t)b * a.h + yy) * a.w + xx) * CIN + c]);
    if (MODE == GEA_CONV_POOL) {
        const size_t W2 = (size_t)2 * a.w;
        const uint16_t *s = a.x0 + (((size_t)b * 2 * a.h + 2 * yy) * W2 + 2 * xx) * CIN + c;
        return round_bf(0.25f * ((bf2f(s[0]) + bf2f(s[CIN])) + (bf2f(s[W2 * CIN]) + bf2f(s[W2 * CIN + CIN]))));
    }
    const int hc = a.h / 2, wc = a.w / 2;
    return round_bf(bf2f(a.x0[(((size_t)b * a.h + yy) * a.w + xx) * CIN + c]) +
                    bf2f(a.x1[(((size_t)b * hc + yy / 2) * wc + xx / 2) * CIN + c]));
}

// Block (tap, slice): dW[tap][co][ci] += sum over the slice's tiles of
// g[p][co] x[p + off(tap)][ci]; the centre tap's blocks also sum db.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kWgThreads) k_wgrad(WgArgs a)
{
    constexpr int NOUT = CIN * COUT;
    constexpr int PER = (NOUT + kWgThreads - 1) / kWgThreads;
    constexpr int XS = CIN + (CIN > 1 ? 1 : 0);       // padded row of the input tile
    extern __shared__ float wsm[];
    float *gs = wsm;                                  // [kWgTile][COUT]
    float *xs = wsm + kWgTile * COUT;                 // [kWgTile][XS]
    const int tap = blockIdx.x, ntap = gridDim.x;
    const int dy = ntap == 9 ? tap / 3 - 1 : 0, dx = ntap == 9 ? tap % 3 - 1 : 0;
    const bool centre = (ntap == 9 && tap == 4) || ntap == 1;
    const int tid = threadIdx.x;
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.0f;
    float accb = 0.0f;
    for (int t = blockIdx.y; t < a.ntiles; t += a.nslices) {
        const int tx = t % a.tiles_per_row, row = t / a.tiles_per_row;
        const int y = row % a.h, b = row / a.h;
        const int x0 = tx * kWgTile;
        for (int e = tid; e < kWgTile * COUT; e += kWgThreads) {
            const int p = e / COUT, c = e % COUT;
            const int xx = x0 + p;
            gs[e] = xx < a.w ? a.g[(((size_t)b * a.h + y) * a.w + xx) * COUT + c] : 0.0f;
        }
        for (int e = tid; e < kWgTile * CIN; e += kWgThreads) {
            const int p = e / CIN, c = e % CIN;
            xs[p * XS + c] = (x0 + p < a.w) ? wg_input<CIN, MODE>(a, b, y + dy, x0 + p + dx, c) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int j = tid + q * kWgThreads;
            if (j < NOUT) {
                const int co = j / CIN, ci = j % CIN;
                float s = 0.0f;
#pragma unroll 8
                for (int p = 0; p < kWgTile; ++p) s = fmaf(gs[p * COUT + co], xs[p * XS + ci], s);
                acc[q] += s;
            }
        }
        if (centre && tid < COUT) {
            float s = 0.0f;
            for (int p = 0; p < kWgTile; ++p) s += gs[p * COUT + tid];
            accb += s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int j = tid + q * kWgThreads;
        if (j < NOUT) a.part[((size_t)blockIdx.y * ntap + tap) * NOUT + j] = acc[q];
    }
    if (centre && tid < COUT) a.partb[(size_t)blockIdx.y * COUT + tid] = accb;
}

// dW[co][tap][ci] (parameter order) from the slice partials
__global__ void k_wgrad_reduce(const float *part, int nslices, int ntap, int cin, int cout, float *dw)
{
    const int nout = cin * cout;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    if (j >= ntap * nout) return;
    const int tap = j / nout, r = j % nout;
    const int co = r / cin, ci = r % cin;
    float s = 0.0f;
    for (int i = 0; i < nslices; ++i) s += part[((size_t)i * ntap + tap) * nout + r];
    dw[((size_t)co * ntap + tap) * cin + ci] = s;
}

// ---- parameters: bfloat16 weight copies and Adam ----

// wf[co][t][ci] = bf16(W[co][t][ci]); wb[ci][t][co] = bf16(W[co][8 - t][ci])
__global__ void k_pack(const float *W, int cin, int cout, uint16_t *wf, uint16_t *wb)
{
    const int j = blockIdx.x * kThreads + threadIdx.x;
    if (j >= cout * 9 * cin) return;
    const int ci = j % cin, t = (j / cin) % 9, co = j / (9 * cin);
    const uint16_t v = f2bf(W[j]);
    wf[j] = v;
    wb[((size_t)ci * 9 + (8 - t)) * cout + co] = v;
}

__global__ void k_adam(long long np, float *th, float *m, float *v, const float *g, float lr, float b1, float b2,
                       float c1, float c2, float eps)
{
    const long long i = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---- energy loss ----

// q = A y / mean(c); per pixel loss 0.5 y q - y x and gradient (q - x) / (h w n);
// block partials of the loss (double) per sample
__global__ void k_energy(int n, int h, int w, const float *y, const float *x, const float *c, const float *ax,
                         const float *az, const float *cmean, float *dy, double *part)
{
    __shared__ double red[kThreads];
    const int b = blockIdx.y;
    const long long per = (long long)h * w;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < per; i += (long long)gridDim.x * kThreads) {
        const int col = (int)(i % w), row = (int)(i / w);
        const float *ys = y + (size_t)b * per;
        const float yc = ys[i];
        const float *axs = ax + (size_t)b * h * (w + 1);
        const float *azs = az + (size_t)b * (h + 1) * w;
        float q = c[(size_t)b * per + i] * yc;
        if (col > 0) q += axs[(size_t)row * (w + 1) + col] * (yc - ys[i - 1]);
        if (col + 1 < w) q += axs[(size_t)row * (w + 1) + col + 1] * (yc - ys[i + 1]);
        if (row > 0) q += azs[(size_t)row * w + col] * (yc - ys[i - w]);
        if (row + 1 < h) q += azs[(size_t)(row + 1) * w + col] * (yc - ys[i + w]);
        q /= cmean[b];
        const float xv = x[(size_t)b * per + i];
        dy[(size_t)b * per + i] = (q - xv) / (float)((double)per * n);
        s += 0.5 * (double)yc * q - (double)yc * xv;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_energy_finish(const double *part, int nblk, int n, long long per, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot = 0.0;
    for (int b = 0; b < n; ++b) {
        double s = 0.0;
        for (int i = 0; i < nblk; ++i) s += part[(size_t)b * nblk + i];
        tot += s / (double)per;
    }
    *out = tot / n;
}

inline unsigned blocks(long long cnt) { return (unsigned)((cnt + kThreads - 1) / kThreads); }

template <int CIN, int COUT>
cudaError_t wgrad_mode(const WgArgs &a, int mode, int ntap, cudaStream_t st)
{
    const int smem = (kWgTile * COUT + kWgTile * (CIN + (CIN > 1 ? 1 : 0))) * (int)sizeof(float);
    dim3 grid(ntap, a.nslices);
    cudaError_t e = cudaSuccess;
    switch (mode) {
    case GEA_CONV_PLAIN:
        e = cudaFuncSetAttribute(k_wgrad<CIN, COUT, GEA_CONV_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_wgrad<CIN, COUT, GEA_CONV_PLAIN><<<grid, kWgThreads, smem, st>>>(a);
        break;
    case GEA_CONV_POOL:
        e = cudaFuncSetAttribute(k_wgrad<CIN, COUT, GEA_CONV_POOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_wgrad<CIN, COUT, GEA_CONV_POOL><<<grid, kWgThreads, smem, st>>>(a);
        break;
    default:
        e = cudaFuncSetAttribute(k_wgrad<CIN, COUT, GEA_CONV_UPADD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_wgrad<CIN, COUT, GEA_CONV_UPADD><<<grid, kWgThreads, smem, st>>>(a);
        break;
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t wgrad_launch(const WgArgs &a, int cin, int cout, int mode, int ntap, cudaStream_t st)
{
#define GEA_WG(CI, CO) \
    if (cin == CI && cout == CO) return wgrad_mode<CI, CO>(a, mode, ntap, st);
    GEA_WG(1, 16) GEA_WG(16, 16) GEA_WG(16, 32) GEA_WG(32, 32) GEA_WG(32, 64) GEA_WG(64, 64) GEA_WG(64, 32)
    GEA_WG(32, 16)
#undef GEA_WG
    return cudaErrorInvalidValue;
}

}  // namespace gea_net_impl

using namespace gea_net_impl;

struct gea_net {
    int nmax = 0, hmax = 0, wmax = 0, relu = 0;
    cudaStream_t st = nullptr;
    long long np = 0;
    long long offw[L], offb[L];
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *dy = nullptr;
    uint16_t *wf[L] = {}, *wb[L] = {};
    uint16_t *act[L] = {};
    float *gact[L] = {};
    uint16_t *gbf = nullptr, *xbf = nullptr;
    float *gin = nullptr, *xh = nullptr, *rms = nullptr, *cmean = nullptr;
    float *part = nullptr, *partb = nullptr;
    double *dpart = nullptr, *loss = nullptr;
    int *status = nullptr;
    int n = 0, h = 0, w = 0;
    const float *last_y = nullptr;
    int t = 0;
    bool have_fwd = false;
    std::vector<void *> allocs;
};

namespace {

constexpr int kSampleBlocks = 64;
// blocks per sample of the per-sample sums of the forward pass (a read of
// the whole input, as wide as the GPU)
constexpr int kStatBlocks = 608;

long long count_params(long long *offw, long long *offb)
{
    long long o = 0;
    for (int l = 0; l < L; ++l) {
        if (offw) offw[l] = o;
        o += (long long)kL[l].cout * kL[l].k * kL[l].k * kL[l].cin;
        if (offb) offb[l] = o;
        o += kL[l].cout;
    }
    return o;
}

template <class T>
T *take(gea_net *net, size_t count, bool &ok)
{
    void *p = nullptr;
    if (!ok) return nullptr;
    if (cudaMalloc(&p, count * sizeof(T) + 16) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
        return nullptr;
    }
    net->allocs.push_back(p);
    return static_cast<T *>(p);
}

long long level_pix(int n, int h, int w, int lev) { return (long long)n * (h >> lev) * (w >> lev); }

int pack_all(gea_net *net)
{
    for (int l = 1; l < kOut; ++l) {
        const int cnt = kL[l].cout * 9 * kL[l].cin;
        k_pack<<<blocks(cnt), kThreads, 0, net->st>>>(net->theta + net->offw[l], kL[l].cin, kL[l].cout, net->wf[l],
                                                      net->wb[l]);
    }
    return cudaGetLastError() == cudaSuccess ? GEA_OK : GEA_ERR_CUDA;
}

// per-sample reduction of x (n samples of `per` values) into out[b]
void sample_stat(gea_net *net, const float *x, int n, long long per, int mode, float *out)
{
    dim3 g(kStatBlocks, n);
    const int vec = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
    k_sample_partials<<<g, kThreads, 0, net->st>>>(x, per, mode == 0 ? 1 : 0, vec, net->dpart);
    k_sample_finish<<<n, kThreads, 0, net->st>>>(net->dpart, kStatBlocks, per, mode, out);
}

int forward(gea_net *net, int n, int h, int w, const float *r, float *y)
{
    cudaStream_t st = net->st;
    const long long per = (long long)h * w, tot = per * n;
    sample_stat(net, r, n, per, 0, net->rms);
    k_prep<<<blocks(tot), kThreads, 0, st>>>(r, net->rms, per, tot, net->xh, net->xbf);
    k_conv_first<<<blocks(tot / kFirstPix), kThreads, 0, st>>>(n, h, w, net->xbf, net->theta + net->offw[0],
                                                   net->theta + net->offb[0], net->relu && kL[0].act, net->act[0]);
    for (int l = 1; l < kOut; ++l) {
        const LayerDef &d = kL[l];
        const int hl = h >> d.level, wl = w >> d.level;
        const uint16_t *x0 = nullptr, *x1 = nullptr;
        int mode = GEA_CONV_PLAIN;
        if (d.kind == SRC_PREV) x0 = net->act[d.a];
        else if (d.kind == SRC_POOL) { x0 = net->act[d.a]; mode = GEA_CONV_POOL; }
        else { x0 = net->act[d.b]; x1 = net->act[d.a]; mode = GEA_CONV_UPADD; }
        const int flags = (net->relu && d.act) ? GEA_CONV_RELU : 0;
        if (gea_conv3x3_launch(n, hl, wl, d.cin, d.cout, mode, flags, x0, x1, net->wf[l], net->theta + net->offb[l],
                               net->act[l], net->status, st) != cudaSuccess)
            return GEA_ERR_CUDA;
    }
    k_conv_out<<<blocks(tot), kThreads, 0, st>>>(tot, net->act[kOut - 1], net->theta + net->offw[kOut],
                                                 net->theta + net->offb[kOut], y);
    if (cudaGetLastError() != cudaSuccess) return GEA_ERR_CUDA;
    net->n = n; net->h = h; net->w = w;
    net->last_y = y;
    net->have_fwd = true;
    return GEA_OK;
}

int backward(gea_net *net, const float *dy, float *grad)
{
    cudaStream_t st = net->st;
    const int n = net->n, h = net->h, w = net->w;
    const long long tot = (long long)n * h * w;
    for (int l = 0; l < kOut; ++l)
        if (cudaMemsetAsync(net->gact[l], 0, (size_t)level_pix(n, h, w, kL[l].level) * kL[l].cout * sizeof(float),
                            st) != cudaSuccess)
            return GEA_ERR_CUDA;
    // output layer
    {
        const unsigned nb = blocks(tot);
        k_out_backward<<<nb, kThreads, 0, st>>>(tot, dy, net->act[kOut - 1], net->theta + net->offw[kOut],
                                                net->gact[kOut - 1], net->part);
        k_sum_partials<<<1, kThreads, 0, st>>>(net->part, (int)nb, 17, 17, grad + net->offw[kOut]);
    }
    for (int l = kOut - 1; l >= 0; --l) {
        const LayerDef &d = kL[l];
        const int hl = h >> d.level, wl = w >> d.level;
        const long long cnt = level_pix(n, h, w, d.level) * d.cout;
        k_mask<<<blocks(cnt), kThreads, 0, st>>>(cnt, net->gact[l], net->act[l], net->relu && d.act,
                                                 l > 0 ? net->gbf : nullptr);
        // weight gradient
        WgArgs a{};
        a.n = n; a.h = hl; a.w = wl;
        a.g = net->gact[l];
        a.part = net->part; a.partb = net->partb;
        a.tiles_per_row = (wl + kWgTile - 1) / kWgTile;
        a.ntiles = n * hl * a.tiles_per_row;
        a.nslices = a.ntiles < kMaxSlices ? a.ntiles : kMaxSlices;
        int mode = GEA_CONV_PLAIN;
        if (d.kind == SRC_X) a.x0 = net->xbf;
        else if (d.kind == SRC_PREV) a.x0 = net->act[d.a];
        else if (d.kind == SRC_POOL) { a.x0 = net->act[d.a]; mode = GEA_CONV_POOL; }
        else { a.x0 = net->act[d.b]; a.x1 = net->act[d.a]; mode = GEA_CONV_UPADD; }
        if (wgrad_launch(a, d.cin, d.cout, mode, 9, st) != cudaSuccess) return GEA_ERR_CUDA;
        const int nw = 9 * d.cin * d.cout;
        k_wgrad_reduce<<<blocks(nw), kThreads, 0, st>>>(net->part, a.nslices, 9, d.cin, d.cout, grad + net->offw[l]);
        k_sum_partials<<<blocks(d.cout), kThreads, 0, st>>>(net->partb, a.nslices, d.cout, d.cout,
                                                            grad + net->offb[l]);
        if (l == 0) break;
        // data gradient on the tensor cores: correlation of bf16(g) with the
        // mirrored, transposed weights
        if (gea_conv3x3_launch(n, hl, wl, d.cout, d.cin, GEA_CONV_PLAIN, GEA_CONV_OUT_F32, net->gbf, nullptr,
                               net->wb[l], nullptr, net->gin, net->status, st) != cudaSuccess)
            return GEA_ERR_CUDA;
        const long long icnt = level_pix(n, h, w, d.level) * d.cin;
        if (d.kind == SRC_PREV) {
            k_add<<<blocks(icnt), kThreads, 0, st>>>(icnt, net->gact[d.a], net->gin);
        } else if (d.kind == SRC_POOL) {
            k_pool_backward<<<blocks(icnt * 4), kThreads, 0, st>>>(n, hl, wl, d.cin, net->gact[d.a], net->gin);
        } else {
            k_add<<<blocks(icnt), kThreads, 0, st>>>(icnt, net->gact[d.b], net->gin);
            k_up_backward<<<blocks(icnt / 4), kThreads, 0, st>>>(n, hl, wl, d.cin, net->gact[d.a], net->gin);
        }
    }
    return cudaGetLastError() == cudaSuccess ? GEA_OK : GEA_ERR_CUDA;
}

int energy(gea_net *net, const float *c, const float *ax, const float *az, float *dy, float *loss)
{
    if (!net->have_fwd) return GEA_ERR_STATE;
    cudaStream_t st = net->st;
    const int n = net->n, h = net->h, w = net->w;
    const long long per = (long long)h * w;
    sample_stat(net, c, n, per, 1, net->cmean);
    dim3 g(kSampleBlocks, n);
    k_energy<<<g, kThreads, 0, st>>>(n, h, w, net->last_y, net->xh, c, ax, az, net->cmean, dy, net->dpart);
    k_energy_finish<<<1, 32, 0, st>>>(net->dpart, kSampleBlocks, n, per, net->loss);
    double hl = 0.0;
    if (cudaMemcpyAsync(&hl, net->loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GEA_ERR_CUDA;
    if (loss) *loss = (float)hl;
    return GEA_OK;
}

int adam(gea_net *net, const float *grad, float lr)
{
    net->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, net->t)), c2 = (float)(1.0 - pow(b2, net->t));
    k_adam<<<blocks(net->np), kThreads, 0, net->st>>>(net->np, net->theta, net->m, net->v, grad, lr, (float)b1,
                                                      (float)b2, c1, c2, 1e-8f);
    if (cudaGetLastError() != cudaSuccess) return GEA_ERR_CUDA;
    return pack_all(net);
}

bool shape_ok(const gea_net *net, int n, int h, int w)
{
    // every buffer is sized by the total pixel count (and the per-sample
    // arrays by n_max)
    return n >= 1 && n <= net->nmax && h >= 8 && w >= 8 && h % 8 == 0 && w % 8 == 0 &&
           (long long)n * h * w <= (long long)net->nmax * net->hmax * net->wmax;
}

}  // namespace

int gea_net_launches();

int gea_net_run(gea_net *net, cudaStream_t st, int n, int h, int w, const float *r, float *y)
{
    if (!net || !shape_ok(net, n, h, w)) return -1;
    cudaStream_t old = net->st;
    net->st = st;
    const int rc = forward(net, n, h, w, r, y);
    net->st = old;
    return rc ? -1 : gea_net_launches();
}

// per-sample statistics (2), input scaling, first layer, 13 tensor-core
// layers, output layer
int gea_net_launches() { return 2 + 1 + 1 + (kOut - 1) + 1; }

bool gea_net_fits(const gea_net *net, int n, int h, int w) { return net && shape_ok(net, n, h, w); }

extern "C" {

int64_t gea_net_param_count(void) { return count_params(nullptr, nullptr); }

int gea_net_layout(int32_t *desc)
{
    if (!desc) return GEA_ERR_INVAL;
    for (int l = 0; l < L; ++l) {
        const LayerDef &d = kL[l];
        const int32_t v[6] = {d.cin, d.cout, d.k, d.act, d.kind, d.level};
        for (int j = 0; j < 6; ++j) desc[6 * l + j] = v[j];
    }
    return GEA_OK;
}

int gea_net_create(int32_t n_max, int32_t h_max, int32_t w_max, int32_t flags, gea_net **out)
{
    if (!out) return GEA_ERR_INVAL;
    *out = nullptr;
    if (n_max < 1 || h_max < 8 || w_max < 8 || h_max % 8 || w_max % 8 || (flags & ~GEA_NET_RELU) ||
        (long long)n_max * h_max * w_max > (1LL << 31) / 64)
        return GEA_ERR_INVAL;
    gea_net *net = new gea_net();
    net->nmax = n_max; net->hmax = h_max; net->wmax = w_max;
    net->relu = (flags & GEA_NET_RELU) ? 1 : 0;
    net->np = count_params(net->offw, net->offb);
    bool ok = true;
    net->theta = take<float>(net, net->np, ok);
    net->m = take<float>(net, net->np, ok);
    net->v = take<float>(net, net->np, ok);
    net->grad = take<float>(net, net->np, ok);
    const long long pix = (long long)n_max * h_max * w_max;
    net->dy = take<float>(net, pix, ok);
    for (int l = 0; l < L; ++l) {
        const long long lp = level_pix(n_max, h_max, w_max, kL[l].level);
        if (l < kOut) {
            net->act[l] = take<uint16_t>(net, lp * kL[l].cout, ok);
            net->gact[l] = take<float>(net, lp * kL[l].cout, ok);
        }
        if (l >= 1 && l < kOut) {
            net->wf[l] = take<uint16_t>(net, (size_t)kL[l].cout * 9 * kL[l].cin, ok);
            net->wb[l] = take<uint16_t>(net, (size_t)kL[l].cout * 9 * kL[l].cin, ok);
        }
    }
    net->gbf = take<uint16_t>(net, pix * 16, ok);
    net->gin = take<float>(net, pix * 16, ok);
    net->xbf = take<uint16_t>(net, pix, ok);
    net->xh = take<float>(net, pix, ok);
    net->rms = take<float>(net, n_max, ok);
    net->cmean = take<float>(net, n_max, ok);
    const long long ns = kMaxSlices;
    long long pcount = ns * 9 * 64 * 64;
    if (17 * ((pix + kThreads - 1) / kThreads) > pcount) pcount = 17 * ((pix + kThreads - 1) / kThreads);
    net->part = take<float>(net, pcount, ok);
    net->partb = take<float>(net, ns * 64, ok);
    net->dpart = take<double>(net, (size_t)n_max * (kStatBlocks > kSampleBlocks ? kStatBlocks : kSampleBlocks), ok);
    net->loss = take<double>(net, 1, ok);
    net->status = take<int>(net, 1, ok);
    if (!ok) {
        gea_net_destroy(net);
        return GEA_ERR_NOMEM;
    }
    if (cudaMemset(net->theta, 0, net->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(net->m, 0, net->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(net->v, 0, net->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(net->status, 0, sizeof(int)) != cudaSuccess || pack_all(net) != GEA_OK ||
        cudaDeviceSynchronize() != cudaSuccess) {
        gea_net_destroy(net);
        return GEA_ERR_CUDA;
    }
    *out = net;
    return GEA_OK;
}

int gea_net_set_stream(gea_net *net, void *stream)
{
    if (!net) return GEA_ERR_INVAL;
    net->st = (cudaStream_t)stream;
    return GEA_OK;
}

int gea_net_set_params(gea_net *net, const float *theta, int32_t mem)
{
    if (!net || !theta || (mem != GEA_MEM_HOST && mem != GEA_MEM_DEVICE)) return GEA_ERR_INVAL;
    if (cudaMemcpyAsync(net->theta, theta, net->np * sizeof(float), cudaMemcpyDefault, net->st) != cudaSuccess ||
        cudaMemsetAsync(net->m, 0, net->np * sizeof(float), net->st) != cudaSuccess ||
        cudaMemsetAsync(net->v, 0, net->np * sizeof(float), net->st) != cudaSuccess)
        return GEA_ERR_CUDA;
    net->t = 0;
    int rc = pack_all(net);
    if (rc) return rc;
    return cudaStreamSynchronize(net->st) == cudaSuccess ? GEA_OK : GEA_ERR_CUDA;
}

int gea_net_get_params(gea_net *net, float *theta, int32_t mem)
{
    if (!net || !theta || (mem != GEA_MEM_HOST && mem != GEA_MEM_DEVICE)) return GEA_ERR_INVAL;
    if (cudaMemcpyAsync(theta, net->theta, net->np * sizeof(float), cudaMemcpyDefault, net->st) != cudaSuccess ||
        cudaStreamSynchronize(net->st) != cudaSuccess)
        return GEA_ERR_CUDA;
    return GEA_OK;
}

int gea_net_forward(gea_net *net, int32_t n, int32_t h, int32_t w, const float *r, float *y)
{
    if (!net || !r || !y || !shape_ok(net, n, h, w)) return GEA_ERR_INVAL;
    return forward(net, n, h, w, r, y);
}

int gea_net_energy(gea_net *net, const float *c, const float *ax, const float *az, float *dy, float *loss)
{
    if (!net || !c || !ax || !az || !dy) return GEA_ERR_INVAL;
    return energy(net, c, ax, az, dy, loss);
}

int gea_net_backward(gea_net *net, const float *dy, float *grad)
{
    if (!net || !dy || !grad) return GEA_ERR_INVAL;
    if (!net->have_fwd) return GEA_ERR_STATE;
    return backward(net, dy, grad);
}

int gea_net_adam(gea_net *net, const float *grad, float lr)
{
    if (!net || !grad || !(lr >= 0.0f)) return GEA_ERR_INVAL;
    return adam(net, grad, lr);
}

int gea_net_train_step(gea_net *net, int32_t n, int32_t h, int32_t w, const float *r, const float *c,
                       const float *ax, const float *az, float lr, float *loss)
{
    if (!net || !r || !c || !ax || !az || !shape_ok(net, n, h, w) || !(lr >= 0.0f)) return GEA_ERR_INVAL;
    // the network's own output buffer: the gradient buffer's first n h w values
    // are free until the backward pass (which reads dy, not y)
    float *y = net->gin;
    int rc = forward(net, n, h, w, r, y);
    if (!rc) rc = energy(net, c, ax, az, net->dy, loss);
    if (!rc) rc = backward(net, net->dy, net->grad);
    if (!rc) rc = adam(net, net->grad, lr);
    return rc;
}

void gea_net_destroy(gea_net *net)
{
    if (!net) return;
    if (net->st) cudaStreamSynchronize(net->st);
    else cudaDeviceSynchronize();
    for (void *p : net->allocs) cudaFree(p);
    delete net;
}

}  // extern "C"
