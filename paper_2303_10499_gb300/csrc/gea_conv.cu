// gea_conv.cu -- 3x3 convolutions of the learned pressure-correction network
// on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// A layer is an implicit GEMM: the output tile of one CTA is 128 consecutive
// pixels of one image row (M = 128) times all cout channels (N = cout); the
// reduction runs over the 9 taps times cin channels (K), 16 channels per
// tcgen05.mma. The CTA keeps the layer's weights in shared memory for its
// whole life (persistent CTAs walk the row tiles) and stages, per tile, the
// three input rows the tile's taps touch (130 pixels each, zero outside the
// image), with the fused pooling or prolongation of the layer's input done
// while loading.
//
// Both operands use the no-swizzle K-major canonical layout: 8 rows x 16 bytes
// core matrices with consecutive rows (pixels / output channels) 16 bytes
// apart, so that the 8-row groups are 128 bytes apart (SBO) and every row of
// the operand is a linear 16-byte stride. A tap (dy, dx) of the A operand is
// then the staged input rows shifted by dx pixels: the descriptor's start
// address moves by 16 dx bytes, no data is copied per tap. Channel groups of
// 8 are LBO bytes apart. The accumulator (128 lanes x cout FP32 columns)
// lives in tensor memory and is read back by the four warps (one 32-lane
// sub-partition each) for the bias, activation and bfloat16 store.
#include "../../include/gea.h"
#include "../../include/gea_net.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace gea_conv {

constexpr int kM = 128;                  // pixels per tile (MMA M)
constexpr int kNP = kM + 2;              // staged pixels per input row
constexpr int kThreads = 128;
constexpr int kGrpB = kNP * 16;          // bytes between channel groups of a staged row
constexpr unsigned kWaitLimit = 1u << 22;  // x >= 32 ns per try: > 0.1 s

// ---- PTX wrappers ----

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K-direction core
// matrix) and stride (8-row group) byte offsets, descriptor version 1, no
// swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 lanes; the wait is tied to
// the registers so that no use can move above it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// ---- bfloat16 helpers ----

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

__device__ __forceinline__ uint32_t pack_bf2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ void unpack8(const uint4 &v, float (&f)[8])
{
    f[0] = bf_lo(v.x); f[1] = bf_hi(v.x); f[2] = bf_lo(v.y); f[3] = bf_hi(v.y);
    f[4] = bf_lo(v.z); f[5] = bf_hi(v.z); f[6] = bf_lo(v.w); f[7] = bf_hi(v.w);
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8])
{
    return make_uint4(pack_bf2(f[0], f[1]), pack_bf2(f[2], f[3]), pack_bf2(f[4], f[5]), pack_bf2(f[6], f[7]));
}

__device__ __forceinline__ uint4 ld16(const uint16_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

struct ConvArgs {
    int n, h, w;
    const uint16_t *x0, *x1, *wt;
    const float *bias;
    void *y;
    int *status;
    int relu, out_f32;
    int ntiles, tiles_per_row;
};

// Stage the three input rows of tile (b, y, x0): element (row r, pixel p,
// channel c) at r * rowB + (c / 8) * kGrpB + p * 16 + (c % 8) * 2, image
// pixel x0 - 1 + p of row y - 1 + r.
template <int CIN, int MODE>
__device__ __forceinline__ void stage_input(uint8_t *sA, const ConvArgs &a, int b, int y, int x0)
{
    constexpr int G = CIN / 8;
    constexpr int rowB = G * kGrpB;
    for (int e = threadIdx.x; e < 3 * kNP * G; e += kThreads) {
        const int g = e % G;
        const int rest = e / G;
        const int p = rest % kNP, r = rest / kNP;
        const int yy = y + r - 1, xx = x0 + p - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (yy >= 0 && yy < a.h && xx >= 0 && xx < a.w) {
            if (MODE == GEA_CONV_PLAIN) {
                v = ld16(a.x0 + (((size_t)b * a.h + yy) * a.w + xx) * CIN + g * 8);
            } else if (MODE == GEA_CONV_POOL) {
                const size_t W2 = (size_t)2 * a.w;
                const uint16_t *s = a.x0 + (((size_t)b * 2 * a.h + 2 * yy) * W2 + 2 * xx) * CIN + g * 8;
                float f0[8], f1[8], f2[8], f3[8], o[8];
                unpack8(ld16(s), f0);
                unpack8(ld16(s + CIN), f1);
                unpack8(ld16(s + W2 * CIN), f2);
                unpack8(ld16(s + W2 * CIN + CIN), f3);
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = 0.25f * ((f0[j] + f1[j]) + (f2[j] + f3[j]));
                v = pack8(o);
            } else {
                const int hc = a.h / 2, wc = a.w / 2;
                float f0[8], f1[8], o[8];
                unpack8(ld16(a.x0 + (((size_t)b * a.h + yy) * a.w + xx) * CIN + g * 8), f0);
                unpack8(ld16(a.x1 + (((size_t)b * hc + yy / 2) * wc + xx / 2) * CIN + g * 8), f1);
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = f0[j] + f1[j];
                v = pack8(o);
            }
        }
        *reinterpret_cast<uint4 *>(sA + r * rowB + g * kGrpB + p * 16) = v;
    }
}

// NB: output channels per CTA (the CTAs of one tile row split cout when the
// full weight block would leave room for only one CTA per SM)
template <int CIN, int NB>
__host__ __device__ constexpr int smem_bytes()
{
    return 9 * CIN * NB * 2 + 3 * (CIN / 8) * kGrpB + 64;
}

template <int COUT>
__host__ __device__ constexpr uint32_t tmem_cols()
{
    return COUT < 32 ? 32u : (uint32_t)COUT;
}

template <int CIN, int COUT, int MODE, int NB>
__global__ void __launch_bounds__(kThreads) k_conv3x3(ConvArgs a)
{
    static_assert(CIN % 16 == 0 && NB % 16 == 0 && NB <= 256 && COUT % NB == 0, "channel counts");
    constexpr int G = CIN / 8;
    constexpr int rowB = G * kGrpB;
    constexpr uint32_t lboB = (NB / 8) * 128;   // between K-groups of the weight operand
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *sW = smem;
    uint8_t *sA = smem + 9 * CIN * NB * 2;
    const int ob = blockIdx.y * NB;               // this CTA's first output channel
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sA + 3 * rowB);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *okflag = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights of output channels ob .. ob + NB - 1: element (o, k = tap * CIN + c)
    // at (k / 8) * lboB + (o / 8) * 128 + (o % 8) * 16 + (k % 8) * 2
    for (int e = tid; e < NB * 9 * G; e += kThreads) {
        const int kg = e % (9 * G), o = e / (9 * G);
        const uint4 v = ld16(a.wt + (size_t)(ob + o) * 9 * CIN + kg * 8);
        *reinterpret_cast<uint4 *>(sW + kg * lboB + (o / 8) * 128 + (o % 8) * 16) = v;
    }
    if (tid == 0) mbar_init(smem_u32(mbar), 1);
    if (warp == 0) tmem_alloc(smem_u32(tslot), tmem_cols<NB>());
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = instr_desc(NB);

    uint32_t phase = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const int tx = t % a.tiles_per_row;
        const int row = t / a.tiles_per_row;
        const int y = row % a.h, b = row / a.h;
        const int x0 = tx * kM;
        stage_input<CIN, MODE>(sA, a, b, y, x0);
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t aBase = smem_u32(sA), bBase = smem_u32(sW);
            uint32_t acc = 0;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int r = tap / 3, dx = tap % 3 - 1;
#pragma unroll
                for (int kc = 0; kc < CIN / 16; ++kc) {
                    const uint64_t ad = smem_desc(aBase + r * rowB + (1 + dx) * 16 + 2 * kc * kGrpB, kGrpB, 128);
                    const uint64_t bd = smem_desc(bBase + (tap * G + 2 * kc) * lboB, lboB, 128);
                    mma_bf16(tmem, ad, bd, idesc, acc);
                    acc = 1;
                }
            }
            mma_commit(smem_u32(mbar));
            unsigned spins = 0;
            bool ok = true;
            while (!mbar_try_wait(smem_u32(mbar), phase)) {
                if (++spins > kWaitLimit) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
            if (!ok) {
                // gave up: the committed MMA batch may still be running and
                // reading sA/sW and writing TMEM, so wait for it once more
                // (bounded) before the CTA releases its TMEM columns and
                // shared memory. If that wait gives up too, nothing can
                // contain the batch: the status says so, and the caller must
                // treat the CUDA context as lost.
                unsigned drain = 0;
                while (!mbar_try_wait(smem_u32(mbar), phase) && ++drain <= kWaitLimit) __nanosleep(32);
                if (a.status) atomicExch(a.status, GEA_ERR_TIMEOUT);
            }
            *okflag = ok ? 1 : 0;
        }
        __syncthreads();
        tc_fence_after();
        if (!*okflag) break;
        phase ^= 1u;

        const int m = warp * 32 + lane;
        const int xx = x0 + m;
        const bool valid = xx < a.w;
        const size_t pix = ((size_t)b * a.h + y) * a.w + xx;
#pragma unroll
        for (int c0 = 0; c0 < NB; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (a.bias) v[j] += __ldg(&a.bias[ob + c0 + j]);
                if (a.relu) v[j] = fmaxf(v[j], 0.0f);
            }
            if (valid) {
                if (a.out_f32) {
                    float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(a.y) + pix * COUT + ob + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(a.y) + pix * COUT + ob + c0);
                    dst[0] = make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                                        pack_bf2(v[6], v[7]));
                    dst[1] = make_uint4(pack_bf2(v[8], v[9]), pack_bf2(v[10], v[11]), pack_bf2(v[12], v[13]),
                                        pack_bf2(v[14], v[15]));
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols<NB>());
}

template <int CIN, int COUT, int MODE>
cudaError_t launch_one(const ConvArgs &a0, cudaStream_t st)
{
    // 64 x 64 layers: two CTAs per tile row of 32 output channels each, so
    // that two CTAs fit on an SM
    constexpr int NB = (CIN >= 64 && COUT >= 64) ? COUT / 2 : COUT;
    constexpr int NOB = COUT / NB;
    constexpr int smem = smem_bytes<CIN, NB>();
    auto kern = k_conv3x3<CIN, COUT, MODE, NB>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int sms = 0, per_sm = 0;
    std::call_once(once, [&] {
        // resident CTAs per SM from the kernel's own limits: threads, shared
        // memory (with the carveout set to its maximum), registers and the
        // 512 tensor-memory columns of an SM
        attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                            (int)cudaSharedmemCarveoutMaxShared);
        int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0;
        cudaFuncAttributes fa{};
        if (attr_err == cudaSuccess) attr_err = cudaGetDevice(&dev);
        if (attr_err == cudaSuccess) attr_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (attr_err == cudaSuccess)
            attr_err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (attr_err == cudaSuccess)
            attr_err = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (attr_err == cudaSuccess)
            attr_err = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        if (attr_err == cudaSuccess) attr_err = cudaFuncGetAttributes(&fa, kern);
        if (attr_err != cudaSuccess) return;
        per_sm = thr_sm / kThreads;
        const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + 1024);
        const int by_regs = regs_sm / (kThreads * (fa.numRegs > 0 ? fa.numRegs : 1));
        const int by_tmem = 512 / (int)tmem_cols<NB>();
        per_sm = per_sm < by_smem ? per_sm : by_smem;
        per_sm = per_sm < by_regs ? per_sm : by_regs;
        per_sm = per_sm < by_tmem ? per_sm : by_tmem;
        if (per_sm < 1) per_sm = 1;
    });
    if (attr_err != cudaSuccess) return attr_err;
    ConvArgs a = a0;
    a.tiles_per_row = (a.w + kM - 1) / kM;
    a.ntiles = a.n * a.h * a.tiles_per_row;
    int gx = (sms * per_sm + NOB - 1) / NOB;
    if (gx > a.ntiles) gx = a.ntiles;
    kern<<<dim3(gx, NOB), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t launch_mode(const ConvArgs &a, int mode, cudaStream_t st)
{
    switch (mode) {
    case GEA_CONV_PLAIN: return launch_one<CIN, COUT, GEA_CONV_PLAIN>(a, st);
    case GEA_CONV_POOL: return launch_one<CIN, COUT, GEA_CONV_POOL>(a, st);
    default: return launch_one<CIN, COUT, GEA_CONV_UPADD>(a, st);
    }
}

template <int CIN>
cudaError_t launch_cout(const ConvArgs &a, int cout, int mode, cudaStream_t st)
{
    switch (cout) {
    case 16: return launch_mode<CIN, 16>(a, mode, st);
    case 32: return launch_mode<CIN, 32>(a, mode, st);
    default: return launch_mode<CIN, 64>(a, mode, st);
    }
}

}  // namespace gea_conv

using namespace gea_conv;

// Launch helper shared with the network code of this library.
cudaError_t gea_conv3x3_launch(int n, int h, int w, int cin, int cout, int mode, int flags, const uint16_t *x0,
                               const uint16_t *x1, const uint16_t *wt, const float *bias, void *y, int *status,
                               cudaStream_t st)
{
    ConvArgs a{};
    a.n = n; a.h = h; a.w = w;
    a.x0 = x0; a.x1 = x1; a.wt = wt; a.bias = bias; a.y = y; a.status = status;
    a.relu = (flags & GEA_CONV_RELU) != 0;
    a.out_f32 = (flags & GEA_CONV_OUT_F32) != 0;
    switch (cin) {
    case 16: return launch_cout<16>(a, cout, mode, st);
    case 32: return launch_cout<32>(a, cout, mode, st);
    default: return launch_cout<64>(a, cout, mode, st);
    }
}

extern "C" int gea_conv3x3(int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout, int32_t mode,
                           int32_t flags, const uint16_t *x0, const uint16_t *x1, const uint16_t *wt,
                           const float *bias, void *y, int32_t *status, void *stream)
{
    auto okc = [](int c) { return c == 16 || c == 32 || c == 64; };
    if (n < 1 || h < 1 || w < 1 || !okc(cin) || !okc(cout) || mode < 0 || mode > 2 ||
        (flags & ~(GEA_CONV_RELU | GEA_CONV_OUT_F32)) || !x0 || !wt || !y)
        return GEA_ERR_INVAL;
    if (mode == GEA_CONV_UPADD && (!x1 || h % 2 || w % 2)) return GEA_ERR_INVAL;
    if ((long long)n * h * w > (1LL << 31) / 64) return GEA_ERR_INVAL;
    cudaError_t e = gea_conv3x3_launch(n, h, w, cin, cout, mode, flags, x0, x1, wt, bias, y, status,
                                       (cudaStream_t)stream);
    return e == cudaSuccess ? GEA_OK : GEA_ERR_CUDA;
}
