// gea_conv.cu -- 3x3 convolutions of the learned pressure-correction network
// on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// A layer is an implicit GEMM: an output tile is 128 consecutive pixels of
// one image row (M = 128) times all cout channels (N = cout); the reduction
// runs over the 9 taps times cin channels (K), 16 channels per
// tcgen05.mma. A persistent CTA keeps the layer's weights in shared memory
// for its whole life and walks a contiguous range of tiles down the tile
// columns, so that consecutive tiles share two of their three input rows:
// a ring of four staged rows (130 pixels each, zero outside the image, the
// fused pooling or prolongation of the layer's input done while loading)
// takes one new row per tile, copied while the previous tile's MMA batch
// runs, and two accumulator buffers in tensor memory let the store of one
// tile overlap the batch of the next.
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
// threads of a CTA: 128 (one warp per 32-lane sub-partition of tensor
// memory), or 256 (two, splitting the channels) for the 64-channel layers,
// whose rows and epilogues are four times larger
template <int CIN, int COUT>
__host__ __device__ constexpr int threads_of()
{
    return (CIN == 64 || COUT == 64) ? 256 : 128;
}
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

// 16 consecutive FP32 columns of this warp's 32 lanes, without waiting.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Wait for this thread's tensor-memory loads; the wait is tied to the
// registers of one load so that no use of them can move above it (a second
// call for another load's registers returns at once).
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
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

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
// and reads nothing.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Input rows are copied kDist tiles ahead of their first use. The ring
// holds the rows of the batch in flight for the previous tile (y - 2 .. y),
// of the current tile (y - 1 .. y + 1) and the ones in flight (y + 2 ..
// y + 1 + kDist): 4 + kDist slots; a new row takes the slot of row y - 3,
// whose last reader, the batch of tile y - 2, has completed.
constexpr int kDist = 2;
constexpr int kRing = 4 + kDist;
constexpr int kSide = kDist + 1;   // prolongation mode: coarse values of the rows not yet added

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n of this thread's most recent groups are pending
__device__ __forceinline__ void cp_async_wait(int n)
{
    if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 2;" ::: "memory");
}

// Stage image row yy (zeros outside the image) of the tile column starting
// at pixel x0 into a ring slot: element (pixel p, channel c) at
// (c / 8) * kGrpB + p * 16 + (c % 8) * 2 holds image pixel x0 - 1 + p.
// Plain inputs are copied asynchronously; in the prolongation mode the
// fine values go to the slot and the coarse value of each fine pixel to the
// same place of a side slot, both asynchronously, and finish_row adds them;
// pooled inputs are averaged in registers and stored. Every thread handles
// the same chunks of every row, so a thread's own wait covers what it
// finishes.
template <int CIN, int MODE, int NT>
__device__ __forceinline__ void stage_row(uint8_t *slot, uint8_t *side, const ConvArgs &a, int b, int yy, int x0)
{
    constexpr int G = CIN / 8;
    const bool row_in = yy >= 0 && yy < a.h;
    for (int e = threadIdx.x; e < kNP * G; e += NT) {
        const int g = e % G, p = e / G;
        const int xx = x0 + p - 1;
        const bool in = row_in && xx >= 0 && xx < a.w;
        const int off = g * kGrpB + p * 16;
        if (MODE == GEA_CONV_PLAIN || MODE == GEA_CONV_UPADD) {
            const uint16_t *src = in ? a.x0 + (((size_t)b * a.h + yy) * a.w + xx) * CIN + g * 8 : a.x0;
            cp_async16(smem_u32(slot + off), src, in ? 16u : 0u);
            if (MODE == GEA_CONV_UPADD) {
                const int hc = a.h / 2, wc = a.w / 2;
                const uint16_t *s1 = in ? a.x1 + (((size_t)b * hc + yy / 2) * wc + xx / 2) * CIN + g * 8 : a.x1;
                cp_async16(smem_u32(side + off), s1, in ? 16u : 0u);
            }
        } else {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (in) {
                const size_t W2 = (size_t)2 * a.w;
                const uint16_t *s0 = a.x0 + (((size_t)b * 2 * a.h + 2 * yy) * W2 + 2 * xx) * CIN + g * 8;
                float f0[8], f1[8], f2[8], f3[8], o[8];
                unpack8(ld16(s0), f0);
                unpack8(ld16(s0 + CIN), f1);
                unpack8(ld16(s0 + W2 * CIN), f2);
                unpack8(ld16(s0 + W2 * CIN + CIN), f3);
#pragma unroll
                for (int j = 0; j < 8; ++j) o[j] = 0.25f * ((f0[j] + f1[j]) + (f2[j] + f3[j]));
                v = pack8(o);
            }
            *reinterpret_cast<uint4 *>(slot + off) = v;
        }
    }
}

// Prolongation mode: slot += side, in FP32 rounded to bfloat16 (this
// thread's chunks, after its wait for the row's copies).
template <int CIN, int MODE, int NT>
__device__ __forceinline__ void finish_row(uint8_t *slot, const uint8_t *side)
{
    if (MODE != GEA_CONV_UPADD) return;
    constexpr int G = CIN / 8;
    for (int e = threadIdx.x; e < kNP * G; e += NT) {
        const int off = (e % G) * kGrpB + (e / G) * 16;
        float f0[8], f1[8], o[8];
        unpack8(*reinterpret_cast<const uint4 *>(slot + off), f0);
        unpack8(*reinterpret_cast<const uint4 *>(side + off), f1);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = f0[j] + f1[j];
        *reinterpret_cast<uint4 *>(slot + off) = pack8(o);
    }
}

// Tensor-memory columns of one accumulator buffer (allocation granule 32)
template <int COUT>
__host__ __device__ constexpr uint32_t tmem_buf_cols()
{
    return COUT < 32 ? 32u : (uint32_t)COUT;
}

// weights, the ring of input rows (and the side slots of the prolongation
// mode), the bias, two mbarriers, the TMEM slot and the wait flag
template <int CIN, int COUT, int MODE>
__host__ __device__ constexpr int smem_bytes()
{
    return 9 * CIN * COUT * 2 + (kRing + (MODE == GEA_CONV_UPADD ? kSide : 0)) * (CIN / 8) * kGrpB + COUT * 4 + 64;
}

// A CTA takes a contiguous range of tiles in (image, tile column, row)
// order, the row fastest, so that consecutive tiles of a column share two
// of their three input rows: a tile needs one new row, copied kDist tiles
// ahead. The CTA's warps have two roles. One extra warp issues the MMA
// batches (one thread); the other NT threads copy rows and, from the second
// of two accumulator buffers in tensor memory, apply the bias and activation
// and store the previous tile, while the batch runs:
//   loaders: wait for and finish the new row of tile i | barrier | copy the
//   row of tile i + kDist | wait for batch i-1 (mbarrier), store tile i-1
//   MMA warp: barrier | issue batch i into buffer i&1, commit to its mbarrier
// The first tile of a column run stages its three rows (and the next kDist
// - 1 rows) once the batch of the tile before it has completed. A wait that
// runs out (bounded polls) sets a flag that every thread reads after the
// next barrier, and the CTA leaves the loop.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(threads_of<CIN, COUT>() + 32) k_conv3x3(ConvArgs a)
{
    constexpr int NT = threads_of<CIN, COUT>();   // loaders (and epilogue)
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 256, "channel counts");
    constexpr int G = CIN / 8;
    constexpr int rowB = G * kGrpB;
    constexpr uint32_t lboB = (COUT / 8) * 128;   // between K-groups of the weight operand
    constexpr uint32_t bufC = tmem_buf_cols<COUT>();
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *sW = smem;
    uint8_t *sR = smem + 9 * CIN * COUT * 2;
    uint8_t *sX = sR + kRing * rowB;   // side slots (prolongation mode)
    float *sBias = reinterpret_cast<float *>(sX + (MODE == GEA_CONV_UPADD ? kSide : 0) * rowB);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sBias + COUT);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    int *sfail = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool loader = tid < NT;

    // weights: element (o, k = tap * CIN + c) at
    // (k / 8) * lboB + (o / 8) * 128 + (o % 8) * 16 + (k % 8) * 2
    for (int e = tid; e < COUT * 9 * G; e += NT + 32) {
        const int kg = e % (9 * G), o = e / (9 * G);
        const uint4 v = ld16(a.wt + (size_t)o * 9 * CIN + kg * 8);
        *reinterpret_cast<uint4 *>(sW + kg * lboB + (o / 8) * 128 + (o % 8) * 16) = v;
    }
    for (int o = tid; o < COUT; o += NT + 32) sBias[o] = a.bias ? __ldg(&a.bias[o]) : 0.0f;
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        *sfail = 0;
    }
    if (warp == 0) tmem_alloc(smem_u32(tslot), 2 * bufC);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = instr_desc(COUT);
    auto slot = [&](int yy) { return sR + ((yy + 1) % kRing) * rowB; };
    auto side = [&](int yy) { return sX + ((yy + 1) % kSide) * rowB; };

    // phase bits and outstanding batches of the two buffers (the loaders
    // track them; thread 0's copy drains the batches after a failed wait)
    uint32_t phase = 0, pending = 0;
    // a loader's bounded wait for buffer j's batch
    auto wait_batch = [&](int j) -> bool {
        const uint32_t mb = smem_u32(&mbar[j]);
        const uint32_t ph = (phase >> j) & 1u;
        unsigned spins = 0;
        while (!mbar_try_wait(mb, ph)) {
            if (++spins > kWaitLimit) {
                *sfail = 1;
                return false;
            }
            __nanosleep(32);
        }
        tc_fence_after();
        return true;
    };
    // bias, activation and store of the tile (b, y, x0) held in buffer j:
    // warp w reads the lanes (pixels) of sub-partition w % 4; with 256
    // loaders warps w and w + 4 split the channels. A thread's columns (16
    // or 32) are loaded before one wait
    auto epilogue = [&](int j, int b, int y, int x0) {
        constexpr int CH = (NT == 256 && COUT >= 32) ? COUT / 2 : COUT;   // channels per warp
        constexpr int NL = CH / 16;                                         // 16-column loads per thread
        static_assert(NL >= 1 && NL <= 2, "one or two tensor-memory loads per thread");
        const int half = warp >> 2;
        if (half * CH >= COUT) return;
        const int m = (warp & 3) * 32 + lane;
        const int xx = x0 + m;
        const bool valid = xx < a.w;
        const size_t pix = ((size_t)b * a.h + y) * a.w + xx;
        const int cb = half * CH;
        uint32_t r[2][16];
#pragma unroll
        for (int l = 0; l < NL; ++l)
            tmem_ld16_issue(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)j * bufC + (uint32_t)(cb + 16 * l),
                            r[l]);
#pragma unroll
        for (int l = 0; l < NL; ++l) tmem_ld_wait(r[l]);
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const int c0 = cb + 16 * l;
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                v[q] = __uint_as_float(r[l][q]) + sBias[c0 + q];
                if (a.relu) v[q] = fmaxf(v[q], 0.0f);
            }
            if (valid) {
                if (a.out_f32) {
                    float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(a.y) + pix * COUT + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(a.y) + pix * COUT + c0);
                    dst[0] = make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                                        pack_bf2(v[6], v[7]));
                    dst[1] = make_uint4(pack_bf2(v[8], v[9]), pack_bf2(v[10], v[11]), pack_bf2(v[12], v[13]),
                                        pack_bf2(v[14], v[15]));
                }
            }
        }
    };

    const long long T = (long long)a.n * a.tiles_per_row * a.h;
    const long long t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;
    // the copy of row yy (one commit group), and whether the tile k rows
    // below tile t (row y) belongs to the same column run of this CTA
    auto issue = [&](int yy, int b, int x0) {
        stage_row<CIN, MODE, NT>(slot(yy), side(yy), a, b, yy, x0);
        cp_async_commit();
    };
    auto in_run = [&](long long t, int y, int k) { return y + k < a.h && t + k < t1; };
    // tile coordinates, advanced without divisions
    int y = (int)(t0 % a.h);
    int col = (int)(t0 / a.h);
    int pb = 0, py = 0, px0 = 0;   // the previous tile
    for (long long t = t0; t < t1; ++t) {
        const int i = (int)(t - t0);
        if (i > 0 && ++y == a.h) {
            y = 0;
            ++col;
        }
        const int x0 = (col % a.tiles_per_row) * kM, b = col / a.tiles_per_row;
        const int j = i & 1;
        if (loader) {
            if (i == 0 || y == 0) {
                // first tile of a column run: its three rows, once the
                // previous tile's batch no longer reads the ring, then the
                // rows of the next kDist - 1 tiles
                if (i == 0 || wait_batch(j ^ 1)) {
                    for (int r = 0; r < 3; ++r) issue(y - 1 + r, b, x0);
                    cp_async_wait(0);
                    for (int r = 0; r < 3; ++r) finish_row<CIN, MODE, NT>(slot(y - 1 + r), side(y - 1 + r));
                    for (int k = 1; k < kDist; ++k)
                        if (in_run(t, y, k)) issue(y + 1 + k, b, x0);
                }
            } else {
                // row y + 1: the groups issued after it are those of the
                // rows of tiles t + 1 .. t + kDist - 1 of the run
                int newer = 0;
                for (int k = 1; k < kDist; ++k) newer += in_run(t, y, k) ? 1 : 0;
                cp_async_wait(newer);
                finish_row<CIN, MODE, NT>(slot(y + 1), side(y + 1));
            }
            fence_proxy_async();
        }
        tc_fence_before();
        __syncthreads();
        if (*sfail) break;
        if (warp == NT / 32) {
            if (lane == 0) {
                tc_fence_after();
                // the descriptors differ only in their start address field
                // (address / 16, below 2^14 in the shared window), so each
                // is a base descriptor plus a constant
                const uint64_t bD = smem_desc(smem_u32(sW), lboB, 128);
                const uint64_t aD[3] = {smem_desc(smem_u32(slot(y - 1)), kGrpB, 128),
                                        smem_desc(smem_u32(slot(y)), kGrpB, 128),
                                        smem_desc(smem_u32(slot(y + 1)), kGrpB, 128)};
                uint32_t acc = 0;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int r = tap / 3, dx = tap % 3 - 1;
#pragma unroll
                    for (int kc = 0; kc < CIN / 16; ++kc) {
                        const uint64_t ad = aD[r] + (uint64_t)(((1 + dx) * 16 + 2 * kc * kGrpB) >> 4);
                        const uint64_t bd = bD + (uint64_t)(((tap * G + 2 * kc) * lboB) >> 4);
                        mma_bf16(tmem + (uint32_t)j * bufC, ad, bd, idesc, acc);
                        acc = 1;
                    }
                }
                mma_commit(smem_u32(&mbar[j]));
            }
            __syncwarp();
        } else {
            pending |= 1u << j;
            // the row of tile t + kDist, into the slot of row y - 3 (read
            // last by the batch of tile t - 2, which has completed), while
            // the batch runs
            if (in_run(t, y, kDist)) issue(y + 1 + kDist, b, x0);
            if (i > 0) {
                const int jp = j ^ 1;
                if (wait_batch(jp)) {
                    epilogue(jp, pb, py, px0);
                    phase ^= 1u << jp;
                    pending &= ~(1u << jp);
                }
            }
            tc_fence_before();
        }
        pb = b;
        py = y;
        px0 = x0;
    }
    // the last tile
    if (loader && !*sfail && t1 > t0) {
        const int jl = (int)((t1 - 1 - t0) & 1);
        if (wait_batch(jl)) {
            epilogue(jl, pb, py, px0);
            phase ^= 1u << jl;
            pending &= ~(1u << jl);
        }
        tc_fence_before();
    }
    cp_async_wait(0);
    __syncthreads();
    if (*sfail && tid == 0) {
        // a wait ran out: the committed batches may still be running and
        // reading shared memory and writing tensor memory, so wait once more,
        // bounded, for every batch still outstanding before the CTA frees
        // them. If that also runs out nothing can contain the batches: the
        // status says so, and the caller must treat the CUDA context as lost.
        for (int q = 0; q < 2; ++q) {
            if (!((pending >> q) & 1u)) continue;
            unsigned drain = 0;
            while (!mbar_try_wait(smem_u32(&mbar[q]), (phase >> q) & 1u) && ++drain <= kWaitLimit) __nanosleep(32);
        }
        if (a.status) atomicExch(a.status, GEA_ERR_TIMEOUT);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 2 * bufC);
}

template <int CIN, int COUT, int MODE>
cudaError_t launch_one(const ConvArgs &a0, cudaStream_t st)
{
    constexpr int smem = smem_bytes<CIN, COUT, MODE>();
    auto kern = k_conv3x3<CIN, COUT, MODE>;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int sms = 0, per_sm = 0;
    std::call_once(once, [&] {
        // resident CTAs per SM from the kernel's own limits: threads, shared
        // memory (with the carveout set to its maximum), registers and the
        // 512 tensor-memory columns of an SM (two buffers a CTA)
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
        constexpr int NT = threads_of<CIN, COUT>() + 32;
        per_sm = thr_sm / NT;
        const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + 1024);
        const int by_regs = regs_sm / (NT * (fa.numRegs > 0 ? fa.numRegs : 1));
        const int by_tmem = 512 / (int)(2 * tmem_buf_cols<COUT>());
        per_sm = per_sm < by_smem ? per_sm : by_smem;
        per_sm = per_sm < by_regs ? per_sm : by_regs;
        per_sm = per_sm < by_tmem ? per_sm : by_tmem;
        if (per_sm < 1) per_sm = 1;
    });
    if (attr_err != cudaSuccess) return attr_err;
    ConvArgs a = a0;
    a.tiles_per_row = (a.w + kM - 1) / kM;
    a.ntiles = a.n * a.h * a.tiles_per_row;
    int gx = sms * per_sm;
    if (gx > a.ntiles) gx = a.ntiles;
    kern<<<gx, threads_of<CIN, COUT>() + 32, smem, st>>>(a);
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
