// cnn.cu -- the learned warm start: a stack of 3 x 3 convolutions on BF16
// tensor cores (tcgen05.mma, FP32 accumulate in tensor memory), its backward
// pass (weight gradients on mma.sync m16n8k16) and Adam. Not part of the paper; Theorem 1 (convergence from any u0, d0) is
// what lets a predicted start feed Algorithm 2.
//
// Layout. Activations and their gradients are BF16 in planes of eight
// channels: [image][C / 8][H][W][8], C padded to 8 (the network's input),
// 16 or 32. One plane row is
// W x 16 contiguous bytes, so a halo tile of a plane is a few long row
// segments (one TMA box of 160-byte rows for the tensor-core layers), and a
// pixel's eight channels are the 16-byte K slice the MMAs consume. The
// network's 4-channel output is FP32 [image][H][W][4]. Packed weights are
// BF16 [tap][cout][cin] (cin contiguous), the order in which the B operand of
// the MMA consumes them.
//
// Every convolution of the forward pass and every input gradient runs on
// tcgen05 (conv3x3_tc below): the 32-channel layers with bias and ReLU, the
// input gradients gated by the ReLU of the layer below, and the last layer
// (4 outputs padded to 16) with bias into FP32.
//
// Weight-gradient kernel: per tap, dW_tap = G^T A_tap, a contraction over
// pixels. A CTA of 9 warps (one per tap) loops over tiles; the gradient and
// activation tiles are stored channel-major in shared memory so the MMA
// operands are pixel pairs of one channel; the CTA's FP32 partial sums go to
// global memory with one atomic add per element at the end.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/admm_warmstart.h"

namespace admm {
bool alloc_fault_fire();   // ADMM_OPT_FAIL_ALLOC (engine.cu)
}

namespace {

using bf16 = __nv_bfloat16;

constexpr int kLayers = ADMM_CNN_LAYERS;
constexpr int kWidth = ADMM_CNN_WIDTH;
constexpr int kIn = 2, kOut = 4;
constexpr int kTile = 16;

// real (cout, cin) and padded channel counts of layer l
__host__ __device__ constexpr int layer_cin(int l) { return l == 0 ? kIn : kWidth; }
__host__ __device__ constexpr int layer_cout(int l) { return l == kLayers - 1 ? kOut : kWidth; }
constexpr int pad16(int c) { return c <= 16 ? 16 : 32; }
// the first layer's 2 input channels fill one plane of eight
constexpr int layer_cinp(int l) { return l == 0 ? 8 : pad16(layer_cin(l)); }
constexpr int layer_coutp(int l) { return l == kLayers - 1 ? 16 : kWidth; }

long long param_offset(int l) {
    long long o = 0;
    for (int j = 0; j < l; ++j) o += (long long)layer_cout(j) * layer_cin(j) * 9 + layer_cout(j);
    return o;
}
long long param_count() { return param_offset(kLayers); }

std::mutex g_cnn_mutex;
long long g_cnn_launches = 0;

int fail(cudaError_t) { return ADMM_ECUDA; }
#define CKC(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return fail(e_);    \
    } while (0)

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// network input: [M^T y, mask] in channels 0 and 1 of one plane of eight
// ---------------------------------------------------------------------------
__global__ void cnn_input_kernel(const float* __restrict__ ybar, const uint8_t* __restrict__ mask,
                                 bf16* __restrict__ a0, long long npx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    const bool obs = mask[i] != 0;
    const float y = obs ? ybar[i] : 0.f;
    reinterpret_cast<uint4*>(a0)[i] =
        make_uint4(pack2(__float2bfloat16(y), __float2bfloat16(obs ? 1.f : 0.f)), 0u, 0u, 0u);
}

enum { kModeReluBf16 = 0, kModeOutF32 = 1, kModeGateBf16 = 2 };   // epilogues of conv3x3_tc

// ---------------------------------------------------------------------------
// 3 x 3 convolution on the fifth-generation tensor cores (tcgen05.mma,
// accumulator in tensor memory).
//
// A CTA of four warps walks output tiles of 8 x 16 pixels (M = 128, one
// accumulator row per pixel: tile row oy, column ox at M row 8 oy + ox), N =
// COUT output channels (32, or 16 for the last layer's 4 outputs), K = 9 taps
// x CIN input channels. Operands sit in shared
// memory in the no-swizzle K-major layout of 8-row x 16-byte core matrices:
//   A: the 10 x 18 halo tile as [CIN/8][180 halo pixels][8 channels]; the A
//      matrix of tap (dy, dx) starts at halo pixel 10 dy + dx, its 8-row
//      groups (one tile row each) are 10 pixels = 160 B apart and its K
//      chunks 180 x 16 B apart, so no im2col copy is needed;
//   B: the weights as [tap][CIN/8][COUT output channels][8].
// With one plane of input channels (CIN = 8, the first layer) the taps go in
// pairs, one per K = 16 MMA: the A descriptor's K-chunk offset is then the
// pixel distance from the pair's first tap to its second (5 MMAs per tile,
// the ninth tap paired with a zero weight slot).
// The halo tile arrives by one TMA copy (cp.async.bulk.tensor, a 4-D view of
// the eight-channel planes whose innermost dimension merges a plane row's
// columns and channels, so each box row is 10 pixels x 16 B = 160 contiguous
// bytes and the box lands in shared memory already in the A layout; rows and
// columns outside the image read as zero), double-buffered. One thread issues
// the 9 x CIN/16 MMAs of a tile (K = 16 each; 5 for CIN = 8) and commits them
// to an mbarrier; the four warps wait (bounded), read their 32 lanes of the
// accumulator (tcgen05.ld) and apply bias + ReLU (forward) or the ReLU gate of
// the layer below (input gradient), storing four BF16 planes, or bias alone
// into the network's FP32 output (last layer).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets >> 4, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: F32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n (a multiple of 16)
__host__ __device__ constexpr uint32_t idesc_m128(uint32_t n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ unsigned long long gtimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for phase `parity` of the mbarrier, at most about a second; try_wait
// suspends the thread in hardware until the phase completes or a short
// hardware time limit passes, so the loop does not spin
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = gtimer_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (gtimer_ns() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's accumulator lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's accumulator lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kTcTW = 8, kTcTH = 16;                 // output tile (M = 128)
constexpr int kTcHW = kTcTW + 2, kTcHH = kTcTH + 2;  // halo tile
constexpr int kTcNP = kTcHW * kTcHH;                 // 180 halo pixels

// tin: TMA view of the input [img][CIN / 8][H][W][8] (see conv_tc); wpk:
// [9][COUT][CIN]; MODE kModeReluBf16 (bias, ReLU; out bf16 [img][4][H][W][8]),
// kModeGateBf16 (gate and out bf16 [img][4][H][W][8]) or kModeOutF32 (bias of
// the 4 outputs; out float [img][H][W][4]); err: set to 1 if a wait ran out (the CTA then stops,
// after a bounded wait for its own copies and MMAs still in flight).
//
// Pipeline of the CTA's i-th tile (halo buffer and accumulator i & 1): thread
// 0 waits for the halo of tile i + 1 and issues its MMAs into the other
// accumulator; all four warps then wait for tile i's MMAs, thread 0 starts the
// copy of tile i + 2's halo into the buffer they have finished reading, and
// the warps read tile i's accumulator and store it while the tensor cores work
// on tile i + 1.
template <int CIN, int MODE>
__global__ void __launch_bounds__(128)
conv3x3_tc(const __grid_constant__ CUtensorMap tin, const bf16* __restrict__ wpk, const float* __restrict__ bias,
           void* __restrict__ out, const bf16* __restrict__ gate, int H, int W, int count, int* __restrict__ err) {
    constexpr int COUT = MODE == kModeOutF32 ? 16 : 32, CH = CIN / 8;
    constexpr int BOXBYTES = CH * kTcNP * 16;                  // one halo box
    constexpr int ABYTES = (BOXBYTES + 127) / 128 * 128;        // (each halo buffer on a 128-byte boundary)
    constexpr uint32_t kTmemCols = 2 * COUT;   // two accumulators
    // weight slots: the 9 taps, or with one plane of input channels (CIN = 8)
    // taps 0..7, a zero slot and tap 8, so that the MMAs take the taps in
    // pairs (0,1) (2,3) (4,5) (6,7) (zero,8), one per K = 16
    constexpr int NSLOT = CIN == 8 ? 10 : 9;
    static_assert(CIN == 8 || CIN == 16 || CIN == 32, "input channels");
    __shared__ __align__(128) unsigned char smA[2][ABYTES];
    __shared__ __align__(128) unsigned char smW[NSLOT * CH * COUT * 16];
    __shared__ float smB[32];
    // 0, 1: halo of buffer 0 / 1 landed; 2, 3: MMAs into accumulator 0 / 1 done
    __shared__ __align__(8) unsigned long long bars[4];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < NSLOT * COUT * CH; e += 128) {
        const int sc = e / CH, k = e - sc * CH;       // sc = slot * COUT + output channel
        const int slot = sc / COUT, co = sc - slot * COUT;
        const int tap = CIN == 8 ? (slot < 8 ? slot : (slot == 9 ? 8 : -1)) : slot;
        unsigned char* dst = smW + ((slot * CH + k) * COUT + co) * 16;
        if (tap >= 0)
            cp_async16(dst, wpk + ((size_t)tap * COUT + co) * CIN + k * 8);
        else
            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    if ((MODE == kModeReluBf16 && tid < COUT) || (MODE == kModeOutF32 && tid < kOut)) smB[tid] = bias[tid];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sh_addr(&tmem_base)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const int tiles_x = W / kTcTW, per_img = tiles_x * (H / kTcTH);
    const int ntiles = per_img * count, G = gridDim.x;
    const uint64_t tmap = reinterpret_cast<uint64_t>(&tin);
    // phase bits (bit b: barrier of buffer / accumulator b) and, in thread 0,
    // the copies and MMA groups issued but not yet seen complete
    uint32_t hph = 0, mph = 0, pend_h = 0, pend_m = 0;
    // one TMA copy of tile t's halo into buffer b (thread 0)
    auto issue = [&](int t, int b) {
        const int img = t / per_img, rem = t - img * per_img;
        const int y0 = (rem / tiles_x) * kTcTH, x0 = (rem % tiles_x) * kTcTW;
        const uint32_t bar = sh_addr(&bars[b]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(BOXBYTES) : "memory");
        // x: element (column x0 - 1, channel 0) of the merged row, a multiple of 8
        // elements (16 B); column -1 and columns past W - 1 read as zero
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
            "%5}], [%6];" ::"r"(sh_addr(smA[b])),
            "l"(tmap), "r"((x0 - 1) * 8), "r"(y0 - 1), "r"(0), "r"(img), "r"(bar)
            : "memory");
        pend_h |= 1u << b;
    };
    if (tid == 0) {
        for (int i = 0; i < 4; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_addr(&bars[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if ((int)blockIdx.x + G < ntiles) issue(blockIdx.x + G, 1);
    }
    cp_async_wait_all();
    fence_async_shared();        // the weights (generic proxy) are visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t wBase = sh_addr(smW);
    // thread 0: wait for the halo in buffer b, then issue the tile's MMAs into
    // accumulator b (columns COUT b) and commit them to bars[2 + b]
    auto mma_tile = [&](int b) -> bool {
        if (!mbar_wait_bounded(sh_addr(&bars[b]), (hph >> b) & 1u)) return false;
        hph ^= 1u << b;
        pend_h &= ~(1u << b);
        tc_fence_after();
        const uint32_t aBase = sh_addr(smA[b]), d = tmem + (uint32_t)COUT * b;
        if constexpr (CIN == 8) {
            // K chunk 0 of pair j is tap a (or the zero slot), chunk 1 tap b: the
            // A descriptor starts at tap a's halo pixel and steps to tap b's by
            // its K-chunk offset (halo pixel of a tap (dy, dx): 10 dy + dx)
            constexpr int pa[5] = {0, 2, 11, 20, 21};   // chunk 0: taps 0, 2, 4, 6; any pixel for the zero slot
            constexpr int pd[5] = {1, 8, 1, 1, 1};      // chunk 1: taps 1, 3, 5, 7, 8
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const uint64_t a = umma_desc(aBase + pa[j] * 16, pd[j] * 16, kTcHW * 16);
                const uint64_t bd = umma_desc(wBase + 2 * j * COUT * 16, COUT * 16, 8 * 16);
                umma_f16(d, a, bd, idesc_m128(COUT), j != 0 ? 1u : 0u);
            }
        } else {
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap - 3 * (tap / 3);
#pragma unroll
                for (int j = 0; j < CH / 2; ++j) {
                    const uint64_t a =
                        umma_desc(aBase + (2 * j * kTcNP + dy * kTcHW + dx) * 16, kTcNP * 16, kTcHW * 16);
                    const uint64_t bd = umma_desc(wBase + (tap * CH + 2 * j) * COUT * 16, COUT * 16, 8 * 16);
                    umma_f16(d, a, bd, idesc_m128(COUT), (tap | j) != 0 ? 1u : 0u);
                }
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         sh_addr(&bars[2 + b]))
                     : "memory");
        pend_m |= 1u << b;
        return true;
    };
    bool ok = true;
    if (tid == 0 && (int)blockIdx.x < ntiles) ok = mma_tile(0);
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, ++it) {
        const int b = it & 1;
        // accumulator b ^ 1 was last read by the previous tile's epilogue,
        // which ended at the block barrier below
        if (tid == 0 && ok && tile + G < ntiles) ok = mma_tile(b ^ 1);
        const bool got = mbar_wait_bounded(sh_addr(&bars[2 + b]), (mph >> b) & 1u);
        if (got) {
            mph ^= 1u << b;
            pend_m &= ~(1u << b);
        }
        ok = __syncthreads_and(got && ok) != 0;
        if (!ok) break;
        // tile's MMAs are complete, so its halo buffer is free
        if (tid == 0 && tile + 2 * G < ntiles) issue(tile + 2 * G, b);
        tc_fence_after();
        const int img = tile / per_img, rem = tile - img * per_img;
        const int y0 = (rem / tiles_x) * kTcTH, x0 = (rem % tiles_x) * kTcTW;
        const int oy = 4 * warp + (lane >> 3), ox = lane & 7;
        const size_t hw = (size_t)H * W;
        const uint32_t tacc = tmem + (uint32_t)COUT * b + ((uint32_t)(32 * warp) << 16);
        if constexpr (MODE == kModeOutF32) {
            float v[16];
            tmem_ld16(tacc, v);
            const size_t px = (size_t)img * hw + (size_t)(y0 + oy) * W + (x0 + ox);
            reinterpret_cast<float4*>(out)[px] =
                make_float4(v[0] + smB[0], v[1] + smB[1], v[2] + smB[2], v[3] + smB[3]);
        } else {
            float v[32];
            tmem_ld32(tacc, v);
            // pixel's slot in plane 0 of its image; plane q is q hw slots further
            const size_t px = (size_t)img * 4 * hw + (size_t)(y0 + oy) * W + (x0 + ox);
            uint32_t pk[16];
            if (MODE == kModeReluBf16) {
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    pk[c] = pack2(__float2bfloat16(fmaxf(v[2 * c] + smB[2 * c], 0.f)),
                                  __float2bfloat16(fmaxf(v[2 * c + 1] + smB[2 * c + 1], 0.f)));
            } else {
                const uint4* gp = reinterpret_cast<const uint4*>(gate) + px;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 gv = gp[q * hw];
                    const uint32_t gw[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int c = 8 * q + 2 * h;
                        const float g0 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(gw[h] & 0xFFFFu)));
                        const float g1 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(gw[h] >> 16)));
                        pk[4 * q + h] = pack2(__float2bfloat16(g0 > 0.f ? v[c] : 0.f),
                                              __float2bfloat16(g1 > 0.f ? v[c + 1] : 0.f));
                    }
                }
            }
            uint4* op = reinterpret_cast<uint4*>(out) + px;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                op[q * hw] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        }
        tc_fence_before();
        __syncthreads();             // accumulator b is free for tile + 2 G's MMAs
    }
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        // let this CTA's own copies and MMAs still in flight finish (bounded)
        // before its tensor memory is released
        for (int b = 0; b < 2; ++b) {
            if (pend_h & (1u << b)) mbar_wait_bounded(sh_addr(&bars[b]), (hph >> b) & 1u);
            if (pend_m & (1u << b)) mbar_wait_bounded(sh_addr(&bars[2 + b]), (mph >> b) & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// weight and bias gradients of one layer
// a: [img][H][W][CIN] (layer input), g: [img][H][W][COUT] (gradient in the
// layer's pre-activation output). dw: FP32 [cout_real][cin_real][9] slice of
// the gradient vector, db: [cout_real].
// ---------------------------------------------------------------------------
template <int CIN, int COUT>
struct WgradCfg {
    static constexpr int HALO = kTile + 2;
    static constexpr int PA = HALO * HALO + 4;       // activation plane stride (elements)
    static constexpr int PG = kTile * kTile + 8;     // gradient plane stride
    static constexpr size_t SMEM = (size_t)(CIN * PA + COUT * PG) * sizeof(bf16) + COUT * sizeof(float);
    static_assert(SMEM <= 48 * 1024, "fits the default shared-memory window");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(288)
conv3x3_wgrad_kernel(const bf16* __restrict__ a, const bf16* __restrict__ gr, float* __restrict__ dw,
                     float* __restrict__ db, int cin_real, int cout_real, int H, int W, int images) {
    using C = WgradCfg<CIN, COUT>;
    extern __shared__ __align__(16) bf16 sm[];
    bf16* sA = sm;                                   // [CIN][PA]
    bf16* sG = sm + CIN * C::PA;                     // [COUT][PG]
    float* sDb = reinterpret_cast<float*>(sG + COUT * C::PG);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;     // warp = tap
    const int g = lane >> 2, t = lane & 3;
    const int p = warp / 3, q = warp % 3;
    constexpr int MT = COUT / 16, NT = CIN / 8;
    float acc[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[mt][nt][j] = 0.f;
    for (int o = tid; o < COUT; o += 288) sDb[o] = 0.f;

    const int tx = W / kTile, ty = H / kTile;
    const int tiles = tx * ty * images;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int im = tile / (tx * ty), rem = tile % (tx * ty);
        const int r0 = (rem / tx) * kTile, c0 = (rem % tx) * kTile;
        const size_t hw = (size_t)H * W;
        __syncthreads();                             // previous tile's operands are consumed
        // activation tile with halo, channel-major (8 channels of one plane per
        // thread and pixel)
        constexpr int NPA = C::HALO * C::HALO;
        for (int e = tid; e < NPA * (CIN / 8); e += 288) {
            const int pl = e / NPA, pix = e - pl * NPA, ch = pl * 8;
            const int yy = pix / C::HALO, xx = pix % C::HALO;
            const int gy = r0 + yy - 1, gx = c0 + xx - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                v = *reinterpret_cast<const uint4*>(a + (((size_t)im * (CIN / 8) + pl) * hw + (size_t)gy * W + gx) * 8);
            const bf16* vv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) sA[(ch + j) * C::PA + pix] = vv[j];
        }
        for (int e = tid; e < kTile * kTile * (COUT / 8); e += 288) {
            const int pl = e / (kTile * kTile), pix = e - pl * (kTile * kTile), ch = pl * 8;
            const int gy = r0 + pix / kTile, gx = c0 + pix % kTile;
            const uint4 v =
                *reinterpret_cast<const uint4*>(gr + (((size_t)im * (COUT / 8) + pl) * hw + (size_t)gy * W + gx) * 8);
            const bf16* vv = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) sG[(ch + j) * C::PG + pix] = vv[j];
        }
        __syncthreads();
        // bias gradient: channel o = tid % 32 sums every 9th pixel row
        if ((tid & 31) < COUT) {
            const int o = tid & 31;
            float s = 0.f;
            for (int px = warp; px < kTile * kTile; px += 9) s += __bfloat162float(sG[o * C::PG + px]);
            atomicAdd(sDb + o, s);
        }
        // K loop: one output row of 16 pixels per step
#pragma unroll 2
        for (int rr = 0; rr < kTile; ++rr) {
            uint32_t af[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                // A[m][k] = G[pixel k][channel m]
                const bf16* gp = sG + (mt * 16 + g) * C::PG + rr * kTile + 2 * t;
                af[mt][0] = ld32(gp);
                af[mt][1] = ld32(gp + 8 * C::PG);
                af[mt][2] = ld32(gp + 8);
                af[mt][3] = ld32(gp + 8 * C::PG + 8);
            }
            const int base = (rr + p) * C::HALO + q + 2 * t;  // pixel (rr + p - 1, 2t + q - 1) + halo
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                // B[k][n] = A_tap[pixel k][channel n]: two pixels of one channel
                const bf16* ap = sA + (nt * 8 + g) * C::PA + base;
                const uint32_t b0 = pack2(ap[0], ap[1]);
                const uint32_t b1 = pack2(ap[8], ap[9]);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) mma_bf16(acc[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], b0, b1);
            }
        }
    }
    // C[m][n] = dW[o = m][i = n] of this tap
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = mt * 16 + g + (j >= 2 ? 8 : 0);
                const int i = nt * 8 + 2 * t + (j & 1);
                if (o < cout_real && i < cin_real) atomicAdd(dw + ((size_t)o * cin_real + i) * 9 + warp, acc[mt][nt][j]);
            }
        }
    }
    __syncthreads();
    for (int o = tid; o < cout_real; o += 288) atomicAdd(db + o, sDb[o]);
}

// ---------------------------------------------------------------------------
// loss and its gradient in the output: g = 2 c_k (o - t) / npx (16 channels
// in two planes, 4 used; hw = H W); per-block FP64 partial sums of the loss
// ---------------------------------------------------------------------------
__global__ void cnn_loss_kernel(const float* __restrict__ o, const float* __restrict__ tg, float4 cw,
                                bf16* __restrict__ gout, double* __restrict__ loss, long long npx, long long hw) {
    __shared__ double red[8];
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < npx) {
        const float4 ov = reinterpret_cast<const float4*>(o)[i];
        const float4 tv = reinterpret_cast<const float4*>(tg)[i];
        const float e0 = ov.x - tv.x, e1 = ov.y - tv.y, e2 = ov.z - tv.z, e3 = ov.w - tv.w;
        l = (double)cw.x * e0 * e0 + (double)cw.y * e1 * e1 + (double)cw.z * e2 * e2 + (double)cw.w * e3 * e3;
        const float s = 2.0f / (float)npx;
        const long long img = i / hw, px = i - img * hw;
        uint4* dst = reinterpret_cast<uint4*>(gout + (img * 2 * hw + px) * 8);
        dst[0] = make_uint4(pack2(__float2bfloat16(s * cw.x * e0), __float2bfloat16(s * cw.y * e1)),
                            pack2(__float2bfloat16(s * cw.z * e2), __float2bfloat16(s * cw.w * e3)), 0u, 0u);
        dst[hw] = make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s / (double)npx);
    }
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba, Algorithm 1) on the FP32 parameter vector
// ---------------------------------------------------------------------------
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ gd, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = gd[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ---------------------------------------------------------------------------
// BF16 weight packing: forward [tap][coutp][cinp], and for the input
// gradient the flipped transpose [tap'][cinp][coutp_g] with
// w'[tap'][i][o] = w[o][i][8 - tap'] (zero in the padding)
// ---------------------------------------------------------------------------
__global__ void pack_kernel(const float* __restrict__ w, bf16* __restrict__ fwd, bf16* __restrict__ bwd,
                            int cin, int cout, int cinp, int coutp, int coutg) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nf = 9 * coutp * cinp;
    if (e < nf) {
        const int tap = e / (coutp * cinp), o = (e / cinp) % coutp, i = e % cinp;
        const float x = (o < cout && i < cin) ? w[((size_t)o * cin + i) * 9 + tap] : 0.f;
        fwd[e] = __float2bfloat16(x);
    }
    const int nb = 9 * cinp * coutg;
    if (bwd && e < nb) {
        const int tap = e / (cinp * coutg), i = (e / coutg) % cinp, o = e % coutg;
        const float x = (o < cout && i < cin) ? w[((size_t)o * cin + i) * 9 + (8 - tap)] : 0.f;
        bwd[e] = __float2bfloat16(x);
    }
}

// ---------------------------------------------------------------------------
// output -> warm start (x0, d1, (d2h, d2v) interleaved)
// ---------------------------------------------------------------------------
__global__ void split_start_kernel(const float* __restrict__ o, float s0, float s1, float s2,
                                   float* __restrict__ x0, float* __restrict__ d0, long long n, long long npx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    const long long im = i / n, px = i % n;
    const float4 v = reinterpret_cast<const float4*>(o)[i];
    x0[i] = s0 * v.x;
    float* d = d0 + im * 3 * n;
    d[px] = s1 * v.y;
    reinterpret_cast<float2*>(d + n)[px] = make_float2(s2 * v.z, s2 * v.w);
}

// the same two steps for a group of separately stored problems (the learned
// start of a batch solve): per-image device pointers, passed by value
constexpr int kWsBatch = 16;
struct ImgPtrs {
    const float* y[kWsBatch];
    const uint8_t* m[kWsBatch];
    float* x0[kWsBatch];
    float* d0[kWsBatch];
};

// grid (ceil(hw / 256), images)
__global__ void cnn_input_ptrs_kernel(ImgPtrs P, bf16* __restrict__ a0, long long hw) {
    const long long px = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= hw) return;
    const int img = blockIdx.y;
    const bool obs = P.m[img][px] != 0;
    const float y = obs ? P.y[img][px] : 0.f;
    reinterpret_cast<uint4*>(a0)[(long long)img * hw + px] =
        make_uint4(pack2(__float2bfloat16(y), __float2bfloat16(obs ? 1.f : 0.f)), 0u, 0u, 0u);
}

// grid (ceil(hw / 256), images)
__global__ void split_start_ptrs_kernel(const float* __restrict__ o, float s0, float s1, float s2, ImgPtrs P,
                                        long long hw) {
    const long long px = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= hw) return;
    const int img = blockIdx.y;
    const float4 v = reinterpret_cast<const float4*>(o)[(long long)img * hw + px];
    P.x0[img][px] = s0 * v.x;
    float* d = P.d0[img];
    d[px] = s1 * v.y;
    reinterpret_cast<float2*>(d + hw)[px] = make_float2(s2 * v.z, s2 * v.w);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
// the driver's tensor-map encoder (through the runtime, no link to the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// One layer on tcgen05 (persistent CTAs over 8 x 16 tiles, as many per SM as
// registers, shared memory and tensor memory allow). The input planes [img][CIN / 8][H][W][8] are viewed by TMA as a 4-D tensor
// (8 W elements of a plane row, H, CIN / 8 planes, images) with strides
// (16 W, 16 W H, 16 W H CIN / 8) bytes, and a box of (80, 18, CIN / 8, 1):
// one halo tile per copy, laid out in shared memory as
// [plane][halo row][halo column][8 channels].
template <int CIN, int MODE>
cudaError_t conv_tc(const bf16* in, const bf16* w, const float* bias, void* out, const bf16* gate, int count, int H,
                    int W, int sms, int* err, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        // CTAs one SM holds, from the kernel's registers and static shared
        // memory (the whole unified L1 / shared array given to shared memory)
        // and the 2 x cout tensor-memory columns each CTA allocates of 512
        cudaFuncAttributes fa;
        int dev = 0, smem_sm = 0, smem_rsv = 0, regs_sm = 0;
        if (cudaFuncSetAttribute(conv3x3_tc<CIN, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, conv3x3_tc<CIN, MODE>) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
            return cudaErrorInvalidConfiguration;
        const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * 128;
        const int by_regs = regs_sm / std::max(regs_cta, 1);
        const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + smem_rsv);
        const int cout = MODE == kModeOutF32 ? 16 : 32;
        per_sm = std::max(1, std::min({by_regs, by_smem, 16, 512 / (2 * cout)}));
    }
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tm;
    const cuuint64_t plane = (cuuint64_t)W * H * 16;
    const cuuint64_t dims[4] = {(cuuint64_t)W * 8, (cuuint64_t)H, (cuuint64_t)(CIN / 8), (cuuint64_t)count};
    const cuuint64_t strides[3] = {(cuuint64_t)W * 16, plane, plane * (CIN / 8)};
    const cuuint32_t box[4] = {(cuuint32_t)kTcHW * 8, (cuuint32_t)kTcHH, (cuuint32_t)(CIN / 8), 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(in), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int ntiles = (W / kTcTW) * (H / kTcTH) * count;
    const int grid = std::min(ntiles, per_sm * sms);
    conv3x3_tc<CIN, MODE><<<grid, 128, 0, s>>>(tm, w, bias, out, gate, H, W, count, err);
    ++g_cnn_launches;
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t wgrad(const bf16* a, const bf16* g, float* dw, float* db, int cin_real, int cout_real, int count,
                  int H, int W, int sms, cudaStream_t s) {
    const int tiles = (H / kTile) * (W / kTile) * count;
    const int grid = std::min(tiles, 2 * sms);
    conv3x3_wgrad_kernel<CIN, COUT><<<grid, 288, WgradCfg<CIN, COUT>::SMEM, s>>>(a, g, dw, db, cin_real, cout_real, H,
                                                                                  W, count);
    ++g_cnn_launches;
    return cudaGetLastError();
}

}  // namespace

struct admm_cnn_s {
    int device = 0;
    int sms = 152;
    long long max_px = 0;
    bool training = false;
    float* params = nullptr;       // FP32 master vector
    float* grads = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    long long adam_t = 0;
    bf16* wf[kLayers] = {};        // packed forward weights
    bf16* wb[kLayers] = {};        // packed input-gradient weights (layers 1..)
    bf16* a0 = nullptr;            // input, one plane of 8 channels
    bf16* act[kLayers - 1] = {};   // activations after layers 0..6 (training keeps all)
    float* out = nullptr;          // output, 4 channels FP32
    bf16* gbuf[2] = {};            // gradient ping-pong, 32 channels
    bf16* gout = nullptr;          // output gradient, 16 channels
    double* loss = nullptr;        // device accumulator
    double* h_loss = nullptr;      // pinned
    int* tc_err = nullptr;         // set by a tensor-core convolution whose bounded wait ran out
    std::vector<void*> allocs;
};

namespace {

template <typename T>
int dalloc(admm_cnn_s* n, T** p, size_t count) {
    void* q = nullptr;
    if (admm::alloc_fault_fire()) return ADMM_ENOMEM;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ADMM_ENOMEM;
    }
    n->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return ADMM_OK;
}

int check_shape(const admm_cnn_s* n, int count, int H, int W) {
    if (count <= 0 || H < kTile || W < kTile || H % kTile || W % kTile) return ADMM_EINVAL;
    if ((long long)count * H * W > n->max_px) return ADMM_EINVAL;
    return ADMM_OK;
}

int pack_all(admm_cnn_s* n, cudaStream_t s) {
    for (int l = 0; l < kLayers; ++l) {
        const int cin = layer_cin(l), cout = layer_cout(l);
        const int cinp = layer_cinp(l), coutp = layer_coutp(l);
        const int coutg = pad16(cout);
        const int nmax = std::max(9 * coutp * cinp, 9 * cinp * coutg);
        pack_kernel<<<(nmax + 255) / 256, 256, 0, s>>>(n->params + param_offset(l), n->wf[l], n->wb[l], cin, cout,
                                                        cinp, coutp, coutg);
        ++g_cnn_launches;
        CKC(cudaGetLastError());
    }
    return ADMM_OK;
}

// the eight layers on the prepared input n->a0; with `keep` every activation
// is stored for the backward pass, otherwise two buffers alternate
int run_layers(admm_cnn_s* n, int count, int H, int W, bool keep, cudaStream_t s) {
    const bf16* cur = n->a0;
    for (int l = 0; l < kLayers; ++l) {
        const float* b = n->params + param_offset(l) + (long long)layer_cout(l) * layer_cin(l) * 9;
        if (l == kLayers - 1) {
            CKC((conv_tc<32, kModeOutF32>(cur, n->wf[l], b, n->out, nullptr, count, H, W, n->sms, n->tc_err, s)));
        } else {
            bf16* dst = keep ? n->act[l] : n->act[l & 1];
            if (l == 0)
                CKC((conv_tc<8, kModeReluBf16>(cur, n->wf[l], b, dst, nullptr, count, H, W, n->sms, n->tc_err, s)));
            else
                CKC((conv_tc<32, kModeReluBf16>(cur, n->wf[l], b, dst, nullptr, count, H, W, n->sms, n->tc_err, s)));
            cur = dst;
        }
    }
    return ADMM_OK;
}

// forward pass from [M^T y, mask] stored contiguously for the count images
int forward(admm_cnn_s* n, int count, int H, int W, const float* ybar, const uint8_t* mask, bool keep,
            cudaStream_t s) {
    const long long npx = (long long)count * H * W;
    cnn_input_kernel<<<(unsigned)((npx + 255) / 256), 256, 0, s>>>(ybar, mask, n->a0, npx);
    ++g_cnn_launches;
    CKC(cudaGetLastError());
    return run_layers(n, count, H, W, keep, s);
}

// loss, gradients into n->grads (zeroed first)
int backward(admm_cnn_s* n, int count, int H, int W, const float* target, const float* chan_w, cudaStream_t s) {
    const long long npx = (long long)count * H * W;
    CKC(cudaMemsetAsync(n->loss, 0, sizeof(double), s));
    CKC(cudaMemsetAsync(n->grads, 0, param_count() * sizeof(float), s));
    const float4 cw = make_float4(chan_w[0], chan_w[1], chan_w[2], chan_w[3]);
    cnn_loss_kernel<<<(unsigned)((npx + 255) / 256), 256, 0, s>>>(n->out, target, cw, n->gout, n->loss, npx,
                                                                   (long long)H * W);
    ++g_cnn_launches;
    CKC(cudaGetLastError());
    const bf16* g = n->gout;                        // gradient in the output of layer l
    for (int l = kLayers - 1; l >= 0; --l) {
        float* dw = n->grads + param_offset(l);
        float* db = dw + (long long)layer_cout(l) * layer_cin(l) * 9;
        const bf16* a_in = l == 0 ? n->a0 : n->act[l - 1];
        if (l == kLayers - 1)
            CKC((wgrad<32, 16>(a_in, g, dw, db, kWidth, kOut, count, H, W, n->sms, s)));
        else if (l == 0)
            CKC((wgrad<8, 32>(a_in, g, dw, db, kIn, kWidth, count, H, W, n->sms, s)));
        else
            CKC((wgrad<32, 32>(a_in, g, dw, db, kWidth, kWidth, count, H, W, n->sms, s)));
        if (l == 0) break;
        bf16* gnext = n->gbuf[l & 1];
        if (l == kLayers - 1)
            CKC((conv_tc<16, kModeGateBf16>(g, n->wb[l], nullptr, gnext, a_in, count, H, W, n->sms, n->tc_err, s)));
        else
            CKC((conv_tc<32, kModeGateBf16>(g, n->wb[l], nullptr, gnext, a_in, count, H, W, n->sms, n->tc_err, s)));
        g = gnext;
    }
    return ADMM_OK;
}

}  // namespace

extern "C" {

long long admm_cnn_param_count(void) { return param_count(); }

long long admm_cnn_launches(void) {
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    return g_cnn_launches;
}

void admm_cnn_destroy(admm_cnn_t net) {
    if (!net) return;
    for (void* p : net->allocs) cudaFree(p);
    if (net->h_loss) cudaFreeHost(net->h_loss);
    delete net;
}

int admm_cnn_create(admm_cnn_t* out, long long max_pixels, int training) {
    if (!out || max_pixels <= 0) return ADMM_EINVAL;
    *out = nullptr;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    admm_cnn_s* n = new (std::nothrow) admm_cnn_s();
    if (!n) return ADMM_ENOMEM;
    int rc = ADMM_OK;
    auto bail = [&](int r) {
        admm_cnn_destroy(n);
        return r;
    };
    if (cudaGetDevice(&n->device) != cudaSuccess) return bail(ADMM_ECUDA);
    cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, n->device);
    n->max_px = max_pixels;
    n->training = training != 0;
    const long long P = param_count();
    const size_t px = (size_t)max_pixels;
    if ((rc = dalloc(n, &n->params, P)) || (rc = dalloc(n, &n->a0, px * 8)) || (rc = dalloc(n, &n->out, px * 4)) ||
        (rc = dalloc(n, &n->tc_err, 1)))
        return bail(rc);
    for (int l = 0; l < kLayers; ++l) {
        if ((rc = dalloc(n, &n->wf[l], (size_t)9 * layer_coutp(l) * layer_cinp(l)))) return bail(rc);
        if (l > 0 && (rc = dalloc(n, &n->wb[l], (size_t)9 * layer_cinp(l) * pad16(layer_cout(l))))) return bail(rc);
    }
    const int nact = n->training ? kLayers - 1 : 2;
    for (int l = 0; l < nact; ++l)
        if ((rc = dalloc(n, &n->act[l], px * kWidth))) return bail(rc);
    if (n->training) {
        if ((rc = dalloc(n, &n->grads, P)) || (rc = dalloc(n, &n->m, P)) || (rc = dalloc(n, &n->v, P)) ||
            (rc = dalloc(n, &n->gbuf[0], px * kWidth)) || (rc = dalloc(n, &n->gbuf[1], px * kWidth)) ||
            (rc = dalloc(n, &n->gout, px * 16)) || (rc = dalloc(n, &n->loss, 1)))
            return bail(rc);
        if (admm::alloc_fault_fire() || cudaHostAlloc(&n->h_loss, sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
            n->h_loss = nullptr;
            return bail(ADMM_ENOMEM);
        }
    }
    if (cudaMemset(n->params, 0, P * sizeof(float)) != cudaSuccess) return bail(ADMM_ECUDA);
    if (cudaMemset(n->tc_err, 0, sizeof(int)) != cudaSuccess) return bail(ADMM_ECUDA);
    if (pack_all(n, nullptr) != ADMM_OK || cudaDeviceSynchronize() != cudaSuccess) return bail(ADMM_ECUDA);
    *out = n;
    return ADMM_OK;
}

int admm_cnn_set_params(admm_cnn_t net, const float* params) {
    if (!net || !params) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    const long long P = param_count();
    CKC(cudaMemcpy(net->params, params, P * sizeof(float), cudaMemcpyDefault));
    if (net->training) {
        CKC(cudaMemset(net->m, 0, P * sizeof(float)));
        CKC(cudaMemset(net->v, 0, P * sizeof(float)));
        net->adam_t = 0;
    }
    const int rc = pack_all(net, nullptr);
    if (rc != ADMM_OK) return rc;
    CKC(cudaDeviceSynchronize());
    return ADMM_OK;
}

int admm_cnn_get_params(admm_cnn_t net, float* params) {
    if (!net || !params) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    CKC(cudaMemcpy(params, net->params, param_count() * sizeof(float), cudaMemcpyDefault));
    return ADMM_OK;
}

int admm_cnn_forward(admm_cnn_t net, int count, int H, int W, const float* ybar, const uint8_t* mask, float* out,
                     void* stream) {
    if (!net || !ybar || !mask || !out) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    int rc = check_shape(net, count, H, W);
    if (rc != ADMM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = forward(net, count, H, W, ybar, mask, false, s)) != ADMM_OK) return rc;
    CKC(cudaMemcpyAsync(out, net->out, (size_t)count * H * W * 4 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return ADMM_OK;
}

int admm_cnn_gradients(admm_cnn_t net, int count, int H, int W, const float* ybar, const uint8_t* mask,
                       const float* target, const float* chan_w, float* grads, double* loss, void* stream) {
    if (!net || !ybar || !mask || !target || !chan_w || !grads || !net->training) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    int rc = check_shape(net, count, H, W);
    if (rc != ADMM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = forward(net, count, H, W, ybar, mask, true, s)) != ADMM_OK) return rc;
    if ((rc = backward(net, count, H, W, target, chan_w, s)) != ADMM_OK) return rc;
    CKC(cudaMemcpyAsync(grads, net->grads, param_count() * sizeof(float), cudaMemcpyDefault, s));
    CKC(cudaMemcpyAsync(net->h_loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKC(cudaStreamSynchronize(s));
    if (loss) *loss = *net->h_loss;
    return ADMM_OK;
}

int admm_cnn_train_step(admm_cnn_t net, int count, int H, int W, const float* ybar, const uint8_t* mask,
                        const float* target, const float* chan_w, float lr, double* loss, void* stream) {
    if (!net || !ybar || !mask || !target || !chan_w || !net->training || !(lr > 0.f)) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    int rc = check_shape(net, count, H, W);
    if (rc != ADMM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = forward(net, count, H, W, ybar, mask, true, s)) != ADMM_OK) return rc;
    if ((rc = backward(net, count, H, W, target, chan_w, s)) != ADMM_OK) return rc;
    net->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)net->adam_t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)net->adam_t));
    const long long P = param_count();
    adam_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(net->params, net->grads, net->m, net->v, P, lr, b1, b2,
                                                            1e-8f, c1, c2);
    ++g_cnn_launches;
    CKC(cudaGetLastError());
    if ((rc = pack_all(net, s)) != ADMM_OK) return rc;
    if (loss) {
        CKC(cudaMemcpyAsync(net->h_loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CKC(cudaStreamSynchronize(s));
        *loss = *net->h_loss;
    }
    return ADMM_OK;
}

int admm_cnn_predict_start(admm_cnn_t net, int count, int H, int W, const float* ybar, const uint8_t* mask,
                           const float* scales, float* x0, float* d0, void* stream) {
    if (!net || !ybar || !mask || !scales || !x0 || !d0) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_cnn_mutex);
    int rc = check_shape(net, count, H, W);
    if (rc != ADMM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = forward(net, count, H, W, ybar, mask, false, s)) != ADMM_OK) return rc;
    const long long n = (long long)H * W, npx = n * count;
    split_start_kernel<<<(unsigned)((npx + 255) / 256), 256, 0, s>>>(net->out, scales[0], scales[1], scales[2], x0,
                                                                     d0, n, npx);
    ++g_cnn_launches;
    CKC(cudaGetLastError());
    return ADMM_OK;
}

// ---------------------------------------------------------------------------
// The library-global warm-start network of admm_warmstart_load, used by
// admm_deconv_solve_batch(..., use_warmstart = 1, ...): parameters and scales
// on the host; the inference network is created on first use on the current
// device and grown to the largest image it meets.
// ---------------------------------------------------------------------------
namespace {
struct WarmStartNet {
    bool loaded = false;
    std::vector<float> params;
    float scales[4] = {0.f, 0.f, 0.f, 0.f};
    admm_cnn_t net = nullptr;
    int device = -1;
    long long cap = 0;
};
std::mutex g_ws_mutex;
WarmStartNet g_ws;
}  // namespace

int admm_warmstart_load(const char* path) {
    std::lock_guard<std::mutex> lk(g_ws_mutex);
    if (!path) {
        if (g_ws.net) admm_cnn_destroy(g_ws.net);
        g_ws = WarmStartNet();
        return ADMM_OK;
    }
    FILE* f = std::fopen(path, "rb");
    if (!f) return ADMM_EINVAL;
    char magic[8];
    int32_t version = 0, reserved = 0;
    int64_t count = 0;
    float scales[4];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "ADMMCNN1", 8) == 0 &&
              std::fread(&version, sizeof(version), 1, f) == 1 && version == 1 &&
              std::fread(&reserved, sizeof(reserved), 1, f) == 1 &&
              std::fread(&count, sizeof(count), 1, f) == 1 && count == param_count() &&
              std::fread(scales, sizeof(float), 4, f) == 4;
    std::vector<float> params;
    if (ok) {
        params.resize((size_t)count);
        ok = std::fread(params.data(), sizeof(float), params.size(), f) == params.size();
        char extra;
        ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing after the parameters
    }
    std::fclose(f);
    if (!ok) return ADMM_EINVAL;
    for (float v : params)
        if (!std::isfinite(v)) return ADMM_EINVAL;
    if (g_ws.net) admm_cnn_destroy(g_ws.net);
    g_ws = WarmStartNet();
    g_ws.params.swap(params);
    std::memcpy(g_ws.scales, scales, sizeof(scales));
    g_ws.loaded = true;
    return ADMM_OK;
}

}  // extern "C"

namespace admm {
// the driver's tensor-map encoder, for the other translation units (null when
// the driver does not provide it)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encode_fn() { return tensor_map_encoder(); }

bool ws_loaded() {
    std::lock_guard<std::mutex> lk(g_ws_mutex);
    return g_ws.loaded;
}

// images of H x W that one ws_predict_starts call takes: up to 16, and no
// more than 16 x 512 x 512 pixels (the network's buffers hold about 180 B per
// pixel)
int ws_batch_limit(int H, int W) {
    const long long px = std::max(1LL, (long long)H * W);
    return (int)std::max(1LL, std::min((long long)kWsBatch, 16LL * 512 * 512 / px));
}

// predicted starts of `count` H x W TV problems (count <= ws_batch_limit):
// for image i, [M^T y, mask] from ybar[i], mask[i], and x0[i] (H W floats)
// and d0[i] (3 H W floats in the layout of admm_deconv_get_state) written,
// device pointers, on `s`. One pass of the network over the group; each
// image's result has the bits of a pass over that image alone.
int ws_predict_starts(int count, int H, int W, const float* const* ybar, const uint8_t* const* mask,
                      float* const* x0, float* const* d0, cudaStream_t s) {
    if (count < 1 || count > ws_batch_limit(H, W)) return ADMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_ws_mutex);
    if (!g_ws.loaded) return ADMM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADMM_ECUDA;
    const long long hw = (long long)H * W, px = hw * count;
    if (!g_ws.net || g_ws.device != dev || g_ws.cap < px) {
        if (g_ws.net) admm_cnn_destroy(g_ws.net);
        g_ws.net = nullptr;
        const long long cap = std::max(px, 512LL * 512LL);
        admm_cnn_t n = nullptr;
        int rc = admm_cnn_create(&n, cap, 0);
        if (rc != ADMM_OK) return rc;
        rc = admm_cnn_set_params(n, g_ws.params.data());
        if (rc != ADMM_OK) {
            admm_cnn_destroy(n);
            return rc;
        }
        g_ws.net = n;
        g_ws.device = dev;
        g_ws.cap = cap;
    }
    admm_cnn_s* net = g_ws.net;
    std::lock_guard<std::mutex> lk2(g_cnn_mutex);
    int rc = check_shape(net, count, H, W);
    if (rc != ADMM_OK) return rc;
    ImgPtrs P{};
    for (int i = 0; i < count; ++i) {
        if (!ybar[i] || !mask[i] || !x0[i] || !d0[i]) return ADMM_EINVAL;
        P.y[i] = ybar[i];
        P.m[i] = mask[i];
        P.x0[i] = x0[i];
        P.d0[i] = d0[i];
    }
    const dim3 grid((unsigned)((hw + 255) / 256), (unsigned)count);
    cnn_input_ptrs_kernel<<<grid, 256, 0, s>>>(P, net->a0, hw);
    ++g_cnn_launches;
    CKC(cudaGetLastError());
    if ((rc = run_layers(net, count, H, W, false, s)) != ADMM_OK) return rc;
    split_start_ptrs_kernel<<<grid, 256, 0, s>>>(net->out, g_ws.scales[0], g_ws.scales[1], g_ws.scales[2], P, hw);
    ++g_cnn_launches;
    CKC(cudaGetLastError());
    return ADMM_OK;
}
}  // namespace admm
