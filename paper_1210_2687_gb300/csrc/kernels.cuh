// kernels.cuh -- device kernels of one ADMM iteration for a batch of problems.
//
// One iteration of TV-MD (Algorithm 3 with line 7 replaced by eq. new_line)
// or FA-MD (Algorithm 2 with H1 = A, H2 = P) is split into two phases that
// each stream the batch once through HBM:
//
//  column phase  (col_phase):  the row-DFTs of (zeta1, w) -> forward column
//                 DFTs -> x^ = K (conj(Lambda) Z1^ + W^)  [eq. fast_inversion /
//                 eq. invAnalysisp1, 1/(HW) folded into K] and (A x)^ = Lambda x^
//                 -> inverse column DFTs -> row-DFTs of (x, A x)
//  row phase     (row_phase_tv):  inverse row DFT -> x, A x on a strip of rows
//                 -> mask-decoupled prox + dual update (eq. new_line, Alg. 3
//                 line 8) -> TV differences, vector-soft, dual update (Alg. 3
//                 lines 9-11) -> zeta1 = u1 + d1, w = gamma (Dh^T dh + Dv^T dv)
//                 with delta = u2 + d2 (Alg. 3 lines 3-5 of the next iteration)
//                 -> forward row DFT of the packed p = zeta1 + i w, split into
//                 the half spectra of zeta1 and w.
//
// Both real signals of each phase share one complex transform: a real pair
// (a, b) is carried as a + i b and separated with the Hermitian symmetry of
// real-signal spectra. Only the half spectrum k_c = 0..W/2 is stored between
// phases, as float4 (Re, Im of the first signal, Re, Im of the second).
//
// Persistent state per problem is the scaled dual d = (d1, d2) only; u is
// formed on the fly (zeta = u + d, Algorithm 2 line 3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "fft.cuh"

namespace admm {

constexpr int kThreads = 256;
constexpr int kNumPartials = 5;   // data term, regulariser sum, ||x||^2, ||x - x_prev||^2, ||d - d_prev||^2

// Mutable per-problem control block.
struct ProbCtl {
    int iter;          // iterations completed
    int active;        // 1 while iterating
    int converged;
    int status;        // 0 or ADMM_ENONFINITE
    unsigned arrive;   // row-phase CTAs of the current iteration that finished
    int have_obj;      // obj_prev valid
    double obj;        // objective at the last evaluation
    double obj_prev;
    double rel_x;      // -1 until evaluated
    double rel_obj;    // -1 until evaluated
    double primal_res; // ||d_k - d_{k-1}|| = ||H z_k - u_k|| (Alg. 2), -1 until evaluated
    int input_bad;     // set by prepare_kernel: an observed value is not finite
    int pad_;
    unsigned cg_arrive;  // Reeves-Sorel variants: row CTAs that have added their share of alpha's denominator
    float cg_alpha;      // ... and the step of the iteration's conjugate-gradient update
    unsigned long long t0;       // device clock (ns) when the batch was set up
    unsigned long long t_start;  // ... when the problem took a slot
    unsigned long long t_done;   // ... when it retired
};

__device__ __forceinline__ unsigned long long device_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-problem constants and buffers (all device pointers).
struct ProbDesc {
    float4* Sa;               // H x Wp: column-phase output (row-DFTs of x, A x)
    float4* Sb;               // H x Wp: row-phase output (row-DFTs of zeta1, w)
    float* d1;                // H x W
    float* d2;                // two buffers of d2_stride floats each (TV: H x W float2
                              // (h, v); frame: nb x H x W planes). TV: iteration k
                              // reads buffer (k+1)&1 and writes buffer k&1, so CTAs
                              // that recompute a neighbour's halo always see the old
                              // d2. Frame priors: zeta2 in place in buffer 0, beside
                              // zbits (haar.cuh)
    long long d2_stride;
    const float* ybar;        // H x W, M^T y (0 where unobserved)
    const uint8_t* mask;      // H x W, 1 = observed (effective mask); the iteration
                              // kernels read the same information from ybar (NaN =
                              // unobserved), which saves the mask's byte per pixel
    const float2* lamT;       // Wc x H, Lambda (column-major half spectrum)
    const float* kT;          // Wc x H, diagonal inverse with 1/(HW) folded in
    float* xprev;             // H x W, x of the previous iteration (rel-x rule)
    float* work;              // frame prior and Reeves-Sorel variants: 3 x H x W scratch
                              // planes (x, zeta1, w)
    float* cg;                // Reeves-Sorel variants: 6 x H x W planes (x~, A x~, v, A v, s, z)
    double* cg_part;          // ... and 2 x (row CTAs) partial sums of the CG step
    double* partials;         // n_strips x kNumPartials
    ProbCtl* ctl;
    float lam, mu1, mu2, gamma, tau, inv1pmu1;
    int stop, max_iters, check_every;
    int n_strips;             // CTAs per problem of the kernel that finishes an iteration
    int n_slots;              // partial-sum slots to reduce (0: n_strips)
    int warm;                 // 1: start from x1 = x0, d0 given (Sb holds the row-DFTs
                              // of x0, d1/d2 buffer 0 hold d0); 2: resume a saved
                              // state (Sb holds the row-DFTs of the right-hand side,
                              // d1/d2 buffer 0 the duals: the first x-step solves as
                              // usual); 0: u0 = d0 = 0
    int ll_free;              // frame prior: 1 = the last low-low band unpenalised
    double tol;
    // frame prior, per band b (3 L + 1 bands): the threshold lambda / mu_b and
    // the factor gamma_b / gamma applied to zeta_b before the synthesis, so that
    // w = gamma P^T (scaled zeta2) = sum_b gamma_b P_b^T zeta_b (one penalty per
    // band, eq. diagonal_penalty); tau and 1 when every band has mu2
    float band_tau[13];
    float band_zs[13];
    float band_izs[13];       // gamma / gamma_b (1 when every band has mu2)
    uint32_t* zbits;          // frame analysis prior: H x W words, two bits per band of the
                              // last analysis (threshold passed; argument negative), beside
                              // zeta2 in d2 buffer 0; null for FS-MD and the TV priors
    int test_stall;           // test hook (ADMM_OPT_TEST_STALL): the TV row phase withholds
                              // one of its bulk copies, so that its bounded wait runs out
    const void* zmap;         // frame prior: L + 1 TMA tensor maps (128 bytes each) of the d2
                              // buffers, the synthesis tile's halo boxes (null: cp.async)
};

// Continuous batching: a launch covers gridDim.y slots; slot s works on
// problem map[s] (or nothing when map[s] < 0). When a problem retires, the
// CTA that finishes its iteration hands the slot to the next queued problem,
// so launches stay full until the queue drains. A problem's first iteration
// (k = 1) treats its whole state as zero (u0 = d0 = 0), so a slot needs no
// reset before it starts a new problem.
struct SlotTable {
    int* map;       // gridDim.y entries
    int* queue;     // next problem index to hand out
    int pool;       // problems in the descriptor table
};

// stop rules (values of ADMM_STOP_*)
constexpr int kStopIters = 0, kStopRelX = 1, kStopRelObj = 2;
constexpr int kStatusNonFinite = -5;
constexpr int kStatusTimeout = -6;     // a bounded wait for an asynchronous copy ran out

__device__ __forceinline__ bool is_check_iter(const ProbDesc& P, int k) {
    return P.stop == kStopRelX && ((k % P.check_every) == 0 || k == P.max_iters);
}
__device__ __forceinline__ bool store_prev_iter(const ProbDesc& P, int k) {
    return P.stop == kStopRelX && (((k + 1) % P.check_every) == 0 || k + 1 == P.max_iters);
}
__device__ __forceinline__ bool need_obj_iter(const ProbDesc& P, int k) {
    return P.stop == kStopRelObj || is_check_iter(P, k) || k == P.max_iters;
}

// Neumaier-compensated FP32 accumulator
struct CompSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float t = s + v;
        c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Asynchronous global->shared copies (cp.async); completion is tracked per
// thread with commit/wait groups, so a thread that only reads what it copied
// itself needs no block barrier.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// wait until at most n of this thread's groups are pending (n folds to a
// constant where the caller's loop is unrolled; larger n wait for more)
__device__ __forceinline__ void cp_async_wait_n(int n) {
    switch (n) {
        case 0: cp_async_wait<0>(); break;
        case 1: cp_async_wait<1>(); break;
        case 2: cp_async_wait<2>(); break;
        case 3: cp_async_wait<3>(); break;
        case 4: cp_async_wait<4>(); break;
        case 5: cp_async_wait<5>(); break;
        case 6: cp_async_wait<6>(); break;
        default: cp_async_wait<7>(); break;
    }
}

// Programmatic dependent launch of the iteration's kernel chain (column
// phase, row side, next column phase, ...). A chain kernel may be launched
// before its predecessor in the stream has completed: its CTAs are scheduled
// once every CTA of the predecessor has exited, and the first thing they do
// is wait for the predecessor's completion and the visibility of its writes
// (chain_wait), so nothing the predecessor writes is touched before that.
// The launch processing overlaps the predecessor's completion. (Releasing the
// successor earlier, from the top of each kernel, measured slower: its
// waiting CTAs held resources the predecessor's last wave could use.)
// Launched without the attribute, the wait is a no-op.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Host side: while `t_chain_overlap` is set on the launching thread, chain
// kernels go out with programmatic stream serialization (the batch engine
// sets it around its iteration launches and graph captures).
inline thread_local bool t_chain_overlap = false;
template <typename... KArgs, typename... Args>
cudaError_t launch_chain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    if (!t_chain_overlap) {
        kern<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Bulk asynchronous copies (the copy engine, cp.async.bulk) completing on an
// mbarrier: `bytes` a multiple of 16, both addresses 16-byte aligned.
__device__ __forceinline__ void mbar_init1(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// TMA (cp.async.bulk.tensor) load of one box of a 4-D tensor map at the
// coordinates (c0 innermost .. c3), completing on an mbarrier; `tmap` is the
// address of a 64-byte-aligned CUtensorMap in global memory, `dst` 128-byte
// aligned shared memory
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
// order this thread's earlier generic accesses to shared memory before its
// later asynchronous-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// wait for phase `parity` of an mbarrier, at most about a second; false if
// the wait ran out (the caller then marks the problem and carries on)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = device_clock_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (device_clock_ns() - t0 > 1000000000ull) return false;
        __nanosleep(20);
    }
}

// Bulk prefetch of a contiguous global range into L2 (no shared memory and no
// completion to wait for); `bytes` a multiple of 16, `p` 16-byte aligned.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// prox of the TV term at s = D_i x - d2_i (Alg. 3 line 10): vector-soft
// with threshold tau (isotropic; 0/0 = 0, via the scale max(0, 1 - tau/|s|)
// from one reciprocal square root, |s| = 0 giving -inf inside the max) or
// eq. soft per component (anisotropic)
__device__ __forceinline__ void tv_prox(float sh, float sv, float tau, bool aniso, float& uh, float& uv) {
    if (aniso) {
        uh = copysignf(fmaxf(fabsf(sh) - tau, 0.f), sh);
        uv = copysignf(fmaxf(fabsf(sv) - tau, 0.f), sv);
    } else {
        const float sc = fmaxf(0.f, fmaf(-tau, rsqrtf(fmaf(sh, sh, sv * sv)), 1.f));
        uh = sc * sh;
        uv = sc * sv;
    }
}
// the TV term of the objective at D_i x = (gh, gv)
__device__ __forceinline__ float tv_norm(float gh, float gv, bool aniso) {
    return aniso ? fabsf(gh) + fabsf(gv) : sqrtf(fmaf(gh, gh, gv * gv));
}

// observed pixels carry M^T y, unobserved ones a quiet NaN (eq. prox_g_1_uBC)
__device__ __forceinline__ bool is_observed(float yb) { return yb == yb; }

// largest PSF side the plan accepts (the spectra kernel keeps one row of
// phase factors per thread)
constexpr int kMaxPsfSide = 63;

// ---------------------------------------------------------------------------
// Column phase. Grid: (ceil(Wc / CB), problems). CTA = CB spectrum columns of
// one problem, whole height H.
// ---------------------------------------------------------------------------
template <int H, int CB>
struct ColCfg {
    static constexpr int FT = H / 8;                 // threads per transform
    static constexpr int G = kThreads / FT;          // transforms in flight
    static_assert(G >= 1 && (kThreads % FT) == 0, "H");
    static_assert(CB % G == 0 && (CB & (CB - 1)) == 0, "column block");
    static constexpr int CPG = CB / G;               // columns per group
    static constexpr int SIG = H;                     // float2 per exchange buffer
    // with one column per group, the transforms exchange through the tile
    // itself once every group holds its column in registers (the tile is
    // exactly G pairs of length-H buffers); otherwise separate buffers
    static constexpr bool ALIAS = CPG == 1;
    // columns of 1024 and more read their per-pass twiddle table from the
    // device buffer (through L1): the 8-16 KB go to more CTAs per SM
    static constexpr bool TWG = H >= 1024;
    static constexpr int TWN = TWG ? 0 : H;          // float2 of staged twiddles
    static constexpr size_t SMEM = (size_t)H * CB * sizeof(float4)
                                 + (size_t)((ALIAS ? 0 : G * 2 * SIG) + TWN) * sizeof(float2);
    static constexpr int MINB = ALIAS ? 4 : 2;       // CTAs per SM the registers are sized for
};

// Grid: (Wp / CB, problems). Wp (the stored half-spectrum width) is a
// multiple of CB; columns >= Wc = W/2 + 1 are padding, transformed but never
// read by the row phase. The H x CB tile is staged in shared memory by
// cp.async with row r's CB entries rotated (tile_slot), so that the
// column-wise float4 reads of the transforms hit distinct banks.
template <int CB>
__device__ __forceinline__ int tile_slot(int r, int c) {
    // eight consecutive rows must fill the eight 16-byte slots of a 128-byte
    // window: rows that share a window position get distinct rotations
    constexpr int SH = CB >= 8 ? 0 : (CB == 4 ? 1 : (CB == 2 ? 2 : 3));
    return r * CB + ((c + (r >> SH)) & (CB - 1));
}
// MB > 0 overrides the CTAs per SM that the registers are sized for
template <int H, int CB, int MB = 0>
__global__ void __launch_bounds__(kThreads, (MB > 0 ? MB : ColCfg<H, CB>::MINB))
col_phase(const ProbDesc* __restrict__ probs, SlotTable sl, int Wc, int Wp, const float2* __restrict__ tw_g) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using C = ColCfg<H, CB>;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const bool it0 = P.ctl->iter == 0;
    const bool warm0 = it0 && P.warm == 1;       // the first x-step returns x0
    if (it0 && !P.warm) {
        // first iteration from u0 = d0 = 0: the right-hand side is zero, so x1 = 0
        const int c0 = blockIdx.x * CB;
        for (int e = threadIdx.x; e < H * CB; e += kThreads)
            P.Sa[(size_t)(e / CB) * Wp + c0 + e % CB] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    extern __shared__ __align__(16) float4 smem4[];
    float4* stage = smem4;                                       // H x CB
    float2* xb = C::ALIAS ? reinterpret_cast<float2*>(stage)     // G x 2 exchange buffers
                          : reinterpret_cast<float2*>(stage + H * CB);
    float2* tws = reinterpret_cast<float2*>(stage + H * CB) + (C::ALIAS ? 0 : C::G * 2 * C::SIG);
    const float2* tw = C::TWG ? tw_g + pass_table_offset<H>() : tws;
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * CB;
    const float4* __restrict__ src = P.Sb;
    for (int e = tid; e < H * CB; e += kThreads) {
        const int r = e / CB, c = e % CB;
        cp_async16(stage + tile_slot<CB>(r, c), src + (size_t)r * Wp + c0 + c);
    }
    cp_async_commit();
    if (!C::TWG) load_twiddles<H>(tws, tw_g, tid, kThreads);
    const int g = tid / C::FT, t = tid % C::FT;
    float2* bz = xb + (2 * g) * C::SIG;
    float2* bw = xb + (2 * g + 1) * C::SIG;
    cp_async_wait<0>();
    __syncthreads();
    for (int j = 0; j < C::CPG; ++j) {
        const int c = g + j * C::G;
        const int kc = c0 + c;
        const bool spec = kc < Wc;
        // spectra of this column, requested before the transforms
        float2 L[8];
        float Kv[8];
        if (spec) {
            const float2* __restrict__ lcol = P.lamT + (size_t)kc * H;
            const float* __restrict__ kcol = P.kT + (size_t)kc * H;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                L[m] = lcol[t + m * C::FT];
                Kv[m] = kcol[t + m * C::FT];
            }
        }
        float2 v[8], u[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int r = t + m * C::FT;
            const float4 f = stage[tile_slot<CB>(r, c)];
            v[m] = make_float2(f.x, f.y);
            u[m] = make_float2(f.z, f.w);
        }
        if (C::ALIAS) __syncthreads();   // every column is in registers: the tile is free
        fft_group2<H, -1>(v, u, bz, bw, tw, t, g);
        if (spec) {
            // warm start: u0 = H x0 - d0 makes the first x-step return x0, whose
            // 2-D DFT is the first signal here (1/(HW) for the inverse)
            const float inv_hw = 1.0f / (float)(H * 2 * (Wc - 1));
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                // x^ = K (conj(Lambda) Z1^ + W^);  (A x)^ = Lambda x^
                const float2 xh = warm0 ? inv_hw * v[m] : Kv[m] * (cmulc(v[m], L[m]) + u[m]);
                v[m] = xh;
                u[m] = cmul(L[m], xh);
            }
        }
        fft_group2<H, 1>(v, u, bz, bw, tw, t, g);
        if (C::ALIAS) __syncthreads();   // every group is done exchanging through the tile
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int r = t + m * C::FT;
            stage[tile_slot<CB>(r, c)] = make_float4(v[m].x, v[m].y, u[m].x, u[m].y);
        }
    }
    __syncthreads();
    float4* __restrict__ dst = P.Sa;
    for (int e = tid; e < H * CB; e += kThreads) {
        const int r = e / CB, c = e % CB;
        dst[(size_t)r * Wp + c0 + c] = stage[tile_slot<CB>(r, c)];
    }
}

// ---------------------------------------------------------------------------
// Persistent column phase (configurations with one column per transform
// group): gridDim.x CTAs walk the launch's items (column block, slot), item
// it = slot * nblk + block. The tile of the next item is requested with
// cp.async into a second stage while the current one is transformed, so a
// CTA's loads overlap its own arithmetic. The work per item is that of
// col_phase.
// ---------------------------------------------------------------------------
template <int H, int CB>
__global__ void __launch_bounds__(kThreads, 3)
col_phase_pers(const ProbDesc* __restrict__ probs, SlotTable sl, int Wc, int Wp, const float2* __restrict__ tw_g,
               int nblk, int nitems) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using C = ColCfg<H, CB>;
    static_assert(C::ALIAS, "one column per transform group");
    extern __shared__ __align__(16) float4 smem4[];
    float2* tws = reinterpret_cast<float2*>(smem4 + 2 * H * CB);
    const float2* tw = C::TWG ? tw_g + pass_table_offset<H>() : tws;
    const int tid = threadIdx.x;
    const int g = tid / C::FT, t = tid % C::FT;
    // what an item needs: 0 nothing (no problem in the slot, or retired),
    // 1 zeros (first iteration from u0 = d0 = 0: x1 = 0), 2 the transforms
    auto classify = [&](int it, const ProbDesc*& q) -> int {
        const int pi = sl.map[it / nblk];
        if (pi < 0) return 0;
        q = probs + pi;
        if (q->ctl->active == 0) return 0;
        return (q->ctl->iter == 0 && !q->warm) ? 1 : 2;
    };
    auto request = [&](int it, const ProbDesc* q, float4* stage) {
        const int c0 = (it % nblk) * CB;
        const float4* __restrict__ src = q->Sb;
        for (int e = tid; e < H * CB; e += kThreads) {
            const int r = e / CB, c = e % CB;
            cp_async16(stage + tile_slot<CB>(r, c), src + (size_t)r * Wp + c0 + c);
        }
    };
    int it = blockIdx.x, cur = 0;
    const ProbDesc* Pc = nullptr;
    int mode = it < nitems ? classify(it, Pc) : 0;
    if (mode == 2) request(it, Pc, smem4);
    cp_async_commit();
    if (!C::TWG) load_twiddles<H>(tws, tw_g, tid, kThreads);
    for (; it < nitems; it += gridDim.x) {
        const int nx = it + gridDim.x;
        const ProbDesc* Pn = nullptr;
        const int mode_n = nx < nitems ? classify(nx, Pn) : 0;
        float4* stage = smem4 + cur * H * CB;
        if (mode_n == 2) request(nx, Pn, smem4 + (cur ^ 1) * H * CB);
        cp_async_commit();
        cp_async_wait<1>();          // this item's tile (the next one may still be in flight)
        __syncthreads();             // ... for every thread; the twiddles too
        const int c0 = (it % nblk) * CB;
        if (mode == 1) {
            for (int e = tid; e < H * CB; e += kThreads)
                Pc->Sa[(size_t)(e / CB) * Wp + c0 + e % CB] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (mode == 2) {
            const ProbDesc& P = *Pc;
            const bool warm0 = P.ctl->iter == 0 && P.warm == 1;   // the first x-step returns x0
            float2* bz = reinterpret_cast<float2*>(stage) + (2 * g) * C::SIG;
            float2* bw = reinterpret_cast<float2*>(stage) + (2 * g + 1) * C::SIG;
            const int kc = c0 + g;
            const bool spec = kc < Wc;
            float2 L[8];
            float Kv[8];
            if (spec) {
                const float2* __restrict__ lcol = P.lamT + (size_t)kc * H;
                const float* __restrict__ kcol = P.kT + (size_t)kc * H;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    L[m] = lcol[t + m * C::FT];
                    Kv[m] = kcol[t + m * C::FT];
                }
            }
            float2 v[8], u[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float4 f = stage[tile_slot<CB>(t + m * C::FT, g)];
                v[m] = make_float2(f.x, f.y);
                u[m] = make_float2(f.z, f.w);
            }
            __syncthreads();         // every column is in registers: the tile is free
            fft_group2<H, -1>(v, u, bz, bw, tw, t, g);
            if (spec) {
                const float inv_hw = 1.0f / (float)(H * 2 * (Wc - 1));
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    // x^ = K (conj(Lambda) Z1^ + W^);  (A x)^ = Lambda x^  (warm start: x0's DFT)
                    const float2 xh = warm0 ? inv_hw * v[m] : Kv[m] * (cmulc(v[m], L[m]) + u[m]);
                    v[m] = xh;
                    u[m] = cmul(L[m], xh);
                }
            }
            fft_group2<H, 1>(v, u, bz, bw, tw, t, g);
            __syncthreads();         // every group is done exchanging through the tile
#pragma unroll
            for (int m = 0; m < 8; ++m)
                stage[tile_slot<CB>(t + m * C::FT, g)] = make_float4(v[m].x, v[m].y, u[m].x, u[m].y);
            __syncthreads();
            float4* __restrict__ dst = P.Sa;
            for (int e = tid; e < H * CB; e += kThreads) {
                const int r = e / CB, c = e % CB;
                dst[(size_t)r * Wp + c0 + c] = stage[tile_slot<CB>(r, c)];
            }
        }
        __syncthreads();             // the stage is free before the next request into it
        cur ^= 1;
        mode = mode_n;
        Pc = Pn;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Shared pieces of the row phase.
// ---------------------------------------------------------------------------
// Rebuild the full row spectrum of the complex row x + i (A x) from the
// stored half spectra of the two real rows and return it in fft_group order.
template <int W>
__device__ __forceinline__ void load_row_xax(float2 (&v)[8], const float4* __restrict__ srow, int t) {
    constexpr int FT = W / 8;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int k = t + m * FT;
        if (k <= W / 2) {
            const float4 s = srow[k];             // (X, AX) at k
            v[m] = make_float2(s.x - s.w, s.y + s.z);
        } else {
            const float4 s = srow[W - k];         // X[k] = conj X[W-k], same for AX
            v[m] = make_float2(s.x + s.w, s.z - s.y);
        }
    }
}

// Split the spectrum P of p = a + i b (stored natural order in `row`) into
// the half spectra A[k] = (P[k] + conj P[W-k]) / 2, B[k] = (P[k] - conj P[W-k]) / 2i.
template <int W>
__device__ __forceinline__ void store_split(float4* __restrict__ drow, const float2* row, int t) {
    constexpr int FT = W / 8;
#pragma unroll
    for (int m = 0; m <= 4; ++m) {
        const int k = t + m * FT;
        if (k > W / 2) break;
        const float2 pk = row[swz(k)];
        const float2 pn = row[swz((W - k) & (W - 1))];
        const float2 a = 0.5f * make_float2(pk.x + pn.x, pk.y - pn.y);
        const float2 dd = make_float2(pk.x - pn.x, pk.y + pn.y);
        drow[k] = make_float4(a.x, a.y, 0.5f * dd.y, -0.5f * dd.x);
    }
}

// Block reduction of kNumPartials compensated FP32 sums: the running sums
// and their compensation terms are reduced separately in FP32 within each
// warp (FP64 arithmetic is slow on this part); across the warps, lane l of
// warp 0 adds series l (a running sum or a compensation term) in FP64, so
// the dependent FP64 chain is one add per warp, and thread 0 receives the
// block's totals (sum + compensation) in `out`.
template <int NT = kThreads>
__device__ __forceinline__ void block_reduce_comp(const CompSum (&a)[kNumPartials], float* red,
                                                  double (&out)[kNumPartials]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float s[kNumPartials], c[kNumPartials];
#pragma unroll
    for (int j = 0; j < kNumPartials; ++j) {
        s[j] = a[j].s;
        c[j] = a[j].c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s[j] += __shfl_down_sync(0xffffffffu, s[j], o);
            c[j] += __shfl_down_sync(0xffffffffu, c[j], o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < kNumPartials; ++j) {
            red[warp * 2 * kNumPartials + j] = s[j];
            red[warp * 2 * kNumPartials + kNumPartials + j] = c[j];
        }
    }
    __syncthreads();
    if (warp == 0) {
        double acc = 0.0;
        if (lane < 2 * kNumPartials) {
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) acc += (double)red[w * 2 * kNumPartials + lane];
        }
        const double tot = acc + __shfl_down_sync(0xffffffffu, acc, kNumPartials);   // lanes j < K
#pragma unroll
        for (int j = 0; j < kNumPartials; ++j) out[j] = __shfl_sync(0xffffffffu, tot, j);
    }
}

// Called by every thread of a CTA that finishes an iteration, with the
// CTA's partial sums in v (valid in thread 0): thread 0 publishes them; the
// last CTA of the problem to arrive reduces all slots (every thread takes a
// fixed strided share, then a fixed tree, so the order is reproducible),
// evaluates the stop rule of iteration k and advances the control block.
template <int NT>
__device__ void finish_iteration(const ProbDesc& P, int k, bool chk, bool nobj,
                                 const double (&v)[kNumPartials], int* n_active, int slot,
                                 const ProbDesc* __restrict__ probs, SlotTable sl) {
    __shared__ int s_last;
    __shared__ double s_red[NT / 32][kNumPartials];
    ProbCtl* ctl = P.ctl;
    const int tid = threadIdx.x;
    // the partial sums matter only where the stop rule or the objective is
    // evaluated; elsewhere the CTAs only count their arrival
    const bool need = chk || nobj;
    if (tid == 0) {
        if (need) {
#pragma unroll
            for (int j = 0; j < kNumPartials; ++j) P.partials[slot * kNumPartials + j] = v[j];
            __threadfence();
        }
        const unsigned prev = atomicAdd(&ctl->arrive, 1u);
        s_last = prev == (unsigned)(P.n_strips - 1);
    }
    __syncthreads();
    if (!s_last) return;
    double acc[kNumPartials] = {0.0};
    if (need) {
        __threadfence();
        const int nslots = P.n_slots > 0 ? P.n_slots : P.n_strips;
        for (int s = tid; s < nslots; s += NT) {
#pragma unroll
            for (int j = 0; j < kNumPartials; ++j) acc[j] += __ldcg(P.partials + s * kNumPartials + j);
        }
#pragma unroll
        for (int j = 0; j < kNumPartials; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_down_sync(0xffffffffu, acc[j], o);
        }
        if ((tid & 31) == 0) {
#pragma unroll
            for (int j = 0; j < kNumPartials; ++j) s_red[tid >> 5][j] = acc[j];
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < NT / 32; ++w) {
#pragma unroll
                for (int j = 0; j < kNumPartials; ++j) acc[j] += s_red[w][j];
            }
        }
    }
    if (tid != 0) return;
    bool done = ctl->status != 0;     // a timed-out copy marked the problem
    bool conv = false;
    if (nobj) {
        const double f = acc[0] + (double)P.lam * acc[1];
        if (!isfinite(f)) {
            ctl->status = kStatusNonFinite;
            done = true;
        }
        if (P.stop == kStopRelObj && ctl->have_obj) {
            const double ro = (f != 0.0) ? fabs(f - ctl->obj_prev) / fabs(f) : INFINITY;
            ctl->rel_obj = ro;
            if (ro < P.tol) conv = true;
        }
        ctl->obj_prev = f;
        ctl->obj = f;
        ctl->have_obj = 1;
        ctl->primal_res = sqrt(fmax(acc[4], 0.0));
    }
    if (chk) {
        if (!isfinite(acc[2]) || !isfinite(acc[3])) {
            ctl->status = kStatusNonFinite;
            done = true;
        }
        const double rx = (acc[2] > 0.0) ? sqrt(acc[3] / acc[2]) : INFINITY;
        ctl->rel_x = rx;
        if (rx < P.tol) conv = true;
    }
    ctl->iter = k;
    if (conv && !done) ctl->converged = 1;
    if (conv || done || k >= P.max_iters) {
        const unsigned long long now = device_clock_ns();
        ctl->active = 0;
        ctl->t_done = now;
        atomicSub(n_active, 1);
        // hand this slot to the next queued problem that is still active
        // (bounded: every pass consumes one queue entry)
        int nx = atomicAdd(sl.queue, 1);
        while (nx < sl.pool && probs[nx].ctl->active == 0) nx = atomicAdd(sl.queue, 1);
        sl.map[blockIdx.y] = nx < sl.pool ? nx : -1;
        if (nx < sl.pool) probs[nx].ctl->t_start = now;
    }
    ctl->arrive = 0u;
}

// ---------------------------------------------------------------------------
// TV row phase. Grid: (H / R, slots). CTA = strip of R rows of one problem;
// the inverse transforms also cover one halo row above and below (the
// forward differences and their adjoints reach one row each way).
//
// Data movement: at entry the walk's rows go to L2 in bulk; every
// half-spectrum row of the strip (R + 2 rows) is requested with cp.async into
// the row buffers by the transform group that will transform it (one
// cp.async group per round of transforms); and the per-pixel inputs of the
// first D rows of the walk (d2, d1, M^T y) go into a per-thread ring of D row
// slots. Each walk step consumes one slot and refills it with the row D ahead,
// so D rows of loads stay in flight behind the arithmetic; x_prev, needed on
// check iterations only, is read one row ahead into registers.
//
// The walk needs no block barrier: warp w owns the contiguous columns
// [w W/NWARP, (w+1) W/NWARP) and walks its rows on its own (lane by lane at
// stride 32, or as pairs of adjacent columns when the warp owns at least 64).
// The left neighbour's delta_h comes by shuffle from the next lower lane; the
// first lane recomputes the pixel left of the chunk itself (its d2 is in the
// ring's halo entry). x values of the neighbouring warps' boundary columns
// are captured in registers before any warp overwrites its rows with p.
// ---------------------------------------------------------------------------
template <int W, int R, int D, int NT>
struct RowCfg {
    static constexpr int FT = W / 8;
    static constexpr int G = NT / FT;                              // row transforms in flight
    static_assert(G >= 1 && NT % FT == 0, "block too small for one row transform");
    static constexpr int NB = R + 2;                               // buffer rows
    static constexpr int NR = (R + 2 + 2 * G - 1) / (2 * G);       // rounds of inverse transforms
    static constexpr int ROW = W + 2;                              // float2 per buffer row (raw spectrum fits)
    static constexpr int RAW = W / 2 + 1;                          // float4 per half-spectrum row
    static constexpr int NWARP = NT / 32;
    static constexpr int CW = W / NWARP;                           // columns per warp
    static constexpr int CPT = CW >= 32 ? CW / 32 : 1;              // columns per thread
    static constexpr int SLOT = 4 * W + 2 * NWARP;                 // floats per ring slot
    static constexpr int DR = D > 0 ? D : 1;                       // ring slots addressed (D = 0: none used)
    // warps of at least 64 columns walk them as pairs of adjacent columns
    // (lane l of pair p: columns w CW + 64 p + 2 l, + 1): 16-byte ring copies,
    // global accesses and shared-memory reads and writes
    static constexpr bool PAIRS = CW >= 64 && D > 0;
    static constexpr int NPAIR = CPT / 2;
    static_assert(!PAIRS || (SLOT * 4) % 16 == 0, "16-byte ring copies need 16-byte slots");
    static_assert(RAW * 16 <= ROW * 8, "raw row must fit a buffer row");
    static_assert(R + 2 <= 32, "boundary capture holds one row per lane");
    static_assert(((size_t)NB * ROW * 8 + (size_t)W * 8) % 16 == 0, "ring alignment");
    static_assert(((size_t)NB * ROW * 8 + (size_t)W * 8 + (size_t)D * SLOT * 4) % 8 == 0, "scratch alignment");
    static constexpr size_t SMEM = (size_t)NB * ROW * sizeof(float2) + (size_t)W * sizeof(float2)
                                 + (size_t)D * SLOT * sizeof(float) + NWARP * 2 * kNumPartials * sizeof(float);
    // CTAs per SM the registers are sized for (128-thread CTAs without the
    // ring fit a fifth CTA in shared memory)
    static constexpr int MINB = NT == 128 ? (D == 0 ? 5 : 4) : (NT == 64 ? 8 : 2);
};

// ANISO: anisotropic TV (soft threshold per difference component)
template <int W, int R, int D, int NT, bool ANISO = false>
__global__ void __launch_bounds__(NT, (RowCfg<W, R, D, NT>::MINB))
row_phase_tv(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g,
             int* __restrict__ n_active) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using C = RowCfg<W, R, D, NT>;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    ProbCtl* ctl = P.ctl;
    if (ctl->active == 0) return;
    const int k = ctl->iter + 1;                 // iteration being completed
    const bool first = k == 1;                   // x_prev = 0 (no earlier iterate)
    const bool cold = first && !P.warm;          // d1 = d2 = 0 (u0 = d0 = 0)
    const bool chk = is_check_iter(P, k), sprev = store_prev_iter(P, k), nobj = need_obj_iter(P, k);
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = buf + C::NB * C::ROW;
    float* ring = reinterpret_cast<float*>(tw + W);
    double* red = reinterpret_cast<double*>(ring + D * C::SLOT);
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int r0 = blockIdx.x * R;
    const bool colthr = lane < C::CW;            // narrow rows leave some lanes idle
    const int cbase = wid * C::CW + lane;        // column j of this thread: cbase + 32 j
    const int chalo = (wid * C::CW - 1) & (W - 1);
    const float2* __restrict__ d2in = reinterpret_cast<const float2*>(P.d2 + ((k + 1) & 1) * P.d2_stride);
    float2* __restrict__ d2out = reinterpret_cast<float2*>(P.d2 + (k & 1) * P.d2_stride);

    // ring slot of walk row i: d2 (float2 per column), d1, M^T y, and per
    // warp the d2 of the pixel left of its chunk (x_prev, read on check
    // iterations only, goes through registers one row ahead)
    auto issue = [&](int i) {
        if (D > 0 && i <= R && colthr) {
            const int q = (r0 - 1 + i + H) & (H - 1);
            float* slot = ring + (i % C::DR) * C::SLOT;
            if constexpr (C::PAIRS) {
#pragma unroll
                for (int pp = 0; pp < C::NPAIR; ++pp) {
                    const int c = wid * C::CW + 64 * pp + 2 * lane;
                    const size_t pix = (size_t)q * W + c;
                    if (!cold) cp_async16(slot + 2 * c, d2in + pix);
                    if (i >= 1) {
                        if (!cold) cp_async8(slot + 2 * W + c, P.d1 + pix);
                        cp_async8(slot + 3 * W + c, P.ybar + pix);
                    }
                }
            } else {
#pragma unroll
            for (int j = 0; j < C::CPT; ++j) {
                const int c = cbase + 32 * j;
                const size_t pix = (size_t)q * W + c;
                if (!cold) cp_async8(slot + 2 * c, d2in + pix);
                if (i >= 1) {
                    if (!cold) cp_async4(slot + 2 * W + c, P.d1 + pix);
                    cp_async4(slot + 3 * W + c, P.ybar + pix);
                }
            }
            }
            if (lane == 0 && !cold) cp_async8(slot + 4 * W + 2 * wid, d2in + (size_t)q * W + chalo);
        }
        cp_async_commit();   // possibly empty: keeps one group per walk row
    };

    // (0) requests: the walk's rows go to L2 in bulk (they are consumed after
    // the inverse transforms), the half spectra of rows r0-1 .. r0+R into
    // shared memory, then the first D walk rows into the ring. The L2
    // prefetches are spread over lane 0 of the warps after the first, whose
    // thread 0 issues the spectrum rows' bulk copies (the first transforms
    // wait for those) without queueing behind them.
    {
        constexpr int NPF = C::NWARP > 1 ? C::NWARP - 1 : 1;   // prefetching warps
        const int pw = C::NWARP > 1 ? wid - 1 : 0;
        if (lane == 0 && pw >= 0) {
            if (!cold && pw == 0) prefetch_l2(d2in + (size_t)((r0 - 1 + H) & (H - 1)) * W, W * sizeof(float2));
            for (int i = pw; i < R; i += NPF) {
                if (!cold) {
                    prefetch_l2(d2in + (size_t)(r0 + i) * W, W * sizeof(float2));
                    prefetch_l2(P.d1 + (size_t)(r0 + i) * W, W * sizeof(float));
                    if (chk && !first) prefetch_l2(P.xprev + (size_t)(r0 + i) * W, W * sizeof(float));
                }
                prefetch_l2(P.ybar + (size_t)(r0 + i) * W, W * sizeof(float));
            }
        }
    }
    const int g = tid / C::FT, t = tid % C::FT;
    constexpr int NR = C::NR;
    // The half-spectrum rows go to shared memory by bulk copies (one per row,
    // RAW float4 = the buffer row's bytes), issued by one thread; the rows of
    // round rd of transform group g complete on mbarrier g NR + rd, so a
    // round starts as soon as its own two rows have landed.
    __shared__ __align__(8) unsigned long long spec_bar[C::G * C::NR];
    if (tid == 0) {
        for (int b = 0; b < C::G * NR; ++b) mbar_init1(smem_u32(&spec_bar[b]));
        mbar_init_fence();
        for (int gg = 0; gg < C::G; ++gg) {
            for (int rd = 0; rd < NR; ++rd) {
                const int i0 = gg + 2 * C::G * rd, i1 = i0 + C::G;
                if (i0 >= R + 2) continue;
                const uint32_t bar = smem_u32(&spec_bar[gg * NR + rd]);
                mbar_expect_tx(bar, (uint32_t)((i1 < R + 2 ? 2 : 1) * C::RAW * sizeof(float4)));
                // (test hook: the first round of group 0 gets no copy, its wait runs out)
                if (P.test_stall && gg == 0 && rd == 0) continue;
                for (int i = i0; i < R + 2 && i <= i1; i += C::G) {
                    const int q = (r0 - 1 + i + H) & (H - 1);
                    bulk_copy_g2s(buf + i * C::ROW, P.Sa + (size_t)q * Wp, C::RAW * sizeof(float4), bar);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) issue(i);
    load_twiddles<W>(tw, tw_g, tid, NT);
    __syncthreads();             // the twiddles

    // (1) x + i A x on buffer rows 0..R+1 = image rows r0-1..r0+R: inverse row
    // DFTs, two rows per group at a time (interleaved: twice the independent
    // work between the group's barriers)
#pragma unroll 1
    for (int rd = 0; rd < NR; ++rd) {
        const int i = g + 2 * C::G * rd;
        if (i >= R + 2) continue;
        // this round's rows have landed (every thread of the group waits itself)
        if (!mbar_wait_bounded(smem_u32(&spec_bar[g * NR + rd]), 0u) && t == 0)
            atomicExch(&ctl->status, kStatusTimeout);
        float2* row = buf + i * C::ROW;
        float2 v[8];
        load_row_xax<W>(v, reinterpret_cast<const float4*>(row), t);
        if (i + C::G < R + 2) {
            float2* row2 = row + C::G * C::ROW;
            float2 u[8];
            load_row_xax<W>(u, reinterpret_cast<const float4*>(row2), t);
            fft_group2<W, 1>(v, u, row, row2, tw, t, g);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                row[swz(t + m * C::FT)] = v[m];
                row2[swz(t + m * C::FT)] = u[m];
            }
        } else {
            fft_group<W, 1>(v, row, tw, t, g);
#pragma unroll
            for (int m = 0; m < 8; ++m) row[swz(t + m * C::FT)] = v[m];
        }
    }
    __syncthreads();
    // x of the neighbouring warps' boundary columns, one row per lane
    float xnb_right = 0.f, xnb_left = 0.f;
    if (lane < R + 2) {
        xnb_right = buf[lane * C::ROW + swz((wid * C::CW + C::CW) & (W - 1))].x;
        xnb_left = buf[lane * C::ROW + swz(chalo)].x;
    }
    __syncthreads();             // nobody overwrites a row before every warp captured

    // (2) proxes and dual updates, each warp walking down its columns
    const float tau = P.tau, gam = P.gamma, mu1 = P.mu1, inv1 = P.inv1pmu1;
    constexpr bool aniso = ANISO;
    CompSum s_data, s_reg, s_xx, s_dxx, s_pr;
    float dvprev[C::CPT];
    const bool need_xp = chk && !first;
    float xpn[C::CPT];               // x_prev of the next owned row
    // column of entry j of the thread's per-column arrays
    auto colj = [&](int j) {
        return C::PAIRS ? wid * C::CW + 64 * (j >> 1) + 2 * lane + (j & 1) : cbase + 32 * j;
    };
#pragma unroll
    for (int j = 0; j < C::CPT; ++j) {
        dvprev[j] = 0.f;
        xpn[j] = (need_xp && colthr) ? P.xprev[(size_t)r0 * W + colj(j)] : 0.f;
    }
    for (int i = 0; i <= R; ++i) {
        const int q = (r0 - 1 + i + H) & (H - 1);
        const bool owned = i >= 1;
        float xpc[C::CPT];
#pragma unroll
        for (int j = 0; j < C::CPT; ++j) xpc[j] = xpn[j];
        if (need_xp && owned && i < R && colthr) {
            // requested a row ahead (row q + 1 is still unwritten by this iteration)
#pragma unroll
            for (int j = 0; j < C::CPT; ++j) xpn[j] = P.xprev[(size_t)(q + 1) * W + colj(j)];
        }
        if (D > 0) cp_async_wait<(D > 0 ? D - 1 : 0)>();   // this thread's copies of walk row i have landed
        const float* slot = ring + (i % C::DR) * C::SLOT;
        const float xr_nb = __shfl_sync(0xffffffffu, xnb_right, i);
        const float xl_nb = __shfl_sync(0xffffffffu, xnb_left, i);
        const float xl_nb_dn = __shfl_sync(0xffffffffu, xnb_left, i + 1);
        float dhcur[C::CPT], dvcur[C::CPT], z1cur[C::CPT];
#pragma unroll
        for (int j = 0; j < C::CPT; ++j) dhcur[j] = dvcur[j] = z1cur[j] = 0.f;
        float dh_halo = 0.f;
        if constexpr (C::PAIRS) {
            // x, A x of both columns of each pair (row i) and x below them (row
            // i + 1): one 16-byte read each. swz keeps an even/odd column pair
            // together (positions swz(c) ^ {0, 1}); bit 3 of c says which is first.
            float4 xa[C::NPAIR];
            float2 xdn[C::NPAIR];
#pragma unroll
            for (int pp = 0; pp < C::NPAIR; ++pp) {
                const int c = wid * C::CW + 64 * pp + 2 * lane;
                const int base = swz(c) & ~1;
                const bool sw = (c >> 3) & 1;
                const float4 t4 = *reinterpret_cast<const float4*>(buf + i * C::ROW + base);
                const float4 u4 = *reinterpret_cast<const float4*>(buf + (i + 1) * C::ROW + base);
                xa[pp] = sw ? make_float4(t4.z, t4.w, t4.x, t4.y) : t4;
                xdn[pp] = sw ? make_float2(u4.z, u4.x) : make_float2(u4.x, u4.z);
            }
            // x right of each pair: the next lane's first column, for lane 31 the
            // next pair's lane 0 or, after the last pair, the next warp's first
            float xrp[C::NPAIR];
#pragma unroll
            for (int pp = 0; pp < C::NPAIR; ++pp) {
                const float nx = __shfl_down_sync(0xffffffffu, xa[pp].x, 1);
                const float wr = pp + 1 < C::NPAIR ? __shfl_sync(0xffffffffu, xa[pp + 1 < C::NPAIR ? pp + 1 : pp].x, 0)
                                                   : xr_nb;
                xrp[pp] = lane == 31 ? wr : nx;
            }
#pragma unroll
            for (int pp = 0; pp < C::NPAIR; ++pp) {
                const int c = wid * C::CW + 64 * pp + 2 * lane;
                const size_t pix = (size_t)q * W + c;
                const float4 dd = cold ? make_float4(0.f, 0.f, 0.f, 0.f)
                                       : *reinterpret_cast<const float4*>(slot + 2 * c);
                const float xs[2] = {xa[pp].x, xa[pp].z}, axs[2] = {xa[pp].y, xa[pp].w};
                const float xrs[2] = {xa[pp].z, xrp[pp]}, xds[2] = {xdn[pp].x, xdn[pp].y};
                const float ddh[2] = {dd.x, dd.z}, ddv[2] = {dd.y, dd.w};
                float nh[2], nv[2];
                float prp = 0.f;         // the pair's share of ||d_k - d_{k-1}||^2
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    // D_i x, u2 = prox(D_i x - d2, lambda/mu2), d2 <- d2 - (D_i x - u2),
                    // delta = u2 + d2  (Alg. 3 lines 3-5, 9-11; as in the single-column walk)
                    const float gh = xrs[e] - xs[e], gv = xds[e] - xs[e];
                    const float sh = gh - ddh[e], sv = gv - ddv[e];
                    float uh, uv;
                    tv_prox(sh, sv, tau, aniso, uh, uv);
                    nh[e] = uh - sh;
                    nv[e] = uv - sv;
                    dhcur[2 * pp + e] = uh + nh[e];
                    dvcur[2 * pp + e] = uv + nv[e];
                    if (owned && nobj) {
                        s_reg.add(tv_norm(gh, gv, aniso));
                        const float eh = nh[e] - ddh[e], ev = nv[e] - ddv[e];
                        prp = fmaf(eh, eh, fmaf(ev, ev, prp));
                    }
                }
                if (owned) {
                    *reinterpret_cast<float4*>(d2out + pix) = make_float4(nh[0], nv[0], nh[1], nv[1]);
                    const float2 d1p = cold ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(slot + 2 * W + c);
                    const float2 ybp = *reinterpret_cast<const float2*>(slot + 3 * W + c);
                    const float d1s[2] = {d1p.x, d1p.y}, ybs[2] = {ybp.x, ybp.y};
                    float nd1[2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        // mask prox (eq. new_line) and d1 update (Alg. 3 line 8)
                        const float s1 = axs[e] - d1s[e];
                        const bool obs = is_observed(ybs[e]);
                        const float u1 = obs ? fmaf(mu1, s1, ybs[e]) * inv1 : s1;
                        nd1[e] = d1s[e] - (axs[e] - u1);
                        z1cur[2 * pp + e] = u1 + nd1[e];
                        if (nobj) {
                            if (obs) {
                                const float er = axs[e] - ybs[e];
                                s_data.add(0.5f * er * er);
                            }
                            const float e1 = nd1[e] - d1s[e];
                            prp = fmaf(e1, e1, prp);
                        }
                        if (chk) {
                            const float dx = first ? xs[e] : xs[e] - xpc[2 * pp + e];
                            s_dxx.add(dx * dx);
                            s_xx.add(xs[e] * xs[e]);
                        }
                    }
                    *reinterpret_cast<float2*>(P.d1 + pix) = make_float2(nd1[0], nd1[1]);
                    if (sprev) *reinterpret_cast<float2*>(P.xprev + pix) = make_float2(xs[0], xs[1]);
                    if (nobj) s_pr.add(prp);
                }
            }
            if (lane == 0 && owned) {
                // delta_h of the pixel left of the chunk (its owner updates its d2)
                const float xh = xl_nb;
                const float xhr = xa[0].x;
                const float2 dd = cold ? make_float2(0.f, 0.f) : *reinterpret_cast<const float2*>(slot + 4 * W + 2 * wid);
                const float sh = (xhr - xh) - dd.x, sv = (xl_nb_dn - xh) - dd.y;
                float uh, uv;
                tv_prox(sh, sv, tau, aniso, uh, uv);
                dh_halo = 2.f * uh - sh;
            }
            issue(i + D);            // slot (i % D) is consumed: refill it D rows ahead
            // delta_h left of each column: the pair's own first column for the
            // second; the previous lane (pair) or the chunk's halo for the first
            float dhl[C::CPT];
#pragma unroll
            for (int pp = 0; pp < C::NPAIR; ++pp) {
                const float up = __shfl_up_sync(0xffffffffu, dhcur[2 * pp + 1], 1);
                const float wr = pp > 0 ? __shfl_sync(0xffffffffu, dhcur[pp > 0 ? 2 * pp - 1 : 1], 31) : dh_halo;
                dhl[2 * pp] = lane == 0 ? wr : up;
                dhl[2 * pp + 1] = dhcur[2 * pp];
            }
            __syncwarp();            // every lane has read rows i, i + 1 before row i is overwritten
            if (owned) {
                // w = gamma (Dh^T delta_h + Dv^T delta_v); p = zeta1 + i w over row i
#pragma unroll
                for (int pp = 0; pp < C::NPAIR; ++pp) {
                    const int c = wid * C::CW + 64 * pp + 2 * lane;
                    const float w0 = gam * ((dhl[2 * pp] - dhcur[2 * pp]) + (dvprev[2 * pp] - dvcur[2 * pp]));
                    const float w1 =
                        gam * ((dhl[2 * pp + 1] - dhcur[2 * pp + 1]) + (dvprev[2 * pp + 1] - dvcur[2 * pp + 1]));
                    const bool sw = (c >> 3) & 1;
                    *reinterpret_cast<float4*>(buf + i * C::ROW + (swz(c) & ~1)) =
                        sw ? make_float4(z1cur[2 * pp + 1], w1, z1cur[2 * pp], w0)
                           : make_float4(z1cur[2 * pp], w0, z1cur[2 * pp + 1], w1);
                }
            }
#pragma unroll
            for (int j = 0; j < C::CPT; ++j) dvprev[j] = dvcur[j];
            continue;
        }
        if (colthr) {
#pragma unroll
            for (int j = 0; j < C::CPT; ++j) {
                const int c = cbase + 32 * j;
                const float2 z = buf[i * C::ROW + swz(c)];
                const float x = z.x, ax = z.y;
                const bool last_col = (lane == C::CW - 1 || lane == 31) && j == C::CPT - 1;
                const float xr = last_col ? xr_nb : buf[i * C::ROW + swz(c + 1)].x;
                const float xd = buf[(i + 1) * C::ROW + swz(c)].x;
                // D_i x (forward periodic differences)
                const float gh = xr - x, gv = xd - x;
                const size_t pix = (size_t)q * W + c;
                const float2 dd = cold ? make_float2(0.f, 0.f)
                                       : (D > 0 ? *reinterpret_cast<const float2*>(slot + 2 * c) : d2in[pix]);
                // u2 = prox(D_i x - d2, lambda/mu2)  (Alg. 3 line 10)
                const float sh = gh - dd.x, sv = gv - dd.y;
                float uh, uv;
                tv_prox(sh, sv, tau, aniso, uh, uv);
                // d2 <- d2 - (D_i x - u2)  (Alg. 3 line 11)
                const float nh = uh - sh, nv = uv - sv;
                // delta = u2 + d2 for the next x-step (Alg. 3 lines 3-5)
                dhcur[j] = uh + nh;
                dvcur[j] = uv + nv;
                z1cur[j] = 0.f;
                if (owned) {
                    d2out[pix] = make_float2(nh, nv);
                    // u1 = (M^T M + mu1 I)^{-1} (M^T y + mu1 (A x - d1))  (eq. new_line)
                    const float dd1 = cold ? 0.f : (D > 0 ? slot[2 * W + c] : P.d1[pix]);
                    const float yb = D > 0 ? slot[3 * W + c] : P.ybar[pix];
                    const float s1 = ax - dd1;
                    const bool obs = is_observed(yb);
                    const float u1 = obs ? fmaf(mu1, s1, yb) * inv1 : s1;
                    // d1 <- d1 - (A x - u1)  (Alg. 3 line 8)
                    const float nd1 = dd1 - (ax - u1);
                    P.d1[pix] = nd1;
                    z1cur[j] = u1 + nd1;
                    if (nobj) {
                        if (obs) {
                            const float e = ax - yb;
                            s_data.add(0.5f * e * e);
                        }
                        s_reg.add(tv_norm(gh, gv, aniso));
                        // d_k - d_{k-1} of both splits (Alg. 2: H z - u)
                        const float e1 = nd1 - dd1, eh = nh - dd.x, ev = nv - dd.y;
                        s_pr.add(fmaf(e1, e1, fmaf(eh, eh, ev * ev)));
                    }
                    if (chk) {
                        const float dx = first ? x : x - xpc[j];
                        s_dxx.add(dx * dx);
                        s_xx.add(x * x);
                    }
                    if (sprev) P.xprev[pix] = x;
                }
            }
            if (lane == 0 && owned) {
                // delta_h of the pixel left of the chunk (its owner updates its d2)
                const float xh = xl_nb;
                const float xhr = buf[i * C::ROW + swz(wid * C::CW)].x;
                const float2 dd = cold ? make_float2(0.f, 0.f)
                                        : (D > 0 ? *reinterpret_cast<const float2*>(slot + 4 * W + 2 * wid)
                                                 : d2in[(size_t)q * W + chalo]);
                const float sh = (xhr - xh) - dd.x, sv = (xl_nb_dn - xh) - dd.y;
                float uh, uv;
                tv_prox(sh, sv, tau, aniso, uh, uv);
                dh_halo = 2.f * uh - sh;
            }
        }
        issue(i + D);                // slot (i % D) is consumed: refill it D rows ahead
        // left neighbours' delta_h within the warp
        float dhl[C::CPT];
#pragma unroll
        for (int j = 0; j < C::CPT; ++j) {
            const float up = __shfl_up_sync(0xffffffffu, dhcur[j], 1);
            const float wrap = j > 0 ? __shfl_sync(0xffffffffu, dhcur[j > 0 ? j - 1 : 0], 31) : dh_halo;
            dhl[j] = lane == 0 ? wrap : up;
        }
        __syncwarp();                // every lane has read row i before it is overwritten
        if (owned && colthr) {
            // w = gamma (Dh^T delta_h + Dv^T delta_v): adjoint of forward differences
#pragma unroll
            for (int j = 0; j < C::CPT; ++j) {
                const int c = cbase + 32 * j;
                const float w = gam * ((dhl[j] - dhcur[j]) + (dvprev[j] - dvcur[j]));
                buf[i * C::ROW + swz(c)] = make_float2(z1cur[j], w);
            }
        }
#pragma unroll
        for (int j = 0; j < C::CPT; ++j) dvprev[j] = dvcur[j];
    }
    cp_async_wait<0>();              // only empty groups remain; nothing left in flight
    __syncthreads();

    // (3) block partial sums (published after the transforms below), only
    // where the stop rule or the objective is evaluated
    double part[kNumPartials] = {0.0};
    if (nobj || chk) {
        const CompSum acc[kNumPartials] = {s_data, s_reg, s_xx, s_dxx, s_pr};
        block_reduce_comp<NT>(acc, reinterpret_cast<float*>(red), part);
    }

    // (4) forward row DFTs of p = zeta1 + i w on rows 1..R and split, two
    // rows per group at a time
    for (int i = 1 + g; i <= R; i += 2 * C::G) {
        float2* row = buf + i * C::ROW;
        float2 v[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = row[swz(t + m * C::FT)];
        if (i + C::G <= R) {
            float2* row2 = row + C::G * C::ROW;
            float2 u[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) u[m] = row2[swz(t + m * C::FT)];
            fft_group2<W, -1>(v, u, row, row2, tw, t, g);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                row[swz(t + m * C::FT)] = v[m];
                row2[swz(t + m * C::FT)] = u[m];
            }
            group_sync<W>(g);        // the split reads this group's rows only
            store_split<W>(P.Sb + (size_t)(r0 - 1 + i) * Wp, row, t);
            store_split<W>(P.Sb + (size_t)(r0 - 1 + i + C::G) * Wp, row2, t);
        } else {
            fft_group<W, -1>(v, row, tw, t, g);
#pragma unroll
            for (int m = 0; m < 8; ++m) row[swz(t + m * C::FT)] = v[m];
            group_sync<W>(g);
            store_split<W>(P.Sb + (size_t)(r0 - 1 + i) * Wp, row, t);
        }
    }

    // (5) the last CTA of the problem evaluates the stop rule; done last so
    // that the memory fence it needs does not hold up the transforms
    finish_iteration<NT>(P, k, chk, nobj, part, n_active, blockIdx.x, probs, sl);
}

// ---------------------------------------------------------------------------
// Final iterate: x from the last column-phase output by inverse row DFTs.
// Grid: (H / G, problems) with G rows per CTA.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
finalize_x(const ProbDesc* __restrict__ probs, float* const* __restrict__ xout, int H, int Wp,
           const float2* __restrict__ tw_g) {
    constexpr int FT = W / 8, G = kThreads / FT, ROW = W;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = buf + G * ROW;
    const ProbDesc& P = probs[blockIdx.y];
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    load_twiddles<W>(tw, tw_g, tid, kThreads);
    __syncthreads();
    const int q = blockIdx.x * G + g;
    float2 v[8];
    if (q < H) {
        load_row_xax<W>(v, P.Sa + (size_t)q * Wp, t);
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = make_float2(0.f, 0.f);
    }
    fft_group<W, 1>(v, buf + g * ROW, tw, t, g);
    if (q < H) {
        float* xo = xout[blockIdx.y] + (size_t)q * W;
#pragma unroll
        for (int m = 0; m < 8; ++m) xo[t + m * FT] = v[m].x;
    }
}

// ---------------------------------------------------------------------------
// Warm start: the row-DFTs of a real starting image x0 (first signal; the
// second signal is zero) into Sb, where the first iteration's column phase
// finds them. Grid: ceil(H / G) CTAs, one row per group of W/8 threads.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
warm_rows(const float* __restrict__ x0, float4* __restrict__ Sb, int H, int Wp, const float2* __restrict__ tw_g) {
    constexpr int FT = W / 8, G = kThreads / FT, ROW = W;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = buf + G * ROW;
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    load_twiddles<W>(tw, tw_g, tid, kThreads);
    __syncthreads();
    const int q = blockIdx.x * G + g;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = make_float2(q < H ? x0[(size_t)q * W + t + m * FT] : 0.f, 0.f);
    float2* row = buf + g * ROW;
    fft_group<W, -1>(v, row, tw, t, g);
#pragma unroll
    for (int m = 0; m < 8; ++m) row[swz(t + m * FT)] = v[m];
    group_sync<W>(g);                // the split reads this group's row only
    if (q < H) store_split<W>(Sb + (size_t)q * Wp, row, t);
}

}  // namespace admm
