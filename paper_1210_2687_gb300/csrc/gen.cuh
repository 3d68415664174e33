// gen.cuh -- the iteration on exact domains whose sides are not both powers
// of two (Sec. IV-A: the unknown domain only has to hold the image and the
// kernel support, so its size is free). Sides m 2^k, m in {1, 3, 5} (gfft.cuh).
//
// One TV-MD or FA-MD iteration (Algorithm 3 with eq. new_line; Algorithm 2
// with H2 = P) runs as
//   gcol_phase   the column phase: forward column DFTs of the row spectra of
//                (zeta1, w), x^ = K (conj(Lambda) Z1^ + W^), (A x)^ = Lambda x^,
//                inverse column DFTs (as col_phase in kernels.cuh)
//   grow_inv     inverse row DFTs -> x, A x; mask prox and d1 update (eq.
//                new_line, Alg. 3 line 8); x and zeta1 = u1 + d1 to the scratch
//                planes (as haar_row_inverse)
//   regulariser  TV: tv_tile (cg.cuh); frame: haar_analysis, haar_synthesis
//   grow_fwd     forward row DFTs of zeta1 + i w, split into half spectra
// with the same buffers, descriptors and reductions as the power-of-two
// kernels; the half spectrum k = 0..W/2 of two real rows is stored as float4.
#pragma once
#include "cg.cuh"
#include "gfft.cuh"

namespace admm {

// rows per CTA of the generic row kernels (one row per transform group)
template <int W> struct GRow {
    static constexpr int T = GShape<W>::T, E = GShape<W>::E;
    static constexpr int G = kThreads / T;
    static_assert(G >= 1 && kThreads % T == 0, "row length");
};

// ---------------------------------------------------------------------------
// column phase. Grid (Wp / CB, slots), CB = columns per CTA = one per group.
// The H x CB tile, the twiddles and the spectra Lambda, K of the CB columns
// are requested with cp.async at entry (the spectra are read from shared
// memory between the transforms instead of from global memory there); once
// every group holds its column in registers the tile doubles as the groups'
// exchange buffers.
// ---------------------------------------------------------------------------
template <int H> struct GCol {
    static constexpr int T = GShape<H>::T, E = GShape<H>::E;
    static constexpr int CB = kThreads / T;
    static constexpr size_t SMEM = (size_t)H * CB * sizeof(float4) + (size_t)H * sizeof(float2)
                                 + (size_t)H * CB * (sizeof(float2) + sizeof(float));
};

template <int H>
__global__ void __launch_bounds__(kThreads)
gcol_phase(const ProbDesc* __restrict__ probs, SlotTable sl, int Wc, int Wp, const float2* __restrict__ twH) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using C = GCol<H>;
    constexpr int CB = C::CB, T = C::T, E = C::E;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const int c0 = blockIdx.x * CB;
    const bool it0 = P.ctl->iter == 0;
    if (it0 && !P.warm) {
        // first iteration from u0 = d0 = 0: the right-hand side is zero, so x1 = 0
        for (int e = threadIdx.x; e < H * CB; e += kThreads)
            P.Sa[(size_t)(e / CB) * Wp + c0 + e % CB] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const bool warm0 = it0 && P.warm == 1;       // the first x-step returns x0
    extern __shared__ __align__(16) float4 gsm4[];
    float4* stage = gsm4;                        // H x CB, row-major
    float2* tw = reinterpret_cast<float2*>(stage + H * CB);
    float2* lks = tw + H;                        // Lambda of the CB columns (H each), then K
    float* kks = reinterpret_cast<float*>(lks + H * CB);
    const int tid = threadIdx.x, g = tid / T, t = tid % T;
    for (int e = tid; e < H * CB; e += kThreads) {
        const int r = e / CB, c = e % CB;
        cp_async16(stage + e, P.Sb + (size_t)r * Wp + c0 + c);
    }
    for (int e = tid; e < H / 2; e += kThreads) cp_async16(tw + 2 * e, twH + 2 * e);
#pragma unroll 1
    for (int c = 0; c < CB; ++c) {
        if (c0 + c >= Wc) break;
        const float2* __restrict__ lcol = P.lamT + (size_t)(c0 + c) * H;
        const float* __restrict__ kcol = P.kT + (size_t)(c0 + c) * H;
        for (int e = tid; e < H / 2; e += kThreads) cp_async16(lks + c * H + 2 * e, lcol + 2 * e);
        for (int e = tid; e < H / 4; e += kThreads) cp_async16(kks + c * H + 4 * e, kcol + 4 * e);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int kc = c0 + g;
    const bool spec = kc < Wc;
    float2 v[E], u[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const float4 f = stage[(t + T * e) * CB + g];
        v[e] = make_float2(f.x, f.y);
        u[e] = make_float2(f.z, f.w);
    }
    __syncthreads();                             // every column is in registers: the tile is free
    float2* bv = reinterpret_cast<float2*>(stage) + (size_t)(2 * g) * H;
    float2* bu = bv + H;
    gfft<H, -1>(v, t, g, tw, bv);
    gfft<H, -1>(u, t, g, tw, bu);
    if (spec) {
        const float2* lcol = lks + g * H;
        const float* kcol = kks + g * H;
        const float inv_hw = 1.0f / (float)(H * 2 * (Wc - 1));
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 L = lcol[t + T * e];
            // x^ = K (conj(Lambda) Z1^ + W^);  (A x)^ = Lambda x^  (warm start: x0's DFT)
            const float2 xh = warm0 ? inv_hw * v[e] : kcol[t + T * e] * (cmulc(v[e], L) + u[e]);
            v[e] = xh;
            u[e] = cmul(L, xh);
        }
    }
    gfft<H, 1>(v, t, g, tw, bv);
    gfft<H, 1>(u, t, g, tw, bu);
    __syncthreads();                             // every group is done exchanging through the tile
#pragma unroll
    for (int e = 0; e < E; ++e) stage[(t + T * e) * CB + g] = make_float4(v[e].x, v[e].y, u[e].x, u[e].y);
    __syncthreads();
    for (int e = tid; e < H * CB; e += kThreads) {
        const int r = e / CB, c = e % CB;
        P.Sa[(size_t)r * Wp + c0 + c] = stage[e];
    }
}

// ---------------------------------------------------------------------------
// inverse row DFTs + mask prox + d1 dual. Grid (H / G, slots).
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
grow_inv(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ twW) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using R = GRow<W>;
    constexpr int T = R::T, E = R::E, G = R::G;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const int k = P.ctl->iter + 1;
    const bool first = k == 1;                   // x_prev = 0 (no earlier iterate)
    const bool cold = first && !P.warm;          // d1 = 0 (u0 = d0 = 0)
    const bool chk = is_check_iter(P, k), sprev = store_prev_iter(P, k), nobj = need_obj_iter(P, k);
    extern __shared__ __align__(16) float2 gsm2[];
    float2* buf = gsm2;                          // G x W
    float2* tw = buf + G * W;
    // d1, M^T y and x_prev of this thread's own pixels, requested before the
    // transform (the thread reads back only what it copied itself)
    float* pre = reinterpret_cast<float*>(tw + W);   // 3 x G x W
    __shared__ float red[kThreads / 32 * 2 * kNumPartials];
    const int tid = threadIdx.x, g = tid / T, t = tid % T;
    const int q = blockIdx.x * G + g;
    const size_t n = (size_t)H * W;
    float* pd1 = pre + (size_t)(3 * g) * W;
    float* pyb = pd1 + W;
    float* pxp = pyb + W;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int c = t + T * e;
        const size_t pix = (size_t)q * W + c;
        if (!cold) cp_async4(pd1 + c, P.d1 + pix);
        cp_async4(pyb + c, P.ybar + pix);
        if (chk && !first) cp_async4(pxp + c, P.xprev + pix);
    }
    cp_async_commit();
    for (int e = tid; e < W; e += kThreads) tw[e] = twW[e];
    __syncthreads();
    // the full spectrum of the complex row x + i A x from the two stored halves
    const float4* __restrict__ srow = P.Sa + (size_t)q * Wp;
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int kk = t + T * e;
        if (kk <= W / 2) {
            const float4 s = srow[kk];
            v[e] = make_float2(s.x - s.w, s.y + s.z);
        } else {
            const float4 s = srow[W - kk];
            v[e] = make_float2(s.x + s.w, s.z - s.y);
        }
    }
    gfft<W, 1>(v, t, g, tw, buf + (size_t)g * W);
    cp_async_wait<0>();          // this thread's staged inputs have landed
    float* __restrict__ xw = P.work;
    float* __restrict__ z1w = P.work + n;
    const float mu1 = P.mu1, inv1 = P.inv1pmu1;
    CompSum s_data, s_xx, s_dxx, s_pr;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const size_t pix = (size_t)q * W + t + T * e;
        const float x = v[e].x, ax = v[e].y;
        // u1 = (M^T M + mu1 I)^{-1} (M^T y + mu1 (A x - d1)); d1 <- d1 - (A x - u1)
        const float dd1 = cold ? 0.f : pd1[t + T * e];
        const float s1 = ax - dd1;
        const float yb = pyb[t + T * e];
        const bool obs = is_observed(yb);
        const float u1 = obs ? fmaf(mu1, s1, yb) * inv1 : s1;
        const float nd1 = dd1 - (ax - u1);
        P.d1[pix] = nd1;
        z1w[pix] = u1 + nd1;
        xw[pix] = x;
        if (nobj) {
            if (obs) {
                const float er = ax - yb;
                s_data.add(0.5f * er * er);
            }
            const float e1 = nd1 - dd1;
            s_pr.add(e1 * e1);
        }
        if (chk) {
            const float dx = first ? x : x - pxp[t + T * e];
            s_dxx.add(dx * dx);
            s_xx.add(x * x);
        }
        if (sprev) P.xprev[pix] = x;
    }
    if (nobj || chk) {
        const CompSum acc[kNumPartials] = {s_data, CompSum(), s_xx, s_dxx, s_pr};
        double pv[kNumPartials];
        block_reduce_comp(acc, red, pv);
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < kNumPartials; ++j) P.partials[blockIdx.x * kNumPartials + j] = pv[j];
        }
    }
}

// ---------------------------------------------------------------------------
// forward row DFTs of p = a + i b and the Hermitian split into half spectra
// A[k] = (P[k] + conj P[W-k]) / 2, B[k] = (P[k] - conj P[W-k]) / 2i, k <= W/2.
// WARM = false: a = zeta1, b = w from the scratch planes (the end of an
// iteration; skipped for an inactive problem or one that has just taken
// over the slot). WARM = true: a = x0, b = 0 from `x0` (warm start; no
// control block). Grid (H / G, slots or 1).
// ---------------------------------------------------------------------------
template <int W, bool WARM = false>
__global__ void __launch_bounds__(kThreads)
grow_fwd(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ twW,
         const float* __restrict__ x0, float4* __restrict__ Sb0) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using R = GRow<W>;
    constexpr int T = R::T, E = R::E, G = R::G;
    const float* za;
    const float* wb = nullptr;
    float4* Sb;
    if constexpr (WARM) {
        za = x0;
        Sb = Sb0;
    } else {
        const int pi = sl.map[blockIdx.y];
        if (pi < 0) return;
        const ProbDesc& P = probs[pi];
        if (P.ctl->active == 0 || P.ctl->iter == 0) return;
        const size_t n = (size_t)H * W;
        za = P.work + n;
        wb = P.work + 2 * n;
        Sb = P.Sb;
    }
    extern __shared__ __align__(16) float2 gsm2[];
    float2* buf = gsm2;
    float2* tw = buf + G * W;
    const int tid = threadIdx.x, g = tid / T, t = tid % T;
    const int q = blockIdx.x * G + g;
    for (int e = tid; e < W; e += kThreads) tw[e] = twW[e];
    __syncthreads();
    float2 v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const size_t pix = (size_t)q * W + t + T * e;
        v[e] = make_float2(za[pix], WARM ? 0.f : wb[pix]);
    }
    float2* row = buf + (size_t)g * W;
    gfft<W, -1>(v, t, g, tw, row);
#pragma unroll
    for (int e = 0; e < E; ++e) row[t + T * e] = v[e];
    ggroup_sync<T>(g);
    float4* __restrict__ drow = Sb + (size_t)q * Wp;
    for (int kk = t; kk <= W / 2; kk += T) {
        const float2 pk = row[kk];
        const float2 pn = row[kk == 0 ? 0 : W - kk];
        const float2 a = 0.5f * make_float2(pk.x + pn.x, pk.y - pn.y);
        const float2 dd = make_float2(pk.x - pn.x, pk.y + pn.y);
        drow[kk] = make_float4(a.x, a.y, 0.5f * dd.y, -0.5f * dd.x);
    }
}

template <int W> constexpr size_t grow_smem() { return (size_t)(GRow<W>::G * W + W) * sizeof(float2); }
// the inverse rows also stage d1, M^T y and x_prev of their G rows
template <int W> constexpr size_t grow_inv_smem() {
    return grow_smem<W>() + (size_t)3 * GRow<W>::G * W * sizeof(float);
}

// Launch chain of one iteration on an exact generic domain (gen.cu).
cudaError_t launch_gen_iteration(int W, int H, int Wc, int Wp, const ProbDesc* d, SlotTable sl, int count,
                                 int reg, int levels, const float2* twH, const float2* twW, int* n_active,
                                 cudaStream_t s);
// The kernels after the one that finishes an iteration (the frame synthesis
// with synth = true, and the forward row DFTs), for admm_deconv_get_full_state.
cudaError_t launch_gen_tail(int W, int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels,
                            bool synth, const float2* twW, cudaStream_t s);
// The row DFTs of a warm-start image into Sb.
cudaError_t launch_gen_warm_rows(int W, int H, int Wp, const float* x0, float4* Sb, const float2* twW,
                                 cudaStream_t s);
// Columns per column-phase CTA and rows per row CTA of a generic domain.
int gen_col_block(int H);
int gen_rows_per_cta(int W);

}  // namespace admm
