// haar.cuh -- row side of FA-MD (frame-based analysis prior, Sec. IV-C).
//
// One FA-MD iteration (Algorithm 2 with H1 = A, H2 = P) after the column
// phase has produced the row spectra of (x, A x):
//
//   haar_row_inverse   inverse row DFTs -> x, A x; mask-decoupled prox and
//                      dual update (eq. prox_g_1_uBC, Alg. 2 lines 6-7, j = 1);
//                      writes x and zeta1 = u1 + d1 to two scratch planes
//   haar_analysis      32 x 32 tile: analysis c = P x (a-trous Haar), u2 =
//                      soft(c - d2, lambda/mu2) (eq. soft), d2 <- d2 - (c - u2);
//                      zeta2 = u2 + d2 and two bits per coefficient replace
//                      the previous state in place (see below); the last CTA
//                      of the problem finishes the iteration
//   haar_synthesis     32 x 32 tile: w = gamma P^T zeta2 (the x-step right-
//                      hand side of eq. invAnalysis divided by mu1)
//   haar_row_forward   forward row DFT of zeta1 + i w, split into half spectra
//
// P is the undecimated Haar frame with periodic wrap: level j filters with
// h = [1/2, 1/2] and g = [1/2, -1/2] at taps {0, 2^j}, emits three detail
// bands and passes the low-low band on; the last low-low band is kept
// (3 L + 1 bands, P^T P = I). Band order per level: rows low / columns high,
// rows high / columns low, rows high / columns high; final band low-low.
//
// State of the analysis prior: with s = c - d2 the argument of the soft
// threshold (tau = lambda/mu_b of the band), the new dual is d2' = u2 - s =
// -clamp(s, -tau, tau): -tau sign(s) where the threshold passes s (u2 != 0),
// -s elsewhere, where zeta2 = u2 + d2' = d2'. So zeta2 and two bits per
// coefficient (u2 != 0; s < 0) carry d2' exactly: the analysis stores
// (gamma_b/gamma) zeta2 in d2 buffer 0 over the state it has just read (each
// coefficient is read and replaced by the thread that owns it) and the bits
// of all bands of a pixel in one word (zbits); the synthesis (a separate
// launch) reads zeta2 there with its halo. Iteration 1 reads d2 itself from
// buffer 0 (zero, a warm start or a restored state). The synthesis
// formulation (FS-MD) keeps the same state: its analysis also needs the
// previous zeta2, which is the value it reads there (at iteration 1 of a
// restored state, from buffer 1).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include "kernels.cuh"

namespace admm {

constexpr int kMaxHaarLevels = 4;
constexpr int kHaarTile = 32;

// periodic index for x in [-n, 2n): sides are multiples of 32, not
// necessarily powers of two (exact generic domains)
__device__ __forceinline__ int hwrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// rows per CTA of the two row kernels: one row transform per thread group
inline int haar_rows_per_cta(int W) { return kThreads / (W / 8); }
inline int haar_row_strip(int W) { return haar_rows_per_cta(W); }
inline int haar_num_row_ctas(int H, int W) { return H / haar_rows_per_cta(W); }
inline int haar_num_tiles(int H, int W) { return (H / kHaarTile) * (W / kHaarTile); }

// Rows of 1024 and more read their per-pass twiddle table from the device
// buffer (through L1) instead of staging W float2 in shared memory: the
// 8-16 KB go to more CTAs per SM on these latency-bound row kernels.
template <int W> __host__ __device__ constexpr bool haar_tw_global() { return W >= 1024; }
template <int W> __host__ __device__ constexpr int haar_tw_smem() { return haar_tw_global<W>() ? 0 : W; }
template <int W> constexpr size_t haar_inv_smem() {
    constexpr int G = kThreads / (W / 8);
    return (size_t)(G * W + haar_tw_smem<W>()) * sizeof(float2) + 8 * kNumPartials * sizeof(double) +
           (size_t)3 * G * W * sizeof(float);   // + staged d1, M^T y, x_prev
}
template <int W> constexpr size_t haar_fwd_smem() {
    constexpr int G = kThreads / (W / 8);
    return (size_t)(2 * G * W + haar_tw_smem<W>()) * sizeof(float2);   // two rows per group
}

// ---------------------------------------------------------------------------
// inverse row DFT + mask prox + d1 dual (no halo: every row is owned)
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
haar_row_inverse(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    constexpr int FT = W / 8, G = kThreads / FT, ROW = W;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const int k = P.ctl->iter + 1;
    const bool first = k == 1;                   // x_prev = 0 (no earlier iterate)
    const bool cold = first && !P.warm;          // d1 = 0 (u0 = d0 = 0)
    const bool chk = is_check_iter(P, k), sprev = store_prev_iter(P, k), nobj = need_obj_iter(P, k);
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tws = buf + G * ROW;
    const float2* tw = haar_tw_global<W>() ? tw_g + pass_table_offset<W>() : tws;
    double* red = reinterpret_cast<double*>(tws + haar_tw_smem<W>());
    // per-pixel inputs of the prox (d1, M^T y, x_prev), staged by the thread
    // that uses them while the transform runs
    float* pre = reinterpret_cast<float*>(red + 8 * kNumPartials);
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    const int q = blockIdx.x * G + g;
    const size_t n = (size_t)H * W;
    float* pd1 = pre + (size_t)(3 * g) * W;
    float* pyb = pd1 + W;
    float* pxp = pyb + W;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int c = t + m * FT;
        const size_t pix = (size_t)q * W + c;
        if (!cold) cp_async4(pd1 + c, P.d1 + pix);
        cp_async4(pyb + c, P.ybar + pix);
        if (chk && !first) cp_async4(pxp + c, P.xprev + pix);
    }
    cp_async_commit();
    if (!haar_tw_global<W>()) load_twiddles<W>(tws, tw_g, tid, kThreads);
    __syncthreads();
    float2 v[8];
    load_row_xax<W>(v, P.Sa + (size_t)q * Wp, t);
    fft_group<W, 1>(v, buf + g * ROW, tw, t, g);
    cp_async_wait<0>();          // this thread's staged inputs have landed
    float* __restrict__ xw = P.work;
    float* __restrict__ z1w = P.work + n;
    const float mu1 = P.mu1, inv1 = P.inv1pmu1;
    CompSum s_data, s_xx, s_dxx, s_pr;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int c = t + m * FT;
        const size_t pix = (size_t)q * W + c;
        const float x = v[m].x, ax = v[m].y;
        // u1 = (M^T M + mu1 I)^{-1} (M^T y + mu1 (A x - d1)); d1 <- d1 - (A x - u1)
        const float dd1 = cold ? 0.f : pd1[c];
        const float s1 = ax - dd1;
        const float yb = pyb[c];
        const bool obs = is_observed(yb);
        const float u1 = obs ? fmaf(mu1, s1, yb) * inv1 : s1;
        const float nd1 = dd1 - (ax - u1);
        P.d1[pix] = nd1;
        z1w[pix] = u1 + nd1;
        xw[pix] = x;
        if (nobj) {
            if (obs) {
                const float e = ax - yb;
                s_data.add(0.5f * e * e);
            }
            const float e1 = nd1 - dd1;       // d1 part of d_k - d_{k-1}
            s_pr.add(e1 * e1);
        }
        if (chk) {
            const float dx = first ? x : x - pxp[c];
            s_dxx.add(dx * dx);
            s_xx.add(x * x);
        }
        if (sprev) P.xprev[pix] = x;
    }
    // partial sums only where the tile kernel evaluates the stop rule
    if (nobj || chk) {
        const CompSum acc[kNumPartials] = {s_data, CompSum(), s_xx, s_dxx, s_pr};
        double pv[kNumPartials];
        block_reduce_comp(acc, reinterpret_cast<float*>(red), pv);
        if (tid == 0) {
#pragma unroll
            for (int j = 0; j < kNumPartials; ++j) P.partials[blockIdx.x * kNumPartials + j] = pv[j];
        }
    }
}

__device__ __forceinline__ float soft_thresh(float v, float t) {
    const float a = fabsf(v) - t;
    return a > 0.f ? copysignf(a, v) : 0.f;
}

// the two state bits of a coefficient: bit 0 the threshold passed s (|s| >
// tau), bit 1 the sign bit of s
__device__ __forceinline__ uint32_t state_bits(float sv, float tau) {
    return (fabsf(sv) > tau ? 1u : 0u) | ((__float_as_uint(sv) >> 30) & 2u);
}
// d2 of one coefficient from its stored (gamma_b/gamma) zeta2 `z` and its two
// bits: -tau sign(s) where the threshold passed, else zeta2 itself (izs =
// gamma / gamma_b)
__device__ __forceinline__ float dual_from_zeta(float z, uint32_t bits, float tau, float izs) {
    const float dt = __uint_as_float(__float_as_uint(tau) ^ ((~bits & 2u) << 30));   // -tau sign(s)
    return (bits & 1u) ? dt : z * izs;
}

// ---------------------------------------------------------------------------
// analysis c = P x on a T x T tile (a-trous Haar), soft threshold, dual
// update. Every coefficient of the tile is owned by this CTA: the previous d2
// is read and zeta2 = u2 + d2 written back in its place by the same thread,
// the new d2 goes to the other buffer. a_{j+1}(r, c) averages a_j at
// (r + {0, s}, c + {0, s}), so the tile needs x on [0, T + 2^L - 1)^2 only.
// ---------------------------------------------------------------------------
template <int L>
struct HaarAnaCfg {
    static constexpr int T = kHaarTile;
    static constexpr int HALO = (1 << L) - 1;
    static constexpr int XA = T + 16;              // stride (16-byte rows); x needs T + HALO columns
    static constexpr int XR = T + HALO;            // rows of x
    static_assert(HALO < 16, "halo fits the 16-column margin");
    static constexpr int NBAND = 3 * L + 1;
    // previous d2 of the tile: two slots of four bands; level j's bands (and
    // the low-low band with the last level) in slot j % 2
    static constexpr int D2S_OFF = 2 * XR * XA;
    static constexpr int SLOT = 4 * T * T;
    static constexpr int RED_OFF = D2S_OFF + 2 * SLOT;
    static_assert((RED_OFF * sizeof(float)) % sizeof(double) == 0, "double alignment");
    static constexpr size_t SMEM = (size_t)RED_OFF * sizeof(float) + 8 * kNumPartials * sizeof(double);
};


// FS: the frame synthesis formulation (FS-MD, Sec. IV-B). There the thresholded
// coefficients are theta = P (x - P^T zeta2) + zeta2 (the theta-step of the
// synthesis problem with W = P^T, reduced with W W^T = I and the x-step's
// equation A^T (zeta1 - A x) = gamma (x - P^T zeta2)); P^T zeta2 = w / gamma
// is the previous synthesis output and zeta2 the previous iteration's: the
// stored state the tile reads anyway (buffer 1 at iteration 1 of a restored
// state).
template <int L, bool FS = false>
__global__ void __launch_bounds__(kThreads, 4)
haar_analysis(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int W, int n_row_ctas,
              int* __restrict__ n_active) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using C = HaarAnaCfg<L>;
    constexpr int T = C::T, XA = C::XA, XR = C::XR;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    ProbCtl* ctl = P.ctl;
    if (ctl->active == 0) return;
    const int k = ctl->iter + 1;
    const bool first = k == 1 && !P.warm;        // d2 = 0 (cold start: u0 = d0 = 0)
    const bool raw = k == 1;                     // buffer holds d2 itself (not zeta2 and bits)
    const bool chk = is_check_iter(P, k), nobj = need_obj_iter(P, k);
    extern __shared__ __align__(16) float sm[];
    float* Ain = sm;
    float* Aout = sm + XR * XA;
    float* d2s = sm + C::D2S_OFF;
    double* red = reinterpret_cast<double*>(sm + C::RED_OFF);
    const int tid = threadIdx.x;
    const int tiles_x = W / T;
    const int R0 = (blockIdx.x / tiles_x) * T, C0 = (blockIdx.x % tiles_x) * T;
    const size_t n = (size_t)H * W;
    // previous state in, zeta2 out; FS-MD at iteration 1 of a restored state:
    // the previous zeta2 in buffer 1
    float* __restrict__ d2io = P.d2;
    const float* __restrict__ z1in = P.d2 + P.d2_stride;

    // x on [0, T + HALO) x [0, T + 16) with periodic wrap, 16-byte copies (the
    // tile origin is a multiple of 32 columns)
    constexpr int CH = XA / 4;
    for (int e = tid; e < XR * CH; e += kThreads) {
        const int rr = e / CH, ch = e - rr * CH;
        const float* src = P.work + (size_t)hwrap(R0 + rr, H) * W + hwrap(C0 + 4 * ch, W);
        cp_async16(Ain + rr * XA + 4 * ch, src);
        if (FS && !first) {
            // w = gamma P^T zeta2 of the previous iteration on the same region (zero at the start)
            const float* wsrc = P.work + 2 * n + (size_t)hwrap(R0 + rr, H) * W + hwrap(C0 + 4 * ch, W);
            cp_async16(Aout + rr * XA + 4 * ch, wsrc);
        }
    }
    cp_async_commit();
    // thread t owns the four adjacent tile pixels of row t / 8, columns
    // 4 (t % 8) .. + 3: 16-byte reads of x and of the staged d2, 16-byte
    // stores of the new d2 and of zeta2. Every thread stages the previous d2
    // of its own pixels, one cp.async group per level (the last with the
    // low-low band), two levels ahead in two slots: it reads only what it
    // copied itself, so neither the copies nor the reuse of a slot need a
    // block barrier.
    static_assert(T * T == 4 * kThreads, "four owned pixels per thread");
    const int orow = tid >> 3, ocol = 4 * (tid & 7);
    const size_t gq = (size_t)(R0 + orow) * W + (C0 + ocol);
    // the bits of the previous iteration at the owned pixels (two per band)
    uint32_t obits[4] = {0u, 0u, 0u, 0u};
    if (!raw) {
        const uint4 bv = *reinterpret_cast<const uint4*>(P.zbits + gq);
        obits[0] = bv.x; obits[1] = bv.y; obits[2] = bv.z; obits[3] = bv.w;
    }
    uint32_t nbits[4] = {0u, 0u, 0u, 0u};
    auto stage = [&](int lvl) {
        if (!first) {
            const int nb = lvl == L - 1 ? 4 : 3;
#pragma unroll
            for (int j = 0; j < nb; ++j) {
                const int b = 3 * lvl + j;
                cp_async16(d2s + (lvl & 1) * C::SLOT + j * T * T + orow * T + ocol, d2io + (size_t)b * n + gq);
            }
        }
        cp_async_commit();
    };
    stage(0);
    if (L >= 2) stage(1);
    cp_async_wait_n(L >= 2 ? 2 : 1);   // x has landed (the d2 groups may still be in flight)
    __syncthreads();
    if (FS && !first) {
        // v = x - P^T zeta2, whose analysis the levels below compute
        const float inv_g = 1.0f / P.gamma;
        for (int e = tid; e < XR * XA; e += kThreads) Ain[e] = fmaf(-inv_g, Aout[e], Ain[e]);
        __syncthreads();
    }

    CompSum l1, pr;
#pragma unroll
    for (int lvl = 0; lvl < L; ++lvl) {
        const int s = 1 << lvl;
        // this level's previous d2 at the owned pixels (the next level's
        // group may still be in flight)
        if (lvl + 1 < L) cp_async_wait<1>();
        else cp_async_wait<0>();
        float dold[3][4];
        // FS: the previous iteration's zeta2 of this level's bands (own pixels)
        float zprev[3][4] = {};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float4 v = first ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : *reinterpret_cast<const float4*>(d2s + (lvl & 1) * C::SLOT + j * T * T + orow * T + ocol);
            dold[j][0] = v.x; dold[j][1] = v.y; dold[j][2] = v.z; dold[j][3] = v.w;
            if (!raw) {
                const int b = 3 * lvl + j;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (FS) zprev[j][e] = dold[j][e];
                    dold[j][e] = dual_from_zeta(dold[j][e], obits[e] >> (2 * b), P.band_tau[b], P.band_izs[b]);
                }
            } else if (FS && !first) {
                const float4 zv = *reinterpret_cast<const float4*>(z1in + (size_t)(3 * lvl + j) * n + gq);
                zprev[j][0] = zv.x; zprev[j][1] = zv.y; zprev[j][2] = zv.z; zprev[j][3] = zv.w;
            }
        }
        // the slot is consumed (the last level's low-low entries are read
        // after the loop, and nothing is staged after the last level)
        if (lvl + 2 < L) stage(lvl + 2);
        const int D = T + (1 << L) - 2 * s;      // a_{lvl+1} is needed on [0, D)^2
        // owned pixels: approximation, detail bands, soft threshold and dual
        // updates. a_lvl on rows orow and orow + s, columns ocol .. ocol + 3 + s
        float w0[12], w1[12];
        const int NW = s > 4 ? 3 : 2;            // float4 words covering 4 + s columns
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (q < NW) {
                const float4 u0 = *reinterpret_cast<const float4*>(Ain + orow * XA + ocol + 4 * q);
                const float4 u1 = *reinterpret_cast<const float4*>(Ain + (orow + s) * XA + ocol + 4 * q);
                w0[4 * q] = u0.x; w0[4 * q + 1] = u0.y; w0[4 * q + 2] = u0.z; w0[4 * q + 3] = u0.w;
                w1[4 * q] = u1.x; w1[4 * q + 1] = u1.y; w1[4 * q + 2] = u1.z; w1[4 * q + 3] = u1.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) w0[4 * q + e] = w1[4 * q + e] = 0.f;
            }
        }
        float ao[4], nd4[3][4], z4[3][4];
        float prl = 0.f;                         // this level's share of ||d_k - d_{k-1}||^2
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float a00 = w0[e], a01 = w0[e + s], a10 = w1[e], a11 = w1[e + s];
            const float p0 = a00 + a01, m0 = a00 - a01, p1 = a10 + a11, m1 = a10 - a11;
            ao[e] = 0.25f * (p0 + p1);
            // detail bands: rows low / cols high, rows high / cols low, both high
            float cb[3] = {0.25f * (m0 + m1), 0.25f * (p0 - p1), 0.25f * (m0 - m1)};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (FS) cb[j] += zprev[j][e];                   // theta = P v + zeta2
                const float sv = cb[j] - dold[j][e];
                const float tb = P.band_tau[3 * lvl + j];
                // d2 - (c - u2) = -clamp(s, -tau, tau), exactly, and u2 = s +
                // that (= soft(s, tau), eq. soft, with its rounding)
                nd4[j][e] = copysignf(fminf(fabsf(sv), tb), -sv);
                const float u = sv + nd4[j][e];
                nbits[e] |= state_bits(sv, tb) << (2 * (3 * lvl + j));
                // zeta2 = u2 + d2, times gamma_b / gamma for the synthesis
                z4[j][e] = (u + nd4[j][e]) * P.band_zs[3 * lvl + j];
                if (nobj) {
                    l1.add(fabsf(cb[j]));
                    const float e2 = nd4[j][e] - dold[j][e];    // d2 part of d_k - d_{k-1}
                    prl = fmaf(e2, e2, prl);
                }
            }
        }
        if (nobj) pr.add(prl);
        *reinterpret_cast<float4*>(Aout + orow * XA + ocol) = make_float4(ao[0], ao[1], ao[2], ao[3]);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const size_t bo = (size_t)(3 * lvl + j) * n + gq;
            *reinterpret_cast<float4*>(d2io + bo) = make_float4(z4[j][0], z4[j][1], z4[j][2], z4[j][3]);
        }
        // the approximation on the rest of [0, D)^2 that later levels read
        // (rows [0, T) x columns [T, D), then rows [T, D) x columns [0, D)),
        // spread evenly over the block
        const int DT = D - T;
        const int n1 = T * DT, nh = n1 + DT * D;
        for (int e = tid; e < nh; e += kThreads) {
            int rr, cc;
            if (e < n1) {
                rr = e / (DT > 0 ? DT : 1);
                cc = T + (e - rr * DT);
            } else {
                const int f = e - n1;
                rr = T + f / D;
                cc = f - (rr - T) * D;
            }
            const int i00 = rr * XA + cc;
            const float a00 = Ain[i00], a01 = Ain[i00 + s];
            const float a10 = Ain[i00 + s * XA], a11 = Ain[i00 + s * XA + s];
            Aout[i00] = 0.25f * ((a00 + a01) + (a10 + a11));
        }
        __syncthreads();
        float* tmp = Ain;
        Ain = Aout;
        Aout = tmp;
    }
    // the last low-low band a_L on the tile (threshold 0 when it is unpenalised)
    {
        const bool ll_free = P.ll_free != 0;
        const float tau_ll = ll_free ? 0.f : P.band_tau[3 * L];
        const float4 dv = first ? make_float4(0.f, 0.f, 0.f, 0.f)
                                : *reinterpret_cast<const float4*>(d2s + ((L - 1) & 1) * C::SLOT + 3 * T * T +
                                                                   orow * T + ocol);
        const float4 cv = *reinterpret_cast<const float4*>(Ain + orow * XA + ocol);
        float dold[4] = {dv.x, dv.y, dv.z, dv.w};
        float cb[4] = {cv.x, cv.y, cv.z, cv.w};
        if (!raw) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (FS) cb[e] += dold[e];                     // theta = P v + zeta2
                dold[e] = dual_from_zeta(dold[e], obits[e] >> (2 * 3 * L), tau_ll, P.band_izs[3 * L]);
            }
        } else if (FS && !first) {
            const float4 zv = *reinterpret_cast<const float4*>(z1in + (size_t)(3 * L) * n + gq);
            cb[0] += zv.x; cb[1] += zv.y; cb[2] += zv.z; cb[3] += zv.w;
        }
        float nd[4], z[4];
        float prl = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float sv = cb[e] - dold[e];
            nd[e] = copysignf(fminf(fabsf(sv), tau_ll), -sv);
            const float u = sv + nd[e];
            nbits[e] |= state_bits(sv, tau_ll) << (2 * 3 * L);
            z[e] = (u + nd[e]) * P.band_zs[3 * L];
            if (nobj) {
                if (!ll_free) l1.add(fabsf(cb[e]));
                const float e2 = nd[e] - dold[e];
                prl = fmaf(e2, e2, prl);
            }
        }
        if (nobj) pr.add(prl);
        const size_t bo = (size_t)(3 * L) * n + gq;
        *reinterpret_cast<float4*>(d2io + bo) = make_float4(z[0], z[1], z[2], z[3]);
        *reinterpret_cast<uint4*>(P.zbits + gq) = make_uint4(nbits[0], nbits[1], nbits[2], nbits[3]);
    }
    double pv[kNumPartials] = {0.0};
    if (nobj || chk) {
        const CompSum acc[kNumPartials] = {CompSum(), l1, CompSum(), CompSum(), pr};
        block_reduce_comp(acc, reinterpret_cast<float*>(red), pv);
    }
    finish_iteration<kThreads>(P, k, chk, nobj, pv, n_active, n_row_ctas + blockIdx.x, probs, sl);
}

// ---------------------------------------------------------------------------
// w = gamma P^T zeta2 on a T x T tile (adjoint synthesis, coarse to fine).
// The adjoint of level j reads the coarser approximation and the level-j
// bands at (r - {0, s}, c - {0, s}), so the tile needs zeta2 of level j on
// [-(2^{j+1} - 1), T)^2 and the low-low band on [-(2^L - 1), T)^2.
// Runs after haar_analysis has finished the iteration (ctl->iter = k).
// ---------------------------------------------------------------------------
template <int L>
struct HaarSynCfg {
    static constexpr int T = kHaarTile;
    static constexpr int HALO = (1 << L) - 1;
    static_assert(HALO < 16, "halo fits the 16-column margin");
    // every array spans the columns [-16, T) (16-byte copies from a tile
    // origin that is a multiple of 32 columns) and the rows it needs
    static constexpr int XS = T + 16;              // row stride of every array
    static constexpr int AR = T + HALO;            // approximation arrays: rows [-HALO, T)
    __host__ __device__ static constexpr int band_rows(int lvl) { return T + 2 * (1 << lvl) - 1; }
    // two band slots, each sized for the coarsest level: level j lives in slot
    // j % 2, and the bands of level j - 1 are requested into the other slot as
    // soon as level j + 1 has released it. Array sizes are rounded to 32
    // floats, so that the TMA destinations (the low-low array and the two
    // slots) start on 128-byte boundaries; two mbarriers follow.
    static constexpr int ARS = (AR * XS + 31) / 32 * 32;
    static constexpr int SLOT = (3 * band_rows(L - 1) * XS + 31) / 32 * 32;
    static constexpr size_t BAR_OFF = (size_t)(2 * ARS + 2 * SLOT) * sizeof(float);
    static constexpr size_t SMEM = BAR_OFF + 2 * sizeof(unsigned long long);
};

// Host: the L + 1 tensor maps the synthesis tile loads its halo boxes with,
// over both d2 buffers of a problem viewed as a 4-D tensor (W columns, H rows,
// 3 L + 1 bands, 2 buffers; FP32): map 0 the low-low band's box (T + 16
// columns x T + 2^L - 1 rows x 1 band), map 1 + j level j's three bands
// (T + 16 columns x T + 2^{j+1} - 1 rows x 3 bands). `enc` is the driver's
// cuTensorMapEncodeTiled; false if a map cannot be encoded.
template <typename Enc, typename Map>
bool haar_synthesis_maps(Enc enc, Map* maps, float* d2, int H, int W, int levels) {
    const int nb = 3 * levels + 1;
    const uint64_t n = (uint64_t)H * W;
    const uint64_t dims[4] = {(uint64_t)W, (uint64_t)H, (uint64_t)nb, 2};
    const uint64_t strides[3] = {(uint64_t)W * 4, n * 4, (uint64_t)nb * n * 4};
    const uint32_t es[4] = {1, 1, 1, 1};
    for (int i = 0; i <= levels; ++i) {
        const uint32_t rows = i == 0 ? (uint32_t)(kHaarTile + (1 << levels) - 1)
                                     : (uint32_t)(kHaarTile + 2 * (1 << (i - 1)) - 1);
        const uint32_t box[4] = {(uint32_t)(kHaarTile + 16), rows, i == 0 ? 1u : 3u, 1u};
        if (!enc(&maps[i], d2, dims, strides, box, es)) return false;
    }
    return true;
}

template <int L>
__global__ void __launch_bounds__(kThreads)
haar_synthesis(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int W) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    using C = HaarSynCfg<L>;
    constexpr int T = C::T, HALO = C::HALO, XS = C::XS, AR = C::AR;
    constexpr int CH = XS / 4;                     // 16-byte chunks per array row
    constexpr int NWARP = kThreads / 32;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    // retired in this iteration, or a problem that has just taken over the slot
    if (P.ctl->active == 0 || P.ctl->iter == 0) return;
    extern __shared__ __align__(128) float syn_sm[];
    float* sm = syn_sm;
    float* At = sm;
    float* Ao = sm + C::ARS;
    float* Z = sm + 2 * C::ARS;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(sm) + C::BAR_OFF);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tiles_x = W / T;
    const int R0 = (blockIdx.x / tiles_x) * T, C0 = (blockIdx.x % tiles_x) * T;
    const size_t n = (size_t)H * W;
    // zeta2: in d2 buffer 0, where the analysis has just written it
    constexpr int zb = 0;
    const float* __restrict__ zeta = P.d2;
    // Tiles whose halo stays inside the image (every tile but the first row
    // and column; the halo lies above and to the left) take their boxes by
    // TMA, one thread issuing one copy per level (and one for the low-low
    // band) on the level slot's mbarrier; the others copy with cp.async and
    // wrap periodically.
    const bool tma = P.zmap != nullptr && R0 > 0 && C0 > 0 && (smem_u32(sm) & 127u) == 0;
    const char* zmaps = static_cast<const char*>(P.zmap);
    auto tma_request = [&](int lvl) {
        const int BO = 2 * (1 << lvl) - 1;
        const uint32_t bar = smem_u32(&bars[lvl & 1]);
        const uint32_t bytes = 3u * (uint32_t)((T + BO) * XS) * 4u + (lvl == L - 1 ? (uint32_t)(AR * XS) * 4u : 0u);
        mbar_expect_tx(bar, bytes);
        if (lvl == L - 1) tma_load_4d(At, zmaps, C0 - 16, R0 - HALO, 3 * L, zb, bar);
        tma_load_4d(Z + (lvl & 1) * C::SLOT, zmaps + 128 * (1 + lvl), C0 - 16, R0 - BO, 3 * lvl, zb, bar);
    };

    // low-low band on rows [-HALO, T) and each level's bands on rows [-BO, T),
    // all on the columns [-16, T), one cp.async group per level (the low-low
    // band with the coarsest). Two levels are requested at entry; each later
    // level goes into the slot the level before last has just released, so
    // its loads overlap the adjoint of the level in between.
    auto request = [&](int lvl) {
        const int BO = 2 * (1 << lvl) - 1, BR = T + BO;
        float* Zl = Z + (lvl & 1) * C::SLOT;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float* band = zeta + (size_t)(3 * lvl + j) * n;
            for (int e = tid; e < BR * CH; e += kThreads) {
                const int rr = e / CH, ch = e - rr * CH;
                cp_async16(Zl + (j * BR + rr) * XS + 4 * ch,
                           band + (size_t)hwrap(R0 + rr - BO, H) * W + hwrap(C0 - 16 + 4 * ch, W));
            }
        }
        cp_async_commit();
    };
    if (tma) {
        if (tid == 0) {
            mbar_init1(smem_u32(&bars[0]));
            mbar_init1(smem_u32(&bars[1]));
            mbar_init_fence();
            tma_request(L - 1);
            if (L >= 2) tma_request(L - 2);
        }
        __syncthreads();             // the barriers are initialised before anyone waits on them
    } else {
        const float* band = zeta + (size_t)(3 * L) * n;
        for (int e = tid; e < AR * CH; e += kThreads) {
            const int rr = e / CH, ch = e - rr * CH;
            cp_async16(At + rr * XS + 4 * ch,
                       band + (size_t)hwrap(R0 + rr - HALO, H) * W + hwrap(C0 - 16 + 4 * ch, W));
        }
        request(L - 1);
        if (L >= 2) request(L - 2);
    }

#pragma unroll
    for (int lvl = L - 1; lvl >= 0; --lvl) {
        // this level's bands have landed (at the first level the next one may
        // still be in flight; later, the next level is requested only below)
        if (tma) {
            // slot lvl % 2 completes its ((L - 1 - lvl) / 2)-th phase with this level
            const uint32_t parity = (uint32_t)((L - 1 - lvl) >> 1) & 1u;
            if (!mbar_wait_bounded(smem_u32(&bars[lvl & 1]), parity) && tid == 0)
                atomicExch(&P.ctl->status, kStatusTimeout);
        } else if (lvl == L - 1 && L >= 2) {
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();             // ... for every thread; level lvl + 1 is done and its slot free
        if (lvl <= L - 2 && lvl >= 1) {
            if (!tma) {
                request(lvl - 1);
            } else if (tid == 0) {
                fence_proxy_async_smem();   // the slot's generic reads before the copy's writes
                tma_request(lvl - 1);
            }
        }
        const int s = 1 << lvl;
        const int D = T + s - 1;                       // output on [-(s-1), T)
        const int BO = 2 * s - 1, BR = T + BO;
        const float* Z0 = Z + (lvl & 1) * C::SLOT;
        const float* Z1 = Z0 + BR * XS;
        const float* Z2 = Z1 + BR * XS;
        const int ra = s * XS, rz = s * XS;
        // the outputs on [-(s-1), T)^2. Columns [0, T) in groups of four
        // adjacent columns, eight groups per row, so that the eight threads of
        // a 16-byte access phase read one 128-byte row segment: 16-byte reads of
        // the eight input rows (At, Z0, Z1, Z2 at rows r and r - s) over columns
        // c - s .. c + 3 and one 16-byte store. The s - 1 halo columns left of
        // the tile one output per thread. (s, D are constants where the level
        // loop is unrolled.)
        static_assert(T == 32, "eight column groups per row");
        const int nwd = s > 4 ? 3 : 2;                 // float4 words covering 4 + s columns
        const int wb = -4 * (nwd - 1);                 // the window starts this many columns before c
        for (int e = tid; e < D * 8; e += kThreads) {
            const int r = (e >> 3) - (s - 1), c = 4 * (e & 7);
            const int ia = (r + HALO) * XS + (c + 16);
            const int iz = (r + BO) * XS + (c + 16);
            float a0[12], a1[12], q0[12], q1[12], y0[12], y1[12], v0[12], v1[12];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (q < nwd) {
                    const int o = wb + 4 * q;
                    const float4 t0 = *reinterpret_cast<const float4*>(At + ia + o);
                    const float4 t1 = *reinterpret_cast<const float4*>(At + ia - ra + o);
                    const float4 u0 = *reinterpret_cast<const float4*>(Z1 + iz + o);
                    const float4 u1 = *reinterpret_cast<const float4*>(Z1 + iz - rz + o);
                    const float4 g0 = *reinterpret_cast<const float4*>(Z0 + iz + o);
                    const float4 g1 = *reinterpret_cast<const float4*>(Z0 + iz - rz + o);
                    const float4 h0 = *reinterpret_cast<const float4*>(Z2 + iz + o);
                    const float4 h1 = *reinterpret_cast<const float4*>(Z2 + iz - rz + o);
                    a0[4 * q] = t0.x; a0[4 * q + 1] = t0.y; a0[4 * q + 2] = t0.z; a0[4 * q + 3] = t0.w;
                    a1[4 * q] = t1.x; a1[4 * q + 1] = t1.y; a1[4 * q + 2] = t1.z; a1[4 * q + 3] = t1.w;
                    q0[4 * q] = u0.x; q0[4 * q + 1] = u0.y; q0[4 * q + 2] = u0.z; q0[4 * q + 3] = u0.w;
                    q1[4 * q] = u1.x; q1[4 * q + 1] = u1.y; q1[4 * q + 2] = u1.z; q1[4 * q + 3] = u1.w;
                    y0[4 * q] = g0.x; y0[4 * q + 1] = g0.y; y0[4 * q + 2] = g0.z; y0[4 * q + 3] = g0.w;
                    y1[4 * q] = g1.x; y1[4 * q + 1] = g1.y; y1[4 * q + 2] = g1.z; y1[4 * q + 3] = g1.w;
                    v0[4 * q] = h0.x; v0[4 * q + 1] = h0.y; v0[4 * q + 2] = h0.z; v0[4 * q + 3] = h0.w;
                    v1[4 * q] = h1.x; v1[4 * q + 1] = h1.y; v1[4 * q + 2] = h1.z; v1[4 * q + 3] = h1.w;
                }
            }
            float out[4];
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4) {
                const int kc = -wb + e4, kl = kc - s;  // window positions of columns c + e4 and c + e4 - s
                // rows adjoint at columns c and c - s
                const float lo_c = (a0[kc] + a1[kc]) + (q0[kc] - q1[kc]);
                const float lo_l = (a0[kl] + a1[kl]) + (q0[kl] - q1[kl]);
                const float hi_c = (y0[kc] + y1[kc]) + (v0[kc] - v1[kc]);
                const float hi_l = (y0[kl] + y1[kl]) + (v0[kl] - v1[kl]);
                out[e4] = 0.25f * ((lo_c + lo_l) + (hi_c - hi_l));
            }
            *reinterpret_cast<float4*>(Ao + ia) = make_float4(out[0], out[1], out[2], out[3]);
        }
        for (int e = tid; e < D * (s - 1); e += kThreads) {
            const int rr = e / (s > 1 ? s - 1 : 1), cc = e - rr * (s - 1);
            const int r = rr - (s - 1), c = cc - (s - 1);
            const int ia = (r + HALO) * XS + (c + 16);
            const int iz = (r + BO) * XS + (c + 16);
            const float lo_c = (At[ia] + At[ia - ra]) + (Z1[iz] - Z1[iz - rz]);
            const float lo_l = (At[ia - s] + At[ia - ra - s]) + (Z1[iz - s] - Z1[iz - rz - s]);
            const float hi_c = (Z0[iz] + Z0[iz - rz]) + (Z2[iz] - Z2[iz - rz]);
            const float hi_l = (Z0[iz - s] + Z0[iz - rz - s]) + (Z2[iz - s] - Z2[iz - rz - s]);
            Ao[ia] = 0.25f * ((lo_c + lo_l) + (hi_c - hi_l));
        }
        float* tmp = At;
        At = Ao;
        Ao = tmp;
    }
    __syncthreads();                 // the finest level is complete
    // w = gamma P^T zeta2 on the tile
    const float gam = P.gamma;
    float* __restrict__ ww = P.work + 2 * n;
    for (int r = warp; r < T; r += NWARP)
        ww[(size_t)(R0 + r) * W + (C0 + lane)] = gam * At[(r + HALO) * XS + (lane + 16)];
}

// ---------------------------------------------------------------------------
// forward row DFT of zeta1 + i w and Hermitian split into the half spectra;
// each transform group takes two rows (g and g + G of the CTA's 2 G rows)
// interleaved pass by pass (fft_group2)
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
haar_row_forward(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    constexpr int FT = W / 8, G = kThreads / FT, ROW = W;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    // a problem that has just taken over this slot starts with the column phase
    if (P.ctl->active == 0 || P.ctl->iter == 0) return;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tws = buf + 2 * G * ROW;
    const float2* tw = haar_tw_global<W>() ? tw_g + pass_table_offset<W>() : tws;
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    const int q0 = blockIdx.x * 2 * G + g, q1 = q0 + G;
    const size_t n = (size_t)H * W;
    const float* __restrict__ z1a = P.work + n + (size_t)q0 * W;
    const float* __restrict__ wa = P.work + 2 * n + (size_t)q0 * W;
    const float* __restrict__ z1b = P.work + n + (size_t)q1 * W;
    const float* __restrict__ wb = P.work + 2 * n + (size_t)q1 * W;
    float2 v[8], u[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        v[m] = make_float2(z1a[t + m * FT], wa[t + m * FT]);
        u[m] = make_float2(z1b[t + m * FT], wb[t + m * FT]);
    }
    if (!haar_tw_global<W>()) load_twiddles<W>(tws, tw_g, tid, kThreads);
    __syncthreads();
    float2* row0 = buf + g * ROW;
    float2* row1 = buf + (g + G) * ROW;
    fft_group2<W, -1>(v, u, row0, row1, tw, t, g);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        row0[swz(t + m * FT)] = v[m];
        row1[swz(t + m * FT)] = u[m];
    }
    group_sync<W>(g);                // the split reads this group's rows only
    store_split<W>(P.Sb + (size_t)q0 * Wp, row0, t);
    store_split<W>(P.Sb + (size_t)q1 * Wp, row1, t);
}

// ---------------------------------------------------------------------------
// d2 of every band from the analysis prior's state (zeta2 in d2 buffer 0 and
// the bits), for the state read-out calls
// ---------------------------------------------------------------------------
struct BandConv {
    float tau[3 * kMaxHaarLevels + 1];   // threshold per band (0 on an unpenalised low-low band)
    float izs[3 * kMaxHaarLevels + 1];   // gamma / gamma_b
};

static __global__ void __launch_bounds__(kThreads)
haar_dual_from_state(const float* __restrict__ zeta, const uint32_t* __restrict__ bits, float* __restrict__ d2,
                     long long n, int nb, BandConv c) {
    for (long long p = (long long)blockIdx.x * kThreads + threadIdx.x; p < n; p += (long long)gridDim.x * kThreads) {
        const uint32_t w = bits[p];
        for (int b = 0; b < nb; ++b) d2[b * n + p] = dual_from_zeta(zeta[b * n + p], w >> (2 * b), c.tau[b], c.izs[b]);
    }
}

// ---------------------------------------------------------------------------
// host-side launch of the three row-side kernels of one FA-MD iteration
// ---------------------------------------------------------------------------
template <int W>
cudaError_t launch_haar_rows_t(int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels, bool fs,
                               const float2* tw, int* n_active, cudaStream_t s) {
    constexpr int FT = W / 8, G = kThreads / FT;
    constexpr size_t smem_inv = haar_inv_smem<W>(), smem_fwd = haar_fwd_smem<W>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(haar_row_inverse<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_inv);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(haar_row_forward<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fwd);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nrow = H / G;
    cudaError_t e = launch_chain(haar_row_inverse<W>, dim3(nrow, count), dim3(kThreads), smem_inv, s, d, sl, H, Wp, tw);
    if (e != cudaSuccess) return e;
    const dim3 tgrid(haar_num_tiles(H, W), count);
    switch (levels * 2 + (fs ? 1 : 0)) {
        case 2: e = launch_chain(haar_analysis<1>, tgrid, dim3(kThreads), HaarAnaCfg<1>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        case 4: e = launch_chain(haar_analysis<2>, tgrid, dim3(kThreads), HaarAnaCfg<2>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        case 6: e = launch_chain(haar_analysis<3>, tgrid, dim3(kThreads), HaarAnaCfg<3>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        case 3: e = launch_chain(haar_analysis<1, true>, tgrid, dim3(kThreads), HaarAnaCfg<1>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        case 5: e = launch_chain(haar_analysis<2, true>, tgrid, dim3(kThreads), HaarAnaCfg<2>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        case 7: e = launch_chain(haar_analysis<3, true>, tgrid, dim3(kThreads), HaarAnaCfg<3>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        case 9: e = launch_chain(haar_analysis<4, true>, tgrid, dim3(kThreads), HaarAnaCfg<4>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        default: e = launch_chain(haar_analysis<4>, tgrid, dim3(kThreads), HaarAnaCfg<4>::SMEM, s, d, sl, H, W, nrow, n_active); break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (levels) {
        case 1: e = launch_chain(haar_synthesis<1>, tgrid, dim3(kThreads), HaarSynCfg<1>::SMEM, s, d, sl, H, W); break;
        case 2: e = launch_chain(haar_synthesis<2>, tgrid, dim3(kThreads), HaarSynCfg<2>::SMEM, s, d, sl, H, W); break;
        case 3: e = launch_chain(haar_synthesis<3>, tgrid, dim3(kThreads), HaarSynCfg<3>::SMEM, s, d, sl, H, W); break;
        default: e = launch_chain(haar_synthesis<4>, tgrid, dim3(kThreads), HaarSynCfg<4>::SMEM, s, d, sl, H, W); break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_chain(haar_row_forward<W>, dim3(nrow / 2, count), dim3(kThreads), smem_fwd, s, d, sl, H, Wp, tw);
}

// The kernels of an iteration that run after the one that finishes it: for
// the frame prior the synthesis (w = gamma P^T zeta2) and the forward row
// DFTs of zeta1 + i w; with synth = false only the forward row DFTs. A
// problem that retires skips them in its last iteration (it is inactive by
// then); admm_deconv_get_full_state runs them for it afterwards, so that the
// saved state holds the right-hand side the next x-step would read.
template <int W>
cudaError_t launch_row_tail_t(int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels, bool synth,
                              const float2* tw, cudaStream_t s) {
    constexpr int FT = W / 8, G = kThreads / FT;
    constexpr size_t smem_fwd = haar_fwd_smem<W>();
    cudaError_t e = cudaFuncSetAttribute(haar_row_forward<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_fwd);
    if (e != cudaSuccess) return e;
    if (synth) {
        const dim3 tgrid(haar_num_tiles(H, W), count);
        switch (levels) {
            case 1: haar_synthesis<1><<<tgrid, kThreads, HaarSynCfg<1>::SMEM, s>>>(d, sl, H, W); break;
            case 2: haar_synthesis<2><<<tgrid, kThreads, HaarSynCfg<2>::SMEM, s>>>(d, sl, H, W); break;
            case 3: haar_synthesis<3><<<tgrid, kThreads, HaarSynCfg<3>::SMEM, s>>>(d, sl, H, W); break;
            default: haar_synthesis<4><<<tgrid, kThreads, HaarSynCfg<4>::SMEM, s>>>(d, sl, H, W); break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    haar_row_forward<W><<<dim3(H / G / 2, count), kThreads, smem_fwd, s>>>(d, sl, H, Wp, tw);
    return cudaGetLastError();
}

// Each translation unit has its own copy (internal linkage): a kernel
// launched from two translation units is registered once per unit, and the
// attribute must be set on the copy that the unit launches. A flag shared
// across units (an inline function's static) left one unit's copies unset.
static cudaError_t haar_tile_attributes() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e;
    e = cudaFuncSetAttribute(haar_synthesis<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarSynCfg<1>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_synthesis<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarSynCfg<2>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_synthesis<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarSynCfg<3>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_synthesis<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarSynCfg<4>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarAnaCfg<1>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarAnaCfg<2>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarAnaCfg<3>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarAnaCfg<4>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HaarAnaCfg<1>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HaarAnaCfg<2>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HaarAnaCfg<3>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_analysis<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HaarAnaCfg<4>::SMEM);
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

static inline cudaError_t launch_row_tail(int W, int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels,
                                   bool synth, const float2* tw, cudaStream_t s) {
    cudaError_t e = haar_tile_attributes();
    if (e != cudaSuccess) return e;
    switch (W) {
        case 64: return launch_row_tail_t<64>(H, Wp, d, sl, count, levels, synth, tw, s);
        case 128: return launch_row_tail_t<128>(H, Wp, d, sl, count, levels, synth, tw, s);
        case 256: return launch_row_tail_t<256>(H, Wp, d, sl, count, levels, synth, tw, s);
        case 512: return launch_row_tail_t<512>(H, Wp, d, sl, count, levels, synth, tw, s);
        case 1024: return launch_row_tail_t<1024>(H, Wp, d, sl, count, levels, synth, tw, s);
        case 2048: return launch_row_tail_t<2048>(H, Wp, d, sl, count, levels, synth, tw, s);
    }
    return cudaErrorInvalidValue;
}

// fs: the synthesis formulation (FS-MD) analysis tile
static inline cudaError_t launch_haar_iteration_rows(int W, int H, int Wp, const ProbDesc* d, SlotTable sl, int count,
                                              int levels, bool fs, const float2* tw, int* n_active, cudaStream_t s) {
    cudaError_t e = haar_tile_attributes();
    if (e != cudaSuccess) return e;
    switch (W) {
        case 64: return launch_haar_rows_t<64>(H, Wp, d, sl, count, levels, fs, tw, n_active, s);
        case 128: return launch_haar_rows_t<128>(H, Wp, d, sl, count, levels, fs, tw, n_active, s);
        case 256: return launch_haar_rows_t<256>(H, Wp, d, sl, count, levels, fs, tw, n_active, s);
        case 512: return launch_haar_rows_t<512>(H, Wp, d, sl, count, levels, fs, tw, n_active, s);
        case 1024: return launch_haar_rows_t<1024>(H, Wp, d, sl, count, levels, fs, tw, n_active, s);
        case 2048: return launch_haar_rows_t<2048>(H, Wp, d, sl, count, levels, fs, tw, n_active, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace admm
