// haar.cuh -- row side of FA-MD (frame-based analysis prior, Sec. IV-C).
//
// One FA-MD iteration (Algorithm 2 with H1 = A, H2 = P) after the column
// phase has produced the row spectra of (x, A x):
//
//   haar_row_inverse   inverse row DFTs -> x, A x; mask-decoupled prox and
//                      dual update (eq. prox_g_1_uBC, Alg. 2 lines 6-7, j = 1);
//                      writes x and zeta1 = u1 + d1 to two scratch planes
//   haar_tile          32 x 32 output tile with a halo of 2^L - 1 pixels:
//                      analysis c = P x (a-trous Haar), u2 = soft(c - d2,
//                      lambda/mu2) (eq. soft), d2 <- d2 - (c - u2), zeta2 =
//                      u2 + d2, then w = gamma P^T zeta2 (the x-step right-hand
//                      side of eq. invAnalysis divided by mu1) on the tile
//   haar_row_forward   forward row DFT of zeta1 + i w, split into half spectra
//
// P is the undecimated Haar frame with periodic wrap: level j filters with
// h = [1/2, 1/2] and g = [1/2, -1/2] at taps {0, 2^j}, emits three detail
// bands and passes the low-low band on; the last low-low band is kept
// (3 L + 1 bands, P^T P = I). Band order per level: rows low / columns high,
// rows high / columns low, rows high / columns high; final band low-low.
//
// The tile recomputes the coefficients of its halo from x and the previous
// iteration's d2, so d2 is double-buffered by iteration parity (a CTA never
// reads a d2 value a neighbouring CTA has already replaced).
#pragma once
#include <cuda_runtime.h>
#include "kernels.cuh"

namespace admm {

constexpr int kMaxHaarLevels = 4;
constexpr int kHaarTile = 32;

// rows per CTA of the two row kernels: one row transform per thread group
inline int haar_rows_per_cta(int W) { return kThreads / (W / 8); }
inline int haar_row_strip(int W) { return haar_rows_per_cta(W); }
inline int haar_num_row_ctas(int H, int W) { return H / haar_rows_per_cta(W); }
inline int haar_num_tiles(int H, int W) { return (H / kHaarTile) * (W / kHaarTile); }

// ---------------------------------------------------------------------------
// inverse row DFT + mask prox + d1 dual (no halo: every row is owned)
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
haar_row_inverse(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g) {
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
    float2* tw = buf + G * ROW;
    double* red = reinterpret_cast<double*>(tw + W);
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    load_twiddles<W>(tw, tw_g, tid, kThreads);
    __syncthreads();
    const int q = blockIdx.x * G + g;
    float2 v[8];
    load_row_xax<W>(v, P.Sa + (size_t)q * Wp, t);
    fft_group<W, 1>(v, buf + g * ROW, tw, t, g);
    const size_t n = (size_t)H * W;
    float* __restrict__ xw = P.work;
    float* __restrict__ z1w = P.work + n;
    const float mu1 = P.mu1, inv1 = P.inv1pmu1;
    CompSum s_data, s_xx, s_dxx;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int c = t + m * FT;
        const size_t pix = (size_t)q * W + c;
        const float x = v[m].x, ax = v[m].y;
        // u1 = (M^T M + mu1 I)^{-1} (M^T y + mu1 (A x - d1)); d1 <- d1 - (A x - u1)
        const float dd1 = cold ? 0.f : P.d1[pix];
        const float s1 = ax - dd1;
        const float yb = P.ybar[pix];
        const bool obs = is_observed(yb);
        const float u1 = obs ? fmaf(mu1, s1, yb) * inv1 : s1;
        const float nd1 = dd1 - (ax - u1);
        P.d1[pix] = nd1;
        z1w[pix] = u1 + nd1;
        xw[pix] = x;
        if (nobj && obs) {
            const float e = ax - yb;
            s_data.add(0.5f * e * e);
        }
        if (chk) {
            const float dx = first ? x : x - P.xprev[pix];
            s_dxx.add(dx * dx);
            s_xx.add(x * x);
        }
        if (sprev) P.xprev[pix] = x;
    }
    const CompSum acc[kNumPartials] = {s_data, CompSum(), s_xx, s_dxx};
    double pv[kNumPartials];
    block_reduce_comp(acc, reinterpret_cast<float*>(red), pv);
    if (tid == 0) {
#pragma unroll
        for (int j = 0; j < kNumPartials; ++j) P.partials[blockIdx.x * kNumPartials + j] = pv[j];
    }
}

// ---------------------------------------------------------------------------
// frame analysis, soft threshold, dual update and adjoint synthesis on a tile
// ---------------------------------------------------------------------------
template <int L>
struct HaarTileCfg {
    static constexpr int T = kHaarTile;
    static constexpr int HALO = (1 << L) - 1;
    static constexpr int XD = T + 2 * HALO;       // side of the x / approximation arrays
    __host__ __device__ static constexpr int band_side(int lvl) { return T + 2 * (1 << lvl) - 1; }
    __host__ __device__ static constexpr int zoff(int lvl) {
        int o = 0;
        for (int i = 0; i < lvl; ++i) o += 3 * band_side(i) * band_side(i);
        return o;
    }
    static constexpr int ZTOT = zoff(L);
    static constexpr int LLD = T + HALO;          // side of the low-low band region
    // the reduction scratch follows the float arrays: round up to 8 bytes
    static constexpr int RED_OFF = (2 * XD * XD + ZTOT + LLD * LLD + 1) & ~1;   // in floats
    static_assert((RED_OFF * sizeof(float)) % sizeof(double) == 0, "double alignment");
    static constexpr size_t SMEM = (size_t)RED_OFF * sizeof(float) + 8 * kNumPartials * sizeof(double);
};

__device__ __forceinline__ float soft_thresh(float v, float t) {
    const float a = fabsf(v) - t;
    return a > 0.f ? copysignf(a, v) : 0.f;
}

template <int L>
__global__ void __launch_bounds__(kThreads)
haar_tile(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int W, int n_row_ctas, int* __restrict__ n_active) {
    using C = HaarTileCfg<L>;
    constexpr int T = C::T, HALO = C::HALO, XD = C::XD;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    ProbCtl* ctl = P.ctl;
    if (ctl->active == 0) return;
    const int k = ctl->iter + 1;
    const bool first = k == 1 && !P.warm;        // d2 = 0 (cold start: u0 = d0 = 0)
    const bool chk = is_check_iter(P, k), nobj = need_obj_iter(P, k);
    extern __shared__ __align__(16) float sm[];
    float* A0 = sm;
    float* A1 = A0 + XD * XD;
    float* Z = A1 + XD * XD;                     // detail bands: d2 staged, then zeta2
    float* ZLL = Z + C::ZTOT;                    // low-low band: d2 staged
    double* red = reinterpret_cast<double*>(sm + C::RED_OFF);
    const int tid = threadIdx.x;
    const int tiles_x = W / T;
    const int R0 = (blockIdx.x / tiles_x) * T, C0 = (blockIdx.x % tiles_x) * T;
    const size_t n = (size_t)H * W;
    const float* __restrict__ xw = P.work;
    float* __restrict__ ww = P.work + 2 * n;
    const float* __restrict__ d2in = P.d2 + ((k + 1) & 1) * P.d2_stride;
    float* __restrict__ d2out = P.d2 + (k & 1) * P.d2_stride;
    const float tau = P.tau;

    // Regions are visited two-dimensionally: warp w takes rows w, w + 8, ...
    // and lane l columns l, l + 32, ... of the region, so positions come from
    // counters rather than divisions, and the wrapped global row is computed
    // once per row.
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NWARP = kThreads / 32;

    // every input of the tile is requested at once (cp.async): x on
    // [-HALO, T + HALO)^2 and the previous d2 of each band on the region where
    // its zeta2 is needed (periodic wrap)
    for (int rr = warp; rr < XD; rr += NWARP) {
        const float* src = xw + (size_t)((R0 + rr - HALO) & (H - 1)) * W;
        for (int cc = lane; cc < XD; cc += 32) cp_async4(A0 + rr * XD + cc, src + ((C0 + cc - HALO) & (W - 1)));
    }
    if (!first) {
#pragma unroll
        for (int lvl = 0; lvl < L; ++lvl) {
            const int BO = 2 * (1 << lvl) - 1, BD = T + 2 * (1 << lvl) - 1;
            float* Zl = Z + C::zoff(lvl);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float* band = d2in + (size_t)(3 * lvl + j) * n;
                for (int rr = warp; rr < BD; rr += NWARP) {
                    const float* src = band + (size_t)((R0 + rr - BO) & (H - 1)) * W;
                    for (int cc = lane; cc < BD; cc += 32)
                        cp_async4(Zl + j * BD * BD + rr * BD + cc, src + ((C0 + cc - BO) & (W - 1)));
                }
            }
        }
        const float* band = d2in + (size_t)(3 * L) * n;
        for (int rr = warp; rr < C::LLD; rr += NWARP) {
            const float* src = band + (size_t)((R0 + rr - HALO) & (H - 1)) * W;
            for (int cc = lane; cc < C::LLD; cc += 32)
                cp_async4(ZLL + rr * C::LLD + cc, src + ((C0 + cc - HALO) & (W - 1)));
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();

    CompSum l1;
    float* Ain = A0;
    float* Aout = A1;
    // analysis, level by level: a_{j+1} and the three detail bands from a_j
    // (levels unrolled: every region size below is a compile-time constant)
#pragma unroll
    for (int lvl = 0; lvl < L; ++lvl) {
        const int s = 1 << lvl;
        const int D = T + 2 * HALO + 1 - 2 * s;       // a_{j+1} is needed on [-HALO, D - HALO)
        const int BO = 2 * s - 1, BD = T + 2 * s - 1;  // band region [-BO, T)
        float* Zl = Z + C::zoff(lvl);
        for (int rr = warp; rr < D; rr += NWARP) {
            const int r = rr - HALO;
            const bool band_row = r >= -BO && r < T;
            const size_t grow = (size_t)((R0 + r) & (H - 1)) * W;
            for (int cc = lane; cc < D; cc += 32) {
                const int c = cc - HALO;
                const int i00 = rr * XD + cc;
                const float a00 = Ain[i00], a01 = Ain[i00 + s];
                const float a10 = Ain[i00 + s * XD], a11 = Ain[i00 + s * XD + s];
                const float p0 = a00 + a01, m0 = a00 - a01, p1 = a10 + a11, m1 = a10 - a11;
                Aout[i00] = 0.25f * (p0 + p1);
                if (band_row && c >= -BO && c < T) {
                    const float cb[3] = {0.25f * (m0 + m1), 0.25f * (p0 - p1), 0.25f * (m0 - m1)};
                    const size_t gpix = grow + ((C0 + c) & (W - 1));
                    const bool own = r >= 0 && c >= 0;
                    const int iz = (r + BO) * BD + (c + BO);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float sv = first ? cb[j] : cb[j] - Zl[j * BD * BD + iz];
                        const float u = soft_thresh(sv, tau);
                        const float nd = u - sv;                   // d2 - (c - u2)
                        Zl[j * BD * BD + iz] = u + nd;              // zeta2 = u2 + d2
                        if (own) {
                            d2out[(size_t)(3 * lvl + j) * n + gpix] = nd;
                            if (nobj) l1.add(fabsf(cb[j]));
                        }
                    }
                }
            }
        }
        __syncthreads();
        float* tmp = Ain; Ain = Aout; Aout = tmp;
    }
    // last low-low band (a_L on [-HALO, T)), thresholded in place
    {
        constexpr int D = T + HALO;
        for (int rr = warp; rr < D; rr += NWARP) {
            const int r = rr - HALO;
            const size_t grow = (size_t)((R0 + r) & (H - 1)) * W;
            for (int cc = lane; cc < D; cc += 32) {
                const int c = cc - HALO;
                const int i = rr * XD + cc;
                const float cb = Ain[i];
                const float sv = first ? cb : cb - ZLL[rr * C::LLD + cc];
                const float u = soft_thresh(sv, tau);
                const float nd = u - sv;
                Ain[i] = u + nd;
                if (r >= 0 && c >= 0) {
                    d2out[(size_t)(3 * L) * n + grow + ((C0 + c) & (W - 1))] = nd;
                    if (nobj) l1.add(fabsf(cb));
                }
            }
        }
        __syncthreads();
    }
    // synthesis (adjoint), coarse to fine: a~_j from a~_{j+1} and the zeta bands of level j
    float* At = Ain;
    float* Ao = Aout;
#pragma unroll
    for (int lvl = L - 1; lvl >= 0; --lvl) {
        const int s = 1 << lvl;
        const int D = T + s - 1;                       // output on [-(s-1), T)
        const int BO = 2 * s - 1, BD = T + 2 * s - 1;
        const float* Z0 = Z + C::zoff(lvl);
        const float* Z1 = Z0 + BD * BD;
        const float* Z2 = Z1 + BD * BD;
        const int ra = s * XD, rz = s * BD;
        for (int rr = warp; rr < D; rr += NWARP) {
            const int r = rr - (s - 1);
            for (int cc = lane; cc < D; cc += 32) {
                const int c = cc - (s - 1);
                const int ia = (r + HALO) * XD + (c + HALO);
                const int iz = (r + BO) * BD + (c + BO);
                // rows adjoint at columns c and c - s
                const float lo_c = (At[ia] + At[ia - ra]) + (Z1[iz] - Z1[iz - rz]);
                const float lo_l = (At[ia - s] + At[ia - ra - s]) + (Z1[iz - s] - Z1[iz - rz - s]);
                const float hi_c = (Z0[iz] + Z0[iz - rz]) + (Z2[iz] - Z2[iz - rz]);
                const float hi_l = (Z0[iz - s] + Z0[iz - rz - s]) + (Z2[iz - s] - Z2[iz - rz - s]);
                Ao[ia] = 0.25f * ((lo_c + lo_l) + (hi_c - hi_l));
            }
        }
        __syncthreads();
        float* tmp = At; At = Ao; Ao = tmp;
    }
    // w = gamma P^T zeta2 on the tile
    const float gam = P.gamma;
    for (int r = warp; r < T; r += NWARP)
        ww[(size_t)(R0 + r) * W + (C0 + lane)] = gam * At[(r + HALO) * XD + (lane + HALO)];
    const CompSum acc[kNumPartials] = {CompSum(), l1, CompSum(), CompSum()};
    double pv[kNumPartials];
    block_reduce_comp(acc, reinterpret_cast<float*>(red), pv);
    finish_iteration<kThreads>(P, k, chk, nobj, pv, n_active, n_row_ctas + blockIdx.x, probs, sl);
}

// ---------------------------------------------------------------------------
// forward row DFT of zeta1 + i w and Hermitian split into the half spectra
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
haar_row_forward(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g) {
    constexpr int FT = W / 8, G = kThreads / FT, ROW = W;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    // a problem that has just taken over this slot starts with the column phase
    if (P.ctl->active == 0 || P.ctl->iter == 0) return;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = buf + G * ROW;
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    load_twiddles<W>(tw, tw_g, tid, kThreads);
    __syncthreads();
    const int q = blockIdx.x * G + g;
    const size_t n = (size_t)H * W;
    const float* __restrict__ z1w = P.work + n + (size_t)q * W;
    const float* __restrict__ ww = P.work + 2 * n + (size_t)q * W;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = make_float2(z1w[t + m * FT], ww[t + m * FT]);
    float2* row = buf + g * ROW;
    fft_group<W, -1>(v, row, tw, t, g);
#pragma unroll
    for (int m = 0; m < 8; ++m) row[swz(t + m * FT)] = v[m];
    group_sync<W>(g);                // the split reads this group's row only
    store_split<W>(P.Sb + (size_t)q * Wp, row, t);
}

// ---------------------------------------------------------------------------
// host-side launch of the three row-side kernels of one FA-MD iteration
// ---------------------------------------------------------------------------
template <int W>
cudaError_t launch_haar_rows_t(int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels,
                               const float2* tw, int* n_active, cudaStream_t s) {
    constexpr int FT = W / 8, G = kThreads / FT;
    const size_t smem_row = (size_t)(G * W + W) * sizeof(float2) + 8 * kNumPartials * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(haar_row_inverse<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(haar_row_forward<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nrow = H / G;
    haar_row_inverse<W><<<dim3(nrow, count), kThreads, smem_row, s>>>(d, sl, H, Wp, tw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 tgrid(haar_num_tiles(H, W), count);
    switch (levels) {
        case 1: haar_tile<1><<<tgrid, kThreads, HaarTileCfg<1>::SMEM, s>>>(d, sl, H, W, nrow, n_active); break;
        case 2: haar_tile<2><<<tgrid, kThreads, HaarTileCfg<2>::SMEM, s>>>(d, sl, H, W, nrow, n_active); break;
        case 3: haar_tile<3><<<tgrid, kThreads, HaarTileCfg<3>::SMEM, s>>>(d, sl, H, W, nrow, n_active); break;
        default: haar_tile<4><<<tgrid, kThreads, HaarTileCfg<4>::SMEM, s>>>(d, sl, H, W, nrow, n_active); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    haar_row_forward<W><<<dim3(nrow, count), kThreads, smem_row, s>>>(d, sl, H, Wp, tw);
    return cudaGetLastError();
}

inline cudaError_t haar_tile_attributes() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e;
    e = cudaFuncSetAttribute(haar_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarTileCfg<1>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_tile<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarTileCfg<2>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_tile<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarTileCfg<3>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(haar_tile<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HaarTileCfg<4>::SMEM);
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

inline cudaError_t launch_haar_iteration_rows(int W, int H, int Wp, const ProbDesc* d, SlotTable sl, int count,
                                              int levels, const float2* tw, int* n_active, cudaStream_t s) {
    cudaError_t e = haar_tile_attributes();
    if (e != cudaSuccess) return e;
    switch (W) {
        case 64: return launch_haar_rows_t<64>(H, Wp, d, sl, count, levels, tw, n_active, s);
        case 128: return launch_haar_rows_t<128>(H, Wp, d, sl, count, levels, tw, n_active, s);
        case 256: return launch_haar_rows_t<256>(H, Wp, d, sl, count, levels, tw, n_active, s);
        case 512: return launch_haar_rows_t<512>(H, Wp, d, sl, count, levels, tw, n_active, s);
        case 1024: return launch_haar_rows_t<1024>(H, Wp, d, sl, count, levels, tw, n_active, s);
        case 2048: return launch_haar_rows_t<2048>(H, Wp, d, sl, count, levels, tw, n_active, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace admm
