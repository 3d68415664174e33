// cg.cuh -- the Reeves-Sorel variants TV-CG and FA-CG (Sec. IV-C/IV-D,
// "Using the Reeves-Sorel technique").
//
// There the observation split is u1 = M A x with g1(u) = 1/2 ||y - u||^2 on
// the observed pixels (eq. H_1_analysis_sorel), and the x-step inverse
// (A^T M^T M A + gamma D^T D)^{-1} (TV) or (A^T M^T M A + gamma I)^{-1}
// (frame) is applied as C - C B^T (B C B^T - I)^{-1} B C (eqs. ReevesTV,
// reeves3), C the circulant inverse the column phase already applies and B
// the rows of A at the unobserved pixels U. The inner system takes one
// conjugate-gradient iteration per outer iteration, warm-started from the
// previous one (Sec. IV-B).
//
// The kernels carry the inner unknown as z = -xi (xi the paper's unknown),
// which solves the positive definite (I - B C B^T) z = B C r; CG takes the
// same steps on either sign. With r = A^T M^T zeta1 + w (w = gamma D^T delta
// or gamma P^T zeta2) one outer iteration is:
//   1. x~ = C (r + B^T z)            -- the column phase on the row DFTs of
//                                       zeta~ + i w, where zeta~ holds zeta1
//                                       on observed pixels and z on U (so
//                                       A^T zeta~ = A^T M^T zeta1 + B^T z)
//   2. s = B x~ - z                   -- the CG residual at the warm start
//                                       (cg_row_a, which also sends s + i 0
//                                       to the row DFTs for step 3)
//   3. v = C A^T s, A v               -- the column phase again
//   4. alpha = s.s / s.(s - B v)      -- the exact step along s (cg_row_b;
//                                       its last CTA divides)
//   5. x = x~ + alpha v, A x likewise, z += alpha s; then the observation
//      prox and dual update on the observed pixels (cg_obs), and the
//      regulariser side as for the MD methods (tv_tile for TV; the frame
//      analysis and synthesis tiles for the frame prior), which finishes
//      the iteration; the forward row DFTs of zeta~ + i w close it.
// Per-pixel planes (ProbDesc::cg): x~, A x~, v, A v, s, z.
#pragma once
#include "haar.cuh"
#include "variants.cuh"

namespace admm {

// Block sum of one compensated FP32 accumulator into thread 0 (FP64).
__device__ __forceinline__ double block_sum_comp(const CompSum& a, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float s = a.s, c = a.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) red[warp] = (double)s + (double)c;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}

// ---------------------------------------------------------------------------
// step 2: inverse row DFTs -> x~, A x~; s = A x~ - z on U (0 elsewhere);
// forward row DFTs of s + i 0 -> Sb. Grid: (H / G, slots), G rows per CTA.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
cg_row_a(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    constexpr int FT = W / 8, G = kThreads / FT;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const int k = P.ctl->iter + 1;
    const bool cold = k == 1 && !P.warm;         // z = 0 at the start
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = buf + G * W;
    double* red = reinterpret_cast<double*>(tw + W);
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    const int q = blockIdx.x * G + g;
    const size_t n = (size_t)H * W;
    load_twiddles<W>(tw, tw_g, tid, kThreads);
    __syncthreads();
    float2 v[8];
    load_row_xax<W>(v, P.Sa + (size_t)q * Wp, t);
    float2* row = buf + g * W;
    fft_group<W, 1>(v, row, tw, t, g);
    float* __restrict__ X = P.cg;
    float* __restrict__ AX = P.cg + n;
    float* __restrict__ Sv = P.cg + 4 * n;
    const float* __restrict__ Z = P.cg + 5 * n;
    CompSum ss;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const size_t pix = (size_t)q * W + t + m * FT;
        const float x = v[m].x, ax = v[m].y;
        const bool obs = is_observed(P.ybar[pix]);
        const float s = obs ? 0.f : ax - (cold ? 0.f : Z[pix]);
        X[pix] = x;
        AX[pix] = ax;
        Sv[pix] = s;
        ss.add(s * s);
        v[m] = make_float2(s, 0.f);
    }
    fft_group<W, -1>(v, row, tw, t, g);
#pragma unroll
    for (int m = 0; m < 8; ++m) row[swz(t + m * FT)] = v[m];
    group_sync<W>(g);                // the split reads this group's row only
    store_split<W>(P.Sb + (size_t)q * Wp, row, t);
    const double tot = block_sum_comp(ss, red);
    if (tid == 0) P.cg_part[blockIdx.x] = tot;
}

// ---------------------------------------------------------------------------
// step 4: inverse row DFTs -> v = C A^T s, A v; the CTA's share of
// s.(s - A v) over U; the last CTA of the problem reduces both sums in a
// fixed order and sets alpha. Grid: (H / G, slots).
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
cg_row_b(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int Wp, const float2* __restrict__ tw_g) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    constexpr int FT = W / 8, G = kThreads / FT;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    ProbCtl* ctl = P.ctl;
    if (ctl->active == 0) return;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = buf + G * W;
    double* red = reinterpret_cast<double*>(tw + W);
    __shared__ int s_last;
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    const int q = blockIdx.x * G + g;
    const int nrow = H / G;
    const size_t n = (size_t)H * W;
    load_twiddles<W>(tw, tw_g, tid, kThreads);
    __syncthreads();
    float2 v[8];
    load_row_xax<W>(v, P.Sa + (size_t)q * Wp, t);
    fft_group<W, 1>(v, buf + g * W, tw, t, g);
    float* __restrict__ V = P.cg + 2 * n;
    float* __restrict__ AV = P.cg + 3 * n;
    const float* __restrict__ Sv = P.cg + 4 * n;
    CompSum den;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const size_t pix = (size_t)q * W + t + m * FT;
        V[pix] = v[m].x;
        AV[pix] = v[m].y;
        const float s = Sv[pix];                  // 0 on observed pixels
        den.add(s * (s - v[m].y));
    }
    const double tot = block_sum_comp(den, red);
    if (tid == 0) {
        P.cg_part[nrow + blockIdx.x] = tot;
        __threadfence();
        s_last = atomicAdd(&ctl->cg_arrive, 1u) == (unsigned)(nrow - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // the last CTA: both sums over all row CTAs, each thread a fixed strided
    // share, then a fixed tree (reproducible)
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = tid; i < nrow; i += kThreads) {
        a += __ldcg(P.cg_part + i);
        b += __ldcg(P.cg_part + nrow + i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red[warp] = a;
        red[kThreads / 32 + warp] = b;
    }
    __syncthreads();
    if (tid == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            ta += red[w];
            tb += red[kThreads / 32 + w];
        }
        // s = 0 (nothing unobserved, or already solved): no step
        ctl->cg_alpha = (ta > 0.0 && tb > 0.0) ? (float)(ta / tb) : 0.f;
        ctl->cg_arrive = 0u;
    }
}

// ---------------------------------------------------------------------------
// step 5, observation side: x = x~ + alpha v, A x = A x~ + alpha A v; on
// observed pixels u1 = (y + mu1 (A x - d1)) / (1 + mu1), d1 <- d1 - (A x - u1)
// (prox of g1 = 1/2 ||y - u||^2 and Alg. 3 line 8 with M A); on U z += alpha s.
// Writes x and zeta~ (zeta1 = u1 + d1 on observed pixels, z on U) to the
// scratch planes, and the data-term, rel-x and d1 partial sums in the slots
// of the row kernels. Grid: (H / G, slots), the row kernels' layout.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads)
cg_obs(const ProbDesc* __restrict__ probs, SlotTable sl, int H) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    constexpr int FT = W / 8, G = kThreads / FT;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const int k = P.ctl->iter + 1;
    const bool first = k == 1;                   // x_prev = 0 (no earlier iterate)
    const bool cold = first && !P.warm;          // d1 = 0, z = 0
    const bool chk = is_check_iter(P, k), sprev = store_prev_iter(P, k), nobj = need_obj_iter(P, k);
    __shared__ float red[kThreads / 32 * 2 * kNumPartials];
    const int tid = threadIdx.x, g = tid / FT, t = tid % FT;
    const int q = blockIdx.x * G + g;
    const size_t n = (size_t)H * W;
    const float alpha = P.ctl->cg_alpha;
    const float* __restrict__ X = P.cg;
    const float* __restrict__ AX = P.cg + n;
    const float* __restrict__ V = P.cg + 2 * n;
    const float* __restrict__ AV = P.cg + 3 * n;
    const float* __restrict__ Sv = P.cg + 4 * n;
    float* __restrict__ Z = P.cg + 5 * n;
    float* __restrict__ xw = P.work;
    float* __restrict__ z1w = P.work + n;
    const float mu1 = P.mu1, inv1 = P.inv1pmu1;
    CompSum s_data, s_xx, s_dxx, s_pr;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const size_t pix = (size_t)q * W + t + m * FT;
        const float x = fmaf(alpha, V[pix], X[pix]);
        const float ax = fmaf(alpha, AV[pix], AX[pix]);
        const float yb = P.ybar[pix];
        float z1;
        if (is_observed(yb)) {
            const float dd1 = cold ? 0.f : P.d1[pix];
            const float u1 = fmaf(mu1, ax - dd1, yb) * inv1;
            const float nd1 = dd1 - (ax - u1);
            P.d1[pix] = nd1;
            z1 = u1 + nd1;
            if (nobj) {
                const float e = ax - yb;
                s_data.add(0.5f * e * e);
                const float e1 = nd1 - dd1;
                s_pr.add(e1 * e1);
            }
        } else {
            z1 = fmaf(alpha, Sv[pix], cold ? 0.f : Z[pix]);
            Z[pix] = z1;
            P.d1[pix] = 0.f;
        }
        xw[pix] = x;
        z1w[pix] = z1;
        if (chk) {
            const float dx = first ? x : x - P.xprev[pix];
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
// TV regulariser side on a 32 x 32 tile (Alg. 3 lines 9-11 and lines 3-5 of
// the next iteration), for TV-CG and for TV-MD on domains whose sides are
// not both powers of two: D x with forward periodic differences, vector-soft
// (ANISO: eq. soft per component) with tau = lambda / mu2, d2 <- d2 -
// (D x - u2), delta = u2 + d2 and w = gamma (Dh^T delta_h + Dv^T delta_v).
// w at a pixel needs delta one column left and one row up, so the tile
// recomputes delta on that halo from x (one more row and column of x) and
// the previous d2 (double-buffered by iteration parity, so a neighbour's halo
// always sees the old d2). Finishes the iteration. Grid: (tiles, slots).
// H and W are multiples of 32 (not necessarily powers of two).
// ---------------------------------------------------------------------------
constexpr int kCgTile = 32;
// periodic index for x in [-n, 2n)
__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }
template <bool ANISO = false>
__global__ void __launch_bounds__(kThreads)
tv_tile(const ProbDesc* __restrict__ probs, SlotTable sl, int H, int W, int n_row_ctas,
        int* __restrict__ n_active) {
    chain_wait();   // (launch chain: the predecessor's writes are visible)
    constexpr int T = kCgTile, XR = T + 2, XS = T + 3, DR = T + 1;
    const int pi = sl.map[blockIdx.y];
    if (pi < 0) return;
    const ProbDesc& P = probs[pi];
    if (P.ctl->active == 0) return;
    const int k = P.ctl->iter + 1;
    const bool first = k == 1 && !P.warm;        // d2 = 0 (cold start)
    const bool chk = is_check_iter(P, k), nobj = need_obj_iter(P, k);
    __shared__ float xs[XR * XS];                // x on rows R0-1 .. R0+T, columns C0-1 .. C0+T
    __shared__ float2 dl[DR * DR];               // delta on rows R0-1 .. R0+T-1, columns C0-1 .. C0+T-1
    __shared__ __align__(8) float2 d2s[DR * DR]; // the previous d2 on the same region
    __shared__ float red[kThreads / 32 * 2 * kNumPartials];
    const int tid = threadIdx.x;
    const int tiles_x = W / T;
    const int R0 = (blockIdx.x / tiles_x) * T, C0 = (blockIdx.x % tiles_x) * T;
    const size_t n = (size_t)H * W;
    const float* __restrict__ xw = P.work;
    const float2* __restrict__ d2in = reinterpret_cast<const float2*>(P.d2 + ((k + 1) & 1) * P.d2_stride);
    float2* __restrict__ d2out = reinterpret_cast<float2*>(P.d2 + (k & 1) * P.d2_stride);
    // x and the previous d2 of the region requested together (cp.async)
    for (int e = tid; e < XR * XR; e += kThreads) {
        const int rr = e / XR, cc = e - rr * XR;
        const int r = wrapi(R0 - 1 + rr, H), c = wrapi(C0 - 1 + cc, W);
        cp_async4(&xs[rr * XS + cc], xw + (size_t)r * W + c);
    }
    if (!first) {
        for (int e = tid; e < DR * DR; e += kThreads) {
            const int rr = e / DR, cc = e - rr * DR;
            const int r = wrapi(R0 - 1 + rr, H), c = wrapi(C0 - 1 + cc, W);
            cp_async8(&d2s[e], d2in + (size_t)r * W + c);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const float tau = P.tau;
    CompSum tvs, prs;
    for (int e = tid; e < DR * DR; e += kThreads) {
        const int rr = e / DR, cc = e - rr * DR;
        const int r = wrapi(R0 - 1 + rr, H), c = wrapi(C0 - 1 + cc, W);
        const size_t pix = (size_t)r * W + c;
        const float x0 = xs[rr * XS + cc];
        const float gh = xs[rr * XS + cc + 1] - x0;
        const float gv = xs[(rr + 1) * XS + cc] - x0;
        const float2 dold = first ? make_float2(0.f, 0.f) : d2s[e];
        float uh, uv;
        tv_prox(gh - dold.x, gv - dold.y, tau, ANISO, uh, uv);
        const float ndh = dold.x - (gh - uh), ndv = dold.y - (gv - uv);
        dl[rr * DR + cc] = make_float2(uh + ndh, uv + ndv);
        if (rr >= 1 && cc >= 1) {                // a pixel of the tile: owned
            d2out[pix] = make_float2(ndh, ndv);
            if (nobj) {
                tvs.add(tv_norm(gh, gv, ANISO));
                const float eh = ndh - dold.x, ev = ndv - dold.y;
                prs.add(fmaf(eh, eh, ev * ev));
            }
        }
    }
    __syncthreads();
    const float gam = P.gamma;
    float* __restrict__ ww = P.work + 2 * n;
    for (int e = tid; e < T * T; e += kThreads) {
        const int rr = e / T + 1, cc = e % T + 1;
        const float2 d = dl[rr * DR + cc];
        const float wv = gam * ((dl[rr * DR + cc - 1].x - d.x) + (dl[(rr - 1) * DR + cc].y - d.y));
        ww[(size_t)(R0 + rr - 1) * W + (C0 + cc - 1)] = wv;
    }
    double pv[kNumPartials] = {0.0};
    if (nobj || chk) {
        const CompSum acc[kNumPartials] = {CompSum(), tvs, CompSum(), CompSum(), prs};
        block_reduce_comp(acc, red, pv);
    }
    finish_iteration<kThreads>(P, k, chk, nobj, pv, n_active, n_row_ctas + blockIdx.x, probs, sl);
}

inline int cg_num_tiles(int H, int W) { return (H / kCgTile) * (W / kCgTile); }

// One TV-CG (tv = true) or FA-CG iteration of a lane: the two column phases
// (col_fn) and the row-side kernels, as a launch chain (cg.cu).
cudaError_t launch_cg_iteration(int W, int H, int Wc, int Wp, const ProbDesc* d, SlotTable sl, int count,
                                int levels, bool tv, ColLaunchFn col_fn, const float2* tw, int* n_active,
                                cudaStream_t s);

}  // namespace admm
