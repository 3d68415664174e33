// setup.cuh -- per-plan and per-solve set-up kernels (spectra of the
// x-step, M^T y, control blocks, slot assignment). Included by the engine's
// translation unit only; the iteration kernels live in kernels.cuh / haar.cuh.
#pragma once
#include "kernels.cuh"

namespace admm {

// ---------------------------------------------------------------------------
// a0: plan precompute. Lambda[kr,kc] = sum_{a,b} h[a+lr,b+lc] exp(-2 pi i (kr a/H + kc b/W))
// (DFT of the kernel centred at (0,0), eq. DFT_fact) for the half spectrum
// kc = 0..W/2, and the diagonal inverse of eq. fast_inversion (TV, divided by
// mu1) or eq. invAnalysisp1 (frame), times 1/(HW). FP64, rounded once to FP32.
// ---------------------------------------------------------------------------
// Per-band weights gamma_b = mu_b / mu1 of the frame prior (one penalty per
// band, eq. diagonal_penalty): sum_b gamma_b |H_b|^2 replaces gamma in the
// denominator, |H_b|^2 the power spectrum of band b of the a-trous Haar frame
// (per axis cos^2 / sin^2 of pi k 2^j / N for the low / high filter of
// level j, the low filters of the earlier levels in front). levels = 0: off.
struct BandWeights {
    double g[13];
    int levels;
};

__device__ __forceinline__ double band_weighted_power(const BandWeights& bw, int kr, int kc, int H, int W) {
    double acc = 0.0, chain = 1.0;
    for (int j = 0; j < bw.levels; ++j) {
        const long long mr = ((long long)kr << j) % H, mc = ((long long)kc << j) % W;
        const double cr = cospi((double)mr / (double)H), cc = cospi((double)mc / (double)W);
        const double lr = cr * cr, lc = cc * cc;          // low-pass power of level j per axis
        const double hr = 1.0 - lr, hc = 1.0 - lc;        // high-pass power
        acc += chain * (bw.g[3 * j] * lr * hc + bw.g[3 * j + 1] * hr * lc + bw.g[3 * j + 2] * hr * hc);
        chain *= lr * lc;
    }
    return acc + bw.g[3 * bw.levels] * chain;
}

__global__ void spectra_kernel(float2* __restrict__ lamT, float* __restrict__ kT,
                               const float* __restrict__ psf, int ph, int pw, int H, int W, int Wc,
                               int reg, double gamma, BandWeights bw) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= H * Wc) return;
    const int kc = idx / H, kr = idx % H;
    const int lr = ph / 2, lc = pw / 2;
    double fre[kMaxPsfSide], fim[kMaxPsfSide];
    for (int b = -lc; b <= lc; ++b) {
        long long m = ((long long)kc * b) % W;
        if (m < 0) m += W;
        double s, c;
        sincospi(-2.0 * (double)m / (double)W, &s, &c);
        fre[b + lc] = c;
        fim[b + lc] = s;
    }
    double re = 0.0, im = 0.0;
    for (int a = -lr; a <= lr; ++a) {
        double sre = 0.0, sim = 0.0;
        const float* hr = psf + (a + lr) * pw;
        for (int b = 0; b < pw; ++b) {
            sre += (double)hr[b] * fre[b];
            sim += (double)hr[b] * fim[b];
        }
        long long m = ((long long)kr * a) % H;
        if (m < 0) m += H;
        double s, c;
        sincospi(-2.0 * (double)m / (double)H, &s, &c);
        re += sre * c - sim * s;
        im += sre * s + sim * c;
    }
    double den = re * re + im * im;
    if (reg == 0) {
        double sh = sinpi((double)kc / (double)W), sv = sinpi((double)kr / (double)H);
        den += gamma * 4.0 * (sh * sh + sv * sv);
    } else if (bw.levels > 0) {
        den += band_weighted_power(bw, kr, kc, H, W);
    } else {
        den += gamma;
    }
    lamT[idx] = make_float2((float)re, (float)im);
    kT[idx] = (float)(1.0 / (den * (double)H * (double)W));
}

// ---------------------------------------------------------------------------
// Per-solve preparation: effective mask (optionally ANDed with the valid
// region of Sec. IV-A) and M^T y (observations zero-extended, eq.
// prox_g_1_uBC), stored as ybar with a quiet NaN on unobserved pixels. A
// non-finite observed value marks the problem (it then retires at once with
// ADMM_ENONFINITE). ctl must be zeroed before this kernel runs.
// The caller's image is Hu x Wu (row stride Wu) in the top-left corner of the
// H x W domain; pixels outside it are never observed (more unknown boundary),
// and the valid region is that of the caller's image.
// ---------------------------------------------------------------------------
__global__ void prepare_kernel(float* __restrict__ ybar, uint8_t* __restrict__ mask_eff,
                               const float* __restrict__ y, const uint8_t* __restrict__ mask_in,
                               int H, int W, int Hu, int Wu, int lr, int lc, int raw_mask,
                               ProbCtl* __restrict__ ctl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * W) return;
    const int r = i / W, c = i % W;
    const bool inside = r < Hu && c < Wu;
    const size_t iu = (size_t)r * Wu + c;
    bool obs = inside && ((mask_in == nullptr) ? true : (mask_in[iu] != 0));
    if (!raw_mask || mask_in == nullptr)
        obs = obs && r >= lr && r < Hu - lr && c >= lc && c < Wu - lc;
    mask_eff[i] = obs ? 1 : 0;
    const float v = obs ? y[iu] : 0.0f;
    if (obs && !isfinite(v)) atomicOr(&ctl->input_bad, 1);
    ybar[i] = obs ? v : __int_as_float(0x7fc00000);
}

// The same preparation for many problems in one launch (grid.y = problem),
// after zero_ctl_kernel has cleared their control blocks: a batch call then
// issues two launches instead of a copy and a launch per problem.
struct PrepItem {
    float* ybar;
    uint8_t* mask;
    const float* y;
    const uint8_t* m;
    ProbCtl* ctl;
    int H, W, Hu, Wu, lr, lc, raw;
};

__global__ void zero_ctl_kernel(const PrepItem* __restrict__ items, int count) {
    constexpr int words = (int)(sizeof(ProbCtl) / sizeof(int));
    static_assert(sizeof(ProbCtl) % sizeof(int) == 0, "control block of whole words");
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count * words) return;
    reinterpret_cast<int*>(items[i / words].ctl)[i % words] = 0;
}

__global__ void prepare_items_kernel(const PrepItem* __restrict__ items) {
    const PrepItem it = items[blockIdx.y];
    const int n = it.H * it.W;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = i / it.W, c = i % it.W;
        const bool inside = r < it.Hu && c < it.Wu;
        const size_t iu = (size_t)r * it.Wu + c;
        bool obs = inside && ((it.m == nullptr) ? true : (it.m[iu] != 0));
        if (!it.raw || it.m == nullptr)
            obs = obs && r >= it.lr && r < it.Hu - it.lr && c >= it.lc && c < it.Wu - it.lc;
        it.mask[i] = obs ? 1 : 0;
        const float v = obs ? it.y[iu] : 0.0f;
        if (obs && !isfinite(v)) atomicOr(&it.ctl->input_bad, 1);
        it.ybar[i] = obs ? v : __int_as_float(0x7fc00000);
    }
}

__global__ void init_ctl_kernel(ProbDesc* __restrict__ probs, int count, int* __restrict__ n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    ProbCtl* c = probs[b].ctl;
    const bool bad = c->input_bad != 0;
    c->iter = 0;
    c->active = bad ? 0 : 1;
    c->converged = 0;
    c->status = bad ? kStatusNonFinite : 0;
    c->arrive = 0;
    c->have_obj = 0;
    c->obj = 0.0;
    c->obj_prev = 0.0;
    c->rel_x = -1.0;
    c->rel_obj = -1.0;
    c->primal_res = -1.0;
    c->t0 = device_clock_ns();
    c->t_start = 0;
    c->t_done = bad ? c->t0 : 0;
    if (bad) atomicSub(n_active, 1);
}

// first `nslots` problems that are still active go to the slots (one thread)
__global__ void assign_slots_kernel(const ProbDesc* __restrict__ probs, SlotTable sl, int nslots) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int next = 0;
    const unsigned long long now = device_clock_ns();
    for (int s = 0; s < nslots; ++s) {
        while (next < sl.pool && probs[next].ctl->active == 0) ++next;
        sl.map[s] = next < sl.pool ? next : -1;
        if (next < sl.pool) probs[next++].ctl->t_start = now;
    }
    *sl.queue = next;
}

}  // namespace admm
