// gfft.cuh -- shared-memory Stockham FFTs of mixed radix for the lengths
// N = m 2^k, m in {1, 3, 5}, that the exact (unpadded) domains use.
//
// The x-update of the ADMM is diagonal in the DFT domain for any domain size
// (Sec. IV-A: the domain only has to hold the image and the kernel support);
// the power-of-two kernels (fft.cuh) serve sides 64..2048, these serve the
// others (192, 384, 768, 1536; 320, 640, 1280) and, in a domain with one
// such side, the power-of-two side too.
//
// Layout: one length-N transform is owned by a group of T = N / E threads;
// thread t holds, in registers, the E elements t + e T, e = 0..E-1, before
// and after the transform (natural order). E is 8 (m = 1), 12 (m = 3) or 20
// (m = 5), so that every pass radix r in {2, 3, 4, 5} divides E: each thread
// then takes E / r whole butterflies of every pass. Passes: radix m first
// (no twiddles), then radix 4 as long as possible, then one radix 2 if
// needed. Exchanges go through a plain shared buffer of N float2 per group.
//
// Stockham pass of radix r with Ns = product of the earlier radices:
// butterfly j in [0, N / r) takes x[j + q N / r], q = 0..r-1, k = j mod Ns,
// multiplies input q by exp(DIR 2 pi i q k / (r Ns)), applies the r-point DFT
// and writes output q to position (j - k) r + k + q Ns.
//
// DIR = -1: X[k] = sum_n x[n] exp(-2 pi i k n / N) (unnormalised forward)
// DIR = +1: x[n] = sum_k X[k] exp(+2 pi i k n / N) (unnormalised inverse)
//
// Twiddles come from a per-length table exp(-2 pi i k / N), k < N, computed
// in FP64 on the host and staged in shared memory by the kernels.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace admm {

__host__ __device__ constexpr int gfft_odd(int n) { return (n & 1) ? n : gfft_odd(n >> 1); }
__host__ __device__ constexpr int gfft_log2(int n) { return n <= 1 ? 0 : 1 + gfft_log2(n >> 1); }

// lengths the generic kernels take: m 2^k with m in {1, 3, 5}, a multiple of
// 32 (the tile kernels' tile) and of 16 E / 8 threads' worth, within 64..2048
__host__ __device__ constexpr bool gfft_length_ok(int n) {
    return n >= 64 && n <= 2048 && n % 32 == 0 &&
           (gfft_odd(n) == 1 || gfft_odd(n) == 3 || gfft_odd(n) == 5) &&
           (n / gfft_odd(n)) >= 32;
}

template <int N> struct GShape {
    static_assert(gfft_length_ok(N), "unsupported generic FFT length");
    static constexpr int M = gfft_odd(N);                 // odd factor
    static constexpr int P2 = N / M;                      // power-of-two factor
    static constexpr int E = M == 1 ? 8 : (M == 3 ? 12 : 20);   // elements per thread
    static constexpr int T = N / E;                       // threads per transform
    static constexpr int L2 = gfft_log2(P2);
    static constexpr int NP4 = L2 / 2, NP2 = L2 % 2;
    static constexpr int NPASS = (M > 1 ? 1 : 0) + NP4 + NP2;
    static_assert(T >= 8 && (T <= 32 || T % 32 == 0), "group size");
    __host__ __device__ static constexpr int radix(int p) {
        return M > 1 ? (p == 0 ? M : (p - 1 < NP4 ? 4 : 2)) : (p < NP4 ? 4 : 2);
    }
};

// r-point DFTs in registers (natural order in and out)
template <int DIR> __device__ __forceinline__ void gdft3(float2& a, float2& b, float2& c) {
    // w = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
    const float s = 0.86602540378443864676f;
    const float2 sbc = b + c, dbc = b - c;
    const float2 m = make_float2(a.x - 0.5f * sbc.x, a.y - 0.5f * sbc.y);
    const float2 r = mul_i<DIR>(s * dbc);
    a = a + sbc;
    b = m + r;
    c = m - r;
}

template <int DIR> __device__ __forceinline__ void gdft5(float2& x0, float2& x1, float2& x2, float2& x3, float2& x4) {
    // w = exp(DIR 2 pi i / 5): cos and sin of 2 pi / 5 and 4 pi / 5
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 t1 = x1 + x4, t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3;
    const float2 a1 = make_float2(x0.x + c1 * t1.x + c2 * t2.x, x0.y + c1 * t1.y + c2 * t2.y);
    const float2 a2 = make_float2(x0.x + c2 * t1.x + c1 * t2.x, x0.y + c2 * t1.y + c1 * t2.y);
    const float2 b1 = mul_i<DIR>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    const float2 b2 = mul_i<DIR>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    x0 = x0 + t1 + t2;
    x1 = a1 + b1;
    x4 = a1 - b1;
    x2 = a2 + b2;
    x3 = a2 - b2;
}

// barrier over the T threads of transform group g (T <= 32: the group's
// lanes of one warp; else named barrier 1 + g)
template <int T> __device__ __forceinline__ void ggroup_sync(int g) {
    if constexpr (T <= 32) {
        constexpr unsigned lanes = T == 32 ? 0xffffffffu : ((1u << T) - 1u);
        __syncwarp(lanes << ((g * T) & 31));
    } else {
        asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "n"(T) : "memory");
    }
}

// one pass of radix R on the registers; outputs exchanged through buf so
// that v again holds elements t + e T
template <int N, int R, int DIR>
__device__ __forceinline__ void gpass(float2 (&v)[GShape<N>::E], int t, int g, int Ns, const float2* tw,
                                      float2* buf) {
    using S = GShape<N>;
    constexpr int E = S::E, T = S::T, B = E / R;
    static_assert(E % R == 0, "radix must divide the elements per thread");
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + T * b;
        const int k = j % Ns;
        float2 x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = v[b + q * B];
        if (Ns > 1) {
            const int step = N / (Ns * R);
#pragma unroll
            for (int q = 1; q < R; ++q) x[q] = cmul(x[q], twid<DIR>(tw, q * k * step));
        }
        if constexpr (R == 2) {
            dft2<DIR>(x[0], x[1]);
        } else if constexpr (R == 3) {
            gdft3<DIR>(x[0], x[1], x[2]);
        } else if constexpr (R == 4) {
            dft4<DIR>(x[0], x[1], x[2], x[3]);
        } else {
            static_assert(R == 5, "radix");
            gdft5<DIR>(x[0], x[1], x[2], x[3], x[4]);
        }
        const int base = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) buf[base + q * Ns] = x[q];
    }
    ggroup_sync<T>(g);
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = buf[t + T * e];
    ggroup_sync<T>(g);       // buf may be written again right away
}

template <int N, int DIR, int P>
__device__ __forceinline__ void gfft_passes(float2 (&v)[GShape<N>::E], int t, int g, int Ns, const float2* tw,
                                            float2* buf) {
    if constexpr (P < GShape<N>::NPASS) {
        constexpr int R = GShape<N>::radix(P);
        gpass<N, R, DIR>(v, t, g, Ns, tw, buf);
        gfft_passes<N, DIR, P + 1>(v, t, g, Ns * R, tw, buf);
    }
}

// Full length-N transform for the T threads of group g.
//   v   : in/out, element t + e T in v[e] (natural order both ways)
//   tw  : exp(-2 pi i k / N), k < N (shared memory)
//   buf : the group's exchange buffer, N float2
// The leading barrier orders any earlier reads of buf by the group.
template <int N, int DIR>
__device__ __forceinline__ void gfft(float2 (&v)[GShape<N>::E], int t, int g, const float2* tw, float2* buf) {
    ggroup_sync<GShape<N>::T>(g);
    gfft_passes<N, DIR, 0>(v, t, g, 1, tw, buf);
}

}  // namespace admm
