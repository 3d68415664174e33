// fft.cuh -- shared-memory Stockham FFTs for power-of-two lengths 64..2048.
//
// The x-update of the ADMM (Algorithm 2 line 4; eq. fast_inversion for TV,
// eq. invAnalysisp1 for the frame prior) is diagonal in the DFT domain. These
// routines provide the 1-D transforms that the row and column phases apply to
// whole image rows / spectrum columns.
//
// Layout: one length-N transform is owned by a group of N/8 threads. Thread t
// holds, in registers, the 8 elements t + m*(N/8), m = 0..7, both before and
// after the transform (natural order), so that the first pass reads and the
// last pass writes registers directly; intermediate passes exchange through a
// swizzled shared-memory buffer of N float2 owned by the group.
// Pass radices: the leading pass (no twiddles) is 2, 4 or 8 so that the
// remaining passes are all radix 8: 64=8.8, 128=2.8.8, 256=4.8.8, 512=8.8.8,
// 1024=2.8.8.8, 2048=4.8.8.8.
//
// DIR = -1: X[k] = sum_n x[n] exp(-2 pi i k n / N) (unnormalised forward)
// DIR = +1: x[n] = sum_k X[k] exp(+2 pi i k n / N) (unnormalised inverse)
#pragma once
#include <cuda_runtime.h>

namespace admm {

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Shared-memory position of element i of a transform buffer: an XOR swizzle
// of the low four index bits with bits 3..6 (a bijection on every power-of-two
// length >= 64). It keeps the radix-8 scatters and the sequential accesses of
// the exchanges on distinct banks (conflict-free for length 512, within 1.2x
// of the minimum wavefronts for the other lengths) without padding.
__host__ __device__ constexpr int swz(int i) { return i ^ ((i >> 3) & 15); }

template <int N> struct FftShape {
    static constexpr int LOG = (N == 64) ? 6 : (N == 128) ? 7 : (N == 256) ? 8 : (N == 512) ? 9
                             : (N == 1024) ? 10 : (N == 2048) ? 11 : -1;
    static_assert(LOG > 0, "unsupported FFT length");
    static constexpr int R0 = (LOG % 3 == 0) ? 8 : (LOG % 3 == 1) ? 2 : 4;  // leading radix
    static constexpr int NP8 = (LOG - (R0 == 8 ? 3 : R0 == 4 ? 2 : 1)) / 3; // radix-8 passes after it
    static constexpr int THREADS = N / 8;
};

// multiply by DIR * i
template <int DIR> __device__ __forceinline__ float2 mul_i(float2 a) {
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR> __device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = t + b;
    b = t - b;
}

template <int DIR> __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3, d13 = a1 - a3;
    float2 j13 = mul_i<DIR>(d13);
    a0 = s02 + s13;
    a2 = s02 - s13;
    a1 = d02 + j13;
    a3 = d02 - j13;
}

// natural-order 8-point DFT in registers (radix-2 split of two 4-point DFTs)
template <int DIR> __device__ __forceinline__ void dft8(float2 (&v)[8]) {
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    const float c = 0.70710678118654752440f;
    // o_k *= exp(DIR * 2 pi i k / 8)
    o1 = make_float2(c * (o1.x - (float)DIR * o1.y), c * (o1.y + (float)DIR * o1.x));
    o2 = mul_i<DIR>(o2);
    o3 = make_float2(c * (-o3.x - (float)DIR * o3.y), c * ((float)DIR * o3.x - o3.y));
    v[0] = e0 + o0; v[4] = e0 - o0;
    v[1] = e1 + o1; v[5] = e1 - o1;
    v[2] = e2 + o2; v[6] = e2 - o2;
    v[3] = e3 + o3; v[7] = e3 - o3;
}

// twiddle tw[idx] of a forward table, conjugated for the inverse direction
template <int DIR> __device__ __forceinline__ float2 twid(const float2* tw, int idx) {
    float2 w = tw[idx];
    return DIR < 0 ? w : conjf2(w);
}

// Per-pass twiddle table of a length-N transform. The radix-8 pass p runs
// with stride Ns = R0 8^p; its entries off(p) + (r - 1) Ns + k hold
// exp(-2 pi i r k / (8 Ns)) for r = 1..7, k < Ns, so the lanes of a warp
// (consecutive k = t mod Ns) read consecutive entries: no bank conflicts,
// where indexing one length-N table by r k N / (8 Ns) put up to eight lanes
// on one bank. At most N entries.
template <int N> struct TwiddleLayout {
    __host__ __device__ static constexpr int off(int p) {
        int o = 0, ns = FftShape<N>::R0;
        for (int q = 0; q < p; ++q) {
            o += 7 * ns;
            ns *= 8;
        }
        return o;
    }
    static constexpr int SIZE = off(FftShape<N>::NP8);
    static_assert(SIZE <= N, "table fits a length-N buffer");
};

// The device twiddle buffer holds the 2048-entry table exp(-2 pi i k / 2048)
// followed by the per-pass table of every length 64..2048, each in a slot of
// 2048 entries (filled on the host from the same float values that
// load_twiddles copies). Kernels whose shared memory is better spent on
// concurrency read their transform's table there, through L1, instead of
// staging it.
constexpr int kTwiddleEntries = 2048 * 7;
template <int N>
__host__ __device__ constexpr int pass_table_offset() {
    return 2048 * (1 + FftShape<N>::LOG - 6);
}
// host: the per-pass table of length n (a power of two, 64..2048) into dst
// from the 2048-entry table tw2048 (the order load_twiddles produces)
inline void fill_pass_table(int n, const float2* tw2048, float2* dst) {
    int log = 0;
    while ((1 << log) < n) ++log;
    const int r0 = (log % 3 == 0) ? 8 : (log % 3 == 1) ? 2 : 4;
    const int np8 = (log - (r0 == 8 ? 3 : r0 == 4 ? 2 : 1)) / 3;
    int ns = r0, o = 0;
    for (int p = 0; p < np8; ++p) {
        const int step = n / (ns * 8);
        for (int e = 0; e < 7 * ns; ++e) {
            const int r = e / ns + 1, k = e - (r - 1) * ns;
            dst[o + e] = tw2048[r * k * step * (2048 / n)];
        }
        o += 7 * ns;
        ns *= 8;
    }
}

// Fill the per-pass table from the 2048-entry table exp(-2 pi i k / 2048)
// (threads tid of nthr cooperate; the caller synchronises afterwards).
template <int N>
__device__ __forceinline__ void load_twiddles(float2* dst, const float2* __restrict__ tw2048, int tid, int nthr) {
    using S = FftShape<N>;
    int ns = S::R0, o = 0;
#pragma unroll
    for (int p = 0; p < S::NP8; ++p) {
        const int step = N / (ns * 8);
        for (int e = tid; e < 7 * ns; e += nthr) {
            const int r = e / ns + 1, k = e - (r - 1) * ns;
            dst[o + e] = tw2048[r * k * step * (2048 / N)];
        }
        o += 7 * ns;
        ns *= 8;
    }
}

// One Stockham pass on the registers of thread t (elements t + m N/8 as
// input): twiddles, butterflies, and the output index of every register.
template <int N, int R, int DIR>
__device__ __forceinline__ void stockham_compute(float2 (&v)[8], int t, int Ns, const float2* tw,
                                                 int (&oidx)[8]) {
    constexpr int Q = N / 8;
    if constexpr (R == 8) {
        // tw: this pass's block of the per-pass table (TwiddleLayout)
        const int j = t, k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], twid<DIR>(tw, (r - 1) * Ns + k));
        }
        dft8<DIR>(v);
        const int base = (j - k) * 8 + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) oidx[r] = base + r * Ns;
    } else if constexpr (R == 4) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int j = t + b * Q, k = j & (Ns - 1);   // leading pass only: Ns = 1, no twiddles
            dft4<DIR>(v[b], v[2 + b], v[4 + b], v[6 + b]);
            const int base = (j - k) * 4 + k;
#pragma unroll
            for (int r = 0; r < 4; ++r) oidx[2 * r + b] = base + r * Ns;
        }
    } else {
        static_assert(R == 2, "radix");
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int j = t + s * Q, k = j & (Ns - 1);   // leading pass only: Ns = 1, no twiddles
            dft2<DIR>(v[s], v[s + 4]);
            const int base = (j - k) * 2 + k;
            oidx[s] = base;
            oidx[s + 4] = base + Ns;
        }
    }
}

// Barrier over the N/8 threads of one transform group (group g of the
// block, threads g*N/8 .. g*N/8 + N/8 - 1): a warp barrier when the group
// fits in one warp, else named barrier 1 + g (barrier 0 is __syncthreads).
template <int N>
__device__ __forceinline__ void group_sync(int g) {
    constexpr int FT = N / 8;
    if constexpr (FT <= 32) {
        constexpr unsigned lanes = FT == 32 ? 0xffffffffu : ((1u << FT) - 1u);
        const unsigned mask = lanes << ((g * FT) & 31);
        __syncwarp(mask);
    } else {
        asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "n"(FT) : "memory");
    }
}

// Full length-N transform for a group of N/8 threads.
//   v    : in/out registers, element t + m N/8 in v[m] (natural order both ways)
//   buf  : the group's shared buffer, >= N float2 (swizzled positions)
//   tw   : per-pass twiddle table of length N (TwiddleLayout, load_twiddles)
//   g    : index of the group in the block (threads g*N/8 .. g*N/8 + N/8 - 1)
// Only the threads of the group synchronise (group_sync); the other groups of
// the block run independently. Block-wide ordering is the caller's business.
template <int N, int DIR>
__device__ __forceinline__ void fft_group(float2 (&v)[8], float2* buf, const float2* tw, int t, int g) {
    using S = FftShape<N>;
    constexpr int Q = N / 8;
    int oidx[8];
    int Ns = 1;
    stockham_compute<N, S::R0, DIR>(v, t, Ns, tw, oidx);
    Ns *= S::R0;
#pragma unroll
    for (int p = 0; p < S::NP8; ++p) {
        // exchange through shared memory into the input order of the next
        // pass; the leading barrier also orders any reads of `buf` the caller
        // made before the transform
        group_sync<N>(g);
#pragma unroll
        for (int m = 0; m < 8; ++m) buf[swz(oidx[m])] = v[m];
        group_sync<N>(g);
#pragma unroll
        for (int m = 0; m < 8; ++m) v[m] = buf[swz(t + m * Q)];
        stockham_compute<N, 8, DIR>(v, t, Ns, tw + TwiddleLayout<N>::off(p), oidx);
        Ns *= 8;
    }
    // after the last radix-8 pass (Ns = N/8 before it) oidx[m] = t + m N/8:
    // registers already hold the natural-order output. The trailing barrier
    // lets the group overwrite `buf` right away.
    group_sync<N>(g);
}

// Two transforms of the same length and direction on one group, interleaved
// pass by pass: the twiddles, index arithmetic and barriers are shared and the
// two dependency chains overlap. Same layout and contract as fft_group.
template <int N, int DIR>
__device__ __forceinline__ void fft_group2(float2 (&v)[8], float2 (&u)[8], float2* bv, float2* bu,
                                           const float2* tw, int t, int g) {
    using S = FftShape<N>;
    constexpr int Q = N / 8;
    int oidx[8];
    int Ns = 1;
    stockham_compute<N, S::R0, DIR>(v, t, Ns, tw, oidx);
    stockham_compute<N, S::R0, DIR>(u, t, Ns, tw, oidx);
    Ns *= S::R0;
#pragma unroll
    for (int p = 0; p < S::NP8; ++p) {
        group_sync<N>(g);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            bv[swz(oidx[m])] = v[m];
            bu[swz(oidx[m])] = u[m];
        }
        group_sync<N>(g);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            v[m] = bv[swz(t + m * Q)];
            u[m] = bu[swz(t + m * Q)];
        }
        // shared twiddles: exp(DIR 2 pi i r k / (8 Ns)), k = t mod Ns
        const int k = t & (Ns - 1);
        if (Ns > 1) {
            const float2* twp = tw + TwiddleLayout<N>::off(p);
#pragma unroll
            for (int r = 1; r < 8; ++r) {
                const float2 w = twid<DIR>(twp, (r - 1) * Ns + k);
                v[r] = cmul(v[r], w);
                u[r] = cmul(u[r], w);
            }
        }
        dft8<DIR>(v);
        dft8<DIR>(u);
        const int base = (t - k) * 8 + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) oidx[r] = base + r * Ns;
        Ns *= 8;
    }
    group_sync<N>(g);
}

}  // namespace admm
