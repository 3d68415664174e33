// variants.cuh -- the kernel configurations the engine chooses between for a
// size class, and their launchers.
//
// Every side length has a short list of compiled configurations of the TV
// row phase (rows per strip R, walk rows in flight D, threads per CTA NT) and
// of the column phase (columns per CTA CB); entry 0 of each list is the
// default. The autotuner (admm_deconv_autotune) times the combinations on the
// device and records the fastest per (device, H, W, regulariser, levels);
// plans created afterwards use it. The instantiations are spread over
// several translation units (rows_small.cu, rows_512.cu, rows_large.cu,
// cols.cu) so that they compile in parallel.
#pragma once
#include <algorithm>

#include "kernels.cuh"

namespace admm {

using RowLaunchFn = cudaError_t (*)(const ProbDesc* d, SlotTable sl, int count, int H, int Wp, const float2* tw,
                                    int* n_active, cudaStream_t s);
using ColLaunchFn = cudaError_t (*)(const ProbDesc* d, SlotTable sl, int count, int Wc, int Wp, const float2* tw,
                                    cudaStream_t s);

struct RowVariant {
    int R, D, NT;
    RowLaunchFn fn;          // isotropic TV
    RowLaunchFn fn_aniso;    // anisotropic TV
};
struct ColVariant {
    int CB;
    int MB;   // CTAs per SM the registers are sized for (0: the default of the block)
    int persistent;   // 1: persistent CTAs with a double-buffered tile (col_phase_pers)
    ColLaunchFn fn;
};

// candidates for one side length (entry 0 = default); returns their number,
// 0 for an unsupported side
int tv_row_variants(int W, const RowVariant** out);
int col_variants(int H, const ColVariant** out);

// per translation unit
int tv_row_variants_small(int W, const RowVariant** out);   // W = 64, 128, 256
int tv_row_variants_512(const RowVariant** out);            // W = 512
int tv_row_variants_large(int W, const RowVariant** out);   // W = 1024, 2048

template <int W, int R, int D, int NT, bool ANISO>
cudaError_t launch_row_tv_t(const ProbDesc* d, SlotTable sl, int count, int H, int Wp, const float2* tw,
                            int* n_active, cudaStream_t s) {
    static bool attr = false;
    const size_t smem = RowCfg<W, R, D, NT>::SMEM;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(row_phase_tv<W, R, D, NT, ANISO>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(H / R, count);
    return launch_chain(row_phase_tv<W, R, D, NT, ANISO>, grid, dim3(NT), smem, s, d, sl, H, Wp, tw, n_active);
}

template <int H, int CB, int MB>
cudaError_t launch_col_t(const ProbDesc* d, SlotTable sl, int count, int Wc, int Wp, const float2* tw,
                         cudaStream_t s) {
    static bool attr = false;
    const size_t smem = ColCfg<H, CB>::SMEM;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(col_phase<H, CB, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid(Wp / CB, count);
    return launch_chain(col_phase<H, CB, MB>, grid, dim3(kThreads), smem, s, d, sl, Wc, Wp, tw);
}

// persistent column phase: three CTAs per SM (two tiles and the twiddles in
// shared memory) over the items of the launch
int device_sm_count();
template <int H, int CB>
cudaError_t launch_col_pers_t(const ProbDesc* d, SlotTable sl, int count, int Wc, int Wp, const float2* tw,
                              cudaStream_t s) {
    static bool attr = false;
    const size_t smem = (size_t)2 * H * CB * sizeof(float4) + (size_t)ColCfg<H, CB>::TWN * sizeof(float2);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(col_phase_pers<H, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nblk = Wp / CB, nitems = nblk * count;
    const int grid = std::min(nitems, 3 * device_sm_count());
    if (grid <= 0) return cudaSuccess;
    return launch_chain(col_phase_pers<H, CB>, dim3(grid), dim3(kThreads), smem, s, d, sl, Wc, Wp, tw, nblk, nitems);
}

template <int W, int R, int D, int NT>
constexpr RowVariant row_variant() {
    return RowVariant{R, D, NT, &launch_row_tv_t<W, R, D, NT, false>, &launch_row_tv_t<W, R, D, NT, true>};
}
// MB > 0: registers sized for MB CTAs per SM instead of the default
template <int H, int CB, int MB = 0>
constexpr ColVariant col_variant() {
    return ColVariant{CB, MB, 0, &launch_col_t<H, CB, MB>};
}
template <int H>
constexpr ColVariant col_variant_pers() {
    return ColVariant{ColCfg<H, kThreads / (H / 8)>::G, 3, 1, &launch_col_pers_t<H, kThreads / (H / 8)>};
}

}  // namespace admm
