// cg.cu -- launch chain of one TV-CG / FA-CG iteration (kernels in cg.cuh).
#include "cg.cuh"

namespace admm {

namespace {

template <int W>
cudaError_t launch_cg_t(int H, int Wc, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels, bool tv,
                        ColLaunchFn col_fn, const float2* tw, int* n_active, cudaStream_t s) {
    constexpr int FT = W / 8, G = kThreads / FT;
    const size_t smem_row = (size_t)(G * W + W) * sizeof(float2) + 2 * (kThreads / 32) * sizeof(double);
    constexpr size_t smem_fwd = haar_fwd_smem<W>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(cg_row_a<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cg_row_b<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(haar_row_forward<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_fwd);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int nrow = H / G;
    const dim3 rgrid(nrow, count), blk(kThreads);
    cudaError_t e = col_fn(d, sl, count, Wc, Wp, tw, s);                       // x~ = C (r + B^T z)
    if (e == cudaSuccess) e = launch_chain(cg_row_a<W>, rgrid, blk, smem_row, s, d, sl, H, Wp, tw);
    if (e == cudaSuccess) e = col_fn(d, sl, count, Wc, Wp, tw, s);              // v = C A^T s
    if (e == cudaSuccess) e = launch_chain(cg_row_b<W>, rgrid, blk, smem_row, s, d, sl, H, Wp, tw);
    if (e == cudaSuccess) e = launch_chain(cg_obs<W>, rgrid, blk, (size_t)0, s, d, sl, H);
    if (e != cudaSuccess) return e;
    if (tv) {
        e = launch_chain(tv_tile<false>, dim3(cg_num_tiles(H, W), count), blk, (size_t)0, s, d, sl, H, W, nrow,
                         n_active);
    } else {
        e = haar_tile_attributes();
        if (e != cudaSuccess) return e;
        const dim3 tgrid(haar_num_tiles(H, W), count);
        switch (levels) {
            case 1: e = launch_chain(haar_analysis<1>, tgrid, blk, HaarAnaCfg<1>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 2: e = launch_chain(haar_analysis<2>, tgrid, blk, HaarAnaCfg<2>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 3: e = launch_chain(haar_analysis<3>, tgrid, blk, HaarAnaCfg<3>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            default: e = launch_chain(haar_analysis<4>, tgrid, blk, HaarAnaCfg<4>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        }
        if (e != cudaSuccess) return e;
        switch (levels) {
            case 1: e = launch_chain(haar_synthesis<1>, tgrid, blk, HaarSynCfg<1>::SMEM, s, d, sl, H, W); break;
            case 2: e = launch_chain(haar_synthesis<2>, tgrid, blk, HaarSynCfg<2>::SMEM, s, d, sl, H, W); break;
            case 3: e = launch_chain(haar_synthesis<3>, tgrid, blk, HaarSynCfg<3>::SMEM, s, d, sl, H, W); break;
            default: e = launch_chain(haar_synthesis<4>, tgrid, blk, HaarSynCfg<4>::SMEM, s, d, sl, H, W); break;
        }
    }
    if (e != cudaSuccess) return e;
    return launch_chain(haar_row_forward<W>, dim3(nrow / 2, count), blk, smem_fwd, s, d, sl, H, Wp, tw);
}

}  // namespace

cudaError_t launch_cg_iteration(int W, int H, int Wc, int Wp, const ProbDesc* d, SlotTable sl, int count,
                                int levels, bool tv, ColLaunchFn col_fn, const float2* tw, int* n_active,
                                cudaStream_t s) {
    switch (W) {
        case 64: return launch_cg_t<64>(H, Wc, Wp, d, sl, count, levels, tv, col_fn, tw, n_active, s);
        case 128: return launch_cg_t<128>(H, Wc, Wp, d, sl, count, levels, tv, col_fn, tw, n_active, s);
        case 256: return launch_cg_t<256>(H, Wc, Wp, d, sl, count, levels, tv, col_fn, tw, n_active, s);
        case 512: return launch_cg_t<512>(H, Wc, Wp, d, sl, count, levels, tv, col_fn, tw, n_active, s);
        case 1024: return launch_cg_t<1024>(H, Wc, Wp, d, sl, count, levels, tv, col_fn, tw, n_active, s);
        case 2048: return launch_cg_t<2048>(H, Wc, Wp, d, sl, count, levels, tv, col_fn, tw, n_active, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace admm
