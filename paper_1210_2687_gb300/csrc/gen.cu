// gen.cu -- launch chains of the iteration on exact domains whose sides are
// not both powers of two (kernels in gen.cuh).
#include "gen.cuh"

namespace admm {

namespace {

// the sides the generic kernels are compiled for
#define ADMM_GEN_SIDES(X) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384) X(512) X(640) X(768) \
                          X(1024) X(1280) X(1536) X(2048)

template <int H>
cudaError_t col_t(const ProbDesc* d, SlotTable sl, int count, int Wc, int Wp, const float2* twH, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gcol_phase<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)GCol<H>::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    return launch_chain(gcol_phase<H>, dim3(Wp / GCol<H>::CB, count), dim3(kThreads), GCol<H>::SMEM, s, d, sl, Wc,
                        Wp, twH);
}

cudaError_t launch_gcol(int H, const ProbDesc* d, SlotTable sl, int count, int Wc, int Wp, const float2* twH,
                        cudaStream_t s) {
    switch (H) {
#define ADMM_CASE(N) case N: return col_t<N>(d, sl, count, Wc, Wp, twH, s);
        ADMM_GEN_SIDES(ADMM_CASE)
#undef ADMM_CASE
    }
    return cudaErrorInvalidValue;
}

template <int W>
cudaError_t set_row_attrs() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    constexpr int smem = (int)grow_smem<W>();
    cudaError_t e = cudaFuncSetAttribute(grow_inv<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)grow_inv_smem<W>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(grow_fwd<W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(grow_fwd<W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) attr = true;
    return e;
}

template <int W>
cudaError_t rows_t(int H, int Wc, int Wp, const ProbDesc* d, SlotTable sl, int count, int reg, int levels,
                   const float2* twH, const float2* twW, int* n_active, cudaStream_t s) {
    cudaError_t e = set_row_attrs<W>();
    if (e != cudaSuccess) return e;
    constexpr int G = GRow<W>::G;
    const int nrow = H / G;
    const dim3 rgrid(nrow, count), blk(kThreads);
    const size_t smem = grow_smem<W>();
    e = launch_chain(grow_inv<W>, rgrid, blk, grow_inv_smem<W>(), s, d, sl, H, Wp, twW);
    if (e != cudaSuccess) return e;
    if (reg == 0 || reg == 2) {          // ADMM_REG_TV, ADMM_REG_TV_ANISO
        const dim3 tg(cg_num_tiles(H, W), count);
        e = reg == 2 ? launch_chain(tv_tile<true>, tg, blk, (size_t)0, s, d, sl, H, W, nrow, n_active)
                     : launch_chain(tv_tile<false>, tg, blk, (size_t)0, s, d, sl, H, W, nrow, n_active);
    } else {
        e = haar_tile_attributes();
        if (e != cudaSuccess) return e;
        const bool fs = reg == 4;        // ADMM_REG_HAAR_SYNTHESIS
        const dim3 tg(haar_num_tiles(H, W), count);
        switch (levels * 2 + (fs ? 1 : 0)) {
            case 2: e = launch_chain(haar_analysis<1>, tg, blk, HaarAnaCfg<1>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 4: e = launch_chain(haar_analysis<2>, tg, blk, HaarAnaCfg<2>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 6: e = launch_chain(haar_analysis<3>, tg, blk, HaarAnaCfg<3>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 3: e = launch_chain(haar_analysis<1, true>, tg, blk, HaarAnaCfg<1>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 5: e = launch_chain(haar_analysis<2, true>, tg, blk, HaarAnaCfg<2>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 7: e = launch_chain(haar_analysis<3, true>, tg, blk, HaarAnaCfg<3>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            case 9: e = launch_chain(haar_analysis<4, true>, tg, blk, HaarAnaCfg<4>::SMEM, s, d, sl, H, W, nrow, n_active); break;
            default: e = launch_chain(haar_analysis<4>, tg, blk, HaarAnaCfg<4>::SMEM, s, d, sl, H, W, nrow, n_active); break;
        }
        if (e != cudaSuccess) return e;
        switch (levels) {
            case 1: e = launch_chain(haar_synthesis<1>, tg, blk, HaarSynCfg<1>::SMEM, s, d, sl, H, W); break;
            case 2: e = launch_chain(haar_synthesis<2>, tg, blk, HaarSynCfg<2>::SMEM, s, d, sl, H, W); break;
            case 3: e = launch_chain(haar_synthesis<3>, tg, blk, HaarSynCfg<3>::SMEM, s, d, sl, H, W); break;
            default: e = launch_chain(haar_synthesis<4>, tg, blk, HaarSynCfg<4>::SMEM, s, d, sl, H, W); break;
        }
    }
    if (e != cudaSuccess) return e;
    return launch_chain(grow_fwd<W, false>, rgrid, blk, smem, s, d, sl, H, Wp, twW, (const float*)nullptr,
                        (float4*)nullptr);
}

template <int W>
cudaError_t tail_t(int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels, bool synth,
                   const float2* twW, cudaStream_t s) {
    cudaError_t e = set_row_attrs<W>();
    if (e != cudaSuccess) return e;
    constexpr int G = GRow<W>::G;
    if (synth) {
        e = haar_tile_attributes();
        if (e != cudaSuccess) return e;
        const dim3 tg(haar_num_tiles(H, W), count);
        switch (levels) {
            case 1: haar_synthesis<1><<<tg, kThreads, HaarSynCfg<1>::SMEM, s>>>(d, sl, H, W); break;
            case 2: haar_synthesis<2><<<tg, kThreads, HaarSynCfg<2>::SMEM, s>>>(d, sl, H, W); break;
            case 3: haar_synthesis<3><<<tg, kThreads, HaarSynCfg<3>::SMEM, s>>>(d, sl, H, W); break;
            default: haar_synthesis<4><<<tg, kThreads, HaarSynCfg<4>::SMEM, s>>>(d, sl, H, W); break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    grow_fwd<W, false><<<dim3(H / G, count), kThreads, grow_smem<W>(), s>>>(d, sl, H, Wp, twW, nullptr, nullptr);
    return cudaGetLastError();
}

template <int W>
cudaError_t warm_t(int H, int Wp, const float* x0, float4* Sb, const float2* twW, cudaStream_t s) {
    cudaError_t e = set_row_attrs<W>();
    if (e != cudaSuccess) return e;
    constexpr int G = GRow<W>::G;
    grow_fwd<W, true><<<dim3(H / G, 1), kThreads, grow_smem<W>(), s>>>(nullptr, SlotTable{}, H, Wp, twW, x0, Sb);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gen_iteration(int W, int H, int Wc, int Wp, const ProbDesc* d, SlotTable sl, int count, int reg,
                                 int levels, const float2* twH, const float2* twW, int* n_active, cudaStream_t s) {
    cudaError_t e = launch_gcol(H, d, sl, count, Wc, Wp, twH, s);
    if (e != cudaSuccess) return e;
    switch (W) {
#define ADMM_CASE(N) case N: return rows_t<N>(H, Wc, Wp, d, sl, count, reg, levels, twH, twW, n_active, s);
        ADMM_GEN_SIDES(ADMM_CASE)
#undef ADMM_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_gen_tail(int W, int H, int Wp, const ProbDesc* d, SlotTable sl, int count, int levels, bool synth,
                            const float2* twW, cudaStream_t s) {
    switch (W) {
#define ADMM_CASE(N) case N: return tail_t<N>(H, Wp, d, sl, count, levels, synth, twW, s);
        ADMM_GEN_SIDES(ADMM_CASE)
#undef ADMM_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_gen_warm_rows(int W, int H, int Wp, const float* x0, float4* Sb, const float2* twW,
                                 cudaStream_t s) {
    switch (W) {
#define ADMM_CASE(N) case N: return warm_t<N>(H, Wp, x0, Sb, twW, s);
        ADMM_GEN_SIDES(ADMM_CASE)
#undef ADMM_CASE
    }
    return cudaErrorInvalidValue;
}

int gen_col_block(int H) {
    switch (H) {
#define ADMM_CASE(N) case N: return GCol<N>::CB;
        ADMM_GEN_SIDES(ADMM_CASE)
#undef ADMM_CASE
    }
    return 0;
}

int gen_rows_per_cta(int W) {
    switch (W) {
#define ADMM_CASE(N) case N: return GRow<N>::G;
        ADMM_GEN_SIDES(ADMM_CASE)
#undef ADMM_CASE
    }
    return 0;
}

}  // namespace admm
