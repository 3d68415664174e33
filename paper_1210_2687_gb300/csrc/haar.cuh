// haar.cuh -- frame-prior (FA-MD) row-side kernels. Placeholder interface.
#pragma once
#include <cuda_runtime.h>
#include "kernels.cuh"

namespace admm {
constexpr int kMaxHaarLevels = 4;
inline int haar_row_strip(int W) { (void)W; return 16; }
inline int haar_num_partial_blocks(int H, int W) { (void)W; return H / 16; }
inline cudaError_t launch_haar_iteration_rows(int, int, int, const ProbDesc*, int, int, const float2*, int*,
                                              cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace admm
