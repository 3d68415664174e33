// rows_512.cu -- compiled TV row-phase configurations for W = 512 (rows per
// strip, walk rows in flight, threads per CTA); entry 0 is the default.
// D = 0 reads the walk's inputs straight from global memory (no ring), which
// frees shared memory for a fifth CTA per SM.
#include "variants.cuh"

namespace admm {

namespace {
const RowVariant k512[] = {row_variant<512, 8, 1, 128>(), row_variant<512, 8, 0, 128>(),
                           row_variant<512, 8, 2, 128>(), row_variant<512, 16, 2, 256>(),
                           row_variant<512, 16, 3, 256>(), row_variant<512, 16, 4, 256>()};
}  // namespace

int tv_row_variants_512(const RowVariant** out) {
    *out = k512;
    return (int)(sizeof(k512) / sizeof(k512[0]));
}

}  // namespace admm
