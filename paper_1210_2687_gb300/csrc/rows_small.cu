// rows_small.cu -- compiled TV row-phase configurations for W = 64, 128, 256
// (rows per strip, walk rows in flight, threads per CTA); entry 0 is the
// default of each width.
#include "variants.cuh"

namespace admm {

namespace {
const RowVariant k64[] = {row_variant<64, 16, 4, 256>(), row_variant<64, 16, 2, 128>(),
                          row_variant<64, 8, 2, 64>()};
const RowVariant k128[] = {row_variant<128, 16, 4, 256>(), row_variant<128, 16, 2, 128>(),
                           row_variant<128, 8, 2, 128>()};
const RowVariant k256[] = {row_variant<256, 8, 4, 256>(), row_variant<256, 8, 2, 128>(),
                           row_variant<256, 16, 2, 256>(), row_variant<256, 16, 4, 256>()};
}  // namespace

int tv_row_variants_small(int W, const RowVariant** out) {
    switch (W) {
        case 64: *out = k64; return (int)(sizeof(k64) / sizeof(k64[0]));
        case 128: *out = k128; return (int)(sizeof(k128) / sizeof(k128[0]));
        case 256: *out = k256; return (int)(sizeof(k256) / sizeof(k256[0]));
    }
    return 0;
}

}  // namespace admm
