// rows_large.cu -- compiled TV row-phase configurations for W = 1024, 2048
// (rows per strip, walk rows in flight, threads per CTA); entry 0 is the
// default of each width.
#include "variants.cuh"

namespace admm {

namespace {
const RowVariant k1024[] = {row_variant<1024, 4, 2, 256>(), row_variant<1024, 8, 1, 256>(),
                            row_variant<1024, 4, 1, 128>(), row_variant<1024, 4, 3, 256>()};
const RowVariant k2048[] = {row_variant<2048, 4, 1, 256>(), row_variant<2048, 4, 0, 256>(),
                            row_variant<2048, 2, 1, 256>()};
}  // namespace

int tv_row_variants_large(int W, const RowVariant** out) {
    switch (W) {
        case 1024: *out = k1024; return (int)(sizeof(k1024) / sizeof(k1024[0]));
        case 2048: *out = k2048; return (int)(sizeof(k2048) / sizeof(k2048[0]));
    }
    return 0;
}

}  // namespace admm
