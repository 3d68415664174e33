// cols.cu -- compiled column-phase configurations (columns per CTA) for every
// height, and the dispatch of the row-phase tables; entry 0 of each list is
// the default.
#include "variants.cuh"

namespace admm {

namespace {
// (the third template argument: registers sized for that many CTAs per SM)
const ColVariant c64[] = {col_variant<64, 32>(), col_variant<64, 64>(), col_variant<64, 32, 3>(),
                          col_variant_pers<64>()};
const ColVariant c128[] = {col_variant<128, 16>(), col_variant<128, 32>(), col_variant<128, 16, 3>(),
                           col_variant_pers<128>()};
const ColVariant c256[] = {col_variant<256, 8>(), col_variant<256, 16>(), col_variant<256, 8, 3>(),
                           col_variant_pers<256>()};
const ColVariant c512[] = {col_variant<512, 4>(), col_variant<512, 8>(), col_variant<512, 4, 3>(),
                           col_variant_pers<512>()};
const ColVariant c1024[] = {col_variant<1024, 4>(), col_variant<1024, 2>(), col_variant<1024, 8>(),
                            col_variant<1024, 2, 3>(), col_variant_pers<1024>()};
const ColVariant c2048[] = {col_variant<2048, 2>(), col_variant<2048, 1>(), col_variant<2048, 4>(),
                            col_variant<2048, 1, 3>(), col_variant_pers<2048>()};
template <int N>
int take(const ColVariant (&t)[N], const ColVariant** out) {
    *out = t;
    return N;
}
}  // namespace

int col_variants(int H, const ColVariant** out) {
    switch (H) {
        case 64: return take(c64, out);
        case 128: return take(c128, out);
        case 256: return take(c256, out);
        case 512: return take(c512, out);
        case 1024: return take(c1024, out);
        case 2048: return take(c2048, out);
    }
    return 0;
}

int device_sm_count() {
    static int sms = 0;   // the library runs on one device type per process
    if (sms == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            return 1;
    }
    return sms;
}

int tv_row_variants(int W, const RowVariant** out) {
    if (W <= 256) return tv_row_variants_small(W, out);
    if (W == 512) return tv_row_variants_512(out);
    return tv_row_variants_large(W, out);
}

}  // namespace admm
