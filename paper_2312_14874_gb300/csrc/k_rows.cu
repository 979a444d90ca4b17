// k_rows.cu — row-wise scans along the last dim (forward cumsum) and their
// gradients (reverse suffix scans), fp32 and fp64: rows that fit a tile go to
// the row-block kernel, longer rows to the chained kernel with row heads.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kRowsF32[] = {
    GBSCAN_VARIANT_ROWS(OpF32, 8, 20, 3, 8, 3, false, 10, 28, 3, 2),
    GBSCAN_VARIANT_ROWS(OpF32, 8, 20, 4, 8, 2, false, 12, 28, 2, 2),
    GBSCAN_VARIANT_ROWS(OpF32, 16, 20, 2, 8, 2, false, 16, 20, 2, 2),
};

static const Variant kRowsRevF32[] = {
    GBSCAN_VARIANT_ROWS(OpF32, 8, 20, 3, 8, 3, true, 10, 28, 3, 2),
    GBSCAN_VARIANT_ROWS(OpF32, 8, 20, 4, 8, 2, true, 12, 28, 2, 2),
    GBSCAN_VARIANT_ROWS(OpF32, 16, 20, 2, 8, 2, true, 16, 20, 2, 2),
};

static const Variant kRowsF64[] = {
    GBSCAN_VARIANT_ROWS(OpF64, 8, 10, 3, 8, 3, false, 10, 14, 3, 2),
    GBSCAN_VARIANT_ROWS(OpF64, 8, 10, 4, 8, 2, false, 12, 14, 2, 2),
    GBSCAN_VARIANT_ROWS(OpF64, 16, 10, 2, 8, 2, false, 16, 10, 2, 2),
};

static const Variant kRowsRevF64[] = {
    GBSCAN_VARIANT_ROWS(OpF64, 8, 10, 3, 8, 3, true, 10, 14, 3, 2),
    GBSCAN_VARIANT_ROWS(OpF64, 8, 10, 4, 8, 2, true, 12, 14, 2, 2),
    GBSCAN_VARIANT_ROWS(OpF64, 16, 10, 2, 8, 2, true, 16, 10, 2, 2),
};

const Family& family_rows_f32() {
    static const Family f{3, kRowsF32, nullptr};
    return f;
}

const Family& family_rows_rev_f32() {
    static const Family f{3, kRowsRevF32, nullptr};
    return f;
}

const Family& family_rows_f64() {
    static const Family f{3, kRowsF64, nullptr};
    return f;
}

const Family& family_rows_rev_f64() {
    static const Family f{3, kRowsRevF64, nullptr};
    return f;
}

}  // namespace gbscan
