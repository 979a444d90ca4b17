// k_rows.cu — row-wise scans along the last dim (forward cumsum) and their
// gradients (reverse suffix scans), fp32 and fp64.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kRowsF32[] = {
    GBSCAN_VARIANT_SP(OpF32, 8, 20, 3, 8, 3, kRowHeads, false),
    GBSCAN_VARIANT_SP(OpF32, 8, 20, 4, 8, 2, kRowHeads, false),
    GBSCAN_VARIANT_SP(OpF32, 16, 20, 2, 8, 2, kRowHeads, false),
};

static const Variant kRowsRevF32[] = {
    GBSCAN_VARIANT_SP(OpF32, 8, 20, 3, 8, 3, kRowHeads, true),
    GBSCAN_VARIANT_SP(OpF32, 8, 20, 4, 8, 2, kRowHeads, true),
    GBSCAN_VARIANT_SP(OpF32, 16, 20, 2, 8, 2, kRowHeads, true),
};

static const Variant kRowsF64[] = {
    GBSCAN_VARIANT_SP(OpF64, 8, 10, 3, 8, 3, kRowHeads, false),
    GBSCAN_VARIANT_SP(OpF64, 8, 10, 4, 8, 2, kRowHeads, false),
    GBSCAN_VARIANT_SP(OpF64, 16, 10, 2, 8, 2, kRowHeads, false),
};

static const Variant kRowsRevF64[] = {
    GBSCAN_VARIANT_SP(OpF64, 8, 10, 3, 8, 3, kRowHeads, true),
    GBSCAN_VARIANT_SP(OpF64, 8, 10, 4, 8, 2, kRowHeads, true),
    GBSCAN_VARIANT_SP(OpF64, 16, 10, 2, 8, 2, kRowHeads, true),
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
