// k_i32.cu — int32 kernel instantiations: plain scans (single-pass and
// two-pass) and offset-segmented scans.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanI32[] = {
    GBSCAN_VARIANT_ALL(OpI32, 8, 20, 3, 3, 2, 3, 2),
    GBSCAN_VARIANT_ALL(OpI32, 8, 20, 5, 2, 2, 4, 2),
    GBSCAN_VARIANT_ALL(OpI32, 8, 12, 6, 2, 3, 4, 2),
    GBSCAN_VARIANT_ALL(OpI32, 16, 20, 5, 1, 1, 3, 2),
    GBSCAN_VARIANT_ALL(OpI32, 4, 28, 4, 3, 3, 4, 2),
    GBSCAN_VARIANT_ALL(OpI32, 8, 28, 4, 2, 2, 3, 2),
};

const Family& family_scan_i32() {
    static const Family f{6, kScanI32, &launch_scan_sums<OpI32>, GBSCAN_RESIDENT(OpI32)};
    return f;
}

static const Variant kSegI32[] = {
    GBSCAN_VARIANT_SEG_PT(OpI32, 8, 20, 4, 2),
    GBSCAN_VARIANT_SEG_PT(OpI32, 8, 20, 3, 2),
    GBSCAN_VARIANT_SP(OpI32, 8, 20, 3, 8, 3, kOffsetHeads, false),
    GBSCAN_VARIANT_SP(OpI32, 8, 20, 4, 8, 2, kOffsetHeads, false),
    GBSCAN_VARIANT_SP(OpI32, 16, 20, 2, 8, 2, kOffsetHeads, false),
};

const Family& family_seg_i32() {
    static const Family f{5, kSegI32, nullptr};
    return f;
}

}  // namespace gbscan
