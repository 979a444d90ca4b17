// k_i32.cu — int32 kernel instantiations: plain scans (single-pass and
// two-pass) and offset-segmented scans.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanI32[] = {
    GBSCAN_VARIANT_ALL(OpI32, 256, 20, 2),
    GBSCAN_VARIANT_ALL(OpI32, 256, 12, 3),
    GBSCAN_VARIANT_ALL(OpI32, 512, 20, 1),
};
const Family& family_scan_i32() {
    static const Family f{3, kScanI32, &launch_scan_sums<OpI32>};
    return f;
}

static const Variant kSegI32[] = {
    GBSCAN_VARIANT_SP(OpI32, 256, 20, 2, kOffsetHeads, false),
    GBSCAN_VARIANT_SP(OpI32, 256, 12, 3, kOffsetHeads, false),
    GBSCAN_VARIANT_SP(OpI32, 512, 20, 1, kOffsetHeads, false),
};
const Family& family_seg_i32() {
    static const Family f{3, kSegI32, nullptr};
    return f;
}

}  // namespace gbscan
