// k_f32.cu — fp32 kernel instantiations: plain scans (single-pass and two-pass)
// and offset-segmented scans.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanF32[] = {
    GBSCAN_VARIANT_ALL(OpF32, 256, 20, 2),
    GBSCAN_VARIANT_ALL(OpF32, 256, 12, 3),
    GBSCAN_VARIANT_ALL(OpF32, 512, 20, 1),
};
const Family& family_scan_f32() {
    static const Family f{3, kScanF32, &launch_scan_sums<OpF32>};
    return f;
}

static const Variant kSegF32[] = {
    GBSCAN_VARIANT_SP(OpF32, 256, 20, 2, kOffsetHeads, false),
    GBSCAN_VARIANT_SP(OpF32, 256, 12, 3, kOffsetHeads, false),
    GBSCAN_VARIANT_SP(OpF32, 512, 20, 1, kOffsetHeads, false),
};
const Family& family_seg_f32() {
    static const Family f{3, kSegF32, nullptr};
    return f;
}

}  // namespace gbscan
