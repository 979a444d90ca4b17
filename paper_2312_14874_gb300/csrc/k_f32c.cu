// k_f32c.cu — compensated fp32 kernel instantiations (TwoSum pair carries),
// single-pass and two-pass.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanF32C[] = {
    GBSCAN_VARIANT_ALL(OpF32C, 8, 20, 3, 3, 2, 3, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 8, 20, 5, 2, 2, 4, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 8, 12, 6, 2, 3, 4, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 16, 20, 5, 1, 1, 3, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 4, 28, 4, 3, 3, 4, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 8, 28, 4, 2, 2, 3, 2),
};

const Family& family_scan_f32c() {
    static const Family f{6, kScanF32C, &launch_scan_sums<OpF32C>, GBSCAN_RESIDENT(OpF32C)};
    return f;
}

}  // namespace gbscan
