// k_f32c.cu — compensated fp32 kernel instantiations (TwoSum pair carries),
// single-pass and two-pass.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanF32C[] = {
    GBSCAN_VARIANT_ALL(OpF32C, 8, 20, 3, 8, 3, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 8, 20, 4, 8, 2, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 8, 12, 4, 8, 3, 3),
    GBSCAN_VARIANT_ALL(OpF32C, 16, 20, 2, 8, 2, 1),
    GBSCAN_VARIANT_ALL(OpF32C, 4, 28, 4, 16, 4, 3),
};

const Family& family_scan_f32c() {
    static const Family f{5, kScanF32C, &launch_scan_sums<OpF32C>};
    return f;
}

}  // namespace gbscan
