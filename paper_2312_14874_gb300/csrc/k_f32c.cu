// k_f32c.cu — compensated fp32 kernel instantiations (TwoSum pair carries),
// single-pass and two-pass.
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanF32C[] = {
    GBSCAN_VARIANT_ALL(OpF32C, 256, 20, 2),
    GBSCAN_VARIANT_ALL(OpF32C, 256, 12, 3),
    GBSCAN_VARIANT_ALL(OpF32C, 512, 20, 1),
};
const Family& family_scan_f32c() {
    static const Family f{3, kScanF32C, &launch_scan_sums<OpF32C>};
    return f;
}

}  // namespace gbscan
