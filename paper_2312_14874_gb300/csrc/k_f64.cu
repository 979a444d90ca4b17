// k_f64.cu — fp64 kernel instantiations: plain scans (single-pass and two-pass).
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanF64[] = {
    GBSCAN_VARIANT_ALL(OpF64, 256, 10, 2),
    GBSCAN_VARIANT_ALL(OpF64, 256, 6, 3),
    GBSCAN_VARIANT_ALL(OpF64, 512, 10, 1),
};
const Family& family_scan_f64() {
    static const Family f{3, kScanF64, &launch_scan_sums<OpF64>};
    return f;
}

}  // namespace gbscan
