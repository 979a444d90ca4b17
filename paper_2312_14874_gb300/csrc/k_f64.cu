// k_f64.cu — fp64 kernel instantiations: plain scans (single-pass and two-pass).
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanF64[] = {
    GBSCAN_VARIANT_ALL(OpF64, 8, 10, 3, 8, 3, 2),
    GBSCAN_VARIANT_ALL(OpF64, 8, 10, 4, 8, 2, 2),
    GBSCAN_VARIANT_ALL(OpF64, 8, 6, 4, 8, 3, 3),
    GBSCAN_VARIANT_ALL(OpF64, 16, 10, 2, 8, 2, 1),
    GBSCAN_VARIANT_ALL(OpF64, 4, 14, 4, 16, 4, 3),
};

const Family& family_scan_f64() {
    static const Family f{5, kScanF64, &launch_scan_sums<OpF64>};
    return f;
}

}  // namespace gbscan
