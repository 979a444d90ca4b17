// k_i64.cu — int64 kernel instantiations: plain scans (single-pass and two-pass).
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanI64[] = {
    GBSCAN_VARIANT_ALL(OpI64, 8, 10, 3, 8, 3, 2),
    GBSCAN_VARIANT_ALL(OpI64, 8, 10, 4, 8, 2, 2),
    GBSCAN_VARIANT_ALL(OpI64, 8, 6, 4, 8, 3, 3),
    GBSCAN_VARIANT_ALL(OpI64, 16, 10, 2, 8, 2, 1),
    GBSCAN_VARIANT_ALL(OpI64, 4, 14, 4, 16, 4, 3),
};

const Family& family_scan_i64() {
    static const Family f{5, kScanI64, &launch_scan_sums<OpI64>};
    return f;
}

}  // namespace gbscan
