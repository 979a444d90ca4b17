// k_i64.cu — int64 kernel instantiations: plain scans (single-pass and two-pass).
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanI64[] = {
    GBSCAN_VARIANT_ALL(OpI64, 8, 10, 3, 3, 2, 3, 2),
    GBSCAN_VARIANT_ALL(OpI64, 8, 10, 5, 2, 2, 4, 2),
    GBSCAN_VARIANT_ALL(OpI64, 8, 6, 6, 2, 3, 4, 2),
    GBSCAN_VARIANT_ALL(OpI64, 16, 10, 5, 1, 1, 3, 2),
    GBSCAN_VARIANT_ALL(OpI64, 4, 14, 4, 3, 3, 4, 2),
    GBSCAN_VARIANT_ALL(OpI64, 8, 14, 4, 2, 2, 3, 2),
};

const Family& family_scan_i64() {
    static const Family f{6, kScanI64, &launch_scan_sums<OpI64>, GBSCAN_RESIDENT(OpI64)};
    return f;
}

}  // namespace gbscan
