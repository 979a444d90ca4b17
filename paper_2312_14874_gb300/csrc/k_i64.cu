// k_i64.cu — int64 kernel instantiations: plain scans (single-pass and two-pass).
#include "gbscan_launch.cuh"

namespace gbscan {

static const Variant kScanI64[] = {
    GBSCAN_VARIANT_ALL(OpI64, 256, 10, 2),
    GBSCAN_VARIANT_ALL(OpI64, 256, 6, 3),
    GBSCAN_VARIANT_ALL(OpI64, 512, 10, 1),
};
const Family& family_scan_i64() {
    static const Family f{3, kScanI64, &launch_scan_sums<OpI64>};
    return f;
}

}  // namespace gbscan
