// k_ops.cu — scans under other associative operators than +: running maximum
// and running minimum of int32 and fp32 arrays (single-pass, two-pass and
// partitioned, three launch shapes each); and stream compaction, the scan of
// keep flags fused with the gather it drives.
#include "gbscan_launch.cuh"

namespace gbscan {

#define GBSCAN_OP_FAMILY(FN, OP)                                                                \
    static const Variant kVariants##OP[] = {                                                    \
        GBSCAN_VARIANT_ALL(OP, 8, 20, 3, 3, 2, 3, 2),                                           \
        GBSCAN_VARIANT_ALL(OP, 8, 20, 5, 2, 2, 4, 2),                                           \
        GBSCAN_VARIANT_ALL(OP, 8, 28, 4, 2, 2, 3, 2),                                           \
    };                                                                                          \
    const Family& FN() {                                                                        \
        static const Family f{3, kVariants##OP, &launch_scan_sums<OP>, GBSCAN_RESIDENT(OP)};                         \
        return f;                                                                               \
    }

GBSCAN_OP_FAMILY(family_max_i32, OpMaxI32)
GBSCAN_OP_FAMILY(family_min_i32, OpMinI32)
GBSCAN_OP_FAMILY(family_max_f32, OpMaxF32)
GBSCAN_OP_FAMILY(family_min_f32, OpMinF32)

static const Variant kCompact[] = {
    GBSCAN_VARIANT_COMPACT(8, 20, 3, 2),
    GBSCAN_VARIANT_COMPACT(16, 28, 2, 1),
    GBSCAN_VARIANT_COMPACT(8, 28, 3, 2),
};

const Family& family_compact() {
    static const Family f{3, kCompact, nullptr};
    return f;
}

}  // namespace gbscan
