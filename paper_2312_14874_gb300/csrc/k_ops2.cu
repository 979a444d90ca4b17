// k_ops2.cu — more scans under maximum and minimum: running maximum and
// minimum of int64 and uint32 arrays (single-pass, two-pass and partitioned,
// three launch shapes each), and segmented running maximum and minimum of
// int32 and fp32 (the partitioned kernel with the head bitmap, two shapes).
#include "gbscan_launch.cuh"

namespace gbscan {

#define GBSCAN_OP_FAMILY_W(FN, OP, I_A, I_B)                                                    \
    static const Variant kVariants##OP[] = {                                                    \
        GBSCAN_VARIANT_ALL(OP, 8, I_A, 3, 3, 2, 3, 2),                                          \
        GBSCAN_VARIANT_ALL(OP, 8, I_A, 5, 2, 2, 4, 2),                                          \
        GBSCAN_VARIANT_ALL(OP, 8, I_B, 4, 2, 2, 3, 2),                                          \
    };                                                                                          \
    const Family& FN() {                                                                        \
        static const Family f{3, kVariants##OP, &launch_scan_sums<OP>, GBSCAN_RESIDENT(OP)};                         \
        return f;                                                                               \
    }

// 4-byte elements: 20 / 28 items per thread; 8-byte: 10 / 14 (the same bytes)
GBSCAN_OP_FAMILY_W(family_max_i64, OpMaxI64, 10, 14)
GBSCAN_OP_FAMILY_W(family_min_i64, OpMinI64, 10, 14)
GBSCAN_OP_FAMILY_W(family_max_u32, OpMaxU32, 20, 28)
GBSCAN_OP_FAMILY_W(family_min_u32, OpMinU32, 20, 28)

#define GBSCAN_SEG_OP_FAMILY(FN, OP)                                                            \
    static const Variant kSegVariants##OP[] = {                                                 \
        GBSCAN_VARIANT_SEG_PT(OP, 8, 20, 4, 2),                                                 \
        GBSCAN_VARIANT_SEG_PT(OP, 8, 20, 3, 2),                                                 \
    };                                                                                          \
    const Family& FN() {                                                                        \
        static const Family f{2, kSegVariants##OP, nullptr};                                    \
        return f;                                                                               \
    }

GBSCAN_SEG_OP_FAMILY(family_seg_max_i32, OpMaxI32)
GBSCAN_SEG_OP_FAMILY(family_seg_min_i32, OpMinI32)
GBSCAN_SEG_OP_FAMILY(family_seg_max_f32, OpMaxF32)
GBSCAN_SEG_OP_FAMILY(family_seg_min_f32, OpMinF32)

}  // namespace gbscan
