// k_ops.cu — scans under other associative operators than +: running maximum
// and running minimum of int32 and fp32 arrays (single-pass, two-pass and
// partitioned, three launch shapes each); and stream compaction, the scan of
// keep flags fused with the gather it drives (on the partitioned scan and on
// the single-pass chained scan).
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

// The compaction on the single-pass chained scan: NW consumer warps x NV
// 16-byte vectors, S stages (one agent warp each), MB blocks per SM.
template <int NW, int NV, int STAGES, int MINB>
cudaError_t launch_lbc(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(lb_compact_kernel<NW, NV, STAGES, 1, MINB>, lbc_threads<NW, STAGES>(),
                             lbc_smem_bytes<NW, NV, STAGES>(), occ_cache, p, stream);
}
#define GBSCAN_VARIANT_COMPACT_LB(NW, NV, S, MB)                                                 \
    Variant {                                                                                  \
        lbc_threads<NW, S>(), NV * 4, S, lbc_tile<NW, NV>(), &launch_lbc<NW, NV, S, MB>, nullptr, \
            nullptr, nullptr, 0                                                                \
    }

// Variants 0-2: the partitioned compaction (the faster from 2^26 elements
// up); 3: the single-pass one (the faster below, where its one pass and
// smaller fixed cost count for more; of the shapes measured, 8 consumer warps
// x 5 vectors, 4 stages, 2 blocks per SM was the fastest at every size).
static const Variant kCompact[] = {
    GBSCAN_VARIANT_COMPACT(8, 20, 3, 2),
    GBSCAN_VARIANT_COMPACT(16, 28, 2, 1),
    GBSCAN_VARIANT_COMPACT(8, 28, 3, 2),
    GBSCAN_VARIANT_COMPACT_LB(8, 5, 4, 2),
};

const Family& family_compact() {
    static const Family f{4, kCompact, nullptr};
    return f;
}

}  // namespace gbscan
