// gbscan_launch.cuh — host-side launch templates and the variant tables.
#pragma once

#include <atomic>
#include <cstdint>

#include "kernels.cuh"
#include "lookback.cuh"
#include "resident.cuh"
#include "partitioned.cuh"
#include "rows.cuh"
#include "compact.cuh"

namespace gbscan {

using LaunchFn = cudaError_t (*)(const Params&, cudaStream_t);
using SumsFn = cudaError_t (*)(unsigned long long*, int64_t, cudaStream_t);
using CapacityFn = int64_t (*)();

// One launch shape of a kernel family.
struct Variant {
    int threads, items, stages, tile;  // single-pass kernel: block threads (with the
                                       // loader warp and one agent warp per stage)
    LaunchFn single_pass;  // chained scan with decoupled look-back
    LaunchFn reduce;       // two-pass: tile sums (null where not built)
    LaunchFn scan_offset;  // two-pass: scan with the scanned tile sums
    LaunchFn partitioned;  // cache-friendly partitioned scan (null where not built)
    int max_chunk_tiles;   // partitioned: most tiles a chunk may have
    LaunchFn rowblock;     // row kinds: whole rows per tile, no look-back (null elsewhere)
    int rowblock_tile;     // row kinds: the longest row the row-block kernel takes
};

struct Family {
    int num_variants;
    const Variant* variants;
    SumsFn scan_sums;  // two-pass: exclusive scan of the tile sums (null where not built)
    LaunchFn resident;            // the resident scan (one block per tile of resident_tile
    int resident_tile;            //   elements), or null where not built;
    CapacityFn resident_capacity; //   the most tiles it takes on the current device
};

int device_sm_count(int device);

// Launch a kernel as a persistent grid: one block per resident slot, never
// more blocks than tiles.  Shared-memory opt-in and occupancy are queried once
// per device and kernel.  A cooperative launch guarantees that all blocks are
// resident at once (or fails), for kernels whose blocks take work statically.
template <class Kernel>
cudaError_t launch_persistent(Kernel kern, int threads, int smem, std::atomic<int>* occ_cache,
                              const Params& p, cudaStream_t stream, bool cooperative = false) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int occ = (dev >= 0 && dev < 64) ? occ_cache[dev].load(std::memory_order_relaxed) : 0;
    if (occ <= 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
        if (e != cudaSuccess) return e;
        if (occ <= 0) return cudaErrorInvalidConfiguration;
        if (dev >= 0 && dev < 64) occ_cache[dev].store(occ, std::memory_order_relaxed);
    }
    const int sms = device_sm_count(dev);
    if (sms <= 0) return cudaErrorInvalidDevice;
    int64_t grid = static_cast<int64_t>(sms) * occ;
    if (grid > p.num_tiles) grid = p.num_tiles;
    if (grid < 1) grid = 1;
    if (!cooperative) {
        kern<<<static_cast<unsigned>(grid), threads, smem, stream>>>(p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <class Op, int CWARPS, int ITEMS, int STAGES, int HEADS, bool REVERSE, int LB, int MINB>
cudaError_t launch_ws(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(ws_scan_kernel<Op, CWARPS, ITEMS, STAGES, HEADS, REVERSE, LB, MINB>,
                             ws_threads<CWARPS, STAGES>(), ws_smem_bytes<Op, CWARPS, ITEMS, STAGES>(),
                             occ_cache, p, stream);
}

template <class Op, int NW, int NV, int STAGES, int LB, int MINB>
cudaError_t launch_lb(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(lb_scan_kernel<Op, NW, NV, STAGES, LB, MINB>, lb_threads<NW, STAGES>(),
                             lb_smem_bytes<Op, NW, NV, STAGES>(), occ_cache, p, stream);
}

// Blocks of the resident scan that fit the current device at once (SMs x
// blocks per SM, at most kResidentMaxTiles), or -1 if CUDA cannot say.
template <class Op, int THREADS, int ITEMS, int MINB>
int64_t resident_capacity() {
    static std::atomic<int> occ_cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    int occ = (dev >= 0 && dev < 64) ? occ_cache[dev].load(std::memory_order_relaxed) : 0;
    if (occ <= 0) {
        auto kern = resident_scan_kernel<Op, THREADS, ITEMS, MINB>;
        const int smem = resident_smem_bytes<Op, THREADS, ITEMS>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem) != cudaSuccess)
            return -1;
        if (occ <= 0) return -1;
        if (dev >= 0 && dev < 64) occ_cache[dev].store(occ, std::memory_order_relaxed);
    }
    const int sms = device_sm_count(dev);
    if (sms <= 0) return -1;
    const int64_t cap = static_cast<int64_t>(sms) * occ;
    return cap < kResidentMaxTiles ? cap : kResidentMaxTiles;
}

// One block per tile, all resident: a cooperative launch, which the runtime
// starts only when every block can run at once.  The host checks the tile
// count against resident_capacity first.
template <class Op, int THREADS, int ITEMS, int MINB>
cudaError_t launch_resident(const Params& p, cudaStream_t stream) {
    const int64_t cap = resident_capacity<Op, THREADS, ITEMS, MINB>();
    if (cap < 0) return cudaErrorInvalidConfiguration;
    if (p.num_tiles < 1 || p.num_tiles > cap) return cudaErrorCooperativeLaunchTooLarge;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(p.num_tiles));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = static_cast<size_t>(resident_smem_bytes<Op, THREADS, ITEMS>());
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, resident_scan_kernel<Op, THREADS, ITEMS, MINB>, p);
}

// The resident scan of a plain family: 256 threads x 80 bytes of items (20
// KB tiles: 5120 4-byte or 2560 8-byte elements); 4 blocks per SM (608 tiles
// on 152 SMs) for 4-byte accumulators, 3 for 8-byte and pair accumulators.
#define GBSCAN_RESIDENT_ITEMS(OP) (80 / static_cast<int>(sizeof(OP::T)))
#define GBSCAN_RESIDENT_MINB(OP) (sizeof(OP::Acc) == 4 ? 4 : 3)
#define GBSCAN_RESIDENT(OP)                                                                    \
    &launch_resident<OP, 256, GBSCAN_RESIDENT_ITEMS(OP), GBSCAN_RESIDENT_MINB(OP)>,              \
        256 * GBSCAN_RESIDENT_ITEMS(OP),                                                       \
        &resident_capacity<OP, 256, GBSCAN_RESIDENT_ITEMS(OP), GBSCAN_RESIDENT_MINB(OP)>

template <class Op, int THREADS, int ITEMS, int STAGES, int MODE>
cudaError_t launch_tp(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(two_pass_kernel<Op, THREADS, ITEMS, STAGES, MODE>, THREADS,
                             tp_smem_bytes<Op, THREADS, ITEMS, STAGES>(), occ_cache, p, stream);
}

template <class Op, int CWARPS, int ITEMS, int STAGES, int MINB, int HEADS>
cudaError_t launch_pt(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(partitioned_kernel<Op, CWARPS, ITEMS, STAGES, MINB, HEADS>,
                             pt_threads<CWARPS>(), pt_smem_bytes<Op, CWARPS, ITEMS, STAGES, HEADS>(),
                             occ_cache, p, stream);
}

template <class Op, int CWARPS, int ITEMS, int STAGES, bool REVERSE, int MINB>
cudaError_t launch_rb(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(rowblock_kernel<Op, CWARPS, ITEMS, STAGES, REVERSE, MINB>,
                             rb_threads<CWARPS>(), rb_smem_bytes<Op, CWARPS, ITEMS, STAGES>(),
                             occ_cache, p, stream);
}

template <int CWARPS, int ITEMS, int STAGES, int MINB>
cudaError_t launch_cp(const Params& p, cudaStream_t stream) {
    static std::atomic<int> occ_cache[64];
    return launch_persistent(compact_kernel<CWARPS, ITEMS, STAGES, MINB>, pt_threads<CWARPS>(),
                             cp_smem_bytes<CWARPS, ITEMS, STAGES>(), occ_cache, p, stream);
}

template <class Op>
cudaError_t launch_scan_sums(unsigned long long* rec, int64_t num_tiles, cudaStream_t stream) {
    scan_tile_sums_kernel<Op, 1024><<<1, 1024, 0, stream>>>(rec, num_tiles);
    return cudaGetLastError();
}

// Variant descriptors.  A variant names the single-pass kernel's shape
// (consumer warps CW, items per thread I, pipeline stages S, look-back tiles per
// lane LB, minimum resident blocks MB) and, for plain scans, the two-pass
// kernels of the same tile (CW * 32 threads, I items, TS stages).  Item counts
// fill whole 16-byte vectors, an odd number of them per thread so that the
// 128-bit shared-memory reads are bank-conflict free.
#define GBSCAN_VARIANT_SP(OP, CW, I, S, LB, MB, HEADS_, REV_)                                   \
    Variant {                                                                                  \
        (CW + 1 + S) * 32, I, S, CW * 32 * I, &launch_ws<OP, CW, I, S, HEADS_, REV_, LB, MB>, nullptr, \
            nullptr, nullptr, 0                                                                \
    }
// Batched segmented scans with the partitioned kernel (a head bitmap in place
// of the offsets lookups): CW consumer warps x I items, S stages, MB blocks per
// SM; threads counts the consumer, loader and chunk scanner warps.
#define GBSCAN_VARIANT_SEG_PT(OP, CW, I, S, MB)                                                 \
    Variant {                                                                                  \
        (CW + 2) * 32, I, S, CW * 32 * I, nullptr, nullptr, nullptr,                           \
            &launch_pt<OP, CW, I, S, MB, kOffsetHeads>, kMaxChunkTiles                         \
    }

// Stream compaction (4-byte payloads): CW consumer warps x I items, S stages,
// MB blocks per SM; threads counts the consumer, loader and scanner warps.
#define GBSCAN_VARIANT_COMPACT(CW, I, S, MB)                                                    \
    Variant {                                                                                  \
        (CW + 2) * 32, I, S, CW * 32 * I, nullptr, nullptr, nullptr, &launch_cp<CW, I, S, MB>,   \
            kMaxChunkTiles                                                                     \
    }

// Row kinds: the chained kernel with row heads (any row length) and the
// row-block kernel (RCW consumer warps x RI items, RS stages, RMB blocks per
// SM) for rows of at most RCW * 32 * RI elements.
#define GBSCAN_VARIANT_ROWS(OP, CW, I, S, LB, MB, REV_, RCW, RI, RS, RMB)                      \
    Variant {                                                                                  \
        (CW + 1 + S) * 32, I, S, CW * 32 * I, &launch_ws<OP, CW, I, S, kRowHeads, REV_, LB, MB>, \
            nullptr, nullptr, nullptr, 0, &launch_rb<OP, RCW, RI, RS, REV_, RMB>, RCW * 32 * RI   \
    }
// Plain scans: one tile (CW consumer warps x I items) for all three
// algorithms.  Single-pass: the look-back kernel with SPS stages and SPMB
// blocks per SM (CW consumer warps, a loader warp and SPS agent warps; the
// group walk reads one group word per lane and round).  Two-pass: CW * 32
// threads, TS stages.  Partitioned: PTS stages, PTMB blocks per SM.
#define GBSCAN_VARIANT_ALL(OP, CW, I, SPS, SPMB, TS, PTS, PTMB)                                  \
    Variant {                                                                                   \
        (CW + 1 + SPS) * 32, I, SPS, CW * 32 * I,                                               \
            &launch_lb<OP, CW, I / (16 / static_cast<int>(sizeof(OP::T))), SPS, 1, SPMB>,        \
            &launch_tp<OP, CW * 32, I, TS, kReduce>, &launch_tp<OP, CW * 32, I, TS, kScanOffset>, \
            &launch_pt<OP, CW, I, PTS, PTMB, kNoHeads>, kMaxChunkTiles                           \
    }

// Families, one per translation unit group.
const Family& family_scan_i32();
const Family& family_scan_i64();
const Family& family_scan_f32();
const Family& family_scan_f32c();
const Family& family_scan_f64();
const Family& family_seg_i32();
const Family& family_seg_f32();
const Family& family_rows_f32();
const Family& family_rows_f64();
const Family& family_rows_rev_f32();
const Family& family_rows_rev_f64();
const Family& family_max_i32();
const Family& family_min_i32();
const Family& family_max_f32();
const Family& family_min_f32();
const Family& family_compact();
const Family& family_max_i64();
const Family& family_min_i64();
const Family& family_max_u32();
const Family& family_min_u32();
const Family& family_seg_max_i32();
const Family& family_seg_min_i32();
const Family& family_seg_max_f32();
const Family& family_seg_min_f32();

// Smallest tile (in elements) of any variant for an element size: sizes the
// workspace so that every variant fits.
constexpr int kMinTile4 = 256 * 12;  // 8 consumer warps x 12 items
constexpr int kMinTile8 = 256 * 6;

}  // namespace gbscan
