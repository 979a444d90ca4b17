// gbscan_launch.cuh — host-side launch templates and the variant tables.
#pragma once

#include <atomic>
#include <cstdint>

#include "gbscan_device.cuh"

namespace gbscan {

using LaunchFn = cudaError_t (*)(const Params&, cudaStream_t);
using SumsFn = cudaError_t (*)(TileRecord*, int64_t, cudaStream_t);

// One launch shape of a kernel family.
struct Variant {
    int threads, items, stages, tile;
    LaunchFn single_pass;  // chained scan with decoupled look-back
    LaunchFn reduce;       // two-pass: tile sums (null where not built)
    LaunchFn scan_offset;  // two-pass: scan with the scanned tile sums
};

struct Family {
    int num_variants;
    const Variant* variants;
    SumsFn scan_sums;  // two-pass: exclusive scan of the tile sums (null where not built)
};

int device_sm_count(int device);

// Launch a tile kernel as a persistent grid: one block per resident slot,
// never more blocks than tiles.  Shared-memory opt-in and occupancy are
// queried once per device and kernel.
template <class Op, int THREADS, int ITEMS, int STAGES, int MODE, int HEADS, bool REVERSE>
cudaError_t launch_tile(const Params& p, cudaStream_t stream) {
    auto kern = tile_scan_kernel<Op, THREADS, ITEMS, STAGES, MODE, HEADS, REVERSE>;
    constexpr int smem = tile_smem_bytes<Op, THREADS, ITEMS, STAGES, HEADS>();
    static std::atomic<int> occ_cache[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int occ = (dev >= 0 && dev < 64) ? occ_cache[dev].load(std::memory_order_relaxed) : 0;
    if (occ <= 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem);
        if (e != cudaSuccess) return e;
        if (occ <= 0) return cudaErrorInvalidConfiguration;
        if (dev >= 0 && dev < 64) occ_cache[dev].store(occ, std::memory_order_relaxed);
    }
    const int sms = device_sm_count(dev);
    if (sms <= 0) return cudaErrorInvalidDevice;
    int64_t grid = static_cast<int64_t>(sms) * occ;
    if (grid > p.num_tiles) grid = p.num_tiles;
    if (grid < 1) grid = 1;
    kern<<<static_cast<unsigned>(grid), THREADS, smem, stream>>>(p);
    return cudaGetLastError();
}

template <class Op>
cudaError_t launch_scan_sums(TileRecord* rec, int64_t num_tiles, cudaStream_t stream) {
    scan_tile_sums_kernel<Op, 1024><<<1, 1024, 0, stream>>>(rec, num_tiles);
    return cudaGetLastError();
}

// Variant descriptors.  VEC-filling item counts: 4-byte elements take multiples
// of 4 items, 8-byte elements multiples of 2; an odd number of 16-byte vectors
// per thread keeps the 128-bit shared-memory reads bank-conflict free.
#define GBSCAN_VARIANT_SP(OP, T_, I_, S_, HEADS_, REV_)                                     \
    Variant {                                                                              \
        T_, I_, S_, T_ * I_, &launch_tile<OP, T_, I_, S_, kSinglePass, HEADS_, REV_>, nullptr, \
            nullptr                                                                        \
    }
#define GBSCAN_VARIANT_ALL(OP, T_, I_, S_)                                          \
    Variant {                                                                      \
        T_, I_, S_, T_ * I_, &launch_tile<OP, T_, I_, S_, kSinglePass, kNoHeads, false>, \
            &launch_tile<OP, T_, I_, S_, kReduce, kNoHeads, false>,                \
            &launch_tile<OP, T_, I_, S_, kScanOffset, kNoHeads, false>             \
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

// Smallest tile (in elements) of any variant for an element size: sizes the
// workspace so that every variant fits.
constexpr int kMinTile4 = 256 * 12;
constexpr int kMinTile8 = 256 * 6;

}  // namespace gbscan
