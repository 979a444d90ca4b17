// capi.cu — the C ABI declared in include/gbscan.h: argument checks, workspace
// layout, and dispatch to the tile kernels.  Host code plus three small
// kernels (segment locator, debug-field writer, copy reference).
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gbscan_launch.cuh"

namespace gbscan {

int device_sm_count(int device) {
    static std::atomic<int> cache[64];
    if (device >= 0 && device < 64) {
        const int c = cache[device].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    if (device >= 0 && device < 64) cache[device].store(sms, std::memory_order_relaxed);
    return sms;
}

// aux[t] = first segment whose start is >= t * tile (lower bound over the
// offsets), for t = 0..num_tiles; the tile kernel marks the starts of
// segments [aux[t], aux[t+1]) as heads.  Also checks the CSR offsets.
__global__ void segment_locate_kernel(const int64_t* offsets, int64_t num_segments, int64_t n,
                                      int64_t tile, int64_t num_tiles, unsigned long long* rec,
                                      Header* hdr) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t t = first; t <= num_tiles; t += stride) {
        int64_t pos = t * tile;
        if (pos > n) pos = n;
        int64_t lo = 0, hi = num_segments + 1;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (offsets[mid] < pos)
                lo = mid + 1;
            else
                hi = mid;
        }
        *rec_aux(rec, t) = static_cast<unsigned long long>(lo);
    }
    bool bad = false;
    for (int64_t j = first; j < num_segments; j += stride)
        if (offsets[j] > offsets[j + 1]) bad = true;
    if (first == 0 && (offsets[0] != 0 || offsets[num_segments] != n)) bad = true;
    if (bad) record_error(hdr, GBSCAN_ERR_INVALID_ARG, -1);
}

// Head bitmap of a batched segmented scan: bit i of word i / 32 is set when
// element i starts a segment.  Block b builds words [1024 b, 1024 b + 1024)
// in shared memory and writes each once (no clearing pass, no global
// atomics): it finds the first segment starting in its range with a 256-way
// search (two rounds for 65,536 segments), then sets the bits of the segments
// that start in the range.  Starts outside [0, n) set nothing.  The blocks
// also check the offsets (monotone, offsets[0] = 0, offsets[S] = n) and record
// GBSCAN_ERR_INVALID_ARG for malformed ones.  256 threads per block.
constexpr int kBitmapBlockWords = 1024;

__global__ void __launch_bounds__(256) segment_bitmap_kernel(const int64_t* offsets, int64_t num_segments,
                                                             int64_t n, uint32_t* bitmap, int64_t words,
                                                             Header* hdr) {
    __shared__ uint32_t w[kBitmapBlockWords];
    const int tid = threadIdx.x;
    const int64_t w0 = static_cast<int64_t>(blockIdx.x) * kBitmapBlockWords;
    const int64_t start = w0 * 32;
    const int64_t end = start + 32ll * kBitmapBlockWords;
    for (int i = tid; i < kBitmapBlockWords; i += 256) w[i] = 0u;
    // j0 = the number of segments that start before `start`
    int64_t lo = 0, len = num_segments;
    while (len > 0) {
        const int64_t step = (len + 255) / 256;
        const int64_t idx = lo + static_cast<int64_t>(tid) * step;
        const int below = (idx < lo + len && offsets[idx] < start) ? 1 : 0;
        const int cnt = __syncthreads_count(below);
        if (cnt == 0) break;
        const int64_t nlo = lo + static_cast<int64_t>(cnt - 1) * step + 1;
        const int64_t nhi = (lo + cnt * step) < (lo + len) ? (lo + cnt * step) : (lo + len);
        lo = nlo;
        len = nhi - nlo;
    }
    __syncthreads();
    for (int64_t j = lo + tid; j < num_segments; j += 256) {
        const int64_t pos = offsets[j];
        if (pos >= end) break;
        if (pos >= start && pos < n) atomicOr(&w[(pos - start) >> 5], 1u << (pos & 31));
    }
    __syncthreads();
    for (int i = tid; i < kBitmapBlockWords && w0 + i < words; i += 256) bitmap[w0 + i] = w[i];
    // this block's share of the offset checks
    bool bad = false;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * 256;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * 256 + tid; j < num_segments; j += stride)
        if (offsets[j] > offsets[j + 1]) bad = true;
    if (blockIdx.x == 0 && tid == 0 && (offsets[0] != 0 || offsets[num_segments] != n)) bad = true;
    if (bad) record_error(hdr, GBSCAN_ERR_INVALID_ARG, -1);
}

__global__ void set_debug_kernel(Header* hdr, uint32_t spin_limit_us, int64_t drop_tile,
                                 uint32_t delay_ns_max) {
    hdr->spin_limit_us = spin_limit_us;
    hdr->drop_tile_plus1 = drop_tile < 0 ? 0 : drop_tile + 1;
    hdr->delay_ns_max = delay_ns_max;
}

__global__ void __launch_bounds__(256) copy_kernel(const uint4* __restrict__ src,
                                                   uint4* __restrict__ dst, int64_t n16) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const uint4 a = __ldcs(src + i), b = __ldcs(src + i + stride);
        const uint4 c = __ldcs(src + i + 2 * stride), d = __ldcs(src + i + 3 * stride);
        __stcs(dst + i, a);
        __stcs(dst + i + stride, b);
        __stcs(dst + i + 2 * stride, c);
        __stcs(dst + i + 3 * stride, d);
    }
    for (; i < n16; i += stride) __stcs(dst + i, __ldcs(src + i));
}

namespace {

// An NVTX range around each C-ABI call that launches work, named after the
// entry point, so that a profiler's timeline shows which call a kernel came
// from.  Without a tool attached a range costs a pointer test.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define GBSCAN_NVTX_RANGE(name) NvtxRange gbscan_nvtx_range_(name)

constexpr size_t kHeaderBytes = sizeof(Header);
constexpr int64_t kMaxTiles = (int64_t(1) << 31) - (int64_t(1) << 24);

int min_tile(gbscan_dtype dt) {
    return (dt == GBSCAN_I64 || dt == GBSCAN_F64) ? kMinTile8 : kMinTile4;
}

bool valid_dtype(int dt) { return dt >= GBSCAN_I32 && dt <= GBSCAN_U32; }

// Records needed for n elements at tile size `tile`: one per tile plus the
// segment locator's end sentinel; they come in blocks of 16.
constexpr int64_t records_for(int64_t n, int tile) { return (n + tile - 1) / tile + 1; }

constexpr size_t record_bytes(int64_t records) {
    return static_cast<size_t>((records + 15) / 16) * kRecBlockBytes;
}

// scan_inclusive_i32_noalloc runs the int32 plain family's variant 0 (8
// consumer warps x 20 items); its scratch must hold the header and that
// tile's records for GBSCAN_NOALLOC_MAX_N elements.  The tile is checked
// against the variant table when the entry point runs.
constexpr int kNoallocTile = 8 * 32 * 20;
static_assert(sizeof(Header) + record_bytes(records_for(GBSCAN_NOALLOC_MAX_N, kNoallocTile)) <=
                  GBSCAN_NOALLOC_SCRATCH_BYTES,
              "the no-allocation scratch must hold GBSCAN_NOALLOC_MAX_N elements' records");

// The head bitmap of a segmented scan sits after the largest record region a
// call on n elements of this size can use, and covers every variant's last
// tile: bits for n + kSegBitmapPad elements, in whole 16-byte units.
constexpr int64_t kSegBitmapPad = 16384;

size_t seg_bitmap_offset(int64_t n, size_t esz) {
    return kHeaderBytes + record_bytes(records_for(n, esz == 8 ? kMinTile8 : kMinTile4));
}

size_t seg_bitmap_bytes(int64_t n) {
    return static_cast<size_t>((n + kSegBitmapPad + 127) / 128) * 16;
}

gbscan_status check_ws(void* ws, size_t ws_bytes, int64_t records) {
    if (ws == nullptr) return GBSCAN_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return GBSCAN_ERR_WORKSPACE;
    if (ws_bytes < kHeaderBytes + record_bytes(records)) return GBSCAN_ERR_WORKSPACE;
    return GBSCAN_OK;
}

bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

// in/out checks shared by every entry point: null, alignment to the element
// size, and overlap other than exact aliasing.
gbscan_status check_io(const void* in, const void* out, int64_t n, size_t esz) {
    if (in == nullptr || out == nullptr) return GBSCAN_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(in) % esz || reinterpret_cast<uintptr_t>(out) % esz)
        return GBSCAN_ERR_ALIGNMENT;
    const size_t bytes = static_cast<size_t>(n) * esz;
    if (in != out && ranges_overlap(in, bytes, out, bytes)) return GBSCAN_ERR_INVALID_ARG;
    return GBSCAN_OK;
}

gbscan_status from_cuda(cudaError_t e) { return e == cudaSuccess ? GBSCAN_OK : GBSCAN_ERR_CUDA; }

Params make_params(const void* in, void* out, int64_t n, int tile, void* ws, size_t ws_bytes) {
    Params p{};
    p.in = in;
    p.out = out;
    p.n = n;
    p.num_tiles = (n + tile - 1) / tile;
    p.hdr = static_cast<Header*>(ws);
    p.rec = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(ws) + kHeaderBytes);
    p.rec_capacity = static_cast<int64_t>((ws_bytes - kHeaderBytes) / kRecBlockBytes) * 16;
    p.fast = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    return p;
}

// Tiles per chunk of the partitioned scan: about GBSCAN_CHUNK_BYTES of input
// (default 8 MiB: with the default four-chunk lag, five chunks of input,
// 40 MiB, are live in the 129 MB L2 at a time, next to the streaming stores),
// at least 16 tiles.
static long long env_cached(std::atomic<long long>& cache, const char* name, long long dflt) {
    long long v = cache.load(std::memory_order_relaxed);
    if (v == 0) {
        v = dflt;
        if (const char* e = getenv(name)) {
            const long long b = atoll(e);
            if (b > 0) v = b;
        }
        cache.store(v, std::memory_order_relaxed);
    }
    return v;
}

// GBSCAN_ALGO_AUTO: the resident scan wherever it fits; above that the
// single-pass scan (measured on GB300 with the L2 prefetch ahead of each
// claim: the fastest of the four for int32, fp32, compensated fp32 and int64
// from 2^24 to 2^30 elements).  fp64, whose scans are bound by its adds on
// this part, takes the two-pass scan above the resident size (its entry
// points decide that before calling scan_flat).

int64_t partition_chunk_tiles(const Variant& v, size_t esz) {
    static std::atomic<long long> bytes_cache{0};
    const long long bytes = env_cached(bytes_cache, "GBSCAN_CHUNK_BYTES", 8ll << 20);
    int64_t k = bytes / (static_cast<long long>(v.tile) * static_cast<long long>(esz));
    if (k < kGroup) k = kGroup;
    if (k > v.max_chunk_tiles) k = v.max_chunk_tiles;
    return k;
}

// Chunks between a chunk's reduction and its scan (GBSCAN_CHUNK_LAG, default 4,
// at most 8): the slack the chunk scanner has to publish a chunk's offsets
// before the chunk's second pass starts.
int64_t partition_chunk_lag() {
    static std::atomic<long long> lag_cache{0};
    const long long lag = env_cached(lag_cache, "GBSCAN_CHUNK_LAG", 4);
    return lag > 8 ? 8 : lag;
}

// Whether the family's resident scan takes n elements on the current device.
bool resident_fits(const Family& fam, int64_t n) {
    if (!fam.resident) return false;
    const int64_t cap = fam.resident_capacity();
    return cap > 0 && (n + fam.resident_tile - 1) / fam.resident_tile <= cap;
}

// GBSCAN_ALGO_AUTO for the scans bound by arithmetic (fp64): the resident
// scan where it fits, the two-pass scan above.
gbscan_algo auto_arith_bound(const Family& fam, int64_t n, gbscan_algo algo) {
    if (algo != GBSCAN_ALGO_AUTO) return algo;
    return resident_fits(fam, n) ? GBSCAN_ALGO_RESIDENT : GBSCAN_ALGO_TWO_PASS;
}

// Single-pass, partitioned and compaction scans: how far ahead of each claim
// the loader prefetches a tile into L2, in bytes of input
// (GBSCAN_PREFETCH_BYTES, default 12 MiB; 1 turns the prefetch off).
// Measured on GB300 at int32 2^30 with 28 KB tiles, single-pass: 0.80 of a
// device copy without it, 0.92 at 7-14 MiB ahead; at 56 MiB the prefetched
// lines start to leave L2 before their copy.  The two-pass kernels take no
// prefetch: their static schedule already keeps several grid-wide steps of
// copies in flight, and a prefetch only added requests (0.57 -> 0.53).
constexpr long long kDefaultPrefetchBytes = 12ll << 20;

int64_t single_pass_prefetch_tiles(int tile, size_t esz) {
    static std::atomic<long long> cache{0};
    const long long bytes = env_cached(cache, "GBSCAN_PREFETCH_BYTES", kDefaultPrefetchBytes);
    const long long tile_bytes = static_cast<long long>(tile) * static_cast<long long>(esz);
    return bytes > tile_bytes ? bytes / tile_bytes : 0;
}

gbscan_status scan_flat(const Family& fam, const void* in, void* out, int64_t n, size_t esz,
                        int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                        cudaStream_t stream) {
    if (n < 0) return GBSCAN_ERR_INVALID_ARG;
    if (algo != GBSCAN_ALGO_AUTO && algo != GBSCAN_ALGO_SINGLE_PASS &&
        algo != GBSCAN_ALGO_TWO_PASS && algo != GBSCAN_ALGO_PARTITIONED &&
        algo != GBSCAN_ALGO_RESIDENT)
        return GBSCAN_ERR_INVALID_ARG;
    if (variant < 0 || variant >= fam.num_variants) return GBSCAN_ERR_INVALID_ARG;
    if (n == 0) return GBSCAN_OK;
    gbscan_status st = check_io(in, out, n, esz);
    if (st != GBSCAN_OK) return st;
    const Variant& v = fam.variants[variant];
    if (algo == GBSCAN_ALGO_AUTO) {
        algo = resident_fits(fam, n) ? GBSCAN_ALGO_RESIDENT : GBSCAN_ALGO_SINGLE_PASS;
    }
    if (algo == GBSCAN_ALGO_RESIDENT && !resident_fits(fam, n)) return GBSCAN_ERR_UNSUPPORTED;
    const int tile = algo == GBSCAN_ALGO_RESIDENT ? fam.resident_tile : v.tile;
    if ((n + tile - 1) / tile > kMaxTiles) return GBSCAN_ERR_UNSUPPORTED;
    st = check_ws(ws, ws_bytes, records_for(n, tile));
    if (st != GBSCAN_OK) return st;
    Params p = make_params(in, out, n, tile, ws, ws_bytes);
    p.exclusive = exclusive;
    cudaGetLastError();  // clear a stale, non-sticky error of an earlier call
    if (algo == GBSCAN_ALGO_RESIDENT) return from_cuda(fam.resident(p, stream));
    if (algo == GBSCAN_ALGO_PARTITIONED) {
        if (!v.partitioned) return GBSCAN_ERR_UNSUPPORTED;
        p.chunk_tiles = partition_chunk_tiles(v, esz);
        p.chunk_lag = partition_chunk_lag();
        p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, esz);
        return from_cuda(v.partitioned(p, stream));
    }
    if (algo == GBSCAN_ALGO_TWO_PASS) {
        if (!v.reduce || !v.scan_offset || !fam.scan_sums) return GBSCAN_ERR_UNSUPPORTED;
        cudaError_t e = v.reduce(p, stream);
        if (e == cudaSuccess) e = fam.scan_sums(p.rec, p.num_tiles, stream);
        if (e == cudaSuccess) e = v.scan_offset(p, stream);
        return from_cuda(e);
    }
    p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, esz);
    return from_cuda(v.single_pass(p, stream));
}

gbscan_status scan_rows_impl(const Family& fam, const void* in, void* out, int64_t rows,
                             int64_t cols, size_t esz, int exclusive, void* ws, size_t ws_bytes,
                             int variant, cudaStream_t stream) {
    if (rows < 0 || cols < 0) return GBSCAN_ERR_INVALID_ARG;
    if (variant < 0 || variant >= fam.num_variants) return GBSCAN_ERR_INVALID_ARG;
    if (rows == 0 || cols == 0) return GBSCAN_OK;
    if (rows > INT64_MAX / cols) return GBSCAN_ERR_UNSUPPORTED;
    const int64_t n = rows * cols;
    gbscan_status st = check_io(in, out, n, esz);
    if (st != GBSCAN_OK) return st;
    const Variant& v = fam.variants[variant];
    if ((n + v.tile - 1) / v.tile > kMaxTiles) return GBSCAN_ERR_UNSUPPORTED;
    st = check_ws(ws, ws_bytes, records_for(n, v.tile));
    if (st != GBSCAN_OK) return st;
    Params p = make_params(in, out, n, v.tile, ws, ws_bytes);
    p.exclusive = exclusive;
    p.cols = cols;
    cudaGetLastError();
    if (v.rowblock && cols <= v.rowblock_tile) return from_cuda(v.rowblock(p, stream));
    p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, esz);
    return from_cuda(v.single_pass(p, stream));
}

gbscan_status scan_seg_impl(const Family& fam, const void* in, void* out, int64_t n,
                            const int64_t* offsets, int64_t num_segments, size_t esz,
                            int exclusive, void* ws, size_t ws_bytes, int variant,
                            cudaStream_t stream) {
    if (n < 0 || num_segments < 0 || num_segments > INT32_MAX) return GBSCAN_ERR_INVALID_ARG;
    if (variant < 0 || variant >= fam.num_variants) return GBSCAN_ERR_INVALID_ARG;
    if (n == 0) return GBSCAN_OK;  // every segment is empty
    if (num_segments == 0 || offsets == nullptr) return GBSCAN_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(offsets) % 8) return GBSCAN_ERR_ALIGNMENT;
    gbscan_status st = check_io(in, out, n, esz);
    if (st != GBSCAN_OK) return st;
    const Variant& v = fam.variants[variant];
    if ((n + v.tile - 1) / v.tile > kMaxTiles) return GBSCAN_ERR_UNSUPPORTED;
    st = check_ws(ws, ws_bytes, records_for(n, v.tile));
    if (st != GBSCAN_OK) return st;
    Params p = make_params(in, out, n, v.tile, ws, ws_bytes);
    p.exclusive = exclusive;
    p.offsets = offsets;
    p.num_segments = num_segments;
    cudaGetLastError();
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sm_count(dev);
    int64_t work = num_segments > p.num_tiles + 1 ? num_segments : p.num_tiles + 1;
    int64_t blocks = (work + 255) / 256;
    const int64_t max_blocks = static_cast<int64_t>(sms > 0 ? sms : 1) * 8;
    if (blocks > max_blocks) blocks = max_blocks;
    if (v.partitioned) {
        // the head bitmap (which also checks the offsets), then the scan
        const size_t boff = seg_bitmap_offset(n, esz), bbytes = seg_bitmap_bytes(n);
        if (ws_bytes < boff + bbytes) return GBSCAN_ERR_WORKSPACE;
        uint32_t* bitmap = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(ws) + boff);
        const int64_t words = static_cast<int64_t>(bbytes / 4);
        const int64_t bb = (words + kBitmapBlockWords - 1) / kBitmapBlockWords;
        segment_bitmap_kernel<<<static_cast<unsigned>(bb), 256, 0, stream>>>(offsets, num_segments, n,
                                                                             bitmap, words, p.hdr);
        if (cudaGetLastError() != cudaSuccess) return GBSCAN_ERR_CUDA;
        p.bitmap = bitmap;
        p.chunk_tiles = partition_chunk_tiles(v, esz);
        p.chunk_lag = partition_chunk_lag();
        p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, esz);
        return from_cuda(v.partitioned(p, stream));
    }
    // each tile's first segment for the single-pass kernel (also checks the
    // offsets)
    segment_locate_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        offsets, num_segments, n, v.tile, p.num_tiles, p.rec, p.hdr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return GBSCAN_ERR_CUDA;
    p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, esz);
    return from_cuda(v.single_pass(p, stream));
}

gbscan_status compact_impl(const void* in, const uint8_t* flags, void* out, int64_t n,
                           int64_t* count, void* ws, size_t ws_bytes, int variant,
                           cudaStream_t stream) {
    const Family& fam = family_compact();
    if (n < 0 || count == nullptr || variant < 0 || variant >= fam.num_variants)
        return GBSCAN_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(count) % 8) return GBSCAN_ERR_ALIGNMENT;
    cudaGetLastError();
    if (n == 0) return from_cuda(cudaMemsetAsync(count, 0, sizeof(int64_t), stream));
    if (flags == nullptr || in == out) return GBSCAN_ERR_INVALID_ARG;
    gbscan_status st = check_io(in, out, n, 4);
    if (st != GBSCAN_OK) return st;
    const Variant& v = fam.variants[variant];
    if ((n + v.tile - 1) / v.tile > kMaxTiles) return GBSCAN_ERR_UNSUPPORTED;
    st = check_ws(ws, ws_bytes, records_for(n, v.tile));
    if (st != GBSCAN_OK) return st;
    Params p = make_params(in, out, n, v.tile, ws, ws_bytes);
    p.flags = flags;
    p.total_out = reinterpret_cast<unsigned long long*>(count);
    p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, 4);
    if (v.single_pass) return from_cuda(v.single_pass(p, stream));  // the single-pass compaction
    // whole R groups per chunk
    p.chunk_tiles = (partition_chunk_tiles(v, 4) + kCpGroup - 1) / kCpGroup * kCpGroup;
    p.chunk_lag = partition_chunk_lag();
    return from_cuda(v.partitioned(p, stream));
}

const Family* family_for(gbscan_dtype dt, gbscan_kind kind) {
    switch (kind) {
    case GBSCAN_KIND_SCAN:
        switch (dt) {
        case GBSCAN_I32: return &family_scan_i32();
        case GBSCAN_U32: return &family_scan_i32();  // sums: the same bits
        case GBSCAN_I64: return &family_scan_i64();
        case GBSCAN_F32: return &family_scan_f32();
        case GBSCAN_F64: return &family_scan_f64();
        }
        break;
    case GBSCAN_KIND_SEGMENTED:
        if (dt == GBSCAN_I32) return &family_seg_i32();
        if (dt == GBSCAN_F32) return &family_seg_f32();
        break;
    case GBSCAN_KIND_ROWS:
        if (dt == GBSCAN_F32) return &family_rows_f32();
        if (dt == GBSCAN_F64) return &family_rows_f64();
        break;
    case GBSCAN_KIND_SCAN_MAX:
        if (dt == GBSCAN_I32) return &family_max_i32();
        if (dt == GBSCAN_F32) return &family_max_f32();
        if (dt == GBSCAN_I64) return &family_max_i64();
        if (dt == GBSCAN_U32) return &family_max_u32();
        break;
    case GBSCAN_KIND_SCAN_MIN:
        if (dt == GBSCAN_I32) return &family_min_i32();
        if (dt == GBSCAN_F32) return &family_min_f32();
        if (dt == GBSCAN_I64) return &family_min_i64();
        if (dt == GBSCAN_U32) return &family_min_u32();
        break;
    case GBSCAN_KIND_COMPACT:
        if (dt == GBSCAN_I32 || dt == GBSCAN_F32) return &family_compact();
        break;
    case GBSCAN_KIND_SEGMENTED_MAX:
        if (dt == GBSCAN_I32) return &family_seg_max_i32();
        if (dt == GBSCAN_F32) return &family_seg_max_f32();
        break;
    case GBSCAN_KIND_SEGMENTED_MIN:
        if (dt == GBSCAN_I32) return &family_seg_min_i32();
        if (dt == GBSCAN_F32) return &family_seg_min_f32();
        break;
    }
    return nullptr;
}

}  // namespace
// Scratch of scan_inclusive_i32_noalloc: a header and tile records for up to
// GBSCAN_NOALLOC_MAX_N elements at the default int32 tile.  Zero at module
// load, like a zeroed workspace.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GBSCAN_NOALLOC_SCRATCH_BYTES];

}  // namespace gbscan

using namespace gbscan;

extern "C" {

gbscan_status gbscan_workspace_size(gbscan_dtype dtype, gbscan_kind kind, int64_t n,
                                    int64_t num_segments, size_t* bytes) {
    if (bytes == nullptr || n < 0 || num_segments < 0 || !valid_dtype(dtype))
        return GBSCAN_ERR_INVALID_ARG;
    if (kind < GBSCAN_KIND_SCAN || kind > GBSCAN_KIND_SEGMENTED_MIN) return GBSCAN_ERR_INVALID_ARG;
    if (num_segments > INT32_MAX) return GBSCAN_ERR_UNSUPPORTED;
    const int tile = min_tile(dtype);
    if ((n + tile - 1) / tile > kMaxTiles) return GBSCAN_ERR_UNSUPPORTED;
    *bytes = kHeaderBytes + record_bytes(records_for(n, tile));
    if (kind == GBSCAN_KIND_SEGMENTED || kind == GBSCAN_KIND_SEGMENTED_MAX ||
        kind == GBSCAN_KIND_SEGMENTED_MIN)
        *bytes += seg_bitmap_bytes(n);
    return GBSCAN_OK;
}

gbscan_status gbscan_workspace_init(void* ws, size_t ws_bytes, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("gbscan_workspace_init");
    if (ws == nullptr || ws_bytes < kHeaderBytes) return GBSCAN_ERR_WORKSPACE;
    return from_cuda(cudaMemsetAsync(ws, 0, ws_bytes, stream));
}

#define GBSCAN_FLAT(NAME, TYPE, FAMILY, EXCL)                                                  \
    gbscan_status NAME(const TYPE* in, TYPE* out, int64_t n, void* ws, size_t ws_bytes,       \
                       gbscan_algo algo, int variant, cudaStream_t stream) {                  \
        GBSCAN_NVTX_RANGE(#NAME);                                                             \
        return scan_flat(FAMILY(), in, out, n, sizeof(TYPE), EXCL, ws, ws_bytes, algo, variant, \
                         stream);                                                             \
    }

GBSCAN_FLAT(scan_inclusive_i32, int32_t, family_scan_i32, 0)
GBSCAN_FLAT(scan_exclusive_i32, int32_t, family_scan_i32, 1)
GBSCAN_FLAT(scan_inclusive_i64, int64_t, family_scan_i64, 0)
GBSCAN_FLAT(scan_exclusive_i64, int64_t, family_scan_i64, 1)
GBSCAN_FLAT(scan_inclusive_u32, uint32_t, family_scan_i32, 0)
GBSCAN_FLAT(scan_exclusive_u32, uint32_t, family_scan_i32, 1)
// fp64 is bound by its adds on this part: AUTO takes the two-pass scan
#define GBSCAN_FLAT_F64(NAME, EXCL)                                                            \
    gbscan_status NAME(const double* in, double* out, int64_t n, void* ws, size_t ws_bytes,   \
                       gbscan_algo algo, int variant, cudaStream_t stream) {                  \
        GBSCAN_NVTX_RANGE(#NAME);                                                             \
        const Family& fam = family_scan_f64();                                                \
        return scan_flat(fam, in, out, n, sizeof(double), EXCL, ws, ws_bytes,                 \
                         auto_arith_bound(fam, n, algo), variant, stream);                    \
    }

GBSCAN_FLAT_F64(scan_inclusive_f64, 0)
GBSCAN_FLAT_F64(scan_exclusive_f64, 1)

static gbscan_status scan_f32_impl(const float* in, float* out, int64_t n, gbscan_f32_mode mode,
                                   int excl, void* ws, size_t ws_bytes, gbscan_algo algo,
                                   int variant, cudaStream_t stream) {
    if (mode != GBSCAN_F32_PLAIN && mode != GBSCAN_F32_COMPENSATED) return GBSCAN_ERR_INVALID_ARG;
    const Family& fam = mode == GBSCAN_F32_COMPENSATED ? family_scan_f32c() : family_scan_f32();
    return scan_flat(fam, in, out, n, sizeof(float), excl, ws, ws_bytes, algo, variant, stream);
}

gbscan_status scan_inclusive_f32(const float* in, float* out, int64_t n, gbscan_f32_mode mode,
                                 void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_inclusive_f32");
    return scan_f32_impl(in, out, n, mode, 0, ws, ws_bytes, algo, variant, stream);
}

gbscan_status scan_exclusive_f32(const float* in, float* out, int64_t n, gbscan_f32_mode mode,
                                 void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                                 cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_exclusive_f32");
    return scan_f32_impl(in, out, n, mode, 1, ws, ws_bytes, algo, variant, stream);
}

// Pieces of the host pipeline: at most 16 Mi elements (64 MiB) each.
constexpr int64_t kHostPieceElems = 16ll << 20;

gbscan_status scan_inclusive_i32_host(const int32_t* h_in, int32_t* h_out, int64_t n,
                                      int32_t* d_buf, int64_t d_elems, void* ws, size_t ws_bytes,
                                      cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_inclusive_i32_host");
    if (n < 0 || d_elems < 0) return GBSCAN_ERR_INVALID_ARG;
    if (n == 0) return GBSCAN_OK;
    if (h_in == nullptr || h_out == nullptr || d_buf == nullptr) return GBSCAN_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_buf) % 16) return GBSCAN_ERR_ALIGNMENT;
    int64_t m = n < kHostPieceElems ? n : kHostPieceElems;
    if (d_elems < n) {
        // a ring of at least two slots
        if (m > d_elems / 2) m = d_elems / 2;
        m &= ~int64_t(3);  // slots stay 16-byte aligned
        if (m < 4096) return GBSCAN_ERR_INVALID_ARG;
    }
    const int64_t P = (n + m - 1) / m;
    int64_t R = d_elems / m;
    if (R > P) R = P;
    const Family& fam = family_scan_i32();
    const Variant& v = fam.variants[1];  // the partitioned shape tuned for large int32 scans
    gbscan_status st = check_ws(ws, ws_bytes, records_for(m, v.tile));
    if (st != GBSCAN_OK) return st;
    Header* hdr = static_cast<Header*>(ws);
    cudaGetLastError();

    cudaStream_t s_cmp = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> evs;
    auto event = [&]() -> cudaEvent_t {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        evs.push_back(e);
        return e;
    };
    cudaError_t e = cudaStreamCreateWithFlags(&s_cmp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
    std::vector<cudaEvent_t> ev_cmp(P, nullptr), ev_out(P, nullptr);
    cudaEvent_t ev_start = event();
    if (e == cudaSuccess && !ev_start) e = cudaErrorMemoryAllocation;
    // the internal streams start after the work already queued on `stream`
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_cmp, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_start, 0);
    for (int64_t k = 0; k < P && e == cudaSuccess; ++k) {
        const int64_t off = k * m;
        const int64_t len = (n - off) < m ? (n - off) : m;
        int32_t* slot = d_buf + (k % R) * m;
        // upload (on `stream`) once the slot's previous piece is downloaded
        if (k >= R) e = cudaStreamWaitEvent(stream, ev_out[k - R], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slot, h_in + off, static_cast<size_t>(len) * 4, cudaMemcpyHostToDevice,
                                stream);
        cudaEvent_t ev_in = event();
        if (e == cudaSuccess && !ev_in) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaEventRecord(ev_in, stream);
        // scan in place, continuing from the pieces before it
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_cmp, ev_in, 0);
        if (e == cudaSuccess) {
            Params p = make_params(slot, slot, len, v.tile, ws, ws_bytes);
            p.chunk_tiles = partition_chunk_tiles(v, 4);
            p.chunk_lag = partition_chunk_lag();
            p.prefetch_tiles = single_pass_prefetch_tiles(v.tile, 4);
            p.carry_in = k > 0 ? &hdr->host_carry : nullptr;
            e = v.partitioned(p, s_cmp);
        }
        // its last prefix carries into the next piece
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hdr->host_carry, slot + len - 1, 4, cudaMemcpyDeviceToDevice, s_cmp);
        ev_cmp[k] = event();
        if (e == cudaSuccess && !ev_cmp[k]) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaEventRecord(ev_cmp[k], s_cmp);
        // download
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_cmp[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_out + off, slot, static_cast<size_t>(len) * 4, cudaMemcpyDeviceToHost,
                                s_out);
        ev_out[k] = event();
        if (e == cudaSuccess && !ev_out[k]) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaEventRecord(ev_out[k], s_out);
    }
    // `stream` continues once every download is done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_out[P - 1], 0);
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (s_cmp) cudaStreamDestroy(s_cmp);
    if (s_out) cudaStreamDestroy(s_out);
    return from_cuda(e);
}

gbscan_status compact_i32(const int32_t* in, const uint8_t* flags, int32_t* out, int64_t n,
                          int64_t* count, void* ws, size_t ws_bytes, int variant,
                          cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("compact_i32");
    return compact_impl(in, flags, out, n, count, ws, ws_bytes, variant, stream);
}

gbscan_status compact_f32(const float* in, const uint8_t* flags, float* out, int64_t n,
                          int64_t* count, void* ws, size_t ws_bytes, int variant,
                          cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("compact_f32");
    return compact_impl(in, flags, out, n, count, ws, ws_bytes, variant, stream);
}

gbscan_status scan_op_i32(const int32_t* in, int32_t* out, int64_t n, gbscan_op op,
                          int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo,
                          int variant, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_op_i32");
    const Family* fam = op == GBSCAN_OP_SUM ? &family_scan_i32()
                        : op == GBSCAN_OP_MAX ? &family_max_i32()
                        : op == GBSCAN_OP_MIN ? &family_min_i32()
                                              : nullptr;
    if (!fam) return GBSCAN_ERR_INVALID_ARG;
    return scan_flat(*fam, in, out, n, sizeof(int32_t), exclusive != 0, ws, ws_bytes, algo,
                     variant, stream);
}

gbscan_status scan_op_f32(const float* in, float* out, int64_t n, gbscan_op op, int exclusive,
                          void* ws, size_t ws_bytes, gbscan_algo algo, int variant,
                          cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_op_f32");
    const Family* fam = op == GBSCAN_OP_SUM ? &family_scan_f32()
                        : op == GBSCAN_OP_MAX ? &family_max_f32()
                        : op == GBSCAN_OP_MIN ? &family_min_f32()
                                              : nullptr;
    if (!fam) return GBSCAN_ERR_INVALID_ARG;
    return scan_flat(*fam, in, out, n, sizeof(float), exclusive != 0, ws, ws_bytes, algo, variant,
                     stream);
}

gbscan_status scan_op_i64(const int64_t* in, int64_t* out, int64_t n, gbscan_op op,
                          int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo,
                          int variant, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_op_i64");
    const Family* fam = op == GBSCAN_OP_SUM ? &family_scan_i64()
                        : op == GBSCAN_OP_MAX ? &family_max_i64()
                        : op == GBSCAN_OP_MIN ? &family_min_i64()
                                              : nullptr;
    if (!fam) return GBSCAN_ERR_INVALID_ARG;
    return scan_flat(*fam, in, out, n, sizeof(int64_t), exclusive != 0, ws, ws_bytes, algo,
                     variant, stream);
}

gbscan_status scan_op_u32(const uint32_t* in, uint32_t* out, int64_t n, gbscan_op op,
                          int exclusive, void* ws, size_t ws_bytes, gbscan_algo algo,
                          int variant, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_op_u32");
    const Family* fam = op == GBSCAN_OP_SUM ? &family_scan_i32()
                        : op == GBSCAN_OP_MAX ? &family_max_u32()
                        : op == GBSCAN_OP_MIN ? &family_min_u32()
                                              : nullptr;
    if (!fam) return GBSCAN_ERR_INVALID_ARG;
    return scan_flat(*fam, in, out, n, sizeof(uint32_t), exclusive != 0, ws, ws_bytes, algo,
                     variant, stream);
}

gbscan_status scan_segmented_op_i32(const int32_t* in, int32_t* out, int64_t n,
                                    const int64_t* offsets, int64_t num_segments, gbscan_op op,
                                    int exclusive, void* ws, size_t ws_bytes, int variant,
                                    cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_segmented_op_i32");
    const Family* fam = op == GBSCAN_OP_SUM ? &family_seg_i32()
                        : op == GBSCAN_OP_MAX ? &family_seg_max_i32()
                        : op == GBSCAN_OP_MIN ? &family_seg_min_i32()
                                              : nullptr;
    if (!fam) return GBSCAN_ERR_INVALID_ARG;
    return scan_seg_impl(*fam, in, out, n, offsets, num_segments, sizeof(int32_t), exclusive != 0,
                         ws, ws_bytes, variant, stream);
}

gbscan_status scan_segmented_op_f32(const float* in, float* out, int64_t n,
                                    const int64_t* offsets, int64_t num_segments, gbscan_op op,
                                    int exclusive, void* ws, size_t ws_bytes, int variant,
                                    cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_segmented_op_f32");
    const Family* fam = op == GBSCAN_OP_SUM ? &family_seg_f32()
                        : op == GBSCAN_OP_MAX ? &family_seg_max_f32()
                        : op == GBSCAN_OP_MIN ? &family_seg_min_f32()
                                              : nullptr;
    if (!fam) return GBSCAN_ERR_INVALID_ARG;
    return scan_seg_impl(*fam, in, out, n, offsets, num_segments, sizeof(float), exclusive != 0,
                         ws, ws_bytes, variant, stream);
}

gbscan_status scan_segmented_batched_i32(const int32_t* in, int32_t* out, int64_t n,
                                         const int64_t* offsets, int64_t num_segments,
                                         int exclusive, void* ws, size_t ws_bytes, int variant,
                                         cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_segmented_batched_i32");
    return scan_seg_impl(family_seg_i32(), in, out, n, offsets, num_segments, sizeof(int32_t),
                         exclusive != 0, ws, ws_bytes, variant, stream);
}

gbscan_status scan_segmented_batched_f32(const float* in, float* out, int64_t n,
                                         const int64_t* offsets, int64_t num_segments,
                                         int exclusive, void* ws, size_t ws_bytes, int variant,
                                         cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_segmented_batched_f32");
    return scan_seg_impl(family_seg_f32(), in, out, n, offsets, num_segments, sizeof(float),
                         exclusive != 0, ws, ws_bytes, variant, stream);
}

gbscan_status scan_rows_f32(const float* in, float* out, int64_t rows, int64_t cols,
                            int exclusive, void* ws, size_t ws_bytes, int variant,
                            cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_rows_f32");
    return scan_rows_impl(family_rows_f32(), in, out, rows, cols, sizeof(float), exclusive != 0,
                          ws, ws_bytes, variant, stream);
}

gbscan_status scan_rows_f64(const double* in, double* out, int64_t rows, int64_t cols,
                            int exclusive, void* ws, size_t ws_bytes, int variant,
                            cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_rows_f64");
    return scan_rows_impl(family_rows_f64(), in, out, rows, cols, sizeof(double), exclusive != 0,
                          ws, ws_bytes, variant, stream);
}

gbscan_status scan_backward_f32(const float* grad_out, float* grad_in, int64_t rows, int64_t cols,
                                int exclusive, void* ws, size_t ws_bytes, int variant,
                                cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_backward_f32");
    return scan_rows_impl(family_rows_rev_f32(), grad_out, grad_in, rows, cols, sizeof(float),
                          exclusive != 0, ws, ws_bytes, variant, stream);
}

gbscan_status scan_backward_f64(const double* grad_out, double* grad_in, int64_t rows,
                                int64_t cols, int exclusive, void* ws, size_t ws_bytes,
                                int variant, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_backward_f64");
    return scan_rows_impl(family_rows_rev_f64(), grad_out, grad_in, rows, cols, sizeof(double),
                          exclusive != 0, ws, ws_bytes, variant, stream);
}

gbscan_status scan_get_device_status(void* ws, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_get_device_status");
    if (ws == nullptr) return GBSCAN_ERR_WORKSPACE;
    Header* hdr = static_cast<Header*>(ws);
    if (cudaStreamSynchronize(stream) != cudaSuccess) return GBSCAN_ERR_CUDA;
    int32_t err = 0;
    if (cudaMemcpy(&err, &hdr->error, sizeof(err), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GBSCAN_ERR_CUDA;
    if (err != 0) {
        if (cudaMemsetAsync(&hdr->error, 0, sizeof(int32_t), stream) != cudaSuccess)
            return GBSCAN_ERR_CUDA;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return GBSCAN_ERR_CUDA;
    }
    return static_cast<gbscan_status>(err);
}

gbscan_status gbscan_set_debug(void* ws, size_t ws_bytes, uint32_t spin_limit_us,
                               int64_t drop_tile, uint32_t delay_ns_max, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("gbscan_set_debug");
    if (ws == nullptr || ws_bytes < kHeaderBytes) return GBSCAN_ERR_WORKSPACE;
    cudaGetLastError();
    set_debug_kernel<<<1, 1, 0, stream>>>(static_cast<Header*>(ws), spin_limit_us, drop_tile,
                                          delay_ns_max);
    return from_cuda(cudaGetLastError());
}

int gbscan_num_variants(gbscan_dtype dtype, gbscan_kind kind) {
    if (!valid_dtype(dtype)) return 0;
    const Family* f = family_for(dtype, kind);
    return f ? f->num_variants : 0;
}

gbscan_status gbscan_variant_info(gbscan_dtype dtype, gbscan_kind kind, int variant, int* threads,
                                  int* items, int* stages, int* tile) {
    if (!valid_dtype(dtype)) return GBSCAN_ERR_INVALID_ARG;
    const Family* f = family_for(dtype, kind);
    if (!f) return GBSCAN_ERR_UNSUPPORTED;
    if (variant < 0 || variant >= f->num_variants) return GBSCAN_ERR_INVALID_ARG;
    const Variant& v = f->variants[variant];
    if (threads) *threads = v.threads;
    if (items) *items = v.items;
    if (stages) *stages = v.stages;
    if (tile) *tile = v.tile;
    return GBSCAN_OK;
}

gbscan_status gbscan_copy(const void* src, void* dst, size_t bytes, cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("gbscan_copy");
    if (bytes == 0) return GBSCAN_OK;
    if (src == nullptr || dst == nullptr) return GBSCAN_ERR_INVALID_ARG;
    if (ranges_overlap(src, bytes, dst, bytes)) return GBSCAN_ERR_INVALID_ARG;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) || (bytes & 15))
        return GBSCAN_ERR_ALIGNMENT;
    cudaGetLastError();
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sm_count(dev);
    const int64_t n16 = static_cast<int64_t>(bytes / 16);
    int64_t blocks = static_cast<int64_t>(sms > 0 ? sms : 1) * 8;
    const int64_t need = (n16 + 255) / 256;
    if (blocks > need) blocks = need;
    copy_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        static_cast<const uint4*>(src), static_cast<uint4*>(dst), n16);
    return from_cuda(cudaGetLastError());
}

const char* gbscan_status_string(gbscan_status status) {
    switch (status) {
    case GBSCAN_OK: return "ok";
    case GBSCAN_ERR_INVALID_ARG: return "invalid argument";
    case GBSCAN_ERR_ALIGNMENT: return "misaligned pointer";
    case GBSCAN_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case GBSCAN_ERR_CUDA: return "CUDA error";
    case GBSCAN_ERR_TIMEOUT: return "bounded wait on another tile ran out";
    case GBSCAN_ERR_UNSUPPORTED: return "unsupported size or option";
    }
    return "unknown status";
}

gbscan_status gbscan_resident_max_n(gbscan_dtype dtype, gbscan_kind kind, gbscan_f32_mode mode,
                                    int64_t* n) {
    if (n == nullptr || !valid_dtype(dtype)) return GBSCAN_ERR_INVALID_ARG;
    if (mode != GBSCAN_F32_PLAIN && mode != GBSCAN_F32_COMPENSATED) return GBSCAN_ERR_INVALID_ARG;
    if (kind != GBSCAN_KIND_SCAN && kind != GBSCAN_KIND_SCAN_MAX && kind != GBSCAN_KIND_SCAN_MIN)
        return GBSCAN_ERR_UNSUPPORTED;
    const Family* f = (kind == GBSCAN_KIND_SCAN && dtype == GBSCAN_F32 && mode == GBSCAN_F32_COMPENSATED)
                          ? &family_scan_f32c()
                          : family_for(dtype, kind);
    if (f == nullptr || !f->resident) return GBSCAN_ERR_UNSUPPORTED;
    const int64_t cap = f->resident_capacity();
    if (cap <= 0) return GBSCAN_ERR_CUDA;
    *n = cap * f->resident_tile;
    return GBSCAN_OK;
}

int gbscan_abi_version(void) { return GBSCAN_ABI_VERSION; }

// The device address of the static scratch array differs per device; it is
// looked up once per device (with that device current) and cached.  In host
// code the array's name is only a host-side stand-in, never passed to a kernel.
static void* noalloc_scratch_address(int device) {
    static std::atomic<void*> cache[64];
    if (device < 0 || device >= 64) return nullptr;
    void* p = cache[device].load(std::memory_order_acquire);
    if (p) return p;
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr) {
        cudaGetLastError();
        return nullptr;
    }
    cache[device].store(addr, std::memory_order_release);
    return addr;
}

gbscan_status scan_inclusive_i32_noalloc(const int32_t* in, int32_t* out, int64_t n,
                                         cudaStream_t stream) {
    GBSCAN_NVTX_RANGE("scan_inclusive_i32_noalloc");
    if (n < 0) return GBSCAN_ERR_INVALID_ARG;
    if (n > GBSCAN_NOALLOC_MAX_N) return GBSCAN_ERR_UNSUPPORTED;
    const Family& fam = family_scan_i32();
    if (fam.variants[0].tile != kNoallocTile) return GBSCAN_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GBSCAN_ERR_CUDA;
    // the per-device address lookup, also for n == 0 (a warm-up call)
    void* ws = noalloc_scratch_address(dev);
    if (ws == nullptr) return GBSCAN_ERR_CUDA;
    if (n == 0) return GBSCAN_OK;
    // the same argument checks as the scan itself, before the shared array is
    // touched: a call that is rejected changes nothing in it
    gbscan_status st = check_io(in, out, n, sizeof(int32_t));
    if (st != GBSCAN_OK) return st;
    // Launch state that must start at zero: the tile and done counters and the
    // error word (header bytes 4..15).  The epoch (bytes 0..3) is kept: it is
    // what makes the status records of earlier calls stale.
    if (cudaMemsetAsync(static_cast<unsigned char*>(ws) + 4, 0, 12, stream) != cudaSuccess)
        return GBSCAN_ERR_CUDA;
    return scan_flat(fam, in, out, n, sizeof(int32_t), 0, ws, GBSCAN_NOALLOC_SCRATCH_BYTES,
                     GBSCAN_ALGO_SINGLE_PASS, 0, stream);
}

}  // extern "C"
