// gbscan_device.cuh — device code of the prefix-sum library (sm_103a).
//
// One templated tile kernel implements every scan in the library:
//
//   tile load    : 1-D TMA bulk copy (cp.async.bulk) of a whole tile into shared
//                  memory, completing on an mbarrier; an element-wise path covers
//                  the ragged last tile and misaligned arrays.
//   thread scan  : each thread owns ITEMS consecutive elements (the "vertical"
//                  per-lane chunk of Section 3.2) read with conflict-free 128-bit
//                  shared loads, and reduces them sequentially in registers.
//   warp scan    : Hillis-Steele log-step scan over the 32 thread totals with
//                  __shfl_up_sync (the in-register scan of Section 3.1, Listing 1,
//                  with warp lanes in place of AVX-512 lanes).
//   block scan   : warp totals through shared memory, scanned by warp 0; the last
//                  value is the tile total, broadcast like the carry vector of
//                  Section 3.1.
//   look-back    : the tile publishes its total, then warp 0 reads the status of
//                  up to 32 predecessors at a time and adds their totals until it
//                  meets a published inclusive prefix; the tile then publishes its
//                  own inclusive prefix.  This is the "synchronise only with
//                  adjacent threads" alternative to the counting barrier that
//                  Section 2.2.1 mentions (StreamScan), with the decoupled
//                  aggregate/prefix states of Merrill and Garland's single-pass
//                  scan, and it plays the role of the paper's sums array
//                  (Section 2.1, Figure 1).
//   store        : results are written back over the tile in shared memory and
//                  leave with one TMA bulk store.
//
// The same kernel, with a mode parameter, gives the two-pass comparison of the
// paper's "Accumulate + Prefix Sum" (Figure 1b): a reduce-only pass and a
// scan-with-offset pass around a one-block scan of the tile sums.
//
// Every wait is bounded (a %globaltimer deadline); a wait that runs out records
// GBSCAN_ERR_TIMEOUT in the workspace and the kernel still finishes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbscan.h"

namespace gbscan {

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------

// Header at the start of the workspace (zeroed once by the caller).
struct alignas(256) Header {
    uint32_t epoch;         // launches completed, mod 2^29; 0 only before the first
    uint32_t tile_counter;  // dynamic tile ids of the running launch (0 between launches)
    uint32_t done_counter;  // blocks that finished the running launch
    int32_t error;          // first device-side error (gbscan_status), 0 = none
    int64_t error_tile;     // tile that recorded it
    uint32_t spin_limit_us; // bound on every wait, 0 = default
    uint32_t delay_ns_max;  // race-stress sleeps before publishing, 0 = off
    int64_t drop_tile_plus1;// debug: this tile (minus one) never publishes, 0 = none
    uint32_t reserved[54];
};
static_assert(sizeof(Header) == 256, "header size");

// One record per tile.  The status word of tile i lives only in `word` of record
// i, whatever the element type, kind or size of the call, so a later call can
// never read a value written by another layout as a status word.
//   word : bits 0..31  tile value (4-byte accumulators: aggregate or inclusive prefix)
//          bits 32..33 state (0 = not ready, 1 = aggregate, 2 = inclusive prefix)
//          bit  34     the tile contains a segment head
//          bits 35..63 epoch of the launch that wrote it
//   agg, inc : 8-byte accumulators (aggregate / inclusive prefix), written before
//          the word is released.
//   aux  : two-pass tile sums, or the first segment of the tile.
struct alignas(32) TileRecord {
    unsigned long long word;
    unsigned long long agg;
    unsigned long long inc;
    unsigned long long aux;
};
static_assert(sizeof(TileRecord) == 32, "record size");

constexpr uint32_t kStateX = 0, kStateA = 1, kStateP = 2;
constexpr uint32_t kEpochBits = 29;
constexpr uint32_t kEpochMask = (1u << kEpochBits) - 1;
constexpr uint64_t kDefaultSpinLimitNs = 200ull * 1000 * 1000;  // 200 ms

enum Mode : int { kSinglePass = 0, kReduce = 1, kScanOffset = 2 };
enum Heads : int { kNoHeads = 0, kOffsetHeads = 1, kRowHeads = 2 };

struct Params {
    const void* in;
    void* out;
    int64_t n;
    int64_t num_tiles;
    Header* hdr;
    TileRecord* rec;
    int64_t rec_capacity;   // records the workspace holds
    const int64_t* offsets; // segmented: CSR offsets (num_segments + 1)
    int64_t num_segments;
    int64_t cols;           // row kinds: row length
    int exclusive;
    int fast;               // in and out are 16-byte aligned: TMA path for full tiles
};

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global -> shared bulk copy; completion is signalled on `bar` (complete_tx).
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Shared -> global bulk copy, tracked as a bulk group.
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) reads of them.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ int32_t ld_relaxed_s32(const int32_t* p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void record_error(Header* hdr, int code, int64_t tile) {
    if (atomicCAS(&hdr->error, 0, code) == 0) hdr->error_tile = tile;
}

// ---------------------------------------------------------------------------
// Operators: + over each element type, with the accumulator it is summed in.
//   combine(a, b)     : a (earlier elements) followed by b
//   accumulate(r, x)  : r = r + x for one element
//   output(c, l)      : the element value of carry c followed by local sum l
// ---------------------------------------------------------------------------

struct OpI32 {
    using T = int32_t;
    using Acc = uint32_t;  // modular: two's complement wraparound
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    __device__ static Acc identity() { return 0u; }
    __device__ static Acc lift(T x) { return static_cast<uint32_t>(x); }
    __device__ static Acc combine(Acc a, Acc b) { return a + b; }
    __device__ static void accumulate(Acc& r, T x) { r += static_cast<uint32_t>(x); }
    __device__ static T output(Acc c, Acc l) { return static_cast<T>(c + l); }
    __device__ static T output1(Acc v) { return static_cast<T>(v); }
    __device__ static Bits to_bits(Acc a) { return a; }
    __device__ static Acc from_bits(Bits b) { return b; }
};

struct OpI64 {
    using T = int64_t;
    using Acc = unsigned long long;
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    __device__ static Acc identity() { return 0ull; }
    __device__ static Acc lift(T x) { return static_cast<Acc>(x); }
    __device__ static Acc combine(Acc a, Acc b) { return a + b; }
    __device__ static void accumulate(Acc& r, T x) { r += static_cast<Acc>(x); }
    __device__ static T output(Acc c, Acc l) { return static_cast<T>(c + l); }
    __device__ static T output1(Acc v) { return static_cast<T>(v); }
    __device__ static Bits to_bits(Acc a) { return a; }
    __device__ static Acc from_bits(Bits b) { return b; }
};

struct OpF32 {
    using T = float;
    using Acc = float;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    __device__ static Acc identity() { return 0.0f; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return __fadd_rn(a, b); }
    __device__ static void accumulate(Acc& r, T x) { r = __fadd_rn(r, x); }
    __device__ static T output(Acc c, Acc l) { return __fadd_rn(c, l); }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return __float_as_uint(a); }
    __device__ static Acc from_bits(Bits b) { return __uint_as_float(b); }
};

struct OpF64 {
    using T = double;
    using Acc = double;
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    __device__ static Acc identity() { return 0.0; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return __dadd_rn(a, b); }
    __device__ static void accumulate(Acc& r, T x) { r = __dadd_rn(r, x); }
    __device__ static T output(Acc c, Acc l) { return __dadd_rn(c, l); }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return static_cast<Bits>(__double_as_longlong(a)); }
    __device__ static Acc from_bits(Bits b) { return __longlong_as_double(static_cast<long long>(b)); }
};

// Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b).  Every operation is an
// explicitly rounded add, so the compiler can neither contract nor reorder it.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float ab = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, ab), __fsub_rn(b, bb));
}

// Compensated fp32: the accumulator is an unevaluated pair hi + lo, where hi
// carries the rounded sum and lo the exact rounding errors of the additions into
// hi (rounded once more when summed).  Per-thread running sums, warp and block
// carries, and the tile prefixes passed between tiles are all pairs; each
// output is rounded once, from the pair.
struct OpF32C {
    using T = float;
    using Acc = float2;  // x = hi, y = lo
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    __device__ static Acc identity() { return make_float2(0.0f, 0.0f); }
    __device__ static Acc lift(T x) { return make_float2(x, 0.0f); }
    __device__ static Acc combine(Acc a, Acc b) {
        float s, e;
        two_sum(a.x, b.x, s, e);
        float lo = __fadd_rn(__fadd_rn(a.y, b.y), e);
        float h2, l2;
        two_sum(s, lo, h2, l2);  // renormalise so |lo| stays below half an ulp of hi
        return make_float2(h2, l2);
    }
    __device__ static void accumulate(Acc& r, T x) {
        float s, e;
        two_sum(r.x, x, s, e);
        r.x = s;
        r.y = __fadd_rn(r.y, e);
    }
    __device__ static T output(Acc c, Acc l) {
        float s, e;
        two_sum(c.x, l.x, s, e);
        return __fadd_rn(s, __fadd_rn(e, __fadd_rn(c.y, l.y)));
    }
    __device__ static T output1(Acc v) { return __fadd_rn(v.x, v.y); }
    __device__ static Bits to_bits(Acc a) {
        return (static_cast<Bits>(__float_as_uint(a.y)) << 32) | __float_as_uint(a.x);
    }
    __device__ static Acc from_bits(Bits b) {
        return make_float2(__uint_as_float(static_cast<uint32_t>(b)),
                           __uint_as_float(static_cast<uint32_t>(b >> 32)));
    }
};

template <class Op>
__device__ __forceinline__ typename Op::Acc shfl_up_acc(typename Op::Acc v, int d) {
    return Op::from_bits(__shfl_up_sync(0xffffffffu, Op::to_bits(v), d));
}
template <class Op>
__device__ __forceinline__ typename Op::Acc shfl_down_acc(typename Op::Acc v, int d) {
    return Op::from_bits(__shfl_down_sync(0xffffffffu, Op::to_bits(v), d));
}
template <class Op>
__device__ __forceinline__ typename Op::Acc shfl_idx_acc(typename Op::Acc v, int src) {
    return Op::from_bits(__shfl_sync(0xffffffffu, Op::to_bits(v), src));
}

// Segmented combine of (flag, value) pairs, a earlier than b: a segment head in
// b discards everything before it.
template <class Op>
__device__ __forceinline__ void seg_combine(bool fa, typename Op::Acc va, bool& fb,
                                            typename Op::Acc& vb) {
    if (!fb) vb = Op::combine(va, vb);
    fb = fb || fa;
}

// ---------------------------------------------------------------------------
// Tile status: publish / read
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t make_meta(uint32_t epoch, bool head, uint32_t state) {
    return (epoch << 3) | (head ? 4u : 0u) | state;
}

template <class Op>
__device__ __forceinline__ void publish(TileRecord* rec, int64_t tile, uint32_t epoch,
                                        uint32_t state, bool head, typename Op::Acc v) {
    TileRecord* r = rec + tile;
    const unsigned long long meta = make_meta(epoch, head, state);
    if constexpr (Op::kPacked) {
        st_relaxed_u64(&r->word, (meta << 32) | static_cast<unsigned long long>(Op::to_bits(v)));
    } else {
        // Value first, then the status word with release order, so that a
        // reader that acquires the word sees the value.  Aggregate and prefix
        // have separate slots: a reader that saw state A never reads a prefix.
        st_relaxed_u64(state == kStateP ? &r->inc : &r->agg,
                       static_cast<unsigned long long>(Op::to_bits(v)));
        st_release_u64(&r->word, meta << 32);
    }
}

template <class Op>
__device__ __forceinline__ void read_status(const TileRecord* rec, int64_t tile, uint32_t epoch,
                                            uint32_t& state, bool& head, typename Op::Acc& v) {
    const TileRecord* r = rec + tile;
    unsigned long long w;
    if constexpr (Op::kPacked)
        w = ld_relaxed_u64(&r->word);
    else
        w = ld_acquire_u64(&r->word);
    const uint32_t meta = static_cast<uint32_t>(w >> 32);
    if ((meta >> 3) != epoch) {
        state = kStateX;
        head = false;
        v = Op::identity();
        return;
    }
    state = meta & 3u;
    head = (meta & 4u) != 0;
    if constexpr (Op::kPacked) {
        v = Op::from_bits(static_cast<typename Op::Bits>(w & 0xffffffffull));
    } else {
        v = Op::from_bits(static_cast<typename Op::Bits>(
            ld_relaxed_u64(state == kStateP ? &r->inc : &r->agg)));
    }
}

__device__ __forceinline__ uint32_t mix32(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    return static_cast<uint32_t>(x);
}

// ---------------------------------------------------------------------------
// Shared-memory control block of the tile kernel
// ---------------------------------------------------------------------------

template <class Op, int STAGES, int NWARPS, int TILE>
struct Ctrl {
    using Acc = typename Op::Acc;
    uint64_t mbar[STAGES];
    int64_t tile_id[STAGES];
    Acc wtot_v[NWARPS];
    Acc tex_v;  // tile exclusive prefix
    uint32_t wtot_f[NWARPS];
    uint32_t tex_f;
    uint32_t epoch;
    uint32_t pad;
    uint32_t bitmap[TILE / 32 + 2];
};

template <class Op, int THREADS, int ITEMS, int STAGES, int HEADS>
constexpr int tile_smem_bytes() {
    return STAGES * THREADS * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(Ctrl<Op, STAGES, THREADS / 32, THREADS * ITEMS>));
}

// ---------------------------------------------------------------------------
// The tile kernel
// ---------------------------------------------------------------------------

template <class Op, int THREADS, int ITEMS, int STAGES, int MODE, int HEADS, bool REVERSE>
__global__ void __launch_bounds__(THREADS) tile_scan_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int NVEC = ITEMS / VEC;
    constexpr int NWARPS = THREADS / 32;
    constexpr bool DYNAMIC = (MODE == kSinglePass);
    static_assert(ITEMS % VEC == 0, "items per thread must fill 16-byte vectors");
    static_assert(ITEMS <= 32, "head flags are kept in one 32-bit mask");
    static_assert(NWARPS <= 32, "warp totals are scanned by one warp");
    static_assert(TILE_BYTES % 16 == 0, "tiles must be 16-byte multiples");
    static_assert(!(REVERSE && HEADS == kOffsetHeads), "offset segments run forward");
    using CtrlT = Ctrl<Op, STAGES, NWARPS, TILE>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * TILE_BYTES);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const T* __restrict__ in = static_cast<const T*>(p.in);
    T* out = static_cast<T*>(p.out);
    Header* hdr = p.hdr;
    const int64_t num_tiles = p.num_tiles;

    uint64_t spin_limit_ns = kDefaultSpinLimitNs;
    uint32_t delay_max = 0;
    int64_t drop_tile = -1;
    if constexpr (MODE == kSinglePass) {
        const uint32_t lim = hdr->spin_limit_us;
        if (lim) spin_limit_ns = static_cast<uint64_t>(lim) * 1000ull;
        delay_max = hdr->delay_ns_max;
        drop_tile = hdr->drop_tile_plus1 - 1;
    }

    auto claim = [&](uint32_t k) -> int64_t {
        if constexpr (DYNAMIC)
            return static_cast<int64_t>(atomicAdd(&hdr->tile_counter, 1u));
        else
            return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(k) * gridDim.x;
    };
    auto phys_of = [&](int64_t tile) -> int64_t { return REVERSE ? num_tiles - 1 - tile : tile; };
    auto count_of = [&](int64_t phys) -> int {
        const int64_t rem = p.n - phys * TILE;
        return rem < TILE ? static_cast<int>(rem) : TILE;
    };
    // Thread 0: record the k-th tile of this block in stage s and start its load.
    auto issue = [&](int s, uint32_t k) {
        const int64_t tile = claim(k);
        c.tile_id[s] = tile;
        if (tile < num_tiles) {
            const int64_t ph = phys_of(tile);
            if (p.fast && count_of(ph) == TILE) {
                T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
                mbar_arrive_expect_tx(&c.mbar[s], TILE_BYTES);
                bulk_load(buf, in + ph * TILE, TILE_BYTES, &c.mbar[s]);
            }
        }
    };

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&c.mbar[s], 1);
        fence_mbar_init();
        c.epoch = hdr->epoch;
    }
    __syncthreads();
    uint32_t epoch = (c.epoch + 1) & kEpochMask;
    if (epoch == 0) epoch = 1;
    if (tid == 0)
        for (int s = 0; s < STAGES; ++s) issue(s, static_cast<uint32_t>(s));
    __syncthreads();

    uint32_t phase = 0;      // parity of each stage's mbarrier
    int pending_refill = -1; // stage whose refill is deferred to the next iteration

    for (uint32_t k = 0;; ++k) {
        const int s = static_cast<int>(k % STAGES);
        const int64_t tile = c.tile_id[s];
        if (tile >= num_tiles) break;
        const int64_t ph = phys_of(tile);
        const int64_t tb = ph * TILE;
        const int cnt = count_of(ph);
        const bool tile_fast = p.fast && cnt == TILE;
        T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);

        // ---- a1: tile load ------------------------------------------------
        if (tile_fast) {
            const uint32_t par = (phase >> s) & 1u;
            phase ^= 1u << s;
            if (!mbar_try_wait(&c.mbar[s], par)) {
                const uint64_t t0 = global_timer_ns();
                while (!mbar_try_wait(&c.mbar[s], par)) {
                    if (global_timer_ns() - t0 > spin_limit_ns) {
                        if (tid == 0) record_error(hdr, GBSCAN_ERR_TIMEOUT, tile);
                        break;
                    }
                }
            }
        } else {
            const int off = REVERSE ? TILE - cnt : 0;
            for (int i = tid; i < cnt; i += THREADS) buf[off + i] = in[tb + i];
            __syncthreads();
        }

        // Thread t owns logical items [t*ITEMS, (t+1)*ITEMS).  Forward they sit at
        // buf[t*ITEMS + j]; reverse, logical item L sits at buf[TILE-1-L].
        T x[ITEMS];
        {
            const int base = REVERSE ? TILE - (tid + 1) * ITEMS : tid * ITEMS;
            const uint4* v4 = reinterpret_cast<const uint4*>(buf + base);
#pragma unroll
            for (int v = 0; v < NVEC; ++v) {
                const uint4 q = v4[v];
                const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
                for (int j = 0; j < VEC; ++j) {
                    if (REVERSE)
                        x[ITEMS - 1 - (v * VEC + j)] = e[j];
                    else
                        x[v * VEC + j] = e[j];
                }
            }
        }
        uint32_t valid_mask = 0xffffffffu;
        if (cnt < TILE) {
            const int first = tid * ITEMS;
            const int nvalid = cnt - first;
            valid_mask = nvalid <= 0 ? 0u : (nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u));
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (!((valid_mask >> j) & 1u)) x[j] = T(0);
        }

        // Pending TMA refill of the stage used in the previous iteration: its
        // store has had a full iteration to read shared memory.
        if (STAGES > 1 && tid == 0 && pending_refill >= 0) {
            bulk_wait_read_all();
            issue(pending_refill, k - 1 + STAGES);
            pending_refill = -1;
        }

        // ---- segment heads ----------------------------------------------
        uint32_t hm = 0;
        if constexpr (HEADS == kOffsetHeads) {
            for (int i = tid; i < TILE / 32 + 2; i += THREADS) c.bitmap[i] = 0u;
            __syncthreads();
            const int64_t s_lo = static_cast<int64_t>(p.rec[ph].aux);
            const int64_t s_hi = static_cast<int64_t>(p.rec[ph + 1].aux);
            for (int64_t sg = s_lo + tid; sg < s_hi; sg += THREADS) {
                const int64_t pos = p.offsets[sg] - tb;
                if (pos >= 0 && pos < cnt)
                    atomicOr(&c.bitmap[pos >> 5], 1u << (pos & 31));
            }
            __syncthreads();
            const int b = tid * ITEMS;
            const uint32_t w0 = c.bitmap[b >> 5], w1 = c.bitmap[(b >> 5) + 1];
            const uint32_t bits = __funnelshift_r(w0, w1, b & 31);
            hm = (ITEMS == 32 ? bits : (bits & ((1u << ITEMS) - 1u))) & valid_mask;
        } else if constexpr (HEADS == kRowHeads) {
            const int64_t cols = p.cols;
            if constexpr (!REVERSE) {
                int64_t r = (tb + static_cast<int64_t>(tid) * ITEMS) % cols;
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    if (r == 0) hm |= 1u << j;
                    r = (r + 1 == cols) ? 0 : r + 1;
                }
            } else {
                // logical L is physical tb + cnt - 1 - L; a head is a row's last element
                int64_t q = (tb + cnt - static_cast<int64_t>(tid) * ITEMS) % cols;
                if (q < 0) q += cols;
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    if (q == 0) hm |= 1u << j;
                    q = (q == 0) ? cols - 1 : q - 1;
                }
            }
            hm &= valid_mask;
        }

        // ---- a2: thread reduction -----------------------------------------
        bool tf = false;
        Acc tv = Op::identity();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (HEADS != kNoHeads && ((hm >> j) & 1u)) {
                tv = Op::lift(x[j]);
                tf = true;
            } else {
                Op::accumulate(tv, x[j]);
            }
        }

        // ---- a3: warp scan (inclusive, Hillis-Steele) ---------------------
        bool wf = tf;
        Acc wv = tv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const bool fo = __shfl_up_sync(0xffffffffu, wf ? 1 : 0, d) != 0;
            const Acc vo = shfl_up_acc<Op>(wv, d);
            if (lane >= d) {
                if (HEADS != kNoHeads)
                    seg_combine<Op>(fo, vo, wf, wv);
                else
                    wv = Op::combine(vo, wv);
            }
        }
        bool ef = __shfl_up_sync(0xffffffffu, wf ? 1 : 0, 1) != 0;
        Acc ev = shfl_up_acc<Op>(wv, 1);
        if (lane == 0) {
            ef = false;
            ev = Op::identity();
        }
        if (lane == 31) {
            c.wtot_v[warp] = wv;
            c.wtot_f[warp] = wf ? 1u : 0u;
        }
        __syncthreads();  // sync 1: warp totals

        // ---- a4/a5: block scan of warp totals, then look-back (warp 0) -----
        if (warp == 0) {
            bool bf = lane < NWARPS ? c.wtot_f[lane] != 0 : false;
            Acc bv = lane < NWARPS ? c.wtot_v[lane] : Op::identity();
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const bool fo = __shfl_up_sync(0xffffffffu, bf ? 1 : 0, d) != 0;
                const Acc vo = shfl_up_acc<Op>(bv, d);
                if (lane >= d) {
                    if (HEADS != kNoHeads)
                        seg_combine<Op>(fo, vo, bf, bv);
                    else
                        bv = Op::combine(vo, bv);
                }
            }
            // tile aggregate: inclusive value at lane NWARPS-1
            const bool agg_f = __shfl_sync(0xffffffffu, bf ? 1 : 0, NWARPS - 1) != 0;
            const Acc agg_v = shfl_idx_acc<Op>(bv, NWARPS - 1);
            // exclusive prefix of each warp within the tile
            bool xf = __shfl_up_sync(0xffffffffu, bf ? 1 : 0, 1) != 0;
            Acc xv = shfl_up_acc<Op>(bv, 1);
            if (lane == 0) {
                xf = false;
                xv = Op::identity();
            }
            if (lane < NWARPS) {
                c.wtot_v[lane] = xv;
                c.wtot_f[lane] = xf ? 1u : 0u;
            }

            bool pf = false;  // tile exclusive prefix
            Acc pv = Op::identity();
            if constexpr (MODE == kReduce) {
                if (lane == 0) p.rec[tile].aux = static_cast<unsigned long long>(Op::to_bits(agg_v));
            } else if constexpr (MODE == kScanOffset) {
                pv = Op::from_bits(static_cast<typename Op::Bits>(p.rec[tile].aux));
            } else {
                const bool dropped = (tile == drop_tile);
                const uint32_t dly = delay_max ? mix32(static_cast<uint64_t>(tile) * 0x9e3779b97f4a7c15ull) % (delay_max + 1) : 0u;
                if (tile == 0) {
                    if (lane == 0 && !dropped) {
                        if (dly) __nanosleep(dly);
                        publish<Op>(p.rec, tile, epoch, kStateP, agg_f, agg_v);
                    }
                } else {
                    if (lane == 0 && !dropped) {
                        if (dly) __nanosleep(dly);
                        publish<Op>(p.rec, tile, epoch, kStateA, agg_f, agg_v);
                    }
                    int64_t base = tile - 1;
                    uint64_t t0 = 0;
                    bool gave_up = false;
                    while (true) {
                        const int64_t idx = base - lane;
                        uint32_t st;
                        bool hf;
                        Acc hv;
                        uint32_t need, stop;
                        uint32_t ns = 32;
                        while (true) {
                            if (idx >= 0) {
                                read_status<Op>(p.rec, idx, epoch, st, hf, hv);
                            } else {
                                st = kStateP;  // before the first tile: the identity
                                hf = false;
                                hv = Op::identity();
                            }
                            const uint32_t valid = __ballot_sync(0xffffffffu, st != kStateX);
                            stop = __ballot_sync(0xffffffffu,
                                                 st == kStateP || (st == kStateA && hf));
                            need = stop ? (((stop & (0u - stop)) << 1) - 1u) : 0xffffffffu;
                            if ((valid & need) == need) break;
                            // bounded wait: give up after the spin limit or once
                            // another tile has recorded an error
                            int quit = 0;
                            if (lane == 0) {
                                const uint64_t now = global_timer_ns();
                                if (t0 == 0) t0 = now;
                                if (now - t0 > spin_limit_ns) {
                                    record_error(hdr, GBSCAN_ERR_TIMEOUT, tile);
                                    quit = 1;
                                } else if (ld_relaxed_s32(&hdr->error) != 0) {
                                    quit = 1;
                                }
                            }
                            if (__shfl_sync(0xffffffffu, quit, 0)) {
                                gave_up = true;
                                break;
                            }
                            __nanosleep(ns);
                            ns = ns < 512 ? ns * 2 : 512;
                        }
                        if (gave_up) break;
                        // fold lanes need..0 in tile order (higher lane = earlier tile)
                        bool rf = ((need >> lane) & 1u) ? hf : false;
                        Acc rv = ((need >> lane) & 1u) ? hv : Op::identity();
#pragma unroll
                        for (int d = 1; d < 32; d <<= 1) {
                            const bool fo = __shfl_down_sync(0xffffffffu, rf ? 1 : 0, d) != 0;
                            const Acc vo = shfl_down_acc<Op>(rv, d);
                            if (lane + d < 32) {
                                if (HEADS != kNoHeads)
                                    seg_combine<Op>(fo, vo, rf, rv);
                                else
                                    rv = Op::combine(vo, rv);
                            }
                        }
                        const bool wf0 = __shfl_sync(0xffffffffu, rf ? 1 : 0, 0) != 0;
                        const Acc wv0 = shfl_idx_acc<Op>(rv, 0);
                        if (HEADS != kNoHeads)
                            seg_combine<Op>(wf0, wv0, pf, pv);
                        else
                            pv = Op::combine(wv0, pv);
                        if (stop) break;
                        base -= 32;
                    }
                    bool incf = agg_f;
                    Acc incv = agg_v;
                    if (HEADS != kNoHeads)
                        seg_combine<Op>(pf, pv, incf, incv);
                    else
                        incv = Op::combine(pv, incv);
                    if (lane == 0 && !dropped) {
                        if (dly) __nanosleep(dly);
                        publish<Op>(p.rec, tile, epoch, kStateP, incf, incv);
                    }
                }
            }
            if (lane == 0) {
                c.tex_v = pv;
                c.tex_f = pf ? 1u : 0u;
            }
        }
        __syncthreads();  // sync 2: tile prefix and warp prefixes ready

        if constexpr (MODE == kReduce) {
            // every thread read its items before sync 1: the stage is free
            if (tid == 0) issue(s, k + STAGES);
            if (STAGES == 1) __syncthreads();
            continue;
        }

        // ---- a6: carry add, outputs into shared memory -----------------------
        bool cf = c.wtot_f[warp] != 0;  // warp's prefix within the tile
        Acc cv = c.wtot_v[warp];
        {
            if (HEADS != kNoHeads)
                seg_combine<Op>(cf, cv, ef, ev);
            else
                ev = Op::combine(cv, ev);
            // ev/ef: thread exclusive prefix within the tile
            bool gf = ef;
            Acc gv = ev;
            const bool tf2 = c.tex_f != 0;
            const Acc tv2 = c.tex_v;
            if (HEADS != kNoHeads)
                seg_combine<Op>(tf2, tv2, gf, gv);
            else
                gv = Op::combine(tv2, gv);
            // (gf, gv): everything before this thread's first item.  A local
            // head (rf) makes later items independent of it.
            bool rf = false;
            Acc rv = Op::identity();
            const bool excl = p.exclusive != 0;
            T y[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool h = HEADS != kNoHeads && ((hm >> j) & 1u);
                if (excl) {
                    if (h)
                        y[j] = T(0);
                    else if (rf)
                        y[j] = Op::output1(rv);
                    else
                        y[j] = Op::output(gv, rv);
                }
                if (h) {
                    rv = Op::lift(x[j]);
                    rf = true;
                } else {
                    Op::accumulate(rv, x[j]);
                }
                if (!excl) y[j] = rf ? Op::output1(rv) : Op::output(gv, rv);
            }
            const int base = REVERSE ? TILE - (tid + 1) * ITEMS : tid * ITEMS;
            uint4* v4 = reinterpret_cast<uint4*>(buf + base);
#pragma unroll
            for (int v = 0; v < NVEC; ++v) {
                uint4 q;
                T* e = reinterpret_cast<T*>(&q);
#pragma unroll
                for (int j = 0; j < VEC; ++j) e[j] = REVERSE ? y[ITEMS - 1 - (v * VEC + j)] : y[v * VEC + j];
                v4[v] = q;
            }
        }
        if (tile_fast) fence_proxy_async_smem();
        __syncthreads();  // sync 3: outputs in shared memory

        if (tile_fast) {
            if (tid == 0) {
                bulk_store(out + tb, buf, TILE_BYTES);
                bulk_commit();
            }
        } else {
            const int off = REVERSE ? TILE - cnt : 0;
            for (int i = tid; i < cnt; i += THREADS) out[tb + i] = buf[off + i];
            __syncthreads();
        }
        if (STAGES == 1) {
            if (tid == 0) {
                if (tile_fast) bulk_wait_read_all();
                issue(s, k + 1);
            }
            __syncthreads();
        } else {
            pending_refill = s;  // thread 0 refills it next iteration
        }
    }

    // ---- block exit: the last block to finish resets the launch state -----
    if (tid == 0) {
        bulk_wait_all();
        c.pad = 0u;
        if constexpr (MODE == kSinglePass) {
            __threadfence();
            const uint32_t prev = atomicAdd(&hdr->done_counter, 1u);
            if (prev == gridDim.x - 1) {
                __threadfence();
                hdr->tile_counter = 0;
                hdr->done_counter = 0;
                // The next launch tags its words with epoch + 1.  Before the tag
                // wraps, clear every status word so that no word written 2^29
                // launches ago can pass for a current one.
                const bool wrap = (epoch == kEpochMask);
                hdr->epoch = wrap ? 0u : epoch;
                c.pad = wrap ? 1u : 0u;
            }
        }
    }
    if constexpr (MODE == kSinglePass) {
        __syncthreads();
        if (c.pad) {
            for (int64_t i = tid; i < p.rec_capacity; i += THREADS) p.rec[i].word = 0ull;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Two-pass helper: exclusive scan of the tile sums (record aux fields), one block.
// ---------------------------------------------------------------------------

template <class Op, int THREADS>
__global__ void __launch_bounds__(THREADS) scan_tile_sums_kernel(TileRecord* rec, int64_t num_tiles) {
    using Acc = typename Op::Acc;
    constexpr int NWARPS = THREADS / 32;
    __shared__ Acc wsum[NWARPS];
    __shared__ Acc carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Acc carry = Op::identity();
    for (int64_t base = 0; base < num_tiles; base += THREADS) {
        const int64_t i = base + tid;
        Acc v = i < num_tiles ? Op::from_bits(static_cast<typename Op::Bits>(rec[i].aux))
                              : Op::identity();
        Acc inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Acc o = shfl_up_acc<Op>(inc, d);
            if (lane >= d) inc = Op::combine(o, inc);
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            Acc w = lane < NWARPS ? wsum[lane] : Op::identity();
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Acc o = shfl_up_acc<Op>(w, d);
                if (lane >= d) w = Op::combine(o, w);
            }
            Acc wx = shfl_up_acc<Op>(w, 1);
            if (lane == 0) wx = Op::identity();
            if (lane < NWARPS) wsum[lane] = wx;
            const Acc total = shfl_idx_acc<Op>(w, NWARPS - 1);
            if (lane == 0) carry_s = Op::combine(carry, total);
        }
        __syncthreads();
        Acc ex = shfl_up_acc<Op>(inc, 1);
        if (lane == 0) ex = Op::identity();
        ex = Op::combine(wsum[warp], ex);
        ex = Op::combine(carry, ex);
        if (i < num_tiles) rec[i].aux = static_cast<unsigned long long>(Op::to_bits(ex));
        carry = carry_s;
        __syncthreads();
    }
}

}  // namespace gbscan
