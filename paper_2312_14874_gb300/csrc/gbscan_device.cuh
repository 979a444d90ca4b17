// gbscan_device.cuh — shared device definitions of the prefix-sum library
// (sm_103a): the workspace layout (header, tile records, epoch-tagged status
// words and pairs), the PTX helpers (mbarriers, 1-D TMA bulk copies, L2
// policies, polling loads, relaxed stores), the operators (+ over int32,
// int64, fp32, fp64 and compensated fp32 pairs; running maximum and minimum),
// status publication and reading, and the two-level decoupled look-back:
//
//   look-back : a tile publishes its aggregate, then one warp reads the status
//               of its predecessors and folds their values until it meets a
//               published inclusive prefix, in two levels (the tiles of its
//               16-tile group, then group words); the tile then publishes its
//               own inclusive prefix.  This is the adjacent-only
//               synchronisation that Section 2.2.1 offers in place of a
//               counting barrier (citing StreamScan), with the decoupled
//               aggregate / prefix states of Merrill and Garland's single-pass
//               scan, and it plays the role of the paper's sums array
//               (Section 2.1, Figure 1).
//
// The kernels are in lookback.cuh (single-pass chained scan), kernels.cuh
// (two-pass comparison, and the warp-specialised chained kernel used by the
// segmented and long-row scans), partitioned.cuh (the cache-partitioned scan,
// Section 2.2), rows.cuh (row scans and their backward) and compact.cuh
// (stream compaction).
//
// Every wait is bounded (a %globaltimer deadline); a wait that runs out records
// GBSCAN_ERR_TIMEOUT in the workspace, aborts the launch, and the kernel still
// finishes.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>
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
    uint32_t abort_epoch;   // epoch of a launch in which a bounded wait ran out
    uint32_t reserved0;
    int64_t host_carry;     // host pipeline: the inclusive total of the pieces scanned so far
    uint32_t reserved[50];
};
static_assert(sizeof(Header) == 256, "header size");

// Tile records, 16 tiles to a 512-byte block (block b = tile / 16, also the
// tile's group; slot = tile % 16):
//   words  0..31  tile status words: with 4-byte accumulators the word of a
//                 tile is word `slot` (words 16..31 unused); with 8-byte
//                 accumulators a tile has the pair of words 2 slot, 2 slot + 1
//   words 32..47  aux[slot]: two-pass tile sums, or the first segment of the tile
//   words 48, 49  the group's status pair (the block's 16 tiles)
//   words 50..53  partitioned scan: chunk prefixes E and P (see rec_chunk)
//   words 54..63  unused
// A status word holds
//   bits 0..31  the value (4-byte accumulators), or one 32-bit half of an
//               8-byte accumulator (first word: bits 0..31, second: 32..63)
//   bits 32..33 state (0 = not ready, 1 = aggregate, 2 = inclusive prefix)
//   bit  34     the tile (or group) contains a segment head
//   bits 35..63 epoch of the launch that wrote it
// Every pair starts on a 16-byte boundary and moves with one 16-byte access.
// Each half is single-copy atomic on its own, so a reader takes a pair only
// when both words carry the same bits 32..63, which identifies one
// publication (each state is published once per launch).  Status words live
// only in words 0..31 and 48..53 of a block, whatever the element type, kind or
// size of a call, and nothing else is written there, so no call can read
// another call's data as a status word (a word another layout left behind
// carries an older epoch).  Sixteen 4-byte-accumulator tile words, or eight
// pairs, share one 128-byte line.
constexpr int kGroup = 16;                 // tiles per group (and per block)
constexpr int kRecBlockWords = 64;         // u64 words per block
constexpr int kRecBlockBytes = kRecBlockWords * 8;

template <class Op>
__device__ __forceinline__ unsigned long long* rec_tile(unsigned long long* rec, int64_t t) {
    return rec + (t >> 4) * kRecBlockWords + (Op::kPacked ? (t & 15) : 2 * (t & 15));
}
__device__ __forceinline__ unsigned long long* rec_aux(unsigned long long* rec, int64_t t) {
    return rec + (t >> 4) * kRecBlockWords + 32 + (t & 15);
}
// Partitioned scan: chunk c keeps two status pairs in the spare words of
// block c: its exclusive prefix E (words 50, 51: w = 0) and inclusive prefix P
// (words 52, 53: w = 2).  A chunk has at least 16 tiles, so block c always
// exists.
__device__ __forceinline__ unsigned long long* rec_chunk(unsigned long long* rec, int64_t c, int w) {
    return rec + c * kRecBlockWords + 50 + w;
}
__device__ __forceinline__ unsigned long long* rec_group(unsigned long long* rec, int64_t g) {
    return rec + g * kRecBlockWords + 48;
}

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
    unsigned long long* rec; // tile records (blocks of 16, see above)
    int64_t rec_capacity;    // tiles the workspace holds records for
    const int64_t* offsets; // segmented: CSR offsets (num_segments + 1)
    const uint32_t* bitmap; // segmented, partitioned: head bitmap (bit i: element i starts a segment)
    int64_t num_segments;
    int64_t cols;           // row kinds: row length
    int64_t chunk_tiles;    // partitioned scan: tiles per chunk
    int64_t chunk_lag;      // partitioned scan: chunk c is scanned beside the reduction of c + lag
    const uint8_t* flags;   // compaction: keep flags (nonzero = keep)
    unsigned long long* total_out; // compaction: the number kept (the last chunk prefix), or null
    const void* carry_in;   // partitioned scan: one element (device) folded in before element 0, or null
    int64_t prefetch_tiles; // single-pass scan: the loader asks L2 for the tile this far ahead of
                            // each claim (0: no prefetch)
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

// Non-blocking test of the same phase condition: never suspends the thread.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, but the thread may be suspended in hardware for up to
// `hint_ns` while the phase is incomplete; it resumes as soon as the phase
// completes.  Waiting threads then do not keep the shared-memory pipe busy.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity,
                                                    uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
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

// L2 eviction-priority policies for the bulk copies: keep (data that will be
// read again soon) or drop first (data read or written for the last time).
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Asks L2 to fetch `bytes` bytes at `src` (16-byte aligned, a multiple of 16
// bytes); nothing waits for it.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load_hint(void* dst_smem, const void* src, uint32_t bytes,
                                               uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void bulk_store_hint(void* dst, const void* src_smem, uint32_t bytes,
                                                uint64_t policy) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(smem_addr(src_smem)), "r"(bytes), "l"(policy)
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

// Status-word poll: a plain 64-bit load served by L2, the point of coherence
// (.cg: not cached in L1, so every poll sees the latest value L2 holds).
// Unlike a .relaxed/.acquire load, consecutive .cg loads of one thread are
// pipelined, so a lane can read several status words in one round trip.  An
// aligned 8-byte word is read whole; a word that is stale or not yet written
// fails the epoch check and is read again on the next poll, and every poll
// round ends with a fence so that no re-read can be merged away.
__device__ __forceinline__ unsigned long long ld_poll_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

// Both words of a status pair in one 16-byte access (see ld_poll_u64).
__device__ __forceinline__ void ld_poll_pair(const unsigned long long* p, unsigned long long& a,
                                             unsigned long long& b) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}

__device__ __forceinline__ void st_relaxed_pair(unsigned long long* p, unsigned long long a,
                                                unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void poll_round_fence() {
    asm volatile("fence.acq_rel.cta;" ::: "memory");
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

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Set in the claim counter by an abort: every later claim of the launch
// returns at least 2^31, past any tile or item count (all below 2^31), so that
// no block takes new work.  The last block to finish resets the counter.
constexpr uint32_t kClaimPoison = 0x80000000u;

// A bounded wait ran out in the launch tagged `epoch`: record the error (kept
// until scan_get_device_status reads it), mark the launch aborted, so that its
// other waits give up at once instead of each running into the bound, and
// poison the claim counter, so that the blocks finish the items they hold and
// claim no more.  The mark names the launch, so later launches are not
// affected.
__device__ __forceinline__ void record_timeout(Header* hdr, uint32_t epoch, int64_t tile) {
    record_error(hdr, GBSCAN_ERR_TIMEOUT, tile);
    atomicExch(&hdr->abort_epoch, epoch);
    atomicOr(&hdr->tile_counter, kClaimPoison);
}

__device__ __forceinline__ bool launch_aborted(const Header* hdr, uint32_t epoch) {
    return ld_relaxed_u32(&hdr->abort_epoch) == epoch;
}

// ---------------------------------------------------------------------------
// Operators: + over each element type, with the accumulator it is summed in.
//   combine(a, b)     : a (earlier elements) followed by b
//   accumulate(r, x)  : r = r + x for one element
//   output(c, l)      : the element value of carry c followed by local sum l
// ---------------------------------------------------------------------------

struct OpI32 {
    using T = int32_t;
    __device__ static T pad() { return T(0); }  // neutral element value
    using Acc = uint32_t;  // modular: two's complement wraparound
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
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
    __device__ static T pad() { return T(0); }  // neutral element value
    using Acc = unsigned long long;
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
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
    __device__ static T pad() { return T(0.0f); }  // neutral element value
    using Acc = float;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
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
    __device__ static T pad() { return T(0.0); }  // neutral element value
    using Acc = double;
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
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

// Running maximum and minimum (the scan of any associative operator, of which
// Section 1 takes +; identities -inf / +inf and INT32_MIN / INT32_MAX).  The
// fp32 versions follow IEEE maxNum / minNum (fmaxf / fminf): a NaN operand
// yields the other operand.
struct OpMaxI32 {
    using T = int32_t;
    using Acc = int32_t;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return INT32_MIN; }
    __device__ static Acc identity() { return INT32_MIN; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return a > b ? a : b; }
    __device__ static void accumulate(Acc& r, T x) { r = r > x ? r : x; }
    __device__ static T output(Acc c, Acc l) { return c > l ? c : l; }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return static_cast<uint32_t>(a); }
    __device__ static Acc from_bits(Bits b) { return static_cast<int32_t>(b); }
};

struct OpMinI32 {
    using T = int32_t;
    using Acc = int32_t;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return INT32_MAX; }
    __device__ static Acc identity() { return INT32_MAX; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return a < b ? a : b; }
    __device__ static void accumulate(Acc& r, T x) { r = r < x ? r : x; }
    __device__ static T output(Acc c, Acc l) { return c < l ? c : l; }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return static_cast<uint32_t>(a); }
    __device__ static Acc from_bits(Bits b) { return static_cast<int32_t>(b); }
};

struct OpMaxF32 {
    using T = float;
    using Acc = float;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return -__int_as_float(0x7f800000); }
    __device__ static Acc identity() { return -__int_as_float(0x7f800000); }
    // a run (or a segment) starts from the identity: a NaN first element is skipped
    __device__ static Acc lift(T x) { return fmaxf(identity(), x); }
    __device__ static Acc combine(Acc a, Acc b) { return fmaxf(a, b); }
    __device__ static void accumulate(Acc& r, T x) { r = fmaxf(r, x); }
    __device__ static T output(Acc c, Acc l) { return fmaxf(c, l); }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return __float_as_uint(a); }
    __device__ static Acc from_bits(Bits b) { return __uint_as_float(b); }
};

struct OpMinF32 {
    using T = float;
    using Acc = float;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return __int_as_float(0x7f800000); }
    __device__ static Acc identity() { return __int_as_float(0x7f800000); }
    // a run (or a segment) starts from the identity: a NaN first element is skipped
    __device__ static Acc lift(T x) { return fminf(identity(), x); }
    __device__ static Acc combine(Acc a, Acc b) { return fminf(a, b); }
    __device__ static void accumulate(Acc& r, T x) { r = fminf(r, x); }
    __device__ static T output(Acc c, Acc l) { return fminf(c, l); }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return __float_as_uint(a); }
    __device__ static Acc from_bits(Bits b) { return __uint_as_float(b); }
};

// Running maximum and minimum of int64 (identities INT64_MIN / INT64_MAX) and
// of uint32 (unsigned order; identities 0 / UINT32_MAX).
struct OpMaxI64 {
    using T = int64_t;
    using Acc = long long;
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return INT64_MIN; }
    __device__ static Acc identity() { return INT64_MIN; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return a > b ? a : b; }
    __device__ static void accumulate(Acc& r, T x) { r = r > x ? r : x; }
    __device__ static T output(Acc c, Acc l) { return c > l ? c : l; }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return static_cast<Bits>(a); }
    __device__ static Acc from_bits(Bits b) { return static_cast<Acc>(b); }
};

struct OpMinI64 {
    using T = int64_t;
    using Acc = long long;
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return INT64_MAX; }
    __device__ static Acc identity() { return INT64_MAX; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return a < b ? a : b; }
    __device__ static void accumulate(Acc& r, T x) { r = r < x ? r : x; }
    __device__ static T output(Acc c, Acc l) { return c < l ? c : l; }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return static_cast<Bits>(a); }
    __device__ static Acc from_bits(Bits b) { return static_cast<Acc>(b); }
};

struct OpMaxU32 {
    using T = uint32_t;
    using Acc = uint32_t;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return 0u; }
    __device__ static Acc identity() { return 0u; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return a > b ? a : b; }
    __device__ static void accumulate(Acc& r, T x) { r = r > x ? r : x; }
    __device__ static T output(Acc c, Acc l) { return c > l ? c : l; }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return a; }
    __device__ static Acc from_bits(Bits b) { return b; }
};

struct OpMinU32 {
    using T = uint32_t;
    using Acc = uint32_t;
    using Bits = uint32_t;
    static constexpr bool kPacked = true;
    static constexpr int kSplit = 1;  // independent chains a thread sums its items in
    __device__ static T pad() { return 0xffffffffu; }
    __device__ static Acc identity() { return 0xffffffffu; }
    __device__ static Acc lift(T x) { return x; }
    __device__ static Acc combine(Acc a, Acc b) { return a < b ? a : b; }
    __device__ static void accumulate(Acc& r, T x) { r = r < x ? r : x; }
    __device__ static T output(Acc c, Acc l) { return c < l ? c : l; }
    __device__ static T output1(Acc v) { return v; }
    __device__ static Bits to_bits(Acc a) { return a; }
    __device__ static Acc from_bits(Bits b) { return b; }
};

// Compensated fp32.  Every carry is an unevaluated pair hi + lo combined with
// Knuth's TwoSum and renormalised: the sub-block, thread, warp, block, tile and
// chunk prefixes, so no error accumulates along the array beyond O(u^2) per
// combination.  Below them, a thread sums runs of at most seven of its own
// elements (a sub-block, see kSplit; a 16-byte vector) in plain fp32
// (`accumulate` leaves lo untouched), and each output is c.hi + ((l + c.lo)),
// rounded twice.  With u = 2^-24 the error of an output is then at most about
// (6 + 6 + 3) u = 9e-7 of sum |a_i| up to it (runs of <= 7 elements inside a
// thread and inside the tile sums, two output roundings), within the 1e-6
// bound, while a thread does TwoSum work only once per run instead of once per
// element (measured: 3.8x the instructions of plain fp32 when every element
// went through TwoSum).
struct OpF32C {
    using T = float;
    __device__ static T pad() { return 0.0f; }  // neutral element value
    using Acc = float2;  // x = hi, y = lo
    using Bits = unsigned long long;
    static constexpr bool kPacked = false;
    static constexpr int kSplit = 4;  // independent chains a thread sums its items in
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
    // short chains inside a tile: the exact error of the hi sum joins lo, and
    // the pair is not renormalised (after the at most few tens of combines of
    // a tile's warp and block scans, |lo| stays within a few ulps of hi, and
    // lo's own rounding is of order eps^2 |hi|)
    __device__ static Acc combine_local(Acc a, Acc b) {
        float s, e;
        two_sum(a.x, b.x, s, e);
        return make_float2(s, __fadd_rn(__fadd_rn(a.y, b.y), e));
    }
    // a thread-local run of outputs: it starts from the carry's lo (run_init)
    // and sums its elements in plain fp32 on hi, and each output is the
    // carry's hi plus the run: one add per element, as in the plain scan
    __device__ static Acc run_init(Acc c) { return make_float2(c.y, 0.0f); }
    __device__ static void accumulate(Acc& r, T x) { r.x = __fadd_rn(r.x, x); }
    __device__ static T output(Acc c, Acc l) { return __fadd_rn(c.x, l.x); }
    __device__ static T output1(Acc v) { return __fadd_rn(v.x, v.y); }
    // in-tile sums of at most a warp row of 16-byte vectors (32 x 4 elements)
    // run in plain fp32 and join the pairs exactly (lift): a row result is at
    // most seven roundings deep (two in a vector, five across the row)
    __device__ static T row_add(T a, T b) { return __fadd_rn(a, b); }
    __device__ static Bits to_bits(Acc a) {
        return (static_cast<Bits>(__float_as_uint(a.y)) << 32) | __float_as_uint(a.x);
    }
    __device__ static Acc from_bits(Bits b) {
        return make_float2(__uint_as_float(static_cast<uint32_t>(b)),
                           __uint_as_float(static_cast<uint32_t>(b >> 32)));
    }
};

// The combine for the short dependent chains inside a tile (a thread's
// sub-block sums and carries, warp scans, block carries): the operator's own
// combine, unless the operator has a cheaper form for short chains
// (compensated pairs: one TwoSum and no renormalisation).  Long chains (tile
// and chunk prefixes, look-back folds, the scan of the tile sums across
// blocks) keep the full combine.
template <class Op, class = void>
struct HasLocalCombine : std::false_type {};
template <class Op>
struct HasLocalCombine<Op, std::void_t<decltype(Op::combine_local(std::declval<typename Op::Acc>(),
                                                                  std::declval<typename Op::Acc>()))>>
    : std::true_type {};

template <class Op>
__device__ __forceinline__ typename Op::Acc combine_local(typename Op::Acc a, typename Op::Acc b) {
    if constexpr (HasLocalCombine<Op>::value)
        return Op::combine_local(a, b);
    else
        return Op::combine(a, b);
}

// The accumulator a thread's run of outputs starts from, given the carry c
// into the run (everything before the run's first element): the identity,
// unless the operator folds part of the carry into the run (compensated
// pairs: c's lo, so that an output is c's hi plus the run).  Every
// output(c, r) takes r from run_init(c) followed by accumulate steps.
template <class Op, class = void>
struct HasRunInit : std::false_type {};
template <class Op>
struct HasRunInit<Op, std::void_t<decltype(Op::run_init(std::declval<typename Op::Acc>()))>>
    : std::true_type {};

template <class Op>
__device__ __forceinline__ typename Op::Acc run_init(typename Op::Acc c) {
    if constexpr (HasRunInit<Op>::value)
        return Op::run_init(c);
    else
        return Op::identity();
}

// Whether short in-tile sums (a warp row of vectors, a group of a lane's
// vectors) run in the element type (Op::row_add) and are lifted to the
// accumulator afterwards: compensated pairs, for which such sums are short
// enough for plain fp32.
template <class Op, class = void>
struct HasPlainRow : std::false_type {};
template <class Op>
struct HasPlainRow<Op, std::void_t<decltype(Op::row_add(std::declval<typename Op::T>(),
                                                         std::declval<typename Op::T>()))>>
    : std::true_type {};

template <class Op>
__device__ __forceinline__ typename Op::Acc shfl_up_acc(typename Op::Acc v, int d) {
    return Op::from_bits(__shfl_up_sync(0xffffffffu, Op::to_bits(v), d));
}
template <class Op>
__device__ __forceinline__ typename Op::Acc shfl_down_acc(typename Op::Acc v, int d) {
    return Op::from_bits(__shfl_down_sync(0xffffffffu, Op::to_bits(v), d));
}
template <class Op>
__device__ __forceinline__ typename Op::Acc shfl_xor_acc(typename Op::Acc v, int m) {
    return Op::from_bits(__shfl_xor_sync(0xffffffffu, Op::to_bits(v), m));
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

// Publishes (state, head, v) into the status word (4-byte accumulators) or
// pair (8-byte accumulators) at w.
template <class Op>
__device__ __forceinline__ void publish_words(unsigned long long* w, uint32_t epoch, uint32_t state,
                                              bool head, typename Op::Acc v) {
    const unsigned long long meta = static_cast<unsigned long long>(make_meta(epoch, head, state)) << 32;
    const unsigned long long bits = static_cast<unsigned long long>(Op::to_bits(v));
    if constexpr (Op::kPacked) {
        st_relaxed_u64(w, meta | bits);
    } else {
        // each half travels in its own 64-bit word together with the same
        // status meta; a reader accepts the pair only when both metas agree
        st_relaxed_pair(w, meta | (bits & 0xffffffffull), meta | (bits >> 32));
    }
}

// Decodes a status word pair already in registers (see read_words).
template <class Op>
__device__ __forceinline__ void parse_words(unsigned long long w0, unsigned long long w1,
                                            uint32_t epoch, uint32_t& state, bool& head,
                                            typename Op::Acc& v) {
    const uint32_t meta = static_cast<uint32_t>(w0 >> 32);
    bool ok = (meta >> 3) == epoch;
    if constexpr (!Op::kPacked) ok = ok && static_cast<uint32_t>(w1 >> 32) == meta;
    if (!ok) {
        state = kStateX;
        head = false;
        v = Op::identity();
        return;
    }
    state = meta & 3u;
    head = (meta & 4u) != 0;
    if constexpr (Op::kPacked)
        v = Op::from_bits(static_cast<typename Op::Bits>(w0 & 0xffffffffull));
    else
        v = Op::from_bits(static_cast<typename Op::Bits>((w1 << 32) | (w0 & 0xffffffffull)));
}

// Polls the status word or pair at w: state X when it is not a publication of
// this launch (stale epoch, or halves from two publications).
template <class Op>
__device__ __forceinline__ void read_words(const unsigned long long* w, uint32_t epoch, uint32_t& state,
                                           bool& head, typename Op::Acc& v) {
    unsigned long long w0, w1 = 0;
    if constexpr (Op::kPacked)
        w0 = ld_poll_u64(w);
    else
        ld_poll_pair(w, w0, w1);
    parse_words<Op>(w0, w1, epoch, state, head, v);
}

template <class Op>
__device__ __forceinline__ void publish(unsigned long long* rec, int64_t tile, uint32_t epoch,
                                        uint32_t state, bool head, typename Op::Acc v) {
    publish_words<Op>(rec_tile<Op>(rec, tile), epoch, state, head, v);
}

template <class Op>
__device__ __forceinline__ void publish_group(unsigned long long* rec, int64_t g, uint32_t epoch,
                                              uint32_t state, bool head, typename Op::Acc v) {
    publish_words<Op>(rec_group(rec, g), epoch, state, head, v);
}

__device__ __forceinline__ uint32_t mix32(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    return static_cast<uint32_t>(x);
}

// ---------------------------------------------------------------------------
// Decoupled look-back (all 32 lanes of one warp)
// ---------------------------------------------------------------------------

// Launch-wide knobs read from the workspace header.
struct LookbackCfg {
    uint64_t spin_limit_ns;
    uint32_t delay_max;
    int64_t drop_tile;
};

__device__ __forceinline__ LookbackCfg read_lookback_cfg(const Header* hdr) {
    LookbackCfg c;
    const uint32_t lim = hdr->spin_limit_us;
    c.spin_limit_ns = lim ? static_cast<uint64_t>(lim) * 1000ull : kDefaultSpinLimitNs;
    c.delay_max = hdr->delay_ns_max;
    c.drop_tile = hdr->drop_tile_plus1 - 1;
    return c;
}

// Publishes a tile's aggregate (agg_f, agg_v): state A, or for tile 0, whose
// inclusive prefix is its aggregate, state P.  Lane 0 only.
template <class Op>
__device__ __forceinline__ void publish_aggregate(unsigned long long* rec, int64_t tile,
                                                  uint32_t epoch, const LookbackCfg& cfg,
                                                  bool agg_f, typename Op::Acc agg_v) {
    if (tile == cfg.drop_tile) return;
    if (cfg.delay_max) {
        const uint32_t dly =
            mix32(static_cast<uint64_t>(tile) * 0x9e3779b97f4a7c15ull) % (cfg.delay_max + 1);
        if (dly) __nanosleep(dly);
    }
    publish<Op>(rec, tile, epoch, tile == 0 ? kStateP : kStateA, agg_f, agg_v);
}

// One backward walk of the decoupled look-back over status entries
// base, base-1, ... (tiles or groups; `group` selects which words are read).
// Each round, lane l reads the LB consecutive entries at distances
// l*LB .. l*LB+LB-1 back from the round's start; the walk stops at the nearest
// entry that ends it: an inclusive prefix, or an aggregate that contains a
// segment head.  Entries below `floor` end the walk as the identity.  All
// entries from the start down to the stop must be ready (at least an
// aggregate); a round whose needed entries are not all ready is polled again,
// re-reading only the lanes that were incomplete.  The fold of the walked
// entries (earlier entries combined first) is returned in every lane, with
// `real_stop` telling whether the walk ended at a status entry (true) or at
// `floor` (false).  A wait that runs out, or a launch already aborted by
// another wait, ends the walk early (returns false).
template <class Op, int HEADS, int LB>
__device__ __forceinline__ bool walk_back(unsigned long long* rec, bool group, int64_t base,
                                          int64_t floor, uint32_t epoch, const LookbackCfg& cfg,
                                          Header* hdr, int64_t tile, int lane, uint64_t& t0,
                                          bool& out_f, typename Op::Acc& out_v, bool& real_stop) {
    using Acc = typename Op::Acc;
    bool pf = false;
    Acc pv = Op::identity();
    real_stop = false;
    while (true) {
        uint32_t st[LB];
        bool hf[LB];
        Acc hv[LB];
        int jstop = LB;  // this lane's first stopping entry (LB: none)
        bool complete = false;
        uint32_t need = 0, stop_lanes = 0;
        uint32_t ns = 20;
        while (true) {
            if (!complete) {
#pragma unroll
                for (int j = 0; j < LB; ++j) {
                    const int64_t idx = base - static_cast<int64_t>(lane) * LB - j;
                    if (idx >= floor) {
                        read_words<Op>(group ? rec_group(rec, idx) : rec_tile<Op>(rec, idx), epoch, st[j],
                                       hf[j], hv[j]);
                    } else {
                        st[j] = kStateP;  // below the floor: the identity
                        hf[j] = false;
                        hv[j] = Op::identity();
                    }
                }
                jstop = LB;
#pragma unroll
                for (int j = LB - 1; j >= 0; --j)
                    if (st[j] == kStateP || (st[j] == kStateA && hf[j])) jstop = j;
                complete = true;
#pragma unroll
                for (int j = 0; j < LB; ++j)
                    if (j <= jstop && st[j] == kStateX) complete = false;
            }
            stop_lanes = __ballot_sync(0xffffffffu, jstop < LB);
            need = stop_lanes ? (((stop_lanes & (0u - stop_lanes)) << 1) - 1u) : 0xffffffffu;
            const uint32_t incomplete = __ballot_sync(0xffffffffu, !complete);
            if ((incomplete & need) == 0) break;
            // bounded wait: give up after the spin limit or once another wait
            // has aborted the launch
            int quit = 0;
            if (lane == 0) {
                const uint64_t now = global_timer_ns();
                if (t0 == 0) t0 = now;
                if (now - t0 > cfg.spin_limit_ns) {
                    record_timeout(hdr, epoch, tile);
                    quit = 1;
                } else if (launch_aborted(hdr, epoch)) {
                    quit = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, quit, 0)) {
                out_f = pf;
                out_v = pv;
                return false;
            }
            __nanosleep(ns);
            ns = ns < 160 ? ns * 2 : 160;
            poll_round_fence();
        }
        // this lane's share, earliest entry first (higher j = earlier)
        bool rf = false;
        Acc rv = Op::identity();
        if ((need >> lane) & 1u) {
#pragma unroll
            for (int j = LB - 1; j >= 0; --j) {
                if (j <= jstop) {
                    if (HEADS != kNoHeads) {
                        bool f2 = hf[j];
                        Acc v2 = hv[j];
                        seg_combine<Op>(rf, rv, f2, v2);
                        rf = f2;
                        rv = v2;
                    } else {
                        rv = Op::combine(rv, hv[j]);
                    }
                }
            }
        }
        // fold the lanes in order (higher lane = earlier entries)
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
        if (stop_lanes) {
            // the stop is real unless it is the first entry below the floor
            const int sl = __ffs(stop_lanes) - 1;
            const int js = __shfl_sync(0xffffffffu, jstop, sl);
            real_stop = (base - static_cast<int64_t>(sl) * LB - js) >= floor;
            break;
        }
        base -= 32 * LB;
    }
    out_f = pf;
    out_v = pv;
    return true;
}

// Finds the exclusive prefix of `tile` and publishes the tile's inclusive
// prefix (its aggregate must already be published), in two levels:
//   1. the tile's own group (16 tiles): walk back over the tiles of the group
//      before this one; a stop there settles the prefix.  If the walk reaches
//      the group start and this is the group's last tile, the fold plus the
//      tile's own aggregate is the group aggregate: publish it.
//   2. earlier groups: walk back over group status words (32 * LBG groups per
//      round) to the nearest group inclusive prefix.
// The group's last tile also publishes its inclusive prefix as the group's.
// So a look-back costs about two round trips however many tiles are in
// flight.  A wait that runs out (or a launch already aborted by another wait)
// ends the look-back with the prefix found so far, which is then wrong, but
// successors are released and the launch finishes; the host learns of it from
// the workspace.  Returns the exclusive prefix in every lane.
template <class Op, int HEADS, int LB>
__device__ __forceinline__ void lookback(unsigned long long* rec, Header* hdr, int64_t tile,
                                         uint32_t epoch, const LookbackCfg& cfg, bool agg_f,
                                         typename Op::Acc agg_v, int lane, bool& out_f,
                                         typename Op::Acc& out_v) {
    using Acc = typename Op::Acc;
    const bool dropped = (tile == cfg.drop_tile);
    const int64_t g = tile / kGroup;
    const bool last_in_group = (tile % kGroup) == kGroup - 1;
    bool pf = false;
    Acc pv = Op::identity();
    uint64_t t0 = 0;
    bool real = false;
    bool ok = true;
    if (tile % kGroup != 0) {
        ok = walk_back<Op, HEADS, 1>(rec, false, tile - 1, g * kGroup, epoch, cfg, hdr, tile, lane,
                                     t0, pf, pv, real);
        if (ok && !real && last_in_group && lane == 0 && !dropped) {
            bool gf = agg_f;
            Acc gv = agg_v;
            if (HEADS != kNoHeads)
                seg_combine<Op>(pf, pv, gf, gv);
            else
                gv = Op::combine(pv, gv);
            publish_group<Op>(rec, g, epoch, kStateA, gf, gv);
        }
    } else if (last_in_group && lane == 0 && !dropped) {
        publish_group<Op>(rec, g, epoch, kStateA, agg_f, agg_v);  // one-tile groups
    }
    if (ok && !real && g > 0) {
        bool qf;
        Acc qv;
        ok = walk_back<Op, HEADS, LB>(rec, true, g - 1, 0, epoch, cfg, hdr, tile, lane, t0, qf, qv,
                                      real);
        if (HEADS != kNoHeads)
            seg_combine<Op>(qf, qv, pf, pv);
        else
            pv = Op::combine(qv, pv);
    }
    bool incf = agg_f;
    Acc incv = agg_v;
    if (HEADS != kNoHeads)
        seg_combine<Op>(pf, pv, incf, incv);
    else
        incv = Op::combine(pv, incv);
    if (lane == 0 && !dropped && tile != 0) {
        if (cfg.delay_max) {
            const uint32_t dly =
                mix32(static_cast<uint64_t>(tile) * 0xc2b2ae3d27d4eb4full) % (cfg.delay_max + 1);
            if (dly) __nanosleep(dly);
        }
        publish<Op>(rec, tile, epoch, kStateP, incf, incv);
    }
    if (last_in_group && lane == 0 && !dropped) publish_group<Op>(rec, g, epoch, kStateP, incf, incv);
    out_f = pf;
    out_v = pv;
}

// Epoch bookkeeping at the end of a single-pass launch: the last block to
// finish resets the tile counter and records the epoch; before the 29-bit tag
// wraps it clears every status word, so that no word written 2^29 launches
// ago can pass for a current one.  Called by one thread per block; returns
// true in the block that must clear.
__device__ __forceinline__ bool finish_launch(Header* hdr, uint32_t epoch) {
    __threadfence();
    const uint32_t prev = atomicAdd(&hdr->done_counter, 1u);
    if (prev != gridDim.x - 1) return false;
    __threadfence();
    hdr->tile_counter = 0;
    hdr->done_counter = 0;
    const bool wrap = (epoch == kEpochMask);
    hdr->epoch = wrap ? 0u : epoch;
    if (wrap) hdr->abort_epoch = 0u;
    return wrap;
}

// Zero every status word (words 0..31 and 48..53 of each block) of
// `capacity` tile records, by `nthreads` threads of one block.
__device__ __forceinline__ void clear_status_words(unsigned long long* rec, int64_t capacity,
                                                   int tid, int nthreads) {
    const int64_t blocks = (capacity + kGroup - 1) / kGroup;
    for (int64_t i = tid; i < blocks * 38; i += nthreads) {
        const int64_t b = i / 38;
        const int w = static_cast<int>(i % 38);
        rec[b * kRecBlockWords + (w < 32 ? w : 48 + (w - 32))] = 0ull;
    }
    __threadfence();
}

__device__ __forceinline__ uint32_t launch_epoch(uint32_t completed) {
    const uint32_t e = (completed + 1) & kEpochMask;
    return e == 0 ? 1u : e;
}

}  // namespace gbscan
