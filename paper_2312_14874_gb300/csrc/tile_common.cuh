// tile_common.cuh — per-thread pieces shared by the tile kernels: moving a
// thread's items between shared memory and registers, segment heads, the
// sequential thread scan, the warp scan, and the per-element outputs.
#pragma once

#include "gbscan_device.cuh"

namespace gbscan {

// Thread t owns the logical items [t*ITEMS, (t+1)*ITEMS) of a tile.  Forward,
// logical item L sits at buf[L]; reverse, at buf[TILE-1-L] (a partial tile is
// stored right-aligned, so the same mapping holds).  The 16-byte reads of a
// thread are contiguous; with an odd number of vectors per thread, the eight
// lanes of a shared-memory wavefront hit eight different 16-byte bank groups.
template <class T, int ITEMS, int TILE, bool REVERSE>
__device__ __forceinline__ void load_items(const T* buf, int tid, T (&x)[ITEMS]) {
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int NVEC = ITEMS / VEC;
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

template <class T, int ITEMS, int TILE, bool REVERSE>
__device__ __forceinline__ void store_items(T* buf, int tid, const T (&y)[ITEMS]) {
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int NVEC = ITEMS / VEC;
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

// Bit j set: the thread's item j is inside the tile's cnt valid elements.
template <int ITEMS>
__device__ __forceinline__ uint32_t valid_items(int cnt, int tid) {
    const int nvalid = cnt - tid * ITEMS;
    return nvalid <= 0 ? 0u : (nvalid >= 32 ? 0xffffffffu : ((1u << nvalid) - 1u));
}

// Segment heads of rows of `cols` elements.  Forward: a head is a row's first
// element (physical index % cols == 0).  Reverse: logical item L is physical
// tb + cnt - 1 - L and a head is a row's last element.
template <int ITEMS, bool REVERSE>
__device__ __forceinline__ uint32_t row_heads(int64_t tb, int cnt, int64_t cols, int tid) {
    uint32_t hm = 0;
    if constexpr (!REVERSE) {
        int64_t r = (tb + static_cast<int64_t>(tid) * ITEMS) % cols;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (r == 0) hm |= 1u << j;
            r = (r + 1 == cols) ? 0 : r + 1;
        }
    } else {
        int64_t q = (tb + cnt - static_cast<int64_t>(tid) * ITEMS) % cols;
        if (q < 0) q += cols;
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (q == 0) hm |= 1u << j;
            q = (q == 0) ? cols - 1 : q - 1;
        }
    }
    return hm;
}

// Sequential reduction of the thread's items; a head restarts the sum.
// Operators whose accumulation is a long dependent chain (Op::kSplit > 1, the
// compensated TwoSum pairs) sum a thread's items as kSplit contiguous
// sub-blocks in independent chains, combined once at the end: the chain a
// thread waits for is ITEMS / kSplit accumulations long instead of ITEMS.
template <class Op, int ITEMS>
__device__ __forceinline__ void split_sums(const typename Op::T (&x)[ITEMS],
                                           typename Op::Acc (&part)[Op::kSplit]) {
    constexpr int K = Op::kSplit, L = ITEMS / K;
#pragma unroll
    for (int k = 0; k < K; ++k) part[k] = Op::lift(x[k * L]);
#pragma unroll
    for (int j = 1; j < L; ++j) {
#pragma unroll
        for (int k = 0; k < K; ++k) Op::accumulate(part[k], x[k * L + j]);
    }
}

template <class Op, int ITEMS, int HEADS>
__device__ __forceinline__ void thread_reduce(const typename Op::T (&x)[ITEMS], uint32_t hm,
                                              bool& f, typename Op::Acc& v) {
    f = false;
    if constexpr (HEADS == kNoHeads && Op::kSplit > 1 && ITEMS % Op::kSplit == 0) {
        typename Op::Acc part[Op::kSplit];
        split_sums<Op, ITEMS>(x, part);
        v = part[0];
#pragma unroll
        for (int k = 1; k < Op::kSplit; ++k) v = combine_local<Op>(v, part[k]);
        return;
    }
    v = Op::identity();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if (HEADS != kNoHeads && ((hm >> j) & 1u)) {
            v = Op::lift(x[j]);
            f = true;
        } else {
            Op::accumulate(v, x[j]);
        }
    }
}

// Inclusive Hillis-Steele scan over the 32 lanes (log2(32) = 5 shift-and-add
// steps, the in-register scan of Section 3.1 with lanes for SIMD slots).
// Segmented: one ballot of the head flags gives each lane the last lane at or
// before it that holds a head (`start`, 0 if none), and a step adds lane
// lane-d only when lane-d >= start.  That is the condition under which the
// flag-carrying form (shuffle the flag with the value, add while no head has
// been seen) adds, so the results are the same, without five flag shuffles.
template <class Op, int HEADS>
__device__ __forceinline__ void warp_inclusive_scan(bool& f, typename Op::Acc& v, int lane) {
    using Acc = typename Op::Acc;
    if constexpr (HEADS != kNoHeads) {
        const uint32_t upto = __ballot_sync(0xffffffffu, f) & (0xffffffffu >> (31 - lane));
        const int start = upto ? 31 - __clz(upto) : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Acc vo = shfl_up_acc<Op>(v, d);
            if (lane - d >= start) v = combine_local<Op>(vo, v);
        }
        f = upto != 0u;
    } else {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Acc vo = shfl_up_acc<Op>(v, d);
            if (lane >= d) v = combine_local<Op>(vo, v);
        }
    }
}

// Outputs of the thread's items given everything before its first item
// (gf, gv).  Inclusive: y_j = prefix through item j; exclusive: before item j
// (a segment head starts at 0).  Each output is the carry combined once with
// the thread's local running sum.
template <class Op, int ITEMS, int HEADS, bool EXCL>
__device__ __forceinline__ void thread_outputs_t(const typename Op::T (&x)[ITEMS], uint32_t hm,
                                                 typename Op::Acc gv, typename Op::T (&y)[ITEMS]) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    if constexpr (HEADS == kNoHeads && Op::kSplit > 1 && ITEMS % Op::kSplit == 0) {
        // sub-block sums, the carry into each sub-block, then each sub-block's
        // outputs from its own carry: K independent chains of ITEMS / K
        constexpr int K = Op::kSplit, L = ITEMS / K;
        Acc part[K];
        split_sums<Op, ITEMS>(x, part);
        Acc cin[K];
        cin[0] = gv;
#pragma unroll
        for (int k = 1; k < K; ++k) cin[k] = combine_local<Op>(cin[k - 1], part[k - 1]);
        Acc r[K];
#pragma unroll
        for (int k = 0; k < K; ++k) r[k] = run_init<Op>(cin[k]);
#pragma unroll
        for (int j = 0; j < L; ++j) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (EXCL) y[k * L + j] = Op::output(cin[k], r[k]);
                Op::accumulate(r[k], x[k * L + j]);
                if (!EXCL) y[k * L + j] = Op::output(cin[k], r[k]);
            }
        }
        return;
    }
    bool rf = false;
    Acc rv = run_init<Op>(gv);
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const bool h = HEADS != kNoHeads && ((hm >> j) & 1u);
        if (EXCL) y[j] = h ? Op::output1(Op::identity()) : (rf ? Op::output1(rv) : Op::output(gv, rv));
        if (h) {
            rv = Op::lift(x[j]);
            rf = true;
        } else {
            Op::accumulate(rv, x[j]);
        }
        if (!EXCL) y[j] = rf ? Op::output1(rv) : Op::output(gv, rv);
    }
}

template <class Op, int ITEMS, int HEADS>
__device__ __forceinline__ void thread_outputs(const typename Op::T (&x)[ITEMS], uint32_t hm,
                                               typename Op::Acc gv, bool excl,
                                               typename Op::T (&y)[ITEMS]) {
    // excl is the same for the whole launch: one branch, two straight loops
    if (excl)
        thread_outputs_t<Op, ITEMS, HEADS, true>(x, hm, gv, y);
    else
        thread_outputs_t<Op, ITEMS, HEADS, false>(x, hm, gv, y);
}

// The part of staging a tile that the lanes of one warp do when the tile is
// not a whole, aligned tile (a ragged last tile, or arrays that are not
// 16-byte aligned).  Elements [0, cnt) of src go to dst.  With `bulk_ok` (src
// and dst 16-byte aligned) the largest 16-byte multiple prefix is left to one
// bulk copy that the caller issues on its barrier: its byte count is
// returned.  The lanes copy the rest with B loads in flight each (one
// dependent load at a time made a ragged tile cost about 15 us, which then
// gated the end of every launch), and write `pad` into [cnt, fill).  The
// caller orders these generic writes before its barrier arrive (__syncwarp).
template <class T>
__device__ __forceinline__ uint32_t warp_stage_partial(T* dst, const T* src, int cnt, int fill,
                                                       bool bulk_ok, T pad, int lane) {
    constexpr int B = 16;
    const uint32_t bulk =
        bulk_ok ? (static_cast<uint32_t>(cnt) * static_cast<uint32_t>(sizeof(T))) & ~15u : 0u;
    const int first = static_cast<int>(bulk / sizeof(T));
    for (int base = first; base < cnt; base += 32 * B) {
        T v[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = base + b * 32 + lane;
            if (i < cnt) v[b] = src[i];
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int i = base + b * 32 + lane;
            if (i < cnt) dst[i] = v[b];
        }
    }
    for (int i = cnt + lane; i < fill; i += 32) dst[i] = pad;
    return bulk;
}

// Named barrier `id` over NTHREADS threads that also ORs a predicate over them:
// every thread gets true if any thread passed true.
template <int NTHREADS>
__device__ __forceinline__ bool named_barrier_or(int id, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred ? 1u : 0u), "r"(id), "n"(NTHREADS)
        : "memory");
    return r != 0;
}

template <int NTHREADS>
__device__ __forceinline__ void named_barrier_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NTHREADS) : "memory");
}

#ifndef GBSCAN_SUSPEND_NS
#define GBSCAN_SUSPEND_NS 20000u
#endif

// Bounded mbarrier wait; returns false if the phase did not complete within
// the limit (or, with epoch != 0, once the launch has been aborted by another
// wait).  With `report`, a wait that runs out records a timeout for `epoch`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns, Header* hdr, uint32_t epoch,
                                                  bool report) {
#ifdef GBSCAN_WAIT_POLL
    if (mbar_test_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    uint32_t polls = 0;
    while (!mbar_test_wait(bar, parity)) {
        __nanosleep(64);
        if ((polls & 31) != 31) { ++polls; continue; }
#else
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    uint32_t polls = 0;
    while (!mbar_try_wait_sleep(bar, parity, GBSCAN_SUSPEND_NS)) {
#endif
        if ((++polls & 7) == 0 && epoch != 0 && launch_aborted(hdr, epoch)) return false;
        if (global_timer_ns() - t0 > limit_ns) {
            if (report) {
                if (epoch != 0)
                    record_timeout(hdr, epoch, -1);
                else
                    record_error(hdr, GBSCAN_ERR_TIMEOUT, -1);
            }
            return false;
        }
    }
    return true;
}

// Warp-uniform bounded wait: lane 0 alone observes the mbarrier phase (with
// the bound), the warp learns the outcome, and __syncwarp orders lane 0's
// view of memory (including the bulk-copied data the phase covers) before the
// other lanes' accesses.  Only one thread per warp touches the mbarrier:
// redundant waits by every lane would park the other lanes in the barrier
// unit for about a microsecond.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                          Header* hdr, uint32_t epoch, int lane) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_bounded(bar, parity, limit_ns, hdr, epoch, true) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Before a block exits, the bulk copies it started into shared memory must
// have landed: a copy still in flight would write into shared memory that the
// next block on the SM may own.  The loader calls this once its loop has
// ended, with fills = the number of times it filled the stages in order (fill
// k went to stage k % STAGES and completes phase k / STAGES of full[stage]).
// Only the last fill of each stage can still be pending: a stage is refilled
// only after its previous fill was consumed.  Each wait is bounded; one that
// runs out is recorded (an earlier error is kept).
template <int STAGES>
__device__ __forceinline__ void drain_fills(uint64_t* full, uint32_t fills, uint64_t limit_ns,
                                            Header* hdr) {
    for (int s = 0; s < STAGES; ++s) {
        if (static_cast<uint32_t>(s) >= fills) break;
        const uint32_t last = (fills - 1 - static_cast<uint32_t>(s)) / STAGES * STAGES + s;
        mbar_wait_bounded(&full[s], (last / STAGES) & 1u, limit_ns, hdr, 0, true);
    }
}

// Warp-uniform dispatch for segmented kinds.  The flagged versions cost
// several instructions per element more than the plain ones; a warp none of
// whose items is a segment head (warp_heads false, decided with __any_sync by
// the whole warp) takes the plain code, which gives the same result because no
// flag is ever set in it.
template <class Op, int ITEMS, int HEADS>
__device__ __forceinline__ void thread_reduce_w(const typename Op::T (&x)[ITEMS], uint32_t hm,
                                                bool warp_heads, bool& f, typename Op::Acc& v) {
    if (HEADS != kNoHeads && warp_heads)
        thread_reduce<Op, ITEMS, HEADS>(x, hm, f, v);
    else
        thread_reduce<Op, ITEMS, kNoHeads>(x, 0u, f, v);
}

template <class Op, int HEADS>
__device__ __forceinline__ void warp_inclusive_scan_w(bool warp_heads, bool& f, typename Op::Acc& v,
                                                      int lane) {
    if (HEADS != kNoHeads && warp_heads)
        warp_inclusive_scan<Op, HEADS>(f, v, lane);
    else
        warp_inclusive_scan<Op, kNoHeads>(f, v, lane);
}

template <class Op, int ITEMS, int HEADS>
__device__ __forceinline__ void thread_outputs_w(const typename Op::T (&x)[ITEMS], uint32_t hm,
                                                 bool warp_heads, typename Op::Acc gv, bool excl,
                                                 typename Op::T (&y)[ITEMS]) {
    if (HEADS != kNoHeads && warp_heads)
        thread_outputs<Op, ITEMS, HEADS>(x, hm, gv, excl, y);
    else
        thread_outputs<Op, ITEMS, kNoHeads>(x, 0u, gv, excl, y);
}

}  // namespace gbscan
