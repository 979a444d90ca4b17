// Small inputs: the two-pass scan with the whole array resident in shared
// memory, in one launch.
//
// resident_scan_kernel: one block per tile, and every block resident at once
// (a cooperative launch of at most SMs x blocks-per-SM tiles).  Each block
// copies its tile into shared memory (one bulk copy; a ragged or misaligned
// tile by the threads), sums each thread's run of items, scans the thread
// sums across the block and publishes the tile's sum as the tile's status
// word.  Warp 0 then waits for the sums of all tiles before its own and folds
// them: lane l reads the words of tiles l, l + 32, ... (32 consecutive words
// per read, coalesced) and re-reads only the words not yet published.  The
// block writes its outputs from the items it kept, through shared memory and
// one bulk store.  This is the two-pass scan of Figure 1b, accumulate then
// prefix sum, with each block scanning the tile sums it needs, combined with
// the partitioning of Section 2.2: the second pass over a partition reads it
// from the cache, and here the whole array is one partition and the SMs'
// shared memory is the cache.  The array is read from memory once and written
// once.
//
// Waiting on sums only, never on another block's prefix, keeps the wait as
// short as the slowest copy: there is no chain of inclusive prefixes.  Every
// block of the launch is resident, so the tiles a block waits for always make
// progress.  Compared with the look-back of the persistent kernels (lanes
// reading LB consecutive entries each, LB apart across the warp), the
// coalesced rows need a few requests per poll where the look-back's need one
// per lane and entry; with hundreds of blocks polling the same few lines at
// once, those requests queue in the L2 slices that hold the lines.
#pragma once

#include "lookback.cuh"

namespace gbscan {

template <class Op, int NWARPS>
struct ResCtrl {
    using Acc = typename Op::Acc;
    uint64_t full;
    alignas(16) Acc wtot[NWARPS];
    Acc prefix;
    uint32_t epoch;
    uint32_t clear;
};

template <class Op, int THREADS, int ITEMS>
constexpr int resident_smem_bytes() {
    return THREADS * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(ResCtrl<Op, THREADS / 32>));
}

// Most tiles a launch takes: lane l of the waiting warp keeps a 32-bit mask of
// its unread rows (tiles l + 32 k, k < 32).
constexpr int64_t kResidentMaxTiles = 1024;

// The fold of the sums of tiles 0 .. tile-1 (all lanes of one warp, every
// lane returns it): each poll round reads the unread rows of the lane, four
// loads in flight, and folds the published ones (the operators are
// commutative, so the order of the fold changes float rounding only).
// Bounded: after the spin limit it records a timeout and returns what it has;
// a launch already aborted by another wait ends it at once.  `ok` tells which.
template <class Op>
__device__ __forceinline__ typename Op::Acc resident_prefix(unsigned long long* rec, Header* hdr,
                                                            int64_t tile, uint32_t epoch,
                                                            const LookbackCfg& cfg, int lane, bool& ok) {
    using Acc = typename Op::Acc;
    const int rows = tile > lane ? static_cast<int>((tile - 1 - lane) / 32) + 1 : 0;
    uint32_t pending = rows >= 32 ? 0xffffffffu : ((1u << rows) - 1u);
    Acc s = Op::identity();
    const uint64_t t0 = global_timer_ns();
    ok = true;
    while (true) {
        for (int k0 = 0; k0 < rows; k0 += 4) {
            if (((pending >> k0) & 15u) == 0) continue;
            uint32_t st[4];
            bool hf[4];
            Acc v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                st[q] = kStateX;
                if ((pending >> (k0 + q)) & 1u)
                    read_words<Op>(rec_tile<Op>(rec, lane + 32 * (k0 + q)), epoch, st[q], hf[q], v[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (st[q] != kStateX) {
                    s = combine_local<Op>(s, v[q]);
                    pending &= ~(1u << (k0 + q));
                }
            }
        }
        if (__all_sync(0xffffffffu, pending == 0)) break;
        int quit = 0;
        if (lane == 0) {
            if (global_timer_ns() - t0 > cfg.spin_limit_ns) {
                record_timeout(hdr, epoch, tile);
                quit = 1;
            } else if (launch_aborted(hdr, epoch)) {
                quit = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, quit, 0)) {
            ok = false;
            break;
        }
        __nanosleep(32);
        poll_round_fence();
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) s = combine_local<Op>(s, shfl_xor_acc<Op>(s, d));
    return s;
}

template <class Op, int THREADS, int ITEMS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) resident_scan_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int NWARPS = THREADS / 32;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    static_assert(ITEMS * sizeof(T) % 16 == 0, "a thread's items are whole 16-byte vectors");
    using CtrlT = ResCtrl<Op, NWARPS>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + TILE_BYTES);
    T* buf = reinterpret_cast<T*>(smem);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t tile = blockIdx.x;
    const T* __restrict__ in = static_cast<const T*>(p.in) + tile * TILE;
    T* out = static_cast<T*>(p.out) + tile * TILE;
    const int64_t rem = p.n - tile * TILE;
    const int cnt = rem < TILE ? static_cast<int>(rem) : TILE;
    const bool whole = p.fast && cnt == TILE;

    // the tile's copy goes out first, so that its latency overlaps the set-up
    if (tid == 0) {
        mbar_init(&c.full, 1);
        fence_mbar_init();
        if (whole) {
            mbar_arrive_expect_tx(&c.full, TILE_BYTES);
            bulk_load_hint(buf, in, TILE_BYTES, &c.full, l2_policy_evict_first());
        }
        c.epoch = hdr->epoch;
        c.clear = 0;
    }
    if (!whole) {
        // ragged or misaligned: the threads copy, all ITEMS loads of a thread
        // in flight at once, padding the tile
        T v[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            const int i = k * THREADS + tid;
            v[k] = i < cnt ? in[i] : Op::pad();
        }
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) buf[k * THREADS + tid] = v[k];
    }
    __syncthreads();
    const uint32_t epoch = launch_epoch(c.epoch);
    const LookbackCfg cfg = read_lookback_cfg(hdr);
    const uint64_t role_limit = 4 * cfg.spin_limit_ns + 10000000ull;
    // every warp polls the copy's phase (bounded; after a failed wait the
    // launch is aborted, its output is not used, and the copy is drained
    // before the block exits)
    if (whole) warp_spin_wait(&c.full, 0, role_limit, hdr, epoch, lane);

    // ---- pass 1: the thread's items, its sum, the warp scan, the tile's sum -
    T x[ITEMS];
    load_items<T, ITEMS, TILE, false>(buf, tid, x);
    bool tf;
    Acc tv;
    thread_reduce<Op, ITEMS, kNoHeads>(x, 0u, tf, tv);
    bool wf = false;
    Acc wv = tv;
    warp_inclusive_scan<Op, kNoHeads>(wf, wv, lane);
    if (lane == 31) c.wtot[warp] = wv;
    __syncthreads();
    Acc agg = Op::identity(), woff = Op::identity();
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) {
        const Acc wt = c.wtot[w];
        agg = combine_local<Op>(agg, wt);
        if (w < warp) woff = combine_local<Op>(woff, wt);
    }

    // ---- the tile's sum out, the sums of the tiles before it in ----------
    if (warp == 0) {
        // (debug hook: the drop tile never publishes)
        if (lane == 0 && tile != cfg.drop_tile)
            publish_words<Op>(rec_tile<Op>(p.rec, tile), epoch, kStateA, false, agg);
        bool ok;
        const Acc s = resident_prefix<Op>(p.rec, hdr, tile, epoch, cfg, lane, ok);
        if (lane == 0) c.prefix = s;
        // The last tile's block, once its wait has ended, makes this launch's
        // epoch the completed one (the next launch takes the one after).
        // Every block reads the epoch in its first instructions, and the
        // thread that read it later tags its tile's sum with it, so the sums
        // this block has waited for show that their blocks have read it; all
        // blocks are resident from the start of the launch, so a wait that
        // ran out (200 ms by default) leaves no block unstarted.  Only the
        // epoch wrap, which must clear every status word after the last block
        // is done with them, goes through the done count (finish_launch).
        if (lane == 0 && tile == static_cast<int64_t>(gridDim.x) - 1 && epoch != kEpochMask)
            hdr->epoch = epoch;
    }
    __syncthreads();

    // ---- pass 2: outputs from the kept items, stored from shared memory ---
    Acc ev = shfl_up_acc<Op>(wv, 1);
    if (lane == 0) ev = Op::identity();
    const Acc gv = Op::combine(Op::combine(c.prefix, woff), ev);
    T y[ITEMS];
    thread_outputs<Op, ITEMS, kNoHeads>(x, 0u, gv, p.exclusive != 0, y);
    store_items<T, ITEMS, TILE, false>(buf, tid, y);
    if (whole) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_store(out, buf, TILE_BYTES);
            bulk_commit();
        }
    } else {
        __syncthreads();
        for (int i = tid; i < cnt; i += THREADS) out[i] = buf[i];
    }

    if (tid == 0) {
        if (whole) drain_fills<1>(&c.full, 1u, role_limit, hdr);
        bulk_wait_read_all();  // the store has read the block's shared memory before it is given up
    }
    if (epoch == kEpochMask) {  // the same for every block of the launch
        __syncthreads();
        if (tid == 0) c.clear = finish_launch(hdr, epoch) ? 1u : 0u;
        __syncthreads();
        if (c.clear) clear_status_words(p.rec, p.rec_capacity, tid, blockDim.x);
    }
}

}  // namespace gbscan
