// partitioned.cuh — the cache-friendly partitioned scan.
//
// The paper's central proposal (Section 2.2, Figure 2): split the data into
// cache-sized partitions and make both passes of the two-pass scheme over one
// partition before moving on, so that the second pass reads from cache instead
// of memory; keep two `sums` arrays so that the second pass of iteration k
// overlaps the first pass of iteration k+1 (Section 2.2.1).  Here the cache is
// the GPU's L2 (129 MB): a chunk is a run of chunk_tiles tiles of a few tens of
// MB, and one persistent launch processes a work list in which the second pass
// (scan) of chunk c is interleaved with the first pass (reduce, "Accumulate")
// of chunk c+2 (a lag of two chunks, so that the scan of chunk c's tile sums
// has a whole chunk of reductions to finish in):
//
//   R(0) R(1) | S(0) R(2) S(0) R(2) ... | S(1) R(3) ... | ... | S(C-1)
//
// R item:  TMA-load the tile with L2 evict-last priority (it will be read again),
//          sum it, publish the sum in the tile's status word.  The last R item of
//          a chunk then scans the chunk's tile sums (the per-partition `sums`
//          array): waits until all are published, publishes each tile's
//          exclusive offset within the chunk in the tile's status word, and
//          chains the chunk prefixes (E, P) from the previous chunk.
// S item:  TMA-load the tile again (from L2, evict-first) together with the two
//          status words it needs (its in-chunk offset and the chunk prefix E),
//          which are self-validating (epoch-tagged), so no global round trip is
//          left on the scan's path; scan, store with a TMA bulk store.
//
// There is no per-tile dependency chain: a tile's S item waits only for its
// chunk's prefix, published once per chunk, which is why this scheme reaches
// copy bandwidth where a per-tile chained scan is bound by status round trips.
// Plain (unsegmented, forward) scans only.
#pragma once

#include "tile_common.cuh"

namespace gbscan {

enum : uint32_t { kItemReduce = 0, kItemScan = 1 };

constexpr int64_t kLag = 2;  // S(c) is interleaved with R(c + kLag)

// Work item w of the list above, for num_tiles tiles in chunks of K:
//   R(0) .. R(kLag-1) in tile order, then for each chunk c the slot
//   S(c) / R(c+kLag) alternating (S first) while both have items, then the rest.
__device__ __forceinline__ void partitioned_item(int64_t w, int64_t num_tiles, int64_t K,
                                                 uint32_t& phase, int64_t& tile) {
    const int64_t C = (num_tiles + K - 1) / K;
    const int64_t nlast = num_tiles - (C - 1) * K;
    const int64_t pre = kLag < C ? kLag : C;
    const int64_t npre = pre < C ? pre * K : (C - 1) * K + nlast;
    if (w < npre) {
        phase = kItemReduce;
        tile = w;
        return;
    }
    w -= npre;
    const int64_t F = C - 1 - kLag > 0 ? C - 1 - kLag : 0;  // slots with both parts full
    if (w < F * 2 * K) {
        const int64_t c = w / (2 * K), off = w % (2 * K), j = off / 2;
        phase = (off & 1) ? kItemReduce : kItemScan;
        tile = ((off & 1) ? c + kLag : c) * K + j;
        return;
    }
    w -= F * 2 * K;
    int64_t c = F;
    if (C - 1 - kLag >= 0) {
        // slot F: S(F) (K items) alternating with R(C-1) (nlast items)
        if (w < 2 * nlast) {
            const int64_t j = w / 2;
            phase = (w & 1) ? kItemReduce : kItemScan;
            tile = ((w & 1) ? C - 1 : F) * K + j;
            return;
        }
        if (w < K + nlast) {
            phase = kItemScan;
            tile = F * K + nlast + (w - 2 * nlast);
            return;
        }
        w -= K + nlast;
        c = F + 1;
    }
    phase = kItemScan;  // the remaining slots hold scans only, in tile order
    tile = c * K + w;
}

template <class Op, int CWARPS, int STAGES, int TILE>
struct PtCtrl {
    using Acc = typename Op::Acc;
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int64_t tile_id[STAGES];
    uint32_t phase[STAGES];
    // per stage, for a scan item: copies of the tile's status word pair (the
    // 16-byte pair holding lo[t], and the one holding hi[t]) and of the chunk's
    // E words, brought in by the loader's bulk copies
    alignas(16) unsigned long long stat[STAGES][6];
    Acc wtot_v[CWARPS];
    Acc prefix_v;
    uint32_t epoch;
    uint32_t clear;
    uint32_t cflag;
};

template <class Op, int CWARPS, int ITEMS, int STAGES>
constexpr int pt_smem_bytes() {
    return STAGES * CWARPS * 32 * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(PtCtrl<Op, CWARPS, STAGES, CWARPS * 32 * ITEMS>));
}

template <int CWARPS>
constexpr int pt_threads() {
    return (CWARPS + 1) * 32;
}

// Most tiles a chunk may have: the chunk scan gives each consumer thread up to
// kChunkPerThread tile sums.
constexpr int kChunkPerThread = 16;

template <class Op, int CWARPS, int ITEMS, int STAGES, int MINB>
__global__ void __launch_bounds__((CWARPS + 1) * 32, MINB) partitioned_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int CTHREADS = CWARPS * 32;
    constexpr int TILE = CTHREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int LOAD_WARP = CWARPS;
    static_assert(STAGES >= 2, "a stage is released one store later: at least two stages");
    using CtrlT = PtCtrl<Op, CWARPS, STAGES, TILE>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * TILE_BYTES);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t num_tiles = p.num_tiles;
    const int64_t K = p.chunk_tiles;
    const int64_t num_items = 2 * num_tiles;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&c.full[s], 1);
            mbar_init(&c.empty[s], 1);
        }
        fence_mbar_init();
        c.epoch = hdr->epoch;
        c.clear = 0;
    }
    __syncthreads();
    const uint32_t epoch = launch_epoch(c.epoch);
    const LookbackCfg cfg = read_lookback_cfg(hdr);
    const uint64_t role_limit = 4 * cfg.spin_limit_ns + 10000000ull;
    auto count_of = [&](int64_t t) -> int {
        const int64_t rem = p.n - t * TILE;
        return rem < TILE ? static_cast<int>(rem) : TILE;
    };

    if (warp == LOAD_WARP) {
        const T* __restrict__ in = static_cast<const T*>(p.in);
        const uint64_t keep = l2_policy_evict_last();
        const uint64_t drop = l2_policy_evict_first();
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (use > 0 && !warp_wait(&c.empty[s], (use - 1) & 1u, role_limit, hdr, epoch, lane))
                break;
            long long claimed = 0;
            if (lane == 0) claimed = static_cast<long long>(atomicAdd(&hdr->tile_counter, 1u));
            const int64_t w = __shfl_sync(0xffffffffu, claimed, 0);
            if (w >= num_items) {
                // end: a sentinel stage ends the consumers' loop
                if (lane == 0) {
                    c.tile_id[s] = num_tiles;
                    mbar_arrive(&c.full[s]);
                }
                break;
            }
            uint32_t phase;
            int64_t t;
            partitioned_item(w, num_tiles, K, phase, t);
            const int cnt = count_of(t);
            const bool fast = p.fast && cnt == TILE;
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
            if (!fast) {
                for (int i = lane; i < cnt; i += 32) buf[i] = in[t * TILE + i];
                __syncwarp();
            }
            if (lane == 0) {
                c.tile_id[s] = t;
                c.phase[s] = phase;
                const uint32_t stat_bytes = phase == kItemScan ? (Op::kPacked ? 32u : 48u) : 0u;
                const uint32_t tx = (fast ? TILE_BYTES : 0u) + stat_bytes;
                if (tx == 0) {
                    mbar_arrive(&c.full[s]);
                } else {
                    mbar_arrive_expect_tx(&c.full[s], tx);
                    if (fast)
                        bulk_load_hint(buf, in + t * TILE, TILE_BYTES, &c.full[s],
                                       phase == kItemReduce ? keep : drop);
                    if (stat_bytes) {
                        // the 16-byte pairs holding the tile's status words, and E
                        unsigned long long* pair = rec_lo(p.rec, t & ~int64_t(1));
                        bulk_load(&c.stat[s][0], pair, 16, &c.full[s]);
                        bulk_load(&c.stat[s][4], rec_chunk(p.rec, t / K, 0), 16, &c.full[s]);
                        if (!Op::kPacked)
                            bulk_load(&c.stat[s][2], rec_hi(p.rec, t & ~int64_t(1)), 16, &c.full[s]);
                    }
                }
            }
        }
    } else {
        T* out = static_cast<T*>(p.out);
        const bool excl = p.exclusive != 0;
        const uint64_t drop = l2_policy_evict_first();
        int pending = -1;
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (tid == 0) {
                if (pending >= 0) {
                    bulk_wait_read_all();
                    mbar_arrive(&c.empty[pending]);
                    pending = -1;
                }
                c.cflag = mbar_wait_bounded(&c.full[s], use & 1u, role_limit, hdr, epoch, true) ? 1u : 0u;
            }
            named_barrier_sync<CTHREADS>(1);
            if (!c.cflag) break;
            const int64_t t = c.tile_id[s];
            if (t >= num_tiles) break;
            const uint32_t phase = c.phase[s];
            const int cnt = count_of(t);
            const bool tile_fast = p.fast && cnt == TILE;
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
            T x[ITEMS];
            load_items<T, ITEMS, TILE, false>(buf, tid, x);
            if (cnt < TILE) {
                const uint32_t valid = valid_items<ITEMS>(cnt, tid);
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (!((valid >> j) & 1u)) x[j] = T(0);
            }
            bool tf;
            Acc tv;
            thread_reduce<Op, ITEMS, kNoHeads>(x, 0u, tf, tv);

            if (phase == kItemReduce) {
                // ---- first pass: the tile sum ------------------------------
                Acc wv = tv;
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) wv = Op::combine(wv, shfl_down_acc<Op>(wv, d));
                if (lane == 0) c.wtot_v[warp] = wv;
                named_barrier_sync<CTHREADS>(1);
                if (tid == 0) {
                    Acc total = Op::identity();
                    for (int w = 0; w < CWARPS; ++w) total = Op::combine(total, c.wtot_v[w]);
                    publish<Op>(p.rec, t, epoch, kStateA, false, total);
                    mbar_arrive(&c.empty[s]);  // every thread holds its items: stage free
                }
                const int64_t ch = t / K;
                const int64_t first = ch * K;
                const int64_t nch = (num_tiles - first) < K ? (num_tiles - first) : K;
                if (t == first + nch - 1) {
                    // ---- the chunk's sums: in-chunk offsets, chunk prefixes -----
                    named_barrier_sync<CTHREADS>(1);  // thread 0 has read wtot_v
                    Acc sv[kChunkPerThread];
                    const int64_t per = (nch + CTHREADS - 1) / CTHREADS;
                    const int64_t i0 = first + static_cast<int64_t>(tid) * per;
                    Acc run = Op::identity();
                    bool ok = true;
#pragma unroll
                    for (int q = 0; q < kChunkPerThread; ++q) {
                        sv[q] = Op::identity();
                        const int64_t i = i0 + q;
                        if (q < per && i < first + nch) {
                            uint32_t st = kStateX;
                            bool hf;
                            const uint64_t t0 = global_timer_ns();
                            while (true) {
                                read_words<Op>(rec_lo(p.rec, i), rec_hi(p.rec, i), epoch, st, hf,
                                               sv[q]);
                                if (st != kStateX) break;
                                if (global_timer_ns() - t0 > cfg.spin_limit_ns ||
                                    launch_aborted(hdr, epoch)) {
                                    ok = false;
                                    break;
                                }
                                __nanosleep(64);
                                poll_round_fence();
                            }
                            run = Op::combine(run, sv[q]);
                        }
                    }
                    if (!ok) record_timeout(hdr, epoch, t);
                    // block exclusive scan of the thread sums `run`
                    Acc inc = run;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const Acc o = shfl_up_acc<Op>(inc, d);
                        if (lane >= d) inc = Op::combine(o, inc);
                    }
                    if (lane == 31) c.wtot_v[warp] = inc;
                    named_barrier_sync<CTHREADS>(1);
                    Acc ex = shfl_up_acc<Op>(inc, 1);
                    if (lane == 0) ex = Op::identity();
                    Acc wpre = Op::identity();
                    for (int w = 0; w < warp; ++w) wpre = Op::combine(wpre, c.wtot_v[w]);
                    ex = Op::combine(wpre, ex);
                    Acc chunk_total = Op::identity();
                    for (int w = 0; w < CWARPS; ++w) chunk_total = Op::combine(chunk_total, c.wtot_v[w]);
#pragma unroll
                    for (int q = 0; q < kChunkPerThread; ++q) {
                        const int64_t i = i0 + q;
                        if (q < per && i < first + nch) {
                            // the in-chunk offset replaces the sum (state P)
                            publish<Op>(p.rec, i, epoch, kStateP, false, ex);
                            ex = Op::combine(ex, sv[q]);
                        }
                    }
                    named_barrier_sync<CTHREADS>(1);
                    if (tid == 0) {
                        Acc e = Op::identity();
                        if (ch > 0) {
                            uint32_t st = kStateX;
                            bool hf;
                            const uint64_t t0 = global_timer_ns();
                            while (true) {
                                read_words<Op>(rec_chunk(p.rec, ch - 1, 2), rec_chunk(p.rec, ch - 1, 3),
                                               epoch, st, hf, e);
                                if (st == kStateP) break;
                                if (global_timer_ns() - t0 > cfg.spin_limit_ns ||
                                    launch_aborted(hdr, epoch)) {
                                    record_timeout(hdr, epoch, t);
                                    e = Op::identity();
                                    break;
                                }
                                __nanosleep(64);
                                poll_round_fence();
                            }
                        }
                        publish_words<Op>(rec_chunk(p.rec, ch, 0), rec_chunk(p.rec, ch, 1), epoch,
                                          kStateP, false, e);
                        publish_words<Op>(rec_chunk(p.rec, ch, 2), rec_chunk(p.rec, ch, 3), epoch,
                                          kStateP, false, Op::combine(e, chunk_total));
                    }
                }
                continue;
            }

            // ---- second pass: scan the tile with its offset -----------------
            if (tid == 0) {
                // the prefetched copies first; poll the status words themselves
                // only if a copy was taken before its word was published
                const int64_t ch = t / K;
                Acc e, off;
                uint32_t se, so;
                bool hf;
                parse_words<Op>(c.stat[s][4], c.stat[s][5], epoch, se, hf, e);
                parse_words<Op>(c.stat[s][t & 1], c.stat[s][2 + (t & 1)], epoch, so, hf, off);
                const uint64_t t0 = global_timer_ns();
                while (se != kStateP || so != kStateP) {
                    if (global_timer_ns() - t0 > cfg.spin_limit_ns || launch_aborted(hdr, epoch)) {
                        record_timeout(hdr, epoch, t);
                        break;
                    }
                    __nanosleep(64);
                    poll_round_fence();
                    if (se != kStateP)
                        read_words<Op>(rec_chunk(p.rec, ch, 0), rec_chunk(p.rec, ch, 1), epoch, se, hf, e);
                    if (so != kStateP)
                        read_words<Op>(rec_lo(p.rec, t), rec_hi(p.rec, t), epoch, so, hf, off);
                }
                c.prefix_v = Op::combine(e, off);
            }
            bool wf = false;
            Acc wv = tv;
            warp_inclusive_scan<Op, kNoHeads>(wf, wv, lane);
            Acc ev = shfl_up_acc<Op>(wv, 1);
            if (lane == 0) ev = Op::identity();
            if (lane == 31) c.wtot_v[warp] = wv;
            named_barrier_sync<CTHREADS>(1);
            Acc gv = c.prefix_v;
            for (int w = 0; w < warp; ++w) gv = Op::combine(gv, c.wtot_v[w]);
            ev = Op::combine(gv, ev);
            T y[ITEMS];
            thread_outputs<Op, ITEMS, kNoHeads>(x, 0u, ev, excl, y);
            store_items<T, ITEMS, TILE, false>(buf, tid, y);
            if (tile_fast) fence_proxy_async_smem();
            named_barrier_sync<CTHREADS>(1);
            if (tile_fast) {
                if (tid == 0) {
                    bulk_store_hint(out + t * TILE, buf, TILE_BYTES, drop);
                    bulk_commit();
                    pending = s;
                }
            } else {
                for (int i = tid; i < cnt; i += CTHREADS) out[t * TILE + i] = buf[i];
                named_barrier_sync<CTHREADS>(1);
                if (tid == 0) mbar_arrive(&c.empty[s]);
            }
        }
        if (tid == 0 && pending >= 0) {
            bulk_wait_read_all();
            mbar_arrive(&c.empty[pending]);
        }
    }

    __syncthreads();
    if (tid == 0) {
        bulk_wait_all();
        c.clear = finish_launch(hdr, epoch) ? 1u : 0u;
    }
    __syncthreads();
    if (c.clear) clear_status_words(p.rec, p.rec_capacity, tid, blockDim.x);
}

}  // namespace gbscan
