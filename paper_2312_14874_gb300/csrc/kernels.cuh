// kernels.cuh — the tile kernels.
//
// ws_scan_kernel: a chained scan with decoupled look-back, warp-specialised,
//   for the segmented (offset heads) and long-row (row heads, forward and
//   reverse) scans; the plain scans use lookback.cuh, which holds waiting
//   tiles in registers instead of shared memory.
//   loader warp     claims tiles in order (dynamic tile ids) and starts a TMA
//                   bulk copy of each into a free pipeline stage;
//   stage agents    one warp per pipeline stage: as soon as the stage's data
//                   lands, it sums the tile and publishes the sum, then runs the
//                   decoupled look-back and publishes the inclusive prefix.  An
//                   agent never waits for the consumers or for the other
//                   stages, so every tile's aggregate is visible one data
//                   latency after its claim and the look-backs of a block's
//                   tiles run concurrently;
//   consumer warps  scan the tile (thread, warp and block level), add the
//                   tile's exclusive prefix, write the results back over the
//                   stage and store it with one TMA bulk store, then release
//                   the stage to the loader.
//   This is the paper's two-pass partition scheme (Section 2.1, Figure 1)
//   turned inside out: the per-partition sums and the scan of the sums
//   (the `sums` array) run ahead of the per-element pass, and adjacent
//   partitions synchronise through status words instead of a barrier
//   (Section 2.2.1).
//
// two_pass_kernel: the comparison scheme "Accumulate + Prefix Sum"
//   (Section 2.1, Figure 1b): a reduce-only pass writes the tile sums, one block
//   scans them, and a second pass scans every tile with its offset.
#pragma once

#include "tile_common.cuh"

namespace gbscan {

template <class Op, int CWARPS, int STAGES, int TILE>
struct WsCtrl {
    using Acc = typename Op::Acc;
    uint64_t full[STAGES];    // stage data landed (loader arrive + TMA bytes)
    uint64_t ready[STAGES];   // tile prefix known (stage agent arrive)
    uint64_t empty[STAGES];   // stage stored and free (consumer arrive)
    int64_t tile_id[STAGES];
    int64_t seg_lo[STAGES], seg_hi[STAGES], seg_last[STAGES];
    Acc excl_v[STAGES];
    Acc wtot_v[CWARPS];
    uint32_t excl_f[STAGES];
    uint32_t wtot_f[CWARPS];
    uint32_t epoch;
    uint32_t clear;
    uint32_t cflag;
    uint32_t bitmap[TILE / 32 + 2];
};

template <class Op, int CWARPS, int ITEMS, int STAGES>
constexpr int ws_smem_bytes() {
    return STAGES * CWARPS * 32 * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(WsCtrl<Op, CWARPS, STAGES, CWARPS * 32 * ITEMS>));
}

// Threads of a single-pass block: the consumer warps, the loader warp and one
// agent warp per pipeline stage.
template <int CWARPS, int STAGES>
constexpr int ws_threads() {
    return (CWARPS + 1 + STAGES) * 32;
}

template <class Op, int CWARPS, int ITEMS, int STAGES, int HEADS, bool REVERSE, int LB, int MINB>
__global__ void __launch_bounds__((CWARPS + 1 + STAGES) * 32, MINB) ws_scan_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int CTHREADS = CWARPS * 32;
    constexpr int TILE = CTHREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int LOAD_WARP = CWARPS;  // warps CWARPS+1+s: the agent of stage s
    static_assert(ITEMS % VEC == 0, "items per thread must fill 16-byte vectors");
    static_assert(ITEMS <= 32, "head flags are kept in one 32-bit mask");
    static_assert(TILE_BYTES % 16 == 0, "tiles must be 16-byte multiples");
    static_assert(!(REVERSE && HEADS == kOffsetHeads), "offset segments run forward");
    static_assert(STAGES >= 2, "a stage is released one store later: at least two stages");
    static_assert((TILE / VEC) % 32 == 0, "an agent warp reads whole rounds of vectors");
    using CtrlT = WsCtrl<Op, CWARPS, STAGES, TILE>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * TILE_BYTES);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t num_tiles = p.num_tiles;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&c.full[s], HEADS == kOffsetHeads ? 2 : 1);
            mbar_init(&c.ready[s], 1);
            mbar_init(&c.empty[s], 1);
        }
        fence_mbar_init();
        c.epoch = hdr->epoch;
        c.clear = 0;
    }
    __syncthreads();
    const uint32_t epoch = launch_epoch(c.epoch);
    const LookbackCfg cfg = read_lookback_cfg(hdr);
    // pipeline waits outlast a look-back that runs into its own bound
    const uint64_t role_limit = 4 * cfg.spin_limit_ns + 10000000ull;
    auto phys_of = [&](int64_t tile) -> int64_t { return REVERSE ? num_tiles - 1 - tile : tile; };
    auto count_of = [&](int64_t ph) -> int {
        const int64_t rem = p.n - ph * TILE;
        return rem < TILE ? static_cast<int>(rem) : TILE;
    };

    if (warp == LOAD_WARP) {
        // ---- a1: claim tiles in order and start their loads --------------------
        const T* __restrict__ in = static_cast<const T*>(p.in);
        uint32_t fills = 0;  // stage fills made, in order (see drain_fills)
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (use > 0 && !warp_wait(&c.empty[s], (use - 1) & 1u, role_limit, hdr, epoch, lane))
                break;
            long long claimed = 0;
            if (lane == 0) claimed = static_cast<long long>(atomicAdd(&hdr->tile_counter, 1u));
            const int64_t tile = __shfl_sync(0xffffffffu, claimed, 0);
            if (tile >= num_tiles) {
                // no tiles left: mark this stage and the next STAGES-1 (once
                // they are free) with an end sentinel, so that every stage
                // agent and the consumers leave their loops
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    mbar_arrive(&c.full[s]);
                    if (HEADS == kOffsetHeads) mbar_arrive(&c.full[s]);
                }
                ++fills;
                for (uint32_t k2 = k + 1; k2 < k + STAGES; ++k2) {
                    const int s2 = static_cast<int>(k2 % STAGES);
                    const uint32_t use2 = k2 / STAGES;
                    if (use2 > 0 &&
                        !warp_wait(&c.empty[s2], (use2 - 1) & 1u, role_limit, hdr, epoch, lane))
                        break;
                    if (lane == 0) {
                        c.tile_id[s2] = num_tiles;
                        mbar_arrive(&c.full[s2]);
                        if (HEADS == kOffsetHeads) mbar_arrive(&c.full[s2]);
                    }
                    ++fills;
                }
                break;
            }
            const int64_t ph = phys_of(tile);
            const int64_t tb = ph * TILE;
            const int cnt = count_of(ph);
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
            if (p.fast && cnt == TILE) {
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    mbar_arrive_expect_tx(&c.full[s], TILE_BYTES);
                    bulk_load(buf, in + tb, TILE_BYTES, &c.full[s]);
                    // the tile prefetch_tiles claims ahead goes to L2 now, for
                    // whichever block claims it (no claim is made)
                    const int64_t pt = tile + p.prefetch_tiles;
                    if (p.prefetch_tiles > 0 && pt < num_tiles) {
                        const int64_t pph = phys_of(pt);
                        const uint32_t pb =
                            (static_cast<uint32_t>(count_of(pph)) * static_cast<uint32_t>(sizeof(T))) & ~15u;
                        if (pb) bulk_prefetch_l2(in + pph * TILE, pb);
                    }
                }
            } else {
                // ragged or misaligned: the aligned body by one bulk copy where
                // the stage offset allows, the rest by the lanes
                const int off = REVERSE ? TILE - cnt : 0;
                const bool bulk_ok = p.fast && ((off * static_cast<int>(sizeof(T))) & 15) == 0;
                const uint32_t bulk = warp_stage_partial<T>(buf + off, in + tb, cnt, cnt, bulk_ok, Op::pad(), lane);
                __syncwarp();
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    if (bulk) {
                        mbar_arrive_expect_tx(&c.full[s], bulk);
                        bulk_load(buf + off, in + tb, bulk, &c.full[s]);
                    } else {
                        mbar_arrive(&c.full[s]);
                    }
                }
            }
            if constexpr (HEADS == kOffsetHeads) {
                if (lane == 0) {
                    const int64_t lo = static_cast<int64_t>(*rec_aux(p.rec, ph));
                    const int64_t hi = static_cast<int64_t>(*rec_aux(p.rec, ph + 1));
                    c.seg_lo[s] = lo;
                    c.seg_hi[s] = hi;
                    c.seg_last[s] = hi > lo ? p.offsets[hi - 1] : -1;
                    mbar_arrive(&c.full[s]);
                }
            }
            ++fills;
        }
        if (lane == 0) drain_fills<STAGES>(c.full, fills, role_limit, hdr);
    } else if (warp > LOAD_WARP) {
        // ---- a5: stage agent: tile sum as soon as the data lands, look-back --
        const int s = warp - LOAD_WARP - 1;
        for (uint32_t use = 0;; ++use) {
            if (!warp_wait(&c.full[s], use & 1u, role_limit, hdr, epoch, lane)) break;
            const int64_t tile = c.tile_id[s];
            if (tile >= num_tiles) {
                if (lane == 0) mbar_arrive(&c.ready[s]);
                break;
            }
            const int64_t ph = phys_of(tile);
            const int64_t tb = ph * TILE;
            const int cnt = count_of(ph);
            const T* buf = reinterpret_cast<const T*>(smem + s * TILE_BYTES);
            // The tile's aggregate is (head in tile, sum after its last head).
            int a = 0;  // logical start of the summed range
            bool f = false;
            if constexpr (HEADS == kOffsetHeads) {
                const int64_t pos = c.seg_last[s] - tb;
                if (c.seg_last[s] >= 0 && pos >= 0 && pos < cnt) {
                    a = static_cast<int>(pos);
                    f = true;
                }
            } else if constexpr (HEADS == kRowHeads) {
                const int64_t cols = p.cols;
                if constexpr (!REVERSE) {
                    const int64_t m = ((tb + cnt - 1) / cols) * cols;  // last row start
                    if (m >= tb) {
                        a = static_cast<int>(m - tb);
                        f = true;
                    }
                } else {
                    const int64_t q = (tb / cols) * cols + cols - 1;  // first row end
                    if (q <= tb + cnt - 1) {
                        a = static_cast<int>(tb + cnt - 1 - q);
                        f = true;
                    }
                }
            }
            const int lo = REVERSE ? TILE - cnt : a;
            const int hi = REVERSE ? TILE - a : cnt;
            Acc v = Op::identity();
            if (lo == 0 && hi == TILE) {
                // whole tile: 16-byte reads, consecutive lanes on consecutive
                // vectors, SUMU independent accumulators so that the reads of a
                // batch are in flight together
                constexpr int PER_LANE = TILE / VEC / 32;
                constexpr int SUMU = PER_LANE < 8 ? PER_LANE : 8;
                const uint4* v4 = reinterpret_cast<const uint4*>(buf) + lane;
                Acc part[SUMU];
#pragma unroll
                for (int u = 0; u < SUMU; ++u) part[u] = Op::identity();
#pragma unroll
                for (int q0 = 0; q0 < PER_LANE; q0 += SUMU) {
                    uint4 w[SUMU];
#pragma unroll
                    for (int u = 0; u < SUMU; ++u)
                        if (q0 + u < PER_LANE) w[u] = v4[(q0 + u) * 32];
#pragma unroll
                    for (int u = 0; u < SUMU; ++u) {
                        if (q0 + u < PER_LANE) {
                            const T* e = reinterpret_cast<const T*>(&w[u]);
#pragma unroll
                            for (int j = 0; j < VEC; ++j) Op::accumulate(part[u], e[j]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < SUMU; ++u) v = combine_local<Op>(v, part[u]);
            } else {
                for (int i = lo + lane; i < hi; i += 32) Op::accumulate(v, buf[i]);
            }
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) v = combine_local<Op>(v, shfl_down_acc<Op>(v, d));
            v = shfl_idx_acc<Op>(v, 0);
            if (lane == 0) publish_aggregate<Op>(p.rec, tile, epoch, cfg, f, v);
            bool ef;
            Acc ev;
            lookback<Op, HEADS, LB>(p.rec, hdr, tile, epoch, cfg, f, v, lane, ef, ev);
            if (lane == 0) {
                c.excl_v[s] = ev;
                c.excl_f[s] = ef ? 1u : 0u;
                mbar_arrive(&c.ready[s]);
            }
        }
    } else {
        // ---- a2-a4, a6: scan the tile, add its prefix, store ------------------
        T* out = static_cast<T*>(p.out);
        const bool excl = p.exclusive != 0;
        int pending = -1;  // stage whose TMA store may still be reading shared memory
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (tid == 0) {
                // release the stage of the previous bulk store once it has read
                // shared memory (before waiting: the loader may need that stage
                // to make progress)
                if (pending >= 0) {
                    bulk_wait_read_all();
                    mbar_arrive(&c.empty[pending]);
                    pending = -1;
                }
                // thread 0 alone observes the tile prefix (ready) and the
                // bulk-copied data (full) with the bound; the named barrier then
                // orders its view of memory before every consumer's accesses and
                // tells all of them whether to go on, so they leave together
                bool ok = mbar_wait_bounded(&c.ready[s], use & 1u, role_limit, hdr, epoch, true);
                ok = ok && mbar_wait_bounded(&c.full[s], use & 1u, role_limit, hdr, epoch, true);
                c.cflag = ok ? 1u : 0u;
            }
            named_barrier_sync<CTHREADS>(1);
            if (!c.cflag) break;
            const int64_t tile = c.tile_id[s];
            if (tile >= num_tiles) break;
            const int64_t ph = phys_of(tile);
            const int64_t tb = ph * TILE;
            const int cnt = count_of(ph);
            const bool tile_fast = p.fast && cnt == TILE;
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);

            T x[ITEMS];
            load_items<T, ITEMS, TILE, REVERSE>(buf, tid, x);
            uint32_t valid = 0xffffffffu;
            if (cnt < TILE) {
                valid = valid_items<ITEMS>(cnt, tid);
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (!((valid >> j) & 1u)) x[j] = Op::pad();
            }
            uint32_t hm = 0;
            if constexpr (HEADS == kOffsetHeads) {
                for (int i = tid; i < TILE / 32 + 2; i += CTHREADS) c.bitmap[i] = 0u;
                named_barrier_sync<CTHREADS>(1);
                const int64_t s_lo = c.seg_lo[s], s_hi = c.seg_hi[s];
                for (int64_t sg = s_lo + tid; sg < s_hi; sg += CTHREADS) {
                    const int64_t pos = p.offsets[sg] - tb;
                    if (pos >= 0 && pos < cnt) atomicOr(&c.bitmap[pos >> 5], 1u << (pos & 31));
                }
                named_barrier_sync<CTHREADS>(1);
                const int b = tid * ITEMS;
                const uint32_t bits = __funnelshift_r(c.bitmap[b >> 5], c.bitmap[(b >> 5) + 1], b & 31);
                hm = (ITEMS == 32 ? bits : (bits & ((1u << ITEMS) - 1u))) & valid;
            } else if constexpr (HEADS == kRowHeads) {
                hm = row_heads<ITEMS, REVERSE>(tb, cnt, p.cols, tid) & valid;
            }

            bool tf;
            Acc tv;
            const bool wh = HEADS != kNoHeads && __any_sync(0xffffffffu, hm != 0u);
            thread_reduce_w<Op, ITEMS, HEADS>(x, hm, wh, tf, tv);
            bool wf = tf;
            Acc wv = tv;
            warp_inclusive_scan_w<Op, HEADS>(wh, wf, wv, lane);
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
            named_barrier_sync<CTHREADS>(1);
            // everything before this thread's first item: tile prefix, then the
            // warps before this one, then the lanes before this one
            bool gf = c.excl_f[s] != 0;
            Acc gv = c.excl_v[s];
            for (int w = 0; w < warp; ++w) {
                if (HEADS != kNoHeads) {
                    bool f2 = c.wtot_f[w] != 0;
                    Acc v2 = c.wtot_v[w];
                    seg_combine<Op>(gf, gv, f2, v2);
                    gf = f2;
                    gv = v2;
                } else {
                    gv = combine_local<Op>(gv, c.wtot_v[w]);
                }
            }
            if (HEADS != kNoHeads)
                seg_combine<Op>(gf, gv, ef, ev);
            else
                ev = combine_local<Op>(gv, ev);
            T y[ITEMS];
            thread_outputs_w<Op, ITEMS, HEADS>(x, hm, wh, ev, excl, y);
            store_items<T, ITEMS, TILE, REVERSE>(buf, tid, y);
            if (tile_fast) fence_proxy_async_smem();
            named_barrier_sync<CTHREADS>(1);
            if (tile_fast) {
                if (tid == 0) {
                    bulk_store(out + tb, buf, TILE_BYTES);
                    bulk_commit();
                    pending = s;  // released at the top of the next iteration
                }
            } else {
                const int off = REVERSE ? TILE - cnt : 0;
                for (int i = tid; i < cnt; i += CTHREADS) out[tb + i] = buf[off + i];
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

// ---------------------------------------------------------------------------
// Two-pass comparison kernel (no segments, forward).  Tile k of block b is
// tile b + k * gridDim.x.  kReduce: rec aux[tile] = tile sum.  kScanOffset:
// scan the tile starting from aux[tile] (the scanned tile sums).
// ---------------------------------------------------------------------------

template <class Op, int STAGES, int NWARPS>
struct TpCtrl {
    using Acc = typename Op::Acc;
    uint64_t mbar[STAGES];
    Acc wtot_v[2][NWARPS];
    uint32_t cflag;  // thread 0 -> block: the stage wait succeeded
};

template <class Op, int THREADS, int ITEMS, int STAGES>
constexpr int tp_smem_bytes() {
    return STAGES * THREADS * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(TpCtrl<Op, STAGES, THREADS / 32>));
}

template <class Op, int THREADS, int ITEMS, int STAGES, int MODE>
__global__ void __launch_bounds__(THREADS) two_pass_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int TILE = THREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int NWARPS = THREADS / 32;
    static_assert(MODE == kReduce || MODE == kScanOffset, "two-pass modes only");
    using CtrlT = TpCtrl<Op, STAGES, NWARPS>;
    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * TILE_BYTES);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T* __restrict__ in = static_cast<const T*>(p.in);
    T* out = static_cast<T*>(p.out);
    const int64_t num_tiles = p.num_tiles;
    // The blocks of a two-pass launch never wait for one another: the only
    // waits are a block's own stage loads.  A stage wait that runs out records
    // GBSCAN_ERR_TIMEOUT and ends the block's loop at once (its remaining
    // tiles are not computed, and the error tells the host so); the block
    // then waits, again bounded, for the loads it still has in flight, so a
    // launch lasts at most its normal time plus two spin limits.  A stage
    // whose wait failed is never re-armed: arming it again while the late
    // load's bytes are still owed to the old phase would leave the barrier's
    // phase and the expected parity out of step, and every later wait of the
    // block would then run to its bound.
    const LookbackCfg cfg = read_lookback_cfg(p.hdr);
    const uint64_t limit_ns = cfg.spin_limit_ns;
    uint32_t armed = 0;  // thread 0: stages with a load issued and not yet consumed

    auto tile_of = [&](uint32_t k) -> int64_t {
        return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(k) * gridDim.x;
    };
    auto count_of = [&](int64_t t) -> int {
        const int64_t rem = p.n - t * TILE;
        return rem < TILE ? static_cast<int>(rem) : TILE;
    };
    auto issue = [&](uint32_t k) {
        const int64_t t = tile_of(k);
        if (t < num_tiles && p.fast && count_of(t) == TILE) {
            if (t == cfg.drop_tile) return;  // test hook: this tile's stage never fills
            const int s = static_cast<int>(k % STAGES);
            mbar_arrive_expect_tx(&c.mbar[s], TILE_BYTES);
            bulk_load(smem + s * TILE_BYTES, in + t * TILE, TILE_BYTES, &c.mbar[s]);
            armed |= 1u << s;
        }
    };
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&c.mbar[s], 1);
        fence_mbar_init();
        for (int s = 0; s < STAGES; ++s) issue(static_cast<uint32_t>(s));
    }
    __syncthreads();
    uint32_t phase = 0;  // per stage: the parity of the next phase to wait for
    bool refill_pending = false;
    for (uint32_t k = 0;; ++k) {
        const int64_t tile = tile_of(k);
        if (tile >= num_tiles) break;
        const int s = static_cast<int>(k % STAGES);
        const int cnt = count_of(tile);
        const bool tile_fast = p.fast && cnt == TILE;
        T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
        if (tile_fast) {
            // one thread observes the phase; the block barrier passes its view
            // of the bulk-copied data (and the outcome) on to every thread
            if (tid == 0) {
                const bool ok =
                    mbar_wait_bounded(&c.mbar[s], (phase >> s) & 1u, limit_ns, p.hdr, 0, false);
                if (ok)
                    armed &= ~(1u << s);
                else
                    record_error(p.hdr, GBSCAN_ERR_TIMEOUT, tile);
                c.cflag = ok ? 1u : 0u;
            }
            __syncthreads();
            if (!c.cflag) break;
            phase ^= 1u << s;
        } else {
            for (int i = tid; i < cnt; i += THREADS) buf[i] = in[tile * TILE + i];
            __syncthreads();
        }
        T x[ITEMS];
        load_items<T, ITEMS, TILE, false>(buf, tid, x);
        uint32_t valid = 0xffffffffu;
        if (cnt < TILE) {
            valid = valid_items<ITEMS>(cnt, tid);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if (!((valid >> j) & 1u)) x[j] = Op::pad();
        }
        if (MODE == kScanOffset && refill_pending && tid == 0) {
            // the previous stage's store has had this block's whole load to
            // read shared memory; refill it
            bulk_wait_read_all();
            issue(k - 1 + STAGES);
            refill_pending = false;
        }
        bool tf;
        Acc tv;
        thread_reduce<Op, ITEMS, kNoHeads>(x, 0u, tf, tv);
        bool wf = false;
        Acc wv = tv;
        warp_inclusive_scan<Op, kNoHeads>(wf, wv, lane);
        if (lane == 31) c.wtot_v[k & 1][warp] = wv;
        __syncthreads();
        if constexpr (MODE == kReduce) {
            if (tid == 0) issue(k + STAGES);  // every thread holds its items: stage free
            if (warp == 0) {
                Acc b = lane < NWARPS ? c.wtot_v[k & 1][lane] : Op::identity();
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) b = combine_local<Op>(b, shfl_down_acc<Op>(b, d));
                if (lane == 0) *rec_aux(p.rec, tile) = static_cast<unsigned long long>(Op::to_bits(b));
            }
            if (STAGES == 1) __syncthreads();
            continue;
        } else {
            Acc gv = Op::from_bits(static_cast<typename Op::Bits>(*rec_aux(p.rec, tile)));
            for (int w = 0; w < warp; ++w) gv = combine_local<Op>(gv, c.wtot_v[k & 1][w]);
            Acc ev = shfl_up_acc<Op>(wv, 1);
            if (lane == 0) ev = Op::identity();
            ev = combine_local<Op>(gv, ev);
            T y[ITEMS];
            thread_outputs<Op, ITEMS, kNoHeads>(x, 0u, ev, p.exclusive != 0, y);
            store_items<T, ITEMS, TILE, false>(buf, tid, y);
            if (tile_fast) fence_proxy_async_smem();
            __syncthreads();
            if (tile_fast) {
                if (tid == 0) {
                    bulk_store(out + tile * TILE, buf, TILE_BYTES);
                    bulk_commit();
                }
            } else {
                for (int i = tid; i < cnt; i += THREADS) out[tile * TILE + i] = buf[i];
                __syncthreads();
            }
            if (STAGES == 1) {
                if (tid == 0) {
                    bulk_wait_read_all();
                    issue(k + 1);
                }
                __syncthreads();
            } else {
                refill_pending = true;
            }
        }
    }
    if (tid == 0) {
        // loads still in flight (only after a failed wait) must land before
        // the block's shared memory is given up
        for (int s = 0; s < STAGES; ++s)
            if ((armed >> s) & 1u) mbar_wait_bounded(&c.mbar[s], (phase >> s) & 1u, limit_ns, p.hdr, 0, false);
        bulk_wait_all();
    }
}

// Exclusive scan of the two-pass tile sums (aux fields), one block.
template <class Op, int THREADS>
__global__ void __launch_bounds__(THREADS) scan_tile_sums_kernel(unsigned long long* rec,
                                                                 int64_t num_tiles) {
    using Acc = typename Op::Acc;
    constexpr int NWARPS = THREADS / 32;
    __shared__ Acc wsum[NWARPS];
    __shared__ Acc carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Acc carry = Op::identity();
    for (int64_t base = 0; base < num_tiles; base += THREADS) {
        const int64_t i = base + tid;
        const Acc v = i < num_tiles ? Op::from_bits(static_cast<typename Op::Bits>(*rec_aux(rec, i)))
                                    : Op::identity();
        Acc inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Acc o = shfl_up_acc<Op>(inc, d);
            if (lane >= d) inc = combine_local<Op>(o, inc);
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            Acc w = lane < NWARPS ? wsum[lane] : Op::identity();
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const Acc o = shfl_up_acc<Op>(w, d);
                if (lane >= d) w = combine_local<Op>(o, w);
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
        ex = combine_local<Op>(wsum[warp], ex);
        ex = Op::combine(carry, ex);
        if (i < num_tiles) *rec_aux(rec, i) = static_cast<unsigned long long>(Op::to_bits(ex));
        carry = carry_s;
        __syncthreads();
    }
}

}  // namespace gbscan
