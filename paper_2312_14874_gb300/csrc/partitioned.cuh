// partitioned.cuh — the cache-friendly partitioned scan.
//
// The paper's central proposal (Section 2.2, Figure 2): split the data into
// cache-sized partitions and make both passes of the two-pass scheme over one
// partition before moving on, so that the second pass reads from cache instead
// of memory; keep two `sums` arrays so that the second pass of iteration k
// overlaps the first pass of iteration k+1 (Section 2.2.1).  Here the cache is
// the GPU's L2 (129 MB): a chunk is a run of chunk_tiles tiles of a few MB (8 MiB
// by default), and one persistent launch processes a work list in which the
// second pass (scan) of chunk c is interleaved with the first pass (reduce,
// "Accumulate") of chunk c+lag (4 by default: the scan of chunk c's tile sums
// has several slots of work to finish in), e.g. with a lag of two:
//
//   R(0) R(1) | S(0) R(2) S(0) R(2) ... | S(1) R(3) ... | ... | S(C-1)
//
// R item:  TMA-load the tile with L2 evict-last priority (it will be read again),
//          sum it, publish the sum in the tile's status word.  The last R item of
//          a chunk hands the chunk to its block's scanner warp, which scans the
//          chunk's tile sums (the per-partition `sums` array): waits until all
//          are published, publishes each tile's exclusive offset within the
//          chunk in the tile's status word, and chains the chunk prefixes (E, P)
//          from the previous chunk.
// S item:  TMA-load the tile again (from L2, evict-first) together with the two
//          status words it needs (its in-chunk offset and the chunk prefix E),
//          which are self-validating (epoch-tagged), so no global round trip is
//          left on the scan's path; scan, store with a TMA bulk store.
// The scanner warp runs beside the block's consumers, so no item waits behind
// a chunk scan.
//
// There is no per-tile dependency chain: a tile's S item waits only for its
// chunk's prefix, published once per chunk, which is why this scheme comes
// close to copy bandwidth where a per-tile chained scan is bound by status
// round trips.  Forward scans, plain or segmented (HEADS = kOffsetHeads: a
// head bitmap travels with each tile and the chunk scan uses the segmented
// operator).
#pragma once

#include "tile_common.cuh"

namespace gbscan {

enum : uint32_t { kItemReduce = 0, kItemScan = 1 };

// The constants of the work list for one launch: num_tiles tiles in chunks of
// K, the scan of chunk c interleaved with the reduction of chunk c + lag
// (lag >= 1).  Every count fits 32 bits (fewer than 2^31 tiles).
struct PtOrder {
    uint32_t K, lag, C, nlast, npre, F;
};

__device__ __forceinline__ PtOrder make_order(int64_t num_tiles, int64_t K, int64_t lag) {
    PtOrder o;
    o.K = static_cast<uint32_t>(K);
    o.lag = static_cast<uint32_t>(lag);
    o.C = static_cast<uint32_t>((num_tiles + K - 1) / K);
    o.nlast = static_cast<uint32_t>(num_tiles - static_cast<int64_t>(o.C - 1) * K);
    const uint32_t pre = o.lag < o.C ? o.lag : o.C;
    o.npre = pre < o.C ? pre * o.K : (o.C - 1) * o.K + o.nlast;
    o.F = o.C > o.lag + 1 ? o.C - 1 - o.lag : 0;  // slots with both parts full
    return o;
}

// Work item w of the list above:
//   R(0) .. R(lag-1) in tile order, then for each chunk c the slot
//   S(c) / R(c+lag) alternating (S first) while both have items, then the rest.
__device__ __forceinline__ void partitioned_item(uint32_t w, const PtOrder& o, uint32_t& phase,
                                                 int64_t& tile) {
    if (w < o.npre) {
        phase = kItemReduce;
        tile = w;
        return;
    }
    w -= o.npre;
    const uint32_t K2 = 2 * o.K;
    if (w < o.F * K2) {
        const uint32_t c = w / K2, off = w - c * K2, j = off >> 1;
        phase = (off & 1) ? kItemReduce : kItemScan;
        tile = static_cast<int64_t>((off & 1) ? c + o.lag : c) * o.K + j;
        return;
    }
    w -= o.F * K2;
    uint32_t c = o.F;
    if (o.C >= o.lag + 1) {
        // slot F: S(F) (K items) alternating with R(C-1) (nlast items)
        if (w < 2 * o.nlast) {
            const uint32_t j = w >> 1;
            phase = (w & 1) ? kItemReduce : kItemScan;
            tile = static_cast<int64_t>((w & 1) ? o.C - 1 : o.F) * o.K + j;
            return;
        }
        if (w < o.K + o.nlast) {
            phase = kItemScan;
            tile = static_cast<int64_t>(o.F) * o.K + o.nlast + (w - 2 * o.nlast);
            return;
        }
        w -= o.K + o.nlast;
        c = o.F + 1;
    }
    phase = kItemScan;  // the remaining slots hold scans only, in tile order
    tile = static_cast<int64_t>(c) * o.K + w;
}

template <class Op, int CWARPS, int STAGES, int TILE, int HEADS>
struct PtCtrl {
    using Acc = typename Op::Acc;
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int64_t tile_id[STAGES];
    uint32_t phase[STAGES];
    // per stage, for a scan item: copies of the 16-byte unit holding the
    // tile's status word (or pair) and of the chunk's E pair, brought in by
    // the loader's bulk copies
    alignas(16) unsigned long long stat[STAGES][6];
    // segmented scans: per stage, the tile's slice of the head bitmap (bit i =
    // element i starts a segment), then zero words for the reads past its end
    alignas(16) uint32_t bits[HEADS != kNoHeads ? STAGES : 1][HEADS != kNoHeads ? TILE / 32 + 4 : 4];
    alignas(16) Acc wtot_v[CWARPS];
    alignas(16) uint32_t wtot_f[CWARPS];
    Acc prefix_v;
    uint64_t scan_req;   // consumers -> scanner warp: a chunk to scan (or -1: stop)
    uint64_t scan_idle;  // scanner warp -> consumers: the request is done
    int64_t scan_chunk;
    uint32_t epoch;
    uint32_t clear;
    uint32_t cflag;
    unsigned int claim_sink;
};

template <class Op, int CWARPS, int ITEMS, int STAGES, int HEADS>
constexpr int pt_smem_bytes() {
    return STAGES * CWARPS * 32 * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(PtCtrl<Op, CWARPS, STAGES, CWARPS * 32 * ITEMS, HEADS>));
}

// Consumer warps, the loader warp and the chunk scanner warp.
template <int CWARPS>
constexpr int pt_threads() {
    return (CWARPS + 2) * 32;
}

// Work items a loader claims with one atomic.
constexpr int kClaim = 2;

// Most tiles a chunk may have.
constexpr int kMaxChunkTiles = 1 << 16;

// Publishes tile t's sum (state A; with segments, the head flag and the sum
// after the tile's last head) for the chunk scan, with the test hooks of
// the workspace header: the dropped tile never publishes, and a pseudo-random
// sleep of up to delay_max ns precedes every publication (race stress).
template <class Op>
__device__ __forceinline__ void publish_sum_hooked(unsigned long long* rec, int64_t t, uint32_t epoch,
                                                   const LookbackCfg& cfg, bool head,
                                                   typename Op::Acc sum) {
    if (t == cfg.drop_tile) return;
    if (cfg.delay_max) {
        const uint32_t dly = mix32(static_cast<uint64_t>(t) * 0x9e3779b97f4a7c15ull) % (cfg.delay_max + 1);
        if (dly) __nanosleep(dly);
    }
    publish<Op>(rec, t, epoch, kStateA, head, sum);
}

// Issues the reads of R status-word rows (32 tiles each, row q of the batch
// holding tiles r0 + 32q .. r0 + 32q + 31 of the chunk that starts at tile
// `first`); tiles at or past nch are left as zero words.
template <class Op, int R>
__device__ __forceinline__ void chunk_rows_issue(const unsigned long long* rec, int64_t first,
                                                 int64_t nch, int64_t r0, int lane,
                                                 unsigned long long (&w0)[R],
                                                 unsigned long long (&w1)[R]) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int64_t i = r0 + q * 32 + lane;
        w0[q] = 0ull;
        w1[q] = 0ull;
        if (i < nch) {
            const unsigned long long* w = rec_tile<Op>(const_cast<unsigned long long*>(rec), first + i);
            if constexpr (Op::kPacked)
                w0[q] = ld_poll_u64(w);
            else
                ld_poll_pair(w, w0[q], w1[q]);
        }
    }
}

// The scan of one chunk's tile sums (the partition's `sums` array), by one
// warp: waits until every tile of chunk ch has published its sum, replaces
// each sum by the tile's exclusive offset within the chunk (state P), then
// chains the chunk prefixes: E(ch) = P(ch-1) (the sum of all earlier chunks)
// and P(ch) = E(ch) + the chunk's total.  The sums are read in batches of R
// rows of 32 consecutive tiles (the next batch's reads go out before the
// current batch is scanned); the rows of a batch are scanned independently
// with warp shuffles, and a running carry joins them in the publishing loop.
// Segmented scans carry (head flag, value) pairs through the same steps with
// the segmented operator: a value after a head does not add what came before.
template <class Op, int HEADS>
__device__ void chunk_scan_warp(const Params& p, int64_t ch, Header* hdr, uint32_t epoch,
                                const LookbackCfg& cfg, int lane) {
    using Acc = typename Op::Acc;
    constexpr int R = 8;
    const int64_t K = p.chunk_tiles;
    const int64_t first = ch * K;
    const int64_t nch = (p.num_tiles - first) < K ? (p.num_tiles - first) : K;
    Acc carry = Op::identity();
    bool carry_f = false;
    bool ok = true;
    unsigned long long w0[R], w1[R];
    chunk_rows_issue<Op, R>(p.rec, first, nch, 0, lane, w0, w1);
    for (int64_t r0 = 0; r0 < nch; r0 += 32 * R) {
        Acc v[R];
        uint32_t st[R];
        bool hfl[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            v[q] = Op::identity();
            hfl[q] = false;
            st[q] = kStateA;  // entries past the chunk count as published
            if (r0 + q * 32 + lane < nch) parse_words<Op>(w0[q], w1[q], epoch, st[q], hfl[q], v[q]);
        }
        if (r0 + 32 * R < nch) chunk_rows_issue<Op, R>(p.rec, first, nch, r0 + 32 * R, lane, w0, w1);
        const uint64_t t0 = global_timer_ns();
        while (true) {
            bool missing = false;
#pragma unroll
            for (int q = 0; q < R; ++q) missing |= st[q] == kStateX;
            if (!missing) break;
            if (global_timer_ns() - t0 > cfg.spin_limit_ns || launch_aborted(hdr, epoch)) {
                ok = false;
                break;
            }
            __nanosleep(64);
            poll_round_fence();
#pragma unroll
            for (int q = 0; q < R; ++q) {
                if (st[q] == kStateX) {
                    const int64_t i = first + r0 + q * 32 + lane;
                    read_words<Op>(rec_tile<Op>(p.rec, i), epoch, st[q], hfl[q], v[q]);
                }
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        // row scans (independent of one another): ex = exclusive within the
        // row, v = the row's total
        Acc ex[R];
        bool exf[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            bool f = hfl[q];
            Acc inc = v[q];
            warp_inclusive_scan<Op, HEADS>(f, inc, lane);
            exf[q] = false;
            if constexpr (HEADS != kNoHeads) exf[q] = __shfl_up_sync(0xffffffffu, f ? 1 : 0, 1) != 0;
            ex[q] = shfl_up_acc<Op>(inc, 1);
            if (lane == 0) {
                exf[q] = false;
                ex[q] = Op::identity();
            }
            v[q] = shfl_idx_acc<Op>(inc, 31);
            if constexpr (HEADS != kNoHeads) hfl[q] = __shfl_sync(0xffffffffu, f ? 1 : 0, 31) != 0;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int64_t i = r0 + q * 32 + lane;
            // the in-chunk offset replaces the sum (state P)
            bool of = exf[q];
            Acc ov = ex[q];
            if constexpr (HEADS != kNoHeads)
                seg_combine<Op>(carry_f, carry, of, ov);
            else
                ov = Op::combine(carry, ov);
            if (i < nch) publish<Op>(p.rec, first + i, epoch, kStateP, of, ov);
            if constexpr (HEADS != kNoHeads) {
                bool f2 = hfl[q];
                Acc v2 = v[q];
                seg_combine<Op>(carry_f, carry, f2, v2);
                carry_f = f2;
                carry = v2;
            } else {
                carry = Op::combine(carry, v[q]);
            }
        }
    }
    if (lane == 0) {
        if (!ok) {
            record_timeout(hdr, epoch, first);
            return;
        }
        Acc e = Op::identity();
        bool ef = false;
        if (ch == 0 && p.carry_in != nullptr) {
            // a scan that continues an earlier one: everything before element 0
            e = Op::lift(*static_cast<const typename Op::T*>(p.carry_in));
        } else if (ch > 0) {
            uint32_t st = kStateX;
            const uint64_t t0 = global_timer_ns();
            while (true) {
                read_words<Op>(rec_chunk(p.rec, ch - 1, 2), epoch, st, ef, e);
                if (st == kStateP) break;
                if (global_timer_ns() - t0 > cfg.spin_limit_ns || launch_aborted(hdr, epoch)) {
                    record_timeout(hdr, epoch, first);
                    return;
                }
                __nanosleep(64);
                poll_round_fence();
            }
        }
        if (cfg.delay_max) {
            const uint32_t dly = mix32(static_cast<uint64_t>(ch) * 0x2545f4914f6cdd1dull) % (cfg.delay_max + 1);
            if (dly) __nanosleep(dly);
        }
        publish_words<Op>(rec_chunk(p.rec, ch, 0), epoch, kStateP, ef, e);
        bool pf = carry_f;
        Acc pv = carry;
        if constexpr (HEADS != kNoHeads)
            seg_combine<Op>(ef, e, pf, pv);
        else
            pv = Op::combine(e, carry);
        publish_words<Op>(rec_chunk(p.rec, ch, 2), epoch, kStateP, pf, pv);
        // the last chunk's inclusive prefix is the total (stream compaction:
        // the number of elements kept)
        if (p.total_out != nullptr && first + nch == p.num_tiles)
            *p.total_out = static_cast<unsigned long long>(Op::to_bits(pv));
    }
}

template <class Op, int CWARPS, int ITEMS, int STAGES, int MINB, int HEADS>
__global__ void __launch_bounds__((CWARPS + 2) * 32, MINB) partitioned_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int CTHREADS = CWARPS * 32;
    constexpr int TILE = CTHREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int LOAD_WARP = CWARPS;
    constexpr int SCAN_WARP = CWARPS + 1;
    static_assert(STAGES >= 2, "a stage is released one store later: at least two stages");
    static_assert(HEADS == kNoHeads || HEADS == kOffsetHeads, "plain or offset segments");
    static_assert(HEADS == kNoHeads || (TILE / 8) % 16 == 0, "bitmap slices are bulk copies");
    static_assert(ITEMS <= 32, "head flags are kept in one 32-bit mask");
    constexpr uint32_t BITS_BYTES = HEADS != kNoHeads ? TILE / 8 : 0;
    using CtrlT = PtCtrl<Op, CWARPS, STAGES, TILE, HEADS>;

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
        mbar_init(&c.scan_req, 1);
        mbar_init(&c.scan_idle, 1);
        fence_mbar_init();
        if constexpr (HEADS != kNoHeads)
            for (int s = 0; s < STAGES; ++s)
                for (int w = TILE / 32; w < TILE / 32 + 4; ++w) c.bits[s][w] = 0u;
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
        // The loader claims kClaim consecutive items per atomic and keeps the
        // next batch's claim in flight while it issues the current batch, so
        // that the atomic's round trip (about a microsecond under load) neither
        // paces the loads (one atomic per item would) nor sits between a stage
        // coming free and its next load.
        const PtOrder order = make_order(num_tiles, K, p.chunk_lag);
        unsigned int cur = 0, nxt = 0;
        if (lane == 0) {
            cur = atomicAdd(&hdr->tile_counter, static_cast<unsigned int>(kClaim));
            nxt = atomicAdd(&hdr->tile_counter, static_cast<unsigned int>(kClaim));
        }
        int in_batch = 0;
        uint32_t fills = 0;  // stage fills made, in order (see drain_fills)
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (use > 0 && !warp_wait(&c.empty[s], (use - 1) & 1u, role_limit, hdr, epoch, lane))
                break;
            const int64_t w = static_cast<int64_t>(__shfl_sync(0xffffffffu, cur, 0)) + in_batch;
            if (++in_batch == kClaim) {
                in_batch = 0;
                if (lane == 0) {
                    cur = nxt;
                    nxt = atomicAdd(&hdr->tile_counter, static_cast<unsigned int>(kClaim));
                }
            }
            ++fills;
            if (w >= num_items) {
                // end (or an aborted launch: poisoned claims): a sentinel
                // stage ends the consumers' loop
                if (lane == 0) {
                    c.tile_id[s] = num_tiles;
                    mbar_arrive(&c.full[s]);
                }
                break;
            }
            uint32_t phase;
            int64_t t;
            partitioned_item(static_cast<uint32_t>(w), order, phase, t);
            const int cnt = count_of(t);
            const bool fast = p.fast && cnt == TILE;
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
            // a whole aligned tile moves by one bulk copy; a ragged one by a
            // bulk copy of its aligned body and the lanes for the rest
            uint32_t body = fast ? static_cast<uint32_t>(TILE_BYTES) : 0u;
            if (!fast) {
                body = warp_stage_partial<T>(buf, in + t * TILE, cnt, cnt, p.fast, Op::pad(), lane);
                __syncwarp();
            }
            if (lane == 0) {
                c.tile_id[s] = t;
                c.phase[s] = phase;
                const uint32_t stat_bytes = phase == kItemScan ? 32u : 0u;
                const uint32_t tx = body + stat_bytes + BITS_BYTES;
                if (tx == 0) {
                    mbar_arrive(&c.full[s]);
                } else {
                    mbar_arrive_expect_tx(&c.full[s], tx);
                    if (body)
                        bulk_load_hint(buf, in + t * TILE, body, &c.full[s],
                                       phase == kItemReduce ? keep : drop);
                    // a reduce item's copy is the tile's first read: the tile
                    // prefetch_tiles ahead goes to L2 now, so that its reduce
                    // item's copy comes from L2 (no item is claimed for it)
                    const int64_t pt = t + p.prefetch_tiles;
                    if (phase == kItemReduce && p.prefetch_tiles > 0 && p.fast && pt < num_tiles) {
                        const uint32_t pbytes =
                            (static_cast<uint32_t>(count_of(pt)) * static_cast<uint32_t>(sizeof(T))) & ~15u;
                        if (pbytes) bulk_prefetch_l2(in + pt * TILE, pbytes);
                    }
                    if constexpr (HEADS != kNoHeads)
                        bulk_load(&c.bits[s][0], p.bitmap + t * (TILE / 32), BITS_BYTES, &c.full[s]);
                    if (stat_bytes) {
                        // the 16-byte unit holding the tile's status word (its
                        // pair for 8-byte accumulators), and the chunk's E pair
                        unsigned long long* unit =
                            Op::kPacked ? rec_tile<Op>(p.rec, t & ~int64_t(1)) : rec_tile<Op>(p.rec, t);
                        bulk_load(&c.stat[s][0], unit, 16, &c.full[s]);
                        const uint32_t ch = static_cast<uint32_t>(t) / order.K;
                        bulk_load(&c.stat[s][4], rec_chunk(p.rec, ch, 0), 16, &c.full[s]);
                    }
                }
            }
        }
        // the claims still in flight must land before this block reports itself
        // done (the last block to finish resets the counter): the store waits
        // for the atomics' results
        if (lane == 0) {
            *static_cast<volatile unsigned int*>(&c.claim_sink) = cur ^ nxt;
            drain_fills<STAGES>(c.full, fills, role_limit, hdr);
        }
    } else if (warp < CWARPS) {
        T* out = static_cast<T*>(p.out);
        const bool excl = p.exclusive != 0;
        const uint64_t drop = l2_policy_evict_first();
        // The segmented kernel spreads its serial duties over lanes of three
        // warps, so that they overlap instead of adding up on the path every
        // item waits for: thread 0 waits for the stages and reads a scan
        // item's prefixes, kPubTid publishes tile sums and hands chunks to the
        // scanner warp, kStoreTid issues the bulk stores and releases their
        // stages (measured: +2-3% segmented).  The plain kernel keeps them all
        // on thread 0, with the store's stage released before the next stage
        // wait (measured: 1-1.5% faster there).
        constexpr bool kSpread = HEADS != kNoHeads;
        constexpr int kPubTid = kSpread ? 32 : 0;
        constexpr int kStoreTid = kSpread ? 64 : 0;
        static_assert(!kSpread || CWARPS >= 3, "the serial duties take lanes of three warps");
        int pending = -1;        // kStoreTid: the stage of its last bulk store
        uint32_t scan_uses = 0;  // kPubTid: requests sent to the scanner warp
        bool scan_ok = true;
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (tid == 0) {
                if (!kSpread && pending >= 0) {
                    bulk_wait_read_all();
                    mbar_arrive(&c.empty[pending]);
                    pending = -1;
                }
                c.cflag = mbar_wait_bounded(&c.full[s], use & 1u, role_limit, hdr, epoch, true) ? 1u : 0u;
            }
            named_barrier_sync<CTHREADS>(1);
            if (kSpread && tid == kStoreTid && pending >= 0) {
                // the previous item's store has read its stage by now, mostly
                bulk_wait_read_all();
                mbar_arrive(&c.empty[pending]);
                pending = -1;
            }
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
                    if (!((valid >> j) & 1u)) x[j] = Op::pad();
            }
            uint32_t hm = 0;
            if constexpr (HEADS != kNoHeads) {
                // this thread's items in the tile's head bitmap
                const int b = tid * ITEMS;
                const uint32_t w = __funnelshift_r(c.bits[s][b >> 5], c.bits[s][(b >> 5) + 1], b & 31);
                hm = (ITEMS == 32 ? w : (w & ((1u << ITEMS) - 1u)));
                if (cnt < TILE) hm &= valid_items<ITEMS>(cnt, tid);
            }
            bool tf;
            Acc tv;
            const bool wh = HEADS != kNoHeads && __any_sync(0xffffffffu, hm != 0u);
            thread_reduce_w<Op, ITEMS, HEADS>(x, hm, wh, tf, tv);

            if (phase == kItemReduce) {
                // ---- first pass: the tile sum (with segments: head flag and
                // the sum after the tile's last head) --------------------------
                bool wf = tf;
                Acc wv = tv;
                if constexpr (HEADS != kNoHeads) {
                    warp_inclusive_scan_w<Op, HEADS>(wh, wf, wv, lane);  // lane 31: the warp's
                    if (lane == 31) {
                        c.wtot_v[warp] = wv;
                        c.wtot_f[warp] = wf ? 1u : 0u;
                    }
                } else {
#pragma unroll
                    for (int d = 16; d >= 1; d >>= 1) wv = combine_local<Op>(wv, shfl_down_acc<Op>(wv, d));
                    if (lane == 0) c.wtot_v[warp] = wv;
                }
                named_barrier_sync<CTHREADS>(1);
                if (tid == kPubTid) {
                    Acc wt[CWARPS];
                    uint32_t wtf[CWARPS];
#pragma unroll
                    for (int w = 0; w < CWARPS; ++w) {
                        wt[w] = c.wtot_v[w];
                        if constexpr (HEADS != kNoHeads) wtf[w] = c.wtot_f[w];
                    }
                    Acc total = Op::identity();
                    bool total_f = false;
#pragma unroll
                    for (int w = 0; w < CWARPS; ++w) {
                        if constexpr (HEADS != kNoHeads) {
                            bool f2 = wtf[w] != 0u;
                            Acc v2 = wt[w];
                            seg_combine<Op>(total_f, total, f2, v2);
                            total_f = f2;
                            total = v2;
                        } else {
                            total = combine_local<Op>(total, wt[w]);
                        }
                    }
                    publish_sum_hooked<Op>(p.rec, t, epoch, cfg, total_f, total);
                    mbar_arrive(&c.empty[s]);  // every thread holds its items: stage free
                    const int64_t ch = static_cast<uint32_t>(t) / static_cast<uint32_t>(K);
                    const int64_t first = ch * K;
                    const int64_t nch = (num_tiles - first) < K ? (num_tiles - first) : K;
                    if (t == first + nch - 1) {
                        // the chunk's last tile: its sums go to the scanner warp,
                        // and the consumers go on with the next item meanwhile
                        if (scan_uses > 0 &&
                            !mbar_wait_bounded(&c.scan_idle, (scan_uses - 1) & 1u, role_limit, hdr, epoch,
                                               true))
                            scan_ok = false;
                        if (scan_ok) {
                            c.scan_chunk = ch;
                            mbar_arrive(&c.scan_req);
                            ++scan_uses;
                        }
                    }
                }
                continue;
            }

            // ---- second pass: scan the tile with its offset -----------------
            if (tid == 0) {
                // the prefetched copies first; poll the status words themselves
                // only if a copy was taken before its word was published
                const int64_t ch = static_cast<uint32_t>(t) / static_cast<uint32_t>(K);
                Acc e, off;
                uint32_t se, so;
                bool ef, of;
                parse_words<Op>(c.stat[s][4], c.stat[s][5], epoch, se, ef, e);
                if constexpr (Op::kPacked)
                    parse_words<Op>(c.stat[s][t & 1], 0ull, epoch, so, of, off);
                else
                    parse_words<Op>(c.stat[s][0], c.stat[s][1], epoch, so, of, off);
                const uint64_t t0 = global_timer_ns();
                while (se != kStateP || so != kStateP) {
                    if (global_timer_ns() - t0 > cfg.spin_limit_ns || launch_aborted(hdr, epoch)) {
                        record_timeout(hdr, epoch, t);
                        break;
                    }
                    __nanosleep(64);
                    poll_round_fence();
                    if (se != kStateP)
                        read_words<Op>(rec_chunk(p.rec, ch, 0), epoch, se, ef, e);
                    if (so != kStateP)
                        read_words<Op>(rec_tile<Op>(p.rec, t), epoch, so, of, off);
                }
                // the tile's carry: the chunk prefix, then the in-chunk offset
                if constexpr (HEADS != kNoHeads) {
                    seg_combine<Op>(ef, e, of, off);
                    c.prefix_v = off;
                } else {
                    c.prefix_v = Op::combine(e, off);
                }
            }
            bool wf = tf;
            Acc wv = tv;
            warp_inclusive_scan_w<Op, HEADS>(wh, wf, wv, lane);
            // xf: a head among the lanes before this one
            bool xf = false;
            if constexpr (HEADS != kNoHeads) xf = __shfl_up_sync(0xffffffffu, wf ? 1 : 0, 1) != 0;
            Acc ev = shfl_up_acc<Op>(wv, 1);
            if (lane == 0) {
                xf = false;
                ev = Op::identity();
            }
            if (lane == 31) {
                c.wtot_v[warp] = wv;
                if constexpr (HEADS != kNoHeads) c.wtot_f[warp] = wf ? 1u : 0u;
            }
            named_barrier_sync<CTHREADS>(1);
            // everything before this thread's first item: the tile's carry, the
            // warps before this one, the lanes before this one (a head cuts
            // what comes before it).  Every warp total is read, with 16-byte
            // loads, and the loop over them is unrolled: a loop bounded by the
            // warp index issued one dependent load per warp, on the path that
            // every scan item waits for.
            Acc wt[CWARPS];
            uint32_t wtf[CWARPS];
#pragma unroll
            for (int w = 0; w < CWARPS; ++w) {
                wt[w] = c.wtot_v[w];
                if constexpr (HEADS != kNoHeads) wtf[w] = c.wtot_f[w];
            }
            Acc gv = c.prefix_v;
#pragma unroll
            for (int w = 0; w < CWARPS; ++w) {
                if (w < warp) {
                    if constexpr (HEADS != kNoHeads) {
                        if (wtf[w] != 0u) gv = wt[w];
                        else gv = combine_local<Op>(gv, wt[w]);
                    } else {
                        gv = combine_local<Op>(gv, wt[w]);
                    }
                }
            }
            if (!xf) ev = combine_local<Op>(gv, ev);
            T y[ITEMS];
            thread_outputs_w<Op, ITEMS, HEADS>(x, hm, wh, ev, excl, y);
            store_items<T, ITEMS, TILE, false>(buf, tid, y);
            if (tile_fast) fence_proxy_async_smem();
            named_barrier_sync<CTHREADS>(1);
            if (tile_fast) {
                if (tid == kStoreTid) {
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
        if (tid == kStoreTid) {
            bulk_wait_all();
            if (pending >= 0) mbar_arrive(&c.empty[pending]);
        }
        if (tid == kPubTid) {
            // stop the scanner warp once its last request is done
            if (scan_uses > 0 && scan_ok)
                scan_ok = mbar_wait_bounded(&c.scan_idle, (scan_uses - 1) & 1u, role_limit, hdr, epoch, true);
            c.scan_chunk = -1;
            mbar_arrive(&c.scan_req);
        }
    } else if (warp == SCAN_WARP) {
        for (uint32_t u = 0;; ++u) {
            if (!warp_wait(&c.scan_req, u & 1u, role_limit, hdr, epoch, lane)) break;
            const int64_t ch = *static_cast<volatile int64_t*>(&c.scan_chunk);
            if (ch < 0) break;
            chunk_scan_warp<Op, HEADS>(p, ch, hdr, epoch, cfg, lane);
            __syncwarp();
            if (lane == 0) mbar_arrive(&c.scan_idle);
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
