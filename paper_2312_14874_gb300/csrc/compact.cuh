// compact.cuh — stream compaction, the scan applied: out = the elements of `in`
// whose keep flag is nonzero, in order, and the number kept.
//
// The exclusive scan of the 0/1 keep flags (Section 1's definition over the
// flags) gives every kept element its position in the output.  Two kernels:
// compact_kernel runs the partitioned scan (Section 2.2), and lb_compact_kernel
// (at the end of this file) the single-pass chained scan, the faster below
// about 2^26 elements.  compact_kernel: a work list of reduce items R and scan items
// S, S(c) interleaved with R(c + lag); the chunk scanner warp turns a chunk's
// tile counts into tile offsets and chains the chunk prefixes.  An R item
// counts the kept elements of kCpGroup consecutive tiles from their flags alone
// (read with L2 evict-last priority): the flags of one tile are a fifth of its
// payload, and a work item costs a pipeline stage whatever its size, so a group
// of four tiles' flags makes an R item as big as an S item's payload.  An S item loads the tile's payload and flags (the flags again,
// from L2) with its two prefetched status words, gives each thread's kept
// elements their positions (block exclusive scan of the thread counts),
// gathers them into shared memory in order, and writes the tile's run of kept
// elements to out[offset ...] with coalesced stores: the scan is fused with its
// consumer and no flag prefix ever reaches global memory.  Counts are 64-bit.
// Payload elements are 4 bytes, copied bit for bit (int32 and fp32 alike).
// The loader asks L2 for the payload and flags about 12 MiB ahead of its
// copies (nothing is claimed for them).  The tuned shape from 2^24 up is 16
// consumer warps x 28 items at one block per SM: the per-tile costs (three
// block barriers, the warp scans, item decoding, status words) spread over
// 14336 elements.
#pragma once

#include "lookback.cuh"
#include "partitioned.cuh"

namespace gbscan {

constexpr int kCpGroup = 4;  // tiles whose flags one R item counts
constexpr uint32_t kCpEnd = 2;  // stage phase: no more items

// The work list of the compaction (tiles in chunks of K, a multiple of
// kCpGroup, so that R groups never straddle chunks; R item q counts tiles
// [q G, q G + G)):
//   the R items of chunks 0 .. lag-1, then for each chunk c the slot of its
//   S items and the R items of chunk c + lag, repeating G S items then one R
//   item while both last, then the rest.
struct CpOrder {
    uint32_t K, lag, C, nlast, RK, pre, F, U;
};

__device__ __forceinline__ CpOrder make_cp_order(int64_t num_tiles, int64_t K, int64_t lag) {
    CpOrder o;
    o.K = static_cast<uint32_t>(K);
    o.lag = static_cast<uint32_t>(lag);
    o.C = static_cast<uint32_t>((num_tiles + K - 1) / K);
    o.nlast = static_cast<uint32_t>(num_tiles - static_cast<int64_t>(o.C - 1) * K);
    o.RK = o.K / kCpGroup;
    const uint32_t L = o.lag < o.C ? o.lag : o.C;
    o.pre = L < o.C ? L * o.RK : (o.C - 1) * o.RK + (o.nlast + kCpGroup - 1) / kCpGroup;
    o.F = o.C > o.lag + 1 ? o.C - 1 - o.lag : 0;
    o.U = o.K + o.RK;
    return o;
}

// Item w: phase kItemReduce with idx = the R group, or kItemScan with idx = the tile.
__device__ __forceinline__ void compact_item(uint32_t w, const CpOrder& o, uint32_t& phase,
                                             int64_t& idx) {
    constexpr uint32_t G = kCpGroup;
    if (w < o.pre) {
        phase = kItemReduce;
        idx = w;
        return;
    }
    w -= o.pre;
    if (w < o.F * o.U) {
        const uint32_t c = w / o.U, p = w - c * o.U, q = p / (G + 1), rr = p - q * (G + 1);
        if (rr < G) {
            phase = kItemScan;
            idx = static_cast<int64_t>(c) * o.K + q * G + rr;
        } else {
            phase = kItemReduce;
            idx = static_cast<int64_t>(c + o.lag) * o.RK + q;
        }
        return;
    }
    w -= o.F * o.U;
    for (uint32_t c = o.F; c < o.C; ++c) {
        const uint32_t nS = c < o.C - 1 ? o.K : o.nlast;
        const uint32_t cr = c + o.lag;
        const uint32_t nR = cr < o.C ? (cr < o.C - 1 ? o.RK : (o.nlast + G - 1) / G) : 0;
        if (w < nS + nR) {
            const int64_t sbase = static_cast<int64_t>(c) * o.K;
            const int64_t rbase = static_cast<int64_t>(cr) * o.RK;
            const uint32_t full = nR < nS / G ? nR : nS / G;
            if (w < full * (G + 1)) {
                const uint32_t q = w / (G + 1), rr = w - q * (G + 1);
                phase = rr < G ? kItemScan : kItemReduce;
                idx = rr < G ? sbase + q * G + rr : rbase + q;
                return;
            }
            const uint32_t p = w - full * (G + 1), remS = nS - full * G;
            phase = p < remS ? kItemScan : kItemReduce;
            idx = p < remS ? sbase + full * G + p : rbase + full + (p - remS);
            return;
        }
        w -= nS + nR;
    }
    phase = kItemScan;  // not reached for w below the item count
    idx = 0;
}

template <int CWARPS, int STAGES>
struct CpCtrl {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int64_t tile_id[STAGES];
    uint32_t phase[STAGES];
    alignas(16) unsigned long long stat[STAGES][6];
    uint32_t wtot[CWARPS];    // S item: the warps' kept counts
    uint32_t gtot[kCpGroup][CWARPS];  // R item: per tile of the group, the warps' counts
    unsigned long long base;  // S item: the output position of the tile's first kept element
    uint64_t scan_req;
    uint64_t scan_idle;
    int64_t scan_chunk;
    uint32_t epoch;
    uint32_t clear;
    uint32_t cflag;
    unsigned int claim_sink;
};

template <int CWARPS, int ITEMS, int STAGES>
constexpr int cp_smem_bytes() {
    return STAGES * CWARPS * 32 * ITEMS * 5 + static_cast<int>(sizeof(CpCtrl<CWARPS, STAGES>));
}

// The number of nonzero bytes among the thread's ITEMS flags, four at a time
// (each byte's bits ORed down into its bit 0; ITEMS a multiple of 4, the flag
// run 4-byte aligned).
template <int ITEMS>
__device__ __forceinline__ uint32_t keep_count(const uint8_t* f) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(f);
    uint32_t n = 0;
#pragma unroll
    for (int q = 0; q < ITEMS / 4; ++q) {
        uint32_t t = w[q];
        t |= t >> 4;
        t |= t >> 2;
        t |= t >> 1;
        n += __popc(t & 0x01010101u);
    }
    return n;
}

// Bit j set: the thread's flag j is nonzero.
template <int ITEMS>
__device__ __forceinline__ uint32_t keep_mask(const uint8_t* f) {
    static_assert(ITEMS % 4 == 0 && ITEMS <= 32, "whole flag words, one 32-bit mask");
    const uint32_t* w = reinterpret_cast<const uint32_t*>(f);
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < ITEMS / 4; ++q) {
        // bit 0 of each byte: the byte is nonzero (its bits ORed down), then
        // the multiply gathers the four bits 0, 8, 16, 24 into bits 24..27
        // (each product term lands on its own bit: no carries reach them)
        uint32_t t = w[q];
        t |= t >> 4;
        t |= t >> 2;
        t |= t >> 1;
        t &= 0x01010101u;
        m |= ((t * 0x01020408u) >> 24) << (4 * q);
    }
    return m;
}

template <int CWARPS, int ITEMS, int STAGES, int MINB>
__global__ void __launch_bounds__((CWARPS + 2) * 32, MINB) compact_kernel(const Params p) {
    using Op = OpI64;  // the counts
    using T = uint32_t;
    constexpr int CTHREADS = CWARPS * 32;
    constexpr int TILE = CTHREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * 4;
    constexpr int STAGE_BYTES = TILE_BYTES + TILE;  // payload, then flags
    constexpr int LOAD_WARP = CWARPS;
    constexpr int SCAN_WARP = CWARPS + 1;
    static_assert(TILE % 16 == 0, "flag slices are bulk copies");
    using CtrlT = CpCtrl<CWARPS, STAGES>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * STAGE_BYTES);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t num_tiles = p.num_tiles;
    const int64_t K = p.chunk_tiles;
    const int64_t num_groups = (num_tiles + kCpGroup - 1) / kCpGroup;
    const int64_t num_items = num_tiles + num_groups;
    static_assert(kCpGroup * TILE <= TILE_BYTES, "an R group's flags fill the payload area");

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&c.full[s], 1);
            mbar_init(&c.empty[s], 1);
        }
        mbar_init(&c.scan_req, 1);
        mbar_init(&c.scan_idle, 1);
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
    auto payload = [&](int s) { return reinterpret_cast<T*>(smem + s * STAGE_BYTES); };
    auto flagbuf = [&](int s) { return smem + s * STAGE_BYTES + TILE_BYTES; };

    if (warp == LOAD_WARP) {
        const T* __restrict__ in = static_cast<const T*>(p.in);
        const uint8_t* __restrict__ fl = p.flags;
        const uint64_t keep = l2_policy_evict_last();
        const uint64_t drop = l2_policy_evict_first();
        const CpOrder order = make_cp_order(num_tiles, K, p.chunk_lag);
        // claims as in the partitioned scan: two items per atomic, the next
        // claim in flight
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
                if (lane == 0) {
                    c.phase[s] = kCpEnd;
                    mbar_arrive(&c.full[s]);
                }
                break;
            }
            uint32_t phase;
            int64_t t;  // the tile of an S item, the group of an R item
            compact_item(static_cast<uint32_t>(w), order, phase, t);
            // an R item's flags (kCpGroup tiles) go to the payload area, an S
            // item's flags to the flag area; flags move by TMA when the slice
            // is whole and 16-byte aligned, the payload when `in` is aligned and
            // the tile whole
            const int64_t f0 = phase == kItemReduce ? t * kCpGroup * TILE : t * TILE;
            const int64_t fcap = phase == kItemReduce ? static_cast<int64_t>(kCpGroup) * TILE : TILE;
            const int fcnt = static_cast<int>((p.n - f0) < fcap ? (p.n - f0) : fcap);
            const int cnt = phase == kItemScan ? count_of(t) : 0;
            const bool ffast = fcnt == fcap && (reinterpret_cast<uintptr_t>(fl) & 15) == 0;
            const bool xfast = p.fast && phase == kItemScan && cnt == TILE;
            T* xb = payload(s);
            uint8_t* fb = phase == kItemReduce ? reinterpret_cast<uint8_t*>(xb) : flagbuf(s);
            // ragged or misaligned parts: aligned bodies by bulk copies, the
            // rest by the lanes
            uint32_t fbytes = ffast ? static_cast<uint32_t>(fcap) : 0u;
            uint32_t xbytes = xfast ? static_cast<uint32_t>(TILE_BYTES) : 0u;
            if (!ffast)
                fbytes = warp_stage_partial<uint8_t>(fb, fl + f0, fcnt, fcnt,
                                                     (reinterpret_cast<uintptr_t>(fl) & 15) == 0,
                                                     uint8_t(0), lane);
            if (phase == kItemScan && !xfast)
                xbytes = warp_stage_partial<T>(xb, in + t * TILE, cnt, cnt, p.fast, T(0), lane);
            __syncwarp();
            if (lane == 0) {
                c.tile_id[s] = t;
                c.phase[s] = phase;
                const uint32_t stat_bytes = phase == kItemScan ? 32u : 0u;
                const uint32_t tx = fbytes + xbytes + stat_bytes;
                if (tx == 0) {
                    mbar_arrive(&c.full[s]);
                } else {
                    mbar_arrive_expect_tx(&c.full[s], tx);
                    if (fbytes)
                        bulk_load_hint(fb, fl + f0, fbytes, &c.full[s], phase == kItemReduce ? keep : drop);
                    if (xbytes) bulk_load_hint(xb, in + t * TILE, xbytes, &c.full[s], drop);
                    // the first DRAM reads (an S item's payload, an R item's
                    // flags) of the item prefetch_tiles tiles ahead go to L2 now,
                    // so that its copy comes from L2 (no item is claimed for it)
                    if (p.prefetch_tiles > 0) {
                        if (phase == kItemScan && p.fast) {
                            const int64_t pt = t + p.prefetch_tiles;
                            if (pt < num_tiles) {
                                const uint32_t pb = (static_cast<uint32_t>(count_of(pt)) * 4u) & ~15u;
                                if (pb) bulk_prefetch_l2(in + pt * TILE, pb);
                            }
                        } else if (phase == kItemReduce && (reinterpret_cast<uintptr_t>(fl) & 15) == 0) {
                            const int64_t pf0 = f0 + p.prefetch_tiles * static_cast<int64_t>(TILE);
                            if (pf0 < p.n) {
                                const int64_t rem = p.n - pf0;
                                const uint32_t pb = static_cast<uint32_t>(rem < fcap ? rem : fcap) & ~15u;
                                if (pb) bulk_prefetch_l2(fl + pf0, pb);
                            }
                        }
                    }
                    if (stat_bytes) {
                        // the tile's status pair and the chunk's E pair
                        bulk_load(&c.stat[s][0], rec_tile<OpI64>(p.rec, t), 16, &c.full[s]);
                        const uint32_t ch = static_cast<uint32_t>(t) / order.K;
                        bulk_load(&c.stat[s][4], rec_chunk(p.rec, ch, 0), 16, &c.full[s]);
                    }
                }
            }
        }
        if (lane == 0) {
            *static_cast<volatile unsigned int*>(&c.claim_sink) = cur ^ nxt;
            drain_fills<STAGES>(c.full, fills, role_limit, hdr);
        }
    } else if (warp < CWARPS) {
        T* out = static_cast<T*>(p.out);
        uint32_t scan_uses = 0;
        bool scan_ok = true;
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (tid == 0) {
                c.cflag = mbar_wait_bounded(&c.full[s], use & 1u, role_limit, hdr, epoch, true) ? 1u : 0u;
                if (c.cflag && c.phase[s] == kItemScan) {
                    // the output position of the tile's run: the chunk prefix
                    // plus the tile's offset within the chunk, from the
                    // prefetched copies (the words themselves only if a copy was
                    // taken before its word was published)
                    const int64_t ts = c.tile_id[s];
                    const int64_t ch = static_cast<uint32_t>(ts) / static_cast<uint32_t>(K);
                    unsigned long long e, off;
                    uint32_t se, so;
                    bool hf;
                    parse_words<Op>(c.stat[s][4], c.stat[s][5], epoch, se, hf, e);
                    parse_words<Op>(c.stat[s][0], c.stat[s][1], epoch, so, hf, off);
                    const uint64_t t0 = global_timer_ns();
                    while (se != kStateP || so != kStateP) {
                        if (global_timer_ns() - t0 > cfg.spin_limit_ns || launch_aborted(hdr, epoch)) {
                            record_timeout(hdr, epoch, ts);
                            break;
                        }
                        __nanosleep(64);
                        poll_round_fence();
                        if (se != kStateP)
                            read_words<Op>(rec_chunk(p.rec, ch, 0), epoch, se, hf, e);
                        if (so != kStateP)
                            read_words<Op>(rec_tile<Op>(p.rec, ts), epoch, so, hf, off);
                    }
                    c.base = e + off;
                }
            }
            named_barrier_sync<CTHREADS>(1);
            if (!c.cflag) break;
            const uint32_t phase = c.phase[s];
            if (phase == kCpEnd) break;
            const int64_t t = c.tile_id[s];
            if (phase == kItemReduce) {
                // ---- R item: the kept counts of the group's tiles ------------
                const uint8_t* fb = reinterpret_cast<const uint8_t*>(payload(s));
                // the thread's kept counts of the four tiles (at most ITEMS
                // each, a warp's at most 640), two to a word, so that the warp
                // sums take two shuffle reductions instead of four
                uint32_t packed[kCpGroup / 2] = {};
#pragma unroll
                for (int g = 0; g < kCpGroup; ++g) {
                    const int64_t tg = t * kCpGroup + g;
                    const int cg = tg < num_tiles ? count_of(tg) : 0;
                    uint32_t v = 0;
                    if (cg == TILE) {
                        v = keep_count<ITEMS>(fb + g * TILE + tid * ITEMS);
                    } else if (cg > 0) {
                        v = __popc(keep_mask<ITEMS>(fb + g * TILE + tid * ITEMS) & valid_items<ITEMS>(cg, tid));
                    }
                    packed[g / 2] |= v << (16 * (g & 1));
                }
                static_assert(kCpGroup % 2 == 0 && 32 * ITEMS < 65536, "two warp counts fit one word");
#pragma unroll
                for (int q = 0; q < kCpGroup / 2; ++q) {
                    uint32_t v = packed[q];
#pragma unroll
                    for (int d = 16; d >= 1; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
                    if (lane == 0) {
                        c.gtot[2 * q][warp] = v & 0xffffu;
                        c.gtot[2 * q + 1][warp] = v >> 16;
                    }
                }
                named_barrier_sync<CTHREADS>(1);  // group counts written, flags read
                if (tid == 0) {
                    for (int g = 0; g < kCpGroup; ++g) {
                        const int64_t tg = t * kCpGroup + g;
                        if (tg >= num_tiles) break;
                        unsigned long long total = 0;
                        for (int w = 0; w < CWARPS; ++w) total += c.gtot[g][w];
                        publish_sum_hooked<Op>(p.rec, tg, epoch, cfg, false, total);
                    }
                    mbar_arrive(&c.empty[s]);
                    // the group holding its chunk's last tile hands the chunk to
                    // the scanner warp
                    const int64_t g0 = t * kCpGroup;
                    const int64_t ch = static_cast<uint32_t>(g0) / static_cast<uint32_t>(K);
                    const int64_t first = ch * K;
                    const int64_t nch = (num_tiles - first) < K ? (num_tiles - first) : K;
                    const int64_t last = first + nch - 1;
                    if (last >= g0 && last < g0 + kCpGroup) {
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
            const int cnt = count_of(t);
            uint32_t m = keep_mask<ITEMS>(flagbuf(s) + tid * ITEMS);
            if (cnt < TILE) m &= valid_items<ITEMS>(cnt, tid);
            const uint32_t mine = __popc(m);
            // block exclusive scan of the thread counts
            uint32_t inc = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += o;
            }
            if (lane == 31) c.wtot[warp] = inc;
            T x[ITEMS];
            load_items<T, ITEMS, TILE, false>(payload(s), tid, x);
            named_barrier_sync<CTHREADS>(1);  // warp totals written, payload read
            // ---- scan item: positions of the kept elements, gather, write --
            // The run is gathered at stage index shift + (position in the run),
            // shift = base mod 4, so that stage index i and output element
            // base - shift + i share their 16-byte alignment; the up to three
            // elements past the payload area land in the flag area, whose flags
            // every thread has read.
            const unsigned long long base = c.base;
            const uint32_t shift = static_cast<uint32_t>(base & 3ull);
            uint32_t pos = shift + inc - mine;  // this thread's first stage index
            uint32_t kept = 0;                  // the tile's kept count
#pragma unroll
            for (int w = 0; w < CWARPS; ++w) {
                const uint32_t wt = c.wtot[w];
                kept += wt;
                if (w < warp) pos += wt;
            }
            // pos + the thread's kept count <= shift + the tile's kept count
            // <= 3 + TILE: every counted flag is one of this tile's
            T* xb = payload(s);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                if ((m >> j) & 1u) xb[pos] = x[j];
                pos += (m >> j) & 1u;
            }
            named_barrier_sync<CTHREADS>(1);  // the run is gathered
            // a run that would leave the output (only after a failed wait, which
            // has recorded its error) is not written
            if (kept > static_cast<uint32_t>(TILE) || base > static_cast<unsigned long long>(p.n) ||
                kept > static_cast<unsigned long long>(p.n) - base) {
                if (tid == 0) record_error(hdr, GBSCAN_ERR_INVALID_ARG, t);
                kept = 0;
            }
            const uint32_t span = shift + kept;  // stage indices [shift, span) hold the run
            T* og = out + (base - shift);        // output element of stage index 0
            if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
                // 16-byte stores for the whole groups of four, single elements
                // at the two ends of the run
                for (uint32_t i0 = 4u * tid; i0 < span; i0 += 4u * CTHREADS) {
                    if (i0 >= shift && i0 + 4u <= span) {
                        *reinterpret_cast<uint4*>(og + i0) = *reinterpret_cast<const uint4*>(xb + i0);
                    } else {
#pragma unroll
                        for (uint32_t q = 0; q < 4u; ++q)
                            if (i0 + q >= shift && i0 + q < span) og[i0 + q] = xb[i0 + q];
                    }
                }
            } else {
                for (uint32_t i = shift + tid; i < span; i += CTHREADS) og[i] = xb[i];
            }
            named_barrier_sync<CTHREADS>(1);  // the stage is read
            if (tid == 0) mbar_arrive(&c.empty[s]);
        }
        if (tid == 0) {
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
            chunk_scan_warp<Op, kNoHeads>(p, ch, hdr, epoch, cfg, lane);
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

// ---- the compaction on the single-pass chained scan ------------------------
//
// lb_compact_kernel: the roles of the single-pass look-back kernel
// (lookback.cuh) applied to the keep flags, one pass over the data.
//   loader     claims a tile when a stage is free and copies the tile's
//              payload and its flags into the stage (bulk copies; a ragged or
//              misaligned tile partly by the lanes, its flags padded with 0);
//              it asks L2 for the payload and flags about 12 MiB ahead;
//   agents     one warp per stage: counts the tile's kept elements from the
//              staged flags, publishes the count and looks back over the
//              earlier tiles' counts (the exclusive scan of the counts, Section
//              1's definition over the flags); the tile's exclusive count is
//              its first output position.  The last tile's agent writes the
//              total;
//   consumers  NW warps read the stage at once (lane l of warp w: the 16-byte
//              payload vectors w*NV*32 + j*32 + l and their four flags) and
//              give it back; three ballots of the lane counts per row of 32
//              vectors give every lane its kept elements' places in the row,
//              and the warps exchange their kept counts.  Once the tile's
//              position is known, every lane stores its kept elements at
//              their places straight from registers (consecutive lanes'
//              elements are adjacent, so each store instruction covers a
//              few hundred contiguous bytes).
// A tile waits for its position in registers, not in a stage, so the stages
// are refilled as soon as they are read and the shared memory holds stages
// only (the bytes in flight per SM set the rate of a chained scan here).
// Measured against placing each row in a shared-memory row buffer first and
// storing it with one coalesced store per 32 elements: fewer instructions,
// 4366 against 3868 GB/s at int32 2^30 with half kept.  Warp 0 alone polls
// for the tile's position; the other consumer warps wait in the block's named
// barrier and spend no issue slots (4468 GB/s).
template <int NW, int STAGES>
struct LbcCtrl {
    uint64_t full[STAGES];   // stage data landed
    uint64_t empty[STAGES];  // count 2: the consumers have read the stage, its agent is idle
    uint64_t ready[STAGES];  // the agent has put the tile's position in excl
    int64_t tile_id[STAGES];
    unsigned long long excl[STAGES][2];  // by use parity, as in the look-back scan
    uint32_t wtot[NW];
    uint32_t epoch;
    uint32_t clear;
};

template <int NW, int NV>
__host__ __device__ constexpr int lbc_tile() {
    return NW * 32 * NV * 4;
}

// Stages (payload, then flags), then the control block.
template <int NW, int NV, int STAGES>
constexpr int lbc_smem_bytes() {
    return STAGES * lbc_tile<NW, NV>() * 5 + static_cast<int>(sizeof(LbcCtrl<NW, STAGES>));
}

template <int NW, int STAGES>
constexpr int lbc_threads() {
    return (NW + 1 + STAGES) * 32;
}

// The number of nonzero bytes of a word (each byte's bits ORed into its bit 0).
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t t) {
    t |= t >> 4;
    t |= t >> 2;
    t |= t >> 1;
    return __popc(t & 0x01010101u);
}

template <int NW, int NV, int STAGES, int LB, int MINB>
__global__ void __launch_bounds__((NW + 1 + STAGES) * 32, MINB) lb_compact_kernel(const Params p) {
    using Op = OpI64;  // the counts
    using T = uint32_t;
    constexpr int NT = NW * 32;
    constexpr int TILE = lbc_tile<NW, NV>();
    constexpr int TILE_BYTES = TILE * 4;
    constexpr int STAGE_BYTES = TILE_BYTES + TILE;  // payload, then flags
    constexpr int LOAD_WARP = NW;                   // warps NW+1+s: the agent of stage s
    static_assert(STAGES >= 2, "at least two stages");
    static_assert((TILE / 16) % 32 == 0, "whole rows of flag vectors for the agents");
    using CtrlT = LbcCtrl<NW, STAGES>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * STAGE_BYTES);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t num_tiles = p.num_tiles;

    unsigned int first_claim = 0;
    if (warp == LOAD_WARP && lane == 0) first_claim = atomicAdd(&hdr->tile_counter, 1u);
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&c.full[s], 1);
            mbar_init(&c.empty[s], 2);
            mbar_init(&c.ready[s], 1);
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
    auto payload = [&](int s) { return reinterpret_cast<T*>(smem + s * STAGE_BYTES); };
    auto flagbuf = [&](int s) { return smem + s * STAGE_BYTES + TILE_BYTES; };

    if (warp == LOAD_WARP) {
        const T* __restrict__ in = static_cast<const T*>(p.in);
        const uint8_t* __restrict__ fl = p.flags;
        const bool in_al = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
        const bool fl_al = (reinterpret_cast<uintptr_t>(fl) & 15) == 0;
        const uint64_t evict_first = l2_policy_evict_first();
        uint32_t fills = 0;
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (use > 0 && !warp_wait(&c.empty[s], (use - 1) & 1u, role_limit, hdr, epoch, lane))
                break;
            long long claimed = 0;
            if (lane == 0)
                claimed = static_cast<long long>(k == 0 ? first_claim : atomicAdd(&hdr->tile_counter, 1u));
            const int64_t tile = __shfl_sync(0xffffffffu, claimed, 0);
            if (tile >= num_tiles) {
                // an end sentinel in this stage and the next STAGES-1
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    mbar_arrive(&c.full[s]);
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
                    }
                    ++fills;
                }
                break;
            }
            const int cnt = count_of(tile);
            T* xb = payload(s);
            uint8_t* fb = flagbuf(s);
            if (in_al && fl_al && cnt == TILE) {
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    mbar_arrive_expect_tx(&c.full[s], TILE_BYTES + TILE);
                    bulk_load_hint(xb, in + tile * TILE, TILE_BYTES, &c.full[s], evict_first);
                    bulk_load_hint(fb, fl + tile * TILE, TILE, &c.full[s], evict_first);
                    // the tile prefetch_tiles ahead, into L2 for whichever block
                    // claims it (no claim is made)
                    const int64_t pt = tile + p.prefetch_tiles;
                    if (p.prefetch_tiles > 0 && pt < num_tiles) {
                        const uint32_t pc = static_cast<uint32_t>(count_of(pt));
                        if ((pc * 4u) & ~15u) bulk_prefetch_l2(in + pt * TILE, (pc * 4u) & ~15u);
                        if (pc & ~15u) bulk_prefetch_l2(fl + pt * TILE, pc & ~15u);
                    }
                }
            } else {
                // ragged or misaligned: aligned bodies by bulk copies, the rest
                // by the lanes; the flags padded with 0 to the whole tile
                const uint32_t xbytes = warp_stage_partial<T>(xb, in + tile * TILE, cnt, cnt, in_al, T(0), lane);
                const uint32_t fbytes =
                    warp_stage_partial<uint8_t>(fb, fl + tile * TILE, cnt, TILE, fl_al, uint8_t(0), lane);
                __syncwarp();
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    if (xbytes + fbytes) {
                        mbar_arrive_expect_tx(&c.full[s], xbytes + fbytes);
                        if (xbytes) bulk_load(xb, in + tile * TILE, xbytes, &c.full[s]);
                        if (fbytes) bulk_load(fb, fl + tile * TILE, fbytes, &c.full[s]);
                    } else {
                        mbar_arrive(&c.full[s]);
                    }
                }
            }
            ++fills;
        }
        if (lane == 0) drain_fills<STAGES>(c.full, fills, role_limit, hdr);
    } else if (warp > LOAD_WARP) {
        // ---- the stage's agent: the tile's count, look-back, position -------
        const int s = warp - LOAD_WARP - 1;
        for (uint32_t use = 0;; ++use) {
            if (!warp_spin_wait(&c.full[s], use & 1u, role_limit, hdr, epoch, lane)) break;
            const int64_t tile = *static_cast<volatile int64_t*>(&c.tile_id[s]);
            if (tile >= num_tiles) break;
            const uint4* f4 = reinterpret_cast<const uint4*>(flagbuf(s)) + lane;
            uint32_t kept = 0;
#pragma unroll
            for (int q = 0; q < TILE / 16 / 32; ++q) {
                const uint4 w = f4[q * 32];
                kept += nonzero_bytes(w.x) + nonzero_bytes(w.y) + nonzero_bytes(w.z) + nonzero_bytes(w.w);
            }
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, d);
            const unsigned long long agg = kept;
            __syncwarp();
            if (lane == 0) publish_aggregate<Op>(p.rec, tile, epoch, cfg, false, agg);
            bool ef;
            unsigned long long ev;
            lookback<Op, kNoHeads, LB>(p.rec, hdr, tile, epoch, cfg, false, agg, lane, ef, ev);
            if (lane == 0) {
                c.excl[s][use & 1u] = ev;
                if (tile == num_tiles - 1 && p.total_out) *p.total_out = ev + agg;
                mbar_arrive(&c.ready[s]);
                mbar_arrive(&c.empty[s]);  // idle again: the stage may be refilled
            }
        }
    } else {
        // ---- consumers: places, the warps' runs, stores -----------------------
        T* out = static_cast<T*>(p.out);
        const int vbase = warp * NV * 32 + lane;  // this lane's first vector in the tile
        const uint32_t below = (1u << lane) - 1u;
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            const bool ok = warp_spin_wait(&c.full[s], use & 1u, role_limit, hdr, epoch, lane);
            const int64_t tile = *static_cast<volatile int64_t*>(&c.tile_id[s]);
            bool stop = !ok || tile >= num_tiles;
            const uint4* x4 = reinterpret_cast<const uint4*>(payload(s));
            const uint32_t* f1 = reinterpret_cast<const uint32_t*>(flagbuf(s));
            uint4 x[NV];
            uint32_t m[NV];   // the vector's four keep bits (bit i: element 4v+i)
            uint32_t ex[NV];  // the row's kept elements before this lane's
            uint32_t rt[NV];  // the row's kept elements
            uint32_t wk = 0;  // the warp's kept elements (the same in every lane)
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const int v = vbase + j * 32;
                x[j] = x4[v];
                // the bytes' ORed-down bits, gathered by one multiply
                uint32_t t = f1[v];
                t |= t >> 4;
                t |= t >> 2;
                t |= t >> 1;
                t &= 0x01010101u;
                m[j] = (t * 0x01020408u) >> 24;
                const uint32_t n = __popc(m[j]);
                const uint32_t b0 = __ballot_sync(0xffffffffu, n & 1u);
                const uint32_t b1 = __ballot_sync(0xffffffffu, n & 2u);
                const uint32_t b2 = __ballot_sync(0xffffffffu, n & 4u);
                ex[j] = __popc(b0 & below) + 2u * __popc(b1 & below) + 4u * __popc(b2 & below);
                rt[j] = __popc(b0) + 2u * __popc(b1) + 4u * __popc(b2);
                wk += rt[j];
            }
            if (lane == 0) c.wtot[warp] = wk;
            // kept counts exchanged; every consumer warp agrees on going on
            stop = named_barrier_or<NT>(1, stop);
            if (stop) break;
            if (tid == 0) mbar_arrive(&c.empty[s]);  // every consumer has read the stage
            uint32_t woff = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (w < warp) woff += c.wtot[w];
            // warp 0 alone polls for the tile's position; the barrier releases
            // the others (and orders the counts' reads before the next tile's
            // writes), so the waiting warps take no issue slots
            const bool bad = named_barrier_or<NT>(
                1, warp == 0 && !warp_spin_wait(&c.ready[s], use & 1u, role_limit, hdr, epoch, lane));
            const unsigned long long base = c.excl[s][use & 1u] + woff;
            // a run that would leave the output (only after a failed wait, which
            // has recorded its error) is not written
            if (!bad && base <= static_cast<unsigned long long>(p.n) &&
                wk <= static_cast<unsigned long long>(p.n) - base) {
                T* o = out + base;
                // each lane stores its kept elements at their places
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    uint32_t q = ex[j];
                    if (m[j] & 1u) o[q++] = x[j].x;
                    if (m[j] & 2u) o[q++] = x[j].y;
                    if (m[j] & 4u) o[q++] = x[j].z;
                    if (m[j] & 8u) o[q] = x[j].w;
                    o += rt[j];
                }
            }
        }
    }

    __syncthreads();
    if (tid == 0) c.clear = finish_launch(hdr, epoch) ? 1u : 0u;
    __syncthreads();
    if (c.clear) clear_status_words(p.rec, p.rec_capacity, tid, blockDim.x);
}

}  // namespace gbscan
