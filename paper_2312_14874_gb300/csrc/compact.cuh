// compact.cuh — stream compaction, the scan applied: out = the elements of `in`
// whose keep flag is nonzero, in order, and the number kept.
//
// The exclusive scan of the 0/1 keep flags (Section 1's definition over the
// flags) gives every kept element its position in the output.  The scan is the
// partitioned one (Section 2.2): a work list of reduce items R (count the kept
// elements of a tile from its flags alone, flags read with L2 evict-last
// priority) and scan items S, S(c) interleaved with R(c + lag); the chunk
// scanner warp turns a chunk's tile counts into tile offsets and chains the
// chunk prefixes.  An S item loads the tile's payload and flags (the flags again,
// from L2) with its two prefetched status words, gives each thread's kept
// elements their positions (block exclusive scan of the thread counts),
// gathers them into shared memory in order, and writes the tile's run of kept
// elements to out[offset ...] with coalesced stores: the scan is fused with its
// consumer and no flag prefix ever reaches global memory.  Counts are 64-bit.
// Payload elements are 4 bytes, copied bit for bit (int32 and fp32 alike).
#pragma once

#include "partitioned.cuh"

namespace gbscan {

template <int CWARPS, int STAGES>
struct CpCtrl {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int64_t tile_id[STAGES];
    uint32_t phase[STAGES];
    alignas(16) unsigned long long stat[STAGES][6];
    unsigned long long wtot[CWARPS];
    unsigned long long base;  // S item: the output position of the tile's first kept element
    uint32_t kept;            // S item: the tile's kept count
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

// Nonzero bytes among the thread's ITEMS flags (ITEMS a multiple of 4; the flag
// run starts 4-byte aligned).
template <int ITEMS>
__device__ __forceinline__ uint32_t keep_mask(const uint8_t* f) {
    static_assert(ITEMS % 4 == 0 && ITEMS <= 32, "whole flag words, one 32-bit mask");
    const uint32_t* w = reinterpret_cast<const uint32_t*>(f);
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < ITEMS / 4; ++q) {
        const uint32_t v = w[q];
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if ((v >> (8 * b)) & 0xffu) m |= 1u << (4 * q + b);
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
    const int64_t num_items = 2 * num_tiles;

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
        const PtOrder order = make_order(num_tiles, K, p.chunk_lag);
        // claims as in the partitioned scan: two items per atomic, the next
        // claim in flight
        unsigned int cur = 0, nxt = 0;
        if (lane == 0) {
            cur = atomicAdd(&hdr->tile_counter, static_cast<unsigned int>(kClaim));
            nxt = atomicAdd(&hdr->tile_counter, static_cast<unsigned int>(kClaim));
        }
        int in_batch = 0;
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
            if (w >= num_items) {
                if (lane == 0) {
                    c.tile_id[s] = num_tiles;  // end
                    mbar_arrive(&c.full[s]);
                }
                break;
            }
            uint32_t phase;
            int64_t t;
            partitioned_item(static_cast<uint32_t>(w), order, phase, t);
            const int cnt = count_of(t);
            // flags move by TMA when the slice is whole and 16-byte aligned;
            // the payload (scan items only) when `in` is aligned and whole too
            const bool ffast = cnt == TILE && (reinterpret_cast<uintptr_t>(fl) & 15) == 0;
            const bool xfast = p.fast && cnt == TILE;
            T* xb = payload(s);
            uint8_t* fb = flagbuf(s);
            if (!ffast) {
                for (int i = lane; i < cnt; i += 32) fb[i] = fl[t * TILE + i];
            }
            if (phase == kItemScan && !xfast) {
                for (int i = lane; i < cnt; i += 32) xb[i] = in[t * TILE + i];
            }
            __syncwarp();
            if (lane == 0) {
                c.tile_id[s] = t;
                c.phase[s] = phase;
                const uint32_t stat_bytes = phase == kItemScan ? 48u : 0u;
                const uint32_t tx = (ffast ? static_cast<uint32_t>(TILE) : 0u) +
                                    (phase == kItemScan && xfast ? static_cast<uint32_t>(TILE_BYTES) : 0u) +
                                    stat_bytes;
                if (tx == 0) {
                    mbar_arrive(&c.full[s]);
                } else {
                    mbar_arrive_expect_tx(&c.full[s], tx);
                    if (ffast)
                        bulk_load_hint(fb, fl + t * TILE, TILE, &c.full[s],
                                       phase == kItemReduce ? keep : drop);
                    if (phase == kItemScan && xfast)
                        bulk_load_hint(xb, in + t * TILE, TILE_BYTES, &c.full[s], drop);
                    if (stat_bytes) {
                        bulk_load(&c.stat[s][0], rec_lo(p.rec, t & ~int64_t(1)), 16, &c.full[s]);
                        const uint32_t ch = static_cast<uint32_t>(t) / order.K;
                        bulk_load(&c.stat[s][4], rec_chunk(p.rec, ch, 0), 16, &c.full[s]);
                        bulk_load(&c.stat[s][2], rec_hi(p.rec, t & ~int64_t(1)), 16, &c.full[s]);
                    }
                }
            }
        }
        if (lane == 0) *static_cast<volatile unsigned int*>(&c.claim_sink) = cur ^ nxt;
    } else if (warp < CWARPS) {
        T* out = static_cast<T*>(p.out);
        uint32_t scan_uses = 0;
        bool scan_ok = true;
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            if (tid == 0)
                c.cflag = mbar_wait_bounded(&c.full[s], use & 1u, role_limit, hdr, epoch, true) ? 1u : 0u;
            named_barrier_sync<CTHREADS>(1);
            if (!c.cflag) break;
            const int64_t t = c.tile_id[s];
            if (t >= num_tiles) break;
            const uint32_t phase = c.phase[s];
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
            if (phase == kItemScan) {
                const T* xb = payload(s);
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) x[j] = xb[tid * ITEMS + j];
            }
            named_barrier_sync<CTHREADS>(1);  // warp totals written, payload read
            if (phase == kItemReduce) {
                if (tid == 0) {
                    unsigned long long total = 0;
                    for (int w = 0; w < CWARPS; ++w) total += c.wtot[w];
                    publish_sum_hooked<Op>(p.rec, t, epoch, cfg, false, total);
                    mbar_arrive(&c.empty[s]);
                    const int64_t ch = static_cast<uint32_t>(t) / static_cast<uint32_t>(K);
                    const int64_t first = ch * K;
                    const int64_t nch = (num_tiles - first) < K ? (num_tiles - first) : K;
                    if (t == first + nch - 1) {
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
            // ---- scan item: positions of the kept elements, gather, write --
            if (tid == 0) {
                const int64_t ch = static_cast<uint32_t>(t) / static_cast<uint32_t>(K);
                unsigned long long e, off;
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
                c.base = e + off;
                uint32_t total = 0;
                for (int w = 0; w < CWARPS; ++w) total += static_cast<uint32_t>(c.wtot[w]);
                c.kept = total;
            }
            uint32_t pos = inc - mine;  // this thread's first position in the tile's run
            for (int w = 0; w < warp; ++w) pos += static_cast<uint32_t>(c.wtot[w]);
            T* xb = payload(s);
#pragma unroll
            for (int j = 0; j < ITEMS; ++j)
                if ((m >> j) & 1u) {
                    if (pos < static_cast<uint32_t>(TILE)) xb[pos] = x[j];
                    ++pos;
                }
            named_barrier_sync<CTHREADS>(1);  // the run is gathered; base and kept are set
            const unsigned long long base = c.base;
            uint32_t kept = c.kept;
            // a run that would leave the output (only after a failed wait, which
            // has recorded its error) is not written
            if (kept > static_cast<uint32_t>(TILE) || base > static_cast<unsigned long long>(p.n) ||
                kept > static_cast<unsigned long long>(p.n) - base) {
                if (tid == 0) record_error(hdr, GBSCAN_ERR_INVALID_ARG, t);
                kept = 0;
            }
            for (uint32_t i = tid; i < kept; i += CTHREADS) out[base + i] = xb[i];
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

}  // namespace gbscan
