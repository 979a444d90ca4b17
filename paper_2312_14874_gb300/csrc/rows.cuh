// rows.cuh — row-wise scans of rows that fit in a tile: torch.cumsum(x, -1)
// forward, and its gradient, the reverse (suffix) scan of each row.
//
// A work item is k whole rows (k = TILE / cols, at least one), so no item needs
// anything from another: there is no look-back and no status word.  The
// loader warp takes items b, b + G, b + 2G, ... (static assignment: nothing
// waits on another block) and TMA-loads each into a shared-memory stage,
// right-aligned for the reverse scan; the consumer warps scan it with row-head
// flags (the segmented operator of the batched scan), the carry into every
// item being the identity because an item starts on a row boundary, and the
// result leaves with one TMA bulk store.  Rows longer than the tile go to the
// chained single-pass kernel with row heads instead.
//
// The gradient of y_k = sum_{i<=k} x_i is dx_i = sum_{k>=i} g_k (exclusive
// forward: sum_{k>i} g_k), the suffix scan of the row (Section 1's definition
// read right to left).
#pragma once

#include "tile_common.cuh"

namespace gbscan {

template <class Op, int CWARPS, int STAGES>
struct RbCtrl {
    using Acc = typename Op::Acc;
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int64_t item[STAGES];
    Acc wtot_v[CWARPS];
    uint32_t wtot_f[CWARPS];
    uint32_t epoch;
    uint32_t clear;
    uint32_t cflag;
};

template <class Op, int CWARPS, int ITEMS, int STAGES>
constexpr int rb_smem_bytes() {
    return STAGES * CWARPS * 32 * ITEMS * static_cast<int>(sizeof(typename Op::T)) +
           static_cast<int>(sizeof(RbCtrl<Op, CWARPS, STAGES>));
}

template <int CWARPS>
constexpr int rb_threads() {
    return (CWARPS + 1) * 32;
}

template <class Op, int CWARPS, int ITEMS, int STAGES, bool REVERSE, int MINB>
__global__ void __launch_bounds__((CWARPS + 1) * 32, MINB) rowblock_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int CTHREADS = CWARPS * 32;
    constexpr int TILE = CTHREADS * ITEMS;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int LOAD_WARP = CWARPS;
    static_assert(ITEMS % VEC == 0, "items per thread must fill 16-byte vectors");
    static_assert(ITEMS <= 32, "head flags are kept in one 32-bit mask");
    static_assert(STAGES >= 2, "a stage is released one store later: at least two stages");
    using CtrlT = RbCtrl<Op, CWARPS, STAGES>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * TILE_BYTES);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t cols = p.cols;
    const int64_t rows = p.n / cols;
    const int64_t k = TILE / cols;  // rows per item (the host sends cols <= TILE)
    const int64_t num_items = (rows + k - 1) / k;
    // whole items move with TMA when every row starts on a 16-byte boundary
    const bool fast = p.fast && (cols * static_cast<int64_t>(sizeof(T))) % 16 == 0;

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
    // item i: rows [i*k, min(rows, (i+1)*k)), elements [tb, tb + cnt)
    auto item_count = [&](int64_t i) -> int {
        const int64_t r = (rows - i * k) < k ? (rows - i * k) : k;
        return static_cast<int>(r * cols);
    };

    if (warp == LOAD_WARP) {
        const T* __restrict__ in = static_cast<const T*>(p.in);
        int64_t i = blockIdx.x;
        uint32_t fills = 0;  // stage fills made, in order (see drain_fills)
        for (uint32_t u = 0;; ++u, i += gridDim.x) {
            const int s = static_cast<int>(u % STAGES);
            const uint32_t use = u / STAGES;
            if (use > 0 && !warp_wait(&c.empty[s], (use - 1) & 1u, role_limit, hdr, epoch, lane))
                break;
            ++fills;
            if (i >= num_items) {
                if (lane == 0) {
                    c.item[s] = -1;  // end
                    mbar_arrive(&c.full[s]);
                }
                break;
            }
            const int cnt = item_count(i);
            const int64_t tb = i * k * cols;
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES) + (REVERSE ? TILE - cnt : 0);
            uint32_t bytes = fast ? static_cast<uint32_t>(cnt) * static_cast<uint32_t>(sizeof(T)) : 0u;
            if (!fast) {
                // rows not in whole 16-byte units: the aligned body of the item
                // by one bulk copy where source and stage allow, the rest by the
                // lanes
                const bool bulk_ok = p.fast && ((tb * static_cast<int64_t>(sizeof(T))) & 15) == 0 &&
                                     (reinterpret_cast<uintptr_t>(buf) & 15) == 0;
                bytes = warp_stage_partial<T>(buf, in + tb, cnt, cnt, bulk_ok, Op::pad(), lane);
                __syncwarp();
            }
            if (lane == 0) {
                c.item[s] = i;
                if (bytes) {
                    mbar_arrive_expect_tx(&c.full[s], bytes);
                    bulk_load(buf, in + tb, bytes, &c.full[s]);
                } else {
                    mbar_arrive(&c.full[s]);
                }
            }
        }
        if (lane == 0) drain_fills<STAGES>(c.full, fills, role_limit, hdr);
    } else {
        T* out = static_cast<T*>(p.out);
        const bool excl = p.exclusive != 0;
        int pending = -1;
        for (uint32_t u = 0;; ++u) {
            const int s = static_cast<int>(u % STAGES);
            const uint32_t use = u / STAGES;
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
            const int64_t i = c.item[s];
            if (i < 0) break;
            const int cnt = item_count(i);
            const int64_t tb = i * k * cols;
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
            const uint32_t hm = row_heads<ITEMS, REVERSE>(tb, cnt, cols, tid) & valid;
            bool tf;
            Acc tv;
            const bool wh = __any_sync(0xffffffffu, hm != 0u);
            thread_reduce_w<Op, ITEMS, kRowHeads>(x, hm, wh, tf, tv);
            bool wf = tf;
            Acc wv = tv;
            warp_inclusive_scan_w<Op, kRowHeads>(wh, wf, wv, lane);
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
            // everything before this thread's first item within the item: the
            // warps before this one, then the lanes before this one (the item
            // itself starts on a row boundary, so nothing comes from before it)
            bool gf = false;
            Acc gv = Op::identity();
            for (int w = 0; w < warp; ++w) {
                bool f2 = c.wtot_f[w] != 0;
                Acc v2 = c.wtot_v[w];
                seg_combine<Op>(gf, gv, f2, v2);
                gf = f2;
                gv = v2;
            }
            seg_combine<Op>(gf, gv, ef, ev);
            T y[ITEMS];
            thread_outputs_w<Op, ITEMS, kRowHeads>(x, hm, wh, ev, excl, y);
            store_items<T, ITEMS, TILE, REVERSE>(buf, tid, y);
            const int off = REVERSE ? TILE - cnt : 0;
            if (fast) fence_proxy_async_smem();
            named_barrier_sync<CTHREADS>(1);
            if (fast) {
                if (tid == 0) {
                    bulk_store(out + tb, buf + off,
                               static_cast<uint32_t>(cnt) * static_cast<uint32_t>(sizeof(T)));
                    bulk_commit();
                    pending = s;
                }
            } else {
                for (int j = tid; j < cnt; j += CTHREADS) out[tb + j] = buf[off + j];
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
