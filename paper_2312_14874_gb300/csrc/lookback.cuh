// lookback.cuh — the single-pass chained scan with decoupled look-back.
//
// One persistent block per resident slot, warp-specialised:
//
//   loader warp   claims a tile (one atomic per tile, only once a stage is
//                 free) and starts a 1-D TMA bulk copy of it into that stage
//                 (a ragged or misaligned tile: its aligned body by one bulk
//                 copy, the rest by the lanes, padded with the operator's
//                 neutral element); with each claim it also asks L2 for the
//                 tile about 12 MiB further on, claiming nothing, so that the
//                 copy of that tile, whichever block claims it, comes from L2
//                 instead of DRAM;                                          [a1]
//   stage agents  one warp per stage: as soon as the stage's data lands it
//                 sums the tile from shared memory, publishes the aggregate,
//                 runs the two-level decoupled look-back (tiles of its 16-tile
//                 group, then group words) and publishes the inclusive prefix:
//                 the adjacent-only synchronisation that Section 2.2.1 sets
//                 against a counting barrier, with Merrill and Garland's
//                 aggregate / inclusive-prefix states.  The agent hands the
//                 tile's exclusive prefix to the consumers and only then frees
//                 the stage: a stage is refilled only when its agent is idle,
//                 so every claimed tile publishes its aggregate one copy
//                 latency after its claim, whatever other tiles are doing;  [a5]
//   consumers     NW warps read each tile out of its stage at once, in a
//                 warp-striped order (lane l of warp w takes the 16-byte
//                 vectors w*NV*32 + j*32 + l, j < NV: 512 contiguous bytes per
//                 warp and row), scan it (per-vector sums in registers, one
//                 Hillis-Steele shuffle scan per row, warp totals through
//                 shared memory), wait in registers for the tile's prefix, and
//                 write the results with 16-byte streaming stores straight
//                 from registers (again 512 contiguous bytes per warp store).
//                                                             [a2, a3, a4, a6]
//
// The consumers give the stage back as soon as they have read it, before the
// prefix is known, so while a tile waits for its prefix it occupies registers
// only; the stores hold no on-chip buffer.  On this part the rate of a chained
// scan is set by the bytes each SM keeps between a tile's claim and its
// prefix (copy latency, aggregate, look-back round trips), so the stages plus
// one tile of registers per block are what the launch shapes trade, and the
// L2 prefetch ahead of the claims takes the DRAM latency out of that time.
//
// Waits are bounded.  The consumers' stage wait and the sentinel that ends the
// work are OR-reduced across the consumer warps in the named barrier that also
// exchanges the warp totals, so every consumer warp leaves the loop at the same
// point.  The look-back honours the launch's abort mark, and an abort poisons
// the claim counter, so a launch that runs into a bound finishes the tiles its
// blocks hold and claims no more.
#pragma once

#include "tile_common.cuh"

namespace gbscan {

template <class Op, int NW, int STAGES>
struct LbCtrl {
    using Acc = typename Op::Acc;
    uint64_t full[STAGES];   // stage data landed (loader arrive + TMA bytes)
    uint64_t empty[STAGES];  // count 2: the consumers have read the stage, its agent is idle
    uint64_t ready[STAGES];  // the agent has put the tile's exclusive prefix in excl
    int64_t tile_id[STAGES];
    Acc excl[STAGES][2];     // by use parity: an agent's next write to a slot comes two uses later
    alignas(16) Acc wtot[NW];
    uint32_t epoch;
    uint32_t clear;
};

template <class Op, int NW, int NV, int STAGES>
constexpr int lb_smem_bytes() {
    return STAGES * NW * 32 * NV * 16 + static_cast<int>(sizeof(LbCtrl<Op, NW, STAGES>));
}

// Consumer warps, the loader warp and one agent warp per stage.
template <int NW, int STAGES>
constexpr int lb_threads() {
    return (NW + 1 + STAGES) * 32;
}

// 16-byte streaming store (the output is not read again by this launch).
__device__ __forceinline__ void st_stream_v4(void* p, const uint4& v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// Warp-uniform bounded wait by polling (lane 0 tests the phase, sleeping a
// few tens of nanoseconds between tests): for the waits on the critical path
// of every tile, where waking from a hardware suspend was measured to cost
// more than polling.  Gives up at `limit_ns` (recording a timeout for the
// launch) or once the launch has been aborted.
__device__ __forceinline__ bool warp_spin_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                               Header* hdr, uint32_t epoch, int lane) {
    int ok = 1;
    if (lane == 0 && !mbar_test_wait(bar, parity)) {
        const uint64_t t0 = global_timer_ns();
        uint32_t polls = 0;
        while (!mbar_test_wait(bar, parity)) {
            __nanosleep(32);
            if ((++polls & 255) == 0) {
                if (launch_aborted(hdr, epoch)) {
                    ok = 0;
                    break;
                }
                if (global_timer_ns() - t0 > limit_ns) {
                    record_timeout(hdr, epoch, -1);
                    ok = 0;
                    break;
                }
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// Sum of a whole stage by one warp: consecutive lanes on consecutive 16-byte
// vectors, SU vectors in flight per lane with independent partial sums; each
// vector is summed on its own (a run of VEC elements) and joined to its
// partial sum with `combine`.  Compensated pairs instead sum groups of four
// of a lane's vectors as a tree in plain fp32 (four roundings deep) and join
// each group's sum to one of two partial pairs.
template <class Op, int TILE, int SU>
__device__ __forceinline__ typename Op::Acc stage_sum(const unsigned char* stage, int lane) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int PER_LANE = TILE / VEC / 32;
    constexpr int U = PER_LANE < SU ? PER_LANE : SU;
    static_assert((TILE / VEC) % 32 == 0, "whole rows of vectors");
    const uint4* v4 = reinterpret_cast<const uint4*>(stage) + lane;
    if constexpr (HasPlainRow<Op>::value) {
        static_assert(VEC == 4 && PER_LANE % 4 == 0, "groups of four 4-element vectors");
        constexpr int NG = PER_LANE / 4;
        Acc part[2] = {Op::identity(), Op::identity()};
#pragma unroll
        for (int g0 = 0; g0 < NG; g0 += 2) {
            uint4 w[2][4];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (g0 + u < NG) w[u][k] = v4[((g0 + u) * 4 + k) * 32];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (g0 + u < NG) {
                    T sv[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const T* e = reinterpret_cast<const T*>(&w[u][k]);
                        sv[k] = Op::row_add(Op::row_add(e[0], e[1]), Op::row_add(e[2], e[3]));
                    }
                    const T t = Op::row_add(Op::row_add(sv[0], sv[1]), Op::row_add(sv[2], sv[3]));
                    part[u] = combine_local<Op>(part[u], Op::lift(t));
                }
            }
        }
        Acc v = combine_local<Op>(part[0], part[1]);
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) v = combine_local<Op>(v, shfl_down_acc<Op>(v, d));
        return shfl_idx_acc<Op>(v, 0);
    }
    Acc part[U];
#pragma unroll
    for (int u = 0; u < U; ++u) part[u] = Op::identity();
#pragma unroll
    for (int q0 = 0; q0 < PER_LANE; q0 += U) {
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (q0 + u < PER_LANE) w[u] = v4[(q0 + u) * 32];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (q0 + u < PER_LANE) {
                const T* e = reinterpret_cast<const T*>(&w[u]);
                Acc vs = Op::lift(e[0]);
#pragma unroll
                for (int j = 1; j < VEC; ++j) Op::accumulate(vs, e[j]);
                part[u] = combine_local<Op>(part[u], vs);
            }
        }
    }
    Acc v = part[0];
#pragma unroll
    for (int u = 1; u < U; ++u) v = combine_local<Op>(v, part[u]);
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v = combine_local<Op>(v, shfl_down_acc<Op>(v, d));
    return shfl_idx_acc<Op>(v, 0);
}

template <class Op, int NW, int NV, int STAGES, int LB, int MINB>
__global__ void __launch_bounds__((NW + 1 + STAGES) * 32, MINB) lb_scan_kernel(const Params p) {
    using T = typename Op::T;
    using Acc = typename Op::Acc;
    constexpr int NT = NW * 32;
    constexpr int VEC = 16 / static_cast<int>(sizeof(T));
    constexpr int TILE = NT * NV * VEC;
    constexpr int TILE_BYTES = TILE * static_cast<int>(sizeof(T));
    constexpr int LOAD_WARP = NW;  // warps NW+1+s: the agent of stage s
    static_assert(STAGES >= 2, "at least two stages");
    using CtrlT = LbCtrl<Op, NW, STAGES>;

    extern __shared__ __align__(128) unsigned char smem[];
    CtrlT& c = *reinterpret_cast<CtrlT*>(smem + STAGES * TILE_BYTES);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    Header* hdr = p.hdr;
    const int64_t num_tiles = p.num_tiles;

    // the loader's first claim goes out before the block's set-up, so that
    // its round trip overlaps it
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
    // pipeline waits outlast a look-back that runs into its own bound
    const uint64_t role_limit = 4 * cfg.spin_limit_ns + 10000000ull;
    auto count_of = [&](int64_t t) -> int {
        const int64_t rem = p.n - t * TILE;
        return rem < TILE ? static_cast<int>(rem) : TILE;
    };

    if (warp == LOAD_WARP) {
        // ---- a1: claim a tile whenever a stage is free, start its copy ------
        // The claim is made only when the stage is free (no claim is kept in
        // flight): a tile claimed ahead would publish its aggregate a stage
        // period late, and every later tile's look-back would wait for it
        // (measured: 0.65 instead of 0.80 of copy bandwidth).
        const T* __restrict__ in = static_cast<const T*>(p.in);
        const uint64_t evict_first = l2_policy_evict_first();
        uint32_t fills = 0;  // stage fills made, in order (see drain_fills)
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
                // no tiles left (or an aborted launch): an end sentinel in this
                // stage and in the next STAGES-1 once they are free, so that
                // every agent and the consumers leave their loops
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
            T* buf = reinterpret_cast<T*>(smem + s * TILE_BYTES);
            if (p.fast && cnt == TILE) {
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    mbar_arrive_expect_tx(&c.full[s], TILE_BYTES);
                    bulk_load_hint(buf, in + tile * TILE, TILE_BYTES, &c.full[s], evict_first);
                    // the tile prefetch_tiles ahead, into L2 for whichever block
                    // claims it: its copy then comes from L2 (no claim is made,
                    // so no tile's aggregate is delayed)
                    const int64_t pt = tile + p.prefetch_tiles;
                    if (p.prefetch_tiles > 0 && pt < num_tiles) {
                        const uint32_t pbytes =
                            (static_cast<uint32_t>(count_of(pt)) * static_cast<uint32_t>(sizeof(T))) & ~15u;
                        if (pbytes) bulk_prefetch_l2(in + pt * TILE, pbytes);
                    }
                }
            } else {
                // ragged or misaligned: the aligned body by one bulk copy where
                // possible, the rest by the lanes, padded to a whole tile
                const uint32_t bulk = warp_stage_partial<T>(buf, in + tile * TILE, cnt, TILE, p.fast,
                                                            Op::pad(), lane);
                __syncwarp();
                if (lane == 0) {
                    c.tile_id[s] = tile;
                    if (bulk) {
                        mbar_arrive_expect_tx(&c.full[s], bulk);
                        bulk_load(buf, in + tile * TILE, bulk, &c.full[s]);
                    } else {
                        mbar_arrive(&c.full[s]);
                    }
                }
            }
            ++fills;
        }
        if (lane == 0) drain_fills<STAGES>(c.full, fills, role_limit, hdr);
    } else if (warp > LOAD_WARP) {
        // ---- a5: the stage's agent: aggregate, look-back, prefix -----------
        const int s = warp - LOAD_WARP - 1;
        for (uint32_t use = 0;; ++use) {
            if (!warp_spin_wait(&c.full[s], use & 1u, role_limit, hdr, epoch, lane)) break;
            const int64_t tile = *static_cast<volatile int64_t*>(&c.tile_id[s]);
            if (tile >= num_tiles) break;
            const Acc agg = stage_sum<Op, TILE, 2 * NV>(smem + s * TILE_BYTES, lane);
            __syncwarp();
            if (lane == 0) publish_aggregate<Op>(p.rec, tile, epoch, cfg, false, agg);
            bool ef;
            Acc ev;
            lookback<Op, kNoHeads, LB>(p.rec, hdr, tile, epoch, cfg, false, agg, lane, ef, ev);
            if (lane == 0) {
                c.excl[s][use & 1u] = ev;
                mbar_arrive(&c.ready[s]);
                mbar_arrive(&c.empty[s]);  // idle again: the stage may be refilled
            }
        }
    } else {
        // ---- a2-a4, a6: consumers -------------------------------------------
        T* out = static_cast<T*>(p.out);
        const bool excl = p.exclusive != 0;
        const int vbase = warp * NV * 32 + lane;  // this lane's first vector in the tile
        for (uint32_t k = 0;; ++k) {
            const int s = static_cast<int>(k % STAGES);
            const uint32_t use = k / STAGES;
            const bool ok = warp_spin_wait(&c.full[s], use & 1u, role_limit, hdr, epoch, lane);
            const int64_t tile = *static_cast<volatile int64_t*>(&c.tile_id[s]);
            bool stop = !ok || tile >= num_tiles;
            const int cnt = stop ? 0 : count_of(tile);
            const int64_t tb = stop ? 0 : tile * TILE;
            // the lane's vectors (a ragged tile was padded in the stage)
            T x[NV][VEC];
            const uint4* st4 = reinterpret_cast<const uint4*>(smem + s * TILE_BYTES);
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const uint4 q = st4[vbase + j * 32];
                const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
                for (int i = 0; i < VEC; ++i) x[j][i] = e[i];
            }
            // vector sums, then one shuffle scan per row of the warp
            Acc ex[NV];  // everything of the row before this lane's vector
            Acc rt[NV];  // row totals
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                if constexpr (HasPlainRow<Op>::value) {
                    // the row in the element type, its results lifted
                    static_assert(VEC == 4, "4-element vectors");
                    T inc = Op::row_add(Op::row_add(x[j][0], x[j][1]), Op::row_add(x[j][2], x[j][3]));
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const T o = __shfl_up_sync(0xffffffffu, inc, d);
                        if (lane >= d) inc = Op::row_add(o, inc);
                    }
                    const T e = __shfl_up_sync(0xffffffffu, inc, 1);
                    ex[j] = lane == 0 ? Op::identity() : Op::lift(e);
                    rt[j] = Op::lift(__shfl_sync(0xffffffffu, inc, 31));
                } else {
                    Acc v = Op::lift(x[j][0]);
#pragma unroll
                    for (int i = 1; i < VEC; ++i) Op::accumulate(v, x[j][i]);
                    Acc inc = v;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const Acc o = shfl_up_acc<Op>(inc, d);
                        if (lane >= d) inc = combine_local<Op>(o, inc);
                    }
                    ex[j] = shfl_up_acc<Op>(inc, 1);
                    if (lane == 0) ex[j] = Op::identity();
                    rt[j] = shfl_idx_acc<Op>(inc, 31);
                }
            }
            Acc wtot = rt[0];
#pragma unroll
            for (int j = 1; j < NV; ++j) wtot = combine_local<Op>(wtot, rt[j]);
            if (lane == 0) c.wtot[warp] = wtot;
            // warp totals exchanged; every consumer warp agrees on going on
            stop = named_barrier_or<NT>(1, stop);
            if (stop) break;
            if (tid == 0) mbar_arrive(&c.empty[s]);  // every consumer has read the stage
            Acc woff = Op::identity();
#pragma unroll
            for (int w = 0; w < NW; ++w)
                if (w < warp) woff = combine_local<Op>(woff, c.wtot[w]);
            warp_spin_wait(&c.ready[s], use & 1u, role_limit, hdr, epoch, lane);
            Acc base = Op::combine(c.excl[s][use & 1u], woff);  // before the warp's first row
            named_barrier_sync<NT>(1);  // warp totals read before the next tile writes them
            T* o = static_cast<T*>(out) + tb;
            const bool whole = p.fast && cnt == TILE;
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const Acc carry = combine_local<Op>(base, ex[j]);
                base = combine_local<Op>(base, rt[j]);
                T y[VEC];
                Acc r = run_init<Op>(carry);
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    if (excl) {
                        y[i] = i == 0 ? Op::output1(carry) : Op::output(carry, r);
                        Op::accumulate(r, x[j][i]);
                    } else {
                        Op::accumulate(r, x[j][i]);
                        y[i] = Op::output(carry, r);
                    }
                }
                const int v = vbase + j * 32;
                if (whole) {
                    uint4 q;
                    T* e = reinterpret_cast<T*>(&q);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) e[i] = y[i];
                    st_stream_v4(o + v * VEC, q);
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; ++i)
                        if (v * VEC + i < cnt) o[v * VEC + i] = y[i];
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
