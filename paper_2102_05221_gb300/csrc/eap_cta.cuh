// eap_cta.cuh -- CTA-per-pair EAPruned DP for long series.
//
// The eight warps of a CTA share one (A, B) pair.  The columns are cut into
// panels of 32*W as in the warp-per-pair kernel; warp w sweeps panels
// w, w+8, w+16, ... each as the same skewed wavefront (lane k at row r0+t-k,
// left input from lane k-1 by shuffle).  Panel p's left boundary is panel
// p-1's last column, written by another warp: inside a round of eight panels
// through a 512-row ring in shared memory, and from the last warp of a round
// to warp 0 of the next round through a full column.
//
// The warps advance in lockstep "ticks" of kTick wavefront steps separated by
// __syncthreads_and, which both publishes the boundary rows written during
// the tick and takes the CTA-wide abandon vote.  A static schedule makes every
// read safe: panel p starts at tick S(p) = (p / 8) * T_round + (p % 8) * lag,
// with lag = 1 + ceil((dr0 + 31) / kTick) (dr0 = how much later panel p's
// rows start than panel p-1's) and T_round >= max(sweep ticks + lag,
// 8 * lag).  Then a boundary row is always written at least one tick before
// it is read, and a ring slot is rewritten only after its reader is done.
// No warp ever spins on another.
//
// Pruning: the pair is abandoned as soon as every lane's frontier is dead
// (Section 4: no live cell can be reached) -- the frontier being each lane's
// newest cells, the live boundary rows its panel has not read yet, and the
// live boundary rows waiting for each warp's next panel -- and a warp whose
// panel frontier is dead while its left neighbour has finished stops that
// panel early (pruning on the right); its consumer then reads +inf past the
// last live row.
#pragma once

#include "eap_device.cuh"

namespace eapd {

constexpr int kCtaWarps = 8;
constexpr int kCtaThreads = 32 * kCtaWarps;
// Wavefront steps per tick.  128: unwindowed (the only form this kernel
// runs), a panel's producer leads its consumer by lag = 2 ticks plus 31 rows
// at most, inside the 512-row ring; against 64, half the barriers and votes
// (1-NN at L = 8192: DTW 12.2 -> 11.3 ms, MSM 63.0 -> 61.3 ms, TWE 56.4 ->
// 54.9 ms; 32 is slower still).
constexpr int kTick = 128;
constexpr int kRing = 512;         // rows per in-round link
constexpr int kCtaMaxPanels = 512;

struct CtaShared {
    float ring[kCtaWarps - 1][kRing];
    int live_hi[kCtaMaxPanels];    // last row of panel p's output column with a value <= cut
    int done[kCtaMaxPanels];       // panel p has written everything it will write
    float cut_next;
    float result;
    unsigned long long item;
};

// Packed row constants in the CTA wavefront: MSM gains (one load instead of
// the per-row reciprocals); TWE, whose carried costs already hold many
// registers, is measured faster computing them per row.
template <class F>
constexpr bool kCtaPacked = F::kPacked && !F::kCarry;

template <class F, int W, bool PRUNE, bool WIN>
__device__ float cta_pair(const PairIn& in, CtaShared& sh, float* __restrict__ wrapcol, const KParams& kp,
                          unsigned long long& cells, bool& abandoned) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int La = in.La, Lb = in.Lb, w = in.w;
    constexpr int P = 32 * W;
    constexpr int kCtaChunk = 64 / W;      // unrolled steps per chunk (16 at W = 4, 8 at W = 8)
    static_assert(kTick % kCtaChunk == 0, "chunks tile a tick");
    const int npan = (Lb + P - 1) / P;
    float cut = PRUNE ? in.cut : EAP_FINF;   // the caller passes a CTA-uniform value
    abandoned = false;

    auto pr0 = [&](int p) { return WIN ? max(1, p * P + 1 - w) : 1; };
    auto pr1 = [&](int p) { return WIN ? min(La, min(p * P + P, Lb) + w) : La; };
    auto plen = [&](int p) { return max(0, pr1(p) - pr0(p) + 1) + 31; };   // sweep steps of panel p
    const int dr0 = WIN ? min(P, La) : 0;
    const int lag = 1 + (dr0 + 31 + kTick - 1) / kTick;
    // The ring holds a round's boundary rows between producer and consumer:
    // the lead lag * kTick + 31 must stay below kRing.  Unwindowed, dr0 = 0
    // and lag = 2; a window would shift every panel's rows by a panel width
    // (the window keeps the warp or band mappings).
    static_assert(!WIN, "the CTA mapping runs unwindowed series only");
    static_assert(2 * kTick + 31 < kRing, "ring too short for the tick");
    int len_max = 0;
    for (int q = 0; q < npan; ++q) len_max = max(len_max, plen(q));
    const int T_round = max((len_max + kTick - 1) / kTick + lag, kCtaWarps * lag);
    auto S = [&](int p) { return (p / kCtaWarps) * T_round + (p % kCtaWarps) * lag; };
    const int total_ticks = S(npan - 1) + (plen(npan - 1) + kTick - 1) / kTick;

    // Vertical border (ERP): live rows 1..bhi0 of column 0, read from global.
    int bhi0 = 0;
    if (F::kBorders) {
        const int vmax = min(La, w + 1);
        int live = 0;
        for (int r0 = 1; r0 <= vmax; r0 += 32) {
            const int r = r0 + lane;
            const float x = r <= vmax ? __ldg(in.bA + r - 1) : EAP_FINF;
            live += __popc(__ballot_sync(EAP_FULL, r <= vmax && x <= cut));
        }
        bhi0 = live;
    }
    for (int p = threadIdx.x; p < npan; p += blockDim.x) { sh.live_hi[p] = 0; sh.done[p] = 0; }
    if (threadIdx.x == 0) sh.result = EAP_FINF;
    __syncthreads();

    // Lane and cell of the last panel that hold M(La, Lb).
    const int res_lane = (Lb - 1 - (npan - 1) * P) / W;
    const int res_u = (Lb - 1 - (npan - 1) * P) % W;

    // Per-warp panel state.
    int p = warp;            // current panel of this warp
    bool have = false, pdead = false;
    int t = 0, r0 = 1, r1 = 0, c0 = 1, len = 0, my_live_hi = 0;
    bool wrote_live = false;   // this lane handed a live boundary row to its consumer during this tick
    typename F::Col cc[W];
    float v[W], cy[W], wr[W];
    float dg = EAP_FINF, sp = 0.f, s_next = 0.f, fd = 0.f;
    float4 pk_next = make_float4(0.f, 0.f, 0.f, 0.f);   // packed row constants, one row ahead (F::kPacked)
    bool lane_out = false;

    // Where lane 0 reads its left input and lane 31 writes its output during
    // a tick.  They change only at the tick barriers: the producer's live
    // rows seen at the start of a tick cover every row read in it (a
    // boundary row is written at least one tick before it is read, and a row
    // past the producer's last live row is above the cut-off, so +inf stands
    // in for it).
    const float* lsrc = nullptr;   // shared-memory column of the left neighbour (panels > 0)
    int lmask = 0, llo = 1, lhi = 0;
    float* odst = nullptr;         // shared-memory column this panel feeds (null for the last panel)
    int omask = 0;
    auto left_in = [&](int row) -> float {   // lane 0's left input at `row` of panel p
        if (row < llo || row > lhi) return EAP_FINF;
        return p == 0 ? __ldg(in.bA + row - 1) : lsrc[row & lmask];
    };
    auto put_out = [&](int row, float x) {   // lane 31's output at `row` of panel p
        if (odst == nullptr) return;
        odst[row & omask] = x;
        if (x <= cut) { my_live_hi = row; wrote_live = true; }
    };

    for (int tick = 0; tick < total_ticks; ++tick) {
        wrote_live = false;
        const bool active = p < npan && tick >= S(p);
        if (active) {
            if (!have) {
                have = true;
                pdead = false;
                t = 0;
                r0 = pr0(p);
                r1 = pr1(p);
                len = plen(p);
                c0 = p * P + 1 + lane * W;
                my_live_hi = 0;
                const int cf = p * P + 1;
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const int c = c0 + u;
                    const float tv = c <= Lb ? __ldg(in.B + c - 1) : kPadValue;
                    const float tprev = c == 1 ? 0.f : (c - 1 <= Lb ? __ldg(in.B + c - 2) : kPadValue);
                    cc[u] = F::col(tv, tprev, kp);
                    v[u] = (r0 == 1) ? hborder<F>(in, c <= Lb ? c : Lb + 1) : EAP_FINF;
                }
                const float s_before = r0 >= 2 ? __ldg(in.A + r0 - 2) : 0.f;
                init_weights<F, W, WIN>(wr, in.wt, kp, r0, c0, fd, w);
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    if constexpr (F::kCarry) cy[u] = F::carry_init(s_before, cc[u]);
                    else cy[u] = 0.f;
                }
                if (r0 == 1) dg = hborder<F>(in, c0 - 1 <= Lb ? c0 - 1 : Lb + 1);
                else dg = (lane == 0) ? left_in(r0 - 1) : EAP_FINF;
                (void)cf;
                sp = s_before;
                s_next = __ldg(in.A + r0 - 1);
                if constexpr (kCtaPacked<F>) pk_next = __ldg(in.rp + r0 - 1);
                lane_out = c0 > Lb;
            }
            const bool is_last = p == npan - 1;
            const int t_end = min((tick - S(p) + 1) * kTick, len);
            if (!pdead) {
                if (p == 0) {
                    llo = 1;
                    lhi = bhi0;
                } else {
                    const int q = p - 1;
                    const bool wrap = q % kCtaWarps == kCtaWarps - 1;
                    lsrc = wrap ? wrapcol : sh.ring[q % kCtaWarps];
                    lmask = wrap ? 0x7fffffff : kRing - 1;
                    llo = pr0(q);
                    lhi = min(pr1(q), sh.live_hi[q]);
                }
                const bool owrap = p % kCtaWarps == kCtaWarps - 1;
                odst = is_last ? nullptr : (owrap ? wrapcol : sh.ring[p % kCtaWarps]);
                omask = owrap ? 0x7fffffff : kRing - 1;
                // One wavefront step; CHECK predicates the lanes outside the
                // panel's rows (ramp at the start, rows past r1 at the end).
                auto step = [&](int tt, auto check) {
                    constexpr bool kCheck = decltype(check)::value;
                    const int row = r0 + tt - lane;
                    const bool act = kCheck ? (row >= r0 && row <= r1) : true;
                    const float bv = (lane == 0 && act) ? left_in(row) : EAP_FINF;
                    float x = __shfl_up_sync(EAP_FULL, v[W - 1], 1);
                    if (lane == 0) x = bv;
                    if (act) {
                        typename F::Row rc;
                        if constexpr (kCtaPacked<F>) {
                            rc = F::unpack(pk_next);
                            pk_next = __ldg(in.rp + row);   // row <= La: the entry past La is readable
                        } else {
                            const float s = s_next;
                            s_next = __ldg(in.A + min(row, La - 1));
                            rc = F::row(s, sp, kp, in.wt);
                            sp = s;
                        }
                        shift_weights<F, W, WIN>(wr, in.wt, kp, row, c0, fd, w);
                        strip_row<F, W, WIN>(v, cy, wr, cc, rc, dg, x, row - c0, w, kp);
                        dg = x;
                        if (lane == 31) put_out(row, v[W - 1]);
                    }
                };
                // A step of an unpredicated chunk: lane 0 takes its left input
                // (loaded for the chunk, one row per lane) from lane k, and
                // lane k keeps lane 31's output of the step.
                auto chunk_step = [&](int tt, int k, float lb, float& ob) {
                    const int row = r0 + tt - lane;
                    float x = __shfl_up_sync(EAP_FULL, v[W - 1], 1);
                    const float xb = __shfl_sync(EAP_FULL, lb, k);
                    if (lane == 0) x = xb;
                    typename F::Row rc;
                    if constexpr (kCtaPacked<F>) {
                        rc = F::unpack(pk_next);
                        pk_next = __ldg(in.rp + row);   // row <= La: the entry past La is readable
                    } else {
                        const float s = s_next;
                        s_next = __ldg(in.A + min(row, La - 1));
                        rc = F::row(s, sp, kp, in.wt);
                        sp = s;
                    }
                    shift_weights<F, W, WIN>(wr, in.wt, kp, row, c0, fd, w);
                    strip_row<F, W, WIN>(v, cy, wr, cc, rc, dg, x, row - c0, w, kp);
                    dg = x;
                    const float o = __shfl_sync(EAP_FULL, v[W - 1], 31);
                    if (lane == k) ob = o;
                };
                // Unpredicated chunks of kCtaChunk steps while every lane's
                // rows stay inside [r0, r1]; single predicated steps otherwise.
                // A chunk reads lane 0's left inputs and writes lane 31's
                // outputs with one coalesced access each (lane j: step j).
                while (t < t_end) {
                    if (t >= 31 && t + kCtaChunk <= t_end && t + kCtaChunk - 1 <= r1 - r0) {
                        float lb = EAP_FINF, ob = 0.f;
                        {
                            const int brow = r0 + t + lane;   // lane 0's row at step t + lane
                            if (lane < kCtaChunk && brow >= llo && brow <= lhi)
                                lb = p == 0 ? __ldg(in.bA + brow - 1) : lsrc[brow & lmask];
                        }
#pragma unroll
                        for (int k = 0; k < kCtaChunk; ++k) chunk_step(t + k, k, lb, ob);
                        if (odst != nullptr) {
                            const int orow = r0 + t + lane - 31;   // lane 31's row at step t + lane
                            if (lane < kCtaChunk) odst[orow & omask] = ob;
                            const unsigned live = __ballot_sync(EAP_FULL, lane < kCtaChunk && ob <= cut);
                            if (live != 0u && lane == 31) {
                                my_live_hi = r0 + t + (31 - __clz(live)) - 31;
                                wrote_live = true;
                            }
                        }
                        t += kCtaChunk;
                    } else {
                        step(t, BoolC<true>{});
                        ++t;
                    }
                }
                // M(La, Lb), once the lane holding it has computed row La (its
                // strip is not touched again: later rows are past r1).
                if (is_last && lane == res_lane && min(r1, r0 + t - 1 - lane) == La) {
                    float res = EAP_FINF;
#pragma unroll
                    for (int u = 0; u < W; ++u) if (u == res_u) res = v[u];
                    sh.result = res;
                }
            } else {
                t = t_end;
            }
            // Panel finished (or stopped dead) after this tick?
            if (t >= len) {
                const int lastrow = min(r1, r0 + t - 1 - lane);
                if (!pdead && lastrow >= r0)
                    cells += (unsigned long long)(lastrow - r0 + 1) * (unsigned)max(0, min(W, Lb - c0 + 1));
                if (lane == 31) sh.live_hi[p] = max(sh.live_hi[p], my_live_hi);
                if (lane == 0) sh.done[p] = 1;
                p += kCtaWarps;
                have = false;
            } else if (lane == 31) {
                sh.live_hi[p] = my_live_hi;
            }
        }
        // CTA-wide vote: every lane's frontier dead means no live cell is reachable.
        // A live boundary row written during this tick counts as frontier until
        // its consumer can see it (after this tick's barrier).
        bool dead = !wrote_live;
        if (have && !pdead) {
            const int row = r0 + t - 1 - lane;   // last row this lane processed (or < r0: not started)
            if (row <= r1 && !lane_out) {
                float m = dg;
#pragma unroll
                for (int u = 0; u < W; ++u) m = fminf(m, v[u]);
                dead = dead && m > cut;
                if (lane == 0) {
                    const int nxt = r0 + t;   // lane 0's next row
                    const int live_left = (p == 0) ? bhi0 : sh.live_hi[p - 1];
                    if (nxt <= live_left) dead = false;
                }
            }
        }
        if (lane == 0) {
            // The next panel this warp has not started yet (the one after its
            // current panel, or the one it waits for): live rows its producer
            // has already written, or a live top border above it, are still
            // frontier.  The producer can be far ahead of this warp: the last
            // panel of a round starts 7 lags into the round, long before warp
            // 0 finishes its panel of that round and takes up the next.
            const int pn = have ? p + kCtaWarps : p;
            if (pn < npan) {
                if (pn > 0 && sh.live_hi[pn - 1] > 0) dead = false;
                if (hborder<F>(in, pn * P) <= cut) dead = false;
            }
        }
        if (threadIdx.x == 0) {
            if (PRUNE && in.cut_src) sh.cut_next = __uint_as_float((unsigned)(*(volatile const unsigned long long*)in.cut_src >> 32));
            else sh.cut_next = cut;
        }
        const int all_dead = __syncthreads_and(dead ? 1 : 0);
        if (PRUNE && all_dead) break;   // nothing live is left to compute
        if (PRUNE) cut = fminf(cut, sh.cut_next);
        // A warp whose panel frontier is dead, with its left neighbour done and
        // no unread live boundary row, stops the rest of that panel.
        if (PRUNE && have && !pdead) {
            bool wdead = dead;
            if (lane == 0) {
                const bool left_done = (p == 0) || sh.done[p - 1];
                const int live_left = (p == 0) ? bhi0 : sh.live_hi[p - 1];
                wdead = wdead && left_done && (r0 + t > live_left);
            }
            if (__all_sync(EAP_FULL, wdead)) {
                pdead = true;
                const int lastrow = min(r1, r0 + t - 1 - lane);
                if (lastrow >= r0)
                    cells += (unsigned long long)(lastrow - r0 + 1) * (unsigned)max(0, min(W, Lb - c0 + 1));
                if (lane == 31) sh.live_hi[p] = my_live_hi;
                __syncwarp();
                if (lane == 0) sh.done[p] = 1;
                p += kCtaWarps;
                have = false;
            }
        }
    }
    __syncthreads();
    float res = sh.result;
    __syncthreads();
    if (PRUNE && !(res <= cut)) res = EAP_FINF;
    if (res == EAP_FINF) abandoned = true;
    return res;
}

}  // namespace eapd

namespace eapd {

// Persistent CTA-per-pair kernel (1-NN, all-pairs and explicit pairs as
// dp_kernel); one pair per CTA at a time.
template <class F, int W, bool PRUNE>
__global__ void __launch_bounds__(kCtaThreads, F::kCtaBlocks) cta_dp_kernel(const DPJob job, const KParams kp) {
    __shared__ CtaShared sh;
    extern __shared__ float wrapcol[];
    unsigned long long cells = 0, npairs = 0, nab = 0, nlb = 0;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(job.counter, 1ULL);
        __syncthreads();
        const unsigned long long item = sh.item;
        if (item >= job.nitems) break;
        int ai, bi;
        const unsigned long long* cut_src = nullptr;
        float cut = EAP_FINF;
        if (job.mode == kModeNN1) {
            const unsigned long long rank = item / (unsigned)job.A.n;
            ai = (int)(item - rank * (unsigned)job.A.n);
            bi = job.order ? __ldg(job.order + (size_t)ai * job.B.n + rank) : (int)rank;
            cut_src = job.best + ai;
            if (PRUNE && threadIdx.x == 0) sh.cut_next = __uint_as_float((unsigned)(*(volatile const unsigned long long*)cut_src >> 32));
        } else if (job.mode == kModePairwise) {
            tri_decode(item, job.A.n, ai, bi);
            if (PRUNE && job.cut && threadIdx.x == 0) sh.cut_next = __ldg(job.cut + item);
            else if (threadIdx.x == 0) sh.cut_next = EAP_FINF;
        } else {
            ai = __ldg(job.ia + item);
            bi = __ldg(job.ib + item);
            if (PRUNE && job.cut && threadIdx.x == 0) sh.cut_next = __ldg(job.cut + item);
            else if (threadIdx.x == 0) sh.cut_next = EAP_FINF;
        }
        __syncthreads();
        if (PRUNE) cut = sh.cut_next;
        __syncthreads();
        if (job.mode == kModeNN1 && PRUNE && job.lb && __ldg(job.lb + (size_t)ai * job.B.n + bi) > cut) {
            ++nlb;
            continue;
        }
        PairIn in;
        const int64_t oa = __ldg(job.A.off + ai), ob = __ldg(job.B.off + bi);
        in.A = job.A.data + oa;
        in.B = job.B.data + ob;
        in.La = __ldg(job.A.len + ai);
        in.Lb = __ldg(job.B.len + bi);
        in.bA = job.A.border ? job.A.border + oa : nullptr;
        in.bB = job.B.border ? job.B.border + ob : nullptr;
        in.wt = job.wdtw_table ? job.wdtw_table + kWdtwOff - max(in.La, in.Lb) : nullptr;
        in.cut_src = cut_src;
        in.rp = job.rowpack ? job.rowpack + oa : nullptr;
        in.w = pair_window(kp, in.La, in.Lb);
        in.cut = cut;
        bool ab = false;
        float d;
        if (in.w < abs(in.La - in.Lb)) { d = EAP_FINF; ab = true; }
        else d = cta_pair<F, W, PRUNE, false>(in, sh, wrapcol, kp, cells, ab);
        ++npairs;
        nab += ab ? 1 : 0;
        if (threadIdx.x == 0) {
            if (job.mode == kModeNN1) {
                if (d != EAP_FINF) atomicMin(job.best + ai, pack_best(d, (unsigned)bi));
            } else if (job.mode == kModePairwise) {
                const int n = job.A.n;
                job.out[(size_t)ai * n + bi] = d;
                job.out[(size_t)bi * n + ai] = d;
            } else {
                job.out[item] = d;
            }
        }
        __syncthreads();
    }
    if (job.stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cells += __shfl_xor_sync(EAP_FULL, cells, o);
        if ((threadIdx.x & 31) == 0 && cells) atomicAdd(job.stats + kStatCells, cells);
        if (threadIdx.x == 0) {
            if (npairs) atomicAdd(job.stats + kStatPairs, npairs);
            if (nab) atomicAdd(job.stats + kStatAbandoned, nab);
            if (nlb) atomicAdd(job.stats + kStatLbPruned, nlb);
        }
    }
}

}  // namespace eapd
