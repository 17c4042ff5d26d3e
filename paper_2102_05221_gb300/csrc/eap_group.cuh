// eap_group.cuh -- EAPruned DP with G = 8 or 16 lanes per pair (32/G pairs per
// warp), for series short enough that pruning granularity, not per-step
// overhead, decides the cost.
//
// The skewed wavefront of a pair is a staircase whose cells span about
// lanes x (W + 1) diagonals; everything the pair computes is the union of
// those staircases over the panel, so a narrower staircase wastes fewer
// cells outside the band of live cells (left of the first live row and
// right of the pruning point).  A G-lane group halves or quarters the span
// of the warp-per-pair mapping at the same strip width W.
//
// The groups of a warp run different pairs, so their panels start and end at
// different times.  To keep the warp converged, the kernel is one flat loop:
// (1) each group that needs a new pair or a new panel sets it up (divergent,
// group-local collectives only), (2) the warp re-converges and runs U
// wavefront steps in lock-step, every lane predicated by its own group's
// state, (3) one ballot gives each group its frontier vote, and groups whose
// panel ended process its end (divergent).  Per round a group also refreshes
// its cut-off from the query's best-so-far (a load issued one vote earlier,
// so the warp never waits for it), and the shared-memory boundary column is
// never cleared in full: rows past those the pair has written are set to
// +inf in blocks, ahead of the rows the group's first lane reads.  The
// arithmetic of a cell, the pruning rules and the results are those of
// warp_pair in the EAPruned mode (with DPJob::no_cut, of the Base mode: the
// cut-off is +inf, so every panel runs to its last row and nothing is
// abandoned).
#pragma once

#include "eap_device.cuh"

namespace eapd {

#ifndef EAP_GROUP_ROUNDS
#define EAP_GROUP_ROUNDS 2
#endif
// Register-rotation cycles (W + 1 steps each) per lock-step round.
constexpr int kGroupRounds = EAP_GROUP_ROUNDS;

template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
    return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

template <class F, int W>
constexpr int group_min_blocks() { return W <= 5 ? F::kGroupBlocks : 0; }

template <class F, int W, int G, bool WIN>
__global__ void __launch_bounds__(kThreads, (group_min_blocks<F, W>())) group_dp_kernel(const DPJob job, const KParams kp) {
    static_assert(G == 8 || G == 16, "group width");
    constexpr int P = G * W;                 // columns per panel
    constexpr int NG = 32 / G;               // groups per warp
    constexpr int U = kGroupRounds * (W + 1);   // steps per round (the strip registers rotate back every W + 1)
    constexpr int kFillRows = 64;            // boundary rows set to +inf at a time (>= U)
    static_assert(U <= kFillRows && kFillRows % G == 0, "boundary fill");
    enum { kNeedPair = 0, kNeedPanel = 1, kStep = 2, kDone = 3 };
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);           // lane within the group
    const unsigned gmask = group_mask<G>(lane);
    float* bnd = smem + ((threadIdx.x >> 5) * NG + lane / G) * job.bnd_stride;

    // Group state that only the set-up and the end of a pair or a panel read
    // lives in shared memory, so that the registers of the wavefront loop
    // hold only what a step uses (more resident warps per SM).  Every lane of
    // the group writes the same values and reads back its own writes; the
    // counters belong to the group's first lane.
    struct Cold {
        PairIn in;
        const unsigned* cut_hi;   // high word (the distance) of the query's best-so-far, or null
        unsigned long long item;
        int ai, bi, npan, p, blo, cf, cl;
        bool last;
        unsigned long long npairs, nab, nlb;
    };
    __shared__ Cold cold_all[kThreads / G];
    Cold& gc = cold_all[threadIdx.x / G];
    if (gl == 0) gc.npairs = gc.nab = gc.nlb = 0;
    unsigned long long cells = 0;

    int state = kNeedPair;
    float cut = EAP_FINF;
    unsigned cut_next = 0x7f800000u;   // best-so-far read at the last vote, taken at the next one
    int bhi = 0;
    int vhi = 0;   // rows 1..vhi of the boundary column hold this pair's values (see begin_panel)
    // What a wavefront step reads of the pair.
    const float4* rp = nullptr;   // packed row constants (F::kPacked)
    const float* Ar = nullptr;    // row series (rows computed in place)
    int La = 0;
    const float* wt = nullptr;    // WDTW weights
    int w = 0;                    // window
    // Panel state.
    int r0 = 1, r1 = 0, t = 0, nsteps = 0, c0 = 0;
    bool lane_out = true, stG = false;
    typename F::Col cc[W];
    float v[W], wr[W], cy[W];
#pragma unroll
    for (int u = 0; u < W; ++u) { v[u] = EAP_FINF; wr[u] = 0.f; cy[u] = 0.f; cc[u] = F::col(0.f, 0.f, kp); }
    float dg = EAP_FINF, sp = 0.f, s_next = 0.f, fd = 0.f;
    float4 pk_next = make_float4(0.f, 0.f, 0.f, 0.f);

    // The group leader publishes a pair's result.
    auto finish_pair = [&](float d, bool ab) {
        if (gl == 0) {
            ++gc.npairs;
            gc.nab += ab ? 1 : 0;
            const int ai = gc.ai, bi = gc.bi;
            if (job.mode == kModeNN1) {
                if (d != EAP_FINF) atomicMin(job.best + ai, pack_best(d, (unsigned)bi));
            } else if (job.mode == kModePairwise) {
                const int n = job.A.n;
                job.out[(size_t)ai * n + bi] = d;
                job.out[(size_t)bi * n + ai] = d;
            } else {
                job.out[gc.item] = d;
            }
        }
        __syncwarp(gmask);
        state = kNeedPair;
    };

    auto begin_pair = [&]() {
        unsigned long long it = 0;
        if (gl == 0) it = atomicAdd(job.counter, 1ULL);
        it = __shfl_sync(gmask, it, 0, G);
        if (it >= job.nitems) { state = kDone; return; }
        const unsigned long long item = it;
        int ai, bi;
        const unsigned long long* cut_src = nullptr;
        float c = EAP_FINF;
        if (job.mode == kModeNN1) {
            const unsigned long long rank = item / (unsigned)job.A.n;
            ai = (int)(item - rank * (unsigned)job.A.n);
            bi = job.order ? __ldg(job.order + (size_t)ai * job.B.n + rank) : (int)rank;
            if (job.cut) {
                c = __ldg(job.cut + (size_t)ai * job.B.n + bi);   // the pair's own bound (Prune)
            } else {
                cut_src = job.best + ai;
                unsigned long long cv = 0;
                if (gl == 0) cv = *(volatile const unsigned long long*)cut_src;
                cv = __shfl_sync(gmask, cv, 0, G);
                c = __uint_as_float((unsigned)(cv >> 32));
                if (job.lb && __ldg(job.lb + (size_t)ai * job.B.n + bi) > c) {   // Alg. 2
                    if (gl == 0) ++gc.nlb;
                    return;   // still kNeedPair
                }
            }
        } else if (job.mode == kModePairwise) {
            tri_decode(item, job.A.n, ai, bi);
            if (job.cut) c = __ldg(job.cut + item);
        } else {
            ai = __ldg(job.ia + item);
            bi = __ldg(job.ib + item);
            if (job.cut) c = __ldg(job.cut + item);
        }
        if (job.no_cut) { c = EAP_FINF; cut_src = nullptr; }   // Base: nothing is pruned or abandoned
        const int64_t oa = __ldg(job.A.off + ai), ob = __ldg(job.B.off + bi);
        PairIn in;
        in.A = job.A.data + oa;
        in.B = job.B.data + ob;
        in.La = __ldg(job.A.len + ai);
        in.Lb = __ldg(job.B.len + bi);
        in.bA = job.A.border ? job.A.border + oa : nullptr;
        in.bB = job.B.border ? job.B.border + ob : nullptr;
        in.wt = job.wdtw_table ? job.wdtw_table + kWdtwOff - max(in.La, in.Lb) : nullptr;
        in.rp = job.rowpack ? job.rowpack + oa : nullptr;
        in.cut_src = cut_src;
        in.w = pair_window(kp, in.La, in.Lb);
        in.cut = c;
        gc.in = in;
        gc.cut_hi = cut_src ? reinterpret_cast<const unsigned*>(cut_src) + 1 : nullptr;
        cut_next = 0x7f800000u;
        gc.item = item;
        gc.ai = ai;
        gc.bi = bi;
        gc.p = 0;
        rp = in.rp;
        Ar = in.A;
        La = in.La;
        wt = in.wt;
        w = in.w;
        cut = c;
        if (in.w < abs(in.La - in.Lb)) { finish_pair(EAP_FINF, true); return; }   // no alignment in the window
        gc.npan = (in.Lb + P - 1) / P;
        // Left boundary of panel 0: the vertical border M(r, 0) (ERP), else +inf.
        int blo = 1;
        bhi = 0;
        if (F::kBorders) {
            const int vmax = min(in.La, in.w + 1);
            int live = 0;
            for (int rr = 1; rr <= vmax; rr += G) {
                const int r = rr + gl;
                const float x = r <= vmax ? __ldg(in.bA + r - 1) : EAP_FINF;
                if (r <= vmax) bnd[r] = x;
                live += __popc(__ballot_sync(gmask, r <= vmax && x <= cut));
            }
            if (live > 0) { blo = 1; bhi = live; }   // the border increases: live rows are a prefix
        }
        vhi = F::kBorders ? min(in.La, in.w + 1) : 0;
        gc.blo = blo;
        __syncwarp(gmask);
        state = kNeedPanel;
    };

    auto begin_panel = [&]() {
        const PairIn in = gc.in;
        const int Lb = in.Lb;
        const int p = gc.p, blo = gc.blo;
        const int cf = p * P + 1;
        const int cl = min(cf + P - 1, Lb);
        const bool last = (p == gc.npan - 1);
        gc.cf = cf;
        gc.cl = cl;
        gc.last = last;
        const bool top_live = hborder<F>(in, cf - 1) <= cut;
        if (!top_live && blo > bhi) { finish_pair(EAP_FINF, true); return; }
        r0 = top_live ? 1 : blo;
        r1 = La;
        if (WIN) { r0 = max(r0, cf - w); r1 = min(La, cl + w); }
        if (r0 > r1) {
            if (last) { finish_pair(EAP_FINF, true); return; }
            __syncwarp(gmask);   // every lane has read p and blo
            gc.blo = 1;
            bhi = 0;
            vhi = 0;          // the skipped panel's cells are all outside the window
            gc.p = p + 1;
            return;   // still kNeedPanel
        }
        // The boundary column is not cleared: its rows r0 - 1 .. vhi hold this
        // pair's values of column cf - 1 (rows the previous panel computed, or
        // rows it treated as dead, whose stored value is then above the
        // cut-off or +inf), and the rows past vhi are set to +inf one round
        // ahead of the group's first lane (fill_boundary).  A value above the
        // cut-off in place of +inf changes no value at or below the cut-off.
        if (r0 - 1 > vhi) {
            if (gl == 0) bnd[r0 - 1] = EAP_FINF;
            vhi = r0 - 1;
        }
        c0 = cf + gl * W;
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int c = c0 + u;
            const float tv = c <= Lb ? __ldg(in.B + c - 1) : kPadValue;
            const float tprev = c == 1 ? 0.f : (c - 1 <= Lb ? __ldg(in.B + c - 2) : kPadValue);
            cc[u] = F::col(tv, tprev, kp);
            v[u] = (r0 == 1) ? hborder<F>(in, c <= Lb ? c : Lb + 1) : EAP_FINF;
        }
        init_weights<F, W, WIN>(wr, wt, kp, r0, c0, fd, w);
        {
            const float s_before = r0 >= 2 ? __ldg(in.A + r0 - 2) : 0.f;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if constexpr (F::kCarry) cy[u] = F::carry_init(s_before, cc[u]);
                else cy[u] = 0.f;
            }
        }
        if (r0 == 1) dg = hborder<F>(in, c0 - 1 <= Lb ? c0 - 1 : Lb + 1);
        else dg = (gl == 0) ? bnd[r0 - 1] : EAP_FINF;
        lane_out = c0 > Lb;
        stG = !last && gl == G - 1;
        if constexpr (F::kPacked) {
            pk_next = __ldg(rp + r0 - 1);
        } else {
            sp = r0 >= 2 ? __ldg(Ar + r0 - 2) : 0.f;
            s_next = __ldg(Ar + r0 - 1);
        }
        nsteps = r1 - r0 + G;
        t = 0;
        state = kStep;
    };

    // End of the current panel after `done` steps.
    auto end_panel = [&](int done) {
        const int Lb = gc.in.Lb, cf = gc.cf, p = gc.p;
        {
            const int lastrow = min(r1, r0 + done - 1 - gl);
            const int nvalid = max(0, min(W, Lb - c0 + 1));
            if (lastrow >= r0) cells += (unsigned long long)(lastrow - r0 + 1) * (unsigned)nvalid;
        }
        __syncwarp(gmask);
        if (gc.last) {
            const int off = Lb - cf;         // offset of column Lb inside the panel
            const int lr = off / W, ur = off % W;
            float res = EAP_FINF;
#pragma unroll
            for (int u = 0; u < W; ++u) if (u == ur) res = v[u];
            res = __shfl_sync(gmask, res, lr, G);
            const int lastrow = min(r1, r0 + done - 1 - lr);
            if (lastrow != La) res = EAP_FINF;
            if (!(res <= cut)) res = EAP_FINF;
            finish_pair(res, res == EAP_FINF);
            return;
        }
        // Live rows of the column handed to the next panel.
        const int wlast = min(r1, r0 + done - 1 - (G - 1));
        int lo = 0x7fffffff, hi = -1;
        for (int r = r0 + gl; r <= wlast; r += G) {
            if (bnd[r] <= cut) { lo = min(lo, r); hi = max(hi, r); }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(gmask, lo, o, G));
            hi = max(hi, __shfl_xor_sync(gmask, hi, o, G));
        }
        if (hi < 0) { gc.blo = 1; bhi = 0; } else { gc.blo = lo; bhi = hi; }
        vhi = max(wlast, r0 - 1);   // the next panel reads rows from r0 - 1 on
        gc.p = p + 1;
        __syncwarp(gmask);
        state = kNeedPanel;
    };

    // One wavefront step for every group, predicated by each lane's state
    // (CHECK) or, when every lane of the warp is inside its panel's rows for
    // the whole round, unpredicated.
    auto step = [&](int tt, auto check) {
        constexpr bool kCheck = decltype(check)::value;
        const int row = r0 + tt - gl;
        const bool act = kCheck ? (state == kStep && row >= r0 && row <= r1) : true;
        // Every lane loads (the first lane's value is used) into a register
        // of its own, independent of the shuffle's result.
        const float bv = act ? bnd[row] : EAP_FINF;
        float x = __shfl_up_sync(EAP_FULL, v[W - 1], 1, G);
        if (gl == 0) x = bv;
        if (act) {
            typename F::Row rc;
            if constexpr (F::kPacked) {
                rc = F::unpack(pk_next);
                pk_next = __ldg(rp + row);   // row <= La: the entry past La is readable
            } else {
                const float s = s_next;
                s_next = __ldg(Ar + min(row, La - 1));
                rc = F::row(s, sp, kp, wt);
                sp = s;
            }
            shift_weights<F, W, WIN>(wr, wt, kp, row, c0, fd, w);
            strip_row<F, W, WIN>(v, cy, wr, cc, rc, dg, x, row - c0, w, kp);
            dg = x;
            if (stG) bnd[row] = v[W - 1];
        }
    };

    for (;;) {
        // (1) Set-up, per group; every pass consumes a work item or a panel.
        while (state == kNeedPair || state == kNeedPanel) {
            if (state == kNeedPair) begin_pair();
            else begin_panel();
        }
        // fill_boundary: +inf into the rows of the boundary column that the
        // group's first lane reads this round and no panel of the pair wrote.
        if (state == kStep && min(r0 + t + U - 1, r1) > vhi) {
#pragma unroll
            for (int k = 0; k < kFillRows / G; ++k) {
                const int r = vhi + 1 + gl + k * G;
                if (r <= r1) bnd[r] = EAP_FINF;
            }
            vhi = min(vhi + kFillRows, r1);
        }
        __syncwarp();
        if (__ballot_sync(EAP_FULL, state == kStep) == 0u) break;   // every group is done
        // (2) U lock-step wavefront steps; unpredicated when every group is
        // stepping with all its lanes inside the panel's rows (no ramp).
        const bool steady = __all_sync(EAP_FULL, state == kStep && t >= G - 1 && t + U <= r1 - r0 + 1);
        if (steady) {
#pragma unroll
            for (int k = 0; k < U; ++k) step(t + k, BoolC<false>{});
        } else {
#pragma unroll
            for (int k = 0; k < U; ++k) step(t + k, BoolC<true>{});
        }
        // (3) Frontier vote: every cell a later row of this panel could depend
        // on (each lane's strip and left input, the group's first lane's
        // unread boundary rows) is above the cut-off.
        bool dead = true;
        if (state == kStep) {
            // The best-so-far read at the previous vote (its load had a round
            // to complete) tightens the cut-off; the next read starts now.
            cut = fminf(cut, __uint_as_float(cut_next));
            const unsigned* ch = gc.cut_hi;
            if (ch) cut_next = *(volatile const unsigned*)ch;
            const int row = r0 + t + U - 1 - gl;
            if (row <= r1 && !lane_out) {
                float m = dg;
#pragma unroll
                for (int u = 0; u < W; ++u) m = fminf(m, v[u]);
                dead = m > cut;
                if (gl == 0 && row < bhi) dead = false;
            }
        }
        const bool gdead = (__ballot_sync(EAP_FULL, dead) & gmask) == gmask;
        if (state == kStep) {
            t += U;
            if (gdead || t >= nsteps) end_panel(gdead ? t : nsteps);
        }
    }
    if (job.stats) {
        unsigned long long npairs = 0, nab = 0, nlb = 0;
        if (gl == 0) { npairs = gc.npairs; nab = gc.nab; nlb = gc.nlb; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cells += __shfl_xor_sync(EAP_FULL, cells, o);
            npairs += __shfl_xor_sync(EAP_FULL, npairs, o);
            nab += __shfl_xor_sync(EAP_FULL, nab, o);
            nlb += __shfl_xor_sync(EAP_FULL, nlb, o);
        }
        if (lane == 0) {
            if (npairs) atomicAdd(job.stats + kStatPairs, npairs);
            if (nab) atomicAdd(job.stats + kStatAbandoned, nab);
            if (cells) atomicAdd(job.stats + kStatCells, cells);
            if (nlb) atomicAdd(job.stats + kStatLbPruned, nlb);
        }
    }
}

}  // namespace eapd
