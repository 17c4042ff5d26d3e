// eap_band.cuh -- the DP of a windowed distance (CDTW, ERP) in band
// coordinates: Base (Alg. 3, every cell) and, with a cut-off, early
// abandoning with the EAPruned result contract.
//
// Layout.  Cell (i, j) is stored at band position p = j - i + w + 1 of row i.
// The window |i - j| <= w is p in [1, 2w + 1]; p = 0 is the cell left of the
// window, (i, i - w - 1), which is the vertical border M(w + 1, 0) in row
// w + 1 (ERP's computed border reaches index w + 1, Section 2.3.2) and +inf in
// every later row.  A group of G lanes holds P = G * W positions of a row, W
// consecutive positions per lane, and runs the pair's rows as a skewed
// wavefront: lane l computes row s - l at step s.
//
// In these coordinates the diagonal predecessor (i-1, j-1) is (i-1, p), the
// vertical one (i-1, j) is (i-1, p+1) and the horizontal one (i, j-1) is
// (i, p-1).  A lane's last cell needs the vertical predecessor that the next
// lane computes in the same step as its first cell, so each step computes
// the lane's first cell, hands it to the left neighbour (shuffle down),
// then the other cells; the last cell reaches the right neighbour (shuffle
// up) as the next step's horizontal input.  A cell's column j = i + p - w - 1
// grows by one per row, so the column constants move one position to the
// left per step and each lane loads one new column per step.  Columns
// outside the series (j < 1 or j > L_B) are +inf, which makes the cell's
// point cost +inf: the recurrence then yields +inf there and, at j = 0,
// ERP's vertical border (its own prefix sum).  Row 0 holds M(0, 0) = 0 and
// the top border.
//
// Right of the window.  An exact launch has P = 2w + 2: the window's last
// cell is the last position of the last lane, its vertical predecessor from
// row i - 1 is outside the window (+inf), except in row 1, where it is ERP's
// top border cell M(0, w + 1).  A padded launch (P >= 2w + 3) adds a +inf
// addend to the positions right of the window; that addend stays off the
// row's left-to-right chain, because those positions are a suffix of the row.
//
// Lock-step groups.  The 32 / G groups of a warp run different pairs.  The
// kernel is one flat loop: groups that need a pair set one up (divergent,
// group-local collectives only), then the whole warp runs W wavefront steps
// (the column registers rotate back after W steps), unpredicated when every
// lane of every group is inside its pair's rows 2 .. L_A - 1 for the whole
// round, predicated otherwise; one ballot gives each group its abandoning
// vote and every group whose pair ended publishes its result.  Every cell
// applies the distance's recurrence to the same predecessor values as the
// column-panel kernels, with the same roundings, so the results are
// bit-identical to theirs.
//
// With a cut-off (PM = kPmPruned: 1-NN with the shared best-so-far, or
// explicit per-item cut-offs) a pair is abandoned as soon as every cell of
// the wavefront's current cut exceeds the cut-off, and the kernel returns
// D(A, B) when D <= cut-off, else +inf -- the EAPruned contract.  The cut is
// each lane's newest row: a path leaving the computed region does so from a
// lane's newest row (the left lane is a row ahead, so a vertical step into it
// stays inside; a horizontal step into the right lane, a row behind, leaves
// from the newest row), so when all of them exceed the cut-off, so does D
// (Alg. 4's abandoning test on this cut).  Pruning inside a row (Alg. 5's
// skipped cells) would save no work here: the lanes compute the band row in
// lock-step either way.
#pragma once

#include "eap_device.cuh"

namespace eapd {

#ifndef EAP_BAND_MINB
#define EAP_BAND_MINB 0
#endif


template <int G>
__device__ __forceinline__ unsigned band_group_mask(int lane) {
    return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// One row of a lane's strip in band coordinates, per distance: `first` is
// the lane's first cell (diagonal dg, vertical tp, horizontal lf); `rest`
// updates cells 1 .. W-1 in place (v[u] is the diagonal predecessor,
// v[u+1] -- or y, the next lane's first cell, for the last one -- the
// vertical predecessor, the cell to the left the horizontal one) with an
// optional +inf addend per position.  The terms that do not depend on the
// cell to the left run on neighbouring cells in pairs (f32x2).
template <class F>
struct BandCell;

template <int COST>
struct BandCell<FDtw<COST>> {
    using F = FDtw<COST>;
    __device__ static float first(float dg, float tp, float lf, const typename F::Row& r,
                                  const typename F::Col& c) {
        const float m = min3f(dg, tp, lf);
        const float d = __fsub_rn(r.s, c.t);
        return COST == 0 ? __fmaf_rn(d, d, m) : __fadd_rn(fabsf(d), m);
    }
    template <int W, bool MSK>
    __device__ static void rest(float (&v)[W], float y, float lf, const typename F::Row& r,
                                const typename F::Col (&cc)[W], const float (&msk)[W]) {
        float d[W];
#pragma unroll
        for (int u = 1; u + 1 < W; u += 2) {
            const float2 d2 = sub2_rn(make_float2(r.s, r.s), make_float2(cc[u].t, cc[u + 1].t));
            d[u] = d2.x;
            d[u + 1] = d2.y;
        }
        if constexpr ((W - 1) % 2 == 1) d[W - 1] = __fsub_rn(r.s, cc[W - 1].t);
#pragma unroll
        for (int u = 1; u < W; ++u) {
            const float tp = u + 1 < W ? v[u + 1] : y;
            const float m = min3f(v[u], tp, lf);
            float nv = COST == 0 ? __fmaf_rn(d[u], d[u], m) : __fadd_rn(fabsf(d[u]), m);
            if (MSK) nv = __fadd_rn(nv, msk[u]);
            v[u] = nv;
            lf = nv;
        }
    }
};

template <int COST>
struct BandCell<FErp<COST>> {
    using F = FErp<COST>;
    __device__ static float diag(float d, float g) { return COST == 0 ? __fmaf_rn(d, d, g) : __fadd_rn(g, fabsf(d)); }
    __device__ static float first(float dg, float tp, float lf, const typename F::Row& r,
                                  const typename F::Col& c) {
        const float a = diag(__fsub_rn(r.s2.x, c.t), dg);
        return min3f(a, __fadd_rn(tp, r.cs2.x), __fadd_rn(lf, c.ct));
    }
    template <int W, bool MSK>
    __device__ static void rest(float (&v)[W], float y, float lf, const typename F::Row& r,
                                const typename F::Col (&cc)[W], const float (&msk)[W]) {
        auto fin = [&](int u, float a, float b) {
            float nv = min3f(a, b, __fadd_rn(lf, cc[u].ct));
            if (MSK) nv = __fadd_rn(nv, msk[u]);
            v[u] = nv;
            lf = nv;
        };
#pragma unroll
        for (int u = 1; u + 1 < W; u += 2) {
            const float2 d2 = sub2_rn(r.s2, make_float2(cc[u].t, cc[u + 1].t));
            const float tp1 = u + 2 < W ? v[u + 2] : y;
            const float2 b2 = __fadd2_rn(make_float2(v[u + 1], tp1), r.cs2);
            const float a0 = diag(d2.x, v[u]), a1 = diag(d2.y, v[u + 1]);
            fin(u, a0, b2.x);
            fin(u + 1, a1, b2.y);
        }
        if constexpr ((W - 1) % 2 == 1) {
            constexpr int u = W - 1;
            fin(u, diag(__fsub_rn(r.s2.x, cc[u].t), v[u]), __fadd_rn(y, r.cs2.x));
        }
    }
};

template <class F, int W, int G, int PM, bool EXACT>
__global__ void __launch_bounds__(kThreads, EAP_BAND_MINB) band_dp_kernel(const DPJob job, const KParams kp) {
    static_assert(G == 4 || G == 8 || G == 16, "group width");
    static_assert(W >= 2, "strip width");
    static_assert(PM == kPmBase || PM == kPmPruned, "mode");
    using BC = BandCell<F>;
    using Col = typename F::Col;
    constexpr bool CUT = PM == kPmPruned;
    constexpr int P = G * W;   // band positions per row
    constexpr int U = W;       // wavefront steps per lock-step round
    enum { kNeedPair = 0, kStep = 1, kDone = 2 };
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = band_group_mask<G>(lane);
    const int c0 = gl * W;     // first band position of this lane

    // What only the set-up and the end of a pair read lives in shared
    // memory (every lane writes the same values; the counters belong to the
    // group's first lane), so the wavefront's registers hold what a step uses.
    struct Cold {
        unsigned long long item;
        int ai, bi;
        unsigned long long npairs, nab, nlb, nerr;
    };
    __shared__ Cold cold_all[kThreads / G];
    Cold& gc = cold_all[threadIdx.x / G];
    if (gl == 0) gc.npairs = gc.nab = gc.nlb = gc.nerr = 0;
    unsigned long long cells = 0;

    int state = kNeedPair;
    float cut = EAP_FINF;
    const unsigned long long* cut_src = nullptr;
    int La = 0, Lb = 0, w = 0;
    int s = 1;                       // next wavefront step of the group's pair
    const float* Ar = nullptr;       // row series
    const float4* rp = nullptr;      // packed row constants (F::kPacked)
    const float* Bp = nullptr;       // column series
    int jb = 0;                      // the column this lane loads in step t is j = t + jb
    float yR = EAP_FINF;             // exact launch, ERP: M(0, w + 1)
    Col cc[W];
    float v[W], msk[W];
#pragma unroll
    for (int u = 0; u < W; ++u) { v[u] = EAP_FINF; msk[u] = 0.f; cc[u] = F::col(EAP_FINF, 0.f, kp); }
    float s_next = 0.f;
    float4 pk_next = make_float4(0.f, 0.f, 0.f, 0.f);

    auto column = [&](int j) -> Col {
        return F::col((unsigned)(j - 1) < (unsigned)Lb ? __ldg(Bp + (j - 1)) : EAP_FINF, 0.f, kp);
    };

    // The group's first lane publishes a pair's result; `rows` wavefront
    // steps were run (0: the pair was decided before any).
    auto finish = [&](float d, bool ab, int steps) {
        const int rows = max(0, min(La, steps - gl));
        const int nvalid = max(0, min(c0 + W - 1, 2 * w + 1) - max(c0, 1) + 1);
        cells += (unsigned long long)rows * (unsigned)nvalid;
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
        int ai, bi;
        float c = EAP_FINF;
        cut_src = nullptr;
        if (job.mode == kModeNN1) {
            const unsigned long long rank = it / (unsigned)job.A.n;
            ai = (int)(it - rank * (unsigned)job.A.n);
            bi = job.order ? __ldg(job.order + (size_t)ai * job.B.n + rank) : (int)rank;
            if (CUT) {
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
            }
        } else if (job.mode == kModePairwise) {
            tri_decode(it, job.A.n, ai, bi);
            if (CUT && job.cut) c = __ldg(job.cut + it);
        } else {
            ai = __ldg(job.ia + it);
            bi = __ldg(job.ib + it);
            if (CUT && job.cut) c = __ldg(job.cut + it);
        }
        gc.item = it;
        gc.ai = ai;
        gc.bi = bi;
        const int64_t oa = __ldg(job.A.off + ai), ob = __ldg(job.B.off + bi);
        La = __ldg(job.A.len + ai);
        Lb = __ldg(job.B.len + bi);
        w = pair_window(kp, La, Lb);
        cut = c;
        if (w < abs(La - Lb)) { finish(EAP_FINF, true, 0); return; }   // no alignment in the window
        if (EXACT ? 2 * w + 2 != P : 2 * w + 3 > P) {
            // Band and launch do not match: never chosen by the host.
            if (gl == 0) ++gc.nerr;
            finish(__int_as_float(0x7fc00000), false, 0);
            return;
        }
        Ar = job.A.data + oa;
        rp = job.rowpack ? job.rowpack + oa : nullptr;
        Bp = job.B.data + ob;
        const float* bB = job.B.border ? job.B.border + ob : nullptr;
        // Row 0: M(0, j) at p = j + w + 1.
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int p = c0 + u, j = p - w - 1;
            float top = EAP_FINF;
            if (j == 0) top = 0.f;
            else if (F::kBorders && j >= 1 && j <= w + 1 && j <= Lb) top = __ldg(bB + j - 1);
            v[u] = top;
            if (!EXACT) msk[u] = p <= 2 * w + 1 ? 0.f : EAP_FINF;
        }
        yR = (EXACT && F::kBorders && w + 1 <= Lb) ? __ldg(bB + w) : EAP_FINF;
        // Before step 1 the lane is at row 1 - gl; cell u has column
        // j = (1 - gl) + c0 + u - w - 1, and step t loads the column of its
        // last cell for the next row, j = t + jb.
        jb = c0 - gl + W - w - 1;
#pragma unroll
        for (int u = 0; u < W; ++u) cc[u] = column(jb + 1 - W + u);
        if constexpr (F::kPacked) pk_next = __ldg(rp);
        else s_next = __ldg(Ar);
        s = 1;
        state = kStep;
    };

    // One wavefront step t for every group: lane gl computes row t - gl.
    // CHECK: predicated by each lane's state; else every lane of the warp is
    // inside rows 2 .. L_A - 1 of its pair.
    auto step = [&](int t, auto check) {
        constexpr bool kCheck = decltype(check)::value;
        const int i = t - gl;
        const bool live = !kCheck || state == kStep;
        const bool act = !kCheck || (live && i >= 1 && i <= La);
        float x = __shfl_up_sync(EAP_FULL, v[W - 1], 1, G);
        if (gl == 0) x = EAP_FINF;   // left of p = 0 is outside the matrix or the window
        typename F::Row rc;
        if constexpr (F::kPacked) {
            rc = F::unpack(pk_next);
            if (!kCheck) pk_next = __ldg(rp + i);
            else if (live) pk_next = __ldg(rp + min(max(i, 0), La - 1));
        } else {
            rc = F::row(s_next, 0.f, kp, nullptr);
            if (!kCheck) s_next = __ldg(Ar + i);
            else if (live) s_next = __ldg(Ar + min(max(i, 0), La - 1));
        }
        float nv0 = BC::first(v[0], v[1], x, rc, cc[0]);
        if (!EXACT) nv0 = __fadd_rn(nv0, msk[0]);
        // p = 0 is +inf once it lies inside the matrix (row w + 2 on); before
        // that it is +inf (DTW) or ERP's vertical border by the recurrence.
        if (gl == 0 && (!F::kBorders || i >= w + 2)) nv0 = EAP_FINF;
        const float pub = act ? nv0 : v[0];
        float y = __shfl_down_sync(EAP_FULL, pub, 1, G);
        if (gl == G - 1) y = (EXACT && F::kBorders && kCheck && i == 1) ? yR : EAP_FINF;
        if (act) {
            v[0] = nv0;
            BC::template rest<W, !EXACT>(v, y, nv0, rc, cc, msk);
        }
        // Columns for the next step, on every step (they follow t, not the
        // lane's activity).
#pragma unroll
        for (int u = 0; u + 1 < W; ++u) cc[u] = cc[u + 1];
        if (live) cc[W - 1] = column(t + jb);
    };

    for (;;) {
        while (state == kNeedPair) begin_pair();
        __syncwarp();
        if (__ballot_sync(EAP_FULL, state == kStep) == 0u) break;   // every group is done
        const bool steady = __all_sync(EAP_FULL, state == kStep && s >= G + 1 && s + U <= La);
        if (steady) {
#pragma unroll
            for (int k = 0; k < U; ++k) step(s + k, BoolC<false>{});
        } else {
            // Predicated rounds (pair starts and ends) stay rolled: explicit
            // register moves for the column shift in a minority of rounds buy
            // half the kernel's code (instruction-cache misses otherwise).
#pragma unroll 1
            for (int k = 0; k < U; ++k) step(s + k, BoolC<true>{});
        }
        s += U;
        // Abandoning vote on the cut of each lane's newest row, with the
        // refreshed best-so-far.
        bool keep = true;
        if (CUT) {
            unsigned long long cv = 0;
            if (gl == 0 && state == kStep && cut_src) cv = *(volatile const unsigned long long*)cut_src;
            cv = __shfl_sync(EAP_FULL, cv, 0, G);
            if (state == kStep && cut_src) cut = fminf(cut, __uint_as_float((unsigned)(cv >> 32)));
            float m = v[0];
#pragma unroll
            for (int u = 1; u < W; ++u) m = fminf(m, v[u]);
            keep = !(m > cut);
        }
        const bool gkeep = (__ballot_sync(EAP_FULL, keep) & gmask) != 0u;
        if (state == kStep) {
            if (s > La + G - 1) {
                // M(L_A, L_B) sits at p = L_B - L_A + w + 1.
                const int pf = Lb - La + w + 1;
                const int lane_f = pf / W, uf = pf - lane_f * W;
                float r = EAP_FINF;
#pragma unroll
                for (int u = 0; u < W; ++u) if (u == uf) r = v[u];
                float d = __shfl_sync(gmask, r, lane_f, G);
                if (CUT && !(d <= cut)) d = EAP_FINF;
                finish(d, CUT && d == EAP_FINF, s - 1);
            } else if (CUT && !gkeep) {
                finish(EAP_FINF, true, s - 1);
            }
        }
    }
    if (job.stats) {
        unsigned long long npairs = 0, nab = 0, nlb = 0, nerr = 0;
        if (gl == 0) { npairs = gc.npairs; nab = gc.nab; nlb = gc.nlb; nerr = gc.nerr; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cells += __shfl_xor_sync(EAP_FULL, cells, o);
            npairs += __shfl_xor_sync(EAP_FULL, npairs, o);
            nab += __shfl_xor_sync(EAP_FULL, nab, o);
            nlb += __shfl_xor_sync(EAP_FULL, nlb, o);
            nerr += __shfl_xor_sync(EAP_FULL, nerr, o);
        }
        if (lane == 0) {
            if (npairs) atomicAdd(job.stats + kStatPairs, npairs);
            if (nab) atomicAdd(job.stats + kStatAbandoned, nab);
            if (cells) atomicAdd(job.stats + kStatCells, cells);
            if (nlb) atomicAdd(job.stats + kStatLbPruned, nlb);
            if (nerr) atomicAdd(job.stats + kStatErrors, nerr);
        }
    }
}

}  // namespace eapd
