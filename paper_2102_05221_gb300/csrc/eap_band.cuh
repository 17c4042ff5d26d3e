// eap_band.cuh -- the DP of a windowed distance (CDTW, ERP) in band
// coordinates: Base (Alg. 3, every cell) and, with a cut-off, early
// abandoning with the EAPruned result contract.
//
// Cell (i, j) of the window |i - j| <= w, together with the two border cells
// that Section 2.3.2's computed borders reach (M(w+1, 0) and M(0, w+1)), is
// stored at (i, k) with k = j - i + w + 1, k in [0, 2w + 2].  A row of the
// band is then one contiguous run of cells, and a group of G lanes covers it
// with P = G * W >= 2w + 3 cells (W consecutive k per lane).  The pair's rows
// run as a skewed wavefront: lane l computes row s - l at step s.
//
// In these coordinates the diagonal predecessor (i-1, j-1) is (i-1, k), the
// vertical one (i-1, j) is (i-1, k+1) and the horizontal one (i, j-1) is
// (i, k-1).  A lane's last cell needs the vertical predecessor held by the
// next lane's first cell one row up, which that lane computes in the same
// step; so each step computes the lane's first cell, hands it to the left
// neighbour (shuffle down), then computes the other cells, and the last
// cell reaches the right neighbour (shuffle up) for the next step.  A cell's
// column j = i + k - w - 1 grows by one per row, so the column constants move
// one cell to the left per step and each lane loads one new column per step
// (from L1: a shuffle from the right neighbour measured slower).
//
// Cells outside the series (j < 1 or j > L_B) see the column value +inf:
// their point cost is +inf.  The recurrence then gives +inf everywhere it
// should, and at k = 0 for i <= w + 1 it gives the vertical border: ERP's
// min(+inf, M(i-1, 0) + cost(s_i, g), +inf) is the border's own prefix sum,
// DTW's is +inf.  Cells with k >= 2w + 2 (right of the window) get a +inf
// addend; the cell k = 0 is set to +inf from row w + 2 on (left of the
// window).  Row 0 holds M(0, 0) = 0 and the horizontal border.  Every cell
// applies the distance's own cell() to the same predecessor values as the
// other Base kernels, so the results are bit-identical to theirs.
//
// With a cut-off (PM = kPmPruned: 1-NN with the shared best-so-far, or
// explicit per-item cut-offs) the kernel abandons a pair as soon as every
// cell of the wavefront's current cut exceeds the cut-off, and returns
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


template <class F, int W, int G, int PM>
__global__ void __launch_bounds__(kThreads, EAP_BAND_MINB) band_dp_kernel(const DPJob job, const KParams kp) {
    static_assert(G == 8 || G == 16 || G == 32, "group width");
    static_assert(W >= 2, "strip width");
    static_assert(PM == kPmBase || PM == kPmPruned, "mode");
    constexpr bool CUT = PM == kPmPruned;
    constexpr int P = G * W;   // band cells per row
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = group_mask<G>(lane);
    const int c0 = gl * W;     // first band cell of this lane
    unsigned long long cells = 0, npairs = 0, nab = 0, nlb = 0, nerr = 0;

    for (;;) {
        unsigned long long it = 0;
        if (gl == 0) it = atomicAdd(job.counter, 1ULL);
        it = __shfl_sync(gmask, it, 0, G);
        if (it >= job.nitems) break;
        int ai, bi;
        if (job.mode == kModeNN1) {
            const unsigned long long rank = it / (unsigned)job.A.n;
            ai = (int)(it - rank * (unsigned)job.A.n);
            bi = job.order ? __ldg(job.order + (size_t)ai * job.B.n + rank) : (int)rank;
        } else if (job.mode == kModePairwise) {
            tri_decode(it, job.A.n, ai, bi);
        } else {
            ai = __ldg(job.ia + it);
            bi = __ldg(job.ib + it);
        }
        const int64_t oa = __ldg(job.A.off + ai), ob = __ldg(job.B.off + bi);
        const float* A = job.A.data + oa;
        const float* B = job.B.data + ob;
        const float* bB = job.B.border ? job.B.border + ob : nullptr;
        const float4* rp = job.rowpack ? job.rowpack + oa : nullptr;
        // Cut-off: the pair's own (Prune, explicit pairs) or the query's
        // shared best-so-far (1-NN), refreshed at every abandoning test.
        float cut = EAP_FINF;
        const unsigned long long* cut_src = nullptr;
        if (CUT) {
            if (job.mode == kModeNN1) {
                if (job.cut) {
                    cut = __ldg(job.cut + (size_t)ai * job.B.n + bi);
                } else {
                    cut_src = job.best + ai;
                    unsigned long long cv = 0;
                    if (gl == 0) cv = *(volatile const unsigned long long*)cut_src;
                    cv = __shfl_sync(gmask, cv, 0, G);
                    cut = __uint_as_float((unsigned)(cv >> 32));
                    if (job.lb && __ldg(job.lb + (size_t)ai * job.B.n + bi) > cut) {   // Alg. 2
                        if (gl == 0) ++nlb;
                        continue;
                    }
                }
            } else if (job.cut) {
                cut = __ldg(job.cut + it);
            }
        }
        const int La = __ldg(job.A.len + ai), Lb = __ldg(job.B.len + bi);
        const int w = pair_window(kp, La, Lb);
        float d = EAP_FINF;
        if (w >= abs(La - Lb) && 2 * w + 3 > P) {
            d = __int_as_float(0x7fc00000);   // band wider than the launch: never chosen by the host
            if (gl == 0) ++nerr;
        } else if (w >= abs(La - Lb)) {
            // +inf addend right of the window (k >= 2w + 2); fixed per cell.
            float msk[W];
#pragma unroll
            for (int u = 0; u < W; ++u) msk[u] = (c0 + u <= 2 * w + 1) ? 0.f : EAP_FINF;
            auto column = [&](int j) {
                return F::col(j >= 1 && j <= Lb ? __ldg(B + j - 1) : EAP_FINF, 0.f, kp);
            };
            // Row 0 (M(0, j), j = k - w - 1) and the columns of row 1 (j = k - w).
            float v[W];
            typename F::Col cc[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const int j = c0 + u - w - 1;
                float top = EAP_FINF;
                if (j == 0) top = 0.f;
                else if (F::kBorders && j >= 1 && j <= w + 1 && j <= Lb) top = __ldg(bB + j - 1);
                v[u] = top;
                cc[u] = column(j + 1);
            }
            float s_next = 0.f;
            float4 pk_next = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (F::kPacked) pk_next = __ldg(rp);
            else s_next = __ldg(A);
            // One step: row i = s - gl of this lane (inactive outside 1..La).
            auto step = [&](int s, auto check) {
                constexpr bool kCheck = decltype(check)::value;
                const int i = s - gl;
                const bool act = kCheck ? (i >= 1 && i <= La) : true;
                float x = __shfl_up_sync(gmask, v[W - 1], 1, G);
                if (gl == 0) x = EAP_FINF;
                typename F::Row rc;
                if constexpr (F::kPacked) {
                    rc = F::unpack(pk_next);
                    if (act) pk_next = __ldg(rp + min(i, La));   // entry La is readable
                } else {
                    rc = F::row(s_next, 0.f, kp, nullptr);
                    if (act) s_next = __ldg(A + min(i, La - 1));
                }
                // The +inf addend right of the window stays off the row's
                // left-to-right chain: the cells it applies to are a suffix of
                // the row, so a masked cell's right neighbour is masked too.
                float nv[W];
                float lf = F::cell(v[0], v[1], x, rc, cc[0], 0, 0.f, kp);
                if (gl == 0 && i >= w + 2) lf = EAP_FINF;   // (i, i - w - 1): left of the window
                nv[0] = __fadd_rn(lf, msk[0]);
                const float pub = act ? nv[0] : v[0];
                float y = __shfl_down_sync(gmask, pub, 1, G);
                if (gl == G - 1) y = EAP_FINF;
#pragma unroll
                for (int u = 1; u < W; ++u) {
                    lf = F::cell(v[u], u + 1 < W ? v[u + 1] : y, lf, rc, cc[u], 0, 0.f, kp);
                    nv[u] = __fadd_rn(lf, msk[u]);
                }
                if (act) {
#pragma unroll
                    for (int u = 0; u < W; ++u) v[u] = nv[u];
#pragma unroll
                    for (int u = 0; u + 1 < W; ++u) cc[u] = cc[u + 1];
                    cc[W - 1] = column(i + 1 + c0 + W - 1 - w - 1);   // column of the last cell in row i + 1
                }
            };
            // Abandoning test on the cut of each lane's newest row.
            auto dead = [&]() -> bool {
                if (cut_src) {
                    unsigned long long cv = 0;
                    if (gl == 0) cv = *(volatile const unsigned long long*)cut_src;
                    cv = __shfl_sync(gmask, cv, 0, G);
                    cut = fminf(cut, __uint_as_float((unsigned)(cv >> 32)));
                }
                float m = v[0];
#pragma unroll
                for (int u = 1; u < W; ++u) m = fminf(m, v[u]);
                return (__ballot_sync(gmask, !(m > cut)) & gmask) == 0u;
            };
            const int nsteps = La + G - 1;
            int s = 1;
            bool ab = false;
            // Ramp-in: lanes start one step apart.
            for (; s < G && s <= nsteps; ++s) step(s, BoolC<true>{});
            if (CUT) ab = dead();
            // Every lane active: steps G .. La, W at a time (the column
            // registers rotate back after W steps).
            for (; !ab && s + W - 1 <= La; s += W) {
#pragma unroll
                for (int k = 0; k < W; ++k) step(s + k, BoolC<false>{});
                if (CUT) ab = dead();
            }
            if (!ab) {
                for (; s <= nsteps; ++s) step(s, BoolC<true>{});
            }
            cells += (unsigned long long)max(0, min(La, s - 1 - gl)) * W;   // rows this lane computed
            if (!ab) {
                // M(L_A, L_B) sits at k = L_B - L_A + w + 1.
                const int kf = Lb - La + w + 1;
                const int lane_f = kf / W, uf = kf - lane_f * W;
                float r = EAP_FINF;
#pragma unroll
                for (int u = 0; u < W; ++u) if (u == uf) r = v[u];
                d = __shfl_sync(gmask, r, lane_f, G);
                if (CUT && !(d <= cut)) d = EAP_FINF;
            }
        }
        if (gl == 0) {
            ++npairs;
            nab += (CUT && d == EAP_FINF) ? 1 : 0;
            if (job.mode == kModeNN1) {
                if (d != EAP_FINF) atomicMin(job.best + ai, pack_best(d, (unsigned)bi));
            } else if (job.mode == kModePairwise) {
                const int n = job.A.n;
                job.out[(size_t)ai * n + bi] = d;
                job.out[(size_t)bi * n + ai] = d;
            } else {
                job.out[it] = d;
            }
        }
        __syncwarp(gmask);
    }
    if (job.stats) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            cells += __shfl_xor_sync(gmask, cells, o, G);
            npairs += __shfl_xor_sync(gmask, npairs, o, G);
            nab += __shfl_xor_sync(gmask, nab, o, G);
            nlb += __shfl_xor_sync(gmask, nlb, o, G);
            nerr += __shfl_xor_sync(gmask, nerr, o, G);
        }
        if (gl == 0) {
            if (npairs) atomicAdd(job.stats + kStatPairs, npairs);
            if (nab) atomicAdd(job.stats + kStatAbandoned, nab);
            if (cells) atomicAdd(job.stats + kStatCells, cells);
            if (nlb) atomicAdd(job.stats + kStatLbPruned, nlb);
            if (nerr) atomicAdd(job.stats + kStatErrors, nerr);
        }
    }
}

}  // namespace eapd
