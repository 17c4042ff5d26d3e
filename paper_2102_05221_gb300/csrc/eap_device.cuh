// eap_device.cuh -- device side of libeap: per-distance cell functors and the
// warp-per-pair EAPruned wavefront (sm_103a).
//
// Method: Herrmann & Webb, arXiv 2102.05221.  The recurrence is Eq. (Common):
//   M(i,j) = min( M(i-1,j-1) + Canonical, M(i-1,j) + AlternateRow, M(i,j-1) + AlternateColumn )
// with each distance's borders and step costs (Section 2.3).
//
// Pruning on the GPU.  Alg. 5 prunes with left-to-right row scans
// (next_start / pruning_point).  A warp cannot scan a row serially, so the
// kernel uses the fact both of Alg. 5's strategies rest on (Section 4.1/4.2):
// every step cost is >= 0, so a cell is never below its smallest dependency.
// Hence (a) a cell whose dependencies all exceed the cut-off exceeds it too,
// and (b) replacing any value above the cut-off by +inf changes no value at or
// below the cut-off (the dependency a live cell takes its minimum from is
// itself <= the cell <= cut-off; float rounding is monotone, so this holds
// bit for bit).  The kernel therefore prunes whole blocks of cells whenever
// all their inputs are dead, abandons when no live cell can be reached
// (the row-abandon of Alg. 5), and returns D exactly when D <= cut-off,
// +inf otherwise -- the EAPruned contract of Section 2.2.
//
// Mapping.  One warp owns one (row series A, column series B) pair.  Columns
// are cut into panels of 32*W; in a panel lane k owns W consecutive columns
// and the warp sweeps the panel's rows as a skewed wavefront: at step t lane
// k computes row r0 + t - k, taking its left input from lane k-1 through
// __shfl_up_sync (lane 0 takes it from the previous panel's last column,
// kept in shared memory).  A panel starts at the first row where its left
// boundary (or top border) can be live -- pruning from the left -- and stops
// as soon as every cell a later row could depend on is dead -- pruning on
// the right; the pair is abandoned when a panel hands no live cell to the
// next one.  The dead-frontier test is a __all_sync over the lanes every
// few steps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define EAP_FINF __int_as_float(0x7f800000)
#define EAP_FULL 0xffffffffu

namespace eapd {

// Window value that means "no constraint" (kept small enough that 2*w fits in int).
constexpr int kNoWindow = 1 << 28;

// ---------------------------------------------------------------------------
// Parameters as the kernels see them (filled by the host from eap_params).
// ---------------------------------------------------------------------------
struct KParams {
    float wdtw_g, wdtw_wmax;
    float erp_gap;
    float msm_c;
    float twe_nu2;       // 2 * nu (the match cost's nu * (|i-j| + |(i-1)-(j-1)|))
    float twe_nu, twe_lambda;
    const float* wdtw_w; // WDTW weights: wdtw_w[2*d + kWdtwOff - L] = wmax / (1 + exp(-g (d - L/2)))
    int window_abs;      // >= 0 absolute window
    float window_ratio;  // used when window_abs < 0 (< 0: none)
    int windowed;        // CDTW / ERP
    int pad_;
};

constexpr int kWdtwOff = 1 << 14;   // index offset of the universal WDTW table (covers |2d - L| <= 16384)
template <bool B>
struct BoolC { static constexpr bool value = B; };

#ifndef EAP_STEADY_UNROLL
#define EAP_STEADY_UNROLL 0
#endif
// Steps per unrolled steady-state iteration (0: W + 1).
constexpr int kSteadyUnroll = EAP_STEADY_UNROLL;

constexpr float kPadValue = 1.0e30f; // value of the columns past a series' end inside a panel

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

#ifndef EAP_X2
#define EAP_X2 1
#endif
#ifndef EAP_X2_TWE
#define EAP_X2_TWE EAP_X2
#endif
#ifndef EAP_X2_DTW
#define EAP_X2_DTW EAP_X2
#endif
// Resident blocks per SM that group_dp_kernel asks the register allocator
// for (strip widths up to 5; 0 leaves the choice to the compiler, which then
// takes the fewest registers that do not spill).  With the group's cold state
// in shared memory every distance's default is the fastest measured on
// 1000 x 1000 x 512 (TWE: 88 registers, 34.8 ms; capped at 80, 35.2 ms).
// Each functor's kCtaBlocks is the same for cta_dp_kernel (256 threads): 0
// for every distance but MSM, which asks for 3 (80 registers at W = 8 instead
// of 104, 3 CTAs per SM instead of 2: 1-NN at L = 8192, 66.2 -> 62.9 ms; TWE
// capped the same way measured slower, 56.5 -> 58.6 ms).
#ifndef EAP_MINB_DTW
#define EAP_MINB_DTW 0
#endif
#ifndef EAP_MINB_WDTW
#define EAP_MINB_WDTW 0
#endif
#ifndef EAP_MINB_ERP
#define EAP_MINB_ERP 0
#endif
#ifndef EAP_MINB_MSM
#define EAP_MINB_MSM 0
#endif
#ifndef EAP_MINB_TWE
#define EAP_MINB_TWE 0
#endif
// Two-cell FP32 arithmetic (add/sub/fma .f32x2 of the sm_100 family): one
// instruction applies the same operation, with the same rounding, to two
// neighbouring cells of a strip, halving the issue slots of the cost terms
// that do not depend on the cell to the left.
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

template <int COST>
__device__ __forceinline__ float pcost(float a, float b) {
    const float d = __fsub_rn(a, b);
    return COST == 0 ? __fmul_rn(d, d) : fabsf(d);
}

// Window of one pair: w = floor(r * max(L_S, L_T)) in double, or the absolute value.
__device__ __forceinline__ int pair_window(const KParams& kp, int la, int lb) {
    if (!kp.windowed) return kNoWindow;
    long long w;
    if (kp.window_abs >= 0) w = kp.window_abs;
    else if (kp.window_ratio >= 0.f) w = (long long)floor((double)kp.window_ratio * (double)(la > lb ? la : lb));
    else w = kNoWindow;
    return (int)(w < kNoWindow ? w : kNoWindow);
}

// ---------------------------------------------------------------------------
// Cell functors.  Each gives per-column constants (from t_j, t_{j-1}), per-row
// constants (from s_i, s_{i-1}) and the cell update from the three
// dependencies.  `dij` is i - j, `fdij` the same as a float.  Every operation
// uses an explicit-rounding intrinsic, so the compiler never re-associates or
// contracts differently between the DP and the diagonal upper bound, which
// evaluate the same functor along the same path.
// ---------------------------------------------------------------------------

// Eq. DTW (also CDTW, whose window is applied by the caller).
template <int COST>
struct FDtw {
    static constexpr bool kWeights = false;
    static constexpr bool kCarry = false;
    static constexpr bool kPen = false;
    static constexpr bool kBorders = false;
    static constexpr bool kPacked = false;   // the row constant is s_i itself
    static constexpr bool kX2 = EAP_X2_DTW;
    static constexpr int kGroupBlocks = EAP_MINB_DTW;
    static constexpr int kCtaBlocks = 0;
    struct Col { float t; };
    struct Row { float s; const float* wt; };
    __device__ static Col col(float t, float, const KParams&) { return {t}; }
    __device__ static Row row(float s, float, const KParams&, const float*) { return {s, nullptr}; }
    // Constants enough for the diagonal candidate alone (the diagonal-path bound).
    __device__ static Col col_diag(float t, float tp, const KParams& kp) { return col(t, tp, kp); }
    __device__ static Row row_diag(float s, float sp, const KParams& kp, const float* wt) { return row(s, sp, kp, wt); }
    __device__ static float cell(float dg, float tp, float lf, const Row& r, const Col& c, int, float,
                                 const KParams&) {
        const float m = min3f(dg, tp, lf);
        const float d = __fsub_rn(r.s, c.t);
        return COST == 0 ? __fmaf_rn(d, d, m) : __fadd_rn(fabsf(d), m);
    }
    // One row of a strip, cell() for every cell with the same operations;
    // s_i - t_j runs on neighbouring cells in pairs.
    template <int W, bool WIN>
    __device__ static void strip(float (&v)[W], float (&)[W], const float (&wr)[W], const Col (&cc)[W],
                                 const Row& rc, float dg, float lf, const KParams&) {
        float d[W];
#pragma unroll
        for (int u = 0; u + 1 < W; u += 2) {
            const float2 d2 = sub2_rn(make_float2(rc.s, rc.s), make_float2(cc[u].t, cc[u + 1].t));
            d[u] = d2.x;
            d[u + 1] = d2.y;
        }
        if constexpr (W % 2 == 1) d[W - 1] = __fsub_rn(rc.s, cc[W - 1].t);
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const float top = v[u];
            const float m = min3f(dg, top, lf);
            float nv = COST == 0 ? __fmaf_rn(d[u], d[u], m) : __fadd_rn(fabsf(d[u]), m);
            if (WIN) nv = __fadd_rn(nv, wr[u]);
            dg = top;
            v[u] = nv;
            lf = nv;
        }
    }
};

// Eq. WDTW: the point cost is weighted by w(|i-j|).
template <int COST>
struct FWdtw {
    // The weight of a cell depends on |i-j| only, so the wavefront keeps the
    // W weights of a lane's strip in registers and shifts them by one cell per
    // row (cell_w); the table lookup in cell() serves the diagonal bound.
    static constexpr bool kWeights = true;
    static constexpr bool kCarry = false;
    static constexpr bool kPen = false;
    static constexpr bool kBorders = false;
    static constexpr bool kPacked = false;
    static constexpr bool kX2 = EAP_X2_DTW;
    static constexpr int kGroupBlocks = EAP_MINB_WDTW;
    static constexpr int kCtaBlocks = 0;
    struct Col { float t; };
    struct Row { float s; const float* wt; };
    __device__ static Col col(float t, float, const KParams&) { return {t}; }
    __device__ static Row row(float s, float, const KParams&, const float* wt) { return {s, wt}; }
    __device__ static Col col_diag(float t, float tp, const KParams& kp) { return col(t, tp, kp); }
    __device__ static Row row_diag(float s, float sp, const KParams& kp, const float* wt) { return row(s, sp, kp, wt); }
    __device__ static float cell(float dg, float tp, float lf, const Row& r, const Col& c, int dij, float,
                                 const KParams&) {
        const float m = min3f(dg, tp, lf);
        const float wgt = __ldg(r.wt + 2 * abs(dij));
        return __fmaf_rn(wgt, pcost<COST>(r.s, c.t), m);
    }
    __device__ static float cell_w(float dg, float tp, float lf, const Row& r, const Col& c, float wgt) {
        return __fmaf_rn(wgt, pcost<COST>(r.s, c.t), min3f(dg, tp, lf));
    }
    // One row of a strip, cell_w() for every cell with the same operations;
    // s_i - t_j and the point cost run on neighbouring cells in pairs.
    template <int W, bool WIN>
    __device__ static void strip(float (&v)[W], float (&)[W], const float (&wr)[W], const Col (&cc)[W],
                                 const Row& rc, float dg, float lf, const KParams&) {
        static_assert(!WIN, "WDTW has no window");
        float c[W];
#pragma unroll
        for (int u = 0; u + 1 < W; u += 2) {
            const float2 d2 = sub2_rn(make_float2(rc.s, rc.s), make_float2(cc[u].t, cc[u + 1].t));
            if constexpr (COST == 0) {
                const float2 c2 = __fmul2_rn(d2, d2);
                c[u] = c2.x;
                c[u + 1] = c2.y;
            } else {
                c[u] = fabsf(d2.x);
                c[u + 1] = fabsf(d2.y);
            }
        }
        if constexpr (W % 2 == 1) c[W - 1] = pcost<COST>(rc.s, cc[W - 1].t);
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const float top = v[u];
            const float nv = __fmaf_rn(wr[u], c[u], min3f(dg, top, lf));
            dg = top;
            v[u] = nv;
            lf = nv;
        }
    }
};

// Eq. ERP: gap value g; borders are the prefix sums of cost(x_k, g).
template <int COST>
struct FErp {
    static constexpr bool kWeights = false;
    static constexpr bool kCarry = false;
    static constexpr bool kPen = false;
    static constexpr bool kBorders = true;
    static constexpr bool kPacked = true;    // row constants precomputed per point (rowpack_kernel)
    static constexpr bool kX2 = EAP_X2;
    static constexpr int kGroupBlocks = EAP_MINB_ERP;
    static constexpr int kCtaBlocks = 0;
    struct Col { float t, ct; };
    struct Row { float2 s2, cs2; };          // (s_i, s_i), (cost(s_i, g), cost(s_i, g))
    __device__ static float4 pack(const Row& r) { return make_float4(r.s2.x, r.s2.y, r.cs2.x, r.cs2.y); }
    __device__ static Row unpack(const float4& p) { return {make_float2(p.x, p.y), make_float2(p.z, p.w)}; }
    __device__ static Col col(float t, float, const KParams& kp) { return {t, pcost<COST>(t, kp.erp_gap)}; }
    __device__ static Row row(float s, float, const KParams& kp, const float*) {
        const float cs = pcost<COST>(s, kp.erp_gap);
        return {make_float2(s, s), make_float2(cs, cs)};
    }
    // On the diagonal path the vertical and horizontal candidates add to +inf:
    // their gap costs are not needed (0 keeps those candidates +inf).
    __device__ static Col col_diag(float t, float, const KParams&) { return {t, 0.f}; }
    __device__ static Row row_diag(float s, float, const KParams&, const float*) {
        return {make_float2(s, s), make_float2(0.f, 0.f)};
    }
    __device__ static float cell(float dg, float tp, float lf, const Row& r, const Col& c, int, float,
                                 const KParams&) {
        const float d = __fsub_rn(r.s2.x, c.t);
        const float a = COST == 0 ? __fmaf_rn(d, d, dg) : __fadd_rn(dg, fabsf(d));
        return min3f(a, __fadd_rn(tp, r.cs2.x), __fadd_rn(lf, c.ct));
    }
    // One row of a strip, cell() for every cell with the same operations;
    // s_i - t_j and the vertical candidate run on neighbouring cells in pairs.
    template <int W, bool WIN>
    __device__ static void strip(float (&v)[W], float (&)[W], const float (&wr)[W], const Col (&cc)[W],
                                 const Row& rc, float dg, float lf, const KParams&) {
        auto diag = [](float d, float g) { return COST == 0 ? __fmaf_rn(d, d, g) : __fadd_rn(g, fabsf(d)); };
        auto finish = [&](int u, float a, float b) {
            float nv = min3f(a, b, __fadd_rn(lf, cc[u].ct));
            if (WIN) nv = __fadd_rn(nv, wr[u]);
            v[u] = nv;
            lf = nv;
        };
#pragma unroll
        for (int u = 0; u + 1 < W; u += 2) {
            const float2 d2 = sub2_rn(rc.s2, make_float2(cc[u].t, cc[u + 1].t));
            const float2 b2 = __fadd2_rn(make_float2(v[u], v[u + 1]), rc.cs2);
            const float a0 = diag(d2.x, dg), a1 = diag(d2.y, v[u]);
            dg = v[u + 1];
            finish(u, a0, b2.x);
            finish(u + 1, a1, b2.y);
        }
        if constexpr (W % 2 == 1) {
            constexpr int u = W - 1;
            finish(u, diag(__fsub_rn(rc.s2.x, cc[u].t), dg), __fadd_rn(v[u], rc.cs2.x));
        }
    }
};

// Eq. MSM with Eq. MSMCost.  C(np, x, y) = c + dist(np, [min(x,y), max(x,y)]),
// dist = 0 when np lies between x and y, else min(|np-x|, |np-y|).  With
// e = x - np (fixed along a row for the AlternateRow cost, x = s_{i-1}, or
// along a column for the AlternateColumn cost, x = t_{j-1}) and f = y - np,
// np is between x and y exactly when f / e <= 0, and otherwise
// min(|e|, |f|) = |e| * min(f / e, 1).  So dist = |e| * sat(f * (1/e)),
// sat = clamp to [0, 1], which is one multiply with saturation (a modifier
// of the FMA pipe, no min/max) and one fused multiply-add for c + |e| * (.).
// 1/e is a per-row or per-column constant (0 when e = 0: then np is always
// between).  The products round where the printed min does not (a few ulps
// of that term); every path, the DP's and the diagonal bound's, evaluates
// this same function.
__device__ __forceinline__ float mul_sat(float a, float b) {
    float d;
    asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

struct FMsm {
    static constexpr bool kWeights = false;
    static constexpr bool kCarry = false;
    static constexpr bool kPen = false;
    static constexpr bool kBorders = false;
    static constexpr bool kPacked = true;
    static constexpr bool kX2 = EAP_X2;
    static constexpr int kGroupBlocks = EAP_MINB_MSM;
    static constexpr int kCtaBlocks = 3;
    struct Col { float t, ig, ag; };   // g = t_{j-1} - t_j: ig = 1/g (0 if g = 0), ag = |g|
    struct Row { float2 s2; float ie, ae; };   // s2 = (s_i, s_i); e = s_{i-1} - s_i: ie = 1/e (0 if e = 0), ae = |e|
    __device__ static float4 pack(const Row& r) { return make_float4(r.s2.x, r.s2.y, r.ie, r.ae); }
    __device__ static Row unpack(const float4& p) { return {make_float2(p.x, p.y), p.z, p.w}; }
    __device__ static Col col(float t, float tprev, const KParams&) {
        const float g = __fsub_rn(tprev, t);
        return {t, g != 0.f ? __frcp_rn(g) : 0.f, fabsf(g)};
    }
    __device__ static Row row(float s, float sprev, const KParams&, const float*) {
        const float e = __fsub_rn(sprev, s);
        return {make_float2(s, s), e != 0.f ? __frcp_rn(e) : 0.f, fabsf(e)};
    }
    // On the diagonal path the split/merge candidates add to +inf: no
    // reciprocals needed (0 makes those costs c, finite, and the candidates +inf).
    __device__ static Col col_diag(float t, float, const KParams&) { return {t, 0.f, 0.f}; }
    __device__ static Row row_diag(float s, float, const KParams&, const float*) { return {make_float2(s, s), 0.f, 0.f}; }
    __device__ static float cell(float dg, float tp, float lf, const Row& r, const Col& c, int, float,
                                 const KParams& kp) {
        const float f = __fsub_rn(c.t, r.s2.x);                                // t_j - s_i
        const float a = __fadd_rn(dg, fabsf(f));                               // move |s_i - t_j|
        const float tc = __fmaf_rn(r.ae, mul_sat(r.ie, f), kp.msm_c);          // C(s_i, s_{i-1}, t_j)
        const float lc = __fmaf_rn(c.ag, mul_sat(c.ig, -f), kp.msm_c);  // C(t_j, t_{j-1}, s_i)
        return min3f(a, __fadd_rn(tp, tc), __fadd_rn(lf, lc));
    }
    // One row of a strip, cell() for every cell with the same operations:
    // the terms that do not depend on the cell to the left (t_j - s_i, both
    // split/merge costs, the vertical candidate) run on neighbouring cells in
    // pairs, then the left-to-right chain (horizontal candidate and minimum).
    template <int W, bool WIN>
    __device__ static void strip(float (&v)[W], float (&)[W], const float (&wr)[W], const Col (&cc)[W],
                                 const Row& rc, float dg, float lf, const KParams& kp) {
        float a[W], b[W], lc[W];
        const float2 c2 = make_float2(kp.msm_c, kp.msm_c);
        const float2 ae2 = make_float2(rc.ae, rc.ae);
#pragma unroll
        for (int u = 0; u + 1 < W; u += 2) {
            const float2 f2 = sub2_rn(make_float2(cc[u].t, cc[u + 1].t), rc.s2);
            const float2 tc2 = __ffma2_rn(ae2, make_float2(mul_sat(rc.ie, f2.x), mul_sat(rc.ie, f2.y)), c2);
            const float2 lc2 = __ffma2_rn(make_float2(cc[u].ag, cc[u + 1].ag),
                                          make_float2(mul_sat(cc[u].ig, -f2.x), mul_sat(cc[u + 1].ig, -f2.y)), c2);
            const float2 b2 = __fadd2_rn(make_float2(v[u], v[u + 1]), tc2);
            a[u] = __fadd_rn(u == 0 ? dg : v[u - 1], fabsf(f2.x));
            a[u + 1] = __fadd_rn(v[u], fabsf(f2.y));
            b[u] = b2.x;
            b[u + 1] = b2.y;
            lc[u] = lc2.x;
            lc[u + 1] = lc2.y;
        }
        if constexpr (W % 2 == 1) {
            constexpr int u = W - 1;
            const float f = __fsub_rn(cc[u].t, rc.s2.x);
            a[u] = __fadd_rn(u == 0 ? dg : v[u - 1], fabsf(f));
            b[u] = __fadd_rn(v[u], __fmaf_rn(rc.ae, mul_sat(rc.ie, f), kp.msm_c));
            lc[u] = __fmaf_rn(cc[u].ag, mul_sat(cc[u].ig, -f), kp.msm_c);
        }
#pragma unroll
        for (int u = 0; u < W; ++u) {
            float nv = min3f(a[u], b[u], __fadd_rn(lf, lc[u]));
            if (WIN) nv = __fadd_rn(nv, wr[u]);
            v[u] = nv;
            lf = nv;
        }
    }
};

// Eq. TWE with Eq. TWECost, tau_i = i, s_0 = t_0 = 0.
template <int COST>
struct FTwe {
    static constexpr bool kWeights = false;
    // cost(s_{i-1}, t_{j-1}) of the match cost is cost(s_i, t_j) of the cell's
    // diagonal predecessor: the strip carries it from the previous row.
    static constexpr bool kCarry = true;
    // The stiffness penalty nu * (|i-j| + |(i-1)-(j-1)|) = 2 nu |i-j| is
    // constant along a diagonal: the wavefront keeps it per cell in registers
    // and shifts it by one cell per row, like WDTW's weights.
    static constexpr bool kPen = true;
    static constexpr bool kBorders = false;
    static constexpr bool kPacked = true;
    static constexpr bool kX2 = EAP_X2_TWE;
    static constexpr int kGroupBlocks = EAP_MINB_TWE;
    static constexpr int kCtaBlocks = 0;
    struct Col { float t, tprev, gb; };   // gb = cost(t_j, t_{j-1}) + nu + lambda
    struct Row { float s, sprev; float2 ga2; };   // ga2 = (ga, ga), ga = cost(s_i, s_{i-1}) + nu + lambda
    __device__ static float4 pack(const Row& r) { return make_float4(r.s, r.sprev, r.ga2.x, r.ga2.y); }
    __device__ static Row unpack(const float4& p) { return {p.x, p.y, make_float2(p.z, p.w)}; }
    __device__ static Col col(float t, float tprev, const KParams& kp) {
        return {t, tprev, __fadd_rn(__fadd_rn(pcost<COST>(t, tprev), kp.twe_nu), kp.twe_lambda)};
    }
    __device__ static Row row(float s, float sprev, const KParams& kp, const float*) {
        const float ga = __fadd_rn(__fadd_rn(pcost<COST>(s, sprev), kp.twe_nu), kp.twe_lambda);
        return {s, sprev, make_float2(ga, ga)};
    }
    // On the diagonal path the deletion candidates add to +inf: their costs
    // are not needed (0 keeps them +inf); the match cost uses s, t and their
    // predecessors as in the DP.
    __device__ static Col col_diag(float t, float tprev, const KParams&) { return {t, tprev, 0.f}; }
    __device__ static Row row_diag(float s, float sprev, const KParams&, const float*) {
        return {s, sprev, make_float2(0.f, 0.f)};
    }
    // 2 nu |i - j| for a cell with i - j = d (an integer, or its exact float).
    __device__ static float pen(const KParams& kp, int d) { return __fmul_rn(kp.twe_nu2, (float)abs(d)); }
    __device__ static float pen_f(const KParams& kp, float d) { return __fmul_rn(kp.twe_nu2, fabsf(d)); }
    __device__ static float cell(float dg, float tp, float lf, const Row& r, const Col& c, int dij, float,
                                 const KParams& kp) {
        const float gm0 = __fadd_rn(pcost<COST>(r.s, c.t), pcost<COST>(r.sprev, c.tprev));
        const float gm = __fadd_rn(gm0, pen(kp, dij));
        return min3f(__fadd_rn(dg, gm), __fadd_rn(tp, r.ga2.x), __fadd_rn(lf, c.gb));
    }
    // The same cell with cost(s_{i-1}, t_{j-1}) given (carry_in), the
    // penalty given (pn = pen(i - j)) and cost(s_i, t_j) returned for the
    // next row (carry_out).
    __device__ static float cell_c(float dg, float tp, float lf, const Row& r, const Col& c, float pn,
                                   float carry_in, float& carry_out) {
        const float c1 = pcost<COST>(r.s, c.t);
        carry_out = c1;
        const float gm = __fadd_rn(__fadd_rn(c1, carry_in), pn);
        return min3f(__fadd_rn(dg, gm), __fadd_rn(tp, r.ga2.x), __fadd_rn(lf, c.gb));
    }
    __device__ static float carry_first(const Row& r, const Col& c0) { return pcost<COST>(r.sprev, c0.tprev); }
    __device__ static float carry_init(float sprev, const Col& c) { return pcost<COST>(sprev, c.t); }
    // One row of a strip, cell_c() for every cell with the same operations:
    // s_i - t_j and the vertical candidate run on neighbouring cells in
    // pairs.  Up to W = 5 (the 16-lane groups) every term that does not
    // depend on the cell to the left comes first, then the left-to-right
    // chain (horizontal candidate and minimum): 35.1 -> 34.7 ms on
    // 1000 x 1000 x 512.  At W = 8 (the CTA mapping) the cells are finished
    // one by one, which measured faster there (L = 8192: 54.8 against
    // 56.9 ms).  Pairing the match cost and the diagonal candidate as well
    // measured slower (96 registers, register moves: 36.7 ms).
    template <int W, bool WIN>
    __device__ static void strip(float (&v)[W], float (&cy)[W], const float (&wr)[W], const Col (&cc)[W],
                                 const Row& rc, float dg, float lf, const KParams&) {
        static_assert(!WIN, "TWE has no window");
        auto pc = [](float d) { return COST == 0 ? __fmul_rn(d, d) : fabsf(d); };
        float cin = carry_first(rc, cc[0]);
        if constexpr (W > 5) {
            auto finish = [&](int u, float dgu, float c1, float bu) {
                const float gm = __fadd_rn(__fadd_rn(c1, cin), wr[u]);
                cin = cy[u];
                cy[u] = c1;
                const float nv = min3f(__fadd_rn(dgu, gm), bu, __fadd_rn(lf, cc[u].gb));
                v[u] = nv;
                lf = nv;
            };
#pragma unroll
            for (int u = 0; u + 1 < W; u += 2) {
                const float2 d2 = sub2_rn(make_float2(rc.s, rc.s), make_float2(cc[u].t, cc[u + 1].t));
                const float2 b2 = __fadd2_rn(make_float2(v[u], v[u + 1]), rc.ga2);
                const float dg0 = dg, dg1 = v[u];
                dg = v[u + 1];
                finish(u, dg0, pc(d2.x), b2.x);
                finish(u + 1, dg1, pc(d2.y), b2.y);
            }
            if constexpr (W % 2 == 1) {
                constexpr int u = W - 1;
                finish(u, dg, pc(__fsub_rn(rc.s, cc[u].t)), __fadd_rn(v[u], rc.ga2.x));
            }
            return;
        }
        float a[W], b[W];
#pragma unroll
        for (int u = 0; u + 1 < W; u += 2) {
            const float2 d2 = sub2_rn(make_float2(rc.s, rc.s), make_float2(cc[u].t, cc[u + 1].t));
            const float c1a = pc(d2.x), c1b = pc(d2.y);
            const float cina = cin, cinb = cy[u];   // cost(s_{i-1}, t_{j-1}) of both cells
            cin = cy[u + 1];
            cy[u] = c1a;
            cy[u + 1] = c1b;
            a[u] = __fadd_rn(u == 0 ? dg : v[u - 1], __fadd_rn(__fadd_rn(c1a, cina), wr[u]));
            a[u + 1] = __fadd_rn(v[u], __fadd_rn(__fadd_rn(c1b, cinb), wr[u + 1]));
            const float2 b2 = __fadd2_rn(make_float2(v[u], v[u + 1]), rc.ga2);
            b[u] = b2.x;
            b[u + 1] = b2.y;
        }
        if constexpr (W % 2 == 1) {
            constexpr int u = W - 1;
            const float c1 = pc(__fsub_rn(rc.s, cc[u].t));
            a[u] = __fadd_rn(u == 0 ? dg : v[u - 1], __fadd_rn(__fadd_rn(c1, cin), wr[u]));
            b[u] = __fadd_rn(v[u], rc.ga2.x);
            cy[u] = c1;
        }
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const float nv = min3f(a[u], b[u], __fadd_rn(lf, cc[u].gb));
            v[u] = nv;
            lf = nv;
        }
    }
};

// ---------------------------------------------------------------------------
// One pair, one warp.
// ---------------------------------------------------------------------------
struct PairIn {
    const float* A;      // row series (length La)
    const float* B;      // column series (length Lb)
    const float* bA;     // ERP: bA[k] = M(k+1, 0) unwindowed prefix sum over A (else unused)
    const float* bB;     // ERP: bB[k] = M(0, k+1)
    const float* wt;     // WDTW: weight of |i-j| = d is wt[2d]
    const float4* rp;    // packed row constants of A (rp[i-1] for row i; one readable entry past La) when F::kPacked
    const unsigned long long* cut_src;  // best-so-far to refresh from (nn1), or null
    int La, Lb;
    int w;               // window (kNoWindow when none)
    float cut;           // cut-off at the start
};

// Top border M(0, j) of the column series (j >= 0).
template <class F>
__device__ __forceinline__ float hborder(const PairIn& in, int j) {
    if (j == 0) return 0.f;
    if (F::kBorders && j <= in.w + 1 && j <= in.Lb) return __ldg(in.bB + j - 1);
    return EAP_FINF;
}

// Applies one row of a lane's strip: v[u] holds M(row-1, c0+u) on entry and
// M(row, c0+u) on exit; dg = M(row-1, c0-1), lf = M(row, c0-1).
template <class F, int W, bool WIN>
__device__ __forceinline__ void strip_row(float (&v)[W], float (&cy)[W], const float (&wr)[W],
                                          const typename F::Col (&cc)[W], const typename F::Row& rc, float dg,
                                          float lf, int dr, int w, const KParams& kp) {
    if constexpr (F::kX2) {
        F::template strip<W, WIN>(v, cy, wr, cc, rc, dg, lf, kp);
        return;
    }
    const float fdr = (float)dr;
    float carry_prev = 0.f;
    if constexpr (F::kCarry) carry_prev = F::carry_first(rc, cc[0]);
#pragma unroll
    for (int u = 0; u < W; ++u) {
        const float top = v[u];
        float nv;
        if constexpr (F::kCarry) {
            const float cin = carry_prev;
            carry_prev = cy[u];
            nv = F::cell_c(dg, top, lf, rc, cc[u], wr[u], cin, cy[u]);
        } else if constexpr (F::kWeights) {
            nv = F::cell_w(dg, top, lf, rc, cc[u], wr[u]);
        } else {
            nv = F::cell(dg, top, lf, rc, cc[u], dr - u, __fsub_rn(fdr, (float)u), kp);
        }
        if (WIN) nv = __fadd_rn(nv, wr[u]);   // 0 inside the window, +inf outside (see shift_weights)
        dg = top;
        v[u] = nv;
        lf = nv;
    }
}

// Per-cell diagonal factors of a strip for the next row: wr[u] <- wr[u-1],
// wr[0] <- the factor of i - j = row - c0.  They are WDTW's weights, TWE's
// penalties, or for the windowed distances the window itself: 0 for
// |i - j| <= w and +inf outside, added to each cell (a float add instead of a
// per-cell integer test; x + 0 = x exactly, x + inf = inf).  For TWE, fd
// holds row - 1 - c0 as a float (an exact integer) and steps by one per row,
// so the penalty of the new cell needs no integer conversion.
template <class F, int W, bool WIN>
__device__ __forceinline__ void shift_weights(float (&wr)[W], const float* wt, const KParams& kp, int row, int c0,
                                              float& fd, int w) {
    if constexpr (F::kWeights || F::kPen || WIN) {
#pragma unroll
        for (int u = W - 1; u > 0; --u) wr[u] = wr[u - 1];
        if constexpr (F::kWeights) {
            wr[0] = __ldg(wt + 2 * abs(row - c0));
        } else if constexpr (F::kPen) {
            fd = __fadd_rn(fd, 1.f);
            wr[0] = F::pen_f(kp, fd);
        } else {
            wr[0] = abs(row - c0) <= w ? 0.f : EAP_FINF;
        }
    }
}
// Factors before a strip's first row r0: those of i - j = r0 - 1 - (c0 + u).
template <class F, int W, bool WIN>
__device__ __forceinline__ void init_weights(float (&wr)[W], const float* wt, const KParams& kp, int r0, int c0,
                                             float& fd, int w) {
    fd = (float)(r0 - 1 - c0);
#pragma unroll
    for (int u = 0; u < W; ++u) {
        if constexpr (F::kWeights) wr[u] = __ldg(wt + 2 * abs(r0 - 1 - c0 - u));
        else if constexpr (F::kPen) wr[u] = F::pen(kp, r0 - 1 - c0 - u);
        else if constexpr (WIN) wr[u] = abs(r0 - 1 - c0 - u) <= w ? 0.f : EAP_FINF;
        else wr[u] = 0.f;
    }
}

// Modes of the pair DP: Base (Alg. 3, every cell), EAPruned (Alg. 5) and
// EABase (Alg. 4: every cell until a cut of the lattice exceeds the cut-off).
constexpr int kPmBase = 0, kPmPruned = 1, kPmEA = 2;

// Returns D(A,B) if it is <= in.cut (EAPruned) or always (Base); EABase
// returns D or +inf, +inf only when D > in.cut.
// bnd: this warp's shared-memory column of La+1 floats.  cells: per-lane
// running count of evaluated cells.
template <class F, int W, int PM, bool WIN>
__device__ float warp_pair(const PairIn& in, float* __restrict__ bnd, const KParams& kp,
                           unsigned long long& cells, bool& abandoned) {
    constexpr bool PRUNE = PM == kPmPruned;
    constexpr bool EA = PM == kPmEA;
    const int lane = threadIdx.x & 31;
    const int La = in.La, Lb = in.Lb, w = in.w;
    constexpr int P = 32 * W;
    const int npan = (Lb + P - 1) / P;
    float cut = PRUNE ? in.cut : EAP_FINF;     // pruning threshold (EAPruned)
    float eacut = EA ? in.cut : EAP_FINF;      // abandoning threshold (EABase)
    abandoned = false;
    // EABase: last row of the boundary column this panel reads whose value is <= eacut.
    int ea_bl = 0;

    // Left boundary of panel 0 is the vertical border M(r, 0): rows [blo, bhi]
    // of bnd hold readable values, everything else is +inf.
    int blo = 1, bhi = 0;
    if (F::kBorders) {
        const int vmax = min(La, w + 1);
        int live = 0;
        for (int r0 = 1; r0 <= vmax; r0 += 32) {
            const int r = r0 + lane;
            const float x = r <= vmax ? __ldg(in.bA + r - 1) : EAP_FINF;
            if (r <= vmax) bnd[r] = x;
            live += __popc(__ballot_sync(EAP_FULL, r <= vmax && x <= cut));
            if (EA) ea_bl += __popc(__ballot_sync(EAP_FULL, r <= vmax && x <= eacut));
        }
        if (live > 0) { blo = 1; bhi = live; }   // the border is monotone: live rows are a prefix
    }
    __syncwarp();

    for (int p = 0; p < npan; ++p) {
        const int cf = p * P + 1;
        const int cl = min(cf + P - 1, Lb);
        const bool last = (p == npan - 1);
        if ((PRUNE || EA) && in.cut_src) {
            // One lane reads the shared best-so-far and broadcasts it, so the
            // whole warp takes the same pruning decisions.
            unsigned long long cv = 0;
            if (lane == 0) cv = *(volatile const unsigned long long*)in.cut_src;
            cv = __shfl_sync(EAP_FULL, cv, 0);
            const float c2 = __uint_as_float((unsigned)(cv >> 32));
            if (PRUNE) cut = fminf(cut, c2);
            else eacut = fminf(eacut, c2);
        }
        // EABase: a top-border cell right of this panel at or below the
        // cut-off (ERP; the border increases, so the first one decides).
        const bool ea_top_beyond = EA && !last && hborder<F>(in, cl + 1) <= eacut;
        // Rows of this panel that can hold a live cell start at row 1 if the
        // top border left of / inside it is live, else at the first live row
        // of the left boundary (pruning from the left).
        const bool top_live = hborder<F>(in, cf - 1) <= cut;
        if (!top_live && blo > bhi) { abandoned = true; return EAP_FINF; }
        int r0 = top_live ? 1 : blo;
        int r1 = La;
        if (WIN) { r0 = max(r0, cf - w); r1 = min(La, cl + w); }
        if (r0 > r1) {
            if (last) return EAP_FINF;
            blo = 1; bhi = 0;
            ea_bl = 0;
            continue;
        }

        // Lane 0 reads the boundary column unconditionally: rows of this panel
        // outside the live range [blo, bhi] are set to +inf first.
        for (int r = r0 + lane; r <= r1; r += 32)
            if (r < blo || r > bhi) bnd[r] = EAP_FINF;
        __syncwarp();

        const int c0 = cf + lane * W;   // first column of this lane's strip
        typename F::Col cc[W];
        float v[W];
#pragma unroll
        for (int u = 0; u < W; ++u) {
            const int c = c0 + u;
            // Columns past Lb get a huge value: their cells stay far above any
            // finite cut-off and never feed a real cell (they lie to the right).
            const float t = c <= Lb ? __ldg(in.B + c - 1) : kPadValue;
            const float tprev = c == 1 ? 0.f : (c - 1 <= Lb ? __ldg(in.B + c - 2) : kPadValue);
            cc[u] = F::col(t, tprev, kp);
            v[u] = (r0 == 1) ? hborder<F>(in, c <= Lb ? c : Lb + 1) : EAP_FINF;
        }
        float wr[W];   // diagonal factors of the strip's cells for the current row (WDTW, TWE)
        float fd;      // row - 1 - c0 as a float (TWE)
        init_weights<F, W, WIN>(wr, in.wt, kp, r0, c0, fd, w);
        float cy[W];   // carried per-cell values of the previous row (TWE)
        {
            const float s_before = r0 >= 2 ? __ldg(in.A + r0 - 2) : 0.f;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                if constexpr (F::kCarry) cy[u] = F::carry_init(s_before, cc[u]);
                else cy[u] = 0.f;
            }
        }
        float dg;
        if (r0 == 1) dg = hborder<F>(in, c0 - 1 <= Lb ? c0 - 1 : Lb + 1);
        else dg = (lane == 0) ? bnd[r0 - 1] : EAP_FINF;
        const bool lane_out = c0 > Lb;             // strip entirely past the last column
        const int nvalid = max(0, min(W, Lb - c0 + 1));
        const bool st31 = !last && lane == 31;     // this lane hands its last column to the next panel
        // Row constants: computed from s_i, s_{i-1} per step, or (F::kPacked)
        // loaded precomputed, one step ahead.
        float sp = 0.f, s_next = 0.f;
        float4 pk_next = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (F::kPacked) {
            pk_next = __ldg(in.rp + r0 - 1);
        } else {
            sp = r0 >= 2 ? __ldg(in.A + r0 - 2) : 0.f;
            s_next = __ldg(in.A + r0 - 1);
        }
        const int nsteps = r1 - r0 + 32;
        bool ea_handed = false;   // EABase: lane 31 handed a value <= eacut to the next panel

        // One step of the skewed wavefront; ACTIVE_CHECK for the ramps, where
        // some lanes have not started or have finished.
        auto step = [&](int t, auto active_check) {
            const int row = r0 + t - lane;
            constexpr bool kCheck = decltype(active_check)::value;
            const bool act = kCheck ? (row >= r0 && row <= r1) : true;
            const float bv = act ? bnd[row] : EAP_FINF;
            float x = __shfl_up_sync(EAP_FULL, v[W - 1], 1);
            if (lane == 0) x = bv;
            if (act) {
                typename F::Row rc;
                if constexpr (F::kPacked) {
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
                if (st31) {
                    bnd[row] = v[W - 1];
                    if (EA) ea_handed = ea_handed || v[W - 1] <= eacut;
                }
            }
        };
        // Dead-frontier vote: every cell a later row of this panel could
        // depend on (each lane's current strip and left input, and lane 0's
        // future boundary rows) is above the cut-off.
        auto frontier_dead = [&](int t) -> bool {
            const int row = r0 + t - lane;
            bool dead = true;
            if (row <= r1 && !lane_out) {
                float m = dg;
#pragma unroll
                for (int u = 0; u < W; ++u) m = fminf(m, v[u]);
                dead = m > cut;
                if (lane == 0 && row < bhi) dead = false;
            }
            return __all_sync(EAP_FULL, dead);
        };
        // EABase: every cell of the current cut of the lattice exceeds the
        // cut-off.  The cut is the staircase of each lane's newest strip
        // values and left input (a lane that has finished the panel keeps
        // its last row, which holds M(L_A, L_B) once the pair is done), the
        // boundary rows lane 0 has not consumed, the rows already handed to
        // the next panel and the top border right of the panel; every
        // alignment path crosses it, so D > cut-off.
        auto ea_dead = [&](int t) -> bool {
            const int row = r0 + t - lane;
            bool dead = !ea_top_beyond && !ea_handed;
            if (dead && !lane_out) {
                float m = dg;
#pragma unroll
                for (int u = 0; u < W; ++u) m = fminf(m, v[u]);
                dead = m > eacut;
            }
            if (lane == 0 && row < ea_bl) dead = false;
            return __all_sync(EAP_FULL, dead);
        };
        int done = nsteps;   // steps executed
        int t = 0;
        bool stop = false;
        const int ramp_end = min(31, nsteps);
        bool ea_ab = false;
        for (; t < ramp_end; ++t) {
            step(t, BoolC<true>{});
            if (PRUNE && (t & 3) == 3 && frontier_dead(t)) { done = t + 1; stop = true; break; }
            if (EA && (t & 3) == 3 && ea_dead(t)) { done = t + 1; stop = ea_ab = true; break; }
        }
        const int steady_end = r1 - r0 + 1;   // steps [31, steady_end) have every lane active
        if (!stop) {
            // Unrolled so that the strip's registers rotate back to their
            // starting assignment at the back-edge (one new value per cell
            // per step: W + 1 steps close the cycle); W = 16 unrolls 4 steps
            // to keep the code and the register count in check.
            constexpr int U = kSteadyUnroll > 0 ? kSteadyUnroll : (W <= 8 ? W + 1 : 4);
            for (; t + U <= steady_end; t += U) {
#pragma unroll
                for (int k = 0; k < U; ++k) step(t + k, BoolC<false>{});
                if (PRUNE && frontier_dead(t + U - 1)) { done = t + U; stop = true; break; }
                if (EA && ea_dead(t + U - 1)) { done = t + U; stop = ea_ab = true; break; }
            }
        }
        if (!stop) {
            for (; t < nsteps; ++t) {
                step(t, BoolC<true>{});
                if (PRUNE && (t & 3) == 3 && frontier_dead(t)) { done = t + 1; break; }
                if (EA && (t & 3) == 3 && ea_dead(t)) { done = t + 1; ea_ab = true; break; }
            }
        }
        t = done;
        // Rows this lane evaluated in the panel.
        {
            const int lastrow = min(r1, r0 + t - 1 - lane);
            if (lastrow >= r0) cells += (unsigned long long)(lastrow - r0 + 1) * (unsigned)nvalid;
        }
        __syncwarp();
        if (EA && ea_ab) { abandoned = true; return EAP_FINF; }
        if (last) {
            const int off = Lb - cf;         // offset of column Lb inside the panel
            const int lr = off / W, ur = off % W;
            float res = EAP_FINF;
#pragma unroll
            for (int u = 0; u < W; ++u) if (u == ur) res = v[u];
            res = __shfl_sync(EAP_FULL, res, lr);
            const int lastrow = min(r1, r0 + t - 1 - lr);
            if (lastrow != La) res = EAP_FINF;
            if (PRUNE && !(res <= cut)) res = EAP_FINF;
            if (res == EAP_FINF) abandoned = true;
            return res;
        }
        // Live rows of the column handed to the next panel.
        const int wlast = min(r1, r0 + t - 1 - 31);
        int lo = 0x7fffffff, hi = -1, ea_hi = 0;
        for (int r = r0 + lane; r <= wlast; r += 32) {
            const float b = bnd[r];
            if (b <= cut) { lo = min(lo, r); hi = max(hi, r); }
            if (EA && b <= eacut) ea_hi = max(ea_hi, r);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(EAP_FULL, lo, o));
            hi = max(hi, __shfl_xor_sync(EAP_FULL, hi, o));
            if (EA) ea_hi = max(ea_hi, __shfl_xor_sync(EAP_FULL, ea_hi, o));
        }
        if (hi < 0) { blo = 1; bhi = 0; } else { blo = lo; bhi = hi; }
        if (EA) {
            // The whole handed column (and the top border beyond it) above the cut-off.
            if (ea_hi == 0 && !ea_top_beyond) { abandoned = true; return EAP_FINF; }
            ea_bl = ea_hi;
        }
        __syncwarp();
    }
    return EAP_FINF;   // not reached: the last panel returns
}

// ---------------------------------------------------------------------------
// Diagonal-path upper bound (Section 4 intro: any warping path's cost bounds
// D from above).  The path is (1,1)..(m,m), m = min(La,Lb), then straight
// along the longer axis.  It is evaluated with the same functor as the DP,
// with the off-path dependencies at +inf, so the DP's value is <= this bound
// exactly (min and float addition are monotone).
// ---------------------------------------------------------------------------
// The same path cost with the column series read from `Bs` (any address space,
// used by the tiled bound kernel with the candidates staged in shared memory).
template <class F>
__device__ float diag_path_cost_b(const PairIn& in, const float* Bs, const KParams& kp) {
    const int La = in.La, Lb = in.Lb;
    const int m = min(La, Lb);
    if (in.w < abs(La - Lb)) return EAP_FINF;
    float acc = 0.f;
    float sp = 0.f, tp = 0.f;
    for (int k = 1; k <= m; ++k) {
        const float s = __ldg(in.A + k - 1), t = Bs[k - 1];
        const typename F::Row rc = F::row_diag(s, sp, kp, in.wt);
        const typename F::Col c = F::col_diag(t, tp, kp);
        acc = F::cell(acc, EAP_FINF, EAP_FINF, rc, c, 0, 0.f, kp);
        sp = s; tp = t;
    }
    if (La > Lb) {
        const typename F::Col c = F::col(Bs[Lb - 1], Lb >= 2 ? Bs[Lb - 2] : 0.f, kp);
        for (int i = m + 1; i <= La; ++i) {
            const float s = __ldg(in.A + i - 1);
            const typename F::Row rc = F::row(s, sp, kp, in.wt);
            acc = F::cell(EAP_FINF, acc, EAP_FINF, rc, c, i - Lb, (float)(i - Lb), kp);
            sp = s;
        }
    } else if (Lb > La) {
        const typename F::Row rc = F::row(__ldg(in.A + La - 1), La >= 2 ? __ldg(in.A + La - 2) : 0.f, kp, in.wt);
        for (int j = m + 1; j <= Lb; ++j) {
            const float t = Bs[j - 1];
            const typename F::Col c = F::col(t, tp, kp);
            acc = F::cell(EAP_FINF, EAP_FINF, acc, rc, c, La - j, (float)(La - j), kp);
            tp = t;
        }
    }
    return acc;
}

template <class F>
__device__ float diag_path_cost(const PairIn& in, const KParams& kp) {
    const int La = in.La, Lb = in.Lb;
    const int m = min(La, Lb);
    if (in.w < abs(La - Lb)) return EAP_FINF;
    float acc = 0.f;   // M(0,0)
    float sp = 0.f, tp = 0.f;
    for (int k = 1; k <= m; ++k) {
        const float s = __ldg(in.A + k - 1), t = __ldg(in.B + k - 1);
        const typename F::Row rc = F::row_diag(s, sp, kp, in.wt);
        const typename F::Col c = F::col_diag(t, tp, kp);
        acc = F::cell(acc, EAP_FINF, EAP_FINF, rc, c, 0, 0.f, kp);
        sp = s; tp = t;
    }
    if (La > Lb) {   // down steps along column Lb (AlternateRow)
        const typename F::Col c = F::col(__ldg(in.B + Lb - 1), Lb >= 2 ? __ldg(in.B + Lb - 2) : 0.f, kp);
        for (int i = m + 1; i <= La; ++i) {
            const float s = __ldg(in.A + i - 1);
            const typename F::Row rc = F::row(s, sp, kp, in.wt);
            acc = F::cell(EAP_FINF, acc, EAP_FINF, rc, c, i - Lb, (float)(i - Lb), kp);
            sp = s;
        }
    } else if (Lb > La) {   // right steps along row La (AlternateColumn)
        const typename F::Row rc = F::row(__ldg(in.A + La - 1), La >= 2 ? __ldg(in.A + La - 2) : 0.f, kp, in.wt);
        for (int j = m + 1; j <= Lb; ++j) {
            const float t = __ldg(in.B + j - 1);
            const typename F::Col c = F::col(t, tp, kp);
            acc = F::cell(EAP_FINF, EAP_FINF, acc, rc, c, La - j, (float)(La - j), kp);
            tp = t;
        }
    }
    return acc;
}

}  // namespace eapd
