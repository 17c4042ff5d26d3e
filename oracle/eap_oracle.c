/*
 * oracle/eap_oracle.c -- plain, slow, FP64 CPU oracle for the elastic distances
 * of Herrmann & Webb, "Early Abandoning and Pruning for Elastic Distances
 * including Dynamic Time Warping" (arXiv 2102.05221).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (all in double precision, inputs widened exactly from
 * float32):
 *   orc_distance   the cost matrix of Eq. (Common) filled row by row from its
 *                  definition, with each distance's own borders and step costs
 *                  (Eq. DTW, Section 2.3.2 for the window, Eq. WDTW, Eq. ERP,
 *                  Eq. MSMCost + Eq. MSM, Eq. TWECost + Eq. TWE).  No pruning,
 *                  no early abandoning.  Two rolling rows hold the matrix; the
 *                  arithmetic and its order are the definition's.
 *   orc_eapruned   Algorithm 5 (generic EAPruned) step by step in the paper's
 *                  stages, with a counter of computed cells (used to pin the
 *                  paper's worked-example counts, Section 4.2).
 *   orc_eabase     Algorithm 4 (Base with a window and the usual early
 *                  abandoning on the row minimum), with a cell counter.
 *   orc_nn1        Algorithm 1 (NN search) over candidates in index order with
 *                  the strict "<" update; threads split the queries.
 *   orc_nn1_eapruned  Algorithm 1 with Algorithm 5 as the distance and the
 *                  best-so-far as its cut-off, single-threaded: the paper's
 *                  own search (the like-for-like CPU baseline).
 *   orc_pairwise   the full distance matrix (the exact values that prune-only
 *                  mode must reproduce, Section 4 intro).
 *   orc_subseq     sub-sequence search (Section 5.3): every z-normalised
 *                  window of a long series against a z-normalised query.
 *   orc_envelope / orc_lb_keogh   the textbook LB_Keogh (Section 2.1, Section
 *                  4.2): windowed min/max envelope, then the sum of the costs
 *                  to the envelope outside it.
 *
 * Readings of the paper taken here:
 *   - cost(a,b) is squared for DTW/CDTW/WDTW (pinned by DTW(S,T)=9 in the
 *     Fig. DTW caption), absolute for ERP and TWE (their metric forms); MSM
 *     uses |.| as printed.  Either cost can be chosen explicitly.
 *   - Eq. ERP's "cost(t_i, g)" in the AlternateColumn case is read as
 *     cost(t_j, g).
 *   - Window (Sections 2.3.2, Alg. 4/5): interior cells with |i-j| > w are
 *     +inf; computed borders (ERP) are initialised for indices 1..w+1 exactly
 *     as Alg. 4 and Alg. 5 do, and are +inf beyond.  w < |L_S - L_T| gives +inf.
 *   - WDTW: M(i,j) = w(|i-j|) * cost(s_i,t_j) + min(three deps) with
 *     w(d) = wmax / (1 + exp(-g (d - L/2))), L = max(L_S, L_T).
 *   - TWE: tau_i = i; s_0 = t_0 = 0 (only reached at (1,1) where it adds
 *     cost(0,0) = 0).
 *   - A window ratio r gives w = floor(r * max(L_S, L_T)).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_DTW = 0, O_CDTW = 1, O_WDTW = 2, O_ERP = 3, O_MSM = 4, O_TWE = 5 };
enum { O_COST_SQ = 0, O_COST_ABS = 1 };

/* Parameters as the oracle sees them.  Laid out independently of the CUDA
 * library's own parameter struct (the Python wrapper fills this one). */
typedef struct {
    int32_t kind;
    int32_t cost;          /* O_COST_SQ / O_COST_ABS */
    int32_t window;        /* >= 0: absolute window; < 0: use window_ratio */
    int32_t derivative;    /* 1: the distance of the first-derivative series (DDTW, DCDTW, ...) */
    double window_ratio;   /* < 0 with window < 0: unconstrained */
    double wdtw_g, wdtw_wmax;
    double erp_gap;
    double msm_c;
    double twe_nu, twe_lambda;
} orc_params;

static const double OINF = INFINITY;

static double o_cost(int cost, double a, double b) {
    double d = a - b;
    return cost == O_COST_SQ ? d * d : fabs(d);
}

static double o_min2(double a, double b) { return a < b ? a : b; }
static double o_min3(double a, double b, double c) { return o_min2(o_min2(a, b), c); }

/* Effective window for a pair: a huge value means "no constraint". */
static long o_window(const orc_params* p, int ls, int lt) {
    if (p->kind != O_CDTW && p->kind != O_ERP) return 1L << 40;
    if (p->window >= 0) return p->window;
    if (p->window_ratio >= 0) {
        int L = ls > lt ? ls : lt;
        return (long)floor(p->window_ratio * (double)L);
    }
    return 1L << 40;
}

/* Eq. MSMCost: C_c(np, x, y). */
static double o_msm_c(double c, double np, double x, double y) {
    if ((x <= np && np <= y) || (x >= np && np >= y)) return c;
    return c + o_min2(fabs(np - x), fabs(np - y));
}

/* Eq. WDTW, weight of a cell at distance d from the diagonal. */
static double o_wdtw_weight(double wmax, double g, long d, int L) {
    return wmax / (1.0 + exp(-g * ((double)d - (double)L / 2.0)));
}

/* First-derivative estimate of a series (the derivative distances of Section
 * 2.3: "taking the first derivative of the series", after Keogh & Pazzani):
 * d_i = ((x_i - x_{i-1}) + (x_{i+1} - x_{i-1}) / 2) / 2 for interior points;
 * the first and last points take the estimate of their neighbour; series of
 * length 1 or 2 have no interior point and give zeros. */
static void o_derivative(const double* x, int n, double* d) {
    for (int i = 1; i + 1 < n; i++) d[i] = ((x[i] - x[i - 1]) + (x[i + 1] - x[i - 1]) / 2.0) / 2.0;
    if (n <= 2) { for (int i = 0; i < n; i++) d[i] = 0.0; return; }
    d[0] = d[1];
    d[n - 1] = d[n - 2];
}

static double orc_distance_d(const orc_params* p, const double* s0, int ls, const double* t0, int lt);

/* Full cost matrix of Eq. (Common) for D(S,T): S on the rows (index i),
 * T on the columns (index j).  Returns M(L_S, L_T). */
double orc_distance(const orc_params* p, const float* sf, int ls, const float* tf, int lt) {
    if (ls <= 0 || lt <= 0) return NAN;
    double* a = (double*)malloc(sizeof(double) * (size_t)ls);
    double* b = (double*)malloc(sizeof(double) * (size_t)lt);
    for (int i = 0; i < ls; i++) a[i] = (double)sf[i];
    for (int j = 0; j < lt; j++) b[j] = (double)tf[j];
    if (p->derivative) {
        double* da = (double*)malloc(sizeof(double) * (size_t)ls);
        double* db = (double*)malloc(sizeof(double) * (size_t)lt);
        o_derivative(a, ls, da);
        o_derivative(b, lt, db);
        free(a); free(b);
        a = da; b = db;
    }
    const double r = orc_distance_d(p, a, ls, b, lt);
    free(a); free(b);
    return r;
}

/* The definition itself, on series already in double. */
static double orc_distance_d(const orc_params* p, const double* s0, int ls, const double* t0, int lt) {
    const long w = o_window(p, ls, lt);
    const int L = ls > lt ? ls : lt;
    const int k = p->kind;
    const int cost = p->cost;
    /* 1-indexed copies with s[0] = t[0] = 0 (TWE's s_0, t_0). */
    double* s = (double*)calloc((size_t)ls + 1, sizeof(double));
    double* t = (double*)calloc((size_t)lt + 1, sizeof(double));
    double* prev = (double*)malloc(((size_t)lt + 1) * sizeof(double));
    double* curr = (double*)malloc(((size_t)lt + 1) * sizeof(double));
    for (int i = 1; i <= ls; i++) s[i] = s0[i - 1];
    for (int j = 1; j <= lt; j++) t[j] = t0[j - 1];

    /* Row 0: M(0,0) = 0 and the horizontal border (InitHBorder). */
    curr[0] = 0.0;
    for (int j = 1; j <= lt; j++) {
        if (k == O_ERP && (long)j <= w + 1)
            curr[j] = curr[j - 1] + o_cost(cost, p->erp_gap, t[j]);    /* Eq. ERP hborder */
        else
            curr[j] = OINF;                                            /* +inf border */
    }
    for (int i = 1; i <= ls; i++) {
        double* tmp = prev; prev = curr; curr = tmp;
        /* Column 0: the vertical border (InitVBorder). */
        if (k == O_ERP && (long)i <= w + 1)
            curr[0] = prev[0] + o_cost(cost, s[i], p->erp_gap);            /* Eq. ERP vborder */
        else
            curr[0] = OINF;
        for (int j = 1; j <= lt; j++) {
            long dij = (long)i - (long)j;
            if (dij < 0) dij = -dij;
            if (dij > w) { curr[j] = OINF; continue; }   /* outside the window */
            const double diag = prev[j - 1], top = prev[j], left = curr[j - 1];
            double v;
            switch (k) {
            case O_DTW:
            case O_CDTW:   /* Eq. DTW */
                v = o_cost(cost, s[i], t[j]) + o_min3(diag, top, left);
                break;
            case O_WDTW:   /* Eq. WDTW: weighted cell cost */
                v = o_wdtw_weight(p->wdtw_wmax, p->wdtw_g, dij, L) * o_cost(cost, s[i], t[j])
                    + o_min3(diag, top, left);
                break;
            case O_ERP:    /* Eq. ERP */
                v = o_min3(diag + o_cost(cost, s[i], t[j]),
                           top + o_cost(cost, s[i], p->erp_gap),
                           left + o_cost(cost, t[j], p->erp_gap));
                break;
            case O_MSM:    /* Eq. MSM with Eq. MSMCost; s_0 only meets top = +inf */
                v = o_min3(diag + fabs(s[i] - t[j]),
                           top + o_msm_c(p->msm_c, s[i], s[i - 1], t[j]),
                           left + o_msm_c(p->msm_c, t[j], s[i], t[j - 1]));
                break;
            case O_TWE: {  /* Eq. TWECost + Eq. TWE with tau_i = i */
                const double nu = p->twe_nu, lam = p->twe_lambda;
                const double gm = o_cost(cost, s[i], t[j]) + o_cost(cost, s[i - 1], t[j - 1])
                                  + nu * ((double)labs((long)i - (long)j)
                                          + (double)labs((long)(i - 1) - (long)(j - 1)));
                const double ga = o_cost(cost, s[i], s[i - 1]) + nu * 1.0 + lam;
                const double gb = o_cost(cost, t[j], t[j - 1]) + nu * 1.0 + lam;
                v = o_min3(diag + gm, top + ga, left + gb);
                break;
            }
            default:
                v = NAN;
            }
            curr[j] = v;
        }
    }
    const double res = curr[lt];
    free(s); free(t); free(prev); free(curr);
    return res;
}

/* ------------------------------------------------------------------------
 * Algorithm 5 (generic EAPruned), taken stage by stage.  co = the shorter
 * series (columns), li = the longer (rows); the six distances are symmetric
 * so D(S,T) = D(T,S).  Counts every computed cell of the main matrix in
 * *cells (borders excluded, as in the paper's cell counts).
 *
 * The initial pruning point is the first index of the top border whose
 * value exceeds the cut-off (the top border is monotone, Eq. Common).  For
 * +inf borders this is 1, as printed; for ERP's computed border it is the
 * first dead border index (the paper defines pruning points as the start of
 * a dead block reaching the end of the row, Section 4.2).
 * ------------------------------------------------------------------------ */
typedef struct {
    const orc_params* p;
    const double* r;   /* rows (li), 1-indexed, r[0] = 0 */
    const double* c;   /* columns (co), 1-indexed, c[0] = 0 */
    int L;             /* max length for WDTW */
} o_ctx;

/* Canonical (diag), AlternateRow (top), AlternateColumn (left) step costs
 * for cell (i,j) with rows r and columns c. */
static double o_canon(const o_ctx* x, int i, int j) {
    const orc_params* p = x->p;
    switch (p->kind) {
    case O_DTW: case O_CDTW: return o_cost(p->cost, x->r[i], x->c[j]);
    case O_WDTW: return o_wdtw_weight(p->wdtw_wmax, p->wdtw_g, labs((long)i - j), x->L)
                        * o_cost(p->cost, x->r[i], x->c[j]);
    case O_ERP: return o_cost(p->cost, x->r[i], x->c[j]);
    case O_MSM: return fabs(x->r[i] - x->c[j]);
    case O_TWE: return o_cost(p->cost, x->r[i], x->c[j]) + o_cost(p->cost, x->r[i - 1], x->c[j - 1])
                       + p->twe_nu * 2.0 * (double)labs((long)i - j);
    }
    return NAN;
}
static double o_altrow(const o_ctx* x, int i, int j) {
    const orc_params* p = x->p;
    switch (p->kind) {
    case O_DTW: case O_CDTW: case O_WDTW: return o_canon(x, i, j);
    case O_ERP: return o_cost(p->cost, x->r[i], p->erp_gap);
    case O_MSM: return o_msm_c(p->msm_c, x->r[i], x->r[i - 1], x->c[j]);
    case O_TWE: return o_cost(p->cost, x->r[i], x->r[i - 1]) + p->twe_nu + p->twe_lambda;
    }
    return NAN;
}
static double o_altcol(const o_ctx* x, int i, int j) {
    const orc_params* p = x->p;
    switch (p->kind) {
    case O_DTW: case O_CDTW: case O_WDTW: return o_canon(x, i, j);
    case O_ERP: return o_cost(p->cost, x->c[j], p->erp_gap);
    case O_MSM: return o_msm_c(p->msm_c, x->c[j], x->r[i], x->c[j - 1]);
    case O_TWE: return o_cost(p->cost, x->c[j], x->c[j - 1]) + p->twe_nu + p->twe_lambda;
    }
    return NAN;
}

/* Series of Alg. 4 / Alg. 5 in double, 1-indexed: *r = the longest ("li",
 * rows), *c = the shortest ("co", columns), derivative applied if asked. */
static void o_setup(const orc_params* p, const float* sf, int ls, const float* tf, int lt,
                    double** r_out, double** c_out, int* Lli_out, int* Lco_out) {
    const float* cof = lt <= ls ? tf : sf;
    const float* lif = lt <= ls ? sf : tf;
    const int Lco = lt <= ls ? lt : ls;
    const int Lli = lt <= ls ? ls : lt;
    double* r = (double*)calloc((size_t)Lli + 1, sizeof(double));
    double* c = (double*)calloc((size_t)Lco + 1, sizeof(double));
    for (int i = 1; i <= Lli; i++) r[i] = (double)lif[i - 1];
    for (int j = 1; j <= Lco; j++) c[j] = (double)cof[j - 1];
    if (p->derivative) {
        double* dr = (double*)malloc(sizeof(double) * (size_t)Lli);
        double* dc = (double*)malloc(sizeof(double) * (size_t)Lco);
        o_derivative(r + 1, Lli, dr);
        o_derivative(c + 1, Lco, dc);
        for (int i = 1; i <= Lli; i++) r[i] = dr[i - 1];
        for (int j = 1; j <= Lco; j++) c[j] = dc[j - 1];
        free(dr); free(dc);
    }
    *r_out = r; *c_out = c; *Lli_out = Lli; *Lco_out = Lco;
}

double orc_eapruned(const orc_params* p, const float* sf, int ls, const float* tf, int lt,
                    double cutoff, int64_t* cells) {
    int64_t n = 0;
    if (ls <= 0 || lt <= 0) return NAN;
    const long w = o_window(p, ls, lt);
    if (cells) *cells = 0;
    /* co: shortest series on the columns; li: longest on the rows. */
    const int Lco = lt <= ls ? lt : ls;
    const int Lli = lt <= ls ? ls : lt;
    if (w < (long)(Lli - Lco)) return OINF;
    double *r, *c;
    int Lli_, Lco_;
    o_setup(p, sf, ls, tf, lt, &r, &c, &Lli_, &Lco_);
    o_ctx x = {p, r, c, Lli};
    double* prev = (double*)malloc(((size_t)Lco + 1) * sizeof(double));
    double* curr = (double*)malloc(((size_t)Lco + 1) * sizeof(double));
    for (int j = 0; j <= Lco; j++) prev[j] = curr[j] = OINF;
    curr[0] = 0.0;
    const long hb_end = w + 1 < (long)Lco ? w + 1 : (long)Lco;
    for (long j = 1; j <= hb_end; j++)
        curr[j] = (p->kind == O_ERP) ? curr[j - 1] + o_cost(p->cost, p->erp_gap, c[j]) : OINF;
    long next_start = 1;
    long pruning_point = 1;
    /* Only computed border cells (ERP, indices 1..w+1) can be <= cut-off;
     * +inf border cells are the dead block that starts at (0,1). */
    if (p->kind == O_ERP)
        while (pruning_point <= hb_end && curr[pruning_point] <= cutoff) pruning_point++;
    long next_pruning_point = pruning_point;
    double result = OINF;
    int abandoned = 0;
    for (long i = 1; i <= Lli && !abandoned; i++) {
        double* tmp = prev; prev = curr; curr = tmp;
        const long j_start = (i - w) > next_start ? (i - w) : next_start;
        const long j_stop = (i + w) < (long)Lco ? (i + w) : (long)Lco;
        long j = j_start;
        /* Stage 1: the vertical border (computed, or +inf outside the window). */
        if (j_start == 1)
            curr[0] = (p->kind == O_ERP) ? prev[0] + o_cost(p->cost, r[i], p->erp_gap) : OINF;
        else
            curr[j_start - 1] = OINF;
        /* Stage 2: discard points, up to (excluding) the pruning point. */
        if (curr[j_start - 1] > cutoff) {
            for (; j < pruning_point && j == next_start; j++) {
                curr[j] = o_min2(prev[j - 1] + o_canon(&x, i, j), prev[j] + o_altrow(&x, i, j));
                n++;
                if (curr[j] <= cutoff) next_pruning_point = j + 1; else next_start++;
            }
        }
        /* Stage 3: up to (excluding) the pruning point, all dependencies. */
        for (; j < pruning_point; j++) {
            curr[j] = o_min3(prev[j - 1] + o_canon(&x, i, j), prev[j] + o_altrow(&x, i, j),
                             curr[j - 1] + o_altcol(&x, i, j));
            n++;
            if (curr[j] <= cutoff) next_pruning_point = j + 1;
        }
        /* A computed vertical border cell (ERP, column 0 of this row) that is
         * <= cut-off belongs to the row's live cells: a path can run down the
         * border and enter the interior in a later row. */
        const int border_live = (j_start == 1) && curr[0] <= cutoff;
        /* Stage 4: at the pruning point. */
        if (j <= j_stop) {
            if (j == next_start && !border_live) {
                curr[j] = prev[j - 1] + o_canon(&x, i, j);
                n++;
                if (curr[j] <= cutoff) next_pruning_point = j + 1;
                else { abandoned = 1; break; }
            } else {
                curr[j] = o_min2(prev[j - 1] + o_canon(&x, i, j), curr[j - 1] + o_altcol(&x, i, j));
                n++;
                if (curr[j] <= cutoff) next_pruning_point = j + 1;
            }
            j++;
        } else if (j == next_start && !border_live) {
            abandoned = 1;
            break;
        }
        /* Stage 5: after the pruning point, left dependency only. */
        for (; j <= j_stop && j == next_pruning_point; j++) {
            curr[j] = curr[j - 1] + o_altcol(&x, i, j);
            n++;
            if (curr[j] <= cutoff) next_pruning_point = j + 1;
        }
        pruning_point = next_pruning_point;
    }
    if (!abandoned) {
        /* The last row's pruning point must lie beyond L_co for curr[L_co]
         * to hold a value computed in that row that is <= cutoff. */
        result = (pruning_point > Lco) ? curr[Lco] : OINF;
        if (!(result <= cutoff)) result = OINF;
    }
    if (cells) *cells = n;
    free(r); free(c); free(prev); free(curr);
    return result;
}

/* ------------------------------------------------------------------------
 * Algorithm 4: the Base DP with a window and the usual early abandoning
 * (EABase).  Rows are the longest series, columns the shortest; after each
 * row, the computation is abandoned (+inf) when the smallest value of the
 * row exceeds the cut-off.  Otherwise M(L_li, L_co) is returned, which may
 * itself exceed the cut-off.  The row minimum includes the row's vertical
 * border cell while the window covers column 0 (ERP's computed border): a
 * path can run down that border, so leaving it out could abandon a distance
 * that is below the cut-off.  *cells counts the interior cells computed.
 * ------------------------------------------------------------------------ */
double orc_eabase(const orc_params* p, const float* sf, int ls, const float* tf, int lt,
                  double cutoff, int64_t* cells) {
    int64_t n = 0;
    if (ls <= 0 || lt <= 0) return NAN;
    const long w = o_window(p, ls, lt);
    if (cells) *cells = 0;
    const int Lco = lt <= ls ? lt : ls;
    const int Lli = lt <= ls ? ls : lt;
    if (w < (long)(Lli - Lco)) return OINF;
    double *r, *c;
    int Lli_, Lco_;
    o_setup(p, sf, ls, tf, lt, &r, &c, &Lli_, &Lco_);
    o_ctx x = {p, r, c, Lli};
    double* prev = (double*)malloc(((size_t)Lco + 1) * sizeof(double));
    double* curr = (double*)malloc(((size_t)Lco + 1) * sizeof(double));
    for (int j = 0; j <= Lco; j++) prev[j] = curr[j] = OINF;
    curr[0] = 0.0;
    const long hb_end = w + 1 < (long)Lco ? w + 1 : (long)Lco;
    for (long j = 1; j <= hb_end; j++)
        curr[j] = (p->kind == O_ERP) ? curr[j - 1] + o_cost(p->cost, p->erp_gap, c[j]) : OINF;
    double result = OINF;
    int abandoned = 0;
    for (long i = 1; i <= Lli; i++) {
        double* tmp = prev; prev = curr; curr = tmp;
        const long j_start = (i - w) > 1 ? (i - w) : 1;
        const long j_stop = (i + w) < (long)Lco ? (i + w) : (long)Lco;
        if (j_start == 1)
            curr[0] = (p->kind == O_ERP) ? prev[0] + o_cost(p->cost, r[i], p->erp_gap) : OINF;
        else
            curr[j_start - 1] = OINF;
        double minv = (j_start == 1) ? curr[0] : OINF;
        for (long j = j_start; j <= j_stop; j++) {
            curr[j] = o_min3(prev[j - 1] + o_canon(&x, i, j), prev[j] + o_altrow(&x, i, j),
                             curr[j - 1] + o_altcol(&x, i, j));
            n++;
            if (curr[j] < minv) minv = curr[j];
        }
        if (minv > cutoff) { abandoned = 1; break; }
    }
    if (!abandoned) result = curr[Lco];
    if (cells) *cells = n;
    free(r); free(c); free(prev); free(curr);
    return result;
}

/* ------------------------------------------------------------------------
 * Algorithm 1 (NN search), queries split across threads.
 * ------------------------------------------------------------------------ */
typedef struct {
    const orc_params* p;
    const float* qd; const int64_t* qo; const int32_t* ql;
    const float* rd; const int64_t* ro; const int32_t* rl;
    int nr;
    int32_t* out_idx; double* out_dist;
    int q_begin, q_end;
} o_nn_job;

static void* o_nn_worker(void* arg) {
    o_nn_job* jb = (o_nn_job*)arg;
    for (int q = jb->q_begin; q < jb->q_end; q++) {
        double dnn = OINF;
        int32_t cnn = -1;
        for (int c = 0; c < jb->nr; c++) {
            double d = orc_distance(jb->p, jb->qd + jb->qo[q], jb->ql[q], jb->rd + jb->ro[c], jb->rl[c]);
            if (d < dnn) { dnn = d; cnn = c; }
        }
        jb->out_idx[q] = cnn;
        jb->out_dist[q] = dnn;
    }
    return NULL;
}

int orc_nn1(const orc_params* p,
            const float* qd, const int64_t* qo, const int32_t* ql, int nq,
            const float* rd, const int64_t* ro, const int32_t* rl, int nr,
            int32_t* out_idx, double* out_dist, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nq) nthreads = nq > 0 ? nq : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    o_nn_job* jobs = (o_nn_job*)malloc(sizeof(o_nn_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = (o_nn_job){p, qd, qo, ql, rd, ro, rl, nr, out_idx, out_dist,
                             (int)((long)nq * k / nthreads), (int)((long)nq * (k + 1) / nthreads)};
        pthread_create(&th[k], NULL, o_nn_worker, &jobs[k]);
    }
    for (int k = 0; k < nthreads; k++) pthread_join(th[k], NULL);
    free(th); free(jobs);
    return 0;
}

/* ------------------------------------------------------------------------
 * Algorithm 1 with Algorithm 5 as the distance, on one thread: the paper's
 * own NN search.  Candidates are scanned in index order; each call gets the
 * current d_nn as its cut-off (Section 2.2: the best-so-far is the cut-off)
 * and a candidate replaces the best only when its result is strictly below
 * it.  Returns the total number of computed cells in *cells.  An abandoned
 * call returns +inf, which never wins, so the result is Algorithm 1's.
 * ------------------------------------------------------------------------ */
int orc_nn1_eapruned(const orc_params* p,
                     const float* qd, const int64_t* qo, const int32_t* ql, int nq,
                     const float* rd, const int64_t* ro, const int32_t* rl, int nr,
                     int32_t* out_idx, double* out_dist, int64_t* cells) {
    int64_t total = 0;
    for (int q = 0; q < nq; q++) {
        double dnn = OINF;
        int32_t cnn = -1;
        for (int c = 0; c < nr; c++) {
            int64_t n = 0;
            const double d = orc_eapruned(p, qd + qo[q], ql[q], rd + ro[c], rl[c], dnn, &n);
            total += n;
            if (d < dnn) { dnn = d; cnn = c; }
        }
        out_idx[q] = cnn;
        out_dist[q] = dnn;
    }
    if (cells) *cells = total;
    return 0;
}

/* ------------------------------------------------------------------------
 * Full distance matrix D(set_i, set_j) (rows i, columns j).
 * ------------------------------------------------------------------------ */
typedef struct {
    const orc_params* p;
    const float* d; const int64_t* o; const int32_t* l;
    int n; double* out; int i_begin, i_end;
} o_pw_job;

static void* o_pw_worker(void* arg) {
    o_pw_job* jb = (o_pw_job*)arg;
    for (int i = jb->i_begin; i < jb->i_end; i++)
        for (int j = 0; j < jb->n; j++)
            jb->out[(size_t)i * jb->n + j] =
                orc_distance(jb->p, jb->d + jb->o[i], jb->l[i], jb->d + jb->o[j], jb->l[j]);
    return NULL;
}

int orc_pairwise(const orc_params* p, const float* d, const int64_t* o, const int32_t* l, int n,
                 double* out, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = n > 0 ? n : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    o_pw_job* jobs = (o_pw_job*)malloc(sizeof(o_pw_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = (o_pw_job){p, d, o, l, n, out,
                             (int)((long)n * k / nthreads), (int)((long)n * (k + 1) / nthreads)};
        pthread_create(&th[k], NULL, o_pw_worker, &jobs[k]);
    }
    for (int k = 0; k < nthreads; k++) pthread_join(th[k], NULL);
    free(th); free(jobs);
    return 0;
}

/* ------------------------------------------------------------------------
 * LB_Keogh (textbook form): envelope of Q with window w, then the cost of
 * each point of C that lies outside it to the nearest envelope edge.
 * ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------
 * Sub-sequence search (Section 5.3): the start position i of the window of
 * the long series T that minimises D(znorm(Q), znorm(T[i .. i+m-1])).
 * z-normalisation: subtract the mean, divide by the population standard
 * deviation (two passes, in double); a window whose deviation is at most
 * 1e-8 normalises to zeros.  Every position is evaluated in full with the
 * definition of D (orc_distance on the normalised windows); ties keep the
 * lowest position.  Threads split the positions.
 * ------------------------------------------------------------------------ */
static void o_znorm(const float* x, int m, double* z) {
    double mu = 0.0;
    for (int k = 0; k < m; k++) mu += (double)x[k];
    mu /= (double)m;
    double var = 0.0;
    for (int k = 0; k < m; k++) var += ((double)x[k] - mu) * ((double)x[k] - mu);
    var /= (double)m;
    const double sd = sqrt(var);
    for (int k = 0; k < m; k++) z[k] = sd > 1e-8 ? ((double)x[k] - mu) / sd : 0.0;
}

typedef struct {
    const orc_params* p;
    const float* T; const double* zq;
    int m;
    int64_t begin, end;
    int64_t best_pos; double best;
} o_ss_job;

static void* o_ss_worker(void* arg) {
    o_ss_job* jb = (o_ss_job*)arg;
    double* z = (double*)malloc(sizeof(double) * (size_t)jb->m);
    jb->best = OINF;
    jb->best_pos = -1;
    for (int64_t i = jb->begin; i < jb->end; i++) {
        o_znorm(jb->T + i, jb->m, z);
        const double d = orc_distance_d(jb->p, jb->zq, jb->m, z, jb->m);
        if (d < jb->best) { jb->best = d; jb->best_pos = i; }
    }
    free(z);
    return NULL;
}

int orc_subseq(const orc_params* p, const float* T, int64_t n, const float* q, int m,
               int64_t* out_pos, double* out_dist, int nthreads) {
    *out_pos = -1;
    *out_dist = OINF;
    if (m <= 0) return -1;
    const int64_t npos = n - m + 1;
    if (npos <= 0) return 0;
    double* zq = (double*)malloc(sizeof(double) * (size_t)m);
    o_znorm(q, m, zq);
    if (p->derivative) {
        /* Not defined for sub-sequence search here. */
        free(zq);
        return -1;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > npos) nthreads = (int)npos;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    o_ss_job* jobs = (o_ss_job*)malloc(sizeof(o_ss_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = (o_ss_job){p, T, zq, m, npos * k / nthreads, npos * (k + 1) / nthreads, -1, OINF};
        pthread_create(&th[k], NULL, o_ss_worker, &jobs[k]);
    }
    for (int k = 0; k < nthreads; k++) {
        pthread_join(th[k], NULL);
        /* Threads cover increasing positions: strict < keeps the lowest on ties. */
        if (jobs[k].best < *out_dist) { *out_dist = jobs[k].best; *out_pos = jobs[k].best_pos; }
    }
    free(th); free(jobs); free(zq);
    return 0;
}

void orc_envelope(const float* q, int L, long w, double* upper, double* lower) {
    for (int i = 0; i < L; i++) {
        double u = -OINF, lo = OINF;
        for (long k = (long)i - w; k <= (long)i + w; k++) {
            if (k < 0 || k >= L) continue;
            if ((double)q[k] > u) u = (double)q[k];
            if ((double)q[k] < lo) lo = (double)q[k];
        }
        upper[i] = u;
        lower[i] = lo;
    }
}

double orc_lb_keogh(const float* q, const float* c, int L, long w, int cost) {
    double* U = (double*)malloc(sizeof(double) * (size_t)L);
    double* Lo = (double*)malloc(sizeof(double) * (size_t)L);
    orc_envelope(q, L, w, U, Lo);
    double lb = 0.0;
    for (int i = 0; i < L; i++) {
        const double ci = (double)c[i];
        if (ci > U[i]) lb += o_cost(cost, ci, U[i]);
        else if (ci < Lo[i]) lb += o_cost(cost, ci, Lo[i]);
    }
    free(U); free(Lo);
    return lb;
}


/* ------------------------------------------------------------------------
 * Cross matrix D(A_a, B_b) for every a, b (rows a), threads split the rows.
 * ------------------------------------------------------------------------ */
typedef struct {
    const orc_params* p;
    const float* ad; const int64_t* ao; const int32_t* al;
    const float* bd; const int64_t* bo; const int32_t* bl;
    int nb; double* out; int a_begin, a_end;
} o_cross_job;

static void* o_cross_worker(void* arg) {
    o_cross_job* jb = (o_cross_job*)arg;
    for (int a = jb->a_begin; a < jb->a_end; a++)
        for (int b = 0; b < jb->nb; b++)
            jb->out[(size_t)a * jb->nb + b] =
                orc_distance(jb->p, jb->ad + jb->ao[a], jb->al[a], jb->bd + jb->bo[b], jb->bl[b]);
    return NULL;
}

int orc_cross(const orc_params* p,
              const float* ad, const int64_t* ao, const int32_t* al, int na,
              const float* bd, const int64_t* bo, const int32_t* bl, int nb,
              double* out, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > na) nthreads = na > 0 ? na : 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    o_cross_job* jobs = (o_cross_job*)malloc(sizeof(o_cross_job) * (size_t)nthreads);
    for (int k = 0; k < nthreads; k++) {
        jobs[k] = (o_cross_job){p, ad, ao, al, bd, bo, bl, nb, out,
                                (int)((long)na * k / nthreads), (int)((long)na * (k + 1) / nthreads)};
        pthread_create(&th[k], NULL, o_cross_worker, &jobs[k]);
    }
    for (int k = 0; k < nthreads; k++) pthread_join(th[k], NULL);
    free(th); free(jobs);
    return 0;
}

int orc_abi_version(void) { return 1; }
