/*
 * eap.h -- C ABI of libeap: batched elastic-distance 1-NN search and distance
 * matrices with EAPruned (pruning + early abandoning) on one GB300 GPU.
 *
 * Method: Herrmann & Webb, "Early Abandoning and Pruning for Elastic
 * Distances including Dynamic Time Warping" (arXiv 2102.05221).
 *
 * Conventions for every entry point
 *   - Return value: EAP_OK (0) or a negative EAP_E* code; eap_strerror()
 *     names it.  No C++ exception ever crosses this boundary.
 *   - Ownership: the caller owns every buffer it passes in and keeps it alive
 *     until the call's work on the stream has finished.  The library owns only
 *     its own scratch (stream-ordered device allocations released on the same
 *     stream) and eap_server objects.
 *   - Memory spaces: pointers documented "device" must be CUDA device (or
 *     managed) memory of the current device; "host" pointers are ordinary host
 *     memory.  eap_nn1_host() is the one entry point that takes host buffers
 *     for everything.
 *   - Asynchrony: device-pointer entry points enqueue work on `cuda_stream`
 *     (a cudaStream_t; NULL = the legacy default stream) and return without
 *     waiting, unless `opt_stats` is non-NULL, in which case they synchronise
 *     the stream to fill it.
 *   - Series sets: a concatenated float32 buffer plus int64 element offsets
 *     and int32 lengths (one per series), given both on the device (read by
 *     the kernels) and on the host (read by the scheduler, never written).
 *   - Numerics: the kernels compute in float32; +inf is the "abandoned / no
 *     alignment" value.  Inputs must be finite.
 */
#ifndef EAP_H
#define EAP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define EAP_OK          0
#define EAP_EINVAL     (-1)  /* invalid argument (null pointer, length <= 0, bad parameter, size mismatch) */
#define EAP_ENOMEM     (-2)  /* device or host allocation failed */
#define EAP_EAGAIN     (-3)  /* serving: not admitted now / result not ready yet */
#define EAP_ETIMEOUT   (-4)  /* a bounded device wait or a serving deadline expired */
#define EAP_EDEVICE    (-5)  /* a CUDA call failed (no device, launch failure, ...) */
#define EAP_EINTERNAL  (-6)  /* an internal consistency check failed */

/* ---- distances (Section 2.3 of the paper) -------------------------------
 * EAP_DTW   Eq. DTW: cost(s_i,t_j) + min of the three dependencies, +inf borders.
 * EAP_CDTW  DTW restricted to the Sakoe-Chiba window |i-j| <= w (Section 2.3.2).
 * EAP_WDTW  Eq. WDTW: cell cost weighted by wmax/(1+exp(-g(|i-j| - L/2))), L = max length.
 * EAP_ERP   Eq. ERP: gap value g, computed borders, window w.
 * EAP_MSM   Eq. MSM with the split/merge cost Eq. MSMCost (penalty c).
 * EAP_TWE   Eq. TWE with Eq. TWECost (stiffness nu, penalty lambda, timestamps tau_i = i). */
typedef enum { EAP_DTW = 0, EAP_CDTW = 1, EAP_WDTW = 2, EAP_ERP = 3, EAP_MSM = 4, EAP_TWE = 5 } eap_kind;

/* Point cost "cost(a,b)" of Section 2.3.  EAP_COST_DEFAULT picks squared
 * for DTW/CDTW/WDTW and absolute for ERP/TWE; MSM always uses |a-b|. */
typedef enum { EAP_COST_DEFAULT = -1, EAP_COST_SQ = 0, EAP_COST_ABS = 1 } eap_cost;

/* Optional lower-bound cascade ahead of the DP (Alg. 2; LB_Keogh of
 * Section 5.2).  Only for DTW/CDTW with equal-length series; ignored otherwise. */
typedef enum { EAP_LB_NONE = 0, EAP_LB_KEOGH = 1, EAP_LB_KEOGH2 = 2 } eap_lb;

typedef struct {
    int32_t kind;          /* eap_kind */
    int32_t cost;          /* eap_cost */
    float   window_ratio;  /* CDTW/ERP: w = floor(ratio * max(L_S, L_T)) when window < 0; < 0 = no window */
    int32_t window;        /* CDTW/ERP: absolute window w >= 0; < 0 = use window_ratio */
    float   wdtw_g;        /* WDTW g >= 0 */
    float   wdtw_wmax;     /* WDTW weight scale wmax > 0 (the paper's form has wmax = 1) */
    float   erp_gap;       /* ERP gap value g (any finite value) */
    float   msm_c;         /* MSM penalty c >= 0 */
    float   twe_nu;        /* TWE stiffness nu >= 0 */
    float   twe_lambda;    /* TWE penalty lambda >= 0 */
    int32_t lb;            /* eap_lb */
    int32_t prune;         /* 1 = EAPruned (Alg. 5 semantics: D if D <= cut-off, else +inf);
                            * 0 = Base (Alg. 3: no pruning, no abandoning);
                            * 2 = EABase (Alg. 4: every cell until the computation is abandoned; returns
                            *     D, or +inf when a cut of the cost matrix -- on the device, the
                            *     wavefront's staircase of newest cells -- lies entirely above the
                            *     cut-off; +inf only if D > cut-off, and a returned D may exceed it).
                            *     Warp mapping only; not accepted by eap_nn1_batch;
                            * 3 = Prune (pruning only: EAPruned with each pair's own diagonal-path cost as
                            *     cut-off, never abandoning; every distance exact).  eap_nn1 family and
                            *     serving only (eap_pairs: EAP_EINVAL; all-pairs: eap_pairwise with
                            *     EAP_PRUNE_ONLY). */
    int32_t derivative;    /* 1 = derivative variant (DDTW, DCDTW, DWDTW, ...; Section 2.3): the distance of
                            * the first-derivative series d_i = ((x_i - x_{i-1}) + (x_{i+1} - x_{i-1})/2)/2
                            * (Keogh & Pazzani's estimate; the end points copy their neighbour, series of
                            * one or two points give zeros), computed on the device in float32 into
                            * stream-ordered scratch of 4 bytes per element of each set; 0 = plain */
} eap_params;

/* Fills *p with the defaults of the distance: window ratio 0.1 for CDTW/ERP,
 * g = 0.05 and wmax = 1 for WDTW, gap 0 for ERP, c = 0.5 for MSM,
 * nu = 0.001 and lambda = 1 for TWE, default cost, no LB, prune = 1,
 * derivative = 0. */
void eap_params_default(eap_params* p, int32_t kind);

typedef struct {
    const float*   data;       /* device: all series back to back (float32) */
    const int64_t* offsets;    /* device: element offset of series k in data */
    const int32_t* lengths;    /* device: length of series k (>= 1) */
    const int64_t* h_offsets;  /* host mirror of offsets */
    const int32_t* h_lengths;  /* host mirror of lengths */
    int64_t        data_len;   /* number of floats in data (bounds check) */
    int32_t        count;      /* number of series (>= 0) */
    int32_t        reserved_;
} eap_series_set;

/* Work counters of one call (filled when a non-NULL pointer is passed). */
typedef struct {
    uint64_t pairs;            /* (query, candidate) or (i, j) pairs given to the DP */
    uint64_t pairs_lb_pruned;  /* pairs skipped because their lower bound exceeded the cut-off */
    uint64_t pairs_abandoned;  /* pairs the DP early-abandoned (returned +inf) */
    uint64_t cells_effective;  /* sum over all pairs of L_S * L_T */
    uint64_t cells_computed;   /* cells the DP kernels evaluated (after pruning) */
    double   dp_ms;            /* device time of the DP kernel launch(es), CUDA events on the call's stream */
    double   lb_ms;            /* device time of the envelope + LB_Keogh launches (eap_nn1 with a lower
                                * bound), CUDA events on the call's stream; 0 otherwise */
} eap_stats;

/* Inputs must be finite.  Validation mode -- the environment variable
 * EAP_CHECK_INPUTS=1 -- makes every entry point scan its input series for
 * NaN / Inf first (after a device-wide synchronisation, so not inside a
 * stream capture) and return EAP_EINVAL if it finds any; otherwise non-finite
 * values are not detected and give unspecified results. */

/* ---- entry points -------------------------------------------------------- */

/* 1-NN search (Alg. 1, each distance evaluation Alg. 5 with the query's
 * current best-so-far as cut-off).  For every query q, finds the candidate c
 * minimising D(Q_q, C_c); ties go to the lowest candidate index; D values
 * that are +inf (infeasible window) never win.
 *   queries, refs : series sets (device + host mirrors).
 *   out_idx       : device int32[queries->count]; -1 when no candidate is finite.
 *   out_dist      : device float[queries->count]; +inf when none.
 * The cut-off starts at the smallest diagonal-path cost of the query over all
 * candidates (a valid upper bound, Section 4 intro), candidates are evaluated
 * nearest-diagonal-cost first, and concurrent candidates of one query share
 * the cut-off through a packed 64-bit atomicMin. */
int eap_nn1(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs,
            int32_t* out_idx, float* out_dist, void* cuda_stream, eap_stats* opt_stats);

/* The same search with every buffer in host memory: copies the sets to the
 * device, runs eap_nn1 on an internal stream, copies the results back and
 * waits.  q_data/r_data: host float32; offsets/lengths: host; out_*: host. */
int eap_nn1_host(const eap_params* p,
                 const float* q_data, const int64_t* q_offsets, const int32_t* q_lengths, int32_t nq,
                 const float* r_data, const int64_t* r_offsets, const int32_t* r_lengths, int32_t nr,
                 int32_t* out_idx, float* out_dist, eap_stats* opt_stats);

/* Which kernel mapping, and which strip width, an eap_nn1 call with these
 * parameters and sizes runs.  The paper has no counterpart (its search runs
 * one pair at a time on one CPU thread); this reports the library's own
 * choice.  Host only: it reads no device memory, launches nothing and works
 * without a GPU.  The choice follows eap_nn1 exactly: distance and mode
 * (p), number of queries, the shortest series of both sets, the longest
 * query and the longest candidate, the EAP_MAP / EAP_W / EAP_G / EAP_BAND*
 * environment overrides and the autotuner's table.
 *   out->mapping        : EAP_PLAN_BAND (band coordinates, windowed CDTW/ERP),
 *                         EAP_PLAN_GROUP (several pairs per warp over column
 *                         panels), EAP_PLAN_WARP (a warp per pair),
 *                         EAP_PLAN_CTA (8 warps per pair, long series).
 *   out->strip_width    : cells a lane computes per row.
 *   out->lanes_per_pair : 4, 8 or 16 (band, groups), 32 (warp), 256 (CTA).
 *   out->band_exact     : 1 when a band launch covers exactly the 2w + 2
 *                         positions of a band row, else 0.
 * Returns EAP_EINVAL for invalid parameters, out == NULL, n_queries < 0,
 * or lengths outside 1..8192 with min_len above either maximum. */
typedef enum { EAP_PLAN_BAND = 1, EAP_PLAN_GROUP = 2, EAP_PLAN_WARP = 3, EAP_PLAN_CTA = 4 } eap_plan_mapping;
typedef struct {
    int32_t mapping;
    int32_t strip_width;
    int32_t lanes_per_pair;
    int32_t band_exact;
} eap_plan;
int eap_nn1_plan(const eap_params* p, int32_t n_queries, int32_t min_len, int32_t max_query_len,
                 int32_t max_ref_len, eap_plan* out);

/* 1-NN against one shard of the candidates, as packed keys for the one
 * exchange step of candidate sharding (Alg. 1 over the union of the shards
 * is the per-query minimum of the shards' keys).  Same search as eap_nn1;
 * instead of (index, distance) it writes, per query,
 *     out_keys[q] = (float bits of D) << 32 | (local index + index_offset)
 * or (+inf bits) << 32 | 0xffffffff when no candidate of the shard is
 * finite.  Distances are >= 0, so the keys order like (distance, global
 * index) both as unsigned and as signed 64-bit integers: an element-wise MIN
 * over the shards (e.g. an all-reduce) keeps the smallest distance and, among
 * equal ones, the lowest global index -- Alg. 1's strict "<" over the
 * candidates in index order.
 *   out_keys      device uint64[queries->count]
 *   index_offset  global index of refs' first series; index_offset >= 0 and
 *                 index_offset + refs->count < 2^32 - 1, else EAP_EINVAL.
 * Asynchronous on the stream like eap_nn1. */
int eap_nn1_keys(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs,
                 int64_t index_offset, uint64_t* out_keys, void* cuda_stream, eap_stats* opt_stats);

/* Keys of eap_nn1_keys (after the min-reduction) to results:
 * out_idx[q] = the key's index, or -1 for "none"; out_dist[q] = D, or +inf.
 * keys, out_idx, out_dist: device arrays of n elements. */
int eap_keys_unpack(const uint64_t* keys, int32_t n, int32_t* out_idx, float* out_dist, void* cuda_stream);

#define EAP_PRUNE_ONLY 0   /* EAPruned with each pair's own diagonal-path cost as cut-off: exact, prunes but never abandons (Section 4 intro) */
#define EAP_BASE       1   /* plain Base DP (Alg. 3) */

/* All-pairs distance matrix of one set: out_matrix is device float
 * [count * count], row-major, symmetric, zero diagonal.  Each unordered pair
 * is computed once (D(set_i, set_j) with i < j, set_i on the rows).  `mode`
 * decides the computation (p->prune is not used): EAP_PRUNE_ONLY or
 * EAP_BASE; both give the same matrix bit for bit. */
int eap_pairwise(const eap_params* p, const eap_series_set* set, float* out_matrix, int32_t mode,
                 void* cuda_stream, eap_stats* opt_stats);

/* Raw EAPruned on an explicit list of n pairs: out[k] = D(A_ia[k], B_ib[k])
 * if it is <= cutoff[k], else +inf (Section 2.2: an early-abandoned
 * distance signals abandoning by returning +inf).  ia, ib, cutoff, out are
 * device arrays of n elements.  With p->prune = 0 the cut-off is ignored and
 * the plain D is returned; with p->prune = 2 (EABase) out[k] is D, or +inf
 * only if D > cutoff[k]; p->prune = 3 is rejected (EAP_EINVAL). */
int eap_pairs(const eap_params* p, const eap_series_set* a, const eap_series_set* b,
              const int32_t* ia, const int32_t* ib, const float* cutoff, float* out, int32_t n,
              void* cuda_stream, eap_stats* opt_stats);

/* LB_Keogh(A_ia[k], B_ib[k]) for n pairs of equal length (textbook form,
 * Section 5.2): the envelope of A_ia[k] with window w = floor(ratio * L) (or
 * the absolute window) bounds the points of B_ib[k].  Squared or absolute
 * cost as the parameters say.  out: device float[n]; pairs whose lengths
 * differ get 0 (no bound). */
int eap_lb_keogh(const eap_params* p, const eap_series_set* a, const eap_series_set* b,
                 const int32_t* ia, const int32_t* ib, float* out, int32_t n, void* cuda_stream);

/* The lower-bound pass of the 1-NN search (Alg. 2; the lb-keogh2 cascade of
 * Section 5.2), as eap_nn1 runs it ahead of the DP when p->lb is set:
 *   out_lb[q * refs->count + c] = max(LB_Keogh(Q_q, C_c), LB_Keogh(C_c, Q_q))
 * (only the first term when two_way = 0), each the textbook bound -- the
 * envelope U/L of one series over |k - i| <= w bounds the points of the
 * other, cost(c_i, U_i) above U, cost(c_i, L_i) below L -- with
 * w = floor(ratio * L) (CDTW) or the whole series (DTW), and the distance's
 * cost; multiplied by 1 - (4L + 16) 2^-24 so that float32 rounding never
 * lifts it above the pair's float32 DP value.  Pairs of unequal length get 0.
 *   out_lb  device float[queries->count * refs->count], row-major by query.
 * p->kind must be EAP_DTW or EAP_CDTW (else EAP_EINVAL); p->prune and p->lb
 * are not used.  Envelopes are stream-ordered scratch (8 bytes per element of
 * each set); asynchronous on the stream. */
int eap_lb_matrix(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs, int32_t two_way,
                  float* out_lb, void* cuda_stream);

/* eap_pairs without any allocation.  (The paper has no counterpart: this is
 * a deployment variant of eap_pairs.)
 *
 * For callers that cannot allocate device memory during the call -- code with
 * a fixed memory budget committed at start-up, code inside a framework that
 * owns every allocation on the device, or a path where cudaMalloc could block
 * or fail at the wrong time.  Same arguments and results as eap_pairs; the
 * scratch it needs (work-queue head, counters, ERP border sums, WDTW weight
 * table) comes from one 4 MiB array in device memory that is part of the
 * library and that every device loading libeap holds until the process
 * exits.  Nothing is allocated by the call: no cudaMalloc, cudaMallocAsync
 * or cudaFree.
 *   - Limit: the scratch must fit in 4 MiB (4,194,304 bytes).  With
 *     na = a->data_len and nb = b->data_len, it is the sum of these pieces,
 *     each rounded up to a multiple of 256 bytes:
 *         8 + 64                        always (queue head, counters)
 *         4*na + 4*nb                   ERP (border prefix sums)
 *         4 * 32769                     WDTW (weight table, 131,076 bytes)
 *         4*na + 4*nb                   any distance with derivative = 1
 *         16*(na + 1)                   ERP, MSM, TWE (packed row constants)
 *     So DTW and CDTW need 512 bytes at any size; MSM and TWE allow na up
 *     to about 262,000; ERP needs 20*na + 4*nb (+ 4*na + 4*nb with the
 *     derivative).  Larger requests return EAP_EINVAL without launching
 *     anything.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture.
 *   - All calls share the one array, which keeps the previous call's
 *     contents (the call resets what must start at zero).  Calls that overlap
 *     on the GPU -- on different streams, or from different host threads --
 *     race on it; serialise them.
 *   - opt_stats->dp_ms is left at 0 (timing events would be allocations). */
int eap_pairs_noalloc(const eap_params* p, const eap_series_set* a, const eap_series_set* b,
                      const int32_t* ia, const int32_t* ib, const float* cutoff, float* out, int32_t n,
                      void* cuda_stream, eap_stats* opt_stats);

/* ---- sub-sequence search ---------------------------------------------------
 * Sub-sequence search (Section 5.3): for every query Q_q, the start position
 * i in [0, n - L_q] of the long series `ref` that minimises
 * D(znorm(Q_q), znorm(ref[i .. i + L_q - 1])), D = DTW or CDTW (p->kind;
 * window w = floor(window_ratio * L_q) or p->window), computed with
 * EAPruned (p->prune must be 1; p->derivative 0; p->lb is ignored: both
 * LB_Keogh directions are always used).  znorm subtracts the window's mean
 * and divides by its population standard deviation; a deviation of at most
 * 1e-8 normalises the window to zeros.  Ties keep the lowest position.
 * Per query, on the stream (window statistics and the series' envelope are
 * reused by consecutive queries of the same length): sliding means and
 * deviations of every window;
 * for every window the squared Euclidean distance of the normalised window
 * (its diagonal path: an upper bound of D) and LB_Keogh both ways (query
 * envelope vs window, the series' running envelope normalised like the
 * window vs query); the smallest upper bound seeds the cut-off; the windows
 * whose bound does not exceed it are compacted in position order, normalised
 * into scratch in chunks of at most 256 MB and searched by the 1-NN DP with
 * the shared best-so-far (the bound skips a window once the best-so-far
 * falls below it, Alg. 2).
 *   ref       device float[n], 0 <= n < 2^31
 *   queries   series set (device + host mirrors), lengths 1..8192
 *   out_pos   device int64[queries->count]: start position, -1 when L_q > n
 *   out_dist  device float[queries->count]: D, +inf when L_q > n
 * Scratch: about 44 bytes per point of ref plus the chunk buffer, stream-
 * ordered.  The call synchronises the stream once per query (to size the
 * chunks).  opt_stats: pairs = windows, pairs_lb_pruned = windows the bounds
 * removed, cells as in eap_nn1 (effective = windows x L_q^2).
 * Errors: EAP_EINVAL for other distances or modes, EAP_ENOMEM, EAP_EDEVICE. */
int eap_subseq(const eap_params* p, const float* ref, int64_t n, const eap_series_set* queries,
               int64_t* out_pos, float* out_dist, void* cuda_stream, eap_stats* opt_stats);

/* ---- batched uneven workloads ---------------------------------------------
 * Many independent 1-NN problems (datasets of different lengths, sizes and
 * distances) in one persistent DP launch: every (task, query, candidate)
 * item goes through one work queue, tasks ordered longest series first, each
 * task's candidates ranked by diagonal-path cost and sharing its queries'
 * cut-offs (the same search as eap_nn1, Alg. 1 with Alg. 5).  All work is
 * enqueued on the stream with stream-ordered scratch and no host
 * synchronisation, so the whole call can be captured in a CUDA graph.
 * Requirements: every task has prune = 1; LB_Keogh options apply to
 * DTW/CDTW tasks as in eap_nn1. */
typedef struct {
    eap_params     params;
    eap_series_set queries;   /* device + host mirrors */
    eap_series_set refs;
    int32_t*       out_idx;   /* device int32[queries.count] */
    float*         out_dist;  /* device float[queries.count] */
} eap_nn1_task;

int eap_nn1_batch(const eap_nn1_task* tasks, int32_t ntasks, void* cuda_stream, eap_stats* opt_stats);

/* Autotuner for the DP mapping: for each distance and each power-of-two
 * length bucket that `tasks` contain, times the wavefront with strip width
 * W = 4, 5, 8 and 16 (16 lanes per pair for W = 4, 5, 8 when the rows fit,
 * else a warp per pair) and, for unwindowed buckets of 2048 and longer, the
 * CTA-per-pair wavefront with W = 4 and 8, on
 * a sample of that task's own work (at most 64 queries x 512 candidates), and
 * keeps the fastest in a process-wide table that eap_nn1, eap_pairwise,
 * eap_pairs and eap_nn1_batch (W only) then use.  Synchronises the stream;
 * call it before any capture.  With a non-NULL `cache_path` the table is also
 * appended to that text file (one line per entry: kind cost length_bucket W
 * mapping, mapping 1 = warp, 2 = CTA). */
int eap_autotune(const eap_nn1_task* tasks, int32_t ntasks, void* cuda_stream, const char* cache_path);
/* Loads a table written by eap_autotune (missing file: EAP_EINVAL). */
int eap_autotune_load(const char* cache_path);
/* Forgets the tuned table (heuristic defaults again). */
void eap_autotune_reset(void);

/* ---- serving ------------------------------------------------------------- */
typedef struct eap_server eap_server;

typedef struct {
    int64_t hbm_budget_bytes;   /* admission budget for resident sets + in-flight queries (0 = 1/2 of free HBM) */
    int32_t max_inflight;       /* queries in flight at once (0 = 4096) */
    int32_t max_query_len;      /* longest admissible query (0 = 8192) */
    int32_t device;             /* CUDA device ordinal */
    int32_t reserved_;
} eap_serve_config;

eap_server* eap_serve_create(const eap_serve_config* cfg, int* status);
/* Copies a host reference set into HBM and keeps it resident; *set_id names it. */
int eap_serve_add_refset(eap_server* s, const float* h_data, const int64_t* h_offsets,
                         const int32_t* h_lengths, int32_t count, int32_t* set_id);
/* Enqueues one 1-NN query (host buffer, copied) against a resident set.
 * EAP_EAGAIN when the query cannot be admitted now (slots or HBM budget). */
int eap_serve_submit(eap_server* s, int32_t set_id, const eap_params* p, const float* h_query,
                     int32_t len, uint64_t* ticket);
/* EAP_OK with the result once the query is done, EAP_EAGAIN before. */
int eap_serve_poll(eap_server* s, uint64_t ticket, int32_t* idx, float* dist);
/* Blocks until every submitted query is done (bounded by timeout_ms; EAP_ETIMEOUT). */
int eap_serve_drain(eap_server* s, int32_t timeout_ms);
int eap_serve_destroy(eap_server* s);

/* Counters and latency of a server.  Latency is measured from
 * eap_serve_submit to the moment the result is on the host (before any
 * poll), over the queries completed since the last reset. */
typedef struct {
    uint64_t submitted;        /* admitted queries */
    uint64_t rejected;         /* submits answered EAP_EAGAIN */
    uint64_t completed;
    uint64_t batches;          /* device batches launched */
    double   lat_p50_ms, lat_p99_ms, lat_max_ms;
    int64_t  inflight_bytes;   /* HBM footprint charged to admitted, unfinished queries */
    int32_t  inflight;         /* admitted, unfinished queries */
    int32_t  reserved_;
} eap_serve_stats;
/* Fills *out; reset != 0 clears the latency samples and counters afterwards. */
int eap_serve_stats_get(eap_server* s, eap_serve_stats* out, int32_t reset);

const char* eap_strerror(int code);
int32_t eap_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EAP_H */
