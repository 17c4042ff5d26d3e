// eap_internal.h -- host-side interface between the C-ABI layer (eap_api.cu)
// and the per-distance launch units (eap_dp_*.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/eap.h"
#include "eap_kernels.cuh"

namespace eaph {

struct LaunchCtx {
    eapd::DPJob job;
    eapd::KParams kp;
    int kind;            // eap_kind
    int cost;            // resolved: 0 squared, 1 absolute
    int W;               // strip width per lane (4, 8 or 16)
    int prune;           // 1 EAPruned, 0 Base, 2 EABase (eapd::kPm*)
    float4* rowpack;     // scratch of A.data_len + 1 float4 for the packed row constants (ERP, MSM, TWE)
    int group;           // EAPruned with 8 or 16 lanes per pair (group_dp_kernel); 0 = a warp per pair
    int sms;             // multiprocessors of the device
    int max_rows;        // longest row series (sizes the per-warp shared column)
    int max_cols;        // longest column series (sizes the tiled bound kernel's shared tile)
    int cta;             // 1: CTA-per-pair mapping (long, unwindowed series); 0: warp per pair
    int band = 0;        // windowed DP in band coordinates (Base, EAPruned): strip width (0 = not used)
    int band_g = 0;      // lanes per pair of the band mapping
    int band_exact = 0;  // 1: the launch holds exactly 2w + 2 band positions (no right-of-window addend)
    cudaStream_t stream;
    float* ub;           // diagonal-path upper bounds (output of launch_ub)
};

}  // namespace eaph

namespace eaph {

// 1-NN on device-resident sets (eap_api.cu); returns an EAP_* code.
int nn1_device(const ::eap_params* p, const ::eap_series_set* queries, const ::eap_series_set* refs,
               int32_t* out_idx, float* out_dist, cudaStream_t stream);

// Parameter validation shared with the serving loop; returns an EAP_* code.
int validate_params_ext(const ::eap_params* p);
int validate_set_ext(const ::eap_series_set* s, int* max_len);
// Validation mode only (EAP_CHECK_INPUTS): EAP_EINVAL if data[0..n) holds a NaN or Inf.
int check_finite_run(const float* data, long long n);
int resolve_cost_ext(const ::eap_params* p);

// Strip-width table filled by the autotuner (eap_api.cu).
int tune_get(int kind, int cost, int bucket);
void tune_set(int kind, int cost, int bucket, int w);
void tune_reset();
void map_set(int kind, int cost, int bucket, int m);   // 0 untuned, 1 warp, 2 CTA
int pick_w(int kind, int cost, int max_cols, int prune);
int pick_cta(int kind, int cost, int max_rows, int max_cols, int prune);
int pick_w_cta(int kind, int cost, int max_cols, int prune);
int pick_group(int kind, int cost, int max_rows, int max_cols, int prune, int W);
void pick_w_group(int kind, int cost, int max_rows, int max_cols, int prune, int* W, int* G);
// Band mapping of the windowed DP: strip width and lanes per pair, or 0
// (min_len / max_len: shortest and longest series of the call).
void pick_band(int kind, int prune, const eapd::KParams& kp, int min_len, int max_len, int* W, int* G, int* exact);
int bucket_of(int len);

// Pre-pass launches shared with the batched path (eap_api.cu).
void launch_erp_border(const ::eap_series_set* s, float gap, int cost, float* border, cudaStream_t st);
void launch_wdtw_table(float* tab, float g, float wmax, cudaStream_t st);
// First-derivative series of every series of s into out (same layout as s->data).
void launch_derivative(const ::eap_series_set* s, float* out, cudaStream_t st);
// Whether a distance's DP takes packed row constants (LaunchCtx::rowpack), and
// their computation for one set (kind/cost resolved; out: data_len + 1 float4).
bool kind_packed(int kind);
int launch_rowpack(int kind, int cost, const ::eap_series_set* s, const eapd::KParams& kp, float4* out,
                   cudaStream_t st);
void launch_lb(const ::eap_params* p, const ::eap_series_set* qs, const ::eap_series_set* rs, int two_way,
               float* qU, float* qL, float* rU, float* rL, float* lb, cudaStream_t st);
eapd::KParams kparams_of(const ::eap_params* p);
// One task's EAPruned 1-NN DP launch with eap_nn1's mapping choice (eap_api.cu).
int nn1_dp_launch(const ::eap_params* p, const ::eap_series_set* qs, const ::eap_series_set* rs, const float* bq,
                  const float* br, const float* wt, const int32_t* order, unsigned long long* best, const float* lb,
                  float4* rowpack, unsigned long long* counter, unsigned long long* stats, int max_rows, int max_cols,
                  cudaStream_t st);
int nn1_timed(const ::eap_params* p, const ::eap_series_set* qs, const ::eap_series_set* rs, int32_t* idx,
              float* dist, cudaStream_t st, double* dp_ms);

// Each returns 0 or a CUDA error code (cudaError_t as int).
int launch_dp_dtw(const LaunchCtx& c, bool ub_only);
int launch_dp_cdtw(const LaunchCtx& c, bool ub_only);
int launch_dp_wdtw(const LaunchCtx& c, bool ub_only);
int launch_dp_erp(const LaunchCtx& c, bool ub_only);
int launch_dp_msm(const LaunchCtx& c, bool ub_only);
int launch_dp_twe(const LaunchCtx& c, bool ub_only);

// Shared launch code for one functor (used by the units above).
template <class F, int W, bool WIN>
int run_dp(const LaunchCtx& c) {
    using namespace eapd;
    void (*kern)(const DPJob, const KParams) = c.prune == kPmPruned ? dp_kernel<F, W, kPmPruned, WIN>
                                               : c.prune == kPmEA    ? dp_kernel<F, W, kPmEA, WIN>
                                                                     : dp_kernel<F, W, kPmBase, WIN>;
    const size_t smem = (size_t)kWarpsPerBlock * c.job.bnd_stride * sizeof(float);
    cudaError_t e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    unsigned long long grid = (unsigned long long)per_sm * c.sms;
    const unsigned long long need = (c.job.nitems + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, smem, c.stream>>>(c.job, c.kp);
    return (int)cudaGetLastError();
}

// DP of a windowed distance in band coordinates (band_dp_kernel): Base, or
// early abandoning for EAPruned and EABase (every cell of a row is computed
// either way), G lanes per pair.
template <class F, int W, int G, bool EXACT>
int run_band(const LaunchCtx& c) {
    using namespace eapd;
    void (*kern)(const DPJob, const KParams) =
        c.prune == kPmBase ? band_dp_kernel<F, W, G, kPmBase, EXACT> : band_dp_kernel<F, W, G, kPmPruned, EXACT>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    unsigned long long grid = (unsigned long long)per_sm * c.sms;
    const unsigned long long per_block = (unsigned long long)kWarpsPerBlock * (32 / G);
    const unsigned long long need = (c.job.nitems + per_block - 1) / per_block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, 0, c.stream>>>(c.job, c.kp);
    return (int)cudaGetLastError();
}

// G-lane groups (32/G pairs per warp), EAPruned only; one boundary column per group.
template <class F, int W, int G, bool WIN>
int run_group(const LaunchCtx& c) {
    using namespace eapd;
    void (*kern)(const DPJob, const KParams) = group_dp_kernel<F, W, G, WIN>;
    const size_t smem = (size_t)kWarpsPerBlock * (32 / G) * c.job.bnd_stride * sizeof(float);
    cudaError_t e;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return (int)e;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    unsigned long long grid = (unsigned long long)per_sm * c.sms;
    const unsigned long long per_block = (unsigned long long)kWarpsPerBlock * (32 / G);
    const unsigned long long need = (c.job.nitems + per_block - 1) / per_block;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, smem, c.stream>>>(c.job, c.kp);
    return (int)cudaGetLastError();
}

template <class F>
int run_ub(const LaunchCtx& c) {
    using namespace eapd;
    if (c.job.mode == kModeNN1 && c.max_cols > 0 && c.max_cols <= 1024) {
        // Tiled path: 32 candidates per block in shared memory.
        const size_t smem = (size_t)kUbTileCands * (c.max_cols + 1) * sizeof(float);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(ub_tile_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
        }
        const unsigned gx = (unsigned)((c.job.B.n + kUbTileCands - 1) / kUbTileCands);
        unsigned gy = (unsigned)((c.job.A.n + kUbTileWarps - 1) / kUbTileWarps);
        const unsigned cap = (unsigned)std::max(1, 8 * c.sms / (int)std::max(1u, gx));
        if (gy > cap) gy = cap;
        ub_tile_kernel<F><<<dim3(gx, gy), 32 * kUbTileWarps, smem, c.stream>>>(c.job, c.kp, c.max_cols, c.ub);
        return (int)cudaGetLastError();
    }
    const unsigned long long total = c.job.mode == kModeNN1
        ? (unsigned long long)c.job.A.n * c.job.B.n : c.job.nitems;
    if (total == 0) return 0;
    unsigned long long blocks = (total + 255) / 256;
    const unsigned long long cap = (unsigned long long)c.sms * 16;
    if (blocks > cap) blocks = cap;
    ub_kernel<F><<<(unsigned)blocks, 256, 0, c.stream>>>(c.job, c.kp, c.ub);
    return (int)cudaGetLastError();
}

// CTA-per-pair launch: 8 warps per pair, one full boundary column in shared memory.
template <class F, int W>
int run_cta(const LaunchCtx& c) {
    using namespace eapd;
    void (*kern)(const DPJob, const KParams) = c.prune ? cta_dp_kernel<F, W, true> : cta_dp_kernel<F, W, false>;
    const size_t smem = (size_t)(c.max_rows + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1));
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCtaThreads, smem);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    unsigned long long grid = (unsigned long long)per_sm * c.sms;
    if (grid > c.job.nitems) grid = c.job.nitems;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kCtaThreads, smem, c.stream>>>(c.job, c.kp);
    return (int)cudaGetLastError();
}

// Packed row constants of the row set (F::kPacked) into c.rowpack.
template <class F>
int run_rowpack(const LaunchCtx& c) {
    using namespace eapd;
    if (!c.rowpack) return (int)cudaErrorInvalidValue;
    if (c.job.A.n <= 0) return 0;
    const int blocks = std::min(c.job.A.n, std::max(1, c.sms) * 8);
    rowpack_kernel<F><<<blocks, 128, 0, c.stream>>>(c.job.A, c.kp, c.rowpack);
    return (int)cudaGetLastError();
}

template <class F, bool WIN>
int run_kind(const LaunchCtx& c, bool ub_only) {
    if (ub_only) return run_ub<F>(c);
    LaunchCtx d = c;
    if constexpr (F::kPacked) {
        const int e = run_rowpack<F>(c);
        if (e) return e;
        d.job.rowpack = c.rowpack;
    }
    if constexpr (!WIN) {
        if (c.cta) return c.W >= 8 ? run_cta<F, 8>(d) : run_cta<F, 4>(d);
    } else {
        if (c.band) {
            if (c.band_exact) {
                if (c.band_g == 8 && c.band == 13) return run_band<F, 13, 8, true>(d);
                if (c.band_g == 4 && c.band == 26) return run_band<F, 26, 4, true>(d);
            } else if (c.band_g == 8) {
                if (c.band == 4) return run_band<F, 4, 8, false>(d);
                if (c.band == 8) return run_band<F, 8, 8, false>(d);
                if (c.band == 14) return run_band<F, 14, 8, false>(d);
                if (c.band == 16) return run_band<F, 16, 8, false>(d);
            } else if (c.band_g == 16) {
                if (c.band == 7) return run_band<F, 7, 16, false>(d);
                if (c.band == 16) return run_band<F, 16, 16, false>(d);
            }
            return (int)cudaErrorInvalidValue;
        }
    }
    if (c.group && (c.prune == eapd::kPmPruned || c.prune == eapd::kPmBase)) {
        d.job.no_cut = c.prune == eapd::kPmBase ? 1 : 0;
        if (c.group == 8) {
            if (c.W == 4) return run_group<F, 4, 8, WIN>(d);
            if (c.W == 8) return run_group<F, 8, 8, WIN>(d);
        } else if (c.group == 16) {
            if (c.W == 4) return run_group<F, 4, 16, WIN>(d);
            if (c.W == 5) return run_group<F, 5, 16, WIN>(d);
            if (c.W == 8) return run_group<F, 8, 16, WIN>(d);
        }
        return (int)cudaErrorInvalidValue;
    }
    switch (c.W) {
        case 4: return run_dp<F, 4, WIN>(d);
        case 8: return run_dp<F, 8, WIN>(d);
        case 16: return run_dp<F, 16, WIN>(d);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace eaph
