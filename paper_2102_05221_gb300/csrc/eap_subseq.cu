// eap_subseq.cu -- sub-sequence search under EAPruned DTW / CDTW (Section 5.3):
// the window of a long series closest to a query, both z-normalised.
//
// Per query of length m over a series of n points (npos = n - m + 1 windows):
//   1. subseq_norm_kernel: mean and 1/deviation of every window, from double
//      sums slid along a run of positions per thread;
//   2. subseq_query_kernel: the normalised query and its envelope;
//      envelope_blocks_kernel / envelope_combine_kernel: the running max/min
//      of the series over +-w in O(n);
//   3. subseq_ub_kernel: over shared-memory tiles of the series, the squared
//      Euclidean distance of each normalised window (its diagonal path: an
//      upper bound of D), abandoned once above the smallest found so far;
//      the smallest, inflated by its rounding bound, seeds the best-so-far;
//   4. subseq_lb_kernel: LB_Keogh both ways (query envelope vs window; the
//      series' envelope, normalised with the window's mean and deviation,
//      vs query), abandoned once above the seed, and the order-preserving
//      compaction of the windows whose bound does not exceed it;
//   5. chunks of survivors are normalised into scratch and run through the
//      1-NN DP kernel (EAPruned, one query, shared best-so-far, the lower
//      bound as Alg. 2's filter before each pair).
// The normalised values of a window are the same float expression in the
// bound pass and in the DP input, so the bounds hold for the DP's own values.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/eap.h"
#include "eap_internal.h"

using namespace eapd;

namespace {

constexpr int kNormRun = 256;            // windows per thread in the mean / deviation pass
constexpr int kBoundThreads = 256;       // windows per block in the bound pass
constexpr int kCompactBlock = 1024;      // windows per block in the compaction
constexpr double kFlatSd = 1e-8;         // deviation at or below which a window normalises to zeros
constexpr size_t kChunkBytes = 256u << 20;   // normalised survivor windows materialised at once

__device__ __forceinline__ float znorm1(float x, float mu, float isd) {
    return __fmul_rn(__fsub_rn(x, mu), isd);
}

__device__ __forceinline__ float cost_rt(float a, float b, int cost) {
    return cost == 0 ? pcost<0>(a, b) : pcost<1>(a, b);
}

// Mean and 1/deviation (population) of every window T[i .. i+m-1].
__global__ void subseq_norm_kernel(const float* __restrict__ T, long long npos, int m, float* __restrict__ mu,
                                   float* __restrict__ isd) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long i0 = t * kNormRun;
    if (i0 >= npos) return;
    const long long i1 = min(npos, i0 + (long long)kNormRun);
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < m; ++k) {
        const double x = __ldg(T + i0 + k);
        s1 += x;
        s2 += x * x;
    }
    const double inv_m = 1.0 / m;
    for (long long i = i0; i < i1; ++i) {
        // Sums in FP64 (the variance is a difference of large terms); the
        // scale 1/deviation only needs float accuracy.
        const double mean = s1 * inv_m;
        const double var = fmax(fma(-mean, mean, s2 * inv_m), 0.0);
        mu[i] = (float)mean;
        isd[i] = var > kFlatSd * kFlatSd ? __frsqrt_rn((float)var) : 0.f;
        if (i + 1 < i1) {
            const double a = __ldg(T + i), b = __ldg(T + i + m);
            s1 += b - a;
            s2 += b * b - a * a;
        }
    }
}

// One block: the query normalised (two passes in double) and its envelope
// over +-w (LB_Keogh, Section 5.2).
__global__ void subseq_query_kernel(const float* __restrict__ q, int m, int w, float* __restrict__ zq,
                                    float* __restrict__ U, float* __restrict__ L) {
    __shared__ double red[32];
    __shared__ double s_mu, s_sd;
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(EAP_FULL, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        double s = 0.0;
        if (threadIdx.x == 0)
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
        __syncthreads();
        return s;
    };
    double a = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) a += (double)q[k];
    const double sum = block_sum(a);
    if (threadIdx.x == 0) s_mu = sum / m;
    __syncthreads();
    double b = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const double d = (double)q[k] - s_mu;
        b += d * d;
    }
    const double ss = block_sum(b);
    if (threadIdx.x == 0) s_sd = sqrt(ss / m);
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x)
        zq[k] = s_sd > kFlatSd ? (float)(((double)q[k] - s_mu) / s_sd) : 0.f;
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        float u = -EAP_FINF, l = EAP_FINF;
        for (int j = max(0, k - w); j <= min(m - 1, k + w); ++j) {
            u = fmaxf(u, zq[j]);
            l = fminf(l, zq[j]);
        }
        U[k] = u;
        L[k] = l;
    }
}

// Running max / min of the raw series over +-w in O(n) (van Herk / Gil-Werman):
// blocks of K = 2w + 1 points; per block the prefix (g) and suffix (h)
// extrema; the window [i - w, i + w] clipped to the series spans at most two
// blocks, and max(h[a], g[b]) over its ends a, b bounds it (exactly when it
// spans two blocks, from above when it lies inside one: a wider envelope
// still gives a valid lower bound).
__global__ void envelope_blocks_kernel(const float* __restrict__ T, long long n, long long K, float* __restrict__ gU,
                                       float* __restrict__ gL, float* __restrict__ hU, float* __restrict__ hL) {
    const long long nblk = (n + K - 1) / K;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nblk;
         b += (long long)gridDim.x * blockDim.x) {
        const long long a0 = b * K, a1 = min(n, a0 + K);
        float u = -EAP_FINF, l = EAP_FINF;
        for (long long i = a0; i < a1; ++i) {
            const float x = __ldg(T + i);
            u = fmaxf(u, x);
            l = fminf(l, x);
            gU[i] = u;
            gL[i] = l;
        }
        u = -EAP_FINF;
        l = EAP_FINF;
        for (long long i = a1 - 1; i >= a0; --i) {
            const float x = __ldg(T + i);
            u = fmaxf(u, x);
            l = fminf(l, x);
            hU[i] = u;
            hL[i] = l;
        }
    }
}

__global__ void envelope_combine_kernel(long long n, int w, const float* __restrict__ gU, const float* __restrict__ gL,
                                        const float* __restrict__ hU, const float* __restrict__ hL,
                                        float* __restrict__ U, float* __restrict__ L) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = max(0LL, i - w), b = min(n - 1, i + (long long)w);
        U[i] = fmaxf(hU[a], gU[b]);
        L[i] = fminf(hL[a], gL[b]);
    }
}

// Shared-memory tile of the series for the windows of one block: the block's
// kBoundThreads windows start at i0 and span kBoundThreads + m - 1 points.
__device__ __forceinline__ void load_tile(float* dst, const float* __restrict__ src, long long i0, long long nT,
                                          int tile) {
    for (int k = threadIdx.x; k < tile; k += blockDim.x) {
        const long long g = i0 + k;
        dst[k] = g < nT ? __ldg(src + g) : 0.f;
    }
}

// Upper bound of every window: the squared Euclidean distance of the
// normalised window (its diagonal path, summed in the order of the path),
// abandoned as soon as the partial sum exceeds the smallest bound found so
// far; only the minimum is kept (one atomicMin per improvement).  Shared
// memory: the block's tile of T and the normalised query.
__global__ void __launch_bounds__(kBoundThreads) subseq_ub_kernel(
        const float* __restrict__ T, long long npos, int m, const float* __restrict__ mu,
        const float* __restrict__ isd, const float* __restrict__ zq, int cost, unsigned* __restrict__ ub_min) {
    extern __shared__ float sm[];
    const int tile = kBoundThreads + m - 1;
    float* sT = sm;
    float* sq = sT + tile;
    const long long i0 = (long long)blockIdx.x * kBoundThreads;
    load_tile(sT, T, i0, npos + m - 1, tile);
    for (int k = threadIdx.x; k < m; k += blockDim.x) sq[k] = zq[k];
    __syncthreads();
    const long long i = i0 + threadIdx.x;
    if (i >= npos) return;
    const float mi = mu[i], si = isd[i];
    // The running minimum as bits: sums are >= 0, whose floats order as their
    // bit patterns, and the initial all-ones pattern is above every one.
    unsigned best = *(volatile const unsigned*)ub_min;
    float acc = 0.f;
    int k = 0;
    for (; k + 32 <= m; k += 32) {
#pragma unroll 8
        for (int u = 0; u < 32; ++u) acc = __fadd_rn(acc, cost_rt(sq[k + u], znorm1(sT[threadIdx.x + k + u], mi, si), cost));
        if (__float_as_uint(acc) > best) {
            best = *(volatile const unsigned*)ub_min;
            if (__float_as_uint(acc) > best) return;   // this window cannot hold the minimum
        }
    }
    for (; k < m; ++k) acc = __fadd_rn(acc, cost_rt(sq[k], znorm1(sT[threadIdx.x + k], mi, si), cost));
    if (__float_as_uint(acc) < best) atomicMin(ub_min, __float_as_uint(acc));
}

// LB_Keogh both ways for every window (query envelope vs window; the series'
// envelope, normalised like the window, vs query), shrunk by the rounding of
// the sums so the bound stays below the DP's float D.  A window is abandoned
// as soon as its partial bound exceeds the cut-off thr: the partial sum is
// itself a lower bound, larger than thr, which is all the compaction and the
// DP's filter need.  (Both bounds in one pass: the larger of the two crosses
// the cut-off sooner than either alone.)  Shared memory: tiles of T and of
// its envelope, the query's envelope.
__global__ void __launch_bounds__(kBoundThreads) subseq_lb_kernel(
        const float* __restrict__ T, const float* __restrict__ UT, const float* __restrict__ LT,
        long long npos, int m, const float* __restrict__ mu, const float* __restrict__ isd,
        const float* __restrict__ zq, const float* __restrict__ Uq, const float* __restrict__ Lq, int cost,
        const float* __restrict__ thr_p, float* __restrict__ lb) {
    extern __shared__ float sm[];
    const int tile = kBoundThreads + m - 1;
    float* sT = sm;
    float* sU = sT + tile;
    float* sL = sU + tile;
    float* sq = sL + tile;
    float* sqU = sq + m;
    float* sqL = sqU + m;
    const long long i0 = (long long)blockIdx.x * kBoundThreads;
    const long long nT = npos + m - 1;
    load_tile(sT, T, i0, nT, tile);
    load_tile(sU, UT, i0, nT, tile);
    load_tile(sL, LT, i0, nT, tile);
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        sq[k] = zq[k];
        sqU[k] = Uq[k];
        sqL[k] = Lq[k];
    }
    __syncthreads();
    const long long i = i0 + threadIdx.x;
    if (i >= npos) return;
    const float mi = mu[i], si = isd[i];
    const float shrink = 1.f - (float)(4 * m + 16) * 5.9604645e-8f;
    const float thr = *thr_p;
    float lq = 0.f, lc = 0.f;
    auto point = [&](int k) {
        const float z = znorm1(sT[threadIdx.x + k], mi, si);
        const float qk = sq[k];
        const float ex = z > sqU[k] ? cost_rt(z, sqU[k], cost) : (z < sqL[k] ? cost_rt(z, sqL[k], cost) : 0.f);
        lq = __fadd_rn(lq, ex);
        const float uz = znorm1(sU[threadIdx.x + k], mi, si), lz = znorm1(sL[threadIdx.x + k], mi, si);
        const float ec = qk > uz ? cost_rt(qk, uz, cost) : (qk < lz ? cost_rt(qk, lz, cost) : 0.f);
        lc = __fadd_rn(lc, ec);
    };
    int k = 0;
    for (; k + 32 <= m; k += 32) {
#pragma unroll 8
        for (int u = 0; u < 32; ++u) point(k + u);
        const float part = fmaxf(lq, lc) * shrink;
        if (part > thr) { lb[i] = part; return; }
    }
    for (; k < m; ++k) point(k);
    lb[i] = fmaxf(lq, lc) * shrink;
}

// Cut-off seed: the smallest upper bound, inflated by the rounding bound of
// an m-term sum, so that the window achieving it has a float D below it.
__global__ void subseq_seed_kernel(const unsigned* __restrict__ ub_min, int m, float* __restrict__ thr,
                                   unsigned long long* __restrict__ best) {
    const float u = __uint_as_float(*ub_min);
    const float s = u == EAP_FINF ? EAP_FINF : __fmul_ru(u, 1.f + (float)(4 * m + 16) * 5.9604645e-8f);
    *thr = s;
    *best = ((unsigned long long)__float_as_uint(s) << 32) | kNoIndex;
}

// Order-preserving compaction of the windows with lb <= thr, in three steps:
// per-block counts, one-block exclusive scan, per-block writes.
__global__ void compact_count_kernel(const float* __restrict__ lb, long long npos, const float* __restrict__ thr,
                                     int* __restrict__ counts) {
    const float t = *thr;
    const long long base = (long long)blockIdx.x * kCompactBlock;
    int c = 0;
    for (int k = threadIdx.x; k < kCompactBlock; k += blockDim.x) {
        const long long i = base + k;
        c += (i < npos && lb[i] <= t) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(EAP_FULL, c, o);
    __shared__ int wsum[32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += wsum[k];
        counts[blockIdx.x] = s;
    }
}

__global__ void compact_scan_kernel(int* __restrict__ counts, int nb, int* __restrict__ total) {
    // One block of 1024 threads: chunked Hillis-Steele scan with a running carry.
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int k = base + threadIdx.x;
        const int v = k < nb ? counts[k] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int a = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += a;
            __syncthreads();
        }
        if (k < nb) counts[k] = carry + buf[threadIdx.x] - v;   // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void compact_write_kernel(const float* __restrict__ lb, long long npos, const float* __restrict__ thr,
                                     const int* __restrict__ offsets, int* __restrict__ surv,
                                     float* __restrict__ surv_lb) {
    const float t = *thr;
    const long long base = (long long)blockIdx.x * kCompactBlock;
    __shared__ int wsum[32];
    __shared__ int run;
    if (threadIdx.x == 0) run = offsets[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k0 = 0; k0 < kCompactBlock; k0 += blockDim.x) {
        const long long i = base + k0 + threadIdx.x;
        const bool keep = i < npos && lb[i] <= t;
        const unsigned bal = __ballot_sync(EAP_FULL, keep);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = run;
        for (int k = 0; k < warp; ++k) before += wsum[k];
        if (keep) {
            const int at = before + __popc(bal & ((1u << lane) - 1u));
            surv[at] = (int)i;
            surv_lb[at] = lb[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int k = 0; k < nw; ++k) s += wsum[k];
            run += s;
        }
        __syncthreads();
    }
}

// Normalised windows of survivors [s0, s0 + cnt) into buf, their offsets and
// lengths (indexed by survivor number) and the chunk's evaluation order.
// Survivors whose bound already exceeds the best-so-far are skipped (the DP
// skips them by the same test before reading their data).
__global__ void subseq_gather_kernel(const float* __restrict__ T, const int* __restrict__ surv,
                                     const float* __restrict__ surv_lb, const float* __restrict__ mu,
                                     const float* __restrict__ isd, int m, int s0, int cnt,
                                     const unsigned long long* __restrict__ best, float* __restrict__ buf,
                                     int64_t* __restrict__ offs, int32_t* __restrict__ lens,
                                     int32_t* __restrict__ order) {
    const float cut = __uint_as_float((unsigned)(*(volatile const unsigned long long*)best >> 32));
    for (int c = blockIdx.x; c < cnt; c += gridDim.x) {
        const int s = s0 + c;
        if (threadIdx.x == 0) {
            offs[s] = (int64_t)c * m;
            lens[s] = m;
            order[c] = s;
        }
        if (surv_lb[s] > cut) continue;
        const int pos = surv[s];
        const float mi = mu[pos], si = isd[pos];
        float* dst = buf + (size_t)c * m;
        for (int k = threadIdx.x; k < m; k += blockDim.x) dst[k] = znorm1(__ldg(T + pos + k), mi, si);
    }
}

__global__ void subseq_result_kernel(const unsigned long long* __restrict__ best, const int* __restrict__ surv,
                                     int q, int64_t* __restrict__ out_pos, float* __restrict__ out_dist,
                                     unsigned long long* __restrict__ stats) {
    const unsigned long long b = *best;
    const unsigned ix = (unsigned)(b & 0xffffffffu);
    if (ix == kNoIndex) {
        out_pos[q] = -1;
        out_dist[q] = EAP_FINF;
        if (stats) atomicAdd(stats + kStatErrors, 1ULL);   // the seed's own window always beats the seed
    } else {
        out_pos[q] = surv[ix];
        out_dist[q] = __uint_as_float((unsigned)(b >> 32));
    }
}

__global__ void subseq_none_kernel(int q, int64_t* out_pos, float* out_dist) {
    out_pos[q] = -1;
    out_dist[q] = EAP_FINF;
}

int sms_of_device() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return sms;
}

}  // namespace

extern "C" int eap_subseq(const eap_params* p, const float* ref, int64_t n, const eap_series_set* queries,
                          int64_t* out_pos, float* out_dist, void* cuda_stream, eap_stats* opt_stats) {
    int rc = eaph::validate_params_ext(p);
    if (rc) return rc;
    if (p->kind != EAP_DTW && p->kind != EAP_CDTW) return EAP_EINVAL;
    if (p->prune != 1 || p->derivative != 0) return EAP_EINVAL;
    int mq = 0;
    if ((rc = eaph::validate_set_ext(queries, &mq))) return rc;
    if (n < 0 || n >= (1LL << 31) || (n > 0 && !ref)) return EAP_EINVAL;
    if ((rc = eaph::check_finite_run(ref, n))) return rc;
    if (queries->count > 0 && (!out_pos || !out_dist)) return EAP_EINVAL;
    if (opt_stats) std::memset(opt_stats, 0, sizeof(*opt_stats));
    const int nq = queries->count;
    if (nq == 0) return EAP_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int sms = sms_of_device();
    if (sms <= 0) return EAP_EDEVICE;
    const int cost = eaph::resolve_cost_ext(p);

    // Scratch for the longest query; windows of shorter ones fit in it.
    const int mmax = mq;
    const long long npos_max = n;   // a query of length 1 has n windows
    const int nb_max = (int)std::max<long long>(1, (npos_max + kCompactBlock - 1) / kCompactBlock);
    size_t used = 0;
    auto take = [&](size_t bytes) { const size_t o = (used + 255) & ~(size_t)255; used = o + bytes; return o; };
    const size_t o_mu = take(sizeof(float) * std::max<long long>(npos_max, 1));
    const size_t o_isd = take(sizeof(float) * std::max<long long>(npos_max, 1));
    const size_t o_lb = take(sizeof(float) * std::max<long long>(npos_max, 1));
    const size_t o_UT = take(sizeof(float) * std::max<int64_t>(n, 1));
    const size_t o_LT = take(sizeof(float) * std::max<int64_t>(n, 1));
    const size_t o_gU = take(sizeof(float) * std::max<int64_t>(n, 1));
    const size_t o_gL = take(sizeof(float) * std::max<int64_t>(n, 1));
    const size_t o_hU = take(sizeof(float) * std::max<int64_t>(n, 1));
    const size_t o_hL = take(sizeof(float) * std::max<int64_t>(n, 1));
    const size_t o_zq = take(sizeof(float) * mmax);
    const size_t o_Uq = take(sizeof(float) * mmax);
    const size_t o_Lq = take(sizeof(float) * mmax);
    const size_t o_qoff = take(sizeof(int64_t));
    const size_t o_qlen = take(sizeof(int32_t));
    const size_t o_umin = take(sizeof(unsigned));
    const size_t o_thr = take(sizeof(float));
    const size_t o_best = take(sizeof(unsigned long long));
    const size_t o_ctr = take(sizeof(unsigned long long));
    const size_t o_stats = take(sizeof(unsigned long long) * kStatCount);
    const size_t o_cnt = take(sizeof(int) * nb_max);
    const size_t o_total = take(sizeof(int));
    const size_t o_surv = take(sizeof(int) * std::max<long long>(npos_max, 1));
    const size_t o_slb = take(sizeof(float) * std::max<long long>(npos_max, 1));
    const size_t o_offs = take(sizeof(int64_t) * std::max<long long>(npos_max, 1));
    const size_t o_lens = take(sizeof(int32_t) * std::max<long long>(npos_max, 1));
    const size_t chunk_cap = std::max<size_t>(1024, kChunkBytes / (sizeof(float) * (size_t)std::max(1, mmax)));
    const size_t o_order = take(sizeof(int32_t) * chunk_cap);
    const size_t o_buf = take(sizeof(float) * chunk_cap * (size_t)std::max(1, mmax));
    char* base = nullptr;
    if (cudaMallocAsync((void**)&base, used, st) != cudaSuccess) { cudaGetLastError(); return EAP_ENOMEM; }
    auto F = [&](size_t o) { return (float*)(base + o); };
    unsigned long long* d_stats = (unsigned long long*)(base + o_stats);
    int e = (int)cudaMemsetAsync(d_stats, 0, sizeof(unsigned long long) * kStatCount, st);
    unsigned long long h_lbskip = 0, h_pos = 0, h_eff = 0;
    // Window statistics and the series' envelope depend on the query only
    // through its length (and the window it implies): reused across
    // consecutive queries of the same length.
    int stats_m = -1, stats_w = -1;
    for (int q = 0; q < nq && !e && rc == EAP_OK; ++q) {
        const int m = queries->h_lengths[q];
        const long long npos = n - m + 1;
        if (npos <= 0) {
            subseq_none_kernel<<<1, 1, 0, st>>>(q, out_pos, out_dist);
            e |= (int)cudaGetLastError();
            continue;
        }
        // Window of the pair (m, m).
        const KParams kp = eaph::kparams_of(p);
        long long w = m;
        if (p->kind == EAP_CDTW) {
            if (p->window >= 0) w = p->window;
            else if (p->window_ratio >= 0.f) w = (long long)std::floor((double)p->window_ratio * (double)m);
        }
        const int wenv = (int)std::min<long long>(w, m);
        const float* qd = queries->data + queries->h_offsets[q];
        if (m != stats_m)
            subseq_norm_kernel<<<(unsigned)((npos + (long long)kNormRun * 128 - 1) / ((long long)kNormRun * 128)), 128,
                                 0, st>>>(ref, npos, m, F(o_mu), F(o_isd));
        subseq_query_kernel<<<1, 256, 0, st>>>(qd, m, wenv, F(o_zq), F(o_Uq), F(o_Lq));
        if (wenv != stats_w) {
            const long long K = 2LL * wenv + 1, nblk = (n + K - 1) / K;
            envelope_blocks_kernel<<<(unsigned)std::min<long long>((nblk + 127) / 128, (long long)sms * 8), 128, 0, st>>>(
                ref, n, K, F(o_gU), F(o_gL), F(o_hU), F(o_hL));
            envelope_combine_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, (long long)sms * 32), 256, 0, st>>>(
                n, wenv, F(o_gU), F(o_gL), F(o_hU), F(o_hL), F(o_UT), F(o_LT));
        }
        stats_m = m;
        stats_w = wenv;
        e |= (int)cudaMemsetAsync(base + o_umin, 0xff, sizeof(unsigned), st);   // all ones: above every sum's bits
        const unsigned gridb = (unsigned)((npos + kBoundThreads - 1) / kBoundThreads);
        const size_t smem_ub = sizeof(float) * ((size_t)(kBoundThreads + m - 1) + (size_t)m);
        if (smem_ub > 48 * 1024)
            e |= (int)cudaFuncSetAttribute(subseq_ub_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ub);
        subseq_ub_kernel<<<gridb, kBoundThreads, smem_ub, st>>>(ref, npos, m, F(o_mu), F(o_isd), F(o_zq), cost,
                                                                (unsigned*)(base + o_umin));
        subseq_seed_kernel<<<1, 1, 0, st>>>((const unsigned*)(base + o_umin), m, F(o_thr),
                                             (unsigned long long*)(base + o_best));
        const size_t smem_lb = sizeof(float) * (3 * (size_t)(kBoundThreads + m - 1) + 3 * (size_t)m);
        if (smem_lb > 48 * 1024)
            e |= (int)cudaFuncSetAttribute(subseq_lb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_lb);
        subseq_lb_kernel<<<gridb, kBoundThreads, smem_lb, st>>>(ref, F(o_UT), F(o_LT), npos, m, F(o_mu), F(o_isd),
                                                                F(o_zq), F(o_Uq), F(o_Lq), cost, F(o_thr), F(o_lb));
        const int nb = (int)((npos + kCompactBlock - 1) / kCompactBlock);
        compact_count_kernel<<<nb, 256, 0, st>>>(F(o_lb), npos, F(o_thr), (int*)(base + o_cnt));
        compact_scan_kernel<<<1, 1024, 0, st>>>((int*)(base + o_cnt), nb, (int*)(base + o_total));
        compact_write_kernel<<<nb, 256, 0, st>>>(F(o_lb), npos, F(o_thr), (const int*)(base + o_cnt),
                                                 (int*)(base + o_surv), F(o_slb));
        e |= (int)cudaGetLastError();
        int S = 0;
        if (!e) e |= (int)cudaMemcpyAsync(&S, base + o_total, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (!e) e |= (int)cudaStreamSynchronize(st);
        if (e) break;
        h_pos += (unsigned long long)npos;
        h_lbskip += (unsigned long long)(npos - S);
        h_eff += (unsigned long long)npos * (unsigned long long)m * (unsigned long long)m;
        // The query as a one-series set.
        const int64_t zero = 0;
        e |= (int)cudaMemcpyAsync(base + o_qoff, &zero, sizeof(int64_t), cudaMemcpyHostToDevice, st);
        e |= (int)cudaMemcpyAsync(base + o_qlen, &m, sizeof(int32_t), cudaMemcpyHostToDevice, st);
        for (int s0 = 0; s0 < S && !e; s0 += (int)chunk_cap) {
            const int cnt = (int)std::min<long long>((long long)chunk_cap, (long long)S - s0);
            subseq_gather_kernel<<<(unsigned)std::min(cnt, sms * 16), 128, 0, st>>>(
                ref, (const int*)(base + o_surv), F(o_slb), F(o_mu), F(o_isd), m, s0, cnt,
                (const unsigned long long*)(base + o_best), F(o_buf), (int64_t*)(base + o_offs),
                (int32_t*)(base + o_lens), (int32_t*)(base + o_order));
            e |= (int)cudaMemsetAsync(base + o_ctr, 0, sizeof(unsigned long long), st);
            eaph::LaunchCtx c;
            std::memset(&c, 0, sizeof(c));
            c.job.mode = kModeNN1;
            c.job.A = SeriesDev{F(o_zq), (const int64_t*)(base + o_qoff), (const int32_t*)(base + o_qlen), nullptr, 1};
            c.job.B = SeriesDev{F(o_buf), (const int64_t*)(base + o_offs), (const int32_t*)(base + o_lens), nullptr, S};
            c.job.nitems = (unsigned long long)cnt;
            c.job.counter = (unsigned long long*)(base + o_ctr);
            c.job.order = (const int32_t*)(base + o_order);
            c.job.best = (unsigned long long*)(base + o_best);
            c.job.lb = F(o_slb);
            c.job.stats = d_stats;
            c.job.bnd_stride = ((m + 1) + 31) & ~31;
            c.kp = kp;
            c.kind = p->kind;
            c.cost = cost;
            c.prune = kPmPruned;
            eaph::pick_w_group(p->kind, cost, m, m, kPmPruned, &c.W, &c.group);
            c.sms = sms;
            c.max_rows = m;
            c.max_cols = m;
            c.cta = eaph::pick_cta(p->kind, cost, m, m, kPmPruned);
            if (c.cta) { c.W = eaph::pick_w_cta(p->kind, cost, m, kPmPruned); c.group = 0; }
            c.stream = st;
            e |= p->kind == EAP_DTW ? eaph::launch_dp_dtw(c, false) : eaph::launch_dp_cdtw(c, false);
        }
        subseq_result_kernel<<<1, 1, 0, st>>>((const unsigned long long*)(base + o_best), (const int*)(base + o_surv),
                                              q, out_pos, out_dist, d_stats);
        e |= (int)cudaGetLastError();
    }
    unsigned long long h[kStatCount] = {};
    if (!e) e |= (int)cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(base, st);
    if (!e) e |= (int)cudaStreamSynchronize(st);
    if (e) return EAP_EDEVICE;
    if (opt_stats) {
        opt_stats->pairs = h_pos;
        opt_stats->pairs_lb_pruned = h_lbskip + h[kStatLbPruned];
        opt_stats->pairs_abandoned = h[kStatAbandoned];
        opt_stats->cells_computed = h[kStatCells];
        opt_stats->cells_effective = h_eff;
    }
    if (h[kStatErrors]) return EAP_EINTERNAL;
    return EAP_OK;
}
