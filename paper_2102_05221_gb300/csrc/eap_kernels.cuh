// eap_kernels.cuh -- kernels of libeap around the warp-per-pair DP:
// the persistent work-queue DP kernel (1-NN / all-pairs / explicit pairs),
// the diagonal upper-bound kernel, the per-query candidate sort that seeds
// each query's cut-off, and the small set-up / unpack kernels.
//
// Included by one translation unit per distance (eap_dp_*.cu), which
// instantiates launch_dp<F, ...>() for its functors.
#pragma once

#include "eap_device.cuh"

namespace eapd {

enum { kModeNN1 = 0, kModePairwise = 1, kModePairs = 2 };
enum { kStatPairs = 0, kStatAbandoned = 1, kStatCells = 2, kStatLbPruned = 3, kStatErrors = 4, kStatCount = 8 };

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;
constexpr unsigned kNoIndex = 0xffffffffu;

struct SeriesDev {
    const float* data;
    const int64_t* off;
    const int32_t* len;
    const float* border;   // ERP prefix sums (same offsets as data), else null
    int n;
};

struct DPJob {
    int mode;
    SeriesDev A, B;                    // A = rows (queries / set), B = columns (candidates / set)
    unsigned long long nitems;
    unsigned long long* counter;       // work-queue head
    const int32_t* order;              // nn1: candidates of query q by rank, [A.n x B.n] (null = index order)
    unsigned long long* best;          // nn1: packed (float bits << 32 | index) per query
    const float* cut;                  // pairwise / pairs: per-item cut-off (null = +inf); nn1: the pair's
                                       // own cut-off [A.n x B.n] instead of the shared best-so-far ("Prune")
    float* out;                        // pairwise: n x n matrix; pairs: n results
    const int32_t* ia;                 // pairs
    const int32_t* ib;
    unsigned long long* stats;         // kStatCount counters
    const float* wdtw_table;           // universal WDTW weight table (or null)
    const float* lb;                   // optional per-item lower bound (nn1: [A.n x B.n] by candidate), or null
    const float4* rowpack;             // packed row constants of A (F::kPacked), laid out like A.data, or null
    int bnd_stride;                    // floats of shared memory per warp (per group for group_dp_kernel)
    int no_cut;                        // group_dp_kernel: run the Base DP (no cut-off, every cell)
    int pad_;
};

__device__ __forceinline__ unsigned long long pack_best(float d, unsigned idx) {
    return ((unsigned long long)__float_as_uint(d) << 32) | idx;
}

// Upper-triangle index k -> (i, j), i < j, row-major over i.
__device__ __forceinline__ void tri_decode(unsigned long long k, int n, int& i, int& j) {
    // Rows i hold n-1-i items; find i with S(i) <= k < S(i+1), S(i) = i*(2n-i-1)/2.
    const double nn = (double)n;
    double di = floor(((2.0 * nn - 1.0) - sqrt((2.0 * nn - 1.0) * (2.0 * nn - 1.0) - 8.0 * (double)k)) / 2.0);
    long long ii = (long long)di;
    if (ii < 0) ii = 0;
    auto S = [&](long long r) { return (unsigned long long)(r * (2LL * n - r - 1) / 2); };
    while (ii > 0 && S(ii) > k) --ii;
    while (S(ii + 1) <= k) ++ii;
    i = (int)ii;
    j = (int)(k - S(ii) + (unsigned long long)ii + 1ULL);
}

template <class F, int W, int PM, bool WIN>
__global__ void __launch_bounds__(kThreads) dp_kernel(const DPJob job, const KParams kp) {
    constexpr bool CUTS = PM != kPmBase;   // EAPruned and EABase take a cut-off
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    float* bnd = smem + (threadIdx.x >> 5) * job.bnd_stride;
    unsigned long long cells = 0, npairs = 0, nab = 0, nlb = 0;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(job.counter, 1ULL);
        item = __shfl_sync(EAP_FULL, item, 0);
        if (item >= job.nitems) break;
        int ai, bi;
        float cut = EAP_FINF;
        const unsigned long long* cut_src = nullptr;
        if (job.mode == kModeNN1) {
            const unsigned long long rank = item / (unsigned)job.A.n;
            ai = (int)(item - rank * (unsigned)job.A.n);
            bi = job.order ? __ldg(job.order + (size_t)ai * job.B.n + rank) : (int)rank;
            cut_src = job.best + ai;
            if (CUTS && job.cut) {
                // Pruning only: the pair's own diagonal-path cost, never the shared best-so-far.
                cut = __ldg(job.cut + (size_t)ai * job.B.n + bi);
                cut_src = nullptr;
            } else if (CUTS) {
                unsigned long long cv = 0;
                if (lane == 0) cv = *(volatile const unsigned long long*)cut_src;
                cv = __shfl_sync(EAP_FULL, cv, 0);   // warp-uniform cut-off
                cut = __uint_as_float((unsigned)(cv >> 32));
                if (job.lb && __ldg(job.lb + (size_t)ai * job.B.n + bi) > cut) {   // Alg. 2: LB >= cut-off skips D
                    ++nlb;
                    continue;
                }
            }
        } else if (job.mode == kModePairwise) {
            tri_decode(item, job.A.n, ai, bi);
            if (CUTS && job.cut) cut = __ldg(job.cut + item);
        } else {
            ai = __ldg(job.ia + item);
            bi = __ldg(job.ib + item);
            if (CUTS && job.cut) cut = __ldg(job.cut + item);
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
        if (in.w < abs(in.La - in.Lb)) { d = EAP_FINF; ab = true; }   // no alignment inside the window
        else d = warp_pair<F, W, PM, WIN>(in, bnd, kp, cells, ab);
        ++npairs;
        nab += ab ? 1 : 0;
        if (lane == 0) {
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
        __syncwarp();
    }
    if (job.stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cells += __shfl_xor_sync(EAP_FULL, cells, o);
        if (lane == 0) {
            if (npairs) atomicAdd(job.stats + kStatPairs, npairs);
            if (nab) atomicAdd(job.stats + kStatAbandoned, nab);
            if (cells) atomicAdd(job.stats + kStatCells, cells);
            if (nlb) atomicAdd(job.stats + kStatLbPruned, nlb);
        }
    }
}

// Row constants of every point of a set, precomputed once for the DP
// (F::kPacked): out[off + i] = F::row(x_i, x_{i-1}) with x_{-1} = 0, the
// same function the wavefront would evaluate per step.  One block per series.
template <class F>
__global__ void rowpack_kernel(const SeriesDev S, const KParams kp, float4* __restrict__ out) {
    for (int k = blockIdx.x; k < S.n; k += gridDim.x) {
        const float* x = S.data + S.off[k];
        float4* o = out + S.off[k];
        const int L = S.len[k];
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const float sp = i > 0 ? __ldg(x + i - 1) : 0.f;
            o[i] = F::pack(F::row(__ldg(x + i), sp, kp, nullptr));
        }
    }
}

// Diagonal-path upper bound for every nn1 item (q, c), stored [q][c], or for
// every upper-triangle pair of an all-pairs job.
template <class F>
__global__ void ub_kernel(const DPJob job, const KParams kp, float* __restrict__ ub) {
    const unsigned long long total = job.mode == kModeNN1
        ? (unsigned long long)job.A.n * job.B.n : job.nitems;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < total;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        int ai, bi;
        if (job.mode == kModeNN1) {
            ai = (int)(k / (unsigned)job.B.n);
            bi = (int)(k - (unsigned long long)ai * job.B.n);
        } else {
            tri_decode(k, job.A.n, ai, bi);
        }
        PairIn in;
        const int64_t oa = job.A.off[ai], ob = job.B.off[bi];
        in.A = job.A.data + oa;
        in.B = job.B.data + ob;
        in.La = job.A.len[ai];
        in.Lb = job.B.len[bi];
        in.bA = in.bB = nullptr;
        in.wt = job.wdtw_table ? job.wdtw_table + kWdtwOff - max(in.La, in.Lb) : nullptr;
        in.cut_src = nullptr;
        in.w = pair_window(kp, in.La, in.Lb);
        in.cut = EAP_FINF;
        ub[k] = diag_path_cost<F>(in, kp);
    }
}

// Tiled diagonal bounds for 1-NN: a block stages 32 candidates in shared
// memory (row stride L+1, so lane c reading element k of its own row hits
// bank (c + k) mod 32 when L is a multiple of 32), then each warp runs one
// query against those 32 candidates, lane = candidate, in the same order and
// with the same functor as the untiled kernel (bit-identical bounds).
constexpr int kUbTileCands = 32;
constexpr int kUbTileWarps = 8;

template <class F>
__global__ void __launch_bounds__(32 * kUbTileWarps) ub_tile_kernel(const DPJob job, const KParams kp, int max_lb,
                                                                     float* __restrict__ ub) {
    extern __shared__ float tile[];
    const int stride = max_lb + 1;
    const int c0 = blockIdx.x * kUbTileCands;
    const int ncand = min(kUbTileCands, job.B.n - c0);
    for (int c = threadIdx.x >> 5; c < ncand; c += kUbTileWarps) {
        const float* src = job.B.data + job.B.off[c0 + c];
        const int L = job.B.len[c0 + c];
        for (int k = threadIdx.x & 31; k < L; k += 32) tile[c * stride + k] = __ldg(src + k);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int q = blockIdx.y * kUbTileWarps + (threadIdx.x >> 5); q < job.A.n; q += gridDim.y * kUbTileWarps) {
        if (lane < ncand) {
            const int c = c0 + lane;
            PairIn in;
            in.A = job.A.data + job.A.off[q];
            in.B = nullptr;
            in.La = job.A.len[q];
            in.Lb = job.B.len[c];
            in.bA = in.bB = nullptr;
            in.wt = job.wdtw_table ? job.wdtw_table + kWdtwOff - max(in.La, in.Lb) : nullptr;
            in.cut_src = nullptr;
            in.w = pair_window(kp, in.La, in.Lb);
            in.cut = EAP_FINF;
            ub[(size_t)q * job.B.n + c] = diag_path_cost_b<F>(in, tile + lane * stride, kp);
        }
    }
}

}  // namespace eapd

#include "eap_cta.cuh"
#include "eap_group.cuh"
#include "eap_band.cuh"
