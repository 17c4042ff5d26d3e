// eap_api.cu -- the C ABI of libeap (declared in include/eap.h): argument
// validation, stream-ordered scratch, and the launch sequence of each entry
// point, plus the small kernels that do not depend on the distance.
//
// 1-NN (Alg. 1 with Alg. 5 as the distance) runs as
//   init best-so-far  ->  [ERP borders | WDTW weights]  ->  diagonal upper
//   bounds (every query x candidate)  ->  per-query sort of the candidates by
//   that bound + cut-off seed  ->  persistent DP over (rank, query) items  ->
//   unpack of the packed best-so-far into (index, distance).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/eap.h"
#include "eap_internal.h"

using namespace eapd;

namespace {

constexpr int kMaxSeriesLen = 8192;   // longest series a call accepts (shared-memory column of the DP)

// ---------------------------------------------------------------------------
// Distance-independent kernels.
// ---------------------------------------------------------------------------
__global__ void init_best_kernel(unsigned long long* best, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        best[i] = pack_best(EAP_FINF, kNoIndex);
}

// One block per query: sorts that query's candidates by their diagonal-path
// cost (bitonic sort of packed (bound bits, index) keys in shared memory, in
// chunks of `chunk` candidates), writes the evaluation order, and seeds the
// query's cut-off with the smallest bound (no index: any real D <= bound wins).
__global__ void sort_seed_kernel(const float* __restrict__ ub, int nb, int chunk, int32_t* __restrict__ order,
                                 unsigned long long* __restrict__ best) {
    extern __shared__ unsigned long long keys[];
    const int q = blockIdx.x;
    const float* u = ub + (size_t)q * nb;
    int32_t* o = order + (size_t)q * nb;
    unsigned long long gmin = ~0ULL;
    for (int base = 0; base < nb; base += chunk) {
        const int cnt = min(chunk, nb - base);
        for (int i = threadIdx.x; i < chunk; i += blockDim.x)
            keys[i] = i < cnt ? pack_best(u[base + i], (unsigned)(base + i)) : ~0ULL;
        __syncthreads();
        for (int k = 2; k <= chunk; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const unsigned long long a = keys[i], b = keys[l];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) { keys[i] = b; keys[l] = a; }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) o[base + i] = (int32_t)(keys[i] & 0xffffffffu);
        if (keys[0] < gmin) gmin = keys[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned bits = (unsigned)(gmin >> 32);
        best[q] = ((unsigned long long)bits << 32) | kNoIndex;
    }
}

__global__ void unpack_kernel(const unsigned long long* __restrict__ best, int n, int32_t* __restrict__ idx,
                              float* __restrict__ dist, unsigned long long* stats) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long b = best[i];
        const unsigned ix = (unsigned)(b & 0xffffffffu);
        const float d = __uint_as_float((unsigned)(b >> 32));
        if (ix == kNoIndex) {
            idx[i] = -1;
            dist[i] = EAP_FINF;
            // A finite seed left in place means no candidate met its own bound.
            if (d != EAP_FINF && stats) atomicAdd(stats + kStatErrors, 1ULL);
        } else {
            idx[i] = (int32_t)ix;
            dist[i] = d;
        }
    }
}

// Per-query result as a packed key for a min-reduction across candidate
// shards: (distance bits << 32) | (index + offset), or (+inf bits << 32) |
// 0xffffffff when no candidate of the shard is finite.  Distances are >= 0,
// so the keys order like (distance, index) -- Alg. 1's strict "<" over
// candidates in index order -- as unsigned and as signed 64-bit integers.
__global__ void keys_kernel(const unsigned long long* __restrict__ best, int n, long long offset,
                            unsigned long long* __restrict__ keys, unsigned long long* stats) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long b = best ? best[i] : pack_best(EAP_FINF, kNoIndex);   // null: an empty shard
        const unsigned ix = (unsigned)(b & 0xffffffffu);
        if (ix == kNoIndex) {
            if (__uint_as_float((unsigned)(b >> 32)) != EAP_FINF && stats) atomicAdd(stats + kStatErrors, 1ULL);
            keys[i] = pack_best(EAP_FINF, kNoIndex);
        } else {
            keys[i] = (b & 0xffffffff00000000ULL) | (unsigned long long)((long long)ix + offset);
        }
    }
}

__global__ void keys_unpack_kernel(const unsigned long long* __restrict__ keys, int n, int32_t* __restrict__ idx,
                                   float* __restrict__ dist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const unsigned ix = (unsigned)(k & 0xffffffffu);
        idx[i] = ix == kNoIndex ? -1 : (int32_t)ix;
        dist[i] = ix == kNoIndex ? EAP_FINF : __uint_as_float((unsigned)(k >> 32));
    }
}

// ERP borders (Eq. ERP): border[off + k] = sum_{m <= k+1} cost(x_m, g), in order.
__global__ void erp_border_kernel(const float* __restrict__ data, const int64_t* __restrict__ off,
                                  const int32_t* __restrict__ len, int n, float g, int cost,
                                  float* __restrict__ border) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float* x = data + off[s];
        float* b = border + off[s];
        float acc = 0.f;
        const int L = len[s];
        for (int k = 0; k < L; ++k) {
            const float c = cost == 0 ? pcost<0>(x[k], g) : pcost<1>(x[k], g);
            acc = __fadd_rn(acc, c);
            b[k] = acc;
        }
    }
}

// Universal WDTW weight table (Eq. WDTW): entry kWdtwOff + u holds
// wmax / (1 + exp(-g u / 2)), u = 2d - L, evaluated in double and rounded.
// First-derivative estimate of every series of a set, for the derivative
// distances (DDTW and the others, Section 2.3; Keogh & Pazzani's estimate):
// d_i = ((x_i - x_{i-1}) + (x_{i+1} - x_{i-1}) / 2) / 2 at interior points,
// the first and last points take their neighbour's estimate, and series of
// one or two points (no interior point) give zeros.  Blocks stride over the
// series, threads over the points (coalesced); out has the layout of data.
__global__ void derivative_kernel(const float* __restrict__ data, const int64_t* __restrict__ off,
                                  const int32_t* __restrict__ len, int n, float* __restrict__ out) {
    for (int s = blockIdx.x; s < n; s += gridDim.x) {
        const float* x = data + off[s];
        float* d = out + off[s];
        const int L = len[s];
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            float v = 0.f;
            if (L > 2) {
                const int k = min(max(i, 1), L - 2);
                // In double, rounded to float once: the differences of float
                // inputs and the halvings are exact in double, so each value is
                // the float nearest the estimate.  (Rounded in float at every
                // step, a distance much smaller than the derivative values --
                // cancellation -- missed 1e-4 relative against the FP64
                // oracle: 1.1e-4 for ERP between two 3-point series.)
                const double xl = __ldg(x + k - 1), xc = __ldg(x + k), xr = __ldg(x + k + 1);
                v = __double2float_rn(((xc - xl) + (xr - xl) * 0.5) * 0.5);
            }
            d[i] = v;
        }
    }
}

__global__ void wdtw_table_kernel(float* tab, double g, double wmax) {
    const int n = 2 * kWdtwOff + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double u = (double)(i - kWdtwOff);
        tab[i] = (float)(wmax / (1.0 + exp(-g * (u / 2.0))));
    }
}

__global__ void diag_zero_kernel(float* m, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m[(size_t)i * n + i] = 0.f;
}

__global__ void fill_nn_empty_kernel(int32_t* idx, float* dist, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        idx[i] = -1;
        dist[i] = EAP_FINF;
    }
}

// LB_Keogh for explicit pairs (textbook form): envelope of A over
// |k - i| <= w, bound on the points of B.  One warp per pair.
__global__ void lb_keogh_pairs_kernel(const SeriesDev A, const SeriesDev B, const int32_t* __restrict__ ia,
                                      const int32_t* __restrict__ ib, int n, KParams kp, int cost,
                                      float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps) {
        const int a = ia[k], b = ib[k];
        const int L = A.len[a];
        float acc = 0.f;
        if (B.len[b] == L) {
            const float* x = A.data + A.off[a];
            const float* y = B.data + B.off[b];
            const int w = pair_window(kp, L, L);
            for (int i = lane; i < L; i += 32) {
                float U = -EAP_FINF, Lo = EAP_FINF;
                const int k0 = max(0, i - w), k1 = min(L - 1, i + w);
                for (int j = k0; j <= k1; ++j) {
                    const float v = __ldg(x + j);
                    U = fmaxf(U, v);
                    Lo = fminf(Lo, v);
                }
                const float c = __ldg(y + i);
                float e = 0.f;
                if (c > U) e = cost == 0 ? pcost<0>(c, U) : pcost<1>(c, U);
                else if (c < Lo) e = cost == 0 ? pcost<0>(c, Lo) : pcost<1>(c, Lo);
                acc = __fadd_rn(acc, e);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(EAP_FULL, acc, o));
        }
        if (lane == 0) out[k] = acc;
    }
}

// Envelope of every series for LB_Keogh (Section 5.2): U[k] / Lo[k] = max /
// min of x over |m - k| <= w, w the pair window of an equal-length pair.
// One block per series.  With `smem_len` > 0 (the launch's longest series,
// 4 floats per point of shared memory) the van Herk / Gil-Werman form runs in
// O(L): the series is cut into blocks of k = 2w + 1 points, each block keeps
// running maxima / minima from its start (g) and from its end (h), and a
// window [a, b] -- at most k points, so it spans at most two blocks -- is
// max(h[a], g[b]); a window inside one block starts at the block (then g[b])
// or ends at the series' end (then h[a]).  Max and min are exact, so the
// result is the same as scanning each window.  Without shared memory each
// point scans its window.
__global__ void envelope_kernel(const SeriesDev S, KParams kp, float* __restrict__ U, float* __restrict__ Lo,
                                int smem_len) {
    extern __shared__ float env_sh[];
    const int s = blockIdx.x;
    const int L = S.len[s];
    const float* x = S.data + S.off[s];
    float* u = U + S.off[s];
    float* lo = Lo + S.off[s];
    int w = pair_window(kp, L, L);
    if (w > L) w = L;
    if (smem_len > 0) {
        const int k = 2 * w + 1;
        float* gmax = env_sh;
        float* hmax = gmax + smem_len;
        float* gmin = hmax + smem_len;
        float* hmin = gmin + smem_len;
        const int nb = (L + k - 1) / k;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const int a0 = b * k, a1 = min(L, a0 + k);
            float m = -EAP_FINF, n = EAP_FINF;
            for (int i = a0; i < a1; ++i) {
                const float v = __ldg(x + i);
                m = fmaxf(m, v);
                n = fminf(n, v);
                gmax[i] = m;
                gmin[i] = n;
            }
            m = -EAP_FINF;
            n = EAP_FINF;
            for (int i = a1 - 1; i >= a0; --i) {
                const float v = __ldg(x + i);
                m = fmaxf(m, v);
                n = fminf(n, v);
                hmax[i] = m;
                hmin[i] = n;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const int a = max(0, i - w), b = min(L - 1, i + w);
            float mu, ml;
            if (a / k != b / k) {
                mu = fmaxf(hmax[a], gmax[b]);
                ml = fminf(hmin[a], gmin[b]);
            } else if (a % k == 0) {
                mu = gmax[b];
                ml = gmin[b];
            } else {
                mu = hmax[a];
                ml = hmin[a];
            }
            u[i] = mu;
            lo[i] = ml;
        }
        return;
    }
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        float uu = -EAP_FINF, ll = EAP_FINF;
        const int a = max(0, k - w), b = min(L - 1, k + w);
        for (int m = a; m <= b; ++m) {
            const float v = __ldg(x + m);
            uu = fmaxf(uu, v);
            ll = fminf(ll, v);
        }
        u[k] = uu;
        lo[k] = ll;
    }
}

// Envelopes of every series of a set (max_len: its longest series).
void launch_envelope(const SeriesDev& S, const KParams& ke, int max_len, float* U, float* Lo, cudaStream_t st) {
    if (S.n <= 0) return;
    const size_t smem = (size_t)4 * max_len * sizeof(float);
    const bool fast = smem <= 48 * 1024;
    envelope_kernel<<<S.n, 128, fast ? smem : 0, st>>>(S, ke, U, Lo, fast ? max_len : 0);
}

// Lower bound of every (query, candidate) pair, [q][c]: LB_Keogh(Q, C) (the
// query's envelope bounds C), and with two_way also LB_Keogh(C, Q); the
// larger one is kept (the lb-keogh2 cascade of Section 5.2 in one pass).
// Pairs of unequal length get 0.  The bound is shrunk by 1 - (4L + 16) 2^-24
// so float rounding can never lift it above the float32 DP value of the pair.
//
// Tiled like a matrix product: a block owns TQ queries x TC candidates and
// walks the points in chunks of kLbK, staging the chunk of every series of
// the tile (query: U, L, x; candidate: y, U, L) in shared memory once, so each
// candidate chunk is read from memory once per query tile instead of once per
// query.  Thread (ty, tx) of the (TQ/4) x (TC/4) block accumulates the 4 x 4
// pairs (ty + (TQ/4) a, tx + (TC/4) b).  Per point and direction, the textbook
// case split "cost(c_i, U_i) if c_i > U_i, cost(c_i, L_i) if c_i < L_i, else
// 0" is cost(c_i, clamp(c_i, L_i, U_i)): the same difference, rounded the same
// way.  Points past a series' end are padded so that they add 0.
constexpr int kLbK = 32;
constexpr int kLbStride = kLbK + 1;   // shared-memory row pitch (conflict-free column reads)

__device__ __forceinline__ float lb_term(float y, float lo, float up, int cost, float acc) {
    const float d = __fsub_rn(y, fminf(fmaxf(y, lo), up));
    return cost == 0 ? __fmaf_rn(d, d, acc) : __fadd_rn(acc, fabsf(d));
}

template <int TQ, int TC>
constexpr size_t lb_smem_bytes() { return sizeof(float) * 3 * (TQ + TC) * kLbStride; }

template <int TQ, int TC>
__global__ void __launch_bounds__((TQ / 4) * (TC / 4)) lb_matrix_kernel(
        const SeriesDev Q, const SeriesDev R, const float* __restrict__ qU, const float* __restrict__ qL,
        const float* __restrict__ rU, const float* __restrict__ rL, int cost, int two_way, float* __restrict__ lb) {
    constexpr int NX = TC / 4, NY = TQ / 4, NT = NX * NY;
    extern __shared__ float lbs[];
    float* sqU = lbs;                          // [TQ][kLbStride]
    float* sqL = sqU + TQ * kLbStride;
    float* sqx = sqL + TQ * kLbStride;
    float* scy = sqx + TQ * kLbStride;         // [TC][kLbStride]
    float* scU = scy + TC * kLbStride;
    float* scL = scU + TC * kLbStride;
    __shared__ int s_len[TQ + TC];
    __shared__ int64_t s_off[TQ + TC];
    __shared__ int s_max;
    const int q0 = blockIdx.y * TQ, c0 = blockIdx.x * TC;
    const int tx = threadIdx.x % NX, ty = threadIdx.x / NX;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < TQ + TC; k += NT) {
        int len = 0;
        int64_t off = 0;
        if (k < TQ) {
            if (q0 + k < Q.n) { len = Q.len[q0 + k]; off = Q.off[q0 + k]; }
        } else if (c0 + k - TQ < R.n) {
            len = R.len[c0 + k - TQ];
            off = R.off[c0 + k - TQ];
        }
        s_len[k] = len;
        s_off[k] = off;
        atomicMax(&s_max, len);
    }
    __syncthreads();
    const int maxlen = s_max;
    float acc1[4][4], acc2[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) { acc1[a][b] = 0.f; acc2[a][b] = 0.f; }
    const int warp = threadIdx.x >> 5, nwarps = NT / 32;
    for (int i0 = 0; i0 < maxlen; i0 += kLbK) {
        // Stage the chunk: TQ + TC series x 32 points, one warp per series row at a time.
        for (int r = warp; r < TQ + TC; r += nwarps) {
            const int col = threadIdx.x & 31;
            const int i = i0 + col;
            const bool in = i < s_len[r];
            const int64_t o = s_off[r] + i;
            if (r < TQ) {
                sqU[r * kLbStride + col] = in ? __ldg(qU + o) : EAP_FINF;
                sqL[r * kLbStride + col] = in ? __ldg(qL + o) : -EAP_FINF;
                if (two_way) sqx[r * kLbStride + col] = in ? __ldg(Q.data + o) : 0.f;
            } else {
                const int rc = r - TQ;
                scy[rc * kLbStride + col] = in ? __ldg(R.data + o) : 0.f;
                if (two_way) {
                    scU[rc * kLbStride + col] = in ? __ldg(rU + o) : EAP_FINF;
                    scL[rc * kLbStride + col] = in ? __ldg(rL + o) : -EAP_FINF;
                }
            }
        }
        __syncthreads();
        const int kend = min(kLbK, maxlen - i0);
        for (int k = 0; k < kend; ++k) {
            float u[4], l[4], x[4], y[4], cu[4], cl[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                u[a] = sqU[(ty + NY * a) * kLbStride + k];
                l[a] = sqL[(ty + NY * a) * kLbStride + k];
                if (two_way) x[a] = sqx[(ty + NY * a) * kLbStride + k];
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                y[b] = scy[(tx + NX * b) * kLbStride + k];
                if (two_way) { cu[b] = scU[(tx + NX * b) * kLbStride + k]; cl[b] = scL[(tx + NX * b) * kLbStride + k]; }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc1[a][b] = lb_term(y[b], l[a], u[a], cost, acc1[a][b]);
                    if (two_way) acc2[a][b] = lb_term(x[a], cl[b], cu[b], cost, acc2[a][b]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int qa = ty + NY * a, q = q0 + qa;
        if (q >= Q.n) continue;
        const int Lq = s_len[qa];
        const float shrink = 1.0f - (float)(4 * Lq + 16) * 5.9604645e-8f;   // 1 - (4L + 16) 2^-24
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int cb = tx + NX * b, c = c0 + cb;
            if (c >= R.n) continue;
            const float v = s_len[TQ + cb] == Lq ? __fmul_rn(fmaxf(acc1[a][b], acc2[a][b]), shrink) : 0.f;
            lb[(size_t)q * R.n + c] = v;
        }
    }
}

template <int TQ, int TC>
void lb_launch(const SeriesDev& Q, const SeriesDev& R, const float* qU, const float* qL, const float* rU,
               const float* rL, int cost, int two_way, float* lb, cudaStream_t st) {
    const dim3 grid((unsigned)((R.n + TC - 1) / TC), (unsigned)((Q.n + TQ - 1) / TQ));
    lb_matrix_kernel<TQ, TC><<<grid, (TQ / 4) * (TC / 4), lb_smem_bytes<TQ, TC>(), st>>>(Q, R, qU, qL, rU, rL, cost,
                                                                                         two_way, lb);
}

void launch_lb_matrix(const SeriesDev& Q, const SeriesDev& R, const float* qU, const float* qL, const float* rU,
                      const float* rL, int cost, int two_way, float* lb, cudaStream_t st) {
    if (Q.n <= 0 || R.n <= 0) return;
    // 64 x 64 tiles: smaller ones (better wave fill for few queries) measured
    // slower -- less reuse of each staged chunk, fewer warps per SM.
    cudaFuncSetAttribute(lb_matrix_kernel<64, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)lb_smem_bytes<64, 64>());
    lb_launch<64, 64>(Q, R, qU, qL, rU, rL, cost, two_way, lb, st);
}

// ---------------------------------------------------------------------------
// Host helpers.
// ---------------------------------------------------------------------------
int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return sms;
}

int resolve_cost(const eap_params* p) {
    if (p->kind == EAP_MSM) return 1;
    if (p->cost == EAP_COST_SQ || p->cost == EAP_COST_ABS) return p->cost;
    return (p->kind == EAP_ERP || p->kind == EAP_TWE) ? 1 : 0;
}

bool finite_f(float x) { return std::isfinite(x); }

int validate_params(const eap_params* p) {
    if (!p) return EAP_EINVAL;
    if (p->kind < EAP_DTW || p->kind > EAP_TWE) return EAP_EINVAL;
    if (p->cost != EAP_COST_DEFAULT && p->cost != EAP_COST_SQ && p->cost != EAP_COST_ABS) return EAP_EINVAL;
    if (p->prune < 0 || p->prune > 3) return EAP_EINVAL;
    if (p->derivative != 0 && p->derivative != 1) return EAP_EINVAL;
    if (p->lb < EAP_LB_NONE || p->lb > EAP_LB_KEOGH2) return EAP_EINVAL;
    if (!finite_f(p->window_ratio)) return EAP_EINVAL;
    if (p->kind == EAP_WDTW && !(finite_f(p->wdtw_g) && p->wdtw_g >= 0.f && finite_f(p->wdtw_wmax) && p->wdtw_wmax > 0.f))
        return EAP_EINVAL;
    if (p->kind == EAP_ERP && !finite_f(p->erp_gap)) return EAP_EINVAL;
    if (p->kind == EAP_MSM && !(finite_f(p->msm_c) && p->msm_c >= 0.f)) return EAP_EINVAL;
    if (p->kind == EAP_TWE && !(finite_f(p->twe_nu) && p->twe_nu >= 0.f && finite_f(p->twe_lambda) && p->twe_lambda >= 0.f))
        return EAP_EINVAL;
    return EAP_OK;
}

// Validation mode (EAP_CHECK_INPUTS=1 in the environment): input series are
// scanned for NaN / Inf before any work, after a device-wide synchronisation
// (so data produced on any stream is complete), on the legacy stream.
__device__ unsigned g_nonfinite_flag;

__global__ void nonfinite_kernel(const float* __restrict__ data, const int64_t* __restrict__ off,
                                 const int32_t* __restrict__ len, int n, long long span) {
    // n series at (off, len), or, with off == nullptr, one run of `span` values.
    const int count = off ? n : 1;
    for (int s = blockIdx.x; s < count; s += gridDim.x) {
        const float* x = off ? data + off[s] : data;
        const long long L = off ? (long long)len[s] : span;
        bool bad = false;
        for (long long i = threadIdx.x; i < L; i += blockDim.x) bad |= !isfinite(__ldg(x + i));
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&g_nonfinite_flag, 1u);
    }
}

bool check_inputs_enabled() {
    const char* e = std::getenv("EAP_CHECK_INPUTS");
    return e && e[0] && e[0] != '0';
}

// EAP_OK when every value is finite, EAP_EINVAL otherwise, EAP_EDEVICE on a CUDA error.
int check_finite(const float* data, const int64_t* off, const int32_t* len, int n, long long span) {
    if ((off && n <= 0) || (!off && span <= 0)) return EAP_OK;
    const unsigned zero = 0;
    unsigned flag = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return EAP_EDEVICE;
    if (cudaMemcpyToSymbol(g_nonfinite_flag, &zero, sizeof(zero)) != cudaSuccess) return EAP_EDEVICE;
    const int blocks = off ? std::min(n, 4096) : 1;
    nonfinite_kernel<<<blocks, 256>>>(data, off, len, n, span);
    if (cudaGetLastError() != cudaSuccess) return EAP_EDEVICE;
    if (cudaMemcpyFromSymbol(&flag, g_nonfinite_flag, sizeof(flag)) != cudaSuccess) return EAP_EDEVICE;
    return flag ? EAP_EINVAL : EAP_OK;
}

int validate_set(const eap_series_set* s, int* max_len) {
    if (!s || s->count < 0) return EAP_EINVAL;
    int mx = 0;
    if (s->count == 0) { *max_len = 0; return EAP_OK; }
    if (!s->data || !s->offsets || !s->lengths || !s->h_offsets || !s->h_lengths) return EAP_EINVAL;
    for (int i = 0; i < s->count; ++i) {
        const int32_t L = s->h_lengths[i];
        const int64_t o = s->h_offsets[i];
        if (L <= 0 || L > kMaxSeriesLen || o < 0 || o + L > s->data_len) return EAP_EINVAL;
        if (L > mx) mx = L;
    }
    *max_len = mx;
    if (check_inputs_enabled()) return check_finite(s->data, s->offsets, s->lengths, s->count, 0);
    return EAP_OK;
}

KParams make_kparams(const eap_params* p) {
    KParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.wdtw_g = p->wdtw_g;
    kp.wdtw_wmax = p->wdtw_wmax;
    kp.erp_gap = p->erp_gap;
    kp.msm_c = p->msm_c;
    kp.twe_nu = p->twe_nu;
    kp.twe_nu2 = 2.0f * p->twe_nu;
    kp.twe_lambda = p->twe_lambda;
    kp.windowed = (p->kind == EAP_CDTW || p->kind == EAP_ERP) ? 1 : 0;
    kp.window_abs = p->window;
    kp.window_ratio = p->window_ratio;
    return kp;
}

// Strip width per lane (32*W columns per panel): the autotuned choice for the
// distance and the power-of-two length bucket when eap_autotune has measured
// one, else a default; EAP_W overrides both (tuning runs).
std::mutex g_tune_mu;
int g_tune[6][2][16] = {};   // [kind][cost][bucket] -> W, 0 = not tuned

int length_bucket(int len) {
    int b = 0;
    while ((1 << b) < len && b < 15) ++b;
    return b;
}

// Warp-per-pair or CTA-per-pair for unwindowed series (EAP_MAP=warp|cta and
// the autotuner's map override the defaults).  CTA from 6144 points, where a
// warp's boundary column no longer fits beside enough warps.  For a 1-NN
// search of at most 32 queries (n_queries; 0 = not a 1-NN search) also from
// 2048 points for DTW and MSM: with few queries the warp mapping runs most of
// a query's candidates at once, before any of them has tightened the
// query's cut-off, while the CTA mapping runs about three pairs per SM.
// Measured, 16 queries x 300-600 candidates: DTW 4.8 -> 2.5 ms at L = 2048,
// 10.1 -> 4.0 ms at 4096; MSM 14.3 -> 12.1 and 32.0 -> 21.2 ms.  With 128
// queries the warp mapping is faster up to 4096 points (DTW 9.9 against
// 15.6 ms at 2048), and TWE gains nothing consistent below 6144.  Windowed
// bands keep the warp mapping: their panels' rows shift by a panel width,
// which starves the CTA pipeline.
int length_bucket(int len);
std::mutex g_map_mu;
int g_map[6][2][16] = {};   // [kind][cost][bucket] -> 0 untuned, 1 warp, 2 CTA (set by the autotuner)

int choose_cta(int kind, int cost, int max_rows, int max_cols, int prune, int n_queries = 0) {
    if (kind == EAP_CDTW || kind == EAP_ERP) return 0;
    if (prune == kPmEA) return 0;   // EABase runs on the warp mapping only
    const char* e = std::getenv("EAP_MAP");
    if (e && std::strcmp(e, "warp") == 0) return 0;
    if (e && std::strcmp(e, "cta") == 0) return 1;
    if (kind >= 0 && kind < 6 && (cost == 0 || cost == 1)) {
        std::lock_guard<std::mutex> lk(g_map_mu);
        const int m = g_map[kind][cost][length_bucket(std::max(max_rows, max_cols))];
        if (m) return m == 2 ? 1 : 0;
    }
    if (max_rows >= 6144 && max_cols >= 6144) return 1;
    if (n_queries > 0 && n_queries <= 32 && prune == kPmPruned && (kind == EAP_DTW || kind == EAP_MSM) &&
        max_rows >= 2048 && max_cols >= 2048)
        return 1;
    return 0;
}

int choose_w(int kind, int cost, int max_cols, int prune) {
    const char* e = std::getenv("EAP_W");
    if (e) {
        const int w = std::atoi(e);
        if (w == 4 || w == 5 || w == 8 || w == 16) return w;
    }
    if (prune == kPmPruned && kind >= 0 && kind < 6 && (cost == 0 || cost == 1)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        const int t = g_tune[kind][cost][length_bucket(max_cols)];
        if (t) return t;
    }
    // Base and EABase compute (nearly) every cell: wide strips, except for the
    // windowed distances, whose Base DP runs in 8-lane groups (a narrow
    // staircase wastes fewer cells outside the band |i - j| <= w; measured on
    // 1000 x 1000 x 512: CDTW W = 8, ERP W = 4 fastest).
    if (prune == kPmBase && kind == EAP_CDTW) return 8;
    if (prune == kPmBase && kind == EAP_ERP) return 4;
    if (prune != kPmPruned) return max_cols > 256 ? 16 : (max_cols > 128 ? 8 : 4);
    // TWE's 7-op cell amortises the per-step work better at W = 8 when the
    // 16-lane groups do not apply.
    if (kind == EAP_TWE && max_cols > 2048) return 8;
    // With 16-lane groups, W = 5 is faster for DTW, MSM and TWE (1000 x 1000
    // x 512: 4.9 / 39.6 / 34.8 ms against 5.0 / 40.5 / 36.4 at W = 4), W = 4
    // for WDTW (4.0 ms against 4.2) and the windowed distances.
    if (kind == EAP_CDTW || kind == EAP_ERP || kind == EAP_WDTW) return 4;
    return 5;
}

// Strip width of the CTA-per-pair mapping: EAP_W, else the autotuner's width
// for the length bucket, else 8.  Measured on 16 x 200 1-NN at L = 8192 with
// the CTA kernel: W = 8 against 4, DTW 26.1 -> 16.5 ms, MSM 97.1 -> 75.0 ms
// (TWE already ran at 8); the per-step work of the CTA wavefront (boundary
// read and write, row constants, shuffle) is spread over twice the cells.
int choose_w_cta(int kind, int cost, int max_cols, int prune) {
    const char* e = std::getenv("EAP_W");
    if (e) {
        const int w = std::atoi(e);
        if (w == 4 || w == 5 || w == 8 || w == 16) return w;
    }
    if (prune == kPmPruned && kind >= 0 && kind < 6 && (cost == 0 || cost == 1)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        const int t = g_tune[kind][cost][length_bucket(max_cols)];
        if (t) return t;
    }
    return 8;
}

// Lanes per pair for the EAPruned DP: 8 or 16 (group_dp_kernel, several pairs
// per warp) or 0 (a warp per pair).  EAP_G overrides (8, 16, or 32 = warp).
// Groups keep one boundary column per group in shared memory, so they are
// limited to rows <= 2048 (16 lanes) and <= 1024 (8 lanes); strip widths
// 4, 5, 8 (16 lanes) and 4, 8 (8 lanes) are built.  Default: 16 lanes
// (measured on the 1000 x 1000 x 512 workload: 9-17% less DP time than a
// warp per pair for every distance; 8 lanes and W = 8 were slower).
int choose_group(int kind, int cost, int max_rows, int max_cols, int prune, int W) {
    (void)cost; (void)max_cols;
    const bool windowed = kind == EAP_CDTW || kind == EAP_ERP;
    const bool base_windowed = prune == kPmBase && windowed;
    if (prune != kPmPruned && !base_windowed) return 0;
    int g = base_windowed ? (max_rows <= 1024 ? 8 : 16) : ((W == 4 || W == 5) ? 16 : 0);
    const char* e = std::getenv("EAP_G");
    if (e) g = std::atoi(e);
    if (g == 8 && max_rows <= 1024 && (W == 4 || W == 8)) return 8;
    if (g == 16 && max_rows <= 2048 && (W == 4 || W == 5 || W == 8)) return 16;
    return 0;
}

// Band mapping (band_dp_kernel) for the DP of CDTW and ERP in every mode
// (Base; EAPruned and EABase abandon on the band's cut, and the lanes compute
// whole band rows either way).  A row of the window plus the cell left of it
// is 2w + 2 positions.  When every pair of the call has the same window and
// a built launch holds exactly 2w + 2 positions, that exact launch is taken
// (no addend right of the window); otherwise the narrowest built launch with
// at least 2w + 3 positions for the widest pair.  A launch is sized for the
// widest band, so it is used only where every pair fills at least half of it
// and every series is at least as long as the widest band (else the
// column-panel kernels do less work).  EAP_BAND=0 turns it off, EAP_BAND=2
// takes it whenever the band fits a launch (tests); EAP_BAND_EXACT=0 skips
// the exact launches; EAP_BAND_G = 4, 8 or 16 restricts the lanes per pair.
void choose_band(int kind, int prune, const KParams& kp, int min_len, int max_len, int* W, int* G, int* exact) {
    *W = 0;
    *G = 0;
    *exact = 0;
    if (kind != EAP_CDTW && kind != EAP_ERP) return;
    if (prune != kPmBase && prune != kPmPruned && prune != kPmEA) return;
    const char* e = std::getenv("EAP_BAND");
    const int mode = e ? std::atoi(e) : 1;
    if (mode == 0) return;
    auto window = [&](int L) -> long long {
        if (kp.window_abs >= 0) return kp.window_abs;
        if (kp.window_ratio >= 0.f) return (long long)std::floor((double)kp.window_ratio * (double)L);
        return -1;
    };
    const long long w_hi = window(max_len), w_lo = window(min_len);
    if (w_hi < 0) return;
    const char* g = std::getenv("EAP_BAND_G");
    const int gsel = g ? std::atoi(g) : 0;
    const char* ex = std::getenv("EAP_BAND_EXACT");
    const bool try_exact = !(ex && ex[0] == '0');
    // Exact launches (W, G): 8 lanes x 13 and 4 lanes x 26 hold 104 = 2w + 2
    // positions (w = 51).  8 lanes first (measured on 1000 x 1000 x 512).
    static const int kExact[][2] = {{13, 8}, {26, 4}};
    if (try_exact && w_lo == w_hi && (mode == 2 || 2 * w_hi + 2 <= min_len)) {
        for (const auto& b : kExact) {
            if (gsel && gsel != b[1]) continue;
            if ((long long)b[0] * b[1] != 2 * w_hi + 2) continue;
            *W = b[0];
            *G = b[1];
            *exact = 1;
            return;
        }
    }
    const long long B = 2 * w_hi + 3;
    static const int kBands8[][2] = {{4, 8}, {8, 8}, {14, 8}, {16, 8}, {16, 16}};     // (W, G), padded
    static const int kBands16[][2] = {{4, 8}, {7, 16}, {16, 16}};
    // 8 lanes per pair except for the abandoning ERP DP, whose wider cells
    // need fewer per lane to keep registers and occupancy up.
    const int gpref = gsel ? gsel : ((kind == EAP_ERP && prune != kPmBase) ? 16 : 8);
    const int (*bands)[2] = gpref == 16 ? kBands16 : kBands8;
    const int nb = gpref == 16 ? (int)(sizeof(kBands16) / sizeof(kBands16[0])) : (int)(sizeof(kBands8) / sizeof(kBands8[0]));
    for (int k = 0; k < nb; ++k) {
        const int* b = bands[k];
        const long long P = (long long)b[0] * b[1];
        if (P < B) continue;
        if (mode != 2 && (B > min_len || P > 2 * (2 * w_lo + 3))) return;
        *W = b[0];
        *G = b[1];
        return;
    }
}

// Shortest series of a set (host mirror of the lengths); 0 for an empty set.
int set_min_len(const eap_series_set* s) {
    if (!s || s->count <= 0 || !s->h_lengths) return 0;
    int m = s->h_lengths[0];
    for (int i = 1; i < s->count; ++i) m = std::min(m, (int)s->h_lengths[i]);
    return m;
}

// Strip width and lanes per pair together: W = 5 exists only for 16-lane
// groups, so where those do not apply it becomes 4.
void choose_w_group(int kind, int cost, int max_rows, int max_cols, int prune, int* W, int* G) {
    *W = choose_w(kind, cost, max_cols, prune);
    *G = choose_group(kind, cost, max_rows, max_cols, prune, *W);
    if (*W == 5 && *G != 16) {
        *W = 4;
        *G = choose_group(kind, cost, max_rows, max_cols, prune, *W);
    }
}

// The kernel mapping of a 1-NN search (c.kp must be set): CTA per pair,
// groups of 8 or 16 lanes, a warp per pair, or band coordinates for the
// windowed distances, with their strip widths.  eap_nn1, the batched
// per-task launch and eap_nn1_plan all take it from here.
void nn1_mapping(int kind, int cost, int prune, bool own_cut, int n_queries, int max_rows, int max_cols,
                 int min_len, eaph::LaunchCtx& c) {
    c.cta = own_cut ? 0 : choose_cta(kind, cost, max_rows, max_cols, prune, n_queries);
    choose_w_group(kind, cost, max_rows, max_cols, prune, &c.W, &c.group);
    if (c.cta) { c.W = choose_w_cta(kind, cost, max_cols, prune); c.group = 0; }
    choose_band(kind, prune, c.kp, min_len, std::max(max_rows, max_cols), &c.band, &c.band_g, &c.band_exact);
}

// DP launch bracketed by CUDA events on the call's stream when timing is asked.
struct DpTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool on = false;
    explicit DpTimer(bool enable) {
        if (enable && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) on = true;
    }
    void start(cudaStream_t s) { if (on) cudaEventRecord(a, s); }
    void stop(cudaStream_t s) { if (on) cudaEventRecord(b, s); }
    double ms() {   // after the stream has been synchronised
        float t = 0.f;
        if (on && cudaEventElapsedTime(&t, a, b) == cudaSuccess) return (double)t;
        return 0.0;
    }
    ~DpTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int dispatch(const eaph::LaunchCtx& c, bool ub_only) {
    switch (c.kind) {
        case EAP_DTW: return eaph::launch_dp_dtw(c, ub_only);
        case EAP_CDTW: return eaph::launch_dp_cdtw(c, ub_only);
        case EAP_WDTW: return eaph::launch_dp_wdtw(c, ub_only);
        case EAP_ERP: return eaph::launch_dp_erp(c, ub_only);
        case EAP_MSM: return eaph::launch_dp_msm(c, ub_only);
        case EAP_TWE: return eaph::launch_dp_twe(c, ub_only);
    }
    return (int)cudaErrorInvalidValue;
}

// One stream-ordered scratch block carved into aligned pieces.
struct Scratch {
    char* base = nullptr;
    size_t size = 0, used = 0;
    cudaStream_t st = nullptr;
    int err = 0;
    void* take(size_t bytes) {
        const size_t a = (used + 255) & ~(size_t)255;
        used = a + bytes;
        return base ? base + a : nullptr;
    }
    int alloc(cudaStream_t s) {
        st = s;
        size = used;
        used = 0;
        if (size == 0) return EAP_OK;
        if (cudaMallocAsync((void**)&base, size, s) != cudaSuccess) { cudaGetLastError(); base = nullptr; return EAP_ENOMEM; }
        return EAP_OK;
    }
    void release() {
        if (base) cudaFreeAsync(base, st);
        base = nullptr;
    }
};

SeriesDev dev_set(const eap_series_set* s, const float* border) {
    return SeriesDev{s->data, s->offsets, s->lengths, border, s->count};
}

unsigned long long sum_cells(const eap_series_set* a, const eap_series_set* b) {
    unsigned long long sa = 0, sb = 0;
    for (int i = 0; i < a->count; ++i) sa += (unsigned long long)a->h_lengths[i];
    for (int i = 0; i < b->count; ++i) sb += (unsigned long long)b->h_lengths[i];
    return sa * sb;
}

int cuda_status(int e) { return e == 0 ? EAP_OK : EAP_EDEVICE; }

void launch_derivative_set(const eap_series_set* s, float* out, int sms, cudaStream_t st) {
    if (s->count <= 0) return;
    const int blocks = std::min(s->count, std::max(1, sms) * 8);
    derivative_kernel<<<blocks, 128, 0, st>>>(s->data, s->offsets, s->lengths, s->count, out);
}

// The derivative variants (p->derivative = 1) run `body` unchanged on copies
// of the sets whose data are the first-derivative series (derivative_kernel),
// with p->derivative cleared; the copies live in one stream-ordered block
// freed after the body.  b may be null (single-set calls) or equal to a.
template <class Body>
int with_derivative(const eap_params* p, const eap_series_set* a, const eap_series_set* b, cudaStream_t st,
                    Body&& body) {
    if (!p || p->derivative == 0) return body(p, a, b);
    int rc = validate_params(p);
    if (rc) return rc;
    int ma = 0, mb = 0;
    if ((rc = validate_set(a, &ma)) || (b && b != a && (rc = validate_set(b, &mb)))) return rc;
    eap_params q = *p;
    q.derivative = 0;
    const bool own_b = b && b != a;
    const size_t na = a->count > 0 ? (size_t)a->data_len : 0;
    const size_t nb = own_b && b->count > 0 ? (size_t)b->data_len : 0;
    const size_t ob = (na + 63) & ~(size_t)63;
    float* buf = nullptr;
    if (na + nb > 0 && cudaMallocAsync((void**)&buf, sizeof(float) * (ob + nb), st) != cudaSuccess) {
        cudaGetLastError();
        return EAP_ENOMEM;
    }
    const int sms = device_sms();
    eap_series_set da = *a, db = own_b ? *b : *a;
    if (na) { da.data = buf; launch_derivative_set(a, buf, sms, st); }
    if (nb) { db.data = buf + ob; launch_derivative_set(b, buf + ob, sms, st); }
    if (cudaGetLastError() != cudaSuccess) {
        if (buf) cudaFreeAsync(buf, st);
        return EAP_EDEVICE;
    }
    rc = body(&q, &da, b ? (own_b ? &db : &da) : nullptr);
    if (buf) cudaFreeAsync(buf, st);
    return rc;
}

// Shared body of 1-NN for device-resident sets.
// keys_out (with key_offset) replaces out_idx / out_dist by packed keys.
int nn1_core(const eap_params* p, const eap_series_set* qs, const eap_series_set* rs, int32_t* out_idx,
             float* out_dist, cudaStream_t st, eap_stats* stats, unsigned long long* dev_stats_keep,
             unsigned long long* keys_out = nullptr, long long key_offset = 0) {
    int rc = validate_params(p);
    if (rc) return rc;
    int mq = 0, mr = 0;
    if ((rc = validate_set(qs, &mq)) || (rc = validate_set(rs, &mr))) return rc;
    if (qs->count > 0 && !keys_out && (!out_idx || !out_dist)) return EAP_EINVAL;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    const int nq = qs->count, nr = rs->count;
    if (nq == 0) return EAP_OK;
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    if (nr == 0) {
        if (keys_out) {   // every key says "none": +inf bits, no index
            keys_kernel<<<(nq + 255) / 256, 256, 0, st>>>(nullptr, nq, 0, keys_out, nullptr);
            return cuda_status((int)cudaGetLastError());
        }
        fill_nn_empty_kernel<<<(nq + 255) / 256, 256, 0, st>>>(out_idx, out_dist, nq);
        return cuda_status((int)cudaGetLastError());
    }
    const bool prune = p->prune != 0;
    const bool erp = p->kind == EAP_ERP, wdtw = p->kind == EAP_WDTW;
    const int cost = resolve_cost(p);
    const unsigned long long items = (unsigned long long)nq * nr;
    // Alg. 2's lower bound (LB_Keogh) ahead of the DP: DTW / CDTW, pruned runs.
    const bool use_lb = prune && p->lb != EAP_LB_NONE && (p->kind == EAP_DTW || p->kind == EAP_CDTW);
    const bool use_lb2 = use_lb && p->lb == EAP_LB_KEOGH2;

    Scratch sc;
    auto layout = [&]() {
        struct { unsigned long long *best, *ctr, *stats; float* ub; int32_t* order; float *bq, *br, *wt, *lb, *qU, *qL, *rU, *rL; float4* rp; } L;
        L.best = (unsigned long long*)sc.take(sizeof(unsigned long long) * nq);
        L.ctr = (unsigned long long*)sc.take(sizeof(unsigned long long));
        L.stats = (unsigned long long*)sc.take(sizeof(unsigned long long) * kStatCount);
        L.ub = prune ? (float*)sc.take(sizeof(float) * items) : nullptr;
        L.order = prune ? (int32_t*)sc.take(sizeof(int32_t) * items) : nullptr;
        L.bq = erp ? (float*)sc.take(sizeof(float) * (size_t)qs->data_len) : nullptr;
        L.br = erp ? (float*)sc.take(sizeof(float) * (size_t)rs->data_len) : nullptr;
        L.wt = wdtw ? (float*)sc.take(sizeof(float) * (2 * kWdtwOff + 1)) : nullptr;
        L.lb = use_lb ? (float*)sc.take(sizeof(float) * items) : nullptr;
        L.qU = use_lb ? (float*)sc.take(sizeof(float) * (size_t)qs->data_len) : nullptr;
        L.qL = use_lb ? (float*)sc.take(sizeof(float) * (size_t)qs->data_len) : nullptr;
        L.rU = use_lb2 ? (float*)sc.take(sizeof(float) * (size_t)rs->data_len) : nullptr;
        L.rL = use_lb2 ? (float*)sc.take(sizeof(float) * (size_t)rs->data_len) : nullptr;
        L.rp = eaph::kind_packed(p->kind) ? (float4*)sc.take(sizeof(float4) * ((size_t)qs->data_len + 1)) : nullptr;
        return L;
    };
    layout();
    if ((rc = sc.alloc(st))) return rc;
    const auto L = layout();
    unsigned long long* d_best = L.best;
    unsigned long long* d_ctr = L.ctr;
    unsigned long long* d_stats = L.stats;
    float* d_ub = L.ub;
    int32_t* d_order = L.order;
    float* d_bq = L.bq;
    float* d_br = L.br;
    float* d_wt = L.wt;

    int e = 0;
    e |= (int)cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long), st);
    e |= (int)cudaMemsetAsync(d_stats, 0, sizeof(unsigned long long) * kStatCount, st);
    init_best_kernel<<<(nq + 255) / 256, 256, 0, st>>>(d_best, nq);
    if (erp) {
        erp_border_kernel<<<(nq + 127) / 128, 128, 0, st>>>(qs->data, qs->offsets, qs->lengths, nq, p->erp_gap, cost, d_bq);
        erp_border_kernel<<<(nr + 127) / 128, 128, 0, st>>>(rs->data, rs->offsets, rs->lengths, nr, p->erp_gap, cost, d_br);
    }
    if (wdtw) wdtw_table_kernel<<<(2 * kWdtwOff + 256) / 256, 256, 0, st>>>(d_wt, (double)p->wdtw_g, (double)p->wdtw_wmax);
    e |= (int)cudaGetLastError();
    if (e) { sc.release(); return EAP_EDEVICE; }

    eaph::LaunchCtx c;
    std::memset(&c, 0, sizeof(c));
    c.job.mode = kModeNN1;
    c.job.A = dev_set(qs, d_bq);
    c.job.B = dev_set(rs, d_br);
    c.job.nitems = items;
    c.job.counter = d_ctr;
    c.job.order = d_order;
    c.job.best = d_best;
    c.job.stats = d_stats;
    c.job.wdtw_table = d_wt;
    c.job.bnd_stride = ((mq + 1) + 31) & ~31;
    c.kp = make_kparams(p);
    c.kp.wdtw_w = d_wt;
    c.rowpack = L.rp;
    c.kind = p->kind;
    c.cost = cost;
    // Prune (3) runs the EAPruned kernel with each pair's own diagonal bound as cut-off.
    const bool own_cut = p->prune == 3;
    c.prune = own_cut ? kPmPruned : p->prune;
    c.job.cut = own_cut ? d_ub : nullptr;
    c.sms = sms;
    c.max_rows = mq;
    c.max_cols = mr;
    nn1_mapping(p->kind, cost, c.prune, own_cut, nq, mq, mr, std::min(set_min_len(qs), set_min_len(rs)), c);
    c.stream = st;
    c.ub = d_ub;
    if (prune) {
        if ((e = dispatch(c, true))) { sc.release(); return cuda_status(e); }
        int chunk = 1;
        while (chunk < nr && chunk < 4096) chunk <<= 1;
        sort_seed_kernel<<<nq, 512, sizeof(unsigned long long) * chunk, st>>>(d_ub, nr, chunk, d_order, d_best);
        if ((e = (int)cudaGetLastError())) { sc.release(); return cuda_status(e); }
    }
    DpTimer tm(stats != nullptr), tlb(stats != nullptr && use_lb);
    if (use_lb) {
        tlb.start(st);
        KParams ke = make_kparams(p);
        ke.windowed = 1;
        if (p->kind == EAP_DTW) { ke.window_abs = -1; ke.window_ratio = -1.f; }   // DTW: the whole series
        launch_envelope(dev_set(qs, nullptr), ke, mq, L.qU, L.qL, st);
        if (use_lb2) launch_envelope(dev_set(rs, nullptr), ke, mr, L.rU, L.rL, st);
        launch_lb_matrix(dev_set(qs, nullptr), dev_set(rs, nullptr), L.qU, L.qL, L.rU, L.rL, cost, use_lb2 ? 1 : 0,
                         L.lb, st);
        if ((e = (int)cudaGetLastError())) { sc.release(); return cuda_status(e); }
        tlb.stop(st);
        c.job.lb = L.lb;
    }
    tm.start(st);
    if ((e = dispatch(c, false))) { sc.release(); return cuda_status(e); }
    tm.stop(st);
    if (keys_out) keys_kernel<<<(nq + 255) / 256, 256, 0, st>>>(d_best, nq, key_offset, keys_out, d_stats);
    else unpack_kernel<<<(nq + 255) / 256, 256, 0, st>>>(d_best, nq, out_idx, out_dist, d_stats);
    if ((e = (int)cudaGetLastError())) { sc.release(); return cuda_status(e); }
    unsigned long long h[kStatCount];
    if (stats || dev_stats_keep) {
        if (cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) { sc.release(); return EAP_EDEVICE; }
    }
    sc.release();
    if (stats || dev_stats_keep) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return EAP_EDEVICE;
        if (stats) {
            stats->pairs = h[kStatPairs] + h[kStatLbPruned];
            stats->pairs_lb_pruned = h[kStatLbPruned];
            stats->pairs_abandoned = h[kStatAbandoned];
            stats->cells_computed = h[kStatCells];
            stats->cells_effective = sum_cells(qs, rs);
            stats->dp_ms = tm.ms();
            stats->lb_ms = tlb.ms();
        }
        if (dev_stats_keep) std::memcpy(dev_stats_keep, h, sizeof(h));
        if (h[kStatErrors]) return EAP_EINTERNAL;
    }
    return EAP_OK;
}

int nn1_impl(const eap_params* p, const eap_series_set* qs, const eap_series_set* rs, int32_t* out_idx,
             float* out_dist, cudaStream_t st, eap_stats* stats, unsigned long long* dev_stats_keep,
             unsigned long long* keys_out = nullptr, long long key_offset = 0) {
    return with_derivative(p, qs, rs, st, [&](const eap_params* q, const eap_series_set* a, const eap_series_set* b) {
        return nn1_core(q, a, b, out_idx, out_dist, st, stats, dev_stats_keep, keys_out, key_offset);
    });
}

int pairwise_core(const eap_params* p, const eap_series_set* set, float* out_matrix, int32_t mode, cudaStream_t st,
                  eap_stats* opt_stats);
int pairs_core(const eap_params* p, const eap_series_set* a, const eap_series_set* b, const int32_t* ia,
               const int32_t* ib, const float* cutoff, float* out, int32_t n, cudaStream_t st, eap_stats* opt_stats);
int lb_keogh_core(const eap_params* p, const eap_series_set* a, const eap_series_set* b, const int32_t* ia,
                  const int32_t* ib, float* out, int32_t n, cudaStream_t st);

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void eap_params_default(eap_params* p, int32_t kind) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->kind = kind;
    p->cost = EAP_COST_DEFAULT;
    p->window_ratio = (kind == EAP_CDTW || kind == EAP_ERP) ? 0.1f : -1.0f;
    p->window = -1;
    p->wdtw_g = 0.05f;
    p->wdtw_wmax = 1.0f;
    p->erp_gap = 0.0f;
    p->msm_c = 0.5f;
    p->twe_nu = 0.001f;
    p->twe_lambda = 1.0f;
    p->lb = EAP_LB_NONE;
    p->prune = 1;
}

const char* eap_strerror(int code) {
    switch (code) {
        case EAP_OK: return "ok";
        case EAP_EINVAL: return "invalid argument";
        case EAP_ENOMEM: return "out of memory";
        case EAP_EAGAIN: return "try again (not admitted / not ready)";
        case EAP_ETIMEOUT: return "timed out";
        case EAP_EDEVICE: return "CUDA device error";
        case EAP_EINTERNAL: return "internal consistency check failed";
    }
    return "unknown error";
}

int32_t eap_version(void) { return 1; }

int eap_nn1(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs, int32_t* out_idx,
            float* out_dist, void* cuda_stream, eap_stats* opt_stats) {
    return nn1_impl(p, queries, refs, out_idx, out_dist, (cudaStream_t)cuda_stream, opt_stats, nullptr);
}

int eap_nn1_plan(const eap_params* p, int32_t n_queries, int32_t min_len, int32_t max_query_len,
                 int32_t max_ref_len, eap_plan* out) {
    if (!out || validate_params(p) != EAP_OK || n_queries < 0) return EAP_EINVAL;
    if (min_len < 1 || max_query_len < min_len || max_ref_len < min_len || max_query_len > kMaxSeriesLen ||
        max_ref_len > kMaxSeriesLen)
        return EAP_EINVAL;
    eaph::LaunchCtx c{};
    c.kp = make_kparams(p);
    const bool own_cut = p->prune == 3;
    const int prune = own_cut ? kPmPruned : p->prune;
    nn1_mapping(p->kind, resolve_cost(p), prune, own_cut, n_queries, max_query_len, max_ref_len, min_len, c);
    // The order run_kind follows: band (windowed) or CTA (unwindowed) first,
    // then groups (EAPruned and Base), then a warp per pair.
    const bool windowed = p->kind == EAP_CDTW || p->kind == EAP_ERP;
    eap_plan r{};
    if (windowed && c.band) {
        r.mapping = EAP_PLAN_BAND;
        r.strip_width = c.band;
        r.lanes_per_pair = c.band_g;
        r.band_exact = c.band_exact;
    } else if (!windowed && c.cta) {
        r.mapping = EAP_PLAN_CTA;
        r.strip_width = c.W >= 8 ? 8 : 4;
        r.lanes_per_pair = eapd::kCtaThreads;
    } else if (c.group && (prune == kPmPruned || prune == kPmBase)) {
        r.mapping = EAP_PLAN_GROUP;
        r.strip_width = c.W;
        r.lanes_per_pair = c.group;
    } else {
        r.mapping = EAP_PLAN_WARP;
        r.strip_width = c.W;
        r.lanes_per_pair = 32;
    }
    *out = r;
    return EAP_OK;
}

int eap_nn1_keys(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs,
                 int64_t index_offset, uint64_t* out_keys, void* cuda_stream, eap_stats* opt_stats) {
    if (!queries || !refs) return EAP_EINVAL;
    if (queries->count > 0 && !out_keys) return EAP_EINVAL;
    if (index_offset < 0 || index_offset + (int64_t)refs->count >= (int64_t)kNoIndex) return EAP_EINVAL;
    return nn1_impl(p, queries, refs, nullptr, nullptr, (cudaStream_t)cuda_stream, opt_stats, nullptr,
                    (unsigned long long*)out_keys, (long long)index_offset);
}

int eap_lb_matrix(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs, int32_t two_way,
                  float* out_lb, void* cuda_stream) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (two_way != 0 && two_way != 1) return EAP_EINVAL;
    return with_derivative(p, queries, refs, st, [&](const eap_params* q, const eap_series_set* qs,
                                                     const eap_series_set* rs) {
        int rc = validate_params(q);
        if (rc) return rc;
        int mq = 0, mr = 0;
        if ((rc = validate_set(qs, &mq)) || (rc = validate_set(rs, &mr))) return rc;
        if (q->kind != EAP_DTW && q->kind != EAP_CDTW) return EAP_EINVAL;
        if (qs->count == 0 || rs->count == 0) return EAP_OK;
        if (!out_lb) return EAP_EINVAL;
        Scratch sc;
        auto layout = [&]() {
            struct { float *qU, *qL, *rU, *rL; } L;
            L.qU = (float*)sc.take(sizeof(float) * (size_t)qs->data_len);
            L.qL = (float*)sc.take(sizeof(float) * (size_t)qs->data_len);
            L.rU = two_way ? (float*)sc.take(sizeof(float) * (size_t)rs->data_len) : nullptr;
            L.rL = two_way ? (float*)sc.take(sizeof(float) * (size_t)rs->data_len) : nullptr;
            return L;
        };
        layout();
        if ((rc = sc.alloc(st))) return rc;
        const auto L = layout();
        KParams ke = make_kparams(q);
        ke.windowed = 1;
        if (q->kind == EAP_DTW) { ke.window_abs = -1; ke.window_ratio = -1.f; }   // DTW: the whole series
        launch_envelope(dev_set(qs, nullptr), ke, mq, L.qU, L.qL, st);
        if (two_way) launch_envelope(dev_set(rs, nullptr), ke, mr, L.rU, L.rL, st);
        launch_lb_matrix(dev_set(qs, nullptr), dev_set(rs, nullptr), L.qU, L.qL, L.rU, L.rL, resolve_cost(q),
                         two_way, out_lb, st);
        const int e = (int)cudaGetLastError();
        sc.release();
        return cuda_status(e);
    });
}

int eap_keys_unpack(const uint64_t* keys, int32_t n, int32_t* out_idx, float* out_dist, void* cuda_stream) {
    if (n < 0) return EAP_EINVAL;
    if (n == 0) return EAP_OK;
    if (!keys || !out_idx || !out_dist) return EAP_EINVAL;
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    const int blocks = std::min((n + 255) / 256, sms * 8);
    keys_unpack_kernel<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>((const unsigned long long*)keys, n, out_idx,
                                                                        out_dist);
    return cuda_status((int)cudaGetLastError());
}

int eap_nn1_host(const eap_params* p, const float* q_data, const int64_t* q_offsets, const int32_t* q_lengths,
                 int32_t nq, const float* r_data, const int64_t* r_offsets, const int32_t* r_lengths, int32_t nr,
                 int32_t* out_idx, float* out_dist, eap_stats* opt_stats) {
    if (nq < 0 || nr < 0) return EAP_EINVAL;
    if (nq > 0 && (!q_data || !q_offsets || !q_lengths || !out_idx || !out_dist)) return EAP_EINVAL;
    if (nr > 0 && (!r_data || !r_offsets || !r_lengths)) return EAP_EINVAL;
    int64_t qlen = 0, rlen = 0;
    for (int i = 0; i < nq; ++i) qlen = std::max<int64_t>(qlen, q_offsets[i] + std::max(0, q_lengths[i]));
    for (int i = 0; i < nr; ++i) rlen = std::max<int64_t>(rlen, r_offsets[i] + std::max(0, r_lengths[i]));
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return EAP_EDEVICE;
    const size_t bytes = sizeof(float) * (size_t)(qlen + rlen) + (sizeof(int64_t) + sizeof(int32_t)) * (size_t)(nq + nr)
                         + (sizeof(int32_t) + sizeof(float)) * (size_t)nq + 6 * 256;
    char* d = nullptr;
    if (cudaMallocAsync((void**)&d, bytes, st) != cudaSuccess) { cudaGetLastError(); cudaStreamDestroy(st); return EAP_ENOMEM; }
    size_t used = 0;
    auto take = [&](size_t b) { const size_t a = (used + 255) & ~(size_t)255; used = a + b; return d + a; };
    float* dq = (float*)take(sizeof(float) * qlen);
    float* dr = (float*)take(sizeof(float) * rlen);
    int64_t* dqo = (int64_t*)take(sizeof(int64_t) * nq);
    int32_t* dql = (int32_t*)take(sizeof(int32_t) * nq);
    int64_t* dro = (int64_t*)take(sizeof(int64_t) * nr);
    int32_t* drl = (int32_t*)take(sizeof(int32_t) * nr);
    int32_t* didx = (int32_t*)take(sizeof(int32_t) * nq);
    float* ddist = (float*)take(sizeof(float) * nq);
    int e = 0;
    if (qlen) e |= (int)cudaMemcpyAsync(dq, q_data, sizeof(float) * qlen, cudaMemcpyHostToDevice, st);
    if (rlen) e |= (int)cudaMemcpyAsync(dr, r_data, sizeof(float) * rlen, cudaMemcpyHostToDevice, st);
    if (nq) {
        e |= (int)cudaMemcpyAsync(dqo, q_offsets, sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st);
        e |= (int)cudaMemcpyAsync(dql, q_lengths, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st);
    }
    if (nr) {
        e |= (int)cudaMemcpyAsync(dro, r_offsets, sizeof(int64_t) * nr, cudaMemcpyHostToDevice, st);
        e |= (int)cudaMemcpyAsync(drl, r_lengths, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, st);
    }
    int rc = e ? EAP_EDEVICE : EAP_OK;
    if (rc == EAP_OK) {
        eap_series_set qs{dq, dqo, dql, q_offsets, q_lengths, qlen, nq, 0};
        eap_series_set rs{dr, dro, drl, r_offsets, r_lengths, rlen, nr, 0};
        rc = nn1_impl(p, &qs, &rs, didx, ddist, st, opt_stats, nullptr);
    }
    if (rc == EAP_OK && nq) {
        e = (int)cudaMemcpyAsync(out_idx, didx, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, st);
        e |= (int)cudaMemcpyAsync(out_dist, ddist, sizeof(float) * nq, cudaMemcpyDeviceToHost, st);
        if (e) rc = EAP_EDEVICE;
    }
    cudaFreeAsync(d, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == EAP_OK) rc = EAP_EDEVICE;
    cudaStreamDestroy(st);
    return rc;
}

int eap_pairwise(const eap_params* p, const eap_series_set* set, float* out_matrix, int32_t mode, void* cuda_stream,
                 eap_stats* opt_stats) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    return with_derivative(p, set, nullptr, st, [&](const eap_params* q, const eap_series_set* a, const eap_series_set*) {
        return pairwise_core(q, a, out_matrix, mode, st, opt_stats);
    });
}

int eap_pairs(const eap_params* p, const eap_series_set* a, const eap_series_set* b, const int32_t* ia,
              const int32_t* ib, const float* cutoff, float* out, int32_t n, void* cuda_stream, eap_stats* opt_stats) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n <= 0) return pairs_core(p, a, b, ia, ib, cutoff, out, n, st, opt_stats);   // validation only, nothing to derive
    return with_derivative(p, a, b, st, [&](const eap_params* q, const eap_series_set* x, const eap_series_set* y) {
        return pairs_core(q, x, y, ia, ib, cutoff, out, n, st, opt_stats);
    });
}

int eap_lb_keogh(const eap_params* p, const eap_series_set* a, const eap_series_set* b, const int32_t* ia,
                 const int32_t* ib, float* out, int32_t n, void* cuda_stream) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n <= 0) return lb_keogh_core(p, a, b, ia, ib, out, n, st);
    return with_derivative(p, a, b, st, [&](const eap_params* q, const eap_series_set* x, const eap_series_set* y) {
        return lb_keogh_core(q, x, y, ia, ib, out, n, st);
    });
}

}  // extern "C"

namespace {

int pairwise_core(const eap_params* p, const eap_series_set* set, float* out_matrix, int32_t mode, cudaStream_t st,
                  eap_stats* opt_stats) {
    int rc = validate_params(p);
    if (rc) return rc;
    int mx = 0;
    if ((rc = validate_set(set, &mx))) return rc;
    if (mode != EAP_PRUNE_ONLY && mode != EAP_BASE) return EAP_EINVAL;
    if (set->count > 0 && !out_matrix) return EAP_EINVAL;
    if (opt_stats) std::memset(opt_stats, 0, sizeof(*opt_stats));
    const int n = set->count;
    if (n == 0) return EAP_OK;
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    const bool prune = mode == EAP_PRUNE_ONLY;
    const bool erp = p->kind == EAP_ERP, wdtw = p->kind == EAP_WDTW;
    const int cost = resolve_cost(p);
    const unsigned long long items = (unsigned long long)n * (n - 1) / 2;

    Scratch sc;
    auto layout = [&]() {
        struct { unsigned long long *ctr, *stats; float *ub, *bs, *wt; float4* rp; } L;
        L.ctr = (unsigned long long*)sc.take(sizeof(unsigned long long));
        L.stats = (unsigned long long*)sc.take(sizeof(unsigned long long) * kStatCount);
        L.ub = prune ? (float*)sc.take(sizeof(float) * (items ? items : 1)) : nullptr;
        L.bs = erp ? (float*)sc.take(sizeof(float) * (size_t)set->data_len) : nullptr;
        L.wt = wdtw ? (float*)sc.take(sizeof(float) * (2 * kWdtwOff + 1)) : nullptr;
        L.rp = eaph::kind_packed(p->kind) ? (float4*)sc.take(sizeof(float4) * ((size_t)set->data_len + 1)) : nullptr;
        return L;
    };
    layout();
    if ((rc = sc.alloc(st))) return rc;
    auto L = layout();
    int e = 0;
    e |= (int)cudaMemsetAsync(L.ctr, 0, sizeof(unsigned long long), st);
    e |= (int)cudaMemsetAsync(L.stats, 0, sizeof(unsigned long long) * kStatCount, st);
    diag_zero_kernel<<<(n + 255) / 256, 256, 0, st>>>(out_matrix, n);
    if (erp) erp_border_kernel<<<(n + 127) / 128, 128, 0, st>>>(set->data, set->offsets, set->lengths, n, p->erp_gap, cost, L.bs);
    if (wdtw) wdtw_table_kernel<<<(2 * kWdtwOff + 256) / 256, 256, 0, st>>>(L.wt, (double)p->wdtw_g, (double)p->wdtw_wmax);
    e |= (int)cudaGetLastError();
    if (e) { sc.release(); return EAP_EDEVICE; }
    DpTimer tm(opt_stats != nullptr);
    if (items > 0) {
        eaph::LaunchCtx c;
        std::memset(&c, 0, sizeof(c));
        c.job.mode = kModePairwise;
        c.job.A = dev_set(set, L.bs);
        c.job.B = dev_set(set, L.bs);
        c.job.nitems = items;
        c.job.counter = L.ctr;
        c.job.cut = L.ub;
        c.job.out = out_matrix;
        c.job.stats = L.stats;
        c.job.wdtw_table = L.wt;
        c.job.bnd_stride = ((mx + 1) + 31) & ~31;
        c.kp = make_kparams(p);
        c.kp.wdtw_w = L.wt;
        c.rowpack = L.rp;
        c.kind = p->kind;
        c.cost = cost;
        c.prune = prune ? 1 : 0;
        // Prune-only keeps the Base strip width: a diagonal-path cut-off
        // prunes far less than a 1-NN best-so-far, so per-cell speed matters more.
        c.W = choose_w(p->kind, cost, mx, 0);
        c.sms = sms;
        c.max_rows = mx;
        c.max_cols = mx;
        c.cta = choose_cta(p->kind, cost, mx, mx, c.prune);
        c.group = c.cta ? 0 : choose_group(p->kind, cost, mx, mx, c.prune, c.W);
        if (c.cta) c.W = choose_w_cta(p->kind, cost, mx, 0);
        choose_band(p->kind, c.prune, c.kp, set_min_len(set), mx, &c.band, &c.band_g, &c.band_exact);
        c.stream = st;
        c.ub = L.ub;
        if (prune && (e = dispatch(c, true))) { sc.release(); return cuda_status(e); }
        tm.start(st);
        if ((e = dispatch(c, false))) { sc.release(); return cuda_status(e); }
        tm.stop(st);
    }
    unsigned long long h[kStatCount];
    if (opt_stats && cudaMemcpyAsync(h, L.stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        sc.release();
        return EAP_EDEVICE;
    }
    sc.release();
    if (opt_stats) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return EAP_EDEVICE;
        opt_stats->pairs = h[kStatPairs];
        opt_stats->pairs_abandoned = h[kStatAbandoned];
        opt_stats->cells_computed = h[kStatCells];
        unsigned long long eff = 0, tot = 0, sq = 0;
        for (int i = 0; i < n; ++i) { tot += (unsigned long long)set->h_lengths[i]; sq += (unsigned long long)set->h_lengths[i] * set->h_lengths[i]; }
        eff = (tot * tot - sq) / 2;
        opt_stats->cells_effective = eff;
        opt_stats->dp_ms = tm.ms();
    }
    return EAP_OK;
}

int pairs_core(const eap_params* p, const eap_series_set* a, const eap_series_set* b, const int32_t* ia,
               const int32_t* ib, const float* cutoff, float* out, int32_t n, cudaStream_t st, eap_stats* opt_stats) {
    int rc = validate_params(p);
    if (rc) return rc;
    int ma = 0, mb = 0;
    if ((rc = validate_set(a, &ma)) || (rc = validate_set(b, &mb))) return rc;
    if (n < 0) return EAP_EINVAL;
    if (opt_stats) std::memset(opt_stats, 0, sizeof(*opt_stats));
    if (n == 0) return EAP_OK;
    if (!ia || !ib || !out || (p->prune && !cutoff) || a->count == 0 || b->count == 0) return EAP_EINVAL;
    if (p->prune == 3) return EAP_EINVAL;   // pruning-only with own bounds: eap_pairwise(EAP_PRUNE_ONLY) / eap_nn1
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    const bool erp = p->kind == EAP_ERP, wdtw = p->kind == EAP_WDTW;
    const int cost = resolve_cost(p);
    Scratch sc;
    auto layout = [&]() {
        struct { unsigned long long *ctr, *stats; float *ba, *bb, *wt; float4* rp; } L;
        L.ctr = (unsigned long long*)sc.take(sizeof(unsigned long long));
        L.stats = (unsigned long long*)sc.take(sizeof(unsigned long long) * kStatCount);
        L.ba = erp ? (float*)sc.take(sizeof(float) * (size_t)a->data_len) : nullptr;
        L.bb = erp ? (float*)sc.take(sizeof(float) * (size_t)b->data_len) : nullptr;
        L.wt = wdtw ? (float*)sc.take(sizeof(float) * (2 * kWdtwOff + 1)) : nullptr;
        L.rp = eaph::kind_packed(p->kind) ? (float4*)sc.take(sizeof(float4) * ((size_t)a->data_len + 1)) : nullptr;
        return L;
    };
    layout();
    if ((rc = sc.alloc(st))) return rc;
    auto L = layout();
    int e = 0;
    e |= (int)cudaMemsetAsync(L.ctr, 0, sizeof(unsigned long long), st);
    e |= (int)cudaMemsetAsync(L.stats, 0, sizeof(unsigned long long) * kStatCount, st);
    if (erp) {
        erp_border_kernel<<<(a->count + 127) / 128, 128, 0, st>>>(a->data, a->offsets, a->lengths, a->count, p->erp_gap, cost, L.ba);
        erp_border_kernel<<<(b->count + 127) / 128, 128, 0, st>>>(b->data, b->offsets, b->lengths, b->count, p->erp_gap, cost, L.bb);
    }
    if (wdtw) wdtw_table_kernel<<<(2 * kWdtwOff + 256) / 256, 256, 0, st>>>(L.wt, (double)p->wdtw_g, (double)p->wdtw_wmax);
    e |= (int)cudaGetLastError();
    if (e) { sc.release(); return EAP_EDEVICE; }
    eaph::LaunchCtx c;
    std::memset(&c, 0, sizeof(c));
    c.job.mode = kModePairs;
    c.job.A = dev_set(a, L.ba);
    c.job.B = dev_set(b, L.bb);
    c.job.nitems = (unsigned long long)n;
    c.job.counter = L.ctr;
    c.job.cut = p->prune ? cutoff : nullptr;
    c.job.out = out;
    c.job.ia = ia;
    c.job.ib = ib;
    c.job.stats = L.stats;
    c.job.wdtw_table = L.wt;
    c.job.bnd_stride = ((ma + 1) + 31) & ~31;
    c.kp = make_kparams(p);
    c.kp.wdtw_w = L.wt;
    c.rowpack = L.rp;
    c.kind = p->kind;
    c.cost = cost;
    c.prune = p->prune;
    c.sms = sms;
    c.max_rows = ma;
    c.max_cols = mb;
    c.cta = choose_cta(p->kind, cost, ma, mb, c.prune);
    choose_w_group(p->kind, cost, ma, mb, c.prune, &c.W, &c.group);
    if (c.cta) { c.W = choose_w_cta(p->kind, cost, mb, c.prune); c.group = 0; }
    choose_band(p->kind, c.prune, c.kp, std::min(set_min_len(a), set_min_len(b)), std::max(ma, mb), &c.band, &c.band_g, &c.band_exact);
    c.stream = st;
    DpTimer tm(opt_stats != nullptr);
    tm.start(st);
    if ((e = dispatch(c, false))) { sc.release(); return cuda_status(e); }
    tm.stop(st);
    unsigned long long h[kStatCount];
    if (opt_stats && cudaMemcpyAsync(h, L.stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        sc.release();
        return EAP_EDEVICE;
    }
    sc.release();
    if (opt_stats) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return EAP_EDEVICE;
        opt_stats->pairs = h[kStatPairs];
        opt_stats->pairs_abandoned = h[kStatAbandoned];
        opt_stats->cells_computed = h[kStatCells];
        opt_stats->dp_ms = tm.ms();
    }
    return EAP_OK;
}

int lb_keogh_core(const eap_params* p, const eap_series_set* a, const eap_series_set* b, const int32_t* ia,
                  const int32_t* ib, float* out, int32_t n, cudaStream_t st) {
    int rc = validate_params(p);
    if (rc) return rc;
    int ma = 0, mb = 0;
    if ((rc = validate_set(a, &ma)) || (rc = validate_set(b, &mb))) return rc;
    if (n < 0) return EAP_EINVAL;
    if (n == 0) return EAP_OK;
    if (!ia || !ib || !out || a->count == 0 || b->count == 0) return EAP_EINVAL;
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    KParams kp = make_kparams(p);
    kp.windowed = 1;
    const int blocks = std::min((n + 7) / 8, sms * 8);
    lb_keogh_pairs_kernel<<<blocks, 256, 0, st>>>(dev_set(a, nullptr), dev_set(b, nullptr), ia, ib, n, kp,
                                                  resolve_cost(p), out);
    return cuda_status((int)cudaGetLastError());
}

}  // namespace

// ===========================================================================
// Allocation-free variant of eap_pairs.
//
// Some callers cannot allocate device memory while they call us: code that
// runs with a fixed, pre-committed memory budget (no cudaMalloc after
// start-up), code called from inside a framework that owns every allocation
// on the device, or code on a path where an allocation could block or fail
// at the wrong moment.  eap_pairs_noalloc gives them the raw EAPruned pairs
// call with every piece of scratch (the work-queue head, the work counters,
// ERP's border prefix sums and WDTW's weight table) taken from one fixed
// array in device memory that is part of this library, so the call itself
// allocates nothing.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;   // 4 MiB, held by every device that loads libeap
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};   // device address of g_noalloc_scratch, per device ordinal

// Once per device, with that device current: the host-side symbol is only a
// stand-in, so the kernels must be given the address the runtime reports.
int noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return EAP_EDEVICE;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return EAP_EDEVICE;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return EAP_OK;
}

}  // namespace

extern "C" int eap_pairs_noalloc(const eap_params* p, const eap_series_set* a, const eap_series_set* b,
                                 const int32_t* ia, const int32_t* ib, const float* cutoff, float* out, int32_t n,
                                 void* cuda_stream, eap_stats* opt_stats) {
    int rc = validate_params(p);
    if (rc) return rc;
    int ma = 0, mb = 0;
    if ((rc = validate_set(a, &ma)) || (rc = validate_set(b, &mb))) return rc;
    if (n < 0) return EAP_EINVAL;
    if (opt_stats) std::memset(opt_stats, 0, sizeof(*opt_stats));
    if (n == 0) return EAP_OK;
    if (!ia || !ib || !out || (p->prune && !cutoff) || a->count == 0 || b->count == 0) return EAP_EINVAL;
    if (p->prune == 3) return EAP_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    const bool erp = p->kind == EAP_ERP, wdtw = p->kind == EAP_WDTW;
    const int cost = resolve_cost(p);

    // Carve the fixed array; reject calls whose scratch would not fit.
    size_t used = 0;
    auto take = [&](size_t bytes) { const size_t o = (used + 255) & ~(size_t)255; used = o + bytes; return o; };
    const size_t o_ctr = take(sizeof(unsigned long long));
    const size_t o_stats = take(sizeof(unsigned long long) * kStatCount);
    const size_t o_ba = erp ? take(sizeof(float) * (size_t)a->data_len) : 0;
    const size_t o_bb = erp ? take(sizeof(float) * (size_t)b->data_len) : 0;
    const size_t o_wt = wdtw ? take(sizeof(float) * (2 * kWdtwOff + 1)) : 0;
    const bool deriv = p->derivative != 0;
    const size_t o_da = deriv ? take(sizeof(float) * (size_t)a->data_len) : 0;
    const size_t o_db = deriv ? take(sizeof(float) * (size_t)b->data_len) : 0;
    const bool packed = eaph::kind_packed(p->kind);
    const size_t o_rp = packed ? take(sizeof(float4) * ((size_t)a->data_len + 1)) : 0;
    if (used > kNoAllocScratchBytes) return EAP_EINVAL;
    void* base = nullptr;
    if ((rc = noalloc_scratch(&base))) return rc;
    char* s = (char*)base;
    unsigned long long* d_ctr = (unsigned long long*)(s + o_ctr);
    unsigned long long* d_stats = (unsigned long long*)(s + o_stats);
    float* d_ba = erp ? (float*)(s + o_ba) : nullptr;
    float* d_bb = erp ? (float*)(s + o_bb) : nullptr;
    float* d_wt = wdtw ? (float*)(s + o_wt) : nullptr;

    // The array keeps the previous call's contents: reset what must start at zero.
    int e = 0;
    e |= (int)cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long), st);
    e |= (int)cudaMemsetAsync(d_stats, 0, sizeof(unsigned long long) * kStatCount, st);
    // Derivative variants: the sets' first-derivative series, also from the fixed array.
    eap_series_set da = *a, db = *b;
    if (deriv) {
        da.data = (const float*)(s + o_da);
        db.data = (const float*)(s + o_db);
        launch_derivative_set(a, (float*)(s + o_da), sms, st);
        launch_derivative_set(b, (float*)(s + o_db), sms, st);
        a = &da;
        b = &db;
    }
    if (erp) {
        erp_border_kernel<<<(a->count + 127) / 128, 128, 0, st>>>(a->data, a->offsets, a->lengths, a->count, p->erp_gap, cost, d_ba);
        erp_border_kernel<<<(b->count + 127) / 128, 128, 0, st>>>(b->data, b->offsets, b->lengths, b->count, p->erp_gap, cost, d_bb);
    }
    if (wdtw) wdtw_table_kernel<<<(2 * kWdtwOff + 256) / 256, 256, 0, st>>>(d_wt, (double)p->wdtw_g, (double)p->wdtw_wmax);
    e |= (int)cudaGetLastError();
    if (e) return EAP_EDEVICE;

    eaph::LaunchCtx c;
    std::memset(&c, 0, sizeof(c));
    c.job.mode = kModePairs;
    c.job.A = dev_set(a, d_ba);
    c.job.B = dev_set(b, d_bb);
    c.job.nitems = (unsigned long long)n;
    c.job.counter = d_ctr;
    c.job.cut = p->prune ? cutoff : nullptr;
    c.job.out = out;
    c.job.ia = ia;
    c.job.ib = ib;
    c.job.stats = d_stats;
    c.job.wdtw_table = d_wt;
    c.job.bnd_stride = ((ma + 1) + 31) & ~31;
    c.kp = make_kparams(p);
    c.kp.wdtw_w = d_wt;
    c.rowpack = packed ? (float4*)(s + o_rp) : nullptr;
    c.kind = p->kind;
    c.cost = cost;
    c.prune = p->prune;
    // The same mapping as eap_pairs: CTA per pair for long unwindowed series
    // (the autotuned map or the default), else warp groups or band.
    c.cta = choose_cta(p->kind, cost, ma, mb, c.prune);
    choose_w_group(p->kind, cost, ma, mb, c.prune, &c.W, &c.group);
    if (c.cta) { c.W = choose_w_cta(p->kind, cost, mb, c.prune); c.group = 0; }
    choose_band(p->kind, c.prune, c.kp, std::min(set_min_len(a), set_min_len(b)), std::max(ma, mb), &c.band, &c.band_g, &c.band_exact);
    c.sms = sms;
    c.max_rows = ma;
    c.max_cols = mb;
    c.stream = st;
    if ((e = dispatch(c, false))) return cuda_status(e);
    if (opt_stats) {
        unsigned long long h[kStatCount];
        if (cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return EAP_EDEVICE;
        if (cudaStreamSynchronize(st) != cudaSuccess) return EAP_EDEVICE;
        opt_stats->pairs = h[kStatPairs];
        opt_stats->pairs_abandoned = h[kStatAbandoned];
        opt_stats->cells_computed = h[kStatCells];
    }
    return EAP_OK;
}

// Entry used by the serving loop (eap_serve.cu): 1-NN on device-resident sets
// on a given stream, no statistics.
namespace eaph {
int nn1_device(const eap_params* p, const eap_series_set* queries, const eap_series_set* refs, int32_t* out_idx,
               float* out_dist, cudaStream_t stream) {
    return nn1_impl(p, queries, refs, out_idx, out_dist, stream, nullptr, nullptr);
}
}  // namespace eaph

namespace eaph {
int validate_params_ext(const eap_params* p) { return validate_params(p); }
}  // namespace eaph

namespace eaph {
int tune_get(int kind, int cost, int bucket) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune[kind][cost][bucket];
}
void tune_set(int kind, int cost, int bucket, int w) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[kind][cost][bucket] = w;
}
void tune_reset() {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        std::memset(g_tune, 0, sizeof(g_tune));
    }
    std::lock_guard<std::mutex> lk(g_map_mu);
    std::memset(g_map, 0, sizeof(g_map));
}
void map_set(int kind, int cost, int bucket, int m) {
    std::lock_guard<std::mutex> lk(g_map_mu);
    g_map[kind][cost][bucket] = m;
}
int pick_w(int kind, int cost, int max_cols, int prune) { return choose_w(kind, cost, max_cols, prune); }
int pick_cta(int kind, int cost, int max_rows, int max_cols, int prune) {
    return choose_cta(kind, cost, max_rows, max_cols, prune);
}
int pick_w_cta(int kind, int cost, int max_cols, int prune) { return choose_w_cta(kind, cost, max_cols, prune); }
int pick_group(int kind, int cost, int max_rows, int max_cols, int prune, int W) {
    return choose_group(kind, cost, max_rows, max_cols, prune, W);
}
void pick_band(int kind, int prune, const KParams& kp, int min_len, int max_len, int* W, int* G, int* exact) {
    choose_band(kind, prune, kp, min_len, max_len, W, G, exact);
}

void pick_w_group(int kind, int cost, int max_rows, int max_cols, int prune, int* W, int* G) {
    choose_w_group(kind, cost, max_rows, max_cols, prune, W, G);
}
int bucket_of(int len) { return length_bucket(len); }
int resolve_cost_ext(const eap_params* p) { return resolve_cost(p); }
int validate_set_ext(const eap_series_set* s, int* max_len) { return validate_set(s, max_len); }
int check_finite_run(const float* data, long long n) {
    return check_inputs_enabled() ? check_finite(data, nullptr, nullptr, 0, n) : EAP_OK;
}
}  // namespace eaph

// Launch helpers for the batched path (eap_batch.cu), wrapping the kernels above.
namespace eaph {
void launch_erp_border(const eap_series_set* s, float gap, int cost, float* border, cudaStream_t st) {
    if (s->count > 0)
        erp_border_kernel<<<(s->count + 127) / 128, 128, 0, st>>>(s->data, s->offsets, s->lengths, s->count, gap, cost, border);
}
void launch_derivative(const eap_series_set* s, float* out, cudaStream_t st) {
    launch_derivative_set(s, out, device_sms(), st);
}
bool kind_packed(int kind) { return kind == EAP_ERP || kind == EAP_MSM || kind == EAP_TWE; }
int launch_rowpack(int kind, int cost, const eap_series_set* s, const KParams& kp, float4* out, cudaStream_t st) {
    if (s->count <= 0) return 0;
    const SeriesDev S{s->data, s->offsets, s->lengths, nullptr, s->count};
    const int blocks = std::min(s->count, std::max(1, device_sms()) * 8);
    switch (kind) {
        case EAP_ERP:
            if (cost) rowpack_kernel<FErp<1>><<<blocks, 128, 0, st>>>(S, kp, out);
            else rowpack_kernel<FErp<0>><<<blocks, 128, 0, st>>>(S, kp, out);
            break;
        case EAP_MSM: rowpack_kernel<FMsm><<<blocks, 128, 0, st>>>(S, kp, out); break;
        case EAP_TWE:
            if (cost) rowpack_kernel<FTwe<1>><<<blocks, 128, 0, st>>>(S, kp, out);
            else rowpack_kernel<FTwe<0>><<<blocks, 128, 0, st>>>(S, kp, out);
            break;
        default: return 0;
    }
    return (int)cudaGetLastError();
}
void launch_wdtw_table(float* tab, float g, float wmax, cudaStream_t st) {
    wdtw_table_kernel<<<(2 * kWdtwOff + 256) / 256, 256, 0, st>>>(tab, (double)g, (double)wmax);
}
void launch_lb(const eap_params* p, const eap_series_set* qs, const eap_series_set* rs, int two_way, float* qU,
               float* qL, float* rU, float* rL, float* lb, cudaStream_t st) {
    KParams ke = make_kparams(p);
    ke.windowed = 1;
    if (p->kind == EAP_DTW) { ke.window_abs = -1; ke.window_ratio = -1.f; }
    int mq = 0, mr = 0;
    for (int i = 0; i < qs->count; ++i) mq = std::max(mq, (int)qs->h_lengths[i]);
    for (int i = 0; i < rs->count; ++i) mr = std::max(mr, (int)rs->h_lengths[i]);
    launch_envelope(dev_set(qs, nullptr), ke, mq, qU, qL, st);
    if (two_way) launch_envelope(dev_set(rs, nullptr), ke, mr, rU, rL, st);
    launch_lb_matrix(dev_set(qs, nullptr), dev_set(rs, nullptr), qU, qL, rU, rL, resolve_cost(p), two_way, lb, st);
}
KParams kparams_of(const eap_params* p) { return make_kparams(p); }
// The EAPruned 1-NN DP of one task on its own pre-computed order, seeds and
// bounds (the batched path's per-task launch): the same mapping choice as
// eap_nn1 -- CTA per pair for long unwindowed series (autotuned or default),
// band coordinates for the windowed distances, 16-lane groups, or a warp per
// pair -- so a batch runs every task on the kernel eap_nn1 would use.
int nn1_dp_launch(const eap_params* p, const eap_series_set* qs, const eap_series_set* rs, const float* bq,
                  const float* br, const float* wt, const int32_t* order, unsigned long long* best, const float* lb,
                  float4* rowpack, unsigned long long* counter, unsigned long long* stats, int max_rows, int max_cols,
                  cudaStream_t st) {
    const int sms = device_sms();
    if (sms <= 0) return EAP_EDEVICE;
    const int cost = resolve_cost(p);
    eaph::LaunchCtx c;
    std::memset(&c, 0, sizeof(c));
    c.job.mode = kModeNN1;
    c.job.A = dev_set(qs, bq);
    c.job.B = dev_set(rs, br);
    c.job.nitems = (unsigned long long)qs->count * rs->count;
    c.job.counter = counter;
    c.job.order = order;
    c.job.best = best;
    c.job.stats = stats;
    c.job.wdtw_table = wt;
    c.job.lb = lb;
    c.job.bnd_stride = ((max_rows + 1) + 31) & ~31;
    c.kp = make_kparams(p);
    c.kp.wdtw_w = wt;
    c.rowpack = rowpack;
    c.kind = p->kind;
    c.cost = cost;
    c.prune = kPmPruned;
    c.sms = sms;
    c.max_rows = max_rows;
    c.max_cols = max_cols;
    nn1_mapping(p->kind, cost, c.prune, false, qs->count, max_rows, max_cols,
                std::min(set_min_len(qs), set_min_len(rs)), c);
    c.stream = st;
    return cuda_status(dispatch(c, false));
}


int nn1_timed(const eap_params* p, const eap_series_set* qs, const eap_series_set* rs, int32_t* idx, float* dist,
              cudaStream_t st, double* dp_ms) {
    eap_stats s;
    const int rc = nn1_impl(p, qs, rs, idx, dist, st, &s, nullptr);
    if (dp_ms) *dp_ms = s.dp_ms;
    return rc;
}
}  // namespace eaph
