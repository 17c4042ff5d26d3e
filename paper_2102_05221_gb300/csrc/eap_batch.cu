// eap_batch.cu -- many 1-NN problems in one call (eap_nn1_batch) and the
// mapping autotuner (eap_autotune).
//
// Every task (queries, references, one distance and its parameters) is a
// 1-NN search of its own.  The pre-passes run as one launch each over all
// tasks: cut-off init, the diagonal upper bound of every (query, candidate)
// pair, the per-query candidate sort with the cut-off seed, and the result
// unpack.  The DP then runs task by task, longest series first, each as one
// persistent launch of the kernel eap_nn1 would pick for it -- CTA per pair
// for long unwindowed series (by the autotuned table or the default), band
// coordinates for the windowed distances, 16-lane groups or a warp per pair
// otherwise -- with the strip width of the autotuned table.  Everything is
// enqueued on the caller's stream with stream-ordered scratch and no host
// synchronisation, so the whole call can be captured in one CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/eap.h"
#include "eap_internal.h"

using namespace eapd;

namespace {

enum {
    kFnDtwSq, kFnDtwAbs, kFnCdtwSq, kFnCdtwAbs, kFnWdtwSq, kFnWdtwAbs, kFnErpSq, kFnErpAbs, kFnMsm, kFnTweSq, kFnTweAbs
};

int fn_of(int kind, int cost) {
    switch (kind) {
        case EAP_DTW: return cost ? kFnDtwAbs : kFnDtwSq;
        case EAP_CDTW: return cost ? kFnCdtwAbs : kFnCdtwSq;
        case EAP_WDTW: return cost ? kFnWdtwAbs : kFnWdtwSq;
        case EAP_ERP: return cost ? kFnErpAbs : kFnErpSq;
        case EAP_MSM: return kFnMsm;
        default: return cost ? kFnTweAbs : kFnTweSq;
    }
}

struct TaskDev {
    SeriesDev A, B;              // queries (rows), references (columns)
    KParams kp;
    const float* wt;             // WDTW weight table or null
    unsigned long long* best;    // per query
    int32_t* order;              // [nq x nr]
    float* ub;                   // [nq x nr]
    const float* lb;             // [nq x nr] or null
    const float4* rp;            // packed row constants of the queries (ERP, MSM, TWE) or null
    int32_t* out_idx;
    float* out_dist;
    unsigned long long begin;    // first work item of the task
    int qbegin;                  // first query of the task in the batch numbering
    int fn, nq, nr;
};

constexpr int kUploadChunk = 96;   // tasks per parameter block (kernel parameters are limited to ~32 KB)
struct TaskChunk {
    TaskDev t[kUploadChunk];
    int n, base;
};
static_assert(sizeof(TaskChunk) < 32000, "task chunk must fit in the kernel parameter space");

__global__ void upload_tasks_kernel(const __grid_constant__ TaskChunk ch, TaskDev* dst) {
    for (int i = threadIdx.x; i < ch.n; i += blockDim.x) dst[ch.base + i] = ch.t[i];
}

// Last task whose first work item (or first query) is <= x.
__device__ __forceinline__ int find_task_item(const TaskDev* __restrict__ T, int n, unsigned long long x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T[mid].begin <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int find_task_query(const TaskDev* __restrict__ T, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T[mid].qbegin <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ void fill_pair(const TaskDev& T, int q, int c, PairIn& in) {
    const int64_t oa = T.A.off[q], ob = T.B.off[c];
    in.A = T.A.data + oa;
    in.B = T.B.data + ob;
    in.La = T.A.len[q];
    in.Lb = T.B.len[c];
    in.bA = T.A.border ? T.A.border + oa : nullptr;
    in.bB = T.B.border ? T.B.border + ob : nullptr;
    in.wt = T.wt ? T.wt + kWdtwOff - max(in.La, in.Lb) : nullptr;
    in.cut_src = T.best + q;
    in.rp = T.rp ? T.rp + oa : nullptr;
    in.w = pair_window(T.kp, in.La, in.Lb);
    in.cut = EAP_FINF;
}

template <class F>
__device__ float ub_of(const PairIn& in, const KParams& kp) { return diag_path_cost<F>(in, kp); }

__device__ float ub_by_fn(int fn, const PairIn& in, const KParams& kp) {
    switch (fn) {
        case kFnDtwSq: case kFnCdtwSq: return ub_of<FDtw<0>>(in, kp);
        case kFnDtwAbs: case kFnCdtwAbs: return ub_of<FDtw<1>>(in, kp);
        case kFnWdtwSq: return ub_of<FWdtw<0>>(in, kp);
        case kFnWdtwAbs: return ub_of<FWdtw<1>>(in, kp);
        case kFnErpSq: return ub_of<FErp<0>>(in, kp);
        case kFnErpAbs: return ub_of<FErp<1>>(in, kp);
        case kFnMsm: return ub_of<FMsm>(in, kp);
        case kFnTweSq: return ub_of<FTwe<0>>(in, kp);
        default: return ub_of<FTwe<1>>(in, kp);
    }
}

__global__ void batch_init_kernel(const TaskDev* __restrict__ T, int nt, int total_q) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_q; g += gridDim.x * blockDim.x) {
        const TaskDev& t = T[find_task_query(T, nt, g)];
        t.best[g - t.qbegin] = pack_best(EAP_FINF, kNoIndex);
    }
}

__global__ void batch_ub_kernel(const TaskDev* __restrict__ T, int nt, unsigned long long total) {
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < total;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const TaskDev& t = T[find_task_item(T, nt, k)];
        const unsigned long long local = k - t.begin;
        const int q = (int)(local / (unsigned)t.nr);
        const int c = (int)(local - (unsigned long long)q * t.nr);
        PairIn in;
        fill_pair(t, q, c, in);
        in.cut_src = nullptr;
        t.ub[local] = ub_by_fn(t.fn, in, t.kp);
    }
}

// One block per query of the batch: candidates sorted by upper bound, and the
// smallest bound as the query's first cut-off (same as eap_nn1).
__global__ void batch_sort_kernel(const TaskDev* __restrict__ T, int nt) {
    extern __shared__ unsigned long long keys[];
    const TaskDev& t = T[find_task_query(T, nt, blockIdx.x)];
    const int q = blockIdx.x - t.qbegin;
    const int nb = t.nr;
    int chunk = 1;
    while (chunk < nb && chunk < 4096) chunk <<= 1;
    const float* u = t.ub + (size_t)q * nb;
    int32_t* o = t.order + (size_t)q * nb;
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
                        if ((a > b) == ((i & k) == 0)) { keys[i] = b; keys[l] = a; }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) o[base + i] = (int32_t)(keys[i] & 0xffffffffu);
        if (keys[0] < gmin) gmin = keys[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) t.best[q] = nb > 0 ? (((gmin >> 32) << 32) | kNoIndex) : pack_best(EAP_FINF, kNoIndex);
}

__global__ void batch_unpack_kernel(const TaskDev* __restrict__ T, int nt, int total_q, unsigned long long* stats) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_q; g += gridDim.x * blockDim.x) {
        const TaskDev& t = T[find_task_query(T, nt, g)];
        const int q = g - t.qbegin;
        const unsigned long long b = t.best[q];
        const unsigned ix = (unsigned)(b & 0xffffffffu);
        const float d = __uint_as_float((unsigned)(b >> 32));
        if (ix == kNoIndex) {
            t.out_idx[q] = -1;
            t.out_dist[q] = EAP_FINF;
            if (d != EAP_FINF && stats) atomicAdd(stats + kStatErrors, 1ULL);
        } else {
            t.out_idx[q] = (int32_t)ix;
            t.out_dist[q] = d;
        }
    }
}

struct HostTask {
    int src;            // index in the caller's array
    int fn, cost;
    int nq, nr, mq, mr;
    bool erp, wdtw, lb, lb2, deriv, packed;
};

int device_sms_b() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    return sms;
}

}  // namespace

extern "C" int eap_nn1_batch(const eap_nn1_task* tasks, int32_t ntasks, void* cuda_stream, eap_stats* opt_stats) {
    if (ntasks < 0 || (ntasks > 0 && !tasks)) return EAP_EINVAL;
    if (opt_stats) std::memset(opt_stats, 0, sizeof(*opt_stats));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<HostTask> ht;
    for (int i = 0; i < ntasks; ++i) {
        const eap_nn1_task& tk = tasks[i];
        int rc = eaph::validate_params_ext(&tk.params);
        if (rc) return rc;
        if (tk.params.prune != 1) return EAP_EINVAL;
        int mq = 0, mr = 0;
        if ((rc = eaph::validate_set_ext(&tk.queries, &mq)) || (rc = eaph::validate_set_ext(&tk.refs, &mr))) return rc;
        if (tk.queries.count > 0 && (!tk.out_idx || !tk.out_dist)) return EAP_EINVAL;
        if (tk.queries.count == 0) continue;
        HostTask h{};
        h.src = i;
        h.cost = eaph::resolve_cost_ext(&tk.params);
        h.fn = fn_of(tk.params.kind, h.cost);
        h.nq = tk.queries.count;
        h.nr = tk.refs.count;
        h.mq = mq;
        h.mr = mr;
        h.erp = tk.params.kind == EAP_ERP;
        h.wdtw = tk.params.kind == EAP_WDTW;
        h.lb = tk.params.lb != EAP_LB_NONE && (tk.params.kind == EAP_DTW || tk.params.kind == EAP_CDTW);
        h.lb2 = h.lb && tk.params.lb == EAP_LB_KEOGH2;
        h.deriv = tk.params.derivative != 0;
        h.packed = eaph::kind_packed(tk.params.kind);
        ht.push_back(h);
    }
    const int sms = device_sms_b();
    if (sms <= 0) return EAP_EDEVICE;
    const int nt = (int)ht.size();
    if (nt == 0) return EAP_OK;
    // Work-queue order: longest series first, then the larger tasks.
    std::stable_sort(ht.begin(), ht.end(), [](const HostTask& a, const HostTask& b) {
        const int la = std::max(a.mq, a.mr), lb = std::max(b.mq, b.mr);
        if (la != lb) return la > lb;
        return (long long)a.nq * a.nr > (long long)b.nq * b.nr;
    });

    // One stream-ordered scratch block for every task.
    size_t used = 0;
    auto take = [&](size_t bytes) { const size_t o = (used + 255) & ~(size_t)255; used = o + bytes; return o; };
    const size_t o_tasks = take(sizeof(TaskDev) * nt);
    const size_t o_ctr = take(sizeof(unsigned long long) * nt);   // one work-queue head per task
    const size_t o_stats = take(sizeof(unsigned long long) * kStatCount);
    struct Off { size_t best, ub, order, lb, qU, qL, rU, rL, bq, br, wt, dq, dr, rp; };
    std::vector<Off> off(nt);
    for (int k = 0; k < nt; ++k) {
        const HostTask& h = ht[k];
        const eap_nn1_task& tk = tasks[h.src];
        const size_t pairs = (size_t)h.nq * h.nr;
        Off& o = off[k];
        o = Off{};
        o.best = take(sizeof(unsigned long long) * h.nq);
        o.ub = take(sizeof(float) * std::max<size_t>(pairs, 1));
        o.order = take(sizeof(int32_t) * std::max<size_t>(pairs, 1));
        if (h.lb && h.nr > 0) {
            o.lb = take(sizeof(float) * pairs);
            o.qU = take(sizeof(float) * (size_t)tk.queries.data_len);
            o.qL = take(sizeof(float) * (size_t)tk.queries.data_len);
            if (h.lb2) {
                o.rU = take(sizeof(float) * (size_t)tk.refs.data_len);
                o.rL = take(sizeof(float) * (size_t)tk.refs.data_len);
            }
        }
        if (h.erp) {
            o.bq = take(sizeof(float) * (size_t)tk.queries.data_len);
            o.br = take(sizeof(float) * std::max<int64_t>(tk.refs.data_len, 1));
        }
        if (h.wdtw) o.wt = take(sizeof(float) * (2 * kWdtwOff + 1));
        if (h.deriv) {
            o.dq = take(sizeof(float) * (size_t)tk.queries.data_len);
            o.dr = take(sizeof(float) * std::max<int64_t>(tk.refs.data_len, 1));
        }
        if (h.packed) o.rp = take(sizeof(float4) * ((size_t)tk.queries.data_len + 1));
    }
    // The sets each task's kernels read: the caller's, or (derivative variants,
    // Section 2.3) copies whose data are the first-derivative series.
    std::vector<eap_series_set> qset(nt), rset(nt);
    for (int k = 0; k < nt; ++k) {
        qset[k] = tasks[ht[k].src].queries;
        rset[k] = tasks[ht[k].src].refs;
    }
    char* base = nullptr;
    if (cudaMallocAsync((void**)&base, used, st) != cudaSuccess) { cudaGetLastError(); return EAP_ENOMEM; }
    for (int k = 0; k < nt; ++k) {
        if (!ht[k].deriv) continue;
        eaph::launch_derivative(&qset[k], (float*)(base + off[k].dq), st);
        eaph::launch_derivative(&rset[k], (float*)(base + off[k].dr), st);
        qset[k].data = (const float*)(base + off[k].dq);
        rset[k].data = (const float*)(base + off[k].dr);
    }

    std::vector<TaskDev> td(nt);
    unsigned long long items = 0;
    int total_q = 0;
    for (int k = 0; k < nt; ++k) {
        const HostTask& h = ht[k];
        const eap_nn1_task& tk = tasks[h.src];
        const Off& o = off[k];
        TaskDev& t = td[k];
        std::memset(&t, 0, sizeof(t));
        float* bq = h.erp ? (float*)(base + o.bq) : nullptr;
        float* br = h.erp ? (float*)(base + o.br) : nullptr;
        t.A = SeriesDev{qset[k].data, tk.queries.offsets, tk.queries.lengths, bq, tk.queries.count};
        t.B = SeriesDev{rset[k].data, tk.refs.offsets, tk.refs.lengths, br, tk.refs.count};
        t.kp = eaph::kparams_of(&tk.params);
        t.wt = h.wdtw ? (const float*)(base + o.wt) : nullptr;
        t.best = (unsigned long long*)(base + o.best);
        t.ub = (float*)(base + o.ub);
        t.order = (int32_t*)(base + o.order);
        t.lb = (h.lb && h.nr > 0) ? (const float*)(base + o.lb) : nullptr;
        t.rp = h.packed ? (const float4*)(base + o.rp) : nullptr;
        t.out_idx = tk.out_idx;
        t.out_dist = tk.out_dist;
        t.begin = items;
        t.qbegin = total_q;
        t.fn = h.fn;
        t.nq = h.nq;
        t.nr = h.nr;
        items += (unsigned long long)h.nq * h.nr;
        total_q += h.nq;
    }
    TaskDev* d_tasks = (TaskDev*)(base + o_tasks);
    unsigned long long* d_ctr = (unsigned long long*)(base + o_ctr);
    unsigned long long* d_stats = (unsigned long long*)(base + o_stats);
    int e = 0;
    for (int b0 = 0; b0 < nt; b0 += kUploadChunk) {
        TaskChunk ch;
        std::memset(&ch, 0, sizeof(ch));
        ch.n = std::min(kUploadChunk, nt - b0);
        ch.base = b0;
        for (int i = 0; i < ch.n; ++i) ch.t[i] = td[b0 + i];
        upload_tasks_kernel<<<1, 128, 0, st>>>(ch, d_tasks);
    }
    e |= (int)cudaMemsetAsync(d_ctr, 0, sizeof(unsigned long long) * nt, st);
    e |= (int)cudaMemsetAsync(d_stats, 0, sizeof(unsigned long long) * kStatCount, st);
    batch_init_kernel<<<(total_q + 255) / 256, 256, 0, st>>>(d_tasks, nt, total_q);
    // DP time (stats only: events are not created for calls without stats).
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (opt_stats && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess)) {
        cudaGetLastError();
        ev[0] = ev[1] = nullptr;
    }
    for (int k = 0; k < nt; ++k) {
        const HostTask& h = ht[k];
        const eap_nn1_task& tk = tasks[h.src];
        const Off& o = off[k];
        if (h.erp) {
            eaph::launch_erp_border(&qset[k], tk.params.erp_gap, h.cost, (float*)(base + o.bq), st);
            eaph::launch_erp_border(&rset[k], tk.params.erp_gap, h.cost, (float*)(base + o.br), st);
        }
        if (h.wdtw) eaph::launch_wdtw_table((float*)(base + o.wt), tk.params.wdtw_g, tk.params.wdtw_wmax, st);
        if (h.lb && h.nr > 0)
            eaph::launch_lb(&tk.params, &qset[k], &rset[k], h.lb2 ? 1 : 0, (float*)(base + o.qU), (float*)(base + o.qL),
                            h.lb2 ? (float*)(base + o.rU) : nullptr, h.lb2 ? (float*)(base + o.rL) : nullptr,
                            (float*)(base + o.lb), st);
    }
    if (items > 0) {
        unsigned long long ub_blocks = std::min<unsigned long long>((items + 255) / 256, (unsigned long long)sms * 16);
        batch_ub_kernel<<<(unsigned)ub_blocks, 256, 0, st>>>(d_tasks, nt, items);
        int max_nr = 0;
        for (auto& h : ht) max_nr = std::max(max_nr, h.nr);
        int chunk = 1;
        while (chunk < max_nr && chunk < 4096) chunk <<= 1;
        batch_sort_kernel<<<total_q, 512, sizeof(unsigned long long) * chunk, st>>>(d_tasks, nt);
        // The DP, task by task (longest series first), each on eap_nn1's kernel
        // for it; the packed row constants are computed by that launch.
        if (ev[0]) cudaEventRecord(ev[0], st);
        for (int k = 0; k < nt && !e; ++k) {
            const HostTask& h = ht[k];
            if (h.nr == 0) continue;
            const eap_nn1_task& tk = tasks[h.src];
            const Off& o = off[k];
            const int rc = eaph::nn1_dp_launch(&tk.params, &qset[k], &rset[k],
                                               h.erp ? (const float*)(base + o.bq) : nullptr,
                                               h.erp ? (const float*)(base + o.br) : nullptr,
                                               h.wdtw ? (const float*)(base + o.wt) : nullptr, td[k].order, td[k].best,
                                               td[k].lb, h.packed ? (float4*)(base + o.rp) : nullptr, d_ctr + k, d_stats,
                                               h.mq, h.mr, st);
            if (rc) e |= 1;
        }
        if (ev[1]) cudaEventRecord(ev[1], st);
    }
    batch_unpack_kernel<<<(total_q + 255) / 256, 256, 0, st>>>(d_tasks, nt, total_q, d_stats);
    e |= (int)cudaGetLastError();
    unsigned long long hs[kStatCount];
    if (!e && opt_stats) e |= (int)cudaMemcpyAsync(hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(base, st);
    if (e) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        return EAP_EDEVICE;
    }
    if (opt_stats) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return EAP_EDEVICE;
        opt_stats->pairs = hs[kStatPairs] + hs[kStatLbPruned];
        opt_stats->pairs_lb_pruned = hs[kStatLbPruned];
        opt_stats->pairs_abandoned = hs[kStatAbandoned];
        opt_stats->cells_computed = hs[kStatCells];
        unsigned long long eff = 0;
        for (auto& h : ht) {
            const eap_nn1_task& tk = tasks[h.src];
            unsigned long long a = 0, b = 0;
            for (int i = 0; i < tk.queries.count; ++i) a += (unsigned long long)tk.queries.h_lengths[i];
            for (int i = 0; i < tk.refs.count; ++i) b += (unsigned long long)tk.refs.h_lengths[i];
            eff += a * b;
        }
        opt_stats->cells_effective = eff;
        float ms = 0.f;
        if (ev[0] && ev[1] && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) opt_stats->dp_ms = ms;
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        if (hs[kStatErrors]) return EAP_EINTERNAL;
    }
    return EAP_OK;
}

// ---------------------------------------------------------------------------
// Strip-width autotuner.
// ---------------------------------------------------------------------------
extern "C" int eap_autotune(const eap_nn1_task* tasks, int32_t ntasks, void* cuda_stream, const char* cache_path) {
    if (ntasks < 0 || (ntasks > 0 && !tasks)) return EAP_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    struct Key { int kind, cost, bucket, src; long long work; };
    std::vector<Key> keys;
    for (int i = 0; i < ntasks; ++i) {
        const eap_nn1_task& tk = tasks[i];
        int rc = eaph::validate_params_ext(&tk.params);
        if (rc) return rc;
        int mq = 0, mr = 0;
        if ((rc = eaph::validate_set_ext(&tk.queries, &mq)) || (rc = eaph::validate_set_ext(&tk.refs, &mr))) return rc;
        if (tk.queries.count == 0 || tk.refs.count == 0) continue;
        const int cost = eaph::resolve_cost_ext(&tk.params);
        const int b = eaph::bucket_of(mr);
        const long long work = (long long)tk.queries.count * tk.refs.count;
        bool found = false;
        for (auto& k : keys) {
            if (k.kind == tk.params.kind && k.cost == cost && k.bucket == b) {
                found = true;
                if (work > k.work) { k.work = work; k.src = i; }
            }
        }
        if (!found) keys.push_back(Key{tk.params.kind, cost, b, i, work});
    }
    int32_t* d_idx = nullptr;
    float* d_dist = nullptr;
    if (cudaMalloc((void**)&d_idx, 64 * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&d_dist, 64 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_idx);
        return EAP_ENOMEM;
    }
    FILE* f = cache_path ? std::fopen(cache_path, "a") : nullptr;
    int rc = EAP_OK;
    for (const Key& k : keys) {
        const eap_nn1_task& tk = tasks[k.src];
        eap_series_set qs = tk.queries, rs = tk.refs;
        qs.count = std::min(qs.count, 64);
        rs.count = std::min(rs.count, 512);
        eap_params p = tk.params;
        p.prune = 1;
        int best_w = 0, best_map = 1;
        double best_ms = 1e300;
        // W = 4, 5, 8, 16 (16-lane groups where they apply, else a warp per
        // pair); CTA-per-pair with W = 4, 8 for long unwindowed buckets.
        const bool try_cta = k.bucket >= 11 && k.kind != EAP_CDTW && k.kind != EAP_ERP;
        const int cands[6][2] = {{4, 1}, {5, 1}, {8, 1}, {16, 1}, {4, 2}, {8, 2}};
        for (int ci = 0; ci < (try_cta ? 6 : 4); ++ci) {
            eaph::tune_set(k.kind, k.cost, k.bucket, cands[ci][0]);
            eaph::map_set(k.kind, k.cost, k.bucket, cands[ci][1]);
            double ms = 0.0;
            if ((rc = eaph::nn1_timed(&p, &qs, &rs, d_idx, d_dist, st, &ms))) break;
            if ((rc = eaph::nn1_timed(&p, &qs, &rs, d_idx, d_dist, st, &ms))) break;
            if (ms < best_ms) { best_ms = ms; best_w = cands[ci][0]; best_map = cands[ci][1]; }
        }
        if (rc) break;
        eaph::tune_set(k.kind, k.cost, k.bucket, best_w);
        eaph::map_set(k.kind, k.cost, k.bucket, best_map);
        if (f) std::fprintf(f, "%d %d %d %d %d\n", k.kind, k.cost, k.bucket, best_w, best_map);
    }
    if (f) std::fclose(f);
    cudaFree(d_idx);
    cudaFree(d_dist);
    return rc;
}

extern "C" int eap_autotune_load(const char* cache_path) {
    if (!cache_path) return EAP_EINVAL;
    FILE* f = std::fopen(cache_path, "r");
    if (!f) return EAP_EINVAL;
    int kind, cost, bucket, w, m;
    while (std::fscanf(f, "%d %d %d %d %d", &kind, &cost, &bucket, &w, &m) == 5) {
        if (kind >= 0 && kind < 6 && (cost == 0 || cost == 1) && bucket >= 0 && bucket < 16 && (w == 4 || w == 5 || w == 8 || w == 16)
            && (m == 1 || m == 2)) {
            eaph::tune_set(kind, cost, bucket, w);
            eaph::map_set(kind, cost, bucket, m);
        }
    }
    std::fclose(f);
    return EAP_OK;
}

extern "C" void eap_autotune_reset(void) { eaph::tune_reset(); }
