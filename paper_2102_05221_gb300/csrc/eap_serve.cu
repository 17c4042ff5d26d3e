// eap_serve.cu -- the serving loop behind eap_serve_* (include/eap.h).
//
// Reference sets are copied to HBM once and stay resident.  Clients submit
// single 1-NN queries (any length, any distance) from host memory; a query is
// admitted only while the number of queries in flight and their HBM footprint
// (query bytes + per-candidate scratch of the 1-NN search) stay inside the
// configured budget, otherwise the submit answers EAP_EAGAIN.
//
// Continuous batching: a worker thread keeps up to kSlots launches in flight,
// each on its own stream.  Whenever a slot is free it takes the pending query
// with the least work (query length x set elements) -- or the oldest one, once
// it has waited kMaxWaitMs -- and with it every pending query of the same work
// class (at most kClassFactor times the lead's work), whatever its reference
// set or distance.  Those queries are grouped by (set, parameters) into tasks
// and run as one eap_nn1_batch call: one pass of upper bounds, candidate sort
// and cut-off seeds over all of them, then each task's DP on the kernel
// eap_nn1 would pick.  Queries that arrive while launches are on the GPU join
// the next free slot, so their work overlaps the running ones.  A result is
// the same float32 distance and index whether its query runs alone or in a
// batch: the DP's value of a pair does not depend on the cut-off it ran with,
// and ties go to the lowest index.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <limits>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/eap.h"
#include "eap_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kSlots = 8;                    // streams with a launch in flight
constexpr int kBatchMaxQueries = 512;
constexpr int64_t kBatchMaxFloats = 1 << 22; // query floats per launch (16 MiB)
constexpr double kClassFactor = 2.0;         // a launch takes queries with up to this much the lead's work
constexpr double kMaxWaitMs = 200.0;         // a query waiting this long leads the next launch

struct RefSet {
    float* d_data = nullptr;
    int64_t* d_off = nullptr;
    int32_t* d_len = nullptr;
    std::vector<int64_t> h_off;
    std::vector<int32_t> h_len;
    int64_t data_len = 0;
    int32_t count = 0;
};

struct Req {
    uint64_t ticket;
    int32_t set_id;
    eap_params p;
    std::vector<float> q;
    int64_t bytes;
    Clock::time_point t0;
};

struct Result {
    int32_t idx;
    float dist;
    int rc;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    float* h_q = nullptr;        // pinned staging
    int64_t* h_off = nullptr;
    int32_t* h_len = nullptr;
    int32_t* h_idx = nullptr;
    float* h_dist = nullptr;
    float* d_q = nullptr;
    int64_t* d_off = nullptr;
    int32_t* d_len = nullptr;
    int32_t* d_idx = nullptr;
    float* d_dist = nullptr;
    std::vector<Req> reqs;
    bool busy = false;
    int rc = EAP_OK;
};

bool same_params(const eap_params& a, const eap_params& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

}  // namespace

struct eap_server {
    eap_serve_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;       // worker wake-up and completion notices
    std::thread worker;
    bool stop = false;
    std::vector<RefSet> sets;
    std::deque<Req> pending;
    std::unordered_map<uint64_t, Result> done;
    std::unordered_map<uint64_t, int> live;   // admitted and not yet completed
    int64_t inflight_bytes = 0;
    int32_t inflight = 0;
    uint64_t next_ticket = 1;
    Slot slots[kSlots];
    eap_serve_stats st{};
    std::vector<double> lat;

    void run();
    bool launch(Slot& s);
    void complete(Slot& s, bool ok);
};

namespace {

int64_t query_footprint(const eap_server* s, int32_t set_id, int32_t len) {
    const int64_t nr = s->sets[set_id].count;
    // query data + per-candidate upper bound and order + best-so-far and outputs
    return (int64_t)len * 4 + nr * 8 + 64;
}

}  // namespace

bool eap_server::launch(Slot& sl) {
    std::vector<Req> batch;
    std::vector<RefSet> views;   // pointers and host mirrors of the resident sets the launch reads
    std::vector<int32_t> view_of_set;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (pending.empty()) return false;
        auto work = [&](const Req& r) { return (double)r.q.size() * (double)sets[r.set_id].data_len; };
        // Lead: the oldest query once it has waited kMaxWaitMs, else the least work.
        const auto now = Clock::now();
        auto lead = pending.begin();
        if (std::chrono::duration<double, std::milli>(now - lead->t0).count() < kMaxWaitMs) {
            for (auto it = pending.begin(); it != pending.end(); ++it)
                if (work(*it) < work(*lead)) lead = it;
        }
        const double lead_work = work(*lead);
        int64_t floats = (int64_t)lead->q.size();
        batch.push_back(std::move(*lead));
        pending.erase(lead);
        for (auto it = pending.begin(); it != pending.end() && (int)batch.size() < kBatchMaxQueries;) {
            if (work(*it) <= lead_work * kClassFactor && floats + (int64_t)it->q.size() <= kBatchMaxFloats) {
                floats += (int64_t)it->q.size();
                batch.push_back(std::move(*it));
                it = pending.erase(it);
            } else {
                ++it;
            }
        }
        view_of_set.assign(sets.size(), -1);
        for (const Req& r : batch) {
            if (view_of_set[r.set_id] >= 0) continue;
            view_of_set[r.set_id] = (int32_t)views.size();
            const RefSet& rs = sets[r.set_id];
            RefSet v;
            v.d_data = rs.d_data;
            v.d_off = rs.d_off;
            v.d_len = rs.d_len;
            v.h_off = rs.h_off;
            v.h_len = rs.h_len;
            v.data_len = rs.data_len;
            v.count = rs.count;
            views.push_back(std::move(v));
        }
    }
    // Group the queries by (set, parameters): each group is one task.
    std::stable_sort(batch.begin(), batch.end(), [](const Req& x, const Req& y) {
        if (x.set_id != y.set_id) return x.set_id < y.set_id;
        return std::memcmp(&x.p, &y.p, sizeof(eap_params)) < 0;
    });
    const int nq = (int)batch.size();
    int64_t off = 0;
    for (int i = 0; i < nq; ++i) {
        std::memcpy(sl.h_q + off, batch[i].q.data(), batch[i].q.size() * sizeof(float));
        sl.h_off[i] = off;
        sl.h_len[i] = (int32_t)batch[i].q.size();
        off += (int64_t)batch[i].q.size();
    }
    int e = 0;
    e |= (int)cudaMemcpyAsync(sl.d_q, sl.h_q, sizeof(float) * off, cudaMemcpyHostToDevice, sl.st);
    e |= (int)cudaMemcpyAsync(sl.d_off, sl.h_off, sizeof(int64_t) * nq, cudaMemcpyHostToDevice, sl.st);
    e |= (int)cudaMemcpyAsync(sl.d_len, sl.h_len, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, sl.st);
    int rc = e ? EAP_EDEVICE : EAP_OK;
    std::vector<eap_nn1_task> tasks;
    for (int b0 = 0; b0 < nq && rc == EAP_OK;) {
        int b1 = b0 + 1;
        while (b1 < nq && batch[b1].set_id == batch[b0].set_id && same_params(batch[b1].p, batch[b0].p)) ++b1;
        const RefSet& rs = views[view_of_set[batch[b0].set_id]];
        eap_series_set qs{sl.d_q, sl.d_off + b0, sl.d_len + b0, sl.h_off + b0, sl.h_len + b0, off, b1 - b0, 0};
        eap_series_set rset{rs.d_data, rs.d_off, rs.d_len, rs.h_off.data(), rs.h_len.data(), rs.data_len, rs.count, 0};
        if (batch[b0].p.prune == 1) {
            tasks.push_back(eap_nn1_task{batch[b0].p, qs, rset, sl.d_idx + b0, sl.d_dist + b0});
        } else {
            // Base, EABase and Prune groups run as their own search.
            rc = eaph::nn1_device(&batch[b0].p, &qs, &rset, sl.d_idx + b0, sl.d_dist + b0, sl.st);
        }
        b0 = b1;
    }
    if (rc == EAP_OK && !tasks.empty()) rc = eap_nn1_batch(tasks.data(), (int32_t)tasks.size(), sl.st, nullptr);
    if (rc == EAP_OK) {
        e = (int)cudaMemcpyAsync(sl.h_idx, sl.d_idx, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, sl.st);
        e |= (int)cudaMemcpyAsync(sl.h_dist, sl.d_dist, sizeof(float) * nq, cudaMemcpyDeviceToHost, sl.st);
        e |= (int)cudaEventRecord(sl.ev, sl.st);
        if (e) rc = EAP_EDEVICE;
    }
    sl.reqs = std::move(batch);
    sl.rc = rc;
    sl.busy = true;
    {
        std::lock_guard<std::mutex> lk(mu);
        st.batches++;
    }
    if (rc != EAP_OK) complete(sl, false);
    return true;
}

void eap_server::complete(Slot& sl, bool ok) {
    const auto now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        const Req& r = sl.reqs[i];
        Result res{-1, std::numeric_limits<float>::infinity(), ok ? EAP_OK : (sl.rc != EAP_OK ? sl.rc : EAP_EDEVICE)};
        if (ok) { res.idx = sl.h_idx[i]; res.dist = sl.h_dist[i]; }
        done[r.ticket] = res;
        live.erase(r.ticket);
        inflight--;
        inflight_bytes -= r.bytes;
        st.completed++;
        lat.push_back(std::chrono::duration<double, std::milli>(now - r.t0).count());
    }
    sl.reqs.clear();
    sl.busy = false;
    cv.notify_all();
}

void eap_server::run() {
    cudaSetDevice(device);
    for (;;) {
        bool progress = false;
        for (auto& sl : slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaSuccess) { complete(sl, true); progress = true; }
            else if (q != cudaErrorNotReady) { cudaGetLastError(); sl.rc = EAP_EDEVICE; complete(sl, false); progress = true; }
        }
        for (auto& sl : slots) {
            if (!sl.busy && launch(sl)) progress = true;
        }
        std::unique_lock<std::mutex> lk(mu);
        bool any_busy = false;
        for (auto& sl : slots) any_busy |= sl.busy;
        if (stop && pending.empty() && !any_busy) break;
        if (!progress) {
            if (pending.empty() && !any_busy) cv.wait_for(lk, std::chrono::milliseconds(2));
            else cv.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

extern "C" {

eap_server* eap_serve_create(const eap_serve_config* cfg, int* status) {
    auto fail = [&](int code) -> eap_server* { if (status) *status = code; return nullptr; };
    if (!cfg) return fail(EAP_EINVAL);
    if (cfg->max_inflight < 0 || cfg->max_query_len < 0 || cfg->hbm_budget_bytes < 0 || cfg->device < 0)
        return fail(EAP_EINVAL);
    eap_server* s = new (std::nothrow) eap_server();
    if (!s) return fail(EAP_ENOMEM);
    s->cfg = *cfg;
    if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 4096;
    if (s->cfg.max_query_len == 0) s->cfg.max_query_len = 8192;
    if (s->cfg.max_query_len > 8192) { delete s; return fail(EAP_EINVAL); }
    s->device = cfg->device;
    if (cudaSetDevice(s->device) != cudaSuccess) { cudaGetLastError(); delete s; return fail(EAP_EDEVICE); }
    if (s->cfg.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete s; return fail(EAP_EDEVICE); }
        s->cfg.hbm_budget_bytes = (int64_t)(fr / 2);
    }
    const int64_t qcap = std::max<int64_t>(kBatchMaxFloats, s->cfg.max_query_len);
    for (auto& sl : s->slots) {
        int e = 0;
        e |= (int)cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        e |= (int)cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        e |= (int)cudaMallocHost((void**)&sl.h_q, sizeof(float) * qcap);
        e |= (int)cudaMallocHost((void**)&sl.h_off, sizeof(int64_t) * kBatchMaxQueries);
        e |= (int)cudaMallocHost((void**)&sl.h_len, sizeof(int32_t) * kBatchMaxQueries);
        e |= (int)cudaMallocHost((void**)&sl.h_idx, sizeof(int32_t) * kBatchMaxQueries);
        e |= (int)cudaMallocHost((void**)&sl.h_dist, sizeof(float) * kBatchMaxQueries);
        e |= (int)cudaMalloc((void**)&sl.d_q, sizeof(float) * qcap);
        e |= (int)cudaMalloc((void**)&sl.d_off, sizeof(int64_t) * kBatchMaxQueries);
        e |= (int)cudaMalloc((void**)&sl.d_len, sizeof(int32_t) * kBatchMaxQueries);
        e |= (int)cudaMalloc((void**)&sl.d_idx, sizeof(int32_t) * kBatchMaxQueries);
        e |= (int)cudaMalloc((void**)&sl.d_dist, sizeof(float) * kBatchMaxQueries);
        if (e) { cudaGetLastError(); eap_serve_destroy(s); return fail(EAP_ENOMEM); }
    }
    s->worker = std::thread([s] { s->run(); });
    if (status) *status = EAP_OK;
    return s;
}

int eap_serve_add_refset(eap_server* s, const float* h_data, const int64_t* h_offsets, const int32_t* h_lengths,
                         int32_t count, int32_t* set_id) {
    if (!s || !set_id || count <= 0 || !h_data || !h_offsets || !h_lengths) return EAP_EINVAL;
    RefSet rs;
    rs.count = count;
    rs.h_off.assign(h_offsets, h_offsets + count);
    rs.h_len.assign(h_lengths, h_lengths + count);
    int64_t len = 0;
    for (int i = 0; i < count; ++i) {
        if (h_lengths[i] <= 0 || h_lengths[i] > 8192 || h_offsets[i] < 0) return EAP_EINVAL;
        len = std::max<int64_t>(len, h_offsets[i] + h_lengths[i]);
    }
    rs.data_len = len;
    if (cudaSetDevice(s->device) != cudaSuccess) return EAP_EDEVICE;
    int e = 0;
    e |= (int)cudaMalloc((void**)&rs.d_data, sizeof(float) * len);
    e |= (int)cudaMalloc((void**)&rs.d_off, sizeof(int64_t) * count);
    e |= (int)cudaMalloc((void**)&rs.d_len, sizeof(int32_t) * count);
    if (e) {
        cudaGetLastError();
        cudaFree(rs.d_data); cudaFree(rs.d_off); cudaFree(rs.d_len);
        return EAP_ENOMEM;
    }
    e |= (int)cudaMemcpy(rs.d_data, h_data, sizeof(float) * len, cudaMemcpyHostToDevice);
    e |= (int)cudaMemcpy(rs.d_off, h_offsets, sizeof(int64_t) * count, cudaMemcpyHostToDevice);
    e |= (int)cudaMemcpy(rs.d_len, h_lengths, sizeof(int32_t) * count, cudaMemcpyHostToDevice);
    if (e) { cudaFree(rs.d_data); cudaFree(rs.d_off); cudaFree(rs.d_len); return EAP_EDEVICE; }
    std::lock_guard<std::mutex> lk(s->mu);
    s->sets.push_back(std::move(rs));
    *set_id = (int32_t)s->sets.size() - 1;
    return EAP_OK;
}

int eap_serve_submit(eap_server* s, int32_t set_id, const eap_params* p, const float* h_query, int32_t len,
                     uint64_t* ticket) {
    if (!s || !p || !h_query || !ticket || len <= 0) return EAP_EINVAL;
    int rc = eaph::validate_params_ext(p);
    if (rc) return rc;
    if (len > s->cfg.max_query_len) return EAP_EINVAL;
    Req r;
    r.set_id = set_id;
    r.p = *p;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (set_id < 0 || set_id >= (int32_t)s->sets.size()) return EAP_EINVAL;
        r.bytes = query_footprint(s, set_id, len);
        if (s->inflight >= s->cfg.max_inflight || s->inflight_bytes + r.bytes > s->cfg.hbm_budget_bytes) {
            s->st.rejected++;
            return EAP_EAGAIN;
        }
        r.ticket = s->next_ticket++;
        s->inflight++;
        s->inflight_bytes += r.bytes;
        s->live[r.ticket] = 1;
        s->st.submitted++;
    }
    r.q.assign(h_query, h_query + len);
    r.t0 = Clock::now();
    *ticket = r.ticket;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->pending.push_back(std::move(r));
    }
    s->cv.notify_all();
    return EAP_OK;
}

int eap_serve_poll(eap_server* s, uint64_t ticket, int32_t* idx, float* dist) {
    if (!s) return EAP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return s->live.count(ticket) ? EAP_EAGAIN : EAP_EINVAL;
    const Result r = it->second;
    s->done.erase(it);
    if (r.rc != EAP_OK) return r.rc;
    if (idx) *idx = r.idx;
    if (dist) *dist = r.dist;
    return EAP_OK;
}

int eap_serve_drain(eap_server* s, int32_t timeout_ms) {
    if (!s) return EAP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (s->inflight > 0) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout && s->inflight > 0) return EAP_ETIMEOUT;
    }
    return EAP_OK;
}

int eap_serve_stats_get(eap_server* s, eap_serve_stats* out, int32_t reset) {
    if (!s || !out) return EAP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->inflight = s->inflight;
    out->inflight_bytes = s->inflight_bytes;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
        out->lat_p50_ms = pct(0.50);
        out->lat_p99_ms = pct(0.99);
        out->lat_max_ms = v.back();
    }
    if (reset) {
        s->lat.clear();
        s->st = eap_serve_stats{};
    }
    return EAP_OK;
}

int eap_serve_destroy(eap_server* s) {
    if (!s) return EAP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        cudaFreeHost(sl.h_q); cudaFreeHost(sl.h_off); cudaFreeHost(sl.h_len);
        cudaFreeHost(sl.h_idx); cudaFreeHost(sl.h_dist);
        cudaFree(sl.d_q); cudaFree(sl.d_off); cudaFree(sl.d_len); cudaFree(sl.d_idx); cudaFree(sl.d_dist);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    for (auto& rs : s->sets) { cudaFree(rs.d_data); cudaFree(rs.d_off); cudaFree(rs.d_len); }
    delete s;
    return EAP_OK;
}

}  // extern "C"
