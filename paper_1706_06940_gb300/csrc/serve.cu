// serve.cu -- a continuous-batching request server over resident arrays.
//
// Arrays are admitted while their plain-BbST state (block table and coarse
// table) plus the array itself fit in a device-memory budget; their tables
// stay resident until evicted.  Requests (an array id and host l, r, out
// buffers) are queued on submit.  A scheduler thread packs every pending
// request into one batch per tick -- one multi-request query launch
// (rmq_query_multi) between an upload and a download on one of several
// streams -- while earlier batches are still on the GPU, so new requests are
// admitted as slots free up and their work overlaps on the device.  A
// completion thread waits for each batch's event, copies the answers into the
// requests' buffers and records each request's latency (submit to answers).
#include <condition_variable>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "rmq_internal.cuh"

namespace rmq {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    int32_t array;
    const int32_t *l, *r;
    int32_t *out;
    int64_t q;
    Clock::time_point t_submit;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int32_t *h_l = nullptr, *h_r = nullptr, *h_out = nullptr;   // pinned staging
    int32_t *d_l = nullptr, *d_r = nullptr, *d_out = nullptr;   // device staging
    std::vector<Request> reqs;
    std::vector<int64_t> offs;
};

struct Resident {
    rmq_handle h;
    int64_t bytes;
};

}  // namespace
}  // namespace rmq

using namespace rmq;

struct rmq_server_s {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    int64_t cap = 0;                       // queries per batch
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_slot;
    std::deque<Request> pending;
    std::vector<Slot> slots;
    std::deque<int> free_slots, inflight;
    std::map<int32_t, Resident> arrays;
    int32_t next_id = 0;
    int64_t next_ticket = 0;
    std::map<int64_t, double> finished;    // ticket -> latency (s), until collected
    std::map<int64_t, rmq_status> failed;
    bool stop = false;
    std::thread sched, compl_;
    rmq_server_stats stats{};
};

namespace {

void scheduler(rmq_server_s *S) {
    cudaSetDevice(S->device);
    for (;;) {
        int si;
        std::vector<Request> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_sched.wait(lk, [&] { return S->stop || (!S->pending.empty() && !S->free_slots.empty()); });
            if (S->stop) return;
            si = S->free_slots.front();
            S->free_slots.pop_front();
            int64_t total = 0;
            while (!S->pending.empty() && (int)batch.size() < kReqMax) {
                const Request &rq = S->pending.front();
                if (!batch.empty() && total + rq.q > S->cap) break;
                total += rq.q;
                batch.push_back(rq);
                S->pending.pop_front();
            }
        }
        Slot &sl = S->slots[si];
        sl.reqs = batch;
        sl.offs.assign(1, 0);
        std::vector<QueryReq> qr;
        rmq_status st = RMQ_OK;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (const Request &rq : batch) {
                auto it = S->arrays.find(rq.array);
                const rmq_handle h = it->second.h;
                qr.push_back(QueryReq{h_array(h), h_table(h), h_coarse(h), h_n(h), rq.q, h_logk(h)});
            }
        }
        for (const Request &rq : batch) {
            const int64_t o = sl.offs.back();
            std::memcpy(sl.h_l + o, rq.l, (size_t)rq.q * 4);
            std::memcpy(sl.h_r + o, rq.r, (size_t)rq.q * 4);
            sl.offs.push_back(o + rq.q);
        }
        const int64_t total = sl.offs.back();
        cudaError_t e = cudaMemcpyAsync(sl.d_l, sl.h_l, (size_t)total * 4, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_r, sl.h_r, (size_t)total * 4, cudaMemcpyHostToDevice, sl.stream);
        int64_t qdone = 0;
        for (size_t g0 = 0; e == cudaSuccess && g0 < qr.size(); g0 += kReqMax) {
            const int cnt = (int)std::min<size_t>(kReqMax, qr.size() - g0);
            int64_t qg = 0;
            for (int i = 0; i < cnt; ++i) qg += qr[g0 + i].q;
            e = launch_query_handles(qr.data() + g0, cnt, sl.d_l + qdone, sl.d_r + qdone, sl.d_out + qdone, sl.stream);
            qdone += qg;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)total * 4, cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (e != cudaSuccess) st = RMQ_ERR_CUDA;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (st != RMQ_OK)
                for (const Request &rq : batch) S->failed[rq.ticket] = st;
            S->inflight.push_back(si);
            S->stats.batches += 1;
        }
        S->cv_done.notify_all();
    }
}

void completer(rmq_server_s *S) {
    cudaSetDevice(S->device);
    for (;;) {
        int si;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_done.wait(lk, [&] { return S->stop || !S->inflight.empty(); });
            if (S->stop && S->inflight.empty()) return;
            si = S->inflight.front();
        }
        Slot &sl = S->slots[si];
        const cudaError_t e = cudaEventSynchronize(sl.done);
        const Clock::time_point now = Clock::now();
        for (size_t i = 0; i < sl.reqs.size(); ++i)
            std::memcpy(sl.reqs[i].out, sl.h_out + sl.offs[i], (size_t)sl.reqs[i].q * 4);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->inflight.pop_front();
            for (const Request &rq : sl.reqs) {
                if (e != cudaSuccess) S->failed[rq.ticket] = RMQ_ERR_CUDA;
                else if (!S->failed.count(rq.ticket))
                    S->finished[rq.ticket] = std::chrono::duration<double>(now - rq.t_submit).count();
                S->stats.requests += 1;
                S->stats.queries += rq.q;
            }
            sl.reqs.clear();
            S->free_slots.push_back(si);
        }
        S->cv_sched.notify_all();
        S->cv_slot.notify_all();
    }
}

void destroy_server(rmq_server_s *S) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (const Request &rq : S->pending) S->failed[rq.ticket] = RMQ_ERR_INVALID_ARG;   // never scheduled
        S->pending.clear();
    }
    S->cv_slot.notify_all();
    S->cv_sched.notify_all();
    S->cv_done.notify_all();
    if (S->sched.joinable()) S->sched.join();
    if (S->compl_.joinable()) S->compl_.join();
    cudaSetDevice(S->device);
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        cudaFreeHost(sl.h_l); cudaFreeHost(sl.h_r); cudaFreeHost(sl.h_out);
        cudaFree(sl.d_l); cudaFree(sl.d_r); cudaFree(sl.d_out);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto &kv : S->arrays) rmq_free(kv.second.h);
    delete S;
}

}  // namespace

#pragma GCC visibility push(default)
extern "C" {

rmq_status rmq_server_create(const rmq_server_opts *opts, rmq_server *out) {
    if (!out) return RMQ_ERR_INVALID_ARG;
    *out = nullptr;
    rmq_server_opts o{};
    if (opts) o = *opts;
    if (o.budget_bytes < 0 || o.inflight < 0 || o.inflight > 64 || o.max_batch_queries < 0 || o.flags != 0)
        return RMQ_ERR_INVALID_ARG;
    rmq_server_s *S = new (std::nothrow) rmq_server_s();
    if (!S) return RMQ_ERR_OOM;
    cudaGetDevice(&S->device);
    S->budget = o.budget_bytes;
    S->cap = o.max_batch_queries ? o.max_batch_queries : (1 << 22);
    const int ns = o.inflight ? o.inflight : 4;
    S->slots.resize(ns);
    for (int i = 0; i < ns; ++i) {
        Slot &sl = S->slots[i];
        const size_t b = (size_t)S->cap * 4;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_l, b) != cudaSuccess || cudaMallocHost(&sl.h_r, b) != cudaSuccess ||
            cudaMallocHost(&sl.h_out, b) != cudaSuccess || cudaMalloc(&sl.d_l, b) != cudaSuccess ||
            cudaMalloc(&sl.d_r, b) != cudaSuccess || cudaMalloc(&sl.d_out, b) != cudaSuccess) {
            cudaGetLastError();
            destroy_server(S);
            return RMQ_ERR_OOM;
        }
        S->free_slots.push_back(i);
    }
    S->sched = std::thread(scheduler, S);
    S->compl_ = std::thread(completer, S);
    *out = S;
    return RMQ_OK;
}

rmq_status rmq_server_admit(rmq_server S, const int32_t *A, int64_t n, int32_t k, int32_t *id_out) {
    if (!S || !A || n <= 0 || !id_out) return RMQ_ERR_INVALID_ARG;
    cudaSetDevice(S->device);
    rmq_opts o{RMQ_VARIANT_PLAIN, k, 0, 0};
    {
        // reserve: the array's own cells and an upper bound of its tables
        std::lock_guard<std::mutex> lk(S->mu);
        rmq_opts t;
        rmq_tune(n, 0, &t);
        const int32_t kk = k ? k : t.k;
        const int64_t tb = rmq_table_bytes(n, kk);
        if (tb < 0) return RMQ_ERR_INVALID_ARG;
        const int64_t bytes = 4 * n + tb + 8 * kCoarseCap;
        if (S->budget > 0 && S->in_use + bytes > S->budget) return RMQ_ERR_BUDGET;
        S->in_use += bytes;
        o.k = kk;
    }
    rmq_handle h = nullptr;
    cudaStream_t bs = nullptr;
    cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
    rmq_status st = rmq_build(A, n, &o, bs, &h);
    if (st == RMQ_OK && cudaStreamSynchronize(bs) != cudaSuccess) st = RMQ_ERR_CUDA;
    cudaStreamDestroy(bs);
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t bytes = 4 * n + rmq_table_bytes(n, o.k) + 8 * kCoarseCap;
    if (st != RMQ_OK) {
        S->in_use -= bytes;
        if (h) rmq_free(h);
        return st;
    }
    const int32_t id = S->next_id++;
    S->arrays[id] = Resident{h, bytes};
    S->stats.table_bytes_in_use = S->in_use;
    *id_out = id;
    return RMQ_OK;
}

rmq_status rmq_server_evict(rmq_server S, int32_t id) {
    if (!S) return RMQ_ERR_INVALID_ARG;
    rmq_handle h = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->arrays.find(id);
        if (it == S->arrays.end()) return RMQ_ERR_INVALID_ARG;
        // wait until no queued or running request uses the array
        S->cv_slot.wait(lk, [&] {
            for (const Request &rq : S->pending) if (rq.array == id) return false;
            for (int si : S->inflight) for (const Request &rq : S->slots[si].reqs) if (rq.array == id) return false;
            return true;
        });
        h = it->second.h;
        S->in_use -= it->second.bytes;
        S->stats.table_bytes_in_use = S->in_use;
        S->arrays.erase(it);
    }
    cudaSetDevice(S->device);
    rmq_free(h);
    return RMQ_OK;
}

rmq_status rmq_server_submit(rmq_server S, int32_t id, const int32_t *l_host, const int32_t *r_host, int64_t q,
                             int32_t *out_host, int64_t *ticket_out) {
    if (!S || !ticket_out || q < 0) return RMQ_ERR_INVALID_ARG;
    if (q > 0 && (!l_host || !r_host || !out_host)) return RMQ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->arrays.count(id) || q > S->cap) return RMQ_ERR_INVALID_ARG;
    const int64_t t = S->next_ticket++;
    *ticket_out = t;
    if (q == 0) {
        S->finished[t] = 0.0;
        return RMQ_OK;
    }
    S->pending.push_back(Request{t, id, l_host, r_host, out_host, q, Clock::now()});
    S->cv_sched.notify_one();
    return RMQ_OK;
}

rmq_status rmq_server_wait(rmq_server S, int64_t ticket, double *latency_s) {
    if (!S || ticket < 0) return RMQ_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket >= S->next_ticket) return RMQ_ERR_INVALID_ARG;
    S->cv_slot.wait(lk, [&] { return S->finished.count(ticket) || S->failed.count(ticket); });
    auto f = S->failed.find(ticket);
    if (f != S->failed.end()) {
        const rmq_status st = f->second;
        S->failed.erase(f);
        return st;
    }
    auto it = S->finished.find(ticket);
    if (latency_s) *latency_s = it->second;
    S->finished.erase(it);
    return RMQ_OK;
}

rmq_status rmq_server_stats_get(rmq_server S, rmq_server_stats *out) {
    if (!S || !out) return RMQ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->table_bytes_in_use = S->in_use;
    out->resident_arrays = (int64_t)S->arrays.size();
    return RMQ_OK;
}

void rmq_server_destroy(rmq_server S) {
    if (S) destroy_server(S);
}

}  // extern "C"
#pragma GCC visibility pop
