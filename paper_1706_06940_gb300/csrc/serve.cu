// serve.cu -- a continuous-batching request server over resident arrays.
//
// Arrays are admitted while their plain-BbST state (block table and coarse
// table) plus the array itself fit in a device-memory budget; their tables
// stay resident until evicted.  Requests (an array id and host l, r, out
// buffers) are queued on submit.  A scheduler thread packs every pending
// request into one batch per tick -- one multi-request query launch between
// an upload and a download on one of several streams -- while earlier
// batches are still on the GPU, so new requests are admitted as slots free up
// and their work overlaps on the device.  A completion thread waits for each
// batch's event, copies the answers into the requests' buffers and records
// each request's latency (submit to answers).
//
// Lifetime of an array's tables: a request pins its array from the moment the
// scheduler takes it off the queue (under the server lock, where its table
// pointers are also resolved) until the completion thread has copied its
// answers.  rmq_server_evict first closes the array to new requests, then
// waits until no queued request names it and no taken request pins it, and
// only then frees the tables.
#include <chrono>
#include <condition_variable>
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
    std::vector<QueryReq> qr;     // the requests' table pointers, resolved when they were taken
    std::vector<int64_t> offs;
};

struct Resident {
    rmq_handle h;
    int64_t bytes;
    int64_t n;
    int64_t pinned = 0;    // requests taken off the queue and not yet completed
    bool closing = false;  // evict has begun: no new requests
};

}  // namespace
}  // namespace rmq

using namespace rmq;

struct rmq_server_s {
    int device = 0;
    int64_t budget = 0, in_use = 0;
    int64_t cap = 0;                       // queries per batch
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_slot, cv_budget;
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

// Copies q entries of l and r into the staging buffers and reports whether
// every query is valid for an array of n cells (0 <= l <= r < n).
bool stage_and_check(const int32_t *l, const int32_t *r, int64_t q, int64_t n, int32_t *dl, int32_t *dr) {
    bool ok = true;
    for (int64_t i = 0; i < q; ++i) {
        const int32_t a = l[i], b = r[i];
        dl[i] = a;
        dr[i] = b;
        ok &= a >= 0 && b >= a && (int64_t)b < n;
    }
    return ok;
}

// Whether a ticket is still to complete: queued, or taken into a slot that
// has not been handed back (a slot's requests are set and cleared under the
// server lock, in the same critical sections that take it from and return it
// to free_slots).  The caller holds the lock.
bool outstanding(const rmq_server_s *S, int64_t t) {
    for (const Request &rq : S->pending)
        if (rq.ticket == t) return true;
    std::vector<char> is_free(S->slots.size(), 0);
    for (int f : S->free_slots) is_free[f] = 1;
    for (size_t i = 0; i < S->slots.size(); ++i)
        if (!is_free[i])
            for (const Request &rq : S->slots[i].reqs)
                if (rq.ticket == t) return true;
    return false;
}

void scheduler(rmq_server_s *S) {
    cudaSetDevice(S->device);
    for (;;) {
        int si;
        std::vector<int64_t> arr_n;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_sched.wait(lk, [&] { return S->stop || (!S->pending.empty() && !S->free_slots.empty()); });
            if (S->stop) return;
            si = S->free_slots.front();
            S->free_slots.pop_front();
            Slot &sl = S->slots[si];
            sl.reqs.clear();
            sl.qr.clear();
            int64_t total = 0;
            while (!S->pending.empty() && (int)sl.reqs.size() < kReqMax) {
                const Request &rq = S->pending.front();
                if (!sl.reqs.empty() && total + rq.q > S->cap) break;
                // the array cannot be freed while the request pins it
                Resident &res = S->arrays.at(rq.array);
                res.pinned += 1;
                const rmq_handle h = res.h;
                sl.qr.push_back(QueryReq{h_array(h), h_table(h), h_coarse(h), h_n(h), rq.q, h_logk(h)});
                arr_n.push_back(res.n);
                total += rq.q;
                sl.reqs.push_back(rq);
                S->pending.pop_front();
            }
        }
        Slot &sl = S->slots[si];
        sl.offs.assign(1, 0);
        std::vector<int64_t> bad_tickets;
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            const Request &rq = sl.reqs[i];
            const int64_t o = sl.offs.back();
            if (!stage_and_check(rq.l, rq.r, rq.q, arr_n[i], sl.h_l + o, sl.h_r + o)) bad_tickets.push_back(rq.ticket);
            sl.offs.push_back(o + rq.q);
        }
        const int64_t total = sl.offs.back();
        cudaError_t e = cudaMemcpyAsync(sl.d_l, sl.h_l, (size_t)total * 4, cudaMemcpyHostToDevice, sl.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_r, sl.h_r, (size_t)total * 4, cudaMemcpyHostToDevice, sl.stream);
        int64_t qdone = 0;
        for (size_t g0 = 0; e == cudaSuccess && g0 < sl.qr.size(); g0 += kReqMax) {
            const int cnt = (int)std::min<size_t>(kReqMax, sl.qr.size() - g0);
            int64_t qg = 0;
            for (int i = 0; i < cnt; ++i) qg += sl.qr[g0 + i].q;
            e = launch_query_handles(sl.qr.data() + g0, cnt, sl.d_l + qdone, sl.d_r + qdone, sl.d_out + qdone,
                                     sl.stream);
            qdone += qg;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)total * 4, cudaMemcpyDeviceToHost, sl.stream);
        if (e == cudaSuccess && !bad_tickets.empty()) {
            // the invalid queries were reported per request above (from the
            // host check); the kernels also raised the slot stream's error
            // word, which is cleared here so that it reports nothing later
            unsigned *ew = err_word_ptr(sl.stream);
            if (ew) e = cudaMemsetAsync(ew, 0, sizeof(unsigned), sl.stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (e != cudaSuccess)
                for (const Request &rq : sl.reqs) S->failed[rq.ticket] = RMQ_ERR_CUDA;
            else
                for (int64_t t : bad_tickets) S->failed[t] = RMQ_ERR_QUERY_RANGE;
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
                auto it = S->arrays.find(rq.array);
                if (it != S->arrays.end()) it->second.pinned -= 1;
            }
            sl.reqs.clear();
            sl.qr.clear();
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
    S->cv_budget.notify_all();
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

// Bytes an admitted array holds against the budget: its cells and exactly the
// tables rmq_build allocates for it.
int64_t admit_bytes(int64_t n, int32_t k) { return 4 * n + handle_bytes_for(n, ilog2_host((uint64_t)k)); }

rmq_status admit_impl(rmq_server S, const int32_t *A, int64_t n, int32_t k, double timeout_s, int32_t *id_out) {
    if (!S || !A || n <= 0 || n > 2147483647ll || !id_out) return RMQ_ERR_INVALID_ARG;
    if (k != 0 && (k < 32 || k > 65536 || (k & (k - 1)))) return RMQ_ERR_INVALID_ARG;
    cudaSetDevice(S->device);
    rmq_opts o{RMQ_VARIANT_PLAIN, k, 0, 0};
    if (!k) {
        rmq_opts t;
        rmq_tune(n, 0, &t);
        o.k = t.k;
    }
    const int64_t bytes = admit_bytes(n, o.k);
    {
        // reserve the array's bytes; with a timeout, wait for evictions to free them
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->budget > 0 && bytes > S->budget) return RMQ_ERR_BUDGET;
        auto fits = [&] { return S->stop || S->budget <= 0 || S->in_use + bytes <= S->budget; };
        if (!fits()) {
            if (timeout_s <= 0) return RMQ_ERR_BUDGET;
            if (!S->cv_budget.wait_for(lk, std::chrono::duration<double>(timeout_s), fits) || S->stop)
                return RMQ_ERR_BUDGET;
        }
        S->in_use += bytes;
    }
    rmq_handle h = nullptr;
    cudaStream_t bs = nullptr;
    rmq_status st = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess ? RMQ_OK : RMQ_ERR_CUDA;
    if (st == RMQ_OK) st = rmq_build(A, n, &o, bs, &h);
    if (st == RMQ_OK && cudaStreamSynchronize(bs) != cudaSuccess) st = RMQ_ERR_CUDA;
    if (bs) cudaStreamDestroy(bs);
    std::lock_guard<std::mutex> lk(S->mu);
    if (st != RMQ_OK) {
        S->in_use -= bytes;
        if (h) rmq_free(h);
        S->cv_budget.notify_all();
        return st;
    }
    const int32_t id = S->next_id++;
    Resident res;
    res.h = h;
    res.bytes = bytes;
    res.n = n;
    S->arrays[id] = res;
    S->stats.table_bytes_in_use = S->in_use;
    *id_out = id;
    return RMQ_OK;
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
    return admit_impl(S, A, n, k, 0.0, id_out);
}

rmq_status rmq_server_admit_wait(rmq_server S, const int32_t *A, int64_t n, int32_t k, double timeout_s,
                                 int32_t *id_out) {
    if (timeout_s < 0) return RMQ_ERR_INVALID_ARG;
    return admit_impl(S, A, n, k, timeout_s, id_out);
}

rmq_status rmq_server_evict(rmq_server S, int32_t id) {
    if (!S) return RMQ_ERR_INVALID_ARG;
    rmq_handle h = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->arrays.find(id);
        if (it == S->arrays.end() || it->second.closing) return RMQ_ERR_INVALID_ARG;
        it->second.closing = true;   // new submits on id are refused from here on
        // wait until no queued request names the array and no taken one pins it
        S->cv_slot.wait(lk, [&] {
            if (it->second.pinned > 0) return false;
            for (const Request &rq : S->pending)
                if (rq.array == id) return false;
            return true;
        });
        h = it->second.h;
        S->in_use -= it->second.bytes;
        S->stats.table_bytes_in_use = S->in_use;
        S->arrays.erase(it);
    }
    cudaSetDevice(S->device);
    rmq_free(h);
    S->cv_budget.notify_all();
    return RMQ_OK;
}

rmq_status rmq_server_submit(rmq_server S, int32_t id, const int32_t *l_host, const int32_t *r_host, int64_t q,
                             int32_t *out_host, int64_t *ticket_out) {
    if (!S || !ticket_out || q < 0) return RMQ_ERR_INVALID_ARG;
    if (q > 0 && (!l_host || !r_host || !out_host)) return RMQ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->arrays.find(id);
    if (it == S->arrays.end() || it->second.closing || q > S->cap) return RMQ_ERR_INVALID_ARG;
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
    // a ticket that is neither done nor outstanding was collected before
    if (!S->finished.count(ticket) && !S->failed.count(ticket) && !outstanding(S, ticket))
        return RMQ_ERR_INVALID_ARG;
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
