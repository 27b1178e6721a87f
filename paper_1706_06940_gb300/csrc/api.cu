// api.cu -- the C ABI declared in include/rmq.h: argument checks, the choice
// of form and block size, stream-ordered workspace, resident handles and the
// sticky device error word.  Every computation is done by the kernels of
// plain.cu and contract.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "rmq_internal.cuh"

namespace rmq {

// Sticky error words (ERR_* bits), one per stream slot on each device:
// raised by kernels, read and cleared by rmq_stream_status on the stream.
__device__ unsigned g_err_words[kErrSlots];

namespace {

std::atomic<int64_t> g_launches{0};
std::once_flag g_dev_once[kMaxDev];
int g_sms[kMaxDev];
unsigned *g_err_base[kMaxDev];

// Stream -> error-word slot of one device.  Slot 0 is the legacy default
// stream; other streams get slots 1 .. kErrSlots - 1 in order of first use,
// and once those are taken, further streams share them round-robin.
struct ErrSlots {
    std::mutex mu;
    uintptr_t stream[kErrSlots] = {};
    int used = 1;
    int next_shared = 1;
    int slot_of(uintptr_t s) {
        if (s == 0 || s == 1) return 0;   // NULL and cudaStreamLegacy: the legacy stream
        std::lock_guard<std::mutex> lk(mu);
        for (int i = 1; i < used; ++i)
            if (stream[i] == s) return i;
        if (used < kErrSlots) {
            stream[used] = s;
            return used++;
        }
        const int i = next_shared;
        next_shared = next_shared + 1 < kErrSlots ? next_shared + 1 : 1;
        return i;
    }
};
ErrSlots g_slots[kMaxDev];

// Once per device: its SM count and the address of its error words.
void device_setup(int d) {
    once_per_device(g_dev_once, d, [d] {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            sms = 148;
        }
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_err_words) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (d >= 0 && d < kMaxDev) {
            g_sms[d] = sms;
            g_err_base[d] = static_cast<unsigned *>(p);
        }
    });
}

}  // namespace

void note_launches(int count) { g_launches.fetch_add(count, std::memory_order_relaxed); }

DevInfo dev_info() {
    int d = 0;
    cudaGetDevice(&d);
    if (d < 0 || d >= kMaxDev) return DevInfo{d, 148};
    device_setup(d);
    return DevInfo{d, g_sms[d]};
}

unsigned *err_word_ptr(cudaStream_t s) {
    int d = 0;
    cudaGetDevice(&d);
    if (d < 0 || d >= kMaxDev) return nullptr;
    device_setup(d);
    if (!g_err_base[d]) return nullptr;
    return g_err_base[d] + g_slots[d].slot_of(reinterpret_cast<uintptr_t>(s));
}

namespace {

// Workspace from the device's default stream-ordered pool; freed memory
// stays cached in the pool for the next call.
std::once_flag g_pool_once[kMaxDev];

void pool_setup() {
    int d = 0;
    cudaGetDevice(&d);
    once_per_device(g_pool_once, d, [d] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        } else {
            cudaGetLastError();
        }
    });
}

struct Workspace {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    rmq_status alloc(size_t bytes, cudaStream_t stream) {
        pool_setup();
        s = stream;
        cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(bytes, 256), stream);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); p = nullptr; return RMQ_ERR_OOM; }
        if (e != cudaSuccess) { p = nullptr; return RMQ_ERR_CUDA; }
        return RMQ_OK;
    }
    ~Workspace() {
        if (p) cudaFreeAsync(p, s);
    }
};

bool pow2_in_range(int32_t k) {
    return k >= (1 << MIN_LOGK) && k <= (1 << MAX_LOGK) && (k & (k - 1)) == 0;
}

int64_t table_entries(int64_t n, int logk) {
    const int64_t nb = cdiv(n, 1ll << logk);
    return nb * (ilog2_host((uint64_t)nb) + 1);
}

int pow2_log_near(double x, int lo, int hi) {
    int t = (int)std::lround(std::log2(std::max(x, 1.0)));
    return std::min(hi, std::max(lo, t));
}

}  // namespace

}  // namespace rmq

using namespace rmq;

namespace {

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

constexpr int64_t kMaxN = 2147483647ll;
constexpr int64_t kMaxQ = 2147483647ll;   // positions and query indices fit in int32

rmq_status check_batch_args(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                            const int32_t *out, const rmq_opts *opts) {
    if (n <= 0 || n > kMaxN || q < 0 || q > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (!A) return RMQ_ERR_INVALID_ARG;
    if (q > 0 && (!l || !r || !out)) return RMQ_ERR_INVALID_ARG;
    if (opts) {
        if (opts->variant < RMQ_VARIANT_AUTO || opts->variant > RMQ_VARIANT_CONTRACTED) return RMQ_ERR_INVALID_ARG;
        if (opts->k != 0 && !pow2_in_range(opts->k)) return RMQ_ERR_INVALID_ARG;
        if (opts->k_con != 0 && !pow2_in_range(opts->k_con)) return RMQ_ERR_INVALID_ARG;
        if (opts->flags != 0) return RMQ_ERR_INVALID_ARG;
        const int32_t t = opts->threads_per_query;
        if (t != 0 && t != 8 && t != 16 && t != 32) return RMQ_ERR_INVALID_ARG;
        if (opts->k1 != 0 && opts->k1 != -1 && !pow2_in_range(opts->k1)) return RMQ_ERR_INVALID_ARG;
        if (opts->k1 > 0 && opts->k != 0 && opts->k1 > opts->k) return RMQ_ERR_INVALID_ARG;
    }
    return RMQ_OK;
}

rmq_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RMQ_OK;
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return RMQ_ERR_OOM; }
    return RMQ_ERR_CUDA;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;   // unknown: do not read the batch back
    }
    return cs != cudaStreamCaptureStatusNone;
}

// The tuner's choice for a batch: the remembered one for its shape, and when
// the shape holds choices for several width classes and l, r are given (an
// AUTO call), the one for the batch's width class, from a sample of its
// queries (not while the stream is being captured: then the lowest class).
rmq_opts tuned_for(int64_t n, int64_t q, const int32_t *l, const int32_t *r, cudaStream_t s) {
    rmq_opts t;
    rmq_tune(n, q, &t);
    rmq_opts m;
    if (q > 0 && l && r && tuned_lookup(n, q, -1, &m) == TUNE_AMBIGUOUS && !stream_capturing(s)) {
        const int w = sample_width_class(l, r, q, n, s);
        if (w >= 0 && tuned_lookup(n, q, w, &m) == TUNE_FOUND) t = m;
    }
    return t;
}

// Fill zero fields of opts with the tuner's choice.  The batch is sampled
// only for an AUTO form (l, r may be null).  A choice's threads_per_query and
// k1 were measured with its form and block size, so they are taken only with
// those.
rmq_opts resolve_opts(int64_t n, int64_t q, const rmq_opts *opts, const int32_t *l = nullptr,
                      const int32_t *r = nullptr, cudaStream_t s = nullptr) {
    const bool auto_form = !opts || opts->variant == RMQ_VARIANT_AUTO;
    rmq_opts t = tuned_for(n, q, auto_form ? l : nullptr, auto_form ? r : nullptr, s);
    if (opts) {
        if (opts->variant != RMQ_VARIANT_AUTO && opts->variant != t.variant) {
            t.variant = opts->variant;
            t.threads_per_query = 0;
            t.k1 = 0;
        }
        if (opts->k) {
            if (opts->k != t.k) t.k1 = 0;
            t.k = opts->k;
        }
        if (opts->k_con) t.k_con = opts->k_con;
        if (opts->threads_per_query) t.threads_per_query = opts->threads_per_query;
        if (opts->k1) t.k1 = opts->k1;
    }
    return t;
}

// Teams of partial-block scans (1, 2 or 4 per warp) for threads_per_query.
int max_teams_of(int32_t tpq) { return tpq == 32 ? 1 : (tpq == 16 ? 2 : 4); }

// log2 of the small blocks of the two-level layout for k1 and k = 2^logk
// (-1: none): k1 = 0 is 128 cells when k >= 128.
int logk1_of(int32_t k1, int logk) {
    if (k1 < 0) return -1;
    if (k1 == 0) return logk >= 7 ? 7 : -1;
    return ilog2_host((uint64_t)k1);
}

// Keys of a plain batch call's workspace: levels 0..lc of the block table,
// then the small-block minima of the two-level layout (Sec. 3.3), one per
// 2^logk1 cells (none for logk1 < 0).
int64_t plain_table_keys(int64_t n, int logk) { return two_level_entries(cdiv(n, 1ll << logk)); }
int64_t plain_m1_keys(int64_t n, int logk1) { return logk1 >= 0 ? cdiv(n, 1ll << logk1) : 0; }
int64_t plain_workspace_bytes(int64_t n, int logk, int logk1) {
    return (plain_table_keys(n, logk) + plain_m1_keys(n, logk1)) * 8;
}

rmq_status batch_plain(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                       int logk, int logk1, int max_teams, cudaStream_t s, Stages *sg,
                       unsigned long long *counts = nullptr) {
    const int64_t nb = cdiv(n, 1ll << logk);
    Workspace ws;
    const int64_t te = plain_table_keys(n, logk);
    const int64_t m1 = plain_m1_keys(n, logk1);
    rmq_status st = ws.alloc((size_t)plain_workspace_bytes(n, logk, logk1), s);
    if (st != RMQ_OK) return st;
    uint64_t *T = static_cast<uint64_t *>(ws.p);
    uint64_t *M1 = m1 ? T + te : nullptr;
    cudaError_t e;
    sg->mark(s);
    if ((e = launch_block_minima_i32(A, n, logk, T, s, M1, logk1)) != cudaSuccess) return cuda_status(e);
    sg->mark(s);
    if ((e = launch_sparse_table(T, Len{n, nullptr}, logk, nb, s, true)) != cudaSuccess) return cuda_status(e);
    sg->mark(s);
    e = launch_query_plain(A, n, logk, T, nullptr, l, r, q, out, s, M1, kCoarseCap, counts, logk1, max_teams);
    sg->mark(s);
    return cuda_status(e);
}

rmq_status batch_contracted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                            int logk_con, int max_teams, cudaStream_t s, Stages *sg,
                            unsigned long long *counts = nullptr) {
    Workspace ws;
    rmq_status st = ws.alloc(con_workspace_bytes(n, q, logk_con), s);
    if (st != RMQ_OK) return st;
    return cuda_status(run_contracted(A, n, l, r, q, out, logk_con, ws.p, s, sg, counts, max_teams));
}

rmq_status batch_dispatch(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                          const rmq_opts *opts, cudaStream_t s, Stages *sg, unsigned long long *counts = nullptr) {
    rmq_status st = check_batch_args(A, n, l, r, q, out, opts);
    if (st != RMQ_OK) return st;
    if (q == 0) return RMQ_OK;
    const rmq_opts o = resolve_opts(n, q, opts, l, r, s);
    const int teams = max_teams_of(o.threads_per_query);
    if (o.variant == RMQ_VARIANT_CONTRACTED)
        return batch_contracted(A, n, l, r, q, out, ilog2_host((uint64_t)o.k_con), teams, s, sg, counts);
    if (o.k1 > o.k) return RMQ_ERR_INVALID_ARG;   // small blocks larger than the blocks
    const int logk = ilog2_host((uint64_t)o.k);
    return batch_plain(A, n, l, r, q, out, logk, logk1_of(o.k1, logk), teams, s, sg, counts);
}

}  // namespace

struct rmq_handle_s {
    const int32_t *A;
    int64_t n;
    int logk;
    int64_t nb;
    uint64_t *T;
    uint64_t *Cs;  // coarse summary, right after the table
    int64_t bytes;
    int device;
};

namespace rmq {
int64_t handle_bytes_for(int64_t n, int logk) { return (two_level_entries(cdiv(n, 1ll << logk)) + kCoarseCap) * 8; }
const int32_t *h_array(rmq_handle h) { return h->A; }
const uint64_t *h_table(rmq_handle h) { return h->T; }
const uint64_t *h_coarse(rmq_handle h) { return h->Cs; }
int64_t h_n(rmq_handle h) { return h->n; }
int32_t h_logk(rmq_handle h) { return h->logk; }
}  // namespace rmq

#pragma GCC visibility push(default)
extern "C" {

rmq_status rmq_batch(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                     void *stream) {
    return rmq_batch_ex(A, n, l, r, q, out, nullptr, stream);
}

rmq_status rmq_batch_ex(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                        const rmq_opts *opts, void *stream) {
    Stages none;
    return batch_dispatch(A, n, l, r, q, out, opts, as_stream(stream), &none);
}

rmq_status rmq_batch_timed(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                           const rmq_opts *opts, void *stream, void *const *events, int32_t n_events) {
    if (n_events < 0 || (n_events > 0 && !events)) return RMQ_ERR_INVALID_ARG;
    Stages sg;
    sg.ev = reinterpret_cast<cudaEvent_t *>(const_cast<void **>(events));
    sg.n = n_events;
    return batch_dispatch(A, n, l, r, q, out, opts, as_stream(stream), &sg);
}

rmq_status rmq_batch_counted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                             int32_t *out, const rmq_opts *opts, void *stream, rmq_scan_stats *stats) {
    if (!stats) return RMQ_ERR_INVALID_ARG;
    rmq_status st = check_batch_args(A, n, l, r, q, out, opts);
    if (st != RMQ_OK) return st;
    *stats = rmq_scan_stats{};
    if (q == 0) return RMQ_OK;
    if (((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(r) |
          reinterpret_cast<uintptr_t>(out)) & 15) != 0)
        return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    Workspace ws;
    if ((st = ws.alloc(CNT_N * sizeof(unsigned long long), s)) != RMQ_OK) return st;
    unsigned long long *c = static_cast<unsigned long long *>(ws.p);
    if (cudaMemsetAsync(c, 0, CNT_N * sizeof(unsigned long long), s) != cudaSuccess) return RMQ_ERR_CUDA;
    Stages none;
    if ((st = batch_dispatch(A, n, l, r, q, out, opts, s, &none, c)) != RMQ_OK) return st;
    unsigned long long h[CNT_N] = {};
    if (cudaMemcpyAsync(h, c, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RMQ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMQ_ERR_CUDA;
    stats->open_queries = (int64_t)h[CNT_OPEN];
    stats->table_reads = (int64_t)h[CNT_TABLE];
    stats->m1_reads = (int64_t)h[CNT_M1];
    stats->scan_elems = (int64_t)h[CNT_ELEMS];
    stats->rank_reads = (int64_t)h[CNT_RANKS];
    return RMQ_OK;
}

int64_t rmq_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

rmq_status rmq_batch_host(const int32_t *A_host, int64_t n, const int32_t *l_host, const int32_t *r_host, int64_t q,
                          int32_t *out_host, const rmq_opts *opts, void *stream) {
    rmq_status st = check_batch_args(A_host, n, l_host, r_host, q, out_host, opts);
    if (st != RMQ_OK) return st;
    if (q == 0) return RMQ_OK;
    cudaStream_t s = as_stream(stream);
    const size_t bA = (size_t)n * 4, bq = (size_t)q * 4;
    const size_t oA = 0, oL = (bA + 255) & ~(size_t)255, oR = oL + ((bq + 255) & ~(size_t)255),
                 oO = oR + ((bq + 255) & ~(size_t)255);
    char *base = nullptr;
    {
        Workspace ws;
        if ((st = ws.alloc(oO + bq, s)) != RMQ_OK) return st;
        base = static_cast<char *>(ws.p);
        int32_t *dA = reinterpret_cast<int32_t *>(base + oA), *dl = reinterpret_cast<int32_t *>(base + oL),
                *dr = reinterpret_cast<int32_t *>(base + oR), *dout = reinterpret_cast<int32_t *>(base + oO);
        cudaError_t e;
        if ((e = cudaMemcpyAsync(dA, A_host, bA, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaMemcpyAsync(dl, l_host, bq, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaMemcpyAsync(dr, r_host, bq, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
        if ((st = rmq_batch_ex(dA, n, dl, dr, q, dout, opts, stream)) != RMQ_OK) return st;
        if ((e = cudaMemcpyAsync(out_host, dout, bq, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_status(e);
    }
    // invalid queries were counted in the device error word: report (and
    // clear) it, as rmq_stream_status does, without scanning out_host
    return rmq_stream_status(stream);
}

rmq_status rmq_batch_multi(const rmq_array *arrays, int32_t H, const int32_t *l, const int32_t *r, int32_t *out,
                           const rmq_opts *opts, void *stream) {
    if (H < 0 || (H > 0 && !arrays)) return RMQ_ERR_INVALID_ARG;
    uint32_t flags = 0;
    int32_t kforce = 0;
    if (opts) {
        if (opts->flags & ~(int32_t)RMQ_FLAG_TEST_WITHHOLD_READY) return RMQ_ERR_INVALID_ARG;
        if (opts->k != 0 && (!pow2_in_range(opts->k) || opts->k > (1 << multi_max_logk()))) return RMQ_ERR_INVALID_ARG;
        flags = (uint32_t)opts->flags;
        kforce = opts->k;
    }
    int64_t qtot = 0;
    for (int32_t h = 0; h < H; ++h) {
        const rmq_array &a = arrays[h];
        if (a.q < 0 || a.q > kMaxQ || a.n < 0 || a.n > kMaxN) return RMQ_ERR_INVALID_ARG;
        if (a.q > 0 && (a.n < 1 || !a.A)) return RMQ_ERR_INVALID_ARG;
        qtot += a.q;
    }
    if (qtot > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (qtot == 0) return RMQ_OK;
    if (!l || !r || !out) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    int64_t qoff = 0;
    for (int32_t g0 = 0; g0 < H; g0 += kMultiMax) {
        const int cnt = (int)std::min<int64_t>(kMultiMax, H - g0);
        const int32_t *Ap[kMultiMax];
        int64_t nn[kMultiMax], qq[kMultiMax];
        int32_t lk[kMultiMax];
        int64_t gq = 0;
        for (int i = 0; i < cnt; ++i) {
            const rmq_array &a = arrays[g0 + i];
            Ap[i] = a.A;
            nn[i] = a.q > 0 ? a.n : 0;
            qq[i] = a.q;
            lk[i] = a.q > 0 ? (kforce ? ilog2_host((uint64_t)kforce) : multi_logk(a.n)) : MIN_LOGK;
            gq += a.q;
        }
        if (gq > 0) {
            Workspace ws;
            rmq_status st = ws.alloc(multi_workspace_bytes(nn, qq, lk, cnt), s);
            if (st != RMQ_OK) return st;
            cudaError_t e = launch_multi(Ap, nn, qq, lk, cnt, l + qoff, r + qoff, out + qoff, flags, ws.p, s);
            if (e != cudaSuccess) return cuda_status(e);
        }
        qoff += gq;
    }
    return RMQ_OK;
}

rmq_status rmq_build(const int32_t *A, int64_t n, const rmq_opts *opts, void *stream, rmq_handle *out_handle) {
    if (!out_handle) return RMQ_ERR_INVALID_ARG;
    *out_handle = nullptr;
    rmq_status st = check_batch_args(A, n, nullptr, nullptr, 0, nullptr, opts);
    if (st != RMQ_OK) return st;
    const rmq_opts o = resolve_opts(n, 0, opts);
    const int logk = ilog2_host((uint64_t)o.k);
    rmq_handle h = new (std::nothrow) rmq_handle_s();
    if (!h) return RMQ_ERR_OOM;
    h->A = A;
    h->n = n;
    h->logk = logk;
    h->nb = cdiv(n, 1ll << logk);
    const int64_t te = two_level_entries(h->nb);
    h->bytes = handle_bytes_for(n, logk);
    cudaGetDevice(&h->device);
    cudaError_t e = cudaMalloc(&h->T, (size_t)h->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return e == cudaErrorMemoryAllocation ? RMQ_ERR_OOM : RMQ_ERR_CUDA;
    }
    cudaStream_t s = as_stream(stream);
    h->Cs = h->T + te;
    if ((e = launch_block_minima_i32(A, n, logk, h->T, s)) != cudaSuccess ||
        (e = launch_sparse_table(h->T, Len{n, nullptr}, logk, h->nb, s, true, h->Cs)) != cudaSuccess) {
        cudaFree(h->T);
        delete h;
        return cuda_status(e);
    }
    *out_handle = h;
    return RMQ_OK;
}

rmq_status rmq_query(rmq_handle h, const int32_t *l, const int32_t *r, int64_t q, int32_t *out, void *stream) {
    if (!h || q < 0 || q > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (q == 0) return RMQ_OK;
    if (!l || !r || !out) return RMQ_ERR_INVALID_ARG;
    return cuda_status(launch_query_plain(h->A, h->n, h->logk, h->T, h->Cs, l, r, q, out, as_stream(stream)));
}

rmq_status rmq_query_host(rmq_handle h, const int32_t *l_host, const int32_t *r_host, int64_t q, int32_t *out_host,
                          void *stream) {
    if (!h || q < 0 || q > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (q == 0) return RMQ_OK;
    if (!l_host || !r_host || !out_host) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const size_t bq = (size_t)q * 4, pad = (bq + 255) & ~(size_t)255;
    {
        Workspace ws;
        rmq_status st = ws.alloc(3 * pad, s);
        if (st != RMQ_OK) return st;
        char *base = static_cast<char *>(ws.p);
        int32_t *dl = reinterpret_cast<int32_t *>(base), *dr = reinterpret_cast<int32_t *>(base + pad),
                *dout = reinterpret_cast<int32_t *>(base + 2 * pad);
        cudaError_t e;
        if ((e = cudaMemcpyAsync(dl, l_host, bq, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaMemcpyAsync(dr, r_host, bq, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_status(e);
        if ((st = rmq_query(h, dl, dr, q, dout, stream)) != RMQ_OK) return st;
        if ((e = cudaMemcpyAsync(out_host, dout, bq, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_status(e);
    }
    return rmq_stream_status(stream);
}

rmq_status rmq_query_multi(const rmq_handle *hs, const int64_t *q_counts, int32_t H, const int32_t *l,
                           const int32_t *r, int32_t *out, void *stream) {
    if (H < 0 || (H > 0 && (!hs || !q_counts))) return RMQ_ERR_INVALID_ARG;
    int64_t qtot = 0;
    for (int32_t h = 0; h < H; ++h) {
        if (!hs[h] || q_counts[h] < 0 || q_counts[h] > kMaxQ) return RMQ_ERR_INVALID_ARG;
        qtot += q_counts[h];
    }
    if (qtot > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (qtot == 0) return RMQ_OK;
    if (!l || !r || !out) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    int64_t off = 0;
    std::vector<QueryReq> reqs;
    for (int32_t g0 = 0; g0 < H; g0 += kReqMax) {
        const int cnt = (int)std::min<int64_t>(kReqMax, H - g0);
        reqs.clear();
        int64_t gq = 0;
        for (int i = 0; i < cnt; ++i) {
            const rmq_handle h = hs[g0 + i];
            reqs.push_back(QueryReq{h->A, h->T, h->Cs, h->n, q_counts[g0 + i], h->logk});
            gq += q_counts[g0 + i];
        }
        if (gq > 0) {
            cudaError_t e = launch_query_handles(reqs.data(), cnt, l + off, r + off, out + off, s);
            if (e != cudaSuccess) return cuda_status(e);
        }
        off += gq;
    }
    return RMQ_OK;
}

int64_t rmq_handle_bytes(rmq_handle h) { return h ? h->bytes : 0; }

int32_t rmq_handle_k(rmq_handle h) { return h ? (int32_t)(1 << h->logk) : 0; }

void rmq_free(rmq_handle h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaFree(h->T);
    if (cur != h->device) cudaSetDevice(cur);
    delete h;
}

rmq_status rmq_stream_status(void *stream) {
    cudaStream_t s = as_stream(stream);
    unsigned *p = err_word_ptr(s);
    if (!p) return RMQ_ERR_CUDA;
    // read and clear the stream's own word in the stream's order, after its work
    unsigned w = 0;
    if (cudaMemcpyAsync(&w, p, sizeof(w), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RMQ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RMQ_ERR_CUDA;
    if (w) {
        if (cudaMemsetAsync(p, 0, sizeof(w), s) != cudaSuccess) return RMQ_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return RMQ_ERR_CUDA;
    }
    if (w & ERR_TIMEOUT) return RMQ_ERR_TIMEOUT;
    if (w & ERR_QUERY_RANGE) return RMQ_ERR_QUERY_RANGE;
    return RMQ_OK;
}

const char *rmq_strerror(rmq_status s) {
    switch (s) {
        case RMQ_OK: return "ok";
        case RMQ_ERR_INVALID_ARG: return "invalid argument (pointer, size or option)";
        case RMQ_ERR_QUERY_RANGE: return "a query had l < 0, r >= n or l > r (its answer is -1)";
        case RMQ_ERR_OOM: return "out of device memory";
        case RMQ_ERR_CUDA: return "a CUDA runtime call failed";
        case RMQ_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case RMQ_ERR_BUDGET: return "the memory budget would be exceeded";
        case RMQ_ERR_SCRATCH_LIMIT: return "the table does not fit the fixed buffer of rmq_batch_noalloc";
    }
    return "unknown status";
}

int64_t rmq_table_bytes(int64_t n, int32_t k) {
    if (n <= 0 || n > kMaxN || !pow2_in_range(k)) return -1;
    return table_entries(n, ilog2_host((uint64_t)k)) * 8;
}

rmq_status rmq_batch_lary(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                          int32_t k, int32_t ell, void *stream) {
    if (check_batch_args(A, n, l, r, q, out, nullptr) != RMQ_OK) return RMQ_ERR_INVALID_ARG;
    if (!pow2_in_range(k) || ell < 2 || ell > 256 || (ell & (ell - 1))) return RMQ_ERR_INVALID_ARG;
    const int logk = ilog2_host((uint64_t)k), logell = ilog2_host((uint64_t)ell);
    const int64_t nb = cdiv(n, 1ll << logk);
    cudaStream_t s = as_stream(stream);
    Workspace ws;
    rmq_status st = ws.alloc((size_t)(lary_levels(nb, logell) * nb) * 8, s);
    if (st != RMQ_OK) return st;
    return cuda_status(run_lary(A, n, logk, logell, l, r, q, out, static_cast<uint64_t *>(ws.p), s));
}

// Block sizes of the multi-level layout: logk[1 .. h] from ks[0 .. h-1];
// false when they break the rules of rmq_batch_hlevel.
static bool hlevel_logks(const int32_t *ks, int32_t h, int *logk) {
    if (!ks || h < 1 || h > kHLevelMax) return false;
    for (int i = 0; i < h; ++i) {
        const int32_t k = ks[i];
        if (k < 1 || (k & (k - 1))) return false;
        logk[i + 1] = ilog2_host((uint64_t)k);
        if (i == 0 ? (logk[1] < MIN_LOGK || logk[1] > MAX_LOGK) : (logk[i + 1] <= logk[i] || logk[i + 1] > kHLevelMaxLogK))
            return false;
    }
    return true;
}

int64_t rmq_hlevel_bytes(int64_t n, const int32_t *ks, int32_t h) {
    int logk[kHLevelMax + 1];
    if (n <= 0 || n > kMaxN || !hlevel_logks(ks, h, logk)) return -1;
    return hlevel_entries(n, logk, h) * 8;
}

rmq_status rmq_batch_hlevel(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                            const int32_t *ks, int32_t h, void *stream) {
    if (check_batch_args(A, n, l, r, q, out, nullptr) != RMQ_OK) return RMQ_ERR_INVALID_ARG;
    int logk[kHLevelMax + 1];
    if (!hlevel_logks(ks, h, logk)) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    Workspace ws;
    rmq_status st = ws.alloc((size_t)hlevel_entries(n, logk, h) * 8, s);
    if (st != RMQ_OK) return st;
    return cuda_status(run_hlevel(A, n, logk, h, l, r, q, out, static_cast<uint64_t *>(ws.p), s));
}

rmq_status rmq_hlevel_paper_ks(int64_t n, int32_t h, int32_t *ks_out) {
    if (!ks_out || n < 2 || n > kMaxN || h < 2 || h > kHLevelMax) return RMQ_ERR_INVALID_ARG;
    const double lg = std::log2((double)n), sq = std::sqrt((double)n);
    int prev = 0;
    for (int i = 1; i <= h; ++i) {
        const double e = (double)(i - 1) / (h - 1) - 1.0 / (h + 1);
        int t = pow2_log_near(sq * std::pow(lg, e), i == 1 ? MIN_LOGK : 1, i == 1 ? MAX_LOGK : kHLevelMaxLogK);
        if (i > 1 && t <= prev) t = prev + 1;
        if (t > kHLevelMaxLogK) return RMQ_ERR_INVALID_ARG;
        ks_out[i - 1] = 1 << t;
        prev = t;
    }
    return RMQ_OK;
}

int64_t rmq_batch_workspace_bytes(int64_t n, int64_t q, const rmq_opts *opts) {
    int32_t dummy = 0;
    if (check_batch_args(&dummy, n, &dummy, &dummy, q, &dummy, opts) != RMQ_OK) return -1;
    if (q == 0) return 0;
    const rmq_opts o = resolve_opts(n, q, opts);
    if (o.variant == RMQ_VARIANT_CONTRACTED) return (int64_t)con_workspace_bytes(n, q, ilog2_host((uint64_t)o.k_con));
    if (o.k1 > o.k) return -1;
    const int logk = ilog2_host((uint64_t)o.k);
    return plain_workspace_bytes(n, logk, logk1_of(o.k1, logk));
}

// The tuner: a choice measured by rmq_autotune for this (n, q) shape when
// there is one; otherwise the plain form over A with k near sqrt(n)/8 (a few
// extra reads per query against a table that stays small next to A), and,
// for the contracted form, k_con near sqrt(2q) capped at the paper's default
// 512.
rmq_status rmq_tune(int64_t n, int64_t q, rmq_opts *out) {
    if (!out || n <= 0) return RMQ_ERR_INVALID_ARG;
    if (q > 0) {   // a measured choice for this shape (the lowest width class if several)
        const int st = tuned_lookup(n, q, -1, out);
        if (st == TUNE_FOUND || (st == TUNE_AMBIGUOUS && tuned_lookup(n, q, 0, out) == TUNE_FOUND)) return RMQ_OK;
    }
    out->variant = RMQ_VARIANT_PLAIN;
    out->k = 1 << pow2_log_near(std::sqrt((double)n) / 8.0, MIN_LOGK, 12);
    out->k_con = 1 << pow2_log_near(std::sqrt(2.0 * (double)std::max<int64_t>(q, 1)), MIN_LOGK, 9);
    out->flags = 0;
    out->threads_per_query = 0;
    out->k1 = 0;
    return RMQ_OK;
}

rmq_status rmq_tune_batch(const int32_t *l, const int32_t *r, int64_t q, int64_t n, void *stream, rmq_opts *out) {
    if (!out || n <= 0 || n > kMaxN || q < 0 || q > kMaxQ || (q > 0 && (!l || !r))) return RMQ_ERR_INVALID_ARG;
    *out = resolve_opts(n, q, nullptr, l, r, as_stream(stream));
    return RMQ_OK;
}

rmq_status rmq_block_minima(const int32_t *A, int64_t n, int32_t k, uint64_t *T0, void *stream) {
    if (!A || !T0 || n <= 0 || n > kMaxN || !pow2_in_range(k)) return RMQ_ERR_INVALID_ARG;
    return cuda_status(launch_block_minima_i32(A, n, ilog2_host((uint64_t)k), T0, as_stream(stream)));
}

rmq_status rmq_sparse_table_build(uint64_t *T, int64_t nb, void *stream) {
    if (!T || nb <= 0 || nb > kMaxN) return RMQ_ERR_INVALID_ARG;
    return cuda_status(launch_sparse_table(T, Len{nb, nullptr}, 0, nb, as_stream(stream)));
}

rmq_status rmq_sort_endpoints(const int32_t *l, const int32_t *r, int64_t q, int64_t n, uint32_t *pos_out,
                              uint32_t *tag_out, void *stream) {
    if (n <= 0 || n > kMaxN || q < 0 || q > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (q == 0) return RMQ_OK;
    if (!l || !r || !pos_out || !tag_out) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    Workspace ws;
    const size_t bytes = sort_workspace_bytes(q);
    rmq_status st = ws.alloc(bytes, s);
    if (st != RMQ_OK) return st;
    return cuda_status(sort_endpoints(l, r, q, n, pos_out, tag_out, ws.p, bytes, s));
}

rmq_status rmq_rank_endpoints(const uint32_t *pos_sorted, const uint32_t *tag_sorted, int64_t q, uint32_t *P_out,
                              int64_t *m_dev, int32_t *rank_l, int32_t *rank_r, void *stream) {
    if (q < 0 || q > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (!m_dev) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (q == 0) return cuda_status(cudaMemsetAsync(m_dev, 0, sizeof(int64_t), s));
    if (!pos_sorted || !tag_sorted || !P_out || !rank_l || !rank_r) return RMQ_ERR_INVALID_ARG;
    Workspace ws;
    rmq_status st = ws.alloc(rank_workspace_bytes(q), s);
    if (st != RMQ_OK) return st;
    return cuda_status(rank_endpoints(pos_sorted, tag_sorted, q, P_out, m_dev, rank_l, rank_r, ws.p, s));
}

rmq_status rmq_endpoint_bitmap(const int32_t *l, const int32_t *r, int64_t q, int64_t n, uint32_t *BP,
                               int64_t *m_dev, void *stream) {
    if (!BP || !m_dev || n <= 0 || n > kMaxN || q < 0 || q > kMaxQ) return RMQ_ERR_INVALID_ARG;
    if (q > 0 && (!l || !r)) return RMQ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(BP) & 3) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    Workspace ws;
    rmq_status st = ws.alloc(endpoint_bitmap_workspace_bytes(n), s);
    if (st != RMQ_OK) return st;
    return cuda_status(endpoint_bitmap(l, r, q, n, BP, BP + bitmap_entries(n), m_dev, nullptr, ws.p, s));
}

rmq_status rmq_contract(const int32_t *A, int64_t n, const uint32_t *P, const int64_t *m_dev, int64_t m_max,
                        uint64_t *AQ, void *stream) {
    if (!A || !P || !m_dev || !AQ || n <= 0 || n > kMaxN || m_max < 0) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    Workspace ws;
    rmq_status st = ws.alloc(contract_workspace_bytes(n), s);
    if (st != RMQ_OK) return st;
    return cuda_status(contract(A, n, P, m_dev, m_max, AQ, ws.p, s));
}

}  // extern "C"
#pragma GCC visibility pop
