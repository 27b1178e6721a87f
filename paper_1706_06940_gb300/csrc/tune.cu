// tune.cu -- the autotuner: measures block sizes, both forms, the lanes per
// partial-block scan and the small-block size of the two-level layout on a
// batch, keeps the fastest choice per batch shape, and lets rmq_tune and the
// AUTO batch calls answer from those measurements (the automated selection
// of k that the paper leaves open, Sec. 5).
//
// A shape is (round(log2 n), round(log2 q), width class), the width class
// being round(log2 of the median query width r - l + 1) over a sample of the
// batch: a uniform batch and a batch of short ranges of the same n and q are
// tuned and remembered apart.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "rmq_internal.cuh"

namespace rmq {
namespace {

std::mutex g_tune_mu;
// (round(log2 n), round(log2 q)) -> width class -> choice; width class -1 is
// a choice loaded without one (it serves every width class of the shape)
std::map<std::pair<int, int>, std::map<int, rmq_opts>> g_tuned;

// Reads `vecs` 16-byte vectors (their values do not matter) so that L2 holds
// this buffer's clean lines and none of a batch's; the xor of what it read
// is stored only in the impossible case that it equals the buffer's address.
__global__ void k_l2_evict(const int4 *__restrict__ p, int64_t vecs, int4 *sink) {
    unsigned acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < vecs; i += (int64_t)gridDim.x * blockDim.x) {
        int4 v;
        asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p + i));
        acc ^= (unsigned)(v.x ^ v.y ^ v.z ^ v.w);
    }
    if (acc == (unsigned)reinterpret_cast<uintptr_t>(p) && threadIdx.x == 0) sink->x = (int)acc;
}

std::pair<int, int> shape_key(int64_t n, int64_t q) {
    auto lg = [](int64_t x) { return (int)std::lround(std::log2((double)x)); };   // nearest log2
    return {lg(std::max<int64_t>(n, 1)), lg(std::max<int64_t>(q, 1))};
}

// The entry of `byw` for width class w: the same class, else the class-less
// entry, else the nearest class.
const rmq_opts *pick_width(const std::map<int, rmq_opts> &byw, int w) {
    auto it = byw.find(w);
    if (it != byw.end()) return &it->second;
    auto any = byw.find(-1);
    if (any != byw.end()) return &any->second;
    const rmq_opts *best = nullptr;
    int dist = 1 << 30;
    for (auto &kv : byw)
        if (std::abs(kv.first - w) < dist) {
            dist = std::abs(kv.first - w);
            best = &kv.second;
        }
    return best;
}

}  // namespace

int width_class_of(const int32_t *l, const int32_t *r, int64_t count, int64_t n) {
    std::vector<int64_t> w;
    w.reserve((size_t)count);
    for (int64_t i = 0; i < count; ++i)
        if (l[i] >= 0 && r[i] >= l[i] && (int64_t)r[i] < n) w.push_back((int64_t)r[i] - l[i] + 1);
    if (w.empty()) return 0;
    std::nth_element(w.begin(), w.begin() + w.size() / 2, w.end());
    return (int)std::lround(std::log2((double)w[w.size() / 2]));
}

int sample_width_class(const int32_t *l, const int32_t *r, int64_t q, int64_t n, cudaStream_t s) {
    // 128 queries from the start of the batch and 128 from its middle
    const int64_t half = std::min<int64_t>(q, kWidthSample / 2);
    const int64_t mid = q / 2 + half <= q ? q / 2 : q - half;
    int32_t hl[kWidthSample], hr[kWidthSample];
    if (cudaMemcpyAsync(hl, l, half * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hr, r, half * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hl + half, l + mid, half * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hr + half, r + mid, half * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return width_class_of(hl, hr, 2 * half, n);
}

int tuned_lookup(int64_t n, int64_t q, int wclass, rmq_opts *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(shape_key(n, q));
    if (it == g_tuned.end() || it->second.empty()) return TUNE_NONE;
    if (wclass < 0) {
        if (it->second.size() > 1) return TUNE_AMBIGUOUS;
        *out = it->second.begin()->second;
        return TUNE_FOUND;
    }
    *out = *pick_width(it->second, wclass);
    return TUNE_FOUND;
}

}  // namespace rmq

using namespace rmq;
#pragma GCC visibility push(default)
extern "C" {

rmq_status rmq_autotune(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q, int32_t *out,
                        int32_t variant, int32_t k_min, int32_t k_max, void *stream, rmq_opts *best,
                        float *best_ms) {
    if (!best || variant < RMQ_VARIANT_AUTO || variant > RMQ_VARIANT_CONTRACTED) return RMQ_ERR_INVALID_ARG;
    if (k_min == 0) k_min = 32;
    if (k_max == 0) k_max = 4096;
    if (k_min < 32 || k_max > 65536 || k_min > k_max || (k_min & (k_min - 1)) || (k_max & (k_max - 1)))
        return RMQ_ERR_INVALID_ARG;
    if (!A || n <= 0 || q <= 0 || !l || !r || !out) return RMQ_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int wclass = std::max(0, sample_width_class(l, r, q, n, s));
    // every timed run starts from an L2 holding none of the batch, as a call
    // on fresh data does: a read of twice the L2 size evicts it and leaves
    // only clean lines (skipped if that buffer cannot be had)
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const size_t flush_bytes = 2 * (size_t)std::max(l2, 0);
    void *flush = nullptr;
    if (flush_bytes && cudaMallocAsync(&flush, flush_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        flush = nullptr;
    }
    if (flush && cudaMemsetAsync(flush, 0, flush_bytes, s) != cudaSuccess) {   // no read of unset memory
        cudaGetLastError();
        cudaFreeAsync(flush, s);
        flush = nullptr;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (flush) cudaFreeAsync(flush, s);
        return RMQ_ERR_CUDA;
    }
    // best of three timed runs after one untimed run (which warms the pool)
    auto time_opts = [&](const rmq_opts &o, float &ms) -> rmq_status {
        ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            if (flush) {
                k_l2_evict<<<(unsigned)(dev_info().sms * 8), 256, 0, s>>>(static_cast<const int4 *>(flush),
                                                                         (int64_t)(flush_bytes / 16),
                                                                         static_cast<int4 *>(flush));
                note_launches(1);
            }
            cudaEventRecord(e0, s);
            const rmq_status st = rmq_batch_ex(A, n, l, r, q, out, &o, stream);
            cudaEventRecord(e1, s);
            if (st != RMQ_OK) return st;
            if (cudaEventSynchronize(e1) != cudaSuccess) return RMQ_ERR_CUDA;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);
        }
        return RMQ_OK;
    };
    rmq_opts win{RMQ_VARIANT_PLAIN, k_min, 512, 0, 0, 0};
    float win_ms = 1e30f;
    rmq_status st = RMQ_OK;
    // the form and its block size
    for (int form = RMQ_VARIANT_PLAIN; form <= RMQ_VARIANT_CONTRACTED && st == RMQ_OK; ++form) {
        if (variant != RMQ_VARIANT_AUTO && variant != form) continue;
        for (int32_t k = k_min; k <= k_max && st == RMQ_OK; k *= 2) {
            const rmq_opts o{form, form == RMQ_VARIANT_PLAIN ? k : 0, form == RMQ_VARIANT_CONTRACTED ? k : 0, 0, 0, 0};
            float ms;
            st = time_opts(o, ms);
            if (st == RMQ_OK && ms < win_ms) {
                win_ms = ms;
                win = o;
            }
        }
    }
    // the lanes that scan one partial block (threads per query of phase B)
    const rmq_opts base = win;
    for (int32_t tpq : {16, 32}) {
        if (st != RMQ_OK) break;
        rmq_opts o = base;
        o.threads_per_query = tpq;
        float ms;
        st = time_opts(o, ms);
        if (st == RMQ_OK && ms < win_ms) {
            win_ms = ms;
            win = o;
        }
    }
    // the small blocks of the two-level layout (plain form, Sec. 3.3)
    if (win.variant == RMQ_VARIANT_PLAIN) {
        const rmq_opts base1 = win;
        for (int32_t k1 : {-1, 32, 64, 128, 256, 512}) {
            if (st != RMQ_OK) break;
            if (k1 > 0 && (k1 > base1.k / 2 || (k1 == 128 && base1.k >= 128))) continue;   // 128: the default
            if (k1 < 0 && base1.k < 128) continue;                                       // none: the default
            rmq_opts o = base1;
            o.k1 = k1;
            float ms;
            st = time_opts(o, ms);
            if (st == RMQ_OK && ms < win_ms) {
                win_ms = ms;
                win = o;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (flush) cudaFreeAsync(flush, s);
    if (st != RMQ_OK) return st;
    // remember the winner; both block sizes are filled in for later calls
    rmq_opts fill;
    rmq_tune(n, q, &fill);
    if (win.k == 0) win.k = fill.k;
    if (win.k_con == 0) win.k_con = fill.k_con;
    if (variant == RMQ_VARIANT_AUTO) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[shape_key(n, q)][wclass] = win;
    }
    *best = win;
    if (best_ms) *best_ms = win_ms;
    return RMQ_OK;
}

rmq_status rmq_tune_save(const char *path) {
    if (!path) return RMQ_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) return RMQ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::fprintf(f, "# log2n log2q wclass variant k k_con threads_per_query k1\n");
    for (auto &shape : g_tuned)
        for (auto &kv : shape.second)
            std::fprintf(f, "%d %d %d %d %d %d %d %d\n", shape.first.first, shape.first.second, kv.first,
                         kv.second.variant, kv.second.k, kv.second.k_con, kv.second.threads_per_query, kv.second.k1);
    std::fclose(f);
    return RMQ_OK;
}

rmq_status rmq_tune_load(const char *path) {
    if (!path) return RMQ_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return RMQ_ERR_INVALID_ARG;
    char line[256];
    std::vector<std::tuple<int, int, int, rmq_opts>> t;
    rmq_status st = RMQ_OK;
    auto pow2 = [](int x) { return x >= 32 && x <= 65536 && (x & (x - 1)) == 0; };
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int a, b, w, v, k, kc, tpq = 0, k1 = 0;
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d", &a, &b, &w, &v, &k, &kc, &tpq, &k1);
        if (got == 5) {   // "log2n log2q variant k k_con": a choice without a width class
            std::sscanf(line, "%d %d %d %d %d", &a, &b, &v, &k, &kc);
            w = -1; tpq = 0; k1 = 0;
        } else if (got != 8) {
            st = RMQ_ERR_INVALID_ARG;
            break;
        }
        if (v < 1 || v > 2 || !pow2(k) || !pow2(kc) || w < -1 || (tpq != 0 && tpq != 8 && tpq != 16 && tpq != 32) ||
            (k1 != 0 && k1 != -1 && (!pow2(k1) || k1 > k))) {
            st = RMQ_ERR_INVALID_ARG;
            break;
        }
        t.emplace_back(a, b, w, rmq_opts{v, k, kc, 0, tpq, k1});
    }
    std::fclose(f);
    if (st != RMQ_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &e : t) g_tuned[{std::get<0>(e), std::get<1>(e)}][std::get<2>(e)] = std::get<3>(e);
    return RMQ_OK;
}

void rmq_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

}  // extern "C"
#pragma GCC visibility pop
