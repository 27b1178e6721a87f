// tune.cu -- the autotuner: measures block sizes and both forms on a batch,
// keeps the fastest choice per (n, q) shape, and lets rmq_tune answer from
// those measurements (the automated selection of k that the paper leaves
// open, Sec. 5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include "rmq_internal.cuh"

namespace rmq {
namespace {

std::mutex g_tune_mu;
std::map<std::pair<int, int>, rmq_opts> g_tuned;   // (round(log2 n), round(log2 q)) -> choice

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

}  // namespace

bool tuned_lookup(int64_t n, int64_t q, rmq_opts *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(shape_key(n, q));
    if (it == g_tuned.end()) return false;
    *out = it->second;
    return true;
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
    rmq_opts win{RMQ_VARIANT_PLAIN, k_min, 512, 0};
    float win_ms = 1e30f;
    rmq_status st = RMQ_OK;
    for (int form = RMQ_VARIANT_PLAIN; form <= RMQ_VARIANT_CONTRACTED && st == RMQ_OK; ++form) {
        if (variant != RMQ_VARIANT_AUTO && variant != form) continue;
        for (int32_t k = k_min; k <= k_max && st == RMQ_OK; k *= 2) {
            rmq_opts o{form, form == RMQ_VARIANT_PLAIN ? k : 0, form == RMQ_VARIANT_CONTRACTED ? k : 0, 0};
            float ms = 1e30f;
            for (int rep = 0; rep < 4 && st == RMQ_OK; ++rep) {   // the first run warms the pool
                if (flush) {
                    k_l2_evict<<<(unsigned)(dev_info().sms * 8), 256, 0, s>>>(static_cast<const int4 *>(flush),
                                                                             (int64_t)(flush_bytes / 16),
                                                                             static_cast<int4 *>(flush));
                    note_launches(1);
                }
                cudaEventRecord(e0, s);
                st = rmq_batch_ex(A, n, l, r, q, out, &o, stream);
                cudaEventRecord(e1, s);
                if (st != RMQ_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) { st = RMQ_ERR_CUDA; break; }
                float t = 0;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);
            }
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
        g_tuned[shape_key(n, q)] = win;
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
    std::fprintf(f, "# log2n log2q variant k k_con\n");
    for (auto &kv : g_tuned)
        std::fprintf(f, "%d %d %d %d %d\n", kv.first.first, kv.first.second, kv.second.variant, kv.second.k,
                     kv.second.k_con);
    std::fclose(f);
    return RMQ_OK;
}

rmq_status rmq_tune_load(const char *path) {
    if (!path) return RMQ_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return RMQ_ERR_INVALID_ARG;
    char line[256];
    std::map<std::pair<int, int>, rmq_opts> t;
    rmq_status st = RMQ_OK;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int a, b, v, k, kc;
        if (std::sscanf(line, "%d %d %d %d %d", &a, &b, &v, &k, &kc) != 5 || v < 1 || v > 2 || k < 32 || k > 65536 ||
            (k & (k - 1)) || kc < 32 || kc > 65536 || (kc & (kc - 1))) {
            st = RMQ_ERR_INVALID_ARG;
            break;
        }
        t[{a, b}] = rmq_opts{v, k, kc, 0};
    }
    std::fclose(f);
    if (st != RMQ_OK) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : t) g_tuned[kv.first] = kv.second;
    return RMQ_OK;
}

void rmq_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
}

}  // extern "C"
#pragma GCC visibility pop
