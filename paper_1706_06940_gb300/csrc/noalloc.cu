// noalloc.cu -- rmq_batch_noalloc: the plain BbST batch for callers that may
// not allocate device memory.  Its only scratch, the sparse table over the
// block minima, lives in a fixed buffer of this library's device image, so a
// call issues kernel launches and nothing else.
#include <mutex>

#include "rmq_internal.cuh"

namespace rmq {

namespace {

// The fixed buffer: RMQ_NOALLOC_TABLE_ENTRIES packed keys for the table (4 MiB)
// followed by the table's coarse summary (kCoarseCap keys, 32 KiB).  It exists
// on every GPU on which the library is loaded, for the life of the process,
// and all calls on a device share it.
static __device__ __align__(256) unsigned long long g_noalloc_table[RMQ_NOALLOC_TABLE_ENTRIES + kCoarseCap];

constexpr int kMaxDev = 64;
std::mutex g_noalloc_mu;
uint64_t *g_noalloc_ptr[kMaxDev];

// In host code `g_noalloc_table` names a host-side stand-in, not device
// memory, so kernels must be given the address the runtime reports for the
// current device.  Looked up once per device, with that device current.
cudaError_t noalloc_table(uint64_t **out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[d]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_table);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[d] = static_cast<uint64_t *>(p);
    }
    *out = g_noalloc_ptr[d];
    return cudaSuccess;
}

bool noalloc_k_ok(int32_t k) {
    return k >= (1 << MIN_LOGK) && k <= (1 << MAX_LOGK) && (k & (k - 1)) == 0;
}

int64_t noalloc_entries(int64_t n, int logk) {
    const int64_t nb = cdiv(n, 1ll << logk);
    return nb * (ilog2_host((uint64_t)nb) + 1);
}

}  // namespace

}  // namespace rmq

using namespace rmq;

#pragma GCC visibility push(default)
extern "C" rmq_status rmq_batch_noalloc(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                                        int32_t *out, int32_t k, void *stream) {
    if (!A || n <= 0 || n > 2147483647ll || q < 0 || q > 2147483647ll) return RMQ_ERR_INVALID_ARG;
    if (q > 0 && (!l || !r || !out)) return RMQ_ERR_INVALID_ARG;
    if (k != 0 && !noalloc_k_ok(k)) return RMQ_ERR_INVALID_ARG;
    int logk;
    if (k != 0) {
        logk = ilog2_host((uint64_t)k);
        if (noalloc_entries(n, logk) > RMQ_NOALLOC_TABLE_ENTRIES) return RMQ_ERR_SCRATCH_LIMIT;
    } else {
        rmq_opts t;
        if (rmq_tune(n, q, &t) != RMQ_OK) return RMQ_ERR_INVALID_ARG;
        logk = ilog2_host((uint64_t)t.k);
        while (logk <= MAX_LOGK && noalloc_entries(n, logk) > RMQ_NOALLOC_TABLE_ENTRIES) ++logk;
        if (logk > MAX_LOGK) return RMQ_ERR_SCRATCH_LIMIT;
    }
    // the buffer's address on this device (the first call per device looks it
    // up, which loads this module and commits the buffer); q == 0 does only that
    uint64_t *T = nullptr;
    if (noalloc_table(&T) != cudaSuccess) return RMQ_ERR_CUDA;
    if (q == 0) return RMQ_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nb = cdiv(n, 1ll << logk);
    // Every table entry the queries read is written by these launches first,
    // so the buffer needs no clearing between calls.
    if (launch_block_minima_i32(A, n, logk, T, s) != cudaSuccess) return RMQ_ERR_CUDA;
    uint64_t *Cs = T + RMQ_NOALLOC_TABLE_ENTRIES;
    if (launch_sparse_table(T, Len{n, nullptr}, logk, nb, s, true, Cs) != cudaSuccess) return RMQ_ERR_CUDA;
    if (launch_query_plain(A, n, logk, T, Cs, l, r, q, out, s) != cudaSuccess) return RMQ_ERR_CUDA;
    return RMQ_OK;
}
#pragma GCC visibility pop
