// lary.cu -- the l-ary generalisation of the block sparse table (Sec. 3.1,
// the variant the paper describes but does not implement).  Level t holds,
// for block j, the minimum over the l^t consecutive blocks from j (level 0:
// the block minima of step 3), so the inner span of a query is covered by at
// most l values of one level instead of two values of a binary table, and
// the table has floor(log_l nb) + 1 levels instead of floor(log2 nb) + 1.
// This first GPU path builds one level per launch and answers one query per
// thread.
#include <algorithm>

#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kThreads = 256;

// Level t (spans of l^t blocks) from level t - 1 (spans of span_prev =
// l^(t-1)): entry j is the minimum of the l entries j, j + span_prev, ...,
// j + (l - 1) span_prev of the level below.  Only the starts whose span ends
// inside the block range are written.
__global__ void __launch_bounds__(kThreads) k_lary_level(uint64_t *__restrict__ T, int64_t nb, int t,
                                                         int64_t span_prev, int ell) {
    pdl_wait();
    const unsigned long long *prev = reinterpret_cast<const unsigned long long *>(T) + (int64_t)(t - 1) * nb;
    uint64_t *cur = T + (int64_t)t * nb;
    const int64_t cnt = nb - span_prev * ell + 1;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t m = __ldg(prev + j);
        for (int i = 1; i < ell; ++i) m = kmin(m, __ldg(prev + j + i * span_prev));
        cur[j] = m;
    }
}

// Minimum key over A[lo .. hi], by one thread.
__device__ __forceinline__ uint64_t thread_scan(const int32_t *__restrict__ A, int64_t lo, int64_t hi) {
    uint64_t m = KEY_MAX;
    for (int64_t i = lo; i <= hi; ++i) m = kmin(m, make_key(__ldg(A + i), (uint32_t)i));
    return m;
}

// One thread per query, in the steps of Sec. 3.1 step 4.  The inner span of
// blocks bl+1 .. br-1 (length len) is covered by spans of the level t =
// floor(log_l len), placed from bl+1 and then one more ending at br-1, so at
// most l table values are read.  An end block whose minimum beats the inner
// span's is taken when that minimum lies inside the query (R5); otherwise
// its part of the query is scanned.  Invalid queries answer -1 and raise the
// error word.
__global__ void __launch_bounds__(kThreads) k_lary_query(const int32_t *__restrict__ A, int64_t n, int logk,
                                                         int logell, int levels, const uint64_t *__restrict__ T,
                                                         int64_t nb, const int32_t *__restrict__ L,
                                                         const int32_t *__restrict__ R, int64_t q,
                                                         int32_t *__restrict__ out, unsigned *err) {
    pdl_wait();
    const unsigned long long *Tu = reinterpret_cast<const unsigned long long *>(T);
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = L[i], r = R[i];
        if (l < 0 || r < l || (int64_t)r >= n) {
            out[i] = -1;
            bad = true;
            continue;
        }
        const int64_t bl = (int64_t)l >> logk, br = (int64_t)r >> logk;
        uint64_t best;
        if (bl == br) {
            best = thread_scan(A, l, r);
        } else {
            best = KEY_MAX;
            if (br - bl >= 2) {
                const int64_t a = bl + 1, b = br - 1, len = b - a + 1;
                int t = 0;
                while (t + 1 < levels && ((int64_t)1 << ((t + 1) * logell)) <= len) ++t;
                const int64_t span = (int64_t)1 << (t * logell);
                const unsigned long long *row = Tu + (int64_t)t * nb;
                for (int64_t s0 = a;; s0 += span) {
                    const int64_t start = s0 + span - 1 <= b ? s0 : b - span + 1;   // the last ends at b
                    best = kmin(best, __ldg(row + start));
                    if (start + span - 1 >= b) break;
                }
            }
            const uint64_t tl = __ldg(Tu + bl);
            if (tl < best)
                best = key_pos(tl) >= (uint32_t)l ? tl : kmin(best, thread_scan(A, l, ((bl + 1) << logk) - 1));
            const uint64_t tr = __ldg(Tu + br);
            if (tr < best)
                best = key_pos(tr) <= (uint32_t)r ? tr : kmin(best, thread_scan(A, br << logk, r));
        }
        out[i] = (int32_t)key_pos(best);
    }
    if (bad) atomicOr(err, ERR_QUERY_RANGE);
}

}  // namespace

int lary_levels(int64_t nb, int logell) {
    if (nb < 1) return 0;
    int lv = 1;
    for (int64_t span = (int64_t)1 << logell; span <= nb; span <<= logell) ++lv;
    return lv;
}

cudaError_t run_lary(const int32_t *A, int64_t n, int logk, int logell, const int32_t *l, const int32_t *r,
                     int64_t q, int32_t *out, uint64_t *T, cudaStream_t s) {
    const int64_t nb = cdiv(n, (int64_t)1 << logk);
    const int levels = lary_levels(nb, logell);
    const DevInfo di = dev_info();
    unsigned *err = err_word_ptr(s);
    if (!err) return cudaErrorUnknown;
    cudaError_t e = launch_block_minima_i32(A, n, logk, T, s);
    if (e != cudaSuccess) return e;
    for (int t = 1; t < levels; ++t) {
        const int64_t span_prev = (int64_t)1 << ((t - 1) * logell);
        const int64_t cnt = nb - (span_prev << logell) + 1;
        const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(cnt, kThreads), (int64_t)di.sms * 8));
        launch_pdl(k_lary_level, (unsigned)ctas, kThreads, 0, s, T, nb, t, span_prev, 1 << logell);
        note_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (q <= 0) return cudaSuccess;
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(q, kThreads), (int64_t)di.sms * 8));
    launch_pdl(k_lary_query, (unsigned)ctas, kThreads, 0, s, A, n, logk, logell, levels, T, nb, l, r, q, out, err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rmq
