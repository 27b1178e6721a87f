// query_plain.cu -- query answering of plain BbST (Sec. 3.1 step 4 over
// blocks of A, Sec. 3.2).
#include <algorithm>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

namespace {
constexpr int kThreads = 256;
}  // namespace

// ------------------------------------------------------------------ queries
// Four queries per thread: l and r come in as 16-byte vectors when aligned,
// every query issues its table reads before any is used, and the partial
// block scans are then drained warp-cooperatively.
namespace {

template <bool VECQ, bool VEC>
__global__ void __launch_bounds__(kThreads) k_query_plain(SrcI32 src, int64_t n, int logk,
                                                         const uint64_t *__restrict__ T, int64_t nb,
                                                         const int32_t *__restrict__ L, const int32_t *__restrict__ R,
                                                         int32_t *__restrict__ out, int64_t q, unsigned *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wb = warp * 128; wb < q; wb += nwarps * 128) {
        const int64_t base = wb + lane * 4;
        int32_t lq[4], rq[4];
        bool present[4];
        if (VECQ && base + 3 < q) {
            const int4 a = __ldcs(reinterpret_cast<const int4 *>(L + base));
            const int4 c = __ldcs(reinterpret_cast<const int4 *>(R + base));
            lq[0] = a.x; lq[1] = a.y; lq[2] = a.z; lq[3] = a.w;
            rq[0] = c.x; rq[1] = c.y; rq[2] = c.z; rq[3] = c.w;
#pragma unroll
            for (int i = 0; i < 4; ++i) present[i] = true;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                present[i] = base + i < q;
                lq[i] = present[i] ? __ldcs(L + base + i) : 0;
                rq[i] = present[i] ? __ldcs(R + base + i) : 0;
            }
        }
        uint64_t best[4];
        Pending pl[4], pr[4];
        bool hl[4], hr[4], ok[4];
        bool bad = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ok[i] = present[i] && lq[i] >= 0 && rq[i] >= lq[i] && (int64_t)rq[i] < n;
            bad |= present[i] && !ok[i];
            hl[i] = hr[i] = false;
            best[i] = KEY_MAX;
            if (ok[i]) best[i] = resolve_query(T, nb, logk, lq[i], rq[i], (uint32_t)lq[i], (uint32_t)rq[i], pl[i], pr[i], hl[i], hr[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            warp_drain_scans<SrcI32, VEC>(src, n, hl[i], pl[i], best[i]);
            warp_drain_scans<SrcI32, VEC>(src, n, hr[i], pr[i], best[i]);
        }
        int32_t o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = ok[i] ? (int32_t)key_pos(best[i]) : -1;
        if (VECQ && base + 3 < q) {
            __stcs(reinterpret_cast<int4 *>(out + base), make_int4(o[0], o[1], o[2], o[3]));
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (present[i]) out[base + i] = o[i];
        }
        if (bad) atomicOr(err, ERR_QUERY_RANGE);
    }
}

}  // namespace

cudaError_t launch_query_plain(const int32_t *A, int64_t n, int logk, const uint64_t *T, int64_t nb,
                               const int32_t *l, const int32_t *r, int64_t q, int32_t *out, cudaStream_t s) {
    if (q <= 0) return cudaSuccess;
    const DevInfo di = dev_info();
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(q, 128 * (kThreads / 32)), (int64_t)di.sms * 8));
    const bool vecq = ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    const bool vec = (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    unsigned *err = err_word_ptr();
    if (!err) return cudaErrorUnknown;
    SrcI32 src{A};
#define RMQ_LQ(VQ, V) k_query_plain<VQ, V><<<(unsigned)ctas, kThreads, 0, s>>>(src, n, logk, T, nb, l, r, out, q, err)
    if (vecq && vec) RMQ_LQ(true, true);
    else if (vecq) RMQ_LQ(true, false);
    else if (vec) RMQ_LQ(false, true);
    else RMQ_LQ(false, false);
#undef RMQ_LQ
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rmq
