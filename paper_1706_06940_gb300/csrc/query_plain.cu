// query_plain.cu -- query answering of plain BbST (Sec. 3.1 step 4 over
// blocks of A, Sec. 3.2, with the coarse level of Sec. 3.3).
#include <algorithm>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

// The kernel is the generic k_query_two of query.cuh over the int32 source.
cudaError_t launch_query_plain(const int32_t *A, int64_t n, int logk, const uint64_t *T, const uint64_t *Cs,
                               const int32_t *l, const int32_t *r, int64_t q, int32_t *out, cudaStream_t s,
                               const uint64_t *M1, int cap, unsigned long long *counts, int logk1, int max_teams) {
    if (q <= 0) return cudaSuccess;
    if (cap < 1 || cap > kCoarseCapMax || (Cs && cap != kCoarseCap)) return cudaErrorInvalidValue;
    if (M1 && (logk1 < MIN_LOGK || logk1 > logk)) return cudaErrorInvalidValue;
    if (max_teams != 1 && max_teams != 2 && max_teams != 4) return cudaErrorInvalidValue;
    const DevInfo di = dev_info();
    const bool vecq = ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    const bool vec = (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    unsigned *err = err_word_ptr(s);
    if (!err) return cudaErrorUnknown;
    SrcI32 src{A};
    const Len len{n, nullptr};
    const int64_t ctas = query_ctas(q, di.sms);
    const int64_t nb = n > 0 ? ((n - 1) >> logk) + 1 : 0;
    const size_t cs_bytes = (size_t)coarse_geom(nb, cap).size() * sizeof(uint64_t);
    cudaError_t e;
#define RMQ_LQ2(VQ, V)                                                                                    \
    e = launch_query_two<SrcI32, false, VQ, V>(di.device, (unsigned)ctas,                                \
                                               query_ring_bytes<false, VQ>() + cs_bytes, s, src, len, logk, \
                                               cap, T, Cs, l, r, nullptr, nullptr, nullptr, nullptr, M1, logk1, \
                                               max_teams, n, out, q, err, (unsigned long long *)nullptr)
    if (counts) {   // the instrumented kernel (aligned buffers only)
        if (!(vecq && vec)) return cudaErrorInvalidValue;
        e = launch_query_two<SrcI32, false, true, true, Count>(di.device, (unsigned)ctas,
                                                               query_ring_bytes<false, true>() + cs_bytes, s, src, len,
                                                               logk, cap, T, Cs, l, r, nullptr, nullptr, nullptr,
                                                               nullptr, M1, logk1, max_teams, n, out, q, err, counts);
    } else if (vecq && vec) RMQ_LQ2(true, true);
    else if (vecq) RMQ_LQ2(true, false);
    else if (vec) RMQ_LQ2(false, true);
    else RMQ_LQ2(false, false);
#undef RMQ_LQ2
    if (e != cudaSuccess) return e;
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rmq
