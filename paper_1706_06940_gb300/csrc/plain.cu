// plain.cu -- BbST over fixed blocks (Sec. 3.2): block minima (Sec. 3.1
// step 3, level 0), the sparse table over block minima (step 3, all levels)
// and query answering (step 4).  The block-minimum and table kernels are
// generic over the source, so the contracted form reuses them over A_Q.
#include <algorithm>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------- block minima
// Warp per block (k / EPV >= 32 vectors): every lane reads k/(32*EPV)
// consecutive-lane 16-byte vectors (coalesced, streaming), keeps the minimum
// packed key, and a shuffle reduction gives the block minimum.  UNR vectors
// are loaded before any is used to keep enough bytes in flight.
template <class Src, int UNR, bool VEC>
__global__ void __launch_bounds__(kThreads) k_block_min_warp(Src src, Len len, int logk, uint64_t *__restrict__ T0) {
    constexpr int EPV = Src::EPV;
    const int64_t n = len.get();
    const int64_t K = 1ll << logk;
    const int64_t nfull = n >> logk;
    const int64_t nb = (n + K - 1) >> logk;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int vpb = (int)(K / EPV);
    const int vpl = vpb >> 5;
    for (int64_t b = warp; b < nfull; b += nwarps) {
        const int64_t v0 = b * vpb + lane;
        uint64_t best = KEY_MAX;
        for (int u = 0; u < vpl; u += UNR) {
            uint64_t kk[UNR][EPV];
#pragma unroll
            for (int x = 0; x < UNR; ++x) src.template vec<VEC>(v0 + (int64_t)(u + x) * 32, kk[x]);
#pragma unroll
            for (int x = 0; x < UNR; ++x)
#pragma unroll
                for (int e = 0; e < EPV; ++e) best = kmin(best, kk[x][e]);
        }
        best = warp_min(best);
        if (lane == 0) T0[b] = best;
    }
    if (nfull < nb && warp == nfull % nwarps) {  // the short last block
        uint64_t best = KEY_MAX;
        for (int64_t i = nfull * K + lane; i < n; i += 32) best = kmin(best, src.one(i));
        best = warp_min(best);
        if (lane == 0) T0[nfull] = best;
    }
}

// Small blocks (k / EPV < 32 vectors): G = k/EPV lanes per block, 32/G blocks
// per warp row, 4 rows in flight; the reduction is a width-G shuffle.
template <class Src, bool VEC>
__global__ void __launch_bounds__(kThreads) k_block_min_group(Src src, Len len, int logk, uint64_t *__restrict__ T0) {
    constexpr int EPV = Src::EPV;
    const int64_t n = len.get();
    const int64_t K = 1ll << logk;
    const int64_t nfull = n >> logk;
    const int64_t nb = (n + K - 1) >> logk;
    const int G = (int)(K / EPV);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nvec = nfull * G;
    for (int64_t base = warp * 128; base < nvec; base += nwarps * 128) {
        uint64_t best[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t vi = base + x * 32 + lane;
            best[x] = KEY_MAX;
            if (vi < nvec) {
                uint64_t kk[EPV];
                src.template vec<VEC>(vi, kk);
#pragma unroll
                for (int e = 0; e < EPV; ++e) best[x] = kmin(best[x], kk[e]);
            }
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            for (int off = G >> 1; off > 0; off >>= 1) best[x] = kmin(best[x], __shfl_xor_sync(0xffffffffu, best[x], off));
            const int64_t vi = base + x * 32 + lane;
            if (vi < nvec && (lane % G) == 0) T0[vi / G] = best[x];
        }
    }
    if (nfull < nb && warp == nfull % nwarps) {
        uint64_t best = KEY_MAX;
        for (int64_t i = nfull * K + lane; i < n; i += 32) best = kmin(best, src.one(i));
        best = warp_min(best);
        if (lane == 0) T0[nfull] = best;
    }
}

template <class Src, bool VEC>
cudaError_t block_min_dispatch(Src src, Len len, int64_t n_max, int logk, uint64_t *T0, cudaStream_t s) {
    constexpr int EPV = Src::EPV;
    const DevInfo di = dev_info();
    const int64_t K = 1ll << logk;
    const int64_t nb = cdiv(n_max, K);
    if (nb <= 0) return cudaSuccess;
    const int vpb = (int)(K / EPV);
    if (vpb >= 32) {
        const int64_t ctas = std::min<int64_t>(cdiv(nb, kThreads / 32), (int64_t)di.sms * 8);
        const int vpl = vpb / 32;
        if (vpl >= 8) k_block_min_warp<Src, 8, VEC><<<(unsigned)ctas, kThreads, 0, s>>>(src, len, logk, T0);
        else if (vpl >= 4) k_block_min_warp<Src, 4, VEC><<<(unsigned)ctas, kThreads, 0, s>>>(src, len, logk, T0);
        else if (vpl >= 2) k_block_min_warp<Src, 2, VEC><<<(unsigned)ctas, kThreads, 0, s>>>(src, len, logk, T0);
        else k_block_min_warp<Src, 1, VEC><<<(unsigned)ctas, kThreads, 0, s>>>(src, len, logk, T0);
    } else {
        const int64_t nvec = nb * vpb;
        const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(nvec, 128 * (kThreads / 32)), (int64_t)di.sms * 8));
        k_block_min_group<Src, VEC><<<(unsigned)ctas, kThreads, 0, s>>>(src, len, logk, T0);
    }
    note_launches(1);
    return cudaGetLastError();
}

// ------------------------------------------------------------ sparse table
// Level t holds, for block j, the minimum over the 2^t blocks starting at j
// (Sec. 3.1 step 3).  Levels are produced in rounds; a round starting from
// level b computes levels b+1 .. b+nlev in shared memory by doubling:
//   level b+u at j = min over i < 2^u of level b at j + i * 2^b.
// A CTA owns R residues rho (mod 2^b) and S consecutive strides s, i.e. the
// entries j = rho0 + rho + (s0 + s) * 2^b; it loads the S + 2^nlev rows it
// needs once (coalesced along rho for R = 32, along s for R = 1), doubles in
// ping-pong buffers and writes every level's rows < S.  Round 0 uses R = 1
// (contiguous tiles); later rounds start at b >= 5, so R = 32 divides 2^b.
template <int R, int LV>
__global__ void __launch_bounds__(kThreads) k_st_round(uint64_t *__restrict__ T, Len len, int logk, int b, int S) {
    const int64_t n = len.get();
    const int64_t nb = (n + (1ll << logk) - 1) >> logk;
    if (nb < 2) return;
    const int top = ilog2_dev((uint64_t)nb);
    if (b >= top) return;
    const int nlev = min(LV, top - b);
    const int rows = S + (1 << nlev);
    const int64_t stride = 1ll << b;
    const int64_t ngroups = (R == 1) ? 1 : (stride / R);
    const int64_t g = blockIdx.x % ngroups;
    const int64_t st = blockIdx.x / ngroups;
    const int64_t rho0 = g * R;
    const int64_t s0 = st * (int64_t)S;
    if (rho0 + s0 * stride >= nb) return;
    extern __shared__ uint64_t smem[];
    uint64_t *X = smem;
    uint64_t *Y = smem + (size_t)rows * R;
    const uint64_t *Tb = T + (int64_t)b * nb;
    for (int i = threadIdx.x; i < rows * R; i += blockDim.x) {
        const int srow = i / R, c = i % R;
        const int64_t j = rho0 + c + (s0 + srow) * stride;
        X[i] = (j < nb) ? Tb[j] : KEY_MAX;
    }
    __syncthreads();
    for (int u = 1; u <= nlev; ++u) {
        const int half = 1 << (u - 1);
        const int cnt = rows - (1 << u) + 1;
        for (int i = threadIdx.x; i < cnt * R; i += blockDim.x) Y[i] = kmin(X[i], X[i + half * R]);
        __syncthreads();
        const int64_t span = 1ll << (b + u);
        uint64_t *Tu = T + (int64_t)(b + u) * nb;
        for (int i = threadIdx.x; i < S * R; i += blockDim.x) {
            const int srow = i / R, c = i % R;
            const int64_t j = rho0 + c + (s0 + srow) * stride;
            if (j + span <= nb) Tu[j] = Y[i];
        }
        uint64_t *tmp = X; X = Y; Y = tmp;
    }
}

constexpr int kLV0 = 12, kS0 = 256;   // round 0: levels 1..12, 256 outputs per CTA
constexpr int kLV1 = 6, kS1 = 64;     // later rounds: 6 levels, 32 residues x 64 strides

}  // namespace

cudaError_t launch_block_minima_i32(const int32_t *A, int64_t n, int logk, uint64_t *T0, cudaStream_t s) {
    SrcI32 src{A};
    Len len{n, nullptr};
    if ((reinterpret_cast<uintptr_t>(A) & 15) == 0) return block_min_dispatch<SrcI32, true>(src, len, n, logk, T0, s);
    return block_min_dispatch<SrcI32, false>(src, len, n, logk, T0, s);
}

cudaError_t launch_block_minima_u64(const uint64_t *AQ, Len len, int64_t n_max, int logk, uint64_t *T0,
                                    cudaStream_t s) {
    return block_min_dispatch<SrcU64, true>(SrcU64{AQ}, len, n_max, logk, T0, s);
}

cudaError_t launch_sparse_table(uint64_t *T, Len len, int logk, int64_t nb_max, cudaStream_t s) {
    if (nb_max < 2) return cudaSuccess;
    const int top = ilog2_host((uint64_t)nb_max);
    static bool attr_done[64] = {false};
    const DevInfo di = dev_info();
    const size_t smem0 = 2ull * (kS0 + (1 << kLV0)) * 1 * sizeof(uint64_t);
    const size_t smem1 = 2ull * (kS1 + (1 << kLV1)) * 32 * sizeof(uint64_t);
    if (di.device < 64 && !attr_done[di.device]) {
        cudaFuncSetAttribute(k_st_round<1, kLV0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0);
        cudaFuncSetAttribute(k_st_round<32, kLV1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
        attr_done[di.device] = true;
    }
    {
        const int64_t ctas = cdiv(nb_max, kS0);
        k_st_round<1, kLV0><<<(unsigned)ctas, kThreads, smem0, s>>>(T, len, logk, 0, kS0);
        note_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int b = kLV0; b < top; b += kLV1) {
        const int64_t stride = 1ll << b;
        const int64_t ngroups = stride / 32;
        const int64_t nstr = cdiv(nb_max, stride);
        const int64_t ctas = ngroups * cdiv(nstr, kS1);
        k_st_round<32, kLV1><<<(unsigned)ctas, kThreads, smem1, s>>>(T, len, logk, b, kS1);
        note_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

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
