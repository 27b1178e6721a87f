// block_min.cu -- block minima (Sec. 3.1 step 3, level 0; Sec. 3.2): for every
// block of k cells, the minimum packed key.  Generic over the source, so the
// contracted form reuses it over A_Q.
#include <algorithm>

#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------- block minima
// Warp per block (k / EPV >= 32 vectors): every lane reads k/(32*EPV)
// consecutive-lane 16-byte vectors (coalesced, streaming), keeps the minimum
// packed key, and a shuffle reduction gives the block minimum.  UNR vectors
// are loaded before any is used to keep enough bytes in flight; when a block
// gives each lane fewer than 8 vectors, a warp takes G = 8 / UNR consecutive
// blocks at once, so that it still reads 4 KB of contiguous memory per round.
// With REV the blocks are visited from the end (a sequence just written is
// then read while its most recent part is still in L2).
// With M1 (int32 source) the kernel also stores the minimum of every small
// block of k1 = 2^logk1 consecutive cells (32 <= k1 <= k), the small blocks of
// the paper's two-level layout (Sec. 3.3, k1 dividing k2 = k).  A row of 128
// cells is one vector per lane: k1 = 128 is a 32-bit warp reduction of the
// values, then the leftmost lane holding the minimum; smaller k1 reduce
// groups of k1/4 lanes; larger k1 combine k1/128 rows.  M1 has
// ceil(n / k1) entries.  WM: 0 = no M1; 1 = k1 = 128 (the default, compiled
// on its own so that it keeps the registers of the one-row case); 2 = any k1.
template <class Src, int UNR, bool VEC, bool REV, int WM, int G>
__global__ void __launch_bounds__(kThreads) k_block_min_warp(Src src, Len len, int logk, uint64_t *__restrict__ T0,
                                                             uint64_t *__restrict__ M1, int logk1) {
    static_assert(G == 1 || UNR * G == 8, "a group of blocks is 8 vectors per lane");
    pdl_wait();
    constexpr int EPV = Src::EPV;
    const int64_t n = len.get();
    const int64_t K = 1ll << logk;
    const int64_t nfull = n >> logk;
    const int64_t nb = (n + K - 1) >> logk;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int vpb = (int)(K / EPV);
    const int vpl = vpb >> 5;   // == UNR when G > 1
    // reduce the UNR vectors of row group u of block b already loaded in kk
    // (acc1: the running minimum of a small block of several rows)
    auto fold = [&](int64_t b, int u, uint64_t (&kk)[UNR][EPV], uint64_t &best, uint64_t &acc1) {
#pragma unroll
        for (int x = 0; x < UNR; ++x) {
            uint64_t rk = KEY_MAX;
#pragma unroll
            for (int e = 0; e < EPV; ++e) rk = kmin(rk, kk[x][e]);
            best = kmin(best, rk);
            if (WM == 1) {   // the row of 128 cells this vector belongs to is a small block
                const uint32_t hv = (uint32_t)(rk >> 32);
                const uint32_t mh = __reduce_min_sync(0xffffffffu, hv);
                const int f = __ffs(__ballot_sync(0xffffffffu, hv == mh)) - 1;
                const uint64_t rowkey = __shfl_sync(0xffffffffu, rk, f);
                if (lane == 0) M1[b * (K >> 7) + u + x] = rowkey;
            } else if (WM == 2) {
                const int row = u + x;   // the row of 128 cells of block b this vector belongs to
                if (logk1 < 7) {         // small blocks of k1/4 lanes
                    uint64_t v = rk;
                    for (int off = 1; off < (1 << (logk1 - 2)); off <<= 1) v = kmin(v, __shfl_xor_sync(0xffffffffu, v, off));
                    if ((lane & ((1 << (logk1 - 2)) - 1)) == 0) M1[((b << logk) + row * 128 + 4 * lane) >> logk1] = v;
                } else {
                    const uint32_t hv = (uint32_t)(rk >> 32);
                    const uint32_t mh = __reduce_min_sync(0xffffffffu, hv);
                    const int f = __ffs(__ballot_sync(0xffffffffu, hv == mh)) - 1;
                    const uint64_t rowkey = __shfl_sync(0xffffffffu, rk, f);
                    acc1 = kmin(acc1, rowkey);
                    const int rb = 1 << (logk1 - 7);   // rows per small block
                    if (((row + 1) & (rb - 1)) == 0) {
                        if (lane == 0) M1[((b << logk) + (int64_t)(row + 1 - rb) * 128) >> logk1] = acc1;
                        acc1 = KEY_MAX;
                    }
                }
            }
        }
    };
    auto one_block = [&](int64_t b) {
        const int64_t v0 = b * vpb + lane;
        uint64_t best = KEY_MAX, acc1 = KEY_MAX;
        for (int u = 0; u < vpl; u += UNR) {
            uint64_t kk[UNR][EPV];
#pragma unroll
            for (int x = 0; x < UNR; ++x) src.template vec<VEC>(v0 + (int64_t)(u + x) * 32, kk[x]);
            fold(b, u, kk, best, acc1);
        }
        best = warp_min(best);
        if (lane == 0) T0[b] = best;
    };
    const int64_t ngrp = nfull / G;   // whole groups of G blocks
    for (int64_t gi = warp; gi < ngrp; gi += nwarps) {
        const int64_t b0 = (REV ? ngrp - 1 - gi : gi) * G;
        // the warp's next group is fetched into L2 while this one is reduced
        if (VEC && lane == 0 && gi + nwarps < ngrp) {
            const int64_t bn = (REV ? ngrp - 1 - (gi + nwarps) : gi + nwarps) * G;
            prefetch_l2_bulk(src.a + bn * K, (uint32_t)(G * K * sizeof(*src.a)));
        }
        if (G == 1) {
            one_block(b0);
        } else {
            uint64_t kk[G][UNR][EPV];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int x = 0; x < UNR; ++x) src.template vec<VEC>((b0 + g) * vpb + lane + x * 32, kk[g][x]);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                uint64_t best = KEY_MAX, acc1 = KEY_MAX;
                fold(b0 + g, 0, kk[g], best, acc1);
                best = warp_min(best);
                if (lane == 0) T0[b0 + g] = best;
            }
        }
    }
    for (int64_t b = ngrp * G + warp; b < nfull; b += nwarps) one_block(b);   // fewer than G left
    if (nfull < nb && warp == nfull % nwarps) {  // the short last block
        uint64_t best = KEY_MAX;
        for (int64_t i = nfull * K + lane; i < n; i += 32) best = kmin(best, src.one(i));
        best = warp_min(best);
        if (lane == 0) T0[nfull] = best;
        if (WM) {   // the small blocks of the short last block
            for (int64_t sb = (nfull * K) >> logk1; (sb << logk1) < n; ++sb) {
                uint64_t rk = KEY_MAX;
                for (int64_t i = (sb << logk1) + lane; i < n && i < ((sb + 1) << logk1); i += 32) rk = kmin(rk, src.one(i));
                rk = warp_min(rk);
                if (lane == 0) M1[sb] = rk;
            }
        }
    }
}

// Small blocks (k / EPV < 32 vectors): G = k/EPV lanes per block, 32/G blocks
// per warp row, 4 rows in flight; the reduction is a width-G shuffle.
// With M1 (int32 source, k1 <= k): the minima of the small blocks of k1 cells
// are taken on the way, once the reduction has covered k1/4 lanes.
template <class Src, bool VEC, bool REV>
__global__ void __launch_bounds__(kThreads) k_block_min_group(Src src, Len len, int logk, uint64_t *__restrict__ T0,
                                                              uint64_t *__restrict__ M1, int logk1) {
    pdl_wait();
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
    const int64_t last = nvec > 0 ? ((nvec - 1) >> 7) << 7 : 0;
    for (int64_t bi = warp * 128; bi < nvec; bi += nwarps * 128) {
        const int64_t base = REV ? last - bi : bi;
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
        const int W1 = M1 ? 1 << (logk1 - 2) : 0;   // lanes of a small block (k1 = 4 W1 cells)
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t vi = base + x * 32 + lane;
            for (int off = 1; off < G; off <<= 1) {
                best[x] = kmin(best[x], __shfl_xor_sync(0xffffffffu, best[x], off));
                if (2 * off == W1 && vi < nvec && (lane & (W1 - 1)) == 0) M1[(vi * EPV) >> logk1] = best[x];
            }
            if (vi < nvec && (lane % G) == 0) T0[vi / G] = best[x];
        }
    }
    if (nfull < nb && warp == nfull % nwarps) {
        uint64_t best = KEY_MAX;
        for (int64_t i = nfull * K + lane; i < n; i += 32) best = kmin(best, src.one(i));
        best = warp_min(best);
        if (lane == 0) T0[nfull] = best;
        if (M1) {   // the small blocks of the short last block
            for (int64_t sb = (nfull * K) >> logk1; (sb << logk1) < n; ++sb) {
                uint64_t rk = KEY_MAX;
                for (int64_t i = (sb << logk1) + lane; i < n && i < ((sb + 1) << logk1); i += 32) rk = kmin(rk, src.one(i));
                rk = warp_min(rk);
                if (lane == 0) M1[sb] = rk;
            }
        }
    }
}

template <class Src, bool VEC, bool REV>
cudaError_t block_min_dispatch(Src src, Len len, int64_t n_max, int logk, uint64_t *T0, cudaStream_t s,
                               uint64_t *M1 = nullptr, int logk1 = 7) {
    constexpr int EPV = Src::EPV;
    const DevInfo di = dev_info();
    const int64_t K = 1ll << logk;
    const int64_t nb = cdiv(n_max, K);
    if (nb <= 0) return cudaSuccess;
    const int vpb = (int)(K / EPV);
    if (vpb >= 32) {
        const int64_t ctas = std::min<int64_t>(cdiv(nb, kThreads / 32), (int64_t)di.sms * 8);
        const int vpl = vpb / 32;
#define RMQ_BMW(U, G)                                                                                          \
    (M1 && logk1 == 7                                                                                          \
         ? launch_pdl(k_block_min_warp<Src, U, VEC, REV, Src::EPV == 4 ? 1 : 0, G>, (unsigned)ctas, kThreads, 0, s,  \
                      src, len, logk, T0, M1, logk1)                                                            \
     : M1 ? launch_pdl(k_block_min_warp<Src, U, VEC, REV, Src::EPV == 4 ? 2 : 0, G>, (unsigned)ctas, kThreads, 0, s, \
                       src, len, logk, T0, M1, logk1)                                                           \
          : launch_pdl(k_block_min_warp<Src, U, VEC, REV, 0, G>, (unsigned)ctas, kThreads, 0, s, src, len, logk, T0, \
                       M1, logk1))
        if (vpl >= 8) RMQ_BMW(8, 1);
        else if (vpl >= 4) RMQ_BMW(4, 2);
        else if (vpl >= 2) RMQ_BMW(2, 4);
        else RMQ_BMW(1, 8);
#undef RMQ_BMW
    } else {
        const int64_t nvec = nb * vpb;
        const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(nvec, 128 * (kThreads / 32)), (int64_t)di.sms * 8));
        launch_pdl(k_block_min_group<Src, VEC, REV>, (unsigned)ctas, kThreads, 0, s, src, len, logk, T0,
                   Src::EPV == 4 && logk1 <= logk ? M1 : nullptr, logk1);
    }
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_block_minima_i32(const int32_t *A, int64_t n, int logk, uint64_t *T0, cudaStream_t s,
                                    uint64_t *M1, int logk1) {
    SrcI32 src{A};
    Len len{n, nullptr};
    if (M1 && (logk1 < MIN_LOGK || logk1 > logk)) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(A) & 15) == 0) return block_min_dispatch<SrcI32, true, false>(src, len, n, logk, T0, s, M1, logk1);
    return block_min_dispatch<SrcI32, false, false>(src, len, n, logk, T0, s, M1, logk1);
}

cudaError_t launch_block_minima_u64(const uint64_t *AQ, Len len, int64_t n_max, int logk, uint64_t *T0,
                                    cudaStream_t s) {
    return block_min_dispatch<SrcU64, true, true>(SrcU64{AQ}, len, n_max, logk, T0, s);
}

}  // namespace rmq
