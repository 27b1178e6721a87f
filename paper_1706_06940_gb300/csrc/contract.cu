// contract.cu -- BbST_CON (Sec. 3.1): sort the 2q query endpoints (step 1),
// remap them to ranks in the distinct sorted positions P (step 1), contract A
// to A_Q[j] = min over A[P_j .. P_{j+1}] (step 2), then the block table over
// A_Q (step 3, kernels of plain.cu) and query answering over A_Q (step 4).
#include <algorithm>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kT = 256;                 // threads per CTA
constexpr int kIPT = 16;                // items per thread
constexpr int kTile = kT * kIPT;        // 4096 items per CTA tile
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kATile = 1024;            // elements of A per warp in the contraction

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread CTA.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < kT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        if (lane < kT / 32) wsum[lane] = s;
    }
    __syncthreads();
    const uint32_t pre = w > 0 ? wsum[w - 1] : 0;
    total = wsum[kT / 32 - 1];
    __syncthreads();
    return pre + x - v;
}

// ------------------------------------------------ device-wide exclusive scan
// Three launches: per-chunk sums, a one-CTA scan of the chunk sums, and the
// per-chunk scans offset by their chunk's prefix.  In place is allowed.
__global__ void __launch_bounds__(kT) k_scan_partial(const uint32_t *__restrict__ in, int64_t count,
                                                     uint32_t *__restrict__ partial) {
    __shared__ uint32_t wsum[kT / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kIPT;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kIPT; ++i)
        if (base + i < count) s += in[base + i];
    uint32_t total;
    block_excl_scan(s, wsum, total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kT) k_scan_top(uint32_t *__restrict__ partial, int64_t nc, int64_t *total_out) {
    __shared__ uint32_t wsum[kT / 32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < nc; b += kTile) {
        const int64_t base = b + (int64_t)threadIdx.x * kIPT;
        uint32_t v[kIPT];
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            v[i] = (base + i < nc) ? partial[base + i] : 0;
            s += v[i];
        }
        uint32_t total;
        uint32_t ex = block_excl_scan(s, wsum, total) + carry;
#pragma unroll
        for (int i = 0; i < kIPT; ++i) {
            if (base + i < nc) partial[base + i] = ex;
            ex += v[i];
        }
        carry += total;
    }
    if (total_out && threadIdx.x == 0) *total_out = (int64_t)carry;
}

__global__ void __launch_bounds__(kT) k_scan_final(const uint32_t *in, uint32_t *out, int64_t count,
                                                   const uint32_t *__restrict__ partial) {
    __shared__ uint32_t wsum[kT / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kIPT;
    uint32_t v[kIPT];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
        v[i] = (base + i < count) ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t total;
    uint32_t ex = block_excl_scan(s, wsum, total) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
        if (base + i < count) out[base + i] = ex;
        ex += v[i];
    }
}

size_t scan_aux_words(int64_t count) { return (size_t)cdiv(std::max<int64_t>(count, 1), kTile) + 1; }

cudaError_t scan_exclusive(const uint32_t *in, uint32_t *out, int64_t count, uint32_t *aux, int64_t *total_out,
                           cudaStream_t s) {
    const int64_t nc = cdiv(std::max<int64_t>(count, 1), kTile);
    k_scan_partial<<<(unsigned)nc, kT, 0, s>>>(in, count, aux);
    k_scan_top<<<1, kT, 0, s>>>(aux, nc, total_out);
    k_scan_final<<<(unsigned)nc, kT, 0, s>>>(in, out, count, aux);
    note_launches(3);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- pack
// Endpoint e = 2i + side gets key = its position and tag = e.  An invalid
// query enters as (0, 0) and raises the error word.
__global__ void __launch_bounds__(kT) k_pack(const int32_t *__restrict__ L, const int32_t *__restrict__ R, int64_t q,
                                             int64_t n, uint32_t *__restrict__ keys, uint32_t *__restrict__ tags,
                                             unsigned *err) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t l = L[i], r = R[i];
        if (!(l >= 0 && r >= l && (int64_t)r < n)) { l = 0; r = 0; bad = true; }
        keys[2 * i] = (uint32_t)l;
        keys[2 * i + 1] = (uint32_t)r;
        tags[2 * i] = (uint32_t)(2 * i);
        tags[2 * i + 1] = (uint32_t)(2 * i + 1);
    }
    if (bad) atomicOr(err, ERR_QUERY_RANGE);
}

// ------------------------------------------------------------- radix sort
// LSD radix sort of (key, tag) pairs, 8-bit digits, one upsweep / scan /
// downsweep per digit.  Within a tile items keep their input order (warp w
// owns items [512w, 512w + 512) in rows of 32), so every pass is stable.
__global__ void __launch_bounds__(kT) k_rs_upsweep(const uint32_t *__restrict__ keys, int64_t cnt, int shift,
                                                   uint32_t *__restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[kT / 32][kRadix];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kT / 32) * kRadix; i += kT) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
#pragma unroll 4
    for (int i = 0; i < kIPT; ++i) {
        const int64_t idx = base + i * kT + threadIdx.x;
        if (idx < cnt) atomicAdd(&h[w][(keys[idx] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kT) {
        uint32_t s = 0;
#pragma unroll
        for (int x = 0; x < kT / 32; ++x) s += h[x][d];
        hist[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kT) k_rs_downsweep(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                     int64_t cnt, int shift, const uint32_t *__restrict__ goff,
                                                     int64_t ntiles, uint32_t *__restrict__ kout,
                                                     uint32_t *__restrict__ vout) {
    __shared__ uint32_t wcnt[kT / 32][kRadix];
    __shared__ uint32_t dstart[kRadix];
    __shared__ uint32_t gbase[kRadix];
    __shared__ uint32_t ks[kTile];
    __shared__ uint32_t vs[kTile];
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (int i = threadIdx.x; i < (kT / 32) * kRadix; i += kT) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t kr[kIPT], vr[kIPT], lo[kIPT];
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + w * (32 * kIPT) + row * 32 + lane;
        const bool valid = idx < cnt;
        const uint32_t k = valid ? kin[idx] : 0u;
        const uint32_t v = valid ? vin[idx] : 0u;
        const uint32_t d = (k >> shift) & (kRadix - 1);
        const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u);
        const uint32_t rank = __popc(peers & lt);
        const uint32_t before = valid ? wcnt[w][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        kr[row] = k;
        vr[row] = v;
        lo[row] = before + rank;
    }
    __syncthreads();
    uint32_t run = 0;
    for (int x = 0; x < kT / 32; ++x) {
        const uint32_t c = wcnt[x][threadIdx.x];
        wcnt[x][threadIdx.x] = run;
        run += c;
    }
    uint32_t total;
    const uint32_t ex = block_excl_scan(run, wsum, total);
    dstart[threadIdx.x] = ex;
    gbase[threadIdx.x] = goff[(int64_t)threadIdx.x * ntiles + blockIdx.x] - ex;
    __syncthreads();
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + w * (32 * kIPT) + row * 32 + lane;
        if (idx < cnt) {
            const uint32_t d = (kr[row] >> shift) & (kRadix - 1);
            const uint32_t p = dstart[d] + wcnt[w][d] + lo[row];
            ks[p] = kr[row];
            vs[p] = vr[row];
        }
    }
    __syncthreads();
    const int tcnt = (int)((cnt - base) < kTile ? (cnt - base) : kTile);
    for (int i = threadIdx.x; i < tcnt; i += kT) {
        const uint32_t k = ks[i];
        const uint32_t g = gbase[(k >> shift) & (kRadix - 1)] + (uint32_t)i;
        kout[g] = k;
        vout[g] = vs[i];
    }
}

// ------------------------------------------------------------------ rank
// flag(i) = (i == 0 || key[i] != key[i-1]); rank(i) = (#flags in [0, i]) - 1.
__device__ __forceinline__ bool rank_flag(const uint32_t *K, int64_t idx, int64_t cnt, uint32_t &k) {
    if (idx >= cnt) return false;
    k = K[idx];
    return idx == 0 || K[idx - 1] != k;
}

__global__ void __launch_bounds__(kT) k_rank_count(const uint32_t *__restrict__ K, int64_t cnt,
                                                   uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTile + w * (32 * kIPT);
    uint32_t c = 0;
#pragma unroll 4
    for (int row = 0; row < kIPT; ++row) {
        uint32_t k;
        c += __popc(__ballot_sync(0xffffffffu, rank_flag(K, base + row * 32 + lane, cnt, k)));
    }
    uint32_t total;
    block_excl_scan(lane == 0 ? c : 0u, wsum, total);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kT) k_rank_scatter(const uint32_t *__restrict__ K, const uint32_t *__restrict__ V,
                                                     int64_t cnt, const uint32_t *__restrict__ tile_off,
                                                     uint32_t *__restrict__ P, int32_t *__restrict__ rank_l,
                                                     int32_t *__restrict__ rank_r) {
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t base = (int64_t)blockIdx.x * kTile + w * (32 * kIPT);
    unsigned bal[kIPT];
    uint32_t c = 0;
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        uint32_t k;
        bal[row] = __ballot_sync(0xffffffffu, rank_flag(K, base + row * 32 + lane, cnt, k));
        c += __popc(bal[row]);
    }
    uint32_t total;
    const uint32_t wpre = block_excl_scan(lane == 0 ? c : 0u, wsum, total);
    uint32_t run = tile_off[blockIdx.x] + __shfl_sync(0xffffffffu, wpre, 0);
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + row * 32 + lane;
        if (idx < cnt) {
            const bool f = (bal[row] >> lane) & 1u;
            const int32_t rank = (int32_t)(run + __popc(bal[row] & lt) + (f ? 1u : 0u)) - 1;
            if (f) P[rank] = K[idx];
            const uint32_t tag = V[idx];
            if (tag & 1u) rank_r[tag >> 1] = rank;
            else rank_l[tag >> 1] = rank;
        }
        run += __popc(bal[row]);
    }
}

// ----------------------------------------------------------- contraction
// so[t] = (number of P_j < t * kATile) - 1: the segment open just before
// tile t.  Segments that are open at some tile start span several tiles and
// are combined with atomicMin, so they start at KEY_MAX here; all other
// segments lie in one tile and are written exactly once, by a plain store.
__global__ void __launch_bounds__(kT) k_con_prep(const uint32_t *__restrict__ P, const int64_t *m_dev, int64_t ntA,
                                                 int32_t *__restrict__ so, uint64_t *__restrict__ H) {
    const int64_t m = *m_dev;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntA; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ts = t * kATile;
        int64_t lo = 0, hi = m;  // first j with P[j] >= ts
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)P[mid] < ts) lo = mid + 1;
            else hi = mid;
        }
        const int64_t s = lo - 1;
        so[t] = (int32_t)s;
        if (s >= 0 && s <= m - 2) H[s] = KEY_MAX;
    }
}

__device__ __forceinline__ void emit_atomic(uint64_t *H, int64_t s, uint64_t v) {
    if (v < __ldcg(reinterpret_cast<const unsigned long long *>(H) + s))
        atomicMin(reinterpret_cast<unsigned long long *>(H) + s, (unsigned long long)v);
}

// One warp per tile of kATile = 1024 cells: 8 rows of 32 lanes x 4 cells.
// Segment j covers A[P_j .. P_{j+1}]; a boundary cell P_j closes segment j-1
// (it is its last cell) and opens segment j.  Each row finds its lanes'
// boundary bits in a per-warp bitmap, every lane folds its 4 cells into the
// segment open at its start (head), closes segments that begin and end inside
// it, and leaves its last segment open (tail); a segmented min-scan over the
// lanes then carries each open value to the lane that closes it.
template <bool VEC>
__global__ void __launch_bounds__(kT) k_contract(SrcI32 src, int64_t n, const uint32_t *__restrict__ P,
                                                 const int64_t *m_dev, const int32_t *__restrict__ so, int64_t ntA,
                                                 uint64_t *__restrict__ H) {
    __shared__ uint32_t bm[kT / 32][kATile / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t m = *m_dev;
    const int64_t nv = n / 4;  // vectors wholly inside [0, n)
    for (int64_t t = warp; t < ntA; t += nwarps) {
        const int64_t s_t = so[t], s_n = so[t + 1];
        if (s_t == s_n && (s_t < 0 || s_t > m - 2)) continue;
        const int64_t ts = t * kATile;
        uint64_t kk[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t vi = ts / 4 + u * 32 + lane;
            if (vi < nv) {
                src.template vec<VEC>(vi, kk[u]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) kk[u][e] = (vi * 4 + e < n) ? src.one(vi * 4 + e) : KEY_MAX;
            }
        }
        if (s_t == s_n) {  // no boundary in the tile: one partial minimum
            uint64_t v = KEY_MAX;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int e = 0; e < 4; ++e) v = kmin(v, kk[u][e]);
            v = warp_min(v);
            if (lane == 0) emit_atomic(H, s_t, v);
            continue;
        }
        __syncwarp();  // every lane is done reading the previous tile's bitmap
        bm[w][lane] = 0;
        __syncwarp();
        for (int64_t j = s_t + 1 + lane; j <= s_n; j += 32) {
            const uint32_t off = (uint32_t)((int64_t)P[j] - ts);
            atomicOr(&bm[w][off >> 5], 1u << (off & 31));
        }
        __syncwarp();
        int64_t open = s_t;
        uint64_t carry = KEY_MAX;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned bits = (bm[w][4 * u + (lane >> 3)] >> ((lane & 7) * 4)) & 0xFu;
            const unsigned nb1 = __popc(bits);
            const unsigned b0 = __ballot_sync(0xffffffffu, nb1 & 1u);
            const unsigned b1 = __ballot_sync(0xffffffffu, nb1 & 2u);
            const unsigned b2 = __ballot_sync(0xffffffffu, nb1 & 4u);
            const int tot = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
            if (tot == 0) {
                uint64_t v = kmin(kmin(kk[u][0], kk[u][1]), kmin(kk[u][2], kk[u][3]));
                carry = kmin(carry, warp_min(v));
                continue;
            }
            const int pre = __popc(b0 & lt) + 2 * __popc(b1 & lt) + 4 * __popc(b2 & lt);
            const int64_t seg0 = open + pre;
            uint64_t head = KEY_MAX, cur = KEY_MAX;
            int64_t s = seg0;
            bool closed = false;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint64_t k = kk[u][e];
                if ((bits >> e) & 1u) {
                    const uint64_t v = kmin(cur, k);
                    if (!closed) { head = v; closed = true; }
                    else if (s >= 0 && s <= m - 2) H[s] = v;  // opened and closed inside this lane
                    ++s;
                    cur = k;
                } else {
                    cur = kmin(cur, k);
                }
            }
            bool f = closed;
            uint64_t val = cur;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const bool of = __shfl_up_sync(0xffffffffu, f, d);
                const uint64_t ov = __shfl_up_sync(0xffffffffu, val, d);
                if (lane >= d) {
                    if (!f) val = kmin(val, ov);
                    f = f || of;
                }
            }
            bool exf = __shfl_up_sync(0xffffffffu, f, 1);
            uint64_t exv = __shfl_up_sync(0xffffffffu, val, 1);
            if (lane == 0) { exf = false; exv = KEY_MAX; }
            const uint64_t carry_in = exf ? exv : kmin(carry, exv);
            if (closed && seg0 >= 0 && seg0 <= m - 2) {
                const uint64_t tv = kmin(carry_in, head);
                if (seg0 == s_t) emit_atomic(H, seg0, tv);
                else H[seg0] = tv;
            }
            const bool lf = __shfl_sync(0xffffffffu, f, 31);
            const uint64_t lv = __shfl_sync(0xffffffffu, val, 31);
            carry = lf ? lv : kmin(carry, lv);
            open += tot;
        }
        if (lane == 0 && open >= 0 && open <= m - 2) emit_atomic(H, open, carry);
    }
}

// ------------------------------------------------------ contracted queries
// Query i covers A_Q[a .. b-1] with a = rank(l_i), b = rank(r_i); a == b
// means l_i == r_i.  The answer is the position inside the minimum key.
template <bool VECQ>
__global__ void __launch_bounds__(kT) k_query_con(SrcU64 src, Len lenq, int logk, const uint64_t *__restrict__ T,
                                                  const int32_t *__restrict__ L, const int32_t *__restrict__ R,
                                                  const int32_t *__restrict__ RL, const int32_t *__restrict__ RR,
                                                  int64_t n, int32_t *__restrict__ out, int64_t q) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t mq = lenq.get();
    const int64_t nb = (mq + (1ll << logk) - 1) >> logk;
    for (int64_t wb = warp * 128; wb < q; wb += nwarps * 128) {
        const int64_t base = wb + lane * 4;
        int32_t lq[4], rq[4], aq[4], bq[4];
        bool present[4];
        if (VECQ && base + 3 < q) {
            const int4 x0 = __ldcs(reinterpret_cast<const int4 *>(L + base));
            const int4 x1 = __ldcs(reinterpret_cast<const int4 *>(R + base));
            const int4 x2 = __ldcs(reinterpret_cast<const int4 *>(RL + base));
            const int4 x3 = __ldcs(reinterpret_cast<const int4 *>(RR + base));
            lq[0] = x0.x; lq[1] = x0.y; lq[2] = x0.z; lq[3] = x0.w;
            rq[0] = x1.x; rq[1] = x1.y; rq[2] = x1.z; rq[3] = x1.w;
            aq[0] = x2.x; aq[1] = x2.y; aq[2] = x2.z; aq[3] = x2.w;
            bq[0] = x3.x; bq[1] = x3.y; bq[2] = x3.z; bq[3] = x3.w;
#pragma unroll
            for (int i = 0; i < 4; ++i) present[i] = true;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                present[i] = base + i < q;
                lq[i] = present[i] ? __ldcs(L + base + i) : 0;
                rq[i] = present[i] ? __ldcs(R + base + i) : 0;
                aq[i] = present[i] ? __ldcs(RL + base + i) : 0;
                bq[i] = present[i] ? __ldcs(RR + base + i) : 0;
            }
        }
        uint64_t best[4];
        Pending pl[4], pr[4];
        bool hl[4], hr[4], ok[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ok[i] = present[i] && lq[i] >= 0 && rq[i] >= lq[i] && (int64_t)rq[i] < n;
            hl[i] = hr[i] = false;
            best[i] = KEY_MAX;
            if (ok[i] && aq[i] < bq[i])
                best[i] = resolve_query(T, nb, logk, aq[i], bq[i] - 1, (uint32_t)lq[i], (uint32_t)rq[i], pl[i], pr[i],
                                        hl[i], hr[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            warp_drain_scans<SrcU64, true>(src, mq, hl[i], pl[i], best[i]);
            warp_drain_scans<SrcU64, true>(src, mq, hr[i], pr[i], best[i]);
        }
        int32_t o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = !ok[i] ? -1 : (aq[i] < bq[i] ? (int32_t)key_pos(best[i]) : lq[i]);
        if (VECQ && base + 3 < q) {
            __stcs(reinterpret_cast<int4 *>(out + base), make_int4(o[0], o[1], o[2], o[3]));
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (present[i]) out[base + i] = o[i];
        }
    }
}

int sort_passes(int64_t n) {
    const int bits = n > 1 ? ilog2_host((uint64_t)(n - 1)) + 1 : 0;
    return (bits + kRadixBits - 1) / kRadixBits;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carver {
    char *p;
    size_t used = 0;
    template <class T>
    T *take(size_t count) {
        T *r = reinterpret_cast<T *>(p + used);
        used += align256(std::max<size_t>(count, 1) * sizeof(T));
        return r;
    }
};

}  // namespace

// ------------------------------------------------------------ host side

size_t sort_workspace_bytes(int64_t q) {
    const int64_t cnt = 2 * q;
    const int64_t ntiles = cdiv(std::max<int64_t>(cnt, 1), kTile);
    const int64_t hist = kRadix * ntiles;
    return align256(cnt * 4) * 2 + align256(hist * 4) + align256(scan_aux_words(hist) * 4);
}

cudaError_t sort_endpoints(const int32_t *l, const int32_t *r, int64_t q, int64_t n, uint32_t *pos_out,
                           uint32_t *tag_out, void *ws, size_t, cudaStream_t s) {
    const int64_t cnt = 2 * q;
    const int64_t ntiles = cdiv(std::max<int64_t>(cnt, 1), kTile);
    const int64_t nhist = kRadix * ntiles;
    Carver c{static_cast<char *>(ws)};
    uint32_t *tk = c.take<uint32_t>(cnt), *tv = c.take<uint32_t>(cnt);
    uint32_t *hist = c.take<uint32_t>(nhist);
    uint32_t *aux = c.take<uint32_t>(scan_aux_words(nhist));
    const int P = sort_passes(n);
    const DevInfo di = dev_info();
    uint32_t *pk = (P & 1) ? tk : pos_out, *pv = (P & 1) ? tv : tag_out;
    const int64_t pctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(q, kT), (int64_t)di.sms * 8));
    unsigned *err = err_word_ptr();
    if (!err) return cudaErrorUnknown;
    k_pack<<<(unsigned)pctas, kT, 0, s>>>(l, r, q, n, pk, pv, err);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int p = 0; p < P; ++p) {
        const bool to_out = ((P - 1 - p) & 1) == 0;
        uint32_t *ok = to_out ? pos_out : tk, *ov = to_out ? tag_out : tv;
        const int shift = p * kRadixBits;
        k_rs_upsweep<<<(unsigned)ntiles, kT, 0, s>>>(pk, cnt, shift, hist, ntiles);
        if ((e = scan_exclusive(hist, hist, nhist, aux, nullptr, s)) != cudaSuccess) return e;
        k_rs_downsweep<<<(unsigned)ntiles, kT, 0, s>>>(pk, pv, cnt, shift, hist, ntiles, ok, ov);
        note_launches(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        pk = ok;
        pv = ov;
    }
    return cudaSuccess;
}

size_t rank_workspace_bytes(int64_t q) {
    const int64_t ntiles = cdiv(std::max<int64_t>(2 * q, 1), kTile);
    return align256(ntiles * 4) + align256(scan_aux_words(ntiles) * 4);
}

cudaError_t rank_endpoints(const uint32_t *pos, const uint32_t *tag, int64_t q, uint32_t *P, int64_t *m_dev,
                           int32_t *rank_l, int32_t *rank_r, void *ws, cudaStream_t s) {
    const int64_t cnt = 2 * q;
    const int64_t ntiles = cdiv(std::max<int64_t>(cnt, 1), kTile);
    Carver c{static_cast<char *>(ws)};
    uint32_t *tc = c.take<uint32_t>(ntiles);
    uint32_t *aux = c.take<uint32_t>(scan_aux_words(ntiles));
    k_rank_count<<<(unsigned)ntiles, kT, 0, s>>>(pos, cnt, tc);
    cudaError_t e = scan_exclusive(tc, tc, ntiles, aux, m_dev, s);
    if (e != cudaSuccess) return e;
    k_rank_scatter<<<(unsigned)ntiles, kT, 0, s>>>(pos, tag, cnt, tc, P, rank_l, rank_r);
    note_launches(2);
    return cudaGetLastError();
}

size_t contract_workspace_bytes(int64_t n) { return align256((cdiv(n, kATile) + 2) * 4); }

cudaError_t contract(const int32_t *A, int64_t n, const uint32_t *P, const int64_t *m_dev, uint64_t *AQ, void *ws,
                     cudaStream_t s) {
    const int64_t ntA = cdiv(n, kATile);
    int32_t *so = static_cast<int32_t *>(ws);
    const DevInfo di = dev_info();
    const int64_t pctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(ntA + 1, kT), (int64_t)di.sms * 8));
    k_con_prep<<<(unsigned)pctas, kT, 0, s>>>(P, m_dev, ntA, so, AQ);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(ntA, kT / 32), (int64_t)di.sms * 8));
    SrcI32 src{A};
    if ((reinterpret_cast<uintptr_t>(A) & 15) == 0)
        k_contract<true><<<(unsigned)ctas, kT, 0, s>>>(src, n, P, m_dev, so, ntA, AQ);
    else
        k_contract<false><<<(unsigned)ctas, kT, 0, s>>>(src, n, P, m_dev, so, ntA, AQ);
    note_launches(2);
    return cudaGetLastError();
}

size_t con_workspace_bytes(int64_t n, int64_t q, int logk_con) {
    const int64_t cnt = 2 * q;
    const int64_t mq_max = std::max<int64_t>(cnt - 1, 1);
    const int64_t nbq = cdiv(mq_max, 1ll << logk_con);
    const int64_t lv = ilog2_host((uint64_t)nbq) + 1;
    size_t b = 0;
    b += align256(cnt * 4) * 2;                       // sorted endpoints
    b += align256(cnt * 4);                           // P
    b += align256(8);                                 // m
    b += align256(q * 4) * 2;                         // ranks
    b += align256(mq_max * 8);                        // A_Q
    b += align256(nbq * lv * 8);                      // table over A_Q
    b += std::max({sort_workspace_bytes(q), rank_workspace_bytes(q), contract_workspace_bytes(n)});
    return b;
}

cudaError_t run_contracted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                           int32_t *out, int logk_con, void *ws, cudaStream_t s, Stages *st) {
    const int64_t cnt = 2 * q;
    const int64_t mq_max = std::max<int64_t>(cnt - 1, 1);
    const int64_t nbq = cdiv(mq_max, 1ll << logk_con);
    const int64_t lv = ilog2_host((uint64_t)nbq) + 1;
    Carver c{static_cast<char *>(ws)};
    uint32_t *sk = c.take<uint32_t>(cnt), *sv = c.take<uint32_t>(cnt);
    uint32_t *P = c.take<uint32_t>(cnt);
    int64_t *m_dev = c.take<int64_t>(1);
    int32_t *ra = c.take<int32_t>(q), *rb = c.take<int32_t>(q);
    uint64_t *AQ = c.take<uint64_t>(mq_max);
    uint64_t *T = c.take<uint64_t>(nbq * lv);
    void *scratch = c.p + c.used;
    cudaError_t e;
    Stages none;
    if (!st) st = &none;
    st->mark(s);
    if ((e = sort_endpoints(l, r, q, n, sk, sv, scratch, 0, s)) != cudaSuccess) return e;                 // step 1
    st->mark(s);
    if ((e = rank_endpoints(sk, sv, q, P, m_dev, ra, rb, scratch, s)) != cudaSuccess) return e;           // step 1
    st->mark(s);
    if ((e = contract(A, n, P, m_dev, AQ, scratch, s)) != cudaSuccess) return e;                          // step 2
    st->mark(s);
    const Len lenq{0, m_dev};
    if ((e = launch_block_minima_u64(AQ, lenq, mq_max, logk_con, T, s)) != cudaSuccess) return e;         // step 3
    if ((e = launch_sparse_table(T, lenq, logk_con, nbq, s)) != cudaSuccess) return e;                    // step 3
    st->mark(s);
    const DevInfo di = dev_info();
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(q, 128 * (kT / 32)), (int64_t)di.sms * 8));
    const bool vecq = ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(r) |
                        reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    SrcU64 src{AQ};
    if (vecq) k_query_con<true><<<(unsigned)ctas, kT, 0, s>>>(src, lenq, logk_con, T, l, r, ra, rb, n, out, q);  // step 4
    else k_query_con<false><<<(unsigned)ctas, kT, 0, s>>>(src, lenq, logk_con, T, l, r, ra, rb, n, out, q);
    note_launches(1);
    e = cudaGetLastError();
    st->mark(s);
    return e;
}

}  // namespace rmq
