// contract.cu -- BbST_CON (Sec. 3.1): sort the 2q query endpoints (step 1),
// remap them to ranks in the distinct sorted positions P (step 1), contract A
// to A_Q[j] = min over A[P_j .. P_{j+1}] (step 2), then the block table over
// A_Q (step 3, kernels of plain.cu) and query answering over A_Q (step 4).
#include <algorithm>
#include <climits>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kT = 256;                 // threads per CTA
constexpr int kIPT = 16;                // items per thread
constexpr int kTile = kT * kIPT;        // 4096 items per CTA tile
constexpr int kRadixBits = 9;           // digits of at most 9 bits: 3 passes for positions below 2^27
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
                                                   uint32_t mask, uint32_t *__restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t h[kT / 32][kRadix];
    const int w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kT / 32) * kRadix; i += kT) (&h[0][0])[i] = 0;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t kr[kIPT];
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
        const int64_t idx = base + i * kT + threadIdx.x;
        kr[i] = idx < cnt ? __ldcs(keys + idx) : 0xffffffffu;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kIPT; ++i)
        if (base + i * kT + threadIdx.x < cnt) atomicAdd(&h[w][(kr[i] >> shift) & mask], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kT) {
        uint32_t s = 0;
#pragma unroll
        for (int x = 0; x < kT / 32; ++x) s += h[x][d];
        hist[(int64_t)d * ntiles + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kT, 3) k_rs_downsweep(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                     int64_t cnt, int shift, int width,
                                                     const uint32_t *__restrict__ goff,
                                                     int64_t ntiles, uint32_t *__restrict__ kout,
                                                     uint32_t *__restrict__ vout) {
    __shared__ uint16_t wcnt[kT / 32][kRadix];   // per warp and digit: count, then tile offset (< 4096)
    __shared__ uint32_t gbase[kRadix];
    __shared__ uint32_t ks[kTile];
    __shared__ uint32_t vs[kTile];
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const uint32_t mask = (1u << width) - 1u;
    for (int i = threadIdx.x; i < (kT / 32) * kRadix; i += kT) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t kr[kIPT], vr[kIPT], lo[kIPT];
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {             // every load of the tile is in flight at once
        const int64_t idx = base + w * (32 * kIPT) + row * 32 + lane;
        kr[row] = idx < cnt ? __ldcs(kin + idx) : 0u;
        vr[row] = idx < cnt ? __ldcs(vin + idx) : 0u;
    }
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + w * (32 * kIPT) + row * 32 + lane;
        const bool valid = idx < cnt;
        const uint32_t k = kr[row];
        const uint32_t d = (k >> shift) & mask;
        // lanes holding the same digit: intersect one ballot per digit bit
        unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < kRadixBits; ++b) {  // bits above the digit width are 0 in every lane
            const bool bit = (d >> b) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        const uint32_t rank = __popc(peers & lt);
        const uint32_t before = valid ? wcnt[w][d] : 0u;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][d] = (uint16_t)(before + __popc(peers));
        __syncwarp();
        lo[row] = before + rank;
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, then over the digits
    constexpr int DPT = kRadix / kT;  // digits per thread
    uint32_t run[DPT], tsum = 0;
#pragma unroll
    for (int x = 0; x < DPT; ++x) {
        const int d = threadIdx.x * DPT + x;
        uint32_t r = 0;
        for (int y = 0; y < kT / 32; ++y) r += wcnt[y][d];
        run[x] = r;
        tsum += r;
    }
    uint32_t total;
    uint32_t ex = block_excl_scan(tsum, wsum, total);
#pragma unroll
    for (int x = 0; x < DPT; ++x) {
        const int d = threadIdx.x * DPT + x;
        gbase[d] = goff[(int64_t)d * ntiles + blockIdx.x] - ex;
        uint32_t r = ex;                       // tile offset of digit d for each warp
        for (int y = 0; y < kT / 32; ++y) {
            const uint32_t c = wcnt[y][d];
            wcnt[y][d] = (uint16_t)r;
            r += c;
        }
        ex += run[x];
    }
    __syncthreads();
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + w * (32 * kIPT) + row * 32 + lane;
        if (idx < cnt) {
            const uint32_t d = (kr[row] >> shift) & mask;
            const uint32_t p = wcnt[w][d] + lo[row];
            ks[p] = kr[row];
            vs[p] = vr[row];
        }
    }
    __syncthreads();
    const int tcnt = (int)((cnt - base) < kTile ? (cnt - base) : kTile);
    for (int i = threadIdx.x; i < tcnt; i += kT) {
        const uint32_t k = ks[i];
        const uint32_t g = gbase[(k >> shift) & mask] + (uint32_t)i;
        kout[g] = k;
        vout[g] = vs[i];
    }
}

// ------------------------------------------------------------------ rank
// flag(i) = (i == 0 || key[i] != key[i-1]); rank(i) = (#flags in [0, i]) - 1.
__global__ void __launch_bounds__(kT) k_rank_count(const uint32_t *__restrict__ K, int64_t cnt,
                                                   uint32_t *__restrict__ tile_cnt) {
    __shared__ uint32_t wsum[kT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kTile + w * (32 * kIPT);
    uint32_t kr[kIPT], pv[kIPT];
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + row * 32 + lane;
        kr[row] = idx < cnt ? K[idx] : 0u;
        pv[row] = (idx < cnt && idx > 0) ? K[idx - 1] : ~kr[row];
    }
    uint32_t c = 0;
#pragma unroll
    for (int row = 0; row < kIPT; ++row)
        c += __popc(__ballot_sync(0xffffffffu, base + row * 32 + lane < cnt && kr[row] != pv[row]));
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
    uint32_t kr[kIPT], vr[kIPT];
    unsigned bal[kIPT];
    uint32_t c = 0;
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        const int64_t idx = base + row * 32 + lane;
        kr[row] = idx < cnt ? K[idx] : 0u;
        vr[row] = idx < cnt ? __ldcs(V + idx) : 0u;
        bal[row] = (idx < cnt && idx > 0) ? K[idx - 1] : ~kr[row];   // previous key, for the flag below
    }
#pragma unroll
    for (int row = 0; row < kIPT; ++row) {
        bal[row] = __ballot_sync(0xffffffffu, base + row * 32 + lane < cnt && kr[row] != bal[row]);
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
            if (f) P[rank] = kr[row];
            const uint32_t tag = vr[row];
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

// One warp per tile of kATile = 1024 cells; lane L owns the 32 consecutive
// cells [32L, 32L + 32) of the tile.  Segment j covers A[P_j .. P_{j+1}]; a
// boundary cell P_j closes segment j-1 (it is its last cell) and opens
// segment j.  The tile is read with coalesced 16-byte loads and handed to the
// lanes through shared memory (swizzled so that neither side has bank
// conflicts); the boundaries of the tile form a 1024-bit bitmap, one word per
// lane.  The b-th boundary of the tile closes segment s_t + b, so every lane
// writes the value of each segment it closes into slot b of a per-warp array;
// a segmented min-scan over the lanes adds, to the first slot of each lane,
// the part of that segment held by the lanes before it; the slots are then
// stored to A_Q in order (coalesced).  Only the first segment (begun in an
// earlier tile) and the one left open at the end are combined with atomics.
__device__ __forceinline__ int swz(int x) { return (x & ~7) | ((x & 7) ^ ((x >> 3) & 7)); }

constexpr int kContractSmem = (kT / 32) * kATile * 8 + (kT / 32) * 32 * 4;   // slots (tile view) + bitmaps

template <bool VEC>
__global__ void __launch_bounds__(kT) k_contract(SrcI32 src, int64_t n, const uint32_t *__restrict__ P,
                                                 const int64_t *m_dev, const int32_t *__restrict__ so, int64_t ntA,
                                                 uint64_t *__restrict__ H) {
    extern __shared__ uint64_t csmem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t *slot = csmem + (size_t)w * kATile;                      // 1024 slots per warp
    int4 *tile = reinterpret_cast<int4 *>(slot);                      // the same memory, first 4 KB
    uint32_t *bm = reinterpret_cast<uint32_t *>(csmem + (size_t)(kT / 32) * kATile) + w * 32;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t m = *m_dev;
    const int64_t nv = n / 4;  // vectors wholly inside [0, n)
    for (int64_t t = warp; t < ntA; t += nwarps) {
        // the tile's cells are requested together with its segment numbers (one
        // round trip); tiles outside [P_0, P_{m-1}] are skipped after the fact
        const int64_t s_t = so[t], s_n = so[t + 1];
        const int64_t ts = t * kATile;
        int4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t vi = ts / 4 + u * 32 + lane;
            if (vi < nv) {
                v[u] = VEC ? ld_stream_v4(reinterpret_cast<const int4 *>(src.a) + vi)
                           : make_int4(__ldg(src.a + 4 * vi), __ldg(src.a + 4 * vi + 1), __ldg(src.a + 4 * vi + 2),
                                       __ldg(src.a + 4 * vi + 3));
            } else {
                const int64_t e = 4 * vi;
                v[u] = make_int4(e < n ? __ldg(src.a + e) : INT_MAX, e + 1 < n ? __ldg(src.a + e + 1) : INT_MAX,
                                 e + 2 < n ? __ldg(src.a + e + 2) : INT_MAX, e + 3 < n ? __ldg(src.a + e + 3) : INT_MAX);
            }
        }
        if (s_t == s_n && (s_t < 0 || s_t > m - 2)) continue;
        if (s_t == s_n) {  // no boundary in the tile: one partial minimum of segment s_t
            uint64_t best = KEY_MAX;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t e = (uint32_t)(ts + 4 * (u * 32 + lane));
                best = kmin(best, kmin(kmin(make_key(v[u].x, e), make_key(v[u].y, e + 1)),
                                       kmin(make_key(v[u].z, e + 2), make_key(v[u].w, e + 3))));
            }
            best = warp_min(best);
            if (lane == 0) emit_atomic(H, s_t, best);
            continue;
        }
        __syncwarp();  // the previous tile's slots are no longer read
#pragma unroll
        for (int u = 0; u < 8; ++u) tile[swz(u * 32 + lane)] = v[u];
        bm[lane] = 0;
        __syncwarp();
        const int cnt = (int)(s_n - s_t);
        for (int64_t j0 = s_t + 1; j0 <= s_n; j0 += 256) {
            uint32_t pp[8];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const int64_t j = j0 + x * 32 + lane;
                pp[x] = j <= s_n ? P[j] : 0xffffffffu;
            }
#pragma unroll
            for (int x = 0; x < 8; ++x)
                if (pp[x] != 0xffffffffu) {
                    const uint32_t off = (uint32_t)((int64_t)pp[x] - ts);
                    atomicOr(&bm[off >> 5], 1u << (off & 31));
                }
        }
        __syncwarp();
        const uint32_t word = bm[lane];
        const uint32_t nbits = __popc(word);
        uint32_t pre = nbits;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, pre, d);
            if (lane >= d) pre += y;
        }
        pre -= nbits;
        int32_t vals[32];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int4 q4 = tile[swz(8 * lane + x)];
            vals[4 * x] = q4.x; vals[4 * x + 1] = q4.y; vals[4 * x + 2] = q4.z; vals[4 * x + 3] = q4.w;
        }
        __syncwarp();  // the tile is read; its memory now holds the slots
        // running minimum of the open segment as (value, cell); cells are met in
        // increasing order, so a strict comparison keeps the leftmost
        const uint32_t cell0 = (uint32_t)(ts + 32 * lane);
        int32_t cv = vals[0];
        uint32_t cp = cell0;
        uint32_t k = pre;
        if (word & 1u) { slot[k++] = make_key(cv, cp); }
#pragma unroll
        for (int c = 1; c < 32; ++c) {
            const int32_t vv = vals[c];
            if (word & (1u << c)) {
                // boundary cell: last cell of the open segment, first of the next
                const bool keep = cv <= vv;
                slot[k++] = make_key(keep ? cv : vv, keep ? cp : cell0 + c);
                cv = vv;
                cp = cell0 + c;
            } else if (vv < cv) {
                cv = vv;
                cp = cell0 + c;
            }
        }
        bool f = nbits != 0;
        uint64_t val = make_key(cv, cp);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const bool of = __shfl_up_sync(0xffffffffu, f, d);
            const uint64_t ov = __shfl_up_sync(0xffffffffu, val, d);
            if (lane >= d) {
                if (!f) val = kmin(val, ov);
                f = f || of;
            }
        }
        uint64_t carry_in = __shfl_up_sync(0xffffffffu, val, 1);
        if (lane == 0) carry_in = KEY_MAX;
        if (nbits) slot[pre] = kmin(slot[pre], carry_in);
        const uint64_t tail = __shfl_sync(0xffffffffu, val, 31);
        __syncwarp();
        for (int b = lane; b < cnt; b += 32) {
            const int64_t sg = s_t + b;
            if (sg < 0 || sg > m - 2) continue;
            if (b == 0) emit_atomic(H, sg, slot[0]);
            else H[sg] = slot[b];
        }
        if (lane == 0 && s_n >= 0 && s_n <= m - 2) emit_atomic(H, s_n, tail);
    }
}

int key_bits(int64_t n) { return n > 1 ? ilog2_host((uint64_t)(n - 1)) + 1 : 0; }
int sort_passes(int64_t n) { return (key_bits(n) + kRadixBits - 1) / kRadixBits; }

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
    const int bits = key_bits(n);
    const int width = P ? (bits + P - 1) / P : 0;      // equal digit widths, at most kRadixBits
    for (int p = 0; p < P; ++p) {
        const bool to_out = ((P - 1 - p) & 1) == 0;
        uint32_t *ok = to_out ? pos_out : tk, *ov = to_out ? tag_out : tv;
        const int shift = p * width;
        const uint32_t mask = (1u << width) - 1u;
        k_rs_upsweep<<<(unsigned)ntiles, kT, 0, s>>>(pk, cnt, shift, mask, hist, ntiles);
        if ((e = scan_exclusive(hist, hist, nhist, aux, nullptr, s)) != cudaSuccess) return e;
        k_rs_downsweep<<<(unsigned)ntiles, kT, 0, s>>>(pk, pv, cnt, shift, width, hist, ntiles, ok, ov);
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
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(ntA, kT / 32), (int64_t)di.sms * 3));
    SrcI32 src{A};
    static bool attr[64] = {false};
    if (di.device >= 0 && di.device < 64 && !attr[di.device]) {
        cudaFuncSetAttribute(k_contract<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        cudaFuncSetAttribute(k_contract<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        attr[di.device] = true;
    }
    if ((reinterpret_cast<uintptr_t>(A) & 15) == 0)
        k_contract<true><<<(unsigned)ctas, kT, kContractSmem, s>>>(src, n, P, m_dev, so, ntA, AQ);
    else
        k_contract<false><<<(unsigned)ctas, kT, kContractSmem, s>>>(src, n, P, m_dev, so, ntA, AQ);
    note_launches(2);
    return cudaGetLastError();
}

size_t con_workspace_bytes(int64_t n, int64_t q, int logk_con) {
    const int64_t cnt = 2 * q;
    const int64_t mq_max = std::max<int64_t>(cnt - 1, 1);
    const int64_t nbq = cdiv(mq_max, 1ll << logk_con);
    const int64_t lv = coarse_geom(nbq).lc + 1;
    size_t b = 0;
    b += align256(cnt * 4) * 2;                       // sorted endpoints
    b += align256(cnt * 4);                           // P
    b += align256(8);                                 // m
    b += align256(q * 4) * 2;                         // ranks
    b += align256(mq_max * 8);                        // A_Q
    b += align256(nbq * lv * 8);                      // table over A_Q
    b += align256(kCoarseCap * 8);                    // its coarse summary
    b += align256(query_residual_bytes(q, dev_info().sms));  // residual list of the query
    b += std::max({sort_workspace_bytes(q), rank_workspace_bytes(q), contract_workspace_bytes(n)});
    return b;
}

cudaError_t run_contracted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                           int32_t *out, int logk_con, void *ws, cudaStream_t s, Stages *st) {
    const int64_t cnt = 2 * q;
    const int64_t mq_max = std::max<int64_t>(cnt - 1, 1);
    const int64_t nbq = cdiv(mq_max, 1ll << logk_con);
    const int64_t lv = coarse_geom(nbq).lc + 1;
    Carver c{static_cast<char *>(ws)};
    uint32_t *sk = c.take<uint32_t>(cnt), *sv = c.take<uint32_t>(cnt);
    uint32_t *P = c.take<uint32_t>(cnt);
    int64_t *m_dev = c.take<int64_t>(1);
    int32_t *ra = c.take<int32_t>(q), *rb = c.take<int32_t>(q);
    uint64_t *AQ = c.take<uint64_t>(mq_max);
    uint64_t *T = c.take<uint64_t>(nbq * lv);
    uint64_t *Cs = c.take<uint64_t>(kCoarseCap);
    char *resw = c.take<char>(query_residual_bytes(q, dev_info().sms));
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
    if ((e = launch_sparse_table(T, lenq, logk_con, nbq, s, Cs)) != cudaSuccess) return e;                // step 3
    st->mark(s);
    const DevInfo di = dev_info();
    const bool vecq = ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(r) |
                        reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    SrcU64 src{AQ};
    const ResidualPlan rp = residual_plan(q, di.sms);                                                    // step 4
    Residual *res = reinterpret_cast<Residual *>(resw);
    if (vecq)
        k_query_two<SrcU64, true, true, true><<<(unsigned)rp.ctas, kT, 0, s>>>(src, lenq, logk_con, T, Cs, l, r, ra, rb, n, out, q, res, rp.region, nullptr);
    else
        k_query_two<SrcU64, true, false, true><<<(unsigned)rp.ctas, kT, 0, s>>>(src, lenq, logk_con, T, Cs, l, r, ra, rb, n, out, q, res, rp.region, nullptr);
    note_launches(1);
    e = cudaGetLastError();
    st->mark(s);
    return e;
}

}  // namespace rmq
