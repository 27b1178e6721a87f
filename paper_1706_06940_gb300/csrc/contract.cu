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

// ------------------------------------------------------- endpoint bitmap
// The batch path replaces the comparison of endpoints by a bitmap over the
// positions of A (a counting sort of keys drawn from [0, n)): bit p of the
// bitmap is set when p is an endpoint.  The set bits, in increasing order,
// are exactly the distinct sorted positions P of step 1, and the rank of an
// endpoint is the number of set bits below it.  BW holds one bit word per 32
// positions and BC, for each word, the set bits in all earlier words; a final
// entry (word 0, count m) keeps every rank lookup in bounds.
__device__ __forceinline__ void mark_bit(uint32_t *bw, uint32_t p) {
    // fire-and-forget OR into word p / 32
    asm volatile("red.global.or.b32 [%0], %1;" ::"l"(bw + (p >> 5)), "r"(1u << (p & 31)) : "memory");
}

// Marks both ends of every query.  An invalid query marks position 0 (the
// pair (0, 0) of the sort) and raises the error word.  The warp moves in
// steps of 32 consecutive vectors (4 queries per lane).  Endpoints that crowd
// into few bit words (many queries sharing an end) would serialise their
// reductions on one address; when neighbouring lanes of the warp hit the same
// word, each lane first reads the word and skips the reduction if its bit is
// already set.
__global__ void __launch_bounds__(kT) k_mark_endpoints(const int32_t *__restrict__ L, const int32_t *__restrict__ R,
                                                       int64_t q, int64_t n, uint32_t *__restrict__ bw,
                                                       unsigned *err) {
    pdl_wait();
    bool bad = false;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto mark1 = [&](bool has, uint32_t p) {
        const uint32_t w = has ? (p >> 5) : 0xffffffffu - (uint32_t)lane;   // an absent end shares no word
        const bool crowded = __any_sync(0xffffffffu, __shfl_xor_sync(0xffffffffu, w, 1) == w);
        if (!has) return;
        const uint32_t bit = 1u << (p & 31);
        if (crowded && (__ldcg(bw + w) & bit)) return;
        mark_bit(bw, p);
    };
    auto mark = [&](bool has, int32_t l, int32_t r) {
        const bool ok = l >= 0 && r >= l && (int64_t)r < n;
        bad |= has && !ok;
        mark1(has, ok ? (uint32_t)l : 0u);
        mark1(has, ok ? (uint32_t)r : 0u);
    };
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(L) | reinterpret_cast<uintptr_t>(R)) & 15) == 0) {
        const int64_t nv = q / 4;
        for (int64_t v0 = warp * 32; v0 < nv; v0 += nwarps * 32) {
            const int64_t v = v0 + lane;
            const bool has = v < nv;
            const int4 l4 = has ? __ldcs(reinterpret_cast<const int4 *>(L) + v) : make_int4(0, 0, 0, 0);
            const int4 r4 = has ? __ldcs(reinterpret_cast<const int4 *>(R) + v) : make_int4(0, 0, 0, 0);
            mark(has, l4.x, r4.x); mark(has, l4.y, r4.y); mark(has, l4.z, r4.z); mark(has, l4.w, r4.w);
        }
        done = nv * 4;
    }
    for (int64_t i0 = done + warp * 32; i0 < q; i0 += nwarps * 32) {
        const int64_t i = i0 + lane;
        const bool has = i < q;
        mark(has, has ? __ldcs(L + i) : 0, has ? __ldcs(R + i) : 0);
    }
    if (bad) atomicOr(err, ERR_QUERY_RANGE);
}

// Marks given positions P[0 .. m) (the step-level contraction takes P).
__global__ void __launch_bounds__(kT) k_mark_positions(const uint32_t *__restrict__ P, const int64_t *m_dev,
                                                       uint32_t *__restrict__ bw) {
    const int64_t m = *m_dev;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        mark_bit(bw, P[j]);
}

// Rank counts: the exclusive scan of popc(BW[w]) into BC[w], over the
// nbp = ceil(n / 32) + 1 entries, in tiles of kTile entries (warp w of a CTA
// owns 512 consecutive entries, lane-interleaved rows of 32).
__global__ void __launch_bounds__(kT) k_bits_partial(const uint32_t *__restrict__ BW, int64_t nbp,
                                                     uint32_t *__restrict__ partial) {
    pdl_wait();
    __shared__ uint32_t wsum[kT / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
        const int64_t e = base + i * kT + threadIdx.x;
        if (e < nbp) c += __popc(BW[e]);
    }
    uint32_t total;
    block_excl_scan(c, wsum, total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Position of word i (0 <= i < 32 kIPT) in a warp's staging buffer, which
// is written by rows of 32 words and read back as kIPT consecutive words per
// lane: the 16-byte chunk index is XORed with its bits 3..5, so that neither
// pattern has bank conflicts.
__device__ __forceinline__ int stage_pos(int i) {
    const int ch = i >> 2;
    return ((ch ^ ((ch >> 3) & 7)) << 2) | (i & 3);
}

// Also sets to KEY_MAX every A_Q entry that the contraction combines with
// atomics: the segment open just before each tile of kATile cells (the
// segment whose left end P_j lies below the tile, when j <= m - 2).
// With CP given, also writes the coarse index of the query over A_Q with
// blocks of 2^logk_q entries: CP (where each coarse block of A_Q begins) and
// CB (the coarse block at each bucket start).
// The tile's offset and the total m come from the tile counts of
// k_bits_partial (every CTA adds up the counts of the tiles before it);
// block 0 stores m.
// bs, nbk: bucket_shift(n), bucket_count(n) (word indices are below 2^26, so
// the per-word arithmetic is 32-bit).
__global__ void __launch_bounds__(kT, 6) k_bits_final(const uint32_t *__restrict__ BW, uint32_t *__restrict__ BC,
                                                      int64_t nbp,
                                                      const uint32_t *__restrict__ partial, int64_t *m_dev,
                                                      int64_t ntA, uint64_t *__restrict__ AQ, int logk_q,
                                                      uint32_t *__restrict__ CP, uint16_t *__restrict__ CB, int bs,
                                                      int64_t nbk) {
    pdl_wait();
    __shared__ uint32_t wsum[kT / 32], wbefore[kT / 32], wall[kT / 32];
    __shared__ __align__(16) uint32_t stage[2][kT / 32][32 * kIPT];   // words, exclusive counts
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t *st = stage[0][w], *sx = stage[1][w];
    // a warp's 32 kIPT words: loaded by rows of 32, counted kIPT per lane
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)w * (32 * kIPT);
    uint32_t words[kIPT];
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
        const int64_t e = base + i * 32 + lane;
        words[i] = e < nbp ? BW[e] : 0u;
    }
    uint32_t before = 0, all = 0;
    for (int64_t i = threadIdx.x; i < gridDim.x; i += kT) {
        const uint32_t v = __ldg(partial + i);
        all += v;
        before += i < blockIdx.x ? v : 0u;
    }
#pragma unroll
    for (int i = 0; i < kIPT; ++i) st[stage_pos(i * 32 + lane)] = words[i];
    __syncwarp();
    uint32_t cnt[kIPT];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kIPT; j += 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(st + stage_pos(kIPT * lane + j));
        cnt[j] = __popc(v.x); cnt[j + 1] = __popc(v.y); cnt[j + 2] = __popc(v.z); cnt[j + 3] = __popc(v.w);
        s += cnt[j] + cnt[j + 1] + cnt[j + 2] + cnt[j + 3];
    }
    // thread order is word order: one scan of the per-thread counts, plus
    // the offset of this tile and the total m from the tile counts
    uint32_t x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    before = __reduce_add_sync(0xffffffffu, before);
    all = __reduce_add_sync(0xffffffffu, all);
    if (lane == 31) wsum[w] = x;
    if (lane == 0) { wbefore[w] = before; wall[w] = all; }
    __syncthreads();
    uint32_t run = x - s, tile_off = 0, m32 = 0;
#pragma unroll
    for (int v = 0; v < kT / 32; ++v) {
        run += v < w ? wsum[v] : 0u;
        tile_off += wbefore[v];
        m32 += wall[v];
    }
    run += tile_off;
    const int64_t m = m32;
    if (blockIdx.x == 0 && threadIdx.x == 0) *m_dev = m;
    const uint32_t r0 = run;   // marks before the lane's first word
    // exclusive counts of the lane's words, back in row order
#pragma unroll
    for (int j = 0; j < kIPT; j += 4) {
        uint4 v;
        v.x = run; run += cnt[j];
        v.y = run; run += cnt[j + 1];
        v.z = run; run += cnt[j + 2];
        v.w = run; run += cnt[j + 3];
        *reinterpret_cast<uint4 *>(sx + stage_pos(kIPT * lane + j)) = v;
    }
    // coarse geometry of the table over A_Q (m - 1 entries)
    const int64_t nbq = m >= 2 ? (m - 2 + (1ll << logk_q)) >> logk_q : 0;
    const bool index = CP != nullptr && nbq > 0;
    // the coarse index serves the batch query, whose geometry is kCoarseCapCon's
    const Coarse g = coarse_geom(nbq > 0 ? nbq : 1, kCoarseCapCon);
    const int sh = logk_q + g.lc;
    const uint32_t nbc = (uint32_t)g.nbc;
    const uint32_t bmask = (1u << (bs - 5)) - 1u;   // word e starts a bucket iff (e & bmask) == 0
    if (index && blockIdx.x == 0 && threadIdx.x == 0) CB[nbk] = (uint16_t)(nbc - 1);
    // The lane's kIPT consecutive words e0 .. e0 + kIPT - 1 hold marks r0 .. r0 + s - 1.
    const uint32_t ue0 = (uint32_t)base + (uint32_t)(kIPT * lane);   // word indices are below 2^27
    // A_Q entries the contraction combines with atomics: the segment open at
    // the first word of each contraction tile (32 words); with kIPT = 16 that
    // word is the first of an even lane
    if (AQ && (ue0 & 31u) == 0 && (int64_t)ue0 < nbp && (int64_t)(ue0 >> 5) < ntA) {
        const int64_t sg = (int64_t)r0 - 1;
        if (sg >= 0 && sg <= m - 2) AQ[sg] = KEY_MAX;
    }
    if (index) {
        // a coarse block of A_Q begins at the (j 2^sh)-th mark: only a lane
        // whose marks contain a multiple of 2^sh looks at its words (for
        // r0 = 0, r0 - 1 wraps and mark 0 counts)
        const bool cp_here = s && ((r0 - 1u) >> sh) != ((r0 + s - 1u) >> sh);
        // a bucket starts at word e when (e & bmask) == 0 (not the end entry)
        const uint32_t first_b = (ue0 + bmask) & ~bmask;
        const bool cb_here = first_b < ue0 + (uint32_t)kIPT && (int64_t)first_b < nbp - 1;
        if (cp_here || cb_here) {
            uint32_t ex = r0;
#pragma unroll
            for (int j = 0; j < kIPT; ++j) {
                const uint32_t e = ue0 + (uint32_t)j;
                const uint32_t word = st[stage_pos(kIPT * lane + j)];
                const uint32_t c = __popc(word);
                if (cp_here && c && ((ex + c - 1u) >> sh) != ((ex - 1u) >> sh)) {
                    // at most one multiple of 2^sh among ex .. ex + c - 1 (2^sh >= 32)
                    const uint32_t jb = (ex + (1u << sh) - 1u) >> sh;
                    const uint32_t t = (jb << sh) - ex;
                    if (jb < nbc) {
                        uint32_t wd = word;
                        for (uint32_t d = 0; d < t; ++d) wd &= wd - 1u;   // drop the t lower marks
                        CP[jb] = e * 32u + (uint32_t)(__ffs(wd) - 1);
                    }
                }
                // bucket start: the last coarse block that begins at or before it
                if (cb_here && (e & bmask) == 0 && (int64_t)e < nbp - 1) {
                    const uint32_t upto = ex + (word & 1u);   // marks <= 32e
                    const uint32_t cb = upto >= 1u ? (upto - 1u) >> sh : 0u;
                    CB[e >> (bs - 5)] = (uint16_t)(cb < nbc - 1u ? cb : nbc - 1u);
                }
                ex += c;
            }
        }
    }
    __syncwarp();
    // the counts, stored by rows (coalesced)
    const uint32_t ebase = (uint32_t)base;
    const bool all_in = base + 32 * kIPT <= nbp;
#pragma unroll
    for (int i = 0; i < kIPT; ++i) {
        const uint32_t e = ebase + (uint32_t)(i * 32 + lane);
        if (all_in || (int64_t)e < nbp) BC[e] = sx[stage_pos(i * 32 + lane)];
    }
}

// ----------------------------------------------------------- contraction
__device__ __forceinline__ void emit_atomic(uint64_t *H, int64_t s, uint64_t v) {
    if (v < __ldcg(reinterpret_cast<const unsigned long long *>(H) + s))
        atomicMin(reinterpret_cast<unsigned long long *>(H) + s, (unsigned long long)v);
}

// One warp per tile of kATile = 1024 cells; lane L owns the 32 consecutive
// cells [32L, 32L + 32) of the tile, whose endpoint marks are exactly the
// bitmap word BW[32t + L], and BC[32t + L] - 1 is the segment open at the
// lane's first cell.  Segment j covers A[P_j .. P_{j+1}]; a marked cell P_j
// closes segment j-1 (it is its last cell) and opens segment j.  The tile is
// read with coalesced 16-byte loads and handed to the lanes through shared
// memory (swizzled so that neither side has bank conflicts).  Each lane walks
// its 32 cells branch-free, keeping the running minimum of the open segment
// and writing the value of each segment it closes into its slot of a per-warp
// array; a segmented min-scan over the lanes adds, to the first slot of each
// lane, the part of that segment held by the lanes before it; the slots are
// then stored to A_Q in order (coalesced).  Only the first segment (begun in
// an earlier tile) and the one left open at the end are combined with
// atomics (those entries were set to KEY_MAX by k_bits_final).
// A warp's shared memory is 4 KB: the tile, then (once the lanes hold their
// cells) the slots of at most kSlots segments.  A tile with more marks than
// that (more than half of its cells are endpoints) stores its segments to A_Q
// straight from the walk instead.
__device__ __forceinline__ int swz(int x) { return (x & ~7) | ((x & 7) ^ ((x >> 3) & 7)); }

constexpr int kSlots = kATile * 4 / 8;                   // 512 slots of 8 bytes in the tile's 4 KB
constexpr int kContractSmem = (kT / 32) * kATile * 4;    // per warp: the tile, then its slots

// The walk of one lane over its 32 cells (vals), from cell0: the running
// (value, cell) minimum of the open segment; a marked cell closes the open
// segment (as its last cell) and opens the next.  Slot k (k from pre) gets
// the key of the k-th segment the tile closes.  DIRECT: slots are entries
// s_t + k of H, stored at once, except the lane's first one, returned in
// `first` (the segmented scan completes it).
template <bool DIRECT>
__device__ __forceinline__ void contract_walk(const int32_t (&vals)[32], uint32_t word, uint32_t cell0, uint32_t pre,
                                              uint64_t *slot, uint64_t *__restrict__ H, int32_t s_t, int32_t m,
                                              int32_t &cv, uint32_t &cp, uint64_t &first) {
    cv = INT_MAX;
    cp = 0;
    uint32_t k = pre;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        const int32_t vv = vals[c];
        const bool lt = vv < cv;
        const int32_t mv = lt ? vv : cv;
        const uint32_t mp = lt ? (uint32_t)c : cp;
        const bool b = (word >> c) & 1u;
        if (DIRECT) {
            if (b) {
                const uint64_t key = make_key(mv, cell0 + mp);
                const int32_t sg = s_t + (int32_t)k;
                if (k == pre) first = key;
                else if (sg >= 0 && sg <= m - 2) H[sg] = key;
            }
        } else {
            if (b) slot[k] = make_key(mv, cell0 + mp);
        }
        k += b ? 1u : 0u;
        cv = b ? vv : mv;
        cp = b ? (uint32_t)c : mp;
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kT, 4) k_contract(SrcI32 src, int64_t n, const uint32_t *__restrict__ BW,
                                                 const uint32_t *__restrict__ BC,
                                                 const int64_t *m_dev, int64_t t_begin, int64_t ntA,
                                                 uint64_t *__restrict__ H) {
    pdl_wait();
    extern __shared__ uint64_t csmem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t *slot = csmem + (size_t)w * kSlots;                      // the warp's 4 KB: tile, then slots
    int4 *tile = reinterpret_cast<int4 *>(slot);                      // the same memory, first 4 KB
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t m = (int32_t)*m_dev;       // m <= n < 2^31: segment numbers fit in 32 bits
    const int64_t nfull = n / kATile;        // tiles wholly inside [0, n)
    const int64_t nv = n / 4;                // vectors wholly inside [0, n)
    const int64_t nw = (n + 31) >> 5;        // bitmap words; entry nw is the end entry
    // a tile's cells and its bitmap words, requested together
    auto load_tile = [&](int64_t t, int4 (&v)[8], uint2 &e) {
        const int64_t wi = t * 32 + lane;
        const int64_t ei = wi < nw ? wi : nw;
        e = make_uint2(__ldg(BW + ei), __ldg(BC + ei));
        const int64_t ts = t * kATile;
        if (VEC && t < nfull) {
            const int4 *tp = reinterpret_cast<const int4 *>(src.a) + ts / 4 + lane;
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = ld_stream_v4(tp + u * 32);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t vi = ts / 4 + u * 32 + lane;
                if (vi < nv) {
                    v[u] = VEC ? ld_stream_v4(reinterpret_cast<const int4 *>(src.a) + vi)
                               : make_int4(__ldg(src.a + 4 * vi), __ldg(src.a + 4 * vi + 1),
                                           __ldg(src.a + 4 * vi + 2), __ldg(src.a + 4 * vi + 3));
                } else {
                    const int64_t c = 4 * vi;
                    v[u] = make_int4(c < n ? __ldg(src.a + c) : INT_MAX, c + 1 < n ? __ldg(src.a + c + 1) : INT_MAX,
                                     c + 2 < n ? __ldg(src.a + c + 2) : INT_MAX,
                                     c + 3 < n ? __ldg(src.a + c + 3) : INT_MAX);
                }
            }
        }
    };
    for (int64_t t = t_begin + warp; t < ntA; t += nwarps) {
        const int64_t ts = t * kATile;
        int4 v[8];
        uint2 e;
        load_tile(t, v, e);
        const uint32_t word = e.x;
        const int32_t s_t = (int32_t)__shfl_sync(0xffffffffu, e.y, 0) - 1;      // open before the tile
        const uint32_t nbits = __popc(word);
        const int32_t cnt = (int32_t)__reduce_add_sync(0xffffffffu, nbits);     // boundaries in the tile
        const int32_t s_n = s_t + cnt;                                           // open after the tile
        if (cnt == 0 && (s_t < 0 || s_t > m - 2)) continue;
        if (cnt == 0) {  // no boundary in the tile: one partial minimum of segment s_t
            uint64_t best = KEY_MAX;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t c = (uint32_t)(ts + 4 * (u * 32 + lane));
                best = kmin(best, kmin(kmin(make_key(v[u].x, c), make_key(v[u].y, c + 1)),
                                       kmin(make_key(v[u].z, c + 2), make_key(v[u].w, c + 3))));
            }
            best = warp_min(best);
            if (lane == 0) emit_atomic(H, s_t, best);
            continue;
        }
        __syncwarp();  // the previous tile's slots are no longer read
#pragma unroll
        for (int u = 0; u < 8; ++u) tile[swz(u * 32 + lane)] = v[u];
        __syncwarp();
        const uint32_t pre = e.y - (uint32_t)(s_t + 1);   // slot of this lane's first boundary
        int32_t vals[32];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int4 q4 = tile[swz(8 * lane + x)];
            vals[4 * x] = q4.x; vals[4 * x + 1] = q4.y; vals[4 * x + 2] = q4.z; vals[4 * x + 3] = q4.w;
        }
        __syncwarp();  // the tile is read; its memory now holds the slots
        const uint32_t cell0 = (uint32_t)(ts + 32 * lane);
        int32_t cv;
        uint32_t cp;
        uint64_t first = KEY_MAX;
        const bool direct = cnt > kSlots;   // warp-uniform
        if (!direct) contract_walk<false>(vals, word, cell0, pre, slot, H, s_t, m, cv, cp, first);
        else contract_walk<true>(vals, word, cell0, pre, slot, H, s_t, m, cv, cp, first);
        // segmented min-scan over the lanes: the part of each lane's first
        // segment held by the lanes before it
        bool f = nbits != 0;
        uint64_t val = make_key(cv, cell0 + cp);
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
        const uint64_t tail = __shfl_sync(0xffffffffu, val, 31);
        if (!direct) {
            if (nbits) slot[pre] = kmin(slot[pre], carry_in);
            __syncwarp();
            for (int32_t b = lane; b < cnt; b += 32) {
                const int32_t sg = s_t + b;
                if (sg < 0 || sg > m - 2) continue;
                if (b == 0) emit_atomic(H, sg, slot[0]);
                else H[sg] = slot[b];
            }
        } else if (nbits) {
            const int32_t sg = s_t + (int32_t)pre;
            const uint64_t v0 = kmin(first, carry_in);
            if (sg >= 0 && sg <= m - 2) {
                if (pre == 0) emit_atomic(H, sg, v0);
                else H[sg] = v0;
            }
        }
        if (lane == 0 && s_n >= 0 && s_n <= m - 2) emit_atomic(H, s_n, tail);
    }
}

// The same contraction for a 16-byte aligned A, with the next tile of each
// warp in flight while the warp walks the current one: a warp's shared memory is a 4 KB tile buffer (swizzled as
// above) and, apart from it, the slots of at most kSlotsPf segments.  As
// soon as the lanes hold their cells the buffer is free, and the warp's next
// tile is requested into it with 16-byte cp.async copies, and its bit words
// and counts into registers.  6.5 KB per warp keeps 32 warps per SM (an
// earlier version with two tile buffers had 16).
constexpr int kSlotsPf = 320;                                            // slots of 8 bytes
constexpr int kPfWarpBytes = kATile * 4 + kSlotsPf * 8;                  // 6.5 KB per warp
constexpr int kContractPfSmem = (kT / 32) * kPfWarpBytes;

__global__ void __launch_bounds__(kT, 4) k_contract_pf(SrcI32 src, int64_t n, int64_t ntA,
                                                    const uint32_t *__restrict__ BW,
                                                    const uint32_t *__restrict__ BC, const int64_t *m_dev,
                                                    uint64_t *__restrict__ H) {
    extern __shared__ __align__(16) uint8_t pfsmem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int4 *tile = reinterpret_cast<int4 *>(pfsmem + (size_t)w * kPfWarpBytes);
    uint64_t *slot = reinterpret_cast<uint64_t *>(pfsmem + (size_t)w * kPfWarpBytes + kATile * 4);
    const uint32_t tile_sh = (uint32_t)__cvta_generic_to_shared(tile);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int4 *A4 = reinterpret_cast<const int4 *>(src.a);
    // A is read once: its lines go first when L2 needs room, so that A_Q,
    // written by this kernel and read by the next, stays there longer
    uint64_t evict_first;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
    // one commit group per request (empty past the last tile).  In the last,
    // partial tile a vector copies only its cells below n and the rest of it
    // is zero-filled: such cells follow the last endpoint, so they only ever
    // fall in the open segment after it, which is no entry of A_Q.
    const int64_t nv = (n + 3) >> 2;   // vectors holding at least one cell
    const int64_t nfull = n / kATile;  // tiles wholly inside [0, n)
    auto request = [&](int64_t t) {
        if (t < nfull) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;"
                             ::"r"(tile_sh + (uint32_t)swz(u * 32 + lane) * 16u),
                             "l"(A4 + t * (kATile / 4) + u * 32 + lane), "l"(evict_first) : "memory");
        } else if (t < ntA) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t vi = t * (kATile / 4) + u * 32 + lane;
                const int64_t cells = n - 4 * vi;
                const uint32_t bytes = cells >= 4 ? 16u : (cells > 0 ? (uint32_t)cells * 4u : 0u);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             ::"r"(tile_sh + (uint32_t)swz(u * 32 + lane) * 16u),
                             "l"(A4 + (vi < nv ? vi : 0)), "r"(bytes) : "memory");
            }
        }
        cp_async_commit();
    };
    // the bit word and count of each lane's 32 cells of tile t
    const int64_t nw = (n + 31) >> 5;   // bitmap words; entry nw is the end entry
    auto words_of = [&](int64_t t) {
        const int64_t wi = t * 32 + lane;
        const int64_t ei = wi < nw ? wi : nw;
        return t < ntA ? make_uint2(__ldg(BW + ei), __ldg(BC + ei)) : make_uint2(0u, 0u);
    };
    // A is the caller's: the first tile is requested before the wait for the
    // kernels that write the bitmap
    request(warp);
    pdl_wait();
    const int32_t m = (int32_t)*m_dev;
    uint2 e_next = words_of(warp);
    for (int64_t t = warp; t < ntA; t += nwarps) {
        const int64_t ts = t * kATile;
        const uint2 e = e_next;
        cp_async_wait<0>();
        __syncwarp();   // every lane's copies of the tile have landed
        int32_t vals[32];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int4 q4 = tile[swz(8 * lane + x)];
            vals[4 * x] = q4.x; vals[4 * x + 1] = q4.y; vals[4 * x + 2] = q4.z; vals[4 * x + 3] = q4.w;
        }
        __syncwarp();   // the tile is read: the buffer takes the next one
        request(t + nwarps);
        e_next = words_of(t + nwarps);   // the next tile's words, in flight during this walk
        const uint32_t word = e.x;
        const int32_t s_t = (int32_t)__shfl_sync(0xffffffffu, e.y, 0) - 1;      // open before the tile
        const uint32_t nbits = __popc(word);
        const int32_t cnt = (int32_t)__reduce_add_sync(0xffffffffu, nbits);     // boundaries in the tile
        const int32_t s_n = s_t + cnt;                                           // open after the tile
        const uint32_t cell0 = (uint32_t)(ts + 32 * lane);
        if (cnt == 0) {
            if (s_t >= 0 && s_t <= m - 2) {   // no boundary in the tile: one partial minimum of segment s_t
                int32_t mv = INT_MAX;
                uint32_t mp = 0;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const bool lt = vals[c] < mv;
                    mp = lt ? (uint32_t)c : mp;
                    mv = lt ? vals[c] : mv;
                }
                const uint64_t best = warp_min(make_key(mv, cell0 + mp));
                if (lane == 0) emit_atomic(H, s_t, best);
            }
            continue;
        }
        const uint32_t pre = e.y - (uint32_t)(s_t + 1);   // slot of this lane's first boundary
        int32_t cv;
        uint32_t cp;
        uint64_t first = KEY_MAX;
        const bool direct = cnt > kSlotsPf;   // warp-uniform
        if (!direct) contract_walk<false>(vals, word, cell0, pre, slot, H, s_t, m, cv, cp, first);
        else contract_walk<true>(vals, word, cell0, pre, slot, H, s_t, m, cv, cp, first);
        bool f = nbits != 0;
        uint64_t val = make_key(cv, cell0 + cp);
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
        const uint64_t tail = __shfl_sync(0xffffffffu, val, 31);
        if (!direct) {
            if (nbits) slot[pre] = kmin(slot[pre], carry_in);
            __syncwarp();
            for (int32_t b = lane; b < cnt; b += 32) {
                const int32_t sg = s_t + b;
                if (sg < 0 || sg > m - 2) continue;
                if (b == 0) emit_atomic(H, sg, slot[0]);
                else H[sg] = slot[b];
            }
            __syncwarp();   // the slots are read before the next walk writes them
        } else if (nbits) {
            const int32_t sg = s_t + (int32_t)pre;
            const uint64_t v0 = kmin(first, carry_in);
            if (sg >= 0 && sg <= m - 2) {
                if (pre == 0) emit_atomic(H, sg, v0);
                else H[sg] = v0;
            }
        }
        if (lane == 0 && s_n >= 0 && s_n <= m - 2) emit_atomic(H, s_n, tail);
    }
    cp_async_wait<0>();   // nothing is left in flight (the last request was empty)
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
    unsigned *err = err_word_ptr(s);
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

int64_t bitmap_entries(int64_t n) { return cdiv(n, 32) + 1; }

namespace {

// BC[w] = set bits in words before w, *m_dev = all set bits; A_Q entries
// that the contraction combines with atomics are set to KEY_MAX (AQ may be
// null when no contraction follows).  aux: scan_aux_words(tiles) words.
cudaError_t bitmap_ranks(const uint32_t *BW, uint32_t *BC, int64_t n, int64_t *m_dev, uint64_t *AQ, uint32_t *aux,
                         cudaStream_t s,
                         int logk_q = 0, uint32_t *CP = nullptr, uint16_t *CB = nullptr) {
    const int64_t nbp = bitmap_entries(n);
    const int64_t tiles = cdiv(nbp, kTile);
    launch_pdl(k_bits_partial, (unsigned)tiles, kT, 0, s, BW, nbp, aux);
    launch_pdl(k_bits_final, (unsigned)tiles, kT, 0, s, BW, BC, nbp, aux, m_dev, AQ ? cdiv(n, kATile) : 0, AQ, logk_q, CP, CB,
               bucket_shift(n), bucket_count(n));
    note_launches(2);
    return cudaGetLastError();
}

size_t bitmap_aux_bytes(int64_t n) { return align256(cdiv(bitmap_entries(n), kTile) * 4); }

cudaError_t contract_bitmap(const int32_t *A, int64_t n, const uint32_t *BW, const uint32_t *BC,
                            const int64_t *m_dev, uint64_t *AQ,
                            cudaStream_t s) {
    const int64_t ntA = cdiv(n, kATile);
    const DevInfo di = dev_info();
    SrcI32 src{A};
    static std::once_flag once[kMaxDev];
    static int occ[kMaxDev];
    int per_sm = 1;   // one resident wave
    once_per_device(once, di.device, [&] {
        cudaFuncSetAttribute(k_contract<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        cudaFuncSetAttribute(k_contract<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kContractSmem);
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_contract<true>, kT, kContractSmem);
        if (di.device >= 0 && di.device < kMaxDev) occ[di.device] = std::max(1, o);
    });
    if (di.device >= 0 && di.device < kMaxDev) per_sm = occ[di.device];
    // a 16-byte aligned A goes to the prefetching kernel, an unaligned one to
    // the register-staged one
    int64_t t_begin = 0;
    if ((reinterpret_cast<uintptr_t>(A) & 15) == 0) {
        static std::once_flag pf_once[kMaxDev];
        static int pf_occ[kMaxDev];
        once_per_device(pf_once, di.device, [&] {
            cudaFuncSetAttribute(k_contract_pf, cudaFuncAttributeMaxDynamicSharedMemorySize, kContractPfSmem);
            int o = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_contract_pf, kT, kContractPfSmem);
            if (di.device >= 0 && di.device < kMaxDev) pf_occ[di.device] = std::max(1, o);
        });
        const int per = (di.device >= 0 && di.device < kMaxDev) ? pf_occ[di.device] : 1;
        const int64_t pctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(ntA, kT / 32), (int64_t)di.sms * per));
        launch_pdl(k_contract_pf, (unsigned)pctas, kT, kContractPfSmem, s, src, n, ntA, BW, BC, m_dev, AQ);
        note_launches(1);
        return cudaGetLastError();
    }
    const int64_t ctas =
        std::max<int64_t>(1, std::min<int64_t>(cdiv(ntA - t_begin, kT / 32), (int64_t)di.sms * per_sm));
    if ((reinterpret_cast<uintptr_t>(A) & 15) == 0)
        launch_pdl(k_contract<true>, (unsigned)ctas, kT, kContractSmem, s, src, n, BW, BC, m_dev, t_begin, ntA, AQ);
    else
        launch_pdl(k_contract<false>, (unsigned)ctas, kT, kContractSmem, s, src, n, BW, BC, m_dev, t_begin, ntA, AQ);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

size_t endpoint_bitmap_workspace_bytes(int64_t n) { return bitmap_aux_bytes(n); }

cudaError_t endpoint_bitmap(const int32_t *l, const int32_t *r, int64_t q, int64_t n, uint32_t *BW, uint32_t *BC,
                            int64_t *m_dev, uint64_t *AQ, void *ws, cudaStream_t s, Stages *st, int logk_q,
                            uint32_t *CP, uint16_t *CB) {
    unsigned *err = err_word_ptr(s);
    if (!err) return cudaErrorUnknown;
    // only the bit words need clearing: k_bits_final writes every count
    cudaError_t e = cudaMemsetAsync(BW, 0, (size_t)bitmap_entries(n) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    if (st) st->extra(s, kEventAfterClear);
    const DevInfo di = dev_info();
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(cdiv(q, 4), kT), (int64_t)di.sms * 8));
    launch_pdl(k_mark_endpoints, (unsigned)ctas, kT, 0, s, l, r, q, n, BW, err);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (st) st->mark(s);
    return bitmap_ranks(BW, BC, n, m_dev, AQ, static_cast<uint32_t *>(ws), s, logk_q, CP, CB);
}

size_t contract_workspace_bytes(int64_t n) {
    return 2 * align256(bitmap_entries(n) * sizeof(uint32_t)) + align256(8) + bitmap_aux_bytes(n);
}

cudaError_t contract(const int32_t *A, int64_t n, const uint32_t *P, const int64_t *m_dev, int64_t m_max,
                     uint64_t *AQ, void *ws, cudaStream_t s) {
    // P -> bitmap -> ranks, then the same contraction as the batch path
    Carver c{static_cast<char *>(ws)};
    uint32_t *BW = c.take<uint32_t>(bitmap_entries(n));
    uint32_t *BC = c.take<uint32_t>(bitmap_entries(n));
    int64_t *m2 = c.take<int64_t>(1);
    uint32_t *aux = reinterpret_cast<uint32_t *>(c.p + c.used);
    cudaError_t e = cudaMemsetAsync(BW, 0, (size_t)bitmap_entries(n) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const DevInfo di = dev_info();
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(std::max<int64_t>(m_max, 1), kT), (int64_t)di.sms * 8));
    k_mark_positions<<<(unsigned)ctas, kT, 0, s>>>(P, m_dev, BW);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = bitmap_ranks(BW, BC, n, m2, AQ, aux, s)) != cudaSuccess) return e;
    return contract_bitmap(A, n, BW, BC, m2, AQ, s);
}

size_t con_workspace_bytes(int64_t n, int64_t q, int logk_con) {
    const int64_t mq_max = std::max<int64_t>(std::min<int64_t>(2 * q, n) - 1, 1);
    const int64_t nbq = cdiv(mq_max, 1ll << logk_con);
    const int64_t lv = coarse_geom(nbq, kCoarseCapCon).lc + 1;
    size_t b = 0;
    b += 2 * align256(bitmap_entries(n) * sizeof(uint32_t));  // endpoint bitmap words, rank counts
    b += align256(8);                                 // m
    b += align256(mq_max * 8);                        // A_Q
    b += align256(nbq * lv * 8);                      // table over A_Q
    b += align256(kCoarseBlocksMax * 4) + align256((kBucketsMax + 1) * 2);   // coarse index
    b += bitmap_aux_bytes(n);
    return b;
}

cudaError_t run_contracted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                           int32_t *out, int logk_con, void *ws, cudaStream_t s, Stages *st,
                           unsigned long long *counts, int max_teams) {
    if (max_teams != 1 && max_teams != 2 && max_teams != 4) return cudaErrorInvalidValue;
    const int64_t mq_max = std::max<int64_t>(std::min<int64_t>(2 * q, n) - 1, 1);
    const int64_t nbq = cdiv(mq_max, 1ll << logk_con);
    const int64_t lv = coarse_geom(nbq, kCoarseCapCon).lc + 1;
    Carver c{static_cast<char *>(ws)};
    uint32_t *BW = c.take<uint32_t>(bitmap_entries(n));
    uint32_t *BC = c.take<uint32_t>(bitmap_entries(n));
    int64_t *m_dev = c.take<int64_t>(1);
    uint64_t *AQ = c.take<uint64_t>(mq_max);
    uint64_t *T = c.take<uint64_t>(nbq * lv);
    uint32_t *CP = c.take<uint32_t>(kCoarseBlocksMax);
    uint16_t *CB = c.take<uint16_t>(kBucketsMax + 1);
    uint32_t *aux = reinterpret_cast<uint32_t *>(c.p + c.used);
    cudaError_t e;
    Stages none;
    if (!st) st = &none;
    const DevInfo di = dev_info();
    st->mark(s);
    // step 1: the endpoint bitmap (marks), then the rank counts
    if ((e = endpoint_bitmap(l, r, q, n, BW, BC, m_dev, AQ, aux, s, st, logk_con, CP, CB)) != cudaSuccess) return e;
    st->mark(s);
    if ((e = contract_bitmap(A, n, BW, BC, m_dev, AQ, s)) != cudaSuccess) return e;         // step 2
    st->mark(s);
    const Len lenq{0, m_dev};
    if ((e = launch_block_minima_u64(AQ, lenq, mq_max, logk_con, T, s)) != cudaSuccess) return e;         // step 3
    if ((e = launch_sparse_table(T, lenq, logk_con, nbq, s, true, nullptr, kCoarseCapCon)) != cudaSuccess)
        return e;                                                                                         // step 3
    st->mark(s);
    const bool vecq = ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(r) |
                        reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    SrcU64 src{AQ};
    const int64_t qctas = query_ctas(q, di.sms);                                                        // step 4
    // m is known on the device only: room for the largest coarse table
    const size_t smem = (size_t)kCoarseCapCon * sizeof(uint64_t);
    unsigned long long *no_counts = nullptr;
    if (counts) {   // the instrumented kernel (aligned l, r, out only)
        if (!vecq) return cudaErrorInvalidValue;
        e = launch_query_two<SrcU64, true, true, true, Count>(di.device, (unsigned)qctas,
                                                              smem + query_ring_bytes<true, true>(), s, src, lenq,
                                                              logk_con, kCoarseCapCon, T, nullptr, l, r, BW, BC, CP, CB,
                                                              nullptr, 7, max_teams, n, out, q, nullptr, counts);
    } else if (vecq)
        e = launch_query_two<SrcU64, true, true, true>(di.device, (unsigned)qctas,
                                                       smem + query_ring_bytes<true, true>(), s, src, lenq, logk_con,
                                                       kCoarseCapCon, T, nullptr, l, r, BW, BC, CP, CB, nullptr, 7,
                                                       max_teams, n, out, q, nullptr, no_counts);
    else
        e = launch_query_two<SrcU64, true, false, true>(di.device, (unsigned)qctas, smem, s, src, lenq, logk_con,
                                                        kCoarseCapCon, T, nullptr, l, r, BW, BC, CP, CB, nullptr, 7,
                                                        max_teams, n, out, q, nullptr, no_counts);
    if (e != cudaSuccess) return e;
    note_launches(1);
    e = cudaGetLastError();
    st->mark(s);
    return e;
}

}  // namespace rmq
