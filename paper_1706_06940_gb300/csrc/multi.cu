// multi.cu -- many independent arrays, each with its own batch of queries,
// answered in one persistent kernel launch (plain BbST per array, Sec. 3.2,
// with a coarse level as in Sec. 3.3).
//
// Work is a queue of warp-sized items taken in order through one atomic
// counter; every warp works on its own, with no barrier between warps.  The
// queue holds every array's phase-1 items, then every array's phase-3 items
// (interleaving an array's queries with later arrays' slices measured slower:
// warps answering queries then stall while the others stream).
//   phase 1: (array h, one slice of 2^li cells, li = max(13, log2 k)) -- the
//            block minima of the slice (Sec. 3.1 step 3, level 0) into h's
//            T0, and the minima of its coarse blocks (2^lc blocks each) into
//            level 0 of h's coarse table: stored when the coarse blocks lie
//            inside the slice, else folded in with one atomicMin per slice.
//            The warp that finishes h's last slice builds the upper levels of
//            h's coarse table (doubling, in L2) and then sets ready[h];
//   phase 3: (array h, 128 queries) -- waits for ready[h] (a bounded spin: on
//            timeout the item's answers are -1 and the stream's error word
//            gets ERR_TIMEOUT), then answers (Sec. 3.1 step 4 on the coarse
//            table; the open end parts on T0 with lane-local scans; partial
//            blocks by warp scans).
// Every phase-1 item of array h precedes its phase-3 items in the queue, so
// when a warp waits for ready[h], every item h depends on was taken earlier
// by a running warp, and phase-1 items never wait: the wait always ends
// unless a flag is withheld on purpose (the test hook below).
#include <algorithm>
#include <vector>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kMT = 256;
constexpr int kLogSlice = 12;             // phase-1 item: 4096 cells (or one block when k is larger)
constexpr int kMaxLogK = 15;              // block sizes the launch accepts (k <= 32768)
constexpr int kQueriesPerItem = 1024;     // k_query_handles: queries per CTA item
constexpr int kWarpQueries = 128;         // k_multi: queries per warp item (4 per lane)
constexpr int kMultiLcMax = 5;            // coarse blocks of at most 32 blocks: short T0 scans

struct MultiDesc {
    const int32_t *A;
    int32_t n, q;
    int32_t logk, lc;       // blocks of 2^logk cells, coarse blocks of 2^lc blocks
    int32_t item1, item3;   // first phase-1 and phase-3 item of the array
    int32_t n1, n3;         // its phase-1 and phase-3 items
    int64_t t0off, qoff;    // offsets of the array's T0 and of its queries
};

struct MultiParams {
    int32_t H;
    uint32_t flags;
    int64_t spin_limit;
    int32_t total;               // items in all
    uint64_t *T0;                // concatenated level-0 tables
    uint64_t *Cs;                // H coarse tables of kCoarseCap entries (level 0 preset to KEY_MAX)
    uint32_t *done1;             // per array: finished phase-1 items
    uint32_t *ready;             // per array: coarse table complete
    unsigned long long *next;    // work counter
    const int32_t *L, *R;
    int32_t *out;
    unsigned *err;
    MultiDesc d[kMultiMax];
};

__device__ __forceinline__ bool wait_flag(const uint32_t *flag, int64_t limit) {
    for (int64_t it = 0;; ++it) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v) return true;
        if (it >= limit) return false;
        __nanosleep(256);
    }
}

__device__ __forceinline__ void set_flag(uint32_t *flag) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(1u) : "memory");
}

// Exclusive prefix over the H arrays of a per-array count (H <= CAP), into
// shared memory pre[0 .. H] (pre[H] = total).
template <class T, int CAP, class F>
__device__ void array_prefix_n(T *pre, int H, F count, T *wsum) {
    constexpr int PER = CAP / kMT;
    T v[PER], tsum = 0;
#pragma unroll
    for (int x = 0; x < PER; ++x) {
        const int i = threadIdx.x * PER + x;
        v[x] = i < H ? count(i) : (T)0;
        tsum += v[x];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T xs = tsum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, xs, d);
        if (lane >= d) xs += y;
    }
    if (lane == 31) wsum[w] = xs;
    __syncthreads();
    T run = xs - tsum;
    for (int y = 0; y < w; ++y) run += wsum[y];
#pragma unroll
    for (int x = 0; x < PER; ++x) {
        const int i = threadIdx.x * PER + x;
        if (i <= H) pre[i] = run;
        run += v[x];
    }
    if (threadIdx.x == kMT - 1 && H == CAP) pre[H] = run;
    __syncthreads();
}

template <class T>
__device__ __forceinline__ int find_array(const T *pre, int H, T item) {  // last h with pre[h] <= item
    int lo = 0, hi = H - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The last array h whose phase-1 (P3 = false) or phase-3 items start at or
// before `item` (the descriptors are read uniformly by the warp).
template <bool P3>
__device__ __forceinline__ int item_array(const MultiParams &p, int32_t item) {
    int lo = 0, hi = p.H - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((P3 ? p.d[mid].item3 : p.d[mid].item1) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The array and phase of an item: the run (of phase-1 or phase-3 items) that
// starts last at or before it.  Runs are never empty where it matters: an
// array without items of a phase shares its start with the next run, which
// begins later in the queue or at the same item.
__device__ __forceinline__ int item_owner(const MultiParams &p, int32_t item, bool &p3) {
    const int h1 = item_array<false>(p, item);
    const int h3 = item_array<true>(p, item);
    const int32_t s1 = p.d[h1].item1, s3 = p.d[h3].item3;
    p3 = s3 <= item && s3 > s1;
    if (s3 <= item && s3 == s1) p3 = p.d[h1].n1 == 0;   // an empty phase-1 run at the same start
    return p3 ? h3 : h1;
}

// Coarse geometry of an array from its block count and coarse shift.
__device__ __forceinline__ Coarse coarse_from(int64_t nb, int lc) {
    Coarse g;
    g.lc = lc;
    g.nbc = (nb + (1ll << lc) - 1) >> lc;
    g.lvc = ilog2_dev((uint64_t)g.nbc) + 1;
    g.nbc_full = nb >> lc;
    return g;
}

// Minimum key over T0[a .. b] read by one lane (the range spans at most one
// coarse block, i.e. at most 32 entries).
__device__ __forceinline__ uint64_t lane_min(const uint64_t *T0, int64_t a, int64_t b) {
    uint64_t m = KEY_MAX;
    for (int64_t j = a; j <= b; j += 8) {
        uint64_t v[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) v[x] = (j + x <= b) ? __ldcg(reinterpret_cast<const unsigned long long *>(T0) + j + x) : KEY_MAX;
#pragma unroll
        for (int x = 0; x < 8; ++x) m = kmin(m, v[x]);
    }
    return m;
}

// Step 4 on T0 alone for a part [lo, hi] inside one coarse block: inner blocks
// by a lane-local scan, end blocks speculatively (as resolve_query).
__device__ __forceinline__ uint64_t resolve_t0(const uint64_t *T0, int logk, int64_t lo, int64_t hi, uint32_t la,
                                               uint32_t ra, Pending &pl, Pending &pr, bool &hl, bool &hr) {
    const int64_t bl = lo >> logk, br = hi >> logk;
    const unsigned long long *Tu = reinterpret_cast<const unsigned long long *>(T0);
    if (bl == br) {
        const uint64_t t0 = __ldcg(Tu + bl);
        const uint32_t p = key_pos(t0);
        if (p >= la && p <= ra) return t0;
        pl.lo = lo; pl.hi = hi; pl.lb = key_hi(t0);
        hl = true;
        return KEY_MAX;
    }
    uint64_t best = br - bl >= 2 ? lane_min(T0, bl + 1, br - 1) : KEY_MAX;
    const uint64_t tl = __ldcg(Tu + bl), tr = __ldcg(Tu + br);
    if (tl < best) {
        if (key_pos(tl) >= la) best = tl;
        else { pl.lo = lo; pl.hi = ((bl + 1) << logk) - 1; pl.lb = key_hi(tl); hl = true; }
    }
    if (tr < best) {
        if (key_pos(tr) <= ra) best = tr;
        else { pr.lo = br << logk; pr.hi = hi; pr.lb = key_hi(tr); hr = true; }
    }
    return best;
}

// The coarse steps of query.cuh (coarse_blocks_min, resolve_coarse) over a
// coarse table in global memory that this kernel wrote (read through L2).
__device__ __forceinline__ uint64_t gcs(const uint64_t *C, int64_t i) {
    return __ldcg(reinterpret_cast<const unsigned long long *>(C) + i);
}

__device__ __forceinline__ bool gcoarse_span_min(const uint64_t *C, const Coarse &g, int sh, uint32_t lo, uint32_t hi,
                                                 uint64_t &m) {
    const uint32_t BL = lo >> sh, BR = hi >> sh;
    const int t = 31 - __clz((int)(BR - BL + 1));
    const int64_t row = g.row(t);
    m = kmin(gcs(C, row + BL), gcs(C, row + BR + 1 - (1u << t)));
    const uint32_t p = key_pos(m);
    return p >= lo && p <= hi;
}

__device__ __forceinline__ uint64_t gresolve_coarse(const uint64_t *C, const Coarse &g, int sh, uint32_t lo,
                                                    uint32_t hi, int &sub) {
    const uint32_t BL = lo >> sh, BR = hi >> sh;
    if (BL == BR) {
        const uint64_t c0 = gcs(C, BL);
        const uint32_t p = key_pos(c0);
        if (p >= lo && p <= hi) { sub = SUB_NONE; return c0; }
        sub = SUB_WHOLE;
        return KEY_MAX;
    }
    sub = SUB_NONE;
    uint64_t best = KEY_MAX;
    if (BR - BL >= 2) {
        const int t = 31 - __clz((int)(BR - BL - 1));
        const int64_t row = g.row(t);
        best = kmin(gcs(C, row + BL + 1), gcs(C, row + BR - (1u << t)));
    }
    const uint64_t cl = gcs(C, BL), cr = gcs(C, BR);
    if (cl < best) {
        if (key_pos(cl) >= lo) best = cl;
        else sub |= SUB_LEFT;
    }
    if (cr < best) {
        if (key_pos(cr) <= hi) best = cr;
        else sub |= SUB_RIGHT;
    }
    return best;
}

// One round of 1024 cells [r0, r0 + 1024) reduced into segments of 2^s cells
// (s >= 5, segments aligned to their size): key4[u] is the minimum key of the
// lane's 4 cells of row u (cells r0 + 128u + 4 lane .. + 3; KEY_MAX past the
// array's end).  emit(seg, v) is called for every segment that ends in this
// round and begins before the end of the array (cell n):
//   s <= 6: by the segment's first lane (2^(s-2) lanes per segment);
//   7 <= s <= 10: by lane 0, after a warp reduction over 2^(s-7) rows;
//   s > 10: the segment spans rounds: acc keeps the lane's minimum, and the
//     warp reduces it at the segment's last round or when `last` is set.
// The minimum key over the warp's lanes in 32-bit steps: the smallest value
// (the keys' high words order as the values), then the smallest position
// among the lanes that hold it.  Positions are unique, so this is the key
// of the leftmost minimum whatever cells the lanes hold (KEY_MAX lanes take
// part harmlessly: their position is the largest).
__device__ __forceinline__ uint64_t warp_min_key(uint64_t k) {
    const uint32_t hv = key_hi(k);
    const uint32_t mv = __reduce_min_sync(0xffffffffu, hv);
    const uint32_t mp = __reduce_min_sync(0xffffffffu, hv == mv ? key_pos(k) : 0xffffffffu);
    return ((uint64_t)mv << 32) | mp;
}

// The same within aligned groups of G consecutive lanes (G <= 16), by
// shuffles of the 32-bit value, then of the candidates' positions.
__device__ __forceinline__ uint64_t group_min_key(uint64_t k, int G) {
    const uint32_t hv = key_hi(k);
    uint32_t mv = hv;
    for (int off = G >> 1; off > 0; off >>= 1) mv = min(mv, __shfl_xor_sync(0xffffffffu, mv, off));
    uint32_t mp = hv == mv ? key_pos(k) : 0xffffffffu;
    for (int off = G >> 1; off > 0; off >>= 1) mp = min(mp, __shfl_xor_sync(0xffffffffu, mp, off));
    return ((uint64_t)mv << 32) | mp;
}

// Key of the leftmost minimum of 4 consecutive cells starting at position e.
__device__ __forceinline__ uint64_t min4_key(int4 x, uint32_t e) {
    const int32_t m = min(min(x.x, x.y), min(x.z, x.w));
    const uint32_t off = x.x == m ? 0u : (x.y == m ? 1u : (x.z == m ? 2u : 3u));
    return make_key(m, e + off);
}

template <class Emit>
__device__ __forceinline__ void seg_round(const uint64_t (&key4)[8], int64_t r0, int64_t n, int s, bool last,
                                          uint64_t &acc, Emit emit) {
    const int lane = threadIdx.x & 31;
    if (s <= 6) {
        const int G = 1 << (s - 2);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint64_t v = group_min_key(key4[u], G);
            const int64_t c = r0 + 128 * u + 4 * lane;
            if ((lane & (G - 1)) == 0 && c < n) emit(c >> s, v);
        }
    } else if (s <= 10) {
        const int RB = 1 << (s - 7);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            acc = kmin(acc, key4[u]);
            if (((u + 1) & (RB - 1)) == 0) {
                const uint64_t w = warp_min_key(acc);
                acc = KEY_MAX;
                const int64_t c = r0 + 128 * (u + 1 - RB);
                if (lane == 0 && c < n) emit(c >> s, w);
            }
        }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = kmin(acc, key4[u]);
        if (last || (((r0 + 1024) >> s) << s) == r0 + 1024) {
            const uint64_t w = warp_min_key(acc);
            acc = KEY_MAX;
            if (lane == 0) emit(r0 >> s, w);
        }
    }
}

// Phase 1 of array d for the slice [c0, c1) (c0 a multiple of 2^li).
__device__ __forceinline__ void multi_slice(const MultiParams &p, int h, int64_t c0, int64_t c1, int li) {
    const MultiDesc &d = p.d[h];
    const int lane = threadIdx.x & 31;
    const int64_t n = d.n;
    const int logk = d.logk, cs = d.logk + d.lc;
    uint64_t *T0h = p.T0 + d.t0off;
    unsigned long long *C0 = reinterpret_cast<unsigned long long *>(p.Cs) + (int64_t)h * kCoarseCap;
    const bool aligned = (reinterpret_cast<uintptr_t>(d.A) & 15) == 0;
    const int4 *v4 = reinterpret_cast<const int4 *>(d.A);
    uint64_t bacc = KEY_MAX, cacc = KEY_MAX;
    for (int64_t r0 = c0; r0 < c1; r0 += 1024) {
        uint64_t key4[8];
        if (aligned && r0 + 1024 <= n) {
            int4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = ld_stream_v4(v4 + (r0 >> 2) + u * 32 + lane);
            // the next round of this slice is fetched into L2 while this one is reduced
            if (lane == 0 && r0 + 2048 <= c1 && r0 + 2048 <= n) prefetch_l2_bulk(d.A + r0 + 1024, 4096);
#pragma unroll
            for (int u = 0; u < 8; ++u) key4[u] = min4_key(x[u], (uint32_t)(r0 + 128 * u + 4 * lane));
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t e = r0 + 128 * u + 4 * lane;
                uint64_t m = KEY_MAX;
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    if (e + x < n) m = kmin(m, make_key(__ldg(d.A + e + x), (uint32_t)(e + x)));
                key4[u] = m;
            }
        }
        const bool last = r0 + 1024 >= c1;
        seg_round(key4, r0, n, logk, last, bacc, [&](int64_t b, uint64_t v) { T0h[b] = v; });
        if (cs <= li) {   // whole coarse blocks inside the slice: stored
            seg_round(key4, r0, n, cs, last, cacc, [&](int64_t c, uint64_t v) { C0[c] = v; });
        } else {          // the slice lies inside one coarse block: one atomicMin at its end
#pragma unroll
            for (int u = 0; u < 8; ++u) cacc = kmin(cacc, key4[u]);
            if (last) {
                const uint64_t w = warp_min_key(cacc);
                if (lane == 0) atomicMin(C0 + (c0 >> cs), (unsigned long long)w);
            }
        }
    }
}

// The upper levels of array h's coarse table (level 0 complete), by the warp
// that finished its last slice: doubling in global memory, one level after
// the other (the lanes' stores of a level are ordered before the next level's
// loads by the warp barrier).
__device__ __forceinline__ void multi_coarse_levels(uint64_t *C, const Coarse &g) {
    const int lane = threadIdx.x & 31;
    for (int t = 1; t < g.lvc; ++t) {
        const int64_t half = 1ll << (t - 1), cnt = g.nbc - (1ll << t) + 1;
        const int64_t cur = g.row(t), prev = g.row(t - 1);
        for (int64_t J = lane; J < cnt; J += 32) C[cur + J] = kmin(gcs(C, prev + J), gcs(C, prev + J + half));
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kMT, 4) k_multi(const __grid_constant__ MultiParams p) {
    const int lane = threadIdx.x & 31;
    const int32_t total = p.total;
    // lane 0 asks for the warp's next item while the warp works on the current one
    int32_t ahead = 0;
    if (lane == 0) ahead = (int32_t)atomicAdd(p.next, 1ull);
    for (;;) {
        const int32_t item = __shfl_sync(0xffffffffu, ahead, 0);
        if (item >= total) break;
        if (lane == 0) ahead = (int32_t)atomicAdd(p.next, 1ull);
        bool p3;
        const int h = item_owner(p, item, p3);
        const MultiDesc &d = p.d[h];
        if (!p3) {
            // ---------------------------------------------------- phase 1
            const int li = max(kLogSlice, d.logk);
            const int64_t c0 = (int64_t)(item - d.item1) << li;
            const int64_t c1 = min((int64_t)d.n, c0 + ((int64_t)1 << li));
            multi_slice(p, h, c0, c1, li);
            __threadfence();
            uint32_t fin = 0;
            if (lane == 0) {
                const uint32_t items_h = (uint32_t)((((int64_t)d.n - 1) >> li) + 1);
                fin = atomicAdd(p.done1 + h, 1u) == items_h - 1;
            }
            fin = __shfl_sync(0xffffffffu, fin, 0);
            if (fin) {   // the array's last slice: its coarse table's upper levels
                __threadfence();
                const int64_t nb = (((int64_t)d.n - 1) >> d.logk) + 1;
                multi_coarse_levels(p.Cs + (int64_t)h * kCoarseCap, coarse_from(nb, d.lc));
                __threadfence();
                const bool withhold = (p.flags & RMQ_FLAG_TEST_WITHHOLD_READY) && h == 0;
                if (lane == 0 && !withhold) set_flag(p.ready + h);
            }
        } else {
            // ---------------------------------------------------- phase 3
            const int64_t c0 = (int64_t)(item - d.item3) * kWarpQueries;
            const int64_t qn = min((int64_t)kWarpQueries, (int64_t)d.q - c0);
            const int64_t qbase = d.qoff + c0;
            uint32_t ok_flag = 0;
            if (lane == 0) ok_flag = wait_flag(p.ready + h, p.spin_limit);
            ok_flag = __shfl_sync(0xffffffffu, ok_flag, 0);
            if (!ok_flag) {  // the table never became ready: answers -1, error word
                for (int64_t i = lane; i < qn; i += 32) p.out[qbase + i] = -1;
                if (lane == 0 && p.err) atomicOr(p.err, ERR_TIMEOUT);
                continue;
            }
            __threadfence();
            const int64_t nb = (((int64_t)d.n - 1) >> d.logk) + 1;
            const Coarse g = coarse_from(nb, d.lc);
            const uint64_t *C = p.Cs + (int64_t)h * kCoarseCap;
            const uint64_t *T0 = p.T0 + d.t0off;
            const int sh = d.logk + d.lc;
            const SrcI32 src{d.A};
            const bool vecA = (reinterpret_cast<uintptr_t>(d.A) & 15) == 0;
            int32_t lq[4], rq[4], o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t qi = lane * 4 + i;
                lq[i] = qi < qn ? __ldcs(p.L + qbase + qi) : 0;
                rq[i] = qi < qn ? __ldcs(p.R + qbase + qi) : -1;   // absent: reads as invalid
            }
            bool bad = false;
            // the coarse check of the lanes' 4 queries at once; then one slot
            // at a time, the open queries are resolved and their parts drained
            unsigned open = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool ok = lq[i] >= 0 && rq[i] >= lq[i] && rq[i] < d.n;
                bad |= (lane * 4 + i < qn) && !ok;
                uint64_t m = KEY_MAX;
                const bool inside = ok && gcoarse_span_min(C, g, sh, (uint32_t)lq[i], (uint32_t)rq[i], m);
                o[i] = !ok ? -1 : (int32_t)key_pos(m);
                open |= (ok && !inside ? 1u : 0u) << i;
            }
            // the settled (and invalid) queries' answers; the open ones follow
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t qi = lane * 4 + i;
                if (qi < qn && !((open >> i) & 1u)) p.out[qbase + qi] = o[i];
            }
            if (bad && p.err) atomicOr(p.err, ERR_QUERY_RANGE);
            // the open queries of all four slots, one per lane (slot-major
            // order), resolved in one round and their edge parts drained
            // together (more rounds only past 32 open queries)
            const unsigned m0 = __ballot_sync(0xffffffffu, open & 1u), m1 = __ballot_sync(0xffffffffu, open & 2u);
            const unsigned m2 = __ballot_sync(0xffffffffu, open & 4u), m3 = __ballot_sync(0xffffffffu, open & 8u);
            const int n0 = __popc(m0), n1 = __popc(m1), n2 = __popc(m2);
            const int total = n0 + n1 + n2 + __popc(m3);
            for (int b = 0; b < total; b += 32) {
                const int k = b + lane;
                const bool has = k < total;
                int slot = 0, owner = 0;
                if (has) {   // the (kk + 1)-th set bit of the slot's mask is the owner lane
                    int kk = k;
                    unsigned mm = m0;
                    if (kk >= n0) {
                        kk -= n0; mm = m1; slot = 1;
                        if (kk >= n1) {
                            kk -= n1; mm = m2; slot = 2;
                            if (kk >= n2) { kk -= n2; mm = m3; slot = 3; }
                        }
                    }
                    owner = (int)__fns(mm, 0u, kk + 1);
                }
                int32_t l = 0, r = 0;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int32_t li = __shfl_sync(0xffffffffu, lq[i], owner);
                    const int32_t ri = __shfl_sync(0xffffffffu, rq[i], owner);
                    if (slot == i) { l = li; r = ri; }
                }
                Pending pl, pr;
                bool hl = false, hr = false;
                uint64_t best = KEY_MAX;
                if (has) {
                    int sub;
                    best = gresolve_coarse(C, g, sh, (uint32_t)l, (uint32_t)r, sub);
                    if (sub == SUB_WHOLE) {
                        best = resolve_t0(T0, d.logk, l, r, (uint32_t)l, (uint32_t)r, pl, pr, hl, hr);
                    } else {
                        Pending unused;
                        bool unused_flag = false;
                        if (sub & SUB_LEFT) {
                            const int64_t end_l = ((((int64_t)l >> sh) + 1) << sh) - 1;
                            best = kmin(best, resolve_t0(T0, d.logk, l, end_l, (uint32_t)l, 0xffffffffu, pl, unused,
                                                         hl, unused_flag));
                        }
                        if (sub & SUB_RIGHT) {
                            const int64_t start_r = ((int64_t)r >> sh) << sh;
                            Pending a, b2;
                            bool ha = false, hb = false;
                            best = kmin(best, resolve_t0(T0, d.logk, start_r, r, 0u, (uint32_t)r, a, b2, ha, hb));
                            if (ha) { pr = a; hr = true; }
                            if (hb) { pr = b2; hr = true; }
                        }
                    }
                }
                if (vecA) {
                    warp_drain_scans<SrcI32, true>(src, d.n, hl, pl, best);
                    warp_drain_scans<SrcI32, true>(src, d.n, hr, pr, best);
                } else {
                    warp_drain_scans<SrcI32, false>(src, d.n, hl, pl, best);
                    warp_drain_scans<SrcI32, false>(src, d.n, hr, pr, best);
                }
                if (has) p.out[qbase + owner * 4 + slot] = (int32_t)key_pos(best);
            }
        }
    }
}

}  // namespace

// Block size for an array of the multi-array launch: the smallest power of
// two >= 32 whose coarse blocks hold at most 32 blocks (short T0 scans).
int multi_logk(int64_t n) {
    for (int lk = MIN_LOGK; lk < kMaxLogK; ++lk) {
        const int64_t nb = cdiv(n, 1ll << lk);
        if (coarse_geom(nb).lc <= kMultiLcMax) return lk;
    }
    return kMaxLogK;
}

int multi_max_logk() { return kMaxLogK; }

size_t multi_workspace_bytes(const int64_t *n, const int64_t *q, const int32_t *logk, int H) {
    int64_t t0 = 0;
    for (int h = 0; h < H; ++h)
        if (q[h] > 0) t0 += cdiv(n[h], 1ll << logk[h]);
    return 256 + (size_t)H * 8 + (size_t)t0 * 8 + (size_t)H * kCoarseCap * 8 + 256;
}

cudaError_t launch_multi(const int32_t *const *A, const int64_t *n, const int64_t *q, const int32_t *logk, int H,
                         const int32_t *l, const int32_t *r, int32_t *out, uint32_t flags, void *ws, cudaStream_t s) {
    if (H < 1 || H > kMultiMax) return cudaErrorInvalidValue;
    const DevInfo di = dev_info();
    unsigned *err = err_word_ptr(s);
    if (!err) return cudaErrorUnknown;
    MultiParams *p = new MultiParams();
    p->H = H;
    p->flags = flags;
    p->spin_limit = (flags & RMQ_FLAG_TEST_WITHHOLD_READY) ? (1ll << 12) : (1ll << 24);
    char *base = static_cast<char *>(ws);
    p->next = reinterpret_cast<unsigned long long *>(base);
    p->done1 = reinterpret_cast<uint32_t *>(base + 256);
    p->ready = p->done1 + H;
    const size_t ctl = 256 + (((size_t)H * 8 + 255) & ~(size_t)255);
    int64_t t0 = 0, qo = 0;
    for (int h = 0; h < H; ++h) {
        MultiDesc &dd = p->d[h];
        dd.A = A[h];
        dd.n = (int32_t)n[h];
        dd.q = (int32_t)q[h];
        dd.logk = logk[h];
        const int64_t nb = q[h] > 0 && n[h] > 0 ? cdiv(n[h], 1ll << logk[h]) : 0;
        dd.lc = nb > 0 ? coarse_geom(nb).lc : 0;
        dd.n1 = nb > 0 ? (int32_t)cdiv(n[h], 1ll << std::max(kLogSlice, (int)logk[h])) : 0;
        dd.n3 = (int32_t)cdiv(q[h], kWarpQueries);
        dd.t0off = t0;
        dd.qoff = qo;
        t0 += nb;
        qo += q[h];
    }
    // the queue: every phase-1 run in array order, then every phase-3 run
    int64_t it = 0;
    for (int j = 0; j < H; ++j) {
        p->d[j].item1 = (int32_t)it;
        it += p->d[j].n1;
    }
    for (int j = 0; j < H; ++j) {
        p->d[j].item3 = (int32_t)it;
        it += p->d[j].n3;
    }
    static std::once_flag once[kMaxDev];
    static int occ[kMaxDev];
    once_per_device(once, di.device, [&] {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_multi, kMT, 0);
        if (di.device >= 0 && di.device < kMaxDev) occ[di.device] = std::max(1, o);
    });
    const int ctas = (di.device >= 0 && di.device < kMaxDev ? occ[di.device] : 1) * di.sms;
    if (it >= (1ll << 31) - (1ll << 20)) {   // the item counter is 32-bit on the device
        delete p;
        return cudaErrorInvalidValue;
    }
    p->total = (int32_t)it;
    p->T0 = reinterpret_cast<uint64_t *>(base + ctl);
    p->Cs = p->T0 + t0;
    p->L = l;
    p->R = r;
    p->out = out;
    p->err = err;
    cudaError_t e = cudaMemsetAsync(base, 0, ctl, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->Cs, 0xff, (size_t)H * kCoarseCap * 8, s);
    if (e == cudaSuccess) {
        // every CTA resident at once (the waits of phase 3 rely on the warps
        // that hold phase-1 items running)
        k_multi<<<ctas, kMT, 0, s>>>(*p);
        note_launches(1);
        e = cudaGetLastError();
    }
    delete p;
    return e;
}

}  // namespace rmq

// ---------------------------------------------------------------------------
// Queries of many requests against resident handles, in one launch.  Item =
// (request h, 1024 queries); no item depends on another.  Each item copies
// its handle's coarse table into shared memory, answers what the coarse level
// settles, and finishes the rest (at most 1024, kept in shared memory) with
// the handle's block table and partial-block scans.
namespace rmq {
namespace {

struct ReqDesc {
    const int32_t *A;
    const uint64_t *T;
    const uint64_t *Cs;
    int32_t n;
    int32_t q;
    int32_t logk;
    int32_t pad;
};

struct ReqParams {
    int32_t H;
    int32_t pad;
    const int32_t *L, *R;
    int32_t *out;
    unsigned *err;
    ReqDesc d[kReqMax];
};

__global__ void __launch_bounds__(kMT, 3) k_query_handles(const __grid_constant__ ReqParams p) {
    __shared__ uint64_t cs[kCoarseCap];
    __shared__ int64_t qoff[kReqMax + 1];
    __shared__ int32_t pre[kReqMax + 1];
    __shared__ int64_t wsum64[kMT / 32];
    __shared__ int32_t wsum32[kMT / 32];
    __shared__ uint16_t open_q[kQueriesPerItem];   // indices (inside the item) of the open queries
    __shared__ int n_open;
    const int H = p.H;
    const int lane = threadIdx.x & 31;
    array_prefix_n<int64_t, kReqMax>(qoff, H, [&](int h) { return (int64_t)p.d[h].q; }, wsum64);
    array_prefix_n<int32_t, kReqMax>(pre, H, [&](int h) { return (p.d[h].q + kQueriesPerItem - 1) / kQueriesPerItem; }, wsum32);
    const int64_t items = pre[H];
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int h = find_array<int32_t>(pre, H, (int32_t)it);
        const ReqDesc d = p.d[h];
        const int64_t nb = ((int64_t)d.n + (1ll << d.logk) - 1) >> d.logk;
        const Coarse g = coarse_geom(nb);
        const int64_t c0 = (it - pre[h]) * kQueriesPerItem;
        const int64_t qn = min((int64_t)kQueriesPerItem, (int64_t)d.q - c0);
        const int64_t qbase = qoff[h] + c0;
        if (threadIdx.x == 0) n_open = 0;
        load_coarse(cs, d.Cs, (int)g.size());
        __syncthreads();
        bool bad = false;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int64_t qi = threadIdx.x * 4 + x;
            if (qi >= qn) continue;
            const int32_t l = p.L[qbase + qi], r = p.R[qbase + qi];
            const bool ok = l >= 0 && r >= l && r < d.n;
            int32_t o = -1;
            bad |= !ok;
            if (ok) {
                uint64_t m;
                if (coarse_span_min(cs, g, d.logk, (uint32_t)l, (uint32_t)r, (uint32_t)l, (uint32_t)r, m)) {
                    o = (int32_t)key_pos(m);
                } else {
                    open_q[atomicAdd(&n_open, 1)] = (uint16_t)qi;
                    continue;
                }
            }
            p.out[qbase + qi] = o;
        }
        if (bad && p.err) atomicOr(p.err, ERR_QUERY_RANGE);
        __syncthreads();
        const int cnt = n_open;
        const int sh = d.logk + g.lc;
        const SrcI32 src{d.A};
        const bool vecA = (reinterpret_cast<uintptr_t>(d.A) & 15) == 0;
        for (int wb = (threadIdx.x >> 5) * 32; wb < cnt; wb += (kMT >> 5) * 32) {
            const int idx = wb + lane;
            const bool has = idx < cnt;
            Pending pl, pr;
            bool hl = false, hr = false;
            uint64_t best = KEY_MAX;
            struct { int32_t i, l, r; } e{0, 0, 0};
            if (has) {
                e.i = open_q[idx];
                e.l = p.L[qbase + e.i];
                e.r = p.R[qbase + e.i];
                int sub;
                best = resolve_coarse(cs, g, d.logk, (uint32_t)e.l, (uint32_t)e.r, (uint32_t)e.l, (uint32_t)e.r, sub);
                if (sub == SUB_WHOLE) {
                    best = resolve_query(d.T, nb, d.logk, e.l, e.r, (uint32_t)e.l, (uint32_t)e.r, pl, pr, hl, hr);
                } else if (sub != SUB_NONE) {
                    Pending unused;
                    bool unused_flag = false;
                    if (sub & SUB_LEFT) {
                        const int64_t end_l = ((((int64_t)e.l >> sh) + 1) << sh) - 1;
                        best = kmin(best, resolve_query(d.T, nb, d.logk, e.l, end_l, (uint32_t)e.l, 0xffffffffu, pl,
                                                        unused, hl, unused_flag));
                    }
                    if (sub & SUB_RIGHT) {
                        const int64_t start_r = ((int64_t)e.r >> sh) << sh;
                        Pending a, b2;
                        bool ha = false, hb = false;
                        best = kmin(best, resolve_query(d.T, nb, d.logk, start_r, e.r, 0u, (uint32_t)e.r, a, b2, ha, hb));
                        if (ha) { pr = a; hr = true; }
                        if (hb) { pr = b2; hr = true; }
                    }
                }
            }
            if (vecA) {
                warp_drain_scans<SrcI32, true>(src, d.n, hl, pl, best);
                warp_drain_scans<SrcI32, true>(src, d.n, hr, pr, best);
            } else {
                warp_drain_scans<SrcI32, false>(src, d.n, hl, pl, best);
                warp_drain_scans<SrcI32, false>(src, d.n, hr, pr, best);
            }
            if (has) p.out[qbase + e.i] = (int32_t)key_pos(best);
        }
        __syncthreads();  // shared memory is reused by the next item
    }
}

}  // namespace

cudaError_t launch_query_handles(const QueryReq *reqs, int H, const int32_t *l, const int32_t *r, int32_t *out,
                                 cudaStream_t s) {
    const DevInfo di = dev_info();
    unsigned *err = err_word_ptr(s);
    if (!err) return cudaErrorUnknown;
    ReqParams *p = new ReqParams();
    p->H = H;
    p->L = l;
    p->R = r;
    p->out = out;
    p->err = err;
    int64_t items = 0;
    for (int h = 0; h < H; ++h) {
        p->d[h] = ReqDesc{reqs[h].A, reqs[h].T, reqs[h].Cs, (int32_t)reqs[h].n, (int32_t)reqs[h].q, reqs[h].logk, 0};
        items += cdiv(reqs[h].q, kQueriesPerItem);
    }
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)di.sms * 3));
    k_query_handles<<<(unsigned)ctas, kMT, 0, s>>>(*p);
    note_launches(1);
    delete p;
    return cudaGetLastError();
}

}  // namespace rmq
