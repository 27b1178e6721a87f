// query.cuh -- device code of BbST query answering (Sec. 3.1 step 4), shared
// by the plain form (over A) and the contracted form (over A_Q).
#pragma once

#include "rmq_internal.cuh"

namespace rmq {

// Work counters of the instrumented query kernel (rmq_batch_counted), which
// counts what phase B reads: NoCount compiles to nothing; Count keeps each
// thread's counts in registers, and the kernel adds them up at its end.
struct NoCount {
    static constexpr bool on = false;
    __device__ __forceinline__ void add(int, int64_t) const {}
};
struct Count {
    static constexpr bool on = true;
    mutable unsigned long long v[CNT_N] = {0, 0, 0, 0, 0};
    __device__ __forceinline__ void add(int i, int64_t x) const { v[i] += (unsigned long long)x; }
};

// A partial-block scan still to do: inclusive index range [lo, hi] of the
// source sequence, and the hi32 of the block minimum that contains it (the
// smallest value the scan can possibly meet).
struct Pending {
    int64_t lo = 0, hi = -1;
    uint32_t lb = 0;
};

// Edge parts a CTA's warps defer to the end of the kernel, when all its
// warps drain them together: the number of parts per warp varies a lot
// (about 1.6 on average for a uniform batch, up to 8 on some warps), and a
// warp that drained its own parts at once would hold the whole kernel back.
// A part's result is combined into its query's entry with a shared-memory
// atomicMin; the entries' answers are written after the drain.
constexpr int kPoolParts = 256;
constexpr int kPoolQueries = 256;
struct PartPool {
    uint32_t lo[kPoolParts], hi[kPoolParts], lb[kPoolParts];
    uint16_t q[kPoolParts];
    unsigned long long best[kPoolQueries];
    uint32_t qid[kPoolQueries];
    int nparts, nq;   // reserved so far (may exceed the capacities)
};

// Step 4 on the block table for one valid (sub)query, before any scan.
// [lo, hi] is the range in the source's index space; [la, ra] bound its ends
// in A's positions (equal to [lo, hi] for the plain form; for A_Q, entry j
// covers A[P_j .. P_{j+1}], so a key whose position lies in [la, ra] is always
// attained inside the range; a caller passes la = 0 or ra = UINT32_MAX for an
// end that is a whole block inside the query).
//
//   * blocks bl = lo/k, br = hi/k;
//   * m' = min over the blocks strictly between them, from two overlapping
//     table lookups at level t = floor(log2(br - bl - 1));
//   * speculative reads of the two end-block minima: an end block is only
//     looked at when its minimum beats m'.  If that minimum's position lies
//     inside the query it is the end part's minimum and no scan is needed
//     (this check is ours; the paper scans whenever the end block wins);
//     otherwise the partial block is queued for a scan.
//   * bl == br: the block minimum answers if it lies in the range, else the
//     range is scanned.
template <class Ctr = NoCount>
__device__ __forceinline__ uint64_t resolve_query(const uint64_t *__restrict__ T, int64_t nb, int logk,
                                                  int64_t lo, int64_t hi, uint32_t la, uint32_t ra,
                                                  Pending &pl, Pending &pr, bool &hl, bool &hr,
                                                  const Ctr &ctr = Ctr{}) {
    const int64_t bl = lo >> logk, br = hi >> logk;
    const unsigned long long *Tu = reinterpret_cast<const unsigned long long *>(T);
    ctr.add(CNT_TABLE, bl == br ? 1 : (br - bl >= 2 ? 4 : 2));
    if (bl == br) {
        const uint64_t t0 = __ldg(Tu + bl);
        const uint32_t p = key_pos(t0);
        if (p >= la && p <= ra) return t0;
        pl.lo = lo; pl.hi = hi; pl.lb = key_hi(t0);
        hl = true;
        return KEY_MAX;
    }
    uint64_t best = KEY_MAX;
    const uint64_t tl = __ldg(Tu + bl);
    const uint64_t tr = __ldg(Tu + br);
    if (br - bl >= 2) {
        const int t = ilog2_dev((uint64_t)(br - bl - 1));
        const int64_t row = (int64_t)t * nb;
        best = kmin(__ldg(Tu + row + bl + 1), __ldg(Tu + row + br - (1ll << t)));
    }
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

// The same step one level up, on the coarse summary in shared memory (coarse
// blocks of 2^lc blocks).  Returns the best key found so far and which parts
// still need the block table: the whole range (when it lies in one coarse
// block whose minimum is outside it), or the part in the left / right end
// coarse block (when that block's minimum beats the inner coarse span but
// lies outside the query).
enum : int { SUB_NONE = 0, SUB_WHOLE = 1, SUB_LEFT = 2, SUB_RIGHT = 4 };

__device__ __forceinline__ uint64_t resolve_coarse(const uint64_t *cs, const Coarse &g, int logk, uint32_t lo,
                                                   uint32_t hi, uint32_t la, uint32_t ra, int &sub) {
    // all indices fit in 32 bits: positions < 2^31, coarse blocks < kCoarseCap
    const int sh = logk + g.lc;
    const uint32_t BL = lo >> sh, BR = hi >> sh;
    if (BL == BR) {
        const uint64_t c0 = cs[BL];
        const uint32_t p = key_pos(c0);
        if (p >= la && p <= ra) { sub = SUB_NONE; return c0; }
        sub = SUB_WHOLE;
        return KEY_MAX;
    }
    sub = SUB_NONE;
    uint64_t best = KEY_MAX;
    if (BR - BL >= 2) {
        const int t = 31 - __clz((int)(BR - BL - 1));
        const uint64_t *row = cs + g.row32(t);
        best = kmin(row[BL + 1], row[BR - (1u << t)]);
    }
    const uint64_t cl = cs[BL], cr = cs[BR];
    if (cl < best) {
        if (key_pos(cl) >= la) best = cl;
        else sub |= SUB_LEFT;
    }
    if (cr < best) {
        if (key_pos(cr) <= ra) best = cr;
        else sub |= SUB_RIGHT;
    }
    return best;
}

// Minimum key over src[lo .. hi], computed by the whole warp (all 32 lanes
// call it with the same arguments).  Lanes read consecutive 16-byte vectors;
// the scan stops early once some lane has met the value `lb`, the minimum of
// the enclosing block: nothing further right can then be smaller.
template <class Src, bool VEC, class Ctr = NoCount>
__device__ __forceinline__ uint64_t warp_scan_min(const Src &src, int64_t n, int64_t lo, int64_t hi, uint32_t lb,
                                                  const Ctr &ctr = Ctr{}) {
    constexpr int EPV = Src::EPV;
    const int lane = threadIdx.x & 31;
    uint64_t best = KEY_MAX;
    const int64_t vlo = lo / EPV, vhi = hi / EPV;
    const int64_t nvfull = n / EPV;  // vectors that lie wholly inside [0, n)
    constexpr int U = EPV == 2 ? 4 : 2;   // vectors per lane and round (8-byte keys: 256 per round)
    for (int64_t v0 = vlo; v0 <= vhi; v0 += 32 * U) {
#pragma unroll
        for (int x = 0; x < U; ++x) {
            const int64_t vi = v0 + x * 32 + lane;
            if (vi <= vhi) {
                uint64_t kk[EPV];
                ctr.add(CNT_ELEMS, EPV);
                if (vi < nvfull) {
                    src.template vec<VEC>(vi, kk);
                } else {
#pragma unroll
                    for (int e = 0; e < EPV; ++e) {
                        const int64_t i = vi * EPV + e;
                        kk[e] = (i < n) ? src.one(i) : KEY_MAX;
                    }
                }
#pragma unroll
                for (int e = 0; e < EPV; ++e) {
                    const int64_t i = vi * EPV + e;
                    if (i >= lo && i <= hi) best = kmin(best, kk[e]);
                }
            }
        }
        if (__any_sync(0xffffffffu, key_hi(best) == lb)) break;
    }
    return warp_min(best);
}

// Minimum key of A[lo .. hi] (clipped to [0, n)) over the lanes' vectors
// vlo + lane, vlo + lane + 32, ...: a part of at most 128 cells costs one
// load per lane (two for the lane at an unaligned end).
template <bool VEC, class Ctr = NoCount>
__device__ __forceinline__ uint64_t lane_part_min(const SrcI32 &src, int64_t n, int64_t lo, int64_t hi,
                                                  const Ctr &ctr = Ctr{}) {
    const int lane = threadIdx.x & 31;
    uint64_t m = KEY_MAX;
    const int64_t nvfull = n / 4;
    for (int64_t vi = lo / 4 + lane; vi <= hi / 4; vi += 32) {
        uint64_t kk[4];
        ctr.add(CNT_ELEMS, 4);
        if (vi < nvfull) {
            src.template vec<VEC>(vi, kk);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) kk[e] = vi * 4 + e < n ? src.one(vi * 4 + e) : KEY_MAX;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t i = vi * 4 + e;
            if (i >= lo && i <= hi) m = kmin(m, kk[e]);
        }
    }
    return m;
}

// Minimum key over A[lo .. hi], a part of one block, with the minima M1 of
// the small blocks of k1 = 2^logk1 cells of the two-level layout (Sec. 3.3):
// the small blocks strictly inside come from M1; an end small block's
// minimum is taken when it lies in the range, else (and only when it could
// matter) its part of at most k1 cells is scanned.  Two rounds of loads for
// k1 <= 128 and k / k1 <= 32: M1, then the end parts.  The whole warp calls
// it with the same arguments.
template <bool VEC, class Ctr = NoCount>
__device__ __forceinline__ uint64_t warp_range_min_m1(const SrcI32 &src, const uint64_t *__restrict__ M1, int logk1,
                                                      int64_t n, int64_t lo, int64_t hi, const Ctr &ctr = Ctr{}) {
    const int lane = threadIdx.x & 31;
    const unsigned long long *Mu = reinterpret_cast<const unsigned long long *>(M1);
    const int64_t ml = lo >> logk1, mh = hi >> logk1;
    uint64_t best = KEY_MAX;
    bool scan_l = false, scan_r = false;
    int64_t l_end = hi, r_beg = lo;
    if (lane == 0) ctr.add(CNT_M1, mh - ml + 1);   // the loads below, counted once per warp
    if (ml == mh) {
        const uint64_t e0 = __ldg(Mu + ml);
        const uint32_t p = key_pos(e0);
        if (p >= lo && p <= hi) return e0;
        scan_l = true;                              // the whole range, at most k1 cells
    } else {
        uint64_t inner = KEY_MAX;
        for (int64_t j = ml + 1 + lane; j < mh; j += 32) inner = kmin(inner, __ldg(Mu + j));
        const uint64_t el = __ldg(Mu + ml), er = __ldg(Mu + mh);
        best = warp_min(inner);
        if (el < best) {
            if (key_pos(el) >= lo) best = el;
            else scan_l = true;
        }
        if (er < best) {
            if (key_pos(er) <= hi) best = er;
            else scan_r = true;
        }
        l_end = ((ml + 1) << logk1) - 1;
        r_beg = mh << logk1;
    }
    uint64_t sc = KEY_MAX;
    if (scan_l) sc = lane_part_min<VEC>(src, n, lo, l_end, ctr);
    if (scan_r) sc = kmin(sc, lane_part_min<VEC>(src, n, r_beg, hi, ctr));
    return kmin(best, warp_min(sc));
}

// Run every queued scan of the warp.  Long scans, or a single one, run one at
// a time on the whole warp (warp_scan_min).  When several are queued and all
// are short enough for one round of a smaller team, the warp splits into 2 or
// 4 teams of 16 or 8 lanes that run as many scans at once (consecutive-lane
// 16-byte vectors, two per lane), so that their latencies overlap.
// With M1 (the int32 source only), a scan of a part of a block goes through
// warp_range_min_m1 instead.
template <class Src, bool VEC, class Ctr = NoCount>
__device__ __forceinline__ void warp_drain_scans(const Src &src, int64_t n, bool has, const Pending &p,
                                                 uint64_t &best, const uint64_t *M1 = nullptr, int logk1 = 7,
                                                 int max_teams = 4, const Ctr &ctr = Ctr{}) {
    constexpr int EPV = Src::EPV;
    const int lane = threadIdx.x & 31;
    unsigned pend = __ballot_sync(0xffffffffu, has);
    const int64_t nvfull = n / EPV;
    if (!pend) return;
    // the longest queued scan, in 16-byte vectors, decides whether teams pay
    int fit = 1;
    if (pend & (pend - 1)) {
        const uint32_t len = has ? (uint32_t)(p.hi / EPV - p.lo / EPV + 1) : 0u;
        const uint32_t maxlen = __reduce_max_sync(0xffffffffu, len);
        fit = maxlen <= 16u ? 4 : (maxlen <= 32u ? 2 : 1);   // teams whose one round covers it
        fit = min(fit, max_teams);                           // lanes per scan at least 32 / max_teams
    }
    while (pend) {
        const int cnt = __popc(pend);
        if (cnt == 1 || fit == 1) {
            const int s = __ffs(pend) - 1;
            pend &= pend - 1;
            const int64_t lo = __shfl_sync(0xffffffffu, p.lo, s);
            const int64_t hi = __shfl_sync(0xffffffffu, p.hi, s);
            const uint32_t lb = __shfl_sync(0xffffffffu, p.lb, s);
            uint64_t v;
            if constexpr (EPV == 4) {
                v = M1 ? warp_range_min_m1<VEC>(src, M1, logk1, n, lo, hi, ctr) : warp_scan_min<Src, VEC>(src, n, lo, hi, lb, ctr);
            } else {
                v = warp_scan_min<Src, VEC>(src, n, lo, hi, lb, ctr);
            }
            if (lane == s) best = kmin(best, v);
            continue;
        }
        const int nteams = cnt >= 4 ? fit : min(2, fit);
        const int ts = 32 / nteams;                  // lanes per team
        const int team = lane / ts, tl = lane % ts;
        // the scans taken now: the nteams lowest pending lanes
        unsigned taken = 0, x = pend;
        for (int t = 0; t < nteams && x; ++t) {
            taken |= x & (~x + 1u);
            x &= x - 1;
        }
        pend &= ~taken;
        unsigned y = taken;
        for (int t = 0; t < team && y; ++t) y &= y - 1;
        const int s = y ? __ffs(y) - 1 : -1;         // the lane whose scan this team runs
        const int src_lane = s < 0 ? 0 : s;
        const int64_t lo = __shfl_sync(0xffffffffu, p.lo, src_lane);
        const int64_t hi = s < 0 ? lo - 1 : __shfl_sync(0xffffffffu, p.hi, src_lane);
        const uint32_t lb = __shfl_sync(0xffffffffu, p.lb, src_lane);
        const int64_t vlo = lo / EPV, vhi = hi / EPV;
        const unsigned tmask = (ts == 32 ? 0xffffffffu : ((1u << ts) - 1u)) << (team * ts);
        uint64_t tb = KEY_MAX;
        bool live = s >= 0 && hi >= lo;
        for (int64_t v0 = vlo; __any_sync(0xffffffffu, live); v0 += 2 * ts) {
            if (live) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t vi = v0 + u * ts + tl;
                    if (vi <= vhi) {
                        uint64_t kk[EPV];
                        ctr.add(CNT_ELEMS, EPV);
                        if (vi < nvfull) {
                            src.template vec<VEC>(vi, kk);
                        } else {
#pragma unroll
                            for (int e = 0; e < EPV; ++e) kk[e] = vi * EPV + e < n ? src.one(vi * EPV + e) : KEY_MAX;
                        }
#pragma unroll
                        for (int e = 0; e < EPV; ++e) {
                            const int64_t i = vi * EPV + e;
                            if (i >= lo && i <= hi) tb = kmin(tb, kk[e]);
                        }
                    }
                }
            }
            // a team stops when its range is done or it met its block minimum
            const unsigned met = __ballot_sync(0xffffffffu, live && key_hi(tb) == lb) & tmask;
            if (v0 + 2 * ts > vhi || met) live = false;
        }
        for (int off = ts / 2; off > 0; off >>= 1) tb = kmin(tb, __shfl_xor_sync(0xffffffffu, tb, off));
        // the lane of each taken scan collects its team's result
        const bool mine = (taken >> lane) & 1u;
        const int my_team = __popc(taken & ((1u << lane) - 1u));
        const uint64_t v = __shfl_sync(0xffffffffu, tb, (mine ? my_team : 0) * ts);
        if (mine) best = kmin(best, v);
    }
}

// Build the coarse table in shared memory from level lc of the block table
// (Sec. 3.3's upper level): level 0 holds the coarse block minima (the last,
// partial coarse block from two overlapping lookups of a lower level), the
// levels above come by doubling.  Ends with a barrier.
__device__ __forceinline__ void build_coarse(uint64_t *cs, const uint64_t *__restrict__ T, int64_t nb, const Coarse &g) {
    const unsigned long long *Tu = reinterpret_cast<const unsigned long long *>(T);
    for (int J = threadIdx.x; J < g.nbc; J += blockDim.x) {
        uint64_t v;
        if (J < g.nbc_full) {
            v = __ldg(Tu + (int64_t)g.lc * nb + ((int64_t)J << g.lc));
        } else {
            const int64_t s0 = (int64_t)J << g.lc;
            const int tt = ilog2_dev((uint64_t)(nb - s0));
            v = kmin(__ldg(Tu + (int64_t)tt * nb + s0), __ldg(Tu + (int64_t)tt * nb + nb - (1ll << tt)));
        }
        cs[J] = v;
    }
    __syncthreads();
    for (int t = 1; t < g.lvc; ++t) {
        const int half = 1 << (t - 1), cnt = (int)g.nbc - (1 << t) + 1;
        uint64_t *cur = cs + g.row(t);
        const uint64_t *prev = cs + g.row(t - 1);
        for (int J = threadIdx.x; J < cnt; J += blockDim.x) cur[J] = kmin(prev[J], prev[J + half]);
        __syncthreads();
    }
}

// Copy the coarse table into shared memory: each thread has 8 loads in
// flight before it stores them.
__device__ __forceinline__ void load_coarse(uint64_t *cs, const uint64_t *__restrict__ Cs, int total) {
    constexpr int PER = 8;
    for (int b = 0; b < total; b += PER * (int)blockDim.x) {
        uint64_t tmp[PER];
#pragma unroll
        for (int x = 0; x < PER; ++x) {
            const int i = b + threadIdx.x + x * (int)blockDim.x;
            tmp[x] = i < total ? __ldg(reinterpret_cast<const unsigned long long *>(Cs) + i) : 0ull;
        }
#pragma unroll
        for (int x = 0; x < PER; ++x) {
            const int i = b + threadIdx.x + x * (int)blockDim.x;
            if (i < total) cs[i] = tmp[x];
        }
    }
}

// ------------------------------------------------------------ query kernel
// Phase A settles most queries from the coarse table in shared memory alone;
// phase B finishes the others on the block table and with edge scans.

// Phase A's test: the minimum over the coarse blocks BL .. BR the query touches,
// from two reads of the coarse table.  When its position lies inside the
// query it is the answer; this settles most queries of a long batch.
__device__ __forceinline__ bool coarse_blocks_min(const uint64_t *cs, const Coarse &g, uint32_t BL, uint32_t BR,
                                                  uint32_t la, uint32_t ra, uint64_t &m) {
    const int t = 31 - __clz((int)(BR - BL + 1));
    const uint64_t *row = cs + g.row32(t);
    m = kmin(row[BL], row[BR + 1 - (1u << t)]);
    const uint32_t p = key_pos(m);
    return p >= la && p <= ra;
}

// The same test for a range [lo, hi] of the source, its coarse blocks taken
// from the indices.
__device__ __forceinline__ bool coarse_span_min(const uint64_t *cs, const Coarse &g, int logk, uint32_t lo, uint32_t hi,
                                                uint32_t la, uint32_t ra, uint64_t &m) {
    const int sh = logk + g.lc;
    return coarse_blocks_min(cs, g, lo >> sh, hi >> sh, la, ra, m);
}

// Rank of a marked position p in the endpoint bitmap: the number of distinct
// endpoint positions below p, i.e. the index of p in the sorted list P.
// BW[w] is bit word w (bit b set: position 32w + b is an endpoint) and BC[w]
// the number of set bits in the words before w.
__device__ __forceinline__ uint32_t bitmap_rank(const uint32_t *__restrict__ BW, const uint32_t *__restrict__ BC,
                                                uint32_t p) {
    return __ldg(BC + (p >> 5)) + __popc(__ldg(BW + (p >> 5)) & ((1u << (p & 31)) - 1u));
}

// Coarse block of A_Q holding the A_Q entry that begins at the last mark
// <= p (p >= P_0): the last j with CP[j] <= p, searched between the bucket
// bounds CB[p >> bs] and CB[(p >> bs) + 1] (usually equal or adjacent),
// which cbp[i] holds as one word (low and high 16 bits).
__device__ __forceinline__ uint32_t coarse_of(const uint32_t *cp, const uint32_t *cbp, int bs, uint32_t p) {
    const uint32_t pr = cbp[p >> bs];
    uint32_t lo = pr & 0xffffu, hi = pr >> 16;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (cp[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Phase B of the query kernel for `take` (<= 32) queued queries whose indices
// are at q_ids: each lane resolves one on the fine table, then the warp runs
// the edge scans.
template <class Src, bool CON, bool VEC, class Ctr>
__device__ __forceinline__ void resolve_queued(const Src src, int64_t n, int logk, const uint64_t *__restrict__ T,
                                            int64_t nb, const uint64_t *cs, const Coarse g,
                                            const int32_t *__restrict__ L, const int32_t *__restrict__ R,
                                            const uint32_t *__restrict__ BW, const uint32_t *__restrict__ BC,
                                            int32_t *__restrict__ out,
                                            const uint32_t *q_ids, int take, const uint64_t *M1,
                                            int logk1, int max_teams, PartPool *pool, const Ctr &ctr) {
    const int lane = threadIdx.x & 31;
    const int sh = logk + g.lc;
    const bool has = lane < take;
    Pending pl, pr;
    bool hl = false, hr = false;
    uint64_t best = KEY_MAX;
    uint32_t qid = 0;
    int sub = SUB_NONE;
    int64_t r_lo = 0, r_hi = -1, r_start = 0, hi_q = -1;
    uint32_t r_la = 0, r_ra = 0, r_r = 0;
    if (has) {
        qid = q_ids[lane];
        ctr.add(CNT_OPEN, 1);
        if (CON) ctr.add(CNT_RANKS, 4);   // bit word and count of each end
        const int32_t l = L[qid], r = R[qid];
        const int64_t lo = CON ? (int64_t)bitmap_rank(BW, BC, (uint32_t)l) : l;
        const int64_t hi = CON ? (int64_t)bitmap_rank(BW, BC, (uint32_t)r) - 1 : r;
        hi_q = hi;
        best = resolve_coarse(cs, g, logk, (uint32_t)lo, (uint32_t)hi, (uint32_t)l, (uint32_t)r, sub);
        const int64_t end_l = (((lo >> sh) + 1) << sh) - 1, start_r = (hi >> sh) << sh;
        // the first (sub)range on the block table: the whole range, else the
        // left end part, else the right end part; a part ending at a whole
        // coarse block takes that end as inside (la = 0 or ra = ~0), so it
        // leaves at most one scan, in the first slot (a part inside one
        // block) or the second
        r_lo = sub == SUB_WHOLE || (sub & SUB_LEFT) ? lo : start_r;
        r_hi = sub == SUB_WHOLE ? hi : ((sub & SUB_LEFT) ? end_l : hi);
        r_la = sub == SUB_WHOLE || (sub & SUB_LEFT) ? (uint32_t)l : 0u;
        r_ra = sub == SUB_WHOLE ? (uint32_t)r : ((sub & SUB_LEFT) ? 0xffffffffu : (uint32_t)r);
        r_start = start_r;
        r_r = (uint32_t)r;
    }
    // one call site for the first resolution of every lane that needs one
    if (has && sub != SUB_NONE)
        best = kmin(best, resolve_query(T, nb, logk, r_lo, r_hi, r_la, r_ra, pl, pr, hl, hr, ctr));
    // both end parts: the right one second; the left one used only the first slot
    if (has && (sub & SUB_LEFT) && (sub & SUB_RIGHT)) {
        Pending a, b;
        bool ha = false, hb = false;
        best = kmin(best, resolve_query(T, nb, logk, r_start, hi_q, 0u, r_r, a, b, ha, hb, ctr));
        if (ha) { pr = a; hr = true; }
        if (hb) { pr = b; hr = true; }
    }
    // a query with edge parts goes to the CTA's pool when both fit; its
    // answer is then written after the pool's drain
    bool defer = false;
    const int np = (hl ? 1 : 0) + (hr ? 1 : 0);
    if (np) {
        const int pi = atomicAdd(&pool->nparts, np);
        const int qi = atomicAdd(&pool->nq, 1);
        defer = pi + np <= kPoolParts && qi < kPoolQueries;
        if (defer) {
            pool->qid[qi] = qid;
            pool->best[qi] = best;
        } else if (qi < kPoolQueries) {
            pool->qid[qi] = 0xffffffffu;   // reserved, unused
        }
        int w = pi;
        for (int side = 0; side < 2; ++side) {
            if (!(side == 0 ? hl : hr)) continue;
            if (w < kPoolParts) {
                const Pending &pp = side == 0 ? pl : pr;
                pool->lo[w] = defer ? (uint32_t)pp.lo : 1u;   // 1 > 0: an empty part
                pool->hi[w] = defer ? (uint32_t)pp.hi : 0u;
                pool->lb[w] = pp.lb;
                pool->q[w] = (uint16_t)(defer ? qi : 0);
            }
            ++w;
        }
    }
    // the two slots' scans, by one copy of the drain
#pragma unroll 1
    for (int side = 0; side < 2; ++side)
        warp_drain_scans<Src, VEC>(src, n, (side == 0 ? hl : hr) && !defer, side == 0 ? pl : pr, best, M1, logk1,
                                   max_teams, ctr);
    if (has && !defer) out[qid] = (int32_t)key_pos(best);
    __syncwarp();
}

// The CTA's warps drain the pooled edge parts (warp w takes parts w, w + W,
// ...), then write the pooled queries' answers.  Called by all threads of
// the CTA, after every warp has finished its queries.
template <class Src, bool VEC, class Ctr>
__device__ __forceinline__ void drain_pool(const Src src, int64_t n, const uint64_t *M1, int logk1, PartPool *pool,
                                           int32_t *__restrict__ out, const Ctr &ctr) {
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int parts = min(pool->nparts, kPoolParts);
    for (int p = w; p < parts; p += nw) {
        const uint32_t lo = pool->lo[p], hi = pool->hi[p];
        if (lo > hi) continue;   // reserved, unused
        uint64_t v;
        if constexpr (Src::EPV == 4) {
            v = M1 ? warp_range_min_m1<VEC>(src, M1, logk1, n, lo, hi, ctr)
                   : warp_scan_min<Src, VEC>(src, n, lo, hi, pool->lb[p], ctr);
        } else {
            v = warp_scan_min<Src, VEC>(src, n, lo, hi, pool->lb[p], ctr);
        }
        if (lane == 0) atomicMin(&pool->best[pool->q[p]], (unsigned long long)v);
    }
    __syncthreads();
    const int nq = min(pool->nq, kPoolQueries);
    for (int e = threadIdx.x; e < nq; e += blockDim.x) {
        const uint32_t qid = pool->qid[e];
        if (qid != 0xffffffffu) out[qid] = (int32_t)key_pos(pool->best[e]);
    }
}

//   plain (CON = false): the source is A; query i covers [l_i, r_i].
//   contracted (CON = true): the source is A_Q; query i covers
//     A_Q[a_i .. b_i - 1] with a_i, b_i the ranks of l_i, r_i in the
//     endpoint bitmap (BW, BC); a_i == b_i means l_i == r_i and the answer is l_i.
//     Phase A needs only the coarse blocks of a_i and b_i - 1, which the
//     coarse index (CP, CB) gives from l_i and r_i - 1; the ranks themselves
//     are looked up in the bitmap for the queries left to phase B.
//   cap: the coarse geometry of the table (coarse_geom(nb, cap)).
// Dynamic shared memory: for the plain form with VECQ, each warp's ring of
// the l, r of its next kQueryRing steps (query_ring_bytes in all), then the
// coarse table (coarse_geom(...).size() keys at most).  The contracted form
// loads the next step's l, r into registers instead: the ring's 64 KB per SM
// cost its phase B more than the deeper prefetch saved.
constexpr int kQueryRing = 4;
template <bool CON, bool VECQ>
__host__ __device__ constexpr bool query_uses_ring() { return VECQ && !CON; }
template <bool CON, bool VECQ>
__host__ __device__ constexpr size_t query_ring_bytes() {
    return query_uses_ring<CON, VECQ>() ? (size_t)(kQueryThreads / 32) * kQueryRing * 2 * 32 * 16 : 0;
}

template <class Src, bool CON, bool VECQ, bool VEC, class Ctr = NoCount>
__global__ void __launch_bounds__(kQueryThreads, kQueryCtasPerSm)
k_query_two(Src src, Len len, int logk, int cap, const uint64_t *__restrict__ T,
                                                    const uint64_t *__restrict__ Cs,
                                                    const int32_t *__restrict__ L, const int32_t *__restrict__ R,
                                                    const uint32_t *__restrict__ BW, const uint32_t *__restrict__ BC,
                                                    const uint32_t *__restrict__ CP,
                                                    const uint16_t *__restrict__ CB, const uint64_t *__restrict__ M1,
                                                    int logk1, int max_teams,
                                                    int64_t n_a, int32_t *__restrict__ out, int64_t q,
                                                    unsigned *err, unsigned long long *counts) {
    const Ctr ctr{};
    // Phase A answers the queries the coarse table settles.  Each warp queues
    // the others (their indices) in its own shared-memory queue, and as soon
    // as 32 are queued it resolves them (phase B: fine table and edge scans),
    // so the latency of that work overlaps the streaming of other warps.
    constexpr int kQueue = 160;   // a step adds at most 128
    constexpr bool RING = query_uses_ring<CON, VECQ>();
    constexpr int kRing = kQueryRing;
    extern __shared__ __align__(16) uint64_t query_dyn_smem[];
    int4 *ring = reinterpret_cast<int4 *>(query_dyn_smem);
    uint64_t *cs = query_dyn_smem + query_ring_bytes<CON, VECQ>() / sizeof(uint64_t);
    __shared__ uint32_t cp[CON ? kCoarseBlocksMax : 1];
    __shared__ uint32_t cbp[CON ? kBucketsMax : 1];   // bucket bounds (CB[i], CB[i + 1])
    __shared__ uint32_t queue[kQueryThreads / 32][kQueue];
    __shared__ PartPool pool;
    if (threadIdx.x == 0) pool.nparts = pool.nq = 0;   // visible after the barrier below
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // RING: the l, r of the warp's next kRing steps are in flight at any
    // time: each lane copies its 16 bytes of l and of r into its slots of the
    // warp's ring (one commit group per step, empty past the end of the
    // batch).  Otherwise the next step's l, r are loaded into registers
    // before the current step is processed.  The first loads are issued
    // before the coarse table is built, so that they overlap its build.
    const int64_t stride = nwarps * 128;
    int4 *wring = ring + (threadIdx.x >> 5) * (kRing * 64);
    const uint32_t ring_sh = RING ? (uint32_t)__cvta_generic_to_shared(wring) : 0u;
    auto issue = [&](int64_t b, int slot) {
        if (b + 3 < q) {
            cp_async16(ring_sh + (uint32_t)(slot * 64 + lane) * 16u, L + b);
            cp_async16(ring_sh + (uint32_t)(slot * 64 + 32 + lane) * 16u, R + b);
        }
        cp_async_commit();
    };
    int4 p0 = make_int4(0, 0, 0, 0), p1 = p0;
    auto fetch = [&](int64_t b) {
        if (VECQ && b + 3 < q) {
            p0 = __ldcs(reinterpret_cast<const int4 *>(L + b));
            p1 = __ldcs(reinterpret_cast<const int4 *>(R + b));
        }
    };
    if (RING) {
#pragma unroll
        for (int j = 0; j < kRing; ++j) issue(warp * 128 + j * stride + lane * 4, j);
    } else {
        fetch(warp * 128 + lane * 4);
    }
    // l and r are the caller's: they are requested above, before the wait
    // for the kernels of this call that build the table (and, for the
    // contracted form, write the length of A_Q)
    pdl_wait();
    const int64_t n = len.get();
    const int64_t nb = (n + (1ll << logk) - 1) >> logk;
    const Coarse g = coarse_geom(nb, cap);
    // the contracted form's coarse index (read before the table is built,
    // whose barriers it does not need)
    const int bs = CON ? bucket_shift(n_a) : 0;
    if (CON && nb > 0) {
        for (int i = threadIdx.x; i < g.nbc; i += blockDim.x) cp[i] = __ldg(CP + i);
        const int nbk = (int)bucket_count(n_a);
        for (int i = threadIdx.x; i < nbk; i += blockDim.x)
            cbp[i] = (uint32_t)__ldg(CB + i) | ((uint32_t)__ldg(CB + i + 1) << 16);
    }
    // the coarse table: copied when the caller keeps one, else built here
    if (Cs) load_coarse(cs, Cs, (int)g.size());
    else if (nb > 0) build_coarse(cs, T, nb, g);
    __syncthreads();
    uint32_t *my = queue[threadIdx.x >> 5];
    int nq = 0;   // queued (warp-uniform)
    const int sh = logk + g.lc;
    auto resolve = [&](int take) {
        resolve_queued<Src, CON, VEC>(src, n, logk, T, nb, cs, g, L, R, BW, BC, out, my + nq - take, take, M1,
                                      logk1, max_teams, &pool, ctr);
        nq -= take;
    };
    int slot = 0;
    const int32_t na = (int32_t)n_a;
    for (int64_t wb = warp * 128; wb < q; wb += stride) {
        const int64_t base = wb + lane * 4;
        const bool full = VECQ && base + 3 < q;
        int32_t lq[4], rq[4];
        if (RING) {
            cp_async_wait<kRing - 1>();   // this step's copies have landed
            if (full) {
                p0 = wring[slot * 64 + lane];
                p1 = wring[slot * 64 + 32 + lane];
            }
        }
        if (full) {
            lq[0] = p0.x; lq[1] = p0.y; lq[2] = p0.z; lq[3] = p0.w;
            rq[0] = p1.x; rq[1] = p1.y; rq[2] = p1.z; rq[3] = p1.w;
        }
        if (!RING) fetch(base + stride);
        if (!full) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const bool p = base + i < q;
                lq[i] = p ? __ldcs(L + base + i) : 0;
                rq[i] = p ? __ldcs(R + base + i) : -1;   // absent: reads as invalid
            }
        }
        int32_t o[4];
        unsigned need = 0;
        bool bad = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool present = full || base + i < q;
            const bool ok = present && lq[i] >= 0 && rq[i] >= lq[i] && rq[i] < na;
            bad |= present && !ok;
            const bool single = CON && ok && lq[i] == rq[i];          // contracted a == b
            // straight-line: an invalid or single query reads block 0 harmlessly
            const bool use = ok && !single;
            uint32_t BL, BR;
            if (CON) {
                BL = use ? coarse_of(cp, cbp, bs, (uint32_t)lq[i]) : 0u;
                BR = use ? coarse_of(cp, cbp, bs, (uint32_t)rq[i] - 1u) : 0u;
            } else {
                BL = use ? (uint32_t)lq[i] >> sh : 0u;
                BR = use ? (uint32_t)rq[i] >> sh : 0u;
            }
            uint64_t m;
            const bool inside = coarse_blocks_min(cs, g, BL, BR, (uint32_t)lq[i], (uint32_t)rq[i], m);
            o[i] = !ok ? -1 : (single ? lq[i] : (inside ? (int32_t)key_pos(m) : -1));
            need |= (use && !inside ? 1u : 0u) << i;
        }
        if (RING) {   // the slot's values are used: it takes the step kRing on
            issue(base + kRing * stride, slot);
            slot = slot + 1 == kRing ? 0 : slot + 1;
        }
        if (full) {
            __stcs(reinterpret_cast<int4 *>(out + base), make_int4(o[0], o[1], o[2], o[3]));
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (base + i < q) out[base + i] = o[i];
        }
        // queue the open queries' indices: slots from four ballots
        const unsigned lt = (1u << lane) - 1u;
        const unsigned b0 = __ballot_sync(0xffffffffu, need & 1u), b1 = __ballot_sync(0xffffffffu, need & 2u);
        const unsigned b2 = __ballot_sync(0xffffffffu, need & 4u), b3 = __ballot_sync(0xffffffffu, need & 8u);
        const int c0 = __popc(b0), c1 = __popc(b1), c2 = __popc(b2), c3 = __popc(b3);
        if (c0 + c1 + c2 + c3) {
            if (need & 1u) my[nq + __popc(b0 & lt)] = (uint32_t)base;
            if (need & 2u) my[nq + c0 + __popc(b1 & lt)] = (uint32_t)(base + 1);
            if (need & 4u) my[nq + c0 + c1 + __popc(b2 & lt)] = (uint32_t)(base + 2);
            if (need & 8u) my[nq + c0 + c1 + c2 + __popc(b3 & lt)] = (uint32_t)(base + 3);
            nq += c0 + c1 + c2 + c3;
            __syncwarp();
            while (nq >= 32) resolve(32);
        }
        if (!CON && bad && err) atomicOr(err, ERR_QUERY_RANGE);
    }
    if (nq > 0) resolve(nq);
    if (RING) cp_async_wait<0>();   // no copy is left in flight (all were empty)
    drain_pool<Src, VEC>(src, n, M1, logk1, &pool, out, ctr);
    if constexpr (Ctr::on) {   // the instrumented kernel: one atomic per warp and counter
#pragma unroll
        for (int i = 0; i < CNT_N; ++i) {
            unsigned long long v = ctr.v[i];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0 && v) atomicAdd(counts + i, v);
        }
    }
}

// Launches k_query_two with `smem` bytes of dynamic shared memory (the ring
// plus at most kCoarseCapMax keys of coarse table); the first launch of each
// instantiation on a device raises the kernel's limit to that maximum.
template <class Src, bool CON, bool VECQ, bool VEC, class Ctr = NoCount, class... Args>
inline cudaError_t launch_query_two(int device, unsigned ctas, size_t smem, cudaStream_t s, Args... args) {
    static std::once_flag once[kMaxDev];
    static cudaError_t raised[kMaxDev];
    auto kern = k_query_two<Src, CON, VECQ, VEC, Ctr>;
    cudaError_t e = cudaSuccess;
    once_per_device(once, device, [&] {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(query_ring_bytes<CON, VECQ>() + kCoarseCapMax * sizeof(uint64_t)));
        if (device >= 0 && device < kMaxDev) raised[device] = e;
    });
    if (device >= 0 && device < kMaxDev) e = raised[device];
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, ctas, kQueryThreads, smem, s, args...);
}

}  // namespace rmq
