// query.cuh -- device code of BbST query answering (Sec. 3.1 step 4), shared
// by the plain form (over A) and the contracted form (over A_Q).
#pragma once

#include "rmq_internal.cuh"

namespace rmq {

// A partial-block scan still to do: inclusive index range [lo, hi] of the
// source sequence, and the hi32 of the block minimum that contains it (the
// smallest value the scan can possibly meet).
struct Pending {
    int64_t lo = 0, hi = -1;
    uint32_t lb = 0;
};

// Step 4 for one valid query, before any scan.  [lo, hi] is the query in the
// source's index space; [la, ra] are its ends in A's positions (equal to
// [lo, hi] for the plain form; for A_Q, entry j covers A[P_j .. P_{j+1}], so a
// key whose position lies in [la, ra] is always attained inside the range).
//
//   * blocks bl = lo/k, br = hi/k;
//   * m' = min over the blocks strictly between them, from two overlapping
//     table lookups at level t = floor(log2(br - bl - 1)) (Sec. 3.1 step 4);
//   * speculative reads of the two end-block minima: an end block is only
//     looked at when its minimum beats m'.  If that minimum's position lies
//     inside the query it is the end part's minimum and no scan is needed
//     (this check is ours; the paper scans whenever the end block wins);
//     otherwise the partial block is queued for a scan.
//   * bl == br: the block minimum answers if it lies in the range, else the
//     range is scanned.
__device__ __forceinline__ uint64_t resolve_query(const uint64_t *__restrict__ T, int64_t nb, int logk,
                                                  int64_t lo, int64_t hi, uint32_t la, uint32_t ra,
                                                  Pending &pl, Pending &pr, bool &hl, bool &hr) {
    const int64_t bl = lo >> logk, br = hi >> logk;
    hl = hr = false;
    if (bl == br) {
        const uint64_t t0 = __ldg(reinterpret_cast<const unsigned long long *>(T) + bl);
        const uint32_t p = key_pos(t0);
        if (p >= la && p <= ra) return t0;
        pl.lo = lo; pl.hi = hi; pl.lb = key_hi(t0);
        hl = true;
        return KEY_MAX;
    }
    uint64_t best = KEY_MAX;
    const unsigned long long *Tu = reinterpret_cast<const unsigned long long *>(T);
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

// Minimum key over src[lo .. hi], computed by the whole warp (all 32 lanes
// call it with the same arguments).  Lanes read consecutive 16-byte vectors;
// the scan stops early once some lane has met the value `lb`, the minimum of
// the enclosing block: nothing further right can then be smaller.
template <class Src, bool VEC>
__device__ __forceinline__ uint64_t warp_scan_min(const Src &src, int64_t n, int64_t lo, int64_t hi, uint32_t lb) {
    constexpr int EPV = Src::EPV;
    const int lane = threadIdx.x & 31;
    uint64_t best = KEY_MAX;
    const int64_t vlo = lo / EPV, vhi = hi / EPV;
    const int64_t nvfull = n / EPV;  // vectors that lie wholly inside [0, n)
    for (int64_t v0 = vlo; v0 <= vhi; v0 += 64) {
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            const int64_t vi = v0 + x * 32 + lane;
            if (vi <= vhi) {
                uint64_t kk[EPV];
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

// Run every queued scan of the warp, one at a time, each with all 32 lanes.
template <class Src, bool VEC>
__device__ __forceinline__ void warp_drain_scans(const Src &src, int64_t n, bool has, const Pending &p,
                                                 uint64_t &best) {
    const int lane = threadIdx.x & 31;
    unsigned pend = __ballot_sync(0xffffffffu, has);
    while (pend) {
        const int s = __ffs(pend) - 1;
        pend &= pend - 1;
        const int64_t lo = __shfl_sync(0xffffffffu, p.lo, s);
        const int64_t hi = __shfl_sync(0xffffffffu, p.hi, s);
        const uint32_t lb = __shfl_sync(0xffffffffu, p.lb, s);
        const uint64_t v = warp_scan_min<Src, VEC>(src, n, lo, hi, lb);
        if (lane == s) best = kmin(best, v);
    }
}

}  // namespace rmq
