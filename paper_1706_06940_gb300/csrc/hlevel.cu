// hlevel.cu -- the multi-level block-based sparse table (Sec. 3.3): block
// sizes k_1 < k_2 < ... < k_h, powers of two, so each divides the next.  The
// minima of the non-overlapping blocks of k_i are kept for i < h (level i),
// and over the blocks of k_h a sparse table (its level 0 being their minima).
// The table shrinks by the factor k_h / k of the one-level form; a query's
// unlucky end parts cost k_h / k_{h-1} + ... + k_2 / k_1 + k_1 reads instead
// of k cells.
//
// Build: the minima of levels 1 and 2 are one pass over A (the block-minima
// kernel of the plain form, which writes the minima of small blocks beside
// those of its blocks); each higher level, and the table's level 0, reduces
// the level below (n / k_2 keys at most, a small fraction of A); the sparse
// table is the plain form's.
//
// Query: one thread per query takes the whole blocks of k_h inside it from
// two table values, then walks each end part down the levels.  At every level
// the part lies inside one block whose minimum is known: a part is skipped
// when that minimum cannot beat the best key so far, and answered by it when
// it lies inside the part (the speculative check of Sec. 3.2, here on every
// level); otherwise the whole sub-blocks one level down are read and the walk
// goes on with the partial one.  Parts left open at level 1 (fewer than k_1
// cells) are scanned by the whole warp together (warp_drain_scans).
#include <algorithm>

#include "query.cuh"

namespace rmq {

namespace {

constexpr int kThreads = 256;
constexpr size_t kSmem = kCoarseCap * sizeof(uint64_t);   // the coarse summary (32 KB)

// Level i of the structure: minima keys of its blocks of 2^logk[i] cells,
// M[i] for 1 <= i < h; the table T over the blocks of level h (level 0 of T,
// nbh entries per table level).
struct HDesc {
    const uint64_t *M[kHLevelMax];   // M[0] unused
    int logk[kHLevelMax + 1];        // logk[1 .. h]
    int h;
    const uint64_t *T;
    int64_t nbh;
    Coarse g;                        // coarse summary of T kept in shared memory
};

__device__ __forceinline__ uint64_t ld_key(const uint64_t *p, int64_t j) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p) + j);
}
__device__ __forceinline__ const uint64_t *level_keys(const HDesc &d, int i) { return i == d.h ? d.T : d.M[i]; }

// Level i from level i - 1: entry j is the minimum of the 2^shift keys j 2^shift
// .. (j + 1) 2^shift - 1 of the level below (fewer for the last block).
__global__ void __launch_bounds__(kThreads) k_level_reduce(const uint64_t *__restrict__ lower, int64_t nlow,
                                                           uint64_t *__restrict__ upper, int64_t nup, int shift) {
    pdl_wait();
    const unsigned long long *lo = reinterpret_cast<const unsigned long long *>(lower);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nup; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = j << shift, e = (j + 1) << shift, b = e < nlow ? e : nlow;
        uint64_t m = KEY_MAX;
        for (int64_t i = a; i < b; ++i) m = kmin(m, __ldg(lo + i));   // levels are 8-byte aligned only
        upper[j] = m;
    }
}

// The part [a, E] of a query, E the last cell of block b of level i whose
// minimum key is m (the suffix chain of a left end).
__device__ __forceinline__ void suffix_chain(const HDesc &d, int i, int64_t a, int64_t E, uint64_t m, uint64_t &best,
                                            Pending &p, bool &has) {
    for (;;) {
        if (m >= best) return;                       // the part cannot win
        if (key_pos(m) >= (uint64_t)a) { best = m; return; }
        if (i == 1) { p.lo = a; p.hi = E; p.lb = key_hi(m); has = true; return; }
        const int s = d.logk[i - 1];
        const uint64_t *Ml = level_keys(d, i - 1);
        const int64_t first = a >> s, last = E >> s;
        for (int64_t j = first + 1; j <= last; ++j) best = kmin(best, ld_key(Ml, j));
        m = ld_key(Ml, first);
        E = ((first + 1) << s) - 1;
        --i;
    }
}

// The part [S, b] of a query, S the first cell of a block of level i whose
// minimum key is m (the prefix chain of a right end).
__device__ __forceinline__ void prefix_chain(const HDesc &d, int i, int64_t S, int64_t b, uint64_t m, uint64_t &best,
                                            Pending &p, bool &has) {
    for (;;) {
        if (m >= best) return;
        if (key_pos(m) <= (uint64_t)b) { best = m; return; }
        if (i == 1) { p.lo = S; p.hi = b; p.lb = key_hi(m); has = true; return; }
        const int s = d.logk[i - 1];
        const uint64_t *Ml = level_keys(d, i - 1);
        const int64_t first = S >> s, last = b >> s;
        for (int64_t j = first; j < last; ++j) best = kmin(best, ld_key(Ml, j));
        m = ld_key(Ml, last);
        S = last << s;
        --i;
    }
}

// One valid query [l, r]: the best key from the structure, and at most two
// level-1 parts still to scan (pl, pr).
__device__ __forceinline__ uint64_t hlevel_resolve(const HDesc &d, int64_t l, int64_t r, Pending &pl, bool &hl,
                                                   Pending &pr, bool &hr) {
    const int lh = d.logk[d.h];
    int64_t bl = l >> lh, br = r >> lh;
    uint64_t best = KEY_MAX;
    if (bl != br) {
        if (br - bl >= 2) {
            const int t = ilog2_dev((uint64_t)(br - bl - 1));
            const int64_t row = (int64_t)t * d.nbh;
            best = kmin(ld_key(d.T, row + bl + 1), ld_key(d.T, row + br - (1ll << t)));
        }
        const uint64_t tl = ld_key(d.T, bl), tr = ld_key(d.T, br);
        suffix_chain(d, d.h, l, ((bl + 1) << lh) - 1, tl, best, pl, hl);
        prefix_chain(d, d.h, br << lh, r, tr, best, pr, hr);
        return best;
    }
    // [l, r] inside one block of level i with minimum m: go down while it
    // stays inside one block; at the first level where it spans several,
    // the whole ones are read and the two ends become chains.
    int i = d.h;
    uint64_t m = ld_key(d.T, bl);
    for (;;) {
        const uint32_t pm = key_pos(m);
        if (pm >= (uint64_t)l && pm <= (uint64_t)r) return m;
        if (i == 1) { pl.lo = l; pl.hi = r; pl.lb = key_hi(m); hl = true; return best; }
        const int s = d.logk[i - 1];
        const uint64_t *Ml = level_keys(d, i - 1);
        bl = l >> s;
        br = r >> s;
        if (bl == br) { m = ld_key(Ml, bl); --i; continue; }
        for (int64_t j = bl + 1; j < br; ++j) best = kmin(best, ld_key(Ml, j));
        const uint64_t ml = ld_key(Ml, bl), mr = ld_key(Ml, br);
        suffix_chain(d, i - 1, l, ((bl + 1) << s) - 1, ml, best, pl, hl);
        prefix_chain(d, i - 1, br << s, r, mr, best, pr, hr);
        return best;
    }
}

// Each CTA first builds the coarse summary of the table over blocks of k_h in
// shared memory (the plain form's upper level); a query whose minimum over
// the coarse blocks it touches lies inside it is answered from there (most
// queries of a long batch), the others walk the levels.  Warps take 32
// consecutive queries at a time (all lanes stay in the loop together so that
// they can scan for one another).  Invalid queries answer -1 and raise the
// error word.
template <bool VEC>
__global__ void __launch_bounds__(kThreads) k_hlevel_query(const int32_t *__restrict__ A, int64_t n,
                                                           const __grid_constant__ HDesc d,
                                                           const int32_t *__restrict__ L, const int32_t *__restrict__ R,
                                                           int64_t q, int32_t *__restrict__ out, unsigned *err) {
    extern __shared__ uint64_t cs[];
    pdl_wait();
    build_coarse(cs, d.T, d.nbh, d.g);
    const SrcI32 src{A};
    const int lane = threadIdx.x & 31;
    const int lh = d.logk[d.h];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    int32_t ln = 0, rn = -1;   // the next batch's query, loaded while this one runs
    if (warp * 32 + lane < q) {
        ln = L[warp * 32 + lane];
        rn = R[warp * 32 + lane];
    }
    for (int64_t base = warp * 32; base < q; base += nwarps * 32) {
        const int64_t i = base + lane;
        const int32_t l = ln, r = rn;
        const int64_t inext = i + nwarps * 32;
        if (inext < q) {
            ln = L[inext];
            rn = R[inext];
        }
        bool valid = false;
        if (i < q) {
            valid = l >= 0 && r >= l && (int64_t)r < n;
            bad |= !valid;
        }
        Pending pl, pr;
        bool hl = false, hr = false;
        uint64_t best = KEY_MAX;
        if (valid) {
            uint64_t m;
            if (coarse_span_min(cs, d.g, lh, (uint32_t)l, (uint32_t)r, (uint32_t)l, (uint32_t)r, m)) best = m;
            else best = hlevel_resolve(d, l, r, pl, hl, pr, hr);
        }
        warp_drain_scans<SrcI32, VEC>(src, n, hl, pl, best);
        warp_drain_scans<SrcI32, VEC>(src, n, hr, pr, best);
        if (i < q) out[i] = valid ? (int32_t)key_pos(best) : -1;
    }
    if (bad) atomicOr(err, ERR_QUERY_RANGE);
}

}  // namespace

int64_t hlevel_entries(int64_t n, const int *logk, int h) {
    if (n <= 0 || h < 1 || h > kHLevelMax) return -1;
    int64_t e = 0;
    for (int i = 1; i < h; ++i) e += cdiv(n, 1ll << logk[i]);
    const int64_t nbh = cdiv(n, 1ll << logk[h]);
    return e + nbh * (ilog2_host((uint64_t)nbh) + 1);
}

cudaError_t run_hlevel(const int32_t *A, int64_t n, const int *logk, int h, const int32_t *l, const int32_t *r,
                       int64_t q, int32_t *out, uint64_t *W, cudaStream_t s) {
    if (h < 1 || h > kHLevelMax || logk[1] < MIN_LOGK || logk[1] > MAX_LOGK) return cudaErrorInvalidValue;
    for (int i = 2; i <= h; ++i)
        if (logk[i] <= logk[i - 1] || logk[i] > kHLevelMaxLogK) return cudaErrorInvalidValue;
    const DevInfo di = dev_info();
    unsigned *err = err_word_ptr(s);
    if (!err) return cudaErrorUnknown;
    HDesc d{};
    d.h = h;
    int64_t nb[kHLevelMax + 1] = {0};
    uint64_t *lev[kHLevelMax + 1] = {nullptr};   // level i's keys; level h: the table's level 0
    uint64_t *p = W;
    for (int i = 1; i <= h; ++i) {
        d.logk[i] = logk[i];
        nb[i] = cdiv(n, 1ll << logk[i]);
        lev[i] = p;
        if (i < h) { d.M[i] = p; p += nb[i]; }
    }
    d.T = lev[h];
    d.nbh = nb[h];
    d.g = coarse_geom(nb[h], kCoarseCap);
    // levels 1 and 2 in one pass over A (the block minima of k_2 with the
    // minima of k_1 beside them) when k_2 <= 65536 and there are blocks of k_2
    // for every warp the GPU holds at once (a warp reduces one block at a
    // time); else level 1 alone
    const bool pair = h >= 2 && logk[2] <= MAX_LOGK && nb[2] >= (int64_t)di.sms * 32;
    cudaError_t e = pair ? launch_block_minima_i32(A, n, logk[2], lev[2], s, lev[1], logk[1])
                         : launch_block_minima_i32(A, n, logk[1], lev[1], s);
    if (e != cudaSuccess) return e;
    for (int i = pair ? 3 : 2; i <= h; ++i) {
        const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(nb[i], kThreads), (int64_t)di.sms * 8));
        launch_pdl(k_level_reduce, (unsigned)ctas, kThreads, 0, s, (const uint64_t *)lev[i - 1], nb[i - 1], lev[i],
                   nb[i], logk[i] - logk[i - 1]);
        note_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = launch_sparse_table(lev[h], Len{n, nullptr}, logk[h], nb[h], s)) != cudaSuccess) return e;
    if (q <= 0) return cudaSuccess;
    // one wave of the CTAs that fit on an SM at once (registers decide), each
    // warp walking the batch in steps of 32 queries
    static std::once_flag once[kMaxDev];
    static int resident[kMaxDev][2];
    once_per_device(once, di.device, [&] {
        int dv = di.device < kMaxDev ? di.device : 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[dv][0], k_hlevel_query<false>, kThreads, kSmem) !=
            cudaSuccess)
            resident[dv][0] = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[dv][1], k_hlevel_query<true>, kThreads, kSmem) !=
            cudaSuccess)
            resident[dv][1] = 1;
    });
    const bool vec = (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const int per_sm = std::max(1, resident[di.device < kMaxDev ? di.device : 0][vec ? 1 : 0]);
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(cdiv(q, kThreads), (int64_t)di.sms * per_sm));
    if (vec)
        launch_pdl(k_hlevel_query<true>, (unsigned)ctas, kThreads, kSmem, s, A, n, d, l, r, q, out, err);
    else
        launch_pdl(k_hlevel_query<false>, (unsigned)ctas, kThreads, kSmem, s, A, n, d, l, r, q, out, err);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace rmq
