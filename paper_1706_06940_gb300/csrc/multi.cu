// multi.cu -- many independent arrays, each with its own batch of queries,
// answered in one persistent kernel launch (plain BbST per array, Sec. 3.2,
// with a coarse level as in Sec. 3.3).
//
// Work is a queue of items taken in order through one atomic counter:
//   phase 1: (array h, 32768 consecutive cells) -- block minima (Sec. 3.1 step 3,
//            level 0) written to the array's T0, and folded with atomicMin into
//            level 0 of its coarse table (coarse blocks of 2^lc blocks);
//            the CTA that finishes the last phase-1 item of array h builds the
//            upper levels of h's coarse table in shared memory and then sets
//            ready[h];
//   phase 3: (array h, 1024 queries) -- waits for ready[h] (a bounded spin: on
//            timeout the item's answers are -1 and the device error word gets
//            ERR_TIMEOUT), copies h's coarse table into shared memory and
//            answers (Sec. 3.1 step 4 on the coarse table; the open end parts
//            on T0 with lane-local scans; partial blocks by warp scans).
// Every phase-1 item precedes every phase-3 item in the queue, so when a CTA
// waits for ready[h] every item h depends on is already held by a running
// CTA that never waits: the wait always ends unless a flag is withheld on
// purpose (the test hook below).
#include <algorithm>

#include "query.cuh"
#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kMT = 256;
constexpr int kLogChunk = 15;             // phase-1 item: 32768 cells of one array (k <= 32768)
constexpr int kQueriesPerItem = 1024;     // 4 per thread
constexpr int kMultiLcMax = 5;            // coarse blocks of at most 32 blocks: short T0 scans

struct MultiDesc {
    const int32_t *A;
    int32_t n;
    int32_t q;
    int32_t logk;
    int32_t pad;
};

struct MultiParams {
    int32_t H;
    uint32_t flags;
    int64_t spin_limit;
    uint64_t *T0;                // concatenated level-0 tables
    uint64_t *Cs;                // H coarse tables of kCoarseCap entries
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

template <class T, class F>
__device__ void array_prefix(T *pre, int H, F count, T *wsum) {
    array_prefix_n<T, kMultiMax>(pre, H, count, wsum);
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

__device__ __forceinline__ int64_t nblocks(const MultiDesc &d) {
    return ((int64_t)d.n + (1ll << d.logk) - 1) >> d.logk;
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

__global__ void __launch_bounds__(kMT, 3) k_multi(const __grid_constant__ MultiParams p) {
    extern __shared__ uint64_t msm[];
    uint64_t *cs = msm;                                             // kCoarseCap
    int64_t *t0off = reinterpret_cast<int64_t *>(cs + kCoarseCap);   // kMultiMax + 1
    int64_t *qoff = t0off + kMultiMax + 1;                           // kMultiMax + 1
    int32_t *pre1 = reinterpret_cast<int32_t *>(qoff + kMultiMax + 1);
    int32_t *pre3 = pre1 + kMultiMax + 1;
    __shared__ int64_t wsum64[kMT / 32];
    __shared__ int32_t wsum32[kMT / 32];
    __shared__ long long s_item;
    __shared__ int s_flag;
    const int H = p.H;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

    array_prefix<int64_t>(t0off, H, [&](int h) { return p.d[h].q > 0 ? nblocks(p.d[h]) : 0ll; }, wsum64);
    array_prefix<int64_t>(qoff, H, [&](int h) { return (int64_t)p.d[h].q; }, wsum64);
    array_prefix<int32_t>(pre1, H, [&](int h) {
        return p.d[h].q > 0 ? (int32_t)(((int64_t)p.d[h].n + (1 << kLogChunk) - 1) >> kLogChunk) : 0; }, wsum32);
    array_prefix<int32_t>(pre3, H, [&](int h) { return (p.d[h].q + kQueriesPerItem - 1) / kQueriesPerItem; }, wsum32);
    const int64_t tot1 = pre1[H], tot3 = pre3[H];

    // thread 0 asks for the next item while the CTA works on the current one
    long long ahead = 0;
    if (threadIdx.x == 0) ahead = (long long)atomicAdd(p.next, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = ahead;
            if (ahead < tot1 + tot3) ahead = (long long)atomicAdd(p.next, 1ull);
        }
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= tot1 + tot3) break;
        if (item < tot1) {
            // ---------------------------------------------------- phase 1
            const int h = find_array<int32_t>(pre1, H, (int32_t)item);
            const MultiDesc d = p.d[h];
            const int64_t nb = nblocks(d);
            const Coarse g = coarse_geom(nb);
            const int64_t c0 = (item - pre1[h]) << kLogChunk;
            const int64_t c1 = min((int64_t)d.n, (int64_t)(c0 + (1ll << kLogChunk)));
            const int64_t K = 1ll << d.logk;
            const bool aligned = (reinterpret_cast<uintptr_t>(d.A) & 15) == 0;
            uint64_t *T0h = p.T0 + t0off[h];
            unsigned long long *C0 = reinterpret_cast<unsigned long long *>(p.Cs + (int64_t)h * kCoarseCap);
            const int64_t s0 = c0 + (int64_t)w * 4096;  // this warp's slice: 32 rows of 32 16-byte vectors
            if (K <= 2048 && aligned && s0 + 4096 <= d.n) {
                // streaming slice: rows of 128 cells; blocks of k cells are groups of
                // k/4 lanes (k < 128) or of k/128 whole rows (k >= 128)
                const int4 *v4 = reinterpret_cast<const int4 *>(d.A + s0);
                const int G = (int)(K >> 2);                  // lanes per block when k < 128
                const int rpb = K >= 128 ? (int)(K >> 7) : 1;  // rows per block when k >= 128
                uint64_t acc = KEY_MAX;
#pragma unroll 1
                for (int r0 = 0; r0 < 32; r0 += 8) {
                    int4 x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = ld_stream_v4(v4 + (r0 + u) * 32 + lane);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int r = r0 + u;
                        const uint32_t e = (uint32_t)(s0 + 128 * r + 4 * lane);
                        uint64_t v = kmin(kmin(make_key(x[u].x, e), make_key(x[u].y, e + 1)),
                                          kmin(make_key(x[u].z, e + 2), make_key(x[u].w, e + 3)));
                        if (K < 128) {
                            for (int off = G >> 1; off > 0; off >>= 1) v = kmin(v, __shfl_xor_sync(0xffffffffu, v, off));
                            if ((lane % G) == 0) {
                                const int64_t b = (s0 + 128 * r + 4 * lane) >> d.logk;
                                T0h[b] = v;
                                atomicMin(C0 + (b >> g.lc), (unsigned long long)v);
                            }
                        } else {
                            acc = kmin(acc, v);
                            if ((r + 1) % rpb == 0) {
                                const uint64_t bm = warp_min(acc);
                                acc = KEY_MAX;
                                if (lane == 0) {
                                    const int64_t b = (s0 + 128 * r) >> d.logk;
                                    T0h[b] = bm;
                                    atomicMin(C0 + (b >> g.lc), (unsigned long long)bm);
                                }
                            }
                        }
                    }
                }
            } else {
                // block by block (large k, an unaligned array, or the array's last slice)
                const int64_t first = K <= 2048 ? (s0 >> d.logk) : (c0 >> d.logk) + w;
                const int64_t step = K <= 2048 ? 1 : kMT / 32;
                const int64_t end = K <= 2048 ? min(c1, s0 + 4096) : c1;
                for (int64_t b = first; (b << d.logk) < end; b += step) {
                    const int64_t lo = b << d.logk;
                    const int64_t hi = min((int64_t)d.n, lo + K) - 1;
                    uint64_t best = KEY_MAX;
                    if (aligned && hi - lo + 1 == K) {
                        const int4 *v4 = reinterpret_cast<const int4 *>(d.A + lo);
                        const int nv = (int)(K >> 2);
                        for (int v0 = lane; v0 < nv; v0 += 128) {
                            int4 x[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) x[u] = (v0 + 32 * u < nv) ? ld_stream_v4(v4 + v0 + 32 * u) : make_int4(0, 0, 0, 0);
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                if (v0 + 32 * u >= nv) continue;
                                const uint32_t e = (uint32_t)(lo + 4 * (v0 + 32 * u));
                                best = kmin(best, kmin(kmin(make_key(x[u].x, e), make_key(x[u].y, e + 1)),
                                                       kmin(make_key(x[u].z, e + 2), make_key(x[u].w, e + 3))));
                            }
                        }
                    } else {
                        for (int64_t i = lo + lane; i <= hi; i += 32) best = kmin(best, make_key(__ldg(d.A + i), (uint32_t)i));
                    }
                    best = warp_min(best);
                    if (lane == 0) {
                        T0h[b] = best;
                        atomicMin(C0 + (b >> g.lc), (unsigned long long)best);
                    }
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const int32_t items_h = pre1[h + 1] - pre1[h];
                s_flag = atomicAdd(p.done1 + h, 1u) == (uint32_t)(items_h - 1);
            }
            __syncthreads();
            if (s_flag) {  // last phase-1 item of array h: the coarse table's upper levels
                __threadfence();
                uint64_t *C = p.Cs + (int64_t)h * kCoarseCap;
                for (int64_t J = threadIdx.x; J < g.nbc; J += kMT) cs[J] = __ldcg(reinterpret_cast<const unsigned long long *>(C) + J);
                __syncthreads();
                for (int t = 1; t < g.lvc; ++t) {
                    const int64_t half = 1ll << (t - 1), cnt = g.nbc - (1ll << t) + 1;
                    uint64_t *cur = cs + g.row(t);
                    const uint64_t *prev = cs + g.row(t - 1);
                    for (int64_t J = threadIdx.x; J < cnt; J += kMT) cur[J] = kmin(prev[J], prev[J + half]);
                    __syncthreads();
                }
                for (int64_t i = g.nbc + threadIdx.x; i < g.size(); i += kMT) C[i] = cs[i];
                __threadfence();
                __syncthreads();
                const bool withhold = (p.flags & RMQ_FLAG_TEST_WITHHOLD_READY) && h == 0;
                if (threadIdx.x == 0 && !withhold) atomicExch(p.ready + h, 1u);
            }
        } else {
            // ---------------------------------------------------- phase 3
            const int64_t it3 = item - tot1;
            const int h = find_array<int32_t>(pre3, H, (int32_t)it3);
            const MultiDesc d = p.d[h];
            const int64_t nb = nblocks(d);
            const Coarse g = coarse_geom(nb);
            const int64_t c0 = (it3 - pre3[h]) * kQueriesPerItem;
            const int64_t qn = min((int64_t)kQueriesPerItem, (int64_t)d.q - c0);
            const int64_t qbase = qoff[h] + c0;
            if (threadIdx.x == 0) s_flag = wait_flag(p.ready + h, p.spin_limit);
            __syncthreads();
            if (!s_flag) {  // the table never became ready: answers -1, error word
                for (int64_t i = threadIdx.x; i < qn; i += kMT) p.out[qbase + i] = -1;
                if (threadIdx.x == 0 && p.err) atomicOr(p.err, ERR_TIMEOUT);
                __syncthreads();
                continue;
            }
            __threadfence();
            const uint64_t *C = p.Cs + (int64_t)h * kCoarseCap;
            for (int64_t i = threadIdx.x; i < g.size(); i += kMT) cs[i] = __ldcg(reinterpret_cast<const unsigned long long *>(C) + i);
            __syncthreads();
            const uint64_t *T0 = p.T0 + t0off[h];
            const int sh = d.logk + g.lc;
            uint64_t best[4];
            Pending pl[4], pr[4];
            bool hl[4], hr[4], ok[4];
            bool bad = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t qi = threadIdx.x * 4 + i;
                const bool present = qi < qn;
                const int32_t l = present ? p.L[qbase + qi] : 0, r = present ? p.R[qbase + qi] : -1;
                ok[i] = present && l >= 0 && r >= l && r < d.n;
                bad |= present && !ok[i];
                hl[i] = hr[i] = false;
                best[i] = KEY_MAX;
                if (!ok[i]) continue;
                if (coarse_span_min(cs, g, d.logk, (uint32_t)l, (uint32_t)r, (uint32_t)l, (uint32_t)r, best[i])) continue;
                int sub;
                best[i] = resolve_coarse(cs, g, d.logk, (uint32_t)l, (uint32_t)r, (uint32_t)l, (uint32_t)r, sub);
                if (sub == SUB_WHOLE) {
                    best[i] = resolve_t0(T0, d.logk, l, r, (uint32_t)l, (uint32_t)r, pl[i], pr[i], hl[i], hr[i]);
                } else {
                    Pending unused;
                    bool unused_flag = false;
                    if (sub & SUB_LEFT) {
                        const int64_t end_l = ((((int64_t)l >> sh) + 1) << sh) - 1;
                        best[i] = kmin(best[i], resolve_t0(T0, d.logk, l, end_l, (uint32_t)l, 0xffffffffu, pl[i], unused,
                                                           hl[i], unused_flag));
                    }
                    if (sub & SUB_RIGHT) {
                        const int64_t start_r = ((int64_t)r >> sh) << sh;
                        Pending a, b2;
                        bool ha = false, hb = false;
                        best[i] = kmin(best[i], resolve_t0(T0, d.logk, start_r, r, 0u, (uint32_t)r, a, b2, ha, hb));
                        if (ha) { pr[i] = a; hr[i] = true; }
                        if (hb) { pr[i] = b2; hr[i] = true; }
                    }
                }
            }
            const SrcI32 src{d.A};
            const bool vecA = (reinterpret_cast<uintptr_t>(d.A) & 15) == 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (vecA) {
                    warp_drain_scans<SrcI32, true>(src, d.n, hl[i], pl[i], best[i]);
                    warp_drain_scans<SrcI32, true>(src, d.n, hr[i], pr[i], best[i]);
                } else {
                    warp_drain_scans<SrcI32, false>(src, d.n, hl[i], pl[i], best[i]);
                    warp_drain_scans<SrcI32, false>(src, d.n, hr[i], pr[i], best[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t qi = threadIdx.x * 4 + i;
                if (qi < qn) p.out[qbase + qi] = ok[i] ? (int32_t)key_pos(best[i]) : -1;
            }
            if (bad && p.err) atomicOr(p.err, ERR_QUERY_RANGE);
            __syncthreads();  // the coarse table in shared memory is free again
        }
    }
}

constexpr size_t kMultiSmem = (size_t)kCoarseCap * 8 + (size_t)(kMultiMax + 1) * (8 + 8 + 4 + 4);

}  // namespace

// Block size for an array of the multi-array launch: the smallest power of
// two >= 32 whose coarse blocks hold at most 32 blocks (short T0 scans).
int multi_logk(int64_t n) {
    for (int lk = MIN_LOGK; lk < kLogChunk; ++lk) {
        const int64_t nb = cdiv(n, 1ll << lk);
        if (coarse_geom(nb).lc <= kMultiLcMax) return lk;
    }
    return kLogChunk;
}

int multi_max_logk() { return kLogChunk; }

size_t multi_workspace_bytes(const int64_t *n, const int64_t *q, const int32_t *logk, int H) {
    int64_t t0 = 0;
    for (int h = 0; h < H; ++h)
        if (q[h] > 0) t0 += cdiv(n[h], 1ll << logk[h]);
    return 256 + (size_t)H * 8 + (size_t)t0 * 8 + (size_t)H * kCoarseCap * 8 + 256;
}

cudaError_t launch_multi(const int32_t *const *A, const int64_t *n, const int64_t *q, const int32_t *logk, int H,
                         const int32_t *l, const int32_t *r, int32_t *out, uint32_t flags, void *ws, cudaStream_t s) {
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
    int64_t t0 = 0;
    for (int h = 0; h < H; ++h)
        if (q[h] > 0) t0 += cdiv(n[h], 1ll << logk[h]);
    p->T0 = reinterpret_cast<uint64_t *>(base + ctl);
    p->Cs = p->T0 + t0;
    p->L = l;
    p->R = r;
    p->out = out;
    p->err = err;
    for (int h = 0; h < H; ++h) p->d[h] = MultiDesc{A[h], (int32_t)n[h], (int32_t)q[h], logk[h], 0};
    cudaError_t e = cudaMemsetAsync(base, 0, ctl, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->Cs, 0xff, (size_t)H * kCoarseCap * 8, s);
    static std::once_flag once[kMaxDev];
    static int occ[kMaxDev];
    static cudaError_t attr_err[kMaxDev];
    once_per_device(once, di.device, [&] {
        const cudaError_t ea = cudaFuncSetAttribute(k_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMultiSmem);
        int o = 0;
        if (ea == cudaSuccess) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_multi, kMT, kMultiSmem);
        if (di.device >= 0 && di.device < kMaxDev) {
            attr_err[di.device] = ea;
            occ[di.device] = std::max(1, o);
        }
    });
    if (e == cudaSuccess && di.device >= 0 && di.device < kMaxDev) e = attr_err[di.device];
    if (e == cudaSuccess) {
        const int ctas = (di.device >= 0 && di.device < kMaxDev ? occ[di.device] : 1) * di.sms;
        k_multi<<<ctas, kMT, kMultiSmem, s>>>(*p);
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
