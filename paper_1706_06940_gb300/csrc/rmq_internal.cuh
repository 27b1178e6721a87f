// rmq_internal.cuh -- shared device helpers and host launcher prototypes of
// the GB300 BbST library.  Not part of the public ABI (include/rmq.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <utility>

#include "../../include/rmq.h"

namespace rmq {

constexpr uint64_t KEY_MAX = ~0ull;
constexpr int MIN_LOGK = 5;    // k >= 32
constexpr int MAX_LOGK = 16;   // k <= 65536

// Counters of the instrumented query kernel (rmq_batch_counted), in the
// order of rmq_scan_stats.
enum : int { CNT_OPEN = 0, CNT_TABLE, CNT_M1, CNT_ELEMS, CNT_RANKS, CNT_N };

// Bits of the sticky device error word.
constexpr unsigned ERR_QUERY_RANGE = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;

// Packed key: unsigned order == (value, position) order; low 32 bits = position.
__device__ __forceinline__ uint64_t make_key(int32_t v, uint32_t pos) {
    return ((uint64_t)((uint32_t)v ^ 0x80000000u) << 32) | (uint64_t)pos;
}
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t key_pos(uint64_t k) { return (uint32_t)k; }
__device__ __forceinline__ uint32_t key_hi(uint64_t k) { return (uint32_t)(k >> 32); }

__device__ __forceinline__ uint64_t warp_min(uint64_t v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = kmin(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__device__ __forceinline__ int ilog2_dev(uint64_t x) { return 63 - __clzll((long long)x); }

__host__ __device__ __forceinline__ int ilog2_hd(uint64_t x) {
#ifdef __CUDA_ARCH__
    return 63 - __clzll((long long)x);
#else
    return 63 - __builtin_clzll(x);
#endif
}

// Coarse summary of a block sparse table (the two-level scheme of Sec. 3.3
// applied to the memory hierarchy): coarse blocks are 2^lc consecutive
// blocks, and the summary holds levels lc .. lc + lvc - 1 of the table at the
// coarse block starts, i.e. a sparse table over nbc coarse blocks, small
// enough (<= cap entries) to live in shared memory while queries run.  Level
// t keeps only its nbc - 2^t + 1 defined entries, stored one level after the
// other.  lc is the smallest shift for which the summary fits.
//   kCoarseCap: every plain-form table (the summary of a table that outlives
//     a call is kept in memory; a batch call's query CTAs build it in shared
//     memory);
//   kCoarseCapCon: the table over A_Q of a contracted batch call.  A query
//     the summary leaves open costs more there (two rank lookups, 8-byte
//     scans), so its summary is finer.
constexpr int kCoarseCap = 4096;
constexpr int kCoarseCapCon = 6656;
constexpr int kCoarseCapMax = kCoarseCapCon;
struct Coarse {
    int lc;            // log2 of blocks per coarse block
    int lvc;           // levels of the coarse table
    int64_t nbc;       // coarse blocks (the last may be partial)
    int64_t nbc_full;  // coarse blocks made of 2^lc whole blocks
    // first entry of level t; row(lvc) is the size of the summary
    __host__ __device__ __forceinline__ int64_t row(int t) const { return (int64_t)t * (nbc + 1) - ((1ll << t) - 1); }
    __host__ __device__ __forceinline__ int64_t size() const { return nbc > 0 ? row(lvc) : 0; }
    __device__ __forceinline__ uint32_t row32(int t) const {
        return (uint32_t)t * ((uint32_t)nbc + 1u) - ((1u << t) - 1u);
    }
};
__host__ __device__ __forceinline__ Coarse coarse_geom(int64_t nb, int cap = kCoarseCap) {
    Coarse g{0, 1, nb, nb};
    if (nb < 1) { g.nbc = g.nbc_full = 0; return g; }
    for (int lc = 0;; ++lc) {
        g.nbc = (nb + (1ll << lc) - 1) >> lc;
        g.lvc = ilog2_hd((uint64_t)g.nbc) + 1;
        if (g.size() <= cap) {
            g.lc = lc; g.nbc_full = nb >> lc;
            return g;
        }
    }
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the previous kernel of the stream drains (its launch and
// set-up overlap that kernel's tail); it calls pdl_wait() before it reads or
// writes anything, which waits for the previous kernel to complete and its
// memory to be visible.  For a kernel launched without the attribute the wait
// is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Streaming 128-bit load that does not allocate in L1 (data read once).
__device__ __forceinline__ int4 ld_stream_v4(const int4 *p) {
    int4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ ulonglong2 ld_stream_v2u64(const ulonglong2 *p) {
    ulonglong2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0,%1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
    return v;
}

// Asks L2 to fetch [p, p + bytes) ahead of its use; p and bytes must be
// multiples of 16 and the range must lie inside one allocation.  Nothing is
// waited for and nothing lands in shared memory.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Asynchronous 16-byte copy global -> shared (dst: shared-window address),
// grouped by commit; wait<N> returns once at most N of this thread's groups
// are still in flight.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- sources
// A "source" yields packed keys of a sequence: the int32 input A (key built
// from value and index) or an array of ready keys (the contracted A_Q).

struct SrcI32 {
    const int32_t *a;
    static constexpr int EPV = 4;  // elements per 16-byte vector
    __device__ __forceinline__ uint64_t one(int64_t i) const { return make_key(__ldg(a + i), (uint32_t)i); }
    // vector vi covers elements [4vi, 4vi + 4); the caller guarantees 4vi + 3 < n
    template <bool VEC>
    __device__ __forceinline__ void vec(int64_t vi, uint64_t (&k)[4]) const {
        const int64_t e = vi * 4;
        if (VEC) {
            int4 v = ld_stream_v4(reinterpret_cast<const int4 *>(a) + vi);
            k[0] = make_key(v.x, (uint32_t)e);
            k[1] = make_key(v.y, (uint32_t)(e + 1));
            k[2] = make_key(v.z, (uint32_t)(e + 2));
            k[3] = make_key(v.w, (uint32_t)(e + 3));
        } else {
#pragma unroll
            for (int x = 0; x < 4; ++x) k[x] = make_key(__ldg(a + e + x), (uint32_t)(e + x));
        }
    }
};

struct SrcU64 {
    const uint64_t *a;
    static constexpr int EPV = 2;
    __device__ __forceinline__ uint64_t one(int64_t i) const { return __ldg(reinterpret_cast<const unsigned long long *>(a) + i); }
    template <bool VEC>
    __device__ __forceinline__ void vec(int64_t vi, uint64_t (&k)[2]) const {
        ulonglong2 v = ld_stream_v2u64(reinterpret_cast<const ulonglong2 *>(a) + vi);
        k[0] = v.x;
        k[1] = v.y;
    }
};

// Length of a sequence that may live on the device: n = m_dev ? (*m_dev - 1)
// clamped at 0 : n_host.  The contracted array's length is only known on the
// device (m - 1), so its kernels read it there and the host sizes launches
// for the bound.
struct Len {
    int64_t n_host;
    const int64_t *m_dev;
    __device__ __forceinline__ int64_t get() const {
        if (!m_dev) return n_host;
        int64_t m = *m_dev;
        return m > 1 ? m - 1 : 0;
    }
};

// ---------------------------------------------------------------- host side

// Stage boundaries: when the caller supplies CUDA events, one is recorded
// on the stream after each stage of the method.
struct Stages {
    cudaEvent_t *ev = nullptr;
    int n = 0;
    int i = 0;
    void mark(cudaStream_t s) {
        if (ev && i < n) cudaEventRecord(ev[i], s);
        ++i;
    }
    // An event outside the sequence (a boundary inside a stage), at index idx.
    void extra(cudaStream_t s, int idx) {
        if (ev && idx < n) cudaEventRecord(ev[idx], s);
    }
};
// Index of the optional event recorded after the clearing of the endpoint
// bitmap, inside step 1 of the contracted form.
constexpr int kEventAfterClear = 6;

// Process-wide count of kernel launches issued by this library.
void note_launches(int count);

// One-time set-up per device (kernel attributes, occupancy, symbol
// addresses): f runs once per device and process, and a thread that calls
// while another runs it waits for it; what f stores is then visible to every
// caller.  Devices beyond kMaxDev run f on every call.
constexpr int kMaxDev = 64;
template <class F>
inline void once_per_device(std::once_flag (&flags)[kMaxDev], int dev, F &&f) {
    if (dev >= 0 && dev < kMaxDev) std::call_once(flags[dev], std::forward<F>(f));
    else f();
}

struct DevInfo {
    int device;
    int sms;
};
DevInfo dev_info();                      // current device, cached SM count
// Device address of the sticky error word (ERR_* bits) of stream s on the
// current device.  Each stream has a word of its own (up to kErrSlots - 1
// streams per device; more streams share words), so that the errors of one
// stream's calls are reported by rmq_stream_status on that stream only.
constexpr int kErrSlots = 256;
unsigned *err_word_ptr(cudaStream_t s);

inline int ilog2_host(uint64_t x) { int t = -1; while (x) { x >>= 1; ++t; } return t; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Launchers (plain.cu).  All enqueue on `s` and return the launch status.
// M1 (optional): minima of every small block of 2^logk1 cells (5 <= logk1 <=
// logk), ceil(n / 2^logk1) entries.
cudaError_t launch_block_minima_i32(const int32_t *A, int64_t n, int logk, uint64_t *T0, cudaStream_t s,
                                    uint64_t *M1 = nullptr, int logk1 = 7);
cudaError_t launch_block_minima_u64(const uint64_t *AQ, Len len, int64_t n_max, int logk, uint64_t *T0,
                                    cudaStream_t s);
// The table's block count is nb = ceil(len / 2^logk), read on the device from
// `len`; nb_max bounds it on the host and sizes the launches.
// two_level == false: every level 1 .. floor(log2 nb) of the block table.
// two_level == true: the two-level layout -- levels 1 .. lc of the block
//   table for the coarse geometry of cap; with Cs (cap == kCoarseCap only),
//   also the coarse table in Cs (else each query CTA builds it in shared
//   memory from level lc).
cudaError_t launch_sparse_table(uint64_t *T, Len len, int logk, int64_t nb_max, cudaStream_t s,
                                bool two_level = false, uint64_t *Cs = nullptr, int cap = kCoarseCap);
// Entries of the two-level block table (levels 0 .. lc) for nb blocks.
inline int64_t two_level_entries(int64_t nb, int cap = kCoarseCap) {
    return nb < 1 ? 0 : nb * (coarse_geom(nb, cap).lc + 1);
}
// Query kernel: kQueryCtasPerSm CTAs of kQueryThreads per SM (<= 113 KB of
// shared memory each: coarse table, l, r ring, queues and part pool; <= 64
// registers), one wave, 16 warps of 128 queries per step.
constexpr int kQueryThreads = 512;
constexpr int kQueryCtasPerSm = 2;
inline int64_t query_ctas(int64_t q, int sms) {
    const int64_t steps = (q + 127) / 128;
    int64_t ctas = (steps + kQueryThreads / 32 - 1) / (kQueryThreads / 32);
    const int64_t cap = (int64_t)sms * kQueryCtasPerSm;
    if (ctas > cap) ctas = cap;
    return ctas < 1 ? 1 : ctas;
}
// Coarse index of the contracted form: CP[j] = P_{j 2^sh}, the position in A
// where coarse block j of A_Q begins (sh = logk_con + lc), and for buckets of
// 2^s positions, CB[i] = the last coarse block that begins at or before
// position i 2^s (0 if none); CB[nbk] = nbc - 1.  A query's coarse blocks
// follow from l and r through these two small arrays, without its ranks.
// A summary of at most kCoarseCapCon entries has nbc <= 766.
constexpr int kCoarseBlocksMax = 768;
constexpr int64_t coarse_size_of(int64_t nbc) {
    int lvc = 0;
    while ((nbc >> lvc) > 0) ++lvc;
    return lvc * (nbc + 1) - ((1ll << lvc) - 1);
}
constexpr int64_t coarse_blocks_fitting(int64_t cap) {
    int64_t nbc = 1;
    while (coarse_size_of(nbc + 1) <= cap) ++nbc;
    return nbc;
}
static_assert(coarse_blocks_fitting(kCoarseCapCon) <= kCoarseBlocksMax, "coarse index too small");
constexpr int kBucketsMax = 2048;
__host__ __device__ inline int bucket_shift(int64_t n) {
    int s = 5;
    while (((n - 1) >> s) + 1 >= kBucketsMax) ++s;
    return s;
}
__host__ __device__ inline int64_t bucket_count(int64_t n) { return ((n - 1) >> bucket_shift(n)) + 1; }
// Plain-form query over a two-level table; Cs == nullptr: the coarse table is
// built by every query CTA from level lc of T.
// M1 (optional): the 128-cell minima of A, used for the partial-block parts.
// cap: the coarse geometry the table was built for (kCoarseCap when Cs is given).
// counts (optional): 5 device counters; when given, the instrumented kernel
// runs and adds its work counts there (rmq_scan_stats order; aligned
// buffers only, else cudaErrorInvalidValue).
// logk1: the small blocks of M1; max_teams: partial-block scans run by
// teams of at least 32 / max_teams lanes (1, 2 or 4).
cudaError_t launch_query_plain(const int32_t *A, int64_t n, int logk, const uint64_t *T, const uint64_t *Cs,
                               const int32_t *l, const int32_t *r, int64_t q, int32_t *out, cudaStream_t s,
                               const uint64_t *M1 = nullptr, int cap = kCoarseCap,
                               unsigned long long *counts = nullptr, int logk1 = 7, int max_teams = 4);

// Multi-level layout (hlevel.cu, Sec. 3.3): logk[1 .. h] the logs of the
// block sizes, strictly increasing, 5 <= logk[1] <= 16, logk[h] <= kHLevelMaxLogK.
// W holds the minima of levels 1 .. h-1, then the table over blocks of
// 2^logk[h]; hlevel_entries gives its size in 8-byte keys (-1 on bad h).
constexpr int kHLevelMax = 8;
constexpr int kHLevelMaxLogK = 30;
int64_t hlevel_entries(int64_t n, const int *logk, int h);
cudaError_t run_hlevel(const int32_t *A, int64_t n, const int *logk, int h, const int32_t *l, const int32_t *r,
                       int64_t q, int32_t *out, uint64_t *W, cudaStream_t s);
// The l-ary block sparse table (lary.cu): levels of the table for nb blocks
// and l = 2^logell; the whole batch with the table T (lary_levels * nb keys).
int lary_levels(int64_t nb, int logell);
cudaError_t run_lary(const int32_t *A, int64_t n, int logk, int logell, const int32_t *l, const int32_t *r,
                     int64_t q, int32_t *out, uint64_t *T, cudaStream_t s);

// Many arrays in one persistent launch (multi.cu).
constexpr int kMultiMax = 512;    // arrays per launch (their descriptors travel as a kernel parameter)
int multi_logk(int64_t n);
int multi_max_logk();   // the largest block size the multi-array launch accepts
size_t multi_workspace_bytes(const int64_t *n, const int64_t *q, const int32_t *logk, int H);
cudaError_t launch_multi(const int32_t *const *A, const int64_t *n, const int64_t *q, const int32_t *logk, int H,
                         const int32_t *l, const int32_t *r, int32_t *out, uint32_t flags, void *ws, cudaStream_t s);

// Queries against many resident handles in one launch (multi.cu).
constexpr int kReqMax = 512;      // requests per launch (descriptors travel as a kernel parameter)
struct QueryReq {
    const int32_t *A;
    const uint64_t *T;
    const uint64_t *Cs;
    int64_t n;
    int64_t q;
    int32_t logk;
};
cudaError_t launch_query_handles(const QueryReq *reqs, int H, const int32_t *l, const int32_t *r, int32_t *out,
                                 cudaStream_t s);

// Measured choices of the autotuner (tune.cu), remembered per shape
// (round(log2 n), round(log2 q), width class = round(log2 of the median query
// width)).  tuned_lookup with wclass < 0: TUNE_AMBIGUOUS when the shape holds
// choices for several width classes (the batch must be sampled).
enum : int { TUNE_NONE = 0, TUNE_FOUND = 1, TUNE_AMBIGUOUS = 2 };
constexpr int kWidthSample = 256;   // queries read back to find a batch's width class
int tuned_lookup(int64_t n, int64_t q, int wclass, rmq_opts *out);
int width_class_of(const int32_t *l, const int32_t *r, int64_t count, int64_t n);
// Width class of a device batch from kWidthSample of its queries (waits for
// the stream); -1 if they cannot be read.
int sample_width_class(const int32_t *l, const int32_t *r, int64_t q, int64_t n, cudaStream_t s);

// Device bytes rmq_build allocates for an array of n cells with blocks of
// 2^logk cells (levels 0 .. lc of the block table and the coarse summary).
int64_t handle_bytes_for(int64_t n, int logk);
// Internals of a resident handle (api.cu), for the multi-request paths.
const int32_t *h_array(rmq_handle h);
const uint64_t *h_table(rmq_handle h);
const uint64_t *h_coarse(rmq_handle h);
int64_t h_n(rmq_handle h);
int32_t h_logk(rmq_handle h);

// Contracted form (contract.cu).
size_t con_workspace_bytes(int64_t n, int64_t q, int logk_con);
cudaError_t run_contracted(const int32_t *A, int64_t n, const int32_t *l, const int32_t *r, int64_t q,
                           int32_t *out, int logk_con, void *ws, cudaStream_t s, Stages *st,
                           unsigned long long *counts = nullptr, int max_teams = 4);
cudaError_t sort_endpoints(const int32_t *l, const int32_t *r, int64_t q, int64_t n, uint32_t *pos_out,
                           uint32_t *tag_out, void *ws, size_t ws_bytes, cudaStream_t s);
size_t sort_workspace_bytes(int64_t q);
cudaError_t rank_endpoints(const uint32_t *pos, const uint32_t *tag, int64_t q, uint32_t *P, int64_t *m_dev,
                           int32_t *rank_l, int32_t *rank_r, void *ws, cudaStream_t s);
size_t rank_workspace_bytes(int64_t q);
cudaError_t contract(const int32_t *A, int64_t n, const uint32_t *P, const int64_t *m_dev, int64_t m_max,
                     uint64_t *AQ, void *ws, cudaStream_t s);
// Endpoint bitmap of the batch path: BW, the bitmap_entries(n) bit words
// (the last one 0), and BC, the set bits before each word (BC[last] = m);
// *m_dev = m, the number of distinct endpoint positions; AQ entries combined
// by the contraction are reset when AQ is given.
int64_t bitmap_entries(int64_t n);
size_t endpoint_bitmap_workspace_bytes(int64_t n);
cudaError_t endpoint_bitmap(const int32_t *l, const int32_t *r, int64_t q, int64_t n, uint32_t *BW, uint32_t *BC,
                            int64_t *m_dev, uint64_t *AQ, void *ws, cudaStream_t s, Stages *st = nullptr,
                            int logk_q = 0, uint32_t *CP = nullptr, uint16_t *CB = nullptr);
size_t contract_workspace_bytes(int64_t n);

}  // namespace rmq
