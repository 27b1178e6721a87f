// sparse_table.cu -- the sparse table over block minima (Sec. 3.1 step 3):
// level t at block j is the minimum over the 2^t blocks starting at j.
#include <algorithm>

#include "rmq_internal.cuh"

namespace rmq {

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------ sparse table
// Level t holds, for block j, the minimum over the 2^t blocks starting at j
// (Sec. 3.1 step 3).  Levels are produced in rounds; a round starting from
// level b computes levels b+1 .. b+nlev in shared memory by doubling:
//   level b+u at j = min over i < 2^u of level b at j + i * 2^b.
// A CTA owns R residues rho (mod 2^b) and S consecutive strides s, i.e. the
// entries j = rho0 + rho + (s0 + s) * 2^b; it loads the S + 2^nlev rows it
// needs once (coalesced along rho for R = 32, along s for R = 1), doubles in
// ping-pong buffers and writes every level's rows < S.  Round 0 (R = 1,
// contiguous tiles) runs as k_st_first below; later rounds start at b >= 5,
// so R = 32 divides 2^b.
// cap > 0: levels up to lc of the two-level layout for that coarse geometry;
// cap == 0: every level.
template <int R, int LV>
__global__ void __launch_bounds__(kThreads) k_st_round(uint64_t *__restrict__ T, Len len, int logk, int b, int S,
                                                      int cap) {
    pdl_wait();
    const int64_t n = len.get();
    const int64_t nb = (n + (1ll << logk) - 1) >> logk;
    if (nb < 2) return;
    const int top = cap > 0 ? coarse_geom(nb, cap).lc : ilog2_dev((uint64_t)nb);
    if (b >= top) return;
    const int nlev = min(LV, top - b);
    const int rows = S + (1 << nlev);
    const int64_t stride = 1ll << b;
    const int64_t ngroups = (R == 1) ? 1 : (stride / R);
    const int64_t g = blockIdx.x % ngroups;
    const int64_t st = blockIdx.x / ngroups;
    const int64_t rho0 = g * R;
    const int64_t s0 = st * (int64_t)S;
    if (rho0 + s0 * stride >= nb) return;
    extern __shared__ uint64_t smem[];
    uint64_t *X = smem;
    uint64_t *Y = smem + (size_t)rows * R;
    const uint64_t *Tb = T + (int64_t)b * nb;
    for (int i = threadIdx.x; i < rows * R; i += blockDim.x) {
        const int srow = i / R, c = i % R;
        const int64_t j = rho0 + c + (s0 + srow) * stride;
        X[i] = (j < nb) ? Tb[j] : KEY_MAX;
    }
    __syncthreads();
    for (int u = 1; u <= nlev; ++u) {
        const int half = 1 << (u - 1);
        const int cnt = rows - (1 << u) + 1;
        for (int i = threadIdx.x; i < cnt * R; i += blockDim.x) Y[i] = kmin(X[i], X[i + half * R]);
        __syncthreads();
        const int64_t span = 1ll << (b + u);
        uint64_t *Tu = T + (int64_t)(b + u) * nb;
        for (int i = threadIdx.x; i < S * R; i += blockDim.x) {
            const int srow = i / R, c = i % R;
            const int64_t j = rho0 + c + (s0 + srow) * stride;
            if (j + span <= nb) Tu[j] = Y[i];
        }
        uint64_t *tmp = X; X = Y; Y = tmp;
    }
}

// The first round (levels 1 .. nlev from level 0, contiguous tiles of S
// outputs): the same doubling as k_st_round with R = 1, b = 0, laid out for a
// short dependent chain, which is what bounds this kernel (a few hundred
// bytes per CTA).  The loads of the tile and its halo are issued first: the
// halo is sized for nlev_max, the host's bound on the level count (from the
// largest possible block count; the coarse shift grows with it), and the
// exact count is worked out from the device-side length while they are in
// flight.  Index arithmetic inside the tile is 32-bit.
template <int S>
__global__ void __launch_bounds__(kThreads) k_st_first(uint64_t *__restrict__ T, Len len, int logk, int nlev_max,
                                                      int cap) {
    pdl_wait();
    const int64_t n = len.get();
    const int64_t nb = (n + (1ll << logk) - 1) >> logk;
    const int64_t s0 = (int64_t)blockIdx.x * S;
    if (nb < 2 || s0 >= nb) return;
    extern __shared__ uint64_t smem[];
    const int rows = S + (1 << nlev_max);
    uint64_t *X = smem, *Y = smem + rows;
    const int64_t left = nb - s0;   // entries of level 0 from the tile's start
    const unsigned long long *T0 = reinterpret_cast<const unsigned long long *>(T) + s0;
    for (int i = threadIdx.x; i < rows; i += kThreads) X[i] = i < left ? __ldg(T0 + i) : KEY_MAX;
    const int top = cap > 0 ? coarse_geom(nb, cap).lc : ilog2_dev((uint64_t)nb);
    const int nlev = min(nlev_max, top);
    __syncthreads();
    uint64_t *Tu = T + s0;
    for (int u = 1; u <= nlev; ++u) {
        const int half = 1 << (u - 1);
        const int cnt = rows - (1 << u) + 1;
        for (int i = threadIdx.x; i < cnt; i += kThreads) Y[i] = kmin(X[i], X[i + half]);
        __syncthreads();
        Tu += nb;
        const int64_t valid = left - (1ll << u) + 1;   // entries j with j + 2^u <= nb
        for (int i = threadIdx.x; i < S; i += kThreads)
            if (i < valid) Tu[i] = Y[i];
        uint64_t *t = X; X = Y; Y = t;
    }
}

// Coarse table of the two-level layout: level 0 holds the minima of the
// coarse blocks (level lc of the block table at the coarse block starts; the
// last, partial coarse block from two overlapping lookups of lower levels),
// and the levels above come by doubling over the coarse blocks -- all in one
// CTA's shared memory, since the coarse table has at most kCoarseCap entries.
__global__ void __launch_bounds__(1024) k_coarse_table(const uint64_t *__restrict__ T, Len len, int logk,
                                                       uint64_t *__restrict__ Cs) {
    pdl_wait();
    __shared__ uint64_t c[kCoarseCap];
    const int64_t n = len.get();
    const int64_t nb = (n + (1ll << logk) - 1) >> logk;
    if (nb < 1) return;
    const Coarse g = coarse_geom(nb);
    for (int64_t J = threadIdx.x; J < g.nbc; J += blockDim.x) {
        uint64_t v;
        if (J < g.nbc_full) {
            v = T[(int64_t)g.lc * nb + (J << g.lc)];
        } else {
            const int64_t s0 = J << g.lc;
            const int tt = ilog2_dev((uint64_t)(nb - s0));
            v = kmin(T[(int64_t)tt * nb + s0], T[(int64_t)tt * nb + nb - (1ll << tt)]);
        }
        c[J] = v;
    }
    __syncthreads();
    for (int t = 1; t < g.lvc; ++t) {
        const int64_t half = 1ll << (t - 1), cnt = g.nbc - (1ll << t) + 1;
        uint64_t *cur = c + g.row(t);
        const uint64_t *prev = c + g.row(t - 1);
        for (int64_t J = threadIdx.x; J < cnt; J += blockDim.x) cur[J] = kmin(prev[J], prev[J + half]);
        __syncthreads();
    }
    for (int64_t i = threadIdx.x; i < g.size(); i += blockDim.x) Cs[i] = c[i];
}

constexpr int kLV0 = 12, kS0 = 256;   // round 0: levels 1..12, 256 outputs per CTA
constexpr int kLV1 = 6, kS1 = 64;     // later rounds: 6 levels, 32 residues x 64 strides

}  // namespace

cudaError_t launch_sparse_table(uint64_t *T, Len len, int logk, int64_t nb_max, cudaStream_t s, bool two,
                                uint64_t *Cs, int cap) {
    if (nb_max < 1) return cudaSuccess;
    if (cap < 1 || cap > kCoarseCapMax || (Cs && cap != kCoarseCap)) return cudaErrorInvalidValue;
    const int top = two ? coarse_geom(nb_max, cap).lc : (nb_max >= 2 ? ilog2_host((uint64_t)nb_max) : 0);
    const int kcap = two ? cap : 0;
    static std::once_flag once[kMaxDev];
    const DevInfo di = dev_info();
    const int nlev0 = std::min(top, kLV0);   // levels of the first round, at most
    const size_t smem0 = 2ull * (kS0 + (1 << nlev0)) * sizeof(uint64_t);
    const size_t smem1 = 2ull * (kS1 + (1 << kLV1)) * 32 * sizeof(uint64_t);
    once_per_device(once, di.device, [&] {
        cudaFuncSetAttribute(k_st_first<kS0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2ull * (kS0 + (1 << kLV0)) * sizeof(uint64_t)));
        cudaFuncSetAttribute(k_st_round<32, kLV1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    });
    {
        const int64_t ctas = cdiv(nb_max, kS0);
        if (top > 0) {
            launch_pdl(k_st_first<kS0>, (unsigned)ctas, kThreads, smem0, s, T, len, logk, nlev0, kcap);
            note_launches(1);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int b = kLV0; b < top; b += kLV1) {
        const int64_t stride = 1ll << b;
        const int64_t ngroups = stride / 32;
        const int64_t nstr = cdiv(nb_max, stride);
        const int64_t ctas = ngroups * cdiv(nstr, kS1);
        launch_pdl(k_st_round<32, kLV1>, (unsigned)ctas, kThreads, smem1, s, T, len, logk, b, kS1, kcap);
        note_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (two && Cs) {
        launch_pdl(k_coarse_table, 1, 1024, 0, s, T, len, logk, Cs);
        note_launches(1);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace rmq
