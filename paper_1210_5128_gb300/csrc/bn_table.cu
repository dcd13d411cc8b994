// bn_table.cu -- the preprocessing step of Sec. III.A on the GPU: data staging, joint
// counting (N_ijk of Eq. (3)), the FP64 local score of Eq. (4) with the structure
// penalty, and the pairwise prior of Eq. (9)-(10), for every (node, parent set of size
// <= k).  The paper keeps these in a host hash table keyed by (node, parent set); here
// they are a dense device array indexed by (node, rank), plus the parent-set table
// (Sec. V.B) of candidate-space masks shared by all nodes.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "bn_table.cuh"

namespace bn {

static constexpr double LN10 = 2.302585092994045684017991454684364208;
static constexpr int BUILD_RANGE = 64;     // consecutive ranks per warp work unit
static constexpr int BUILD_THREADS = 256;

// ---------------------------------------------------------------------------------
// rank <-> set on the device (sizes ascending, combinatorial number system)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void unrank_dev(int N, int64_t rank, int& j, uint64_t& mask)
{
    j = 0;
    while (rank >= (int64_t)c_binom.v[N][j]) { rank -= (int64_t)c_binom.v[N][j]; ++j; }
    mask = 0;
    for (int t = j; t >= 1; --t) {
        int a = N - 1;
        while ((int64_t)c_binom.v[a][t] > rank) --a;
        mask |= 1ull << a;
        rank -= (int64_t)c_binom.v[a][t];
    }
}

// next set in rank order: colex successor within a size (Gosper's hack), then the
// first set {0..j} of the next size
__device__ __forceinline__ void next_set(int N, int& j, uint64_t& mask)
{
    if (j == 0) { j = 1; mask = 1; return; }
    uint64_t c = mask & (~mask + 1);
    uint64_t r = mask + c;
    uint64_t nxt = (((r ^ mask) >> 2) >> (__ffsll((long long)mask) - 1)) | r;
    if ((nxt >> N) != 0) { ++j; mask = (j >= 64) ? ~0ull : ((1ull << j) - 1); }
    else mask = nxt;
}

// ---------------------------------------------------------------------------------
// a1: data staging.  m x n row-major uint8 -> [n][mw] words of 16 two-bit values.  Row
// 16w + b sits at bits 8(b & 3) + 2(b >> 2), so one shift by 2s and a mask 0x03030303
// yields rows 16w + 4s .. 16w + 4s + 3 as four bytes.  Rows past m are 0 (every variable
// in state 0); the counting kernel takes their number back out of cell 0.
// ---------------------------------------------------------------------------------
__global__ void k_pack(const uint8_t* __restrict__ data, int m, int n, int mw,
                       const uint8_t* __restrict__ arity, uint32_t* __restrict__ packed,
                       uint32_t* status)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * mw) return;
    int v = idx / mw, w = idx - v * mw;
    int av = arity[v];
    uint32_t word = 0;
    bool bad = false;
    for (int b = 0; b < 16; ++b) {
        int row = 16 * w + b;
        if (row < m) {
            uint32_t x = data[(size_t)row * n + v];
            if (x >= (uint32_t)av) { bad = true; x = 0; }   // never let a bad value index a count table
            word |= x << (8 * (b & 3) + 2 * (b >> 2));
        }
    }
    if (bad) atomicOr(status, STATUS_BADINPUT);
    packed[idx] = word;
}

// PPF of Eq. (10): ppf[i][m] = 100 (R[i][m] - 0.5)^3, evaluated left to right.
__global__ void k_ppf(const double* __restrict__ R, int n, double* __restrict__ ppf)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    double d = __dsub_rn(R[idx], 0.5);
    ppf[idx] = __dmul_rn(__dmul_rn(__dmul_rn(100.0, d), d), d);
}

// lgamma lookup: lut[l][N] = lgamma(N + alpha_l) - lgamma(alpha_l) in 64.64 fixed point
__global__ void k_lut(const double* __restrict__ alpha, int nlut, int m1, fx128* __restrict__ lut)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nlut * m1) return;
    int l = (int)(idx / m1), N = (int)(idx - (int64_t)l * m1);
    double a = alpha[l];
    double g = (N == 0) ? 0.0 : __dsub_rn(lgamma((double)N + a), lgamma(a));
    lut[idx] = fx_from_double(g);
}

// a4: parent-set table, candidate-space mask of every rank; padding ranks get ~0 (they
// can never be consistent with an order)
__global__ void k_pst(int N, int64_t S, int64_t Sp, uint64_t* __restrict__ pst)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= Sp) return;
    if (r >= S) { pst[r] = ~0ull; return; }
    int j;
    uint64_t m;
    unrank_dev(N, r, j, m);
    pst[r] = m;
}

__global__ void k_pad_keys(int64_t* __restrict__ keys, int n, int64_t S, int64_t Sp)
{
    int64_t pad = Sp - S;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * pad) return;
    int64_t i = idx / pad, e = idx - i * pad;
    keys[i * Sp + S + e] = KEY_NONE;
}

struct BuildArgs {
    const uint32_t* packed;
    int m, n, mw, k;
    int64_t S, Sp;
    int units_per_node;
    int cells_cap;
    int cells_max;           // largest histogram (q * r) of any entry
    const uint8_t* arity;
    const double* ppf;        // n*n or null
    double log10g;
    const fx128* lut;
    int lut_stride;           // m + 1
    const int16_t* cell_lut;  // [(qmax+1) * 5], index q*5 + r
    const int16_t* cfg_lut;
    int64_t* keys;
};

// an entry from its exact lgamma sum: / ln 10, the size penalty, the prior of every
// parent (candidate mask -> node ids, ascending), as one FP64 value in key form
__device__ __forceinline__ void finish_entry(const BuildArgs& A, int i, fx128 acc, int j, uint64_t mask, int64_t rho)
{
    double ls = __dadd_rn(__ddiv_rn(fx_to_double(acc), LN10), __dmul_rn((double)j, A.log10g));
    if (A.ppf) {
        uint64_t mm = mask;
        while (mm) {
            const int c = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            ls = __dadd_rn(ls, A.ppf[(size_t)i * A.n + c + (c >= i ? 1 : 0)]);
        }
    }
    A.keys[(size_t)i * A.Sp + rho] = double_to_key(ls);
}

// Counts of one packed word (16 rows).  cell = child state + sum_t parent state_t * cs[t];
// with cells <= 256 four rows' cells are formed at once as the bytes of one 32-bit
// integer (no byte can carry: each is a cell index < 256), otherwise two rows' as 16-bit
// halves.  Parents past the set's size have cs = 0.
template <int KT, bool WARP_AGG>
__device__ __forceinline__ void count_word(uint32_t* hist, uint32_t cw, const uint32_t (&pw)[KT],
                                           const uint32_t (&cs)[KT], bool bytes, int lane)
{
    if (bytes) {
#pragma unroll
        for (int sft = 0; sft < 8; sft += 2) {
            uint32_t c4 = (cw >> sft) & 0x03030303u;
#pragma unroll
            for (int t = 0; t < KT; ++t) c4 += ((pw[t] >> sft) & 0x03030303u) * cs[t];
            if (WARP_AGG) {
                // tiny histograms: one add per distinct cell of the warp
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const uint32_t cell = (c4 >> (8 * r)) & 0xffu;
                    const unsigned grp = __match_any_sync(__activemask(), cell);
                    if ((__ffs(grp) - 1) == lane) atomicAdd(&hist[cell], (uint32_t)__popc(grp));
                }
            } else {
                atomicAdd(&hist[c4 & 0xffu], 1u);
                atomicAdd(&hist[(c4 >> 8) & 0xffu], 1u);
                atomicAdd(&hist[(c4 >> 16) & 0xffu], 1u);
                atomicAdd(&hist[c4 >> 24], 1u);
            }
        }
    } else {
#pragma unroll
        for (int h = 0; h < 16; h += 8) {
#pragma unroll
            for (int sft = 0; sft < 8; sft += 2) {
                uint32_t c2 = (cw >> (h + sft)) & 0x00030003u;
#pragma unroll
                for (int t = 0; t < KT; ++t) c2 += ((pw[t] >> (h + sft)) & 0x00030003u) * cs[t];
                atomicAdd(&hist[c2 & 0xffffu], 1u);
                atomicAdd(&hist[c2 >> 16], 1u);
            }
        }
    }
}

// The lgamma terms of one count table: per configuration c, sum_x L_cell[N_cx] -
// L_cfg[sum_x N_cx], exactly in 128-bit fixed point.  Every cell read is set back to 0,
// so the warp's histogram is all zero again for the next entry.
template <int RI>
__device__ __forceinline__ fx128 score_cells(uint32_t* hist, int q, const fx128* __restrict__ Lx,
                                             const fx128* __restrict__ Lc, int lane)
{
    fx128 acc = 0;
    for (int c = lane; c < q; c += 32) {
        uint32_t v[RI], Nc = 0;
#pragma unroll
        for (int x = 0; x < RI; ++x) {
            v[x] = hist[c * RI + x];
            Nc += v[x];
        }
#pragma unroll
        for (int x = 0; x < RI; ++x) {
            hist[c * RI + x] = 0u;
            acc += Lx[v[x]];
        }
        acc -= Lc[Nc];
    }
    return acc;
}

// a2 + a3: one warp per work unit of BUILD_RANGE consecutive ranks of one node.  Per
// parent set: a warp-private shared-memory histogram of (parent configuration, child
// state) counts over all m rows, then the lgamma terms summed exactly in 128-bit fixed
// point (the sum is independent of the cell order), one rounding to FP64, the
// structure penalty, and the prior terms in ascending parent id.
// Shared memory holds the warps' histograms, then (when it fits) the packed data.
template <int KT, bool SMEM_DATA, bool WARP_AGG>
__global__ void __launch_bounds__(BUILD_THREADS) k_build(BuildArgs A)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* hist = sm + warp * A.cells_cap;
    const uint32_t* D = A.packed;
    for (int c = lane; c < A.cells_cap; c += 32) hist[c] = 0u;
    if (SMEM_DATA) {
        uint32_t* sd = sm + nw * A.cells_cap;
        for (int t = threadIdx.x; t < A.n * A.mw; t += blockDim.x) sd[t] = A.packed[t];
        D = sd;
    }
    __syncthreads();
    const int N = A.n - 1;
    const uint32_t pad = (uint32_t)(16 * A.mw - A.m);   // zero rows of the last word, all in cell 0
    const int64_t units = (int64_t)A.n * A.units_per_node;
    for (int64_t u = (int64_t)blockIdx.x * nw + warp; u < units; u += (int64_t)gridDim.x * nw) {
        const int i = (int)(u / A.units_per_node);
        const int64_t r0 = (u - (int64_t)i * A.units_per_node) * BUILD_RANGE;
        const int64_t r1 = min(r0 + (int64_t)BUILD_RANGE, A.S);
        const int ri = A.arity[i];
        const uint32_t* Di = D + (size_t)i * A.mw;
        int j;
        uint64_t mask;
        unrank_dev(N, r0, j, mask);
        fx128 my_acc = 0;
        int my_j = 0;
        uint64_t my_mask = 0;
        int64_t my_rho = 0;
        for (int64_t rho = r0; rho < r1; ++rho) {
            int poff[KT];
            uint32_t cs[KT];
            int q = 1;
            uint64_t mm = mask;
#pragma unroll
            for (int t = 0; t < KT; ++t) {
                poff[t] = 0;
                cs[t] = 0u;
                if (t < j) {
                    const int c = __ffsll((long long)mm) - 1;
                    mm &= mm - 1;
                    const int p = c + (c >= i ? 1 : 0);
                    poff[t] = p * A.mw;
                    cs[t] = (uint32_t)(q * ri);
                    q *= __ldg(&A.arity[p]);
                }
            }
            const bool bytes = q * ri <= 256;
            for (int w = lane; w < A.mw; w += 32) {
                const uint32_t cw = Di[w];
                uint32_t pw[KT];
#pragma unroll
                for (int t = 0; t < KT; ++t) pw[t] = D[poff[t] + w];
                count_word<KT, WARP_AGG>(hist, cw, pw, cs, bytes, lane);
            }
            __syncwarp();
            if (lane == 0 && pad) hist[0] -= pad;
            const fx128* Lx = A.lut + (size_t)A.cell_lut[q * 5 + ri] * A.lut_stride;
            const fx128* Lc = A.lut + (size_t)A.cfg_lut[q * 5 + ri] * A.lut_stride;
            fx128 acc;
            if (ri == 2) acc = score_cells<2>(hist, q, Lx, Lc, lane);
            else if (ri == 3) acc = score_cells<3>(hist, q, Lx, Lc, lane);
            else acc = score_cells<4>(hist, q, Lx, Lc, lane);
            // warp sum, exact mod 2^128: five limbs (26, 26, 26, 26, 24 bits) of every lane's
            // value summed by one 32-bit reduction instruction each (32 lanes x 2^26 < 2^32)
            {
                const uint64_t lo = (uint64_t)acc, hi = (uint64_t)(acc >> 64);
                constexpr uint64_t M26 = (1ull << 26) - 1;
                const uint32_t s0 = __reduce_add_sync(0xffffffffu, (uint32_t)(lo & M26));
                const uint32_t s1 = __reduce_add_sync(0xffffffffu, (uint32_t)((lo >> 26) & M26));
                const uint32_t s2 = __reduce_add_sync(0xffffffffu, (uint32_t)(((lo >> 52) | (hi << 12)) & M26));
                const uint32_t s3 = __reduce_add_sync(0xffffffffu, (uint32_t)((hi >> 14) & M26));
                const uint32_t s4 = __reduce_add_sync(0xffffffffu, (uint32_t)(hi >> 40));
                acc = (fx128)s0 + ((fx128)s1 << 26) + ((fx128)s2 << 52) + ((fx128)s3 << 78) + ((fx128)s4 << 104);
            }
            // every lane holds the sum; lane (rho - r0) % 32 finishes this entry, 32 entries
            // at a time (the FP64 tail runs on all lanes instead of on one)
            const int slot = (int)((rho - r0) & 31);
            if (lane == slot) {
                my_acc = acc;
                my_j = j;
                my_mask = mask;
                my_rho = rho;
            }
            if (slot == 31 || rho + 1 == r1) {
                if (lane <= slot) finish_entry(A, i, my_acc, my_j, my_mask, my_rho);
                __syncwarp();
            }
            __syncwarp();
            next_set(N, j, mask);
        }
    }
}

// score table upload / readout
__global__ void k_keys_from_scores(const double* __restrict__ sc, int n, int64_t S, int64_t Sp,
                                   int64_t* __restrict__ keys, uint32_t* status)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * S) return;
    int64_t i = idx / S, r = idx - i * S;
    double v = sc[idx];
    if (isnan(v) || v == INFINITY) atomicOr(status, STATUS_BADINPUT);
    keys[i * Sp + r] = double_to_key(v);
}

__global__ void k_scores_from_keys(const int64_t* __restrict__ keys, int n0, int nn, int64_t S,
                                   int64_t Sp, double* __restrict__ out)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nn * S) return;
    int64_t i = idx / S, r = idx - i * S;
    out[idx] = key_to_double(keys[(n0 + i) * Sp + r]);
}

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------
static int table_alloc(int n, int k, bn_table** out)
{
    bn_table* t = new bn_table();
    t->n = n;
    t->k = k;
    t->dev = device_id();
    t->S = num_sets_host(n - 1, k);
    t->Sp = round_up(t->S, SUBQ);
    cudaError_t e = cudaMalloc(&t->keys, sizeof(int64_t) * (size_t)n * (size_t)t->Sp);
    if (e == cudaSuccess) e = cudaMalloc(&t->pst, sizeof(uint64_t) * (size_t)t->Sp);
    if (e == cudaSuccess) e = cudaMalloc(&t->spos, sizeof(uint32_t) * (size_t)n * (size_t)t->Sp);
    if (e == cudaSuccess) e = cudaMalloc(&t->srank, sizeof(uint32_t) * (size_t)n * (size_t)t->Sp);
    if (e == cudaSuccess) e = cudaMalloc(&t->spos_t, sizeof(uint32_t) * (size_t)n * (size_t)t->Sp);
    if (e != cudaSuccess) {
        cudaFree(t->keys);
        cudaFree(t->pst);
        cudaFree(t->spos);
        cudaFree(t->srank);
        cudaFree(t->spos_t);
        delete t;
        cudaGetLastError();
        return set_error(BN_ENOMEM, "table allocation of %lld entries failed: %s",
                         (long long)((int64_t)n * num_sets_host(n - 1, k)), cudaGetErrorString(e));
    }
    t->bytes = (sizeof(int64_t) + 3 * sizeof(uint32_t)) * (size_t)n * (size_t)t->Sp + sizeof(uint64_t) * (size_t)t->Sp;
    *out = t;
    return BN_OK;
}

static int build_pst(bn_table* t, cudaStream_t s)
{
    int thr = 256;
    int64_t blocks = (t->Sp + thr - 1) / thr;
    k_pst<<<(unsigned)blocks, thr, 0, s>>>(t->n - 1, t->S, t->Sp, t->pst);
    BN_LAUNCH_CHECK("k_pst");
    if (t->Sp > t->S) {
        int64_t tot = (int64_t)t->n * (t->Sp - t->S);
        k_pad_keys<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(t->keys, t->n, t->S, t->Sp);
        BN_LAUNCH_CHECK("k_pad_keys");
    }
    return BN_OK;
}

// RAII list of stream-ordered temporaries
struct Temps {
    cudaStream_t s;
    std::vector<void*> p;
    explicit Temps(cudaStream_t st) : s(st) {}
    template <class T>
    int get(T** out, size_t count)
    {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(BN_ENOMEM, "cudaMallocAsync(%zu bytes) failed: %s", count * sizeof(T),
                             cudaGetErrorString(e));
        }
        p.push_back(q);
        *out = (T*)q;
        return BN_OK;
    }
    ~Temps()
    {
        for (void* q : p) cudaFreeAsync(q, s);
    }
};

// Counting: plain shared-memory atomics, except for tiny histograms (<= 8 cells), where
// the lanes of a warp collide on a few cells and warp-aggregated adds (one atomic per
// distinct cell, __match_any_sync) win.  Measured on GB300 at n = 60, k = 4, m = 1000
// (243-cell histograms): 0.070 s plain against 0.224 s aggregated for the whole table.
template <int KT>
static int launch_build_kt(const BuildArgs& A, bool smem_data, size_t smem, int grid, cudaStream_t s)
{
    const bool agg = A.cells_max <= 8;
    if (smem_data) {
        if (agg) {
            cudaFuncSetAttribute(k_build<KT, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_build<KT, true, true><<<grid, BUILD_THREADS, smem, s>>>(A);
        } else {
            cudaFuncSetAttribute(k_build<KT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_build<KT, true, false><<<grid, BUILD_THREADS, smem, s>>>(A);
        }
    } else {
        if (agg) {
            cudaFuncSetAttribute(k_build<KT, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_build<KT, false, true><<<grid, BUILD_THREADS, smem, s>>>(A);
        } else {
            cudaFuncSetAttribute(k_build<KT, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_build<KT, false, false><<<grid, BUILD_THREADS, smem, s>>>(A);
        }
    }
    BN_LAUNCH_CHECK("k_build");
    return BN_OK;
}

static int copy_in(void* dst, const void* src, size_t bytes, int mem, cudaStream_t s)
{
    if (bytes == 0) return BN_OK;
    BN_CUDA(cudaMemcpyAsync(dst, src, bytes, mem == BN_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                                 : cudaMemcpyHostToDevice, s));
    return BN_OK;
}

static int read_status(const uint32_t* d_status, uint32_t* h, cudaStream_t s)
{
    BN_CUDA(cudaMemcpyAsync(h, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    return BN_OK;
}

}  // namespace bn

using namespace bn;

// Host half of a table build: argument checks and the plan of the lgamma tables.
struct BuildPlan {
    const uint8_t* data = nullptr;
    int m = 0, n = 0, k = 0, mem = BN_MEM_HOST, kind = 0;
    double log10g = 0.0;
    const double* R = nullptr;
    std::vector<uint8_t> ar;
    std::vector<double> Rh;
    int64_t S = 0;
    int cells_max = 1;
    std::vector<int16_t> cell_lut, cfg_lut;
    std::vector<double> alpha;
};

static int build_plan(const uint8_t* data, int m, int n, const uint8_t* arity, int k, const double* R,
                      const bn_score_params* params, int mem, cudaStream_t s, BuildPlan* P)
{
    if (n < 2 || n > MAXN) return set_error(BN_EINVAL, "bn_build_scores: n=%d outside [2, 64]", n);
    if (m < 0 || (m > 0 && !data)) return set_error(BN_EINVAL, "bn_build_scores: bad data/m");
    if (k < 0 || k > n - 1) return set_error(BN_EINVAL, "bn_build_scores: k=%d outside [0, n-1]", k);
    if (!arity) return set_error(BN_EINVAL, "bn_build_scores: arity is NULL");
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_build_scores: bad mem");
    if (k > MAXK) return set_error(BN_EUNSUPPORTED, "bn_build_scores: k=%d above %d", k, MAXK);
    int kind = params ? params->score_kind : 0;
    double ess = params ? params->ess : 1.0;
    double log10g = params ? params->log10_gamma : 0.0;
    if (kind != 0 && kind != 1) return set_error(BN_EINVAL, "bn_build_scores: score_kind %d", kind);
    if (kind == 1 && !(ess > 0.0 && std::isfinite(ess))) return set_error(BN_EINVAL, "bn_build_scores: ess must be > 0");
    if (!std::isfinite(log10g)) return set_error(BN_EINVAL, "bn_build_scores: log10_gamma not finite");
    P->data = data;
    P->m = m;
    P->n = n;
    P->k = k;
    P->mem = mem;
    P->kind = kind;
    P->log10g = log10g;
    P->R = R;
    // small arrays are checked on the host
    std::vector<uint8_t>& ar = P->ar;
    std::vector<double>& Rh = P->Rh;
    ar.resize(n);
    if (mem == BN_MEM_DEVICE) {
        BN_CUDA(cudaMemcpyAsync(ar.data(), arity, n, cudaMemcpyDeviceToHost, s));
        if (R) {
            Rh.resize((size_t)n * n);
            BN_CUDA(cudaMemcpyAsync(Rh.data(), R, sizeof(double) * n * n, cudaMemcpyDeviceToHost, s));
        }
        BN_CUDA(cudaStreamSynchronize(s));
    } else {
        memcpy(ar.data(), arity, n);
        if (R) Rh.assign(R, R + (size_t)n * n);
    }
    for (int i = 0; i < n; ++i)
        if (ar[i] < 2 || ar[i] > 4) return set_error(BN_EINVAL, "bn_build_scores: arity[%d]=%d outside [2,4]", i, ar[i]);
    for (size_t t = 0; t < Rh.size(); ++t) {
        if ((int)(t / n) == (int)(t % n)) continue;
        if (!(Rh[t] >= 0.0 && Rh[t] <= 1.0)) return set_error(BN_EINVAL, "bn_build_scores: R[%zu] outside [0,1]", t);
    }
    if (mem == BN_MEM_HOST && m > 0) {
        for (int64_t r = 0; r < (int64_t)m; ++r)
            for (int i = 0; i < n; ++i)
                if (data[r * n + i] >= ar[i])
                    return set_error(BN_EINVAL, "bn_build_scores: data[%lld][%d]=%d >= arity %d", (long long)r, i,
                                     data[r * n + i], ar[i]);
    }
    const int64_t S = num_sets_host(n - 1, k);
    if (S >= (int64_t)1 << 31) return set_error(BN_EUNSUPPORTED, "bn_build_scores: %lld sets per node", (long long)S);
    P->S = S;
    // count-table size bound: r_i times the product of the k largest other arities
    int cells_max = 1;
    for (int i = 0; i < n; ++i) {
        std::vector<int> o;
        for (int p = 0; p < n; ++p)
            if (p != i) o.push_back(ar[p]);
        std::sort(o.rbegin(), o.rend());
        int64_t c = ar[i];
        for (int t = 0; t < k && t < (int)o.size(); ++t) c *= o[t];
        if (c > MAX_CELLS) return set_error(BN_EUNSUPPORTED, "bn_build_scores: count tables up to %lld cells (max %d)",
                                            (long long)c, MAX_CELLS);
        cells_max = std::max<int>(cells_max, (int)c);
    }
    P->cells_max = cells_max;

    // LUT plan: K2 uses alpha = 1 for cells and alpha = r for configurations; BDeu uses
    // ess/(q r) and ess/q for every reachable q (products of <= k arities)
    std::set<int> qs = {1};
    for (int t = 0; t < k; ++t) {
        std::set<int> nq = qs;
        for (int q : qs)
            for (int a = 2; a <= 4; ++a)
                if ((int64_t)q * a <= MAX_CELLS / 2) nq.insert(q * a);
        qs.swap(nq);
    }
    const int qmax = *qs.rbegin();
    std::vector<int16_t>& cell_lut = P->cell_lut;
    std::vector<int16_t>& cfg_lut = P->cfg_lut;
    std::vector<double>& alpha = P->alpha;
    cell_lut.assign((size_t)(qmax + 1) * 5, 0);
    cfg_lut.assign((size_t)(qmax + 1) * 5, 0);
    if (kind == 0) {
        alpha = {1.0, 2.0, 3.0, 4.0};
        for (int q : qs)
            for (int r = 2; r <= 4; ++r) {
                cell_lut[(size_t)q * 5 + r] = 0;
                cfg_lut[(size_t)q * 5 + r] = (int16_t)(r - 1);
            }
    } else {
        for (int q : qs) {
            int cfg_id = (int)alpha.size();
            alpha.push_back(ess / (double)q);
            for (int r = 2; r <= 4; ++r) {
                cfg_lut[(size_t)q * 5 + r] = (int16_t)cfg_id;
                cell_lut[(size_t)q * 5 + r] = (int16_t)alpha.size();
                alpha.push_back(ess / ((double)q * (double)r));
            }
        }
    }
    if (alpha.size() > 32000) return set_error(BN_EUNSUPPORTED, "bn_build_scores: too many lgamma tables");
    return BN_OK;
}

// Device half: every kernel of the build on stream s, writing t (allocated) and OR-ing
// STATUS_BADINPUT into *d_status for a data value at or above its arity.  Temporaries
// are stream-ordered; nothing here waits for the device.
static int build_enqueue(const BuildPlan& P, bn_table* t, uint32_t* d_status, cudaStream_t s,
                         cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr)
{
    const int n = P.n, m = P.m, k = P.k;
    const std::vector<double>& alpha = P.alpha;
    int rc = BN_OK;
    Temps tmp(s);
    const int mw = (m + 15) / 16;
    uint8_t *d_data = nullptr, *d_ar = nullptr;
    uint32_t* d_packed = nullptr;
    double *d_ppf = nullptr, *d_R = nullptr, *d_alpha = nullptr;
    fx128* d_lut = nullptr;
    int16_t *d_cell = nullptr, *d_cfg = nullptr;
    if ((rc = tmp.get(&d_ar, n)) || (rc = tmp.get(&d_packed, (size_t)n * mw)) ||
        (rc = tmp.get(&d_alpha, alpha.size())) || (rc = tmp.get(&d_lut, alpha.size() * (size_t)(m + 1))) ||
        (rc = tmp.get(&d_cell, P.cell_lut.size())) || (rc = tmp.get(&d_cfg, P.cfg_lut.size())))
        return rc;
    BN_CUDA(cudaMemcpyAsync(d_ar, P.ar.data(), n, cudaMemcpyHostToDevice, s));
    BN_CUDA(cudaMemcpyAsync(d_alpha, alpha.data(), sizeof(double) * alpha.size(), cudaMemcpyHostToDevice, s));
    BN_CUDA(cudaMemcpyAsync(d_cell, P.cell_lut.data(), sizeof(int16_t) * P.cell_lut.size(), cudaMemcpyHostToDevice, s));
    BN_CUDA(cudaMemcpyAsync(d_cfg, P.cfg_lut.data(), sizeof(int16_t) * P.cfg_lut.size(), cudaMemcpyHostToDevice, s));
    if (m > 0) {
        if (P.mem == BN_MEM_DEVICE) d_data = (uint8_t*)P.data;
        else {
            if ((rc = tmp.get(&d_data, (size_t)m * n))) return rc;
            if ((rc = copy_in(d_data, P.data, (size_t)m * n, BN_MEM_HOST, s))) return rc;
        }
        k_pack<<<(n * mw + 255) / 256, 256, 0, s>>>(d_data, m, n, mw, d_ar, d_packed, d_status);
        BN_LAUNCH_CHECK("k_pack");
    }
    if (P.R) {
        if ((rc = tmp.get(&d_ppf, (size_t)n * n)) || (rc = tmp.get(&d_R, (size_t)n * n))) return rc;
        BN_CUDA(cudaMemcpyAsync(d_R, P.Rh.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, s));
        k_ppf<<<(n * n + 255) / 256, 256, 0, s>>>(d_R, n, d_ppf);
        BN_LAUNCH_CHECK("k_ppf");
    }
    {
        int64_t tot = (int64_t)alpha.size() * (m + 1);
        k_lut<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_alpha, (int)alpha.size(), m + 1, d_lut);
        BN_LAUNCH_CHECK("k_lut");
    }
    if ((rc = build_pst(t, s))) return rc;

    BuildArgs A;
    A.packed = d_packed;
    A.m = m;
    A.n = n;
    A.mw = mw;
    A.k = k;
    A.S = P.S;
    A.Sp = t->Sp;
    A.units_per_node = (int)((P.S + BUILD_RANGE - 1) / BUILD_RANGE);
    A.cells_cap = (int)round_up(P.cells_max, 32);
    A.cells_max = (int)P.cells_max;
    A.arity = d_ar;
    A.ppf = d_ppf;
    A.log10g = P.log10g;
    A.lut = d_lut;
    A.lut_stride = m + 1;
    A.cell_lut = d_cell;
    A.cfg_lut = d_cfg;
    A.keys = t->keys;
    const int nwarps = BUILD_THREADS / 32;
    size_t data_bytes = sizeof(uint32_t) * (size_t)n * mw;
    size_t hist_bytes = sizeof(uint32_t) * (size_t)A.cells_cap * nwarps;
    bool smem_data = data_bytes + hist_bytes <= 160 * 1024;
    size_t smem = hist_bytes + (smem_data ? data_bytes : 0);   // histograms, then the data
    int per_sm = std::max(1, std::min(8, (int)((220 * 1024) / std::max<size_t>(smem + 1024, 1))));
    int64_t units = (int64_t)n * A.units_per_node;
    int grid = (int)std::min<int64_t>((int64_t)sm_count() * per_sm, (units + nwarps - 1) / nwarps);
    if (grid < 1) grid = 1;
    int kt = k <= 2 ? 2 : k <= 4 ? 4 : k <= 8 ? 8 : 12;
    if (ev0) BN_CUDA(cudaEventRecord(ev0, s));
    switch (kt) {
        case 2: rc = launch_build_kt<2>(A, smem_data, smem, grid, s); break;
        case 4: rc = launch_build_kt<4>(A, smem_data, smem, grid, s); break;
        case 8: rc = launch_build_kt<8>(A, smem_data, smem, grid, s); break;
        default: rc = launch_build_kt<12>(A, smem_data, smem, grid, s); break;
    }
    if (rc) return rc;
    if (ev1) BN_CUDA(cudaEventRecord(ev1, s));
    return rank_entries(t, s);
}

static int build_scores_impl(const uint8_t* data, int m, int n, const uint8_t* arity, int k, const double* R,
                             const bn_score_params* params, int mem, void* stream, bn_table** out,
                             cudaEvent_t ev0, cudaEvent_t ev1)
{
    set_error(BN_OK, "");
    if (!out) return set_error(BN_EINVAL, "bn_build_scores: out is NULL");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    BuildPlan P;
    int rc = build_plan(data, m, n, arity, k, R, params, mem, s, &P);
    if (rc) return rc;
    bn_table* t = nullptr;
    if ((rc = table_alloc(n, k, &t))) return rc;
    struct Guard {
        bn_table*& t;
        bool ok = false;
        ~Guard()
        {
            if (!ok && t) bn_table_free(t);
        }
    } guard{t};
    uint32_t* d_status = nullptr;
    {
        Temps tmp(s);
        if ((rc = tmp.get(&d_status, 1))) return rc;
        BN_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
        if ((rc = build_enqueue(P, t, d_status, s, ev0, ev1))) return rc;
        uint32_t st = 0;
        if ((rc = read_status(d_status, &st, s))) return rc;
        if (st & STATUS_BADINPUT) return set_error(BN_EINVAL, "bn_build_scores: a data value is >= its arity");
    }
    guard.ok = true;
    *out = t;
    return BN_OK;
}

extern "C" int bn_build_scores(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                               const double* R, const bn_score_params* params, int mem,
                               void* stream, bn_table** out)
{
    return build_scores_impl(data, m, n, arity, k, R, params, mem, stream, out, nullptr, nullptr);
}

extern "C" int bn_build_scores_profiled(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                                        const double* R, const bn_score_params* params, int mem,
                                        void* stream, bn_table** out, double* build_ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
    }
    int rc = build_scores_impl(data, m, n, arity, k, R, params, mem, stream, out, e0, e1);
    float ms = 0.f;
    if (rc == BN_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "cudaEventElapsedTime", __FILE__, __LINE__);
    if (build_ms) *build_ms = (double)ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" int bn_build_scores_batch(int count, const uint8_t* const* data, const int* m, const int* n,
                                     const uint8_t* const* arity, const int* k, const double* const* R,
                                     const bn_score_params* params, int mem, void* stream, bn_table** out)
{
    set_error(BN_OK, "");
    if (count < 1 || !data || !m || !n || !arity || !k || !out)
        return set_error(BN_EINVAL, "bn_build_scores_batch: bad arguments");
    for (int i = 0; i < count; ++i) out[i] = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<BuildPlan> plans(count);
    for (int i = 0; i < count; ++i) {
        int rc = build_plan(data[i], m[i], n[i], arity[i], k[i], R ? R[i] : nullptr, params ? &params[i] : nullptr,
                            mem, s, &plans[i]);
        if (rc) {
            std::string msg = bn_last_error();
            return set_error(rc, "bn_build_scores_batch: network %d: %s", i, msg.c_str());
        }
    }
    std::vector<bn_table*> tabs(count, nullptr);
    struct Guard {
        std::vector<bn_table*>& t;
        bool ok = false;
        ~Guard()
        {
            if (!ok)
                for (bn_table* x : t) bn_table_free(x);
        }
    } guard{tabs};
    for (int i = 0; i < count; ++i) {
        int rc = table_alloc(n[i], k[i], &tabs[i]);
        if (rc) return rc;
    }
    // the builds run on a few side streams that fork from and join into `stream`; the
    // largest networks are spread over the streams first
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)n[a] * (double)plans[a].S * (double)(m[a] + 1) > (double)n[b] * (double)plans[b].S * (double)(m[b] + 1);
    });
    const int ns = std::min(count, 4);
    std::vector<cudaStream_t> side(ns, nullptr);
    std::vector<cudaEvent_t> ev(ns + 1, nullptr);
    struct Streams {
        std::vector<cudaStream_t>& s;
        std::vector<cudaEvent_t>& e;
        ~Streams()
        {
            for (cudaStream_t x : s)
                if (x) cudaStreamDestroy(x);
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } sg{side, ev};
    uint32_t* d_status = nullptr;
    BN_CUDA(cudaMallocAsync((void**)&d_status, sizeof(uint32_t) * count, s));
    struct Free {
        uint32_t* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{d_status, s};
    BN_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t) * count, s));
    for (int j = 0; j <= ns; ++j) BN_CUDA(cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming));
    BN_CUDA(cudaEventRecord(ev[ns], s));
    for (int j = 0; j < ns; ++j) {
        BN_CUDA(cudaStreamCreateWithFlags(&side[j], cudaStreamNonBlocking));
        BN_CUDA(cudaStreamWaitEvent(side[j], ev[ns], 0));
    }
    int rc = BN_OK;
    for (int q = 0; q < count && !rc; ++q) {
        const int i = order[q];
        rc = build_enqueue(plans[i], tabs[i], d_status + i, side[q % ns]);
    }
    for (int j = 0; j < ns; ++j) {
        cudaEventRecord(ev[j], side[j]);
        cudaStreamWaitEvent(s, ev[j], 0);
    }
    if (rc) {
        cudaStreamSynchronize(s);
        return rc;
    }
    std::vector<uint32_t> st(count, 0);
    BN_CUDA(cudaMemcpyAsync(st.data(), d_status, sizeof(uint32_t) * count, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i)
        if (st[i] & STATUS_BADINPUT)
            return set_error(BN_EINVAL, "bn_build_scores_batch: network %d: a data value is >= its arity", i);
    guard.ok = true;
    for (int i = 0; i < count; ++i) out[i] = tabs[i];
    return BN_OK;
}

extern "C" int bn_table_from_scores(const double* scores, int n, int k, int mem, void* stream, bn_table** out)
{
    set_error(BN_OK, "");
    if (!out) return set_error(BN_EINVAL, "bn_table_from_scores: out is NULL");
    *out = nullptr;
    if (n < 2 || n > MAXN || k < 0 || k > n - 1 || !scores)
        return set_error(BN_EINVAL, "bn_table_from_scores: bad n/k/scores");
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_table_from_scores: bad mem");
    const int64_t S = num_sets_host(n - 1, k);
    if (S >= (int64_t)1 << 31) return set_error(BN_EUNSUPPORTED, "bn_table_from_scores: too many sets");
    cudaStream_t s = (cudaStream_t)stream;
    bn_table* t = nullptr;
    int rc = table_alloc(n, k, &t);
    if (rc) return rc;
    Temps tmp(s);
    double* d_sc = nullptr;
    uint32_t* d_status = nullptr;
    if ((rc = tmp.get(&d_status, 1))) { bn_table_free(t); return rc; }
    if (mem == BN_MEM_DEVICE) d_sc = (double*)scores;
    else {
        if ((rc = tmp.get(&d_sc, (size_t)n * S))) { bn_table_free(t); return rc; }
        if ((rc = copy_in(d_sc, scores, sizeof(double) * (size_t)n * S, BN_MEM_HOST, s))) { bn_table_free(t); return rc; }
    }
    if (cudaMemsetAsync(d_status, 0, 4, s) != cudaSuccess) { bn_table_free(t); return cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__); }
    int64_t tot = (int64_t)n * S;
    k_keys_from_scores<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_sc, n, S, t->Sp, t->keys, d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { bn_table_free(t); return cuda_fail(e, "k_keys_from_scores", __FILE__, __LINE__); }
    count_launches(1);
    if ((rc = build_pst(t, s))) { bn_table_free(t); return rc; }
    if ((rc = rank_entries(t, s))) { bn_table_free(t); return rc; }
    uint32_t st = 0;
    if ((rc = read_status(d_status, &st, s))) { bn_table_free(t); return rc; }
    if (st) { bn_table_free(t); return set_error(BN_EINVAL, "bn_table_from_scores: NaN or +inf score"); }
    *out = t;
    return BN_OK;
}

extern "C" int bn_table_info(const bn_table* t, int* n, int* k, int64_t* sets_per_node, int64_t* device_bytes)
{
    if (!t) return set_error(BN_EINVAL, "bn_table_info: NULL table");
    if (n) *n = t->n;
    if (k) *k = t->k;
    if (sets_per_node) *sets_per_node = t->S;
    if (device_bytes) *device_bytes = (int64_t)t->bytes;
    return BN_OK;
}

extern "C" int bn_table_scores(const bn_table* t, int node, double* out, int mem, void* stream)
{
    set_error(BN_OK, "");
    if (!t || !out) return set_error(BN_EINVAL, "bn_table_scores: NULL argument");
    if (node < -1 || node >= t->n) return set_error(BN_EINVAL, "bn_table_scores: node %d", node);
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_table_scores: bad mem");
    cudaStream_t s = (cudaStream_t)stream;
    int n0 = node < 0 ? 0 : node, nn = node < 0 ? t->n : 1;
    int64_t tot = (int64_t)nn * t->S;
    Temps tmp(s);
    double* d = nullptr;
    int rc;
    if (mem == BN_MEM_DEVICE) d = out;
    else if ((rc = tmp.get(&d, (size_t)tot))) return rc;
    k_scores_from_keys<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(t->keys, n0, nn, t->S, t->Sp, d);
    BN_LAUNCH_CHECK("k_scores_from_keys");
    if (mem == BN_MEM_HOST) BN_CUDA(cudaMemcpyAsync(out, d, sizeof(double) * tot, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    return BN_OK;
}

extern "C" void bn_table_free(bn_table* t)
{
    if (!t) return;
    cudaFree(t->keys);
    cudaFree(t->pst);
    cudaFree(t->spos);
    cudaFree(t->srank);
    cudaFree(t->spos_t);
    cudaFree(t->sset);
    cudaFree(t->alive_block);
    cudaFree(t->gcache);
    delete t;
}
