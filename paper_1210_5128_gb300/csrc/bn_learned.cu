// bn_learned.cu -- the MH sampler with the learned swap proposal, built for latency.
//
// One MH step of every chain is three kernels, chained by programmatic dependent launch
// and captured as a CUDA graph:
//   k_learned_chain  one warp per chain: finishes the previous step (reverse proposal
//                    probability from the network's outputs on the proposed order, the
//                    exact MH test, state update, best graph, dwell-time edge counts,
//                    trace/records), then starts the next one (pair drawn from the cached
//                    q(. | current order), swap, re-scoring of the swapped span through the
//                    surviving parent sets, the first layer of the network on the proposed
//                    order written as the next GEMM's operand)
//   k_learned_gemm   hidden layer 2 (bias, ReLU, bf16) on the tensor cores
//   k_learned_gemm   output layer (bias) on the tensor cores, with per-tile softmax
//                    partials (max logit, sum of exp) for the row normaliser
// The first layer never multiplies the one-hot-like input: z1 = sum_p W1_p E[sigma(p)] is a
// sum of n table rows T[p][v] = W1_p E[v], and a swap of positions a, b changes four of
// them.  The rows are held in 32-bit fixed point so the running sum is exact: z1 is a
// function of the order alone, whatever path of swaps led to it, and so is q(. | order),
// which keeps the MH ratio exact.
//
// Operands of the GEMMs live in HBM/L2 in the no-swizzle K-major core-matrix layout the
// tensor core reads, so each CTA pulls its A tile (128 chains x H) and B tile (32 outputs
// x H) with 1-D bulk copies, one mbarrier per 64-wide K block, and issues the MMAs as the
// blocks land.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bn_chain.cuh"
#include "bn_tc.cuh"

namespace bn {

typedef __nv_bfloat16 bf16;

static constexpr int LR_TM = 128;        // chains per GEMM tile (tcgen05 M)
static constexpr int LR_TN = 32;         // outputs per GEMM CTA (tcgen05 N)
static constexpr int LR_MAX_H = 640;     // hidden width whose tiles fit in shared memory
static constexpr int LR_WARPS = 4;       // chains per block of k_learned_chain
static constexpr int LR_GRAPH_ITERS = 32;
static constexpr int LR_STAGE_MAX = 160 * 1024;   // survivors staged in shared memory up to this size
static constexpr uint32_t LR_IDESC = tc_idesc_bf16_f32(LR_TM, LR_TN);

enum { LF_FINISH = 1, LF_START = 2, LF_FLUSH = 4 };

struct LearnArgs {
    int H, P, Pp, NT;
    float eps;
    float scale;              // 2^-shift: fixed-point layer-1 sums to float
    const int32_t* T;         // [n][n][H] fixed point of W1_p E[v]
    const float* b1;
    uint8_t* h1;              // layer-2 A operand, core-matrix layout
    int32_t* z1;              // [C][H] fixed-point sum of the current order's rows
    int32_t* z1p;             // [C][H] ... of the proposed order
    const float* logits;      // [2][C][Pp]
    const float2* part;       // [2][C][NT] per 32-column tile: max logit, sum exp(l - max)
    uint8_t* cur_buf;         // [C] buffer holding the current order's network outputs
    int64_t* since;           // [C][n] step since which node i holds its parent set
    uint32_t* prank;          // [C][n] proposal: ranks of the re-scored nodes
    int64_t* pkey;            // [C][n] ... and their keys
    uint8_t* pab;             // [C][2] swapped positions a < b
    uint32_t* ppair;          // [C] pair index
    float* plqf;              // [C] ln q(pair | current order)
    double* pu;               // [C] the MH uniform
    double* pdpart;           // [C] change of the re-scored entries (any order)
    const uint64_t* smask;    // survivors in score order: candidate masks,
    const uint32_t* srk;      //   ranks,
    const int64_t* skey;      //   keys,
    const uint32_t* soff;     //   node offsets [n + 1]; one region (masks first):
    const uint8_t* sreg;      //   the region, staged into shared memory when it fits
    uint32_t sreg_bytes;      //   (0: not staged)
    uint32_t so_key, so_rk, so_off;   // byte offsets of keys, ranks, offsets in it
    double margin_x;
    uint32_t* done;           // ticket of the block that advances the step
};

struct LGemmArgs {
    const uint8_t* A;         // M tiles of 128 rows x K (core-matrix layout)
    const uint8_t* B;         // N tiles of 32 rows x K (core-matrix layout)
    const float* bias;
    int K;
    int mode;                 // 0: hidden layer -> bf16 ReLU into out_h; 1: output layer
    uint8_t* out_h;
    float* logits;
    float2* part;
    const uint8_t* cur_buf;
    int prime;                // output layer: write the current buffer (else the other)
    int C, P, Pp, NT;
    uint32_t* status;
};

// ---------------------------------------------------------------------------------
// layouts and small helpers
// ---------------------------------------------------------------------------------

// byte offset of the 8-element chunk (row, k..k+7) in a core-matrix operand whose tiles
// hold `rows` rows x K: 64-wide K blocks of rows/8 groups x 8 chunks x 8 rows x 16 bytes
__host__ __device__ __forceinline__ size_t cm_off(int row, int k, int K, int rows)
{
    const int tile = row / rows, rr = row - tile * rows;
    return (size_t)tile * rows * K * 2 + (size_t)(k >> 6) * (rows * 128) + (size_t)(rr >> 3) * 1024 +
           (size_t)((k & 63) >> 3) * 128 + (size_t)(rr & 7) * 16;
}

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const uint32_t a = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

// ln q(pair | order) of the mixture (1 - eps) softmax + eps / P from the pair's logit
__device__ __forceinline__ float log_q(float l, float lse, float eps, int P)
{
    return logf((1.f - eps) * expf(l - lse) + eps / (float)P);
}

// layer-1 output of one chain for hidden units h0..h0+7: bf16(relu(z * 2^-shift + b1))
// into the layer-2 operand
__device__ __forceinline__ void store_h1(const LearnArgs& L, int c, int h0, const int32_t z[8])
{
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = fmaxf((float)z[j] * L.scale + L.b1[h0 + j], 0.f);
    uint4 q;
    q.x = pack_bf16x2(v[0], v[1]);
    q.y = pack_bf16x2(v[2], v[3]);
    q.z = pack_bf16x2(v[4], v[5]);
    q.w = pack_bf16x2(v[6], v[7]);
    *(uint4*)(L.h1 + cm_off(c, h0, L.H, LR_TM)) = q;
}

// ---------------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------------

// T[p][v][h] = sum_j W1[h][p d + j] E[v][j]  (bf16 products are exact in FP32; j ascending)
__global__ void k_l1_table(const bf16* __restrict__ W1b, int ndp, const bf16* __restrict__ Eb, int n, int d, int H,
                           float* __restrict__ T)
{
    const int pv = blockIdx.x, p = pv / n, v = pv - p * n;
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        float acc = 0.f;
        for (int j = 0; j < d; ++j)
            acc = fmaf(__bfloat162float(W1b[(size_t)h * ndp + p * d + j]), __bfloat162float(Eb[(size_t)v * d + j]), acc);
        T[((size_t)p * n + v) * H + h] = acc;
    }
}

// bound on |z1| before the bias: max over h of sum_p max_v |T[p][v][h]| (float bits of a
// non-negative value order like unsigned integers)
__global__ void k_l1_bound(const float* __restrict__ T, int n, int H, uint32_t* __restrict__ out)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    float s = 0.f;
    for (int p = 0; p < n; ++p) {
        float m = 0.f;
        for (int v = 0; v < n; ++v) m = fmaxf(m, fabsf(T[((size_t)p * n + v) * H + h]));
        s += m;
    }
    atomicMax(out, __float_as_uint(s));
}

// in place: float -> round-to-nearest integer of value * 2^shift
__global__ void k_l1_fix(float* __restrict__ T, int64_t count, float mul)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int32_t q = __float2int_rn(T[i] * mul);
    ((int32_t*)T)[i] = q;
}

// row-major rows x K bf16 -> 32-row core-matrix tiles (rows >= valid are zero)
__global__ void k_pack_b(const bf16* __restrict__ src, int valid, int rows, int K, uint8_t* __restrict__ dst)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int kc = K / 8;
    if (idx >= (int64_t)rows * kc) return;
    const int r = (int)(idx / kc), k = (int)(idx - (int64_t)r * kc) * 8;
    uint4 q = make_uint4(0, 0, 0, 0);
    if (r < valid) q = *(const uint4*)(src + (size_t)r * K + k);
    *(uint4*)(dst + cm_off(r, k, K, LR_TN)) = q;
}

// survivors of every node in score order: rank and key next to the candidate mask
__global__ void k_surv_compact(const uint64_t* __restrict__ amask, const uint32_t* __restrict__ aspos,
                               const uint32_t* __restrict__ aoff, const uint32_t* __restrict__ acnt,
                               const uint32_t* __restrict__ srank, const int64_t* __restrict__ keys, int64_t Sp,
                               int n, uint64_t* __restrict__ smask, uint32_t* __restrict__ srk,
                               int64_t* __restrict__ skey, uint32_t* __restrict__ soff)
{
    const int v = blockIdx.x;
    for (uint32_t j = threadIdx.x; j < acnt[v]; j += blockDim.x) {
        const uint32_t r = srank[(size_t)v * Sp + aspos[aoff[v] + j]];
        smask[aoff[v] + j] = amask[aoff[v] + j];
        srk[aoff[v] + j] = r;
        skey[aoff[v] + j] = keys[(size_t)v * Sp + r];
    }
    if (threadIdx.x == 0) {
        soff[v] = aoff[v];
        if (v == n - 1) soff[n] = aoff[v] + acnt[v];
    }
}

// the current orders' layer-1 sums from scratch and their layer-2 operand rows; dwell
// starts at the current step
__global__ void k_learned_prime(ChainState S, LearnArgs L)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * LR_WARPS + warp;
    if (c >= S.C) return;
    const int n = S.n;
    const uint8_t* o = S.cur_order + (size_t)c * n;
    for (int h0 = lane * 8; h0 < L.H; h0 += 256) {
        uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int p = 0; p < n; ++p) {
            const int32_t* row = L.T + ((size_t)p * n + o[p]) * L.H + h0;
            const int4 q0 = *(const int4*)row, q1 = *(const int4*)(row + 4);
            z[0] += (uint32_t)q0.x; z[1] += (uint32_t)q0.y; z[2] += (uint32_t)q0.z; z[3] += (uint32_t)q0.w;
            z[4] += (uint32_t)q1.x; z[5] += (uint32_t)q1.y; z[6] += (uint32_t)q1.z; z[7] += (uint32_t)q1.w;
        }
        int32_t zi[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) zi[j] = (int32_t)z[j];
        int32_t* dst = L.z1 + (size_t)c * L.H + h0;
        *(int4*)dst = make_int4(zi[0], zi[1], zi[2], zi[3]);
        *(int4*)(dst + 4) = make_int4(zi[4], zi[5], zi[6], zi[7]);
        store_h1(L, c, h0, zi);
    }
    const int64_t t = *S.step;
    for (int i = lane; i < n; i += 32) L.since[(size_t)c * n + i] = t;
    if (lane == 0) L.cur_buf[c] = 0;
}

// ---------------------------------------------------------------------------------
// dense layers on the tensor cores: C[128 x 32] = A[128 x K] B[32 x K]^T per CTA
// ---------------------------------------------------------------------------------
__host__ __device__ constexpr size_t lgemm_smem(int K)
{
    return (size_t)LR_TM * K * 2 + (size_t)LR_TN * K * 2 + 8 * (size_t)(K / 64 + 1) + 16 + 1024;
}

// epilogue of one 128 x 32 tile: TMEM -> bias (+ ReLU -> bf16 operand of the next layer, or
// logits + per-tile softmax partials of the output layer); warp w holds rows 32w..32w+31
__device__ __forceinline__ void lgemm_epilogue(const LGemmArgs& g, uint32_t tmem, int warp, int lane, int mt, int nt)
{
    uint32_t r[32];
    tc_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16), r);
    tc_wait_ld();
    const int row = mt * LR_TM + warp * 32 + lane;
    const int n0 = nt * LR_TN;
    if (g.mode == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaxf(__uint_as_float(r[q * 8 + j]) + g.bias[n0 + q * 8 + j], 0.f);
            uint4 o;
            o.x = pack_bf16x2(v[0], v[1]);
            o.y = pack_bf16x2(v[2], v[3]);
            o.z = pack_bf16x2(v[4], v[5]);
            o.w = pack_bf16x2(v[6], v[7]);
            *(uint4*)(g.out_h + cm_off(row, n0 + q * 8, g.K, LR_TM)) = o;
        }
    } else if (row < g.C) {
        const int cb = g.cur_buf[row];
        const int buf = g.prime ? cb : 1 - cb;
        float* dst = g.logits + ((size_t)buf * g.C + row) * g.Pp + n0;
        float v[32];
        float mx = -INFINITY;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            v[j] = __uint_as_float(r[j]) + g.bias[n0 + j];
            if (n0 + j < g.P) mx = fmaxf(mx, v[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; j += 4) *(float4*)(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (n0 + j < g.P) s += expf(v[j] - mx);
        g.part[((size_t)buf * g.C + row) * g.NT + nt] = make_float2(mx, s);
    }
}

__global__ void __launch_bounds__(128) k_learned_gemm(LGemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int KB = g.K >> 6;
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)LR_TM * g.K * 2;
    uint64_t* bar = (uint64_t*)(sB + (size_t)LR_TN * g.K * 2);
    uint32_t* tslot = (uint32_t*)(bar + KB + 1);
    int* s_ok = (int*)(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockIdx.x, mt = blockIdx.y;

    if (warp == 0) {
        tc_alloc(tslot, 32);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int kb = 0; kb <= KB; ++kb) mbar_init(&bar[kb], 1);
        fence_mbar_init();
        *s_ok = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        const uint64_t pol = l2_policy_evict_last();
        const uint8_t* gB = g.B + (size_t)nt * LR_TN * g.K * 2;
        // the weights do not depend on the previous kernel: fetch them before waiting on it
        for (int kb = 0; kb < KB; ++kb) {
            mbar_arrive_expect_tx(&bar[kb], LR_TM * 128 + LR_TN * 128);
            bulk_g2s(sB + (size_t)kb * LR_TN * 128, gB + (size_t)kb * LR_TN * 128, LR_TN * 128, &bar[kb], pol);
        }
        griddep_wait();
        const uint8_t* gA = g.A + (size_t)mt * LR_TM * g.K * 2;
        for (int kb = 0; kb < KB; ++kb)
            bulk_g2s(sA + (size_t)kb * LR_TM * 128, gA + (size_t)kb * LR_TM * 128, LR_TM * 128, &bar[kb], pol);
        griddep_launch();
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            ok = mbar_wait_bounded(&bar[kb], 0, WAIT_TIMEOUT_NS);
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = tc_smem_desc(sA + (size_t)kb * LR_TM * 128 + kk * 256, 128, 1024);
                const uint64_t bd = tc_smem_desc(sB + (size_t)kb * LR_TN * 128 + kk * 256, 128, 1024);
                tc_mma_bf16(tmem, ad, bd, LR_IDESC, (kb | kk) != 0);
            }
        }
        tc_commit(&bar[KB]);
        if (!ok) {
            *s_ok = 0;
            // copies still in flight land before the block leaves (bounded)
            for (int kb = 0; kb < KB; ++kb) mbar_wait_bounded(&bar[kb], 0, WAIT_TIMEOUT_NS);
        }
    } else {
        griddep_wait();
        griddep_launch();
    }
    const bool done_ok = mbar_wait_bounded(&bar[KB], 0, WAIT_TIMEOUT_NS);
    tc_fence_after();
    const bool all_ok = __syncthreads_and(done_ok && *s_ok);
    if (all_ok) {
        lgemm_epilogue(g, tmem, warp, lane, mt, nt);
    } else if (tid == 0) {
        atomicOr(g.status, STATUS_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 32);
}

// ---------------------------------------------------------------------------------
// the per-chain kernel
// ---------------------------------------------------------------------------------
struct LWarp {
    uint8_t ord[MAXN];
    uint32_t rank[MAXN];
    int64_t key[MAXN];
    int64_t nkey[MAXN];
};

// ln sum_j exp(l_j) of a row from the lane's two tile partials (tiles lane, lane + 32);
// M = the largest tile max, w = the lane's tile weights sum_t exp(m_t - M).  Butterfly
// sums: every lane gets the same bits, and the value depends on the partials alone.
__device__ __forceinline__ float row_lse_v(float2 p0, float2 p1, float& M, float w[2])
{
    float m = fmaxf(p0.x, p1.x);
#pragma unroll
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    M = m;
    w[0] = p0.y > 0.f ? p0.y * expf(p0.x - m) : 0.f;
    w[1] = p1.y > 0.f ? p1.y * expf(p1.x - m) : 0.f;
    float s = w[0] + w[1];
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return m + logf(s);
}

static constexpr int LR_HCH = 3;          // 256-wide hidden chunks per lane (H <= 768)

__device__ __forceinline__ void load_z(const int32_t* row, int lane, int H, int32_t (&z)[LR_HCH][8])
{
#pragma unroll
    for (int q = 0; q < LR_HCH; ++q) {
        const int h0 = lane * 8 + 256 * q;
        if (h0 < H) {
            const int4 u = *(const int4*)(row + h0), v = *(const int4*)(row + h0 + 4);
            z[q][0] = u.x; z[q][1] = u.y; z[q][2] = u.z; z[q][3] = u.w;
            z[q][4] = v.x; z[q][5] = v.y; z[q][6] = v.z; z[q][7] = v.w;
        }
    }
}

// One block's share of a learned MH step: warp w runs chain block * LR_WARPS + w; it
// finishes the previous step (LF_FINISH) and starts the next (LF_START).  The survivors
// are read from `sreg` once the staged copy has landed on `s_bar` (when `staged`), else
// from global memory.  Thread 0 adds the block's re-scored items, and the last of the
// `nblocks` blocks to finish advances the step counter.
__device__ __forceinline__ void learned_chain_block(const ChainState& S, const LearnArgs& L, int flags, int block,
                                                    int nblocks, const uint8_t* sreg, LWarp* sw, int64_t* s_items,
                                                    uint64_t* s_bar, bool staged, bool stage_wait_at_end)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = block * LR_WARPS + warp;
    const int n = S.n, H = L.H, NT = L.NT;
    const int64_t t_dev = *S.step;
    int64_t items = 0;
    if (c < S.C) {
        LWarp& W = sw[warp];
        // ---------------- every load that depends on nothing computed here -------------
        for (int i = lane; i < n; i += 32) {
            W.ord[i] = S.cur_order[(size_t)c * n + i];
            W.rank[i] = S.cur_rank[(size_t)c * n + i];
            W.key[i] = S.cur_key[(size_t)c * n + i];
        }
        double score = S.cur_score[c];
        const double best = S.best_score[c];   // read once: lane 0 updates it below
        int cb = L.cur_buf[c];
        const float2 none = make_float2(-INFINITY, 0.f);
        const float2* pr0 = L.part + (size_t)c * NT;
        const float2* pr1 = L.part + ((size_t)S.C + c) * NT;
        const float2 q00 = lane < NT ? pr0[lane] : none, q01 = lane + 32 < NT ? pr0[lane + 32] : none;
        const float2 q10 = lane < NT ? pr1[lane] : none, q11 = lane + 32 < NT ? pr1[lane + 32] : none;
        int32_t zc[LR_HCH][8], zq[LR_HCH][8];
        load_z(L.z1 + (size_t)c * H, lane, H, zc);
        const bool fin = (flags & LF_FINISH) != 0;
        int af = 0, bf = 0;
        uint32_t pairf = 0;
        float lf0 = 0.f, lf1 = 0.f, lqff = 0.f;
        double uf = 0.0, dpf = 0.0;
        int64_t pk[2] = {0, 0};
        uint32_t prk[2] = {0, 0};
        if (fin) {
            load_z(L.z1p + (size_t)c * H, lane, H, zq);
            af = L.pab[2 * c];
            bf = L.pab[2 * c + 1];
            pairf = L.ppair[c];
            lf0 = L.logits[(size_t)c * L.Pp + pairf];
            lf1 = L.logits[((size_t)S.C + c) * L.Pp + pairf];
            lqff = L.plqf[c];
            uf = L.pu[c];
            dpf = L.pdpart[c];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = lane + 32 * h;
                if (p < n) {
                    pk[h] = L.pkey[(size_t)c * n + p];
                    prk[h] = L.prank[(size_t)c * n + p];
                }
            }
        }
        const int64_t ts = fin ? t_dev + 1 : t_dev;
        U64x4 x;
        if (flags & LF_START) x = philox4x64((uint64_t)ts, (uint64_t)c, 0, 0, S.seed, 0);
        __syncwarp();
        // ---------------- finish step tf: the MH test with the reverse proposal ----------
        if (fin) {
            const int64_t tf = t_dev;
            const int a = af, b = bf;
            const int nb = 1 - cb;
            float M, w[2];
            const float lse = nb ? row_lse_v(q10, q11, M, w) : row_lse_v(q00, q01, M, w);
            const float lrev = log_q(nb ? lf1 : lf0, lse, L.eps, L.P);
            const double corr = (double)lrev - (double)lqff;
            // the proposal's keys: positions a..b hold its re-scored nodes, the rest keep theirs
            uint32_t nrank[2] = {0, 0};
            int node[2] = {-1, -1};
            bool mv = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = lane + 32 * h;
                if (p < n) {
                    if (p >= a && p <= b) {
                        const int v = (p == a) ? W.ord[b] : (p == b) ? W.ord[a] : W.ord[p];
                        node[h] = v;
                        nrank[h] = prk[h];
                        W.nkey[v] = pk[h];
                        mv |= prk[h] != W.rank[v];
                    } else {
                        const int v = W.ord[p];
                        W.nkey[v] = W.key[v];
                    }
                }
            }
            const bool moved = __any_sync(0xffffffffu, mv);
            __syncwarp();
            int acc = 0;
            double s2 = 0.0;
            if (lane == 0) {
                const float luf = logf((float)uf);
                const double xa = (S.literal_log ? dpf : LN10 * dpf) + corr;
                const double margin = 1e-6 * (1.0 + fabs((double)luf)) + (moved ? L.margin_x : 0.0);
                const double gap = (double)luf - xa;
                int exact = 0;
                if (gap > margin) acc = 0;
                else if (gap < -margin) { acc = 1; exact = 1; }
                else exact = 2;
                if (exact && !moved) {
                    // no parent set changes: s' = s bit for bit, the test is ln u < corr
                    s2 = score;
                    if (exact == 2) acc = log(uf) < __dadd_rn(S.literal_log ? 0.0 : __dmul_rn(LN10, 0.0), corr);
                } else if (exact) {
                    for (int i = 0; i < n; ++i) s2 = __dadd_rn(s2, key_to_double(W.nkey[i]));
                    if (exact == 2) {
                        const double delta = __dsub_rn(s2, score);
                        const double lu = log(uf);
                        acc = S.literal_log ? (lu < __dadd_rn(delta, corr))
                                            : (lu < __dadd_rn(__dmul_rn(LN10, delta), corr));
                    }
                }
            }
            acc = __shfl_sync(0xffffffffu, acc, 0);
            s2 = __shfl_sync(0xffffffffu, s2, 0);
            items = b - a + 1;
            if (acc) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int v = node[h];
                    if (v >= 0 && nrank[h] != W.rank[v]) {
                        const size_t si = (size_t)c * n + v;
                        credit_edges(S, c, v, W.rank[v], L.since[si], tf);
                        L.since[si] = tf;
                        W.rank[v] = nrank[h];
                        W.key[v] = W.nkey[v];
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    const uint8_t oa = W.ord[a];
                    W.ord[a] = W.ord[b];
                    W.ord[b] = oa;
                }
                __syncwarp();
                // the proposal's layer-1 sums and network outputs become the current ones
#pragma unroll
                for (int q = 0; q < LR_HCH; ++q) {
                    const int h0 = lane * 8 + 256 * q;
                    if (h0 < H) {
                        int32_t* dst = L.z1 + (size_t)c * H + h0;
                        *(int4*)dst = make_int4(zq[q][0], zq[q][1], zq[q][2], zq[q][3]);
                        *(int4*)(dst + 4) = make_int4(zq[q][4], zq[q][5], zq[q][6], zq[q][7]);
#pragma unroll
                        for (int j = 0; j < 8; ++j) zc[q][j] = zq[q][j];
                    }
                }
                cb = nb;
                score = s2;
                for (int i = lane; i < n; i += 32) {
                    S.cur_order[(size_t)c * n + i] = W.ord[i];
                    S.cur_rank[(size_t)c * n + i] = W.rank[i];
                    S.cur_key[(size_t)c * n + i] = W.key[i];
                }
                if (s2 > best) {
                    for (int i = lane; i < n; i += 32) {
                        S.best_order[(size_t)c * n + i] = W.ord[i];
                        S.best_rank[(size_t)c * n + i] = W.rank[i];
                    }
                    if (lane == 0) S.best_score[c] = s2;
                }
                if (lane == 0) {
                    L.cur_buf[c] = (uint8_t)cb;
                    S.cur_score[c] = s2;
                    S.accepts[c] += 1;
                }
            }
            if (lane == 0 && tf < S.trace_cap) {
                S.trace_score[(size_t)c * S.trace_cap + tf] = score;
                S.trace_accept[(size_t)c * S.trace_cap + tf] = (uint8_t)acc;
            }
            if (tf >= S.burn_in && S.record_every > 0 && ((tf - S.burn_in) % S.record_every) == 0 &&
                (tf - S.burn_in) / S.record_every < S.record_cap) {
                const int64_t ridx = (tf - S.burn_in) / S.record_every;
                for (int i = lane; i < n; i += 32) {
                    uint64_t m = S.pst[W.rank[i]];
                    while (m) {
                        const int slot = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        const int par = slot + (slot >= i ? 1 : 0);
                        atomicOr((unsigned long long*)&S.rec_bits[(((size_t)c * n + i) * n + par) * S.rec_words + (ridx >> 6)],
                                 1ull << (ridx & 63));
                    }
                }
            }
            if (flags & LF_FLUSH) {
                for (int i = lane; i < n; i += 32) {
                    const size_t si = (size_t)c * n + i;
                    credit_edges(S, c, i, W.rank[i], L.since[si], tf + 1);
                    L.since[si] = tf + 1;
                }
            }
            __syncwarp();
        }
        // ---------------- start step ts: draw, swap, re-score, layer 1 ---------------------
        if (flags & LF_START) {
            const float* lrow = L.logits + ((size_t)cb * S.C + c) * L.Pp;
            const float2 p0 = cb ? q10 : q00, p1 = cb ? q11 : q01;
            float M, w[2];
            const float lse = row_lse_v(p0, p1, M, w);
            uint32_t pair;
            float lpair;
            const double umix = __dmul_rn(__dadd_rn((double)(x.x[3] >> 11), 0.5), 0x1p-53);
            if (umix < (double)L.eps) {
                pair = (uint32_t)__umul64hi(x.x[0], (uint64_t)L.P);
                lpair = lrow[pair];
            } else {
                // softmax component: the tile by the tile weights, then the pair within it
                float i0 = w[0], i1 = w[1];
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float t0 = __shfl_up_sync(0xffffffffu, i0, off);
                    const float t1 = __shfl_up_sync(0xffffffffu, i1, off);
                    if (lane >= off) { i0 += t0; i1 += t1; }
                }
                const float tot0 = __shfl_sync(0xffffffffu, i0, 31);
                i1 += tot0;
                const float total = __shfl_sync(0xffffffffu, i1, 31);
                const double u2 = __dmul_rn(__dadd_rn((double)(x.x[2] >> 11), 0.5), 0x1p-53);
                const float target = (float)(u2 * (double)total);
                const unsigned b0 = __ballot_sync(0xffffffffu, i0 > target && w[0] > 0.f);
                const unsigned b1 = __ballot_sync(0xffffffffu, i1 > target && w[1] > 0.f);
                int tsel;
                if (b0) tsel = __ffs(b0) - 1;
                else if (b1) tsel = 32 + __ffs(b1) - 1;
                else {
                    const unsigned nz1 = __ballot_sync(0xffffffffu, w[1] > 0.f);
                    const unsigned nz0 = __ballot_sync(0xffffffffu, w[0] > 0.f);
                    tsel = nz1 ? 63 - __clz(nz1) : (nz0 ? 31 - __clz(nz0) : 0);
                }
                const bool hi = tsel >= 32;
                const float wsel = __shfl_sync(0xffffffffu, hi ? w[1] : w[0], tsel & 31);
                const float before = __shfl_sync(0xffffffffu, hi ? i1 : i0, tsel & 31) - wsel;
                const float mt = __shfl_sync(0xffffffffu, hi ? p1.x : p0.x, tsel & 31);
                const int col = tsel * 32 + lane;
                const bool valid = col < L.P;
                const float lv = valid ? lrow[col] : 0.f;
                const float e = valid ? expf(lv - mt) : 0.f;
                float ie = e;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float tt = __shfl_up_sync(0xffffffffu, ie, off);
                    if (lane >= off) ie += tt;
                }
                const float tin = (target - before) / expf(mt - M);
                const unsigned bw = __ballot_sync(0xffffffffu, valid && ie > tin);
                const unsigned bv = __ballot_sync(0xffffffffu, valid && e > 0.f);
                const int j = bw ? __ffs(bw) - 1 : (bv ? 31 - __clz(bv) : 0);
                pair = (uint32_t)(tsel * 32 + j);
                lpair = __shfl_sync(0xffffffffu, lv, j);
                if (pair >= (uint32_t)L.P) {                      // only with non-finite logits
                    pair = (uint32_t)L.P - 1;
                    lpair = lrow[pair];
                }
            }
            const float lqf = log_q(lpair, lse, L.eps, L.P);
            int a, b;
            pair_decode(n, (uint64_t)pair, a, b);
            // proposed order on the lanes (positions lane, lane + 32) and prefix masks
            int v[2];
            uint64_t bit[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = lane + 32 * h;
                v[h] = 0;
                bit[h] = 0;
                if (p < n) {
                    v[h] = W.ord[(p == a) ? b : (p == b) ? a : p];
                    bit[h] = 1ull << v[h];
                }
            }
            uint64_t s0 = bit[0], s1 = bit[1];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint64_t t0 = __shfl_up_sync(0xffffffffu, s0, off);
                const uint64_t t1 = __shfl_up_sync(0xffffffffu, s1, off);
                if (lane >= off) { s0 |= t0; s1 |= t1; }
            }
            const uint64_t first_half = __shfl_sync(0xffffffffu, s0, 31);
            // survivors: shared-memory copy once it has landed, else the global arrays
            const uint64_t* smask = L.smask;
            const int64_t* skey = L.skey;
            const uint32_t* srk = L.srk;
            const uint32_t* soff = L.soff;
            if (staged && mbar_wait_bounded(s_bar, 0, WAIT_TIMEOUT_NS)) {
                smask = (const uint64_t*)sreg;
                skey = (const int64_t*)(sreg + L.so_key);
                srk = (const uint32_t*)(sreg + L.so_rk);
                soff = (const uint32_t*)(sreg + L.so_off);
            }
            // survivors in score order: the first consistent one wins (the empty set, always
            // consistent, is the last survivor)
            uint32_t wj[2] = {0, 0}, wj1[2] = {0, 0};
            uint64_t wnpc[2] = {0, 0};
            bool act[2] = {false, false};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int p = lane + 32 * h;
                if (p < n && p >= a && p <= b) {
                    const int nd = v[h];
                    const uint64_t excl = (h == 0 ? s0 : (s1 | first_half)) & ~bit[h];
                    wnpc[h] = ~compress_pred(excl, nd);
                    wj[h] = soff[nd];
                    wj1[h] = soff[nd + 1];
                    act[h] = true;
                }
            }
            span_walk(smask, wj, wj1, wnpc, act, lane, 8);
            double dpart = 0.0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!act[h]) continue;
                const int p = lane + 32 * h;
                const int nd = v[h];
                const uint32_t r = srk[wj[h]];
                const int64_t k = skey[wj[h]];
                L.prank[(size_t)c * n + p] = r;
                L.pkey[(size_t)c * n + p] = k;
                dpart += key_to_double(k) - key_to_double(W.key[nd]);
            }
#pragma unroll
            for (int off = 16; off; off >>= 1) dpart += __shfl_down_sync(0xffffffffu, dpart, off);
            // layer 1 of the proposal: four table rows change
            const int va = W.ord[a], vb = W.ord[b];
            const int32_t* Ta_new = L.T + ((size_t)a * n + vb) * H;
            const int32_t* Tb_new = L.T + ((size_t)b * n + va) * H;
            const int32_t* Ta_old = L.T + ((size_t)a * n + va) * H;
            const int32_t* Tb_old = L.T + ((size_t)b * n + vb) * H;
#pragma unroll
            for (int q = 0; q < LR_HCH; ++q) {
                const int h0 = lane * 8 + 256 * q;
                if (h0 < H) {
                    int32_t zi[8];
#pragma unroll
                    for (int o = 0; o < 8; o += 4) {
                        const int4 an = *(const int4*)(Ta_new + h0 + o), bn = *(const int4*)(Tb_new + h0 + o);
                        const int4 ao = *(const int4*)(Ta_old + h0 + o), bo = *(const int4*)(Tb_old + h0 + o);
                        zi[o + 0] = (int32_t)((uint32_t)zc[q][o + 0] + (uint32_t)an.x + (uint32_t)bn.x - (uint32_t)ao.x - (uint32_t)bo.x);
                        zi[o + 1] = (int32_t)((uint32_t)zc[q][o + 1] + (uint32_t)an.y + (uint32_t)bn.y - (uint32_t)ao.y - (uint32_t)bo.y);
                        zi[o + 2] = (int32_t)((uint32_t)zc[q][o + 2] + (uint32_t)an.z + (uint32_t)bn.z - (uint32_t)ao.z - (uint32_t)bo.z);
                        zi[o + 3] = (int32_t)((uint32_t)zc[q][o + 3] + (uint32_t)an.w + (uint32_t)bn.w - (uint32_t)ao.w - (uint32_t)bo.w);
                    }
                    int32_t* zp = L.z1p + (size_t)c * H + h0;
                    *(int4*)zp = make_int4(zi[0], zi[1], zi[2], zi[3]);
                    *(int4*)(zp + 4) = make_int4(zi[4], zi[5], zi[6], zi[7]);
                    store_h1(L, c, h0, zi);
                }
            }
            if (lane == 0) {
                L.pab[2 * c] = (uint8_t)a;
                L.pab[2 * c + 1] = (uint8_t)b;
                L.ppair[c] = pair;
                L.plqf[c] = lqf;
                L.pu[c] = __dmul_rn(__dadd_rn((double)(x.x[1] >> 12), 0.5), 0x1p-52);
                L.pdpart[c] = dpart;
            }
        }
    }
    if (lane == 0) s_items[warp] = items;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (staged && stage_wait_at_end) mbar_wait_bounded(s_bar, 0, WAIT_TIMEOUT_NS);   // no copy left in flight
        if (flags & LF_FINISH) {
            int64_t tot = 0;
            for (int w = 0; w < LR_WARPS; ++w) tot += s_items[w];
            if (tot) atomicAdd((unsigned long long*)S.items_total, (unsigned long long)tot);
            // the last block advances the step counter
            __threadfence();
            const uint32_t ticket = atomicAdd(L.done, 1u);
            if (ticket == (uint32_t)nblocks - 1) {
                const int64_t t_end = t_dev + 1;
                *S.step = t_end;
                if (S.record_every > 0 && t_end > S.burn_in) {
                    const int64_t r = (t_end - 1 - S.burn_in) / S.record_every + 1;
                    *S.rec_count = r < S.record_cap ? r : S.record_cap;
                }
                *L.done = 0;
                __threadfence();
            }
        }
    }
}


__global__ void __launch_bounds__(32 * LR_WARPS) k_learned_chain(ChainState S, LearnArgs L, int flags)
{
    extern __shared__ __align__(16) uint8_t sreg[];        // the survivors, staged
    __shared__ LWarp sw[LR_WARPS];
    __shared__ int64_t s_items[LR_WARPS];
    __shared__ __align__(8) uint64_t s_bar;
    const bool staged = L.sreg_bytes > 0;
    if (threadIdx.x == 0 && staged) {
        // the survivors do not change between launches: fetch them before the wait
        mbar_init(&s_bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&s_bar, L.sreg_bytes);
        bulk_g2s(sreg, L.sreg, L.sreg_bytes, &s_bar, l2_policy_evict_last());
    }
    griddep_wait();
    griddep_launch();
    __syncthreads();
    learned_chain_block(S, L, flags, blockIdx.x, gridDim.x, sreg, sw, s_items, &s_bar, staged, true);
}

// ---------------------------------------------------------------------------------
// the persistent learned step
// ---------------------------------------------------------------------------------
// One cooperative launch runs many MH steps.  A step is three phases -- layer 2 on the
// proposals' layer-1 outputs, the output layer, then the chains (finish the step, start
// the next) -- separated by grid-wide barriers instead of kernel boundaries.  Every CTA
// keeps its layer-2 or output-layer weight tile in shared memory and its TMEM columns for
// the whole launch, and the chain CTAs keep the survivors staged; only the activations
// and the chains' outputs pass through L2.  CTAs [0, n3) own output-layer tiles, CTAs
// [n3, n3 + n2) layer-2 tiles, and CTAs [0, nc) four chains each.
struct PersistArgs {
    int iters;
    int n2, n3, nc;
    int nt2, nt3;                 // N tiles of layer 2 (H / 32) and of the output layer (NT)
    uint32_t* gsync;              // grid barrier counter, zero at launch
    uint32_t a_off, b_off, bar_off;   // dynamic shared memory: A tile, B tile, barriers
    int staged;                   // chain CTAs stage the survivors at [0, L.sreg_bytes)
};

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid-wide barrier number k (1, 2, ...) of the launch: every CTA's writes before it are
// visible after it, to generic loads and to the bulk copies (async proxy) issued after
// it.  Bounded: false once the wait has run out (status gets STATUS_TIMEOUT).
__device__ __forceinline__ bool grid_barrier(uint32_t* counter, uint32_t target, uint32_t* status, int* s_ok)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        bool ok = true;
        if (ld_acquire_gpu(counter) < target) {
            const uint64_t t0 = global_timer_ns();
            while (ld_acquire_gpu(counter) < target) {
                if (global_timer_ns() - t0 > WAIT_TIMEOUT_NS) {
                    ok = false;
                    break;
                }
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!ok) atomicOr(status, STATUS_TIMEOUT);
        *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// one GEMM tile of a phase: A (128 rows x K) by bulk copies, one mbarrier per 64-wide K
// block (phase `parity`), MMAs into `tmem` as the blocks land, commit, epilogue
__device__ __forceinline__ bool persist_gemm(const LGemmArgs& g, int mt, int nt, uint8_t* sA, const uint8_t* sB,
                                             uint64_t* bar, uint32_t parity, uint32_t tmem, int* s_okg)
{
    const int KB = g.K >> 6, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        *s_okg = 1;
        const uint64_t pol = l2_policy_evict_last();
        const uint8_t* gA = g.A + (size_t)mt * LR_TM * g.K * 2;
        for (int kb = 0; kb < KB; ++kb) {
            mbar_arrive_expect_tx(&bar[kb], LR_TM * 128);
            bulk_g2s(sA + (size_t)kb * LR_TM * 128, gA + (size_t)kb * LR_TM * 128, LR_TM * 128, &bar[kb], pol);
        }
        bool ok = true;
        for (int kb = 0; kb < KB && ok; ++kb) {
            ok = mbar_wait_bounded(&bar[kb], parity, WAIT_TIMEOUT_NS);
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = tc_smem_desc(sA + (size_t)kb * LR_TM * 128 + kk * 256, 128, 1024);
                const uint64_t bd = tc_smem_desc(sB + (size_t)kb * LR_TN * 128 + kk * 256, 128, 1024);
                tc_mma_bf16(tmem, ad, bd, LR_IDESC, (kb | kk) != 0);
            }
        }
        tc_commit(&bar[KB]);
        if (!ok) {
            *s_okg = 0;
            for (int kb = 0; kb < KB; ++kb) mbar_wait_bounded(&bar[kb], parity, WAIT_TIMEOUT_NS);
        }
    }
    __syncthreads();
    const bool done_ok = mbar_wait_bounded(&bar[KB], parity, WAIT_TIMEOUT_NS);
    tc_fence_after();
    const bool all_ok = __syncthreads_and(done_ok && *s_okg);
    if (all_ok) lgemm_epilogue(g, tmem, warp, lane, mt, nt);
    else if (tid == 0) atomicOr(g.status, STATUS_TIMEOUT);
    tc_fence_before();
    return all_ok;
}

__global__ void __launch_bounds__(32 * LR_WARPS, 1)
    k_learned_persist(ChainState S, LearnArgs L, LGemmArgs g2, LGemmArgs g3, PersistArgs P)
{
    extern __shared__ __align__(1024) uint8_t psm_raw[];
    uint8_t* psm = (uint8_t*)(((uintptr_t)psm_raw + 1023) & ~(uintptr_t)1023);
    __shared__ LWarp sw[LR_WARPS];
    __shared__ int64_t s_items[LR_WARPS];
    __shared__ uint32_t s_tslot;
    __shared__ int s_okg, s_okb;                       // GEMM and grid-barrier outcomes
    const int cta = blockIdx.x, tid = threadIdx.x;
    const bool is3 = cta < P.n3, is2 = !is3 && cta < P.n3 + P.n2, isc = cta < P.nc;
    const bool gemm = is3 || is2;
    const LGemmArgs& g = is3 ? g3 : g2;
    const int tile = is3 ? cta : cta - P.n3;
    const int ntiles = is3 ? P.nt3 : P.nt2;
    const int mt = gemm ? tile / ntiles : 0, nt = gemm ? tile - mt * ntiles : 0;
    const int KB = g2.K >> 6;
    uint8_t* sA = psm + P.a_off;
    uint8_t* sB = psm + P.b_off;
    uint64_t* bar = (uint64_t*)(psm + P.bar_off);      // [KB] A blocks, [KB] commit, [KB+1] B, [KB+2] survivors
    const bool staged = isc && P.staged;
    if (gemm && tid < 32) {
        tc_alloc(&s_tslot, 32);
        tc_relinquish();
    }
    if (tid == 0) {
        for (int kb = 0; kb < KB + 3; ++kb) mbar_init(&bar[kb], 1);
        fence_mbar_init();
        if (gemm) {
            // the CTA's weight tile, resident for the launch
            const uint8_t* gB = g.B + (size_t)nt * LR_TN * g.K * 2;
            mbar_arrive_expect_tx(&bar[KB + 1], (uint32_t)(KB * LR_TN * 128));
            for (int kb = 0; kb < KB; ++kb)
                bulk_g2s(sB + (size_t)kb * LR_TN * 128, gB + (size_t)kb * LR_TN * 128, LR_TN * 128, &bar[KB + 1],
                         l2_policy_evict_last());
        }
        if (staged) {
            mbar_arrive_expect_tx(&bar[KB + 2], L.sreg_bytes);
            bulk_g2s(psm, L.sreg, L.sreg_bytes, &bar[KB + 2], l2_policy_evict_last());
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tslot;
    bool ok = true;
    if (gemm) ok = mbar_wait_bounded(&bar[KB + 1], 0, WAIT_TIMEOUT_NS);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(g2.status, STATUS_TIMEOUT);
    } else {
        const uint32_t G = (uint32_t)gridDim.x;
        uint32_t nb = 0;                                // barriers passed
        for (int it = 0; it < P.iters; ++it) {
            const uint32_t parity = (uint32_t)(it & 1);
            if (is2 && !persist_gemm(g2, mt, nt, sA, sB, bar, parity, tmem, &s_okg)) ok = false;
            if (!grid_barrier(P.gsync, G * ++nb, g2.status, &s_okb) || !ok) break;
            if (is3 && !persist_gemm(g3, mt, nt, sA, sB, bar, parity, tmem, &s_okg)) ok = false;
            if (!grid_barrier(P.gsync, G * ++nb, g2.status, &s_okb) || !ok) break;
            if (isc)
                learned_chain_block(S, L, LF_FINISH | LF_START, cta, P.nc, psm, sw, s_items, &bar[KB + 2], staged,
                                    false);
            if (it + 1 < P.iters && !grid_barrier(P.gsync, G * ++nb, g2.status, &s_okb)) break;
        }
    }
    if (tid == 0 && staged) mbar_wait_bounded(&bar[KB + 2], 0, WAIT_TIMEOUT_NS);   // no copy left in flight
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (gemm && tid < 32) tc_dealloc(tmem, 32);
}

// current logits of every chain (row stride P)
__global__ void k_gather_logits(const float* __restrict__ logits, const uint8_t* __restrict__ cur_buf, int C, int P,
                                int Pp, float* __restrict__ out)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)C * P) return;
    const int c = (int)(idx / P), j = (int)(idx - (int64_t)c * P);
    out[idx] = logits[((size_t)cur_buf[c] * C + c) * Pp + j];
}

struct LearnedPath {
    void* block = nullptr;
    size_t bytes = 0;
    int C = 0, n = 0, H = 0, d = 0, P = 0, Pp = 0, NT = 0, Mt = 0;
    int64_t alive = 0;
    int shift = 0;
    LearnArgs L{};
    LGemmArgs g2{}, g3{};
    uint8_t *wp2 = nullptr, *wp3 = nullptr, *h2 = nullptr;
    uint32_t* bound = nullptr;
    uint32_t* status = nullptr;
    const bn_table* table = nullptr;
    const uint64_t* amask = nullptr;     // the table's survivors the path was built from
    bool weights_ok = false;
    bool primed = false;
    bool pdl = true;
    cudaGraphExec_t exec = nullptr;
    uint32_t* gsync = nullptr;           // grid barrier counter of the persistent launch
    int persist = -1;                    // persistent launch: -1 not checked, 0 no, 1 yes
    PersistArgs pa{};
    size_t persist_smem = 0;
};

}  // namespace bn

using namespace bn;

static bool learned_fits(const bn_chains* ch)
{
    const bn_mlp* m = ch->mlp;
    return m && ch->t->scan_mode == BN_SCAN_PRUNED && ch->t->amask && m->H % 64 == 0 && m->H <= LR_MAX_H &&
           m->n == ch->S.n;
}

bool bn::learned_path(const bn_chains* ch) { return ch->S.mode == BN_PROPOSAL_LEARNED && learned_fits(ch); }

void bn::learned_invalidate(LearnedPath* lp, bool weights)
{
    if (!lp) return;
    lp->primed = false;
    if (weights) lp->weights_ok = false;
}

void bn::learned_free(LearnedPath* lp)
{
    if (!lp) return;
    if (lp->exec) cudaGraphExecDestroy(lp->exec);
    cudaFree(lp->block);
    delete lp;
}

// device buffers of the path (sizes from the chains, the network and the table)
static int learned_alloc(bn_chains* ch)
{
    const bn_mlp* m = ch->mlp;
    const bn_table* t = ch->t;
    LearnedPath* lp = ch->lp;
    const int C = ch->S.C, n = ch->S.n, H = m->H, P = m->P, Pp = m->Pp;
    if (lp && lp->C == C && lp->n == n && lp->H == H && lp->d == m->d && lp->table == t &&
        lp->alive == t->alive_total && lp->amask == t->amask)
        return BN_OK;
    if (lp) {
        learned_free(lp);
        ch->lp = nullptr;
    }
    lp = new LearnedPath();
    lp->C = C;
    lp->n = n;
    lp->H = H;
    lp->d = m->d;
    lp->P = P;
    lp->Pp = Pp;
    lp->NT = Pp / LR_TN;
    lp->Mt = (C + LR_TM - 1) / LR_TM;
    lp->table = t;
    lp->alive = t->alive_total;
    const size_t nn = (size_t)n * n, Cs = (size_t)C, A_bytes = (size_t)lp->Mt * LR_TM * H * 2;
    const size_t alive = (size_t)std::max<int64_t>(t->alive_total, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_T = take(4 * nn * H), o_wp2 = take((size_t)H * H * 2), o_wp3 = take((size_t)Pp * H * 2),
                 o_h1 = take(A_bytes), o_h2 = take(A_bytes), o_z1 = take(4 * Cs * H), o_z1p = take(4 * Cs * H),
                 o_lg = take(4 * 2 * Cs * Pp), o_part = take(8 * 2 * Cs * lp->NT), o_cb = take(Cs),
                 o_since = take(8 * Cs * n), o_prank = take(4 * Cs * n), o_pkey = take(8 * Cs * n), o_pab = take(2 * Cs),
                 o_pair = take(4 * Cs), o_lqf = take(4 * Cs), o_pu = take(8 * Cs), o_dp = take(8 * Cs),
                 o_done = take(4), o_bound = take(4), o_status = take(4), o_gsync = take(4);
    // survivors region [masks | keys | ranks | node offsets], each part 16-byte aligned
    const size_t r_key = (size_t)round_up((int64_t)(8 * alive), 16), r_rk = r_key + (size_t)round_up((int64_t)(8 * alive), 16),
                 r_off = r_rk + (size_t)round_up((int64_t)(4 * alive), 16),
                 r_end = r_off + (size_t)round_up((int64_t)(4 * (n + 1)), 16);
    const size_t o_sreg = take(r_end);
    cudaError_t e = cudaMalloc(&lp->block, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete lp;
        return set_error(BN_ENOMEM, "learned proposal: %zu bytes: %s", off, cudaGetErrorString(e));
    }
    lp->bytes = off;
    uint8_t* B = (uint8_t*)lp->block;
    LearnArgs& L = lp->L;
    L.H = H;
    L.P = P;
    L.Pp = Pp;
    L.NT = lp->NT;
    L.T = (const int32_t*)(B + o_T);
    L.b1 = m->b1;
    L.h1 = B + o_h1;
    L.z1 = (int32_t*)(B + o_z1);
    L.z1p = (int32_t*)(B + o_z1p);
    L.logits = (const float*)(B + o_lg);
    L.part = (const float2*)(B + o_part);
    L.cur_buf = B + o_cb;
    L.since = (int64_t*)(B + o_since);
    L.prank = (uint32_t*)(B + o_prank);
    L.pkey = (int64_t*)(B + o_pkey);
    L.pab = B + o_pab;
    L.ppair = (uint32_t*)(B + o_pair);
    L.plqf = (float*)(B + o_lqf);
    L.pu = (double*)(B + o_pu);
    L.pdpart = (double*)(B + o_dp);
    L.sreg = B + o_sreg;
    L.smask = (const uint64_t*)(B + o_sreg);
    L.skey = (const int64_t*)(B + o_sreg + r_key);
    L.srk = (const uint32_t*)(B + o_sreg + r_rk);
    L.soff = (const uint32_t*)(B + o_sreg + r_off);
    L.so_key = (uint32_t)r_key;
    L.so_rk = (uint32_t)r_rk;
    L.so_off = (uint32_t)r_off;
    L.sreg_bytes = r_end <= (size_t)LR_STAGE_MAX ? (uint32_t)r_end : 0u;
    lp->amask = t->amask;
    L.margin_x = mh_margin(n, t->max_abs_survivor);
    L.done = (uint32_t*)(B + o_done);
    lp->wp2 = B + o_wp2;
    lp->wp3 = B + o_wp3;
    lp->h2 = B + o_h2;
    lp->bound = (uint32_t*)(B + o_bound);
    lp->status = (uint32_t*)(B + o_status);
    lp->gsync = (uint32_t*)(B + o_gsync);
    ch->lp = lp;
    return BN_OK;
}

static unsigned blocks_of(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// the network's weights in the path's layouts: the layer-1 table in fixed point, the
// packed layer-2/3 tiles, and the survivors next to their ranks and keys
static int learned_weights(bn_chains* ch, cudaStream_t s)
{
    LearnedPath* lp = ch->lp;
    const bn_mlp* m = ch->mlp;
    const bn_table* t = ch->t;
    const int n = lp->n, H = lp->H;
    BN_CUDA(cudaMemsetAsync(lp->block, 0, lp->bytes, s));
    float* Tf = (float*)lp->L.T;
    k_l1_table<<<n * n, 256, 0, s>>>(m->W1b, m->ndp, m->Eb, n, m->d, H, Tf);
    BN_LAUNCH_CHECK("k_l1_table");
    k_l1_bound<<<blocks_of(H), 256, 0, s>>>(Tf, n, H, lp->bound);
    BN_LAUNCH_CHECK("k_l1_bound");
    uint32_t hb = 0;
    BN_CUDA(cudaMemcpyAsync(&hb, lp->bound, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    float bnd;
    std::memcpy(&bnd, &hb, 4);
    if (!(bnd < 0x1p29f)) return set_error(BN_EUNSUPPORTED, "learned proposal: layer-1 weights too large (%g)", bnd);
    // |z| <= bound 2^shift + n/2 < 2^31
    int shift = 24;
    while (shift > 0 && (double)bnd * std::ldexp(1.0, shift) >= 0x1p30) --shift;
    lp->shift = shift;
    lp->L.scale = std::ldexp(1.0f, -shift);
    const int64_t cnt = (int64_t)n * n * H;
    k_l1_fix<<<blocks_of(cnt), 256, 0, s>>>(Tf, cnt, std::ldexp(1.0f, shift));
    BN_LAUNCH_CHECK("k_l1_fix");
    k_pack_b<<<blocks_of((int64_t)H * (H / 8)), 256, 0, s>>>(m->W2b, H, H, H, lp->wp2);
    BN_LAUNCH_CHECK("k_pack_b");
    k_pack_b<<<blocks_of((int64_t)lp->Pp * (H / 8)), 256, 0, s>>>(m->W3b, lp->Pp, lp->Pp, H, lp->wp3);
    BN_LAUNCH_CHECK("k_pack_b");
    k_surv_compact<<<n, 128, 0, s>>>(t->amask, t->aspos, t->aoff, t->acnt, t->srank, t->keys, t->Sp, n,
                                     (uint64_t*)lp->L.smask, (uint32_t*)lp->L.srk, (int64_t*)lp->L.skey,
                                     (uint32_t*)lp->L.soff);
    BN_LAUNCH_CHECK("k_surv_compact");
    lp->L.b1 = m->b1;
    lp->L.eps = ch->S.eps_mix;
    LGemmArgs g{};
    g.K = H;
    g.C = lp->C;
    g.P = lp->P;
    g.Pp = lp->Pp;
    g.NT = lp->NT;
    g.cur_buf = lp->L.cur_buf;
    g.status = lp->status;
    lp->g2 = g;
    lp->g2.A = lp->L.h1;
    lp->g2.B = lp->wp2;
    lp->g2.bias = m->b2;
    lp->g2.mode = 0;
    lp->g2.out_h = lp->h2;
    lp->g3 = g;
    lp->g3.A = lp->h2;
    lp->g3.B = lp->wp3;
    lp->g3.bias = m->b3;
    lp->g3.mode = 1;
    lp->g3.logits = (float*)lp->L.logits;
    lp->g3.part = (float2*)lp->L.part;
    static unsigned long long ctx[64] = {0};
    if (first_in_context(ctx)) {
        BN_CUDA(cudaFuncSetAttribute(k_learned_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)lgemm_smem(LR_MAX_H)));
        BN_CUDA(cudaFuncSetAttribute(k_learned_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, LR_STAGE_MAX));
    }
    if (lp->exec) {
        cudaGraphExecDestroy(lp->exec);
        lp->exec = nullptr;
    }
    lp->weights_ok = true;
    lp->primed = false;
    return BN_OK;
}

static int launch_gemm(LearnedPath* lp, const LGemmArgs& g, int prime, cudaStream_t s)
{
    LGemmArgs a = g;
    a.prime = prime;
    const unsigned nx = (unsigned)(g.mode == 0 ? lp->H / LR_TN : lp->NT);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nx, (unsigned)lp->Mt, 1);
    cfg.blockDim = dim3(128, 1, 1);
    cfg.dynamicSmemBytes = lgemm_smem(lp->H);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = lp->pdl ? 1 : 0;
    BN_CUDA(cudaLaunchKernelEx(&cfg, k_learned_gemm, a));
    BN_LAUNCH_CHECK("k_learned_gemm");
    return BN_OK;
}

static int launch_chain(bn_chains* ch, int flags, cudaStream_t s)
{
    LearnedPath* lp = ch->lp;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((lp->C + LR_WARPS - 1) / LR_WARPS), 1, 1);
    cfg.blockDim = dim3(32 * LR_WARPS, 1, 1);
    cfg.dynamicSmemBytes = lp->L.sreg_bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = lp->pdl ? 1 : 0;
    BN_CUDA(cudaLaunchKernelEx(&cfg, k_learned_chain, ch->S, lp->L, flags));
    BN_LAUNCH_CHECK("k_learned_chain");
    return BN_OK;
}

// one step's network on the proposals, then finish it and start the next
static int launch_iter(bn_chains* ch, int flags, cudaStream_t s)
{
    int rc;
    if ((rc = launch_gemm(ch->lp, ch->lp->g2, 0, s))) return rc;
    if ((rc = launch_gemm(ch->lp, ch->lp->g3, 0, s))) return rc;
    return launch_chain(ch, flags, s);
}

// the current orders' layer-1 sums and network outputs
static int learned_prime(bn_chains* ch, cudaStream_t s)
{
    LearnedPath* lp = ch->lp;
    k_learned_prime<<<(lp->C + LR_WARPS - 1) / LR_WARPS, 32 * LR_WARPS, 0, s>>>(ch->S, lp->L);
    BN_LAUNCH_CHECK("k_learned_prime");
    int rc;
    if ((rc = launch_gemm(lp, lp->g2, 1, s))) return rc;
    if ((rc = launch_gemm(lp, lp->g3, 1, s))) return rc;
    lp->primed = true;
    return BN_OK;
}

int bn::learned_setup(bn_chains* ch, cudaStream_t s)
{
    int rc = learned_alloc(ch);
    if (rc) return rc;
    if (!ch->lp->weights_ok && (rc = learned_weights(ch, s))) return rc;
    if (!ch->lp->primed && (rc = learned_prime(ch, s))) return rc;
    return BN_OK;
}

// the G-iteration graph of the steady state (captured once per set-up)
static int learned_graph(bn_chains* ch, cudaStream_t s)
{
    LearnedPath* lp = ch->lp;
    if (lp->exec) return BN_OK;
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaGraph_t g = nullptr;
        BN_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = BN_OK;
        const int64_t l0 = bn_kernel_launches();
        for (int i = 0; i < LR_GRAPH_ITERS && rc == BN_OK; ++i) rc = launch_iter(ch, LF_FINISH | LF_START, s);
        count_launches(-(bn_kernel_launches() - l0));       // captured, not run
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (rc == BN_OK && ce == cudaSuccess) {
            cudaError_t ie = cudaGraphInstantiate(&lp->exec, g, 0);
            cudaGraphDestroy(g);
            if (ie == cudaSuccess) return BN_OK;
            lp->exec = nullptr;
        } else if (g) {
            cudaGraphDestroy(g);
        }
        cudaGetLastError();
        if (!lp->pdl) return set_error(BN_ECUDA, "learned proposal: graph capture failed");
        lp->pdl = false;                                   // retry with plain stream order
    }
    return set_error(BN_ECUDA, "learned proposal: graph capture failed");
}

// the persistent launch's plan: CTAs per role, shared-memory layout, and whether every
// CTA can be resident at once (a cooperative launch needs that)
static int persist_setup(bn_chains* ch)
{
    LearnedPath* lp = ch->lp;
    if (lp->persist >= 0) return BN_OK;
    lp->persist = 0;
    PersistArgs& P = lp->pa;
    P.nt2 = lp->H / LR_TN;
    P.nt3 = lp->NT;
    P.n2 = P.nt2 * lp->Mt;
    P.n3 = P.nt3 * lp->Mt;
    P.nc = (lp->C + LR_WARPS - 1) / LR_WARPS;
    P.gsync = lp->gsync;
    const size_t sreg = lp->L.sreg_bytes;
    const size_t a_bytes = (size_t)LR_TM * lp->H * 2, b_bytes = (size_t)LR_TN * lp->H * 2;
    const size_t bars = 8 * (size_t)(lp->H / 64 + 3);
    const int dev = device_id();
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return BN_OK;
    }
    const size_t static_smem = sizeof(LWarp) * LR_WARPS + 64 + 1024;   // + alignment slack
    auto layout = [&](bool stage) {
        P.staged = stage ? 1 : 0;
        const size_t a = stage ? (size_t)round_up((int64_t)sreg, 1024) : 0;
        P.a_off = (uint32_t)a;
        P.b_off = (uint32_t)(a + a_bytes);
        P.bar_off = (uint32_t)(a + a_bytes + b_bytes);
        return a + a_bytes + b_bytes + bars + 1024;
    };
    size_t smem = layout(sreg > 0);
    if (smem + static_smem > (size_t)optin) smem = layout(false);     // survivors from global memory
    if (smem + static_smem > (size_t)optin) return BN_OK;
    if (cudaFuncSetAttribute(k_learned_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return BN_OK;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_learned_persist, 32 * LR_WARPS, smem) != cudaSuccess) {
        cudaGetLastError();
        return BN_OK;
    }
    const int grid = std::max(P.n2 + P.n3, P.nc);
    if ((int64_t)per_sm * sm_count() < grid) return BN_OK;
    lp->persist_smem = smem;
    lp->persist = 1;
    return BN_OK;
}

// `iters` learned steps (each: layer 2, output layer, finish + start) in one cooperative
// launch
static int launch_persist(bn_chains* ch, int iters, cudaStream_t s)
{
    LearnedPath* lp = ch->lp;
    PersistArgs P = lp->pa;
    P.iters = iters;
    BN_CUDA(cudaMemsetAsync(lp->gsync, 0, sizeof(uint32_t), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::max(P.n2 + P.n3, P.nc), 1, 1);
    cfg.blockDim = dim3(32 * LR_WARPS, 1, 1);
    cfg.dynamicSmemBytes = lp->persist_smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BN_CUDA(cudaLaunchKernelEx(&cfg, k_learned_persist, ch->S, lp->L, lp->g2, lp->g3, P));
    BN_LAUNCH_CHECK("k_learned_persist");
    return BN_OK;
}

static constexpr int LR_PERSIST_ITERS = 256;   // learned steps per persistent launch

int bn::learned_step(bn_chains* ch, int64_t steps, cudaStream_t s)
{
    int rc = learned_setup(ch, s);
    if (rc) return rc;
    if (steps <= 0) return BN_OK;
    if ((rc = launch_chain(ch, LF_START, s))) return rc;
    int64_t mid = steps - 1;
    if (ch->learned_launch == BN_LEARNED_LAUNCH_AUTO && mid > 0 && (rc = persist_setup(ch))) return rc;
    if (ch->learned_launch == BN_LEARNED_LAUNCH_AUTO && ch->lp->persist == 1) {
        for (; mid > 0;) {
            const int k = (int)std::min<int64_t>(mid, LR_PERSIST_ITERS);
            if ((rc = launch_persist(ch, k, s))) return rc;
            mid -= k;
        }
    }
    if (mid >= LR_GRAPH_ITERS) {
        if ((rc = learned_graph(ch, s))) return rc;
        for (; mid >= LR_GRAPH_ITERS; mid -= LR_GRAPH_ITERS) {
            BN_CUDA(cudaGraphLaunch(ch->lp->exec, s));
            count_launches(3 * LR_GRAPH_ITERS);
        }
    }
    for (; mid > 0; --mid)
        if ((rc = launch_iter(ch, LF_FINISH | LF_START, s))) return rc;
    if ((rc = launch_gemm(ch->lp, ch->lp->g2, 0, s)) || (rc = launch_gemm(ch->lp, ch->lp->g3, 0, s)) ||
        (rc = launch_chain(ch, LF_FINISH | LF_FLUSH, s)))
        return rc;
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, ch->lp->status, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "learned proposal: a bounded device wait expired");
    return BN_OK;
}

int bn::learned_read_logits(const bn_chains* ch, float* out, int mem, cudaStream_t s)
{
    const LearnedPath* lp = ch->lp;
    if (!lp || !lp->primed) return set_error(BN_EINVAL, "bn_chains_read: no learned-proposal outputs (set a learned proposal on a pruned table and step)");
    const int64_t cnt = (int64_t)lp->C * lp->P;
    float* d = out;
    float* tmp = nullptr;
    if (mem == BN_MEM_HOST) {
        BN_CUDA(cudaMallocAsync((void**)&tmp, 4 * (size_t)cnt, s));
        d = tmp;
    }
    k_gather_logits<<<blocks_of(cnt), 256, 0, s>>>(lp->L.logits, lp->L.cur_buf, lp->C, lp->P, lp->Pp, d);
    BN_LAUNCH_CHECK("k_gather_logits");
    if (mem == BN_MEM_HOST) {
        BN_CUDA(cudaMemcpyAsync(out, tmp, 4 * (size_t)cnt, cudaMemcpyDeviceToHost, s));
        BN_CUDA(cudaFreeAsync(tmp, s));
    }
    BN_CUDA(cudaStreamSynchronize(s));
    return BN_OK;
}
