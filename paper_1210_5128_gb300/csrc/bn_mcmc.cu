// bn_mcmc.cu -- Algorithm 1's iteration on the device: Metropolis-Hastings over node
// orders with the two-position swap proposal of Sec. III.C, the order score of Eq. (6),
// best-graph tracking and (after burn-in) edge counts of the current greedy DAG.
//
// The paper scores one order per iteration on the GPU and keeps the MH test, the
// best-graph update and the proposal on the CPU (Sec. V.A), crossing the bus every
// iteration.  Here every chain's state lives on the device and one step of all chains
// is three kernels, captured once as a CUDA graph and replayed:
//   k_propose  Philox draw, swap, and the work list of nodes whose predecessor sets
//              changed (the nodes between the two swapped positions; all others keep
//              their best parent sets, which is exact)
//   k_scan     the order-score scan of those (node, chain) items
//   k_accept   chunk combine, FP64 order score (ascending node id), MH test, best
//              graph, edge counts, trace/ESS records; the last block advances the step
// On a pruned table with the uniform proposal one kernel does all of it instead:
//   k_chain_fused  one warp per chain, up to 1024 steps per launch, the network's
//              survivors in shared memory; per step only the span's nodes that cannot
//              keep their parent sets are re-scored, the MH test is decided on exact
//              fixed-point changes against thresholds prepared with the Philox draws,
//              and FP64 order scores are formed only where a decision or an output needs
//              them (every decision equal to the per-step path's)
//   k_batch_fused  the same for many networks' chains in one launch
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bn_chain.cuh"

namespace bn {

// initial orders: Fisher-Yates from the identity driven by the Philox init stream
__global__ void k_init_orders(ChainState S)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S.C) return;
    uint8_t o[MAXN];
    for (int p = 0; p < S.n; ++p) o[p] = (uint8_t)p;
    U64x4 buf;
    int used = 4;
    uint64_t blk = 0;
    for (int i = S.n - 1; i >= 1; --i) {
        if (used == 4) { buf = philox4x64(blk++, (uint64_t)c, 1, 0, S.seed, 0); used = 0; }
        uint64_t x = buf.x[used++];
        int j = (int)mulhi64(x, (uint64_t)(i + 1));
        uint8_t tmp = o[i]; o[i] = o[j]; o[j] = tmp;
    }
    for (int p = 0; p < S.n; ++p) S.cur_order[(size_t)c * S.n + p] = o[p];
}

// scan result of one (node, item): the chosen rank and its entry's key
__device__ __forceinline__ void item_result(const ChainState& S, int i, uint32_t p, int64_t& bk, uint32_t& br)
{
    if ((int64_t)p >= S.Sp) p = 0;                     // only after a timed-out scan
    br = S.srank[(size_t)i * S.Sp + p];
    bk = S.keys[(size_t)i * S.Sp + br];
}

// full scoring of the initial orders (items of node i are chains 0..C-1)
__global__ void k_init_state(ChainState S)
{
    __shared__ int64_t s_key[8][MAXN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + warp;
    if (c >= S.C) return;
    for (int i = lane; i < S.n; i += 32) {
        int64_t bk;
        uint32_t br;
        item_result(S, i, S.list_best[(size_t)i * S.C + c], bk, br);
        s_key[warp][i] = bk;
        S.cur_key[(size_t)c * S.n + i] = bk;
        S.cur_rank[(size_t)c * S.n + i] = br;
        S.best_rank[(size_t)c * S.n + i] = br;
    }
    for (int p = lane; p < S.n; p += 32) S.best_order[(size_t)c * S.n + p] = S.cur_order[(size_t)c * S.n + p];
    __syncwarp();
    if (lane == 0) {
        double sum = 0.0;
        for (int i = 0; i < S.n; ++i) sum = __dadd_rn(sum, key_to_double(s_key[warp][i]));
        S.cur_score[c] = sum;
        S.best_score[c] = sum;
        S.accepts[c] = 0;
    }
}

// the swapped order and the work items of the positions a..b (their predecessor sets
// changed), one warp per chain: lane l owns positions l and l + 32, prefix masks by a
// warp OR-scan, the list appends in parallel
__device__ __forceinline__ void swap_and_list(const ChainState& S, int c, int a, int b, int lane)
{
    const int n = S.n;
    uint8_t* po = S.prop_order + (size_t)c * n;
    const uint8_t* co = S.cur_order + (size_t)c * n;
    int v[2];
    uint64_t bit[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = lane + 32 * h;
        v[h] = -1;
        bit[h] = 0;
        if (p < n) {
            v[h] = (p == a) ? co[b] : (p == b) ? co[a] : co[p];
            po[p] = (uint8_t)v[h];
            bit[h] = 1ull << v[h];
        }
    }
    // inclusive OR-scan over positions 0..31, then 32..63 on top of the first half's total
    uint64_t s0 = bit[0], s1 = bit[1];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint64_t t0 = __shfl_up_sync(0xffffffffu, s0, off);
        const uint64_t t1 = __shfl_up_sync(0xffffffffu, s1, off);
        if (lane >= off) { s0 |= t0; s1 |= t1; }
    }
    const uint64_t first_half = __shfl_sync(0xffffffffu, s0, 31);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = lane + 32 * h;
        if (p < n && p >= a && p <= b) {
            const uint64_t excl = (h == 0 ? s0 : (s1 | first_half)) & ~bit[h];   // nodes before position p
            const uint32_t slot = atomicAdd(&S.list_count[v[h]], 1u);
            S.list_pc[(size_t)v[h] * S.C + slot] = compress_pred(excl, v[h]);
            S.list_best[(size_t)v[h] * S.C + slot] = SPOS_NONE;
            S.slot_of[(size_t)c * n + v[h]] = slot;
        }
    }
    if (lane == 0) {
        S.prop_ab[2 * c] = (uint8_t)a;
        S.prop_ab[2 * c + 1] = (uint8_t)b;
    }
}

// step 1: proposal and work lists (one warp per chain)
__global__ void k_propose(ChainState S)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= S.C) return;
    const int n = S.n;
    const int64_t t = *S.step;
    const U64x4 x = philox4x64((uint64_t)t, (uint64_t)c, 0, 0, S.seed, 0);
    const uint64_t P = (uint64_t)n * (uint64_t)(n - 1) / 2;
    int a, b;
    pair_decode(n, mulhi64(x.x[0], P), a, b);
    swap_and_list(S, c, a, b, lane);
    if (lane == 0) S.prop_u[c] = __dmul_rn(__dadd_rn((double)(x.x[1] >> 12), 0.5), 0x1p-52);
}

// step 3: combine, MH test, bookkeeping; the last block advances the step counter
__global__ void k_accept(ChainState S)
{
    __shared__ int64_t s_key[8][MAXN];
    __shared__ uint32_t s_rank[8][MAXN];
    __shared__ int s_acc[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + warp;
    const int n = S.n;
    const int64_t t = *S.step;
    if (c < S.C) {
        const int a = S.prop_ab[2 * c], b = S.prop_ab[2 * c + 1];
        const uint8_t* po = S.prop_order + (size_t)c * n;
        bool moved = false;
        for (int p = lane; p < n; p += 32) {
            const int v = po[p];
            int64_t bk;
            uint32_t br;
            if (p >= a && p <= b) {
                const uint32_t slot = S.slot_of[(size_t)c * n + v];
                item_result(S, v, S.list_best[(size_t)v * S.C + slot], bk, br);
                moved |= br != S.cur_rank[(size_t)c * n + v];
            } else {
                bk = S.cur_key[(size_t)c * n + v];
                br = S.cur_rank[(size_t)c * n + v];
            }
            s_key[warp][v] = bk;
            s_rank[warp][v] = br;
        }
        moved = __any_sync(0xffffffffu, moved);
        if (S.changed && lane == 0) S.changed[c] = moved ? 1 : 0;
        __syncwarp();
        if (lane == 0) {
            double s2 = 0.0;
            for (int i = 0; i < n; ++i) s2 = __dadd_rn(s2, key_to_double(s_key[warp][i]));
            const double s1 = S.cur_score[c];
            const double delta = __dsub_rn(s2, s1);
            const double lu = log(S.prop_u[c]);
            // learned proposal: ln q(pair | proposed) - ln q(pair | current)
            const double corr = S.mode == BN_PROPOSAL_LEARNED
                                    ? (double)S.prop_lq[(size_t)c * S.P + S.prop_pair[c]] - (double)S.prop_lqf[c]
                                    : 0.0;
            const bool acc = S.literal_log ? (lu < __dadd_rn(delta, corr))
                                           : (lu < __dadd_rn(__dmul_rn(LN10, delta), corr));
            if (S.delta) S.delta[c] = (float)delta;
            s_acc[warp] = acc ? 1 : 0;
            if (acc) {
                S.cur_score[c] = s2;
                S.accepts[c] += 1;
                if (s2 > S.best_score[c]) { S.best_score[c] = s2; s_acc[warp] = 2; }
            }
            if (t < S.trace_cap) {
                S.trace_score[(size_t)c * S.trace_cap + t] = acc ? s2 : s1;
                S.trace_accept[(size_t)c * S.trace_cap + t] = acc ? 1 : 0;
            }
        }
        __syncwarp();
        const int acc = s_acc[warp];
        if (acc && S.mode == BN_PROPOSAL_LEARNED) {
            for (int j = lane; j < S.P; j += 32) S.cur_lq[(size_t)c * S.P + j] = S.prop_lq[(size_t)c * S.P + j];
        }
        if (acc) {
            for (int p = lane; p < n; p += 32) {
                S.cur_order[(size_t)c * n + p] = po[p];
                S.cur_key[(size_t)c * n + p] = s_key[warp][p];
                S.cur_rank[(size_t)c * n + p] = s_rank[warp][p];
                if (acc == 2) {
                    S.best_order[(size_t)c * n + p] = po[p];
                    S.best_rank[(size_t)c * n + p] = s_rank[warp][p];
                }
            }
        }
        if (t >= S.burn_in) {
            const bool rec = S.record_every > 0 && ((t - S.burn_in) % S.record_every) == 0 &&
                             (t - S.burn_in) / S.record_every < S.record_cap;
            const int64_t ridx = rec ? (t - S.burn_in) / S.record_every : 0;
            for (int i = lane; i < n; i += 32) {
                uint32_t r = acc ? s_rank[warp][i] : S.cur_rank[(size_t)c * n + i];
                if ((int64_t)r >= S.Sp) r = 0;          // only after a timed-out scan
                uint64_t m = S.pst[r];
                uint32_t* E = S.edge + ((size_t)c * n + i) * n;
                while (m) {
                    const int slot = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    const int par = slot + (slot >= i ? 1 : 0);
                    E[par] += 1u;
                    if (rec) {
                        S.rec_bits[(((size_t)c * n + i) * n + par) * S.rec_words + (ridx >> 6)] |= 1ull << (ridx & 63);
                    }
                }
            }
        }
    }
    // the last block to finish advances the step and clears the work lists
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t ticket = atomicAdd(S.done, 1u);
        if (ticket == gridDim.x - 1) {
            int64_t items = 0;
            for (int i = 0; i < n; ++i) {
                items += S.list_count[i];
                S.list_count[i] = 0;
            }
            *S.items_total += items;
            if (t >= S.burn_in && S.record_every > 0 && ((t - S.burn_in) % S.record_every) == 0 &&
                (t - S.burn_in) / S.record_every < S.record_cap)
                *S.rec_count = (t - S.burn_in) / S.record_every + 1;
            *S.step = t + 1;
            *S.done = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------------
// Fused steps for the pruned table and the uniform proposal: one warp per chain runs
// `iters` MH steps without leaving the kernel (chains are independent).  Per step: the
// Philox draw, the swapped span's nodes re-scored by their lanes (each walks its node's
// survivors in score order to the first consistent one), the FP64 order score summed in
// ascending node id by lane 0, the MH test, the best graph.  Edge counts are accumulated
// by dwell time: when a node's parent set changes at step t, its old set is credited
// with the post-burn-in steps it was held; everything is flushed at the end of the
// launch, so the counts equal per-step counting exactly.
// ---------------------------------------------------------------------------------
struct FusedArgs {
    const uint64_t* amask;
    const uint32_t* aspos;
    const uint32_t* aoff;
    const uint32_t* acnt;
    int64_t t0;          // first step of this launch
    int iters;
    int staged;          // 1: the network's survivors fit the warp's shared-memory cache
    int cap;             // survivors per warp cache (shared-memory layout of the launch;
                         // the table's survivor count for a global-memory cache)
    const uint8_t* gcache;   // not staged: the same cache in global memory, or null
    const uint16_t* gfirst;  // with gcache: [node][v] first survivor of the node whose set
                             // contains node v (the node's survivor count if none)
    double margin_x;     // bound on |ln10 (dpart - (s' - s))| (rounding of the two sums)
    int64_t guard_fx;    // two order scores whose exact fixed-point sums differ by more than
                         // this (2^-32 units) compare the same way as their FP64 sums
};

// shared-memory cache of a network's survivors: parent mask in node space (bit v = node v;
// the table's candidate-space masks with a 0 inserted at the child's own bit, so the span's
// predecessor masks test against it directly), the entry in 64-bit fixed point (2^-32
// units), the OR of the masks of the node's survivors before it, and rank of every
// survivor (score order), and the node offsets
__host__ __device__ constexpr size_t surv_cache_bytes(int cap)
{
    return (size_t)cap * (8 + 8 + 8 + 4) + 4 * (MAXN + 1);
}
static constexpr int SURV_CAP_MAX = 2400;
// cached networks sum entry changes in 64-bit fixed point (2^-32 units): entries below 2^22
// in magnitude keep every sum of up to 2 x 64 changes inside int64
static constexpr double FX_LIMIT = 4194304.0;

static constexpr int FUSED_WARPS = 2;      // chains per block of one network's fused launch
static constexpr int BATCH_WARPS = 8;      // chains per block of a many-network launch

struct FusedSmem {
    uint8_t ord[MAXN];
    uint32_t rank[MAXN];
    int64_t key[MAXN];
    int64_t nkey[MAXN];
    int64_t since[MAXN];
    uint64_t pre[MAXN];        // nodes at positions < p of the current order
    uint32_t cj[MAXN];         // cache index of each node's current best survivor,
    uint64_t cmask[MAXN];      //   its parent mask (node space, cached networks)
    uint64_t corb[MAXN];       //   and the OR of the masks of the node's survivors before it
    int64_t fx[MAXN];          // each node's current entry in fixed point (cached networks)
    uint8_t ra[32], rb[32];    // the next 32 steps: the swapped positions a < b,
    double ru[32];             //   the MH uniform from x1,
    int64_t tlo[32], thi[32];  //   and the fast test's thresholds (ln u -/+ its margin) in
                               //   the fixed-point units of the change, 2^-32 of a score
    uint32_t brank[MAXN];      // ranks of the best state so far
    uint32_t coff[MAXN + 1];   // cached networks: the nodes' first survivor indices (a copy
                               // of the cache's, which may sit in global memory)
    uint8_t kst[MAXN];         // 1: key[i] (and nkey[i]) not yet read for the node's rank
};

// Cached networks leave the FP64 order score of an accepted move for later when the fast
// test already decided it (the exact fixed-point sum tracks the state); these recover it.
// Keys of nodes whose parent set changed in such moves, read for their ranks:
__device__ __forceinline__ void refresh_keys(const ChainState& S, FusedSmem& W, int n, int lane)
{
    for (int i = lane; i < n; i += 32)
        if (W.kst[i]) {
            const int64_t k = S.keys[(size_t)i * S.Sp + W.rank[i]];
            W.key[i] = k;
            W.nkey[i] = k;
            W.kst[i] = 0;
        }
    __syncwarp();
}
// the FP64 order score: entries in ascending node id, summed left to right (lane 0)
__device__ __forceinline__ double seq_score(const int64_t* k, int n, int lane)
{
    double s = 0.0;
    if (lane == 0)
        for (int i = 0; i < n; ++i) s = __dadd_rn(s, key_to_double(k[i]));
    return __shfl_sync(0xffffffffu, s, 0);
}
// the same for the best state, from its ranks
__device__ __forceinline__ double best_score_of(const ChainState& S, const FusedSmem& W, int n, int lane)
{
    int64_t k0 = 0, k1 = 0;
    if (lane < n) k0 = S.keys[(size_t)lane * S.Sp + W.brank[lane]];
    if (lane + 32 < n) k1 = S.keys[(size_t)(lane + 32) * S.Sp + W.brank[lane + 32]];
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        const int64_t v = __shfl_sync(0xffffffffu, i < 32 ? k0 : k1, i & 31);
        if (lane == 0) s = __dadd_rn(s, key_to_double(v));
    }
    return __shfl_sync(0xffffffffu, s, 0);
}

// an entry (order-preserving key) in fixed point, 2^-32 units, rounded to nearest; exact
// sums of these decide most MH tests (entries below 2^22 in magnitude, see FX_LIMIT)
__device__ __forceinline__ int64_t entry_fx(int64_t key)
{
    return __double2ll_rn(key_to_double(key) * 4294967296.0);
}

// a network's survivors (mask, rank, key in score order; node offsets) into the block's
// shared-memory cache, by all `nthr` threads of the block
__device__ __forceinline__ void fill_surv_cache(const ChainState& S, const FusedArgs& F, uint8_t* cache, int tid,
                                                int nthr)
{
    const int n = S.n;
    uint64_t* c_mask = (uint64_t*)cache;
    int64_t* c_fx = (int64_t*)(cache + 8 * (size_t)F.cap);
    uint64_t* c_orb = (uint64_t*)(cache + 16 * (size_t)F.cap);
    uint32_t* c_rank = (uint32_t*)(cache + 24 * (size_t)F.cap);
    uint32_t* c_off = (uint32_t*)(cache + 28 * (size_t)F.cap);
    const uint32_t o0 = F.aoff[0];
    const uint32_t total = F.aoff[n - 1] + F.acnt[n - 1] - o0;
    for (uint32_t j = tid; j < total; j += nthr) {
        // node of survivor j: offsets are ascending
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (F.aoff[mid] - o0 <= j) lo = mid;
            else hi = mid;
        }
        const uint32_t r = S.srank[(size_t)lo * S.Sp + F.aspos[o0 + j]];
        const uint64_t cm = F.amask[o0 + j];
        const uint64_t below = lo ? (~0ull >> (64 - lo)) : 0ull;
        c_mask[j] = (cm & below) | ((cm & ~below) << 1);
        c_rank[j] = r;
        c_fx[j] = entry_fx(S.keys[(size_t)lo * S.Sp + r]);
    }
    for (int v = tid; v < n; v += nthr) c_off[v] = F.aoff[v] - o0;
    if (tid == 0) c_off[n] = total;
    __syncthreads();
    // per node, the OR of the masks of the survivors before each one
    for (int v = tid; v < n; v += nthr) {
        uint64_t acc = 0ull;
        for (uint32_t j = c_off[v]; j < c_off[v + 1]; ++j) {
            c_orb[j] = acc;
            acc |= c_mask[j];
        }
    }
}

// The survivors in the cache layout above, in global memory (one thread per survivor; the
// prefix ORs one thread per node, in a second launch)
__global__ void k_gcache_fill(const int64_t* __restrict__ keys, const uint32_t* __restrict__ srank, int64_t Sp,
                              int n, const uint64_t* __restrict__ amask, const uint32_t* __restrict__ aspos,
                              const uint32_t* __restrict__ aoff, uint32_t total, int cap, uint8_t* __restrict__ cache)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t* c_mask = (uint64_t*)cache;
    int64_t* c_fx = (int64_t*)(cache + 8 * (size_t)cap);
    uint32_t* c_rank = (uint32_t*)(cache + 24 * (size_t)cap);
    uint32_t* c_off = (uint32_t*)(cache + 28 * (size_t)cap);
    if (j < total) {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (aoff[mid] <= j) lo = mid;
            else hi = mid;
        }
        const uint32_t r = srank[(size_t)lo * Sp + aspos[j]];
        const uint64_t cm = amask[j];
        const uint64_t below = lo ? (~0ull >> (64 - lo)) : 0ull;
        c_mask[j] = (cm & below) | ((cm & ~below) << 1);
        c_rank[j] = r;
        c_fx[j] = entry_fx(keys[(size_t)lo * Sp + r]);
    }
    if (j <= (uint32_t)n) c_off[j] = j < (uint32_t)n ? aoff[j] : total;
}

__global__ void k_gcache_first(int n, int cap, const uint8_t* __restrict__ cache, uint16_t* __restrict__ first)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * 64) return;
    const int nd = idx >> 6, v = idx & 63;
    const uint64_t* c_mask = (const uint64_t*)cache;
    const uint32_t* c_off = (const uint32_t*)(cache + 28 * (size_t)cap);
    const uint32_t j0 = c_off[nd], j1 = c_off[nd + 1];
    uint32_t j = j0;
    while (j < j1 && ((c_mask[j] >> v) & 1ull) == 0ull) ++j;
    first[idx] = (uint16_t)min(j - j0, 65535u);
}

__global__ void k_gcache_orb(int n, int cap, uint8_t* __restrict__ cache)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint64_t* c_mask = (const uint64_t*)cache;
    uint64_t* c_orb = (uint64_t*)(cache + 16 * (size_t)cap);
    const uint32_t* c_off = (const uint32_t*)(cache + 28 * (size_t)cap);
    uint64_t acc = 0ull;
    for (uint32_t j = c_off[v]; j < c_off[v + 1]; ++j) {
        c_orb[j] = acc;
        acc |= c_mask[j];
    }
}

// JUMP (global-memory caches): `first` = F.gfirst, the first survivor of every node that
// contains each node, where a restarted walk with one gained predecessor begins
template <bool STAGED, bool JUMP = false>
__device__ __forceinline__ void chain_fused_body(const ChainState& S, const FusedArgs& F, int c, int lane,
                                                 FusedSmem& W, const uint8_t* cache)
{
    const int n = S.n;
    const uint64_t P = (uint64_t)n * (uint64_t)(n - 1) / 2;
    const uint64_t* c_mask = (const uint64_t*)cache;
    const int64_t* c_fx = (const int64_t*)(cache + 8 * (size_t)F.cap);
    const uint64_t* c_orb = (const uint64_t*)(cache + 16 * (size_t)F.cap);
    const uint32_t* c_rank = (const uint32_t*)(cache + 24 * (size_t)F.cap);
    const uint32_t* c_off = (const uint32_t*)(cache + 28 * (size_t)F.cap);
    if (STAGED)
        for (int i = lane; i <= n; i += 32) W.coff[i] = c_off[i];
    for (int i = lane; i < n; i += 32) {
        W.ord[i] = S.cur_order[(size_t)c * n + i];
        W.rank[i] = S.cur_rank[(size_t)c * n + i];
        W.key[i] = S.cur_key[(size_t)c * n + i];
        W.nkey[i] = W.key[i];
        W.since[i] = F.t0;
        W.brank[i] = S.best_rank[(size_t)c * n + i];
        W.kst[i] = 0;
        // the cache index of node i's current best survivor
        uint32_t cj = 0;
        if (STAGED) {
            for (cj = c_off[i]; cj + 1 < c_off[i + 1] && c_rank[cj] != W.rank[i]; ++cj) {}
            W.cmask[i] = c_mask[cj];
            W.corb[i] = c_orb[cj];
            W.fx[i] = c_fx[cj];
        }
        W.cj[i] = cj;
    }
    __syncwarp();
    {
        // prefix masks of the current order (positions lane, lane + 32): exclusive OR-scan
        uint64_t b0 = lane < n ? 1ull << W.ord[lane] : 0ull;
        uint64_t b1 = lane + 32 < n ? 1ull << W.ord[lane + 32] : 0ull;
        uint64_t s0 = b0, s1 = b1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t t0 = __shfl_up_sync(0xffffffffu, s0, off);
            const uint64_t t1 = __shfl_up_sync(0xffffffffu, s1, off);
            if (lane >= off) { s0 |= t0; s1 |= t1; }
        }
        const uint64_t first_half = __shfl_sync(0xffffffffu, s0, 31);
        if (lane < n) W.pre[lane] = s0 & ~b0;
        if (lane + 32 < n) W.pre[lane + 32] = (s1 | first_half) & ~b1;
    }
    double score = S.cur_score[c], best = S.best_score[c];
    // Cached networks: Fcur = the exact fixed-point sum of the current entries; `dirty`: score
    // not yet summed in FP64 for the current state; bestF / `bdirty` the same for the best
    // state (bestF within guard_fx / 2 of best * 2^32 either way); `stale`: some kst[i] set
    int64_t Fcur = 0, bestF = INT64_MIN / 4;
    bool dirty = false, bdirty = false, stale = false;
    if (STAGED) {
        for (int i = lane; i < n; i += 32) Fcur += W.fx[i];
#pragma unroll
        for (int off = 16; off; off >>= 1) Fcur += __shfl_xor_sync(0xffffffffu, Fcur, off);
        if (isfinite(best)) bestF = __double2ll_rn(best * 4294967296.0);
    }
    int64_t acc_count = 0, items = 0;
    // next recorded step and its index (recording: every record_every-th step from burn-in)
    int64_t rec_next = INT64_MAX, rec_idx = 0;
    if (S.record_every > 0) {
        const int64_t from = F.t0 > S.burn_in ? F.t0 : S.burn_in;
        rec_idx = (from - S.burn_in + S.record_every - 1) / S.record_every;
        rec_next = rec_idx < S.record_cap ? S.burn_in + rec_idx * S.record_every : INT64_MAX;
    }
    __syncwarp();
    for (int it = 0; it < F.iters; ++it) {
        const int64_t t = F.t0 + it;
        if ((it & 31) == 0) {
            // the next 32 steps' Philox blocks, one per lane, and what the MH test needs of
            // them: u, and ln u within the FP32 log's error plus the rounding bound of the
            // change, divided by ln 10 (the test's factor) and scaled to the change's
            // fixed-point units, one unit further out on each side than the conversion's
            // rounding needs (the fast test is decided outside [tlo, thi] by two integer
            // compares; the FP64 work runs here, once per 32 steps, in all lanes at once)
            const U64x4 xr = philox4x64((uint64_t)(t + lane), (uint64_t)c, 0, 0, S.seed, 0);
            const double u = __dmul_rn(__dadd_rn((double)(xr.x[1] >> 12), 0.5), 0x1p-52);
            const float luf = logf((float)u);
            const double mg = 1e-6 * (1.0 + fabs((double)luf)) + F.margin_x;
            const double to_fx = S.literal_log ? 4294967296.0 : 4294967296.0 / LN10;
            int pa, pb;
            pair_decode(n, __umul64hi(xr.x[0], P), pa, pb);
            W.ra[lane] = (uint8_t)pa;
            W.rb[lane] = (uint8_t)pb;
            W.ru[lane] = u;
            W.tlo[lane] = (int64_t)floor(((double)luf - mg) * to_fx) - 1;
            W.thi[lane] = (int64_t)ceil(((double)luf + mg) * to_fx) + 1;
            __syncwarp();
        }
        const int a = W.ra[it & 31], b = W.rb[it & 31];
        const int va = W.ord[a], vb = W.ord[b];
        const uint64_t bva = 1ull << va, bvb = 1ull << vb;
        // the span a..b of the proposed order: its nodes and their predecessor sets (the
        // current prefix with node va replaced by vb between a and b)
        // lane l holds span positions a + l and, for spans longer than 32, a + l + 32
        int node[2] = {-1, -1};
        uint32_t nrank[2] = {0, 0};
        uint32_t wj[2] = {0, 0}, wj1[2] = {0, 0};
        uint64_t wnpc[2] = {0, 0};
        bool act[2] = {false, false};
        bool kept[2] = {false, false};
        uint32_t cjv[2] = {0, 0};        // cached networks: the node's current survivor index
        const int halves = b - a >= 32 ? 2 : 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h >= halves) break;
            const int p = a + lane + 32 * h;
            if (p <= b) {
                const int nd = (p == a) ? vb : (p == b) ? va : W.ord[p];
                const uint64_t excl = (p == a) ? W.pre[a] : ((W.pre[p] & ~bva) | bvb);
                // cached networks test node-space masks; the table's are in candidate space
                wnpc[h] = STAGED ? ~excl : ~compress_pred(excl, nd);
                node[h] = nd;
                if (STAGED) {
                    // The node's best set so far is the first survivor consistent with its
                    // old predecessors.  A survivor before it can only become consistent by
                    // containing a gained predecessor; if none does, the answer is that set
                    // again (still consistent) or lies after it.
                    const uint64_t old_pred = (p == a) ? W.pre[b] : (p == b) ? W.pre[a] : W.pre[p];
                    const uint64_t gained = excl & ~old_pred;
                    const uint32_t cj = W.cj[nd];
                    cjv[h] = cj;
                    const bool none_before = (W.corb[nd] & gained) == 0ull;
                    const bool stays = (W.cmask[nd] & wnpc[h]) == 0ull;
                    uint32_t restart = W.coff[nd];
                    if (JUMP && !none_before && (gained & (gained - 1)) == 0ull) {   // (gained != 0 here)
                        // one gained predecessor v: survivors before the first one containing
                        // v stay inconsistent (they were before the first consistent one)
                        restart += F.gfirst[nd * 64 + (__ffsll((long long)gained) - 1)];
                    }
                    wj[h] = none_before ? (stays ? cj : cj + 1) : restart;
                    wj1[h] = W.coff[nd + 1];
                    kept[h] = none_before && stays;
                    act[h] = !kept[h];
                } else {
                    wj[h] = F.aoff[nd];
                    wj1[h] = F.aoff[nd] + F.acnt[nd];
                    act[h] = true;
                }
            }
        }
        // survivors of each node in score order: the first consistent one wins
        span_walk(STAGED ? c_mask : F.amask, wj, wj1, wnpc, act, lane, STAGED ? 64 : 8);
        bool moved = false;
        int64_t nfx[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (!act[h] && !kept[h]) continue;
            const int nd = node[h];
            if (STAGED) {
                // the new key is fetched only if the exact test needs it; survivor indices
                // are unique per node, so the set changed iff the index did
                nrank[h] = c_rank[wj[h]];
                nfx[h] = c_fx[wj[h]];
                moved |= wj[h] != cjv[h];
            } else {
                nrank[h] = S.srank[(size_t)nd * S.Sp + F.aspos[wj[h]]];
                W.nkey[nd] = S.keys[(size_t)nd * S.Sp + nrank[h]];
                moved |= nrank[h] != W.rank[nd];
            }
        }
        moved = __any_sync(0xffffffffu, moved);
        items += b - a + 1;
        int acc = 1;
        double s2 = score;
        bool lazy = false;
        int exact = 0;
        long long dfx = 0;
        if (moved) {
            __syncwarp();
            // MH test.  The exact test compares ln u with ln10 (s' - s), s' the FP64 sum over
            // nodes in ascending id.  Most steps are decided without it: the change of the
            // re-scored nodes alone (exact in fixed point for cached networks, within n 2^-32
            // of the true change; an FP64 sum in any order otherwise) is within the margin of
            // s' - s, and an FP32 log(u) within 1e-6 (1 + |ln u|) of ln u; when the two sides
            // are farther apart than both errors the decision is the exact one.  Close calls
            // and accepted moves (whose new score the state keeps) take the exact path, which
            // fetches the span's new FP64 entries.
            acc = 0;
            if (STAGED) {
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (node[h] >= 0) dfx += nfx[h] - W.fx[node[h]];
                // warp sum in three 21-bit limbs (|lane value| < 2^56, so no limb sum
                // overflows 32 bits), one reduction instruction each
                {
                    const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(dfx & 0x1fffff));
                    const unsigned mid = __reduce_add_sync(0xffffffffu, (unsigned)((dfx >> 21) & 0x1fffff));
                    const int hi = __reduce_add_sync(0xffffffffu, (int)(dfx >> 42));
                    dfx = (long long)hi * (1ll << 42) + (long long)mid * (1ll << 21) + (long long)lo;
                }
                {
                    const int q = it & 31;
                    exact = dfx < W.tlo[q] ? 0 : (dfx > W.thi[q] ? 1 : 2);     // equal in every lane
                }
                // a move the fast test accepts needs no FP64 score now, unless per-step
                // scores are traced
                lazy = exact == 1 && t >= S.trace_cap;
                if (exact && !lazy) {
                    if (stale) {
                        refresh_keys(S, W, n, lane);
                        stale = false;
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (node[h] >= 0) W.nkey[node[h]] = S.keys[(size_t)node[h] * S.Sp + nrank[h]];
                    __syncwarp();
                }
            } else {
                double dpart = 0.0;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (node[h] >= 0) dpart += key_to_double(W.nkey[node[h]]) - key_to_double(W.key[node[h]]);
#pragma unroll
                for (int off = 16; off; off >>= 1) dpart += __shfl_down_sync(0xffffffffu, dpart, off);
                if (lane == 0) {
                    const double xa = S.literal_log ? dpart : LN10 * dpart;
                    const int q = it & 31;
                    // the thresholds back in ln units (a little further out than ln u -/+ the
                    // margin, so still sound for this FP64 change)
                    const double back = S.literal_log ? 0x1p-32 : LN10 * 0x1p-32;
                    exact = xa < (double)W.tlo[q] * back ? 0 : (xa > (double)W.thi[q] * back ? 1 : 2);
                }
                exact = __shfl_sync(0xffffffffu, exact, 0);
            }
            if (exact && !lazy) {
                if (dirty) {
                    score = seq_score(W.key, n, lane);
                    dirty = false;
                }
                if (lane == 0) {
                    // the proposal's keys: nkey holds the span's new keys and everyone else's
                    s2 = 0.0;
                    for (int i = 0; i < n; ++i) s2 = __dadd_rn(s2, key_to_double(W.nkey[i]));
                    if (exact == 2) {
                        const double delta = __dsub_rn(s2, score);
                        const double lu = log(W.ru[it & 31]);
                        acc = S.literal_log ? (lu < delta) : (lu < __dmul_rn(LN10, delta));
                    } else {
                        acc = 1;
                    }
                }
                acc = __shfl_sync(0xffffffffu, acc, 0);
                s2 = __shfl_sync(0xffffffffu, s2, 0);
            } else if (lazy) {
                acc = 1;
            }
        }
        // (not moved: no parent set changes, s' = s bit for bit and ln u < 0 accepts)
        if (!acc && (!STAGED || exact)) {
            // the rejected proposal's keys: nkey equals key again outside any span (cached
            // networks change nkey only on the exact path)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (node[h] >= 0) W.nkey[node[h]] = W.key[node[h]];
        }
        if (acc) {
            if (moved) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int nd = node[h];
                    if (nd >= 0 && nrank[h] != W.rank[nd]) {
                        credit_edges(S, c, nd, W.rank[nd], W.since[nd], t);
                        W.since[nd] = t;
                        W.rank[nd] = nrank[h];
                        if (lazy) W.kst[nd] = 1;
                        else W.key[nd] = W.nkey[nd];
                        W.cj[nd] = wj[h];
                        if (STAGED) {
                            W.cmask[nd] = c_mask[wj[h]];
                            W.corb[nd] = c_orb[wj[h]];
                            W.fx[nd] = nfx[h];
                        }
                    }
                }
            }
            // prefixes of positions a+1..b now hold vb instead of va (lane l: a + 1 + l and,
            // for b - a > 32, a + 33 + l)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && b - a <= 32) break;
                const int p = a + 1 + lane + 32 * h;
                if (p <= b) W.pre[p] = (W.pre[p] & ~bva) | bvb;
            }
            if (lane == 0) {
                W.ord[a] = (uint8_t)vb;
                W.ord[b] = (uint8_t)va;
            }
            __syncwarp();
            ++acc_count;
            bool newbest;
            if (!STAGED) {
                score = s2;
                newbest = s2 > best;
            } else if (!moved) {
                newbest = false;                        // s' = s <= best
            } else {
                Fcur += dfx;
                if (lazy) {
                    dirty = true;
                    stale = true;
                } else {
                    score = s2;
                }
                const int64_t d = Fcur - bestF;
                if (!dirty && !bdirty) {
                    newbest = score > best;
                } else if (d > F.guard_fx) {
                    newbest = true;
                } else if (d < -F.guard_fx) {
                    newbest = false;
                } else if (__all_sync(0xffffffffu, (lane >= n || W.rank[lane] == W.brank[lane]) &&
                                                       (lane + 32 >= n || W.rank[lane + 32] == W.brank[lane + 32]))) {
                    newbest = false;                    // the best state's parent sets: equal scores
                } else {
                    // too close to call in fixed point: both FP64 sums
                    if (stale) {
                        refresh_keys(S, W, n, lane);
                        stale = false;
                    }
                    if (dirty) {
                        score = seq_score(W.key, n, lane);
                        dirty = false;
                    }
                    if (bdirty) {
                        best = best_score_of(S, W, n, lane);
                        bdirty = false;
                    }
                    newbest = score > best;
                }
            }
            if (newbest) {
                best = score;                           // (the FP64 value when !dirty)
                bdirty = dirty;
                bestF = Fcur;
                for (int i = lane; i < n; i += 32) {
                    S.best_order[(size_t)c * n + i] = W.ord[i];
                    S.best_rank[(size_t)c * n + i] = W.rank[i];
                    W.brank[i] = W.rank[i];
                }
            }
        }
        if (lane == 0 && t < S.trace_cap) {
            S.trace_score[(size_t)c * S.trace_cap + t] = score;
            S.trace_accept[(size_t)c * S.trace_cap + t] = (uint8_t)acc;
        }
        if (t == rec_next) {
            const int64_t ridx = rec_idx;
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
            ++rec_idx;
            rec_next = rec_idx < S.record_cap ? rec_next + S.record_every : INT64_MAX;
        }
        __syncwarp();
    }
    const int64_t t_end = F.t0 + F.iters;
    __syncwarp();
    if (stale) refresh_keys(S, W, n, lane);
    if (dirty) score = seq_score(W.key, n, lane);
    if (bdirty) best = best_score_of(S, W, n, lane);
    for (int i = lane; i < n; i += 32) {
        credit_edges(S, c, i, W.rank[i], W.since[i], t_end);
        S.cur_order[(size_t)c * n + i] = W.ord[i];
        S.cur_rank[(size_t)c * n + i] = W.rank[i];
        S.cur_key[(size_t)c * n + i] = W.key[i];
    }
    if (lane == 0) {
        S.cur_score[c] = score;
        S.best_score[c] = best;
        S.accepts[c] += acc_count;
        atomicAdd((unsigned long long*)S.items_total, (unsigned long long)items);
    }
}

__host__ __device__ constexpr size_t surv_cache_stride(int cap) { return (surv_cache_bytes(cap) + 15) / 16 * 16; }

// MODE 1: the network's survivors in the block's shared-memory cache (F.staged); 2: the
// same layout in global memory (F.gcache); 0: the table's survivor arrays
template <int MODE>
__global__ void __launch_bounds__(32 * FUSED_WARPS) k_chain_fused(ChainState S, FusedArgs F)
{
    __shared__ FusedSmem sm[FUSED_WARPS];
    extern __shared__ __align__(16) uint8_t fcache[];     // one survivor cache per block
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * FUSED_WARPS + warp;
    if (MODE == 1) {
        fill_surv_cache(S, F, fcache, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    if (c >= S.C) return;
    chain_fused_body<MODE != 0, MODE == 2>(S, F, c, lane, sm[warp], MODE == 2 ? F.gcache : fcache);
}

// many networks' chains in one launch: block g belongs to the network i with
// cta_base[i] <= g < cta_base[i + 1]; its warps run chains (g - cta_base[i]) * BATCH_WARPS + warp
// of that network, all sharing the block's copy of the network's survivors
__global__ void __launch_bounds__(32 * BATCH_WARPS) k_batch_fused(const ChainState* __restrict__ Ss,
                                                                 const FusedArgs* __restrict__ Fs,
                                                                 const int64_t* __restrict__ cta_base, int nnet)
{
    __shared__ FusedSmem sm[BATCH_WARPS];
    extern __shared__ __align__(16) uint8_t fcache[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = blockIdx.x;
    if (g >= cta_base[nnet]) return;                                  // block-uniform
    int lo = 0, hi = nnet;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cta_base[mid] <= g) lo = mid;
        else hi = mid;
    }
    const ChainState S = Ss[lo];
    const FusedArgs F = Fs[lo];
    if (F.staged) {
        fill_surv_cache(S, F, fcache, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    const int64_t c = (g - cta_base[lo]) * BATCH_WARPS + warp;
    if (c >= S.C) return;
    if (F.staged) chain_fused_body<true>(S, F, (int)c, lane, sm[warp], fcache);
    else if (F.gcache) chain_fused_body<true, true>(S, F, (int)c, lane, sm[warp], F.gcache);
    else chain_fused_body<false>(S, F, (int)c, lane, sm[warp], fcache);
}

// ---------------------------------------------------------------------------------
// Speculative fused steps (cached networks, uniform proposal): SPEC_WARPS warps per chain.
// Step t's proposal and uniform are Philox draws keyed by (t, chain), independent of the
// state, so warp j evaluates step t + j -- the span walk, the exact fixed-point change and
// the fast MH decision -- against the current state at the same time as the others, as if
// steps t .. t + j - 1 were all rejected (a rejection leaves the state as it was).  The
// first step that is not rejected ends the round: its warp applies it (a close call first
// takes the exact FP64 test, on the state it applies to, and may turn out a rejection), the
// evaluations after it are dropped, and the rejected steps before it only leave their
// records.  Every decision, state and output is the one-warp kernel's (and the per-step
// path's); with acceptance rate r a round commits 1 + (1 - r) + ... + (1 - r)^(W - 1)
// steps for about the latency of one.
// ---------------------------------------------------------------------------------
static constexpr int SPEC_WARPS = 4;       // warps per chain
static constexpr int SPEC_BATCH = 64;      // Philox draws prepared at a time
static constexpr int SPEC_PROBE = 8;      // survivors each lane tests of its own walks first

struct SpecBatch {                         // steps base .. base + SPEC_BATCH - 1
    uint8_t ra[SPEC_BATCH], rb[SPEC_BATCH];
    double ru[SPEC_BATCH];
    int64_t tlo[SPEC_BATCH], thi[SPEC_BATCH];
};

struct SpecTasks {                         // a round's re-scoring walks, shared by the warps
    uint32_t js[SPEC_WARPS][MAXN], je[SPEC_WARPS][MAXN], hit[SPEC_WARPS][MAXN];
    uint64_t np[SPEC_WARPS][MAXN];
    int cnt[SPEC_WARPS];
};

struct SpecChain {                         // the chain's running values (any warp commits)
    double score, best;
    long long Fcur, bestF, acc_count;
    int dirty, bdirty, stale;
    int dec[SPEC_WARPS];                   // 0 rejected, 1 accepted, 2 close call
    int prog;
};

// step t's records: the traced score and accept flag, and the recorded state's edges
__device__ __forceinline__ void spec_records(const ChainState& S, const FusedSmem& W, int c, int n, int64_t t,
                                             double score, int acc, int lane)
{
    if (lane == 0 && t < S.trace_cap) {
        S.trace_score[(size_t)c * S.trace_cap + t] = score;
        S.trace_accept[(size_t)c * S.trace_cap + t] = (uint8_t)acc;
    }
    if (S.record_every > 0 && t >= S.burn_in && (t - S.burn_in) % S.record_every == 0) {
        const int64_t ridx = (t - S.burn_in) / S.record_every;
        if (ridx < S.record_cap)
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
}

// credit_edges for a parent set given in node space (bit u: parent u), as the survivor
// cache holds it -- no read of the parent-set table
__device__ __forceinline__ void credit_edges_nodes(const ChainState& S, int c, int v, uint64_t m, int64_t from,
                                                   int64_t to)
{
    const int64_t lo = max(from, S.burn_in);
    if (to <= lo) return;
    const uint32_t d = (uint32_t)(to - lo);
    uint32_t* E = S.edge + ((size_t)c * S.n + v) * S.n;
    while (m) {
        const int u = __ffsll((long long)m) - 1;
        m &= m - 1;
        atomicAdd(&E[u], d);
    }
}

template <bool JUMP>
__device__ __forceinline__ void chain_spec_body(const ChainState& S, const FusedArgs& F, int c, int warp, int lane,
                                                FusedSmem& W, SpecBatch& PB, SpecChain& K, SpecTasks& TK,
                                                const uint8_t* cache)
{
    const int n = S.n;
    const uint64_t P = (uint64_t)n * (uint64_t)(n - 1) / 2;
    const uint64_t* c_mask = (const uint64_t*)cache;
    const int64_t* c_fx = (const int64_t*)(cache + 8 * (size_t)F.cap);
    const uint64_t* c_orb = (const uint64_t*)(cache + 16 * (size_t)F.cap);
    const uint32_t* c_rank = (const uint32_t*)(cache + 24 * (size_t)F.cap);
    const uint32_t* c_off = (const uint32_t*)(cache + 28 * (size_t)F.cap);
    if (warp == 0) {
        for (int i = lane; i <= n; i += 32) W.coff[i] = c_off[i];
        for (int i = lane; i < n; i += 32) {
            W.ord[i] = S.cur_order[(size_t)c * n + i];
            W.rank[i] = S.cur_rank[(size_t)c * n + i];
            W.key[i] = S.cur_key[(size_t)c * n + i];
            W.nkey[i] = W.key[i];
            W.since[i] = F.t0;
            W.brank[i] = S.best_rank[(size_t)c * n + i];
            W.kst[i] = 0;
            uint32_t cj;
            for (cj = c_off[i]; cj + 1 < c_off[i + 1] && c_rank[cj] != W.rank[i]; ++cj) {}
            W.cmask[i] = c_mask[cj];
            W.corb[i] = c_orb[cj];
            W.fx[i] = c_fx[cj];
            W.cj[i] = cj;
        }
        __syncwarp();
        uint64_t b0 = lane < n ? 1ull << W.ord[lane] : 0ull;
        uint64_t b1 = lane + 32 < n ? 1ull << W.ord[lane + 32] : 0ull;
        uint64_t s0 = b0, s1 = b1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint64_t t0 = __shfl_up_sync(0xffffffffu, s0, off);
            const uint64_t t1 = __shfl_up_sync(0xffffffffu, s1, off);
            if (lane >= off) { s0 |= t0; s1 |= t1; }
        }
        const uint64_t first_half = __shfl_sync(0xffffffffu, s0, 31);
        if (lane < n) W.pre[lane] = s0 & ~b0;
        if (lane + 32 < n) W.pre[lane + 32] = (s1 | first_half) & ~b1;
        long long Fcur = 0;
        for (int i = lane; i < n; i += 32) Fcur += W.fx[i];
#pragma unroll
        for (int off = 16; off; off >>= 1) Fcur += __shfl_xor_sync(0xffffffffu, Fcur, off);
        if (lane == 0) {
            K.score = S.cur_score[c];
            K.best = S.best_score[c];
            K.Fcur = Fcur;
            K.bestF = isfinite(K.best) ? __double2ll_rn(K.best * 4294967296.0) : INT64_MIN / 4;
            K.acc_count = 0;
            K.dirty = K.bdirty = K.stale = 0;
        }
    }
    __syncthreads();
    const int64_t t_end = F.t0 + F.iters;
    int64_t pbase = INT64_MIN / 2;         // step of PB's entry 0 (the same in every thread)
    long long items = 0;                   // this warp's committed span lengths
    for (int64_t t = F.t0; t < t_end;) {
        if (t + SPEC_WARPS > pbase + SPEC_BATCH) {
            // the next SPEC_BATCH steps' Philox blocks and what the MH test needs of them
            // (u, and the fast test's fixed-point thresholds; see the one-warp kernel)
            pbase = t;
            for (int q = warp * 32 + lane; q < SPEC_BATCH; q += 32 * SPEC_WARPS) {
                const U64x4 xr = philox4x64((uint64_t)(t + q), (uint64_t)c, 0, 0, S.seed, 0);
                const double u = __dmul_rn(__dadd_rn((double)(xr.x[1] >> 12), 0.5), 0x1p-52);
                const float luf = logf((float)u);
                const double mg = 1e-6 * (1.0 + fabs((double)luf)) + F.margin_x;
                const double to_fx = S.literal_log ? 4294967296.0 : 4294967296.0 / LN10;
                int pa, pb;
                pair_decode(n, __umul64hi(xr.x[0], P), pa, pb);
                PB.ra[q] = (uint8_t)pa;
                PB.rb[q] = (uint8_t)pb;
                PB.ru[q] = u;
                PB.tlo[q] = (int64_t)floor(((double)luf - mg) * to_fx) - 1;
                PB.thi[q] = (int64_t)ceil(((double)luf + mg) * to_fx) + 1;
            }
            __syncthreads();
        }
        const int nact = (int)min((int64_t)SPEC_WARPS, t_end - t);
        // ---- evaluation of step t + warp against the current state --------------------
        const int64_t tj = t + warp;
        const int q = (int)(tj - pbase);
        int a = 0, b = 0, va = 0, vb = 0;
        int node[2] = {-1, -1};
        uint32_t nrank[2] = {0, 0}, wj[2] = {0, 0};
        int64_t nfx[2] = {0, 0};
        bool moved = false;
        long long dfx = 0;
        int exact = 1;
        uint32_t wj1[2] = {0, 0}, cjv[2] = {0, 0};
        uint64_t wnpc[2] = {0, 0};
        bool act[2] = {false, false};
        if (warp < nact) {
            a = PB.ra[q];
            b = PB.rb[q];
            va = W.ord[a];
            vb = W.ord[b];
            const uint64_t bva = 1ull << va, bvb = 1ull << vb;
            const int halves = b - a >= 32 ? 2 : 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h >= halves) break;
                const int p = a + lane + 32 * h;
                if (p <= b) {
                    const int nd = (p == a) ? vb : (p == b) ? va : W.ord[p];
                    const uint64_t excl = (p == a) ? W.pre[a] : ((W.pre[p] & ~bva) | bvb);
                    wnpc[h] = ~excl;
                    node[h] = nd;
                    const uint64_t old_pred = (p == a) ? W.pre[b] : (p == b) ? W.pre[a] : W.pre[p];
                    const uint64_t gained = excl & ~old_pred;
                    const uint32_t cj = W.cj[nd];
                    cjv[h] = cj;
                    const bool none_before = (W.corb[nd] & gained) == 0ull;
                    const bool stays = (W.cmask[nd] & wnpc[h]) == 0ull;
                    uint32_t restart = W.coff[nd];
                    if (JUMP && !none_before && (gained & (gained - 1)) == 0ull)
                        restart += F.gfirst[nd * 64 + (__ffsll((long long)gained) - 1)];
                    wj[h] = none_before ? (stays ? cj : cj + 1) : restart;
                    wj1[h] = W.coff[nd + 1];
                    act[h] = !(none_before && stays);
                }
            }
            // each lane first tests the first SPEC_PROBE survivors of its own walks, all loads
            // independent: a walk whose answer lies there is done without the warp-wide
            // walk (the same answer: the first consistent survivor in index order); the
            // others go on from the first survivor not probed
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!act[h]) continue;
                uint64_t pm[SPEC_PROBE];
#pragma unroll
                for (int r = 0; r < SPEC_PROBE; ++r) pm[r] = wj[h] + r < wj1[h] ? c_mask[wj[h] + r] : ~0ull;
                int first = SPEC_PROBE;
#pragma unroll
                for (int r = SPEC_PROBE - 1; r >= 0; --r)
                    if ((pm[r] & wnpc[h]) == 0ull) first = r;
                if (first < SPEC_PROBE) {
                    wj[h] += first;
                    act[h] = false;
                } else {
                    wj[h] += SPEC_PROBE;
                }
            }
        }
        // the round's remaining re-scoring walks are shared by the four warps, so a step with
        // many of them does not hold the round back: each warp posts its own, all walk them
        // in turn, each takes its answers
        int ti[2] = {0, 0};
        {
            const unsigned m0 = __ballot_sync(0xffffffffu, act[0]), m1 = __ballot_sync(0xffffffffu, act[1]);
            const unsigned lt = (1u << lane) - 1u;
            ti[0] = __popc(m0 & lt);
            ti[1] = __popc(m0) + __popc(m1 & lt);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (act[h]) {
                    TK.js[warp][ti[h]] = wj[h];
                    TK.je[warp][ti[h]] = wj1[h];
                    TK.np[warp][ti[h]] = wnpc[h];
                }
            if (lane == 0) TK.cnt[warp] = __popc(m0) + __popc(m1);
        }
        __syncthreads();
        {
            int base[SPEC_WARPS + 1];
            base[0] = 0;
#pragma unroll
            for (int w = 0; w < SPEC_WARPS; ++w) base[w + 1] = base[w] + TK.cnt[w];
            for (int g = warp; g < base[SPEC_WARPS]; g += SPEC_WARPS) {
                int w = 0, i = g;
#pragma unroll
                for (int x = 1; x < SPEC_WARPS; ++x)
                    if (g >= base[x]) {
                        w = x;
                        i = g - base[x];
                    }
                const uint32_t hit = warp_walk(c_mask, TK.js[w][i], TK.je[w][i], TK.np[w][i], lane);
                if (lane == 0) TK.hit[w][i] = hit;
            }
        }
        __syncthreads();
        if (warp < nact) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (act[h]) wj[h] = TK.hit[warp][ti[h]];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (node[h] < 0) continue;
                nrank[h] = c_rank[wj[h]];
                nfx[h] = c_fx[wj[h]];
                moved |= wj[h] != cjv[h];
                dfx += nfx[h] - W.fx[node[h]];
            }
            moved = __any_sync(0xffffffffu, moved);
            if (moved) {
                const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(dfx & 0x1fffff));
                const unsigned mid = __reduce_add_sync(0xffffffffu, (unsigned)((dfx >> 21) & 0x1fffff));
                const int hi = __reduce_add_sync(0xffffffffu, (int)(dfx >> 42));
                dfx = (long long)hi * (1ll << 42) + (long long)mid * (1ll << 21) + (long long)lo;
                exact = dfx < PB.tlo[q] ? 0 : (dfx > PB.thi[q] ? 1 : 2);
            }
            if (lane == 0) K.dec[warp] = exact;
        }
        __syncthreads();
        // ---- the first step not rejected ends the round --------------------------------
        int f = 0;
        while (f < nact && K.dec[f] == 0) ++f;
        // close calls: the exact FP64 test by that step's warp, on the current state
        while (f < nact && K.dec[f] == 2) {
            if (warp == f) {
                if (K.stale) {
                    refresh_keys(S, W, n, lane);
                    if (lane == 0) K.stale = 0;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (node[h] >= 0) W.nkey[node[h]] = S.keys[(size_t)node[h] * S.Sp + nrank[h]];
                __syncwarp();
                double score = K.score;
                if (K.dirty) score = seq_score(W.key, n, lane);
                int acc = 0;
                double s2 = 0.0;
                if (lane == 0) {
                    for (int i = 0; i < n; ++i) s2 = __dadd_rn(s2, key_to_double(W.nkey[i]));
                    const double delta = __dsub_rn(s2, score);
                    const double lu = log(PB.ru[q]);
                    acc = S.literal_log ? (lu < delta) : (lu < __dmul_rn(LN10, delta));
                    K.score = score;
                    K.dirty = 0;
                    K.dec[f] = acc ? 3 : 0;             // 3: accepted, s' in W.nkey
                }
                acc = __shfl_sync(0xffffffffu, acc, 0);
                if (!acc) {
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (node[h] >= 0) W.nkey[node[h]] = W.key[node[h]];
                }
            }
            __syncthreads();
            while (f < nact && K.dec[f] == 0) ++f;
        }
        const int prog = f < nact ? f + 1 : nact;
        // ---- records and the accepted step --------------------------------------------
        if (f < nact) {
            if (warp == f) {
                // the rejected steps before it, in order, on the state they saw
                for (int j = 0; j < f; ++j) {
                    spec_records(S, W, c, n, t + j, K.score, 0, lane);
                    items += PB.rb[q - f + j] - PB.ra[q - f + j] + 1;
                }
                items += b - a + 1;
                const uint64_t bva = 1ull << va, bvb = 1ull << vb;
                double score = K.score, best = K.best;
                long long Fcur = K.Fcur, bestF = K.bestF;
                bool dirty = K.dirty, bdirty = K.bdirty, stale = K.stale;
                const int d = K.dec[f];
                bool lazy = false;
                double s2 = score;
                if (moved) {
                    lazy = d == 1 && tj >= S.trace_cap;
                    if (d == 1 && !lazy) {
                        // an accepted traced step: its FP64 score s'
                        if (stale) {
                            refresh_keys(S, W, n, lane);
                            stale = false;
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            if (node[h] >= 0) W.nkey[node[h]] = S.keys[(size_t)node[h] * S.Sp + nrank[h]];
                        __syncwarp();
                    }
                    if (!lazy) {
                        if (dirty) {
                            score = seq_score(W.key, n, lane);
                            dirty = false;
                        }
                        if (lane == 0) {
                            s2 = 0.0;
                            for (int i = 0; i < n; ++i) s2 = __dadd_rn(s2, key_to_double(W.nkey[i]));
                        }
                        s2 = __shfl_sync(0xffffffffu, s2, 0);
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int nd = node[h];
                        if (nd >= 0 && nrank[h] != W.rank[nd]) {
                            credit_edges_nodes(S, c, nd, W.cmask[nd], W.since[nd], tj);
                            W.since[nd] = tj;
                            W.rank[nd] = nrank[h];
                            if (lazy) W.kst[nd] = 1;
                            else W.key[nd] = W.nkey[nd];
                            W.cj[nd] = wj[h];
                            W.cmask[nd] = c_mask[wj[h]];
                            W.corb[nd] = c_orb[wj[h]];
                            W.fx[nd] = nfx[h];
                        }
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h == 1 && b - a <= 32) break;
                    const int p = a + 1 + lane + 32 * h;
                    if (p <= b) W.pre[p] = (W.pre[p] & ~bva) | bvb;
                }
                __syncwarp();
                if (lane == 0) {
                    W.ord[a] = (uint8_t)vb;
                    W.ord[b] = (uint8_t)va;
                }
                __syncwarp();
                bool newbest;
                if (!moved) {
                    newbest = false;                        // s' = s <= best
                } else {
                    Fcur += dfx;
                    if (lazy) {
                        dirty = true;
                        stale = true;
                    } else {
                        score = s2;
                    }
                    const long long dd = Fcur - bestF;
                    if (!dirty && !bdirty) {
                        newbest = score > best;
                    } else if (dd > F.guard_fx) {
                        newbest = true;
                    } else if (dd < -F.guard_fx) {
                        newbest = false;
                    } else if (__all_sync(0xffffffffu, (lane >= n || W.rank[lane] == W.brank[lane]) &&
                                                           (lane + 32 >= n || W.rank[lane + 32] == W.brank[lane + 32]))) {
                        newbest = false;
                    } else {
                        if (stale) {
                            refresh_keys(S, W, n, lane);
                            stale = false;
                        }
                        if (dirty) {
                            score = seq_score(W.key, n, lane);
                            dirty = false;
                        }
                        if (bdirty) {
                            best = best_score_of(S, W, n, lane);
                            bdirty = false;
                        }
                        newbest = score > best;
                    }
                }
                if (newbest) {
                    best = score;
                    bdirty = dirty;
                    bestF = Fcur;
                    for (int i = lane; i < n; i += 32) {
                        S.best_order[(size_t)c * n + i] = W.ord[i];
                        S.best_rank[(size_t)c * n + i] = W.rank[i];
                        W.brank[i] = W.rank[i];
                    }
                }
                spec_records(S, W, c, n, tj, score, 1, lane);
                if (lane == 0) {
                    K.score = score;
                    K.best = best;
                    K.Fcur = Fcur;
                    K.bestF = bestF;
                    K.dirty = dirty;
                    K.bdirty = bdirty;
                    K.stale = stale;
                    K.acc_count += 1;
                }
            }
        } else if (warp < nact) {
            // every step rejected: each warp its own records (the state is unchanged)
            spec_records(S, W, c, n, tj, K.score, 0, lane);
            items += b - a + 1;
        }
        __syncthreads();
        t += prog;
    }
    if (lane == 0) atomicAdd((unsigned long long*)S.items_total, (unsigned long long)items);
    if (warp == 0) {
        __syncwarp();
        double score = K.score, best = K.best;
        if (K.stale) refresh_keys(S, W, n, lane);
        if (K.dirty) score = seq_score(W.key, n, lane);
        if (K.bdirty) best = best_score_of(S, W, n, lane);
        for (int i = lane; i < n; i += 32) {
            credit_edges(S, c, i, W.rank[i], W.since[i], t_end);
            S.cur_order[(size_t)c * n + i] = W.ord[i];
            S.cur_rank[(size_t)c * n + i] = W.rank[i];
            S.cur_key[(size_t)c * n + i] = W.key[i];
        }
        if (lane == 0) {
            S.cur_score[c] = score;
            S.best_score[c] = best;
            S.accepts[c] += K.acc_count;
        }
    }
}

// MODE 1: the network's survivors in the block's shared-memory cache; 2: the same layout
// in global memory.  One chain per block.
template <int MODE>
__global__ void __launch_bounds__(32 * SPEC_WARPS, 1) k_chain_spec(ChainState S, FusedArgs F)
{
    __shared__ FusedSmem W;
    __shared__ SpecBatch PB;
    __shared__ SpecChain K;
    __shared__ SpecTasks TK;
    extern __shared__ __align__(16) uint8_t fcache[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x;
    if (MODE == 1) {
        fill_surv_cache(S, F, fcache, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    if (c >= S.C) return;                                  // block-uniform
    chain_spec_body<MODE == 2>(S, F, c, warp, lane, W, PB, K, TK, MODE == 2 ? F.gcache : fcache);
}

int build_survivor_cache(bn_table* t, cudaStream_t s)
{
    // every pruned table whose entries fit the fixed point gets one (28 B per survivor):
    // a many-network launch may keep fewer survivors in shared memory than one network does
    if (t->gcache || !t->amask || t->alive_total < 1 || !(t->max_abs_survivor < FX_LIMIT)) return BN_OK;
    const int cap = (int)t->alive_total;
    uint8_t* g = nullptr;
    // the cache, then the [n][64] first-survivor table (16-bit offsets within a node)
    cudaError_t e = cudaMalloc((void**)&g, surv_cache_stride(cap) + sizeof(uint16_t) * 64 * MAXN);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BN_OK;                       // no cache: the uncached walk still works
    }
    const uint32_t total = (uint32_t)cap;
    const unsigned blocks = (unsigned)((std::max<uint32_t>(total, (uint32_t)t->n + 1) + 255) / 256);
    k_gcache_fill<<<blocks, 256, 0, s>>>(t->keys, t->srank, t->Sp, t->n, t->amask, t->aspos, t->aoff, total, cap, g);
    BN_LAUNCH_CHECK("k_gcache_fill");
    k_gcache_orb<<<(t->n + 63) / 64, 64, 0, s>>>(t->n, cap, g);
    BN_LAUNCH_CHECK("k_gcache_orb");
    k_gcache_first<<<(t->n * 64 + 255) / 256, 256, 0, s>>>(t->n, cap, g, (uint16_t*)(g + surv_cache_stride(cap)));
    BN_LAUNCH_CHECK("k_gcache_first");
    t->gcache = g;
    return BN_OK;
}

static int fused_smem_setup(int cap, size_t* smem)
{
    static unsigned long long ctx[64] = {0};
    const size_t mx = surv_cache_stride(SURV_CAP_MAX);
    if (first_in_context(ctx)) {
        BN_CUDA(cudaFuncSetAttribute(k_chain_fused<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
        BN_CUDA(cudaFuncSetAttribute(k_chain_spec<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
        BN_CUDA(cudaFuncSetAttribute(k_batch_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
    }
    *smem = surv_cache_stride(cap);
    return BN_OK;
}

__global__ void k_batch_advance(const ChainState* __restrict__ Ss, const int* __restrict__ iters, int nnet)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnet || iters[i] == 0) return;
    const ChainState& S = Ss[i];
    const int64_t t_end = *S.step + iters[i];
    *S.step = t_end;
    if (S.record_every > 0 && t_end > S.burn_in) {
        const int64_t r = (t_end - 1 - S.burn_in) / S.record_every + 1;
        *S.rec_count = r < S.record_cap ? r : S.record_cap;
    }
}

// after a fused launch: the step counter and the number of recorded states
__global__ void k_step_advance(ChainState S, int64_t iters)
{
    const int64_t t_end = *S.step + iters;
    *S.step = t_end;
    if (S.record_every > 0 && t_end > S.burn_in) {
        const int64_t r = (t_end - 1 - S.burn_in) / S.record_every + 1;
        *S.rec_count = r < S.record_cap ? r : S.record_cap;
    }
}

// learned proposal, step 1: draw the pair from the cached q(. | current order) by inverse
// CDF (one warp per chain), then the same swap and work lists as k_propose
__global__ void k_propose_learned(ChainState S)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= S.C) return;
    const int n = S.n, P = S.P;
    const int64_t t = *S.step;
    const U64x4 x = philox4x64((uint64_t)t, (uint64_t)c, 0, 0, S.seed, 0);
    const float* lq = S.cur_lq + (size_t)c * P;
    const int blk = (P + 31) / 32;
    const int j0 = lane * blk, j1 = min(P, j0 + blk);
    float part = 0.f;
    for (int j = j0; j < j1; ++j) part += expf(lq[j]);
    float incl = part;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const float total = __shfl_sync(0xffffffffu, incl, 31);
    const double u = __dmul_rn(__dadd_rn((double)(x.x[2] >> 11), 0.5), 0x1p-53);
    const float target = (float)(u * (double)total);
    const unsigned over = __ballot_sync(0xffffffffu, incl > target && j1 > j0);
    int owner = over ? __ffs(over) - 1 : 31;
    while (owner > 0 && (owner * blk >= P)) --owner;            // a lane that holds pairs
    int pair = -1;
    if (lane == owner) {
        float cum = incl - part;
        for (int j = j0; j < j1; ++j) {
            cum += expf(lq[j]);
            if (cum > target) { pair = j; break; }
        }
        if (pair < 0) pair = j1 - 1;
    }
    pair = __shfl_sync(0xffffffffu, pair, owner);
    int a, b;
    pair_decode(n, (uint64_t)pair, a, b);
    swap_and_list(S, c, a, b, lane);
    if (lane == 0) {
        S.prop_u[c] = __dmul_rn(__dadd_rn((double)(x.x[1] >> 12), 0.5), 0x1p-52);
        S.prop_pair[c] = (uint32_t)pair;
        S.prop_lqf[c] = lq[pair];
    }
}

// log q(. | order) of every chain from the network's logits (row stride ldl):
// log((1 - eps) softmax + eps / P), one warp per chain
__global__ void k_log_q(const float* __restrict__ L, int ldl, int C, int P, float eps, float* __restrict__ out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= C) return;
    const float* l = L + (size_t)c * ldl;
    float mx = -INFINITY;
    for (int j = lane; j < P; j += 32) mx = fmaxf(mx, l[j]);
#pragma unroll
    for (int off = 16; off; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    float s = 0.f;
    for (int j = lane; j < P; j += 32) s += __expf(l[j] - mx);
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const float lse = mx + __logf(s);
    const float w = 1.f - eps, e = eps / (float)P;
    for (int j = lane; j < P; j += 32) out[(size_t)c * P + j] = __logf(w * __expf(l[j] - lse) + e);
}

// training batch of the last uniform step: the pre-step order (the proposal with the
// pair swapped back), the pair index and alpha = min(1, 10^delta)
__global__ void k_train_batch(ChainState S)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S.C) return;
    const int n = S.n;
    const int a = S.prop_ab[2 * c], b = S.prop_ab[2 * c + 1];
    const uint8_t* po = S.prop_order + (size_t)c * n;
    uint8_t* o = S.train_orders + (size_t)c * n;
    for (int p = 0; p < n; ++p) o[p] = po[p == a ? b : p == b ? a : p];
    S.train_pairs[c] = (uint32_t)(a * (2 * n - a - 1) / 2 + (b - a - 1));
    // the swap's acceptance probability, but 0 for swaps that change no parent set
    // (always accepted, they move nothing)
    const float d = S.delta[c];
    S.train_alpha[c] = S.changed[c] ? (d >= 0.f ? 1.f : exp10f(d)) : 0.f;
}

// Geyer initial monotone sequence ESS of each recorded edge-indicator series, summed over
// chains.  Autocovariances are exact integers: T^3 g_k = T^2 P_k - T S (S1_k + S2_k) + (T-k) S^2
// with P_k = sum_t x_t x_{t+k}, S = sum x, S1_k = sum_{t<T-k} x_t, S2_k = sum_{t>=k} x_t.
__device__ __forceinline__ int bit_at(const uint64_t* w, int64_t t) { return (int)((w[t >> 6] >> (t & 63)) & 1ull); }

__device__ int64_t lag_products(const uint64_t* w, int words, int64_t T, int64_t k)
{
    // sum_{t=0}^{T-1-k} x_t x_{t+k}
    int64_t s = 0;
    const int64_t ws = k >> 6, bs = k & 63;
    for (int64_t q = 0; q < words; ++q) {
        const int64_t qs = q + ws;
        if (qs >= words) break;
        uint64_t sh = w[qs] >> bs;
        if (bs && qs + 1 < words) sh |= w[qs + 1] << (64 - bs);
        uint64_t v = w[q] & sh;
        // keep only t with t + k < T
        const int64_t t0 = q * 64;
        const int64_t lim = T - k - t0;
        if (lim <= 0) break;
        if (lim < 64) v &= (1ull << lim) - 1;
        s += __popcll(v);
    }
    return s;
}

__global__ void k_ess(const uint64_t* __restrict__ bits, int C, int n, int words, int64_t T, double* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;     // edge index i*n + m
    if (e >= n * n) return;
    if (T < 2) { out[e] = NAN; return; }
    double total = 0.0;
    bool any = false;
    const double T3 = (double)T * (double)T * (double)T;
    for (int c = 0; c < C; ++c) {
        const uint64_t* w = bits + ((size_t)c * n * n + e) * words;
        int64_t Ssum = 0;
        for (int q = 0; q < words; ++q) Ssum += __popcll(w[q]);
        if (Ssum == 0 || Ssum == T) continue;                  // constant series
        // prefix counts for S1_k (first T-k) and S2_k (last T-k) computed incrementally
        int64_t head = Ssum, tail = Ssum;                       // k = 0
        auto gk = [&](int64_t k, int64_t P) -> double {
            const __int128 v = (__int128)T * T * P - (__int128)T * Ssum * (head + tail) + (__int128)(T - k) * Ssum * Ssum;
            return (double)v / T3;
        };
        const double g0 = gk(0, Ssum);
        double sum = 0.0, prev = INFINITY;
        for (int64_t j = 0; 2 * j + 1 < T; ++j) {
            double g[2];
            for (int h = 0; h < 2; ++h) {
                const int64_t k = 2 * j + h;
                if (k > 0) {
                    head -= bit_at(w, T - k);                   // drop x_{T-k} from the first T-k
                    tail -= bit_at(w, k - 1);                   // drop x_{k-1} from the last T-k
                }
                g[h] = (k == 0) ? g0 : gk(k, lag_products(w, words, T, k));
            }
            double G = g[0] + g[1];
            if (!(G > 0.0)) break;
            if (G > prev) G = prev;
            sum += G;
            prev = G;
        }
        const double sigma2 = -g0 + 2.0 * sum;
        if (sigma2 > 0.0) { total += (double)T * g0 / sigma2; any = true; }
    }
    out[e] = any ? total : NAN;
}

__global__ void k_edge_freq(const uint32_t* __restrict__ edge, int C, int n, double denom, double* __restrict__ out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    uint64_t s = 0;
    for (int c = 0; c < C; ++c) s += edge[(size_t)c * n * n + e];
    out[e] = denom > 0 ? (double)s / denom : 0.0;
}

// best chain (highest best score, lowest chain id on ties) and its greedy DAG
__global__ void k_pick_best(const double* __restrict__ best_score, const uint8_t* __restrict__ best_order,
                            const uint32_t* __restrict__ best_rank, const uint64_t* __restrict__ pst, int C, int n,
                            uint8_t* __restrict__ out_order, uint8_t* __restrict__ out_dag, double* __restrict__ out_score)
{
    __shared__ int s_c;
    if (threadIdx.x == 0) {
        int bc = 0;
        for (int c = 1; c < C; ++c)
            if (best_score[c] > best_score[bc]) bc = c;
        s_c = bc;
        *out_score = best_score[bc];
    }
    __syncthreads();
    const int bc = s_c;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        out_order[i] = best_order[(size_t)bc * n + i];
        for (int m = 0; m < n; ++m) out_dag[(size_t)i * n + m] = 0;
        uint64_t msk = pst[best_rank[(size_t)bc * n + i]];
        while (msk) {
            const int slot = __ffsll((long long)msk) - 1;
            msk &= msk - 1;
            out_dag[(size_t)i * n + slot + (slot >= i ? 1 : 0)] = 1;
        }
    }
}

}  // namespace bn

using namespace bn;

static constexpr int FUSED_ITERS = 1024;    // MH steps per fused launch

static bool fused_path(const bn_chains* ch)
{
    return ch->S.mode == BN_PROPOSAL_UNIFORM && ch->t->scan_mode == BN_SCAN_PRUNED;
}

// `iters` fused steps starting at step t0; ev0/ev1 (optional) bracket the fused kernel
static int fused_launch(bn_chains* ch, int64_t t0, int iters, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                        cudaEvent_t ev1 = nullptr)
{
    FusedArgs F;
    F.amask = ch->t->amask;
    F.aspos = ch->t->aspos;
    F.aoff = ch->t->aoff;
    F.acnt = ch->t->acnt;
    F.t0 = t0;
    F.iters = iters;
    F.staged = ch->t->alive_total <= SURV_CAP_MAX && ch->t->max_abs_survivor < FX_LIMIT ? 1 : 0;
    F.gcache = F.staged ? nullptr : ch->t->gcache;
    F.gfirst = F.gcache ? (const uint16_t*)(F.gcache + surv_cache_stride((int)ch->t->alive_total)) : nullptr;
    F.cap = (F.staged || F.gcache) ? (int)ch->t->alive_total : 0;
    F.margin_x = mh_margin(ch->S.n, ch->t->max_abs_survivor);
    F.guard_fx = score_guard_fx(ch->S.n, ch->t->max_abs_survivor);
    size_t smem = 0;
    int rc = fused_smem_setup(F.staged ? F.cap : 0, &smem);
    if (rc) return rc;
    if (!F.staged) smem = 0;
    const unsigned grid = (unsigned)((ch->S.C + FUSED_WARPS - 1) / FUSED_WARPS);
    if (ev0) BN_CUDA(cudaEventRecord(ev0, s));
    if (F.staged || F.gcache) {
        // cached networks: several warps per chain evaluate consecutive steps at once
        if (F.staged) k_chain_spec<1><<<(unsigned)ch->S.C, 32 * SPEC_WARPS, smem, s>>>(ch->S, F);
        else k_chain_spec<2><<<(unsigned)ch->S.C, 32 * SPEC_WARPS, 0, s>>>(ch->S, F);
        BN_LAUNCH_CHECK("k_chain_spec");
    } else {
        k_chain_fused<0><<<grid, 32 * FUSED_WARPS, 0, s>>>(ch->S, F);
        BN_LAUNCH_CHECK("k_chain_fused");
    }
    if (ev1) BN_CUDA(cudaEventRecord(ev1, s));
    k_step_advance<<<1, 1, 0, s>>>(ch->S, iters);
    BN_LAUNCH_CHECK("k_step_advance");
    return BN_OK;
}

// one MH step of every chain; ev0/ev1 (optional) bracket the scan launch
static int sweep_launch(bn_chains* ch, cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr)
{
    const ChainState& S = ch->S;
    const int64_t l0 = bn_kernel_launches();
    int rc;
    if (S.mode == BN_PROPOSAL_LEARNED) {
        k_propose_learned<<<(S.C + 7) / 8, 256, 0, s>>>(S);
        BN_LAUNCH_CHECK("k_propose_learned");
        if ((rc = mlp_forward_dev(ch->mlp, S.prop_order, S.C, false, s))) return rc;
        k_log_q<<<(S.C + 7) / 8, 256, 0, s>>>(ch->mlp->L, ch->mlp->Pp, S.C, S.P, S.eps_mix, S.prop_lq);
        BN_LAUNCH_CHECK("k_log_q");
    } else {
        k_propose<<<(S.C + 7) / 8, 256, 0, s>>>(S);
        BN_LAUNCH_CHECK("k_propose");
    }
    if (ev0) BN_CUDA(cudaEventRecord(ev0, s));
    rc = launch_scan(ch->t, ch->plan, S.list_count, S.list_pc, S.list_best, S.C, S.status, s);
    if (rc) return rc;
    if (ev1) BN_CUDA(cudaEventRecord(ev1, s));
    k_accept<<<(S.C + 7) / 8, 256, 0, s>>>(S);
    BN_LAUNCH_CHECK("k_accept");
    if (S.mode == BN_PROPOSAL_TRAIN) {
        k_train_batch<<<(S.C + 127) / 128, 128, 0, s>>>(S);
        BN_LAUNCH_CHECK("k_train_batch");
        if ((rc = mlp_loss_grad_dev(ch->mlp, S.train_orders, S.train_pairs, S.train_alpha, S.C, s))) return rc;
        if ((rc = mlp_adam_dev(ch->mlp, s))) return rc;
    }
    ch->per_sweep = (int)(bn_kernel_launches() - l0);
    return BN_OK;
}

// q(. | current order) of every chain for the graph path of the learned proposal
static int refresh_lq(bn_chains* ch, cudaStream_t s)
{
    ChainState& S = ch->S;
    int rc = mlp_forward_dev(ch->mlp, S.cur_order, S.C, false, s);
    if (rc) return rc;
    k_log_q<<<(S.C + 7) / 8, 256, 0, s>>>(ch->mlp->L, ch->mlp->Pp, S.C, S.P, S.eps_mix, S.cur_lq);
    BN_LAUNCH_CHECK("k_log_q");
    ch->lq_valid = true;
    return BN_OK;
}

extern "C" int bn_chains_create(const bn_table* t, const bn_mcmc_params* p, const uint8_t* init_orders, int mem,
                                void* stream, bn_chains** out)
{
    set_error(BN_OK, "");
    if (!out) return set_error(BN_EINVAL, "bn_chains_create: out is NULL");
    *out = nullptr;
    if (!t || !p) return set_error(BN_EINVAL, "bn_chains_create: NULL table/params");
    if (p->chains < 1 || p->chains > 65536) return set_error(BN_EINVAL, "bn_chains_create: chains=%d", p->chains);
    if (p->burn_in < 0 || p->record_every < 0 || p->record_cap < 0 || p->trace_cap < 0)
        return set_error(BN_EINVAL, "bn_chains_create: negative burn_in/record/trace");
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_chains_create: bad mem");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->chains <= 2048) {                          // the full-table scan's tiling, once per table
        int rt = ensure_tuned(t, p->chains, s);
        if (rt) return rt;
    }
    bn_chains* ch = new bn_chains();
    ch->t = t;
    ch->p = *p;
    ch->dev = device_id();
    const int n = t->n, C = p->chains;
    ch->plan = plan_scan(t, C);
    ChainState& S = ch->S;
    S.n = n;
    S.C = C;
    S.seed = p->seed;
    S.burn_in = p->burn_in;
    S.literal_log = p->literal_log;
    S.trace_cap = p->trace ? p->trace_cap : 0;
    S.record_every = p->record_cap > 0 ? p->record_every : 0;
    S.record_cap = S.record_every > 0 ? p->record_cap : 0;
    S.rec_words = (S.record_cap + 63) / 64;
    S.keys = t->keys;
    S.pst = t->pst;
    S.srank = t->srank;
    S.Sp = t->Sp;

    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up((int64_t)(off + bytes), 256); return o; };
    const size_t Cn = (size_t)C * n;
    size_t o_cur_order = take(Cn), o_cur_rank = take(4 * Cn), o_cur_key = take(8 * Cn), o_cur_score = take(8 * C);
    size_t o_best_order = take(Cn), o_best_rank = take(4 * Cn), o_best_score = take(8 * C), o_acc = take(8 * C);
    size_t o_edge = take(4 * Cn * n), o_prop_order = take(Cn), o_prop_ab = take(2 * C), o_prop_u = take(8 * C);
    size_t o_cnt = take(4 * (size_t)n), o_pc = take(8 * Cn), o_slot = take(4 * Cn);
    size_t o_best = take(4 * Cn);
    size_t o_step = take(8), o_status = take(4), o_done = take(4), o_rec_count = take(8), o_items = take(8);
    size_t o_ts = take(8 * (size_t)C * S.trace_cap), o_ta = take((size_t)C * S.trace_cap);
    size_t o_rec = take(8 * Cn * n * S.rec_words);
    size_t o_init = take(mem == BN_MEM_HOST && init_orders ? Cn : 0);
    cudaError_t e = cudaMalloc(&ch->block, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ch;
        return set_error(BN_ENOMEM, "bn_chains_create: %zu bytes of chain state: %s", off, cudaGetErrorString(e));
    }
    uint8_t* B = (uint8_t*)ch->block;
    S.cur_order = B + o_cur_order;
    S.cur_rank = (uint32_t*)(B + o_cur_rank);
    S.cur_key = (int64_t*)(B + o_cur_key);
    S.cur_score = (double*)(B + o_cur_score);
    S.best_order = B + o_best_order;
    S.best_rank = (uint32_t*)(B + o_best_rank);
    S.best_score = (double*)(B + o_best_score);
    S.accepts = (int64_t*)(B + o_acc);
    S.edge = (uint32_t*)(B + o_edge);
    S.prop_order = B + o_prop_order;
    S.prop_ab = B + o_prop_ab;
    S.prop_u = (double*)(B + o_prop_u);
    S.list_count = (uint32_t*)(B + o_cnt);
    S.list_pc = (uint64_t*)(B + o_pc);
    S.slot_of = (uint32_t*)(B + o_slot);
    S.list_best = (uint32_t*)(B + o_best);
    S.step = (int64_t*)(B + o_step);
    S.status = (uint32_t*)(B + o_status);
    S.done = (uint32_t*)(B + o_done);
    S.rec_count = (int64_t*)(B + o_rec_count);
    S.items_total = (int64_t*)(B + o_items);
    S.trace_score = (double*)(B + o_ts);
    S.trace_accept = B + o_ta;
    S.rec_bits = (uint64_t*)(B + o_rec);

    auto fail = [&](int rc) { bn_chains_free(ch); return rc; };
    if (cudaMemsetAsync(ch->block, 0, off, s) != cudaSuccess) return fail(cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__));
    if (init_orders) {
        const uint8_t* src = init_orders;
        if (mem == BN_MEM_HOST) {
            if (cudaMemcpyAsync(B + o_init, init_orders, Cn, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return fail(cuda_fail(cudaGetLastError(), "copy init orders", __FILE__, __LINE__));
            src = B + o_init;
        }
        if (cudaMemcpyAsync(S.cur_order, src, Cn, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return fail(cuda_fail(cudaGetLastError(), "copy init orders", __FILE__, __LINE__));
    } else {
        k_init_orders<<<(C + 127) / 128, 128, 0, s>>>(S);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return fail(cuda_fail(le, "k_init_orders", __FILE__, __LINE__));
        count_launches(1);
    }
    // full scoring of the initial orders through the node-major lists
    int rc = launch_pred_lists(S.cur_order, C, n, S.list_pc, S.list_best, S.list_count, S.status, s);
    if (rc) return fail(rc);
    if ((rc = launch_scan(t, ch->plan, S.list_count, S.list_pc, S.list_best, C, S.status, s))) return fail(rc);
    k_init_state<<<(C + 7) / 8, 256, 0, s>>>(S);
    {
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return fail(cuda_fail(le, "k_init_state", __FILE__, __LINE__));
        count_launches(1);
    }
    if (cudaMemsetAsync(S.list_count, 0, 4 * (size_t)n, s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "memset", __FILE__, __LINE__));
    uint32_t st = 0;
    if (cudaMemcpyAsync(&st, S.status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "bn_chains_create sync", __FILE__, __LINE__));
    if (st & STATUS_BADINPUT) return fail(set_error(BN_EINVAL, "bn_chains_create: an initial order is not a permutation"));
    if (st & STATUS_TIMEOUT) return fail(set_error(BN_ETIMEOUT, "bn_chains_create: a bounded device wait expired"));
    *out = ch;
    return BN_OK;
}

extern "C" int bn_chains_step(bn_chains* ch, int64_t steps, void* stream)
{
    set_error(BN_OK, "");
    if (!ch) return set_error(BN_EINVAL, "bn_chains_step: NULL chains");
    if (steps < 0) return set_error(BN_EINVAL, "bn_chains_step: steps < 0");
    if (steps == 0) return BN_OK;
    cudaStream_t user = (cudaStream_t)stream;
    cudaStream_t s = user;
    cudaStream_t own = nullptr;
    if (user == nullptr) {
        BN_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        BN_CUDA(cudaDeviceSynchronize());
        s = own;
    }
    struct Own {
        cudaStream_t s;
        ~Own()
        {
            if (s) cudaStreamDestroy(s);
        }
    } own_guard{own};
    if (learned_path(ch)) {
        int rc = learned_step(ch, steps, s);
        if (rc) return rc;
        ch->steps += steps;
        ch->lq_valid = false;
        return BN_OK;
    }
    learned_invalidate(ch->lp, false);         // the orders move outside the learned path
    if (ch->S.mode == BN_PROPOSAL_LEARNED && !ch->lq_valid) {
        int rc = refresh_lq(ch, s);
        if (rc) return rc;
    }
    if (fused_path(ch)) {
        for (int64_t done = 0; done < steps;) {
            const int it = (int)std::min<int64_t>(FUSED_ITERS, steps - done);
            int rc = fused_launch(ch, ch->steps + done, it, s);
            if (rc) return rc;
            done += it;
        }
        ch->steps += steps;
        BN_CUDA(cudaStreamSynchronize(s));
        return BN_OK;
    }
    if (ch->exec && ch->exec_scan_mode != ch->t->scan_mode) {
        cudaGraphExecDestroy(ch->exec);
        ch->exec = nullptr;
    }
    if (!ch->exec) {
        cudaGraph_t g = nullptr;
        ch->exec_scan_mode = ch->t->scan_mode;
        BN_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = sweep_launch(ch, s);
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
        cudaError_t ie = cudaGraphInstantiate(&ch->exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate", __FILE__, __LINE__);
        count_launches(-ch->per_sweep);     // the captured launches did not run
    }
    for (int64_t i = 0; i < steps; ++i) BN_CUDA(cudaGraphLaunch(ch->exec, s));
    count_launches(ch->per_sweep * steps);
    ch->steps += steps;
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, ch->S.status, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_chains_step: a bounded device wait expired");
    return BN_OK;
}

extern "C" int bn_chains_step_profiled(bn_chains* ch, int64_t steps, void* stream, double* scan_ms,
                                       int64_t* scan_launches)
{
    set_error(BN_OK, "");
    if (!ch) return set_error(BN_EINVAL, "bn_chains_step_profiled: NULL chains");
    if (steps < 0) return set_error(BN_EINVAL, "bn_chains_step_profiled: steps < 0");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<cudaEvent_t> ev(2 * (size_t)std::max<int64_t>(steps, 1));
    for (auto& e : ev) BN_CUDA(cudaEventCreate(&e));
    struct Ev {
        std::vector<cudaEvent_t>& v;
        ~Ev()
        {
            for (auto e : v) cudaEventDestroy(e);
        }
    } ev_guard{ev};
    int64_t launches = steps;
    if (learned_path(ch)) {
        // the whole learned step (three kernels per MH step) between one pair of events
        BN_CUDA(cudaEventRecord(ev[0], s));
        int rc = learned_step(ch, steps, s);
        if (rc) return rc;
        BN_CUDA(cudaEventRecord(ev[1], s));
        ch->lq_valid = false;
        launches = 1;
    } else if (fused_path(ch)) {
        // the fused kernel is the whole step: its launches are what the events bracket
        launches = 0;
        for (int64_t done = 0; done < steps; ++launches) {
            const int it = (int)std::min<int64_t>(FUSED_ITERS, steps - done);
            int rc = fused_launch(ch, ch->steps + done, it, s, ev[2 * launches], ev[2 * launches + 1]);
            if (rc) return rc;
            done += it;
        }
    } else {
        learned_invalidate(ch->lp, false);
        if (ch->S.mode == BN_PROPOSAL_LEARNED && !ch->lq_valid) {
            int rc = refresh_lq(ch, s);
            if (rc) return rc;
        }
        for (int64_t i = 0; i < steps; ++i) {
            int rc = sweep_launch(ch, s, ev[2 * i], ev[2 * i + 1]);
            if (rc) return rc;
        }
    }
    ch->steps += steps;
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, ch->S.status, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    double tot = 0.0;
    for (int64_t i = 0; i < launches; ++i) {
        float ms = 0.f;
        BN_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        tot += ms;
    }
    if (scan_ms) *scan_ms = tot;
    if (scan_launches) *scan_launches = launches;
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_chains_step_profiled: a bounded device wait expired");
    return BN_OK;
}

extern "C" int bn_chains_read(const bn_chains* ch, int what, void* out, int mem, void* stream)
{
    set_error(BN_OK, "");
    if (!ch || !out) return set_error(BN_EINVAL, "bn_chains_read: NULL argument");
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_chains_read: bad mem");
    cudaStream_t s = (cudaStream_t)stream;
    const ChainState& S = ch->S;
    const size_t Cn = (size_t)S.C * S.n;
    const void* src = nullptr;
    size_t bytes = 0;
    switch (what) {
        case BN_OUT_ORDERS: src = S.cur_order; bytes = Cn; break;
        case BN_OUT_SCORES: src = S.cur_score; bytes = 8 * (size_t)S.C; break;
        case BN_OUT_RANKS: src = S.cur_rank; bytes = 4 * Cn; break;
        case BN_OUT_BEST_ORDERS: src = S.best_order; bytes = Cn; break;
        case BN_OUT_BEST_SCORES: src = S.best_score; bytes = 8 * (size_t)S.C; break;
        case BN_OUT_BEST_RANKS: src = S.best_rank; bytes = 4 * Cn; break;
        case BN_OUT_EDGE_COUNTS: src = S.edge; bytes = 4 * Cn * S.n; break;
        case BN_OUT_ACCEPTS: src = S.accepts; bytes = 8 * (size_t)S.C; break;
        case BN_OUT_TRACE_SCORE: src = S.trace_score; bytes = 8 * (size_t)S.C * S.trace_cap; break;
        case BN_OUT_TRACE_ACCEPT: src = S.trace_accept; bytes = (size_t)S.C * S.trace_cap; break;
        case BN_OUT_STEPS: src = S.step; bytes = 8; break;
        case BN_OUT_RECORD: src = S.rec_bits; bytes = 8 * Cn * S.n * S.rec_words; break;
        case BN_OUT_RECORD_LEN: src = S.rec_count; bytes = 8; break;
        case BN_OUT_ITEMS: src = S.items_total; bytes = 8; break;
        case BN_OUT_ESS: {
            int64_t T = 0;
            BN_CUDA(cudaMemcpyAsync(&T, S.rec_count, 8, cudaMemcpyDeviceToHost, s));
            BN_CUDA(cudaStreamSynchronize(s));
            double* d = (double*)out;
            double* tmp = nullptr;
            if (mem == BN_MEM_HOST) {
                BN_CUDA(cudaMallocAsync((void**)&tmp, 8 * (size_t)S.n * S.n, s));
                d = tmp;
            }
            const int nn = S.n * S.n;
            k_ess<<<(nn + 127) / 128, 128, 0, s>>>(S.rec_bits, S.C, S.n, std::max(S.rec_words, 1), T, d);
            BN_LAUNCH_CHECK("k_ess");
            if (mem == BN_MEM_HOST) {
                BN_CUDA(cudaMemcpyAsync(out, tmp, 8 * (size_t)nn, cudaMemcpyDeviceToHost, s));
                BN_CUDA(cudaFreeAsync(tmp, s));
            }
            BN_CUDA(cudaStreamSynchronize(s));
            return BN_OK;
        }
        case BN_OUT_LOGITS: return learned_read_logits(ch, (float*)out, mem, s);
        default: return set_error(BN_EINVAL, "bn_chains_read: unknown output %d", what);
    }
    if (bytes) BN_CUDA(cudaMemcpyAsync(out, src, bytes, mem == BN_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    BN_CUDA(cudaStreamSynchronize(s));
    return BN_OK;
}

extern "C" void bn_chains_free(bn_chains* ch)
{
    if (!ch) return;
    if (ch->exec) cudaGraphExecDestroy(ch->exec);
    learned_free(ch->lp);
    cudaFree(ch->block);
    cudaFree(ch->prop_block);
    delete ch;
}

extern "C" int bn_chains_set_proposal(bn_chains* ch, bn_mlp* m, int mode, double eps_mix, void* stream)
{
    set_error(BN_OK, "");
    if (!ch) return set_error(BN_EINVAL, "bn_chains_set_proposal: NULL chains");
    if (mode != BN_PROPOSAL_UNIFORM && mode != BN_PROPOSAL_LEARNED && mode != BN_PROPOSAL_TRAIN)
        return set_error(BN_EINVAL, "bn_chains_set_proposal: mode %d", mode);
    ChainState& S = ch->S;
    if (mode != BN_PROPOSAL_UNIFORM) {
        if (!m) return set_error(BN_EINVAL, "bn_chains_set_proposal: the learned modes need a network");
        if (m->n != S.n) return set_error(BN_EINVAL, "bn_chains_set_proposal: network n=%d, chains n=%d", m->n, S.n);
        if (m->cap < S.C) return set_error(BN_EINVAL, "bn_chains_set_proposal: batch_cap %d < %d chains", m->cap, S.C);
        if (!(eps_mix > 0.0 && eps_mix <= 1.0)) return set_error(BN_EINVAL, "bn_chains_set_proposal: eps_mix in (0, 1]");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (ch->exec) {                                   // the step graph changes shape
        cudaGraphExecDestroy(ch->exec);
        ch->exec = nullptr;
    }
    S.P = S.n * (S.n - 1) / 2;
    if (!ch->prop_block) {
        const size_t C = (size_t)S.C, P = (size_t)S.P;
        size_t off = 0;
        auto take = [&](size_t bytes) {
            const size_t o = off;
            off = (size_t)round_up((int64_t)(off + bytes), 256);
            return o;
        };
        const size_t o_cur = take(4 * C * P), o_prop = take(4 * C * P), o_pair = take(4 * C), o_lqf = take(4 * C),
                     o_delta = take(4 * C), o_to = take(C * S.n), o_tp = take(4 * C), o_ta = take(4 * C),
                     o_ch = take(C);
        cudaError_t e = cudaMalloc(&ch->prop_block, off);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ch->prop_block = nullptr;
            return set_error(BN_ENOMEM, "bn_chains_set_proposal: %zu bytes: %s", off, cudaGetErrorString(e));
        }
        uint8_t* B = (uint8_t*)ch->prop_block;
        S.cur_lq = (float*)(B + o_cur);
        S.prop_lq = (float*)(B + o_prop);
        S.prop_pair = (uint32_t*)(B + o_pair);
        S.prop_lqf = (float*)(B + o_lqf);
        S.delta = (float*)(B + o_delta);
        S.train_orders = B + o_to;
        S.train_pairs = (uint32_t*)(B + o_tp);
        S.train_alpha = (float*)(B + o_ta);
        S.changed = B + o_ch;
        BN_CUDA(cudaMemsetAsync(ch->prop_block, 0, off, s));
    }
    ch->mlp = m;
    S.mode = mode;
    S.eps_mix = (float)eps_mix;
    learned_invalidate(ch->lp, true);                 // network or proposal changed
    ch->lq_valid = false;
    if (mode == BN_PROPOSAL_LEARNED) {
        // q(. | current order) of every chain from the network as it is now
        int rc = learned_path(ch) ? learned_setup(ch, s) : refresh_lq(ch, s);
        if (rc) return rc;
    }
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, m ? m->status : S.status, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_chains_set_proposal: a bounded device wait expired");
    return BN_OK;
}

// seeded initial weights of the proposal network bn_mcmc_run creates when none is given:
// uniform in [-1, 1) (fan-in scaled for the dense layers) from splitmix64, zero biases
static void default_mlp_weights(int n, int d, int H, uint64_t seed, std::vector<float>* w)
{
    const int P = n * (n - 1) / 2;
    uint64_t x = seed ^ 0x6a09e667f3bcc909ull;
    auto next = [&]() {
        uint64_t z = (x += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    };
    const size_t sz[7] = {(size_t)n * d, (size_t)H * n * d, (size_t)H, (size_t)H * H, (size_t)H, (size_t)P * H, (size_t)P};
    const float scale[7] = {1.f, 1.f / std::sqrt((float)(n * d)), 0.f, 1.f / std::sqrt((float)H), 0.f,
                            1.f / std::sqrt((float)H), 0.f};
    for (int i = 0; i < 7; ++i) {
        w[i].resize(sz[i]);
        for (size_t j = 0; j < sz[i]; ++j) w[i][j] = scale[i] == 0.f ? 0.f : next() * scale[i];
    }
}

extern "C" int bn_chains_set_learned_launch(bn_chains* ch, int mode)
{
    set_error(BN_OK, "");
    if (!ch || (mode != BN_LEARNED_LAUNCH_AUTO && mode != BN_LEARNED_LAUNCH_GRAPH))
        return set_error(BN_EINVAL, "bn_chains_set_learned_launch: bad arguments");
    ch->learned_launch = mode;
    return BN_OK;
}

// checks of the run-level fields of bn_mcmc_params (bn_mcmc_run, bn_mcmc_run_batch)
static int run_params_check(const bn_table* t, const bn_mcmc_params* p, const char* who)
{
    const bool learned = p->proposal == BN_PROPOSAL_LEARNED;
    if (!learned && p->proposal != BN_PROPOSAL_UNIFORM)
        return set_error(BN_EINVAL, "%s: proposal %d (BN_PROPOSAL_UNIFORM or BN_PROPOSAL_LEARNED)", who, p->proposal);
    if (learned && (!(p->eps_mix > 0.0 && p->eps_mix <= 1.0) || p->train_iters < 0))
        return set_error(BN_EINVAL, "%s: eps_mix in (0, 1] and train_iters >= 0 for the learned proposal", who);
    if (p->thin < 0) return set_error(BN_EINVAL, "%s: thin=%d", who, p->thin);
    if (learned && p->net && (p->net->n != t->n || p->net->cap < p->chains))
        return set_error(BN_EINVAL, "%s: the network's n or batch_cap does not fit the run", who);
    return BN_OK;
}

// the chain parameters of a run: traces off, recording from `thin` over all its steps
static bn_mcmc_params run_chain_params(const bn_mcmc_params* p, int64_t total)
{
    bn_mcmc_params cp = *p;
    cp.trace = 0;
    cp.trace_cap = 0;
    cp.record_every = p->thin;
    cp.record_cap = p->thin > 0 ? (int)std::max<int64_t>(1, (total - p->burn_in + p->thin - 1) / p->thin) : 0;
    return cp;
}

// the learned proposal's set-up of a run: the caller's network or one created from the
// seed (d = 32, H = 512), then train_iters training steps of the chains alone
static int run_learned_setup(bn_chains* ch, const bn_mcmc_params* p, void* stream, bn_mlp** own)
{
    bn_mlp* net = p->net;
    int rc;
    if (!net) {
        const int n = ch->S.n, d = 32, H = 512;
        std::vector<float> w[7];
        default_mlp_weights(n, d, H, p->seed, w);
        bn_mlp_params mp = {d, H, p->chains, 2e-3f, 0.f, 0.f, 0.f};
        if ((rc = bn_mlp_create(n, &mp, w[0].data(), w[1].data(), w[2].data(), w[3].data(), w[4].data(),
                                w[5].data(), w[6].data(), BN_MEM_HOST, stream, own)))
            return rc;
        net = *own;
    }
    if ((rc = bn_chains_set_proposal(ch, net, BN_PROPOSAL_TRAIN, p->eps_mix, stream))) return rc;
    if ((rc = bn_chains_step(ch, p->train_iters, stream))) return rc;
    return bn_chains_set_proposal(ch, net, BN_PROPOSAL_LEARNED, p->eps_mix, stream);
}

// a run's outputs from its chains: the best state over all chains and its greedy DAG,
// edge frequencies over the post-burn-in steps, and the summary (acc0: the chains'
// accept counters before the sampling steps)
static int run_collect(bn_chains* ch, const bn_mcmc_params* p, int64_t total, int64_t steps,
                       const std::vector<int64_t>& acc0, double sample_ms, double train_ms, uint8_t* best_order,
                       uint8_t* best_dag, double* best_score, double* edge_freq, bn_mcmc_stats* stats, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const bn_table* t = ch->t;
    const int n = t->n, C = p->chains;
    uint8_t *d_o = nullptr, *d_dag = nullptr;
    double *d_s = nullptr, *d_f = nullptr;
    BN_CUDA(cudaMallocAsync((void**)&d_o, n, s));
    BN_CUDA(cudaMallocAsync((void**)&d_dag, (size_t)n * n, s));
    BN_CUDA(cudaMallocAsync((void**)&d_s, 8, s));
    BN_CUDA(cudaMallocAsync((void**)&d_f, 8 * (size_t)n * n, s));
    k_pick_best<<<1, 64, 0, s>>>(ch->S.best_score, ch->S.best_order, ch->S.best_rank, t->pst, C, n, d_o, d_dag, d_s);
    BN_LAUNCH_CHECK("k_pick_best");
    const double denom = (double)C * (double)std::max<int64_t>(0, total - p->burn_in);
    k_edge_freq<<<(n * n + 127) / 128, 128, 0, s>>>(ch->S.edge, C, n, denom, d_f);
    BN_LAUNCH_CHECK("k_edge_freq");
    std::vector<double> f((size_t)n * n);
    std::vector<int64_t> acc1(C);
    if (best_order) BN_CUDA(cudaMemcpyAsync(best_order, d_o, n, cudaMemcpyDeviceToHost, s));
    if (best_dag) BN_CUDA(cudaMemcpyAsync(best_dag, d_dag, (size_t)n * n, cudaMemcpyDeviceToHost, s));
    if (best_score) BN_CUDA(cudaMemcpyAsync(best_score, d_s, 8, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaMemcpyAsync(f.data(), d_f, 8 * (size_t)n * n, cudaMemcpyDeviceToHost, s));
    if (stats) BN_CUDA(cudaMemcpyAsync(acc1.data(), ch->S.accepts, 8 * (size_t)C, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(d_o, s);
    cudaFreeAsync(d_dag, s);
    cudaFreeAsync(d_s, s);
    cudaFreeAsync(d_f, s);
    BN_CUDA(cudaStreamSynchronize(s));
    if (edge_freq) std::copy(f.begin(), f.end(), edge_freq);
    if (stats) {
        bn_mcmc_stats st;
        int64_t acc = 0;
        for (int c = 0; c < C; ++c) acc += acc1[c] - acc0[c];
        st.acceptance = steps > 0 ? (double)acc / ((double)C * (double)steps) : 0.0;
        st.train_ms = train_ms;
        st.sample_ms = sample_ms;
        st.order_evals = (int64_t)C * total;
        st.ess_median = st.ess_min = std::nan("");
        st.uncertain_edges = 0;
        if (p->thin > 0) {
            std::vector<double> ess((size_t)n * n);
            int rc = bn_chains_read(ch, BN_OUT_ESS, ess.data(), BN_MEM_HOST, stream);
            if (rc) return rc;
            std::vector<double> unc;
            for (size_t e = 0; e < ess.size(); ++e)
                if (f[e] >= 0.05 && f[e] <= 0.95 && !std::isnan(ess[e])) unc.push_back(ess[e]);
            if (!unc.empty()) {
                std::sort(unc.begin(), unc.end());
                const size_t h = unc.size() / 2;
                st.ess_median = unc.size() % 2 ? unc[h] : 0.5 * (unc[h - 1] + unc[h]);
                st.ess_min = unc[0];
                st.uncertain_edges = (int64_t)unc.size();
            }
        }
        *stats = st;
    }
    return BN_OK;
}

struct RunEvents {
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    ~RunEvents()
    {
        for (int i = 0; i < 3; ++i)
            if (e[i]) cudaEventDestroy(e[i]);
    }
    int create()
    {
        for (int i = 0; i < 3; ++i) BN_CUDA(cudaEventCreate(&e[i]));
        return BN_OK;
    }
    double ms(int a, int b) const
    {
        float v = 0.f;
        cudaEventElapsedTime(&v, e[a], e[b]);
        return v;
    }
};

extern "C" int bn_mcmc_run(const bn_table* t, const bn_mcmc_params* p, int64_t steps, uint8_t* best_order,
                           uint8_t* best_dag, double* best_score, double* edge_freq, bn_mcmc_stats* stats,
                           void* stream)
{
    set_error(BN_OK, "");
    if (!t || !p || steps < 0) return set_error(BN_EINVAL, "bn_mcmc_run: bad arguments");
    int rc = run_params_check(t, p, "bn_mcmc_run");
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool learned = p->proposal == BN_PROPOSAL_LEARNED;
    const int C = p->chains;
    const int64_t total = (learned ? p->train_iters : 0) + steps;
    const bn_mcmc_params cp = run_chain_params(p, total);
    bn_chains* ch = nullptr;
    if ((rc = bn_chains_create(t, &cp, nullptr, BN_MEM_HOST, stream, &ch))) return rc;
    bn_mlp* own = nullptr;
    RunEvents ev;
    struct G {
        bn_chains* c;
        bn_mlp** m;
        ~G()
        {
            bn_chains_free(c);
            bn_mlp_free(*m);
        }
    } g{ch, &own};
    if ((rc = ev.create())) return rc;
    BN_CUDA(cudaEventRecord(ev.e[0], s));
    if (learned && (rc = run_learned_setup(ch, p, stream, &own))) return rc;
    std::vector<int64_t> acc0(C);
    if (stats) BN_CUDA(cudaMemcpyAsync(acc0.data(), ch->S.accepts, 8 * (size_t)C, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaEventRecord(ev.e[1], s));
    if ((rc = bn_chains_step(ch, steps, stream))) return rc;
    BN_CUDA(cudaEventRecord(ev.e[2], s));
    BN_CUDA(cudaEventSynchronize(ev.e[2]));
    return run_collect(ch, p, total, steps, acc0, ev.ms(1, 2), learned ? ev.ms(0, 1) : 0.0, best_order, best_dag,
                       best_score, edge_freq, stats, stream);
}

// ---------------------------------------------------------------------------------
// batches of networks of uneven size
// ---------------------------------------------------------------------------------
struct bn_batch {
    std::vector<bn_chains*> chains;
    void* dev = nullptr;            // device arrays: ChainState[], FusedArgs[], base[], iters[]
    size_t dev_bytes = 0;
};

extern "C" int bn_batch_create(int count, const bn_table* const* tables, const bn_mcmc_params* params, void* stream,
                               bn_batch** out)
{
    set_error(BN_OK, "");
    if (!out || count < 1 || !tables || !params) return set_error(BN_EINVAL, "bn_batch_create: bad arguments");
    *out = nullptr;
    bn_batch* b = new bn_batch();
    for (int i = 0; i < count; ++i) {
        bn_chains* c = nullptr;
        int rc = bn_chains_create(tables[i], &params[i], nullptr, BN_MEM_HOST, stream, &c);
        if (rc) {
            bn_batch_free(b);
            return rc;
        }
        b->chains.push_back(c);
    }
    const size_t bytes = (sizeof(ChainState) + sizeof(FusedArgs) + 2 * sizeof(int64_t)) * (size_t)(count + 1) + 1024;
    cudaError_t e = cudaMalloc(&b->dev, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        bn_batch_free(b);
        return set_error(BN_ENOMEM, "bn_batch_create: %zu bytes", bytes);
    }
    b->dev_bytes = bytes;
    *out = b;
    return BN_OK;
}

extern "C" int bn_batch_chains(bn_batch* b, int i, bn_chains** out)
{
    if (!b || !out || i < 0 || i >= (int)b->chains.size()) return set_error(BN_EINVAL, "bn_batch_chains: bad index");
    *out = b->chains[i];
    return BN_OK;
}

extern "C" int bn_batch_step(bn_batch* b, int64_t steps, void* stream)
{
    set_error(BN_OK, "");
    if (!b || steps < 0) return set_error(BN_EINVAL, "bn_batch_step: bad arguments");
    if (steps == 0) return BN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<bn_chains*> fused, other;
    for (bn_chains* c : b->chains) (fused_path(c) ? fused : other).push_back(c);
    // networks on other proposals step through their own per-network path
    for (bn_chains* c : other) {
        int rc = bn_chains_step(c, steps, stream);
        if (rc) return rc;
    }
    if (fused.empty()) return BN_OK;
    const int nf = (int)fused.size();
    std::vector<ChainState> hs(nf);
    std::vector<int64_t> base(nf + 1, 0);        // first block of every network
    for (int i = 0; i < nf; ++i) {
        hs[i] = fused[i]->S;
        base[i + 1] = base[i] + (fused[i]->S.C + BATCH_WARPS - 1) / BATCH_WARPS;
    }
    uint8_t* d = (uint8_t*)b->dev;
    ChainState* d_states = (ChainState*)d;
    int64_t* d_base = (int64_t*)(d + sizeof(ChainState) * (nf + 1));
    BN_CUDA(cudaMemcpyAsync(d_states, hs.data(), sizeof(ChainState) * nf, cudaMemcpyHostToDevice, s));
    BN_CUDA(cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * (nf + 1), cudaMemcpyHostToDevice, s));
    const unsigned blocks = (unsigned)base[nf];
    // shared-memory survivor caches up to `limit` survivors: SURV_CAP_MAX, or less when that
    // lets every block of the launch be resident at once (networks above the limit use
    // their global-memory cache)
    int limit = SURV_CAP_MAX;
    {
        const int per_sm = (int)((blocks + sm_count() - 1) / sm_count());
        if (per_sm > 2) {
            const long room = (long)(227 * 1024) / per_sm - (long)sizeof(FusedSmem) * BATCH_WARPS - 1024;
            const long fit = (room - 4 * (MAXN + 1) - 16) / 28;
            if (fit > 0) limit = (int)std::min<long>(limit, fit);
        }
    }
    int cap = 0;
    for (bn_chains* c : fused)
        if (c->t->alive_total <= limit && c->t->max_abs_survivor < FX_LIMIT)
            cap = std::max(cap, (int)c->t->alive_total);
    size_t smem = 0;
    {
        int rc = fused_smem_setup(cap, &smem);
        if (rc) return rc;
    }
    // every launch's arguments up front (one upload, no synchronisation between launches)
    const int64_t nl = (steps + FUSED_ITERS - 1) / FUSED_ITERS;
    std::vector<FusedArgs> hf((size_t)nl * nf);
    std::vector<int> hit((size_t)nl * nf);
    for (int64_t l = 0; l < nl; ++l) {
        const int64_t done = l * FUSED_ITERS;
        const int it = (int)std::min<int64_t>(FUSED_ITERS, steps - done);
        for (int i = 0; i < nf; ++i) {
            const bn_table* t = fused[i]->t;
            FusedArgs& f = hf[(size_t)l * nf + i];
            f.amask = t->amask;
            f.aspos = t->aspos;
            f.aoff = t->aoff;
            f.acnt = t->acnt;
            f.t0 = fused[i]->steps + done;
            f.iters = it;
            f.staged = t->alive_total <= cap && t->max_abs_survivor < FX_LIMIT ? 1 : 0;
            f.gcache = f.staged ? nullptr : t->gcache;
            f.gfirst = f.gcache ? (const uint16_t*)(f.gcache + surv_cache_stride((int)t->alive_total)) : nullptr;
            f.cap = f.gcache ? (int)t->alive_total : cap;
            f.margin_x = mh_margin(t->n, t->max_abs_survivor);
            f.guard_fx = score_guard_fx(t->n, t->max_abs_survivor);
            hit[(size_t)l * nf + i] = it;
        }
    }
    uint8_t* args = nullptr;
    const size_t fbytes = sizeof(FusedArgs) * hf.size(), ibytes = sizeof(int) * hit.size();
    BN_CUDA(cudaMallocAsync((void**)&args, fbytes + ibytes + 16, s));
    struct Free {
        uint8_t* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{args, s};
    FusedArgs* d_fargs = (FusedArgs*)args;
    int* d_iters = (int*)(args + fbytes);
    BN_CUDA(cudaMemcpyAsync(d_fargs, hf.data(), fbytes, cudaMemcpyHostToDevice, s));
    BN_CUDA(cudaMemcpyAsync(d_iters, hit.data(), ibytes, cudaMemcpyHostToDevice, s));
    for (int64_t l = 0; l < nl; ++l) {
        k_batch_fused<<<blocks, 32 * BATCH_WARPS, smem, s>>>(d_states, d_fargs + (size_t)l * nf, d_base, nf);
        BN_LAUNCH_CHECK("k_batch_fused");
        k_batch_advance<<<(nf + 127) / 128, 128, 0, s>>>(d_states, d_iters + (size_t)l * nf, nf);
        BN_LAUNCH_CHECK("k_batch_advance");
    }
    BN_CUDA(cudaStreamSynchronize(s));     // the host argument arrays are released after this
    for (bn_chains* c : fused) c->steps += steps;
    return BN_OK;
}

extern "C" void bn_batch_free(bn_batch* b)
{
    if (!b) return;
    for (bn_chains* c : b->chains) bn_chains_free(c);
    cudaFree(b->dev);
    delete b;
}

extern "C" int bn_mcmc_run_batch(int count, const bn_table* const* tables, const bn_mcmc_params* params,
                                 int64_t steps, uint8_t* const* best_order, uint8_t* const* best_dag,
                                 double* best_score, double* const* edge_freq, bn_mcmc_stats* stats, void* stream)
{
    set_error(BN_OK, "");
    if (count < 1 || !tables || !params || steps < 0) return set_error(BN_EINVAL, "bn_mcmc_run_batch: bad arguments");
    int rc;
    for (int i = 0; i < count; ++i) {
        if (!tables[i]) return set_error(BN_EINVAL, "bn_mcmc_run_batch: network %d has no table", i);
        if ((rc = run_params_check(tables[i], &params[i], "bn_mcmc_run_batch"))) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<bn_mcmc_params> cps(count);
    std::vector<int64_t> total(count);
    for (int i = 0; i < count; ++i) {
        const bool learned = params[i].proposal == BN_PROPOSAL_LEARNED;
        total[i] = (learned ? params[i].train_iters : 0) + steps;
        cps[i] = run_chain_params(&params[i], total[i]);
    }
    bn_batch* b = nullptr;
    if ((rc = bn_batch_create(count, tables, cps.data(), stream, &b))) return rc;
    std::vector<bn_mlp*> own(count, nullptr);
    struct G {
        bn_batch* b;
        std::vector<bn_mlp*>& m;
        ~G()
        {
            bn_batch_free(b);
            for (bn_mlp* x : m) bn_mlp_free(x);
        }
    } g{b, own};
    RunEvents ev;
    if ((rc = ev.create())) return rc;
    BN_CUDA(cudaEventRecord(ev.e[0], s));
    for (int i = 0; i < count; ++i)
        if (params[i].proposal == BN_PROPOSAL_LEARNED &&
            (rc = run_learned_setup(b->chains[i], &params[i], stream, &own[i])))
            return rc;
    std::vector<std::vector<int64_t>> acc0(count);
    for (int i = 0; i < count; ++i) {
        acc0[i].resize(params[i].chains);
        if (stats)
            BN_CUDA(cudaMemcpyAsync(acc0[i].data(), b->chains[i]->S.accepts, 8 * (size_t)params[i].chains,
                                    cudaMemcpyDeviceToHost, s));
    }
    BN_CUDA(cudaEventRecord(ev.e[1], s));
    if ((rc = bn_batch_step(b, steps, stream))) return rc;
    BN_CUDA(cudaEventRecord(ev.e[2], s));
    BN_CUDA(cudaEventSynchronize(ev.e[2]));
    const double sample_ms = ev.ms(1, 2), train_ms = ev.ms(0, 1);
    for (int i = 0; i < count; ++i) {
        const bool learned = params[i].proposal == BN_PROPOSAL_LEARNED;
        if ((rc = run_collect(b->chains[i], &params[i], total[i], steps, acc0[i], sample_ms, learned ? train_ms : 0.0,
                              best_order ? best_order[i] : nullptr, best_dag ? best_dag[i] : nullptr,
                              best_score ? &best_score[i] : nullptr, edge_freq ? edge_freq[i] : nullptr,
                              stats ? &stats[i] : nullptr, stream)))
            return rc;
    }
    return BN_OK;
}
