// bn_chain.cuh -- device state of a set of MH chains over node orders, shared by the
// uniform-proposal sampler (bn_mcmc.cu) and the learned-proposal sampler (bn_learned.cu).
#pragma once

#include <cmath>

#include "bn_mlp.cuh"
#include "bn_table.cuh"

namespace bn {

static constexpr double LN10 = 2.302585092994045684017991454684364208;

struct ChainState {
    int n, C;
    uint64_t seed;
    int64_t burn_in;
    int literal_log;
    int64_t trace_cap;
    int record_every, record_cap, rec_words;
    const int64_t* keys;       // table
    const uint64_t* pst;
    const uint32_t* srank;
    int64_t Sp;
    uint8_t* cur_order;        // C*n
    uint32_t* cur_rank;        // C*n
    int64_t* cur_key;          // C*n
    double* cur_score;         // C
    uint8_t* best_order;
    uint32_t* best_rank;
    double* best_score;
    int64_t* accepts;
    uint32_t* edge;            // C*n*n
    uint8_t* prop_order;       // C*n
    uint8_t* prop_ab;          // C*2
    double* prop_u;            // C
    uint32_t* list_count;      // n
    uint64_t* list_pc;         // n*C
    uint32_t* slot_of;         // C*n
    uint32_t* list_best;       // n*C  scan results (sorted positions)
    int64_t* step;             // 1
    uint32_t* status;          // 1
    uint32_t* done;            // 1
    double* trace_score;       // C*trace_cap
    uint8_t* trace_accept;
    uint64_t* rec_bits;        // C*n*n*rec_words
    int64_t* rec_count;        // 1
    int64_t* items_total;      // 1  (node, chain) items scanned so far
    // proposal (BN_PROPOSAL_*): learned draws and their log proposal probabilities
    int mode;
    int P;                     // n(n-1)/2
    float eps_mix;
    float* cur_lq;             // C*P  log q(. | current order)
    float* prop_lq;            // C*P  log q(. | proposed order)
    uint32_t* prop_pair;       // C
    float* prop_lqf;           // C  log q(pair | current)
    float* delta;              // C  s' - s of the last step (training target)
    uint8_t* changed;          // C  1 if the last proposal changed some node's parent set
    uint8_t* train_orders;     // C*n  pre-step orders of the last step
    uint32_t* train_pairs;     // C
    float* train_alpha;        // C
};

__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

__device__ __forceinline__ uint64_t compress_pred(uint64_t pred, int i)
{
    uint64_t lowm = (i == 0) ? 0ull : ((1ull << i) - 1);
    return (pred & lowm) | ((i + 1 < 64) ? ((pred >> (i + 1)) << i) : 0ull);
}

// credit the post-burn-in steps [from, to) during which node v held parent set `rank`
__device__ __forceinline__ void credit_edges(const ChainState& S, int c, int v, uint32_t rank, int64_t from, int64_t to)
{
    const int64_t lo = max(from, S.burn_in);
    if (to <= lo) return;
    const uint32_t d = (uint32_t)(to - lo);
    uint64_t m = S.pst[rank];
    uint32_t* E = S.edge + ((size_t)c * S.n + v) * S.n;
    while (m) {
        const int slot = __ffsll((long long)m) - 1;
        m &= m - 1;
        atomicAdd(&E[slot + (slot >= v ? 1 : 0)], d);     // no read-back: the warp does not wait
    }
}

// The whole warp walks one node's survivors [js, je), 32 a round; returns the first j with
// (m[j] & np) == 0 (je - 1, the empty set, if none before it).
__device__ __forceinline__ uint32_t warp_walk(const uint64_t* m, uint32_t js, uint32_t je, uint64_t np, int lane)
{
    for (uint32_t base = js; base < je; base += 32) {
        const uint32_t idx = base + lane;
        const unsigned b = __ballot_sync(0xffffffffu, idx < je && (m[idx] & np) == 0ull);
        if (b) return base + __ffs(b) - 1;
    }
    return je - 1;
}

// The span's re-scoring walks: every lane has up to two nodes (h = 0, 1; act[h]) and finds
// for each the first survivor j in [j[h], j1[h]) with (m[j] & npc[h]) == 0 (the last
// survivor, the empty set, always qualifies); on return j[h] holds the answer.  All 32
// lanes must call it.  With at most `warp_max` such nodes the whole warp walks them one
// after another, 32 survivors a round (the fused sampler on a cached network, whose
// kept-set test leaves ~3 nodes per step: measured on GB300 at n = 60, 1.66 us per step
// with warp walks always against 1.70 us with lane walks above 8 nodes and 1.73 us above
// 3); with more, every lane first walks its own nodes for 16 survivors and the warp then
// walks those still open (every span node re-scored: uncached networks, learned steps).
constexpr int WALK_PROBE = 8;   // survivors each lane tests of its own nodes before the warp walks
__device__ __forceinline__ void span_walk(const uint64_t* m, uint32_t (&j)[2], const uint32_t (&j1)[2],
                                          const uint64_t (&npc)[2], const bool (&act)[2], int lane,
                                          int warp_max)
{
    {
        const unsigned p0 = __ballot_sync(0xffffffffu, act[0]), p1 = __ballot_sync(0xffffffffu, act[1]);
        if (__popc(p0) + __popc(p1) <= warp_max) {
            // each lane first tests the first WALK_PROBE survivors of its own nodes, all loads
            // independent; a node whose answer lies there needs no warp walk (the same answer:
            // the first qualifying survivor in index order), the others go on after them
            bool open[2] = {act[0], act[1]};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!open[h]) continue;
                uint64_t pm[WALK_PROBE];
#pragma unroll
                for (int r = 0; r < WALK_PROBE; ++r) pm[r] = j[h] + r < j1[h] ? m[j[h] + r] : ~0ull;
                int first = WALK_PROBE;
#pragma unroll
                for (int r = WALK_PROBE - 1; r >= 0; --r)
                    if ((pm[r] & npc[h]) == 0ull) first = r;
                if (first < WALK_PROBE) {
                    j[h] += first;
                    open[h] = false;
                } else {
                    j[h] += WALK_PROBE;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned pend = __ballot_sync(0xffffffffu, open[h]);
                while (pend) {
                    const int src = __ffs(pend) - 1;
                    pend &= pend - 1;
                    const uint32_t js = __shfl_sync(0xffffffffu, j[h], src), je = __shfl_sync(0xffffffffu, j1[h], src);
                    const uint64_t np = __shfl_sync(0xffffffffu, npc[h], src);
                    const uint32_t hit = warp_walk(m, js, je, np, lane);
                    if (lane == src) j[h] = hit;
                }
            }
            return;
        }
    }
    bool open[2] = {false, false};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!act[h]) continue;
        uint32_t x = j[h];
        bool found = false;
        for (int r = 0; r < 4 && !found; ++r) {
            if (x + 4 <= j1[h]) {
                const uint64_t a0 = m[x], a1 = m[x + 1], a2 = m[x + 2], a3 = m[x + 3];
                if ((a0 & npc[h]) == 0ull) found = true;
                else if ((a1 & npc[h]) == 0ull) { x += 1; found = true; }
                else if ((a2 & npc[h]) == 0ull) { x += 2; found = true; }
                else if ((a3 & npc[h]) == 0ull) { x += 3; found = true; }
                else x += 4;
            } else {
                while (x + 1 < j1[h] && (m[x] & npc[h]) != 0ull) ++x;
                found = true;
            }
        }
        j[h] = x;
        open[h] = !found;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned pend = __ballot_sync(0xffffffffu, open[h]);
        while (pend) {
            const int src = __ffs(pend) - 1;
            pend &= pend - 1;
            const uint32_t js = __shfl_sync(0xffffffffu, j[h], src), je = __shfl_sync(0xffffffffu, j1[h], src);
            const uint64_t np = __shfl_sync(0xffffffffu, npc[h], src);
            const uint32_t hit = warp_walk(m, js, je, np, lane);
            if (lane == src) j[h] = hit;
        }
    }
}

// rounding bound of the MH test's right-hand side: two sequential sums of n entries of
// magnitude <= max_abs (each within (n - 1) 2^-53 n max_abs) and the change summed over
// the re-scored nodes, times ln 10, with a factor 8 to spare; plus, for a change summed in
// fixed point, its rounding (2n entries each within 2^-33), times ln 10 with a factor 2
inline double mh_margin(int n, double max_abs)
{
    return 8.0 * 2.31 * (double)(n + 8) * (double)n * max_abs * 0x1p-52 + 2.0 * 2.31 * (double)n * 0x1p-32;
}

// Guard of fixed-point order-score comparisons, in 2^-32 units: an order score summed left
// to right in FP64 from n entries of magnitude <= max_abs is within (n-1) 2^-53 n max_abs
// (x 1.01) of the exact sum, and the sum of the entries rounded to 2^-32 within n 2^-33 of
// it; G bounds both in 2^-32 units, and two scores whose fixed-point sums differ by more
// than 2G + 1 compare the same way in FP64.  One unit to spare.
inline int64_t score_guard_fx(int n, double max_abs)
{
    const double g = (1.01 * (double)(n - 1) * (double)n * max_abs * 0x1p-53 + (double)n * 0x1p-33) * 0x1p32;
    const int64_t G = (int64_t)std::ceil(g) + 1;
    return 2 * G + 2;
}

struct LearnedPath;                       // bn_learned.cu
int learned_setup(::bn_chains* ch, cudaStream_t s);
int learned_step(::bn_chains* ch, int64_t steps, cudaStream_t s);
void learned_free(LearnedPath* lp);
// the path's network outputs (and with `weights` its copies of the network) are stale
void learned_invalidate(LearnedPath* lp, bool weights);
bool learned_path(const ::bn_chains* ch);
int learned_read_logits(const ::bn_chains* ch, float* out, int mem, cudaStream_t s);

}  // namespace bn

struct bn_chains {
    const bn_table* t = nullptr;
    bn_mcmc_params p{};
    bn::ChainState S{};
    bn::ScanPlan plan{};
    void* block = nullptr;          // one device allocation holding all state
    void* prop_block = nullptr;     // learned-proposal buffers (bn_chains_set_proposal)
    bn_mlp* mlp = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_scan_mode = -1;        // table scan mode the graph was captured with
    int per_sweep = 3;              // kernel launches per step
    int64_t steps = 0;
    int dev = 0;
    bn::LearnedPath* lp = nullptr;  // fast learned-proposal path (bn_learned.cu)
    bool lq_valid = false;          // S.cur_lq matches the current orders (graph path)
    int learned_launch = BN_LEARNED_LAUNCH_AUTO;   // bn_chains_set_learned_launch
};

