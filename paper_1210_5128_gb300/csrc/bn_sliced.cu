// bn_sliced.cu -- the order score of Eq. (6) with the orders bit-sliced.
//
// In a node's entries ordered by sorted position (score descending, rank ascending; see
// bn_sort.cu) the answer for an order is the FIRST entry whose parent set lies inside
// the node's predecessors.  So the (entry, order) tests need not each keep a running
// minimum: slice the orders into 32-bit words instead.  For node i, group g of 32 work
// items and node v, the word P[v][g] has bit r set when v precedes i in item 32g + r.
// An entry with parent nodes {v1, .., vj} (j <= k <= 4) is consistent with exactly the
// items of P[v1][g] & .. & P[vj][g]: four shared-memory words and three ANDs test one
// entry against 32 orders at once.  Of those items, the ones this warp has not found
// yet take the entry's sorted position (a shared-memory atomicMin, by the lowest lane of
// a step that hits the item), and a warp-wide OR marks them found.  Every later entry of
// the warp lies further down the sorted list, so it can only lose.  Blocks of the same
// node also trade positions across chunks through the work list: an item that already
// holds a position above a block's chunk is not tested there at all.
//
// The entries reach shared memory as one 4-byte word each (the parent node ids, a byte
// apiece, in sorted-position order; `sset`), streamed by 1-D bulk (TMA) copies, so a
// full pass reads 4 B per (node, entry) -- as the mask-test scan does -- but tests 32
// items per shared-memory word instead of one.  The per-lane copies of the P words
// (each lane reads its own bank) keep the four loads free of bank conflicts.
//
// Two modes.  The full pass tests every entry of the table (Eq. (6) taken literally).
// The sorted mode (BN_SCAN_SORTED) stops early, with identical results: nothing past the
// empty set's sorted position can be chosen (the empty set is consistent with every
// order), a block stops streaming once each of its items has taken an entry (every
// entry still unread lies further down the list), and a block whose items all hold a
// position above its chunk already (from blocks of earlier chunks) does nothing.
#include <algorithm>

#include "bn_table.cuh"

namespace bn {

static constexpr int SL_CWARPS = 8;                 // consumer warps
static constexpr int SL_THREADS = 32 * (SL_CWARPS + 1);   // and one producer warp
static constexpr int SL_SUB = 2048;                 // entries per stage
static constexpr int SL_STAGES = 4;
static constexpr int SL_PER_WARP = SL_SUB / SL_CWARPS;  // 256 entries of a stage per consumer warp
static constexpr int SL_ROWS = 66;                  // nodes 0..63, "no parent" (64), "never" (65)
static constexpr int SL_ROW_BYTES = 256;            // two groups' 32 lanes per row
static constexpr uint32_t SL_ROW_ONES = 64;
static constexpr uint32_t SL_WORD_NEVER = 0x41414141u;  // four bytes of row 65 (all zero)
static constexpr int SL_MAX_K = 4;

// The P copies of up to four groups sit in static shared memory, whose address the
// compiler knows, so a byte-permute result addresses a row directly; eight groups do not
// fit the static limit and use the dynamic region.
__host__ __device__ constexpr bool sl_static_p(int G) { return G <= 4; }
__host__ __device__ constexpr size_t sl_p_bytes(int G) { return (size_t)((G + 1) / 2) * SL_ROWS * SL_ROW_BYTES; }
// dynamic shared memory of a block
__host__ __device__ constexpr size_t sl_smem(int G)
{
    return (size_t)SL_STAGES * SL_SUB * 4            // staged entry words
           + (sl_static_p(G) ? 0 : sl_p_bytes(G))    // per-lane copies of P[v][g]
           + (size_t)32 * G * 4                      // per-item best sorted position
           + 16 * SL_STAGES + 64;                    // full/empty mbarriers, flags, skip words
}


struct SlicedArgs {
    const uint32_t* sset;          // [n][Ssp] parent node ids of the entry at each sorted position
    const uint32_t* spos;          // [n][Sp] sorted position of each rank (rank 0 = empty set)
    int64_t Sp, S;
    int64_t Ssp;                   // sset row stride: S rounded up to whole stages
    int n;
    int64_t chunk;                 // entries per block (multiple of SL_SUB)
    int nchunk;
    const uint32_t* list_count;
    const uint64_t* list_pc;
    uint32_t* list_best;
    int cap;
    uint32_t* status;
};

// ---------------------------------------------------------------------------------
// sset[i][p]: byte j = the j-th smallest parent node id of the entry at sorted position
// p of node i (node space: candidate c is node c + (c >= i)), SL_ROW_ONES for j >= the
// set's size; positions at or past S (padding up to the row stride Ssp, a whole number of
// stages) hold SL_WORD_NEVER, which no order is consistent with.
// ---------------------------------------------------------------------------------
__global__ void k_sset(const uint32_t* __restrict__ srank, const uint64_t* __restrict__ pst, int n, int64_t S,
                       int64_t Sp, int64_t Ssp, uint32_t* __restrict__ sset)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * Ssp) return;
    const int i = (int)(g / Ssp);
    const int64_t p = g - (int64_t)i * Ssp;
    uint32_t w = SL_WORD_NEVER;
    if (p < S) {
        uint64_t m = pst[srank[(size_t)i * Sp + p]];
        w = 0;
        for (int j = 0; j < SL_MAX_K; ++j) {
            uint32_t v = SL_ROW_ONES;
            if (m) {
                const int c = __ffsll((long long)m) - 1;
                m &= m - 1;
                v = (uint32_t)(c + (c >= i));
            }
            w |= v << (8 * j);
        }
    }
    sset[g] = w;
}

int build_sset(bn_table* t, cudaStream_t s)
{
    if (t->k > SL_MAX_K || t->n > 64) return BN_OK;          // the mask-test scans serve these
    const int64_t Ssp = round_up(t->S, SL_SUB);
    if (!t->sset) {
        cudaError_t e = cudaMalloc(&t->sset, sizeof(uint32_t) * (size_t)t->n * (size_t)Ssp);
        if (e != cudaSuccess) {
            t->sset = nullptr;
            cudaGetLastError();
            return set_error(BN_ENOMEM, "sorted parent sets: %zu bytes: %s",
                             sizeof(uint32_t) * (size_t)t->n * (size_t)Ssp, cudaGetErrorString(e));
        }
        t->sset_stride = Ssp;
        t->bytes += sizeof(uint32_t) * (size_t)t->n * (size_t)Ssp;
    }
    const int64_t tot = (int64_t)t->n * Ssp;
    k_sset<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(t->srank, t->pst, t->n, t->S, t->Sp, Ssp, t->sset);
    BN_LAUNCH_CHECK("k_sset");
    // the empty set's sorted position per node, for the sorted mode's launch shape: ranks
    // 0 and 1 of every node are the first 2 n words of the entry-major copy spos_t
    uint32_t h[2 * 64];
    BN_CUDA(cudaMemcpyAsync(h, t->spos_t, sizeof(uint32_t) * 2 * (size_t)t->n, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < t->n; ++i) t->cut[i] = h[2 * i] + 1;
    return BN_OK;
}

// word index of P[v][g] for lane 0
__device__ __forceinline__ int Pw(int g, int v)
{
    return (g >> 1) * SL_ROWS * (SL_ROW_BYTES / 4) + v * (SL_ROW_BYTES / 4) + (g & 1) * 32;
}

// Block (chunk c, node i) = blockIdx.x = c * n + i, item set blockIdx.y: items
// 32 G y .. 32 G y + 32 G - 1 of node i.  Eight consumer warps and one producer warp:
// consumer warp w tests entries w * 256 .. w * 256 + 255 of every stage, 128 a step, so
// each warp walks its entries in increasing sorted position; the producer refills a stage
// as soon as every consumer has released it (an empty mbarrier per stage), so no
// consumer waits for a refill.
template <int G, bool CUT>
__global__ void __launch_bounds__(SL_THREADS) k_scan_sliced(SlicedArgs A)
{
    // one record per item and step (measured: faster everywhere but in the full pass over
    // eight groups, where hits are sparse and the prefix ORs cost more than the duplicates)
    constexpr bool DEDUP = CUT || G <= 4;
    // positions traded with the node's other chunks after each refill (measured: faster
    // but for the full pass over eight groups, whose short, load-bound stages the trade's
    // global round trip would hold back)
    constexpr bool TRADE = CUT || G <= 4;
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t* s_ent = (uint32_t*)smem;                                            // [STAGES][SUB]
    // P[v][g] for lane l at word (g / 2) * ROWS * 64 + v * 64 + (g % 2) * 32 + l: a row of
    // 256 bytes per node, so an entry's byte v and the lane's offset make the row address
    // in one byte permute
    __shared__ __align__(256) uint32_t s_Pst[sl_static_p(G) ? sl_p_bytes(G) / 4 : 1];
    uint32_t* s_P = sl_static_p(G) ? s_Pst : s_ent + SL_STAGES * SL_SUB;
    uint32_t* s_best = s_ent + SL_STAGES * SL_SUB + (sl_static_p(G) ? 0 : sl_p_bytes(G) / 4);   // [32 G]
    uint64_t* bar = (uint64_t*)(s_best + 32 * G);                                 // full, per stage
    uint64_t* ebar = bar + SL_STAGES;                                             // empty, per stage
    int* s_flags = (int*)(ebar + SL_STAGES);                                      // abort, last, nrec
    uint32_t* s_skip = (uint32_t*)(s_flags + 4);                                  // [G]

    const int node = blockIdx.x % A.n;
    const int chunk = blockIdx.x / A.n;
    const int cnt = (int)A.list_count[node];
    const int g0 = blockIdx.y * 32 * G;
    if (g0 >= cnt) return;                                                        // block-uniform
    const int64_t e0 = (int64_t)chunk * A.chunk;
    int64_t e1 = min(e0 + A.chunk, A.S);
    if (CUT) e1 = min(e1, (int64_t)A.spos[(size_t)node * A.Sp] + 1);              // the empty set's position
    if (e0 >= e1) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvalid = min(cnt - g0, 32 * G);
    const int nsub = (int)((e1 - e0 + SL_SUB - 1) / SL_SUB);
    const bool producer = warp == SL_CWARPS;
    const uint32_t* src = A.sset + (size_t)node * A.Ssp;
    uint64_t pol_stream = 0;
    // the producer stages `it` into buffer st: always a whole stage (the row stride Ssp is
    // a whole number of stages).  Words past S are SL_WORD_NEVER; in the sorted mode the
    // last stage may run past the empty set's position, and those entries cannot win
    // (the empty set, in the same stage, is consistent with every item and ranks above
    // them), so no lane needs a bounds test.
    auto issue = [&](int it, int st) {
        const int64_t base = e0 + (int64_t)it * SL_SUB;
        mbar_arrive_expect_tx(&bar[st], SL_SUB * 4u);
        bulk_g2s(s_ent + st * SL_SUB, src + base, SL_SUB * 4u, &bar[st], pol_stream);
    };

    if (producer) {
        // Items this block need not test: in the sorted mode those holding a position above
        // this chunk already (from blocks of earlier chunks).  The producer decides for
        // every warp, so all skip the same items and the count of items holding a position
        // stays exact.  Then the first copies go out while the consumers set up.
        int pre = 0;
        if (CUT) {
            for (int g = 0; g < G; ++g) {
                const int item = g0 + 32 * g + lane;
                const bool done = item < cnt && *(volatile const uint32_t*)&A.list_best[(size_t)node * A.cap + item] <
                                                    (uint32_t)e0;
                const uint32_t d = __ballot_sync(0xffffffffu, done);
                if (lane == 0) s_skip[g] = d;
                pre += __popc(d);
            }
        } else if (lane < G) {
            s_skip[lane] = 0;
        }
        if (lane == 0) {
            s_flags[0] = 0;                                                       // abort
            s_flags[1] = 0x7fffffff;                                              // first stage never issued
            s_flags[2] = pre;                                                     // items holding a position
            pol_stream = l2_policy_evict_first();
            for (int s = 0; s < SL_STAGES; ++s) {
                mbar_init(&bar[s], 1);
                mbar_init(&ebar[s], SL_CWARPS);
            }
            fence_mbar_init();
            if (!(CUT && pre == nvalid))
                for (int it = 0; it < SL_STAGES && it < nsub; ++it) issue(it, it);
        }
    } else {
        // the items' predecessor words: warp g builds group g (rows 0..63 from ballots of
        // the 32 items' masks, row 64 all ones, row 65 zero)
        if (warp < G) {
            const int item = g0 + warp * 32 + lane;
            const uint64_t pc = item < cnt ? A.list_pc[(size_t)node * A.cap + item] : 0ull;
            for (int v = 0; v < 64; ++v) {
                const int c = v - (v > node);
                const bool bit = v < A.n && v != node && ((pc >> c) & 1ull);
                const uint32_t word = __ballot_sync(0xffffffffu, bit);
                s_P[Pw(warp, v) + lane] = word;
            }
            s_P[Pw(warp, 64) + lane] = 0xffffffffu;
            s_P[Pw(warp, 65) + lane] = 0u;
        }
        for (int j = threadIdx.x; j < 32 * G; j += 32 * SL_CWARPS) s_best[j] = SPOS_NONE;
    }
    __syncthreads();
    if (CUT && s_flags[2] == nvalid) return;                                      // block-uniform; nothing issued

    if (producer && !TRADE) {
        // lane 0 alone refills each stage once every consumer has released it
        if (lane == 0) {
            int issued = min(SL_STAGES, nsub);
            for (int it = 0; it + SL_STAGES < nsub; ++it) {
                const int st = it % SL_STAGES;
                if (*(volatile int*)&s_flags[0]) break;
                if (!mbar_wait_bounded(&ebar[st], (uint32_t)((it / SL_STAGES) & 1), WAIT_TIMEOUT_NS)) {
                    *(volatile int*)&s_flags[0] = 1;
                    atomicOr(A.status, STATUS_TIMEOUT);
                    break;
                }
                issue(it + SL_STAGES, st);
                issued = it + SL_STAGES + 1;
            }
            // no copy may still be in flight when the block's shared memory goes away
            for (int j = max(0, issued - SL_STAGES); j < issued; ++j)
                mbar_wait_bounded(&bar[j % SL_STAGES], (uint32_t)((j / SL_STAGES) & 1), WAIT_TIMEOUT_NS);
        }
    } else if (producer) {
        // Lane 0 refills each stage once every consumer has released it.  Then, while the
        // copy is in flight, the whole warp trades positions with the blocks of the node's
        // other chunks: it publishes this block's new positions (atomicMin) and marks as
        // skipped every item that already holds a position above this chunk -- no entry
        // of the chunk can win for it, so the consumers stop testing it (they still read
        // every entry).
        int issued = min(SL_STAGES, nsub);
        uint32_t pub[G], known[G];         // last published position; items already skipped
#pragma unroll
        for (int g = 0; g < G; ++g) {
            pub[g] = SPOS_NONE;
            known[g] = s_skip[g];          // (the sorted mode's items skipped at the start are
        }                                  // counted already)
        for (int it = 0; it + SL_STAGES < nsub; ++it) {
            const int st = it % SL_STAGES;
            int go = 1;
            if (lane == 0) {
                if (*(volatile int*)&s_flags[0]) {
                    go = 0;
                } else if (!mbar_wait_bounded(&ebar[st], (uint32_t)((it / SL_STAGES) & 1), WAIT_TIMEOUT_NS)) {
                    *(volatile int*)&s_flags[0] = 1;
                    atomicOr(A.status, STATUS_TIMEOUT);
                    go = 0;
                } else if (CUT && *(volatile int*)&s_flags[2] >= nvalid) {
                    // every item holds a position: no unread entry can win; release the
                    // consumers of this buffer's next phase without a copy
                    *(volatile int*)&s_flags[1] = it + SL_STAGES;
                    mbar_arrive(&bar[st]);
                    issued = it + SL_STAGES + 1;
                    go = 0;
                } else {
                    issue(it + SL_STAGES, st);
                    issued = it + SL_STAGES + 1;
                }
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) break;
            // every load first (one round trip for all groups), then the updates
            uint32_t mine[G], other[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int item = g0 + 32 * g + lane;
                const bool live = item < cnt && !((known[g] >> lane) & 1u);
                mine[g] = live ? *(volatile const uint32_t*)&s_best[g * 32 + lane] : SPOS_NONE;
                other[g] = live ? *(volatile const uint32_t*)&A.list_best[(size_t)node * A.cap + item] : SPOS_NONE;
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int item = g0 + 32 * g + lane;
                if (mine[g] < pub[g] && mine[g] < other[g]) {
                    atomicMin(&A.list_best[(size_t)node * A.cap + item], mine[g]);
                    pub[g] = mine[g];
                }
                const bool sk = other[g] < (uint32_t)e0;
                // in the sorted mode the item now holds a position (for the stop)
                if (CUT && sk && atomicMin(&s_best[g * 32 + lane], other[g]) == SPOS_NONE) atomicAdd(&s_flags[2], 1);
                const uint32_t bits = __ballot_sync(0xffffffffu, sk);
                known[g] |= bits;
                if (lane == 0 && bits) *(volatile uint32_t*)&s_skip[g] |= bits;
            }
        }
        if (lane == 0) {
            // no copy may still be in flight when the block's shared memory goes away
            for (int j = max(0, issued - SL_STAGES); j < issued; ++j)
                mbar_wait_bounded(&bar[j % SL_STAGES], (uint32_t)((j / SL_STAGES) & 1), WAIT_TIMEOUT_NS);
        }
    } else {
        uint32_t found[G];                 // items of group g this warp no longer tests
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int nv = min(max(cnt - g0 - 32 * g, 0), 32);
            found[g] = nv >= 32 ? 0u : (0xffffffffu << nv);
            found[g] |= s_skip[g];
        }
        const uint32_t lane4 = (uint32_t)lane * 4u;
        const uint8_t* Pb = (const uint8_t*)s_P;
        for (int it = 0; it < nsub; ++it) {
            const int st = it % SL_STAGES;
            const uint32_t parity = (uint32_t)((it / SL_STAGES) & 1);
            if (__shfl_sync(0xffffffffu, *(volatile int*)&s_flags[0], 0)) break;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], parity, WAIT_TIMEOUT_NS))) {
                if (lane == 0) {
                    *(volatile int*)&s_flags[0] = 1;
                    atomicOr(A.status, STATUS_TIMEOUT);
                }
                break;
            }
            if (CUT && it >= __shfl_sync(0xffffffffu, *(volatile int*)&s_flags[1], 0)) break;
            const int64_t base = e0 + (int64_t)it * SL_SUB + warp * SL_PER_WARP;
            const uint4* E4 = (const uint4*)(s_ent + st * SL_SUB + warp * SL_PER_WARP);
            uint32_t all_found = 0xffffffffu;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if constexpr (TRADE) found[g] |= *(volatile const uint32_t*)&s_skip[g];
                all_found &= found[g];
            }
            if (all_found != 0xffffffffu) {
                // a step: 128 entries, four consecutive ones a lane (one 16-byte load); one
                // warp vote per step, then one warp-wide OR per group marks the step's new
                // items found (two records of an item in one step: the atomicMin keeps the
                // earlier position)
#pragma unroll 1
                for (int q = 0; q < SL_PER_WARP / 128; ++q) {
                    const uint4 w4 = E4[q * 32 + lane];
                    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
                    // byte 1 = the parent's node id, byte 0 = this lane's offset: the byte
                    // address of P[v][g] minus the group's constant part
                    auto word = [&](uint32_t wu, uint32_t sel, int g) {
                        return *(const uint32_t*)(Pb + 4 * Pw(g, 0) + __byte_perm(wu, lane4, sel));
                    };
                    uint32_t raw[G];
#pragma unroll
                    for (int g = 0; g < G; ++g) raw[g] = 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            raw[g] |= word(w[u], 0x5504, g) & word(w[u], 0x5514, g) & word(w[u], 0x5524, g) &
                                      word(w[u], 0x5534, g);
                    }
                    uint32_t any = 0;
#pragma unroll
                    for (int g = 0; g < G; ++g) any |= raw[g] & ~found[g];
                    if (__any_sync(0xffffffffu, any != 0)) {
                        const uint32_t pos0 = (uint32_t)(base + q * 128 + 4 * lane);
                        if constexpr (DEDUP) {
                            // rare: record the step's new items.  Positions run lane-major
                            // (lane l holds pos0 .. pos0 + 3), so of the lanes hitting an
                            // item only the lowest records it (an exclusive prefix OR over
                            // the lanes), at its first entry that hits: one atomicMin per
                            // item and step, however densely the top of a node's list
                            // matches the orders
#pragma unroll
                            for (int g = 0; g < G; ++g) {
                                const uint32_t hit = raw[g] & ~found[g];
                                uint32_t incl = hit;
#pragma unroll
                                for (int d = 1; d < 32; d <<= 1) {
                                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                                    if (lane >= d) incl |= y;
                                }
                                const uint32_t before = __shfl_up_sync(0xffffffffu, incl, 1);   // lanes below
                                uint32_t mine = lane == 0 ? hit : hit & ~before;
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    if (!mine) break;
                                    uint32_t m = word(w[u], 0x5504, g) & word(w[u], 0x5514, g) &
                                                 word(w[u], 0x5524, g) & word(w[u], 0x5534, g) & mine;
                                    mine &= ~m;
                                    while (m) {
                                        const int b = __ffs(m) - 1;
                                        m &= m - 1;
                                        const uint32_t old = atomicMin(&s_best[g * 32 + b], pos0 + u);
                                        if (CUT && old == SPOS_NONE) atomicAdd(&s_flags[2], 1);
                                    }
                                }
                                found[g] |= __shfl_sync(0xffffffffu, incl, 31);
                            }
                        } else {
                            // every lane records its own new items (duplicates of one step
                            // lose the atomicMin); cheaper where hits are sparse
#pragma unroll
                            for (int g = 0; g < G; ++g) {
                                const uint32_t hit = raw[g] & ~found[g];
                                if (hit) {
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        uint32_t m = word(w[u], 0x5504, g) & word(w[u], 0x5514, g) &
                                                     word(w[u], 0x5524, g) & word(w[u], 0x5534, g) & hit;
                                        while (m) {
                                            const int b = __ffs(m) - 1;
                                            m &= m - 1;
                                            const uint32_t old = atomicMin(&s_best[g * 32 + b], pos0 + u);
                                            if (CUT && old == SPOS_NONE) atomicAdd(&s_flags[2], 1);
                                        }
                                    }
                                }
                                found[g] |= __reduce_or_sync(0xffffffffu, hit);
                            }
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ebar[st]);
        }
    }
    __syncthreads();
    if (s_flags[0]) return;                                                       // block-uniform
    for (int j = threadIdx.x; j < nvalid; j += SL_THREADS) {
        const uint32_t b = s_best[j];
        if (b != SPOS_NONE) atomicMin(&A.list_best[(size_t)node * A.cap + g0 + j], b);
    }
}

// Launch shape: as many blocks as are resident at once (the occupancy calculator: threads,
// registers and shared memory), one wave of long blocks, so each block's set-up is paid
// once; the sorted mode spreads its chunks (at least four stages each) over the nodes'
// live ranges [0, cut), and the blocks past a node's cut leave at once.
template <int G, bool CUT>
static int sliced_launch(const bn_table* t, const uint32_t* list_count, const uint64_t* list_pc,
                         uint32_t* list_best, int cap, int sets, uint32_t* status, cudaStream_t s)
{
    static unsigned long long ctx[64] = {0};
    static int resident[64] = {0};
    const int d = device_id();
    if (first_in_context(ctx)) {
        BN_CUDA(cudaFuncSetAttribute(k_scan_sliced<G, CUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sl_smem(G)));
        int nb = 0;
        BN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_scan_sliced<G, CUT>, SL_THREADS, sl_smem(G)));
        if (d >= 0 && d < 64) resident[d] = std::max(1, nb);
    }
    const int per_sm = (d >= 0 && d < 64 && resident[d] > 0) ? resident[d] : 1;
    const int64_t want = (int64_t)sm_count() * per_sm;
    int64_t chunk, nchunk;
    if (!CUT) {
        nchunk = std::max<int64_t>(1, want / ((int64_t)t->n * sets));
        chunk = round_up((t->S + nchunk - 1) / nchunk, SL_SUB);
        nchunk = (t->S + chunk - 1) / chunk;
    } else {
        int64_t live = 0, longest = 0;
        for (int i = 0; i < t->n; ++i) {
            live += t->cut[i];
            longest = std::max<int64_t>(longest, t->cut[i]);
        }
        chunk = std::max<int64_t>(4 * SL_SUB, round_up((live * sets + want - 1) / want, SL_SUB));
        nchunk = (longest + chunk - 1) / chunk;
    }
    SlicedArgs A{t->sset, t->spos, t->Sp, t->S, t->sset_stride, t->n, chunk, (int)nchunk, list_count, list_pc,
                 list_best, cap, status};
    dim3 grid((unsigned)(nchunk * t->n), (unsigned)sets);
    k_scan_sliced<G, CUT><<<grid, SL_THREADS, sl_smem(G), s>>>(A);
    BN_LAUNCH_CHECK("k_scan_sliced");
    return BN_OK;
}

int launch_scan_sliced(const bn_table* t, const uint32_t* list_count, const uint64_t* list_pc, uint32_t* list_best,
                       int cap, bool cut, uint32_t* status, cudaStream_t s)
{
    if (!t->sset) return set_error(BN_EUNSUPPORTED, "sliced scan: needs k <= 4 (k = %d)", t->k);
    if (cap < 1) return BN_OK;
    const int per = std::min(cap, 256);
    const int G = per <= 32 ? 1 : (per <= 64 ? 2 : (per <= 128 ? 4 : 8));
    const int sets = (cap + 32 * G - 1) / (32 * G);
    if (sets > 65535) return set_error(BN_EUNSUPPORTED, "sliced scan: %d items per node (at most %d)", cap, 65535 * 256);
#define BN_SL(GG)                                                                                               \
    return cut ? sliced_launch<GG, true>(t, list_count, list_pc, list_best, cap, sets, status, s)               \
               : sliced_launch<GG, false>(t, list_count, list_pc, list_best, cap, sets, status, s)
    switch (G) {
        case 1: BN_SL(1);
        case 2: BN_SL(2);
        case 4: BN_SL(4);
        default: BN_SL(8);
    }
#undef BN_SL
}

}  // namespace bn
