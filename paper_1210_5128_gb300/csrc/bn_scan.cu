// bn_scan.cu -- the order score of Eq. (6) (scoring loop of Algorithm 1).
//
// For node i and an order, the best entry is the maximum of entry(i, rho) over the ranks
// rho whose parent set lies inside the node's predecessors, ties to the lowest rank.
// With every entry's sorted position spos (score descending, rank ascending; unique per
// node) that is the entry of minimum spos among the consistent ones.
//
// The paper assigns h blocks per node and splits one order's consistent sets over their
// threads (Sec. V.B), then reduces an argmax in shared memory.  Here a block owns a
// contiguous chunk of one node's table and up to 256 (order, node) work items, one per
// thread.  The chunk's spos values and parent-set masks are streamed once into shared
// memory by 1-D bulk (TMA) copies; every thread tests each staged entry's candidate mask
// against its item's predecessor mask and keeps a running min of spos.  So the table is
// read once per 256 orders instead of once per order, and a test is a 64-bit AND-NOT,
// a zero test and one unsigned min.  When a block holds fewer than 256 items, its spare
// warps take a share of the entries of the same items, and below 32 items the lanes of a
// warp split each item's entries as well (so a batch of a few orders streams the table at
// memory speed instead of one active lane per warp).  Chunks combine with atomicMin.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "bn_table.cuh"

namespace bn {

// best = min(best, sp) if (m & npc) == 0, npc = (nhi:nlo): the two halves ANDed and ORed
// by two three-input logic ops, the zero test on that word, a predicated min
__device__ __forceinline__ void test_min(uint32_t& best, uint32_t mlo, uint32_t mhi, uint32_t nlo, uint32_t nhi,
                                         uint32_t sp)
{
    asm("{\n\t.reg .pred p;\n\t.reg .b32 t, u;\n\t"
        "lop3.b32 t, %1, %3, 0, 0xC0;\n\t"
        "lop3.b32 u, %2, %4, t, 0xEA;\n\t"
        "setp.eq.u32 p, u, 0;\n\t"
        "@p min.u32 %0, %0, %5;\n\t}"
        : "+r"(best)
        : "r"(mlo), "r"(mhi), "r"(nlo), "r"(nhi), "r"(sp));
}

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_WARPS = SCAN_THREADS / 32;
// stage size (entries) and pipeline depth; 48 KB of shared memory for the 1024 and 512
// variants, 72 KB for 2048
template <int SUB>
struct ScanCfg {
    static constexpr int STAGES = SUB >= 2048 ? 3 : (SUB >= 1024 ? 4 : 8);
    // stages, then a full and an empty mbarrier per stage
    static constexpr size_t SMEM = (size_t)STAGES * SUB * (sizeof(uint32_t) + sizeof(uint64_t)) + 16 * STAGES;
};

struct ScanArgs {
    const uint32_t* spos;
    const uint64_t* pst;
    int64_t Sp;
    int64_t S;             // parent sets per node (entries at or past S are padding)
    int N, k;              // candidates per node (n - 1) and the size limit
    int nchunk;
    int64_t chunk;
    const uint32_t* list_count;
    const uint64_t* list_pc;
    uint32_t* list_best;
    int cap;
    uint32_t* status;
};

static ScanPlan plan_for(const bn_table* t, int groups, int64_t target, int sub)
{
    ScanPlan p;
    p.sub = sub;
    const int64_t units = t->Sp / SUBQ;
    // whole waves: at most `target` blocks
    int64_t nchunk = target / ((int64_t)t->n * groups);
    nchunk = std::max<int64_t>(1, std::min<int64_t>(nchunk, units));
    const int64_t chunk = round_up((t->Sp + nchunk - 1) / nchunk, SUBQ);
    p.chunk = chunk;
    p.nchunk = (int)((t->Sp + chunk - 1) / chunk);
    return p;
}

ScanPlan plan_scan(const bn_table* t, int max_items)
{
    const int groups = std::max(1, (max_items + SCAN_THREADS - 1) / SCAN_THREADS);
    if (groups <= 8 && t->tuned_sub[groups]) {
        ScanPlan p;
        p.sub = t->tuned_sub[groups];
        p.nchunk = t->tuned_nchunk[groups];
        p.chunk = t->tuned_chunk[groups];
        return p;
    }
    // four blocks per SM: one wave for a few items per node (the scan streams the table at
    // memory speed, and a second, partial wave would idle most SMs), else two
    const int waves = max_items <= 32 ? 1 : 2;
    return plan_for(t, groups, (int64_t)sm_count() * 4 * waves, 1024);
}

template <int SCAN_SUB, bool UNRANK>
__device__ __forceinline__ void scan_issue(const ScanArgs& A, int node, int64_t base, int64_t e1, uint32_t* s_sp,
                                           uint64_t* s_msk, uint64_t* bar, uint64_t pol_stream, uint64_t pol_keep)
{
    const uint32_t cnt = (uint32_t)min((int64_t)SCAN_SUB, e1 - base);
    mbar_arrive_expect_tx(bar, cnt * (UNRANK ? 4u : 12u));
    bulk_g2s(s_sp, A.spos + (size_t)node * A.Sp + base, cnt * 4u, bar, pol_stream);
    if (!UNRANK) bulk_g2s(s_msk, A.pst + base, cnt * 8u, bar, pol_keep);
}

// ---------------------------------------------------------------------------------
// Parent sets computed instead of read (the paper's first strategy, Sec. V.B, against
// the table of its second): the candidate-space mask of rank r in the size-ascending
// combinatorial number system, and the next rank's from the previous one.
// bin[c * (k + 1) + t] = C(c, t), c <= 64, t <= k.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t unrank_set(uint64_t r, int N, int k, const uint64_t* bin, int& size)
{
    int j = 0;
    while (j <= k && r >= bin[N * (k + 1) + j]) {
        r -= bin[N * (k + 1) + j];
        ++j;
    }
    size = j;
    if (j > k) return ~0ull;                              // padding
    uint64_t m = 0;
    int hi = N - 1;
    for (int t = j; t >= 1; --t) {                        // largest element first
        int lo = t - 1, h = hi;
        while (lo < h) {
            const int mid = (lo + h + 1) >> 1;
            if (bin[mid * (k + 1) + t] <= r) lo = mid;
            else h = mid - 1;
        }
        m |= 1ull << lo;
        r -= bin[lo * (k + 1) + t];
        hi = lo - 1;
    }
    return m;
}

// the set after m in rank order: the next set of the same size in colex order (the next
// larger mask with as many bits, Gosper's construction), else the first set one larger
__device__ __forceinline__ uint64_t next_set(uint64_t m, int N, int k, int& size)
{
    if (size > k) return ~0ull;
    uint64_t nm = 0;
    bool roll = true;
    if (size > 0) {
        const uint64_t c = m & (~m + 1ull);
        const uint64_t r = m + c;
        nm = (((r ^ m) >> 2) >> (__ffsll((long long)c) - 1)) | r;
        roll = (r == 0ull) || (N < 64 && (nm >> N) != 0ull);
    }
    if (roll) {
        ++size;
        if (size > k) return ~0ull;
        nm = (size >= 64) ? ~0ull : ((1ull << size) - 1ull);
    }
    return nm;
}

template <int SCAN_SUB, bool UNRANK>
__global__ void __launch_bounds__(SCAN_THREADS, 4) k_scan(ScanArgs A)
{
    constexpr int SCAN_STAGES = ScanCfg<SCAN_SUB>::STAGES;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* s_msk = (uint64_t*)smem;                                          // [STAGES][SUB]
    uint32_t* s_sp = (uint32_t*)(smem + sizeof(uint64_t) * SCAN_STAGES * SCAN_SUB);
    uint64_t* bar = (uint64_t*)(smem + (sizeof(uint64_t) + sizeof(uint32_t)) * SCAN_STAGES * SCAN_SUB);
    uint64_t* ebar = bar + SCAN_STAGES;                                         // stage consumed by every warp
    uint64_t* s_bin = ebar + SCAN_STAGES;                                       // C(c, t) (UNRANK)

    const int node = blockIdx.x / A.nchunk;
    const int chunk = blockIdx.x - node * A.nchunk;
    const int cnt = (int)A.list_count[node];
    const int g0 = blockIdx.y * SCAN_THREADS;
    if (g0 >= cnt) return;                                                      // block-uniform
    const int64_t e0 = (int64_t)chunk * A.chunk;
    const int64_t e1 = min(e0 + A.chunk, A.Sp);
    if (e0 >= e1) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // G warps' worth of items; the spare warps split the entries of the same items.  With
    // fewer than 32 items a warp holds all of them, LPI lanes per item, and the LPI lanes
    // of an item split its entries too.
    const int here = min(SCAN_THREADS, cnt - g0);
    const int ipw = here >= 32 ? 32 : (here <= 1 ? 1 : 1 << (32 - __clz(here - 1)));   // items per warp
    const int LPI = 32 / ipw;                                                          // lanes per item
    const int G = (here + ipw - 1) / ipw;
    const int split = SCAN_WARPS / G;
    const int ig = warp % G, sp = warp / G;
    const bool warp_on = sp < split;
    const int item = g0 + ig * ipw + lane / LPI;
    const int sub = lane % LPI;
    const bool active = warp_on && item < cnt;
    const uint64_t npc = active ? ~A.list_pc[(size_t)node * A.cap + item] : ~0ull;
    const uint32_t nlo = (uint32_t)npc, nhi = (uint32_t)(npc >> 32);
    const int nsub = (int)((e1 - e0 + SCAN_SUB - 1) / SCAN_SUB);

    uint64_t pol_stream = 0, pol_keep = 0;
    if (threadIdx.x == 0) {
        pol_stream = l2_policy_evict_first();
        pol_keep = l2_policy_evict_last();
        for (int s = 0; s < SCAN_STAGES; ++s) {
            mbar_init(&bar[s], 1);
            mbar_init(&ebar[s], SCAN_WARPS);
        }
        fence_mbar_init();
    }
    if (UNRANK)
        for (int q = threadIdx.x; q < 65 * (A.k + 1); q += SCAN_THREADS)
            s_bin[q] = c_binom.v[q / (A.k + 1)][q % (A.k + 1)];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < SCAN_STAGES && s < nsub; ++s)
            scan_issue<SCAN_SUB, UNRANK>(A, node, e0 + (int64_t)s * SCAN_SUB, e1, s_sp + s * SCAN_SUB, s_msk + s * SCAN_SUB, &bar[s],
                       pol_stream, pol_keep);
    }

    uint32_t b0 = SPOS_NONE, b1 = SPOS_NONE;
    if constexpr (!UNRANK) {
        // Warps run decoupled: each waits for a stage to land (full barrier), tests it,
        // and releases it (empty barrier, one arrival per warp); thread 0 re-fills a stage
        // once every warp has released it, SCAN_STAGES stages ahead of its own position.
        // A wait that runs out sets s_abort, and every warp leaves at its next stage.
        __shared__ int s_abort;
        if (threadIdx.x == 0) s_abort = 0;
        __syncthreads();
        int issued = min(nsub, SCAN_STAGES);
        for (int it = 0; it < nsub; ++it) {
            const int st = it % SCAN_STAGES;
            const uint32_t parity = (uint32_t)((it / SCAN_STAGES) & 1);
            // warp-uniform decisions: lane 0's view of the abort flag, all lanes' waits
            if (__shfl_sync(0xffffffffu, *(volatile int*)&s_abort, 0)) break;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], parity, WAIT_TIMEOUT_NS))) {
                if (lane == 0) {
                    *(volatile int*)&s_abort = 1;
                    atomicOr(A.status, STATUS_TIMEOUT);
                }
                break;
            }
            if (warp_on) {
                const int64_t base = e0 + (int64_t)it * SCAN_SUB;
                const int pairs = (int)min((int64_t)SCAN_SUB, e1 - base) >> 1;
                const uint2* P = (const uint2*)(s_sp + st * SCAN_SUB);
                const ulonglong2* M = (const ulonglong2*)(s_msk + st * SCAN_SUB);
#pragma unroll 32
                for (int j = sp * LPI + sub; j < pairs; j += split * LPI) {
                    const uint2 pp = P[j];
                    const uint4 mm = ((const uint4*)M)[j];
                    test_min(b0, mm.x, mm.y, nlo, nhi, pp.x);
                    test_min(b1, mm.z, mm.w, nlo, nhi, pp.y);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ebar[st]);
            if (threadIdx.x == 0 && it + SCAN_STAGES < nsub) {
                // (on a timeout no break here: warp 0 leaves together at the next check)
                if (!mbar_wait_bounded(&ebar[st], parity, WAIT_TIMEOUT_NS)) {
                    *(volatile int*)&s_abort = 1;
                    atomicOr(A.status, STATUS_TIMEOUT);
                } else {
                    const int64_t nb = e0 + (int64_t)(it + SCAN_STAGES) * SCAN_SUB;
                    scan_issue<SCAN_SUB, UNRANK>(A, node, nb, e1, s_sp + st * SCAN_SUB, s_msk + st * SCAN_SUB,
                                                 &bar[st], pol_stream, pol_keep);
                    issued = it + SCAN_STAGES + 1;
                }
            }
        }
        if (threadIdx.x == 0) {
            // no copy may still be in flight when the block's shared memory goes away
            for (int j = max(0, issued - SCAN_STAGES); j < issued; ++j)
                mbar_wait_bounded(&bar[j % SCAN_STAGES], (uint32_t)((j / SCAN_STAGES) & 1), WAIT_TIMEOUT_NS);
        }
        __syncthreads();
        if (s_abort) return;                                        // block-uniform after the barrier
    } else {
        int it = 0;
        bool timed_out = false;
        for (; it < nsub; ++it) {
            const int st = it % SCAN_STAGES;
            const uint32_t parity = (uint32_t)((it / SCAN_STAGES) & 1);
            if (UNRANK) {
                // this stage's masks: every thread a run of SUB / 256 consecutive ranks
                constexpr int PER = SCAN_SUB / SCAN_THREADS;
                const int64_t base = e0 + (int64_t)it * SCAN_SUB;
                const int64_t r0 = base + (int64_t)threadIdx.x * PER;
                uint64_t* dst = s_msk + st * SCAN_SUB + threadIdx.x * PER;
                if (r0 < e1) {
                    int size = 0;
                    uint64_t m = r0 < A.S ? unrank_set((uint64_t)r0, A.N, A.k, s_bin, size) : ~0ull;
                    if (r0 >= A.S) size = A.k + 1;
                    dst[0] = m;
    #pragma unroll
                    for (int q = 1; q < PER; ++q) {
                        m = next_set(m, A.N, A.k, size);
                        dst[q] = m;
                    }
                }
                __syncthreads();
            }
            const bool ok = mbar_wait_bounded(&bar[st], parity, WAIT_TIMEOUT_NS);
            if (ok && warp_on) {
                const int64_t base = e0 + (int64_t)it * SCAN_SUB;
                const int pairs = (int)min((int64_t)SCAN_SUB, e1 - base) >> 1;
                const uint2* P = (const uint2*)(s_sp + st * SCAN_SUB);
                const ulonglong2* M = (const ulonglong2*)(s_msk + st * SCAN_SUB);
    #pragma unroll 32
                for (int j = sp * LPI + sub; j < pairs; j += split * LPI) {
                    const uint2 pp = P[j];
                    const uint4 mm = ((const uint4*)M)[j];
                    test_min(b0, mm.x, mm.y, nlo, nhi, pp.x);
                    test_min(b1, mm.z, mm.w, nlo, nhi, pp.y);
                }
            }
            if (__syncthreads_or(!ok)) { timed_out = true; break; }
            if (threadIdx.x == 0 && it + SCAN_STAGES < nsub) {
                const int64_t base = e0 + (int64_t)(it + SCAN_STAGES) * SCAN_SUB;
                scan_issue<SCAN_SUB, UNRANK>(A, node, base, e1, s_sp + st * SCAN_SUB, s_msk + st * SCAN_SUB, &bar[st],
                                             pol_stream, pol_keep);
            }
        }
        if (timed_out) {
            if (threadIdx.x == 0) {
                atomicOr(A.status, STATUS_TIMEOUT);
                // let copies already in flight land before the CTA's shared memory goes away
                for (int j = it; j < nsub && j < it + SCAN_STAGES; ++j)
                    mbar_wait_bounded(&bar[j % SCAN_STAGES], (uint32_t)((j / SCAN_STAGES) & 1), WAIT_TIMEOUT_NS);
            }
            return;
        }
    }
    uint32_t b = min(b0, b1);
    for (int off = 1; off < LPI; off <<= 1) b = min(b, __shfl_xor_sync(0xffffffffu, b, off));
    if (active && sub == 0 && b != SPOS_NONE) atomicMin(&A.list_best[(size_t)node * A.cap + item], b);
}

static constexpr size_t SCAN_BIN_BYTES = 8 * 65 * (MAXK + 1);   // binomial table (UNRANK)

template <int SUB, bool UNRANK>
static int scan_variant(const ScanArgs& A, dim3 grid, cudaStream_t s)
{
    static unsigned long long ctx[64] = {0};
    const size_t smem = ScanCfg<SUB>::SMEM + (UNRANK ? SCAN_BIN_BYTES : 0);
    if (first_in_context(ctx))
        BN_CUDA(cudaFuncSetAttribute(k_scan<SUB, UNRANK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_scan<SUB, UNRANK><<<grid, SCAN_THREADS, smem, s>>>(A);
    BN_LAUNCH_CHECK("k_scan");
    return BN_OK;
}

int launch_scan(const bn_table* t, const ScanPlan& pl, const uint32_t* list_count, const uint64_t* list_pc,
                uint32_t* list_best, int cap, uint32_t* status, cudaStream_t s)
{
    if (t->scan_mode == BN_SCAN_PRUNED) return launch_scan_pruned(t, list_count, list_pc, list_best, cap, s);
    if (t->scan_mode == BN_SCAN_SLICED || t->scan_mode == BN_SCAN_SORTED)
        return launch_scan_sliced(t, list_count, list_pc, list_best, cap, t->scan_mode == BN_SCAN_SORTED, status, s);
    ScanArgs A;
    A.spos = t->spos;
    A.pst = t->pst;
    A.Sp = t->Sp;
    A.S = t->S;
    A.N = t->n - 1;
    A.k = t->k;
    A.nchunk = pl.nchunk;
    A.chunk = pl.chunk;
    A.list_count = list_count;
    A.list_pc = list_pc;
    A.list_best = list_best;
    A.cap = cap;
    A.status = status;
    dim3 grid((unsigned)(t->n * pl.nchunk), (unsigned)((cap + SCAN_THREADS - 1) / SCAN_THREADS));
    const bool unrank = t->scan_mode == BN_SCAN_UNRANK;
    if (pl.sub >= 2048) return unrank ? scan_variant<2048, true>(A, grid, s) : scan_variant<2048, false>(A, grid, s);
    if (pl.sub >= 1024) return unrank ? scan_variant<1024, true>(A, grid, s) : scan_variant<1024, false>(A, grid, s);
    return unrank ? scan_variant<512, true>(A, grid, s) : scan_variant<512, false>(A, grid, s);
}

// ---------------------------------------------------------------------------------
// Up to 1,024 (node, order group) items (bn_score_orders; order groups of up to eight
// orders): a block owns a slice of the rank range for all nodes and orders, so the
// shared candidate-mask table is read once per slice instead of once per node, and the
// slice's sorted positions of all nodes come from the entry-major copy spos_t as one
// contiguous bulk copy per stage.  spos_t keeps the two positions of ranks 2j and 2j + 1
// of node i side by side ([Sp / 2][n][2]), so a thread takes an entry pair's two masks by
// one 16-byte and its node's two positions by one 8-byte shared-memory load, and tests
// them against the R orders of its group held in registers.
// ---------------------------------------------------------------------------------
static constexpr int NS_SUB = 128;             // entries per stage
static constexpr int NS_STAGES = 3;
static constexpr int NS_RMAX = 8;              // orders per thread
static constexpr int NS_MAX_ITEMS = 1024;      // (node, order group) items: one thread each

__host__ __device__ constexpr size_t ns_stage_bytes(int n) { return (size_t)NS_SUB * 8 + (size_t)n * NS_SUB * 4; }
__host__ __device__ constexpr size_t ns_smem(int n) { return NS_STAGES * ns_stage_bytes(n) + 8 * NS_STAGES; }

struct NodeScanArgs {
    const uint32_t* spos_t;        // [Sp / 2][n][2]
    const uint64_t* pst;
    int64_t Sp;
    int n, B;
    int64_t chunk;                 // entries per block (multiple of NS_SUB)
    const uint64_t* list_pc;       // [n][B]
    uint32_t* list_best;           // [n][B]
    uint32_t* status;
};

// Item g = i * BG + c (node i, order group c: orders c * R .. c * R + R - 1, those below
// B) takes T consecutive threads; thread `sub` of an item tests the entry pairs
// (2j, 2j + 1), j = sub mod T, of every staged slice against the group's orders.
template <int T, int R>
__global__ void __launch_bounds__(T == 1 ? 1024 : 256) k_scan_nodes(NodeScanArgs A)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const size_t SB = ns_stage_bytes(A.n);
    uint64_t* bar = (uint64_t*)(smem + NS_STAGES * SB);
    const int64_t e0 = (int64_t)blockIdx.x * A.chunk;
    const int64_t e1 = min(e0 + A.chunk, A.Sp);
    if (e0 >= e1) return;                                           // block-uniform
    const int nsub = (int)((e1 - e0) / NS_SUB);
    const int tid = threadIdx.x;
    const int BG = (A.B + R - 1) / R;
    const int g = tid / T, sub = tid - g * T;
    const bool active = g < A.n * BG;
    const int i = active ? g / BG : 0, c = active ? g - i * BG : 0;
    // predecessor masks of the group's orders, complemented (an unused slot tests only
    // the empty set and is never written back)
    uint32_t nlo[R], nhi[R], best0[R], best1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int b = c * R + r;
        const uint64_t pc = (active && b < A.B) ? A.list_pc[(size_t)i * A.B + b] : 0ull;
        nlo[r] = ~(uint32_t)pc;
        nhi[r] = ~(uint32_t)(pc >> 32);
        best0[r] = SPOS_NONE;
        best1[r] = SPOS_NONE;
    }
    const uint32_t rows = (uint32_t)(A.n * NS_SUB * 4);
    uint64_t pol_stream = 0, pol_keep = 0;
    if (tid == 0) {
        pol_stream = l2_policy_evict_first();
        pol_keep = l2_policy_evict_last();
        for (int st = 0; st < NS_STAGES; ++st) mbar_init(&bar[st], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // thread 0 stages slice `it` in buffer `st`: the masks, then all nodes' positions
    auto issue = [&](int it, int st) {
        uint8_t* base = smem + (size_t)st * SB;
        const int64_t e = e0 + (int64_t)it * NS_SUB;
        mbar_arrive_expect_tx(&bar[st], (uint32_t)(NS_SUB * 8) + rows);
        bulk_g2s(base, A.pst + e, NS_SUB * 8, &bar[st], pol_keep);
        bulk_g2s(base + NS_SUB * 8, A.spos_t + (size_t)e * A.n, rows, &bar[st], pol_stream);
    };
    if (tid == 0)
        for (int st = 0; st < NS_STAGES && st < nsub; ++st) issue(st, st);
    const int n = A.n;
    int it = 0;
    bool timed_out = false;
    for (; it < nsub; ++it) {
        const int st = it % NS_STAGES;
        const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((it / NS_STAGES) & 1), WAIT_TIMEOUT_NS);
        if (ok && active) {
            const uint4* M2 = (const uint4*)(smem + (size_t)st * SB);
            const uint2* P2 = (const uint2*)(smem + (size_t)st * SB + NS_SUB * 8) + i;
#pragma unroll(R >= 4 ? 4 : 8)
            for (int q = 0; q < NS_SUB / 2 / T; ++q) {
                const int j = q * T + sub;
                const uint4 mm = M2[j];
                const uint2 pp = P2[j * n];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    test_min(best0[r], mm.x, mm.y, nlo[r], nhi[r], pp.x);
                    test_min(best1[r], mm.z, mm.w, nlo[r], nhi[r], pp.y);
                }
            }
        }
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        if (tid == 0 && it + NS_STAGES < nsub) issue(it + NS_STAGES, st);
    }
    if (timed_out) {
        if (tid == 0) {
            atomicOr(A.status, STATUS_TIMEOUT);
            for (int j = it; j < nsub && j < it + NS_STAGES; ++j)
                mbar_wait_bounded(&bar[j % NS_STAGES], (uint32_t)((j / NS_STAGES) & 1), WAIT_TIMEOUT_NS);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint32_t best = min(best0[r], best1[r]);
#pragma unroll
        for (int off = 1; off < T; off <<= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, off));
        const int b = c * R + r;
        if (active && sub == 0 && b < A.B && best != SPOS_NONE) atomicMin(&A.list_best[(size_t)i * A.B + b], best);
    }
}

// launch shape of k_scan_nodes for n nodes and B orders: R orders per thread (as few
// groups as eight orders a thread allow, the orders spread evenly over them), T threads an
// item while 256 threads hold them, else one thread an item in blocks of up to 1,024
struct NsShape {
    int T, R, threads;
};

static NsShape ns_shape(int n, int B)
{
    const int BG = (B + NS_RMAX - 1) / NS_RMAX;
    const int R = (B + BG - 1) / BG;
    const int items = n * BG;
    int T = 1;
    while (T < 8 && 2 * T * items <= 256) T *= 2;
    return {T, R, items * T <= 256 ? 256 : (int)round_up(items, 32)};
}

bool scan_nodes_fits(const bn_table* t, int B)
{
    return t->scan_mode == BN_SCAN_FULL && B >= 1 && (int64_t)t->n * ((B + NS_RMAX - 1) / NS_RMAX) <= NS_MAX_ITEMS;
}

template <int T, int R>
static void ns_launch(unsigned grid, int threads, size_t smem, cudaStream_t s, const NodeScanArgs& A)
{
    k_scan_nodes<T, R><<<grid, threads, smem, s>>>(A);
}

typedef void (*NsLaunchFn)(unsigned, int, size_t, cudaStream_t, const NodeScanArgs&);
typedef void (*NsKernelFn)(NodeScanArgs);

template <int T>
static void ns_table_row(NsLaunchFn* l, NsKernelFn* k)
{
    l[0] = ns_launch<T, 1>; l[1] = ns_launch<T, 2>; l[2] = ns_launch<T, 3>; l[3] = ns_launch<T, 4>;
    l[4] = ns_launch<T, 5>; l[5] = ns_launch<T, 6>; l[6] = ns_launch<T, 7>; l[7] = ns_launch<T, 8>;
    k[0] = k_scan_nodes<T, 1>; k[1] = k_scan_nodes<T, 2>; k[2] = k_scan_nodes<T, 3>; k[3] = k_scan_nodes<T, 4>;
    k[4] = k_scan_nodes<T, 5>; k[5] = k_scan_nodes<T, 6>; k[6] = k_scan_nodes<T, 7>; k[7] = k_scan_nodes<T, 8>;
}

int launch_scan_nodes(const bn_table* t, int B, const uint64_t* list_pc, uint32_t* list_best, uint32_t* status,
                      cudaStream_t s)
{
    static_assert(NS_RMAX == 8, "one table row per T holds R = 1..8");
    static NsLaunchFn launch[4][NS_RMAX];
    static NsKernelFn kern[4][NS_RMAX];
    static std::once_flag once;
    std::call_once(once, [] {
        ns_table_row<1>(launch[0], kern[0]);
        ns_table_row<2>(launch[1], kern[1]);
        ns_table_row<4>(launch[2], kern[2]);
        ns_table_row<8>(launch[3], kern[3]);
    });
    const size_t smem = ns_smem(t->n);
    static unsigned long long ctx[64] = {0};
    if (first_in_context(ctx))
        for (int a = 0; a < 4; ++a)
            for (int r = 0; r < NS_RMAX; ++r)
                BN_CUDA(cudaFuncSetAttribute(kern[a][r], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ns_smem(MAXN)));
    const NsShape sh = ns_shape(t->n, B);
    // whole waves: as many blocks per SM as its 2,048 threads and shared memory hold (at
    // most four)
    const int per_sm = (int)std::max<size_t>(
        1, std::min<size_t>({(size_t)4, (size_t)(2048 / sh.threads), (size_t)(220 * 1024) / smem}));
    const int64_t want = (int64_t)sm_count() * per_sm;
    const int64_t chunk = round_up((t->Sp + want - 1) / want, NS_SUB);
    NodeScanArgs A{t->spos_t, t->pst, t->Sp, t->n, B, chunk, list_pc, list_best, status};
    const unsigned grid = (unsigned)((t->Sp + chunk - 1) / chunk);
    const int a = sh.T == 8 ? 3 : (sh.T == 4 ? 2 : (sh.T == 2 ? 1 : 0));
    launch[a][sh.R - 1](grid, sh.threads, smem, s, A);
    BN_LAUNCH_CHECK("k_scan_nodes");
    return BN_OK;
}

// synthetic work lists for tuning: every node holds `items` items with pseudo-random
// predecessor masks (a fixed integer hash of (node, item))
__global__ void k_tune_lists(int n, int items, uint64_t* list_pc, uint32_t* list_best, uint32_t* list_count)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) list_count[idx] = (uint32_t)items;
    if (idx >= n * items) return;
    uint64_t h = (uint64_t)idx * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    h ^= h >> 29;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 32;
    list_pc[idx] = h;
    list_best[idx] = SPOS_NONE;
}

// a5: candidate-space predecessor masks, written straight into the node-major work
// lists (item b of node i is order b); also checks each row is a permutation.
__global__ void k_pred_lists(const uint8_t* __restrict__ orders, int B, int n, uint64_t* __restrict__ list_pc,
                             uint32_t* __restrict__ list_best, uint32_t* __restrict__ list_count, uint32_t* status)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n && blockIdx.x == 0) list_count[idx] = (uint32_t)B;
    if (idx >= B * n) return;
    const int b = idx / n, i = idx - b * n;
    const uint8_t* o = orders + (size_t)b * n;
    uint64_t pred = 0, seen = 0;
    bool found = false;
    for (int p = 0; p < n; ++p) {
        const int v = o[p];
        if (v >= n) {
            atomicOr(status, STATUS_BADINPUT);
            break;
        }
        seen |= 1ull << v;
        if (v == i) found = true;
        else if (!found) pred |= 1ull << v;
    }
    const uint64_t full = (n == 64) ? ~0ull : ((1ull << n) - 1);
    if (seen != full) atomicOr(status, STATUS_BADINPUT);
    const uint64_t lowm = (i == 0) ? 0ull : ((1ull << i) - 1);
    const uint64_t pc = (pred & lowm) | ((i + 1 < 64) ? ((pred >> (i + 1)) << i) : 0ull);
    list_pc[(size_t)i * B + b] = pc;
    list_best[(size_t)i * B + b] = SPOS_NONE;
}

int launch_pred_lists(const uint8_t* orders, int B, int n, uint64_t* list_pc, uint32_t* list_best,
                      uint32_t* list_count, uint32_t* status, cudaStream_t s)
{
    const int tot = B * n;
    k_pred_lists<<<(tot + 255) / 256, 256, 0, s>>>(orders, B, n, list_pc, list_best, list_count, status);
    BN_LAUNCH_CHECK("k_pred_lists");
    return BN_OK;
}

// a7: per order, the chosen rank of every node and the FP64 sum over nodes in ascending
// node id of their entries
__global__ void k_reduce_orders(const uint32_t* __restrict__ list_best, const uint32_t* __restrict__ srank,
                                const int64_t* __restrict__ keys, int64_t Sp, int n, int B,
                                uint32_t* __restrict__ best_rank, double* __restrict__ score)
{
    __shared__ int64_t s_key[8][MAXN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= B) return;
    for (int i = lane; i < n; i += 32) {
        uint32_t p = list_best[(size_t)i * B + b];
        if ((int64_t)p >= Sp) p = 0;                  // only after a timed-out scan
        const uint32_t r = srank[(size_t)i * Sp + p];
        s_key[warp][i] = keys[(size_t)i * Sp + r];
        if (best_rank) best_rank[(size_t)b * n + i] = r;
    }
    __syncwarp();
    if (lane == 0 && score) {
        double sum = 0.0;
        for (int i = 0; i < n; ++i) sum = __dadd_rn(sum, key_to_double(s_key[warp][i]));
        score[b] = sum;
    }
}

// the full-table scan's tiling for up to max_items items per node, tuned on first use: the
// first scan with a new number of 256-item groups (<= 8) times every tiling the autotuner
// knows on this table (tens of milliseconds once) and keeps the fastest.  BN_AUTOTUNE=0 in
// the environment keeps the fixed plan.
int ensure_tuned(const bn_table* t, int max_items, cudaStream_t s)
{
    if (!t || (t->scan_mode != BN_SCAN_FULL && t->scan_mode != BN_SCAN_UNRANK) || max_items < 1) return BN_OK;
    const int groups = (max_items + SCAN_THREADS - 1) / SCAN_THREADS;
    if (groups > 8 || t->tuned_sub[groups]) return BN_OK;
    static const bool off = [] {
        const char* e = getenv("BN_AUTOTUNE");
        return e && e[0] == '0';
    }();
    if (off) return BN_OK;
    return bn_table_autotune(const_cast<bn_table*>(t), groups * SCAN_THREADS, s, nullptr);
}

// The peak rate of the scan's consistency test on this GPU, for its roofline: the scan's
// own inner loop (two entries per step: their sorted positions by one 8-byte and their
// masks by one 16-byte shared-memory load, then two test_min) over 1,024 entries that
// stay in shared memory, so nothing waits on HBM or on the staging barriers.  The loads
// stay inside the loop (1,024 entries do not fit in registers).
static constexpr int TEST_RATE_ENTRIES = 1024;

__global__ void __launch_bounds__(256) k_test_rate(uint32_t iters, uint32_t salt, uint32_t* sink)
{
    __shared__ uint2 s_p[TEST_RATE_ENTRIES / 2];
    __shared__ uint4 s_m[TEST_RATE_ENTRIES / 2];
    for (int j = threadIdx.x; j < TEST_RATE_ENTRIES / 2; j += blockDim.x) {
        const uint32_t h = (uint32_t)j * 0x9e3779b9u ^ salt;
        s_p[j] = make_uint2(h >> 1, (h * 0x85ebca6bu) >> 1);
        s_m[j] = make_uint4(h & 0x0f0f0f0fu, h & 0x00ff00ffu, (h * 3u) & 0x0f0f0f0fu, (h * 5u) & 0x00ff00ffu);
    }
    __syncthreads();
    const uint32_t x = (threadIdx.x + blockIdx.x * 256u) * 0x27d4eb2du;
    const uint32_t nlo = ~(x & 0xf0f0f0f0u), nhi = ~(x & 0xff00ff00u);
    uint32_t b0 = ~0u, b1 = ~0u;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll 32
        for (int j = 0; j < TEST_RATE_ENTRIES / 2; ++j) {
            const uint2 pp = s_p[j];
            const uint4 mm = s_m[j];
            test_min(b0, mm.x, mm.y, nlo, nhi, pp.x);
            test_min(b1, mm.z, mm.w, nlo, nhi, pp.y);
        }
    }
    if (min(b0, b1) == 0x12345678u) sink[0] = 1u;     // keeps the results live
}

int launch_reduce_orders(const bn_table* t, const uint32_t* list_best, int B, uint32_t* best_rank, double* score,
                         cudaStream_t s)
{
    k_reduce_orders<<<(B + 7) / 8, 256, 0, s>>>(list_best, t->srank, t->keys, t->Sp, t->n, B, best_rank, score);
    BN_LAUNCH_CHECK("k_reduce_orders");
    return BN_OK;
}

}  // namespace bn

using namespace bn;

// the stream-ordered pool keeps freed scratch mapped (its default release threshold of 0
// would unmap it at every synchronisation and map it again on the next call)
static void keep_pool_mapped()
{
    static unsigned long long ctx[64] = {0};
    if (!first_in_context(ctx)) return;
    const int d = device_id();
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
        uint64_t thr = (uint64_t)256 << 20;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

static int score_orders_impl(const bn_table* t, const uint8_t* orders, int B, uint32_t* best_rank,
                             double* order_score, int mem, void* stream, cudaEvent_t ev0, cudaEvent_t ev1)
{
    set_error(BN_OK, "");
    if (!t) return set_error(BN_EINVAL, "bn_score_orders: NULL table");
    if (B < 0) return set_error(BN_EINVAL, "bn_score_orders: B=%d", B);
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_score_orders: bad mem");
    if (B == 0) return BN_OK;
    if (!orders) return set_error(BN_EINVAL, "bn_score_orders: orders is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = t->n;
    if (!scan_nodes_fits(t, B)) {
        int rt = ensure_tuned(t, B, s);
        if (rt) return rt;
    }
    const ScanPlan pl = plan_scan(t, B);
    keep_pool_mapped();

    // one scratch block: orders | list_pc | list_best | counts | status | ranks | scores
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    const size_t o_orders = take(mem == BN_MEM_HOST ? (size_t)B * n : 0);
    const size_t o_pc = take(sizeof(uint64_t) * (size_t)n * B);
    const size_t o_best = take(sizeof(uint32_t) * (size_t)n * B);
    const size_t o_cnt = take(sizeof(uint32_t) * n);
    const size_t o_st = take(sizeof(uint32_t));
    const size_t o_rank = take(mem == BN_MEM_HOST && best_rank ? sizeof(uint32_t) * (size_t)B * n : 0);
    const size_t o_score = take(mem == BN_MEM_HOST && order_score ? sizeof(double) * B : 0);
    uint8_t* base = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&base, off, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BN_ENOMEM, "bn_score_orders: scratch of %zu bytes: %s", off, cudaGetErrorString(e));
    }
    struct Free {
        uint8_t* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{base, s};
    const uint8_t* d_orders = orders;
    if (mem == BN_MEM_HOST) {
        BN_CUDA(cudaMemcpyAsync(base + o_orders, orders, (size_t)B * n, cudaMemcpyHostToDevice, s));
        d_orders = base + o_orders;
    }
    uint64_t* d_pc = (uint64_t*)(base + o_pc);
    uint32_t* d_best = (uint32_t*)(base + o_best);
    uint32_t* d_cnt = (uint32_t*)(base + o_cnt);
    uint32_t* d_st = (uint32_t*)(base + o_st);
    uint32_t* d_rank = mem == BN_MEM_HOST ? (best_rank ? (uint32_t*)(base + o_rank) : nullptr) : best_rank;
    double* d_score = mem == BN_MEM_HOST ? (order_score ? (double*)(base + o_score) : nullptr) : order_score;
    BN_CUDA(cudaMemsetAsync(d_st, 0, sizeof(uint32_t), s));
    int rc = launch_pred_lists(d_orders, B, n, d_pc, d_best, d_cnt, d_st, s);
    if (rc) return rc;
    if (ev0) BN_CUDA(cudaEventRecord(ev0, s));
    rc = scan_nodes_fits(t, B) ? launch_scan_nodes(t, B, d_pc, d_best, d_st, s)
                               : launch_scan(t, pl, d_cnt, d_pc, d_best, B, d_st, s);
    if (rc) return rc;
    if (ev1) BN_CUDA(cudaEventRecord(ev1, s));
    if ((rc = launch_reduce_orders(t, d_best, B, d_rank, d_score, s))) return rc;
    if (mem == BN_MEM_HOST) {
        if (best_rank)
            BN_CUDA(cudaMemcpyAsync(best_rank, d_rank, sizeof(uint32_t) * (size_t)B * n, cudaMemcpyDeviceToHost, s));
        if (order_score) BN_CUDA(cudaMemcpyAsync(order_score, d_score, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    }
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, d_st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_BADINPUT) return set_error(BN_EINVAL, "bn_score_orders: an order is not a permutation of 0..n-1");
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_score_orders: a bounded device wait expired");
    return BN_OK;
}

extern "C" int bn_score_orders(const bn_table* t, const uint8_t* orders, int B, uint32_t* best_rank,
                               double* order_score, int mem, void* stream)
{
    return score_orders_impl(t, orders, B, best_rank, order_score, mem, stream, nullptr, nullptr);
}

extern "C" int bn_score_orders_profiled(const bn_table* t, const uint8_t* orders, int B, uint32_t* best_rank,
                                        double* order_score, int mem, void* stream, double* scan_ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
    }
    int rc = score_orders_impl(t, orders, B, best_rank, order_score, mem, stream, e0, e1);
    float ms = 0.f;
    if (rc == BN_OK && B > 0 && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = cuda_fail(cudaGetLastError(), "cudaEventElapsedTime", __FILE__, __LINE__);
    if (scan_ms) *scan_ms = (double)ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" int bn_measure_test_rate(void* stream, double* tests_per_s)
{
    set_error(BN_OK, "");
    if (!tests_per_s) return set_error(BN_EINVAL, "bn_measure_test_rate: NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* sink = nullptr;
    BN_CUDA(cudaMallocAsync((void**)&sink, 4, s));
    struct Free {
        uint32_t* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{sink, s};
    cudaEvent_t e0, e1;
    BN_CUDA(cudaEventCreate(&e0));
    BN_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev()
        {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};
    const unsigned grid = (unsigned)sm_count() * 8u;
    const uint32_t iters = 16;
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {                 // the first launch warms up
        BN_CUDA(cudaEventRecord(e0, s));
        k_test_rate<<<grid, 256, 0, s>>>(iters, (uint32_t)rep, sink);
        BN_LAUNCH_CHECK("k_test_rate");
        BN_CUDA(cudaEventRecord(e1, s));
        BN_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        BN_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    *tests_per_s = (double)grid * 256.0 * iters * TEST_RATE_ENTRIES / (best * 1e-3);
    return BN_OK;
}

extern "C" int bn_table_autotune(bn_table* t, int max_items, void* stream, int64_t* chosen)
{
    set_error(BN_OK, "");
    if (!t || max_items < 1) return set_error(BN_EINVAL, "bn_table_autotune: bad arguments");
    const int groups = std::max(1, (max_items + SCAN_THREADS - 1) / SCAN_THREADS);
    if (groups > 8) return set_error(BN_EUNSUPPORTED, "bn_table_autotune: at most 2048 items");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = t->n, items = std::min(max_items, groups * SCAN_THREADS);
    uint8_t* blk = nullptr;
    const size_t o_pc = 0, o_best = (size_t)round_up(8 * (int64_t)n * items, 256),
                 o_cnt = o_best + (size_t)round_up(4 * (int64_t)n * items, 256), o_st = o_cnt + 256;
    BN_CUDA(cudaMallocAsync((void**)&blk, o_st + 256, s));
    struct Free {
        uint8_t* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{blk, s};
    uint64_t* pc = (uint64_t*)(blk + o_pc);
    uint32_t* best = (uint32_t*)(blk + o_best);
    uint32_t* cnt = (uint32_t*)(blk + o_cnt);
    uint32_t* st = (uint32_t*)(blk + o_st);
    BN_CUDA(cudaMemsetAsync(st, 0, 4, s));
    cudaEvent_t e0, e1;
    BN_CUDA(cudaEventCreate(&e0));
    BN_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev()
        {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } ev{e0, e1};
    const int saved_mode = t->scan_mode;
    t->scan_mode = BN_SCAN_FULL;
    float best_ms = 1e30f;
    ScanPlan best_pl = plan_for(t, groups, (int64_t)sm_count() * 8, 1024);
    const int subs[3] = {512, 1024, 2048};
    const int per_sm[5] = {1, 2, 4, 8, 16};
    int rc = BN_OK;
    for (int si = 0; si < 3 && !rc; ++si) {
        for (int bi = 0; bi < 5 && !rc; ++bi) {
            const ScanPlan pl = plan_for(t, groups, (int64_t)sm_count() * per_sm[bi], subs[si]);
            float tot = 0.f;
            for (int rep = 0; rep < 4 && !rc; ++rep) {
                k_tune_lists<<<(n * items + 255) / 256, 256, 0, s>>>(n, items, pc, best, cnt);
                if (cudaGetLastError() != cudaSuccess) { rc = set_error(BN_ECUDA, "k_tune_lists"); break; }
                count_launches(1);
                if (cudaEventRecord(e0, s) != cudaSuccess) { rc = set_error(BN_ECUDA, "event"); break; }
                rc = launch_scan(t, pl, cnt, pc, best, items, st, s);
                if (rc) break;
                if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = set_error(BN_ECUDA, "event sync");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;          // first launch warms up
            }
            if (!rc && tot < best_ms) { best_ms = tot; best_pl = pl; }
        }
    }
    t->scan_mode = saved_mode;
    if (rc) return rc;
    t->tuned_sub[groups] = best_pl.sub;
    t->tuned_nchunk[groups] = best_pl.nchunk;
    t->tuned_chunk[groups] = best_pl.chunk;
    if (chosen) {
        chosen[0] = best_pl.sub;
        chosen[1] = best_pl.nchunk;
        chosen[2] = (int64_t)(1000.0f * best_ms / 3.0f);   // microseconds per launch
    }
    uint32_t hs = 0;
    BN_CUDA(cudaMemcpyAsync(&hs, st, 4, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (hs & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_table_autotune: a bounded device wait expired");
    return BN_OK;
}
