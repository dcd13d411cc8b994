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
// warps take a share of the entries of the same items.  Chunks combine with atomicMin.
#include <algorithm>
#include <cstring>

#include "bn_table.cuh"

namespace bn {

static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_WARPS = SCAN_THREADS / 32;
// stage size (entries) and pipeline depth; 48 KB of shared memory for the 1024 and 512
// variants, 72 KB for 2048
template <int SUB>
struct ScanCfg {
    static constexpr int STAGES = SUB >= 2048 ? 3 : (SUB >= 1024 ? 4 : 8);
    static constexpr size_t SMEM = (size_t)STAGES * SUB * (sizeof(uint32_t) + sizeof(uint64_t)) + 8 * STAGES;
};

struct ScanArgs {
    const uint32_t* spos;
    const uint64_t* pst;
    int64_t Sp;
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
    int64_t nchunk = (target + (int64_t)t->n * groups - 1) / ((int64_t)t->n * groups);
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
    return plan_for(t, groups, (int64_t)sm_count() * 4 * 2, 1024);   // two waves of four blocks per SM
}

template <int SCAN_SUB>
__device__ __forceinline__ void scan_issue(const ScanArgs& A, int node, int64_t base, int64_t e1, uint32_t* s_sp,
                                           uint64_t* s_msk, uint64_t* bar, uint64_t pol_stream, uint64_t pol_keep)
{
    const uint32_t cnt = (uint32_t)min((int64_t)SCAN_SUB, e1 - base);
    mbar_arrive_expect_tx(bar, cnt * 12u);
    bulk_g2s(s_sp, A.spos + (size_t)node * A.Sp + base, cnt * 4u, bar, pol_stream);
    bulk_g2s(s_msk, A.pst + base, cnt * 8u, bar, pol_keep);
}

template <int SCAN_SUB>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(ScanArgs A)
{
    constexpr int SCAN_STAGES = ScanCfg<SCAN_SUB>::STAGES;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* s_msk = (uint64_t*)smem;                                          // [STAGES][SUB]
    uint32_t* s_sp = (uint32_t*)(smem + sizeof(uint64_t) * SCAN_STAGES * SCAN_SUB);
    uint64_t* bar = (uint64_t*)(smem + (sizeof(uint64_t) + sizeof(uint32_t)) * SCAN_STAGES * SCAN_SUB);

    const int node = blockIdx.x / A.nchunk;
    const int chunk = blockIdx.x - node * A.nchunk;
    const int cnt = (int)A.list_count[node];
    const int g0 = blockIdx.y * SCAN_THREADS;
    if (g0 >= cnt) return;                                                      // block-uniform
    const int64_t e0 = (int64_t)chunk * A.chunk;
    const int64_t e1 = min(e0 + A.chunk, A.Sp);
    if (e0 >= e1) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // G warps' worth of items; the spare warps split the entries of the same items
    const int here = min(SCAN_THREADS, cnt - g0);
    const int G = (here + 31) >> 5;
    const int split = SCAN_WARPS / G;
    const int ig = warp % G, sp = warp / G;
    const bool warp_on = sp < split;
    const int item = g0 + ig * 32 + lane;
    const bool active = warp_on && item < cnt;
    const uint64_t npc = active ? ~A.list_pc[(size_t)node * A.cap + item] : ~0ull;
    const int nsub = (int)((e1 - e0 + SCAN_SUB - 1) / SCAN_SUB);

    uint64_t pol_stream = 0, pol_keep = 0;
    if (threadIdx.x == 0) {
        pol_stream = l2_policy_evict_first();
        pol_keep = l2_policy_evict_last();
        for (int s = 0; s < SCAN_STAGES; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int s = 0; s < SCAN_STAGES && s < nsub; ++s)
            scan_issue<SCAN_SUB>(A, node, e0 + (int64_t)s * SCAN_SUB, e1, s_sp + s * SCAN_SUB, s_msk + s * SCAN_SUB, &bar[s],
                       pol_stream, pol_keep);
    }

    uint32_t b0 = SPOS_NONE, b1 = SPOS_NONE;
    int it = 0;
    bool timed_out = false;
    for (; it < nsub; ++it) {
        const int st = it % SCAN_STAGES;
        const uint32_t parity = (uint32_t)((it / SCAN_STAGES) & 1);
        const bool ok = mbar_wait_bounded(&bar[st], parity, WAIT_TIMEOUT_NS);
        if (ok && warp_on) {
            const int64_t base = e0 + (int64_t)it * SCAN_SUB;
            const int pairs = (int)min((int64_t)SCAN_SUB, e1 - base) >> 1;
            const uint2* P = (const uint2*)(s_sp + st * SCAN_SUB);
            const ulonglong2* M = (const ulonglong2*)(s_msk + st * SCAN_SUB);
#pragma unroll 4
            for (int j = sp; j < pairs; j += split) {
                const uint2 pp = P[j];
                const ulonglong2 mm = M[j];
                if ((mm.x & npc) == 0ull) b0 = min(b0, pp.x);
                if ((mm.y & npc) == 0ull) b1 = min(b1, pp.y);
            }
        }
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        if (threadIdx.x == 0 && it + SCAN_STAGES < nsub) {
            const int64_t base = e0 + (int64_t)(it + SCAN_STAGES) * SCAN_SUB;
            scan_issue<SCAN_SUB>(A, node, base, e1, s_sp + st * SCAN_SUB, s_msk + st * SCAN_SUB, &bar[st], pol_stream,
                       pol_keep);
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
    const uint32_t b = min(b0, b1);
    if (active && b != SPOS_NONE) atomicMin(&A.list_best[(size_t)node * A.cap + item], b);
}

int launch_scan(const bn_table* t, const ScanPlan& pl, const uint32_t* list_count, const uint64_t* list_pc,
                uint32_t* list_best, int cap, uint32_t* status, cudaStream_t s)
{
    if (t->scan_mode == BN_SCAN_PRUNED) return launch_scan_pruned(t, list_count, list_pc, list_best, cap, s);
    ScanArgs A;
    A.spos = t->spos;
    A.pst = t->pst;
    A.Sp = t->Sp;
    A.nchunk = pl.nchunk;
    A.chunk = pl.chunk;
    A.list_count = list_count;
    A.list_pc = list_pc;
    A.list_best = list_best;
    A.cap = cap;
    A.status = status;
    static bool attr_set[64][3] = {{false}};
    const int d = device_id();
    const int v = pl.sub >= 2048 ? 2 : (pl.sub >= 1024 ? 1 : 0);
    if (d < 64 && !attr_set[d][v]) {
        if (v == 2) BN_CUDA(cudaFuncSetAttribute(k_scan<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ScanCfg<2048>::SMEM));
        if (v == 1) BN_CUDA(cudaFuncSetAttribute(k_scan<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ScanCfg<1024>::SMEM));
        if (v == 0) BN_CUDA(cudaFuncSetAttribute(k_scan<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ScanCfg<512>::SMEM));
        attr_set[d][v] = true;
    }
    dim3 grid((unsigned)(t->n * pl.nchunk), (unsigned)((cap + SCAN_THREADS - 1) / SCAN_THREADS));
    if (v == 2) k_scan<2048><<<grid, SCAN_THREADS, ScanCfg<2048>::SMEM, s>>>(A);
    else if (v == 1) k_scan<1024><<<grid, SCAN_THREADS, ScanCfg<1024>::SMEM, s>>>(A);
    else k_scan<512><<<grid, SCAN_THREADS, ScanCfg<512>::SMEM, s>>>(A);
    BN_LAUNCH_CHECK("k_scan");
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

}  // namespace bn

using namespace bn;

// the stream-ordered pool keeps freed scratch mapped (its default release threshold of 0
// would unmap it at every synchronisation and map it again on the next call)
static void keep_pool_mapped()
{
    static bool done[64] = {false};
    const int d = device_id();
    if (d < 0 || d >= 64 || done[d]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
        uint64_t thr = (uint64_t)256 << 20;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[d] = true;
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
    if ((rc = launch_scan(t, pl, d_cnt, d_pc, d_best, B, d_st, s))) return rc;
    if (ev1) BN_CUDA(cudaEventRecord(ev1, s));
    k_reduce_orders<<<(B + 7) / 8, 256, 0, s>>>(d_best, t->srank, t->keys, t->Sp, n, B, d_rank, d_score);
    BN_LAUNCH_CHECK("k_reduce_orders");
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
