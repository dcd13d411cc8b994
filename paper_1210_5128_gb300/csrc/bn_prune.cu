// bn_prune.cu -- exact pruning of the table and the scan over what is left.
//
// An entry (i, pi) can never be the answer of Eq. (6) if some proper subset pi' of pi
// scores at least as well: whenever pi lies inside a node's predecessors so does pi',
// and pi' wins (a higher score, or an equal score at a lower rank -- ranks are
// size-ascending).  Removing every such "dominated" entry leaves every order's result
// unchanged.  For each node the surviving entries are kept in sorted-position order
// (score descending, rank ascending), so a scan over them can stop at its first
// consistent entry.
//
// best_le(pi) = max over all subsets of pi (pi included) of the entry key, computed size
// class by size class from the j immediate subsets; pi survives iff key(pi) >
// max_t best_le(pi minus its t-th element).
#include <algorithm>
#include <cstring>
#include <vector>

#include "bn_table.cuh"

namespace bn {

static constexpr int PR_RANGE = 64;       // consecutive ranks per thread
static constexpr int PR_CHUNK = 4096;     // sorted positions per compaction block
static constexpr int PS_CHUNK = 2048;     // surviving entries per pruned-scan block

__device__ __forceinline__ void pr_unrank(int N, int64_t rank, int& j, uint64_t& mask)
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

// one size class j: ranks [base, base + C(N, j)) of every node
__global__ void k_dominance(const int64_t* __restrict__ keys, int64_t Sp, int N, int j, int64_t base, int64_t count,
                            int units_per_node, const uint64_t* __restrict__ binom /*[65][j+1]*/,
                            int64_t* __restrict__ best_le, uint8_t* __restrict__ alive)
{
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(u / units_per_node);
    const int64_t r0 = (u - (int64_t)i * units_per_node) * PR_RANGE;
    if (r0 >= count || i >= N + 1) return;
    const int64_t r1 = min(r0 + (int64_t)PR_RANGE, count);
    const int64_t* K = keys + (size_t)i * Sp;
    int64_t* BL = best_le + (size_t)i * Sp;
    uint8_t* AL = alive + (size_t)i * Sp;
    if (j == 0) {
        BL[0] = K[0];
        AL[0] = 1;
        return;
    }
    int jj;
    uint64_t mask;
    pr_unrank(N, base + r0, jj, mask);
    const int64_t sub_base = base - (int64_t)binom[(size_t)N * 8 + (j - 1)];   // first rank of size j-1
    for (int64_t r = r0; r < r1; ++r) {
        // elements a_1 < ... < a_j and the combinatorial part of the rank
        int el[MAXK];
        uint64_t m = mask;
#pragma unroll
        for (int t = 0; t < MAXK; ++t) {
            el[t] = 0;
            if (t < j) { el[t] = __ffsll((long long)m) - 1; m &= m - 1; }
        }
        int64_t sub_max = KEY_NONE;
#pragma unroll
        for (int drop = 0; drop < MAXK; ++drop) {
            if (drop < j) {
                int64_t rr = sub_base;
                int pos = 1;
#pragma unroll
                for (int t = 0; t < MAXK; ++t) {
                    if (t < j && t != drop) { rr += (int64_t)binom[(size_t)el[t] * 8 + pos]; ++pos; }
                }
                sub_max = max(sub_max, BL[rr]);
            }
        }
        const int64_t key = K[base + r];
        AL[base + r] = key > sub_max ? 1 : 0;
        BL[base + r] = max(key, sub_max);
        // colex successor within the size class
        const uint64_t c = mask & (~mask + 1);
        const uint64_t rs = mask + c;
        mask = (((rs ^ mask) >> 2) >> (__ffsll((long long)mask) - 1)) | rs;
    }
}

// survivors per (node, chunk of sorted positions)
__global__ void k_alive_count(const uint8_t* __restrict__ alive, const uint32_t* __restrict__ srank, int64_t S,
                              int64_t Sp, int nch, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t s;
    const int i = blockIdx.x / nch, ch = blockIdx.x - i * nch;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    uint32_t c = 0;
    for (int64_t p = (int64_t)ch * PR_CHUNK + threadIdx.x; p < min((int64_t)(ch + 1) * PR_CHUNK, S); p += blockDim.x)
        c += alive[(size_t)i * Sp + srank[(size_t)i * Sp + p]];
    atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// ordered compaction: block-level scan of the flags in sorted-position order
__global__ void __launch_bounds__(256) k_alive_write(const uint8_t* __restrict__ alive,
                                                     const uint32_t* __restrict__ srank,
                                                     const uint64_t* __restrict__ pst, int64_t S, int64_t Sp, int nch,
                                                     const uint32_t* __restrict__ offs, uint64_t* __restrict__ amask,
                                                     uint32_t* __restrict__ aspos)
{
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t running;
    const int i = blockIdx.x / nch, ch = blockIdx.x - i * nch;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) running = offs[blockIdx.x];
    __syncthreads();
    const int64_t p0 = (int64_t)ch * PR_CHUNK, p1 = min(p0 + PR_CHUNK, S);
    for (int64_t base = p0; base < p1; base += 256) {
        const int64_t p = base + threadIdx.x;
        uint32_t r = 0, f = 0;
        if (p < p1) {
            r = srank[(size_t)i * Sp + p];
            f = alive[(size_t)i * Sp + r];
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f != 0);
        const uint32_t before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        uint32_t off = running;
        for (int w = 0; w < warp; ++w) off += wsum[w];
        if (f) {
            amask[off + before] = pst[r];
            aspos[off + before] = (uint32_t)p;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int w = 0; w < 8; ++w) tot += wsum[w];
            running += tot;
        }
        __syncthreads();
    }
}

// largest |entry| among the survivors (positive doubles order like their bit patterns)
__global__ void k_survivor_maxabs(const uint32_t* __restrict__ aspos, const uint32_t* __restrict__ aoff,
                                  const uint32_t* __restrict__ acnt, const uint32_t* __restrict__ srank,
                                  const int64_t* __restrict__ keys, int64_t Sp, int n, unsigned long long* out)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    for (uint32_t j = threadIdx.x; j < acnt[i]; j += blockDim.x) {
        const uint32_t r = srank[(size_t)i * Sp + aspos[aoff[i] + j]];
        const double v = fabs(key_to_double(keys[(size_t)i * Sp + r]));
        atomicMax(out, (unsigned long long)__double_as_longlong(v));
    }
}

struct PrunedArgs {
    const uint64_t* amask;
    const uint32_t* aspos;
    const uint32_t* aoff;      // [n] first survivor of node i
    const uint32_t* acnt;      // [n]
    int max_chunks;
    const uint32_t* list_count;
    const uint64_t* list_pc;
    uint32_t* list_best;
    int cap;
};

// scan over a node's survivors in sorted-position order: each thread stops at its first
// consistent entry (the minimum sorted position within this chunk); warps leave when all
// their items have one; chunks combine with atomicMin
__global__ void __launch_bounds__(256) k_scan_pruned(PrunedArgs A)
{
    const int node = blockIdx.x / A.max_chunks, ch = blockIdx.x - node * A.max_chunks;
    const int cnt = (int)A.list_count[node];
    const int g0 = blockIdx.y * 256;
    if (g0 >= cnt) return;
    const int64_t acount = A.acnt[node];
    const int64_t e0 = (int64_t)ch * PS_CHUNK;
    if (e0 >= acount) return;
    const int64_t e1 = min(acount, e0 + PS_CHUNK);
    const int item = g0 + (int)threadIdx.x;
    const bool active = item < cnt;
    if (!__any_sync(0xffffffffu, active)) return;
    const uint64_t npc = active ? ~A.list_pc[(size_t)node * A.cap + item] : 0ull;
    const uint64_t* M = A.amask + A.aoff[node];
    const uint32_t* P = A.aspos + A.aoff[node];
    bool found = !active;
    uint32_t best = SPOS_NONE;
    for (int64_t e = e0; e < e1; e += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t ee = e + u;
            if (ee < e1) {
                const uint64_t m = __ldg(M + ee);
                if (!found && (m & npc) == 0ull) { best = __ldg(P + ee); found = true; }
            }
        }
        if (__all_sync(0xffffffffu, found)) break;
    }
    if (active && best != SPOS_NONE) atomicMin(&A.list_best[(size_t)node * A.cap + item], best);
}

int launch_scan_pruned(const bn_table* t, const uint32_t* list_count, const uint64_t* list_pc, uint32_t* list_best,
                       int cap, cudaStream_t s)
{
    PrunedArgs A;
    A.amask = t->amask;
    A.aspos = t->aspos;
    A.aoff = t->aoff;
    A.acnt = t->acnt;
    A.max_chunks = t->alive_chunks;
    A.list_count = list_count;
    A.list_pc = list_pc;
    A.list_best = list_best;
    A.cap = cap;
    dim3 grid((unsigned)(t->n * t->alive_chunks), (unsigned)((cap + 255) / 256));
    k_scan_pruned<<<grid, 256, 0, s>>>(A);
    BN_LAUNCH_CHECK("k_scan_pruned");
    return BN_OK;
}

int prune_table(bn_table* t, cudaStream_t s)
{
    if (t->amask) return BN_OK;
    const int n = t->n, N = n - 1, k = t->k;
    const int64_t S = t->S, Sp = t->Sp;
    const int nch = (int)((S + PR_CHUNK - 1) / PR_CHUNK);
    int64_t* best_le = nullptr;
    uint8_t* alive = nullptr;
    uint32_t *counts = nullptr, *offs = nullptr;
    uint64_t* binom = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&best_le, 8 * (size_t)n * Sp, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&alive, (size_t)n * Sp, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&counts, 4 * (size_t)n * nch, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&binom, 8 * 65 * 8, s);
    struct F {
        cudaStream_t s;
        void* p[4];
        ~F()
        {
            for (void* q : p)
                if (q) cudaFreeAsync(q, s);
        }
    } fr{s, {best_le, alive, counts, binom}};
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BN_ENOMEM, "prune: %zu bytes of work space", (size_t)n * Sp * 9);
    }
    if (k > 7) return set_error(BN_EUNSUPPORTED, "prune: k=%d above 7", k);
    std::vector<uint64_t> hb(65 * 8);
    for (int a = 0; a <= 64; ++a)
        for (int q = 0; q < 8; ++q) hb[(size_t)a * 8 + q] = h_binom.v[a][q];
    BN_CUDA(cudaMemcpyAsync(binom, hb.data(), 8 * hb.size(), cudaMemcpyHostToDevice, s));
    int64_t base = 0;
    for (int j = 0; j <= k && j <= N; ++j) {
        const int64_t count = (int64_t)h_binom.v[N][j];
        const int upn = (int)((count + PR_RANGE - 1) / PR_RANGE);
        const int64_t threads = (int64_t)n * upn;
        k_dominance<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(t->keys, Sp, N, j, base, count, upn, binom,
                                                                    best_le, alive);
        BN_LAUNCH_CHECK("k_dominance");
        base += count;
    }
    k_alive_count<<<n * nch, 256, 0, s>>>(alive, t->srank, S, Sp, nch, counts);
    BN_LAUNCH_CHECK("k_alive_count");
    std::vector<uint32_t> hc((size_t)n * nch);
    BN_CUDA(cudaMemcpyAsync(hc.data(), counts, 4 * hc.size(), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    std::vector<uint32_t> ho(hc.size()), hoff(n), hcnt(n);
    uint64_t run = 0;
    uint32_t mx = 0;
    for (int i = 0; i < n; ++i) {
        hoff[i] = (uint32_t)run;
        for (int c = 0; c < nch; ++c) {
            ho[(size_t)i * nch + c] = (uint32_t)run;
            run += hc[(size_t)i * nch + c];
        }
        hcnt[i] = (uint32_t)(run - hoff[i]);
        mx = std::max(mx, hcnt[i]);
    }
    if (run >= 0xffffffffull) return set_error(BN_EUNSUPPORTED, "prune: too many surviving entries");
    uint8_t* blk = nullptr;
    const size_t bytes = 8 * (size_t)std::max<uint64_t>(run, 1) + 4 * (size_t)std::max<uint64_t>(run, 1) + 8 * (size_t)n + 64;
    BN_CUDA(cudaMalloc((void**)&blk, bytes));
    t->amask = (uint64_t*)blk;
    t->aspos = (uint32_t*)(blk + 8 * std::max<uint64_t>(run, 1));
    t->aoff = (uint32_t*)((uint8_t*)t->aspos + 4 * std::max<uint64_t>(run, 1));
    t->acnt = t->aoff + n;
    t->alive_total = (int64_t)run;
    t->alive_max = mx;
    t->alive_chunks = (int)std::max<uint32_t>(1, (mx + PS_CHUNK - 1) / PS_CHUNK);
    t->alive_block = blk;
    BN_CUDA(cudaMemcpyAsync(t->aoff, hoff.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    BN_CUDA(cudaMemcpyAsync(t->acnt, hcnt.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    uint32_t* d_offs = counts;                    // reuse: per-chunk output offsets
    BN_CUDA(cudaMemcpyAsync(d_offs, ho.data(), 4 * ho.size(), cudaMemcpyHostToDevice, s));
    k_alive_write<<<n * nch, 256, 0, s>>>(alive, t->srank, t->pst, S, Sp, nch, d_offs, t->amask, t->aspos);
    BN_LAUNCH_CHECK("k_alive_write");
    unsigned long long* d_mx = (unsigned long long*)binom;          // reuse: one word
    BN_CUDA(cudaMemsetAsync(d_mx, 0, 8, s));
    k_survivor_maxabs<<<n, 128, 0, s>>>(t->aspos, t->aoff, t->acnt, t->srank, t->keys, Sp, n, d_mx);
    BN_LAUNCH_CHECK("k_survivor_maxabs");
    unsigned long long hmx = 0;
    BN_CUDA(cudaMemcpyAsync(&hmx, d_mx, 8, cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    double mx_abs;
    memcpy(&mx_abs, &hmx, 8);
    t->max_abs_survivor = mx_abs;
    (void)offs;
    return build_survivor_cache(t, s);
}

}  // namespace bn

using namespace bn;

extern "C" int bn_table_set_scan(bn_table* t, int mode, void* stream)
{
    set_error(BN_OK, "");
    if (!t) return set_error(BN_EINVAL, "bn_table_set_scan: NULL table");
    if (mode != BN_SCAN_FULL && mode != BN_SCAN_PRUNED && mode != BN_SCAN_UNRANK && mode != BN_SCAN_SLICED &&
        mode != BN_SCAN_SORTED)
        return set_error(BN_EINVAL, "bn_table_set_scan: mode %d", mode);
    if ((mode == BN_SCAN_SLICED || mode == BN_SCAN_SORTED) && !t->sset)
        return set_error(BN_EUNSUPPORTED, "bn_table_set_scan: the bit-sliced scans need k <= 4 (k = %d)", t->k);
    if (mode == BN_SCAN_PRUNED) {
        int rc = prune_table(t, (cudaStream_t)stream);
        if (rc) return rc;
    }
    t->scan_mode = mode;
    return BN_OK;
}

extern "C" int bn_table_pruned(const bn_table* t, int64_t* survivors_per_node)
{
    set_error(BN_OK, "");
    if (!t || !survivors_per_node) return set_error(BN_EINVAL, "bn_table_pruned: NULL argument");
    if (!t->amask) return set_error(BN_EINVAL, "bn_table_pruned: the table has not been pruned");
    std::vector<uint32_t> h(t->n);
    BN_CUDA(cudaMemcpy(h.data(), t->acnt, 4 * (size_t)t->n, cudaMemcpyDeviceToHost));
    for (int i = 0; i < t->n; ++i) survivors_per_node[i] = h[i];
    return BN_OK;
}
