// bn_sort.cu -- per-node ranking of the table entries for the scan.
//
// Every entry (i, rho) gets spos[i][rho]: its position when node i's entries are ordered
// by score descending, ties by rank ascending.  spos is unique within a node and
// "smaller spos" means "higher score, or equal score and lower rank", so the order-score
// scan's (max score, lowest rank) reduction becomes a single unsigned min over spos.
// srank[i][p] is the inverse (the rank at sorted position p).
//
// The ordering is a stable least-significant-digit radix sort (8-bit digits) of
// (node, ~key) with the global index as value: eight passes over the 64-bit
// order-inverted score keys, then one over the node, each pass = digit histogram per
// tile, per-digit scan over tiles, stable scatter.  Input order is (node, rank), so
// stability keeps equal scores in rank order.
#include <algorithm>
#include <vector>

#include "bn_table.cuh"

namespace bn {

static constexpr int RS_THREADS = 256;
static constexpr int RS_ROUNDS = 16;
static constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096 elements per tile

struct RsPass {
    const uint64_t* kin;
    const uint32_t* vin;
    uint64_t* kout;
    uint32_t* vout;
    int64_t N;
    int shift;          // digit = (key >> shift) & 255, or the node (value / S) when < 0
    int64_t S;
    int node0;          // first node of this batch
    uint32_t* counts;   // [256][T]
    uint32_t* totals;   // [256]
    int T;
};

__device__ __forceinline__ int rs_digit(const RsPass& P, uint64_t k, uint32_t v)
{
    return P.shift >= 0 ? (int)((k >> P.shift) & 255ull) : (int)(v / (uint32_t)P.S);
}

__global__ void k_rs_init(const int64_t* __restrict__ keys, int64_t Sp, int64_t S, int node0, int64_t N,
                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const int64_t i = g / S, r = g - i * S;
    const uint64_t u = (uint64_t)keys[(node0 + i) * Sp + r] ^ 0x8000000000000000ull;  // ascending as unsigned
    kout[g] = ~u;                                                                        // descending score
    vout[g] = (uint32_t)g;
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(RsPass P)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t e = base + (int64_t)r * RS_THREADS + threadIdx.x;
        if (e < P.N) atomicAdd(&h[rs_digit(P, P.kin[e], P.vin[e])], 1u);
    }
    __syncthreads();
    P.counts[(size_t)threadIdx.x * P.T + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of counts[d][0..T) for one digit d per block; totals[d] = the sum
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t* __restrict__ counts, int T, uint32_t* __restrict__ totals)
{
    __shared__ uint32_t part[1024];
    uint32_t* c = counts + (size_t)blockIdx.x * T;
    const int per = (T + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(T, b + per);
    uint32_t s = 0;
    for (int j = b; j < e; ++j) s += c[j];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;   // exclusive prefix of this thread's range
    for (int j = b; j < e; ++j) {
        const uint32_t v = c[j];
        c[j] = run;
        run += v;
    }
    if (threadIdx.x == 1023) totals[blockIdx.x] = part[1023];
}

// stable scatter of one tile: round-major order (element base + r*256 + t), ranks
// within a round from warp match groups plus the earlier warps' counts of the digit
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(RsPass P)
{
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_w[RS_THREADS / 32][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        // digit base = exclusive scan of totals (256 values, Hillis-Steele in shared)
        __shared__ uint32_t t[256];
        const uint32_t mine = P.totals[threadIdx.x];
        t[threadIdx.x] = mine;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            uint32_t v = threadIdx.x >= off ? t[threadIdx.x - off] : 0u;
            __syncthreads();
            t[threadIdx.x] += v;
            __syncthreads();
        }
        s_run[threadIdx.x] = t[threadIdx.x] - mine + P.counts[(size_t)threadIdx.x * P.T + blockIdx.x];
    }
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        for (int j = threadIdx.x; j < (RS_THREADS / 32) * 256; j += RS_THREADS) (&s_w[0][0])[j] = 0u;
        __syncthreads();
        const int64_t e = base + (int64_t)r * RS_THREADS + threadIdx.x;
        const bool valid = e < P.N;
        uint64_t k = 0;
        uint32_t v = 0;
        int d = 256;                                  // sentinel for the tail
        if (valid) {
            k = P.kin[e];
            v = P.vin[e];
            d = rs_digit(P, k, v);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lrank = (uint32_t)__popc(peers & lt);
        if (valid && lrank == 0) s_w[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = s_run[d] + lrank;
            for (int w = 0; w < warp; ++w) off += s_w[w][d];
            P.kout[off] = k;
            P.vout[off] = v;
        }
        __syncthreads();
        {
            uint32_t add = 0;
            for (int w = 0; w < RS_THREADS / 32; ++w) add += s_w[w][threadIdx.x];
            s_run[threadIdx.x] += add;
        }
        __syncthreads();
    }
}

__global__ void k_rs_finish(const uint32_t* __restrict__ vals, int64_t N, int64_t S, int64_t Sp, int node0,
                            uint32_t* __restrict__ srank, uint32_t* __restrict__ spos)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const int64_t i = g / S, p = g - i * S;      // sorted by node first: position p of node i
    const uint32_t v = vals[g];
    const int64_t r = (int64_t)v - i * S;
    srank[(node0 + i) * Sp + p] = (uint32_t)r;
    spos[(node0 + i) * Sp + r] = (uint32_t)p;
}

// spos_t[r / 2][i][r % 2] = spos[i][r]: 32 x 32 tiles through shared memory, a thread
// storing the two positions of a rank pair of one node as one 8-byte word (coalesced both
// ways)
__global__ void k_spos_transpose(const uint32_t* __restrict__ spos, int n, int64_t Sp, uint32_t* __restrict__ spos_t)
{
    __shared__ uint32_t tile[32][33];                      // [node][rank]
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8 threads
    for (int y = ty; y < 32; y += 8) {
        const int i = i0 + y;
        if (i < n) tile[y][tx] = spos[(size_t)i * Sp + r0 + tx];
    }
    __syncthreads();
    uint2* out = (uint2*)spos_t;
    for (int y2 = ty; y2 < 16; y2 += 8) {
        const int i = i0 + tx;
        if (i < n) out[(size_t)(r0 / 2 + y2) * n + i] = make_uint2(tile[tx][2 * y2], tile[tx][2 * y2 + 1]);
    }
}

__global__ void k_spos_pad(uint32_t* __restrict__ spos, uint32_t* __restrict__ srank, int n, int64_t S, int64_t Sp)
{
    const int64_t pad = Sp - S;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * pad) return;
    const int64_t i = idx / pad, e = idx - i * pad;
    spos[i * Sp + S + e] = 0xffffffffu;
    srank[i * Sp + S + e] = 0u;
}

// Ranks every node's entries (see the file comment).  Temporaries are stream-ordered.
int rank_entries(bn_table* t, cudaStream_t s)
{
    const int64_t S = t->S;
    if (S > 0xffffffffLL) return set_error(BN_EUNSUPPORTED, "rank_entries: too many sets per node");
    // nodes per batch so that batch * S fits the 32-bit value
    const int per = (int)std::max<int64_t>(1, std::min<int64_t>(t->n, 0x7fffffffLL / S));
    const int64_t Nmax = (int64_t)per * S;
    const int Tmax = (int)((Nmax + RS_TILE - 1) / RS_TILE);
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *counts = nullptr, *totals = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&k0, 8 * (size_t)Nmax, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&k1, 8 * (size_t)Nmax, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&v0, 4 * (size_t)Nmax, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&v1, 4 * (size_t)Nmax, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&counts, 4 * (size_t)256 * Tmax, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&totals, 4 * 256, s);
    struct F {
        cudaStream_t s;
        void* p[6];
        ~F()
        {
            for (void* q : p)
                if (q) cudaFreeAsync(q, s);
        }
    } fr{s, {k0, k1, v0, v1, counts, totals}};
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BN_ENOMEM, "rank_entries: %zu bytes of sort buffers: %s", (size_t)Nmax * 24,
                         cudaGetErrorString(e));
    }
    for (int node0 = 0; node0 < t->n; node0 += per) {
        const int nb = std::min(per, t->n - node0);
        const int64_t N = (int64_t)nb * S;
        const int T = (int)((N + RS_TILE - 1) / RS_TILE);
        k_rs_init<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(t->keys, t->Sp, S, node0, N, k0, v0);
        BN_LAUNCH_CHECK("k_rs_init");
        uint64_t *ki = k0, *ko = k1;
        uint32_t *vi = v0, *vo = v1;
        for (int pass = 0; pass < 9; ++pass) {
            RsPass P;
            P.kin = ki;
            P.vin = vi;
            P.kout = ko;
            P.vout = vo;
            P.N = N;
            P.shift = pass < 8 ? 8 * pass : -1;
            P.S = S;
            P.node0 = node0;
            P.counts = counts;
            P.totals = totals;
            P.T = T;
            if (pass == 8 && nb == 1) break;        // a single node needs no node pass
            k_rs_hist<<<T, RS_THREADS, 0, s>>>(P);
            BN_LAUNCH_CHECK("k_rs_hist");
            k_rs_scan<<<256, 1024, 0, s>>>(counts, T, totals);
            BN_LAUNCH_CHECK("k_rs_scan");
            k_rs_scatter<<<T, RS_THREADS, 0, s>>>(P);
            BN_LAUNCH_CHECK("k_rs_scatter");
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
        k_rs_finish<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(vi, N, S, t->Sp, node0, t->srank, t->spos);
        BN_LAUNCH_CHECK("k_rs_finish");
    }
    if (t->Sp > S) {
        const int64_t tot = (int64_t)t->n * (t->Sp - S);
        k_spos_pad<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(t->spos, t->srank, t->n, S, t->Sp);
        BN_LAUNCH_CHECK("k_spos_pad");
    }
    k_spos_transpose<<<dim3((unsigned)(t->Sp / 32), (unsigned)((t->n + 31) / 32)), dim3(32, 8), 0, s>>>(t->spos, t->n, t->Sp,
                                                                                                    t->spos_t);
    BN_LAUNCH_CHECK("k_spos_transpose");
    return build_sset(t, s);
}

}  // namespace bn
