// bn_sum.cu -- the sum-based order score of the prior scorer the paper compares its own
// against (Sec. III.B): log10 of the sum over every graph consistent with an order of
// 10^(graph score), which factorises over nodes into
//     sum_i log10 sum_{parent sets pi of i drawn from its predecessors} 10^entry(i, pi).
// The paper's argument against it is its cost (exponentials and logarithms instead of
// comparisons) and that its best order need not carry the best graph; this scan makes the
// first point measurable on the same table and the same hardware.
//
// A block owns a chunk of one node's table and up to SUM_OB orders: every thread streams
// entries (FP64 entry from the order-preserving key, candidate mask from the parent-set
// table) and keeps, per order, a running (max m, sum of 10^(entry - m)) over the
// consistent entries; warps, then the block, then the chunks merge those pairs in a
// fixed order, so results are deterministic for a given launch shape.
#include <algorithm>
#include <cmath>

#include "bn_table.cuh"

namespace bn {

static constexpr int SUM_OB = 8;          // orders per pass
static constexpr int SUM_THREADS = 256;

struct SumScanArgs {
    const int64_t* keys;
    const uint64_t* pst;
    int64_t Sp;
    int n, B, b0, nb;                     // all orders, the pass's first and count
    int nchunk;
    int64_t chunk;
    const uint64_t* list_pc;              // [n][B] candidate-space predecessor masks
    double2* part;                        // [n][B][nchunk] (m, sum)
};

// (m, s) += 10^v
__device__ __forceinline__ void lse_push(double& m, double& s, double v)
{
    if (v > m) {
        s = s * exp10(m - v) + 1.0;       // m = -inf: 0 * 0 + 1
        m = v;
    } else {
        s += exp10(v - m);
    }
}

// (m, s) += (m2, s2)
__device__ __forceinline__ void lse_merge(double& m, double& s, double m2, double s2)
{
    if (s2 == 0.0) return;
    if (s == 0.0) {
        m = m2;
        s = s2;
        return;
    }
    if (m2 > m) {
        s = s * exp10(m - m2) + s2;
        m = m2;
    } else {
        s += s2 * exp10(m2 - m);
    }
}

__global__ void __launch_bounds__(SUM_THREADS) k_scan_sum(SumScanArgs A)
{
    __shared__ double s_m[SUM_THREADS / 32][SUM_OB], s_s[SUM_THREADS / 32][SUM_OB];
    const int node = blockIdx.x / A.nchunk, chunk = blockIdx.x - node * A.nchunk;
    const int64_t e0 = (int64_t)chunk * A.chunk, e1 = min(e0 + A.chunk, A.Sp);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t npc[SUM_OB];
    double m[SUM_OB], s[SUM_OB];
#pragma unroll
    for (int b = 0; b < SUM_OB; ++b) {
        npc[b] = b < A.nb ? ~A.list_pc[(size_t)node * A.B + A.b0 + b] : ~0ull;
        m[b] = -INFINITY;
        s[b] = 0.0;
    }
    const int64_t* K = A.keys + (size_t)node * A.Sp;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += SUM_THREADS) {
        const uint64_t mask = __ldg(&A.pst[e]);
        const double v = key_to_double(K[e]);
#pragma unroll
        for (int b = 0; b < SUM_OB; ++b)
            if (b < A.nb && (mask & npc[b]) == 0ull) lse_push(m[b], s[b], v);
    }
#pragma unroll
    for (int b = 0; b < SUM_OB; ++b) {
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            const double m2 = __shfl_down_sync(0xffffffffu, m[b], off);
            const double s2 = __shfl_down_sync(0xffffffffu, s[b], off);
            lse_merge(m[b], s[b], m2, s2);
        }
        if (lane == 0) {
            s_m[warp][b] = m[b];
            s_s[warp][b] = s[b];
        }
    }
    __syncthreads();
    if (threadIdx.x < A.nb) {
        const int b = threadIdx.x;
        double mm = -INFINITY, ss = 0.0;
        for (int w = 0; w < SUM_THREADS / 32; ++w) lse_merge(mm, ss, s_m[w][b], s_s[w][b]);
        A.part[((size_t)node * A.B + A.b0 + b) * A.nchunk + chunk] = make_double2(mm, ss);
    }
}

// chunks in order, then nodes in ascending id
__global__ void k_sum_finish(const double2* __restrict__ part, int n, int B, int nchunk,
                             double* __restrict__ node_score, double* __restrict__ order_score)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        double mm = -INFINITY, ss = 0.0;
        for (int c = 0; c < nchunk; ++c) {
            const double2 p = part[((size_t)i * B + b) * nchunk + c];
            lse_merge(mm, ss, p.x, p.y);
        }
        const double v = mm + log10(ss);
        if (node_score) node_score[(size_t)b * n + i] = v;
        total += v;
    }
    if (order_score) order_score[b] = total;
}

}  // namespace bn

using namespace bn;

extern "C" int bn_score_orders_sum(const bn_table* t, const uint8_t* orders, int B, double* order_score,
                                   double* node_score, int mem, void* stream)
{
    set_error(BN_OK, "");
    if (!t) return set_error(BN_EINVAL, "bn_score_orders_sum: NULL table");
    if (B < 0) return set_error(BN_EINVAL, "bn_score_orders_sum: B=%d", B);
    if (mem != BN_MEM_HOST && mem != BN_MEM_DEVICE) return set_error(BN_EINVAL, "bn_score_orders_sum: bad mem");
    if (B == 0) return BN_OK;
    if (!orders) return set_error(BN_EINVAL, "bn_score_orders_sum: orders is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = t->n;
    // chunks per node: about two blocks per SM in all
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(t->Sp / SUBQ, (int64_t)sm_count() * 2 / n + 1));
    const int64_t chunk = round_up((t->Sp + nchunk - 1) / nchunk, SUBQ);
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
    const size_t o_part = take(sizeof(double2) * (size_t)n * B * nchunk);
    const size_t o_os = take(mem == BN_MEM_HOST && order_score ? sizeof(double) * B : 0);
    const size_t o_ns = take(mem == BN_MEM_HOST && node_score ? sizeof(double) * (size_t)B * n : 0);
    uint8_t* base = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&base, off, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BN_ENOMEM, "bn_score_orders_sum: scratch of %zu bytes: %s", off, cudaGetErrorString(e));
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
    uint32_t* d_st = (uint32_t*)(base + o_st);
    double2* d_part = (double2*)(base + o_part);
    double* d_os = mem == BN_MEM_HOST ? (order_score ? (double*)(base + o_os) : nullptr) : order_score;
    double* d_ns = mem == BN_MEM_HOST ? (node_score ? (double*)(base + o_ns) : nullptr) : node_score;
    BN_CUDA(cudaMemsetAsync(d_st, 0, sizeof(uint32_t), s));
    int rc = launch_pred_lists(d_orders, B, n, d_pc, (uint32_t*)(base + o_best), (uint32_t*)(base + o_cnt), d_st, s);
    if (rc) return rc;
    for (int b0 = 0; b0 < B; b0 += SUM_OB) {
        SumScanArgs A{t->keys, t->pst, t->Sp, n, B, b0, std::min(SUM_OB, B - b0), nchunk, chunk, d_pc, d_part};
        k_scan_sum<<<(unsigned)(n * nchunk), SUM_THREADS, 0, s>>>(A);
        BN_LAUNCH_CHECK("k_scan_sum");
    }
    k_sum_finish<<<(B + 127) / 128, 128, 0, s>>>(d_part, n, B, nchunk, d_ns, d_os);
    BN_LAUNCH_CHECK("k_sum_finish");
    if (mem == BN_MEM_HOST) {
        if (order_score) BN_CUDA(cudaMemcpyAsync(order_score, d_os, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
        if (node_score)
            BN_CUDA(cudaMemcpyAsync(node_score, d_ns, sizeof(double) * (size_t)B * n, cudaMemcpyDeviceToHost, s));
    }
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, d_st, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_BADINPUT) return set_error(BN_EINVAL, "bn_score_orders_sum: an order is not a permutation of 0..n-1");
    return BN_OK;
}
