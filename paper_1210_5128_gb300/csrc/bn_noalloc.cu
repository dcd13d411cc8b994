// bn_noalloc.cu -- bn_score_orders_noalloc: order scoring that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they score orders: a
// host framework that owns all device memory through its own pool and forbids other
// allocations, a latency-critical loop that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree, or a plugin whose host hands it
// pre-allocated input and output buffers only.  This entry point serves them: the
// work lists and per-chunk partial results the scan needs live in one file-scope
// __device__ array (SCRATCH_BYTES, below), which every GPU that loads the library
// holds until the process exits.
#include <algorithm>
#include <mutex>

#include "bn_table.cuh"

namespace bn {

static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;   // 8 MiB

static __device__ __align__(256) uint8_t g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Per-device address of g_noalloc_scratch.  In host code the array's name is only a
// host-side stand-in for the symbol, never a device address, so it is resolved once per
// device with that device current.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

static int noalloc_scratch(void** out)
{
    const int d = device_id();
    if (d < 0 || d >= 64) return set_error(BN_EUNSUPPORTED, "bn_score_orders_noalloc: device id %d", d);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[d]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_noalloc_ptr[d] = p;
    }
    *out = g_noalloc_ptr[d];
    return BN_OK;
}

__global__ void k_noalloc_reduce(const uint32_t* __restrict__ list_best, const uint32_t* __restrict__ srank,
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

extern "C" int bn_score_orders_noalloc(const bn_table* t, const uint8_t* orders, int B, uint32_t* best_rank,
                                       double* order_score, void* stream)
{
    set_error(BN_OK, "");
    if (!t) return set_error(BN_EINVAL, "bn_score_orders_noalloc: NULL table");
    if (B < 0) return set_error(BN_EINVAL, "bn_score_orders_noalloc: B=%d", B);
    if (B == 0) return BN_OK;
    if (!orders) return set_error(BN_EINVAL, "bn_score_orders_noalloc: orders is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = t->n;

    // scratch: status | counts | predecessor masks | per-item results
    const size_t o_status = 0;
    const size_t o_cnt = 256;
    const size_t o_pc = (size_t)round_up((int64_t)(o_cnt + sizeof(uint32_t) * n), 256);
    const size_t o_best = (size_t)round_up((int64_t)(o_pc + sizeof(uint64_t) * (size_t)n * B), 256);
    const size_t need = o_best + sizeof(uint32_t) * (size_t)n * B;
    if (need > NOALLOC_SCRATCH_BYTES)
        return set_error(BN_EINVAL,
                         "bn_score_orders_noalloc: B=%d orders of n=%d nodes need %zu bytes of scratch; the "
                         "static scratch holds %zu (at most %zu orders at this n)",
                         B, n, need, NOALLOC_SCRATCH_BYTES, (NOALLOC_SCRATCH_BYTES - 1024 - 4 * (size_t)n) / (12 * (size_t)n));
    const ScanPlan pl = plan_scan(t, B);

    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    uint8_t* sb = (uint8_t*)base;
    uint32_t* d_status = (uint32_t*)(sb + o_status);
    uint32_t* d_cnt = (uint32_t*)(sb + o_cnt);
    uint64_t* d_pc = (uint64_t*)(sb + o_pc);
    uint32_t* d_best = (uint32_t*)(sb + o_best);

    // the array keeps the previous call's contents: the status word must start at zero;
    // counts, masks and per-item results are rewritten by k_pred_lists before use
    BN_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    if ((rc = launch_pred_lists(orders, B, n, d_pc, d_best, d_cnt, d_status, s))) return rc;
    rc = scan_nodes_fits(t, B) ? launch_scan_nodes(t, B, d_pc, d_best, d_status, s)
                               : launch_scan(t, pl, d_cnt, d_pc, d_best, B, d_status, s);
    if (rc) return rc;
    k_noalloc_reduce<<<(B + 7) / 8, 256, 0, s>>>(d_best, t->srank, t->keys, t->Sp, n, B, best_rank, order_score);
    BN_LAUNCH_CHECK("k_noalloc_reduce");
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_BADINPUT) return set_error(BN_EINVAL, "bn_score_orders_noalloc: an order is not a permutation");
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_score_orders_noalloc: a bounded device wait expired");
    return BN_OK;
}
