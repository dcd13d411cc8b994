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

__global__ void k_noalloc_reduce(const ScanPartial* __restrict__ part, int n, int cap, int nchunk, int B,
                                 uint32_t* __restrict__ best_rank, double* __restrict__ score)
{
    __shared__ int64_t s_key[8][MAXN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + warp;
    if (b >= B) return;
    for (int i = lane; i < n; i += 32) {
        const ScanPartial* p = part + ((size_t)i * cap + b) * nchunk;
        int64_t bk = KEY_NONE;
        uint32_t br = 0xffffffffu;
        for (int c = 0; c < nchunk; ++c) {
            const ScanPartial q = p[c];
            if (q.key > bk || (q.key == bk && q.rank < br)) { bk = q.key; br = q.rank; }
        }
        s_key[warp][i] = bk;
        if (best_rank) best_rank[(size_t)b * n + i] = br;
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

    // fixed part of the scratch: status | counts | predecessor masks; the rest holds the
    // partials, so the chunking is coarsened until they fit
    const size_t o_status = 0;
    const size_t o_cnt = 256;
    const size_t o_pc = (size_t)round_up((int64_t)(o_cnt + sizeof(uint32_t) * n), 256);
    const size_t o_part = (size_t)round_up((int64_t)(o_pc + sizeof(uint64_t) * (size_t)n * B), 256);
    const size_t per_chunk = sizeof(ScanPartial) * (size_t)n * B;
    if (o_part + per_chunk > NOALLOC_SCRATCH_BYTES)
        return set_error(BN_EINVAL,
                         "bn_score_orders_noalloc: B=%d orders of n=%d nodes need %zu bytes of scratch; the "
                         "static scratch holds %zu (at most %zu orders at this n)",
                         B, n, o_part + per_chunk, NOALLOC_SCRATCH_BYTES,
                         (NOALLOC_SCRATCH_BYTES - 1024 - 4 * (size_t)n) / ((sizeof(ScanPartial) + 8) * (size_t)n));
    ScanPlan pl = plan_scan(t, B);
    const int64_t max_chunks = (int64_t)((NOALLOC_SCRATCH_BYTES - o_part) / per_chunk);
    if (pl.nchunk > max_chunks) {
        pl.chunk = round_up((t->Sp + max_chunks - 1) / max_chunks, SUBQ);
        pl.nchunk = (int)((t->Sp + pl.chunk - 1) / pl.chunk);
    }

    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    uint8_t* sb = (uint8_t*)base;
    uint32_t* d_status = (uint32_t*)(sb + o_status);
    uint32_t* d_cnt = (uint32_t*)(sb + o_cnt);
    uint64_t* d_pc = (uint64_t*)(sb + o_pc);
    ScanPartial* d_part = (ScanPartial*)(sb + o_part);

    // the array keeps the previous call's contents: the status word must start at zero;
    // counts, masks and partials are fully rewritten before they are read
    BN_CUDA(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
    if ((rc = launch_pred_lists(orders, B, n, d_pc, d_cnt, d_status, s))) return rc;
    if ((rc = launch_scan(t, pl, d_cnt, d_pc, B, d_part, d_status, s))) return rc;
    k_noalloc_reduce<<<(B + 7) / 8, 256, 0, s>>>(d_part, n, B, pl.nchunk, B, best_rank, order_score);
    BN_LAUNCH_CHECK("k_noalloc_reduce");
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_BADINPUT) return set_error(BN_EINVAL, "bn_score_orders_noalloc: an order is not a permutation");
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_score_orders_noalloc: a bounded device wait expired");
    return BN_OK;
}
