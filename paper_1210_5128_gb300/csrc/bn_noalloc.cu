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
// host-side stand-in for the symbol, never a device address, so the address is looked up
// with the device current and kept per device together with the identity of the CUDA
// context it belongs to: a context destroyed and created again (cudaDeviceReset, or the
// primary context released and retained anew) has a new identity, and the address is
// looked up again.  Without the driver's context identity the lookup runs on every call.
struct NoallocSlot {
    unsigned long long ctx = 0;
    void* ptr = nullptr;
};
static std::mutex g_noalloc_mu;
static NoallocSlot g_noalloc_slot[64];

static int noalloc_scratch(void** out)
{
    const int d = device_id();
    if (d < 0 || d >= 64) return set_error(BN_EUNSUPPORTED, "bn_score_orders_noalloc: device id %d", d);
    const unsigned long long ctx = context_id();
    const bool known = ctx != 0;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    NoallocSlot& slot = g_noalloc_slot[d];
    if (!known || !slot.ptr || slot.ctx != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        slot.ctx = ctx;
        slot.ptr = p;
    }
    *out = slot.ptr;
    return BN_OK;
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
    if ((rc = launch_reduce_orders(t, d_best, B, best_rank, order_score, s))) return rc;
    uint32_t st = 0;
    BN_CUDA(cudaMemcpyAsync(&st, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    BN_CUDA(cudaStreamSynchronize(s));
    if (st & STATUS_BADINPUT) return set_error(BN_EINVAL, "bn_score_orders_noalloc: an order is not a permutation");
    if (st & STATUS_TIMEOUT) return set_error(BN_ETIMEOUT, "bn_score_orders_noalloc: a bounded device wait expired");
    return BN_OK;
}
