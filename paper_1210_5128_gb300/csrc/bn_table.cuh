// bn_table.cuh -- the device-resident local-score table shared by the scan and the sampler.
#pragma once

#include "bn_internal.cuh"

struct bn_table {
    int n = 0, k = 0, dev = 0;
    int64_t S = 0;             // parent sets per node, S(n-1, k)
    int64_t Sp = 0;            // per-node stride, S rounded up to a multiple of SUBQ
    int64_t* keys = nullptr;   // [n][Sp] order-preserving keys of the FP64 entries, rank
                               // order; padding entries hold KEY_NONE
    uint64_t* pst = nullptr;   // [Sp] candidate-space mask of each rank (padding: ~0)
    uint32_t* spos = nullptr;  // [n][Sp] position of the entry when the node's entries are
                               // ordered by score descending, rank ascending (padding: ~0)
    uint32_t* srank = nullptr; // [n][Sp] inverse of spos: rank at sorted position p
    uint32_t* spos_t = nullptr;// [Sp / 2][n][2] spos entry-major, rank pairs side by side (k_scan_nodes)
    uint32_t* sset = nullptr;  // [n][sset_stride] parent node ids (a byte each) of the entry at each
                               // sorted position, k <= 4 only (bn_sliced.cu); null otherwise
    int64_t sset_stride = 0;   // S rounded up to whole stages of the sliced scan
    uint32_t cut[64] = {0};    // per node: sorted position of the empty set + 1 (host copy); no
                               // entry at or past it can be a node's best
    size_t bytes = 0;
    int scan_mode = 0;         // BN_SCAN_FULL, _PRUNED, _UNRANK, _SLICED or _SORTED
    // entries not dominated by a proper subset, per node in sorted-position order
    // (bn_prune.cu): candidate masks and sorted positions, node offsets and counts
    uint64_t* amask = nullptr;
    uint32_t* aspos = nullptr;
    uint32_t* aoff = nullptr;
    uint32_t* acnt = nullptr;
    int64_t alive_total = 0;
    uint32_t alive_max = 0;
    int alive_chunks = 1;
    void* alive_block = nullptr;
    double max_abs_survivor = 0.0;   // largest |entry| among the survivors
    // the survivors in the fused sampler's cache layout (bn_mcmc.cu), in global memory, for
    // launches whose shared memory cannot hold them (null if the entries exceed its fixed
    // point)
    uint8_t* gcache = nullptr;
    // full-scan tiling chosen by bn_table_autotune, per number of 256-item groups (1..8);
    // tuned_sub == 0: not tuned
    int tuned_sub[9] = {0};
    int tuned_nchunk[9] = {0};
    int64_t tuned_chunk[9] = {0};
};

namespace bn {

// Sorted positions and their inverse for every node (bn_sort.cu).
int rank_entries(bn_table* t, cudaStream_t s);

// The bit-sliced scans (bn_sliced.cu): the parent sets in sorted-position order (k <= 4;
// nothing for larger k), and the scan of work lists in the layout of launch_scan, as a
// full pass (cut = false) or stopping early with identical results (cut = true).
int build_sset(bn_table* t, cudaStream_t s);
int launch_scan_sliced(const bn_table* t, const uint32_t* list_count, const uint64_t* list_pc, uint32_t* list_best,
                       int cap, bool cut, uint32_t* status, cudaStream_t s);

// Dominance pruning and the scan over the surviving entries (bn_prune.cu).
int prune_table(bn_table* t, cudaStream_t s);
// The survivors in the fused sampler's cache layout in global memory (t->gcache) when their
// entries fit its fixed point (bn_mcmc.cu).
int build_survivor_cache(bn_table* t, cudaStream_t s);
int launch_scan_pruned(const bn_table* t, const uint32_t* list_count, const uint64_t* list_pc, uint32_t* list_best,
                       int cap, cudaStream_t s);

struct ScanPlan {
    int nchunk;        // blocks per node along the table
    int64_t chunk;     // entries per block (multiple of SUBQ)
    int sub = 1024;    // entries per shared-memory stage (512, 1024 or 2048)
};
ScanPlan plan_scan(const bn_table* t, int max_items);
// tune the full-table scan's tiling for up to max_items items on first use (bn_scan.cu)
int ensure_tuned(const bn_table* t, int max_items, cudaStream_t s);

constexpr uint32_t SPOS_NONE = 0xffffffffu;

// Scan all list items of every node against the table (the consistent-max of Eq. (6)):
//   list_count[i]          number of items of node i
//   list_pc[i * cap + j]   candidate-space predecessor mask of item j of node i
//   list_best[i * cap + j] in: SPOS_NONE (set by the list builder);
//                          out: smallest sorted position among the consistent entries
int launch_scan(const bn_table* t, const ScanPlan& pl, const uint32_t* list_count,
                const uint64_t* list_pc, uint32_t* list_best, int cap, uint32_t* status,
                cudaStream_t s);

// The same for B orders of every node when n * ceil(B / 8) <= 1,024 and the table is
// scanned in full (scan_nodes_fits): one pass over the rank range for all nodes and
// orders, up to eight orders a thread (list layout [n][B]).
bool scan_nodes_fits(const bn_table* t, int B);
int launch_scan_nodes(const bn_table* t, int B, const uint64_t* list_pc, uint32_t* list_best, uint32_t* status,
                      cudaStream_t s);

// Candidate-space predecessor masks of B orders written as node-major work lists:
// list_pc[i * B + b] (item b of node i is order b), list_best[i * B + b] = SPOS_NONE,
// list_count[i] = B; rows that are not permutations of 0..n-1 set STATUS_BADINPUT.
int launch_pred_lists(const uint8_t* orders, int B, int n, uint64_t* list_pc, uint32_t* list_best,
                      uint32_t* list_count, uint32_t* status, cudaStream_t s);

// a7: per order b, the chosen rank of every node (best_rank[b * n + i], may be null) and
// the FP64 sum over nodes, ascending node id, of their entries (score[b], may be null),
// from the scan's smallest sorted positions list_best[i * B + b]
int launch_reduce_orders(const bn_table* t, const uint32_t* list_best, int B, uint32_t* best_rank, double* score,
                         cudaStream_t s);

// best rank and FP64 entry of (node i, sorted position p)
__device__ __forceinline__ uint32_t spos_rank(const bn_table& t, int i, uint32_t p)
{
    return t.srank[(size_t)i * t.Sp + p];
}

}  // namespace bn
