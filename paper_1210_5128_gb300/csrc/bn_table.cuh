// bn_table.cuh -- the device-resident local-score table shared by the scan and the sampler.
#pragma once

#include "bn_internal.cuh"

struct bn_table {
    int n = 0, k = 0, dev = 0;
    int64_t S = 0;            // parent sets per node, S(n-1, k)
    int64_t Sp = 0;           // per-node stride, S rounded up to a multiple of SUBQ
    int64_t* keys = nullptr;  // [n][Sp] order-preserving keys of the FP64 entries;
                              // padding entries hold KEY_NONE
    uint64_t* pst = nullptr;  // [Sp] candidate-space mask of each rank (padding: ~0)
    size_t bytes = 0;
};

namespace bn {

// Scratch-free bits of the order scan used by bn_score_orders and the sampler.
struct ScanPlan {
    int nchunk;        // blocks per node along the table
    int64_t chunk;     // entries per block (multiple of SUBQ)
    int sub;           // entries per shared-memory stage
    int stages;
    int group;         // orders per block (threads)
};
ScanPlan plan_scan(const bn_table* t, int max_items);

struct ScanPartial {
    int64_t key;
    uint32_t rank;
    uint32_t pad;
};

// Scan all list items of every node against the table:
//   list_count[i]             number of items of node i
//   list_pc[i * cap + j]      candidate-space predecessor mask of item j of node i
//   part[(i * cap + j) * nchunk + c]  best (key, rank) of item j over chunk c
int launch_scan(const bn_table* t, const ScanPlan& pl, const uint32_t* list_count,
                const uint64_t* list_pc, int cap, ScanPartial* part, uint32_t* status,
                cudaStream_t s);

// candidate-space predecessor masks of B orders written as node-major work lists:
// list_pc[i * B + b] (item b of node i is order b), list_count[i] = B; rows that are not
// permutations of 0..n-1 set STATUS_BADINPUT
int launch_pred_lists(const uint8_t* orders, int B, int n, uint64_t* list_pc, uint32_t* list_count,
                      uint32_t* status, cudaStream_t s);

}  // namespace bn
