/*
 * bn.h -- C ABI of the GB300 order-space Bayesian-network scorer.
 *
 * The library implements the data-parallel hot path of the order-space MCMC learner of
 * Wang, Zhang, Qian and Yuan, "A Novel Learning Algorithm for Bayesian Network and Its
 * Efficient Implementation on GPU" (arXiv:1210.5128):
 *   - the local-score table of every (node, parent set of size <= k)     Sec. III.A, Eq. (3)-(4)
 *     with the pairwise prior folded in                                  Sec. IV, Eq. (9)-(10)
 *   - the order score: per node the best parent set drawn from its
 *     predecessors, summed over nodes                                    Sec. III.B, Eq. (6)
 *   - the Metropolis-Hastings swap sampler and best-graph tracking       Sec. III.C, Algorithm 1
 * All compute runs in CUDA kernels for sm_103a; every entry point is synchronous with
 * respect to the stream it is given (it returns after its work on that stream is done).
 *
 * Conventions shared by every entry point
 *   - Return value: BN_OK (0) or a negative BN_E* code; bn_last_error() then holds a
 *     one-line message for the calling thread.  No entry point aborts the process.
 *   - `mem` says where the caller's array arguments live: BN_MEM_HOST (ordinary or
 *     pinned host memory) or BN_MEM_DEVICE (device memory of the current device, e.g. a
 *     torch tensor's data_ptr()).  All array arguments of one call use the same `mem`.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Nodes are numbered 0..n-1, 2 <= n <= 64.  Parent sets of node i live in its
 *     "candidate space": slot c (0 <= c < n-1) stands for node c + (c >= i).
 *   - A parent set's rank orders all subsets of size <= k of the n-1 candidate slots:
 *     sizes ascending (the empty set is rank 0), and within one size the
 *     combinatorial number system, rank {a_1 < ... < a_j} = sum_t C(a_t, t)
 *     (Sec. V.B asks for such a regular, invertible indexing; this is the choice made).
 *     S(n-1, k) = sum_{j<=k} C(n-1, j) sets per node (Sec. III.B).
 *   - Ties between equal local scores always go to the lowest rank.
 *   - Orders are arrays of n node ids, position -> node.
 */
#ifndef BN_H
#define BN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BN_OK            0
#define BN_EINVAL       -1   /* invalid argument (sizes, values, NaN, NULL) */
#define BN_ENOMEM       -2   /* a device or host allocation failed */
#define BN_ECUDA        -3   /* a CUDA runtime call failed (message has the CUDA error) */
#define BN_ETIMEOUT     -4   /* a bounded device-side wait expired; the kernel gave up */
#define BN_EUNSUPPORTED -5   /* valid request outside the library's limits */

#define BN_MEM_HOST   0
#define BN_MEM_DEVICE 1

/* ---------------------------------------------------------------------------------- */
/* Local-score table                                                                   */
/* ---------------------------------------------------------------------------------- */

typedef struct bn_table bn_table;   /* opaque, device-resident, owned by the library */

typedef struct {
    int    score_kind;   /* 0 = K2 (alpha_cx = 1, alpha_c = r_i); 1 = BDeu(ess)          */
    double ess;          /* BDeu equivalent sample size (> 0); ignored for K2           */
    double log10_gamma;  /* log10 of the structure penalty gamma of Eq. (3); 0 = none   */
} bn_score_params;

/* Build the local-score table of Eq. (4) plus the prior of Eq. (9) for every node and
 * every parent set of size <= k (the preprocessing step of Sec. III.A):
 *   entry(i, pi) = ls(i, pi) + sum_{m in pi} PPF(i, m),  PPF = 100 (R[i][m] - 0.5)^3.
 *   data   m x n uint8, row-major, data[r*n + i] < arity[i]   (m >= 0; complete data)
 *   arity  n uint8 in [2, 4]
 *   k      0 <= k <= n-1, and the per-node set count and q*r count table must fit
 *   R      n x n float64 in [0, 1], R[i*n + m] = prior belief in the edge m -> i
 *          (Sec. IV: 0.5 = no bias); NULL = 0.5 everywhere; the diagonal is ignored
 *   params NULL = K2 with gamma = 1
 * Scores are FP64.  Counts are exact integers; the lgamma terms of one entry are summed
 * exactly (128-bit fixed point) before one rounding to FP64.
 * Errors: BN_EINVAL for n, k, arity, data or R out of range (R NaN included);
 * BN_EUNSUPPORTED if S(n-1,k) >= 2^31 or a count table needs more than 4096 cells;
 * BN_ENOMEM; BN_ECUDA.  On error *out is NULL. */
int bn_build_scores(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                    const double* R, const bn_score_params* params, int mem,
                    void* stream, bn_table** out);

/* bn_build_scores with the device time of its counting-and-scoring kernel (the table
 * build of Eq. (3)-(4), the call's dominant launch) measured by CUDA events on `stream`
 * around that launch: *build_ms receives it (build_ms may be NULL).  Outputs and errors as
 * bn_build_scores. */
int bn_build_scores_profiled(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                             const double* R, const bn_score_params* params, int mem,
                             void* stream, bn_table** out, double* build_ms);

/* bn_build_scores for `count` networks of uneven size in one call (many-network batches,
 * the paper learns one network at a time): network i has data[i] (m[i] x n[i]), arity[i],
 * k[i], R[i] (R may be NULL, or R[i] NULL: no prior) and params[i] (params may be NULL:
 * K2).  The host checks every network first; the builds then run concurrently on a few
 * internal streams that fork from and join into `stream`.  Each table equals the one
 * bn_build_scores builds from the same arguments, entry for entry.  out: count table
 * pointers (all NULL on error).  Errors: as bn_build_scores, the message naming the
 * network. */
int bn_build_scores_batch(int count, const uint8_t* const* data, const int* m, const int* n,
                          const uint8_t* const* arity, const int* k, const double* const* R,
                          const bn_score_params* params, int mem, void* stream, bn_table** out);

/* Wrap an existing table of scores (n x S(n-1,k) float64, node-major, rank order; the
 * layout bn_table_scores returns).  Used to score orders against an externally built
 * table.  Errors: BN_EINVAL (NaN or +inf scores, sizes), BN_ENOMEM, BN_ECUDA. */
int bn_table_from_scores(const double* scores, int n, int k, int mem, void* stream,
                         bn_table** out);

/* n, k, S(n-1,k) and the device bytes the table holds (any output may be NULL). */
int bn_table_info(const bn_table* t, int* n, int* k, int64_t* sets_per_node,
                  int64_t* device_bytes);

/* Copy out the S(n-1,k) FP64 scores of one node (rank order), or of all nodes when
 * node == -1 (n x S, node-major). */
int bn_table_scores(const bn_table* t, int node, double* out, int mem, void* stream);

void bn_table_free(bn_table* t);

/* ---------------------------------------------------------------------------------- */
/* Order scoring                                                                       */
/* ---------------------------------------------------------------------------------- */

/* Score B orders (Eq. (6), the scoring loop of Algorithm 1):
 *   orders      B x n uint8, each row a permutation of 0..n-1 (position -> node)
 *   best_rank   B x n uint32 out: best_rank[b*n + i] = rank of node i's best parent
 *               set among those drawn from its predecessors in order b (lowest rank
 *               among equal scores); its greedy best graph (Sec. III.B)
 *   order_score B float64 out: sum over nodes, ascending node id, of those entries
 * Either output may be NULL.  B = 0 is a no-op.  Scratch is allocated per call.
 * Errors: BN_EINVAL (not a permutation, B < 0), BN_ENOMEM, BN_ECUDA. */
int bn_score_orders(const bn_table* t, const uint8_t* orders, int B, uint32_t* best_rank,
                    double* order_score, int mem, void* stream);

/* bn_score_orders with the device time of its scan (the consistent-max kernel of Eq. (6),
 * the call's dominant launch) measured by CUDA events on `stream` around that launch:
 * *scan_ms receives it (0 for B = 0; scan_ms may be NULL).  Outputs and errors as
 * bn_score_orders. */
int bn_score_orders_profiled(const bn_table* t, const uint8_t* orders, int B, uint32_t* best_rank,
                             double* order_score, int mem, void* stream, double* scan_ms);

/* The sum-based order score of the prior scorer the paper compares its own against
 * (Sec. III.B): for each order, the log10 of the sum over all graphs consistent with it
 * of 10^(graph score) = sum_i log10 sum_{parent sets of node i drawn from its
 * predecessors} 10^entry(i, pi), in FP64.  Per (order, node) the consistent entries are
 * accumulated as a running (max, shifted sum); partial sums merge in a fixed order (the
 * result is deterministic for a table and a batch, not bit-equal to a sequential sum).
 *   orders      B x n uint8 permutations (position -> node)
 *   order_score B float64 out (may be NULL)
 *   node_score  B x n float64 out, [b][i] = node i's term (may be NULL)
 * Scratch is allocated per call.  Errors: BN_EINVAL, BN_ENOMEM, BN_ECUDA. */
int bn_score_orders_sum(const bn_table* t, const uint8_t* orders, int B, double* order_score,
                        double* node_score, int mem, void* stream);

/* bn_score_orders without any allocation.  The paper has no counterpart to this call.
 * It is for callers that cannot allocate device memory when they score orders: a host
 * framework whose memory pool owns the device and forbids outside allocations, a
 * latency-critical loop that cannot take the implicit device synchronisation of
 * cudaMalloc/cudaFree, a plugin handed pre-allocated buffers only.
 *   orders, best_rank, order_score: DEVICE pointers, same layouts as bn_score_orders
 *   (best_rank and order_score may be NULL).
 * The work lists and partial results live in one static 8 MiB device array that every
 * GPU loading the library holds until the process exits; B is limited to what fits
 * (about 8 MiB / (12 n) orders: 11,600 at n = 60), larger B returns BN_EINVAL with the
 * limit in the message.  Nothing is allocated or freed: no cudaMalloc, cudaFree or
 * allocating library routine.
 * The first call on each device (and the first after that device's CUDA context was
 * destroyed and created again) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call waits for its stream
 * (it reads a status word back), so it must not be made while the stream is being
 * captured.  All calls share the one array and it keeps the previous call's contents
 * (the call clears what must start at zero), so calls that overlap on the GPU (other
 * streams, other host threads) race: serialise them.
 * Errors: as bn_score_orders. */
int bn_score_orders_noalloc(const bn_table* t, const uint8_t* orders, int B,
                            uint32_t* best_rank, double* order_score, void* stream);

/* Scan mode of a table (used by bn_score_orders, bn_score_orders_noalloc and samplers
 * whose next step is captured after the change):
 *   BN_SCAN_FULL    every entry of a node's table is tested against every order (the
 *                   default; Eq. (6) taken literally)
 *   BN_SCAN_PRUNED  only entries that no proper subset of their parent set matches or
 *                   beats are tested.  A dominated entry can never be chosen: whenever
 *                   its set lies in a node's predecessors so does the subset, which has
 *                   a score at least as high and a lower rank.  Results are identical.
 *                   The surviving entries are kept in score order, so each order stops
 *                   at its first consistent one.  The first switch builds them (k <= 7),
 *                   with a copy laid out for the fused sampler (28 B per survivor plus
 *                   8 KB, device memory owned by the table).
 *   BN_SCAN_UNRANK  every entry, as BN_SCAN_FULL, but each parent set is computed from
 *                   its rank on the fly (the paper's first strategy, Sec. V.B / Algorithm
 *                   2, in this library's size-ascending combinatorial number system)
 *                   instead of read from the parent-set table.  Results are identical. 
 *   BN_SCAN_SLICED  every entry, as BN_SCAN_FULL, with the orders bit-sliced (k <= 4):
 *                   a node's entries are visited in score order (each entry's parent
 *                   nodes, a byte apiece, 4 B per entry from HBM) and for every group of
 *                   32 orders one word per parent node says in which of them that node
 *                   precedes the scored one; the AND of at most four such words tests an
 *                   entry against 32 orders, and an order takes the first consistent
 *                   entry, which is the (max score, lowest rank) one.  Results are
 *                   identical.
 *   BN_SCAN_SORTED  BN_SCAN_SLICED that stops early: no entry ranked below the empty
 *                   set (consistent with every order) is read, and a tile of orders
 *                   stops reading a node's entries once every order has its first
 *                   consistent one.  Results are identical.
 * Errors: BN_EINVAL (unknown mode), BN_ENOMEM, BN_EUNSUPPORTED (the sliced modes with
 * k > 4), BN_ECUDA. */
#define BN_SCAN_FULL   0
#define BN_SCAN_PRUNED 1
#define BN_SCAN_UNRANK 2
#define BN_SCAN_SLICED 3
#define BN_SCAN_SORTED 4
int bn_table_set_scan(bn_table* t, int mode, void* stream);
/* surviving entries per node after pruning (n int64) */
int bn_table_pruned(const bn_table* t, int64_t* survivors_per_node);

/* Autotuner of the full-table scan: times every (shared-memory stage size in
 * {512, 1024, 2048} entries) x (blocks per SM target in {1, 2, 4, 8, 16}) tiling on this
 * table with synthetic work lists of max_items (node, order) items per node, and keeps
 * the fastest for later scans of up to that many items (per 256-item group, up to 2048).
 * It also runs by itself: the first bn_score_orders call that takes the full-table scan
 * and the first bn_chains_create on a table not in BN_SCAN_PRUNED mode tune the tiling
 * for their number of 256-item groups (tens of milliseconds once per table and group
 * count; BN_AUTOTUNE=0 in the environment keeps the fixed tiling).  Results do not depend
 * on the tiling.
 * chosen (3 int64, may be NULL): stage size, blocks per node, microseconds per launch.
 * The table's scan mode is unchanged.  Errors: BN_EINVAL, BN_EUNSUPPORTED, BN_ECUDA. */
int bn_table_autotune(bn_table* t, int max_items, void* stream, int64_t* chosen);

/* Candidate-space mask of a rank and back (host-side helpers, no GPU needed).
 * mask bit c = candidate slot c.  Errors: BN_EINVAL if rank >= S(N,k) or the mask has
 * more than k bits or bits at or above N. */
int bn_unrank(int N, int k, int64_t rank, uint64_t* mask);
int bn_rank(int N, int k, uint64_t mask, int64_t* rank);

/* ---------------------------------------------------------------------------------- */
/* Metropolis-Hastings swap sampler                                                    */
/* ---------------------------------------------------------------------------------- */

typedef struct bn_chains bn_chains;  /* opaque, device-resident chain state */

/* Random numbers (one definition, key = {seed, 0}, Philox4x64-10):
 *   initial order of chain c: Fisher-Yates from the identity; for i = n-1..1 swap
 *     positions i and floor(x*(i+1)/2^64), x the next word of the blocks
 *     Philox(ctr = {j, c, 1, 0}), j = 0, 1, ...
 *   step t of chain c: x = Philox(ctr = {t, c, 0, 0}); the swapped positions are pair
 *     floor(x0 * P / 2^64) of the P = n(n-1)/2 pairs (a < b) in lexicographic order;
 *     u = ((x1 >> 12) + 0.5) 2^-52. */
typedef struct {
    int      chains;      /* independent chains, 1 .. 65536                             */
    int64_t  burn_in;     /* steps before edge counting starts                          */
    uint64_t seed;
    int      literal_log; /* 0: accept iff ln u < ln10 (s' - s)  (exact MH for the target
                             proportional to 10^score); 1: ln u < s' - s as printed     */
    int      record_every;/* >0: record every record_every-th post-burn-in state's edge
                             indicators for the ESS estimate; 0: off                     */
    int      record_cap;  /* max recorded states per chain (ESS series length)          */
    int      trace;       /* 1: keep per-step score and accept flag (chains x steps cap) */
    int64_t  trace_cap;   /* steps of trace kept per chain                              */
    /* bn_mcmc_run only (bn_chains_create and bn_batch_create ignore these):           */
    int      proposal;    /* BN_PROPOSAL_UNIFORM (0, the paper's swap) or
                             BN_PROPOSAL_LEARNED (1): train_iters uniform steps that train
                             the network (BN_PROPOSAL_TRAIN), then the sampling steps with
                             the learned proposal                                        */
    double   eps_mix;     /* learned: weight of the uniform component, in (0, 1]         */
    int64_t  train_iters; /* learned: training steps before the sampling steps           */
    int      thin;        /* > 0: record every thin-th post-burn-in state and fill the
                             ESS fields of bn_mcmc_stats; 0: no ESS                       */
    struct bn_mlp* net;   /* learned: the proposal network (its n, batch_cap >= chains);
                             NULL: the call creates one (d = 32, H = 512, Adam lr 2e-3,
                             weights drawn from seed) and frees it                        */
} bn_mcmc_params;

/* Create chains over a table.  init_orders: chains x n (NULL = Philox initial orders,
 * see above).  The table must outlive the chains. */
int bn_chains_create(const bn_table* t, const bn_mcmc_params* p, const uint8_t* init_orders,
                     int mem, void* stream, bn_chains** out);

/* Advance every chain by `steps` MH steps (Algorithm 1 iterations).  Each step
 * proposes a swap, re-scores only the nodes between the swapped positions (the
 * others keep their predecessor sets, so their best parent sets are unchanged),
 * applies the MH test, updates the best graph (strictly better replaces; candidates are
 * the initial and the accepted orders) and, after burn-in, the edge counts of the
 * current state's greedy DAG.  Steps are replayed from a captured CUDA graph; on a
 * pruned table (BN_SCAN_PRUNED) with the uniform proposal one fused kernel advances every
 * chain up to 1024 steps per launch instead, with identical results (it forms a step's
 * FP64 order score only where the MH test, a trace, the best state or the chain's saved
 * state needs it).  Synchronous with `stream`.
 * Errors: BN_ETIMEOUT, BN_ECUDA. */
int bn_chains_step(bn_chains* c, int64_t steps, void* stream);

/* bn_chains_step without the graph: the step's kernels are launched one by one on
 * `stream` and every scan launch (on the fused path: every fused launch) is bracketed by
 * a pair of CUDA events; *scan_ms receives the summed device time of those launches and
 * *scan_launches their number (either may be NULL).  Results are identical to
 * bn_chains_step. */
int bn_chains_step_profiled(bn_chains* c, int64_t steps, void* stream, double* scan_ms,
                            int64_t* scan_launches);

#define BN_OUT_ORDERS       1  /* chains x n uint8    current orders                     */
#define BN_OUT_SCORES       2  /* chains float64      current order scores               */
#define BN_OUT_RANKS        3  /* chains x n uint32   current best parent-set ranks      */
#define BN_OUT_BEST_ORDERS  4  /* chains x n uint8                                       */
#define BN_OUT_BEST_SCORES  5  /* chains float64                                         */
#define BN_OUT_BEST_RANKS   6  /* chains x n uint32                                      */
#define BN_OUT_EDGE_COUNTS  7  /* chains x n x n uint32, [c][i][m]: steps with m -> i    */
#define BN_OUT_ACCEPTS      8  /* chains int64                                           */
#define BN_OUT_TRACE_SCORE  9  /* chains x trace_cap float64 (score after each step)     */
#define BN_OUT_TRACE_ACCEPT 10 /* chains x trace_cap uint8                               */
#define BN_OUT_STEPS        11 /* 1 int64: steps taken so far                            */
#define BN_OUT_ESS          12 /* n x n float64: Geyer initial-monotone-sequence ESS of
                                  each edge indicator series, summed over the chains in
                                  which it is not constant (NaN where all are constant) */
#define BN_OUT_RECORD       13 /* chains x n x n x ceil(record_cap/64) uint64: recorded
                                  edge-indicator series, bit r of [c][i][m] = edge m -> i
                                  in chain c's r-th recorded state                       */
#define BN_OUT_RECORD_LEN   14 /* 1 int64: states recorded so far per chain              */
#define BN_OUT_ITEMS        15 /* 1 int64: (node, chain) items re-scored so far (every
                                  step re-scores the nodes between the swapped positions) */
#define BN_OUT_LOGITS       16 /* chains x n(n-1)/2 float32: the proposal network's logits
                                  on each chain's current order, as the learned proposal
                                  on a pruned table holds them (BN_EINVAL otherwise)    */
int bn_chains_read(const bn_chains* c, int what, void* out, int mem, void* stream);

void bn_chains_free(bn_chains* c);

/* Summary of a bn_mcmc_run (the sampler's acceptance and edge-posterior ESS):
 * acceptance over the sampling steps; per directed edge m -> i the Geyer initial-
 * monotone-sequence ESS of its indicator series (every thin-th post-burn-in state),
 * summed over the chains in which the series is not constant; median and minimum over
 * the uncertain edges, those with frequency 0.05 <= f <= 0.95 and a defined ESS. */
typedef struct {
    double  acceptance;      /* accepted / proposed over the sampling steps, all chains   */
    double  ess_median;      /* NaN when thin == 0 or no edge is uncertain                */
    double  ess_min;
    int64_t uncertain_edges;
    double  sample_ms;       /* device time of the sampling steps (CUDA events)           */
    double  train_ms;        /* device time of the training steps (0 for uniform)         */
    int64_t order_evals;     /* chains x (train_iters + steps): every step scores a full order */
} bn_mcmc_stats;

/* One-shot run (Algorithm 1): chains from Philox initial orders; with the learned
 * proposal first p->train_iters training steps, then `steps` sampling steps; edge counts
 * from step p->burn_in on (counted over both phases); then
 *   best_order  n uint8       the best order over all chains
 *   best_dag    n x n uint8   its greedy DAG, best_dag[i*n + m] = 1 iff m -> i
 *   best_score  1 float64
 *   edge_freq   n x n float64 fraction of post-burn-in steps (all chains) with m -> i
 *   stats       the summary above
 * Any output may be NULL.  Outputs are host memory.  p->trace and the record fields are
 * ignored (thin sets the recording).  Errors: BN_EINVAL (proposal, eps_mix, a network of
 * the wrong size), BN_ENOMEM, BN_ETIMEOUT, BN_ECUDA. */
int bn_mcmc_run(const bn_table* t, const bn_mcmc_params* p, int64_t steps,
                uint8_t* best_order, uint8_t* best_dag, double* best_score,
                double* edge_freq, bn_mcmc_stats* stats, void* stream);

/* bn_mcmc_run for `count` networks of uneven size stepped together (the paper learns one
 * network at a time): network i runs on tables[i] with params[i] (learned networks train
 * first, on their own chains), then every network takes `steps` sampling steps in one
 * batch (bn_batch_step: the uniform-proposal networks on pruned tables share one fused
 * launch per 1,024 steps).  Outputs per network, any array or entry may be NULL:
 * best_order[i] (n_i uint8), best_dag[i] (n_i x n_i), best_score[i], edge_freq[i]
 * (n_i x n_i), stats[i] (sample_ms and train_ms are the whole batch's).  Each network's
 * results equal its own bn_mcmc_run with the same parameters.  Errors: as bn_mcmc_run,
 * naming the network. */
int bn_mcmc_run_batch(int count, const bn_table* const* tables, const bn_mcmc_params* params,
                      int64_t steps, uint8_t* const* best_order, uint8_t* const* best_dag,
                      double* best_score, double* const* edge_freq, bn_mcmc_stats* stats,
                      void* stream);

/* Batches of networks of uneven size (the paper samples one network at a time): count
 * networks, each with its own table and chain parameters.  bn_batch_step advances every
 * network by `steps` MH steps; the networks whose chains use the uniform proposal on a
 * pruned table (BN_SCAN_PRUNED) advance together in one fused launch per 1024 steps (one
 * warp per chain of every network), the others through their own per-network steps.
 * Results equal stepping each network's chains alone.  bn_batch_chains gives network
 * i's chains (for bn_chains_read / bn_chains_set_proposal); they are freed with the
 * batch.  The tables must outlive the batch. */
typedef struct bn_batch bn_batch;
int bn_batch_create(int count, const bn_table* const* tables, const bn_mcmc_params* params,
                    void* stream, bn_batch** out);
int bn_batch_chains(bn_batch* b, int i, bn_chains** out);
int bn_batch_step(bn_batch* b, int64_t steps, void* stream);
void bn_batch_free(bn_batch* b);

/* ---------------------------------------------------------------------------------- */
/* Learned swap proposal                                                               */
/* ---------------------------------------------------------------------------------- */

/* The paper proposes a new order by swapping two uniformly chosen nodes (Sec. III.C).
 * The learned proposal replaces the uniform choice of the pair by a small network over
 * the current order, used inside an exact MH ratio (forward and reverse proposal
 * probabilities), so the target distribution is unchanged:
 *   x      = concat over positions p of E[sigma(p)]        (E: n x d node embeddings)
 *   h1     = relu(W1 x + b1),  h2 = relu(W2 h1 + b2)        (W1: H x (n d), W2: H x H)
 *   logits = W3 h2 + b3                                     (W3: P x H, P = n(n-1)/2 pairs
 *                                                            a < b, lexicographic)
 *   q(pair | sigma) = (1 - eps) softmax(logits)[pair] + eps / P
 * Dense layers run on the tensor cores with bf16 weights and activations and FP32
 * accumulation; master weights, biases, softmax and Adam are FP32.
 * Training target: a logged uniform-swap step (sigma, pair, delta) fits the pair's logit
 * by binary cross-entropy to alpha = min(1, 10^delta), the swap's acceptance probability;
 * the loss is the batch mean. */
typedef struct bn_mlp bn_mlp;

typedef struct {
    int   d;          /* embedding width                                              */
    int   hidden;     /* H, a positive multiple of 128                                */
    int   batch_cap;  /* largest batch of orders a forward/backward call takes         */
    float lr;         /* Adam learning rate                                           */
    float beta1, beta2, adam_eps;   /* 0 = defaults 0.9, 0.999, 1e-8                  */
} bn_mlp_params;

/* Weights are FP32, row-major, unpadded (E n x d, W1 H x (n d), b1 H, W2 H x H, b2 H,
 * W3 P x H, b3 P), host or device per `mem`; the network keeps its own copies. */
int bn_mlp_create(int n, const bn_mlp_params* p, const float* E, const float* W1,
                  const float* b1, const float* W2, const float* b2, const float* W3,
                  const float* b3, int mem, void* stream, bn_mlp** out);
/* logits of B <= batch_cap orders: B x P float32 */
int bn_mlp_forward(bn_mlp* m, const uint8_t* orders, int B, float* logits, int mem,
                   void* stream);
/* loss and gradients (kept inside; read them with bn_mlp_read) of B logged steps:
 * orders B x n, pairs B uint32 (pair index), alpha B float32 in [0, 1] */
int bn_mlp_loss_grad(bn_mlp* m, const uint8_t* orders, const uint32_t* pairs,
                     const float* alpha, int B, float* loss, int mem, void* stream);
/* one Adam step on every parameter with the last gradients */
int bn_mlp_adam_step(bn_mlp* m, void* stream);
#define BN_MLP_E 0
#define BN_MLP_W1 1
#define BN_MLP_B1 2
#define BN_MLP_W2 3
#define BN_MLP_B2 4
#define BN_MLP_W3 5
#define BN_MLP_B3 6
#define BN_MLP_GRAD_E 7   /* + the tensor id above: its gradient */
/* copy a parameter or gradient out (FP32, unpadded layout as in bn_mlp_create) */
int bn_mlp_read(const bn_mlp* m, int what, float* out, int mem, void* stream);
void bn_mlp_free(bn_mlp* m);

/* Proposal of a chain set's subsequent steps:
 *   BN_PROPOSAL_UNIFORM  the paper's uniform two-position swap (the default)
 *   BN_PROPOSAL_LEARNED  the pair is drawn from q(. | sigma) of the (frozen) network m;
 *                        the MH test becomes  ln u < ln10 (s' - s) + ln q(pair | sigma')
 *                        - ln q(pair | sigma)  (the reverse move swaps the same pair)
 *   BN_PROPOSAL_TRAIN    uniform swaps; after every step the network takes one Adam step
 *                        on that step's proposals (sigma, pair, alpha = min(1, 10^delta))
 * Random numbers of the learned draw, from the step's Philox block: on a pruned table
 * (bn_table_set_scan) the mixture component is drawn first, uniform iff
 * ((x3 >> 11) + 0.5) 2^-53 < eps_mix (pair = floor(x0 P / 2^64)), else the softmax pair is
 * inverted from u = ((x2 >> 11) + 0.5) 2^-53 through the cumulative softmax, tile of 32
 * pairs first; on a full table u inverts the cumulative mixture q in pair order.  On a
 * pruned table the network's first layer is evaluated as a sum of per-(position, node)
 * rows held in 32-bit fixed point (scale 2^-s, s <= 24 chosen so no sum can overflow),
 * so q(. | sigma) depends on sigma alone; the network is read when this call is made
 * (later training needs another call).  m must have the chains' n and
 * batch_cap >= chains; it must outlive the chains (or the next call here).  eps_mix in
 * (0, 1] keeps every pair proposable.  Errors: BN_EINVAL, BN_ENOMEM, BN_ECUDA. */
#define BN_PROPOSAL_UNIFORM 0
#define BN_PROPOSAL_LEARNED 1
#define BN_PROPOSAL_TRAIN   2
int bn_chains_set_proposal(bn_chains* c, bn_mlp* m, int mode, double eps_mix, void* stream);

/* How the learned proposal's steps on a pruned table are launched (the results are the
 * same either way):
 *   BN_LEARNED_LAUNCH_AUTO   (default) one cooperative persistent kernel runs up to 256
 *                            steps per launch -- per step the layer-2 tiles, the output-layer
 *                            tiles and the chains, separated by grid-wide barriers, with the
 *                            weight tiles resident in shared memory and TMEM -- when all its
 *                            CTAs fit on the GPU at once (at most 256 chains at H = 512);
 *                            otherwise as BN_LEARNED_LAUNCH_GRAPH
 *   BN_LEARNED_LAUNCH_GRAPH  three kernels per step (chains, layer 2, output layer),
 *                            chained by programmatic dependent launch in a CUDA graph
 * Errors: BN_EINVAL. */
#define BN_LEARNED_LAUNCH_AUTO  0
#define BN_LEARNED_LAUNCH_GRAPH 1
int bn_chains_set_learned_launch(bn_chains* c, int mode);

/* C (M x N float32) = A (M x K bf16) * B (N x K bf16)^T on the tensor cores (tcgen05,
 * TMEM accumulator); device pointers, row-major, M and N multiples of 128, K of 64.
 * The proposal network's dense-layer GEMM, exposed for testing. */
int bn_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C, int M, int N, int K,
                 void* stream);

/* ---------------------------------------------------------------------------------- */
/* Misc                                                                                */
/* ---------------------------------------------------------------------------------- */

/* Failure-detection self test (the paper has no counterpart): one kernel waits, with the
 * library's bounded-wait helpers, on an mbarrier no thread arrives at and on a device
 * flag no one sets; each wait gives up after timeout_ns (<= 2 s) and records it in a
 * status word.  Returns BN_ETIMEOUT when both waits ran out as intended (the context
 * stays usable), BN_ECUDA otherwise. */
int bn_selftest_timeout(int64_t timeout_ns, void* stream);

/* Measured peak rate of the scan's consistency test on this GPU (the paper has no
 * counterpart; it is the denominator of the full-table scan's roofline): a kernel that
 * runs the scan's own inner loop -- per two entries one 8-byte load of their sorted
 * positions and one 16-byte load of their masks from shared memory, then per entry two
 * three-input logic ops folding the 64-bit AND-NOT, a zero test and a predicated
 * unsigned min -- over 1,024 entries resident in shared memory (no HBM, no staging),
 * 8 blocks of 256 threads per SM, timed by CUDA events on `stream` (best of three
 * launches after one warm-up).  *tests_per_s receives (tests per launch) / (time). */
int bn_measure_test_rate(void* stream, double* tests_per_s);

const char* bn_last_error(void);     /* thread-local; "" when no error                 */
const char* bn_version(void);
/* Number of kernel launches the library issued on behalf of the calling process so far
 * (graph replays count their kernel nodes). */
int64_t bn_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* BN_H */
