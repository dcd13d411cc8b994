/*
 * oracle.h -- plain, slow CPU oracle for the order-space Bayesian-network scorer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load this library.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written directly from the paper:
 *   Eq. (3)-(4)   local score (Bayesian-Dirichlet, log10 space)
 *   Eq. (5)-(6)   graph score and order score (sum over nodes of the best consistent set)
 *   Sec. III.B    the sum-based order score of the prior scorer the paper compares against
 *   Eq. (7)-(10)  pairwise prior, PPF = 100 (R - 0.5)^3
 *   Algorithm 1   learner loop: score, Metropolis-Hastings test, best graph, swap
 *   Algorithm 2   unranking of the l-th k-combination in lexicographic order
 * Everything is FP64 / exact integers, single-threaded, no blocking or fusion.
 */
#ifndef BN_ORACLE_H
#define BN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- combinatorics (Sec. V.B subset indexing) ---------------------------------- */
uint64_t orc_binom(int N, int j);
/* number of subsets of an N-set with size <= k */
int64_t  orc_num_sets(int N, int k);
/* rank of a sorted subset of {0..N-1} (size j <= k) in size-ascending,
 * combinatorial-number-system (colex) order */
int64_t  orc_rank(int N, int k, const int* set, int j);
/* inverse of orc_rank; returns the size, writes the sorted elements */
int      orc_unrank(int N, int k, int64_t rank, int* set_out);
/* Algorithm 2, 1-based: l-th (1-based) k-combination of {1..n} in lexicographic order */
void     orc_comb_alg2(int n, int k, int64_t l, int* comb_out);

/* ---- counts and local score (Eq. 3-4, Eq. 9-10) ---------------------------------- */
/* counts[c * r + x]: rows whose parent configuration is c (mixed radix, parents in the
 * given order, first parent least significant) and whose child state is x */
void   orc_counts(const uint8_t* data, int m, int n, const uint8_t* arity,
                  int child, const int* parents, int np, uint32_t* counts);
/* kind 0 = K2 (alpha_cx = 1, alpha_c = r), kind 1 = BDeu(ess); R may be NULL */
double orc_local_score(const uint8_t* data, int m, int n, const uint8_t* arity,
                       int child, const int* parents, int np, int kind, double ess,
                       double log10_gamma, const double* R);
double orc_ppf(double r);
/* one node's row of the table (S(n-1,k) entries, rank order) */
void   orc_build_table_node(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                            int kind, double ess, double log10_gamma, const double* R,
                            int i, double* row);
/* all n * S(n-1,k) entries, node-major, rank order (candidate space of each node) */
void   orc_build_table(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                       int kind, double ess, double log10_gamma, const double* R,
                       double* table);
/* candidate slot c of node i <-> node id c + (c >= i) */
int    orc_cand_to_node(int i, int c);

/* ---- order score (Eq. 6, Algorithm 1 scoring loop) ----------------------------- */
double orc_order_score(const double* table, int n, int k, const uint8_t* order,
                       uint32_t* best_rank);
/* parents of the greedy DAG: adj[i*n + m] = 1 iff m -> i */
void   orc_greedy_dag(int n, int k, const uint32_t* best_rank, uint8_t* adj);
/* Eq. (9) score of a DAG given per-node ranks: sum over nodes ascending */
double orc_graph_score(const double* table, int n, int k, const uint32_t* ranks);
/* The sum-based order score of the prior scorer the paper compares against (Sec. III.B):
 * log10 of the sum over all graphs consistent with the order of 10^score(G), which
 * factorises over nodes into sum_i log10 sum_{consistent pi} 10^ls(i, pi).  Per node the
 * consistent sets are enumerated as in orc_order_score, the terms summed in that order
 * after shifting by the node's maximum; nodes summed in ascending id.  node_score (n,
 * may be NULL) receives the per-node values. */
double orc_order_score_sum(const double* table, int n, int k, const uint8_t* order, double* node_score);

/* ---- Philox4x64-10 (Salmon et al., SC'11) --------------------------------------- */
void   orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* ---- Metropolis-Hastings swap sampler (Sec. III.C) ------------------------------ */
typedef struct {
    int      chains;
    int64_t  iters;
    int64_t  burn_in;
    uint64_t seed;
    int      literal_log;     /* 1: accept iff ln u < delta (un-scaled), as printed */
    int      chain0;          /* chain c of the call draws the Philox streams of chain
                                 chain0 + c (lets chains run in separate calls)      */
} orc_mcmc_params;

/* init_orders: chains x n (NULL = draw from the Philox init stream);
 * outputs (any may be NULL):
 *   final_orders chains*n, final_score chains, best_order chains*n, best_score chains,
 *   best_rank chains*n, edge_counts chains*n*n (uint64, [c][i][m]),
 *   accepts chains, trace_score chains*iters (score of the state after step t),
 *   trace_accept chains*iters */
void   orc_mcmc_run(const double* table, int n, int k, const orc_mcmc_params* p,
                    const uint8_t* init_orders,
                    uint8_t* final_orders, double* final_score,
                    uint8_t* best_order, double* best_score, uint32_t* best_rank,
                    uint64_t* edge_counts, int64_t* accepts,
                    double* trace_score, uint8_t* trace_accept);
void   orc_init_order(uint64_t seed, int chain, int n, uint8_t* order);
void   orc_pair_decode(int n, uint64_t idx, int* a, int* b);

/* ---- effective sample size (Geyer initial monotone sequence) -------------------- */
double orc_ess(const double* x, int64_t T);

/* ---- Table I: number of labelled DAGs (Robinson's recurrence) ------------------- */
double orc_count_dags(int n);

#ifdef __cplusplus
}
#endif
#endif
