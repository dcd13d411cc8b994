/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load it.
 * It shares no code with the CUDA library.  Every function follows a passage of the
 * paper (section / equation / algorithm named beside it); where the paper is silent the
 * reading taken is stated in place.  FP64 for all floating point, exact integers for
 * counts and indices, single thread, no blocking/fusion/reordering.
 *
 * Parity pins (tests/test_oracle_*.py) tie each function to something other than
 * itself: closed forms with exact big-integer factorials, scipy's gammaln, brute force
 * over all orders and all DAGs, numpy's Philox4x64 generator, AR(1) series with a known
 * autocorrelation time, and the values printed in the paper (Sec. V.B example,
 * Table I).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LN10 2.302585092994045684017991454684364208

/* ------------------------------------------------------------------------------ */
/* combinatorics                                                                  */
/* ------------------------------------------------------------------------------ */

/* C(N, j) by the multiplicative formula; exact for N <= 64 (each partial product
 * C(N-j+i, i) is an integer and the final value fits in 64 bits). */
uint64_t orc_binom(int N, int j)
{
    if (j < 0 || N < 0 || j > N) return 0;
    if (j > N - j) j = N - j;
    unsigned __int128 r = 1;
    for (int i = 1; i <= j; ++i) {
        r = r * (unsigned __int128)(N - j + i);
        r = r / (unsigned __int128)i;
    }
    return (uint64_t)r;
}

/* Sec. III.B: the number of candidate parent sets of size <= s is sum_j C(N, j). */
int64_t orc_num_sets(int N, int k)
{
    int64_t s = 0;
    for (int j = 0; j <= k && j <= N; ++j) s += (int64_t)orc_binom(N, j);
    return s;
}

/* Rank of a parent set among all subsets of size <= k of an N-set.  Sec. V.B asks for
 * a regular indexing of all <=s-subsets that can be inverted from the index alone; the
 * reading taken here is: sizes ascending (the empty set first), and within one size
 * the combinatorial number system, rank {a_1 < ... < a_j} = sum_t C(a_t, t). */
int64_t orc_rank(int N, int k, const int* set, int j)
{
    (void)k;
    int64_t base = 0;
    for (int t = 0; t < j; ++t) base += (int64_t)orc_binom(N, t);
    int64_t r = 0;
    for (int t = 0; t < j; ++t) r += (int64_t)orc_binom(set[t], t + 1);
    return base + r;
}

/* Inverse of orc_rank: find the size class, then peel the largest element first
 * (largest a with C(a, t) <= remainder). */
int orc_unrank(int N, int k, int64_t rank, int* set_out)
{
    int j = 0;
    while (j <= k && rank >= (int64_t)orc_binom(N, j)) {
        rank -= (int64_t)orc_binom(N, j);
        ++j;
    }
    int64_t rem = rank;
    for (int t = j; t >= 1; --t) {
        int a = t - 1;
        while (a + 1 < N && (int64_t)orc_binom(a + 1, t) <= rem) ++a;
        set_out[t - 1] = a;
        rem -= (int64_t)orc_binom(a, t);
    }
    return j;
}

/* Algorithm 2 (non-recursive unranking of the l-th k-combination of n elements in
 * lexicographic order), read with 1-based l and elements {1..n}.  For each position but
 * the last it finds the shift s: the largest s such that the blocks of combinations
 * starting with low+1 .. low+s-1 together hold fewer than l combinations; then it
 * recurses on the (k-1)-combinations of the remaining n-s elements.  The last element
 * is low + l, using the remaining l. */
void orc_comb_alg2(int n, int k, int64_t l, int* comb_out)
{
    int low = 0;
    int kk = k;
    int nn = n;
    int64_t ll = l;
    for (int pos = 1; pos <= k - 1; ++pos) {
        int64_t sum = 0;
        int s;
        for (s = 1; s <= nn; ++s) {
            int64_t blk = (int64_t)orc_binom(nn - s, kk - 1);
            if (sum + blk < ll) sum += blk;
            else break;
        }
        comb_out[pos - 1] = low + s;
        nn -= s;
        kk -= 1;
        ll -= sum;
        low = comb_out[pos - 1];
    }
    comb_out[k - 1] = low + (int)ll;
}

/* ------------------------------------------------------------------------------ */
/* counts and local score                                                         */
/* ------------------------------------------------------------------------------ */

int orc_cand_to_node(int i, int c) { return c + (c >= i ? 1 : 0); }

/* N_ijk of Eq. (3): a direct pass over the m rows. */
void orc_counts(const uint8_t* data, int m, int n, const uint8_t* arity,
                int child, const int* parents, int np, uint32_t* counts)
{
    int q = 1;
    for (int t = 0; t < np; ++t) q *= arity[parents[t]];
    int r = arity[child];
    memset(counts, 0, sizeof(uint32_t) * (size_t)q * (size_t)r);
    for (int row = 0; row < m; ++row) {
        const uint8_t* x = data + (size_t)row * (size_t)n;
        int c = 0, stride = 1;
        for (int t = 0; t < np; ++t) {
            c += x[parents[t]] * stride;
            stride *= arity[parents[t]];
        }
        counts[c * r + x[child]] += 1;
    }
}

/* Eq. (10): PPF = 100 (R - 0.5)^3. */
double orc_ppf(double r)
{
    double d = r - 0.5;
    return 100.0 * d * d * d;
}

typedef struct { double arg; int sign; } orc_term;

static int orc_term_cmp(const void* a, const void* b)
{
    const orc_term* x = (const orc_term*)a;
    const orc_term* y = (const orc_term*)b;
    if (x->arg < y->arg) return -1;
    if (x->arg > y->arg) return 1;
    return x->sign - y->sign;
}

/* Eq. (4) plus the prior term of Eq. (9):
 *   ls = |pi| log10(gamma)
 *      + sum_c [ log10 G(a_c) - log10 G(a_c + N_c)
 *                + sum_x ( log10 G(N_cx + a_cx) - log10 G(a_cx) ) ]
 *      + sum_{m in pi} PPF(i, m)
 * with G = Gamma.  The paper does not fix the Dirichlet hyper-parameters; kind 0 is the
 * K2 choice (a_cx = 1, a_c = r), kind 1 BDeu (a_cx = ess/(q r), a_c = ess/q).  Terms
 * whose count is zero cancel exactly and are left out.  The remaining lgamma terms are
 * summed in natural log, in ascending order of their argument (a permutation of the
 * count table therefore gives a bit-identical sum), then divided by ln 10.  R[i*n+m]
 * is the prior belief in the edge m -> i (NULL: none). */
double orc_local_score(const uint8_t* data, int m, int n, const uint8_t* arity,
                       int child, const int* parents, int np, int kind, double ess,
                       double log10_gamma, const double* R)
{
    int q = 1;
    for (int t = 0; t < np; ++t) q *= arity[parents[t]];
    int r = arity[child];
    uint32_t* cnt = (uint32_t*)calloc((size_t)q * (size_t)r, sizeof(uint32_t));
    orc_counts(data, m, n, arity, child, parents, np, cnt);
    double a_cx, a_c;
    if (kind == 0) { a_cx = 1.0; a_c = (double)r; }
    else { a_cx = ess / ((double)q * (double)r); a_c = ess / (double)q; }

    orc_term* terms = (orc_term*)malloc(sizeof(orc_term) * (size_t)(2 * q * r + 2 * q + 1));
    int nt = 0;
    for (int c = 0; c < q; ++c) {
        uint32_t Nc = 0;
        for (int x = 0; x < r; ++x) Nc += cnt[c * r + x];
        if (Nc == 0) continue;
        terms[nt].arg = a_c; terms[nt].sign = +1; ++nt;
        terms[nt].arg = a_c + (double)Nc; terms[nt].sign = -1; ++nt;
        for (int x = 0; x < r; ++x) {
            uint32_t N = cnt[c * r + x];
            if (N == 0) continue;
            terms[nt].arg = (double)N + a_cx; terms[nt].sign = +1; ++nt;
            terms[nt].arg = a_cx; terms[nt].sign = -1; ++nt;
        }
    }
    qsort(terms, (size_t)nt, sizeof(orc_term), orc_term_cmp);
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += (double)terms[t].sign * lgamma(terms[t].arg);
    free(terms);
    free(cnt);

    double ls = s / ORC_LN10 + (double)np * log10_gamma;
    if (R) {
        for (int t = 0; t < np; ++t) ls += orc_ppf(R[(size_t)child * (size_t)n + (size_t)parents[t]]);
    }
    return ls;
}

/* Preprocessing of Sec. III.A for one node: every local score of node i, by rank. */
void orc_build_table_node(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                          int kind, double ess, double log10_gamma, const double* R,
                          int i, double* row)
{
    int64_t S = orc_num_sets(n - 1, k);
    int slots[64], parents[64];
    for (int64_t rho = 0; rho < S; ++rho) {
        int j = orc_unrank(n - 1, k, rho, slots);
        for (int t = 0; t < j; ++t) parents[t] = orc_cand_to_node(i, slots[t]);
        row[rho] = orc_local_score(data, m, n, arity, i, parents, j, kind, ess, log10_gamma, R);
    }
}

/* Preprocessing of Sec. III.A: every local score of every (node, parent set), stored
 * here densely by (node, rank) instead of in a hash table. */
void orc_build_table(const uint8_t* data, int m, int n, const uint8_t* arity, int k,
                     int kind, double ess, double log10_gamma, const double* R,
                     double* table)
{
    int64_t S = orc_num_sets(n - 1, k);
    for (int i = 0; i < n; ++i)
        orc_build_table_node(data, m, n, arity, k, kind, ess, log10_gamma, R, i,
                             table + (size_t)i * (size_t)S);
}

/* ------------------------------------------------------------------------------ */
/* order score                                                                    */
/* ------------------------------------------------------------------------------ */

/* Eq. (6) / Algorithm 1 scoring loop: for every node, the best local score among the
 * parent sets drawn from its predecessors in the order (size <= k); the order score is
 * their sum over nodes in ascending node id.  The enumeration here is brute force over
 * the subsets of the predecessor set (not a table scan).  Ties between equal scores go
 * to the lowest rank. */
double orc_order_score(const double* table, int n, int k, const uint8_t* order,
                       uint32_t* best_rank)
{
    int64_t S = orc_num_sets(n - 1, k);
    int pos[64];
    for (int p = 0; p < n; ++p) pos[order[p]] = p;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        int pred[64], np = 0;
        for (int c = 0; c < n - 1; ++c) {               /* candidate slots ascending */
            int node = orc_cand_to_node(i, c);
            if (pos[node] < pos[i]) pred[np++] = c;
        }
        double best = -INFINITY;
        int64_t bestr = -1;
        int maxj = k < np ? k : np;
        for (int j = 0; j <= maxj; ++j) {
            /* all j-subsets of pred[0..np), index combinations in lexicographic order */
            int idx[64], set[64];
            for (int t = 0; t < j; ++t) idx[t] = t;
            for (;;) {
                for (int t = 0; t < j; ++t) set[t] = pred[idx[t]];
                int64_t rho = orc_rank(n - 1, k, set, j);
                double v = table[(size_t)i * (size_t)S + (size_t)rho];
                if (v > best || (v == best && rho < bestr)) { best = v; bestr = rho; }
                int t = j - 1;
                while (t >= 0 && idx[t] == np - j + t) --t;
                if (t < 0) break;
                idx[t] += 1;
                for (int u = t + 1; u < j; ++u) idx[u] = idx[u - 1] + 1;
            }
        }
        if (best_rank) best_rank[i] = (uint32_t)bestr;
        total += best;
    }
    return total;
}

double orc_order_score_sum(const double* table, int n, int k, const uint8_t* order, double* node_score)
{
    int64_t S = orc_num_sets(n - 1, k);
    int pos[64];
    for (int p = 0; p < n; ++p) pos[order[p]] = p;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        int pred[64], np = 0;
        for (int c = 0; c < n - 1; ++c) {
            int node = orc_cand_to_node(i, c);
            if (pos[node] < pos[i]) pred[np++] = c;
        }
        int maxj = k < np ? k : np;
        /* two passes over the same enumeration: the maximum, then the shifted sum */
        double mx = -INFINITY, sum = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = 0; j <= maxj; ++j) {
                int idx[64], set[64];
                for (int t = 0; t < j; ++t) idx[t] = t;
                for (;;) {
                    for (int t = 0; t < j; ++t) set[t] = pred[idx[t]];
                    double v = table[(size_t)i * (size_t)S + (size_t)orc_rank(n - 1, k, set, j)];
                    if (pass == 0) { if (v > mx) mx = v; }
                    else sum += pow(10.0, v - mx);
                    int t = j - 1;
                    while (t >= 0 && idx[t] == np - j + t) --t;
                    if (t < 0) break;
                    idx[t] += 1;
                    for (int u = t + 1; u < j; ++u) idx[u] = idx[u - 1] + 1;
                }
            }
        }
        double node = mx + log10(sum);
        if (node_score) node_score[i] = node;
        total += node;
    }
    return total;
}

void orc_greedy_dag(int n, int k, const uint32_t* best_rank, uint8_t* adj)
{
    memset(adj, 0, (size_t)n * (size_t)n);
    int slots[64];
    for (int i = 0; i < n; ++i) {
        int j = orc_unrank(n - 1, k, best_rank[i], slots);
        for (int t = 0; t < j; ++t) adj[(size_t)i * (size_t)n + (size_t)orc_cand_to_node(i, slots[t])] = 1;
    }
}

/* Eq. (9) score of one DAG given by its per-node parent-set ranks. */
double orc_graph_score(const double* table, int n, int k, const uint32_t* ranks)
{
    int64_t S = orc_num_sets(n - 1, k);
    double total = 0.0;
    for (int i = 0; i < n; ++i) total += table[(size_t)i * (size_t)S + ranks[i]];
    return total;
}

/* ------------------------------------------------------------------------------ */
/* Philox4x64-10                                                                   */
/* ------------------------------------------------------------------------------ */

/* Philox4x64 with 10 rounds as published by Salmon, Moraes, Dror and Shaw (SC'11):
 * per round two 64x64->128 multiplications of counter words 0 and 2 by fixed
 * multipliers, the high halves xor-ed with the other counter words and the key, the
 * key bumped by two Weyl constants between rounds. */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint64_t orc_mulhi(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* ------------------------------------------------------------------------------ */
/* Metropolis-Hastings swap sampler                                               */
/* ------------------------------------------------------------------------------ */

/* Random numbers the sampler draws (a fixed definition both implementations follow):
 *   key = {seed, 0}
 *   initial order of chain c: Fisher-Yates, for i = n-1 .. 1 swap order[i] with
 *     order[floor(x * (i+1) / 2^64)], x the next 64-bit word of the stream of blocks
 *     Philox(ctr = {j, c, 1, 0}), j = 0, 1, ...; identity start.
 *   step t of chain c: x = Philox(ctr = {t, c, 0, 0});
 *     (chain c of a call is chain p->chain0 + c of these streams)
 *     pair index floor(x0 * P / 2^64), P = n(n-1)/2, pairs (a<b) in lexicographic order;
 *     u = ((x1 >> 12) + 0.5) * 2^-52 in (0, 1). */
void orc_init_order(uint64_t seed, int chain, int n, uint8_t* order)
{
    uint64_t key[2] = {seed, 0};
    uint64_t buf[4];
    int used = 4;
    uint64_t blk = 0;
    for (int p = 0; p < n; ++p) order[p] = (uint8_t)p;
    for (int i = n - 1; i >= 1; --i) {
        if (used == 4) {
            uint64_t ctr[4] = {blk++, (uint64_t)chain, 1, 0};
            orc_philox4x64(ctr, key, buf);
            used = 0;
        }
        uint64_t x = buf[used++];
        int j = (int)orc_mulhi(x, (uint64_t)(i + 1));
        uint8_t tmp = order[i]; order[i] = order[j]; order[j] = tmp;
    }
}

void orc_pair_decode(int n, uint64_t idx, int* a, int* b)
{
    for (int x = 0; x < n - 1; ++x) {
        uint64_t cnt = (uint64_t)(n - 1 - x);
        if (idx < cnt) { *a = x; *b = x + 1 + (int)idx; return; }
        idx -= cnt;
    }
    *a = -1; *b = -1;
}

/* Algorithm 1 with the steps of Sec. III.C: score the proposed order, accept with
 * probability min(1, P(new)/P(old)), keep the best graph among the initial and the
 * accepted orders (strictly better replaces), propose by swapping two positions.
 * The scores are log10 values, so the exact acceptance test for the target
 * proportional to 10^score is  ln u < ln(10) * (score_new - score_old); the
 * literal_log flag takes the printed test  ln u < score_new - score_old  instead.
 * Edge counts: after the decision of every step t >= burn_in, every edge of the
 * current state's greedy DAG is counted once. */
void orc_mcmc_run(const double* table, int n, int k, const orc_mcmc_params* p,
                  const uint8_t* init_orders,
                  uint8_t* final_orders, double* final_score,
                  uint8_t* best_order, double* best_score, uint32_t* best_rank,
                  uint64_t* edge_counts, int64_t* accepts,
                  double* trace_score, uint8_t* trace_accept)
{
    uint64_t key[2] = {p->seed, 0};
    const uint64_t P = (uint64_t)n * (uint64_t)(n - 1) / 2;
    uint8_t cur[64], prop[64], best[64];
    uint32_t cur_r[64], prop_r[64], best_r[64];
    int slots[64];
    for (int c = 0; c < p->chains; ++c) {
        const uint64_t cg = (uint64_t)p->chain0 + (uint64_t)c;    /* the chain's stream */
        if (init_orders) memcpy(cur, init_orders + (size_t)c * (size_t)n, (size_t)n);
        else orc_init_order(p->seed, (int)cg, n, cur);
        double s = orc_order_score(table, n, k, cur, cur_r);
        double bs = s;
        memcpy(best, cur, (size_t)n);
        memcpy(best_r, cur_r, sizeof(uint32_t) * (size_t)n);
        int64_t acc = 0;
        uint64_t* E = edge_counts ? edge_counts + (size_t)c * (size_t)n * (size_t)n : NULL;
        if (E) memset(E, 0, sizeof(uint64_t) * (size_t)n * (size_t)n);
        for (int64_t t = 0; t < p->iters; ++t) {
            uint64_t ctr[4] = {(uint64_t)t, cg, 0, 0};
            uint64_t x[4];
            orc_philox4x64(ctr, key, x);
            int a, b;
            orc_pair_decode(n, orc_mulhi(x[0], P), &a, &b);
            double u = ((double)(x[1] >> 12) + 0.5) * (1.0 / 4503599627370496.0);
            memcpy(prop, cur, (size_t)n);
            uint8_t tmp = prop[a]; prop[a] = prop[b]; prop[b] = tmp;
            double s2 = orc_order_score(table, n, k, prop, prop_r);
            double delta = s2 - s;
            int ok = p->literal_log ? (log(u) < delta) : (log(u) < ORC_LN10 * delta);
            if (ok) {
                memcpy(cur, prop, (size_t)n);
                memcpy(cur_r, prop_r, sizeof(uint32_t) * (size_t)n);
                s = s2;
                ++acc;
                if (s > bs) {
                    bs = s;
                    memcpy(best, cur, (size_t)n);
                    memcpy(best_r, cur_r, sizeof(uint32_t) * (size_t)n);
                }
            }
            if (trace_score) trace_score[(size_t)c * (size_t)p->iters + (size_t)t] = s;
            if (trace_accept) trace_accept[(size_t)c * (size_t)p->iters + (size_t)t] = (uint8_t)ok;
            if (E && t >= p->burn_in) {
                for (int i = 0; i < n; ++i) {
                    int j = orc_unrank(n - 1, k, cur_r[i], slots);
                    for (int q = 0; q < j; ++q) E[(size_t)i * (size_t)n + (size_t)orc_cand_to_node(i, slots[q])] += 1;
                }
            }
        }
        if (final_orders) memcpy(final_orders + (size_t)c * (size_t)n, cur, (size_t)n);
        if (final_score) final_score[c] = s;
        if (best_order) memcpy(best_order + (size_t)c * (size_t)n, best, (size_t)n);
        if (best_score) best_score[c] = bs;
        if (best_rank) memcpy(best_rank + (size_t)c * (size_t)n, best_r, sizeof(uint32_t) * (size_t)n);
        if (accepts) accepts[c] = acc;
    }
}

/* ------------------------------------------------------------------------------ */
/* effective sample size                                                          */
/* ------------------------------------------------------------------------------ */

/* Geyer's (1992) initial monotone sequence estimator: autocovariances g_k (divisor T),
 * pair sums G_j = g_{2j} + g_{2j+1} taken while positive and made non-increasing;
 * variance of the mean sigma^2 = -g_0 + 2 sum_j G_j; ESS = T g_0 / sigma^2.
 * A constant series has no defined ESS (NaN). */
double orc_ess(const double* x, int64_t T)
{
    if (T < 2) return NAN;
    double mu = 0.0;
    for (int64_t t = 0; t < T; ++t) mu += x[t];
    mu /= (double)T;
    double g0 = 0.0;
    for (int64_t t = 0; t < T; ++t) g0 += (x[t] - mu) * (x[t] - mu);
    g0 /= (double)T;
    if (!(g0 > 0.0)) return NAN;
    double sum = 0.0, prev = INFINITY;
    for (int64_t j = 0; 2 * j + 1 < T; ++j) {
        double gk[2];
        for (int h = 0; h < 2; ++h) {
            int64_t lag = 2 * j + h;
            double acc = 0.0;
            for (int64_t t = 0; t + lag < T; ++t) acc += (x[t] - mu) * (x[t + lag] - mu);
            gk[h] = acc / (double)T;
        }
        double G = gk[0] + gk[1];
        if (!(G > 0.0)) break;
        if (G > prev) G = prev;
        sum += G;
        prev = G;
    }
    double sigma2 = -g0 + 2.0 * sum;
    if (!(sigma2 > 0.0)) return NAN;
    return (double)T * g0 / sigma2;
}

/* ------------------------------------------------------------------------------ */
/* Table I                                                                        */
/* ------------------------------------------------------------------------------ */

/* Robinson's recurrence for labelled DAGs on n nodes:
 * a(0) = 1, a(n) = sum_{j=1..n} (-1)^{j+1} C(n,j) 2^{j(n-j)} a(n-j). */
double orc_count_dags(int n)
{
    double a[65];
    a[0] = 1.0;
    for (int N = 1; N <= n; ++N) {
        double s = 0.0;
        for (int j = 1; j <= N; ++j) {
            double term = (double)orc_binom(N, j) * ldexp(1.0, j * (N - j)) * a[N - j];
            s += (j % 2 == 1) ? term : -term;
        }
        a[N] = s;
    }
    return a[n];
}
