"""Pins of the oracle's subset indexing (Sec. V.B, Algorithm 2) and of Table I."""
import itertools
import json
import math
import os

import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_binomial_matches_math_comb():
    for N in range(0, 65):
        for j in range(0, N + 1):
            assert oracle.binom(N, j) == math.comb(N, j)


def test_num_sets_is_sum_of_binomials_and_paper_example():
    ex = json.load(open(os.path.join(GOLD, "subset_index_example.json")))
    # Sec. V.B: 6 candidates, size limit 4 -> 57 subsets
    assert oracle.num_sets(6, 4) == ex["total"] == 57
    # brute-force count of subsets
    for N in range(0, 9):
        for k in range(0, N + 1):
            brute = sum(1 for j in range(k + 1) for _ in itertools.combinations(range(N), j))
            assert oracle.num_sets(N, k) == brute
    # per-node table sizes of the workloads (Sec. III.B: sum_{j<=s} C(n-1, j))
    assert oracle.num_sets(5, 2) == 16
    assert oracle.num_sets(19, 4) == 5036
    assert oracle.num_sets(39, 4) == 92171
    assert oracle.num_sets(59, 4) == 489406


def test_pst_memory_of_paper():
    # Sec. V.B: a 60-node graph at s = 4 needs 7.99 MB of parent-set table.  The paper's
    # table spans all 60 labels, one int32 per slot of a 4-slot record.
    ex = json.load(open(os.path.join(GOLD, "subset_index_example.json")))
    mib = oracle.num_sets(60, 4) * 4 * 4 / 2**20
    assert round(mib, 2) == ex["pst_memory"]["megabytes"]


@pytest.mark.parametrize("N,k", [(1, 1), (5, 2), (6, 4), (8, 3), (10, 10), (12, 4)])
def test_rank_unrank_bijection_and_order(N, k):
    S = oracle.num_sets(N, k)
    # independent definition of the ordering: size ascending, then colex (compare the
    # sorted tuples from their largest element down)
    subsets = [c for j in range(k + 1) for c in itertools.combinations(range(N), j)]
    subsets.sort(key=lambda c: (len(c), tuple(reversed(c))))
    assert len(subsets) == S
    for r, c in enumerate(subsets):
        assert oracle.rank(N, k, list(c)) == r
        assert oracle.unrank(N, k, r) == list(c)


def test_rank_prefix_property():
    # colex: all j-subsets of {0..a-1} come before any j-subset containing a
    N, k = 9, 4
    base = [oracle.num_sets(N, j - 1) if j else 0 for j in range(k + 1)]
    for j in range(1, k + 1):
        for a in range(j, N + 1):
            for c in itertools.combinations(range(a), j):
                assert oracle.rank(N, k, list(c)) - base[j] < math.comb(a, j)


@pytest.mark.parametrize("n,k", [(6, 4), (7, 3), (9, 2), (10, 5), (5, 1), (6, 6)])
def test_algorithm2_is_lexicographic(n, k):
    # Algorithm 2 read with a 1-based index l and elements {1..n} reproduces the
    # lexicographic order of itertools.combinations exactly
    for l, c in enumerate(itertools.combinations(range(1, n + 1), k), start=1):
        assert oracle.comb_alg2(n, k, l) == list(c)


def test_paper_subset_index_example():
    """Sec. V.B example: subsets of {0..5} of size <= 4 indexed size-descending and
    lexicographically within a size, the empty set last.  Algorithm 2 (1-based) gives
    the sets within one size; the oracle's own rank is a different bijection onto the
    same 57 subsets."""
    ex = json.load(open(os.path.join(GOLD, "subset_index_example.json")))
    N, s = 6, 4
    paper = []
    for j in range(s, 0, -1):
        for l in range(1, math.comb(N, j) + 1):
            paper.append([x - 1 for x in oracle.comb_alg2(N, j, l)])
    paper.append([])
    assert len(paper) == ex["total"]
    for e in ex["examples"]:
        assert paper[e["index"]] == e["set"]
    # bijection between the paper's index and the oracle's rank
    ranks = {oracle.rank(N, s, st) for st in paper}
    assert ranks == set(range(ex["total"]))


def test_table1_orders_and_graphs():
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    for row in g["rows"]:
        n = row["n"]
        f = math.factorial(n)
        # orders: n!, as printed to its printed precision
        op = row["orders_printed"]
        digits = 3 if op >= 1e6 else len(str(int(op)))
        assert float(f"{f:.{digits - 1}e}") == pytest.approx(op, rel=10 ** (1 - digits))
        dags = oracle.count_dags(n)
        if row["graphs_true"] is not None:
            assert dags == pytest.approx(row["graphs_true"], rel=1e-12)
        if n not in (4, 10):          # the two errata
            gp = row["graphs_printed"]
            assert dags == pytest.approx(gp, rel=5e-3)


def test_count_dags_brute_force_small():
    # enumerate all digraphs without self loops on n nodes and keep the acyclic ones
    for n in (1, 2, 3, 4):
        pairs = [(i, j) for i in range(n) for j in range(n) if i != j]
        cnt = 0
        for bits in range(1 << len(pairs)):
            par = [0] * n
            for t, (i, j) in enumerate(pairs):
                if bits >> t & 1:
                    par[i] |= 1 << j
            removed = 0
            for _ in range(n):
                for i in range(n):
                    if not removed >> i & 1 and par[i] & ~removed == 0:
                        removed |= 1 << i
            cnt += removed == (1 << n) - 1
        assert oracle.count_dags(n) == cnt
