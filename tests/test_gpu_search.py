"""Exact structure search on the GPU against the oracle's search (needs a GPU).

* best parents: the subset minimum of every child block equals the oracle's on the same
  FP32 table exactly (a minimum of stored values has no rounding), and every argmin is a
  subset of its candidate set holding that minimum; the sizes cover one, two and three
  passes of the transform;
* the search: the GPU's DAG is acyclic, its score (the table entries it chose) equals the
  reported total, and the total equals the oracle's optimum on the same table (FP64 sums of
  the same FP32 values, in a different order: 1e-9 relative);
* on tables scored by the walk from SEM data, the optimum of the FP32 table agrees with the
  optimum of the oracle's FP64 scores within the walk's tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import search
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


def _random_table(m, seed):
    return np.random.default_rng(seed).standard_normal(m << (m - 1)).astype(np.float32)


@pytest.mark.parametrize("m", [2, 3, 9, 13, 14, 17, 22, 23])
def test_best_parents_equal_the_oracle(m):
    t = _random_table(m, 100 + m)
    best, bset = binding.best_parents(torch.from_numpy(t).cuda())
    best = best.cpu().numpy()
    bset = bset.cpu().numpy().astype(np.int64) & 0xffffffff
    want, _ = search.best_parents(t.astype(np.float64), m)
    assert np.array_equal(best.astype(np.float64), want)
    half = 1 << (m - 1)
    u = np.arange(m * half) % half
    assert np.all((bset & ~u) == 0)  # the argmin is a subset of the candidate set
    c = np.arange(m * half) // half
    assert np.array_equal(t[c * half + bset], best)


def _check_network(t, m, parents, order, total):
    assert search.is_acyclic(parents, m)
    assert sorted(order) == list(range(m))
    pos = {v: i for i, v in enumerate(order)}
    assert all(pos[p] < pos[c] for c in range(m) for p in range(m) if (parents[c] >> p) & 1)
    assert search.network_score(t.astype(np.float64), m, parents) == pytest.approx(total, rel=1e-12)


@pytest.mark.parametrize("m,seed", [(2, 1), (4, 2), (7, 3), (11, 4), (15, 5), (18, 6)])
def test_search_on_random_tables(m, seed):
    t = _random_table(m, seed)
    parents, order, total = binding.structure_search(torch.from_numpy(t).cuda())
    _check_network(t, m, parents, order, total)
    wp, _, wt = search.optimal_network(t.astype(np.float64), m)
    assert total == pytest.approx(wt, rel=1e-9)
    assert parents == wp


@pytest.mark.parametrize("m,n,p", [(8, 300, 0.4), (12, 500, 0.3), (16, 2000, 0.25),
                                   (20, 1000, 0.2)])
def test_search_on_walk_scores(m, n, p):
    X = synthetic.sem_sample(m, n, p, 8800 + m)
    table = binding.score_all_families(torch.from_numpy(X).cuda())
    parents, order, total = binding.structure_search(table)
    t = table.cpu().numpy()
    _check_network(t, m, parents, order, total)
    _, _, wt = search.optimal_network(t.astype(np.float64), m)
    assert total == pytest.approx(wt, rel=1e-9)
    if m <= 12:  # against the optimum of the oracle's FP64 scores (walk tolerance 1e-4 * n)
        _, ref = oracle.scores(X)
        _, _, rt = search.optimal_network(ref, m)
        assert abs(total - rt) <= 1e-4 * n * m


def test_search_respects_forbidden_families():
    """A table whose families with more than K parents hold +inf (a bounded-in-degree call
    into a table filled with +inf first): the optimum uses at most K parents per variable."""
    m, n, K = 14, 600, 2
    X = synthetic.sem_sample(m, n, 0.4, 8900)
    out = torch.full((m << (m - 1),), float("inf"), dtype=torch.float32, device="cuda")
    binding.score_all_families(torch.from_numpy(X).cuda(), out, max_parents=K)
    parents, order, total = binding.structure_search(out)
    assert max(bin(p).count("1") for p in parents) <= K
    t = out.cpu().numpy()
    _, _, wt = search.optimal_network(t.astype(np.float64), m)
    assert np.isfinite(total) and total == pytest.approx(wt, rel=1e-9)
