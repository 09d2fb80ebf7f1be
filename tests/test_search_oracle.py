"""The structure-search oracle pinned without the CUDA path (no GPU): the one-bit-at-a-time
best-parent minimum against listing every subset, the dynamic programme against every
acyclic assignment of parent sets, and a table whose optimum is known in closed form."""
import numpy as np
import pytest

from oracle import search


def _table(m, seed):
    return np.random.default_rng(seed).standard_normal(m << (m - 1))


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6, 7])
def test_best_parents_recursion_equals_enumeration(m):
    t = _table(m, m)
    b1, a1 = search.best_parents(t, m)
    b2, a2 = search.best_parents_by_enumeration(t, m)
    assert np.array_equal(b1, b2) and np.array_equal(a1, a2)


@pytest.mark.parametrize("m,seed", [(2, 0), (3, 1), (3, 2), (4, 3), (4, 4), (4, 5)])
def test_dynamic_programme_equals_brute_force(m, seed):
    t = _table(m, seed)
    parents, order, total = search.optimal_network(t, m)
    bp, btotal = search.brute_force_network(t, m)
    assert search.is_acyclic(parents, m)
    assert total == pytest.approx(btotal, rel=0, abs=1e-12)
    assert search.network_score(t, m, parents) == pytest.approx(total, abs=1e-12)
    assert parents == bp  # continuous random scores: the optimum is unique
    pos = {v: i for i, v in enumerate(order)}
    assert all(pos[p] < pos[c] for c in range(m) for p in range(m) if (parents[c] >> p) & 1)


def test_known_chain_is_found():
    """score(c, S) = 0 for S = {c - 1} (and S = {} for c = 0), 1 otherwise: the chain
    0 -> 1 -> ... -> m-1 is the unique optimum, with score 0."""
    m = 6
    half = 1 << (m - 1)
    t = np.ones(m * half)
    t[0 * half + 0] = 0.0
    for c in range(1, m):
        t[c * half + search.compress(1 << (c - 1), c)] = 0.0
    parents, order, total = search.optimal_network(t, m)
    assert total == 0.0
    assert parents == [0] + [1 << (c - 1) for c in range(1, m)]
    assert order == list(range(m))


def test_forbidden_families_are_avoided():
    """+inf entries are never chosen: forbid every parent set but the empty one."""
    m = 5
    half = 1 << (m - 1)
    t = np.full(m * half, np.inf)
    t[np.arange(m) * half] = np.arange(m, dtype=float)
    parents, _, total = search.optimal_network(t, m)
    assert parents == [0] * m and total == float(sum(range(m)))
