"""Pins of the FP64 oracle against things other than itself (no GPU).

* exact rational normal equations on integer data (m <= 4), independent of
  floating point and of QR;
* numpy/LAPACK least squares (an SVD-based solver the oracle does not use);
* invariants: RSS(empty) = centred sum of squares, RSS never grows when a
  parent is added, RSS >= 0;
* metamorphic relations: row permutation and orthogonal mixing of the centred
  rows leave every RSS unchanged, scaling one column by a scales the RSS of
  that child by a^2 and leaves every other RSS unchanged, mutually orthogonal
  centred columns give RSS(c|S) = |x_c|^2;
* the score against the Gaussian profile log-likelihood evaluated by scipy
  (BIC = -2 log L + |S| log n up to the constants n log(2 pi) + n);
* the table layout against a direct enumeration of (child, parent set);
* planted mistakes: each deliberate error in the oracle fails at least one pin.
"""
from fractions import Fraction
from itertools import combinations

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1901_07643_gb300 import synthetic


def _families(m):
    for c in range(m):
        others = [v for v in range(m) if v != c]
        for r in range(m):
            for S in combinations(others, r):
                mask = 0
                for v in S:
                    mask |= 1 << v
                yield c, S, mask


def _frac_rss(Xi, c, S):
    """Exact RSS via normal equations in rational arithmetic."""
    n, m = len(Xi), len(Xi[0])
    cols = [[Fraction(int(Xi[t][j])) for t in range(n)] for j in range(m)]
    cols = [[v - sum(col, Fraction(0)) / n for v in col] for col in cols]
    y = cols[c]
    yy = sum(v * v for v in y)
    if not S:
        return yy
    A = [cols[j] for j in S]
    k = len(S)
    G = [[sum(a * b for a, b in zip(A[i], A[j])) for j in range(k)] for i in range(k)]
    h = [sum(a * b for a, b in zip(A[i], y)) for i in range(k)]
    # Gauss-Jordan on [G | h]
    M = [G[i][:] + [h[i]] for i in range(k)]
    for col in range(k):
        piv = next(r for r in range(col, k) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [v / p for v in M[col]]
        for r in range(k):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * b for a, b in zip(M[r], M[col])]
    beta = [M[i][k] for i in range(k)]
    return yy - sum(b * hh for b, hh in zip(beta, h))


def _pin_rational(seed=7):
    for m, n in [(3, 6), (4, 7)]:
        X = synthetic.integer_sample(m, n, seed + m)
        rss, _ = oracle.scores(X, nthreads=1)
        for c, S, mask in _families(m):
            exact = _frac_rss(X.tolist(), c, S)
            got = rss[oracle.table_index(c, mask, m)]
            if abs(got - float(exact)) > 1e-12 * max(1.0, abs(float(exact))):
                return False
    return True


def _pin_lstsq(X):
    n, m = X.shape
    Xc = X - X.mean(0)
    rss, _ = oracle.scores(X, nthreads=2)
    for c, S, mask in _families(m):
        y = Xc[:, c]
        if S:
            A = Xc[:, list(S)]
            beta = np.linalg.lstsq(A, y, rcond=None)[0]
            e = y - A @ beta
        else:
            e = y
        ref = float(e @ e)
        if abs(rss[oracle.table_index(c, mask, m)] - ref) > 1e-9 * ref:
            return False
    return True


def _pin_invariants(X):
    n, m = X.shape
    Xc = X - X.mean(0)
    rss, _ = oracle.scores(X, nthreads=2)
    if (rss < 0).any():
        return False
    for c in range(m):
        ss = float(Xc[:, c] @ Xc[:, c])
        if abs(rss[oracle.table_index(c, 0, m)] - ss) > 1e-12 * ss:
            return False
    for c, S, mask in _families(m):
        for p in range(m):
            if p == c or (mask >> p) & 1:
                continue
            big = rss[oracle.table_index(c, mask | (1 << p), m)]
            small = rss[oracle.table_index(c, mask, m)]
            if big > small * (1 + 1e-12) + 1e-12:
                return False
    return True


def _pin_loglik(X):
    n, m = X.shape
    Xc = X - X.mean(0)
    rss, sc = oracle.scores(X, nthreads=2)
    for c, S, mask in _families(m):
        y = Xc[:, c]
        if S:
            A = Xc[:, list(S)]
            e = y - A @ np.linalg.lstsq(A, y, rcond=None)[0]
        else:
            e = y
        sigma = np.sqrt(float(e @ e) / n)
        minus2ll = -2.0 * stats.norm.logpdf(e, scale=sigma).sum()
        bic = minus2ll - n * np.log(2 * np.pi) - n + len(S) * np.log(n)
        if abs(sc[oracle.table_index(c, mask, m)] - bic) > 1e-8 * max(1.0, abs(bic)):
            return False
    return True


def _pin_layout(m=5):
    X = synthetic.sem_sample(m, 40, 0.4, 11)
    Xc = X - X.mean(0)
    rss, _ = oracle.scores(X, nthreads=1)
    slots = []
    for c, S, mask in _families(m):
        y = Xc[:, c]
        if S:
            A = Xc[:, list(S)]
            e = y - A @ np.linalg.lstsq(A, y, rcond=None)[0]
        else:
            e = y
        # slot computed by hand: drop bit c, keep the order of the other bits
        slot = c * 2 ** (m - 1) + sum(1 << (v if v < c else v - 1) for v in S)
        slots.append(slot)
        if abs(rss[slot] - float(e @ e)) > 1e-9 * float(e @ e):
            return False
    return sorted(slots) == list(range(m * 2 ** (m - 1)))


SMALL = synthetic.sem_sample(6, 30, 0.4, 3)


def test_exact_rational_normal_equations():
    assert _pin_rational()


def test_against_lapack_lstsq():
    assert _pin_lstsq(synthetic.sem_sample(8, 50, 0.3, 5))


def test_invariants_m10():
    assert _pin_invariants(synthetic.workload_sample(synthetic.SMALL_M10))


def test_score_is_gaussian_bic():
    assert _pin_loglik(SMALL)


def test_table_layout():
    assert _pin_layout()


def test_row_permutation_and_orthogonal_mixing():
    X = synthetic.sem_sample(7, 40, 0.3, 21)
    rss, _ = oracle.scores(X)
    rng = np.random.default_rng(0)
    rss_p, _ = oracle.scores(X[rng.permutation(len(X))])
    np.testing.assert_allclose(rss_p, rss, rtol=1e-11)
    # Householder reflector with v orthogonal to the ones vector keeps centring
    v = rng.standard_normal(len(X))
    v -= v.mean()
    H = np.eye(len(X)) - 2.0 * np.outer(v, v) / (v @ v)
    rss_h, _ = oracle.scores(H @ (X - X.mean(0)))
    np.testing.assert_allclose(rss_h, rss, rtol=1e-10)


def test_column_scaling():
    m = 6
    X = synthetic.sem_sample(m, 40, 0.4, 31)
    rss, _ = oracle.scores(X)
    a = 3.7
    Y = X.copy()
    Y[:, 2] *= a
    rss_s, _ = oracle.scores(Y)
    half = 2 ** (m - 1)
    for c in range(m):
        blk = slice(c * half, (c + 1) * half)
        f = a * a if c == 2 else 1.0
        np.testing.assert_allclose(rss_s[blk], f * rss[blk], rtol=1e-10)


def test_orthogonal_columns():
    n, m = 16, 4
    Hd = np.array([[1.0]])
    while Hd.shape[0] < n:
        Hd = np.block([[Hd, Hd], [Hd, -Hd]])
    X = Hd[:, 1:m + 1] * np.array([1.0, 2.0, 0.5, 3.0])  # centred, orthogonal
    rss, _ = oracle.scores(X)
    for c, S, mask in _families(m):
        np.testing.assert_allclose(rss[oracle.table_index(c, mask, m)], X[:, c] @ X[:, c],
                                   rtol=1e-12)


def test_reduced_equals_direct():
    X = synthetic.sem_sample(9, 80, 0.3, 41, collinear=1)
    r1, s1 = oracle.scores(X)
    r2, s2 = oracle.scores(X, reduced=True)
    np.testing.assert_allclose(r2, r1, rtol=1e-8)
    np.testing.assert_allclose(s2, s1, rtol=1e-10, atol=1e-8)


def test_sampled_equals_full():
    X = synthetic.sem_sample(8, 60, 0.3, 51)
    m = 8
    rss, sc = oracle.scores(X)
    rng = np.random.default_rng(1)
    child = rng.integers(0, m, 200)
    mask = np.array([int(rng.integers(0, 1 << m)) & ~(1 << int(c)) for c in child], np.uint64)
    r, s = oracle.scores_sampled(X, child, mask)
    idx = [oracle.table_index(int(c), int(k), m) for c, k in zip(child, mask)]
    np.testing.assert_array_equal(r, rss[idx])
    np.testing.assert_array_equal(s, sc[idx])


def test_gradient_against_finite_differences():
    m, n = 4, 12
    X = synthetic.sem_sample(m, n, 0.5, 61)
    w = np.random.default_rng(2).standard_normal(m << (m - 1))
    g = oracle.grad(X, w)

    def f(Z):
        return float(w @ oracle.scores(Z)[1])

    h = 1e-6
    for t in range(n):
        for j in range(m):
            Zp = X.copy(); Zp[t, j] += h
            Zm = X.copy(); Zm[t, j] -= h
            fd = (f(Zp) - f(Zm)) / (2 * h)
            assert abs(fd - g[t, j]) <= 1e-5 * max(1.0, abs(fd)), (t, j, fd, g[t, j])


@pytest.mark.parametrize("code", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(code):
    X8 = synthetic.sem_sample(8, 50, 0.3, 5)
    X10 = synthetic.workload_sample(synthetic.SMALL_M10)
    oracle.set_mutation(code)
    try:
        results = [_pin_rational(), _pin_lstsq(X8), _pin_invariants(X10), _pin_loglik(SMALL),
                   _pin_layout()]
    finally:
        oracle.set_mutation(0)
    assert not all(results), f"mutation {code} passed every pin"


def _pin_penalised_scores(X, lam):
    """The penalised score against -2 * (Gaussian profile log-likelihood, scipy) + |S| * lam."""
    n, m = X.shape
    Xc = X - X.mean(0)
    _, sc = oracle.scores(X, nthreads=2, penalty=lam)
    for c, S, mask in _families(m):
        y = Xc[:, c]
        e = y - Xc[:, list(S)] @ np.linalg.lstsq(Xc[:, list(S)], y, rcond=None)[0] if S else y
        sigma = np.sqrt(float(e @ e) / n)
        minus2ll = -2.0 * stats.norm.logpdf(e, scale=sigma).sum()
        want = minus2ll - n * np.log(2 * np.pi) - n + len(S) * lam
        if abs(sc[oracle.table_index(c, mask, m)] - want) > 1e-8 * max(1.0, abs(want)):
            return False
    return True


@pytest.mark.parametrize("lam", [2.0, 0.0, 7.5])
def test_penalised_scores_are_gaussian_information_criteria(lam):
    assert _pin_penalised_scores(SMALL, lam)


def _pin_coefficients(X, count=200, seed=0):
    """Coefficients and intercept against LAPACK lstsq on the UNcentred data with a column of
    ones (a different formulation of the same regression), and the RSS of that fit."""
    n, m = X.shape
    rng = np.random.default_rng(seed)
    child = rng.integers(0, m, count).astype(np.int32)
    mask = np.array([int(rng.integers(0, 1 << m)) & ~(1 << int(c)) for c in child], np.uint64)
    beta, rss = oracle.coefficients(X, child, mask, nthreads=2)
    for i, (c, S) in enumerate(zip(child, mask)):
        cols = [v for v in range(m) if (int(S) >> v) & 1]
        A = np.column_stack([X[:, cols], np.ones(n)])
        sol = np.linalg.lstsq(A, X[:, c], rcond=None)[0]
        e = X[:, c] - A @ sol
        want = np.zeros(m + 1)
        want[cols] = sol[:-1]
        want[m] = sol[-1]
        if np.max(np.abs(beta[i] - want) / np.maximum(np.abs(want), 1.0)) > 1e-9:
            return False
        if abs(rss[i] - float(e @ e)) > 1e-9 * float(e @ e):
            return False
    return True


def test_coefficients_against_lstsq_with_intercept():
    assert _pin_coefficients(synthetic.sem_sample(8, 60, 0.4, 21))
    assert _pin_coefficients(synthetic.sem_sample(12, 300, 0.3, 22) + 5.0, seed=1)


def test_coefficients_of_an_exact_linear_model():
    """y = 3 + 2 x0 - x2 exactly: the coefficients are recovered, RSS is zero."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((40, 4))
    X[:, 3] = 3.0 + 2.0 * X[:, 0] - X[:, 2]
    beta, rss = oracle.coefficients(X, [3], [0b101])
    np.testing.assert_allclose(beta[0], [2.0, 0.0, -1.0, 0.0, 3.0], atol=1e-12)
    assert rss[0] < 1e-20


def test_coefficients_with_dependent_parents_are_nan():
    X = synthetic.sem_sample(5, 40, 0.4, 23)
    X[:, 4] = X[:, 1]
    beta, rss = oracle.coefficients(X, [0], [(1 << 1) | (1 << 4)])
    assert np.isnan(beta[0, 1]) and np.isnan(beta[0, 4]) and np.isfinite(rss[0])


def test_sampled_reduced_equals_direct():
    X = synthetic.sem_sample(14, 400, 0.3, 24)
    rng = np.random.default_rng(3)
    child = rng.integers(0, 14, 3000).astype(np.int32)
    mask = np.array([int(rng.integers(0, 1 << 14)) & ~(1 << int(c)) for c in child], np.uint64)
    r1, s1 = oracle.scores_sampled(X, child, mask)
    r2, s2 = oracle.scores_sampled(X, child, mask, reduced=True)
    np.testing.assert_allclose(r2, r1, rtol=1e-10)
    np.testing.assert_allclose(s2, s1, rtol=0, atol=1e-8)
