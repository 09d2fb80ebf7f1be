"""Pins of the BGe oracle (oracle/bge.py) against facts that do not come from it.

* one variable: ln p(d) equals the marginal likelihood integrated numerically over the
  normal-gamma prior (mu, w) -- the constants, the gamma ratio and the determinant powers;
* two variables: ln p(d_{x0}) and ln p(d_{x0,x1}) equal Monte Carlo averages of the
  likelihood over draws of (mu, W) from the two-variable normal-Wishart prior -- the
  degrees of freedom alpha_w - m + |Y| of a marginal block (a shift by one moves ln p by
  far more than the tolerance);
* three variables: Markov-equivalent DAGs get equal totals and a v-structure does not, read
  through the table layout (a wrong slot breaks the equalities).
"""
import math

import numpy as np
import pytest

from oracle import bge


def _normal_pdf(x, mu, var):
    return np.exp(-0.5 * (x - mu) ** 2 / var) / np.sqrt(2 * np.pi * var)


def test_one_variable_equals_numerical_integration():
    integrate = pytest.importorskip("scipy.integrate")
    x = np.array([0.3, -1.2, 0.8, 0.5])
    X = x[:, None]
    am, aw, t = bge.prior(1)  # alpha_mu 1, alpha_w 3, t = 0.5
    nu = x.mean()

    def integrand(mu, w):  # likelihood x normal(mu | nu, 1/(am w)) x gamma(w | aw/2, rate t/2)
        lik = np.prod(_normal_pdf(x, mu, 1.0 / w))
        prior_mu = _normal_pdf(mu, nu, 1.0 / (am * w))
        prior_w = (t / 2) ** (aw / 2) * w ** (aw / 2 - 1) * math.exp(-t * w / 2) / math.gamma(aw / 2)
        return lik * prior_mu * prior_w

    val, err = integrate.dblquad(integrand, 0.0, 200.0, lambda w: nu - 12.0, lambda w: nu + 12.0,
                                 epsabs=1e-14, epsrel=1e-10)
    assert err < 1e-6 * val
    assert bge.ln_marginal(X, [0]) == pytest.approx(math.log(val), abs=1e-7)
    assert bge.scores(X)[0] == pytest.approx(math.log(val), abs=1e-7)


def test_two_variable_marginals_equal_monte_carlo():
    stats = pytest.importorskip("scipy.stats")
    X = np.array([[0.21, -0.05], [-0.33, -0.41], [0.12, 0.30]])
    n, m = X.shape
    am, aw, t = bge.prior(m)  # alpha_w 4, t = 0.5
    nu = X.mean(axis=0)
    N = 400_000
    W = stats.wishart(df=aw, scale=np.eye(m) / t).rvs(size=N, random_state=np.random.default_rng(7))
    Sigma = np.linalg.inv(W)
    rng = np.random.default_rng(8)
    L = np.linalg.cholesky(Sigma / am)
    mu = nu + np.einsum("nij,nj->ni", L, rng.standard_normal((N, m)))
    # the first variable alone
    lik0 = np.prod(_normal_pdf(X[None, :, 0], mu[:, None, 0], Sigma[:, 0, 0][:, None]), axis=1)
    assert bge.ln_marginal(X, [0]) == pytest.approx(math.log(lik0.mean()), abs=0.03)
    # both variables
    d = X[None, :, :] - mu[:, None, :]
    P = np.linalg.inv(Sigma)
    quad = np.einsum("nki,nij,nkj->nk", d, P, d)
    dens = np.exp(-0.5 * quad) / (2 * np.pi * np.sqrt(np.linalg.det(Sigma)))[:, None]
    lik01 = np.prod(dens, axis=1)
    assert bge.ln_marginal(X, [0, 1]) == pytest.approx(math.log(lik01.mean()), abs=0.03)
    # the degrees of freedom matter: alpha_w one higher moves ln p(d_{x0}) well past 0.03
    assert abs(bge.ln_marginal(X, [0], alpha_w=aw + 1) - bge.ln_marginal(X, [0])) > 0.1


def _total(table, m, parents):
    half = 1 << (m - 1)
    tot = 0.0
    for c, S in enumerate(parents):
        cm = (S & ((1 << c) - 1)) | ((S >> (c + 1)) << c)
        tot += table[c * half + cm]
    return tot


def test_markov_equivalent_dags_score_alike():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 3)) @ np.array([[1.0, 0.5, 0.2], [0.0, 1.0, 0.7], [0.0, 0.0, 1.0]])
    t = bge.scores(X)
    a, b, c = 1, 2, 4  # variable bits
    chain = [0, a, b]          # 0 -> 1 -> 2
    rev = [b, c, 0]            # 0 <- 1 <- 2
    fork = [b, 0, b]           # 0 <- 1 -> 2
    vee = [0, a | c, 0]        # 0 -> 1 <- 2
    full_orders = [[0, a, a | b], [b | c, 0, b], [b | c, c, 0]]  # orders 012, 120, 210
    tc = _total(t, 3, chain)
    assert _total(t, 3, rev) == pytest.approx(tc, abs=1e-9)
    assert _total(t, 3, fork) == pytest.approx(tc, abs=1e-9)
    assert abs(_total(t, 3, vee) - tc) > 1e-6
    full = [_total(t, 3, p) for p in full_orders]
    assert full == pytest.approx([bge.ln_marginal(X, [0, 1, 2])] * 3, abs=1e-9)


def test_improper_prior_is_refused():
    with pytest.raises(ValueError):
        bge.prior(4, alpha_w=5.0)
