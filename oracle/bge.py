"""BGe local scores of every family, in plain FP64 numpy (TEST INFRASTRUCTURE ONLY).

The BGe score (Geiger and Heckerman, "Parameter priors for directed acyclic graphical
models and the characterization of several probability distributions", Ann. Statist.
2002; with the correction of Kuipers, Moffa and Heckerman, "Addendum on the scoring of
Gaussian directed acyclic graphical models", Ann. Statist. 2014) is the log marginal
likelihood of Gaussian data under a normal-Wishart prior on (mu, W), W the precision:

    W ~ Wishart(alpha_w, T0^-1),   mu | W ~ N(nu, (alpha_mu W)^-1).

For a set Y of |Y| variables, with n samples, m variables in the network,
R = T0 + S_n + (n alpha_mu / (n + alpha_mu)) (nu - xbar)(nu - xbar)^T (S_n the centred
scatter matrix) and Gamma_p the multivariate gamma function,

    ln p(d_Y) = (|Y|/2) ln(alpha_mu / (n + alpha_mu)) - (n |Y| / 2) ln pi
                + ln Gamma_|Y|((n + alpha_w - m + |Y|) / 2) - ln Gamma_|Y|((alpha_w - m + |Y|) / 2)
                + ((alpha_w - m + |Y|) / 2) ln det T0_YY - ((n + alpha_w - m + |Y|) / 2) ln det R_YY,

and the local score of child c with parents S is ln p(d_{S u c}) - ln p(d_S).

Readings (the common defaults of the published BGe implementations):
  * nu = xbar, so the mean term of R vanishes and R = T0 + S_n;
  * T0 = t I with t = alpha_mu (alpha_w - m - 1) / (alpha_mu + 1) (Kuipers et al. 2014);
  * alpha_mu = 1 and alpha_w = m + 2 unless given (alpha_w > m + 1 keeps t > 0).

The determinants come straight from numpy's slogdet of each principal submatrix; nothing
here uses the walk or a Cholesky update, so the GPU path (a walk over a factor of R plus a
log-determinant recursion) is checked against an independent computation.
"""
from __future__ import annotations

import math

import numpy as np


def prior(m: int, alpha_mu: float = 1.0, alpha_w: float | None = None):
    """(alpha_mu, alpha_w, t) with the defaults above; raises on an improper prior."""
    aw = float(m + 2) if alpha_w is None else float(alpha_w)
    am = float(alpha_mu)
    if not (am > 0 and aw > m + 1):
        raise ValueError("BGe needs alpha_mu > 0 and alpha_w > m + 1")
    return am, aw, am * (aw - m - 1) / (am + 1)


def ln_mvgamma(p: int, x: float) -> float:
    """ln Gamma_p(x) = p(p-1)/4 ln pi + sum_{j=1..p} ln Gamma(x + (1 - j)/2)."""
    return p * (p - 1) / 4.0 * math.log(math.pi) + sum(math.lgamma(x + (1 - j) / 2.0)
                                                       for j in range(1, p + 1))


def _posterior(X, alpha_mu, alpha_w):
    """(n, m, alpha_mu, alpha_w, t, R) with R = t I + S_n (nu = xbar)."""
    X = np.asarray(X, dtype=np.float64)
    n, m = X.shape
    am, aw, t = prior(m, alpha_mu, alpha_w)
    Xc = X - X.mean(axis=0)
    return n, m, am, aw, t, t * np.eye(m) + Xc.T @ Xc


def _ln_p(R, Y, n, m, am, aw, t) -> float:
    """ln p(d_Y) from the posterior matrix R (the formula of the module docstring)."""
    k = len(Y)
    if k == 0:
        return 0.0
    sign, logdet_r = np.linalg.slogdet(R[np.ix_(Y, Y)])
    if sign <= 0:
        raise ValueError("R_YY is not positive definite")
    return (k / 2.0 * math.log(am / (n + am)) - n * k / 2.0 * math.log(math.pi)
            + ln_mvgamma(k, (n + aw - m + k) / 2.0) - ln_mvgamma(k, (aw - m + k) / 2.0)
            + (aw - m + k) / 2.0 * k * math.log(t) - (n + aw - m + k) / 2.0 * logdet_r)


def ln_marginal(X, Y, alpha_mu: float = 1.0, alpha_w: float | None = None) -> float:
    """ln p(d_Y) for the variable set Y (a list of column indices) of data X (n x m)."""
    n, m, am, aw, t, R = _posterior(X, alpha_mu, alpha_w)
    return _ln_p(R, list(Y), n, m, am, aw, t)


def scores(X, alpha_mu: float = 1.0, alpha_w: float | None = None) -> np.ndarray:
    """Every family's BGe local score in table layout: slot c * 2^(m-1) + the parent mask
    with bit c removed (the layout of the library's score table)."""
    n, m, am, aw, t, R = _posterior(X, alpha_mu, alpha_w)
    lnp = np.empty(1 << m)
    for S in range(1 << m):
        lnp[S] = _ln_p(R, [v for v in range(m) if (S >> v) & 1], n, m, am, aw, t)
    half = 1 << (m - 1)
    out = np.empty(m * half)
    for c in range(m):
        for cm in range(half):
            S = (cm & ((1 << c) - 1)) | ((cm >> c) << (c + 1))
            out[c * half + cm] = lnp[S | (1 << c)] - lnp[S]
    return out


def scores_sampled(X, child, mask, alpha_mu: float = 1.0, alpha_w: float | None = None):
    """BGe scores of listed families (child[i], parent bitmask mask[i]) of data X."""
    n, m, am, aw, t, R = _posterior(X, alpha_mu, alpha_w)
    out = np.empty(len(child))
    for i, (c, S) in enumerate(zip(child, mask)):
        par = [v for v in range(m) if (int(S) >> v) & 1]
        out[i] = _ln_p(R, sorted(par + [int(c)]), n, m, am, aw, t) - _ln_p(R, par, n, m, am, aw, t)
    return out
