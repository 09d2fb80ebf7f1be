"""BGe scores on the GPU against the BGe oracle (needs a GPU).

The oracle (oracle/bge.py) takes numpy log-determinants of every principal block of the
posterior matrix; the GPU walks a factor of it and forms the determinants by a recursion
over the table, so the two share nothing but the definition.  Tolerance as for the RSS
scores: |gpu - oracle| <= tol * max(|oracle|, n), 1e-4 for the FP32 walk, 1e-10 for FP64.
"""
import numpy as np
import pytest
import torch

from oracle import bge
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}


def _check(got, ref, n, tol):
    got = np.asarray(got, np.float64)
    assert np.all(np.isfinite(got)), "non-finite GPU scores"
    err = np.abs(got - ref) / np.maximum(np.abs(ref), n)
    worst = int(np.argmax(err))
    assert err[worst] <= tol, f"max scaled error {err[worst]:.3e} at slot {worst}"


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,q", [(2, 7, 2), (3, 12, 3), (5, 30, 3), (7, 60, 4), (9, 80, 5),
                                   (11, 200, 6), (13, 150, 7), (14, 300, 8)])
def test_bge_equals_the_oracle(precision, m, n, q):
    X = synthetic.sem_sample(m, n, 0.35, 5100 + m)
    got = binding.score_all_families(torch.from_numpy(X).cuda(), precision=precision, q=q,
                                     score="bge")
    _check(got.double().cpu().numpy(), bge.scores(X), n, TOL[precision])


@pytest.mark.parametrize("alpha_mu,alpha_w", [(2.5, 0.0), (0.0, 20.0), (0.3, 13.5)])
def test_bge_prior_parameters(alpha_mu, alpha_w):
    m, n = 10, 120
    X = synthetic.sem_sample(m, n, 0.3, 5200)
    got = binding.score_all_families(torch.from_numpy(X).cuda(), score="bge",
                                     bge_alpha_mu=alpha_mu, bge_alpha_w=alpha_w)
    ref = bge.scores(X, alpha_mu=alpha_mu or 1.0, alpha_w=alpha_w or None)
    _check(got.double().cpu().numpy(), ref, n, TOL[0])


@pytest.mark.parametrize("m,q,K", [(12, 6, 2), (13, 7, 0), (10, 4, 5)])
def test_bge_bounded_in_degree(m, q, K):
    n = 100
    X = synthetic.sem_sample(m, n, 0.3, 5300 + K)
    out = torch.full((m << (m - 1),), float("nan"), dtype=torch.float32, device="cuda")
    binding.score_all_families(torch.from_numpy(X).cuda(), out, q=q, score="bge", max_parents=K)
    got = out.double().cpu().numpy()
    half = 1 << (m - 1)
    k = np.array([bin(x).count("1") for x in range(half)])[np.arange(m * half) % half]
    assert np.all(np.isnan(got[k > K]))
    _check(got[k <= K], bge.scores(X)[k <= K], n, TOL[0])


def test_bge_collinear_data():
    """Two near-collinear columns: the prior's t I keeps every block well conditioned."""
    m, n = 9, 200
    X = synthetic.sem_sample(m, n, 0.3, 5400)
    X[:, 4] = X[:, 1] + 1e-7 * np.random.default_rng(1).standard_normal(n)
    got = binding.score_all_families(torch.from_numpy(X).cuda(), score="bge")
    _check(got.double().cpu().numpy(), bge.scores(X), n, TOL[0])


def test_bge_refusals():
    X = torch.from_numpy(synthetic.sem_sample(6, 40, 0.3, 1)).cuda()
    with pytest.raises(binding.GivensBNError):  # alpha_w must exceed m + 1
        binding.score_all_families(X, score="bge", bge_alpha_w=7.0)
    with pytest.raises(binding.GivensBNError):  # every family is needed for the log-determinants
        binding.score_all_families(X, score="bge", shard=(0, 2))
    with pytest.raises(binding.GivensBNError):
        binding.score_all_families_batched([X, X], score="bge")
