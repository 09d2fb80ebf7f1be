"""Data of extreme scale (needs a GPU).

The FP32 stages square R entries, so a column near 2^70 or 2^-70 would overflow or flush
them; the library scales such columns of R0 by powers of two and corrects the children's
scores exactly afterwards.  Here the scores of such data match the FP64 oracle at the usual
tolerance (|gpu - oracle| <= tol * max(|oracle|, n)), with the in-degree bound, shards and
the BGe score too.
"""
import numpy as np
import pytest
import torch

import oracle
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


def _scaled(m, n, seed, exps):
    X = synthetic.sem_sample(m, n, 0.35, seed)
    for j, e in exps.items():
        X[:, j] = np.ldexp(X[:, j], e)
    return X


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("e", [70, -70, 100, -100])
def test_whole_data_scaled(precision, e):
    m, n = 10, 200
    X = _scaled(m, n, 7000, {j: e for j in range(m)})
    _, ref = oracle.scores(X)
    got = binding.score_all_families(torch.from_numpy(X).cuda(), precision=precision, q=5)
    _check(got.double().cpu().numpy(), ref, n, TOL[precision])


@pytest.mark.parametrize("m,q", [(11, 6), (14, 7)])
def test_mixed_column_scales(m, q):
    n = 150
    X = _scaled(m, n, 7100 + m, {0: 45, 3: 80, 5: -75, m - 1: -40})
    _, ref = oracle.scores(X)
    got = binding.score_all_families(torch.from_numpy(X).cuda(), q=q)
    _check(got.double().cpu().numpy(), ref, n, TOL[0])


def test_scaled_with_bound_and_shards():
    m, n, K = 12, 120, 3
    X = _scaled(m, n, 7200, {2: 90, 7: -90})
    _, ref = oracle.scores(X)
    Xt = torch.from_numpy(X).cuda()
    out = torch.full((m << (m - 1),), float("nan"), dtype=torch.float32, device="cuda")
    binding.score_all_families(Xt, out, q=6, max_parents=K)
    got = out.double().cpu().numpy()
    half = 1 << (m - 1)
    k = np.array([bin(x).count("1") for x in range(half)])[np.arange(m * half) % half]
    assert np.all(np.isnan(got[k > K]))
    _check(got[k <= K], ref[k <= K], n, TOL[0])
    whole = binding.score_all_families(Xt, q=6)
    parts = torch.full_like(whole, float("nan"))
    for i in range(2):
        binding.score_all_families(Xt, parts, q=6, shard=(i, 2))
    assert torch.equal(parts, whole)


def test_scaled_bge():
    m, n = 9, 150
    X = _scaled(m, n, 7300, {1: 60, 4: -50})
    got = binding.score_all_families(torch.from_numpy(X).cuda(), score="bge")
    _check(got.double().cpu().numpy(), bge.scores(X), n, TOL[0])
