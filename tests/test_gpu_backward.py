"""The adjoint walk (gradient of sum_f w_f * score_f with respect to X), needs a GPU.

Checked against the oracle's closed-form FP64 gradient and against FP64 central
finite differences of the GPU's own FP64 forward scores (h = 1e-6, 50 entries),
on the gradient workload's shape (m = 16, n = 2000).

Tolerance: |g - g_ref| <= tol * max|g_ref| per entry, tol = 1e-4 for the FP32
walk state and 1e-9 for the FP64 walk (the scale is the gradient's largest
entry because individual entries can cross zero).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-9}


def _bwd(X, w, precision, q=0):
    Xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    g = binding.score_all_families_backward(Xt, wt, precision=precision, q=q)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def _check(g, ref, tol):
    scale = float(np.abs(ref).max())
    err = float(np.abs(g - ref).max())
    assert err <= tol * scale, f"max error {err:.3e} vs scale {scale:.3e}"


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,q", [(2, 5, 0), (3, 9, 0), (4, 12, 2), (5, 20, 5), (6, 30, 3),
                                   (8, 60, 0), (8, 60, 8), (10, 200, 4), (11, 150, 0),
                                   (12, 300, 7)])
def test_backward_matches_oracle_gradient(precision, m, n, q):
    X = synthetic.sem_sample(m, n, 0.4, 600 + m)
    w = np.random.default_rng(m).standard_normal(m << (m - 1))
    ref = oracle.grad(X, w)
    _check(_bwd(X, w, precision, q), ref, TOL[precision])


def test_backward_gradient_workload_against_oracle():
    Xs, w = synthetic.gradient_workload(count=2)
    for X in Xs:
        ref = oracle.grad(X, w)
        _check(_bwd(X, w, 1), ref, TOL[1])
        _check(_bwd(X, w, 0), ref, TOL[0])


def test_backward_finite_differences_gradient_workload():
    """FP64 central differences (h = 1e-6) of the GPU FP64 forward on 50 entries of X."""
    Xs, w = synthetic.gradient_workload(count=1)
    X = Xs[0]
    n, m = X.shape
    wt = torch.from_numpy(w).cuda()
    g64 = _bwd(X, w, 1)
    g32 = _bwd(X, w, 0)
    rng = np.random.default_rng(5)
    ts = rng.integers(0, n, 50)
    js = rng.integers(0, m, 50)
    h = 1e-6

    def loss(Z):
        s = binding.score_all_families(torch.from_numpy(Z).cuda(), precision=1, check=False)
        return float(torch.dot(s, wt))

    scale = float(np.abs(g64).max())
    for t, j in zip(ts, js):
        Zp = X.copy()
        Zp[t, j] += h
        Zm = X.copy()
        Zm[t, j] -= h
        fd = (loss(Zp) - loss(Zm)) / (2 * h)
        assert abs(fd - g64[t, j]) <= 1e-5 * scale + 1e-6 * abs(fd), (t, j, fd, g64[t, j])
        assert abs(fd - g32[t, j]) <= 1e-4 * scale, (t, j, fd, g32[t, j])


def test_autograd_function_matches_entry_point():
    X = synthetic.sem_sample(9, 120, 0.3, 909)
    w = np.random.default_rng(9).standard_normal(9 << 8)
    Xt = torch.from_numpy(X).cuda().requires_grad_(True)
    for precision in (0, 1):
        Xt.grad = None
        s = binding.all_family_scores(Xt, precision=precision)
        (s.double() * torch.from_numpy(w).cuda()).sum().backward()
        direct = _bwd(X, w, precision)
        np.testing.assert_array_equal(Xt.grad.cpu().numpy(), direct)


def test_backward_deterministic():
    X = synthetic.sem_sample(14, 400, 0.3, 1414)
    w = np.random.default_rng(14).standard_normal(14 << 13)
    a = _bwd(X, w, 0)
    b = _bwd(X, w, 0)
    np.testing.assert_array_equal(a, b)


def test_backward_gradient_workload_all_datasets():
    """All 64 datasets of the gradient workload: finite, and FP32 close to FP64."""
    Xs, w = synthetic.gradient_workload()
    for X in Xs:
        g64 = _bwd(X, w, 1)
        g32 = _bwd(X, w, 0)
        assert np.all(np.isfinite(g64))
        _check(g32, g64, TOL[0])


def test_batched_backward_equals_single_calls():
    """Uneven datasets in one batched backward call: each gradient bit-equal to its own
    single-dataset call (same R0 kernels, same sub-walks on the same warps, same sums)."""
    shapes = [(8, 60), (12, 300), (10, 200), (14, 500), (9, 90)]
    Xs = [synthetic.sem_sample(m, n, 0.3, 990 + i) for i, (m, n) in enumerate(shapes)]
    rng = np.random.default_rng(99)
    ws = [rng.standard_normal(m << (m - 1)) for m, _ in shapes]
    for precision in (0, 1):
        Xt = [torch.from_numpy(X).cuda() for X in Xs]
        wt = [torch.from_numpy(w).cuda() for w in ws]
        got = binding.score_all_families_backward_batched(Xt, wt, precision=precision)
        torch.cuda.synchronize()
        for X, w, g in zip(Xs, ws, got):
            single = _bwd(X, w, precision)
            np.testing.assert_array_equal(g.cpu().numpy(), single)
            if precision == 0:
                _check(g.cpu().numpy(), oracle.grad(X, w), TOL[0])


def test_batched_backward_gradient_workload():
    """The 64-dataset gradient workload in one batched call, against single calls."""
    Xs, w = synthetic.gradient_workload()
    Xt = [torch.from_numpy(X).cuda() for X in Xs]
    wt = torch.from_numpy(w).cuda()
    got = binding.score_all_families_backward_batched(Xt, wt)
    for i in (0, 31, 63):
        np.testing.assert_array_equal(got[i].cpu().numpy(), _bwd(Xs[i], w, 0))
