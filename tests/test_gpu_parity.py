"""Parity of the CUDA path with the FP64 oracle (needs a GPU).

Tolerance (written here, derived in the design notes): a score matches when
|score_gpu - score_oracle| <= tol * max(|score_oracle|, n), tol = 1e-4 for the
FP32 walk and 1e-10 for the FP64 walk (the relative bound breaks down where a
score crosses zero, so it is taken against max(|score|, n)).  RSS == 0 gives
-inf on both sides.  Coverage counters are compared bit-exactly.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}


def _gpu(X, **kw):
    Xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    out = binding.score_all_families(Xt, **kw)
    torch.cuda.synchronize()
    return out


def _check(got, ref, n, tol):
    got = np.asarray(got, np.float64)
    both = np.isneginf(got) & np.isneginf(ref)
    assert np.all(np.isfinite(got) | both), "non-finite GPU scores"
    err = np.abs(got - ref) / np.maximum(np.abs(ref), n)
    err[both] = 0.0
    worst = int(np.argmax(err))
    assert err[worst] <= tol, f"max scaled error {err[worst]:.3e} at slot {worst}"
    return float(err.max())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,n,q", [(2, 5, 2), (3, 9, 2), (3, 9, 3), (4, 12, 2), (4, 12, 4),
                                   (5, 20, 3), (6, 25, 2), (6, 25, 6), (7, 40, 4), (8, 50, 3),
                                   (9, 60, 5), (10, 200, 4), (11, 100, 6), (12, 80, 7),
                                   (13, 90, 8), (14, 120, 5), (12, 60, 9), (13, 70, 9),
                                   (14, 80, 8), (15, 90, 9)])
def test_all_families_small(precision, m, n, q):
    if precision == 1 and q > 8:
        pytest.skip("the FP64 walk is compiled for q <= 8")
    X = synthetic.sem_sample(m, n, 0.4, 100 + m)
    _, ref = oracle.scores(X)
    got = _gpu(X, precision=precision, q=q).cpu().numpy()
    _check(got, ref, n, TOL[precision])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,q", [(2, 2), (3, 3), (4, 2), (5, 5), (6, 3), (7, 2), (8, 4), (9, 4),
                                 (10, 5), (11, 2), (12, 7), (13, 8), (14, 6), (16, 8), (18, 7),
                                 (12, 9), (16, 9), (20, 9), (21, 9), (22, 8)])
def test_coverage_exactly_once(precision, m, q):
    if precision == 1 and q > 8:
        pytest.skip("the FP64 walk is compiled for q <= 8")
    X = synthetic.sem_sample(m, 3 * m, 0.3, 7)
    cnt = _gpu(X, precision=precision, q=q, debug_coverage=True)
    assert cnt.numel() == m << (m - 1)
    assert int(cnt.min()) == 1 and int(cnt.max()) == 1


@pytest.mark.parametrize("precision", [0, 1])
def test_workload_m10_full(precision):
    w = synthetic.SMALL_M10
    X = synthetic.workload_sample(w)
    _, ref = oracle.scores(X)
    for q in (0, 3, 5, 7, 9):
        if precision == 1 and q > 8:
            continue
        got = _gpu(X, precision=precision, q=q).cpu().numpy()
        _check(got, ref, w.n, TOL[precision])


def test_workload_m20_full_fp32():
    w = synthetic.MEDIUM_M20
    X = synthetic.workload_sample(w)
    _, ref = oracle.scores(X, reduced=True)
    got = _gpu(X).cpu().numpy()
    _check(got, ref, w.n, TOL[0])
    # direct (non-reduced) oracle on seeded samples
    _sampled_direct(X, got, w.n, TOL[0], 2000, seed=20)


def test_workload_m20_full_fp64():
    w = synthetic.MEDIUM_M20
    X = synthetic.workload_sample(w)
    _, ref = oracle.scores(X, reduced=True)
    got = _gpu(X, precision=1).cpu().numpy()
    _check(got, ref, w.n, 1e-9)  # the reduced oracle itself is one QR away from the direct one
    _sampled_direct(X, got, w.n, TOL[1], 1000, seed=21)


def _sample(m, count, seed, extra=()):
    rng = np.random.default_rng(seed)
    child = rng.integers(0, m, count)
    mask = np.array([int(rng.integers(0, 1 << m)) & ~(1 << int(c)) for c in child], np.uint64)
    if extra:
        child = np.concatenate([child, np.array([e[0] for e in extra], np.int64)])
        mask = np.concatenate([mask, np.array([e[1] for e in extra], np.uint64)])
    return child.astype(np.int32), mask


def _slots(child, mask, m):
    return np.array([oracle.table_index(int(c), int(k), m) for c, k in zip(child, mask)], np.int64)


def _sampled_direct(X, table, n, tol, count, seed, extra=()):
    m = X.shape[1]
    child, mask = _sample(m, count, seed, extra)
    _, ref = oracle.scores_sampled(X, child, mask)
    got = np.asarray(table)[_slots(child, mask, m)]
    return _check(got, ref, n, tol)


def _collinear_families(X, count, seed):
    """Families whose child is one of a near-collinear pair and whose parents hold the other."""
    m = X.shape[1]
    C = np.corrcoef(X, rowvar=False)
    pairs = [(a, b) for a in range(m) for b in range(m) if a != b and abs(C[a, b]) > 0.99]
    assert pairs, "expected near-collinear columns"
    rng = np.random.default_rng(seed)
    fams = []
    for _ in range(count):
        a, b = pairs[int(rng.integers(len(pairs)))]
        mask = (int(rng.integers(0, 1 << m)) & ~(1 << a)) | (1 << b)
        fams.append((a, mask))
    return fams


def _device_gather(table: torch.Tensor, slots: np.ndarray) -> np.ndarray:
    idx = torch.from_numpy(slots).to(table.device)
    return table[idx].double().cpu().numpy()


def _collinear_pairs(X, thresh=0.99):
    m = X.shape[1]
    C = np.corrcoef(X, rowvar=False)
    return [(a, b) for a in range(m) for b in range(m) if a != b and abs(C[a, b]) > thresh]


def _every_collinear_family(X):
    """Every family whose child is one column of a near-collinear pair and whose parent set
    holds the other: 2^(m-2) parent sets per ordered pair."""
    m = X.shape[1]
    child, mask = [], []
    for a, b in _collinear_pairs(X):
        rest = np.arange(1 << (m - 2), dtype=np.uint64)
        lo, hi = min(a, b), max(a, b)
        # spread the (m-2)-bit counter over the variables other than a and b
        full = (rest & np.uint64((1 << lo) - 1)) | ((rest >> np.uint64(lo)) << np.uint64(lo + 1))
        full = (full & np.uint64((1 << hi) - 1)) | ((full >> np.uint64(hi)) << np.uint64(hi + 1))
        child.append(np.full(len(rest), a, np.int32))
        mask.append(full | np.uint64(1 << b))
    return np.concatenate(child), np.concatenate(mask)


@pytest.fixture(scope="module")
def m26_reference():
    """Oracle values on the m=26 workload, shared by the FP32 and FP64 checks: 2^20 seeded
    random families and every collinear-pair family (R0-reduced oracle, pinned to the direct
    one), and 2^17 seeded random families plus 1000 collinear ones solved directly on Xc."""
    w = synthetic.LARGE_M26
    X = synthetic.workload_sample(w)
    child_r, mask_r = _sample(w.m, 1 << 20, 2600)
    child_c, mask_c = _every_collinear_family(X)
    assert len(child_c) >= 1 << 24
    child = np.concatenate([child_r, child_c])
    mask = np.concatenate([mask_r, mask_c])
    _, ref_red = oracle.scores_sampled(X, child, mask, reduced=True)
    extra = _collinear_families(X, 1000, 26)
    child_d, mask_d = _sample(w.m, 1 << 17, 2601, extra)
    _, ref_dir = oracle.scores_sampled(X, child_d, mask_d)
    return {"X": X, "w": w, "red": (child, mask, ref_red), "dir": (child_d, mask_d, ref_dir)}


def _slots_np(child, mask, m):
    """idx(c,S) = c 2^(m-1) + compress(S, c), vectorised."""
    c = child.astype(np.uint64)
    low = mask & ((np.uint64(1) << c) - np.uint64(1))
    high = (mask >> (c + np.uint64(1))) << c
    return ((c << np.uint64(m - 1)) + (low | high)).astype(np.int64)


@pytest.mark.parametrize("precision", [0, 1])
def test_workload_m26_sampled(precision, m26_reference):
    """The benchmark's launch configuration (automatic q) on the m=26 workload, compared
    element by element with the oracle on 2^20 + 2^17 seeded families and on every family
    of a near-collinear pair (child one column, parents holding the other)."""
    ref = m26_reference
    w, X = ref["w"], ref["X"]
    table = _gpu(X, precision=precision)
    assert table.numel() == 26 << 25
    assert bool(torch.isfinite(table).all())  # every slot written, none non-finite
    for key in ("red", "dir"):
        child, mask, want = ref[key]
        got = _device_gather(table, _slots_np(child, mask, w.m))
        _check(got, want, w.n, TOL[precision])
    del table
    torch.cuda.empty_cache()


def test_maximum_m30_sampled():
    m, n = 30, 64
    X = synthetic.sem_sample(m, n, 0.1, 3030)
    table = _gpu(X)
    assert table.numel() == 30 << 29
    child, mask = _sample(m, 1500, 30)
    # include the extreme slots of every child block
    ext = [(c, 0) for c in range(m)] + [(c, ((1 << m) - 1) & ~(1 << c)) for c in range(m)]
    c2 = np.concatenate([child, [e[0] for e in ext]]).astype(np.int32)
    k2 = np.concatenate([mask, np.array([e[1] for e in ext], np.uint64)])
    _, ref = oracle.scores_sampled(X, c2, k2)
    got = _device_gather(table, _slots(c2, k2, m))
    _check(got, ref, n, TOL[0])
    del table
    torch.cuda.empty_cache()


@pytest.mark.parametrize("m,n", [(6, 7), (10, 11), (12, 1037), (9, 4099)])
def test_ragged_and_minimal_n(m, n):
    X = synthetic.sem_sample(m, n, 0.3, 500 + n)
    _, ref = oracle.scores(X)
    for precision in (0, 1):
        got = _gpu(X, precision=precision).cpu().numpy()
        _check(got, ref, n, TOL[precision] * (10 if n == m + 1 else 1))


def test_no_centering_option():
    X = synthetic.sem_sample(8, 60, 0.3, 808)
    Xc = X - X.mean(0)
    _, ref = oracle.scores(X)
    got = _gpu(Xc, center=False, precision=1).cpu().numpy()
    _check(got, ref, 60, 1e-9)


def test_deterministic():
    X = synthetic.sem_sample(16, 300, 0.3, 1616)
    a = _gpu(X)
    b = _gpu(X)
    assert torch.equal(a, b)


def test_scale_invariance_of_shape():
    """Scaling all data by a constant shifts every score by n ln(a^2) exactly in theory."""
    X = synthetic.sem_sample(12, 400, 0.3, 1212)
    a = 8.0  # power of two: the data scale exactly
    s1 = _gpu(X, precision=1).cpu().numpy()
    s2 = _gpu(X * a, precision=1).cpu().numpy()
    np.testing.assert_allclose(s2 - s1, 400 * math.log(a * a), rtol=0, atol=1e-8)


def test_table_written_straight_to_pinned_host_memory():
    X = synthetic.sem_sample(14, 300, 0.3, 1400)
    Xt = torch.from_numpy(X).cuda()
    dev = binding.score_all_families(Xt)
    host = torch.empty(14 << 13, dtype=torch.float32, pin_memory=True)
    binding.score_all_families(Xt, host)
    torch.cuda.synchronize()
    assert torch.equal(host, dev.cpu())


@pytest.mark.parametrize("m,q", [(12, 6), (13, 7), (14, 6), (17, 7), (18, 8), (16, 5)])
def test_fp32_walk_forms_write_every_slot(m, q):
    """The FP32 forms for full warps (the paired walk, its persistent ring at
    q <= 6) over a table first filled with NaN: every slot is written, and the
    table matches the oracle.  Cases span one pair of roots CTAs (m = q + 6),
    several persistent units, and q = 5 .. 8."""
    n = 90
    X = synthetic.sem_sample(m, n, 0.3, 7000 + 10 * m + q)
    Xt = torch.from_numpy(X).cuda()
    out = torch.full((m << (m - 1),), float("nan"), dtype=torch.float32, device="cuda")
    binding.score_all_families(Xt, out, q=q)
    torch.cuda.synchronize()
    assert not bool(torch.isnan(out).any()), "a slot was not written"
    _, ref = oracle.scores(X)
    _check(out.cpu().numpy(), ref, n, TOL[0])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("sigma", [0.06, 0.045, 0.02, 0.005])
def test_r0_one_pass_boundary(precision, sigma):
    """Column 3 = column 1 + sigma * noise, so its smallest RSS is about sigma^2 of its sum of
    squares: above 1e-3 the R0 stage takes one Cholesky QR pass, below it two.  Either way
    every score matches the oracle at the walk's tolerance."""
    m, n = 10, 400
    X = synthetic.sem_sample(m, n, 0.3, 9100)
    X[:, 3] = X[:, 1] + sigma * np.std(X[:, 1]) * np.random.default_rng(3).standard_normal(n)
    _, ref = oracle.scores(X)
    got = _gpu(X, precision=precision, q=5)
    _check(got.double().cpu().numpy(), ref, n, TOL[precision])
