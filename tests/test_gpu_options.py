"""The scoring options through the C ABI against the oracle (needs a GPU).

* score kinds: AIC and a caller's penalty per parent, fused into the walk's store;
* bounded in-degree: only families with |S| <= K are written, the rest of the table is
  left as it was;
* shards of one table (the split of Sec. 6 across calls): each shard writes exactly its
  range of sub-walk CTAs, and the shards together equal one whole call bit for bit;
* the watchdog: a bound shorter than a tape chunk makes the walk's waits expire, the
  kernel records the status and returns, and the next call is unaffected;
* least-squares coefficients of listed families (Sec. 1.1) against the oracle;
* the autotuner: its cached choice is what later calls use, and they stay in parity.

Tolerances as in test_gpu_parity: |d| <= tol * max(|score|, n), tol 1e-4 (FP32 walk),
1e-10 (FP64 walk).
"""
import math
import os
import tempfile
import warnings

import numpy as np
import pytest
import torch

import oracle
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}


def _check(got, ref, n, tol):
    got = np.asarray(got, np.float64)
    both = np.isneginf(got) & np.isneginf(ref)
    assert np.all(np.isfinite(got) | both), "non-finite GPU scores"
    err = np.abs(got - ref) / np.maximum(np.abs(ref), n)
    err[both] = 0.0
    assert float(err.max()) <= tol, f"max scaled error {err.max():.3e} at {int(np.argmax(err))}"


def _parents(m):
    """|S| of every table slot (the popcount of the compressed parent mask)."""
    half = 1 << (m - 1)
    comp = np.arange(m * half) % half
    return np.array([bin(int(x)).count("1") for x in range(half)])[comp]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("score,penalty", [("aic", None), ("penalty", 3.25), ("penalty", 0.0)])
@pytest.mark.parametrize("m,q", [(12, 6), (14, 7), (9, 4)])
def test_score_kinds(precision, score, penalty, m, q):
    n = 150
    X = synthetic.sem_sample(m, n, 0.35, 4100 + m)
    lam = 2.0 if score == "aic" else penalty
    _, ref = oracle.scores(X, penalty=lam)
    Xt = torch.from_numpy(X).cuda()
    got = binding.score_all_families(Xt, precision=precision, q=q, score=score,
                                     penalty=penalty or 0.0)
    _check(got.double().cpu().numpy(), ref, n, TOL[precision])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,q,K", [(12, 6, 0), (12, 6, 1), (13, 7, 3), (14, 6, 5), (16, 8, 2),
                                   (11, 4, 9), (9, 5, 2), (18, 7, 4), (17, 9, 6)])
def test_bounded_in_degree(precision, m, q, K):
    """Slots with |S| <= K carry the oracle's score; every other slot keeps the NaN the table
    was filled with (the walk forms: paired with m >= q + 6, the generic form otherwise, the
    FP64 walk)."""
    if precision == 1 and q > 8:
        pytest.skip("the FP64 walk is compiled for q <= 8")
    n = 120
    X = synthetic.sem_sample(m, n, 0.3, 4200 + 10 * m + K)
    _, ref = oracle.scores(X)
    Xt = torch.from_numpy(X).cuda()
    dt = torch.float64 if precision else torch.float32
    out = torch.full((m << (m - 1),), float("nan"), dtype=dt, device="cuda")
    binding.score_all_families(Xt, out, precision=precision, q=q, max_parents=K)
    got = out.double().cpu().numpy()
    k = _parents(m)
    inside = k <= K
    assert np.all(np.isnan(got[~inside])), "a family above the bound was written"
    _check(got[inside], ref[inside], n, TOL[precision])


@pytest.mark.parametrize("m,q,K", [(12, 6, 2), (16, 7, 3), (9, 4, 1)])
def test_bounded_in_degree_coverage(m, q, K):
    X = synthetic.sem_sample(m, 3 * m, 0.3, 7)
    cnt = binding.score_all_families(torch.from_numpy(X).cuda(), q=q, debug_coverage=True,
                                     max_parents=K).cpu().numpy()
    k = _parents(m)
    assert np.all(cnt[k <= K] == 1) and np.all(cnt[k > K] == 0)


def _shard_slots(m, kfix, W, b, e):
    """Slots a shard writes: families (c, S) with ((S & (2^k - 1)) >> W) in [b, e)."""
    half = 1 << (m - 1)
    idx = np.arange(m * half, dtype=np.int64)
    c = idx // half
    comp = idx % half
    S = (comp & ((1 << c) - 1)) | ((comp >> c) << (c + 1))
    g = (S & ((1 << kfix) - 1)) >> W
    return (g >= b) & (g < e)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("m,q,N", [(14, 6, 2), (15, 7, 3), (16, 6, 4), (18, 8, 5), (13, 7, 4),
                                   (8, 4, 2)])
def test_shards_cover_the_table_once(precision, m, q, N):
    n = 200
    X = synthetic.sem_sample(m, n, 0.3, 4300 + m + N)
    Xt = torch.from_numpy(X).cuda()
    whole = binding.score_all_families(Xt, precision=precision, q=q)
    dt = whole.dtype
    merged = torch.full_like(whole, float("nan"))
    seen = np.zeros(whole.numel(), bool)
    for i in range(N):
        kfix, W, b, e = binding.shard_range(n, m, (i, N), precision, q)
        out = torch.full_like(whole, float("nan"))
        binding.score_all_families(Xt, out, precision=precision, q=q, shard=(i, N))
        mine = _shard_slots(m, kfix, W, b, e)
        got = out.cpu().numpy()
        assert not np.any(np.isnan(got[mine])), f"shard {i}: a slot of its range was not written"
        assert np.all(np.isnan(got[~mine])), f"shard {i}: a slot outside its range was written"
        assert not np.any(seen & mine)
        seen |= mine
        sel = torch.from_numpy(mine).cuda()
        merged[sel] = out[sel]
    assert seen.all()
    assert merged.dtype == dt and torch.equal(merged, whole)


def test_shards_at_m24_bit_equal():
    w = synthetic.PROFILE_M24
    X = torch.from_numpy(synthetic.workload_sample(w)).cuda()
    whole = binding.score_all_families(X)
    merged = torch.empty_like(whole)
    for i in range(2):
        binding.score_all_families(X, merged, shard=(i, 2))  # disjoint slots of one table
    assert torch.equal(merged, whole)


def test_watchdog_expiry_is_reported_and_recoverable():
    """A bound of 1 ns: the consumers' first wait for the producer's tape expires, the
    kernel sets GBN_STATUS_WATCHDOG and returns, the binding raises; the next call with
    the default bound is unaffected."""
    m, n = 20, 400
    X = synthetic.sem_sample(m, n, 0.25, 4400)
    Xt = torch.from_numpy(X).cuda()
    for q in (9, 7):
        with pytest.raises(RuntimeError, match="bounded wait"):
            binding.score_all_families(Xt, q=q, watchdog_ns=1)
    torch.cuda.synchronize()
    got = binding.score_all_families(Xt).cpu().numpy()
    _, ref = oracle.scores(X, reduced=True)
    _check(got, ref, n, TOL[0])


@pytest.mark.parametrize("m,n", [(10, 200), (20, 1000), (26, 5000)])
def test_family_coefficients(m, n):
    X = synthetic.sem_sample(m, n, 0.3, 4500 + m)
    rng = np.random.default_rng(m)
    count = 3000
    child = rng.integers(0, m, count).astype(np.int32)
    mask = np.array([int(rng.integers(0, 1 << m)) & ~(1 << int(c)) for c in child], np.uint64)
    child[:m] = np.arange(m)
    mask[:m] = 0  # empty parent sets
    full = (1 << m) - 1
    child[m:2 * m] = np.arange(m)
    mask[m:2 * m] = [full & ~(1 << c) for c in range(m)]  # every other variable a parent
    want_b, want_r = oracle.coefficients(X, child, mask)
    Xt = torch.from_numpy(X).cuda()
    got_b, got_r = binding.family_coefficients(Xt, child, mask.view(np.int64))
    got_b, got_r = got_b.cpu().numpy(), got_r.cpu().numpy()
    scale = np.maximum(np.abs(want_b), 1.0)
    assert float(np.max(np.abs(got_b - want_b) / scale)) <= 1e-9
    assert float(np.max(np.abs(got_r - want_r) / want_r)) <= 1e-10


def test_family_coefficients_invalid_and_dependent():
    m, n = 8, 60
    X = synthetic.sem_sample(m, n, 0.3, 4600)
    Xt = torch.from_numpy(X).cuda()
    with pytest.raises(ValueError):
        binding.family_coefficients(Xt, [3], [1 << 3])  # parents hold the child
    with pytest.raises(ValueError):
        binding.family_coefficients(Xt, [m], [1])  # child out of range
    X2 = X.copy()
    X2[:, 5] = 2.0 * X2[:, 2]  # an exact dependency between two parents
    with warnings.catch_warnings(record=True) as rec:
        warnings.simplefilter("always")
        b, r = binding.family_coefficients(torch.from_numpy(X2).cuda(), [0], [(1 << 2) | (1 << 5)])
    b = b.cpu().numpy()
    assert any("dependent" in str(x.message) for x in rec)
    assert np.isnan(b[0, 2]) and np.isnan(b[0, 5])
    assert np.isfinite(float(r[0]))


def test_autotune_cache_is_used_and_in_parity():
    m, n = 18, 800
    X = synthetic.sem_sample(m, n, 0.25, 4700)
    Xt = torch.from_numpy(X).cuda()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        q, cw, ms, table = binding.autotune(Xt, tune_cache=path)
        assert len(table) >= 3 and ms > 0
        assert (q, cw) in [(t[0], t[1]) for t in table]
        assert min(t[2] for t in table) == ms
        with open(path) as f:
            lines = f.read().splitlines()
        assert len(lines) == 1 and lines[0].startswith("gbn-tune-v1 ")
        assert binding.plan_choice(n, m, tune_cache=path) == (q, cw)
        tuned = binding.score_all_families(Xt, tune_cache=path)
        explicit = binding.score_all_families(Xt, q=q, consumer_warps=cw)
        assert torch.equal(tuned, explicit)
        _, ref = oracle.scores(X, reduced=True)
        _check(tuned.cpu().numpy(), ref, n, TOL[0])


def test_autotune_batched_cache_is_used():
    Xs_np = [synthetic.sem_sample(m, n, 0.25, 4800 + i)
             for i, (m, n) in enumerate([(12, 300), (14, 500), (13, 200), (15, 700)])]
    Xs = [torch.from_numpy(X).cuda() for X in Xs_np]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.txt")
        q, cw, ms, table = binding.autotune_batched(Xs, tune_cache=path)
        assert (q, cw) in [(t[0], t[1]) for t in table]
        tuned, offs = binding.score_all_families_batched(Xs, tune_cache=path)
        explicit, _ = binding.score_all_families_batched(Xs, q=q, consumer_warps=cw)
        assert torch.equal(tuned, explicit)
        for X, off in zip(Xs_np, offs):
            m, n = X.shape[1], X.shape[0]
            _, ref = oracle.scores(X)
            _check(tuned[off:off + (m << (m - 1))].cpu().numpy(), ref, n, TOL[0])
