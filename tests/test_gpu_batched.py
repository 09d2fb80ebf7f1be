"""Batched scoring of many uneven datasets in one set of launches (needs a GPU).

Each dataset's table must equal the single-dataset call with the same sub-walk
size bit for bit (same kernels, same plan), match the oracle within the FP32
tolerance, cover every slot exactly once, and replay identically from a
captured CUDA graph.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


def _uneven(count, seed, m_lo=3, m_hi=12, n_lo=20, n_hi=600):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(max(n_lo, m + 1), n_hi + 1))
        out.append(synthetic.sem_sample(m, n, 0.3, seed * 100 + i, bootstrap=True))
    return out


def _dev(Xs):
    return [torch.from_numpy(X).cuda() for X in Xs]


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_single_calls(precision):
    Xs = _uneven(12, 7)
    Xd = _dev(Xs)
    q = min(binding.auto_q(X.shape[1], precision) for X in Xs)
    out, offs = binding.score_all_families_batched(Xd, precision=precision)
    torch.cuda.synchronize()
    for X, off in zip(Xd, offs):
        m = X.shape[1]
        single = binding.score_all_families(X, precision=precision, q=min(q, m))
        assert torch.equal(out[off:off + (m << (m - 1))], single)


def test_batched_paired_walk_equals_single_calls():
    # every dataset has W = 5 and an even number of walk CTAs (m >= q + 6), so
    # the batch takes the paired walk; single calls at q = 6 take the paired ring
    Xs = _uneven(5, 17, m_lo=12, m_hi=14, n_lo=40, n_hi=300)
    Xd = _dev(Xs)
    out, offs = binding.score_all_families_batched(Xd, q=6)
    torch.cuda.synchronize()
    for X, off in zip(Xd, offs):
        m = X.shape[1]
        single = binding.score_all_families(X, q=6)
        assert torch.equal(out[off:off + (m << (m - 1))], single)
    got = out.double().cpu().numpy()
    X = Xs[0]
    n, m = X.shape
    _, ref = oracle.scores(X)
    g = got[offs[0]:offs[0] + (m << (m - 1))]
    assert float((np.abs(g - ref) / np.maximum(np.abs(ref), n)).max()) <= 1e-4


def test_batched_against_oracle():
    Xs = _uneven(6, 11, m_hi=10)
    out, offs = binding.score_all_families_batched(_dev(Xs))
    got = out.double().cpu().numpy()
    for X, off in zip(Xs, offs):
        n, m = X.shape
        _, ref = oracle.scores(X)
        g = got[off:off + (m << (m - 1))]
        err = np.abs(g - ref) / np.maximum(np.abs(ref), n)
        assert float(err.max()) <= 1e-4


def test_batched_coverage_exactly_once():
    Xs = _uneven(9, 13, m_hi=14)
    cnt, offs = binding.score_all_families_batched(_dev(Xs), debug_coverage=True)
    assert int(cnt.min()) == 1 and int(cnt.max()) == 1


def test_bootstrap_workload_sampled():
    """The 256-dataset bootstrap workload: every table finite; sampled datasets
    equal their single calls and the R0-reduced oracle."""
    Xs = synthetic.batched_bootstrap()
    Xd = _dev(Xs)
    out, offs = binding.score_all_families_batched(Xd)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    q = min(binding.auto_q(X.shape[1], 0) for X in Xs)
    for i in (0, 17, 101, 255):
        m = Xs[i].shape[1]
        single = binding.score_all_families(Xd[i], q=q)
        assert torch.equal(out[offs[i]:offs[i] + (m << (m - 1))], single)
    small = [i for i, X in enumerate(Xs) if X.shape[1] <= 13][:3]
    got = out.double().cpu().numpy()
    for i in small:
        n, m = Xs[i].shape
        _, ref = oracle.scores(Xs[i], reduced=True)
        g = got[offs[i]:offs[i] + (m << (m - 1))]
        err = np.abs(g - ref) / np.maximum(np.abs(ref), n)
        assert float(err.max()) <= 1e-4


def test_batched_graph_capture_replays():
    Xs = _uneven(10, 17)
    Xd = _dev(Xs)
    offs, total = binding.batch_offsets(Xd)
    out = torch.empty(total, dtype=torch.float32, device="cuda")
    ws = torch.empty(binding.batched_workspace_size(Xd), dtype=torch.uint8, device="cuda")
    binding.score_all_families_batched(Xd, out, workspace=ws)  # eager reference (and warm-up)
    torch.cuda.synchronize()
    ref = out.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out.fill_(0.0)
        with torch.cuda.graph(g, stream=s):
            binding.score_all_families_batched(Xd, out, workspace=ws)
    torch.cuda.synchronize()
    out.fill_(0.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # new data in the same buffers: the replay follows it
    Y = _uneven(10, 17)
    for X, Yn in zip(Xd, Y):
        X.copy_(torch.from_numpy(Yn[:X.shape[0], :X.shape[1]] * 2.0))
    g.replay()
    torch.cuda.synchronize()
    fresh, _ = binding.score_all_families_batched(Xd)
    assert torch.equal(out, fresh)
