"""FP64 fix-up of ill-conditioned families in the FP32 walk (needs a GPU).

A child that is almost a copy of one of its parents has an RSS many orders of
magnitude below its own sum of squares.  Such families are listed after the
walk and recomputed in FP64 from R0: the listed slots then carry the FP64
score (to FP32 rounding of the stored value), every other slot is untouched,
and all families stay within the FP32 tolerance of the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu


def _near_copy(m, n, seed, src, dst, var):
    X = synthetic.sem_sample(m, n, 0.3, seed)
    rng = np.random.default_rng(seed + 1)
    X[:, dst] = X[:, src] + rng.normal(0.0, np.sqrt(var), n)
    return X


def _run(X, **kw):
    Xt = torch.from_numpy(X).cuda()
    n, m = X.shape
    ws = torch.empty(binding.workspace_size(n, m, 0, 0, kw.get("fixup_tau")), dtype=torch.uint8,
                     device="cuda")
    out = binding.score_all_families(Xt, workspace=ws, **kw)
    torch.cuda.synchronize()
    listed = int(ws[16:20].view(torch.int32).item())
    return out.double().cpu().numpy(), listed


def _err(got, ref, n):
    return np.abs(got - ref) / np.maximum(np.abs(ref), n)


def test_fixup_repairs_near_copies():
    m, n = 9, 400
    X = _near_copy(m, n, 4242, src=2, dst=6, var=1e-10)
    _, ref = oracle.scores(X)
    got, listed = _run(X)
    off, none = _run(X, fixup_tau=0.0)
    assert listed > 0 and none == 0
    err = _err(got, ref, n)
    assert float(err.max()) <= 1e-4, float(err.max())
    changed = got != off
    assert 0 < int(changed.sum()) <= listed
    # the recomputed slots hold the FP64 score rounded once to FP32
    assert float(err[changed].max()) <= 1e-6
    # every listed family has child 2 or 6 and the other one among its parents
    slots = np.nonzero(changed)[0]
    half = 1 << (m - 1)
    assert set(int(s // half) for s in slots) <= {2, 6}


def test_fixup_lists_nothing_on_well_conditioned_data():
    X = synthetic.workload_sample(synthetic.MEDIUM_M20)
    _, listed = _run(X)
    assert listed == 0


def test_fixup_on_collinear_workload_sampled():
    """m = 26 with two near-collinear columns: sampled families, including the
    collinear ones, within the FP32 tolerance with the fix-up on."""
    w = synthetic.LARGE_M26
    X = synthetic.workload_sample(w)
    Xt = torch.from_numpy(X).cuda()
    table = binding.score_all_families(Xt)
    C = np.corrcoef(X, rowvar=False)
    pairs = [(a, b) for a in range(w.m) for b in range(w.m) if a != b and abs(C[a, b]) > 0.99]
    rng = np.random.default_rng(77)
    child, mask = [], []
    for _ in range(2000):
        a, b = pairs[int(rng.integers(len(pairs)))]
        child.append(a)
        mask.append((int(rng.integers(0, 1 << w.m)) & ~(1 << a)) | (1 << b))
    child = np.array(child, np.int32)
    mask = np.array(mask, np.uint64)
    _, ref = oracle.scores_sampled(X, child, mask)
    slots = torch.tensor([oracle.table_index(int(c), int(k), w.m) for c, k in zip(child, mask)],
                         device="cuda")
    got = table[slots].double().cpu().numpy()
    assert float(_err(got, ref, w.n).max()) <= 1e-4
    del table
    torch.cuda.empty_cache()
