"""The allocation-free entry point against score_all_families (needs a GPU).

Collected last (file name) so that it also runs after every other GPU test
in the same process; it passes alone as well.
"""
import numpy as np
import pytest
import torch

from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the FP32 walk's score tolerance, |d| <= tol * max(|score|, n)


def _compare(got, ref, n):
    got = got.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref) / np.maximum(np.abs(ref), n)
    assert float(err.max()) <= TOL


@pytest.mark.parametrize("m,n", [(12, 300), (20, 1000)])
def test_noalloc_matches_workspace_entry_twice(m, n):
    X = torch.from_numpy(synthetic.sem_sample(m, n, 0.25, 9000 + m)).cuda()
    ref = binding.score_all_families(X)
    outs = [torch.empty(m << (m - 1), dtype=torch.float32, device="cuda") for _ in range(2)]
    binding.score_all_families_noalloc(X, outs[0])  # first call on the device: symbol lookup
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    binding.score_all_families_noalloc(X, outs[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before  # the second call allocated nothing
    for out in outs:
        _compare(out, ref, n)


def test_noalloc_rejects_oversize_input():
    m, n = 22, 64  # 33 MiB of scratch with the automatic q
    X = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    out = torch.empty(m << (m - 1), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.GivensBNError) as e:
        binding.score_all_families_noalloc(X, out)
    assert e.value.code == -10
