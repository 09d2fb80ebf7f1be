"""The allocation-free entry point against score_all_families (needs a GPU).

score_all_families_noalloc runs the same plan and the same kernels as
score_all_families with the default options, only with its scratch in the
library's static device array, so the two tables must agree bit for bit; one
call is also compared with the oracle directly.  Collected last (file name)
so that it also runs after every other GPU test in the same process; it
passes alone as well.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_07643_gb300 import binding, synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the FP32 walk's score tolerance, |d| <= tol * max(|score|, n)
STATIC_SCRATCH = 16 << 20  # bytes of the static array (csrc/noalloc.cu)


@pytest.mark.parametrize("m,n", [(12, 300), (20, 1000), (20, 12000)])
def test_noalloc_matches_workspace_entry_twice(m, n):
    """Two calls in a row, each bit-equal to the workspace entry point; (20, 12000) is the
    largest scratch it accepts (304 row panels, the cap)."""
    assert binding.workspace_size(n, m) <= STATIC_SCRATCH
    X = torch.from_numpy(synthetic.sem_sample(m, n, 0.25, 9000 + m)).cuda()
    ref = binding.score_all_families(X)
    outs = [torch.empty(m << (m - 1), dtype=torch.float32, device="cuda") for _ in range(2)]
    binding.score_all_families_noalloc(X, outs[0])
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    binding.score_all_families_noalloc(X, outs[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before  # the second call allocated nothing
    for out in outs:
        assert torch.equal(out, ref)


def test_noalloc_against_the_oracle():
    m, n = 12, 300
    Xn = synthetic.sem_sample(m, n, 0.25, 9012)
    out = torch.empty(m << (m - 1), dtype=torch.float32, device="cuda")
    binding.score_all_families_noalloc(torch.from_numpy(Xn).cuda(), out)
    _, ref = oracle.scores(Xn)
    got = out.double().cpu().numpy()
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref) / np.maximum(np.abs(ref), n)
    assert float(err.max()) <= TOL


@pytest.mark.parametrize("m,n", [(21, 64), (22, 64)])
def test_noalloc_rejects_oversize_input(m, n):
    """m = 21 needs about 19.4 MiB of scratch and m = 22 about 38.5 MiB with the automatic
    q, both above the 16 MiB array: rejected before any device work."""
    assert binding.workspace_size(n, m) > STATIC_SCRATCH
    X = torch.zeros((n, m), dtype=torch.float64, device="cuda")
    out = torch.empty(m << (m - 1), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.GivensBNError) as e:
        binding.score_all_families_noalloc(X, out)
    assert e.value.code == -10
