"""The autotuner's cache file on the host (no GPU): which line a plan takes, and the
fallbacks to the automatic choice for a missing, malformed or foreign file."""
import os

import pytest

from paper_1901_07643_gb300 import binding
from paper_1901_07643_gb300 import build as gbn_build


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(binding.LIB_PATH):
        gbn_build.build()
    return binding.load()


def _line(device="*", kind="single", precision=0, m=20, mmin=None, count=1, nlog2=9, q=8, cw=4):
    mmin = m if mmin is None else mmin
    return (f"gbn-tune-v1 device={device} kind={kind} precision={precision} m={m} mmin={mmin} "
            f"count={count} nlog2={nlog2} q={q} cw={cw} ms=1.25\n")


def test_cached_choice_is_taken(tmp_path):
    p = tmp_path / "tune.txt"
    auto = binding.plan_choice(1000, 20)
    p.write_text(_line(q=8, cw=4))  # n = 1000: floor(log2 n) = 9
    assert binding.plan_choice(1000, 20, tune_cache=str(p)) == (8, 4)
    assert binding.plan_choice(1000, 20) == auto  # without the cache: the automatic choice
    # explicit q or consumer_warps win over the cache
    assert binding.plan_choice(1000, 20, q=6, tune_cache=str(p))[0] == 6
    assert binding.plan_choice(1000, 20, consumer_warps=2, tune_cache=str(p)) == (auto[0], 2)


def test_last_matching_line_wins_and_file_changes_are_seen(tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text(_line(q=8, cw=4) + _line(q=7, cw=6))
    assert binding.plan_choice(1000, 20, tune_cache=str(p)) == (7, 6)
    with open(p, "a") as f:
        f.write(_line(q=5, cw=8) + "  \n")
    assert binding.plan_choice(1000, 20, tune_cache=str(p)) == (5, 8)


@pytest.mark.parametrize("text", [
    "garbage\n", "gbn-tune-v1 device=* kind=single\n",
    _line(q=8, cw=4).replace("q=8", "q=x"),
    _line(nlog2=10), _line(m=21), _line(precision=1), _line(kind="batch"),
    _line(device="some_other_gpu"), _line(q=42), _line(q=1), _line(cw=0), _line(cw=9),
])
def test_unusable_lines_fall_back(tmp_path, text):
    p = tmp_path / "tune.txt"
    p.write_text(text)
    assert binding.plan_choice(1000, 20, tune_cache=str(p)) == binding.plan_choice(1000, 20)


def test_missing_file_falls_back(tmp_path):
    assert (binding.plan_choice(1000, 20, tune_cache=str(tmp_path / "none.txt"))
            == binding.plan_choice(1000, 20))


def test_workspace_follows_the_cached_q(tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text(_line(q=8, cw=4))
    assert (binding.workspace_size(1000, 20, tune_cache=str(p))
            == binding.workspace_size(1000, 20, q=8))


@pytest.mark.parametrize("kw", [dict(score="aic"), dict(score="penalty", penalty=1.5),
                                dict(max_parents=3), dict(shard=(1, 3)),
                                dict(consumer_warps=5), dict(watchdog_ns=10 ** 6)])
def test_valid_options_plan(kw):
    assert binding.workspace_size(1000, 20, **kw) > 0


@pytest.mark.parametrize("kw", [dict(shard=(3, 3)), dict(shard=(-1, 2)), dict(shard=(1, 1)),
                                dict(consumer_warps=9), dict(consumer_warps=-1),
                                dict(watchdog_ns=-5), dict(score="penalty", penalty=float("nan"))])
def test_invalid_options_are_rejected(kw):
    with pytest.raises(binding.GivensBNError) as e:
        binding.workspace_size(1000, 20, **kw)
    assert e.value.code == -11


def test_shard_ranges_partition_the_ctas():
    for m, q in ((26, 7), (20, 6), (14, 9), (9, 4), (7, 7)):
        k, W, b0, e0 = binding.shard_range(5000, m, (0, 1), q=q)
        total = 1 << (k - W)
        assert (b0, e0) == (0, total)
        for N in (2, 3, 4, 7, 16):
            ends = []
            prev = 0
            for i in range(N):
                kk, WW, b, e = binding.shard_range(5000, m, (i, N), q=q)
                assert (kk, WW) == (k, W) and b == prev and b <= e
                if total % 2 == 0:
                    assert b % 2 == 0  # pairs of CTAs stay together
                prev = e
                ends.append(e)
            assert prev == total
