"""The C ABI library loads, exports what include/givensbn.h declares, and checks
its arguments on the host (no GPU needed for any of this)."""
import ctypes
import os
import re
import subprocess

import pytest

import oracle
import oracle.sequence as seq
from paper_1901_07643_gb300 import binding
from paper_1901_07643_gb300 import build as gbn_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "givensbn.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(binding.LIB_PATH):
        gbn_build.build()
    return binding.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "score_all_families" in names and len(names) >= 6
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def _ws(n, m, **kw):
    return binding.workspace_size(n, m, **kw)


def test_workspace_size_and_plan(lib):
    assert _ws(200, 10) > 0
    assert _ws(5000, 26) > _ws(1000, 20)
    assert _ws(1000, 20, precision=1) > _ws(1000, 20, precision=0)
    for m in range(2, 31):
        q = binding.auto_q(m, 0)
        assert 2 <= q <= min(9, m)
        assert 2 <= binding.auto_q(m, 1) <= min(8, m)


@pytest.mark.parametrize("n,m,kw,code", [
    (200, 1, {}, -1), (200, 31, {}, -1), (10, 10, {}, -2), (3, 3, {}, -2),
    (200, 10, {"precision": 2}, -8), (200, 14, {"q": 10}, -7), (200, 10, {"q": 1}, -7),
    (200, 4, {"q": 5}, -7), (200, 20, {"q": 9, "precision": 1}, -7),
])
def test_argument_errors(lib, n, m, kw, code):
    with pytest.raises(binding.GivensBNError) as e:
        _ws(n, m, **kw)
    assert e.value.code == code


def test_entry_point_rejects_before_any_device_work(lib):
    o = binding._opts()
    fake = ctypes.c_void_p(1 << 20)
    assert lib.score_all_families(fake, 200, 1, fake, ctypes.byref(o)) == -1
    assert lib.score_all_families(None, 200, 10, fake, ctypes.byref(o)) == -3
    assert lib.score_all_families(fake, 200, 10, fake, None) == -3
    assert lib.score_all_families(fake, 200, 10, fake, ctypes.byref(o)) == -5  # no workspace
    assert lib.score_all_families(ctypes.c_void_p((1 << 20) + 4), 200, 10, fake,
                                  ctypes.byref(o)) == -4
    assert "workspace" in binding.strerror(-5)


def test_device_swap_tables_match_greedy_swaps(tmp_path):
    """The walk's compile-time tables equal Algorithm 1 and the orderings it visits."""
    exe = tmp_path / "seq_dump"
    src = os.path.join(ROOT, "tests", "native", "seq_dump.cu")
    subprocess.run([gbn_build._nvcc(), "-std=c++17", "--expt-relaxed-constexpr", "-o", str(exe),
                    src], check=True, capture_output=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    rows = [list(map(int, ln.split())) for ln in lines if not ln[0] in "US"]
    slots = [list(map(int, ln.split()[1:])) for ln in lines if ln.startswith("S ")]
    for Q in (3, 5, 7, 8):
        sw = seq.greedy_swaps(Q)
        orders = seq.apply_swaps(list(range(Q)), sw)[1:]
        got = {(r[1], r[2]): r[3] for r in slots if r[0] == Q}
        assert len(got) == len(sw) * (Q + 1)
        for t, (o, i) in enumerate(zip(orders, sw)):
            pre = sum(1 << v for v in o[:i])
            for jj in range(Q + 1):
                want = 0xFFFF if (pre >> jj) & 1 else oracle.compress(pre, jj)
                assert got[(t, jj)] == want, (Q, t, jj)
    run = [list(map(int, ln.split()[1:])) for ln in lines if ln.startswith("U ")]
    for Q in range(2, 15):
        got = [r[1] for r in run if r[0] == Q]
        assert got == seq.greedy_swaps(Q) + [0]
    for Q in range(2, 13):
        mine = [r for r in rows if r[0] == Q]
        sw = seq.greedy_swaps(Q)
        assert [r[1] for r in mine] == sw
        orders = seq.apply_swaps(list(range(Q)), sw)[1:]
        for r, o, i in zip(mine, orders, sw):
            assert r[2] == sum(1 << v for v in o[:i])


def test_noalloc_host_rejections(lib):
    """The allocation-free entry point rejects before touching the device."""
    import ctypes
    f = lib.score_all_families_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    assert f(None, 5000, 22, None, None) == -10  # needs more than the 16 MiB static scratch
    assert f(None, 64, 31, None, None) == -1     # m out of range
    assert f(None, 5, 8, None, None) == -2       # n < m + 1
    assert f(None, 100, 12, None, None) == -3    # NULL pointers


def test_batched_host_checks(lib):
    """Batched sizing and argument checks run on the host (no device work)."""
    import ctypes
    B = 3
    ns = (ctypes.c_int64 * B)(100, 50, 400)
    ms = (ctypes.c_int32 * B)(12, 8, 20)
    o = binding.Opts()
    lib.givensbn_default_opts(ctypes.byref(o))
    b = ctypes.c_size_t(0)
    f = lib.givensbn_batched_workspace_size
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(binding.Opts),
                  ctypes.POINTER(ctypes.c_size_t)]
    assert f(ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p), B,
             ctypes.byref(o), ctypes.byref(b)) == 0
    singles = sum(binding.workspace_size(n, m, 0, 6, fixup_tau=0.0) for n, m in zip(ns, ms))
    assert b.value >= singles
    assert f(ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p), 0,
             ctypes.byref(o), ctypes.byref(b)) == -9
    bad = (ctypes.c_int32 * B)(12, 1, 20)
    assert f(ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(bad, ctypes.c_void_p), B,
             ctypes.byref(o), ctypes.byref(b)) == -1
    g = lib.score_all_families_batched
    g.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(binding.Opts)]
    assert g(None, ctypes.cast(ns, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p), B, None,
             None, ctypes.byref(o)) == -3


def test_backward_workspace_and_checks(lib):
    import ctypes
    assert binding.backward_workspace_size(2000, 16, 0, 0) > 0
    o = binding.Opts()
    lib.givensbn_default_opts(ctypes.byref(o))
    f = lib.score_all_families_backward
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.POINTER(binding.Opts)]
    assert f(None, 100, 12, None, None, ctypes.byref(o)) == -3
    assert f(None, 100, 31, None, None, ctypes.byref(o)) == -1
    o.q = 13
    assert f(None, 100, 12, None, None, ctypes.byref(o)) == -7
