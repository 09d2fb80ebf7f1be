"""Reference oracle for the all-families regression scores (arXiv 1901.07643).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library in ``paper_1901_07643_gb300``
and never imports it.

* ``oracle.c``   -- plain FP64 C: centring, Householder QR per family, BIC
  score, the R0-reduced variant, sampled families, closed-form gradient.
* ``sequence.py`` -- the paper's integer algorithms: GreedySwaps (Algorithm 1),
  SeedPathCalculator (Algorithm 2, corrected reading), the families each QRD
  provides (Sec. 2) and the flop count of Sec. 5.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, OpenMP) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.oracle_scores.argtypes = [d, i64, i32, d, d, ctypes.c_int]
            lib.oracle_scores_reduced.argtypes = [d, i64, i32, d, d, ctypes.c_int]
            lib.oracle_scores_sampled.argtypes = [d, i64, i32, d, d, i64, d, d, ctypes.c_int]
            lib.oracle_grad.argtypes = [d, i64, i32, d, d, ctypes.c_int]
            lib.oracle_r_factor.argtypes = [d, i64, i32, d]
            lib.oracle_center.argtypes = [d, i64, i32, d]
            lib.oracle_compress.argtypes = [ctypes.c_uint64, i32]
            lib.oracle_compress.restype = ctypes.c_uint64
            lib.oracle_set_mutation.argtypes = [ctypes.c_int]
            lib.oracle_num_threads.argtypes = [ctypes.c_int]
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_table_scores.argtypes = [d, i64, i32, ctypes.c_double, d]
            lib.oracle_scores_sampled_reduced.argtypes = [d, i64, i32, d, d, i64, d, d,
                                                          ctypes.c_int]
            lib.oracle_coefficients.argtypes = [d, i64, i32, d, d, i64, d, d, ctypes.c_int]
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads(requested: int = 0) -> int:
    return _load().oracle_num_threads(requested)


def set_mutation(code: int) -> None:
    """Plant a deliberate mistake (oracle self-tests only; 0 = none)."""
    _load().oracle_set_mutation(int(code))


def compress(S: int, c: int) -> int:
    return int(_load().oracle_compress(S, c))


def scores(X, nthreads: int = 0, reduced: bool = False, penalty=None):
    """(rss, score) tables of every family, each m*2^(m-1) FP64 in table layout.

    The score is n ln(RSS/n) + |S| * penalty, penalty = ln n (BIC) by default.
    """
    X = _f64(X)
    n, m = X.shape
    rss = np.empty(m << (m - 1), np.float64)
    sc = np.empty_like(rss)
    fn = _load().oracle_scores_reduced if reduced else _load().oracle_scores
    if fn(_ptr(X), n, m, _ptr(rss), _ptr(sc), nthreads) != 0:
        raise ValueError("oracle: invalid shape")
    if penalty is not None:
        _load().oracle_table_scores(_ptr(rss), n, m, float(penalty), _ptr(sc))
    return rss, sc


def coefficients(X, child, mask, nthreads: int = 0):
    """(beta, rss) of the listed families, directly on Xc: beta is count x (m+1)
    (b_v at column v for v in the parent set, 0 elsewhere, intercept in column m)."""
    X = _f64(X)
    n, m = X.shape
    child = np.ascontiguousarray(child, dtype=np.int32)
    mask = np.ascontiguousarray(mask, dtype=np.uint64)
    beta = np.empty((len(child), m + 1), np.float64)
    rss = np.empty(len(child), np.float64)
    if _load().oracle_coefficients(_ptr(X), n, m, _ptr(child), _ptr(mask), len(child),
                                   _ptr(beta), _ptr(rss), nthreads) != 0:
        raise ValueError("oracle: invalid shape")
    return beta, rss


def scores_sampled(X, child, mask, nthreads: int = 0, reduced: bool = False):
    """(rss, score) of the listed families (child[i], parent bitmask[i]), direct on Xc
    (or, reduced=True, on the oracle's own Householder R0 of Xc)."""
    X = _f64(X)
    n, m = X.shape
    child = np.ascontiguousarray(child, dtype=np.int32)
    mask = np.ascontiguousarray(mask, dtype=np.uint64)
    rss = np.empty(len(child), np.float64)
    sc = np.empty_like(rss)
    fn = _load().oracle_scores_sampled_reduced if reduced else _load().oracle_scores_sampled
    if fn(_ptr(X), n, m, _ptr(child), _ptr(mask), len(child), _ptr(rss), _ptr(sc),
          nthreads) != 0:
        raise ValueError("oracle: invalid shape")
    return rss, sc


def grad(X, w, nthreads: int = 0) -> np.ndarray:
    """d/dX of sum_f w_f * score_f (w in table layout)."""
    X = _f64(X)
    n, m = X.shape
    w = _f64(w)
    assert w.shape == (m << (m - 1),)
    g = np.empty_like(X)
    if _load().oracle_grad(_ptr(X), n, m, _ptr(w), _ptr(g), nthreads) != 0:
        raise ValueError("oracle: invalid shape")
    return g


def r_factor(A) -> np.ndarray:
    """Householder R (m x m, upper triangular) of the rows x m matrix A."""
    A = _f64(A)
    rows, m = A.shape
    R = np.empty((m, m), np.float64)
    _load().oracle_r_factor(_ptr(A), rows, m, _ptr(R))
    return R


def center(X) -> np.ndarray:
    X = _f64(X)
    n, m = X.shape
    Xc = np.empty_like(X)
    _load().oracle_center(_ptr(X), n, m, _ptr(Xc))
    return Xc


def table_index(c: int, S: int, m: int) -> int:
    """idx(c,S) = c*2^(m-1) + compress(S,c)."""
    return (c << (m - 1)) + compress(S, c)
