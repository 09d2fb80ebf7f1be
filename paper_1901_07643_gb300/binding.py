"""ctypes binding of libgivensbn (argument marshalling only).

Every step of the scoring path runs in the CUDA library; these functions only
turn torch tensors into pointers, size the workspace and translate error
codes.  There is no CPU fallback: if the library is not built or the tensors
are not on a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
import warnings

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgivensbn.so")
_lock = threading.Lock()
_lib = None

GBN_STATUS_RANK_DEFICIENT = 1
GBN_STATUS_WATCHDOG = 2
GBN_STATUS_FIXUP_OVERFLOW = 4
GBN_STATUS_BAD_FAMILY = 8

SCORE_BIC, SCORE_AIC, SCORE_PENALTY, SCORE_BGE = 0, 1, 2, 3
_SCORES = {"bic": SCORE_BIC, "aic": SCORE_AIC, "penalty": SCORE_PENALTY, "bge": SCORE_BGE}


def _check_status(st: int) -> None:
    if st & GBN_STATUS_WATCHDOG:
        raise RuntimeError("givensbn: a bounded wait in the walk expired; the table is incomplete")
    if st & GBN_STATUS_RANK_DEFICIENT:
        warnings.warn("givensbn: data rank deficient; some RSS are 0 (scores -inf)")
    if st & GBN_STATUS_FIXUP_OVERFLOW:
        warnings.warn("givensbn: more ill-conditioned families than the FP64 fix-up list holds; "
                      "the rest keep FP32 scores")


class Opts(ctypes.Structure):
    """Mirror of givensbn_opts (include/givensbn.h)."""
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("center", ctypes.c_int32),
        ("q", ctypes.c_int32),
        ("debug_coverage", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("stage_events", ctypes.c_void_p),
        ("fixup_tau", ctypes.c_double),
        ("watchdog_ns", ctypes.c_int64),
        ("max_parents", ctypes.c_int32),
        ("score", ctypes.c_int32),
        ("penalty", ctypes.c_double),
        ("shard_index", ctypes.c_int32),
        ("shard_count", ctypes.c_int32),
        ("consumer_warps", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("tune_cache", ctypes.c_char_p),
        ("bge_alpha_mu", ctypes.c_double),
        ("bge_alpha_w", ctypes.c_double),
    ]


class TuneResult(ctypes.Structure):
    """Mirror of givensbn_tune_result."""
    _fields_ = [("q", ctypes.c_int32), ("consumer_warps", ctypes.c_int32), ("ms", ctypes.c_double)]


def load():
    """Load libgivensbn.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libgivensbn.so not found at {LIB_PATH}; build it with "
                    "`python -m paper_1901_07643_gb300.build`")
            lib = ctypes.CDLL(LIB_PATH)
            P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.givensbn_default_opts.argtypes = [ctypes.POINTER(Opts)]
            lib.givensbn_workspace_size.argtypes = [i64, i32, ctypes.POINTER(Opts),
                                                    ctypes.POINTER(ctypes.c_size_t)]
            lib.score_all_families.argtypes = [P, i64, i32, P, ctypes.POINTER(Opts)]
            lib.givensbn_status.argtypes = [ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_int32)]
            lib.givensbn_strerror.argtypes = [ctypes.c_int]
            lib.givensbn_strerror.restype = ctypes.c_char_p
            lib.givensbn_auto_q.argtypes = [i32, i32]
            lib.givensbn_auto_q.restype = i32
            lib.score_all_families_noalloc.argtypes = [P, i64, i32, P, P]
            lib.score_all_families_batched.argtypes = [P, P, P, i32, P, P, ctypes.POINTER(Opts)]
            lib.givensbn_batched_workspace_size.argtypes = [P, P, i32, ctypes.POINTER(Opts),
                                                            ctypes.POINTER(ctypes.c_size_t)]
            lib.score_all_families_backward.argtypes = [P, i64, i32, P, P, ctypes.POINTER(Opts)]
            lib.givensbn_backward_workspace_size.argtypes = [i64, i32, ctypes.POINTER(Opts),
                                                             ctypes.POINTER(ctypes.c_size_t)]
            I32P, I64P = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
            SZP, DP = ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_double)
            OP = ctypes.POINTER(Opts)
            lib.givensbn_plan_choice.argtypes = [i64, i32, OP, I32P, I32P]
            lib.givensbn_shard_range.argtypes = [i64, i32, OP, I32P, I32P, I64P, I64P]
            lib.givensbn_autotune_workspace_size.argtypes = [i64, i32, OP, SZP]
            lib.givensbn_autotune.argtypes = [P, i64, i32, P, OP, I32P, I32P, DP,
                                              ctypes.POINTER(TuneResult), i32, I32P]
            lib.givensbn_autotune_batched_workspace_size.argtypes = [P, P, i32, OP, SZP]
            lib.givensbn_autotune_batched.argtypes = [P, P, P, i32, P, P, OP, I32P, I32P, DP,
                                                      ctypes.POINTER(TuneResult), i32, I32P]
            lib.givensbn_coefficients_workspace_size.argtypes = [i64, i32, OP, SZP]
            lib.givensbn_family_coefficients.argtypes = [P, i64, i32, P, P, i64, P, P, OP]
            lib.givensbn_best_parents.argtypes = [P, i32, P, P, OP]
            lib.givensbn_pipe_peaks.argtypes = [P, P, DP, DP]
            lib.givensbn_dmma_peak.argtypes = [P, P, DP]
            lib.score_all_families_backward_batched.argtypes = [P, P, P, i32, P, P, OP]
            lib.givensbn_backward_batched_workspace_size.argtypes = [P, P, i32, OP, SZP]
            lib.givensbn_structure_search_workspace_size.argtypes = [i32, SZP]
            lib.givensbn_structure_search.argtypes = [P, i32, P, P, P, OP]
            _lib = lib
    return _lib


class GivensBNError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"givensbn error {code}: {strerror(code)}")
        self.code = code


def strerror(code: int) -> str:
    return load().givensbn_strerror(code).decode()


def auto_q(m: int, precision: int = 0) -> int:
    return int(load().givensbn_auto_q(m, precision))


def _opts(precision=0, q=0, center=True, debug_coverage=False, stream=None,
          workspace=None, stage_events=None, fixup_tau=None, *, score="bic", penalty=0.0,
          max_parents=None, shard=None, consumer_warps=0, watchdog_ns=0,
          tune_cache=None, bge_alpha_mu=0.0, bge_alpha_w=0.0) -> Opts:
    o = Opts()
    load().givensbn_default_opts(ctypes.byref(o))
    if fixup_tau is not None:
        o.fixup_tau = float(fixup_tau)
    if score not in _SCORES:
        raise ValueError(f"score must be one of {sorted(_SCORES)}")
    o.score = _SCORES[score]
    o.penalty = float(penalty)
    o.bge_alpha_mu = float(bge_alpha_mu)
    o.bge_alpha_w = float(bge_alpha_w)
    o.max_parents = -1 if max_parents is None else int(max_parents)
    if shard is not None:
        o.shard_index, o.shard_count = int(shard[0]), int(shard[1])
    o.consumer_warps = int(consumer_warps)
    o.watchdog_ns = int(watchdog_ns)
    if tune_cache is not None:
        o._cache_keepalive = os.fsencode(tune_cache)
        o.tune_cache = o._cache_keepalive
    o.precision = int(precision)
    o.q = int(q)
    o.center = 1 if center else 0
    o.debug_coverage = 1 if debug_coverage else 0
    o.stream = stream
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    if stage_events is not None:
        assert len(stage_events) == 4
        arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in stage_events])
        o._events_keepalive = arr
        o.stage_events = ctypes.cast(arr, ctypes.c_void_p)
    return o


# keyword options of the scoring calls that shape the plan (see givensbn_opts)
_PLAN_KEYS = ("score", "penalty", "max_parents", "shard", "consumer_warps", "watchdog_ns",
              "tune_cache", "bge_alpha_mu", "bge_alpha_w")


def workspace_size(n: int, m: int, precision: int = 0, q: int = 0, fixup_tau=None,
                   **plan) -> int:
    o = _opts(precision, q, fixup_tau=fixup_tau, **plan)
    b = ctypes.c_size_t(0)
    rc = load().givensbn_workspace_size(n, m, ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    return int(b.value)


def backward_workspace_size(n: int, m: int, precision: int = 0, q: int = 0) -> int:
    o = _opts(precision, q)
    b = ctypes.c_size_t(0)
    rc = load().givensbn_backward_workspace_size(n, m, ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    return int(b.value)


def _stream_handle(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def plan_choice(n: int, m: int, precision: int = 0, q: int = 0, **plan):
    """(q, consumer warps) a scoring call with these options would use."""
    o = _opts(precision, q, **plan)
    qq, cw = ctypes.c_int32(0), ctypes.c_int32(0)
    rc = load().givensbn_plan_choice(n, m, ctypes.byref(o), ctypes.byref(qq), ctypes.byref(cw))
    if rc:
        raise GivensBNError(rc)
    return int(qq.value), int(cw.value)


def shard_range(n: int, m: int, shard, precision: int = 0, q: int = 0, **plan):
    """(k, W, cta_begin, cta_end) of shard = (index, count): the families (c, S) this shard
    writes are those with ((S & (2^k - 1)) >> W) in [cta_begin, cta_end)."""
    o = _opts(precision, q, shard=shard, **plan)
    k, W = ctypes.c_int32(0), ctypes.c_int32(0)
    b, e = ctypes.c_int64(0), ctypes.c_int64(0)
    rc = load().givensbn_shard_range(n, m, ctypes.byref(o), ctypes.byref(k), ctypes.byref(W),
                                     ctypes.byref(b), ctypes.byref(e))
    if rc:
        raise GivensBNError(rc)
    return int(k.value), int(W.value), int(b.value), int(e.value)


def score_all_families(X: torch.Tensor, out: torch.Tensor | None = None, *, precision: int = 0,
                       q: int = 0, center: bool = True, debug_coverage: bool = False,
                       workspace: torch.Tensor | None = None, stream=None,
                       stage_events=None, check: bool = True, fixup_tau=None,
                       **plan) -> torch.Tensor:
    """Scores of all m * 2^(m-1) families of the n x m data X (CUDA float64, row-major).

    Returns a 1-D tensor in table layout (float32 for precision 0, float64 for
    precision 1, int32 counters for debug_coverage).  `out` may be a pinned host
    tensor: the kernels then write the table straight into host memory.  check=True synchronises
    and warns if the data were rank deficient.  stage_events: four
    torch.cuda.Event(enable_timing=True) recorded at the stage boundaries.
    Further keyword options (givensbn_opts): score ("bic", "aic", "penalty", "bge") with
    penalty or bge_alpha_mu / bge_alpha_w (0 = the defaults 1 and m + 2), max_parents
    (in-degree bound; slots of larger families are left as they are in `out`),
    shard = (index, count), consumer_warps, watchdog_ns, tune_cache (path of the
    autotuner's cache file).
    """
    for key in plan:
        if key not in _PLAN_KEYS:
            raise TypeError(f"unexpected option {key!r}")
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2):
        raise TypeError("X must be a 2-D float64 CUDA tensor")
    X = X.contiguous()
    n, m = X.shape
    dev = X.device
    if out is None:
        size = m << (m - 1)
        if debug_coverage:
            out = torch.zeros(size, dtype=torch.int32, device=dev)
        else:
            out = torch.empty(size, dtype=torch.float64 if precision else torch.float32, device=dev)
    elif not (out.device == dev or (out.device.type == "cpu" and out.is_pinned())):
        raise ValueError("out must be on X's device or in pinned host memory")
    if workspace is None:
        workspace = torch.empty(workspace_size(n, m, precision, q, fixup_tau, **plan),
                                dtype=torch.uint8, device=dev)
    if stage_events is not None:
        for e in stage_events:  # torch creates the CUDA event on its first record()
            if not e.cuda_event:
                e.record(stream if stream is not None else torch.cuda.current_stream(dev))
    o = _opts(precision, q, center, debug_coverage, _stream_handle(stream, dev), workspace,
              stage_events, fixup_tau, **plan)
    rc = load().score_all_families(ctypes.c_void_p(X.data_ptr()), n, m,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    if check:
        st = ctypes.c_int32(0)
        rc = load().givensbn_status(ctypes.byref(o), ctypes.byref(st))
        if rc:
            raise GivensBNError(rc)
        _check_status(st.value)
    return out


def score_all_families_noalloc(X: torch.Tensor, out: torch.Tensor, *, stream=None) -> torch.Tensor:
    """FP32 scores of all families through the library's allocation-free entry point.

    The library uses its own 16 MiB static device scratch (m <= 20) and takes
    no workspace; `out` (float32, m * 2^(m-1) elements, on X's device) must be
    supplied by the caller.  Calls on one device must not overlap.
    """
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2):
        raise TypeError("X must be a 2-D float64 CUDA tensor")
    if not X.is_contiguous():
        raise ValueError("X must be contiguous (row-major)")
    n, m = X.shape
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
            and out.numel() == m << (m - 1) and out.device == X.device):
        raise ValueError("out must be a contiguous float32 tensor of m * 2^(m-1) elements on X's device")
    rc = load().score_all_families_noalloc(ctypes.c_void_p(X.data_ptr()), n, m,
                                           ctypes.c_void_p(out.data_ptr()),
                                           _stream_handle(stream, X.device))
    if rc:
        raise GivensBNError(rc)
    return out


def score_all_families_backward(X: torch.Tensor, w: torch.Tensor, *, precision: int = 0, q: int = 0,
                                center: bool = True, workspace: torch.Tensor | None = None,
                                stream=None, check: bool = True) -> torch.Tensor:
    """Gradient of sum_f w_f * score_f with respect to X (float64, n x m).

    w: weights in table layout (m * 2^(m-1)); float32 for precision 0 (FP32
    walk), float64 for precision 1.
    """
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2):
        raise TypeError("X must be a 2-D float64 CUDA tensor")
    X = X.contiguous()
    n, m = X.shape
    wdt = torch.float64 if precision else torch.float32
    w = w.to(device=X.device, dtype=wdt).contiguous()
    if w.numel() != m << (m - 1):
        raise ValueError("w must hold m * 2^(m-1) weights")
    grad = torch.empty_like(X)
    if workspace is None:
        workspace = torch.empty(backward_workspace_size(n, m, precision, q), dtype=torch.uint8,
                                device=X.device)
    o = _opts(precision, q, center, False, _stream_handle(stream, X.device), workspace)
    rc = load().score_all_families_backward(ctypes.c_void_p(X.data_ptr()), n, m,
                                            ctypes.c_void_p(w.data_ptr()),
                                            ctypes.c_void_p(grad.data_ptr()), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    if check:
        st = ctypes.c_int32(0)
        rc = load().givensbn_status(ctypes.byref(o), ctypes.byref(st))
        if rc:
            raise GivensBNError(rc)
        if st.value & GBN_STATUS_RANK_DEFICIENT:
            warnings.warn("givensbn: singular sub-walk factor or Gram matrix in the backward pass")
    return grad


class AllFamilyScores(torch.autograd.Function):
    """Differentiable scores: forward = score_all_families, backward = the adjoint walk."""

    @staticmethod
    def forward(ctx, X, precision=0, q=0, center=True):
        ctx.save_for_backward(X)
        ctx.opts = (precision, center)
        return score_all_families(X.detach(), precision=precision, q=q, center=center)

    @staticmethod
    def backward(ctx, grad_scores):
        (X,) = ctx.saved_tensors
        precision, center = ctx.opts
        g = score_all_families_backward(X.detach(), grad_scores, precision=precision,
                                        center=center)
        return g, None, None, None


def all_family_scores(X: torch.Tensor, precision: int = 0, q: int = 0,
                      center: bool = True) -> torch.Tensor:
    """Scores of all families with autograd support (gradient through the adjoint walk)."""
    return AllFamilyScores.apply(X, precision, q, center)


def _batch_arrays(Xs):
    B = len(Xs)
    ns = (ctypes.c_int64 * B)(*[int(X.shape[0]) for X in Xs])
    ms = (ctypes.c_int32 * B)(*[int(X.shape[1]) for X in Xs])
    return B, ns, ms


def batched_workspace_size(Xs, precision: int = 0, q: int = 0, **plan) -> int:
    B, ns, ms = _batch_arrays(Xs)
    o = _opts(precision, q, **plan)
    b = ctypes.c_size_t(0)
    rc = load().givensbn_batched_workspace_size(ctypes.cast(ns, ctypes.c_void_p),
                                                ctypes.cast(ms, ctypes.c_void_p), B,
                                                ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    return int(b.value)


def batch_offsets(Xs):
    """Element offsets of each dataset's table in the concatenated output."""
    offs, pos = [], 0
    for X in Xs:
        m = int(X.shape[1])
        offs.append(pos)
        pos += m << (m - 1)
    return offs, pos


def score_all_families_batched(Xs, out: torch.Tensor | None = None, *, precision: int = 0,
                               q: int = 0, center: bool = True, debug_coverage: bool = False,
                               workspace: torch.Tensor | None = None, stream=None, **plan):
    """Scores of every family of every dataset in Xs (list of n_b x m_b float64 CUDA tensors).

    Returns (out, offsets): the tables concatenated in the order of Xs, and the
    element offset of each.  Safe to capture in a CUDA graph when `out` and
    `workspace` are supplied.
    """
    if not Xs:
        raise ValueError("empty batch")
    dev = Xs[0].device
    for X in Xs:
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64
                and X.dim() == 2 and X.is_contiguous() and X.device == dev):
            raise TypeError("every X must be a contiguous 2-D float64 CUDA tensor on one device")
    B, ns, ms = _batch_arrays(Xs)
    offs, total = batch_offsets(Xs)
    if out is None:
        if debug_coverage:
            out = torch.zeros(total, dtype=torch.int32, device=dev)
        else:
            out = torch.empty(total, dtype=torch.float64 if precision else torch.float32, device=dev)
    if out.numel() < total:
        raise ValueError("out is too small for the batch")
    if workspace is None:
        workspace = torch.empty(batched_workspace_size(Xs, precision, q, **plan),
                                dtype=torch.uint8, device=dev)
    ptrs = (ctypes.c_void_p * B)(*[X.data_ptr() for X in Xs])
    offa = (ctypes.c_int64 * B)(*offs)
    o = _opts(precision, q, center, debug_coverage, _stream_handle(stream, dev), workspace,
              **plan)
    rc = load().score_all_families_batched(ctypes.cast(ptrs, ctypes.c_void_p),
                                           ctypes.cast(ns, ctypes.c_void_p),
                                           ctypes.cast(ms, ctypes.c_void_p), B,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.cast(offa, ctypes.c_void_p), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    return out, offs


def _check_x(X):
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64 and X.dim() == 2):
        raise TypeError("X must be a 2-D float64 CUDA tensor")
    return X.contiguous()


def autotune(X: torch.Tensor, *, precision: int = 0, tune_cache=None, center: bool = True,
             stream=None, **plan):
    """Time the candidate (q, consumer warps) plans of score_all_families on X.

    Returns (q, consumer_warps, ms, [(q, cw, ms), ...]); with tune_cache the winner
    is appended to that file and later calls with tune_cache=... take it.
    """
    X = _check_x(X)
    n, m = X.shape
    dev = X.device
    o = _opts(precision, 0, center, False, _stream_handle(stream, dev), None, tune_cache=tune_cache,
              **plan)
    b = ctypes.c_size_t(0)
    rc = load().givensbn_autotune_workspace_size(n, m, ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    ws = torch.empty(int(b.value), dtype=torch.uint8, device=dev)
    o.workspace, o.workspace_bytes = ws.data_ptr(), int(b.value)
    out = torch.empty(m << (m - 1), dtype=torch.float64 if precision else torch.float32, device=dev)
    q, cw, ms, nres = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0), ctypes.c_int32(0)
    res = (TuneResult * 32)()
    rc = load().givensbn_autotune(ctypes.c_void_p(X.data_ptr()), n, m, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.byref(o), ctypes.byref(q), ctypes.byref(cw), ctypes.byref(ms),
                                  res, 32, ctypes.byref(nres))
    if rc:
        raise GivensBNError(rc)
    table = [(r.q, r.consumer_warps, r.ms) for r in res[:min(nres.value, 32)]]
    return int(q.value), int(cw.value), float(ms.value), table


def autotune_batched(Xs, *, precision: int = 0, tune_cache=None, center: bool = True,
                     stream=None, **plan):
    """The batched counterpart of autotune (one common q for the batch)."""
    if not Xs:
        raise ValueError("empty batch")
    dev = Xs[0].device
    B, ns, ms_ = _batch_arrays(Xs)
    offs, total = batch_offsets(Xs)
    o = _opts(precision, 0, center, False, _stream_handle(stream, dev), None, tune_cache=tune_cache,
              **plan)
    b = ctypes.c_size_t(0)
    rc = load().givensbn_autotune_batched_workspace_size(ctypes.cast(ns, ctypes.c_void_p),
                                                         ctypes.cast(ms_, ctypes.c_void_p), B,
                                                         ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    ws = torch.empty(int(b.value), dtype=torch.uint8, device=dev)
    o.workspace, o.workspace_bytes = ws.data_ptr(), int(b.value)
    out = torch.empty(total, dtype=torch.float64 if precision else torch.float32, device=dev)
    ptrs = (ctypes.c_void_p * B)(*[X.data_ptr() for X in Xs])
    offa = (ctypes.c_int64 * B)(*offs)
    q, cw, t, nres = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0), ctypes.c_int32(0)
    res = (TuneResult * 32)()
    rc = load().givensbn_autotune_batched(ctypes.cast(ptrs, ctypes.c_void_p),
                                          ctypes.cast(ns, ctypes.c_void_p),
                                          ctypes.cast(ms_, ctypes.c_void_p), B,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.cast(offa, ctypes.c_void_p), ctypes.byref(o),
                                          ctypes.byref(q), ctypes.byref(cw), ctypes.byref(t), res,
                                          32, ctypes.byref(nres))
    if rc:
        raise GivensBNError(rc)
    table = [(r.q, r.consumer_warps, r.ms) for r in res[:min(nres.value, 32)]]
    return int(q.value), int(cw.value), float(t.value), table


def family_coefficients(X: torch.Tensor, child, parents, *, center: bool = True,
                        stream=None, check: bool = True):
    """Least-squares coefficients of listed families (child[i] on the parent bitmask parents[i]).

    Returns (beta, rss): beta is count x (m + 1) float64 (b_v at column v for v in the
    parent set, 0 elsewhere, the intercept in column m), rss the residual sums of squares.
    """
    X = _check_x(X)
    n, m = X.shape
    dev = X.device
    child = torch.as_tensor(child, dtype=torch.int32).to(dev).contiguous()
    parents = torch.as_tensor(parents, dtype=torch.int64).to(dev).contiguous()  # uint64 bit patterns
    count = int(child.numel())
    if parents.numel() != count:
        raise ValueError("child and parents must have the same length")
    beta = torch.empty((count, m + 1), dtype=torch.float64, device=dev)
    rss = torch.empty(count, dtype=torch.float64, device=dev)
    o = _opts(0, 0, center, False, _stream_handle(stream, dev))
    b = ctypes.c_size_t(0)
    rc = load().givensbn_coefficients_workspace_size(n, m, ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    ws = torch.empty(int(b.value), dtype=torch.uint8, device=dev)
    o.workspace, o.workspace_bytes = ws.data_ptr(), int(b.value)
    rc = load().givensbn_family_coefficients(ctypes.c_void_p(X.data_ptr()), n, m,
                                             ctypes.c_void_p(child.data_ptr()),
                                             ctypes.c_void_p(parents.data_ptr()), count,
                                             ctypes.c_void_p(beta.data_ptr()),
                                             ctypes.c_void_p(rss.data_ptr()), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    if check:
        st = ctypes.c_int32(0)
        rc = load().givensbn_status(ctypes.byref(o), ctypes.byref(st))
        if rc:
            raise GivensBNError(rc)
        if st.value & GBN_STATUS_BAD_FAMILY:
            raise ValueError("givensbn: invalid family in the list (child out of range or parent "
                             "mask holding the child or variables >= m)")
        if st.value & GBN_STATUS_RANK_DEFICIENT:
            warnings.warn("givensbn: linearly dependent parent columns; their coefficients are NaN")
    return beta, rss


def _table_m(scores: torch.Tensor) -> int:
    if not (isinstance(scores, torch.Tensor) and scores.is_cuda and scores.dtype == torch.float32
            and scores.dim() == 1 and scores.is_contiguous()):
        raise TypeError("scores must be a contiguous 1-D float32 CUDA tensor in table layout")
    for m in range(2, 31):
        if m << (m - 1) == scores.numel():
            return m
    raise ValueError("scores must hold m * 2^(m-1) entries")


def best_parents(scores: torch.Tensor, *, stream=None):
    """(best, best_set): per child and candidate set U, the lowest score over the subsets of U
    and that subset's compressed mask (givensbn_best_parents)."""
    m = _table_m(scores)
    best = torch.empty_like(scores)
    bset = torch.empty(scores.numel(), dtype=torch.int32, device=scores.device)
    o = _opts(stream=_stream_handle(stream, scores.device))
    rc = load().givensbn_best_parents(ctypes.c_void_p(scores.data_ptr()), m,
                                      ctypes.c_void_p(best.data_ptr()),
                                      ctypes.c_void_p(bset.data_ptr()), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    return best, bset


def structure_search(scores: torch.Tensor, *, stream=None, workspace=None):
    """Exact structure search over a score table (lower is better): returns (parents, order,
    total), the parent bitmask of each variable in an optimal DAG, an optimal ordering and the
    network's score (givensbn_structure_search)."""
    m = _table_m(scores)
    dev = scores.device
    b = ctypes.c_size_t(0)
    rc = load().givensbn_structure_search_workspace_size(m, ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    if workspace is None:
        workspace = torch.empty(int(b.value), dtype=torch.uint8, device=dev)
    o = _opts(stream=_stream_handle(stream, dev), workspace=workspace)
    parents = torch.empty(m, dtype=torch.int32, device=dev)
    order = torch.empty(m, dtype=torch.int32, device=dev)
    total = torch.empty(1, dtype=torch.float64, device=dev)
    rc = load().givensbn_structure_search(ctypes.c_void_p(scores.data_ptr()), m,
                                          ctypes.c_void_p(parents.data_ptr()),
                                          ctypes.c_void_p(order.data_ptr()),
                                          ctypes.c_void_p(total.data_ptr()), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    return ([int(x) & 0xffffffff for x in parents.cpu().tolist()], order.cpu().tolist(),
            float(total.item()))


def pipe_peaks(device=None, stream=None):
    """Measured FP32 and FP64 FMA throughput of the device, TFLOP/s (givensbn_pipe_peaks)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    scratch = torch.empty(1, dtype=torch.float64, device=dev)
    f32, f64 = ctypes.c_double(0), ctypes.c_double(0)
    rc = load().givensbn_pipe_peaks(ctypes.c_void_p(scratch.data_ptr()), _stream_handle(stream, dev),
                                    ctypes.byref(f32), ctypes.byref(f64))
    if rc:
        raise GivensBNError(rc)
    return float(f32.value), float(f64.value)


def dmma_peak(device=None, stream=None):
    """Measured FP64 tensor-core (mma.sync m8n8k4 f64) throughput, TFLOP/s (givensbn_dmma_peak)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    scratch = torch.empty(1, dtype=torch.float64, device=dev)
    t = ctypes.c_double(0)
    rc = load().givensbn_dmma_peak(ctypes.c_void_p(scratch.data_ptr()), _stream_handle(stream, dev),
                                   ctypes.byref(t))
    if rc:
        raise GivensBNError(rc)
    return float(t.value)


def backward_batched_workspace_size(Xs, precision: int = 0, q: int = 0) -> int:
    B, ns, ms = _batch_arrays(Xs)
    o = _opts(precision, q)
    b = ctypes.c_size_t(0)
    rc = load().givensbn_backward_batched_workspace_size(ctypes.cast(ns, ctypes.c_void_p),
                                                         ctypes.cast(ms, ctypes.c_void_p), B,
                                                         ctypes.byref(o), ctypes.byref(b))
    if rc:
        raise GivensBNError(rc)
    return int(b.value)


def score_all_families_backward_batched(Xs, ws, *, precision: int = 0, q: int = 0,
                                        center: bool = True, workspace=None, stream=None,
                                        grads=None):
    """Gradients of sum_f w_f * score_f for every dataset of a batch (one list of n x m float64
    tensors); ws: one weight tensor per dataset, or one tensor shared by all (same m)."""
    if not Xs:
        raise ValueError("empty batch")
    dev = Xs[0].device
    for X in Xs:
        if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float64
                and X.dim() == 2 and X.is_contiguous() and X.device == dev):
            raise TypeError("every X must be a contiguous 2-D float64 CUDA tensor on one device")
    wdt = torch.float64 if precision else torch.float32
    if isinstance(ws, torch.Tensor):
        ws = [ws] * len(Xs)
    ws = [w.to(device=dev, dtype=wdt).contiguous() for w in ws]
    for X, w in zip(Xs, ws):
        m = int(X.shape[1])
        if w.numel() != m << (m - 1):
            raise ValueError("each weight tensor must hold m * 2^(m-1) entries")
    if grads is None:
        grads = [torch.empty_like(X) for X in Xs]
    B, ns, ms = _batch_arrays(Xs)
    if workspace is None:
        workspace = torch.empty(backward_batched_workspace_size(Xs, precision, q),
                                dtype=torch.uint8, device=dev)
    xp = (ctypes.c_void_p * B)(*[X.data_ptr() for X in Xs])
    wp = (ctypes.c_void_p * B)(*[w.data_ptr() for w in ws])
    gp = (ctypes.c_void_p * B)(*[g.data_ptr() for g in grads])
    o = _opts(precision, q, center, False, _stream_handle(stream, dev), workspace)
    rc = load().score_all_families_backward_batched(ctypes.cast(xp, ctypes.c_void_p),
                                                    ctypes.cast(ns, ctypes.c_void_p),
                                                    ctypes.cast(ms, ctypes.c_void_p), B,
                                                    ctypes.cast(wp, ctypes.c_void_p),
                                                    ctypes.cast(gp, ctypes.c_void_p),
                                                    ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    return grads
