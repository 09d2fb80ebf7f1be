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
    ]


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
          workspace=None, stage_events=None, fixup_tau=None) -> Opts:
    o = Opts()
    load().givensbn_default_opts(ctypes.byref(o))
    if fixup_tau is not None:
        o.fixup_tau = float(fixup_tau)
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


def workspace_size(n: int, m: int, precision: int = 0, q: int = 0, fixup_tau=None) -> int:
    o = _opts(precision, q, fixup_tau=fixup_tau)
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


def score_all_families(X: torch.Tensor, out: torch.Tensor | None = None, *, precision: int = 0,
                       q: int = 0, center: bool = True, debug_coverage: bool = False,
                       workspace: torch.Tensor | None = None, stream=None,
                       stage_events=None, check: bool = True, fixup_tau=None) -> torch.Tensor:
    """Scores of all m * 2^(m-1) families of the n x m data X (CUDA float64, row-major).

    Returns a 1-D tensor in table layout (float32 for precision 0, float64 for
    precision 1, int32 counters for debug_coverage).  `out` may be a pinned host
    tensor: the kernels then write the table straight into host memory.  check=True synchronises
    and warns if the data were rank deficient.  stage_events: four
    torch.cuda.Event(enable_timing=True) recorded at the stage boundaries.
    """
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
        workspace = torch.empty(workspace_size(n, m, precision, q, fixup_tau), dtype=torch.uint8,
                                device=dev)
    if stage_events is not None:
        for e in stage_events:  # torch creates the CUDA event on its first record()
            if not e.cuda_event:
                e.record(stream if stream is not None else torch.cuda.current_stream(dev))
    o = _opts(precision, q, center, debug_coverage, _stream_handle(stream, dev), workspace,
              stage_events, fixup_tau)
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


def batched_workspace_size(Xs, precision: int = 0, q: int = 0) -> int:
    B, ns, ms = _batch_arrays(Xs)
    o = _opts(precision, q)
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
                               workspace: torch.Tensor | None = None, stream=None):
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
        workspace = torch.empty(batched_workspace_size(Xs, precision, q), dtype=torch.uint8,
                                device=dev)
    ptrs = (ctypes.c_void_p * B)(*[X.data_ptr() for X in Xs])
    offa = (ctypes.c_int64 * B)(*offs)
    o = _opts(precision, q, center, debug_coverage, _stream_handle(stream, dev), workspace)
    rc = load().score_all_families_batched(ctypes.cast(ptrs, ctypes.c_void_p),
                                           ctypes.cast(ns, ctypes.c_void_p),
                                           ctypes.cast(ms, ctypes.c_void_p), B,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.cast(offa, ctypes.c_void_p), ctypes.byref(o))
    if rc:
        raise GivensBNError(rc)
    return out, offs
