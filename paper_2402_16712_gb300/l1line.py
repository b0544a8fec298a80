"""Python binding of the C ABI in ``include/l1line.h`` (argument marshalling only).

Every step of the path runs in the CUDA library ``libl1line.so``; PyTorch only
supplies device memory (``tensor.data_ptr()``) and streams.  There is no CPU
fallback: if the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# L1LINE_LIB selects another build of the same library (the bounds-checked
# libl1line_checks.so)
LIB_PATH = os.environ.get("L1LINE_LIB") or os.path.join(_HERE, "libl1line.so")

OK, ERR_ARG, ERR_NONFINITE, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_INTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7)
DTYPE_F32, DTYPE_F64 = 0, 1
FLAG_FORCE_EXACT = 1

# Exported symbols and their ctypes signatures (mirrors include/l1line.h).
_P, _I64, _U32, _SZ, _I = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t,
                           ctypes.c_int)
SIGNATURES = {
    "l1line_max_rows": (_I64, [_I]),
    "l1line_workspace_bytes": (_SZ, [_I, _I64, _I64, _I64]),
    "l1line_scan_f32": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_scan_f64": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_scan_ex_f32": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P, _U32]),
    "l1line_scan_ex_f64": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P, _U32]),
    "l1line_fit_f32": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_fit_f64": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_status": (_I, [_P, _P]),
    "l1line_status_string": (ctypes.c_char_p, [_I]),
    "l1line_last_launch_count": (_I, []),
    "l1line_check_hits": (_I64, [_I, _P]),
    "l1line_profile_events": (_I, [_P, _P]),
    "l1line_path_max_rows": (_I64, [_I]),
    "l1line_probe": (_I, [_I, _P, _SZ, _I, _P, _P, _P]),
    "l1line_fit_noalloc_f32": (_I, [_P, _I64, _I64, _P, _I64, _P, _P, _P, _P]),
    "l1line_noalloc_status": (_I, [_P]),
    "l1line_batched_workspace_bytes": (_SZ, [_I, _I64, _P, _P, _P]),
    "l1line_fit_batched_f32": (_I, [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "l1line_fit_batched_f64": (_I, [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "l1line_fit_subset_f32": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_fit_subset_f64": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_proposer_rows": (_I64, [_I64]),
    "l1line_proposed_workspace_bytes": (_SZ, [_I, _I64, _I64, _I64]),
    "l1line_features_f32": (_I, [_P, _I64, _I64, ctypes.c_double, _P, _P, _P, _SZ, _P]),
    "l1line_features_f64": (_I, [_P, _I64, _I64, ctypes.c_double, _P, _P, _P, _SZ, _P]),
    "l1line_mlp_forward": (_I, [_P, _P, _I64, _P, _P, _P]),
    "l1line_mlp_workspace_bytes": (_SZ, [_I64]),
    "l1line_mlp_backward": (_I, [_P, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1line_rank_loss": (_I, [_P, _P, _P, _P, _I64, _P, _P, _P]),
    "l1line_adam_step": (_I, [_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, ctypes.c_float, _P, _P]),
    "l1line_mlp_pack": (_I, [_P, _P, _P]),
    "l1line_topk": (_I, [_P, _I64, _I64, _P, _P]),
    "l1line_fit_proposed_f32": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _P, _P, _P, _P,
                                     _SZ, _P]),
    "l1line_fit_proposed_f64": (_I, [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _P, _P, _P, _P,
                                     _SZ, _P]),
    "l1line_path_workspace_bytes": (_SZ, [_I, _I64, _I64]),
    "l1line_path_count_f32": (_I, [_P, _I64, _I64, _P, _P, _SZ, _P]),
    "l1line_path_count_f64": (_I, [_P, _I64, _I64, _P, _P, _SZ, _P]),
    "l1line_path_write_f32": (_I, [_P, _I64, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "l1line_path_write_f64": (_I, [_P, _I64, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "l1line_solution_path_workspace_bytes": (_SZ, [_I64, _I64]),
    "l1line_solution_path_f32": (_I, [_I64, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _P, _P,
                                      _I64, _P, _SZ, _P]),
    "l1line_solution_path_f64": (_I, [_I64, _P, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _P, _P,
                                      _I64, _P, _SZ, _P]),
    "l1line_components_workspace_bytes": (_SZ, [_I, _I64, _I64]),
    "l1line_components_f32": (_I, [_P, _I64, _I64, ctypes.c_double, _I64, _P, _P, _P, _P, _SZ,
                                   _P]),
    "l1line_components_f64": (_I, [_P, _I64, _I64, ctypes.c_double, _I64, _P, _P, _P, _P, _SZ,
                                   _P]),
    "l1line_set_tuning": (_I, [_P]),
    "l1line_plan": (_I, [_I, _I64, _I64, _I64, _P]),
    "l1line_plan_for": (_I, [_I, _I64, _I64, _I64, _I, _P]),
}
MLP_FEATURES = 4     # L1L_MLP_FEATURES
MLP_PARAMS = 17281   # L1L_MLP_PARAMS
MLP_BYTES = 35088    # sizeof(l1line_mlp)
NOALLOC_SCRATCH_BYTES = 32 << 20  # L1L_NOALLOC_SCRATCH_BYTES in include/l1line.h

_lib = None


class L1LineError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code) if _lib else code} ({code})")


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with `python -c \"import __graft_entry__ as g; "
                f"g.build()\"` (there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def status_string(code: int) -> str:
    return load().l1line_status_string(int(code)).decode()


def max_rows(dtype) -> int:
    return int(load().l1line_max_rows(_dt(dtype)))


def workspace_bytes(dtype, n: int, m: int, n_lambda: int) -> int:
    return int(load().l1line_workspace_bytes(_dt(dtype), n, m, n_lambda))


def last_launch_count() -> int:
    return int(load().l1line_last_launch_count())


def check_hits(reset: bool = False):
    """(hits, source line of the last) of the bounds-checked build; hits is -1
    in the normal build."""
    line = ctypes.c_int(0)
    h = int(load().l1line_check_hits(1 if reset else 0, ctypes.byref(line)))
    return h, line.value


def _dt(dtype) -> int:
    import torch
    if dtype in (torch.float32, np.float32, "float32", DTYPE_F32):
        return DTYPE_F32
    if dtype in (torch.float64, np.float64, "float64", DTYPE_F64):
        return DTYPE_F64
    raise TypeError(f"unsupported dtype {dtype}")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_x(X):
    import torch
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise TypeError("X must be a CUDA tensor")
    if X.dtype not in (torch.float32, torch.float64) or X.dim() != 2 or not X.is_contiguous():
        raise TypeError("X must be a contiguous 2-D float32/float64 CUDA tensor")


def _lams(lambdas) -> np.ndarray:
    return np.ascontiguousarray(np.atleast_1d(np.asarray(lambdas, dtype=np.float64)))


class Workspace:
    """Caller-owned device workspace (a torch uint8 buffer, 256-byte aligned)."""

    def __init__(self, nbytes: int, device=None):
        import torch
        self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buf.data_ptr()
        self.ptr = (base + 255) & ~255
        self.nbytes = nbytes

    @classmethod
    def for_shape(cls, dtype, n, m, n_lambda, device=None):
        nb = workspace_bytes(dtype, n, m, n_lambda)
        if nb == 0:
            raise ValueError("bad shape for the workspace")
        return cls(nb, device)


def scan(X, lambdas, workspace: Optional[Workspace] = None, stream=None, flags: int = 0,
         out=None, z_only=False):
    """A1-A5: v_all [nl, m, m], s_all [nl, m, m] (double), z_all [nl, m] (double).
    With z_only, v_all and s_all are not returned (None) and stay internal."""
    import torch
    _check_x(X)
    lam = _lams(lambdas)
    n, m = X.shape
    nl = lam.size
    ws = workspace or Workspace.for_shape(X.dtype, n, m, nl, X.device)
    if z_only:
        z_all = out if out is not None else torch.empty((nl, m), dtype=torch.float64,
                                                        device=X.device)
        f = load().l1line_scan_ex_f32 if X.dtype == torch.float32 else load().l1line_scan_ex_f64
        _check(f(X.data_ptr(), n, m, lam.ctypes.data_as(ctypes.c_void_p), nl, None, None,
                 z_all.data_ptr(), ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream), flags),
               "l1line_scan")
        return None, None, z_all, ws
    if out is None:
        v_all = torch.empty((nl, m, m), dtype=X.dtype, device=X.device)
        s_all = torch.empty((nl, m, m), dtype=torch.float64, device=X.device)
        z_all = torch.empty((nl, m), dtype=torch.float64, device=X.device)
    else:
        v_all, s_all, z_all = out
    f = load().l1line_scan_ex_f32 if X.dtype == torch.float32 else load().l1line_scan_ex_f64
    rc = f(X.data_ptr(), n, m, lam.ctypes.data_as(ctypes.c_void_p), nl, v_all.data_ptr(),
           s_all.data_ptr(), z_all.data_ptr(), ctypes.c_void_p(ws.ptr), ws.nbytes,
           _stream_ptr(stream), flags)
    if rc != OK:
        raise L1LineError(rc, "l1line_scan")
    return v_all, s_all, z_all, ws


def fit(X, lambdas, workspace: Optional[Workspace] = None, stream=None, out=None):
    """Algorithm 1 per lambda: v [nl, m], obj [nl] (double), jstar [nl] (int32)."""
    import torch
    _check_x(X)
    lam = _lams(lambdas)
    n, m = X.shape
    nl = lam.size
    ws = workspace or Workspace.for_shape(X.dtype, n, m, nl, X.device)
    if out is None:
        v = torch.empty((nl, m), dtype=X.dtype, device=X.device)
        obj = torch.empty(nl, dtype=torch.float64, device=X.device)
        js = torch.empty(nl, dtype=torch.int32, device=X.device)
    else:
        v, obj, js = out
    f = load().l1line_fit_f32 if X.dtype == torch.float32 else load().l1line_fit_f64
    rc = f(X.data_ptr(), n, m, lam.ctypes.data_as(ctypes.c_void_p), nl, v.data_ptr(),
           obj.data_ptr(), js.data_ptr(), ctypes.c_void_p(ws.ptr), ws.nbytes,
           _stream_ptr(stream))
    if rc != OK:
        raise L1LineError(rc, "l1line_fit")
    return v, obj, js, ws


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(rc, where):
    if rc != OK:
        raise L1LineError(rc, where)


def _fit_outputs(X, nl, out):
    import torch
    if out is not None:
        return out
    m = X.shape[1]
    return (torch.empty((nl, m), dtype=X.dtype, device=X.device),
            torch.empty(nl, dtype=torch.float64, device=X.device),
            torch.empty(nl, dtype=torch.int32, device=X.device))


def fit_subset(X, lambdas, jhat, workspace: Optional[Workspace] = None, stream=None, out=None):
    """Algorithm 1 over the candidate jhat in `jhat` (int32 CUDA tensor) only:
    v [nl, m], obj [nl], jstar [nl]."""
    import torch
    _check_x(X)
    if jhat.dtype != torch.int32 or not jhat.is_cuda or jhat.dim() != 1:
        raise TypeError("jhat must be a 1-D int32 CUDA tensor")
    lam = _lams(lambdas)
    n, m = X.shape
    ws = workspace or Workspace.for_shape(X.dtype, n, m, lam.size, X.device)
    v, obj, js = _fit_outputs(X, lam.size, out)
    f = load().l1line_fit_subset_f32 if X.dtype == torch.float32 else load().l1line_fit_subset_f64
    _check(f(X.data_ptr(), n, m, lam.ctypes.data_as(ctypes.c_void_p), lam.size, _ptr(jhat),
             jhat.numel(), v.data_ptr(), obj.data_ptr(), js.data_ptr(), ctypes.c_void_p(ws.ptr),
             ws.nbytes, _stream_ptr(stream)), "l1line_fit_subset")
    return v, obj, js, ws


def proposer_rows(n: int) -> int:
    return int(load().l1line_proposer_rows(n))


def proposed_workspace(dtype, n: int, m: int, n_lambda: int = 1, device=None) -> "Workspace":
    """Workspace of the proposer calls (features, fit_proposed)."""
    nb = int(load().l1line_proposed_workspace_bytes(_dt(dtype), n, m, n_lambda))
    if nb == 0:
        raise ValueError("bad shape for the proposer workspace")
    return Workspace(nb, device)


def features(X, lam: float, workspace: Optional[Workspace] = None, stream=None, raw=True):
    """The proposer's features of every column of X (the restricted objective
    at penalty lam): (raw [m, 4] or None, standardised [m, 4]) float32."""
    import torch
    _check_x(X)
    n, m = X.shape
    ws = workspace or proposed_workspace(X.dtype, n, m, 1, X.device)
    r = torch.empty((m, MLP_FEATURES), dtype=torch.float32, device=X.device) if raw else None
    z = torch.empty((m, MLP_FEATURES), dtype=torch.float32, device=X.device)
    f = load().l1line_features_f32 if X.dtype == torch.float32 else load().l1line_features_f64
    _check(f(X.data_ptr(), n, m, float(lam), _ptr(r), _ptr(z), ctypes.c_void_p(ws.ptr),
             ws.nbytes, _stream_ptr(stream)), "l1line_features")
    return r, z


def mlp_pack(theta, mlp=None, stream=None):
    """Network image (uint8 CUDA tensor of MLP_BYTES) from flat float32 params."""
    import torch
    if mlp is None:
        mlp = torch.empty(MLP_BYTES, dtype=torch.uint8, device=theta.device)
    _check(load().l1line_mlp_pack(_ptr(theta), _ptr(mlp), _stream_ptr(stream)), "l1line_mlp_pack")
    return mlp


def mlp_forward(feat, mlp, rows=None, n=None, out=None, stream=None):
    import torch
    N = int(rows.numel() if rows is not None else (feat.shape[0] if n is None else n))
    s = out if out is not None else torch.empty(N, dtype=torch.float32, device=feat.device)
    _check(load().l1line_mlp_forward(_ptr(feat), _ptr(rows), N, _ptr(mlp), _ptr(s),
                                     _stream_ptr(stream)), "l1line_mlp_forward")
    return s


class MlpWorkspace:
    def __init__(self, N, device=None):
        nb = int(load().l1line_mlp_workspace_bytes(int(N)))
        if nb == 0:
            raise ValueError("bad sample count")
        self.ws = Workspace(nb, device)


def mlp_backward(feat, mlp, dscores, rows=None, grad=None, workspace=None, stream=None):
    import torch
    N = int(dscores.numel())
    g = grad if grad is not None else torch.empty(MLP_PARAMS, dtype=torch.float32,
                                                  device=feat.device)
    ws = (workspace or MlpWorkspace(N, feat.device)).ws
    _check(load().l1line_mlp_backward(_ptr(feat), _ptr(rows), N, _ptr(mlp), _ptr(dscores),
                                      _ptr(g), ctypes.c_void_p(ws.ptr), ws.nbytes,
                                      _stream_ptr(stream)), "l1line_mlp_backward")
    return g


def rank_loss(scores, targets, offsets, rows=None, dscores=None, loss=None, stream=None):
    import torch
    nb = int(offsets.numel()) - 1
    ds = dscores if dscores is not None else torch.empty_like(scores)
    lo = loss if loss is not None else torch.empty(nb, dtype=torch.float32, device=scores.device)
    _check(load().l1line_rank_loss(_ptr(scores), _ptr(targets), _ptr(rows), _ptr(offsets), nb,
                                   _ptr(ds), _ptr(lo), _stream_ptr(stream)), "l1line_rank_loss")
    return lo, ds


def adam_step(theta, grad, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, mlp=None,
              stream=None):
    _check(load().l1line_adam_step(_ptr(theta), _ptr(grad), _ptr(m1), _ptr(m2), int(step),
                                   float(lr), float(beta1), float(beta2), float(eps), _ptr(mlp),
                                   _stream_ptr(stream)), "l1line_adam_step")


def topk(scores, K, out=None, stream=None):
    import torch
    o = out if out is not None else torch.empty(int(K), dtype=torch.int32, device=scores.device)
    _check(load().l1line_topk(_ptr(scores), scores.numel(), int(K), _ptr(o), _stream_ptr(stream)),
           "l1line_topk")
    return o


def fit_proposed(X, lambdas, mlp, K, workspace: Optional[Workspace] = None, stream=None,
                 out=None, idx=None):
    """The learned path: features, network, top-K, exact fit of the K
    candidates.  Returns v, obj, jstar, candidate indices, workspace."""
    import torch
    _check_x(X)
    lam = _lams(lambdas)
    n, m = X.shape
    ws = workspace or proposed_workspace(X.dtype, n, m, lam.size, X.device)
    v, obj, js = _fit_outputs(X, lam.size, out)
    if idx is None:
        idx = torch.empty(int(K), dtype=torch.int32, device=X.device)
    f = (load().l1line_fit_proposed_f32 if X.dtype == torch.float32
         else load().l1line_fit_proposed_f64)
    _check(f(X.data_ptr(), n, m, lam.ctypes.data_as(ctypes.c_void_p), lam.size, _ptr(mlp), int(K),
             _ptr(idx), v.data_ptr(), obj.data_ptr(), js.data_ptr(), ctypes.c_void_p(ws.ptr),
             ws.nbytes, _stream_ptr(stream)), "l1line_fit_proposed")
    return v, obj, js, idx, ws


def path_workspace(dtype, n: int, m: int, device=None) -> "Workspace":
    nb = int(load().l1line_path_workspace_bytes(_dt(dtype), n, m))
    if nb == 0:
        raise ValueError("bad shape for the path workspace")
    return Workspace(nb, device)


def paths(X, workspace: Optional[Workspace] = None, stream=None, residuals=False):
    """Algorithm 2 for every (jhat, k): returns (offsets [m*m + 1] int64 CUDA,
    lam double CUDA, v CUDA (X's dtype), length [m*m] int32 CUDA, workspace),
    and with residuals=True also the residual of every entry (double CUDA) as
    a sixth item.  Pair p = jhat * m + k owns entries offsets[p] ..
    offsets[p] + length[p].  Reads the entry count back to the host between
    the two library calls."""
    import torch
    _check_x(X)
    n, m = X.shape
    ws = workspace or path_workspace(X.dtype, n, m, X.device)
    off = torch.empty(m * m + 1, dtype=torch.int64, device=X.device)
    f32 = X.dtype == torch.float32
    cnt = load().l1line_path_count_f32 if f32 else load().l1line_path_count_f64
    _check(cnt(X.data_ptr(), n, m, off.data_ptr(), ctypes.c_void_p(ws.ptr), ws.nbytes,
               _stream_ptr(stream)), "l1line_path_count")
    total = int(off[m * m].item())  # synchronises the stream
    lam = torch.empty(max(total, 1), dtype=torch.float64, device=X.device)
    v = torch.empty(max(total, 1), dtype=X.dtype, device=X.device)
    ln = torch.empty(m * m, dtype=torch.int32, device=X.device)
    res = torch.empty(max(total, 1), dtype=torch.float64, device=X.device) if residuals else None
    wr = load().l1line_path_write_f32 if f32 else load().l1line_path_write_f64
    _check(wr(X.data_ptr(), n, m, off.data_ptr(), lam.data_ptr(), v.data_ptr(), _ptr(res),
              ln.data_ptr(), ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream)),
           "l1line_path_write")
    if residuals:
        return off, lam, v, ln, ws, res
    return off, lam, v, ln, ws


def solution_path(X, cap: int = 4096, stream=None):
    """Algorithms 2 and 3: the solution path of X over all lambda >= 0.
    Returns (start, jhat, intercept, slope, v) CPU tensors of the pieces:
    from start[e] on, jhat* = jhat[e], z* = intercept[e] + slope[e] lambda and
    v* = v[e] (on the open interval after the start)."""
    import torch
    _check_x(X)
    n, m = X.shape
    off, lam, v, ln, pws, res = paths(X, stream=stream, residuals=True)
    entries = int(off[m * m].item())
    nb = int(load().l1line_solution_path_workspace_bytes(m, entries))
    if nb == 0:
        raise L1LineError(ERR_UNSUPPORTED, "l1line_solution_path_workspace_bytes")
    ws = Workspace(nb, X.device)
    dev = X.device
    start = torch.empty(cap, dtype=torch.float64, device=dev)
    jh = torch.empty(cap, dtype=torch.int32, device=dev)
    I = torch.empty(cap, dtype=torch.float64, device=dev)
    S = torch.empty(cap, dtype=torch.float64, device=dev)
    vs = torch.empty((cap, m), dtype=X.dtype, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    f = (load().l1line_solution_path_f32 if X.dtype == torch.float32
         else load().l1line_solution_path_f64)
    _check(f(m, off.data_ptr(), lam.data_ptr(), v.data_ptr(), res.data_ptr(), ln.data_ptr(),
             entries, start.data_ptr(), jh.data_ptr(), I.data_ptr(), S.data_ptr(), vs.data_ptr(),
             count.data_ptr(), cap, ctypes.c_void_p(ws.ptr), ws.nbytes, _stream_ptr(stream)),
           "l1line_solution_path")
    c = int(count.item())
    if c > cap:
        return solution_path(X, cap=c, stream=stream)
    return start[:c].cpu(), jh[:c].cpu(), I[:c].cpu(), S[:c].cpu(), vs[:c].cpu()


def components(X, lam: float, ncomp: int, workspace: Optional[Workspace] = None, stream=None):
    """ncomp successive components at one lambda: v [ncomp, m], obj [ncomp],
    jstar [ncomp] (CUDA), workspace."""
    import torch
    _check_x(X)
    n, m = X.shape
    if workspace is None:
        nb = int(load().l1line_components_workspace_bytes(_dt(X.dtype), n, m))
        if nb == 0:
            raise ValueError("bad shape for the components workspace")
        workspace = Workspace(nb, X.device)
    v = torch.empty((ncomp, m), dtype=X.dtype, device=X.device)
    obj = torch.empty(ncomp, dtype=torch.float64, device=X.device)
    js = torch.empty(ncomp, dtype=torch.int32, device=X.device)
    f = load().l1line_components_f32 if X.dtype == torch.float32 else load().l1line_components_f64
    _check(f(X.data_ptr(), n, m, float(lam), int(ncomp), v.data_ptr(), obj.data_ptr(),
             js.data_ptr(), ctypes.c_void_p(workspace.ptr), workspace.nbytes, _stream_ptr(stream)),
           "l1line_components")
    return v, obj, js, workspace


class Tuning(ctypes.Structure):
    """l1line_tuning: pair-kernel launch overrides (0 = the planner's choice)."""
    _fields_ = [("warps", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("kchunk", ctypes.c_int32), ("d0", ctypes.c_int32),
                ("batch_classes", ctypes.c_int32), ("column", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def set_tuning(tuning=None) -> None:
    """Apply a tuning (dict or Tuning) to this thread's later calls; None
    restores the planner."""
    if tuning is None:
        _check(load().l1line_set_tuning(None), "l1line_set_tuning")
        return
    t = tuning if isinstance(tuning, Tuning) else Tuning(**tuning)
    _check(load().l1line_set_tuning(ctypes.byref(t)), "l1line_set_tuning")


def plan(dtype, n: int, m: int, nj: Optional[int] = None) -> dict:
    """The pair-kernel plan the next call of this thread would use."""
    t = Tuning()
    _check(load().l1line_plan(_dt(dtype), n, m, m if nj is None else nj, ctypes.byref(t)),
           "l1line_plan")
    return t.as_dict()


def plan_for(dtype, n: int, m: int, sms: int, nj: Optional[int] = None) -> dict:
    """The plan for a GPU of `sms` SMs, computed on the host (no device)."""
    t = Tuning()
    _check(load().l1line_plan_for(_dt(dtype), n, m, m if nj is None else nj, sms,
                                  ctypes.byref(t)), "l1line_plan_for")
    return t.as_dict()


def status(ws: Workspace, stream=None) -> int:
    """Synchronise and return the device-side status of the last call on ws."""
    return int(load().l1line_status(ctypes.c_void_p(ws.ptr), _stream_ptr(stream)))


def profile_events(start=None, stop=None) -> None:
    """Have later calls record torch.cuda.Event `start`/`stop` around the pair
    kernel (steps A2-A4) on their stream; call with no arguments to stop."""
    if start is None or stop is None:
        load().l1line_profile_events(None, None)
    else:
        load().l1line_profile_events(ctypes.c_void_p(start.cuda_event),
                                     ctypes.c_void_p(stop.cuda_event))


PROBE_L2, PROBE_SMEM = 0, 1


def probe_bandwidth(kind: int, reps: int, buf=None, stream=None) -> float:
    """Run one bandwidth probe (`l1line_probe`) on `stream` and return bytes/s
    from CUDA events around it.  kind PROBE_L2 reads the device tensor `buf`
    `reps` times; PROBE_SMEM ignores `buf`."""
    import torch
    st = stream or torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.int32, device=st.device)
    nbytes = ctypes.c_double(0.0)
    ptr = ctypes.c_void_p(buf.data_ptr()) if buf is not None else None
    size = buf.numel() * buf.element_size() if buf is not None else 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    _check(load().l1line_probe(kind, ptr, size, reps, ctypes.c_void_p(sink.data_ptr()),
                               ctypes.c_void_p(st.cuda_stream), ctypes.byref(nbytes)),
           "l1line_probe")
    b.record(st)
    b.synchronize()
    return nbytes.value / (a.elapsed_time(b) * 1e-3)


class Batched:
    """A batch of independent fits (`l1line_fit_batched_*`), set up once and run
    any number of times (e.g. inside a torch.cuda.CUDAGraph capture after one
    warm-up run).  Xs: list of contiguous CUDA tensors (same dtype), lambdas:
    list of 1-D sequences, one per instance."""

    def __init__(self, Xs, lambdas, device=None):
        import torch
        if len(Xs) != len(lambdas) or not Xs:
            raise ValueError("one lambda list per instance")
        for X in Xs:
            _check_x(X)
        self.dtype = Xs[0].dtype
        if any(X.dtype != self.dtype for X in Xs):
            raise TypeError("all instances must share a dtype")
        device = device or Xs[0].device
        self.Xs = list(Xs)
        self.ns = np.array([X.shape[0] for X in Xs], dtype=np.int64)
        self.ms = np.array([X.shape[1] for X in Xs], dtype=np.int64)
        lams = [_lams(l) for l in lambdas]
        self.nl = np.array([l.size for l in lams], dtype=np.int64)
        self.loff = np.concatenate([[0], np.cumsum(self.nl)]).astype(np.int64)
        self.lam = np.ascontiguousarray(np.concatenate(lams), dtype=np.float64)
        self.xptr = np.array([X.data_ptr() for X in Xs], dtype=np.uint64)
        nb = int(load().l1line_batched_workspace_bytes(
            _dt(self.dtype), len(Xs), self.ns.ctypes.data_as(ctypes.c_void_p),
            self.ms.ctypes.data_as(ctypes.c_void_p), self.loff.ctypes.data_as(ctypes.c_void_p)))
        if nb == 0:
            raise L1LineError(ERR_UNSUPPORTED, "l1line_batched_workspace_bytes")
        self.ws = Workspace(nb, device)
        vlen = int((self.nl * self.ms).sum())
        self.out_v = torch.empty(vlen, dtype=self.dtype, device=device)
        self.out_obj = torch.empty(int(self.nl.sum()), dtype=torch.float64, device=device)
        self.out_jstar = torch.empty(int(self.nl.sum()), dtype=torch.int32, device=device)

    def run(self, stream=None):
        import torch
        f = (load().l1line_fit_batched_f32 if self.dtype == torch.float32
             else load().l1line_fit_batched_f64)
        P = ctypes.c_void_p
        rc = f(len(self.Xs), self.xptr.ctypes.data_as(P), self.ns.ctypes.data_as(P),
               self.ms.ctypes.data_as(P), self.lam.ctypes.data_as(P), self.loff.ctypes.data_as(P),
               self.out_v.data_ptr(), self.out_obj.data_ptr(), self.out_jstar.data_ptr(),
               P(self.ws.ptr), self.ws.nbytes, _stream_ptr(stream))
        if rc != OK:
            raise L1LineError(rc, "l1line_fit_batched")

    def results(self):
        """Per instance: (v [nl, m], obj [nl], jstar [nl]) views of the outputs."""
        out, vo = [], 0
        for b in range(len(self.Xs)):
            nl, m, t0 = int(self.nl[b]), int(self.ms[b]), int(self.loff[b])
            out.append((self.out_v[vo:vo + nl * m].view(nl, m), self.out_obj[t0:t0 + nl],
                        self.out_jstar[t0:t0 + nl]))
            vo += nl * m
        return out

    def status(self, stream=None) -> int:
        return status(self.ws, stream)
