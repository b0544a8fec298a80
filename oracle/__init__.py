"""CPU oracle for the l1-regularised l1 best-fit line (Ling & Brooks, arXiv 2402.16712).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()``, and the
CPU-baseline leg and ``--impl reference`` arm of ``bench.py`` may import this
package (``__graft_entry__.build()`` compiles it).  The product path
(the CUDA library and its binding) never touches it, and it shares no code with
that path.

The arithmetic lives in ``l1line_oracle.c`` (plain C11, exact decisions by a
long fixed-point accumulator, sort-and-scan per (jhat, k) pair as in Lemma 1 and
Algorithm 1).  This module only builds that file and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "l1line_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            for sfx in ("f64", "f32"):
                f = getattr(lib, f"oracle_fit_{sfx}")
                f.restype = ctypes.c_int
                f.argtypes = [P, I64, I64, P, I64, P, I64, P, P, P, P, P, P, ctypes.c_int]
                g = getattr(lib, f"oracle_pair_{sfx}")
                g.restype = ctypes.c_int
                g.argtypes = [P, P, I64, ctypes.c_double, P]
                h = getattr(lib, f"oracle_path_{sfx}")
                h.restype = I64
                h.argtypes = [P, I64, I64, I64, I64, P, P, I64]
            lib.oracle_sign_of_sum.restype = ctypes.c_int
            lib.oracle_sign_of_sum.argtypes = [P, I64]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def sign_of_sum(vals) -> int:
    """Exact sign (-1, 0, +1) of the real sum of the given doubles."""
    a = np.ascontiguousarray(vals, dtype=np.float64)
    return int(_load().oracle_sign_of_sum(_ptr(a), a.size))


def pair(a, b, lam: float):
    """v_k for one (jhat, k) pair: a = column k, b = column jhat (Lemma 1)."""
    a = np.ascontiguousarray(a)
    dt = a.dtype
    if dt not in (np.float32, np.float64):
        raise TypeError("float32 or float64 expected")
    b = np.ascontiguousarray(b, dtype=dt)
    out = np.zeros(1, dtype=dt)
    f = getattr(_load(), "oracle_pair_f32" if dt == np.float32 else "oracle_pair_f64")
    rc = f(_ptr(a), _ptr(b), a.size, float(lam), _ptr(out))
    if rc != 0:
        raise OracleError(f"oracle_pair failed: {rc}")
    return out[0]


def fit(X, lambdas, jlist=None, nthreads=None, want_all=True):
    """Algorithm 1 for every lambda.  X: (n, m) float32/float64, rows = points.

    Returns a dict with v (nl, m), obj (nl,), jstar (nl,) and, when want_all,
    v_all (nl, m, m), s_all (nl, m, m), z_all (nl, m) for every listed jhat.
    """
    X = np.ascontiguousarray(X)
    if X.dtype not in (np.float32, np.float64) or X.ndim != 2:
        raise TypeError("X must be a 2-D float32/float64 array")
    dt = X.dtype
    n, m = X.shape
    lam = np.ascontiguousarray(np.atleast_1d(lambdas), dtype=np.float64)
    nl = lam.size
    jl = None if jlist is None else np.ascontiguousarray(jlist, dtype=np.int32)
    nj = m if jl is None else jl.size
    out_v = np.zeros((nl, m), dtype=dt)
    out_obj = np.zeros(nl, dtype=np.float64)
    out_j = np.zeros(nl, dtype=np.int32)
    v_all = s_all = z_all = None
    if want_all:
        v_all = np.full((nl, m, m), np.nan, dtype=dt)
        s_all = np.full((nl, m, m), np.nan, dtype=np.float64)
        z_all = np.full((nl, m), np.nan, dtype=np.float64)
    if nthreads is None:
        nthreads = max_threads()
    f = getattr(_load(), "oracle_fit_f32" if dt == np.float32 else "oracle_fit_f64")
    rc = f(_ptr(X), n, m, _ptr(lam), nl, _ptr(jl), nj, _ptr(v_all), _ptr(s_all),
           _ptr(z_all), _ptr(out_v), _ptr(out_obj), _ptr(out_j), int(nthreads))
    if rc != 0:
        raise OracleError(f"oracle_fit failed: {rc}")
    res = {"v": out_v, "obj": out_obj, "jstar": out_j}
    if want_all:
        res.update(v_all=v_all, s_all=s_all, z_all=z_all)
    return res


def path(X, jhat: int, k: int):
    """The lambda path of v_k for preserved coordinate jhat (Algorithm 2):
    (lam, v) with lam increasing from 0; v[g] is the value from lam[g] on
    (see oracle_path_* for the conventions)."""
    X = np.ascontiguousarray(X)
    if X.dtype not in (np.float32, np.float64) or X.ndim != 2:
        raise TypeError("X must be a 2-D float32/float64 array")
    n, m = X.shape
    lam = np.zeros(n + 1)
    v = np.zeros(n + 1, dtype=X.dtype)
    f = getattr(_load(), "oracle_path_f32" if X.dtype == np.float32 else "oracle_path_f64")
    r = int(f(_ptr(X), n, m, int(jhat), int(k), _ptr(lam), _ptr(v), n + 1))
    if r < 1:
        raise OracleError(f"oracle_path failed: {r}")
    return lam[:r].copy(), v[:r].copy()
