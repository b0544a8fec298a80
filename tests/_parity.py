"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare it with the oracle element by element.

Bar (stated once, used by every parity test):
  * v (every v^jhat_k, every lambda): bit-identical to the oracle.
  * z_jhat: |z_gpu - z_ref| <= rtol |z_ref| + atol with rtol = 1e-5 (float32
    input) or 1e-12 (float64 input), and atol = 8 u sum_k |v_k| sum_i |x_ijhat|,
    the size of the rounding of the products v_k x_ijhat that a near-perfect
    fit (residuals far below |x|) cannot hide; u = 2^-24 or 2^-53.
  * s_jhat,k (every pair): the same bar term by term, atol = 8 u |v_k| sum_i |x_ijhat|.
  * jhat*: equal, or the two objectives tie within the z tolerance; v* is then
    the bit-exact v^jhat* of the index the GPU chose.
"""
import numpy as np
import torch

import oracle
from paper_2402_16712_gb300 import l1line


def as_bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def tolerances(X, v_all, cols=None):
    """cols: the jhat indices the last axis of v_all's leading part refers to
    (default: all of them)."""
    X = np.asarray(X)
    f32 = X.dtype == np.float32
    u = 2.0 ** -24 if f32 else 2.0 ** -53
    rtol = 1e-5 if f32 else 1e-12
    col = np.abs(X.astype(np.float64)).sum(axis=0)          # [m]
    if cols is not None:
        col = col[np.asarray(cols)]
    vab = np.abs(np.asarray(v_all, dtype=np.float64)).sum(axis=-1)  # [..., m]
    atol = 8.0 * u * vab * col
    return rtol, atol


def gpu_scan(X, lams, flags=0):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    v_all, s_all, z_all, ws = l1line.scan(Xd, lams, flags=flags)
    rc = l1line.status(ws)
    assert rc == l1line.OK, l1line.status_string(rc)
    return v_all.cpu().numpy(), s_all.cpu().numpy(), z_all.cpu().numpy()


def gpu_fit(X, lams):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    v, obj, js, ws = l1line.fit(Xd, lams)
    rc = l1line.status(ws)
    assert rc == l1line.OK, l1line.status_string(rc)
    return v.cpu().numpy(), obj.cpu().numpy(), js.cpu().numpy()


def assert_v_equal(vg, vr, where=""):
    bad = as_bits(vg) != as_bits(vr)
    if bad.any():
        idx = np.argwhere(bad)[:5]
        raise AssertionError(f"{where}: {bad.sum()} v entries differ, e.g. "
                             + ", ".join(f"{tuple(i)}: gpu={vg[tuple(i)]!r} ref={vr[tuple(i)]!r}"
                                         for i in idx))


def assert_z_close(X, zg, zr, v_all, where="", cols=None):
    rtol, atol = tolerances(X, v_all, cols)
    err = np.abs(zg - zr)
    lim = rtol * np.abs(zr) + atol
    if not (err <= lim).all():
        i = np.unravel_index(np.argmax(err - lim), err.shape)
        raise AssertionError(f"{where}: z differs at {i}: gpu={zg[i]!r} ref={zr[i]!r} "
                             f"err={err[i]:.3e} lim={lim[i]:.3e}")


def assert_s_close(X, sg, sr, vr, where="", cols=None):
    """Per-pair residuals s_jhat,k (every entry): the z bar applied to one
    term, |s_gpu - s_ref| <= rtol |s_ref| + 8 u |v_k| sum_i |x_ijhat|."""
    X = np.asarray(X)
    f32 = X.dtype == np.float32
    u = 2.0 ** -24 if f32 else 2.0 ** -53
    rtol = 1e-5 if f32 else 1e-12
    col = np.abs(X.astype(np.float64)).sum(axis=0)
    if cols is not None:
        col = col[np.asarray(cols)]
    lim = rtol * np.abs(sr) + 8.0 * u * np.abs(np.asarray(vr, dtype=np.float64)) * col[:, None]
    err = np.abs(np.asarray(sg) - sr)
    if not (err <= lim).all():
        i = np.unravel_index(np.argmax(err - lim), err.shape)
        raise AssertionError(f"{where}: s differs at {i}: gpu={sg[i]!r} ref={sr[i]!r} "
                             f"err={err[i]:.3e} lim={lim[i]:.3e}")


def check_scan(X, lams, flags=0, where=""):
    vg, sg, zg = gpu_scan(X, lams, flags)
    ref = oracle.fit(X, lams)
    assert_v_equal(vg, ref["v_all"], where + " v_all")
    assert_z_close(X, zg, ref["z_all"], ref["v_all"], where + " z_all")
    assert_s_close(X, sg, ref["s_all"], ref["v_all"], where + " s_all")
    return vg, zg, ref


def check_fit(X, lams, ref=None, where=""):
    v, obj, js = gpu_fit(X, lams)
    if ref is None:
        ref = oracle.fit(X, lams)
    rtol, atol = tolerances(X, ref["v_all"])
    for t in range(len(np.atleast_1d(lams))):
        jg, jr = int(js[t]), int(ref["jstar"][t])
        if jg != jr:
            zr = ref["z_all"][t]
            lim = rtol * abs(zr[jr]) + atol[t, jg] + atol[t, jr]
            assert abs(zr[jg] - zr[jr]) <= lim, f"{where}: jhat* {jg} vs {jr} not a tie"
        assert_v_equal(v[t], ref["v_all"][t, jg], where + f" v*[{t}]")
        lim = rtol * abs(ref["z_all"][t, jg]) + atol[t, jg]
        assert abs(obj[t] - ref["z_all"][t, jg]) <= lim, (where, obj[t], ref["z_all"][t, jg])
    return v, obj, js
