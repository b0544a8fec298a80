"""The no-allocation fit entry point (`l1line_fit_noalloc_f32`).

It serves callers that cannot allocate device memory (their device memory is
owned by another allocator, or an allocation's implicit synchronisation is not
acceptable): it takes no workspace and runs in a fixed scratch array that the
library declares in device memory.  The test calls it through the C ABI twice
in a row and checks both results against the ordinary `l1line_fit_f32`, under
the same bar as the parity tests (v bit-identical, objectives within 1e-5
relative, the same jhat*).  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import __graft_entry__
from paper_2402_16712_gb300 import datagen, l1line


def _call_noalloc(lib, Xd, lams, n_out):
    import torch
    n, m = Xd.shape
    nl = lams.size
    v = torch.full((nl, m), float("nan"), dtype=torch.float32, device=Xd.device)
    obj = torch.full((nl,), float("nan"), dtype=torch.float64, device=Xd.device)
    js = torch.full((nl,), -7, dtype=torch.int32, device=Xd.device)
    stream = torch.cuda.current_stream()
    rc = lib.l1line_fit_noalloc_f32(Xd.data_ptr(), n, m, lams.ctypes.data_as(ctypes.c_void_p),
                                    nl, v.data_ptr(), obj.data_ptr(), js.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream))
    assert rc == l1line.OK, l1line.status_string(rc)
    torch.cuda.synchronize()
    return v.cpu().numpy(), obj.cpu().numpy(), js.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_fit_matches_fit_twice_in_a_row():
    import torch
    __graft_entry__.build()
    lib = l1line.load()
    lams = np.array([0.0, 0.1, 0.7], dtype=np.float64)
    results = []
    for seed in (3, 4):  # two different inputs, one call each, back to back
        X, _, _ = datagen.planted(datagen.Planted(300, 40, 4, 0.1, 0.1, 5.0, seed, "float32"))
        Xd = torch.from_numpy(X).cuda()
        assert l1line.workspace_bytes(np.float32, 300, 40, lams.size) <= l1line.NOALLOC_SCRATCH_BYTES
        results.append((Xd, _call_noalloc(lib, Xd, lams, 0)))
    for Xd, (v, obj, js) in results:
        rv, robj, rjs, ws = l1line.fit(Xd, lams)
        assert l1line.status(ws) == l1line.OK
        rv, robj, rjs = rv.cpu().numpy(), robj.cpu().numpy(), rjs.cpu().numpy()
        assert np.array_equal(js, rjs)
        assert np.array_equal(v.view(np.uint32), rv.view(np.uint32))
        assert np.all(np.abs(obj - robj) <= 1e-5 * np.abs(robj))


@pytest.mark.gpu
def test_noalloc_status_reports_a_nonfinite_input():
    """The call returns before its kernels run; l1line_noalloc_status reads the
    device-side status the fit left in the scratch: NaN in X is reported,
    and the next clean call clears it."""
    import torch
    __graft_entry__.build()
    lib = l1line.load()
    lams = np.array([0.2], dtype=np.float64)
    X, _, _ = datagen.planted(datagen.Planted(200, 12, 3, 0.1, 0.1, 5.0, 9, "float32"))
    bad = X.copy()
    bad[17, 5] = np.nan
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _call_noalloc(lib, torch.from_numpy(bad).cuda(), lams, 0)
    assert lib.l1line_noalloc_status(stream) == l1line.ERR_NONFINITE
    _call_noalloc(lib, torch.from_numpy(X).cuda(), lams, 0)
    assert lib.l1line_noalloc_status(stream) == l1line.OK


def test_noalloc_rejects_sizes_beyond_its_scratch():
    __graft_entry__.build()
    lib = l1line.load()
    lams = np.array([0.5])
    p = ctypes.c_void_p(256)
    # 2000 x 2000 needs ~128 MB of workspace: refused before any device call
    assert l1line.workspace_bytes(np.float32, 2000, 2000, 1) > l1line.NOALLOC_SCRATCH_BYTES
    rc = lib.l1line_fit_noalloc_f32(256, 2000, 2000, lams.ctypes.data_as(ctypes.c_void_p), 1,
                                    p, p, p, None)
    assert rc == l1line.ERR_UNSUPPORTED
    rc = lib.l1line_fit_noalloc_f32(None, 20, 20, lams.ctypes.data_as(ctypes.c_void_p), 1,
                                    p, p, p, None)
    assert rc == l1line.ERR_ARG
