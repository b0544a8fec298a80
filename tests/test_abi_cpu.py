"""CPU-side checks of the C ABI: the library builds, loads without a GPU,
exports every function declared in include/l1line.h, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_2402_16712_gb300 import l1line

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return l1line.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(l1line_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in l1line.SIGNATURES, f"{nm} has no ctypes signature in the binding"


def test_status_strings(lib):
    for code in range(0, -8, -1):
        s = l1line.status_string(code)
        assert s and s != "unknown status"
    assert l1line.status_string(5) == "unknown status"


def test_workspace_and_limits(lib):
    a = l1line.workspace_bytes(np.float32, 2000, 2000, 1)
    b = l1line.workspace_bytes(np.float64, 2000, 2000, 1)
    assert 0 < a < b
    assert l1line.workspace_bytes(np.float32, 0, 10, 1) == 0
    assert l1line.workspace_bytes(np.float32, 10, 10, 0) == 0
    assert l1line.workspace_bytes(np.float32, 1 << 40, 1 << 40, 1) == 0  # overflow caught
    assert l1line.max_rows(np.float32) >= 5000 and l1line.max_rows(np.float64) >= 5000
    assert lib.l1line_max_rows(7) == 0
    # the path kernels stage a column and eight 256-entry lists per CTA: a lower limit
    for dt in (l1line.DTYPE_F32, l1line.DTYPE_F64):
        pm = lib.l1line_path_max_rows(dt)
        assert 5000 <= pm <= lib.l1line_max_rows(dt) and pm % 32 == 0
        assert lib.l1line_path_workspace_bytes(dt, pm, 10) > 0
        assert lib.l1line_path_workspace_bytes(dt, pm + 1, 10) == 0
    assert lib.l1line_path_max_rows(7) == 0


def _scan(lib, X=256, n=4, m=3, lam=(0.5,), nl=None, ws=1024, wsb=1 << 30, flags=0):
    lam = np.asarray(lam, dtype=np.float64)
    return lib.l1line_scan_ex_f32(X, n, m, lam.ctypes.data_as(ctypes.c_void_p),
                                  lam.size if nl is None else nl, None, None, None, ws, wsb,
                                  None, flags)


def test_argument_errors_return_before_launch(lib):
    # pointers here are never dereferenced: validation fails first
    assert _scan(lib, X=None) == l1line.ERR_ARG
    assert _scan(lib, n=0) == l1line.ERR_ARG
    assert _scan(lib, m=0) == l1line.ERR_ARG
    assert _scan(lib, nl=0) == l1line.ERR_ARG
    assert _scan(lib, lam=(-1.0,)) == l1line.ERR_ARG
    assert _scan(lib, lam=(float("nan"),)) == l1line.ERR_ARG
    assert _scan(lib, lam=(float("inf"),)) == l1line.ERR_ARG
    assert _scan(lib, X=258) == l1line.ERR_ARG  # misaligned float pointer
    assert _scan(lib, n=2 ** 31) == l1line.ERR_UNSUPPORTED  # beyond the global-memory path
    assert _scan(lib, ws=None) == l1line.ERR_WORKSPACE
    assert _scan(lib, ws=1024 + 16) == l1line.ERR_WORKSPACE  # not 256-aligned
    assert _scan(lib, wsb=16) == l1line.ERR_WORKSPACE
    v = ctypes.c_void_p(512)
    lam = np.array([0.1])
    assert lib.l1line_fit_f64(256, 4, 3, lam.ctypes.data_as(ctypes.c_void_p), 1, None, v, v,
                              1024, 1 << 30, None) == l1line.ERR_ARG
    assert lib.l1line_status(None, None) == l1line.ERR_WORKSPACE


def test_exact_list_capacity_stays_within_its_uint32_counter(lib):
    # one launch lists at most m * m * min(n_lambda, 256) pairs for the exact
    # path; its counter is a uint32, so shapes past 2^31 entries are refused
    assert lib.l1line_workspace_bytes(0, 10, 2048, 256) > 0        # 2^30 entries
    assert lib.l1line_workspace_bytes(0, 10, 4096, 128) > 0        # 2^31 entries
    assert lib.l1line_workspace_bytes(0, 10, 4096, 256) == 0       # 2^32 entries
    assert lib.l1line_workspace_bytes(0, 10, 65536, 1) == 0        # 2^32 entries
    assert lib.l1line_workspace_bytes(1, 10, 46341, 1) == 0
    assert _scan(lib, m=65536) == l1line.ERR_UNSUPPORTED


def test_binding_has_no_cpu_fallback(tmp_path):
    with pytest.raises(RuntimeError):
        saved = l1line._lib
        try:
            l1line._lib = None
            l1line.load(str(tmp_path / "missing.so"))
        finally:
            l1line._lib = saved


def test_batched_argument_errors(lib):
    I = np.array
    P = ctypes.c_void_p
    ns, ms = I([10, 20], dtype=np.int64), I([3, 4], dtype=np.int64)
    loff = I([0, 1, 3], dtype=np.int64)
    f = lib.l1line_batched_workspace_bytes
    ok = f(0, 2, ns.ctypes.data_as(P), ms.ctypes.data_as(P), loff.ctypes.data_as(P))
    assert ok > 0
    bad = I([1, 1, 3], dtype=np.int64)  # must start at 0
    assert f(0, 2, ns.ctypes.data_as(P), ms.ctypes.data_as(P), bad.ctypes.data_as(P)) == 0
    empty = I([0, 0, 3], dtype=np.int64)  # an instance without lambdas
    assert f(0, 2, ns.ctypes.data_as(P), ms.ctypes.data_as(P), empty.ctypes.data_as(P)) == 0
    big = np.zeros(258, dtype=np.int64) + 4
    offs = np.arange(258, dtype=np.int64)
    assert f(0, 257, big.ctypes.data_as(P), big.ctypes.data_as(P), offs.ctypes.data_as(P)) == 0
    lam = I([0.1, -1.0, 0.2])
    xp = I([256, 512], dtype=np.uint64)
    rc = lib.l1line_fit_batched_f32(2, xp.ctypes.data_as(P), ns.ctypes.data_as(P),
                                    ms.ctypes.data_as(P), lam.ctypes.data_as(P),
                                    loff.ctypes.data_as(P), P(256), P(256), P(256), P(1024),
                                    1 << 30, None)
    assert rc == l1line.ERR_ARG  # negative lambda


def test_proposer_argument_errors(lib):
    P = ctypes.c_void_p
    p = P(256)
    lam = np.array([0.2])
    L = lam.ctypes.data_as(P)
    # top-K: K outside 1..m, null pointers
    assert lib.l1line_topk(p, 10, 0, p, None) == l1line.ERR_ARG
    assert lib.l1line_topk(p, 10, 11, p, None) == l1line.ERR_ARG
    assert lib.l1line_topk(None, 10, 3, p, None) == l1line.ERR_ARG
    # network: null or misaligned image, empty batch
    assert lib.l1line_mlp_forward(p, None, 0, p, p, None) == l1line.ERR_ARG
    assert lib.l1line_mlp_forward(p, None, 10, P(264), p, None) == l1line.ERR_ARG
    assert lib.l1line_mlp_forward(p, None, 10, None, p, None) == l1line.ERR_ARG
    assert lib.l1line_mlp_workspace_bytes(0) == 0
    assert lib.l1line_mlp_workspace_bytes(64) == 17281 * 4 + 252  # one CTA row, 256-aligned
    assert lib.l1line_mlp_backward(p, None, 100, p, p, p, None, 1 << 20, None) == \
        l1line.ERR_WORKSPACE
    assert lib.l1line_mlp_backward(p, None, 100, p, p, p, P(1024), 16, None) == l1line.ERR_WORKSPACE
    # Adam: step >= 1, betas in [0, 1), finite learning rate
    assert lib.l1line_adam_step(p, p, p, p, 0, 1e-3, 0.9, 0.999, 1e-8, None, None) == l1line.ERR_ARG
    assert lib.l1line_adam_step(p, p, p, p, 1, 1e-3, 1.0, 0.999, 1e-8, None, None) == l1line.ERR_ARG
    assert lib.l1line_adam_step(p, p, p, p, 1, float("inf"), 0.9, 0.999, 1e-8, None, None) == \
        l1line.ERR_ARG
    assert lib.l1line_rank_loss(p, p, None, p, 0, p, p, None) == l1line.ERR_ARG
    # subset / proposed fits
    assert lib.l1line_fit_subset_f32(p, 10, 5, L, 1, None, 2, p, p, p, P(1024), 1 << 30,
                                     None) == l1line.ERR_ARG
    assert lib.l1line_fit_subset_f32(p, 10, 5, L, 1, p, 0, p, p, p, P(1024), 1 << 30,
                                     None) == l1line.ERR_ARG
    # more entries than columns (the exact path's pair list holds m per jhat row)
    assert lib.l1line_fit_subset_f32(p, 10, 5, L, 1, p, 6, p, p, p, P(1024), 1 << 30,
                                     None) == l1line.ERR_ARG
    assert lib.l1line_fit_proposed_f32(p, 10, 5, L, 1, p, 6, None, p, p, p, P(1024), 1 << 30,
                                       None) == l1line.ERR_ARG
    assert lib.l1line_fit_proposed_f64(p, 10, 5, L, 1, None, 2, None, p, p, p, P(1024), 1 << 30,
                                       None) == l1line.ERR_ARG
    assert lib.l1line_features_f32(p, 10, 5, 0.2, None, None, P(1024), 1 << 30, None) == \
        l1line.ERR_ARG


def test_probe_argument_errors(lib):
    P = ctypes.c_void_p
    out = ctypes.c_double(0.0)
    ref = ctypes.byref(out)
    assert lib.l1line_probe(2, P(256), 1024, 1, P(256), None, ref) == l1line.ERR_ARG  # kind
    assert lib.l1line_probe(l1line.PROBE_L2, P(256), 1024, 0, P(256), None, ref) == l1line.ERR_ARG
    assert lib.l1line_probe(l1line.PROBE_L2, None, 1024, 1, P(256), None, ref) == l1line.ERR_ARG
    assert lib.l1line_probe(l1line.PROBE_L2, P(264), 1024, 1, P(256), None, ref) == l1line.ERR_ARG
    assert lib.l1line_probe(l1line.PROBE_L2, P(256), 8, 1, P(256), None, ref) == l1line.ERR_ARG
    assert lib.l1line_probe(l1line.PROBE_SMEM, None, 0, 1, None, None, ref) == l1line.ERR_ARG
    assert lib.l1line_probe(l1line.PROBE_SMEM, None, 0, 1, P(258), None, ref) == l1line.ERR_ARG
    assert lib.l1line_probe(l1line.PROBE_SMEM, None, 0, 1, P(256), None, None) == l1line.ERR_ARG


def test_proposer_rows_and_workspace(lib):
    # the restricted fit takes min(n, max(256, ceil(n / 8))) rows
    assert [lib.l1line_proposer_rows(n) for n in (0, 1, 200, 256, 2048, 2049, 5000)] == \
        [0, 1, 200, 256, 256, 257, 625]
    for dt in (0, 1):
        for n, m, nl in ((300, 20, 1), (5000, 1000, 1), (2000, 50, 3)):
            fit = lib.l1line_workspace_bytes(dt, n, m, nl)
            prop = lib.l1line_proposed_workspace_bytes(dt, n, m, nl)
            R = lib.l1line_proposer_rows(n)
            # the fit's workspace, the row norms, row list, row copy and the
            # restricted fit's own workspace
            assert prop >= fit + n * 4 + R * 4 + R * m * (4 if dt == 0 else 8) + \
                lib.l1line_workspace_bytes(dt, R, m, 1)
    assert lib.l1line_proposed_workspace_bytes(2, 10, 10, 1) == 0
    # the proposer keeps the shared-memory row limit; plain fits go past it
    for dt in (0, 1):
        mr = lib.l1line_max_rows(dt)
        assert lib.l1line_proposed_workspace_bytes(dt, mr, 10, 1) > 0
        assert lib.l1line_proposed_workspace_bytes(dt, mr + 1, 10, 1) == 0
        assert lib.l1line_workspace_bytes(dt, mr + 1, 10, 1) > 0
    assert lib.l1line_proposed_workspace_bytes(0, 0, 10, 1) == 0
    P = ctypes.c_void_p
    lam = np.array([0.2])
    small = lib.l1line_proposed_workspace_bytes(0, 10, 5, 1) - 256
    assert lib.l1line_features_f32(P(256), 10, 5, 0.2, None, P(512), P(1024), small, None) == \
        l1line.ERR_WORKSPACE
    assert lib.l1line_features_f32(P(256), 10, 5, 0.2, None, None, P(1024), 1 << 30, None) == \
        l1line.ERR_ARG
    assert lib.l1line_fit_proposed_f32(P(256), 10, 5, lam.ctypes.data_as(P), 1, P(256), 2, None,
                                       P(512), P(512), P(512), P(1024), small, None) == \
        l1line.ERR_WORKSPACE


def test_committed_network_parameters():
    from paper_2402_16712_gb300 import proposer
    th = proposer.load_theta()
    assert th.dtype == np.float32 and th.size == l1line.MLP_PARAMS
    assert np.isfinite(th).all() and np.abs(th).max() < 65504  # binary16-representable range
