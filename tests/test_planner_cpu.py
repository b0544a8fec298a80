"""The pair kernel's launch planner, on the host (no GPU): l1line_plan_for
computes the plan l1line_plan would make on a GPU of the given SM count.

Pinned here are the plans the measurements in the design doc were taken with on
the 152-SM GB300 (the bench's `config.tuning.plan` lines), and invariants that
every plan must meet: a compiled launch shape, the shared-memory budget, a k
split that covers every column, and the caller's tuning taken as given.
"""
import numpy as np
import pytest

import __graft_entry__
from paper_2402_16712_gb300 import l1line

SMS = 152


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    l1line.load()
    yield
    l1line.set_tuning(None)


def _plan(dtype, n, m, d0=0, nj=None, **tune):
    t = dict(tune)
    if d0:
        t["d0"] = d0
    l1line.set_tuning(t or None)
    try:
        return l1line.plan_for(dtype, n, m, SMS, nj)
    finally:
        l1line.set_tuning(None)


@pytest.mark.parametrize("dtype,n,m,d0,want", [
    # the headline fit: 16 warps x 2 CTAs (64 registers), 3 k-chunks, x_ijhat in shared memory
    (np.float32, 2000, 2000, 4, dict(warps=16, ctas_per_sm=2, kchunk=667, column=1)),
    # double input reads x_ijhat from the column copy in global memory
    (np.float64, 2000, 2000, 4, dict(warps=16, ctas_per_sm=2, kchunk=667, column=2)),
    # n = 5000 leaves room for 16 resident warps (128 registers)
    (np.float32, 5000, 1000, 4, dict(warps=16, ctas_per_sm=1, kchunk=334, column=1)),
    (np.float32, 1000, 500, 4, dict(warps=16, ctas_per_sm=2, kchunk=250, column=1)),
    # a small fit whose pairs fill one wave: the latency plan, 8 x 3 warps
    (np.float64, 200, 20, 0, dict(warps=8, ctas_per_sm=3, column=2)),
])
def test_plans_of_the_measured_workloads(dtype, n, m, d0, want):
    p = _plan(dtype, n, m, d0)
    for k, v in want.items():
        assert p[k] == v, (k, p)


def _shape(warps, ctas):
    # the compiled launch shapes: <= 16 resident warps (128 registers),
    # 17-24 in CTAs of <= 8 warps (80), 25-32 (64)
    t = warps * ctas
    if not (1 <= warps <= 16 and 1 <= ctas <= 3):
        return None
    if t <= 16:
        return "r128"
    if t <= 24:
        return "r80" if warps <= 8 else None
    return "r64" if t <= 32 else None


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_every_plan_is_a_compiled_shape_and_covers_every_column(dtype):
    rng = np.random.default_rng(5)
    for _ in range(300):
        n = int(rng.integers(1, l1line.max_rows(dtype) + 1))
        m = int(rng.integers(1, 3000))
        d0 = int(rng.choice([0, 3, 4, 6, 10]))
        p = _plan(dtype, n, m, d0)
        assert _shape(p["warps"], p["ctas_per_sm"]) is not None, (n, m, p)
        assert p["column"] in (1, 2) and (dtype == np.float32 or p["column"] == 2), p
        chunks = -(-m // p["kchunk"])
        assert 1 <= chunks <= m and p["kchunk"] * chunks >= m, (m, p)
        assert p["d0"] == (d0 or 6)


def test_rows_beyond_the_pair_kernel_are_not_planned():
    for dtype in (np.float32, np.float64):
        mr = l1line.max_rows(dtype)
        assert _plan(dtype, mr, 8)["warps"] > 0
        with pytest.raises(l1line.L1LineError):
            _plan(dtype, mr + 1, 8)  # the global-memory path takes these


def test_the_callers_tuning_is_taken_as_given():
    p = _plan(np.float32, 2000, 2000, 4, warps=8, ctas_per_sm=3, kchunk=500, column=2)
    assert (p["warps"], p["ctas_per_sm"], p["kchunk"], p["column"]) == (8, 3, 500, 2)
    # fewer SMs: more k-chunks keep at least four CTAs per SM busy
    l1line.set_tuning({"d0": 4})
    try:
        few = l1line.plan_for(np.float32, 2000, 200, 8, 200)
        many = l1line.plan_for(np.float32, 2000, 200, SMS, 200)
    finally:
        l1line.set_tuning(None)
    assert few["kchunk"] >= many["kchunk"]


def test_plan_for_rejects_bad_arguments():
    lib = l1line.load()
    t = l1line.Tuning()
    import ctypes
    assert lib.l1line_plan_for(0, 100, 10, 10, 0, ctypes.byref(t)) == l1line.ERR_ARG
    assert lib.l1line_plan_for(0, 0, 10, 10, 152, ctypes.byref(t)) == l1line.ERR_ARG
    assert lib.l1line_plan_for(7, 100, 10, 10, 152, ctypes.byref(t)) == l1line.ERR_ARG
    assert lib.l1line_plan_for(0, 100, 10, 10, 152, None) == l1line.ERR_ARG
