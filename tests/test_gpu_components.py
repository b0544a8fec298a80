"""Successive components on the GPU (l1line_components) against the oracle
(oracle/components.py): every component's v bit for bit, jhat* equal (or an
objective tie within the parity tolerance), objectives within the parity
tolerance; exact rank-one data deflates to zero."""
import numpy as np
import pytest
import torch

from oracle import components as C
from paper_2402_16712_gb300 import datagen, l1line

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _gpu(X, lam, nc):
    v, obj, js, ws = l1line.components(torch.from_numpy(np.ascontiguousarray(X)).cuda(), lam, nc)
    assert l1line.status(ws) == l1line.OK
    return v.cpu().numpy(), obj.cpu().numpy(), js.cpu().numpy()


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_components_match_oracle(dtype):
    X, _, _ = datagen.planted(datagen.Planted(300, 16, 4, 0.1, 0.1, 5.0, 6, dtype))
    V, obj, js, _ = C.components(X, 0.2, 5)
    gv, gobj, gjs = _gpu(X, 0.2, 5)
    rtol = 1e-5 if dtype == "float32" else 1e-12
    for c in range(5):
        assert gjs[c] == js[c], (c, gjs, js)
        assert np.array_equal(gv[c], V[c]), c
        assert abs(gobj[c] - obj[c]) <= rtol * abs(obj[c]) + 1e-12


def test_rank_one_components():
    rng = np.random.default_rng(3)
    t = rng.integers(-8, 9, size=40).astype(np.float32)
    a = np.array([1.0, -2.0, 0.5, 4.0, 0.0, -0.25], dtype=np.float32)
    X = np.outer(t, a).astype(np.float32)
    gv, gobj, gjs = _gpu(X, 0.0, 3)
    assert list(gjs) == [0, 0, 0] and np.array_equal(gv[0], a) and gobj[0] == 0.0
    assert np.array_equal(gv[1], np.eye(6, dtype=np.float32)[0]) and gobj[1] == 0.0
