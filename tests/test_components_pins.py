"""Pins of the successive-components oracle (oracle/components.py): the first
component is the fit; the deflated data's jhat column is exactly zero; the
l1 norm of the deflated data is the component's residual (its objective less
the penalty); exact rank-one data deflates to zero; on all-zero data every
later component is e_0 with objective lambda."""
import numpy as np
import pytest

import oracle
from oracle import components as C
from paper_2402_16712_gb300 import datagen


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_components_properties(dtype):
    X, _, _ = datagen.planted(datagen.Planted(80, 9, 3, 0.1, 0.1, 5.0, 2, dtype))
    lam = 0.3
    V, obj, js, mats = C.components(X, lam, 4)
    r = oracle.fit(X, [lam], want_all=False)
    assert np.array_equal(V[0], r["v"][0]) and js[0] == r["jstar"][0] and obj[0] == r["obj"][0]
    prev = X
    for c in range(4):
        D = mats[c]
        assert np.all(D[:, js[c]] == 0)  # v_jhat = 1: the column cancels exactly
        # residual of component c = l1 norm of the deflated data (up to rounding)
        resid = obj[c] - lam * np.abs(V[c].astype(np.float64)).sum()
        l1 = np.abs(D.astype(np.float64)).sum()
        u = 2.0 ** -24 if dtype == "float32" else 2.0 ** -53
        assert abs(l1 - resid) <= 4 * u * (np.abs(prev.astype(np.float64)).sum() + l1)
        prev = D
    # each later component fits the deflated data of the previous one
    r2 = oracle.fit(mats[0], [lam], want_all=False)
    assert np.array_equal(V[1], r2["v"][0]) and js[1] == r2["jstar"][0]


def test_rank_one_data_deflates_to_zero():
    rng = np.random.default_rng(3)
    t = rng.integers(-8, 9, size=30).astype(np.float64)
    a = np.array([1.0, -2.0, 0.5, 4.0, 0.0, -0.25])  # dyadic: every product exact
    X = np.outer(t, a)
    V, obj, js, mats = C.components(X, 0.0, 3)
    # at lambda = 0 every coordinate with a_j != 0 fits exactly (z = 0): the
    # smallest such jhat is chosen, v = a / a_0
    assert js[0] == 0 and np.array_equal(V[0], a) and obj[0] == 0.0
    assert np.all(mats[0] == 0.0)
    # on zero data: v = e_0, z = lambda * 1 = 0 here
    assert js[1] == 0 and np.array_equal(V[1], np.eye(6)[0]) and obj[1] == 0.0
    V2, obj2, js2, _ = C.components(np.zeros((5, 4)), 0.7, 2)
    assert list(js2) == [0, 0] and np.allclose(obj2, 0.7)
