"""CPU oracle of successive components (the paper's closing remark after
Proposition 5: apply Algorithm 1 again to the data projected onto the null
space of the components found so far).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading (the paper does not define the projection): a component (jhat, v)
with v_jhat = 1 represents point x_i by x_ijhat v, the term its objective
measures; the projected point is the residual x_i - x_ijhat v, whose jhat-th
coordinate is 0.  Arithmetic in the input precision, the product rounded
before the subtraction (no fused multiply-add):
    x'_ik = fl(x_ik - fl(v_k x_ijhat)).
"""
from __future__ import annotations

import numpy as np

from . import fit as _fit


def deflate(X, jhat: int, v):
    X = np.asarray(X)
    dt = X.dtype.type
    prod = (np.asarray(v, dtype=X.dtype)[None, :] * X[:, [jhat]]).astype(X.dtype)
    return (X - prod).astype(X.dtype)


def components(X, lam: float, ncomp: int):
    """Returns (V [ncomp, m], obj [ncomp], jstar [ncomp]) and the deflated
    matrices after each component."""
    X = np.ascontiguousarray(X)
    V, objs, js, mats = [], [], [], []
    for _ in range(ncomp):
        r = _fit(X, [lam], want_all=False)
        v, obj, j = r["v"][0], float(r["obj"][0]), int(r["jstar"][0])
        V.append(v)
        objs.append(obj)
        js.append(j)
        X = deflate(X, j, v)
        mats.append(X)
    return np.array(V), np.array(objs), np.array(js), mats
