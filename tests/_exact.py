"""Exact rational restatements used to pin the oracle (pure Python, tiny inputs).

Nothing here imports the oracle or the CUDA path.  Every float is turned into
its exact rational value (``Fraction(float)`` is exact), so these functions
are free of rounding.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def fr(x) -> Fraction:
    return Fraction(float(x))


def pair_objective(a, b, lam, t):
    """f(t) = sum_i |a_i - t b_i| + lam |t|  (the one-variable LP (l1reglp))."""
    t = Fraction(t)
    return sum(abs(fr(ai) - t * fr(bi)) for ai, bi in zip(a, b)) + fr(lam) * abs(t)


def pair_breakpoints(a, b):
    return sorted({fr(ai) / fr(bi) for ai, bi in zip(a, b) if bi != 0} | {Fraction(0)})


def pair_right_endpoint(a, b, lam):
    """Brute force: evaluate f at every breakpoint; return (min value, right end
    point of the minimiser set).  If every weight is zero (f constant) the
    right end point is undefined and Algorithm 1 keeps v = 0: return 0."""
    if all(bi == 0 for bi in b) and lam == 0:
        return pair_objective(a, b, lam, 0), Fraction(0)
    cands = pair_breakpoints(a, b)
    vals = [pair_objective(a, b, lam, t) for t in cands]
    best = min(vals)
    return best, max(t for t, v in zip(cands, vals) if v == best)


def sgn(x):
    return (x > 0) - (x < 0)


def alg1_literal(a, b, lam, order=None):
    """Algorithm 1's inner loop transcribed as printed: sort the ratios over rows
    with x_ijhat != 0, then for each position p test
        sgn(r_p) * lam  in  ( sum_{q>p} w_q - sum_{q<=p} w_q ,
                              sum_{q>=p} w_q - sum_{q<p} w_q ]
    and let the last satisfying position set v (v starts at 0).  ``order``
    breaks ties between equal ratios (a permutation of the row indices)."""
    lam = fr(lam)
    rows = [i for i in range(len(a)) if b[i] != 0]
    if order is not None:
        rank = {i: p for p, i in enumerate(order)}
        rows.sort(key=lambda i: rank[i])
    items = sorted(((fr(a[i]) / fr(b[i]), abs(fr(b[i]))) for i in rows), key=lambda t: t[0])
    w = [it[1] for it in items]
    tot = sum(w)
    v = Fraction(0)
    pre = Fraction(0)
    for p, (r, wp) in enumerate(items):
        below = pre              # sum_{q<p}
        above = tot - pre - wp   # sum_{q>p}
        lo = above - (below + wp)
        hi = (above + wp) - below
        s = sgn(r) * lam
        if lo < s <= hi:
            v = r
        pre += wp
    return v


def dual_certificate_ok(a, b, lam, t):
    """Lemma 1's optimality argument: build a dual point (pi, gamma) of the LP
    (l1reglp) complementary to the primal value t and check dual feasibility and
    equal objectives (exact).  Returns True iff t is certified optimal."""
    lam = fr(lam)
    t = Fraction(t)
    rows = [i for i in range(len(a)) if b[i] != 0]
    r = {i: fr(a[i]) / fr(b[i]) for i in rows}
    w = {i: abs(fr(b[i])) for i in rows}
    pi = {}
    for i in rows:
        if r[i] > t:
            pi[i] = w[i]
        elif r[i] < t:
            pi[i] = -w[i]
    # free multipliers: rows with r_i == t (|pi_i| <= w_i) and gamma (|gamma| <= lam,
    # gamma = -sgn(t) lam when t != 0 for complementary slackness).
    tied = [i for i in rows if r[i] == t]
    fixed = sum(pi.values())
    if t != 0:
        gamma_lo = gamma_hi = -sgn(t) * lam
    else:
        gamma_lo, gamma_hi = -lam, lam
    # need sum_tied pi_i = -(fixed + gamma) with |pi_i| <= w_i
    cap = sum(w[i] for i in tied)
    need_lo = -(fixed + gamma_hi)
    need_hi = -(fixed + gamma_lo)
    if need_hi < -cap or need_lo > cap:
        return False
    need = max(need_lo, -cap)
    gamma = -(fixed + need)
    rem = need
    for i in tied:
        take = max(-w[i], min(w[i], rem))
        pi[i] = take
        rem -= take
    assert rem == 0
    assert sum(pi.values()) + gamma == 0
    assert all(abs(pi[i]) <= w[i] for i in rows) and abs(gamma) <= lam
    dual = sum(r[i] * pi[i] for i in rows)
    primal = sum(w[i] * abs(r[i] - t) for i in rows) + lam * abs(t)
    return dual == primal


def fit_exact(X, lam):
    """Algorithm 1 over every jhat in exact arithmetic with the right-end-point
    rule: returns (z list, v list per jhat) as Fractions."""
    X = np.asarray(X)
    n, m = X.shape
    zs, vs = [], []
    for j in range(m):
        v = []
        for k in range(m):
            if k == j:
                v.append(Fraction(1))
            else:
                v.append(pair_right_endpoint(X[:, k], X[:, j], lam)[1])
        z = sum(abs(fr(X[i, k]) - v[k] * fr(X[i, j])) for i in range(n) for k in range(m))
        z += fr(lam) * sum(abs(x) for x in v)
        zs.append(z)
        vs.append(v)
    return zs, vs


def objective_at(X, j, v, lam):
    """z_j at a given v (exact): sum_i sum_k |x_ik - v_k x_ij| + lam sum_k |v_k|."""
    X = np.asarray(X)
    n, m = X.shape
    vq = [fr(x) for x in v]
    z = sum(abs(fr(X[i, k]) - vq[k] * fr(X[i, j])) for i in range(n) for k in range(m))
    return z + fr(lam) * sum(abs(x) for x in vq)
