"""CPU oracle of Algorithm 3: the solution path over all lambda >= 0.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain Python in exact
rationals, for small instances.

Input, as Algorithm 3 requires: the ordered breakpoints lambda^1 < ... <
lambda^K of Algorithm 2 over every preserved coordinate, and for each jhat
the solution v^jhat on each interval (from oracle.path).  For each interval
[lambda^k, lambda^(k+1)] and each jhat, z^jhat(lambda^k) is the objective of
v^jhat (the value holding just after lambda^k) and ||v^jhat||_1 its slope in
lambda.  For each coordinate j, beta_L (the largest offset at which line j
undercuts a line of larger slope) and beta_U (the smallest offset at which a
line of smaller slope undercuts j) bound where j is the lowest line; j starts
the solution at lambda^k + beta_L when 0 < beta_L < beta_U within the
interval, or at lambda^k when beta_L <= 0 < beta_U, provided no line of equal
slope lies strictly below it.

Readings (the paper is silent): the last interval is [lambda^K, infinity)
(lambda^K = lambda_max, after which every v is e_jhat-like with slope 1);
lines of equal value and equal slope are one line, and the smallest jhat
names it (Algorithm 1's argmin rule); consecutive entries with the same jhat
and the same v are merged.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import path as _path


def _F(x):
    return Fraction(float(x))


def _value_after(lam, v, q):
    """The pair path's value on the open interval just after q."""
    g = int(np.searchsorted(lam, q, side="right")) - 1
    return v[g]


def pair_paths(X):
    m = X.shape[1]
    return {(j, k): _path(X, j, k) for j in range(m) for k in range(m)}


def solution_path(X, paths=None):
    """Returns (entries, breakpoints): entries is a list of (lambda_start
    (Fraction), jhat, v (tuple of floats), z_intercept, slope) ordered by
    lambda_start: from lambda_start on, the solution is v^jhat with objective
    z_intercept + slope * lambda; breakpoints is Algorithm 2's ordered set."""
    X = np.asarray(X)
    n, m = X.shape
    if paths is None:
        paths = pair_paths(X)
    Xf = [[_F(X[i, k]) for k in range(m)] for i in range(n)]
    lams = sorted({_F(l) for (lam, _) in paths.values() for l in lam} | {Fraction(0)})
    ext = lams + [None]  # the last interval is unbounded
    raw = []
    for kk in range(len(lams)):
        lo, hi = ext[kk], ext[kk + 1]
        # v^jhat on (lo, hi): the value just after lo
        V = []
        for jh in range(m):
            V.append(tuple(_F(_value_after(*paths[(jh, k)], float(lo))) for k in range(m)))
        S = [sum(abs(x) for x in V[jh]) for jh in range(m)]
        Z = []
        for jh in range(m):
            r = sum(abs(Xf[i][k] - V[jh][k] * Xf[i][jh]) for i in range(n) for k in range(m))
            Z.append(r + lo * S[jh])  # z^jhat(lambda^k)
        for j in range(m):
            # equal-slope lines strictly below j, or an equal line with a smaller index
            if any(S[h] == S[j] and (Z[h] < Z[j] or (Z[h] == Z[j] and h < j))
                   for h in range(m) if h != j):
                continue
            bl = [(Z[j] - Z[h]) / (S[h] - S[j]) for h in range(m) if S[j] < S[h]]
            bu = [(Z[h] - Z[j]) / (S[j] - S[h]) for h in range(m) if S[j] > S[h]]
            beta_l = max(bl) if bl else None
            beta_u = min(bu) if bu else None
            lt_u = lambda b: beta_u is None or b < beta_u
            if beta_l is not None and 0 < beta_l and lt_u(beta_l) and (
                    hi is None or lo + beta_l <= hi):
                start = lo + beta_l
            elif (beta_l is None or beta_l <= 0) and lt_u(0):
                start = lo
            else:
                continue
            raw.append((start, kk, j, V[j], Z[j] - lo * S[j], S[j]))
    # by start; at one lambda the later interval's line is the one that holds after it
    raw.sort(key=lambda e: (e[0], e[1], e[2]))
    out = []
    for (s0, _, j, v, zi, sl) in raw:
        e = (s0, j, v, zi, sl)
        if out and out[-1][0] == s0:
            out[-1] = e
        else:
            out.append(e)
        if len(out) >= 2 and out[-2][1] == out[-1][1] and out[-2][2] == out[-1][2]:
            out.pop()
    entries = [(s, j, tuple(float(x) for x in v), zi, sl) for (s, j, v, zi, sl) in out]
    return entries, lams
