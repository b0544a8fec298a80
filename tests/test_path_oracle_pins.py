"""Pins of the Algorithm 2 oracle (oracle.path): the lambda path of v_k for
one preserved coordinate jhat, against facts that do not come from it --
the paper's toy breakpoints and Figure 1, Algorithm 1 (the pinned pair
oracle) evaluated on both sides of every breakpoint, and the breakpoints
recomputed in exact rationals from the weighted-median condition."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2402_16712_gb300 import datagen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "toy_example.json")


def _toy():
    d = json.load(open(GOLDEN))
    return np.array(d["points"], dtype=np.float64), d


def test_toy_breakpoints_match_figure_and_text():
    X, d = _toy()
    m = X.shape[1]
    union = set()
    for j in range(m):
        bps = set()
        for k in range(m):
            lam, v = oracle.path(X, j, k)
            bps |= set(lam.tolist())
        union |= bps
        # positive breakpoints = the lambdas where Figure 1's z_jhat line bends
        fig = {float(s["from"]) for s in d["figure1_lines"] if s["jhat"] == j + 1 and
               float(s["from"]) > 0}
        assert {b for b in bps if b > 0} == fig, (j, bps, fig)
        text = set(d["algorithm2_text"]["per_jhat"][str(j + 1)])
        assert text <= bps | {0.0}  # the text's lists (jhat = 1 omits 11)
    assert sorted(union) == d["algorithm2_text"]["collection"]


def test_toy_solution_values_of_table1():
    X, d = _toy()
    # jhat = 4 on [0, 3): v = (-2/3, 1/3, -1/2, 1); at 3.25 v_3 = 0
    for lam_q, want in ((0.0, [-2 / 3, 1 / 3, -0.5, 1.0]), (3.25, [-2 / 3, 1 / 3, 0.0, 1.0])):
        got = []
        for k in range(4):
            lam, v = oracle.path(X, 3, k)
            got.append(_path_value(lam, v, lam_q))
        assert np.allclose(got, want, rtol=0, atol=1e-15)
    # jhat = 1 on (3.5, 11): v = (1, 0, 0, -0.2); beyond 11: (1, 0, 0, 0)
    for lam_q, want in ((5.0, [1.0, 0.0, 0.0, -0.2]), (12.0, [1.0, 0.0, 0.0, 0.0])):
        got = []
        for k in range(4):
            lam, v = oracle.path(X, 0, k)
            got.append(_path_value(lam, v, lam_q))
        assert np.allclose(got, want, rtol=0, atol=1e-15)


def _path_value(lam, v, q):
    """Value of the path at lambda q = 0 or strictly inside a segment."""
    if q == 0.0:
        return v[0]
    return v[np.searchsorted(lam, q, side="left") - 1]


def _check_against_alg1(X, at_breakpoints):
    n, m = X.shape
    for j in range(m):
        for k in range(m):
            lam, v = oracle.path(X, j, k)
            assert lam[0] == 0.0 and (lam[1:] >= lam[:-1]).all()
            if k == j:
                assert list(v) == [1.0]
                continue
            assert v[-1] == 0.0
            # |v| shrinks toward 0 and keeps its sign
            assert (np.abs(v[1:]) < np.abs(v[:-1])).all()
            assert (np.sign(v[:-1]) == np.sign(v[0])).all()
            a, b = X[:, k], X[:, j]
            qs = [0.0] + [0.5 * (lam[g] + lam[g + 1]) for g in range(len(lam) - 1)
                          if lam[g + 1] > lam[g]] + [lam[-1] + 1.0, 2 * lam[-1] + 7.0]
            for q in qs:
                want = oracle.pair(a, b, q)
                assert _path_value(lam, v, q) == want, (j, k, q)
            if at_breakpoints:
                # at a breakpoint the value on the positive side is still the
                # previous one (the test is strict), on the negative side the new one
                for g in range(1, len(lam)):
                    if lam[g] == lam[g - 1]:
                        continue
                    want = oracle.pair(a, b, lam[g])
                    expect = v[g - 1] if v[g - 1] > 0 else v[g]
                    assert want == expect, (j, k, g)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_path_equals_algorithm1_on_tie_heavy_integers(seed):
    X = datagen.small_integers(14, 6, seed, lo=-4, hi=4, zero_frac=0.25, dtype="float64")
    _check_against_alg1(X, at_breakpoints=True)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_path_equals_algorithm1_on_planted_floats(dtype):
    X, _, _ = datagen.planted(datagen.Planted(60, 7, 3, 0.1, 0.1, 5.0, 3, dtype))
    _check_against_alg1(X, at_breakpoints=False)


def _exact_path(a, b):
    """Breakpoints from the weighted-median condition in rationals: for a
    positive start value, v = t from lambda = (weight above t) - (weight at or
    below t) on; for a negative one, v leaves t at (weight at or below t) -
    (weight above t)."""
    rows = [(Fraction(float(x)) / Fraction(float(y)), abs(Fraction(float(y))))
            for x, y in zip(a, b) if y != 0]
    vals = sorted({r for r, _ in rows})
    W = sum(w for _, w in rows)

    def below(t):
        return sum(w for r, w in rows if r <= t)

    # the lambda = 0 median (right end point rule with a zero-weight penalty point)
    cand = sorted(set(vals) | {Fraction(0)})
    v0 = next(t for t in cand if 2 * below(t) > W)
    out = [(Fraction(0), v0)]
    if v0 > 0:
        for t in sorted((t for t in vals if 0 < t < v0), reverse=True):
            out.append((W - 2 * below(t), t))
        out.append((W - 2 * below(Fraction(0)), Fraction(0)))
    elif v0 < 0:
        seq = [t for t in vals if v0 <= t < 0]
        for g, t in enumerate(seq):
            nxt = seq[g + 1] if g + 1 < len(seq) else Fraction(0)
            out.append((2 * below(t) - W, nxt))
    return out


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_breakpoint_lambdas_in_exact_rationals(seed):
    rng = np.random.default_rng(seed)
    X = rng.integers(-9, 10, size=(11, 5)).astype(np.float64) / rng.choice([1, 2, 4, 8], size=(11, 5))
    for j in range(5):
        for k in range(5):
            if j == k:
                continue
            lam, v = oracle.path(X, j, k)
            ex = _exact_path(X[:, k], X[:, j])
            # the oracle merges equal values and clips at 0; compare value by value
            got = list(zip(lam.tolist(), v.tolist()))
            assert len(got) == len(ex), (j, k, got, ex)
            for (gl, gv), (el, ev) in zip(got, ex):
                assert gv == float(ev) and gl == float(max(el, Fraction(0))), (j, k, got, ex)


@pytest.mark.parametrize("c", [1.0, -1.0, 2.0, -0.5, 0.25])
def test_path_of_a_copy_of_the_preserved_column(c):
    """Column k = c x column jhat: every ratio is c with weight |x_ijhat|, so
    v_k is c until the penalty weight lambda reaches S = ||x_jhat||_1 and 0
    from there on: the path is (0, c), (S, 0) for either sign (at lambda = S
    itself the strict test keeps c > 0 and gives 0 for c < 0, the path's
    breakpoint convention).  Rows with x_ijhat = 0 change nothing."""
    base = np.array([3.0, -1.0, 0.0, 2.0, -4.0, 0.0, 1.0])
    X = np.stack([base, c * base, np.ones(7)], axis=1)
    lam, v = oracle.path(X, 0, 1)
    S = float(np.abs(base).sum())
    assert list(lam) == [0.0, S] and list(v) == [c, 0.0], (lam, v)
    # the column of ones: ratios 1/x_i0 (the sign of x_i0) with weights
    # |x_i0|; with no zero ratio, v_k is 0 exactly when the penalty point's
    # weight outweighs the difference of the two sides: lambda_max = |P - N|
    lam1, v1 = oracle.path(X, 0, 2)
    P, N = base[base > 0].sum(), -base[base < 0].sum()
    assert v1[-1] == 0.0 and lam1[0] == 0.0 and lam1[-1] == abs(P - N), (lam1, v1)
