"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- exact rational brute force, the paper's printed toy example, the
Lemma 1 dual certificate, closed forms and invariances.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2402_16712_gb300 import datagen
from tests import _exact as ex

GOLD = os.path.join(os.path.dirname(__file__), "golden", "toy_example.json")


def fl(q: Fraction, dtype):
    """Round an exact rational to the given float type (single rounding)."""
    if dtype == np.float64:
        return np.float64(q.numerator / q.denominator) if q else np.float64(0.0)
    # float32: round the exact rational directly (avoids double rounding)
    if q == 0:
        return np.float32(0.0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    ulp = Fraction(2) ** (e - 23)
    k = a / ulp
    fk = math.floor(k)
    rem = k - fk
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fk % 2 == 1):
        fk += 1
    return np.float32(s * float(fk * ulp))


# ---------------------------------------------------------------------------
# Exact accumulator
# ---------------------------------------------------------------------------
def test_exact_sign_of_sum_matches_rational_sum():
    rng = np.random.default_rng(1)
    for trial in range(400):
        cnt = int(rng.integers(1, 40))
        e = rng.integers(-1074, 1000, size=cnt)
        vals = np.ldexp(rng.uniform(-2, 2, size=cnt), e)
        if trial % 3 == 0:  # force near-cancellation: append the negated rounded sum
            vals = np.append(vals, -math.fsum(vals))
        exact = sum(Fraction(float(x)) for x in vals)
        assert oracle.sign_of_sum(vals) == (exact > 0) - (exact < 0)
    tiny = 5e-324
    assert oracle.sign_of_sum([1e308, -1e308, tiny]) == 1
    assert oracle.sign_of_sum([1e308, 1e308, -1e308, -1e308]) == 0
    assert oracle.sign_of_sum([tiny, tiny, -2 * tiny]) == 0
    assert oracle.sign_of_sum([-tiny]) == -1


# ---------------------------------------------------------------------------
# Lemma 1 / Algorithm 1, one pair at a time, against exact brute force
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pair_matches_bruteforce_right_endpoint(dtype):
    rng = np.random.default_rng(2)
    lams = [0.0, 0.5, 1.0, 2.0, 3.0, 7.0, 0.1, 100.0]
    for trial in range(300):
        n = int(rng.integers(1, 11))
        a = rng.integers(-5, 6, size=n).astype(dtype)
        b = rng.integers(-5, 6, size=n).astype(dtype)
        if trial % 5 == 0:
            b[:] = 0
        lam = lams[trial % len(lams)]
        _, t = ex.pair_right_endpoint(a, b, lam)
        got = oracle.pair(a, b, lam)
        want = fl(t, dtype)
        assert got == want and math.copysign(1, got) == math.copysign(1, want), (a, b, lam)


def test_alg1_literal_scan_equals_right_endpoint_rule():
    """The reading of Algorithm 1's half-open test with 'last index wins' is the
    right end point of the minimiser interval, for every order of tied ratios."""
    rng = np.random.default_rng(3)
    for trial in range(2000):
        n = int(rng.integers(1, 9))
        a = rng.integers(-3, 4, size=n).astype(float)
        b = rng.integers(-3, 4, size=n).astype(float)
        lam = float(rng.choice([0, 0.5, 1, 2, 3, 4, 6]))
        order = list(rng.permutation(n))
        _, t = ex.pair_right_endpoint(a, b, lam)
        assert ex.alg1_literal(a, b, lam, order) == t, (a, b, lam, order)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pair_dual_certificate_random_floats(dtype):
    """Lemma 1's dual construction certifies the oracle's choice as optimal."""
    rng = np.random.default_rng(4)
    for trial in range(200):
        n = int(rng.integers(1, 30))
        a = rng.standard_normal(n).astype(dtype)
        b = rng.standard_normal(n).astype(dtype)
        b[rng.random(n) < 0.1] = 0
        lam = float(rng.choice([0.0, 0.05, 0.3, 1.0, 5.0]))
        v = oracle.pair(a, b, lam)
        if v == 0:
            t = Fraction(0)
        else:
            # the exact ratio whose rounding the oracle returned
            cands = [Fraction(float(ai)) / Fraction(float(bi)) for ai, bi in zip(a, b)
                     if bi != 0 and (a.dtype.type(ai) / a.dtype.type(bi)) == v]
            assert cands, (a, b, v)
            t = max(cands)
        assert ex.dual_certificate_ok(a, b, lam, t)


# ---------------------------------------------------------------------------
# Whole fit: toy example printed in the paper
# ---------------------------------------------------------------------------
def _tol(s: str) -> float:
    # one unit in the last printed place: the paper both rounds (2.17) and
    # truncates (37.66666 for 113/3) its printed values
    return 10.0 ** (-(len(s.split(".")[1]) if "." in s else 0))


def test_toy_example_exact_values_match_paper_figure_and_table():
    g = json.load(open(GOLD))
    X = np.array(g["points"], dtype=np.float64)
    for ln in g["figure1_lines"]:
        lam = Fraction(ln["from"] + ln["to"], 2)
        zs, _ = ex.fit_exact(X, float(lam))
        z = zs[ln["jhat"] - 1]
        pred = float(ln["intercept"]) + float(ln["slope"]) * float(lam)
        tol = _tol(ln["intercept"]) + _tol(ln["slope"]) * float(lam) + 1e-12
        assert abs(float(z) - pred) <= tol, (ln, float(z))
    for row in g["table1"]:
        hi = row["to"] if row["to"] is not None else row["from"] + 5
        lam = (row["from"] + hi) / 2
        zs, vs = ex.fit_exact(X, lam)
        jb = min(range(len(zs)), key=lambda j: (zs[j], j))
        assert jb + 1 == row["jhat"]
        for got, s in zip(vs[jb], row["v"]):
            want = Fraction(s) if "/" in s else float(s)
            tol = 0 if "/" in s else _tol(s)
            assert abs(float(got) - float(want)) <= tol + 1e-12, (row, vs[jb])
        for key, lam_end in (("z_from", row["from"]), ("z_to", row["to"])):
            if row[key] is None:
                continue
            zs_end, _ = ex.fit_exact(X, lam_end)
            zstar = float(min(zs_end))
            tol = _tol(row[key])
            if row.get("inconsistent_with_figure") == key:
                tol = 0.1 + 1e-12  # printed 42.9; the figure's lines give 43.0
            assert abs(zstar - float(row[key])) <= tol, (row, key, zstar)
    # crossing at 3.5: z_1 == z_4 exactly, the tie goes to the smaller jhat
    zs, _ = ex.fit_exact(X, 3.5)
    assert zs[0] == zs[3] == 43
    # beyond lambda max every v^jhat is the unit vector e_jhat
    for lam in (g["lambda_max"], g["lambda_max"] + 7.25):
        _, vs = ex.fit_exact(X, lam)
        for j, v in enumerate(vs):
            assert v == [Fraction(int(k == j)) for k in range(4)]
    _, vs = ex.fit_exact(X, g["lambda_max"] - 0.01)
    assert any(vs[j] != [Fraction(int(k == j)) for k in range(4)] for j in range(4))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_oracle_on_toy_equals_exact(dtype):
    g = json.load(open(GOLD))
    X = np.array(g["points"], dtype=dtype)
    lams = [0.0, 0.5, 1.0, 2.0, 3.0, 3.25, 3.5, 4.0, 5.0, 6.0, 10.9, 11.0, 20.0]
    r = oracle.fit(X, lams)
    for t, lam in enumerate(lams):
        zs, vs = ex.fit_exact(X, lam)
        for j in range(4):
            # exact objective at the oracle's (rounded) v
            zr = ex.objective_at(X, j, r["v_all"][t, j], lam)
            assert abs(r["z_all"][t, j] - float(zr)) <= 1e-14 * float(zr)
            if dtype == np.float64:
                assert abs(r["z_all"][t, j] - float(zs[j])) <= 1e-13 * float(zs[j])
            for k in range(4):
                assert r["v_all"][t, j, k] == fl(vs[j][k], dtype)
        jb = min(range(4), key=lambda j: (zs[j], j))
        assert r["jstar"][t] == jb
    t35 = lams.index(3.5)
    assert r["jstar"][t35] == 0  # tie z_1 = z_4 = 43 resolved to the smaller jhat


# ---------------------------------------------------------------------------
# Whole fit: brute force on tiny random inputs, closed forms, invariances
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_fit_matches_exact_on_tiny_integer_data(dtype):
    for seed in range(25):
        rng = np.random.default_rng(100 + seed)
        n, m = int(rng.integers(1, 7)), int(rng.integers(1, 5))
        X = datagen.small_integers(n, m, seed, dtype=dtype)
        lams = [0.0, 0.5, 2.0, 9.0]
        r = oracle.fit(X, lams)
        for t, lam in enumerate(lams):
            zs, vs = ex.fit_exact(X, lam)
            zr = []
            for j in range(m):
                zr.append(ex.objective_at(X, j, r["v_all"][t, j], lam))
                assert abs(r["z_all"][t, j] - float(zr[j])) <= 1e-14 * max(1.0, float(zr[j]))
                assert [r["v_all"][t, j, k] for k in range(m)] == [fl(q, dtype) for q in vs[j]]
            # argmin: exact objective at the rounded v is minimal up to rounding of z
            js = int(r["jstar"][t])
            scale = float(np.abs(X.astype(np.float64)).sum()) * 2 * m
            assert float(zr[js]) - float(min(zr)) <= 1e-14 * (float(min(zr)) + scale)
            assert js == min(j for j in range(m) if r["z_all"][t, j] == r["z_all"][t].min())
            assert np.array_equal(r["v"][t], r["v_all"][t, js])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_objective_against_exact_recomputation(dtype):
    X, _, _ = datagen.planted(datagen.Planted(40, 6, 2, 0.1, 0.1, 5.0, 7, np.dtype(dtype).name))
    lam = 0.3
    r = oracle.fit(X, [lam])
    for j in range(6):
        v = [Fraction(float(x)) for x in r["v_all"][0, j]]
        z = sum(abs(ex.fr(X[i, k]) - v[k] * ex.fr(X[i, j])) for i in range(40) for k in range(6))
        z += ex.fr(lam) * sum(abs(x) for x in v)
        if dtype == np.float32:  # products exact in double: one rounding per term
            assert abs(r["z_all"][0, j] - float(z)) <= 1e-14 * float(z)
        else:
            assert abs(r["z_all"][0, j] - float(z)) <= 1e-13 * float(z)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_large_lambda_closed_form(dtype):
    X, _, _ = datagen.planted(datagen.Planted(50, 9, 3, 0.1, 0.1, 5.0, 11, np.dtype(dtype).name))
    col = np.abs(X.astype(np.float64)).sum(axis=0)
    lam = float(col.max()) * 1.0001
    r = oracle.fit(X, [lam, 1e6])
    for t, L in enumerate([lam, 1e6]):
        js = int(np.argmax(col))
        assert r["jstar"][t] == js
        assert np.array_equal(r["v"][t], np.eye(9, dtype=dtype)[js])
        want = math.fsum(np.abs(X.astype(np.float64)).ravel()) - col[js] + L
        assert abs(r["obj"][t] - want) <= 1e-12 * want



LAMBDA_GRID = [0.0, 0.05, 0.3, 1.0, 2.5, 7.0, 40.0, 1e4]


def _sandwich(z_all, v_all, lams):
    """Largest violation, over jhat and lambda pairs, of the two bounds that
    make z_jhat(lambda) = min_v [sum_ik |x_ik - v_k x_ijhat| + lambda ||v||_1]
    concave in lambda with supergradient ||v(lambda)||_1 (the objective of
    Algorithm 1 per jhat; v_jhat = 1 is part of ||v||_1):
        z(b) <= z(a) + (b - a) ||v(a)||_1    (v(a) is feasible at b)
        z(b) >= z(a) + (b - a) ||v(b)||_1    (v(b) is feasible at a)
    in units of the objective's scale."""
    P = np.abs(v_all.astype(np.float64)).sum(axis=2)  # [lambda, jhat]
    worst = 0.0
    for a in range(len(lams)):
        for b in range(a + 1, len(lams)):
            d = lams[b] - lams[a]
            scale = np.abs(z_all[a]) + np.abs(z_all[b]) + d * (P[a] + P[b])
            up = z_all[b] - (z_all[a] + d * P[a])
            lo = (z_all[a] + d * P[b]) - z_all[b]
            worst = max(worst, float(np.max(np.maximum(up, lo) / scale)))
    return worst


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_objective_is_concave_in_lambda_with_norm_supergradient(dtype):
    """Per jhat, the oracle's z and v over a lambda grid satisfy both
    feasibility bounds above (Lemma 1 optimality per k, the penalty term and
    v_jhat = 1 of the objective all enter), ||v||_1 never grows with lambda,
    and no z exceeds that of v = e_jhat, feasible at every lambda:
    sum_{k != jhat} ||x_k||_1 + lambda."""
    X, _, _ = datagen.planted(datagen.Planted(40, 7, 3, 0.1, 0.15, 5.0, 23,
                                              np.dtype(dtype).name))
    r = oracle.fit(X, LAMBDA_GRID)
    m = X.shape[1]
    assert np.array_equal(r["v_all"][:, np.arange(m), np.arange(m)], np.ones((len(LAMBDA_GRID), m)))
    assert _sandwich(r["z_all"], r["v_all"], LAMBDA_GRID) <= 1e-12
    P = np.abs(r["v_all"].astype(np.float64)).sum(axis=2)
    assert (np.diff(P, axis=0) <= 1e-12 * P[:-1]).all()
    col = np.abs(X.astype(np.float64)).sum(axis=0)
    for t, lam in enumerate(LAMBDA_GRID):
        e_obj = col.sum() - col + lam
        assert (r["z_all"][t] <= e_obj * (1 + 1e-12)).all(), (lam, r["z_all"][t] - e_obj)


def test_copies_of_the_preserved_column_closed_form():
    """Columns k that are c times column jhat have every ratio equal to c with
    weight |x_ijhat|, plus the penalty point (0, lambda).  With S = ||x_jhat||_1
    the weighted median's right end point is c while lambda <= S when c > 0
    (the cumulative weight at 0 is lambda, at most half of S + lambda), but
    only while lambda < S when c < 0 (at lambda = S the cumulative weight at c
    is exactly half, so the scan moves on to 0): Lemma 1's strict test."""
    base = np.array([3.0, -1.0, 0.0, 2.0, -4.0, 0.0, 1.0])
    other = np.array([1.0, 2.0, -3.0, 0.0, 5.0, -1.0, 2.0])
    X = np.stack([base, base, -base, 2.0 * base, -0.5 * base, other], axis=1)
    S = float(np.abs(base).sum())
    lams = [0.0, S - 0.5, S, S + 0.5]
    r = oracle.fit(X, lams)
    for t, lam in enumerate(lams):
        v = r["v_all"][t, 0]
        assert v[0] == 1.0
        assert v[1] == (1.0 if lam <= S else 0.0), (lam, v)
        assert v[2] == (-1.0 if lam < S else 0.0), (lam, v)
        assert v[3] == (2.0 if lam <= S else 0.0), (lam, v)
        assert v[4] == (-0.5 if lam < S else 0.0), (lam, v)

def test_single_coordinate_and_zero_column():
    X = np.array([[1.5], [-2.0], [0.25]])
    r = oracle.fit(X, [0.0, 0.7])
    assert list(r["obj"]) == [0.0, 0.7] and list(r["v"][:, 0]) == [1.0, 1.0]
    # a column of zeros: Algorithm 1 keeps v = e_jhat and z = sum|x| + lambda
    X = np.array([[1.0, 0.0, 2.0], [-3.0, 0.0, 1.0], [0.5, 0.0, -1.0]])
    for lam in (0.0, 0.4):
        r = oracle.fit(X, [lam])
        assert np.array_equal(r["v_all"][0, 1], [0.0, 1.0, 0.0])
        assert r["z_all"][0, 1] == np.abs(X).sum() + lam


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_invariances(dtype):
    X, _, _ = datagen.planted(datagen.Planted(60, 8, 3, 0.1, 0.1, 5.0, 5, np.dtype(dtype).name))
    lams = [0.0, 0.2, 2.0]
    base = oracle.fit(X, lams)
    rng = np.random.default_rng(0)
    # row sign flips: ratios and weights unchanged -> bit-identical
    S = X * rng.choice([-1, 1], size=(60, 1)).astype(dtype)
    r = oracle.fit(S, lams)
    assert np.array_equal(r["v_all"], base["v_all"]) and np.array_equal(r["z_all"], base["z_all"])
    # row permutation: v bit-identical (exact decisions), z to rounding
    P = X[rng.permutation(60)]
    r = oracle.fit(P, lams)
    assert np.array_equal(r["v_all"], base["v_all"])
    np.testing.assert_allclose(r["z_all"], base["z_all"], rtol=1e-14)
    # power-of-two scaling of X and lambda: v identical, z scaled exactly
    for p in (-7, 5):
        s = dtype(2.0 ** p)
        r = oracle.fit(X * s, [L * 2.0 ** p for L in lams])
        assert np.array_equal(r["v_all"], base["v_all"])
        assert np.array_equal(r["z_all"], base["z_all"] * 2.0 ** p)
    # column permutation permutes jhat and v
    q = rng.permutation(8)
    r = oracle.fit(np.ascontiguousarray(X[:, q]), lams)
    for t in range(len(lams)):
        for jn in range(8):
            assert np.array_equal(r["v_all"][t, jn], base["v_all"][t, q[jn]][q])
            np.testing.assert_allclose(r["z_all"][t, jn], base["z_all"][t, q[jn]], rtol=1e-14)


def test_lambda_zero_is_unregularised_fit():
    """lambda = 0 gives the plain l1 best-fit line of the sort method: every
    pair is the unweighted-penalty weighted median (brute force with lam = 0)."""
    X = datagen.small_integers(7, 4, 99, lo=-6, hi=6, zero_frac=0.1)
    r = oracle.fit(X, [0.0])
    zs, vs = ex.fit_exact(X, 0.0)
    for j in range(4):
        assert [Fraction(float(x)) for x in r["v_all"][0, j]] == [
            Fraction(float(np.float64(q.numerator / q.denominator))) for q in vs[j]]


def test_wide_exponent_columns_exact():
    """Weights spanning the whole float range (subnormals included): decisions
    stay exact (checked against exact brute force)."""
    for dtype in (np.float32, np.float64):
        X = datagen.wide_exponents(6, 3, 21, dtype=dtype)
        for lam in (0.0, float(np.abs(X).max()) * 1e-3):
            r = oracle.fit(X, [lam])
            for j in range(3):
                for k in range(3):
                    if k == j:
                        continue
                    _, t = ex.pair_right_endpoint(X[:, k], X[:, j], lam)
                    # t is an exact ratio; compare the rounded value
                    want = fl(t, dtype) if t else dtype(0)
                    assert r["v_all"][0, j, k] == want


def test_argument_errors():
    X = np.ones((3, 2))
    with pytest.raises(oracle.OracleError):
        oracle.fit(X, [-1.0])
    with pytest.raises(oracle.OracleError):
        oracle.fit(X, [float("inf")])
    Y = X.copy()
    Y[1, 1] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.fit(Y, [0.1])
