"""The float-float residual of double pairs (the pair kernel's residual for
float64 input, step A4): its error bound, checked without a GPU.

The kernel sums |x_ik - v x_ijhat| with every double held as two floats
(x1 = fl(x), x2 = fl(x - x1)) and accepts the sum T_ff only when

    E = 2^-48 (24 C_k + 56 |v| W + (77 + ldn/4096) T_ff) + ldn 2^-146 <= 2^-40 T_ff,

with C_k = sum |x_ik| and W = sum |x_ijhat|; otherwise it sums in double.
This file replays the kernel's float operations exactly (IEEE single
rounding, an exact fused multiply-add, the lanes' row order, blocks of eight
rows, double block sums, the butterfly over 32 lanes) and checks, on exact
rational sums, that |T_ff - T| <= E on random, near-exact, mixed-magnitude
and extreme-v columns, and that an accepted sum is within 9.1e-13 relative.
"""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def rn32(q: Fraction) -> np.float32:
    """Round an exact rational to the nearest float32 (ties to even)."""
    f = F32(float(q))  # within one float32 step of the answer
    best = None
    for c in (np.nextafter(f, F32(-np.inf)), f, np.nextafter(f, F32(np.inf))):
        if not np.isfinite(c):
            continue
        d = abs(Fraction(float(c)) - q)
        if best is None or d < best[0] or (d == best[0] and (int(c.view(np.uint32)) & 1) == 0):
            best = (d, c)
    return F32(best[1])


def fma32(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(x, y):
    s = F32(x + y)
    bb = F32(s - x)
    return s, F32(F32(x - F32(s - bb)) + F32(y - bb))


def ff_row(a1, a2, b1, b2, v1, v2, H, L):
    p1 = F32(v1 * b1)
    e1 = fma32(v1, b1, -p1)
    c = fma32(v1, b2, fma32(v2, b1, e1))
    s, t = two_sum(a1, F32(-p1))
    d = F32(F32(a2 - c) + t)
    if F32(s + d) < 0 or (F32(s + d) == 0 and np.signbit(F32(s + d))):
        s, d = F32(-s), F32(-d)
    h, e = two_sum(H, s)
    return h, F32(L + F32(d + e))


def residual_ff(a, b, v):
    """The kernel's sum over rows padded to a multiple of 128, lane by lane."""
    n = len(a)
    ldn = -(-n // 128) * 128
    A = np.zeros(ldn)
    B = np.zeros(ldn)
    A[:n] = a
    B[:n] = b
    a1 = A.astype(F32)
    a2 = (A - a1.astype(np.float64)).astype(F32)
    b1 = B.astype(F32)
    b2 = (B - b1.astype(np.float64)).astype(F32)
    v1 = F32(v)
    v2 = F32(v - float(v1))
    ng = ldn // 128
    D = np.zeros(32)
    for lane in range(32):
        g = 0
        while g < ng:
            H = L = F32(0.0)
            for gg in range(g, min(g + 2, ng)):
                for r in range(4):
                    i = 128 * gg + 4 * lane + r
                    H, L = ff_row(a1[i], a2[i], b1[i], b2[i], v1, v2, H, L)
            D[lane] = D[lane] + float(H)
            D[lane] = D[lane] + float(L)
            g += 2
    o = 16
    while o:  # butterfly: every lane ends with the same value
        D = np.array([D[ln] + D[ln ^ o] for ln in range(32)])
        o //= 2
    return float(D[0]), ldn


def bound(a, b, v, Tff, ldn):
    Ck = float(np.abs(a).sum())
    W = float(np.abs(b).sum())
    return 2.0 ** -48 * (24 * Ck + 56 * abs(v) * W + (77 + ldn / 4096) * Tff) + ldn * 2.0 ** -146


def exact_T(a, b, v):
    fv = Fraction(v)
    return sum(abs(Fraction(x) - fv * Fraction(y)) for x, y in zip(a.tolist(), b.tolist()))


def cases():
    rng = np.random.default_rng(2402)
    n = 300
    b = rng.standard_normal(n)
    yield "random", rng.standard_normal(n), b, float(rng.standard_normal())
    v = float(rng.standard_normal()) * (1 + 2.0 ** -30)
    yield "near-exact fit", v * b + 1e-9 * rng.standard_normal(n), b, v
    yield "exact fit", v * b, b, v
    mags = np.exp2(rng.integers(-55, 55, n).astype(float))
    yield "mixed magnitudes", rng.standard_normal(n) * mags, rng.standard_normal(n) * mags[::-1], 0.75
    yield "v = 0", rng.standard_normal(n), b, 0.0
    yield "v near 2^59", rng.standard_normal(n) * 2.0 ** 40, b * 2.0 ** -19, 2.0 ** 59 * 1.1
    yield "v near 2^-59", rng.standard_normal(n) * 2.0 ** -40, b * 2.0 ** 19, 2.0 ** -59 * 1.3
    z = rng.standard_normal(n)
    z[::3] = 0.0
    yield "zero rows", z, np.where(np.arange(n) % 5 == 0, 0.0, b), -0.4
    yield "ragged n", rng.standard_normal(133), rng.standard_normal(133), 2.5


@pytest.mark.parametrize("name,a,b,v", list(cases()), ids=[c[0] for c in cases()])
def test_ff_residual_within_bound(name, a, b, v):
    Tff, ldn = residual_ff(a, b, v)
    T = exact_T(a, b, v)
    err = abs(Fraction(Tff) - T)
    E = bound(a, b, v, Tff, ldn)
    assert err <= Fraction(E), (name, float(err), E)
    if E <= 2.0 ** -40 * Tff:  # the kernel keeps T_ff
        assert err <= Fraction(9.1e-13) * T, (name, float(err / T))


def test_certification_rejects_exact_fits_and_keeps_noisy_ones():
    rng = np.random.default_rng(7)
    b = rng.standard_normal(256)
    v = 0.3
    Tff, ldn = residual_ff(v * b, b, v)  # residual 0: only the double sum is trusted
    assert not (bound(v * b, b, v, Tff, ldn) <= 2.0 ** -40 * Tff)
    a = rng.standard_normal(256)
    Tff, ldn = residual_ff(a, b, v)
    assert bound(a, b, v, Tff, ldn) <= 2.0 ** -40 * Tff


def random_cases(count=40, seed=16712):
    """Random columns: n from 1 to 300, magnitudes over +-50 binades per row,
    v from the data's own ratios (a near fit) or random, zero rows, sign mixes."""
    rng = np.random.default_rng(seed)
    for c in range(count):
        n = int(rng.integers(1, 301))
        ea = rng.integers(-50, 51, n) if c % 3 == 0 else np.zeros(n, int)
        eb = rng.integers(-50, 51, n) if c % 4 == 0 else np.zeros(n, int)
        b = rng.standard_normal(n) * np.exp2(eb)
        if c % 2 == 0:  # a near fit: a ~ v b plus noise of random size
            v = float(rng.standard_normal()) * (1 + 2.0 ** -int(rng.integers(20, 50)))
            a = v * b + rng.standard_normal(n) * 10.0 ** float(rng.uniform(-14, 0)) * np.exp2(ea)
        else:
            a = rng.standard_normal(n) * np.exp2(ea)
            v = float(np.median(a / np.where(b == 0, 1, b)))
        a[rng.random(n) < 0.05] = 0.0
        b[rng.random(n) < 0.05] = 0.0
        yield f"random {c}", a, b, v


def test_ff_residual_bound_on_random_columns():
    accepted = 0
    for name, a, b, v in random_cases():
        Tff, ldn = residual_ff(a, b, v)
        T = exact_T(a, b, v)
        err = abs(Fraction(Tff) - T)
        E = bound(a, b, v, Tff, ldn)
        assert err <= Fraction(E), (name, float(err), E)
        if E <= 2.0 ** -40 * Tff:
            accepted += 1
            assert err <= Fraction(9.1e-13) * T, (name, float(err / T))
    assert 5 <= accepted < 40  # both outcomes of the certificate occur


def certified_in_float(Tff, Ck_up, W_up, v, ldn):
    """The kernel's certificate as it evaluates it: float operations, the
    column totals rounded up, |v| from its float rounding, 2^-20 margins."""
    T = F32(Tff)
    if not T < F32(2.0 ** 100):
        return False
    ln = F32(ldn)
    av = abs(F32(v))
    lhs = F32(F32(F32(F32(24.0) * Ck_up) + F32(F32(F32(56.0) * av) * W_up))
              + F32(F32(F32(77.0) + F32(ln * F32(1.0 / 4096.0))) * T))
    lhs = F32(lhs + F32(ln * F32(2.0 ** -98)))
    return bool(F32(lhs * F32(1.0 + 2.0 ** -20)) <= F32(F32(F32(256.0) * T) * F32(1.0 - 2.0 ** -20)))


def round_up32(x: float) -> np.float32:
    f = F32(x)
    return f if float(f) >= x else np.nextafter(f, F32(np.inf))


def test_float_certificate_implies_the_exact_inequality():
    """Whenever the float evaluation accepts, the inequality holds in exact
    arithmetic on the true totals, |v| and T_ff (the margins cover the float
    roundings of the test itself); and it accepts the plainly certifiable."""
    rng = np.random.default_rng(3)
    hits = 0
    for _ in range(20000):
        ldn = int(rng.integers(1, 200)) * 128
        T = float(np.exp2(rng.uniform(-60, 60)))
        Ck = T * float(np.exp2(rng.uniform(-8, 4)))
        W = float(np.exp2(rng.uniform(-60, 60)))
        v = float(rng.choice([-1, 1]) * np.exp2(rng.uniform(-59, 59)))
        ok = certified_in_float(T, round_up32(Ck), round_up32(W), v, ldn)
        exact = (24 * Fraction(Ck) + 56 * abs(Fraction(v)) * Fraction(W)
                 + (77 + Fraction(ldn, 4096)) * Fraction(T) + ldn * Fraction(2) ** -98
                 <= 256 * Fraction(T))
        if ok:
            hits += 1
            assert exact, (T, Ck, W, v, ldn)
    assert hits > 1000
    assert certified_in_float(100.0, round_up32(100.0), round_up32(50.0), 0.01, 2048)
    assert not certified_in_float(0.0, round_up32(100.0), round_up32(50.0), 0.01, 2048)
