"""Seeded synthetic inputs for the l1-regularised l1 best-fit line.

This module only draws random numbers; it holds none of the method's
arithmetic, so both the CUDA path's tests and the CPU oracle's tests can use it.

Planted sparse line model (the workloads' stand-in for the paper's synthetic
studies, Section "Experiments with Synthetic Data"):

    x_i = t_i * v_star + e_i,   t_i ~ N(0, 1),
    v_star: ``nnz`` entries ~ N(0, 1) at seeded positions, divided by their
            l1 norm (unit l1 norm), zeros elsewhere,
    e_i   : i.i.d. Laplace(0, noise_b) per coordinate,
    a seeded subset of round(outlier_frac * n) rows is REPLACED by
    N(0, outlier_std^2 I) outliers.

Rows are the points (n rows, m coordinates), stored row-major.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Planted:
    n: int
    m: int
    nnz: int
    noise_b: float
    outlier_frac: float
    outlier_std: float
    seed: int
    dtype: str = "float32"


def planted(spec: Planted):
    """Return (X, v_star, outlier_rows) for the planted model above."""
    rng = np.random.default_rng(spec.seed)
    n, m = spec.n, spec.m
    nnz = max(1, min(spec.nnz, m))
    v = np.zeros(m)
    pos = rng.choice(m, size=nnz, replace=False)
    v[pos] = rng.standard_normal(nnz)
    s = np.abs(v).sum()
    if s > 0:
        v /= s
    t = rng.standard_normal(n)
    X = np.outer(t, v) + rng.laplace(0.0, spec.noise_b, size=(n, m))
    nout = int(round(spec.outlier_frac * n))
    rows = np.sort(rng.choice(n, size=nout, replace=False)) if nout else np.zeros(0, np.int64)
    if nout:
        X[rows] = rng.normal(0.0, spec.outlier_std, size=(nout, m))
    return np.ascontiguousarray(X.astype(spec.dtype)), v, rows


# ---------------------------------------------------------------------------
# The five workloads (sizes, distributions and lambda choices).
# ---------------------------------------------------------------------------
def one_fit_small(dtype="float64"):
    """n=200 points, m=20, 4-sparse v*, Laplace(0,0.05), 10% N(0,25 I) outliers,
    lambda = 0.1, seed 0."""
    X, v, _ = planted(Planted(200, 20, 4, 0.05, 0.10, 5.0, 0, dtype))
    return X, np.array([0.1]), v


def paper_size(dtype="float32", seed=0, n=2000, m=2000):
    """n = m = 2000 (the paper's 2000x2000 size), 20-sparse v*, Laplace(0,0.1),
    5% N(0,100 I) outlier rows, lambda = 0.5."""
    X, v, _ = planted(Planted(n, m, 20, 0.1, 0.05, 10.0, seed, dtype))
    return X, np.array([0.5]), v


def lambda_path(dtype="float32", seed=0, n=1000, m=500, n_lambda=32):
    """n=1000, m=500, 10-sparse v*, Laplace(0,0.1), 10% N(0,100 I) outliers,
    32 lambdas log-spaced in [1e-3, 10]."""
    X, v, _ = planted(Planted(n, m, 10, 0.1, 0.10, 10.0, seed, dtype))
    return X, np.logspace(-3, 1, n_lambda), v


def uneven_batch(count=256, seed=0, n_range=(100, 5000), m_range=(10, 500), lam=0.2,
                 dtype="float32"):
    """`count` independent instances: n ~ U[100,5000], m ~ U[10,500],
    nnz ~ U[1, max(1, m//10)], outlier fraction ~ U[0, 0.2], Laplace(0,0.1)
    noise, N(0,100 I) outliers, lambda = 0.2 each."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        nnz = int(rng.integers(1, max(1, m // 10) + 1))
        frac = float(rng.uniform(0.0, 0.2))
        X, _, _ = planted(Planted(n, m, nnz, 0.1, frac, 10.0, seed * 100003 + b + 1, dtype))
        out.append((X, np.array([lam])))
    return out


PROPOSER_LAMBDA = 0.2
# Held-out instances of the learned proposer use seeds from here on; training
# instances use seeds 1 .. 20000.
PROPOSER_HELDOUT_SEED0 = 1_000_001


def proposer_spec(seed, n_range=(500, 5000), m_range=(100, 1000), dtype="float32", n=None,
                  m=None) -> Planted:
    """Shape and model parameters of a training / held-out instance of the
    learned proposer: n ~ U[500,5000], m ~ U[100,1000] unless given,
    nnz ~ U[1, m//10], outlier fraction ~ U[0, 0.2], Laplace(0, 0.1) noise,
    N(0, 100 I) outliers; lambda = 0.2."""
    rng = np.random.default_rng(10_000_019 + seed)
    n = int(rng.integers(n_range[0], n_range[1] + 1)) if n is None else n
    m = int(rng.integers(m_range[0], m_range[1] + 1)) if m is None else m
    nnz = int(rng.integers(1, max(1, m // 10) + 1))
    frac = float(rng.uniform(0.0, 0.2))
    return Planted(n, m, nnz, 0.1, frac, 10.0, seed, dtype)


def proposer_instance(seed, n_range=(500, 5000), m_range=(100, 1000), dtype="float32",
                      n=None, m=None):
    """proposer_spec's instance drawn with numpy (host memory)."""
    X, v, _ = planted(proposer_spec(seed, n_range, m_range, dtype, n, m))
    return X, np.array([PROPOSER_LAMBDA]), v


def planted_torch(spec: Planted, device):
    """The planted model of `planted`, drawn on a CUDA device by torch's
    seeded generator (a different random stream from `planted`, same
    distribution), for the learned proposer's many training instances.
    Laplace noise by inversion: -b sgn(u) log(1 - 2|u|), u ~ U[-1/2, 1/2).
    Returns (X, v_star, outlier_rows) as device tensors."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(spec.seed))
    f64 = torch.float64
    n, m = spec.n, spec.m
    nnz = max(1, min(spec.nnz, m))
    pos = torch.randperm(m, generator=g, device=device)[:nnz]
    v = torch.zeros(m, dtype=f64, device=device)
    v[pos] = torch.randn(nnz, generator=g, device=device, dtype=f64)
    v = v / v.abs().sum().clamp_min(1e-300)
    t = torch.randn(n, generator=g, device=device, dtype=f64)
    u = torch.rand((n, m), generator=g, device=device, dtype=f64) - 0.5
    e = -spec.noise_b * torch.sign(u) * torch.log((1.0 - 2.0 * u.abs()).clamp_min(1e-300))
    X = t[:, None] * v[None, :] + e
    nout = int(round(spec.outlier_frac * n))
    rows = torch.sort(torch.randperm(n, generator=g, device=device)[:nout]).values
    if nout:
        X[rows] = torch.randn((nout, m), generator=g, device=device, dtype=f64) * spec.outlier_std
    dt = torch.float32 if spec.dtype == "float32" else torch.float64
    return X.to(dt).contiguous(), v, rows


def comparison(seed, n_outliers, n=100, m=100, dtype="float64"):
    """The paper's comparison-experiment data (Section "Comparison to
    Competing Methods"): v with coordinates ~ U(-10, 10) scaled to unit l2
    norm; each regular point alpha_i v + Laplace(0, 10) noise with alpha_i ~
    U(-100, 100); n_outliers seeded rows are outliers whose first five
    coordinates are ~ U(50, 100), the others 0, plus Laplace(0, 1) noise.
    Returns (X, v, outlier_rows)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-10.0, 10.0, size=m)
    v /= np.sqrt((v * v).sum())
    alpha = rng.uniform(-100.0, 100.0, size=n)
    X = np.outer(alpha, v) + rng.laplace(0.0, 10.0, size=(n, m))
    rows = np.sort(rng.choice(n, size=n_outliers, replace=False))
    out = np.zeros((n_outliers, m))
    out[:, :5] = rng.uniform(50.0, 100.0, size=(n_outliers, 5))
    X[rows] = out + rng.laplace(0.0, 1.0, size=(n_outliers, m))
    return np.ascontiguousarray(X.astype(dtype)), v, rows


def comparison_suite(dtype="float64"):
    """The 30 comparison datasets: five seeds for each outlier count 1..6."""
    return [comparison(1000 * c + s, c, dtype=dtype)[0] for c in range(1, 7) for s in range(5)]


# ---------------------------------------------------------------------------
# Adversarial inputs for parity tests.
# ---------------------------------------------------------------------------
def small_integers(n, m, seed, lo=-4, hi=4, zero_frac=0.2, dtype="float64"):
    """Small integer entries: many exactly tied ratios, zero ratios and zero
    denominators (exact ties exercise the tie rule)."""
    rng = np.random.default_rng(seed)
    X = rng.integers(lo, hi + 1, size=(n, m)).astype(np.float64)
    X[rng.random((n, m)) < zero_frac] = 0.0
    return np.ascontiguousarray(X.astype(dtype))


def wide_exponents(n, m, seed, dtype="float32"):
    """Entries whose magnitudes span many binades (tiny and huge weights in the
    same column), including subnormals for float32."""
    rng = np.random.default_rng(seed)
    if np.dtype(dtype) == np.float32:
        e = rng.integers(-140, 100, size=(n, m))
    else:
        e = rng.integers(-1060, 900, size=(n, m))
    mant = rng.uniform(1.0, 2.0, size=(n, m)) * rng.choice([-1.0, 1.0], size=(n, m))
    X = np.ldexp(mant, e)
    return np.ascontiguousarray(X.astype(dtype))
