"""The seeded input generators draw the stated distributions: the planted
sparse-line model of datagen.planted (numpy) and its torch twin used for the
learned proposer's training instances (checked here on the CPU device)."""
import numpy as np
import pytest

from paper_2402_16712_gb300 import datagen


def _check_planted(X, v, rows, spec):
    X = np.asarray(X, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    rows = np.asarray(rows)
    n, m = X.shape
    assert (n, m) == (spec.n, spec.m)
    # v*: nnz nonzeros, unit l1 norm
    assert np.count_nonzero(v) == max(1, min(spec.nnz, m))
    assert abs(np.abs(v).sum() - 1.0) < 1e-12
    # outliers: round(frac n) distinct rows with N(0, std^2) entries
    assert rows.size == int(round(spec.outlier_frac * n)) == np.unique(rows).size
    if rows.size:
        o = X[rows]
        assert abs(o.std() / spec.outlier_std - 1.0) < 0.05
        assert abs(o.mean()) < 0.05 * spec.outlier_std
    # clean rows, coordinates outside the support: pure Laplace(0, b) noise,
    # mean |e| = b and var = 2 b^2
    clean = np.setdiff1d(np.arange(n), rows)
    off = np.flatnonzero(v == 0)
    e = X[np.ix_(clean, off)]
    b = spec.noise_b
    assert abs(np.abs(e).mean() / b - 1.0) < 0.03
    assert abs(e.var() / (2 * b * b) - 1.0) < 0.06
    # clean rows on the support: t_i v_j + noise; the projection onto v
    # recovers t ~ N(0, 1) up to the noise
    on = np.flatnonzero(v != 0)
    t = X[np.ix_(clean, on)] @ v[on] / (v[on] @ v[on])
    assert abs(t.std() - 1.0) < 0.25 + 3 * b / np.sqrt(v[on] @ v[on])


@pytest.mark.parametrize("seed", [0, 1])
def test_numpy_planted_distribution(seed):
    spec = datagen.Planted(4000, 60, 5, 0.1, 0.1, 10.0, seed, "float64")
    X, v, rows = datagen.planted(spec)
    _check_planted(X, v, rows, spec)


def test_torch_planted_distribution_and_seeding():
    torch = pytest.importorskip("torch")
    spec = datagen.Planted(4000, 60, 5, 0.1, 0.15, 10.0, 3, "float64")
    X, v, rows = datagen.planted_torch(spec, "cpu")
    _check_planted(X.numpy(), v.numpy(), rows.numpy(), spec)
    X2, _, _ = datagen.planted_torch(spec, "cpu")
    assert torch.equal(X, X2)  # same seed, same draw
    X3, _, _ = datagen.planted_torch(datagen.Planted(4000, 60, 5, 0.1, 0.15, 10.0, 4, "float64"),
                                     "cpu")
    assert not torch.equal(X, X3)


def test_proposer_spec_ranges():
    for seed in range(1, 200):
        s = datagen.proposer_spec(seed)
        assert 500 <= s.n <= 5000 and 100 <= s.m <= 1000
        assert 1 <= s.nnz <= max(1, s.m // 10) and 0.0 <= s.outlier_frac <= 0.2
    s = datagen.proposer_spec(datagen.PROPOSER_HELDOUT_SEED0, n=5000, m=1000)
    assert (s.n, s.m) == (5000, 1000)


def test_comparison_workload_distribution():
    X, v, rows = datagen.comparison(7, 4, n=400, m=60)
    assert abs(np.linalg.norm(v) - 1.0) < 1e-12 and np.all(np.abs(v) <= 1.0)
    assert rows.size == 4
    out = X[rows]
    assert np.all((out[:, :5] > 40) & (out[:, :5] < 110))
    assert np.abs(out[:, 5:]).mean() < 2.0  # Laplace(0, 1) noise only
    clean = np.setdiff1d(np.arange(400), rows)
    # projection on v ~ U(-100, 100); residual noise Laplace(0, 10): mean |e| = 10
    Y = X[clean]
    alpha = Y @ v
    assert abs(alpha.std() - 200 / np.sqrt(12)) < 12
    e = Y - np.outer(alpha, v)
    assert abs(np.abs(e).mean() - 10.0) < 1.0
    assert len(datagen.comparison_suite()) == 30
