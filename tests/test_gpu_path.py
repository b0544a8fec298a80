"""Algorithm 2 on the GPU (l1line_path_count/write): every pair's lambda path
against the oracle (oracle.path), under this bar:
  * path lengths and every value v: identical (bit for bit);
  * breakpoint lambdas: identical when the column's weights are exact in the
    kernel's fixed point (small-integer data), else within 2^-40 of the
    column's l1 norm.
Cases: planted data in both precisions, tie-heavy integers with zero
columns and zero ratios, n = 1 and m = 1, pairs with more rows between v0 and
0 than a warp's list holds, and a sampled check at the 2000 x 2000 size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_16712_gb300 import datagen, l1line

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _gpu_paths(X):
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    off, lam, v, ln, ws = l1line.paths(Xd)
    assert l1line.status(ws) == l1line.OK
    return off.cpu().numpy(), lam.cpu().numpy(), v.cpu().numpy(), ln.cpu().numpy()


def _bits(a):
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def _check_pairs(X, pairs, exact_lambda):
    off, lam, v, ln = _gpu_paths(X)
    m = X.shape[1]
    colnorm = np.abs(X.astype(np.float64)).sum(axis=0)
    for j, k in pairs:
        p = j * m + k
        rl, rv = oracle.path(X, j, k)
        L = int(ln[p])
        assert L == rl.size, (j, k, L, rl.size, rl, rv)
        assert L <= off[p + 1] - off[p]
        gl, gv = lam[off[p]:off[p] + L], v[off[p]:off[p] + L]
        assert np.array_equal(_bits(gv), _bits(rv.astype(X.dtype))), (j, k, gv, rv)
        if exact_lambda:
            assert np.array_equal(gl, rl), (j, k, gl, rl)
        else:
            assert np.all(np.abs(gl - rl) <= 2.0 ** -40 * colnorm[j]), (j, k, gl, rl)


def _all_pairs(m):
    return [(j, k) for j in range(m) for k in range(m)]


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_paths_planted(dtype):
    X, _, _ = datagen.planted(datagen.Planted(300, 17, 4, 0.1, 0.1, 5.0, 4, dtype))
    _check_pairs(X, _all_pairs(17), exact_lambda=False)


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_paths_integer_ties_zero_columns(seed, dtype):
    X = datagen.small_integers(120, 9, seed, lo=-4, hi=4, zero_frac=0.3, dtype=dtype)
    X[:, 3] = 0.0  # an all-zero column
    _check_pairs(X, _all_pairs(9), exact_lambda=True)


def test_paths_degenerate_shapes():
    for X in (np.array([[2.0, -3.0, 5.0]], dtype=np.float32),
              np.array([[1.5], [-2.0], [0.0]], dtype=np.float64)):
        _check_pairs(X, _all_pairs(X.shape[1]), exact_lambda=True)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_paths_longer_than_a_warp_list(dtype):
    # column 1 = 2 x column 0 plus a little noise: v0 ~ 2 and about half the
    # rows lie between 0 and v0, more than a warp's 256-entry list
    rng = np.random.default_rng(9)
    n = 900
    x0 = rng.normal(size=n)
    X = np.stack([x0, 2 * x0 + 0.01 * rng.normal(size=n), rng.normal(size=n)], axis=1)
    X = X.astype(dtype)
    off, lam, v, ln = _gpu_paths(X)
    assert ln[0 * 3 + 1] > 256
    _check_pairs(X, _all_pairs(3), exact_lambda=False)


def test_paths_consistent_with_the_fit_at_a_lambda():
    # the path's value at lambda equals the fit's v^jhat_k at that lambda
    X, _, _ = datagen.planted(datagen.Planted(400, 24, 4, 0.1, 0.1, 10.0, 12, "float32"))
    off, lam, v, ln = _gpu_paths(X)
    m = 24
    for q in (0.05, 0.7, 3.0):
        vf, _, _, ws = l1line.scan(torch.from_numpy(X).cuda(), [q])
        vf = vf.cpu().numpy()[0]
        for p in range(m * m):
            L = int(ln[p])
            gl, gv = lam[off[p]:off[p] + L], v[off[p]:off[p] + L]
            g = np.searchsorted(gl, q, side="left") - 1  # q is never a breakpoint here
            assert gv[g] == vf[p // m, p % m], (p, q)


def test_paths_paper_size_sampled():
    X, _, _ = datagen.paper_size("float32")
    off, lam, v, ln = _gpu_paths(X)
    assert int(off[-1]) >= int(ln.sum()) > 2000 * 2000
    rng = np.random.default_rng(1)
    pairs = [tuple(map(int, x)) for x in rng.integers(0, 2000, size=(40, 2))] + [(5, 5)]
    m = 2000
    colnorm = np.abs(X.astype(np.float64)).sum(axis=0)
    for j, k in pairs:
        p = j * m + k
        rl, rv = oracle.path(X, j, k)
        L = int(ln[p])
        assert L == rl.size
        gl, gv = lam[off[p]:off[p] + L], v[off[p]:off[p] + L]
        assert np.array_equal(_bits(gv), _bits(rv))
        assert np.all(np.abs(gl - rl) <= 2.0 ** -40 * colnorm[j])


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_paths_at_the_largest_row_count(dtype):
    # n = the path kernels' row limit (their staged column and lists fill a CTA's
    # shared memory); one more row is refused
    dt = l1line.DTYPE_F32 if dtype == "float32" else l1line.DTYPE_F64
    n = int(l1line.load().l1line_path_max_rows(dt))
    X, _, _ = datagen.planted(datagen.Planted(n, 3, 1, 0.1, 0.1, 5.0, 17, dtype))
    _check_pairs(X, _all_pairs(3), exact_lambda=False)
    assert l1line.load().l1line_path_workspace_bytes(dt, n + 1, 3) == 0
