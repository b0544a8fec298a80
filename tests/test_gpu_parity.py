"""GPU parity: the CUDA path (through the C ABI) against the oracle, element by
element, on seeded inputs -- the small workload, tie-heavy integer data, zero
columns, ragged and degenerate shapes, weights that force the exact slow path,
lambda batches, and the 2000 x 2000 workload on sampled outputs.  The bar is
stated in tests/_parity.py."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_16712_gb300 import datagen, l1line
from tests._parity import (assert_v_equal, assert_z_close, check_fit, check_scan, gpu_fit,
                           gpu_scan)

pytestmark = pytest.mark.gpu

DT = [np.float32, np.float64]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_one_fit_small_workload():
    X, lams, _ = datagen.one_fit_small("float64")
    _, _, ref = check_scan(X, lams, where="n200m20")
    check_fit(X, lams, ref, where="n200m20")
    X32 = X.astype(np.float32)
    _, _, ref = check_scan(X32, lams, where="n200m20 f32")
    check_fit(X32, lams, ref, where="n200m20 f32")


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n,m", [(1, 3), (5, 4), (31, 6), (32, 5), (33, 7), (100, 9), (257, 12)])
def test_integer_ties_and_zeros(dtype, n, m):
    X = datagen.small_integers(n, m, seed=n * 131 + m, dtype=dtype)
    X[:, m // 2] = 0  # an all-zero column
    lams = [0.0, 0.5, 2.0, 9.0, 1e3]
    _, _, ref = check_scan(X, lams, where=f"int {n}x{m}")
    check_fit(X, lams, ref, where=f"int {n}x{m}")


@pytest.mark.parametrize("dtype", DT)
def test_degenerate_shapes(dtype):
    rng = np.random.default_rng(0)
    for n, m in [(1, 1), (7, 1), (1, 2), (2, 2), (63, 2), (65, 3), (3, 40)]:
        X = rng.standard_normal((n, m)).astype(dtype)
        check_scan(X, [0.0, 0.3], where=f"{n}x{m}")
        check_fit(X, [0.0, 0.3], where=f"{n}x{m}")
    X = np.zeros((10, 3), dtype=dtype)  # everything zero
    check_scan(X, [0.0, 1.0], where="zeros")


@pytest.mark.parametrize("dtype", DT)
def test_force_exact_path_matches(dtype):
    X, _, _ = datagen.planted(datagen.Planted(70, 9, 2, 0.1, 0.1, 5.0, 3, np.dtype(dtype).name))
    lams = [0.0, 0.05, 0.7]
    vg, _, zg = gpu_scan(X, lams, flags=l1line.FLAG_FORCE_EXACT)
    ref = oracle.fit(X, lams)
    assert_v_equal(vg, ref["v_all"], "forced exact")
    assert_z_close(X, zg, ref["z_all"], ref["v_all"], "forced exact")
    Xi = datagen.small_integers(40, 6, 5, dtype=dtype)
    vg, _, _ = gpu_scan(Xi, [0.0, 1.0, 2.5], flags=l1line.FLAG_FORCE_EXACT)
    assert_v_equal(vg, oracle.fit(Xi, [0.0, 1.0, 2.5])["v_all"], "forced exact ints")


@pytest.mark.parametrize("dtype", DT)
def test_wide_exponent_columns(dtype):
    """Weights spanning the whole exponent range: truncated fixed-point
    weights, so the decisions go through the certainty band / exact path."""
    X = datagen.wide_exponents(48, 7, 11, dtype=dtype)
    big = float(np.abs(X.astype(np.float64)).max())
    check_scan(X, [0.0, big * 1e-3, big], where="wide")
    # one tiny entry per column in otherwise ordinary data
    Y, _, _ = datagen.planted(datagen.Planted(90, 8, 2, 0.1, 0.1, 5.0, 9, np.dtype(dtype).name))
    Y[3, :] = np.float32(1e-30) if dtype == np.float32 else 1e-200
    check_scan(Y, [0.0, 0.2], where="tiny entries")


@pytest.mark.parametrize("cluster", [12, 31, 32, 200])
def test_double_ratios_equal_in_float(cluster):
    """Double input whose median lies among ratios that differ in double but
    round to one float (one coarse key): up to 31 such rows are decided on
    their 64-bit keys in the final step, more go to the 64-bit selection."""
    rng = np.random.default_rng(cluster)
    n, m = 400, 5
    X = rng.standard_normal((n, m))
    # column 0 / column 1 = 1 + i 2^-45 on the cluster rows: distinct doubles,
    # one float; those rows carry most of the weight of column 1
    rows = rng.choice(n, size=cluster, replace=False)
    X[rows, 1] = 50.0 + rng.random(cluster)
    X[rows, 0] = X[rows, 1] * (1.0 + np.arange(cluster) * 2.0 ** -45)
    X[rows, 2] = -X[rows, 1] * (3.0 - np.arange(cluster)[::-1] * 2.0 ** -44)
    _, _, ref = check_scan(X, [0.0, 0.5, 40.0], where=f"coarse ties {cluster}")
    check_fit(X, [0.0, 0.5, 40.0], ref, where=f"coarse ties {cluster}")


@pytest.mark.parametrize("outliers", [False, True])
@pytest.mark.parametrize("noise", [0.0, 1e-13, 1e-9, 1e-3])
def test_double_near_exact_fits(noise, outliers):
    """Double columns that are (nearly) multiples of one another.  Without
    outlier rows the residuals lie far below the columns' size, where the
    float-float residual's error bound (~2^-48 of the columns) cannot be
    certified, so the pairs are summed again in double; with outliers most
    are certified.  Either way every s meets the 1e-12 bar term by term."""
    rng = np.random.default_rng(int(noise * 1e15) % 1000 + (7 if outliers else 3))
    n, m = 300, 6
    base = rng.standard_normal(n)
    scale = rng.standard_normal(m) * (1 + 2.0 ** -30)
    X = base[:, None] * scale[None, :] + noise * rng.standard_normal((n, m))
    if outliers:
        X[rng.choice(n, 15, replace=False)] += rng.standard_normal((15, m)) * 5
    where = f"near-exact {noise} outliers={outliers}"
    _, _, ref = check_scan(X, [0.0, 0.1], where=where)
    check_fit(X, [0.0, 0.1], ref, where=where)


@pytest.mark.parametrize("dtype", DT)
def test_lambda_batch(dtype):
    X, lams, _ = datagen.lambda_path(np.dtype(dtype).name, n=300, m=24, n_lambda=40)
    _, _, ref = check_scan(X, lams, where="lambda batch")
    check_fit(X, lams, ref, where="lambda batch")


def test_more_lambdas_than_one_launch():
    X, _, _ = datagen.planted(datagen.Planted(64, 5, 2, 0.1, 0.1, 5.0, 4, "float32"))
    lams = np.linspace(0.0, 3.0, 300)
    check_scan(X, lams, where="300 lambdas")


@pytest.mark.parametrize("dtype", DT)
def test_large_lambda_closed_form(dtype):
    X, _, _ = datagen.planted(datagen.Planted(120, 10, 3, 0.1, 0.1, 5.0, 6, np.dtype(dtype).name))
    col = np.abs(X.astype(np.float64)).sum(axis=0)
    lam = float(col.max()) * 1.01
    v, obj, js = gpu_fit(X, [lam])
    assert int(js[0]) == int(np.argmax(col))
    assert np.array_equal(v[0], np.eye(10, dtype=dtype)[int(js[0])])
    want = np.abs(X.astype(np.float64)).sum() - col.max() + lam
    assert abs(obj[0] - want) <= 1e-5 * want


def test_nonfinite_input_reported():
    X = np.ones((16, 4), dtype=np.float32)
    X[3, 2] = np.nan
    Xd = torch.from_numpy(X).cuda()
    _, _, _, ws = l1line.fit(Xd, [0.1])
    assert l1line.status(ws) == l1line.ERR_NONFINITE
    X[3, 2] = np.inf
    _, _, _, ws = l1line.fit(torch.from_numpy(X).cuda(), [0.1])
    assert l1line.status(ws) == l1line.ERR_NONFINITE
    # the next clean call on the same workspace reports ok again
    X[3, 2] = 1.0
    l1line.fit(torch.from_numpy(X).cuda(), [0.1], workspace=ws)
    assert l1line.status(ws) == l1line.OK


def test_workspace_reuse_and_stream():
    ws = l1line.Workspace.for_shape(np.float64, 300, 30, 2)
    s = torch.cuda.Stream()
    for seed in range(3):
        X, _, _ = datagen.planted(datagen.Planted(300 - 7 * seed, 30 - seed, 3, 0.1, 0.1, 5.0,
                                                  seed, "float64"))
        with torch.cuda.stream(s):
            Xd = torch.from_numpy(X).cuda()
            v, obj, js, _ = l1line.fit(Xd, [0.0, 0.4], workspace=ws, stream=s)
        assert l1line.status(ws, s) == l1line.OK
        ref = oracle.fit(X, [0.0, 0.4])
        for t in range(2):
            assert_v_equal(v[t].cpu().numpy(), ref["v_all"][t, int(js[t])], f"reuse {seed}")


@pytest.mark.parametrize("dtype", DT)
def test_paper_size_sampled(dtype):
    """n = m = 2000 (the paper's size, lambda = 0.5): the launch the bench
    times.  The oracle recomputes sampled jhat rows one by one."""
    X, lams, _ = datagen.paper_size(np.dtype(dtype).name)
    vg, _, zg = gpu_scan(X, lams)
    v, obj, js = gpu_fit(X, lams)
    js0 = int(js[0])
    assert js0 == int(np.argmin(zg[0]))  # fit == argmin of the scan's z
    rng = np.random.default_rng(1)
    sample = sorted({js0, 0, 1, 1999, *rng.choice(2000, 4, replace=False).tolist()})
    ref = oracle.fit(X, lams, jlist=sample)
    for j in sample:
        assert_v_equal(vg[0, j], ref["v_all"][0, j], f"2000^2 row {j}")
    zs = zg[:, sample]
    assert_z_close(X, zs, ref["z_all"][:, sample], ref["v_all"][:, sample], "2000^2 z",
                   cols=sample)
    assert_v_equal(v[0], ref["v_all"][0, js0], "2000^2 v*")
    assert abs(obj[0] - ref["z_all"][0, js0]) <= (1e-5 if dtype == np.float32 else 1e-12) * obj[0]
    # the GPU's jhat* is no worse than any sampled jhat under the oracle's z
    assert ref["z_all"][0, js0] <= np.nanmin(ref["z_all"][0, sample]) * (1 + 1e-5)


@pytest.mark.parametrize("dtype", DT)
def test_lambda_batch_unsorted_and_repeated(dtype):
    """Lambdas in arbitrary order, with repeats: results follow the caller's order."""
    X, _, _ = datagen.planted(datagen.Planted(257, 15, 3, 0.1, 0.1, 5.0, 8, np.dtype(dtype).name))
    rng = np.random.default_rng(2)
    lams = rng.permutation(np.concatenate([np.logspace(-3, 1.5, 12), [0.0, 0.3, 0.3]]))
    _, _, ref = check_scan(X, lams, where="unsorted lambdas")
    check_fit(X, lams, ref, where="unsorted lambdas")


@pytest.mark.parametrize("dtype", DT)
@pytest.mark.parametrize("n", [127, 128, 129, 255, 385])
def test_row_padding_boundaries(dtype, n):
    # the staged rows are padded to a multiple of 128; counts around it
    X, _, _ = datagen.planted(datagen.Planted(n, 11, 3, 0.1, 0.1, 5.0, n, np.dtype(dtype).name))
    _, _, ref = check_scan(X, [0.0, 0.4, 3.0], where=f"n={n}")
    check_fit(X, [0.0, 0.4, 3.0], ref, where=f"n={n}")


@pytest.mark.parametrize("dtype", DT)
def test_largest_supported_row_count(dtype):
    # n at the pair kernel's limit (shared memory), a few columns: every pair
    # against the oracle (one row more takes the global-memory path,
    # tests/test_gpu_large.py)
    n = l1line.max_rows(dtype)
    X, _, _ = datagen.planted(datagen.Planted(n, 5, 2, 0.1, 0.1, 5.0, 77, np.dtype(dtype).name))
    _, _, ref = check_scan(X, [0.0, 0.25], where=f"n=max={n}")
    check_fit(X, [0.0, 0.25], ref, where=f"n=max={n}")
