"""GPU parity of the global-memory path (n beyond the pair kernel's shared
memory, Lemma 1 and Algorithm 1 put no limit on n): every v bit-exact, every s
and z within the bar of tests/_parity.py, against the oracle -- one row past
the shared-memory limit, 50,000 x 8, clusters of several CTAs per pair (n
above 65,536 rows), tie-heavy integers with zero columns, weights that send
pairs to the exact path, forced exact path, subset fits, more lambdas than one
launch holds."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_16712_gb300 import datagen, l1line
from tests._parity import (assert_s_close, assert_v_equal, assert_z_close, check_fit, check_scan,
                           gpu_scan)

pytestmark = pytest.mark.gpu

DT = [np.float32, np.float64]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _planted(n, m, seed, dtype, nnz=2):
    X, _, _ = datagen.planted(datagen.Planted(n, m, nnz, 0.1, 0.1, 5.0, seed,
                                              np.dtype(dtype).name))
    return X


@pytest.mark.parametrize("dtype", DT)
def test_one_row_past_shared_memory(dtype):
    n = l1line.max_rows(dtype) + 1
    X = _planted(n, 5, 78, dtype)
    lams = [0.0, 0.25, 3.0]
    _, _, ref = check_scan(X, lams, where=f"n=max+1={n}")
    check_fit(X, lams, ref, where=f"n=max+1={n}")


@pytest.mark.parametrize("dtype", DT)
def test_50000_by_8(dtype):
    X = _planted(50000, 8, 5, dtype, nnz=3)
    lams = [0.0, 0.5]
    _, _, ref = check_scan(X, lams, where="50000x8")
    check_fit(X, lams, ref, where="50000x8")


@pytest.mark.parametrize("dtype,n", [(np.float32, 300000), (np.float64, 600000)])
def test_cluster_of_several_ctas(dtype, n):
    # 300,000 rows: 5 CTAs per pair; 600,000: the cluster limit of 8
    X = _planted(n, 3, 11, dtype)
    lams = [0.0, 0.1]
    _, _, ref = check_scan(X, lams, where=f"{n}x3")
    check_fit(X, lams, ref, where=f"{n}x3")


@pytest.mark.parametrize("dtype", DT)
def test_integer_ties_zero_columns(dtype):
    n = l1line.max_rows(dtype) + 777
    X = datagen.small_integers(n, 6, seed=4242, dtype=dtype)
    X[:, 2] = 0  # an all-zero column: v = 0 against it, lambda or not
    lams = [0.0, 0.5, 9.0, 1e6]
    _, _, ref = check_scan(X, lams, where="int large")
    check_fit(X, lams, ref, where="int large")


@pytest.mark.parametrize("dtype", DT)
def test_wide_exponents_reach_the_exact_path(dtype):
    # weights over many binades: truncated fixed-point weights leave some
    # decisions to the exact wide-accumulator path
    n = l1line.max_rows(dtype) + 129
    X = datagen.wide_exponents(n, 4, seed=9, dtype=dtype)
    check_scan(X, [0.0, 1e-3], where="wide large")


@pytest.mark.parametrize("dtype", DT)
def test_forced_exact_path(dtype):
    n = l1line.max_rows(dtype) + 5
    X = _planted(n, 4, 3, dtype)
    lams = [0.0, 0.7]
    vg, sg, zg = gpu_scan(X, lams, flags=l1line.FLAG_FORCE_EXACT)
    ref = oracle.fit(X, lams)
    assert_v_equal(vg, ref["v_all"], "forced exact v")
    assert_z_close(X, zg, ref["z_all"], ref["v_all"], "forced exact z")
    assert_s_close(X, sg, ref["s_all"], ref["v_all"], "forced exact s")


@pytest.mark.parametrize("dtype", DT)
def test_subset_fit(dtype):
    n = l1line.max_rows(dtype) + 300
    X = _planted(n, 9, 21, dtype, nnz=3)
    jl = np.array([7, 0, 4, 4], dtype=np.int32)
    lams = [0.0, 0.3]
    Xd = torch.from_numpy(X).cuda()
    v, obj, js, ws = l1line.fit_subset(Xd, lams, torch.from_numpy(jl).cuda())
    assert l1line.status(ws) == l1line.OK
    ref = oracle.fit(X, lams, jlist=jl)
    np.testing.assert_array_equal(js.cpu().numpy(), ref["jstar"])
    assert_v_equal(v.cpu().numpy(), ref["v"], "subset v*")
    np.testing.assert_allclose(obj.cpu().numpy(), ref["obj"],
                               rtol=1e-5 if dtype == np.float32 else 1e-12)


def test_more_lambdas_than_one_launch():
    n = l1line.max_rows(np.float32) + 64
    X = _planted(n, 3, 8, np.float32)
    lams = list(np.linspace(0.0, 4.0, 300))
    _, _, ref = check_scan(X, lams, where="300 lambdas")
    check_fit(X, lams, ref, where="300 lambdas")


def test_bad_jhat_entry_is_reported():
    n = l1line.max_rows(np.float32) + 1
    X = torch.from_numpy(_planted(n, 4, 1, np.float32)).cuda()
    _, _, _, ws = l1line.fit_subset(X, [0.1], torch.tensor([1, 9], dtype=torch.int32,
                                                            device="cuda"))
    assert l1line.status(ws) == l1line.ERR_ARG
