"""Batched fit (one persistent pair launch per size class over uneven
instances): every instance's result against the oracle, under the parity bar
of tests/_parity.py; graph capture and replay; degenerate instances; every
number of size classes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_16712_gb300 import datagen, l1line
from tests._parity import assert_v_equal, tolerances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _instances(dtype, count, seed):
    rng = np.random.default_rng(seed)
    Xs, lams = [], []
    for b in range(count):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(1, 30))
        kind = b % 4
        if kind == 3:
            X = datagen.small_integers(n, m, seed + b, dtype=dtype)
        else:
            X, _, _ = datagen.planted(datagen.Planted(n, m, max(1, m // 5), 0.1, 0.1, 5.0,
                                                      seed * 1000 + b, np.dtype(dtype).name))
        nl = int(rng.integers(1, 5))
        Xs.append(X)
        lams.append(np.sort(rng.choice([0.0, 0.05, 0.2, 0.7, 3.0], size=nl, replace=False)))
    return Xs, lams


def _check(Xs, lams, results, where):
    for b, (X, lam) in enumerate(zip(Xs, lams)):
        v, obj, js = (t.cpu().numpy() for t in results[b])
        ref = oracle.fit(X, lam)
        rtol, atol = tolerances(X, ref["v_all"])
        for t in range(len(lam)):
            jg, jr = int(js[t]), int(ref["jstar"][t])
            if jg != jr:
                zr = ref["z_all"][t]
                assert abs(zr[jg] - zr[jr]) <= rtol * abs(zr[jr]) + atol[t, jg] + atol[t, jr], \
                    (where, b, t, jg, jr)
            assert_v_equal(v[t], ref["v_all"][t, jg], f"{where} inst {b} lambda {t}")
            lim = rtol * abs(ref["z_all"][t, jg]) + atol[t, jg]
            assert abs(obj[t] - ref["z_all"][t, jg]) <= lim, (where, b, t)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batched_matches_oracle(dtype):
    Xs, lams = _instances(dtype, 24, 5)
    Xs[0] = np.zeros((7, 3), dtype=dtype)   # all-zero instance
    Xs[1] = Xs[1][:, :1].copy()             # m = 1
    Xs[2] = Xs[2][:1].copy()                # n = 1
    bat = l1line.Batched([torch.from_numpy(np.ascontiguousarray(X)).cuda() for X in Xs], lams)
    bat.run()
    assert bat.status() == l1line.OK
    _check(Xs, lams, bat.results(), "batched")
    assert l1line.last_launch_count() == 6


def test_batched_graph_replay():
    Xs, lams = _instances(np.float32, 16, 11)
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    bat = l1line.Batched(Xd, lams)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bat.run(s)  # warm-up: sets kernel attributes outside the capture
    torch.cuda.synchronize()
    first = [tuple(t.clone() for t in r) for r in bat.results()]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bat.run()
    for X in Xd:  # replay on new data of the same shapes: every row sign-flipped
        X.neg_()
    g.replay()
    torch.cuda.synchronize()
    assert bat.status() == l1line.OK
    # a sign flip of every row leaves ratios, weights and residual terms unchanged
    for (v0, o0, j0), (v1, o1, j1) in zip(first, bat.results()):
        assert torch.equal(j0, j1) and torch.equal(v0, v1) and torch.equal(o0, o1)
    Xs2 = [X.cpu().numpy() for X in Xd]
    _check(Xs2, lams, bat.results(), "graph replay")


def test_comparison_suite_batched():
    # the paper's comparison experiment data (30 datasets of 100 x 100), a
    # sparsity sweep of 8 lambdas each, in one batched call
    Xs = datagen.comparison_suite("float64")
    lams = [np.array([0.0, 5.0, 20.0, 50.0, 100.0, 200.0, 400.0, 800.0])] * len(Xs)
    bat = l1line.Batched([torch.from_numpy(X).cuda() for X in Xs], [l.copy() for l in lams])
    bat.run()
    assert bat.status() == l1line.OK
    _check(Xs, lams, bat.results(), "comparison suite")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_size_classes_give_identical_results(dtype):
    """Instances with n from 60 to 5000 (each shared-memory plan of the pair
    kernel occurs) under every number of size classes: each run matches the
    oracle and the runs agree bit for bit."""
    rng = np.random.default_rng(77)
    Xs, lams = [], []
    for b, n in enumerate((5000, 60, 4700, 700, 3600, 1800, 2600, 130, 4100, 2200, 999, 3100)):
        m = int(rng.integers(2, 20))
        X, _, _ = datagen.planted(datagen.Planted(n, m, max(1, m // 5), 0.1, 0.15, 10.0,
                                                  5000 + b, np.dtype(dtype).name))
        Xs.append(X)
        lams.append(np.array([0.0, 0.2, 1.5]))
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    runs = []
    for k in (0, 1, 2, 3):
        l1line.set_tuning({"batch_classes": k})
        try:
            bat = l1line.Batched(Xd, lams)
            bat.run()
            if k > 0:  # staging 2, one pair launch per class, exact path, sums, argmin
                assert l1line.last_launch_count() == 5 + k
            assert bat.status() == l1line.OK
            runs.append([tuple(t.clone() for t in r) for r in bat.results()])
        finally:
            l1line.set_tuning(None)
    _check(Xs, lams, runs[1], "batch_classes=1")
    ib = torch.int32 if dtype == np.float32 else torch.int64
    for k, r in enumerate(runs):
        for b, (a, c) in enumerate(zip(runs[1], r)):
            assert torch.equal(a[0].view(ib), c[0].view(ib)), (k, b)
            assert torch.equal(a[1], c[1]) and torch.equal(a[2], c[2]), (k, b)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_every_launch_shape_gives_identical_results(dtype):
    """The persistent pair kernel in each compiled register budget (128
    registers: 4 x 2 and 16 x 1 warps; 80: 8 x 3; 64: 16 x 2) on instances
    up to n = 1500 (every shape's lists fit): every shape matches the
    planner's run bit for bit, and the planner's run matches the oracle."""
    rng = np.random.default_rng(91)
    Xs, lams = [], []
    for b, n in enumerate((1500, 80, 1100, 700, 1400, 333)):
        m = int(rng.integers(2, 16))
        X, _, _ = datagen.planted(datagen.Planted(n, m, max(1, m // 4), 0.1, 0.15, 10.0,
                                                  7000 + b, np.dtype(dtype).name))
        Xs.append(X)
        lams.append(np.array([0.0, 0.4]))
    Xd = [torch.from_numpy(X).cuda() for X in Xs]
    l1line.set_tuning(None)
    bat = l1line.Batched(Xd, lams)
    bat.run()
    assert bat.status() == l1line.OK
    ref = [tuple(t.clone() for t in r) for r in bat.results()]
    _check(Xs, lams, ref, "planner")
    ib = torch.int32 if dtype == np.float32 else torch.int64
    for warps, ctas in ((4, 2), (8, 3), (16, 2), (16, 1)):
        l1line.set_tuning({"warps": warps, "ctas_per_sm": ctas, "batch_classes": 1})
        try:
            b2 = l1line.Batched(Xd, lams)
            b2.run()
        finally:
            l1line.set_tuning(None)
        assert b2.status() == l1line.OK
        for b, (a, c) in enumerate(zip(ref, b2.results())):
            assert torch.equal(a[0].view(ib), c[0].view(ib)), (warps, ctas, b)
            assert torch.equal(a[1], c[1]) and torch.equal(a[2], c[2]), (warps, ctas, b)
