"""Autotuner: cache keys and file round trip (CPU), the ABI's tuning checks
(CPU), and on the GPU that every candidate tuning gives the same results as
the planner's plan, bit for bit."""
import numpy as np
import pytest

import __graft_entry__
from paper_2402_16712_gb300 import autotune, datagen, l1line


def test_bucket_and_key():
    assert [autotune.bucket(x) for x in (1, 2, 3, 1000, 1024, 1025)] == [1, 2, 4, 1024, 1024, 2048]
    k = autotune.key("float32", 2000, 2000, 1, gpu="G")
    assert k == "G|f32|fit|n2048|m2048|l1"
    assert autotune.key("float64", 1000, 500, 32, "batch", gpu="G") == "G|f64|batch|n1024|m512|l32"


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "sub" / "cache.json")
    assert autotune.load_cache(p) == {}
    autotune.store("a", {"warps": 4}, 1.5, p)
    autotune.store("b", {}, 2.5, p)
    d = autotune.load_cache(p)
    assert d["a"] == {"tuning": {"warps": 4}, "ms": 1.5} and d["b"]["tuning"] == {}
    (tmp_path / "bad.json").write_text("not json")
    assert autotune.load_cache(str(tmp_path / "bad.json")) == {}


def test_candidates_vary_one_knob_group():
    c = list(autotune.candidates({"warps": 8, "ctas_per_sm": 3, "kchunk": 2000, "d0": 6}))
    assert {"kchunk": 1000} in c and {"d0": 4} in c and {"warps": 4, "ctas_per_sm": 3} in c
    assert all(len(x) <= 2 for x in c)
    assert not any("batch_classes" in x for x in c)
    cb = list(autotune.candidates({"warps": 8, "ctas_per_sm": 3, "kchunk": 0, "d0": 6},
                                  kchunk=False, classes=True))
    assert [x for x in cb if "batch_classes" in x] == [{"batch_classes": k} for k in (1, 2, 3)]
    assert not any("kchunk" in x for x in cb)
    # the other placement of x_ijhat than the plan's
    assert {"column": 2} in c and {"column": 1} in c
    assert [x for x in autotune.candidates({"kchunk": 1, "d0": 6, "column": 2})
            if "column" in x] == [{"column": 1}]


def test_tuning_argument_checks():
    __graft_entry__.build()
    l1line.load()
    for bad in ({"warps": 17}, {"ctas_per_sm": 4}, {"kchunk": -1}, {"d0": 25}, {"warps": -1},
                {"batch_classes": 4}, {"batch_classes": -1}, {"column": 3}, {"column": -1}):
        with pytest.raises(l1line.L1LineError):
            l1line.set_tuning(bad)
    l1line.set_tuning({"warps": 4, "d0": 8})
    l1line.set_tuning(None)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_every_candidate_tuning_gives_identical_results(dtype):
    import torch
    __graft_entry__.build()
    X, _, _ = datagen.planted(datagen.Planted(900, 48, 5, 0.1, 0.1, 10.0, 21, np.dtype(dtype).name))
    Xd = torch.from_numpy(X).cuda()
    lams = [0.0, 0.3, 0.9, 2.0]
    l1line.set_tuning(None)
    v0, s0, z0, ws = l1line.scan(Xd, lams)
    assert l1line.status(ws) == l1line.OK
    base = l1line.plan(Xd.dtype, 900, 48)
    tried = 0
    for cand in autotune.candidates(base):
        l1line.set_tuning(cand)
        try:
            v1, s1, z1, ws1 = l1line.scan(Xd, lams)
        except l1line.L1LineError:
            continue
        finally:
            l1line.set_tuning(None)
        assert l1line.status(ws1) == l1line.OK
        assert torch.equal(v0.view(-1).view(torch.int32 if dtype == np.float32 else torch.int64),
                           v1.view(-1).view(torch.int32 if dtype == np.float32 else torch.int64)), cand
        assert torch.equal(z0, z1), cand
        tried += 1
    assert tried >= 10


@pytest.mark.gpu
def test_apply_tunes_once_and_then_reads_the_cache(tmp_path):
    import torch
    __graft_entry__.build()
    p = str(tmp_path / "tune.json")
    X, lams, _ = datagen.lambda_path("float32", n=600, m=120, n_lambda=8)
    Xd = torch.from_numpy(X).cuda()
    ws = l1line.Workspace.for_shape(torch.float32, 600, 120, lams.size)
    run = lambda: l1line.fit(Xd, lams, workspace=ws)
    t = autotune.apply(torch.float32, 600, 120, lams.size, run=run, path=p)
    assert autotune.key(torch.float32, 600, 120, lams.size) in autotune.load_cache(p)
    v1, o1, j1, _ = l1line.fit(Xd, lams, workspace=ws)
    t2 = autotune.apply(torch.float32, 600, 120, lams.size, path=p)  # cached: no run needed
    assert t2 == t
    l1line.set_tuning(None)
    v0, o0, j0, _ = l1line.fit(Xd, lams, workspace=ws)
    assert torch.equal(v0, v1) and torch.equal(o0, o1) and torch.equal(j0, j1)
