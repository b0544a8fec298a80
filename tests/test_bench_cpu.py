"""The bench's roofline arithmetic on hand-worked numbers: a 2000-row pair
kernel that scores 3,998,000 pairs in 20 ms (1.999e8 pairs/s) against
shared-memory, L2 and issue peaks."""
import pytest


def test_roofline_picks_the_binding_ceiling():
    import bench
    r = bench.roofline(2000, 3_998_000, 20.0, 500, 1, 17_870.0, 40_000.0, None)
    c = r["ceilings"]
    # 16 shared-memory bytes per pair-row: 1.999e8 * 32,000 B = 6,396.8 GB/s
    assert c["smem"]["achieved"] == pytest.approx(6396.8)
    assert c["smem"]["frac"] == pytest.approx(6396.8 / 40_000.0)
    assert c["smem"]["ceiling_pairs_per_s"] == pytest.approx(40_000e9 / 32_000)
    # 4 n (1 + 1/T_k) L2 bytes per pair at T_k = 500: 8,016 B
    assert c["l2"]["achieved"] == pytest.approx(1.999e8 * 8016 / 1e9)
    assert c["l2"]["ceiling_pairs_per_s"] == pytest.approx(17_870e9 / 8016)
    # 8 lane-instructions per pair-row; 152 SMs x 128 lanes x 2070 MHz
    assert c["alu"]["peak"] == pytest.approx(152 * 128 * 2070e6 / 1e12)
    assert c["alu"]["achieved"] == pytest.approx(1.999e8 * 16_000 / 1e12)
    # the binding ceiling (fewest pairs/s) is shared memory here
    assert r["bound"] == "smem" and r["unit"] == "GB/s"
    assert r["frac"] == c["smem"]["frac"] and r["traffic"] is None
    assert r["kernel"] == "k_pairs<float, 0, 1, 0>" and r["kernel_ms"] == 20.0


def test_roofline_names_the_timed_placement_and_binding_l2():
    import bench
    # a slow L2 makes L2 the binding ceiling; column 2 keeps x_ijhat in global memory
    r = bench.roofline(2000, 3_998_000, 20.0, 1000, 2, 1_000.0, 40_000.0, 1.7e7)
    assert r["bound"] == "l2" and r["kernel"] == "k_pairs<float, 0, 0, 0>"
    assert r["achieved"] == pytest.approx(1.999e8 * 4 * 2000 * 1.001 / 1e9)
    assert r["traffic"] == 1.7e7


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_two_ranks_prints_one_line_on_all_cores():
    """The oracle arm launched like the multi-GPU bench: rank 0 alone times the
    oracle, on every host core although torchrun sets OMP_NUM_THREADS=1, and
    prints the one JSON line; the other rank exits 0 without work."""
    import json
    import os
    import subprocess
    import sys

    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == bench._host_cores()
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_cpu_baseline_reports_all_cores_and_one():
    import numpy as np

    import bench
    X = np.random.default_rng(0).normal(size=(300, 60)).astype(np.float32)
    r = bench.cpu_baseline(X, 0.5, target_s=0.2)
    assert r["kind"] == "oracle" and r["unit"] == "pairs/s" and r["value"] > 0
    assert r["cores"] == bench._host_cores()
    one = r["single_core"]
    assert one["cores"] == 1 and one["value"] > 0 and "jhat columns" in one["sample"]


def test_comparison_line_host_logic(monkeypatch):
    """measure_comparison's host code with the CUDA pieces faked: it builds
    one batched call over the 30 datasets x 8 lambdas and reports rates from
    the event times (an error there would only show as an 'error' entry in
    the bench line, so it is checked here)."""
    import contextlib

    import torch

    import bench
    from paper_2402_16712_gb300 import l1line

    calls = {"run": 0}

    class FakeBatched:
        def __init__(self, Xs, lams, device=None):
            assert len(Xs) == 30 and all(tuple(X.shape) == (100, 100) for X in Xs)
            assert all(list(lm) == [0.0, 5.0, 20.0, 50.0, 100.0, 200.0, 400.0, 800.0]
                       for lm in lams)

        def run(self, stream=None):
            calls["run"] += 1

        def status(self, stream=None):
            return l1line.OK

    class FakeEvent:
        n = 0

        def __init__(self, enable_timing=False):
            FakeEvent.n += 1
            self.t = FakeEvent.n

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 2.0  # ms

    class Fill:
        def fill_(self, v):
            pass

    class Stream:
        def synchronize(self):
            pass

    monkeypatch.setattr(l1line, "Batched", FakeBatched)
    monkeypatch.setattr(l1line, "set_tuning", lambda t=None: None)
    monkeypatch.setattr(l1line, "last_launch_count", lambda: 8)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    r = bench.measure_comparison("cpu", Stream(), Fill(), steps=5)
    assert calls["run"] == 3 + 5
    assert r["ms_per_step"] == 2.0 and r["gpu_launches_per_step"] == 8
    assert r["fits_per_s"] == 240 / 2e-3
    assert r["pair_lambdas_per_s"] == 30 * 100 * 99 * 8 / 2e-3


def test_components_line_host_logic(monkeypatch):
    """measure_components' host code with the CUDA pieces faked: one
    workspace for every call, three components per call, rates from the event
    times."""
    import contextlib

    import torch

    import bench
    from paper_2402_16712_gb300 import l1line

    seen = []

    def fake_components(X, lam, ncomp, workspace=None, stream=None):
        assert tuple(X.shape) == (1000, 500) and lam == 0.5 and ncomp == 3
        seen.append(workspace)
        return None, None, torch.tensor([7, 3, 11], dtype=torch.int32), "ws"

    class FakeEvent:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 4.0

    class Fill:
        def fill_(self, v):
            pass

    class Stream:
        def synchronize(self):
            pass

    monkeypatch.setattr(l1line, "components", fake_components)
    monkeypatch.setattr(l1line, "status", lambda ws, stream=None: l1line.OK)
    monkeypatch.setattr(l1line, "set_tuning", lambda t=None: None)
    monkeypatch.setattr(l1line, "last_launch_count", lambda: 17)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    r = bench.measure_components("cpu", Stream(), Fill(), ncomp=3, steps=5)
    assert seen[0] is None and all(w == "ws" for w in seen[1:]) and len(seen) == 1 + 2 + 5
    assert r["ms_per_step"] == 4.0 and r["components_per_s"] == 3 / 4e-3
    assert r["pairs_per_s"] == 3 * 500 * 499 / 4e-3 and r["jhat_star"] == [7, 3, 11]
    assert r["gpu_launches_per_step"] == 17


def _sharded_leg_on_rank(rank, world):
    """bench.measure_sharded on one gloo rank with the CUDA pieces faked: the
    'fit' of a jhat list returns the best of a fixed objective table over it,
    so the sharded result must equal the one-GPU fit's."""
    import numpy as np
    import torch

    import bench
    from paper_2402_16712_gb300 import l1line

    m = 2000
    z = (np.arange(m, dtype=np.float64) - 1234.0) ** 2 + 3.0  # argmin at jhat 1234

    def best(jl, nl=1):
        jl = np.asarray(jl)
        j = int(jl[np.argmin(z[jl])])
        v = torch.full((nl, m), float(j), dtype=torch.float32)
        return v, torch.tensor([z[j]], dtype=torch.float64), torch.tensor([j], dtype=torch.int32)

    def fake_fit_subset(X, lambdas, jhat, workspace=None, stream=None, out=None):
        v, o, j = best(jhat.numpy())
        return v, o, j, workspace

    def fake_fit(X, lambdas, workspace=None, stream=None, out=None):
        v, o, j = best(np.arange(m))
        return v, o, j, workspace

    class FakeEvent:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 1.0 + rank  # ms: the slower rank sets the job's time

    l1line.fit_subset = fake_fit_subset
    l1line.fit = fake_fit
    l1line.Workspace.for_shape = classmethod(lambda cls, *a, **k: None)
    torch.cuda.Event = FakeEvent
    torch.cuda.synchronize = lambda *a, **k: None
    import torch.distributed as dist
    return bench.measure_sharded(torch.device("cpu"), None, dist, 3, 1)


def test_sharded_bench_leg_two_ranks():
    """The bench's one-fit-over-all-ranks leg on two gloo ranks: the jhat
    ranges, the cross-rank argmin, the max-over-ranks step time, the strong-
    scaling value (one fit's pairs per step) and the bit-identity check."""
    from tests._dist import run_ranks
    out = run_ranks(_sharded_leg_on_rank, 2)
    r0, r1 = out[0], out[1]
    assert r0["identical_to_one_gpu"] is True and r1["identical_to_one_gpu"] is None
    for r in (r0, r1):
        assert r["scaling"] == "strong" and r["n_gpus"] == 2 and r["steps"] == 3
        assert r["ms_per_step"] == pytest.approx(2.0)  # rank 1's 2 ms per step
        assert r["value"] == pytest.approx(2000 * 1999 / 2.0e-3)


def test_sharded_summary_arithmetic():
    import bench
    r = bench.sharded_summary(4, 2, 3_998_000, [5.0, 7.0], True)
    assert r["ms_per_step"] == 6.0 and r["fits_per_s"] == pytest.approx(2 / 12e-3)
    assert r["value"] == pytest.approx(2 * 3_998_000 / 12e-3)
    assert r["identical_to_one_gpu"] is True and r["scaling"] == "strong"


def test_path_roofline_arithmetic():
    """Algorithm 2's ceilings on hand-worked numbers: 2000 x 2000 float32,
    2.6e8 breakpoints in 60 ms."""
    import bench
    r = bench.path_roofline(2000, 2000, 260_000_000, 60.0, 4)
    wbytes = 260_000_000 * 12 + 2000 * 2000 * 12
    instr = 2 * 6 * 2000 * (2000 * 1999)
    c = r["ceilings"]
    assert c["hbm"]["traffic_bytes"] == wbytes and c["alu"]["instructions"] == instr
    assert c["hbm"]["achieved"] == pytest.approx(wbytes / 0.060 / 1e9)
    assert c["alu"]["achieved"] == pytest.approx(instr / 0.060 / 1e12)
    assert c["alu"]["peak"] == pytest.approx(152 * 128 * 2070e6 / 1e12)
    # the binding ceiling is the one with the longer minimum time
    t_hbm = wbytes / (c["hbm"]["peak"] * 1e9)
    t_alu = instr / (c["alu"]["peak"] * 1e12)
    assert r["bound"] == ("hbm" if t_hbm > t_alu else "alu")
    assert r["frac"] == c[r["bound"]]["frac"]


def test_pair_shape_label_follows_the_register_budgets():
    import bench
    # 128 registers up to 16 resident warps, 80 up to 24 with <= 8 warps per
    # CTA, 64 up to 32
    assert [bench.pair_shape(w, c) for w, c in ((16, 1), (8, 2), (4, 3), (8, 3), (7, 3),
                                                (16, 2), (13, 2), (10, 3))] == \
        [2, 2, 2, 0, 0, 1, 1, 1]


def test_f64_line_uses_the_pair_kernel_ceilings():
    import bench
    r = bench.roofline(2000, 3_998_000, 26.0, 667, 0, 17_870.0, 40_000.0, None, 1,
                       dtype="double", timed="whole fit")
    assert r["kernel"] == "k_pairs<double, 0, 0, 1>" and r["timed"] == "whole fit"
    # shared memory binds: 16 n bytes per pair at 3,998,000 pairs / 26 ms
    assert r["bound"] == "smem"
    assert r["achieved"] == pytest.approx(16 * 2000 * 3_998_000 / 0.026 / 1e9)
    assert r["traffic"] is None
