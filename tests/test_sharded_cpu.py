"""Multi-rank host logic on CPU (gloo, no GPU): the jhat-sharded fit's shard
ranges and cross-rank argmin (world sizes 2 and 3), and the bench's job time
over ranks."""
import numpy as np
import pytest

from paper_2402_16712_gb300 import sharded
from tests._dist import run_ranks


def test_shard_ranges_cover_every_jhat_once():
    for m in (1, 2, 7, 10, 2000):
        for world in (1, 2, 3, 8):
            spans = [sharded.shard_range(m, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.shard_range(10, 2, 2)


# Per rank and lambda: (objective, local jhat* or -1).  Cases: a strictly
# smaller objective on rank 1; equal objectives (smallest jhat wins); a rank
# with no jhat; objectives of 0; a tie across all three ranks.
LOCAL = {
    0: [(3.0, 2), (4.0, 4), (1.5, 1), (0.0, 1), (7.25, 3)],
    1: [(2.5, 7), (4.0, 5), (9.0, -1), (0.0, 6), (7.25, 6)],
    2: [(2.75, 9), (5.0, 8), (8.0, 9), (0.5, 8), (7.25, 9)],
}


def _combine_on_rank(rank, world):
    import torch
    rows = LOCAL[rank]
    obj = torch.tensor([z for z, _ in rows], dtype=torch.float64)
    js = torch.tensor([j for _, j in rows], dtype=torch.int64)
    v = torch.full((len(rows), 4), float(rank + 1), dtype=torch.float32)
    v[:, 0] = -0.5 * (rank + 1)
    z, j, vg = sharded.combine(obj, js, v)
    return z.numpy(), j.numpy(), vg.numpy()


@pytest.mark.parametrize("world", [2, 3])
def test_combine_picks_the_global_argmin(world):
    out = run_ranks(_combine_on_rank, world)
    for t in range(len(LOCAL[0])):
        # smallest objective, ties to the smallest jhat; v from the rank that owns it
        zw, jw, owner = min((LOCAL[r][t][0], LOCAL[r][t][1], r) for r in range(world)
                            if LOCAL[r][t][1] >= 0)
        want_v = np.full(4, owner + 1, dtype=np.float32)
        want_v[0] = -0.5 * (owner + 1)
        for rank in range(world):
            z, j, v = out[rank]
            assert z[t] == zw and j[t] == jw, (rank, t, z[t], j[t])
            assert np.array_equal(v[t], want_v), (rank, t)


def _bench_aggregate(rank, world):
    import torch.distributed as dist

    import bench
    ms = 10.0 * (rank + 1)  # the slowest rank takes 10 * world ms
    tot = bench.job_ms(ms, dist, "cpu")
    return tot, bench.job_value(world, 4, 1000.0, tot)


def test_bench_job_time_is_the_slowest_rank():
    out = run_ranks(_bench_aggregate, 2)
    for rank in (0, 1):
        tot, value = out[rank]
        assert tot == 20.0
        assert value == 2 * 4 * 1000.0 / 0.020
