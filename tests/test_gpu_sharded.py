"""The jhat-sharded fit on the GPU: without a process group it is the plain
fit; with two gloo ranks (two processes sharing this GPU; their kernels never
wait on each other, the exchange is on the host) every rank gets the plain
fit's result bit for bit, which matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_16712_gb300 import datagen, l1line, sharded
from tests._dist import run_ranks
from tests._parity import assert_v_equal

pytestmark = pytest.mark.gpu

LAMS = [0.0, 0.3, 2.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _data(m, dtype):
    X, _, _ = datagen.planted(datagen.Planted(300, m, max(1, m // 6), 0.1, 0.1, 10.0, 71 + m,
                                              np.dtype(dtype).name))
    return X


def _sharded_on_rank(rank, world, m, dtype):
    X = _data(m, dtype)
    v, z, j = sharded.fit_sharded(torch.from_numpy(X).cuda(), LAMS)
    torch.cuda.synchronize()
    return v.cpu().numpy(), z.cpu().numpy(), j.cpu().numpy()


def test_without_a_group_it_is_the_plain_fit():
    X = torch.from_numpy(_data(37, np.float32)).cuda()
    v0, z0, j0, _ = l1line.fit(X, LAMS)
    v1, z1, j1 = sharded.fit_sharded(X, LAMS)
    assert torch.equal(v0.view(torch.int32), v1.view(torch.int32))
    assert torch.equal(z0, z1) and torch.equal(j0, j1)


@pytest.mark.parametrize("m,dtype", [(37, np.float32), (24, np.float64), (1, np.float32)])
def test_two_ranks_match_the_plain_fit_and_the_oracle(m, dtype):
    X = _data(m, dtype)
    v0, z0, j0, _ = l1line.fit(torch.from_numpy(X).cuda(), LAMS)
    v0, z0, j0 = v0.cpu().numpy(), z0.cpu().numpy(), j0.cpu().numpy()
    out = run_ranks(_sharded_on_rank, 2, m, dtype)
    for rank in (0, 1):
        v, z, j = out[rank]
        assert_v_equal(v, v0, f"rank {rank}")
        assert np.array_equal(z, z0) and np.array_equal(j, j0), rank
    ref = oracle.fit(X, LAMS)
    for t in range(len(LAMS)):
        assert int(j0[t]) == int(ref["jstar"][t]) or \
            abs(ref["z_all"][t][int(j0[t])] - ref["z_all"][t][int(ref["jstar"][t])]) <= \
            1e-5 * abs(ref["obj"][t]), t
        assert_v_equal(v0[t], ref["v_all"][t, int(j0[t])], f"lambda {t}")
