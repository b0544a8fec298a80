"""Bandwidth probes behind the bench's L2 and shared-memory ceilings: they run,
report the bytes they read, and land in a plausible range for one GB300."""
import pytest
import torch

from paper_2402_16712_gb300 import l1line

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_l2_probe():
    buf = torch.ones(16 << 20, dtype=torch.uint8, device="cuda")  # 16 MB, L2-resident
    l1line.probe_bandwidth(l1line.PROBE_L2, 2, buf)  # warm-up
    bw = l1line.probe_bandwidth(l1line.PROBE_L2, 20, buf)
    assert l1line.last_launch_count() == 1
    assert 2e12 < bw < 2e14, bw  # above any HBM rate, below the SMs' load ports


def test_smem_probe():
    l1line.probe_bandwidth(l1line.PROBE_SMEM, 16)
    bw = l1line.probe_bandwidth(l1line.PROBE_SMEM, 2000)
    # 152 SMs x 128 bytes per clock x 2.07 GHz = 40.3 TB/s nominal
    assert 1e13 < bw < 5e13, bw
