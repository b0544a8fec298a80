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
    assert r["kernel"] == "k_pairs<float, 0, 1>" and r["kernel_ms"] == 20.0


def test_roofline_names_the_timed_placement_and_binding_l2():
    import bench
    # a slow L2 makes L2 the binding ceiling; column 2 keeps x_ijhat in global memory
    r = bench.roofline(2000, 3_998_000, 20.0, 1000, 2, 1_000.0, 40_000.0, 1.7e7)
    assert r["bound"] == "l2" and r["kernel"] == "k_pairs<float, 0, 0>"
    assert r["achieved"] == pytest.approx(1.999e8 * 4 * 2000 * 1.001 / 1e9)
    assert r["traffic"] == 1.7e7
