"""The size-class split of a batched fit, compiled for the host from the same
header the planner uses (tests/native/batch_split_check.cpp): on small random
batches the dynamic programme's split matches a brute-force enumeration of
every set of class starts, for each fixed class count and under the
added-class gain rule."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_split_matches_brute_force(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "batch_split_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror",
                    os.path.join(HERE, "native", "batch_split_check.cpp"), "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
