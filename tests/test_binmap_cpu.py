"""The pair kernel's bin layout for the bracket histogram, compiled for the
host from the same header as the kernel (tests/native/binmap_check.cpp):
bins tile every bracket in order, keys map to the bin holding them, the
zero-crossing layout starts a bin at key 0, and the guard-band test by
neighbouring keys equals the test by bin edges."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bin_layout_tiles_every_bracket(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "binmap_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror",
                    os.path.join(HERE, "native", "binmap_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
