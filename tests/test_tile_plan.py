"""The sweep's tile plan (csrc/ase_df_tileplan.h) on the host: the header compiles as plain
C++, and tests/tile_plan_check.cpp checks every plan of a range of grids and slot counts
(exact coverage of every tile column and line, tile heights, filled waves)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2410_05489_gb300", "csrc")


def test_tile_plan_covers_every_face_line_once(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "tile_plan_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I", CSRC, os.path.join(HERE, "tile_plan_check.cpp"),
                    "-o", exe], check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.startswith("ok "), res.stdout
    assert int(res.stdout.split()[1]) == 2 * 29 * 22 * 7  # line floors 16 and 8
