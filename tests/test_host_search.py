"""Host check of the membership search that the search kernels share with the host
(paper_2404_01585_gb300/csrc/search_util.h): compiled as plain C++ and compared with
std::binary_search on sorted runs of many shapes (empty, tiny, uniform, clustered, geometric,
extreme ids), with the bisection bound on the loads it makes."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_interpolation_search_matches_binary_search():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "check")
        subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2404_01585_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "host_search_check.cpp"), "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout
