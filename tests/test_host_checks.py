"""Host logic of the library checked as plain C++ (no GPU): each check program is compiled
with the host sources it tests and compared there with a plain recomputation.

* host_graph_check.cpp -- the data-graph build (csrc/graph.cpp): label ranks, deduplicated and
  sorted adjacency, label runs, vertex records, the root index in both root orders, label pairs,
  dropped self-loops and repeats, on 144 random graphs.
* host_plan_check.cpp -- the pattern compiler (csrc/pattern.cpp): matching orders and their
  masks from their definitions, orbit representatives against brute-force automorphisms, label
  slices, neighbour-label sets, tau special cases, absent labels and invalid inputs."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2404_01585_gb300", "csrc")


def run_check(main_cpp, *sources):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "check")
        subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", main_cpp), *[os.path.join(CSRC, s) for s in sources],
                        "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fails 0" in r.stdout, r.stdout


def test_host_graph_build_matches_plain_recomputation():
    run_check("host_graph_check.cpp", "graph.cpp")


def test_host_pattern_compiler_matches_definitions():
    run_check("host_plan_check.cpp", "pattern.cpp", "graph.cpp")
