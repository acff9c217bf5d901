"""Host-side checks of logic the kernels share (CPU only): the batch
kernel's warp lower bound and owner search (search.cuh), compiled with g++
and checked against std::lower_bound on sorted arrays with repeats."""
import os
import subprocess

from conftest import ROOT


def test_search_helpers(tmp_path):
    exe = str(tmp_path / "search_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_2010_03090_gb300", "csrc"), "-o", exe,
                    os.path.join(ROOT, "tests", "host", "search_check.cpp")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 bad" in r.stdout
