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


def test_all_cores_split_keeps_validity():
    """bench.py's all-cores oracle timing cuts a buffer at character starts;
    the AND over the parts must equal the whole buffer's validity, including
    cuts inside runs of continuation bytes and errors right at a cut."""
    import sys

    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synth
    rng = np.random.default_rng(7)
    cases = []
    base = synth.fill(1 << 16, synth.UNIFORM, seed=11)
    cases.append(base)
    for kind in synth.ERROR_CLASSES:
        b = base.copy()
        synth.inject_any(b, kind, rng)
        cases.append(b)
    # runs of continuation bytes (four or more) and leads at the cut points
    for _ in range(200):
        n = int(rng.integers(1, 64))
        cases.append(rng.choice(np.array([0x41, 0x80, 0xBF, 0xC3, 0xE2, 0xF0, 0x90], np.uint8), n))
    for b in cases:
        whole = oracle.valid(b)
        for pieces in (2, 3, 8, 17):
            cuts = bench.split_at_char_starts(b, pieces)
            assert cuts[0] == 0 and cuts[-1] == b.size and np.all(np.diff(cuts) >= 0)
            parts = oracle.valid_batch(b, cuts, threads=2)
            assert bool(parts.all()) == whole
