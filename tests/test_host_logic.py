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


def test_location_rule_on_every_short_class_string():
    """The rule the error-location kernels use (locate.cuh), restated here:
    take the first position where the Section 6 classification reports an
    error (the lookup aid's per-position special_cases ^ must_be_2_3, with
    the Section 6.3 zero padding), step back at most three bytes to a
    position where no character is cut; that is the oracle's longest valid
    prefix, for every string over the 14 byte classes up to 4 bytes."""
    import itertools
    import sys

    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import lookup_aid

    def first_error(b):
        buf = np.concatenate([np.frombuffer(b, np.uint8), np.zeros(3, np.uint8)])
        prev = np.zeros(3, np.uint8)
        sc = lookup_aid.classify(buf, prev)["special_cases"]
        m = lookup_aid.must_be_2_3_continuation(buf, prev)
        nz = np.nonzero(sc ^ m)[0]
        return int(nz[0]) if nz.size else None

    def whole_characters_before(b, m):
        c1, c2, c3 = (b[m - k] if m >= k else 0 for k in (1, 2, 3))
        return not (c1 >= 0xC0 or c2 >= 0xE0 or c3 >= 0xF0)

    reps = [0x41, 0x85, 0x95, 0xA5, 0xC0, 0xC5, 0xE0, 0xE5, 0xED, 0xEE, 0xF0, 0xF2, 0xF4, 0xF8]
    for length in range(5):
        for t in itertools.product(reps, repeat=length):
            b = bytes(t)
            p = first_error(b)
            if p is None:
                assert oracle.locate(b) == (len(b), 0)
                continue
            m = min(p, len(b))
            steps = 0
            while not whole_characters_before(b, m):
                m -= 1
                steps += 1
            assert steps <= 3 and p - m <= 3
            assert m == oracle.locate(b)[0], b.hex()
