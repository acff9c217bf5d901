"""Each planted mistake in the oracle (compiled with -DORACLE_MUTANT=k) must
fail at least one pin.  The mutants: a wrong 3-byte overlong bound, 5-byte
leads admitted, a truncated tail ignored, any byte >= 0x80 taken as a
continuation, an off-by-one code-point maximum, surrogates admitted; and in
the error location: a too-short character reported at its missing byte
instead of its start, C0/C1 leads reported as rule a instead of d."""
import os

import numpy as np
import pytest

import oracle
from conftest import read_hex_rows
from test_oracle_locate import bad_character, codec_position, random_text
from test_oracle_pins import codec_valid, valid_count_recurrence, _batch


def _pins_failed(mutant, golden_dir):
    failed = []
    for expect, seq in read_hex_rows(os.path.join(golden_dir, "vectors.txt")):
        if oracle.valid(seq, mutant=mutant) != (expect == "valid"):
            failed.append("vectors")
            break
    for length in (1, 2, 3):
        if oracle.count_valid(length, mutant=mutant) != valid_count_recurrence(length):
            failed.append(f"count{length}")
    if oracle.count_valid(4, lead_min=0xF0, mutant=mutant) != \
            oracle.count_valid(4, lead_min=0xF0, which=1, mutant=mutant):
        failed.append("fsm4")
    v2 = oracle.valid_all(2, mutant=mutant)
    if any(v2[r] != codec_valid(bytes([r & 255, r >> 8])) for r in range(65536)):
        failed.append("codec2")
    big = [bytes([0xF4, 0x90, 0x80, 0x80]), bytes([0xF4, 0x90, 0x80, 0x80, 0x41])]
    if oracle.valid_batch(np.frombuffer(b"".join(big), np.uint8),
                          np.array([0, 4, 9]), mutant=mutant).any():
        failed.append("too-large")
    rng = np.random.default_rng(3)
    for rule in range(1, 7):
        for _ in range(50):
            head = random_text(rng, 3)
            b = head + bad_character(rule, rng) + b"A"
            got = oracle.locate(b, mutant=mutant)
            if got != (len(head), rule) or got[0] != codec_position(b):
                failed.append(f"locate-rule{rule}")
                break
    return failed


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7, 8])
def test_mutant_is_caught(mutant, golden_dir):
    assert _pins_failed(mutant, golden_dir), f"mutant {mutant} passed every pin"


def test_unmutated_passes_same_checks(golden_dir):
    assert _pins_failed(0, golden_dir) == []
