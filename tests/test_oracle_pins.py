"""Pins the CPU oracle to things other than itself (CPU only).

* values the paper prints (Table 8 rows; the named sequences of Tables 1-4
  and Section 3),
* the closed-form count of valid strings of each length,
* Python's strict UTF-8 codec (a library routine for the same predicate),
* the Section 5 finite-state validator and the Section 6 ``lookup`` steps,
  exhaustively on short strings and on every byte-class string up to 7,
* encoding every code point (valid) and every surrogate / too-large /
  overlong form (invalid).
``test_oracle_mutants.py`` shows that a planted mistake fails these pins.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import lookup_aid
from conftest import read_hex_rows

# One representative byte per class that the validity predicate can tell
# apart (Table 1 ranges split where rules d-f put their bounds).
CLASS_REPS_LOW = bytes([0x00, 0x80, 0x90, 0xA0, 0xC0, 0xC2, 0xE0, 0xE1, 0xED, 0xEE,
                        0xF0, 0xF1, 0xF4, 0xF5])
CLASS_REPS_HIGH = bytes([0x7F, 0x8F, 0x9F, 0xBF, 0xC1, 0xDF, 0xE0, 0xEC, 0xED, 0xEF,
                         0xF0, 0xF3, 0xF4, 0xFF])


def codec_valid(b: bytes) -> bool:
    try:
        b.decode("utf-8", "strict")
        return True
    except UnicodeDecodeError:
        return False


def valid_count_recurrence(n: int) -> int:
    """V(n) = 128 V(n-1) + 1920 V(n-2) + 61440 V(n-3) + 1048576 V(n-4):
    the number of code points of each encoded length (Table 1: 0x80,
    0x800 - 0x80, 0x10000 - 0x800 - 0x800 surrogates, 0x110000 - 0x10000)."""
    v = [1]
    for k in range(1, n + 1):
        t = 128 * v[k - 1]
        t += 1920 * v[k - 2] if k >= 2 else 0
        t += 61440 * v[k - 3] if k >= 3 else 0
        t += 1048576 * v[k - 4] if k >= 4 else 0
        v.append(t)
    return v[n]


# --------------------------------------------------------------------------
# values the paper prints
# --------------------------------------------------------------------------
def test_named_vectors(golden_dir):
    rows = read_hex_rows(os.path.join(golden_dir, "vectors.txt"))
    assert len(rows) >= 20
    for expect, seq in rows:
        want = expect == "valid"
        assert oracle.valid(seq) == want, seq.hex(" ")
        assert oracle.fsm_valid(seq) == want, seq.hex(" ")
        assert lookup_aid.lookup_valid(seq) == want, seq.hex(" ")
        assert codec_valid(seq) == want, seq.hex(" ")


def test_table8_rows(golden_dir):
    rows = dict(read_hex_rows(os.path.join(golden_dir, "table8.txt")))
    block = np.frombuffer(rows["input"], dtype=np.uint8)
    got = lookup_aid.classify(block, np.zeros(len(block), dtype=np.uint8))
    for name, want in rows.items():
        assert bytes(got[name].astype(np.uint8)) == want, name


def test_tables_cover_table7_exactly():
    """Bit k of the AND is set exactly on the pattern's product set."""
    sc = lookup_aid.pair_special_cases()
    p = np.arange(256)
    for bit, (hi1, lo1, hi2) in lookup_aid.TABLE7_PATTERNS.items():
        want = (np.isin(p >> 4, hi1) & np.isin(p & 15, lo1))[:, None] & \
            np.isin(p >> 4, hi2)[None, :]
        assert np.array_equal((sc & bit) != 0, want), hex(bit)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("length", [1, 2, 3])
def test_count_closed_form(length):
    assert valid_count_recurrence(1) == 128
    assert valid_count_recurrence(2) == 18304
    want = valid_count_recurrence(length)
    assert oracle.count_valid(length) == want
    assert oracle.count_valid(length, which=1) == want


def test_count_closed_form_len4_multibyte_leads():
    # strings of length 4 that start with a 2-, 3- or 4-byte lead:
    # V(4) - 128 V(3) = 1920 V(2) + 61440 V(1) + 1048576 V(0)
    want = valid_count_recurrence(4) - 128 * valid_count_recurrence(3)
    assert want == 44056576
    assert oracle.count_valid(4, lead_min=0xC0) == want


# --------------------------------------------------------------------------
# Python's strict codec
# --------------------------------------------------------------------------
def test_codec_all_len_le2():
    v1 = oracle.valid_all(1)
    v2 = oracle.valid_all(2)
    for r in range(256):
        assert v1[r] == codec_valid(bytes([r]))
    for r in range(65536):
        assert v2[r] == codec_valid(bytes([r & 255, r >> 8])), hex(r)


def test_codec_len3_selected_leads():
    v3 = oracle.valid_all(3)
    for b0 in [0x41, 0x80, 0xBF, 0xC1, 0xC2, 0xDF, 0xE0, 0xE1, 0xEC, 0xED, 0xEE, 0xEF,
               0xF0, 0xF4, 0xF5]:
        for r in range(65536):
            s = bytes([b0, r & 255, r >> 8])
            assert v3[b0 | (r << 8)] == codec_valid(s), s.hex(" ")


def test_codec_random_strings():
    rng = np.random.default_rng(20100309)
    alphabet = np.frombuffer(CLASS_REPS_LOW + CLASS_REPS_HIGH + b"az\n", dtype=np.uint8)
    for _ in range(20000):
        n = int(rng.integers(0, 24))
        s = bytes(alphabet[rng.integers(0, alphabet.size, n)])
        want = codec_valid(s)
        assert oracle.valid(s) == want, s.hex(" ")
        assert lookup_aid.lookup_valid(s, w=8) == want, s.hex(" ")


def test_codec_random_batch():
    rng = np.random.default_rng(7)
    alphabet = np.frombuffer(CLASS_REPS_LOW + CLASS_REPS_HIGH, dtype=np.uint8)
    lens = rng.integers(0, 40, 5000)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    data = alphabet[rng.integers(0, alphabet.size, int(offsets[-1]))]
    got = oracle.valid_batch(data, offsets, threads=3)
    for k in range(lens.size):
        s = bytes(data[offsets[k]:offsets[k + 1]])
        assert got[k] == codec_valid(s)


# --------------------------------------------------------------------------
# independent validators, exhaustively
# --------------------------------------------------------------------------
@pytest.mark.parametrize("length", [1, 2, 3])
def test_fsm_agrees_all_short(length):
    assert np.array_equal(oracle.valid_all(length, which=0), oracle.valid_all(length, which=1))


@pytest.mark.parametrize("reps", [CLASS_REPS_LOW, CLASS_REPS_HIGH])
def test_fsm_agrees_class_strings(reps):
    assert oracle.class_disagreements(reps, 7) == 0


@pytest.mark.parametrize("length", [1, 2, 3])
def test_lookup_agrees_all_short(length):
    want = oracle.valid_all(length).astype(bool)
    r = np.arange(256 ** length, dtype=np.uint32)
    rows = np.stack([(r >> (8 * k)) & 255 for k in range(length)], axis=1).astype(np.uint8)
    for lo in range(0, rows.shape[0], 1 << 21):
        got = lookup_aid.lookup_valid_rows(rows[lo:lo + (1 << 21)])
        assert np.array_equal(got, want[lo:lo + (1 << 21)])


@pytest.mark.parametrize("reps", [CLASS_REPS_LOW, CLASS_REPS_HIGH])
def test_lookup_agrees_class_strings(reps):
    reps = np.frombuffer(reps, dtype=np.uint8)
    for length in range(1, 7):
        idx = np.indices((reps.size,) * length).reshape(length, -1).T
        rows = reps[idx]
        got = lookup_aid.lookup_valid_rows(rows)
        offsets = np.arange(0, rows.size + 1, length, dtype=np.int64)
        want = oracle.valid_batch(rows.reshape(-1), offsets).astype(bool)
        assert np.array_equal(got, want), length


def test_lookup_ascii_blocks_match():
    """Section 6.4's ASCII blocks change nothing: block widths 3..80."""
    rng = np.random.default_rng(11)
    alphabet = np.frombuffer(b"abc" * 20 + CLASS_REPS_LOW + CLASS_REPS_HIGH, dtype=np.uint8)
    for _ in range(600):
        n = int(rng.integers(0, 200))
        s = alphabet[rng.integers(0, alphabet.size, n)]
        w = int(rng.integers(3, 81))
        assert lookup_aid.lookup_valid(s, w=w) == oracle.valid(s)


# --------------------------------------------------------------------------
# encodings of every code point
# --------------------------------------------------------------------------
def _encode_raw(cp: int, length: int) -> bytes:
    """Plain UTF-8 bit layout of cp in `length` bytes (no range checks)."""
    if length == 1:
        return bytes([cp])
    lead_bits = {2: 0xC0, 3: 0xE0, 4: 0xF0}[length]
    out = []
    for _ in range(length - 1):
        out.append(0x80 | (cp & 0x3F))
        cp >>= 6
    out.append(lead_bits | cp)
    return bytes(reversed(out))


def _batch(seqs):
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([len(s) for s in seqs])
    return oracle.valid_batch(np.frombuffer(b"".join(seqs), dtype=np.uint8), offsets)


def test_roundtrip_every_scalar_value():
    cps = [c for c in range(0x110000) if not 0xD800 <= c <= 0xDFFF]
    seqs = [chr(c).encode("utf-8") for c in cps]
    assert _batch(seqs).all()
    assert oracle.valid(b"".join(seqs))
    # our raw encoder agrees with the codec on a stride of them
    for c in cps[::97]:
        n = 1 if c < 0x80 else 2 if c < 0x800 else 3 if c < 0x10000 else 4
        assert _encode_raw(c, n) == chr(c).encode("utf-8")


def test_surrogates_too_large_overlong_invalid():
    sur = [chr(c).encode("utf-8", "surrogatepass") for c in range(0xD800, 0xE000)]
    assert not _batch(sur).any()
    big = [_encode_raw(c, 4) for c in range(0x110000, 0x200000)]
    assert not _batch(big).any()
    over = [_encode_raw(c, 2) for c in range(0x80)]
    over += [_encode_raw(c, 3) for c in range(0x800)]
    over += [_encode_raw(c, 4) for c in range(0x10000)]
    assert not _batch(over).any()


def test_named_error_classes():
    """The error classes the workloads inject, each on a small case."""
    cases = {
        "too short": b"a\xe9\x8fb",
        "too long": b"a\xc3\xa7\xa7",
        "overlong": b"x\xc1\xbf",
        "too large": b"\xf4\x90\x80\x80",
        "too large lead": b"\xf5\x80\x80\x80",
        "surrogate": b"\xed\xa0\x80",
        "stray continuation": b"\x80abc",
        "truncated tail": b"abc\xf0\x9f\x98",
        "5-byte": b"\xf8\x88\x80\x80\x80",
    }
    for name, s in cases.items():
        assert not oracle.valid(s), name
        assert not codec_valid(s), name
