"""The GPU classification's design, restated in numpy, against the oracle
(CPU only).

The kernels (csrc/lookup.cuh) keep the paper's three AND-ed nibble tables for
the five second-byte rows of Table 7 and fold TOO_SHORT, TOO_LONG and
TWO_CONTS / must_be_2_3 (Section 6.2) into one continuation check: a byte is
a continuation exactly when byte i-1 >= 0xC0, byte i-2 >= 0xE0 or byte i-3 >=
0xF0.  ASCII bytes take the values prmt's sign mode gives them (0xFF on the
previous side, 0 on the current side), and the 2/3-bytes-back terms are
combined as the kernels combine them (an XOR, through one integer sum).
This file checks that design decides exactly the oracle's boolean: on every
string of up to three bytes and on every class string of up to six bytes
(validity depends only on the 14 byte classes, so six bytes cover every
window of the 4-byte check with context on both sides).  The GPU tests check
the kernels' per-position values against this design's tables and the
paper's (tests/test_gpu_parity.py)."""
import itertools

import numpy as np

import oracle

OV2, OV3, SUR, TL, OV4, CONT = 0x01, 0x02, 0x04, 0x08, 0x10, 0x40

BYTE1_HIGH = np.array([0xFF] * 8 + [0xC0] * 4 +
                      [0xC0 | OV2, 0xC0, 0xC0 | OV3 | SUR, 0xC0 | TL | OV4], np.uint8)
BYTE1_LOW = np.array([0xC0 | OV2 | OV3 | OV4, 0xC0 | OV2, 0xC0, 0xC0, 0xC0 | TL] +
                     [0xC0 | TL | OV4] * 8 + [0xC0 | TL | OV4 | SUR] + [0xC0 | TL | OV4] * 2,
                     np.uint8)
BYTE2_HIGH = np.array([0] * 8 + [CONT | OV2 | OV3 | OV4, CONT | OV2 | OV3 | TL,
                                 CONT | OV2 | SUR | TL, CONT | OV2 | SUR | TL] + [0] * 4, np.uint8)
LEAD_FLAGS = np.array([0] * 12 + [0x40, 0x40, 0x60, 0x70], np.uint8)

# one representative byte per class that decides validity
CLASSES = np.array([0x41, 0x85, 0x95, 0xA5, 0xC1, 0xC5, 0xE0, 0xE5, 0xED, 0xEE, 0xF0, 0xF2,
                    0xF4, 0xF7], np.uint8)


def model_valid(strings: np.ndarray) -> np.ndarray:
    """Validity of each row (count x n uint8) under the kernels' design."""
    count, n = strings.shape
    v = np.zeros((count, n + 6), np.uint8)  # three zeros before and after
    v[:, 3:3 + n] = strings
    hi, lo = v >> 4, v & 15
    prev = BYTE1_HIGH[hi] & BYTE1_LOW[lo]
    cur = BYTE2_HIGH[hi]
    flags = LEAD_FLAGS[hi].astype(np.uint32)
    bad = np.zeros(count, bool)
    for i in range(3, n + 6):
        back23 = ((2 * flags[:, i - 2] + 4 * flags[:, i - 3]) & 0x40).astype(np.uint8)
        expect = (flags[:, i - 1].astype(np.uint8) | back23) & CONT
        err = (prev[:, i - 1] & cur[:, i]) ^ expect
        bad |= err != 0
    return ~bad


def test_tables_restate_table7_on_non_ascii_pairs():
    """The special bits of every byte pair whose first byte is not ASCII are
    the paper's Table 7 rows (through the oracle's lookup aid)."""
    from oracle import lookup_aid
    paper = lookup_aid.pair_special_cases()  # [prev, cur] -> Table 8 bits
    b = np.arange(256)
    ours = (BYTE1_HIGH[b[:, None] >> 4] & BYTE1_LOW[b[:, None] & 15] &
            BYTE2_HIGH[b[None, :] >> 4]) & 0x1F
    mapped = np.zeros_like(ours)
    for o, p in ((OV2, 0x20), (OV3, 0x04), (SUR, 0x10), (TL, 0x08), (OV4, 0x40)):
        mapped |= np.where(ours & o, p, 0).astype(np.uint8)
    assert np.array_equal(mapped[0x80:], paper[0x80:] & 0x7C)
    # after an ASCII byte a special row can match only a continuation
    assert not np.any(ours[:0x80][:, (b & 0xC0) != 0x80])


def test_every_string_up_to_3_bytes():
    for n in (1, 2, 3):
        s = np.arange(256 ** n, dtype=np.uint32).view(np.uint8).reshape(-1, 4)[:, :n]
        assert np.array_equal(model_valid(np.ascontiguousarray(s)), oracle.valid_all(n) == 1)


def test_every_class_string_up_to_6_bytes():
    for n in (4, 5, 6):
        idx = np.array(list(itertools.product(range(CLASSES.size), repeat=n)), np.int64)
        for part in np.array_split(idx, max(1, idx.shape[0] // 1_000_000)):
            s = CLASSES[part]
            offsets = np.arange(0, s.size + 1, n, dtype=np.int64)
            want = oracle.valid_batch(s.reshape(-1), offsets, threads=4) == 1
            assert np.array_equal(model_valid(s), want), n


# ---------------------------------------------------------------------------
# The byte-permute lookups of the row-quad layout (lut_quad in
# csrc/lookup.cuh), restated with a model of PTX `prmt` (default mode): for
# result byte i, selector nibble i picks byte (nibble & 7) of the eight bytes
# {b, a}; with nibble bit 3 set the result is that byte's sign bit replicated.
# ---------------------------------------------------------------------------
def prmt(a, b, sel):
    a, b, sel = np.broadcast_arrays(np.asarray(a, np.uint64), np.asarray(b, np.uint64),
                                    np.asarray(sel, np.uint64))
    pool = np.stack([(a >> np.uint64(8 * k)) & np.uint64(0xFF) for k in range(4)] +
                    [(b >> np.uint64(8 * k)) & np.uint64(0xFF) for k in range(4)])
    out = np.zeros(a.shape, np.uint64)
    cols = np.arange(a.size)
    for i in range(4):
        nib = (sel >> np.uint64(4 * i)) & np.uint64(0xF)
        v = pool[(nib & np.uint64(7)).astype(np.int64).ravel(), cols].reshape(a.shape)
        sign = np.where(v & np.uint64(0x80), np.uint64(0xFF), np.uint64(0))
        v = np.where(nib & np.uint64(8), sign, v)
        out |= v << np.uint64(8 * i)
    return out


def pack4(t):
    return sum(int(t[k]) << (8 * k) for k in range(4))


def halves(table, reversed_):
    """The two words of an 8-entry prmt table: entries 0..7 (plain selector)
    or 15..8 (complemented selector)."""
    e = table[::-1] if reversed_ else table
    return pack4(e[0:4]), pack4(e[4:8])


def lut_quad(a, b, c, d):
    """Per j = 0..3: (prev_side, cur_side, flags) of W_j = (a_j, b_j, c_j, d_j)."""
    m = np.uint64(0x0F0F0F0F)
    full = np.uint64(0xFFFFFFFF)
    sel_not = lambda x, y: ~((x & m) | (y & ~m)) & full
    sel = lambda x, y: ((x & m) | (y & ~m)) & full
    hab = sel_not(a >> np.uint64(4), b)
    hcd = sel_not(c >> np.uint64(4), d)
    lab = sel(a, (b << np.uint64(4)) & full)
    lcd = sel(c, (d << np.uint64(4)) & full)
    b1h, b2h, flg = halves(BYTE1_HIGH, True), halves(BYTE2_HIGH, True), halves(LEAD_FLAGS, True)
    b1l_plain, b1l_rev = halves(BYTE1_LOW, False), halves(BYTE1_LOW, True)
    words = []
    for j in range(4):
        s = np.uint64(j | ((4 + j) << 4))
        hi_c = prmt(hab, hcd, s)
        lo = prmt(lab, lcd, s)
        lo_c = ~lo & full
        prev = prmt(*b1h, hi_c) & prmt(*b1l_plain, lo) & prmt(*b1l_rev, lo_c)
        words.append((prev, prmt(*b2h, hi_c), prmt(*flg, hi_c)))
    return words


def test_quad_lookups_are_the_tables():
    """Byte r of W_j's lookups is the tables' value for byte j of row r, for
    random words and for every byte value in every byte slot."""
    rng = np.random.default_rng(3)
    rows = rng.integers(0, 1 << 32, (4, 4096), dtype=np.uint64)
    every = np.arange(256, dtype=np.uint64)
    for r in range(4):  # byte value v in byte slot j of row r (j = v % 4)
        rows[r, :256] = every << np.uint64(8 * (int(r) % 4))
    words = lut_quad(*rows)
    for j in range(4):
        for r in range(4):
            byte = ((rows[r] >> np.uint64(8 * j)) & np.uint64(0xFF)).astype(np.int64)
            got = [((w >> np.uint64(8 * r)) & np.uint64(0xFF)).astype(np.int64) for w in words[j]]
            assert np.array_equal(got[0], BYTE1_HIGH[byte >> 4] & BYTE1_LOW[byte & 15])
            assert np.array_equal(got[1], BYTE2_HIGH[byte >> 4])
            assert np.array_equal(got[2], LEAD_FLAGS[byte >> 4])
