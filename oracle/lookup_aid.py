"""The paper's ``lookup`` steps written out plainly (numpy, CPU) — TEST AID.

Part of the oracle package (test infrastructure; the product never imports
it).  It exists to pin two readings of the paper against what the paper
prints, independently of the CUDA path:

1. Section 6.1 / Table 7: each error pattern is a product of three byte-field
   sets (high nibble of the first byte, low nibble of the first byte, high
   nibble of the second byte).  ``derive_tables`` builds the three 16-entry
   tables from those pattern sets alone; the tests check that the result
   reproduces every lookup row of Table 8.
2. The bit positions.  Table 7 numbers its rows 0..7, but the values printed
   in Table 8 (e.g. ``byte_1_high`` = 0x02 for an ASCII first byte, 0x21 for
   a 0xC_ lead) fix a different assignment: TOO_SHORT 0x01, TOO_LONG 0x02,
   OVERLONG_3 0x04, TOO_LARGE 0x08, SURROGATE 0x10, OVERLONG_2 0x20,
   OVERLONG_4 + TOO_LARGE_1000 0x40, TWO_CONTS 0x80.  The boolean does not
   depend on the assignment; Table 8's is used so intermediates can be
   compared with the paper.

``lookup_valid`` runs the algorithm in the paper's order (Fig. 1
classification, the 3-4 byte check of Section 6.2, the incomplete-stream
check of Section 6.3, and the 64-byte ASCII blocks of Section 6.4) over
blocks of ``w`` bytes with a carried previous block.
"""
from __future__ import annotations

import numpy as np

TOO_SHORT = 0x01
TOO_LONG = 0x02
OVERLONG_3 = 0x04
TOO_LARGE = 0x08
SURROGATE = 0x10
OVERLONG_2 = 0x20
OVERLONG_4_OR_TOO_LARGE_1000 = 0x40
TWO_CONTS = 0x80

ANY = tuple(range(16))
_ASCII_HI = tuple(range(0x0, 0x8))     # 0xxx
_CONT_HI = tuple(range(0x8, 0xC))      # 10xx
_LEAD_HI = tuple(range(0xC, 0x10))     # 11xx

# Table 7, one row per bit: (first-byte high nibbles, first-byte low nibbles,
# second-byte high nibbles).  Each row is a product set.
TABLE7_PATTERNS = {
    # ASCII followed by a continuation: 0xxx.... 10xx....
    TOO_LONG: (_ASCII_HI, ANY, _CONT_HI),
    # a lead (11......) not followed by a continuation: 0....... or 11......
    TOO_SHORT: (_LEAD_HI, ANY, _ASCII_HI + _LEAD_HI),
    # 1100000x 10......  (C0, C1)
    OVERLONG_2: ((0xC,), (0x0, 0x1), _CONT_HI),
    # 11101101 101.....  (ED A0..BF)
    SURROGATE: ((0xE,), (0xD,), (0xA, 0xB)),
    # 11100000 100.....  (E0 80..9F)
    OVERLONG_3: ((0xE,), (0x0,), (0x8, 0x9)),
    # 11110000 1000....  (F0 80..8F) and 11110101..11111111 1000....
    OVERLONG_4_OR_TOO_LARGE_1000: ((0xF,), (0x0,) + tuple(range(0x5, 0x10)), (0x8,)),
    # 11110100..11111111 1001.... .. 1011....  (F4..FF 90..BF)
    TOO_LARGE: ((0xF,), tuple(range(0x4, 0x10)), (0x9, 0xA, 0xB)),
    # two continuations in a row (not an error by itself)
    TWO_CONTS: (_CONT_HI, ANY, _CONT_HI),
}


def derive_tables(patterns=TABLE7_PATTERNS):
    """Builds (byte_1_high, byte_1_low, byte_2_high) tables from Table 7."""
    t1h = np.zeros(16, dtype=np.uint8)
    t1l = np.zeros(16, dtype=np.uint8)
    t2h = np.zeros(16, dtype=np.uint8)
    for bit, (hi1, lo1, hi2) in patterns.items():
        for n in hi1:
            t1h[n] |= bit
        for n in lo1:
            t1l[n] |= bit
        for n in hi2:
            t2h[n] |= bit
    return t1h, t1l, t2h


TABLES = derive_tables()


def classify(block: np.ndarray, previous: np.ndarray, tables=TABLES) -> dict:
    """Fig. 1 on one block, with every intermediate vector of Table 8."""
    t1h, t1l, t2h = tables
    block = np.asarray(block, dtype=np.uint8)
    prev1 = np.concatenate([previous[-1:], block[:-1]]).astype(np.uint8)
    hi1 = prev1 >> 4
    lo1 = prev1 & 0x0F
    hi2 = block >> 4
    b1h = t1h[hi1]
    b1l = t1l[lo1]
    b2h = t2h[hi2]
    return {
        "input": block, "prev1": prev1,
        "prev1_high": hi1, "prev1_low": lo1, "input_high": hi2,
        "byte_1_high": b1h, "byte_1_low": b1l, "byte_2_high": b2h,
        "special_cases": b1h & b1l & b2h,
    }


def must_be_2_3_continuation(block: np.ndarray, previous: np.ndarray) -> np.ndarray:
    """Section 6.2: 0x80 where two continuations are expected in a row, i.e.
    where the byte two back is >= 0xE0 (a 3- or 4-byte lead) or the byte
    three back is >= 0xF0 (a 4-byte lead)."""
    both = np.concatenate([previous[-3:], block]).astype(np.int32)
    prev2 = both[1:-2]
    prev3 = both[0:-3]
    need = (prev2 >= 0xE0) | (prev3 >= 0xF0)
    return np.where(need, TWO_CONTS, 0).astype(np.uint8)


def is_incomplete(block: np.ndarray) -> bool:
    """Section 6.3: the block ends inside a character."""
    b = np.asarray(block, dtype=np.int32)
    return bool(b[-1] >= 0xC0 or b[-2] >= 0xE0 or b[-3] >= 0xF0)


def lookup_valid(buf, w: int = 64, tables=TABLES) -> bool:
    """The whole ``lookup`` algorithm over blocks of ``w`` bytes (w >= 3)."""
    data = np.frombuffer(bytes(buf), dtype=np.uint8) if not isinstance(buf, np.ndarray) \
        else np.asarray(buf, dtype=np.uint8).reshape(-1)
    previous = np.zeros(w, dtype=np.uint8)       # zeros at stream start
    prev_incomplete = False
    error = 0
    for start in range(0, data.size, w):
        block = np.zeros(w, dtype=np.uint8)      # a short last block is zero-padded
        chunk = data[start:start + w]
        block[:chunk.size] = chunk
        if int(np.bitwise_or.reduce(block)) < 0x80:
            # ASCII block: no classification, but the previous block must
            # not have ended inside a character.
            error |= int(prev_incomplete)
        else:
            sc = classify(block, previous, tables)["special_cases"]
            m = must_be_2_3_continuation(block, previous)
            error |= int(np.bitwise_or.reduce(sc ^ m))
        prev_incomplete = is_incomplete(block)
        previous = block
    error |= int(prev_incomplete)                # end of stream
    return error == 0


def pair_special_cases(tables=TABLES) -> np.ndarray:
    """special_cases for every (previous byte, current byte) pair, as a
    [256, 256] array indexed [prev1, input]."""
    t1h, t1l, t2h = tables
    p = np.arange(256, dtype=np.uint8)
    return (t1h[p >> 4] & t1l[p & 0x0F])[:, None] & t2h[p >> 4][None, :]


def lookup_valid_rows(rows: np.ndarray, tables=TABLES) -> np.ndarray:
    """``lookup`` on many strings of equal length at once (one string per row
    of a [N, L] uint8 array).  Each string is one zero-padded block with a
    zero previous block, i.e. the algorithm above with w >= L + 3; returns a
    bool per row."""
    t1h, t1l, t2h = tables
    rows = np.asarray(rows, dtype=np.uint8)
    n, length = rows.shape
    padded = np.zeros((n, length + 6), dtype=np.uint8)   # 3 zeros before, 3 after
    padded[:, 3:3 + length] = rows
    cur = padded[:, 3:]
    prev1 = padded[:, 2:-1]
    prev2 = padded[:, 1:-2].astype(np.int32)
    prev3 = padded[:, 0:-3].astype(np.int32)
    sc = t1h[prev1 >> 4] & t1l[prev1 & 0x0F] & t2h[cur >> 4]
    m = np.where((prev2 >= 0xE0) | (prev3 >= 0xF0), TWO_CONTS, 0).astype(np.uint8)
    return np.bitwise_or.reduce(sc ^ m, axis=1) == 0
