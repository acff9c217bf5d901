"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle,
bit-exact, plus the per-position classification against the paper's Table 8
and the Table 7 lookup aid.  Needs a GPU (-m gpu)."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import lookup_aid
from conftest import read_hex_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

CLASS_BYTES = np.frombuffer(bytes([0x00, 0x41, 0x7F, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0,
                                   0xC1, 0xC2, 0xDF, 0xE0, 0xE1, 0xEC, 0xED, 0xEE, 0xEF, 0xF0,
                                   0xF1, 0xF3, 0xF4, 0xF5, 0xFF]), dtype=np.uint8)


def dev(a) -> "torch.Tensor":
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def batch_flags(data: np.ndarray, offsets: np.ndarray) -> np.ndarray:
    d = dev(data) if data.size else torch.zeros(16, dtype=torch.uint8, device="cuda")
    o = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).cuda()
    out = u.utf8_validate_batch(d, o)
    return out.cpu().numpy()


def de_bruijn_256_2() -> np.ndarray:
    """A cyclic sequence in which every ordered byte pair occurs once."""
    k, n = 256, 2
    a = [0] * (k * n)
    seq = []

    def db(t, p):
        if t > n:
            if n % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            db(t + 1, p)
            for j in range(a[t - p] + 1, k):
                a[t] = j
                db(t + 1, t)

    db(1, 1)
    s = np.array(seq, dtype=np.uint8)
    return np.concatenate([s, s[:1]])  # linear form: all 65536 pairs


# --------------------------------------------------------------------------
# classification intermediates
# --------------------------------------------------------------------------
# The kernels' special-row bits, in the order of the paper's Table 8 bits.
PAPER_BIT_OF = ((0x01, 0x20), (0x02, 0x04), (0x04, 0x10), (0x08, 0x08), (0x10, 0x40))


def to_paper_bits(sc: np.ndarray) -> np.ndarray:
    out = np.zeros_like(sc)
    for ours, paper in PAPER_BIT_OF:
        out |= np.where(sc & ours, paper, 0).astype(sc.dtype)
    return out


def check_against_paper(buf: np.ndarray, sc: np.ndarray, cont: np.ndarray):
    """Per position of buf + 3 zeros (zeros before): the special-row bits
    equal the paper's (Table 7 through lookup_aid) except where an ASCII byte
    precedes a continuation (an error either way); cont bit 1 is
    'continuation', cont bit 0 is 'previous byte >= 0xC0, or exactly one of
    the two terms of must_be_2_3' (both terms hold only where a lead follows a
    4-byte lead, an error that position i-2 shows)."""
    zeros = np.zeros(3, np.uint8)
    padded = np.concatenate([buf, zeros])
    paper = lookup_aid.classify(padded, zeros)["special_cases"]
    must23 = lookup_aid.must_be_2_3_continuation(padded, zeros)
    prev1 = np.concatenate([zeros[:1], padded[:-1]])
    is_cont = (padded & 0xC0) == 0x80
    free = (prev1 < 0x80) & is_cont
    want_sc = to_paper_bits(sc)
    assert np.array_equal(np.where(free, 0, want_sc), np.where(free, 0, paper & 0x7C))
    assert np.array_equal((cont >> 1) & 1, is_cont.astype(np.uint8))
    prev2 = np.concatenate([zeros[:2], padded[:-2]])
    prev3 = np.concatenate([zeros, padded[:-3]])
    term2, term3 = prev2 >= 0xE0, prev3 >= 0xF0
    assert np.array_equal(must23 != 0, term2 | term3)  # the paper's must_be_2_3
    want = (prev1 >= 0xC0) | (term2 ^ term3)
    assert np.array_equal(cont & 1, want.astype(np.uint8))
    # where both terms hold, position i-2 is an error: a lead right after a
    # 4-byte lead, where a continuation is expected
    both = np.flatnonzero(term2 & term3)
    assert np.all((cont[both - 2] & 1) == 1) and np.all(((cont[both - 2] >> 1) & 1) == 0)
    assert not np.any(cont & 0xFC) and not np.any(sc & 0xE0)


def test_table8_special_cases(golden_dir):
    rows = dict(read_hex_rows(os.path.join(golden_dir, "table8.txt")))
    buf = np.frombuffer(rows["input"], dtype=np.uint8)
    sc, cont = u.utf8_classify_debug(dev(buf))
    sc, cont = sc.cpu().numpy()[:len(buf)], cont.cpu().numpy()[:len(buf)]
    paper = np.frombuffer(rows["special_cases"], np.uint8)
    # Table 8's text is valid: no special row matches, and bit 7 of the
    # paper's special_cases (two continuations in a row) marks exactly the
    # positions that are continuations and expect one without a lead just
    # before (must_be_2_3)
    assert not np.any(sc) and not np.any(paper & 0x7F)
    assert np.array_equal(cont & 1, (cont >> 1) & 1)
    prev1 = np.concatenate([[0], buf[:-1]]).astype(np.uint8)
    assert np.array_equal((paper >> 7) & 1, ((cont >> 1) & 1) & (prev1 < 0xC0))


def test_classification_every_byte_pair():
    seq = de_bruijn_256_2()
    pairs = set(zip(seq[:-1].tolist(), seq[1:].tolist()))
    assert len(pairs) == 65536
    sc, cont = u.utf8_classify_debug(dev(seq))
    sc, cont = sc.cpu().numpy(), cont.cpu().numpy()
    check_against_paper(seq, sc, cont)
    pair = lookup_aid.pair_special_cases()[seq[:-1], seq[1:]] & 0x7C
    free = (seq[:-1] < 0x80) & ((seq[1:] & 0xC0) == 0x80)
    assert np.array_equal(np.where(free, 0, to_paper_bits(sc[1:len(seq)])), np.where(free, 0, pair))


@pytest.mark.parametrize("shift", [0, 1, 5, 15])
def test_classification_random_misaligned(shift):
    rng = np.random.default_rng(shift)
    buf = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, 100_000)]
    t = torch.zeros(buf.size + 16, dtype=torch.uint8, device="cuda")
    t[shift:shift + buf.size] = dev(buf)
    sc, cont = u.utf8_classify_debug(t[shift:shift + buf.size])
    check_against_paper(buf, sc.cpu().numpy(), cont.cpu().numpy())


# --------------------------------------------------------------------------
# exhaustive short strings
# --------------------------------------------------------------------------
@pytest.mark.parametrize("length", [1, 2, 3])
def test_every_string_up_to_3_bytes(length):
    n = 256 ** length
    r = np.arange(n, dtype=np.uint32)
    data = np.stack([(r >> (8 * k)) & 255 for k in range(length)], axis=1).astype(np.uint8)
    offsets = np.arange(0, n * length + 1, length, dtype=np.int64)
    got = batch_flags(data.reshape(-1), offsets)
    assert np.array_equal(got, oracle.valid_all(length))


def _valid_count_by_lead_len4() -> np.ndarray:
    """Closed-form number of valid 4-byte strings for each first byte, from
    the Table 1 ranges (V(n): valid strings of n bytes)."""
    v = [1, 128, 18304, 2650112]
    out = np.zeros(256, dtype=np.int64)
    for b in range(256):
        if b < 0x80:
            out[b] = v[3]
        elif 0xC2 <= b <= 0xDF:
            out[b] = 64 * v[2]
        elif b == 0xE0 or b == 0xED:
            out[b] = 32 * 64 * v[1]
        elif 0xE1 <= b <= 0xEF:
            out[b] = 64 * 64 * v[1]
        elif b == 0xF0:
            out[b] = 48 * 64 * 64
        elif 0xF1 <= b <= 0xF3:
            out[b] = 64 * 64 * 64
        elif b == 0xF4:
            out[b] = 16 * 64 * 64
    return out


def test_every_4_byte_string_count_by_lead():
    want = _valid_count_by_lead_len4()
    assert want.sum() == 383270912
    per = 1 << 24  # strings per first byte
    tail = torch.arange(per, dtype=torch.int32, device="cuda")
    body = torch.stack([(tail >> (8 * k)) & 255 for k in range(3)], dim=1).to(torch.uint8)
    offsets = torch.arange(0, 4 * per + 1, 4, dtype=torch.int64, device="cuda")
    got = np.zeros(256, dtype=np.int64)
    for b in range(256):
        data = torch.cat([torch.full((per, 1), b, dtype=torch.uint8, device="cuda"), body], dim=1)
        flags = u.utf8_validate_batch(data.reshape(-1), offsets)
        got[b] = int(flags.sum(dtype=torch.int64))
    assert np.array_equal(got, want)
    assert got[0xC0:].sum() == oracle.count_valid(4, lead_min=0xC0)


def test_every_4_byte_string_with_a_lead_flag_by_flag():
    """Every 4-byte string whose first byte is a lead (0xC0..0xFF), flag by
    flag against the oracle on the same bytes.  (A first byte below 0xC0 is
    ASCII, whose string is valid iff its last three bytes are, a case the
    every-3-byte-string test covers flag by flag, or a continuation, which is
    always invalid: the per-lead counts above check both.)"""
    per = 1 << 24
    tails = np.arange(per, dtype=np.uint32).view(np.uint8).reshape(per, 4)[:, :3]
    host = np.empty((per, 4), dtype=np.uint8)
    host[:, 1:] = tails
    offsets = np.arange(0, 4 * per + 1, 4, dtype=np.int64)
    o = torch.from_numpy(offsets).cuda()
    threads = max(len(os.sched_getaffinity(0)), 1)
    for b in range(0xC0, 0x100):
        host[:, 0] = b
        flags = u.utf8_validate_batch(dev(host.reshape(-1)), o).cpu().numpy()
        want = oracle.valid_batch(host.reshape(-1), offsets, threads=threads)
        if not np.array_equal(flags, want):
            bad = np.flatnonzero(flags != want)[:5]
            pytest.fail(f"lead {b:#04x}: {bad.size} strings differ, e.g. "
                        f"{[bytes(host[i]).hex() for i in bad]}")


# --------------------------------------------------------------------------
# single-buffer API: every length and alignment, errors at tile boundaries
# --------------------------------------------------------------------------
def test_every_length_and_alignment_single_api():
    rng = np.random.default_rng(1)
    pool = dev(np.zeros(8192, np.uint8))
    for n in list(range(0, 130)) + list(range(130, 4200, 37)):
        text = synth.fill(n, synth.UNIFORM, seed=n) if rng.random() < 0.5 else \
            CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, n)]
        for shift in range(16):
            pool[shift:shift + n] = dev(text) if n else pool[:0]
            got = u.utf8_validate(pool[shift:shift + n])
            assert got == oracle.valid(text), (n, shift)


def test_every_length_and_alignment_batch_api():
    rng = np.random.default_rng(2)
    lens = np.concatenate([np.arange(0, 300), rng.integers(0, 5000, 2000)])
    strings = []
    for i, n in enumerate(lens):
        if i % 3 == 0:
            strings.append(CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, n)])
        else:
            s = synth.fill(int(n), synth.UNIFORM, seed=i)
            if i % 3 == 1 and n:
                synth.inject_any(s, synth.ERROR_CLASSES[i % 7], rng)
            strings.append(s)
    offsets = synth.offsets_of([s.size for s in strings])
    data = np.concatenate(strings)
    for shift in (0, 1, 7, 13):
        shifted = np.concatenate([np.full(shift, 0x41, np.uint8), data])
        got = batch_flags(shifted, offsets + shift)
        assert np.array_equal(got, oracle.valid_batch(data, offsets)), shift


@pytest.mark.parametrize("model", [synth.CJK, synth.EMOJI, synth.LATIN, synth.ASCII])
def test_errors_around_tile_and_chunk_boundaries(model):
    n = 3 << 20
    base = synth.fill(n, model, seed=model + 100)
    assert u.utf8_validate(dev(base))
    rng = np.random.default_rng(model)
    periods = [512, 1024, 2048, 4096, 65536, n // 7]
    for period in periods:
        for k in (1, 2, 5):
            for d in range(0, 4):
                at = k * period - d
                if at >= n:
                    continue
                buf = base.copy()
                kind = synth.ERROR_CLASSES[int(rng.integers(0, 6))]
                pos = synth.inject_any(buf, kind, rng, at=at)
                assert pos is not None
                assert u.utf8_validate(dev(buf)) == oracle.valid(buf), (period, k, d, kind)


def test_every_error_class_every_model():
    rng = np.random.default_rng(9)
    for model in range(7):
        base = synth.fill(200_000, model, seed=model)
        for kind in synth.ERROR_CLASSES:
            buf = base.copy()
            if synth.inject(buf, kind, rng) is None:
                continue
            assert u.utf8_validate(dev(buf)) == oracle.valid(buf) == False, (model, kind)  # noqa: E712


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def test_workload_1mib():
    bufs, labels = synth.workload_1mib()
    got = [u.utf8_validate(dev(b)) for b in bufs]
    assert got == [oracle.valid(b) for b in bufs] == [True] + [False] * 7, labels


@pytest.mark.parametrize("variant", synth.VARIANTS_1GIB)
def test_workload_1gib(variant):
    n = 1 << 30
    seed = synth.SEED_BASE + 1000 + synth.VARIANTS_1GIB.index(variant)
    buf = synth.fill_variant(n, variant, seed)
    t = dev(buf)
    assert u.utf8_validate(t) == oracle.valid(buf) == True  # noqa: E712
    tail = np.frombuffer(synth.tail_error_bytes(seed), np.uint8)
    t[-3:] = dev(tail)
    buf[-3:] = tail
    assert u.utf8_validate(t) == oracle.valid(buf) == False  # noqa: E712


def test_workload_batch_1m():
    data, offsets, bad = synth.workload_batch_1m()
    got = batch_flags(data, offsets)
    want = oracle.valid_batch(data, offsets, threads=os.cpu_count() or 1)
    assert np.array_equal(got, want)
    assert set(np.nonzero(want == 0)[0]) == set(bad.tolist())


def test_workload_heavy_skew():
    data, offsets, bad = synth.workload_heavy_skew()
    assert offsets[-1] > (3 << 30)
    got = batch_flags(data, offsets)
    want = oracle.valid_batch(data, offsets, threads=os.cpu_count() or 1)
    assert np.array_equal(got, want)
    assert (want == 0).sum() >= 1


# --------------------------------------------------------------------------
# other entry points
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 5, 4096, (64 << 20) + 12345, (130 << 20) + 7])
def test_host_path(n):
    buf = synth.fill(n, synth.UNIFORM, seed=n) if n else np.zeros(0, np.uint8)
    assert u.utf8_validate_host(buf) == oracle.valid(buf)
    if n > 10:
        bad = buf.copy()
        bad[n // 2] = 0xFF
        assert not u.utf8_validate_host(bad)
        pinned = torch.from_numpy(bad).pin_memory()
        assert not u.utf8_validate_host(pinned)
        buf2 = buf.copy()
        buf2[-3:] = np.frombuffer(b"\xf0\x9f\x98", np.uint8)
        assert u.utf8_validate_host(buf2) == oracle.valid(buf2)


def test_host_path_small_windows(monkeypatch):
    """Several staging windows, each with a halo tile copied from the host."""
    monkeypatch.setenv("UTF8GPU_STAGE_CHUNK", str(1 << 16))
    monkeypatch.setenv("UTF8GPU_STAGE_WINDOW", str(1 << 18))
    rng = np.random.default_rng(4)
    for n in [(1 << 18) - 1, 1 << 18, (1 << 20) + 333, 3 << 20]:
        buf = synth.fill(n, synth.CJK, seed=n)
        assert u.utf8_validate_host(buf)
        for at in [(1 << 18) - 2, (1 << 18) + 1, (1 << 16) - 1, n - 2]:
            if at >= n:
                continue
            bad = buf.copy()
            synth.inject_any(bad, "too_short", rng, at=at)
            assert u.utf8_validate_host(bad) == oracle.valid(bad), (n, at)


def test_async_in_cuda_graph():
    a = dev(synth.fill(5 << 20, synth.EMOJI, seed=1))
    out = torch.zeros(1, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        u.utf8_validate_async(a, out)  # first call outside capture (library set-up)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        u.utf8_validate_async(a, out)
    g.replay()
    torch.cuda.synchronize()
    assert out.item() == 1
    a[777] = 0xC0
    g.replay()
    torch.cuda.synchronize()
    assert out.item() == 0


def test_batch_in_cuda_graph():
    data, offsets, _ = synth.workload_batch_1m(count=20_000, total=20_000 * 537)
    d, o = dev(data), torch.from_numpy(offsets).cuda()
    out = torch.empty(offsets.size - 1, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        u.utf8_validate_batch(d, o, out)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        u.utf8_validate_batch(d, o, out)
    for trial in range(3):
        host = data.copy()
        synth.corrupt_strings(host, offsets, 0.02, seed=trial)
        d.copy_(torch.from_numpy(host))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.valid_batch(host, offsets))


def test_invalid_arguments():
    host = torch.zeros(16, dtype=torch.uint8)
    with pytest.raises(u.Utf8Error):
        u.utf8_validate(host)
    lib = u.lib()
    assert lib.utf8_validate(None, 5, None) is False
    assert lib.utf8_last_error() == u.UTF8_ERR_INVALID_ARG
    assert lib.utf8_validate(None, 0, None) is True
    assert lib.utf8_validate_batch(None, None, -1, None, None) == u.UTF8_ERR_INVALID_ARG
    assert lib.utf8_validate_batch(None, None, 0, None, None) == u.UTF8_OK
    buf = np.zeros(64, np.uint8)
    assert lib.utf8_validate(buf.ctypes.data, 64, None) is False  # host pointer
    assert lib.utf8_last_error() == u.UTF8_ERR_INVALID_ARG


def test_autotune_and_cache(tmp_path):
    u.utf8_autotune(1)
    cfg = u.utf8_config_json()
    assert '"rows"' in cfg and '"sm_count"' in cfg
    path = str(tmp_path / "tune.json")
    u.utf8_tune_cache_save(path)
    u.utf8_tune_cache_load(path)
    assert "entries" in open(path).read()
    base = synth.fill(3 << 20, synth.UNIFORM, seed=77)
    assert u.utf8_validate(dev(base))
    base[12345] = 0xBF
    assert not u.utf8_validate(dev(base))


def test_tiny_batches_around_group_sizes():
    """Batches of 1 .. 97 strings (boundary groups of 32 are checked
    together), with empty strings, all-empty batches and errors in the first
    and last strings; flags and error locations against the oracle."""
    rng = np.random.default_rng(23)
    for count in (1, 2, 3, 31, 32, 33, 63, 64, 65, 96, 97):
        for trial in range(3):
            lens = rng.integers(0, 40, count)
            if trial == 1:
                lens[rng.random(count) < 0.5] = 0
            if trial == 2 and count > 2:
                lens[:] = 0
                lens[count // 2] = 7
            strings = [synth.fill(int(n), synth.UNIFORM, seed=count * 10 + trial * 1000 + i)
                       for i, n in enumerate(lens)]
            if strings[0].size:
                strings[0][0] = 0x80
            if strings[-1].size:
                strings[-1][-1] = 0xE2
            offsets = synth.offsets_of([s.size for s in strings])
            data = np.concatenate(strings) if offsets[-1] else np.zeros(0, np.uint8)
            for shift in (0, 5):
                shifted = np.concatenate([np.full(shift, 0x41, np.uint8), data])
                got = batch_flags(shifted, offsets + shift)
                assert np.array_equal(got, oracle.valid_batch(data, offsets)), (count, trial, shift)
                d = dev(shifted) if shifted.size else torch.zeros(16, dtype=torch.uint8, device="cuda")
                pos, rule = u.error_info_fields(u.utf8_locate_errors_batch(
                    d, torch.from_numpy(offsets + shift).cuda()))
                want_pos, want_rule = oracle.locate_batch(data, offsets)
                assert np.array_equal(pos.cpu().numpy(), want_pos), (count, trial, shift)
                assert np.array_equal(rule.cpu().numpy(), want_rule), (count, trial, shift)


def test_batch_dense_errors_short_strings():
    """Many short strings with most tiles holding an error: boundary groups
    then open on tiles whose staged bytes already hold error words, and many
    windows end past a warp's last tile (one tile per warp), so the kernel's
    fallback reads run; errors sit in the first and last three bytes of
    strings too.  Flags and error locations against the oracle."""
    rng = np.random.default_rng(29)
    for shift in (0, 3, 9):
        lens = rng.integers(0, 48, 60_000)
        offsets = synth.offsets_of(lens)
        data = synth.fill_strings(offsets, synth.UNIFORM, seed=shift + 29).copy()
        # 30% of the non-empty strings get one byte replaced: in their first
        # three bytes, their last three or anywhere
        starts, n = offsets[:-1], lens
        hit = (n > 0) & (rng.random(n.size) < 0.3)
        kind = rng.integers(0, 3, n.size)
        r = rng.integers(0, 1 << 30, n.size)
        near = r % np.minimum(np.maximum(n, 1), 3)
        rel = np.where(kind == 0, near, np.where(kind == 1, n - 1 - near, r % np.maximum(n, 1)))
        at = (starts + rel)[hit]
        data[at] = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, at.size)]
        shifted = np.concatenate([np.full(shift, 0x41, np.uint8), data])
        want = oracle.valid_batch(data, offsets)
        assert (want == 0).mean() > 0.1
        assert np.array_equal(batch_flags(shifted, offsets + shift), want), shift
        pos, rule = u.error_info_fields(u.utf8_locate_errors_batch(
            dev(shifted), torch.from_numpy(offsets + shift).cuda()))
        want_pos, want_rule = oracle.locate_batch(data, offsets)
        assert np.array_equal(pos.cpu().numpy(), want_pos), shift
        assert np.array_equal(rule.cpu().numpy(), want_rule), shift


def test_check_offsets():
    ok = [[0, 3, 3, 10], [5], [0, 0, 0]]
    bad = [[0, 5, 3, 10], [-1, 2, 3], [0, 1, 2, 1]]
    for o in ok:
        u.utf8_check_offsets(torch.tensor(o, dtype=torch.int64, device="cuda"))
    for o in bad:
        with pytest.raises(u.Utf8Error) as e:
            u.utf8_check_offsets(torch.tensor(o, dtype=torch.int64, device="cuda"))
        assert e.value.code == 1
    big = torch.arange(0, 3_000_001, dtype=torch.int64, device="cuda")
    u.utf8_check_offsets(big)
    big[-1] = 17  # one decreasing pair at the very end (grid-stride coverage)
    with pytest.raises(u.Utf8Error):
        u.utf8_check_offsets(big)


def test_offsets_debug_mode_rejects_before_launch():
    """UTF8GPU_CHECK_OFFSETS=1 (read once per process, so in a child):
    the batch entry points refuse malformed offsets with status 1.  The
    offsets stay inside the data, so nothing out of range would be read even
    without the check."""
    import subprocess
    import sys
    code = (
        "import torch, paper_2010_03090_gb300 as u\n"
        "d = torch.zeros(16, dtype=torch.uint8, device='cuda')\n"
        "good = torch.tensor([0, 3, 3, 10], dtype=torch.int64, device='cuda')\n"
        "print(u.utf8_validate_batch(d, good).tolist())\n"
        "bad = torch.tensor([0, 5, 3, 10], dtype=torch.int64, device='cuda')\n"
        "for f in (u.utf8_validate_batch, u.utf8_locate_errors_batch):\n"
        "    try:\n"
        "        f(d, bad)\n"
        "        print('launched')\n"
        "    except u.Utf8Error as e:\n"
        "        print('rejected', e.code)\n")
    env = dict(os.environ, UTF8GPU_CHECK_OFFSETS="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split("\n")[:3] == ["[1, 1, 1]", "rejected 1", "rejected 1"], r.stdout


def test_batch_descriptor_graph_replays_other_batches():
    """One CUDA graph of utf8_validate_batch_desc, replayed after the device
    descriptor is rewritten: other pointers and another count each time."""
    rng = np.random.default_rng(61)
    batches = []
    for count in (1000, 37, 5000, 1):
        lens = rng.integers(0, 300, count)
        strings = []
        for i, n in enumerate(lens):
            s = synth.fill(int(n), synth.UNIFORM, seed=count + i)
            if i % 4 == 1 and n:
                synth.inject_any(s, synth.ERROR_CLASSES[i % 7], rng)
            strings.append(s)
        offsets = synth.offsets_of([s.size for s in strings])
        data = np.concatenate(strings) if offsets[-1] else np.zeros(1, np.uint8)
        d, o = dev(data), torch.from_numpy(offsets).cuda()
        out = torch.full((count,), 7, dtype=torch.uint8, device="cuda")
        batches.append((data, offsets, d, o, out))
    desc = torch.tensor(u.batch_desc_values(*batches[0][2:]), dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    u.utf8_validate_batch_desc(desc, stream=s)  # first call outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        u.utf8_validate_batch_desc(desc, stream=s)
    for data, offsets, d, o, out in batches:
        desc.copy_(torch.tensor(u.batch_desc_values(d, o, out), dtype=torch.int64))
        out.fill_(7)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.valid_batch(data[:offsets[-1]], offsets))
