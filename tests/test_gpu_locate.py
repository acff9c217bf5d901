"""GPU parity of the error location (utf8_locate_error*, through the C-ABI)
against the oracle's locate: the longest valid prefix and the Section 3 rule
of the next character must match exactly, for single buffers at every length
and alignment, errors straddling tile boundaries, several errors in one
buffer (the first wins), the 1 GiB buffers, and batches.  Needs a GPU."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

CLASS_BYTES = np.frombuffer(bytes([0x00, 0x41, 0x7F, 0x80, 0x8F, 0x90, 0x9F, 0xA0, 0xBF, 0xC0,
                                   0xC1, 0xC2, 0xDF, 0xE0, 0xE1, 0xEC, 0xED, 0xEE, 0xEF, 0xF0,
                                   0xF1, 0xF3, 0xF4, 0xF5, 0xF8, 0xFF]), dtype=np.uint8)
THREADS = os.cpu_count() or 1


def dev(a) -> "torch.Tensor":
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def locate_batch(data: np.ndarray, offsets: np.ndarray):
    d = dev(data) if data.size else torch.zeros(16, dtype=torch.uint8, device="cuda")
    o = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).cuda()
    pos, rule = u.error_info_fields(u.utf8_locate_errors_batch(d, o))
    return pos.cpu().numpy(), rule.cpu().numpy()


def text_with_errors(n: int, model: int, seed: int, errors: int) -> np.ndarray:
    buf = synth.fill(n, model, seed=seed)
    rng = np.random.default_rng(seed)
    for _ in range(errors):
        synth.inject_any(buf, synth.ERROR_CLASSES[int(rng.integers(0, 7))], rng)
    return buf


def test_every_length_and_alignment():
    rng = np.random.default_rng(11)
    pool = dev(np.zeros(8192, np.uint8))
    for n in list(range(0, 140)) + list(range(140, 4300, 41)):
        r = rng.random()
        if r < 0.4:
            text = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, n)]
        elif r < 0.8 and n:
            text = text_with_errors(n, synth.UNIFORM, seed=n, errors=1)
        else:
            text = synth.fill(n, synth.UNIFORM, seed=n)
        want = oracle.locate(text)
        for shift in range(16):
            pool[shift:shift + n] = dev(text) if n else pool[:0]
            assert u.utf8_locate_error(pool[shift:shift + n]) == want, (n, shift)


@pytest.mark.parametrize("model", [synth.CJK, synth.EMOJI, synth.LATIN, synth.ASCII,
                                   synth.UNIFORM])
def test_errors_around_tile_boundaries(model):
    n = 3 << 20
    base = synth.fill(n, model, seed=model + 200)
    assert u.utf8_locate_error(dev(base)) == (n, 0)
    rng = np.random.default_rng(model + 50)
    for period in (512, 1024, 2048, 4096, 65536, n // 7):
        for k in (1, 3):
            for d in range(0, 5):
                at = k * period - d
                if at >= n:
                    continue
                buf = base.copy()
                kind = synth.ERROR_CLASSES[int(rng.integers(0, 6))]
                assert synth.inject_any(buf, kind, rng, at=at) is not None
                got = u.utf8_locate_error(dev(buf))
                assert got == oracle.locate(buf), (period, k, d, kind)


def test_first_of_many_errors():
    for seed in range(6):
        buf = text_with_errors(1 << 21, seed % 7, seed=300 + seed, errors=40)
        assert u.utf8_locate_error(dev(buf)) == oracle.locate(buf), seed


def test_every_error_class_every_model():
    rng = np.random.default_rng(13)
    for model in range(7):
        base = synth.fill(300_000, model, seed=model + 7)
        for kind in synth.ERROR_CLASSES:
            buf = base.copy()
            if synth.inject(buf, kind, rng) is None:
                continue
            want = oracle.locate(buf)
            assert want[1] != 0
            assert u.utf8_locate_error(dev(buf)) == want, (model, kind)


@pytest.mark.parametrize("variant", synth.VARIANTS_1GIB)
def test_workload_1gib(variant):
    """At the full 1 GiB size, in the launch configuration the benchmark uses:
    the clean buffer, the truncated tail, and a second error in the middle."""
    n = 1 << 30
    seed = synth.SEED_BASE + 1000 + synth.VARIANTS_1GIB.index(variant)
    buf = synth.fill_variant(n, variant, seed)
    t = dev(buf)
    assert u.utf8_locate_error(t) == (n, 0)
    tail = np.frombuffer(synth.tail_error_bytes(seed), np.uint8)
    t[-3:] = dev(tail)
    buf[-3:] = tail
    want = oracle.locate(buf)
    assert want[1] == 2 and want[0] >= n - 3
    assert u.utf8_locate_error(t) == want
    rng = np.random.default_rng(seed)
    at = int(rng.integers(n // 3, 2 * n // 3))
    window = buf[at - 64:at + 64].copy()
    synth.inject_any(window, "stray", rng, at=64)
    t[at - 64:at + 64] = dev(window)
    buf[at - 64:at + 64] = window
    assert u.utf8_locate_error(t) == oracle.locate(buf)


def test_async_and_graph_match_sync():
    buf = text_with_errors(5 << 20, synth.CJK, seed=77, errors=3)
    t = dev(buf)
    want = oracle.locate(buf)
    out = u.utf8_locate_error_async(t)
    pos, rule = u.error_info_fields(out)
    assert (int(pos[0]), int(rule[0])) == want
    s = torch.cuda.Stream()
    out2 = torch.empty(2, dtype=torch.int64, device="cuda")
    u.utf8_locate_error_async(t, out2, stream=s)  # first call on this device outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        u.utf8_locate_error_async(t, out2, stream=s)
    for _ in range(3):
        out2.zero_()
        g.replay()
        torch.cuda.synchronize()
        pos, rule = u.error_info_fields(out2)
        assert (int(pos[0]), int(rule[0])) == want


def test_batch_random_short_strings():
    rng = np.random.default_rng(21)
    count = 300_000
    lens = rng.integers(0, 14, count)
    offsets = synth.offsets_of(lens)
    data = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, int(offsets[-1]))]
    pos, rule = locate_batch(data, offsets)
    want_pos, want_rule = oracle.locate_batch(data, offsets, threads=THREADS)
    assert np.array_equal(pos, want_pos)
    assert np.array_equal(rule, want_rule)


def test_batch_every_length_with_errors_and_shifts():
    rng = np.random.default_rng(22)
    lens = np.concatenate([np.arange(0, 300), rng.integers(0, 9000, 1500)])
    strings = []
    for i, n in enumerate(lens):
        s = synth.fill(int(n), synth.UNIFORM, seed=i + 5)
        if i % 2 == 0 and n:
            for _ in range(1 + i % 3):
                synth.inject_any(s, synth.ERROR_CLASSES[int(rng.integers(0, 7))], rng)
        strings.append(s)
    offsets = synth.offsets_of([s.size for s in strings])
    data = np.concatenate(strings)
    want = oracle.locate_batch(data, offsets)
    for shift in (0, 3, 9):
        shifted = np.concatenate([np.full(shift, 0xE2, np.uint8), data])
        pos, rule = locate_batch(shifted, offsets + shift)
        assert np.array_equal(pos, want[0]) and np.array_equal(rule, want[1]), shift


def test_batch_workload_1m():
    data, offsets, bad = synth.workload_batch_1m()
    pos, rule = locate_batch(data, offsets)
    want_pos, want_rule = oracle.locate_batch(data, offsets, threads=THREADS)
    assert np.array_equal(pos, want_pos)
    assert np.array_equal(rule, want_rule)
    assert set(np.nonzero(rule)[0].tolist()) == set(bad.tolist())


def test_batch_skewed_lengths():
    data, offsets, bad = synth.workload_heavy_skew(total=512 << 20, count=5000)
    pos, rule = locate_batch(data, offsets)
    want_pos, want_rule = oracle.locate_batch(data, offsets, threads=THREADS)
    assert np.array_equal(pos, want_pos)
    assert np.array_equal(rule, want_rule)


def test_invalid_arguments():
    t = dev(np.zeros(64, np.uint8))
    out = torch.empty(4, dtype=torch.int64, device="cuda")
    with pytest.raises(u.Utf8Error) as e:
        u.utf8_locate_error_async(t, (out.data_ptr() + 4, 2))  # misaligned record
    assert e.value.code == 1
    host = np.zeros(64, np.uint8)
    with pytest.raises(u.Utf8Error) as e:
        u.utf8_locate_error((host.ctypes.data, host.size))
    assert e.value.code == 1
    assert u.utf8_locate_error(t[:0]) == (0, 0)


def test_buffer_beyond_4gib():
    """A single 4.5 GiB buffer (positions past 2^32): validity and error
    location of the clean buffer and with an error past 4 GiB, in the launch
    configuration the benchmark uses; the oracle scans the same bytes."""
    n = (9 << 29) + 12345
    buf = synth.fill(n, synth.CJK, seed=99)
    t = dev(buf)
    assert u.utf8_validate(t) == oracle.valid(buf) == True  # noqa: E712
    assert u.utf8_locate_error(t) == (n, 0)
    rng = np.random.default_rng(4)
    at = (1 << 32) + 1000003
    window = buf[at - 64:at + 64].copy()
    synth.inject_any(window, "overlong", rng, at=64)
    t[at - 64:at + 64] = dev(window)
    buf[at - 64:at + 64] = window
    want = oracle.locate(buf)
    assert want[0] > (1 << 32) and want[1] == 4
    assert u.utf8_validate(t) == oracle.valid(buf) == False  # noqa: E712
    assert u.utf8_locate_error(t) == want


def test_batch_beyond_4gib():
    """A batch of about 4.5 GiB (Pareto lengths, CJK and emoji content) whose
    string offsets pass 2^32, with 2% of the strings corrupted, errors placed
    near 2 KiB and 64 KiB multiples: flags and error locations against the
    oracle, in the launch configuration the benchmark uses."""
    data, offsets, _ = synth.workload_heavy_skew(seed=synth.SEED_BASE + 3100, count=4000,
                                                   total=(9 << 29) + 777)
    assert offsets[-1] > (1 << 32)
    rng = np.random.default_rng(5)
    more = synth.corrupt_strings(data, offsets, 0.02, seed=91, at_boundaries=[2048, 65536])
    # strings that straddle or follow the 2^32 offset hold errors too
    late = np.nonzero(offsets[:-1] >= (1 << 32) - (64 << 20))[0]
    for i in late[::7]:
        lo, hi = int(offsets[i]), int(offsets[i + 1])
        if hi > lo:
            synth.inject_any(data, synth.ERROR_CLASSES[int(rng.integers(0, 7))], rng, lo, hi)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(offsets).cuda()
    flags = u.utf8_validate_batch(d, o).cpu().numpy()
    want = oracle.valid_batch(data, offsets, threads=THREADS)
    assert np.array_equal(flags.astype(bool), want.astype(bool))
    assert (~want.astype(bool)).sum() >= len(more) // 2
    pos, rule = u.error_info_fields(u.utf8_locate_errors_batch(d, o))
    want_pos, want_rule = oracle.locate_batch(data, offsets, threads=THREADS)
    assert np.array_equal(pos.cpu().numpy(), want_pos)
    assert np.array_equal(rule.cpu().numpy(), want_rule)
