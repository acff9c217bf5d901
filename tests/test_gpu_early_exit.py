"""Early stop of the single-buffer kernels on invalid input.  With early
exit on (utf8_set_early_exit), warps of the validation kernel poll the result
byte and stop once another warp has cleared it; warps of the location kernel
always stop once the smallest marked position lies before their next tile.
These buffers are large enough that every warp's run of tiles spans several
polls (at least 16 KiB per warp).  In both settings results must equal the
oracle's wherever the errors lie, and the result byte must be reset by every
call; with early exit on, an error at the front of a 1 GiB buffer must be
rejected in a fraction of the time a full pass takes.  Needs a GPU."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

N = 256 << 20


@pytest.fixture(params=[False, True], ids=["early_exit_off", "early_exit_on"])
def early_exit(request):
    before = u.utf8_set_early_exit(request.param)
    assert '"early_exit": %d' % int(request.param) in u.utf8_config_json()
    yield request.param
    u.utf8_set_early_exit(before)


@pytest.fixture(scope="module")
def clean():
    buf = synth.fill(N, synth.CJK, seed=synth.SEED_BASE + 7100)
    return buf, torch.from_numpy(buf).cuda()


def with_errors(buf, t, positions, kind="stray", seed=0):
    """Injects one error of `kind` near each position, on the host copy and
    the device copy alike; returns the saved windows to undo it."""
    rng = np.random.default_rng(seed)
    saved = []
    for at in positions:
        lo = max(at - 64, 0)
        window = buf[lo:lo + 128].copy()
        saved.append((lo, window.copy()))
        synth.inject_any(window, kind, rng, at=at - lo)
        buf[lo:lo + 128] = window
        t[lo:lo + 128] = torch.from_numpy(window).cuda()
    return saved


def undo(buf, t, saved):
    for lo, window in reversed(saved):
        buf[lo:lo + window.size] = window
        t[lo:lo + window.size] = torch.from_numpy(window).cuda()


@pytest.mark.parametrize("where", ["first_byte", "first_kib", "middle", "last_warp",
                                   "every_16k", "last_bytes"])
def test_invalid_buffers_match_oracle(clean, where, early_exit):
    buf, t = clean
    positions = {
        "first_byte": [0],
        "first_kib": [700],
        "middle": [N // 2 + 12345],
        "last_warp": [N - 100_000],
        "every_16k": list(range(5000, N - 200, 16 << 10)),
        "last_bytes": [N - 70],
    }[where]
    saved = with_errors(buf, t, positions, seed=len(positions))
    try:
        want_valid, want_loc = oracle.valid(buf), oracle.locate(buf)
        assert not want_valid
        assert u.utf8_validate(t) is False
        out = torch.full((1,), 7, dtype=torch.uint8, device="cuda")
        u.utf8_validate_async(t, out)
        assert int(out.item()) == 0
        assert u.utf8_locate_error(t) == want_loc
    finally:
        undo(buf, t, saved)
    assert u.utf8_validate(t) is True  # the result byte is reset by each call
    assert u.utf8_locate_error(t) == (N, 0)


def test_random_bytes(early_exit):
    rng = np.random.default_rng(5)
    buf = rng.integers(0, 256, N, dtype=np.uint8)
    t = torch.from_numpy(buf).cuda()
    assert u.utf8_validate(t) is False
    assert u.utf8_locate_error(t) == oracle.locate(buf)


def test_first_error_late_in_first_warp(clean, early_exit):
    """Warp 0 finds its error last (its run ends there), while the warps after
    it each hold errors in their first tiles: the location stays warp 0's."""
    buf, t = clean
    warps = 152 * 2 * 8
    run = N // warps
    positions = [run - 600] + [k * run + 200 for k in range(1, warps, 3)]
    saved = with_errors(buf, t, positions, kind="overlong", seed=9)
    try:
        want = oracle.locate(buf)
        assert want[0] < run and want[1] == 4
        assert u.utf8_locate_error(t) == want
        assert u.utf8_validate(t) is False
    finally:
        undo(buf, t, saved)


def test_host_path_error_in_first_chunk(clean, early_exit):
    buf, _ = clean
    pinned = torch.empty(N, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = buf
    pinned.numpy()[100] = 0xFF
    assert u.utf8_validate_host(pinned) is False
    pinned.numpy()[100] = buf[100]
    assert u.utf8_validate_host(pinned) is True


def kernel_ms(fn, stream, reps=7):
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        stream.synchronize()
        times.append(a.elapsed_time(b))
    return sorted(times)[reps // 2]


def test_error_at_front_stops_early():
    before = u.utf8_set_early_exit(True)
    try:
        front_error_timings()
    finally:
        u.utf8_set_early_exit(before)


def front_error_timings():
    n = 1 << 30
    buf = synth.fill(n, synth.CJK, seed=synth.SEED_BASE + 7200)
    t = torch.from_numpy(buf).cuda()
    out = torch.empty(1, dtype=torch.uint8, device="cuda")
    loc = torch.empty(2, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    for _ in range(3):
        u.utf8_validate_async(t, out, stream=s)
    s.synchronize()
    full = kernel_ms(lambda: u.utf8_validate_async(t, out, stream=s), s)
    full_loc = kernel_ms(lambda: u.utf8_locate_error_async(t, loc, stream=s), s)
    assert int(out.item()) == 1
    t[50] = 0xFF
    buf[50] = 0xFF
    early = kernel_ms(lambda: u.utf8_validate_async(t, out, stream=s), s)
    early_loc = kernel_ms(lambda: u.utf8_locate_error_async(t, loc, stream=s), s)
    assert int(out.item()) == 0
    pos, rule = u.error_info_fields(loc)
    assert (int(pos[0]), int(rule[0])) == oracle.locate(buf)
    assert early < 0.5 * full, (early, full)
    assert early_loc < 0.5 * full_loc, (early_loc, full_loc)


def test_graph_keeps_the_setting_of_its_capture(clean):
    """A graph captured with early exit on replays the polling kernel after the
    setting is switched off, and still gives the oracle's answers as the
    buffer changes under it."""
    buf, t = clean
    out = torch.empty(1, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    before = u.utf8_set_early_exit(True)
    try:
        u.utf8_validate_async(t, out, stream=s)  # first call on this device outside capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            u.utf8_validate_async(t, out, stream=s)
    finally:
        u.utf8_set_early_exit(False)
    try:
        for positions in ([], [123], [N // 3], [N - 50]):
            saved = with_errors(buf, t, positions, seed=3)
            try:
                out.fill_(7)
                g.replay()
                torch.cuda.synchronize()
                assert int(out.item()) == int(oracle.valid(buf)), positions
            finally:
                undo(buf, t, saved)
    finally:
        u.utf8_set_early_exit(before)


def test_every_length_and_alignment_with_early_exit_on():
    """The polling kernel on short and medium buffers (no poll, or a few), at
    every alignment, valid and with injected errors, against the oracle."""
    rng = np.random.default_rng(71)
    pool = torch.zeros(8 << 20, dtype=torch.uint8, device="cuda")
    before = u.utf8_set_early_exit(True)
    try:
        sizes = list(range(0, 80)) + [int(x) for x in rng.integers(80, 6 << 20, 60)]
        for n in sizes:
            text = synth.fill(n, int(rng.integers(0, 7)), seed=n + 3)
            if n and rng.random() < 0.6:
                for _ in range(int(rng.integers(1, 4))):
                    synth.inject_any(text, synth.ERROR_CLASSES[int(rng.integers(0, 7))], rng)
            want = oracle.valid(text)
            for shift in (0, 1, 7, 15):
                if n:
                    pool[shift:shift + n] = torch.from_numpy(text).cuda()
                assert u.utf8_validate(pool[shift:shift + n]) == want, (n, shift)
    finally:
        u.utf8_set_early_exit(before)
