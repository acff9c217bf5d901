"""Chunked validation (GPU): a buffer cut into chunks at arbitrary points
(including inside characters, empty chunks, chunks shorter than 3 bytes,
any alignment) gives the same result as the whole buffer, through the
stateless chunk call and through the device-resident stream state."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

CLASS = np.frombuffer(bytes([0x41, 0x80, 0x90, 0xA0, 0xBF, 0xC1, 0xC3, 0xE0, 0xE9, 0xED, 0xF0,
                             0xF4, 0xF5, 0x00]), np.uint8)


def _cuts(n, rng):
    k = int(rng.integers(0, 12))
    pts = sorted(set([0, n] + [int(x) for x in rng.integers(0, n + 1, k)]))
    if rng.random() < 0.3 and n > 2:  # force tiny chunks
        a = int(rng.integers(0, n - 2))
        pts = sorted(set(pts + [a, a + 1, a + 2]))
    return pts


def _buffers(rng):
    out = []
    for i in range(160):
        n = int(rng.integers(0, 3000)) if i % 4 else int(rng.integers(0, 40))
        if i % 3 == 0:
            b = CLASS[rng.integers(0, CLASS.size, n)]
        else:
            b = synth.fill(n, synth.UNIFORM, seed=i)
            if i % 3 == 1 and n:
                synth.inject_any(b, synth.ERROR_CLASSES[i % 7], rng)
        out.append(b)
    big = synth.fill(5 << 20, synth.CJK, seed=5)
    out.append(big)
    bad = big.copy()
    synth.inject(bad, "too_short", rng, at=(1 << 20) - 1)
    out.append(bad)
    return out


def test_chunks_equal_whole_buffer():
    rng = np.random.default_rng(3)
    flag = torch.ones(1, dtype=torch.uint8, device="cuda")
    pool = torch.zeros((6 << 20) + 64, dtype=torch.uint8, device="cuda")
    for b in _buffers(rng):
        want = oracle.valid(b)
        pts = _cuts(b.size, rng)
        flag.fill_(1)
        for k in range(len(pts) - 1):
            lo, hi = pts[k], pts[k + 1]
            shift = int(rng.integers(0, 16))
            pool[shift:shift + hi - lo] = torch.from_numpy(b[lo:hi].copy()).cuda()
            u.utf8_validate_chunk(pool[shift:shift + hi - lo], bytes(b[max(0, lo - 3):lo]),
                                  k == len(pts) - 2, flag)
        if len(pts) == 1:  # empty buffer: only the final (empty) chunk
            u.utf8_validate_chunk(pool[:0], b"", True, flag)
        torch.cuda.synchronize()
        assert flag.item() == want, (b.size, pts)


def test_stream_state_equals_whole_buffer():
    rng = np.random.default_rng(4)
    h = u.utf8_stream_create()
    out = torch.zeros(1, dtype=torch.uint8, device="cuda")
    ring = torch.zeros((6 << 20) + 64, dtype=torch.uint8, device="cuda")  # one reused buffer
    try:
        for b in _buffers(rng):
            u.utf8_stream_reset(h)
            pts = _cuts(b.size, rng)
            for k in range(len(pts) - 1):
                lo, hi = pts[k], pts[k + 1]
                shift = int(rng.integers(0, 16))
                ring[shift:shift + hi - lo] = torch.from_numpy(b[lo:hi].copy()).cuda()
                u.utf8_stream_update(h, ring[shift:shift + hi - lo])
            u.utf8_stream_finish(h, out)
            torch.cuda.synchronize()
            assert out.item() == oracle.valid(b), (b.size, pts)
    finally:
        u.utf8_stream_destroy(h)


def test_shards_share_one_flag():
    """Shards of one buffer (each given the 3 bytes before it) validated on
    separate streams into one shared flag."""
    rng = np.random.default_rng(5)
    base = synth.fill(32 << 20, synth.UNIFORM, seed=9)
    for trial in range(4):
        b = base.copy()
        if trial:
            synth.inject_any(b, synth.ERROR_CLASSES[trial], rng, at=int(rng.integers(0, b.size)))
        d = torch.from_numpy(b).cuda()
        cuts = np.linspace(0, b.size, 9).astype(int)
        flag = torch.ones(1, dtype=torch.uint8, device="cuda")
        streams = [torch.cuda.Stream() for _ in range(len(cuts) - 1)]
        torch.cuda.synchronize()
        for k, st in enumerate(streams):
            lo, hi = int(cuts[k]), int(cuts[k + 1])
            u.utf8_validate_chunk(d[lo:hi], bytes(b[max(0, lo - 3):lo]), k == len(streams) - 1,
                                  flag, stream=st)
        torch.cuda.synchronize()
        assert flag.item() == oracle.valid(b)


def test_stream_sequence_in_cuda_graph():
    """reset, a run of updates and finish captured once in a CUDA graph and
    replayed: the replays follow the bytes in the buffer at replay time."""
    n, chunk = 3 << 20, 256 << 10
    buf = synth.fill(n, synth.CJK, seed=31)
    d = torch.from_numpy(buf).cuda()
    out = torch.zeros(1, dtype=torch.uint8, device="cuda")
    h = u.utf8_stream_create()
    try:
        s = torch.cuda.Stream()
        u.utf8_stream_reset(h, stream=s)  # first calls outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            u.utf8_stream_reset(h, stream=s)
            for i in range(0, n, chunk):
                u.utf8_stream_update(h, d[i:i + chunk], stream=s)
            u.utf8_stream_finish(h, out, stream=s)
        g.replay()
        torch.cuda.synchronize()
        assert int(out.item()) == 1 == oracle.valid(buf)
        bad = buf.copy()
        synth.inject_any(bad, "surrogate", np.random.default_rng(3), at=5 * chunk - 1)
        d.copy_(torch.from_numpy(bad))
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(out.item()) == int(oracle.valid(bad)) == 0
    finally:
        u.utf8_stream_destroy(h)


def test_chunks_on_both_sides_of_the_tile_switch():
    """Chunks checked in 4 KiB tiles and chunks small enough (about 2.4 MB
    and less on 152 SMs) to be checked in 1 KiB tiles, cut inside
    characters, with errors in either kind of chunk, at the cut and at the
    end; stateless chunks and the stream state both equal the whole buffer."""
    rng = np.random.default_rng(17)
    base = synth.fill(40 << 20, synth.UNIFORM, seed=17)
    cuts = [0, 3, (12 << 20) + 1, (12 << 20) + 5001, (30 << 20) + 7, (31 << 20) + 2, base.size]
    h = u.utf8_stream_create()
    try:
        for bad_at in (None, 5 << 20, (12 << 20) + 2, (20 << 20) + 11, (30 << 20) + 5,
                       (30 << 20) + 100, base.size - 2):
            b = base.copy()
            if bad_at is not None:
                synth.inject_any(b, synth.ERROR_CLASSES[int(rng.integers(0, 7))], rng, at=bad_at)
            want = oracle.valid(b)
            d = torch.from_numpy(b).cuda()
            flag = torch.ones(1, dtype=torch.uint8, device="cuda")
            for k in range(len(cuts) - 1):
                lo, hi = cuts[k], cuts[k + 1]
                u.utf8_validate_chunk(d[lo:hi], bytes(b[max(0, lo - 3):lo]), k == len(cuts) - 2,
                                      flag)
            u.utf8_stream_reset(h)
            for k in range(len(cuts) - 1):
                u.utf8_stream_update(h, d[cuts[k]:cuts[k + 1]])
            out = torch.zeros(1, dtype=torch.uint8, device="cuda")
            u.utf8_stream_finish(h, out)
            torch.cuda.synchronize()
            assert flag.item() == want, bad_at
            assert out.item() == want, bad_at
    finally:
        u.utf8_stream_destroy(h)
