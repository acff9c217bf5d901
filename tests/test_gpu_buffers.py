"""utf8_validate_buffers_async: many independent device buffers in one
launch, each checked as utf8_validate checks it.  Flags against the CPU
oracle, flag by flag.  Needs a GPU (-m gpu)."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

CHUNK = 128 << 10  # the launch's chunk of work
CLASS_BYTES = np.frombuffer(bytes([0x00, 0x41, 0x80, 0x8F, 0x90, 0xBF, 0xC0, 0xC2, 0xDF, 0xE0,
                                   0xE1, 0xED, 0xEF, 0xF0, 0xF1, 0xF4, 0xF5, 0xFF]), np.uint8)


def dev(a) -> "torch.Tensor":
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def make_buffers(rng, count, max_len):
    bufs = []
    for i in range(count):
        n = int(rng.integers(0, max_len)) if i % 5 else int(rng.integers(0, 40))
        b = synth.fill(n, [synth.UNIFORM, synth.CJK, synth.ASCII, synth.EMOJI][i % 4], seed=i + 7)
        if n and rng.random() < 0.4:
            synth.inject_any(b, synth.ERROR_CLASSES[i % 7], rng)
        bufs.append(b)
    return bufs


def placed(bufs, rng):
    """The buffers at random 0..15-byte offsets inside one device pool."""
    offs, total = [], 0
    for b in bufs:
        total += int(rng.integers(0, 16))
        offs.append(total)
        total += b.size
    pool = torch.zeros(total + 16, dtype=torch.uint8, device="cuda")
    views = []
    for b, o in zip(bufs, offs):
        if b.size:
            pool[o:o + b.size] = dev(b)
        views.append(pool[o:o + b.size])
    return pool, views


@pytest.mark.parametrize("count", [1, 2, 7, 63, 64, 65, 130])
def test_flags_against_oracle(count):
    rng = np.random.default_rng(count)
    bufs = make_buffers(rng, count, 300_000)
    pool, views = placed(bufs, rng)
    got = u.utf8_validate_buffers_async(views).cpu().numpy()
    want = np.array([oracle.valid(b) for b in bufs], np.uint8)
    assert np.array_equal(got, want), count
    assert 0 < want.sum() < count or count < 3


def test_errors_at_chunk_boundaries():
    rng = np.random.default_rng(5)
    base = synth.fill(6 * CHUNK + 1000, synth.CJK, seed=3)
    bufs = []
    for k in range(1, 6):
        for d in (-4, -3, -1, 0, 1, 2, 3):
            b = base.copy()
            b[k * CHUNK + d] = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size)]
            bufs.append(b)
    bufs.append(base)
    for shift in (0, 1, 13):
        pool = torch.zeros(len(bufs) * (base.size + 32), dtype=torch.uint8, device="cuda")
        views = []
        for i, b in enumerate(bufs):
            o = i * (base.size + 32) + shift
            pool[o:o + b.size] = dev(b)
            views.append(pool[o:o + b.size])
        got = u.utf8_validate_buffers_async(views).cpu().numpy()
        want = np.array([oracle.valid(b) for b in bufs], np.uint8)
        assert np.array_equal(got, want), shift


def test_same_flags_as_single_calls_and_graph_replay():
    rng = np.random.default_rng(9)
    bufs = make_buffers(rng, 20, 2_000_000)
    pool, views = placed(bufs, rng)
    single = [int(u.utf8_validate(v)) for v in views]
    out = torch.zeros(len(views), dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        u.utf8_validate_buffers_async(views, out, stream=s)
    s.synchronize()
    assert out.cpu().numpy().tolist() == single
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        u.utf8_validate_buffers_async(views, out, stream=s)
    for _ in range(3):
        out.fill_(7)
        g.replay()
        torch.cuda.synchronize()
        assert out.cpu().numpy().tolist() == single


def test_two_streams_at_once():
    rng = np.random.default_rng(10)
    a = make_buffers(rng, 9, 3_000_000)
    b = make_buffers(rng, 11, 3_000_000)
    pa, va = placed(a, rng)
    pb, vb = placed(b, rng)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    oa = torch.zeros(len(va), dtype=torch.uint8, device="cuda")
    ob = torch.zeros(len(vb), dtype=torch.uint8, device="cuda")
    for _ in range(5):
        with torch.cuda.stream(sa):
            u.utf8_validate_buffers_async(va, oa, stream=sa)
        with torch.cuda.stream(sb):
            u.utf8_validate_buffers_async(vb, ob, stream=sb)
        torch.cuda.synchronize()
        assert oa.cpu().numpy().tolist() == [int(oracle.valid(x)) for x in a]
        assert ob.cpu().numpy().tolist() == [int(oracle.valid(x)) for x in b]


def test_writes_only_its_flags_and_rejects_bad_arguments():
    rng = np.random.default_rng(11)
    bufs = make_buffers(rng, 10, 100_000)
    pool, views = placed(bufs, rng)
    canvas = torch.full((64,), 0xA5, dtype=torch.uint8, device="cuda")
    u.utf8_validate_buffers_async(views, canvas[16:26])
    c = canvas.cpu().numpy()
    assert (c[:16] == 0xA5).all() and (c[26:] == 0xA5).all()
    assert c[16:26].tolist() == [int(oracle.valid(b)) for b in bufs]
    L = u.lib()
    ptrs = (ctypes.c_void_p * 2)(views[0].data_ptr(), bufs[1].ctypes.data)  # a host pointer
    lens = (ctypes.c_size_t * 2)(views[0].numel(), max(bufs[1].size, 1))
    out = torch.zeros(2, dtype=torch.uint8, device="cuda")
    assert L.utf8_validate_buffers_async(ptrs, lens, 2, ctypes.c_void_p(out.data_ptr()), None) == 1
    assert L.utf8_validate_buffers_async(ptrs, lens, -1, ctypes.c_void_p(out.data_ptr()), None) == 1
    assert L.utf8_validate_buffers_async(None, None, 0, None, None) == 0


def test_workload_1gib_buffers():
    bufs, names = [], []
    for i, name in enumerate(synth.VARIANTS_1GIB):
        seed = synth.SEED_BASE + 1000 + i
        clean = synth.fill_variant(1 << 30, name, seed)
        bad = clean.copy()
        bad[-3:] = np.frombuffer(synth.tail_error_bytes(seed), np.uint8)
        bufs += [clean, bad]
    views = [dev(b) for b in bufs]
    got = u.utf8_validate_buffers_async(views).cpu().numpy().tolist()
    assert got == [int(oracle.valid(b)) for b in bufs] == [1, 0] * 5
