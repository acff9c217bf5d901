"""The paper's finite-state validator (Section 5) on the GPU
(utf8_validate_fsm_async), a comparison kernel for the `lookup` path, against
the CPU oracle, flag by flag.  Needs a GPU (-m gpu)."""
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
                                   0xF1, 0xF3, 0xF4, 0xF5, 0xFF]), dtype=np.uint8)
REGION = 512  # the kernel's region of one machine


def dev(a) -> "torch.Tensor":
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def fsm(t) -> bool:
    out = torch.empty(1, dtype=torch.uint8, device="cuda")
    u.utf8_validate_fsm_async(t, out)
    return bool(out.item())


def test_every_length_and_alignment():
    rng = np.random.default_rng(11)
    pool = dev(np.zeros(12288, np.uint8))
    for n in list(range(0, 130)) + list(range(130, 4200, 37)) + [8191, 8192, 8193]:
        text = synth.fill(n, synth.UNIFORM, seed=n) if rng.random() < 0.5 else \
            CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, n)]
        for shift in range(16):
            pool[shift:shift + n] = dev(text) if n else pool[:0]
            assert fsm(pool[shift:shift + n]) == oracle.valid(text), (n, shift)


def test_errors_at_region_starts():
    """Characters cut by a region boundary (the region before runs on over
    the continuations), errors on both sides of it, and runs of
    continuations at a region's start."""
    rng = np.random.default_rng(12)
    base = synth.fill(64 * REGION, synth.CJK, seed=3)
    for k in range(1, 60):
        for d in range(-5, 6):
            for shift in (0, 3):
                b = base.copy()
                at = k * REGION + d - shift
                if rng.random() < 0.5:
                    b[at] = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size)]
                else:
                    b[at:at + 4] = 0x80  # four continuations: never valid
                t = torch.zeros(b.size + 16, dtype=torch.uint8, device="cuda")
                t[shift:shift + b.size] = dev(b)
                assert fsm(t[shift:shift + b.size]) == oracle.valid(b), (k, d, shift)
    for shift in range(4):
        t = torch.zeros(base.size + 16, dtype=torch.uint8, device="cuda")
        t[shift:shift + base.size] = dev(base)
        assert fsm(t[shift:shift + base.size]) is True


def test_injected_errors_every_class():
    rng = np.random.default_rng(13)
    for model in (synth.UNIFORM, synth.LATIN, synth.EMOJI):
        for kind in synth.ERROR_CLASSES:
            for _ in range(5):
                b = synth.fill(int(rng.integers(1000, 300_000)), model, seed=int(rng.integers(1 << 30)))
                synth.inject_any(b, kind, rng)
                assert fsm(dev(b)) == oracle.valid(b) == False, kind  # noqa: E712


def test_random_bytes_and_class_strings():
    rng = np.random.default_rng(14)
    for n in (1 << 10, 1 << 16, 3 << 20):
        noise = rng.integers(0, 256, n).astype(np.uint8)
        assert fsm(dev(noise)) == oracle.valid(noise)
        cls = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size, n)]
        assert fsm(dev(cls)) == oracle.valid(cls)


@pytest.mark.parametrize("variant", synth.VARIANTS_1GIB)
def test_workload_1gib(variant):
    n = 1 << 30
    seed = synth.SEED_BASE + 1000 + synth.VARIANTS_1GIB.index(variant)
    buf = synth.fill_variant(n, variant, seed)
    t = dev(buf)
    assert fsm(t) == oracle.valid(buf) == True  # noqa: E712
    tail = np.frombuffer(synth.tail_error_bytes(seed), np.uint8)
    t[-3:] = dev(tail)
    buf[-3:] = tail
    assert fsm(t) == oracle.valid(buf) == False  # noqa: E712
