"""utf8_copy_validate (GPU): the destination receives exactly the source
bytes (nothing outside it is touched), and the flag equals the oracle's,
for aligned (fused single pass) and misaligned (copy then validate) pairs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

CLASS = np.frombuffer(bytes([0x41, 0x80, 0x90, 0xA0, 0xC3, 0xE0, 0xED, 0xF0, 0xF4, 0xFF]), np.uint8)


def test_copy_validate_bytes_and_flags():
    rng = np.random.default_rng(8)
    src_pool = torch.zeros((9 << 20) + 64, dtype=torch.uint8, device="cuda")
    dst_pool = torch.full(((9 << 20) + 128,), 0x5A, dtype=torch.uint8, device="cuda")
    sizes = [0, 1, 2, 3, 15, 16, 17, 100, 4095, 4096, 4097, 70_000, (8 << 20) + 3]
    for i, n in enumerate(sizes * 3):
        if i % 3 == 0:
            b = CLASS[rng.integers(0, CLASS.size, n)]
        else:
            b = synth.fill(n, synth.UNIFORM if i % 2 else synth.CJK, seed=i)
            if i % 3 == 1 and n:
                synth.inject_any(b, synth.ERROR_CLASSES[i % 7], rng)
        so = int(rng.integers(0, 16))
        do = so + 16 * int(rng.integers(0, 3)) if i % 2 == 0 else int(rng.integers(0, 32))
        src = src_pool[so:so + n]
        if n:
            src.copy_(torch.from_numpy(b.copy()))
        dst_pool.fill_(0x5A)
        dst = dst_pool[do + 16:do + 16 + n]
        flag = u.utf8_copy_validate(dst, src)
        torch.cuda.synchronize()
        assert flag.item() == oracle.valid(b), (n, so, do)
        assert torch.equal(dst, src)
        assert (dst_pool[:do + 16] == 0x5A).all() and (dst_pool[do + 16 + n:] == 0x5A).all()


def test_copy_validate_rejects_overlap():
    t = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(u.Utf8Error):
        u.utf8_copy_validate(t[100:600], t[0:500])
