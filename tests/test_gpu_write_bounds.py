"""Write bounds of every output: each call writes into a window of a larger
device buffer filled with a canary byte, and the bytes around the window
must come back untouched while the window holds the oracle's values.  Covers
the batch flags (plain and descriptor-driven), per-string error records, the
single-buffer result byte and error record, and the per-position debug
bytes.  Needs a GPU."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402

CANARY = 0xA5
PAD = 64


def canary(nbytes: int) -> "torch.Tensor":
    return torch.full((nbytes + 2 * PAD,), CANARY, dtype=torch.uint8, device="cuda")


def untouched(buf: "torch.Tensor", lo: int, hi: int) -> bool:
    b = buf.cpu().numpy()
    return bool((b[:lo] == CANARY).all() and (b[hi:] == CANARY).all())


def batches():
    rng = np.random.default_rng(23)
    out = []
    for count in (1, 2, 31, 32, 33, 1000, 40_000):
        lens = rng.integers(0, 300, count)
        lens[:: max(1, count // 7)] = 0  # empty strings among them
        offsets = synth.offsets_of(lens)
        data = synth.fill_strings(offsets, synth.UNIFORM, seed=count)
        synth.corrupt_strings(data, offsets, 0.1, seed=count + 1)
        out.append((data, offsets))
    return out


def test_batch_flags_stay_in_their_window():
    for data, offsets in batches():
        count = offsets.size - 1
        d = torch.from_numpy(data).cuda() if data.size else torch.zeros(16, dtype=torch.uint8,
                                                                        device="cuda")
        o = torch.from_numpy(offsets).cuda()
        want = oracle.valid_batch(data, offsets)
        buf = canary(count)
        u.utf8_validate_batch(d, o, buf[PAD:PAD + count])
        torch.cuda.synchronize()
        assert untouched(buf, PAD, PAD + count), count
        assert np.array_equal(buf[PAD:PAD + count].cpu().numpy(), want), count
        # the descriptor-driven form
        buf2 = canary(count)
        desc = torch.tensor(u.batch_desc_values(d, o, buf2[PAD:PAD + count]), dtype=torch.int64,
                            device="cuda")
        u.utf8_validate_batch_desc(desc)
        torch.cuda.synchronize()
        assert untouched(buf2, PAD, PAD + count), count
        assert np.array_equal(buf2[PAD:PAD + count].cpu().numpy(), want), count


def test_batch_error_records_stay_in_their_window():
    for data, offsets in batches():
        count = offsets.size - 1
        d = torch.from_numpy(data).cuda() if data.size else torch.zeros(16, dtype=torch.uint8,
                                                                        device="cuda")
        o = torch.from_numpy(offsets).cuda()
        rec = torch.full((count + 8, 2), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
        u.utf8_locate_errors_batch(d, o, rec[4:4 + count])
        torch.cuda.synchronize()
        r = rec.cpu().numpy()
        assert (r[:4] == -0x5A5A5A5A5A5A5A5B).all() and (r[4 + count:] == -0x5A5A5A5A5A5A5A5B).all()
        pos, rule = u.error_info_fields(rec[4:4 + count])
        want_pos, want_rule = oracle.locate_batch(data, offsets)
        assert np.array_equal(pos.cpu().numpy(), want_pos)
        assert np.array_equal(rule.cpu().numpy(), want_rule)


def test_single_buffer_outputs_stay_in_their_window():
    rng = np.random.default_rng(29)
    for n in (0, 1, 5, 4096, 3 << 20):
        text = synth.fill(n, synth.CJK, seed=n)
        if n and rng.random() < 0.7:
            synth.inject_any(text, synth.ERROR_CLASSES[int(rng.integers(0, 7))], rng)
        d = torch.from_numpy(text).cuda() if n else torch.zeros(16, dtype=torch.uint8,
                                                               device="cuda")[:0]
        buf = canary(1)
        u.utf8_validate_async(d, buf[PAD:PAD + 1])
        torch.cuda.synchronize()
        assert untouched(buf, PAD, PAD + 1), n
        assert int(buf[PAD].item()) == int(oracle.valid(text)), n
        rec = torch.full((6,), 77, dtype=torch.int64, device="cuda")
        u.utf8_locate_error_async(d, rec[2:4])
        torch.cuda.synchronize()
        r = rec.cpu().numpy()
        assert (r[:2] == 77).all() and (r[4:] == 77).all(), n
        assert (int(r[2]), int(r[3]) & 0xFFFFFFFF) == oracle.locate(text), n


def test_debug_bytes_stay_in_their_window():
    for n in (1, 3, 17, 5000):
        text = synth.fill(n, synth.UNIFORM, seed=n + 40)
        d = torch.from_numpy(text).cuda()
        sc, m = canary(n + 3), canary(n + 3)
        status = u.lib().utf8_classify_debug(d.data_ptr(), n, sc.data_ptr() + PAD,
                                             m.data_ptr() + PAD, None)
        torch.cuda.synchronize()
        assert status == 0
        want_sc, want_m = u.utf8_classify_debug(d)
        assert untouched(sc, PAD, PAD + n + 3) and untouched(m, PAD, PAD + n + 3), n
        assert torch.equal(sc[PAD:PAD + n + 3], want_sc) and torch.equal(m[PAD:PAD + n + 3], want_m)
