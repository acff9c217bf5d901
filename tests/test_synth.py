"""The seeded generators: determinism, exact sizes, valid content, and
injected errors of each class (checked with the oracle)."""
import numpy as np
import pytest

import oracle
import synth


def test_fill_is_deterministic_and_exact():
    a = synth.fill(100_003, synth.UNIFORM, seed=5, threads=1)
    b = synth.fill(100_003, synth.UNIFORM, seed=5, threads=4)
    assert a.size == 100_003 and np.array_equal(a, b)
    assert not np.array_equal(a, synth.fill(100_003, synth.UNIFORM, seed=6))


@pytest.mark.parametrize("name", list(synth.MODEL_NAMES))
def test_models_are_valid(name):
    buf = synth.fill(1 << 20, synth.MODEL_NAMES[name], seed=11)
    assert oracle.valid(buf)


def test_model_mixes():
    ascii_frac = {n: float(np.mean(synth.fill(1 << 20, m, seed=3) < 0x80))
                  for n, m in synth.MODEL_NAMES.items()}
    assert ascii_frac["ascii"] == 1.0
    assert 0.6 < ascii_frac["latin"] < 0.85       # 85% of characters are 1 byte
    assert ascii_frac["cjk"] < 0.15
    assert ascii_frac["uniform"] < 0.2


@pytest.mark.parametrize("kind", synth.ERROR_CLASSES)
def test_injection_makes_invalid(kind):
    rng = np.random.default_rng(1)
    for model in (synth.UNIFORM, synth.CJK, synth.LATIN):
        buf = synth.fill(4096, model, seed=int(rng.integers(1 << 30)))
        pos = synth.inject(buf, kind, rng)
        assert pos is not None
        assert not oracle.valid(buf), (kind, model)


def test_workload_1mib_flags():
    bufs, labels = synth.workload_1mib()
    assert [b.size for b in bufs] == [1 << 20] * 8
    assert [oracle.valid(b) for b in bufs] == [True] + [False] * 7
    assert labels[1:] == list(synth.ERROR_CLASSES)


def test_lognormal_and_pareto_calibration():
    lens, sigma = synth.lognormal_lengths(100_000, 200.0, 100_000 * 537, 1, 65536, 7)
    assert abs(np.median(lens) - 200) < 10
    assert abs(lens.sum() / (100_000 * 537) - 1) < 0.01
    assert 1.2 < sigma < 1.6
    lens, _ = synth.pareto_lengths(2000, 1.1, 1 << 28, 8, 1 << 24, 9)
    assert lens.min() >= 8 and lens.max() <= 1 << 24
    assert abs(lens.sum() / (1 << 28) - 1) < 0.02


def test_batch_corruption_matches_oracle():
    lens, _ = synth.lognormal_lengths(20_000, 200.0, 20_000 * 537, 1, 65536, 3)
    offsets = synth.offsets_of(lens)
    data = synth.fill_strings(offsets, synth.UNIFORM, seed=4)
    assert oracle.valid_batch(data, offsets).all()
    bad = synth.corrupt_strings(data, offsets, 0.01, seed=5)
    flags = oracle.valid_batch(data, offsets)
    assert set(np.nonzero(flags == 0)[0]) == set(bad.tolist())


def test_tail_error_bytes():
    for seed in range(10):
        t = synth.tail_error_bytes(seed)
        buf = synth.fill_variant(1000, "cjk", seed)
        assert oracle.valid(buf)
        buf[-3:] = np.frombuffer(t, np.uint8)
        assert not oracle.valid(buf)
