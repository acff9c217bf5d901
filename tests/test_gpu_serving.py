"""The continuous-batching server (GPU): every request's result in the mix
equals its result alone (utf8_validate) and the oracle's; admission keeps
the admitted bytes within the budget; argument and budget errors."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402
from paper_2010_03090_gb300.serve import Server  # noqa: E402


@pytest.fixture(scope="module")
def pool():
    data, offsets, bad = synth.serving_pool(count=400, lo=64, hi=4 << 20,
                                            invalid_fraction=0.03, seed=99)
    dev = torch.from_numpy(data).cuda()
    return data, offsets, bad, dev


def _requests(offsets, n, seed):
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, offsets.size - 1, n)
    return pick


def test_results_alone_and_in_the_mix(pool):
    data, offsets, bad, dev = pool
    pick = _requests(offsets, 3000, 5)
    base = dev.data_ptr()
    ptrs = base + offsets[pick]
    lens = offsets[pick + 1] - offsets[pick]
    arrivals = synth.poisson_arrivals_ns(pick.size, 20_000.0, 6)
    with Server(window_min_us=50, window_max_us=500, streams=4) as srv:
        mixed, lat = srv.replay(ptrs, lens, arrivals)
        st = srv.stats()
    alone = np.array([u.utf8_validate(dev[offsets[j]:offsets[j + 1]]) for j in range(offsets.size - 1)],
                     dtype=np.uint8)
    want = oracle.valid_batch(data, offsets)
    assert np.array_equal(alone, want)
    assert np.array_equal(mixed, alone[pick])
    assert (mixed == 0).sum() > 0 and (mixed == 1).sum() > 0
    assert st["completed"] == pick.size and st["batches"] >= 1
    assert st["max_batch_seen"] > 1  # requests were batched together
    assert (lat > 0).all()


def test_budget_admission(pool):
    data, offsets, bad, dev = pool
    pick = _requests(offsets, 500, 7)
    lens = offsets[pick + 1] - offsets[pick]
    budget = int(lens.max()) + (1 << 20)
    with Server(budget_bytes=budget, streams=2) as srv:
        valid, _ = srv.replay(dev.data_ptr() + offsets[pick], lens, np.zeros(pick.size, np.int64))
        st = srv.stats()
    assert st["max_admitted_bytes"] <= budget
    assert np.array_equal(valid, oracle.valid_batch(data, offsets)[pick])


def test_submit_result_and_errors(pool):
    data, offsets, bad, dev = pool
    with Server(budget_bytes=1 << 20) as srv:
        j = int(np.argmax(np.diff(offsets) < (1 << 20)))
        t = srv.submit(dev[offsets[j]:offsets[j + 1]])
        ok, lat = srv.result(t, timeout_us=10_000_000)
        assert ok == oracle.valid(data[offsets[j]:offsets[j + 1]])
        with pytest.raises(u.Utf8Error):
            srv.submit(torch.zeros(2 << 20, dtype=torch.uint8, device="cuda"))  # over budget
        with pytest.raises(u.Utf8Error):
            srv.submit(torch.zeros(16, dtype=torch.uint8))  # host memory
        with pytest.raises(u.Utf8Error):
            srv.result(10 ** 9, timeout_us=0)  # unknown ticket
