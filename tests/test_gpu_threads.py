"""Entry points called from many host threads at once (the header promises
thread safety): each thread uses its own stream and mixes the synchronous,
asynchronous, error-location, host-memory, batch and multi-buffer calls on valid and
invalid buffers, while another thread retunes the launch configuration.
Every result must equal the oracle's.  Needs a GPU."""
import json
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2010_03090_gb300 as u  # noqa: E402


def test_concurrent_calls_from_host_threads():
    rng = np.random.default_rng(41)
    bufs = []
    for k in range(12):
        b = synth.fill(int(rng.integers(1 << 10, 6 << 20)), k % 7, seed=900 + k)
        if k % 3 == 1:
            synth.inject_any(b, synth.ERROR_CLASSES[k % 7], rng)
        bufs.append(b)
    want = [oracle.valid(b) for b in bufs]
    where = [oracle.locate(b) for b in bufs]
    dev = [torch.from_numpy(b).cuda() for b in bufs]
    pinned = []
    for b in bufs:
        p = torch.empty(b.size, dtype=torch.uint8, pin_memory=True)
        p.numpy()[:] = b
        pinned.append(p)
    strings = [b[:4096] for b in bufs]
    offsets = synth.offsets_of([s.size for s in strings])
    data = np.concatenate(strings)
    d_data, d_off = torch.from_numpy(data).cuda(), torch.from_numpy(offsets).cuda()
    want_batch = oracle.valid_batch(data, offsets)
    u.utf8_validate(dev[0])  # the device's work areas exist before the threads start
    torch.cuda.synchronize()

    failures = []

    def worker(t):
        try:
            s = torch.cuda.Stream()
            out = torch.empty(1, dtype=torch.uint8, device="cuda")
            flags = torch.empty(len(strings), dtype=torch.uint8, device="cuda")
            three = torch.empty(3, dtype=torch.uint8, device="cuda")
            for it in range(40):
                k = (t * 7 + it) % len(bufs)
                mode = (t + it) % 6
                if mode == 0:
                    got = u.utf8_validate(dev[k], stream=s)
                    ok = got == want[k]
                elif mode == 1:
                    u.utf8_validate_async(dev[k], out, stream=s)
                    s.synchronize()
                    ok = bool(out.item()) == want[k]
                elif mode == 2:
                    ok = u.utf8_locate_error(dev[k], stream=s) == where[k]
                elif mode == 3:
                    ok = u.utf8_validate_host(pinned[k], stream=s) == want[k]
                elif mode == 4:
                    u.utf8_validate_batch(d_data, d_off, flags, stream=s)
                    s.synchronize()
                    ok = np.array_equal(flags.cpu().numpy(), want_batch)
                else:
                    ks = [(k + j) % len(bufs) for j in range(3)]
                    u.utf8_validate_buffers_async([dev[j] for j in ks], three, stream=s)
                    s.synchronize()
                    ok = three.cpu().numpy().tolist() == [int(want[j]) for j in ks]
                if not ok:
                    failures.append((t, it, k, mode))
        except Exception as e:  # noqa: BLE001
            failures.append((t, repr(e)))

    def tuner():
        try:
            u.utf8_autotune(1)
        except Exception as e:  # noqa: BLE001
            failures.append(("tune", repr(e)))

    cfg0 = json.loads(u.utf8_config_json())
    threads = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
    threads.append(threading.Thread(target=tuner))
    try:
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=600)
    finally:
        restore_config(cfg0)
    assert not any(th.is_alive() for th in threads)
    assert failures == []


def restore_config(cfg, tmp_dir=None):
    """Puts the launch configuration back (a cache entry, then a cached
    autotune), so that later tests run with the one they started with."""
    import os
    import tempfile
    name = torch.cuda.get_device_name(0)
    line = (f'{{"gpu": "{name}", "sms": {cfg["sm_count"]}, "rows": {cfg["rows"]}, '
            f'"blocks_per_sm": {cfg["blocks_per_sm"]}, "batch_rows": {cfg["batch_rows"]}, '
            f'"batch_blocks_per_sm": {cfg["batch_blocks_per_sm"]}}}\n')
    fd, path = tempfile.mkstemp(suffix=".json", dir=tmp_dir)
    with os.fdopen(fd, "w") as f:
        f.write(line)
    try:
        u.utf8_tune_cache_load(path)
        u.utf8_autotune(0)
    finally:
        os.remove(path)
    assert json.loads(u.utf8_config_json()) == cfg
