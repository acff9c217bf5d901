"""Tile heights other than the default 8 rows, against the oracle.

A launch configuration (from the autotuner, a tuning cache or the
UTF8GPU_ROWS / UTF8GPU_BATCH_ROWS variables) may pick 4- or 2-row tiles.
At 4 rows the single-buffer, multi-buffer and error-location passes
classify one row quad with register loads, and the batch pass classifies one
quad per tile through its shared-memory ring; at 2 rows every pass
classifies one row pair.  The variables are read when a device is first
used, so each height runs in a child process; the parent checks the child's
answers against the oracle.  Needs a GPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

CHILD = r"""
import json, sys, numpy as np, torch, paper_2010_03090_gb300 as u, synth
cfg = json.loads(u.utf8_config_json())
print(json.dumps([cfg["rows"], cfg["batch_rows"]]))
rng = np.random.default_rng(11)
cls = np.frombuffer(bytes([0x80, 0xBF, 0xC0, 0xE0, 0xED, 0xF0, 0xF4, 0xF5, 0xFF]), np.uint8)
single = []
for i in range(16):
    n = int(rng.integers(0, 6 << 20))
    b = synth.fill(n, [synth.CJK, synth.UNIFORM, synth.ASCII, synth.EMOJI][i % 4], seed=90 + i)
    if n and i % 3:
        b[int(rng.integers(0, n))] = cls[i % cls.size]
    np.save("_rows_case_%d.npy" % i, b)
    pool = torch.zeros(n + 32, dtype=torch.uint8, device="cuda")
    off = int(rng.integers(0, 16))
    if n:
        pool[off:off + n] = torch.from_numpy(b).cuda()
    t = pool[off:off + n]
    single.append([int(u.utf8_validate(t)), u.utf8_validate_buffers_async([t]).item(),
                   list(u.utf8_locate_error(t))])
print(json.dumps(single))
lengths, _ = synth.lognormal_lengths(20000, 200.0, 8 << 20, 1, 65536, 5)
offsets = synth.offsets_of(lengths)
data = synth.fill_strings(offsets, synth.UNIFORM, 5)
synth.corrupt_strings(data, offsets, 0.02, 6)
np.save("_rows_batch_data.npy", data)
np.save("_rows_batch_offsets.npy", offsets)
d = torch.from_numpy(data).cuda()
o = torch.from_numpy(offsets).cuda()
flags = u.utf8_validate_batch(d, o).cpu().numpy().tolist()
pos, rule = u.error_info_fields(u.utf8_locate_errors_batch(d, o))
print(json.dumps([flags, pos.cpu().numpy().tolist(), rule.cpu().numpy().tolist()]))
"""


@pytest.mark.parametrize("rows", [4, 2])
def test_tile_height_in_a_child(rows, tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, UTF8GPU_ROWS=str(rows), UTF8GPU_BATCH_ROWS=str(rows))
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=str(tmp_path),
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().split("\n")
    assert json.loads(lines[0]) == [rows, rows]
    for i, (a, b, loc) in enumerate(json.loads(lines[1])):
        buf = np.load(str(tmp_path / ("_rows_case_%d.npy" % i)))
        want = int(oracle.valid(buf))
        assert a == b == want, (rows, i, a, b, want)
        assert tuple(loc) == tuple(oracle.locate(buf)), (rows, i, loc)
    flags, pos, rule = json.loads(lines[2])
    data = np.load(str(tmp_path / "_rows_batch_data.npy"))
    offsets = np.load(str(tmp_path / "_rows_batch_offsets.npy"))
    want = oracle.valid_batch(data, offsets, threads=4)
    assert np.array_equal(np.array(flags, np.uint8), want)
    assert 0 < int((want == 0).sum()) < want.size
    wpos, wrule = oracle.locate_batch(data, offsets, threads=4)
    assert np.array_equal(np.array(pos, np.int64), wpos)
    assert np.array_equal(np.array(rule, np.int32), wrule)
