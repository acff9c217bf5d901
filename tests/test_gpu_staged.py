"""The two load paths of the 8-row single-buffer, multi-buffer,
error-location and stream-chunk passes.

By default (where the device accepts the shared memory) the warps stage their
coming tiles through shared memory with cp.async, two tiles ahead; with
UTF8GPU_STAGED=0 they keep the next tile in registers.  Both must give the
oracle's answers.  The staged ring is exercised where it is most fragile:
warps whose runs hold 1 to 5 tiles (shorter than, equal to and longer than
the ring), errors in every tile of a run, checked first and last tiles of
unaligned buffers, and tile ranges of the host path.  Needs a GPU."""
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

import paper_2010_03090_gb300 as u  # noqa: E402

TILE = 8 * 512  # bytes of an 8-row tile
CLASS_BYTES = np.frombuffer(bytes([0x80, 0xBF, 0xC0, 0xC2, 0xE0, 0xED, 0xF0, 0xF4, 0xF5, 0xFF]),
                            np.uint8)


def config():
    return json.loads(u.utf8_config_json())


def grid_warps():
    c = config()
    return c["sm_count"] * c["blocks_per_sm"] * 8


def streamed(view, cuts):
    """The stream's flag, the buffer given in chunks cut at `cuts`."""
    h = u.utf8_stream_create()
    try:
        edges = [0] + sorted(cuts) + [view.numel()]
        for a, b in zip(edges[:-1], edges[1:]):
            u.utf8_stream_update(h, view[a:b])
        out = torch.zeros(1, dtype=torch.uint8, device="cuda")
        u.utf8_stream_finish(h, out)
        return int(out.item())
    finally:
        u.utf8_stream_destroy(h)


def check(buf, off=0):
    pool = torch.zeros(buf.size + 32, dtype=torch.uint8, device="cuda")
    if buf.size:
        pool[off:off + buf.size] = torch.from_numpy(buf).cuda()
    view = pool[off:off + buf.size]
    want = bool(oracle.valid(buf))
    assert bool(u.utf8_validate(view)) == want
    assert u.utf8_validate_buffers_async([view]).cpu().tolist() == [int(want)]
    assert u.utf8_locate_error(view) == tuple(oracle.locate(buf))
    # chunks of several tiles each (4 KiB tiles), cut inside characters too
    assert streamed(view, [buf.size // 3 + 1, 2 * buf.size // 3 + 2]) == int(want)
    return want


def test_default_is_staged():
    c = config()
    assert c["rows"] == 8 and c["staged"] == 1, c


@pytest.mark.parametrize("tiles_per_warp", [1, 2, 3, 4, 5])
def test_runs_shorter_and_longer_than_the_ring(tiles_per_warp):
    """Every warp's run holds tiles_per_warp tiles; one error per case, put
    into tile j of some warp's run for every j, and the clean buffer."""
    n = grid_warps() * tiles_per_warp * TILE - 7  # a partial last tile
    base = synth.fill(n, synth.CJK, seed=synth.SEED_BASE + 7300 + tiles_per_warp)
    assert check(base, 3)
    rng = np.random.default_rng(tiles_per_warp)
    for j in range(tiles_per_warp):
        w = int(rng.integers(0, grid_warps()))
        p = (w * tiles_per_warp + j) * TILE + int(rng.integers(0, TILE))
        p = min(p, n - 1)
        b = base.copy()
        b[p] = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size)]
        check(b, int(rng.integers(0, 16)))


def test_host_path_tile_ranges():
    """utf8_validate_host checks its buffer in ranges of tiles as the copies
    arrive; the staged runs then start and end inside the buffer."""
    n = 96 << 20
    base = synth.fill(n, synth.EMOJI, seed=synth.SEED_BASE + 7400)
    assert u.utf8_validate_host(base)
    rng = np.random.default_rng(7)
    for p in (0, TILE - 1, TILE, (1 << 20) - 2, (48 << 20) + 5, n - 1):
        b = base.copy()
        b[p] = CLASS_BYTES[rng.integers(0, CLASS_BYTES.size)]
        assert u.utf8_validate_host(b) == bool(oracle.valid(b)), p


def test_register_path_in_a_child():
    """UTF8GPU_STAGED=0 (read when a device is first used, so in a child):
    the register form answers as the oracle does on the same cases, with
    early exit off and on."""
    code = (
        "import json, numpy as np, torch, paper_2010_03090_gb300 as u, synth\n"
        "print(json.loads(u.utf8_config_json())['staged'])\n"
        "rng = np.random.default_rng(3)\n"
        "cls = np.frombuffer(bytes([0x80, 0xC0, 0xE0, 0xED, 0xF0, 0xF5]), np.uint8)\n"
        "out = []\n"
        "for i in range(24):\n"
        "    n = int(rng.integers(0, 12 << 20))\n"
        "    b = synth.fill(n, [synth.CJK, synth.UNIFORM, synth.ASCII][i % 3], seed=50 + i)\n"
        "    if n and i % 2:\n"
        "        b[int(rng.integers(0, n))] = cls[i % cls.size]\n"
        "    np.save('_staged_case_%d.npy' % i, b)\n"
        "    t = torch.from_numpy(b).cuda()\n"
        "    h = u.utf8_stream_create()\n"
        "    for a, b in ((0, n // 3 + 1), (n // 3 + 1, 2 * n // 3 + 2), (2 * n // 3 + 2, n)):\n"
        "        u.utf8_stream_update(h, t[min(a, n):min(b, n)])\n"
        "    f = torch.zeros(1, dtype=torch.uint8, device='cuda')\n"
        "    u.utf8_stream_finish(h, f)\n"
        "    u.utf8_stream_destroy(h)\n"
        "    u.utf8_set_early_exit(True)\n"
        "    ee = int(u.utf8_validate(t))\n"
        "    u.utf8_set_early_exit(False)\n"
        "    out.append([int(u.utf8_validate(t)), u.utf8_validate_buffers_async([t]).item(),\n"
        "                list(u.utf8_locate_error(t)), int(f.item()), ee])\n"
        "print(json.dumps(out))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, UTF8GPU_STAGED="0")
    work = os.path.join(root, "tests", "_staged_tmp")
    os.makedirs(work, exist_ok=True)
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=work,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        lines = r.stdout.strip().split("\n")
        assert lines[0] == "0", lines[0]
        got = json.loads(lines[1])
        for i, (a, b, loc, st, ee) in enumerate(got):
            buf = np.load(os.path.join(work, "_staged_case_%d.npy" % i))
            want = int(oracle.valid(buf))
            assert a == b == st == ee == want, (i, a, b, st, ee, want)
            assert tuple(loc) == tuple(oracle.locate(buf)), (i, loc)
    finally:
        for i in range(24):
            f = os.path.join(work, "_staged_case_%d.npy" % i)
            if os.path.exists(f):
                os.remove(f)
        if os.path.isdir(work):
            os.rmdir(work)
