"""The C99 example program (tests/host/c_abi_example.c) runs against the
library on the GPU: validation, error location and a batch through the C-ABI
alone, without Python in the call path.  Needs a GPU."""
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from test_abi import _build_c_example  # noqa: E402


def test_c_program_runs(tmp_path):
    exe = _build_c_example(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
