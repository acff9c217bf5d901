"""The C-ABI library builds, loads and exports every symbol that
include/utf8gpu.h declares (CPU only: no compute calls)."""
import os
import re
import subprocess

import paper_2010_03090_gb300 as u
from conftest import ROOT


def declared_functions():
    text = open(os.path.join(ROOT, "include", "utf8gpu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(utf8_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("utf8_validate", "utf8_validate_batch", "utf8_last_error",
                     "utf8_error_string", "utf8_autotune", "utf8_tune_cache_load",
                     "utf8_tune_cache_save"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = u.lib_path()
    u.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(u.lib(), n)


def test_binding_names_match_header():
    for n in declared_functions():
        assert callable(getattr(u, n)), n


def test_error_strings():
    assert u.utf8_error_string(0) == "ok"
    assert u.utf8_error_string(1) == "invalid argument"
    assert u.utf8_error_string(2) == "CUDA error"
    assert u.utf8_error_string(999) == "unknown status"


def test_early_exit_setting_starts_from_the_environment():
    """utf8_set_early_exit touches no device: its default comes from
    UTF8GPU_EARLY_EXIT and it returns the previous setting."""
    import sys
    code = ("import paper_2010_03090_gb300 as u; "
            "print(int(u.utf8_set_early_exit(True)), int(u.utf8_set_early_exit(False)), "
            "int(u.utf8_set_early_exit(False)))")
    for env, first in ((None, "0"), ("1", "1"), ("0", "0"), ("7", "1")):
        e = dict(os.environ)
        e.pop("UTF8GPU_EARLY_EXIT", None)
        if env is not None:
            e["UTF8GPU_EARLY_EXIT"] = env
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                             env=e, cwd=ROOT, check=True).stdout.split()
        assert out == [first, "1", "0"], (env, out)


def test_library_links_no_shared_runtime():
    out = subprocess.run(["readelf", "-d", u.lib_path()], capture_output=True, text=True).stdout
    assert "libcudart" not in out  # static CUDA runtime: only the driver is needed
    assert "libtorch" not in out


def _build_c_example(out_dir):
    """Compiles tests/host/c_abi_example.c as C99 against the header and links
    it with the library (no GPU needed to build)."""
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(str(out_dir), "c_abi_example")
    lib_dir = os.path.dirname(u.lib_path())
    u.lib()
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    os.path.join(ROOT, "tests", "host", "c_abi_example.c"), "-o", exe,
                    "-L", lib_dir, "-lutf8gpu", f"-Wl,-rpath,{lib_dir}",
                    "-L", os.path.join(cuda, "lib64"), "-lcudart", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"],
                   check=True)
    return exe


def test_c_program_compiles_against_the_header(tmp_path):
    assert os.path.exists(_build_c_example(tmp_path))
