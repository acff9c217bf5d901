"""ctypes binding of libutf8gpu.so (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

EXPORTS = (
    "utf8_validate", "utf8_validate_async", "utf8_validate_batch", "utf8_validate_host",
    "utf8_classify_debug", "utf8_last_error", "utf8_error_string", "utf8_autotune",
    "utf8_tune_cache_load", "utf8_tune_cache_save", "utf8_config_json",
    "utf8_validate_host_noalloc", "utf8_server_default_config", "utf8_server_create",
    "utf8_server_submit", "utf8_server_result", "utf8_server_replay", "utf8_server_stats_get",
    "utf8_server_destroy", "utf8_validate_chunk", "utf8_stream_create", "utf8_stream_reset",
    "utf8_stream_update", "utf8_stream_finish", "utf8_stream_destroy", "utf8_copy_validate",
    "utf8_locate_error", "utf8_locate_error_async", "utf8_locate_errors_batch",
    "utf8_check_offsets", "utf8_validate_batch_desc", "utf8_set_early_exit",
    "utf8_validate_fsm_async", "utf8_validate_buffers_async",
)

# Section 3's rules a-f as the library numbers them (enum utf8_rule).
RULES = {0: "valid", 1: "a: 5+ byte", 2: "b: too short", 3: "c: too long", 4: "d: overlong",
         5: "e: too large", 6: "f: surrogate"}


class ErrorInfo(ctypes.Structure):
    """utf8_error_info: longest valid prefix and the rule the next character breaks."""
    _fields_ = [("position", ctypes.c_uint64), ("rule", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Utf8Error(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().utf8_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} (status {code})" if what else f"{msg} (status {code})")


def lib_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Loads the library (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, sz, i64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64, ctypes.c_int
            L.utf8_validate.argtypes = [vp, sz, vp]
            L.utf8_validate.restype = ctypes.c_bool
            L.utf8_validate_async.argtypes = [vp, sz, vp, vp]
            L.utf8_validate_async.restype = i32
            L.utf8_validate_fsm_async.argtypes = [vp, sz, vp, vp]
            L.utf8_validate_fsm_async.restype = i32
            L.utf8_validate_buffers_async.argtypes = [vp, vp, i32, vp, vp]
            L.utf8_validate_buffers_async.restype = i32
            L.utf8_validate_batch.argtypes = [vp, vp, i64, vp, vp]
            L.utf8_validate_batch.restype = i32
            L.utf8_validate_host.argtypes = [vp, sz, vp]
            L.utf8_validate_host.restype = ctypes.c_bool
            L.utf8_classify_debug.argtypes = [vp, sz, vp, vp, vp]
            L.utf8_classify_debug.restype = i32
            L.utf8_last_error.argtypes = []
            L.utf8_last_error.restype = i32
            L.utf8_error_string.argtypes = [i32]
            L.utf8_error_string.restype = ctypes.c_char_p
            L.utf8_autotune.argtypes = [i32]
            L.utf8_autotune.restype = i32
            L.utf8_tune_cache_load.argtypes = [ctypes.c_char_p]
            L.utf8_tune_cache_load.restype = i32
            L.utf8_tune_cache_save.argtypes = [ctypes.c_char_p]
            L.utf8_tune_cache_save.restype = i32
            L.utf8_config_json.argtypes = [ctypes.c_char_p, sz]
            L.utf8_config_json.restype = i32
            L.utf8_set_early_exit.argtypes = [i32]
            L.utf8_set_early_exit.restype = i32
            L.utf8_validate_host_noalloc.argtypes = [vp, sz, vp]
            L.utf8_validate_host_noalloc.restype = ctypes.c_bool
            L.utf8_copy_validate.argtypes = [vp, vp, sz, vp, vp]
            L.utf8_copy_validate.restype = i32
            L.utf8_validate_chunk.argtypes = [vp, sz, ctypes.c_uint32, i32, i32, vp, vp]
            L.utf8_validate_chunk.restype = i32
            L.utf8_stream_create.argtypes = []
            L.utf8_stream_create.restype = vp
            L.utf8_stream_reset.argtypes = [vp, vp]
            L.utf8_stream_reset.restype = i32
            L.utf8_stream_update.argtypes = [vp, vp, sz, vp]
            L.utf8_stream_update.restype = i32
            L.utf8_stream_finish.argtypes = [vp, vp, vp]
            L.utf8_stream_finish.restype = i32
            L.utf8_stream_destroy.argtypes = [vp]
            L.utf8_stream_destroy.restype = None
            L.utf8_locate_error.argtypes = [vp, sz, ctypes.POINTER(ErrorInfo), vp]
            L.utf8_locate_error.restype = i32
            L.utf8_locate_error_async.argtypes = [vp, sz, vp, vp]
            L.utf8_locate_error_async.restype = i32
            L.utf8_locate_errors_batch.argtypes = [vp, vp, i64, vp, vp]
            L.utf8_locate_errors_batch.restype = i32
            L.utf8_check_offsets.argtypes = [vp, i64, vp]
            L.utf8_check_offsets.restype = i32
            L.utf8_validate_batch_desc.argtypes = [vp, vp]
            L.utf8_validate_batch_desc.restype = i32
            _lib = L
    return _lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def _stream(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None  # the library reports UTF8_ERR_CUDA itself
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _dev(t, dtype_name: str, what: str):
    """(pointer, element count) of a contiguous CUDA tensor, or raw (ptr, n)."""
    if isinstance(t, tuple):
        return int(t[0]), int(t[1])
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch tensor")
    if not t.is_cuda:
        raise Utf8Error(1, f"{what} must be CUDA device memory")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"{what}: expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    return t.data_ptr(), t.numel()


def _check(status: int, what: str):
    if status != 0:
        raise Utf8Error(status, what)


# --------------------------------------------------------------------------
# the C-ABI, same names
# --------------------------------------------------------------------------
def utf8_validate(data, stream=None) -> bool:
    """True iff the uint8 CUDA tensor holds valid UTF-8 (synchronises the stream)."""
    p, n = _dev(data, "uint8", "data")
    ok = lib().utf8_validate(p or None, n, _stream(stream))
    _check(lib().utf8_last_error(), "utf8_validate")
    return bool(ok)


def utf8_validate_async(data, out_valid=None, stream=None):
    """Queues validation; returns a 1-element uint8 CUDA tensor (1 = valid)."""
    import torch
    p, n = _dev(data, "uint8", "data")
    if out_valid is None:
        out_valid = torch.empty(1, dtype=torch.uint8, device=data.device)
    q, _ = _dev(out_valid, "uint8", "out_valid")
    _check(lib().utf8_validate_async(p or None, n, q, _stream(stream)), "utf8_validate_async")
    return out_valid


def utf8_validate_buffers_async(buffers, out_valid=None, stream=None):
    """Queues the validation of a list of uint8 CUDA tensors in one launch;
    returns a uint8 CUDA tensor with one flag per buffer (1 = valid)."""
    import torch
    n = len(buffers)
    ptrs = (ctypes.c_void_p * max(n, 1))()
    lens = (ctypes.c_size_t * max(n, 1))()
    for i, t in enumerate(buffers):
        p, m = _dev(t, "uint8", "buffers[%d]" % i)
        ptrs[i], lens[i] = p or None, m
    if out_valid is None:
        dev = buffers[0].device if n else "cuda"
        out_valid = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    q, k = _dev(out_valid, "uint8", "out_valid")
    if k < n:
        raise ValueError("out_valid is too small")
    _check(lib().utf8_validate_buffers_async(ptrs, lens, n, q, _stream(stream)),
           "utf8_validate_buffers_async")
    return out_valid[:n]


def utf8_validate_fsm_async(data, out_valid=None, stream=None):
    """The paper's finite-state validator (Section 5) on the GPU, for
    comparison: queues it; returns a 1-element uint8 CUDA tensor (1 = valid)."""
    import torch
    p, n = _dev(data, "uint8", "data")
    if out_valid is None:
        out_valid = torch.empty(1, dtype=torch.uint8, device=data.device)
    q, _ = _dev(out_valid, "uint8", "out_valid")
    _check(lib().utf8_validate_fsm_async(p or None, n, q, _stream(stream)),
           "utf8_validate_fsm_async")
    return out_valid


def utf8_validate_batch(data, offsets, out_valid=None, stream=None):
    """One uint8 flag per string data[offsets[i]:offsets[i+1]] (asynchronous)."""
    import torch
    if isinstance(data, torch.Tensor) and data.numel() == 0:
        data = torch.zeros(16, dtype=torch.uint8, device=offsets.device)  # any device byte
    p, _ = _dev(data, "uint8", "data")
    q, m = _dev(offsets, "int64", "offsets")
    count = m - 1
    if count < 0:
        raise ValueError("offsets needs at least one entry")
    if out_valid is None:
        out_valid = torch.empty(max(count, 0), dtype=torch.uint8, device=offsets.device)
    r, k = _dev(out_valid, "uint8", "out_valid")
    if k < count:
        raise ValueError("out_valid is too small")
    _check(lib().utf8_validate_batch(p or None, q, count, r, _stream(stream)),
           "utf8_validate_batch")
    return out_valid


def utf8_locate_error(data, stream=None) -> tuple[int, int]:
    """(length of the longest valid prefix, rule 0-6) of a uint8 CUDA tensor;
    synchronises the stream."""
    p, n = _dev(data, "uint8", "data")
    info = ErrorInfo()
    _check(lib().utf8_locate_error(p or None, n, ctypes.byref(info), _stream(stream)),
           "utf8_locate_error")
    return int(info.position), int(info.rule)


def utf8_locate_error_async(data, out=None, stream=None):
    """Queues the error location of data into `out`, an int64 CUDA tensor of
    two elements holding one utf8_error_info (see error_info_fields)."""
    import torch
    p, n = _dev(data, "uint8", "data")
    if out is None:
        out = torch.empty(2, dtype=torch.int64, device=data.device)
    q, k = _dev(out, "int64", "out")
    if k < 2:
        raise ValueError("out needs two int64 elements")
    _check(lib().utf8_locate_error_async(p or None, n, q, _stream(stream)),
           "utf8_locate_error_async")
    return out


def utf8_locate_errors_batch(data, offsets, out=None, stream=None):
    """Per string data[offsets[i]:offsets[i+1]]: one utf8_error_info, as an
    int64 CUDA tensor of shape (count, 2) (asynchronous; see error_info_fields)."""
    import torch
    if isinstance(data, torch.Tensor) and data.numel() == 0:
        data = torch.zeros(16, dtype=torch.uint8, device=offsets.device)  # any device byte
    p, _ = _dev(data, "uint8", "data")
    q, m = _dev(offsets, "int64", "offsets")
    count = m - 1
    if count < 0:
        raise ValueError("offsets needs at least one entry")
    if out is None:
        out = torch.empty((max(count, 0), 2), dtype=torch.int64, device=offsets.device)
    r, k = _dev(out, "int64", "out")
    if k < 2 * count:
        raise ValueError("out is too small")
    _check(lib().utf8_locate_errors_batch(p or None, q, count, r, _stream(stream)),
           "utf8_locate_errors_batch")
    return out


def error_info_fields(out):
    """(positions int64, rules int32) views of utf8_error_info records held in
    an int64 tensor of shape (..., 2)."""
    import torch
    t = out.reshape(-1, 2)
    return t[:, 0], (t[:, 1] & 0xFFFFFFFF).to(torch.int32)  # rule: low half, little-endian


def batch_desc_values(data, offsets, out_valid) -> list:
    """The four int64 fields of a utf8_batch_desc (data, offsets, count,
    out_valid) for CUDA tensors; copy them into a device int64[4] tensor."""
    p, _ = _dev(data, "uint8", "data")
    q, m = _dev(offsets, "int64", "offsets")
    r, k = _dev(out_valid, "uint8", "out_valid")
    if k < m - 1:
        raise ValueError("out_valid is too small")
    return [p, q, m - 1, r]


def utf8_validate_batch_desc(desc, stream=None) -> None:
    """Queues the batch described by `desc`, a device int64[4] tensor holding a
    utf8_batch_desc (see batch_desc_values); the kernels read it when they run,
    so a captured graph of this call replays for whatever the tensor holds."""
    q, m = _dev(desc, "int64", "desc")
    if m < 4:
        raise ValueError("desc needs four int64 elements")
    _check(lib().utf8_validate_batch_desc(q, _stream(stream)), "utf8_validate_batch_desc")


def utf8_check_offsets(offsets, stream=None) -> None:
    """Raises Utf8Error (status 1) unless offsets[0] >= 0 and the int64 CUDA
    tensor is non-decreasing (checked on the device; synchronises)."""
    q, m = _dev(offsets, "int64", "offsets")
    if m < 1:
        raise ValueError("offsets needs at least one entry")
    _check(lib().utf8_check_offsets(q, m - 1, _stream(stream)), "utf8_check_offsets")


def utf8_validate_host(host, stream=None) -> bool:
    """True iff the host buffer (numpy uint8 array, bytes or a CPU tensor,
    pinned or not) is valid UTF-8; the library stages it through the GPU."""
    keep = host
    if isinstance(host, (bytes, bytearray)):
        keep = (ctypes.c_uint8 * len(host)).from_buffer_copy(host)
        p, n = ctypes.addressof(keep), len(host)
    elif hasattr(host, "ctypes"):  # numpy
        p, n = host.ctypes.data, host.nbytes
    else:  # torch CPU tensor
        if host.is_cuda:
            raise Utf8Error(1, "utf8_validate_host needs host memory")
        p, n = host.data_ptr(), host.numel() * host.element_size()
    ok = lib().utf8_validate_host(p or None, n, _stream(stream))
    del keep
    _check(lib().utf8_last_error(), "utf8_validate_host")
    return bool(ok)


def utf8_validate_host_noalloc(host, stream=None) -> bool:
    """utf8_validate_host for callers that cannot allocate GPU memory: stages
    through a fixed 32 MiB array inside the library (longer inputs raise with
    UTF8_ERR_BUDGET).  Calls that overlap on the GPU share that array."""
    if hasattr(host, "ctypes"):  # numpy
        p, n = host.ctypes.data, host.nbytes
    else:  # torch CPU tensor
        p, n = host.data_ptr(), host.numel() * host.element_size()
    ok = lib().utf8_validate_host_noalloc(p or None, n, _stream(stream))
    _check(lib().utf8_last_error(), "utf8_validate_host_noalloc")
    return bool(ok)


def utf8_copy_validate(dst, src, out_valid=None, stream=None):
    """Copies the uint8 CUDA tensor src into dst (same size) and validates it
    in one pass; returns the 1-element result tensor (1 = valid)."""
    import torch
    d, n = _dev(dst, "uint8", "dst")
    s, m = _dev(src, "uint8", "src")
    if n < m:
        raise ValueError("dst is smaller than src")
    if out_valid is None:
        out_valid = torch.empty(1, dtype=torch.uint8, device=src.device)
    q, _ = _dev(out_valid, "uint8", "out_valid")
    _check(lib().utf8_copy_validate(d or None, s or None, m, q, _stream(stream)),
           "utf8_copy_validate")
    return out_valid


def utf8_validate_chunk(data, prefix: bytes, final: bool, out_valid, stream=None) -> None:
    """Validates one chunk of a stream given the (up to 3) bytes before it;
    clears the device byte out_valid on an error (asynchronous)."""
    p, n = _dev(data, "uint8", "data")
    q, _ = _dev(out_valid, "uint8", "out_valid")
    pre = bytes(prefix)[-3:]
    packed = int.from_bytes(pre[::-1], "little")  # byte just before the chunk in bits 0..7
    _check(lib().utf8_validate_chunk(p or None, n, packed, len(pre), int(bool(final)), q,
                                     _stream(stream)), "utf8_validate_chunk")


def utf8_stream_create():
    h = lib().utf8_stream_create()
    if not h:
        raise Utf8Error(lib().utf8_last_error(), "utf8_stream_create")
    return h


def utf8_stream_reset(h, stream=None) -> None:
    _check(lib().utf8_stream_reset(h, _stream(stream)), "utf8_stream_reset")


def utf8_stream_update(h, chunk, stream=None) -> None:
    p, n = _dev(chunk, "uint8", "chunk")
    _check(lib().utf8_stream_update(h, p or None, n, _stream(stream)), "utf8_stream_update")


def utf8_stream_finish(h, out_valid, stream=None) -> None:
    q, _ = _dev(out_valid, "uint8", "out_valid")
    _check(lib().utf8_stream_finish(h, q, _stream(stream)), "utf8_stream_finish")


def utf8_stream_destroy(h) -> None:
    lib().utf8_stream_destroy(h)


def utf8_classify_debug(data, stream=None):
    """Per-position special-row bits and continuation bits (len + 3 each):
    see utf8_classify_debug in utf8gpu.h."""
    import torch
    p, n = _dev(data, "uint8", "data")
    sc = torch.empty(n + 3, dtype=torch.uint8, device=data.device)
    cont = torch.empty(n + 3, dtype=torch.uint8, device=data.device)
    _check(lib().utf8_classify_debug(p or None, n, sc.data_ptr(), cont.data_ptr(),
                                     _stream(stream)), "utf8_classify_debug")
    return sc, cont


def utf8_last_error() -> int:
    return lib().utf8_last_error()


def utf8_error_string(code: int) -> str:
    return lib().utf8_error_string(code).decode()


def utf8_autotune(flags: int = 0) -> None:
    _check(lib().utf8_autotune(flags), "utf8_autotune")


def utf8_tune_cache_load(path: str) -> None:
    _check(lib().utf8_tune_cache_load(os.fsencode(path)), "utf8_tune_cache_load")


def utf8_tune_cache_save(path: str) -> None:
    _check(lib().utf8_tune_cache_save(os.fsencode(path)), "utf8_tune_cache_save")


def utf8_set_early_exit(enable: bool) -> bool:
    """Switches early exit of single-buffer validation on or off (process-
    wide); returns the previous setting."""
    return bool(lib().utf8_set_early_exit(1 if enable else 0))


def utf8_config_json() -> str:
    buf = ctypes.create_string_buffer(512)
    n = lib().utf8_config_json(buf, 512)
    if n < 0:
        raise Utf8Error(lib().utf8_last_error(), "utf8_config_json")
    return buf.value.decode()
