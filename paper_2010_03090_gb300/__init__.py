"""utf8gpu: UTF-8 validation on one GB300 with the `lookup` algorithm
(Keiser & Lemire, arXiv 2010.03090), as hand-written sm_103a CUDA kernels.

This module is a thin binding over the C-ABI library ``libutf8gpu.so``
(declared in ``include/utf8gpu.h``): the functions have the C names and only
marshal arguments (tensor -> device pointer, torch stream -> cudaStream_t).
Every validation step runs in the library's kernels; if the library is
missing or CUDA is unusable the calls raise — there is no CPU fallback.
PyTorch is used for device memory and streams only.
"""
from ._lib import (  # noqa: F401
    Utf8Error,
    lib,
    lib_path,
    utf8_autotune,
    utf8_classify_debug,
    utf8_config_json,
    utf8_set_early_exit,
    utf8_error_string,
    utf8_last_error,
    utf8_tune_cache_load,
    utf8_tune_cache_save,
    utf8_validate,
    utf8_validate_async,
    utf8_validate_fsm_async,
    utf8_validate_buffers_async,
    utf8_validate_batch,
    utf8_validate_host,
    utf8_validate_host_noalloc,
    utf8_validate_chunk,
    utf8_copy_validate,
    utf8_stream_create,
    utf8_stream_reset,
    utf8_stream_update,
    utf8_stream_finish,
    utf8_stream_destroy,
    utf8_locate_error,
    utf8_locate_error_async,
    utf8_locate_errors_batch,
    utf8_check_offsets,
    utf8_validate_batch_desc,
    batch_desc_values,
    error_info_fields,
    ErrorInfo,
    RULES,
)

from .serve import Server  # noqa: E402,F401


def _server_fn(name):
    def call(*args):
        from .serve import _bind
        return getattr(_bind(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"Direct C-ABI call {name}; see include/utf8gpu.h and serve.Server."
    return call


utf8_server_default_config = _server_fn("utf8_server_default_config")
utf8_server_create = _server_fn("utf8_server_create")
utf8_server_submit = _server_fn("utf8_server_submit")
utf8_server_result = _server_fn("utf8_server_result")
utf8_server_replay = _server_fn("utf8_server_replay")
utf8_server_stats_get = _server_fn("utf8_server_stats_get")
utf8_server_destroy = _server_fn("utf8_server_destroy")

UTF8_OK = 0
UTF8_ERR_INVALID_ARG = 1
UTF8_ERR_CUDA = 2
UTF8_ERR_TIMEOUT = 3
UTF8_ERR_BUDGET = 4
UTF8_ERR_NOMEM = 5
