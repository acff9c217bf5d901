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
    utf8_error_string,
    utf8_last_error,
    utf8_tune_cache_load,
    utf8_tune_cache_save,
    utf8_validate,
    utf8_validate_async,
    utf8_validate_batch,
    utf8_validate_host,
    utf8_validate_host_noalloc,
)

UTF8_OK = 0
UTF8_ERR_INVALID_ARG = 1
UTF8_ERR_CUDA = 2
UTF8_ERR_TIMEOUT = 3
UTF8_ERR_BUDGET = 4
UTF8_ERR_NOMEM = 5
