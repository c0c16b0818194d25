"""GB300-native variational loop shrinking (handle/tunnel loops and diffusion Reeb graph).

The compute path is the CUDA library ``libvls.so`` (C ABI in ``include/vls.h``); this
package only marshals arguments to it (``vls.py``).  Build it with ``build.build()``.
"""
from .vls import (STATUS, VLS_FP32_RECHECK, VLS_FP64, detect, load, read_result, vls_constants, vls_create,
                  vls_result_kernel_times,
                  vls_default_options, vls_destroy, vls_detect, vls_detect_batch, vls_result_free)

__all__ = ["STATUS", "vls_result_kernel_times", "VLS_FP32_RECHECK", "VLS_FP64", "detect", "load", "read_result", "vls_constants", "vls_create",
           "vls_default_options", "vls_destroy", "vls_detect", "vls_detect_batch", "vls_result_free"]
