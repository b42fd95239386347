"""GB300 ray marching of relativistic, optically thin emission through meshed
simulation snapshots (the method of the cuDART paper), as a C-ABI library
with hand-written sm_103a CUDA kernels and a thin Python binding."""
from .gbdart import (BEAMING, LOOKBACK, STORE_BF16_F16U, STORE_F32, Context, GbdError, error_string,
                     load_library)

__all__ = ["Context", "GbdError", "load_library", "error_string", "BEAMING", "LOOKBACK", "STORE_F32",
           "STORE_BF16_F16U"]
