"""GB300-native single-conjugate adaptive-optics real-time controller.

The compute path is librtc.so (CUDA kernels for sm_103a behind the C ABI in
include/rtc.h); ``rtc`` is its ctypes binding.  Build the library with
``paper_1805_07254_gb300._build.build()``.
"""
from .rtc import Rtc, Mlp, Server, RtcError, load_library, version, LIB_PATH  # noqa: F401

__all__ = ["Rtc", "Mlp", "Server", "RtcError", "load_library", "version", "LIB_PATH"]
