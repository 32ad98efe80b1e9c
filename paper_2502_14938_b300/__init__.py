"""B300-native structured-3DGS frame renderer (GS-Cache hot path, arXiv 2502.14938).

The compute lives in libgsc.so (hand-written sm_103a CUDA behind a C ABI,
include/gsc.h); `native` is the ctypes binding with the same call names.
"""
from .native import (GscError, Renderer, default_config, exported_symbols, lib, to_camera,
                     FLAG_DEBUG_ATTRS, FLAG_DEBUG_T, FLAG_TIMING, FLAG_REUSE_COLLECT, FLAG_BLEND_WORK,
                     FLAG_UNFUSED, REUSE_NPARAM)

__all__ = ["GscError", "Renderer", "default_config", "exported_symbols", "lib", "to_camera",
           "FLAG_DEBUG_ATTRS", "FLAG_DEBUG_T", "FLAG_TIMING", "FLAG_REUSE_COLLECT", "FLAG_BLEND_WORK",
           "FLAG_UNFUSED", "REUSE_NPARAM"]
