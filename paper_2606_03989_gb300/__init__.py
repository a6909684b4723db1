"""PixVOD synchronous GBP sweeps on GB300 (sm_103a): Python binding.

The compute path is the CUDA library built from csrc/ (C ABI in
include/pixvod.h). This package only marshals arguments. Its attributes load
the library on first use and raise ImportError if it has not been built
(``python -m paper_2606_03989_gb300.build``); the build module itself imports
without the library.
"""
import importlib

_NATIVE = {"ADJOINT_HANDWRITTEN", "ADJOINT_TAPE", "ECUDA", "EINVAL", "ENOMEM", "ENUMERIC", "ESTATE", "ETIMEOUT", "FLAG_NONFINITE",
           "SCHED_PLAIN", "SCHED_BATCHED", "SCHED_PERSISTENT", "SCHED_NAMES",
           "TOPOLOGY_GRID", "TOPOLOGY_QUADTREE", "pixvod_intrinsics",
           "FLAG_NONPOS_PIVOT", "FLAG_TIMEOUT", "FLAG_BOUNDS", "LIB_PATH", "OK", "PixvodError", "StateView",
           "intrinsics", "lib", "params", "params_default", "parse_state", "status_string",
           "workspace_bytes"}

__all__ = sorted(_NATIVE | {"Tracker", "Batch", "track_frame"})


def __getattr__(name):
    if name in _NATIVE:
        return getattr(importlib.import_module("._native", __name__), name)
    if name in ("Tracker", "Batch", "track_frame"):
        return getattr(importlib.import_module(".tracker", __name__), name)
    raise AttributeError(name)
