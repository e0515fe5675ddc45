"""GB300 (sm_103a) row-wise Gustavson SpGEMM: C = A*B on CSR matrices.

The computation lives in the CUDA library ``libspgemm_gb300.so`` (sources in
``csrc/``, C ABI in ``include/spgemm.h``).  ``_native`` binds the ABI with
ctypes under the same names; ``api`` adds torch device containers and plans.
Submodules load on first use, so ``gen`` (the input generators) can be
imported without torch or the CUDA library.
"""
import importlib

__all__ = ["api", "gen", "build", "DeviceCSR", "Plan", "spgemm"]


def __getattr__(name):
    if name in ("api", "gen", "build", "_native"):
        return importlib.import_module("." + name, __name__)
    if name in ("DeviceCSR", "Plan", "spgemm"):
        return getattr(importlib.import_module(".api", __name__), name)
    raise AttributeError(name)
