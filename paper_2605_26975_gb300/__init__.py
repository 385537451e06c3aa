"""GB300-native multiway p-spectral clustering (hot path in CUDA for sm_103a).

The compute lives in the C-ABI library libpspec.so (include/pspec.h); the
Python side is a thin ctypes binding (``api``), a torch.autograd.Function
over it (``autograd``) and seeded synthetic workloads (``workloads``).
Submodules are imported lazily so that ``workloads`` needs neither torch nor
the built library.
"""
import importlib

__all__ = ["api", "autograd", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
