"""GB300-native spin-based MR simulator: per-isochromat Bloch propagation with
the per-ADC-sample signal reduction, behind the C-ABI library ``libmrsim``.

``workloads`` builds seeded synthetic inputs; ``mrsim`` is the thin ctypes
binding of the C-ABI (loaded on first use, never a CPU fallback).
"""
import importlib

__all__ = ["workloads", "mrsim", "autograd", "distributed"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
