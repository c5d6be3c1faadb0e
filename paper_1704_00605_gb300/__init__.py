"""GB300-native base64 codec (Muła & Lemire's method, re-designed for sm_103a).

The codec runs in hand-written CUDA kernels behind a C ABI (``include/gb64.h``);
``gb64`` is the thin Python binding over it. Using a codec entry point loads
the compiled library and raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import importlib

_SUBMODULES = ("build", "gb64", "workloads")


def load():
    """Return the binding module, loading ``libgb64.so`` (raises if absent)."""
    gb = importlib.import_module(".gb64", __name__)
    gb.lib()
    return gb


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module(f".{name}", __name__)
    gb = importlib.import_module(".gb64", __name__)
    if hasattr(gb, name):
        return getattr(gb, name)
    raise AttributeError(name)
