"""GB300-native base64 codec (Muła & Lemire's method, re-designed for sm_103a).

The codec runs in hand-written CUDA kernels behind a C ABI (``include/gb64.h``);
this package is the thin Python binding over it. Import of the codec entry
points loads the compiled library and raises if it is missing: there is no
CPU fallback.
"""
from __future__ import annotations

from . import workloads  # noqa: F401  (seeded inputs; no codec arithmetic)

_BINDING_NAMES = None


def load():
    """Return the binding module, loading ``libgb64.so`` (raises if absent)."""
    from . import gb64

    gb64.lib()
    return gb64


def __getattr__(name):
    if name == "build":
        from . import build as _b

        return _b
    from . import gb64

    if hasattr(gb64, name):
        return getattr(gb64, name)
    raise AttributeError(name)
