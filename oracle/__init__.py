"""Scalar CPU oracle for the base64 codec (test infrastructure only).

The oracle is ``b64_oracle.c``: Algorithm 1 (encode) and Algorithm 2 (decode,
made strict as Section 2 and Appendix B ask) of Muła & Lemire, written one
character at a time with the paper's own division/modulo arithmetic and the
paper's Table 1. This module compiles it with the host C compiler and exposes
it through ctypes over numpy arrays.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product library never does, and it
shares no code with the CUDA sources.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "b64_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_b64.so")

OK = 0
INVALID_CHAR = 1
BAD_LENGTH = 2
NONCANONICAL = 3
FLAG_URL = 1
FLAG_NOPAD = 2
FLAG_STRICT_TAIL = 4
FLAG_SKIP_WS = 8

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "gcc")
    subprocess.check_call([cc, "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c_size = ctypes.c_size_t
        vp = ctypes.c_void_p
        lib.oracle_encoded_len.argtypes = [c_size]
        lib.oracle_encoded_len.restype = c_size
        lib.oracle_decoded_cap.argtypes = [c_size]
        lib.oracle_decoded_cap.restype = c_size
        lib.oracle_encode.argtypes = [vp, c_size, vp]
        lib.oracle_encode.restype = c_size
        lib.oracle_decode.argtypes = [vp, c_size, vp, ctypes.POINTER(c_size), ctypes.POINTER(c_size)]
        lib.oracle_decode.restype = ctypes.c_int
        lib.oracle_table1_value.argtypes = [ctypes.c_ubyte]
        lib.oracle_table1_value.restype = ctypes.c_int
        lib.oracle_table1_char.argtypes = [ctypes.c_uint]
        lib.oracle_table1_char.restype = ctypes.c_char
        lib.oracle_encode_batch.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        lib.oracle_encode_batch.restype = None
        lib.oracle_decode_batch.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        lib.oracle_decode_batch.restype = None
        lib.oracle_encoded_len_ex.argtypes = [c_size, ctypes.c_int]
        lib.oracle_encoded_len_ex.restype = c_size
        lib.oracle_decoded_cap_ex.argtypes = [c_size, ctypes.c_int]
        lib.oracle_decoded_cap_ex.restype = c_size
        lib.oracle_encode_ex.argtypes = [vp, c_size, vp, ctypes.c_int]
        lib.oracle_encode_ex.restype = c_size
        lib.oracle_decode_ex.argtypes = [vp, c_size, vp, ctypes.POINTER(c_size),
                                         ctypes.POINTER(c_size), ctypes.c_int]
        lib.oracle_decode_ex.restype = ctypes.c_int
        lib.oracle_decode_ws.argtypes = [vp, c_size, vp, ctypes.POINTER(c_size),
                                         ctypes.POINTER(c_size), ctypes.c_int]
        lib.oracle_decode_ws.restype = ctypes.c_int
        _lib = lib
        return lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8:
        a = a.view(np.uint8)
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def encoded_len(n: int) -> int:
    return int(_load().oracle_encoded_len(n))


def decoded_cap(m: int) -> int:
    return int(_load().oracle_decoded_cap(m))


def table1_value(x: int) -> int:
    """A of Algorithm 2: the 6-bit value of byte ``x``, or -1 if not in Table 1."""
    return int(_load().oracle_table1_value(x))


def table1_char(v: int) -> int:
    """B of Algorithm 1: the byte of the character for 6-bit value ``v``."""
    return _load().oracle_table1_char(v)[0]


def encode(data) -> np.ndarray:
    """Algorithm 1 over ``data``; returns the characters as a uint8 array."""
    src = _u8(data)
    out = np.empty(encoded_len(src.size), dtype=np.uint8)
    k = _load().oracle_encode(_ptr(src), src.size, _ptr(out))
    assert k == out.size
    return out


def decode(chars):
    """Strict Algorithm 2. Returns ``(status, output_bytes, first_bad)``."""
    src = _u8(chars)
    out = np.empty(max(decoded_cap(src.size), 1), dtype=np.uint8)
    outlen = ctypes.c_size_t(0)
    first_bad = ctypes.c_size_t(0)
    st = _load().oracle_decode(_ptr(src), src.size, out.ctypes.data,
                               ctypes.byref(outlen), ctypes.byref(first_bad))
    return int(st), out[: outlen.value].copy(), int(first_bad.value)


def encode_batch(src, in_off):
    """Encode packed messages; returns ``(dst, out_off)``."""
    src = _u8(src)
    in_off = np.ascontiguousarray(in_off, dtype=np.int64)
    nmsg = in_off.size - 1
    lens = np.diff(in_off)
    total = int(sum(encoded_len(int(n)) for n in lens)) if nmsg < 1000 else \
        int((4 * ((lens + 2) // 3)).sum())
    dst = np.empty(max(total, 1), dtype=np.uint8)
    out_off = np.empty(nmsg + 1, dtype=np.int64)
    _load().oracle_encode_batch(_ptr(src), in_off.ctypes.data, nmsg, dst.ctypes.data,
                                out_off.ctypes.data)
    assert out_off[-1] == total
    return dst[:total], out_off


def decode_batch(src, in_off):
    """Decode packed messages.

    Returns ``(dst, out_off, status, first_bad, outlen)`` with ``out_off`` the
    prefix of per-message capacities ``3*(m//4)``.
    """
    src = _u8(src)
    in_off = np.ascontiguousarray(in_off, dtype=np.int64)
    nmsg = in_off.size - 1
    cap = int((3 * (np.diff(in_off) // 4)).sum())
    dst = np.zeros(max(cap, 1), dtype=np.uint8)
    out_off = np.empty(nmsg + 1, dtype=np.int64)
    status = np.empty(nmsg, dtype=np.int32)
    first_bad = np.empty(nmsg, dtype=np.int64)
    outlen = np.empty(nmsg, dtype=np.int64)
    _load().oracle_decode_batch(_ptr(src), in_off.ctypes.data, nmsg, dst.ctypes.data,
                                out_off.ctypes.data, status.ctypes.data,
                                first_bad.ctypes.data, outlen.ctypes.data)
    return dst[:cap], out_off, status, first_bad, outlen


def encode_ex(data, flags: int) -> np.ndarray:
    """Algorithm 1 with the base64url / no-padding variants of Section 2."""
    src = _u8(data)
    out = np.empty(max(int(_load().oracle_encoded_len_ex(src.size, flags)), 1), dtype=np.uint8)
    k = _load().oracle_encode_ex(_ptr(src), src.size, out.ctypes.data, flags)
    return out[:k].copy()


def decode_ex(chars, flags: int):
    """Strict Algorithm 2 with the Section 2 variants and Appendix A's check.
    Returns ``(status, output_bytes, first_bad)``."""
    src = _u8(chars)
    out = np.empty(max(int(_load().oracle_decoded_cap_ex(src.size, flags)), 1), dtype=np.uint8)
    outlen = ctypes.c_size_t(0)
    first_bad = ctypes.c_size_t(0)
    fn = _load().oracle_decode_ws if flags & FLAG_SKIP_WS else _load().oracle_decode_ex
    st = fn(_ptr(src), src.size, out.ctypes.data, ctypes.byref(outlen), ctypes.byref(first_bad),
            flags)
    return int(st), out[: outlen.value].copy(), int(first_bad.value)
