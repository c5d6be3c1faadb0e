"""Thin ctypes binding of libgb64 (the C ABI in include/gb64.h).

Every function here only marshals arguments: it allocates output tensors
with torch when the caller did not pass them, turns tensors into raw device
pointers and the current torch stream into a ``cudaStream_t``, and calls the
C entry point of the same name. All coding runs in the library's CUDA
kernels; when ``libgb64.so`` is missing, loading raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

B64_OK = 0
B64_ERR_INVALID_CHAR = 1
B64_ERR_BAD_LENGTH = 2
B64_ERR_NONCANONICAL = 3
B64_FLAG_URL = 1
B64_FLAG_NOPAD = 2
B64_FLAG_STRICT_TAIL = 4
B64_ERR_ARG = -1
B64_ERR_CUDA = -2
B64_ERR_NOMEM = -3
B64_ERR_TIMEOUT = -4
SIZE_MAX = (1 << 64) - 1

_lib = None

B64_KIND_ENCODE = 0
B64_KIND_DECODE = 1
B64_KIND_ENCODE_BATCH = 2
B64_KIND_DECODE_BATCH = 3
B64_KIND_DECODE_WS = 4


class b64_server_config(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_int64), ("streams", ctypes.c_int32),
                ("max_batch_msgs", ctypes.c_int32), ("max_batch_bytes", ctypes.c_int64),
                ("auto_release", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class b64_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("kind", ctypes.c_int32), ("status", ctypes.c_int32),
                ("first_bad", ctypes.c_int64), ("outlen", ctypes.c_int64),
                ("out", ctypes.c_void_p), ("len", ctypes.c_int64), ("batch", ctypes.c_int64),
                ("t_arrival_us", ctypes.c_double), ("t_admit_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class b64_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "requests_submitted", "requests_launched", "requests_done", "rejected", "batches",
        "memory_waits", "arena_bytes", "arena_in_use", "arena_high_water", "bytes_in")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class b64_shape(ctypes.Structure):
    """Launch shape (mirrors ``b64_shape`` in include/gb64.h)."""

    _fields_ = [("threads", ctypes.c_int32), ("units_per_thread", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("tile", ctypes.c_int64), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Gb64Error(RuntimeError):
    """A call of the C ABI returned an error code."""

    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load ``libgb64.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1704_00605_gb300.build.build(); "
                           "the codec has no CPU fallback")
    L = ctypes.CDLL(path)
    sz, vp, i64, i32 = ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    psz = ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "b64_encoded_len": (sz, [sz]),
        "b64_decoded_cap": (sz, [sz]),
        "b64_encode": (sz, [vp, sz, vp, vp]),
        "b64_decode": (i32, [vp, sz, vp, psz, psz, vp]),
        "b64_decode_async": (i32, [vp, sz, vp, vp, vp]),
        "b64_encode_host": (sz, [vp, sz, vp, vp]),
        "b64_decode_host": (i32, [vp, sz, vp, psz, psz, vp]),
        "b64_batch_out_offsets": (i32, [i32, vp, i64, vp, vp]),
        "b64_encode_batch": (i32, [vp, vp, i64, vp, vp, vp]),
        "b64_decode_batch": (i32, [vp, vp, i64, vp, vp, vp, vp, vp, vp]),
        "b64_status_str": (ctypes.c_char_p, [i32]),
        "b64_last_error": (ctypes.c_char_p, []),
        "b64_device_fault": (i32, []),
        "b64_release_scratch": (i32, []),
        "b64_test_stall_copies": (i32, [i32, ctypes.c_uint64]),
        "b64_shape_get": (i32, [i32, i64, i64, ctypes.POINTER(b64_shape)]),
        "b64_shape_set": (i32, [i32, i64, i64, ctypes.POINTER(b64_shape)]),
        "b64_tune": (i32, [i32, i64, i64, ctypes.POINTER(b64_shape), i32,
                           ctypes.POINTER(ctypes.c_int), vp]),
        "b64_tune_save": (i32, [ctypes.c_char_p]),
        "b64_tune_load": (i32, [ctypes.c_char_p]),
        "b64_server_create": (vp, [ctypes.POINTER(b64_server_config)]),
        "b64_server_now_us": (ctypes.c_double, [vp]),
        "b64_server_submit": (i32, [vp, i32, vp, i64, ctypes.c_double, ctypes.POINTER(i64)]),
        "b64_server_poll": (i32, [vp, ctypes.POINTER(b64_completion), i32, i32]),
        "b64_server_release": (i32, [vp, i64]),
        "b64_server_stats_get": (i32, [vp, ctypes.POINTER(b64_server_stats)]),
        "b64_server_replay": (i32, [vp, i64, vp, vp, vp, vp, vp, vp]),
        "b64_server_destroy": (None, [vp]),
        "b64_decode_batch_noalloc": (i32, [vp, vp, i64, vp, vp, vp, vp, vp, vp]),
        "b64_encoded_len_ex": (sz, [sz, i32]),
        "b64_decoded_cap_ex": (sz, [sz, i32]),
        "b64_encode_ex": (sz, [vp, sz, vp, i32, vp]),
        "b64_decode_ex": (i32, [vp, sz, vp, psz, psz, i32, vp]),
        "b64_decode_async_ex": (i32, [vp, sz, vp, vp, i32, vp]),
        "b64_batch_out_offsets_ex": (i32, [i32, vp, i64, vp, i32, vp]),
        "b64_encode_batch_ex": (i32, [vp, vp, i64, vp, vp, i32, vp]),
        "b64_decode_batch_ex": (i32, [vp, vp, i64, vp, vp, vp, vp, vp, i32, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_name(status: int) -> str:
    try:
        return lib().b64_status_str(status).decode()
    except Exception:
        return str(status)


def b64_last_error() -> str:
    return lib().b64_last_error().decode()


def b64_status_str(status: int) -> str:
    return lib().b64_status_str(status).decode()


def b64_encoded_len(n: int) -> int:
    return int(lib().b64_encoded_len(n))


def b64_decoded_cap(m: int) -> int:
    return int(lib().b64_decoded_cap(m))


def b64_device_fault() -> int:
    return int(lib().b64_device_fault())


def b64_release_scratch() -> None:
    """Frees the scratch that the whitespace decode keeps on the current
    device (after its last user)."""
    st = int(lib().b64_release_scratch())
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())


def b64_test_stall_copies(stall: bool, wait_limit_ns: int = 0) -> None:
    """Test hook: while ``stall`` is set, pipelined kernels leave out the
    first copy of their first CTA (warp) so its bounded wait runs out."""
    lib().b64_test_stall_copies(1 if stall else 0, int(wait_limit_ns))


# ------------------------------------------------------------ marshalling
def _torch():
    import torch

    return torch


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


_NULL = _Null()


def _on(device):
    """Device guard that costs nothing when ``device`` is already current."""
    torch = _torch()
    if isinstance(device, int):
        idx = device
    else:
        idx = device.index if device.index is not None else torch.cuda.current_device()
    return _NULL if idx == torch.cuda.current_device() else torch.cuda.device(idx)


def _ptr(t) -> int:
    return t.data_ptr() if t is not None and t.numel() else 0


def _stream(stream, device):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream


def _check_u8(t, name):
    torch = _torch()
    if t.dtype != torch.uint8 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous uint8 CUDA tensor")


def b64_encode(src, dst=None, stream=None):
    """Encode ``src`` (uint8 CUDA tensor); returns the characters (uint8)."""
    torch = _torch()
    _check_u8(src, "src")
    n = src.numel()
    m = b64_encoded_len(n)
    if dst is None:
        dst = torch.empty(m, dtype=torch.uint8, device=src.device)
    _check_u8(dst, "dst")
    if dst.numel() < m:
        raise ValueError("dst is too small")
    with _on(src.device):
        r = lib().b64_encode(_ptr(src), n, _ptr(dst), _stream(stream, src.device))
    if r == SIZE_MAX:
        raise Gb64Error(B64_ERR_ARG, b64_last_error())
    return dst[:m]


def b64_decode(src, dst=None, stream=None):
    """Synchronous decode. Returns ``(status, outlen, first_bad, dst)``."""
    torch = _torch()
    _check_u8(src, "src")
    m = src.numel()
    cap = b64_decoded_cap(m)
    if dst is None:
        dst = torch.empty(max(cap, 1), dtype=torch.uint8, device=src.device)
    _check_u8(dst, "dst")
    if dst.numel() < cap:
        raise ValueError(f"dst holds {dst.numel()} bytes; decoding may write {cap}")
    outlen = ctypes.c_size_t(0)
    first_bad = ctypes.c_size_t(0)
    with _on(src.device):
        st = lib().b64_decode(_ptr(src), m, _ptr(dst) if cap else 0, ctypes.byref(outlen),
                              ctypes.byref(first_bad), _stream(stream, src.device))
    if st < 0:
        raise Gb64Error(st, b64_last_error())
    return st, int(outlen.value), int(first_bad.value), dst


def b64_decode_async(src, dst, result, stream=None):
    """Enqueue a decode; ``result`` is an int64 CUDA tensor of 3 entries that
    receives (first_bad, outlen, status | internal << 32)."""
    torch = _torch()
    _check_u8(src, "src")
    if result.dtype != torch.int64 or result.numel() < 3 or not result.is_cuda:
        raise ValueError("result must be an int64 CUDA tensor with 3 entries")
    m = src.numel()
    with _on(src.device):
        st = lib().b64_decode_async(_ptr(src), m, _ptr(dst) if b64_decoded_cap(m) else 0,
                                    result.data_ptr(), _stream(stream, src.device))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())


def parse_result(result) -> tuple:
    """(status, outlen, first_bad) from a result tensor of b64_decode_async."""
    r = result.cpu().numpy()
    status = int(np.int32(r[2] & 0xFFFFFFFF))
    return status, int(r[1]), int(r[0])


def _host_u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    if hasattr(a, "numpy") and not isinstance(a, np.ndarray):  # torch CPU tensor
        a = a.numpy()
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8:
        a = a.view(np.uint8)
    return a


def b64_encode_host(h_src, h_dst=None, stream=None):
    """Encode host memory (numpy/bytes/CPU tensor); returns a numpy array."""
    torch = _torch()
    src = _host_u8(h_src)
    m = b64_encoded_len(src.size)
    dst = np.empty(max(m, 1), dtype=np.uint8) if h_dst is None else _host_u8(h_dst)
    if dst.size < m:
        raise ValueError(f"h_dst holds {dst.size} bytes; the encoding needs {m}")
    r = lib().b64_encode_host(src.ctypes.data if src.size else 0, src.size, dst.ctypes.data,
                              _stream(stream, torch.cuda.current_device()))
    if r == SIZE_MAX:
        raise Gb64Error(B64_ERR_ARG, b64_last_error())
    return dst[:m]


def b64_decode_host(h_src, h_dst=None, stream=None):
    """Decode host memory; returns ``(status, outlen, first_bad, dst)``."""
    torch = _torch()
    src = _host_u8(h_src)
    cap = b64_decoded_cap(src.size)
    dst = np.empty(max(cap, 1), dtype=np.uint8) if h_dst is None else _host_u8(h_dst)
    if dst.size < cap:
        raise ValueError(f"h_dst holds {dst.size} bytes; decoding may write {cap}")
    outlen = ctypes.c_size_t(0)
    first_bad = ctypes.c_size_t(0)
    st = lib().b64_decode_host(src.ctypes.data if src.size else 0, src.size, dst.ctypes.data,
                               ctypes.byref(outlen), ctypes.byref(first_bad),
                               _stream(stream, torch.cuda.current_device()))
    if st < 0:
        raise Gb64Error(st, b64_last_error())
    return st, int(outlen.value), int(first_bad.value), dst


def _nonempty(t):
    """A tensor with a valid device pointer: batches of empty messages still
    pass real buffers to the C ABI."""
    torch = _torch()
    return t if t.numel() else torch.empty(1, dtype=t.dtype, device=t.device)


def _check_off(t, name):
    torch = _torch()
    if t.dtype != torch.int64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous int64 CUDA tensor")


def b64_batch_out_offsets(decode: bool, in_off, out_off=None, stream=None):
    """Output offsets (exclusive prefix of encoded lengths or decode
    capacities) of packed messages; returns an int64 CUDA tensor."""
    torch = _torch()
    _check_off(in_off, "in_off")
    nmsg = in_off.numel() - 1
    if out_off is None:
        out_off = torch.empty(nmsg + 1, dtype=torch.int64, device=in_off.device)
    with _on(in_off.device):
        st = lib().b64_batch_out_offsets(1 if decode else 0, in_off.data_ptr(), nmsg,
                                         out_off.data_ptr(), _stream(stream, in_off.device))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return out_off


def b64_encode_batch(src, in_off, dst=None, out_off=None, stream=None, check_dst=False):
    """Encode packed messages; returns ``(dst, out_off)``."""
    torch = _torch()
    _check_u8(src, "src")
    _check_off(in_off, "in_off")
    nmsg = in_off.numel() - 1
    if out_off is None:
        out_off = torch.empty(nmsg + 1, dtype=torch.int64, device=in_off.device)
    if dst is None or check_dst:
        b64_batch_out_offsets(False, in_off, out_off, stream)
        need = int(out_off[-1].item())
        if dst is None:
            dst = torch.empty(max(need, 1), dtype=torch.uint8, device=src.device)
        elif dst.numel() < need:
            raise ValueError(f"dst holds {dst.numel()} bytes; the batch needs {need}")
    with _on(src.device):
        src, dst = _nonempty(src), _nonempty(dst)
        st = lib().b64_encode_batch(_ptr(src), in_off.data_ptr(), nmsg, _ptr(dst),
                                    out_off.data_ptr(), _stream(stream, src.device))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return dst, out_off


def b64_decode_batch(src, in_off, dst=None, out_off=None, status=None, first_bad=None,
                     outlen=None, stream=None, check_dst=False):
    """Decode packed messages; returns ``(dst, out_off, status, first_bad, outlen)``.
    A caller-provided ``dst`` must hold the sum of the decode capacities
    (``out_off[-1]``); ``check_dst=True`` verifies that first (one scan and a
    host read)."""
    torch = _torch()
    _check_u8(src, "src")
    _check_off(in_off, "in_off")
    nmsg = in_off.numel() - 1
    dev = src.device
    if out_off is None:
        out_off = torch.empty(nmsg + 1, dtype=torch.int64, device=dev)
    if dst is None or check_dst:
        b64_batch_out_offsets(True, in_off, out_off, stream)
        need = int(out_off[-1].item())
        if dst is None:
            dst = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        elif dst.numel() < need:
            raise ValueError(f"dst holds {dst.numel()} bytes; the batch needs {need}")
    if status is None:
        status = torch.empty(max(nmsg, 1), dtype=torch.int32, device=dev)
    if first_bad is None:
        first_bad = torch.empty(max(nmsg, 1), dtype=torch.int64, device=dev)
    if outlen is None:
        outlen = torch.empty(max(nmsg, 1), dtype=torch.int64, device=dev)
    with _on(dev):
        src, dst = _nonempty(src), _nonempty(dst)
        st = lib().b64_decode_batch(_ptr(src), in_off.data_ptr(), nmsg, _ptr(dst),
                                    out_off.data_ptr(), status.data_ptr(), first_bad.data_ptr(),
                                    outlen.data_ptr(), _stream(stream, dev))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return dst, out_off, status[:nmsg], first_bad[:nmsg], outlen[:nmsg]


# ------------------------------------------------------------------ tuner
def b64_shape_get(kind: int, total: int, nmsg: int = 1) -> dict:
    out = b64_shape()
    st = lib().b64_shape_get(kind, total, nmsg, ctypes.byref(out))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return out.as_dict()


def b64_shape_set(kind: int, total: int, nmsg: int = 1, **shape) -> None:
    cur = b64_shape(**{k: v for k, v in b64_shape_get(kind, total, nmsg).items()})
    for k, v in shape.items():
        setattr(cur, k, v)
    st = lib().b64_shape_set(kind, total, nmsg, ctypes.byref(cur))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())


def b64_tune(kind: int, total: int, nmsg: int = 1, stream=None, max_trials: int = 256):
    """Autotune the bucket of (kind, total, nmsg); returns the timed trials."""
    torch = _torch()
    trials = (b64_shape * max_trials)()
    n = ctypes.c_int(0)
    st = lib().b64_tune(kind, total, nmsg, trials, max_trials, ctypes.byref(n),
                        _stream(stream, torch.cuda.current_device()))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return [trials[i].as_dict() for i in range(n.value)]


def b64_tune_save(path: str) -> None:
    if lib().b64_tune_save(path.encode()) != B64_OK:
        raise Gb64Error(B64_ERR_ARG, b64_last_error())


def b64_tune_load(path: str) -> None:
    if lib().b64_tune_load(path.encode()) != B64_OK:
        raise Gb64Error(B64_ERR_ARG, b64_last_error())


# ---------------------------------------------------------------- server
def device_view(addr: int, n: int):
    """A uint8 CUDA tensor viewing ``n`` bytes at device address ``addr``
    (no copy; e.g. a completion's output, valid until it is released)."""
    torch = _torch()

    class _View:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (addr, False),
                                    "version": 3, "strides": None}

    return torch.as_tensor(_View(), device="cuda")



class Server:
    """Handle of a serving engine (``b64_server_create``); ``close()`` or the
    context manager destroys it."""

    def __init__(self, memory_budget=8 << 30, streams=4, max_batch_msgs=4096,
                 max_batch_bytes=256 << 20, auto_release=False):
        cfg = b64_server_config(memory_budget, streams, max_batch_msgs, max_batch_bytes,
                                1 if auto_release else 0, 0)
        h = lib().b64_server_create(ctypes.byref(cfg))
        if not h:
            raise Gb64Error(B64_ERR_ARG, b64_last_error())
        self.h = ctypes.c_void_p(h)
        self._keep = []

    def now_us(self) -> float:
        return float(lib().b64_server_now_us(self.h))

    def submit(self, kind: int, src, length: int | None = None, t_arrival_us: float = -1.0) -> int:
        """Queue a request on device memory ``src`` (tensor or address)."""
        ptr = src if isinstance(src, int) else src.data_ptr()
        n = length if length is not None else src.numel()
        rid = ctypes.c_int64(-1)
        st = lib().b64_server_submit(self.h, kind, ptr, n, t_arrival_us, ctypes.byref(rid))
        if st != B64_OK:
            raise Gb64Error(st, b64_last_error())
        return int(rid.value)

    def poll(self, max_items: int = 4096, timeout_us: int = 1000) -> list:
        buf = (b64_completion * max_items)()
        k = lib().b64_server_poll(self.h, buf, max_items, timeout_us)
        if k < 0:
            raise Gb64Error(k, b64_last_error())
        return [buf[i].as_dict() for i in range(k)]

    def release(self, rid: int) -> None:
        st = lib().b64_server_release(self.h, rid)
        if st != B64_OK:
            raise Gb64Error(st, b64_last_error())

    def stats(self) -> dict:
        out = b64_server_stats()
        lib().b64_server_stats_get(self.h, ctypes.byref(out))
        return out.as_dict()

    def replay(self, t_arrival_us, kind, src_ptrs, length):
        """Open-loop replay from native threads; returns (latency_us, status)."""
        t = np.ascontiguousarray(t_arrival_us, dtype=np.float64)
        k = np.ascontiguousarray(kind, dtype=np.int32)
        sp = np.ascontiguousarray(src_ptrs, dtype=np.uint64)
        ln = np.ascontiguousarray(length, dtype=np.int64)
        lat = np.full(t.size, -1.0)
        st = np.zeros(t.size, dtype=np.int32)
        rc = lib().b64_server_replay(self.h, t.size, t.ctypes.data, k.ctypes.data, sp.ctypes.data,
                                     ln.ctypes.data, lat.ctypes.data, st.ctypes.data)
        if rc != B64_OK:
            raise Gb64Error(rc, b64_last_error())
        return lat, st

    def close(self):
        if self.h:
            lib().b64_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def b64_server_create(**cfg) -> Server:
    return Server(**cfg)


# ------------------------------------------------ variants (flags, _ex calls)
def b64_encoded_len_ex(n: int, flags: int) -> int:
    return int(lib().b64_encoded_len_ex(n, flags))


def b64_decoded_cap_ex(m: int, flags: int) -> int:
    return int(lib().b64_decoded_cap_ex(m, flags))


def b64_encode_ex(src, flags: int, dst=None, stream=None):
    torch = _torch()
    _check_u8(src, "src")
    n = src.numel()
    m = b64_encoded_len_ex(n, flags)
    if dst is None:
        dst = torch.empty(max(m, 1), dtype=torch.uint8, device=src.device)
    _check_u8(dst, "dst")
    if dst.numel() < m:
        raise ValueError("dst is too small")
    with _on(src.device):
        r = lib().b64_encode_ex(_ptr(src), n, _ptr(dst), flags, _stream(stream, src.device))
    if r == SIZE_MAX:
        raise Gb64Error(B64_ERR_ARG, b64_last_error())
    return dst[:m]


def b64_decode_ex(src, flags: int, dst=None, stream=None):
    """Synchronous decode with flags. Returns ``(status, outlen, first_bad, dst)``."""
    torch = _torch()
    _check_u8(src, "src")
    m = src.numel()
    cap = b64_decoded_cap_ex(m, flags)
    if dst is None:
        dst = torch.empty(max(cap, 1), dtype=torch.uint8, device=src.device)
    _check_u8(dst, "dst")
    if dst.numel() < cap:
        raise ValueError(f"dst holds {dst.numel()} bytes; decoding may write {cap}")
    outlen = ctypes.c_size_t(0)
    first_bad = ctypes.c_size_t(0)
    with _on(src.device):
        st = lib().b64_decode_ex(_ptr(src), m, _ptr(dst) if cap else 0, ctypes.byref(outlen),
                                 ctypes.byref(first_bad), flags, _stream(stream, src.device))
    if st < 0:
        raise Gb64Error(st, b64_last_error())
    return st, int(outlen.value), int(first_bad.value), dst


def b64_decode_async_ex(src, dst, result, flags: int, stream=None):
    torch = _torch()
    _check_u8(src, "src")
    m = src.numel()
    with _on(src.device):
        st = lib().b64_decode_async_ex(_ptr(src), m, _ptr(dst) if b64_decoded_cap_ex(m, flags) else 0,
                                       result.data_ptr(), flags, _stream(stream, src.device))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())


def b64_batch_out_offsets_ex(decode: bool, in_off, flags: int, out_off=None, stream=None):
    torch = _torch()
    _check_off(in_off, "in_off")
    nmsg = in_off.numel() - 1
    if out_off is None:
        out_off = torch.empty(nmsg + 1, dtype=torch.int64, device=in_off.device)
    with _on(in_off.device):
        st = lib().b64_batch_out_offsets_ex(1 if decode else 0, in_off.data_ptr(), nmsg,
                                            out_off.data_ptr(), flags, _stream(stream, in_off.device))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return out_off


def b64_encode_batch_ex(src, in_off, flags: int, dst=None, out_off=None, stream=None):
    torch = _torch()
    _check_u8(src, "src")
    _check_off(in_off, "in_off")
    nmsg = in_off.numel() - 1
    if out_off is None:
        out_off = torch.empty(nmsg + 1, dtype=torch.int64, device=in_off.device)
    if dst is None:
        b64_batch_out_offsets_ex(False, in_off, flags, out_off, stream)
        dst = torch.empty(max(int(out_off[-1].item()), 1), dtype=torch.uint8, device=src.device)
    with _on(src.device):
        src, dst = _nonempty(src), _nonempty(dst)
        st = lib().b64_encode_batch_ex(_ptr(src), in_off.data_ptr(), nmsg, _ptr(dst),
                                       out_off.data_ptr(), flags, _stream(stream, src.device))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return dst, out_off


def b64_decode_batch_ex(src, in_off, flags: int, dst=None, out_off=None, status=None,
                        first_bad=None, outlen=None, stream=None, check_dst=False):
    torch = _torch()
    _check_u8(src, "src")
    _check_off(in_off, "in_off")
    nmsg = in_off.numel() - 1
    dev = src.device
    if out_off is None:
        out_off = torch.empty(nmsg + 1, dtype=torch.int64, device=dev)
    if dst is None or check_dst:
        b64_batch_out_offsets_ex(True, in_off, flags, out_off, stream)
        need = int(out_off[-1].item())
        if dst is None:
            dst = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        elif dst.numel() < need:
            raise ValueError(f"dst holds {dst.numel()} bytes; the batch needs {need}")
    status = torch.empty(max(nmsg, 1), dtype=torch.int32, device=dev) if status is None else status
    first_bad = torch.empty(max(nmsg, 1), dtype=torch.int64, device=dev) if first_bad is None else first_bad
    outlen = torch.empty(max(nmsg, 1), dtype=torch.int64, device=dev) if outlen is None else outlen
    with _on(dev):
        src, dst = _nonempty(src), _nonempty(dst)
        st = lib().b64_decode_batch_ex(_ptr(src), in_off.data_ptr(), nmsg, _ptr(dst),
                                       out_off.data_ptr(), status.data_ptr(), first_bad.data_ptr(),
                                       outlen.data_ptr(), flags, _stream(stream, dev))
    if st != B64_OK:
        raise Gb64Error(st, b64_last_error())
    return dst, out_off, status[:nmsg], first_bad[:nmsg], outlen[:nmsg]
