"""Seeded synthetic inputs for the base64 codec.

This module is shared by the tests, the benchmark and the CPU oracle checks,
so it holds no base64 arithmetic at all: it only draws bytes, lengths,
positions and arrival times. Every array is a pure function of its seed.

Workloads (uniform random bytes, the input model of the paper's length sweep
in Section 5):

* ``single_message``   1 MiB of uniform bytes, seed 0, plus one seeded
  position for an injected '!' (0x21).
* ``large_buffer``     1 GiB + 2 uniform bytes, seed 1; the three lengths
  2^30, 2^30+1, 2^30+2 are prefixes of the same array.
* ``batched``          100,000 messages, log-normal lengths (median 2 KiB,
  sigma 1.5, clipped to [1, 2^20]), uniform bytes, seed 2.
* ``error_batch``      messages of uniform length in [16, 65536] with 1% of
  them carrying one byte outside the alphabet and not '=' (seed 3). Payload
  bytes come from ``counter_bytes`` so that any slice can be regenerated on
  the host or on the device without materialising the whole set.
* ``serving``          Poisson arrivals, 50/50 encode/decode, log-normal
  payload lengths (median 4 KiB, sigma 2, clipped to [1, 2^24]), seed 4.
"""
from __future__ import annotations

import numpy as np

MIB = 1 << 20
GIB = 1 << 30

# Byte values that are neither in the RFC 4648 base64 alphabet nor '='
# (0x3D): the 191 values an error is drawn from. This is input data of the
# error workloads, listed as ranges of the byte table.
_NON_ALPHABET_RANGES = [(0x00, 0x2A), (0x2C, 0x2E), (0x3A, 0x3C), (0x3E, 0x40),
                        (0x5B, 0x60), (0x7B, 0xFF)]
NON_ALPHABET_NON_PAD = np.concatenate(
    [np.arange(lo, hi + 1, dtype=np.uint8) for lo, hi in _NON_ALPHABET_RANGES])
assert NON_ALPHABET_NON_PAD.size == 191


def uniform_bytes(n: int, seed: int) -> np.ndarray:
    """``n`` uniform random bytes from ``numpy.random.default_rng(seed)``."""
    return np.random.default_rng(seed).integers(0, 256, size=n, dtype=np.uint8)


# ---------------------------------------------------------------- config 1
def single_message(n: int = MIB, seed: int = 0) -> np.ndarray:
    """1 MiB of uniform bytes (seed 0)."""
    return uniform_bytes(n, seed)


def single_message_error_offset(limit: int, seed: int = 0) -> int:
    """Offset of the injected '!' in [0, limit), from its own stream [seed, 1].

    The caller passes ``limit`` = encoded length minus its padding count so
    that the expected first bad index equals the offset.
    """
    return int(np.random.default_rng([seed, 1]).integers(0, limit))


# ---------------------------------------------------------------- config 2
LARGE_LENGTHS = (GIB, GIB + 1, GIB + 2)


def large_buffer(seed: int = 1) -> np.ndarray:
    """2^30 + 2 uniform bytes (seed 1); each config length is a prefix."""
    return uniform_bytes(GIB + 2, seed)


# ---------------------------------------------------------------- config 3
def lognormal_lengths(rng: np.random.Generator, nmsg: int, median: float, sigma: float,
                      lo: int, hi: int) -> np.ndarray:
    z = rng.standard_normal(nmsg)
    lens = np.rint(np.exp(np.log(median) + sigma * z))
    return np.clip(lens, lo, hi).astype(np.int64)


def offsets_from_lengths(lens: np.ndarray) -> np.ndarray:
    off = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def batched(nmsg: int = 100_000, seed: int = 2, median: float = 2048.0, sigma: float = 1.5,
            max_len: int = MIB):
    """Packed messages: ``(payload_bytes, in_off)`` with int64 offsets."""
    rng = np.random.default_rng(seed)
    lens = lognormal_lengths(rng, nmsg, median, sigma, 1, max_len)
    off = offsets_from_lengths(lens)
    data = rng.integers(0, 256, size=int(off[-1]), dtype=np.uint8)
    return data, off


# ------------------------------------------------- counter-based byte stream
_M64 = (1 << 64) - 1
_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_MUL1 = 0xBF58476D1CE4E5B9
_SM_MUL2 = 0x94D049BB133111EB


def _splitmix64_np(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 counters."""
    with np.errstate(over="ignore"):
        z = x + np.uint64(_SM_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_MUL2)
        return z ^ (z >> np.uint64(31))


def counter_bytes(key: int, start: int, n: int) -> np.ndarray:
    """Bytes ``start .. start+n`` of the stream for ``key`` (host, numpy).

    Byte ``i`` of the stream is byte ``i % 8`` (little-endian) of
    SplitMix64(key * 2^40 + i // 8).
    """
    if n <= 0:
        return np.zeros(0, dtype=np.uint8)
    w0 = start // 8
    w1 = (start + n + 7) // 8
    ctr = np.arange(w0, w1, dtype=np.uint64) + np.uint64((key << 40) & _M64)
    words = _splitmix64_np(ctr).astype("<u8")
    b = words.view(np.uint8)
    s = start - 8 * w0
    return b[s:s + n].copy()


def _i64(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def counter_bytes_torch(key: int, start: int, n: int, device, chunk_words: int = 1 << 26):
    """Same stream as :func:`counter_bytes`, generated with torch int64 ops on
    ``device`` (so a large input never has to exist in host memory)."""
    import torch

    out = torch.empty(n, dtype=torch.uint8, device=device)
    if n <= 0:
        return out
    w0 = start // 8
    w1 = (start + n + 7) // 8
    s = start - 8 * w0
    pos = 0
    base = _i64((key << 40) & _M64)
    m30 = (1 << 34) - 1
    m27 = (1 << 37) - 1
    m31 = (1 << 33) - 1
    for c0 in range(w0, w1, chunk_words):
        c1 = min(w1, c0 + chunk_words)
        x = torch.arange(c0, c1, dtype=torch.int64, device=device) + base
        z = x + _i64(_SM_GAMMA)
        z = (z ^ ((z >> 30) & m30)) * _i64(_SM_MUL1)
        z = (z ^ ((z >> 27) & m27)) * _i64(_SM_MUL2)
        z = z ^ ((z >> 31) & m31)
        b = z.view(torch.uint8)  # little-endian on every target of this build
        lo = s if c0 == w0 else 0
        take = min(b.numel() - lo, n - pos)
        out[pos:pos + take] = b[lo:lo + take]
        pos += take
    assert pos == n
    return out


# ---------------------------------------------------------------- config 4
def error_batch(nmsg: int = 1_000_000, seed: int = 3, lo: int = 16, hi: int = 65536,
                err_fraction: float = 0.01):
    """Recipe of the batched-decode-with-errors workload.

    Returns ``dict(in_off, payload_key, err_msg, err_frac, err_byte)``:
    payload message ``j`` is ``counter_bytes(payload_key, in_off[j], len_j)``;
    message ``err_msg[k]`` gets byte ``err_byte[k]`` written over character
    ``floor(err_frac[k] * m)`` of its encoding of length ``m``
    (see :func:`inject_errors`).
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=nmsg, dtype=np.int64)
    in_off = offsets_from_lengths(lens)
    nerr = int(round(err_fraction * nmsg))
    err_msg = np.sort(rng.choice(nmsg, size=nerr, replace=False)).astype(np.int64)
    err_frac = rng.random(nerr)
    err_byte = NON_ALPHABET_NON_PAD[rng.integers(0, NON_ALPHABET_NON_PAD.size, size=nerr)]
    return dict(in_off=in_off, payload_key=seed, err_msg=err_msg, err_frac=err_frac,
                err_byte=err_byte)


def error_positions(enc_off: np.ndarray, err_msg: np.ndarray, err_frac: np.ndarray) -> np.ndarray:
    """Absolute character positions of the injected errors, given the encoded
    messages' offsets ``enc_off`` (length nmsg + 1)."""
    m = enc_off[err_msg + 1] - enc_off[err_msg]
    rel = np.floor(err_frac * m).astype(np.int64)
    rel = np.minimum(rel, np.maximum(m - 1, 0))
    return enc_off[err_msg] + rel


def inject_errors(encoded, enc_off: np.ndarray, err_msg: np.ndarray, err_frac: np.ndarray,
                  err_byte: np.ndarray):
    """Overwrite one character per chosen message, in place (numpy or torch)."""
    pos = error_positions(enc_off, err_msg, err_frac)
    if isinstance(encoded, np.ndarray):
        encoded[pos] = err_byte
    else:
        import torch

        encoded[torch.as_tensor(pos, device=encoded.device)] = torch.as_tensor(
            err_byte, device=encoded.device)
    return pos


# ---------------------------------------------------------------- config 5
def serving(duration_s: float = 30.0, rate_hz: float = 200_000.0, seed: int = 4,
            median: float = 4096.0, sigma: float = 2.0, max_len: int = 1 << 24):
    """Request stream: ``dict(t_arrival, is_decode, length, pool_pos)``.

    ``pool_pos`` in [0, 1) places each request's payload in a resident pool
    of random bytes (the pool itself is ``counter_bytes(seed, ...)``).
    """
    rng = np.random.default_rng(seed)
    nexp = int(duration_s * rate_hz * 1.2) + 16
    gaps = rng.exponential(1.0 / rate_hz, size=nexp)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    nreq = t.size
    is_decode = rng.random(nreq) < 0.5
    length = lognormal_lengths(rng, nreq, median, sigma, 1, max_len)
    pool_pos = rng.random(nreq)
    return dict(t_arrival=t, is_decode=is_decode, length=length, pool_pos=pool_pos)
