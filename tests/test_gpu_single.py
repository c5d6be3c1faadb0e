"""GPU parity of the single-buffer codec against the CPU oracle.

Integer codec: every comparison is exact (bytes, status, first_bad, outlen).
Cases: the paper's examples, brute force over all 2^24 three-byte groups and
all 64^4 valid quads, every byte value at every position of a quad, lengths
across several tiles with ragged tails, every alignment of src and dst,
guard bytes around dst, injected errors, the 1 MiB and 1 GiB workloads.
"""
import base64

import numpy as np
import pytest

from tests import golden

pytestmark = pytest.mark.gpu

GUARD = 64
ENC_TILE = 256 * 4 * 12    # input bytes per tile of the TMA encode kernel
DEC_TILE = 256 * 4 * 16    # characters per tile of the TMA decode kernel


def to_dev(a, offset=0, extra=0):
    """Device copy of host bytes starting at byte ``offset`` of a fresh
    allocation (so ``offset`` sets the pointer's alignment)."""
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint8)
    buf = torch.empty(offset + a.size + extra + 1, dtype=torch.uint8, device="cuda")
    t = buf[offset:offset + a.size]
    if a.size:
        t.copy_(torch.from_numpy(a))
    return t


def guarded(n, offset=0, fill=0xA5):
    import torch

    buf = torch.full((GUARD + offset + n + GUARD,), fill, dtype=torch.uint8, device="cuda")
    return buf, buf[GUARD + offset:GUARD + offset + n]


def check_guards(buf, offset, n, fill=0xA5):
    h = buf.cpu().numpy()
    assert (h[:GUARD + offset] == fill).all(), "write before dst"
    assert (h[GUARD + offset + n:] == fill).all(), "write after dst"


def gpu_encode(gb64, raw, src_off=0, dst_off=0):
    import torch

    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    src = to_dev(raw, src_off)
    m = gb64.b64_encoded_len(raw.size)
    buf, dst = guarded(max(m, 1), dst_off)
    out = gb64.b64_encode(src, dst)
    torch.cuda.synchronize()
    check_guards(buf, dst_off, max(m, 1))
    return out.cpu().numpy()[:m]


def gpu_decode(gb64, chars, src_off=0, dst_off=0):
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    src = to_dev(chars, src_off)
    cap = gb64.b64_decoded_cap(chars.size)
    buf, dst = guarded(max(cap, 1), dst_off)
    st, outlen, fb, d = gb64.b64_decode(src, dst)
    check_guards(buf, dst_off, max(cap, 1))
    return st, d.cpu().numpy()[:outlen], fb


# ------------------------------------------------------------ the paper
def test_paper_examples(gb64, oracle):
    out = gpu_encode(gb64, np.array(golden.ints("encode_example_bytes"), dtype=np.uint8))
    assert out.tobytes() == golden.text("encode_example_chars").encode()
    chars = np.frombuffer(golden.text("decode_example_chars").encode(), dtype=np.uint8)
    st, out, fb = gpu_decode(gb64, chars)
    assert st == 0 and fb == chars.size
    assert list(out) == golden.ints("decode_example_bytes")
    chars = np.frombuffer(golden.text("appc_chars").encode(), dtype=np.uint8)
    st, out, fb = gpu_decode(gb64, chars)
    assert st == 0 and np.array_equal(out, oracle.decode(chars)[1])


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("src_off,dst_off", [(0, 0), (1, 0), (0, 4), (5, 7)])
def test_encode_all_three_byte_groups(gb64, oracle, src_off, dst_off):
    g = np.arange(1 << 24, dtype=np.uint32)
    raw = np.empty((1 << 24, 3), dtype=np.uint8)
    raw[:, 0] = g >> 16
    raw[:, 1] = (g >> 8) & 0xFF
    raw[:, 2] = g & 0xFF
    raw = raw.reshape(-1)
    out = gpu_encode(gb64, raw, src_off, dst_off)
    assert np.array_equal(out, oracle.encode(raw))


@pytest.mark.parametrize("src_off,dst_off", [(0, 0), (3, 1)])
def test_decode_all_valid_quads(gb64, oracle, src_off, dst_off):
    alpha = np.array([oracle.table1_char(v) for v in range(64)], dtype=np.uint8)
    q = np.arange(64 ** 4, dtype=np.uint32)
    chars = np.empty((64 ** 4, 4), dtype=np.uint8)
    chars[:, 0] = alpha[q >> 18]
    chars[:, 1] = alpha[(q >> 12) & 63]
    chars[:, 2] = alpha[(q >> 6) & 63]
    chars[:, 3] = alpha[q & 63]
    chars = chars.reshape(-1)
    st, out, fb = gpu_decode(gb64, chars, src_off, dst_off)
    ost, oout, ofb = oracle.decode(chars)
    assert st == ost == 0 and fb == ofb
    assert np.array_equal(out, oout)


CONTEXTS = [b"QUJDREVGR0lG", b"R0lGQUJD", b"R0lGQUI=", b"R0lGQQ=="]


def test_every_byte_at_every_quad_position(gb64, oracle):
    """256 byte values x each position of the final quad and of a middle quad
    (the same cases the oracle is pinned on), one GPU decode each."""
    for base in CONTEXTS:
        for q in range(len(base)):
            for x in range(256):
                s = bytearray(base)
                s[q] = x
                s = np.frombuffer(bytes(s), dtype=np.uint8)
                got = gpu_decode(gb64, s)
                exp = oracle.decode(s)
                assert got[0] == exp[0] and got[2] == exp[2], (bytes(s), got, exp)
                if exp[0] == 0:
                    assert np.array_equal(got[1], exp[1])


# ------------------------------------------------- lengths and alignment
def _lengths():
    ls = list(range(0, 80))
    for k in (1, 2, 3, 7):
        for d in (-13, -12, -3, -2, -1, 0, 1, 2, 3, 12, 13, 16, 17):
            ls.append(k * ENC_TILE + d)
            ls.append(k * DEC_TILE + d)
    return sorted(set(l for l in ls if l >= 0))


@pytest.mark.parametrize("n", _lengths())
def test_round_trip_lengths(gb64, oracle, n):
    rng = np.random.default_rng(n)
    raw = rng.integers(0, 256, n, dtype=np.uint8)
    enc = gpu_encode(gb64, raw)
    assert np.array_equal(enc, oracle.encode(raw))
    st, out, fb = gpu_decode(gb64, enc)
    assert st == 0 and fb == enc.size and np.array_equal(out, raw)


@pytest.mark.parametrize("src_off", range(16))
@pytest.mark.parametrize("dst_off", [0, 1, 2, 3, 4, 8, 12, 15])
def test_every_alignment(gb64, oracle, src_off, dst_off):
    rng = np.random.default_rng(100 * src_off + dst_off)
    n = int(rng.integers(3 * ENC_TILE, 3 * ENC_TILE + 100))
    raw = rng.integers(0, 256, n, dtype=np.uint8)
    enc = gpu_encode(gb64, raw, src_off, dst_off)
    assert np.array_equal(enc, oracle.encode(raw))
    st, out, fb = gpu_decode(gb64, enc, src_off, dst_off)
    assert st == 0 and np.array_equal(out, raw)


def test_random_lengths(gb64, oracle):
    rng = np.random.default_rng(5)
    for _ in range(60):
        n = int(rng.integers(0, 100_000))
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        so, do = int(rng.integers(0, 16)), int(rng.integers(0, 16))
        enc = gpu_encode(gb64, raw, so, do)
        assert np.array_equal(enc, oracle.encode(raw))
        st, out, fb = gpu_decode(gb64, enc, do, so)
        assert st == 0 and np.array_equal(out, raw)


# ------------------------------------------------------------------ errors
def test_injected_errors_multi_tile(gb64, oracle):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    rng = np.random.default_rng(11)
    for trial in range(120):
        n = int(rng.integers(1, 6 * DEC_TILE))
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        enc = oracle.encode(raw).copy()
        k = int(rng.integers(1, 4))
        pos = rng.integers(0, enc.size, k)
        enc[pos] = NON_ALPHABET_NON_PAD[rng.integers(0, 191, k)]
        if trial % 3 == 0:  # sometimes also a misplaced '='
            enc[int(rng.integers(0, enc.size))] = 0x3D
        off = int(rng.integers(0, 16)) if trial % 2 else 0
        got = gpu_decode(gb64, enc, off, off)
        exp = oracle.decode(enc)
        assert got[0] == exp[0] and got[2] == exp[2], (trial, got[:1], got[2], exp[0], exp[2])


@pytest.mark.parametrize("m", list(range(1, 40)) + [DEC_TILE + 1, DEC_TILE + 2, DEC_TILE + 3,
                                                    3 * DEC_TILE + 5])
def test_bad_lengths_and_tails(gb64, oracle, m):
    rng = np.random.default_rng(m)
    alpha = np.array([oracle.table1_char(v) for v in range(64)], dtype=np.uint8)
    s = alpha[rng.integers(0, 64, m)]
    for variant in range(4):
        t = s.copy()
        if variant == 1 and m >= 1:
            t[-1] = 0x3D
        if variant == 2 and m >= 2:
            t[-2:] = 0x3D
        if variant == 3 and m >= 3:
            t[-3:] = 0x3D
        got = gpu_decode(gb64, t)
        exp = oracle.decode(t)
        assert got[0] == exp[0] and got[2] == exp[2], (m, variant, got, exp)
        if exp[0] == 0:
            assert np.array_equal(got[1], exp[1])


def test_degenerate(gb64, oracle):
    import torch

    assert gb64.b64_encode(torch.empty(0, dtype=torch.uint8, device="cuda")).numel() == 0
    st, outlen, fb, _ = gb64.b64_decode(torch.empty(0, dtype=torch.uint8, device="cuda"))
    assert (st, outlen, fb) == (0, 0, 0)
    for s in [b"=", b"==", b"===", b"====", b"A", b"AA", b"AAA", b"AA==", b"AAA=", b"A===",
              b"AAAA====", b"\x00\x00\x00\x00", b"\xff" * 8, b"AAAA\n", b" AAA"]:
        a = np.frombuffer(s, dtype=np.uint8)
        got = gpu_decode(gb64, a)
        exp = oracle.decode(a)
        assert got[0] == exp[0] and got[2] == exp[2], (s, got, exp)


# -------------------------------------------------------- other entry points
def test_decode_async_result(gb64, oracle):
    import torch

    raw = np.random.default_rng(1).integers(0, 256, 100_001, dtype=np.uint8)
    enc = oracle.encode(raw).copy()
    enc[77_777] = ord("!")
    src = to_dev(enc)
    dst = torch.empty(gb64.b64_decoded_cap(enc.size), dtype=torch.uint8, device="cuda")
    res = torch.empty(3, dtype=torch.int64, device="cuda")
    gb64.b64_decode_async(src, dst, res)
    assert gb64.parse_result(res) == (1, 0, 77_777)
    enc[77_777] = oracle.encode(raw)[77_777]
    gb64.b64_decode_async(to_dev(enc), dst, res)
    st, outlen, fb = gb64.parse_result(res)
    assert (st, outlen, fb) == (0, raw.size, enc.size)
    assert np.array_equal(dst.cpu().numpy()[:outlen], raw)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 1000, (48 << 20) + 7, (100 << 20) + 1])
def test_host_buffer_forms(gb64, oracle, n):
    rng = np.random.default_rng(n % 1000)
    raw = rng.integers(0, 256, n, dtype=np.uint8)
    enc = gb64.b64_encode_host(raw)
    if n < (1 << 20):
        assert np.array_equal(enc, oracle.encode(raw))
    else:
        assert enc.tobytes() == base64.b64encode(raw.tobytes())
    st, outlen, fb, out = gb64.b64_decode_host(enc)
    assert st == 0 and outlen == n and fb == enc.size
    assert np.array_equal(out[:outlen], raw)
    if enc.size > 8:
        bad = enc.copy()
        p = enc.size - 5
        bad[p] = 0x00
        st, outlen, fb, _ = gb64.b64_decode_host(bad)
        assert (st, outlen, fb) == (1, 0, p)


# ----------------------------------------------------------- the workloads
def test_workload_single_1mib(gb64, oracle):
    from paper_1704_00605_gb300 import workloads as W

    raw = W.single_message()
    enc = gpu_encode(gb64, raw)
    assert np.array_equal(enc, oracle.encode(raw))
    assert enc.size == 1_398_104 and enc[-2:].tobytes() == b"=="
    st, out, fb = gpu_decode(gb64, enc)
    assert st == 0 and np.array_equal(out, raw)
    pos = W.single_message_error_offset(enc.size - 2)
    bad = enc.copy()
    bad[pos] = 0x21
    st, out, fb = gpu_decode(gb64, bad)
    assert (st, fb) == (1, pos)
    assert oracle.decode(bad)[0] == 1 and oracle.decode(bad)[2] == pos


def test_workload_large_1gib(gb64, oracle):
    """Full size, in the launch shapes the benchmark times, every byte: for
    each of the three lengths the whole encoding is compared with the
    oracle's, and the whole decode output with the oracle's decode of that
    encoding (so an encode bug that the decode undid would still show), the
    oracle running over aligned chunks (48 MiB of bytes, 64 Mi characters)
    on all host cores; then one injected error is located exactly."""
    import concurrent.futures as cf
    import os

    import torch

    from paper_1704_00605_gb300 import workloads as W

    data = W.large_buffer()
    src_all = torch.from_numpy(data).cuda()
    rng = np.random.default_rng(77)
    threads = os.cpu_count() or 4
    CB, CC = 48 << 20, 64 << 20  # chunk of bytes (multiple of 3) and of characters (of 4)
    for n in W.LARGE_LENGTHS:
        src = src_all[:n]
        enc = gb64.b64_encode(src)
        m = enc.numel()
        assert m == 1_431_655_768
        enc_h = enc.cpu().numpy()
        assert enc_h[-4:].tobytes().count(b"=") == (3 - n % 3) % 3

        def check_enc(i):
            a = i * CB
            exp = oracle.encode(data[a:min(n, a + CB)])
            return np.array_equal(enc_h[a // 3 * 4:a // 3 * 4 + exp.size], exp)

        with cf.ThreadPoolExecutor(threads) as ex:
            ok = list(ex.map(check_enc, range((n + CB - 1) // CB)))
        assert all(ok), [i for i, x in enumerate(ok) if not x]
        dst = torch.empty(gb64.b64_decoded_cap(m), dtype=torch.uint8, device="cuda")
        st, outlen, fb, dst = gb64.b64_decode(enc, dst)
        assert (st, outlen, fb) == (0, n, m)
        dec_h = dst[:n].cpu().numpy()
        del dst

        def check_dec(i):
            a = i * CC
            ost, oout, ofb = oracle.decode(enc_h[a:min(m, a + CC)])
            return ost == 0 and np.array_equal(dec_h[a // 4 * 3:a // 4 * 3 + oout.size], oout)

        with cf.ThreadPoolExecutor(threads) as ex:
            ok = list(ex.map(check_dec, range((m + CC - 1) // CC)))
        assert all(ok), [i for i, x in enumerate(ok) if not x]
        del enc_h, dec_h
    # one error at a random place of the last encoding
    pos = int(rng.integers(0, enc.numel() - 4))
    enc[pos] = 0x21
    st, outlen, fb, _ = gb64.b64_decode(enc)
    assert (st, outlen, fb) == (1, 0, pos)
    assert gb64.b64_device_fault() == 0
