"""GPU parity of the codec variants (base64url, omitted padding, Appendix A's
tail check) against the oracle's variant functions, exact, on the single-
buffer kernels (TMA and generic), the batched kernels and a large buffer."""
import itertools

import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

URL, NOPAD, STRICT = 1, 2, 4
ALL_FLAGS = [URL, NOPAD, STRICT, URL | NOPAD, URL | STRICT, NOPAD | STRICT, URL | NOPAD | STRICT]


def dev(a, off=0):
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint8)
    buf = torch.empty(off + a.size + 1, dtype=torch.uint8, device="cuda")
    t = buf[off:off + a.size]
    if a.size:
        t.copy_(torch.from_numpy(a.copy()))
    return t


def test_url_encode_all_three_byte_groups(gb64, oracle):
    g = np.arange(1 << 24, dtype=np.uint32)
    raw = np.empty((1 << 24, 3), dtype=np.uint8)
    raw[:, 0], raw[:, 1], raw[:, 2] = g >> 16, (g >> 8) & 0xFF, g & 0xFF
    raw = raw.reshape(-1)
    for off in (0, 3):
        out = gb64.b64_encode_ex(dev(raw, off), URL).cpu().numpy()
        assert np.array_equal(out, oracle.encode_ex(raw, URL))


def test_url_decode_all_valid_quads(gb64, oracle):
    alpha = oracle.encode_ex(np.frombuffer(
        int("".join(f"{v:06b}" for v in range(64)), 2).to_bytes(48, "big"), dtype=np.uint8), URL)
    q = np.arange(64 ** 4, dtype=np.uint32)
    chars = np.empty((64 ** 4, 4), dtype=np.uint8)
    chars[:, 0], chars[:, 1] = alpha[q >> 18], alpha[(q >> 12) & 63]
    chars[:, 2], chars[:, 3] = alpha[(q >> 6) & 63], alpha[q & 63]
    chars = chars.reshape(-1)
    st, outlen, fb, d = gb64.b64_decode_ex(dev(chars), URL)
    ost, oout, ofb = oracle.decode_ex(chars, URL)
    assert (st, fb) == (ost, ofb) == (0, chars.size)
    assert np.array_equal(d[:outlen].cpu().numpy(), oout)


@pytest.mark.parametrize("flags", [URL, NOPAD, URL | NOPAD])
def test_encode_decode_lengths_and_alignments(gb64, oracle, flags):
    rng = np.random.default_rng(flags)
    lens = list(range(0, 60)) + [12287, 12288, 12289, 3 * 12288 + 2, 16383, 16384, 16385,
                                 3 * 16384 + 3, 200_001]
    for i, n in enumerate(lens):
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        off = (0, 0, 5, 3)[i % 4]
        enc = gb64.b64_encode_ex(dev(raw, off), flags).cpu().numpy()
        exp = oracle.encode_ex(raw, flags)
        assert np.array_equal(enc, exp), (n, flags)
        for dflags in (flags, flags | STRICT):
            st, outlen, fb, d = gb64.b64_decode_ex(dev(exp, off), dflags)
            ost, oout, ofb = oracle.decode_ex(exp, dflags)
            assert (st, fb, outlen) == (ost, ofb, oout.size), (n, dflags)
            assert np.array_equal(d[:outlen].cpu().numpy(), oout)


def _batch_check(gb64, oracle, msgs, flags):
    """Decode a list of byte strings as one batch with flags; compare every
    message's status, first_bad and bytes with the oracle."""
    import torch

    lens = np.array([len(m) for m in msgs], dtype=np.int64)
    off = W.offsets_from_lengths(lens)
    chars = np.frombuffer(b"".join(msgs), dtype=np.uint8) if off[-1] else np.zeros(0, np.uint8)
    dst, out_off, st, fb, ol = gb64.b64_decode_batch_ex(dev(chars), torch.from_numpy(off).cuda(),
                                                        flags)
    st, fb, ol, oo = st.cpu().numpy(), fb.cpu().numpy(), ol.cpu().numpy(), out_off.cpu().numpy()
    h = dst.cpu().numpy()
    for j, m in enumerate(msgs):
        ost, oout, ofb = oracle.decode_ex(m, flags)
        assert (st[j], fb[j]) == (ost, ofb), (m, flags, st[j], fb[j], ost, ofb)
        if ost == 0:
            assert ol[j] == oout.size and np.array_equal(h[oo[j]:oo[j] + ol[j]], oout), (m, flags)


@pytest.mark.parametrize("flags", ALL_FLAGS)
def test_every_byte_at_every_position_batched(gb64, oracle, flags):
    bases = [b"QUJDREVGR0lG", b"R0lGQUI=", b"R0lGQQ==", b"_-_-R0lG", b"+/+/R0lG", b"R0lGQUI",
             b"R0lGQQ", b"R0lGQ"]
    msgs = []
    for base in bases:
        for q in range(len(base)):
            for x in range(256):
                s = bytearray(base)
                s[q] = x
                msgs.append(bytes(s))
    _batch_check(gb64, oracle, msgs, flags)


@pytest.mark.parametrize("flags", [STRICT, STRICT | NOPAD, STRICT | URL, STRICT | URL | NOPAD])
def test_strict_tail_all_final_groups(gb64, oracle, flags):
    """Every final group of two characters + "==" and of three + "=" (strided
    over the alphabet), decoded in one batch and one by one."""
    enc = lambda b: oracle.encode_ex(np.frombuffer(b, dtype=np.uint8), flags & (URL | NOPAD)).tobytes()
    alpha = enc(int("".join(f"{v:06b}" for v in range(64)), 2).to_bytes(48, "big"))
    pad = (lambda s: s) if flags & NOPAD else (lambda s: s + b"=" * (4 - len(s)))
    msgs = [b"R0lG" + pad(bytes([a, b])) for a, b in itertools.product(alpha[::7], alpha)]
    msgs += [pad(bytes([a, b, c])) for a, b, c in itertools.product(alpha[::9], alpha[::5], alpha)]
    _batch_check(gb64, oracle, msgs, flags)
    for m in msgs[::97]:
        st, outlen, fb, d = gb64.b64_decode_ex(dev(np.frombuffer(m, dtype=np.uint8)), flags)
        ost, oout, ofb = oracle.decode_ex(m, flags)
        assert (st, fb) == (ost, ofb), m


@pytest.mark.parametrize("flags", [URL, NOPAD, URL | NOPAD])
def test_encode_batch_variants(gb64, oracle, flags):
    import torch

    data, off = W.batched(nmsg=2000, seed=60 + flags, median=400.0)
    dst, out_off = gb64.b64_encode_batch_ex(dev(data), torch.from_numpy(off).cuda(), flags)
    oo, h = out_off.cpu().numpy(), dst.cpu().numpy()
    for j in range(off.size - 1):
        exp = oracle.encode_ex(data[off[j]:off[j + 1]], flags)
        assert oo[j + 1] - oo[j] == exp.size
        assert np.array_equal(h[oo[j]:oo[j + 1]], exp), j
    msgs = [h[oo[j]:oo[j + 1]].tobytes() for j in range(off.size - 1)]
    _batch_check(gb64, oracle, msgs[:600], flags | STRICT)


def test_large_buffer_url_nopad(gb64, oracle):
    """300 MiB through the big-tile shapes with base64url and no padding."""
    import torch

    flags = URL | NOPAD
    n = (300 << 20) + 1
    src = W.counter_bytes_torch(61, 0, n, device="cuda")
    enc = gb64.b64_encode_ex(src, flags)
    assert enc.numel() == gb64.b64_encoded_len_ex(n, flags)
    rng = np.random.default_rng(1)
    for _ in range(50):
        w = int(rng.integers(0, n // 3 - 2000))
        L = 3 * int(rng.integers(1, 1000))
        exp = oracle.encode_ex(src[3 * w:3 * w + L].cpu().numpy(), flags)
        assert np.array_equal(enc[4 * w:4 * w + exp.size].cpu().numpy(), exp)
    k = (n // 3 - 100) * 3  # the last groups, including the partial one
    exp_tail = oracle.encode_ex(src[k:].cpu().numpy(), flags)
    assert np.array_equal(enc[-exp_tail.size:].cpu().numpy(), exp_tail)
    st, outlen, fb, dec = gb64.b64_decode_ex(enc, flags | STRICT)
    assert (st, outlen, fb) == (0, n, enc.numel())
    assert torch.equal(dec[:n], src)
