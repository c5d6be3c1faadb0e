"""GPU parity of whitespace removal before decoding (Appendix B): status,
first_bad (an index into the original input) and bytes equal the oracle's,
for sprinkled whitespace, line-wrapped input, injected errors, the other
flags, every alignment class, and inputs spanning many tiles."""
import base64

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SKIP_WS, URL, NOPAD, STRICT = 8, 1, 2, 4
WS = b" \n\r"


def dev(a, off=0):
    import torch

    a = np.ascontiguousarray(np.frombuffer(bytes(a), dtype=np.uint8) if isinstance(a, bytes) else a,
                             dtype=np.uint8)
    buf = torch.empty(off + a.size + 1, dtype=torch.uint8, device="cuda")
    t = buf[off:off + a.size]
    if a.size:
        t.copy_(torch.from_numpy(a.copy()))
    return t


def sprinkle(rng, s: bytes, rate):
    out = bytearray()
    for ch in s:
        while rng.random() < rate:
            out.append(WS[int(rng.integers(0, 3))])
        out.append(ch)
    return bytes(out)


def check(gb64, oracle, s: bytes, flags, off=0):
    st, outlen, fb, d = gb64.b64_decode_ex(dev(s, off), flags)
    ost, oout, ofb = oracle.decode_ex(s, flags)
    assert (st, fb) == (ost, ofb), (len(s), flags, st, fb, ost, ofb)
    if ost == 0:
        assert outlen == oout.size and np.array_equal(d[:outlen].cpu().numpy(), oout)
    return st


@pytest.mark.parametrize("rate", [0.0, 0.03, 0.3])
def test_sprinkled_whitespace(gb64, oracle, rate):
    rng = np.random.default_rng(int(rate * 100))
    for i, n in enumerate(list(range(0, 40)) + [3071, 3072, 3073, 6000, 12289, 100_000]):
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        s = sprinkle(rng, base64.b64encode(raw), rate)
        assert check(gb64, oracle, s, SKIP_WS, off=i % 5) == 0


def test_line_wrapped_input(gb64, oracle):
    """MIME-style: 76 characters per line, CRLF line ends."""
    rng = np.random.default_rng(4)
    for n in (57, 1000, 57 * 1000 + 5, 3 << 20):
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        e = base64.b64encode(raw)
        s = b"\r\n".join(e[i:i + 76] for i in range(0, len(e), 76)) + b"\r\n"
        assert check(gb64, oracle, s, SKIP_WS) == 0


def test_errors_in_original_offsets(gb64, oracle):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    bad_set = [b for b in NON_ALPHABET_NON_PAD.tolist() if b not in WS]
    rng = np.random.default_rng(5)
    for trial in range(150):
        n = int(rng.integers(1, 50_000))
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        s = bytearray(sprinkle(rng, base64.b64encode(raw), 0.05))
        for _ in range(int(rng.integers(1, 3))):
            q = int(rng.integers(0, len(s)))
            s[q] = bad_set[int(rng.integers(0, len(bad_set)))]
        if trial % 4 == 0:
            s += b"QQ"  # an incomplete final group
        check(gb64, oracle, bytes(s), SKIP_WS, off=trial % 3)


@pytest.mark.parametrize("flags", [SKIP_WS | URL, SKIP_WS | NOPAD, SKIP_WS | STRICT,
                                   SKIP_WS | URL | NOPAD | STRICT])
def test_with_the_other_flags(gb64, oracle, flags):
    rng = np.random.default_rng(flags)
    for n in list(range(0, 30)) + [4097, 20_000]:
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        e = oracle.encode_ex(np.frombuffer(raw, dtype=np.uint8), flags & (URL | NOPAD)).tobytes()
        s = sprinkle(rng, e, 0.05)
        assert check(gb64, oracle, s, flags) == 0
        if len(e) >= 2:  # a noncanonical tail under STRICT, or just another error
            t = bytearray(s)
            t[-1 if t[-1] not in WS else -2] ^= 1
            check(gb64, oracle, bytes(t), flags)


def test_degenerate(gb64, oracle):
    for s in [b"", b" ", b"\r\n\r\n", b" " * 5000, b"QQ==\n", b"\nQQ==", b"Q Q = =", b"QQ=\n=",
              b"=\n===", b"A\nB\nC", b"AB CD\r\n", b"A" * 4096 + b" " * 4096 + b"AAAA"]:
        check(gb64, oracle, s, SKIP_WS)


def test_whitespace_runs_across_tiles(gb64, oracle):
    """The decode reads the kept characters just after its tile (the rest of
    a unit, or the final quads) from the following tiles: runs of
    whitespace longer than a tile (16,384 characters), tiles that keep a
    single character, errors and final groups among those characters."""
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    tile = 16384
    rng = np.random.default_rng(21)
    e = base64.b64encode(rng.integers(0, 256, 3001, dtype=np.uint8).tobytes())
    bad = bytes([[b for b in NON_ALPHABET_NON_PAD.tolist() if b not in WS][7]])
    cases = []
    for cut in (1, 3, 15, 16, 17, 1001, len(e) - 3, len(e) - 1):
        for gap in (tile - 1, 3 * tile + 5):
            cases.append(e[:cut] + b" " * gap + e[cut:])
    sparse = b"".join(e[i:i + 1] + b"\n" * (tile - 1) for i in range(40)) + e[40:]
    cases += [sparse, b" " * (2 * tile - 7) + e[:9] + b" " * tile + e[9:],
              b"".join(e[i:i + 1] + b" " * (tile - 1) for i in range(len(e) - 6, len(e)))]
    for k, s in enumerate(cases):
        check(gb64, oracle, s, SKIP_WS, off=k % 3)
        t = bytearray(s)
        kept = [i for i, c in enumerate(t) if c not in WS]
        t[kept[min(len(kept) - 1, 17 + k)]] = bad[0]  # an error among the halo's characters
        check(gb64, oracle, bytes(t), SKIP_WS)


def test_rejected_where_not_supported(gb64):
    import torch

    src = dev(b"QUJD")
    with pytest.raises(gb64.Gb64Error):
        gb64.b64_encode_ex(src, SKIP_WS)
    off = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    with pytest.raises(gb64.Gb64Error):
        gb64.b64_decode_batch_ex(src, off, SKIP_WS)


def test_large_with_whitespace(gb64, oracle):
    """~64 MB of line-wrapped text (many tiles), checked against the oracle
    on sampled windows and by the round trip."""
    import torch

    from paper_1704_00605_gb300 import workloads as W

    raw = W.counter_bytes(9, 0, 48 << 20)
    e = base64.b64encode(raw.tobytes())
    s = b"\n".join(e[i:i + 64] for i in range(0, len(e), 64))
    st, outlen, fb, d = gb64.b64_decode_ex(dev(s), SKIP_WS)
    assert (st, outlen, fb) == (0, raw.size, len(s))
    assert torch.equal(d[:outlen].cpu(), torch.from_numpy(raw))
    t = bytearray(s)
    t[len(s) // 2 + 7] = ord("!") if t[len(s) // 2 + 7] != 0x0A else t[len(s) // 2 + 7]
    t[len(s) - 1000] = ord("*")
    st, outlen, fb, d = gb64.b64_decode_ex(dev(bytes(t)), SKIP_WS)
    ost, _, ofb = oracle.decode_ex(bytes(t), SKIP_WS)
    assert (st, fb) == (ost, ofb)
