"""GPU parity of the one-pass line-model path of the whitespace-removing
decode (Appendix B). Line-wrapped input of the common shapes (MIME 76 + CR
LF, PEM 64 + LF, other line lengths and separators, trailing whitespace)
decodes exactly as the oracle does, through the line-model kernel; input
that breaks the model anywhere (a short or long line, a missing or extra
separator, whitespace inside a line, leading whitespace, long trailing runs)
gives the same exact result through the general path. Errors, padding, the
length rule and the other flags are checked on wrapped input, at every
source alignment and across many tiles."""
import base64

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SKIP_WS, URL, NOPAD, STRICT = 8, 1, 2, 4
LINE_MARK = 0x4C494E45  # b64_result.internal after the line-model kernel finished a decode


def dev(a, off=0, dst_off=0):
    import torch

    a = np.frombuffer(bytes(a), dtype=np.uint8)
    buf = torch.empty(off + a.size + 1, dtype=torch.uint8, device="cuda")
    t = buf[off:off + a.size]
    if a.size:
        t.copy_(torch.from_numpy(a.copy()))
    return t


def wrap(e: bytes, L: int, sep: bytes, trail: bytes = b"") -> bytes:
    return sep.join(e[i:i + L] for i in range(0, len(e), L)) + trail


def run(gb64, s: bytes, flags=SKIP_WS, off=0, dst_off=0):
    """(status, outlen, first_bad, decoded bytes, line path taken)."""
    import torch

    src = dev(s, off)
    cap = gb64.b64_decoded_cap_ex(len(s), flags)
    dbuf = torch.zeros(cap + dst_off + 16, dtype=torch.uint8, device="cuda")
    dst = dbuf[dst_off:dst_off + max(cap, 1)]
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    gb64.b64_decode_async_ex(src, dst, res, flags)
    torch.cuda.synchronize()
    st, outlen, fb = gb64.parse_result(res)
    internal = int(res.view(torch.int32)[5].item()) & 0xFFFFFFFF
    return st, outlen, fb, dst[:max(outlen, 0)].cpu().numpy(), internal == LINE_MARK


def check(gb64, oracle, s: bytes, flags=SKIP_WS, off=0, dst_off=0, line=None):
    st, outlen, fb, d, took = run(gb64, s, flags, off, dst_off)
    ost, oout, ofb = oracle.decode_ex(s, flags)
    assert (st, fb) == (ost, ofb), (len(s), flags, st, fb, ost, ofb, took)
    if ost == 0:
        assert outlen == oout.size and np.array_equal(d, oout)
    if line is not None:
        assert took == line, (len(s), took)
    return st


SHAPES = [(76, b"\r\n"), (64, b"\n"), (76, b"\n"), (60, b"\r\n"), (16, b"\n"), (17, b"\r\n"),
          (57, b" "), (100, b"\r"), (1000, b"\r\n"), (4095, b"\n")]


@pytest.mark.parametrize("L,sep", SHAPES)
def test_line_shapes(gb64, oracle, L, sep):
    rng = np.random.default_rng(L * 7 + len(sep))
    for i, n in enumerate([1, 2, 3, 12, 45, 57 * 10 + 1, 12_289, 100_000, 1_000_003]):
        e = base64.b64encode(rng.integers(0, 256, n, dtype=np.uint8).tobytes())
        for trail in (b"", sep, b"\r\n", b" \n\t"[:2], b" " * 15):
            s = wrap(e, L, sep, trail)
            # one line only (no break before the end) is the no-breaks model
            check(gb64, oracle, s, off=(i + len(trail)) % 16, line=True)


def test_no_line_breaks(gb64, oracle):
    rng = np.random.default_rng(3)
    e = base64.b64encode(rng.integers(0, 256, 300_001, dtype=np.uint8).tobytes())
    for trail in (b"", b"\n", b"\r\n", b" " * 15):
        check(gb64, oracle, e + trail, line=True)
    # a trailing run of 16 or more may be longer than the model looks: general path
    for trail in (b" " * 16, b"\n" * 40):
        check(gb64, oracle, e + trail, line=False)
    # whitespace past the probed prefix: the model breaks
    t = e[:200_000] + b"\n" + e[200_000:]
    check(gb64, oracle, t, line=False)
    # all whitespace, short and long
    for s in (b" ", b"\r\n", b"\n" * 15, b" " * 16, b" " * 5000):
        check(gb64, oracle, s)


def test_model_breaks_fall_back(gb64, oracle):
    rng = np.random.default_rng(5)
    e = base64.b64encode(rng.integers(0, 256, 57 * 400, dtype=np.uint8).tobytes())
    s = wrap(e, 76, b"\r\n", b"\r\n")
    lines = s.split(b"\r\n")
    mid = len(lines) // 2
    cases = {
        "short line": b"\r\n".join(lines[:mid] + [lines[mid][:-4] + b"\r\n" + lines[mid][-4:]] +
                                   lines[mid + 1:]),
        "joined lines": b"\r\n".join(lines[:mid] + [lines[mid] + lines[mid + 1]] + lines[mid + 2:]),
        "extra break": s[:5000] + b"\n" + s[5000:],
        "space in a line": s[:7001] + b" " + s[7001:],
        "first line short": s[20:],
        "leading whitespace": b"\n" + s,
        "three-byte break": s.replace(b"\r\n", b"\r\n\n", 1),
        "break shorter later": s[:9000] + s[9000:].replace(b"\r\n", b"\n", 1),
        "last line too long": s[:-2] + b"QUJD\r\n",
    }
    for name, c in cases.items():
        # (the oracle decides the status; the kernel must not take the line path)
        st, outlen, fb, d, took = run(gb64, c)
        ost, oout, ofb = oracle.decode_ex(c, SKIP_WS)
        assert (st, fb) == (ost, ofb), name
        if ost == 0:
            assert np.array_equal(d, oout), name
        assert not took, name
    # other whitespace bytes of the same length at a separator still fit the model
    t = s[:3000] + s[3000:].replace(b"\r\n", b" \n", 1)
    check(gb64, oracle, t, line=True)
    t = s[:3000] + s[3000:].replace(b"\r\n", b"\n\r", 3)
    check(gb64, oracle, t, line=True)


def test_errors_on_wrapped_input(gb64, oracle):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    ws = b" \n\r"
    bad_set = [b for b in NON_ALPHABET_NON_PAD.tolist() if b not in ws]
    rng = np.random.default_rng(6)
    for trial in range(120):
        n = int(rng.integers(1, 60_000))
        L, sep = SHAPES[trial % len(SHAPES)]
        e = base64.b64encode(rng.integers(0, 256, n, dtype=np.uint8).tobytes())
        s = bytearray(wrap(e, L, sep, sep if trial % 2 else b""))
        kept = [i for i, c in enumerate(s) if c not in ws]
        for _ in range(int(rng.integers(1, 4))):
            q = kept[int(rng.integers(0, len(kept)))]
            s[q] = bad_set[int(rng.integers(0, len(bad_set)))] if trial % 5 else ord("=")
        check(gb64, oracle, bytes(s), off=trial % 16, line=True)
    # a bad byte in place of a separator byte breaks the model
    s = bytearray(wrap(base64.b64encode(bytes(range(256)) * 40), 64, b"\n"))
    s[64 * 5 + 5 - 1] = ord("!")
    check(gb64, oracle, bytes(s), line=False)


@pytest.mark.parametrize("flags", [SKIP_WS | URL, SKIP_WS | NOPAD, SKIP_WS | STRICT,
                                   SKIP_WS | URL | NOPAD | STRICT])
def test_flags_and_final_groups(gb64, oracle, flags):
    rng = np.random.default_rng(flags + 40)
    for n in list(range(1, 80)) + [4097, 20_000, 20_001, 20_002]:
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        e = oracle.encode_ex(raw, flags & (URL | NOPAD)).tobytes()
        for L, sep in ((16, b"\n"), (76, b"\r\n")):
            s = wrap(e, L, sep, b"\n" if n % 2 else b"")
            check(gb64, oracle, s, flags, line=True)
            if len(e) >= 2:  # a noncanonical final group under STRICT
                t = bytearray(s)
                k = max(i for i, c in enumerate(t) if c not in b"\r\n=")
                t[k] ^= 1
                check(gb64, oracle, bytes(t), flags)
            # the length rule: a dropped last character
            t = s.rstrip(b"\r\n")[:-1]
            if t:
                check(gb64, oracle, t, flags)


def test_alignments(gb64, oracle):
    rng = np.random.default_rng(8)
    e = base64.b64encode(rng.integers(0, 256, 50_000, dtype=np.uint8).tobytes())
    s = wrap(e, 76, b"\r\n", b"\r\n")
    for off in range(16):
        check(gb64, oracle, s, off=off, line=True)
    for dst_off in (1, 2, 3, 8):  # an unaligned output goes to the general path
        check(gb64, oracle, s, dst_off=dst_off, line=False)


def test_large_mime(gb64, oracle):
    """~72 MB of MIME lines (the 512-thread shape, hundreds of tiles): exact
    round trip through the line path; then errors near the start and the
    end; then a model break near the end (general path)."""
    import torch

    from paper_1704_00605_gb300 import workloads as W

    raw = W.counter_bytes(11, 0, 52 << 20)
    e = base64.b64encode(raw.tobytes())
    s = wrap(e, 76, b"\r\n", b"\r\n")
    st, outlen, fb, d, took = run(gb64, s)
    assert (st, outlen, fb, took) == (0, raw.size, len(s), True)
    assert np.array_equal(d, raw)
    t = bytearray(s)
    t[len(s) - 1003] = ord("*") if t[len(s) - 1003] not in b"\r\n" else t[len(s) - 1003]
    t[123_457] = ord("#") if t[123_457] not in b"\r\n" else t[123_457]
    st, outlen, fb, d, took = run(gb64, bytes(t))
    ost, _, ofb = oracle.decode_ex(bytes(t), SKIP_WS)
    assert (st, fb, took) == (ost, ofb, True)
    t = s[:len(s) - 5000] + b"\n" + s[len(s) - 5000:]
    st, outlen, fb, d, took = run(gb64, t)
    assert (st, outlen, took) == (0, raw.size, False)
    assert torch.equal(torch.from_numpy(d), torch.from_numpy(raw))


@pytest.mark.parametrize("shape", [(256, 4, 3), (256, 1, 6), (512, 1, 4), (512, 2, 4),
                                   (512, 4, 3), (512, 7, 2)])
def test_line_kernel_shapes(gb64, oracle, shape):
    """Every tile shape the shape table accepts for the line-model kernel
    (threads, 16-character units per thread, stages) decodes exactly: MIME
    and PEM lines, unaligned input, errors."""
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    threads, upt, stages = shape
    kind = gb64.B64_KIND_DECODE_WS
    rng = np.random.default_rng(sum(shape))
    cases = []
    for n, L, sep in ((300_001, 76, b"\r\n"), (200_000, 64, b"\n"), (150_000, 57, b"\n")):
        e = base64.b64encode(rng.integers(0, 256, n, dtype=np.uint8).tobytes())
        cases.append(wrap(e, L, sep, sep))
    t = bytearray(cases[0])
    for q in rng.integers(0, len(t), 3):
        if t[q] not in b"\r\n":
            t[q] = int(NON_ALPHABET_NON_PAD[int(rng.integers(0, 191))])
    cases.append(bytes(t))
    saved = [gb64.b64_shape_get(kind, len(c), 1) for c in cases]
    try:
        for k, c in enumerate(cases):
            gb64.b64_shape_set(kind, len(c), 1, threads=threads, units_per_thread=upt,
                               stages=stages, blocks_per_sm=0, tile=threads * upt * 16)
            check(gb64, oracle, c, off=k * 5 % 16, line=True)
    finally:
        for c, sh in zip(cases, saved):
            gb64.b64_shape_set(kind, len(c), 1, **{f: sh[f] for f in (
                "threads", "units_per_thread", "stages", "blocks_per_sm", "tile")})


def test_line_kernel_shape_validation(gb64):
    kind = gb64.B64_KIND_DECODE_WS
    for bad in ((128, 4, 3), (1024, 2, 3), (512, 9, 2), (512, 4, 1), (512, 4, 7),
                (512, 8, 2)):  # the last needs more shared memory than a CTA has
        with pytest.raises(gb64.Gb64Error):
            gb64.b64_shape_set(kind, 1 << 20, 1, threads=bad[0], units_per_thread=bad[1],
                               stages=bad[2], blocks_per_sm=0, tile=bad[0] * bad[1] * 16)


@pytest.mark.parametrize("threads", [256, 512])
def test_general_path_in_each_block_size(gb64, oracle, threads):
    """The general path runs in the line kernel's own launch, so with its
    block size: sprinkled whitespace (no line model), a model broken late in
    a long input, and an output the bulk stores cannot take (general path
    alone) decode exactly with both block sizes."""
    kind = gb64.B64_KIND_DECODE_WS
    rng = np.random.default_rng(threads)
    e = base64.b64encode(rng.integers(0, 256, 400_000, dtype=np.uint8).tobytes())
    sprinkled = bytearray()
    for i in range(0, len(e), 40):
        sprinkled += e[i:i + 40] + b" \r\n"[int(rng.integers(0, 3)):][:int(rng.integers(0, 3))]
    mime = wrap(e, 76, b"\r\n", b"\r\n")
    late = mime[:len(mime) - 777] + b" " + mime[len(mime) - 777:]
    cases = [bytes(sprinkled), late, mime]
    saved = [gb64.b64_shape_get(kind, len(c), 1) for c in cases]
    try:
        for c in cases:
            gb64.b64_shape_set(kind, len(c), 1, threads=threads, units_per_thread=2, stages=3,
                               blocks_per_sm=0, tile=threads * 2 * 16)
        check(gb64, oracle, cases[0], line=False)
        check(gb64, oracle, cases[1], off=3, line=False)
        check(gb64, oracle, cases[2], dst_off=5, line=False)
        check(gb64, oracle, cases[2], line=True)
    finally:
        for c, sh in zip(cases, saved):
            gb64.b64_shape_set(kind, len(c), 1, **{f: sh[f] for f in (
                "threads", "units_per_thread", "stages", "blocks_per_sm", "tile")})
