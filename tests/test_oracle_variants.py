"""Pins of the oracle's variants (Section 2: base64url and omitted padding;
Appendix A: the extra check of the final group) against independent
sources: Python's urlsafe codec and strict decoder, Python's own encodings
with their padding stripped, and brute force over every 1- and 2-byte input
for the set of canonical final groups."""
import base64
import binascii
import itertools

import numpy as np
import pytest

URL, NOPAD, STRICT = 1, 2, 4


def _py_strict(s: bytes, url: bool):
    """Python's strict decoder on s; in url mode '+' and '/' are outside the
    alphabet, so they are mapped to '!' before translating '-' and '_'."""
    if url:
        s = s.replace(b"+", b"!").replace(b"/", b"!").replace(b"-", b"+").replace(b"_", b"/")
    try:
        return binascii.a2b_base64(s, strict_mode=True)
    except binascii.Error:
        return None


def test_flags_zero_equal_the_base_functions(oracle):
    rng = np.random.default_rng(0)
    for n in list(range(0, 40)) + [1000, 1001, 1002]:
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        assert np.array_equal(oracle.encode_ex(raw, 0), oracle.encode(raw))
    for base in (b"QUJDREVG", b"R0lGQUI=", b"R0lGQQ==", b"QUJ", b"Q"):
        for q in range(len(base)):
            for x in range(256):
                s = bytearray(base)
                s[q] = x
                a, b = oracle.decode_ex(bytes(s), 0), oracle.decode(bytes(s))
                assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])


def test_url_encode_all_three_byte_groups(oracle):
    g = np.arange(1 << 24, dtype=np.uint32)
    raw = np.empty((1 << 24, 3), dtype=np.uint8)
    raw[:, 0], raw[:, 1], raw[:, 2] = g >> 16, (g >> 8) & 0xFF, g & 0xFF
    raw = raw.reshape(-1)
    assert oracle.encode_ex(raw, URL).tobytes() == base64.urlsafe_b64encode(raw.tobytes())


@pytest.mark.parametrize("flags", [URL, NOPAD, URL | NOPAD])
def test_encode_variants_lengths(oracle, flags):
    rng = np.random.default_rng(flags)
    for n in list(range(0, 80)) + [4095, 4096, 4097]:
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        py = base64.urlsafe_b64encode(raw) if flags & URL else base64.b64encode(raw)
        if flags & NOPAD:
            py = py.rstrip(b"=")
        assert oracle.encode_ex(raw, flags).tobytes() == py


def test_url_decode_all_valid_quads(oracle):
    alpha = np.frombuffer(base64.urlsafe_b64encode(
        int("".join(f"{v:06b}" for v in range(64)), 2).to_bytes(48, "big")), dtype=np.uint8)
    q = np.arange(64 ** 4, dtype=np.uint32)
    chars = np.empty((64 ** 4, 4), dtype=np.uint8)
    chars[:, 0], chars[:, 1] = alpha[q >> 18], alpha[(q >> 12) & 63]
    chars[:, 2], chars[:, 3] = alpha[(q >> 6) & 63], alpha[q & 63]
    chars = chars.reshape(-1)
    st, out, fb = oracle.decode_ex(chars, URL)
    assert st == 0 and fb == chars.size
    assert out.tobytes() == base64.urlsafe_b64decode(chars.tobytes())


@pytest.mark.parametrize("flags", [URL, URL | NOPAD, NOPAD])
def test_decode_variants_every_byte_at_every_position(oracle, flags):
    """Accept/reject and output equal Python's strict decoder (padding
    re-added for unpadded inputs); rejections point at the written byte."""
    url = bool(flags & URL)
    bases = [b"QUJDREVGR0lG", b"R0lGQUI=", b"R0lGQQ=="] if not url else \
        [b"QUJDREVGR0lG", b"R0lGQUI=", b"R0lGQQ==", b"_-_-R0lG"]
    if flags & NOPAD:
        bases += [b"R0lGQUI", b"R0lGQQ"]
    for base in bases:
        for q in range(len(base)):
            for x in range(256):
                s = bytearray(base)
                s[q] = x
                s = bytes(s)
                st, out, fb = oracle.decode_ex(s, flags)
                padded = s + b"=" * ((-len(s)) % 4) if (flags & NOPAD) and len(s) % 4 in (2, 3) else s
                if (flags & NOPAD) and len(s) % 4 in (2, 3) and b"=" in s:
                    py = None  # '=' is not allowed inside an unpadded final group
                else:
                    py = _py_strict(padded, url)
                if py is not None:
                    assert st == 0 and out.tobytes() == py and fb == len(s), (s, st)
                    continue
                assert st == 1, (s, st, fb)
                exp = q
                if base.endswith(b"==") and q == len(s) - 1 and x != 0x3D:
                    exp = len(s) - 2
                assert fb == exp, (s, fb, exp)


def test_nopad_round_trip_and_length_rule(oracle):
    rng = np.random.default_rng(3)
    for n in range(0, 300):
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        s = base64.b64encode(raw).rstrip(b"=")
        st, out, fb = oracle.decode_ex(s, NOPAD)
        assert (st, fb) == (0, len(s)) and out.tobytes() == raw
        st, out, fb = oracle.decode_ex(base64.b64encode(raw), NOPAD)  # padded still accepted
        assert st == 0 and out.tobytes() == raw
        if len(s) % 4 == 0 and len(s):
            t = s + b"Q"  # one character past whole groups: BAD_LENGTH there
            st, out, fb = oracle.decode_ex(t, NOPAD)
            assert (st, fb) == (2, len(t) - 1) and _py_strict(t + b"===", False) is None


@pytest.mark.parametrize("flags", [STRICT, STRICT | NOPAD, STRICT | URL])
def test_strict_tail_accepts_exactly_the_canonical_groups(oracle, flags):
    """Appendix A: the final groups accepted are exactly those Python's
    encoder produces for some 1- or 2-byte input; any other group of valid
    characters is NONCANONICAL at its last data character."""
    enc = base64.urlsafe_b64encode if flags & URL else base64.b64encode
    strip = (lambda b: b.rstrip(b"=")) if flags & NOPAD else (lambda b: b)
    alpha = enc(int("".join(f"{v:06b}" for v in range(64)), 2).to_bytes(48, "big"))
    canon1 = {strip(enc(bytes([a]))) for a in range(256)}
    canon2 = {strip(enc(bytes([a, b]))) for a in range(256) for b in range(256)}
    for c0, c1 in itertools.product(alpha[::3], alpha):
        s = strip(bytes([c0, c1]) + b"==")
        st, out, fb = oracle.decode_ex(b"R0lG" + s, flags)
        if s in canon1:
            assert st == 0 and len(out) == 4
        else:
            assert (st, fb) == (3, 4 + 1), s
    for c0, c1, c2 in itertools.product(alpha[::5], alpha[::3], alpha):
        s = strip(bytes([c0, c1, c2]) + b"=")
        st, out, fb = oracle.decode_ex(s, flags)
        if s in canon2:
            assert st == 0 and len(out) == 2
        else:
            assert (st, fb) == (3, 2), s


def test_strict_tail_precedence(oracle):
    # invalid characters and the length rule come before Appendix A's check
    assert oracle.decode_ex(b"!WJ=", STRICT)[0::2] == (1, 0)
    assert oracle.decode_ex(b"YWJ", STRICT)[0::2] == (2, 0)
    assert oracle.decode_ex(b"YWJ", STRICT | NOPAD)[0::2] == (3, 2)
    assert oracle.decode_ex(b"YWI", STRICT | NOPAD)[0] == 0


# ------------------------------------------------------- whitespace (App. B)
SKIP_WS = 8
WS = b" \n\r"


def _sprinkle(rng, s: bytes, rate=0.03):
    """Insert space/LF/CR before characters with probability `rate`
    (Appendix B's test input has about 3 % whitespace); returns the string
    and, for every character of s, its index in the result."""
    out, where = bytearray(), []
    for ch in s:
        while rng.random() < rate:
            out.append(WS[int(rng.integers(0, 3))])
        where.append(len(out))
        out.append(ch)
    if rng.random() < 0.5:
        out.extend(b"\r\n")
    return bytes(out), where


def test_skip_ws_matches_python_nonstrict(oracle):
    rng = np.random.default_rng(21)
    for n in list(range(0, 120)) + [999, 4096]:
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        s, _ = _sprinkle(rng, base64.b64encode(raw))
        st, out, fb = oracle.decode_ex(s, SKIP_WS)
        assert (st, fb) == (0, len(s)) and out.tobytes() == raw
        assert binascii.a2b_base64(s) == raw  # Python drops the whitespace too
        assert _py_strict(bytes(c for c in s if c not in WS), False) == raw


def test_skip_ws_first_bad_in_original_offsets(oracle):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    bad_set = [b for b in NON_ALPHABET_NON_PAD.tolist() if b not in WS]
    rng = np.random.default_rng(22)
    for trial in range(400):
        raw = rng.integers(0, 256, int(rng.integers(1, 300)), dtype=np.uint8).tobytes()
        enc = bytearray(base64.b64encode(raw))
        q = int(rng.integers(0, len(enc) - 2))  # not the padding positions
        enc[q] = bad_set[int(rng.integers(0, len(bad_set)))]
        s, where = _sprinkle(rng, bytes(enc))
        st, out, fb = oracle.decode_ex(s, SKIP_WS)
        assert (st, fb) == (1, where[q]), (s, fb, where[q])


def test_skip_ws_length_rule_and_equivalence(oracle):
    rng = np.random.default_rng(23)
    s, where = _sprinkle(rng, b"QUJDREVGQ", rate=0.3)
    st, out, fb = oracle.decode_ex(s, SKIP_WS)
    assert (st, fb) == (2, where[8])  # start of the incomplete group, original index
    assert oracle.decode_ex(b" \n\r", SKIP_WS)[0::2] == (0, 3)  # nothing left: empty input
    for base in (b"R0lGQUI=", b"R0lGQQ==", b"QUJDREVG"):
        for q in range(len(base)):
            for x in range(256):
                t = bytearray(base)
                t[q] = x
                t = bytes(t)
                if x in WS:
                    continue
                a, b = oracle.decode_ex(t, SKIP_WS), oracle.decode_ex(t, 0)
                assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])
    # combined with the other flags: url alphabet, no padding, strict tail
    raw = bytes(range(200))
    s, _ = _sprinkle(rng, base64.urlsafe_b64encode(raw).rstrip(b"="))
    st, out, fb = oracle.decode_ex(s, SKIP_WS | URL | NOPAD | STRICT)
    assert st == 0 and out.tobytes() == raw
