"""Pins of the CPU oracle against things other than itself.

Each test fixes a part of the oracle by an independent source: Python's
base64/binascii (an RFC 4648 implementation), the paper's worked examples
and printed constants (tests/golden/paper_examples.txt), closed forms, and
errors whose position is known by construction.
"""
import base64
import binascii

import numpy as np
import pytest

from tests import golden

ALL = np.arange(256, dtype=np.int64)


def python_alphabet() -> bytes:
    """The 64 characters in value order, obtained from Python's encoder: pack
    the values 0..63 as consecutive 6-bit fields and encode the 48 bytes."""
    bits = 0
    for v in range(64):
        bits = (bits << 6) | v
    raw = bits.to_bytes(48, "big")
    return base64.b64encode(raw)


# ------------------------------------------------------------ Table 1 pins
def test_table1_matches_python_alphabet(oracle):
    alpha = python_alphabet()
    assert bytes(oracle.table1_char(v) for v in range(64)) == alpha
    for x in range(256):
        expect = alpha.index(bytes([x])) if bytes([x]) in alpha and x != 0x3D else -1
        assert oracle.table1_value(x) == expect


def test_table1_spot_entries_from_paper(oracle):
    for v, code in golden.rows("table1_entry"):
        assert oracle.table1_char(v) == code
        assert oracle.table1_value(code) == v


def test_table3_offsets_reproduce_table1(oracle):
    """Table 3: each 6-bit range maps to ASCII by one offset."""
    covered = set()
    for lo, hi, off in golden.rows("table3_row"):
        for v in range(lo, hi + 1):
            assert oracle.table1_char(v) == v + off
            covered.add(v)
    assert covered == set(range(64))


def test_algorithm3_bitsets_classify_all_bytes(oracle):
    """Algorithm 3 / Appendix C: a byte is outside Table 1 exactly when
    lut_lo[low nibble] AND lut_hi[high nibble] is non-zero (high nibble taken
    as floor(x / 16)); for valid bytes x + roll[h + (x == '/' ? -1 : 0)] is
    the 6-bit value."""
    lut_lo = golden.ints("lut_lo")
    lut_hi = golden.ints("lut_hi")
    roll = golden.ints("roll")
    nvalid = 0
    for x in range(256):
        h = x // 16
        invalid = (lut_lo[x % 16] & lut_hi[h]) != 0
        v = oracle.table1_value(x)
        assert invalid == (v < 0), hex(x)
        if not invalid:
            nvalid += 1
            c = -1 if x == 0x2F else 0
            assert (x + roll[h + c]) % 256 == v, hex(x)
    assert nvalid == 64


def test_appendix_c_example_intermediates(oracle):
    chars = golden.text("appc_chars").encode()
    hi = golden.ints("appc_hi_nibbles")
    roll_vals = golden.ints("appc_roll")
    values = golden.ints("appc_values")
    lut_hi = golden.ints("lut_hi")
    lut_lo = golden.ints("lut_lo")
    assert [c >> 4 for c in chars] == hi
    assert [(c + r) % 256 for c, r in zip(chars, roll_vals)] == values
    assert [oracle.table1_value(c) for c in chars] == values
    assert [lut_hi[c >> 4] for c in chars] == golden.ints("appc_lut_hi_lookup")
    assert [lut_lo[c & 15] for c in chars] == golden.ints("appc_lut_lo_lookup")
    # the 24 bytes the 32 characters decode to
    st, out, fb = oracle.decode(chars)
    assert st == oracle.OK and fb == len(chars)
    assert out.tobytes() == base64.b64decode(chars, validate=True)


# ----------------------------------------------------------- encode pins
def test_encode_worked_example(oracle):
    src = bytes(golden.ints("encode_example_bytes"))
    out = oracle.encode(src).tobytes()
    assert out == golden.text("encode_example_chars").encode()
    assert [oracle.table1_value(c) for c in out] == golden.ints("encode_example_values")


def test_encode_all_three_byte_groups(oracle):
    """Brute force: all 2^24 groups of three bytes, concatenated (groups are
    independent because every group starts at a multiple of 3)."""
    g = np.arange(1 << 24, dtype=np.uint32)
    raw = np.empty((1 << 24, 3), dtype=np.uint8)
    raw[:, 0] = g >> 16
    raw[:, 1] = (g >> 8) & 0xFF
    raw[:, 2] = g & 0xFF
    raw = raw.reshape(-1)
    out = oracle.encode(raw)
    assert out.tobytes() == base64.b64encode(raw.tobytes())


@pytest.mark.parametrize("n", list(range(0, 70)) + [1000, 1001, 1002, 4095, 4096, 4097])
def test_encode_lengths_and_padding(oracle, n):
    rng = np.random.default_rng(1234 + n)
    raw = rng.integers(0, 256, n, dtype=np.uint8)
    out = oracle.encode(raw).tobytes()
    # closed form: m = 4 * ceil(n / 3), with (3 - n mod 3) mod 3 padding chars
    assert len(out) == 4 * -(-n // 3)
    npad = (3 - n % 3) % 3
    assert out.count(b"=") == npad and (npad == 0 or out.endswith(b"=" * npad))
    assert out == base64.b64encode(raw.tobytes())


# ----------------------------------------------------------- decode pins
def test_decode_worked_example(oracle):
    chars = golden.text("decode_example_chars").encode()
    values = golden.ints("decode_example_values")
    assert [oracle.table1_value(c) for c in chars[:-1]] == values
    st, out, fb = oracle.decode(chars)
    assert st == oracle.OK and fb == len(chars)
    assert list(out) == golden.ints("decode_example_bytes")


def test_decode_all_valid_quads(oracle):
    """Brute force: all 64^4 quads of alphabet characters decode as Python
    decodes them, and re-encode to themselves."""
    alpha = np.frombuffer(python_alphabet(), dtype=np.uint8)
    q = np.arange(64 ** 4, dtype=np.uint32)
    chars = np.empty((64 ** 4, 4), dtype=np.uint8)
    chars[:, 0] = alpha[q >> 18]
    chars[:, 1] = alpha[(q >> 12) & 63]
    chars[:, 2] = alpha[(q >> 6) & 63]
    chars[:, 3] = alpha[q & 63]
    chars = chars.reshape(-1)
    st, out, fb = oracle.decode(chars)
    assert st == oracle.OK and fb == chars.size
    assert out.tobytes() == base64.b64decode(chars.tobytes(), validate=True)
    assert np.array_equal(oracle.encode(out), chars)


# Contexts for single-character injection: a quad in the middle of the
# stream, and the three kinds of final quad.
CONTEXTS = {
    "mid": b"QUJDREVG" + b"R0lG",      # inject into the first quad
    "final_nopad": b"R0lG" + b"QUJD",  # inject into the last quad
    "final_pad1": b"R0lG" + b"QUI=",
    "final_pad2": b"R0lG" + b"QQ==",
}
INJECT_QUAD = {"mid": 0, "final_nopad": 4, "final_pad1": 4, "final_pad2": 4}


def _py_strict(s: bytes):
    try:
        return binascii.a2b_base64(s, strict_mode=True)
    except binascii.Error:
        return None


@pytest.mark.parametrize("ctx", sorted(CONTEXTS))
@pytest.mark.parametrize("pos", range(4))
def test_decode_every_byte_at_every_quad_position(oracle, ctx, pos):
    """All 256 byte values at each position of a quad, in four contexts.

    Accept/reject and the output bytes must equal Python's strict decoder.
    When the result is a rejection, the first bad index is the injected
    position, by construction - with one exception that the strict padding
    reading fixes: in an "xx==" final quad, replacing the last '=' by anything
    but '=' leaves the '=' before it outside an accepted padding position, so
    that earlier '=' is the first bad character.
    """
    base = bytearray(CONTEXTS[ctx])
    q = INJECT_QUAD[ctx] + pos
    m = len(base)
    for x in range(256):
        s = bytearray(base)
        s[q] = x
        s = bytes(s)
        st, out, fb = oracle.decode(s)
        py = _py_strict(s)
        if py is not None:
            assert st == oracle.OK, (s, st)
            assert out.tobytes() == py
            assert fb == m
            continue
        assert st == oracle.INVALID_CHAR, (s, st)
        expect = q
        if ctx == "final_pad2" and q == m - 1 and x != 0x3D:
            expect = m - 2
        assert fb == expect, (s, fb, expect)


@pytest.mark.parametrize("m", range(0, 65))
def test_decode_length_rule(oracle, m):
    """Alphabet-only strings: a length that is not a multiple of 4 is
    BAD_LENGTH at the start of the incomplete group; Python rejects the same
    strings."""
    rng = np.random.default_rng(m)
    alpha = np.frombuffer(python_alphabet(), dtype=np.uint8)
    s = alpha[rng.integers(0, 64, m)].tobytes()
    st, out, fb = oracle.decode(s)
    if m % 4 == 0:
        assert st == oracle.OK and fb == m and out.tobytes() == _py_strict(s)
    else:
        assert _py_strict(s) is None
        assert st == oracle.BAD_LENGTH and fb == m - m % 4 and out.size == 0


def test_decode_padding_readings(oracle):
    """Consequences of the strict padding reading on small cases (each is
    rejected by Python's strict decoder as well)."""
    cases = {
        b"A===": 1, b"AB=A": 2, b"====": 0, b"QQ==QQ==": 2, b"R0lGQ===": 5,
        b"R0lGQQ=x": 6, b"R0lG=QQ=": 4, b"QQ=": 2, b"QQ==\n": 2,
    }
    for s, fb_expect in cases.items():
        st, out, fb = oracle.decode(s)
        assert _py_strict(s) is None
        assert st == oracle.INVALID_CHAR and fb == fb_expect, (s, st, fb)


def test_decode_first_bad_brute_force(oracle):
    """Tiny inputs with 1-3 bytes from outside the alphabet and not '='
    written at random positions of a valid string: first_bad is the smallest
    written position (known by construction)."""
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    rng = np.random.default_rng(7)
    for trial in range(4000):
        n = int(rng.integers(1, 10))
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        s = bytearray(base64.b64encode(raw.tobytes()))
        k = int(rng.integers(1, 4))
        pos = rng.choice(len(s), size=min(k, len(s)), replace=False)
        for p in pos:
            s[p] = int(NON_ALPHABET_NON_PAD[rng.integers(0, 191)])
        # positions written over a padding '=' may turn an earlier '=' into
        # a bad character; exclude those by construction here
        npad = base64.b64encode(raw.tobytes()).count(b"=")
        if any(p >= len(s) - npad for p in pos) and npad == 2:
            continue
        st, out, fb = oracle.decode(bytes(s))
        assert st == oracle.INVALID_CHAR
        assert fb == int(pos.min()), (bytes(s), fb, pos)


def test_decode_non_alphabet_set_is_complement(oracle):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    outside = {x for x in range(256) if oracle.table1_value(x) < 0 and x != 0x3D}
    assert set(NON_ALPHABET_NON_PAD.tolist()) == outside


def test_round_trip(oracle):
    rng = np.random.default_rng(99)
    for n in list(range(0, 300)) + [int(v) for v in rng.integers(300, 5000, 50)]:
        raw = rng.integers(0, 256, n, dtype=np.uint8)
        enc = oracle.encode(raw)
        st, out, fb = oracle.decode(enc)
        assert st == oracle.OK and fb == enc.size
        assert np.array_equal(out, raw)


def test_trailing_bits_accepted(oracle):
    """Appendix A's extra tail check is not applied: non-zero trailing bits
    decode like Python does (the bits are dropped)."""
    for s in (b"QR==", b"QUJ=", b"R0lGQR=="):
        st, out, fb = oracle.decode(s)
        assert st == oracle.OK and out.tobytes() == _py_strict(s)


# ------------------------------------------------------------ batch pins
def test_batch_matches_python_per_message(oracle):
    from paper_1704_00605_gb300 import workloads

    data, off = workloads.batched(nmsg=300, seed=5, median=200.0)
    enc, eoff = oracle.encode_batch(data, off)
    for j in range(300):
        raw = data[off[j]:off[j + 1]].tobytes()
        assert enc[eoff[j]:eoff[j + 1]].tobytes() == base64.b64encode(raw)
    dst, doff, st, fb, ol = oracle.decode_batch(enc, eoff)
    assert (st == 0).all()
    for j in range(300):
        raw = data[off[j]:off[j + 1]].tobytes()
        assert ol[j] == len(raw) and fb[j] == eoff[j + 1] - eoff[j]
        assert dst[doff[j]:doff[j] + ol[j]].tobytes() == raw


def test_batch_errors_by_construction(oracle):
    from paper_1704_00605_gb300 import workloads

    rec = workloads.error_batch(nmsg=2000, seed=11, lo=16, hi=600, err_fraction=0.05)
    off = rec["in_off"]
    payload = workloads.counter_bytes(rec["payload_key"], 0, int(off[-1]))
    enc, eoff = oracle.encode_batch(payload, off)
    npad = np.array([enc[eoff[j + 1] - 2:eoff[j + 1]].tobytes().count(b"=")
                     for j in rec["err_msg"]])
    pos = workloads.inject_errors(enc, eoff, rec["err_msg"], rec["err_frac"], rec["err_byte"])
    dst, doff, st, fb, ol = oracle.decode_batch(enc, eoff)
    bad = np.zeros(off.size - 1, dtype=bool)
    bad[rec["err_msg"]] = True
    assert (st[~bad] == 0).all()
    assert (st[bad] == 1).all()
    rel = pos - eoff[rec["err_msg"]]
    m = eoff[rec["err_msg"] + 1] - eoff[rec["err_msg"]]
    # an error written over the last '=' of an "==" tail makes the '=' before
    # it the first bad character (strict padding reading); else it is exact
    expect = np.where((npad == 2) & (rel == m - 1), m - 2, rel)
    assert np.array_equal(fb[rec["err_msg"]], expect)
