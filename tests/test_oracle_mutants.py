"""The oracle's pins are strong enough to catch plausible mistakes.

Each mutant is a copy of the oracle source with one planted error (a dropped
term, a wrong shift or modulus, a swapped operand, a wrong padding rule),
compiled on the CPU into a temporary library. A subset of the independent
pins (Python's base64/binascii, the paper's worked examples) must reject
every mutant, and must accept the unmodified source.
"""
import base64
import binascii
import ctypes
import os
import subprocess

import numpy as np
import pytest

from tests import golden

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "b64_oracle.c")
VARIANTS_MARK = "/* ------------------------------------------------------------------------\n * Variants"


def mutate(text: str, old: str, new: str, variants: bool) -> str:
    """Replace the single occurrence of `old` in the base functions (or, with
    variants=True, in the variant functions) of the oracle source."""
    cut = text.index(VARIANTS_MARK)
    head, tail = text[:cut], text[cut:]
    region = tail if variants else head
    assert region.count(old) == 1, f"mutation anchor not found exactly once: {old!r}"
    region = region.replace(old, new)
    return head + region if variants else region + tail

MUTANTS = {
    "enc_drop_hi_term": ("B(((s[i] * 16) % 64) + (s[i + 1] / 16));\n    p[k++] = B(((s[i + 1]",
                         "B(((s[i] * 16) % 64));\n    p[k++] = B(((s[i + 1]"),
    "enc_wrong_div": ("(s[i + 2] / 64)", "(s[i + 2] / 32)"),
    "enc_wrong_mod": ("B(s[i + 2] % 64)", "B(s[i + 2] % 63)"),
    "enc_swap_operands": ("p[k++] = B(s[i] / 4);\n    p[k++] = B(((s[i] * 16)",
                          "p[k++] = B(s[i + 1] / 4);\n    p[k++] = B(((s[i] * 16)"),
    "enc_tail_one_pad": ("      p[k++] = B((s[i] * 16) % 64);\n      p[k++] = PAD;",
                         "      p[k++] = B((s[i] * 16) % 64);\n      p[k++] = 'A';"),
    "table_swap_plus_slash": ("'8', '9', '+', '/'}", "'8', '9', '/', '+'}"),
    "dec_wrong_shift": ("(uint8_t)((a * 4) + (b / 16))", "(uint8_t)((a * 4) + (b / 8))"),
    "dec_wrong_mod": ("(((b * 16) % 256) + (cc / 4))", "(((b * 16) % 128) + (cc / 4))"),
    "dec_swap_cd": ("(((cc * 64) % 256) + d)", "(((d * 64) % 256) + cc)"),
    "dec_pad_anywhere": ("int is_padding = (npad > 0) && (i >= m - npad);",
                         "int is_padding = (c[i] == PAD);"),
    "dec_len_rule": ("*first_bad = m - m % 4;", "*first_bad = m;"),
    "dec_first_bad_off_by_one": ("*first_bad = i;\n", "*first_bad = i + 1;\n"),
    "dec_pad2_without_pad1": ("if (c[m - 2] != PAD) return 1;", "if (c[m - 3] != PAD) return 1;"),
}


def _compile(tmp_path, name, text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", str(c), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    lib.oracle_encode.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    lib.oracle_encode.restype = ctypes.c_size_t
    lib.oracle_decode.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
    lib.oracle_decode.restype = ctypes.c_int
    return lib


def _enc(lib, raw: bytes) -> bytes:
    out = ctypes.create_string_buffer(4 * (len(raw) // 3 + 1) + 4)
    k = lib.oracle_encode(raw, len(raw), out)
    return out.raw[:k]


def _dec(lib, s: bytes):
    out = ctypes.create_string_buffer(3 * (len(s) // 4) + 4)
    ol, fb = ctypes.c_size_t(), ctypes.c_size_t()
    st = lib.oracle_decode(s, len(s), out, ctypes.byref(ol), ctypes.byref(fb))
    return st, out.raw[:ol.value], fb.value


def _pins_pass(lib) -> bool:
    rng = np.random.default_rng(3)
    # encode: Python's encoder on random inputs of every length class
    for n in (0, 1, 2, 3, 4, 5, 47, 48, 49, 3000):
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        if _enc(lib, raw) != base64.b64encode(raw):
            return False
    if _enc(lib, bytes(golden.ints("encode_example_bytes"))) != golden.text("encode_example_chars").encode():
        return False
    # decode: the paper's example and Python's strict decoder on injections
    st, out, fb = _dec(lib, golden.text("decode_example_chars").encode())
    if st != 0 or list(out) != golden.ints("decode_example_bytes"):
        return False
    for base in (b"QUJDREVGR0lG", b"R0lGQUI=", b"R0lGQQ=="):
        for q in range(len(base)):
            for x in range(256):
                s = bytearray(base)
                s[q] = x
                s = bytes(s)
                try:
                    py = binascii.a2b_base64(s, strict_mode=True)
                except binascii.Error:
                    py = None
                st, out, fb = _dec(lib, s)
                if (py is None) != (st != 0):
                    return False
                if py is not None and (out != py or fb != len(s)):
                    return False
                if py is None and x not in b"=" and base[q:q + 1] != b"=" and fb != q:
                    return False
    # length rule: construction gives the start of the incomplete group
    for m in (1, 2, 3, 5, 6, 7, 9):
        st, out, fb = _dec(lib, b"QUJD" * 3 + b"Q"[:0] + (b"QUJD" * 3)[: m])
        mm = 12 + m
        if st != 2 or fb != mm - mm % 4:
            return False
    return True


def test_unmodified_oracle_passes(tmp_path):
    assert _pins_pass(_compile(tmp_path, "orig", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _compile(tmp_path, name, mutate(open(SRC).read(), old, new, variants=False))
    assert not _pins_pass(lib), f"planted mistake {name} survived the pins"


# --------------------------------------------------- the variant functions
VARIANT_MUTANTS = {
    "url_swap_62_63": ("if (v == 62) return '-';", "if (v == 63) return '-';"),
    "url_accepts_plus_slash": ("    if (x == '+' || x == '/') return -1;\n", "\n"),
    "strict_tail_wrong_multiplier": ("      mult = 16;", "      mult = 32;"),
    "strict_tail_wrong_index": ("idx = (npad == 1) ? m - 2 : m - 1;", "idx = (npad == 1) ? m - 3 : m - 1;"),
    "nopad_length_rule": ("if (m % 4 != 0 && (!nopad || m % 4 == 1)) {", "if (m % 4 != 0 && !nopad) {"),
    "nopad_keeps_padding": ("      if (pad) p[k++] = PAD;\n    } else if", "      p[k++] = PAD;\n    } else if"),
    "nopad_tail_shift": ("      p[k++] = (uint8_t)(((b * 16) % 256) + (cc / 4));\n    }\n  }",
                         "      p[k++] = (uint8_t)(((b * 16) % 256) + (cc / 8));\n    }\n  }"),
    "ws_misses_cr": ("return x == ' ' || x == '\\n' || x == '\\r';", "return x == ' ' || x == '\\n';"),
    "ws_first_bad_not_mapped": ("*first_bad = (st == ORACLE_OK) ? m : from[fb];",
                                "*first_bad = (st == ORACLE_OK) ? m : fb;"),
}


def _bind_ex(lib):
    lib.oracle_encode_ex.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int]
    lib.oracle_encode_ex.restype = ctypes.c_size_t
    lib.oracle_decode_ex.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t), ctypes.c_int]
    lib.oracle_decode_ex.restype = ctypes.c_int
    lib.oracle_decode_ws.argtypes = lib.oracle_decode_ex.argtypes
    lib.oracle_decode_ws.restype = ctypes.c_int
    return lib


def _enc_ex(lib, raw: bytes, flags: int) -> bytes:
    out = ctypes.create_string_buffer(4 * (len(raw) // 3 + 1) + 4)
    k = lib.oracle_encode_ex(raw, len(raw), out, flags)
    return out.raw[:k]


def _dec_ex(lib, s: bytes, flags: int):
    out = ctypes.create_string_buffer(3 * (len(s) // 4) + 8)
    ol, fb = ctypes.c_size_t(), ctypes.c_size_t()
    fn = lib.oracle_decode_ws if flags & 8 else lib.oracle_decode_ex
    st = fn(s, len(s), out, ctypes.byref(ol), ctypes.byref(fb), flags)
    return st, out.raw[:ol.value], fb.value


def _variant_pins_pass(lib) -> bool:
    rng = np.random.default_rng(8)
    for n in (0, 1, 2, 3, 4, 5, 62, 63, 64, 700):
        raw = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        for flags, py in ((1, base64.urlsafe_b64encode(raw)), (2, base64.b64encode(raw).rstrip(b"=")),
                          (3, base64.urlsafe_b64encode(raw).rstrip(b"="))):
            if _enc_ex(lib, raw, flags) != py:
                return False
            st, out, fb = _dec_ex(lib, py, flags)
            if st != 0 or out != raw:
                return False
    if _dec_ex(lib, b"ab+c", 1)[0] != 1:  # '+' is outside the url alphabet
        return False
    if _dec_ex(lib, b"QUJDQ", 2)[0::2] != (2, 4):  # one character past whole groups
        return False
    canon1 = {base64.b64encode(bytes([a])) for a in range(256)}
    canon2 = {base64.b64encode(bytes([a, b])) for a in range(256) for b in range(0, 256, 7)}
    for s in canon1:
        if _dec_ex(lib, s, 4)[0] != 0:
            return False
    for s in canon2:
        if _dec_ex(lib, s, 4)[0] != 0:
            return False
    for s, fb in ((b"QR==", 1), (b"QI==", 1), (b"QUJ=", 2), (b"QUB=", 2), (b"R0lGQR==", 5)):
        if _dec_ex(lib, s, 4)[0::2] != (3, fb):
            return False
    # whitespace removal (Appendix B): space, LF and CR anywhere; first_bad in
    # original offsets
    if _dec_ex(lib, b"QU\r\nJD R E\nVG\r\n", 8)[:2] != (0, b"ABCDEF"):
        return False
    if _dec_ex(lib, b"QU\r\nJD R!\nVG", 8)[0::2] != (1, 8):
        return False
    return True


def test_unmodified_variants_pass(tmp_path):
    assert _variant_pins_pass(_bind_ex(_compile(tmp_path, "orig_ex", open(SRC).read())))


@pytest.mark.parametrize("name", sorted(VARIANT_MUTANTS))
def test_variant_mutant_is_caught(tmp_path, name):
    old, new = VARIANT_MUTANTS[name]
    lib = _bind_ex(_compile(tmp_path, name, mutate(open(SRC).read(), old, new, variants=True)))
    assert not _variant_pins_pass(lib), f"planted mistake {name} survived the pins"
