"""The C-ABI library builds, loads and exports every symbol the header
declares; host-side argument checks run without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1704_00605_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gb64.h")


@pytest.fixture(scope="module")
def libpath():
    return build.ensure_built()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(b64_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["b64_encode", "b64_decode", "b64_decode_async", "b64_encode_batch",
              "b64_decode_batch", "b64_batch_out_offsets", "b64_encoded_len", "b64_decoded_cap",
              "b64_encode_host", "b64_decode_host", "b64_status_str", "b64_last_error",
              "b64_device_fault"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (b64_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_header_compiles_as_c(tmp_path):
    c = tmp_path / "t.c"
    c.write_text('#include "gb64.h"\nint main(void){return (int)b64_encoded_len(3) - 4;}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(c), "-o", str(tmp_path / "t.o")], check=True)


@pytest.fixture(scope="module")
def g(libpath):
    from paper_1704_00605_gb300 import gb64

    gb64.lib()
    return gb64


def test_length_closed_forms(g):
    for n in range(0, 100):
        assert g.b64_encoded_len(n) == 4 * -(-n // 3)
        assert g.b64_decoded_cap(n) == 3 * (n // 4)
    assert g.b64_encoded_len((1 << 64) - 1) == g.SIZE_MAX
    assert g.b64_encoded_len(1 << 30) == 1431655768
    assert g.b64_encoded_len((1 << 30) + 2) == 1431655768


def test_status_strings(g):
    assert g.b64_status_str(0) == "B64_OK"
    assert g.b64_status_str(1) == "B64_ERR_INVALID_CHAR"
    assert g.b64_status_str(2) == "B64_ERR_BAD_LENGTH"
    assert g.b64_status_str(-4) == "B64_ERR_TIMEOUT"
    assert g.b64_status_str(99) == "B64_UNKNOWN_STATUS"


def test_argument_errors_need_no_gpu(g):
    L = g.lib()
    # encode: null pointers, overlap; n = 0 is legal and enqueues nothing
    assert L.b64_encode(None, 0, None, None) == 0
    assert L.b64_encode(None, 5, None, None) == g.SIZE_MAX
    assert "null" in g.b64_last_error()
    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    assert L.b64_encode(p, 9, p + 4, None) == g.SIZE_MAX
    assert "overlap" in g.b64_last_error()
    # decode: null result pointers; m = 0 answers on the host
    ol, fb = ctypes.c_size_t(7), ctypes.c_size_t(7)
    assert L.b64_decode(None, 4, None, None, None, None) == g.B64_ERR_ARG
    assert L.b64_decode(None, 0, None, ctypes.byref(ol), ctypes.byref(fb), None) == g.B64_OK
    assert ol.value == 0 and fb.value == 0
    assert L.b64_decode_async(p, 8, p + 16, None, None) == g.B64_ERR_ARG
    assert L.b64_decode_async(p, 8, p + 16, p + 3, None) == g.B64_ERR_ARG  # misaligned result
    assert L.b64_decode_async(p, 8, p + 4, p + 32, None) == g.B64_ERR_ARG  # overlap
    # batch: negative count, null or misaligned offsets
    assert L.b64_encode_batch(p, p, -1, p, p, None) == g.B64_ERR_ARG
    assert L.b64_encode_batch(p, None, 3, p, p, None) == g.B64_ERR_ARG
    assert L.b64_decode_batch(p, p + 4, 3, p, p, p, p, p, None) == g.B64_ERR_ARG
    assert L.b64_batch_out_offsets(0, None, 1, p, None) == g.B64_ERR_ARG
    # host forms
    assert L.b64_encode_host(None, 3, None, None) == g.SIZE_MAX
    assert L.b64_decode_host(p, 4, p, None, None, None) == g.B64_ERR_ARG
    assert L.b64_decode_host(None, 0, None, ctypes.byref(ol), ctypes.byref(fb), None) == g.B64_OK


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1704_00605_gb300 import gb64

    monkeypatch.setattr(gb64, "_lib", None)
    monkeypatch.setattr(gb64._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gb64.lib()


def test_shape_table_host_side(g, tmp_path):
    """The shape table (no GPU needed): defaults, set/get per bucket,
    rejection of invalid shapes, save/load round trip."""
    d = g.b64_shape_get(g.B64_KIND_ENCODE, 1 << 30)
    assert d["threads"] in (128, 256, 512) and d["tile"] == d["threads"] * d["units_per_thread"] * 12
    g.b64_shape_set(g.B64_KIND_ENCODE, 1 << 20, threads=128, units_per_thread=2, stages=3)
    assert g.b64_shape_get(g.B64_KIND_ENCODE, (1 << 20) + 5)["threads"] == 128  # same bucket
    assert g.b64_shape_get(g.B64_KIND_ENCODE, 1 << 30)["threads"] == d["threads"]  # other bucket
    with pytest.raises(g.Gb64Error):
        g.b64_shape_set(g.B64_KIND_ENCODE, 1 << 20, threads=100)
    with pytest.raises(g.Gb64Error):
        g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 10_000, 10, threads=256, tile=1000)
    with pytest.raises(g.Gb64Error):  # not a whole number of warp rows (512 characters)
        g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 10_000, 10, threads=128, tile=768)
    with pytest.raises(g.Gb64Error):  # 16 warps x 4 stages x 14 KiB: more shared memory than a CTA has
        g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 10_000, 10, threads=512, tile=8192, stages=4)
    with pytest.raises(g.Gb64Error):
        g.b64_shape_set(g.B64_KIND_ENCODE_BATCH, 10_000, 10, threads=128, tile=1536, stages=7)
    with pytest.raises(g.Gb64Error):  # 16 warps x 3 stages x 4.5 KiB: no room left for the
        # encode kernel's static tables (17.4 KiB with the 8 KiB pair table) under 227 KiB
        g.b64_shape_set(g.B64_KIND_ENCODE_BATCH, 10_000, 10, threads=512, tile=12 * 384, stages=3)
    g.b64_shape_set(g.B64_KIND_ENCODE_BATCH, 10_000, 10, threads=512, tile=16 * 384, stages=2)
    # unstaged tiles (kernel choice 2) use no shared memory: up to 64 rows
    g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 10_000, 10, threads=512, tile=64 * 512, stages=2,
                    units_per_thread=2)
    with pytest.raises(g.Gb64Error):
        g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 10_000, 10, threads=128, tile=65 * 512,
                        units_per_thread=2)
    with pytest.raises(g.Gb64Error):  # staged tiles: at most 16 rows
        g.b64_shape_set(g.B64_KIND_ENCODE_BATCH, 10_000, 10, threads=128, tile=17 * 384,
                        units_per_thread=0)
    with pytest.raises(g.Gb64Error):  # kernel choices are 0 .. 3
        g.b64_shape_set(g.B64_KIND_ENCODE_BATCH, 10_000, 10, units_per_thread=4)
    g.b64_shape_set(g.B64_KIND_ENCODE_BATCH, 10_000, 10, threads=256, tile=16 * 384, stages=2,
                    units_per_thread=3)  # the flat encode, unstaged tiles otherwise
    g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 40_000, 10, threads=512, tile=1024, stages=2,
                    blocks_per_sm=4)
    assert g.b64_shape_get(g.B64_KIND_DECODE_BATCH, 40_000, 10)["stages"] == 2
    path = str(tmp_path / "shapes.txt")
    g.b64_tune_save(path)
    text = open(path).read()
    assert "512" in text and "128" in text
    g.b64_shape_set(g.B64_KIND_DECODE_BATCH, 40_000, 10, threads=256, tile=2048, blocks_per_sm=8)
    g.b64_tune_load(path)
    assert g.b64_shape_get(g.B64_KIND_DECODE_BATCH, 40_000, 10)["threads"] == 512


def test_default_shapes_need_no_gpu(g):
    """The defaults the shape table answers with when nothing was set or
    tuned (no GPU needed): batched decode takes the flat decode (kernel
    choice 3, unstaged 32-row tiles for batches it leaves alone), batched
    encode the staged 16-row tiles (16 warps), the whitespace line kernel 512 threads
    x 7 units x 2 stages for large inputs."""
    d = g.b64_shape_get(g.B64_KIND_DECODE_BATCH, 123_456_789, 1000)
    assert (d["units_per_thread"], d["threads"], d["tile"]) == (3, 128, 32 * 512)
    e = g.b64_shape_get(g.B64_KIND_ENCODE_BATCH, 123_456_789, 1000)
    assert (e["units_per_thread"], e["threads"], e["tile"], e["stages"]) == (0, 512, 16 * 384, 2)
    w = g.b64_shape_get(g.B64_KIND_DECODE_WS, 367_332_732, 1)
    assert (w["threads"], w["units_per_thread"], w["stages"]) == (512, 7, 2)
