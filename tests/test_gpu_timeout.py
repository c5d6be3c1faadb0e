"""The timeout path of the bounded waits, without a GPU fault: the test hook
b64_test_stall_copies makes the first CTA (warp) of each pipelined kernel
leave out its first input copy, so that CTA's wait on it runs out after a
short limit. The kernel records the fault word, waits (bounded) for its other
copies and returns; the call reports B64_ERR_TIMEOUT and b64_device_fault()
returns it once. With the hook off, the next calls are exact against the
oracle again."""
import contextlib

import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LIMIT_NS = 2_000_000  # 2 ms


@contextlib.contextmanager
def stalled(gb64):
    assert gb64.b64_device_fault() == 0  # nothing left from earlier tests
    gb64.b64_test_stall_copies(True, LIMIT_NS)
    try:
        yield
    finally:
        gb64.b64_test_stall_copies(False, 0)


def _payload(n, seed):
    import torch

    raw = W.uniform_bytes(n, seed)
    return raw, torch.from_numpy(raw).cuda()


def test_single_decode_times_out_then_recovers(gb64, oracle):
    import torch

    raw, src = _payload(1 << 20, 41)
    enc = gb64.b64_encode(src)
    exp = oracle.encode(raw)
    assert np.array_equal(enc.cpu().numpy(), exp)
    dst = torch.empty(gb64.b64_decoded_cap(enc.numel()), dtype=torch.uint8, device="cuda")
    res = torch.empty(3, dtype=torch.int64, device="cuda")
    with stalled(gb64):
        gb64.b64_decode_async(enc, dst, res)
        torch.cuda.synchronize()
        st, outlen, fb = gb64.parse_result(res)
    assert st == gb64.B64_ERR_TIMEOUT, (st, outlen, fb)
    assert outlen == 0
    assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
    assert gb64.b64_device_fault() == 0  # read and cleared
    # the next call is exact
    st, outlen, fb, d = gb64.b64_decode(enc)
    assert (st, outlen, fb) == (0, raw.size, exp.size)
    assert np.array_equal(d[:outlen].cpu().numpy(), raw)


def test_single_encode_times_out_then_recovers(gb64, oracle):
    raw, src = _payload((1 << 20) + 1, 42)
    with stalled(gb64):
        gb64.b64_encode(src)
        assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
    assert gb64.b64_device_fault() == 0
    enc = gb64.b64_encode(src)
    assert np.array_equal(enc.cpu().numpy(), oracle.encode(raw))


def test_staged_batch_times_out_then_recovers(gb64, oracle):
    """Encode batches use the staged tile kernel by default; the decode batch
    is sent to it through the shape table. Every message then reports
    B64_ERR_TIMEOUT until the fault word is read."""
    import torch

    data, off = W.batched(nmsg=3000, seed=43, median=4000.0, sigma=1.0)
    src, doff = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    oenc, ooff = oracle.encode_batch(data, off)
    kinds = (gb64.B64_KIND_ENCODE_BATCH, gb64.B64_KIND_DECODE_BATCH)
    saved = [gb64.b64_shape_get(k, -1, 1) for k in kinds]
    try:
        for k in kinds:
            dec = k == gb64.B64_KIND_DECODE_BATCH
            gb64.b64_shape_set(k, -1, 1, units_per_thread=1, threads=128, stages=2,
                               tile=8 * 512 if dec else 16 * 384)
        with stalled(gb64):
            gb64.b64_encode_batch(src, doff)
            assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
        benc, boff = gb64.b64_encode_batch(src, doff)
        assert np.array_equal(boff.cpu().numpy(), ooff)
        assert np.array_equal(benc.cpu().numpy()[:oenc.size], oenc)
        with stalled(gb64):
            _, _, st, fb, ol = gb64.b64_decode_batch(benc, boff)
            torch.cuda.synchronize()
            assert bool((st == gb64.B64_ERR_TIMEOUT).all())
            assert int(ol.abs().sum()) == 0
            assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
        ddst, doff2, st, fb, ol = gb64.b64_decode_batch(benc, boff)
        assert int((st != 0).sum()) == 0
        assert np.array_equal(ol.cpu().numpy(), np.diff(off))
        h, oo = ddst.cpu().numpy(), doff2.cpu().numpy()
        for j in range(0, off.size - 1, 37):
            assert np.array_equal(h[oo[j]:oo[j] + off[j + 1] - off[j]], data[off[j]:off[j + 1]])
    finally:
        for k, sh in zip(kinds, saved):
            gb64.b64_shape_set(k, -1, 1, **{f: sh[f] for f in ("threads", "units_per_thread",
                                                                 "stages", "blocks_per_sm",
                                                                 "tile")})
    assert gb64.b64_device_fault() == 0


def test_whitespace_decode_times_out_then_recovers(gb64, oracle):
    """The line-model kernel of the whitespace decode: CTA 0's first stage
    wait runs out, the CTAs still meet at the grid barrier, and the call
    reports B64_ERR_TIMEOUT with first_bad = m; then the same input decodes
    exactly through the line path."""
    import base64

    import torch

    raw = W.uniform_bytes(3 << 20, 44)
    e = base64.b64encode(raw.tobytes())
    s = b"\r\n".join(e[i:i + 76] for i in range(0, len(e), 76)) + b"\r\n"
    src = torch.from_numpy(np.frombuffer(s, dtype=np.uint8).copy()).cuda()
    dst = torch.zeros(raw.size + 16, dtype=torch.uint8, device="cuda")
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    with stalled(gb64):
        gb64.b64_decode_async_ex(src, dst, res, 8)
        torch.cuda.synchronize()
        st, outlen, fb = gb64.parse_result(res)
        assert (st, outlen, fb) == (gb64.B64_ERR_TIMEOUT, 0, len(s))
        assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
    assert gb64.b64_device_fault() == 0
    gb64.b64_decode_async_ex(src, dst, res, 8)
    torch.cuda.synchronize()
    assert gb64.parse_result(res) == (0, raw.size, len(s))
    assert int(res.view(torch.int32)[5].item()) & 0xFFFFFFFF == 0x4C494E45
    assert np.array_equal(dst[:raw.size].cpu().numpy(), raw)
    ost, oout, ofb = oracle.decode_ex(s, 8)
    assert (ost, ofb) == (0, len(s)) and np.array_equal(oout, raw)


def test_flat_batch_decode_times_out_then_recovers(gb64, oracle):
    """The flat decode of a padded batch (the default decode of such
    batches): CTA 0's first copy is left out, its wait runs out, every
    message reports B64_ERR_TIMEOUT; then the batch decodes exactly."""
    import torch

    data, off = W.batched(nmsg=3000, seed=45, median=6000.0, sigma=1.0)
    src, doff = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    benc, boff = gb64.b64_encode_batch(src, doff)
    with stalled(gb64):
        _, _, st, fb, ol = gb64.b64_decode_batch(benc, boff)
        torch.cuda.synchronize()
        assert bool((st == gb64.B64_ERR_TIMEOUT).all())
        assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
    ddst, doff2, st, fb, ol = gb64.b64_decode_batch(benc, boff)
    assert int((st != 0).sum()) == 0
    assert np.array_equal(ol.cpu().numpy(), np.diff(off))
    h, oo = ddst.cpu().numpy(), doff2.cpu().numpy()
    for j in range(0, off.size - 1, 29):
        assert np.array_equal(h[oo[j]:oo[j] + off[j + 1] - off[j]], data[off[j]:off[j + 1]])
    assert gb64.b64_device_fault() == 0


def test_flat_batch_encode_times_out_then_recovers(gb64, oracle):
    """The flat encode (kernel choice 3, set through the shape table) of a
    batch of long messages: CTA 0's first copy is left out and its wait runs
    out; then the batch encodes exactly."""
    import torch

    data, off = W.batched(nmsg=3000, seed=46, median=6000.0, sigma=1.0)
    src, doff = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    kind = gb64.B64_KIND_ENCODE_BATCH
    saved = gb64.b64_shape_get(kind, -1, 1)
    try:
        gb64.b64_shape_set(kind, -1, 1, threads=256, units_per_thread=3, stages=2, tile=16 * 384)
        with stalled(gb64):
            gb64.b64_encode_batch(src, doff)
            assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
        assert gb64.b64_device_fault() == 0
        benc, boff = gb64.b64_encode_batch(src, doff)
    finally:
        gb64.b64_shape_set(kind, -1, 1, **{f: saved[f] for f in (
            "threads", "units_per_thread", "stages", "blocks_per_sm", "tile")})
    oenc, ooff = oracle.encode_batch(data, off)
    assert np.array_equal(boff.cpu().numpy(), ooff)
    assert np.array_equal(benc.cpu().numpy()[:oenc.size], oenc)
