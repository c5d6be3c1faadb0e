"""The flat kernels of packed batches (kernel choice 3; the decode default).

Decode: a batch whose encoded lengths are all multiples of 4 decodes as one
buffer, the last quad of each message (its final group) decoded by the
finish kernel. Exact against the oracle per message (status, first_bad,
outlen, bytes) with errors in bodies, in final groups and on padding
positions, '=' inside a body, empty messages, messages that end on and
next to tile boundaries, the decode flags; the same batches through the
unstaged tiles agree; batches that do not qualify (a length not a multiple
of 4, short messages on average, buffers off a 16-byte boundary) fall back
to the tile walk and stay exact.

Encode (kernel choice 3 through the shape table; the staged tiles stay the
default): padded output is one flat sequence of quads; exact against the
oracle with empty messages, tile-boundary lengths, a tile holding more
messages than its segment table, the url alphabet, and the fallbacks
(unpadded output, an unaligned output, short messages)."""
import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

URL, NOPAD, STRICT = 1, 2, 4
TILE = 480 * 8 * 16  # characters per tile of the flat decode


def _dev(a, shift=0):
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint8)
    buf = torch.zeros(a.size + 512, dtype=torch.uint8, device="cuda")
    base = (-buf.data_ptr()) % 256
    t = buf[base + shift:base + shift + a.size]
    if a.size:
        t.copy_(torch.from_numpy(a.copy()))
    return t


def _decode(gb64, chars, off, flags=0, shift=0, kernel=3):
    import torch

    kind = gb64.B64_KIND_DECODE_BATCH
    saved = gb64.b64_shape_get(kind, -1, 1)
    try:
        gb64.b64_shape_set(kind, -1, 1, units_per_thread=kernel, threads=128, stages=2,
                           tile=32 * 512)
        dst, oo, st, fb, ol = gb64.b64_decode_batch_ex(
            _dev(chars, shift), torch.from_numpy(np.ascontiguousarray(off)).cuda(), flags)
        torch.cuda.synchronize()
    finally:
        gb64.b64_shape_set(kind, -1, 1, **{f: saved[f] for f in (
            "threads", "units_per_thread", "stages", "blocks_per_sm", "tile")})
    return dst.cpu().numpy(), oo.cpu().numpy(), st.cpu().numpy(), fb.cpu().numpy(), ol.cpu().numpy()


def _check(oracle, chars, off, res, flags):
    h, oo, st, fb, ol = res
    for j in range(off.size - 1):
        m = chars[off[j]:off[j + 1]]
        est, eout, efb = oracle.decode_ex(m, flags)
        assert (st[j], fb[j]) == (est, efb), (j, m.size, flags, st[j], fb[j], est, efb)
        if est == 0:
            assert ol[j] == eout.size and np.array_equal(h[oo[j]:oo[j] + ol[j]], eout), (j, flags)


def _padded_batch(oracle, seed, nmsg, flags=0, mean=6000):
    """Encodings (padded unless NOPAD, whose raw lengths are then multiples of
    3 so every encoded length is a multiple of 4) of log-normal lengths, with
    empty messages and messages ending on and next to tile boundaries."""
    rng = np.random.default_rng(seed)
    lens = np.maximum(0, rng.lognormal(np.log(mean), 1.0, nmsg)).astype(np.int64)
    lens[rng.integers(0, nmsg, nmsg // 20)] = 0
    raw_at_tile = TILE // 4 * 3
    lens[:6] = [raw_at_tile, raw_at_tile - 3, raw_at_tile + 3, 2 * raw_at_tile, 1, 2]
    if flags & NOPAD:
        lens = lens // 3 * 3
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), seed + 100)
    enc = [oracle.encode_ex(data[off[j]:off[j + 1]], flags & (URL | NOPAD)) for j in range(nmsg)]
    coff = W.offsets_from_lengths(np.array([e.size for e in enc], dtype=np.int64))
    assert (np.diff(coff) % 4 == 0).all()
    return np.concatenate(enc), coff


def _inject(rng, chars, coff, frac=0.08):
    """Errors in a fraction of the messages: a byte outside the alphabet in
    the body or the final group, '=' inside the body, '=' before a final
    character, or a space."""
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    chars = chars.copy()
    for j in range(coff.size - 1):
        a, b = int(coff[j]), int(coff[j + 1])
        if b - a < 8 or rng.random() >= frac:
            continue
        k = rng.integers(0, 5)
        if k == 0:
            chars[int(rng.integers(a, b - 4))] = NON_ALPHABET_NON_PAD[int(rng.integers(0, 191))]
        elif k == 1:
            chars[int(rng.integers(b - 4, b))] = NON_ALPHABET_NON_PAD[int(rng.integers(0, 191))]
        elif k == 2:
            chars[int(rng.integers(a, b - 4))] = 0x3D
        elif k == 3:
            chars[b - 3] = 0x3D
        else:
            chars[int(rng.integers(a, b))] = 0x20
    return chars


@pytest.mark.parametrize("flags", [0, URL, STRICT, NOPAD, URL | STRICT])
def test_flat_decode_exact_with_errors(gb64, oracle, flags):
    chars, coff = _padded_batch(oracle, 3 + flags, 1200, flags)
    _check(oracle, chars, coff, _decode(gb64, chars, coff, flags), flags)
    bad = _inject(np.random.default_rng(9 + flags), chars, coff)
    _check(oracle, bad, coff, _decode(gb64, bad, coff, flags), flags)


def test_flat_and_tile_walk_agree(gb64, oracle):
    """One padded batch with errors through the flat decode and through the
    unstaged tiles: the same results and the same decoded bytes."""
    chars, coff = _padded_batch(oracle, 21, 3000)
    bad = _inject(np.random.default_rng(22), chars, coff, 0.05)
    a = _decode(gb64, bad, coff, kernel=3)
    b = _decode(gb64, bad, coff, kernel=2)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)
    h1, h2, oo, ol = a[0], b[0], a[1], a[4]
    for j in range(coff.size - 1):
        if a[2][j] == 0:
            assert np.array_equal(h1[oo[j]:oo[j] + ol[j]], h2[oo[j]:oo[j] + ol[j]])


def test_batches_that_do_not_qualify(gb64, oracle):
    """Kernel choice 3 on batches the flat decode leaves to the tile walk:
    one message of a length not a multiple of 4, short messages on average,
    and a source off a 16-byte boundary; all exact."""
    chars, coff = _padded_batch(oracle, 31, 800)
    odd = np.concatenate([chars, np.frombuffer(b"QUJD", dtype=np.uint8)[:3]])
    ooff = np.concatenate([coff, [coff[-1] + 3]])
    _check(oracle, odd, ooff, _decode(gb64, odd, ooff), 0)
    short, soff = _padded_batch(oracle, 32, 4000, mean=60)
    _check(oracle, short, soff, _decode(gb64, short, soff), 0)
    _check(oracle, chars, coff, _decode(gb64, chars, coff, shift=4), 0)


def test_flat_decode_large(gb64, oracle):
    """About 300 MB of padded messages (the 100,000-message mix), every
    message exact against the oracle in a bounded sample and the whole
    round trip exact."""
    import torch

    data, off = W.batched()
    src, doff = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    enc, eoff = gb64.b64_encode_batch(src, doff)
    dst, oo, st, fb, ol = gb64.b64_decode_batch(enc, eoff)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0
    assert np.array_equal(ol.cpu().numpy(), np.diff(off))
    h, ooh, e, eo = dst.cpu().numpy(), oo.cpu().numpy(), enc.cpu().numpy(), eoff.cpu().numpy()
    for j in range(off.size - 1):
        assert np.array_equal(h[ooh[j]:ooh[j] + off[j + 1] - off[j]], data[off[j]:off[j + 1]]), j
    for j in range(0, off.size - 1, 997):
        est, eout, efb = oracle.decode_ex(e[eo[j]:eo[j + 1]], 0)
        assert (est, efb) == (0, eo[j + 1] - eo[j]) and np.array_equal(eout, data[off[j]:off[j + 1]])


def _enc_flat(gb64, data, off, flags=0, shift=0, kernel=3):
    import torch

    kind = gb64.B64_KIND_ENCODE_BATCH
    saved = gb64.b64_shape_get(kind, -1, 1)
    try:
        gb64.b64_shape_set(kind, -1, 1, units_per_thread=kernel, threads=256, stages=2,
                           tile=16 * 384)
        doff = torch.from_numpy(np.ascontiguousarray(off)).cuda()
        out_off = torch.empty(off.size, dtype=torch.int64, device="cuda")
        gb64.b64_batch_out_offsets_ex(False, doff, flags, out_off)
        need = int(out_off[-1].item())
        buf = torch.zeros(need + 512, dtype=torch.uint8, device="cuda")
        base = (-buf.data_ptr()) % 256
        dst = buf[base + shift:base + shift + max(need, 1)]
        gb64.b64_encode_batch_ex(_dev(data), doff, flags, dst=dst, out_off=out_off)
        torch.cuda.synchronize()
    finally:
        gb64.b64_shape_set(kind, -1, 1, **{f: saved[f] for f in (
            "threads", "units_per_thread", "stages", "blocks_per_sm", "tile")})
    return dst.cpu().numpy()[:need], out_off.cpu().numpy()


def _enc_lengths(seed, nmsg, mean=5000):
    """Log-normal lengths (empty ones among them), lengths whose encodings
    end on and next to the flat encode's tile boundary (53,760 characters),
    and a run of a thousand tiny messages (more messages in one tile than
    its segment table holds)."""
    rng = np.random.default_rng(seed)
    lens = np.maximum(0, rng.lognormal(np.log(mean), 1.0, nmsg)).astype(np.int64)
    lens[rng.integers(0, nmsg, nmsg // 20)] = 0
    at = 53760 // 4 * 3
    lens[:6] = [at, at - 1, at + 1, at - 2, 2 * at, 3]
    lens[100:1100] = rng.integers(0, 12, 1000)
    return lens


@pytest.mark.parametrize("flags", [0, URL])
def test_flat_encode_exact(gb64, oracle, flags):
    lens = _enc_lengths(40 + flags, 3000)
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), 41 + flags)
    exp = np.concatenate([oracle.encode_ex(data[off[j]:off[j + 1]], flags)
                          for j in range(off.size - 1)])
    out, out_off = _enc_flat(gb64, data, off, flags)
    assert np.array_equal(out_off, W.offsets_from_lengths(4 * ((lens + 2) // 3)))
    assert np.array_equal(out, exp)
    walk, _ = _enc_flat(gb64, data, off, flags, kernel=2)
    assert np.array_equal(walk, exp)


def test_flat_encode_fallbacks(gb64, oracle):
    """Kernel choice 3 where the flat encode does not apply: unpadded output,
    an output off a 16-byte boundary, short messages on average."""
    lens = _enc_lengths(50, 1500)
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), 51)
    nopad = np.concatenate([oracle.encode_ex(data[off[j]:off[j + 1]], NOPAD)
                            for j in range(off.size - 1)])
    assert np.array_equal(_enc_flat(gb64, data, off, NOPAD)[0], nopad)
    exp, _ = oracle.encode_batch(data, off)
    assert np.array_equal(_enc_flat(gb64, data, off, shift=4)[0], exp)
    short = np.random.default_rng(52).integers(0, 200, 20_000).astype(np.int64)
    soff = W.offsets_from_lengths(short)
    sdata = W.uniform_bytes(int(soff[-1]), 53)
    assert np.array_equal(_enc_flat(gb64, sdata, soff)[0], oracle.encode_batch(sdata, soff)[0])


def test_flat_encode_large(gb64, oracle):
    """The 100,000-message mix through the flat encode: the encoding equals
    the oracle's in full."""
    data, off = W.batched()
    exp, exp_off = oracle.encode_batch(data, off)
    out, out_off = _enc_flat(gb64, data, off)
    assert np.array_equal(out_off, exp_off)
    assert np.array_equal(out, exp)
