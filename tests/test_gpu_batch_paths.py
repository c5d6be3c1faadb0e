"""The kernels of the batched codec against the oracle (exact), on the same
batches: short messages one thread each with staged per-warp tiles for the
rest, staged tiles for every message, short messages with unstaged tiles
(of 8 and of 64 rows), and the flat kernels of padded batches (unstaged
tiles for the others), chosen through the shape table's kernel choice (0,
1, 2, 3), each with buffers on and off a 16-byte boundary. Batches mix empty, tiny and large messages, lengths of
every class mod 3 and mod 4, messages that straddle tiles and tiles that
hold hundreds of messages, padding, errors at every kind of position, and
the decode flags."""
import contextlib

import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

URL, NOPAD, STRICT = 1, 2, 4
# kernel choice, and tile rows of encode and decode
STAGED, STAGED_ALL, DIRECT, DIRECT_LONG = (0, 16, 8), (1, 16, 8), (2, 8, 8), (2, 64, 64)
FLAT = (3, 8, 32)  # the flat kernels where the batch qualifies, else unstaged tiles
MODES = (STAGED, STAGED_ALL, DIRECT, DIRECT_LONG, FLAT)


@contextlib.contextmanager
def kernel_choice(gb64, mode):
    """Batch calls (whose total size the library does not know) use the
    given kernel choice and tile rows while the block runs."""
    kernel, enc_rows, dec_rows = mode
    kinds = (gb64.B64_KIND_ENCODE_BATCH, gb64.B64_KIND_DECODE_BATCH)
    saved = [gb64.b64_shape_get(k, -1, 1) for k in kinds]
    try:
        for k in kinds:
            dec = k == gb64.B64_KIND_DECODE_BATCH
            gb64.b64_shape_set(k, -1, 1, units_per_thread=kernel, threads=128, stages=2,
                               tile=dec_rows * 512 if dec else enc_rows * 384)
        yield
    finally:
        for k, sh in zip(kinds, saved):
            gb64.b64_shape_set(k, -1, 1, **{f: sh[f] for f in ("threads", "units_per_thread",
                                                                 "stages", "blocks_per_sm",
                                                                 "tile")})


def _dev_at(a, shift):
    """A device copy of a whose first byte is `shift` bytes past a 256-byte
    boundary."""
    import torch

    a = np.ascontiguousarray(a, dtype=np.uint8)
    buf = torch.zeros(a.size + 512, dtype=torch.uint8, device="cuda")
    base = (-buf.data_ptr()) % 256
    t = buf[base + shift:base + shift + a.size]
    if a.size:
        t.copy_(torch.from_numpy(a.copy()))
    return t


def _off(off):
    import torch

    return torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda()


def _encode(gb64, data, off, dst_shift, flags=0):
    """Encode with the output starting dst_shift bytes past a 256-byte
    boundary; returns the output and its offsets."""
    import torch

    out_off = torch.empty(off.size, dtype=torch.int64, device="cuda")
    gb64.b64_batch_out_offsets_ex(False, _off(off), flags, out_off)
    need = int(out_off[-1].item())
    buf = torch.zeros(need + 512, dtype=torch.uint8, device="cuda")
    base = (-buf.data_ptr()) % 256
    dst = buf[base + dst_shift:base + dst_shift + max(need, 1)]
    gb64.b64_encode_batch_ex(_dev_at(data, 0), _off(off), flags, dst=dst, out_off=out_off)
    return dst.cpu().numpy()[:need], out_off.cpu().numpy()


def _decode(gb64, chars, off, src_shift, flags=0):
    dst, out_off, st, fb, ol = gb64.b64_decode_batch_ex(_dev_at(chars, src_shift), _off(off), flags)
    return (dst.cpu().numpy(), out_off.cpu().numpy(), st.cpu().numpy(), fb.cpu().numpy(),
            ol.cpu().numpy())


def _check_decode(oracle, chars, off, res, flags):
    h, oo, st, fb, ol = res
    for j in range(off.size - 1):
        m = chars[off[j]:off[j + 1]]
        est, eout, efb = oracle.decode_ex(m, flags)
        assert (st[j], fb[j]) == (est, efb), (j, m.size, flags, st[j], fb[j], est, efb)
        if est == 0:
            assert ol[j] == eout.size and np.array_equal(h[oo[j]:oo[j] + ol[j]], eout), (j, flags)


def _mixed_lengths(rng, nmsg):
    """Tiny, empty and large messages in runs, so that some tiles hold one
    message and others hundreds."""
    kind = rng.integers(0, 6, nmsg)
    lens = np.where(kind == 0, 0, 0)
    lens = np.where(kind == 1, rng.integers(1, 16, nmsg), lens)
    lens = np.where(kind == 2, rng.integers(16, 200, nmsg), lens)
    lens = np.where(kind == 3, rng.integers(200, 5000, nmsg), lens)
    lens = np.where(kind == 4, rng.integers(5000, 70000, nmsg), lens)
    lens = np.where(kind == 5, rng.integers(0, 4, nmsg) * 4096 + rng.integers(0, 3, nmsg), lens)
    runs = rng.integers(0, 2, nmsg // 50 + 1)
    for r, v in enumerate(runs):  # every other stretch of 50: tiny messages only
        if v:
            lens[50 * r:50 * r + 50] = rng.integers(0, 20, len(lens[50 * r:50 * r + 50]))
    return lens.astype(np.int64)


@pytest.mark.parametrize("seed", [1, 2])
def test_encode_both_paths(gb64, oracle, seed):
    rng = np.random.default_rng(seed)
    lens = _mixed_lengths(rng, 1500)
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), 40 + seed)
    exp, exp_off = oracle.encode_batch(data, off)
    exp_url = np.concatenate([oracle.encode_ex(data[off[j]:off[j + 1]], URL)
                              for j in range(off.size - 1)])
    for mode in MODES:
        with kernel_choice(gb64, mode):
            for shift in (0, 4, 8, 12, 1):  # outputs on and off a 16-byte boundary
                out, out_off = _encode(gb64, data, off, shift)
                assert np.array_equal(out_off, exp_off)
                assert np.array_equal(out, exp), (mode, shift)
            out, _ = _encode(gb64, data, off, 0, URL)
            assert np.array_equal(out, exp_url), mode


@pytest.mark.parametrize("seed", [3, 4])
def test_decode_both_paths_valid_and_errors(gb64, oracle, seed):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    rng = np.random.default_rng(seed)
    lens = _mixed_lengths(rng, 1500)
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), 50 + seed)
    chars, coff = oracle.encode_batch(data, off)
    chars = chars.copy()
    nbad = 0
    for j in range(coff.size - 1):
        a, b = coff[j], coff[j + 1]
        if b > a and rng.random() < 0.05:
            # an error in the body, in the final quad, or on a padding position
            p = int(rng.integers(a, b)) if rng.random() < 0.7 else int(b - 1 - rng.integers(0, min(4, b - a)))
            chars[p] = NON_ALPHABET_NON_PAD[int(rng.integers(0, NON_ALPHABET_NON_PAD.size))]
            nbad += 1
    assert nbad > 10
    for mode in MODES:
        with kernel_choice(gb64, mode):
            for shift in (0, 3, 8):  # inputs on and off a 16-byte boundary
                _check_decode(oracle, chars, coff, _decode(gb64, chars, coff, shift), 0)


@pytest.mark.parametrize("flags", [0, URL, NOPAD, STRICT, URL | NOPAD | STRICT])
def test_decode_both_paths_lengths_not_multiple_of_4(gb64, oracle, flags):
    """Messages of every length mod 4 (so later messages start off a
    multiple of 4), with random '=' and other bytes mixed in."""
    rng = np.random.default_rng(7 + flags)
    alpha = oracle.encode_ex(np.frombuffer(int("".join(f"{v:06b}" for v in range(64)), 2)
                                           .to_bytes(48, "big"), dtype=np.uint8), flags & URL)
    nmsg = 2500
    lens = np.where(rng.random(nmsg) < 0.2, rng.integers(2000, 40000, nmsg), rng.integers(0, 90, nmsg))
    off = W.offsets_from_lengths(lens.astype(np.int64))
    chars = alpha[rng.integers(0, 64, int(off[-1]))]
    for j in range(nmsg):
        a, b = off[j], off[j + 1]
        r = rng.random()
        if b - a >= 2 and r < 0.15:
            chars[b - 2:b] = 0x3D
        elif b - a >= 1 and r < 0.3:
            chars[b - 1] = 0x3D
        elif b > a and r < 0.4:
            chars[int(rng.integers(a, b))] = int(rng.integers(0, 256))
    for mode in MODES:
        with kernel_choice(gb64, mode):
            for shift in (0, 5):
                _check_decode(oracle, chars, off, _decode(gb64, chars, off, shift, flags), flags)


def test_decode_tiles_of_tiny_messages(gb64, oracle):
    """100,000 messages of 0-24 characters (one thread each): every final
    group and padding form, buffers on and off a 16-byte boundary."""
    rng = np.random.default_rng(11)
    lens = rng.integers(0, 19, 100_000)
    off = W.offsets_from_lengths(lens.astype(np.int64))
    data = W.uniform_bytes(int(off[-1]), 12)
    chars, coff = oracle.encode_batch(data, off)
    for shift in (0, 1):
        res = _decode(gb64, chars, coff, shift)
        h, oo, st, fb, ol = res
        assert (st == 0).all() and np.array_equal(ol, np.diff(off))
        assert np.array_equal(np.concatenate([h[oo[j]:oo[j] + ol[j]] for j in range(0, 100_000, 97)]),
                              np.concatenate([data[off[j]:off[j + 1]] for j in range(0, 100_000, 97)]))
    out, out_off = _encode(gb64, data, off, 0)
    assert np.array_equal(out, chars) and np.array_equal(out_off, coff)


def test_mixed_short_and_long_batches(gb64, oracle):
    """The same content cut into short messages (one thread each) and into
    long ones (the tile kernels), and a batch of mostly tiny messages with a
    few large ones, code exactly by default."""
    rng = np.random.default_rng(13)
    data = W.uniform_bytes(3 << 20, 14)
    for lens in (rng.integers(0, 200, 40_000), rng.integers(5000, 60000, 100),
                 np.concatenate([rng.integers(0, 30, 30_000), [300_000, 70_001, 1 << 20]])):
        lens = lens.astype(np.int64)
        off = W.offsets_from_lengths(lens)
        d = data[:off[-1]] if off[-1] <= data.size else W.uniform_bytes(int(off[-1]), 15)
        exp, exp_off = oracle.encode_batch(d, off)
        out, out_off = _encode(gb64, d, off, 0)
        assert np.array_equal(out_off, exp_off) and np.array_equal(out, exp)
        _check_decode(oracle, exp, exp_off, _decode(gb64, exp, exp_off, 0), 0)


@pytest.mark.parametrize("flags", [0, URL | NOPAD, STRICT])
def test_lengths_around_the_short_message_limit(gb64, oracle, flags):
    """Messages just below, at and above the longest length the short-message
    kernel takes (256 bytes, 344 characters), mixed with tiny and long ones,
    with errors: both sides of the split code exactly."""
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    rng = np.random.default_rng(31 + flags)
    lens = np.concatenate([rng.integers(230, 290, 600), rng.integers(0, 40, 300),
                           rng.integers(250, 262, 300), rng.integers(250, 260, 200),
                           [5000, 70000, 0, 1, 2]])
    rng.shuffle(lens)
    off = W.offsets_from_lengths(lens.astype(np.int64))
    data = W.uniform_bytes(int(off[-1]), 60 + flags)
    enc = [oracle.encode_ex(data[off[j]:off[j + 1]], flags & (URL | NOPAD)) for j in range(off.size - 1)]
    if not flags & NOPAD:
        out, out_off = _encode(gb64, data, off, 0, flags & URL)
        assert np.array_equal(out, np.concatenate(enc))
    chars = [e.copy() for e in enc]
    for j in rng.integers(0, len(chars), 60):
        if chars[j].size:
            chars[j][int(rng.integers(0, chars[j].size))] = NON_ALPHABET_NON_PAD[int(rng.integers(0, 191))]
    coff = W.offsets_from_lengths(np.array([c.size for c in chars], dtype=np.int64))
    allc = np.concatenate(chars)
    for mode in MODES:
        with kernel_choice(gb64, mode):
            _check_decode(oracle, allc, coff, _decode(gb64, allc, coff, 0, flags), flags)


@pytest.mark.parametrize("mode", MODES)
def test_weight_split_edge_cases(gb64, oracle, mode):
    """The warps' equal shares of the batch weight (bytes + a fixed cost per
    tile): batches whose total weight is below the number of warps (most
    shares empty), one huge message among tiny ones (its tiles spread over
    many warps), and lengths at tile boundaries, at the short-message limit
    and at 0 between them; every message codes exactly."""
    kernel, enc_rows, dec_rows = mode
    rng = np.random.default_rng(77 + kernel + enc_rows)
    enc_tile, dec_tile = 384 * enc_rows, 512 * dec_rows
    cases = [
        np.array([257, 258, 259], dtype=np.int64),                      # 3 small tiles, most warps idle
        np.array([0, 0, 345, 0], dtype=np.int64),
        np.concatenate([rng.integers(0, 40, 5000), [3 << 20], rng.integers(0, 40, 5000)]),
        np.array([k * enc_tile + d for k in (1, 2, 3) for d in (-1, 0, 1)] * 7 + [0] * 5),
        np.array([k * dec_tile // 4 * 3 + d for k in (1, 2, 5) for d in (-2, -1, 0, 1, 2)] * 5),
    ]
    with kernel_choice(gb64, mode):
        for lens in cases:
            lens = lens.astype(np.int64)
            off = W.offsets_from_lengths(lens)
            data = W.uniform_bytes(int(off[-1]), int(lens.sum() % 1000) + 3)
            exp, exp_off = oracle.encode_batch(data, off)
            out, out_off = _encode(gb64, data, off, 0)
            assert np.array_equal(out_off, exp_off) and np.array_equal(out, exp), lens[:8]
            _check_decode(oracle, exp, exp_off, _decode(gb64, exp, exp_off, 0), 0)
