"""Long messages (256 KiB to 3 MiB) in the batched codec, against the oracle,
exactly: lengths around 256 KiB and at multiples of 48 KiB and 64 Ki
characters (where the per-warp tiles and the staged copies split them),
long messages mixed with short and medium ones, every alignment of the
packed buffers, errors in their first and last tiles and in the final
group, the variant flags, a batch of 1 MiB messages round trip, and the
timeout path on a batch of long messages."""
import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu

URL, NOPAD, STRICT = 1, 2, 4
BIG = 256 << 10
ENC_CT, DEC_CT = 48 << 10, 64 << 10  # multiples of the tile sizes (input bytes / characters)


def _dev_at(a, shift):
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


def _long_lengths(rng, n_long, n_other):
    """Long messages at the threshold and at tile boundaries, between
    short and medium ones."""
    special = [BIG - 1, BIG, BIG + 1, BIG + 2, 6 * ENC_CT, 6 * ENC_CT + 1, 6 * ENC_CT - 383,
               4 * DEC_CT, 4 * DEC_CT + 3, 5 * DEC_CT - 512, (1 << 20), (1 << 20) + 2,
               3 * (1 << 20) + 5]
    longs = special + [int(x) for x in rng.integers(BIG, 2 << 20, max(0, n_long - len(special)))]
    others = [int(x) for x in rng.integers(0, 70_000, n_other)]
    lens = longs + others
    rng.shuffle(lens)
    return np.array(lens, dtype=np.int64)


def _encode(gb64, data, off, src_shift, dst_shift, flags=0):
    import torch

    out_off = torch.empty(off.size, dtype=torch.int64, device="cuda")
    gb64.b64_batch_out_offsets_ex(False, _off(off), flags, out_off)
    need = int(out_off[-1].item())
    buf = torch.zeros(need + 512, dtype=torch.uint8, device="cuda")
    base = (-buf.data_ptr()) % 256
    dst = buf[base + dst_shift:base + dst_shift + max(need, 1)]
    gb64.b64_encode_batch_ex(_dev_at(data, src_shift), _off(off), flags, dst=dst, out_off=out_off)
    return dst.cpu().numpy()[:need], out_off.cpu().numpy()


def _check_decode(gb64, oracle, chars, coff, shift, flags=0):
    dst, oo, st, fb, ol = gb64.b64_decode_batch_ex(_dev_at(chars, shift), _off(coff), flags)
    h, oo, st, fb, ol = (dst.cpu().numpy(), oo.cpu().numpy(), st.cpu().numpy(), fb.cpu().numpy(),
                         ol.cpu().numpy())
    for j in range(coff.size - 1):
        m = chars[coff[j]:coff[j + 1]]
        est, eout, efb = oracle.decode_ex(m, flags)
        assert (st[j], fb[j]) == (est, efb), (j, m.size, shift, flags, st[j], fb[j], est, efb)
        if est == 0:
            assert ol[j] == eout.size and np.array_equal(h[oo[j]:oo[j] + ol[j]], eout), (j, shift)


def test_encode_long_messages(gb64, oracle):
    rng = np.random.default_rng(61)
    lens = _long_lengths(rng, 16, 200)
    off = W.offsets_from_lengths(lens)
    data = W.counter_bytes(61, 0, int(off[-1]))
    exp, exp_off = oracle.encode_batch(data, off)
    for src_shift, dst_shift in ((0, 0), (5, 4), (3, 8), (1, 12), (7, 0)):
        out, out_off = _encode(gb64, data, off, src_shift, dst_shift)
        assert np.array_equal(out_off, exp_off)
        assert np.array_equal(out, exp), (src_shift, dst_shift)


@pytest.mark.parametrize("flags", [URL, NOPAD, URL | NOPAD])
def test_encode_long_messages_flags(gb64, oracle, flags):
    rng = np.random.default_rng(62 + flags)
    lens = _long_lengths(rng, 13, 60)
    off = W.offsets_from_lengths(lens)
    data = W.counter_bytes(62, 0, int(off[-1]))
    exp = np.concatenate([oracle.encode_ex(data[off[j]:off[j + 1]], flags)
                          for j in range(off.size - 1)])
    out, _ = _encode(gb64, data, off, 3, 4, flags)
    assert np.array_equal(out, exp)


def test_decode_long_messages_with_errors(gb64, oracle):
    from paper_1704_00605_gb300.workloads import NON_ALPHABET_NON_PAD

    rng = np.random.default_rng(63)
    lens = _long_lengths(rng, 20, 150)
    off = W.offsets_from_lengths(lens)
    data = W.counter_bytes(63, 0, int(off[-1]))
    chars, coff = oracle.encode_batch(data, off)
    chars = chars.copy()
    longs = [j for j in range(coff.size - 1) if coff[j + 1] - coff[j] >= BIG]
    assert len(longs) >= 15
    # errors in long messages: first tile, a tile boundary, the last 64 Ki
    # tile, the final group; and one in a few short ones
    for i, j in enumerate(longs[:12]):
        a, b = int(coff[j]), int(coff[j + 1])
        where = [a + 5, a + 8192 - 1, a + 8192, a + DEC_CT + 17, b - 1 - (b - a) % DEC_CT,
                 b - 2, b - 1, a + int(rng.integers(0, b - a))][i % 8]
        chars[where] = NON_ALPHABET_NON_PAD[int(rng.integers(0, NON_ALPHABET_NON_PAD.size))]
    for j in range(0, coff.size - 1, 23):
        if coff[j + 1] > coff[j] and coff[j + 1] - coff[j] < BIG:
            chars[int(rng.integers(coff[j], coff[j + 1]))] = ord("*")
    for shift in (0, 1, 4, 8, 13):
        _check_decode(gb64, oracle, chars, coff, shift)


@pytest.mark.parametrize("flags", [URL, NOPAD, STRICT, URL | NOPAD | STRICT])
def test_decode_long_messages_flags(gb64, oracle, flags):
    rng = np.random.default_rng(64 + flags)
    lens = _long_lengths(rng, 13, 40)
    off = W.offsets_from_lengths(lens)
    data = W.counter_bytes(64, 0, int(off[-1]))
    enc = [oracle.encode_ex(data[off[j]:off[j + 1]], flags & (URL | NOPAD))
           for j in range(off.size - 1)]
    coff = W.offsets_from_lengths(np.array([e.size for e in enc], dtype=np.int64))
    chars = np.concatenate(enc).copy()
    if flags & STRICT:  # noncanonical final groups in some long messages
        for j in range(0, coff.size - 1, 3):
            a, b = int(coff[j]), int(coff[j + 1])
            if b - a >= BIG:
                k = b - 1
                while chars[k] == ord("="):
                    k -= 1
                chars[k] ^= 1
    _check_decode(gb64, oracle, chars, coff, 4, flags)


def test_batch_of_long_messages_round_trip(gb64):
    """64 messages of 1 MiB (the sweep's batch): round trip on the device."""
    import torch

    n, L = 64, 1 << 20
    src = W.counter_bytes_torch(65, 0, n * L, device=torch.device("cuda"))
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda") * L
    enc, eoff = gb64.b64_encode_batch(src, off)
    dst, doff, st, fb, ol = gb64.b64_decode_batch(enc, eoff)
    assert int((st != 0).sum()) == 0 and bool((ol == L).all())
    do = doff.cpu().numpy()  # decode outputs sit at capacity offsets
    for j in range(n):
        assert torch.equal(dst[do[j]:do[j] + L], src[j * L:(j + 1) * L]), j


def test_long_messages_time_out_then_recover(gb64, oracle):
    import torch

    lens = np.array([BIG + 7, 100, 3 * BIG], dtype=np.int64)
    off = W.offsets_from_lengths(lens)
    data = W.counter_bytes(66, 0, int(off[-1]))
    src, doff = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    assert gb64.b64_device_fault() == 0
    gb64.b64_test_stall_copies(True, 2_000_000)
    try:
        gb64.b64_encode_batch(src, doff)
        assert gb64.b64_device_fault() == gb64.B64_ERR_TIMEOUT
    finally:
        gb64.b64_test_stall_copies(False, 0)
    benc, boff = gb64.b64_encode_batch(src, doff)
    exp, exp_off = oracle.encode_batch(data, off)
    assert np.array_equal(benc.cpu().numpy()[:exp.size], exp)
    assert gb64.b64_device_fault() == 0
