"""GPU parity of the batched codec against the CPU oracle (exact).

Each message's output, status, first_bad and outlen must equal the oracle's
for that message alone; batches include empty and 1-byte messages, messages
that straddle tiles, every length class mod 3 / mod 4, injected errors, and
the batched workloads at reduced and full message counts.
"""
import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def check_encode_batch(gb64, oracle, data, off):
    dst, out_off = gb64.b64_encode_batch(dev(data), dev(off))
    exp, exp_off = oracle.encode_batch(data, off)
    assert np.array_equal(out_off.cpu().numpy(), exp_off)
    assert np.array_equal(dst.cpu().numpy()[:exp.size], exp)
    return exp, exp_off


def check_decode_batch(gb64, oracle, chars, off):
    dst, out_off, st, fb, ol = gb64.b64_decode_batch(dev(chars), dev(off))
    edst, eoff, est, efb, eol = oracle.decode_batch(chars, off)
    assert np.array_equal(out_off.cpu().numpy(), eoff)
    st, fb, ol = st.cpu().numpy(), fb.cpu().numpy(), ol.cpu().numpy()
    bad = np.nonzero((st != est) | (fb != efb) | (ol != eol))[0]
    assert bad.size == 0, (bad[:5], st[bad[:5]], est[bad[:5]], fb[bad[:5]], efb[bad[:5]])
    h = dst.cpu().numpy()
    okm = np.nonzero(est == 0)[0]
    for j in okm:
        a, n = eoff[j], eol[j]
        if n:
            assert np.array_equal(h[a:a + n], edst[a:a + n]), j
    return est, efb


def test_small_mixed_batch(gb64, oracle):
    lens = np.array([0, 1, 2, 3, 4, 5, 0, 11, 12, 13, 47, 48, 49, 6143, 6144, 6145, 20000, 0, 1,
                     12289, 100000, 7], dtype=np.int64)
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), 9)
    enc, eoff = check_encode_batch(gb64, oracle, data, off)
    check_decode_batch(gb64, oracle, enc, eoff)


def test_empty_and_single_message_batches(gb64, oracle):
    import torch

    off = np.zeros(1, dtype=np.int64)
    dst, out_off = gb64.b64_encode_batch(dev(np.zeros(1, np.uint8)), dev(off))
    assert out_off.cpu().tolist() == [0]
    for n in [0, 1, 2, 3, 100, 65537]:
        off = np.array([0, n], dtype=np.int64)
        data = W.uniform_bytes(n, n)
        enc, eoff = check_encode_batch(gb64, oracle, data, off)
        check_decode_batch(gb64, oracle, enc, eoff)
    _ = torch


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_batches(gb64, oracle, seed):
    rng = np.random.default_rng(seed)
    nmsg = int(rng.integers(1, 3000))
    lens = W.lognormal_lengths(rng, nmsg, 300.0, 2.0, 0, 200_000)
    off = W.offsets_from_lengths(lens)
    data = W.uniform_bytes(int(off[-1]), seed)
    enc, eoff = check_encode_batch(gb64, oracle, data, off)
    check_decode_batch(gb64, oracle, enc, eoff)


def test_decode_batch_arbitrary_lengths_and_bytes(gb64, oracle):
    """Strings that are not encodings: random lengths (any mod 4) of mostly
    alphabet characters with random '=' and other bytes mixed in."""
    rng = np.random.default_rng(21)
    alpha = np.array([oracle.table1_char(v) for v in range(64)], dtype=np.uint8)
    nmsg = 4000
    lens = rng.integers(0, 300, nmsg)
    off = W.offsets_from_lengths(lens.astype(np.int64))
    chars = alpha[rng.integers(0, 64, int(off[-1]))]
    for j in range(nmsg):
        a, b = off[j], off[j + 1]
        r = rng.random()
        if b - a >= 2 and r < 0.2:
            chars[b - 2:b] = 0x3D
        elif b - a >= 1 and r < 0.4:
            chars[b - 1] = 0x3D
        elif b > a and r < 0.5:
            chars[int(rng.integers(a, b))] = int(rng.integers(0, 256))
    check_decode_batch(gb64, oracle, chars, off)


def test_workload_batched_reduced(gb64, oracle):
    data, off = W.batched(nmsg=5000, seed=2)
    enc, eoff = check_encode_batch(gb64, oracle, data, off)
    check_decode_batch(gb64, oracle, enc, eoff)


def test_workload_batched_full(gb64, oracle):
    """100,000 messages (seed 2) through the shapes the benchmark times:
    outputs equal the single-buffer calls on sampled messages and the oracle
    on sampled messages; the decode round trip is exact for all."""
    import torch

    data, off = W.batched()
    src, doff = dev(data), dev(off)
    enc, eoff = gb64.b64_encode_batch(src, doff)
    dst, out_off, st, fb, ol = gb64.b64_decode_batch(enc, eoff)
    assert int((st != 0).sum()) == 0
    lens = torch.diff(doff)
    assert torch.equal(ol, lens)
    eo = eoff.cpu().numpy()
    oo = out_off.cpu().numpy()
    rng = np.random.default_rng(0)
    for j in rng.integers(0, off.size - 1, 300):
        raw = data[off[j]:off[j + 1]]
        exp = oracle.encode(raw)
        assert np.array_equal(enc[eo[j]:eo[j + 1]].cpu().numpy(), exp)
        single = gb64.b64_encode(src[int(off[j]):int(off[j + 1])])
        assert np.array_equal(single.cpu().numpy(), exp)
        assert np.array_equal(dst[oo[j]:oo[j] + raw.size].cpu().numpy(), raw)
    # every decoded message equals its payload: compare packed views
    keep = torch.zeros(int(oo[-1]), dtype=torch.bool, device="cuda")
    starts = out_off[:-1]
    idx = torch.repeat_interleave(starts, lens) + (
        torch.arange(int(lens.sum()), device="cuda") -
        torch.repeat_interleave(doff[:-1], lens))
    keep[idx] = True
    assert torch.equal(dst[:int(oo[-1])][keep], src)


def test_workload_error_batch_reduced(gb64, oracle):
    """Config 4 recipe at 20,000 messages: per-message status and first_bad
    exactly as the oracle's."""
    rec = W.error_batch(nmsg=20_000, seed=3)
    off = rec["in_off"]
    payload = W.counter_bytes(rec["payload_key"], 0, int(off[-1]))
    enc, eoff = oracle.encode_batch(payload, off)
    genc, geoff = gb64.b64_encode_batch(dev(payload), dev(off))
    assert np.array_equal(genc.cpu().numpy(), enc)
    W.inject_errors(enc, eoff, rec["err_msg"], rec["err_frac"], rec["err_byte"])
    est, efb = check_decode_batch(gb64, oracle, enc, eoff)
    assert (est != 0).sum() == rec["err_msg"].size


def test_workload_error_batch_full(gb64, oracle):
    """Config 4 at full size: 1,000,000 messages of 16 B .. 64 KiB (about
    33 GB of payload, generated on the device from the counter-based
    stream), encoded and decoded in one launch per direction in the default
    shapes. Every message: status, first_bad and outlen exact (the 10,000
    injected errors at their known offsets, every other message OK with its
    length); sampled messages (with and without an error) against the oracle
    one by one; the round trip of every clean message is checked on the
    device."""
    import torch

    rec = W.error_batch(seed=3)
    off = rec["in_off"]
    nmsg = off.size - 1
    doff = dev(off)
    payload = W.counter_bytes_torch(rec["payload_key"], 0, int(off[-1]), device="cuda")
    enc, eoff = gb64.b64_encode_batch(payload, doff)
    eo = eoff.cpu().numpy()
    rng = np.random.default_rng(5)
    sample = np.concatenate([rng.integers(0, nmsg, 120), rec["err_msg"][:40]])
    for j in sample:  # encodings against the oracle before any error is written
        raw = W.counter_bytes(rec["payload_key"], int(off[j]), int(off[j + 1] - off[j]))
        assert np.array_equal(enc[eo[j]:eo[j + 1]].cpu().numpy(), oracle.encode(raw)), j
    pos = W.inject_errors(enc, eo, rec["err_msg"], rec["err_frac"], rec["err_byte"])
    dst, out_off, st, fb, ol = gb64.b64_decode_batch(enc, eoff)
    st, fb, ol = st.cpu().numpy(), fb.cpu().numpy(), ol.cpu().numpy()
    bad = np.zeros(nmsg, dtype=bool)
    bad[rec["err_msg"]] = True
    assert (st[~bad] == 0).all() and (ol[~bad] == np.diff(off)[~bad]).all()
    assert (fb[~bad] == np.diff(eo)[~bad]).all()
    assert (st[bad] == 1).all()  # an injected byte is never in the alphabet nor '='
    assert np.array_equal(fb[rec["err_msg"]], pos - eo[rec["err_msg"]])
    oo = out_off.cpu().numpy()
    for j in sample:  # decode results against the oracle
        m = enc[eo[j]:eo[j + 1]].cpu().numpy()
        est, eout, efb = oracle.decode(m)
        assert (st[j], fb[j]) == (est, efb), j
        if est == 0:
            assert np.array_equal(dst[oo[j]:oo[j] + ol[j]].cpu().numpy(), eout), j
    # every clean message decodes to its payload: gather the decoded bytes of
    # 20,000 messages at a time (at most ~1.3 GB of payload, 10 GB of int64
    # indices) and blank the messages with an error on both sides
    lens = torch.diff(doff)
    badd = torch.from_numpy(bad).cuda()
    step = 20_000
    for a in range(0, nmsg, step):
        b = min(nmsg, a + step)
        ln = lens[a:b]
        n = int(off[b] - off[a])
        idx = torch.repeat_interleave(out_off[a:b], ln) + (
            torch.arange(n, device="cuda") - torch.repeat_interleave(doff[a:b] - doff[a], ln))
        got = dst[idx]
        want = payload[int(off[a]):int(off[b])].clone()
        mask = torch.repeat_interleave(badd[a:b], ln)
        got[mask] = 0
        want[mask] = 0
        assert torch.equal(got, want), a
        del idx, got, want, mask


def test_batch_deterministic_and_stream_ordered(gb64, oracle):
    import torch

    data, off = W.batched(nmsg=3000, seed=7)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a, ao = gb64.b64_encode_batch(dev(data), dev(off), stream=s)
        b, bo = gb64.b64_encode_batch(dev(data), dev(off), stream=s)
    s.synchronize()
    assert torch.equal(a, b) and torch.equal(ao, bo)


def test_batch_calls_capture_into_a_cuda_graph(gb64, oracle):
    """The batched calls enqueue only stream-ordered work (kernels, the
    stream-ordered allocator), so they can be captured once and replayed:
    a replay after new data was written into the same buffers codes it."""
    import torch

    data, off = W.batched(nmsg=3000, seed=71, median=600.0)
    src, doff = dev(data), dev(off)
    eoff = gb64.b64_batch_out_offsets(False, doff)
    enc = torch.empty(int(eoff[-1].item()), dtype=torch.uint8, device="cuda")
    dec_off = gb64.b64_batch_out_offsets(True, eoff)
    dec = torch.empty(int(dec_off[-1].item()) + 16, dtype=torch.uint8, device="cuda")
    n = off.size - 1
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    fb = torch.empty(n, dtype=torch.int64, device="cuda")
    ol = torch.empty(n, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gb64.b64_encode_batch(src, doff, enc, eoff, stream=s)  # warm-up outside capture
        gb64.b64_decode_batch(enc, eoff, dec, dec_off, st, fb, ol, stream=s)
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            gb64.b64_encode_batch(src, doff, enc, eoff, stream=s)
            gb64.b64_decode_batch(enc, eoff, dec, dec_off, st, fb, ol, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for seed in (72, 73):
        new = W.uniform_bytes(data.size, seed)
        src.copy_(torch.from_numpy(new))
        enc.zero_()
        graph.replay()
        torch.cuda.synchronize()
        exp, exp_off = oracle.encode_batch(new, off)
        assert np.array_equal(enc.cpu().numpy(), exp)
        assert int((st != 0).sum()) == 0
        do = dec_off.cpu().numpy()
        h = dec.cpu().numpy()
        for j in range(0, n, 97):
            assert np.array_equal(h[do[j]:do[j] + off[j + 1] - off[j]], new[off[j]:off[j + 1]])
