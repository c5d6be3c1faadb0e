"""The autotuner: it times every candidate shape, keeps the fastest for the
bucket, and every candidate shape it may pick codes bit-exactly (checked
against the oracle with the shape forced for its bucket)."""
import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def restore_shapes(gb64, tmp_path):
    path = str(tmp_path / "before.txt")
    gb64.b64_tune_save(path)
    yield
    gb64.b64_tune_load(path)


def _check_single(gb64, oracle, raw):
    import torch

    src = torch.from_numpy(raw).cuda()
    enc = gb64.b64_encode(src)
    exp = oracle.encode(raw)
    assert np.array_equal(enc.cpu().numpy(), exp)
    st, outlen, fb, dst = gb64.b64_decode(enc)
    assert (st, outlen, fb) == (0, raw.size, exp.size)
    assert torch.equal(dst[:outlen], src)
    bad = enc.clone()
    p = exp.size - 3 * exp.size // 7
    bad[p] = 0x2A
    st, outlen, fb, _ = gb64.b64_decode(bad)
    assert (st, fb) == (1, p)


@pytest.mark.parametrize("kind", [0, 1])
def test_tune_single_and_every_candidate_is_exact(gb64, oracle, restore_shapes, kind):
    size = 3 << 20  # the 1-16 MiB bucket
    trials = gb64.b64_tune(kind, size)
    assert len(trials) >= 20 and all(t["ms"] > 0 for t in trials)
    best = min(trials, key=lambda t: t["ms"])
    got = gb64.b64_shape_get(kind, size)
    assert (got["threads"], got["units_per_thread"], got["stages"], got["blocks_per_sm"]) == \
        (best["threads"], best["units_per_thread"], best["stages"], best["blocks_per_sm"])
    n = 3 * (1 << 20) // 4 * 3 + 7 if kind == 1 else (3 << 20) + 2
    raw = W.uniform_bytes(n, 40 + kind)
    bucket_size = n if kind == 0 else gb64.b64_encoded_len(n)
    for t in trials:
        gb64.b64_shape_set(kind, bucket_size, threads=t["threads"],
                           units_per_thread=t["units_per_thread"], stages=t["stages"],
                           blocks_per_sm=t["blocks_per_sm"])
        _check_single(gb64, oracle, raw)


def test_shape_that_does_not_fit_is_rejected(gb64, restore_shapes):
    with pytest.raises(gb64.Gb64Error, match="shared memory"):
        gb64.b64_shape_set(1, 1 << 30, threads=512, units_per_thread=8, stages=6)


@pytest.mark.parametrize("kind", [2, 3])
def test_tune_batch_and_every_candidate_is_exact(gb64, oracle, restore_shapes, kind):
    import torch

    data, off = W.batched(nmsg=1500, seed=50 + kind, median=1500.0)
    total, nmsg = int(off[-1]), off.size - 1
    trials = gb64.b64_tune(kind, total, nmsg)
    assert len(trials) >= 10 and all(t["ms"] > 0 for t in trials)
    exp_enc, exp_off = oracle.encode_batch(data, off)
    src, doff = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    # packed batch calls (offsets on the device: mean length unknown to the
    # host) take the shape of the unknown-size bucket: force it there
    fields = ("threads", "units_per_thread", "stages", "blocks_per_sm", "tile")
    saved = gb64.b64_shape_get(kind, -1, 1)
    try:
        for t in trials:
            gb64.b64_shape_set(kind, -1, 1, **{f: t[f] for f in fields})
            enc, eoff = gb64.b64_encode_batch(src, doff)
            assert np.array_equal(enc.cpu().numpy()[:exp_enc.size], exp_enc), t
            dst, out_off, st, fb, ol = gb64.b64_decode_batch(enc, eoff)
            assert int((st != 0).sum()) == 0, t
            assert torch.equal(ol.cpu(), torch.from_numpy(np.diff(off))), t
            assert all(np.array_equal(dst[out_off[j]:out_off[j] + ol[j]].cpu().numpy(),
                                      data[off[j]:off[j + 1]]) for j in range(0, nmsg, 97)), t
    finally:
        gb64.b64_shape_set(kind, -1, 1, **{f: saved[f] for f in fields})
