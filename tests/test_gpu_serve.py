"""The serving engine: every request's result in a continuous-batching mix
equals the oracle's and equals the same request served alone; admission
keeps device memory within the budget; oversized requests are refused."""
import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pools(gb64, nbytes, seed):
    import torch

    raw = W.counter_bytes_torch(seed, 0, nbytes, device="cuda")
    enc = gb64.b64_encode(raw)
    return raw, enc


def _requests(gb64, n, seed, raw, enc, err_every=0):
    """(kind, device address, length, host payload) per request; decode
    payloads are quad-aligned slices of the encoded pool, some with a byte
    from outside the alphabet written in (kept in a side buffer)."""
    import torch

    rng = np.random.default_rng(seed)
    lens = W.lognormal_lengths(rng, n, 700.0, 2.0, 0, 1 << 20)
    kinds = (rng.random(n) < 0.5).astype(np.int32)
    pos = rng.random(n)
    reqs = []
    bad_chunks = []
    for i in range(n):
        L = int(lens[i])
        if kinds[i] == 0:
            off = int(pos[i] * (raw.numel() - L))
            reqs.append((0, raw[off:off + L]))
        else:
            m = 4 * -(-L // 3)
            q = int(pos[i] * ((enc.numel() - m) // 4))
            t = enc[4 * q:4 * q + m]
            if err_every and i % err_every == 0 and m > 0:
                t = t.clone()
                t[int(rng.integers(0, m))] = int(W.NON_ALPHABET_NON_PAD[rng.integers(0, 191)])
                bad_chunks.append(t)
            reqs.append((1, t))
    return reqs, bad_chunks


def _serve(gb64, server, reqs):
    ids = [server.submit(k, t) for k, t in reqs]
    out = {}
    while len(out) < len(ids):
        for c in server.poll(timeout_us=20000):
            data = None
            if c["status"] == 0 and c["outlen"] > 0:
                data = _copy_out(c["out"], c["outlen"])
            out[c["id"]] = (c["status"], c["first_bad"], c["outlen"], data, c["batch"])
            server.release(c["id"])
    return [out[i] for i in ids]


def _copy_out(addr, n):
    """Host copy of n bytes of a completion's device output."""
    from paper_1704_00605_gb300 import gb64

    return gb64.device_view(addr, n).cpu().numpy().copy()


def test_mix_equals_oracle_and_alone(gb64, oracle):
    raw, enc = _pools(gb64, 64 << 20, seed=41)
    reqs, _ = _requests(gb64, 3000, 1, raw, enc, err_every=37)
    with gb64.Server(memory_budget=1 << 30, streams=4, max_batch_msgs=512) as srv:
        mix = _serve(gb64, srv, reqs)
        st = srv.stats()
        assert st["batches"] > 1 and st["requests_done"] == len(reqs)
    nbatches = len({r[4] for r in mix})
    assert nbatches > 1
    for (kind, t), (status, fb, outlen, data, _) in zip(reqs, mix):
        h = t.cpu().numpy()
        if kind == 0:
            exp = oracle.encode(h)
            assert status == 0 and outlen == exp.size
            assert exp.size == 0 or np.array_equal(data, exp)
        else:
            ost, oout, ofb = oracle.decode(h)
            assert (status, fb) == (ost, ofb)
            if ost == 0:
                assert outlen == oout.size and (oout.size == 0 or np.array_equal(data, oout))
    # the same requests, each served alone, give the same bytes and status
    rng = np.random.default_rng(5)
    sample = rng.choice(len(reqs), 60, replace=False)
    with gb64.Server(memory_budget=1 << 30, streams=1, max_batch_msgs=1) as srv:
        for i in sample:
            (status, fb, outlen, data, _), = _serve(gb64, srv, [reqs[i]])
            m = mix[i]
            assert (status, fb, outlen) == m[:3]
            assert (data is None and m[3] is None) or np.array_equal(data, m[3])


def test_admission_stays_within_budget(gb64, oracle):
    raw, enc = _pools(gb64, 40 << 20, seed=42)
    budget = 48 << 20
    rng = np.random.default_rng(2)
    reqs = []
    for i in range(40):
        L = int(rng.integers(1, 6 << 20))
        off = int(rng.integers(0, raw.numel() - L))
        reqs.append((0, raw[off:off + L]))
    with gb64.Server(memory_budget=budget, streams=4, max_batch_msgs=8) as srv:
        res = _serve(gb64, srv, reqs)
        st = srv.stats()
        assert st["arena_high_water"] <= budget
        assert st["memory_waits"] > 0  # some batches had to wait for memory
        with pytest.raises(gb64.Gb64Error, match="budget"):
            srv.submit(0, raw[: 40 << 20])
        assert srv.stats()["rejected"] == 1
    for (kind, t), (status, fb, outlen, data, _) in zip(reqs[:5], res[:5]):
        assert np.array_equal(data, oracle.encode(t.cpu().numpy()))


def test_open_loop_replay(gb64):
    raw, enc = _pools(gb64, 64 << 20, seed=43)
    r = W.serving(duration_s=0.1, rate_hz=200_000.0, seed=4, max_len=1 << 20)
    n = r["t_arrival"].size
    kind = r["is_decode"].astype(np.int32)
    length = r["length"].astype(np.int64)
    src = np.empty(n, dtype=np.uint64)
    ln = np.empty(n, dtype=np.int64)
    for i in range(n):
        L = int(length[i])
        if kind[i] == 0:
            src[i] = raw.data_ptr() + int(r["pool_pos"][i] * (raw.numel() - L))
            ln[i] = L
        else:
            m = 4 * -(-L // 3)
            src[i] = enc.data_ptr() + 4 * int(r["pool_pos"][i] * ((enc.numel() - m) // 4))
            ln[i] = m
    with gb64.Server(memory_budget=8 << 30, streams=4, max_batch_msgs=4096,
                     auto_release=True) as srv:
        lat, st = srv.replay(r["t_arrival"] * 1e6, kind, src, ln)
        stats = srv.stats()
    assert (st == 0).all() and (lat >= 0).all()
    assert stats["requests_done"] == n and stats["batches"] >= 2
    assert np.percentile(lat, 50) < 50_000  # microseconds
