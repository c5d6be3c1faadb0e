"""The seeded input generators are deterministic and self-consistent."""
import numpy as np

from paper_1704_00605_gb300 import workloads as W


def test_uniform_bytes_deterministic():
    a = W.single_message(4096, seed=0)
    b = W.single_message(4096, seed=0)
    assert np.array_equal(a, b) and a.dtype == np.uint8
    assert not np.array_equal(a, W.single_message(4096, seed=1))


def test_counter_bytes_slices_agree():
    full = W.counter_bytes(3, 0, 10_000)
    for s, n in [(0, 1), (1, 7), (5, 100), (8, 8), (13, 4000), (9999, 1), (3, 0)]:
        assert np.array_equal(W.counter_bytes(3, s, n), full[s:s + n])


def test_counter_bytes_torch_matches_numpy():
    import torch

    for s, n in [(0, 1000), (3, 999), (17, 64), (1 << 33, 100)]:
        a = W.counter_bytes(5, s, n)
        b = W.counter_bytes_torch(5, s, n, device="cpu", chunk_words=37).numpy()
        assert np.array_equal(a, b), (s, n)
    assert W.counter_bytes_torch(5, 0, 0, device="cpu").numel() == 0
    _ = torch


def test_counter_bytes_look_uniform():
    b = W.counter_bytes(1, 0, 1 << 20)
    hist = np.bincount(b, minlength=256)
    assert hist.min() > 3500 and hist.max() < 4700


def test_batched_lengths_recipe():
    data, off = W.batched(nmsg=20000, seed=2)
    lens = np.diff(off)
    assert lens.min() >= 1 and lens.max() <= W.MIB
    assert 1700 < np.median(lens) < 2400
    frac = np.bincount(lens % 3, minlength=3) / lens.size
    assert np.all(np.abs(frac - 1 / 3) < 0.02)
    assert data.size == off[-1]


def test_error_batch_recipe():
    rec = W.error_batch(nmsg=10000, seed=3)
    lens = np.diff(rec["in_off"])
    assert lens.min() >= 16 and lens.max() <= 65536
    assert rec["err_msg"].size == 100 and np.unique(rec["err_msg"]).size == 100
    assert set(rec["err_byte"].tolist()) <= set(W.NON_ALPHABET_NON_PAD.tolist())
    assert 0x3D not in rec["err_byte"]


def test_error_positions_inside_messages():
    off = np.array([0, 8, 8, 20, 24], dtype=np.int64)
    pos = W.error_positions(off, np.array([0, 2, 3]), np.array([0.0, 0.999, 0.5]))
    assert pos.tolist() == [0, 19, 22]


def test_serving_recipe():
    r = W.serving(duration_s=0.05, rate_hz=200_000.0)
    n = r["t_arrival"].size
    assert 8000 < n < 12000
    assert np.all(np.diff(r["t_arrival"]) >= 0)
    assert r["length"].min() >= 1 and r["length"].max() <= 1 << 24
    assert 0.45 < r["is_decode"].mean() < 0.55
