"""The scratch buffer that the whitespace-removing decode keeps per device:
calls of growing size reuse and grow it, b64_release_scratch frees it (the
next call allocates it again), calls on two streams that share it stay
exact, and a call captured into a CUDA graph (which takes its scratch from
the stream-ordered allocator instead) replays exactly."""
import base64

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SKIP_WS = 8


def _mime(n, seed, L=76, sep=b"\r\n"):
    rng = np.random.default_rng(seed)
    raw = rng.integers(0, 256, n, dtype=np.uint8)
    e = base64.b64encode(raw.tobytes())
    return raw, sep.join(e[i:i + L] for i in range(0, len(e), L)) + sep


def _sprinkled(n, seed):
    rng = np.random.default_rng(seed)
    raw = rng.integers(0, 256, n, dtype=np.uint8)
    e = base64.b64encode(raw.tobytes())
    cut = np.sort(rng.integers(0, len(e), max(1, len(e) // 50)))
    parts, last = [], 0
    for c in cut:
        parts.append(e[last:c])
        last = int(c)
    parts.append(e[last:])
    return raw, b" ".join(parts)


def _dev(s):
    import torch

    return torch.from_numpy(np.frombuffer(s, dtype=np.uint8).copy()).cuda()


def _decode_into(gb64, src, stream=None):
    import torch

    dst = torch.zeros(gb64.b64_decoded_cap_ex(src.numel(), SKIP_WS) + 16, dtype=torch.uint8,
                      device="cuda")
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    gb64.b64_decode_async_ex(src, dst, res, SKIP_WS, stream=stream)
    return dst, res


def test_grow_release_and_reuse(gb64):
    import torch

    for n, seed in ((1000, 1), (3 << 20, 2), (100, 3), (5 << 20, 4)):
        for make in (_mime, _sprinkled):
            raw, s = make(n, seed)
            dst, res = _decode_into(gb64, _dev(s))
            torch.cuda.synchronize()
            assert gb64.parse_result(res) == (0, n, len(s))
            assert np.array_equal(dst[:n].cpu().numpy(), raw)
        if seed % 2 == 0:
            gb64.b64_release_scratch()
    gb64.b64_release_scratch()
    gb64.b64_release_scratch()  # nothing kept: still fine


def test_two_streams_share_the_scratch(gb64):
    """Calls alternate between two streams with no host synchronisation in
    between; the kept scratch orders them, and every result is exact."""
    import torch

    inputs = [_mime(2 << 20, 10), _sprinkled(1 << 20, 11), _mime(600_000, 12, 64, b"\n"),
              _sprinkled(3 << 20, 13)]
    devs = [_dev(s) for _, s in inputs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    outs = []
    for rep in range(3):
        for i, src in enumerate(devs):
            st = streams[(i + rep) % 2]
            with torch.cuda.stream(st):
                outs.append((i, _decode_into(gb64, src, stream=st)))
    torch.cuda.synchronize()
    for i, (dst, res) in outs:
        raw, s = inputs[i]
        assert gb64.parse_result(res) == (0, raw.size, len(s)), i
        assert np.array_equal(dst[:raw.size].cpu().numpy(), raw), i


def test_captured_into_a_cuda_graph(gb64):
    import torch

    for make, seed in ((_mime, 20), (_sprinkled, 21)):
        raw, s = make(1 << 20, seed)
        src = _dev(s)
        dst = torch.zeros(gb64.b64_decoded_cap_ex(len(s), SKIP_WS) + 16, dtype=torch.uint8,
                          device="cuda")
        res = torch.zeros(3, dtype=torch.int64, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            gb64.b64_decode_async_ex(src, dst, res, SKIP_WS, stream=side)  # warm-up, uncaptured
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=side):
                gb64.b64_decode_async_ex(src, dst, res, SKIP_WS, stream=side)
        torch.cuda.synchronize()
        for _ in range(2):
            dst.zero_()
            res.zero_()
            graph.replay()
            torch.cuda.synchronize()
            assert gb64.parse_result(res) == (0, raw.size, len(s))
            assert np.array_equal(dst[:raw.size].cpu().numpy(), raw)
