"""b64_decode_batch_noalloc (the batched decode for callers that cannot
allocate device memory during the call) gives exactly the results of
b64_decode_batch and of the CPU oracle, on two calls in a row that share its
fixed scratch, and on a batch of the largest size it accepts.

Kept in a file of its own that pytest collects last; it loads the library
itself, so it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_00605_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.b64_decode_batch_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _batch(gb64, seed, nmsg, nerr, median=900.0, sigma=1.5, max_len=1 << 20):
    import torch

    data, off = W.batched(nmsg=nmsg, seed=seed, median=median, sigma=sigma, max_len=max_len)
    enc, eoff = gb64.b64_encode_batch(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda())
    enc_h = enc.cpu().numpy().copy()
    eo = eoff.cpu().numpy()
    rng = np.random.default_rng(seed)
    err_msg = np.sort(rng.choice(nmsg, nerr, replace=False))
    W.inject_errors(enc_h, eo, err_msg, rng.random(nerr), W.NON_ALPHABET_NON_PAD[
        rng.integers(0, 191, nerr)])
    return torch.from_numpy(enc_h).cuda(), eoff


def _run_and_compare(gb64, oracle, f, chars, eoff, nmsg, nerr, call):
    import torch

    ref = gb64.b64_decode_batch(chars, eoff)
    cap = int(ref[1][-1].item())
    dst = torch.zeros(max(cap, 1), dtype=torch.uint8, device="cuda")
    out_off = torch.full((nmsg + 1,), -1, dtype=torch.int64, device="cuda")
    status = torch.full((nmsg,), 99, dtype=torch.int32, device="cuda")
    first_bad = torch.full((nmsg,), -1, dtype=torch.int64, device="cuda")
    outlen = torch.full((nmsg,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = f(chars.data_ptr(), eoff.data_ptr(), nmsg, dst.data_ptr(), out_off.data_ptr(),
           status.data_ptr(), first_bad.data_ptr(), outlen.data_ptr(),
           ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, gb64.b64_last_error()
    torch.cuda.synchronize()
    rdst, roff, rst, rfb, rol = ref
    assert torch.equal(out_off, roff), call
    assert torch.equal(status, rst), call
    assert torch.equal(first_bad, rfb), call
    assert torch.equal(outlen, rol), call
    assert int((rst != 0).sum()) == nerr
    # and against the oracle, message by message
    odst, odoff, ost, ofb, ool = oracle.decode_batch(chars.cpu().numpy(), eoff.cpu().numpy())
    assert np.array_equal(out_off.cpu().numpy(), odoff), call
    assert np.array_equal(status.cpu().numpy(), ost), call
    assert np.array_equal(first_bad.cpu().numpy(), ofb), call
    assert np.array_equal(outlen.cpu().numpy(), ool), call
    ro, rl, rs = roff.cpu().numpy(), rol.cpu().numpy(), rst.cpu().numpy()
    a, b = dst.cpu().numpy(), rdst.cpu().numpy()
    for j in np.nonzero(rs == 0)[0]:
        assert np.array_equal(a[ro[j]:ro[j] + rl[j]], b[ro[j]:ro[j] + rl[j]]), (call, j)
        assert np.array_equal(a[ro[j]:ro[j] + rl[j]], odst[odoff[j]:odoff[j] + ool[j]]), (call, j)


def test_noalloc_matches_decode_batch_on_two_calls(gb64, oracle):
    f = _noalloc(gb64.lib())
    for call, (seed, nmsg) in enumerate([(31, 5000), (32, 1700)]):
        chars, eoff = _batch(gb64, seed, nmsg, nerr=nmsg // 50)
        _run_and_compare(gb64, oracle, f, chars, eoff, nmsg, nmsg // 50, call)


def test_noalloc_at_its_message_limit(gb64, oracle):
    """65,536 messages, the most one call accepts (the largest scratch):
    short ones, so that both the one-thread-per-message pass and the tiles
    run."""
    f = _noalloc(gb64.lib())
    nmsg = 65536
    chars, eoff = _batch(gb64, 33, nmsg, nerr=nmsg // 100, median=200.0, sigma=1.0,
                         max_len=20_000)
    _run_and_compare(gb64, oracle, f, chars, eoff, nmsg, nmsg // 100, "limit")


def test_noalloc_rejects_batches_over_its_limit(gb64):
    import torch

    f = _noalloc(gb64.lib())
    nmsg = 65537
    off = torch.zeros(nmsg + 1, dtype=torch.int64, device="cuda")
    res = torch.zeros(nmsg + 1, dtype=torch.int64, device="cuda")
    st = torch.zeros(nmsg, dtype=torch.int32, device="cuda")
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = f(buf.data_ptr(), off.data_ptr(), nmsg, buf.data_ptr(), res.data_ptr(), st.data_ptr(),
           res.data_ptr(), res.data_ptr(), None)
    assert rc == gb64.B64_ERR_ARG
    assert "65536" in gb64.b64_last_error()
