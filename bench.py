#!/usr/bin/env python
"""Benchmark of the base64 codec on a GB300 (one JSON line on rank 0).

A step is one pass of the whole hot path over the 1 GiB workload: encode a
buffer of uniform random bytes (seed 1) and decode the encoding. Steps
rotate over the three lengths 2^30, 2^30+1, 2^30+2 so every padding case
("==", "=", none) is timed. Inputs (>= 1 GiB) are larger than the 129 MB L2,
so no flush is needed between steps.

  value      enc+dec input GB/s: (n + m) bytes per step / device time, all ranks
  roofline   the dominant kernel's algorithmic bytes (read + write) per launch
             / its CUDA-event duration, against the measured HBM copy peak
  e2e        the same metric through b64_encode_host / b64_decode_host on
             pinned host buffers (host<->device copies inside the timing)
  cpu_baseline  the CPU oracle on a bounded prefix of the workload, all cores,
             and on one core for the 1 MiB message and a 24 MiB prefix

The same line also carries (unless --no-extras): `batched` (the 100,000
log-normal messages, one launch per direction against one per message),
`whitespace` (Appendix B's removal on 367 MB of MIME lines), `sweep` (Fig.
10's length sweep 16 B .. 256 MiB, single calls and 256 MiB batches,
checked against the oracle), `config1_1mib` (the 1 MiB message's amortised
rate) and `serve` (200k requests/s Poisson for 30 s).

--impl reference times the CPU oracle itself (the reference arm of this
build): it has no GPU code; under torchrun only rank 0 runs it.
--config batched runs the 100,000-message workload: one batched launch per
direction against one launch per message.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GIB = 1 << 30
FALLBACK_HBM_GBS = 6800.0


# ------------------------------------------------------------------ setup
def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1200)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", choices=["large", "batched", "serve", "sweep", "variants",
                                        "whitespace"],
                   default="large")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the batched and serving sub-measurements of the default line")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--serve-seconds", type=float, default=30.0,
                   help="length of the serving replay in the default line (config 5: 30 s)")
    p.add_argument("--small", action="store_true",
                   help="384 MiB instead of 1 GiB (profiling captures; same launch shapes as "
                        "1 GiB); not a bench value")
    p.add_argument("--no-plain", action="store_true",
                   help="with --config batched: the 100,000-message batched calls only, without "
                        "the one-launch-per-message comparison (profiling captures)")
    p.add_argument("--tiny", action="store_true",
                   help="with --config batched --small: 1,000,000 messages of about 40 bytes "
                        "(one thread each); a profiling case")
    return p.parse_args(argv)


class Dist:
    """Rank bookkeeping; torch.distributed only for barrier and max/sum."""

    def __init__(self, backend=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False
        if self.world > 1:
            import datetime

            import torch.distributed as dist

            if backend is None:
                import torch

                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend, timeout=datetime.timedelta(seconds=600))
            self.pg = True
            self.backend = backend

    def barrier(self):
        if self.pg:
            import torch.distributed as dist

            dist.barrier()

    def reduce(self, x: float, op: str) -> float:
        if not self.pg:
            return x
        import torch
        import torch.distributed as dist

        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            import torch.distributed as dist

            dist.destroy_process_group()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.path = None
        self.uuid = None
        try:
            import torch

            self.uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            if self.uuid and not self.uuid.startswith("GPU-"):
                self.uuid = "GPU-" + self.uuid
        except Exception:
            self.uuid = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd[1:1] = ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------- CPU oracle timing
def oracle_throughput(data: np.ndarray, sample_bytes: int, threads: int):
    """Encode a prefix of ``sample_bytes`` (multiple of 3) and decode its
    encoding with the CPU oracle, split in aligned chunks over ``threads``
    threads. Returns (input GB/s of encode+decode, seconds)."""
    import oracle

    oracle.build()
    sample = np.ascontiguousarray(data[:sample_bytes])
    per = (sample_bytes // threads) // 3 * 3
    cuts = [i * per for i in range(threads)] + [sample_bytes]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        encs = list(ex.map(lambda i: oracle.encode(sample[cuts[i]:cuts[i + 1]]), range(threads)))
        decs = list(ex.map(lambda e: oracle.decode(e), encs))
    dt = time.perf_counter() - t0
    assert all(d[0] == 0 for d in decs)
    moved = sample_bytes + sum(e.size for e in encs)
    return moved / dt / 1e9, dt


def traffic_from_profile(kernel_tag: str, src_hash: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic_1gib.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != src_hash:
            return None
        return float(kv[f"{kernel_tag}_dram_bytes_per_launch"])
    except Exception:
        return None


def kernel_source_hash() -> str:
    """Hash of the sources that define the single-buffer kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1704_00605_gb300", "csrc")
    for name in ("common.cuh", "single.cu"):
        h.update(name.encode())
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()


# ------------------------------------------------------------ our codec
def run_large(args, d: Dist):
    import torch

    import paper_1704_00605_gb300 as pkg
    from paper_1704_00605_gb300 import workloads as W

    torch.cuda.set_device(d.local_rank)
    pkg.build.ensure_built()
    g = pkg.load()
    dev = torch.device("cuda", d.local_rank)
    base = (384 << 20) if args.small else GIB
    lengths = (base, base + 1, base + 2)
    data = W.uniform_bytes(base + 2, 1)  # the 1 GiB workload's stream (prefix when --small)
    src_all = torch.from_numpy(data).to(dev)
    m_max = g.b64_encoded_len(base + 2)
    enc = torch.empty(m_max, dtype=torch.uint8, device=dev)
    dec = torch.empty(g.b64_decoded_cap(m_max), dtype=torch.uint8, device=dev)
    res = torch.empty(3, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(i, evs=None):
        n = lengths[i % 3]
        if evs is not None:
            evs[0].record(stream)
        g.b64_encode(src_all[:n], enc)
        if evs is not None:
            evs[1].record(stream)
        m = g.b64_encoded_len(n)
        g.b64_decode_async(enc[:m], dec, res)
        if evs is not None:
            evs[2].record(stream)
        return n, m

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    # correctness of the path being timed (full round trip, all three lengths)
    for i in range(3):
        n, m = step(i)
        st, outlen, fb = g.parse_result(res)
        assert (st, outlen, fb) == (0, n, m), (st, outlen, fb)
        assert torch.equal(dec[:n], src_all[:n])

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(d.local_rank)
    d.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start.record(stream)
    moved_in = 0
    for i in range(args.steps):
        n, m = step(i, evs[i])
        moved_in += n + m
    t_end.record(stream)
    torch.cuda.synchronize()
    d.barrier()
    clk = clocks.stop()
    st, outlen, fb = g.parse_result(res)
    n_last = lengths[(args.steps - 1) % 3]
    assert (st, outlen) == (0, n_last), (st, outlen)

    total_ms = t_start.elapsed_time(t_end)
    enc_ms = [e[0].elapsed_time(e[1]) for e in evs]
    dec_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms_max = d.reduce(total_ms, "max")
    moved_all = d.reduce(float(moved_in), "sum")
    value = moved_all / (total_ms_max / 1e3) / 1e9

    peak, peak_kind = measured_peaks()
    alg_enc = [lengths[i % 3] + g.b64_encoded_len(lengths[i % 3]) for i in range(args.steps)]
    alg_dec = alg_enc  # decode reads m characters and writes n bytes
    enc_gbs = sum(alg_enc) / (sum(enc_ms) / 1e3) / 1e9
    dec_gbs = sum(alg_dec) / (sum(dec_ms) / 1e3) / 1e9
    dominant = "decode" if sum(dec_ms) >= sum(enc_ms) else "encode"
    dom_gbs = dec_gbs if dominant == "decode" else enc_gbs
    src_hash = kernel_source_hash()
    traffic = traffic_from_profile(dominant, src_hash)

    line = {
        "metric": "enc+dec input GB/s (1 GiB buffer, encode then decode)",
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": d.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms_max / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic: uniform random bytes, numpy default_rng(1), 2^30+2 bytes",
        "config": {"workload": ("single large buffer: 1 GiB (+1, +2) encode + decode (config 2)"
                                if not args.small else "384 MiB profiling case (not a bench value)"),
                   "lengths": list(lengths), "encoded_chars": g.b64_encoded_len(base),
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{d.world}",
                   "cpu_baseline_sample": "96 MiB prefix of this workload on all host cores; one "
                                          "core on the 1 MiB single message and a 24 MiB prefix",
                   "reference_arm_sample": "24 MiB prefix of this workload per step, all host "
                                           "cores (bench.py --impl reference)"},
        "roofline": {"bound": "hbm", "kernel": f"k_{dominant}_tma", "achieved": round(dom_gbs, 1),
                     "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs (copy, read+write)",
                     "unit": "GB/s", "frac": round(dom_gbs / peak, 4), "traffic": traffic},
        "encode": {"ms_per_launch": round(float(np.mean(enc_ms)), 4),
                   "input_gbs": round(sum(lengths[i % 3] for i in range(args.steps)) /
                                      (sum(enc_ms) / 1e3) / 1e9, 1),
                   "hbm_gbs": round(enc_gbs, 1), "hbm_frac": round(enc_gbs / peak, 4)},
        "decode": {"ms_per_launch": round(float(np.mean(dec_ms)), 4),
                   "input_gbs": round(sum(g.b64_encoded_len(lengths[i % 3])
                                          for i in range(args.steps)) /
                                      (sum(dec_ms) / 1e3) / 1e9, 1),
                   "hbm_gbs": round(dec_gbs, 1), "hbm_frac": round(dec_gbs / peak, 4)},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }

    if not args.no_e2e and not args.small:
        line["e2e"] = run_e2e(g, data, d)
    if d.rank == 0 and d.world == 1 and not args.no_cpu and not args.small:
        line["cpu_baseline"] = run_cpu_baseline(data)
    return line


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def run_cpu_baseline(data: np.ndarray):
    """The CPU oracle on the host cores: all cores on a 96 MiB prefix of the
    1 GiB workload (the line's value), and one core on the 1 MiB single
    message (config 1, seed 0) and on a 24 MiB prefix of the 1 GiB workload
    (config 2), each the median of 5 runs of encode + decode of the
    encoding."""
    import oracle
    from paper_1704_00605_gb300 import workloads as W

    oracle.build()
    threads = os.cpu_count() or 1
    sample = 96 << 20
    v, dt = oracle_throughput(data, sample, threads)

    def one_core(buf):
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            e = oracle.encode(buf)
            st, out, fb = oracle.decode(e)
            ts.append(time.perf_counter() - t0)
            assert st == 0 and out.size == buf.size
        return (buf.size + e.size) / float(np.median(ts)) / 1e9

    cfg1 = W.single_message(1 << 20, 0)
    cfg2 = np.ascontiguousarray(data[:24 << 20])
    return {"value": round(v, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"first {sample} bytes of the 1 GiB workload: encode, then decode of its "
                      f"encoding; {threads} threads over 3-/4-aligned chunks; {dt:.2f} s wall",
            "single_thread_gbs": {"config1_1mib": round(one_core(cfg1), 4),
                                  "config2_24mib_prefix": round(one_core(cfg2), 4)},
            "unit_note": "input bytes + encoded characters per second (encode + decode)"}


def run_e2e(g, data, d: Dist):
    """Host-buffer round trip through the C ABI (pinned memory)."""
    import torch

    lengths = (GIB, GIB + 1, GIB + 2)
    h_src = torch.empty(GIB + 2, dtype=torch.uint8, pin_memory=True)
    h_src.numpy()[:] = data
    m_max = g.b64_encoded_len(GIB + 2)
    h_enc = torch.empty(m_max, dtype=torch.uint8, pin_memory=True)
    h_dec = torch.empty(g.b64_decoded_cap(m_max), dtype=torch.uint8, pin_memory=True)
    src_np, enc_np, dec_np = h_src.numpy(), h_enc.numpy(), h_dec.numpy()

    def step(i):
        n = lengths[i % 3]
        m = len(g.b64_encode_host(src_np[:n], enc_np))
        st, outlen, fb, _ = g.b64_decode_host(enc_np[:m], dec_np)
        assert st == 0 and outlen == n
        return n, m

    step(0)
    assert np.array_equal(dec_np[:GIB], data[:GIB])
    # the host link's own rate right now (pinned torch copies of 1 GiB), from
    # and into each host buffer the round trip uses: the pages behind one
    # pinned buffer have been seen to take device-to-host writes at a
    # quarter of the rate of another's on the same box
    dbuf = torch.empty(GIB, dtype=torch.uint8, device="cuda")
    link = {}
    # (the best of five single copies: one copy has been seen to run at
    # under half the rate of the next from the same buffer)
    for name, fn in (("h2d", lambda: dbuf.copy_(h_src[:GIB], non_blocking=True)),
                     ("d2h", lambda: h_dec[:GIB].copy_(dbuf, non_blocking=True)),
                     ("h2d_from_encoded", lambda: dbuf.copy_(h_enc[:GIB], non_blocking=True)),
                     ("d2h_into_encoded", lambda: h_enc[:GIB].copy_(dbuf, non_blocking=True))):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(5):
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t)
        link[name] = round(GIB / best / 1e9, 1)
    # both directions at once (two streams): the combined rate of the link
    dbuf2 = torch.empty(GIB, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def both():
        with torch.cuda.stream(s1):
            dbuf.copy_(h_src[:GIB], non_blocking=True)
        with torch.cuda.stream(s2):
            h_dec[:GIB].copy_(dbuf2, non_blocking=True)

    both()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(5):
        t = time.perf_counter()
        both()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
    link["both_directions_total"] = round(2 * GIB / best / 1e9, 1)
    del dbuf, dbuf2
    k = 6
    d.barrier()
    t0 = time.perf_counter()
    moved = 0
    hb = 0
    t_enc = t_dec = 0.0
    for i in range(k):
        n = lengths[i % 3]
        ta = time.perf_counter()
        m = len(g.b64_encode_host(src_np[:n], enc_np))
        tb = time.perf_counter()
        st, outlen, fb, _ = g.b64_decode_host(enc_np[:m], dec_np)
        t_enc += tb - ta
        t_dec += time.perf_counter() - tb
        assert st == 0 and outlen == n
        moved += n + m
        hb += n + m
    dt = time.perf_counter() - t0
    # the bound the host link sets on one step, with copies in both
    # directions overlapped: the encode moves n bytes in and m out, the
    # decode m in and n out, each at the rate measured from and into its
    # own host buffers
    # (and at most the combined rate of both directions at once)
    bound_ms = 0.0
    both = link["both_directions_total"]
    for i in range(k):
        n = lengths[i % 3]
        m = g.b64_encoded_len(n)
        bound_ms += max(n / link["h2d"], m / link["d2h_into_encoded"], (n + m) / both) / 1e6
        bound_ms += max(m / link["h2d_from_encoded"], n / link["d2h"], (n + m) / both) / 1e6
    step_ms = dt / k * 1e3
    dt = d.reduce(dt, "max")
    moved = d.reduce(float(moved), "sum")
    return {"value": round(moved / dt / 1e9, 2), "unit": "GB/s",
            "link_bound_ms_per_step": round(bound_ms / k, 3), "ms_per_step": round(step_ms, 3),
            "frac_of_link_bound": round(bound_ms / k / step_ms, 4),
            "h2d_bytes_per_step": int(hb // k), "d2h_bytes_per_step": int(hb // k),
            "steps": k, "api": "b64_encode_host + b64_decode_host (pinned host buffers)",
            "encode_host_ms": round(t_enc / k * 1e3, 2), "decode_host_ms": round(t_dec / k * 1e3, 2),
            "link_copy_gbs": link}


# ------------------------------------------------------ batched workload
def run_batched(args, d: Dist, steps: int = 20, plain_msgs: int = 20_000, nmsg_override=None,
                lengths=None):
    """Config 3: 100,000 packed messages (seed 2). Batched: one launch per
    direction (b64_encode_batch + b64_decode_batch), direct and replayed from
    a CUDA graph. Plain: one b64_encode + one b64_decode_async per message,
    through the C ABI in a host loop and captured in a CUDA graph, on the
    first ``plain_msgs`` messages (a rate, so a prefix suffices). Outputs of
    the two forms are compared byte for byte on that prefix."""
    import torch

    import paper_1704_00605_gb300 as pkg
    from paper_1704_00605_gb300 import workloads as W

    torch.cuda.set_device(d.local_rank)
    g = pkg.load()
    dev = torch.device("cuda", d.local_rank)
    kw = {} if nmsg_override is None else {"nmsg": nmsg_override}
    if lengths is not None:  # (median, sigma, max_len) of the log-normal lengths
        kw.update(median=lengths[0], sigma=lengths[1], max_len=lengths[2])
    data, off = W.batched(**kw)
    nmsg = off.size - 1
    src = torch.from_numpy(data).to(dev)
    doff = torch.from_numpy(off).to(dev)
    eoff = g.b64_batch_out_offsets(False, doff)
    enc = torch.empty(int(eoff[-1].item()), dtype=torch.uint8, device=dev)
    dec_off = g.b64_batch_out_offsets(True, eoff)  # decode outputs sit at capacity offsets
    dec = torch.empty(int(dec_off[-1].item()) + 16, dtype=torch.uint8, device=dev)
    st = torch.empty(nmsg, dtype=torch.int32, device=dev)
    fb = torch.empty(nmsg, dtype=torch.int64, device=dev)
    ol = torch.empty(nmsg, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def batched_step():
        g.b64_encode_batch(src, doff, enc, eoff)
        g.b64_decode_batch(enc, eoff, dec, dec_off, st, fb, ol)

    def timed(fn, k):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    batched_ms = timed(batched_step, steps)
    assert int((st != 0).sum()) == 0 and torch.equal(ol, torch.diff(doff))
    graph = torch.cuda.CUDAGraph()
    s2 = torch.cuda.Stream(dev)
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        batched_step()  # warm the allocator pool on the capture stream
        s2.synchronize()
        with torch.cuda.graph(graph, stream=s2):
            batched_step()
    stream.wait_stream(s2)
    graph_ms = timed(graph.replay, steps)

    if plain_msgs == 0:  # profiling case: the batched calls only
        return {"nmsg": nmsg, "batched_ms_per_step": round(batched_ms, 4),
                "batched_msgs_per_s": round(2 * nmsg / (batched_ms / 1e3), 1)}
    # plain: one launch per message on the prefix
    k = min(plain_msgs, nmsg)
    o = off[:k + 1]
    eo = eoff[:k + 1].cpu().numpy()
    penc = torch.empty(int(eo[-1]), dtype=torch.uint8, device=dev)
    pdo = np.concatenate([[0], np.cumsum(3 * (np.diff(eo) // 4))])
    pdec = torch.empty(int(pdo[-1]) + 16, dtype=torch.uint8, device=dev)
    pres = torch.empty((k, 3), dtype=torch.int64, device=dev)
    views = [(src[o[j]:o[j + 1]], penc[eo[j]:eo[j + 1]], pdec[pdo[j]:pdo[j + 1]], pres[j])
             for j in range(k)]

    def plain_step():
        for s_, e_, d_, r_ in views:
            g.b64_encode(s_, e_)
            g.b64_decode_async(e_, d_, r_)

    t0 = time.perf_counter()
    plain_step()
    torch.cuda.synchronize()
    plain_loop_ms = (time.perf_counter() - t0) * 1e3
    assert torch.equal(penc, enc[:int(eo[-1])])
    assert int((pres[:, 2] & 0xFFFFFFFF).sum()) == 0
    pgraph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s2):
        plain_step()
        s2.synchronize()
        with torch.cuda.graph(pgraph, stream=s2):
            plain_step()
    stream.wait_stream(s2)
    plain_graph_ms = timed(pgraph.replay, 3)
    assert torch.equal(penc, enc[:int(eo[-1])])
    pol = pres[:, 1].cpu().numpy()
    assert np.array_equal(pol, np.diff(o))
    for j in range(0, k, max(1, k // 200)):  # plain decode output equals the payload
        assert torch.equal(pdec[pdo[j]:pdo[j] + pol[j]], src[o[j]:o[j + 1]])

    msgs = 2 * nmsg  # one encode and one decode per message
    moved = float(data.size + enc.numel())
    # algorithmic bytes of a step: each direction reads its input and writes
    # its output once; the metadata adds, per message, the offsets read and
    # written by each direction (16 B each) and the decode's status,
    # first_bad and outlen (20 B)
    alg = 2.0 * moved
    meta = 52.0 * nmsg
    peak, peak_kind = measured_peaks()
    alg_gbs = alg / (batched_ms / 1e3) / 1e9
    return {
        "nmsg": nmsg, "bytes": int(data.size), "encoded": int(enc.numel()),
        "batched_ms_per_step": round(batched_ms, 4),
        "batched_msgs_per_s": round(msgs / (batched_ms / 1e3), 1),
        "batched_graph_msgs_per_s": round(msgs / (graph_ms / 1e3), 1),
        "batched_input_gbs": round(moved / (batched_ms / 1e3) / 1e9, 1),
        "hbm_gbs": round(alg_gbs, 1), "frac": round(alg_gbs / peak, 4),
        "frac_with_metadata": round((alg + meta) / (batched_ms / 1e3) / 1e9 / peak, 4),
        "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs",
        "plain_msgs_measured": k,
        "plain_loop_msgs_per_s": round(2 * k / (plain_loop_ms / 1e3), 1),
        "plain_graph_msgs_per_s": round(2 * k / (plain_graph_ms / 1e3), 1),
        "speedup_vs_plain_graph": round((msgs / batched_ms) / (2 * k / plain_graph_ms), 1),
        # encode: the scan kernel and the staged tile walk; decode: the
        # scan kernel, the flat decode, the tile walk (which returns at once
        # after a flat batch) and the finish kernel
        "gpu_launches_per_batched_step": BATCHED_LAUNCHES,
    }


BATCHED_LAUNCHES = 6  # kernels of one batched encode + decode step


def batched_line(args, d: Dist):
    if args.small and args.tiny:  # 1,000,000 short messages, batched calls only
        b = run_batched(args, d, steps=max(args.steps, 5), plain_msgs=0, nmsg_override=1_000_000,
                        lengths=(40.0, 0.3, 64))
        return {"metric": "batched msgs/s (profiling case, not a bench value)",
                "value": b["batched_msgs_per_s"], "unit": "msgs/s", "batched": b}
    if args.no_plain:  # the 100,000 messages, batched calls only (profiling captures)
        b = run_batched(args, d, steps=max(args.steps, 5), plain_msgs=0)
        return {"metric": "batched msgs/s (profiling case, not a bench value)",
                "value": b["batched_msgs_per_s"], "unit": "msgs/s", "batched": b}
    if args.small:  # 20,000 messages, batched calls only (profiling captures)
        b = run_batched(args, d, steps=max(args.steps, 5), plain_msgs=0, nmsg_override=20_000)
        return {"metric": "batched msgs/s (profiling case, not a bench value)",
                "value": b["batched_msgs_per_s"], "unit": "msgs/s", "batched": b}
    b = run_batched(args, d, steps=max(args.steps, 5))
    return {
        "metric": "batched encode+decode msgs/s (100,000 messages, one launch per direction)",
        "value": b["batched_msgs_per_s"], "unit": "msgs/s", "n_gpus": d.world,
        "steps": max(args.steps, 5), "warmup": 3, "ms_per_step": b["batched_ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic: log-normal lengths (median 2 KiB, sigma 1.5), uniform bytes, seed 2",
        "config": {"workload": "batched encode+decode: 100,000 messages (config 3)",
                   "l2": "600 MiB of input > L2 (no flush)"},
        "batched": b, "gpu_launches": BATCHED_LAUNCHES * max(args.steps, 5),
    }


# ------------------------------------------------------ serving workload
def run_serve(args, d: Dist, duration_s: float):
    """Config 5: Poisson arrivals at 200k requests/s, 50/50 encode/decode,
    log-normal payloads (median 4 KiB, sigma 2, clipped to 1 B..16 MiB),
    seed 4, replayed open-loop by native threads against the continuous
    batching server with an 8 GiB memory budget. Payloads live in resident
    device pools: a 1 GiB byte pool and its encoding (decode requests are
    quad-aligned slices of it, 4*ceil(len/3) characters)."""
    import torch

    import paper_1704_00605_gb300 as pkg
    from paper_1704_00605_gb300 import workloads as W

    torch.cuda.set_device(d.local_rank)
    g = pkg.load()
    raw = W.counter_bytes_torch(4, 0, GIB, device=torch.device("cuda", d.local_rank))
    enc = g.b64_encode(raw)
    r = W.serving(duration_s=duration_s, rate_hz=200_000.0, seed=4)
    n = r["t_arrival"].size
    kind = r["is_decode"].astype(np.int32)
    length = r["length"].astype(np.int64)
    m = 4 * ((length + 2) // 3)
    enc_pos = 4 * np.floor(r["pool_pos"] * ((enc.numel() - m) // 4)).astype(np.int64)
    raw_pos = np.floor(r["pool_pos"] * (raw.numel() - length)).astype(np.int64)
    src = np.where(kind == 1, enc.data_ptr() + enc_pos, raw.data_ptr() + raw_pos).astype(np.uint64)
    ln = np.where(kind == 1, m, length)
    with g.Server(memory_budget=8 << 30, streams=4, max_batch_msgs=8192,
                  max_batch_bytes=512 << 20, auto_release=True) as srv:
        t0 = time.perf_counter()
        lat, st = srv.replay(r["t_arrival"] * 1e6, kind, src, ln)
        wall = time.perf_counter() - t0
        stats = srv.stats()
    ok = st == 0
    lat_ok = lat[ok]
    return {
        "requests": int(n), "duration_s": duration_s, "offered_rps": 200_000.0,
        "completed_rps": round(int(ok.sum()) / wall, 1),
        "p50_us": round(float(np.percentile(lat_ok, 50)), 1),
        "p99_us": round(float(np.percentile(lat_ok, 99)), 1),
        "p999_us": round(float(np.percentile(lat_ok, 99.9)), 1),
        "mean_us": round(float(lat_ok.mean()), 1),
        "sustained_gbs": round(float(ln[ok].sum()) / wall / 1e9, 3),
        "batches": stats["batches"], "mean_batch": round(stats["requests_launched"] /
                                                         max(stats["batches"], 1), 1),
        "memory_waits": stats["memory_waits"], "rejected": stats["rejected"],
        "arena_high_water_bytes": stats["arena_high_water"], "memory_budget_bytes": 8 << 30,
        "status_ok": int(ok.sum()),
    }


def serve_line(args, d: Dist):
    s = run_serve(args, d, duration_s=30.0)
    return {
        "metric": "serving p99 latency (200k req/s Poisson, 50/50 encode/decode)",
        "value": s["p99_us"], "unit": "us", "n_gpus": d.world, "steps": 1, "warmup": 0,
        "ms_per_step": s["duration_s"] * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8",
        "data": "synthetic: Poisson arrivals, log-normal payloads (median 4 KiB, sigma 2), seed 4",
        "config": {"workload": "serving: 200k req/s for 30 s, 8 GiB admission budget (config 5)"},
        "serve": s,
    }


# ------------------------------------------------------ length sweep
SWEEP_LENGTHS = [16, 64, 256, 1 << 10, 4 << 10, 16 << 10, 64 << 10, 256 << 10, 1 << 20,
                 4 << 20, 16 << 20, 64 << 20, 256 << 20, 1 << 30]
# the default line's sweep: every decade of Fig. 10's range up to 256 MiB
SWEEP_COMPACT = [16, 256, 4 << 10, 64 << 10, 1 << 20, 16 << 20, 256 << 20]
SWEEP_KEY = 7  # counter-based stream of the sweep's bytes (regenerated on the host to check)


def _sweep_checks(g, big, enc, L, m, bsrc_len, benc, eoff, bdec, doff, st, ol, nmsg):
    """The sweep's outputs against the oracle: the single call's encoding on
    its first and last 4 KiB of characters and its round trip; the batch's
    status and lengths for every message and, on sampled messages, the
    encoding against the oracle and the decode against the payload."""
    import torch

    import oracle
    from paper_1704_00605_gb300 import workloads as W

    oracle.build()
    head = W.counter_bytes(SWEEP_KEY, 0, min(L, 3 * 1024))
    exp = oracle.encode(head)
    got = enc[:exp.size].cpu().numpy() if L > 3 * 1024 else enc[:m].cpu().numpy()
    assert np.array_equal(got[:min(exp.size, got.size)], exp[:min(exp.size, got.size)]), L
    if L > 3 * 1024:  # the last whole groups and the padded tail
        t0 = (L - 3 * 1024) // 3 * 3
        tail = W.counter_bytes(SWEEP_KEY, t0, L - t0)
        exp = oracle.encode(tail)
        assert np.array_equal(enc[t0 // 3 * 4:m].cpu().numpy(), exp), L
    checked = 0
    if benc is not None:
        assert int((st != 0).sum()) == 0 and bool((ol == L).all()), L
        eo, do = eoff.cpu().numpy(), doff.cpu().numpy()
        for j in np.unique(np.linspace(0, nmsg - 1, 24).astype(np.int64)):
            raw = W.counter_bytes(SWEEP_KEY, int(j) * L, L)
            assert np.array_equal(benc[eo[j]:eo[j + 1]].cpu().numpy(), oracle.encode(raw)), (L, j)
            assert np.array_equal(bdec[do[j]:do[j] + L].cpu().numpy(), raw), (L, j)
            checked += 1
    return checked


def run_sweep(args, d: Dist, lengths=SWEEP_LENGTHS, check: bool = False):
    """Fig. 10's experiment on the GPU: encode and decode time against the
    input length (uniform random bytes). For every length: one single-buffer
    call (CUDA-event time per call, averaged over back-to-back calls; small
    calls are launch-bound) and, up to 16 MiB, the same calls replayed from a
    CUDA graph (device time per call without the host's share); and a batch
    of messages of that length totalling 256 MiB through the batched calls
    (lengths <= 1 MiB). With check, every row's outputs are compared with
    the oracle (_sweep_checks) after its timing."""
    import torch

    import paper_1704_00605_gb300 as pkg
    from paper_1704_00605_gb300 import workloads as W

    torch.cuda.set_device(d.local_rank)
    g = pkg.load()
    dev = torch.device("cuda", d.local_rank)
    stream = torch.cuda.current_stream(dev)
    top = max(lengths)
    big = W.counter_bytes_torch(SWEEP_KEY, 0, max(top, 256 << 20), device=dev)
    enc = torch.empty(g.b64_encoded_len(top), dtype=torch.uint8, device=dev)
    dec = torch.empty(top + 16, dtype=torch.uint8, device=dev)
    res = torch.empty(3, dtype=torch.int64, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e3  # microseconds per call

    rows = []
    for L in lengths:
        reps = max(3, min(2000, (256 << 20) // L))
        src = big[:L]
        m = g.b64_encoded_len(L)
        e_us = timed(lambda: g.b64_encode(src, enc), reps)
        d_us = timed(lambda: g.b64_decode_async(enc[:m], dec, res), reps)
        st_, outlen_, fb_ = g.parse_result(res)
        assert (st_, outlen_, fb_) == (0, L, m) and torch.equal(dec[:L], src), L
        row = {"length": L, "encode_us": round(e_us, 3), "decode_us": round(d_us, 3),
               "encode_gbs": round(L / e_us / 1e3, 2), "decode_gbs": round(m / d_us / 1e3, 2)}
        if L <= (16 << 20):
            # the same calls replayed from a CUDA graph: device time per call
            # without the host-side cost of issuing it
            k = 64
            side = torch.cuda.Stream(dev)
            side.wait_stream(stream)
            ge, gd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(ge, stream=side):
                    for _ in range(k):
                        g.b64_encode(src, enc)
                with torch.cuda.graph(gd, stream=side):
                    for _ in range(k):
                        g.b64_decode_async(enc[:m], dec, res)
            stream.wait_stream(side)
            row["encode_us_graph"] = round(timed(ge.replay, 10) / k, 3)
            row["decode_us_graph"] = round(timed(gd.replay, 10) / k, 3)
            row["encode_gbs_graph"] = round(L / row["encode_us_graph"] / 1e3, 2)
            row["decode_gbs_graph"] = round(m / row["decode_us_graph"] / 1e3, 2)
        benc = eoff = bdec = doff = st = ol = None
        nmsg = 0
        if L <= (1 << 20):
            nmsg = max(1, (256 << 20) // L)
            off = torch.arange(nmsg + 1, dtype=torch.int64, device=dev) * L
            bsrc = big[:nmsg * L]
            eoff = g.b64_batch_out_offsets(False, off)
            benc = torch.empty(int(eoff[-1].item()), dtype=torch.uint8, device=dev)
            doff = g.b64_batch_out_offsets(True, eoff)  # decode outputs sit at capacity offsets
            bdec = torch.empty(int(doff[-1].item()) + 16, dtype=torch.uint8, device=dev)
            st = torch.empty(nmsg, dtype=torch.int32, device=dev)
            fb = torch.empty(nmsg, dtype=torch.int64, device=dev)
            ol = torch.empty(nmsg, dtype=torch.int64, device=dev)
            be = timed(lambda: g.b64_encode_batch(bsrc, off, benc, eoff), 5)
            bd = timed(lambda: g.b64_decode_batch(benc, eoff, bdec, doff, st, fb, ol), 5)
            row.update({"batch_msgs": nmsg,
                        "batch_encode_gbs": round(nmsg * L / be / 1e3, 1),
                        "batch_decode_gbs": round(benc.numel() / bd / 1e3, 1),
                        "batch_encode_msgs_per_s": round(nmsg / be * 1e6, 1),
                        "batch_decode_msgs_per_s": round(nmsg / bd * 1e6, 1)})
        if check:
            row["oracle_checked_msgs"] = _sweep_checks(g, big, enc, L, m, L, benc, eoff, bdec,
                                                       doff, st, ol, nmsg)
        rows.append(row)
        del benc, bdec
    return rows


def run_variants(args, d: Dist):
    """The variant flags on 256 MiB of uniform random bytes (single-buffer
    calls, CUDA-event time per call): base64url, unpadded, Appendix A's
    strict tail, and Appendix B's whitespace removal on MIME-style input
    (CRLF after every 76 characters) against the plain decode of the same
    characters without the line breaks."""
    import torch

    import paper_1704_00605_gb300 as pkg
    from paper_1704_00605_gb300 import workloads as W

    torch.cuda.set_device(d.local_rank)
    g = pkg.load()
    dev = torch.device("cuda", d.local_rank)
    stream = torch.cuda.current_stream(dev)
    n = 256 << 20
    src = W.counter_bytes_torch(8, 0, n, device=dev)
    res = torch.empty(3, dtype=torch.int64, device=dev)

    def timed(fn, reps=20):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e3  # microseconds per call

    out = {"bytes": n}
    dec = torch.empty(n + 16, dtype=torch.uint8, device=dev)

    def result():  # (first_bad, outlen, status) of the last decode
        return int(res[0]), int(res[1]), int(res.view(torch.int32)[4])

    for name, flags in (("plain", 0), ("url", 1), ("nopad", 2), ("strict", 4)):
        enc = g.b64_encode_ex(src, flags & 3)
        e_us = timed(lambda: g.b64_encode_ex(src, flags & 3, enc))
        d_us = timed(lambda: g.b64_decode_async_ex(enc, dec, res, flags))
        assert result() == (enc.numel(), n, 0), name
        out[name] = {"encode_us": round(e_us, 2), "decode_us": round(d_us, 2),
                     "encode_input_gbs": round(n / e_us / 1e3, 1),
                     "decode_input_gbs": round(enc.numel() / d_us / 1e3, 1)}
    out["whitespace"] = run_whitespace(args, d, src=src, plain_us=out["plain"]["decode_us"])
    return out


def mime_lines(enc, line: int = 76):
    """The characters enc cut into lines of `line` characters, each ended by
    CR LF (the last line too), built on the device."""
    import torch

    m = enc.numel()
    rows = (m + line - 1) // line
    body = torch.zeros(rows * line, dtype=torch.uint8, device=enc.device)
    body[:m] = enc
    lines = torch.empty(rows, line + 2, dtype=torch.uint8, device=enc.device)
    lines[:, :line] = body.view(rows, line)
    lines[:, line] = 13
    lines[:, line + 1] = 10
    wrapped = lines.view(-1)
    last = m - (rows - 1) * line  # characters on the last line
    if last != line:
        wrapped = torch.cat([wrapped[:(rows - 1) * (line + 2) + last], wrapped.new_tensor([13, 10])])
    return wrapped


def run_whitespace(args, d: Dist, src=None, plain_us=None):
    """Appendix B's whitespace removal before decoding, on the MIME form of
    the encoding of 256 MiB of uniform random bytes (76 characters and CR LF
    per line: 367,332,732 characters): CUDA-event time per call, the
    algorithmic bytes (characters read + bytes written) against the HBM
    peak, and an exact round trip; then the same input with one space
    inside a line, which breaks the line model and takes the general path."""
    import torch

    import paper_1704_00605_gb300 as pkg
    from paper_1704_00605_gb300 import workloads as W

    torch.cuda.set_device(d.local_rank)
    g = pkg.load()
    dev = torch.device("cuda", d.local_rank)
    stream = torch.cuda.current_stream(dev)
    n = 256 << 20
    if src is None:
        src = W.counter_bytes_torch(8, 0, n, device=dev)
    enc = g.b64_encode(src)
    wrapped = mime_lines(enc, 76)
    dec = torch.empty(n + 16, dtype=torch.uint8, device=dev)
    res = torch.zeros(3, dtype=torch.int64, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps * 1e3  # microseconds per call

    w_us = timed(lambda: g.b64_decode_async_ex(wrapped, dec, res, 8), 20)
    st, outlen, fb = g.parse_result(res)
    line_path = (int(res.view(torch.int32)[5].item()) & 0xFFFFFFFF) == 0x4C494E45
    assert (st, outlen, fb) == (0, n, wrapped.numel()), (st, outlen, fb)
    assert torch.equal(dec[:n], src)
    # the same lines with one space inside the second line: the model breaks
    # in the first tile, so the call decodes the input by the general path
    broken = torch.cat([wrapped[:100], wrapped.new_tensor([32]), wrapped[100:]])
    dec.zero_()
    g_us = timed(lambda: g.b64_decode_async_ex(broken, dec, res, 8), 10)
    st, outlen, fb = g.parse_result(res)
    g_line = (int(res.view(torch.int32)[5].item()) & 0xFFFFFFFF) == 0x4C494E45
    assert (st, outlen, fb, g_line) == (0, n, broken.numel(), False), (st, outlen, fb, g_line)
    assert torch.equal(dec[:n], src)
    del broken
    if plain_us is None:
        plain_us = timed(lambda: g.b64_decode_async(enc, dec, res), 20)
    peak, peak_kind = measured_peaks()
    alg = wrapped.numel() + n
    return {"chars": int(wrapped.numel()), "line": 76, "separator": "CR LF",
            "decode_us": round(w_us, 2), "decode_input_gbs": round(wrapped.numel() / w_us / 1e3, 1),
            "alg_bytes": int(alg), "hbm_gbs": round(alg / w_us / 1e3, 1),
            "frac": round(alg / w_us / 1e3 / peak, 4), "peak": peak,
            "peak_kind": f"{peak_kind} hbm_gbs", "line_model_path": line_path,
            "general_path_us": round(g_us, 2),
            "general_path_frac": round((alg + 1) / g_us / 1e3 / peak, 4),
            "plain_decode_us": round(plain_us, 2),
            "gpu_launches_per_call": 1, "memsets_per_call": 2}


def sweep_line(args, d: Dist):
    rows = run_sweep(args, d)
    variants = run_variants(args, d)
    top = rows[-1]
    return {
        "metric": "encode/decode input GB/s against input length (Fig. 10 sweep)",
        "value": top["encode_gbs"], "unit": "GB/s", "n_gpus": d.world, "steps": 1, "warmup": 1,
        "ms_per_step": top["encode_us"] / 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic: uniform random bytes",
        "config": {"workload": "length sweep 16 B .. 1 GiB, single calls and 256 MiB batches"},
        "sweep": rows, "variants_256mib": variants,
    }


def whitespace_line(args, d: Dist):
    w = run_whitespace(args, d)
    return {
        "metric": "decode input GB/s with whitespace removal (Appendix B, MIME lines)",
        "value": w["decode_input_gbs"], "unit": "GB/s", "n_gpus": d.world, "steps": 20,
        "warmup": 1, "ms_per_step": w["decode_us"] / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic: uniform random bytes",
        "config": {"workload": "whitespace removal on the MIME-wrapped encoding of 256 MiB "
                               "(CRLF after every 76 characters)"},
        "whitespace": w,
    }


def variants_line(args, d: Dist):
    v = run_variants(args, d)
    ws = v["whitespace"]
    return {
        "metric": "decode input GB/s with whitespace removal (Appendix B, MIME lines)",
        "value": ws["decode_input_gbs"], "unit": "GB/s", "n_gpus": d.world, "steps": 10,
        "warmup": 1, "ms_per_step": ws["decode_us"] / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic: uniform random bytes",
        "config": {"workload": "variant flags on 256 MiB; whitespace removal on its MIME-wrapped "
                               "encoding (CRLF after every 76 characters)"},
        "variants_256mib": v,
    }


# ------------------------------------------------------ reference arm
def run_reference(args, d: Dist):
    """The CPU oracle as it stands, on the host cores, on bounded samples of
    the same workload (the reference arm of this build)."""
    from paper_1704_00605_gb300 import workloads as W

    data = W.uniform_bytes(48 << 20, 1)  # prefix of the workload stream
    threads = os.cpu_count() or 1
    sample = 24 << 20
    for _ in range(args.warmup):
        oracle_throughput(data, 3 << 20, threads)
    t0 = time.perf_counter()
    moved = 0
    for _ in range(args.steps):
        oracle_throughput(data, sample, threads)
        moved += sample + 4 * sample // 3
    dt = time.perf_counter() - t0
    v = moved / dt / 1e9
    return {
        "impl": "reference",
        "metric": "enc+dec input GB/s (1 GiB buffer, encode then decode)",
        "value": round(v, 4), "unit": "GB/s", "n_gpus": d.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic: uniform random bytes, numpy default_rng(1)",
        "config": {"workload": "single large buffer: 1 GiB (+1, +2) encode + decode (config 2)",
                   "sample": f"{sample} bytes per step"},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"{sample}-byte prefix of the 1 GiB workload per step, "
                                   f"encode + decode, {threads} threads"},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return 0  # rank 0 alone runs the CPU reference
        os.environ["WORLD_SIZE"] = "1"
        d = Dist()
        print(json.dumps(run_reference(args, d)), flush=True)
        return 0
    d = Dist()
    if args.config == "batched":
        line = batched_line(args, d)
    elif args.config == "serve":
        line = serve_line(args, d)
    elif args.config == "sweep":
        line = sweep_line(args, d)
    elif args.config == "variants":
        line = variants_line(args, d)
    elif args.config == "whitespace":
        line = whitespace_line(args, d)
    else:
        line = run_large(args, d)
        if not args.small and not args.no_extras:
            line["batched"] = run_batched(args, d)
            line["whitespace"] = run_whitespace(args, d)
            sweep = run_sweep(args, d, lengths=SWEEP_COMPACT, check=True)
            line["sweep"] = sweep
            r1 = [r for r in sweep if r["length"] == 1 << 20][0]
            line["config1_1mib"] = {
                "length": 1 << 20, "encoded_chars": 1398104,
                "encode_gbs_graph": r1["encode_gbs_graph"], "decode_gbs_graph": r1["decode_gbs_graph"],
                "encode_us_graph": r1["encode_us_graph"], "decode_us_graph": r1["decode_us_graph"],
                "encode_gbs_host_loop": r1["encode_gbs"], "decode_gbs_host_loop": r1["decode_gbs"],
                "note": "one call of the 1 MiB length, amortised over 64 graph-replayed calls "
                        "(device time) and over back-to-back calls from the host"}
            line["serve"] = run_serve(args, d, duration_s=args.serve_seconds)
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
