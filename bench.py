#!/usr/bin/env python
"""Benchmark of the PFB channeliser on GB300.

Default workload (N=1): one channelisation of 2^24 complex64 samples,
P=1024 branches, T=16 taps, Hamming-windowed sinc prototype, FP32 FIR + FFT
path (the paper-scale configuration).  One step = one pass of the fused
FIR + DFT over that stream (load/dequant, polyphase FIR, DFT, store).

Printed as one JSON line (rank 0).  Besides the headline value it reports:
  roofline      dominant kernel vs the measured HBM copy bandwidth
  e2e           same metric through pfb_execute_host (H2D + kernel + D2H per step)
  paths         GSample/s and rel. L2 error vs the FP64 oracle of the three DFT
                paths (FP32 FFT, FP32 DFT-GEMM, split-bf16 tensor-core DFT-GEMM)
  serving       p50/p99 request latency and GSample/s of a Poisson request
                stream through pfb_submit/pfb_poll
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample
  clocks        SM clocks and throttle reasons sampled during the timed region

--impl reference times the FP64 oracle (the reference arm of this repo) on the
same workload, one bounded sample per step.
"""

from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PFB GSample/s split-BF16 DFT vs FP32 at rel err ≤1e-5; serving p50/p99 latency"
UNIT = "GSample/s"


def load_json(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return None


def peaks():
    p = load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"))
    if p and "hbm_gbs" in p:
        return float(p["hbm_gbs"]), float(p.get("bf16_tflops", 1955.4)), float(p.get("bf16_tflops_sustained", 1702.1)), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


def source_hash(files=None) -> str:
    """Hash of the given source files of the library (default: all of csrc/)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2408_16551_gb300", "csrc")
    paths = sorted(os.path.join(csrc, f) for f in files) if files else sorted(glob.glob(os.path.join(csrc, "*")))
    for f in paths:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def gpu_local_cpus(dev_index: int):
    """CPUs local to the GPU (sysfs local_cpulist of its PCI function), or None."""
    try:
        import torch
        p = torch.cuda.get_device_properties(dev_index)
        path = f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0/local_cpulist"
        cpus = set()
        for part in open(path).read().strip().split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        cur = os.sched_getaffinity(0)
        cpus &= cur
        return cpus if cpus and cpus != cur else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if smax and s > 0.5 * smax] or sm
        load.sort()
        return {"sm_mhz": load[len(load) // 2] if load else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def gpu_index_for(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def sampled_rel_l2(X_dev, x_host, in_dtype, P, T, window, rows):
    import numpy as np
    import oracle
    h = oracle.prototype(P, T, window)
    xs = oracle.dequant(x_host, in_dtype)
    got = X_dev[rows].cpu().numpy()
    ref = np.concatenate([oracle.pfb(xs, P, T, h, s0=int(r), ns=1) for r in rows])
    return oracle.rel_l2(got, ref)


def cpu_baseline_oracle(x_host, in_dtype, P, T, window, target_s=12.0):
    """Time the FP64 oracle on a bounded prefix of the workload's spectra."""
    import oracle
    h = oracle.prototype(P, T, window)
    xs = oracle.dequant(x_host, in_dtype)
    S = oracle.num_spectra(xs[0].size, P, T)
    ns = min(S, 16)
    t0 = time.perf_counter()
    oracle.pfb(xs, P, T, h, s0=0, ns=ns)
    dt = time.perf_counter() - t0
    ns2 = int(min(S, max(ns, ns * target_s / max(dt, 1e-3))))
    if ns2 > ns:
        t0 = time.perf_counter()
        oracle.pfb(xs, P, T, h, s0=0, ns=ns2)
        dt = time.perf_counter() - t0
        ns = ns2
    gsps = ns * P / dt / 1e9
    return {"value": gsps, "unit": UNIT, "cores": cores(), "kind": "oracle",
            "sample": f"FP64 oracle (explicit FIR then naive DFT) on spectra 0..{ns - 1} of the workload "
                      f"({ns * P} input samples consumed at hop P), {dt:.1f} s"}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def workload_c2():
    from paper_2408_16551_gb300 import synth
    spec = synth.config_c2()
    return spec, spec.generate()


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    spec, x = workload_c2()
    h = oracle.prototype(spec.P, spec.T, spec.window)
    xs = oracle.dequant(x, spec.in_dtype)
    ns = 64  # spectra per step: a bounded sample of the workload
    n_windows = oracle.num_spectra(x.size, spec.P, spec.T) - ns + 1  # sample starts, wrapped for long runs
    for i in range(args.warmup):
        oracle.pfb(xs, spec.P, spec.T, h, s0=(i * ns) % n_windows, ns=ns)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.pfb(xs, spec.P, spec.T, h, s0=((args.warmup + i) * ns) % n_windows, ns=ns)
    dt = (time.perf_counter() - t0) / args.steps
    value = ns * spec.P / dt / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "c2: 2^24 complex64 samples, P=1024, T=16, Hamming-windowed sinc; "
                               f"each step = {ns} spectra of it through the FP64 oracle",
                   "P": spec.P, "T": spec.T, "n_samples": int(x.size)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores(), "kind": "oracle",
                         "sample": f"{ns} spectra ({ns * spec.P} input samples at hop P) per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_path(pkg, plan, xs, outs, steps, warmup, stream):
    """Per-launch CUDA-event timing of plan.execute over rotating buffers."""
    import torch
    for i in range(warmup):
        plan.execute(xs[i % len(xs)], out=outs[i % len(outs)], stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(steps):
        plan.execute(xs[i % len(xs)], out=outs[i % len(outs)], stream=stream)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[-1]) / steps, per


def run_serving(pkg, n_requests, rate_hz, warm_requests, device):
    """Open-loop Poisson requests (P=4096, T=16, complex int8, 2^20 samples in
    16 chunks of 2^16, state resident across chunks); latency = arrival ->
    completion of the request's last chunk, observed by polling."""
    import numpy as np
    import torch
    from paper_2408_16551_gb300 import synth
    wl = synth.config_c5(n_requests=n_requests + warm_requests, rate_hz=rate_hz)
    plan = pkg.Plan(wl.P, wl.T, pkg.PFB_IN_CI8, wl.window, pkg.PFB_DFT_FFT_F32)
    srv = pkg.Server(hbm_budget_bytes=40 << 30, max_slots=32, timeout_ms=5000, queue_when_busy=True)
    nbuf = 32
    rng = np.random.default_rng(wl.seed)
    bufs = [torch.from_numpy(rng.integers(-127, 128, size=2 * wl.request_samples, dtype=np.int16).astype(np.int8)).to(device)
            for _ in range(nbuf)]
    nch = wl.request_samples // wl.chunk_samples
    s_req = plan.out_spectra(wl.request_samples)      # spectra of a whole request (state starts empty)
    outs = [torch.empty((s_req, wl.P), dtype=torch.complex64, device=device) for _ in range(nbuf)]
    arrivals = wl.arrivals()
    torch.cuda.synchronize()
    pending = []  # (req index, sid, last ticket, t_arrival)
    lat = []
    t_start = time.perf_counter()
    i = 0
    done_samples = 0
    t_first = None
    while i < len(arrivals) or pending:
        now = time.perf_counter() - t_start
        if i < len(arrivals) and now >= arrivals[i]:
            b = i % nbuf
            sid = srv.open_stream(plan)
            last = None
            row = 0
            for c in range(nch):
                S = srv.next_spectra(sid, wl.chunk_samples)
                o = outs[b][row:row + S]
                row += S
                last = srv.submit(sid, bufs[b][2 * c * wl.chunk_samples: 2 * (c + 1) * wl.chunk_samples],
                                  wl.chunk_samples, o if S > 0 else None)
            pending.append((i, sid, last, t_start + arrivals[i]))
            i += 1
            continue
        still = []
        for (ri, sid, tk, ta) in pending:
            st = srv.poll(tk)
            if st == pkg.PFB_PENDING:
                still.append((ri, sid, tk, ta))
                continue
            tdone = time.perf_counter()
            srv.close_stream(sid)
            if st == pkg.PFB_OK and ri >= warm_requests:
                lat.append((tdone - ta) * 1e6)
                done_samples += wl.request_samples
                if t_first is None:
                    t_first = ta
        pending = still
    t_end = time.perf_counter()
    stats = srv.stats()
    srv.close()
    lat.sort()
    if not lat:
        return None
    span = t_end - (t_first or t_start)
    return {"workload": f"Poisson {rate_hz:.0f} req/s, {n_requests} requests (+{warm_requests} warm-up discarded); "
                        f"request = P={wl.P}, T={wl.T} channelisation of {wl.request_samples} complex int8 samples "
                        f"in {nch} chunks of {wl.chunk_samples}, filter state resident on the device",
            "p50_us": lat[len(lat) // 2], "p99_us": lat[min(len(lat) - 1, int(0.99 * (len(lat) - 1) + 0.5))],
            "gsps": done_samples / span / 1e9, "chunk_p50_us": stats["p50_latency_us"],
            "mean_batch": stats["batched_requests"] / max(stats["batches"], 1),
            "chunk_p99_us": stats["p99_latency_us"], "failed": stats["failed"],
            "peak_reserved_bytes": stats["peak_reserved_bytes"]}


def run_c3(pkg, device, reps=3, paths=("fft_f32", "gemm_bf16x3", "gemm_f32"), rel_err=True):
    """Configuration 3: 64 streams x 2^20 complex64, P=4096, T=16, Blackman; every
    DFT path as one batched launch over the 64 streams; rel. L2 on sampled spectra."""
    import numpy as np
    import torch
    from paper_2408_16551_gb300 import synth
    specs = synth.config_c3()
    xs_host = [sp.generate() for sp in specs]
    xs = [torch.from_numpy(x).to(device) for x in xs_host]
    P, T, win = specs[0].P, specs[0].T, specs[0].window
    n_total = sum(x.size for x in xs_host)
    out = {"workload": "c3: 64 streams x 2^20 complex64 samples (CN(0,1) + 2 tones each), P=4096, T=16, "
                       "Blackman-windowed sinc; one batched launch per DFT path", "n_samples": int(n_total)}
    rows = [0, 120, 240]
    for name, path in (("fft_f32", pkg.PFB_DFT_FFT_F32), ("gemm_bf16x3", pkg.PFB_DFT_GEMM_BF16X3),
                       ("gemm_f32", pkg.PFB_DFT_GEMM_F32)):
        if name not in paths:
            continue
        try:
            plan = pkg.Plan(P, T, pkg.PFB_IN_C64, win, path)
            S = plan.out_spectra(xs_host[0].size)
            outs = [torch.empty((S, P), dtype=torch.complex64, device=device) for _ in xs]
            entries = [(plan, x, o) for x, o in zip(xs, outs)]
            batch = pkg.Batch(entries)
            batch.launch()
            torch.cuda.synchronize()
            r = 1 if path == pkg.PFB_DFT_GEMM_F32 else reps
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(r):
                batch.launch()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / r
            errs = [sampled_rel_l2(outs[i], xs_host[i], pkg.PFB_IN_C64, P, T, win, rows) for i in (0, 37)] \
                if rel_err else [None]
            out[name] = {"gsps": n_total / (ms * 1e-3) / 1e9, "ms": ms, "rel_l2": max(errs) if rel_err else None,
                         "kernel": plan.kernel_name, "variant": plan.variant,
                         "hbm_frac": (n_total * 8 + len(xs) * S * P * 8) / (ms * 1e-3) / (peaks()[0] * 1e9)}
            batch.close(); plan.close()
            del outs
        except pkg.PFBError as e:
            out[name] = {"gsps": None, "unavailable": str(e)}
    return out


def run_oversampled(pkg, device, xs, x_host, spec, reps=50):
    """The c2 stream through a 2x oversampled plan (hop P/2, twice the spectra),
    FFT path; rel. L2 on sampled spectra against the FP64 oracle."""
    import numpy as np
    import torch
    import oracle
    P, T, D = spec.P, spec.T, spec.P // 2
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, spec.window, pkg.PFB_DFT_FFT_F32, hop=D)
    n = int(x_host.size)
    S = plan.out_spectra(n)
    outs = [torch.empty((S, P), dtype=torch.complex64, device=device) for _ in range(2)]
    for i in range(5):
        plan.execute(xs[i % len(xs)], out=outs[i % 2])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(reps):
        plan.execute(xs[i % len(xs)], out=outs[i % 2])
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    last = outs[(reps - 1) % 2]
    rows = [0, 1, S // 2, S // 2 + 1, S - 2, S - 1]
    h = oracle.prototype(P, T, spec.window)
    xs64 = oracle.dequant(x_host, oracle.IN_C64)
    ref = np.concatenate([oracle.pfb_hop(xs64, P, T, h, D, s0=r, ns=1) for r in rows])
    err = oracle.rel_l2(last[rows].cpu().numpy(), ref)
    alg = n * 8 + S * P * 8
    out = {"workload": f"c2 stream, hop P/2 = {D} (2x oversampled), FFT path", "spectra": S, "ms": ms,
           "gsps": n / (ms * 1e-3) / 1e9, "spectra_per_s": S / (ms * 1e-3), "rel_l2": err,
           "hbm_frac": alg / (ms * 1e-3) / (peaks()[0] * 1e9), "kernel": plan.kernel_name, "variant": plan.variant}
    plan.close()
    return out


def run_synthesis(pkg, device, X_spectra, spec, reps=50):
    """The synthesis (inverse) filter bank of the c2 analysis output: spectra
    [16369, 1024] back to (S + T - 1) * P samples; rel. L2 on sampled frames."""
    import numpy as np
    import torch
    import oracle
    P, T = spec.P, spec.T
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, spec.window, pkg.PFB_DFT_FFT_F32)
    S = X_spectra.shape[0]
    n_out = plan.synth_out_samples(S)
    outs = [torch.empty((n_out,), dtype=torch.complex64, device=device) for _ in range(2)]
    for i in range(5):
        plan.synthesize(X_spectra, out=outs[i % 2])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(reps):
        plan.synthesize(X_spectra, out=outs[i % 2])
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    last = outs[(reps - 1) % 2]
    h = oracle.prototype(P, T, spec.window)
    frames = [0, 7, S // 2, S - 1, S + T - 2]
    rows_needed = sorted({s for f in frames for s in range(max(0, f - T + 1), min(S, f + 1))})
    Xh = np.zeros((S, P), dtype=np.complex128)
    Xh[rows_needed] = X_spectra[rows_needed].cpu().numpy()
    ref = np.concatenate([oracle.synth(Xh, P, T, h, f0=f, nf=1) for f in frames])
    got = np.concatenate([last[f * P:(f + 1) * P].cpu().numpy() for f in frames])
    alg = S * P * 8 + n_out * 8
    out = {"workload": f"synthesis of the c2 analysis output: {S} spectra x P={P} -> {n_out} samples, T={T}",
           "ms": ms, "gsps": n_out / (ms * 1e-3) / 1e9, "rel_l2": oracle.rel_l2(got, ref),
           "hbm_frac": alg / (ms * 1e-3) / (peaks()[0] * 1e9), "kernel": "k_synth_ws"}
    plan.close()
    return out


def run_c4(pkg, device, reps=5):
    """Configuration 4: 256 uneven streams (P in {256,512,1024,4096}, T in {8,16},
    lengths log-uniform 2^14..2^22) as one captured CUDA graph over per-variant
    persistent launches, tile shapes from the autotuner."""
    import torch
    from paper_2408_16551_gb300 import synth
    specs = synth.config_c4()
    plans = {}
    entries = []
    n_total = 0
    for sp in specs:
        key = (sp.P, sp.T, sp.window)  # one plan per shape; streams of a shape share it
        if key not in plans:
            plans[key] = pkg.Plan(sp.P, sp.T, pkg.PFB_IN_C64, sp.window, pkg.PFB_DFT_FFT_F32)
            plans[key].autotune(min(sp.P * 4096, 1 << 24))
        plan = plans[key]
        x = torch.from_numpy(sp.generate()).to(device)
        S = plan.out_spectra(sp.n_samples)
        o = torch.empty((max(S, 1), sp.P), dtype=torch.complex64, device=device)
        entries.append((plan, x, o))
        n_total += sp.n_samples
    batch = pkg.Batch(entries)
    batch.launch()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    zero = sum(1 for (p, x, o) in entries if p.out_spectra(x.numel()) == 0)
    return {"workload": "c4: 256 uneven complex64 streams, P~U{256,512,1024,4096}, T~U{8,16}, N=2^U, U~U(14,22); "
                        "one CUDA graph of per-variant persistent launches, autotuned tile shapes",
            "n_samples": int(n_total), "gsps": n_total / (ms * 1e-3) / 1e9, "ms": ms,
            "streams_with_zero_spectra": zero}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-paths", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--no-configs", action="store_true", help="skip the c3/c4 lines")
    ap.add_argument("--minimal", action="store_true", help="headline timing only (for profiler runs)")
    ap.add_argument("--nsets", type=int, default=4, help="rotating input/output buffer sets")
    ap.add_argument("--variant", type=int, default=-1, help="kernel variant of the headline path (-1: autotune / default)")
    ap.add_argument("--path", default="fft", choices=["fft", "bf16x3"],
                    help="DFT route of the headline step: FP32 FFT, or the split-bf16 tensor-core DFT")
    ap.add_argument("--c3-only", action="store_true",
                    help="time only configuration 3 (64 x 2^20, P=4096) through the --path route (profiler runs)")
    ap.add_argument("--synth-only", action="store_true",
                    help="time only the synthesis filter bank of the c2 analysis output (profiler runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    from paper_2408_16551_gb300 import build as pbuild
    pbuild.build()
    import paper_2408_16551_gb300 as pkg
    from paper_2408_16551_gb300 import replicas

    if args.c3_only:
        paths = ("fft_f32",) if args.path == "fft" else ("gemm_bf16x3",)
        print(json.dumps({"c3": run_c3(pkg, device, paths=paths, rel_err=False)}), flush=True)
        return

    spec, x = workload_c2()
    P, T = spec.P, spec.T
    n = int(x.size)
    if args.synth_only:
        p0 = pkg.Plan(P, T, pkg.PFB_IN_C64, spec.window, pkg.PFB_DFT_FFT_F32)
        X0 = p0.execute(torch.from_numpy(x).to(device))
        torch.cuda.synchronize()
        print(json.dumps({"synthesis": run_synthesis(pkg, device, X0, spec, reps=max(3, args.steps // 4))}), flush=True)
        return
    tc_path = args.path == "bf16x3"
    plan = pkg.Plan(P, T, pkg.PFB_IN_C64, spec.window, pkg.PFB_DFT_GEMM_BF16X3 if tc_path else pkg.PFB_DFT_FFT_F32)
    S = plan.out_spectra(n)
    if args.variant >= 0:
        plan.variant = args.variant
    elif not tc_path:
        plan.autotune(n)  # tile shape (kernel variant) from the autotuner
    # (split-bf16: the factored tensor-core DFT is the plan's default variant at P = 1024)
    nsets = max(1, args.nsets)  # rotating input/output sets: 4 x 256 MiB > 129 MB L2
    xd0 = torch.from_numpy(x).to(device)
    xs = [xd0] + [xd0.clone() for _ in range(nsets - 1)]
    outs = [torch.empty((S, P), dtype=torch.complex64, device=device) for _ in range(nsets)]
    stream = torch.cuda.current_stream()

    # ---------------- headline: device-resident inputs -----------------
    for i in range(args.warmup):
        plan.execute(xs[i % nsets], out=outs[i % nsets], stream=stream)
    # two events around the K steps (events between launches would add gaps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(gpu_index_for(local_rank)) if not args.minimal else None
    if sampler:
        # nvidia-smi's start-up (NVML initialisation) must be over before the timed region
        sampler.start()
        time.sleep(1.0)
    replicas.barrier()
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    ev[0].record(stream)
    for i in range(args.steps):
        plan.execute(xs[i % nsets], out=outs[i % nsets], stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    replicas.barrier()
    gpu_launches = pkg.launch_count() - launches0
    # hold the clock sampler on a loaded GPU for a moment (not timed)
    if sampler:
        t_end = time.perf_counter() + 1.0
        while time.perf_counter() < t_end:
            for i in range(20):
                plan.execute(xs[i % nsets], out=outs[i % nsets], stream=stream)
            torch.cuda.synchronize()
        clocks = sampler.stop()
    else:
        clocks = None
    total_ms = ev[0].elapsed_time(ev[1])
    ms_step_local = total_ms / args.steps
    # per-launch durations (median, min, max) from a separate untimed pass with an
    # event between launches; the headline stays the two-event mean above
    per_launch = sorted(time_path(pkg, plan, xs, outs, 50, 0, stream)[1]) if not args.minimal else []
    ms_step = replicas.max_over_ranks(ms_step_local)
    value = world * n / (ms_step * 1e-3) / 1e9

    hbm, bf16, bf16s, peak_kind = peaks()
    alg_bytes = n * 8 + S * P * 8
    kern_ms = ms_step_local  # one kernel launch per step: the average launch duration
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    traffic = None
    prof = load_json(os.path.join(ROOT, "profiles", "traffic.json"))
    kkey = f"{plan.kernel_name}:{plan.variant}"
    kent = (prof or {}).get("kernels", {}).get(kkey)
    if kent and kent.get("source_hash") == source_hash(kent.get("sources")):
        traffic = kent.get("dram_bytes_per_launch")  # counters taken on these very sources
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": f"{plan.kernel_name} variant {plan.variant}",
                "algorithmic_bytes_per_launch": alg_bytes,
                "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    if tc_path and plan.variant == 1:
        # executed bf16 tensor work of the factored DFT per spectrum: 2 products
        # (32 rows x 64 x 64 real block form each) x 3 split terms x 2 flop/MAC
        # = 1,572,864 flop per 1024 samples = 1536 flop per sample
        flop = n * (2 * 3 * 2 * 32 * 64 * 64 // 1024)
        tfl = flop / (kern_ms * 1e-3) / 1e12
        roofline["tensor"] = {"executed_tflops": tfl, "peak_tflops": bf16s, "frac": tfl / bf16s,
                              "flop_per_sample": flop // n, "peak_source": "sustained bf16 (MEASURED_PEAKS.json)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3/f32acc" if tc_path else "f32", "data": "synthetic",
        "config": {"workload": "c2: one stream of 2^24 complex64 samples (CN(0,1) + 8 channel-centre tones), "
                               "P=1024, T=16, Hamming-windowed sinc prototype; "
                               + ("FIR + split-bf16 tensor-core DFT path" if tc_path else "FIR + FFT path (FP32)"),
                   "P": P, "T": T, "n_samples": n, "spectra": S, "path": "gemm_bf16x3" if tc_path else "fft_f32",
                   "variant": plan.variant,
                   "l2": f"{nsets} rotating input/output buffer sets ({nsets * (n * 8 + S * P * 8) >> 20} MiB) > 129 MB L2",
                   "replicas": "each rank channelises its own copy of the workload (weak scaling, no collective)"},
        "roofline": roofline,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if per_launch:
        line["per_launch_ms"] = {"launches": len(per_launch), "median": per_launch[len(per_launch) // 2],
                                 "min": per_launch[0], "max": per_launch[-1],
                                 "note": "separate untimed pass, an event between launches"}

    if not args.minimal:
        import numpy as np
        rows = sorted(set([0, S // 3, S // 2, S - 1] + list(np.random.default_rng(1).integers(0, S, 6))))
        head = "gemm_bf16x3" if tc_path else "fft_f32"
        paths = {head: {"gsps": value / world, "rel_l2": sampled_rel_l2(outs[(args.steps - 1) % nsets], x,
                                                                       spec.in_dtype, P, T, spec.window, rows),
                        "dtype": "bf16x3/f32acc" if tc_path else "f32", "kernel": plan.kernel_name}}
        others = (("fft_f32", pkg.PFB_DFT_FFT_F32, "f32"),) if tc_path else \
            (("gemm_bf16x3", pkg.PFB_DFT_GEMM_BF16X3, "bf16x3/f32acc"),)
        if not args.no_paths:
            for name, path, dt in others + (("gemm_f32", pkg.PFB_DFT_GEMM_F32, "f32"),):
                try:
                    p2 = pkg.Plan(P, T, pkg.PFB_IN_C64, spec.window, path)
                    if path == pkg.PFB_DFT_FFT_F32:
                        p2.autotune(n)
                    ms, per = time_path(pkg, p2, xs, outs, max(3, args.steps // 4), 2, stream)
                    err = sampled_rel_l2(outs[(max(3, args.steps // 4) - 1) % nsets], x, spec.in_dtype, P, T,
                                         spec.window, rows)
                    paths[name] = {"gsps": n / (ms * 1e-3) / 1e9, "rel_l2": err, "dtype": dt, "kernel": p2.kernel_name,
                                   "variant": p2.variant, "ms_per_step": ms,
                                   "hbm_frac": alg_bytes / (ms * 1e-3) / 1e9 / hbm}
                    if path == pkg.PFB_DFT_GEMM_BF16X3 and p2.variant == 1:
                        # factored tensor-core DFT: 1536 executed bf16 flop per sample (see the roofline note)
                        tfl = n * 1536 / (ms * 1e-3) / 1e12
                        paths[name]["tensor"] = {"executed_tflops": tfl, "frac_of_sustained_bf16": tfl / bf16s}
                    elif path == pkg.PFB_DFT_GEMM_F32:
                        # complex x complex FMA against the DFT matrix: 8P flop per sample on the FP32 SIMT cores
                        tfl = n * 8 * P / (ms * 1e-3) / 1e12
                        paths[name]["fp32_tflops"] = tfl
                    p2.close()
                except pkg.PFBError as e:
                    paths[name] = {"gsps": None, "unavailable": str(e)}
        line["paths"] = paths

        if not args.no_e2e:
            # pinned buffers on the GPU's local CPU node (first touch by this
            # thread while its affinity is that node), then the old affinity back
            local = gpu_local_cpus(gpu_index_for(local_rank))
            old_aff = os.sched_getaffinity(0)
            if local:
                os.sched_setaffinity(0, local)
            hin = torch.empty(x.shape, dtype=torch.complex64).pin_memory()
            hin.numpy()[...] = x
            hout = torch.empty((S, P), dtype=torch.complex64).pin_memory()
            hout.numpy()[...] = 0
            xin = hin.numpy()
            xout = hout.numpy()
            for _ in range(2):
                plan.execute_host(xin, xout)
            k2 = max(3, args.steps // 4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(k2):
                plan.execute_host(xin, xout)
            dt = (time.perf_counter() - t0) / k2
            if local:
                os.sched_setaffinity(0, old_aff)
            line["e2e"] = {"value": n / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": n * 8,
                           "d2h_bytes_per_step": S * P * 8, "api": "pfb_execute_host (pinned host buffers)",
                           "host_buffers": f"pinned, first touched on the GPU-local CPUs ({len(local)} cpus)"
                           if local else "pinned"}

        if not args.no_configs and rank == 0:
            line["oversampled"] = run_oversampled(pkg, device, xs, x, spec)
            line["synthesis"] = run_synthesis(pkg, device, outs[(args.steps - 1) % nsets], spec)
            del xs, outs
            torch.cuda.empty_cache()
            line["c3"] = run_c3(pkg, device)
            line["c4"] = run_c4(pkg, device)

        if not args.no_serving and rank == 0:
            try:
                line["serving"] = run_serving(pkg, args.serving_requests, 2000.0, max(100, args.serving_requests // 10),
                                              device)
            except Exception as e:  # reported, not hidden
                line["serving"] = {"error": repr(e)}

        if not args.no_cpu_baseline and rank == 0 and world == 1:
            line["cpu_baseline"] = cpu_baseline_oracle(x, spec.in_dtype, P, T, spec.window)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
