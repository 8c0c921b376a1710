#!/usr/bin/env python
"""Benchmark: FFCz correction to certified feasibility on B300.

Workload (default ``lognormal512``): a 512^3 float32 lognormal density field
(exp of a unit-variance GRF with P(k) ~ k^-2.5), base-compressor error from a
uniform quantiser with eps_s = 1e-4 * range, eps_f = 1e-3 * max|FFT(x)|.
One step = one ``ffcz_correct`` call (the whole loop plus FP64 certification)
on a fresh copy of e0 already resident in HBM (the copy is outside the event
pair).  The field (537 MB) is larger than L2, so no flush is needed.

Printed JSON line (rank 0): value = field GB/s (4 N bytes per step, summed
over ranks), e2e = the same through the host-buffer entry point with the
copies inside the timed region, roofline of the dominant kernel (CUDA events
around each launch, live), per-iteration roofline from forced iterations,
and the oracle timed on the host cores (cpu_baseline).

Multi-GPU: a single field does not shard; ``--gpus N`` runs N independent
replicas (one process per GPU under torchrun) and reports their aggregate.
``--impl reference`` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2601_01596_b300 import workloads as W  # noqa: E402

METRIC = "field GB/s to certified feasibility, 512^3 fp32; % HBM roofline/iteration"
FP64_TFLOPS_NOMINAL = 1.25   # nominal dense FP64 rate of a B300 (context only)

# DRAM bytes (read + write) per 512^3 launch and FP64-pipe utilisation from
# one ncu capture of each kernel (summaries in profiles/), taken on half-size
# fields of the same kernels (512x256x512 for the x and z passes, 256x512x512
# for the y passes, 268 MB each) and scaled by 2: every pass touches each
# value once, so its traffic grows with the values processed.  The figures
# describe the kernel sources as they were at that capture: NCU_SRC_SHA is the
# digest of those sources (kernel_sources_sha()), and when the current
# sources differ the figures are reported as null.
NCU_CAPTURE = "ncu capture of 2026-12-04 (profiles/roofline_*.md; half-size fields, traffic x 2)"
NCU_SRC_SHA = "a3922083cc7ba78a"
NCU_TRAFFIC = {
    "chk<f32,512>": 2 * (280047616 + 223072256),      # k_chk_tma<512, 8, lean>
    "axis_fwd<f32,512>": 2 * (268473856 + 215547904),  # k_axis_tma<512, -1, 8>
    "px<f32,256>": 2 * (268479232 + 208703744),        # k_px_tma<256, 2, lean>
    "xfwd<f64,256>": 2 * (269651712 + 479538688),      # k_xfwd<double, 256, 2, X2>
    "xfwd<f32,256>": 2 * (268478720 + 217321472),      # k_xfwd_tma<256, 2> (entry)
    "axis_fwd<f64,512>": 2 * (537792512 + 481961984),  # k_axis<double, 512, -1, 4>
    "chk_cert<f64,512>": 2 * (551576576 + 3133184),    # k_chk<double, 512, 4> (check only)
}
NCU_FP64_PIPE = {"xfwd<f64,256>": 0.854, "axis_fwd<f64,512>": 0.854, "chk_cert<f64,512>": 0.848}


def kernel_sources_sha():
    """Digest of the device-code sources (the kernels whose counters
    NCU_TRAFFIC records)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2601_01596_b300", "csrc")
    for f in ("fft_core.cuh", "passes.cuh", "tma.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_figures(key, n):
    """(traffic, fp64 pipe fraction, note) for the top kernel: the recorded
    ncu figures when they describe the current kernel sources at 512^3."""
    if n != 512 ** 3:
        return None, None, "no capture at this size"
    if kernel_sources_sha() != NCU_SRC_SHA:
        return None, None, "kernel sources changed since the " + NCU_CAPTURE
    return NCU_TRAFFIC.get(key), NCU_FP64_PIPE.get(key), "from the " + NCU_CAPTURE


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def make_workload(name):
    if name == "lognormal512":
        return W.lognormal_field(512)
    if name == "lognormal512s":
        return W.lognormal_field(512, stress=0.2)
    if name == "lognormal256":
        return W.lognormal_field(256)
    if name == "grf32":
        return W.grf_field(32)
    if name == "turbulence256":
        return W.turbulence_field(256)
    if name.startswith("lognormal:"):
        # the same recipe on another 3D shape, e.g. lognormal:512x256x512
        # (smaller cases of the 512-point kernels for profiling)
        return W.lognormal_shape([int(v) for v in name.split(":", 1)[1].split("x")])
    raise SystemExit(f"unknown workload {name}")


# ---------------------------------------------------------------- clocks
class _NvmlC:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes)."""

    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2 failed")

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.c.c_void_p()
        if self.lib.nvmlDeviceGetHandleByIndex_v2(self.c.c_uint(i), self.c.byref(h)) != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex_v2 failed")
        return h

    def nvmlDeviceGetClockInfo(self, h, kind):
        v = self.c.c_uint()
        if self.lib.nvmlDeviceGetClockInfo(h, self.c.c_int(kind), self.c.byref(v)) != 0:
            raise RuntimeError("nvmlDeviceGetClockInfo failed")
        return v.value

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        v = self.c.c_uint()
        if self.lib.nvmlDeviceGetMaxClockInfo(h, self.c.c_int(kind), self.c.byref(v)) != 0:
            raise RuntimeError("nvmlDeviceGetMaxClockInfo failed")
        return v.value

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.c.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        if fn(h, self.c.byref(v)) != 0:
            raise RuntimeError("clock event reasons query failed")
        return v.value


class Clocks:
    """SM clocks and throttle reasons sampled DURING a region (read-only).

    NVML is polled from a thread every 10 ms, so even a region of a few tens of
    milliseconds gets samples; without NVML, nvidia-smi is polled at 200 ms.
    """

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.thread = None
        self.samples = []
        self.stop_evt = threading.Event()
        self.nvml = None
        self.err = None
        # the CUDA ordinal of this process maps to the NVML index through
        # CUDA_VISIBLE_DEVICES when it is set
        idx = dev
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            ids = [x.strip() for x in vis.split(",") if x.strip()]
            if dev < len(ids) and ids[dev].isdigit():
                idx = int(ids[dev])
        for make in (lambda: __import__("pynvml"), _NvmlC):
            try:
                n = make()
                if hasattr(n, "nvmlInit"):
                    n.nvmlInit()
                self.handle = n.nvmlDeviceGetHandleByIndex(idx)
                self.nvml = n
                break
            except Exception as ex:   # try the next binding, else nvidia-smi
                self.err = f"{type(ex).__name__}: {ex}"

    def _poll(self):
        n = self.nvml
        bits = [n.nvmlClocksEventReasonHwSlowdown, n.nvmlClocksEventReasonHwThermalSlowdown,
                n.nvmlClocksEventReasonSwThermalSlowdown, n.nvmlClocksEventReasonSwPowerCap]
        while not self.stop_evt.is_set():
            try:
                sm = n.nvmlDeviceGetClockInfo(self.handle, n.NVML_CLOCK_SM)
                smax = n.nvmlDeviceGetMaxClockInfo(self.handle, n.NVML_CLOCK_SM)
                r = n.nvmlDeviceGetCurrentClocksEventReasons(self.handle)
                self.samples.append((float(sm), float(smax), [nm for nm, b in zip(self.NAMES, bits) if r & b]))
            except Exception:
                pass
            self.stop_evt.wait(0.01)

    def start(self):
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_evt.set()
            self.thread.join(timeout=5)
            sm = [x[0] for x in self.samples]
            smax = [x[1] for x in self.samples]
            reasons = sorted({r for x in self.samples for r in x[2]})
            return {"sm_mhz": float(np.median(sm)) if sm else None,
                    "sm_max_mhz": max(smax) if smax else None,
                    "reasons": reasons, "samples": len(sm), "source": "nvml"}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "nvml_error": self.err}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(self.NAMES, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi",
                "nvml_error": self.err}


# ---------------------------------------------------------------- oracle arm
def oracle_run(it):
    """One oracle call (Alg. 1 in FP64 plus certification) on the item."""
    from oracle import ffcz_oracle as O
    t0 = time.perf_counter()
    r = O.correct(it["e0"], it["E"], it["D"])
    ok, _, _ = O.certify(r.e, it["E"], it["D"])
    return time.perf_counter() - t0, r.iters, ok


def cpu_baseline(it):
    from oracle import ffcz_oracle as O
    dt, iters, ok = oracle_run(it)
    n = int(np.prod(it["shape"]))
    return {"value": round(4 * n / dt / 1e9, 4), "unit": "GB/s", "cores": O.workers(),
            "kind": "oracle",
            "sample": f"one full call on the {it['name']} field (FP64 loop, {iters} iterations, "
                      f"+ certification{' ok' if ok else ' FAILED'}), {dt:.1f} s"}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    it = make_workload(args.workload)
    n = int(np.prod(it["shape"]))
    for _ in range(args.warmup):
        oracle_run(it)
    times = []
    for _ in range(args.steps):
        dt, iters, ok = oracle_run(it)
        times.append(dt)
    from oracle import ffcz_oracle as O
    ms = 1e3 * float(np.mean(times))
    val = 4 * n / (ms / 1e3) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": it["name"], "shape": list(it["shape"]), "eps_s": it["E"],
                   "eps_f": it["D"], "l2": "input larger than L2"},
        "cpu_baseline": {"value": round(val, 4), "unit": "GB/s", "cores": O.workers(),
                         "kind": "oracle",
                         "sample": f"full {it['name']} call per step ({iters} iterations)"},
        "e2e": {"value": round(val, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def bytes_per_launch(key, n):
    """Algorithmic HBM bytes of one launch on an n-point item (read + write).

    Packed spectra hold n/2 complex values: 4n bytes in FP32, 8n in FP64."""
    kind, rest = key.split("<")
    prec = int(rest.split(",")[0][1:])
    sb = 4 * n if prec == 32 else 8 * n
    if kind == "xfwd":
        return 4 * n + sb            # float32 e in, spectrum out
    if kind == "xexit":
        return sb + 4 * n
    if kind == "chk_cert":
        return sb                    # read only
    return 2 * sb                    # px, axis_*, chk: spectrum in and out


def fft_flops_per_point(L):
    """Algorithmic real operations per complex point of one length-L
    transform, a conventional count independent of the kernels' schedule
    (radix-8 stages, one or two radix-4 stages first): radix-8 butterfly 56
    flops per 8 points, radix-4 16 per 4, twiddle products 6 flops each for
    all but one input of every stage after the first."""
    lg = int(round(math.log2(L)))
    a, b = divmod(lg, 3)
    radices = [8] * a if b == 0 else ([4] + [8] * a if b == 2 else [4, 4] + [8] * (a - 1))
    f = 0.0
    for i, r in enumerate(radices):
        f += 7.0 if r == 8 else 4.0
        if i > 0:
            f += 6.0 * (r - 1) / r
    return f


def flops_per_launch(key, n):
    """Algorithmic floating-point work of one launch on an n-point 2D/3D item
    (n/2 packed complex points)."""
    kind, rest = key.split("<")
    L = int(rest.split(",")[1].rstrip(">"))
    pts = n / 2
    f = fft_flops_per_point(L)
    if kind in ("xfwd", "xexit"):
        f += 16.0                      # R2C / C2R pre- or post-processing
    elif kind == "px":
        f = 2 * f + 32.0
    elif kind in ("chk", "chk_adj"):
        f = 2 * f
    return f * pts


def _timed(torch, fn, reps=2, warm=1):
    for _ in range(warm):
        fn()
    out = []
    for _ in range(reps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out)), r


def _batch_form(ffcz, torch, items, name, rank=0, world=1, dist=None):
    """One batched call over the items (each item's own loop, Alg. 1 per
    item).  With N ranks the items are spread over the GPUs by
    ``shard_items`` (no data crosses ranks); the step time is the slowest
    rank's and the throughput all items' bytes over it."""
    all_bytes = 4 * sum(int(x["e0"].size) for x in items)
    if world > 1:
        items = [items[i] for i in shard_items([4 * int(x["e0"].size) for x in items], rank, world)]
    shapes = [x["shape"] for x in items]
    host = np.concatenate([x["e0"].reshape(-1) for x in items])
    d0 = torch.from_numpy(host).cuda()
    d = torch.empty_like(d0)
    Es = [x["E"] for x in items]
    Ds = [x["D"] for x in items]
    plan = ffcz.Plan(shapes)
    desc = plan.describe().strip()

    def call():
        d.copy_(d0)
        return plan.correct(d, Es, Ds)

    call()
    ms_total, st = _timed(torch, lambda: plan.correct(d.copy_(d0), Es, Ds))
    copy_ms, _ = _timed(torch, lambda: d.copy_(d0))
    ms = ms_total - copy_ms
    iters = [x["iters"] for x in st]
    if world > 1 and dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    byts = all_bytes
    del plan
    return {"workload": name, "items": len(items), "ranks": world, "field_bytes": int(byts),
            "ms_per_call": round(ms, 3), "GBps": round(byts / (ms / 1e3) / 1e9, 3),
            "ms_device": round(float(st[0]["ms_total"]), 3),
            "iters_min": int(min(iters)), "iters_max": int(max(iters)),
            "iters_mean": round(float(np.mean(iters)), 3),
            "certified": int(sum(x["certified"] for x in st)),
            "ms_cert": round(float(st[0]["ms_cert"]), 3), "variants": desc}


def aggregate_ranks(torch, dist, local_ms, bytes_per_rank, world, device="cpu"):
    """Whole-job figure of N replicas (one process per GPU, each doing the same
    step): the step time is the MAX over ranks, the value the bytes all ranks
    processed divided by it (GB/s).  ``dist`` is torch.distributed or None."""
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * bytes_per_rank / (ms / 1e3) / 1e9


def shard_items(nbytes, rank, world):
    """Items of a batched workload for one rank when a batch is spread over
    GPUs: greedy bin packing by bytes (largest first onto the least loaded
    rank); every item lands on exactly one rank and no data crosses ranks."""
    order = sorted(range(len(nbytes)), key=lambda i: (-nbytes[i], i))
    load = [0] * world
    owner = [0] * len(nbytes)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += nbytes[i]
    return [i for i in range(len(nbytes)) if owner[i] == rank]


def paper_design_cufft(torch, it, D, hbm, K=20):
    """Bench-only comparator (not on the product path): the paper's loop body
    as separate library kernels on the same B300 -- cuFFT R2C (torch.fft),
    CheckConvergence (one max-reduction), ProjectOntoFCube (clamp of Re and
    Im in place), cuFFT C2R with 1/N, ProjectOntoSCube (clamp) -- timed over
    K forced iterations with CUDA events and no per-iteration host check."""
    shape, E = it["shape"], it["E"]
    e = torch.from_numpy(it["e0"]).cuda()
    Es, Ds = float(E) * (1 - 2.0 ** -16), float(D) * (1 - 2.0 ** -16)

    def body():
        X = torch.fft.rfftn(e)
        Xr = torch.view_as_real(X)
        v = torch.linalg.vector_norm(Xr, ord=float("inf"))
        Xr.clamp_(-Ds, Ds)
        e.copy_(torch.fft.irfftn(X, s=shape))
        e.clamp_(-Es, Es)
        return v

    for _ in range(3):
        body()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(K):
        body()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    design = 32.0 * int(np.prod(shape))   # 4-pass fused design: 4 x (read + write 4 bytes/point)
    return {"workload": it["name"] + " stress bounds, K forced iterations",
            "kernels": "cuFFT R2C, max-reduce, clamp Re/Im, cuFFT C2R (+1/N), clamp",
            "ms_per_iteration": round(ms, 4),
            "frac_hbm_of_fused_design_bytes": round(design / (ms / 1e3) / 1e9 / hbm, 4),
            "iterations": K}


def edits_form(ffcz, torch, it, D):
    """Alg. 1 edits on the stress variant: the call with edit recording vs
    without, CompactEdits + QuantizeEdits (m = 16), and the decompression
    side x_hat += S~ + IFFT(F~) (CUDA events; median of 2 after 1 warm-up)."""
    shape, E = it["shape"], it["E"]
    n = int(np.prod(shape))
    d0 = torch.from_numpy(it["e0"].reshape(-1)).cuda()
    d = torch.empty_like(d0)
    plain = ffcz.Plan([shape])
    ms_plain, _ = _timed(torch, lambda: plain.correct(d.copy_(d0), [E], [D]))
    del plain
    plan = ffcz.Plan([shape], edits=1)
    ms_edits, st = _timed(torch, lambda: plan.correct(d.copy_(d0), [E], [D])[0])
    copy_ms, _ = _timed(torch, lambda: d.copy_(d0))
    ms_compact, stored = _timed(torch, lambda: plan.edits_compact(16))
    xhat = torch.zeros_like(d0)
    ms_apply, _ = _timed(torch, lambda: plan.apply_edits(xhat, [E], [D], stored, 16))
    ns, nf = (int(v) for v in stored["counts"][0])
    tot = plan.edit_layout(-1)
    stored_bytes = tot[2] + tot[4] + 2 * ns + 4 * nf      # flags + 16-bit codes (Re, Im for bins)
    del plan
    return {"workload": it["name"] + " stress bounds, edits recorded",
            "iters": st["iters"], "ms_correct_plain": round(ms_plain - copy_ms, 3),
            "ms_correct_with_edits": round(ms_edits - copy_ms, 3),
            "ms_compact_quantize": round(ms_compact, 3), "ms_apply": round(ms_apply, 3),
            "spatial_edits": ns, "frequency_edits": nf,
            "stored_bytes_before_lossless": int(stored_bytes),
            "field_bytes": 4 * n}


def pointwise_form(ffcz, torch, it, D, hbm, K=20):
    """Pointwise bounds (ffcz_correct_pw) on the stress variant: per-iteration
    time from K forced iterations minus 0, and its fraction of the HBM peak
    for the 4-pass traffic plus the bound reads (E_n in the x pass, the
    (Delta^Re, Delta^Im) pairs in the check pass): 40N bytes per iteration."""
    shape, E = it["shape"], it["E"]
    n = int(np.prod(shape))
    d0 = torch.from_numpy(it["e0"].reshape(-1)).cuda()
    d = torch.empty_like(d0)
    eb = torch.full((n,), float(E), dtype=torch.float32, device="cuda")
    out = {}
    kernels = {}
    for k in (K, 0):
        plan = ffcz.Plan([shape], pointwise=1, min_iters=k, max_iters=k, certify=0)
        nb = plan.edit_layout(-1)[1]
        db = torch.full((2 * nb,), float(D), dtype=torch.float32, device="cuda")
        ms, st = _timed(torch, lambda: plan.correct_pw(d.copy_(d0), eb, db)[0], reps=3)
        out[k] = (ms, st)
        if k == K:
            # one call with every launch timed by CUDA events (direct launches,
            # outside the graph): the per-kernel split of the iteration
            plan.profile(True)
            plan.correct_pw(d.copy_(d0), eb, db)
            torch.cuda.synchronize()
            kernels = {name: {"ms_per_launch": round(tms / cnt, 4), "launches": cnt}
                       for name, (tms, cnt) in plan.profile_table().items()}
            plan.profile(False)
        del plan, db
    it_ms = (out[K][0] - out[0][0]) / K
    design = 40.0 * n
    return {"workload": it["name"] + " stress bounds as uniform pointwise arrays",
            "forced_iters": K, "ms_per_iteration": round(it_ms, 4),
            "design_bytes": int(design),
            "frac_hbm_design": round(design / (it_ms / 1e3) / 1e9 / hbm, 4),
            "kernels": kernels}


def fp64_form(ffcz, torch, it, D, K=4):
    """The float32 loop with FP64 certification against an all-FP64 GPU run
    (ffcz_opts.precision = 64: the loop in float64, then the same
    certification) on the stress variant: time to certified feasibility
    (the copy of e0 subtracted), iterations, per-iteration time from K forced
    iterations minus 0, and the largest difference between the two corrected
    fields relative to eps_s."""
    shape, E = it["shape"], it["E"]
    d0 = torch.from_numpy(it["e0"].reshape(-1)).cuda()
    d = torch.empty_like(d0)
    copy_ms, _ = _timed(torch, lambda: d.copy_(d0))
    out, fields = {}, {}
    for prec in (32, 64):
        plan = ffcz.Plan([shape], precision=prec)
        ms, st = _timed(torch, lambda: plan.correct(d.copy_(d0), [E], [D])[0])
        fields[prec] = d.clone()
        del plan
        per = {}
        for k in (K, 0):
            fp = ffcz.Plan([shape], precision=prec, min_iters=k, max_iters=k, certify=0)
            per[k], _ = _timed(torch, lambda: fp.correct(d.copy_(d0), [E], [D])[0])
            del fp
        out[f"fp{prec}_loop"] = {"ms_to_certified": round(ms - copy_ms, 3), "iters": st["iters"],
                                 "certified": st["certified"], "ms_cert": round(st["ms_cert"], 3),
                                 "ms_per_iteration": round((per[K] - per[0]) / K, 4)}
        torch.cuda.empty_cache()
    diff = float((fields[32] - fields[64]).abs().max().item()) / E
    del fields, d, d0
    return {"workload": it["name"] + " stress eps_f = 0.2 max box violation of e0", **out,
            "max_abs_diff_over_eps_s": diff, "forced_iters": K}


def variants_form(ffcz, torch, it, D, hbm, K=20):
    """The projection variants of Sec. III (ffcz_opts.method) on the stress
    variant: time to certified feasibility (the copy of e0 subtracted),
    iterations, the size of the correction relative to e0, and per-iteration
    time from K forced iterations minus 0 against the design traffic (Alg. 1
    32N bytes; Dykstra + the residual spectrum and q read and written 48N;
    Douglas-Rachford + the residual 40N; ADMM + u 40N)."""
    shape, E = it["shape"], it["E"]
    n = int(np.prod(shape))
    d0 = torch.from_numpy(it["e0"].reshape(-1)).cuda()
    d = torch.empty_like(d0)
    copy_ms, _ = _timed(torch, lambda: d.copy_(d0))
    nrm0 = float(torch.linalg.vector_norm(d0.double()))
    design = {"pocs": 32.0, "dykstra": 48.0, "dr": 40.0, "admm": 40.0}
    out = {"workload": it["name"] + " stress eps_f = 0.2 max box violation of e0"}
    for m, bpn in design.items():
        plan = ffcz.Plan([shape], method=m)
        ms, st = _timed(torch, lambda: plan.correct(d.copy_(d0), [E], [D])[0])
        edit = float(torch.linalg.vector_norm((d - d0).double())) / nrm0
        del plan
        per, kernels = {}, {}
        for k in (K, 0):
            plan = ffcz.Plan([shape], method=m, min_iters=k, max_iters=k, certify=0)
            per[k], _ = _timed(torch, lambda: plan.correct(d.copy_(d0), [E], [D])[0], reps=3)
            if k == K:
                # one call with every launch timed by CUDA events (direct
                # launches, outside the graph): the per-kernel split
                plan.profile(True)
                plan.correct(d.copy_(d0), [E], [D])
                torch.cuda.synchronize()
                kernels = {name: {"ms_per_launch": round(tms / cnt, 4), "launches": cnt}
                           for name, (tms, cnt) in plan.profile_table().items()}
                plan.profile(False)
            del plan
        it_ms = (per[K] - per[0]) / K
        out[m] = {"ms_to_certified": round(ms - copy_ms, 3), "iters": st["iters"],
                  "certified": st["certified"], "repairs": st["repairs"],
                  "edit_norm_rel": round(edit, 6), "ms_per_iteration": round(it_ms, 4),
                  "design_bytes": int(design[m] * n),
                  "frac_hbm_design": round(design[m] * n / (it_ms / 1e3) / 1e9 / hbm, 4),
                  "kernels": kernels}
        torch.cuda.empty_cache()
    return out


FORMS = ("stress", "cufft", "edits", "pointwise", "variants", "fp64", "batched_2d", "batched_1d",
         "differentiable")


def measure_forms(ffcz, torch, fin, it, hbm, which=FORMS, rank=0, world=1, dist=None):
    """The stress variant, the batched and the differentiable forms (each a
    median of 2 calls after 1 warm-up; CUDA events on the current stream);
    `which` selects some of them.  The batched forms shard their items over
    the ranks; the others run as replicas."""
    out = {}
    shape, E = it["shape"], it["E"]
    n = int(np.prod(shape))
    if "stress" in which:
        d0 = torch.from_numpy(it["e0"].reshape(-1)).cuda()
        d = torch.empty_like(d0)
        plan = ffcz.Plan([shape])
        Dst = fin["stress_D"]
        ms_total, st = _timed(torch, lambda: plan.correct(d.copy_(d0), [E], [Dst])[0])
        copy_ms, _ = _timed(torch, lambda: d.copy_(d0))
        ms = ms_total - copy_ms
        out["stress_512"] = {"workload": it["name"] + " stress eps_f = 0.2 max box violation of e0",
                             "ms_per_call": round(ms, 3), "GBps": round(4 * n / (ms / 1e3) / 1e9, 3),
                             "iters": st["iters"], "certified": st["certified"],
                             "ms_cert": round(st["ms_cert"], 3)}
        del plan, d, d0
        torch.cuda.empty_cache()
    if "cufft" in which:
        out["paper_design_cufft"] = paper_design_cufft(torch, it, fin["stress_D"], hbm)
        torch.cuda.empty_cache()
    if "edits" in which:
        out["edits_stress_512"] = edits_form(ffcz, torch, it, fin["stress_D"])
        torch.cuda.empty_cache()
    if "pointwise" in which:
        out["pointwise_512"] = pointwise_form(ffcz, torch, it, fin["stress_D"], hbm)
        torch.cuda.empty_cache()
    if "variants" in which:
        out["variants_512"] = variants_form(ffcz, torch, it, fin["stress_D"], hbm)
        torch.cuda.empty_cache()
    if "fp64" in which:
        out["fp64_512"] = fp64_form(ffcz, torch, it, fin["stress_D"])
        torch.cuda.empty_cache()
    if "batched_2d" in which:
        out["batched_2d"] = _batch_form(ffcz, torch, fin["c3"],
                                        "512 diffraction images 171x256^2 + 171x512^2 + 170x1024^2",
                                        rank, world, dist)
        torch.cuda.empty_cache()
    if "batched_1d" in which:
        out["batched_1d"] = _batch_form(ffcz, torch, fin["c4"],
                                        "4096 EEG-like signals, lengths U{1024..65536} (Bluestein)",
                                        rank, world, dist)
        torch.cuda.empty_cache()
    if "differentiable" not in which:
        return out
    # differentiable: K = 50 forced iterations, checkpoint every 10, loss on the
    # log power spectrum of x + e_K (torch.fft in the loss only)
    from paper_2601_01596_b300.autograd import FFCzCorrect, power_spectrum_loss
    c5 = fin["c5"]
    x = torch.from_numpy(c5["x"]).cuda()
    e0 = torch.from_numpy(c5["e0"]).cuda()
    K, m = 50, 10

    def fwd():
        return FFCzCorrect.apply(e0, c5["E"], c5["D"], K, m)

    fwd_ms, _ = _timed(torch, fwd)

    def fwd_bwd():
        ee = e0.clone().requires_grad_(True)
        eK = FFCzCorrect.apply(ee, c5["E"], c5["D"], K, m)
        loss = power_spectrum_loss(x, eK)
        loss.backward()
        return float(loss.item())

    fb_ms, loss = _timed(torch, fwd_bwd)
    # the library's vector-Jacobian product alone (ffcz_correct_backward_ckpt
    # from the forward's checkpoints), without the torch loss and its backward
    from paper_2601_01596_b300.autograd import _plan
    vplan = _plan(tuple(e0.shape), K, m)
    ck = torch.empty(vplan.ckpt_floats(), dtype=torch.float32, device="cuda")
    ek = e0.reshape(-1).clone()
    vplan.correct_ckpt(ek, [c5["E"]], [c5["D"]], ck)
    gvec = torch.ones_like(ek)
    gin = torch.empty_like(ek)
    vjp_ms, _ = _timed(torch, lambda: vplan.backward(e0.reshape(-1), gvec, gin, [c5["E"]], [c5["D"]], ckpt=ck))
    # the same with every step's masks kept by the forward (opts.keep_masks):
    # one forward writing checkpoints and masks, then the adjoint steps alone
    kplan = _plan(tuple(e0.shape), K, m, 1)
    kfwd_ms, _ = _timed(torch, lambda: kplan.correct_ckpt(e0.reshape(-1).clone(), [c5["E"]], [c5["D"]], ck))
    ek = e0.reshape(-1).clone()
    kplan.correct_ckpt(ek, [c5["E"]], [c5["D"]], ck)
    kvjp_ms, _ = _timed(torch, lambda: kplan.backward(e0.reshape(-1), gvec, gin, [c5["E"]], [c5["D"]], ckpt=ck))
    del ck, ek, gvec, gin
    n5 = int(np.prod(c5["shape"]))
    out["differentiable"] = {"workload": c5["name"] + f", K={K} forced iterations, checkpoint every {m}",
                             "forward_ms": round(fwd_ms, 3),
                             "backward_vjp_ms": round(vjp_ms, 3),
                             "vjp_over_forward": round(vjp_ms / fwd_ms, 3),
                             "forward_backward_ms": round(fb_ms, 3),
                             "backward_over_forward": round((fb_ms - fwd_ms) / fwd_ms, 3),
                             "note": "forward_backward includes the float64 torch power-spectrum loss and its backward",
                             "forward_ms_per_iteration": round(fwd_ms / K, 4),
                             "kept_masks": {"forward_ms": round(kfwd_ms, 3), "backward_vjp_ms": round(kvjp_ms, 3),
                                            "forward_plus_vjp_ms": round(kfwd_ms + kvjp_ms, 3),
                                            "replay_forward_plus_vjp_ms": round(fwd_ms + vjp_ms, 3)},
                             "field_GBps_forward": round(4 * n5 / (fwd_ms / 1e3) / 1e9, 3),
                             "loss": loss}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ffcz", choices=["ffcz", "reference"])
    ap.add_argument("--workload", default="lognormal512")
    ap.add_argument("--forced", type=int, default=20, help="forced iterations for the per-iteration roofline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the stress, batched and differentiable forms")
    ap.add_argument("--forms", default=",".join(FORMS),
                    help="comma-separated forms to run: " + ",".join(FORMS))
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    # every input is generated on the host before the first CUDA call
    it = make_workload(args.workload)
    # the labelled stress bound (eps_f = 0.2 max box violation of e0): the
    # per-iteration cost of a field whose clips are active
    stress_D = W.max_box_fft(it["e0"]) * 0.2
    forms_in = None
    which = tuple(f for f in args.forms.split(",") if f)
    unknown = [f for f in which if f not in FORMS]
    if unknown:
        ap.error(f"unknown forms {unknown}; choose from {FORMS}")
    if not args.no_forms and which:
        workers = min(8, os.cpu_count() or 1)
        forms_in = {"stress_D": stress_D}
        if "batched_2d" in which:
            forms_in["c3"] = W.diffraction_batch(workers=workers)
        if "batched_1d" in which:
            forms_in["c4"] = W.eeg_batch(workers=workers)
        if "differentiable" in which:
            forms_in["c5"] = W.turbulence_field(256)

    import torch
    import paper_2601_01596_b300 as ffcz

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    hbm, peak_kind = load_peaks()
    shape, E, D = it["shape"], it["E"], it["D"]
    n = int(np.prod(shape))
    field_bytes = 4 * n
    h_e0 = torch.from_numpy(it["e0"].reshape(-1)).pin_memory()
    d_e0 = h_e0.cuda()
    d_e = torch.empty_like(d_e0)
    plan = ffcz.Plan([shape])
    plan_desc = plan.describe().strip()

    def step():
        return plan.correct(d_e, [E], [D])[0]

    for _ in range(max(3, args.warmup)):
        d_e.copy_(d_e0)
        st = step()
    torch.cuda.synchronize()

    # -- timed region: K calls, events on the launching stream ------------------
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = ffcz.launch_count()
    stats = []
    for k in range(args.steps):
        d_e.copy_(d_e0)
        ev[k][0].record()
        stats.append(step())
        ev[k][1].record()
    torch.cuda.synchronize()
    launches = ffcz.launch_count() - l0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms, value = aggregate_ranks(torch, dist, ms, field_bytes, world, device="cuda")
    st = stats[-1]

    # -- per-kernel profile of the same step (live CUDA events per launch) -----
    plan.profile(True)
    for _ in range(args.steps):
        d_e.copy_(d_e0)
        step()
    torch.cuda.synchronize()
    prof = plan.profile_table()
    plan.profile(False)
    tot = sum(v[0] for v in prof.values())
    top_key, (top_ms, top_n) = max(prof.items(), key=lambda kv: kv[1][0])
    top_avg = top_ms / top_n
    top_bytes = bytes_per_launch(top_key, n)
    traffic, pipe, ncu_note = ncu_figures(top_key, n)
    if "f64" in top_key:
        # FP64 kernels are bound by the FP64 pipe: measured FP64 FMA rate of
        # this GPU (ffcz_fp64_peak), the add-only rate beside it
        fma_tf = ffcz.fp64_peak("fma") / 1e12
        add_tf = ffcz.fp64_peak("add") / 1e12
        top_flops = flops_per_launch(top_key, n)
        ach = top_flops / (top_avg / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": top_key,
                "achieved": round(ach, 4), "peak": round(fma_tf, 4), "unit": "TFLOP/s (FP64)",
                "frac": round(ach / fma_tf, 4),
                "traffic": traffic, "fp64_pipe_active_ncu": pipe, "ncu_note": ncu_note,
                "peak_kind": "measured: FP64 FMA chains on this GPU (ffcz_fp64_peak), 2 flops per FMA",
                "fp64_add_peak_tflops": round(add_tf, 4),
                "fp64_nominal_tflops": FP64_TFLOPS_NOMINAL,
                "avg_launch_ms": round(top_avg, 4), "algorithmic_flops": top_flops,
                "algorithmic_bytes": top_bytes,
                "achieved_GBps": round(top_bytes / (top_avg / 1e3) / 1e9, 1),
                "share_of_step": round(top_ms / tot, 3) if tot else None}
    else:
        roof = {"bound": "hbm", "kernel": top_key,
                "achieved": round(top_bytes / (top_avg / 1e3) / 1e9, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(top_bytes / (top_avg / 1e3) / 1e9 / hbm, 4),
                "traffic": traffic, "ncu_note": ncu_note,
                "peak_kind": peak_kind, "avg_launch_ms": round(top_avg, 4),
                "algorithmic_bytes": top_bytes,
                "share_of_step": round(top_ms / tot, 3) if tot else None}

    # -- per-iteration roofline: forced iterations, no certification -----------
    fplan = ffcz.Plan([shape], min_iters=args.forced, max_iters=args.forced, certify=0)
    zplan = ffcz.Plan([shape], min_iters=0, max_iters=0, certify=0)   # t(0): entry + exit only
    for p_ in (fplan, zplan):
        d_e.copy_(d_e0)
        p_.correct(d_e, [E], [D])
    def per_iter(Dv):
        tf, tz = [], []
        for _ in range(max(2, args.steps)):
            for p_, acc in ((fplan, tf), (zplan, tz)):
                d_e.copy_(d_e0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                p_.correct(d_e, [E], [Dv])
                b.record()
                torch.cuda.synchronize()
                acc.append(a.elapsed_time(b))
        return (float(np.median(tf)) - float(np.median(tz))) / args.forced
    it_ms = per_iter(D)
    it_ms_stress = per_iter(stress_D)   # every clip active: no warp skips its clip arithmetic
    fplan.profile(True)
    d_e.copy_(d_e0)
    fplan.correct(d_e, [E], [D])
    torch.cuda.synchronize()
    fprof = fplan.profile_table()
    fplan.profile(False)
    passes = 4 if len(shape) == 3 else 2
    design = passes * 8 * n                 # each pass reads and writes the packed spectrum
    minimum = 2 * 8 * n                     # two passes: the fewest an nD FFT loop can do
    body = {k: v for k, v in fprof.items() if k.split("<")[0] in ("px", "chk", "axis_fwd", "axis_inv")
            and "f32" in k}
    body_ms = sum(v[0] for v in body.values()) / args.forced
    body_kernels = {}
    for k, (tms, cnt) in body.items():
        # loop-body launches (the entry's axis/chk launch is one of them)
        avg = tms / cnt
        body_kernels[k] = {"ms_per_launch": round(avg, 4), "launches": cnt,
                           "GBps": round(bytes_per_launch(k, n) / (avg / 1e3) / 1e9, 1),
                           "frac_hbm": round(bytes_per_launch(k, n) / (avg / 1e3) / 1e9 / hbm, 4)}

    # -- end to end through the host-buffer entry point -----------------------
    h_work = torch.empty_like(h_e0).pin_memory()
    hw = h_work.numpy()
    src = h_e0.numpy()
    np.copyto(hw, src)
    plan.correct_host(hw, [E], [D])
    e2e_t, e2e_copies = [], []
    for _ in range(args.steps):
        np.copyto(hw, src)
        t0 = time.perf_counter()
        sth = plan.correct_host(hw, [E], [D])
        e2e_t.append(time.perf_counter() - t0)
        e2e_copies.append(sth[0]["host_copies"])
    e2e_ms = 1e3 * float(np.mean(e2e_t))
    e2e_ms_t = torch.tensor([e2e_ms], device="cuda")
    if dist:
        dist.all_reduce(e2e_ms_t, op=dist.ReduceOp.MAX)
    e2e_val = world * field_bytes / (float(e2e_ms_t.item()) / 1e3) / 1e9
    # the same on the labelled stress bound: the field iterates, so every
    # call copies it back (the device-to-host leg of an iterating field)
    np.copyto(hw, src)
    plan.correct_host(hw, [E], [stress_D])
    s2e_t, s2e_copies, s2e_iters = [], [], []
    for _ in range(max(2, args.steps // 2)):
        np.copyto(hw, src)
        t0 = time.perf_counter()
        sth = plan.correct_host(hw, [E], [stress_D])
        s2e_t.append(time.perf_counter() - t0)
        s2e_copies.append(sth[0]["host_copies"])
        s2e_iters.append(sth[0]["iters"])
    s2e_ms_t = torch.tensor([1e3 * float(np.mean(s2e_t))], device="cuda")
    if dist:
        dist.all_reduce(s2e_ms_t, op=dist.ReduceOp.MAX)
    s2e_val = world * field_bytes / (float(s2e_ms_t.item()) / 1e3) / 1e9

    forms = measure_forms(ffcz, torch, forms_in, it, hbm, which, rank, world, dist) if forms_in else None
    if forms and "paper_design_cufft" in forms:
        forms["paper_design_cufft"]["fused_speedup_per_iteration"] = round(
            forms["paper_design_cufft"]["ms_per_iteration"] / it_ms, 3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(it)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": it["name"], "shape": list(shape), "eps_s": E, "eps_f": D,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"input {field_bytes / 1e6:.0f} MB {'>' if field_bytes > 126e6 else '<'} 126 MB L2, no flush",
                   "certify": "fp64",
                   "iters": st["iters"], "certified": st["certified"],
                   "step": "ffcz_correct (loop + FP64 certification), e0 resident in HBM",
                   "variants": plan_desc},
        "e2e": {"value": round(e2e_val, 3), "unit": "GB/s", "h2d_bytes_per_step": field_bytes + 64,
                "d2h_bytes_per_step": int(round(field_bytes * float(np.mean(e2e_copies)))) + 4 + 160,
                "field_copies_back": float(np.mean(e2e_copies)),
                "stress": {"value": round(s2e_val, 3), "unit": "GB/s",
                           "eps_f": stress_D, "iters": int(s2e_iters[-1]),
                           "h2d_bytes_per_step": field_bytes + 64,
                           "d2h_bytes_per_step": int(round(field_bytes * float(np.mean(s2e_copies)))) + 4 + 160,
                           "field_copies_back": float(np.mean(s2e_copies))}},
        "roofline": roof,
        "per_iteration": {"ms": round(it_ms, 4), "body_kernels_ms": round(body_ms, 4),
                          "design_bytes": design, "passes": passes,
                          "design_GBps": round(design / (it_ms / 1e3) / 1e9, 1),
                          "frac_hbm_design": round(design / (it_ms / 1e3) / 1e9 / hbm, 4),
                          "frac_hbm_two_pass_minimum": round(minimum / (it_ms / 1e3) / 1e9 / hbm, 4),
                          "frac_nominal_8TBps": round(design / (it_ms / 1e3) / 8e12, 4),
                          # R2C + C2R per iteration: 2 x 2.5 N log2 N
                          "gflops_achieved": round(5.0 * n * np.log2(n) / (it_ms / 1e3) / 1e9, 1),
                          "stress_ms": round(it_ms_stress, 4),
                          "stress_frac_hbm_design": round(design / (it_ms_stress / 1e3) / 1e9 / hbm, 4),
                          "forced_iters": args.forced, "kernels": body_kernels},
        "kernels": {k: {"ms_per_launch": round(v[0] / v[1], 4), "launches": v[1],
                        "share": round(v[0] / tot, 3)} for k, v in prof.items()},
        "ms_cert": round(st["ms_cert"], 4),
        "clocks": clk,
        "gpu_launches": int(launches),
        "cpu_baseline": cpu,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
