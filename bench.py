#!/usr/bin/env python
"""Benchmark of the SRP-map hot path on one GB300 (or N replicas under torchrun).

Workload (default): M=8 uniform circular array (r=5 cm), 3-D grid of 0.1 m cells over
5x4x3 m (J=60000), N=512 Hann frames, F=2000 frames per step, AR(10) speech-like source
with on/off envelope and 10 dB diffuse noise (synthetic, seeded).  One step computes,
for the whole batch, the maps of conv. FD-SRP, SLRI-SRP (R=16) and SSPI-SRP (t=4 taps
per location and pair), each through the full path (STFT + PHAT, cross-spectra / iFFT
sampling, contraction, argmax).  ``value`` counts every map cell produced: 3 * J * F per
step and rank.  The default precision is FP32-class for every method: FP16 hi+lo on the
tensor cores (three products, FP32 accumulation), whose maps stay within 1e-5 of the FP64
oracle.  A BF16 point of the same step is measured after the timed region and reported
as an extra key (``bf16_point``); ``--precision`` picks another headline precision.

Timing: every step is bracketed by CUDA events on the launching stream, with an L2 flush
(a 512 MB write) before each step outside the events.  Prints one JSON line (rank 0).
``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SRP map cells·frames/s, SLRI/SSPI vs conv FD-SRP at matched error; p50/p99 latency"
UNIT = "cells*frames/s"
FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS = 6800.0, 1900.0
PEAKS_K, PEAKS_DMIN = 4, 0.5  # several-peak estimates timed beside the argmax
FFMA_LANES = 152 * 128  # SMs x FP32 lanes


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libsrp", choices=["libsrp", "reference"])
    ap.add_argument("--workload", default="uca8")
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--cells", type=int, default=None,
                    help="keep the first CELLS grid cells (small profiling captures of a kernel)")
    ap.add_argument("--rank", type=int, default=16, help="SLRI rank R")
    ap.add_argument("--taps", type=float, default=4.0, help="SSPI taps per location and pair")
    ap.add_argument("--precision", default="fp16x3",
                    help="fp32 | bf16 | fp16 | tf32 | bf16x3 | fp16x3 | tf32x3")
    ap.add_argument("--conv-precision", default=None)
    ap.add_argument("--slri-precision", default=None)
    ap.add_argument("--sspi-precision", default=None)
    ap.add_argument("--methods", default="conv,slri,sspi")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-bf16-point", action="store_true",
                    help="skip the extra BF16 measurement of the same step")
    ap.add_argument("--argmax-frames", type=int, default=1024,
                    help="frames whose argmax is compared with the FP64 oracle's")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--clock-ms", type=int, default=20,
                    help="nvidia-smi sampling interval during the timed region (0: no sampling)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the heuristic kernel variants")
    ap.add_argument("--variant", type=int, default=None,
                    help="pin the tensor-core kernel variant of every plan (0..11, as srp_plan_autotune)")
    ap.add_argument("--serving", action="store_true", help="run the serving workload instead")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving run")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the walls16 / nested32 points")
    ap.add_argument("--curve", action="store_true", help="map error vs throughput over R / t")
    ap.add_argument("--sessions", type=int, default=64)
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=62.5, help="serving: frames/s per session")
    ap.add_argument("--serving-precision", default="auto",
                    help="serving: a precision for every session, or auto (FP32 for M <= 8, "
                         "BF16 otherwise)")
    return ap.parse_args(argv)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), \
            d.get("sm_max_mhz", 2070.0), "measured"
    return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, 1700.0, 2070.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, interval_ms=20):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = None
        self.index = index
        self.interval_ms = interval_ms

    def start(self):
        """Starts the sampler (every interval_ms) and returns once it has written its first sample
        (nvidia-smi takes a while to start), so that the timed region that follows is
        sampled from its beginning; mark() then sets where the timed region's samples begin."""
        self.n0 = 0
        if self.interval_ms <= 0:
            return
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms",
                                          str(self.interval_ms)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None and self._lines() < 1:
            time.sleep(0.01)

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for line in f if line.strip())
        except OSError:
            return 0

    def mark(self):
        self.n0 = self._lines() if self.proc is not None else 0

    def stop(self):
        if self.proc is None:
            if getattr(self, "f", None):
                self.f.close()
            if os.path.exists(self.path):
                os.unlink(self.path)
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [line for line in open(self.path) if line.strip()]
        if len(lines) > self.n0:  # the samples taken from the start of the timed region on
            lines = lines[self.n0:]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_seed(base: int, rank: int) -> int:
    """Each rank processes its own batch of frames (weak scaling, no data exchange)."""
    return base + 7919 * rank


def reduce_max(values, world, device):
    if world == 1:
        return values
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


# ------------------------------------------------------------------------------------
class OracleRefs:
    """FP64 oracle maps of sampled frames (CPU), for the error report."""

    def __init__(self, w, R, t):
        import oracle as O
        self.O = O
        self.w = w
        self.fs, self.K = w["fs"], w["N"] // 2
        self.dt = O.tdoa_nf(w["mic_xyz"], w["grid_xyz"])
        self.lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], self.fs))
        self.Lam = O.interp_matrix(self.dt, self.fs, self.lags)
        self.tall, self.fat, _ = O.slri_factors(self.Lam, R)
        self.Lsp = O.sspi_matrix(self.Lam, self.lags, int(round(t * self.Lam.shape[0] * len(self.lags))))

    def maps(self, method, frames, cells=slice(None)):
        """The oracle's maps of `method` for `frames` on the grid cells `cells` (all by
        default), or None where the oracle's factors are out of reach at this size (LR-SRP
        needs the SVD of the whole SRP matrix)."""
        O = self.O
        psi = O.gcc_phat(O.stft(frames, "hann"))
        if method == "conv":
            return O.srp_conv(psi, self.dt[cells], self.fs)
        if method == "lr":
            return None
        xi, _ = O.gcc_samples_ifft(psi, self.lags, self.K)
        if method == "slri":
            return O.srp_slri(self.tall[cells], self.fat, xi)
        if method == "si":
            return O.srp_si(self.Lam[cells], xi)
        if method == "td":
            return xi @ O.td_matrix(self.dt[cells], self.fs, self.lags).T
        return O.srp_sspi(self.Lsp[cells], xi)


def cpu_baseline(refs, frames, stride=1):
    """The FP64 oracle as it stands: per-frame work of all three methods on a bounded
    sample (every `stride`-th grid cell).  The SLRI / SSPI fits are made beforehand, like
    the GPU plans'; the oracle's conv. FD-SRP builds its SRP matrix inside every call."""
    cells = slice(None, None, stride)
    t0 = time.perf_counter()
    out = {m: refs.maps(m, frames, cells) for m in ("conv", "slri", "sspi")}
    el = time.perf_counter() - t0
    J = len(range(refs.w["grid_xyz"].shape[0])[cells])
    try:
        import threadpoolctl
        cores = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or 1
    except Exception:  # no threadpoolctl: the BLAS thread setting, else the usable CPUs
        env = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or ""
        cores = int(env) if env.isdigit() and int(env) > 0 else len(os.sched_getaffinity(0))
    n = frames.shape[0]
    return out, {"value": 3 * J * n / el, "unit": UNIT, "cores": int(cores), "kind": "oracle",
                 "sample": f"{n} frame(s) x {J} cells"
                           + (f" (1 in {stride} of the grid)" if stride > 1 else "")
                           + " x 3 methods: conv. FD-SRP with its SRP matrix H built inside the"
                             " call (the oracle generates H per call), SLRI and SSPI from factors"
                             " fitted beforehand (the SVD and the top-Q selection are not timed)",
                 "seconds": el}


REF_FULL_STEPS = 12


def reference_stride(warmup: int, steps: int) -> int:
    """Grid-cell stride of the reference arm: up to REF_FULL_STEPS warm-up plus timed steps
    take every cell; longer runs take one cell in ceil((W + K) / REF_FULL_STEPS) per step,
    so the whole run does about REF_FULL_STEPS frames of full work."""
    return max(1, -(-(warmup + steps) // REF_FULL_STEPS))


def arm_methods(a):
    methods = [m for m in a.methods.split(",") if m]
    return methods, {m: getattr(a, f"{m}_precision", None) or a.precision for m in methods}


def workload_config(a, M, J, N, F, methods, prec):
    """The benchmark's `config`, shared by both arms (the reference arm times the same
    workload on a bounded sample of it)."""
    return {"workload": f"{a.workload}: M={M}, J={J}, N={N} Hann, F={F} frames/step/rank; "
                        + ", ".join(f"{m} {prec[m]}" for m in methods)
                        + f" (SLRI R={a.rank}, SSPI t={a.taps})",
            "maps_per_frame": len(methods),
            "l2": "flushed before every step (512 MB write, outside the timed events)"
            if not a.no_flush else "not flushed"}


def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import synth
    w = synth.workload(a.workload, F=a.frames)  # the libsrp arm's workload (rank 0)
    methods, prec = arm_methods(a)
    config = workload_config(a, w["mic_xyz"].shape[0], w["grid_xyz"].shape[0], w["N"], w["F"],
                             methods, prec)
    refs = OracleRefs(w, a.rank, a.taps)
    # a bounded run: beyond REF_FULL_STEPS steps, each step takes every stride-th cell, so
    # the whole run does about REF_FULL_STEPS full frames of work (about 2 min on 8 cores)
    stride = reference_stride(a.warmup, a.steps)
    J = len(range(w["grid_xyz"].shape[0])[::stride])
    times = []
    r = None
    for s in range(a.warmup + a.steps):
        f = s % w["F"]
        _, r = cpu_baseline(refs, w["frames"][f:f + 1], stride)
        if s >= a.warmup:
            times.append(r["seconds"])
    ms = 1e3 * float(np.mean(times))
    value = 3 * J / (ms / 1e3)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                            "sample": "per step: " + r["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------
def measured_traffic(workload, F, method, prec):
    """DRAM bytes (read + write) per launch of the method's contraction from the committed
    ncu capture (profiles/traffic_*.json), or None when there is no capture of this launch
    or its kernel source changed since (sha256 mismatch)."""
    import glob
    import hashlib
    key = f"{workload}:F{F}:{method}:{prec}"
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "traffic_*.json"))):
        try:
            d = json.load(open(path))
        except Exception:
            continue
        rec = d.get("launches", {}).get(key)
        if not rec:
            continue
        src = rec["source"]
        want = d.get("sources_sha256", {}).get(src)
        try:
            have = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
        except OSError:
            return None
        if want != have:
            return None
        return rec["dram_read"] + rec["dram_write"]
    return None


def contraction_work(m, prec, info, F, R):
    """(kind, amount per launch) of the dominant kernel of method m: the algorithm's FLOPs
    of the contraction, 2JP(K-1) real MACs per frame for conv. FD-SRP (Eq. SRPomp) whatever
    the precision, or the bytes of the map write that bounds SLRI / SSPI."""
    J, P, K, L = info.J, info.P, info.K, info.L
    if m == "conv":
        return "flop", 4.0 * J * P * (K - 1) * F
    if m == "slri":
        return "byte", 4.0 * J * F  # the map write; 2R(J+L) flop per frame is far below
    if m == "sspi":
        if prec == "fp32":
            return "flop", 2.0 * info.nnz * F
        return "byte", 4.0 * J * F
    return "byte", 4.0 * J * F


def contraction_peak(prec, kind, peaks_):
    """(peak, unit, bound, source) the dominant kernel is measured against.  A hi+lo split
    runs three products per algorithmic MAC, so its peak in algorithmic FLOP/s is the
    operand type's tensor rate / 3.  Kernels timed per step (a few ms, L2 flushed between
    steps) take the burst figure."""
    hbm, bf16, _bf16s, smmax, src = peaks_
    if kind == "byte":
        return hbm, "GB/s", "hbm", f"{src} copy"
    if prec == "fp32":
        return (FFMA_LANES * 2 * smmax * 1e6 / 1e12, "TFLOP/s", "alu",
                "derived: 152 SMs x 128 FP32 FMA/clk x 2 x max SM clock")
    split = 3.0 if prec.endswith("x3") else 1.0
    if prec.startswith("tf32"):
        # no TF32 peak is measured: the measured BF16 burst x the nominal ratio 1.1 / 2.25
        base, what = bf16 * 1.1 / 2.25, f"{src} bf16 burst x 1.1/2.25 (nominal TF32 / BF16 dense rates)"
    else:
        base, what = bf16, f"{src} bf16 burst (FP16 runs at the BF16 rate)"
    if split > 1:
        what += " / 3 (hi+lo: three products per algorithmic MAC)"
    return base / split, "TFLOP/s", "tensor", what


def roofline_of(dom, prec, info, F, R, t_launch, peaks_):
    """The roofline object of the dominant kernel: algorithmic work per launch over the
    launch's CUDA-event duration, against the matching peak."""
    kind, work = contraction_work(dom, prec, info, F, R)
    peak, unit, bound, what = contraction_peak(prec, kind, peaks_)
    achieved = work / t_launch / (1e12 if kind == "flop" else 1e9)
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "peak_source": what, "frac": achieved / peak,
            "work_per_launch": {"kind": kind, "amount": work}}


def grid_pitch(grid_xyz):
    """Per-axis spacing of a regular grid of cell centres (inf on an axis with one value)."""
    h = []
    for ax in range(3):
        u = np.unique(np.round(np.asarray(grid_xyz)[:, ax], 9))
        h.append(float(np.min(np.diff(u))) if len(u) > 1 else np.inf)
    return np.array(h)


TIE_REL = 1e-9


def argmax_report(idx, ref, grid_xyz):
    """Agreement of per-frame estimates `idx` with the maxima of the FP64 maps `ref`
    [frames][J] (Eq. imax).  A map can hold several exact maxima (the uca8 array lies in a
    mirror plane of its grid, so every map has mirror-image twins): the oracle's maxima are
    the cells within TIE_REL of its peak height above the map's median -- ties in exact
    arithmetic that FP64 rounding resolves arbitrarily.  Reported: the exact index, the
    pick being one of the oracle's maxima, the pick within one grid cell (on every axis)
    of one of them, its distance in metres to the nearest, and the map value lost at the
    pick relative to the peak's height above the median."""
    idx = np.asarray(idx, np.int64)
    g = np.asarray(grid_xyz, float)
    h = grid_pitch(g)
    r = np.arange(len(idx))
    io = np.argmax(ref, axis=1)
    top = ref[r, io]
    prom = np.maximum(top - np.median(ref, axis=1), 1e-300)
    gap = (top - ref[r, idx]) / prom
    cells = np.empty(len(idx))
    metres = np.empty(len(idx))
    for f in range(len(idx)):
        ties = np.flatnonzero(ref[f] >= top[f] - TIE_REL * prom[f])
        d = g[ties] - g[idx[f]]
        cells[f] = np.min(np.max(np.abs(d) / h[None, :], axis=1))
        metres[f] = np.min(np.linalg.norm(d, axis=1))
    return {"frames": int(len(idx)), "exact_index": float(np.mean(idx == io)),
            "agree_up_to_ties": float(np.mean(gap <= TIE_REL)),
            "within_one_cell": float(np.mean(cells <= 1.0 + 1e-6)),
            "dist_m_median": float(np.median(metres)),
            "dist_m_p99": float(np.percentile(metres, 99)), "dist_m_max": float(metres.max()),
            "peak_gap_median": float(np.median(gap)), "peak_gap_max": float(gap.max())}


PLAN_KW = {"conv": lambda a: dict(method="conv"), "slri": lambda a: dict(method="slri", rank=a.rank),
           "sspi": lambda a: dict(method="sspi", taps=a.taps), "si": lambda a: dict(method="si"),
           "td": lambda a: dict(method="td"), "lr": lambda a: dict(method="lr", rank=a.rank)}


def make_plans(S, a, w, methods, prec, F):
    """One plan per method at its precision, each tuned (tile shape) for batches of F."""
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    plans = {m: S.Plan(*args, max_frames=F, precision=prec[m], **PLAN_KW[m](a)) for m in methods}
    if a.variant is not None:
        for m in methods:
            plans[m].set_variant(a.variant)
        return plans, {m: {"variant": a.variant, "pinned": True} for m in methods}
    tuned = {m: plans[m].autotune(F) for m in methods} if not a.no_autotune else {}
    return plans, tuned


def per_method(plans, methods, prec, steps, J, F):
    """Per-method stage times (CUDA events on the launching stream, averaged per step)."""
    per = {}
    for m in methods:
        st = plans[m].stage_ms()
        ms_m = sum(st[k] for k in ("frontend", "spectra", "contract", "argmax")) / steps
        per[m] = {"precision": prec[m], "ms_per_step": ms_m, "cells_frames_per_s": J * F / (ms_m / 1e3),
                  "stage_ms": {k: st[k] / steps for k in ("frontend", "spectra", "contract", "argmax")}}
    return per


def dominant(per, methods):
    return max(methods, key=lambda m: per[m]["stage_ms"]["contract"])


def kernel_name(dom, p):
    tc = p != "fp32"
    return {"conv": "tc_gemm_kernel (conv SRP matrix)" if tc else "sgemm_nt_argmax_kernel",
            "slri": "SLRI fat + pack + tc_gemm_kernel" if tc else "SLRI fat + tall",
            "sspi": "SSPI pack + tc_gemm_kernel" if tc else "sspi_kernel",
            }.get(dom, f"{dom} contraction ({'tc_gemm_kernel' if tc else 'sgemm_nt_argmax_kernel'})")


def speedups(per):
    out = {}
    for m in ("slri", "sspi", "si", "td", "lr"):
        if "conv" in per and m in per:
            out[f"speedup_{m}_vs_conv"] = per[m]["cells_frames_per_s"] / per["conv"]["cells_frames_per_s"]
    return out


def extra_point(S, a, w, methods, precision, frames, stream, flush, peaks_, steps=8, warmup=3):
    """The same step at another precision, measured after the timed region (L2 flushed
    before every step, CUDA events): its throughput, per-method times and roofline.
    Returns (summary, maps, argmax) with the maps kept for the error report."""
    import torch
    F, J = w["F"], w["grid_xyz"].shape[0]
    prec = {m: precision for m in methods}
    plans, tuned = make_plans(S, a, w, methods, prec, F)
    maps = {m: torch.empty((F, J), dtype=torch.float32, device=frames.device) for m in methods}
    am = {m: torch.empty((F,), dtype=torch.int32, device=frames.device) for m in methods}
    for _ in range(warmup):
        for m in methods:
            plans[m].map(frames, maps[m], am[m], stream=stream)
    torch.cuda.synchronize()
    for m in methods:
        plans[m].status()
        plans[m].set_profiling(True)
    tot = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for m in methods:
            plans[m].map(frames, maps[m], am[m], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    per = per_method(plans, methods, prec, steps, J, F)
    ms = tot / steps
    dom = dominant(per, methods)
    roof = roofline_of(dom, precision, plans[dom].info, F, a.rank,
                       per[dom]["stage_ms"]["contract"] / 1e3, peaks_)
    roof["kernel"] = kernel_name(dom, precision)
    for m in methods:
        plans[m].set_profiling(False)
        plans[m].status()
        plans[m].close()
    out = {"precision": precision, "steps": steps, "warmup": warmup, "ms_per_step": ms,
           "value": len(methods) * J * F / (ms / 1e3), "methods": per, "autotune": tuned,
           "roofline": roof, **speedups(per)}
    return out, maps, am


# The other workloads, measured after the headline (the default run includes them): each
# point is (method, precision, plan keywords, frames timed), on the workload's frames.
OTHER_WORKLOADS = [
    ("walls16", 1024, [("conv", "bf16", {}, None), ("conv", "fp16x3", {}, None),
                       ("slri", "bf16", {"rank": 16}, None), ("slri", "fp16x3", {"rank": 16}, None),
                       ("sspi", "bf16", {"taps": 4.0}, None)]),
    ("nested32", 1024, [("conv", "fp32", {}, 64), ("conv", "fp16x3", {}, None),
                        ("conv", "bf16", {}, None), ("slri", "bf16", {"rank": 16}, None),
                        ("slri", "bf16", {"rank": 64}, None), ("sspi", "bf16", {"taps": 8.0}, None)]),
]


def other_workloads(a, S, stream, flush, pk, steps=3):
    """The large workloads (16 wall microphones, N = 1024, J = 72000; 32 microphones on two
    nested circles, N = 2048, J = 240000) at a batch of 1024 frames: per point the plan is
    built (fit included, not timed), tuned, warmed once, and `steps` steps are timed with
    CUDA events (L2 flushed before each).  On the 32-microphone grid the SRP matrix is not
    stored: conv. FD-SRP in FP32 generates it inside the GEMM (timed on the first 64
    frames), on the tensor cores it is generated in chunks of cells."""
    import torch
    import synth
    out = {}
    for name, F, points in OTHER_WORKLOADS:
        t0 = time.perf_counter()
        w = synth.workload(name, F=F)
        J = w["grid_xyz"].shape[0]
        frames_all = torch.from_numpy(w["frames"]).cuda()
        rows = []
        fits = {}  # (method, rank / taps) -> a saved plan: later precisions read the fit back
        tmpdir = tempfile.mkdtemp()
        for method, prec, kw, nf in points:
            n = nf or F
            frames = frames_all[:n].contiguous()
            tb = time.perf_counter()
            fit_key = (method, tuple(sorted(kw.items())))
            plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method=method,
                          precision=prec, max_frames=n, plan_file=fits.get(fit_key), **kw)
            build_s = time.perf_counter() - tb
            if method in ("slri", "sspi") and fit_key not in fits:
                fits[fit_key] = os.path.join(tmpdir, f"{method}_{len(fits)}.plan")
                plan.save(fits[fit_key])
            if method != "conv":  # conv keeps the heuristic's variant (calls of seconds)
                plan.autotune(n)
            maps = torch.empty((n, J), dtype=torch.float32, device="cuda")
            am = torch.empty((n,), dtype=torch.int32, device="cuda")
            tw = time.perf_counter()
            plan.map(frames, maps, am, stream=stream)
            torch.cuda.synchronize()
            nsteps = steps if time.perf_counter() - tw < 0.5 else 1
            plan.status()
            plan.set_profiling(True)
            tot = 0.0
            for _ in range(nsteps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.map(frames, maps, am, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            st = plan.stage_ms()
            plan.set_profiling(False)
            plan.status()
            ms = tot / nsteps
            stage = {k: st[k] / nsteps for k in ("frontend", "spectra", "contract", "argmax")}
            roof = roofline_of(method, prec, plan.info, n, kw.get("rank", 0),
                               stage["contract"] / 1e3, pk)
            rows.append({"method": method, "precision": prec, **kw, "frames": n, "steps": nsteps,
                         "ms_per_step": ms, "cells_frames_per_s": J * n / (ms / 1e3),
                         "stage_ms": stage, "plan_build_s": build_s, "roofline": roof})
            plan.close()
            del maps, am
        conv = {r["precision"]: r["cells_frames_per_s"] for r in rows if r["method"] == "conv"}
        for r in rows:
            if r["method"] != "conv" and conv:
                ref = conv.get(r["precision"]) or max(conv.values())
                r["speedup_vs_conv"] = r["cells_frames_per_s"] / ref
        for path in fits.values():
            os.unlink(path)
        os.rmdir(tmpdir)
        out[name] = {"F": F, "J": J, "M": int(w["mic_xyz"].shape[0]), "N": int(w["N"]),
                     "points": rows, "seconds": time.perf_counter() - t0}
        del frames_all
        torch.cuda.empty_cache()
    return out


def oracle_report(a, w, methods, variants):
    """Each variant's maps against the FP64 oracle of the same method: the relative map
    error over 32 frames spread over the batch, and the argmax agreement (exact, within
    one grid cell, distance in metres) over `a.argmax_frames` frames.  `variants` maps a
    name to (precision per method, host maps accessor, host argmax per method)."""
    import oracle as O
    F = w["F"]
    sel_arg = np.unique(np.linspace(0, F - 1, min(F, a.argmax_frames)).astype(int))
    sel_err = sel_arg[np.unique(np.linspace(0, len(sel_arg) - 1, min(32, len(sel_arg))).astype(int))]
    pos_err = np.searchsorted(sel_arg, sel_err)
    refs = OracleRefs(w, a.rank, a.taps)
    rep = {v: {} for v in variants}
    rc = None
    for m in methods:
        ref = refs.maps(m, w["frames"][sel_arg])
        if m == "conv":
            rc = ref
        for v, (prec, get_maps, idx) in variants.items():
            if ref is None:
                rep[v][m] = {"frames_checked": 0, "note": "no FP64 oracle factors at this size"}
                continue
            z = get_maps(m, sel_err).astype(np.float64)
            rel = O.rel_err(z, ref[pos_err], axis=-1)
            rep[v][m] = {"precision": prec[m], "frames_checked": int(len(sel_err)),
                         "rel_err_max": float(rel.max()), "rel_err_median": float(np.median(rel)),
                         "argmax": argmax_report(idx[m][sel_arg], ref, w["grid_xyz"])}
            if m != "conv" and rc is not None:
                rep[v][m]["eps_z_vs_conv_db"] = float(np.median(O.eps_db(ref[pos_err], rc[pos_err], axis=-1)))
    return refs, rep


def run_libsrp(a):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_2306_08514_gb300 as S
    import synth

    w = synth.workload(a.workload, F=a.frames, seed=None if rank == 0 else shard_seed(1002, rank))
    if a.cells:
        w["grid_xyz"] = w["grid_xyz"][:a.cells]
    F, J, N, M = w["F"], w["grid_xyz"].shape[0], w["N"], w["mic_xyz"].shape[0]
    methods, prec = arm_methods(a)
    plans, tuned = make_plans(S, a, w, methods, prec, F)
    frames = torch.from_numpy(w["frames"]).to(dev)
    maps = {m: torch.empty((F, J), dtype=torch.float32, device=dev) for m in methods}
    am = {m: torch.empty((F,), dtype=torch.int32, device=dev) for m in methods}
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)

    def step():
        for m in methods:
            plans[m].map(frames, maps[m], am[m], stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    for m in methods:
        plans[m].status()
        plans[m].set_profiling(True)
    launches0 = {m: plans[m].info_now().launches for m in methods}
    clocks = Clocks(local, a.clock_ms)
    if rank == 0:
        clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    if rank == 0:
        clocks.mark()
    t0 = time.perf_counter()
    for e0, e1 in ev:
        if not a.no_flush:
            flush.fill_(1.0)  # L2 flush, outside the events
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop() if rank == 0 else None
    dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / a.steps
    launches = sum(plans[m].info_now().launches - launches0[m] for m in methods)
    per = per_method(plans, methods, prec, a.steps, J, F)
    for m in methods:
        plans[m].set_profiling(False)
        plans[m].status()
    dev_ms, wall = reduce_max([dev_ms, wall], world, dev)

    # estimates only (srp_map with maps = NULL: argmax per frame, no map written)
    for m in methods:
        for _ in range(2):
            plans[m].map(frames, None, am[m], stream=stream, want_maps=False)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(5):
            plans[m].map(frames, None, am[m], stream=stream, want_maps=False)
        q1.record(stream)
        torch.cuda.synchronize()
        per_est = q0.elapsed_time(q1) / 5
        per[m]["estimates_only_ms"] = per_est
        per[m]["estimates_only_frames_per_s"] = F / (per_est / 1e3)
        # several peaks per frame (srp_map_peaks: 4 picks at least 0.5 m apart), with the
        # maps written and estimates only (maps through L2-sized plan scratch)
        for want, key in ((True, "peaks_ms"), (False, "peaks_estimates_only_ms")):
            pk_maps = maps[m] if want else None
            plans[m].peaks(frames, PEAKS_K, PEAKS_DMIN, maps=pk_maps, want_maps=want, stream=stream)
            q0.record(stream)
            for _ in range(5):
                plans[m].peaks(frames, PEAKS_K, PEAKS_DMIN, maps=pk_maps, want_maps=want, stream=stream)
            q1.record(stream)
            torch.cuda.synchronize()
            per[m][key] = q0.elapsed_time(q1) / 5
        per[m]["peaks"] = {"K": PEAKS_K, "d_min_m": PEAKS_DMIN,
                           "estimates_only_frames_per_s": F / (per[m]["peaks_estimates_only_ms"] / 1e3)}
    for m in methods:  # the maps of the last full step are restored for the error report
        plans[m].map(frames, maps[m], am[m], stream=stream)
    torch.cuda.synchronize()

    # e2e through the host-buffer entry point (H2D frames + D2H maps inside the timing): a
    # step is one srp_map_host call per method, the calls issued together from one host
    # thread each on streams of their own (srp_map_host returns once its maps are on the
    # host), so that one method's computation overlaps another's map copies
    import concurrent.futures as cf
    hframes = torch.from_numpy(w["frames"]).pin_memory()
    hmaps = {m: torch.empty((F, J), dtype=torch.float32).pin_memory() for m in methods}
    ham = {m: torch.empty((F,), dtype=torch.int32).pin_memory() for m in methods}
    hstreams = {m: torch.cuda.Stream(device=dev) for m in methods}
    pool = cf.ThreadPoolExecutor(max_workers=len(methods),
                                 initializer=torch.cuda.set_device, initargs=(dev,))

    def e2e_step():
        futs = [pool.submit(plans[m].map_host, hframes, hmaps[m], ham[m], hstreams[m])
                for m in methods]
        for f in futs:
            f.result()

    e2e_step()  # warm the staging buffers
    e2e_steps = max(1, min(a.steps, 3))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    pool.shutdown()
    e2e_s = reduce_max([e2e_s], world, dev)[0]

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cells = len(methods) * J * F * world
    value = cells / (dev_ms / 1e3)
    pk = peaks()

    # dominant kernel: the contraction with the largest time (its CUDA-event duration on the
    # launching stream, per launch; one launch per method and step)
    dom = dominant(per, methods)
    roof = roofline_of(dom, prec[dom], plans[dom].info, F, a.rank,
                       per[dom]["stage_ms"]["contract"] / 1e3, pk)
    roof["traffic"] = measured_traffic(a.workload, F, dom, prec[dom])
    roof["kernel"] = kernel_name(dom, prec[dom])

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dev_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "/".join(sorted(set(prec.values()))), "data": "synthetic",
        "config": workload_config(a, M, J, N, F, methods, prec),
        "wall_ms_per_step": 1e3 * wall / a.steps,
        "methods": per,
        "autotune": tuned,
        "roofline": roof,
        "e2e": {"value": cells / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": len(methods) * F * M * N * 4,
                "d2h_bytes_per_step": len(methods) * F * (J * 4 + 4),
                "how": "srp_map_host per method (pinned host frames in, maps and argmax out), "
                       "the methods' calls concurrent on their own streams, wall clock"},
        "gpu_launches": launches // a.steps * a.steps,
        "clocks": ck,
        **speedups(per),
    }
    for m in methods:  # the e2e staging buffers are no longer needed
        plans[m].close()
    del hmaps, ham

    bmaps = bam = None
    variants = {"headline": (prec, lambda m, s: maps[m][torch.from_numpy(s).to(dev)].cpu().numpy(),
                             {m: am[m].cpu().numpy() for m in methods})}
    if world == 1 and not a.no_bf16_point and any(p != "bf16" for p in prec.values()):
        bp, bmaps, bam = extra_point(S, a, w, methods, "bf16", frames, stream, flush, pk)
        out["bf16_point"] = bp
        variants["bf16_point"] = ({m: "bf16" for m in methods},
                                  lambda m, s: bmaps[m][torch.from_numpy(s).to(dev)].cpu().numpy(),
                                  {m: bam[m].cpu().numpy() for m in methods})

    if world == 1 and not (a.no_oracle_check and a.no_cpu_baseline):
        refs = None
        if not a.no_oracle_check:
            refs, rep = oracle_report(a, w, methods, variants)
            out["vs_oracle"] = rep["headline"]
            if "bf16_point" in rep:
                out["bf16_point"]["vs_oracle"] = rep["bf16_point"]
        if not a.no_cpu_baseline:
            refs = refs or OracleRefs(w, a.rank, a.taps)
            _, cb = cpu_baseline(refs, w["frames"][:1])
            out["cpu_baseline"] = {k: v for k, v in cb.items() if k != "seconds"}
    del maps, variants, bmaps, bam
    torch.cuda.empty_cache()
    if world == 1 and not a.no_other_workloads:
        out["other_workloads"] = other_workloads(a, S, stream, flush, pk)
    if world == 1 and not a.no_serving:
        # the serving workload: the full mix of 64 sessions, Poisson arrivals, 5 s
        res = run_serving(a, sessions=64, seconds=5.0)
        res.pop("mix", None)
        out["serving"] = dict(res, note="64 sessions (M in {4, 8, 16, 32}), Poisson 62.5 frames/s "
                                        "each, 5 s")
        # the same mix at four times the real-time rate: launches overlap, so batches carry
        # several frames and grouped launches several sessions
        hi = run_serving(a, sessions=64, seconds=2.0, rate=4 * 62.5)
        hi.pop("mix", None)
        hi.pop("slowest_sessions", None)
        out["serving"]["high_load"] = dict(hi, note="the same 64 sessions at 250 frames/s each, 2 s")
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------------------
def serving_sessions(n, seed=1005, Ms=(4, 8, 16, 32)):
    """Seeded session mix of the serving workload: per session M in Ms (geometries of the
    square4 / uca8 / walls16 / nested32 workloads), J log-uniform in [2500, 100000] (box
    grids over the workload's room, or a plane grid for the square), N in {512, 1024}
    (1024 where the array needs it), hop 256, SLRI (R in {16, 32}) where L <= 768, else
    SSPI (t in {2, 4}); a white source at a random position plus 20 dB sensor noise."""
    import synth
    g = synth.rng(seed)
    out = []
    for i in range(n):
        M = int(g.choice(Ms))
        J = int(round(np.exp(g.uniform(np.log(2500), np.log(100000)))))
        N = int(g.choice([512, 1024]))
        if M == 4:
            mics = synth.mics_square()
            side = int(round(np.sqrt(J)))
            grid = synth.grid_plane((0.0, 0.0), (4.0, 4.0), (side, side))
            room = (4.0, 4.0, 0.0)
        elif M == 8:
            mics = synth.mics_uca(8, 0.05, (2.5, 2.0, 1.5))
            room = (5.0, 4.0, 3.0)
        elif M == 16:
            room = (6.0, 4.0, 3.0)
            mics = synth.mics_walls(g, room)
            N = 1024
        else:
            mics = synth.mics_nested_uca(16, 0.04, 16, 0.12, (2.0, 1.5, 1.25))
            room = (4.0, 3.0, 2.5)
        if M != 4:
            h = (np.prod(room) / J) ** (1.0 / 3.0)
            grid = synth.grid_box((0, 0, 0), room, h)
        d = np.linalg.norm(mics[:, None, :] - mics[None, :, :], axis=-1)
        iu = np.triu_indices(M, 1)
        L = int(np.sum(2 * (np.floor(d[iu] * 16000.0 / 340.0).astype(int) + 2) + 1))
        if L <= 768 and g.uniform() < 0.5:
            kw = dict(method="slri", rank=int(g.choice([16, 32])))
        else:
            kw = dict(method="sspi", taps=float(g.choice([2.0, 4.0])))
        out.append(dict(M=M, mics=mics, grid=grid, N=N, hop=256, kw=kw, room=room,
                        seed=seed * 1000 + i))
    return out


def session_signal(sess, seconds, fs=16000.0):
    import synth
    g = synth.rng(sess["seed"])
    n = int(seconds * fs) + sess["N"]
    lo = np.array([0.3, 0.3, 0.0 if sess["M"] == 4 else 0.3])
    hi = np.maximum(np.array(sess["room"]) - 0.3, lo + 1e-3)
    src = g.uniform(lo, hi)
    x = synth.propagate([(synth.white(g, n), src)], fs, sess["mics"], n)
    x = synth.add_noise_snr(x, g.standard_normal(x.shape), 20.0)
    return np.ascontiguousarray(x.astype(np.float32))


def slowest_sessions(mix, lats, n=6):
    """Per-session p99 frame-to-map latency, the n worst sessions with their shapes."""
    rows = []
    for k, ls in enumerate(lats):
        if not ls:
            continue
        v = np.concatenate(ls) * 1e3
        s = mix[k]
        rows.append({"session": k, "M": s["M"], "J": int(s["grid"].shape[0]), "N": s["N"],
                     "method": s["kw"]["method"], "frames": int(v.size),
                     "p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99)),
                     "max_ms": float(v.max())})
    rows.sort(key=lambda r: -r["p99_ms"])
    return rows[:n]


def session_precision(sess, precision):
    """precision "auto": FP32 on the CUDA cores for the 4- and 8-microphone arrays, whose
    plans use the fused front end and share grouped launches; BF16 on the tensor cores for
    the 16- and 32-microphone arrays (long sample vectors or many pairs)."""
    if precision != "auto":
        return precision
    return "fp32" if sess["M"] <= 8 else "bf16"


def run_serving(a, sessions=64, seconds=10.0, rate=62.5, precision="auto", max_batch=16,
                Ms=(4, 8, 16, 32), quiet=False):
    """Serving workload: `sessions` sessions with Poisson frame arrivals (`rate` frames/s
    each) pushed in real time by a feeder thread, results drained (argmax and latency) by a
    poller thread.  Returns the serving summary."""
    import threading
    import torch
    import paper_2306_08514_gb300 as S
    torch.cuda.set_device(0)
    mix = serving_sessions(sessions, Ms=Ms)
    # hop 256 at 16 kHz: 62.5 frames/s is real time; Poisson counts stay below 1.5x the mean
    # at most 6 s of signal per session; a session that reaches its end starts it again
    sigs = [session_signal(s, min(1.5 * seconds * rate * s["hop"] / 16000.0 + 1.0, 6.0)) for s in mix]
    free, total = torch.cuda.mem_get_info()
    srv = S.Server(hbm_budget=int(0.6 * free), max_sessions=sessions, max_batch=max_batch,
                   streams=8, slots_per_session=3, pending_frames=16 * max_batch)
    t_build = time.perf_counter()
    sids = [srv.open(s["mics"], s["grid"], 16000.0, s["N"], s["hop"],
                     precision=session_precision(s, precision), **s["kw"]) for s in mix]
    while True:
        infos = [srv.session_info(x)["state"] for x in sids]
        if all(st == "active" for st in infos):
            break
        if time.perf_counter() - t_build > 600:
            raise RuntimeError(f"sessions not admitted: {infos}")
        time.sleep(0.05)
    build_s = time.perf_counter() - t_build
    # the first frame of every session (the window of N samples) before the clock starts
    pos = []
    for sid, s, x in zip(sids, mix, sigs):
        srv.push(sid, x[:, :s["N"] - s["hop"]])
        pos.append(s["N"] - s["hop"])
    rng = np.random.default_rng(7)
    events = []
    for k, s in enumerate(mix):
        t = rng.exponential(1.0 / rate)
        while t < seconds:
            events.append((t, k))
            t += rng.exponential(1.0 / rate)
    events.sort()
    Js = [s["grid"].shape[0] for s in mix]
    done = {"frames": 0, "cells": 0}
    stop = threading.Event()

    errors = {}
    lats = [[] for _ in mix]

    def poller():
        while not stop.is_set():
            for k, sid in enumerate(sids):
                try:
                    _, am, idx, lat = srv.poll(sid, max_frames=16 * max_batch, want_maps=False)
                except S.SrpError as e:  # a failed session: record it, keep serving the rest
                    errors.setdefault(k, str(e))
                    continue
                done["frames"] += len(idx)
                done["cells"] += len(idx) * Js[k]
                if len(lat):
                    lats[k].append(lat.copy())
            time.sleep(0.0002)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    srv.reset_stats()
    t0 = S.srp_server_now()
    w0 = time.perf_counter()
    refused = 0
    for t, k in events:
        while S.srp_server_now() < t0 + t:
            time.sleep(0.0001)
        s = mix[k]
        if pos[k] + s["hop"] > sigs[k].shape[1]:
            pos[k] = s["N"] - s["hop"]
        seg = sigs[k][:, pos[k]:pos[k] + s["hop"]]
        if k in errors:
            continue
        try:
            while not srv.push(sids[k], seg, t0 + t):
                refused += 1
                time.sleep(0.0002)
        except S.SrpError as e:
            errors.setdefault(k, str(e))
        pos[k] += s["hop"]
    # let the last frames finish
    deadline = time.perf_counter() + 30
    while done["frames"] < len(events) and time.perf_counter() < deadline and not errors:
        time.sleep(0.01)
    wall = time.perf_counter() - w0
    stop.set()
    th.join()
    st = srv.stats()
    srv.close()
    res = {"sessions": sessions, "seconds": seconds, "rate_frames_per_s_per_session": rate,
           "precision": precision, "max_batch": max_batch, "frames": st["frames_done"],
           "frames_expected": len(events), "cells_frames_per_s": done["cells"] / wall,
           "frames_per_s": st["frames_done"] / wall,
           "latency_p50_ms": 1e3 * st["latency_p50_s"], "latency_p99_ms": 1e3 * st["latency_p99_s"],
           "latency_max_ms": 1e3 * st["latency_max_s"], "launches": st["launches"],
           "graph_launches": st["graph_launches"],
           "mean_frames_per_launch": st["frames_launched"] / max(1, st["launches"]),
           "group_launches": st["group_launches"], "group_frames": st["group_frames"],
           "mean_sessions_per_group_launch": st["group_sessions"] / max(1, st["group_launches"]),
           "mean_frames_per_group_launch": st["group_frames"] / max(1, st["group_launches"]),
           "precision_by_M": {str(M): session_precision({"M": M}, precision) for M in Ms},
           "admission_build_s": build_s, "push_retries": refused,
           "failed_sessions": {str(k): v for k, v in errors.items()},
           "slowest_sessions": slowest_sessions(mix, lats),
           "mix": {"M": [s["M"] for s in mix], "J": Js, "N": [s["N"] for s in mix],
                   "method": [s["kw"]["method"] for s in mix]}}
    return res


def run_curve(a):
    """Map error vs throughput over the methods' complexity parameters (the paper's
    trade-off, Sec. V): every point times srp_map on the workload's F frames (L2 flushed,
    CUDA events) and compares sampled frames with the FP64 conv. FD-SRP oracle: eps_z in dB
    (Sec. V-A) and the distance of the argmax location to the true source."""
    import torch
    import oracle as O
    import paper_2306_08514_gb300 as S
    import synth
    torch.cuda.set_device(0)
    w = synth.workload(a.workload, F=a.frames)
    F, J, N, M = w["F"], w["grid_xyz"].shape[0], w["N"], w["mic_xyz"].shape[0]
    P, K = M * (M - 1) // 2, N // 2
    frames = torch.from_numpy(w["frames"]).cuda()
    sel = np.linspace(0, F - 1, 32).astype(int)
    dt = O.tdoa_nf(w["mic_xyz"], w["grid_xyz"])
    zc = O.srp_conv(O.gcc_phat(O.stft(w["frames"][sel], "hann")), dt, w["fs"])
    src = np.asarray(w["sources"][0], float)
    Nm = O.mean_samples(O.n_p_samples(w["mic_xyz"], w["fs"]))
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    points = [("conv", {}, "fp32"), ("conv", {}, "fp16x3"), ("conv", {}, "bf16")]
    points += [("slri", {"rank": r}, "bf16") for r in (2, 4, 8, 16, 32, 64)]
    points += [("sspi", {"taps": t}, "bf16") for t in (0.5, 1.0, 2.0, 4.0, 8.0)]
    points += [("lr", {"rank": r}, "bf16") for r in (4, 16, 32)]
    points += [("si", {}, "bf16"), ("td", {}, "bf16")]
    out = []
    for method, kw, prec in points:
        plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], N, method=method, precision=prec,
                      max_frames=F, **kw)
        plan.autotune(F)
        maps = torch.empty((F, J), dtype=torch.float32, device="cuda")
        am = torch.empty((F,), dtype=torch.int32, device="cuda")
        for _ in range(2):
            plan.map(frames, maps, am)
        times = []
        for _ in range(5):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.map(frames, maps, am)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        plan.status()
        z = maps[torch.from_numpy(sel).cuda()].double().cpu().numpy()
        idx = am.cpu().numpy()[sel]
        eps = O.eps_db(z, zc, axis=-1)
        loc = np.linalg.norm(w["grid_xyz"][idx] - src[None, :], axis=1)
        loc_c = np.linalg.norm(w["grid_xyz"][np.argmax(zc, axis=1)] - src[None, :], axis=1)
        cx = O.complexity(J, P, K, N_mean=Nm, R=kw.get("rank"), R_H=kw.get("rank"),
                          Q_Lambda=round(kw.get("taps", 0) * J * P) or None)
        key = {"conv": "C", "slri": "C_slri", "sspi": "C_sspi", "lr": "C_lr", "si": "C_si",
               "td": "C_td"}[method]
        ms = float(np.median(times))
        out.append({"method": method, **kw, "precision": prec, "ms": ms,
                    "cells_frames_per_s": J * F / (ms / 1e3),
                    "eps_z_db_median": float(np.median(eps)), "eps_z_db_max": float(np.max(eps)),
                    "loc_err_m_median": float(np.median(loc)),
                    "argmax_agree_conv_oracle": float(np.mean(idx == np.argmax(zc, axis=1))),
                    "C_rel": float(cx[key] / cx["C"])})
        plan.close()
        del maps
        print(json.dumps(out[-1]), file=sys.stderr, flush=True)
    res = {"metric": "SRP map error vs throughput (eps_z vs the FP64 conv. FD-SRP oracle)",
           "unit": UNIT, "workload": a.workload, "F": F, "J": J,
           "conv_oracle_loc_err_m_median": float(np.median(loc_c)), "points": out}
    print(json.dumps(res), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.curve:
        run_curve(a)
    elif a.serving:
        res = run_serving(a, sessions=a.sessions, seconds=a.seconds,
                          precision=a.serving_precision, rate=a.rate)
        out = {"metric": "serving: map cells*frames/s and frame-to-map latency", "value": res["cells_frames_per_s"],
               "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": a.serving_precision,
               "data": "synthetic", "config": {"workload": f"serving: {a.sessions} sessions, Poisson "
                                               f"{a.rate} frames/s each, {a.seconds} s"},
               "serving": res}
        print(json.dumps(out), flush=True)
    else:
        run_libsrp(a)


if __name__ == "__main__":
    main()
