#!/usr/bin/env python
"""Benchmark of the SRP-map hot path on one GB300 (or N replicas under torchrun).

Workload (default): M=8 uniform circular array (r=5 cm), 3-D grid of 0.1 m cells over
5x4x3 m (J=60000), N=512 Hann frames, F=2000 frames per step, AR(10) speech-like source
with on/off envelope and 10 dB diffuse noise (synthetic, seeded).  One step computes,
for the whole batch, the maps of all three methods -- conv. FD-SRP, SLRI-SRP (R=16) and
SSPI-SRP (t=4 taps per location and pair) -- each through the full path (STFT + PHAT,
cross-spectra / iFFT sampling, contraction, argmax).  ``value`` counts every map cell
produced: 3 * J * F per step and rank.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle instead.
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libsrp", choices=["libsrp", "reference"])
    ap.add_argument("--workload", default="uca8")
    ap.add_argument("--frames", type=int, default=None)
    ap.add_argument("--rank", type=int, default=16, help="SLRI rank R")
    ap.add_argument("--taps", type=float, default=4.0, help="SSPI taps per location and pair")
    ap.add_argument("--conv-precision", default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--methods", default="conv,slri,sspi")
    return ap.parse_args()


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

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
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
def cpu_baseline(w, R, t, n_frames=1):
    """The FP64 oracle as it stands, per-frame work of all three methods on a bounded
    sample (n_frames frames, every grid cell); plan-time fits are excluded like the GPU's."""
    import oracle as O
    fs, K = w["fs"], w["N"] // 2
    dt = O.tdoa_nf(w["mic_xyz"], w["grid_xyz"])
    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], fs))
    Lam = O.interp_matrix(dt, fs, lags)
    tall, fat, _ = O.slri_factors(Lam, R)
    Lsp = O.sspi_matrix(Lam, lags, int(round(t * Lam.shape[0] * len(lags))))
    fr = w["frames"][:n_frames]
    t0 = time.perf_counter()
    psi = O.gcc_phat(O.stft(fr, "hann"))
    O.srp_conv(psi, dt, fs)
    xi, _ = O.gcc_samples_ifft(psi, lags, K)
    O.srp_slri(tall, fat, xi)
    O.srp_sspi(Lsp, xi)
    el = time.perf_counter() - t0
    J = w["grid_xyz"].shape[0]
    try:
        import threadpoolctl
        cores = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or 1
    except Exception:
        cores = os.cpu_count()
    return {"value": 3 * J * n_frames / el, "unit": UNIT, "cores": int(cores), "kind": "oracle",
            "sample": f"{n_frames} frame(s) x {J} cells x 3 methods (conv FP64 H, SLRI R={R}, "
                      f"SSPI t={t}); plan-time SVD/selection excluded", "seconds": el}


def run_reference(a):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import synth
    w = synth.workload(a.workload, F=max(4, a.warmup + a.steps))
    J = w["grid_xyz"].shape[0]
    times = []
    for s in range(a.warmup + a.steps):
        sub = dict(w)
        sub["frames"] = w["frames"][s:s + 1]
        r = cpu_baseline(sub, a.rank, a.taps, 1)
        if s >= a.warmup:
            times.append(r["seconds"])
    ms = 1e3 * float(np.mean(times))
    value = 3 * J / (ms / 1e3)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{a.workload}: 1 frame per step, all 3 methods, FP64 oracle on host"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                            "sample": r["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------------------------
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
    F, J, N, M = w["F"], w["grid_xyz"].shape[0], w["N"], w["mic_xyz"].shape[0]
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], N)
    methods = [m for m in a.methods.split(",") if m]
    kw = {"conv": dict(method="conv", precision=a.conv_precision),
          "slri": dict(method="slri", rank=a.rank), "sspi": dict(method="sspi", taps=a.taps)}
    plans = {m: S.Plan(*args, max_frames=F, **kw[m]) for m in methods}
    frames = torch.from_numpy(w["frames"]).to(dev)
    maps = {m: torch.empty((F, J), dtype=torch.float32, device=dev) for m in methods}
    am = {m: torch.empty((F,), dtype=torch.int32, device=dev) for m in methods}
    stream = torch.cuda.current_stream()

    def step():
        for m in methods:
            plans[m].map(frames, maps[m], am[m], stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    for m in methods:
        plans[m].set_profiling(True)
    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop() if rank == 0 else None
    dev_ms = e0.elapsed_time(e1) / a.steps
    stages = {m: plans[m].stage_ms() for m in methods}
    for m in methods:
        plans[m].set_profiling(False)
    dev_ms, wall = reduce_max([dev_ms, wall], world, dev)

    # per-method device time for the breakdown (sum of its stages per step)
    per = {}
    for m in methods:
        st = stages[m]
        ms_m = sum(st[k] for k in ("frontend", "spectra", "contract", "argmax")) / a.steps
        per[m] = {"ms_per_step": ms_m, "cells_frames_per_s": J * F / (ms_m / 1e3),
                  "stage_ms": {k: st[k] / a.steps for k in ("frontend", "spectra", "contract", "argmax")}}
    # map error of SLRI/SSPI relative to the GPU's conv FP32 map (eps_z of Sec. V-A)
    if "conv" in methods:
        zc = maps["conv"].double()
        for m in methods:
            if m == "conv":
                continue
            d = ((maps[m].double() - zc) ** 2).sum(1) / (zc ** 2).sum(1)
            per[m]["eps_z_vs_conv_db_median"] = float(10 * torch.log10(d).median())
            per[m]["argmax_agree_vs_conv"] = float((am[m] == am["conv"]).float().mean())

    # e2e through the host-buffer entry point (H2D frames + D2H maps inside the timing)
    hframes = torch.from_numpy(w["frames"]).pin_memory()
    hmaps = {m: torch.empty((F, J), dtype=torch.float32).pin_memory() for m in methods}
    ham = {m: torch.empty((F,), dtype=torch.int32).pin_memory() for m in methods}
    for m in methods:  # warm the staging buffers
        plans[m].map_host(hframes, hmaps[m], ham[m])
    e2e_steps = max(1, min(a.steps, 3))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        for m in methods:
            plans[m].map_host(hframes, hmaps[m], ham[m])
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    e2e_s = reduce_max([e2e_s], world, dev)[0]

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cells = len(methods) * J * F * world
    value = cells / (dev_ms / 1e3)
    hbm, bf16, bf16s, smmax, src = peaks()
    # dominant kernel: the contraction with the largest time
    dom = max(methods, key=lambda m: per[m]["stage_ms"]["contract"])
    K = N // 2
    P = M * (M - 1) // 2
    t_launch = per[dom]["stage_ms"]["contract"] / 1e3
    info = plans[dom].info
    if dom == "conv":
        flops = 4.0 * J * P * (K - 1) * F  # 2 J P (K-1) real MACs per frame (Eq. SRPomp)
        if a.conv_precision == "fp32":
            peak = 152 * 128 * 2 * smmax * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": flops / t_launch / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 x max SM clock"}
        else:
            roof = {"bound": "tensor", "achieved": flops / t_launch / 1e12, "peak": bf16s,
                    "unit": "TFLOP/s", "peak_source": f"{src} bf16 sustained"}
    elif dom == "slri":
        R = a.rank
        byts = 4.0 * J * F + 4.0 * F * R + 4.0 * J * R  # map write + u read + factors
        roof = {"bound": "hbm", "achieved": byts / t_launch / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": f"{src} copy"}
    else:
        nnz = info.nnz
        flops = 2.0 * nnz * F
        peak = 152 * 128 * 2 * smmax * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / t_launch / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": "152 SMs x 128 FP32 FMA/clk x 2 x max SM clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["kernel"] = {"conv": "conv GEMM", "slri": "SLRI fat+tall", "sspi": "SSPI gather"}[dom]
    per_launch = {"conv": 4, "slri": 5, "sspi": 4}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": dev_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{a.workload}: M={M} UCA r=5cm, J={J} (0.1 m grid), N={N} Hann, "
                               f"F={F} frames/step/rank; conv FD-SRP {a.conv_precision} + SLRI R={a.rank} "
                               f"+ SSPI t={a.taps}",
                   "maps_per_frame": len(methods), "l2": "working set per step > L2 (SRP matrix "
                   f"{plans['conv'].info.device_bytes / 1e9:.1f} GB, maps {len(methods) * 4 * J * F / 1e9:.2f} GB); no flush"
                   if "conv" in plans else "maps written per step exceed L2"},
        "wall_ms_per_step": 1e3 * wall / a.steps,
        "methods": per,
        "roofline": roof,
        "e2e": {"value": cells / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": len(methods) * F * M * N * 4,
                "d2h_bytes_per_step": len(methods) * F * (J * 4 + 4)},
        "gpu_launches": sum(per_launch[m] for m in methods) * a.steps,
        "clocks": ck,
    }
    if "conv" in per and "slri" in per:
        out["speedup_slri_vs_conv"] = per["slri"]["cells_frames_per_s"] / per["conv"]["cells_frames_per_s"]
    if "conv" in per and "sspi" in per:
        out["speedup_sspi_vs_conv"] = per["sspi"]["cells_frames_per_s"] / per["conv"]["cells_frames_per_s"]
    if world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = {k: v for k, v in cpu_baseline(w, a.rank, a.taps, 1).items() if k != "seconds"}
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_libsrp(a)


if __name__ == "__main__":
    main()
