"""Localisation agreement (Eq. imax) of the GPU estimates with the FP64 oracle's, per method
and precision (GPU).

On square4 (M = 4, J = 2500, all 100 frames) and a walls16 subset (M = 16, N = 1024, two
sources, every 37th grid cell, 128 frames) the argmax each plan returns is compared with
the maxima of the oracle's map of the same method.  Both grids hold exact ties (the
square array sits on a symmetry centre of its grid), so agreement is counted against the
set of the oracle's maxima, cells within 1e-9 of its peak height (ties in exact arithmetic
that FP64 rounding resolves either way).  FP32-class precisions (maps within 1e-5 of the
oracle) must agree on every frame; BF16 and FP16, whose maps carry 1e-4..1e-2 of rounding
error, must pick a cell whose oracle value is within the stated fraction of the peak's
height above the map median.  Every figure is written to the test log.
"""
import json

import numpy as np
import pytest

import bench
import oracle as O
from tests import _ref as R
from tests.test_gpu_parity import S, _run, _check_taps  # noqa: F401

pytestmark = pytest.mark.gpu

FP32_CLASS = ("fp32", "fp16x3", "tf32x3", "bf16x3")
# BF16 / FP16 / TF32 operands: the pick may lose at most this fraction of the peak height
GAP_BOUND = {"fp16": 5e-3, "tf32": 5e-3, "bf16": 2e-2}


def _refs(name, F, sub, rank, taps):
    w = R.workload(name, F, sub)
    dt, Np, lags, perm = R.geometry(name, F, sub)
    psi = R.psi_of(w["frames"])
    xi, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    Lam = R.lam(name, F, sub)
    tall, fat, _ = R.slri(name, rank, F, sub)
    mask, _, _, _ = R.sspi(name, taps, F, sub)
    return w, dt, lags, perm, psi, xi, Lam, (tall, fat), mask


@pytest.mark.parametrize("name,F,sub,rank,taps", [("square4", None, 1, 8, 2.0),
                                                  ("walls16", 128, 37, 16, 4.0)])
def test_argmax_agreement_per_method_and_precision(S, name, F, sub, rank, taps):
    w, dt, lags, perm, psi, xi, Lam, (tall, fat), mask = _refs(name, F, sub, rank, taps)
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    zo = {"conv": O.srp_conv(psi, dt, w["fs"]), "slri": O.srp_slri(tall, fat, xi)}
    kws = {"conv": {}, "slri": dict(rank=rank), "sspi": dict(taps=taps)}
    report = {}
    for method in ("conv", "slri", "sspi"):
        for prec in FP32_CLASS + tuple(GAP_BOUND):
            if method != "conv" and prec in ("tf32", "bf16x3"):
                continue
            plan = S.Plan(*args, method=method, precision=prec, max_frames=128, **kws[method])
            if method == "sspi":  # Lambda masked by the plan's own (validated) selection
                ref = O.srp_sspi(np.where(_check_taps(plan, mask, perm, Lam), Lam, 0.0), xi)
            else:
                ref = zo[method]
            z, am = _run(plan, w["frames"])
            plan.status()
            plan.close()
            assert np.array_equal(am, np.argmax(z, axis=1)), (method, prec)
            rep = bench.argmax_report(am, ref, w["grid_xyz"])
            rep["rel_err_max"] = float(R.per_frame_rel(z, ref).max())
            report[f"{method}/{prec}"] = rep
    print(f"\nargmax agreement, {name}: " + json.dumps(report, indent=1))
    for key, rep in report.items():
        method, prec = key.split("/")
        if prec in FP32_CLASS:
            assert rep["agree_up_to_ties"] == 1.0, (key, rep)
        else:
            assert rep["peak_gap_max"] <= GAP_BOUND[prec], (key, rep)
