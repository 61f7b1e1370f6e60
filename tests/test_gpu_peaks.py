"""Several source estimates per frame (srp_map_peaks) against the oracle (GPU).

The oracle's srp_peaks is Eq. (imax) taken K times with exclusion balls of radius d_min,
its distance test in the FP32 the kernel uses.  Given the same map, the picks are integer
decisions taken in the same precision, so the GPU's peaks must equal the oracle's applied
to the GPU's own map exactly, and the values must be the map's values at the picks.
Estimates-only calls (maps = NULL: L2-sized map scratch) must give the same picks as calls
that write the maps (but on near ties: their smaller chunks may split long reductions
differently, which moves map values by FP32 rounding).  Against the FP64 oracle's own maps (walls16 subset, FP32-class
precision) the first pick must be one of the oracle's maxima and the picks must agree
wherever the oracle's greedy choice is not decided within the GPU's map error.
Sizes: square4 (J = 2500, F = 100) and the full walls16 workload (M = 16, J = 72000,
N = 1024, F = 4096, two sources), in the bench's launch configuration.
"""
import numpy as np
import pytest

import oracle as O
from tests import _ref as R
from tests.test_gpu_parity import S, _cuda  # noqa: F401

pytestmark = pytest.mark.gpu


def _check_against_own_map(plan, frames, K, d_min, grid):
    import torch
    pk, val, maps = plan.peaks(frames, K, d_min)
    pk2, val2, none = plan.peaks(frames, K, d_min, want_maps=False)
    torch.cuda.synchronize()
    plan.status()
    assert none is None
    z = maps.cpu().numpy()
    p = pk.cpu().numpy()
    v = val.cpu().numpy()
    io, vo = O.srp_peaks(z, grid, K, d_min)
    assert np.array_equal(p, io), np.argwhere(p != io)[:5]
    assert np.array_equal(np.isnan(v), np.isnan(vo)) and np.array_equal(v[~np.isnan(v)], vo[~np.isnan(vo)])
    # estimates only: the maps go through smaller L2-sized chunks, whose long reductions
    # may be split into (FP64-summed) slices differently, so map values can differ in the
    # last bits; the picks must agree but on near ties, the values to FP32 rounding
    p2, v2 = pk2.cpu().numpy(), val2.cpu().numpy()
    same = np.all(p2 == p, axis=1)
    assert same.mean() >= 0.999, same.mean()
    ok = ~np.isnan(v) & same[:, None]
    assert np.allclose(v2[ok], v[ok], rtol=1e-5, atol=0)
    _, am = plan.map(frames)
    torch.cuda.synchronize()
    assert np.array_equal(am.cpu().numpy(), p[:, 0])  # pick 0 is srp_map's argmax
    return p, z


@pytest.mark.parametrize("method,kw,prec", [("conv", {}, "fp32"), ("slri", dict(rank=8), "bf16"),
                                            ("sspi", dict(taps=2.0), "fp16x3")])
@pytest.mark.parametrize("K,d_min", [(1, 0.0), (4, 0.5), (3, 0.0), (16, 1.3), (5, 9.0)])
def test_peaks_square4_equal_the_oracle_rule_on_the_gpu_map(S, method, kw, prec, K, d_min):
    w = R.workload("square4")
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method=method, precision=prec,
                  max_frames=64, **kw)  # F = 100: two chunks
    p, _ = _check_against_own_map(plan, _cuda(w["frames"]), K, d_min, w["grid_xyz"])
    if d_min >= 9.0:  # beyond the grid's diameter: one pick per frame
        assert np.all(p[:, 1:] == -1)


def test_peaks_walls16_full_size(S):
    """The full walls16 workload (two sources), SLRI R = 16 in FP16 hi+lo and conv in BF16:
    K = 4 picks 1 m apart for all 4096 frames, exactly the oracle's rule on the GPU's maps;
    the estimates-only path (maps in L2-sized chunks) gives the same picks."""
    w = R.workload("walls16")
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    frames = _cuda(w["frames"])
    for kw in (dict(method="slri", rank=16, precision="fp16x3"), dict(method="conv", precision="bf16")):
        plan = S.Plan(*args, max_frames=w["F"], **kw)
        p, _ = _check_against_own_map(plan, frames, 4, 1.0, w["grid_xyz"])
        assert np.all(p[:, 1] >= 0)
        d = np.linalg.norm(w["grid_xyz"][p[:, 0]] - w["grid_xyz"][p[:, 1]], axis=1)
        assert np.all(d >= 1.0 - 1e-6)
        plan.close()


def test_peaks_walls16_subset_against_fp64_oracle_maps(S):
    """Every 37th cell of walls16, 128 frames: the GPU (conv and SLRI in FP16 hi+lo) against
    the oracle's picks on the oracle's FP64 maps.  Pick 0 must be a maximum of the oracle's
    map (ties in exact arithmetic excepted).  Later picks must equal the oracle's in every
    frame where each greedy choice of the oracle wins by more than 2x the GPU's map error
    and no cell lies within 1e-5 m of an exclusion boundary."""
    name, F, sub = "walls16", 128, 37
    w = R.workload(name, F, sub)
    dt, Np, lags, perm = R.geometry(name, F, sub)
    psi = R.psi_of(w["frames"])
    xi, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    tall, fat, _ = R.slri(name, 16, F, sub)
    refs = {"conv": O.srp_conv(psi, dt, w["fs"]), "slri": O.srp_slri(tall, fat, xi)}
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    g = w["grid_xyz"]
    K, d_min = 3, 1.0
    for method, kw in (("conv", {}), ("slri", dict(rank=16))):
        plan = S.Plan(*args, method=method, precision="fp16x3", max_frames=F, **kw)
        import torch
        pk, val, maps = plan.peaks(_cuda(w["frames"]), K, d_min)
        torch.cuda.synchronize()
        p, z = pk.cpu().numpy(), maps.cpu().numpy().astype(np.float64)
        zo = refs[method]
        err = np.abs(z - zo).max(axis=1)
        io, vo = O.srp_peaks(zo, g, K, d_min)
        decided = 0
        for f in range(F):
            top = zo[f, io[f, 0]]
            assert zo[f, p[f, 0]] >= top - 2 * err[f] - 1e-9, (method, f)
            # is every greedy step of the oracle decided by more than the GPU's error?
            clear, allowed = True, np.ones(len(g), bool)
            for k in range(K):
                if io[f, k] < 0:
                    break
                cand = np.sort(np.where(allowed, zo[f], -np.inf))[-2:]
                clear &= cand[1] - cand[0] > 4 * err[f]
                dist = np.linalg.norm(g - g[io[f, k]], axis=1)
                clear &= not np.any(np.abs(dist - d_min) < 1e-5)
                allowed &= dist >= d_min
                allowed[io[f, k]] = False
            if clear:
                decided += 1
                assert np.array_equal(p[f], io[f]), (method, f, p[f], io[f])
        assert decided >= F // 2, (method, decided)
        plan.close()
