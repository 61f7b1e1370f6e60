"""Parity of the tensor-core precisions of every method, and of SI-SRP and conv. TD-SRP,
against the FP64 oracle (through the C-ABI, on the GPU).

Bounds: FP16 hi+lo and FP32 must meet 1e-5 relative per frame; single FP16 / BF16
operands round each operand to 2^-11 / 2^-8 relative, which over sums of many terms gives
about sqrt(2/3) u of map error: stated bounds 2e-3 (FP16) and 1.5e-2 (BF16).  The argmax
returned must be the argmax of the GPU's own map, and a valid maximum of the oracle map
within the measured error.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests import _ref as R
from tests.test_gpu_parity import S, _run, check_argmax, _check_taps, sq, uca_small  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = 1e-5
PRECS = [("fp32", TOL), ("fp16x3", TOL), ("tf32x3", TOL), ("bf16x3", 1e-4), ("fp16", 2e-3),
         ("tf32", 2e-3), ("bf16", 1.5e-2)]
TC_PRECS = PRECS[1:]


@pytest.mark.parametrize("prec,tol", PRECS)
def test_si_square4(S, sq, prec, tol):
    w, psi, dt, lags, perm, xi_o = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="si", precision=prec,
                  max_frames=64)
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = O.srp_si(R.lam("square4"), xi_o)
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_td_square4(S, sq, prec, tol):
    w, psi, dt, lags, perm, xi_o = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="td", precision=prec,
                  max_frames=64)
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = xi_o @ O.td_matrix(dt, w["fs"], lags).T
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)


@pytest.mark.parametrize("prec,tol", TC_PRECS)
@pytest.mark.parametrize("rank", [8, 16])
def test_slri_tensor_cores_square4(S, sq, prec, tol, rank):
    w, psi, dt, lags, perm, xi_o = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="slri", rank=rank,
                  precision=prec, max_frames=64)
    z, am = _run(plan, w["frames"])
    plan.status()
    tall, fat, s = R.slri("square4", rank)
    zo = O.srp_slri(tall, fat, xi_o)
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)


@pytest.mark.parametrize("prec,tol", TC_PRECS)
@pytest.mark.parametrize("t", [0.5, 2.0, 4.0])
def test_sspi_tensor_cores_square4(S, sq, prec, tol, t):
    w, psi, dt, lags, perm, xi_o = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="sspi", taps=t,
                  precision=prec, max_frames=64)
    mask, tied, taken, nnz = R.sspi("square4", t)
    mask_g = _check_taps(plan, mask, perm, R.lam("square4"))
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = O.srp_sspi(np.where(mask_g, R.lam("square4"), 0.0), xi_o)
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)


def test_uca8_small_tensor_cores_all_methods(S, uca_small):
    """Ragged frame tile (70 = 64 + 6) and cell tile (4616 cells), block-sparse SSPI/TD."""
    name, F, sub, w, psi, dt, lags, perm, xi_o = uca_small
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    Lam = R.lam(name, F, sub)
    tall, fat, s = R.slri(name, 16, F, sub)
    mask, tied, taken, nnz = R.sspi(name, 4.0, F, sub)
    refs = {
        "si": (dict(method="si"), O.srp_si(Lam, xi_o)),
        "td": (dict(method="td"), xi_o @ O.td_matrix(dt, w["fs"], lags).T),
        "slri": (dict(method="slri", rank=16), O.srp_slri(tall, fat, xi_o)),
        "sspi": (dict(method="sspi", taps=4.0), None),
    }
    for prec, tol in PRECS:
        for m, (kw, zo) in refs.items():
            if m in ("slri", "sspi") and prec == "fp32":
                continue  # covered by test_gpu_parity
            plan = S.Plan(*args, precision=prec, max_frames=64, **kw)
            if m == "sspi":  # Lambda masked by the plan's own (valid) selection
                zo = O.srp_sspi(np.where(_check_taps(plan, mask, perm, Lam), Lam, 0.0), xi_o)
            z, am = _run(plan, w["frames"])
            plan.status()
            assert R.per_frame_rel(z, zo).max() <= tol, (m, prec)
            check_argmax(z, am, zo)


def test_uca8_full_size_tensor_cores_sampled(S):
    """The benchmark's workload (J=60000, F=2000, one launch per method), tensor-core
    SLRI / SSPI in FP16 hi+lo: sampled frames against the oracle."""
    w = R.workload("uca8")
    F = w["F"]
    frames = w["frames"]
    fsel = np.array([0, 3, 999, 1998, F - 1])
    psi = R.psi_of(frames[fsel])
    dt, Np, lags, perm = R.geometry("uca8")
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    tall, fat, s = R.slri("uca8", 16)
    plan = S.Plan(*args, method="slri", rank=16, precision="fp16x3", max_frames=F)
    z, am = _run(plan, frames)
    plan.status()
    zo = O.srp_slri(tall, fat, xi_o)
    assert R.per_frame_rel(z[fsel], zo).max() <= TOL
    check_argmax(z[fsel], am[fsel], zo)
    mask, tied, taken, nnz = R.sspi("uca8", 4.0)
    plan = S.Plan(*args, method="sspi", taps=4.0, precision="fp16x3", max_frames=F)
    mask_g = _check_taps(plan, mask, perm, R.lam("uca8"))
    z, am = _run(plan, frames)
    plan.status()
    zo = O.srp_sspi(np.where(mask_g, R.lam("uca8"), 0.0), xi_o)
    assert R.per_frame_rel(z[fsel], zo).max() <= TOL
    check_argmax(z[fsel], am[fsel], zo)
    # each kernel alone and in clusters of 2 (and 2 x 2: SLRI's dense reduction; SSPI's
    # block-sparse one runs them as 2 x 1) CTAs that share operand tiles by multicast (16
    # frame tiles per cell tile): the same maps bit for bit
    for base in (0, 1, 3):
        plan.set_variant(base)
        zb, amb = _run(plan, frames)
        for v in (base + 4, base + 8):
            plan.set_variant(v)
            zc, amc = _run(plan, frames)
            plan.status()
            assert np.array_equal(zc, zb) and np.array_equal(amc, amb), v


@pytest.mark.parametrize("prec,base", [("fp16x3", 3), ("bf16", 0), ("tf32x3", 0)])
def test_clusters_with_split_reduction_and_a_tile_past_F(S, prec, base):
    """Conv on 330 frames (three frame tiles, the last ragged: the second cluster of a cell
    tile runs a frame tile past F) and 4616 cells (19 cell tiles, the last ragged: a 2 x 2
    cluster also runs a cell tile past J; 57 output tiles, so the reduction is split into
    slices summed in FP64): the cluster variants' maps equal the unclustered kernel's bit
    for bit, and match the oracle on sampled frames."""
    w = R.workload("uca8", 330, 13)
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    plan = S.Plan(*args, method="conv", precision=prec, max_frames=330)
    plan.set_variant(base)
    zb, ab = _run(plan, w["frames"])
    for v in (base + 4, base + 8):
        plan.set_variant(v)
        zc, ac = _run(plan, w["frames"])
        plan.status()
        assert np.array_equal(zc, zb) and np.array_equal(ac, ab), v
    fsel = np.array([0, 129, 257, 329])
    dt, *_ = R.geometry("uca8", 330, 13)
    zo = O.srp_conv(R.psi_of(w["frames"][fsel]), dt, w["fs"])
    assert R.per_frame_rel(zc[fsel], zo).max() <= dict(PRECS)[prec]
    check_argmax(zc[fsel], ac[fsel], zo)


@pytest.mark.parametrize("name,F,sub,rank,prec", [
    ("nested32", 6, 400, 8, "fp32"), ("nested32", 6, 400, 32, "fp16x3"),
    ("nested32", 6, 400, 16, "bf16"), ("nested32", 6, 400, 16, "fp16"), ("nested32", 6, 400, 16, "tf32"),
    ("walls16", 4, 300, 8, "fp32"), ("walls16", 4, 300, 16, "bf16"), ("walls16", 4, 300, 16, "fp16"),
    ("walls16", 4, 300, 16, "tf32"),
])
def test_slri_long_sample_vectors(S, name, F, sub, rank, prec):
    """L = 7408 (nested32) and 43326 (walls16): the low-rank fit runs as a device subspace
    iteration; its singular values and maps match the oracle's SVD.  The nested32 frames
    (N = 2048) are sampled from spectra in global memory: with the three products of the
    hi + lo split for FP32 and FP16 hi+lo, with one FP16 product for BF16, FP16 and TF32; the
    walls16 frames (N = 1024, lag windows up to 355) by iFFT: radix-8 in FP32, as 32 x 32
    DFTs on the warp-level tensor cores for BF16, FP16 and TF32."""
    w = R.workload(name, F, sub)
    dt, Np, lags, perm = R.geometry(name, F, sub)
    xi_o, _ = O.gcc_samples_ifft(R.psi_of(w["frames"]), lags, w["N"] // 2)
    tall, fat, s = R.slri(name, rank, F, sub)
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="slri", rank=rank,
                  precision=prec, max_frames=4)
    sig = plan.slri_sigma(rank + 1)
    assert np.allclose(sig, s[:rank + 1], rtol=1e-8, atol=1e-8 * s[0])
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = O.srp_slri(tall, fat, xi_o)
    tol = dict(PRECS)[prec]
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)


@pytest.mark.parametrize("method,kw", [("conv", {}), ("slri", dict(rank=16)), ("sspi", dict(taps=4.0)),
                                       ("td", {})])
def test_every_tensor_core_variant_and_the_autotuner(S, uca_small, method, kw):
    """The four tcgen05 variants (128x256 4-stage, 128x256 2-stage 4-box, 128x128, and for
    the hi + lo precisions 128x256 with the hi and lo planes of one k-block per stage), each
    also in clusters of 2 CTAs sharing the B tiles by multicast, give the oracle's maps on
    ragged tiles (70 frames: one frame tile, which the cluster variants run unclustered) and
    equal maps bit for bit; srp_plan_autotune times them and keeps one; a BF16 plan refuses
    the hi + lo variants."""
    name, F, sub, w, psi, dt, lags, perm, xi_o = uca_small
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    Lam = R.lam(name, F, sub)
    if method == "conv":
        zo = O.srp_conv(psi, dt, w["fs"])
    elif method == "slri":
        tall, fat, s = R.slri(name, 16, F, sub)
        zo = O.srp_slri(tall, fat, xi_o)
    elif method == "sspi":
        mask, tied, taken, nnz = R.sspi(name, 4.0, F, sub)
        zo = O.srp_sspi(np.where(mask, Lam, 0.0), xi_o)
    else:
        zo = xi_o @ O.td_matrix(dt, w["fs"], lags).T
    plan = S.Plan(*args, method=method, precision="fp16x3", max_frames=64, **kw)
    if method == "sspi":  # Lambda masked by the plan's own (valid) selection
        zo = O.srp_sspi(np.where(_check_taps(plan, mask, perm, Lam), Lam, 0.0), xi_o)
    base = {}
    for v in list(range(12)) + [-1]:
        plan.set_variant(v)
        z, am = _run(plan, w["frames"])
        plan.status()
        assert R.per_frame_rel(z, zo).max() <= TOL, v
        check_argmax(z, am, zo)
        if 0 <= v < 4:
            base[v] = (z, am)
        elif v >= 4:  # the same kernel with shared operand tiles: the same maps bit for bit
            assert np.array_equal(z, base[v % 4][0]) and np.array_equal(am, base[v % 4][1]), v
    rep = plan.autotune(F=64)
    assert rep["variant"] in rep["ms"] and len(rep["ms"]) == 12
    z, am = _run(plan, w["frames"])
    assert R.per_frame_rel(z, zo).max() <= TOL
    single = S.Plan(*args, method=method, precision="bf16", max_frames=64, **kw)
    for v in (3, 7, 11):
        with pytest.raises(S.SrpError):
            single.set_variant(v)
    assert len(single.autotune(F=64)["ms"]) == 9


@pytest.mark.parametrize("method,kw,prec,tol", [
    ("conv", {}, "fp32", TOL), ("conv", {}, "fp16x3", TOL), ("slri", dict(rank=20), "fp16x3", TOL),
    ("sspi", dict(taps=2.0), "fp32", TOL), ("si", {}, "bf16", 1.5e-2), ("td", {}, "fp16x3", TOL),
])
def test_far_field_grid(S, method, kw, prec, tol):
    """Far field (Eq. Deltat_i second case) on the paper's 2-degree half-sphere grid
    (J = 8101) with the uca8 array."""
    w = R.workload("uca8", 24, 13)
    dirs = synth.grid_ff_halfsphere(2.0)
    dt = O.tdoa_ff(w["mic_xyz"], dirs)
    Np = O.n_p_samples(w["mic_xyz"], w["fs"])
    lags = O.pair_lags(Np)
    psi = R.psi_of(w["frames"])
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    Lam = O.interp_matrix(dt, w["fs"], lags)
    plan = S.Plan(w["mic_xyz"], dirs, w["fs"], w["N"], method=method, precision=prec,
                  max_frames=16, far_field=True, **kw)
    perm = O.lags_to_ascending(lags)
    if method == "conv":
        zo = O.srp_conv(psi, dt, w["fs"])
    elif method == "slri":
        tall, fat, s = O.slri_factors(Lam, 20)  # sigma_16 = sigma_17 here (symmetric array): R = 20 has a gap
        zo = O.srp_slri(tall, fat, xi_o)
    elif method == "sspi":
        nnz = int(round(2.0 * Lam.shape[0] * len(lags)))
        mask, tied, taken = O.sspi_select(Lam, lags, nnz)
        zo = O.srp_sspi(np.where(_check_taps(plan, mask, perm, Lam), Lam, 0.0), xi_o)
    elif method == "si":
        zo = O.srp_si(Lam, xi_o)
    else:
        zo = xi_o @ O.td_matrix(dt, w["fs"], lags).T
    z, am = _run(plan, w["frames"])
    plan.status()
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)


@pytest.mark.parametrize("method,kw,prec", [("conv", {}, "bf16"), ("slri", dict(rank=16), "fp16x3"),
                                            ("sspi", dict(taps=4.0), "bf16"), ("sspi", dict(taps=4.0), "fp32"),
                                            ("conv", {}, "fp32")])
def test_estimates_only(S, uca_small, method, kw, prec):
    """srp_map with maps = NULL: the argmax equals the argmax of the full map call (on the
    tensor cores no map is written at all)."""
    import torch
    name, F, sub, w, psi, dt, lags, perm, xi_o = uca_small
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method=method, precision=prec,
                  max_frames=64, **kw)
    frames = torch.from_numpy(np.ascontiguousarray(w["frames"])).cuda()
    z, am = plan.map(frames)
    _, am2 = plan.map(frames, want_maps=False)
    torch.cuda.synchronize()
    plan.status()
    assert np.array_equal(am.cpu().numpy(), am2.cpu().numpy())
    assert np.array_equal(am2.cpu().numpy(), np.argmax(z.cpu().numpy(), axis=1))


@pytest.mark.parametrize("name,F,sub,rank,prec", [
    ("square4", None, 1, 8, "fp32"), ("square4", None, 1, 16, "fp16x3"), ("square4", None, 1, 8, "bf16"),
    ("uca8", 70, 50, 12, "fp32"), ("uca8", 70, 50, 12, "fp16x3"),
])
def test_lr_srp(S, name, F, sub, rank, prec):
    """LR-SRP (the paper's low-rank competitor, boxed Eq. z_lr): rank-R factors of the complex
    SRP matrix from the device subspace iteration; singular values and maps vs the oracle's
    SVD."""
    w = R.workload(name, F, sub)
    dt, *_ = R.geometry(name, F, sub)
    psi = R.psi_of(w["frames"])
    H = O.steering_matrix_H(dt, w["fs"], w["N"] // 2).reshape(dt.shape[0], -1)
    tall, fat = O.lr_factors(H, rank)
    s = np.linalg.svd(H, compute_uv=False)
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="lr", rank=rank,
                  precision=prec, max_frames=64)
    assert np.allclose(plan.slri_sigma(rank + 1), s[:rank + 1], rtol=1e-8, atol=1e-8 * s[0])
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = O.srp_lr(tall, fat, psi.reshape(psi.shape[0], -1))
    assert R.per_frame_rel(z, zo).max() <= dict(PRECS)[prec]
    check_argmax(z, am, zo)
