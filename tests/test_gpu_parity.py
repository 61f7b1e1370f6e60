"""Parity of the CUDA path (through the C-ABI) against the FP64 oracle, on the GPU.

Tolerances: FP32 paths must match the oracle to <= 1e-5 relative per frame
(sqrt(||z_gpu - z||^2 / ||z||^2)); the argmax the GPU returns must be the argmax of
its own FP32 map exactly (same precision decides), and a valid argmax of the oracle map
within the GPU's measured error.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests import _ref as R

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2306_08514_gb300 as S
    S.lib()
    return S


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(plan, frames):
    import torch
    maps, am = plan.map(_cuda(frames))
    torch.cuda.synchronize()
    return maps.cpu().numpy(), am.cpu().numpy()


def check_argmax(z, am, zo):
    assert np.array_equal(am, np.argmax(z, axis=1)), "argmax differs from the GPU map's own"
    err = np.max(np.abs(z.astype(np.float64) - zo), axis=1)
    picked = zo[np.arange(len(am)), am]
    assert np.all(picked >= zo.max(axis=1) - 2 * err - 1e-9), "argmax is not a valid oracle maximum"
    return float(np.mean(am == np.argmax(zo, axis=1)))


# ------------------------------------------------------------------ sampling stage
@pytest.mark.parametrize("N,half", [(256, 0.1), (512, 0.1), (1024, 0.1), (2048, 0.1),
                                    (512, 0.02), (512, 0.2), (1024, 0.2), (512, 1.0), (1024, 1.0),
                                    (2048, 1.5)])
def test_gcc_samples_match_oracle(S, N, half):
    """Eq. xi_p_ifft / n_prime on the GPU vs the oracle's iFFT sampling.  Square arrays of
    half-side `half` give max N_p of 4 (0.02), 15 (0.1), 28 (0.2) -- the sampling GEMM with
    2, 4 and 9 n-tiles of lags (in the fused front end for N <= 1024, from spectra in global
    memory for N = 2048) -- and 135 / 201 (1.0 / 1.5): the iFFT kernel."""
    mics = synth.mics_square(half=half)
    grid = synth.grid_plane((1, 1), (3, 3), (8, 8))
    g = synth.rng(N)
    frames = g.standard_normal((37, 4, N)).astype(np.float32)
    plan = S.Plan(mics, grid, 16000.0, N, method="si", max_frames=16)
    import torch
    xi = plan.gcc_samples(_cuda(frames)).cpu().numpy()
    torch.cuda.synchronize()
    Np = O.n_p_samples(mics, 16000.0)
    assert np.array_equal(plan.lags(), Np)
    lags = O.pair_lags(Np)
    ref = R.xi_ascending(R.psi_of(frames), lags, O.lags_to_ascending(lags), N // 2)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(xi - ref) / scale) <= TOL


@pytest.mark.parametrize("N,M,diam,prec", [(2048, 40, 0.1, "fp32"), (2048, 40, 0.25, "fp16x3"),
                                           (2048, 40, 0.6, "fp32"), (1024, 40, 0.25, "bf16"),
                                           (256, 48, 0.6, "fp32")])
def test_gcc_samples_many_channels_short_windows(S, N, M, diam, prec):
    """Sampling GEMM from spectra in global memory (frames the fused front end cannot hold:
    N = 2048, or 40-48 channels): 780-1128 pairs (two or more rounds of m-tiles per frame),
    max N_p in each n-tile bucket (15, 31 and 65 lags), against the oracle's iFFT sampling
    (Eq. xi_p_ifft / n_prime).  Bounds: the FP32 1e-5 on each frame's samples as a whole
    (sqrt(sum err^2 / sum xi^2), the measure of the maps); sample by sample 5e-5 of the
    frame's largest sample, because with 10^5-10^6 samples per test the largest single
    error comes from PHAT's division at the weakest bin of a frame (FP32 spectra: a bin
    10^3 below the frame's typical magnitude turns a 1e-7 rounding into a 1e-4 phase
    error), whatever the sampling kernel."""
    g = synth.rng(N + M)
    v = g.standard_normal((M, 3))
    mics = (2.0, 2.0, 1.0) + 0.5 * diam * v / np.linalg.norm(v, axis=1, keepdims=True)
    grid = synth.grid_plane((1, 1), (3, 3), (8, 8))
    frames = g.standard_normal((37, M, N)).astype(np.float32)
    plan = S.Plan(mics, grid, 16000.0, N, method="si", precision=prec, max_frames=16)
    import torch
    xi = plan.gcc_samples(_cuda(frames)).cpu().numpy()
    torch.cuda.synchronize()
    Np = O.n_p_samples(mics, 16000.0)
    assert np.array_equal(plan.lags(), Np)
    assert Np.max() <= 32
    lags = O.pair_lags(Np)
    ref = R.xi_ascending(R.psi_of(frames), lags, O.lags_to_ascending(lags), N // 2)
    assert R.per_frame_rel(xi, ref).max() <= TOL
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(xi - ref) / scale) <= 5 * TOL


# ------------------------------------------------------------------ square4 (full size)
@pytest.fixture(scope="module")
def sq():
    w = R.workload("square4")
    psi = R.psi_of(w["frames"])
    dt, Np, lags, perm = R.geometry("square4")
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    return w, psi, dt, lags, perm, xi_o


def test_conv_fp32_square4(S, sq):
    w, psi, dt, *_ = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv", max_frames=64)
    z, am = _run(plan, w["frames"])
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= TOL
    assert check_argmax(z, am, zo) >= 0.99


# Tensor-core conv bounds: FP16 hi+lo and TF32 hi+lo (22 significant bits) meet the FP32
# bar; single FP16 / TF32 / BF16 operands carry a relative rounding of 2^-11 / 2^-11 / 2^-8
# per operand, i.e. about sqrt(2/3) u of map error for sums of many terms: stated bounds
# 2e-3 (FP16, TF32) and 1.5e-2 (BF16); BF16 hi+lo keeps 16 significant bits (the dropped
# lo*lo and the rounding of lo are ~2^-16 per product): stated bound 1e-4.
TC_CASES = [("fp16x3", TOL), ("tf32x3", TOL), ("bf16x3", 1e-4), ("fp16", 2e-3), ("tf32", 2e-3),
            ("bf16", 1.5e-2)]


@pytest.mark.parametrize("prec,tol", TC_CASES)
def test_conv_tensor_core_square4(S, sq, prec, tol):
    w, psi, dt, *_ = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv", precision=prec,
                  max_frames=64)
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)
    if prec.endswith("x3"):  # the hi + lo per stage kernel, alone and in clusters of two
        for v in (3, 7):
            plan.set_variant(v)
            z, am = _run(plan, w["frames"])
            plan.status()
            assert R.per_frame_rel(z, zo).max() <= tol, v
            check_argmax(z, am, zo)


@pytest.mark.parametrize("rank", [8, 16])
def test_slri_square4(S, sq, rank):
    w, psi, dt, lags, perm, xi_o = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="slri", rank=rank,
                  max_frames=64)
    tall, fat, s = R.slri("square4", rank)
    sig = plan.slri_sigma(rank + 1)
    assert np.allclose(sig, s[:rank + 1], rtol=1e-9, atol=1e-9 * s[0])
    z, am = _run(plan, w["frames"])
    zo = O.srp_slri(tall, fat, xi_o)
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)


def _check_taps(plan, mask_o, perm, lam_o):
    """The plan's SSPI taps against the oracle's global top-Q_Lambda selection (Eq.
    min_Lambda_sp): the same count, Lambda's own values, and the same set except for
    entries tied at the cut (equal quantised magnitudes), where several selections are
    optimal.  Returns the plan's selection as a mask in the oracle's column order, so that
    the map is compared with Lambda masked by the taps the plan actually uses."""
    J, L = mask_o.shape
    row_ptr, col, val = plan.sspi_taps()
    assert row_ptr[-1] == mask_o.sum()
    m = np.zeros((J, L), bool)
    rows = np.repeat(np.arange(J), np.diff(row_ptr))
    m[rows, col] = True
    assert m.sum() == mask_o.sum(), "repeated taps"
    mo = mask_o[:, perm]
    lam_a = lam_o[:, perm]
    diff = m != mo
    if diff.any():  # only ties at the cut may differ (quantised magnitudes equal)
        keys = np.floor(np.abs(lam_a) * 2.0 ** 40 + 0.5)
        kmin = keys[mo].min()
        assert np.all(keys[diff] == kmin)
        assert keys[m].min() == kmin and not np.any(~m & (keys > kmin))
    assert np.allclose(val, lam_a[rows, col].astype(np.float32), rtol=0, atol=0)
    mask_g = np.zeros((J, L), bool)
    mask_g[:, perm] = m
    return mask_g


@pytest.mark.parametrize("t", [0.5, 1.0, 2.0, 4.0])
def test_sspi_square4(S, sq, t):
    w, psi, dt, lags, perm, xi_o = sq
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="sspi", taps=t,
                  max_frames=64)
    mask, tied, taken, nnz = R.sspi("square4", t)
    assert plan.info.nnz == nnz
    mask_g = _check_taps(plan, mask, perm, R.lam("square4"))
    z, am = _run(plan, w["frames"])
    zo = O.srp_sspi(np.where(mask_g, R.lam("square4"), 0.0), xi_o)
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)


# ------------------------------------------------------------------ uca8, several tiles
@pytest.fixture(scope="module")
def uca_small():
    name, F, sub = "uca8", 70, 13
    w = R.workload(name, F, sub)
    psi = R.psi_of(w["frames"])
    dt, Np, lags, perm = R.geometry(name, F, sub)
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    return name, F, sub, w, psi, dt, lags, perm, xi_o


def test_uca8_small_all_methods(S, uca_small):
    name, F, sub, w, psi, dt, lags, perm, xi_o = uca_small
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    z, am = _run(S.Plan(*args, method="conv", max_frames=64), w["frames"])
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)
    for prec, tol in TC_CASES:  # ragged frame tile (70 = 64 + 6) and cell tile (4616 cells)
        plan = S.Plan(*args, method="conv", precision=prec, max_frames=64)
        z, am = _run(plan, w["frames"])
        plan.status()
        assert R.per_frame_rel(z, zo).max() <= tol, prec
        check_argmax(z, am, zo)
    tall, fat, s = R.slri(name, 16, F, sub)
    z, am = _run(S.Plan(*args, method="slri", rank=16, max_frames=64), w["frames"])
    zo = O.srp_slri(tall, fat, xi_o)
    assert R.per_frame_rel(z, zo).max() <= TOL
    mask, tied, taken, nnz = R.sspi(name, 4.0, F, sub)
    plan = S.Plan(*args, method="sspi", taps=4.0, max_frames=64)
    mask_g = _check_taps(plan, mask, perm, R.lam(name, F, sub))
    z, am = _run(plan, w["frames"])
    zo = O.srp_sspi(np.where(mask_g, R.lam(name, F, sub), 0.0), xi_o)
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)


# ------------------------------------------------------------------ edge cases
def test_edge_cases(S):
    import torch
    mics = synth.mics_square()
    grid = synth.grid_plane((0, 0), (4, 4), (5, 5))
    plan = S.Plan(mics, grid, 16000.0, 512, method="conv", max_frames=8)
    empty = torch.empty((0, 4, 512), device="cuda")
    maps, am = plan.map(empty)
    assert maps.shape == (0, 25)
    with pytest.raises(S.SrpError) as e:
        S.srp_map(plan.handle, None, 3, None, None, None)
    assert e.value.status == S.SRP_EINVAL
    with pytest.raises(S.SrpError):
        S.srp_map(plan.handle, None, -1, None, None, None)
    # a single location, a single frame, every method
    g1 = grid[12:13]
    fr = synth.rng(1).standard_normal((1, 4, 512)).astype(np.float32)
    psi = R.psi_of(fr)
    dt = O.tdoa_nf(mics, g1)
    for kw in (dict(method="conv"), dict(method="slri", rank=1), dict(method="sspi", taps=1.0)):
        z, am = _run(S.Plan(mics, g1, 16000.0, 512, max_frames=1, **kw), fr)
        assert am[0] == 0 and np.isfinite(z).all()
    zc, _ = _run(S.Plan(mics, g1, 16000.0, 512, method="conv"), fr)
    assert abs(zc[0, 0] - O.srp_conv(psi, dt, 16000.0)[0, 0]) <= TOL * abs(O.srp_conv(psi, dt, 16000.0)[0, 0]) + 1e-3


def test_silent_channel(S):
    w = R.workload("square4")
    fr = w["frames"][:9].copy()
    fr[:, 2, :] = 0.0
    psi = R.psi_of(fr)
    dt, *_ = R.geometry("square4")
    z, am = _run(S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv"), fr)
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= TOL


def test_invalid_plans_rejected(S):
    mics = synth.mics_square()
    grid = synth.grid_plane((0, 0), (4, 4), (5, 5))
    with pytest.raises(S.SrpError) as e:
        S.Plan(mics, grid, 16000.0, 500)
    assert e.value.status == S.SRP_EINVAL
    far = mics * 40.0  # pairs so far apart that N_p >= K
    with pytest.raises(S.SrpError) as e:
        S.Plan(far, grid, 16000.0, 256)
    assert e.value.status == S.SRP_EINVAL


def test_host_entry_matches_device_entry_and_is_deterministic(S):
    w = R.workload("square4")
    fr = np.ascontiguousarray(w["frames"][:40])
    for kw in (dict(method="conv"), dict(method="slri", rank=8), dict(method="sspi", taps=2.0)):
        plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], max_frames=16, **kw)
        z1, a1 = _run(plan, fr)
        z2, a2 = _run(plan, fr)
        assert np.array_equal(z1, z2) and np.array_equal(a1, a2)
        zh, ah = plan.map_host(fr)
        assert np.array_equal(zh, z1) and np.array_equal(ah, a1)


@pytest.mark.parametrize("kw", [dict(method="conv", precision="bf16"),
                                dict(method="slri", rank=8),
                                dict(method="sspi", taps=2.0, precision="bf16")],
                         ids=["conv-bf16", "slri-fp32", "sspi-bf16"])
def test_host_entry_pipelined_sub_batches(S, kw):
    """srp_map_host splits a chunk into sub-batches whose frames come in and whose maps leave
    on copy streams while the next computes; 1000 frames through 600-frame chunks give
    several sub-batches per chunk and a ragged last one.  Maps agree with the device entry
    (FP32 sums may be ordered differently), argmax is the host map's own."""
    w = R.workload("square4", 1000)
    fr = np.ascontiguousarray(w["frames"])
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], max_frames=600, **kw)
    z1, a1 = _run(plan, fr)
    zh, ah = plan.map_host(fr)
    plan.status()
    assert R.per_frame_rel(zh, z1).max() <= 1e-6
    assert np.array_equal(ah, np.argmax(zh, axis=1))
    gap = np.sort(z1, axis=1)[:, -1] - np.sort(z1, axis=1)[:, -2]
    clear = gap > 1e-5 * np.abs(z1).max(axis=1)
    assert np.array_equal(ah[clear], a1[clear])


def test_largest_fft_and_most_mics_conv(S):
    """N = 2048 and M = 32 (nested arrays) on a reduced grid."""
    w = R.workload("nested32", 6, 400)
    psi = R.psi_of(w["frames"])
    dt, *_ = R.geometry("nested32", 6, 400)
    z, am = _run(S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv",
                        max_frames=4), w["frames"])
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)
    # tensor cores, FP16 hi+lo: 3 output tiles, so the reduction is split into slices summed in FP64
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv",
                  precision="fp16x3", max_frames=4)
    z, am = _run(plan, w["frames"])
    plan.status()
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)


# ------------------------------------------------------------------ full-size uca8 (bench config)
@pytest.fixture(scope="module")
def uca_full():
    w = R.workload("uca8")
    return w


def test_uca8_full_size_sampled(S, uca_full):
    """The benchmark's workload (M=8 UCA, J=60000, F=2000, one launch per method): the
    oracle evaluates sampled frames exactly."""
    w = uca_full
    F = w["F"]
    frames = w["frames"]
    fsel = np.array([0, 1, 777, 1500, F - 1])
    psi = R.psi_of(frames[fsel])
    dt, Np, lags, perm = R.geometry("uca8")
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    # conv, FP32, on all J for the sampled frames
    z, am = _run(S.Plan(*args, method="conv", max_frames=F), frames)
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z[fsel], zo).max() <= TOL
    check_argmax(z[fsel], am[fsel], zo)
    # conv on the tensor cores, FP16 hi+lo, in the benchmark's launch configuration
    plan = S.Plan(*args, method="conv", precision="fp16x3", max_frames=F)
    z, am = _run(plan, frames)
    plan.status()
    assert R.per_frame_rel(z[fsel], zo).max() <= TOL
    check_argmax(z[fsel], am[fsel], zo)
    # the hi + lo per stage kernel alone and in clusters of 2 CTAs sharing the SRP matrix's
    # tiles by multicast (16 frame tiles per cell tile): the same maps bit for bit
    plan.set_variant(3)
    z3, am3 = _run(plan, frames)
    assert R.per_frame_rel(z3[fsel], zo).max() <= TOL
    for v in (7, 11):  # clusters of 2 and of 2 x 2
        plan.set_variant(v)
        zc, amc = _run(plan, frames)
        plan.status()
        assert np.array_equal(zc, z3) and np.array_equal(amc, am3), v
    del z3, zc
    # SLRI, R = 16
    tall, fat, s = R.slri("uca8", 16)
    z, am = _run(S.Plan(*args, method="slri", rank=16, max_frames=F), frames)
    zo = O.srp_slri(tall, fat, xi_o)
    assert R.per_frame_rel(z[fsel], zo).max() <= TOL
    check_argmax(z[fsel], am[fsel], zo)
    # SSPI, t = 4
    mask, tied, taken, nnz = R.sspi("uca8", 4.0)
    plan = S.Plan(*args, method="sspi", taps=4.0, max_frames=F)
    mask_g = _check_taps(plan, mask, perm, R.lam("uca8"))
    z, am = _run(plan, frames)
    zo = O.srp_sspi(np.where(mask_g, R.lam("uca8"), 0.0), xi_o)
    assert R.per_frame_rel(z[fsel], zo).max() <= TOL
    check_argmax(z[fsel], am[fsel], zo)


@pytest.mark.parametrize("method,kw,hop", [("conv", {}, 256), ("sspi", dict(taps=2.0, precision="bf16"), 128),
                                           ("slri", dict(rank=8, precision="fp16x3"), 512)])
def test_stream_push_keeps_overlap(S, method, kw, hop):
    """srp_stream_push on a signal pushed in uneven blocks = srp_map on the frames cut from the
    zero-padded stream (frame b = the N samples ending with block b)."""
    import torch
    w = R.workload("square4")
    N, M = w["N"], w["mic_xyz"].shape[0]
    x = synth.rng(77).standard_normal((M, 41 * hop)).astype(np.float32)
    cat = np.concatenate([np.zeros((M, N - hop), np.float32), x], axis=1)
    nb = x.shape[1] // hop
    frames = np.stack([cat[:, b * hop:b * hop + N] for b in range(nb)])
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], N, method=method, max_frames=16, **kw)
    zr, ar = _run(plan, frames)
    hops = np.ascontiguousarray(x.reshape(M, nb, hop).transpose(1, 0, 2))
    out, outa, b0 = [], [], 0
    for B in [1, 3, 20, 0, 7, 10]:  # 20 > max_frames: chunked inside
        B = min(B, nb - b0)
        m, a = plan.stream_push(_cuda(hops[b0:b0 + B]))
        torch.cuda.synchronize()
        out.append(m.cpu().numpy())
        outa.append(a.cpu().numpy())
        b0 += B
    z = np.concatenate(out)
    am = np.concatenate(outa)
    assert z.shape == zr.shape
    assert np.array_equal(z, zr) or R.per_frame_rel(z, zr.astype(np.float64)).max() <= 1e-6
    assert np.array_equal(am, np.argmax(z, axis=1))
    with pytest.raises(S.SrpError):
        plan.stream_push(_cuda(np.zeros((1, M, hop // 2), np.float32)))  # hop changed
    plan.stream_reset()
    m, a = plan.stream_push(_cuda(hops[:2]))
    torch.cuda.synchronize()
    assert np.array_equal(m.cpu().numpy(), zr[:2])


@pytest.mark.parametrize("name,F,sub", [("square4", None, 1), ("uca8", 70, 13), ("nested32", 6, 400)])
def test_conv_srp_matrix_generated_on_the_fly(S, name, F, sub):
    """conv. FD-SRP with the SRP matrix generated inside the FP32 GEMM (for grids whose
    stored matrix would not fit): same maps as the FP64 oracle, N up to 2048."""
    w = R.workload(name, F, sub)
    dt, *_ = R.geometry(name, F, sub)
    psi = R.psi_of(w["frames"])
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv", h_on_the_fly=1,
                  max_frames=64)
    assert plan.info.device_bytes < w["grid_xyz"].shape[0] * plan.P * w["N"] * 4  # H not stored
    z, am = _run(plan, w["frames"])
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)


@pytest.mark.parametrize("name,F,sub,t", [("walls16", 70, 37, 4.0), ("nested32", 37, 101, 8.0),
                                          ("walls16", 9, 300, 0.5)])
def test_sspi_fp32_long_sample_vectors(S, name, F, sub, t):
    """The FP32 SSPI gather beyond the whole-vector kernel's reach (walls16 L = 43326,
    nested32 L = 7408): each 64-cell block stages only the columns its taps use.  Against
    the oracle masked by the plan's validated taps, FP32 bound; ragged frame and cell
    blocks."""
    w = R.workload(name, F, sub)
    dt, Np, lags, perm = R.geometry(name, F, sub)
    psi = R.psi_of(w["frames"])
    xi_o, _ = O.gcc_samples_ifft(psi, lags, w["N"] // 2)
    mask, tied, taken, nnz = R.sspi(name, t, F, sub)
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="sspi", taps=t,
                  max_frames=64)
    Lam = R.lam(name, F, sub)
    mask_g = _check_taps(plan, mask, perm, Lam)
    z, am = _run(plan, w["frames"])
    zo = O.srp_sspi(np.where(mask_g, Lam, 0.0), xi_o)
    assert R.per_frame_rel(z, zo).max() <= TOL
    check_argmax(z, am, zo)


@pytest.mark.parametrize("prec,tol", [("fp16x3", TOL), ("bf16", 1.5e-2), ("tf32x3", TOL)])
def test_conv_tensor_cores_with_srp_matrix_in_chunks(S, uca_small, prec, tol):
    """Conv. FD-SRP on the tensor cores without the whole SRP matrix stored: the rows of one
    chunk of cells are generated before that chunk's GEMM (h_on_the_fly).  A batch size of
    32768 frames makes the chunks 512 cells (about two waves of tiles), so the 4616 cells
    take ten chunks, the last of 8 cells; maps and estimates-only calls against the oracle."""
    import torch
    name, F, sub, w, psi, dt, lags, perm, xi_o = uca_small
    plan = S.Plan(w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"], method="conv", precision=prec,
                  max_frames=32768, h_on_the_fly=1)
    z, am = _run(plan, w["frames"])
    plan.status()
    zo = O.srp_conv(psi, dt, w["fs"])
    assert R.per_frame_rel(z, zo).max() <= tol
    check_argmax(z, am, zo)
    _, am2 = plan.map(_cuda(w["frames"]), want_maps=False)
    torch.cuda.synchronize()
    assert np.array_equal(am2.cpu().numpy(), am)
