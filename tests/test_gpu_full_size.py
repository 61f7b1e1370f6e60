"""The large workloads at their full sizes, in the launch configuration bench.py times
(BF16; walls16: M = 16, J = 72000, N = 1024, F = 4096; nested32: M = 32, J = 240000,
N = 2048, F = 1024).  The FP64 oracle cannot evaluate these whole (the SVD of walls16's
72000 x 43326 Lambda, nested32's 952 M SSPI taps), so sampled outputs are checked:

* conv: the oracle's map on 256 sampled cells of two sampled frames (walls16 in BF16;
  nested32 in FP16 hi+lo with its SRP matrix generated in chunks of cells);
* SLRI: the plan's own factors (read back from its checkpoint file) applied in FP64 to the
  oracle's GCC samples, the fit on the sampled rows (Lambda_tall = Lambda V, V
  orthonormal), and that V spans the top-R singular subspace of the whole Lambda: the
  Ritz residual of Lambda^T Lambda V and a deflated subspace iteration that finds no
  direction outside span(V) above sigma_R^2, with Lambda streamed from the oracle in row
  blocks (FP64);
* SSPI: the plan's taps applied in FP64 to the oracle's samples, the tap count, and the
  global top-Q_Lambda property on the sampled rows (every entry above the smallest kept
  magnitude is kept, every entry below it dropped).
"""
import numpy as np
import pytest

import oracle as O
from tests import _ref as R
from tests.test_gpu_parity import S, _run  # noqa: F401

pytestmark = pytest.mark.gpu

BF16_TOL = 1.5e-2


def _setup(name):
    w = R.workload(name)
    dt, Np, lags, perm = R.geometry(name)
    F = w["F"]
    rng = np.random.default_rng(2024)
    fsel = np.array([0, F // 2 + 1])
    cells = np.sort(rng.choice(w["grid_xyz"].shape[0], 256, replace=False))
    psi = R.psi_of(w["frames"][fsel])
    xi = R.xi_ascending(psi, lags, perm, w["N"] // 2)  # the GPU's sample order
    lam_cells = O.interp_matrix(dt[cells], w["fs"], lags)[:, perm]
    return w, dt, lags, perm, fsel, cells, psi, xi, lam_cells


def _check_slri(S, w, dt, lags, perm, fsel, cells, xi, lam_cells, rank, tmp_path):
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    plan = S.Plan(*args, method="slri", rank=rank, precision="bf16", max_frames=w["F"])
    z, am = _run(plan, w["frames"])
    plan.status()
    assert np.array_equal(am, np.argmax(z, axis=1))
    plan.save(tmp_path / "slri.plan")
    tall, fat, sigma, Rr = R.read_slri_plan(tmp_path / "slri.plan")
    V = fat[:rank].astype(np.float64).T  # [L][R]
    # the fit: orthonormal V, Lambda_tall = Lambda V on the sampled rows
    assert np.abs(V.T @ V - np.eye(rank)).max() < 1e-5
    want = lam_cells @ V
    got = tall[cells, :rank].astype(np.float64)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    # V spans the top-R right singular subspace of the whole Lambda (Eckart-Young, Eq.
    # min_Lambda_lr).  V is stored in FP32 (2^-24 per entry), so its Ritz residual is
    # bounded by about sigma_1^2 * 2^-24 * sqrt(R); 1e-6 leaves margin for that and nothing
    # for a stalled iteration.  The plan's sigma are the square roots of the Ritz values.
    ritz, resid, mu = R.top_subspace_certificate(
        lambda Y: R.gram_apply(dt, w["fs"], lags, perm, Y), V)
    sig = plan.slri_sigma(rank)
    assert resid <= 1e-6, resid
    assert np.allclose(np.sqrt(ritz), sig, rtol=1e-6, atol=0), (np.sqrt(ritz), sig)
    assert mu < ritz[-1] * (1 - 1e-6), (mu, ritz[-1])
    # the run-time path: z = Lambda_tall (Lambda_fat xi) with the plan's factors, in FP64
    zo = (xi @ V) @ tall[cells, :rank].astype(np.float64).T
    assert R.per_frame_rel(z[fsel][:, cells], zo).max() <= BF16_TOL


def _check_sspi(S, w, fsel, cells, xi, lam_cells, t):
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    plan = S.Plan(*args, method="sspi", taps=t, precision="bf16", max_frames=w["F"])
    z, am = _run(plan, w["frames"])
    plan.status()
    assert np.array_equal(am, np.argmax(z, axis=1))
    row_ptr, col, val = plan.sspi_taps()
    J, P = w["grid_xyz"].shape[0], plan.P
    assert row_ptr[-1] == int(round(t * J * P))
    cut = np.abs(val).min()
    zo = np.zeros((len(fsel), len(cells)))
    for j, i in enumerate(cells):
        c, v = col[row_ptr[i]:row_ptr[i + 1]], val[row_ptr[i]:row_ptr[i + 1]].astype(np.float64)
        row = lam_cells[j]
        assert np.allclose(v, row[c], rtol=1e-6, atol=1e-7)  # the taps are Lambda's entries
        kept = np.zeros(row.size, bool)
        kept[c] = True
        mag = np.abs(row)
        assert not np.any(kept & (mag < cut * (1 - 1e-6)))   # nothing below the cut kept
        assert not np.any(~kept & (mag > cut * (1 + 1e-6)))  # nothing above the cut dropped
        zo[:, j] = xi[:, c] @ v
    assert R.per_frame_rel(z[fsel][:, cells], zo).max() <= BF16_TOL


def test_walls16_full_size_sampled(S, tmp_path):
    w, dt, lags, perm, fsel, cells, psi, xi, lam_cells = _setup("walls16")
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    plan = S.Plan(*args, method="conv", precision="bf16", max_frames=w["F"])
    z, am = _run(plan, w["frames"])
    plan.status()
    assert np.array_equal(am, np.argmax(z, axis=1))
    zo = R.conv_cells(psi, dt, w["fs"], cells)
    assert R.per_frame_rel(z[fsel][:, cells], zo).max() <= BF16_TOL
    del plan, z
    _check_slri(S, w, dt, lags, perm, fsel, cells, xi, lam_cells, 16, tmp_path)
    _check_sspi(S, w, fsel, cells, xi, lam_cells, 4.0)


def test_nested32_full_size_sampled(S, tmp_path):
    w, dt, lags, perm, fsel, cells, psi, xi, lam_cells = _setup("nested32")
    # conv. FD-SRP on the tensor cores in FP16 hi+lo: the SRP matrix (975 GB as hi + lo
    # planes) is generated in chunks of cells before each chunk's GEMM
    args = (w["mic_xyz"], w["grid_xyz"], w["fs"], w["N"])
    plan = S.Plan(*args, method="conv", precision="fp16x3", max_frames=w["F"])
    z, am = _run(plan, w["frames"])
    plan.status()
    assert np.array_equal(am, np.argmax(z, axis=1))
    zo = R.conv_cells(psi, dt, w["fs"], cells)
    assert R.per_frame_rel(z[fsel][:, cells], zo).max() <= 1e-5
    del plan, z
    _check_slri(S, w, dt, lags, perm, fsel, cells, xi, lam_cells, 16, tmp_path)
    _check_sspi(S, w, fsel, cells, xi, lam_cells, 8.0)
