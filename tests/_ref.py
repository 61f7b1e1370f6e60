"""Oracle references for the parity tests (CPU, FP64).  Only calls ``oracle`` and
``synth``; no expected value here comes from the CUDA path.  It also holds a reader of
the plan files the library writes, for tests that check a plan's own factors."""
from __future__ import annotations

import functools
import struct

import numpy as np

import oracle as O
import synth

C = 340.0


@functools.lru_cache(maxsize=8)
def workload(name, F=None, sub=1):
    return synth.workload(name, F=F, grid_subsample=sub)


@functools.lru_cache(maxsize=8)
def geometry(name, F=None, sub=1, n_aux=2):
    w = workload(name, F, sub)
    dt = O.tdoa_nf(w["mic_xyz"], w["grid_xyz"], C)
    Np = O.n_p_samples(w["mic_xyz"], w["fs"], C, n_aux)
    lags = O.pair_lags(Np)
    perm = O.lags_to_ascending(lags)
    return dt, Np, lags, perm


def psi_of(frames, window="hann"):
    return O.gcc_phat(O.stft(frames, window))


def xi_ascending(psi, lags, perm, K):
    """Oracle TD GCC samples (iFFT route, Eq. xi_p_ifft) reordered to ascending lags."""
    xi, _ = O.gcc_samples_ifft(psi, lags, K)
    return xi[:, perm]


@functools.lru_cache(maxsize=8)
def lam(name, F=None, sub=1):
    w = workload(name, F, sub)
    dt, Np, lags, perm = geometry(name, F, sub)
    return O.interp_matrix(dt, w["fs"], lags)


@functools.lru_cache(maxsize=16)
def slri(name, R, F=None, sub=1):
    tall, fat, s = O.slri_factors(lam(name, F, sub), R)
    return tall, fat, s


@functools.lru_cache(maxsize=16)
def sspi(name, t, F=None, sub=1):
    w = workload(name, F, sub)
    dt, Np, lags, perm = geometry(name, F, sub)
    Lam = lam(name, F, sub)
    nnz = int(round(t * Lam.shape[0] * len(lags)))
    mask, tied, taken = O.sspi_select(Lam, lags, nnz)
    return mask, tied, taken, nnz


def conv_cells(psi, dt, fs, cells):
    """conv. FD-SRP on a subset of grid cells (Eq. z_computed restricted to rows)."""
    return O.srp_conv(psi, dt[cells], fs)


def per_frame_rel(a, ref):
    return O.rel_err(np.asarray(a, np.float64), ref, axis=-1)


def gram_apply(dt, fs, lags, perm, Y, rows=256, workers=None):
    """Lambda^T (Lambda Y) in FP64 for Y [L][b], with Lambda (Eq. Lambda, columns in the
    GPU's ascending-lag order) generated by oracle.interp_matrix in blocks of `rows` grid
    cells on a thread pool and never held whole (walls16's Lambda is 25 GB in FP64).
    Blocks are summed in grid order, so the result does not depend on the thread count."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    J = dt.shape[0]
    workers = workers or max(1, min(16, os.cpu_count() or 1))

    def part(j0):
        lam_rows = O.interp_matrix(dt[j0:j0 + rows], fs, lags)[:, perm]
        return lam_rows.T @ (lam_rows @ Y)

    out = None
    with ThreadPoolExecutor(workers) as ex:
        for r in ex.map(part, range(0, J, rows)):
            out = r if out is None else out + r
    return out


def top_subspace_certificate(apply, V, b=16, passes=3, seed=7):
    """Evidence that the orthonormal columns of V [L][R] span the top-R right singular
    subspace of Lambda (the Eckart-Young optimum of Eq. min_Lambda_lr), from products
    G = Lambda^T Lambda Y only (`apply`).

    Returns (ritz, resid, mu):
      ritz  -- eigenvalues of V^T G V (sigma_r^2 of the fit, descending);
      resid -- max over columns of ||G V - V (V^T G V)||, relative to ritz[0]: zero when
               span(V) is an invariant subspace;
      mu    -- the largest Rayleigh quotient found outside span(V) by `passes` steps of a
               block subspace iteration (b random columns, V deflated every step).  It
               approaches sigma_{R+1}^2 when V is the top-R subspace, and the largest
               missed sigma^2 (> sigma_R^2) when it is not."""
    V, _ = np.linalg.qr(np.asarray(V, np.float64))  # the subspace, orthonormal in FP64
    L, R = V.shape
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((L, b))
    X -= V @ (V.T @ X)
    X, _ = np.linalg.qr(X)
    Z = apply(np.hstack([V, X]))
    GV, GX = Z[:, :R], Z[:, R:]
    B = V.T @ GV
    B = 0.5 * (B + B.T)
    ritz = np.sort(np.linalg.eigvalsh(B))[::-1]
    resid = float(np.max(np.linalg.norm(GV - V @ B, axis=0)) / ritz[0])
    for _ in range(passes - 1):
        X = GX - V @ (V.T @ GX)
        X, _ = np.linalg.qr(X)
        GX = apply(X)
    Gd = GX - V @ (V.T @ GX)
    C = X.T @ Gd
    mu = float(np.linalg.eigvalsh(0.5 * (C + C.T)).max())
    return ritz, resid, mu


def read_slri_plan(path):
    """Lambda_tall [J][Rp] and Lambda_fat [Rp][L] from a saved SLRI plan (the little-endian
    format srp_plan_save documents)."""
    b = open(path, "rb").read()
    assert b[:8] == b"SRPPLAN\0"
    pos = 8
    version, method, _h = struct.unpack_from("<Iiq", b, pos)
    pos += 16
    J, P, L, R = struct.unpack_from("<iiii", b, pos)
    pos += 16

    def vec(dtype):
        nonlocal pos
        (n,) = struct.unpack_from("<Q", b, pos)
        pos += 8
        a = np.frombuffer(b, dtype=dtype, count=n, offset=pos)
        pos += n * np.dtype(dtype).itemsize
        return a

    sigma = vec(np.float64)
    tall = vec(np.float32)
    fat = vec(np.float32)
    Rp = tall.size // J
    return tall.reshape(J, Rp), fat.reshape(Rp, L), sigma, R
