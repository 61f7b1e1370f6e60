"""Oracle references for the parity tests (CPU, FP64).  Only calls ``oracle`` and
``synth``; nothing here comes from the CUDA path."""
from __future__ import annotations

import functools

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
