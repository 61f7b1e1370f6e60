"""FP64 reference implementation of conventional FD-SRP, SI-SRP, SLRI-SRP, SSPI-SRP
(and conv. TD-SRP, LR-SRP as comparison points) -- TEST INFRASTRUCTURE ONLY.

Notation follows the paper: M microphones, P = M(M-1)/2 pairs p <-> (m, m') with
m > m', J candidate locations, DFT length 2K, one-sided bins k = 1..K-1, sampling
period T = 1/fs.  Arrays are 0-based; the paper's 1-based "mod[.]+1" indices become
plain "mod[.]".

Readings of points where the paper is silent (both this oracle and the CUDA library take them):
* sinc(x) = sin(pi x)/(pi x), sinc(0) = 1 (Whittaker-Shannon, Eq. SRPinterp).
* The iFFT is the unnormalised inverse DFT, i.e. 2K * numpy.fft.ifft (Eq. xi_p_ifft,
  which must equal S-bar times psi-bar, Appendix).
* psi(0) and psi(+-omega_b) are set to zero (Sec. II-D: bandlimit / negligible DC).
* PHAT with a silent bin: psi = 0 when |y_m|^2 or |y_m'|^2 < 1e-30.
* SSPI keeps the Q_Lambda entries of largest magnitude; magnitudes are compared
  after quantisation to multiples of 2^-40 and ties are broken by ascending
  (location i, pair p, lag n).
* Rounding to nearest (conv. TD-SRP) rounds halves away from zero.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

__all__ = [
    "mic_pairs", "tdoa_nf", "tdoa_ff", "analysis_window", "stft", "gcc_phat",
    "steering_matrix_H", "srp_conv", "dsb_srp_map", "n_p_samples", "mean_samples",
    "pair_lags", "sampling_matrix_S", "two_sided", "gcc_samples_direct",
    "gcc_samples_ifft", "sinc", "dirichlet", "interp_matrix", "srp_si", "slri_factors",
    "srp_slri", "sspi_select", "sspi_matrix", "srp_sspi", "td_matrix", "srp_td",
    "lr_factors", "srp_lr", "argmax_map", "srp_peaks", "eps_db", "rel_err",
    "complexity", "lags_to_ascending", "SPARSE_KEY_SCALE",
]

SPARSE_KEY_SCALE = 2.0 ** 40


# ------------------------------------------------------------------------------
# Sec. II-A: pairs and TDOAs
# ------------------------------------------------------------------------------
def mic_pairs(M: int):
    """Pair index p -> (m, m'), m > m', in the order of the double sum of Eq. (SRP_omegaT):
    m' outer ascending, m = m'+1..M inner ascending.  P = M(M-1)/2 (Sec. II-A)."""
    return [(m, mp) for mp in range(M - 1) for m in range(mp + 1, M)]


def tdoa_nf(mic_xyz, grid_xyz, c=340.0):
    """Eq. (Deltat_i), near field: Delta t_p(i) = (||r_m - q_i|| - ||r_m' - q_i||)/c.
    Returns seconds, [J][P]."""
    mic_xyz = np.asarray(mic_xyz, float)
    grid_xyz = np.asarray(grid_xyz, float)
    pairs = mic_pairs(len(mic_xyz))
    out = np.empty((grid_xyz.shape[0], len(pairs)))
    dist = np.sqrt(((grid_xyz[:, None, :] - mic_xyz[None, :, :]) ** 2).sum(axis=2))  # [J][M]
    for p, (m, mp) in enumerate(pairs):
        out[:, p] = (dist[:, m] - dist[:, mp]) / c
    return out


def tdoa_ff(mic_xyz, dirs, c=340.0):
    """Eq. (Deltat_i), far field: Delta t_p(i) = (r_m - r_m')^T q_i / c, q_i unit vectors."""
    pairs = mic_pairs(len(mic_xyz))
    out = np.empty((dirs.shape[0], len(pairs)))
    for p, (m, mp) in enumerate(pairs):
        out[:, p] = dirs @ (mic_xyz[m] - mic_xyz[mp]) / c
    return out


# ------------------------------------------------------------------------------
# Sec. II-A / II-D: STFT, FD GCC with PHAT
# ------------------------------------------------------------------------------
def analysis_window(N: int, kind: str = "hann"):
    """Periodic Hann, square-root periodic Hann (the paper's STFT window, Sec. V-B) or
    rectangular."""
    n = np.arange(N)
    hann = 0.5 - 0.5 * np.cos(2.0 * np.pi * n / N)
    if kind == "hann":
        return hann
    if kind == "sqrt-hann":
        return np.sqrt(hann)
    if kind == "rect":
        return np.ones(N)
    raise ValueError(kind)


def stft(frames, window="hann"):
    """y_m(omega_k) of each frame: DFT of length 2K = N of the windowed frame,
    Y[f][m][k] = sum_n w[n] x_m[n] exp(-j 2 pi k n / N), k = 0..K (numpy rfft)."""
    frames = np.asarray(frames, dtype=np.float64)
    w = analysis_window(frames.shape[-1], window)
    return np.fft.rfft(frames * w, axis=-1)


def gcc_phat(Y, tiny=1e-30):
    """Eq. (corrmatrix) with the PHAT weight gamma = 1/|y_m y_m'^*|:
    psi_p(omega_k) = gamma y_m(omega_k) y_m'(omega_k)^*, for k = 1..K-1 (Eq. psi_p_single).
    Y: [F][M][K+1].  Returns psi [F][P][K-1] complex128."""
    F, M, K1 = Y.shape
    K = K1 - 1
    pairs = mic_pairs(M)
    psi = np.zeros((F, len(pairs), K - 1), dtype=np.complex128)
    y = Y[:, :, 1:K]
    silent = (np.abs(y) ** 2) < tiny
    for p, (m, mp) in enumerate(pairs):
        prod = y[:, m] * np.conj(y[:, mp])
        mag = np.abs(prod)
        ok = ~(silent[:, m] | silent[:, mp])
        psi[:, p][ok] = prod[ok] / mag[ok]
    return psi


# ------------------------------------------------------------------------------
# Sec. II-B..D: conventional FD-SRP
# ------------------------------------------------------------------------------
def _omega(K, fs):
    """Eq. (w_0), (w_k): omega_k = k omega_b / K with omega_b = pi / T, k = 1..K-1."""
    return np.arange(1, K) * (np.pi * fs) / K


def steering_matrix_H(dt, fs, K):
    """Eq. (H_p_single)-(H_single): [H_p]_{i,k} = exp(j omega_k Delta t_p(i)).
    Returns [J][P][K-1] complex128."""
    w = _omega(K, fs)
    return np.exp(1j * dt[:, :, None] * w[None, None, :])


def srp_conv(psi, dt, fs, chunk=None):
    """Boxed Eq. (z_computed): z = 2 Re[H psi], for each frame.
    psi: [F][P][K-1]; dt: [J][P] seconds.  Returns z [F][J] float64.  H is built in
    row blocks of ``chunk`` locations to bound memory."""
    F, P, Km1 = psi.shape
    K = Km1 + 1
    J = dt.shape[0]
    if chunk is None:
        chunk = max(1, int(2e7 // (P * Km1)))
    z = np.empty((F, J))
    psi_flat = psi.reshape(F, P * Km1)
    for j0 in range(0, J, chunk):
        H = steering_matrix_H(dt[j0:j0 + chunk], fs, K).reshape(-1, P * Km1)
        z[:, j0:j0 + chunk] = 2.0 * np.real(psi_flat @ H.T)
    return z


def dsb_srp_map(Y, mic_xyz, grid_xyz, fs, c=340.0, tiny=1e-30):
    """First line of Eq. (SRP_omegaT) summed over the bins k = 1..K-1: the delay-and-sum
    output power h^H Psi h - tr[Psi] with the steering vector of Eq. (h_steering),
    [h]_m = exp(-j omega Delta t_{m,1}(i)), and the PHAT-weighted GCC matrix of
    Eq. (corrmatrix) built as a full M x M matrix.  Brute force, for small cases.
    Y: [F][M][K+1].  Returns [F][J]."""
    F, M, K1 = Y.shape
    K = K1 - 1
    w = _omega(K, fs)
    dist = np.sqrt(((grid_xyz[:, None, :] - mic_xyz[None, :, :]) ** 2).sum(axis=2))  # [J][M]
    dt_m1 = (dist - dist[:, :1]) / c  # Delta t_{m,1}(i), [J][M]
    out = np.zeros((F, grid_xyz.shape[0]))
    for f in range(F):
        for ki, k in enumerate(range(1, K)):
            y = Y[f, :, k]
            Psi = np.outer(y, np.conj(y))
            mag = np.abs(Psi)
            silent = (np.abs(y) ** 2) < tiny
            bad = silent[:, None] | silent[None, :]
            Psi = np.where(bad, 0.0, Psi / np.where(bad, 1.0, mag))
            h = np.exp(-1j * w[ki] * dt_m1)  # [J][M]
            quad = np.einsum("jm,mn,jn->j", np.conj(h), Psi, h)
            out[f] += np.real(quad) - np.real(np.trace(Psi))
    return out


# ------------------------------------------------------------------------------
# Sec. III-B: sampling
# ------------------------------------------------------------------------------
def n_p_samples(mic_xyz, fs, c=340.0, n_aux=2):
    """Eq. (N_p): N_p = floor(Delta t_{p|0} / T) + N_aux with Delta t_{p|0} = d_p / c."""
    out = []
    for (m, mp) in mic_pairs(len(mic_xyz)):
        d = float(np.linalg.norm(np.asarray(mic_xyz[m], float) - np.asarray(mic_xyz[mp], float)))
        out.append(int(math.floor(d / c * fs)) + n_aux)
    return np.array(out, dtype=np.int64)


def mean_samples(Np):
    """Eq. (N): N = 1 + (2/P) sum_p N_p."""
    return 1.0 + 2.0 * float(np.sum(Np)) / len(Np)


def pair_lags(Np):
    """For each pair the lags n in {-N_p..N_p} listed in the order of the row/column
    index n_mod = mod[n, 2N_p+1] (Eq. nmod): 0, 1, .., N_p, -N_p, .., -1."""
    out = []
    for N_p in Np:
        n = np.arange(-N_p, N_p + 1)
        order = np.argsort(np.mod(n, 2 * N_p + 1), kind="stable")
        out.append(n[order])
    return out


def lags_to_ascending(lags):
    """Permutation that reorders the stacked n_mod-ordered sample vector into pair-major,
    ascending-lag order (a relabelling of Eq. (xi_single); Lambda xi is unchanged)."""
    perm, off = [], 0
    for n in lags:
        perm.extend((off + np.argsort(n, kind="stable")).tolist())
        off += len(n)
    return np.array(perm, dtype=np.int64)


def sampling_matrix_S(n_lags, K):
    """Eq. (S_p_single): [S_p]_{n_mod,k} = exp(j pi k n / K), k = 1..K-1."""
    k = np.arange(1, K)
    return np.exp(1j * np.pi * np.outer(np.asarray(n_lags, float), k) / K)


def two_sided(psi_p, K):
    """Appendix Eq. (psi_p_two): the 2K-vector psi-bar with [psi-bar]_{mod[k,2K]} =
    psi(omega_k) for k = -K+1..K, using psi(omega_{-k}) = psi(omega_k)^* (complex
    symmetry) and psi(0) = psi(omega_K) = 0.  psi_p: [..][K-1]."""
    shape = psi_p.shape[:-1] + (2 * K,)
    out = np.zeros(shape, dtype=np.complex128)
    out[..., 1:K] = psi_p
    out[..., K + 1:] = np.conj(psi_p[..., ::-1])  # k = -K+1..-1  <->  index 2K+k
    return out


def gcc_samples_direct(psi, lags, K):
    """Eq. (xi_computed): xi_p = 2 Re[S_p psi_p], i.e. the TD GCC of Eq. (xi_p_discreteFreq)
    at tau = nT.  psi: [F][P][K-1]; lags: per pair the n values (any order).
    Returns [F][L] with pairs stacked (Eq. xi_single)."""
    cols = []
    for p, n in enumerate(lags):
        S = sampling_matrix_S(n, K)
        cols.append(2.0 * np.real(psi[:, p, :] @ S.T))
    return np.concatenate(cols, axis=1)


def gcc_samples_ifft(psi, lags, K):
    """Eq. (xi_p_ifft)-(n_prime): xi-bar_p = iFFT[psi-bar_p] (unnormalised, length 2K), then
    [xi_p]_{n_mod} = [xi-bar_p]_{n'_mod} with n'_mod = mod[n, 2K].  Returns [F][L]
    (real part; the imaginary part is returned separately for the symmetry check)."""
    re, im = [], []
    for p, n in enumerate(lags):
        xb = np.fft.ifft(two_sided(psi[:, p, :], K), axis=-1) * (2 * K)
        sel = xb[:, np.mod(np.asarray(n), 2 * K)]
        re.append(np.real(sel))
        im.append(np.imag(sel))
    return np.concatenate(re, axis=1), np.concatenate(im, axis=1)


# ------------------------------------------------------------------------------
# Sec. III-B: interpolation, SI-SRP
# ------------------------------------------------------------------------------
def sinc(x):
    """Normalised sinc, sin(pi x)/(pi x) with sinc(0) = 1 (Eq. SRPinterp)."""
    return np.sinc(x)


def dirichlet(x, K):
    """2K-periodic interpolation kernel D(x) = (1/2K) sum_{k=-K+1}^{K-1} exp(j pi k x / K)
    (written as its sum).  With all 2K samples per pair it makes the interpolation of
    Eq. (SRPapprox) exact for the band-limited TD GCC of Eq. (xi_p_discreteFreq); it is a
    test-only kernel that ties SI-SRP to conv. FD-SRP."""
    k = np.arange(-K + 1, K)
    x = np.asarray(x, float)
    return np.real(np.exp(1j * np.pi * x[..., None] * k / K).sum(axis=-1)) / (2 * K)


def interp_matrix(dt, fs, lags, kernel="sinc", K=None):
    """Eq. (Lambda_p)-(Lambda): [Lambda_p]_{i,n_mod} = sinc(Delta t_p(i)/T - n), stacked over
    pairs.  dt: [J][P] seconds; lags: per pair the n values in the column order wanted.
    Returns [J][L] float64."""
    blocks = []
    for p, n in enumerate(lags):
        x = dt[:, p:p + 1] * fs - np.asarray(n, float)[None, :]
        blocks.append(sinc(x) if kernel == "sinc" else dirichlet(x, K))
    return np.concatenate(blocks, axis=1)


def srp_si(Lam, xi):
    """Boxed Eq. (z_circ_computed): z_si = Lambda xi.  xi: [F][L] -> [F][J]."""
    return xi @ Lam.T


# ------------------------------------------------------------------------------
# Sec. IV-A: low-rank and sparse interpolation
# ------------------------------------------------------------------------------
def slri_factors(Lam, R):
    """Eq. (min_Lambda_lr)-(Lambda_lr): the best rank-R approximation of Lambda from its SVD
    (Eckart-Young), split as Lambda_tall = U_R Sigma_R, Lambda_fat = V_R^T (Sec. III-A.1's
    "for instance" split).  Returns (tall [J][R], fat [R][L], all singular values)."""
    U, s, Vt = scipy.linalg.svd(Lam, full_matrices=False)
    return U[:, :R] * s[:R], Vt[:R], s


def srp_slri(tall, fat, xi):
    """Boxed Eq. (z_circlr_computed): z_slri = Lambda_tall (Lambda_fat xi)."""
    u = xi @ fat.T
    return u @ tall.T


def _sparse_keys(Lam):
    return np.floor(np.abs(Lam) * SPARSE_KEY_SCALE + 0.5).astype(np.int64)


def sspi_select(Lam, lags, Q_Lambda):
    """Eq. (min_Lambda_sp): keep the Q_Lambda entries of largest magnitude (Sec. IV-A).
    Equivalent to sorting all J*L entries by (quantised magnitude desc, i, p, n asc) and
    keeping the first Q_Lambda.  Returns (boolean mask [J][L], number of entries tied with
    the smallest kept key, number of those kept)."""
    J, L = Lam.shape
    keys = _sparse_keys(Lam).ravel()
    if Q_Lambda >= keys.size:
        return np.ones((J, L), bool), 0, 0
    if Q_Lambda <= 0:
        return np.zeros((J, L), bool), 0, 0
    kth = np.partition(keys, keys.size - Q_Lambda)[keys.size - Q_Lambda]
    mask = keys > kth
    need = Q_Lambda - int(mask.sum())
    tied = np.flatnonzero(keys == kth)
    # tie-break by (i, p, n) ascending
    col_p = np.concatenate([np.full(len(n), p) for p, n in enumerate(lags)])
    col_n = np.concatenate([np.asarray(n) for n in lags])
    ti, tc = np.divmod(tied, L)
    order = np.lexsort((col_n[tc], col_p[tc], ti))
    mask[tied[order[:need]]] = True
    return mask.reshape(J, L), int(tied.size), int(need)


def sspi_matrix(Lam, lags, Q_Lambda):
    """Lambda_sp: Lambda with all but the kept entries set to zero (Sec. IV-A)."""
    mask, _, _ = sspi_select(Lam, lags, Q_Lambda)
    return np.where(mask, Lam, 0.0)


def srp_sspi(Lsp, xi):
    """Boxed Eq. (z_circsp_computed): z_sspi = Lambda_sp xi."""
    return xi @ Lsp.T


def td_matrix(dt, fs, lags):
    """Sec. III-B.2 remark: conv. TD-SRP as the interpolation matrix with
    [Lambda_p]_{i,n_mod} = 1 if round(Delta t_p(i)/T) = n, else 0 (Eq. TD_SRP)."""
    blocks = []
    for p, n in enumerate(lags):
        x = dt[:, p] * fs
        r = np.sign(x) * np.floor(np.abs(x) + 0.5)
        blocks.append((r[:, None] == np.asarray(n, float)[None, :]).astype(np.float64))
    return np.concatenate(blocks, axis=1)


def srp_td(dt, fs, xi_fn):
    """Boxed Eq. (TD_SRP): z_td(i) = sum_p xi_p(round(Delta t_p(i)/T) T); xi_fn(p, n) gives
    [F] samples of pair p at integer lags n (array)."""
    J, P = dt.shape
    out = None
    for p in range(P):
        x = dt[:, p] * fs
        r = (np.sign(x) * np.floor(np.abs(x) + 0.5)).astype(np.int64)
        v = xi_fn(p, r)  # [F][J]
        out = v if out is None else out + v
    return out


def lr_factors(H2d, R_H):
    """Eq. (min_lr)-(H_lr): best rank-R_H approximation of the complex SRP matrix (LR-SRP,
    Sec. III-A), H_tall = U Sigma, H_fat = V^H."""
    U, s, Vh = scipy.linalg.svd(H2d, full_matrices=False)
    return U[:, :R_H] * s[:R_H], Vh[:R_H]


def srp_lr(H_tall, H_fat, psi_flat):
    """Boxed Eq. (z_lr): z_lr = 2 Re[H_tall H_fat psi]."""
    return 2.0 * np.real((psi_flat @ H_fat.T) @ H_tall.T)


# ------------------------------------------------------------------------------
# Sec. II-B, V-A: estimate and measures
# ------------------------------------------------------------------------------
def argmax_map(z):
    """Eq. (imax): i_max = argmax_i z(i); the lowest index wins a tie."""
    return np.argmax(z, axis=-1)


def srp_peaks(z, grid_xyz, K, d_min):
    """Several source estimates from one map: Eq. (imax) taken K times, each time over the
    candidate locations not yet excluded, where a pick excludes itself and every location
    closer than d_min metres to it (the peak picking behind Eq. (qshat), extended to
    several sources).  The lowest index wins a tie.  The exclusion test takes the
    distance in FP32, as the GPU does: with the coordinates rounded to FP32, the squared
    distance is ((dx*dx + dy*dy) + dz*dz), every operation rounded to FP32, and a location
    is excluded when that is below d_min^2 rounded to FP32.  z: [F][J] (or [J]).
    Returns (indices int64 [F][K], values [F][K]); -1 and NaN where no location is left."""
    z = np.atleast_2d(np.asarray(z))
    F, J = z.shape
    q = np.asarray(grid_xyz, float).astype(np.float32)
    t = np.float32(float(d_min) * float(d_min))
    idx = np.full((F, K), -1, dtype=np.int64)
    val = np.full((F, K), np.nan)
    for f in range(F):
        allowed = np.ones(J, bool)
        for k in range(K):
            if not allowed.any():
                break
            i = int(np.argmax(np.where(allowed, z[f], -np.inf)))
            if not allowed[i]:  # every allowed value is -inf
                i = int(np.flatnonzero(allowed)[0])
            idx[f, k] = i
            val[f, k] = z[f, i]
            d = q - q[i]
            d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
            allowed &= d2 >= t
            allowed[i] = False
    return idx, val


def eps_db(approx, ref, axis=None):
    """Sec. V-A: 10 log10(||approx - ref||^2 / ||ref||^2) dB (eps_z for maps, eps_H for
    matrices)."""
    num = np.sum(np.abs(approx - ref) ** 2, axis=axis)
    den = np.sum(np.abs(ref) ** 2, axis=axis)
    return 10.0 * np.log10(num / den)


def rel_err(approx, ref, axis=-1):
    """sqrt(||approx - ref||^2 / ||ref||^2) along an axis (per frame for maps)."""
    num = np.sum((np.asarray(approx, float) - ref) ** 2, axis=axis)
    den = np.sum(np.asarray(ref, float) ** 2, axis=axis)
    return np.sqrt(num / den)


def complexity(J, P, K, N_mean=None, R=None, Q_Lambda=None, R_H=None, sampling="ifft"):
    """Real-MAC counts of Sec. II-E, III-A.2, III-B.3 and IV-B:
    C = 2JP(K-1) (Eq. SRPomp); C_samp = 8PK log2(2K) by iFFT or 2PN(K-1) by S psi
    (Eq. C_sampling); C_td = JP + C_samp(iFFT) (Eq. tdSRPcomp, with the P iFFTs its text
    counts); C_lr = 2JR_H + 4R_H P(K-1) (Eq. C_lr); C_si = JPN + C_samp; C_slri = JR +
    RPN + C_samp; C_sspi = Q_Lambda + C_samp (boxed equations of Sec. IV-B)."""
    C = 2 * J * P * (K - 1)
    c_fft = 8 * P * K * math.log2(2 * K)
    out = {"C": C, "C_samp_ifft": c_fft, "C_td": J * P + c_fft}
    if N_mean is not None:
        c_mat = 2 * P * N_mean * (K - 1)
        c_samp = c_fft if sampling == "ifft" else c_mat
        out["C_samp_matrix"] = c_mat
        out["C_si"] = J * P * N_mean + c_samp
        if R is not None:
            out["C_slri"] = J * R + R * P * N_mean + c_samp
    if Q_Lambda is not None:
        out["C_sspi"] = Q_Lambda + c_fft
    if R_H is not None:
        out["C_lr"] = 2 * J * R_H + 4 * R_H * P * (K - 1)
    return out
