"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the pin it implements: identities the paper derives (delay-and-sum
power, TD-GCC form, sampling by iFFT, orthogonality of the iDFT rows), closed forms
(a source exactly on a grid point), special cases that reduce to textbook or library
routines (DFT shift theorem, full-rank SVD, full sort), the paper's printed worked
numbers (tests/golden/paper_numbers.json) and monotone behaviour the sampling theorem
implies.  A few tests plant a mistake in the oracle and check that a pin catches it.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def _small(name, F=3, sub=1, seed=None):
    w = synth.workload(name, F=F, grid_subsample=sub, seed=seed)
    Y = O.stft(w["frames"], "hann")
    psi = O.gcc_phat(Y)
    dt = O.tdoa_nf(w["mic_xyz"], w["grid_xyz"], 340.0)
    return w, Y, psi, dt


@pytest.fixture(scope="module")
def sq():
    return _small("square4", F=4, sub=7)


@pytest.fixture(scope="module")
def uca():
    return _small("uca8", F=3, sub=211)


# ---------------------------------------------------------------- Sec. II-A
def test_pair_order_and_count():
    pairs = O.mic_pairs(4)
    assert pairs == [(1, 0), (2, 0), (3, 0), (2, 1), (3, 1), (3, 2)]
    for M in range(2, 12):
        assert len(O.mic_pairs(M)) == M * (M - 1) // 2


def test_tdoa_range_and_colinear_limit():
    """Eq. (Deltat_i_range): |Delta t_p(i)| <= d_p / c, with equality on the pair's line."""
    mics = synth.mics_uca(6, 0.2, (1.0, 1.0, 1.0))
    g = synth.rng(7)
    grid = g.uniform(-3, 3, (500, 3))
    dt = O.tdoa_nf(mics, grid)
    for p, (m, mp) in enumerate(O.mic_pairs(6)):
        d = np.linalg.norm(mics[m] - mics[mp])
        assert np.all(np.abs(dt[:, p]) <= d / 340.0 * (1 + 1e-12))
    # a point beyond mic 0 on the line through mics 1 -> 0: Delta t_{1,0} = +d/c
    q = mics[0] + 2.0 * (mics[0] - mics[1])
    dt1 = O.tdoa_nf(mics, q[None, :])
    d10 = np.linalg.norm(mics[1] - mics[0])
    assert abs(dt1[0, 0] - d10 / 340.0) < 1e-15


def test_tdoa_ff_is_nf_limit():
    """Eq. (Deltat_i): the FF TDOA is the limit of the NF TDOA for a far source."""
    mics = synth.mics_uca(4, 0.1, (0.0, 0.0, 0.0))
    dirs = synth.grid_ff_halfsphere(30.0)
    far = O.tdoa_nf(mics, 1e7 * dirs)
    ff = O.tdoa_ff(mics, dirs)
    # far-field sign: ||r_m - q|| - ||r_m' - q|| -> -(r_m - r_m')^T q / |q|
    assert np.allclose(far, -ff, atol=1e-9)


def test_stft_shift_theorem():
    """The DFT of a circularly delayed frame carries exp(-j 2 pi k tau / N) (textbook)."""
    g = synth.rng(3)
    tau = np.array([0.0, 1.25, -3.5, 7.125])
    f32, f64 = synth.circular_delay_frames(g, tau, 256, 2)
    Y = O.stft(f64, "rect")
    k = np.arange(129)
    for m in range(1, 4):
        expect = np.exp(-2j * np.pi * k[1:128] * (tau[m] - tau[0]) / 256)
        got = Y[:, m, 1:128] / Y[:, 0, 1:128]
        assert np.max(np.abs(got - expect)) < 1e-10


def test_hann_window_closed_form():
    """Reading 4 (periodic Hann): the N-point DFT of 0.5 - 0.5 cos(2 pi n / N) is N/2 at
    k = 0, -N/4 at k = +-1 and zero elsewhere, so the windowed DFT is the three-tap
    modulation 0.5 X[k] - 0.25 X[k-1] - 0.25 X[k+1] of the plain DFT X (numpy's full FFT,
    a library routine).  The square-root Hann window squares to the Hann window."""
    for N in (256, 512, 1024):
        Wk = np.fft.fft(O.analysis_window(N, "hann"))
        expect = np.zeros(N, dtype=np.complex128)
        expect[0], expect[1], expect[-1] = N / 2, -N / 4, -N / 4
        assert np.max(np.abs(Wk - expect)) <= 1e-10 * N
        sq = O.analysis_window(N, "sqrt-hann")
        assert np.all(sq >= 0) and np.allclose(sq ** 2, O.analysis_window(N, "hann"), atol=1e-15)
    x = synth.rng(17).standard_normal((2, 3, 512))
    X = np.fft.fft(x, axis=-1)
    Y = O.stft(x, "hann")
    k = np.arange(257)
    mod = 0.5 * X[..., k] - 0.25 * X[..., (k - 1) % 512] - 0.25 * X[..., (k + 1) % 512]
    assert np.max(np.abs(Y - mod)) <= 1e-12 * np.max(np.abs(X))


# ---------------------------------------------------------------- P1: DSB identity
@pytest.mark.parametrize("case", ["sq", "uca"])
def test_P1_conv_equals_delay_and_sum_power(case, request):
    """Eq. (SRP_omegaT): 2 sum_p Re[psi_p e^{j w dt_p}] = h^H Psi h - tr Psi for every bin."""
    w, Y, psi, dt = request.getfixturevalue(case)
    z = O.srp_conv(psi, dt, w["fs"])
    zd = O.dsb_srp_map(Y, w["mic_xyz"], w["grid_xyz"], w["fs"])
    assert np.max(np.abs(z - zd)) <= 1e-11 * np.max(np.abs(zd))


def test_P1_silent_channel():
    """PHAT of an all-zero channel: its pairs contribute nothing (reading G5), and the
    identity still holds with tr Psi counting only the live channels."""
    w, _, _, _ = _small("square4", F=2, sub=25)
    fr = w["frames"].copy()
    fr[:, 2, :] = 0.0
    Y = O.stft(fr, "hann")
    psi = O.gcc_phat(Y)
    assert np.all(psi[:, [1, 3, 5], :] == 0)  # pairs (2,0), (2,1), (3,2)
    dt = O.tdoa_nf(w["mic_xyz"], w["grid_xyz"])
    z = O.srp_conv(psi, dt, w["fs"])
    zd = O.dsb_srp_map(Y, w["mic_xyz"], w["grid_xyz"], w["fs"])
    assert np.max(np.abs(z - zd)) <= 1e-11 * np.max(np.abs(zd))


def test_P1_planted_sign_flip_is_caught(monkeypatch, sq):
    """Plant a mistake (conjugated steering) in the oracle: P1 must fail."""
    w, Y, psi, dt = sq
    orig = O.srp.steering_matrix_H
    monkeypatch.setattr(O.srp, "steering_matrix_H", lambda d, fs, K: np.conj(orig(d, fs, K)))
    z = O.srp.srp_conv(psi, dt, w["fs"])
    zd = O.dsb_srp_map(Y, w["mic_xyz"], w["grid_xyz"], w["fs"])
    assert np.max(np.abs(z - zd)) > 1e-3 * np.max(np.abs(zd))


# ---------------------------------------------------------------- P2: closed form
def test_P2_source_on_grid_point_is_the_exact_peak():
    """With psi_p(w_k) = exp(-j w_k dt_p(s)) exactly, z(s) = 2P(K-1) and z(i) <= z(s)."""
    mics = synth.mics_square()
    grid = synth.grid_plane((1.0, 1.0), (3.0, 3.0), (12, 12))
    s = 77
    fs, N = 16000.0, 256
    d = np.linalg.norm(mics - grid[s], axis=1)
    tau = d / 340.0 * fs
    _, f64 = synth.circular_delay_frames(synth.rng(11), tau, N, 3)
    psi = O.gcc_phat(O.stft(f64, "rect"))
    dt = O.tdoa_nf(mics, grid)
    z = O.srp_conv(psi, dt, fs)
    P, K = 6, N // 2
    assert np.allclose(z[:, s], 2 * P * (K - 1), rtol=1e-12)
    assert np.all(z <= 2 * P * (K - 1) * (1 + 1e-12))
    assert np.all(O.argmax_map(z) == s)


@pytest.mark.parametrize("window", ["hann", "sqrt-hann"])
def test_P2_windowed_free_field_source_on_a_grid_point_is_the_argmax(window):
    """Time-domain variant of P2: a white source exactly on a grid point, propagated in free
    field (band-limited fractional delays, 1/r gain, no noise), framed with a Hann or
    square-root Hann window.  The PHAT maps of conv. FD-SRP, SI-SRP and full-rank SLRI-SRP
    all peak at that grid point in every frame (Sec. II-B: the true location maximises the
    delay-and-sum power)."""
    mics = synth.mics_square()
    grid = synth.grid_plane((1.0, 1.0), (3.0, 3.0), (9, 9))
    s = 58
    fs, N, hop, F = 16000.0, 512, 256, 6
    sig = synth.white(synth.rng(31), (F - 1) * hop + N + 64)
    x = synth.propagate([(sig, grid[s])], fs, mics, (F - 1) * hop + N)
    frames = synth.cut_frames(x, N, hop, F).astype(np.float64)
    psi = O.gcc_phat(O.stft(frames, window))
    dt = O.tdoa_nf(mics, grid)
    K = N // 2
    z = O.srp_conv(psi, dt, fs)
    lags = O.pair_lags(O.n_p_samples(mics, fs))
    xi = O.gcc_samples_direct(psi, lags, K)
    Lam = O.interp_matrix(dt, fs, lags)
    tall, fat, _ = O.slri_factors(Lam, min(Lam.shape))
    for zz in (z, O.srp_si(Lam, xi), O.srp_slri(tall, fat, xi)):
        assert np.all(O.argmax_map(zz) == s)
    # under PHAT z <= 2P(K-1) everywhere; the true point comes close to it (the delays are
    # exact and there is no noise), and it beats the runner-up (a neighbouring cell)
    P = len(O.mic_pairs(len(mics)))
    assert np.all(z <= 2 * P * (K - 1) * (1 + 1e-12))
    assert np.all(z[:, s] >= 0.98 * 2 * P * (K - 1))
    top2 = np.sort(z, axis=1)[:, -2:]
    assert np.all(top2[:, 1] - top2[:, 0] > 0.005 * top2[:, 1])


# ---------------------------------------------------------------- P3/P4: sampling
def test_P3_samples_direct_equal_ifft_selection(sq):
    """Eq. (xi_computed) = Eq. (xi_p_ifft)-(n_prime): 2 Re[S_p psi_p] equals the
    unnormalised 2K-iFFT of psi-bar at n'_mod = mod[n, 2K]."""
    w, Y, psi, dt = sq
    K = w["N"] // 2
    Np = O.n_p_samples(w["mic_xyz"], w["fs"])
    lags = O.pair_lags(Np)
    a = O.gcc_samples_direct(psi, lags, K)
    b, _ = O.gcc_samples_ifft(psi, lags, K)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_P3_integer_lag_equals_conv_pair_term(sq):
    """Eq. (SRP_T_IFT) at an integer TDOA n: 2 Re[H_p psi_p]_i = xi_p(nT), and the sinc row
    of Lambda_p is one-hot there (Sec. III-B.2)."""
    w, Y, psi, _ = sq
    fs, K = w["fs"], w["N"] // 2
    n_int = np.array([-3, -1, 0, 2, 5])
    dt = np.repeat((n_int / fs)[:, None], psi.shape[1], axis=1)  # J=5 locations, every pair
    Np = np.full(psi.shape[1], 6)
    lags = O.pair_lags(Np)
    xi = O.gcc_samples_direct(psi, lags, K)
    Lam = O.interp_matrix(dt, fs, lags)
    assert np.all((np.abs(Lam) < 1e-15) | (np.abs(Lam - 1) < 1e-15))
    for p in range(psi.shape[1]):
        single = psi.copy()
        single[:, [q for q in range(psi.shape[1]) if q != p]] = 0
        zc = O.srp_conv(single, dt, fs)
        off = sum(len(l) for l in lags[:p])
        col = [off + list(lags[p]).index(n) for n in n_int]
        assert np.allclose(zc, xi[:, col], rtol=0, atol=1e-10 * np.max(np.abs(xi)))
        blk = slice(off, off + len(lags[p]))  # SI-SRP of this pair alone picks the same sample
        assert np.allclose(O.srp_si(Lam[:, blk], xi[:, blk]), zc, rtol=0,
                           atol=1e-10 * np.max(np.abs(xi)))


def test_P4_hermitian_symmetry(uca):
    """psi-bar[2K-k] = psi-bar[k]^* makes the iFFT real (Appendix)."""
    w, Y, psi, _ = uca
    K = w["N"] // 2
    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"]))
    re, im = O.gcc_samples_ifft(psi, lags, K)
    assert np.max(np.abs(im)) <= 1e-13 * np.linalg.norm(re)
    pb = O.two_sided(psi[0, 0], K)
    assert pb[0] == 0 and pb[K] == 0
    assert np.allclose(pb[2 * K - np.arange(1, K)], np.conj(pb[1:K]))


def test_P3_planted_missing_conjugate_is_caught(monkeypatch, sq):
    w, Y, psi, _ = sq
    K = w["N"] // 2

    def bad_two_sided(psi_p, K):
        out = np.zeros(psi_p.shape[:-1] + (2 * K,), dtype=np.complex128)
        out[..., 1:K] = psi_p
        out[..., K + 1:] = psi_p[..., ::-1]  # conjugate dropped
        return out

    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"]))
    a = O.gcc_samples_direct(psi, lags, K)
    monkeypatch.setattr(O.srp, "two_sided", bad_two_sided)
    b, _ = O.srp.gcc_samples_ifft(psi, lags, K)
    assert np.max(np.abs(a - b)) > 1e-3 * np.max(np.abs(a))


def test_lag_order_is_nmod():
    """Eq. (nmod): n_mod = mod[n, 2N_p+1] lists 0..N_p then -N_p..-1."""
    assert list(O.pair_lags([2])[0]) == [0, 1, 2, -2, -1]
    lags = O.pair_lags([1, 2])
    perm = O.lags_to_ascending(lags)
    stacked = np.concatenate(lags)
    assert list(stacked[perm]) == [-1, 0, 1, -2, -1, 0, 1, 2]


# ---------------------------------------------------------------- P5: limits
def test_P5_full_rank_and_full_support_reproduce_si(uca):
    w, Y, psi, dt = uca
    K = w["N"] // 2
    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"]))
    xi = O.gcc_samples_direct(psi, lags, K)
    Lam = O.interp_matrix(dt, w["fs"], lags)
    z_si = O.srp_si(Lam, xi)
    R = min(Lam.shape)
    tall, fat, _ = O.slri_factors(Lam, R)
    z_lr = O.srp_slri(tall, fat, xi)
    assert np.max(np.abs(z_lr - z_si)) <= 1e-10 * np.max(np.abs(z_si))
    Lsp = O.sspi_matrix(Lam, lags, Lam.size)
    assert np.array_equal(O.srp_sspi(Lsp, xi), z_si)


def test_P5_exact_kernel_si_equals_conv(sq):
    """With all 2K samples per pair and the 2K-periodic kernel, Lambda S = H exactly, so
    SI-SRP, full-rank SLRI and full-support SSPI all reproduce conv. FD-SRP (Eq. H_circ)."""
    w, Y, psi, dt = sq
    K = w["N"] // 2
    lags = [np.arange(-K + 1, K + 1)] * psi.shape[1]
    xi = O.gcc_samples_direct(psi, lags, K)
    Lam = O.interp_matrix(dt, w["fs"], lags, kernel="dirichlet", K=K)
    z_si = O.srp_si(Lam, xi)
    z = O.srp_conv(psi, dt, w["fs"])
    assert np.max(np.abs(z_si - z)) <= 1e-10 * np.max(np.abs(z))
    tall, fat, _ = O.slri_factors(Lam, min(Lam.shape))
    assert np.max(np.abs(O.srp_slri(tall, fat, xi) - z)) <= 1e-10 * np.max(np.abs(z))


def test_dirichlet_kernel_closed_form_and_exact_interpolation():
    """The test-only 2K-periodic kernel: its sum equals the closed form
    sin(pi (2K-1) x / 2K) / (2K sin(pi x / 2K)) (the Dirichlet kernel), and it interpolates a
    trigonometric polynomial of degree K-1 with no DC or Nyquist term (the TD GCC of
    Eq. xi_p_discreteFreq with psi(0) = psi(omega_b) = 0) exactly from its 2K integer
    samples n = -K+1..K, at any real x."""
    for K in (4, 8, 16):
        x = np.linspace(-2.3 * K, 2.3 * K, 997)
        x = x[np.abs(np.sin(np.pi * x / (2 * K))) > 1e-3]  # the closed form is 0/0 at 2K m
        closed = np.sin(np.pi * (2 * K - 1) * x / (2 * K)) / (2 * K * np.sin(np.pi * x / (2 * K)))
        assert np.max(np.abs(O.dirichlet(x, K) - closed)) <= 1e-12
        g = synth.rng(K)
        psi = g.standard_normal(K - 1) + 1j * g.standard_normal(K - 1)
        k = np.arange(1, K)

        def xi(t):
            return 2.0 * np.real(np.exp(1j * np.pi * np.outer(t, k) / K) @ psi)

        n = np.arange(-K + 1, K + 1)
        interp = O.dirichlet(x[:, None] - n[None, :], K) @ xi(n)
        assert np.max(np.abs(interp - xi(x))) <= 1e-10 * np.max(np.abs(xi(n)))


def test_td_is_one_hot_interpolation(sq):
    """Sec. III-B.2: conv. TD-SRP = SI with the one-hot Lambda at the rounded lag."""
    w, Y, psi, dt = sq
    K = w["N"] // 2
    Np = O.n_p_samples(w["mic_xyz"], w["fs"])
    lags = O.pair_lags(Np)
    xi = O.gcc_samples_direct(psi, lags, K)
    z1 = O.srp_si(O.td_matrix(dt, w["fs"], lags), xi)

    def xi_fn(p, n):
        S = O.sampling_matrix_S(n, K)
        return 2.0 * np.real(psi[:, p, :] @ S.T)

    z2 = O.srp_td(dt, w["fs"], xi_fn)
    assert np.max(np.abs(z1 - z2)) <= 1e-12 * np.max(np.abs(z2))


def test_lr_full_rank_equals_conv(sq):
    """Eq. (z_lr): with R_H = rank H, LR-SRP is conv. FD-SRP."""
    w, Y, psi, dt = sq
    K = w["N"] // 2
    H = O.steering_matrix_H(dt, w["fs"], K).reshape(dt.shape[0], -1)
    tall, fat = O.lr_factors(H, min(H.shape))
    z = O.srp_lr(tall, fat, psi.reshape(psi.shape[0], -1))
    zc = O.srp_conv(psi, dt, w["fs"])
    assert np.max(np.abs(z - zc)) <= 1e-10 * np.max(np.abs(zc))


def test_lr_rank_R_is_the_best_approximation(sq):
    """Eq. (min_lr): H_tall H_fat is the best rank-R_H approximation of the complex SRP
    matrix: it equals H W_R W_R^H with W_R the top eigenvectors of H^H H (numpy.linalg.eigh,
    another routine than the SVD the oracle calls), and its residual is the sum of the
    dropped squared singular values (Eckart-Young)."""
    w, Y, psi, dt = sq
    K = w["N"] // 2
    H = O.steering_matrix_H(dt[::5], w["fs"], K).reshape(dt[::5].shape[0], -1)
    ev, W = np.linalg.eigh(H.conj().T @ H)
    s = np.sqrt(np.clip(ev[::-1], 0, None))
    for R in (2, 7, 20):
        if s[R - 1] - s[R] < 1e-6 * s[0]:
            continue  # degenerate cut: the rank-R optimum is not unique
        tall, fat = O.lr_factors(H, R)
        WR = W[:, ::-1][:, :R]
        ref = H @ WR @ WR.conj().T
        assert np.max(np.abs(tall @ fat - ref)) <= 1e-8 * np.max(np.abs(H))
        res = np.linalg.norm(H - tall @ fat) ** 2
        assert abs(res - np.sum(s[R:] ** 2)) <= 1e-9 * np.sum(s ** 2)


# ---------------------------------------------------------------- P6: low rank
def test_P6_rank_R_matches_gram_eigenprojector(uca):
    """Eq. (min_Lambda_lr): Lambda_lr = Lambda V_R V_R^T with V_R the top eigenvectors of
    Lambda^T Lambda (a different library routine than the SVD the oracle calls), and no
    random rank-R matrix near it does better (Eckart-Young)."""
    w, Y, psi, dt = uca
    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"]))
    Lam = O.interp_matrix(dt, w["fs"], lags)
    for R in (3, 8, 16):
        tall, fat, s = O.slri_factors(Lam, R)
        if (s[R - 1] - s[R]) < 1e-6 * s[0]:
            continue  # degenerate cut: the rank-R optimum is not unique
        ev, V = np.linalg.eigh(Lam.T @ Lam)
        VR = V[:, ::-1][:, :R]
        ref = Lam @ VR @ VR.T
        assert np.max(np.abs(tall @ fat - ref)) <= 1e-8 * np.max(np.abs(Lam))
        best = np.linalg.norm(Lam - tall @ fat)
        assert abs(best ** 2 - np.sum(s[R:] ** 2)) <= 1e-10 * np.sum(s ** 2)
        g = synth.rng(R)
        for _ in range(5):
            B = (tall + 1e-3 * g.standard_normal(tall.shape)) @ (fat + 1e-3 * g.standard_normal(fat.shape))
            assert np.linalg.norm(Lam - B) >= best - 1e-12


def test_P6_rank_one_by_power_iteration(sq):
    w, Y, psi, dt = sq
    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"]))
    Lam = O.interp_matrix(dt, w["fs"], lags)
    v = np.ones(Lam.shape[1])
    for _ in range(2000):
        v = Lam.T @ (Lam @ v)
        v /= np.linalg.norm(v)
    tall, fat, s = O.slri_factors(Lam, 1)
    assert abs(np.linalg.norm(Lam @ v) - s[0]) <= 1e-10 * s[0]
    assert np.max(np.abs(tall @ fat - np.outer(Lam @ v, v))) <= 1e-8


# ---------------------------------------------------------------- P7: sparse
def test_P7_sparse_selection_matches_full_sort(sq):
    w, Y, psi, dt = sq
    lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"]))
    Lam = O.interp_matrix(dt, w["fs"], lags)
    J, L = Lam.shape
    keys = np.floor(np.abs(Lam) * 2.0 ** 40 + 0.5).astype(np.int64).ravel()
    col_p = np.concatenate([np.full(len(n), p) for p, n in enumerate(lags)])
    col_n = np.concatenate(lags)
    ii, cc = np.divmod(np.arange(J * L), L)
    full = np.lexsort((col_n[cc], col_p[cc], ii, -keys))
    for t in (0.5, 1.0, 2.0, 4.0):
        Q_L = int(round(t * J * len(lags)))
        mask, tied, taken = O.sspi_select(Lam, lags, Q_L)
        ref = np.zeros(J * L, bool)
        ref[full[:Q_L]] = True
        assert np.array_equal(mask.ravel(), ref)
        kept = np.abs(Lam[mask])
        dropped = np.abs(Lam[~mask])
        assert kept.min() >= dropped.max() - 2.0 ** -40
        Lsp = O.sspi_matrix(Lam, lags, Q_L)
        assert math.isclose(np.sum((Lam - Lsp) ** 2), np.sum(dropped ** 2), rel_tol=1e-12)


# ---------------------------------------------------------------- P8: cost simplification
def test_P8_cost_simplification():
    """Eq. (cost_simplified) and the Appendix: S-bar S-bar^H = 2K I, hence
    ||D S-bar||_F^2 = 2K ||D||_F^2 for real D; and the one-sided S drops exactly the
    omega = 0 and omega_b columns: 2 ||D S||^2 = ||D S-bar||^2 - ||D s_0||^2 - ||D s_K||^2."""
    K = 16
    Np = [3, 5]
    lags = O.pair_lags(Np)
    k2 = np.arange(-K + 1, K + 1)
    Sbar_blocks = [np.exp(1j * np.pi * np.outer(n, k2) / K) for n in lags]
    Sbar = np.zeros((sum(len(n) for n in lags), 2 * K * len(lags)), dtype=np.complex128)
    r = 0
    for p, B in enumerate(Sbar_blocks):
        Sbar[r:r + B.shape[0], p * 2 * K:(p + 1) * 2 * K] = B
        r += B.shape[0]
    assert np.allclose(Sbar @ Sbar.conj().T, 2 * K * np.eye(Sbar.shape[0]), atol=1e-12)
    g = synth.rng(5)
    D = g.standard_normal((7, Sbar.shape[0]))
    assert math.isclose(np.linalg.norm(D @ Sbar) ** 2, 2 * K * np.linalg.norm(D) ** 2, rel_tol=1e-12)
    S_one = np.zeros((Sbar.shape[0], (K - 1) * len(lags)), dtype=np.complex128)
    r = 0
    for p, n in enumerate(lags):
        S_one[r:r + len(n), p * (K - 1):(p + 1) * (K - 1)] = O.sampling_matrix_S(n, K)
        r += len(n)
    lhs = 2 * np.linalg.norm(D @ S_one) ** 2
    s0 = np.concatenate([np.ones(len(n)) for n in lags])
    sK = np.concatenate([np.cos(np.pi * n) for n in lags])
    per_pair = 0.0
    off = 0
    for n in lags:
        sl = slice(off, off + len(n))
        per_pair += np.linalg.norm(D[:, sl] @ s0[sl]) ** 2 + np.linalg.norm(D[:, sl] @ sK[sl]) ** 2
        off += len(n)
    rhs = np.linalg.norm(D @ Sbar) ** 2 - per_pair
    assert math.isclose(lhs, rhs, rel_tol=1e-12)


# ---------------------------------------------------------------- P9: worked numbers
def test_P9_paper_worked_numbers():
    G = json.load(open(GOLDEN))
    ff = G["ff_uca_mean_samples"]
    for D, want in zip(ff["diameters_m"], ff["N_mean"]):
        mics = synth.mics_uca(ff["M"], D / 2, (0, 0, 0))
        Np = O.n_p_samples(mics, ff["fs"], ff["c"], ff["n_aux"])
        assert abs(O.mean_samples(Np) - want) <= ff["print_precision"]
    assert len(synth.grid_ff_halfsphere(G["ff_grid_size"]["step_deg"])) == G["ff_grid_size"]["J"]
    t1 = G["table1_complexity"]
    for key in ("nf", "ff"):
        e = t1[key]
        C = O.complexity(e["J"], e["P"], e["K_minus_1"] + 1)["C"]
        assert abs(C / 2 - e["C_printed"]) <= t1["print_precision_rel"] * e["C_printed"]
    for key in ("nf", "ff"):
        e = G["table1_si_crel"][key]
        c = O.complexity(e["J"], e["P"], e["K"], N_mean=e["N_mean"])
        assert abs(c["C_si"] / c["C"] - e["C_rel"]) <= e["tol"]
    tf = G["timing_figure"]
    J, P, K = tf["J"], tf["P"], tf["K"]
    N_mean = 1 + 2 * tf["derived_sum_N_p"] / P
    c = O.complexity(J, P, K, N_mean=N_mean, R=tf["derived_R_Lambda"], Q_Lambda=J * P,
                     R_H=tf["derived_R_H"])
    C = c["C"]
    for key, val in (("C_samp_ifft", "C_rel_samp"), ("C_td", "C_rel_td"), ("C_lr", "C_rel_lr"),
                     ("C_si", "C_rel_si"), ("C_slri", "C_rel_slri"), ("C_sspi", "C_rel_sspi")):
        assert math.isclose(c[key] / C, tf[val], rel_tol=1e-12), key


# ---------------------------------------------------------------- estimate and measures
def test_argmax_takes_the_lowest_index_on_ties():
    """Reading of Eq. (imax) for tied maxima: the lowest location index."""
    z = np.array([[0.0, 3.0, 1.0, 3.0], [5.0, 5.0, 5.0, 5.0], [-2.0, -1.0, -1.0, -3.0]])
    assert list(O.argmax_map(z)) == [1, 0, 1]


def _line(J, h=1.0):
    return np.stack([np.arange(J) * h, np.zeros(J), np.zeros(J)], axis=1)


def test_peaks_worked_example_on_a_line():
    """Eq. (imax) repeated with exclusion, worked by hand on a line of unit spacing with
    d_min = 2: 9 at cell 1 (the lower index of the tie 1 / 3) excludes cells 0..2 (cell 3,
    exactly 2 away, stays); 9 at cell 3 excludes 2..4; 8 at cell 6 excludes 5..7; nothing
    is left for a fourth pick."""
    z = np.array([[4.0, 9.0, 1.0, 9.0, 7.0, 3.0, 8.0, 0.0]])
    idx, val = O.srp_peaks(z, _line(8), 4, 2.0)
    assert idx.tolist() == [[1, 3, 6, -1]]
    assert val[0, :3].tolist() == [9.0, 9.0, 8.0] and np.isnan(val[0, 3])
    # d_min = 1: neighbours exactly 1 away stay, so 7 at cell 4 is the fourth pick
    idx, _ = O.srp_peaks(z, _line(8), 4, 1.0)
    assert idx.tolist() == [[1, 3, 6, 4]]


def test_peaks_without_separation_are_the_sorted_map():
    """d_min = 0 excludes only the picks themselves: the K largest values in descending
    order, ties in ascending index -- a full sort (numpy lexsort)."""
    g = synth.rng(31)
    z = np.round(g.standard_normal((5, 400)), 1)  # many ties
    grid = g.uniform(0, 4, (400, 3))
    idx, val = O.srp_peaks(z, grid, 12, 0.0)
    for f in range(5):
        order = np.lexsort((np.arange(400), -z[f]))
        assert idx[f].tolist() == order[:12].tolist()
        assert np.array_equal(val[f], z[f, order[:12]])


def test_peaks_beyond_the_grid_diameter_leave_the_argmax_only():
    g = synth.rng(32)
    z = g.standard_normal((3, 200))
    grid = g.uniform(0, 2, (200, 3))
    idx, _ = O.srp_peaks(z, grid, 3, 10.0)
    assert idx[:, 0].tolist() == O.argmax_map(z).tolist()
    assert np.all(idx[:, 1:] == -1)


def test_peaks_are_separated_and_greedy_on_a_box_grid():
    """Invariants on a 3-D grid: picks are pairwise at least d_min apart, and each is the
    largest value among the cells at least d_min from every earlier pick (checked with a
    margin of 1e-6 m on both sides, away from the FP32 exclusion boundary)."""
    grid = synth.grid_box((0, 0, 0), (1.0, 0.8, 0.6), 0.1)
    g = synth.rng(33)
    z = g.standard_normal((4, grid.shape[0]))
    d_min = 0.25
    idx, val = O.srp_peaks(z, grid, 5, d_min)
    for f in range(4):
        picks = [i for i in idx[f] if i >= 0]
        assert len(picks) == 5
        for k, i in enumerate(picks):
            d_prev = [np.linalg.norm(grid - grid[j], axis=1) for j in picks[:k]]
            far = np.all([d >= d_min + 1e-6 for d in d_prev], axis=0) if k else np.ones(len(z[f]), bool)
            near = np.any([d < d_min - 1e-6 for d in d_prev], axis=0) if k else np.zeros(len(z[f]), bool)
            assert not near[i]
            assert z[f, i] >= z[f, far].max()
            assert val[f, k] == z[f, i]


def test_peaks_of_two_sources_on_grid_points_are_the_sources():
    """Closed form: with psi the mean of two exactly delayed single-source spectra, the map
    is the mean of two single-source maps, each 2P(K-1) at its source (Eq. SRPomp with
    psi_p(w_k) = exp(-j w_k dt_p(s))).  With d_min = 0.5 m the two picks are the two source
    cells, each with z >= P(K-1) - max|cross term|.  The array is not planar, so no mirror
    image of a source is an exact tie."""
    mics = synth.rng(41).uniform((1.0, 1.0, 0.4), (3.0, 3.0, 1.6), (8, 3))
    grid = synth.grid_box((0.5, 0.5, 0.5), (3.5, 3.5, 1.5), 0.25)
    fs, N = 16000.0, 256
    s1, s2 = 20, 500
    assert np.linalg.norm(grid[s1] - grid[s2]) > 1.5
    psis = []
    for s in (s1, s2):
        tau = np.linalg.norm(mics - grid[s], axis=1) / 340.0 * fs
        _, f64 = synth.circular_delay_frames(synth.rng(40 + s), tau, N, 2)
        psis.append(O.gcc_phat(O.stft(f64, "rect")))
    dt = O.tdoa_nf(mics, grid)
    z1, z2 = (O.srp_conv(p, dt, fs) for p in psis)
    z = O.srp_conv(0.5 * (psis[0] + psis[1]), dt, fs)
    assert np.allclose(z, 0.5 * (z1 + z2), rtol=0, atol=1e-9 * np.abs(z).max())
    P, K = 28, N // 2
    idx, val = O.srp_peaks(z, grid, 2, 0.5)
    for f in range(2):
        assert set(idx[f].tolist()) == {s1, s2}
        cross = max(abs(z2[f, s1]), abs(z1[f, s2])) / 2
        assert np.all(val[f] >= P * (K - 1) - cross - 1e-9)


def test_error_measures_closed_forms():
    """Sec. V-A measures on maps with a known error: a map scaled by (1 + e) is
    10 log10(e^2) dB and e relative away from the original; orthogonal errors add."""
    z = synth.rng(23).standard_normal((4, 300))
    for e in (1e-1, 1e-3, 1e-6):
        assert math.isclose(O.eps_db((1 + e) * z, z), 20.0 * math.log10(e), abs_tol=1e-6)
        assert np.allclose(O.rel_err((1 + e) * z, z), e, rtol=1e-6)
    a = np.zeros((1, 4))
    ref = np.array([[3.0, 0.0, 0.0, 0.0]])
    a[0, 0], a[0, 1] = 3.0, 4.0  # error (0, 4): ||e|| / ||ref|| = 4 / 3
    assert math.isclose(O.rel_err(a, ref)[0], 4.0 / 3.0, rel_tol=1e-15)


# ---------------------------------------------------------------- P10: truncation
def test_P10_si_error_shrinks_with_aux_samples(sq):
    """Eq. (SRPapprox)-(N_p): more auxiliary samples -> SI-SRP closer to conv. FD-SRP."""
    w, Y, psi, dt = sq
    K = w["N"] // 2
    z = O.srp_conv(psi, dt, w["fs"])
    errs = []
    for n_aux in (0, 2, 8, 32):
        lags = O.pair_lags(O.n_p_samples(w["mic_xyz"], w["fs"], n_aux=n_aux))
        xi = O.gcc_samples_direct(psi, lags, K)
        errs.append(O.eps_db(O.srp_si(O.interp_matrix(dt, w["fs"], lags), xi), z))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
