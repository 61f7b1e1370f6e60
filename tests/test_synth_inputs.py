"""The seeded input generator (synth/, shared by the oracle tests, the GPU parity tests and
the benchmark; it holds none of the method's arithmetic).  Its propagation and diffuse
noise apply exact band-limited delays as linear-phase ramps exp(-2 pi i k s / L) computed
as products of two exponentials (k = k0 + j); these tests pin that factorisation to the
direct exponential and the presets to their documented sizes and determinism."""
import numpy as np
import pytest

import synth


def test_phase_ramp_factorisation_is_the_direct_exponential():
    rng = np.random.default_rng(3)
    L = 1 << 16
    shifts = np.concatenate([rng.uniform(0.0, 1500.0, 20), [0.0, 0.5, 1.0, 1234.5678]])
    A, B, nb = synth._ramps(shifts, L)
    k = np.arange(nb)
    ramp = (A[:, None, :] * B.T[None, :, :]).reshape(-1, len(shifts))[:nb]  # [k][s]
    direct = np.exp(-2j * np.pi * np.outer(k, shifts) / L)
    assert np.abs(ramp - direct).max() < 1e-12


def test_free_field_delay_is_exact_for_an_integer_shift():
    """A path of length d = c * D / fs (D integer samples) delays by exactly D samples and
    scales by 1/d."""
    fs, c, D = 16000.0, synth.C_SOUND, 37
    g = synth.rng(5)
    s = g.standard_normal(4000)
    mic = np.zeros((1, 3))
    src = np.array([c * D / fs, 0.0, 0.0])
    x = synth.propagate([(s, src)], fs, mic, 4000)[0]
    d = c * D / fs
    assert np.allclose(x[D:], s[:4000 - D] / d, atol=1e-9)
    assert np.allclose(x[:D], 0.0, atol=1e-9)


@pytest.mark.parametrize("name,M,J,N", [("square4", 4, 2500, 512), ("uca8", 8, 60000, 512)])
def test_presets_are_seeded_and_sized(name, M, J, N):
    a = synth.workload(name, F=12)
    b = synth.workload(name, F=12)
    assert np.array_equal(a["frames"], b["frames"])
    assert a["frames"].shape == (12, M, N) and a["frames"].dtype == np.float32
    assert a["grid_xyz"].shape == (J, 3) and a["mic_xyz"].shape == (M, 3)


def test_image_sources_count_gains_and_first_order_mirrors():
    """Shoebox image method with total reflection order <= 3: per axis one image with no
    reflection and two with r >= 1 reflections, so 1 + 6 + 18 + 38 = 63 images; gains
    beta^order; the six first-order images are the mirrors in the six walls; no duplicates."""
    room = (6.0, 4.0, 3.0)
    src = np.array([1.3, 2.9, 0.7])
    imgs = synth.image_sources(src, room, 3, 0.7)
    assert len(imgs) == 63
    pos = np.array([p for p, _ in imgs])
    assert len(np.unique(np.round(pos, 9), axis=0)) == 63
    gains = sorted(round(g, 12) for _, g in imgs)
    want = [1.0] + [0.7] * 6 + [round(0.7 ** 2, 12)] * 18 + [round(0.7 ** 3, 12)] * 38
    assert gains == sorted(want)
    first = {tuple(np.round(p, 9)) for p, g in imgs if abs(g - 0.7) < 1e-12}
    mirrors = set()
    for ax in range(3):
        for wall in (0.0, room[ax]):
            m = src.copy()
            m[ax] = 2 * wall - src[ax]
            mirrors.add(tuple(np.round(m, 9)))
    assert first == mirrors
    assert any(np.allclose(p, src) and g == 1.0 for p, g in imgs)


def test_noise_is_added_at_the_requested_snr():
    g = synth.rng(9)
    x = g.standard_normal((4, 5000)) * np.array([[1.0], [0.5], [2.0], [1.5]])
    n = g.standard_normal((4, 5000))
    for snr in (10.0, 15.0, 20.0):
        y = synth.add_noise_snr(x, n, snr)
        got = 10 * np.log10(np.mean(x ** 2) / np.mean((y - x) ** 2))
        assert abs(got - snr) < 1e-9
