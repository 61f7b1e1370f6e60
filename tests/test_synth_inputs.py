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
