"""Seeded synthetic inputs for the SRP-map workloads.

This module is shared by the FP64 oracle tests, the GPU parity tests and the
benchmark.  It produces *inputs only*: microphone geometries, candidate-location
grids, source signals, their propagation to the microphones (free field or image
sources), sensor and diffuse noise, and the cut into frames.  It contains none of
the SRP method's arithmetic (no window, no STFT, no PHAT, no cross-spectra, no
TDOA table, no steering/interpolation matrix, no map).

Every generator takes an explicit ``numpy.random.Generator`` or a seed; the
workload presets use seed ``1000 + index`` with numpy's PCG64.  Speed of sound is
c = 340 m/s, as in the paper's simulation setup (Sec. V-B).

Workload presets (the sizes of the paper-derived workloads):

* ``square4``   M=4 mics on a 0.2 m square, 2-D 50x50 grid over 4x4 m (J=2500),
  N=512 Hann / hop 256, F=100, white source, 20 dB sensor noise.
* ``uca8``      M=8 uniform circular array r=5 cm, 3-D 0.1 m grid over 5x4x3 m
  (J=60000), N=512, F=2000, AR(10) speech-like source, 10 dB diffuse noise.
* ``walls16``   M=16 mics on the walls of a 6x4x3 m room, 0.1 m grid (J=72000),
  N=1024, F=4096, two sources, image sources to order 3 (beta=0.7), 15 dB.
* ``nested32``  M=32 as two nested UCAs r=4/12 cm, 0.05 m grid over 4x3x2.5 m
  (J=240000), N=2048, F=1024, one source, 20 dB.

Frames are returned as float32 ``[F][M][N]`` (frame f = samples
``[f*hop, f*hop+N)``), unwindowed.
"""
from __future__ import annotations

import numpy as np

C_SOUND = 340.0

__all__ = [
    "C_SOUND", "rng", "mics_square", "mics_uca", "mics_nested_uca", "mics_walls",
    "grid_box", "grid_plane", "grid_ff_halfsphere", "white", "ar_speech_like",
    "onoff_envelope", "propagate", "image_sources", "diffuse_noise", "add_noise_snr",
    "cut_frames", "circular_delay_frames", "workload", "WORKLOADS",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------------
def mics_square(center=(2.0, 2.0, 0.0), half=0.1) -> np.ndarray:
    """Four microphones at the corners of a square of side 2*half, in a z-plane."""
    cx, cy, cz = center
    return np.array([[cx - half, cy - half, cz], [cx + half, cy - half, cz],
                     [cx + half, cy + half, cz], [cx - half, cy + half, cz]], dtype=np.float64)


def mics_uca(M: int, radius: float, center, phase: float = 0.0) -> np.ndarray:
    """M microphones equally spaced on a horizontal circle."""
    a = phase + 2.0 * np.pi * np.arange(M) / M
    c = np.asarray(center, dtype=np.float64)
    return np.stack([c[0] + radius * np.cos(a), c[1] + radius * np.sin(a),
                     np.full(M, c[2])], axis=1)


def mics_nested_uca(M_inner: int, r_inner: float, M_outer: int, r_outer: float, center) -> np.ndarray:
    """Two coplanar, concentric horizontal UCAs (the outer one rotated by half a step)."""
    inner = mics_uca(M_inner, r_inner, center)
    outer = mics_uca(M_outer, r_outer, center, phase=np.pi / M_outer)
    return np.concatenate([inner, outer], axis=0)


def mics_walls(g: np.random.Generator, room=(6.0, 4.0, 3.0), per_wall=4,
               height=(0.5, 2.5), margin=0.5) -> np.ndarray:
    """per_wall microphones on each of the 4 side walls of a box room, seeded."""
    Lx, Ly, _ = room
    out = []
    for wall in range(4):
        for _ in range(per_wall):
            h = g.uniform(*height)
            if wall == 0:
                out.append([g.uniform(margin, Lx - margin), 0.0, h])
            elif wall == 1:
                out.append([Lx, g.uniform(margin, Ly - margin), h])
            elif wall == 2:
                out.append([g.uniform(margin, Lx - margin), Ly, h])
            else:
                out.append([0.0, g.uniform(margin, Ly - margin), h])
    return np.asarray(out, dtype=np.float64)


def grid_box(lo, hi, h) -> np.ndarray:
    """Cell centres of a regular grid of pitch h over the box [lo, hi] (x fastest-varying last).

    Returns [J][3] with J = prod(round((hi-lo)/h)); index i = (ix*ny + iy)*nz + iz.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = np.rint((hi - lo) / h).astype(int)
    axes = [lo[d] + (np.arange(n[d]) + 0.5) * h for d in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def grid_plane(lo_xy, hi_xy, n_xy, z=0.0) -> np.ndarray:
    """Cell centres of an n_x x n_y grid over a rectangle in the plane z = const."""
    hx = (hi_xy[0] - lo_xy[0]) / n_xy[0]
    hy = (hi_xy[1] - lo_xy[1]) / n_xy[1]
    xs = lo_xy[0] + (np.arange(n_xy[0]) + 0.5) * hx
    ys = lo_xy[1] + (np.arange(n_xy[1]) + 0.5) * hy
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)


def grid_ff_halfsphere(step_deg: float = 2.0) -> np.ndarray:
    """Unit incident directions on the upper half sphere at an angular pitch step_deg.

    Elevation rings at 0, step, ..., 90-step deg each carry 360/step azimuths, plus
    the zenith as a single point: for a 2 deg pitch J = 45*180 + 1 = 8101, the
    far-field grid size of the paper's Table II.
    """
    n_az = int(round(360.0 / step_deg))
    n_el = int(round(90.0 / step_deg))
    dirs = [[0.0, 0.0, 1.0]]
    for e in range(n_el):  # elevations 0, step, ..., 90-step
        el = np.deg2rad(e * step_deg)
        az = np.deg2rad(np.arange(n_az) * step_deg)
        dirs.extend(np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az),
                              np.full(n_az, np.sin(el))], axis=1).tolist())
    return np.asarray(dirs, dtype=np.float64)


# ----------------------------------------------------------------------------------
# source signals
# ----------------------------------------------------------------------------------
def white(g: np.random.Generator, n: int) -> np.ndarray:
    return g.standard_normal(n)


def onoff_envelope(g: np.random.Generator, n: int, fs: float, seg_ms=(200.0, 400.0),
                   ramp_ms=10.0) -> np.ndarray:
    """Alternating on/off segments of U(seg_ms) duration with raised-cosine ramps."""
    env = np.zeros(n)
    pos, on = 0, bool(g.integers(0, 2))
    ramp = max(1, int(round(ramp_ms * 1e-3 * fs)))
    r = 0.5 - 0.5 * np.cos(np.pi * (np.arange(ramp) + 0.5) / ramp)
    while pos < n:
        seg = int(round(g.uniform(*seg_ms) * 1e-3 * fs))
        end = min(n, pos + seg)
        if on:
            env[pos:end] = 1.0
            k = min(ramp, end - pos)
            env[pos:pos + k] *= r[:k]
            env[end - k:end] *= r[::-1][ramp - k:]
        pos, on = end, not on
    return env


def ar_speech_like(g: np.random.Generator, n: int, fs: float, order_pairs: int = 5,
                   envelope: bool = True) -> np.ndarray:
    """AR(2*order_pairs) coloured noise with seeded conjugate pole pairs, gain-normalised.

    Pole radii U(0.7, 0.95), angles U(0.05 pi, 0.95 pi); optional on/off envelope.
    """
    radii = g.uniform(0.7, 0.95, order_pairs)
    angles = g.uniform(0.05 * np.pi, 0.95 * np.pi, order_pairs)
    poles = np.concatenate([radii * np.exp(1j * angles), radii * np.exp(-1j * angles)])
    a = np.real(np.poly(poles))  # denominator coefficients, a[0] = 1
    e = g.standard_normal(n)
    # all-pole filter via scipy (a library primitive for the input model)
    from scipy.signal import lfilter
    s = lfilter([1.0], a, e)
    s /= np.std(s) + 1e-300
    if envelope:
        s *= onoff_envelope(g, n, fs)
    return s


# ----------------------------------------------------------------------------------
# propagation
# ----------------------------------------------------------------------------------
def _fft_len(n: int) -> int:
    return 1 << int(np.ceil(np.log2(max(2, n))))


_CHUNK = 4096


def _ramps(shifts: np.ndarray, L: int) -> tuple:
    """Factors of the linear-phase ramps exp(-2 pi i k s / L), k = 0..L/2, for the shifts s:
    with k = k0 + j (k0 a multiple of _CHUNK, j < _CHUNK) the ramp is A[k0 / _CHUNK, s] *
    B[s, j].  Each factor is one FP64 exponential, so a ramp entry is exact to rounding.
    Returns (A [chunks][S], B [S][_CHUNK], number of bins)."""
    nb = L // 2 + 1
    nch = -(-nb // _CHUNK)
    k0 = np.arange(nch, dtype=np.float64) * _CHUNK
    j = np.arange(_CHUNK, dtype=np.float64)
    s = np.asarray(shifts, dtype=np.float64)
    A = np.exp((-2j * np.pi / L) * np.outer(k0, s))
    B = np.exp((-2j * np.pi / L) * np.outer(s, j))
    return A, B, nb


def propagate(sources, fs: float, mic_xyz: np.ndarray, n_out: int, c: float = C_SOUND,
              images=None) -> np.ndarray:
    """Free-field (or image-source) propagation with exact band-limited fractional delays.

    sources: list of (signal [n_in], position [3]).  images: optional list, per source,
    of (image_position [3], gain) replacing the direct path; by default each source has
    the single direct path with gain 1.  Each path contributes gain * s(t - d/c) / d
    where d is the path length.  The delay is applied as a linear phase on a zero-padded
    FFT whose length exceeds the signal plus the largest delay, so no wrap-around occurs.
    Returns float64 [M][n_out].
    """
    M = mic_xyz.shape[0]
    out = np.zeros((M, n_out))
    for si, (sig, pos) in enumerate(sources):
        paths = [(np.asarray(pos, float), 1.0)] if images is None else images[si]
        dmax = max(np.linalg.norm(mic_xyz - p[0], axis=1).max() for p in paths)
        L = _fft_len(max(len(sig), n_out) + int(np.ceil(dmax / c * fs)) + 64)
        S = np.fft.rfft(sig, L)
        ppos = np.array([p[0] for p in paths])
        pgain = np.array([p[1] for p in paths], dtype=np.float64)
        for m in range(M):
            d = np.linalg.norm(ppos - mic_xyz[m], axis=1)
            # sum over paths of (gain / d) exp(-2 pi i f d fs / c), f = k / L, as one
            # product of the ramp factors
            A, B, nb = _ramps(d / c * fs, L)
            acc = (A @ ((pgain / d)[:, None] * B)).ravel()[:nb]
            out[m] += np.fft.irfft(S * acc, L)[:n_out]
    return out


def image_sources(src, room, max_order: int, beta: float):
    """Image sources of a shoebox room with all walls of reflection coefficient beta.

    An image is kept when its total number of wall reflections (summed over the three
    axes) is at most max_order; its gain is beta**order.  Returns [(position, gain)].
    """
    src = np.asarray(src, float)
    out = []
    rng_a = range(-max_order - 1, max_order + 2)
    for a in rng_a:
        for b in rng_a:
            for cc in rng_a:
                for px in (0, 1):
                    for py in (0, 1):
                        for pz in (0, 1):
                            # per axis: coordinate 2*a*L + (1-2p)*x, reflections |2a-p|
                            ox = abs(2 * a - px)
                            oy = abs(2 * b - py)
                            oz = abs(2 * cc - pz)
                            order = ox + oy + oz
                            if order > max_order:
                                continue
                            pos = np.array([2 * a * room[0] + (1 - 2 * px) * src[0],
                                            2 * b * room[1] + (1 - 2 * py) * src[1],
                                            2 * cc * room[2] + (1 - 2 * pz) * src[2]])
                            out.append((pos, beta ** order))
    # remove duplicates (a=0,p=0 etc. are unique already; keep deterministic order)
    return out


def diffuse_noise(g: np.random.Generator, fs: float, mic_xyz: np.ndarray, n_out: int,
                  n_waves: int = 64, c: float = C_SOUND) -> np.ndarray:
    """Approximate diffuse noise: n_waves far-field plane waves from directions drawn
    uniformly on the sphere, each carrying an independent white signal."""
    M = mic_xyz.shape[0]
    v = g.standard_normal((n_waves, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    ctr = mic_xyz.mean(axis=0)
    rel = mic_xyz - ctr
    L = _fft_len(n_out + 64)
    nb = L // 2 + 1
    nch = -(-nb // _CHUNK)
    acc = np.zeros((M, nch * _CHUNK), dtype=np.complex128)
    for w in range(n_waves):
        S = np.zeros(nch * _CHUNK, dtype=np.complex128)
        S[:nb] = np.fft.rfft(g.standard_normal(n_out), L)
        S = S.reshape(nch, _CHUNK)
        adv = rel @ v[w] / c * fs  # arrival advance in samples for direction v
        A, B, _ = _ramps(-adv, L)  # exp(+2 pi i f adv) as factors
        for m in range(M):
            acc[m] += (S * np.outer(A[:, m], B[m])).ravel()
    return np.fft.irfft(acc[:, :nb], L, axis=1)[:, :n_out] / np.sqrt(n_waves)


def add_noise_snr(x: np.ndarray, noise: np.ndarray, snr_db: float) -> np.ndarray:
    """x + a * noise with a chosen so that mean-over-mics signal power / noise power = snr."""
    ps = np.mean(x ** 2)
    pn = np.mean(noise ** 2)
    a = np.sqrt(ps / (pn * 10.0 ** (snr_db / 10.0))) if pn > 0 else 0.0
    return x + a * noise


def cut_frames(x: np.ndarray, N: int, hop: int, F: int) -> np.ndarray:
    """[M][n] signal -> float32 [F][M][N] frames, frame f = samples [f*hop, f*hop+N)."""
    M = x.shape[0]
    out = np.empty((F, M, N), dtype=np.float32)
    for f in range(F):
        out[f] = x[:, f * hop:f * hop + N]
    return out


def circular_delay_frames(g: np.random.Generator, delays: np.ndarray, N: int, F: int) -> np.ndarray:
    """Frames whose length-N DFTs are exactly S_f[k] * exp(-j 2 pi k delays[m] / N).

    Each frame is one period of a periodic band-limited white signal, circularly delayed
    by delays[m] samples at microphone m; DC and Nyquist bins are zero.  Returns
    (float32 [F][M][N], the same frames in float64).
    """
    K = N // 2
    M = len(delays)
    out = np.empty((F, M, N), dtype=np.float64)
    k = np.arange(K + 1)
    for f in range(F):
        S = g.standard_normal(K + 1) + 1j * g.standard_normal(K + 1)
        S[0] = 0.0
        S[K] = 0.0
        for m in range(M):
            out[f, m] = np.fft.irfft(S * np.exp(-2j * np.pi * k * delays[m] / N), N)
    return out.astype(np.float32), out


# ----------------------------------------------------------------------------------
# workload presets
# ----------------------------------------------------------------------------------
WORKLOADS = ("square4", "uca8", "walls16", "nested32")


def _src_far_from(g, lo, hi, pts, dmin, plane_z=None):
    for _ in range(10000):
        p = g.uniform(lo, hi)
        if plane_z is not None:
            p[2] = plane_z
        if np.min(np.linalg.norm(pts - p, axis=1)) >= dmin:
            return p
    raise RuntimeError("no source position found")


def workload(name: str, F: int | None = None, grid_subsample: int = 1, seed: int | None = None):
    """Build a workload preset.  Returns a dict with keys
    mic_xyz [M][3], grid_xyz [J][3], fs, N, hop, F, frames float32 [F][M][N],
    sources (list of positions), window ('hann'), c.

    F overrides the number of frames (the signal is generated just long enough);
    grid_subsample > 1 keeps every k-th grid point (for oracle-sized parity cases).
    """
    idx = WORKLOADS.index(name) + 1
    g = rng(1000 + idx if seed is None else seed)
    if name == "square4":
        fs, N, hop, F0, snr = 16000.0, 512, 256, 100, 20.0
        mics = mics_square()
        grid = grid_plane((0.0, 0.0), (4.0, 4.0), (50, 50), z=0.0)
        F = F0 if F is None else F
        n = (F - 1) * hop + N
        src = _src_far_from(g, np.array([0.2, 0.2, 0.0]), np.array([3.8, 3.8, 0.0]), mics, 0.3, 0.0)
        s = white(g, n)
        x = propagate([(s, src)], fs, mics, n)
        noise = g.standard_normal(x.shape)
        x = add_noise_snr(x, noise, snr)
        sources = [src]
    elif name == "uca8":
        fs, N, hop, F0, snr = 16000.0, 512, 256, 2000, 10.0
        ctr = np.array([2.5, 2.0, 1.5])
        mics = mics_uca(8, 0.05, ctr)
        grid = grid_box((0, 0, 0), (5.0, 4.0, 3.0), 0.1)
        F = F0 if F is None else F
        n = (F - 1) * hop + N
        src = _src_far_from(g, np.array([0.3, 0.3, 0.3]), np.array([4.7, 3.7, 2.7]), ctr[None, :], 0.5)
        s = ar_speech_like(g, n, fs)
        x = propagate([(s, src)], fs, mics, n)
        x = add_noise_snr(x, diffuse_noise(g, fs, mics, n), snr)
        sources = [src]
    elif name == "walls16":
        fs, N, hop, F0, snr = 16000.0, 1024, 512, 4096, 15.0
        room = (6.0, 4.0, 3.0)
        mics = mics_walls(g, room)
        grid = grid_box((0, 0, 0), room, 0.1)
        F = F0 if F is None else F
        n = (F - 1) * hop + N
        srcs = [_src_far_from(g, np.array([0.5, 0.5, 0.5]), np.array([5.5, 3.5, 2.5]), mics, 0.5)
                for _ in range(2)]
        sigs = [ar_speech_like(g, n, fs) for _ in range(2)]
        imgs = [image_sources(p, room, 3, 0.7) for p in srcs]
        x = propagate(list(zip(sigs, srcs)), fs, mics, n, images=imgs)
        x = add_noise_snr(x, diffuse_noise(g, fs, mics, n), snr)
        sources = srcs
    elif name == "nested32":
        fs, N, hop, F0, snr = 16000.0, 2048, 1024, 1024, 20.0
        ctr = np.array([2.0, 1.5, 1.25])
        mics = mics_nested_uca(16, 0.04, 16, 0.12, ctr)
        grid = grid_box((0, 0, 0), (4.0, 3.0, 2.5), 0.05)
        F = F0 if F is None else F
        n = (F - 1) * hop + N
        src = _src_far_from(g, np.array([0.3, 0.3, 0.3]), np.array([3.7, 2.7, 2.2]), ctr[None, :], 0.5)
        s = ar_speech_like(g, n, fs)
        x = propagate([(s, src)], fs, mics, n)
        x = add_noise_snr(x, diffuse_noise(g, fs, mics, n), snr)
        sources = [src]
    else:  # pragma: no cover
        raise ValueError(name)
    if grid_subsample > 1:
        grid = grid[::grid_subsample].copy()
    frames = cut_frames(x, N, hop, F)
    return dict(name=name, mic_xyz=mics, grid_xyz=grid, fs=fs, N=N, hop=hop, F=F,
                frames=frames, sources=sources, window="hann", c=C_SOUND)
