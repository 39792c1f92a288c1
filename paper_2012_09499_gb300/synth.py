"""Seeded synthetic inputs: array geometries, candidate grids and free-field
STFT frames.

This module holds the signal model only (Sec. 2.1: a bandlimited source
propagating in free field to M microphones, observed through a square-root
Hann STFT).  It holds none of the SRP method's arithmetic (no cross spectra,
no GCC, no interpolation), so both the CUDA path and the FP64 oracle can be
fed from it.

The paper evaluates on a randomised image-method room with speech sources
and diffuse babble noise (Sec. 4); neither the simulator nor the corpora are
available, so white Gaussian sources with exact free-field fractional delays,
1/r gains and white sensor noise stand in for them, at the paper's array
scale, sampling rate and STFT sizes.
"""
from __future__ import annotations

import math

import numpy as np

C_SOUND = 343.0


# --------------------------------------------------------------------------
# geometries and grids
# --------------------------------------------------------------------------

def square_array_2d(side: float = 0.2, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Four microphones at the corners of a side x side square in the z=0 plane."""
    h = side / 2.0
    c = np.asarray(centre, np.float64)
    return np.array([[-h, -h, 0.0], [h, -h, 0.0], [h, h, 0.0], [-h, h, 0.0]]) + c


def plane_grid(extent: float = 4.0, n: int = 41, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n x n candidate points spanning [-extent/2, extent/2]^2 (edges included), z=0."""
    v = np.linspace(-extent / 2.0, extent / 2.0, n)
    gx, gy = np.meshgrid(v, v, indexing="ij")
    g = np.stack([gx.ravel(), gy.ravel(), np.zeros(gx.size)], axis=1)
    return g + np.asarray(centre, np.float64)


def random_cube_array(rng: np.random.Generator, M: int, edge: float, centre) -> np.ndarray:
    """M microphones uniform in an edge^3 cube centred at ``centre``."""
    return rng.uniform(-edge / 2.0, edge / 2.0, size=(M, 3)) + np.asarray(centre, np.float64)


def box_grid(shape=(100, 80, 60), spacing: float = 0.05, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Cell-centre candidate points of a regular 3D grid: origin + (i + 1/2) spacing."""
    axes = [np.asarray(origin[d], np.float64) + (np.arange(shape[d]) + 0.5) * spacing
            for d in range(3)]
    gx, gy, gz = np.meshgrid(*axes, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)


def circular_array(M: int = 6, radius: float = 0.1, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """M microphones equally spaced on a horizontal circle (Sec. 3.3, Sec. 4)."""
    a = 2.0 * np.pi * np.arange(M) / M
    return np.stack([radius * np.cos(a), radius * np.sin(a), np.zeros(M)], axis=1) + \
        np.asarray(centre, np.float64)


def half_sphere_directions(step_deg: float = 2.0) -> np.ndarray:
    """Far-field candidates on the lower half sphere (Sec. 4): theta from 90 to
    180 degrees and phi from 0 to 360-step degrees, r = -(sin t cos p, sin t sin p,
    cos t); the pole theta = 180 is one candidate.  step 2 gives J = 8101."""
    th = np.arange(90.0, 180.0 + 1e-9, step_deg)
    ph = np.arange(0.0, 360.0 - 1e-9, step_deg)
    dirs = []
    for t in th:
        for p in (ph if t < 180.0 - 1e-9 else ph[:1]):
            tr, pr = np.deg2rad(t), np.deg2rad(p)
            dirs.append([-np.sin(tr) * np.cos(pr), -np.sin(tr) * np.sin(pr), -np.cos(tr)])
    return np.asarray(dirs, np.float64)


# --------------------------------------------------------------------------
# signals
# --------------------------------------------------------------------------

def sqrt_hann(K: int) -> np.ndarray:
    """Periodic square-root Hann window of length K."""
    return np.sin(np.pi * np.arange(K) / K)


def _propagation(mic, src, c, far_field):
    """Per-microphone delay (s) and gain of a point source (1/r) or a plane
    wave travelling along unit vector ``src`` (gain 1)."""
    mic = np.asarray(mic, np.float64)
    src = np.asarray(src, np.float64)
    if far_field:
        return mic @ src / c, np.ones(mic.shape[0])
    r = np.linalg.norm(mic - src[None, :], axis=1)
    return r / c, 1.0 / r


def _delay_signal(s: np.ndarray, delays_samples: np.ndarray, gains: np.ndarray) -> np.ndarray:
    """Exact fractional delays applied in the DFT domain (circular over len(s));
    the Nyquist bin is dropped so every output stays real."""
    n = s.size
    S = np.fft.rfft(s)
    k = np.arange(S.size)
    out = np.empty((delays_samples.size, n))
    for m, (d, g) in enumerate(zip(delays_samples, gains)):
        X = S * g * np.exp(-2j * np.pi * k * d / n)
        if n % 2 == 0:
            X[-1] = 0.0
        out[m] = np.fft.irfft(X, n)
    return out


def stft(x: np.ndarray, K: int, L: int) -> np.ndarray:
    """Frames l = 0..L-1 with hop K/2, square-root Hann window, one-sided DFT:
    x[M][n] -> Y[L][M][K/2+1]."""
    hop = K // 2
    w = sqrt_hann(K)
    frames = np.stack([x[:, l * hop: l * hop + K] * w[None, :] for l in range(L)])
    return np.fft.rfft(frames, axis=-1)


def free_field_stft(rng: np.random.Generator, mic, sources, fs: float, K: int, L: int,
                    snr_db: float, c: float = C_SOUND, levels_db=None,
                    far_field: bool = False) -> np.ndarray:
    """STFT frames Y[L][M][K/2+1] (complex64) of white Gaussian sources in free
    field plus independent white sensor noise.

    ``sources`` is a list of positions (or unit propagation directions when
    ``far_field``); ``levels_db`` their relative levels.  SNR is the source
    power averaged over microphones (after the 1/r gains) over the noise power
    per microphone."""
    mic = np.asarray(mic, np.float64)
    M = mic.shape[0]
    n_out = (L - 1) * (K // 2) + K
    if levels_db is None:
        levels_db = [0.0] * len(sources)
    delays = []
    for src in sources:
        d, g = _propagation(mic, src, c, far_field)
        delays.append((d * fs, g))
    max_d = max(float(np.max(np.abs(d))) for d, _ in delays)
    pad = int(math.ceil(max_d)) + 64
    n = n_out + 2 * pad
    n += n % 2
    x = np.zeros((M, n_out))
    for (d, g), lev in zip(delays, levels_db):
        s = rng.standard_normal(n) * 10.0 ** (lev / 20.0)
        x += _delay_signal(s, d, g)[:, pad: pad + n_out]
    p_sig = float(np.mean(x ** 2))
    noise = rng.standard_normal((M, n_out)) * math.sqrt(p_sig / 10.0 ** (snr_db / 10.0))
    return stft(x + noise, K, L).astype(np.complex64)


def circular_frames(rng: np.random.Generator, mic, src, fs: float, K: int, L: int,
                    c: float = C_SOUND, far_field: bool = False) -> np.ndarray:
    """Noiseless frames whose delays are exact circular shifts within each
    frame: Y_m(k) = S_l(k) g_m e^{-j 2 pi k fs tau_m / K} for k < K/2, and the
    Nyquist bin set to zero.  With PHAT weighting the cross spectra are then
    pure phases of the true TDOAs."""
    d, g = _propagation(mic, src, c, far_field)
    Kb = K // 2 + 1
    k = np.arange(Kb)
    Y = np.zeros((L, len(d), Kb), np.complex128)
    for l in range(L):
        S = np.fft.rfft(rng.standard_normal(K))
        for m in range(len(d)):
            Y[l, m] = S * g[m] * np.exp(-2j * np.pi * k * fs * d[m] / K)
        Y[l, :, Kb - 1] = 0.0
    return Y.astype(np.complex64)


# --------------------------------------------------------------------------
# workload configurations (paper-scale synthetic setups)
# --------------------------------------------------------------------------

def tiny_2d(seed: int = 0, L: int = 16, snr_db: float = 20.0, K: int = 512,
            second_source_db=None) -> dict:
    """M=4 at the corners of a 0.2 m square centred in a 4 x 4 m plane; 41 x 41
    grid at 0.1 m (J=1681); fs=16 kHz; c=343 m/s; white source at a random
    in-plane location; optional second source at ``second_source_db``."""
    rng = np.random.default_rng(seed)
    mic = square_array_2d(0.2)
    grid = plane_grid(4.0, 41)
    srcs = [np.array([*rng.uniform(-1.8, 1.8, 2), 0.0])]
    levels = [0.0]
    if second_source_db is not None:
        srcs.append(np.array([*rng.uniform(-1.8, 1.8, 2), 0.0]))
        levels.append(float(second_source_db))
    Y = free_field_stft(rng, mic, srcs, 16000.0, K, L, snr_db, levels_db=levels)
    return dict(mic=mic, grid=grid, fs=16000.0, c=C_SOUND, K=K, L=L, Y=Y,
                sources=np.array(srcs), far_field=False, name="tiny_2d")


def room_3d(seed: int = 0, L: int = 64, K: int = 1024, shape=(100, 80, 60),
            spacing: float = 0.05, M: int = 8, snr_db: float = 10.0) -> dict:
    """M=8 uniform in a 0.5 m cube at the centre of a 5 x 4 x 3 m room; grid
    100 x 80 x 60 cell centres at 0.05 m (J=480000); fs=16 kHz; K=1024."""
    rng = np.random.default_rng(seed)
    room = np.array([5.0, 4.0, 3.0])
    mic = random_cube_array(rng, M, 0.5, room / 2.0)
    grid = box_grid(shape, spacing, (0.0, 0.0, 0.0))
    src = rng.uniform([0.3, 0.3, 0.3], room - 0.3)
    Y = free_field_stft(rng, mic, [src], 16000.0, K, L, snr_db)
    return dict(mic=mic, grid=grid, fs=16000.0, c=C_SOUND, K=K, L=L, Y=Y,
                sources=src[None, :], far_field=False, name="room_3d")


ROOM_MIX = np.array([6.0, 7.0, 3.5])  # the paper's room size (Sec. 4), candidates span it


def uneven_instance(seed: int, J_range=(10_000, 500_000), L: int = 32, dims=None, M=None,
                    K=None, aperture=None) -> dict:
    """One array of the uneven batch mix: M uniform in {4..16} microphones
    uniform in a cube of edge (aperture) uniform in [0.1, 1.0] m at the centre
    of a 6 x 7 x 3.5 m room; K in {512, 1024, 2048} at fs = 16 kHz; a 2D
    (horizontal plane through the array centre) or 3D candidate grid of cell
    centres spanning the room with J log-uniform in J_range; one white
    source at a uniform position (0.3 m from the walls; in the plane for 2D
    grids) at SNR uniform in [0, 30] dB; L frames.  Keyword arguments fix a
    draw."""
    rng = np.random.default_rng(seed)
    M = int(rng.integers(4, 17)) if M is None else int(M)
    aperture = float(rng.uniform(0.1, 1.0)) if aperture is None else float(aperture)
    K = int(rng.choice([512, 1024, 2048])) if K is None else int(K)
    dims = int(rng.choice([2, 3])) if dims is None else int(dims)
    lo, hi = J_range
    J_target = float(np.exp(rng.uniform(np.log(lo), np.log(hi))))
    snr = float(rng.uniform(0.0, 30.0))
    centre = ROOM_MIX / 2.0
    mic = random_cube_array(rng, M, aperture, centre)
    if dims == 2:
        nx = max(2, int(round(np.sqrt(J_target * ROOM_MIX[0] / ROOM_MIX[1]))))
        ny = max(2, int(round(J_target / nx)))
        sp = np.array([ROOM_MIX[0] / nx, ROOM_MIX[1] / ny])
        gx = (np.arange(nx) + 0.5) * sp[0]
        gy = (np.arange(ny) + 0.5) * sp[1]
        X, Yg = np.meshgrid(gx, gy, indexing="ij")
        grid = np.stack([X.ravel(), Yg.ravel(), np.full(X.size, centre[2])], axis=1)
        src = np.array([*rng.uniform(0.3, ROOM_MIX[:2] - 0.3), centre[2]])
    else:
        s = (J_target / float(np.prod(ROOM_MIX))) ** (1.0 / 3.0)
        shape = tuple(max(2, int(round(v * s))) for v in ROOM_MIX)
        axes = [(np.arange(shape[d]) + 0.5) * ROOM_MIX[d] / shape[d] for d in range(3)]
        gx, gy, gz = np.meshgrid(*axes, indexing="ij")
        grid = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
        src = rng.uniform(0.3, ROOM_MIX - 0.3)
    Y = free_field_stft(rng, mic, [src], 16000.0, K, L, snr)
    return dict(mic=mic, grid=grid, fs=16000.0, c=C_SOUND, K=K, L=L, Y=Y,
                sources=src[None, :], far_field=False, snr_db=snr, aperture=aperture,
                dims=dims, name="uneven")


def uneven_mix(seed: int, n: int, J_range=(10_000, 500_000), L: int = 32) -> list:
    """n arrays of the uneven mix (uneven_instance with seeds derived from seed)."""
    return [uneven_instance(seed * 100_003 + i, J_range, L) for i in range(n)]


def random_lower_direction(rng: np.random.Generator) -> np.ndarray:
    """A unit vector of the far-field candidate family of Sec. 4,
    -(sin t cos p, sin t sin p, cos t), with t uniform in [90, 180) degrees and
    p uniform in [0, 360) degrees (so it generally falls between grid points)."""
    t = np.deg2rad(rng.uniform(90.0, 180.0))
    p = np.deg2rad(rng.uniform(0.0, 360.0))
    return -np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])


def paper_circle_setup(seed: int, L: int = 32, K: int = 2048, step_deg: float = 2.0,
                       snr_range=(-3.0, 6.0)) -> dict:
    """The paper's evaluation geometry (Sec. 4) with synthetic signals: M = 6
    microphones on a circle of radius 0.1 m, far-field candidates on the lower
    half sphere at 2 degrees (J = 8101), fs = 16 kHz (omega_0 / 2 pi = 8 kHz),
    K = 2048 with a square-root Hann window.  One white plane-wave source
    from a random direction, with white sensor noise at an SNR uniform in
    snr_range (the paper's babble-noise SNRs; reverberation and speech are not
    modelled)."""
    rng = np.random.default_rng(seed)
    mic = circular_array(6, 0.1)
    grid = half_sphere_directions(step_deg)
    u = random_lower_direction(rng)
    snr = float(rng.uniform(*snr_range))
    Y = free_field_stft(rng, mic, [u], 16000.0, K, L, snr, far_field=True)
    return dict(mic=mic, grid=grid, fs=16000.0, c=C_SOUND, K=K, L=L, Y=Y, sources=u[None, :],
                far_field=True, snr_db=snr, name="paper_circle")
