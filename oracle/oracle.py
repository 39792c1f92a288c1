"""FP64 CPU oracle for SRP mapping (conventional and Nyquist-Shannon).

TEST INFRASTRUCTURE ONLY: the slow, obviously correct definition that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it.  It
shares no code with the product library (it does not import the package and
the package does not import it).

The arithmetic lives in ``srp_oracle.c`` (plain double-precision loops, each
citing its equation); this module only loads it with ctypes, marshals numpy
arrays and composes the steps in the paper's order (Sec. 3.2):
PHAT cross-spectra -> GCC at every TDOA (conventional) or GCC samples at the
critical lags followed by truncated sinc interpolation (Nyquist) -> sum over
pairs -> argmax.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srp_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.orc_set_threads.argtypes = [i32]
            lib.orc_get_threads.restype = i32
            lib.orc_num_pairs.argtypes = [i32]
            lib.orc_num_pairs.restype = i32
            lib.orc_pairs.argtypes = [i32, i32p, i32p]
            lib.orc_lag_counts.argtypes = [i32, f64p, f64, f64, i32p, f64p]
            lib.orc_tdoa_points.argtypes = [i32, f64p, i64, f64p, f64, f64, f64p]
            lib.orc_tdoa_directions.argtypes = [i32, f64p, i64, f64p, f64, f64, f64p]
            lib.orc_phat.argtypes = [i64, i32, i32, f64p, f64p]
            lib.orc_cross_power.argtypes = [i64, i32, i32, f64p, f64p]
            lib.orc_conventional.argtypes = [i64, i32, i32, f64p, i64, f64p, f64p]
            lib.orc_gcc_samples.argtypes = [i64, i32, i32, f64p, i32p, i32, f64p]
            lib.orc_nyquist.argtypes = [i64, i32, i32p, i32, f64p, i64, f64p, f64p]
            lib.orc_argmax.argtypes = [i64, i64, f64p, i64p, f64p]
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (0 = all host cores)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _c64(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def pairs(M: int):
    """(m, m') per pair q, m > m' (Sec. 2.2)."""
    lib = _load()
    Q = lib.orc_num_pairs(M)
    m = np.zeros(Q, np.int32)
    mp = np.zeros(Q, np.int32)
    lib.orc_pairs(M, m, mp)
    return m, mp


def lag_counts(mic_xyz, fs: float, c: float):
    """N_q = floor(d_q fs / c) and d_q per pair (Eq. SRPapprox)."""
    mic = _c64(mic_xyz)
    M = mic.shape[0]
    Q = M * (M - 1) // 2
    Nq = np.zeros(Q, np.int32)
    d = np.zeros(Q, np.float64)
    _load().orc_lag_counts(M, mic, float(fs), float(c), Nq, d)
    return Nq, d


def complexity(mic_xyz, fs: float, c: float, K_b: int, J: int, n_aux: int):
    """Operation counts of Sec. 3.3 (C_conv of Sec. 2.3) for one frame, with
    K_b one-sided frequency bins (the paper's K): the average number of
    critical samples per pair N = (2/P) sum N_q + 2 N_aux + 1, C_samp = N P K_b
    complex multiplications of the partial IDFT, C_int = N P J real
    multiplications of the interpolation, C_conv = J P K_b, and the reduction
    factors R_samp = C_samp / C_conv, R_int = C_int / C_conv, R = their sum."""
    Nq, _ = lag_counts(mic_xyz, fs, c)
    P = len(Nq)
    N = 2.0 / P * float(np.sum(Nq, dtype=np.int64)) + 2.0 * n_aux + 1.0
    C_samp, C_int, C_conv = N * P * K_b, N * P * J, float(J) * P * K_b
    return {"N": N, "P": P, "K_b": K_b, "J": J, "C_samp": C_samp, "C_int": C_int,
            "C_conv": C_conv, "R_samp": C_samp / C_conv, "R_int": C_int / C_conv,
            "R": (C_samp + C_int) / C_conv}


def tdoa(mic_xyz, grid_xyz, fs: float, c: float, far_field: bool = False):
    """TDOAs in samples, [J][Q] (Eq. Deltat_i or Eq. Deltat_i_spher)."""
    mic = _c64(mic_xyz)
    grid = _c64(grid_xyz)
    M, J = mic.shape[0], grid.shape[0]
    x = np.zeros((J, M * (M - 1) // 2), np.float64)
    fn = _load().orc_tdoa_directions if far_field else _load().orc_tdoa_points
    fn(M, mic, J, grid, float(fs), float(c), x)
    return x


def _cplx_to_f64(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64).reshape(a.shape + (2,))


def phat(Y):
    """PHAT cross spectra psi[L][Q][Kb] from STFT frames Y[L][M][Kb] (Eq. corrmatrix)."""
    Y = np.asarray(Y)
    L, M, Kb = Y.shape
    Q = M * (M - 1) // 2
    psi = np.zeros((L, Q, Kb, 2), np.float64)
    _load().orc_phat(L, M, Kb, _c64(_cplx_to_f64(Y)), psi)
    return psi[..., 0] + 1j * psi[..., 1]


def cross_power(Y):
    """Unweighted cross spectra psi[L][Q][Kb] = y_m conj(y_m') (Eq. corrmatrix
    without a GCC weighting)."""
    Y = np.asarray(Y)
    L, M, Kb = Y.shape
    Q = M * (M - 1) // 2
    psi = np.zeros((L, Q, Kb, 2), np.float64)
    _load().orc_cross_power(L, M, Kb, _c64(_cplx_to_f64(Y)), psi)
    return psi[..., 0] + 1j * psi[..., 1]


def cross_spectra(Y, weighting="phat"):
    """PHAT-weighted (default) or unweighted cross spectra of STFT frames."""
    return phat(Y) if weighting == "phat" else cross_power(Y)


def conventional(psi, x, K: int):
    """Conventional SRP map[L][J] from psi[L][Q][Kb] and TDOAs x[J][Q] (Sec. 2.4)."""
    psi = np.asarray(psi)
    L, Q, Kb = psi.shape
    assert Kb == K // 2 + 1
    x = _c64(x)
    J = x.shape[0]
    out = np.zeros((L, J), np.float64)
    _load().orc_conventional(L, Q, K, _c64(_cplx_to_f64(psi)), J, x, out)
    return out


def gcc_samples(psi, Nq, n_aux: int, K: int):
    """Critical GCC samples xi[L][S], pairs concatenated (Sec. 3.2)."""
    psi = np.asarray(psi)
    L, Q, Kb = psi.shape
    Nq = _c64(Nq, np.int32)
    S = int(np.sum(2 * Nq.astype(np.int64) + 2 * n_aux + 1))
    out = np.zeros((L, S), np.float64)
    _load().orc_gcc_samples(L, Q, K, _c64(_cplx_to_f64(psi)), Nq, int(n_aux), out)
    return out


def nyquist(xi, Nq, n_aux: int, x):
    """Nyquist-Shannon SRP approximation map[L][J] (Eq. SRPapprox, Sec. 3.2)."""
    xi = _c64(xi)
    L = xi.shape[0]
    Nq = _c64(Nq, np.int32)
    x = _c64(x)
    J, Q = x.shape
    out = np.zeros((L, J), np.float64)
    _load().orc_nyquist(L, Q, Nq, int(n_aux), xi, J, x, out)
    return out


def refine(xi, mic_xyz, fs, c, Nq, n_aux: int, centres, offsets, levels: int, shrink: float,
           far_field: bool = False):
    """Coarse-to-fine search on the approximation (the refinement Sec. 3.3
    leaves outside the paper's scope), step by step per frame l: level v
    evaluates SRP_appr (Eq. SRPapprox summed over pairs) at the points
    c_v + shrink^v o_f, normalised onto the unit sphere on a direction grid;
    c_0 is the frame's centre and c_{v+1} the first maximiser of level v.
    Returns (best point [L][3], its value [L], values of the last level
    [L][F])."""
    xi = np.atleast_2d(np.asarray(xi, np.float64))
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    offsets = np.asarray(offsets, np.float64).reshape(-1, 3)
    L = xi.shape[0]
    best = np.zeros((L, 3))
    best_val = np.zeros(L)
    last = np.zeros((L, offsets.shape[0]))
    for l in range(L):
        centre = centres[l].copy()
        scale = 1.0
        for v in range(levels):
            pts = centre[None, :] + scale * offsets
            if far_field:
                nrm = np.sqrt(np.sum(pts ** 2, axis=1))
                pts = np.where(nrm[:, None] > 0.0, pts / np.where(nrm > 0.0, nrm, 1.0)[:, None],
                               centre[None, :])
            vals = nyquist(xi[l:l + 1], Nq, n_aux, tdoa(mic_xyz, pts, fs, c, far_field))[0]
            (k,), (val,) = argmax(vals[None, :])
            centre = pts[k].copy()
            scale *= shrink
        best[l], best_val[l], last[l] = centre, val, vals
    return best, best_val, last


def argmax(maps):
    """First maximiser and its value per frame (Sec. 2.2)."""
    maps = _c64(maps)
    L, J = maps.shape
    idx = np.zeros(L, np.int64)
    val = np.zeros(L, np.float64)
    _load().orc_argmax(L, J, maps, idx, val)
    return idx, val


def e_appr_db(srp, srp_appr):
    """Approximation error per frame in dB (Sec. 4):
    10 log10( sum_i (SRP - SRP_appr)^2 / sum_i SRP^2 )."""
    srp = np.atleast_2d(np.asarray(srp, np.float64))
    srp_appr = np.atleast_2d(np.asarray(srp_appr, np.float64))
    num = np.sum((srp - srp_appr) ** 2, axis=-1)
    den = np.sum(srp ** 2, axis=-1)
    return 10.0 * np.log10(num / den)


def srp_map(Y, mic_xyz, grid_xyz, fs, c, K, mode="nyquist", n_aux=2,
            far_field=False, psi=None, weighting="phat"):
    """Whole path for one block of frames: returns (maps[L][J], argmax[L], peak[L]).

    ``Y`` are STFT frames [L][M][Kb]; pass ``psi`` instead to start from
    already weighted cross spectra [L][Q][Kb]."""
    x = tdoa(mic_xyz, grid_xyz, fs, c, far_field)
    if psi is None:
        psi = cross_spectra(Y, weighting)
    if mode == "conventional":
        maps = conventional(psi, x, K)
    elif mode == "nyquist":
        Nq, _ = lag_counts(mic_xyz, fs, c)
        maps = nyquist(gcc_samples(psi, Nq, n_aux, K), Nq, n_aux, x)
    else:
        raise ValueError(mode)
    idx, val = argmax(maps)
    return maps, idx, val
