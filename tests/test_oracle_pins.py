"""Pins of the FP64 oracle to facts fixed outside it: the paper's printed
numbers, closed forms, library routines and invariances.  CPU only.

Each test is chosen so that a plausible slip in the oracle (a dropped bin
weight, a sign of the phase, a pair or lag index, a transposed operand)
breaks at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2012_09499_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _cross(Y):
    """Unweighted cross spectra psi_q = y_m y_m'^* (pairs m > m')."""
    L, M, Kb = Y.shape
    m, mp = oracle.pairs(M)
    return Y[:, m, :] * np.conj(Y[:, mp, :])


# --------------------------------------------------------------------------
# pair table, lag counts, TDOAs
# --------------------------------------------------------------------------

def test_pairs_order_and_count():
    m, mp = oracle.pairs(5)
    assert len(m) == 10  # P = M(M-1)/2, Sec. 2.1
    assert np.all(m > mp)
    assert list(zip(mp, m))[:4] == [(0, 1), (0, 2), (0, 3), (0, 4)]
    assert len(set(zip(m, mp))) == 10


def test_paper_complexity_example():
    """Sec. 3.3 / Sec. 4 worked numbers (tests/golden/paper_complexity_example.txt)."""
    gold = {}
    with open(os.path.join(GOLDEN, "paper_complexity_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v, tol = line.split()
                gold[k] = (float(v), tol)
    mic = synth.circular_array(6, 0.1)
    Nq, d = oracle.lag_counts(mic, 16000.0, 340.0)
    P = len(Nq)
    J = synth.half_sphere_directions(2.0).shape[0]
    K = 1024
    assert sorted(Nq.tolist()) == [4] * 6 + [8] * 6 + [9] * 3

    c0, c1, c2 = (oracle.complexity(mic, 16000.0, 340.0, K, J, n) for n in (0, 1, 2))
    vals = {
        "P": c2["P"], "J": J, "N_at_naux0": c0["N"], "N_slope_per_naux": c1["N"] - c0["N"],
        "C_conv": c2["C_conv"], "C_samp_naux2": c2["C_samp"], "C_int_naux2": c2["C_int"],
        "R_samp_naux2": c2["R_samp"], "R_int_naux2": c2["R_int"],
    }
    assert c2["R"] == pytest.approx(c2["R_samp"] + c2["R_int"], rel=1e-15)
    for k, (v, tol) in gold.items():
        if tol == "exact":
            assert vals[k] == v, k
        else:
            assert abs(vals[k] - v) <= float(tol) + 1e-12 * abs(v), (k, vals[k], v)


def test_complexity_circle_closed_form():
    """Sec. 3.3 for an M = 6 circle of radius r (the setting of Fig. 2): the 15
    chords are r (6 pairs), r sqrt(3) (6) and 2r (3), so N is a closed form in
    r; R_samp grows with the radius, R_int = R_samp J / K_b, and R_samp falls
    as 1/J at fixed r."""
    fs, c, K_b = 16000.0, 340.0, 1024
    prev = 0.0
    for r in np.linspace(0.01, 0.5, 50):
        mic = synth.circular_array(6, r)
        f = lambda dist: np.floor(dist * fs / c)  # noqa: E731
        for naux in (0, 1, 2):
            N = 2.0 / 15.0 * (6 * f(r) + 6 * f(np.sqrt(3.0) * r) + 3 * f(2.0 * r)) + 2 * naux + 1
            for J in (1000, 8101, 100000):
                cx = oracle.complexity(mic, fs, c, K_b, J, naux)
                # chord lengths computed from coordinates may round across an
                # integer boundary: only then may N differ, by 2/15 per pair class
                assert abs(cx["N"] - N) <= 2.0 / 15.0 * 6 + 1e-12
                assert cx["R_samp"] == pytest.approx(cx["N"] / J, rel=1e-15)
                assert cx["R_int"] == pytest.approx(cx["R_samp"] * J / K_b, rel=1e-12)
        cx = oracle.complexity(mic, fs, c, K_b, 8101, 0)
        assert cx["R_samp"] >= prev
        prev = cx["R_samp"]
    # away from integer boundaries the closed form is exact
    for r in (0.03, 0.1, 0.23, 0.41):
        cx = oracle.complexity(synth.circular_array(6, r), fs, c, K_b, 8101, 2)
        f = lambda dist: np.floor(dist * fs / c)  # noqa: E731
        assert cx["N"] == 2.0 / 15.0 * (6 * f(r) + 6 * f(np.sqrt(3.0) * r) + 3 * f(2 * r)) + 5


# --------------------------------------------------------------------------
# coarse-to-fine refinement (oracle.refine)
# --------------------------------------------------------------------------

def test_refine_at_exact_sample_points():
    """Where every pair's TDOA is an integer lag, Eq. SRPapprox returns the
    GCC sample itself (sinc(0) = 1, sinc(k) = 0), so SRP_appr = sum_q xi_q(x_q).
    A linear array along x with spacing c / fs and the far-field directions
    +x and -x give x_q = m - m' and m' - m (Eq. Deltat_i_spher)."""
    fs, c = 8192.0, 256.0
    mic = np.array([[k / 32.0, 0.0, 0.0] for k in range(4)])  # spacing 1/32 m = c / fs
    rng = np.random.default_rng(7)
    psi = oracle.cross_spectra(_rand_cplx(rng, (3, 4, 33)))  # K = 64
    Nq, _ = oracle.lag_counts(mic, fs, c)
    assert Nq.tolist() == [1, 2, 3, 1, 2, 1]
    xi = oracle.gcc_samples(psi, Nq, 1, 64)
    m, mp = oracle.pairs(4)
    offs = np.concatenate([[0], np.cumsum(2 * Nq + 3)[:-1]])
    for sgn in (1, -1):
        centres = np.tile([float(sgn), 0.0, 0.0], (3, 1))
        best, val, last = oracle.refine(xi, mic, fs, c, Nq, 1, centres, np.zeros((1, 3)), 1, 0.5,
                                        far_field=True)
        lag = sgn * (m - mp)
        expect = [sum(xi[l, offs[q] + lag[q] + Nq[q] + 1] for q in range(6)) for l in range(3)]
        assert np.allclose(last[:, 0], expect, rtol=0.0, atol=1e-12)
        assert np.array_equal(best, centres) and np.array_equal(val, last[:, 0])


def _cube(h):
    g = np.array([-1.0, 0.0, 1.0]) * h
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.concatenate([np.zeros((1, 3)), pts[np.any(pts != 0.0, axis=1)]])  # 0 first


def test_refine_level_invariants():
    """Facts the search fixes: with the zero displacement in the stencil the
    best value never falls from one level to the next; on a direction grid
    every point has unit norm; with displacements {0, h e_x} and shrink 1/2
    the result after V levels is c + b h 2^-(V-1) e_x with integer b in
    [0, 2^V - 1]."""
    rng = np.random.default_rng(11)
    mic = rng.uniform(-0.15, 0.15, (5, 3))
    fs, c, K = 16000.0, 343.0, 256
    Nq, _ = oracle.lag_counts(mic, fs, c)
    xi = oracle.gcc_samples(oracle.cross_spectra(_rand_cplx(rng, (2, 5, K // 2 + 1))), Nq, 2, K)
    centres = rng.uniform(-1.0, 1.0, (2, 3))
    vals = [oracle.refine(xi, mic, fs, c, Nq, 2, centres, _cube(0.1), v, 0.5)[1]
            for v in range(1, 5)]
    for a, b in zip(vals, vals[1:]):
        assert np.all(b >= a)
    dirs = centres / np.linalg.norm(centres, axis=1, keepdims=True)
    best, _, _ = oracle.refine(xi, mic, fs, c, Nq, 2, dirs, _cube(0.2), 3, 0.5, far_field=True)
    assert np.allclose(np.linalg.norm(best, axis=1), 1.0, rtol=0.0, atol=1e-12)
    h, V = 0.08, 5
    best, _, _ = oracle.refine(xi, mic, fs, c, Nq, 2, centres, np.array([[0, 0, 0], [h, 0, 0]]),
                               V, 0.5)
    d = best - centres
    assert np.all(d[:, 1:] == 0.0)
    b = d[:, 0] / h * 2 ** (V - 1)
    assert np.allclose(b, np.round(b), atol=1e-9) and np.all((b > -0.5) & (b < 2 ** V - 0.5))


def test_lag_count_exact_integer_boundary():
    # d = 0.5 m, c = 256 m/s, fs = 8192 Hz: d fs / c = 16 exactly in binary.
    mic = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0]])
    Nq, d = oracle.lag_counts(mic, 8192.0, 256.0)
    assert Nq.tolist() == [16] and d[0] == 0.5


def test_tdoa_bounds_and_limits():
    rng = np.random.default_rng(1)
    mic = rng.uniform(-0.3, 0.3, (5, 3))
    fs, c = 16000.0, 343.0
    grid = rng.uniform(-3, 3, (400, 3))
    x = oracle.tdoa(mic, grid, fs, c)
    _, d = oracle.lag_counts(mic, fs, c)
    assert np.all(np.abs(x) <= d[None, :] * fs / c + 1e-9)  # Eq. Deltat_i_range
    # collinear candidate beyond mic m on the line m' -> m: |Delta t| = d/c
    m, mp = oracle.pairs(5)
    q = 3
    u = mic[m[q]] - mic[mp[q]]
    pt = mic[m[q]] + 2.5 * u
    xq = oracle.tdoa(mic, pt[None, :], fs, c)[0, q]
    assert xq == pytest.approx(-d[q] * fs / c, rel=1e-12)
    # far field: r along p_m - p_m' gives +d/c (Eq. Deltat_i_spher)
    r = u / np.linalg.norm(u)
    xf = oracle.tdoa(mic, r[None, :], fs, c, far_field=True)[0, q]
    assert xf == pytest.approx(d[q] * fs / c, rel=1e-12)
    # far field is the limit of near field for a distant source along -r
    far_pt = -1e6 * r
    xn = oracle.tdoa(mic, far_pt[None, :], fs, c)[0]
    xd = oracle.tdoa(mic, r[None, :], fs, c, far_field=True)[0]
    np.testing.assert_allclose(xn, xd, atol=1e-5)


# --------------------------------------------------------------------------
# PHAT
# --------------------------------------------------------------------------

def test_phat_is_pure_phase_difference():
    rng = np.random.default_rng(2)
    L, M, Kb = 3, 4, 9
    phase = rng.uniform(-np.pi, np.pi, (L, M, Kb))
    mag = rng.uniform(0.01, 100.0, (L, M, Kb))
    Y = mag * np.exp(1j * phase)
    Y[1, 2, 4] = 0.0  # zero denominator -> psi = 0
    psi = oracle.phat(Y)
    m, mp = oracle.pairs(M)
    expect = np.exp(1j * (phase[:, m, :] - phase[:, mp, :]))
    zero = np.zeros_like(expect, bool)
    zero[1, (m == 2) | (mp == 2), 4] = True
    expect[zero] = 0.0
    np.testing.assert_allclose(psi, expect, atol=1e-13)


# --------------------------------------------------------------------------
# conventional SRP
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M", [2, 3, 5])
def test_dsb_equivalence_bruteforce(M):
    """Eq. SRP_omegaT: h^H Psi h - tr Psi = 2 sum_{m>m'} Re[psi e^{j w dt}],
    integrated over the two-sided spectrum (Eq. SRP_T), equals 2K times the
    oracle's one-sided conventional map.  Psi is unweighted here: the paper
    states the relation holds for any weighting."""
    rng = np.random.default_rng(10 + M)
    K, L, fs, c = 16, 2, 16000.0, 343.0
    Kb = K // 2 + 1
    mic = rng.uniform(-0.2, 0.2, (M, 3))
    grid = rng.uniform(-2, 2, (7, 3))
    Y = _rand_cplx(rng, (L, M, Kb))
    got = oracle.conventional(_cross(Y), oracle.tdoa(mic, grid, fs, c), K)
    # brute force: steering vector relative to mic 1 (Eq. h_steering)
    ks = np.arange(-K // 2 + 1, K // 2 + 1)
    ref = np.zeros((L, grid.shape[0]))
    for l in range(L):
        for i, g in enumerate(grid):
            dist = np.linalg.norm(mic - g, axis=1)
            dt1 = (dist - dist[0]) / c
            tot = 0.0
            for k in ks:
                y = Y[l, :, k] if k >= 0 else np.conj(Y[l, :, -k])
                Psi = np.outer(y, np.conj(y))
                w = 2 * np.pi * k * fs / K
                h = np.exp(-1j * w * dt1)
                tot += (np.conj(h) @ Psi @ h - np.trace(Psi)).real
            ref[l, i] = tot / (2 * K)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_conventional_single_bin_closed_form():
    """A single bin k0 with psi = e^{j phi}: xi(x) = (a_k0/K) cos(2 pi k0 x/K + phi)."""
    K = 32
    Kb = K // 2 + 1
    x = np.array([[-3.7], [0.0], [1.25], [5.5]])
    for k0, a in [(0, 1.0), (5, 2.0), (K // 2, 1.0)]:
        psi = np.zeros((1, 1, Kb), complex)
        phi = 0.3
        psi[0, 0, k0] = np.exp(1j * phi)
        got = oracle.conventional(psi, x, K)[0]
        np.testing.assert_allclose(got, a / K * np.cos(2 * np.pi * k0 * x[:, 0] / K + phi),
                                   atol=1e-15)


def test_conventional_linear_and_invariant():
    rng = np.random.default_rng(3)
    M, K, L, fs, c = 4, 32, 2, 16000.0, 343.0
    Kb = K // 2 + 1
    mic = rng.uniform(-0.2, 0.2, (M, 3))
    grid = rng.uniform(-2, 2, (25, 3))
    Y1, Y2 = _rand_cplx(rng, (L, M, Kb)), _rand_cplx(rng, (L, M, Kb))
    x = oracle.tdoa(mic, grid, fs, c)
    p1, p2 = oracle.phat(Y1), oracle.phat(Y2)
    lin = oracle.conventional(0.7 * p1 - 1.3 * p2, x, K)
    np.testing.assert_allclose(lin, 0.7 * oracle.conventional(p1, x, K)
                               - 1.3 * oracle.conventional(p2, x, K), atol=1e-12)
    base, _, _ = oracle.srp_map(Y1, mic, grid, fs, c, K, "conventional")
    # common translation of microphones and grid
    t = np.array([1.5, -0.7, 2.0])
    moved, _, _ = oracle.srp_map(Y1, mic + t, grid + t, fs, c, K, "conventional")
    np.testing.assert_allclose(moved, base, atol=1e-11)
    # relabelling the microphones (pairs permute, signs of psi and dt flip together)
    perm = np.array([2, 0, 3, 1])
    rel, _, _ = oracle.srp_map(Y1[:, perm, :], mic[perm], grid, fs, c, K, "conventional")
    np.testing.assert_allclose(rel, base, atol=1e-11)
    # Nyquist map is invariant under the same relabelling
    nb, _, _ = oracle.srp_map(Y1, mic, grid, fs, c, K, "nyquist", n_aux=1)
    nr, _, _ = oracle.srp_map(Y1[:, perm, :], mic[perm], grid, fs, c, K, "nyquist", n_aux=1)
    np.testing.assert_allclose(nr, nb, atol=1e-11)


# --------------------------------------------------------------------------
# GCC samples and the Nyquist-Shannon approximation
# --------------------------------------------------------------------------

def test_gcc_samples_equal_inverse_rfft():
    """At integer lags the discrete GCC is the real inverse DFT of psi."""
    rng = np.random.default_rng(4)
    K, Q, L = 32, 3, 2
    Kb = K // 2 + 1
    psi = _rand_cplx(rng, (L, Q, Kb))
    Nq = np.array([15, 15, 15], np.int32)
    xi = oracle.gcc_samples(psi, Nq, 0, K).reshape(L, Q, 31)
    ref = np.fft.irfft(psi, K, axis=-1)
    n = np.arange(-15, 16)
    np.testing.assert_allclose(xi, ref[:, :, n % K], atol=1e-14)


def test_untruncated_interpolation_is_exact():
    """With psi real at DC and Nyquist, the K-periodic samples interpolated by
    the untruncated sinc series (which sums to the Dirichlet kernel
    sin(pi u)/(K tan(pi u/K))) reproduce the conventional GCC at any lag."""
    rng = np.random.default_rng(5)
    K = 24
    Kb = K // 2 + 1
    psi = _rand_cplx(rng, (1, 1, Kb))
    psi[..., 0] = psi[..., 0].real
    psi[..., -1] = psi[..., -1].real
    xi = oracle.gcc_samples(psi, np.array([K // 2], np.int32), 0, K)[0]
    n = np.arange(-K // 2, K // 2 + 1)
    samples = {int(nn) % K: v for nn, v in zip(n, xi)}
    xs = rng.uniform(-K / 2, K / 2, 9)
    conv = oracle.conventional(psi, xs[:, None], K)[0]
    for xv, cv in zip(xs, conv):
        u = xv - np.arange(K)
        D = np.sin(np.pi * u) / (K * np.tan(np.pi * u / K))
        assert abs(sum(samples[j] * D[j] for j in range(K)) - cv) < 1e-12


def test_truncated_interpolation_converges():
    """Symmetric truncation of the sinc series at +-N approaches the
    conventional value as N grows (Eq. SRPinterp -> Eq. SRPapprox)."""
    rng = np.random.default_rng(6)
    K = 64
    Kb = K // 2 + 1
    psi = _rand_cplx(rng, (1, 1, Kb))
    psi[..., 0] = psi[..., 0].real
    psi[..., -1] = psi[..., -1].real
    xs = rng.uniform(-6, 6, (16, 1))
    conv = oracle.conventional(psi, xs, K)[0]
    peak = np.abs(conv).max()
    errs = []
    for N in [10, 100, 1000, 10000]:
        Nq = np.array([N], np.int32)
        approx = oracle.nyquist(oracle.gcc_samples(psi, Nq, 0, K), Nq, 0, xs)[0]
        errs.append(np.abs(approx - conv).max())
    assert errs[-1] < 1e-4 * peak
    assert errs[-1] < errs[1] < errs[0]


def test_nyquist_single_sample_is_sinc():
    """One nonzero critical sample xi_q(n0) = 1 gives map = sinc(x - n0)."""
    Nq = np.array([3, 2], np.int32)
    n_aux = 1
    S = int(np.sum(2 * Nq + 2 * n_aux + 1))
    x = np.array([[0.3, -1.6], [2.0, 0.0], [-3.9, 2.5]])
    for q, n0 in [(0, -4), (0, 2), (1, 3), (1, -1)]:
        xi = np.zeros((1, S))
        off = 0 if q == 0 else 2 * (Nq[0] + n_aux) + 1
        xi[0, off + n0 + Nq[q] + n_aux] = 1.0
        got = oracle.nyquist(xi, Nq, n_aux, x)[0]
        np.testing.assert_allclose(got, np.sinc(x[:, q] - n0), atol=1e-15)


def test_nyquist_equals_conventional_at_integer_tdoas():
    """Where every TDOA is an integer lag inside the sampled range, the sinc
    weights reduce to a unit impulse and both maps agree exactly."""
    rng = np.random.default_rng(7)
    K, Q, L = 64, 3, 2
    Kb = K // 2 + 1
    psi = _rand_cplx(rng, (L, Q, Kb))
    Nq = np.array([4, 7, 2], np.int32)
    x = np.stack([rng.integers(-n, n + 1, 20) for n in Nq], axis=1).astype(float)
    for n_aux in [0, 2]:
        ny = oracle.nyquist(oracle.gcc_samples(psi, Nq, n_aux, K), Nq, n_aux, x)
        np.testing.assert_allclose(ny, oracle.conventional(psi, x, K), atol=1e-13)


def test_peak_at_true_source_noiseless():
    """Noiseless free field, source on a grid point, exact circular delays:
    the conventional map peaks there at the closed-form value Q (K-1)/K and
    the Nyquist approximation finds the same cell."""
    rng = np.random.default_rng(8)
    mic = synth.square_array_2d(0.2)
    grid = synth.plane_grid(4.0, 41)
    fs, c, K, L = 16000.0, 343.0, 256, 3
    for src_idx in [  # a few grid points at least 0.5 m from the array
        int(np.argmin(np.linalg.norm(grid - p, axis=1)))
        for p in ([1.2, -0.8, 0], [-1.5, 1.7, 0], [0.6, 0.5, 0])
    ]:
        Y = synth.circular_frames(rng, mic, grid[src_idx], fs, K, L)
        maps, idx, val = oracle.srp_map(Y, mic, grid, fs, c, K, "conventional")
        assert np.all(idx == src_idx)
        np.testing.assert_allclose(val, 6 * (K - 1) / K, rtol=1e-12)
        _, idx_n, _ = oracle.srp_map(Y, mic, grid, fs, c, K, "nyquist", n_aux=2)
        assert np.all(idx_n == src_idx)


def test_far_field_peak_on_half_sphere():
    rng = np.random.default_rng(9)
    mic = synth.circular_array(6, 0.1)
    dirs = synth.half_sphere_directions(2.0)
    fs, c, K = 16000.0, 340.0, 512
    src = 1234
    Y = synth.circular_frames(rng, mic, dirs[src], fs, K, 2, c=c, far_field=True)
    _, idx, val = oracle.srp_map(Y, mic, dirs, fs, c, K, "conventional", far_field=True)
    assert np.all(idx == src)
    np.testing.assert_allclose(val, 15 * (K - 1) / K, rtol=1e-12)


def test_approximation_error_small_on_synthetic_scene():
    """e_appr (Sec. 4) on the 2D white-noise scene is small and falls from
    N_aux = 0 to N_aux = 2 (the paper reports the same trend)."""
    cfg = synth.tiny_2d(seed=0, L=4)
    args = (cfg["Y"], cfg["mic"], cfg["grid"], cfg["fs"], cfg["c"], cfg["K"])
    conv, ic, _ = oracle.srp_map(*args, mode="conventional")
    e = []
    for n_aux in [0, 2]:
        ny, _, _ = oracle.srp_map(*args, mode="nyquist", n_aux=n_aux)
        e.append(np.median(oracle.e_appr_db(conv, ny)))
    assert e[1] < e[0] < -15.0


def test_approximation_error_closed_forms():
    """e_appr (Sec. 4, the ratio of the squared-error sum to the map's squared
    sum, in dB) in closed form: an approximation (1 - a) SRP has error a SRP
    at every candidate, so e_appr = 20 log10 |a| dB for any map; a single
    error of size eps at one candidate gives 10 log10(eps^2 / sum_i SRP^2);
    the value is per frame (row) and does not depend on the map's scale."""
    rng = np.random.default_rng(17)
    srp = rng.normal(size=(5, 333))
    for a in (0.5, 0.1, 1e-3, 2.0, -0.25):
        e = oracle.e_appr_db(srp, (1.0 - a) * srp)
        assert e.shape == (5,)
        np.testing.assert_allclose(e, 20.0 * np.log10(abs(a)), rtol=0, atol=1e-10)
    # SRP = (3, 4), SRP_appr = (3, 5): one unit error against a squared sum of 25
    np.testing.assert_allclose(oracle.e_appr_db([3.0, 4.0], [3.0, 5.0]),
                               [10.0 * np.log10(1.0 / 25.0)], rtol=0, atol=1e-12)
    rows = oracle.e_appr_db([[3.0, 4.0], [1.0, 0.0]], [[3.0, 5.0], [1.0, 0.1]])
    np.testing.assert_allclose(rows, [-13.979400086720377, -20.0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.e_appr_db(7.0 * srp, 7.0 * (0.9 * srp)),
                               oracle.e_appr_db(srp, 0.9 * srp), rtol=0, atol=1e-12)


def test_argmax_first_maximum():
    """Ties resolve to the lowest candidate index (the first maximiser)."""
    maps = np.array([[0.0, 2.0, 1.0, 2.0], [-1.0, -1.0, -3.0, -1.0], [5.0, 5.0, 5.0, 5.0]])
    idx, val = oracle.argmax(maps)
    assert idx.tolist() == [1, 0, 0]
    assert val.tolist() == [2.0, -1.0, 5.0]


def test_unweighted_cross_power_closed_form():
    """No GCC weighting (Sec. 2.1: the method holds for any weighting).  In
    noiseless free field with exact circular delays every pair's cross
    spectrum is in phase at the source, so the conventional map there equals
    (1/K) sum_q sum_k a_k |y_m(k)| |y_m'(k)| and is the maximum; the
    unweighted map scales with the square of an input gain, the PHAT map not
    at all; and the unweighted cross spectrum of one pair and bin is
    y_m conj(y_m')."""
    rng = np.random.default_rng(12)
    mic = synth.square_array_2d(0.2)
    grid = synth.plane_grid(4.0, 41)
    fs, c, K, L = 16000.0, 343.0, 256, 2
    src = int(np.argmin(np.linalg.norm(grid - np.array([1.1, -0.7, 0.0]), axis=1)))
    Y = synth.circular_frames(rng, mic, grid[src], fs, K, L).astype(np.complex128)
    args = (mic, grid, fs, c, K)
    maps, idx, val = oracle.srp_map(Y, *args, mode="conventional", weighting="none")
    Kb = K // 2 + 1
    a = np.full(Kb, 2.0)
    a[0] = a[-1] = 1.0
    A = np.abs(Y.astype(np.complex128))
    expect = [sum(np.sum(a * A[l, m] * A[l, mp]) for mp in range(4) for m in range(mp + 1, 4)) / K
              for l in range(L)]
    assert np.all(idx == src)
    np.testing.assert_allclose(val, expect, rtol=1e-12)
    m3, _, _ = oracle.srp_map(3.0 * Y, *args, mode="conventional", weighting="none")
    np.testing.assert_allclose(m3, 9.0 * maps, rtol=1e-12, atol=1e-11 * np.abs(maps).max())
    p1, _, _ = oracle.srp_map(Y, *args, mode="conventional")
    p3, _, _ = oracle.srp_map(3.0 * Y, *args, mode="conventional")
    np.testing.assert_allclose(p3, p1, rtol=1e-12, atol=1e-12)
    psi = oracle.cross_power(Y)  # pairs m' = 0..M-2 outer, m > m' inner: q = 3 is (2, 1)
    np.testing.assert_allclose(psi[1, 3, 7], complex(Y[1, 2, 7]) * np.conj(complex(Y[1, 1, 7])),
                               rtol=1e-12)
