/*
 * FP64 CPU oracle for steered response power (SRP) mapping, conventional and
 * Nyquist-Shannon approximated (Dietzen, De Sena, van Waterschoot,
 * "Low-Complexity Steered Response Power Mapping based on Nyquist-Shannon
 * Sampling", WASPAA 2021).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never does, and this file shares no code, header, table
 * or constant with it.
 *
 * Every routine is a plain loop over the definition it cites, in double
 * precision, with no blocking, fusion or reordering.  The only parallelism is
 * an OpenMP loop over independent candidate locations (or frames), which does
 * not change any per-output arithmetic.
 *
 * Conventions (the readings of the paper that the whole repository follows):
 *  - Pairs q <-> (m, m') with m > m' (Sec. 2.2, Eq. SRP_omegaT), enumerated
 *    m' = 0..M-2 outer, m = m'+1..M-1 inner.
 *  - Critical sampling period T = pi/omega_0 with omega_0 = pi*fs, i.e.
 *    T = 1/fs (Sec. 3.1); lags and TDOAs are expressed in samples,
 *    x = Delta t / T.
 *  - K is the DFT length (even); the one-sided spectrum has Kb = K/2+1 bins.
 *    The frequency integral (Eq. SRP_T / Eq. GCC_IFT) over the two-sided
 *    spectrum becomes (1/K) sum_{k=0}^{K/2} a_k Re[psi_k e^{j 2 pi k x/K}]
 *    with a_0 = a_{K/2} = 1 and a_k = 2 otherwise.  Constant factors (the 2
 *    of Eq. SRP_T_IFT, the bin spacing) are dropped; 1/K keeps |xi| <= 1.
 *  - Truncated interpolation (Eq. SRPapprox) sums n from -(N_q+N_aux) to
 *    N_q+N_aux; N_q = floor(d_q/(cT)) (Eq. SRPapprox, second line).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORC_PI = 3.14159265358979323846264338327950288;

static int g_threads = 0; /* 0 = OpenMP default */

void orc_set_threads(int n) { g_threads = n; }

int orc_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static int nthreads(void) { return orc_get_threads(); }

/* P = M(M-1)/2 microphone pairs (Sec. 2.1). */
int orc_num_pairs(int M) { return M * (M - 1) / 2; }

/* Pair table: q -> (m, m'), m > m' (Sec. 2.2, sum under Eq. SRP_omegaT). */
void orc_pairs(int M, int32_t *m_of_q, int32_t *mp_of_q) {
    int q = 0;
    for (int mp = 0; mp < M - 1; ++mp)
        for (int m = mp + 1; m < M; ++m) {
            m_of_q[q] = m;
            mp_of_q[q] = mp;
            ++q;
        }
}

static double dist3(const double *a, const double *b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* N_q = floor(Delta t_{q|0} / T) with Delta t_{q|0} = d_q / c and T = 1/fs
 * (Eq. Deltat_i_range, Eq. SRPapprox).  Writes d_q too. */
void orc_lag_counts(int M, const double *mic_xyz, double fs, double c,
                    int32_t *Nq, double *d_q) {
    int Q = orc_num_pairs(M);
    int32_t *m_of_q = malloc(sizeof(int32_t) * Q), *mp_of_q = malloc(sizeof(int32_t) * Q);
    orc_pairs(M, m_of_q, mp_of_q);
    for (int q = 0; q < Q; ++q) {
        double d = dist3(&mic_xyz[3 * m_of_q[q]], &mic_xyz[3 * mp_of_q[q]]);
        double T = 1.0 / fs;
        if (d_q) d_q[q] = d;
        Nq[q] = (int32_t)floor((d / c) / T);
    }
    free(m_of_q);
    free(mp_of_q);
}

/* Near-field TDOA in samples, Eq. Deltat_i:
 *   x[i][q] = (||p_m - q_i|| - ||p_m' - q_i||) / (c T).               */
void orc_tdoa_points(int M, const double *mic_xyz, int64_t J, const double *grid_xyz,
                     double fs, double c, double *x /* [J][Q] */) {
    int Q = orc_num_pairs(M);
    int32_t *m_of_q = malloc(sizeof(int32_t) * Q), *mp_of_q = malloc(sizeof(int32_t) * Q);
    orc_pairs(M, m_of_q, mp_of_q);
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int64_t i = 0; i < J; ++i)
        for (int q = 0; q < Q; ++q) {
            double dt = (dist3(&mic_xyz[3 * m_of_q[q]], &grid_xyz[3 * i]) -
                         dist3(&mic_xyz[3 * mp_of_q[q]], &grid_xyz[3 * i])) / c;
            x[i * Q + q] = dt * fs;
        }
    free(m_of_q);
    free(mp_of_q);
}

/* Far-field TDOA in samples, Eq. Deltat_i_spher:
 *   x[i][q] = (p_m - p_m')^T r_i / (c T),  r_i a unit direction.       */
void orc_tdoa_directions(int M, const double *mic_xyz, int64_t J, const double *dir_xyz,
                         double fs, double c, double *x /* [J][Q] */) {
    int Q = orc_num_pairs(M);
    int32_t *m_of_q = malloc(sizeof(int32_t) * Q), *mp_of_q = malloc(sizeof(int32_t) * Q);
    orc_pairs(M, m_of_q, mp_of_q);
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int64_t i = 0; i < J; ++i)
        for (int q = 0; q < Q; ++q) {
            const double *pm = &mic_xyz[3 * m_of_q[q]], *pmp = &mic_xyz[3 * mp_of_q[q]];
            const double *r = &dir_xyz[3 * i];
            double dt = ((pm[0] - pmp[0]) * r[0] + (pm[1] - pmp[1]) * r[1] +
                         (pm[2] - pmp[2]) * r[2]) / c;
            x[i * Q + q] = dt * fs;
        }
    free(m_of_q);
    free(mp_of_q);
}

/* PHAT-weighted cross spectra, Eq. corrmatrix with the PHAT weight of
 * Sec. 2.1:  psi_q(k) = y_m(k) y_m'(k)^* / |y_m(k) y_m'(k)^*|, and 0 where the
 * denominator vanishes (the paper leaves that case open).
 * Y: [L][M][Kb] complex (interleaved re, im); psi: [L][Q][Kb] complex.  */
void orc_phat(int64_t L, int M, int Kb, const double *Y, double *psi) {
    int Q = orc_num_pairs(M);
    int32_t *m_of_q = malloc(sizeof(int32_t) * Q), *mp_of_q = malloc(sizeof(int32_t) * Q);
    orc_pairs(M, m_of_q, mp_of_q);
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int64_t l = 0; l < L; ++l)
        for (int q = 0; q < Q; ++q)
            for (int k = 0; k < Kb; ++k) {
                const double *ym = &Y[2 * ((l * M + m_of_q[q]) * Kb + k)];
                const double *ymp = &Y[2 * ((l * M + mp_of_q[q]) * Kb + k)];
                /* y_m * conj(y_m') */
                double re = ym[0] * ymp[0] + ym[1] * ymp[1];
                double im = ym[1] * ymp[0] - ym[0] * ymp[1];
                double mag = sqrt(re * re + im * im);
                double *out = &psi[2 * ((l * Q + q) * Kb + k)];
                if (mag > 0.0) {
                    out[0] = re / mag;
                    out[1] = im / mag;
                } else {
                    out[0] = 0.0;
                    out[1] = 0.0;
                }
            }
    free(m_of_q);
    free(mp_of_q);
}

/* Unweighted cross spectra (Eq. corrmatrix without a GCC weighting; Sec. 2.1
 * notes that the method holds for any weighting): psi_q(k) = y_m(k) y_m'(k)^*
 * for the pair q = (m, m').  Same layout as orc_phat. */
void orc_cross_power(int64_t L, int M, int Kb, const double *Y, double *psi) {
    int Q = orc_num_pairs(M);
    int32_t *m_of_q = malloc(sizeof(int32_t) * Q), *mp_of_q = malloc(sizeof(int32_t) * Q);
    orc_pairs(M, m_of_q, mp_of_q);
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int64_t l = 0; l < L; ++l)
        for (int q = 0; q < Q; ++q)
            for (int k = 0; k < Kb; ++k) {
                const double *ym = &Y[2 * ((l * M + m_of_q[q]) * Kb + k)];
                const double *ymp = &Y[2 * ((l * M + mp_of_q[q]) * Kb + k)];
                double *out = &psi[2 * ((l * Q + q) * Kb + k)];
                out[0] = ym[0] * ymp[0] + ym[1] * ymp[1];
                out[1] = ym[1] * ymp[0] - ym[0] * ymp[1];
            }
    free(m_of_q);
    free(mp_of_q);
}

/* Bin weight of the one-sided discretisation of the two-sided integral. */
static double bin_weight(int k, int K) { return (k == 0 || 2 * k == K) ? 1.0 : 2.0; }

/* Discrete-frequency GCC of one pair at lag x (in samples), Eq. GCC_IFT:
 *   xi(x) = (1/K) sum_{k=0}^{K/2} a_k Re[psi(k) e^{j 2 pi k x / K}].     */
static double gcc_at(const double *psi_q, int K, double x) {
    int Kb = K / 2 + 1;
    double acc = 0.0;
    for (int k = 0; k < Kb; ++k) {
        double ph = 2.0 * ORC_PI * (double)k * x / (double)K;
        acc += bin_weight(k, K) * (psi_q[2 * k] * cos(ph) - psi_q[2 * k + 1] * sin(ph));
    }
    return acc / (double)K;
}

/* Conventional SRP map (Eq. SRP_T_IFT evaluated with the discrete IFT of
 * Eq. GCC_IFT at every TDOA, Sec. 2.4):
 *   map[l][i] = sum_q xi_q(x[i][q]).
 * psi: [L][Q][Kb] complex; x: [J][Q] samples; map: [L][J].              */
void orc_conventional(int64_t L, int Q, int K, const double *psi, int64_t J,
                      const double *x, double *map) {
    int Kb = K / 2 + 1;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads())
    for (int64_t i = 0; i < J; ++i)
        for (int64_t l = 0; l < L; ++l) {
            double acc = 0.0;
            for (int q = 0; q < Q; ++q)
                acc += gcc_at(&psi[2 * ((l * Q + q) * Kb)], K, x[i * Q + q]);
            map[l * J + i] = acc;
        }
}

/* Critical samples of every pair's GCC, xi_q(nT) for
 * n = -(N_q+N_aux) .. N_q+N_aux (Sec. 3.2, first step of the approximation).
 * Pair q's samples start at offset sum_{q'<q} (2N_q'+2N_aux+1); xi: [L][S]. */
void orc_gcc_samples(int64_t L, int Q, int K, const double *psi, const int32_t *Nq,
                     int n_aux, double *xi) {
    int Kb = K / 2 + 1;
    int64_t S = 0;
    for (int q = 0; q < Q; ++q) S += 2 * (int64_t)Nq[q] + 2 * n_aux + 1;
#pragma omp parallel for schedule(static) num_threads(nthreads())
    for (int64_t l = 0; l < L; ++l) {
        int64_t s = 0;
        for (int q = 0; q < Q; ++q) {
            int nmax = Nq[q] + n_aux;
            for (int n = -nmax; n <= nmax; ++n) {
                xi[l * S + s] = gcc_at(&psi[2 * ((l * Q + q) * Kb)], K, (double)n);
                ++s;
            }
        }
    }
}

/* sinc(u) = sin(pi u)/(pi u), sinc(0) = 1 (Eq. SRPinterp). */
static double sinc(double u) {
    if (u == 0.0) return 1.0;
    return sin(ORC_PI * u) / (ORC_PI * u);
}

/* Nyquist-Shannon SRP approximation (Eq. SRPapprox summed over pairs with
 * Eq. SRP_T_IFT, Sec. 3.2):
 *   map[l][i] = sum_q sum_{n=-(N_q+N_aux)}^{N_q+N_aux} xi_q(nT) sinc(x[i][q] - n). */
void orc_nyquist(int64_t L, int Q, const int32_t *Nq, int n_aux, const double *xi,
                 int64_t J, const double *x, double *map) {
    int64_t S = 0;
    for (int q = 0; q < Q; ++q) S += 2 * (int64_t)Nq[q] + 2 * n_aux + 1;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads())
    for (int64_t i = 0; i < J; ++i)
        for (int64_t l = 0; l < L; ++l) {
            double acc = 0.0;
            int64_t s = 0;
            for (int q = 0; q < Q; ++q) {
                int nmax = Nq[q] + n_aux;
                for (int n = -nmax; n <= nmax; ++n) {
                    acc += xi[l * S + s] * sinc(x[i * Q + q] - (double)n);
                    ++s;
                }
            }
            map[l * J + i] = acc;
        }
}

/* Source location estimate: the first (lowest index) maximiser of the map
 * per frame (Sec. 2.2, last sentence).                                    */
void orc_argmax(int64_t L, int64_t J, const double *map, int64_t *idx, double *val) {
    for (int64_t l = 0; l < L; ++l) {
        int64_t best = 0;
        double bv = map[l * J];
        for (int64_t i = 1; i < J; ++i)
            if (map[l * J + i] > bv) {
                bv = map[l * J + i];
                best = i;
            }
        idx[l] = best;
        val[l] = bv;
    }
}
