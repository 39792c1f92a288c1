// Host side of the SRP library: descriptor validation, the FP64 planner
// (pairs, lag counts, TDOA tables, twiddles), device memory ownership and
// the C-ABI entry points that enqueue the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "srp_internal.h"

namespace srp {
namespace {

thread_local std::string g_err;

constexpr int kMaxM = 64;
constexpr int kMaxK = 8192;
constexpr int kMaxFrames = 65536;
constexpr int64_t kMaxJ = (int64_t)INT32_MAX - (1 << 20);
constexpr int kMaxLagSpan = 8192;  // 2 (N_q + N_aux) + 1 per pair

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

bool finite3(const double *p) { return isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]); }

// Slots of pair q on the tensor-core reduction axis: its critical lags
// 2(N_q + N_aux) + 1 (Nyquist) or its bins as (re, im) pairs, 2 Kb (conventional).
int64_t tc_span(const srp_plan_desc *d, const Layout &lay, int q) {
    if (d->mode == SRP_MODE_NYQUIST) return 2 * ((int64_t)lay.Nq[q] + d->n_aux) + 1;
    return 2 * (int64_t)lay.Kb;
}

// Validate the descriptor and compute every size of the plan.  Host only.
srp_status make_layout(const srp_plan_desc *d, Layout &lay) {
    if (d == nullptr) return fail(SRP_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->M < 2 || d->M > kMaxM) return fail(SRP_ERR_INVALID_ARG, "M must be in [2, 64]");
    if (d->mic_xyz == nullptr) return fail(SRP_ERR_INVALID_ARG, "mic_xyz is NULL");
    if (d->J < 1 || d->J > kMaxJ) return fail(SRP_ERR_INVALID_ARG, "J out of range");
    if (d->grid_xyz == nullptr) return fail(SRP_ERR_INVALID_ARG, "grid_xyz is NULL");
    if (!(d->fs > 0.0) || !isfinite(d->fs)) return fail(SRP_ERR_INVALID_ARG, "fs must be > 0");
    if (!(d->c > 0.0) || !isfinite(d->c)) return fail(SRP_ERR_INVALID_ARG, "c must be > 0");
    if (d->K < 4 || d->K > kMaxK || (d->K & 1))
        return fail(SRP_ERR_INVALID_ARG, "K must be even and in [4, 8192]");
    if (d->mode != SRP_MODE_CONV && d->mode != SRP_MODE_NYQUIST)
        return fail(SRP_ERR_INVALID_ARG, "unknown mode");
    if (d->n_aux < 0) return fail(SRP_ERR_INVALID_ARG, "n_aux must be >= 0");
    if (d->precision != SRP_PREC_FP32 && d->precision != SRP_PREC_BF16 &&
        d->precision != SRP_PREC_FP16)
        return fail(SRP_ERR_INVALID_ARG, "unknown precision");
    if (d->input_kind != SRP_IN_STFT && d->input_kind != SRP_IN_CROSS)
        return fail(SRP_ERR_INVALID_ARG, "unknown input kind");
    if (d->grid_kind != SRP_GRID_POINTS && d->grid_kind != SRP_GRID_DIRECTIONS)
        return fail(SRP_ERR_INVALID_ARG, "unknown grid kind");
    if (d->engine != SRP_ENGINE_AUTO && d->engine != SRP_ENGINE_CUDA_CORES)
        return fail(SRP_ERR_INVALID_ARG, "unknown engine");
    if (d->weighting != SRP_WEIGHT_PHAT && d->weighting != SRP_WEIGHT_NONE)
        return fail(SRP_ERR_INVALID_ARG, "unknown weighting");
    if (d->weighting == SRP_WEIGHT_NONE && d->precision == SRP_PREC_FP16 &&
        d->input_kind == SRP_IN_STFT)
        return fail(SRP_ERR_UNSUPPORTED, "unweighted spectra can exceed the FP16 range");
    if (d->max_frames < 1 || d->max_frames > kMaxFrames)
        return fail(SRP_ERR_INVALID_ARG, "max_frames must be in [1, 65536]");
    for (int m = 0; m < d->M; ++m)
        if (!finite3(d->mic_xyz + 3 * m)) return fail(SRP_ERR_INVALID_ARG, "mic_xyz not finite");

    lay = Layout();
    lay.M = d->M;
    lay.Q = d->M * (d->M - 1) / 2;
    lay.K = d->K;
    lay.Kb = d->K / 2 + 1;
    lay.n_aux = d->mode == SRP_MODE_NYQUIST ? d->n_aux : 0;
    lay.J = d->J;
    lay.J_pad = round_up(d->J, kTileJ);
    lay.n_tiles = (int)(lay.J_pad / kTileJ);
    lay.L_max = d->max_frames;
    lay.L_pad = (int)round_up(d->max_frames, kFramePad);

    // Pairs (m > m', m' outer) and lag counts N_q = floor(d_q fs / c).
    double max_bound = 0.0;
    for (int mp = 0; mp < d->M - 1; ++mp)
        for (int m = mp + 1; m < d->M; ++m) {
            const double *a = d->mic_xyz + 3 * m, *b = d->mic_xyz + 3 * mp;
            const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
            const double dq = sqrt(dx * dx + dy * dy + dz * dz);
            const double bound = dq / d->c * d->fs;
            if (bound > 1.0e6) return fail(SRP_ERR_UNSUPPORTED, "array aperture too large for fs/c");
            lay.pm.push_back(m);
            lay.pmp.push_back(mp);
            lay.Nq.push_back((int32_t)floor(bound));
            max_bound = std::max(max_bound, bound);
        }
    lay.max_nq = *std::max_element(lay.Nq.begin(), lay.Nq.end());
    int64_t S = 0;
    if (d->mode == SRP_MODE_NYQUIST) {
        for (int q = 0; q < lay.Q; ++q) {
            const int64_t span = 2 * (int64_t)lay.Nq[q] + 2 * (int64_t)d->n_aux + 1;
            if (span > kMaxLagSpan)
                return fail(SRP_ERR_UNSUPPORTED, "2(N_q + N_aux) + 1 exceeds 8192 lags");
            lay.off.push_back((int32_t)S);
            S += span;
        }
    } else {
        lay.off.assign(lay.Q, 0);
    }
    lay.S = (int)S;
    lay.S_pad = (int)round_up(S, kLagPad);
    // Both maps run on the tensor cores unless CUDA cores are asked for; the
    // CUDA-core engine is FP32 only.  FP32 accumulation in TMEM carries a
    // systematic relative bias of about kTcAccumBias per accumulated MMA step
    // (measured on GB300), so an FP32 plan whose reduction is long enough for
    // that bias to reach kTcBiasLimit, half of the 1e-4 tolerance (long
    // conventional sums: many pairs x many bins), runs on the exact CUDA-core
    // kernels instead.
    lay.tc = d->engine == SRP_ENGINE_AUTO;
    if (lay.tc) {
        int64_t steps = 0;  // 16-slot MMA steps per tile
        for (int q = 0; q < lay.Q; ++q) steps += round_up(tc_span(d, lay, q), 16) / 16;
        lay.mma_steps = (int)std::min<int64_t>(steps, INT32_MAX);
        const double adds = 3.0 * (double)steps / 2.0;  // 3 products, 2 accumulators
        if (d->precision == SRP_PREC_FP32 && adds * kTcAccumBias > kTcBiasLimit) {
            // A long conventional reduction stays on the tensor cores if its
            // accumulators can be promoted: every kPromoteChunks chunks of 64
            // slots (4 MMA steps, 3 products, over 2 accumulators) they are
            // added into FP32 sums and restarted, which bounds the bias of
            // each partial sum by kPromoteChunks * 6 * kTcAccumBias, a quarter of
            // the limit.  That needs A in TMEM (at most 64 frames per CTA).
            const bool can = d->mode == SRP_MODE_CONV &&
                             interp_tc_frames_per_cta(d->max_frames) <= 64;
            if (can)
                lay.promote = kPromoteChunks;
            else
                lay.tc = false;
        }
    }
    if (!lay.tc && d->precision != SRP_PREC_FP32)
        return fail(SRP_ERR_UNSUPPORTED, "BF16/FP16 need the tensor-core engine");
    if (lay.tc) {
        // reduction axis per pair: the critical lags (Nyquist) or the bins as
        // (re, im) element pairs (conventional), padded to 64-slot chunks
        int64_t sc = 0;
        for (int q = 0; q < lay.Q; ++q) {
            lay.offc.push_back((int32_t)sc);
            sc += round_up(tc_span(d, lay, q), kLagPad);
        }
        // the second accumulator takes every other 16-slot step of the tile
        lay.par1_used = lay.mma_steps >= 2 ? 1 : 0;
        lay.Sc = (int)sc;
        lay.n_chunks = (int)(sc / kLagPad);
        lay.N_tc = interp_tc_frames_per_cta(d->max_frames);
    }
    if (d->argmax != SRP_ARGMAX_RESCORE && d->argmax != SRP_ARGMAX_MAP)
        return fail(SRP_ERR_INVALID_ARG, "unknown argmax mode");
    lay.rescore = lay.tc && d->precision != SRP_PREC_FP32 && d->argmax == SRP_ARGMAX_RESCORE;
    if (!(d->resident_fraction >= 0.0f && d->resident_fraction <= 1.0f))
        return fail(SRP_ERR_INVALID_ARG, "resident_fraction must be in [0, 1]");
    if (d->resident_fraction > 0.0f) {
        if (!lay.tc || d->mode != SRP_MODE_NYQUIST)
            return fail(SRP_ERR_UNSUPPORTED,
                        "resident weights need a Nyquist plan on the tensor cores");
        // whole pairs, interleaved: pair q is streamed when that brings the
        // streamed steps closer to the fraction of the steps so far
        const double frac = d->resident_fraction;
        int64_t total = 0, streamed = 0;
        lay.streamed.assign(lay.Q, 0);
        for (int q = 0; q < lay.Q; ++q) {
            const int64_t s_q = (tc_span(d, lay, q) + 15) / 16;  // 16-slot MMA steps of pair q
            total += s_q;
            const double target = frac * (double)total;
            if (fabs((double)(streamed + s_q) - target) < fabs((double)streamed - target)) {
                lay.streamed[q] = 1;
                streamed += s_q;
            }
        }
        lay.tile_steps = (int)streamed;
        lay.total_steps = (int)total;
    }

    // Fixed-point TDOA: the largest xf <= 24 with (max|x| + 2) 2^xf < 2^31.
    // Far-field directions must be unit vectors so that |x| <= d fs / c.
    int xf = 24;
    while (xf > 8 && (max_bound + 2.0) * ldexp(1.0, xf) >= 2147483648.0) --xf;
    if ((max_bound + 2.0) * ldexp(1.0, xf) >= 2147483648.0)
        return fail(SRP_ERR_UNSUPPORTED, "TDOA range too large");
    lay.xf = xf;

    const bool nyq = d->mode == SRP_MODE_NYQUIST;
    const bool half = d->precision != SRP_PREC_FP32;
    lay.b_pairs = sizeof(int2) * lay.Q;
    lay.b_nq = sizeof(int32_t) * lay.Q;
    lay.b_off = sizeof(int32_t) * lay.Q;
    lay.b_x = lay.tc ? 0 : sizeof(int32_t) * (size_t)lay.Q * (size_t)lay.J_pad;
    lay.b_twid = nyq ? sizeof(float2) * lay.K : 0;
    lay.b_psi = d->input_kind == SRP_IN_STFT
                    ? sizeof(float2) * (size_t)lay.L_max * lay.Q * lay.Kb : 0;
    lay.b_xi = (nyq && !lay.tc) ? sizeof(float) * (size_t)lay.S_pad * lay.L_pad : 0;
    lay.b_xi16 = lay.tc ? sizeof(uint16_t) * (half ? 1 : 2) * (size_t)lay.L_pad * lay.Sc : 0;
    // FP32 re-scoring: the Nyquist samples in FP32 (the conventional map reads
    // the cross spectra, formed into b_psi from STFT input)
    lay.b_xi32 = (lay.rescore && nyq) ? sizeof(float) * (size_t)lay.L_pad * lay.S_pad : 0;
    lay.b_rs = lay.rescore ? (sizeof(unsigned long long) * (1 + kRescoreCtas) + sizeof(int)) *
                                 (size_t)lay.L_pad : 0;
    // the GCC samples of a Nyquist tensor-core plan with PHAT-weighted STFT
    // input by the tensor-core IDFT where its shape allows (else the CUDA-core
    // sample kernel)
    lay.nmax_all = lay.max_nq + lay.n_aux;
    lay.gcc_mma = lay.tc && nyq && d->weighting == SRP_WEIGHT_PHAT &&
                  d->input_kind == SRP_IN_STFT && gcc_mma_fits(lay.K, lay.nmax_all);
    lay.b_gtw = lay.gcc_mma ? gcc_mma_twiddle_bytes(lay.K, lay.nmax_all) : 0;
    lay.b_offc = lay.tc ? sizeof(int32_t) * lay.Q : 0;
    lay.b_xs = lay.tc ? sizeof(int2) * (size_t)lay.Q * (size_t)lay.J_pad : 0;
    lay.b_ctab = lay.tc ? sizeof(int4) * (size_t)lay.n_chunks : 0;
    lay.b_w = lay.tile_steps ? (size_t)lay.n_tiles * lay.tile_steps * (half ? 1 : 2) * 4096 : 0;
    lay.b_woff = lay.tile_steps ? sizeof(int32_t) * (size_t)lay.n_chunks : 0;
    lay.b_status = sizeof(int);
    lay.b_part = sizeof(unsigned long long) * (size_t)lay.L_pad * lay.n_tiles;
    if (d->host_io < 0 || d->host_io > 2) return fail(SRP_ERR_INVALID_ARG, "host_io must be 0, 1 or 2");
    if (d->host_io) {  // host_io staging slots, each 256-byte aligned
        const int rows = d->input_kind == SRP_IN_STFT ? lay.M : lay.Q;
        const size_t slots = (size_t)d->host_io;
        lay.b_in_stage = slots * round_up(sizeof(float2) * (size_t)lay.L_max * rows * lay.Kb, 256);
        lay.b_maps_stage = slots * round_up(sizeof(float) * (size_t)lay.L_max * (size_t)lay.J, 256);
        lay.b_small_stage = slots * 2 * round_up(sizeof(float) * (size_t)lay.L_pad, 256);
    }
    return SRP_OK;
}

srp_status check_grid(const srp_plan_desc *d) {
    for (int64_t i = 0; i < d->J; ++i) {
        const double *g = d->grid_xyz + 3 * i;
        if (!finite3(g)) return fail(SRP_ERR_INVALID_ARG, "grid_xyz not finite");
        if (d->grid_kind == SRP_GRID_DIRECTIONS) {
            const double n = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            if (fabs(n - 1.0) > 1e-6)
                return fail(SRP_ERR_INVALID_ARG, "direction vectors must have unit length");
        }
    }
    return SRP_OK;
}

void fill_info(const Layout &lay, srp_plan_info *info) {
    info->M = lay.M;
    info->Q = lay.Q;
    info->K = lay.K;
    info->Kb = lay.Kb;
    info->J = lay.J;
    info->n_aux = lay.n_aux;
    info->S = lay.S;
    info->max_nq = lay.max_nq;
    info->x_frac_bits = lay.xf;
    info->max_frames = lay.L_max;
    info->tensor_cores = lay.tc ? 1 : 0;
    info->device_bytes = lay.total();
    info->weight_bytes = lay.b_w;
    info->argmax_rescored = lay.rescore ? 1 : 0;
    info->accum_promotion = lay.promote;
    info->gcc_tensor_cores = lay.gcc_mma ? 1 : 0;
}

template <typename T>
cudaError_t dalloc(T **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

void release(srp_plan_s *h) {
    cudaFree(h->d_pairs);
    cudaFree(h->d_nq);
    cudaFree(h->d_off);
    cudaFree(h->d_x);
    cudaFree(h->d_twid);
    cudaFree(h->d_gtw);
    cudaFree(h->d_psi);
    cudaFree(h->d_xi);
    cudaFree(h->d_xi16);
    cudaFree(h->d_xi32);
    cudaFree(h->d_rs_fkey);
    cudaFree(h->d_offc);
    cudaFree(h->d_xs);
    cudaFree(h->d_ctab);
    cudaFree(h->d_w);
    cudaFree(h->d_woff);
    cudaFree(h->d_status);
    cudaFree(h->d_part);
    cudaFree(h->d_in_stage);
    cudaFree(h->d_maps_stage);
    cudaFree(h->d_argmax_stage);
    cudaFree(h->d_peak_stage);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < 2; ++k) {
        if (h->ev_in[k]) cudaEventDestroy(h->ev_in[k]);
        if (h->ev_done[k]) cudaEventDestroy(h->ev_done[k]);
        if (h->ev_out[k]) cudaEventDestroy(h->ev_out[k]);
    }
    if (h->io_in) cudaStreamDestroy(h->io_in);
    if (h->io_out) cudaStreamDestroy(h->io_out);
}

// Build the TDOA table in FP64 (Eq. Deltat_i / Eq. Deltat_i_spher), convert
// x = Delta t fs to fixed point and upload it as [Q][J_pad]: int32 for the
// CUDA-core kernels, or, for the tensor cores, (X, bits of sp) with
// sp = (-1)^x0 sin(pi f) / pi for x = x0 + f decoded exactly as the kernel
// decodes it (f = 0, an exact sample, is taken as 2^-40).  The candidates
// are split over host threads.
srp_status build_tdoa(const srp_plan_desc *d, srp_plan_s *h) {
    const Layout &lay = h->lay;
    std::vector<int32_t> X;
    std::vector<int2> xs;
    if (lay.tc) xs.assign((size_t)lay.Q * lay.J_pad, make_int2(0, 0));
    else X.assign((size_t)lay.Q * lay.J_pad, 0);
    const double scale = ldexp(1.0, lay.xf);
    const bool far = d->grid_kind == SRP_GRID_DIRECTIONS;
    const double pi = 3.141592653589793238462643383279502884;
    const int32_t half = 1 << (lay.xf - 1);
    // entry of a padding candidate (X = 0)
    auto tc_entry = [&](int32_t Xk) {
        const int32_t x0 = (Xk + half) >> lay.xf;
        double f = ldexp((double)(Xk - x0 * (1 << lay.xf)), -lay.xf);
        if (f == 0.0) f = ldexp(1.0, -40);
        float sp = (float)(sin(pi * f) / pi);
        if (x0 & 1) sp = -sp;
        int32_t bits;
        memcpy(&bits, &sp, sizeof bits);
        return make_int2(Xk, bits);
    };
    auto work = [&](int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; ++i) {
            double dist[kMaxM];
            const double *g = i < lay.J ? d->grid_xyz + 3 * i : nullptr;
            if (g != nullptr && !far)
                for (int m = 0; m < lay.M; ++m) {
                    const double *p = d->mic_xyz + 3 * m;
                    const double dx = p[0] - g[0], dy = p[1] - g[1], dz = p[2] - g[2];
                    dist[m] = sqrt(dx * dx + dy * dy + dz * dz);
                }
            for (int q = 0; q < lay.Q; ++q) {
                int32_t Xk = 0;
                if (g != nullptr) {
                    const int m = lay.pm[q], mp = lay.pmp[q];
                    double dt;
                    if (far) {
                        const double *a = d->mic_xyz + 3 * m, *b = d->mic_xyz + 3 * mp;
                        dt = ((a[0] - b[0]) * g[0] + (a[1] - b[1]) * g[1] + (a[2] - b[2]) * g[2]) /
                             d->c;
                    } else {
                        dt = (dist[m] - dist[mp]) / d->c;
                    }
                    Xk = (int32_t)llround(dt * d->fs * scale);
                }
                const size_t k = (size_t)q * lay.J_pad + i;
                if (lay.tc) xs[k] = tc_entry(Xk);
                else X[k] = Xk;
            }
        }
    };
    const int64_t work_items = lay.J_pad * (int64_t)lay.Q;
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 64u));
    if (work_items < (1 << 16)) nt = 1;
    if (nt == 1) {
        work(0, lay.J_pad);
    } else {
        std::vector<std::thread> pool;
        const int64_t per = (lay.J_pad + nt - 1) / nt;
        for (unsigned t = 0; t < nt; ++t) {
            const int64_t a = std::min<int64_t>(lay.J_pad, (int64_t)t * per);
            const int64_t b = std::min<int64_t>(lay.J_pad, a + per);
            if (a < b) pool.emplace_back(work, a, b);
        }
        for (auto &th : pool) th.join();
    }
    if (!lay.tc) {
        SRP_CUDA(cudaMemcpy(h->d_x, X.data(), lay.b_x, cudaMemcpyHostToDevice),
                 "upload TDOA table");
        return SRP_OK;
    }
    SRP_CUDA(cudaMemcpy(h->d_xs, xs.data(), lay.b_xs, cudaMemcpyHostToDevice),
             "upload tensor-core TDOA table");
    // per chunk of 64 slots: pair; nmax_q - first slot as float bits (Nyquist)
    // or the chunk's first bin (conventional); 8-slot groups to generate
    // (even); 16-slot MMA steps holding data
    std::vector<int4> ctab(lay.n_chunks);
    const bool nyq = d->mode == SRP_MODE_NYQUIST;
    for (int q = 0; q < lay.Q; ++q) {
        const int nmax = lay.Nq[q] + lay.n_aux;
        const int span = nyq ? 2 * nmax + 1 : 2 * lay.Kb;
        for (int c0 = 0; c0 < span; c0 += kLagPad) {
            int32_t y;
            if (nyq) {
                const float moff = (float)(nmax - c0);
                memcpy(&y, &moff, sizeof y);
            } else {
                y = c0 / 2;  // first bin: two slots per bin
            }
            const int nk = (std::min(kLagPad, span - c0) + 15) / 16;
            ctab[(lay.offc[q] + c0) / kLagPad] = make_int4(q, y, 2 * nk, nk);
        }
    }
    SRP_CUDA(cudaMemcpy(h->d_ctab, ctab.data(), lay.b_ctab, cudaMemcpyHostToDevice),
             "upload chunk table");
    if (lay.tile_steps) {  // resident interpolation matrix: chunk offsets, then the weights
        std::vector<int32_t> woff(lay.n_chunks);  // -1: the chunk's weights are generated
        int32_t at = 0;
        for (int c = 0; c < lay.n_chunks; ++c) {
            woff[c] = lay.streamed[ctab[c].x] ? at : -1;
            if (woff[c] >= 0) at += ctab[c].w;
        }
        if (at != lay.tile_steps) return fail(SRP_ERR_UNSUPPORTED, "internal: step count");
        SRP_CUDA(cudaMemcpy(h->d_woff, woff.data(), lay.b_woff, cudaMemcpyHostToDevice),
                 "upload chunk offsets");
        SRP_CUDA(launch_build_w(h->d_xs, h->d_ctab, h->d_woff, lay.n_chunks, lay.J_pad, lay.xf,
                                lay.tile_steps, lay.n_tiles, h->precision, h->d_w, 0),
                 "interpolation matrix kernel");
    }
    return SRP_OK;
}

srp_status check_handle(srp_handle h) {
    if (h == nullptr) return fail(SRP_ERR_INVALID_ARG, "handle is NULL");
    return SRP_OK;
}

void record(srp_plan_s *h, int idx, cudaStream_t s) {
    if (h->timing) cudaEventRecord(h->ev[idx], s);
}

// The hot path: K2 + K3 (Nyquist) or K4 (conventional) -> K5; the CUDA-core
// engine runs K1 first on STFT input, the tensor-core operand kernels form the
// cross spectra themselves.
srp_status run_map(srp_plan_s *h, const void *d_in, int L, float *d_maps, int32_t *d_argmax,
                   float *d_peak, cudaStream_t s) {
    const Layout &lay = h->lay;
    int launches = 0;
    for (int &r : h->stage_ran) r = 0;
    record(h, 0, s);
    const float2 *psi = static_cast<const float2 *>(d_in);
    // The tensor-core operand kernels form the weighted cross spectra of STFT
    // input themselves; the CUDA-core engine runs K1 first.
    const bool from_y = lay.tc && h->input_kind == SRP_IN_STFT;
    if (h->input_kind == SRP_IN_STFT && !lay.tc) {
        SRP_CUDA(launch_phat(static_cast<const float2 *>(d_in), L, lay.M, lay.Kb, h->d_pairs,
                             lay.Q, h->weighting, h->d_psi, s), "cross-spectrum kernel");
        psi = h->d_psi;
        h->stage_ran[kStagePhat] = 1;
        ++launches;
    }
    record(h, 1, s);
    const int fmt = h->precision == SRP_PREC_FP32 ? 1 : (h->precision == SRP_PREC_FP16 ? 2 : 0);
    // FP32 re-scoring: per-tile keys instead of one raised key per frame, and
    // the FP32 operands kept beside the 16-bit ones (cross spectra formed from
    // STFT input go to d_psi; cross-spectrum input is read in place)
    unsigned long long *best = lay.rescore ? h->d_rs_fkey : h->d_part;
    float2 *psi32 = (lay.rescore && from_y) ? h->d_psi : nullptr;
    if (h->mode == SRP_MODE_CONV && lay.tc) {
        SRP_CUDA(launch_conv_operand_tc(psi, from_y, lay.M, h->d_pairs, h->weighting, L, lay.Q,
                                        lay.K, h->d_offc, h->d_xi16, lay.L_pad, lay.Sc, fmt,
                                        best, psi32, s), "conventional operand kernel");
        h->stage_ran[kStageGcc] = 1;
        ++launches;
    } else if (h->mode == SRP_MODE_NYQUIST && lay.gcc_mma) {
        SRP_CUDA(launch_gcc_samples_mma(h->gtw_map, psi, from_y, lay.M, h->weighting, L,
                                        lay.Q, lay.K, h->d_nq, h->d_offc,
                                        lay.n_aux, lay.nmax_all, h->d_xi16, lay.L_pad, lay.Sc,
                                        fmt, best, h->d_xi32, h->d_off, lay.S_pad, h->d_status,
                                        h->gcc_zmax, s),
                 "GCC sample kernel");
        h->stage_ran[kStageGcc] = 1;
        ++launches;
    } else if (h->mode == SRP_MODE_NYQUIST && lay.tc) {
        SRP_CUDA(launch_gcc_samples_tc(psi, from_y, lay.M, h->d_pairs, h->weighting, L, lay.Q,
                                       lay.K, h->d_nq, h->d_offc, lay.n_aux, h->d_twid,
                                       h->d_xi16, lay.L_pad, lay.Sc, fmt, best, h->d_xi32,
                                       h->d_off, lay.S_pad, s),
                 "GCC sample kernel");
        h->stage_ran[kStageGcc] = 1;
        ++launches;
    } else if (h->mode == SRP_MODE_NYQUIST) {
        SRP_CUDA(launch_gcc_samples(psi, L, lay.Q, lay.K, h->d_nq, h->d_off, lay.n_aux, h->d_twid,
                                    h->d_xi, lay.L_pad, 1, s), "GCC sample kernel");
        h->stage_ran[kStageGcc] = 1;
        ++launches;
    }
    record(h, 2, s);
    if (lay.tc) {
        SRP_CUDA(launch_interp_tc(h->xi_map, lay.N_tc, h->d_xs, h->d_ctab, lay.par1_used,
                                  lay.J_pad, lay.J, lay.Q, h->d_nq, lay.n_aux, lay.xf, lay.Sc,
                                  lay.L_pad, L, h->precision, h->mode == SRP_MODE_CONV ? 1 : 0,
                                  lay.K, d_maps, h->d_part, lay.n_tiles, h->d_status, h->d_w,
                                  h->d_woff, lay.tile_steps, lay.tile_steps == lay.total_steps,
                                  lay.rescore ? h->d_rs_fkey : nullptr, lay.promote, s),
                 "tensor-core map kernel");
    } else if (h->mode == SRP_MODE_NYQUIST) {
        SRP_CUDA(launch_interp_simt(h->d_x, lay.J_pad, lay.J, lay.Q, h->d_nq, h->d_off, lay.n_aux,
                                    lay.xf, h->d_xi, lay.L_pad, L, d_maps, h->d_part, lay.n_tiles,
                                    s), "interpolation kernel");
    } else {
        SRP_CUDA(launch_conv_simt(h->d_x, lay.J_pad, lay.J, lay.Q, lay.K, lay.xf, psi, L, d_maps,
                                  h->d_part, lay.n_tiles, s), "conventional kernel");
    }
    h->stage_ran[kStageMap] = 1;
    ++launches;
    record(h, 3, s);
    if (lay.rescore) {
        // the maximiser in FP32 among the tiles near the frame's maximum
        const float2 *psi_fp32 = from_y ? h->d_psi : static_cast<const float2 *>(d_in);
        SRP_CUDA(launch_rescore(h->mode == SRP_MODE_CONV, h->d_part, lay.n_tiles, lay.J,
                                lay.J_pad, lay.Q, h->d_xs, lay.xf, h->d_nq, h->d_off, lay.n_aux,
                                h->d_xi32, lay.S_pad, psi_fp32, lay.K, L, kRescoreDelta,
                                h->d_rs_fkey, h->d_rs_slots, h->d_rs_count, d_argmax, d_peak,
                                d_maps, s),
                 "argmax re-scoring kernel");
    } else {
        // tensor-core tiles raise one key per frame (d_part[0, L)); CUDA-core
        // tiles leave one key per (frame, tile)
        SRP_CUDA(launch_argmax(h->d_part, lay.tc ? 1 : lay.n_tiles, L, d_argmax, d_peak, s),
                 "argmax kernel");
    }
    h->stage_ran[kStageArgmax] = 1;
    ++launches;
    record(h, 4, s);
    h->last_launches = launches;
    h->last_L = L;
    return SRP_OK;
}

}  // namespace

srp_status describe_layout(const srp_plan_desc *d, Layout &lay) { return make_layout(d, lay); }

void set_error(const std::string &msg) { g_err = msg; }

srp_status fail(srp_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

srp_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SRP_ERR_OOM : SRP_ERR_CUDA;
}

}  // namespace srp

using namespace srp;

extern "C" {

srp_status srp_plan_describe(const srp_plan_desc *d, srp_plan_info *info, int32_t *Nq_out) {
    Layout lay;
    srp_status st = make_layout(d, lay);
    if (st != SRP_OK) return st;
    if (info != nullptr) fill_info(lay, info);
    if (Nq_out != nullptr) memcpy(Nq_out, lay.Nq.data(), sizeof(int32_t) * lay.Q);
    return SRP_OK;
}

srp_status srp_plan_complexity(const srp_plan_desc *d, srp_complexity *out) {
    if (out == nullptr) return fail(SRP_ERR_INVALID_ARG, "out is NULL");
    if (d == nullptr) return fail(SRP_ERR_INVALID_ARG, "descriptor is NULL");
    Layout lay;
    srp_status st = make_layout(d, lay);
    if (st != SRP_OK) return st;
    // Sec. 3.3: N averages the 2 N_q + 2 N_aux + 1 samples of each pair
    int64_t sum_nq = 0;
    for (int32_t v : lay.Nq) sum_nq += v;
    const double P = (double)lay.Q, Kb = (double)(d->K / 2), J = (double)d->J;
    memset(out, 0, sizeof *out);
    out->N = 2.0 * (double)sum_nq / P + 2.0 * (double)d->n_aux + 1.0;
    out->P = lay.Q;
    out->K_b = d->K / 2;
    out->J = d->J;
    out->C_samp = out->N * P * Kb;
    out->C_int = out->N * P * J;
    out->C_conv = J * P * Kb;
    out->R_samp = out->N / J;
    out->R_int = out->N / Kb;
    out->R = out->R_samp + out->R_int;
    return SRP_OK;
}

srp_status srp_plan_footprint(const srp_plan_desc *d, size_t *device_bytes) {
    if (device_bytes == nullptr) return fail(SRP_ERR_INVALID_ARG, "device_bytes is NULL");
    Layout lay;
    srp_status st = make_layout(d, lay);
    if (st != SRP_OK) return st;
    *device_bytes = lay.total();
    return SRP_OK;
}

srp_status srp_plan(const srp_plan_desc *d, srp_handle *out) {
    if (out == nullptr) return fail(SRP_ERR_INVALID_ARG, "out is NULL");
    Layout lay;
    srp_status st = make_layout(d, lay);
    if (st != SRP_OK) return st;
    if ((st = check_grid(d)) != SRP_OK) return st;
    srp_plan_s *h = new (std::nothrow) srp_plan_s();
    if (h == nullptr) return fail(SRP_ERR_OOM, "host allocation failed");
    h->lay = std::move(lay);
    h->mode = d->mode;
    h->precision = d->precision;
    h->input_kind = d->input_kind;
    h->weighting = d->weighting;
    h->host_io = d->host_io;
    h->fs = d->fs;
    h->c = d->c;
    h->grid_kind = d->grid_kind;
    const Layout &L = h->lay;
    auto bail = [&](srp_status s) {
        release(h);
        delete h;
        return s;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
#define SRP_ALLOC(ptr, bytes)                                            \
    do {                                                                 \
        cudaError_t e_ = dalloc(&(ptr), (bytes));                        \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, "cudaMalloc")); \
    } while (0)
    SRP_ALLOC(h->d_pairs, L.b_pairs);
    SRP_ALLOC(h->d_nq, L.b_nq);
    SRP_ALLOC(h->d_off, L.b_off);
    SRP_ALLOC(h->d_x, L.b_x);
    SRP_ALLOC(h->d_twid, L.b_twid);
    SRP_ALLOC(h->d_gtw, L.b_gtw);
    SRP_ALLOC(h->d_psi, L.b_psi);
    SRP_ALLOC(h->d_xi, L.b_xi);
    SRP_ALLOC(h->d_xi16, L.b_xi16);
    SRP_ALLOC(h->d_xi32, L.b_xi32);
    SRP_ALLOC(h->d_rs_fkey, L.b_rs);  // the slots and the counters follow the frame keys
    if (L.b_rs) {
        h->d_rs_slots = h->d_rs_fkey + L.L_pad;
        h->d_rs_count = reinterpret_cast<int *>(h->d_rs_slots + (size_t)L.L_pad * kRescoreCtas);
    }
    SRP_ALLOC(h->d_offc, L.b_offc);
    SRP_ALLOC(h->d_xs, L.b_xs);
    SRP_ALLOC(h->d_ctab, L.b_ctab);
    SRP_ALLOC(h->d_w, L.b_w);
    SRP_ALLOC(h->d_woff, L.b_woff);
    SRP_ALLOC(h->d_status, L.b_status);
    SRP_ALLOC(h->d_part, L.b_part);
    if (h->host_io) {
        h->n_slots = h->host_io;
        SRP_ALLOC(h->d_in_stage, L.b_in_stage);
        SRP_ALLOC(h->d_maps_stage, L.b_maps_stage);
        SRP_ALLOC(h->d_argmax_stage, L.b_small_stage / 2);
        SRP_ALLOC(h->d_peak_stage, L.b_small_stage / 2);
    }
    if (h->n_slots == 2) {
        if ((e = cudaStreamCreateWithFlags(&h->io_in, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&h->io_out, cudaStreamNonBlocking)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaStreamCreate"));
        for (int k = 0; k < 2; ++k)
            if ((e = cudaEventCreateWithFlags(&h->ev_in[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h->ev_done[k], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&h->ev_out[k], cudaEventDisableTiming)) != cudaSuccess)
                return bail(cuda_fail(e, "cudaEventCreate"));
    }
#undef SRP_ALLOC
    std::vector<int2> pairs(L.Q);
    for (int q = 0; q < L.Q; ++q) pairs[q] = make_int2(L.pm[q], L.pmp[q]);
    auto up = [&](void *dst, const void *src, size_t n) -> cudaError_t {
        return n ? cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    if ((e = up(h->d_pairs, pairs.data(), L.b_pairs)) != cudaSuccess ||
        (e = up(h->d_nq, L.Nq.data(), L.b_nq)) != cudaSuccess ||
        (e = up(h->d_off, L.off.data(), L.b_off)) != cudaSuccess ||
        (e = up(h->d_offc, L.offc.data(), L.b_offc)) != cudaSuccess ||
        (e = cudaMemset(h->d_status, 0, L.b_status)) != cudaSuccess ||
        (L.b_rs && (e = cudaMemset(h->d_rs_fkey, 0, L.b_rs)) != cudaSuccess))
        return bail(cuda_fail(e, "upload pair tables"));
    if (L.b_twid) {
        std::vector<float2> tw(L.K);
        const double two_pi = 6.283185307179586476925286766559;
        for (int j = 0; j < L.K; ++j)
            tw[j] = make_float2((float)cos(two_pi * j / L.K), (float)sin(two_pi * j / L.K));
        if ((e = up(h->d_twid, tw.data(), L.b_twid)) != cudaSuccess)
            return bail(cuda_fail(e, "upload twiddles"));
    }
    if (L.b_gtw) {
        if ((e = gcc_mma_twiddles(L.K, L.nmax_all, h->d_gtw, h->gtw_map)) != cudaSuccess)
            return bail(cuda_fail(e, "tensor-core IDFT twiddles"));
        const int fmt = h->precision == SRP_PREC_FP32 ? 1 : (h->precision == SRP_PREC_FP16 ? 2 : 0);
        if ((h->gcc_zmax = gcc_mma_setup(L.K, L.nmax_all, fmt)) == 0)
            return bail(cuda_fail(cudaErrorInvalidValue, "tensor-core IDFT set-up"));
    }
    // Padding rows and frames of the GCC-sample buffers stay zero for ever.
    if (L.b_xi && (e = cudaMemset(h->d_xi, 0, L.b_xi)) != cudaSuccess)
        return bail(cuda_fail(e, "clear GCC buffer"));
    if (L.b_xi16 && (e = cudaMemset(h->d_xi16, 0, L.b_xi16)) != cudaSuccess)
        return bail(cuda_fail(e, "clear GCC buffer"));
    if (L.tc) {
        const int rows = (h->precision == SRP_PREC_FP32 ? 2 : 1) * L.L_pad;
        if ((e = encode_xi_map(h->d_xi16, rows, L.Sc, L.N_tc, h->xi_map)) != cudaSuccess)
            return bail(cuda_fail(e, "cuTensorMapEncodeTiled"));
    }
    if ((st = build_tdoa(d, h)) != SRP_OK) return bail(st);
    for (auto &ev : h->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(e, "plan upload"));
    *out = h;
    return SRP_OK;
}

srp_status srp_plan_get_info(srp_handle h, srp_plan_info *info) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (info == nullptr) return fail(SRP_ERR_INVALID_ARG, "info is NULL");
    fill_info(h->lay, info);
    return SRP_OK;
}

srp_status srp_plan_tdoa(srp_handle h, double *x_host) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (x_host == nullptr) return fail(SRP_ERR_INVALID_ARG, "x_host is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    const Layout &L = h->lay;
    std::vector<int32_t> X((size_t)L.Q * L.J_pad);
    if (L.tc) {
        std::vector<int2> xs((size_t)L.Q * L.J_pad);
        SRP_CUDA(cudaMemcpy(xs.data(), h->d_xs, L.b_xs, cudaMemcpyDeviceToHost),
                 "download TDOA table");
        for (size_t k = 0; k < xs.size(); ++k) X[k] = xs[k].x;
    } else {
        SRP_CUDA(cudaMemcpy(X.data(), h->d_x, L.b_x, cudaMemcpyDeviceToHost),
                 "download TDOA table");
    }
    const double inv = ldexp(1.0, -L.xf);
    for (int64_t i = 0; i < L.J; ++i)
        for (int q = 0; q < L.Q; ++q) x_host[i * L.Q + q] = X[(size_t)q * L.J_pad + i] * inv;
    return SRP_OK;
}

srp_status srp_map(srp_handle h, const void *d_in, int32_t L, float *d_maps, int32_t *d_argmax,
                   float *d_peak, srp_stream_t s) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (L < 0 || L > h->lay.L_max) return fail(SRP_ERR_INVALID_ARG, "L out of [0, max_frames]");
    if (L == 0) return SRP_OK;
    if (d_in == nullptr || d_argmax == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "d_in and d_argmax must be non-NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    return run_map(h, d_in, L, d_maps, d_argmax, d_peak, reinterpret_cast<cudaStream_t>(s));
}

// Device address of a pinned (page-locked or registered) host buffer on a
// GPU that reaches host memory coherently (NVLink-C2C, host page tables), or
// null: the map kernel then stores the maps straight into the caller's buffer
// instead of into a device staging buffer followed by a copy.
static float *direct_host_maps(int device, float *h_maps) {
    if (h_maps == nullptr) return nullptr;
    int coherent = 0;
    if (cudaDeviceGetAttribute(&coherent, cudaDevAttrPageableMemoryAccessUsesHostPageTables,
                               device) != cudaSuccess || !coherent) {
        cudaGetLastError();
        return nullptr;
    }
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h_maps) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
    return static_cast<float *>(at.devicePointer);
}

srp_status srp_map_host(srp_handle h, const void *h_in, int32_t L, float *h_maps,
                        int32_t *h_argmax, float *h_peak, srp_stream_t s) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (!h->host_io) return fail(SRP_ERR_INVALID_ARG, "plan was built without host_io");
    if (L < 0 || L > h->lay.L_max) return fail(SRP_ERR_INVALID_ARG, "L out of [0, max_frames]");
    if (L == 0) return SRP_OK;
    if (h_in == nullptr || h_argmax == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "h_in and h_argmax must be non-NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    const Layout &lay = h->lay;
    const int rows = h->input_kind == SRP_IN_STFT ? lay.M : lay.Q;
    const size_t in_bytes = sizeof(float2) * (size_t)L * rows * lay.Kb;
    SRP_CUDA(cudaMemcpyAsync(h->d_in_stage, h_in, in_bytes, cudaMemcpyHostToDevice, cs),
             "copy input to device");
    float *direct = direct_host_maps(h->device, h_maps);
    st = run_map(h, h->d_in_stage, L, h_maps ? (direct ? direct : h->d_maps_stage) : nullptr,
                 h->d_argmax_stage, h->d_peak_stage, cs);  // slot 0
    if (st != SRP_OK) return st;
    if (h_maps && !direct)
        SRP_CUDA(cudaMemcpyAsync(h_maps, h->d_maps_stage, sizeof(float) * (size_t)L * lay.J,
                                 cudaMemcpyDeviceToHost, cs), "copy maps to host");
    SRP_CUDA(cudaMemcpyAsync(h_argmax, h->d_argmax_stage, sizeof(int32_t) * L,
                             cudaMemcpyDeviceToHost, cs), "copy argmax to host");
    if (h_peak)
        SRP_CUDA(cudaMemcpyAsync(h_peak, h->d_peak_stage, sizeof(float) * L,
                                 cudaMemcpyDeviceToHost, cs), "copy peak to host");
    SRP_CUDA(cudaStreamSynchronize(cs), "synchronise stream");
    return srp_poll_device_status(h, s);
}

// Byte offsets of staging slot k (see make_layout: slots are 256-byte aligned).
struct SlotPtrs {
    char *in;
    float *maps;
    int32_t *argmax;
    float *peak;
};

static SlotPtrs slot_ptrs(srp_plan_s *h, int k) {
    const Layout &lay = h->lay;
    const size_t n = (size_t)h->n_slots;
    SlotPtrs p;
    p.in = static_cast<char *>(h->d_in_stage) + k * (lay.b_in_stage / n);
    p.maps = reinterpret_cast<float *>(reinterpret_cast<char *>(h->d_maps_stage) +
                                       k * (lay.b_maps_stage / n));
    p.argmax = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(h->d_argmax_stage) +
                                           k * (lay.b_small_stage / 2 / n));
    p.peak = reinterpret_cast<float *>(reinterpret_cast<char *>(h->d_peak_stage) +
                                       k * (lay.b_small_stage / 2 / n));
    return p;
}

srp_status srp_map_host_async(srp_handle h, const void *h_in, int32_t L, float *h_maps,
                              int32_t *h_argmax, float *h_peak, srp_stream_t s) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (h->n_slots != 2) return fail(SRP_ERR_INVALID_ARG, "plan was not built with host_io = 2");
    if (L < 0 || L > h->lay.L_max) return fail(SRP_ERR_INVALID_ARG, "L out of [0, max_frames]");
    if (L == 0) return SRP_OK;
    if (h_in == nullptr || h_argmax == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "h_in and h_argmax must be non-NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    const Layout &lay = h->lay;
    const int k = h->next_slot;
    h->next_slot ^= 1;
    const SlotPtrs sp = slot_ptrs(h, k);
    const int rows = h->input_kind == SRP_IN_STFT ? lay.M : lay.Q;
    const size_t in_bytes = sizeof(float2) * (size_t)L * rows * lay.Kb;
    // input: once the slot's previous map has read it
    SRP_CUDA(cudaStreamWaitEvent(h->io_in, h->ev_done[k], 0), "order input copy");
    SRP_CUDA(cudaMemcpyAsync(sp.in, h_in, in_bytes, cudaMemcpyHostToDevice, h->io_in),
             "copy input to device");
    SRP_CUDA(cudaEventRecord(h->ev_in[k], h->io_in), "record input copy");
    // map: once the input is in and the slot's previous results have left
    SRP_CUDA(cudaStreamWaitEvent(cs, h->ev_in[k], 0), "order map");
    SRP_CUDA(cudaStreamWaitEvent(cs, h->ev_out[k], 0), "order map");
    // (the maps go through the staging slot and a copy even into pinned
    // buffers: stores from the map kernel to host memory would hold the next
    // step's map back, while the copy overlaps it)
    st = run_map(h, sp.in, L, h_maps ? sp.maps : nullptr, sp.argmax, sp.peak, cs);
    if (st != SRP_OK) return st;
    SRP_CUDA(cudaEventRecord(h->ev_done[k], cs), "record map");
    // results
    SRP_CUDA(cudaStreamWaitEvent(h->io_out, h->ev_done[k], 0), "order result copy");
    if (h_maps)
        SRP_CUDA(cudaMemcpyAsync(h_maps, sp.maps, sizeof(float) * (size_t)L * lay.J,
                                 cudaMemcpyDeviceToHost, h->io_out), "copy maps to host");
    SRP_CUDA(cudaMemcpyAsync(h_argmax, sp.argmax, sizeof(int32_t) * L, cudaMemcpyDeviceToHost,
                             h->io_out), "copy argmax to host");
    if (h_peak)
        SRP_CUDA(cudaMemcpyAsync(h_peak, sp.peak, sizeof(float) * L, cudaMemcpyDeviceToHost,
                                 h->io_out), "copy peak to host");
    SRP_CUDA(cudaEventRecord(h->ev_out[k], h->io_out), "record result copy");
    return SRP_OK;
}

srp_status srp_map_host_wait(srp_handle h) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (h->n_slots != 2) return fail(SRP_ERR_INVALID_ARG, "plan was not built with host_io = 2");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    SRP_CUDA(cudaStreamSynchronize(h->io_out), "wait for results");
    return srp_poll_device_status(h, reinterpret_cast<srp_stream_t>(h->io_out));
}

srp_status srp_poll_device_status(srp_handle h, srp_stream_t s) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    int flags = 0;
    SRP_CUDA(cudaMemcpyAsync(&flags, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, cs),
             "read device status");
    SRP_CUDA(cudaMemsetAsync(h->d_status, 0, sizeof(int), cs), "clear device status");
    SRP_CUDA(cudaStreamSynchronize(cs), "synchronise stream");
    if (flags & 1) return fail(SRP_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel gave up");
    if (flags & 2) return fail(SRP_ERR_INVALID_ARG, "a refinement centre index was outside [0, J)");
    return SRP_OK;
}

srp_status srp_cross_spectra(srp_handle h, const void *d_y, int32_t L, void *d_psi,
                             srp_stream_t s) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (h->input_kind != SRP_IN_STFT) return fail(SRP_ERR_INVALID_ARG, "plan takes cross spectra");
    if (L < 0 || L > h->lay.L_max) return fail(SRP_ERR_INVALID_ARG, "L out of [0, max_frames]");
    if (L == 0) return SRP_OK;
    if (d_y == nullptr || d_psi == nullptr) return fail(SRP_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    const Layout &lay = h->lay;
    SRP_CUDA(launch_phat(static_cast<const float2 *>(d_y), L, lay.M, lay.Kb, h->d_pairs, lay.Q,
                         h->weighting, static_cast<float2 *>(d_psi),
                         reinterpret_cast<cudaStream_t>(s)),
             "cross-spectrum kernel");
    return SRP_OK;
}

srp_status srp_gcc_samples(srp_handle h, const void *d_in, int32_t L, float *d_xi,
                           srp_stream_t s) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (h->mode != SRP_MODE_NYQUIST) return fail(SRP_ERR_INVALID_ARG, "plan is conventional");
    if (L < 0 || L > h->lay.L_max) return fail(SRP_ERR_INVALID_ARG, "L out of [0, max_frames]");
    if (L == 0) return SRP_OK;
    if (d_in == nullptr || d_xi == nullptr) return fail(SRP_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    const Layout &lay = h->lay;
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    const float2 *psi = static_cast<const float2 *>(d_in);
    if (h->input_kind == SRP_IN_STFT) {
        SRP_CUDA(launch_phat(psi, L, lay.M, lay.Kb, h->d_pairs, lay.Q, h->weighting, h->d_psi, cs),
                 "PHAT kernel");
        psi = h->d_psi;
    }
    SRP_CUDA(launch_gcc_samples(psi, L, lay.Q, lay.K, h->d_nq, h->d_off, lay.n_aux, h->d_twid,
                                d_xi, 1, lay.S, cs), "GCC sample kernel");
    return SRP_OK;
}

srp_status srp_set_timing(srp_handle h, int32_t enable) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    h->timing = enable != 0;
    return SRP_OK;
}

srp_status srp_stage_times(srp_handle h, float *ms, int32_t n) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (ms == nullptr || n < 0) return fail(SRP_ERR_INVALID_ARG, "bad output buffer");
    if (!h->timing) return fail(SRP_ERR_INVALID_ARG, "timing is disabled");
    DeviceGuard g(h->device);
    SRP_CUDA(cudaEventSynchronize(h->ev[kNumStages]), "wait for timing events");
    for (int k = 0; k < n; ++k) {
        ms[k] = 0.0f;
        if (k < kNumStages && h->stage_ran[k])
            SRP_CUDA(cudaEventElapsedTime(&ms[k], h->ev[k], h->ev[k + 1]), "event elapsed time");
    }
    return SRP_OK;
}

srp_status srp_last_launch_count(srp_handle h, int32_t *n) {
    srp_status st = check_handle(h);
    if (st != SRP_OK) return st;
    if (n == nullptr) return fail(SRP_ERR_INVALID_ARG, "n is NULL");
    *n = h->last_launches;
    return SRP_OK;
}

srp_status srp_destroy(srp_handle h) {
    if (h == nullptr) return SRP_OK;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    release(h);
    delete h;
    return SRP_OK;
}

const char *srp_status_string(srp_status s) {
    switch (s) {
        case SRP_OK: return "ok";
        case SRP_ERR_INVALID_ARG: return "invalid argument";
        case SRP_ERR_OOM: return "out of memory";
        case SRP_ERR_CUDA: return "CUDA error";
        case SRP_ERR_UNSUPPORTED: return "unsupported";
        case SRP_ERR_TIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char *srp_last_error_message(void) { return g_err.c_str(); }

}  // extern "C"
