// Internal declarations shared by the host planner (srp_api.cu) and the
// kernels (srp_kernels.cu, srp_tc.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/srp.h"

namespace srp {

// Candidate tile of every map kernel: one CTA owns 128 consecutive candidates.
constexpr int kTileJ = 128;
// Frame granularity of the GCC-sample buffer (rows of xi are padded to it).
constexpr int kFramePad = 16;
// Lag granularity of the GCC-sample buffer (the tensor-core K step).
constexpr int kLagPad = 64;
// Stages reported by srp_stage_times.
enum Stage { kStagePhat = 0, kStageGcc = 1, kStageMap = 2, kStageArgmax = 3, kNumStages = 4 };

// Host-side sizes of a plan; shared by describe / footprint / plan.
// FP32 accumulation in TMEM carries a systematic relative bias of about
// kTcAccumBias per MMA accumulated into one accumulator (measured on GB300);
// FP32 tensor-core paths keep that bias below kTcBiasLimit, half of the 1e-4
// tolerance of the FP32 maps.
constexpr double kTcAccumBias = 1.5e-8;
constexpr double kTcBiasLimit = 5e-5;
// Chunks per accumulator epoch of promoted FP32 conventional plans:
// 128 * 6 * kTcAccumBias = 1.15e-5 <= kTcBiasLimit / 4.
constexpr int kPromoteChunks = 128;
static_assert(kPromoteChunks * 6 * kTcAccumBias <= kTcBiasLimit / 4, "promotion epoch too long");
// FP32 re-scoring of reduced-precision maps: tiles whose maximum lies within
// kRescoreDelta |max| of the frame's maximum are evaluated again in FP32;
// twice the 1e-2 x peak error bound of BF16/FP16 maps.
constexpr float kRescoreDelta = 2e-2f;
// At most this many tiles per frame are re-scored (more: a nearly flat map,
// which keeps its reduced-precision maximiser).
constexpr int kRescoreMaxTiles = 64;
// CTAs per frame that share the re-scoring of its candidates (at most).
constexpr int kRescoreCtas = 16;

struct Layout {
    int M = 0, Q = 0, K = 0, Kb = 0, n_aux = 0, S = 0, S_pad = 0, max_nq = 0, xf = 0;
    int64_t J = 0, J_pad = 0;
    int L_max = 0, L_pad = 0, n_tiles = 0;
    std::vector<int32_t> Nq, off, pm, pmp;  // per pair
    // tensor-core lag layout: pair q owns ceil(N'_q / 64) chunks of 64 slots
    int Sc = 0, n_chunks = 0, N_tc = 0;
    int par1_used = 0;  // the tile has two or more 16-slot MMA steps (both accumulators written)
    int mma_steps = 0;   // tensor-core plans: 16-slot MMA steps per tile over all pairs
    int tile_steps = 0;  // resident interpolation matrix: 16-slot steps per tile (0: generated)
    int promote = 0;     // FP32 conventional on tensor cores: chunks per accumulator epoch (0: none)
    int total_steps = 0; // 16-slot steps holding lags, per tile, of all pairs (resident plans)
    std::vector<char> streamed;  // per pair: its weights are resident and streamed
    bool tc = false;    // the Nyquist map runs on the tensor cores
    bool rescore = false;  // reduced-precision tensor-core plan choosing its maximiser in FP32
    bool gcc_mma = false;  // Nyquist tensor-core plan: GCC samples by the tensor-core IDFT
    int nmax_all = 0;      // largest N_q + N_aux (the IDFT's lag columns)
    std::vector<int32_t> offc;
    // byte counts of every device buffer, in allocation order
    size_t b_status = 0, b_offc = 0, b_xs = 0, b_ctab = 0, b_w = 0, b_woff = 0;
    size_t b_pairs = 0, b_nq = 0, b_off = 0, b_x = 0, b_twid = 0, b_psi = 0, b_xi = 0,
           b_xi16 = 0, b_xi32 = 0, b_rs = 0, b_part = 0, b_in_stage = 0, b_maps_stage = 0,
           b_small_stage = 0, b_gtw = 0;
    size_t total() const {
        return b_status + b_offc + b_xs + b_ctab + b_w + b_woff + b_pairs + b_nq + b_off + b_x +
               b_twid + b_psi + b_xi + b_xi16 + b_xi32 + b_rs + b_part + b_in_stage +
               b_maps_stage + b_small_stage + b_gtw;
    }
};

}  // namespace srp

struct srp_plan_s {
    int device = 0;
    srp_mode mode = SRP_MODE_NYQUIST;
    srp_precision precision = SRP_PREC_FP32;
    srp_input_kind input_kind = SRP_IN_STFT;
    srp_weighting weighting = SRP_WEIGHT_PHAT;
    int host_io = 0;
    double fs = 0.0, c = 0.0;      // sampling rate and speed of sound of the descriptor
    srp_grid_kind grid_kind = SRP_GRID_POINTS;
    int last_L = 0;                // frames of the last map whose GCC samples the plan holds
    srp::Layout lay;
    // device tables (owned)
    int2 *d_pairs = nullptr;       // [Q] (m, m')
    int32_t *d_nq = nullptr;       // [Q] N_q
    int32_t *d_off = nullptr;      // [Q] first GCC-sample row of pair q
    int32_t *d_x = nullptr;        // [Q][J_pad] TDOA in samples, fixed point with xf fraction bits
    float2 *d_twid = nullptr;      // [K] (cos, sin)(2 pi j / K)
    uint16_t *d_gtw = nullptr;     // [2][N][K] the tensor-core IDFT's twiddle operand (hi, lo)
    alignas(64) unsigned char gtw_map[128] = {};  // CUtensorMap of d_gtw
    int gcc_zmax = 0;              // cluster size limit of the tensor-core IDFT
    // scratch (owned)
    float2 *d_psi = nullptr;       // [L_max][Q][Kb] cross spectra (STFT input only)
    float *d_xi = nullptr;         // [S_pad][L_pad] GCC samples, frames contiguous
    uint16_t *d_xi16 = nullptr;    // [1 or 2][L_pad][Sc] sign-folded GCC samples, 16-bit
    float *d_xi32 = nullptr;       // [L_pad][S_pad] FP32 GCC samples (Nyquist FP32 re-scoring)
    // FP32 re-scoring, one allocation: the frames' largest reduced-precision
    // keys, per (frame, CTA) best keys, per-frame arrival counters
    unsigned long long *d_rs_fkey = nullptr;   // [L_pad]
    unsigned long long *d_rs_slots = nullptr;  // [L_pad][kRescoreCtas]
    int *d_rs_count = nullptr;                 // [L_pad], zero between calls
    int32_t *d_offc = nullptr;     // [Q] first 16-bit lag slot of pair q (a multiple of 64)
    int2 *d_xs = nullptr;          // [Q][J_pad] (fixed-point TDOA, bits of (-1)^x0 sin(pi f)/pi)
    void *d_w = nullptr;           // resident interpolation matrix (resident_weights plans)
    int32_t *d_woff = nullptr;     // [n_chunks] first 16-slot step of each chunk in a tile
    int4 *d_ctab = nullptr;        // [n_chunks] (pair, bits of nmax - first slot, groups, MMA steps)
    int *d_status = nullptr;       // device error flags (bit 0: a bounded wait gave up)
    alignas(64) unsigned char xi_map[128] = {};  // CUtensorMap of d_xi16
    // argmax keys, [L_pad][n_tiles]: one per (frame, tile) on the CUDA-core
    // engine; the tensor-core engine uses the first L, one per frame
    unsigned long long *d_part = nullptr;
    // staging for srp_map_host (slot 0) and srp_map_host_async (slots 0, 1)
    // (owned, optional): n_slots consecutive slots per buffer
    int n_slots = 0;
    void *d_in_stage = nullptr;
    float *d_maps_stage = nullptr;
    int32_t *d_argmax_stage = nullptr;
    float *d_peak_stage = nullptr;
    cudaStream_t io_in = nullptr, io_out = nullptr;  // copy streams of srp_map_host_async
    cudaEvent_t ev_in[2] = {}, ev_done[2] = {}, ev_out[2] = {};
    int next_slot = 0;
    // timing
    int timing = 0;
    cudaEvent_t ev[srp::kNumStages + 1] = {};
    int stage_ran[srp::kNumStages] = {};
    int last_launches = 0;
};

namespace srp {

// Validate a descriptor and compute its layout (host only), as srp_plan does.
srp_status describe_layout(const srp_plan_desc *d, Layout &lay);

void set_error(const std::string &msg);
// Record msg (or the CUDA error text) for srp_last_error_message; return the status.
srp_status fail(srp_status st, const std::string &msg);
srp_status cuda_fail(cudaError_t e, const char *what);

#define SRP_CUDA(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return srp::cuda_fail(e_, (what)); \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---- kernel launchers (srp_kernels.cu); each returns cudaGetLastError() ----
cudaError_t launch_phat(const float2 *y, int L, int M, int Kb, const int2 *pairs, int Q,
                        int weighting, float2 *psi, cudaStream_t s);
cudaError_t launch_gcc_samples(const float2 *psi, int L, int Q, int K, const int32_t *nq,
                               const int32_t *off, int n_aux, const float2 *twid, float *xi,
                               int64_t s_stride, int64_t l_stride, cudaStream_t s);
cudaError_t launch_interp_simt(const int32_t *x, int64_t J_pad, int64_t J, int Q,
                               const int32_t *nq, const int32_t *off, int n_aux, int xf,
                               const float *xi, int L_pad, int L, float *maps,
                               unsigned long long *part, int n_tiles, cudaStream_t s);
cudaError_t launch_conv_simt(const int32_t *x, int64_t J_pad, int64_t J, int Q, int K, int xf,
                             const float2 *psi, int L, float *maps, unsigned long long *part,
                             int n_tiles, cudaStream_t s);
cudaError_t encode_xi_map(void *xi16, int rows, int S_pad, int N, void *map_out);
// Tensor-core operand kernels: src is the cross spectra psi[L][Q][Kb], or with
// from_y the STFT frames y[L][M][Kb] (the weighted cross spectra are formed
// in the kernel).  best (nullable): the L per-frame argmax keys, cleared here.
// xi32 (nullable): the FP32 samples too, [L_pad][S32] at the pair offsets off.
cudaError_t launch_gcc_samples_tc(const float2 *src, bool from_y, int M, const int2 *pairs,
                                  int weighting, int L, int Q, int K, const int32_t *nq,
                                  const int32_t *offc, int n_aux, const float2 *twid,
                                  uint16_t *xi16, int L_pad, int S_pad, int fmt,
                                  unsigned long long *best, float *xi32, const int32_t *off,
                                  int S32, cudaStream_t s);
// The same samples by the tensor-core inverse DFT (srp_gcc_mma.cu), for
// PHAT-weighted STFT input (pairs in the plan's enumeration: m' outer, m > m'
// inner), K a multiple of 64 and 2 nmax + 1 <= 128 lag columns (nmax: the
// largest N_q + N_aux): gcc_mma_fits tells whether the shape qualifies, and
// gcc_mma_twiddles writes its twiddle operand (gcc_mma_twiddle_bytes) and
// the operand's tensor map at plan time.
bool gcc_mma_fits(int K, int nmax);
// Plan time: set the kernel's attributes for output format fmt (0 bf16, 1
// bf16 split, 2 fp16) and return the cluster size limit the launches use
// (16 where the GPU can place such a cluster, else 8; 0 on failure).
int gcc_mma_setup(int K, int nmax, int fmt);
size_t gcc_mma_twiddle_bytes(int K, int nmax);
cudaError_t gcc_mma_twiddles(int K, int nmax, uint16_t *d_tw, void *map_out);
cudaError_t launch_gcc_samples_mma(const void *tw_map, const float2 *src, bool from_y, int M,
                                   int weighting, int L, int Q, int K,
                                   const int32_t *nq, const int32_t *offc, int n_aux, int nmax,
                                   uint16_t *xi16, int L_pad, int S_pad, int fmt,
                                   unsigned long long *best, float *xi32, const int32_t *off,
                                   int S32, int *status, int zmax, cudaStream_t s);
int interp_tc_frames_per_cta(int L);
// frame_keys (nullable, for the FP32 re-scoring): every tile writes its key
// per frame to part[l][tile] and raises frame_keys[l] (cleared by the operand
// kernel), instead of raising part[l].
cudaError_t launch_interp_tc(const void *xi_map, int N, const int2 *xs, const int4 *ctab,
                             int par1_used, int64_t J_pad, int64_t J, int Q, const int32_t *nq,
                             int n_aux, int xf, int S_pad, int L_pad, int L, int precision,
                             int conv, int K, float *maps, unsigned long long *part, int n_tiles,
                             int *status, const void *w, const int32_t *woff, int tile_steps,
                             int all_streamed, unsigned long long *frame_keys, int promote,
                             cudaStream_t s);
// Plan time: the resident interpolation matrix (operand A) of every tile.
cudaError_t launch_build_w(const int2 *xs, const int4 *ctab, const int32_t *woff, int n_chunks,
                           int64_t J_pad, int xf, int tile_steps, int n_tiles, int precision,
                           void *w, cudaStream_t s);
// psi32 (nullable): the weighted cross spectra [L][Q][Kb] in FP32 too.
cudaError_t launch_conv_operand_tc(const float2 *src, bool from_y, int M, const int2 *pairs,
                                   int weighting, int L, int Q, int K, const int32_t *offc,
                                   uint16_t *b16, int L_pad, int S_pad, int fmt,
                                   unsigned long long *best, float2 *psi32, cudaStream_t s);
// FP32 re-scoring of reduced-precision maps (srp_rescore.cu): per frame, the
// tiles whose key is within delta |max| of the frame's largest key are
// evaluated again in FP32, candidate by candidate: Nyquist from xi32
// [L_pad][S32] (off, nq, n_aux), conventional from psi [L][Q][Kb] (the
// weighted cross spectra, a_k / K applied here).  Writes argmax and peak.
cudaError_t launch_rescore(bool conv, const unsigned long long *part, int n_tiles, int64_t J,
                           int64_t J_pad, int Q, const int2 *xs, int xf, const int32_t *nq,
                           const int32_t *off, int n_aux, const float *xi32, int S32,
                           const float2 *psi, int K, int L, float delta,
                           const unsigned long long *fkey, unsigned long long *slots, int *count,
                           int32_t *argmax, float *peak, const float *maps, cudaStream_t s);
cudaError_t launch_argmax(const unsigned long long *part, int n_tiles, int L, int32_t *argmax,
                          float *peak, cudaStream_t s);

}  // namespace srp
