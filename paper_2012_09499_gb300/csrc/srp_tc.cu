// Tensor-core (tcgen05 / TMEM / TMA) kernels of the SRP map:
//   k_gcc_samples_tc  critical GCC samples (Eq. GCC_IFT at tau = nT) as 16-bit
//                     operands, sign-folded and split for the FP32 path
//   k_conv_operand_tc (a_k/K)(Re psi, Im psi) as 16-bit operands for the
//                     conventional map (Eq. GCC_IFT at every TDOA, Sec. 2.4)
//   k_interp_tc       map[l][i] = sum_q sum_n xi_q(n) sinc(x_iq - n)
//                     (Eq. SRPapprox summed over pairs, Eq. SRP_T_IFT) as one
//                     (J x S) x (S x L) contraction with the pair sum as the
//                     reduction axis, accumulated in TMEM; the epilogue
//                     writes the maps and raises each frame's argmax key
//                     (atomicMax over the candidate tiles).
//
// Operand A (sinc weights) is generated on chip.  With x = x0 + f,
//   sinc(x - n) = (-1)^n * [(-1)^x0 sin(pi f) / pi] / (f + x0 - n),
// so (-1)^n moves into the GCC samples (B) and A[i][s] = sp_iq / d with
// sp_iq = (-1)^x0 sin(pi f)/pi and d = f + x0 - n.  Two neighbouring lags
// share one reciprocal: 1/da = db / (da db).  f = 0 (an exact sample) is
// evaluated as f = 2^-40, which gives the unit weight at n = x0 and weights
// below 1e-11 elsewhere.
//
// Lag axis: pair q owns ceil((2(N_q+N_aux)+1)/64) chunks of 64 lag slots
// (one 128-byte swizzle row of 16-bit data), so every pipeline stage holds one
// pair; the slots past the pair's last lag have B = 0.  A plan table gives
// each chunk its pair, its first lag, the 8-lag groups to generate and the
// 16-lag MMA steps to issue (trailing empty steps are skipped).  The plan also
// holds, per (pair, candidate), the fixed-point TDOA and sp = (-1)^x0
// sin(pi f)/pi computed in FP64, so no sine is evaluated here.
//
// The same kernel (kConv) computes the conventional map as the contraction of
// the steering matrix [cos theta, -sin theta], theta = 2 pi k x_iq / K, with
// (a_k/K)(Re psi, Im psi) over (pair, bin, re/im): each thread seeds
// e^{-j theta} exactly every 32 bins (phase ((k x0 mod K) + k f)/K) and
// rotates by e^{-j 2 pi x / K} in between.
//
// FP32 precision uses three BF16 products per step (A_hi B_hi + A_hi B_lo +
// A_lo B_hi, hi = bf16(v), lo = bf16(v - hi)); BF16 and FP16 precision use one.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "srp_device.cuh"
#include "srp_internal.h"
#include "srp_tc_common.cuh"

namespace srp {
namespace {

using namespace dev;
using namespace tc;

// ---------------------------------------------------------------------------
// GCC samples as 16-bit operand B: xi'[row][slot], row = frame (hi) or
// L_pad + frame (lo), slot = offc[q] + t, value (-1)^n xi_q(n).  With kFromY
// the row's cross spectrum is formed here from the STFT frames (the weighted
// y_m conj(y_m') of K1, the same arithmetic), so K1 and its round trip
// through the cross-spectrum scratch are skipped.  CTA (0, 0) also clears
// the per-frame argmax keys that the map kernel's tiles raise with atomicMax.
// ---------------------------------------------------------------------------
// With xi32 the FP32 samples xi_q(n) (not sign-folded) also go to
// xi32[frame][off[q] + t], for the FP32 re-scoring of the maximiser.
template <int kFmt, bool kFromY>  // kFmt 0: bf16, 1: bf16 hi/lo split, 2: fp16
__global__ void __launch_bounds__(128, 12) k_gcc_samples_tc(
    const float2 *__restrict__ src, int M, const int2 *__restrict__ pairs, int weighting, int Q,
    int K, const int32_t *__restrict__ nq, const int32_t *__restrict__ offc, int n_aux,
    const float2 *__restrict__ twid, uint16_t *__restrict__ xi16, int L_pad, int S_pad,
    unsigned long long *__restrict__ best, float *__restrict__ xi32,
    const int32_t *__restrict__ off, int S32) {
    extern __shared__ float2 sm[];
    float2 *tw = sm, *ps = sm + K;
    const int q = blockIdx.x, l = blockIdx.y, Kb = K / 2 + 1;
    grid_dep_launch();  // the map kernel may start its prologue now
    if (best != nullptr && q == 0 && l == 0)
        for (int i = threadIdx.x; i < (int)gridDim.y; i += blockDim.x) best[i] = 0ull;
    if (kFromY) {
        const int2 p = pairs[q];
        const float2 *ym = src + ((size_t)l * M + p.x) * Kb, *yn = src + ((size_t)l * M + p.y) * Kb;
        copy_twiddles_async(twid, K, tw);
        const int nt = blockDim.x;
        for (int k0 = threadIdx.x; k0 < Kb; k0 += kStageUnroll * nt) {
            float2 a[kStageUnroll], b[kStageUnroll];
#pragma unroll
            for (int u = 0; u < kStageUnroll; ++u)
                if (k0 + u * nt < Kb) {
                    a[u] = ym[k0 + u * nt];
                    b[u] = yn[k0 + u * nt];
                }
#pragma unroll
            for (int u = 0; u < kStageUnroll; ++u) {
                const int k = k0 + u * nt;
                if (k >= Kb) continue;
                float2 x = a[u], y = b[u];
                if (weighting == SRP_WEIGHT_PHAT) {
                    x = unit_phase(x);
                    y = unit_phase(y);
                }
                const float2 v = times_conj(x, y);
                const float w = (k == 0 || 2 * k == K) ? 1.0f : 2.0f;
                ps[k] = make_float2(w * v.x, w * v.y);
            }
        }
        wait_async_copies();
    } else {
        stage_gcc_row(src + ((size_t)l * Q + q) * Kb, twid, K, tw, ps);
    }
    __syncthreads();
    const int base = offc[q];
    float *x32 = xi32 != nullptr ? xi32 + (size_t)l * S32 + off[q] : nullptr;
    gcc_row(tw, ps, K, nq[q] + n_aux, [&](int t, int n, float v) {
        if (x32 != nullptr) x32[t] = v;
        if (n & 1) v = -v;
        const size_t hi = (size_t)l * S_pad + base + t;
        if (kFmt == 2) {
            __half h = __float2half_rn(v);
            xi16[hi] = *reinterpret_cast<uint16_t *>(&h);
        } else {
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            xi16[hi] = *reinterpret_cast<uint16_t *>(&h);
            if (kFmt == 1) {
                __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(h));
                xi16[hi + (size_t)L_pad * S_pad] = *reinterpret_cast<uint16_t *>(&lo);
            }
        }
    });
}

// ---------------------------------------------------------------------------
// Conventional operand B: slot offc[q] + 2k (+1) of row l holds
// (a_k/K) Re psi_q(k) (and (a_k/K) Im psi_q(k)), as bf16 (hi, lo) or fp16.
// ---------------------------------------------------------------------------
// With psi32 the weighted cross spectrum formed from STFT input is also
// stored in FP32, psi32[frame][q][k], for the FP32 re-scoring.
template <int kFmt, bool kFromY>  // kFmt 0: bf16, 1: bf16 hi/lo split, 2: fp16
__global__ void __launch_bounds__(128) k_conv_operand_tc(
    const float2 *__restrict__ src, int M, const int2 *__restrict__ pairs, int weighting, int Q,
    int K, const int32_t *__restrict__ offc, uint16_t *__restrict__ b16, int L_pad, int S_pad,
    unsigned long long *__restrict__ best, float2 *__restrict__ psi32) {
    const int Kb = K / 2 + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y, l = blockIdx.z;
    grid_dep_launch();  // the map kernel may start its prologue now
    if (best != nullptr && blockIdx.x == 0 && q == 0 && l == 0)
        for (int i = threadIdx.x; i < (int)gridDim.z; i += blockDim.x) best[i] = 0ull;
    if (k >= Kb) return;
    float2 v;
    if (kFromY) {  // the weighted cross spectrum of K1, formed here
        const int2 p = pairs[q];
        float2 a = src[((size_t)l * M + p.x) * Kb + k], b = src[((size_t)l * M + p.y) * Kb + k];
        if (weighting == SRP_WEIGHT_PHAT) {
            a = unit_phase(a);
            b = unit_phase(b);
        }
        v = times_conj(a, b);
        if (psi32 != nullptr) psi32[((size_t)l * Q + q) * Kb + k] = v;
    } else {
        v = src[((size_t)l * Q + q) * Kb + k];
    }
    const float ak = ((k == 0 || 2 * k == K) ? 1.0f : 2.0f) / (float)K;
    const float re = ak * v.x, im = ak * v.y;
    const size_t hi = (size_t)l * S_pad + offc[q] + 2 * k;
    uint32_t h, lo = 0;
    if (kFmt == 2) {
        h = pack_f16(re, im);
    } else {
        h = pack_bf16(re, im);
        if (kFmt == 1)
            lo = pack_bf16(re - __uint_as_float(h << 16), im - __uint_as_float(h & 0xFFFF0000u));
    }
    *reinterpret_cast<uint32_t *>(b16 + hi) = h;
    if (kFmt == 1) *reinterpret_cast<uint32_t *>(b16 + hi + (size_t)L_pad * S_pad) = lo;
}

// ---------------------------------------------------------------------------
// The contraction.
// ---------------------------------------------------------------------------
struct TcArgs {
    const int2 *xs;         // [Q][J_pad] (fixed-point TDOA, bits of sp)
    int K;                  // DFT length (conventional map)
    const int4 *ctab;       // [n_chunks] (pair, nmax_q - first lag slot as float bits or, for
                            // the conventional map, first bin; groups; MMA steps)
    int64_t J_pad, J;
    int Q;
    const int32_t *nq;      // [Q]
    int n_aux, xf;
    int n_chunks;           // S_pad / 64
    int L_pad, L, N;        // N: frames per CTA (MMA N), multiple of 16, <= 256
    uint32_t idesc;
    uint32_t tmem_cols;
    int stages;
    float *maps;            // [L][J] or null
    unsigned long long *part;  // [L_pad][n_tiles]
    int n_tiles;
    int *status;
    int vec_maps;           // maps rows are 8-byte aligned (float2 stores)
    int bulk_maps;          // maps in device memory, 16-byte aligned, J % 4 == 0: one
                            // bulk store per frame row of a tile
    uint32_t a_col0;        // operand A in TMEM: first column of the A stages
    int par1_used;          // the tile has two or more 16-lag steps: accumulator 1 is written
    const uint4 *w;         // resident operand A (kW): the plan's interpolation matrix
    const int32_t *woff;    // [n_chunks] first 16-slot step of chunk c within a tile's block
    int tile_steps;         // 16-slot steps per 128-candidate tile
    int all_streamed;       // kW with every chunk resident: the generators read no TDOA table
    unsigned long long *fkey;  // non-null: write part[frame][tile], raise fkey[frame]
    int mma_warps;          // 2: two accumulators fed by two warps; 1: one accumulator
    int promote;            // conventional FP32: chunks per accumulator epoch (0: one epoch)
};

// ---------------------------------------------------------------------------
// Plan time: the interpolation matrix (operand A) of a resident-weights plan.
// For every 128-candidate tile t and chunk c, the sinc weights of the chunk's
// nk used 16-slot steps, in the canonical K-major layout without swizzle (one
// kAStep block per step: 16 groups of 8 rows, each two 128-byte core matrices
// of 8 rows x 16 bytes along K), high parts then low parts for the FP32 split.
// Chunk c of tile t starts (t * tile_steps + woff[c]) * hs * kAStep bytes in.
// The weights are the generator's, so the maps equal those of on-chip
// generation.
// ---------------------------------------------------------------------------
template <bool kSplit, bool kHalf>
__global__ void __launch_bounds__(128) k_build_w(const int2 *__restrict__ xs,
                                                 const int4 *__restrict__ ctab,
                                                 const int32_t *__restrict__ woff, int n_chunks,
                                                 int64_t J_pad, int xf, int tile_steps,
                                                 uint4 *__restrict__ w) {
    const int r = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * 128 + r;
    const int hs = kSplit ? 2 : 1;
    const uint32_t row_off = (uint32_t)((r >> 3) * 16 + (r & 7));  // uint4 units in a step
    uint4 *tile = w + (size_t)blockIdx.x * tile_steps * hs * (kAStep / 16);
    int q = -1;
    float sp = 0.0f, f = 0.5f, x0f = 0.0f;
    for (int c = 0; c < n_chunks; ++c) {
        const int4 cur = ctab[c];
        if (cur.x != q) {
            q = cur.x;
            const int2 e = xs[(size_t)q * J_pad + i];
            int x0;
            decode_tdoa(e.x, xf, x0, f);
            if (f == 0.0f) f = 9.094947017729282e-13f;  // 2^-40, as in the plan
            sp = __int_as_float(e.y);
            x0f = (float)x0;
        }
        const int wo = woff[c];
        if (wo < 0) continue;  // generated on chip by the map kernel
        const float mc = x0f + __int_as_float(cur.y);
        uint4 *hi = tile + (size_t)wo * hs * (kAStep / 16);
        uint4 *lo = hi + (size_t)cur.w * (kAStep / 16);
        switch (cur.z) {
            case 2: gen_groups<2, kSplit, kHalf, kAGlobal>(row_off, row_off, 0u, f, mc, sp, 0u, hi, lo); break;
            case 4: gen_groups<4, kSplit, kHalf, kAGlobal>(row_off, row_off, 0u, f, mc, sp, 0u, hi, lo); break;
            case 6: gen_groups<6, kSplit, kHalf, kAGlobal>(row_off, row_off, 0u, f, mc, sp, 0u, hi, lo); break;
            default: gen_groups<8, kSplit, kHalf, kAGlobal>(row_off, row_off, 0u, f, mc, sp, 0u, hi, lo); break;
        }
    }
}


// kTm: operand A is generated into TMEM (32 columns per 64-slot stage and
// part) and the MMAs read only B from shared memory; otherwise A is a
// 128-byte-swizzled shared-memory tile like B.  kW: the chunks whose weights
// are resident in the plan's interpolation matrix are not generated but
// streamed by bulk copies (no swizzle, one block per 16-slot step) into the
// stage's shared-memory A region next to B.  kTm and kW together: generated
// chunks go to TMEM as with kTm alone, streamed chunks are read from shared
// memory, so on-chip generation and HBM streaming share the work.
// kOcc: CTAs per SM the launch is built for (2, or 4 for the 16-bit formats
// with one accumulator and 128 TMEM columns per CTA).
// kPr (FP32 conventional, A in TMEM): the accumulators are promoted every
// a.promote chunks.
template <bool kSplit, bool kHalf, bool kConv, bool kTm, bool kW = false, int kOcc = 2,
          bool kPr = false>
__global__ void __launch_bounds__(kThreads, kOcc) k_interp_tc(const __grid_constant__ CUtensorMap tmap,
                                                              const TcArgs a) {
    static_assert(!kPr || (kConv && kSplit && kTm && !kW), "promotion: FP32 conventional, TMEM A");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // control block, then 1024-aligned stages, then the argmax scratch
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    // full[kMaxStages], empty[kMaxStages], accum, epoch, drained
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + 8 * (2 * kMaxStages + 3));
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t b_tile = (uint32_t)a.N * 128u;
    // (a shared-memory A region unless A only ever comes from TMEM)
    constexpr bool kSmemA = !kTm || kW;
    const uint32_t stage_bytes = (kSplit ? 2u : 1u) * ((kSmemA ? kATile : 0u) + b_tile);
    const uint32_t stage0 = base + 1024u;
    // epilogue tile mt[frame][kMtStride] over the (then idle) stage buffers,
    // then the per-row ring of prefetched (TDOA, sp): xring[slot][row], 8 bytes each
    const uint32_t tile_bytes = ((uint32_t)a.N * (uint32_t)kMtStride * 4u + 1023u) & ~1023u;
    const uint32_t xring = base + 1024u + max(stage_bytes * (uint32_t)a.stages, tile_bytes);
    float *mt = reinterpret_cast<float *>(gbase + 1024u);
    // Accumulator promotion (FP32 conventional maps with long reductions):
    // every a.promote chunks the generator warps add the TMEM accumulators
    // into rs[frame][row] (FP32, round to nearest) and the MMAs start them
    // afresh, so that no accumulator sums more than a.promote chunks.
    constexpr bool promote = kPr;
    float *rs = reinterpret_cast<float *>(gbase + (xring - base) + kXRing * 128 * sizeof(int2));

    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[kMaxStages + s]); };
    const uint32_t accum_bar = smem_u32(&bars[2 * kMaxStages]);
    const uint32_t epoch_bar = smem_u32(&bars[2 * kMaxStages + 1]);    // the epoch's MMAs done
    const uint32_t drained_bar = smem_u32(&bars[2 * kMaxStages + 2]);  // accumulators read
    auto a_hi = [&](int s) { return stage0 + (uint32_t)s * stage_bytes; };
    auto a_lo = [&](int s) { return stage0 + (uint32_t)s * stage_bytes + kATile; };
    auto b_hi = [&](int s) {
        return stage0 + (uint32_t)s * stage_bytes + (kSmemA ? (kSplit ? 2u : 1u) * kATile : 0u);
    };
    // operand A of stage s in TMEM: part 0 (hi) then part 1 (lo), 32 columns each
    auto a_tm = [&](int s, int part) {
        return a.a_col0 + ((uint32_t)s * (kSplit ? 2u : 1u) + (uint32_t)part) * 32u;
    };
    auto b_lo = [&](int s) { return b_hi(s) + b_tile; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l0 = blockIdx.y * a.N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full_bar(s), 128 + 1);
            mbar_init(empty_bar(s), (uint32_t)a.mma_warps);
        }
        mbar_init(accum_bar, (uint32_t)a.mma_warps);
        mbar_init(epoch_bar, (uint32_t)a.mma_warps);
        mbar_init(drained_bar, 128);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kTmaWarp) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    grid_dep_launch();  // the argmax kernel may be scheduled behind this grid
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        const int r = threadIdx.x;
        if (promote)  // the running sums start at zero (each thread owns its row)
            for (int j = 0; j < a.N; ++j) rs[j * 128 + r] = 0.0f;
        {
        // ---------------- A generation: one candidate row per thread ----------------
        // (kW: chunks whose weights are resident are streamed by the TMA warp and
        // only pass through the stage barriers here; with every chunk resident the
        // TDOA table is not read at all)
        const int64_t i = (int64_t)blockIdx.x * 128 + r;
        const uint32_t row = (uint32_t)r * 128u, sw = (uint32_t)(r & 7);
        // d = f + (m - e) for lag e of a group, where m = x0 + nmax - (first lag
        // slot of the group) is an exact integer in FP32: d is rounded once and
        // is never 0 unless f is.
        int q = -1;
        float sp = 0.0f, f = 0.5f, x0f = 0.0f;
        int x0m = 0;              // conventional: x0 mod K
        float wp = 1.0f, wq = 0.0f;  // conventional: e^{-j 2 pi x / K}
        const float two_k = 2.0f / (float)a.K;
        // (TDOA, sp) of the first kXAhead pairs start streaming in now; pair p
        // sits in slot p % kXRing (kXRingW and kXAheadW for kTm with kW, whose
        // stages also hold streamed A blocks).  Pair q + 1 is read from its
        // slot when pair q starts, one chunk or more ahead of its use, and that
        // read issues the load of pair q + 1 + kXAhead (one commit group per
        // pair).
        const int ring_q = (kW && a.all_streamed) ? 0 : a.Q;  // pairs whose TDOAs are read
        constexpr int kRing = (kTm && kW) ? kXRingW : kXRing, kAhead = kRing - 1;
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            if (k < ring_q)
                cp_async8(xring + (uint32_t)(k * 128 + r) * 8u, &a.xs[(size_t)k * a.J_pad + i]);
            cp_async_commit();
        }
        int32_t nX, nsp;  // (TDOA, sp) of the next pair to start
        auto read_ring = [&](int p) {
            cp_async_wait<kAhead - 1>();  // pair p has landed
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];"
                         : "=r"(nX), "=r"(nsp)
                         : "r"(xring + (uint32_t)((p % kRing) * 128 + r) * 8u));
            const int pn = p + kAhead;
            if (pn < ring_q)
                cp_async8(xring + (uint32_t)((pn % kRing) * 128 + r) * 8u,
                          &a.xs[(size_t)pn * a.J_pad + i]);
            cp_async_commit();
        };
        read_ring(0);
        int4 cur = __ldg(&a.ctab[0]);
        int st = 0;        // stage of chunk c, and the parity of its use
        uint32_t ph = 0;
        for (int c = 0; c < a.n_chunks; ++c) {
            const int4 nxt = __ldg(&a.ctab[c + 1 < a.n_chunks ? c + 1 : c]);
            if (cur.x != q && ring_q > 0) {  // uniform: a new pair starts with this chunk
                q = cur.x;
                int x0;
                decode_tdoa(nX, a.xf, x0, f);
                if (kConv) {
                    x0m = ((x0 % a.K) + a.K) % a.K;
                    float sn, cs;
                    sincospif(((float)x0 + f) * two_k, &sn, &cs);
                    wp = cs;
                    wq = -sn;
                } else {
                    if (f == 0.0f) f = 9.094947017729282e-13f;  // 2^-40, as in the plan
                    sp = __int_as_float(nsp);
                    x0f = (float)x0;
                }
                if (q + 1 < a.Q) read_ring(q + 1);
            }
            const float mc = x0f + __int_as_float(cur.y);  // Nyquist: x0 + nmax - first lag slot
            const int ng = cur.z;
            // the stage is reused once the MMAs of chunk c - stages completed; the
            // weights are computed into registers before this wait and stored after
            const uint32_t eb = empty_bar(st), eph = ph ^ 1u;
            const bool reuse = c >= a.stages;
            auto wait_free = [&]() {
                if (reuse && !mbar_try_wait(eb, eph)) mbar_wait(eb, eph, abort_flag, a.status);
            };
            // up to 64 weights, fully unrolled per group count
            const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
            const uint32_t d0 = kTm ? tmem + lane_base + a_tm(st, 0) : a_hi(st) + row;
            const uint32_t d1 = kTm ? tmem + lane_base + a_tm(st, 1) : 0u;
            if (kW && __ldg(&a.woff[c]) >= 0) {
                // resident: the TMA warp brings this chunk's weights
                wait_free();
            } else if (kConv) {
                // exact seed e^{-j theta_k0} for the chunk's first bin k0 = cur.y
                const int k0 = cur.y;
                const int rk = (int)(((long long)k0 * x0m) % a.K);
                float sn, cs;
                sincospif(fmaf((float)rk, two_k, (float)k0 * f * two_k), &sn, &cs);
                switch (ng) {
                    case 2: gen_steer<2, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                    case 4: gen_steer<4, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                    case 6: gen_steer<6, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                    default: gen_steer<8, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                }
            } else {
                switch (ng) {
                    case 2: gen_groups<2, kSplit, kHalf, kTm>(d0, d1, sw, f, mc, sp, 0u, nullptr, nullptr, wait_free); break;
                    case 4: gen_groups<4, kSplit, kHalf, kTm>(d0, d1, sw, f, mc, sp, 0u, nullptr, nullptr, wait_free); break;
                    case 6: gen_groups<6, kSplit, kHalf, kTm>(d0, d1, sw, f, mc, sp, 0u, nullptr, nullptr, wait_free); break;
                    default: gen_groups<8, kSplit, kHalf, kTm>(d0, d1, sw, f, mc, sp, 0u, nullptr, nullptr, wait_free); break;
                }
            }
            if (kTm) {  // TMEM stores complete and ordered before the MMA's reads
                tmem_wait_st();
                tc_fence_before();
            } else {  // generic-proxy smem writes visible to the tensor core
                fence_proxy_async();
            }
            mbar_arrive(full_bar(st));
            cur = nxt;
            if (++st == a.stages) {
                st = 0;
                ph ^= 1u;
            }
            if (promote && c > 0 && c % a.promote == 0) {
                // the epoch ended with chunk c - 1: once its MMAs are done, add
                // the accumulators to the running sums and release them
                const uint32_t eph = (uint32_t)(c / a.promote - 1) & 1u;
                if (!mbar_wait(epoch_bar, eph, abort_flag, a.status)) break;
                tc_fence_after();
                const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes
                for (int j0 = 0; j0 < a.N; j0 += 16) {
                    float v[16];
                    tmem_ld16(trow + (uint32_t)j0, v);
                    if (a.par1_used) {
                        float v1[16];
                        tmem_ld16(trow + (uint32_t)(a.N + j0), v1);
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj) v[jj] += v1[jj];
                    }
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) rs[(j0 + jj) * 128 + r] += v[jj];
                }
                tc_fence_before();
                mbar_arrive(drained_bar);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        }

        // ---------------- epilogue: TMEM -> smem tile -> maps + argmax keys ----------------
        mbar_wait(accum_bar, 0, abort_flag, a.status);
        grid_dep_wait();  // the operand kernel cleared the frames' keys
        tc_fence_after();
        fence_proxy_async();
        // every MMA has completed (and with it every TMA load it consumed), so the
        // stage buffers are free: candidate r's frames go to column r of mt
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j0 = 0; j0 < a.N; j0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)j0, v);
            if (a.par1_used) {
                float v1[16];
                tmem_ld16(trow + (uint32_t)(a.N + j0), v1);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] += v1[jj];
            }
            if (promote) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) v[jj] += rs[(j0 + jj) * 128 + r];
            }
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) mt[(j0 + jj) * kMtStride + r] = v[jj];
        }
        tc_fence_before();
        if (a.bulk_maps) fence_proxy_async();  // mt's stores before the bulk copies read it
        asm volatile("bar.sync 1, 128;" ::: "memory");
        const int64_t tile0 = (int64_t)blockIdx.x * 128;
        const int n_rows = min(a.N, a.L - l0);
        if (a.bulk_maps) {  // warp w's lane 0 copies frame rows w, w + 4, ... out
            if (lane == 0) {
                const uint32_t bytes = 4u * (uint32_t)min((int64_t)128, a.J - tile0);
                for (int fr = warp; fr < n_rows; fr += 4)
                    bulk_store(a.maps + (size_t)(l0 + fr) * a.J + tile0,
                               smem_u32(mt + fr * kMtStride), bytes);
                bulk_commit();
            }
        } else if (a.maps != nullptr) {  // warp w writes frame rows w, w + 4, ...
            for (int fr = warp; fr < n_rows; fr += 4) {
                float *dst = a.maps + (size_t)(l0 + fr) * a.J + tile0;
                const float *srcr = mt + fr * kMtStride;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int k = 2 * (lane + 32 * hh);
                    const float2 val = *reinterpret_cast<const float2 *>(srcr + k);
                    if (a.vec_maps && tile0 + k + 1 < a.J) {
                        *reinterpret_cast<float2 *>(dst + k) = val;
                    } else {
                        if (tile0 + k < a.J) dst[k] = val.x;
                        if (tile0 + k + 1 < a.J) dst[k + 1] = val.y;
                    }
                }
            }
        }
        // first maximiser per frame: threads 2f and 2f+1 scan even / odd candidates
        for (int fr = r >> 1; fr < n_rows + 63 - ((n_rows + 63) % 64); fr += 64) {
            const int h = r & 1;
            unsigned long long key = 0ull;
            if (fr < n_rows) {
                uint32_t bo = 0u;
                int bk = -1;
                const float *row_p = mt + fr * kMtStride;
                const int kmax = (int)min((int64_t)128, a.J - tile0);
                if (kmax == 128) {  // full tile: 64 candidates per thread, unrolled
                    // (FP32 compares: the same first maximiser as the ordered
                    // values for finite maps, -0 equal to +0)
                    const float *rp = row_p + h;
                    int bj = 0;
                    float bv = rp[0];
#pragma unroll
                    for (int j = 1; j < 64; ++j) {
                        const float v = rp[2 * j];
                        if (v > bv) {
                            bv = v;
                            bj = j;
                        }
                    }
                    bo = ordered_value(bv);
                    bk = h + 2 * bj;
                } else {
                    for (int k = h; k < kmax; k += 2) {
                        const uint32_t o = ordered_value(row_p[k]);
                        if (bk < 0 || o > bo) {
                            bo = o;
                            bk = k;
                        }
                    }
                }
                if (bk >= 0)
                    key = ((unsigned long long)bo << 32) |
                          (unsigned long long)(0xFFFFFFFFu - (uint32_t)(tile0 + bk));
            }
            const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, key, 1);
            key = other > key ? other : key;
            if (h == 0 && fr < n_rows) {
                if (a.fkey != nullptr) {
                    a.part[(size_t)(l0 + fr) * a.n_tiles + blockIdx.x] = key;
                    atomicMax(a.fkey + l0 + fr, key);
                } else if (key != 0ull) {
                    atomicMax(a.part + l0 + fr, key);
                }
            }
        }
        if (a.bulk_maps && lane == 0) bulk_wait_read();
    } else if (warp == kTmaWarp) {
        // ---------------- B loads (GCC samples) ----------------
        if (lane == 0) {
            const uint32_t bytes = (kSplit ? 2u : 1u) * b_tile;
            int issued = 0;
            int st = 0;  // stage of chunk c, and the parity of its use
            uint32_t ph = 0;
            grid_dep_wait();  // operand B is written by the previous kernel
            for (int c = 0; c < a.n_chunks; ++c) {
                if (c >= a.stages && !mbar_wait(empty_bar(st), ph ^ 1u, abort_flag, a.status))
                    break;
                if (*abort_flag) break;
                const int wo = kW ? __ldg(&a.woff[c]) : -1;
                if (wo >= 0) {  // the chunk's used steps of the resident A, high then low parts
                    const uint32_t a_bytes = (uint32_t)__ldg(&a.ctab[c]).w * kAStep;
                    const uint4 *src = a.w + ((size_t)blockIdx.x * a.tile_steps + wo) *
                                                 (kSplit ? 2 : 1) * (kAStep / 16);
                    mbar_arrive_expect_tx(full_bar(st), bytes + (kSplit ? 2u : 1u) * a_bytes);
                    bulk_load(a_hi(st), src, a_bytes, full_bar(st));
                    if (kSplit) bulk_load(a_lo(st), src + a_bytes / 16, a_bytes, full_bar(st));
                } else {
                    mbar_arrive_expect_tx(full_bar(st), bytes);
                }
                tma_load_2d(b_hi(st), &tmap, c * kChunk, l0, full_bar(st));
                if (kSplit) tma_load_2d(b_lo(st), &tmap, c * kChunk, a.L_pad + l0, full_bar(st));
                issued = c + 1;
                if (++st == a.stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            if (*abort_flag) {
                // let every copy already issued land before the CTA exits
                for (int c = (issued > a.stages ? issued - a.stages : 0); c < issued; ++c) {
                    const int st = c % a.stages;
                    const uint32_t ph = (uint32_t)(c / a.stages) & 1u;
                    const uint64_t t0 = global_timer();
                    while (!mbar_try_wait(full_bar(st), ph) && global_timer() - t0 < kWaitLimitNs) {
                    }
                }
            }
        }
    } else {
        // ---------------- MMA issue: two warps, by 16-lag step parity ----------------
        // One 128 x N x 16 MMA is small at N = 64, and MMAs into one accumulator
        // form a dependent chain, so the steps are spread over two accumulators
        // (TMEM columns [0, N) and [N, 2N)), each fed by its own issuing warp;
        // the epilogue adds them.  The parity is that of the running step count
        // over the whole tile, which balances the two chains also when every
        // chunk holds an odd number of steps.
        // With a.mma_warps == 1 the first MMA warp sums every step into one
        // accumulator (columns [0, N)) and the second has nothing to do.
        // The whole warp runs the loop and computes every operand alike (the
        // TMEM base and the chunk-table entries broadcast from lane 0), and one
        // elected lane issues the chunk's MMAs and the commits that track them,
        // in the same elected block.
        const int par = warp - kMmaWarp0;
        if (par < a.mma_warps) {
            const uint32_t tm = __shfl_sync(0xFFFFFFFFu, tmem, 0);
            const uint32_t dt = tm + (uint32_t)(par * a.N);
            const int kstep = a.mma_warps;
            uint32_t acc = 0;  // the first MMA into the accumulator overwrites it
            int g0 = 0;        // 16-lag steps of the earlier chunks
            int st = 0;        // stage of chunk c, and the parity of its use
            uint32_t ph = 0;
            int ep = 0;        // promotion: chunks into the current epoch
            uint32_t eph = 0;  // promotion: parity of the epoch that ends next
            bool done = false;
            // the chunk table entry of the next chunk is loaded a chunk ahead,
            // so that its latency overlaps the wait instead of delaying the MMAs
            int nk_next = __shfl_sync(0xFFFFFFFFu, __ldg(&a.ctab[0]).w, 0);
            bool streamed_next = kW && __shfl_sync(0xFFFFFFFFu, __ldg(&a.woff[0]), 0) >= 0;
            for (int c = 0; c < a.n_chunks; ++c) {
                const int nk = nk_next;  // 16-lag steps holding lags of the pair
                const bool streamed = streamed_next;
                if (c + 1 < a.n_chunks) {
                    nk_next = __shfl_sync(0xFFFFFFFFu, __ldg(&a.ctab[c + 1]).w, 0);
                    streamed_next =
                        kW && __shfl_sync(0xFFFFFFFFu, __ldg(&a.woff[c + 1]), 0) >= 0;
                }
                const uint64_t dah = smem_desc_sw128(a_hi(st)), dbh = smem_desc_sw128(b_hi(st));
                const uint64_t dal = smem_desc_sw128(a_lo(st)), dbl = smem_desc_sw128(b_lo(st));
                const uint32_t tah = tm + a_tm(st, 0), tal = tm + a_tm(st, 1);
                if (promote && ep == a.promote) {
                    // the epoch's MMAs were committed to epoch_bar with its last
                    // chunk; once the generators have read the accumulators,
                    // the next MMA into each starts it afresh
                    bool ok = mbar_try_wait(drained_bar, eph) ||
                              mbar_wait(drained_bar, eph, abort_flag, a.status);
                    if (!__all_sync(0xFFFFFFFFu, ok)) break;
                    tc_fence_after();
                    acc = 0;
                    ep = 0;
                    eph ^= 1u;
                }
                bool ok = mbar_try_wait(full_bar(st), ph) ||
                          mbar_wait(full_bar(st), ph, abort_flag, a.status);
                if (!__all_sync(0xFFFFFFFFu, ok)) break;
                tc_fence_after();
                const int kk0 = kstep == 1 ? 0 : (par + g0) & 1;  // this warp's first step
                g0 += nk;
                ++ep;
                const bool last = c + 1 == a.n_chunks;
                const bool epoch_end = promote && ep == a.promote && !last;
                if (elect_one()) {
#pragma unroll
                    for (int s = 0; s < kChunk / 16; ++s) {
                        const int kk = kk0 + s * kstep;
                        if (kk >= nk) break;
                        const uint32_t acc_s = s > 0 ? 1u : acc;
                        const uint64_t adv = (uint64_t)(kk * 2);  // 32 bytes in 16-byte units
                        const uint32_t ac = (uint32_t)(kk * 8);   // 16 values in 8 TMEM columns
                        if (kTm && !streamed) {
                            mma_f16_ts(dt, tah + ac, dbh + adv, a.idesc, acc_s);
                            if (kSplit) {
                                mma_f16_ts(dt, tah + ac, dbl + adv, a.idesc, 1);
                                mma_f16_ts(dt, tal + ac, dbh + adv, a.idesc, 1);
                            }
                        } else if (streamed) {  // A blocks without swizzle, kAStep bytes per step
                            const uint64_t wah = smem_desc_none(a_hi(st) + (uint32_t)kk * kAStep);
                            const uint64_t wal = smem_desc_none(a_lo(st) + (uint32_t)kk * kAStep);
                            mma_f16(dt, wah, dbh + adv, a.idesc, acc_s);
                            if (kSplit) {
                                mma_f16(dt, wah, dbl + adv, a.idesc, 1);
                                mma_f16(dt, wal, dbh + adv, a.idesc, 1);
                            }
                        } else {
                            mma_f16(dt, dah + adv, dbh + adv, a.idesc, acc_s);
                            if (kSplit) {
                                mma_f16(dt, dah + adv, dbl + adv, a.idesc, 1);
                                mma_f16(dt, dal + adv, dbh + adv, a.idesc, 1);
                            }
                        }
                    }
                    mma_commit(empty_bar(st));
                    if (epoch_end) mma_commit(epoch_bar);
                    if (last) mma_commit(accum_bar);
                }
                __syncwarp();
                if (kk0 < nk) acc = 1;
                if (last) done = true;
                if (++st == a.stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            // a loop left early (a wait gave up) still commits, so that the
            // release of TMEM can wait for whatever MMAs were issued
            if (!done && elect_one()) mma_commit(accum_bar);
            __syncwarp();
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == kTmaWarp) {
        tc_fence_after();
        if (*abort_flag) {  // make sure no MMA is still writing TMEM
            const uint64_t t0 = global_timer();
            while (!mbar_try_wait(accum_bar, 0) && global_timer() - t0 < kWaitLimitNs) {
            }
        }
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (fn == nullptr) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

template <bool kSplit, bool kHalf, bool kConv, bool kTm, bool kW = false, int kOcc = 2,
          bool kPr = false>
cudaError_t launch_tc(const CUtensorMap &map, const TcArgs &a, int grid_y, size_t smem,
                      cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_interp_tc<kSplit, kHalf, kConv, kTm, kW, kOcc, kPr>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // programmatic stream serialization: the prologue (TMEM allocation, barrier
    // set-up, the first TDOA loads) overlaps the end of the operand kernel
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.n_tiles, grid_y);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e =
        cudaLaunchKernelEx(&cfg, k_interp_tc<kSplit, kHalf, kConv, kTm, kW, kOcc, kPr>, map, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <bool kSplit, bool kHalf, bool kConv>
cudaError_t launch_tc_a(const CUtensorMap &map, const TcArgs &a, bool tm, int grid_y, size_t smem,
                        cudaStream_t s) {
    if constexpr (!kSplit) {
        if (tm && a.mma_warps == 1)  // four CTAs per SM
            return launch_tc<kSplit, kHalf, kConv, true, false, 4>(map, a, grid_y, smem, s);
    } else if constexpr (kConv) {
        if (tm && a.promote > 0)  // promoted accumulators
            return launch_tc<kSplit, kHalf, kConv, true, false, 2, true>(map, a, grid_y, smem, s);
    }
    return tm ? launch_tc<kSplit, kHalf, kConv, true>(map, a, grid_y, smem, s)
              : launch_tc<kSplit, kHalf, kConv, false>(map, a, grid_y, smem, s);
}

}  // namespace

cudaError_t encode_xi_map(void *xi16, int rows, int S_pad, int N, void *map_out) {
    EncodeTiledFn fn = encode_fn();
    if (fn == nullptr) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)S_pad, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)S_pad * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)N};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap *>(map_out), CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                    xi16, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_gcc_samples_tc(const float2 *src, bool from_y, int M, const int2 *pairs,
                                  int weighting, int L, int Q, int K, const int32_t *nq,
                                  const int32_t *offc, int n_aux, const float2 *twid,
                                  uint16_t *xi16, int L_pad, int S_pad, int fmt,
                                  unsigned long long *best, float *xi32, const int32_t *off,
                                  int S32, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)(K + K / 2 + 1);
    typedef void (*Kern)(const float2 *, int, const int2 *, int, int, int, const int32_t *,
                         const int32_t *, int, const float2 *, uint16_t *, int, int,
                         unsigned long long *, float *, const int32_t *, int);
    static const Kern kerns[6] = {k_gcc_samples_tc<0, false>, k_gcc_samples_tc<1, false>,
                                  k_gcc_samples_tc<2, false>, k_gcc_samples_tc<0, true>,
                                  k_gcc_samples_tc<1, true>,  k_gcc_samples_tc<2, true>};
    static bool attr[6] = {false, false, false, false, false, false};
    const int v = fmt + (from_y ? 3 : 0);
    if (!attr[v]) {
        cudaError_t e = cudaFuncSetAttribute(kerns[v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float2) * (8192 + 4097)));
        if (e != cudaSuccess) return e;
        attr[v] = true;
    }
    kerns[v]<<<dim3(Q, L), 128, smem, s>>>(src, M, pairs, weighting, Q, K, nq, offc, n_aux, twid,
                                           xi16, L_pad, S_pad, best, xi32, off, S32);
    return cudaGetLastError();
}

cudaError_t launch_conv_operand_tc(const float2 *src, bool from_y, int M, const int2 *pairs,
                                   int weighting, int L, int Q, int K, const int32_t *offc,
                                   uint16_t *b16, int L_pad, int S_pad, int fmt,
                                   unsigned long long *best, float2 *psi32, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    const int Kb = K / 2 + 1;
    dim3 grid((Kb + 127) / 128, Q, L);
    typedef void (*Kern)(const float2 *, int, const int2 *, int, int, int, const int32_t *,
                         uint16_t *, int, int, unsigned long long *, float2 *);
    static const Kern kerns[6] = {k_conv_operand_tc<0, false>, k_conv_operand_tc<1, false>,
                                  k_conv_operand_tc<2, false>, k_conv_operand_tc<0, true>,
                                  k_conv_operand_tc<1, true>,  k_conv_operand_tc<2, true>};
    kerns[fmt + (from_y ? 3 : 0)]<<<grid, 128, 0, s>>>(src, M, pairs, weighting, Q, K, offc, b16,
                                                       L_pad, S_pad, best, psi32);
    return cudaGetLastError();
}

int interp_tc_frames_per_cta(int L) {
    const int n = ((L + 15) / 16) * 16;
    return n > 256 ? 256 : n;
}

cudaError_t launch_interp_tc(const void *xi_map, int N, const int2 *xs, const int4 *ctab,
                             int par1_used, int64_t J_pad, int64_t J, int Q, const int32_t *nq,
                             int n_aux, int xf, int S_pad, int L_pad, int L, int precision,
                             int conv, int K, float *maps, unsigned long long *part, int n_tiles,
                             int *status, const void *w, const int32_t *woff, int tile_steps,
                             int all_streamed, unsigned long long *frame_keys, int promote,
                             cudaStream_t s) {
    // N is the plan's frames per CTA: the height of the tensor map's box.
    if (L == 0) return cudaSuccess;
    if (w != nullptr && conv) return cudaErrorInvalidValue;  // resident A: Nyquist only
    if (N < 16 || N > 256 || (N & 15)) return cudaErrorInvalidValue;
    const bool split = precision == SRP_PREC_FP32, half = precision == SRP_PREC_FP16;
    TcArgs a;
    a.xs = xs;
    a.ctab = ctab;
    a.J_pad = J_pad;
    a.J = J;
    a.Q = Q;
    a.nq = nq;
    a.n_aux = n_aux;
    a.xf = xf;
    a.n_chunks = S_pad / kChunk;
    a.L_pad = L_pad;
    a.L = L;
    a.N = N;
    // kind::f16 instruction descriptor: FP32 accumulate (bit 4), A/B BF16 (bits 7, 10)
    // or FP16 (0), both K-major, N >> 3 at bit 17, M = 128 >> 4 at bit 24.
    const uint32_t ab = half ? 0u : 1u;
    a.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
    const int hs = split ? 2 : 1;
    const size_t tile_bytes = ((size_t)N * kMtStride * sizeof(float) + 1023) / 1024 * 1024;
    // Operand A in TMEM when two CTAs per SM keep 2N accumulator columns and at
    // least two A stages (32 columns per part) within 256 columns each.  With
    // resident weights, the generated chunks still go to TMEM (unless every
    // chunk is streamed) and the stages also hold a shared-memory A region.
    const bool streams = w != nullptr;
    const bool tm = (!streams || !all_streamed) && 2 * N + 2 * hs * 32 <= 256;
    const size_t fixed =
        1024 + 1024 + (size_t)((tm && streams) ? kXRingW : kXRing) * 128 * sizeof(int2);
    const size_t a_region = streams ? kATile : 0;  // per part
    // 16-bit formats with up to 64 frames: one accumulator and two or three A
    // stages in 128 TMEM columns, so that four CTAs (four independent
    // generator -> MMA pipelines) share an SM
    // (one accumulator for every 16-bit plan with up to 64 frames, streamed
    // weights included, so that a plan's maps do not depend on where its
    // operand A comes from)
    const bool one_acc = !split && N <= 64;
    const bool quad = tm && one_acc;
    a.mma_warps = one_acc ? 1 : 2;
    int stages;
    size_t smem;
    if (quad) {
        stages = std::min(kMaxStages, (128 - N) / 32);
        a.tmem_cols = 128;
        a.a_col0 = (uint32_t)N;
        const size_t stage = a_region + (size_t)N * 128;
        smem = fixed + std::max(stage * (size_t)stages, tile_bytes);
        // at least 46 KB: no fifth CTA (whose TMEM allocation would wait) on an SM
        smem = std::max(smem, (size_t)(46 * 1024));
    } else if (tm) {
        stages = 4;
        while (2 * N + stages * hs * 32 > 256) --stages;
        a.tmem_cols = 256;
        a.a_col0 = (uint32_t)(2 * N);
        const size_t stage = (size_t)hs * (a_region + (size_t)N * 128);
        smem = fixed + std::max(stage * (size_t)stages, tile_bytes);
        // at least 78 KB: no third CTA (whose TMEM allocation would wait) on an SM
        smem = std::max(smem, (size_t)(78 * 1024));
    } else {
        uint32_t cols = 32;
        while (cols < (uint32_t)(a.mma_warps * N)) cols <<= 1;  // one or two accumulators
        a.tmem_cols = cols;
        a.a_col0 = 0;
        const size_t stage = (size_t)hs * (kATile + (uint32_t)N * 128u);
        // two stages (or more if they fit in half the SM) and at most four; the
        // stages must also hold the epilogue tile
        stages = (int)((113 * 1024 - fixed) / stage);
        if (stages < 2) stages = (int)((227 * 1024 - fixed) / stage);
        if (stages > 4) stages = 4;
        while (stages * stage < tile_bytes && fixed + (stages + 1) * stage <= 227 * 1024) ++stages;
        if (stages < 2 || stages * stage < tile_bytes) return cudaErrorInvalidConfiguration;
        smem = fixed + stage * (size_t)stages;
    }
    // the barrier block holds kMaxStages full and empty barriers
    if (stages < 2 || stages > kMaxStages) return cudaErrorInvalidConfiguration;
    a.stages = stages;
    a.maps = maps;
    a.part = part;
    a.n_tiles = n_tiles;
    a.status = status;
    a.par1_used = a.mma_warps == 2 ? par1_used : 0;
    a.K = K;
    a.vec_maps = (maps != nullptr && (J % 2) == 0 && (reinterpret_cast<uintptr_t>(maps) & 7) == 0);
    a.bulk_maps = 0;
    if (maps != nullptr && (J % 4) == 0 && (reinterpret_cast<uintptr_t>(maps) & 15) == 0) {
        // maps written straight into host memory keep the per-thread stores
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, maps) == cudaSuccess &&
            pa.type == cudaMemoryTypeDevice)
            a.bulk_maps = 1;
        (void)cudaGetLastError();
    }
    a.w = static_cast<const uint4 *>(w);
    a.woff = woff;
    a.tile_steps = tile_steps;
    a.all_streamed = (w != nullptr && all_streamed) ? 1 : 0;
    a.fkey = frame_keys;
    // accumulator promotion: conventional FP32 only, with A in TMEM; its running
    // sums take N x 128 floats after the TDOA ring
    a.promote = (conv && split && tm) ? promote : 0;
    if (promote > 0 && a.promote == 0) return cudaErrorInvalidConfiguration;
    if (a.promote > 0) {
        const size_t need = 1024 + 1024 + std::max((size_t)hs * N * 128 * (size_t)stages,
                                                   tile_bytes) +
                            (size_t)kXRing * 128 * sizeof(int2) + (size_t)N * 128 * sizeof(float);
        smem = std::max(smem, need);
        if (smem > 113 * 1024) return cudaErrorInvalidConfiguration;  // two CTAs per SM
    }
    const int grid_y = (L + N - 1) / N;
    const CUtensorMap &map = *reinterpret_cast<const CUtensorMap *>(xi_map);
    if (conv) {
        if (split) return launch_tc_a<true, false, true>(map, a, tm, grid_y, smem, s);
        if (half) return launch_tc_a<false, true, true>(map, a, tm, grid_y, smem, s);
        return launch_tc_a<false, false, true>(map, a, tm, grid_y, smem, s);
    }
    if (streams && tm) {  // generated chunks in TMEM, streamed ones from shared memory
        if (split) return launch_tc<true, false, false, true, true>(map, a, grid_y, smem, s);
        if (half)
            return quad ? launch_tc<false, true, false, true, true, 4>(map, a, grid_y, smem, s)
                        : launch_tc<false, true, false, true, true>(map, a, grid_y, smem, s);
        return quad ? launch_tc<false, false, false, true, true, 4>(map, a, grid_y, smem, s)
                    : launch_tc<false, false, false, true, true>(map, a, grid_y, smem, s);
    }
    if (streams) {
        if (split) return launch_tc<true, false, false, false, true>(map, a, grid_y, smem, s);
        if (half) return launch_tc<false, true, false, false, true>(map, a, grid_y, smem, s);
        return launch_tc<false, false, false, false, true>(map, a, grid_y, smem, s);
    }
    if (split) return launch_tc_a<true, false, false>(map, a, tm, grid_y, smem, s);
    if (half) return launch_tc_a<false, true, false>(map, a, tm, grid_y, smem, s);
    return launch_tc_a<false, false, false>(map, a, tm, grid_y, smem, s);
}

cudaError_t launch_build_w(const int2 *xs, const int4 *ctab, const int32_t *woff, int n_chunks,
                           int64_t J_pad, int xf, int tile_steps, int n_tiles, int precision,
                           void *w, cudaStream_t s) {
    uint4 *dst = static_cast<uint4 *>(w);
    if (precision == SRP_PREC_FP32)
        k_build_w<true, false><<<n_tiles, 128, 0, s>>>(xs, ctab, woff, n_chunks, J_pad, xf, tile_steps, dst);
    else if (precision == SRP_PREC_FP16)
        k_build_w<false, true><<<n_tiles, 128, 0, s>>>(xs, ctab, woff, n_chunks, J_pad, xf, tile_steps, dst);
    else
        k_build_w<false, false><<<n_tiles, 128, 0, s>>>(xs, ctab, woff, n_chunks, J_pad, xf, tile_steps, dst);
    return cudaGetLastError();
}

}  // namespace srp
