// Batched uneven instances: several plans (arrays with their own M, J, K and
// geometry) mapped by one CUDA-graph launch of three kernels:
//   k_batch_operands  PHAT cross spectra (Eq. corrmatrix, PHAT weight) and the
//                     contraction operand B of every (plan, frame, pair) row:
//                     sign-folded critical GCC samples (Eq. GCC_IFT at
//                     tau = nT, Sec. 3.2) or (a_k/K)(Re psi, Im psi)
//                     (conventional map, Sec. 2.4)
//   k_map_batch_tc    one persistent tcgen05 kernel over a work list of
//                     (plan, 128-candidate tile, frame tile) items: the same
//                     contraction as k_interp_tc (Eq. SRPapprox or Eq. GCC_IFT
//                     summed over pairs, Eq. SRP_T_IFT), items of different
//                     plans back to back through one operand pipeline, the
//                     TMEM accumulator double-buffered across items so that
//                     an item's epilogue overlaps the next item's MMAs
//   k_batch_argmax    per-frame first maximiser (Sec. 2.2) of every plan.
// The host spreads the items over the persistent CTAs longest-first onto the
// least-loaded CTA; an autotuner times the candidate tile shapes (frames per
// item, pipeline depth, CTAs per SM) on a real call and keeps the fastest.
//
// Operand B of every plan lives in one chunk-major buffer of 64-slot rows
// (128 bytes of 16-bit data): row b_row0 + (c * hs + h) * Lb + l holds chunk
// c (64 lag or bin slots) of frame l, h = 0 (BF16/FP16 or the high BF16
// part) or 1 (low part, FP32 split), Lb = max_frames rounded up to the frame
// tile.  One TMA descriptor over the whole buffer serves every plan.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <new>
#include <queue>
#include <string>
#include <utility>
#include <vector>

#include "srp_device.cuh"
#include "srp_internal.h"
#include "srp_rescore.cuh"
#include "srp_tc_common.cuh"

namespace srp {
namespace {

using namespace dev;
using namespace tc;

constexpr int kPairBlock = 4;         // pairs per CTA of the operand kernel
constexpr int kMaxSmemCta = 227 * 1024;
constexpr int kSmemPerSm = 228 * 1024;  // shared memory per SM (1 KB of it reserved per CTA)

// Static description of one plan in the batch (device table).
struct BatchInst {
    const int2 *xs;           // [Q][J_pad] (fixed-point TDOA, bits of sp)
    const int4 *ctab;         // [n_chunks] chunk table
    const int2 *pairs;        // [Q] (m, m')
    const int32_t *nq;        // [Q] N_q
    const int32_t *offc;      // [Q] first slot of pair q on the reduction axis
    const float2 *twid;       // [K] (cos, sin)(2 pi j / K); Nyquist only
    unsigned long long *part; // [max_frames][n_tiles] per-tile argmax keys
    int64_t J, J_pad;
    int64_t b_row0;           // first row of the plan's block of operand B
    int M, Q, K, n_aux, xf, n_chunks, n_tiles, par1_used, input_kind, Lb, max_frames;
    int weighting;            // srp_weighting of STFT input
    const uint4 *w;           // resident interpolation matrix of the plan, or null
    const int32_t *woff;      // [n_chunks] first 16-slot step of each chunk in a tile
    int tile_steps;           // 16-slot steps per tile of w
    int all_streamed;         // every chunk's weights are resident: no TDOA table reads
    int pblocks;              // pair blocks of kPairBlock per frame
    int promote;              // FP32 conventional: chunks per accumulator epoch (0: one epoch)
    int64_t op_row0;          // first block of the plan in the operand kernel's grid
    int64_t frame0;           // first block of the plan in the argmax kernel's grid
    // FP32 re-scoring of the maximiser (BF16 / FP16 Nyquist plans that ask for it)
    const int32_t *off;       // [Q] first slot of pair q among the S unpadded samples
    float *x32;               // [max_frames][S32] FP32 samples written by the operand kernel, or null
    int S32;
};

// Per-call arguments of one plan (device table, rewritten by every call).
struct BatchCall {
    const void *in;
    float *maps;
    int32_t *argmax;
    float *peak;
    int L;
    int vec_maps;             // maps rows 8-byte aligned and J even: float2 stores
};

struct PersistArgs {
    const BatchInst *__restrict__ inst;
    const BatchCall *__restrict__ call;
    const int4 *__restrict__ items;      // {plan, tile, l0, items left in the (plan, l0) run},
                                         // CTA lists back to back
    const int32_t *__restrict__ cta_first;  // [gridDim.x + 1]
    int N, stages;
    uint32_t idesc, tmem_cols;
    uint32_t a_col0;        // operand A in TMEM: first column of the A stages
    int mma_warps;          // MMA-issuing warps, each with its own accumulator (1 or 2)
    int *status;
};

// Binary search: the last entry with key(i) <= v among n sorted entries.
template <typename Key>
__device__ __forceinline__ int find_plan(int n, int64_t v, Key key) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key(mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint16_t to16(float v, int fmt_half) {
    if (fmt_half) {
        __half h = __float2half_rn(v);
        return *reinterpret_cast<uint16_t *>(&h);
    }
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t *>(&h);
}

// ---------------------------------------------------------------------------
// Operand kernel: one CTA per (plan, frame, block of kPairBlock pairs), of
// kOpThreads threads (eight warps share a CTA's twiddles and spectrum rows,
// whose shared memory would otherwise bound the SM to four-warp CTAs).
// ---------------------------------------------------------------------------
constexpr int kOpThreads = 256;

template <int kFmt, bool kConv>  // kFmt 0: bf16, 1: bf16 hi/lo split, 2: fp16
__global__ void __launch_bounds__(kOpThreads) k_batch_operands(const BatchInst *__restrict__ inst,
                                                        const BatchCall *__restrict__ call,
                                                        int n, uint16_t *__restrict__ b16) {
    extern __shared__ float2 sm[];
    const int64_t blk = blockIdx.x;
    const int p = find_plan(n, blk, [&](int i) { return inst[i].op_row0; });
    const BatchInst &I = inst[p];
    const int L = call[p].L;
    const int64_t rr = blk - I.op_row0;
    const int l = (int)(rr / I.pblocks), pb = (int)(rr % I.pblocks);
    if (l >= L) return;
    const int K = I.K, Kb = K / 2 + 1, Q = I.Q;
    const int hs = kFmt == 1 ? 2 : 1;
    const float2 *in = static_cast<const float2 *>(call[p].in);
    float2 *tw = sm, *ps = sm + K;  // Nyquist: twiddles, then kPairBlock spectrum rows
    const int q0 = pb * kPairBlock, np = min(Q, q0 + kPairBlock) - q0;
    // slot s of frame l, part h, lives at row b_row0 + ((s >> 6) hs + h) Lb + l
    auto elem = [&](int s, int h) -> size_t {
        return (size_t)(I.b_row0 + (int64_t)((s >> 6) * hs + h) * I.Lb + l) * 64 + (s & 63);
    };
    // cross spectrum of pair q0 + j, bin k
    auto cross = [&](int j, int k) -> float2 {
        const int q = q0 + j;
        if (I.input_kind == SRP_IN_STFT) {
            const int2 pr = I.pairs[q];
            const float2 ym = in[((size_t)l * I.M + pr.x) * Kb + k];
            const float2 ymp = in[((size_t)l * I.M + pr.y) * Kb + k];
            if (I.weighting == SRP_WEIGHT_NONE) return times_conj(ym, ymp);  // y_m y_m'^*
            return times_conj(unit_phase(ym), unit_phase(ymp));
        }
        return in[((size_t)l * Q + q) * Kb + k];
    };
    if (kConv) {
        for (int j = 0; j < np; ++j)
        for (int k = threadIdx.x; k < Kb; k += blockDim.x) {
            const float2 v = cross(j, k);
            const float a = ((k == 0 || 2 * k == K) ? 1.0f : 2.0f) / (float)K;
            const float re = a * v.x, im = a * v.y;
            const int s = I.offc[q0 + j] + 2 * k;
            uint32_t h, lo = 0;
            if (kFmt == 2) {
                h = pack_f16(re, im);
            } else {
                h = pack_bf16(re, im);
                if (kFmt == 1)
                    lo = pack_bf16(re - __uint_as_float(h << 16),
                                   im - __uint_as_float(h & 0xFFFF0000u));
            }
            *reinterpret_cast<uint32_t *>(b16 + elem(s, 0)) = h;
            if (kFmt == 1) *reinterpret_cast<uint32_t *>(b16 + elem(s, 1)) = lo;
        }
        return;
    }
    // Nyquist: a_k psi of every pair of the block, then its critical samples.
    // The loads of a bin for all the block's pairs are issued before any
    // arithmetic, so that their latencies overlap.
    copy_twiddles_async(I.twid, K, tw);
    const bool stft = I.input_kind == SRP_IN_STFT;
    for (int k = threadIdx.x; k < Kb; k += blockDim.x) {
        float2 u[kPairBlock], v[kPairBlock];
#pragma unroll
        for (int j = 0; j < kPairBlock; ++j) {
            if (j < np) {
                if (stft) {
                    const int2 pr = I.pairs[q0 + j];
                    u[j] = in[((size_t)l * I.M + pr.x) * Kb + k];
                    v[j] = in[((size_t)l * I.M + pr.y) * Kb + k];
                } else {
                    u[j] = in[((size_t)l * Q + q0 + j) * Kb + k];
                }
            }
        }
        const float a = (k == 0 || 2 * k == K) ? 1.0f : 2.0f;
#pragma unroll
        for (int j = 0; j < kPairBlock; ++j) {
            if (j < np) {
                float2 c = u[j];
                if (stft)
                    c = I.weighting == SRP_WEIGHT_NONE ? times_conj(u[j], v[j])
                                                       : times_conj(unit_phase(u[j]), unit_phase(v[j]));
                ps[j * Kb + k] = make_float2(a * c.x, a * c.y);
            }
        }
    }
    wait_async_copies();
    __syncthreads();
    gcc_rows(tw, ps, Kb, np, K, [&](int j) { return I.nq[q0 + j] + I.n_aux; },
             [&](int j, int t, int nl, float v) {
                 if (I.x32 != nullptr) I.x32[(size_t)l * I.S32 + I.off[q0 + j] + t] = v;
                 if (nl & 1) v = -v;
                 const int s = I.offc[q0 + j] + t;
                 const uint16_t h = to16(v, kFmt == 2);
                 b16[elem(s, 0)] = h;
                 if (kFmt == 1) {
                     __nv_bfloat16 hb = *reinterpret_cast<const __nv_bfloat16 *>(&h);
                     b16[elem(s, 1)] = to16(v - __bfloat162float(hb), 0);
                 }
             });
}

// ---------------------------------------------------------------------------
// Argmax kernel: one CTA per (plan, frame).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_batch_argmax(const BatchInst *__restrict__ inst,
                                                      const BatchCall *__restrict__ call, int n) {
    __shared__ unsigned long long red[8];
    const int64_t blk = blockIdx.x;
    const int p = find_plan(n, blk, [&](int i) { return inst[i].frame0; });
    const BatchInst &I = inst[p];
    const int l = (int)(blk - I.frame0);
    if (l >= call[p].L) return;
    const unsigned long long *part = I.part + (size_t)l * I.n_tiles;
    unsigned long long k = 0ull;
    for (int t = threadIdx.x; t < I.n_tiles; t += blockDim.x) {
        const unsigned long long v = part[t];
        k = v > k ? v : k;
    }
    k = warp_max_u64(k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x < 32) {
        k = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
        k = warp_max_u64(k);
        if (threadIdx.x == 0) {
            call[p].argmax[l] = (int32_t)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull));
            if (call[p].peak != nullptr) call[p].peak[l] = key_value(k);
        }
    }
}

// ---------------------------------------------------------------------------
// Argmax with FP32 re-scoring: one CTA of kBrsThreads per (plan, frame).  For
// a plan with FP32 samples (x32), the tiles whose reduced-precision maximum
// is at least m - kRescoreDelta |m| (m the frame's maximum) are evaluated
// again candidate by candidate in FP32 (Eq. SRPapprox, rs::nyquist_at: four
// threads per candidate over quarters of the pairs, added in a fixed order),
// as srp_map does for such a plan; the lowest-index maximiser of those values
// is the frame's argmax and its FP32 value the peak.  Other plans, and frames
// with more than kRescoreMaxTiles such tiles (a nearly flat map), keep the
// reduced-precision maximiser.
// ---------------------------------------------------------------------------
constexpr int kBrsParts = 4, kBrsThreads = kBrsParts * kTileJ, kBrsWarps = kBrsThreads / 32;
constexpr int kBrsSmemFloats = 12 * 1024;  // a frame's FP32 samples staged in shared memory (48 KB)
constexpr int kBrsCandCap = 2048;          // candidates scored one by one (else whole tiles)
static_assert(kBrsThreads >= kRescoreMaxTiles, "one thread per selected tile when sorting");

__device__ __forceinline__ unsigned long long block_max_brs(unsigned long long k,
                                                            unsigned long long *red) {
    k = warp_max_u64(k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
    __syncthreads();
    k = 0ull;
#pragma unroll
    for (int w = 0; w < kBrsWarps; ++w) k = red[w] > k ? red[w] : k;
    __syncthreads();
    return k;
}

__global__ void __launch_bounds__(kBrsThreads) k_batch_rescore(const BatchInst *__restrict__ inst,
                                                                const BatchCall *__restrict__ call,
                                                                int n) {
    __shared__ unsigned long long red[kBrsWarps];
    __shared__ int tiles[kRescoreMaxTiles];
    __shared__ int n_sel, n_cand;
    __shared__ int cand[kBrsCandCap];
    __shared__ float part_sum[kBrsParts * kTileJ];
    extern __shared__ float xi_sm[];
    const int64_t blk = blockIdx.x;
    const int p = find_plan(n, blk, [&](int i) { return inst[i].frame0; });
    const BatchInst &I = inst[p];
    const int l = (int)(blk - I.frame0);
    if (l >= call[p].L) return;
    const unsigned long long *part = I.part + (size_t)l * I.n_tiles;
    unsigned long long k = 0ull;
    for (int t = threadIdx.x; t < I.n_tiles; t += blockDim.x) {
        const unsigned long long v = part[t];
        k = v > k ? v : k;
    }
    const unsigned long long kmax = block_max_brs(k, red);
    const float m = key_value(kmax);
    unsigned long long best = kmax;
    if (I.x32 != nullptr) {
        if (threadIdx.x == 0) n_sel = 0;
        __syncthreads();
        const uint32_t otau = ordered_value(m - kRescoreDelta * fabsf(m));
        for (int t = threadIdx.x; t < I.n_tiles; t += blockDim.x)
            if ((uint32_t)(part[t] >> 32) >= otau) {
                const int slot = atomicAdd(&n_sel, 1);
                if (slot < kRescoreMaxTiles) tiles[slot] = t;
            }
        __syncthreads();
        const int ns = n_sel;
        if (ns <= kRescoreMaxTiles) {
            // ascending tile order (the atomics fill the list in any order)
            int tt = 0, rank = 0;
            if (threadIdx.x < ns) {
                tt = tiles[threadIdx.x];
                for (int j = 0; j < ns; ++j) rank += tiles[j] < tt ? 1 : 0;
            }
            __syncthreads();
            if (threadIdx.x < ns) tiles[rank] = tt;
            __syncthreads();
            // the frame's FP32 samples, in shared memory when they fit
            const float *xr = I.x32 + (size_t)l * I.S32;
            if (I.S32 <= kBrsSmemFloats) {
                for (int t = threadIdx.x; t < I.S32; t += blockDim.x) xi_sm[t] = xr[t];
                __syncthreads();
                xr = xi_sm;
            }
            // the candidates that reach the threshold in the map when it is
            // written, else every candidate of the tiles
            const float *maps_row =
                call[p].maps != nullptr ? call[p].maps + (size_t)l * I.J : nullptr;
            unsigned long long b = rs::score_candidates<kBrsParts>(
                tiles, 0, 1, ns, maps_row, otau, I.J, cand, kBrsCandCap, &n_cand, part_sum,
                [&](int64_t i, int q) {
                    return rs::nyquist_at(I.xs, I.J_pad, i, I.Q, I.xf, I.nq, I.off, I.n_aux, xr,
                                          q, kBrsParts);
                });
            b = block_max_brs(b, red);
            if (b != 0ull) best = b;
        }
    }
    if (threadIdx.x == 0) {
        call[p].argmax[l] = (int32_t)(0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFull));
        if (call[p].peak != nullptr) call[p].peak[l] = key_value(best);
    }
}

// AND of v over the 128 threads of warps 0-3 (named barrier 1).
__device__ __forceinline__ bool and_128(bool v) {
    uint32_t r;
    asm volatile(
        "{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.and.pred q, 1, 128, p; "
        "selp.u32 %0, 1, 0, q; }"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void sync_128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// ---------------------------------------------------------------------------
// The persistent contraction.  Warps 0-3 generate operand A (one candidate
// row per thread) and run the epilogue of the previous item after the
// operands of the current one; warp 4 issues the TMA loads of B; warps 5-6
// issue the MMAs into two accumulators by the parity of the item's running
// 16-slot step count (or warp 5
// alone into one, mma_warps = 1).  TMEM holds two such accumulator sets (item
// parity), columns [b W N, b W N + W N) for W = mma_warps.
// ---------------------------------------------------------------------------
// kTm: operand A is generated into TMEM after the accumulators (32 columns per
// stage and part) and the MMAs read only B from shared memory.  kOcc: CTAs per
// SM the registers are sized for (2, or 4 for the 16-bit formats in 128 TMEM
// columns per CTA).
// kPr (FP32 conventional, A in TMEM): items of plans with I.promote > 0 have
// their accumulators promoted every I.promote chunks into per-row FP32 sums
// rs[frame][row] in shared memory (as in the single-plan kernel), and run
// their epilogue right after their own chunks, so that one set of sums serves
// every item.
template <bool kSplit, bool kHalf, bool kConv, bool kTm, int kOcc = 2, bool kPr = false>
__global__ void __launch_bounds__(kThreads, kOcc) k_map_batch_tc(const __grid_constant__ CUtensorMap tmap,
                                                                 const PersistArgs a) {
    static_assert(!kPr || (kConv && kSplit && kTm), "promotion: FP32 conventional, TMEM A");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    // full[kMaxStages], empty[kMaxStages], acc_full[2], acc_empty[2], drain
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + 128);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + 132);
    const int N = a.N;
    const uint32_t b_tile = (uint32_t)N * 128u;
    const uint32_t stage_bytes = (kSplit ? 2u : 1u) * ((kTm ? 0u : kATile) + b_tile);
    const uint32_t stage0 = base + 1024u;
    const uint32_t xring = stage0 + stage_bytes * (uint32_t)a.stages;
    float *mt = reinterpret_cast<float *>(gbase + 1024u + stage_bytes * (uint32_t)a.stages +
                                          (uint32_t)kXRing * 128u * 8u);
    float *rs = mt + (size_t)N * kMtStride;  // kPr: running sums of the promoted item

    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[kMaxStages + s]); };
    auto acc_full = [&](int b) { return smem_u32(&bars[2 * kMaxStages + b]); };
    auto acc_empty = [&](int b) { return smem_u32(&bars[2 * kMaxStages + 2 + b]); };
    const uint32_t drain = smem_u32(&bars[2 * kMaxStages + 4]);
    const uint32_t epoch_bar = smem_u32(&bars[2 * kMaxStages + 5]);    // kPr: the epoch's MMAs done
    const uint32_t drained_bar = smem_u32(&bars[2 * kMaxStages + 6]);  // kPr: accumulators read
    static_assert((2 * kMaxStages + 7) * 8 <= 128, "barrier block overlaps the TMEM slot");
    auto a_hi = [&](int s) { return stage0 + (uint32_t)s * stage_bytes; };
    auto a_lo = [&](int s) { return stage0 + (uint32_t)s * stage_bytes + kATile; };
    auto b_hi = [&](int s) {
        return stage0 + (uint32_t)s * stage_bytes + (kTm ? 0u : (kSplit ? 2u : 1u) * kATile);
    };
    auto b_lo = [&](int s) { return b_hi(s) + b_tile; };
    auto a_tm = [&](int s, int part) {
        return a.a_col0 + ((uint32_t)s * (kSplit ? 2u : 1u) + (uint32_t)part) * 32u;
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it0 = a.cta_first[blockIdx.x], it1 = a.cta_first[blockIdx.x + 1];
    auto live = [&](const int4 &it) { return it.z < a.call[it.x].L; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full_bar(s), 128 + 1);
            mbar_init(empty_bar(s), a.mma_warps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), a.mma_warps);
            mbar_init(acc_empty(b), 128);
        }
        mbar_init(drain, a.mma_warps);
        mbar_init(epoch_bar, a.mma_warps);
        mbar_init(drained_bar, 128);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kTmaWarp) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        const int r = threadIdx.x;
        const uint32_t row = (uint32_t)r * 128u, sw = (uint32_t)(r & 7);
        // (TDOA, sp) of the pairs of all live items, streamed kXAhead pairs
        // ahead of their use through the ring (entry e in slot e % kXRing, one
        // commit group per entry).
        int li = it0, lq = 0, lQ = 0, seq_load = 0, seq_use = 0;
        const int2 *lxs = nullptr;
        int64_t ljp = 0;
        auto load_next = [&]() {
            if (lq == 0) {
                // dead items, and items of plans whose weights are all resident,
                // read no TDOA table
                // (both hold for a whole (plan, frame tile) run)
                while (li < it1 && (!live(a.items[li]) ||
                                    (!kConv && !kTm && a.inst[a.items[li].x].all_streamed)))
                    li += a.items[li].w;
                if (li < it1) {
                    const int4 it = a.items[li];
                    const BatchInst &I = a.inst[it.x];
                    lxs = I.xs + (int64_t)it.y * 128 + r;
                    ljp = I.J_pad;
                    lQ = I.Q;
                }
            }
            if (li < it1) {
                cp_async8(xring + (uint32_t)((seq_load % kXRing) * 128 + r) * 8u,
                          lxs + (size_t)lq * ljp);
                if (++lq == lQ) {
                    lq = 0;
                    ++li;
                }
            }
            cp_async_commit();
            ++seq_load;
        };
        int32_t nX = 0, nsp = 0;  // (TDOA, sp) of the next pair to start
        auto read_next = [&]() {
            cp_async_wait<kXAhead - 1>();
            asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];"
                         : "=r"(nX), "=r"(nsp)
                         : "r"(xring + (uint32_t)((seq_use % kXRing) * 128 + r) * 8u));
            ++seq_use;
            load_next();
        };
#pragma unroll 1
        for (int k = 0; k < kXAhead; ++k) load_next();
        read_next();

        // epilogue of live item P (the kp-th): TMEM -> mt -> maps and argmax keys
        auto epilogue = [&](const int4 &P, int kp) {
            const int b = kp & 1;
            const bool ok = mbar_wait(acc_full(b), (uint32_t)(kp >> 1) & 1u, abort_flag, a.status);
            if (!and_128(ok)) return;
            tc_fence_after();
            const BatchInst &I = a.inst[P.x];
            const BatchCall &C = a.call[P.x];
            const uint32_t trow =
                tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * a.mma_warps * N);
            const int par1 = a.mma_warps == 2 && I.par1_used;
            for (int j0 = 0; j0 < N; j0 += 16) {
                float v[16];
                tmem_ld16(trow + (uint32_t)j0, v);
                if (par1) {
                    float v1[16];
                    tmem_ld16(trow + (uint32_t)(N + j0), v1);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) v[jj] += v1[jj];
                }
                if (kPr && I.promote > 0) {
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) v[jj] += rs[(j0 + jj) * 128 + r];
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) mt[(j0 + jj) * kMtStride + r] = v[jj];
            }
            tc_fence_before();
            mbar_arrive(acc_empty(b));  // accumulator set b may be overwritten
            sync_128();
            const int64_t J = I.J, tile0 = (int64_t)P.y * 128;
            const int l0 = P.z, n_rows = min(N, C.L - l0);
            if (C.maps != nullptr) {  // warp w writes frame rows w, w + 4, ...
                for (int fr = warp; fr < n_rows; fr += 4) {
                    float *dst = C.maps + (size_t)(l0 + fr) * J + tile0;
                    const float *srcr = mt + fr * kMtStride;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int k = 2 * (lane + 32 * hh);
                        const float2 val = *reinterpret_cast<const float2 *>(srcr + k);
                        if (C.vec_maps && tile0 + k + 1 < J) {
                            *reinterpret_cast<float2 *>(dst + k) = val;
                        } else {
                            if (tile0 + k < J) dst[k] = val.x;
                            if (tile0 + k + 1 < J) dst[k + 1] = val.y;
                        }
                    }
                }
            }
            // first maximiser per frame: threads 2f and 2f+1 scan even / odd candidates
            const int kmax = (int)min((int64_t)128, J - tile0);
            for (int fr = r >> 1; fr < n_rows + 63 - ((n_rows + 63) % 64); fr += 64) {
                const int h = r & 1;
                unsigned long long key = 0ull;
                if (fr < n_rows) {
                    uint32_t bo = 0u;
                    int bk = -1;
                    const float *row_p = mt + fr * kMtStride;
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
                if (h == 0 && fr < n_rows) I.part[(size_t)(l0 + fr) * I.n_tiles + P.y] = key;
            }
            sync_128();  // mt is free for the next epilogue
        };

        int g = 0, kx = 0;   // chunks and live items so far
        int st = 0;          // stage of chunk g, and the parity of its use
        uint32_t ph = 0;
        uint32_t epar = 0;   // kPr: parity of the next accumulator epoch to end
        int4 prev = make_int4(-1, 0, 0, 0);
        for (int t = it0; t < it1; ++t) {
            const int4 it = a.items[t];
            if (!live(it)) {  // skip the rest of this (plan, frame tile) run
                t += it.w - 1;
                continue;
            }
            if (!and_128(*abort_flag == 0)) break;
            const BatchInst &I = a.inst[it.x];
            const int n_chunks = I.n_chunks, xf = I.xf;
            const int4 *ctab = I.ctab;
            const bool resident = !kConv && !kTm && I.w != nullptr;  // some chunks streamed
            const bool skip_ring = resident && I.all_streamed;      // no weights generated
            int q = -1;
            float sp = 0.0f, f = 0.5f, x0f = 0.0f;
            int x0m = 0;
            float wp = 1.0f, wq = 0.0f;
            const int K = I.K;
            const float two_k = 2.0f / (float)K;
            const int prom = kPr ? I.promote : 0;
            if (prom > 0)  // the running sums start at zero (each thread owns its row)
                for (int j = 0; j < N; ++j) rs[j * 128 + r] = 0.0f;
            bool drained_ok = true;
            int4 cur = __ldg(&ctab[0]);
            for (int c = 0; c < n_chunks; ++c, ++g) {
                const int4 nxt = __ldg(&ctab[c + 1 < n_chunks ? c + 1 : c]);
                if (cur.x != q && !skip_ring) {  // uniform: a new pair starts with this chunk
                    q = cur.x;
                    int x0;
                    decode_tdoa(nX, xf, x0, f);
                    if (kConv) {
                        x0m = ((x0 % K) + K) % K;
                        float sn, cs;
                        sincospif(((float)x0 + f) * two_k, &sn, &cs);
                        wp = cs;
                        wq = -sn;
                    } else {
                        if (f == 0.0f) f = 9.094947017729282e-13f;  // 2^-40, as in the plan
                        sp = __int_as_float(nsp);
                        x0f = (float)x0;
                    }
                    read_next();
                }
                // the weights are computed into registers before the stage wait
                const uint32_t eb = empty_bar(st), eph = ph ^ 1u;
                const bool reuse = g >= a.stages;
                auto wait_free = [&]() {
                    if (reuse && !mbar_try_wait(eb, eph)) mbar_wait(eb, eph, abort_flag, a.status);
                };
                const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
                const uint32_t d0 = kTm ? tmem + lane_base + a_tm(st, 0) : a_hi(st) + row;
                const uint32_t d1 = kTm ? tmem + lane_base + a_tm(st, 1) : 0u;
                const int ng = cur.z;
                if (resident && __ldg(&I.woff[c]) >= 0) {
                    // the TMA warp brings this chunk's A; only the stage protocol below
                    wait_free();
                } else if (kConv) {
                    const int k0 = cur.y;
                    const int rk = (int)(((long long)k0 * x0m) % K);
                    float sn, cs;
                    sincospif(fmaf((float)rk, two_k, (float)k0 * f * two_k), &sn, &cs);
                    switch (ng) {
                        case 2: gen_steer<2, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                        case 4: gen_steer<4, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                        case 6: gen_steer<6, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                        default: gen_steer<8, kSplit, kHalf, kTm>(d0, d1, sw, cs, -sn, wp, wq, 0u, nullptr, nullptr, wait_free); break;
                    }
                } else {
                    const float mc = x0f + __int_as_float(cur.y);
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
                if (prom > 0 && c > 0 && c % max(prom, 1) == 0) {
                    // the epoch ended with chunk c - 1: once its MMAs are done,
                    // add the item's accumulators to the running sums and
                    // release them
                    if (!mbar_wait(epoch_bar, epar, abort_flag, a.status)) {
                        drained_ok = false;
                        break;
                    }
                    epar ^= 1u;
                    tc_fence_after();
                    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) +
                                          (uint32_t)((kx & 1) * a.mma_warps * N);
                    for (int j0 = 0; j0 < N; j0 += 16) {
                        float v[16];
                        tmem_ld16(trow + (uint32_t)j0, v);
                        if (a.mma_warps == 2 && I.par1_used) {
                            float v1[16];
                            tmem_ld16(trow + (uint32_t)(N + j0), v1);
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
            if (kPr && !and_128(drained_ok)) break;
            if (prev.x >= 0) epilogue(prev, kx - 1);
            prev = it;
            if (prom > 0) {  // its sums are needed by no later item: finish it now
                epilogue(it, kx);
                prev = make_int4(-1, 0, 0, 0);
            }
            ++kx;
        }
        if (prev.x >= 0) epilogue(prev, kx - 1);
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == kTmaWarp) {
        // ---------------- B loads ----------------
        if (lane == 0) {
            const uint32_t bytes = (kSplit ? 2u : 1u) * b_tile;
            int g = 0, issued = 0;
            int st = 0;  // stage of chunk g, and the parity of its use
            uint32_t ph = 0;
            bool ok = true;
            for (int t = it0; t < it1 && ok; ++t) {
                const int4 it = a.items[t];
                if (!live(it)) {
                    t += it.w - 1;
                    continue;
                }
                const BatchInst &I = a.inst[it.x];
                const int n_chunks = I.n_chunks, Lb = I.Lb;
                const int64_t r0 = I.b_row0 + it.z;
                for (int c = 0; c < n_chunks; ++c, ++g) {
                    if (g >= a.stages && !mbar_wait(empty_bar(st), ph ^ 1u, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const int wo = (!kConv && !kTm && I.w != nullptr) ? __ldg(&I.woff[c]) : -1;
                    if (wo >= 0) {  // resident A: the chunk's used steps
                        const int4 cc = __ldg(&I.ctab[c]);
                        const uint32_t a_bytes = (uint32_t)cc.w * kAStep;
                        const uint4 *src = I.w + ((size_t)it.y * I.tile_steps + wo) *
                                                     (kSplit ? 2 : 1) * (kAStep / 16);
                        mbar_arrive_expect_tx(full_bar(st), bytes + (kSplit ? 2u : 1u) * a_bytes);
                        bulk_load(a_hi(st), src, a_bytes, full_bar(st));
                        if (kSplit) bulk_load(a_lo(st), src + a_bytes / 16, a_bytes, full_bar(st));
                    } else {
                        mbar_arrive_expect_tx(full_bar(st), bytes);
                    }
                    const int y = (int)(r0 + (int64_t)c * (kSplit ? 2 : 1) * Lb);
                    tma_load_2d(b_hi(st), &tmap, 0, y, full_bar(st));
                    if (kSplit) tma_load_2d(b_lo(st), &tmap, 0, y + Lb, full_bar(st));
                    issued = g + 1;
                    if (++st == a.stages) {
                        st = 0;
                        ph ^= 1u;
                    }
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
        // ---------------- MMA issue ----------------
        // The whole warp runs the loop on values broadcast from lane 0 (work
        // items, plan fields, chunk-table entries, the TMEM base), so that
        // every branch and every MMA operand is uniform, and one elected lane
        // issues the chunk's MMAs with the commits that track them.
        const int par = warp - kMmaWarp0, nw = a.mma_warps;
        if (par < nw) {
            const uint32_t tm = __shfl_sync(0xFFFFFFFFu, tmem, 0);
            auto bc = [](int v) { return __shfl_sync(0xFFFFFFFFu, v, 0); };
            auto bcp = [](const void *p) {
                return reinterpret_cast<const void *>(
                    __shfl_sync(0xFFFFFFFFu, reinterpret_cast<unsigned long long>(p), 0));
            };
            int kx = 0, st = 0;  // live items so far; stage of the next chunk
            uint32_t ph = 0;     // parity of the stage's use
            uint32_t eph = 0;    // kPr: parity of the next epoch drain
            bool ok = true;
            for (int t = it0; t < it1 && ok; ++t) {
                int4 it = a.items[t];
                it = make_int4(bc(it.x), bc(it.y), bc(it.z), bc(it.w));
                if (!bc(live(it) ? 1 : 0)) {
                    t += it.w - 1;
                    continue;
                }
                const BatchInst &I = a.inst[it.x];
                const int b = kx & 1;
                const bool e_ok = mbar_wait(acc_empty(b), ((uint32_t)(kx >> 1) & 1u) ^ 1u,
                                            abort_flag, a.status);
                if (!__all_sync(0xFFFFFFFFu, e_ok)) break;
                tc_fence_after();
                const uint32_t dt = tm + (uint32_t)((b * nw + par) * N);
                uint32_t acc = 0;  // the item's first MMA overwrites the accumulator
                int g0 = 0;        // 16-slot steps of the item's earlier chunks
                const int n_chunks = bc(I.n_chunks);
                const int4 *ctab = reinterpret_cast<const int4 *>(bcp(I.ctab));
                const bool resident = !kConv && !kTm && bcp(I.w) != nullptr;
                const int32_t *woff =
                    resident ? reinterpret_cast<const int32_t *>(bcp(I.woff)) : nullptr;
                const int prom = kPr ? bc(I.promote) : 0;
                int ep = 0;  // chunks into the current accumulator epoch
                // the next chunk's table entry is loaded a chunk ahead
                int nk_next = bc(__ldg(&ctab[0]).w);
                bool streamed_next = resident && bc(__ldg(&woff[0])) >= 0;
                for (int c = 0; c < n_chunks; ++c) {
                    const int nk = nk_next;
                    const bool streamed = streamed_next;
                    if (prom > 0 && ep == prom) {
                        // the epoch's MMAs were committed to epoch_bar with its
                        // last chunk; once the generators have read the
                        // accumulators, the next MMA into each starts it afresh
                        const bool d_ok = mbar_try_wait(drained_bar, eph) ||
                                          mbar_wait(drained_bar, eph, abort_flag, a.status);
                        if (!__all_sync(0xFFFFFFFFu, d_ok)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        eph ^= 1u;
                        acc = 0;
                        ep = 0;
                    }
                    if (c + 1 < n_chunks) {
                        nk_next = bc(__ldg(&ctab[c + 1]).w);
                        streamed_next = resident && bc(__ldg(&woff[c + 1])) >= 0;
                    }
                    const uint64_t dah = smem_desc_sw128(a_hi(st)), dbh = smem_desc_sw128(b_hi(st));
                    const uint64_t dal = smem_desc_sw128(a_lo(st)), dbl = smem_desc_sw128(b_lo(st));
                    const uint32_t tah = tm + a_tm(st, 0), tal = tm + a_tm(st, 1);
                    const bool f_ok = mbar_try_wait(full_bar(st), ph) ||
                                      mbar_wait(full_bar(st), ph, abort_flag, a.status);
                    if (!__all_sync(0xFFFFFFFFu, f_ok)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // steps alternate over the nw accumulators by the running
                    // step count of the item (balanced chains)
                    const int kk0 = nw == 1 ? 0 : (par + g0) & 1;
                    g0 += nk;
                    ++ep;
                    const bool last = c + 1 == n_chunks;
                    const bool epoch_end = prom > 0 && ep == prom && !last;
                    if (elect_one()) {
#pragma unroll
                        for (int s = 0; s < kChunk / 16; ++s) {
                            const int kk = kk0 + s * nw;
                            if (kk >= nk) break;
                            const uint32_t acc_s = s > 0 ? 1u : acc;
                            const uint64_t adv = (uint64_t)(kk * 2);
                            const uint32_t ac = (uint32_t)(kk * 8);
                            if (kTm) {
                                mma_f16_ts(dt, tah + ac, dbh + adv, a.idesc, acc_s);
                                if (kSplit) {
                                    mma_f16_ts(dt, tah + ac, dbl + adv, a.idesc, 1);
                                    mma_f16_ts(dt, tal + ac, dbh + adv, a.idesc, 1);
                                }
                            } else if (streamed) {  // A blocks without swizzle, kAStep per step
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
                        if (last) mma_commit(acc_full(b));
                    }
                    __syncwarp();
                    if (kk0 < nk) acc = 1;
                    if (++st == a.stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                if (n_chunks == 0 && elect_one()) mma_commit(acc_full(b));  // (no plan has none)
                __syncwarp();
                ++kx;
            }
            // arrives once every MMA issued above has completed
            if (elect_one()) mma_commit(drain);
            __syncwarp();
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == kTmaWarp) {
        tc_fence_after();
        const uint64_t t0 = global_timer();
        while (!mbar_try_wait(drain, 0) && global_timer() - t0 < kWaitLimitNs) {
        }
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

struct TileChoice {
    int N = 0, stages = 0, cps = 0;
    bool tm = false;  // operand A in TMEM
    int mw = 2;       // MMA-issuing warps = accumulators per item
};

// Bytes of shared memory of the persistent kernel for a tile choice (with
// promote, the running sums of a promoted item after the epilogue tile).
size_t persist_smem(const TileChoice &t, bool split, bool promote) {
    const size_t stage = (split ? 2 : 1) * ((t.tm ? 0 : (size_t)kATile) + (size_t)t.N * 128);
    return 2048 + stage * t.stages + (size_t)kXRing * 128 * 8 + (size_t)t.N * kMtStride * 4 +
           (promote ? (size_t)t.N * 128 * 4 : 0);
}

// TMEM columns: two accumulator sets of mw accumulators (2 mw N) and, with A
// in TMEM, 32 per stage and part; rounded up to a power of two (the
// allocation unit).
uint32_t persist_tmem_cols(const TileChoice &t, bool split) {
    const uint32_t need = (uint32_t)(2 * t.mw * t.N) +
                          (t.tm ? (uint32_t)(t.stages * (split ? 2 : 1) * 32) : 0u);
    uint32_t cols = 32;
    while (cols < need) cols <<= 1;
    return cols;
}

bool tile_fits(const TileChoice &t, bool split, bool any_resident, bool one_acc, bool promote) {
    if (t.N < 16 || t.N > 256 || (t.N & 15)) return false;
    if (t.tm && any_resident) return false;  // streamed A blocks live in shared memory
    if (promote && (!t.tm || t.cps > 2)) return false;  // the promoting kernel: A in TMEM
    if (t.stages < 2 || t.stages > kMaxStages || t.cps < 1 || t.cps > 4 || t.cps == 3)
        return false;
    // four CTAs per SM: 16-bit formats with A in TMEM (the register budget of the
    // FP32 split does not fit)
    if (t.cps == 4 && (split || !t.tm)) return false;
    if (t.mw < 1 || t.mw > 2 || (t.mw == 1 && !one_acc)) return false;
    if (persist_tmem_cols(t, split) * (uint32_t)t.cps > 512u) return false;
    const size_t smem = persist_smem(t, split, promote);
    if (smem > (size_t)kMaxSmemCta) return false;
    return (smem + 1024) * (size_t)t.cps <= (size_t)kSmemPerSm;
}

int round_up_int(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace
}  // namespace srp

using namespace srp;

struct srp_batch_s {
    int device = 0;
    int sm_count = 0;
    std::vector<srp_plan_s *> plans;
    srp_mode mode = SRP_MODE_NYQUIST;
    srp_precision precision = SRP_PREC_FP32;
    bool split = false, half = false;
    int max_L = 0, max_K = 0;
    bool any_resident = false;  // some plan streams its interpolation matrix: A in shared memory
    bool one_acc = true;        // one accumulator per item keeps the FP32 bias within its limit
    bool promote = false;       // some plan's FP32 accumulators are promoted (long conventional sums)
    TileChoice tiles;
    int n_ctas = 0, n_items = 0;
    int64_t op_blocks = 0, frame_blocks = 0, b_rows = 0;
    std::vector<BatchInst> inst;
    BatchInst *d_inst = nullptr;
    BatchCall *d_call = nullptr;
    BatchCall *h_call = nullptr;  // pinned staging of the per-call table
    int4 *d_items = nullptr;
    int32_t *d_cta_first = nullptr;
    size_t items_cap = 0, cta_cap = 0;
    uint16_t *d_b = nullptr;
    size_t b_cap = 0;
    unsigned long long *d_part = nullptr;
    size_t part_bytes = 0;
    float *d_x32 = nullptr;     // FP32 samples of the plans whose maximiser is re-scored
    bool rescore = false;       // some plan re-scores its maximiser (the argmax kernel does)
    int *d_status = nullptr;
    alignas(64) unsigned char b_map[128] = {};
    // the three kernels of a call, as captured in the graph
    void (*operands)(const BatchInst *, const BatchCall *, int, uint16_t *) = nullptr;
    void (*persist)(const CUtensorMap, const PersistArgs) = nullptr;
    size_t op_smem = 0, persist_smem_bytes = 0;
    PersistArgs pargs = {};
    int timing = 0;  // calls launch the kernels directly, with events between them
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[4] = {};
    cudaEvent_t copied = nullptr;
    int tuned = 0;
    float tuned_ms = 0.0f;
};

namespace srp {
namespace {

void batch_release(srp_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto &e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->copied) cudaEventDestroy(b->copied);
    cudaFree(b->d_inst);
    cudaFree(b->d_call);
    cudaFreeHost(b->h_call);
    cudaFree(b->d_items);
    cudaFree(b->d_cta_first);
    cudaFree(b->d_b);
    cudaFree(b->d_part);
    cudaFree(b->d_x32);
    cudaFree(b->d_status);
}

template <typename T>
cudaError_t grow(T **p, size_t &cap, size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
}

// The three kernels of a call on stream s (captured into the graph, or
// launched directly with events around each when timing).
cudaError_t enqueue_kernels(srp_batch_s *b, cudaStream_t s, bool timed) {
    const int n = (int)b->plans.size();
    const CUtensorMap &map = *reinterpret_cast<const CUtensorMap *>(b->b_map);
    if (timed) cudaEventRecord(b->ev[0], s);
    b->operands<<<(unsigned)b->op_blocks, kOpThreads, b->op_smem, s>>>(b->d_inst, b->d_call, n,
                                                                       b->d_b);
    if (timed) cudaEventRecord(b->ev[1], s);
    b->persist<<<(unsigned)b->n_ctas, kThreads, b->persist_smem_bytes, s>>>(map, b->pargs);
    if (timed) cudaEventRecord(b->ev[2], s);
    if (b->rescore)
        k_batch_rescore<<<(unsigned)b->frame_blocks, kBrsThreads, kBrsSmemFloats * sizeof(float),
                          s>>>(b->d_inst, b->d_call, n);
    else
        k_batch_argmax<<<(unsigned)b->frame_blocks, 256, 0, s>>>(b->d_inst, b->d_call, n);
    if (timed) cudaEventRecord(b->ev[3], s);
    return cudaGetLastError();
}

// Lay out operand B, the work list and its schedule for tile choice t, upload
// the tables, encode the TMA descriptor and capture the graph.
srp_status batch_configure(srp_batch_s *b, const TileChoice &t) {
    const int hs = b->split ? 2 : 1;
    const int n = (int)b->plans.size();
    SRP_CUDA(cudaDeviceSynchronize(), "finish earlier batch calls");
    int64_t rows = 0, op = 0, fr = 0;
    std::vector<int4> items;
    std::vector<int64_t> cost;
    for (int i = 0; i < n; ++i) {
        BatchInst &I = b->inst[i];
        I.Lb = round_up_int(I.max_frames, t.N);
        I.b_row0 = rows;
        rows += (int64_t)I.n_chunks * hs * I.Lb;
        I.op_row0 = op;
        op += (int64_t)I.max_frames * I.pblocks;
        I.frame0 = fr;
        fr += I.max_frames;
        for (int tile = 0; tile < I.n_tiles; ++tile)
            for (int l0 = 0; l0 < I.max_frames; l0 += t.N) {
                items.push_back(make_int4(i, tile, l0, 0));
                cost.push_back((int64_t)I.n_chunks * hs + 2);
            }
    }
    if (rows + 256 >= (int64_t)INT32_MAX)
        return fail(SRP_ERR_UNSUPPORTED, "batch operand buffer exceeds 2^31 rows of 64 slots");
    if (items.size() >= (size_t)INT32_MAX) return fail(SRP_ERR_UNSUPPORTED, "too many work items");
    // longest processing time first onto the least-loaded persistent CTA
    const int ctas = std::max(1, std::min<int>(b->sm_count * t.cps, (int)items.size()));
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    typedef std::pair<int64_t, int> Load;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < ctas; ++c) heap.push(Load(0, c));
    std::vector<std::vector<int>> lists(ctas);
    for (int k : order) {
        Load ld = heap.top();
        heap.pop();
        lists[ld.second].push_back(k);
        ld.first += cost[k];
        heap.push(ld);
    }
    std::vector<int4> sched;
    sched.reserve(items.size());
    std::vector<int32_t> first(ctas + 1, 0);
    // Within a CTA the items run grouped by (plan, frame tile), and .w holds
    // the items left in the group: a call that skips a plan (or its later
    // frames) skips the group with one test.
    for (int c = 0; c < ctas; ++c) {
        first[c] = (int32_t)sched.size();
        std::vector<int> &lc = lists[c];
        std::stable_sort(lc.begin(), lc.end(), [&](int x, int y) {
            return items[x].x != items[y].x ? items[x].x < items[y].x : items[x].z < items[y].z;
        });
        for (size_t k = 0; k < lc.size(); ++k) sched.push_back(items[lc[k]]);
        const size_t e = sched.size();
        for (size_t k = first[c]; k < e;) {
            size_t r = k;
            while (r < e && sched[r].x == sched[k].x && sched[r].z == sched[k].z) ++r;
            for (size_t j = k; j < r; ++j) sched[j].w = (int)(r - j);
            k = r;
        }
    }
    first[ctas] = (int32_t)sched.size();
    // every TMA box [y, y + N) of every item stays inside its plan's block,
    // and the blocks inside the buffer
    for (const int4 &it : sched) {
        const BatchInst &I = b->inst[it.x];
        const int64_t y_last = I.b_row0 + (int64_t)((I.n_chunks - 1) * hs + hs - 1) * I.Lb + it.z;
        if (it.y < 0 || it.y >= I.n_tiles || it.z < 0 || it.z + t.N > I.Lb ||
            y_last + t.N > I.b_row0 + (int64_t)I.n_chunks * hs * I.Lb || y_last + t.N > rows)
            return fail(SRP_ERR_UNSUPPORTED, "internal: batch work item out of bounds");
    }

    SRP_CUDA(grow(&b->d_b, b->b_cap, (size_t)(rows + 256) * 128), "cudaMalloc operand buffer");
    SRP_CUDA(cudaMemset(b->d_b, 0, (size_t)(rows + 256) * 128), "clear operand buffer");
    SRP_CUDA(grow(&b->d_items, b->items_cap, sizeof(int4) * sched.size()), "cudaMalloc work list");
    SRP_CUDA(grow(&b->d_cta_first, b->cta_cap, sizeof(int32_t) * first.size()),
             "cudaMalloc work list");
    SRP_CUDA(cudaMemcpy(b->d_items, sched.data(), sizeof(int4) * sched.size(),
                        cudaMemcpyHostToDevice), "upload work list");
    SRP_CUDA(cudaMemcpy(b->d_cta_first, first.data(), sizeof(int32_t) * first.size(),
                        cudaMemcpyHostToDevice), "upload work list");
    SRP_CUDA(cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice),
             "upload batch table");
    SRP_CUDA(encode_xi_map(b->d_b, (int)(rows + 256), 64, t.N, b->b_map), "cuTensorMapEncodeTiled");
    b->tiles = t;
    b->n_ctas = ctas;
    b->n_items = (int)sched.size();
    b->b_rows = rows;
    b->op_blocks = op;
    b->frame_blocks = fr;

    // kernels and their attributes
    PersistArgs pa;
    pa.inst = b->d_inst;
    pa.call = b->d_call;
    pa.items = b->d_items;
    pa.cta_first = b->d_cta_first;
    pa.N = t.N;
    pa.stages = t.stages;
    const uint32_t ab = b->half ? 0u : 1u;
    pa.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(t.N >> 3) << 17) | ((128u >> 4) << 24);
    pa.tmem_cols = persist_tmem_cols(t, b->split);
    pa.a_col0 = (uint32_t)(2 * t.mw * t.N);
    pa.mma_warps = t.mw;
    pa.status = b->d_status;
    // shared memory at launch: at least enough that no more than cps CTAs fit
    // on one SM (so that their TMEM columns always fit, 512 per SM)
    size_t smem = persist_smem(t, b->split, b->promote);
    smem = std::max(smem, ((size_t)kSmemPerSm / (t.cps + 1) - 1024 + 16 + 15) / 16 * 16);
    const bool conv = b->mode == SRP_MODE_CONV;
    void (*persist)(const CUtensorMap, const PersistArgs) =
        b->promote ? k_map_batch_tc<true, false, true, true, 2, true> :
        t.cps == 4 ? (conv ? (b->half ? k_map_batch_tc<false, true, true, true, 4>
                                      : k_map_batch_tc<false, false, true, true, 4>)
                           : (b->half ? k_map_batch_tc<false, true, false, true, 4>
                                      : k_map_batch_tc<false, false, false, true, 4>)) :
        t.tm ? (conv ? (b->split ? k_map_batch_tc<true, false, true, true>
                                 : (b->half ? k_map_batch_tc<false, true, true, true>
                                            : k_map_batch_tc<false, false, true, true>))
                     : (b->split ? k_map_batch_tc<true, false, false, true>
                                 : (b->half ? k_map_batch_tc<false, true, false, true>
                                            : k_map_batch_tc<false, false, false, true>)))
             : (conv ? (b->split ? k_map_batch_tc<true, false, true, false>
                                 : (b->half ? k_map_batch_tc<false, true, true, false>
                                            : k_map_batch_tc<false, false, true, false>))
                     : (b->split ? k_map_batch_tc<true, false, false, false>
                                 : (b->half ? k_map_batch_tc<false, true, false, false>
                                            : k_map_batch_tc<false, false, false, false>)));
    const int fmt = b->split ? 1 : (b->half ? 2 : 0);
    void (*operands)(const BatchInst *, const BatchCall *, int, uint16_t *) =
        conv ? (fmt == 0 ? k_batch_operands<0, true> : (fmt == 1 ? k_batch_operands<1, true> : k_batch_operands<2, true>))
             : (fmt == 0 ? k_batch_operands<0, false> : (fmt == 1 ? k_batch_operands<1, false> : k_batch_operands<2, false>));
    const size_t op_smem =
        conv ? 0 : sizeof(float2) * (size_t)(b->max_K + kPairBlock * (b->max_K / 2 + 1));
    SRP_CUDA(cudaFuncSetAttribute(persist, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemCta),
             "persistent kernel attribute");
    SRP_CUDA(cudaFuncSetAttribute(operands, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::max<size_t>(op_smem, 1)), "operand kernel attribute");

    b->operands = operands;
    b->persist = persist;
    b->op_smem = op_smem;
    b->persist_smem_bytes = smem;
    b->pargs = pa;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    SRP_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin graph capture");
    cudaError_t launch_err = enqueue_kernels(b, b->cap, false);
    cudaError_t cap_err = cudaStreamEndCapture(b->cap, &b->graph);
    if (launch_err != cudaSuccess) return cuda_fail(launch_err, "capture batch kernels");
    if (cap_err != cudaSuccess) return cuda_fail(cap_err, "end graph capture");
    SRP_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate batch graph");
    return SRP_OK;
}

srp_status batch_call_table(srp_batch_s *b, const void *const *d_in, const int32_t *L,
                            float *const *d_maps, int32_t *const *d_argmax, float *const *d_peak) {
    if (d_in == nullptr || L == nullptr || d_argmax == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "d_in, L and d_argmax must be non-NULL arrays");
    const int n = (int)b->plans.size();
    for (int i = 0; i < n; ++i) {
        const BatchInst &I = b->inst[i];
        if (L[i] < 0 || L[i] > I.max_frames)
            return fail(SRP_ERR_INVALID_ARG, "L[i] out of [0, max_frames of plan i]");
        if (L[i] > 0 && (d_in[i] == nullptr || d_argmax[i] == nullptr))
            return fail(SRP_ERR_INVALID_ARG, "d_in[i] and d_argmax[i] must be non-NULL when L[i] > 0");
    }
    // the previous call's copy of the table must have left the staging buffer
    SRP_CUDA(cudaEventSynchronize(b->copied), "wait for the previous batch call");
    for (int i = 0; i < n; ++i) {
        BatchCall &C = b->h_call[i];
        C.in = d_in[i];
        C.maps = d_maps != nullptr ? d_maps[i] : nullptr;
        C.argmax = d_argmax[i];
        C.peak = d_peak != nullptr ? d_peak[i] : nullptr;
        C.L = L[i];
        C.vec_maps = C.maps != nullptr && (b->inst[i].J % 2) == 0 &&
                     (reinterpret_cast<uintptr_t>(C.maps) & 7) == 0;
    }
    return SRP_OK;
}

srp_status batch_launch(srp_batch_s *b, cudaStream_t s) {
    SRP_CUDA(cudaMemcpyAsync(b->d_call, b->h_call, sizeof(BatchCall) * b->plans.size(),
                             cudaMemcpyHostToDevice, s), "upload batch call table");
    SRP_CUDA(cudaEventRecord(b->copied, s), "record batch event");
    if (b->timing) {
        SRP_CUDA(enqueue_kernels(b, s, true), "launch batch kernels");
    } else {
        SRP_CUDA(cudaGraphLaunch(b->exec, s), "launch batch graph");
    }
    return SRP_OK;
}

}  // namespace
}  // namespace srp

extern "C" {

srp_status srp_batch_create(const srp_handle *plans, int32_t n, const srp_batch_tiles *tiles,
                            srp_batch *out) {
    if (out == nullptr) return fail(SRP_ERR_INVALID_ARG, "out is NULL");
    if (plans == nullptr || n < 1) return fail(SRP_ERR_INVALID_ARG, "need at least one plan");
    for (int i = 0; i < n; ++i)
        if (plans[i] == nullptr) return fail(SRP_ERR_INVALID_ARG, "plan handle is NULL");
    const srp_plan_s *p0 = plans[0];
    for (int i = 0; i < n; ++i) {
        const srp_plan_s *p = plans[i];
        if (p->device != p0->device) return fail(SRP_ERR_INVALID_ARG, "plans on different devices");
        if (p->mode != p0->mode || p->precision != p0->precision)
            return fail(SRP_ERR_UNSUPPORTED, "a batch takes plans of one mode and one precision");
        if (!p->lay.tc)
            return fail(SRP_ERR_UNSUPPORTED,
                        "a batch takes tensor-core plans only (this plan runs on CUDA cores)");
    }
    DeviceGuard g(p0->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plans' device");
    srp_batch_s *b = new (std::nothrow) srp_batch_s();
    if (b == nullptr) return fail(SRP_ERR_OOM, "host allocation failed");
    auto bail = [&](srp_status s) {
        batch_release(b);
        delete b;
        return s;
    };
    b->device = p0->device;
    b->mode = p0->mode;
    b->precision = p0->precision;
    b->split = p0->precision == SRP_PREC_FP32;
    b->half = p0->precision == SRP_PREC_FP16;
    b->plans.assign(plans, plans + n);
    cudaError_t e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    size_t part = 0, x32 = 0;
    b->inst.resize(n);
    for (int i = 0; i < n; ++i) {
        const srp_plan_s *p = plans[i];
        const Layout &L = p->lay;
        BatchInst &I = b->inst[i];
        memset(&I, 0, sizeof I);
        I.xs = p->d_xs;
        I.ctab = p->d_ctab;
        I.pairs = p->d_pairs;
        I.nq = p->d_nq;
        I.offc = p->d_offc;
        I.twid = p->d_twid;
        I.J = L.J;
        I.J_pad = L.J_pad;
        I.M = L.M;
        I.Q = L.Q;
        I.K = L.K;
        I.n_aux = L.n_aux;
        I.xf = L.xf;
        I.n_chunks = L.n_chunks;
        I.n_tiles = L.n_tiles;
        I.par1_used = L.par1_used;
        I.input_kind = p->input_kind;
        I.weighting = p->weighting;
        I.w = static_cast<const uint4 *>(p->d_w);
        I.woff = p->d_woff;
        I.tile_steps = L.tile_steps;
        I.all_streamed = (p->d_w != nullptr && L.tile_steps == L.total_steps) ? 1 : 0;
        if (p->d_w != nullptr) b->any_resident = true;
        // FP32 split: 3 products per step, all in one accumulator (per epoch
        // of a promoted plan: at most 4 steps per chunk)
        I.promote = L.promote;
        if (L.promote > 0) b->promote = true;
        const double acc_steps =
            L.promote > 0 ? std::min<double>(L.mma_steps, 4.0 * L.promote) : (double)L.mma_steps;
        if (p0->precision == SRP_PREC_FP32 && 3.0 * acc_steps * kTcAccumBias > kTcBiasLimit)
            b->one_acc = false;
        I.max_frames = L.L_max;
        I.pblocks = (L.Q + kPairBlock - 1) / kPairBlock;
        I.off = p->d_off;
        I.S32 = L.S;
        if (L.rescore && p0->mode == SRP_MODE_NYQUIST) {
            b->rescore = true;
            x32 += sizeof(float) * (size_t)L.L_max * L.S;
        }
        part += sizeof(unsigned long long) * (size_t)L.L_max * L.n_tiles;
        b->max_L = std::max(b->max_L, L.L_max);
        b->max_K = std::max(b->max_K, L.K);
    }
    if (sizeof(float2) * (size_t)(b->max_K + kPairBlock * (b->max_K / 2 + 1)) > (size_t)kMaxSmemCta)
        return bail(fail(SRP_ERR_UNSUPPORTED, "K too large for the batched operand kernel"));
    if ((e = cudaMalloc(&b->d_part, part)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    b->part_bytes = part;
    if (x32 > 0) {
        if ((e = cudaMalloc(&b->d_x32, x32)) != cudaSuccess)
            return bail(cuda_fail(e, "cudaMalloc"));
        size_t off = 0;
        for (int i = 0; i < n; ++i) {
            if (!(plans[i]->lay.rescore && p0->mode == SRP_MODE_NYQUIST)) continue;
            b->inst[i].x32 = b->d_x32 + off / sizeof(float);
            off += sizeof(float) * (size_t)b->inst[i].max_frames * b->inst[i].S32;
        }
        if ((e = cudaFuncSetAttribute(k_batch_rescore, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kBrsSmemFloats * sizeof(float)))) != cudaSuccess)
            return bail(cuda_fail(e, "re-scoring kernel attribute"));
    }
    {
        size_t off = 0;
        for (int i = 0; i < n; ++i) {
            b->inst[i].part = b->d_part + off / sizeof(unsigned long long);
            off += sizeof(unsigned long long) * (size_t)b->inst[i].max_frames * b->inst[i].n_tiles;
        }
    }
    if ((e = cudaMalloc(&b->d_inst, sizeof(BatchInst) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_call, sizeof(BatchCall) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_status, sizeof(int))) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = cudaMallocHost(&b->h_call, sizeof(BatchCall) * n)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMallocHost"));
    memset(b->h_call, 0, sizeof(BatchCall) * n);
    if ((e = cudaMemset(b->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(b->d_call, b->h_call, sizeof(BatchCall) * n, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return bail(cuda_fail(e, "clear batch tables"));
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaStreamCreate"));
    for (auto &ev : b->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate"));
    if ((e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaEventCreate"));

    // tile choice: as given, else N = frames of the largest call (at most
    // 64), two CTAs per SM when two pipeline stages fit, else one CTA
    TileChoice t;
    if (tiles != nullptr && tiles->frames_per_tile != 0) t.N = tiles->frames_per_tile;
    else t.N = std::min(64, round_up_int(b->max_L, 16));
    const bool given_stages = tiles != nullptr && tiles->stages != 0;
    const bool given_cps = tiles != nullptr && tiles->ctas_per_sm != 0;
    const int given_a = tiles != nullptr ? tiles->operand_a : 0;
    if (given_a < 0 || given_a > 2) return bail(fail(SRP_ERR_INVALID_ARG, "operand_a must be 0, 1 or 2"));
    const int given_mw = tiles != nullptr ? tiles->accumulators : 0;
    if (given_mw < 0 || given_mw > 2)
        return bail(fail(SRP_ERR_INVALID_ARG, "accumulators must be 0, 1 or 2"));
    TileChoice best;
    for (int tm = 1; tm >= 0; --tm) {  // A in TMEM first
        if ((given_a == 1 && !tm) || (given_a == 2 && tm)) continue;
        for (int cps = 4; cps >= 1; cps = (cps == 4 ? 2 : cps - 1)) {
            if (given_cps && cps != tiles->ctas_per_sm) continue;
            for (int mw = 2; mw >= 1; --mw) {
                if (given_mw != 0 && mw != given_mw) continue;
                for (int st = 4; st >= 2; --st) {
                    if (given_stages && st != tiles->stages) continue;
                    TileChoice c = t;
                    c.cps = cps;
                    c.stages = st;
                    c.tm = tm != 0;
                    c.mw = mw;
                    if (tile_fits(c, b->split, b->any_resident, b->one_acc, b->promote) && best.N == 0)
                        best = c;
                }
            }
        }
    }
    if (best.N == 0) return bail(fail(SRP_ERR_INVALID_ARG, "tile choice does not fit the SM"));
    srp_status st = batch_configure(b, best);
    if (st != SRP_OK) return bail(st);
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(cuda_fail(e, "batch setup"));
    *out = b;
    return SRP_OK;
}

srp_status srp_map_batch(srp_batch b, const void *const *d_in, const int32_t *L,
                         float *const *d_maps, int32_t *const *d_argmax, float *const *d_peak,
                         srp_stream_t s) {
    if (b == nullptr) return fail(SRP_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the batch's device");
    srp_status st = batch_call_table(b, d_in, L, d_maps, d_argmax, d_peak);
    if (st != SRP_OK) return st;
    return batch_launch(b, reinterpret_cast<cudaStream_t>(s));
}

srp_status srp_batch_tune(srp_batch b, const void *const *d_in, const int32_t *L,
                          float *const *d_maps, int32_t *const *d_argmax, float *const *d_peak,
                          srp_stream_t s) {
    if (b == nullptr) return fail(SRP_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the batch's device");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    srp_status st = batch_call_table(b, d_in, L, d_maps, d_argmax, d_peak);
    if (st != SRP_OK) return st;
    // candidates: frames per item N in {16, 32, 64, 128, 256} up to the
    // largest call, pipeline depth 2..4, one or two CTAs per SM, A in TMEM or
    // shared memory, one or two accumulators
    int maxl = 0;
    for (size_t i = 0; i < b->plans.size(); ++i) maxl = std::max(maxl, L[i]);
    const int nmax = std::min(256, round_up_int(std::max(maxl, 1), 16));
    std::vector<int> Ns;
    for (int N = 16; N <= 256; N *= 2)
        if (N <= nmax) Ns.push_back(N);
    if (std::find(Ns.begin(), Ns.end(), nmax) == Ns.end()) Ns.push_back(nmax);
    cudaEvent_t e0, e1;
    SRP_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    SRP_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    TileChoice best;
    float best_ms = 0.0f;
    srp_status result = SRP_OK;
    for (int N : Ns) {
        if (result != SRP_OK) break;
        for (int tm = 0; tm <= 1 && result == SRP_OK; ++tm)
        for (int cps = 1; cps <= 4 && result == SRP_OK; cps = (cps == 2 ? 4 : cps + 1))
        for (int mw = 1; mw <= 2 && result == SRP_OK; ++mw)
            for (int stg = 2; stg <= 4 && result == SRP_OK; ++stg) {
                TileChoice c;
                c.N = N;
                c.stages = stg;
                c.cps = cps;
                c.tm = tm != 0;
                c.mw = mw;
                if (!tile_fits(c, b->split, b->any_resident, b->one_acc, b->promote)) continue;
                if ((result = batch_configure(b, c)) != SRP_OK) break;
                float ms = 0.0f;
                for (int rep = 0; rep < 3 && result == SRP_OK; ++rep) {
                    cudaEventRecord(e0, cs);
                    result = batch_launch(b, cs);
                    cudaEventRecord(e1, cs);
                    if (result == SRP_OK && cudaEventSynchronize(e1) != cudaSuccess)
                        result = fail(SRP_ERR_CUDA, "batch tuning run failed");
                    float m = 0.0f;
                    cudaEventElapsedTime(&m, e0, e1);
                    if (rep > 0) ms += m / 2.0f;  // first run is a warm-up
                }
                if (result == SRP_OK && (best.N == 0 || ms < best_ms)) {
                    best = c;
                    best_ms = ms;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != SRP_OK) return result;
    if (best.N == 0) return fail(SRP_ERR_UNSUPPORTED, "no tile candidate fits");
    if ((st = batch_configure(b, best)) != SRP_OK) return st;
    if ((st = batch_launch(b, cs)) != SRP_OK) return st;  // outputs of the chosen tiles
    SRP_CUDA(cudaStreamSynchronize(cs), "batch tuning run");
    b->tuned = 1;
    b->tuned_ms = best_ms;
    return SRP_OK;
}

srp_status srp_batch_get_info(srp_batch b, srp_batch_info *info) {
    if (b == nullptr || info == nullptr) return fail(SRP_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof *info);
    info->n = (int32_t)b->plans.size();
    info->items = b->n_items;
    info->ctas = b->n_ctas;
    info->tiles.frames_per_tile = b->tiles.N;
    info->tiles.stages = b->tiles.stages;
    info->tiles.ctas_per_sm = b->tiles.cps;
    info->tiles.operand_a = b->tiles.tm ? 1 : 2;
    info->tiles.accumulators = b->tiles.mw;
    info->launches = 3;
    info->tuned = b->tuned;
    info->tuned_ms = b->tuned_ms;
    info->device_bytes = b->b_cap + b->items_cap + b->cta_cap + b->part_bytes +
                         (sizeof(BatchInst) + sizeof(BatchCall)) * b->plans.size() + sizeof(int);
    return SRP_OK;
}

srp_status srp_batch_set_timing(srp_batch b, int32_t enable) {
    if (b == nullptr) return fail(SRP_ERR_INVALID_ARG, "batch is NULL");
    b->timing = enable ? 1 : 0;
    return SRP_OK;
}

srp_status srp_batch_stage_times(srp_batch b, float *ms, int32_t n) {
    if (b == nullptr || ms == nullptr || n < 0) return fail(SRP_ERR_INVALID_ARG, "bad argument");
    if (!b->timing) return fail(SRP_ERR_INVALID_ARG, "timing is off (srp_batch_set_timing)");
    DeviceGuard g(b->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the batch's device");
    SRP_CUDA(cudaEventSynchronize(b->ev[3]), "wait for the batch call");
    for (int k = 0; k < n && k < 3; ++k) {
        float v = 0.0f;
        SRP_CUDA(cudaEventElapsedTime(&v, b->ev[k], b->ev[k + 1]), "batch stage time");
        ms[k] = v;
    }
    for (int k = 3; k < n; ++k) ms[k] = 0.0f;
    return SRP_OK;
}

srp_status srp_batch_poll_device_status(srp_batch b, srp_stream_t s) {
    if (b == nullptr) return fail(SRP_ERR_INVALID_ARG, "batch is NULL");
    DeviceGuard g(b->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the batch's device");
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    int flags = 0;
    SRP_CUDA(cudaMemcpyAsync(&flags, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, cs),
             "read device status");
    SRP_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int), cs), "clear device status");
    SRP_CUDA(cudaStreamSynchronize(cs), "read device status");
    if (flags & 1) return fail(SRP_ERR_TIMEOUT, "a bounded wait in the batch kernel gave up");
    return SRP_OK;
}

srp_status srp_batch_destroy(srp_batch b) {
    if (b == nullptr) return SRP_OK;
    {
        DeviceGuard g(b->device);
        cudaEventSynchronize(b->copied);
        batch_release(b);
    }
    delete b;
    return SRP_OK;
}

}  // extern "C"
