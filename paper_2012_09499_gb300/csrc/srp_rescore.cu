// FP32 re-scoring of the maximiser of reduced-precision (BF16 / FP16) maps.
//
// A BF16 or FP16 map is within 1e-2 x peak of the exact map, but two
// candidates whose exact values differ by less than that may swap order, and
// on a broad peak the maximiser then moves by several grid cells.  The
// maximiser (Sec. 2.2, last sentence: the candidate of largest SRP) is
// therefore decided in FP32: with m the frame's largest reduced-precision
// value, every 128-candidate tile whose own maximum is at least
// m - delta |m| is evaluated again, candidate by candidate, in FP32 arithmetic:
//   Nyquist:      sum_q sum_n xi_q(n) sinc(x_iq - n)         (Eq. SRPapprox)
//   conventional: sum_q (1/K) sum_k a_k Re[psi_q(k) e^{j 2 pi k x_iq / K}]
//                                                            (Eq. GCC_IFT)
// and the lowest-index maximiser of those values is the frame's argmax, its
// FP32 value the peak.  With delta twice the error bound of the map, the tile
// of the exact maximiser is always among those evaluated (its reduced value
// is at least the exact maximum minus the bound, and m is at most the exact
// maximum plus the bound).
//
// kRescoreCtas CTAs per frame each find the same tiles (from the per-tile keys)
// and split the selected candidates: for the Nyquist map a CTA takes whole
// tiles, four threads per candidate each summing a quarter of the pairs in
// order, the quarters added in a fixed order; for the
// conventional map a warp takes one candidate at a time, its lanes splitting
// each pair's bins, and sums the lanes in a fixed order.  Every value and the
// result are therefore the same on every run.  Each CTA leaves its best
// key in a per-frame slot; the last CTA of the frame to finish (a per-frame
// counter, reset by that CTA) reduces the slots and writes argmax and peak.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "srp_device.cuh"
#include "srp_internal.h"
#include "srp_rescore.cuh"

namespace srp {
namespace {

using namespace dev;
using rs::nyquist_at;

constexpr int kRsParts = 4;                   // Nyquist: threads per candidate
constexpr int kRsThreads = kRsParts * kTileJ;  // Nyquist: one tile per CTA and pass
constexpr int kRsWarps = kRsThreads / 32;
static_assert(kRsThreads >= kRescoreMaxTiles, "one thread per selected tile when sorting");
constexpr int kRsSmemFloats = 12 * 1024;  // a frame's FP32 samples staged in shared memory (48 KB)
constexpr int kRsCandCap = 2048;          // candidates scored one by one (else whole tiles)

// Sum over the warp in a fixed order (the same butterfly every time).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// The conventional map at candidate i, by one warp, for one frame's cross
// spectra psi [Q][Kb]: lane j takes a contiguous run of ceil(Kb / 32) bins of
// each pair.  The phase 2 pi k x / K is formed exactly as
// 2 pi ((k x0 mod K) + k f) / K every kReseed bins and advanced by the
// rotation e^{j 2 pi x / K} in between.
constexpr int kReseed = 32;
constexpr int kRsGroup = 8;  // bins whose loads are in flight together

__device__ float conventional_at(const int2 *__restrict__ xs, int64_t J_pad, int64_t i, int Q,
                                 int xf, int K, const float2 *__restrict__ psi) {
    const int lane = threadIdx.x & 31;
    const int Kb = K / 2 + 1, run = (Kb + 31) / 32;
    const int kbeg = min(Kb, lane * run), kend = min(Kb, kbeg + run);
    const float two_k = 2.0f / (float)K, inv_k = 1.0f / (float)K;
    float acc = 0.0f;
    for (int q0 = 0; q0 < Q; q0 += 32) {
        const int my = q0 + lane < Q ? __ldg(&xs[(size_t)(q0 + lane) * J_pad + i]).x : 0;
        const int nq_here = min(32, Q - q0);
        for (int qq = 0; qq < nq_here; ++qq) {
            int x0;
            float f;
            decode_tdoa(__shfl_sync(0xFFFFFFFFu, my, qq), xf, x0, f);
            const int x0m = ((x0 % K) + K) % K;
            float s1, c1;  // e^{j 2 pi x / K}
            sincospif(fmaf((float)x0m, two_k, f * two_k), &s1, &c1);
            const float2 *row = psi + (size_t)(q0 + qq) * Kb;
            for (int k0 = kbeg; k0 < kend; k0 += kReseed) {
                float s, c;
                sincospif(fmaf((float)(int)(((long long)k0 * x0m) % K), two_k,
                               (float)k0 * f * two_k),
                          &s, &c);
                const int k1 = min(kend, k0 + kReseed);
                for (int kb = k0; kb < k1; kb += kRsGroup) {
                    float2 v[kRsGroup];  // the group's loads are issued before its arithmetic
#pragma unroll
                    for (int u = 0; u < kRsGroup; ++u)
                        v[u] = kb + u < k1 ? __ldg(&row[kb + u]) : make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int u = 0; u < kRsGroup; ++u) {
                        const int k = kb + u;
                        if (k >= k1) break;
                        const float a = (k == 0 || 2 * k == K) ? inv_k : 2.0f * inv_k;
                        acc = fmaf(a * v[u].x, c, fmaf(-a * v[u].y, s, acc));
                        const float cn = c * c1 - s * s1;
                        s = fmaf(s, c1, c * s1);
                        c = cn;
                    }
                }
            }
        }
    }
    return warp_sum(acc);
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long k,
                                                        unsigned long long *red) {
    k = warp_max_u64(k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
    __syncthreads();
    k = 0ull;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) k = red[w] > k ? red[w] : k;
    __syncthreads();
    return k;
}

template <bool kConv>
__global__ void __launch_bounds__(kRsThreads) k_rescore(
    const unsigned long long *__restrict__ part, int n_tiles, int64_t J, int64_t J_pad, int Q,
    const int2 *__restrict__ xs, int xf, const int32_t *__restrict__ nq,
    const int32_t *__restrict__ off, int n_aux, const float *__restrict__ xi32, int S32,
    const float2 *__restrict__ psi, int K, float delta, const unsigned long long *fkey,
    unsigned long long *slots, int *count, int32_t *__restrict__ argmax,
    float *__restrict__ peak, const float *__restrict__ maps) {
    __shared__ unsigned long long red[kRsWarps];
    __shared__ int tiles[kRescoreMaxTiles];
    __shared__ int n_sel, last, n_cand;
    __shared__ int cand[kRsCandCap];
    const int l = blockIdx.x, g = blockIdx.y, G = gridDim.y;
    // launched behind the map kernel with programmatic stream serialization:
    // wait until its tile keys are complete and visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const unsigned long long *pl = part + (size_t)l * n_tiles;
    if (threadIdx.x == 0) n_sel = 0;
    __syncthreads();
    // the frame's largest key (raised by every tile), then the tiles near it;
    // four loads in flight per thread
    const unsigned long long kmax = __ldcg(&fkey[l]);
    const float m = key_value(kmax);
    const uint32_t otau = ordered_value(m - delta * fabsf(m));
    for (int t0 = threadIdx.x; t0 < n_tiles; t0 += 4 * kRsThreads) {
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * kRsThreads;
            v[u] = t < n_tiles ? (uint32_t)(__ldcg(&pl[t]) >> 32) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (v[u] >= otau && t0 + u * kRsThreads < n_tiles) {
                const int slot = atomicAdd(&n_sel, 1);
                if (slot < kRescoreMaxTiles) tiles[slot] = t0 + u * kRsThreads;
            }
    }
    __syncthreads();
    const int ns = n_sel;
    if (ns <= kRescoreMaxTiles) {
        // ascending tile order, the same in every CTA of the frame (the
        // atomics above fill the list in an arbitrary order, and the CTAs
        // split the work by list position)
        int t = 0, rank = 0;
        if (threadIdx.x < ns) {
            t = tiles[threadIdx.x];
            for (int j = 0; j < ns; ++j) rank += tiles[j] < t ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x < ns) tiles[rank] = t;
        __syncthreads();
    }
    if (ns > kRescoreMaxTiles) {  // nearly flat map: the reduced-precision maximiser stands
        if (g == 0 && threadIdx.x == 0) {
            argmax[l] = (int32_t)(0xFFFFFFFFu - (uint32_t)(kmax & 0xFFFFFFFFull));
            if (peak != nullptr) peak[l] = m;
        }
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the frame's FP32 samples, in shared memory when they fit
    extern __shared__ float xi_sm[];
    const float *xr = nullptr;
    if (!kConv) {
        xr = xi32 + (size_t)l * S32;
        if (S32 <= kRsSmemFloats) {
            for (int t = threadIdx.x; t < S32; t += kRsThreads) xi_sm[t] = xr[t];
            __syncthreads();
            xr = xi_sm;
        }
    }
    const float2 *pr = kConv ? psi + (size_t)l * Q * (K / 2 + 1) : nullptr;
    unsigned long long best = 0ull;
    // the order in which candidates are evaluated does not change any value,
    // and the key order picks the largest value, then the lowest index
    if (kConv) {
        // candidate e of the selected tiles goes to warp e mod (G x warps) of CTA g
        for (int e = g * kRsWarps + warp; e < ns * kTileJ; e += G * kRsWarps) {
            const int64_t i = (int64_t)tiles[e / kTileJ] * kTileJ + (e % kTileJ);
            if (i >= J) continue;  // uniform over the warp
            const float v = conventional_at(xs, J_pad, i, Q, xf, K, pr);
            if (lane == 0) {
                const unsigned long long key = argmax_key(v, (uint32_t)i);
                best = key > best ? key : best;
            }
        }
    } else {
        // selected tile j goes to CTA j mod G (its candidates that reach the
        // threshold in the map, when the map is written)
        __shared__ float part_sum[kRsParts * kTileJ];
        best = rs::score_candidates<kRsParts>(
            tiles, g, G, ns, maps != nullptr ? maps + (size_t)l * J : nullptr, otau, J, cand,
            kRsCandCap, &n_cand, part_sum, [&](int64_t i, int p) {
                return nyquist_at(xs, J_pad, i, Q, xf, nq, off, n_aux, xr, p, kRsParts);
            });
    }
    best = block_max(best, red);
    // this CTA's best key; the frame's last CTA to arrive reduces them all
    if (threadIdx.x == 0) {
        slots[(size_t)l * G + g] = best;
        __threadfence();
        last = atomicAdd(&count[l], 1) == G - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    unsigned long long b = 0ull;
    for (int j = threadIdx.x; j < G; j += kRsThreads) {
        const unsigned long long v = __ldcg(&slots[(size_t)l * G + j]);
        b = v > b ? v : b;
    }
    b = block_max(b, red);
    if (threadIdx.x == 0) {
        count[l] = 0;  // ready for the next call
        argmax[l] = (int32_t)(0xFFFFFFFFu - (uint32_t)(b & 0xFFFFFFFFull));
        if (peak != nullptr) peak[l] = key_value(b);
    }
}

}  // namespace

cudaError_t launch_rescore(bool conv, const unsigned long long *part, int n_tiles, int64_t J,
                           int64_t J_pad, int Q, const int2 *xs, int xf, const int32_t *nq,
                           const int32_t *off, int n_aux, const float *xi32, int S32,
                           const float2 *psi, int K, int L, float delta,
                           const unsigned long long *fkey, unsigned long long *slots, int *count,
                           int32_t *argmax, float *peak, const float *maps, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    static bool attr = false;
    if (!attr) {  // up to 48 KB of staged samples beside the static arrays
        cudaError_t e = cudaFuncSetAttribute(k_rescore<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float) * kRsSmemFloats));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    // the conventional map scores a warp per candidate, the Nyquist map a CTA
    // per tile: all kRescoreCtas CTAs per frame, or a quarter of them
    cfg.gridDim = dim3((unsigned)L, (unsigned)(conv ? kRescoreCtas : kRescoreCtas / 4));
    cfg.blockDim = dim3(kRsThreads);
    cfg.dynamicSmemBytes = (conv || S32 > kRsSmemFloats) ? 0 : sizeof(float) * (size_t)S32;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = conv ? cudaLaunchKernelEx(&cfg, k_rescore<true>, part, n_tiles, J, J_pad, Q, xs,
                                              xf, nq, off, n_aux, xi32, S32, psi, K, delta, fkey,
                                              slots, count, argmax, peak, maps)
                         : cudaLaunchKernelEx(&cfg, k_rescore<false>, part, n_tiles, J, J_pad, Q,
                                              xs, xf, nq, off, n_aux, xi32, S32, psi, K, delta,
                                              fkey, slots, count, argmax, peak, maps);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace srp
