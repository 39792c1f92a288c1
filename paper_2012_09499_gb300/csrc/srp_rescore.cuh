// FP32 evaluation of Eq. SRPapprox at one candidate, shared by the FP32
// re-scoring of reduced-precision maps in single-plan calls
// (srp_rescore.cu) and in batches (srp_batch.cu).
#pragma once

#include <stdint.h>

#include "srp_device.cuh"

namespace srp {
namespace rs {

constexpr float kExactF = 9.094947017729282e-13f;  // 2^-40: f of an exact sample, as in the plan

__device__ __forceinline__ float rcp_hw(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Eq. SRPapprox summed over the pairs q_first, q_first + q_step, ... at
// candidate i, by one thread (the threads of a warp take consecutive
// candidates, so the table reads are coalesced), for one frame's FP32
// samples xi (pair q's 2 nmax + 1 samples from off[q], lag n at n + nmax; every thread reads the same sample at the
// same time): with x = x0 + f, sinc(x - n) = (-1)^n sp / (f + x0 - n), sp =
// (-1)^x0 sin(pi f) / pi from the plan's table.  f + (x0 - n) is rounded
// once (x0 - n is an exact integer) and its reciprocal is the hardware
// approximation (within an ulp), as in the tensor-core generator.
static __device__ float nyquist_at(const int2 *__restrict__ xs, int64_t J_pad, int64_t i, int Q,
                                   int xf, const int32_t *__restrict__ nq,
                                   const int32_t *__restrict__ off, int n_aux, const float *xi,
                                   int q_first, int q_step) {
    float acc = 0.0f;
    int2 nxt = q_first < Q ? __ldg(&xs[(size_t)q_first * J_pad + i]) : make_int2(0, 0);
    for (int q = q_first; q < Q; q += q_step) {
        const int2 e = nxt;
        if (q + q_step < Q) nxt = __ldg(&xs[(size_t)(q + q_step) * J_pad + i]);
        int x0;
        float f;
        dev::decode_tdoa(e.x, xf, x0, f);
        if (f == 0.0f) f = kExactF;
        const float sp = __int_as_float(e.y);
        const int nmax = __ldg(&nq[q]) + n_aux;
        const float *r = xi + __ldg(&off[q]);
        const int base = x0 + nmax;  // f + base - t = f + x0 - n for slot t = n + nmax
        const float sg = (nmax & 1) ? -sp : sp;  // (-1)^n sp at n = -nmax
        float s0 = 0.0f, s1 = 0.0f;  // even and odd slots
        int t = 0;
        for (; t + 1 <= 2 * nmax; t += 2) {
            s0 = fmaf(rcp_hw(f + (float)(base - t)), r[t], s0);
            s1 = fmaf(rcp_hw(f + (float)(base - t - 1)), r[t + 1], s1);
        }
        s0 = fmaf(rcp_hw(f + (float)(base - t)), r[t], s0);  // the last slot, t = 2 nmax
        acc = fmaf(sg, s0 - s1, acc);
    }
    return acc;
}

// FP32 scores of candidates of the selected tiles tiles[j], j = j0, j0 +
// jstep, ... < ns, by kTileJ * kParts threads: kParts per candidate, part p
// summing the pairs q = p mod kParts, the parts then added in the order 0,
// 1, ... (the same value for a candidate wherever it is scored).  With the
// frame's row of the reduced-precision map (maps_row), only the candidates
// whose own value reaches the threshold otau are scored: the exact
// maximiser is among them by the same argument that selects the tiles
// (every reduced value is within the map's error bound of the exact one),
// and most of a broad peak's tiles lie below it.  Without maps, or when more
// than cap candidates qualify, every candidate of the tiles is scored.
// cand (cap entries), n_cand and part_sum ([kParts][kTileJ]) are shared
// memory; every thread of the CTA calls this.  Returns the best key among
// the candidates whose parts this thread added up (0 if none).
template <int kParts, typename Nyq>
__device__ __forceinline__ unsigned long long score_candidates(
    const int *tiles, int j0, int jstep, int ns, const float *maps_row, uint32_t otau, int64_t J,
    int *cand, int cap, int *n_cand, float *part_sum, Nyq nyq) {
    const int r = threadIdx.x % kTileJ, p = threadIdx.x / kTileJ;
    unsigned long long best = 0ull;
    int nc = -1;
    if (maps_row != nullptr) {
        if (threadIdx.x == 0) *n_cand = 0;
        __syncthreads();
        if (p == 0)
            for (int j = j0; j < ns; j += jstep) {
                const int64_t i = (int64_t)tiles[j] * kTileJ + r;
                if (i < J && dev::ordered_value(maps_row[i]) >= otau) {
                    const int slot = atomicAdd(n_cand, 1);
                    if (slot < cap) cand[slot] = (int)i;
                }
            }
        __syncthreads();
        nc = *n_cand;
        if (nc > cap) nc = -1;
    }
    auto add = [&](bool valid, int64_t i) {
        if (valid) part_sum[p * kTileJ + r] = nyq(i, p);
        __syncthreads();
        if (p == 0 && valid) {
            float v = part_sum[r];
#pragma unroll
            for (int u = 1; u < kParts; ++u) v += part_sum[u * kTileJ + r];
            const unsigned long long key = dev::argmax_key(v, (uint32_t)i);
            best = key > best ? key : best;
        }
        __syncthreads();
    };
    if (nc >= 0) {
        for (int c0 = 0; c0 < nc; c0 += kTileJ) {
            const int c = c0 + r;
            add(c < nc, c < nc ? (int64_t)cand[c] : 0);
        }
    } else {
        for (int j = j0; j < ns; j += jstep) {
            const int64_t i = (int64_t)tiles[j] * kTileJ + r;
            add(i < J, i);
        }
    }
    return best;
}

}  // namespace rs
}  // namespace srp
