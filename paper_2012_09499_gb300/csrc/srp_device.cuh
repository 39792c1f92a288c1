// Device helpers shared by the CUDA-core and tensor-core kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace srp {
namespace dev {

constexpr float kInvPi = 0.318309886183790671537767526745f;

// Key whose unsigned order is (map value ascending, candidate index
// descending): the maximum key is the first maximiser.  -0 is folded to +0 so
// that equal zeros tie on the index.
__device__ __forceinline__ unsigned long long argmax_key(float v, uint32_t i) {
    if (v == 0.0f) v = 0.0f;
    uint32_t u = __float_as_uint(v);
    uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)o << 32) | (unsigned long long)(0xFFFFFFFFu - i);
}

// The upper half of argmax_key: an unsigned value in the order of v.
__device__ __forceinline__ uint32_t ordered_value(float v) {
    // -0 + 0 = +0 (round to nearest), so both zeros map alike; negative
    // values are complemented, non-negative ones get the top bit
    const uint32_t u = __float_as_uint(v + 0.0f);
    return u ^ ((uint32_t)((int32_t)u >> 31) | 0x80000000u);
}

__device__ __forceinline__ float key_value(unsigned long long k) {
    uint32_t o = (uint32_t)(k >> 32);
    uint32_t u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return __uint_as_float(u);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, k, o);
        k = t > k ? t : k;
    }
    return k;
}

// Decode a fixed-point TDOA X = round(x 2^xf) into x = x0 + f with x0 the
// nearest integer and f in [-1/2, 1/2) exact in FP32.
__device__ __forceinline__ void decode_tdoa(int32_t X, int xf, int &x0, float &f) {
    x0 = (X + (1 << (xf - 1))) >> xf;
    f = (float)(X - x0 * (1 << xf)) * __int_as_float((127 - xf) << 23);
}

// Sum over the warp of 16 values per lane, as a transposed butterfly: 16
// shuffles instead of 80.  Returns to lane l the full sum of value index
// ((l >> 1) & 1) | ((l >> 2) & 1) << 1 | ((l >> 3) & 1) << 2 | ((l >> 4) & 1) << 3
// (lanes l and l ^ 1 hold the same sum).
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int half = 8, m = 16; half >= 1; half >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = up ? v[i] : v[i + half];
            const float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, m);
        }
    }
    return v[0] + __shfl_xor_sync(0xFFFFFFFFu, v[0], 1);
}

// Critical GCC samples of P (frame, pair) rows held in shared memory:
// xi_p(n) = (1/K) sum_k a_k Re[psi_p(k) e^{j 2 pi k n / K}] for
// n = -nmax_p..nmax_p, with ps[p * ps_stride + k] = a_k psi_p(k) and
// tw[j] = (cos, sin)(2 pi j / K).  With theta = 2 pi k n / K,
// C(n) = sum_k a_k Re psi(k) cos theta and S(n) = sum_k a_k Im psi(k) sin theta
// give both xi(n) = (C - S)/K and xi(-n) = (C + S)/K, so only n >= 0 is
// summed.  The work items, blocks of kLagBlock consecutive lags n >= 0 of one
// row, are spread over the warps; lanes stride over the bins.  A lane reads the
// exact twiddle of the block's first lag n0 once per bin (index k n0 mod K,
// stepped by 32 n0 mod K) and steps to the next lags by multiplying with
// e^{j 2 pi k / K} = tw[k], which consecutive lanes read from consecutive
// entries.  emit(p, t, n, value) is called for every lag n, slot
// t = n + nmax_p, by one lane.  nmax_of(p) gives nmax_p.
constexpr int kLagBlock = 8;

template <typename NmaxFn, typename Emit>
__device__ __forceinline__ void gcc_rows(const float2 *tw, const float2 *ps, int ps_stride, int P,
                                         int K, NmaxFn nmax_of, Emit emit) {
    const int Kb = K / 2 + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float inv_k = 1.0f / (float)K;
    auto blocks = [&](int p) { return nmax_of(p) / kLagBlock + 1; };
    int p = 0, blk = warp, nb = blocks(0);
    for (;;) {
        while (p < P && blk >= nb) {  // item -> (row p, lag block blk); uniform per warp
            blk -= nb;
            if (++p < P) nb = blocks(p);
        }
        if (p >= P) break;
        const int nmax = nmax_of(p);
        const int n0 = blk * kLagBlock;
        const int nm0 = n0 % K;
        const int step = (int)((32ll * nm0) % K);
        int idx = (int)(((long long)lane * nm0) % K);
        const float2 *row = ps + (size_t)p * ps_stride;
        float acc[2 * kLagBlock];  // C then S of lag n0 + j at 2j, 2j + 1
#pragma unroll
        for (int j = 0; j < 2 * kLagBlock; ++j) acc[j] = 0.0f;
        for (int k = lane; k < Kb; k += 32) {
            const float2 pv = row[k];
            const float2 r = tw[k];
            float2 w = tw[idx];
#pragma unroll
            for (int j = 0; j < kLagBlock; ++j) {
                acc[2 * j] = fmaf(pv.x, w.x, acc[2 * j]);
                acc[2 * j + 1] = fmaf(pv.y, w.y, acc[2 * j + 1]);
                w = make_float2(fmaf(w.x, r.x, -w.y * r.y), fmaf(w.x, r.y, w.y * r.x));
            }
            idx += step;
            if (idx >= K) idx -= K;
        }
        const float mine = warp_transpose_sum16(acc);
        const float other = __shfl_xor_sync(0xFFFFFFFFu, mine, 2);
        const int c = (lane >> 1) & 1, n = n0 + (lane >> 2);
        if ((lane & 1) == 0 && n <= nmax) {
            const float C = c ? other : mine, S = c ? mine : other;
            if (c == 0) emit(p, nmax + n, n, (C - S) * inv_k);
            else if (n > 0) emit(p, nmax - n, -n, (C + S) * inv_k);
        }
        blk += nw;
    }
}

// One row: emit(t, n, value).
template <typename Emit>
__device__ __forceinline__ void gcc_row(const float2 *tw, const float2 *ps, int K, int nmax,
                                        Emit emit) {
    gcc_rows(tw, ps, 0, 1, K, [&](int) { return nmax; },
             [&](int, int t, int n, float v) { emit(t, n, v); });
}

// PHAT cross spectrum of one bin: times_conj(unit_phase(y_m), unit_phase(y_m'))
// = u_m conj(u_m') with u = y / |y| (0 where y = 0), which equals
// y_m y_m'^* / |y_m y_m'^*| without forming the product of two small
// magnitudes; times_conj(y_m, y_m') is the unweighted cross spectrum.
__device__ __forceinline__ float2 unit_phase(float2 v) {
    const float a2 = fmaf(v.x, v.x, v.y * v.y);
    if (a2 > 1e-30f && a2 < 1e30f) {  // the usual case: one reciprocal square root
        const float r = rsqrtf(a2);
        return make_float2(v.x * r, v.y * r);
    }
    const float a = hypotf(v.x, v.y);  // tiny, huge or zero magnitudes
    return a > 0.0f ? make_float2(v.x / a, v.y / a) : make_float2(0.0f, 0.0f);
}

// a conj(b)
__device__ __forceinline__ float2 times_conj(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Start copying the K twiddles into shared memory tw (16-byte cp.async, two
// per copy; K even, both addresses 16-byte aligned).  The copies complete at
// wait_async_copies().
__device__ __forceinline__ void copy_twiddles_async(const float2 *__restrict__ twid, int K,
                                                    float2 *tw) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(tw);
    for (int j = 2 * (int)threadIdx.x; j < K; j += 2 * (int)blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 8u * (uint32_t)j),
                     "l"(twid + j)
                     : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void wait_async_copies() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Bins of a spectrum row handled together by a thread: their loads are issued
// before any arithmetic, so that the latencies overlap.
constexpr int kStageUnroll = 4;

// Stage one (frame, pair) spectrum row as a_k psi(k) and the twiddles
// (the caller synchronises the block before use).
__device__ __forceinline__ void stage_gcc_row(const float2 *__restrict__ row,
                                              const float2 *__restrict__ twid, int K, float2 *tw,
                                              float2 *ps) {
    const int Kb = K / 2 + 1;
    copy_twiddles_async(twid, K, tw);
    const int nt = blockDim.x;
    for (int k0 = threadIdx.x; k0 < Kb; k0 += kStageUnroll * nt) {
        float2 v[kStageUnroll];
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u)
            if (k0 + u * nt < Kb) v[u] = row[k0 + u * nt];
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
            const int k = k0 + u * nt;
            if (k < Kb) {
                const float a = (k == 0 || 2 * k == K) ? 1.0f : 2.0f;
                ps[k] = make_float2(a * v[u].x, a * v[u].y);
            }
        }
    }
    wait_async_copies();
}

}  // namespace dev
}  // namespace srp
