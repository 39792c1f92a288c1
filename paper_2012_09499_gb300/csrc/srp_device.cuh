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
    if (v == 0.0f) v = 0.0f;
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
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

// Critical GCC samples of one (frame, pair) row held in shared memory:
// xi(n) = (1/K) sum_k a_k Re[psi(k) e^{j 2 pi k n / K}] for n = -nmax..nmax,
// with ps[k] = a_k psi(k) and tw[j] = (cos, sin)(2 pi j / K).  One warp per
// lag, lanes strided over bins; emit(t, value) is called by lane 0 for lag
// slot t = n + nmax.
template <typename Emit>
__device__ __forceinline__ void gcc_row(const float2 *tw, const float2 *ps, int K, int nmax,
                                        Emit emit) {
    const int Kb = K / 2 + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float inv_k = 1.0f / (float)K;
    for (int t = warp; t <= 2 * nmax; t += nw) {
        const int n = t - nmax;
        const int nm = ((n % K) + K) % K;
        // twiddle index k n mod K, stepped by 32 n mod K along the lane's bins
        const int step = (int)((32ll * nm) % K);
        int idx = (int)(((long long)lane * nm) % K);
        float acc = 0.0f;
        for (int k = lane; k < Kb; k += 32) {
            const float2 w = tw[idx];
            const float2 p = ps[k];
            acc = fmaf(p.x, w.x, acc);
            acc = fmaf(-p.y, w.y, acc);
            idx += step;
            if (idx >= K) idx -= K;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) emit(t, n, acc * inv_k);
    }
}

// PHAT cross spectrum of one bin: u_m conj(u_m') with u = y / |y| (0 where
// y = 0), which equals y_m y_m'^* / |y_m y_m'^*| without forming the product
// of two small magnitudes.
__device__ __forceinline__ float2 unit_phase(float2 v) {
    const float a = hypotf(v.x, v.y);
    return a > 0.0f ? make_float2(v.x / a, v.y / a) : make_float2(0.0f, 0.0f);
}

__device__ __forceinline__ float2 phat_cross(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Stage one (frame, pair) spectrum row as a_k psi(k) and the twiddles.
__device__ __forceinline__ void stage_gcc_row(const float2 *__restrict__ row,
                                              const float2 *__restrict__ twid, int K, float2 *tw,
                                              float2 *ps) {
    const int Kb = K / 2 + 1;
    for (int j = threadIdx.x; j < K; j += blockDim.x) tw[j] = twid[j];
    for (int k = threadIdx.x; k < Kb; k += blockDim.x) {
        const float2 v = row[k];
        const float a = (k == 0 || 2 * k == K) ? 1.0f : 2.0f;
        ps[k] = make_float2(a * v.x, a * v.y);
    }
}

}  // namespace dev
}  // namespace srp
