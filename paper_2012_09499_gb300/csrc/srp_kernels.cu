// CUDA-core kernels of the SRP hot path (sm_103a):
//   K1 k_phat          PHAT cross spectra            (Eq. corrmatrix, PHAT weight)
//   K2 k_gcc_samples   GCC at the critical lags      (Eq. GCC_IFT at tau = nT, Sec. 3.2)
//   K3 k_interp_simt   truncated sinc interpolation  (Eq. SRPapprox) + pair sum (Eq. SRP_T_IFT)
//   K4 k_conv_simt     conventional SRP              (Eq. GCC_IFT at every TDOA, Sec. 2.4)
//   K5 k_argmax        per-frame maximiser           (Sec. 2.2)
// K3 and K4 end with a fused per-tile argmax: every CTA reduces its 128
// candidates to one ordered 64-bit key per frame, and K5 reduces the keys.
#include <cuda_runtime.h>
#include <stdint.h>

#include "srp_device.cuh"
#include "srp_internal.h"

namespace srp {
namespace {

using namespace dev;

// ---------------------------------------------------------------------------
// K1: psi_q(k) = u_m(k) conj(u_m'(k)) with u = y / |y| (0 where y = 0).  That
// equals y_m y_m'^* / |y_m y_m'^*| and never forms the product of two small
// magnitudes.  Without a weighting, u = y.  One CTA: one frame, kPhatBins
// bins, all microphones and pairs.
// ---------------------------------------------------------------------------
constexpr int kPhatBins = 64;

__global__ void __launch_bounds__(256) k_phat(const float2 *__restrict__ y, int M, int Kb,
                                              const int2 *__restrict__ pairs, int Q,
                                              int weighting, float2 *__restrict__ psi) {
    extern __shared__ float2 u_sm[];  // [M][kPhatBins]
    const int l = blockIdx.y;
    const int k0 = blockIdx.x * kPhatBins;
    for (int e = threadIdx.x; e < M * kPhatBins; e += blockDim.x) {
        const int m = e / kPhatBins, k = k0 + e % kPhatBins;
        float2 v = make_float2(0.0f, 0.0f);
        if (k < Kb) {
            v = y[((size_t)l * M + m) * Kb + k];
            if (weighting == SRP_WEIGHT_PHAT) v = unit_phase(v);
        }
        u_sm[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Q * kPhatBins; e += blockDim.x) {
        const int q = e / kPhatBins, kk = e % kPhatBins, k = k0 + kk;
        if (k >= Kb) continue;
        const int2 p = pairs[q];
        psi[((size_t)l * Q + q) * Kb + k] =
            times_conj(u_sm[p.x * kPhatBins + kk], u_sm[p.y * kPhatBins + kk]);
    }
}

// ---------------------------------------------------------------------------
// K2: xi_q(n) = (1/K) sum_k a_k Re[psi_q(k) e^{j 2 pi k n / K}] for the
// 2(N_q+N_aux)+1 critical lags of pair q.  One CTA per (pair, frame); the
// twiddle table and the weighted spectrum row sit in shared memory, one warp
// per lag, lanes strided over bins, then a shuffle reduction.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_gcc_samples(
    const float2 *__restrict__ psi, int Q, int K, const int32_t *__restrict__ nq,
    const int32_t *__restrict__ off, int n_aux, const float2 *__restrict__ twid,
    float *__restrict__ xi, int64_t s_stride, int64_t l_stride) {
    extern __shared__ float2 sm[];
    float2 *tw = sm, *ps = sm + K;
    const int q = blockIdx.x, l = blockIdx.y;
    stage_gcc_row(psi + ((size_t)l * Q + q) * (K / 2 + 1), twid, K, tw, ps);
    __syncthreads();
    const int base = off[q];
    gcc_row(tw, ps, K, nq[q] + n_aux, [&](int t, int, float v) {
        xi[(int64_t)(base + t) * s_stride + (int64_t)l * l_stride] = v;
    });
}

// Shared epilogue of the map kernels: write the tile's maps (if requested)
// and reduce its argmax key per frame into part[l][tile].
template <int LT>
__device__ __forceinline__ void map_epilogue(const float (&acc)[LT], int64_t i, int64_t J, int l0,
                                             int L, float *__restrict__ maps,
                                             unsigned long long *__restrict__ part, int n_tiles,
                                             unsigned long long (*red)[LT]) {
    const bool valid = i < J;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        const int l = l0 + j;
        if (l < L) {
            if (maps != nullptr && valid) maps[(size_t)l * J + i] = acc[j];
            unsigned long long k = valid ? argmax_key(acc[j], (uint32_t)i) : 0ull;
            k = warp_max_u64(k);
            if (lane == 0) red[warp][j] = k;
        }
    }
    __syncthreads();
    if (threadIdx.x < LT && l0 + (int)threadIdx.x < L) {
        unsigned long long k = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const unsigned long long t = red[w][threadIdx.x];
            k = t > k ? t : k;
        }
        part[(size_t)(l0 + threadIdx.x) * n_tiles + blockIdx.x] = k;
    }
}

// ---------------------------------------------------------------------------
// K3 (CUDA cores, FP32): map[l][i] = sum_q sum_n xi_q(n) sinc(x_iq - n).
// With x = x0 + f, sinc(x - n) = (-1)^(x0-n) sin(pi f) / (pi (f + x0 - n)):
// one sine per (candidate, pair), one division per lag.  f = 0 reduces the
// series to the single sample n = x0.  One thread per candidate, LT frames
// in registers; xi rows are read as float4 (uniform across the warp).
// ---------------------------------------------------------------------------
template <int LT>
__global__ void __launch_bounds__(kTileJ) k_interp_simt(
    const int32_t *__restrict__ x, int64_t J_pad, int64_t J, int Q,
    const int32_t *__restrict__ nq, const int32_t *__restrict__ off, int n_aux, int xf,
    const float *__restrict__ xi, int L_pad, int L, float *__restrict__ maps,
    unsigned long long *__restrict__ part, int n_tiles) {
    __shared__ unsigned long long red[kTileJ / 32][LT];
    const int64_t i = (int64_t)blockIdx.x * kTileJ + threadIdx.x;
    const int l0 = blockIdx.y * LT;
    float acc[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) acc[j] = 0.0f;
    for (int q = 0; q < Q; ++q) {
        int x0;
        float f;
        decode_tdoa(__ldg(&x[(size_t)q * J_pad + i]), xf, x0, f);
        const int nmax = __ldg(&nq[q]) + n_aux;
        const float *xr = xi + (size_t)__ldg(&off[q]) * L_pad + l0;
        if (f == 0.0f) {
            const int t = x0 + nmax;
            if (t >= 0 && t <= 2 * nmax) {
                const float4 *r4 = reinterpret_cast<const float4 *>(xr + (size_t)t * L_pad);
#pragma unroll
                for (int j = 0; j < LT / 4; ++j) {
                    const float4 v = __ldg(r4 + j);
                    acc[4 * j] += v.x;
                    acc[4 * j + 1] += v.y;
                    acc[4 * j + 2] += v.z;
                    acc[4 * j + 3] += v.w;
                }
            }
        } else {
            const float sp = sinpif(f) * kInvPi;
            float sg = ((x0 + nmax) & 1) ? -sp : sp;  // (-1)^(x0-n) at n = -nmax
            for (int t = 0; t <= 2 * nmax; ++t) {
                const float w = sg / (f + (float)(x0 + nmax - t));
                sg = -sg;
                const float4 *r4 = reinterpret_cast<const float4 *>(xr + (size_t)t * L_pad);
#pragma unroll
                for (int j = 0; j < LT / 4; ++j) {
                    const float4 v = __ldg(r4 + j);
                    acc[4 * j] = fmaf(w, v.x, acc[4 * j]);
                    acc[4 * j + 1] = fmaf(w, v.y, acc[4 * j + 1]);
                    acc[4 * j + 2] = fmaf(w, v.z, acc[4 * j + 2]);
                    acc[4 * j + 3] = fmaf(w, v.w, acc[4 * j + 3]);
                }
            }
        }
    }
    map_epilogue<LT>(acc, i, J, l0, L, maps, part, n_tiles, red);
}

// ---------------------------------------------------------------------------
// K4 (CUDA cores, FP32): map[l][i] = sum_q (1/K) sum_k a_k Re[psi_q(k)
// e^{j 2 pi k x_iq / K}].  The phase is formed exactly per chunk of kConvChunk
// bins as 2 pi ((k x0 mod K) + k f)/K and advanced inside the chunk by a
// rotation e^{j 2 pi x / K}.  The CTA stages (a_k/K) psi for its frames and
// one chunk of bins in shared memory, frames contiguous.
// ---------------------------------------------------------------------------
constexpr int kConvChunk = 32;

template <int LT>
__global__ void __launch_bounds__(kTileJ) k_conv_simt(
    const int32_t *__restrict__ x, int64_t J_pad, int64_t J, int Q, int K, int xf,
    const float2 *__restrict__ psi, int L, float *__restrict__ maps,
    unsigned long long *__restrict__ part, int n_tiles) {
    __shared__ unsigned long long red[kTileJ / 32][LT];
    __shared__ __align__(16) float2 ps[kConvChunk][LT];
    const int Kb = K / 2 + 1;
    const int64_t i = (int64_t)blockIdx.x * kTileJ + threadIdx.x;
    const int l0 = blockIdx.y * LT;
    const float inv_k = 1.0f / (float)K, two_over_k = 2.0f / (float)K;
    float acc[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) acc[j] = 0.0f;
    for (int q = 0; q < Q; ++q) {
        int x0;
        float f;
        decode_tdoa(__ldg(&x[(size_t)q * J_pad + i]), xf, x0, f);
        float s1, c1;  // e^{j 2 pi x / K}
        sincospif(((float)x0 + f) * two_over_k, &s1, &c1);
        const int x0m = ((x0 % K) + K) % K;
        for (int k0 = 0; k0 < Kb; k0 += kConvChunk) {
            __syncthreads();
            for (int e = threadIdx.x; e < kConvChunk * LT; e += blockDim.x) {
                const int j = e / kConvChunk, kk = e % kConvChunk, k = k0 + kk, l = l0 + j;
                float2 v = make_float2(0.0f, 0.0f);
                if (k < Kb && l < L) {
                    v = psi[((size_t)l * Q + q) * Kb + k];
                    const float a = ((k == 0 || 2 * k == K) ? 1.0f : 2.0f) * inv_k;
                    v.x *= a;
                    v.y *= a;
                }
                ps[kk][j] = v;
            }
            __syncthreads();
            float s, c;
            sincospif((float)((k0 * x0m) % K) * two_over_k + (float)k0 * f * two_over_k, &s, &c);
            const int kn = min(kConvChunk, Kb - k0);
            for (int kk = 0; kk < kn; ++kk) {
                const float4 *p4 = reinterpret_cast<const float4 *>(&ps[kk][0]);
#pragma unroll
                for (int j = 0; j < LT / 2; ++j) {
                    const float4 v = p4[j];  // frames 2j, 2j+1: (re, im, re, im)
                    acc[2 * j] = fmaf(c, v.x, fmaf(-s, v.y, acc[2 * j]));
                    acc[2 * j + 1] = fmaf(c, v.z, fmaf(-s, v.w, acc[2 * j + 1]));
                }
                const float cn = c * c1 - s * s1;
                s = fmaf(s, c1, c * s1);
                c = cn;
            }
        }
    }
    map_epilogue<LT>(acc, i, J, l0, L, maps, part, n_tiles, red);
}

// ---------------------------------------------------------------------------
// K5: per frame, the maximum key over all candidate tiles, decoded into the
// first maximiser and its value.  One CTA per frame, shuffle reductions.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_argmax(const unsigned long long *__restrict__ part,
                                                int n_tiles, int32_t *__restrict__ argmax,
                                                float *__restrict__ peak) {
    __shared__ unsigned long long red[8];
    const int l = blockIdx.x;
    unsigned long long k = 0ull;
    // launched behind the map kernel with programmatic stream serialization:
    // wait until that kernel's keys are complete and visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const unsigned long long v = part[(size_t)l * n_tiles + t];
        k = v > k ? v : k;
    }
    k = warp_max_u64(k);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x < 32) {
        k = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
        k = warp_max_u64(k);
        if (threadIdx.x == 0) {
            argmax[l] = (int32_t)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull));
            if (peak != nullptr) peak[l] = key_value(k);
        }
    }
}

constexpr int kFramesPerCta = 16;

}  // namespace

cudaError_t launch_phat(const float2 *y, int L, int M, int Kb, const int2 *pairs, int Q,
                        int weighting, float2 *psi, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    dim3 grid((Kb + kPhatBins - 1) / kPhatBins, L);
    k_phat<<<grid, 256, sizeof(float2) * M * kPhatBins, s>>>(y, M, Kb, pairs, Q, weighting, psi);
    return cudaGetLastError();
}

cudaError_t launch_gcc_samples(const float2 *psi, int L, int Q, int K, const int32_t *nq,
                               const int32_t *off, int n_aux, const float2 *twid, float *xi,
                               int64_t s_stride, int64_t l_stride, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)(K + K / 2 + 1);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_gcc_samples,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float2) * (8192 + 4097)));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_gcc_samples<<<dim3(Q, L), 128, smem, s>>>(psi, Q, K, nq, off, n_aux, twid, xi, s_stride,
                                                 l_stride);
    return cudaGetLastError();
}

cudaError_t launch_interp_simt(const int32_t *x, int64_t J_pad, int64_t J, int Q,
                               const int32_t *nq, const int32_t *off, int n_aux, int xf,
                               const float *xi, int L_pad, int L, float *maps,
                               unsigned long long *part, int n_tiles, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    dim3 grid((unsigned)(J_pad / kTileJ), (L + kFramesPerCta - 1) / kFramesPerCta);
    k_interp_simt<kFramesPerCta><<<grid, kTileJ, 0, s>>>(x, J_pad, J, Q, nq, off, n_aux, xf, xi,
                                                         L_pad, L, maps, part, n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_conv_simt(const int32_t *x, int64_t J_pad, int64_t J, int Q, int K, int xf,
                             const float2 *psi, int L, float *maps, unsigned long long *part,
                             int n_tiles, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    dim3 grid((unsigned)(J_pad / kTileJ), (L + kFramesPerCta - 1) / kFramesPerCta);
    k_conv_simt<kFramesPerCta><<<grid, kTileJ, 0, s>>>(x, J_pad, J, Q, K, xf, psi, L, maps,
                                                       part, n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_argmax(const unsigned long long *part, int n_tiles, int L, int32_t *argmax,
                          float *peak, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_argmax, part, n_tiles, argmax, peak);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace srp
