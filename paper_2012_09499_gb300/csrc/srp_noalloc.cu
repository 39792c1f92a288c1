// srp_gcc_samples_static: the critical GCC samples of STFT frames without any
// device allocation, for callers that may not call cudaMalloc (for example
// code running where the allocator is owned by someone else, or a real-time
// audio thread that must not take the allocator's locks or risk its
// latency).  The cross-spectra scratch between the two kernels lives in a
// file-scope __device__ array of fixed size instead of plan-owned memory, and
// the pair tables travel as a kernel argument.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "srp_internal.h"

namespace srp {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB
constexpr int kStaticMaxM = 16;
constexpr int kStaticMaxQ = kStaticMaxM * (kStaticMaxM - 1) / 2;
constexpr int kMaxDevices = 64;
constexpr int kBins = 64;

// Cross spectra psi[L][Q][Kb] of the call in flight.  Every device that
// loads the library holds these 8 MiB until the process exits.
static __device__ __align__(256) unsigned char g_psi_scratch[kStaticScratchBytes];

struct PairTable {
    int2 mp[kStaticMaxQ];  // (m, m')
    int32_t nq[kStaticMaxQ];
    int32_t off[kStaticMaxQ];
};

// psi_q(k) = u_m(k) conj(u_m'(k)), u = y / |y| (0 where y = 0): the PHAT
// weighted cross spectrum of Eq. corrmatrix.
__global__ void __launch_bounds__(256) k_phat_static(const float2 *__restrict__ y, int M, int Kb,
                                                     int Q, PairTable t, float2 *__restrict__ psi) {
    __shared__ float2 u[kStaticMaxM * kBins];
    const int l = blockIdx.y, k0 = blockIdx.x * kBins;
    for (int e = threadIdx.x; e < M * kBins; e += blockDim.x) {
        const int m = e / kBins, k = k0 + e % kBins;
        float2 v = make_float2(0.0f, 0.0f);
        if (k < Kb) {
            v = y[((size_t)l * M + m) * Kb + k];
            const float a = hypotf(v.x, v.y);
            v = a > 0.0f ? make_float2(v.x / a, v.y / a) : make_float2(0.0f, 0.0f);
        }
        u[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Q * kBins; e += blockDim.x) {
        const int q = e / kBins, kk = e % kBins, k = k0 + kk;
        if (k >= Kb) continue;
        const float2 a = u[t.mp[q].x * kBins + kk], b = u[t.mp[q].y * kBins + kk];
        psi[((size_t)l * Q + q) * Kb + k] =
            make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
    }
}

// xi_q(n) = (1/K) sum_k a_k Re[psi_q(k) e^{j 2 pi k n / K}] at the critical
// lags of Eq. SRPapprox; twiddles are generated into shared memory.
__global__ void __launch_bounds__(128) k_gcc_static(const float2 *__restrict__ psi, int Q, int K,
                                                    int n_aux, PairTable t, float *__restrict__ xi,
                                                    int S) {
    extern __shared__ float2 sm[];
    const int Kb = K / 2 + 1;
    float2 *tw = sm, *ps = sm + K;
    const int q = blockIdx.x, l = blockIdx.y;
    for (int j = threadIdx.x; j < K; j += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)j / (float)K, &s, &c);
        tw[j] = make_float2(c, s);
    }
    const float2 *row = psi + ((size_t)l * Q + q) * Kb;
    for (int k = threadIdx.x; k < Kb; k += blockDim.x) {
        const float2 v = row[k];
        const float a = (k == 0 || 2 * k == K) ? 1.0f : 2.0f;
        ps[k] = make_float2(a * v.x, a * v.y);
    }
    __syncthreads();
    const int nmax = t.nq[q] + n_aux, base = t.off[q];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i <= 2 * nmax; i += (int)(blockDim.x >> 5)) {
        const int n = i - nmax, nm = ((n % K) + K) % K;
        float acc = 0.0f;
        for (int k = lane; k < Kb; k += 32) {
            const float2 w = tw[(k * nm) % K], p = ps[k];
            acc = fmaf(p.x, w.x, acc);
            acc = fmaf(-p.y, w.y, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) xi[(size_t)l * S + base + i] = acc / (float)K;
    }
}

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Largest dynamic shared memory of k_gcc_static: K + K/2 + 1 twiddles and
// bins at K = 8192.
constexpr int kGccStaticMaxSmem = (int)sizeof(float2) * (8192 + 4097);

// Per-device set-up, once, under the lock: the device address of
// g_psi_scratch (host code only sees a host-side stand-in under that name),
// and k_gcc_static's shared-memory limit raised to the largest size any K
// needs, so that no later call changes a process-wide kernel attribute
// while another host thread launches.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        e = cudaFuncSetAttribute(k_gcc_static, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kGccStaticMaxSmem);
        if (e != cudaSuccess) return e;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_psi_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace srp

using namespace srp;

extern "C" SRP_API srp_status srp_gcc_samples_static(int32_t M, int32_t K, int32_t n_aux,
                                                     const int32_t *Nq, const void *d_y, int32_t L,
                                                     float *d_xi, srp_stream_t s) {
    if (M < 2 || M > kStaticMaxM) {
        set_error("srp_gcc_samples_static: M must be in [2, 16]");
        return SRP_ERR_INVALID_ARG;
    }
    if (K < 4 || K > 8192 || (K & 1)) {
        set_error("srp_gcc_samples_static: K must be even and in [4, 8192]");
        return SRP_ERR_INVALID_ARG;
    }
    if (n_aux < 0 || Nq == nullptr || L < 0 || L > 65535) {
        set_error("srp_gcc_samples_static: bad n_aux or Nq, or L outside [0, 65535]");
        return SRP_ERR_INVALID_ARG;
    }
    const int Q = M * (M - 1) / 2, Kb = K / 2 + 1;
    PairTable t = {};
    int64_t S = 0;
    int q = 0;
    for (int mp = 0; mp < M - 1; ++mp)
        for (int m = mp + 1; m < M; ++m, ++q) {
            if (Nq[q] < 0 || 2 * (int64_t)Nq[q] + 2 * n_aux + 1 > 8192) {
                set_error("srp_gcc_samples_static: N_q out of range");
                return SRP_ERR_INVALID_ARG;
            }
            t.mp[q] = make_int2(m, mp);
            t.nq[q] = Nq[q];
            t.off[q] = (int32_t)S;
            S += 2 * (int64_t)Nq[q] + 2 * n_aux + 1;
        }
    const size_t need = sizeof(float2) * (size_t)L * Q * Kb;
    if (need > kStaticScratchBytes) {
        set_error("srp_gcc_samples_static: L*Q*(K/2+1)*8 bytes exceeds the 8 MiB static scratch");
        return SRP_ERR_INVALID_ARG;
    }
    if (L == 0) return SRP_OK;
    if (d_y == nullptr || d_xi == nullptr) {
        set_error("srp_gcc_samples_static: NULL buffer");
        return SRP_ERR_INVALID_ARG;
    }
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_error(std::string("srp_gcc_samples_static: set-up: ") + cudaGetErrorString(e));
        return SRP_ERR_CUDA;
    }
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s);
    float2 *psi = static_cast<float2 *>(scratch);
    k_phat_static<<<dim3((Kb + kBins - 1) / kBins, L), 256, 0, cs>>>(
        static_cast<const float2 *>(d_y), M, Kb, Q, t, psi);
    const size_t smem = sizeof(float2) * (size_t)(K + Kb);  // <= kGccStaticMaxSmem
    k_gcc_static<<<dim3(Q, L), 128, smem, cs>>>(psi, Q, K, n_aux, t, d_xi, (int)S);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("srp_gcc_samples_static: launch: ") + cudaGetErrorString(e));
        return SRP_ERR_CUDA;
    }
    return SRP_OK;
}
