// Critical GCC samples (Eq. GCC_IFT at tau = nT, Sec. 3.2) of every (frame,
// pair) row on the tensor cores.  The partial inverse DFT of all rows is one
// contraction over (bin, re/im):
//
//   D[r][c] = sum_k A[r][2k] B[c][2k] + A[r][2k+1] B[c][2k+1],  k = 0 .. K/2 - 1,
//   A[r][2k] = Re psi_r(k),  A[r][2k+1] = Im psi_r(k)     (row r = l Q + q),
//   B[c][2k] = a_k cos(2 pi k n / K),  B[c][2k+1] = -a_k sin(2 pi k n / K),
//
// with lag n = c - nmax for column c (nmax: the largest N_q + N_aux of the
// plan), a_0 = 1 and a_k = 2, so that xi_r(n) = D[r][c] / K + (1/K) Re
// psi_r(K/2) (-1)^n; the epilogue adds the Nyquist bin's term.  B is a plan
// constant (the twiddles, in FP64 and split into FP16 high and low parts); A,
// the PHAT-weighted cross spectrum (components in [-1, 1]), is formed from the
// STFT frames straight into shared memory in the 128-byte-swizzled K-major
// layout, also split, and each product is the three FP16 MMAs of the split
// (A_hi B_hi + A_hi B_lo + A_lo B_hi), accumulated in FP32 in tensor memory.
// With 11-bit significands the split represents both operands to about 2^-22
// of their range (BF16 high and low parts would leave 2^-17), so the samples
// come out at FP32 accuracy; PHAT bounds A, which FP16 needs (plans without
// PHAT weighting, or with cross-spectrum input, keep the CUDA-core kernel).
//
// Work: a CTA takes 128 rows and cpz chunks of 64 (bin, re/im) slots; the Z
// CTAs that share a row tile form one cluster, and CTA z of the cluster sums
// rows [z 128/Z, (z+1) 128/Z) of the Z partial products, read from the other
// CTAs' shared memory in rank order (the same sum for every run), then writes
// the samples like the CUDA-core sample kernel: sign-folded 16-bit operand B
// of the map (high and low parts for FP32) and, optionally, the FP32 samples.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "srp_device.cuh"
#include "srp_internal.h"
#include "srp_tc_common.cuh"

namespace cg = cooperative_groups;

namespace srp {
namespace {

using namespace dev;
using namespace tc;

constexpr int kGmThreads = 512;   // 16 warps: A formation, then the epilogue
constexpr int kGmHead = 8192;     // barriers, the rows' spectrum pointers and tables
constexpr int kGmMaxZ = 16;       // CTAs per cluster: 16 where the GPU schedules it, else 8
constexpr int kGmPortableZ = 8;
constexpr int kGmSmemMax = 227 * 1024;
// TMEM columns per CTA.  A CTA waits at the cluster barriers for the other
// CTAs of its cluster, which may share its SM; with at most 2048 / 512 = 4
// CTAs of this kernel per SM and 128 columns each, every CTA's allocation
// succeeds whichever of them share an SM, so no CTA can wait for columns
// that a CTA waiting on it holds.
constexpr uint32_t kGmTmemCols = 128;

struct GmArgs {
    const float2 *src;      // STFT frames [L][M][Kb] (kFromY) or cross spectra [L][Q][Kb]
    const int32_t *nq;      // [Q]
    const int32_t *offc;    // [Q] first 16-bit slot of pair q
    const int32_t *off;     // [Q] first FP32 sample of pair q (xi32)
    uint16_t *xi16;         // [1 or 2][L_pad][S_pad]
    float *xi32;            // [L][S32] or null
    unsigned long long *best;  // [L] per-frame argmax keys to clear, or null
    int *status;
    int M, Q, K, L, n_aux, weighting;
    int nmax;               // largest N_q + N_aux
    int N;                  // MMA N: lag columns, a multiple of 32, >= 2 nmax + 1
    int cpz;                // chunks of 64 slots per CTA
    int n_acc;              // TMEM accumulators (N columns each) the 16-slot steps rotate over
    int L_pad, S_pad, S32;
    uint32_t idesc;
    uint32_t a_bytes;       // A region (cpz x (hi, lo) tiles, or the partial sums if larger)
};

// Microphones (m, m') of pair q in the plan's enumeration (m' outer, m > m'
// inner), without a table load: the A loads then depend on no other load.
__device__ __forceinline__ int2 pair_of(int q, int M) {
    int mp = 0, cnt = M - 1;
    while (q >= cnt) {
        q -= cnt;
        ++mp;
        --cnt;
    }
    return make_int2(mp + 1 + q, mp);
}

// Weighted cross spectrum psi_r(k) of row r = (l, q), as K1 forms it.
template <bool kFromY>
__device__ __forceinline__ float2 cross_bin(const GmArgs &a, int l, int q, int k, int Kb) {
    if (kFromY) {
        const int2 p = pair_of(q, a.M);
        float2 x = __ldg(&a.src[((size_t)l * a.M + p.x) * Kb + k]);
        float2 y = __ldg(&a.src[((size_t)l * a.M + p.y) * Kb + k]);
        if (a.weighting == SRP_WEIGHT_PHAT) {
            x = unit_phase(x);
            y = unit_phase(y);
        }
        return times_conj(x, y);
    }
    return __ldg(&a.src[((size_t)l * a.Q + q) * Kb + k]);
}

template <int kFmt, bool kFromY>
__global__ void __launch_bounds__(kGmThreads, 2)
    k_gcc_samples_mma(const __grid_constant__ CUtensorMap tmap, const GmArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    // [0, 1024): barriers, TMEM address, abort flag; [1024, 3072): the tables
    // of the rows this CTA reduces; [4096, 8192): the spectrum pointers of
    // the tile's rows; then the A region (A_hi, A_lo of each chunk, 16 KB
    // each; later the partial sums), then B
    const uint32_t full_bar = base, mma_bar = base + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + 16);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + 20);
    float *row_nyq = reinterpret_cast<float *>(gbase + 1024);       // [128] Re psi(K/2)
    int *row_nmq = reinterpret_cast<int *>(gbase + 1536);           // [128] N_q + N_aux (-1: none)
    int *row_o16 = reinterpret_cast<int *>(gbase + 2048);           // [128] l S_pad + offc[q]
    int *row_o32 = reinterpret_cast<int *>(gbase + 2560);           // [128] l S32 + off[q]
    // [128] the row's two spectra (STFT rows of mics m, m'; null past the last row)
    const float2 **row_sp = reinterpret_cast<const float2 **>(gbase + 4096);
    const uint32_t a0 = base + (uint32_t)kGmHead;
    const uint32_t b0 = a0 + a.a_bytes;
    const uint32_t b_tile = (uint32_t)a.N * 128u;
    float *part = reinterpret_cast<float *>(gbase + kGmHead);  // [128][N + 1], over A
    const int pstride = a.N + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int z = blockIdx.x, tile = blockIdx.y, Z = gridDim.x;
    const int Kb = a.K / 2 + 1, R = a.L * a.Q;
    const int chunk0 = z * a.cpz;
    const int rz = 128 / Z;  // rows this CTA reduces: [z rz, (z + 1) rz)

    if (threadIdx.x == 0) {
        mbar_init(full_bar, 1);
        mbar_init(mma_bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kGmTmemCols);
    if (threadIdx.x >= kGmThreads - 128) {  // the last four warps: one tile row each
        const int r = (int)threadIdx.x - (kGmThreads - 128), rg = tile * 128 + r;
        const float2 *p0 = nullptr, *p1 = nullptr;
        if (rg < R) {
            const int l = rg / a.Q, q = rg - l * a.Q;
            if (kFromY) {
                const int2 p = pair_of(q, a.M);
                p0 = a.src + ((size_t)l * a.M + p.x) * Kb;
                p1 = a.src + ((size_t)l * a.M + p.y) * Kb;
            } else {
                p0 = a.src + ((size_t)l * a.Q + q) * Kb;
            }
        }
        row_sp[2 * r] = p0;
        row_sp[2 * r + 1] = p1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the map kernel may start its prologue once every CTA holds its TMEM
    grid_dep_launch();
    if (threadIdx.x == 0) {  // the twiddle chunks of this k-slice, high and low parts
        mbar_arrive_expect_tx(full_bar, 2u * b_tile * (uint32_t)a.cpz);
        for (int cc = 0; cc < a.cpz; ++cc) {
            const uint32_t bh = b0 + (uint32_t)cc * 2u * b_tile;
            tma_load_2d(bh, &tmap, (chunk0 + cc) * kChunk, 0, full_bar);
            tma_load_2d(bh + b_tile, &tmap, (chunk0 + cc) * kChunk, a.N, full_bar);
        }
    }
    if (a.best != nullptr && z == 0 && tile == 0)
        for (int i = threadIdx.x; i < a.L; i += blockDim.x) a.best[i] = 0ull;

    // ---- A: warp w forms rows w, w + 16, ..., lane = bin of the chunk ----
    // (re, im) of bin 32 chunk + lane are slots 2 lane, 2 lane + 1 of the chunk:
    // bytes 4 lane of the row's 128, in 16-byte unit (lane >> 2) ^ (row & 7).
    // Every load of a chunk (the warp's 8 rows, both spectra) is issued before
    // any arithmetic, so that one memory latency covers the chunk.
    constexpr int kRowsW = 128 / (kGmThreads / 32);  // rows per warp
    for (int cc = 0; cc < a.cpz; ++cc) {
        const int k = (chunk0 + cc) * 32 + lane;
        float2 x[kRowsW], y[kRowsW];
#pragma unroll
        for (int j = 0; j < kRowsW; ++j) {
            const int r = warp + (kGmThreads / 32) * j;
            const float2 *p0 = row_sp[2 * r], *p1 = row_sp[2 * r + 1];
            x[j] = y[j] = make_float2(0.0f, 0.0f);
            if (p0 != nullptr) {
                x[j] = __ldg(p0 + k);
                if (kFromY) y[j] = __ldg(p1 + k);
            }
        }
#pragma unroll
        for (int j = 0; j < kRowsW; ++j) {
            float2 v = x[j];
            if (kFromY) {
                float2 w = y[j];
                if (a.weighting == SRP_WEIGHT_PHAT) {
                    v = unit_phase(v);
                    w = unit_phase(w);
                }
                v = times_conj(v, w);
            }
            const int r = warp + (kGmThreads / 32) * j;
            const __half2 h2 = __floats2half2_rn(v.x, v.y);
            const float2 hf = __half22float2(h2);
            const uint32_t hi = *reinterpret_cast<const uint32_t *>(&h2);
            const float2 lo = make_float2(v.x - hf.x, v.y - hf.y);
            const uint32_t addr = a0 + (uint32_t)cc * 2u * kATile + (uint32_t)r * 128u +
                                  ((((uint32_t)lane >> 2) ^ ((uint32_t)r & 7u)) << 4) +
                                  ((uint32_t)lane & 3u) * 4u;
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(hi) : "memory");
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr + kATile),
                         "r"(pack_f16(lo.x, lo.y))
                         : "memory");
        }
    }
    fence_proxy_async();  // A's generic stores before the tensor core reads them
    __syncthreads();

    // ---- the contraction: warp 0 issues, one lane elected ----
    if (warp == 0) {
        const bool ok = mbar_try_wait(full_bar, 0) || mbar_wait(full_bar, 0, abort_flag, a.status);
        if (__all_sync(0xFFFFFFFFu, ok)) {
            tc_fence_after();
            if (elect_one()) {
                // 16-slot step g goes to accumulator g % n_acc (N columns each):
                // the tensor core rounds each accumulation toward zero, so the
                // fewer steps an accumulator chains, the smaller that bias
                for (int cc = 0; cc < a.cpz; ++cc) {
                    const uint32_t ah = a0 + (uint32_t)cc * 2u * kATile;
                    const uint32_t bh = b0 + (uint32_t)cc * 2u * b_tile;
                    const uint64_t dah = smem_desc_sw128(ah), dal = smem_desc_sw128(ah + kATile);
                    const uint64_t dbh = smem_desc_sw128(bh), dbl = smem_desc_sw128(bh + b_tile);
#pragma unroll
                    for (int s = 0; s < kChunk / 16; ++s) {
                        const int g = cc * (kChunk / 16) + s;
                        const uint32_t d = tmem + (uint32_t)((g % a.n_acc) * a.N);
                        const uint64_t adv = (uint64_t)(s * 2);  // 32 bytes in 16-byte units
                        mma_f16(d, dah + adv, dbh + adv, a.idesc, g >= a.n_acc ? 1u : 0u);
                        mma_f16(d, dah + adv, dbl + adv, a.idesc, 1u);
                        mma_f16(d, dal + adv, dbh + adv, a.idesc, 1u);
                    }
                }
                mma_commit(mma_bar);
            }
            __syncwarp();
        }
    }
    if (threadIdx.x >= kGmThreads - 128 && threadIdx.x - (kGmThreads - 128) < rz) {
        // while the MMAs run, the last four warps look up the rows this CTA
        // reduces (read after the cluster barrier below)
        const int rr = z * rz + (int)threadIdx.x - (kGmThreads - 128);
        const int rg = tile * 128 + rr;
        int nmq = -1, o16 = 0, o32 = 0;
        float nyq = 0.0f;
        if (rg < R) {
            const int l = rg / a.Q, q = rg - l * a.Q;
            nmq = __ldg(&a.nq[q]) + a.n_aux;
            o16 = l * a.S_pad + __ldg(&a.offc[q]);
            o32 = l * a.S32 + __ldg(&a.off[q]);
            nyq = cross_bin<kFromY>(a, l, q, a.K / 2, Kb).x;
        }
        row_nyq[rr] = nyq;
        row_nmq[rr] = nmq;
        row_o16[rr] = o16;
        row_o32[rr] = o32;
    }
    {
        const bool ok = mbar_try_wait(mma_bar, 0) || mbar_wait(mma_bar, 0, abort_flag, a.status);
        (void)ok;  // on a timeout the status is set; the cluster barriers below still run
    }
    tc_fence_after();

    // ---- partial sums: TMEM -> part[row][col] (over the A tiles, now read) ----
    // warp w reads TMEM lanes 32 (w & 3) .. + 31, columns of quarter w >> 2
    if (!*abort_flag) {
        const int row = 32 * (warp & 3) + lane;
        const int qn = a.N / 4, c0 = (warp >> 2) * qn;
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        for (int j0 = 0; j0 < qn; j0 += 8) {
            float v[8], t[8];
            tmem_ld8(trow + (uint32_t)(c0 + j0), v);
            for (int ai = 1; ai < a.n_acc; ++ai) {  // the accumulators, in order
                tmem_ld8(trow + (uint32_t)(ai * a.N + c0 + j0), t);
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) v[jj] += t[jj];
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) part[row * pstride + c0 + j0 + jj] = v[jj];
        }
    }
    tc_fence_before();
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();  // every CTA's partial sums are in its shared memory

    // ---- rows [z rz, (z+1) rz): the sum over the cluster, in rank order ----
    if (!*abort_flag) {
        const float inv_k = 1.0f / (float)a.K;
        for (int e = threadIdx.x; e < rz * a.N; e += blockDim.x) {
            const int rl = e / a.N, col = e - rl * a.N;
            const int rr = z * rz + rl;
            const int n = col - a.nmax, nmq = row_nmq[rr];
            if (n > nmq || n < -nmq) continue;  // also rows past the last (nmq = -1)
            float pv[kGmMaxZ];
#pragma unroll
            for (int src = 0; src < kGmMaxZ; ++src)
                if (src < Z) pv[src] = *cluster.map_shared_rank(&part[rr * pstride + col], src);
            float sum = 0.0f;
#pragma unroll
            for (int src = 0; src < kGmMaxZ; ++src)
                if (src < Z) sum += pv[src];
            const float nyq = row_nyq[rr];
            float v = (sum + ((n & 1) ? -nyq : nyq)) * inv_k;
            const int t = nmq + n;
            if (a.xi32 != nullptr) a.xi32[(size_t)row_o32[rr] + t] = v;
            if (n & 1) v = -v;
            const size_t hi = (size_t)row_o16[rr] + t;
            if (kFmt == 2) {
                __half h = __float2half_rn(v);
                a.xi16[hi] = *reinterpret_cast<uint16_t *>(&h);
            } else {
                __nv_bfloat16 h = __float2bfloat16_rn(v);
                a.xi16[hi] = *reinterpret_cast<uint16_t *>(&h);
                if (kFmt == 1) {
                    __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(h));
                    a.xi16[hi + (size_t)a.L_pad * a.S_pad] = *reinterpret_cast<uint16_t *>(&lo);
                }
            }
        }
    }
    cluster.sync();  // no CTA leaves while another still reads its partial sums
    if (warp == 0) tmem_dealloc(tmem, kGmTmemCols);
}

// IEEE half precision of x (|x| < 65504), rounded to nearest even, and back.
uint16_t host_f16(double x) {
    const uint16_t sign = x < 0.0 ? 0x8000u : 0u;
    const double v = fabs(x);
    if (v == 0.0) return sign;
    int e2;
    frexp(v, &e2);
    int E = e2 - 1;  // v = 1.f 2^E
    if (E < -14) return (uint16_t)(sign | (uint16_t)rint(ldexp(v, 24)));  // subnormal, 2^-24 steps
    double q = rint(ldexp(v, -E) * 1024.0 - 1024.0);
    if (q == 1024.0) {
        q = 0.0;
        ++E;
    }
    return (uint16_t)(sign | (uint16_t)((E + 15) << 10) | (uint16_t)q);
}

double host_f16_value(uint16_t h) {
    const int e = (h >> 10) & 0x1F, m = h & 0x3FF;
    const double v = e == 0 ? ldexp((double)m, -24) : ldexp(1024.0 + m, e - 25);
    return (h & 0x8000u) ? -v : v;
}

struct GmShape {
    int N = 0, Z = 0, cpz = 0;
    uint32_t a_bytes = 0;
    size_t smem = 0;
};

// zmax: the largest cluster the launch may use (8, or 16 where supported);
// plan-time checks use 8, whose CTAs need the most shared memory.
GmShape gm_shape(int K, int nmax, int zmax = kGmPortableZ) {
    GmShape g;
    if (K % kChunk != 0 || K < kChunk) return g;
    const int n_chunks = K / kChunk;  // 32 bins (64 slots) per chunk; the Nyquist bin apart
    const int N = (2 * nmax + 1 + 31) / 32 * 32;
    if (N > (int)kGmTmemCols) return g;
    int Z = std::min(zmax, n_chunks);
    while (n_chunks % Z != 0) --Z;
    const int cpz = n_chunks / Z;
    const size_t a_tiles = (size_t)cpz * 2 * kATile;
    const size_t p_bytes = (size_t)128 * (N + 1) * sizeof(float);
    const size_t a_bytes = std::max(a_tiles, (p_bytes + 1023) / 1024 * 1024);
    const size_t smem = 1024 + kGmHead + a_bytes + (size_t)cpz * 2 * N * 128;
    if (smem > (size_t)kGmSmemMax) return g;
    g.N = N;
    g.Z = Z;
    g.cpz = cpz;
    g.a_bytes = (uint32_t)a_bytes;
    g.smem = smem;
    return g;
}

typedef void (*GmKern)(const CUtensorMap, const GmArgs);

GmKern gm_kernel(int fmt) {
    static const GmKern kerns[3] = {k_gcc_samples_mma<0, true>, k_gcc_samples_mma<1, true>,
                                    k_gcc_samples_mma<2, true>};
    return kerns[fmt];
}

}  // namespace

int gcc_mma_setup(int K, int nmax, int fmt) {
    if (fmt < 0 || fmt > 2 || gm_shape(K, nmax).N == 0) return 0;
    const GmKern k = gm_kernel(fmt);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kGmSmemMax) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    // a cluster of 16 where the GPU can place one of this shape, else the portable 8
    int zmax = kGmPortableZ;
    const GmShape g = gm_shape(K, nmax, kGmMaxZ);
    if (g.Z == kGmMaxZ &&
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3((unsigned)g.Z, 1);
        q.blockDim = dim3(kGmThreads);
        q.dynamicSmemBytes = g.smem;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = (unsigned)g.Z;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int n_clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&n_clusters, k, &q) == cudaSuccess && n_clusters > 0)
            zmax = kGmMaxZ;
    }
    (void)cudaGetLastError();
    return zmax;
}

bool gcc_mma_fits(int K, int nmax) { return gm_shape(K, nmax).N > 0; }

size_t gcc_mma_twiddle_bytes(int K, int nmax) {
    const GmShape g = gm_shape(K, nmax);
    return g.N > 0 ? sizeof(uint16_t) * 2 * (size_t)g.N * K : 0;
}

cudaError_t gcc_mma_twiddles(int K, int nmax, uint16_t *d_tw, void *map_out) {
    const GmShape g = gm_shape(K, nmax);
    if (g.N == 0) return cudaErrorInvalidValue;
    // rows 0 .. N-1: high parts of the lag columns, rows N .. 2N-1: low parts
    std::vector<uint16_t> h((size_t)2 * g.N * K, 0);
    const double two_pi = 6.283185307179586476925286766559;
    for (int c = 0; c <= 2 * nmax; ++c) {
        const long long n = c - nmax;
        for (int k = 0; k < K / 2; ++k) {
            const double ak = k == 0 ? 1.0 : 2.0;
            const long long ph = (((long long)k * n) % K + K) % K;  // k n mod K, exact
            const double th = two_pi * (double)ph / (double)K;
            const double val[2] = {ak * cos(th), -ak * sin(th)};
            for (int p = 0; p < 2; ++p) {
                const uint16_t hi = host_f16(val[p]);
                const uint16_t lo = host_f16(val[p] - host_f16_value(hi));
                h[(size_t)c * K + 2 * k + p] = hi;
                h[((size_t)g.N + c) * K + 2 * k + p] = lo;
            }
        }
    }
    cudaError_t e = cudaMemcpy(d_tw, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return encode_xi_map(d_tw, 2 * g.N, K, g.N, map_out);
}

cudaError_t launch_gcc_samples_mma(const void *tw_map, const float2 *src, bool from_y, int M,
                                   int weighting, int L, int Q, int K,
                                   const int32_t *nq, const int32_t *offc, int n_aux, int nmax,
                                   uint16_t *xi16, int L_pad, int S_pad, int fmt,
                                   unsigned long long *best, float *xi32, const int32_t *off,
                                   int S32, int *status, int zmax, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    if (!from_y || weighting != SRP_WEIGHT_PHAT || fmt < 0 || fmt > 2) return cudaErrorInvalidValue;
    const int v = fmt;
    const GmShape g = gm_shape(K, nmax, zmax);
    if (g.N == 0) return cudaErrorInvalidValue;
    GmArgs a;
    a.src = src;
    a.nq = nq;
    a.offc = offc;
    a.off = off;
    a.xi16 = xi16;
    a.xi32 = xi32;
    a.best = best;
    a.status = status;
    a.M = M;
    a.Q = Q;
    a.K = K;
    a.L = L;
    a.n_aux = n_aux;
    a.weighting = weighting;
    a.nmax = nmax;
    a.N = g.N;
    a.cpz = g.cpz;
    a.L_pad = L_pad;
    a.S_pad = S_pad;
    a.S32 = S32;
    // kind::f16: FP32 accumulate (bit 4), A and B FP16 (0 at bits 7, 10), both
    // K-major, N >> 3 at bit 17, M = 128 >> 4 at bit 24
    a.idesc = (1u << 4) | ((uint32_t)(g.N >> 3) << 17) | ((128u >> 4) << 24);
    a.n_acc = std::max(1, std::min(g.cpz * (kChunk / 16), (int)kGmTmemCols / g.N));
    a.a_bytes = g.a_bytes;
    const int tiles = (L * Q + 127) / 128;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.Z, (unsigned)tiles);
    cfg.blockDim = dim3(kGmThreads);
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)g.Z;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const CUtensorMap &map = *reinterpret_cast<const CUtensorMap *>(tw_map);
    cudaError_t e = cudaLaunchKernelEx(&cfg, gm_kernel(v), map, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace srp
