// Tensor-core (tcgen05 / TMEM / TMA) kernels of the Nyquist SRP path:
//   k_gcc_samples_tc  critical GCC samples (Eq. GCC_IFT at tau = nT) as 16-bit
//                     operands, sign-folded and split for the FP32 path
//   k_interp_tc       map[l][i] = sum_q sum_n xi_q(n) sinc(x_iq - n)
//                     (Eq. SRPapprox summed over pairs, Eq. SRP_T_IFT) as one
//                     (J x S) x (S x L) contraction with the pair sum as the
//                     reduction axis, accumulated in TMEM, with the maps and
//                     the per-tile argmax keys written by the epilogue.
//
// Operand A (sinc weights) is generated on chip.  With x = x0 + f,
//   sinc(x - n) = (-1)^n * [(-1)^x0 sin(pi f) / pi] / (f + x0 - n),
// so (-1)^n moves into the GCC samples (B) and A[i][s] = sp_iq / d with
// sp_iq = (-1)^x0 sin(pi f)/pi and d = f + x0 - n.  Two neighbouring lags
// share one reciprocal: 1/da = db / (da db).  f = 0 (an exact sample) is
// evaluated as f = 2^-40, which gives the unit weight at n = x0 and weights
// below 1e-11 elsewhere.
//
// Lag axis: pair q owns ceil((2(N_q+N_aux)+1)/8) groups of 8 lags (the tail
// of the last group has B = 0), so every 16-byte shared-memory chunk of A
// belongs to one pair.  K is walked in chunks of 64 lags (one 128-byte
// swizzle row of 16-bit data).
//
// FP32 precision uses three BF16 products per step (A_hi B_hi + A_hi B_lo +
// A_lo B_hi, hi = bf16(v), lo = bf16(v - hi)); BF16 and FP16 precision use one.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "srp_device.cuh"
#include "srp_internal.h"

namespace srp {
namespace {

using namespace dev;

constexpr int kThreads = 192;        // warps 0-3: A generation + epilogue; 4: TMA; 5: MMA
constexpr int kTmaWarp = 4, kMmaWarp = 5;
constexpr int kChunk = 64;           // lags per pipeline stage
constexpr uint32_t kATile = 128u * 128u;  // 128 candidates x 64 lags x 2 B
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s per wait

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_timer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
                     bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, "
        "p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: gives up after kWaitLimitNs (or as soon as another thread of
// the CTA gave up), records SRP timeout in *status and returns false.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                       int *status) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort_flag) return false;
            if (global_timer() - t0 > kWaitLimitNs) {
                *abort_flag = 1;
                atomicOr(status, 1);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], "
        "[%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 or FP16 in, FP32 accumulate).
__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), tile base 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ---------------------------------------------------------------------------
// GCC samples as 16-bit operand B: xi'[row][slot], row = frame (hi) or
// L_pad + frame (lo), slot = off8[q] + t, value (-1)^n xi_q(n).
// ---------------------------------------------------------------------------
template <int kFmt>  // 0: bf16, 1: bf16 hi/lo split, 2: fp16
__global__ void __launch_bounds__(128) k_gcc_samples_tc(
    const float2 *__restrict__ psi, int Q, int K, const int32_t *__restrict__ nq,
    const int32_t *__restrict__ off8, int n_aux, const float2 *__restrict__ twid,
    uint16_t *__restrict__ xi16, int L_pad, int S_pad) {
    extern __shared__ float2 sm[];
    float2 *tw = sm, *ps = sm + K;
    const int q = blockIdx.x, l = blockIdx.y;
    stage_gcc_row(psi + ((size_t)l * Q + q) * (K / 2 + 1), twid, K, tw, ps);
    __syncthreads();
    const int base = off8[q];
    gcc_row(tw, ps, K, nq[q] + n_aux, [&](int t, int n, float v) {
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
// The contraction.
// ---------------------------------------------------------------------------
struct TcArgs {
    const int32_t *x;       // [Q][J_pad] fixed-point TDOA
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
};

template <bool kSplit, bool kHalf>
__global__ void __launch_bounds__(kThreads, 1) k_interp_tc(const __grid_constant__ CUtensorMap tmap,
                                                           const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // control block, then 1024-aligned stages, then the argmax scratch
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = smem_raw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase);  // full[4], empty[4], accum
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gbase + 80);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gbase + 84);
    const uint32_t b_tile = (uint32_t)a.N * 128u;
    const uint32_t stage_bytes = (kSplit ? 2u : 1u) * (kATile + b_tile);
    const uint32_t stage0 = base + 1024u;
    unsigned long long *red =
        reinterpret_cast<unsigned long long *>(gbase + 1024u + stage_bytes * (uint32_t)a.stages);

    auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
    auto empty_bar = [&](int s) { return smem_u32(&bars[4 + s]); };
    const uint32_t accum_bar = smem_u32(&bars[8]);
    auto a_hi = [&](int s) { return stage0 + (uint32_t)s * stage_bytes; };
    auto a_lo = [&](int s) { return stage0 + (uint32_t)s * stage_bytes + kATile; };
    auto b_hi = [&](int s) { return stage0 + (uint32_t)s * stage_bytes + (kSplit ? 2u : 1u) * kATile; };
    auto b_lo = [&](int s) { return b_hi(s) + b_tile; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int l0 = blockIdx.y * a.N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(full_bar(s), 128 + 1);
            mbar_init(empty_bar(s), 1);
        }
        mbar_init(accum_bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kTmaWarp) tmem_alloc(smem_u32(tmem_slot), a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ---------------- A generation: one candidate row per thread ----------------
        const int r = threadIdx.x;
        const int64_t i = (int64_t)blockIdx.x * 128 + r;
        const uint32_t row = (uint32_t)r * 128u, sw = (uint32_t)(r & 7);
        int q = -1, g_next = 0;
        // d = f + (mg - e) for lag e of the current group: mg is an exact
        // integer in FP32, so d is rounded once and is never 0 unless f is.
        float sp = 0.0f, f = 0.5f, mg = 0.0f;
        int32_t x_next = __ldg(&a.x[i]);
        int nmax_next = __ldg(&a.nq[0]) + a.n_aux;
        for (int c = 0; c < a.n_chunks; ++c) {
            const int st = c % a.stages;
            const uint32_t ph = (uint32_t)(c / a.stages) & 1u;
            if (c >= a.stages) mbar_wait(empty_bar(st), ph ^ 1u, abort_flag, a.status);
#pragma unroll 1
            for (int cc = 0; cc < 8; ++cc) {
                const int g = c * 8 + cc;
                if (g == g_next) {  // uniform: the next pair starts at this group
                    ++q;
                    if (q < a.Q) {
                        int x0;
                        decode_tdoa(x_next, a.xf, x0, f);
                        if (f == 0.0f) f = 9.094947017729282e-13f;  // 2^-40
                        sp = sinpif(f) * kInvPi;
                        if (x0 & 1) sp = -sp;
                        const int nmax = nmax_next;
                        mg = (float)(x0 + nmax);  // d - f at n = -nmax
                        g_next = g + (2 * nmax + 1 + 7) / 8;
                        if (q + 1 < a.Q) {
                            x_next = __ldg(&a.x[(size_t)(q + 1) * a.J_pad + i]);
                            nmax_next = __ldg(&a.nq[q + 1]) + a.n_aux;
                        }
                    } else {  // padding beyond the last pair
                        sp = 0.0f;
                        f = 0.5f;
                        mg = 0.0f;
                        g_next = 0x7FFFFFFF;
                    }
                }
                float w[8];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const float da = f + (mg - (float)e), db = f + (mg - (float)(e + 1));
                    const float rr = sp * rcp_approx(da * db);
                    w[e] = db * rr;
                    w[e + 1] = da * rr;
                }
                mg -= 8.0f;
                const uint32_t off = row + (((uint32_t)cc ^ sw) << 4);
                if (kHalf) {
                    st_shared_v4(a_hi(st) + off, pack_f16(w[0], w[1]), pack_f16(w[2], w[3]),
                                 pack_f16(w[4], w[5]), pack_f16(w[6], w[7]));
                } else {
                    uint32_t h[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) h[e] = pack_bf16(w[2 * e], w[2 * e + 1]);
                    st_shared_v4(a_hi(st) + off, h[0], h[1], h[2], h[3]);
                    if (kSplit) {
                        uint32_t lo[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float h0 = __uint_as_float(h[e] << 16);
                            const float h1 = __uint_as_float(h[e] & 0xFFFF0000u);
                            lo[e] = pack_bf16(w[2 * e] - h0, w[2 * e + 1] - h1);
                        }
                        st_shared_v4(a_lo(st) + off, lo[0], lo[1], lo[2], lo[3]);
                    }
                }
            }
            fence_proxy_async();
            mbar_arrive(full_bar(st));
        }

        // ---------------- epilogue: TMEM -> maps + argmax keys ----------------
        mbar_wait(accum_bar, 0, abort_flag, a.status);
        tc_fence_after();
        const bool valid = i < a.J;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j0 = 0; j0 < a.N; j0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)j0, v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const int l = l0 + j0 + jj;
                if (l < a.L) {
                    if (a.maps != nullptr && valid) a.maps[(size_t)l * a.J + i] = v[jj];
                    unsigned long long k = valid ? argmax_key(v[jj], (uint32_t)i) : 0ull;
                    k = warp_max_u64(k);
                    if (lane == 0) red[warp * a.N + j0 + jj] = k;
                }
            }
        }
        tc_fence_before();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        for (int j = threadIdx.x; j < a.N && l0 + j < a.L; j += 128) {
            unsigned long long k = red[j];
#pragma unroll
            for (int w2 = 1; w2 < 4; ++w2) {
                const unsigned long long t = red[w2 * a.N + j];
                k = t > k ? t : k;
            }
            a.part[(size_t)(l0 + j) * a.n_tiles + blockIdx.x] = k;
        }
    } else if (warp == kTmaWarp) {
        // ---------------- B loads (GCC samples) ----------------
        if (lane == 0) {
            const uint32_t bytes = (kSplit ? 2u : 1u) * b_tile;
            int issued = 0;
            for (int c = 0; c < a.n_chunks; ++c) {
                const int st = c % a.stages;
                const uint32_t ph = (uint32_t)(c / a.stages) & 1u;
                if (c >= a.stages && !mbar_wait(empty_bar(st), ph ^ 1u, abort_flag, a.status))
                    break;
                if (*abort_flag) break;
                mbar_arrive_expect_tx(full_bar(st), bytes);
                tma_load_2d(b_hi(st), &tmap, c * kChunk, l0, full_bar(st));
                if (kSplit) tma_load_2d(b_lo(st), &tmap, c * kChunk, a.L_pad + l0, full_bar(st));
                issued = c + 1;
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
        if (lane == 0) {
            for (int c = 0; c < a.n_chunks; ++c) {
                const int st = c % a.stages;
                const uint32_t ph = (uint32_t)(c / a.stages) & 1u;
                if (!mbar_wait(full_bar(st), ph, abort_flag, a.status)) break;
                tc_fence_after();
                const uint64_t dah = smem_desc_sw128(a_hi(st)), dbh = smem_desc_sw128(b_hi(st));
                const uint64_t dal = smem_desc_sw128(a_lo(st)), dbl = smem_desc_sw128(b_lo(st));
#pragma unroll
                for (int kk = 0; kk < kChunk / 16; ++kk) {
                    const uint64_t adv = (uint64_t)(kk * 2);  // 32 bytes in 16-byte units
                    mma_f16(tmem, dah + adv, dbh + adv, a.idesc, (c | kk) != 0);
                    if (kSplit) {
                        mma_f16(tmem, dah + adv, dbl + adv, a.idesc, 1);
                        mma_f16(tmem, dal + adv, dbh + adv, a.idesc, 1);
                    }
                }
                mma_commit(empty_bar(st));
            }
            mma_commit(accum_bar);
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

template <bool kSplit, bool kHalf>
cudaError_t launch_tc(const CUtensorMap &map, const TcArgs &a, int grid_y, size_t smem,
                      cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_interp_tc<kSplit, kHalf>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_interp_tc<kSplit, kHalf><<<dim3((unsigned)a.n_tiles, grid_y), kThreads, smem, s>>>(map, a);
    return cudaGetLastError();
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

cudaError_t launch_gcc_samples_tc(const float2 *psi, int L, int Q, int K, const int32_t *nq,
                                  const int32_t *off8, int n_aux, const float2 *twid,
                                  uint16_t *xi16, int L_pad, int S_pad, int fmt, cudaStream_t s) {
    if (L == 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)(K + K / 2 + 1);
    static bool attr[3] = {false, false, false};
    auto kern = fmt == 0 ? k_gcc_samples_tc<0> : (fmt == 1 ? k_gcc_samples_tc<1> : k_gcc_samples_tc<2>);
    if (!attr[fmt]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float2) * (8192 + 4097)));
        if (e != cudaSuccess) return e;
        attr[fmt] = true;
    }
    kern<<<dim3(Q, L), 128, smem, s>>>(psi, Q, K, nq, off8, n_aux, twid, xi16, L_pad, S_pad);
    return cudaGetLastError();
}

int interp_tc_frames_per_cta(int L) {
    const int n = ((L + 15) / 16) * 16;
    return n > 256 ? 256 : n;
}

cudaError_t launch_interp_tc(const void *xi_map, int N, const int32_t *x, int64_t J_pad,
                             int64_t J, int Q, const int32_t *nq, int n_aux, int xf, int S_pad,
                             int L_pad, int L, int precision, float *maps,
                             unsigned long long *part, int n_tiles, int *status, cudaStream_t s) {
    // N is the plan's frames per CTA: the height of the tensor map's box.
    if (L == 0) return cudaSuccess;
    if (N < 16 || N > 256 || (N & 15)) return cudaErrorInvalidValue;
    const bool split = precision == SRP_PREC_FP32, half = precision == SRP_PREC_FP16;
    TcArgs a;
    a.x = x;
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
    uint32_t cols = 32;
    while (cols < (uint32_t)N) cols <<= 1;
    a.tmem_cols = cols;
    const size_t stage = (split ? 2 : 1) * (size_t)(kATile + (uint32_t)N * 128u);
    const size_t fixed = 1024 + 1024 + 4 * sizeof(unsigned long long) * (size_t)N;
    // two stages (or more if they fit in half the SM) and at most four
    int stages = (int)((113 * 1024 - fixed) / stage);
    if (stages < 2) stages = (int)((227 * 1024 - fixed) / stage);
    if (stages > 4) stages = 4;
    if (stages < 2) return cudaErrorInvalidConfiguration;
    a.stages = stages;
    a.maps = maps;
    a.part = part;
    a.n_tiles = n_tiles;
    a.status = status;
    const size_t smem = fixed + stage * (size_t)stages;
    const int grid_y = (L + N - 1) / N;
    const CUtensorMap &map = *reinterpret_cast<const CUtensorMap *>(xi_map);
    if (split) return launch_tc<true, false>(map, a, grid_y, smem, s);
    if (half) return launch_tc<false, true>(map, a, grid_y, smem, s);
    return launch_tc<false, false>(map, a, grid_y, smem, s);
}

}  // namespace srp
