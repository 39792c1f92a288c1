// Building blocks of the tensor-core (tcgen05 / TMEM / TMA) map kernels:
// inline-PTX wrappers, bounded mbarrier waits, shared-memory descriptors, and
// the on-chip generators of operand A (sinc weights of Eq. SRPapprox and the
// steering matrix of Eq. GCC_IFT).  Included by srp_tc.cu (one plan per
// launch) and srp_batch.cu (many plans in one persistent launch).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace srp {
namespace tc {
namespace {

constexpr int kThreads = 224;        // warps 0-3: A generation + epilogue; 4: TMA; 5, 6: MMA
constexpr int kTmaWarp = 4, kMmaWarp0 = 5;
constexpr int kChunk = 64;           // lags per pipeline stage
constexpr uint32_t kATile = 128u * 128u;  // 128 candidates x 64 lags x 2 B
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s per wait
constexpr int kXRing = 8;            // (TDOA, sp) prefetch ring (slots per candidate row)
constexpr int kXAhead = kXRing - 1;  // pairs in flight ahead of the current one
constexpr int kXRingW = 4;           // the same ring in the kernel that also streams A blocks
constexpr int kMtStride = 132;       // floats per frame row of the epilogue tile (rows
                                     // 16-byte aligned for bulk stores)
constexpr int kMaxStages = 4;        // pipeline stages the kernels' barrier blocks hold

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

// One probe of the phase; a waiting thread is suspended in hardware (not
// spinning) until the phase completes or the hint of 20 us runs out.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 20000; "
        "selp.u32 %0, 1, 0, p; }"
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
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_timer() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            atomicOr(status, 1);
            return false;
        }
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel of the stream still runs;
// grid_dep_wait() returns once that kernel has completed and its memory
// operations are visible, grid_dep_launch() lets the next kernel start early.
// Both are no-ops for kernels launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
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

// One lane of the (converged) warp is elected.  A tcgen05.mma issued under
// the elected predicate, with operands the whole warp computed alike, is one
// instruction of the warp; issued under a plain lane test, the compiler must
// assume several active lanes with different operands and serialise them.
__device__ __forceinline__ bool elect_one() {
    uint32_t pred = 0;
    asm volatile(
        "{ .reg .pred P; elect.sync _|P, 0xffffffff; selp.b32 %0, 1, 0, P; }"
        : "=r"(pred));
    return pred != 0;
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

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16: A's rows are TMEM lanes and each
// 32-bit column holds two consecutive K elements (the lower K in the low half).
__device__ __forceinline__ void mma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p; }" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Four consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c,
                                         uint32_t d) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                 "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// 8, 16 or 32 consecutive 32-bit TMEM columns of this thread's lane in one
// instruction (v[0] at column taddr).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {"
        "%1, %2, %3, %4, %5, %6, %7, %8};"
        ::"r"(taddr),
          "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {"
        "%1, %2, %3, %4, %5, %6, %7, %8, "
        "%9, %10, %11, %12, %13, %14, %15, %16};"
        ::"r"(taddr),
          "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {"
        "%1, %2, %3, %4, %5, %6, %7, %8, "
        "%9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, "
        "%25, %26, %27, %28, %29, %30, %31, %32};"
        ::"r"(taddr),
          "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
          "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
          "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
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

// Shared-memory matrix descriptor: K-major without swizzle, core matrices of
// 8 rows x 16 bytes; LBO = 128 bytes between the two core matrices along K
// of a 16-element step, SBO = 256 bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc_none(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46);
}

// Bulk copy of bytes (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on the mbarrier with its byte count.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Bulk copy of bytes (a multiple of 16, both addresses 16-byte aligned) from
// shared to global memory, in this thread's bulk group.  The shared source
// may be reused once bulk_wait_read() has returned.
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (two lanes per instruction on sm_100+).
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 upk2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
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

// Where the weight generators put operand A.
enum ADst : int {
    kASmem = 0,    // shared-memory A tile, 128-byte swizzle
    kATmem = 1,    // tensor memory
    kAGlobal = 2   // global memory, canonical K-major layout without swizzle
};
constexpr uint32_t kAStep = 4096;  // one 16-slot MMA step of a 128-row A tile, 16-bit

// Store group cc of a candidate row of operand A: 8 16-bit values hv (and,
// with kSplit, their low parts lv).
//  kATmem: four 32-bit columns per group from column dst0 (dst1 for the low
//    parts) of this thread's lane.
//  kASmem: the A tile with the 128-byte swizzle: row address dst0, 16-byte
//    chunk cc ^ sw, low parts kATile bytes on.
//  kAGlobal: dst0 / dst1 index this row's first 16 bytes (as a uint4 offset
//    within the step block) in the generic pointers g0 / g1: group cc is
//    k-half cc & 1 of step cc >> 1, and a step block of kAStep bytes holds
//    16 row groups of two k-halves of 8 rows x 16 bytes, so group cc lands
//    (cc >> 1) * kAStep + (cc & 1) * 128 bytes past the row's position.
template <bool kSplit, int kDst>
__device__ __forceinline__ void store_group(uint32_t dst0, uint32_t dst1, uint32_t sw,
                                            uint32_t cc, const uint32_t (&hv)[4],
                                            const uint32_t (&lv)[4], uint4 *g0 = nullptr,
                                            uint4 *g1 = nullptr) {
    if (kDst == kATmem) {
        tmem_st4(dst0 + 4u * cc, hv[0], hv[1], hv[2], hv[3]);
        if (kSplit) tmem_st4(dst1 + 4u * cc, lv[0], lv[1], lv[2], lv[3]);
    } else if (kDst == kASmem) {
        const uint32_t off = dst0 + ((cc ^ sw) << 4);
        st_shared_v4(off, hv[0], hv[1], hv[2], hv[3]);
        if (kSplit) st_shared_v4(off + kATile, lv[0], lv[1], lv[2], lv[3]);
    } else {
        const size_t at = (size_t)dst0 + (size_t)(cc >> 1) * (kAStep / 16) + (size_t)(cc & 1) * 8;
        g0[at] = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        if (kSplit) g1[at] = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
}

// Store the NG groups cc0 .. cc0 + NG - 1 of a candidate row (hv[cc][e], and
// lv with kSplit).  In tensor memory the row's 4 NG columns are consecutive,
// so they go out as one x32 store (NG = 8), x16 + x8 (NG = 6), x16 or x8
// instead of NG x4 stores.
template <int NG, bool kSplit, int kDst>
__device__ __forceinline__ void store_row(uint32_t dst0, uint32_t dst1, uint32_t sw,
                                          uint32_t cc0, const uint32_t (&hv)[NG][4],
                                          const uint32_t (&lv)[NG][4], uint4 *g0, uint4 *g1) {
    if (kDst == kATmem) {
#pragma unroll
        for (int part = 0; part < (kSplit ? 2 : 1); ++part) {
            const uint32_t *v = part ? &lv[0][0] : &hv[0][0];
            const uint32_t t = (part ? dst1 : dst0) + 4u * cc0;
            if (NG == 8) {
                tmem_st32(t, v);
            } else if (NG == 6) {
                tmem_st16(t, v);
                tmem_st8(t + 16u, v + 16);
            } else if (NG == 4) {
                tmem_st16(t, v);
            } else if (NG == 2) {
                tmem_st8(t, v);
            } else {
#pragma unroll
                for (int cc = 0; cc < NG; ++cc)
                    tmem_st4(t + 4u * cc, v[4 * cc], v[4 * cc + 1], v[4 * cc + 2], v[4 * cc + 3]);
            }
        }
    } else {
#pragma unroll
        for (int cc = 0; cc < NG; ++cc)
            store_group<kSplit, kDst>(dst0, dst1, sw, (uint32_t)cc + cc0, hv[cc], lv[cc], g0, g1);
    }
}

// Weights of NG groups of 8 lags for one candidate row of operand A:
// w = sp / d with d = f + (mc - k) for lag slot k of the chunk, two lags per
// reciprocal, stored by store_group (groups cc0 .. cc0 + NG - 1 of the row).
// With kSplit, the low parts bf16(w - hi) are stored too.  Every weight of
// the chunk is computed into registers first; wait() then runs before the
// first store, so a generator that must wait for its stage to drain has its
// arithmetic done by the time the stage is free.
struct NoWait {
    __device__ __forceinline__ void operator()() const {}
};

template <int NG, bool kSplit, bool kHalf, int kDst, class Wait = NoWait>
__device__ __forceinline__ void gen_groups(uint32_t dst0, uint32_t dst1, uint32_t sw, float f,
                                           float mc, float sp, uint32_t cc0 = 0,
                                           uint4 *g0 = nullptr, uint4 *g1 = nullptr,
                                           Wait wait = Wait()) {
    const uint64_t f2 = pk2(f, f);
    const uint64_t two = pk2(2.0f, 2.0f);
    // m2 = (mc - k - 1, mc - k): the second lag of a pair first, so that
    // (db, da) * rr = (w_a, w_b) comes out in lag order
    uint64_t m2 = pk2(mc - 1.0f, mc);
    uint32_t hv[NG][4], lv[NG][4];
#pragma unroll
    for (int cc = 0; cc < NG; ++cc) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint64_t d2 = add2(f2, m2);  // (db, da), each rounded once
            m2 = sub2(m2, two);
            const float2 d = upk2(d2);
            const float rr = sp * rcp_approx(d.x * d.y);
            const float2 w = upk2(mul2(d2, pk2(rr, rr)));  // (w_a, w_b)
            lv[cc][e] = 0u;
            if (kHalf) {
                hv[cc][e] = pack_f16(w.x, w.y);
            } else {
                hv[cc][e] = pack_bf16(w.x, w.y);
                if (kSplit) {
                    const uint64_t h2 = pk2(__uint_as_float(hv[cc][e] << 16),
                                            __uint_as_float(hv[cc][e] & 0xFFFF0000u));
                    const float2 lo = upk2(sub2(pk2(w.x, w.y), h2));
                    lv[cc][e] = pack_bf16(lo.x, lo.y);
                }
            }
        }
    }
    wait();
    store_row<NG, kSplit, kDst>(dst0, dst1, sw, cc0, hv, lv, g0, g1);
}

// Steering weights of NG groups (4 bins each) for this thread's row of A: the
// element pair (cos theta_k, -sin theta_k) of bins k0, k0 + 1, ..., i.e.
// z = e^{-j theta_k}, starting from z0 and multiplied per bin by
// w' = (p, q) = e^{-j 2 pi x / K}: z w' = (a p - b q, b p + a q) for z = (a, b).
// As in gen_groups, the chunk is computed into registers before wait().
template <int NG, bool kSplit, bool kHalf, int kDst, class Wait = NoWait>
__device__ __forceinline__ void gen_steer(uint32_t dst0, uint32_t dst1, uint32_t sw, float za,
                                          float zb, float p, float q, uint32_t cc0 = 0,
                                          uint4 *g0 = nullptr, uint4 *g1 = nullptr,
                                          Wait wait = Wait()) {
    uint64_t z = pk2(za, zb);
    const uint64_t pp = pk2(p, p), qq = pk2(-q, q);
    uint32_t hv[NG][4], lv[NG][4];
#pragma unroll
    for (int cc = 0; cc < NG; ++cc) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 v = upk2(z);
            const uint64_t t = mul2(z, pp);
            uint64_t zn;
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(zn) : "l"(pk2(v.y, v.x)), "l"(qq), "l"(t));
            z = zn;
            lv[cc][e] = 0u;
            if (kHalf) {
                hv[cc][e] = pack_f16(v.x, v.y);
            } else {
                hv[cc][e] = pack_bf16(v.x, v.y);
                if (kSplit) {
                    const uint64_t h2 = pk2(__uint_as_float(hv[cc][e] << 16),
                                            __uint_as_float(hv[cc][e] & 0xFFFF0000u));
                    const float2 lo = upk2(sub2(pk2(v.x, v.y), h2));
                    lv[cc][e] = pack_bf16(lo.x, lo.y);
                }
            }
        }
    }
    wait();
    store_row<NG, kSplit, kDst>(dst0, dst1, sw, cc0, hv, lv, g0, g1);
}

}  // namespace
}  // namespace tc
}  // namespace srp
