// Coarse-to-fine search on the interpolated map.  Sec. 3.3 notes that the
// interpolation cost R_int = N/K falls far lower if, instead of every
// candidate of a fine grid, only points near a coarse maximiser are
// evaluated.  srp_refine does that on top of a Nyquist plan: per frame, the
// approximation of Eq. SRPapprox summed over pairs (Eq. SRP_T_IFT) is
// evaluated at a stencil of points around a centre, the best point becomes
// the next centre, and the stencil shrinks by a constant factor per level.
//
// The GCC samples are the ones the plan's last srp_map computed (K2), read
// in the precision the map itself used and staged per frame in shared
// memory.  The TDOA of each stencil point is computed in FP32 from the
// geometry (Eq. Deltat_i or Eq. Deltat_i_spher), with coordinates relative
// to the microphones' centroid and the distance difference in a form without
// cancellation; the centres themselves are kept in FP64.  The sinc weight of
// Eq. SRPapprox is written, like the map's, as
//   sinc(x - n) = (-1)^n [(-1)^x0 sin(pi f) / pi] / (f + x0 - n),
// x = x0 + f, x0 the nearest integer, f = 0 evaluated as f = 2^-40.
// One cluster of CTAs per frame, one warp per stencil point, its lanes over
// the pairs.
#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "srp_device.cuh"
#include "srp_internal.h"

struct srp_refiner_s {
    srp_plan_s *plan = nullptr;
    int device = 0;
    int F = 0, levels = 0;
    double shrink = 1.0;
    double centroid[3] = {0.0, 0.0, 0.0};  // of the microphones
    float *d_mic = nullptr;       // [M][3] microphones relative to the centroid
    double *d_offsets = nullptr;  // [F][3]
    double *d_grid = nullptr;     // [J][3] or null
    int pstride = 0;              // staged samples per pair (odd)
    size_t smem = 0;              // dynamic shared memory of the kernel
    bool staged = false;          // the frame's samples fit in shared memory
};

namespace srp {
namespace {

using namespace dev;
namespace cg = cooperative_groups;

constexpr int kRefineThreads = 512;
constexpr int kCluster = 4;  // CTAs per frame
constexpr int kRefineWarps = kRefineThreads / 32;
constexpr int kMaxOffsets = 1024;
constexpr int kMaxLevels = 64;
constexpr size_t kRefineSmemMax = 200 * 1024;

// Where the GCC samples of the plan's last map are.
enum XiSource : int {
    kXiF32 = 0,   // CUDA-core plans: FP32 [S_pad][L_pad], not sign-folded
    kXiBf16 = 1,  // tensor-core BF16: [L_pad][Sc] sign-folded (-1)^n xi(n)
    kXiSplit = 2, // tensor-core FP32: high parts as kXiBf16, low parts lo_off further
    kXiF16 = 3    // tensor-core FP16: [L_pad][Sc] sign-folded
};

struct RefineArgs {
    const float *mic;        // [M][3] relative to the centroid
    const int2 *pairs;       // [Q] (m, m')
    const int32_t *nq;       // [Q]
    const int32_t *off;      // [Q] first sample row (kXiF32) or 16-bit slot of pair q
    int M, Q, n_aux;
    float fs_c;              // fs / c: samples per metre of path difference
    int far;                 // candidates are unit directions
    int src;
    const float *xi;         // kXiF32
    const uint16_t *xi16;    // 16-bit sources
    int64_t ld;              // kXiF32: row stride (L_pad); 16-bit: frame stride (Sc)
    int64_t lo_off;          // kXiSplit: offset of the low parts
    int pstride;             // staged samples per pair (odd: pairs start on distinct banks)
    double cx, cy, cz;       // microphone centroid
    const double *offsets;   // [F][3]
    int F, levels;
    double shrink;
    const double *grid;      // [J][3] or null
    int64_t J;
    const int32_t *argmax;   // [L] centre indices, or null
    const double *centres;   // [L][3] centres, or null
    double *best_xyz;        // [L][3]
    float *best_val;         // [L]
    float *values;           // [L][F] last level, or null
    int *status;
};

// Sign-folded GCC sample (-1)^n xi_q(n) of frame l at slot t = n + nmax.
__device__ __forceinline__ float folded_sample(const RefineArgs &a, int l, int q, int t, int n) {
    const int64_t o = (int64_t)__ldg(&a.off[q]) + t;
    if (a.src == kXiF32) {
        const float v = __ldg(&a.xi[o * a.ld + l]);
        return (n & 1) ? -v : v;
    }
    const int64_t k = (int64_t)l * a.ld + o;
    const uint16_t h = __ldg(&a.xi16[k]);
    if (a.src == kXiF16) return __half2float(__ushort_as_half(h));
    float v = __uint_as_float((uint32_t)h << 16);
    if (a.src == kXiSplit) v += __uint_as_float((uint32_t)__ldg(&a.xi16[k + a.lo_off]) << 16);
    return v;
}

// Candidate point of stencil entry f around centre c at stencil scale s, in
// FP64; on a direction grid the displaced point is projected back onto the
// sphere.
__device__ __forceinline__ void stencil_point(const RefineArgs &a, const double *c, int f,
                                              double s, double *p) {
    for (int k = 0; k < 3; ++k) p[k] = c[k] + s * __ldg(&a.offsets[3 * f + k]);
    if (a.far) {
        const double nrm = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        if (nrm > 0.0)
            for (int k = 0; k < 3; ++k) p[k] /= nrm;
        else
            for (int k = 0; k < 3; ++k) p[k] = c[k];
    }
}

// TDOA of pair (m, m') in samples at point p (relative to the centroid on a
// point grid, a unit direction on a direction grid), FP32.  Near field:
// |p - a| - |p - b| = (|p - a|^2 - |p - b|^2) / (|p - a| + |p - b|)
// = (b - a).(2p - a - b) / (|p - a| + |p - b|), which has no cancellation.
__device__ __forceinline__ float pair_tdoa(const RefineArgs &a, const float *mic, const float *p,
                                           int m, int mp) {
    const float ax = mic[3 * m], ay = mic[3 * m + 1], az = mic[3 * m + 2];
    const float bx = mic[3 * mp], by = mic[3 * mp + 1], bz = mic[3 * mp + 2];
    if (a.far) return a.fs_c * ((ax - bx) * p[0] + (ay - by) * p[1] + (az - bz) * p[2]);
    const float dax = p[0] - ax, day = p[1] - ay, daz = p[2] - az;
    const float dbx = p[0] - bx, dby = p[1] - by, dbz = p[2] - bz;
    const float ra = sqrtf(dax * dax + day * day + daz * daz);
    const float rb = sqrtf(dbx * dbx + dby * dby + dbz * dbz);
    const float num = (bx - ax) * (dax + dbx) + (by - ay) * (day + dby) + (bz - az) * (daz + dbz);
    const float den = ra + rb;
    return den > 0.0f ? a.fs_c * num / den : 0.0f;
}

// Eq. SRPapprox for one pair at TDOA x: sum_n xi(n) sinc(x - n) with the
// samples sign-folded, sinc(x - n) = (-1)^n sp / (f + x0 - n).
template <bool kStaged>
__device__ __forceinline__ float pair_value(const RefineArgs &a, const float *xs, int l, int q,
                                            float x) {
    const float x0f = rintf(x);
    float f = x - x0f;  // exact: x0f is the integer nearest x
    if (f == 0.0f) f = 9.094947017729282e-13f;  // 2^-40
    const int x0 = (int)x0f;
    float sp = sinpif(f) * 0.318309886183790671538f;  // sin(pi f) / pi
    if (x0 & 1) sp = -sp;
    const int nmax = __ldg(&a.nq[q]) + a.n_aux;
    const int top = x0 + nmax;  // x0 - n at slot t is top - t, an exact integer in FP32
    auto term = [&](int t) {
        const float v = kStaged ? xs[q * a.pstride + t] : folded_sample(a, l, q, t, t - nmax);
        return v * __fdividef(sp, f + (float)(top - t));
    };
    // four independent partial sums keep several reciprocals in flight
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
    int t = 0;
    for (; t + 3 <= 2 * nmax; t += 4) {
        acc0 += term(t);
        acc1 += term(t + 1);
        acc2 += term(t + 2);
        acc3 += term(t + 3);
    }
    for (; t <= 2 * nmax; ++t) acc0 += term(t);
    return (acc0 + acc1) + (acc2 + acc3);
}

// One cluster of kCluster CTAs per frame: CTA rank r evaluates the stencil
// points of warps r W .. r W + W - 1 of every round of kCluster W points (W
// warps per CTA).  After a level, every CTA sends its best (key, value) to
// all CTAs of the cluster through distributed shared memory, double-buffered
// by level parity (a CTA can rewrite a buffer only after the next cluster
// barrier, which every CTA reaches after reading it), and all of them take
// the same first maximiser and the same next centre.
template <bool kStaged>
__global__ void __launch_bounds__(kRefineThreads) k_refine(const RefineArgs a) {
    extern __shared__ float rsm[];
    float *mic = rsm;                 // [M][3]
    float *vals = rsm + 3 * a.M;      // [F] (this CTA's points)
    float *xs = vals + a.F;           // [Q][pstride] sign-folded samples (kStaged)
    __shared__ double centre[3];
    __shared__ float centre_rel[3];   // centre - centroid (point grid) or centre (directions)
    __shared__ unsigned long long keys[2][kCluster];
    __shared__ float kvals[2][kCluster];
    __shared__ int s_bad;
    __shared__ float s_val;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int l = blockIdx.x / kCluster, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto mine = [&](int f) { return (f / kRefineWarps) % kCluster == rank; };
    for (int i = tid; i < 3 * a.M; i += blockDim.x) mic[i] = a.mic[i];
    if (kStaged)
        for (int i = tid; i < a.Q * a.pstride; i += blockDim.x) {
            const int q = i / a.pstride, t = i - q * a.pstride;
            const int nmax = __ldg(&a.nq[q]) + a.n_aux;
            xs[i] = t <= 2 * nmax ? folded_sample(a, l, q, t, t - nmax) : 0.0f;
        }
    if (tid == 0) {
        s_bad = 0;
        if (a.centres != nullptr) {
            for (int k = 0; k < 3; ++k) centre[k] = a.centres[3 * (int64_t)l + k];
        } else {
            const int idx = a.argmax[l];
            if (idx < 0 || (int64_t)idx >= a.J) {
                s_bad = 1;
                if (rank == 0) atomicOr(a.status, 2);
            } else {
                for (int k = 0; k < 3; ++k) centre[k] = a.grid[3 * (int64_t)idx + k];
            }
        }
    }
    __syncthreads();
    if (s_bad) {  // the same for every CTA of the cluster: NaN outputs, no cluster barrier
        const float nan = __int_as_float(0x7fc00000);
        if (rank == 0 && tid < 3) a.best_xyz[3 * (int64_t)l + tid] = (double)nan;
        if (rank == 0 && tid == 0) a.best_val[l] = nan;
        if (a.values != nullptr)
            for (int f = tid; f < a.F; f += blockDim.x)
                if (mine(f)) a.values[(int64_t)l * a.F + f] = nan;
        return;
    }
    double scale = 1.0;
    for (int v = 0; v < a.levels; ++v) {
        if (tid == 0) {
            centre_rel[0] = (float)(a.far ? centre[0] : centre[0] - a.cx);
            centre_rel[1] = (float)(a.far ? centre[1] : centre[1] - a.cy);
            centre_rel[2] = (float)(a.far ? centre[2] : centre[2] - a.cz);
        }
        __syncthreads();
        const float sf = (float)scale;
        // one warp per stencil point, its lanes over the pairs
        for (int f = rank * kRefineWarps + warp; f < a.F; f += kCluster * kRefineWarps) {
            float p[3];
            for (int k = 0; k < 3; ++k) p[k] = centre_rel[k] + sf * (float)__ldg(&a.offsets[3 * f + k]);
            if (a.far) {
                const float nrm2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
                if (nrm2 > 0.0f) {
                    const float r = rsqrtf(nrm2);
                    for (int k = 0; k < 3; ++k) p[k] *= r;
                } else {
                    for (int k = 0; k < 3; ++k) p[k] = centre_rel[k];
                }
            }
            float acc = 0.0f;
            for (int q = lane; q < a.Q; q += 32) {
                const int2 pr = __ldg(&a.pairs[q]);
                acc += pair_value<kStaged>(a, xs, l, q, pair_tdoa(a, mic, p, pr.x, pr.y));
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (lane == 0) vals[f] = acc;
        }
        __syncthreads();
        const int buf = v & 1;
        if (tid < 32) {  // this CTA's first maximiser: the largest value, lowest index
            unsigned long long key = 0ull;
            for (int f = tid; f < a.F; f += 32) {
                if (!mine(f)) continue;
                const unsigned long long k =
                    ((unsigned long long)ordered_value(vals[f]) << 32) | (0xFFFFFFFFu - (uint32_t)f);
                key = k > key ? k : key;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, key, o);
                key = other > key ? other : key;
            }
            if (tid < kCluster) {  // lane c sends the key to CTA c of the cluster
                const int f = (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu));
                unsigned long long *rk = cluster.map_shared_rank(&keys[buf][0], tid);
                float *rv = cluster.map_shared_rank(&kvals[buf][0], tid);
                rk[rank] = key;
                rv[rank] = key != 0ull ? vals[f] : 0.0f;
            }
        }
        if (v + 1 == a.levels && a.values != nullptr)
            for (int f = tid; f < a.F; f += blockDim.x)
                if (mine(f)) a.values[(int64_t)l * a.F + f] = vals[f];
        cluster.sync();  // every CTA's key has arrived everywhere
        if (tid == 0) {
            int c = 0;
            for (int k = 1; k < kCluster; ++k)
                if (keys[buf][k] > keys[buf][c]) c = k;
            const int best = (int)(0xFFFFFFFFu - (uint32_t)(keys[buf][c] & 0xFFFFFFFFu));
            double p[3];
            stencil_point(a, centre, best, scale, p);
            for (int k = 0; k < 3; ++k) centre[k] = p[k];
            s_val = kvals[buf][c];
        }
        __syncthreads();
        scale *= a.shrink;
    }
    if (rank == 0 && tid < 3) a.best_xyz[3 * (int64_t)l + tid] = centre[tid];
    if (rank == 0 && tid == 0) a.best_val[l] = s_val;
}

}  // namespace
}  // namespace srp

using namespace srp;

static void refiner_release(srp_refiner_s *r) {
    cudaFree(r->d_mic);
    cudaFree(r->d_offsets);
    cudaFree(r->d_grid);
    r->d_mic = nullptr;
    r->d_offsets = r->d_grid = nullptr;
}

static bool all_finite(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

extern "C" {

srp_status srp_refiner_create(srp_handle h, const srp_plan_desc *d, const srp_refine_desc *rd,
                              srp_refiner *out) {
    if (out == nullptr) return fail(SRP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (h == nullptr || d == nullptr || rd == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "NULL handle or descriptor");
    if (h->mode != SRP_MODE_NYQUIST)
        return fail(SRP_ERR_UNSUPPORTED, "refinement interpolates the GCC samples of a Nyquist plan");
    Layout lay;
    srp_status st = describe_layout(d, lay);
    if (st != SRP_OK) return st;
    const Layout &hl = h->lay;
    if (d->mode != h->mode || lay.M != hl.M || lay.J != hl.J || lay.K != hl.K ||
        lay.n_aux != hl.n_aux || lay.Nq != hl.Nq || d->fs != h->fs || d->c != h->c ||
        d->grid_kind != h->grid_kind)
        return fail(SRP_ERR_INVALID_ARG, "descriptor is not the plan's");
    if (rd->n_offsets < 1 || rd->n_offsets > kMaxOffsets || rd->offsets == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "n_offsets must be in [1, 1024] with offsets given");
    if (!all_finite(rd->offsets, 3 * (size_t)rd->n_offsets))
        return fail(SRP_ERR_INVALID_ARG, "offsets not finite");
    if (rd->levels < 1 || rd->levels > kMaxLevels)
        return fail(SRP_ERR_INVALID_ARG, "levels must be in [1, 64]");
    if (!(rd->shrink > 0.0 && rd->shrink <= 1.0))
        return fail(SRP_ERR_INVALID_ARG, "shrink must be in (0, 1]");
    if (rd->keep_grid != 0 && rd->keep_grid != 1)
        return fail(SRP_ERR_INVALID_ARG, "keep_grid must be 0 or 1");
    if (rd->keep_grid && !all_finite(d->grid_xyz, 3 * (size_t)d->J))
        return fail(SRP_ERR_INVALID_ARG, "grid_xyz not finite");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    srp_refiner_s *r = new (std::nothrow) srp_refiner_s();
    if (r == nullptr) return fail(SRP_ERR_OOM, "host allocation failed");
    r->plan = h;
    r->device = h->device;
    r->F = rd->n_offsets;
    r->levels = rd->levels;
    r->shrink = rd->shrink;
    auto bail = [&](srp_status s) {
        refiner_release(r);
        delete r;
        return s;
    };
    // microphones relative to their centroid, in FP32
    std::vector<float> micf(3 * (size_t)d->M);
    for (int k = 0; k < 3; ++k) {
        double c = 0.0;
        for (int m = 0; m < d->M; ++m) c += d->mic_xyz[3 * m + k];
        r->centroid[k] = c / d->M;
    }
    for (int m = 0; m < d->M; ++m)
        for (int k = 0; k < 3; ++k)
            micf[3 * m + k] = (float)(d->mic_xyz[3 * m + k] - r->centroid[k]);
    // per-pair stride of the staged samples: the longest pair, made odd
    int span = 1;
    for (int32_t v : hl.Nq) span = std::max(span, 2 * (v + hl.n_aux) + 1);
    r->pstride = span | 1;
    const size_t base = sizeof(float) * (3 * (size_t)hl.M + (size_t)r->F);
    const size_t staged = base + sizeof(float) * (size_t)hl.Q * r->pstride;
    r->staged = staged <= kRefineSmemMax;
    r->smem = r->staged ? staged : base;
    if (r->smem > 48 * 1024) {
        cudaError_t e = r->staged
            ? cudaFuncSetAttribute(k_refine<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)r->smem)
            : cudaFuncSetAttribute(k_refine<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)r->smem);
        if (e != cudaSuccess) return bail(cuda_fail(e, "refinement kernel attribute"));
    }
    const size_t b_mic = sizeof(float) * 3 * (size_t)d->M;
    const size_t b_off = sizeof(double) * 3 * (size_t)r->F;
    const size_t b_grid = rd->keep_grid ? sizeof(double) * 3 * (size_t)d->J : 0;
    cudaError_t e;
    if ((e = cudaMalloc(&r->d_mic, b_mic)) != cudaSuccess ||
        (e = cudaMalloc(&r->d_offsets, b_off)) != cudaSuccess ||
        (b_grid && (e = cudaMalloc(&r->d_grid, b_grid)) != cudaSuccess))
        return bail(e == cudaErrorMemoryAllocation ? fail(SRP_ERR_OOM, "refiner buffers")
                                                   : cuda_fail(e, "cudaMalloc"));
    if ((e = cudaMemcpy(r->d_mic, micf.data(), b_mic, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(r->d_offsets, rd->offsets, b_off, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (b_grid && (e = cudaMemcpy(r->d_grid, d->grid_xyz, b_grid, cudaMemcpyHostToDevice)) !=
                       cudaSuccess))
        return bail(cuda_fail(e, "upload refiner tables"));
    *out = r;
    return SRP_OK;
}

srp_status srp_refine(srp_refiner r, int32_t L, const int32_t *d_argmax, const double *d_centres,
                      double *d_best_xyz, float *d_best_val, float *d_values, srp_stream_t s) {
    if (r == nullptr) return fail(SRP_ERR_INVALID_ARG, "refiner is NULL");
    srp_plan_s *h = r->plan;
    if (L < 0) return fail(SRP_ERR_INVALID_ARG, "L must be >= 0");
    if (L == 0) return SRP_OK;
    if (L > h->last_L)
        return fail(SRP_ERR_INVALID_ARG, "L exceeds the frames of the plan's last srp_map");
    if ((d_argmax == nullptr) == (d_centres == nullptr))
        return fail(SRP_ERR_INVALID_ARG, "give exactly one of d_argmax and d_centres");
    if (d_argmax != nullptr && r->d_grid == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "centre indices need a refiner built with keep_grid");
    if (d_best_xyz == nullptr || d_best_val == nullptr)
        return fail(SRP_ERR_INVALID_ARG, "d_best_xyz and d_best_val must be non-NULL");
    DeviceGuard g(r->device);
    if (!g.ok) return fail(SRP_ERR_CUDA, "cannot select the plan's device");
    const Layout &lay = h->lay;
    RefineArgs a;
    memset(&a, 0, sizeof a);
    a.mic = r->d_mic;
    a.pairs = h->d_pairs;
    a.nq = h->d_nq;
    a.M = lay.M;
    a.Q = lay.Q;
    a.n_aux = lay.n_aux;
    a.fs_c = (float)(h->fs / h->c);
    a.far = h->grid_kind == SRP_GRID_DIRECTIONS;
    if (lay.tc) {
        a.src = h->precision == SRP_PREC_FP32 ? kXiSplit
                                              : (h->precision == SRP_PREC_FP16 ? kXiF16 : kXiBf16);
        a.off = h->d_offc;
        a.xi16 = h->d_xi16;
        a.ld = lay.Sc;
        a.lo_off = (int64_t)lay.L_pad * lay.Sc;
    } else {
        a.src = kXiF32;
        a.off = h->d_off;
        a.xi = h->d_xi;
        a.ld = lay.L_pad;
    }
    a.pstride = r->pstride;
    a.cx = r->centroid[0];
    a.cy = r->centroid[1];
    a.cz = r->centroid[2];
    a.offsets = r->d_offsets;
    a.F = r->F;
    a.levels = r->levels;
    a.shrink = r->shrink;
    a.grid = r->d_grid;
    a.J = lay.J;
    a.argmax = d_argmax;
    a.centres = d_centres;
    a.best_xyz = d_best_xyz;
    a.best_val = d_best_val;
    a.values = d_values;
    a.status = h->d_status;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)L * kCluster);
    cfg.blockDim = dim3(kRefineThreads);
    cfg.dynamicSmemBytes = r->smem;
    cfg.stream = reinterpret_cast<cudaStream_t>(s);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SRP_CUDA(r->staged ? cudaLaunchKernelEx(&cfg, k_refine<true>, a)
                       : cudaLaunchKernelEx(&cfg, k_refine<false>, a),
             "refinement kernel");
    return SRP_OK;
}

srp_status srp_refiner_destroy(srp_refiner r) {
    if (r == nullptr) return SRP_OK;
    DeviceGuard g(r->device);
    refiner_release(r);
    delete r;
    return SRP_OK;
}

}  // extern "C"
