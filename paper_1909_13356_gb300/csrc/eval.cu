// eval.cu -- Phi and grad Phi at Morton-sorted targets (Sec. 4.4).
//
// The sum over source nodes is split by tile (eq. kerdecomp): a source tile
// whose bounding box lies farther than cutoff * sigma_max(tile) from the
// bounding box of a block of targets contributes through the Laplace double
// layer (eq. kerapprox); every other tile contributes through the full
// smoothed kernel (eq. kerpsi, and its gradient from eq. gradPhi with the
// sign of the second term corrected).  Nothing is dropped: a near tile
// evaluates the full kernel for all of its pairs.
//
// With nw' = nw / (4 pi), a = 1/(sqrt2 sigma), r = y - x, u = |r| a, w = u^2:
//   phi  += (nw'.r) a^3 H(w)
//   grad -= nw' a^3 H(w) + (nw'.r) a^5 K r,    K = H'(u)/u = 2 dH/dw
//   H = g(u)/u^3, g(u) = erf(u) - (2u/sqrt pi) e^{-u^2};
// the Laplace limits are a^3 H -> 1/|r|^3 and a^5 K -> -3/|r|^5.  The FP64
// kernel evaluates H and K from their power series (small u, eq.
// kerpsi_asymp completed with the term eq. kerpsi_asymp2 drops) or the
// erf form; the FP32 and float-float kernels read H from a piecewise
// polynomial table fitted at context creation.
//
// Three kernels share one layout.  A CTA owns a block of consecutive sorted
// targets and walks a range of source tiles; each tile is staged into shared
// memory by the bulk-copy engine (cp.async.bulk, completion on an mbarrier
// with a bounded wait), double buffered.  A grid y-dimension splits the tile
// range when there are too few target blocks to fill the GPU (partials are
// reduced in a fixed order), or a table of work items (target range, tile
// range) drives the grid for batches of meshes.
//   k_eval_fp64   the FP64 reference path.
//   k_eval_mixed  far tiles in FP32 on tile-local coordinates (two targets
//                 per thread in packed f32x2 lanes), near tiles in
//                 float-float; compensated, per-tile renormalised sums.
//   k_eval_ff     Phi to FP64 accuracy on the FP32 pipes: every far and near
//                 pair in float-float; grad Phi to mixed accuracy.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <type_traits>

#include "lsm_internal.cuh"
#include "ff.cuh"

#ifndef LSM_RSQRT_REFINE
#define LSM_RSQRT_REFINE 1
#endif
// near tiles: sources beyond the cutoff from the whole target box take the
// Laplace pair.  On in the mixed kernel (its near pair costs about five far
// pairs: -7% on the torus bench step's mixed launches); off in the float-float
// kernel, where the two pairs cost nearly the same and the tile's
// classification cost more than it saved (+1.7% per launch).
#ifndef LSM_REACH_SPLIT_FF
#define LSM_REACH_SPLIT_FF 0
#endif
#ifndef LSM_REACH_SPLIT_MIXED
#define LSM_REACH_SPLIT_MIXED 1
#endif
// unrolling of the mixed kernel's packed far loop (pairs of sources per step;
// 4 measured no faster and drops the 64-target layout to 4 CTAs per SM)
#ifndef LSM_MIXED_UNROLL
#define LSM_MIXED_UNROLL 2
#endif
#ifndef LSM_PACKED_F32X2
#define LSM_PACKED_F32X2 1
#endif

namespace lsm {
namespace {

constexpr int kSer64 = 14;  // series terms, FP64, used for u^2 < 0.25
constexpr double kUs64 = 0.25;
constexpr double kTwoOverSqrtPi = 1.12837916709551257390;
constexpr double kFourOverSqrtPi = 2.25675833419102514780;

// Hs(u) = sum_m A_m w^m, Ks(u) = sum_m B_m w^m, w = u^2 (filled by the host)
__constant__ double c_A64[kSer64];
__constant__ double c_B64[kSer64];

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared; `bytes` and both addresses are multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each poll may suspend the
// thread for a hardware-defined time slice).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
constexpr int kWaitLimit = 1 << 22;
constexpr int kTestWaitLimit = 1 << 10;   // the test hook's short limit (nothing is in flight then)
constexpr double kSqrt2 = 1.41421356237309505;
// 1 / (2 sqrt2 pi^(3/2)): dPhi/dsigma = -(4 a^4 / (2 sqrt2 pi^(3/2))) sum (nw' . r) e^{-u^2} 4 pi
// with nw' = nw / 4 pi and sigma = 1 / (sqrt2 a), i.e. -16 pi a^4 kSigC sum (nw' . r) e^{-w}
constexpr double kSigC = 0.063493635934240970;
constexpr double kFourPiD = 12.566370614359172954;
constexpr int kChunk = 64;  // far-tile sources summed in FP32 before compensation
constexpr int kMixedUnroll = LSM_MIXED_UNROLL;
constexpr int kErrWaitTimeout = 1;

// ---------------------------------------------------------------- radial factors
__device__ __forceinline__ void radial64(double r2, double a, double sqrt2sig, double& fH, double& FK)
{
    const double w = r2 * a * a;
    double H, K;
    if (w < kUs64) {
        H = c_A64[kSer64 - 1];
        K = c_B64[kSer64 - 1];
#pragma unroll
        for (int m = kSer64 - 2; m >= 0; m--) {
            H = fma(H, w, c_A64[m]);
            K = fma(K, w, c_B64[m]);
        }
    } else {
        const double rinv = rsqrt(r2);
        const double u = r2 * rinv * a;
        const double e = exp(-w);
        const double g = erf(u) - kTwoOverSqrtPi * u * e;
        const double ui = rinv * sqrt2sig;
        const double ui2 = ui * ui;
        H = g * ui2 * ui;
        K = ui2 * (kFourOverSqrtPi * e - 3.0 * H);
    }
    const double a3 = a * a * a;
    fH = a3 * H;
    FK = a3 * a * a * K;
}

// One Newton step on the hardware estimate: the result is within about one
// ulp and carries no systematic bias.
__device__ __forceinline__ float rsqrt_refined(float r2)
{
    // one Newton step on the hardware estimate: the result is within about
    // one ulp and carries no systematic bias
    const float r = rsqrtf(r2);
#if LSM_RSQRT_REFINE
    const float t = r2 * r;
    const float e = fmaf(-t, r, 1.0f);
    return fmaf(0.5f * r, e, r);
#else
    return r;
#endif
}


// Piecewise polynomial table of H(w) = g(u)/u^3, w = u^2 (see build_h_table):
// interval k covers w in [k, k+1)/kHTabPerUnit; per interval three float4:
// {c0h, c0l, c1h, c1l}, {c2h, c2l, c3h, c3l}, {c4h, c4l, c5, c6}, p(t) =
// sum c_j t^j, t = w - centre.  Beyond kHTabWmax, H = 1/u^3 to 1e-14.
constexpr int kHTabPerUnit = 16;
constexpr int kHTabN = 520;                   // covers w < 32.5 (u < 5.70)
constexpr float kHTabWmax = (float)kHTabN / kHTabPerUnit;
__device__ float4 g_htab[kHTabN * 3];         // filled once per device by the host


// Block-wide min/max of three floats each, result in shared s[0..6).
__device__ __forceinline__ void block_bbox(float lo[3], float hi[3], float* s)
{
    __shared__ float part[6][kEvalThreads / 32];
    for (int c = 0; c < 3; c++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; c++) {
            part[c][w] = lo[c];
            part[3 + c][w] = hi[c];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++) {
            float L = part[c][0], H = part[3 + c][0];
            for (int k = 1; k < kEvalThreads / 32; k++) {
                L = fminf(L, part[c][k]);
                H = fmaxf(H, part[3 + c][k]);
            }
            s[c] = L;
            s[3 + c] = H;
        }
    }
    __syncthreads();
}

// Block-wide max of one float, result in *dst (shared); all threads call.
__device__ __forceinline__ void block_max1(float v, float* dst)
{
    __shared__ float part[kEvalThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = part[0];
        for (int k = 1; k < kEvalThreads / 32; k++) m = fmaxf(m, part[k]);
        *dst = m;
    }
    __syncthreads();
}

// The tile box with the near-field width replaced by the target block's
// largest sigma (sigma(x) mode).
__device__ __forceinline__ float4 with_sigma(float4 lo, float smax)
{
    return make_float4(lo.x, lo.y, lo.z, smax);
}

// True when every pair between the target block box and the source tile box
// is at least cutoff * sigma_max(tile) apart (conservative in FP32).
__device__ __forceinline__ bool tile_is_far(const float* bb, float4 lo, float4 hi, float cut2)
{
    const float gx = fmaxf(0.0f, fmaxf(lo.x - bb[3], bb[0] - hi.x));
    const float gy = fmaxf(0.0f, fmaxf(lo.y - bb[4], bb[1] - hi.y));
    const float gz = fmaxf(0.0f, fmaxf(lo.z - bb[5], bb[2] - hi.z));
    const float d2 = gx * gx + gy * gy + gz * gz;
    return d2 > cut2 * lo.w * lo.w * 1.0001f;
}

struct EvalArgs {
    // sigma(x) mode: the targets' sigma [nt] and grad sigma [3][nt] (sorted order)
    const double* tsig = nullptr;
    const double* tgsig = nullptr;
    const float4* tlo;
    const float4* thi;
    const float4* tchi;
    const float4* tclo;
    int ns, ntiles, tiles_per_split;
    const double* tx;  // SoA targets, component stride ld
    int64_t ld;
    int nt;
    float cut2;
    double* out;       // [split][4][nt] (phi, gx, gy, gz) when splitting, else [4][nt]
    int* flag;
    // bounded waits: polls before a stage counts as lost; test_nocopy != 0
    // (test hook) arms the first stage's barrier without issuing its copy,
    // so that the wait runs out with nothing in flight
    int wait_limit = 1 << 22;
    int test_nocopy = 0;
    const int4* items; // optional work items (first target, count, first tile, end tile)
    const int* n_items;
    // float-float kernel only: 0 plain; 1 record the far-tile part into
    // far_io ([split][4][nt] like out); 2 evaluate near tiles only, split 0
    // adding the recorded far part ([4][nt]) moved to x by its gradient
    // (x_old: SoA targets of the record call)
    int ff_mode;
    double* far_io;
    const double* x_old;
    float* bb_io = nullptr;   // [block][8]: block box recorded in mode 1, reused in mode 2
    unsigned long long* pairs;  // [2] pairs evaluated in near / far tiles
    // mixed kernel only: interaction lists of the treecode.  Block b walks the
    // tile ids list[blist[b].x .. + blist[b].y); ids >= ntiles are proxy
    // tiles (positions ppos, weights pnw; always far).  tlo .. tclo then
    // cover source and proxy tiles.
    const int* list = nullptr;
    const int2* blist = nullptr;
    const int* border = nullptr;     // list mode: block of each CTA row (longest lists first)
    const float4* ppos = nullptr;
    const float4* pnw = nullptr;
    const float4* plo = nullptr;     // float-float kernel: proxy remainders
    const float4* pnwlo = nullptr;
};

// Block-wide sums of the pair counts, added once per CTA.
__device__ __forceinline__ void count_pairs(unsigned long long* dst, unsigned long long n, unsigned long long f)
{
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        f += __shfl_xor_sync(0xffffffffu, f, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n) atomicAdd(dst, n);
        if (f) atomicAdd(dst + 1, f);
    }
}

// A stage's copy did not complete within the wait limit: record the error in
// the device word and wait (bounded again) for the lost stage and, when
// `next` was issued, the prefetched next one, so that no bulk copy is
// still writing into shared memory when the CTA exits.  Called by thread 0.
__device__ __forceinline__ void give_up(const EvalArgs& A, uint64_t* bar, int b, int it, bool next)
{
    atomicOr(A.flag, kErrWaitTimeout);
    mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1), A.wait_limit);
    if (next) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1), A.wait_limit);
}
// Targets of a CTA that gave up get NaN results.
constexpr double kNaN = __builtin_nan("");



// One source's Phi term for one target in float-float: the tile-local pair
// difference r, |r|^2, the radial factor (far: 1/|r|^3 from the hardware
// rsqrt plus a float-float Newton step; near: a^3 H(w) from the table),
// nw . r and the product.  Also returns, rounded to FP32, the values the
// gradient uses (r, |r|^2, nw . r) and, for far pairs, the rsqrt estimate.
// FULL: the table's c0..c4 in float-float Horner steps (H to ~1e-15; the
// FP32 c3 t^3 term alone errs by 4e-12 of H near w = 1, |t| <= 1/32); else
// c0..c2 (the mixed path's near Phi, to ~1e-11 of H).
// Also returns the FP32 radial factors of the gradient, fH = a^3 H(w) and
// FK = a^5 K = 2 a^5 dH/dw, from the same table interval (or the Laplace
// limits beyond the table), so that the caller need not look them up again.
template <bool FULL>
__device__ __forceinline__ void ff_pair(const float4& y, const float4& n, const float4& yl, const float4& nl,
                                        const float* qh, const float* ql, bool far,
                                        const float4* __restrict__ tab, float& qhi, float& qlo, float& dxh,
                                        float& dyh, float& dzh, float& rh, float& dh, float& r0, float& gfH,
                                        float& gFK)
{
    float dxl, dyl, dzl, e;
    two_diff(y.x, qh[0], dxh, e);
    dxl = e + (yl.x - ql[0]);
    two_diff(y.y, qh[1], dyh, e);
    dyl = e + (yl.y - ql[1]);
    two_diff(y.z, qh[2], dzh, e);
    dzl = e + (yl.z - ql[2]);
    // |r|^2 as in ff_far_pair_grid: squares' errors, non-negative two-sums,
    // the cross terms summed in FP32
    const float p0 = dxh * dxh, p1 = dyh * dyh, p2 = dzh * dzh;
    const float e0 = fmaf(dxh, dxh, -p0), e1 = fmaf(dyh, dyh, -p1), e2 = fmaf(dzh, dzh, -p2);
    const float cr = fmaf(dxh, dxl, fmaf(dyh, dyl, dzh * dzl));
    float s01, t01, t2;
    two_sum_nonneg(p0, p1, s01, t01);
    two_sum_nonneg(s01, p2, rh, t2);
    const float rl = fmaf(2.0f, cr, ((e0 + e1) + e2) + (t01 + t2));
    float fHh, fHl;
    float wh = 0.0f, aah = 0.0f, aal = 0.0f;
    r0 = 0.0f;
    if (!far) {
        aah = y.w * y.w;
        aal = fmaf(y.w, y.w, -aah) + 2.0f * y.w * yl.w;
        wh = rh * aah;
    }
    if (!far && wh < kHTabWmax) {
        const float wl = fmaf(rh, aah, -wh) + fmaf(rh, aal, rl * aah);
        const int k = min((int)(wh * (float)kHTabPerUnit), kHTabN - 1);
        const float wc = ((float)k + 0.5f) * (1.0f / kHTabPerUnit);
        float th, te;
        two_diff(wh, wc, th, te);
        const float tl = te + wl;
        const float4 c01 = tab[3 * k], c23 = tab[3 * k + 1], c45 = tab[3 * k + 2];
        // tail in FP32, then float-float Horner steps
        float Hh, Hl, mh, ml;
        if (FULL) {
            const float q = fmaf(c45.w, th, c45.z);
            ff_mul(th, tl, q, 0.0f, mh, ml);
            ff_add(c45.x, c45.y, mh, ml, Hh, Hl);
            ff_mul(th, tl, Hh, Hl, mh, ml);
            ff_add(c23.z, c23.w, mh, ml, Hh, Hl);
            ff_mul(th, tl, Hh, Hl, mh, ml);
        } else {
            const float q = fmaf(fmaf(fmaf(c45.w, th, c45.z), th, c45.x), th, c23.z);
            ff_mul(th, tl, q, 0.0f, mh, ml);
        }
        ff_add(c23.x, c23.y, mh, ml, Hh, Hl);
        ff_mul(th, tl, Hh, Hl, mh, ml);
        ff_add(c01.z, c01.w, mh, ml, Hh, Hl);
        ff_mul(th, tl, Hh, Hl, mh, ml);
        ff_add(c01.x, c01.y, mh, ml, Hh, Hl);
        float a3h, a3l;
        ff_mul(aah, aal, y.w, yl.w, a3h, a3l);
        ff_mul(a3h, a3l, Hh, Hl, fHh, fHl);
        const float dH = fmaf(fmaf(fmaf(fmaf(fmaf(6.0f * c45.w, th, 5.0f * c45.z), th, 4.0f * c45.x), th,
                                        3.0f * c23.z), th, 2.0f * c23.x), th, c01.z);
        gfH = fHh;
        gFK = 2.0f * a3h * aah * dH;
    } else {
        // 1/|r| = r0 (1 - delta)^-1/2 = r0 (1 + delta/2 + 3 delta^2/8 + ...),
        // delta = 1 - |r|^2 r0^2 (~5e-7 from the hardware estimate); fH =
        // 1/|r|^3.  The delta^2 term is ~1e-13 of 1/|r| and of one sign for
        // every pair, so dropping it biases the whole far sum
        r0 = rsqrtf(rh);
        const float a = r0 * r0, ae = fmaf(r0, r0, -a);
        const float hh = rh * a;
        float he = fmaf(rh, a, -hh);
        he = fmaf(rh, ae, he);
        he = fmaf(rl, a, he);
        const float delta = (1.0f - hh) - he;
        const float ril = r0 * delta * fmaf(0.375f, delta, 0.5f);
        const float q2l = fmaf(2.0f * r0, ril, ae);
        fHh = a * r0;
        fHl = fmaf(a, r0, -fHh) + fmaf(a, ril, q2l * r0);
        gfH = fHh;
        gFK = -3.0f * fHh * a;
    }
    const float d0 = n.x * dxh, d1 = n.y * dyh, d2 = n.z * dzh;
    const float f0 = fmaf(n.x, dxh, -d0), f1 = fmaf(n.y, dyh, -d1), f2 = fmaf(n.z, dzh, -d2);
    float sd, u1, u2;
    two_sum(d0, d1, sd, u1);
    two_sum(sd, d2, dh, u2);
    const float dl = ((f0 + f1) + f2) + (u1 + u2) + fmaf(n.x, dxl, fmaf(n.y, dyl, n.z * dzl)) +
                     fmaf(nl.x, dxh, fmaf(nl.y, dyh, nl.z * dzh));
    ff_mul(dh, dl, fHh, fHl, qhi, qlo);
    // FP32 values for the gradient: the pair difference with its low part
    dxh += dxl;
    dyh += dyl;
    dzh += dzl;
    rh += rl;
    dh += dl;
}

// One source's far-tile Phi term for one target in float-float (the far
// branch of ff_pair, with fewer instructions): the tile-local pair
// difference r and |r|^2 as float pairs, then 1/|r|^3 from the hardware
// estimate r0 = rsqrt(|r|^2) and its relative defect
//   delta = 1 - |r|^2 r0^2 = (1 - t r0) - (t_err + |r|^2_lo r0) r0,
// with t + t_err = |r|^2_hi r0 exactly (an FMA), as
//   1/|r|^3 = r0^3 (1 - delta)^(-3/2) = r0^3 (1 + 3/2 delta + 15/8 delta^2),
// r0^3 a float pair (r0^2 is exact in two floats); the next term, 35/16
// delta^3 ~ 1e-20, is below float-float precision.  nw . r in float-float,
// and the product.  Returns for the gradient, in FP32, the high parts of r
// and nw . r, r0^2 and r0^3 (the gradient keeps mixed accuracy).
__device__ __forceinline__ void ff_far_pair(const float4& y, const float4& n, const float4& yl, const float4& nl,
                                            const float* qh, const float* ql, float& qhi, float& qlo, float& dxh,
                                            float& dyh, float& dzh, float& dh, float& ri2, float& ri3)
{
    float dxl, dyl, dzl, e;
    two_diff(y.x, qh[0], dxh, e);
    dxl = e + (yl.x - ql[0]);
    two_diff(y.y, qh[1], dyh, e);
    dyl = e + (yl.y - ql[1]);
    two_diff(y.z, qh[2], dzh, e);
    dzl = e + (yl.z - ql[2]);
    const float p0 = dxh * dxh, p1 = dyh * dyh, p2 = dzh * dzh;
    float e0 = fmaf(dxh, dxh, -p0), e1 = fmaf(dyh, dyh, -p1), e2 = fmaf(dzh, dzh, -p2);
    e0 = fmaf(2.0f * dxh, dxl, e0);
    e1 = fmaf(2.0f * dyh, dyl, e1);
    e2 = fmaf(2.0f * dzh, dzl, e2);
    float s01, t01, t2, rh;
    two_sum(p0, p1, s01, t01);
    two_sum(s01, p2, rh, t2);
    const float rl = ((e0 + e1) + e2) + (t01 + t2);
    const float r0 = rsqrtf(rh);
    const float t = rh * r0;
    const float te = fmaf(rh, r0, -t);
    const float u = fmaf(rl, r0, te);
    const float delta = fmaf(-u, r0, fmaf(-t, r0, 1.0f));
    const float a = r0 * r0, ae = fmaf(r0, r0, -a);
    const float fHh = a * r0;
    const float c3l = fmaf(ae, r0, fmaf(a, r0, -fHh));
    const float fHl = fmaf(fHh, delta * fmaf(1.875f, delta, 1.5f), c3l);
    const float d0 = n.x * dxh, d1 = n.y * dyh, d2 = n.z * dzh;
    const float f0 = fmaf(n.x, dxh, -d0), f1 = fmaf(n.y, dyh, -d1), f2 = fmaf(n.z, dzh, -d2);
    float sd, u1, u2;
    two_sum(d0, d1, sd, u1);
    two_sum(sd, d2, dh, u2);
    const float dl = fmaf(n.x, dxl, fmaf(n.y, dyl, fmaf(n.z, dzl, fmaf(nl.x, dxh, fmaf(nl.y, dyh,
                     fmaf(nl.z, dzh, ((f0 + f1) + f2) + (u1 + u2)))))));
    ff_mul(dh, dl, fHh, fHl, qhi, qlo);
    ri2 = a;
    ri3 = fHh;
}

// The far pair when the tile's source offsets and the target's offset have
// been re-split on a common grid (the high parts multiples of one power of two
// 2^k, all below 2^(k+23) in magnitude): the high parts' difference is then
// exact, and the low parts' difference is one addition.  The low part can then
// be as large as 2^(k-1), far above the high part's rounding unit when the
// pair is much closer than the grid's range, and the first-order steps below
// drop its square, so the pair is renormalised (a fast two-sum: the far pair's
// high part dominates).  Four operations per component instead of eight; the
// rest is ff_far_pair.
__device__ __forceinline__ void ff_far_pair_grid(const float4& y, const float4& n, const float4& yl,
                                                 const float4& nl, const float* qh, const float* ql, float& qhi,
                                                 float& qlo, float& dxh, float& dyh, float& dzh, float& dh,
                                                 float& ri2, float& ri3)
{
    float dxl, dyl, dzl;
    {
        const float hx = y.x - qh[0], hy = y.y - qh[1], hz = y.z - qh[2];
        const float lx = yl.x - ql[0], ly = yl.y - ql[1], lz = yl.z - ql[2];
        dxh = hx + lx;
        dyh = hy + ly;
        dzh = hz + lz;
        dxl = lx - (dxh - hx);
        dyl = ly - (dyh - hy);
        dzl = lz - (dzh - hz);
    }
    // |r|^2: the squares' rounding errors, their sum (non-negative terms),
    // and the cross terms 2 r_hi . r_lo summed in FP32 (2^-23 of |r|^2)
    const float p0 = dxh * dxh, p1 = dyh * dyh, p2 = dzh * dzh;
    const float e0 = fmaf(dxh, dxh, -p0), e1 = fmaf(dyh, dyh, -p1), e2 = fmaf(dzh, dzh, -p2);
    const float cr = fmaf(dxh, dxl, fmaf(dyh, dyl, dzh * dzl));
    float s01, t01, t2, rh;
    two_sum_nonneg(p0, p1, s01, t01);
    two_sum_nonneg(s01, p2, rh, t2);
    const float rl = fmaf(2.0f, cr, ((e0 + e1) + e2) + (t01 + t2));
    const float r0 = rsqrtf(rh);
    const float t = rh * r0;
    const float te = fmaf(rh, r0, -t);
    const float u = fmaf(rl, r0, te);
    const float delta = fmaf(-u, r0, fmaf(-t, r0, 1.0f));
    const float a = r0 * r0, ae = fmaf(r0, r0, -a);
    const float fHh = a * r0;
    const float c3l = fmaf(ae, r0, fmaf(a, r0, -fHh));
    const float fHl = fmaf(fHh, delta * fmaf(1.875f, delta, 1.5f), c3l);
    const float d0 = n.x * dxh, d1 = n.y * dyh, d2 = n.z * dzh;
    const float f0 = fmaf(n.x, dxh, -d0), f1 = fmaf(n.y, dyh, -d1), f2 = fmaf(n.z, dzh, -d2);
    float sd, u1, u2;
    two_sum(d0, d1, sd, u1);
    two_sum(sd, d2, dh, u2);
    const float dl = fmaf(n.x, dxl, fmaf(n.y, dyl, fmaf(n.z, dzl, fmaf(nl.x, dxh, fmaf(nl.y, dyh,
                     fmaf(nl.z, dzh, ((f0 + f1) + f2) + (u1 + u2)))))));
    ff_mul(dh, dl, fHh, fHl, qhi, qlo);
    ri2 = a;
    ri3 = fHh;
}

// Round v to a multiple of 2^k given c = 3 * 2^(k+22) and |v| < 2^(k+22):
// v + c lies in [2^(k+23), 2^(k+24)), where the float spacing is 2^k.
__device__ __forceinline__ float round_to_grid(float v, float c) { return (v + c) - c; }

// ---------------------------------------------------------------- mixed kernel
template <int TPT, bool SIGX, int SPL = 1>
__global__ void __launch_bounds__(kEvalThreads, 4) k_eval_mixed(const float4* __restrict__ spos,
                                                            const float4* __restrict__ snw,
                                                            const float4* __restrict__ slo,
                                                            const float4* __restrict__ snwlo, EvalArgs A)
{
    __shared__ __align__(128) float4 sh_pos[2][kTile];
    __shared__ __align__(128) float4 sh_nw[2][kTile];
    __shared__ __align__(128) float4 sh_lo[2][kTile];
    __shared__ __align__(128) float4 sh_nl[2][kTile];
    __shared__ __align__(16) float4 s_htab[kHTabN * 3];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float s_bb[6];
    __shared__ float s_smax;
    __shared__ unsigned char s_perm[kTile];   // near tile: its sources, those within reach of the block first
    __shared__ int s_cnt[2][kEvalThreads / 32];

    // SPL threads share each target (SPL 2: one target per pair of threads,
    // 64 per CTA), each taking its share of every tile's sources
    static_assert(SPL == 1 || (SPL == 2 && TPT == 1), "two threads per target with one target per thread");
    constexpr int TPB = kEvalThreads * TPT / SPL;
    const int tid = threadIdx.x;
    const int lane = SPL == 1 ? 0 : tid / TPB;
    const int tix = SPL == 1 ? tid : tid % TPB;   // the thread's target within its row of the block
    int base, tend, t0, t1;
    if (A.items) {
        if ((int)blockIdx.x >= *A.n_items) return;  // whole CTA, before any barrier
        const int4 w = A.items[blockIdx.x];
        base = w.x;
        tend = w.x + w.y;
        t0 = w.z;
        t1 = w.w;
    } else if (A.list) {
        // this split's part of the block's interaction list
        const int blk = A.border[blockIdx.x];
        base = blk * TPB;
        tend = A.nt;
        const int2 r = A.blist[blk];
        const int per = (r.y + (int)gridDim.y - 1) / (int)gridDim.y;
        t0 = min(r.x + (int)blockIdx.y * per, r.x + r.y);
        t1 = min(r.x + r.y, t0 + per);
    } else {
        base = blockIdx.x * TPB;
        tend = A.nt;
        t0 = blockIdx.y * A.tiles_per_split;
        t1 = min(A.ntiles, t0 + A.tiles_per_split);
    }

    for (int k = tid; k < kHTabN * 3; k += kEvalThreads) s_htab[k] = g_htab[k];
    float xh[TPT][3], xl[TPT][3];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int nvalid = 0;
#pragma unroll
    for (int k = 0; k < TPT; k++) {
        const int i = base + k * kEvalThreads + tix;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double v = i < tend ? A.tx[c * A.ld + i] : 0.0;
            xh[k][c] = __double2float_rn(v);
            xl[k][c] = __double2float_rn(v - (double)xh[k][c]);
            if (i < tend) {
                lo[c] = fminf(lo[c], __double2float_rd(v));
                hi[c] = fmaxf(hi[c], __double2float_ru(v));
            }
        }
        nvalid += i < tend && lane == 0 ? 1 : 0;   // pairs counted once per target
    }
    block_bbox(lo, hi, s_bb);
    // sigma(x) mode: each target's a = 1/(sqrt2 sigma(x)) as a float pair, and
    // the block's largest sigma for the near/far split
    float ta_h[TPT], ta_l[TPT], dsum_h[TPT], dsum_l[TPT];
#pragma unroll
    for (int k = 0; k < TPT; k++) ta_h[k] = ta_l[k] = dsum_h[k] = dsum_l[k] = 0.0f;
    if constexpr (SIGX) {
        float smax = 0.0f;
#pragma unroll
        for (int k = 0; k < TPT; k++) {
            const int i = base + k * kEvalThreads + tix;
            if (i < tend) {
                const double sg = A.tsig[i];
                const double a = 1.0 / (kSqrt2 * sg);
                ta_h[k] = (float)a;
                ta_l[k] = (float)(a - (double)ta_h[k]);
                smax = fmaxf(smax, __double2float_ru(sg));
            }
        }
        block_max1(smax, &s_smax);
    }

    float acc_h[TPT][4], acc_l[TPT][4];
#pragma unroll
    for (int k = 0; k < TPT; k++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc_h[k][c] = acc_l[k][c] = 0.0f;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // thread 0 stages a tile; the low parts of the positions only for near
    // tiles.  Proxy tiles (ids >= ntiles, list mode only) are always far.
    auto tile_at = [&](int j) { return A.list ? A.list[j] : j; };
    auto issue = [&](int t, int b, bool arm_only) {
        const int cnt = (int)A.thi[t].w;
        const uint32_t bytes = (uint32_t)cnt * 16u;
        const bool proxy = t >= A.ntiles;
        const bool far = proxy || tile_is_far(s_bb, SIGX ? with_sigma(A.tlo[t], s_smax) : A.tlo[t], A.thi[t], A.cut2);
        mbar_expect_tx(&bar[b], (far ? 2u : 4u) * bytes);
        if (arm_only) return;
        const float4* gp = proxy ? A.ppos + (size_t)(t - A.ntiles) * kTile : spos + (size_t)t * kTile;
        const float4* gn = proxy ? A.pnw + (size_t)(t - A.ntiles) * kTile : snw + (size_t)t * kTile;
        bulk_g2s(&sh_pos[b][0], gp, bytes, &bar[b]);
        bulk_g2s(&sh_nw[b][0], gn, bytes, &bar[b]);
        if (!far) {
            bulk_g2s(&sh_lo[b][0], slo + (size_t)t * kTile, bytes, &bar[b]);
            bulk_g2s(&sh_nl[b][0], snwlo + (size_t)t * kTile, bytes, &bar[b]);
        }
    };
    if (tid == 0 && t0 < t1) issue(tile_at(t0), 0, A.test_nocopy != 0);

    unsigned long long pairs_near = 0, pairs_far = 0;
    bool failed = false;
    for (int j = t0; j < t1; j++) {
        const int it = j - t0;
        const int b = it & 1;
        const int t = tile_at(j);
        const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1), A.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) give_up(A, bar, b, it, false);
            failed = true;
            break;
        }
        // past this barrier every thread has finished the previous tile, so
        // its stage (b ^ 1) takes the next tile's copy, which lands while this
        // tile is computed (one barrier per tile)
        if (tid == 0 && j + 1 < t1) issue(tile_at(j + 1), b ^ 1, false);
        const float4 tl = A.tlo[t], th = A.thi[t];
        const float4 ch = A.tchi[t], cl = A.tclo[t];
        const int cnt = (int)A.thi[t].w;
        const bool far = t >= A.ntiles || tile_is_far(s_bb, SIGX ? with_sigma(tl, s_smax) : tl, th, A.cut2);
        const float4* sp = sh_pos[b];
        const float4* sn = sh_nw[b];
        if (far) {
            pairs_far += (unsigned long long)cnt * nvalid;
            float xq[TPT][3];
#pragma unroll
            for (int k = 0; k < TPT; k++) {
                xq[k][0] = (xh[k][0] - ch.x) + (xl[k][0] - cl.x);
                xq[k][1] = (xh[k][1] - ch.y) + (xl[k][1] - cl.y);
                xq[k][2] = (xh[k][2] - ch.z) + (xl[k][2] - cl.z);
            }
            // FP32 sums over chunks of kChunk sources, each folded into the
            // float-float accumulator
#if LSM_PACKED_F32X2
            if constexpr (TPT == 2) {
                // the two targets of a thread ride in the two lanes of the packed
                // FP32 instructions (fma/add/mul.f32x2), halving the issue slots
                // of the pair arithmetic; x - y is carried (= -r)
                const float2 qx = make_float2(xq[0][0], xq[1][0]);
                const float2 qy = make_float2(xq[0][1], xq[1][1]);
                const float2 qz = make_float2(xq[0][2], xq[1][2]);
                const float2 one = make_float2(1.0f, 1.0f), half = make_float2(0.5f, 0.5f);
                const float2 p3 = make_float2(3.0f, 3.0f), m1 = make_float2(-1.0f, -1.0f);
                for (int c0 = 0; c0 < cnt; c0 += kChunk) {
                    const int c1 = min(cnt, c0 + kChunk);
                    float2 P0 = make_float2(0.0f, 0.0f), P1 = P0, P2 = P0, P3 = P0;
#pragma unroll 4
                    for (int s = c0; s < c1; s++) {
                        const float4 y = sp[s];
                        const float4 n = sn[s];
                        const float2 ndx = __fadd2_rn(qx, make_float2(-y.x, -y.x));
                        const float2 ndy = __fadd2_rn(qy, make_float2(-y.y, -y.y));
                        const float2 ndz = __fadd2_rn(qz, make_float2(-y.z, -y.z));
                        const float2 r2 = __ffma2_rn(ndx, ndx, __ffma2_rn(ndy, ndy, __fmul2_rn(ndz, ndz)));
                        float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
#if LSM_RSQRT_REFINE
                        const float2 t = __fmul2_rn(r2, ri);
                        const float2 e = __ffma2_rn(t, __fmul2_rn(ri, m1), one);
                        ri = __ffma2_rn(__fmul2_rn(ri, half), e, ri);
#endif
                        const float2 ri2 = __fmul2_rn(ri, ri);
                        const float2 ri3 = __fmul2_rn(ri2, ri);
                        const float2 nx = make_float2(n.x, n.x), ny = make_float2(n.y, n.y),
                                     nz = make_float2(n.z, n.z);
                        const float2 dneg = __ffma2_rn(nx, ndx, __ffma2_rn(ny, ndy, __fmul2_rn(nz, ndz)));
                        const float2 qn = __fmul2_rn(dneg, ri3);          // -(nw . r)/|r|^3
                        P0 = __fadd2_rn(P0, qn);                          // -Phi
                        // grad = 3 q r / |r|^5 - nw/|r|^3 = (3 qn/|r|^2) (x - y) - nw/|r|^3
                        const float2 tq = __fmul2_rn(qn, __fmul2_rn(ri2, p3));
                        const float2 mnx = make_float2(-n.x, -n.x), mny = make_float2(-n.y, -n.y),
                                     mnz = make_float2(-n.z, -n.z);
                        P1 = __ffma2_rn(tq, ndx, __ffma2_rn(mnx, ri3, P1));
                        P2 = __ffma2_rn(tq, ndy, __ffma2_rn(mny, ri3, P2));
                        P3 = __ffma2_rn(tq, ndz, __ffma2_rn(mnz, ri3, P3));
                    }
                    two_sum_acc(acc_h[0][0], acc_l[0][0], -P0.x);
                    two_sum_acc(acc_h[1][0], acc_l[1][0], -P0.y);
                    two_sum_acc(acc_h[0][1], acc_l[0][1], P1.x);
                    two_sum_acc(acc_h[1][1], acc_l[1][1], P1.y);
                    two_sum_acc(acc_h[0][2], acc_l[0][2], P2.x);
                    two_sum_acc(acc_h[1][2], acc_l[1][2], P2.y);
                    two_sum_acc(acc_h[0][3], acc_l[0][3], P3.x);
                    two_sum_acc(acc_h[1][3], acc_l[1][3], P3.y);
                }
            } else if constexpr (TPT == 1) {
                // one target per thread: two consecutive sources ride in the
                // two lanes (an odd tail pairs the last source with a zero
                // weight), and the lanes are added before each chunk's fold.
                // The tile is first rewritten pair-interleaved and negated into
                // this stage's low-part buffers (idle for a far tile): -y and
                // -nw, three planes of 128 floats each, so that every packed
                // operand is one 64-bit shared load with no lane assembly.
                float* tpos = reinterpret_cast<float*>(&sh_lo[b][0]);
                float* tnw = reinterpret_cast<float*>(&sh_nl[b][0]);
                if (tid < ((cnt + 1) & ~1)) {
                    const int s = min(tid, cnt - 1);
                    const float4 y = sp[s];
                    const float4 n = tid < cnt ? sn[s] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    tpos[tid] = -y.x;
                    tpos[kTile + tid] = -y.y;
                    tpos[2 * kTile + tid] = -y.z;
                    tnw[tid] = -n.x;
                    tnw[kTile + tid] = -n.y;
                    tnw[2 * kTile + tid] = -n.z;
                }
                __syncthreads();
                const float2* PX = reinterpret_cast<const float2*>(tpos);
                const float2* PY = PX + kTile / 2;
                const float2* PZ = PX + kTile;
                const float2* MX = reinterpret_cast<const float2*>(tnw);
                const float2* MY = MX + kTile / 2;
                const float2* MZ = MX + kTile;
                const float2 qx = make_float2(xq[0][0], xq[0][0]);
                const float2 qy = make_float2(xq[0][1], xq[0][1]);
                const float2 qz = make_float2(xq[0][2], xq[0][2]);
                const float2 one = make_float2(1.0f, 1.0f), half = make_float2(0.5f, 0.5f);
                const float2 p3 = make_float2(3.0f, 3.0f), m1 = make_float2(-1.0f, -1.0f);
                for (int c0 = 0; c0 < cnt; c0 += kChunk) {
                    const int c1 = min(cnt, c0 + kChunk);
                    // P0 = Phi; grad = P - R (P: -nw/|r|^3 terms, R: the 3 (nw . r) r/|r|^5 terms negated)
                    float2 P0 = make_float2(0.0f, 0.0f), P1 = P0, P2 = P0, P3 = P0, R1 = P0, R2 = P0, R3 = P0;
                    const int k0 = c0 >> 1, npair = (c1 - c0 + 1) >> 1;
#pragma unroll kMixedUnroll
                    for (int q = lane; q < npair; q += SPL) {
                        const int k = k0 + q;
                        const float2 mx = MX[k], my = MY[k], mz = MZ[k];
                        const float2 ndx = __fadd2_rn(qx, PX[k]);   // x - y
                        const float2 ndy = __fadd2_rn(qy, PY[k]);
                        const float2 ndz = __fadd2_rn(qz, PZ[k]);
                        const float2 r2 = __ffma2_rn(ndx, ndx, __ffma2_rn(ndy, ndy, __fmul2_rn(ndz, ndz)));
                        float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
#if LSM_RSQRT_REFINE
                        const float2 t = __fmul2_rn(r2, ri);
                        const float2 e = __ffma2_rn(t, __fmul2_rn(ri, m1), one);
                        ri = __ffma2_rn(__fmul2_rn(ri, half), e, ri);
#endif
                        const float2 ri2 = __fmul2_rn(ri, ri);
                        const float2 ri3 = __fmul2_rn(ri2, ri);
                        const float2 dn = __ffma2_rn(mx, ndx, __ffma2_rn(my, ndy, __fmul2_rn(mz, ndz)));   // nw . r
                        const float2 sv = __fmul2_rn(dn, ri3);            // (nw . r)/|r|^3
                        P0 = __fadd2_rn(P0, sv);
                        const float2 tq = __fmul2_rn(sv, __fmul2_rn(ri2, p3));
                        R1 = __ffma2_rn(tq, ndx, R1);
                        R2 = __ffma2_rn(tq, ndy, R2);
                        R3 = __ffma2_rn(tq, ndz, R3);
                        P1 = __ffma2_rn(mx, ri3, P1);
                        P2 = __ffma2_rn(my, ri3, P2);
                        P3 = __ffma2_rn(mz, ri3, P3);
                    }
                    two_sum_acc(acc_h[0][0], acc_l[0][0], P0.x + P0.y);
                    two_sum_acc(acc_h[0][1], acc_l[0][1], (P1.x + P1.y) - (R1.x + R1.y));
                    two_sum_acc(acc_h[0][2], acc_l[0][2], (P2.x + P2.y) - (R2.x + R2.y));
                    two_sum_acc(acc_h[0][3], acc_l[0][3], (P3.x + P3.y) - (R3.x + R3.y));
                }
            } else
#endif
            for (int c0 = 0; c0 < cnt; c0 += kChunk) {
                const int c1 = min(cnt, c0 + kChunk);
                float p[TPT][4];
#pragma unroll
                for (int k = 0; k < TPT; k++) p[k][0] = p[k][1] = p[k][2] = p[k][3] = 0.0f;
#pragma unroll 4
                for (int s = c0 + lane; s < c1; s += SPL) {
                    const float4 y = sp[s];
                    const float4 n = sn[s];
#pragma unroll
                    for (int k = 0; k < TPT; k++) {
                        const float dx = y.x - xq[k][0], dy = y.y - xq[k][1], dz = y.z - xq[k][2];
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const float ri = rsqrt_refined(r2);
                        const float ri2 = ri * ri;
                        const float ri3 = ri2 * ri;
                        const float d = fmaf(n.x, dx, fmaf(n.y, dy, n.z * dz));
                        const float q = d * ri3;
                        p[k][0] += q;
                        const float tq = 3.0f * q * ri2;
                        p[k][1] = fmaf(tq, dx, fmaf(-n.x, ri3, p[k][1]));
                        p[k][2] = fmaf(tq, dy, fmaf(-n.y, ri3, p[k][2]));
                        p[k][3] = fmaf(tq, dz, fmaf(-n.z, ri3, p[k][3]));
                    }
                }
#pragma unroll
                for (int k = 0; k < TPT; k++)
#pragma unroll
                    for (int c = 0; c < 4; c++) two_sum_acc(acc_h[k][c], acc_l[k][c], p[k][c]);
            }
        } else {
            // A near tile's sources beyond the cutoff from the whole target box
            // take the far field's Laplace pair (Sec. 4.4's split is by
            // distance).  Thread tid tests source tid (FP32 position against
            // the box, with a 1e-3 margin); s_perm lists the sources within
            // reach first, each group in source order.
            bool reach = !LSM_REACH_SPLIT_MIXED;
            if (LSM_REACH_SPLIT_MIXED && tid < cnt) {
                const float4 y = sp[tid];
                const float a = SIGX ? 0.70710678f / s_smax : y.w;
                const float px = ch.x + y.x, py = ch.y + y.y, pz = ch.z + y.z;
                const float gx = fmaxf(0.0f, fmaxf(s_bb[0] - px, px - s_bb[3]));
                const float gy = fmaxf(0.0f, fmaxf(s_bb[1] - py, py - s_bb[4]));
                const float gz = fmaxf(0.0f, fmaxf(s_bb[2] - pz, pz - s_bb[5]));
                reach = !((gx * gx + gy * gy + gz * gz) * (2.0f * a * a) > A.cut2 * 1.001f);
            }
            const int wl = tid & 31, wp = tid >> 5;
            const unsigned bn = __ballot_sync(0xffffffffu, tid < cnt && reach);
            const unsigned bf = __ballot_sync(0xffffffffu, tid < cnt && !reach);
            if (wl == 0) {
                s_cnt[0][wp] = __popc(bn);
                s_cnt[1][wp] = __popc(bf);
            }
            __syncthreads();
            int nn = 0, pn = 0, pf = 0;
#pragma unroll
            for (int w = 0; w < kEvalThreads / 32; w++) {
                nn += s_cnt[0][w];
                if (w < wp) {
                    pn += s_cnt[0][w];
                    pf += s_cnt[1][w];
                }
            }
            const unsigned below = (1u << wl) - 1u;
            if (tid < cnt) s_perm[reach ? pn + __popc(bn & below) : nn + pf + __popc(bf & below)] = (unsigned char)tid;
            __syncthreads();
            // pairs counted by the kernel they take
            pairs_near += (unsigned long long)nn * nvalid;
            pairs_far += (unsigned long long)(cnt - nn) * nvalid;
            // target offset from the tile centre as a float-float pair
            float qh[TPT][3], ql[TPT][3];
#pragma unroll
            for (int k = 0; k < TPT; k++) {
                const float cc[3] = {ch.x, ch.y, ch.z}, cc2[3] = {cl.x, cl.y, cl.z};
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float s0 = xh[k][c] - cc[c];
                    const float bb = s0 - xh[k][c];
                    const float e0 = (xh[k][c] - (s0 - bb)) + (-cc[c] - bb);
                    const float tt = (xl[k][c] - cc2[c]) + e0;
                    const float hh = s0 + tt;
                    qh[k][c] = hh;
                    ql[k][c] = tt - (hh - s0);
                }
            }
            const float4* sl = sh_lo[b];
            const float4* snl = sh_nl[b];
            // near pairs carry the large, often cancelling, terms: Phi in
            // float-float (as the float-float kernel), folded into the
            // accumulator pair by pair; the gradient in FP32 from the table
            float cph[TPT], cpl[TPT], cg[TPT][3], cgl[TPT][3];   // this tile's sums, float-float
#pragma unroll
            for (int k = 0; k < TPT; k++) {
                cph[k] = cpl[k] = 0.0f;
                for (int c = 0; c < 3; c++) cg[k][c] = cgl[k][c] = 0.0f;
            }
            float cd[TPT];   // sigma(x) mode: this tile's sum of (nw . r) e^{-w}
#pragma unroll
            for (int k = 0; k < TPT; k++) cd[k] = 0.0f;
#pragma unroll 1
            for (int k = lane; k < nn; k += SPL) {
                const int s = s_perm[k];
                const float4 y = sp[s];
                const float4 n = sn[s];
                const float4 yl = sl[s];
                const float4 nl = snl[s];
#pragma unroll
                for (int k = 0; k < TPT; k++) {
                    // the pair's a: the source's, or the target's in sigma(x) mode
                    const float4 ya = SIGX ? make_float4(y.x, y.y, y.z, ta_h[k]) : y;
                    const float4 yla = SIGX ? make_float4(yl.x, yl.y, yl.z, ta_l[k]) : yl;
                    float qh_, ql_, dxh, dyh, dzh, rh, dh, r0, fH, FK;
                    ff_pair<false>(ya, n, yla, nl, qh[k], ql[k], false, s_htab, qh_, ql_, dxh, dyh, dzh, rh, dh, r0,
                                   fH, FK);
                    float sph, tph;
                    two_sum(cph[k], qh_, sph, tph);
                    cph[k] = sph;
                    cpl[k] += tph + ql_;
                    const float tq = dh * FK;
                    two_sum_acc(cg[k][0], cgl[k][0], -fmaf(n.x, fH, tq * dxh));
                    two_sum_acc(cg[k][1], cgl[k][1], -fmaf(n.y, fH, tq * dyh));
                    two_sum_acc(cg[k][2], cgl[k][2], -fmaf(n.z, fH, tq * dzh));
                    if constexpr (SIGX) cd[k] = fmaf(dh, expf(-rh * ya.w * ya.w), cd[k]);
                }
            }
            // the rest with the Laplace pair in FP32 (tile-local coordinates,
            // the target offset's high part), folded into the same tile sums
#pragma unroll 2
            for (int k = nn + lane; k < cnt; k += SPL) {
                const int s = s_perm[k];
                const float4 y = sp[s];
                const float4 n = sn[s];
#pragma unroll
                for (int q = 0; q < TPT; q++) {
                    const float dx = y.x - qh[q][0], dy = y.y - qh[q][1], dz = y.z - qh[q][2];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float ri = rsqrt_refined(r2);
                    const float ri2 = ri * ri;
                    const float ri3 = ri2 * ri;
                    const float d = fmaf(n.x, dx, fmaf(n.y, dy, n.z * dz));
                    const float qv = d * ri3;
                    float sph, tph;
                    two_sum(cph[q], qv, sph, tph);
                    cph[q] = sph;
                    cpl[q] += tph;
                    const float tq = 3.0f * qv * ri2;
                    two_sum_acc(cg[q][0], cgl[q][0], fmaf(tq, dx, -n.x * ri3));
                    two_sum_acc(cg[q][1], cgl[q][1], fmaf(tq, dy, -n.y * ri3));
                    two_sum_acc(cg[q][2], cgl[q][2], fmaf(tq, dz, -n.z * ri3));
                }
            }
            if constexpr (SIGX) {
#pragma unroll
                for (int k = 0; k < TPT; k++) {
                    two_sum_acc(dsum_h[k], dsum_l[k], cd[k]);
                    renorm(dsum_h[k], dsum_l[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < TPT; k++) {
                float nh_, nl_;
                ff_add(acc_h[k][0], acc_l[k][0], cph[k], cpl[k], nh_, nl_);
                acc_h[k][0] = nh_;
                acc_l[k][0] = nl_;
                for (int c = 0; c < 3; c++) {
                    ff_add(acc_h[k][c + 1], acc_l[k][c + 1], cg[k][c], cgl[k][c], nh_, nl_);
                    acc_h[k][c + 1] = nh_;
                    acc_l[k][c + 1] = nl_;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < TPT; k++)
#pragma unroll
            for (int c = 0; c < 4; c++) renorm(acc_h[k][c], acc_l[k][c]);
    }
    if constexpr (SPL == 2) {
        // the second thread's sums join the first's, through the stage buffer
        // (idle once every thread is past the last tile: every copy has been
        // waited for unless a stage was lost)
        __syncthreads();
        if (!failed) {
            float* xch = reinterpret_cast<float*>(&sh_pos[0][0]);   // both stages: 1,024 floats
            if (lane == 1) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    xch[(2 * c) * TPB + tix] = acc_h[0][c];
                    xch[(2 * c + 1) * TPB + tix] = acc_l[0][c];
                }
                xch[8 * TPB + tix] = dsum_h[0];
                xch[9 * TPB + tix] = dsum_l[0];
            }
            __syncthreads();
            if (lane == 0) {
                float nh_, nl_;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    ff_add(acc_h[0][c], acc_l[0][c], xch[(2 * c) * TPB + tix], xch[(2 * c + 1) * TPB + tix], nh_, nl_);
                    acc_h[0][c] = nh_;
                    acc_l[0][c] = nl_;
                }
                ff_add(dsum_h[0], dsum_l[0], xch[8 * TPB + tix], xch[9 * TPB + tix], nh_, nl_);
                dsum_h[0] = nh_;
                dsum_l[0] = nl_;
            }
        }
    }
    const int64_t plane = (int64_t)A.nt;
    double* out = A.out + (int64_t)blockIdx.y * 4 * plane;
#pragma unroll
    for (int k = 0; k < TPT; k++) {
        const int i = base + k * kEvalThreads + tix;
        if (i < tend && lane == 0) {
            double r[4];
#pragma unroll
            for (int c = 0; c < 4; c++) r[c] = failed ? kNaN : (double)acc_h[k][c] + (double)acc_l[k][c];
            if constexpr (SIGX) {
                // grad Phi += (dPhi/dsigma) grad sigma (eq. gradPhi, third term)
                const double a = (double)ta_h[k] + (double)ta_l[k];
                const double a2 = a * a;
                const double dps = -4.0 * kFourPiD * kSigC * a2 * a2 * ((double)dsum_h[k] + (double)dsum_l[k]);
#pragma unroll
                for (int c = 0; c < 3; c++) r[c + 1] += dps * A.tgsig[c * plane + i];
            }
#pragma unroll
            for (int c = 0; c < 4; c++) out[c * plane + i] = r[c];
        }
    }
    count_pairs(A.pairs, pairs_near, pairs_far);
}

// ---------------------------------------------------------------- FP64 kernel
template <int TPT, bool SIGX>
__global__ void __launch_bounds__(kEvalThreads) k_eval_fp64(const double4_32a* __restrict__ spos,
                                                           const double4_32a* __restrict__ snw, EvalArgs A)
{
    __shared__ __align__(128) double4_32a sh_pos[2][kTile];
    __shared__ __align__(128) double4_32a sh_nw[2][kTile];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float s_bb[6];
    __shared__ float s_smax;

    const int tid = threadIdx.x;
    int base, tend, t0, t1;
    if (A.items) {
        if ((int)blockIdx.x >= *A.n_items) return;
        const int4 w = A.items[blockIdx.x];
        base = w.x;
        tend = w.x + w.y;
        t0 = w.z;
        t1 = w.w;
    } else {
        base = blockIdx.x * (kEvalThreads * TPT);
        tend = A.nt;
        t0 = blockIdx.y * A.tiles_per_split;
        t1 = min(A.ntiles, t0 + A.tiles_per_split);
    }

    double x[TPT][3];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int k = 0; k < TPT; k++) {
        const int i = base + k * kEvalThreads + tid;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double v = i < tend ? A.tx[c * A.ld + i] : 0.0;
            x[k][c] = v;
            if (i < tend) {
                lo[c] = fminf(lo[c], __double2float_rd(v));
                hi[c] = fmaxf(hi[c], __double2float_ru(v));
            }
        }
    }
    block_bbox(lo, hi, s_bb);
    // sigma(x) mode: each target's a = 1/(sqrt2 sigma(x)) and sqrt2 sigma(x)
    double ta[TPT], ts2[TPT], dsum[TPT], dsuml[TPT];
#pragma unroll
    for (int k = 0; k < TPT; k++) ta[k] = ts2[k] = dsum[k] = dsuml[k] = 0.0;
    if constexpr (SIGX) {
        float smax = 0.0f;
#pragma unroll
        for (int k = 0; k < TPT; k++) {
            const int i = base + k * kEvalThreads + tid;
            if (i < tend) {
                const double sg = A.tsig[i];
                ts2[k] = kSqrt2 * sg;
                ta[k] = 1.0 / ts2[k];
                smax = fmaxf(smax, __double2float_ru(sg));
            } else {
                ts2[k] = 1.0;
                ta[k] = 1.0;
            }
        }
        block_max1(smax, &s_smax);
    }

    double acc[TPT][4], accl[TPT][4];   // running sums, double-double
#pragma unroll
    for (int k = 0; k < TPT; k++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[k][c] = accl[k][c] = 0.0;
    int nvalid = 0;
#pragma unroll
    for (int k = 0; k < TPT; k++) nvalid += (base + k * kEvalThreads + tid) < tend ? 1 : 0;
    unsigned long long pairs_near = 0, pairs_far = 0;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t, int b, bool arm_only) {
        const int cnt = (int)A.thi[t].w;
        const uint32_t bytes = (uint32_t)cnt * 32u;
        mbar_expect_tx(&bar[b], 2u * bytes);
        if (arm_only) return;
        bulk_g2s(&sh_pos[b][0], spos + (size_t)t * kTile, bytes, &bar[b]);
        bulk_g2s(&sh_nw[b][0], snw + (size_t)t * kTile, bytes, &bar[b]);
    };
    if (tid == 0 && t0 < t1) issue(t0, 0, A.test_nocopy != 0);

    bool failed = false;
    for (int t = t0; t < t1; t++) {
        const int it = t - t0;
        const int b = it & 1;
        if (tid == 0 && t + 1 < t1) issue(t + 1, b ^ 1, false);
        const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1), A.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) give_up(A, bar, b, it, t + 1 < t1);
            failed = true;
            break;
        }
        const float4 tl = A.tlo[t], th = A.thi[t];
        const int cnt = (int)A.thi[t].w;
        const bool far = tile_is_far(s_bb, SIGX ? with_sigma(tl, s_smax) : tl, th, A.cut2);
        const double4_32a* sp = sh_pos[b];
        const double4_32a* sn = sh_nw[b];
        if (far) pairs_far += (unsigned long long)cnt * nvalid;
        else pairs_near += (unsigned long long)cnt * nvalid;
        double p[TPT][4];
#pragma unroll
        for (int k = 0; k < TPT; k++) p[k][0] = p[k][1] = p[k][2] = p[k][3] = 0.0;
        if (far) {
#pragma unroll 2
            for (int s = 0; s < cnt; s++) {
                const double4_32a y = sp[s];
                const double4_32a n = sn[s];
#pragma unroll
                for (int k = 0; k < TPT; k++) {
                    const double dx = y.x - x[k][0], dy = y.y - x[k][1], dz = y.z - x[k][2];
                    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    const double ri = rsqrt(r2);
                    const double ri2 = ri * ri;
                    const double ri3 = ri2 * ri;
                    const double d = fma(n.x, dx, fma(n.y, dy, n.z * dz));
                    const double q = d * ri3;
                    p[k][0] += q;
                    const double tq = 3.0 * q * ri2;
                    p[k][1] = fma(tq, dx, fma(-n.x, ri3, p[k][1]));
                    p[k][2] = fma(tq, dy, fma(-n.y, ri3, p[k][2]));
                    p[k][3] = fma(tq, dz, fma(-n.z, ri3, p[k][3]));
                }
            }
        } else {
            double pd[TPT];   // sigma(x) mode: this tile's sum of (nw . r) e^{-w}
#pragma unroll
            for (int k = 0; k < TPT; k++) pd[k] = 0.0;
            for (int s = 0; s < cnt; s++) {
                const double4_32a y = sp[s];
                const double4_32a n = sn[s];
#pragma unroll
                for (int k = 0; k < TPT; k++) {
                    const double dx = y.x - x[k][0], dy = y.y - x[k][1], dz = y.z - x[k][2];
                    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    double fH, FK;
                    // the pair's a and sqrt2 sigma: the source's, or the target's
                    radial64(r2, SIGX ? ta[k] : y.w, SIGX ? ts2[k] : n.w, fH, FK);
                    const double d = fma(n.x, dx, fma(n.y, dy, n.z * dz));
                    p[k][0] = fma(d, fH, p[k][0]);
                    const double tq = d * FK;
                    p[k][1] -= fma(n.x, fH, tq * dx);
                    p[k][2] -= fma(n.y, fH, tq * dy);
                    p[k][3] -= fma(n.z, fH, tq * dz);
                    if constexpr (SIGX) pd[k] = fma(d, exp(-r2 * ta[k] * ta[k]), pd[k]);
                }
            }
            if constexpr (SIGX) {
#pragma unroll
                for (int k = 0; k < TPT; k++) two_sum_acc64(dsum[k], dsuml[k], pd[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < TPT; k++)
#pragma unroll
            for (int c = 0; c < 4; c++) two_sum_acc64(acc[k][c], accl[k][c], p[k][c]);
        __syncthreads();
    }
    const int64_t plane = (int64_t)A.nt;
    double* out = A.out + (int64_t)blockIdx.y * 4 * plane;
#pragma unroll
    for (int k = 0; k < TPT; k++) {
        const int i = base + k * kEvalThreads + tid;
        if (i < tend) {
            double r[4];
#pragma unroll
            for (int c = 0; c < 4; c++) r[c] = failed ? kNaN : acc[k][c] + accl[k][c];
            if constexpr (SIGX) {
                // grad Phi += (dPhi/dsigma) grad sigma (eq. gradPhi, third term)
                const double a2 = ta[k] * ta[k];
                const double dps = -4.0 * kFourPiD * kSigC * a2 * a2 * (dsum[k] + dsuml[k]);
#pragma unroll
                for (int c = 0; c < 3; c++) r[c + 1] += dps * A.tgsig[c * plane + i];
            }
#pragma unroll
            for (int c = 0; c < 4; c++) out[c * plane + i] = r[c];
        }
    }
    count_pairs(A.pairs, pairs_near, pairs_far);
}

// ---------------------------------------------------------------- float-float kernel
// Phi to FP64 accuracy on the FP32 pipes.  Every quantity Phi depends on is
// carried as an unevaluated sum of two floats (about 44 significant bits):
// the tile-local pair difference r, |r|^2, 1/|r| (hardware estimate plus one
// Newton step evaluated in float-float), nw . r and their products.  Far
// tiles use the Laplace factor 1/|r|^3.  Near pairs use a^3 H(w), w = u^2,
// H = g(u)/u^3, read from a piecewise polynomial table (kHTabPerUnit
// intervals per unit of w up to kHTabWmax, degree 6 in the local variable,
// the five leading coefficients in float-float); beyond kHTabWmax H equals
// 1/u^3 to 1e-14.  grad Phi keeps mixed accuracy (FP32, compensated sums):
// it only steers Newton.
constexpr int kFFStage = kTile * 64;  // bytes per stage: 4 float4 arrays
constexpr int kMaxNearTiles = 768;    // near-tile list of one block (incremental mode)

template <bool SIGX, int TPB = kEvalThreads>
__global__ void __launch_bounds__(kEvalThreads) k_eval_ff(
    const float4* __restrict__ spos, const float4* __restrict__ snw, const float4* __restrict__ slo,
    const float4* __restrict__ snwlo, EvalArgs A)
{
    __shared__ __align__(128) unsigned char sh[2][kFFStage];
    __shared__ __align__(16) float4 s_htab[kHTabN * 3];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float s_bb[6];
    __shared__ int s_near[kMaxNearTiles];
    __shared__ int s_warp[kEvalThreads / 32];
    __shared__ int s_nnear;
    __shared__ float s_smax;
    __shared__ float4 s_dref[2][2];   // per stage: tile centre - block reference, float pair
    __shared__ unsigned char s_perm[kTile];   // near tile: its sources, those within reach of the block first
    __shared__ int s_cnt[2][kEvalThreads / 32];

    const int tid = threadIdx.x;
    int base, tend, t0, t1;
    if (A.items) {
        if ((int)blockIdx.x >= *A.n_items) return;
        const int4 w = A.items[blockIdx.x];
        base = w.x;
        tend = w.x + w.y;
        t0 = w.z;
        t1 = w.w;
    } else if (A.list) {
        // this split's part of the block's interaction list (modes 0 and 1)
        const int blk = A.border[blockIdx.x];
        base = blk * TPB;
        tend = A.nt;
        const int2 r = A.blist[blk];
        const int per = (r.y + (int)gridDim.y - 1) / (int)gridDim.y;
        t0 = min(r.x + (int)blockIdx.y * per, r.x + r.y);
        t1 = min(r.x + r.y, t0 + per);
    } else {
        base = blockIdx.x * TPB;
        tend = A.nt;
        t0 = blockIdx.y * A.tiles_per_split;
        t1 = min(A.ntiles, t0 + A.tiles_per_split);
    }
    // SPL threads share each target, each taking every SPL-th source of a tile
    constexpr int SPL = kEvalThreads / TPB;
    static_assert(SPL == 1 || SPL == 2, "64 or 128 targets per CTA");
    const int lane = SPL == 1 ? 0 : tid / TPB;
    const int i = base + (SPL == 1 ? tid : tid % TPB);
    const bool valid = i < tend;
    for (int k = tid; k < kHTabN * 3; k += kEvalThreads) s_htab[k] = g_htab[k];
    int mode = A.ff_mode;

    // the target relative to the block's first target, as a float pair: a
    // float pair of the absolute position would carry only ~48 bits of |x|,
    // an error that grad Phi (~1/sigma) turns into ~1e-13 of Phi
    double bref[3];
    float xh[3], xl[3];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        bref[c] = A.tx[c * A.ld + base];
        const double v = valid ? A.tx[c * A.ld + i] : bref[c];
        const double xb = v - bref[c];
        xh[c] = __double2float_rn(xb);
        xl[c] = __double2float_rn(xb - (double)xh[c]);
        if (valid) {
            lo[c] = __double2float_rd(v);
            hi[c] = __double2float_ru(v);
        }
    }
    block_bbox(lo, hi, s_bb);   // also orders the table fill before its first use
    // sigma(x) mode: the target's a = 1/(sqrt2 sigma(x)) as a float pair, and
    // the block's largest sigma for the near/far split
    float ta_h = 0.0f, ta_l = 0.0f, dsum_h = 0.0f, dsum_l = 0.0f;
    if constexpr (SIGX) {
        float smax = 0.0f;
        if (valid) {
            const double sg = A.tsig[i];
            const double a = 1.0 / (kSqrt2 * sg);
            ta_h = (float)a;
            ta_l = (float)(a - (double)ta_h);
            smax = __double2float_ru(sg);
        }
        block_max1(smax, &s_smax);
    }
    // incremental modes: the record call stores the block's box, the
    // near-only call reuses it (the same near/far split in both)
    if (A.bb_io && mode != 0) {
        // the block's own slot: list mode launches blocks in another order
        const int64_t bslot = A.list ? (int64_t)(base / TPB) : (int64_t)blockIdx.x;
        float* io = A.bb_io + 8 * bslot;
        if (tid == 0) {
            if (mode == 1) {
                for (int c = 0; c < 6; c++) io[c] = s_bb[c];
                io[6] = SIGX ? s_smax : 0.0f;
            } else {
                for (int c = 0; c < 6; c++) s_bb[c] = io[c];
                if (SIGX) s_smax = io[6];
            }
        }
        __syncthreads();
    }

    // incremental mode: the block's near tiles, in tile order
    int nlist = t1 - t0;
    bool scan = false;
    if (mode == 2) {
        if (tid == 0) s_nnear = 0;
        __syncthreads();
        const int lane = tid & 31, wp = tid >> 5;
        for (int tb = t0; tb < t1; tb += kEvalThreads) {
            const int t = tb + tid;
            const bool nr = t < t1 && !tile_is_far(s_bb, SIGX ? with_sigma(A.tlo[t], s_smax) : A.tlo[t], A.thi[t], A.cut2);
            const unsigned bal = __ballot_sync(0xffffffffu, nr);
            if (lane == 0) s_warp[wp] = __popc(bal);
            __syncthreads();
            int off = s_nnear;
            for (int k = 0; k < wp; k++) off += s_warp[k];
            off += __popc(bal & ((1u << lane) - 1u));
            if (nr && off < kMaxNearTiles) s_near[off] = t;
            __syncthreads();
            if (tid == 0) {
                int tot = 0;
                for (int k = 0; k < kEvalThreads / 32; k++) tot += s_warp[k];
                s_nnear += tot;
            }
            __syncthreads();
        }
        nlist = s_nnear;
        if (nlist > kMaxNearTiles) {   // too many to list: walk the whole range, skipping far tiles' pairs
            scan = true;
            nlist = t1 - t0;
        }
    }
    auto tile_at = [&](int k) {
        return mode == 2 && !scan ? s_near[k] : (A.list ? A.list[t0 + k] : t0 + k);
    };

    float ph = 0.0f, pl = 0.0f;                                     // near Phi, float-float
    float gh[3] = {0.0f, 0.0f, 0.0f}, gl[3] = {0.0f, 0.0f, 0.0f};   // near grad, compensated FP32
    float fph = 0.0f, fpl = 0.0f;                                   // far Phi
    float fgh[3] = {0.0f, 0.0f, 0.0f}, fgl[3] = {0.0f, 0.0f, 0.0f}; // far grad

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int t, int b, bool arm_only) {
        const int cnt = (int)A.thi[t].w;
        const uint32_t by = (uint32_t)cnt * 16u;
        // the tile's centre relative to the block reference, in FP64 (read
        // by every thread after the stage's barrier)
        const float4 ch = A.tchi[t], cl = A.tclo[t];
        const double d0 = ((double)ch.x - bref[0]) + (double)cl.x, d1 = ((double)ch.y - bref[1]) + (double)cl.y,
                     d2 = ((double)ch.z - bref[2]) + (double)cl.z;
        const float h0 = (float)d0, h1 = (float)d1, h2 = (float)d2;
        // far tiles re-split the offsets on a grid of spacing 2^k (see
        // ff_far_pair_grid): Q bounds every component of the targets' offsets
        // from the tile centre (block box) and of the tile's own offsets (tile
        // box), 2^(k+22) >= Q, and c = 3 * 2^(k+22)
        float Q = 0.0f;
        {
            const float4 tlo = A.tlo[t], thi = A.thi[t];
            const float cx[3] = {ch.x, ch.y, ch.z}, lo_t[3] = {tlo.x, tlo.y, tlo.z}, hi_t[3] = {thi.x, thi.y, thi.z};
#pragma unroll
            for (int c = 0; c < 3; c++) {
                Q = fmaxf(Q, fmaxf(fabsf(s_bb[c] - cx[c]), fabsf(s_bb[3 + c] - cx[c])));
                Q = fmaxf(Q, fmaxf(fabsf(lo_t[c] - cx[c]), fabsf(hi_t[c] - cx[c])));
            }
        }
        int ex;
        frexpf(fmaxf(Q * 1.0625f, 1e-30f), &ex);   // Q * 1.0625 < 2^ex
        s_dref[b][0] = make_float4(h0, h1, h2, ldexpf(3.0f, ex));
        s_dref[b][1] = make_float4((float)(d0 - (double)h0), (float)(d1 - (double)h1), (float)(d2 - (double)h2), 0.0f);
        mbar_expect_tx(&bar[b], 4u * by);
        if (arm_only) return;
        // proxy tiles (list mode, ids >= ntiles) come from the tree's arrays
        const bool proxy = t >= A.ntiles;
        const size_t o = (size_t)(proxy ? t - A.ntiles : t) * kTile;
        bulk_g2s(sh[b] + 0 * kTile * 16, (proxy ? A.ppos : spos) + o, by, &bar[b]);
        bulk_g2s(sh[b] + 1 * kTile * 16, (proxy ? A.pnw : snw) + o, by, &bar[b]);
        bulk_g2s(sh[b] + 2 * kTile * 16, (proxy ? A.plo : slo) + o, by, &bar[b]);
        bulk_g2s(sh[b] + 3 * kTile * 16, (proxy ? A.pnwlo : snwlo) + o, by, &bar[b]);
    };
    if (tid == 0 && nlist > 0) issue(tile_at(0), 0, A.test_nocopy != 0);

    unsigned long long pairs_near = 0, pairs_far = 0;
    bool failed = false;
    for (int it = 0; it < nlist; it++) {
        const int t = tile_at(it);
        const int b = it & 1;
        const bool ok = mbar_wait_bounded(&bar[b], (uint32_t)((it >> 1) & 1), A.wait_limit);
        const int cnt = (int)A.thi[t].w;
        const bool far =
            t >= A.ntiles || tile_is_far(s_bb, SIGX ? with_sigma(A.tlo[t], s_smax) : A.tlo[t], A.thi[t], A.cut2);
        if (ok && far && !scan && tid < cnt) {
            // this thread's source of a far tile, re-split on the tile's grid
            // (its copy has landed: the thread's own wait succeeded)
            float4* py = reinterpret_cast<float4*>(sh[b]);
            float4* pl = py + 2 * kTile;
            const float gc = s_dref[b][0].w;
            const float4 yh = py[tid], yl = pl[tid];
            const float hx = round_to_grid(yh.x, gc), hy = round_to_grid(yh.y, gc), hz = round_to_grid(yh.z, gc);
            py[tid] = make_float4(hx, hy, hz, yh.w);
            pl[tid] = make_float4((yh.x - hx) + yl.x, (yh.y - hy) + yl.y, (yh.z - hz) + yl.z, yl.w);
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) give_up(A, bar, b, it, false);
            failed = true;
            break;
        }
        // past this barrier every thread has finished the previous tile, so
        // its stage (b ^ 1) takes the next tile's copy, which lands while this
        // tile is computed (one barrier per tile)
        if (tid == 0 && it + 1 < nlist) issue(tile_at(it + 1), b ^ 1, false);
        if (scan && far) continue;   // near-only call walking its whole range: the far part is the recorded one
        if (far) pairs_far += valid && lane == 0 ? cnt : 0;
        const float4 ch = s_dref[b][0], cl = s_dref[b][1];
        const float cc[3] = {ch.x, ch.y, ch.z}, cc2[3] = {cl.x, cl.y, cl.z};
        float qh[3], ql[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float s0, e0;
            two_diff(xh[c], cc[c], s0, e0);
            const float tt = (xl[c] - cc2[c]) + e0;
            qh[c] = s0 + tt;
            ql[c] = tt - (qh[c] - s0);
            if (far) {   // the target's offset on the tile's grid, as the sources'
                const float h = round_to_grid(qh[c], ch.w);
                ql[c] = (qh[c] - h) + ql[c];
                qh[c] = h;
            }
        }
        const float4* sp = reinterpret_cast<const float4*>(sh[b]);
        const float4* sn = sp + kTile;
        const float4* sl = sp + 2 * kTile;
        const float4* snl = sp + 3 * kTile;
        // Pairs k0 .. k1 of the tile in chunks of kChunk (through s_perm when
        // PERM), with the smoothed kernel or the far field's Laplace kernel
        // (FAR), folded into the far sums or the near ones (TO_FAR).
        auto run = [&](int k0, int k1, auto far_c, auto perm_c, bool to_far) {
            constexpr bool FAR = decltype(far_c)::value;
            constexpr bool PERM = decltype(perm_c)::value;
            for (int c0 = k0; c0 < k1; c0 += kChunk) {
                const int c1 = min(k1, c0 + kChunk);
                float g[3] = {0.0f, 0.0f, 0.0f}, gn[3] = {0.0f, 0.0f, 0.0f};
                float cph = 0.0f, cpl = 0.0f;   // this chunk's Phi, float-float
                float cd = 0.0f;                // sigma(x) mode: sum of (nw . r) e^{-w}
#pragma unroll 4
                for (int k = c0 + lane; k < c1; k += SPL) {
                    const int s = PERM ? (int)s_perm[k] : k;
                    const float4 y0 = sp[s], n = sn[s], yl0 = sl[s], nl = snl[s];
                    // the pair's a: the source's, or the target's in sigma(x) mode
                    const float4 y = SIGX ? make_float4(y0.x, y0.y, y0.z, ta_h) : y0;
                    const float4 yl = SIGX ? make_float4(yl0.x, yl0.y, yl0.z, ta_l) : yl0;
                    float qh_, ql_, dxh, dyh, dzh, rh, dh;
                    if constexpr (FAR) {
                        float ri2, ri3;
                        // far tiles are on the grid; far sources of a near tile are not
                        if constexpr (PERM)
                            ff_far_pair(y, n, yl, nl, qh, ql, qh_, ql_, dxh, dyh, dzh, dh, ri2, ri3);
                        else
                            ff_far_pair_grid(y, n, yl, nl, qh, ql, qh_, ql_, dxh, dyh, dzh, dh, ri2, ri3);
                        float sph, tph;
                        two_sum(cph, qh_, sph, tph);
                        cph = sph;
                        cpl += tph + ql_;
                        // grad from the high parts (FP32)
                        const float tq = 3.0f * dh * ri3 * ri2;
                        g[0] = fmaf(tq, dxh, fmaf(-n.x, ri3, g[0]));
                        g[1] = fmaf(tq, dyh, fmaf(-n.y, ri3, g[1]));
                        g[2] = fmaf(tq, dzh, fmaf(-n.z, ri3, g[2]));
                    } else {
                        float r0, fH, FK;
                        ff_pair<true>(y, n, yl, nl, qh, ql, false, s_htab, qh_, ql_, dxh, dyh, dzh, rh, dh, r0, fH,
                                      FK);
                        float sph, tph;
                        two_sum(cph, qh_, sph, tph);
                        cph = sph;
                        cpl += tph + ql_;
                        const float tq = dh * FK;
                        two_sum_acc(g[0], gn[0], -fmaf(n.x, fH, tq * dxh));
                        two_sum_acc(g[1], gn[1], -fmaf(n.y, fH, tq * dyh));
                        two_sum_acc(g[2], gn[2], -fmaf(n.z, fH, tq * dzh));
                        if constexpr (SIGX) cd = fmaf(dh, expf(-rh * y.w * y.w), cd);
                    }
                }
                if constexpr (SIGX && !FAR) {
                    two_sum_acc(dsum_h, dsum_l, cd);
                    renorm(dsum_h, dsum_l);
                }
                // fold the chunk into the running float-float sums, renormalised
                float nh_, nl_;
                if (to_far) {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        two_sum_acc(fgh[c], fgl[c], g[c]);
                        renorm(fgh[c], fgl[c]);
                    }
                    ff_add(fph, fpl, cph, cpl, nh_, nl_);
                    fph = nh_;
                    fpl = nl_;
                } else {
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        float ah, al;
                        ff_add(gh[c], gl[c], g[c], gn[c], ah, al);
                        gh[c] = ah;
                        gl[c] = al;
                    }
                    ff_add(ph, pl, cph, cpl, nh_, nl_);
                    ph = nh_;
                    pl = nl_;
                }
            }
        };
        if (far) {
            run(0, cnt, std::true_type{}, std::false_type{}, true);
        } else if (!LSM_REACH_SPLIT_FF) {
            pairs_near += valid && lane == 0 ? cnt : 0;
            run(0, cnt, std::false_type{}, std::false_type{}, false);
        } else {
            // A near tile's sources beyond the cutoff from the whole target box
            // take the Laplace pair, as in a far tile (Sec. 4.4's split is by
            // distance); they stay in the near sums, which the near-only call
            // recomputes.  Thread tid tests source tid (FP32 position against
            // the box, with a 1e-3 margin), and s_perm lists the sources
            // within reach first, each group in source order.
            bool reach = false;
            if (tid < cnt) {
                const float4 y = sp[tid];
                const float a = SIGX ? 0.70710678f / s_smax : y.w;
                const float px = (float)bref[0] + (ch.x + y.x), py = (float)bref[1] + (ch.y + y.y),
                            pz = (float)bref[2] + (ch.z + y.z);
                const float gx = fmaxf(0.0f, fmaxf(s_bb[0] - px, px - s_bb[3]));
                const float gy = fmaxf(0.0f, fmaxf(s_bb[1] - py, py - s_bb[4]));
                const float gz = fmaxf(0.0f, fmaxf(s_bb[2] - pz, pz - s_bb[5]));
                reach = !((gx * gx + gy * gy + gz * gz) * (2.0f * a * a) > A.cut2 * 1.001f);
            }
            const int wl = tid & 31, wp = tid >> 5;
            const unsigned bn = __ballot_sync(0xffffffffu, tid < cnt && reach);
            const unsigned bf = __ballot_sync(0xffffffffu, tid < cnt && !reach);
            if (wl == 0) {
                s_cnt[0][wp] = __popc(bn);
                s_cnt[1][wp] = __popc(bf);
            }
            __syncthreads();
            int nn = 0, pn = 0, pf = 0;
#pragma unroll
            for (int w = 0; w < kEvalThreads / 32; w++) {
                nn += s_cnt[0][w];
                if (w < wp) {
                    pn += s_cnt[0][w];
                    pf += s_cnt[1][w];
                }
            }
            const unsigned below = (1u << wl) - 1u;
            if (tid < cnt) s_perm[reach ? pn + __popc(bn & below) : nn + pf + __popc(bf & below)] = (unsigned char)tid;
            __syncthreads();
            // pairs counted by the kernel they take
            pairs_near += valid && lane == 0 ? nn : 0;
            pairs_far += valid && lane == 0 ? cnt - nn : 0;
            run(0, nn, std::false_type{}, std::true_type{}, false);
            run(nn, cnt, std::true_type{}, std::true_type{}, false);
        }
    }
    if constexpr (SPL == 2) {
        // the second lane's partial sums join the first's, through the stage
        // buffers (idle once every thread is past the last tile: every copy
        // has been waited for unless a stage was lost)
        __syncthreads();
        if (!failed) {
            float* xch = reinterpret_cast<float*>(sh[0]);
            const int k = tid % TPB;
            if (lane == 1) {
                float v[18] = {ph, pl, fph, fpl, dsum_h, dsum_l};
                for (int c = 0; c < 3; c++) {
                    v[6 + c] = gh[c];
                    v[9 + c] = gl[c];
                    v[12 + c] = fgh[c];
                    v[15 + c] = fgl[c];
                }
#pragma unroll
                for (int q = 0; q < 18; q++) xch[q * TPB + k] = v[q];
            }
            __syncthreads();
            if (lane == 0) {
                float v[18];
#pragma unroll
                for (int q = 0; q < 18; q++) v[q] = xch[q * TPB + k];
                float nh_, nl_;
                ff_add(ph, pl, v[0], v[1], nh_, nl_);
                ph = nh_;
                pl = nl_;
                ff_add(fph, fpl, v[2], v[3], nh_, nl_);
                fph = nh_;
                fpl = nl_;
                ff_add(dsum_h, dsum_l, v[4], v[5], nh_, nl_);
                dsum_h = nh_;
                dsum_l = nl_;
                for (int c = 0; c < 3; c++) {
                    ff_add(gh[c], gl[c], v[6 + c], v[9 + c], nh_, nl_);
                    gh[c] = nh_;
                    gl[c] = nl_;
                    ff_add(fgh[c], fgl[c], v[12 + c], v[15 + c], nh_, nl_);
                    fgh[c] = nh_;
                    fgl[c] = nl_;
                }
            }
        }
    }
    if (valid && lane == 0) {
        const int64_t plane = (int64_t)A.nt;
        double* out = A.out + (int64_t)blockIdx.y * 4 * plane;
        double phi = (double)ph + (double)pl;
        double gr[3];
        for (int c = 0; c < 3; c++) gr[c] = (double)gh[c] + (double)gl[c];
        const double fphi = (double)fph + (double)fpl;
        double fgr[3];
        for (int c = 0; c < 3; c++) fgr[c] = (double)fgh[c] + (double)fgl[c];
        if (failed) {
            // a stage was lost: no partial sums leave the CTA
            phi = kNaN;
            for (int c = 0; c < 3; c++) gr[c] = kNaN;
        } else if (mode == 2) {
            // recorded far part, moved to x along its gradient (once, by split 0)
            if (blockIdx.y == 0) {
                double fp = A.far_io[i];
                for (int c = 0; c < 3; c++) {
                    const double g0 = A.far_io[(c + 1) * plane + i];
                    fp += g0 * (A.tx[c * A.ld + i] - A.x_old[c * A.ld + i]);
                    gr[c] += g0;
                }
                phi += fp;
            }
        } else {
            if (mode == 1) {
                double* fo = A.far_io + (int64_t)blockIdx.y * 4 * plane;
                fo[i] = fphi;
                for (int c = 0; c < 3; c++) fo[(c + 1) * plane + i] = fgr[c];
            }
            phi += fphi;
            for (int c = 0; c < 3; c++) gr[c] += fgr[c];
        }
        if constexpr (SIGX) {
            // grad Phi += (dPhi/dsigma) grad sigma (eq. gradPhi, third term)
            const double a = (double)ta_h + (double)ta_l;
            const double a2 = a * a;
            const double dps = -4.0 * kFourPiD * kSigC * a2 * a2 * ((double)dsum_h + (double)dsum_l);
            for (int c = 0; c < 3; c++) gr[c] += dps * A.tgsig[c * plane + i];
        }
        out[i] = phi;
        for (int c = 0; c < 3; c++) out[(c + 1) * plane + i] = gr[c];
    }
    count_pairs(A.pairs, pairs_near, pairs_far);
}

// Sum of the split partials in split order into res [4][nt].
__global__ void k_reduce_splits(const double* __restrict__ part, int nsplit, int nt, double* __restrict__ res)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < nsplit; k++)
        for (int c = 0; c < 4; c++) s[c] += part[((int64_t)k * 4 + c) * nt + i];
    for (int c = 0; c < 4; c++) res[(int64_t)c * nt + i] = s[c];
}

}  // namespace

// H(w) = g(u)/u^3, w = u^2, in long double: the power series for w < 1,
// the closed form with erfl/expl otherwise.
long double h_of_w(long double w)
{
    const long double tsp = 2.0L / sqrtl(3.14159265358979323846264338327950288L);
    if (w < 1.0L) {
        long double sum = 0.0L, fact = 1.0L, wp = 1.0L;
        for (int k = 1; k < 60; k++) {
            fact *= k;
            const long double ck = ((k & 1) ? 1.0L : -1.0L) * (2.0L * k) / (fact * (2.0L * k + 1.0L));
            const long double term = ck * wp;
            sum += term;
            if (fabsl(term) < 1e-30L) break;
            wp *= w;
        }
        return tsp * sum;
    }
    const long double u = sqrtl(w);
    const long double g = erfl(u) - tsp * u * expl(-w);
    return g / (u * u * u);
}

// Monomial coefficients (about the interval's centre) of the degree-6
// polynomial interpolating H at 7 Chebyshev points of interval k, which
// covers w in [k, k+1)/per_unit; long double throughout.
void h_interval_fit(int k, int per_unit, long double* cf)
{
    const int deg = 6;
    const long double h = 0.5L / per_unit;
    const long double wc = (k + 0.5L) / per_unit;
    long double V[7][8];
    for (int r = 0; r <= deg; r++) {
        const long double t = h * cosl(3.14159265358979323846264338327950288L * (r + 0.5L) / (deg + 1));
        long double tp = 1.0L;
        for (int j = 0; j <= deg; j++) {
            V[r][j] = tp;
            tp *= t;
        }
        V[r][deg + 1] = h_of_w(wc + t);
    }
    // Gaussian elimination with partial pivoting
    for (int c = 0; c <= deg; c++) {
        int piv = c;
        for (int r = c + 1; r <= deg; r++)
            if (fabsl(V[r][c]) > fabsl(V[piv][c])) piv = r;
        for (int j = 0; j <= deg + 1; j++) std::swap(V[c][j], V[piv][j]);
        for (int r = 0; r <= deg; r++) {
            if (r == c) continue;
            const long double f = V[r][c] / V[c][c];
            for (int j = c; j <= deg + 1; j++) V[r][j] -= f * V[c][j];
        }
    }
    for (int j = 0; j <= deg; j++) cf[j] = V[j][deg + 1] / V[j][j];
}

namespace {

// Piecewise polynomial table of H: interval k covers w in [k, k+1)/kHTabPerUnit,
// p(t) = sum_j c_j t^j with t = w - centre, interpolating H at 7 Chebyshev
// points (h_interval_fit).
// Layout per interval: {c0h, c0l, c1h, c1l}, {c2h, c2l, c3h, c3l}, {c4h, c4l, c5, c6}.
void build_h_table(float4* out)
{
    for (int k = 0; k < kHTabN; k++) {
        long double cf[7];
        h_interval_fit(k, kHTabPerUnit, cf);
        auto hi = [](long double v) { return (float)v; };
        auto lo = [](long double v) { return (float)(v - (long double)(float)v); };
        out[3 * k + 0] = make_float4(hi(cf[0]), lo(cf[0]), hi(cf[1]), lo(cf[1]));
        out[3 * k + 1] = make_float4(hi(cf[2]), lo(cf[2]), hi(cf[3]), lo(cf[3]));
        out[3 * k + 2] = make_float4(hi(cf[4]), lo(cf[4]), (float)cf[5], (float)cf[6]);
    }
}

bool g_consts_ready[64] = {false};

int upload_series_constants(Ctx* ctx)
{
    if (ctx->device >= 0 && ctx->device < 64 && g_consts_ready[ctx->device]) return LSM_OK;
    // c_k = (-1)^{k+1} 2k / (k! (2k+1)); Hs = (2/sqrt pi) sum_{k>=1} c_k w^{k-1},
    // Ks = (2/sqrt pi) sum_{k>=2} c_k (2k-2) w^{k-2}
    double A[kSer64 + 1], B[kSer64];
    double fact = 1.0;
    double c[kSer64 + 2];
    for (int k = 1; k <= kSer64 + 1; k++) {
        fact *= k;
        c[k] = ((k % 2) ? 1.0 : -1.0) * (2.0 * k) / (fact * (2.0 * k + 1.0));
    }
    for (int m = 0; m < kSer64; m++) {
        A[m] = kTwoOverSqrtPi * c[m + 1];
        B[m] = kTwoOverSqrtPi * c[m + 2] * (2.0 * (m + 2) - 2.0);
    }
    LSM_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_A64, A, sizeof(double) * kSer64));
    LSM_CUDA_TRY(ctx, cudaMemcpyToSymbol(c_B64, B, sizeof(double) * kSer64));
    {
        std::vector<float4> tab(kHTabN * 3);
        build_h_table(tab.data());
        LSM_CUDA_TRY(ctx, cudaMemcpyToSymbol(g_htab, tab.data(), sizeof(float4) * tab.size()));
    }
    // copies from pageable memory may return before they land, and nothing
    // orders them with kernels on the caller's (possibly non-blocking) stream
    LSM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (ctx->device >= 0 && ctx->device < 64) g_consts_ready[ctx->device] = true;
    return LSM_OK;
}

#ifndef LSM_TPT32
#define LSM_TPT32 2
#endif
constexpr int kTPT32 = LSM_TPT32;
constexpr int kTPT64 = 1;

}  // namespace

int eval_init_constants(Ctx* ctx) { return upload_series_constants(ctx); }

int mixed_tpb(const Ctx* ctx, const Mesh* me)
{
    const int t = ctx->opt.mixed_block > 0 ? ctx->opt.mixed_block : me->tune_tpb;
    // untuned: 64 targets per CTA (the autotuner's choice on the torus and the icosphere)
    return t == kEvalThreads || t == kEvalThreads * kTPT32 ? t : 64;
}
double mixed_cut(const Ctx* ctx, const Mesh* me) { return me->tune_cut > 0.0 ? me->tune_cut : ctx->opt.cutoff_mixed; }

// Phi and grad at n sorted targets (SoA x with stride ld) into res [4][n]
// (phi, then the three gradient components).
int eval_sorted(Ctx* ctx, const Mesh* me, const Targets& t, double* res, int precision, cudaStream_t st,
                const FFIncremental* inc)
{
    if (t.n <= 0) return LSM_OK;
    const bool newton = precision == kPrecMixedNewton;
    if (newton) precision = LSM_MIXED;
    const bool mixed = precision == LSM_MIXED;
    const bool ff = precision == LSM_FF;
    // targets per CTA: the mixed kernel's tuned layout (64, 128 or 256); the
    // float-float kernel's 64 (the option's default) or 128
    const bool ff64 = ff && ctx->opt.ff_block == 64;
    const int tpb = mixed ? mixed_tpb(ctx, me) : (ff64 ? 64 : kEvalThreads * kTPT64);
    const int nblk = (t.n + tpb - 1) / tpb;
    const int ntiles = (int)me->ntiles;
    // split the tile range so that the grid covers the GPU a few times over
    const int want = ctx->num_sms * 16;
    int nsplit = 1;
    if (nblk < want) nsplit = std::min((want + nblk - 1) / nblk, std::max(1, ntiles / 4));
    const int tps = (ntiles + nsplit - 1) / nsplit;
    nsplit = (ntiles + tps - 1) / tps;

    Scratch s(st);
    // sigma(x) mode: sigma and grad sigma of the sorted targets
    double *tsig = nullptr, *tgsig = nullptr;
    if (me->sigx) {
        LSM_CUDA_TRY(ctx, s.get(&tsig, (size_t)t.n));
        LSM_CUDA_TRY(ctx, s.get(&tgsig, 3 * (size_t)t.n));
        int rc = sigma_x_eval(ctx, me, t, tsig, tgsig, st, precision);
        if (rc != LSM_OK) return rc;
    }
    // mixed path on a large mesh: the treecode's interaction lists
    int* list = nullptr;
    int2* blist = nullptr;
    int* border = nullptr;
    // float-float: every mode but the near-only one (which lists near tiles itself)
    const bool use_tree = mixed ? tree_wanted(ctx, me, false)
                                : (ff && !(inc && inc->mode == 2) && tree_wanted(ctx, me, true));
    // treecodes: target clusters take the nodes far from them (tpc a multiple of the block)
    ClusterPlan cp;
    const int tpc = (ff ? ctx->opt.tree_ff_cluster : ctx->opt.tree_cluster) / tpb * tpb;
    const bool clusters = use_tree && (ff || mixed) && tpc > 0 && t.n >= 2 * tpc;
    // the mixed Newton sweeps' coarser treecode and near-field radius
    const bool ntree = use_tree && newton && newton_tree_wanted(ctx, me);
    const double mcut = newton ? std::min(mixed_cut(ctx, me), (double)ctx->opt.newton_cutoff) : mixed_cut(ctx, me);
    const Tree* TT = nullptr;
    if (use_tree) {
        int rc = tree_ensure(ctx, const_cast<Mesh*>(me), st, ff, ntree);
        if (rc != LSM_OK) return rc;
        TT = ff ? me->tree_ff : (ntree ? me->tree_newton : me->tree);
        if (clusters) {
            rc = cluster_setup(ctx, TT, t, tpc, tpb, ff ? ctx->opt.cutoff_fp64 : mcut, tsig, s, &cp, st);
            if (rc != LSM_OK) return rc;
        }
        int64_t total = 0;
        rc = tree_lists(ctx, TT, t, tpb, tsig, s, &list, &blist, &border, &total, st,
                        mixed ? mcut : 0.0, clusters ? &cp : nullptr);
        if (rc != LSM_OK) return rc;
        const int64_t avg = total / nblk;
        nsplit = 1;
        if (nblk < want) nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((want + nblk - 1) / nblk, avg / 4));
    }
    double* part = res;
    if (nsplit > 1) LSM_CUDA_TRY(ctx, s.get(&part, (size_t)nsplit * 4 * t.n));
    // a split record call keeps one far part per split, summed like the results
    const bool split_far = ff && inc && inc->mode == 1 && nsplit > 1;
    double* far_part = nullptr;
    if (split_far) LSM_CUDA_TRY(ctx, s.get(&far_part, (size_t)nsplit * 4 * t.n));
    EvalArgs A;
    A.tlo = me->tile_lo;
    A.thi = me->tile_hi;
    A.tchi = me->tile_chi;
    A.tclo = me->tile_clo;
    A.ns = (int)me->ns;
    A.ntiles = ntiles;
    A.tiles_per_split = tps;
    A.tx = t.x;
    A.ld = t.ld;
    A.nt = t.n;
    const double cut = mixed ? mcut : ctx->opt.cutoff_fp64;
    A.cut2 = (float)(cut * cut);
    A.out = part;
    A.flag = flag_word(ctx);
    A.test_nocopy = ctx->test_nocopy ? 1 : 0;
    A.wait_limit = ctx->test_nocopy ? kTestWaitLimit : kWaitLimit;
    A.pairs = ctx->d_pairs + 2 * (mixed ? 0 : (precision == LSM_FF ? 1 : 2));
    A.items = nullptr;
    A.n_items = nullptr;
    A.ff_mode = 0;
    A.far_io = nullptr;
    A.x_old = nullptr;
    if (ff && inc) {
        A.ff_mode = inc->mode;
        A.far_io = split_far ? far_part : inc->far_io;
        A.x_old = inc->x_old;
        A.bb_io = inc->bb_io;
    }
    if (use_tree) {
        const Tree* T = TT;
        A.tlo = T->tile_lo;
        A.thi = T->tile_hi;
        A.tchi = T->tile_chi;
        A.tclo = T->tile_clo;
        A.list = list;
        A.blist = blist;
        A.border = border;
        A.ppos = T->p_pos;
        A.pnw = T->p_nw;
        A.plo = T->p_lo;
        A.pnwlo = T->p_nwlo;
    }
    A.tsig = tsig;
    A.tgsig = tgsig;
    dim3 grid(nblk, nsplit);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (ctx->profiling) {
        LSM_CUDA_TRY(ctx, cudaEventCreate(&ev0));
        LSM_CUDA_TRY(ctx, cudaEventCreate(&ev1));
        LSM_CUDA_TRY(ctx, cudaEventRecord(ev0, st));
    }
    if (me->sigx) {
        if (mixed && tpb == 64)
            k_eval_mixed<1, true, 2><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                     me->s32_nwlo, A);
        else if (mixed && tpb == kEvalThreads)
            k_eval_mixed<1, true><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo,
                                                                 A);
        else if (mixed)
            k_eval_mixed<kTPT32, true><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                      me->s32_nwlo, A);
        else if (ff64)
            k_eval_ff<true, 64><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, A);
        else if (ff)
            k_eval_ff<true><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, A);
        else
            k_eval_fp64<kTPT64, true><<<grid, kEvalThreads, 0, st>>>(me->s64_pos, me->s64_nw, A);
    } else if (mixed && tpb == 64) {
        k_eval_mixed<1, false, 2><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo,
                                                                  A);
    } else if (mixed && tpb == kEvalThreads) {
        k_eval_mixed<1, false><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, A);
    } else if (mixed) {
        k_eval_mixed<kTPT32, false><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                   me->s32_nwlo, A);
    } else if (ff64) {
        k_eval_ff<false, 64><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, A);
    } else if (ff) {
        k_eval_ff<false><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, A);
    } else {
        k_eval_fp64<kTPT64, false><<<grid, kEvalThreads, 0, st>>>(me->s64_pos, me->s64_nw, A);
    }
    LSM_LAUNCHED(ctx);
    double* rg = nullptr;
    if (clusters && cp.ngblk > 0) {
        // the clusters' grid points against the nodes their clusters took:
        // the same kernel in list mode, every pair far
        LSM_CUDA_TRY(ctx, s.get(&rg, 4 * (size_t)cp.ng));
        EvalArgs G = A;
        G.tx = cp.gx;
        G.ld = cp.ng;
        G.nt = (int)cp.ng;
        G.out = rg;
        G.list = cp.list;
        G.blist = cp.gblist;
        G.border = cp.gorder;
        G.ff_mode = 0;
        G.far_io = nullptr;
        G.x_old = nullptr;
        G.bb_io = nullptr;
        if (ff64)
            k_eval_ff<false, 64><<<cp.ngblk, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, G);
        else if (ff)
            k_eval_ff<false><<<cp.ngblk, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, G);
        else if (tpb == 64)
            k_eval_mixed<1, false, 2><<<cp.ngblk, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                        me->s32_nwlo, G);
        else if (tpb == kEvalThreads)
            k_eval_mixed<1, false><<<cp.ngblk, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                     me->s32_nwlo, G);
        else
            k_eval_mixed<kTPT32, false><<<cp.ngblk, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                          me->s32_nwlo, G);
        LSM_LAUNCHED(ctx);
    }
    if (ctx->profiling) {
        LSM_CUDA_TRY(ctx, cudaEventRecord(ev1, st));
        ctx->prof_events.push_back(Ctx::ProfEvent{ev0, ev1, mixed ? 0 : (ff ? 1 : 2)});
    }
    if (nsplit > 1) {
        k_reduce_splits<<<(t.n + 255) / 256, 256, 0, st>>>(part, nsplit, t.n, res);
        LSM_LAUNCHED(ctx);
    }
    if (split_far) {
        k_reduce_splits<<<(t.n + 255) / 256, 256, 0, st>>>(far_part, nsplit, t.n, inc->far_io);
        LSM_LAUNCHED(ctx);
    }
    if (rg) {
        int rc = cluster_l2p(ctx, cp, t, rg, res, (inc && inc->mode == 1) ? inc->far_io : nullptr, st);
        if (rc != LSM_OK) return rc;
    }
    return LSM_OK;
}

int eval_item_targets(const Ctx* ctx, int precision, int tpb)
{
    if (precision == LSM_MIXED) {
        const int t = tpb > 0 ? tpb : ctx->opt.mixed_block;
        return t == kEvalThreads || t == kEvalThreads * kTPT32 ? t : 64;
    }
    if (precision == LSM_FF) return ctx->opt.ff_block == 64 ? 64 : kEvalThreads;
    return kEvalThreads * kTPT64;
}

int eval_items(Ctx* ctx, const SourceView& v, const Targets& t, const int4* items, const int* n_items,
               int max_items, double* res, int precision, cudaStream_t st, const FFIncremental* inc, int tpb,
               double cut_mixed)
{
    if (max_items <= 0) return LSM_OK;
    EvalArgs A;
    A.tlo = v.tile_lo;
    A.thi = v.tile_hi;
    A.tchi = v.tile_chi;
    A.tclo = v.tile_clo;
    A.ns = 0;
    A.ntiles = v.ntiles;
    A.tiles_per_split = v.ntiles;
    A.tx = t.x;
    A.ld = t.ld;
    A.nt = t.n;
    const bool mixed = precision == LSM_MIXED;
    const double cut = mixed ? (cut_mixed > 0.0 ? cut_mixed : ctx->opt.cutoff_mixed) : ctx->opt.cutoff_fp64;
    A.cut2 = (float)(cut * cut);
    A.out = res;
    A.flag = flag_word(ctx);
    A.test_nocopy = ctx->test_nocopy ? 1 : 0;
    A.wait_limit = ctx->test_nocopy ? kTestWaitLimit : kWaitLimit;
    A.pairs = ctx->d_pairs + 2 * (mixed ? 0 : (precision == LSM_FF ? 1 : 2));
    A.items = items;
    A.n_items = n_items;
    A.ff_mode = 0;
    A.far_io = nullptr;
    A.x_old = nullptr;
    if (precision == LSM_FF && inc) {
        A.ff_mode = inc->mode;
        A.far_io = inc->far_io;
        A.x_old = inc->x_old;
        A.bb_io = inc->bb_io;
    }
    const int bs = eval_item_targets(ctx, precision, tpb);
    if (mixed && bs == 64) {
        k_eval_mixed<1, false, 2><<<max_items, kEvalThreads, 0, st>>>(v.s32_pos, v.s32_nw, v.s32_lo, v.s32_nwlo, A);
    } else if (mixed && bs == kEvalThreads) {
        k_eval_mixed<1, false><<<max_items, kEvalThreads, 0, st>>>(v.s32_pos, v.s32_nw, v.s32_lo, v.s32_nwlo, A);
    } else if (mixed) {
        k_eval_mixed<kTPT32, false><<<max_items, kEvalThreads, 0, st>>>(v.s32_pos, v.s32_nw, v.s32_lo, v.s32_nwlo,
                                                                        A);
    } else if (precision == LSM_FF && bs == 64) {
        k_eval_ff<false, 64><<<max_items, kEvalThreads, 0, st>>>(v.s32_pos, v.s32_nw, v.s32_lo, v.s32_nwlo, A);
    } else if (precision == LSM_FF) {
        k_eval_ff<false><<<max_items, kEvalThreads, 0, st>>>(v.s32_pos, v.s32_nw, v.s32_lo, v.s32_nwlo, A);
    } else {
        k_eval_fp64<kTPT64, false><<<max_items, kEvalThreads, 0, st>>>(v.s64_pos, v.s64_nw, A);
    }
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

// ---------------------------------------------------------------- no-allocation variant
//
// lsm_eval_phi_grad_noalloc runs the same pair kernels without allocating:
// its scratch (SoA targets, result planes, split partials) lives in one
// file-scope device array.  The array's name is a host-side stand-in in host
// code, so its device address is fetched once per device with
// cudaGetSymbolAddress and passed to the kernels.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB on every device that loads the library
constexpr int kNoAllocMaxTargets = 16384;                  // 7 doubles per target for targets and results

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_dev_ptr[64] = {nullptr};

__global__ void k_noalloc_to_soa(const double* __restrict__ x, int n, double* __restrict__ T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; c++) T[(int64_t)c * n + i] = x[3 * (int64_t)i + c];
}

__global__ void k_noalloc_store(const double* __restrict__ R, int n, double* __restrict__ phi,
                                double* __restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    phi[i] = R[i];
    if (grad) {
        for (int c = 0; c < 3; c++) grad[3 * (int64_t)i + c] = R[(int64_t)(c + 1) * n + i];
    }
}

bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

int eval_noalloc(Ctx* ctx, const Mesh* me, const double* x, int64_t n, double* phi, double* grad,
                 int precision, cudaStream_t st)
{
    if (n == 0) return LSM_OK;
    if (n < 0 || n > kNoAllocMaxTargets) {
        ctx->err = "eval_phi_grad_noalloc: n = " + std::to_string(n) + " is outside [0, " +
                   std::to_string(kNoAllocMaxTargets) + "], the size its fixed 8 MiB scratch holds";
        return LSM_E_INVALID_ARG;
    }
    if (!x || !phi || (precision != LSM_FP64 && precision != LSM_MIXED)) {
        ctx->err = "eval_phi_grad_noalloc: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    if (me->sigx) {
        ctx->err = "eval_phi_grad_noalloc: meshes with a target-dependent sigma are not supported";
        return LSM_E_INVALID_ARG;
    }
    if (!on_device(x) || !on_device(phi) || (grad && !on_device(grad))) {
        ctx->err = "eval_phi_grad_noalloc: x, phi and grad must be device pointers";
        return LSM_E_INVALID_ARG;
    }
    if (ctx->device < 0 || ctx->device >= 64) {
        ctx->err = "eval_phi_grad_noalloc: device index out of range";
        return LSM_E_INVALID_ARG;
    }
    // set-up, once per device, with the context's device current
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_dev_ptr[ctx->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                ctx->err = std::string("eval_phi_grad_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return LSM_E_CUDA;
            }
            g_noalloc_dev_ptr[ctx->device] = p;
        }
        base = static_cast<unsigned char*>(g_noalloc_dev_ptr[ctx->device]);
    }
    const int nt = (int)n;
    double* T = reinterpret_cast<double*>(base);
    double* R = T + 3 * (size_t)nt;
    double* part = R + 4 * (size_t)nt;
    const size_t room = kNoAllocScratchBytes - sizeof(double) * 7 * (size_t)nt;
    const int max_split = (int)std::max<size_t>(1, room / (sizeof(double) * 4 * (size_t)nt));

    const bool mixed = precision == LSM_MIXED;
    const int tpb = kEvalThreads * (mixed ? kTPT32 : kTPT64);
    const int nblk = (nt + tpb - 1) / tpb;
    const int ntiles = (int)me->ntiles;
    const int want = ctx->num_sms * 16;
    int nsplit = 1;
    if (nblk < want) nsplit = std::min((want + nblk - 1) / nblk, std::max(1, ntiles / 4));
    nsplit = std::min(nsplit, max_split);
    const int tps = (ntiles + nsplit - 1) / nsplit;
    nsplit = (ntiles + tps - 1) / tps;

    k_noalloc_to_soa<<<(nt + 255) / 256, 256, 0, st>>>(x, nt, T);
    LSM_LAUNCHED(ctx);
    EvalArgs A;
    A.tlo = me->tile_lo;
    A.thi = me->tile_hi;
    A.tchi = me->tile_chi;
    A.tclo = me->tile_clo;
    A.ns = (int)me->ns;
    A.ntiles = ntiles;
    A.tiles_per_split = tps;
    A.tx = T;
    A.ld = nt;
    A.nt = nt;
    const double cut = mixed ? ctx->opt.cutoff_mixed : ctx->opt.cutoff_fp64;
    A.cut2 = (float)(cut * cut);
    A.out = nsplit > 1 ? part : R;
    A.flag = flag_word(ctx);
    A.test_nocopy = ctx->test_nocopy ? 1 : 0;
    A.wait_limit = ctx->test_nocopy ? kTestWaitLimit : kWaitLimit;
    A.pairs = ctx->d_pairs + 2 * (mixed ? 0 : (precision == LSM_FF ? 1 : 2));
    A.items = nullptr;
    A.n_items = nullptr;
    A.ff_mode = 0;
    A.far_io = nullptr;
    A.x_old = nullptr;
    dim3 grid(nblk, nsplit);
    if (mixed) {
        k_eval_mixed<kTPT32, false><<<grid, kEvalThreads, 0, st>>>(me->s32_pos, me->s32_nw, me->s32_lo,
                                                                   me->s32_nwlo, A);
    } else {
        k_eval_fp64<kTPT64, false><<<grid, kEvalThreads, 0, st>>>(me->s64_pos, me->s64_nw, A);
    }
    LSM_LAUNCHED(ctx);
    if (nsplit > 1) {
        k_reduce_splits<<<(nt + 255) / 256, 256, 0, st>>>(part, nsplit, nt, R);
        LSM_LAUNCHED(ctx);
    }
    k_noalloc_store<<<(nt + 255) / 256, 256, 0, st>>>(R, nt, phi, grad);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace lsm
