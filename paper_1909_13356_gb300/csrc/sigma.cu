// sigma.cu -- the target-dependent smoothing width (Sec. 2.3, eq. sigma2):
//   sigma(x) = sum_j sigma_j e_j / sum_j e_j,   e_j = exp(-|x - c_j|^2 / (2 sigma0^2)),
// a Gaussian-weighted mean over the triangle centroids c_j of
// sigma_j = D_j / lambda (D_j the diameter of the smallest ball enclosing
// triangle j), and its gradient
//   grad sigma = (S1 sum_j e_j (x - c_j) - S0 sum_j sigma_j e_j (x - c_j)) / (sigma0^2 S0^2),
// S0 = sum_j e_j, S1 = sum_j sigma_j e_j.
//
// The centroids are Morton-sorted into tiles of kTile with outward-rounded
// FP32 boxes.  A CTA owns a block of sorted targets.  It first bounds, from
// the boxes, the squared distance U within which every target of the block
// has a centroid (the least, over tiles, of the farthest block-to-tile
// distance), then sums only tiles whose nearest distance is below
// U + 2 T sigma0^2: a skipped centroid weighs less than e^-T of each target's
// nearest one (T = 37.5 for the FP64-accurate paths, 20 for the mixed path).  The weights are taken relative to exp(-U / 2
// sigma0^2) (a common factor that cancels in the ratio), so nothing
// underflows however far the targets are.  The FP64 path sums in FP64; the
// mixed and float-float paths sum in float-float on the FP32 pipes, with a
// float-float exponential (FP64 exp on this GPU's FP64 pipe, 1/76 of its FP32
// rate, was most of a sigma(x) evaluation).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lsm_internal.cuh"
#include "ff.cuh"

namespace lsm {
namespace {

constexpr int kSigThreads = 128;

uint32_t spread10(uint32_t v)
{
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ float box_gap2(float4 alo, float4 ahi, const float* bb)
{
    const float gx = fmaxf(0.0f, fmaxf(alo.x - bb[3], bb[0] - ahi.x));
    const float gy = fmaxf(0.0f, fmaxf(alo.y - bb[4], bb[1] - ahi.y));
    const float gz = fmaxf(0.0f, fmaxf(alo.z - bb[5], bb[2] - ahi.z));
    return gx * gx + gy * gy + gz * gz;
}
__device__ __forceinline__ float box_far2(float4 alo, float4 ahi, const float* bb)
{
    const float fx = fmaxf(ahi.x - bb[0], bb[3] - alo.x);
    const float fy = fmaxf(ahi.y - bb[1], bb[4] - alo.y);
    const float fz = fmaxf(ahi.z - bb[2], bb[5] - alo.z);
    return fx * fx + fy * fy + fz * fz;
}

// Constants of the float-float exponential, from the host: ln2/64 = c1 + c2 +
// c3 with c1 of 10 significant bits (so that n c1 is exact for |n| < 2^14)
struct ExpConsts {
    float c1, c2, c3;
};

// e^w for a float pair w <= 60 (the sigma(x) weights), by Tang's table-driven
// reduction (ACM TOMS 15, 1989) carried out in float-float: w = n ln2/64 + r with
// n = 64 k + j, |r| <= ln2/128; e^r - 1 from its Taylor series to r^5 (error
// r^6/720 < 4e-17), the low orders in float-float; then e^w = 2^k 2^(j/64)
// (1 + (e^r - 1)), the power of two applied to both floats exactly.  Below
// w = -87 (e^w < FLT_MIN: 2^k would leave the normal range) the weight is 0;
// the caller's weights are relative to one of at least 1.
__device__ __forceinline__ void ff_exp(float wh, float wl, const ExpConsts& E, const float2* tab, float& eh,
                                       float& el)
{
    if (wh < -87.0f) {
        eh = el = 0.0f;
        return;
    }
    const float nf = rintf(wh * 92.332482616893656f);   // 64 / ln2, rounded: n need only be near
    const int n = (int)nf;
    // r = w - n (c1 + c2 + c3): n c1 is exact (|n| < 2^14, c1 of 10 bits),
    // its difference with w_hi and the product n c2 are taken with their
    // errors, n c3 is below the float-float unit
    float a, ae;
    two_diff(wh, nf * E.c1, a, ae);
    const float b = nf * E.c2;
    const float be = fmaf(nf, E.c2, -b);
    float rh, rl, r2, e3;
    two_diff(a, b, r2, rl);
    two_sum(r2, wl, rh, e3);   // w's low part can be as large as ulp(w_hi) / 2 ~ 2e-6: error-free
    rl = (((rl + e3) + ae) - be) - nf * E.c3;
    const float t = rh + rl;   // renormalise
    rl = rl - (t - rh);
    rh = t;
    // e^r - 1 = r (1 + r (1/2 + r (1/6 + r (1/24 + r/120)))): the inner two
    // orders in FP32, then float-float steps
    const float q = fmaf(rh, 1.0f / 120.0f, 1.0f / 24.0f);
    float uh, ul, mh, ml;
    ff_mul(rh, rl, q, 0.0f, mh, ml);
    ff_add(0.16666667163372040f, -4.9670538793123e-09f, mh, ml, uh, ul);   // 1/6
    ff_mul(rh, rl, uh, ul, mh, ml);
    ff_add(0.5f, 0.0f, mh, ml, uh, ul);
    ff_mul(rh, rl, uh, ul, mh, ml);
    ff_add(1.0f, 0.0f, mh, ml, uh, ul);
    float ph, pl;
    ff_mul(rh, rl, uh, ul, ph, pl);   // e^r - 1
    // 2^(j/64) (1 + p) = T + T p
    const float2 T = tab[n & 63];
    ff_mul(T.x, T.y, ph, pl, mh, ml);
    ff_add(T.x, T.y, mh, ml, uh, ul);
    const float s2 = __int_as_float((((n >> 6) + 127) & 255) << 23);   // 2^k, k = floor(n / 64)
    eh = uh * s2;
    el = ul * s2;
}

// FF: the sums in float-float on the FP32 pipes (the weights from ff_exp,
// sigma and S0 to about 1e-15; the gradient's sums in FP32 with compensated
// accumulation, as the pair kernels' gradients).  A block whose weight range
// could leave the FP32 exponent range (U / 2 sigma0^2 > 60: targets spread
// over more than ~13 sigma0) takes the FP64 loop instead.
template <bool FF>
__global__ void __launch_bounds__(kSigThreads) k_sigma_x(const double4_32a* __restrict__ cent,
                                                         const float4* __restrict__ clo,
                                                         const float4* __restrict__ chi, int64_t ncent, int ntile,
                                                         const double* __restrict__ x, int64_t ld, int n,
                                                         double sigma0, double tail, ExpConsts E,
                                                         double* __restrict__ sig, double* __restrict__ gsig)
{
    __shared__ double4_32a sc[kTile];
    __shared__ float4 s_ch[kTile], s_cl[kTile];   // FF: centroid - block reference (x, y, z, sigma_j) as float pairs
    __shared__ float2 s_tab[64];
    __shared__ float s_bb[6];
    __shared__ float s_red[kSigThreads / 32];
    __shared__ float s_u;
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kSigThreads + tid;
    const bool valid = i < n;
    // 2^(j/64), j = 0..63, as float pairs for the float-float exponential:
    // each block forms its own from the FP64 exp2 (relative error ~1e-16)
    if (FF && tid < 64) {
        const double v = exp2((double)tid * (1.0 / 64.0));
        const float h = (float)v;
        s_tab[tid] = make_float2(h, (float)(v - (double)h));
    }
    double xs[3] = {0.0, 0.0, 0.0};
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = 0; c < 3; c++) {
        if (valid) {
            xs[c] = x[c * ld + i];
            lo[c] = __double2float_rd(xs[c]);
            hi[c] = __double2float_ru(xs[c]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    __shared__ float part[6][kSigThreads / 32];
    const int w = tid >> 5, lane = tid & 31;
    if (lane == 0)
        for (int c = 0; c < 3; c++) {
            part[c][w] = lo[c];
            part[3 + c][w] = hi[c];
        }
    __syncthreads();
    if (tid == 0) {
        for (int c = 0; c < 3; c++) {
            float L = part[c][0], H = part[3 + c][0];
            for (int k = 1; k < kSigThreads / 32; k++) {
                L = fminf(L, part[c][k]);
                H = fmaxf(H, part[3 + c][k]);
            }
            s_bb[c] = L;
            s_bb[3 + c] = H;
        }
    }
    __syncthreads();
    // U: every target of the block has a centroid within sqrt(U)
    float u = INFINITY;
    for (int t = tid; t < ntile; t += kSigThreads) u = fminf(u, box_far2(clo[t], chi[t], s_bb));
    for (int o = 16; o > 0; o >>= 1) u = fminf(u, __shfl_xor_sync(0xffffffffu, u, o));
    if (lane == 0) s_red[w] = u;
    __syncthreads();
    if (tid == 0) {
        float m = s_red[0];
        for (int k = 1; k < kSigThreads / 32; k++) m = fminf(m, s_red[k]);
        s_u = m;
    }
    __syncthreads();
    const double U = (double)s_u;
    const double inv2s2 = 1.0 / (2.0 * sigma0 * sigma0);
    const float reach2 = (float)(U + 2.0 * tail * sigma0 * sigma0) * 1.0001f;
    const bool ff = FF && U * inv2s2 <= 60.0;   // block-uniform
    // FF: the block reference (its first target) and the target's offset
    // from it as a float pair; 1/(2 sigma0^2) as a float pair
    double bref[3] = {0.0, 0.0, 0.0};
    float xh[3] = {0.0f, 0.0f, 0.0f}, xl[3] = {0.0f, 0.0f, 0.0f};
    const float iwh = (float)inv2s2, iwl = (float)(inv2s2 - (double)iwh);
    if (ff) {
        const int i0 = blockIdx.x * kSigThreads;
        for (int c = 0; c < 3; c++) {
            bref[c] = x[c * ld + i0];
            const double d = (valid ? xs[c] : bref[c]) - bref[c];
            xh[c] = (float)d;
            xl[c] = (float)(d - (double)xh[c]);
        }
    }
    double S0 = 0.0, S1 = 0.0, A[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
    float s0h = 0.0f, s0l = 0.0f, s1h = 0.0f, s1l = 0.0f;
    float ah[3] = {0.0f, 0.0f, 0.0f}, al[3] = {0.0f, 0.0f, 0.0f}, bh[3] = {0.0f, 0.0f, 0.0f},
          bl[3] = {0.0f, 0.0f, 0.0f};
    // candidate tiles kSigThreads at a time: each thread tests one, the
    // block compacts the list in tile order, then sums the listed tiles
    __shared__ int s_list[kSigThreads];
    __shared__ int s_wcnt[kSigThreads / 32];
    for (int tb = 0; tb < ntile; tb += kSigThreads) {
        const int tt = tb + tid;
        const bool take = tt < ntile && box_gap2(clo[tt], chi[tt], s_bb) <= reach2;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (lane == 0) s_wcnt[w] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int k = 0; k < kSigThreads / 32; k++) {
            off += k < w ? s_wcnt[k] : 0;
            tot += s_wcnt[k];
        }
        if (take) s_list[off + __popc(bal & ((1u << lane) - 1u))] = tt;
        __syncthreads();
        for (int q = 0; q < tot; q++) {
            const int t = s_list[q];
            const int64_t j0 = (int64_t)t * kTile;
            const int cnt = (int)(ncent - j0 < kTile ? ncent - j0 : kTile);
            if (tid < cnt) {
                const double4_32a cj = cent[j0 + tid];
                if (ff) {
                    const double d0 = cj.x - bref[0], d1 = cj.y - bref[1], d2 = cj.z - bref[2];
                    const float h0 = (float)d0, h1 = (float)d1, h2 = (float)d2, hs = (float)cj.w;
                    s_ch[tid] = make_float4(h0, h1, h2, hs);
                    s_cl[tid] = make_float4((float)(d0 - (double)h0), (float)(d1 - (double)h1),
                                            (float)(d2 - (double)h2), (float)(cj.w - (double)hs));
                } else {
                    sc[tid] = cj;
                }
            }
            __syncthreads();
            if (valid && ff) {
                for (int s = 0; s < cnt; s++) {
                    const float4 ch = s_ch[s], cl = s_cl[s];
                    // r = x - c as float pairs (the FP64 loop's dx)
                    float dh[3], dl[3];
                    const float cch[3] = {ch.x, ch.y, ch.z}, ccl[3] = {cl.x, cl.y, cl.z};
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        float e;
                        two_diff(xh[c], cch[c], dh[c], e);
                        dl[c] = e + (xl[c] - ccl[c]);
                    }
                    // |r|^2: squares' errors, non-negative two-sums, cross terms
                    const float p0 = dh[0] * dh[0], p1 = dh[1] * dh[1], p2 = dh[2] * dh[2];
                    const float e0 = fmaf(dh[0], dh[0], -p0), e1 = fmaf(dh[1], dh[1], -p1),
                                e2 = fmaf(dh[2], dh[2], -p2);
                    const float cr = fmaf(dh[0], dl[0], fmaf(dh[1], dl[1], dh[2] * dl[2]));
                    float s01, t01, t2, rh;
                    two_sum_nonneg(p0, p1, s01, t01);
                    two_sum_nonneg(s01, p2, rh, t2);
                    const float rl = fmaf(2.0f, cr, ((e0 + e1) + e2) + (t01 + t2));
                    // w = (U - |r|^2) / (2 sigma0^2)
                    float gh, gl;
                    two_diff(s_u, rh, gh, gl);
                    gl -= rl;
                    float wh, wl;
                    ff_mul(gh, gl, iwh, iwl, wh, wl);
                    float eh, el;
                    ff_exp(wh, wl, E, s_tab, eh, el);
                    // S0 += e, S1 += sigma_j e (float-float); the gradient's sums (FP32)
                    float nh, nl;
                    ff_add(s0h, s0l, eh, el, nh, nl);
                    s0h = nh;
                    s0l = nl;
                    float se_h, se_l;
                    ff_mul(ch.w, cl.w, eh, el, se_h, se_l);
                    ff_add(s1h, s1l, se_h, se_l, nh, nl);
                    s1h = nh;
                    s1l = nl;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        two_sum_acc(ah[c], al[c], eh * dh[c]);
                        two_sum_acc(bh[c], bl[c], se_h * dh[c]);
                    }
                }
            } else if (valid) {
                for (int s = 0; s < cnt; s++) {
                    const double4_32a cj = sc[s];
                    const double dx = xs[0] - cj.x, dy = xs[1] - cj.y, dz = xs[2] - cj.z;
                    const double e = exp((U - (dx * dx + dy * dy + dz * dz)) * inv2s2);
                    S0 += e;
                    S1 += cj.w * e;
                    A[0] += e * dx;
                    A[1] += e * dy;
                    A[2] += e * dz;
                    B[0] += cj.w * e * dx;
                    B[1] += cj.w * e * dy;
                    B[2] += cj.w * e * dz;
                }
            }
            __syncthreads();
        }
    }
    if (valid) {
        if (ff) {
            S0 = (double)s0h + (double)s0l;
            S1 = (double)s1h + (double)s1l;
            for (int c = 0; c < 3; c++) {
                A[c] = (double)ah[c] + (double)al[c];
                B[c] = (double)bh[c] + (double)bl[c];
            }
        }
        sig[i] = S1 / S0;
        const double den = sigma0 * sigma0 * S0 * S0;
        for (int c = 0; c < 3; c++) gsig[(int64_t)c * n + i] = (S1 * A[c] - S0 * B[c]) / den;
    }
}

}  // namespace

// sigma_j = D_j / lambda and centroids (host, input triangle order); returns
// max_j D_j.  D_j: the longest edge of a right or obtuse triangle, else the
// circumdiameter abc / (2 area).
double sigma_sources_host(const double* verts, const int32_t* tris, int64_t nt, double lambda, double* sj,
                          double* cen)
{
    double dmax = 0.0;
    for (int64_t j = 0; j < nt; j++) {
        const double* p[3] = {verts + 3 * (int64_t)tris[3 * j], verts + 3 * (int64_t)tris[3 * j + 1],
                              verts + 3 * (int64_t)tris[3 * j + 2]};
        double e2[3];
        for (int k = 0; k < 3; k++) {
            const double* a = p[(k + 1) % 3];
            const double* b = p[(k + 2) % 3];
            const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
            e2[k] = dx * dx + dy * dy + dz * dz;
        }
        const double ux = p[1][0] - p[0][0], uy = p[1][1] - p[0][1], uz = p[1][2] - p[0][2];
        const double vx = p[2][0] - p[0][0], vy = p[2][1] - p[0][1], vz = p[2][2] - p[0][2];
        const double cx = uy * vz - uz * vy, cy = uz * vx - ux * vz, cz = ux * vy - uy * vx;
        const double area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
        int kl = 0;
        if (e2[1] > e2[kl]) kl = 1;
        if (e2[2] > e2[kl]) kl = 2;
        const double D = e2[kl] >= e2[(kl + 1) % 3] + e2[(kl + 2) % 3]
                             ? std::sqrt(e2[kl])
                             : std::sqrt(e2[0]) * std::sqrt(e2[1]) * std::sqrt(e2[2]) / (2.0 * area);
        sj[j] = D / lambda;
        for (int c = 0; c < 3; c++) cen[3 * j + c] = (p[0][c] + p[1][c] + p[2][c]) / 3.0;
        dmax = std::max(dmax, D);
    }
    return dmax;
}

// The centroid tiles of a sigma(x) mesh (Morton order, outward-rounded boxes).
int sigma_attach(Ctx* ctx, Mesh* me, const double* sj, const double* cen, int64_t nt, double sigma0,
                 cudaStream_t st)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = 0; j < nt; j++)
        for (int c = 0; c < 3; c++) {
            lo[c] = std::min(lo[c], cen[3 * j + c]);
            hi[c] = std::max(hi[c], cen[3 * j + c]);
        }
    const double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
    std::vector<std::pair<uint32_t, int64_t>> key(nt);
    for (int64_t j = 0; j < nt; j++) {
        uint32_t q[3];
        for (int c = 0; c < 3; c++)
            q[c] = (uint32_t)std::min(1023.0, std::max(0.0, (cen[3 * j + c] - lo[c]) / ext * 1023.0));
        key[j] = {(spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]), j};
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<uint32_t, int64_t>& a, const std::pair<uint32_t, int64_t>& b) {
                         return a.first < b.first;
                     });
    const int64_t ntile = (nt + kTile - 1) / kTile;
    std::vector<double4_32a> hc(nt);
    std::vector<float4> hlo(ntile), hhi(ntile);
    for (int64_t t = 0; t < ntile; t++) {
        float l[3] = {INFINITY, INFINITY, INFINITY}, h[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t k = t * kTile; k < std::min(nt, (t + 1) * kTile); k++) {
            const int64_t j = key[k].second;
            hc[k] = make_double4_32a(cen[3 * j], cen[3 * j + 1], cen[3 * j + 2], sj[j]);
            for (int c = 0; c < 3; c++) {
                const double v = cen[3 * j + c];
                float f = (float)v;
                if ((double)f > v) f = std::nextafter(f, -INFINITY);
                l[c] = std::min(l[c], f);
                float g = (float)v;
                if ((double)g < v) g = std::nextafter(g, INFINITY);
                h[c] = std::max(h[c], g);
            }
        }
        hlo[t] = make_float4(l[0], l[1], l[2], 0.0f);
        hhi[t] = make_float4(h[0], h[1], h[2], 0.0f);
    }
    LSM_CUDA_TRY(ctx, cudaMalloc(&me->cent, sizeof(double4_32a) * nt));
    LSM_CUDA_TRY(ctx, cudaMalloc(&me->cent_lo, sizeof(float4) * ntile));
    LSM_CUDA_TRY(ctx, cudaMalloc(&me->cent_hi, sizeof(float4) * ntile));
    me->bytes += sizeof(double4_32a) * nt + 2 * sizeof(float4) * ntile;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(me->cent, hc.data(), sizeof(double4_32a) * nt, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(me->cent_lo, hlo.data(), sizeof(float4) * ntile, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(me->cent_hi, hhi.data(), sizeof(float4) * ntile, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    me->sigx = true;
    me->sigma0 = sigma0;
    me->ncent = nt;
    me->ncent_tiles = ntile;
    return LSM_OK;
}

namespace {

// The three-float split of ln2/64 for the float-float exponential, from long
// double: c1 of 10 significant bits, so that n c1 is exact for |n| < 2^14
ExpConsts exp_constants()
{
    const long double l = logl(2.0L) / 64.0L;
    const long double c1 = ldexpl(roundl(ldexpl(l, 16)), -16);
    ExpConsts E;
    E.c1 = (float)c1;
    E.c2 = (float)(l - c1);
    E.c3 = (float)(l - c1 - (long double)E.c2);
    return E;
}

}  // namespace

int sigma_x_eval(Ctx* ctx, const Mesh* me, const Targets& t, double* sig, double* gsig, cudaStream_t st,
                 int precision)
{
    if (t.n <= 0) return LSM_OK;
    const int nb = (t.n + kSigThreads - 1) / kSigThreads;
    // truncation: e^-20 (2e-9 relative) suffices for the mixed path's 1e-7,
    // e^-37.5 (5e-17) for the FP64-accurate ones.  The FP64 path keeps its
    // sums in FP64; the mixed and float-float paths sum in float-float.
    const double tail = precision == LSM_MIXED ? 20.0 : 37.5;
    const ExpConsts E = exp_constants();
    if (precision == LSM_FP64)
        k_sigma_x<false><<<nb, kSigThreads, 0, st>>>(me->cent, me->cent_lo, me->cent_hi, me->ncent,
                                                     (int)me->ncent_tiles, t.x, t.ld, t.n, me->sigma0, tail, E, sig,
                                                     gsig);
    else
        k_sigma_x<true><<<nb, kSigThreads, 0, st>>>(me->cent, me->cent_lo, me->cent_hi, me->ncent,
                                                    (int)me->ncent_tiles, t.x, t.ld, t.n, me->sigma0, tail, E, sig,
                                                    gsig);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace lsm
