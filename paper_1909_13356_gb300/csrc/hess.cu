// hess.cu -- the Hessian of Phi at targets (Sec. 3.3: second derivatives of
// the charts need the Hessian of Phi, eq. uu_vector_aux1).
//
// For one pair, with r = y - x, q = nw . r and the radial factors
// f = g(u)/(4 pi rho^3), F = f'(rho)/rho, G = F'(rho)/rho,
//   d2/dx_i dx_j [q f] = F (nw_i r_j + nw_j r_i + q delta_ij) + q G r_i r_j.
// With a = 1/(sqrt2 sigma), w = u^2 = rho^2 a^2, h(w) = g(u)/u^3 and
// nw' = nw / 4 pi (the resident weights):
//   f -> a^3 h,   F -> a^5 k,   G -> a^7 kp,
//   k = h'(u)/u = 2 dh/dw,  kp = k'(u)/u = 2 dk/dw,
// read from a piecewise polynomial table of h in w (FP64); beyond the cutoff
// they are the Laplace limits 1/rho^3, -3/rho^5, 15/rho^7.
//
// Near the level set the Hessian's curvature part is a small fraction of
// its terms, which cancel: near tiles are summed in FP64.  Far tiles (the
// Laplace double layer, no cancellation of note) are summed in FP32 on
// tile-local coordinates with compensated accumulation, and so are the
// sources of a near tile that lie beyond the cutoff from the CTA's whole
// target box (Sec. 4.4, eq. kerdecomp: the split by distance, per source).  A CTA owns 128
// sorted targets and walks a range of tiles (a grid row per split, partials
// reduced in a fixed order): all tiles, or on a large mesh the interaction
// list of the mixed path's treecode built for this kernel's near radius
// (proxy tiles are far; x-derivatives of the interpolated kernel are the
// interpolated derivatives).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kHessThreads = kTile;   // one target per thread, tiles staged by one load per thread
// FP64 table of h(w) = g(u)/u^3: interval k covers w in [k, k+1)/16 up to
// w = 32.5, the degree-6 interpolant about the interval's centre (fitted in
// long double at setup, 8 doubles per interval).  h, dh/dw and d2h/dw2 come
// from the same polynomial: k = 2 dh/dw, kp = 4 d2h/dw2.  Beyond the table
// (|r| > 8 sigma) the Laplace limits hold to about 1e-11 relative.
constexpr int kH64PerUnit = 16;
constexpr int kH64N = 520;
constexpr double kH64Wmax = (double)kH64N / kH64PerUnit;
__device__ double g_htab64[kH64N * 8];

__device__ __forceinline__ void radial3(double r2, double a, const double* __restrict__ tab, double& fH,
                                        double& FK, double& GK)
{
    const double w = r2 * a * a;
    if (w < kH64Wmax) {
        const int k = min((int)(w * (double)kH64PerUnit), kH64N - 1);
        const double t = w - ((double)k + 0.5) * (1.0 / kH64PerUnit);
        const double* c = tab + 8 * k;
        const double h = fma(fma(fma(fma(fma(fma(c[6], t, c[5]), t, c[4]), t, c[3]), t, c[2]), t, c[1]), t, c[0]);
        const double d1 =
            fma(fma(fma(fma(fma(6.0 * c[6], t, 5.0 * c[5]), t, 4.0 * c[4]), t, 3.0 * c[3]), t, 2.0 * c[2]), t, c[1]);
        const double d2 = fma(fma(fma(fma(30.0 * c[6], t, 20.0 * c[5]), t, 12.0 * c[4]), t, 6.0 * c[3]), t, 2.0 * c[2]);
        const double a2 = a * a, a3 = a2 * a;
        fH = a3 * h;
        FK = a3 * a2 * 2.0 * d1;
        GK = a3 * a2 * a2 * 4.0 * d2;
    } else {
        const double ri = rsqrt(r2);
        const double ri2 = ri * ri;
        fH = ri2 * ri;
        FK = -3.0 * fH * ri2;
        GK = 15.0 * fH * ri2 * ri2;
    }
}

__device__ __forceinline__ void tsum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

struct HessArgs {
    const float4* s32_pos;        // tile-local FP32 positions (far tiles)
    const float4* s32_nw;
    const double4_32a* s64_pos;   // FP64 (near tiles): (x, y, z, a)
    const double4_32a* s64_nw;    // (nw / 4 pi, sqrt2 sigma)
    const float4 *tlo, *thi, *tchi, *tclo;
    int ntiles, tiles_per_split;
    const double* tx;
    int64_t ld;
    int nt;
    float cut2;
    double* out;                  // [split][6][nt]
    unsigned long long* pairs;    // [2] pairs in near / far tiles
    // treecode lists (optional): block b walks list[blist[b].x .. + blist[b].y),
    // launched in the order border; ids >= ntiles are proxy tiles (ppos, pnw)
    const int* list;
    const int2* blist;
    const int* border;
    const float4* ppos;
    const float4* pnw;
};

__global__ void __launch_bounds__(kHessThreads) k_eval_hess(HessArgs A)
{
    __shared__ float4 sp[kTile], sn[kTile];
    __shared__ double4_32a dp[kTile], dn[kTile];
    __shared__ double s_tab[kH64N * 8];
    __shared__ float part[6][kHessThreads / 32];
    __shared__ float bb[6];
    __shared__ unsigned char s_far[kTile];   // near tile: the source is beyond the cutoff from the whole block
    const int tid = threadIdx.x;
    int blk = blockIdx.x, t0, t1;
    if (A.list) {
        blk = A.border[blockIdx.x];
        const int2 r = A.blist[blk];
        const int per = (r.y + (int)gridDim.y - 1) / (int)gridDim.y;
        t0 = min(r.x + (int)blockIdx.y * per, r.x + r.y);
        t1 = min(r.x + r.y, t0 + per);
    } else {
        t0 = blockIdx.y * A.tiles_per_split;
        t1 = min(A.ntiles, t0 + A.tiles_per_split);
    }
    const int i = blk * kHessThreads + tid;
    const bool valid = i < A.nt;

    for (int k = tid; k < kH64N * 8; k += kHessThreads) s_tab[k] = g_htab64[k];
    double x[3] = {0.0, 0.0, 0.0};
    float xh[3], xl[3];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int c = 0; c < 3; c++) {
        if (valid) {
            x[c] = A.tx[c * A.ld + i];
            lo[c] = __double2float_rd(x[c]);
            hi[c] = __double2float_ru(x[c]);
        }
        xh[c] = (float)x[c];
        xl[c] = (float)(x[c] - (double)xh[c]);
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    if ((tid & 31) == 0)
        for (int c = 0; c < 3; c++) {
            part[c][tid >> 5] = lo[c];
            part[3 + c][tid >> 5] = hi[c];
        }
    __syncthreads();
    if (tid == 0)
        for (int c = 0; c < 3; c++) {
            float L = part[c][0], H = part[3 + c][0];
            for (int k = 1; k < kHessThreads / 32; k++) {
                L = fminf(L, part[c][k]);
                H = fmaxf(H, part[3 + c][k]);
            }
            bb[c] = L;
            bb[3 + c] = H;
        }
    __syncthreads();

    float fh[6], fl[6];   // far part, float-float
    double nh[6];         // near part, FP64
    for (int c = 0; c < 6; c++) {
        fh[c] = fl[c] = 0.0f;
        nh[c] = 0.0;
    }
    unsigned long long pn = 0, pf = 0;
    for (int jt = t0; jt < t1; jt++) {
        const int t = A.list ? A.list[jt] : jt;
        const bool proxy = t >= A.ntiles;
        const float4 tl = A.tlo[t], th = A.thi[t];
        const float gx = fmaxf(0.0f, fmaxf(tl.x - bb[3], bb[0] - th.x));
        const float gy = fmaxf(0.0f, fmaxf(tl.y - bb[4], bb[1] - th.y));
        const float gz = fmaxf(0.0f, fmaxf(tl.z - bb[5], bb[2] - th.z));
        const bool far = proxy || gx * gx + gy * gy + gz * gz > A.cut2 * tl.w * tl.w * 1.0001f;
        const int cnt = (int)th.w;
        const int64_t j = (int64_t)(proxy ? t - A.ntiles : t) * kTile + tid;
        bool src_far = false;
        if (tid < cnt) {
            if (proxy) {
                sp[tid] = A.ppos[j];
                sn[tid] = A.pnw[j];
            } else {
                sp[tid] = A.s32_pos[j];
                sn[tid] = A.s32_nw[j];
            }
            if (!far) {
                // near tile: a source beyond the cutoff from every point of the
                // block's box (its own sigma, FP64 distance to the outward
                // box) takes the FP32 Laplace pair of the far tiles
                const double4_32a y = A.s64_pos[j], n = A.s64_nw[j];
                dp[tid] = y;
                dn[tid] = n;
                const double gx = fmax(0.0, fmax((double)bb[0] - y.x, y.x - (double)bb[3]));
                const double gy = fmax(0.0, fmax((double)bb[1] - y.y, y.y - (double)bb[4]));
                const double gz = fmax(0.0, fmax((double)bb[2] - y.z, y.z - (double)bb[5]));
                src_far = gx * gx + gy * gy + gz * gz > (double)A.cut2 * 0.5 * n.w * n.w * (1.0 + 1e-9);
                s_far[tid] = src_far ? 1 : 0;
            }
        }
        const int nfar = far ? cnt : __syncthreads_count(src_far);
        if (far) __syncthreads();
        if (valid) {
            pf += nfar;
            pn += cnt - nfar;
        }
        // the FP32 Laplace pair on tile-local coordinates (far tiles, and far
        // sources of a near tile), r = y - x
        auto far_pair = [&](const float4& y, const float4& n, float qx, float qy, float qz, float (&p)[6]) {
            const float r0 = y.x - qx, r1 = y.y - qy, r2c = y.z - qz;
            const float r2 = fmaf(r0, r0, fmaf(r1, r1, r2c * r2c));
            float ri = rsqrtf(r2);
            ri = ri * fmaf(-0.5f * r2 * ri, ri, 1.5f);   // one Newton step for 1/sqrt
            const float ri2 = ri * ri;
            const float ri5 = ri2 * ri2 * ri;
            const float q = fmaf(n.x, r0, fmaf(n.y, r1, n.z * r2c));
            const float F = -3.0f * ri5;
            const float qG = 15.0f * q * ri5 * ri2;
            p[0] += F * (2.0f * n.x * r0 + q) + qG * r0 * r0;
            p[1] += F * (n.x * r1 + n.y * r0) + qG * r0 * r1;
            p[2] += F * (n.x * r2c + n.z * r0) + qG * r0 * r2c;
            p[3] += F * (2.0f * n.y * r1 + q) + qG * r1 * r1;
            p[4] += F * (n.y * r2c + n.z * r1) + qG * r1 * r2c;
            p[5] += F * (2.0f * n.z * r2c + q) + qG * r2c * r2c;
        };
        // target in tile-local coordinates
        const float4 ch = A.tchi[t], cl = A.tclo[t];
        const float qx = (xh[0] - ch.x) + (xl[0] - cl.x);
        const float qy = (xh[1] - ch.y) + (xl[1] - cl.y);
        const float qz = (xh[2] - ch.z) + (xl[2] - cl.z);
        if (far) {
            float p[6] = {0, 0, 0, 0, 0, 0};
            for (int s = 0; s < cnt; s++) far_pair(sp[s], sn[s], qx, qy, qz, p);
            for (int c = 0; c < 6; c++) tsum(fh[c], fl[c], p[c]);
        } else {
            double p[6] = {0, 0, 0, 0, 0, 0};
            float pf32[6] = {0, 0, 0, 0, 0, 0};
            for (int s = 0; s < cnt; s++) {
                if (s_far[s]) {   // uniform over the CTA
                    far_pair(sp[s], sn[s], qx, qy, qz, pf32);
                    continue;
                }
                const double4_32a y = dp[s], n = dn[s];
                const double r0 = y.x - x[0], r1 = y.y - x[1], r2c = y.z - x[2];
                const double r2 = fma(r0, r0, fma(r1, r1, r2c * r2c));
                double fH, F, G;
                radial3(r2, y.w, s_tab, fH, F, G);
                const double q = fma(n.x, r0, fma(n.y, r1, n.z * r2c));
                const double qG = q * G;
                p[0] += F * (2.0 * n.x * r0 + q) + qG * r0 * r0;
                p[1] += F * (n.x * r1 + n.y * r0) + qG * r0 * r1;
                p[2] += F * (n.x * r2c + n.z * r0) + qG * r0 * r2c;
                p[3] += F * (2.0 * n.y * r1 + q) + qG * r1 * r1;
                p[4] += F * (n.y * r2c + n.z * r1) + qG * r1 * r2c;
                p[5] += F * (2.0 * n.z * r2c + q) + qG * r2c * r2c;
            }
            for (int c = 0; c < 6; c++) {
                nh[c] += p[c];
                tsum(fh[c], fl[c], pf32[c]);
            }
        }
        __syncthreads();
    }
    if (valid) {
        double* out = A.out + (int64_t)blockIdx.y * 6 * A.nt;
        for (int c = 0; c < 6; c++) out[(int64_t)c * A.nt + i] = nh[c] + ((double)fh[c] + (double)fl[c]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        pn += __shfl_xor_sync(0xffffffffu, pn, o);
        pf += __shfl_xor_sync(0xffffffffu, pf, o);
    }
    if ((tid & 31) == 0) {
        if (pn) atomicAdd(A.pairs, pn);
        if (pf) atomicAdd(A.pairs + 1, pf);
    }
}

__global__ void k_reduce6(const double* __restrict__ part, int nsplit, int nt, double* __restrict__ res)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    for (int c = 0; c < 6; c++) {
        double s = 0.0;
        for (int k = 0; k < nsplit; k++) s += part[((int64_t)k * 6 + c) * nt + i];
        res[(int64_t)c * nt + i] = s;
    }
}

bool g_hess_consts[64] = {false};

int hess_constants(Ctx* ctx)
{
    if (ctx->device >= 0 && ctx->device < 64 && g_hess_consts[ctx->device]) return LSM_OK;
    std::vector<double> tab((size_t)kH64N * 8, 0.0);
    for (int k = 0; k < kH64N; k++) {
        long double cf[7];
        h_interval_fit(k, kH64PerUnit, cf);
        for (int j = 0; j < 7; j++) tab[8 * (size_t)k + j] = (double)cf[j];
    }
    LSM_CUDA_TRY(ctx, cudaMemcpyToSymbol(g_htab64, tab.data(), sizeof(double) * tab.size()));
    // a copy from pageable memory may return before it lands, and nothing
    // orders it with kernels on the caller's (possibly non-blocking) stream
    LSM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (ctx->device >= 0 && ctx->device < 64) g_hess_consts[ctx->device] = true;
    return LSM_OK;
}

}  // namespace

int hess_sorted(Ctx* ctx, const Mesh* me, const Targets& t, double* res, cudaStream_t st)
{
    if (t.n <= 0) return LSM_OK;
    int rc = hess_constants(ctx);
    if (rc != LSM_OK) return rc;
    const int nblk = (t.n + kHessThreads - 1) / kHessThreads;
    const int ntiles = (int)me->ntiles;
    const int want = ctx->num_sms * 8;
    int nsplit = 1;
    if (nblk < want) nsplit = std::min((want + nblk - 1) / nblk, std::max(1, ntiles / 4));
    const int tps = (ntiles + nsplit - 1) / nsplit;
    nsplit = (ntiles + tps - 1) / tps;
    Scratch s(st);
    // a large mesh: the mixed path's treecode, walked for this kernel's radius
    int *list = nullptr, *border = nullptr;
    int2* blist = nullptr;
    const bool use_tree = tree_wanted(ctx, me, false);
    if (use_tree) {
        rc = tree_ensure(ctx, const_cast<Mesh*>(me), st, false);
        if (rc != LSM_OK) return rc;
        int64_t total = 0;
        rc = tree_lists(ctx, me->tree, t, kHessThreads, nullptr, s, &list, &blist, &border, &total, st,
                        ctx->opt.cutoff_fp64);
        if (rc != LSM_OK) return rc;
        nsplit = 1;
        const int64_t avg = total / nblk;
        if (nblk < want) nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((want + nblk - 1) / nblk, avg / 4));
    }
    double* part = res;
    if (nsplit > 1) LSM_CUDA_TRY(ctx, s.get(&part, (size_t)nsplit * 6 * t.n));
    HessArgs A;
    A.s32_pos = me->s32_pos;
    A.s32_nw = me->s32_nw;
    A.s64_pos = me->s64_pos;
    A.s64_nw = me->s64_nw;
    A.tlo = me->tile_lo;
    A.thi = me->tile_hi;
    A.tchi = me->tile_chi;
    A.tclo = me->tile_clo;
    A.ntiles = ntiles;
    A.tiles_per_split = tps;
    A.tx = t.x;
    A.ld = t.ld;
    A.nt = t.n;
    A.cut2 = (float)(ctx->opt.cutoff_fp64 * ctx->opt.cutoff_fp64);
    A.out = part;
    A.pairs = ctx->d_pairs + 6;
    A.list = nullptr;
    A.blist = nullptr;
    A.border = nullptr;
    A.ppos = A.pnw = nullptr;
    if (use_tree) {
        const Tree* T = me->tree;
        A.tlo = T->tile_lo;
        A.thi = T->tile_hi;
        A.tchi = T->tile_chi;
        A.tclo = T->tile_clo;
        A.list = list;
        A.blist = blist;
        A.border = border;
        A.ppos = T->p_pos;
        A.pnw = T->p_nw;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (ctx->profiling) {
        LSM_CUDA_TRY(ctx, cudaEventCreate(&ev0));
        LSM_CUDA_TRY(ctx, cudaEventCreate(&ev1));
        LSM_CUDA_TRY(ctx, cudaEventRecord(ev0, st));
    }
    k_eval_hess<<<dim3(nblk, nsplit), kHessThreads, 0, st>>>(A);
    LSM_LAUNCHED(ctx);
    if (ctx->profiling) {
        LSM_CUDA_TRY(ctx, cudaEventRecord(ev1, st));
        ctx->prof_events.push_back(Ctx::ProfEvent{ev0, ev1, 3});
    }
    if (nsplit > 1) {
        k_reduce6<<<(t.n + 255) / 256, 256, 0, st>>>(part, nsplit, t.n, res);
        LSM_LAUNCHED(ctx);
    }
    return LSM_OK;
}

}  // namespace lsm
