// frames.cu -- local coordinates of the solved charts and the Gauss flux
// check of their closure (Sec. 3.3 and Sec. 5).
//
// Chart j is x(u,v) = T(u,v) + h(u,v) H(u,v) (eq. chart) over the skeleton
// patch T(u,v) (the flat triangle of eq. tparam, or a quadratic patch), with
// H interpolated linearly from the vertex pseudonormals.  Newton gives h only at the rule
// points; its derivatives follow from x_u being tangent to the level set and
// grad Phi normal to it (x_u . grad Phi = 0):
//   h_u = -((T_u + h H_u) . grad Phi) / (H . grad Phi)         (eq. U_vector_2)
//   x_u = T_u + h H_u + h_u H                                    (eq. u_vector)
// the same in v (eq. v_vector, v_vector_2), and da = |x_u x x_v| du dv
// (eq. da).  The Gauss flux error
//   eps0 = 1 + sum over chart nodes of w_i |x_u x x_v| N . (x0 - x) / (4 pi |x0 - x|^3),
// N = -grad Phi / |grad Phi| the outward normal, is zero for a closed surface
// around x0 (Sec. 5).  Both are elementwise FP64 work over the chart nodes;
// the flux sum is reduced in a fixed order (per-block partials, then one
// block), so it is deterministic.
#include <algorithm>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kFrameThreads = 256;
constexpr double kFourPi = 12.566370614359172954;

// Triangle, parent (u, v) and weight of node s: from the rule shared by all
// triangles (s = j np + i), or given per node (tri, uvw).
__device__ __forceinline__ void node_of(int64_t s, int np, const double* rule, const int32_t* tri,
                                        const double* uvw, int64_t& j, double& u, double& v, double& w)
{
    if (tri) {
        j = tri[s];
        u = uvw[3 * s];
        v = uvw[3 * s + 1];
        w = uvw[3 * s + 2];
    } else {
        j = s / np;
        const int i = (int)(s - j * np);
        u = rule[3 * i];
        v = rule[3 * i + 1];
        w = rule[3 * i + 2];
    }
}

__global__ void k_chart_frames(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                               const int32_t* __restrict__ tris6, const double* __restrict__ vpn, int64_t n, int np,
                               const double* __restrict__ rule, const int32_t* __restrict__ tri,
                               const double* __restrict__ uvw, const double* __restrict__ h,
                               const double* __restrict__ g, double* __restrict__ xu, double* __restrict__ xv,
                               double* __restrict__ jac)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int64_t j;
    double u, v, wq;
    node_of(s, np, rule, tri, uvw, j, u, v, wq);
    const int a = tris[3 * j], b = tris[3 * j + 1], c = tris[3 * j + 2];
    double T[3], tu[3], tv[3], H[3], hu[3], hv[3], gs[3];
    patch_map(verts, tris, tris6, j, u, v, T, tu, tv);   // the patch's tangents at the node
    for (int k = 0; k < 3; k++) {
        const double n1 = vpn[3 * a + k];
        hu[k] = vpn[3 * b + k] - n1;
        hv[k] = vpn[3 * c + k] - n1;
        H[k] = n1 + u * hu[k] + v * hv[k];
        gs[k] = g[3 * s + k];
    }
    const double hs = h[s];
    double au[3], av[3];
    for (int k = 0; k < 3; k++) {
        au[k] = tu[k] + hs * hu[k];
        av[k] = tv[k] + hs * hv[k];
    }
    const double hg = H[0] * gs[0] + H[1] * gs[1] + H[2] * gs[2];
    const double h_u = -(au[0] * gs[0] + au[1] * gs[1] + au[2] * gs[2]) / hg;
    const double h_v = -(av[0] * gs[0] + av[1] * gs[1] + av[2] * gs[2]) / hg;
    double x1[3], x2[3];
    for (int k = 0; k < 3; k++) {
        x1[k] = au[k] + h_u * H[k];
        x2[k] = av[k] + h_v * H[k];
        xu[3 * s + k] = x1[k];
        xv[3 * s + k] = x2[k];
    }
    const double cx = x1[1] * x2[2] - x1[2] * x2[1];
    const double cy = x1[2] * x2[0] - x1[0] * x2[2];
    const double cz = x1[0] * x2[1] - x1[1] * x2[0];
    jac[s] = sqrt(cx * cx + cy * cy + cz * cz);
}

// Second derivatives of the charts and the curvatures of the level set at
// the nodes.  On a flat triangle with linear H (eq. uu_vector and its uv, vv
// analogues, T and H having no second derivatives):
//   x_uu = 2 h_u H_u + h_uu H,  x_uv = h_u H_v + h_v H_u + h_uv H,  x_vv = 2 h_v H_v + h_vv H,
// with h_uu, h_uv, h_vv from differentiating x_u . grad Phi = 0 once more
// (eq. uu_vector_aux1, uu_vector_aux2):
//   h_uu = -(x_u^T Hess x_u + 2 h_u H_u . grad Phi) / (H . grad Phi), etc.
// Then with N = -grad Phi/|grad Phi| (outward) and the fundamental forms
// E, F, G = x_u.x_u, x_u.x_v, x_v.x_v and L, M, Nn = x_uu.N, x_uv.N, x_vv.N:
//   kgauss = (L Nn - M^2)/(EG - F^2),  kmean = -(E Nn - 2 F M + G L)/(EG - F^2)
// (kmean the sum of the principal curvatures, 2/R on a sphere of radius R).
__global__ void k_chart_second(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                               const double* __restrict__ vpn, int64_t m, int np, const double* __restrict__ rule,
                               const double* __restrict__ h, const double* __restrict__ g,
                               const double* __restrict__ hess, double* __restrict__ xuu, double* __restrict__ xuv,
                               double* __restrict__ xvv, double* __restrict__ kmean, double* __restrict__ kgauss)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m * np) return;
    const int64_t j = s / np;
    const int i = (int)(s - j * np);
    const double u = rule[3 * i], v = rule[3 * i + 1];
    const int ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
    double tu[3], tv[3], H[3], hu[3], hv[3], gs[3];
    for (int k = 0; k < 3; k++) {
        const double p1 = verts[3 * ia + k], n1 = vpn[3 * ia + k];
        tu[k] = verts[3 * ib + k] - p1;
        tv[k] = verts[3 * ic + k] - p1;
        hu[k] = vpn[3 * ib + k] - n1;
        hv[k] = vpn[3 * ic + k] - n1;
        H[k] = n1 + u * hu[k] + v * hv[k];
        gs[k] = g[3 * s + k];
    }
    const double* Hs = hess + 6 * s;
    const double S[3][3] = {{Hs[0], Hs[1], Hs[2]}, {Hs[1], Hs[3], Hs[4]}, {Hs[2], Hs[4], Hs[5]}};
    auto dot = [](const double* p, const double* q) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; };
    const double hs = h[s];
    const double hg = dot(H, gs);
    double au[3], av[3], a[3], b[3];
    for (int k = 0; k < 3; k++) {
        au[k] = tu[k] + hs * hu[k];
        av[k] = tv[k] + hs * hv[k];
    }
    const double h_u = -dot(au, gs) / hg, h_v = -dot(av, gs) / hg;
    for (int k = 0; k < 3; k++) {
        a[k] = au[k] + h_u * H[k];
        b[k] = av[k] + h_v * H[k];
    }
    double Sa[3], Sb[3];
    for (int r = 0; r < 3; r++) {
        Sa[r] = S[r][0] * a[0] + S[r][1] * a[1] + S[r][2] * a[2];
        Sb[r] = S[r][0] * b[0] + S[r][1] * b[1] + S[r][2] * b[2];
    }
    const double huu = -(dot(a, Sa) + 2.0 * h_u * dot(hu, gs)) / hg;
    const double huv = -(dot(a, Sb) + h_u * dot(hv, gs) + h_v * dot(hu, gs)) / hg;
    const double hvv = -(dot(b, Sb) + 2.0 * h_v * dot(hv, gs)) / hg;
    double uu[3], uv[3], vv[3];
    for (int k = 0; k < 3; k++) {
        uu[k] = 2.0 * h_u * hu[k] + huu * H[k];
        uv[k] = h_u * hv[k] + h_v * hu[k] + huv * H[k];
        vv[k] = 2.0 * h_v * hv[k] + hvv * H[k];
        xuu[3 * s + k] = uu[k];
        xuv[3 * s + k] = uv[k];
        xvv[3 * s + k] = vv[k];
    }
    const double gn = sqrt(dot(gs, gs));
    const double N[3] = {-gs[0] / gn, -gs[1] / gn, -gs[2] / gn};
    const double E = dot(a, a), F = dot(a, b), G = dot(b, b);
    const double L = dot(uu, N), M = dot(uv, N), Nn = dot(vv, N);
    const double det = E * G - F * F;
    kgauss[s] = (L * Nn - M * M) / det;
    kmean[s] = -(E * Nn - 2.0 * F * M + G * L) / det;
}

// One node's term of the Gauss flux about x0: w jac N . (x0 - x) / (4 pi |x0 - x|^3),
// N = -grad Phi / |grad Phi|.
__device__ __forceinline__ double flux_term(const double* __restrict__ x, const double* __restrict__ g,
                                            const double* __restrict__ jac, int64_t s, double wq, double x0, double y0,
                                            double z0)
{
    const double dx = x0 - x[3 * s], dy = y0 - x[3 * s + 1], dz = z0 - x[3 * s + 2];
    const double gx = g[3 * s], gy = g[3 * s + 1], gz = g[3 * s + 2];
    const double gn = sqrt(gx * gx + gy * gy + gz * gz);
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double r = sqrt(r2);
    const double nd = -(gx * dx + gy * dy + gz * dz) / gn;
    return wq * jac[s] * nd / (kFourPi * r2 * r);
}

// Per-triangle sums of the flux terms: triangle j's nodes are [off[j], off[j+1])
// (nodes grouped by triangle), summed in node order by one thread.
__global__ void k_flux_tri(const double* __restrict__ x, const double* __restrict__ g, const double* __restrict__ jac,
                           const double* __restrict__ uvw, const int64_t* __restrict__ off, int64_t m, double x0,
                           double y0, double z0, double* __restrict__ out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double a = 0.0;
    for (int64_t s = off[j]; s < off[j + 1]; s++) a += flux_term(x, g, jac, s, uvw[3 * s + 2], x0, y0, z0);
    out[j] = a;
}

// Per-block partial sums of the flux terms (block sums in a fixed tree order).
__global__ void __launch_bounds__(kFrameThreads) k_flux_partial(const double* __restrict__ x,
                                                                const double* __restrict__ g,
                                                                const double* __restrict__ jac, int64_t n, int np,
                                                                const double* __restrict__ rule,
                                                                const double* __restrict__ uvw, double x0, double y0,
                                                                double z0, double* __restrict__ part)
{
    __shared__ double sw[kFrameThreads / 32];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double t = 0.0;
    if (s < n) t = flux_term(x, g, jac, s, uvw ? uvw[3 * s + 2] : rule[3 * (s % np) + 2], x0, y0, z0);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < kFrameThreads / 32; k++) a += sw[k];
        part[blockIdx.x] = a;
    }
}

// One block: the partials in index order, then 1 + sum.
__global__ void __launch_bounds__(kFrameThreads) k_flux_final(const double* __restrict__ part, int nb,
                                                              double* __restrict__ out)
{
    __shared__ double sw[kFrameThreads];
    double a = 0.0;
    const int per = (nb + kFrameThreads - 1) / kFrameThreads;
    const int lo = threadIdx.x * per, hi = min(nb, lo + per);
    for (int k = lo; k < hi; k++) a += part[k];
    sw[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kFrameThreads; k++) t += sw[k];
        *out = 1.0 + t;
    }
}

int upload_rule(Ctx* ctx, Scratch& s, int n_gl, double** rule, cudaStream_t st)
{
    const int np = n_gl * n_gl;
    std::vector<double> r(3 * (size_t)np);
    simplex_rule_host(n_gl, 0, r.data());
    LSM_CUDA_TRY(ctx, s.get(rule, r.size()));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(*rule, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, st));
    // the host vector must outlive the copy
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

}  // namespace

int chart_frames_dev(Ctx* ctx, const Mesh* me, int n_gl, const double* h, const double* g, double* xu, double* xv,
                     double* jac, cudaStream_t st, const NodeSpec* spec)
{
    Scratch s(st);
    double* rule = nullptr;
    int rc = upload_rule(ctx, s, std::max(1, n_gl), &rule, st);
    if (rc) return rc;
    const int np = n_gl * n_gl;
    const int64_t n = spec ? spec->n : me->m * np;
    if (n == 0) return LSM_OK;
    k_chart_frames<<<(unsigned)((n + kFrameThreads - 1) / kFrameThreads), kFrameThreads, 0, st>>>(
        me->verts, me->tris, me->tris6, me->vpn, n, np, rule, spec ? spec->tri : nullptr, spec ? spec->uvw : nullptr, h,
        g, xu, xv, jac);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

int chart_second_dev(Ctx* ctx, const Mesh* me, int n_gl, const double* h, const double* g, const double* hess,
                     double* xuu, double* xuv, double* xvv, double* kmean, double* kgauss, cudaStream_t st)
{
    Scratch s(st);
    double* rule = nullptr;
    int rc = upload_rule(ctx, s, n_gl, &rule, st);
    if (rc) return rc;
    const int np = n_gl * n_gl;
    const int64_t n = me->m * np;
    if (n == 0) return LSM_OK;
    k_chart_second<<<(unsigned)((n + kFrameThreads - 1) / kFrameThreads), kFrameThreads, 0, st>>>(
        me->verts, me->tris, me->vpn, me->m, np, rule, h, g, hess, xuu, xuv, xvv, kmean, kgauss);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

int gauss_flux_dev(Ctx* ctx, const Mesh* me, int n_gl, const double* x, const double* g, const double* jac,
                   const double* x0, double* eps0, cudaStream_t st, const NodeSpec* spec)
{
    Scratch s(st);
    double* rule = nullptr;
    int rc = upload_rule(ctx, s, std::max(1, n_gl), &rule, st);
    if (rc) return rc;
    const int np = n_gl * n_gl;
    const int64_t n = spec ? spec->n : me->m * np;
    const int nb = (int)((n + kFrameThreads - 1) / kFrameThreads);
    double *part = nullptr, *out = nullptr;
    LSM_CUDA_TRY(ctx, s.get(&part, std::max(1, nb)));
    LSM_CUDA_TRY(ctx, s.get(&out, 1));
    if (nb > 0) {
        k_flux_partial<<<nb, kFrameThreads, 0, st>>>(x, g, jac, n, np, rule, spec ? spec->uvw : nullptr, x0[0], x0[1],
                                                     x0[2], part);
        LSM_LAUNCHED(ctx);
    }
    k_flux_final<<<1, kFrameThreads, 0, st>>>(part, nb, out);
    LSM_LAUNCHED(ctx);
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(eps0, out, sizeof(double), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

int flux_per_triangle_dev(Ctx* ctx, int64_t m, const int64_t* off, const double* x, const double* g, const double* jac,
                          const double* uvw, const double* x0, double* out, cudaStream_t st)
{
    if (m <= 0) return LSM_OK;
    k_flux_tri<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(x, g, jac, uvw, off, m, x0[0], x0[1], x0[2], out);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace lsm
