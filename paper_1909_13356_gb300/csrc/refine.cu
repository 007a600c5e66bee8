// refine.cu -- a posteriori refinement of the charts (Sec. 3.4) and the
// per-triangle Gauss flux it is driven by.
//
// The paper refines a skeleton triangle 1 -> 4 at its edge midpoints where
// refinement is wanted and leaves the choice to standard a posteriori
// estimates from adaptive interpolation or integration.  The estimate used
// here is one from adaptive integration: the Gauss flux integral about an
// interior point x0 over the charts of triangle j,
//     S_j(L) = sum over the chart nodes of j's 4^L children of w jac N . (x0 - x) / (4 pi |x0 - x|^3),
// with N = -grad Phi/|grad Phi|, is compared with the same integral one level
// finer.  The integrand is smooth over a well-resolved chart, so the two
// agree to the chart rule's accuracy; a difference above the tolerance marks
// the triangle as under-resolved there.  Such triangles are refined (their
// level raised by one) and tested again one level further, up to a maximum
// level; the others keep their level.  Charts of the children keep the
// parent's map (lsm_refined_nodes), so a mixture of levels stays continuous.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lsm_internal.cuh"

using namespace lsm;

namespace lsm {
namespace {

// Nodes (triangle, parent u, v, weight) of the listed triangles at the given
// levels, grouped by triangle in list order; off [k + 1] node offsets.
void refined_node_set(int n_gl, const std::vector<int64_t>& tris, const std::vector<int>& level,
                      std::vector<int32_t>& tri, std::vector<double>& uvw, std::vector<int64_t>& off)
{
    tri.clear();
    uvw.clear();
    off.assign(1, 0);
    std::vector<std::vector<double>> rules(6);
    for (size_t k = 0; k < tris.size(); k++) {
        const int L = level[k];
        std::vector<double>& r = rules[L];
        if (r.empty()) {
            r.resize((size_t)n_gl * n_gl * ((size_t)1 << (2 * L)) * 3);
            simplex_rule_host(n_gl, L, r.data());
        }
        const size_t cnt = r.size() / 3;
        for (size_t i = 0; i < cnt; i++) tri.push_back((int32_t)tris[k]);
        uvw.insert(uvw.end(), r.begin(), r.end());
        off.push_back(off.back() + (int64_t)cnt);
    }
}

// Charts at the nodes of the listed triangles at the given levels, then their
// per-triangle flux sums (host out [k]).
int flux_of_levels(Ctx* ctx, lsm_mesh* mh, int n_gl, double tol, const std::vector<int64_t>& tris,
                   const std::vector<int>& level, const double* x0, std::vector<double>& out, int* failed,
                   cudaStream_t st)
{
    Mesh* me = &mh->m;
    std::vector<int32_t> tri;
    std::vector<double> uvw;
    std::vector<int64_t> off;
    refined_node_set(n_gl, tris, level, tri, uvw, off);
    const int64_t n = (int64_t)tri.size();
    out.assign(tris.size(), 0.0);
    if (n == 0) return LSM_OK;
    Scratch s(st);
    int32_t *d_tri, *d_st;
    double *d_uvw, *d_x, *d_h, *d_phi, *d_g, *d_xu, *d_xv, *d_jac, *d_out;
    int64_t* d_off;
    LSM_CUDA_TRY(ctx, s.get(&d_tri, (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_st, (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_uvw, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_x, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_h, (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_phi, (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_g, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_xu, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_xv, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_jac, (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&d_out, tris.size()));
    LSM_CUDA_TRY(ctx, s.get(&d_off, off.size()));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(d_tri, tri.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(d_uvw, uvw.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st));
    NodeSpec spec{n, d_tri, d_uvw};
    lsm_solve_stats stats;
    int rc = solve_charts_device(ctx, me, 1, tol, 20, LSM_MIXED, d_x, d_h, d_st, &stats, st, &spec);
    if (rc) return rc;
    *failed += stats.n_failed;
    rc = lsm_eval_phi_grad(mh, d_x, n, d_phi, d_g, LSM_FF, st);
    if (rc) return rc;
    rc = chart_frames_dev(ctx, me, 1, d_h, d_g, d_xu, d_xv, d_jac, st, &spec);
    if (rc) return rc;
    rc = flux_per_triangle_dev(ctx, (int64_t)tris.size(), d_off, d_x, d_g, d_jac, d_uvw, x0, d_out, st);
    if (rc) return rc;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(out.data(), d_out, sizeof(double) * tris.size(), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

}  // namespace
}  // namespace lsm

extern "C" {

int lsm_flux_per_triangle(lsm_mesh* mh, int64_t n, const int32_t* tri, const double* uvw, const double* x,
                          const double* grad, const double* jac, const double* x0, double* out, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (n < 0 || !tri || !uvw || !x || !grad || !jac || !x0 || !out) {
        ctx->err = "flux_per_triangle: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "flux_per_triangle: cudaSetDevice failed";
        return LSM_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = LSM_OK;
    do {
        // node offsets per triangle on the host; nodes must come grouped by
        // triangle in increasing triangle order
        std::vector<int32_t> ht((size_t)n);
        cudaPointerAttributes a;
        const bool tdev = cudaPointerGetAttributes(&a, tri) == cudaSuccess &&
                          (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        if (n > 0 && cudaMemcpy(ht.data(), tri, sizeof(int32_t) * n, tdev ? cudaMemcpyDeviceToHost
                                                                          : cudaMemcpyHostToHost) != cudaSuccess) {
            ctx->err = "flux_per_triangle: copy failed";
            rc = LSM_E_CUDA;
            break;
        }
        std::vector<int64_t> off((size_t)me->m + 1, 0);
        for (int64_t s = 0; s < n; s++) {
            if (ht[s] < 0 || ht[s] >= me->m || (s > 0 && ht[s] < ht[s - 1])) {
                ctx->err = "flux_per_triangle: nodes must be grouped by triangle in increasing order";
                rc = LSM_E_INVALID_ARG;
                break;
            }
            off[(size_t)ht[s] + 1]++;
        }
        if (rc) break;
        for (int64_t j = 0; j < me->m; j++) off[j + 1] += off[j];
        Scratch s(st);
        int64_t* d_off;
        const double *dx, *dg, *dj, *du;
        double* d_out;
        auto to_dev = [&](const double* p, size_t cnt, const double** o) -> int {
            cudaPointerAttributes pa;
            const bool dev = cudaPointerGetAttributes(&pa, p) == cudaSuccess &&
                             (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            if (dev) {
                *o = p;
                return LSM_OK;
            }
            double* d;
            if (s.get(&d, cnt) != cudaSuccess ||
                cudaMemcpyAsync(d, p, sizeof(double) * cnt, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return LSM_E_CUDA;
            *o = d;
            return LSM_OK;
        };
        if (s.get(&d_off, off.size()) != cudaSuccess || s.get(&d_out, (size_t)me->m) != cudaSuccess ||
            cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            to_dev(x, 3 * (size_t)n, &dx) || to_dev(grad, 3 * (size_t)n, &dg) || to_dev(jac, (size_t)n, &dj) ||
            to_dev(uvw, 3 * (size_t)n, &du)) {
            ctx->err = "flux_per_triangle: device copies failed";
            rc = LSM_E_CUDA;
            break;
        }
        rc = flux_per_triangle_dev(ctx, me->m, d_off, dx, dg, dj, du, x0, d_out, st);
        if (rc) break;
        if (cudaMemcpyAsync(out, d_out, sizeof(double) * me->m, cudaMemcpyDefault, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            ctx->err = "flux_per_triangle: copy back failed";
            rc = LSM_E_CUDA;
        }
    } while (false);
    cudaSetDevice(prev);
    cudaGetLastError();
    return rc;
}

int lsm_refine_adaptive(lsm_mesh* mh, int order, double newton_tol, double flux_tol, int max_level,
                        const double* x0, int32_t* level_out, int* rounds_out, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (order < 0 || order > 40 || !(newton_tol > 0) || !(flux_tol > 0) || max_level < 0 || max_level > 4 || !x0 ||
        !level_out) {
        ctx->err = "refine_adaptive: bad arguments (max_level 0..4)";
        return LSM_E_INVALID_ARG;
    }
    if (me->sigx) {
        ctx->err = "refine_adaptive: meshes with a target-dependent sigma are not supported";
        return LSM_E_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "refine_adaptive: cudaSetDevice failed";
        return LSM_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n_gl = order / 2 + 2;
    const int64_t m = me->m;
    std::vector<int> level((size_t)m, 0);
    std::vector<char> done((size_t)m, 0);
    std::vector<int64_t> all((size_t)m);
    for (int64_t j = 0; j < m; j++) all[j] = j;
    std::vector<double> cur;
    int failed = 0, rounds = 0;
    int rc = flux_of_levels(ctx, mh, n_gl, newton_tol, all, level, x0, cur, &failed, st);
    while (rc == LSM_OK) {
        // the triangles still open, one level finer
        std::vector<int64_t> cand;
        std::vector<int> lv;
        for (int64_t j = 0; j < m; j++)
            if (!done[j] && level[j] < max_level) {
                cand.push_back(j);
                lv.push_back(level[j] + 1);
            }
        if (cand.empty()) break;
        std::vector<double> fine;
        rc = flux_of_levels(ctx, mh, n_gl, newton_tol, cand, lv, x0, fine, &failed, st);
        if (rc) break;
        rounds++;
        for (size_t k = 0; k < cand.size(); k++) {
            const int64_t j = cand[k];
            if (std::fabs(fine[k] - cur[j]) <= flux_tol) {
                done[j] = 1;            // level[j] resolves the flux to the tolerance
            } else {
                level[j] += 1;          // refine, and test the next level
                cur[j] = fine[k];
            }
        }
    }
    if (rc == LSM_OK) rc = check_flag(ctx, st);
    if (rc == LSM_OK) {
        for (int64_t j = 0; j < m; j++) level_out[j] = level[j];
        if (rounds_out) *rounds_out = rounds;
        if (failed) {
            ctx->err = "refine_adaptive: " + std::to_string(failed) + " chart nodes did not converge";
            rc = LSM_E_NOT_CONVERGED;
        }
    }
    cudaSetDevice(prev);
    cudaGetLastError();
    return rc;
}

}  // extern "C"
