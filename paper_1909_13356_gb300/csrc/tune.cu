// tune.cu -- autotuner of the mixed path's far field.
//
// The paper runs its FMM at one fixed precision (Sec. 4.4).  Here the far
// field of the mixed path is either the direct tiled sum or the treecode,
// and the treecode's speed and error depend on its Chebyshev degree and
// opening parameter in a way that varies with the mesh (grading, curvature,
// size) and with the density of the targets.  The tuner measures instead of
// modelling: on a sample of the caller's targets it times every candidate
// with CUDA events and compares its Phi with the float-float path (the
// direct sum to FP64 accuracy), then keeps the fastest candidate within the
// error budget.  The sample is a few windows of consecutive Morton-sorted
// targets, so its blocks of targets are as compact as in the full workload
// and a candidate's interaction lists (and cost per target) are the ones it
// would have there.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kTuneWindow = 4096;   // targets per window (16 blocks of the mixed kernel)
constexpr int kTuneWindows = 8;

struct Candidate {
    int mode;      // 0 direct, 1 treecode
    int degree;
    float theta;
};
const Candidate kCandidates[] = {
    {0, 0, 0.0f},    {1, 5, 0.35f},  {1, 6, 0.4f},  {1, 6, 0.45f},  {1, 7, 0.4f},
    {1, 7, 0.45f},   {1, 7, 0.5f},   {1, 8, 0.45f}, {1, 8, 0.5f},   {1, 10, 0.55f},
};

// max |a - b| over n entries, as the bit pattern of a non-negative double
// (ordered like the values)
__global__ void k_max_abs_diff(const double* __restrict__ a, const double* __restrict__ b, int n,
                               unsigned long long* __restrict__ out)
{
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = fabs(a[i] - b[i]);
        m = d > m || d != d ? d : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v > m || v != v ? v : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

int max_abs_diff(Ctx* ctx, const double* a, const double* b, int n, unsigned long long* d_word, double* out,
                 cudaStream_t st)
{
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(d_word, 0, sizeof(unsigned long long), st));
    k_max_abs_diff<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(a, b, n, d_word);
    LSM_LAUNCHED(ctx);
    unsigned long long w = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&w, d_word, sizeof(w), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    double v;
    std::memcpy(&v, &w, sizeof(v));
    *out = v;
    return LSM_OK;
}

}  // namespace

// The mixed kernel's near-field radii the tuner tries (in sigma).  A pair
// beyond radius c uses the Laplace double layer; the relative difference of
// the smoothed kernel from it there is erfc(c/sqrt2) + c sqrt(2/pi)
// e^{-c^2/2} (the gradient part; Sec. 4.4's bound without the factor the
// paper drops), and only radii where it is at most kCutBound are tried.
const double kCutCandidates[] = {6.4, 6.5, 7.0};
constexpr double kCutBound = 1e-8;
static double cutoff_bound(double c)
{
    return std::erfc(c / std::sqrt(2.0)) + c * std::sqrt(2.0 / 3.14159265358979323846) * std::exp(-0.5 * c * c);
}

int autotune_sorted(Ctx* ctx, Mesh* me, const Targets& t, double budget, lsm_tune_result* res, cudaStream_t st)
{
    // the sample: windows of consecutive sorted targets, evenly spread
    const int win = std::min(kTuneWindow, t.n);
    const int nw = std::max(1, std::min(kTuneWindows, t.n / std::max(1, win)));
    const int m = nw * win;
    Scratch s(st);
    double *S = nullptr, *Rref = nullptr, *R = nullptr;
    unsigned long long* word = nullptr;
    LSM_CUDA_TRY(ctx, s.get(&S, 3 * (size_t)m));
    LSM_CUDA_TRY(ctx, s.get(&Rref, 4 * (size_t)m));
    LSM_CUDA_TRY(ctx, s.get(&R, 4 * (size_t)m));
    LSM_CUDA_TRY(ctx, s.get(&word, 1));
    for (int w = 0; w < nw; w++) {
        const int64_t off = nw > 1 ? (int64_t)(t.n - win) * w / (nw - 1) : 0;
        for (int c = 0; c < 3; c++)
            LSM_CUDA_TRY(ctx, cudaMemcpyAsync(S + (size_t)c * m + (size_t)w * win, t.x + c * t.ld + off,
                                              sizeof(double) * win, cudaMemcpyDeviceToDevice, st));
    }
    Targets ts{S, m, m};
    int rc = eval_sorted(ctx, me, ts, Rref, LSM_FF, st);
    if (rc != LSM_OK) return rc;

    cudaEvent_t e0, e1;
    LSM_CUDA_TRY(ctx, cudaEventCreate(&e0));
    LSM_CUDA_TRY(ctx, cudaEventCreate(&e1));
    struct Meas {
        Candidate c;
        double ms, err;
    };
    std::vector<Meas> meas;
    const int saved_mode = me->tune_mode, saved_deg = me->tune_degree, saved_tpb = me->tune_tpb;
    const float saved_theta = me->tune_theta;
    const double saved_cut = me->tune_cut;
    me->tune_cut = 0.0;   // the far field is chosen at the default radius and tile
    me->tune_tpb = 0;
    for (const Candidate& c : kCandidates) {
        me->tune_mode = c.mode;
        me->tune_degree = c.degree;
        me->tune_theta = c.theta;
        // the first evaluation builds the candidate's tree; the second is timed
        rc = eval_sorted(ctx, me, ts, R, LSM_MIXED, st);
        if (rc == LSM_OK) {
            cudaEventRecord(e0, st);
            rc = eval_sorted(ctx, me, ts, R, LSM_MIXED, st);
            cudaEventRecord(e1, st);
        }
        if (rc != LSM_OK) break;
        double err = 0.0;
        rc = max_abs_diff(ctx, R, Rref, m, word, &err, st);
        if (rc != LSM_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        meas.push_back(Meas{c, (double)ms, err});
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LSM_OK) {
        me->tune_mode = saved_mode;
        me->tune_degree = saved_deg;
        me->tune_theta = saved_theta;
        me->tune_cut = saved_cut;
        me->tune_tpb = saved_tpb;
        return rc;
    }
    // fastest within the budget; else the most accurate
    int best = -1;
    for (int i = 0; i < (int)meas.size(); i++)
        if (meas[i].err <= budget && (best < 0 || meas[i].ms < meas[best].ms)) best = i;
    if (best < 0) {
        best = 0;
        for (int i = 1; i < (int)meas.size(); i++)
            if (meas[i].err < meas[best].err) best = i;
    }
    const Candidate& c = meas[best].c;
    me->tune_mode = c.mode;
    me->tune_degree = c.degree;
    me->tune_theta = c.theta;
    if (c.mode == 1) {
        rc = tree_ensure(ctx, me, st, false);
        if (rc != LSM_OK) return rc;
    }
    // second stage, with that far field: the near-field radius (among the
    // values whose neglected kernel difference stays within the mixed path's
    // bound, Sec. 4.4) and the targets per CTA of the mixed kernel
    double best_ms = meas[best].ms, best_err = meas[best].err;
    double best_cut = 0.0;
    int best_tpb = 0;
    int stage2 = 0;
    {
        cudaEvent_t f0, f1;
        LSM_CUDA_TRY(ctx, cudaEventCreate(&f0));
        LSM_CUDA_TRY(ctx, cudaEventCreate(&f1));
        for (double cut : kCutCandidates) {
            if (cutoff_bound(cut) > kCutBound) continue;
            for (int tpb : {64, kEvalThreads, 2 * kEvalThreads}) {
                me->tune_cut = cut;
                me->tune_tpb = tpb;
                rc = eval_sorted(ctx, me, ts, R, LSM_MIXED, st);   // warm: lists and launch shapes
                if (rc == LSM_OK) {
                    cudaEventRecord(f0, st);
                    rc = eval_sorted(ctx, me, ts, R, LSM_MIXED, st);
                    cudaEventRecord(f1, st);
                }
                double err = 0.0;
                if (rc == LSM_OK) rc = max_abs_diff(ctx, R, Rref, m, word, &err, st);
                if (rc != LSM_OK) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, f0, f1);
                stage2++;
                if (err <= budget && ms < best_ms) {
                    best_ms = ms;
                    best_err = err;
                    best_cut = cut;
                    best_tpb = tpb;
                }
            }
            if (rc != LSM_OK) break;
        }
        cudaEventDestroy(f0);
        cudaEventDestroy(f1);
        if (rc != LSM_OK) return rc;
    }
    me->tune_cut = best_cut;
    me->tune_tpb = best_tpb;
    if (res) {
        res->use_tree = c.mode;
        res->tree_degree = c.degree;
        res->tree_theta = c.theta;
        res->candidates = (int32_t)meas.size() + stage2;
        res->sample_targets = m;
        res->err_phi = best_err;
        res->ms_sample = best_ms;
        res->ms_direct = meas[0].ms;
        res->err_direct = meas[0].err;
        res->cutoff = mixed_cut(ctx, me);
        res->targets_per_block = mixed_tpb(ctx, me);
    }
    return LSM_OK;
}

namespace {

// mesh of the node at sorted position k (nodes are triangle-major, np per triangle)
__global__ void k_tune_node_mesh(const int32_t* __restrict__ tri_mesh, int np, int n,
                                 const uint32_t* __restrict__ perm, uint32_t* __restrict__ key,
                                 int32_t* __restrict__ mesh_sorted)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int32_t m = tri_mesh[perm[k] / np];
    if (key) key[k] = (uint32_t)m;
    if (mesh_sorted) mesh_sorted[k] = m;
}

__global__ void k_tune_sample_flags(const int32_t* __restrict__ mesh_sorted, int n, int stride,
                                    int32_t* __restrict__ flags)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flags[k] = mesh_sorted[k] % stride == 0 ? 1 : 0;
}

// T (SoA, stride ld) = the starting points of the listed nodes
__global__ void k_tune_gather(const int32_t* __restrict__ L, int n, const uint32_t* __restrict__ perm,
                              const double* __restrict__ x0, int64_t ld, double* __restrict__ T)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm[L[k]];
    for (int c = 0; c < 3; c++) T[c * ld + k] = x0[3 * i + c];
}

inline unsigned nbk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// Autotuner of a batch's mixed kernel (lsm_batch_autotune): on the chart
// nodes' starting points of a sample of the batch's meshes (every stride-th
// mesh, about 64 of them), in the same work items the batched solve uses,
// the mixed evaluation is timed for every near-field radius and target tile
// and compared with the float-float evaluation; the fastest within the
// budget is kept for the batch's solves.  Batches use the direct far field
// (their meshes are below the treecode threshold), so the treecode's degree
// and opening parameter, the mesh autotuner's first stage, do not apply.
int batch_autotune(Ctx* ctx, Batch* b, int n_gl, double budget, lsm_tune_result* res, cudaStream_t st)
{
    const int np = n_gl * n_gl;
    const int64_t N64 = b->m * (int64_t)np;
    if (N64 <= 0 || N64 >= ((int64_t)1 << 31) - 1024) {
        ctx->err = "batch autotune: node count out of range";
        return LSM_E_INVALID_ARG;
    }
    const int N = (int)N64;
    Scratch s(st);
    std::vector<double> rule((size_t)np * 3);
    simplex_rule_host(n_gl, 0, rule.data());
    double *rule_d, *x0a, *hda, *sla;
    LSM_CUDA_TRY(ctx, s.get(&rule_d, rule.size()));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(rule_d, rule.data(), sizeof(double) * rule.size(), cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, s.get(&x0a, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&hda, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&sla, (size_t)N));
    int rc = chart_nodes_raw(ctx, b->verts, b->tris, b->vpn, b->tri_sigma, b->m, rule_d, np, x0a, hda, sla, st);
    if (rc) return rc;
    // the solve's order: mesh, then Morton
    uint32_t *perm, *key;
    int32_t *mesh_sorted, *flags, *L;
    int* cnts;
    LSM_CUDA_TRY(ctx, s.get(&perm, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&key, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&mesh_sorted, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&flags, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&L, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&cnts, 4));
    rc = morton_order_points(ctx, x0a, 3, N, perm, st);
    if (rc) return rc;
    k_tune_node_mesh<<<nbk(N), 256, 0, st>>>(b->tri_mesh, np, N, perm, key, nullptr);
    LSM_LAUNCHED(ctx);
    int bits = 1;
    while ((1 << bits) < b->nmesh) bits++;
    rc = radix_sort_pairs(ctx, key, perm, N, bits, st);
    if (rc) return rc;
    k_tune_node_mesh<<<nbk(N), 256, 0, st>>>(b->tri_mesh, np, N, perm, nullptr, mesh_sorted);
    LSM_LAUNCHED(ctx);
    const int stride = std::max(1, b->nmesh / 64);
    k_tune_sample_flags<<<nbk(N), 256, 0, st>>>(mesh_sorted, N, stride, flags);
    LSM_LAUNCHED(ctx);
    rc = compact_flags(ctx, flags, 1, nullptr, N, L, cnts, st);
    if (rc) return rc;
    int32_t nL = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&nL, cnts, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (nL <= 0) {
        ctx->err = "batch autotune: empty sample";
        return LSM_E_INVALID_ARG;
    }
    double *T, *Rref, *R;
    LSM_CUDA_TRY(ctx, s.get(&T, 3 * (size_t)nL));
    LSM_CUDA_TRY(ctx, s.get(&Rref, 4 * (size_t)nL));
    LSM_CUDA_TRY(ctx, s.get(&R, 4 * (size_t)nL));
    k_tune_gather<<<nbk(nL), 256, 0, st>>>(L, nL, perm, x0a, nL, T);
    LSM_LAUNCHED(ctx);
    const int max_items = nL / 64 + b->nmesh + 1;   // the smallest work item has 64 targets
    int4* items;
    int* n_items;
    uint32_t *cnt, *nblk;
    unsigned long long* word;
    LSM_CUDA_TRY(ctx, s.get(&items, (size_t)max_items));
    LSM_CUDA_TRY(ctx, s.get(&n_items, 1));
    LSM_CUDA_TRY(ctx, s.get(&cnt, 2 * (size_t)b->nmesh));
    LSM_CUDA_TRY(ctx, s.get(&nblk, (size_t)b->nmesh));
    LSM_CUDA_TRY(ctx, s.get(&word, 1));
    const SourceView view = view_of_batch(b);
    Targets tg{T, nL, nL};
    auto evaluate = [&](int prec, int tpb, double cut, double* out) -> int {
        const int bs = eval_item_targets(ctx, prec, tpb);
        int r = build_items(ctx, L, cnts, nL, mesh_sorted, b->mesh_tiles, b->nmesh, bs, cnt, nblk, items, n_items,
                            max_items, st);
        if (r) return r;
        return eval_items(ctx, view, tg, items, n_items, nL / bs + b->nmesh + 1, out, prec, st, nullptr, tpb, cut);
    };
    rc = evaluate(LSM_FF, 0, 0.0, Rref);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    LSM_CUDA_TRY(ctx, cudaEventCreate(&e0));
    LSM_CUDA_TRY(ctx, cudaEventCreate(&e1));
    double best_ms = 1e300, best_err = 0.0, best_cut = 0.0, def_ms = 0.0, def_err = 0.0;
    int best_tpb = 0, tried = 0;
    for (double cut : kCutCandidates) {
        if (cutoff_bound(cut) > kCutBound) continue;
        for (int tpb : {64, 128, 256}) {
            rc = evaluate(LSM_MIXED, tpb, cut, R);   // warm
            if (rc == LSM_OK) {
                cudaEventRecord(e0, st);
                rc = evaluate(LSM_MIXED, tpb, cut, R);
                cudaEventRecord(e1, st);
            }
            double err = 0.0;
            if (rc == LSM_OK) rc = max_abs_diff(ctx, R, Rref, nL, word, &err, st);
            if (rc != LSM_OK) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            tried++;
            if (tpb == 64 && std::fabs(cut - ctx->opt.cutoff_mixed) < 1e-12) {   // the default settings
                def_ms = ms;
                def_err = err;
            }
            if (err <= budget && ms < best_ms) {
                best_ms = ms;
                best_err = err;
                best_cut = cut;
                best_tpb = tpb;
            }
        }
        if (rc != LSM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LSM_OK) return rc;
    if (best_tpb == 0) {   // nothing within the budget: keep the defaults
        best_cut = 0.0;
        best_ms = def_ms;
        best_err = def_err;
    }
    b->cut_mixed = best_cut;
    b->tpb = best_tpb;
    if (res) {
        res->use_tree = 0;
        res->tree_degree = 0;
        res->tree_theta = 0.0f;
        res->candidates = tried;
        res->sample_targets = nL;
        res->err_phi = best_err;
        res->ms_sample = best_ms;
        res->ms_direct = def_ms;
        res->err_direct = def_err;
        res->cutoff = best_cut > 0.0 ? best_cut : ctx->opt.cutoff_mixed;
        res->targets_per_block = eval_item_targets(ctx, LSM_MIXED, best_tpb);
        res->reserved = 0;
    }
    return LSM_OK;
}

}  // namespace lsm
