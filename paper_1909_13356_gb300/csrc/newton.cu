// newton.cu -- batched Newton solve for chart nodes on Phi = 1/2
// (Sec. 3.2, eq. newton, newtonderiv, newtoneq).
//
// Every chart node i carries x0 = T^j(u_i, v_i), its pseudonormal direction
// H = H^j(u_i, v_i) (eq. mkpseudovec), sigma_j and h (h = 0 at start).  A
// sweep evaluates Phi and grad Phi at x = x0 + h H for the active nodes and
// applies h <- h - (Phi - 1/2)/(H . grad Phi), each step clamped to
// 4 sigma_j.  A node stops when |Phi - 1/2| < tol (converged), when the
// derivative vanishes or is not finite, or after max_iter evaluations.
// Stopped nodes leave the active list (Sec. 5), which is compacted stably
// so that it keeps the Morton order the nodes were sorted into once.
//
// Mixed precision: nodes start on the FP32 pair kernels; a node whose
// residual falls below opt.mixed_switch moves to the float-float kernel
// (Phi to FP64 accuracy on the FP32 pipes) for its last steps, unless the
// requested tolerance is one the FP32 kernels already meet (opt.mixed_accept).
#include <algorithm>
#include <cstring>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kPending = -1;

struct NodeState {
    double* x0;    // SoA [3][n]
    double* hd;    // SoA [3][n]
    double* sl;    // [n]
    double* h;     // [n]
    double* dh;    // [n] last |step|
    double* res;   // [n] last |Phi - 1/2|
    int32_t* st;   // [n] status (kPending while active)
    int32_t* it;   // [n] evaluations so far
    int32_t* mode; // [n] 0 = mixed kernels, 1 = FP64 kernels
    int32_t* clamp;// [n] 1 once a step was clamped
    int64_t n;
};

__global__ void k_sort_state(const double* __restrict__ x0a, const double* __restrict__ hda,
                             const double* __restrict__ sla, const uint32_t* __restrict__ perm, int n,
                             NodeState S, int mode0)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = (int)perm[k];
    for (int c = 0; c < 3; c++) {
        S.x0[c * S.n + k] = x0a[3 * (int64_t)i + c];
        S.hd[c * S.n + k] = hda[3 * (int64_t)i + c];
    }
    S.sl[k] = sla[i];
    S.h[k] = 0.0;
    S.dh[k] = 0.0;
    S.res[k] = 0.0;
    S.st[k] = kPending;
    S.it[k] = 0;
    S.mode[k] = mode0;
    S.clamp[k] = 0;
}

// flags[k] = (mode[list[k]] == m) for k < n
__global__ void k_mode_flags(const int32_t* __restrict__ list, const int32_t* __restrict__ mode, int n,
                             int32_t* __restrict__ flags)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flags[k] = mode[list[k]];
}

__global__ void k_pending_flags(const int32_t* __restrict__ list, const int32_t* __restrict__ st, int n,
                                int32_t* __restrict__ flags)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flags[k] = st[list[k]] == kPending ? 1 : 0;
}

// targets T (SoA [3][n]) = x0 + h H for the listed nodes
__global__ void k_gather_targets(const int32_t* __restrict__ list, int n, NodeState S, double* __restrict__ T)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list[k];
    const double h = S.h[i];
    for (int c = 0; c < 3; c++) T[(int64_t)c * n + k] = S.x0[c * S.n + i] + h * S.hd[c * S.n + i];
}

// One Newton update per listed node from res = [phi | gx | gy | gz] ([4][n]).
__global__ void k_newton_update(const int32_t* __restrict__ list, int n, const double* __restrict__ R,
                                NodeState S, int mixed_eval, int accept_mixed, double tol, double sw,
                                int max_iter)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int i = list[k];
    const double r = R[k] - 0.5;
    const int it = S.it[i] + 1;
    S.it[i] = it;
    S.res[i] = fabs(r);
    if (!isfinite(r)) {
        S.st[i] = LSM_NODE_NONFINITE;
        return;
    }
    if ((!mixed_eval || accept_mixed) && fabs(r) < tol) {
        S.st[i] = LSM_NODE_CONVERGED;
        return;
    }
    if (mixed_eval && !accept_mixed && fabs(r) < sw) S.mode[i] = 1;
    const double d = S.hd[i] * R[(int64_t)n + k] + S.hd[S.n + i] * R[2 * (int64_t)n + k] +
                     S.hd[2 * S.n + i] * R[3 * (int64_t)n + k];
    if (!isfinite(d)) {
        S.st[i] = LSM_NODE_NONFINITE;
        return;
    }
    if (d == 0.0) {
        S.st[i] = LSM_NODE_ZERODERIV;
        return;
    }
    double step = -r / d;
    const double lim = 4.0 * S.sl[i];
    if (step > lim || step < -lim) {
        step = step > 0 ? lim : -lim;
        S.clamp[i] = 1;
    }
    S.h[i] += step;
    S.dh[i] = fabs(step);
    if (it >= max_iter) S.st[i] = LSM_NODE_MAXITER;
}

__device__ __forceinline__ void atomic_max_nonneg(double* a, double v)
{
    atomicMax(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// Back to the input order; summary: red[0] = eps_N, red[1] = max residual of
// converged nodes, cnt[0] = converged, cnt[1] = failed.
__global__ void k_unsort_state(const uint32_t* __restrict__ perm, NodeState S, double* __restrict__ xo,
                               double* __restrict__ ho, int32_t* __restrict__ so, double* __restrict__ red,
                               int* __restrict__ cnt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.n) return;
    const int64_t i = perm[k];
    const double h = S.h[k];
    for (int c = 0; c < 3; c++) xo[3 * i + c] = S.x0[c * S.n + k] + h * S.hd[c * S.n + k];
    ho[i] = h;
    int st = S.st[k];
    if (st == kPending) st = LSM_NODE_MAXITER;
    if (S.clamp[k]) st |= LSM_NODE_CLAMPED_BIT;
    so[i] = st;
    atomic_max_nonneg(&red[0], S.dh[k]);
    if ((st & 255) == LSM_NODE_CONVERGED) {
        atomic_max_nonneg(&red[1], S.res[k]);
        atomicAdd(&cnt[0], 1);
    } else {
        atomicAdd(&cnt[1], 1);
    }
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int solve_charts_device(Ctx* ctx, Mesh* me, int n_gl, double tol, int max_iter, int precision,
                        double* x_out, double* h_out, int32_t* status_out, lsm_solve_stats* stats,
                        cudaStream_t st)
{
    const int np = n_gl * n_gl;
    const int64_t N64 = me->m * (int64_t)np;
    if (N64 >= (int64_t)1 << 31) {
        ctx->err = "too many chart nodes";
        return LSM_E_INVALID_ARG;
    }
    const int N = (int)N64;
    lsm_solve_stats S0;
    memset(&S0, 0, sizeof(S0));
    S0.n_nodes = N;
    Scratch s(st);
    // chart rule on the device
    std::vector<double> rule((size_t)np * 3);
    simplex_rule_host(n_gl, 0, rule.data());
    double* rule_d;
    LSM_CUDA_TRY(ctx, s.get(&rule_d, rule.size()));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(rule_d, rule.data(), sizeof(double) * rule.size(),
                                      cudaMemcpyHostToDevice, st));
    double *x0a, *hda, *sla;
    LSM_CUDA_TRY(ctx, s.get(&x0a, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&hda, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&sla, (size_t)N));
    int rc = chart_nodes_init(ctx, me, rule_d, np, x0a, hda, sla, st);
    if (rc) return rc;
    uint32_t* perm;
    LSM_CUDA_TRY(ctx, s.get(&perm, (size_t)N));
    rc = morton_order_points(ctx, x0a, 3, N, perm, st);
    if (rc) return rc;

    NodeState S;
    S.n = N;
    LSM_CUDA_TRY(ctx, s.get(&S.x0, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.hd, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.sl, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.h, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.dh, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.res, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.st, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.it, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.mode, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&S.clamp, (size_t)N));
    const bool mixed = precision == LSM_MIXED;
    k_sort_state<<<nb(N), 256, 0, st>>>(x0a, hda, sla, perm, N, S, mixed ? 0 : 1);
    LSM_LAUNCHED(ctx);

    int32_t *act, *act2, *lst, *flags, *dcount;
    double *T, *R;
    LSM_CUDA_TRY(ctx, s.get(&act, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&act2, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&lst, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&flags, (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&dcount, 4));
    LSM_CUDA_TRY(ctx, s.get(&T, 3 * (size_t)N));
    LSM_CUDA_TRY(ctx, s.get(&R, 4 * (size_t)N));
    int32_t* hcount = nullptr;
    LSM_CUDA_TRY(ctx, cudaMallocHost(&hcount, sizeof(int32_t) * 4));
    struct PinnedFree {
        int32_t* p;
        ~PinnedFree() { cudaFreeHost(p); }
    } pf{hcount};

    // identity active list
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, sizeof(int32_t) * N, st));
    rc = compact_flags(ctx, flags, 0, nullptr, N, act, dcount, st);
    if (rc) return rc;
    int nact = N;
    const int accept_mixed = tol >= ctx->opt.mixed_accept ? 1 : 0;
    int iter = 0;
    for (; iter < max_iter && nact > 0; iter++) {
        if (iter < 32) S0.active_per_iter[iter] = nact;
        for (int m = mixed ? 0 : 1; m <= 1; m++) {
            const int32_t* L = act;
            int nl = nact;
            if (mixed) {
                k_mode_flags<<<nb(nact), 256, 0, st>>>(act, S.mode, nact, flags);
                LSM_LAUNCHED(ctx);
                rc = compact_flags(ctx, flags, m, act, nact, lst, dcount, st);
                if (rc) return rc;
                LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hcount, dcount, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
                nl = hcount[0];
                L = lst;
            }
            if (nl == 0) continue;
            k_gather_targets<<<nb(nl), 256, 0, st>>>(L, nl, S, T);
            LSM_LAUNCHED(ctx);
            Targets tg{T, nl, nl};
            rc = eval_sorted(ctx, me, tg, R, m == 0 ? LSM_MIXED : (mixed ? LSM_FF : LSM_FP64), st);
            if (rc) return rc;
            k_newton_update<<<nb(nl), 256, 0, st>>>(L, nl, R, S, m == 0 ? 1 : 0, accept_mixed, tol,
                                                     ctx->opt.mixed_switch, max_iter);
            LSM_LAUNCHED(ctx);
            if (m == 0) S0.evals_fp32 += nl;
            else S0.evals_fp64 += nl;
        }
        k_pending_flags<<<nb(nact), 256, 0, st>>>(act, S.st, nact, flags);
        LSM_LAUNCHED(ctx);
        rc = compact_flags(ctx, flags, 1, act, nact, act2, dcount, st);
        if (rc) return rc;
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hcount, dcount, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        nact = hcount[0];
        std::swap(act, act2);
    }
    S0.iterations = iter;

    double* red;
    int* cnt;
    LSM_CUDA_TRY(ctx, s.get(&red, 2));
    LSM_CUDA_TRY(ctx, s.get(&cnt, 2));
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(red, 0, sizeof(double) * 2, st));
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, sizeof(int) * 2, st));
    k_unsort_state<<<nb(N), 256, 0, st>>>(perm, S, x_out, h_out, status_out, red, cnt);
    LSM_LAUNCHED(ctx);
    double hred[2];
    int hcnt[2];
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hred, red, sizeof(hred), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hcnt, cnt, sizeof(hcnt), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    S0.eps_newton = hred[0];
    S0.max_residual = hred[1];
    S0.n_converged = hcnt[0];
    S0.n_failed = hcnt[1];
    if (stats) *stats = S0;
    return LSM_OK;
}

}  // namespace lsm
