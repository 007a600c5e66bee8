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

// One Newton update of node i from row k of res = [phi | gx | gy | gz] (plane stride p).
__device__ __forceinline__ void newton_update_one(int i, int k, int64_t p, const double* __restrict__ R,
                                                  NodeState& S, int mixed_eval, int accept_mixed, double tol,
                                                  double sw, int max_iter)
{
    if (S.st[i] != kPending) return;   // listed again after it stopped
    const double r = R[k] - 0.5;
    const int it = S.it[i] + 1;
    S.it[i] = it;
    S.res[i] = fabs(r);
    if (!isfinite(r)) {
        S.st[i] = LSM_NODE_NONFINITE;
        return;
    }
    // the tolerance is met on this evaluation; its update is still applied
    // (eq. newtoneq: each update precedes the stopping test, Sec. 5), so the
    // returned h lies closer to the root than the residual reported
    const bool done = (!mixed_eval || accept_mixed) && fabs(r) < tol;
    if (!done && mixed_eval && !accept_mixed && fabs(r) < sw) S.mode[i] = 1;
    const double d = S.hd[i] * R[p + k] + S.hd[S.n + i] * R[2 * p + k] + S.hd[2 * S.n + i] * R[3 * p + k];
    if (!isfinite(d) || d == 0.0) {
        S.st[i] = done ? LSM_NODE_CONVERGED : (isfinite(d) ? LSM_NODE_ZERODERIV : LSM_NODE_NONFINITE);
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
    if (done) S.st[i] = LSM_NODE_CONVERGED;
    else if (it >= max_iter) S.st[i] = LSM_NODE_MAXITER;
}

__global__ void k_newton_update(const int32_t* __restrict__ list, int n, const double* __restrict__ R,
                                NodeState S, int mixed_eval, int accept_mixed, double tol, double sw,
                                int max_iter)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    newton_update_one(list[k], k, n, R, S, mixed_eval, accept_mixed, tol, sw, max_iter);
}

// ---- device-counted variants (launch shapes fixed by the capacity, so a
// whole sweep can be captured in a CUDA graph)
__global__ void k_newton_update_dev(const int32_t* __restrict__ list, const int* __restrict__ n_dev,
                                    const double* __restrict__ R, int64_t plane, NodeState S, int mixed_eval,
                                    int accept_mixed, double tol, double sw, int max_iter)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *n_dev) return;
    newton_update_one(list[k], k, plane, R, S, mixed_eval, accept_mixed, tol, sw, max_iter);
}

__global__ void k_list_mode_flags(const int32_t* __restrict__ list, const int* __restrict__ n_dev,
                                  const int32_t* __restrict__ mode, int32_t* __restrict__ flags)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < *n_dev) flags[k] = mode[list[k]];
}

__global__ void k_list_pending_flags(const int32_t* __restrict__ list, const int* __restrict__ n_dev,
                                     const int32_t* __restrict__ st, int32_t* __restrict__ flags)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < *n_dev) flags[k] = st[list[k]] == kPending ? 1 : 0;
}

__global__ void k_gather_targets_dev(const int32_t* __restrict__ list, const int* __restrict__ n_dev, NodeState S,
                                     double* __restrict__ T, int64_t ld)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *n_dev) return;
    const int i = list[k];
    const double h = S.h[i];
    for (int c = 0; c < 3; c++) T[(int64_t)c * ld + k] = S.x0[c * S.n + i] + h * S.hd[c * S.n + i];
}

// active-count history: hist[sweep] = n after the sweep (sweeps with work only)
__global__ void k_record_sweep(const int* __restrict__ n_before, const int* __restrict__ n_after,
                               int* __restrict__ counter, int* __restrict__ hist)
{
    if (threadIdx.x == 0 && *n_before > 0) {
        const int s = *counter;
        if (s < 32) hist[s] = *n_before;
        *counter = s + 1;
    }
}

// work items: blocks of at most bs consecutive listed nodes of one mesh
__global__ void k_mesh_hist(const int32_t* __restrict__ list, const int* __restrict__ n_dev,
                            const int32_t* __restrict__ node_mesh, uint32_t* __restrict__ cnt)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < *n_dev) atomicAdd(&cnt[node_mesh[list[k]]], 1u);
}

__global__ void k_mesh_blocks(const uint32_t* __restrict__ cnt, int nmesh, int bs, uint32_t* __restrict__ nblk)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < nmesh) nblk[m] = (cnt[m] + bs - 1) / bs;
}

__global__ void k_write_items(const uint32_t* __restrict__ seg, const uint32_t* __restrict__ cnt,
                              const uint32_t* __restrict__ blk, const int2* __restrict__ mesh_tiles, int nmesh,
                              int bs, int cap, int4* __restrict__ items)
{
    const int m = blockIdx.x;
    if (m >= nmesh) return;
    const int c = (int)cnt[m];
    const int nb = (c + bs - 1) / bs;
    const int2 tr = mesh_tiles[m];
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const int first = (int)seg[m] + j * bs;
        if ((int64_t)blk[m] + j < cap)   // never past the buffer (its size is computed for bs on the host)
            items[blk[m] + j] = make_int4(first, min(bs, c - j * bs), tr.x, tr.y);
    }
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
                        cudaStream_t st, const NodeSpec* spec)
{
    const int np = n_gl * n_gl;
    const int64_t N64 = spec ? spec->n : me->m * (int64_t)np;
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
    int rc = spec ? chart_nodes_at(ctx, me, spec->n, spec->tri, spec->uvw, x0a, hda, sla, st)
                  : chart_nodes_init(ctx, me, rule_d, np, x0a, hda, sla, st);
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
    HostWords hw(ctx);
    LSM_CUDA_TRY(ctx, hw.get());
    int32_t* hcount = hw.p;

    // identity active list
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, sizeof(int32_t) * N, st));
    rc = compact_flags(ctx, flags, 0, nullptr, N, act, dcount, st);
    if (rc) return rc;
    int nact = N;
    const int accept_mixed = tol >= ctx->opt.mixed_accept ? 1 : 0;
    // float-float sweeps come in pairs: the first records the far-tile part
    // of Phi for its list of nodes, the second re-evaluates the same list
    // (same blocks, so the same near/far split) with near tiles only and the
    // recorded far part moved along its gradient; the Newton steps between
    // them are ~1e-8 sigma, where the far part is linear to ~1e-14
    int32_t* Lrec = nullptr;
    double *Trec = nullptr, *Rfar = nullptr;
    float* BBrec = nullptr;   // block boxes of the record sweep (64 or more targets per block)
    int nrec = 0, ff_stage = 0;
    if (mixed) {
        LSM_CUDA_TRY(ctx, s.get(&Lrec, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&Trec, 3 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&Rfar, 4 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&BBrec, 8 * ((size_t)N / 64 + 2)));
    }
    int iter = 0;
    for (; iter < max_iter && nact > 0; iter++) {
        if (iter < 32) S0.active_per_iter[iter] = nact;
        for (int m = mixed ? 0 : 1; m <= 1; m++) {
            const int32_t* L = act;
            int nl = nact;
            if (mixed && m == 1 && ff_stage == 1) {
                // verification sweep on the recorded list
                L = Lrec;
                nl = nrec;
                ff_stage = 0;
                if (nl == 0) continue;
                k_gather_targets<<<nb(nl), 256, 0, st>>>(L, nl, S, T);
                LSM_LAUNCHED(ctx);
                Targets tg{T, nl, nl};
                FFIncremental inc{2, Rfar, Trec, BBrec};
                rc = eval_sorted(ctx, me, tg, R, LSM_FF, st, &inc);
                if (rc) return rc;
                k_newton_update<<<nb(nl), 256, 0, st>>>(L, nl, R, S, 0, accept_mixed, tol, ctx->opt.mixed_switch,
                                                         max_iter);
                LSM_LAUNCHED(ctx);
                S0.evals_fp64 += nl;
                S0.evals_near_only += nl;
                continue;
            }
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
            if (mixed && m == 1) {
                // recording float-float sweep
                FFIncremental inc{1, Rfar, nullptr, BBrec};
                rc = eval_sorted(ctx, me, tg, R, LSM_FF, st, &inc);
                if (rc) return rc;
                LSM_CUDA_TRY(ctx, cudaMemcpyAsync(Lrec, L, sizeof(int32_t) * nl, cudaMemcpyDeviceToDevice, st));
                LSM_CUDA_TRY(ctx, cudaMemcpyAsync(Trec, T, sizeof(double) * 3 * nl, cudaMemcpyDeviceToDevice, st));
                nrec = nl;
                ff_stage = 1;
            } else {
                // mixed sweeps that float-float steps finish take the coarser Newton treecode
                rc = eval_sorted(ctx, me, tg, R, m == 0 ? (accept_mixed ? LSM_MIXED : kPrecMixedNewton) : LSM_FP64,
                                 st);
                if (rc) return rc;
            }
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

// Work items for the listed nodes (the list is ordered by mesh, at most
// n_max long).  Scratch: cnt [2*nmesh] (counts, then segment starts),
// nblk [nmesh] (block counts, then block starts).  *n_items (device) =
// number of items written.  Launch shapes depend on n_max and nmesh only.
int build_items(Ctx* ctx, const int32_t* list, const int* n_list, int n_max, const int32_t* node_mesh,
                const int2* mesh_tiles, int nmesh, int bs, uint32_t* cnt, uint32_t* nblk, int4* items, int* n_items,
                int cap, cudaStream_t st)
{
    uint32_t* seg = cnt + nmesh;
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * nmesh, st));
    k_mesh_hist<<<nb(n_max), 256, 0, st>>>(list, n_list, node_mesh, cnt);
    LSM_LAUNCHED(ctx);
    k_mesh_blocks<<<nb(nmesh), 256, 0, st>>>(cnt, nmesh, bs, nblk);
    LSM_LAUNCHED(ctx);
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(seg, cnt, sizeof(uint32_t) * nmesh, cudaMemcpyDeviceToDevice, st));
    int rc = scan_exclusive(ctx, seg, nmesh, nullptr, st);
    if (rc) return rc;
    rc = scan_exclusive(ctx, nblk, nmesh, reinterpret_cast<uint32_t*>(n_items), st);
    if (rc) return rc;
    k_write_items<<<nmesh, 128, 0, st>>>(seg, cnt, nblk, mesh_tiles, nmesh, bs, cap, items);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

namespace {

// sort key: the mesh of the node at Morton position k
__global__ void k_node_mesh(const int32_t* __restrict__ tri_mesh, int np, int n, const uint32_t* __restrict__ perm,
                            uint32_t* __restrict__ key)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) key[k] = (uint32_t)tri_mesh[perm[k] / np];
}

__global__ void k_gather_mesh(const int32_t* __restrict__ tri_mesh, int np, int n, const uint32_t* __restrict__ perm,
                              int32_t* __restrict__ mesh_of_sorted)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) mesh_of_sorted[k] = tri_mesh[perm[k] / np];
}

// Float-float sweeps of a mixed batch solve come in pairs, as in the
// single-mesh solve: the first (stage 1) evaluates its node list fully and
// records each node's far-tile part; the second (stage 2) re-evaluates the
// same list (same items, so the same near/far split) over near tiles only and
// adds the recorded far part moved along its gradient.
__global__ void k_copy_record(const int32_t* __restrict__ L, const int* __restrict__ nL, int32_t* __restrict__ Lrec,
                              int* __restrict__ n_rec, const double* __restrict__ T, double* __restrict__ Trec, int N)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = *nL;
    if (k == 0) *n_rec = n;
    if (k >= n) return;
    Lrec[k] = L[k];
    for (int c = 0; c < 3; c++) Trec[(int64_t)c * N + k] = T[(int64_t)c * N + k];
}

struct BatchSweep {
    int N, nmesh, max_items_mixed, max_items_other;
    int32_t* Lrec;     // float-float record: node list, its length, targets, far part, block boxes
    int* n_rec;
    double *Trec, *Rfar;
    float* BBrec;
    int32_t *flags, *lst, *node_mesh;
    int *n_lst, *n_items, *sweep_counter, *hist;
    double *T, *R;
    int4* items;
    uint32_t *bc, *cnt, *nblk;
    const int2* mesh_tiles;
    SourceView view;
    NodeState S;
    bool mixed;
    int accept_mixed, max_iter;
    double tol, sw;
    int tpb;          // mixed kernel: targets per work item (0: default)
    double cut;       // mixed kernel: near-field radius in sigma (0: default)
};

int batch_sweep(Ctx* ctx, const BatchSweep& B, const int32_t* act, const int* n_act, int32_t* act_out,
                int* n_act_out, cudaStream_t st, int ff_stage)
{
    int rc;
    for (int m = B.mixed ? 0 : 1; m <= 1; m++) {
        const int prec = m == 0 ? LSM_MIXED : (B.mixed ? LSM_FF : LSM_FP64);
        const int32_t* L = act;
        const int* nL = n_act;
        const bool verify = B.mixed && m == 1 && ff_stage == 2;
        if (verify) {
            L = B.Lrec;
            nL = B.n_rec;
        } else if (B.mixed) {
            k_list_mode_flags<<<nb(B.N), 256, 0, st>>>(act, n_act, B.S.mode, B.flags);
            LSM_LAUNCHED(ctx);
            rc = compact_flags_dev(ctx, B.flags, m, act, n_act, B.N, B.lst, B.n_lst, B.bc, st);
            if (rc) return rc;
            L = B.lst;
            nL = B.n_lst;
        }
        k_gather_targets_dev<<<nb(B.N), 256, 0, st>>>(L, nL, B.S, B.T, B.N);
        LSM_LAUNCHED(ctx);
        const int bs = eval_item_targets(ctx, prec, B.tpb);
        rc = build_items(ctx, L, nL, B.N, B.node_mesh, B.mesh_tiles, B.nmesh, bs, B.cnt, B.nblk, B.items, B.n_items,
                         std::max(B.max_items_mixed, B.max_items_other), st);
        if (rc) return rc;
        Targets tg{B.T, B.N, B.N};
        FFIncremental inc{verify ? 2 : 1, B.Rfar, verify ? B.Trec : nullptr, B.BBrec};
        const bool ffpair = B.mixed && m == 1;
        // mixed sweeps that float-float steps finish take the Newton near-field radius
        const double cut = prec == LSM_MIXED && !B.accept_mixed
                               ? std::min(B.cut > 0.0 ? B.cut : ctx->opt.cutoff_mixed, (double)ctx->opt.newton_cutoff)
                               : B.cut;
        rc = eval_items(ctx, B.view, tg, B.items, B.n_items, prec == LSM_MIXED ? B.max_items_mixed : B.max_items_other,
                        B.R, prec, st, ffpair ? &inc : nullptr, B.tpb, cut);
        if (rc) return rc;
        if (ffpair && !verify) {
            k_copy_record<<<nb(B.N), 256, 0, st>>>(L, nL, B.Lrec, B.n_rec, B.T, B.Trec, B.N);
            LSM_LAUNCHED(ctx);
        }
        k_newton_update_dev<<<nb(B.N), 256, 0, st>>>(L, nL, B.R, B.N, B.S, m == 0 ? 1 : 0, B.accept_mixed, B.tol, B.sw,
                                                     B.max_iter);
        LSM_LAUNCHED(ctx);
    }
    k_list_pending_flags<<<nb(B.N), 256, 0, st>>>(act, n_act, B.S.st, B.flags);
    LSM_LAUNCHED(ctx);
    rc = compact_flags_dev(ctx, B.flags, 1, act, n_act, B.N, act_out, n_act_out, B.bc, st);
    if (rc) return rc;
    k_record_sweep<<<1, 32, 0, st>>>(n_act, n_act_out, B.sweep_counter, B.hist);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace

// Chart solve for every mesh of a batch in one set of launches per sweep.
// With use_graph, two sweeps (A -> B -> A) are captured once as a CUDA graph
// and replayed until no node is active or max_iter sweeps have run.
int solve_charts_batch(Ctx* ctx, Batch* b, int n_gl, double tol, int max_iter, int precision, int use_graph,
                       double* x_out, double* h_out, int32_t* status_out, lsm_solve_stats* stats, cudaStream_t caller)
{
    const int np = n_gl * n_gl;
    const int64_t N64 = b->m * (int64_t)np;
    if (N64 <= 0 || N64 >= ((int64_t)1 << 31) - 1024) {
        ctx->err = "batch chart solve: node count out of range";
        return LSM_E_INVALID_ARG;
    }
    const int N = (int)N64;
    // a private stream (graph capture needs one), ordered after the caller's work
    cudaStream_t st;
    LSM_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamFree {
        cudaStream_t s;
        ~StreamFree() { cudaStreamDestroy(s); }
    } sfree{st};
    cudaEvent_t ev;
    LSM_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    struct EventFree {
        cudaEvent_t e;
        ~EventFree() { cudaEventDestroy(e); }
    } efree{ev};
    LSM_CUDA_TRY(ctx, cudaEventRecord(ev, caller));
    LSM_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ev, 0));

    lsm_solve_stats S0;
    memset(&S0, 0, sizeof(S0));
    S0.n_nodes = N;
    int rc;
    {
        Scratch s(st);
        std::vector<double> rule((size_t)np * 3);
        simplex_rule_host(n_gl, 0, rule.data());
        double* rule_d;
        LSM_CUDA_TRY(ctx, s.get(&rule_d, rule.size()));
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(rule_d, rule.data(), sizeof(double) * rule.size(), cudaMemcpyHostToDevice, st));
        double *x0a, *hda, *sla;
        LSM_CUDA_TRY(ctx, s.get(&x0a, 3 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&hda, 3 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&sla, (size_t)N));
        rc = chart_nodes_raw(ctx, b->verts, b->tris, b->vpn, b->tri_sigma, b->m, rule_d, np, x0a, hda, sla, st);
        if (rc) return rc;
        // order: mesh, then Morton within the batch's box
        uint32_t *perm, *key;
        LSM_CUDA_TRY(ctx, s.get(&perm, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&key, (size_t)N));
        rc = morton_order_points(ctx, x0a, 3, N, perm, st);
        if (rc) return rc;
        k_node_mesh<<<nb(N), 256, 0, st>>>(b->tri_mesh, np, N, perm, key);
        LSM_LAUNCHED(ctx);
        int bits = 1;
        while ((1 << bits) < b->nmesh) bits++;
        rc = radix_sort_pairs(ctx, key, perm, N, bits, st);
        if (rc) return rc;

        BatchSweep B;
        B.N = N;
        B.nmesh = b->nmesh;
        B.mixed = precision == LSM_MIXED;   // before the item sizes, which depend on it
        B.tpb = b->tpb;
        B.cut = b->cut_mixed;
        B.max_items_mixed = (N + eval_item_targets(ctx, LSM_MIXED, B.tpb) - 1) / eval_item_targets(ctx, LSM_MIXED, B.tpb) +
                            b->nmesh;
        const int bs_other = eval_item_targets(ctx, B.mixed ? LSM_FF : LSM_FP64);
        B.max_items_other = (N + bs_other - 1) / bs_other + b->nmesh;
        B.mesh_tiles = b->mesh_tiles;
        B.view = view_of_batch(b);
        B.accept_mixed = tol >= ctx->opt.mixed_accept ? 1 : 0;
        B.max_iter = max_iter;
        B.tol = tol;
        B.sw = ctx->opt.mixed_switch;
        NodeState& S = B.S;
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
        k_sort_state<<<nb(N), 256, 0, st>>>(x0a, hda, sla, perm, N, S, B.mixed ? 0 : 1);
        LSM_LAUNCHED(ctx);
        LSM_CUDA_TRY(ctx, s.get(&B.node_mesh, (size_t)N));
        k_gather_mesh<<<nb(N), 256, 0, st>>>(b->tri_mesh, np, N, perm, B.node_mesh);
        LSM_LAUNCHED(ctx);

        int32_t *actA, *actB;
        int* cnts;  // n_actA, n_actB, n_lst, n_items, sweep counter, hist[32]
        LSM_CUDA_TRY(ctx, s.get(&actA, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&actB, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.lst, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.flags, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.T, 3 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.R, 4 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.items, (size_t)std::max(B.max_items_mixed, B.max_items_other)));
        LSM_CUDA_TRY(ctx, s.get(&B.bc, (size_t)compact_blocks(N) + 1));
        LSM_CUDA_TRY(ctx, s.get(&B.cnt, 2 * (size_t)b->nmesh));
        LSM_CUDA_TRY(ctx, s.get(&B.nblk, (size_t)b->nmesh));
        LSM_CUDA_TRY(ctx, s.get(&cnts, 40));
        LSM_CUDA_TRY(ctx, cudaMemsetAsync(cnts, 0, sizeof(int) * 40, st));
        int* n_actA = cnts;
        int* n_actB = cnts + 1;
        B.n_lst = cnts + 2;
        B.n_items = cnts + 3;
        B.sweep_counter = cnts + 4;
        B.hist = cnts + 5;
        B.n_rec = cnts + 37;
        LSM_CUDA_TRY(ctx, s.get(&B.Lrec, (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.Trec, 3 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.Rfar, 4 * (size_t)N));
        LSM_CUDA_TRY(ctx, s.get(&B.BBrec, 8 * (size_t)B.max_items_other));
        // identity active list
        LSM_CUDA_TRY(ctx, cudaMemsetAsync(B.flags, 0, sizeof(int32_t) * N, st));
        rc = compact_flags(ctx, B.flags, 0, nullptr, N, actA, n_actA, st);
        if (rc) return rc;

        HostWords hw(ctx);
        LSM_CUDA_TRY(ctx, hw.get());
        int32_t* hcount = hw.p;   // 40 words: the batch counters

        int sweeps = 0;
        if (use_graph) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            const int64_t l0 = ctx->launches;
            LSM_CUDA_TRY(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            // sweep 1 records the float-float far parts, sweep 2 verifies
            int rc1 = batch_sweep(ctx, B, actA, n_actA, actB, n_actB, st, 1);
            int rc2 = rc1 ? rc1 : batch_sweep(ctx, B, actB, n_actB, actA, n_actA, st, 2);
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (rc2 || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                if (!rc2) ctx->err = std::string("graph capture: ") + cudaGetErrorString(ce);
                return rc2 ? rc2 : LSM_E_CUDA;
            }
            const int64_t per_replay = ctx->launches - l0;
            ctx->launches = l0;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(ce);
                return LSM_E_CUDA;
            }
            struct ExecFree {
                cudaGraphExec_t e;
                ~ExecFree() { cudaGraphExecDestroy(e); }
            } xfree{exec};
            while (sweeps < max_iter) {
                LSM_CUDA_TRY(ctx, cudaGraphLaunch(exec, st));
                ctx->launches += per_replay;
                sweeps += 2;
                LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hcount, n_actA, sizeof(int), cudaMemcpyDeviceToHost, st));
                LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
                if (hcount[0] == 0) break;
            }
        } else {
            int32_t *a = actA, *c = actB;
            int *na = n_actA, *nc = n_actB;
            while (sweeps < max_iter) {
                rc = batch_sweep(ctx, B, a, na, c, nc, st, (sweeps & 1) ? 2 : 1);
                if (rc) return rc;
                sweeps++;
                LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hcount, nc, sizeof(int), cudaMemcpyDeviceToHost, st));
                LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
                std::swap(a, c);
                std::swap(na, nc);
                if (hcount[0] == 0) break;
            }
        }
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hcount, cnts, sizeof(int) * 40, cudaMemcpyDeviceToHost, st));
        LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        S0.iterations = hcount[4];
        for (int k = 0; k < 32 && k < hcount[4]; k++) S0.active_per_iter[k] = hcount[5 + k];

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
    }
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    LSM_CUDA_TRY(ctx, cudaEventRecord(ev, st));
    LSM_CUDA_TRY(ctx, cudaStreamWaitEvent(caller, ev, 0));
    if (stats) *stats = S0;
    return LSM_OK;
}

}  // namespace lsm
