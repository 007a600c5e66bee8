// api.cu -- the extern "C" entry points declared in include/lsm.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {

// Duffy-collapsed n x n Gauss-Legendre rule on the standard simplex,
// composite over `subdiv` midpoint splits (Sec. 4.3 and 4.5).  For each
// (sub)triangle (A, B, C) with children (A,mAB,mCA), (mAB,B,mBC),
// (mCA,mBC,C), (mBC,mCA,mAB): node A + s (B-A) + t (C-A) with
// s = xi (1 - eta), t = xi eta, weight w_xi w_eta xi |det(B-A, C-A)|.
// Output uvw[cnt][3] = (u, v, w); order: subtriangle, xi, eta.
void simplex_rule_host(int n, int subdiv, double* uvw)
{
    // Gauss-Legendre on [-1, 1] by Newton iteration on P_n, then mapped to [0, 1]
    std::vector<double> xg(n), wg(n);
    for (int i = 0; i < n; i++) {
        double z = std::cos(M_PI * (n - i - 0.25) / (n + 0.5));  // ascending roots
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double pm = 1.0, p = z;
            for (int k = 2; k <= n; k++) {
                const double pk = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
                pm = p;
                p = pk;
            }
            dp = n * (pm - z * p) / (1.0 - z * z);
            const double dz = p / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-16) {
                double q0 = 1.0, q1 = z;
                for (int k = 2; k <= n; k++) {
                    const double qk = ((2 * k - 1) * z * q1 - (k - 1) * q0) / k;
                    q0 = q1;
                    q1 = qk;
                }
                dp = n * (q0 - z * q1) / (1.0 - z * z);
                break;
            }
        }
        xg[i] = 0.5 * (z + 1.0);
        wg[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    struct Tri {
        double a[2], b[2], c[2];
    };
    std::vector<Tri> cur{{{0, 0}, {1, 0}, {0, 1}}}, nxt;
    for (int l = 0; l < subdiv; l++) {
        nxt.clear();
        for (const Tri& t : cur) {
            const double ab[2] = {0.5 * (t.a[0] + t.b[0]), 0.5 * (t.a[1] + t.b[1])};
            const double bc[2] = {0.5 * (t.b[0] + t.c[0]), 0.5 * (t.b[1] + t.c[1])};
            const double ca[2] = {0.5 * (t.c[0] + t.a[0]), 0.5 * (t.c[1] + t.a[1])};
            nxt.push_back({{t.a[0], t.a[1]}, {ab[0], ab[1]}, {ca[0], ca[1]}});
            nxt.push_back({{ab[0], ab[1]}, {t.b[0], t.b[1]}, {bc[0], bc[1]}});
            nxt.push_back({{ca[0], ca[1]}, {bc[0], bc[1]}, {t.c[0], t.c[1]}});
            nxt.push_back({{bc[0], bc[1]}, {ca[0], ca[1]}, {ab[0], ab[1]}});
        }
        cur.swap(nxt);
    }
    size_t o = 0;
    for (const Tri& t : cur) {
        const double e1[2] = {t.b[0] - t.a[0], t.b[1] - t.a[1]};
        const double e2[2] = {t.c[0] - t.a[0], t.c[1] - t.a[1]};
        const double det = std::fabs(e1[0] * e2[1] - e1[1] * e2[0]);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                const double s = xg[i] * (1.0 - xg[j]), q = xg[i] * xg[j];
                uvw[o++] = t.a[0] + s * e1[0] + q * e2[0];
                uvw[o++] = t.a[1] + s * e1[1] + q * e2[1];
                uvw[o++] = wg[i] * wg[j] * xg[i] * det;
            }
    }
}

namespace {

// Makes `dev` current for the scope of a call.  A failure here is left to
// the call's own checks, but its error is cleared, so that it cannot surface
// later as the error of an unrelated launch.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            if (cudaSetDevice(dev) != cudaSuccess) cudaGetLastError();
        } else {
            prev = -1;
            cudaGetLastError();
        }
    }
    ~DeviceGuard() {
        if (prev >= 0 && cudaSetDevice(prev) != cudaSuccess) cudaGetLastError();
    }
};

template <class H>
void reg_add(Ctx* ctx, std::set<H*>& set, H* h)
{
    std::lock_guard<std::mutex> lk(ctx->reg_mu);
    set.insert(h);
}
template <class H>
void reg_remove(Ctx* ctx, std::set<H*>& set, H* h)
{
    std::lock_guard<std::mutex> lk(ctx->reg_mu);
    set.erase(h);
}

bool is_device_ptr(const void* p)
{
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Input array as a device pointer: either the caller's or a stream-ordered copy.
template <class T>
int to_device(Ctx* ctx, Scratch& s, const T* p, size_t count, const T** out, cudaStream_t st)
{
    if (p == nullptr || count == 0) {
        *out = p;
        return LSM_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return LSM_OK;
    }
    T* d;
    LSM_CUDA_TRY(ctx, s.get(&d, count));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, st));
    *out = d;
    return LSM_OK;
}

// Host-side topology check: indices in range, no repeated vertex, and every
// directed edge (a, b) appears exactly once with its reverse (b, a) present:
// the surface is closed, edge-manifold and consistently oriented.
bool check_topology(const int32_t* tris, int64_t m, int64_t nv, std::string& why)
{
    std::vector<uint64_t> e;
    e.reserve(3 * (size_t)m);
    for (int64_t j = 0; j < m; j++) {
        const int32_t a = tris[3 * j], b = tris[3 * j + 1], c = tris[3 * j + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
            why = "triangle index out of range";
            return false;
        }
        if (a == b || b == c || c == a) {
            why = "degenerate triangle (repeated vertex)";
            return false;
        }
        e.push_back((uint64_t)a * (uint64_t)nv + (uint64_t)b);
        e.push_back((uint64_t)b * (uint64_t)nv + (uint64_t)c);
        e.push_back((uint64_t)c * (uint64_t)nv + (uint64_t)a);
    }
    std::sort(e.begin(), e.end());
    for (size_t i = 1; i < e.size(); i++)
        if (e[i] == e[i - 1]) {
            why = "directed edge used twice (inconsistent orientation or non-manifold edge)";
            return false;
        }
    for (uint64_t k : e) {
        const uint64_t a = k / (uint64_t)nv, b = k % (uint64_t)nv;
        if (!std::binary_search(e.begin(), e.end(), b * (uint64_t)nv + a)) {
            why = "open edge (mesh not watertight)";
            return false;
        }
    }
    return true;
}

// SoA sorted targets from AoS x and a permutation
__global__ void k_gather_points(const double* __restrict__ x, const uint32_t* __restrict__ perm, int n,
                                double* __restrict__ T)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm[k];
    for (int c = 0; c < 3; c++) T[(int64_t)c * n + k] = x[3 * i + c];
}

__global__ void k_scatter_results(const double* __restrict__ R, const uint32_t* __restrict__ perm, int n,
                                  double* __restrict__ phi, double* __restrict__ grad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm[k];
    phi[i] = R[k];
    if (grad) {
        grad[3 * i] = R[(int64_t)n + k];
        grad[3 * i + 1] = R[2 * (int64_t)n + k];
        grad[3 * i + 2] = R[3 * (int64_t)n + k];
    }
}

// res [6][n] in sorted order -> out [n][6] in the caller's order
__global__ void k_scatter6(const double* __restrict__ R, const uint32_t* __restrict__ perm, int n,
                           double* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = perm[i];
    for (int c = 0; c < 6; c++) out[6 * o + c] = R[(int64_t)c * n + i];
}

}  // namespace

int check_flag(Ctx* ctx, cudaStream_t st)
{
    int h = 0;
    int* f = flag_word(ctx);
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (h != 0) {
        ctx->err = "device wait limit reached in a pair kernel (error word " + std::to_string(h) +
                   "); the targets of the blocks that gave up hold NaN";
        LSM_CUDA_TRY(ctx, cudaMemsetAsync(f, 0, sizeof(int), st));
        LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        return LSM_E_TIMEOUT;
    }
    return LSM_OK;
}

namespace {

// Edge nodes of quadratic patches: in range, never a patch corner, every
// vertex a corner or an edge node, and the two patches on an edge sharing
// its node (directed edge (a, b) and its reverse carry the same node).
bool check_edge_nodes(const int32_t* t6, int64_t m, int64_t nv, std::string& why)
{
    std::vector<uint8_t> role((size_t)nv, 0);   // 1 corner, 2 edge node
    for (int64_t j = 0; j < m; j++)
        for (int k = 0; k < 3; k++) role[t6[6 * j + k]] |= 1;
    std::vector<std::pair<uint64_t, int32_t>> e;
    e.reserve(3 * (size_t)m);
    for (int64_t j = 0; j < m; j++) {
        for (int k = 0; k < 3; k++) {
            const int32_t a = t6[6 * j + k], b = t6[6 * j + (k + 1) % 3], mid = t6[6 * j + 3 + k];
            if (mid < 0 || mid >= nv) {
                why = "edge node index out of range";
                return false;
            }
            role[mid] |= 2;
            e.push_back({(uint64_t)a * (uint64_t)nv + (uint64_t)b, mid});
        }
    }
    for (int64_t i = 0; i < nv; i++) {
        if (role[i] == 3) {
            why = "a vertex is both a patch corner and an edge node";
            return false;
        }
        if (role[i] == 0) {
            why = "vertex not used by any patch";
            return false;
        }
    }
    std::sort(e.begin(), e.end());
    for (const auto& d : e) {
        const uint64_t a = d.first / (uint64_t)nv, b = d.first % (uint64_t)nv;
        auto it = std::lower_bound(e.begin(), e.end(), std::make_pair(b * (uint64_t)nv + a, INT32_MIN));
        if (it == e.end() || it->first != b * (uint64_t)nv + a || it->second != d.second) {
            why = "the two patches on an edge do not share its edge node";
            return false;
        }
    }
    return true;
}

// Upload after the topology checks: tris holds the triangles' (or patches')
// corners, tris6 (host, or null for flat triangles) the quadratic patches.
int upload_common(Ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tris6,
                  const double* sigma, const lsm_quad* rule, cudaStream_t st, lsm_mesh** out)
{
    lsm_quad q = rule ? *rule : lsm_quad{4, 0};
    if (q.n_gl < 1 || q.n_gl > 32 || q.subdiv < 0 || q.subdiv > 5) {
        ctx->err = "mesh_upload: rule needs 1 <= n_gl <= 32 and 0 <= subdiv <= 5";
        return LSM_E_INVALID_ARG;
    }
    const int nq = q.n_gl * q.n_gl * (1 << (2 * q.subdiv));
    const int64_t ns = nt * (int64_t)nq;
    if (ns >= ((int64_t)1 << 31) - kTile || nv >= ((int64_t)1 << 31)) {
        ctx->err = "mesh_upload: too many source nodes (limit 2^31)";
        return LSM_E_INVALID_ARG;
    }
    lsm_mesh* mh = new (std::nothrow) lsm_mesh();
    if (!mh) return LSM_E_OOM;
    Mesh* me = &mh->m;
    me->ctx = ctx;
    me->nv = nv;
    me->m = nt;
    me->nq = nq;
    me->rule = q;
    me->ns = ns;   // tiles (and the padded source arrays) are laid out by build_mesh_device
    auto fail = [&](int rc) {
        lsm_mesh_free(mh);
        return rc;
    };
    auto alloc = [&](auto** p, size_t count) -> bool {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
        const size_t bytes = count * sizeof(T);
        if (cudaMalloc((void**)p, bytes) != cudaSuccess) return false;
        me->bytes += bytes;
        return true;
    };
    if (!alloc(&me->verts, 3 * nv) || !alloc(&me->tris, 3 * nt) || !alloc(&me->tri_sigma, nt) ||
        !alloc(&me->tri_n, 3 * nt) || !alloc(&me->vpn, 3 * nv) || (tris6 && !alloc(&me->tris6, 6 * nt))) {
        cudaGetLastError();
        ctx->err = "mesh_upload: out of device memory";
        return fail(LSM_E_OOM);
    }
    const cudaMemcpyKind kv = is_device_ptr(verts) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kt = is_device_ptr(tris) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(me->verts, verts, sizeof(double) * 3 * nv, kv, st) != cudaSuccess ||
        cudaMemcpyAsync(me->tris, tris, sizeof(int32_t) * 3 * nt, kt, st) != cudaSuccess ||
        (tris6 && cudaMemcpyAsync(me->tris6, tris6, sizeof(int32_t) * 6 * nt, cudaMemcpyHostToDevice, st) !=
                      cudaSuccess)) {
        ctx->err = "mesh_upload: copy failed";
        return fail(LSM_E_CUDA);
    }
    int rc;
    {
        Scratch s(st);
        const double* sig_d = nullptr;
        rc = to_device(ctx, s, sigma, (size_t)nt, &sig_d, st);
        if (rc) return fail(rc);
        std::vector<double> rh((size_t)nq * 3);
        simplex_rule_host(q.n_gl, q.subdiv, rh.data());
        double* rd;
        if (s.get(&rd, rh.size()) != cudaSuccess ||
            cudaMemcpyAsync(rd, rh.data(), sizeof(double) * rh.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            ctx->err = "mesh_upload: rule upload failed";
            return fail(LSM_E_CUDA);
        }
        double red[8];
        rc = build_mesh_device(ctx, me, sig_d, rd, red, st);
        if (rc == LSM_E_MESH) {
            ctx->err = red[3] > 0 ? "mesh_upload: zero-area triangle or sigma <= 0"
                     : red[4] > 0 ? "mesh_upload: vertex not used by any triangle"
                                  : "mesh_upload: signed volume <= 0 (triangles must be counter-clockwise seen from outside)";
        }
        if (rc) return fail(rc);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        ctx->err = "mesh_upload: stream failed";
        return fail(LSM_E_CUDA);
    }
    reg_add(ctx, ctx->meshes, mh);
    *out = mh;
    return LSM_OK;
}

}  // namespace
}  // namespace lsm

using namespace lsm;

extern "C" {

int lsm_create(lsm_ctx** out, int device, const lsm_options* opt)
{
    if (!out) return LSM_E_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LSM_E_INVALID_ARG;
    lsm_ctx* c = new (std::nothrow) lsm_ctx();
    if (!c) return LSM_E_OOM;
    Ctx* ctx = &c->c;
    ctx->device = device;
    ctx->opt.cutoff_fp64 = 8.0;
    ctx->opt.cutoff_mixed = 6.5;
    ctx->opt.mixed_switch = 1e-4;
    ctx->opt.mixed_accept = 1e-7;
    ctx->opt.tree_degree = 8;
    ctx->opt.tree_theta = 0.45f;
    ctx->opt.tree_min_sources = 262144;
    ctx->opt.tree_ff_degree = 14;
    ctx->opt.tree_ff_theta = 0.45f;
    ctx->opt.tree_ff_min_sources = 262144;
    ctx->opt.tree_grid = 1;
    ctx->opt.tree_ff_cluster = 4096;
    ctx->opt.tree_cluster = 4096;
    ctx->opt.ff_block = 64;
    ctx->opt.newton_tree_degree = 5;
    ctx->opt.newton_tree_theta = 0.5f;
    ctx->opt.newton_cutoff = 5.0f;
    if (opt) {
        if (opt->tree_degree < 0 || opt->tree_degree > 12 || opt->tree_theta < 0.0f ||
            opt->tree_theta >= 1.0f || opt->tree_min_sources < -1 || opt->tree_ff_degree < 0 ||
            opt->tree_ff_degree > kTreeMaxDegree || opt->tree_ff_theta < 0.0f || opt->tree_ff_theta >= 1.0f ||
            opt->tree_ff_min_sources < -1 || opt->tree_grid < 0 || opt->tree_grid > 2 || opt->tree_ff_cluster < -1 ||
            opt->tree_ff_cluster > (1 << 20) || (opt->tree_ff_cluster > 0 && opt->tree_ff_cluster % kEvalThreads) ||
            opt->tree_cluster < -1 || opt->tree_cluster > (1 << 20) ||
            (opt->tree_cluster > 0 && opt->tree_cluster % (2 * kEvalThreads)) ||
            (opt->ff_block != 0 && opt->ff_block != 64 && opt->ff_block != 128) ||
            (opt->mixed_block != 0 && opt->mixed_block != 64 && opt->mixed_block != 128 && opt->mixed_block != 256) ||
            opt->newton_tree_degree < -1 || opt->newton_tree_degree > 12 || opt->newton_tree_theta < 0.0f ||
            opt->newton_tree_theta >= 1.0f || opt->newton_cutoff < 0.0f || opt->newton_cutoff > 16.0f) {
            delete c;
            return LSM_E_INVALID_ARG;
        }
        if (opt->mixed_accept > 0) ctx->opt.mixed_accept = opt->mixed_accept;
        if (opt->cutoff_fp64 > 0) ctx->opt.cutoff_fp64 = opt->cutoff_fp64;
        if (opt->cutoff_mixed > 0) ctx->opt.cutoff_mixed = opt->cutoff_mixed;
        if (opt->mixed_switch > 0) ctx->opt.mixed_switch = opt->mixed_switch;
        if (opt->tree_degree > 0) ctx->opt.tree_degree = opt->tree_degree;
        if (opt->tree_theta > 0.0f) ctx->opt.tree_theta = opt->tree_theta;
        if (opt->tree_min_sources != 0) ctx->opt.tree_min_sources = opt->tree_min_sources;
        if (opt->tree_ff_degree > 0) ctx->opt.tree_ff_degree = opt->tree_ff_degree;
        if (opt->tree_ff_theta > 0.0f) ctx->opt.tree_ff_theta = opt->tree_ff_theta;
        if (opt->tree_ff_min_sources != 0) ctx->opt.tree_ff_min_sources = opt->tree_ff_min_sources;
        if (opt->tree_grid > 0) ctx->opt.tree_grid = opt->tree_grid;
        if (opt->tree_ff_cluster != 0) ctx->opt.tree_ff_cluster = opt->tree_ff_cluster > 0 ? opt->tree_ff_cluster : 0;
        if (opt->tree_cluster != 0) ctx->opt.tree_cluster = opt->tree_cluster > 0 ? opt->tree_cluster : 0;
        if (opt->ff_block != 0) ctx->opt.ff_block = opt->ff_block;
        ctx->opt.mixed_block = opt->mixed_block;
        if (opt->newton_tree_degree != 0) ctx->opt.newton_tree_degree = opt->newton_tree_degree;
        if (opt->newton_tree_theta > 0.0f) ctx->opt.newton_tree_theta = opt->newton_tree_theta;
        if (opt->newton_cutoff > 0.0f) ctx->opt.newton_cutoff = opt->newton_cutoff;
    }
    DeviceGuard g(device);
    int rc = LSM_OK;
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&ctx->d_flag, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_flag, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->d_pairs, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_pairs, 0, 8 * sizeof(unsigned long long)) != cudaSuccess) {
        delete c;
        return LSM_E_CUDA;
    }
    rc = eval_init_constants(ctx);
    if (rc != LSM_OK) {
        cudaFree(ctx->d_flag);
        delete c;
        return rc;
    }
    // keep freed scratch in the stream-ordered pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return LSM_OK;
}

int lsm_destroy(lsm_ctx* c)
{
    if (!c) return LSM_E_INVALID_ARG;
    DeviceGuard g(c->c.device);
    // what the caller did not free: servers first (their workers use meshes
    // of their own), then batches, then meshes
    std::vector<lsm_server*> sv;
    std::vector<lsm_batch*> bt;
    std::vector<lsm_mesh*> ms;
    {
        std::lock_guard<std::mutex> lk(c->c.reg_mu);
        sv.assign(c->c.servers.begin(), c->c.servers.end());
        bt.assign(c->c.batches.begin(), c->c.batches.end());
        ms.assign(c->c.meshes.begin(), c->c.meshes.end());
    }
    for (lsm_server* s : sv) lsm_server_destroy(s);
    for (lsm_batch* b : bt) lsm_batch_free(b);
    for (lsm_mesh* m : ms) lsm_mesh_free(m);
    cudaFree(c->c.d_flag);
    cudaFree(c->c.d_pairs);
    for (int32_t* p : c->c.host_free) cudaFreeHost(p);
    for (auto& e : c->c.prof_events) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    delete c;
    return LSM_OK;
}

int lsm_set_profiling(lsm_ctx* c, int enable)
{
    if (!c) return LSM_E_INVALID_ARG;
    c->c.profiling = enable != 0;
    return LSM_OK;
}

int lsm_read_stats(lsm_ctx* c, lsm_ctx_stats* out, int reset)
{
    if (!c || !out) return LSM_E_INVALID_ARG;
    Ctx* ctx = &c->c;
    DeviceGuard g(ctx->device);
    LSM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    for (auto& e : ctx->prof_events) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) ctx->prof_ms[e.kind] += ms;
        ctx->prof_launches[e.kind]++;
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    ctx->prof_events.clear();
    unsigned long long pr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    LSM_CUDA_TRY(ctx, cudaMemcpy(pr, ctx->d_pairs, sizeof(pr), cudaMemcpyDeviceToHost));
    out->launches = ctx->launches.load();
    out->pairs_near = out->pairs_far = 0;
    out->pair_kernel_launches = 0;
    out->pair_kernel_ms = 0.0;
    for (int k = 0; k < 4; k++) {
        out->kind_pairs_near[k] = (int64_t)pr[2 * k];
        out->kind_pairs_far[k] = (int64_t)pr[2 * k + 1];
        out->kind_launches[k] = ctx->prof_launches[k];
        out->kind_ms[k] = ctx->prof_ms[k];
        out->pairs_near += out->kind_pairs_near[k];
        out->pairs_far += out->kind_pairs_far[k];
        out->pair_kernel_launches += ctx->prof_launches[k];
        out->pair_kernel_ms += ctx->prof_ms[k];
    }
    if (reset) {
        LSM_CUDA_TRY(ctx, cudaMemset(ctx->d_pairs, 0, sizeof(pr)));
        for (int k = 0; k < 4; k++) {
            ctx->prof_ms[k] = 0.0;
            ctx->prof_launches[k] = 0;
        }
    }
    return LSM_OK;
}

const char* lsm_last_error(const lsm_ctx* c)
{
    if (!c) return "null context";
    return c->c.err.c_str();
}

int64_t lsm_launch_count(const lsm_ctx* c) { return c ? c->c.launches.load() : -1; }

int lsm_check_error(lsm_ctx* c, void* stream)
{
    if (!c) return LSM_E_INVALID_ARG;
    DeviceGuard g(c->c.device);
    return check_flag(&c->c, (cudaStream_t)stream);
}

int lsm_test_inject_wait_timeout(lsm_ctx* c, int enable)
{
    if (!c) return LSM_E_INVALID_ARG;
    c->c.test_nocopy = enable != 0;
    return LSM_OK;
}

int lsm_mesh_upload(lsm_ctx* c, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                    const double* sigma, const lsm_quad* rule, void* stream, lsm_mesh** out)
{
    if (!c || !out) return LSM_E_INVALID_ARG;
    *out = nullptr;
    Ctx* ctx = &c->c;
    if (!verts || !tris || nv < 3 || nt < 4) {
        ctx->err = "mesh_upload: need at least 3 vertices and 4 triangles";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    // topology on the host
    std::vector<int32_t> htris;
    const int32_t* tp = tris;
    if (is_device_ptr(tris)) {
        htris.resize(3 * (size_t)nt);
        LSM_CUDA_TRY(ctx, cudaMemcpy(htris.data(), tris, sizeof(int32_t) * 3 * nt, cudaMemcpyDeviceToHost));
        tp = htris.data();
    }
    std::string why;
    if (!check_topology(tp, nt, nv, why)) {
        ctx->err = "mesh_upload: " + why;
        return LSM_E_MESH;
    }
    return upload_common(ctx, verts, nv, tris, nt, nullptr, sigma, rule, (cudaStream_t)stream, out);
}

int lsm_mesh_upload_quadratic(lsm_ctx* c, const double* verts, int64_t nv, const int32_t* tris6, int64_t nt,
                              const double* sigma, const lsm_quad* rule, void* stream, lsm_mesh** out)
{
    if (!c || !out) return LSM_E_INVALID_ARG;
    *out = nullptr;
    Ctx* ctx = &c->c;
    if (!verts || !tris6 || nv < 6 || nt < 4) {
        ctx->err = "mesh_upload_quadratic: need at least 6 vertices and 4 patches";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    std::vector<int32_t> h6;
    const int32_t* t6 = tris6;
    if (is_device_ptr(tris6)) {
        h6.resize(6 * (size_t)nt);
        LSM_CUDA_TRY(ctx, cudaMemcpy(h6.data(), tris6, sizeof(int32_t) * 6 * nt, cudaMemcpyDeviceToHost));
        t6 = h6.data();
    }
    std::vector<int32_t> corners(3 * (size_t)nt);
    for (int64_t j = 0; j < nt; j++)
        for (int k = 0; k < 3; k++) corners[3 * j + k] = t6[6 * j + k];
    std::string why;
    if (!check_topology(corners.data(), nt, nv, why) || !check_edge_nodes(t6, nt, nv, why)) {
        ctx->err = "mesh_upload_quadratic: " + why;
        return LSM_E_MESH;
    }
    return upload_common(ctx, verts, nv, corners.data(), nt, t6, sigma, rule, (cudaStream_t)stream, out);
}

int lsm_mesh_upload_sigmax(lsm_ctx* c, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                           double lambda, double sigma0, const lsm_quad* rule, void* stream, lsm_mesh** out)
{
    if (!c || !out) return LSM_E_INVALID_ARG;
    *out = nullptr;
    Ctx* ctx = &c->c;
    if (!verts || !tris || nv < 3 || nt < 4 || lambda < 0 || sigma0 < 0 || !std::isfinite(lambda) ||
        !std::isfinite(sigma0)) {
        ctx->err = "mesh_upload_sigmax: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    // sigma_j = D_j / lambda and the centroids, on the host
    std::vector<double> hv, sj(nt), cen(3 * (size_t)nt);
    std::vector<int32_t> ht;
    const double* vp = verts;
    const int32_t* tp = tris;
    if (is_device_ptr(verts)) {
        hv.resize(3 * (size_t)nv);
        LSM_CUDA_TRY(ctx, cudaMemcpy(hv.data(), verts, sizeof(double) * 3 * nv, cudaMemcpyDeviceToHost));
        vp = hv.data();
    }
    if (is_device_ptr(tris)) {
        ht.resize(3 * (size_t)nt);
        LSM_CUDA_TRY(ctx, cudaMemcpy(ht.data(), tris, sizeof(int32_t) * 3 * nt, cudaMemcpyDeviceToHost));
        tp = ht.data();
    }
    for (int64_t k = 0; k < 3 * nt; k++)
        if (tp[k] < 0 || tp[k] >= nv) {
            ctx->err = "mesh_upload_sigmax: vertex index out of range";
            return LSM_E_MESH;
        }
    const double lam = lambda > 0 ? lambda : 2.5;
    const double dmax = sigma_sources_host(vp, tp, nt, lam, sj.data(), cen.data());
    // default sigma0: a centroid one diameter away weighs 1/2
    const double s0 = sigma0 > 0 ? sigma0 : dmax / std::sqrt(2.0 * std::log(2.0));
    if (!(dmax > 0) || !(s0 > 0)) {
        ctx->err = "mesh_upload_sigmax: degenerate triangles";
        return LSM_E_MESH;
    }
    lsm_mesh* mh = nullptr;
    int rc = lsm_mesh_upload(c, verts, nv, tris, nt, sj.data(), rule, stream, &mh);
    if (rc != LSM_OK) return rc;
    rc = sigma_attach(ctx, &mh->m, sj.data(), cen.data(), nt, s0, (cudaStream_t)stream);
    if (rc != LSM_OK) {
        lsm_mesh_free(mh);
        return rc;
    }
    *out = mh;
    return LSM_OK;
}

int lsm_eval_sigma(lsm_mesh* mh, const double* x, int64_t n, double* sigma, double* gsigma, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (n == 0) return LSM_OK;
    if (!me->sigx || n < 0 || n >= ((int64_t)1 << 31) || !x || !sigma) {
        ctx->err = "eval_sigma: bad arguments (or not a sigma(x) mesh)";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)n;
    Scratch s(st);
    const double* xd;
    int rc = to_device(ctx, s, x, 3 * (size_t)n, &xd, st);
    if (rc) return rc;
    uint32_t* perm;
    double *T, *R;
    LSM_CUDA_TRY(ctx, s.get(&perm, n));
    LSM_CUDA_TRY(ctx, s.get(&T, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&R, 4 * (size_t)n));
    rc = morton_order_points(ctx, xd, 3, ni, perm, st);
    if (rc) return rc;
    k_gather_points<<<(ni + 255) / 256, 256, 0, st>>>(xd, perm, ni, T);
    LSM_LAUNCHED(ctx);
    Targets tg{T, n, ni};
    rc = sigma_x_eval(ctx, me, tg, R, R + n, st);
    if (rc) return rc;
    const bool sdev = is_device_ptr(sigma);
    const bool gdev = gsigma && is_device_ptr(gsigma);
    double* sd = sigma;
    double* gd = gsigma;
    if (!sdev) LSM_CUDA_TRY(ctx, s.get(&sd, n));
    if (gsigma && !gdev) LSM_CUDA_TRY(ctx, s.get(&gd, 3 * (size_t)n));
    k_scatter_results<<<(ni + 255) / 256, 256, 0, st>>>(R, perm, ni, sd, gd);
    LSM_LAUNCHED(ctx);
    if (!sdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(sigma, sd, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (gsigma && !gdev)
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(gsigma, gd, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    return check_flag(ctx, st);
}

int lsm_mesh_get_sigma0(const lsm_mesh* mh, double* sigma0)
{
    if (!mh || !sigma0) return LSM_E_INVALID_ARG;
    *sigma0 = mh->m.sigx ? mh->m.sigma0 : 0.0;
    return LSM_OK;
}

int lsm_mesh_free(lsm_mesh* mh)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    if (me->ctx) reg_remove(me->ctx, me->ctx->meshes, mh);
    DeviceGuard g(me->ctx ? me->ctx->device : 0);
    tree_free(me->tree);
    me->tree = nullptr;
    tree_free(me->tree_ff);
    me->tree_ff = nullptr;
    tree_free(me->tree_newton);
    me->tree_newton = nullptr;
    for (void* p : {(void*)me->cent, (void*)me->cent_lo, (void*)me->cent_hi})
        if (p) cudaFree(p);
    void* ps[] = {me->verts, me->tris, me->tris6, me->tri_sigma, me->tri_n, me->vpn, me->s64_pos, me->s64_nw,
                  me->s32_pos, me->s32_nw, me->s32_lo, me->s32_nwlo, me->tile_lo, me->tile_hi, me->tile_chi, me->tile_clo};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete mh;
    return LSM_OK;
}

int lsm_mesh_get_info(const lsm_mesh* mh, lsm_mesh_info* out)
{
    if (!mh || !out) return LSM_E_INVALID_ARG;
    const Mesh* me = &mh->m;
    out->n_vertices = me->nv;
    out->n_triangles = me->m;
    out->n_sources = me->ns;
    out->n_tiles = me->ntiles;
    out->device_bytes = (int64_t)me->bytes;
    out->sigma_min = me->sigma_min;
    out->sigma_max = me->sigma_max;
    return LSM_OK;
}

int lsm_eval_phi_grad(lsm_mesh* mh, const double* x, int64_t n, double* phi, double* grad, int precision,
                      void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (n == 0) return LSM_OK;
    if (n < 0 || n >= ((int64_t)1 << 31) || !x || !phi ||
        (precision != LSM_FP64 && precision != LSM_MIXED && precision != LSM_FF)) {
        ctx->err = "eval_phi_grad: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)n;
    Scratch s(st);
    const double* xd;
    int rc = to_device(ctx, s, x, 3 * (size_t)n, &xd, st);
    if (rc) return rc;
    uint32_t* perm;
    double *T, *R;
    LSM_CUDA_TRY(ctx, s.get(&perm, n));
    LSM_CUDA_TRY(ctx, s.get(&T, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&R, 4 * (size_t)n));
    rc = morton_order_points(ctx, xd, 3, ni, perm, st);
    if (rc) return rc;
    k_gather_points<<<(ni + 255) / 256, 256, 0, st>>>(xd, perm, ni, T);
    LSM_LAUNCHED(ctx);
    Targets tg{T, n, ni};
    rc = eval_sorted(ctx, me, tg, R, precision, st);
    if (rc) return rc;
    const bool phi_dev = is_device_ptr(phi);
    const bool grad_dev = grad && is_device_ptr(grad);
    double* pd = phi;
    double* gd = grad;
    if (!phi_dev) LSM_CUDA_TRY(ctx, s.get(&pd, n));
    if (grad && !grad_dev) LSM_CUDA_TRY(ctx, s.get(&gd, 3 * (size_t)n));
    k_scatter_results<<<(ni + 255) / 256, 256, 0, st>>>(R, perm, ni, pd, gd);
    LSM_LAUNCHED(ctx);
    if (!phi_dev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(phi, pd, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (grad && !grad_dev)
        LSM_CUDA_TRY(ctx, cudaMemcpyAsync(grad, gd, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (!phi_dev || (grad && !grad_dev) || !is_device_ptr(x)) return check_flag(ctx, st);
    return LSM_OK;
}

int lsm_autotune(lsm_mesh* mh, const double* x, int64_t n, double err_budget, lsm_tune_result* out, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (n < 1 || n >= ((int64_t)1 << 31) || !x || !(err_budget > 0)) {
        ctx->err = "autotune: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)n;
    Scratch s(st);
    const double* xd;
    int rc = to_device(ctx, s, x, 3 * (size_t)n, &xd, st);
    if (rc) return rc;
    uint32_t* perm;
    double* T;
    LSM_CUDA_TRY(ctx, s.get(&perm, n));
    LSM_CUDA_TRY(ctx, s.get(&T, 3 * (size_t)n));
    rc = morton_order_points(ctx, xd, 3, ni, perm, st);
    if (rc) return rc;
    k_gather_points<<<(ni + 255) / 256, 256, 0, st>>>(xd, perm, ni, T);
    LSM_LAUNCHED(ctx);
    Targets tg{T, n, ni};
    rc = autotune_sorted(ctx, me, tg, err_budget, out, st);
    if (rc) return rc;
    return check_flag(ctx, st);
}

int lsm_chart_frames(lsm_mesh* mh, int order, const double* h, const double* grad, double* xu, double* xv,
                     double* jac, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (order < 0 || order > 40 || !h || !grad || !xu || !xv || !jac) {
        ctx->err = "chart_frames: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_gl = order / 2 + 2;
    const size_t N = (size_t)me->m * n_gl * n_gl;
    Scratch s(st);
    const double *hd, *gd;
    int rc = to_device(ctx, s, h, N, &hd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, grad, 3 * N, &gd, st);
    if (rc) return rc;
    double *a = xu, *b = xv, *c = jac;
    const bool adev = is_device_ptr(xu), bdev = is_device_ptr(xv), cdev = is_device_ptr(jac);
    if (!adev) LSM_CUDA_TRY(ctx, s.get(&a, 3 * N));
    if (!bdev) LSM_CUDA_TRY(ctx, s.get(&b, 3 * N));
    if (!cdev) LSM_CUDA_TRY(ctx, s.get(&c, N));
    rc = chart_frames_dev(ctx, me, n_gl, hd, gd, a, b, c, st);
    if (rc) return rc;
    if (!adev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(xu, a, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    if (!bdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(xv, b, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    if (!cdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(jac, c, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    if (!adev || !bdev || !cdev) LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

int lsm_eval_hessian(lsm_mesh* mh, const double* x, int64_t n, double* hess, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (n == 0) return LSM_OK;
    if (n < 0 || n >= ((int64_t)1 << 31) || !x || !hess || me->sigx) {
        ctx->err = "eval_hessian: bad arguments (meshes with sigma(x) are not supported)";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)n;
    Scratch s(st);
    const double* xd;
    int rc = to_device(ctx, s, x, 3 * (size_t)n, &xd, st);
    if (rc) return rc;
    uint32_t* perm;
    double *T, *R;
    LSM_CUDA_TRY(ctx, s.get(&perm, n));
    LSM_CUDA_TRY(ctx, s.get(&T, 3 * (size_t)n));
    LSM_CUDA_TRY(ctx, s.get(&R, 6 * (size_t)n));
    rc = morton_order_points(ctx, xd, 3, ni, perm, st);
    if (rc) return rc;
    k_gather_points<<<(ni + 255) / 256, 256, 0, st>>>(xd, perm, ni, T);
    LSM_LAUNCHED(ctx);
    Targets tg{T, n, ni};
    rc = hess_sorted(ctx, me, tg, R, st);
    if (rc) return rc;
    const bool hdev = is_device_ptr(hess);
    double* hd = hess;
    if (!hdev) LSM_CUDA_TRY(ctx, s.get(&hd, 6 * (size_t)n));
    k_scatter6<<<(ni + 255) / 256, 256, 0, st>>>(R, perm, ni, hd);
    LSM_LAUNCHED(ctx);
    if (!hdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hess, hd, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
    return check_flag(ctx, st);
}

int lsm_chart_curvature(lsm_mesh* mh, int order, const double* h, const double* grad, const double* hess,
                        double* xuu, double* xuv, double* xvv, double* kmean, double* kgauss, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (order < 0 || order > 40 || !h || !grad || !hess || !xuu || !xuv || !xvv || !kmean || !kgauss) {
        ctx->err = "chart_curvature: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    if (me->tris6) {
        ctx->err = "chart_curvature: the flat-triangle form of eq. uu_vector; quadratic patches are not supported";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_gl = order / 2 + 2;
    const size_t N = (size_t)me->m * n_gl * n_gl;
    Scratch s(st);
    const double *hd, *gd, *sd;
    int rc = to_device(ctx, s, h, N, &hd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, grad, 3 * N, &gd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, hess, 6 * N, &sd, st);
    if (rc) return rc;
    double* outs[5] = {xuu, xuv, xvv, kmean, kgauss};
    const size_t cnt[5] = {3 * N, 3 * N, 3 * N, N, N};
    double* dev[5];
    bool isdev[5];
    for (int k = 0; k < 5; k++) {
        isdev[k] = is_device_ptr(outs[k]);
        dev[k] = outs[k];
        if (!isdev[k]) LSM_CUDA_TRY(ctx, s.get(&dev[k], cnt[k]));
    }
    rc = chart_second_dev(ctx, me, n_gl, hd, gd, sd, dev[0], dev[1], dev[2], dev[3], dev[4], st);
    if (rc) return rc;
    bool any_host = false;
    for (int k = 0; k < 5; k++)
        if (!isdev[k]) {
            any_host = true;
            LSM_CUDA_TRY(ctx, cudaMemcpyAsync(outs[k], dev[k], sizeof(double) * cnt[k], cudaMemcpyDeviceToHost, st));
        }
    if (any_host) LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

int lsm_gauss_flux(lsm_mesh* mh, int order, const double* x, const double* grad, const double* jac,
                   const double* x0, double* eps0, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (order < 0 || order > 40 || !x || !grad || !jac || !x0 || !eps0) {
        ctx->err = "gauss_flux: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_gl = order / 2 + 2;
    const size_t N = (size_t)me->m * n_gl * n_gl;
    Scratch s(st);
    const double *xd, *gd, *jd;
    int rc = to_device(ctx, s, x, 3 * N, &xd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, grad, 3 * N, &gd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, jac, N, &jd, st);
    if (rc) return rc;
    return gauss_flux_dev(ctx, me, n_gl, xd, gd, jd, x0, eps0, st);
}

int lsm_refined_nodes(int order, int64_t m, const int32_t* level, int32_t* tri, double* uvw, int64_t* n_out)
{
    if (order < 0 || order > 40 || m < 1 || !level || !n_out) return LSM_E_INVALID_ARG;
    const int n_gl = order / 2 + 2;
    int64_t n = 0;
    for (int64_t j = 0; j < m; j++) {
        if (level[j] < 0 || level[j] > 4) return LSM_E_INVALID_ARG;
        n += (int64_t)n_gl * n_gl << (2 * level[j]);
    }
    *n_out = n;
    if (!tri || !uvw) return LSM_OK;
    std::vector<double> rules[5];
    int64_t k = 0;
    for (int64_t j = 0; j < m; j++) {
        const int L = level[j];
        if (rules[L].empty()) {
            rules[L].resize(3 * ((size_t)n_gl * n_gl << (2 * L)));
            simplex_rule_host(n_gl, L, rules[L].data());
        }
        const int64_t cnt = (int64_t)rules[L].size() / 3;
        for (int64_t i = 0; i < cnt; i++, k++) {
            tri[k] = (int32_t)j;
            for (int c = 0; c < 3; c++) uvw[3 * k + c] = rules[L][3 * i + c];
        }
    }
    return LSM_OK;
}

namespace {
// Copy explicit nodes to the device and check their triangles.
int node_spec(Ctx* ctx, Scratch& s, const Mesh* me, int64_t n, const int32_t* tri, const double* uvw, NodeSpec* out,
              cudaStream_t st)
{
    if (n < 1 || n >= ((int64_t)1 << 31) || !tri || !uvw) {
        ctx->err = "chart nodes: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    std::vector<int32_t> ht;
    const int32_t* tp = tri;
    if (is_device_ptr(tri)) {
        ht.resize((size_t)n);
        LSM_CUDA_TRY(ctx, cudaMemcpy(ht.data(), tri, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
        tp = ht.data();
    }
    for (int64_t k = 0; k < n; k++)
        if (tp[k] < 0 || tp[k] >= me->m) {
            ctx->err = "chart nodes: triangle index out of range";
            return LSM_E_INVALID_ARG;
        }
    const int32_t* td;
    const double* ud;
    int rc = to_device(ctx, s, tri, (size_t)n, &td, st);
    if (rc) return rc;
    rc = to_device(ctx, s, uvw, 3 * (size_t)n, &ud, st);
    if (rc) return rc;
    *out = NodeSpec{n, td, ud};
    return LSM_OK;
}
}  // namespace

int lsm_solve_charts_nodes(lsm_mesh* mh, int64_t n, const int32_t* tri, const double* uvw, double tol, int max_iter,
                           int precision, double* x_out, double* h_out, int32_t* status, lsm_solve_stats* stats,
                           void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (!(tol > 0) || max_iter < 1 || max_iter > 1000 || (precision != LSM_FP64 && precision != LSM_MIXED)) {
        ctx->err = "solve_charts_nodes: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s(st);
    NodeSpec spec;
    int rc = node_spec(ctx, s, me, n, tri, uvw, &spec, st);
    if (rc) return rc;
    double *xo = x_out, *ho = h_out;
    int32_t* so = status;
    const bool xdev = x_out && is_device_ptr(x_out);
    const bool hdev = h_out && is_device_ptr(h_out);
    const bool sdev = status && is_device_ptr(status);
    if (!xdev) LSM_CUDA_TRY(ctx, s.get(&xo, 3 * (size_t)n));
    if (!hdev) LSM_CUDA_TRY(ctx, s.get(&ho, (size_t)n));
    if (!sdev) LSM_CUDA_TRY(ctx, s.get(&so, (size_t)n));
    rc = solve_charts_device(ctx, me, 1, tol, max_iter, precision, xo, ho, so, stats, st, &spec);
    if (rc) return rc;
    if (x_out && !xdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(x_out, xo, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
    if (h_out && !hdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(h_out, ho, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (status && !sdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(status, so, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    return check_flag(ctx, st);
}

int lsm_chart_frames_nodes(lsm_mesh* mh, int64_t n, const int32_t* tri, const double* uvw, const double* h,
                           const double* grad, double* xu, double* xv, double* jac, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (!h || !grad || !xu || !xv || !jac) {
        ctx->err = "chart_frames_nodes: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s(st);
    NodeSpec spec;
    int rc = node_spec(ctx, s, me, n, tri, uvw, &spec, st);
    if (rc) return rc;
    const size_t N = (size_t)n;
    const double *hd, *gd;
    rc = to_device(ctx, s, h, N, &hd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, grad, 3 * N, &gd, st);
    if (rc) return rc;
    double *a = xu, *b = xv, *c = jac;
    const bool adev = is_device_ptr(xu), bdev = is_device_ptr(xv), cdev = is_device_ptr(jac);
    if (!adev) LSM_CUDA_TRY(ctx, s.get(&a, 3 * N));
    if (!bdev) LSM_CUDA_TRY(ctx, s.get(&b, 3 * N));
    if (!cdev) LSM_CUDA_TRY(ctx, s.get(&c, N));
    rc = chart_frames_dev(ctx, me, 1, hd, gd, a, b, c, st, &spec);
    if (rc) return rc;
    if (!adev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(xu, a, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    if (!bdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(xv, b, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    if (!cdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(jac, c, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

int lsm_gauss_flux_nodes(lsm_mesh* mh, int64_t n, const int32_t* tri, const double* uvw, const double* x,
                         const double* grad, const double* jac, const double* x0, double* eps0, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (!x || !grad || !jac || !x0 || !eps0) {
        ctx->err = "gauss_flux_nodes: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Scratch s(st);
    NodeSpec spec;
    int rc = node_spec(ctx, s, me, n, tri, uvw, &spec, st);
    if (rc) return rc;
    const size_t N = (size_t)n;
    const double *xd, *gd, *jd;
    rc = to_device(ctx, s, x, 3 * N, &xd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, grad, 3 * N, &gd, st);
    if (rc) return rc;
    rc = to_device(ctx, s, jac, N, &jd, st);
    if (rc) return rc;
    return gauss_flux_dev(ctx, me, 1, xd, gd, jd, x0, eps0, st, &spec);
}

int lsm_solve_charts(lsm_mesh* mh, int order, double tol, int max_iter, int precision, double* x_out,
                     double* h_out, int32_t* status, lsm_solve_stats* stats, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    if (order < 0 || order > 40 || !(tol > 0) || max_iter < 1 || max_iter > 1000 ||
        (precision != LSM_FP64 && precision != LSM_MIXED)) {
        ctx->err = "solve_charts: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_gl = order / 2 + 2;
    const int64_t N = me->m * (int64_t)n_gl * n_gl;
    Scratch s(st);
    double *xo = x_out, *ho = h_out;
    int32_t* so = status;
    const bool xdev = x_out && is_device_ptr(x_out);
    const bool hdev = h_out && is_device_ptr(h_out);
    const bool sdev = status && is_device_ptr(status);
    if (!xdev) LSM_CUDA_TRY(ctx, s.get(&xo, 3 * (size_t)N));
    if (!hdev) LSM_CUDA_TRY(ctx, s.get(&ho, (size_t)N));
    if (!sdev) LSM_CUDA_TRY(ctx, s.get(&so, (size_t)N));
    int rc = solve_charts_device(ctx, me, n_gl, tol, max_iter, precision, xo, ho, so, stats, st);
    if (rc) return rc;
    if (x_out && !xdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(x_out, xo, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    if (h_out && !hdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(h_out, ho, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    if (status && !sdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(status, so, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    return check_flag(ctx, st);
}

int lsm_eval_phi_grad_noalloc(lsm_mesh* mh, const double* x, int64_t n, double* phi, double* grad,
                              int precision, void* stream)
{
    if (!mh) return LSM_E_INVALID_ARG;
    Mesh* me = &mh->m;
    Ctx* ctx = me->ctx;
    DeviceGuard g(ctx->device);
    return eval_noalloc(ctx, me, x, n, phi, grad, precision, (cudaStream_t)stream);
}

int lsm_batch_create(lsm_ctx* c, lsm_mesh* const* meshes, int n, void* stream, lsm_batch** out)
{
    if (!c || !out || !meshes || n < 1) return LSM_E_INVALID_ARG;
    *out = nullptr;
    Ctx* ctx = &c->c;
    DeviceGuard g(ctx->device);
    for (int i = 0; i < n; i++)
        if (!meshes[i]) {
            ctx->err = "batch_create: null mesh";
            return LSM_E_INVALID_ARG;
        }
    lsm_batch* bh = new (std::nothrow) lsm_batch();
    if (!bh) return LSM_E_OOM;
    int rc = batch_build(ctx, &bh->b, meshes, n, (cudaStream_t)stream);
    if (rc) {
        batch_release(&bh->b);
        delete bh;
        return rc;
    }
    reg_add(ctx, ctx->batches, bh);
    *out = bh;
    return LSM_OK;
}

int lsm_batch_free(lsm_batch* bh)
{
    if (!bh) return LSM_E_INVALID_ARG;
    if (bh->b.ctx) reg_remove(bh->b.ctx, bh->b.ctx->batches, bh);
    DeviceGuard g(bh->b.ctx ? bh->b.ctx->device : 0);
    batch_release(&bh->b);
    delete bh;
    return LSM_OK;
}

int lsm_batch_solve_charts(lsm_batch* bh, int order, double tol, int max_iter, int precision, int use_graph,
                           double* x_out, double* h_out, int32_t* status, lsm_solve_stats* stats, void* stream)
{
    if (!bh) return LSM_E_INVALID_ARG;
    Batch* b = &bh->b;
    Ctx* ctx = b->ctx;
    if (order < 0 || order > 40 || !(tol > 0) || max_iter < 1 || max_iter > 1000 ||
        (precision != LSM_FP64 && precision != LSM_MIXED)) {
        ctx->err = "batch_solve_charts: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int n_gl = order / 2 + 2;
    const int64_t N = b->m * (int64_t)n_gl * n_gl;
    Scratch s(st);
    double *xo = x_out, *ho = h_out;
    int32_t* so = status;
    const bool xdev = x_out && is_device_ptr(x_out);
    const bool hdev = h_out && is_device_ptr(h_out);
    const bool sdev = status && is_device_ptr(status);
    if (!xdev) LSM_CUDA_TRY(ctx, s.get(&xo, 3 * (size_t)N));
    if (!hdev) LSM_CUDA_TRY(ctx, s.get(&ho, (size_t)N));
    if (!sdev) LSM_CUDA_TRY(ctx, s.get(&so, (size_t)N));
    int rc = solve_charts_batch(ctx, b, n_gl, tol, max_iter, precision, use_graph, xo, ho, so, stats, st);
    if (rc) return rc;
    if (x_out && !xdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(x_out, xo, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
    if (h_out && !hdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(h_out, ho, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    if (status && !sdev) LSM_CUDA_TRY(ctx, cudaMemcpyAsync(status, so, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st));
    return check_flag(ctx, st);
}

int lsm_batch_autotune(lsm_batch* bh, int order, double err_budget, lsm_tune_result* out, void* stream)
{
    if (!bh) return LSM_E_INVALID_ARG;
    Batch* b = &bh->b;
    Ctx* ctx = b->ctx;
    if (order < 0 || order > 40 || !(err_budget > 0)) {
        ctx->err = "batch_autotune: bad arguments";
        return LSM_E_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = batch_autotune(ctx, b, order / 2 + 2, err_budget, out, st);
    if (rc) return rc;
    return check_flag(ctx, st);
}

}  // extern "C"
