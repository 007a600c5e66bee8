// lsm_internal.cuh -- internal types and helpers of liblsm (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <string>
#include <utility>
#include <vector>

#include "lsm.h"

struct lsm_mesh;
struct lsm_batch;
struct lsm_server;

namespace lsm {

// Source nodes per tile.  Tiles are runs of consecutive Morton-sorted source
// nodes; a tile is the unit of the near/far decision and of shared-memory
// staging in the pair kernels.
constexpr int kTile = 128;
// Targets per thread block row of the pair kernels (threads * targets/thread).
constexpr int kEvalThreads = 128;
// Largest Chebyshev degree of the treecode's proxy grids.
constexpr int kTreeMaxDegree = 16;

// Last-error messages of a context, one per host thread: a call records its
// message for the thread that made it, so that threads sharing a context
// (the server's worker slots) never read each other's messages.  c_str()
// returns a copy taken under the lock, owned by the calling thread and valid
// until its next c_str() call.
class ErrorText {
public:
    ErrorText& operator=(const std::string& s) {
        std::lock_guard<std::mutex> lk(mu_);
        text_[std::this_thread::get_id()] = s;
        return *this;
    }
    const char* c_str() const {
        thread_local std::string copy;
        std::lock_guard<std::mutex> lk(mu_);
        auto it = text_.find(std::this_thread::get_id());
        copy = it == text_.end() ? std::string() : it->second;
        return copy.c_str();
    }

private:
    mutable std::mutex mu_;
    std::map<std::thread::id, std::string> text_;
};

struct Ctx {
    int device = 0;
    int num_sms = 0;
    lsm_options opt{};
    ErrorText err;
    std::atomic<int64_t> launches{0};
    int* d_flag = nullptr;   // device error word (bounded waits); see flag_word()
    bool test_nocopy = false;  // test hook: pair kernels arm their first stage without copying
    unsigned long long* d_pairs = nullptr;  // [4 kinds][2]: pairs in near / far tiles
    bool profiling = false;
    struct ProfEvent {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<ProfEvent> prof_events;
    double prof_ms[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t prof_launches[4] = {0, 0, 0, 0};
    // pinned host blocks of kHostWords int32 for counts read back by the
    // solves; several solves may run at once on one context (server slots),
    // so each takes its own block and returns it (freed at lsm_destroy)
    static constexpr int kHostWords = 64;
    std::mutex host_mu;
    std::vector<int32_t*> host_free;
    // handles made from this context and not yet freed; lsm_destroy frees
    // them, so that none outlives the context it points to
    std::mutex reg_mu;
    std::set<lsm_mesh*> meshes;
    std::set<lsm_batch*> batches;
    std::set<lsm_server*> servers;
};

// Device error word of the calling thread: a thread that installed its own
// word for this context (FlagScope) gets that one, every other thread the
// context's.  Kernels launched by the thread set it; check_flag reads it.
struct FlagOverride {
    const Ctx* ctx = nullptr;
    int* flag = nullptr;
};
inline FlagOverride& flag_override()
{
    thread_local FlagOverride f;
    return f;
}
inline int* flag_word(Ctx* ctx)
{
    const FlagOverride& f = flag_override();
    return f.ctx == ctx && f.flag ? f.flag : ctx->d_flag;
}
// Installs `flag` as the calling thread's error word of ctx for its lifetime.
struct FlagScope {
    FlagOverride saved;
    FlagScope(const Ctx* ctx, int* flag) : saved(flag_override()) { flag_override() = FlagOverride{ctx, flag}; }
    ~FlagScope() { flag_override() = saved; }
};

// A pinned block from the context's pool, returned to it on scope exit.
struct HostWords {
    Ctx* ctx;
    int32_t* p = nullptr;
    explicit HostWords(Ctx* c) : ctx(c) {}
    cudaError_t get() {
        {
            std::lock_guard<std::mutex> lk(ctx->host_mu);
            if (!ctx->host_free.empty()) {
                p = ctx->host_free.back();
                ctx->host_free.pop_back();
                return cudaSuccess;
            }
        }
        return cudaMallocHost(&p, sizeof(int32_t) * Ctx::kHostWords);
    }
    ~HostWords() {
        if (!p) return;
        std::lock_guard<std::mutex> lk(ctx->host_mu);
        ctx->host_free.push_back(p);
    }
};

struct Tree;

struct Mesh {
    Ctx* ctx = nullptr;
    Tree* tree = nullptr;        // treecode far field of the mixed path, built on first use
    Tree* tree_ff = nullptr;     // and of the float-float path
    Tree* tree_newton = nullptr; // the coarser mixed treecode of the mixed Newton sweeps
    // target-dependent sigma (eq. sigma2): centroids in Morton order (x, y, z,
    // sigma_j), in tiles of kTile with outward-rounded boxes
    bool sigx = false;
    double sigma0 = 0.0;
    int64_t ncent = 0, ncent_tiles = 0;
    double4_32a* cent = nullptr;
    float4 *cent_lo = nullptr, *cent_hi = nullptr;
    // far-field choice stored by the autotuner: -1 follow the context's
    // options, 0 direct, 1 treecode with tune_degree / tune_theta
    int tune_mode = -1;
    int tune_degree = 0;
    float tune_theta = 0.0f;
    // and its near-field radius (in sigma) and targets per CTA of the mixed
    // kernel (64, 128 or 256; 0: the context's cutoff_mixed, 256)
    double tune_cut = 0.0;
    int tune_tpb = 0;
    int64_t nv = 0, m = 0, ns = 0, ntiles = 0;
    int nq = 0;
    lsm_quad rule{4, 0};
    double sigma_min = 0, sigma_max = 0;
    size_t bytes = 0;
    // geometry, triangle order of the input
    double* verts = nullptr;     // [nv][3]
    int32_t* tris = nullptr;     // [m][3]
    double* tri_sigma = nullptr; // [m]
    double* tri_n = nullptr;     // [m][3] N = T_u x T_v (not normalised)
    double* vpn = nullptr;       // [nv][3] vertex pseudonormals
    // quadratic skeletons (Sec. 5, quadratic skeletons): [m][6] patch nodes,
    // the corners (also in tris) then the nodes of edges 1-2, 2-3, 3-1;
    // nullptr for flat triangles
    int32_t* tris6 = nullptr;
    // sources in Morton order
    double4_32a* s64_pos = nullptr;  // (x, y, z, a = 1/(sqrt2 sigma))
    double4_32a* s64_nw = nullptr;   // (nw / 4 pi, 0)
    float4* s32_pos = nullptr;   // (y - c_tile in FP32, a)
    float4* s32_nw = nullptr;    // (nw / 4 pi, sqrt2 sigma) in FP32
    float4* s32_lo = nullptr;    // FP32 remainders of the tile-local position and of a
    float4* s32_nwlo = nullptr;  // FP32 remainder of nw / 4 pi, 0 (float-float kernel)
    float4* tile_lo = nullptr;   // bbox lower corner rounded down, w = sigma_max rounded up
    float4* tile_hi = nullptr;   // bbox upper corner rounded up, w = number of nodes in the tile
    float4* tile_chi = nullptr;  // tile centre, FP32 high part
    float4* tile_clo = nullptr;  // tile centre, FP32 remainder
};

// Many meshes evaluated and solved together: their tiles and geometry are
// concatenated (each mesh's sources start on a tile boundary).
struct Batch {
    Ctx* ctx = nullptr;
    int nmesh = 0;
    int64_t nv = 0, m = 0, ntiles = 0;
    size_t bytes = 0;
    double* verts = nullptr;     // [nv][3]
    int32_t* tris = nullptr;     // [m][3], global vertex indices
    double* tri_sigma = nullptr; // [m]
    double* vpn = nullptr;       // [nv][3]
    int32_t* tri_mesh = nullptr; // [m] mesh of each triangle
    float4 *s32_pos = nullptr, *s32_nw = nullptr, *s32_lo = nullptr, *s32_nwlo = nullptr;
    double4_32a *s64_pos = nullptr, *s64_nw = nullptr;
    float4 *tile_lo = nullptr, *tile_hi = nullptr, *tile_chi = nullptr, *tile_clo = nullptr;
    int2* mesh_tiles = nullptr;  // [nmesh] (first tile, end tile)
    std::vector<int64_t> tri_off;  // host [nmesh + 1]
    // mixed kernel settings chosen by lsm_batch_autotune (0: defaults): the
    // near-field radius and the targets per work item (64, 128 or 256)
    double cut_mixed = 0.0;
    int tpb = 0;
};

// ---------------------------------------------------------------- patch map
// T(u,v), T_u and T_v of skeleton triangle j.  Flat triangles (tris6 null):
// T = P1 + u (P2 - P1) + v (P3 - P1) (eq. tparam).  Quadratic patches: the
// second-order Lagrange interpolant through the corners P1, P2, P3 and the
// edge nodes P4 (edge 1-2), P5 (2-3), P6 (3-1), written in monomials,
//   T = P1 + u A + v B + u^2 C + u v D + v^2 E,
//   A = 4 P4 - 3 P1 - P2,  B = 4 P6 - 3 P1 - P3,  C = 2 (P1 + P2 - 2 P4),
//   D = 4 (P1 - P4 + P5 - P6),  E = 2 (P1 + P3 - 2 P6),
// which reduces to the flat map when the edge nodes are the midpoints.
__device__ __forceinline__ void patch_map(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                                          const int32_t* __restrict__ tris6, int64_t j, double u, double v,
                                          double T[3], double Tu[3], double Tv[3])
{
    if (!tris6) {
        const int64_t a = tris[3 * j], b = tris[3 * j + 1], c = tris[3 * j + 2];
        for (int k = 0; k < 3; k++) {
            const double p1 = verts[3 * a + k];
            Tu[k] = verts[3 * b + k] - p1;
            Tv[k] = verts[3 * c + k] - p1;
            T[k] = p1 + u * Tu[k] + v * Tv[k];
        }
        return;
    }
    const int32_t* q = tris6 + 6 * j;
    for (int k = 0; k < 3; k++) {
        const double p1 = verts[3 * (int64_t)q[0] + k], p2 = verts[3 * (int64_t)q[1] + k],
                     p3 = verts[3 * (int64_t)q[2] + k], p4 = verts[3 * (int64_t)q[3] + k],
                     p5 = verts[3 * (int64_t)q[4] + k], p6 = verts[3 * (int64_t)q[5] + k];
        const double A = 4.0 * p4 - 3.0 * p1 - p2, B = 4.0 * p6 - 3.0 * p1 - p3;
        const double C = 2.0 * (p1 + p2 - 2.0 * p4), D = 4.0 * (p1 - p4 + p5 - p6), E = 2.0 * (p1 + p3 - 2.0 * p6);
        T[k] = p1 + u * (A + u * C + v * D) + v * (B + v * E);
        Tu[k] = A + 2.0 * u * C + v * D;
        Tv[k] = B + u * D + 2.0 * v * E;
    }
}

// ---------------------------------------------------------------- errors
#define LSM_CUDA_TRY(ctx, call)                                                   \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            return LSM_E_CUDA;                                                    \
        }                                                                         \
    } while (0)

#define LSM_LAUNCHED(ctx)                                                         \
    do {                                                                          \
        cudaError_t e_ = cudaGetLastError();                                      \
        (ctx)->launches++;                                                        \
        if (e_ != cudaSuccess) {                                                  \
            (ctx)->err = std::string("kernel launch: ") + cudaGetErrorString(e_); \
            return LSM_E_CUDA;                                                    \
        }                                                                         \
    } while (0)

// ---------------------------------------------------------------- scratch
// Stream-ordered scratch allocation for one call.
struct Scratch {
    static constexpr int kMax = 64;
    cudaStream_t st;
    void* ptrs[kMax];
    int n = 0;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <class T>
    cudaError_t get(T** p, size_t count) {
        if (n >= kMax) return cudaErrorMemoryAllocation;
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, count * sizeof(T) + 16, st);
        if (e != cudaSuccess) return e;
        ptrs[n++] = q;
        *p = reinterpret_cast<T*>(q);
        return cudaSuccess;
    }
    ~Scratch() {
        for (int i = 0; i < n; i++) cudaFreeAsync(ptrs[i], st);
    }
};

// ---------------------------------------------------------------- launches
// sort.cu
int radix_sort_pairs(Ctx* ctx, uint32_t* keys, uint32_t* vals, int n, int key_bits,
                     cudaStream_t st);
int compact_flags(Ctx* ctx, const int32_t* flags, int want, const int32_t* in, int n,
                  int32_t* out, int32_t* d_count, cudaStream_t st);
int scan_exclusive(Ctx* ctx, uint32_t* a, int64_t len, uint32_t* total, cudaStream_t st);
int compact_blocks(int n_max);
int compact_flags_dev(Ctx* ctx, const int32_t* flags, int want, const int32_t* in, const int* n_dev, int n_max,
                      int32_t* out, int32_t* d_count, uint32_t* bc, cudaStream_t st);

// geometry.cu
int build_mesh_device(Ctx* ctx, Mesh* mesh, const double* sigma_in_dev, const double* rule_dev,
                      double* host_vol, cudaStream_t st);
int morton_order_points(Ctx* ctx, const double* pts, int stride, int n, uint32_t* perm,
                        cudaStream_t st);
int chart_nodes_init(Ctx* ctx, const Mesh* mesh, const double* chart_rule_dev, int np,
                     double* x0, double* hdir, double* sloc, cudaStream_t st);
// chart nodes at explicit (triangle, parent u, v) (device arrays)
int chart_nodes_at(Ctx* ctx, const Mesh* mesh, int64_t n, const int32_t* tri, const double* uvw, double* x0,
                   double* hdir, double* sloc, cudaStream_t st);
int chart_nodes_raw(Ctx* ctx, const double* verts, const int32_t* tris, const double* vpn, const double* tri_sigma,
                    int64_t m, const double* chart_rule_dev, int np, double* x0, double* hdir, double* sloc,
                    cudaStream_t st);

// Source-side arrays the pair kernels read: one mesh, or a batch of meshes
// whose tiles are concatenated.
struct SourceView {
    const float4 *s32_pos, *s32_nw, *s32_lo, *s32_nwlo;
    const double4_32a *s64_pos, *s64_nw;
    const float4 *tile_lo, *tile_hi, *tile_chi, *tile_clo;
    int ntiles;
};
inline SourceView view_of(const Mesh* m)
{
    return SourceView{m->s32_pos, m->s32_nw, m->s32_lo, m->s32_nwlo, m->s64_pos, m->s64_nw,
                      m->tile_lo, m->tile_hi, m->tile_chi, m->tile_clo, (int)m->ntiles};
}
inline SourceView view_of_batch(const Batch* b)
{
    return SourceView{b->s32_pos, b->s32_nw, b->s32_lo, b->s32_nwlo, b->s64_pos, b->s64_nw,
                      b->tile_lo, b->tile_hi, b->tile_chi, b->tile_clo, (int)b->ntiles};
}

// eval.cu
// Explicit chart nodes (device arrays): node s in triangle tri[s] at parent
// coordinates uvw[3s], uvw[3s+1]; replaces the rule of order n_gl
// (weight uvw[3s+2]).
struct NodeSpec {
    int64_t n;
    const int32_t* tri;
    const double* uvw;
};

struct Targets {
    const double* x;  // SoA: x[0..n), y = x + ld, z = x + 2 ld
    int64_t ld;
    int n;
};
int eval_init_constants(Ctx* ctx);
// Float-float evaluation in two calls on the same targets: mode 1 records the
// far-tile part of Phi and grad Phi into far_io [4][n]; mode 2 then
// evaluates only the near tiles and adds the recorded far part moved to the
// new positions along its gradient (x_old = the targets of the mode 1 call).
// bb_io [grid blocks][8]: mode 1 stores each block's box (and its largest
// sigma in sigma(x) mode), mode 2 reuses it, so both calls split near and far
// tiles identically however little the targets moved.
// Internal precision code for eval_sorted: the mixed path as the mixed Newton
// sweeps of a chart solve that finishes with float-float steps take it (their
// own coarser treecode where newton_tree_wanted)
constexpr int kPrecMixedNewton = 16;
struct FFIncremental {
    int mode;
    double* far_io;
    const double* x_old;
    float* bb_io = nullptr;
};
int eval_sorted(Ctx* ctx, const Mesh* mesh, const Targets& t, double* res, int precision,
                cudaStream_t st, const FFIncremental* inc = nullptr);
// Targets grouped by work items (int4: first target, count, first tile, end
// tile; at most eval_item_targets(ctx, precision, tpb) targets each); the
// number of items is read on the device from *n_items, the grid covers
// max_items.  tpb: targets per item of the mixed kernel (64, 128 or 256; 0
// the default 256; the float-float kernel takes the context's ff_block);
// cut: its near-field radius in sigma (0: the context's cutoff_mixed)
int eval_item_targets(const Ctx* ctx, int precision, int tpb = 0);
int eval_items(Ctx* ctx, const SourceView& v, const Targets& t, const int4* items, const int* n_items,
               int max_items, double* res, int precision, cudaStream_t st, const FFIncremental* inc = nullptr,
               int tpb = 0, double cut = 0.0);
// the mixed kernel's settings for a mesh: its autotuned ones, else the defaults
int mixed_tpb(const Ctx* ctx, const Mesh* me);   // targets per CTA of the mixed kernel on this mesh
double mixed_cut(const Ctx* ctx, const Mesh* me);
int eval_noalloc(Ctx* ctx, const Mesh* mesh, const double* x, int64_t n, double* phi, double* grad,
                 int precision, cudaStream_t st);

// tree.cu
// The treecode of a mesh: node boxes over Morton-ordered source tiles and the
// proxy tiles (Chebyshev points with interpolated dipole weights) of the
// nodes large enough to profit.  Tile ids below ntiles are source tiles,
// the rest proxy tiles; tile_* cover both.
struct Tree {
    bool ff = false;                        // float-float proxies (FP64 weights split in two floats)
    int degree = 0;
    float theta = 0.0f;
    int grid = 1;                           // 1 oriented per-axis grids and a degree ladder, 2 full (degree + 1)^3 grids
    int top = 0;                            // level of the root (level 0 = tiles)
    int64_t lev_off[33] = {0};              // first node of each level
    int64_t nnodes = 0;
    int ntiles = 0, nptiles = 0;
    float4* node_lo = nullptr;              // box, rounded down; w = sigma_max
    float4* node_hi = nullptr;              // box, rounded up
    int4* node_info = nullptr;              // first tile, tile count, first proxy tile or -1, proxy tiles
    float4* node_acc = nullptr;             // proxy nodes: frame centre, (radius / theta_n)^2
    float* node_r = nullptr;                // proxy nodes: radius of the frame box, rounded up
    float4 *p_pos = nullptr, *p_nw = nullptr;   // proxies, kTile per proxy tile
    float4 *p_lo = nullptr, *p_nwlo = nullptr;  // float-float trees: remainders of both
    float4 *tile_lo = nullptr, *tile_hi = nullptr, *tile_chi = nullptr, *tile_clo = nullptr;
    size_t bytes = 0;
};
bool tree_wanted(const Ctx* ctx, const Mesh* me, bool ff);
// newton: the mixed Newton sweeps' own treecode (options newton_tree_*)
int tree_ensure(Ctx* ctx, Mesh* me, cudaStream_t st, bool ff, bool newton = false);
// True when the mixed Newton sweeps take their own treecode: on, and coarser
// than the mesh's mixed treecode (lower degree or larger opening parameter,
// neither finer)
bool newton_tree_wanted(const Ctx* ctx, const Mesh* me);
void tree_free(Tree* t);
// Interaction lists of sorted targets in blocks of tpb: for block b, the
// tile ids list[blist[b].x .. + blist[b].y) in tree order; order = the
// blocks by decreasing list length (the launch order); *total = the summed
// list length.
// tsig: the targets' sigma in sigma(x) mode (the near width), else NULL.
// cut_override > 0: the near radius (in sigma) of the kernel that evaluates
// the lists, when it is not the tree's own path's.
// Target clusters of one evaluation (float-float treecode): runs of `tpc`
// consecutive sorted targets, each with an oriented box and a tensor
// Chebyshev grid on it.  A source node far enough from a cluster acts on the
// cluster's grid points (through its proxies), and the cluster's targets
// interpolate that field from the grid (cluster_l2p); the targets' own
// block lists skip such nodes.  Device arrays in the caller's Scratch.
struct ClusterPlan {
    int tpc = 0;                 // targets per cluster (0: no clusters)
    int ncl = 0;
    float4 *box_lo = nullptr, *box_hi = nullptr;   // outward box of each cluster's oriented box
    float4* cacc = nullptr;      // frame centre, (r + q h_max)^2: the target-side opening radius
    double* frame = nullptr;     // [ncl][16]: centre (3), axes (9, rows), half-widths (3), unused
    int4* counts = nullptr;      // grid points per axis; w = first grid point (padded to a block)
    int64_t ng = 0;              // grid points, padded
    double* gx = nullptr;        // grid points, SoA [3][ng]
    int* list = nullptr;         // proxy tiles acting on each cluster's grid
    int2* gblist = nullptr;      // per block of grid points: its cluster's (offset, length) in list
    int* gorder = nullptr;       // grid blocks in launch order
    int ngblk = 0;
    int64_t total = 0;           // summed length of the clusters' lists
    float4 *blo = nullptr, *bhi = nullptr;   // the target blocks' boxes
    uint32_t* cbits = nullptr;   // [ncl][cwords]: bit `node` set when the cluster took the node
    int64_t cwords = 0;
};
// tpb: targets per block of the pair kernel that evaluates the lists (and
// the grid points); cut: its near radius in sigma; tsig: the sorted targets'
// sigma in sigma(x) mode (the near width of a cluster or block is then its
// largest target sigma), else null
int cluster_setup(Ctx* ctx, const Tree* tree, const Targets& t, int tpc, int tpb, double cut, const double* tsig,
                  Scratch& s, ClusterPlan* plan, cudaStream_t st);
// Adds the clusters' interpolated far field to res [4][n] (and to far_io [4][n]
// when not null) from the grid values rg [4][ng].
int cluster_l2p(Ctx* ctx, const ClusterPlan& plan, const Targets& t, const double* rg, double* res,
                double* far_io, cudaStream_t st);
int tree_lists(Ctx* ctx, const Tree* tree, const Targets& t, int tpb, const double* tsig, Scratch& s, int** list,
               int2** blist, int** order, int64_t* total, cudaStream_t st, double cut_override = 0.0,
               const ClusterPlan* clusters = nullptr);

// frames.cu: chart local coordinates and the Gauss flux (lsm_chart_frames,
// lsm_gauss_flux); all arrays on the device, nodes in solve order
// spec: explicit nodes (their parent u, v and weight in uvw) instead of the rule
int chart_frames_dev(Ctx* ctx, const Mesh* me, int n_gl, const double* h, const double* g, double* xu, double* xv,
                     double* jac, cudaStream_t st, const NodeSpec* spec = nullptr);
int gauss_flux_dev(Ctx* ctx, const Mesh* me, int n_gl, const double* x, const double* g, const double* jac,
                   const double* x0, double* eps0, cudaStream_t st, const NodeSpec* spec = nullptr);
// per-triangle sums of the Gauss flux terms (device arrays; nodes grouped by
// triangle, triangle j's nodes [off[j], off[j+1]), weights uvw[3s+2]); x0 host
int flux_per_triangle_dev(Ctx* ctx, int64_t m, const int64_t* off, const double* x, const double* g, const double* jac,
                          const double* uvw, const double* x0, double* out, cudaStream_t st);

// eval.cu: H(w) = g(u)/u^3 in long double, and the degree-6 interpolant of H
// on interval k of width 1/per_unit in w (monomial coefficients about its
// centre)
long double h_of_w(long double w);
void h_interval_fit(int k, int per_unit, long double* cf);

// hess.cu: the Hessian of Phi [6][n] (xx, xy, xz, yy, yz, zz) at sorted
// targets (per-triangle sigma meshes)
int hess_sorted(Ctx* ctx, const Mesh* me, const Targets& t, double* res, cudaStream_t st);
// frames.cu: chart second derivatives and curvatures; device arrays, nodes in
// solve order
int chart_second_dev(Ctx* ctx, const Mesh* me, int n_gl, const double* h, const double* g, const double* hess,
                     double* xuu, double* xuv, double* xvv, double* kmean, double* kgauss, cudaStream_t st);

// sigma.cu: target-dependent sigma (eq. sigma2)
double sigma_sources_host(const double* verts, const int32_t* tris, int64_t nt, double lambda, double* sj,
                          double* cen);
int sigma_attach(Ctx* ctx, Mesh* me, const double* sj, const double* cen, int64_t nt, double sigma0,
                 cudaStream_t st);
// sigma(x) [n] and grad sigma [3][n] (SoA) at sorted targets, for the pair
// kernels of `precision` (LSM_FP64: FP64 sums; else float-float sums)
int sigma_x_eval(Ctx* ctx, const Mesh* me, const Targets& t, double* sig, double* gsig, cudaStream_t st,
                 int precision = LSM_FP64);

// tune.cu: the autotuner on sorted SoA targets (lsm_autotune)
int autotune_sorted(Ctx* ctx, Mesh* me, const Targets& t, double budget, lsm_tune_result* res, cudaStream_t st);
// the batch's mixed-kernel radius and target tile (lsm_batch_autotune)
int batch_autotune(Ctx* ctx, Batch* b, int n_gl, double budget, lsm_tune_result* res, cudaStream_t st);

// newton.cu
int solve_charts_device(Ctx* ctx, Mesh* mesh, int n_gl, double tol, int max_iter,
                        int precision, double* x_out, double* h_out, int32_t* status_out,
                        lsm_solve_stats* stats, cudaStream_t st, const NodeSpec* spec = nullptr);

int solve_charts_batch(Ctx* ctx, Batch* b, int n_gl, double tol, int max_iter, int precision, int use_graph,
                       double* x_out, double* h_out, int32_t* status_out, lsm_solve_stats* stats,
                       cudaStream_t st);
int batch_build(Ctx* ctx, Batch* b, lsm_mesh* const* meshes, int n, cudaStream_t st);
void batch_release(Batch* b);
// Work items of at most bs listed nodes of one mesh each; cap: the items
// buffer's length (no item is written past it)
int build_items(Ctx* ctx, const int32_t* list, const int* n_list, int n_max, const int32_t* node_mesh,
                const int2* mesh_tiles, int nmesh, int bs, uint32_t* cnt, uint32_t* nblk, int4* items, int* n_items,
                int cap, cudaStream_t st);

// host helpers (api.cu)
void simplex_rule_host(int n, int subdiv, double* uvw);  // [cnt][3]
// synchronise st, read and clear the calling thread's device error word:
// LSM_E_TIMEOUT when a bounded wait ran out
int check_flag(Ctx* ctx, cudaStream_t st);

}  // namespace lsm

struct lsm_ctx {
    lsm::Ctx c;
};
struct lsm_mesh {
    lsm::Mesh m;
};
struct lsm_batch {
    lsm::Batch b;
};
