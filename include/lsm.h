/*
 * lsm.h -- C ABI of the GB300 level-set mesher library (liblsm.so).
 *
 * The library evaluates the Gaussian-smoothed indicator function Phi of a
 * closed triangulated solid, and its gradient, at batches of target points,
 * and solves for chart nodes on the level set Phi = 1/2 by Newton's method.
 * It follows Vico, Greengard, O'Neil, Rachh, "A fast boundary integral method
 * for high-order multiscale mesh generation" (arXiv 1909.13356):
 *   Phi(x) = sum_j sum_k w_k |N_j| psi_sigma(x, T^j(u_k, v_k))   (Sec. 4.3,
 *   eq. discrete_int, with psi from eq. kerpsi), i.e. a sum over source nodes
 *   y with weighted normals nw of (nw . (y-x)) g(u) / (4 pi |y-x|^3),
 *   g(u) = erf(u) - (2u/sqrt pi) e^{-u^2}, u = |y-x| / (sqrt2 sigma).
 * sigma belongs to the source triangle (one value per skeleton triangle).
 *
 * Conventions for every entry point:
 *   - Return value: LSM_OK (0) or a negative lsm_status; no exceptions cross
 *     the ABI.  lsm_last_error(ctx) returns the message of the calling
 *     thread's last failed call on that context.
 *   - Every wait of a pair kernel on its staged source tile is bounded.  A
 *     wait that runs out sets the calling thread's device error word of the
 *     context and the targets of the thread blocks that gave up get NaN
 *     results.  Synchronous calls return LSM_E_TIMEOUT for it; calls left
 *     asynchronous (device pointers) report it at lsm_check_error or at the
 *     thread's next synchronous call.
 *   - Handles are opaque.  Device state belongs to the library until the
 *     matching *_free / lsm_destroy.
 *   - Array arguments may be host or device pointers (detected with
 *     cudaPointerGetAttributes).  With device pointers the call is
 *     asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) unless stated otherwise; with host pointers the call copies in
 *     and out and returns after the stream has finished.  Mixing host and
 *     device pointers in one call is allowed.
 *   - Layouts are row-major: points are double[n][3] (x, y, z), triangles
 *     int32[m][3] (0-based vertex indices, counter-clockwise seen from
 *     outside, Sec. 3).
 *   - Calls on the same mesh must be serialised by the caller (one stream at
 *     a time); different meshes may run concurrently on different streams.
 */
#ifndef LSM_H
#define LSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsm_ctx lsm_ctx;
typedef struct lsm_mesh lsm_mesh;
typedef struct lsm_batch lsm_batch;
typedef struct lsm_server lsm_server;

typedef enum {
    LSM_OK = 0,
    LSM_E_INVALID_ARG = -1,
    LSM_E_OOM = -2,
    LSM_E_CUDA = -3,
    LSM_E_MESH = -4,          /* not watertight / not conforming / orientation */
    LSM_E_NOT_CONVERGED = -5, /* reserved: per-node failures go to status arrays */
    LSM_E_TIMEOUT = -6,
    LSM_E_CANCELLED = -7,     /* lsm_server_cancel took the request off the queue */
    LSM_PENDING = 1           /* lsm_server_poll: the request has not finished */
} lsm_status;

typedef enum {
    LSM_FP64 = 0,   /* every kernel in FP64 */
    LSM_MIXED = 1,  /* FP32 pair kernels, compensated per-tile accumulation,
                       FP64 results; Newton finishes with LSM_FF steps when
                       the tolerance asks for more than FP32 gives */
    LSM_FF = 2      /* Phi to FP64 accuracy on the FP32 pipes: every pair in
                       float-float arithmetic (about 44 significant bits),
                       the near pairs' radial factor from a float-float
                       table; grad Phi to mixed accuracy */
} lsm_precision;

/* Per-node status of the chart solve (low byte); bit 8 set when a Newton
 * step was clamped to 4 sigma. */
enum {
    LSM_NODE_CONVERGED = 0,
    LSM_NODE_MAXITER = 1,
    LSM_NODE_ZERODERIV = 2,   /* H . grad Phi == 0 */
    LSM_NODE_NONFINITE = 3,
    LSM_NODE_CLAMPED_BIT = 256
};

/* Source quadrature rule on each skeleton triangle (Sec. 4.3): the triangle
 * is split `subdiv` times into four midpoint children (Sec. 4.5, 0..5) and
 * each (sub)triangle carries the Duffy-collapsed n_gl x n_gl Gauss-Legendre
 * rule, collapsed at its first vertex.  Nodes per triangle:
 * n_gl^2 * 4^subdiv.  (The paper's Vioreanu-Rokhlin rules are not used.) */
typedef struct {
    int32_t n_gl;
    int32_t subdiv;
} lsm_quad;

/* Context options; pass NULL for the defaults shown. */
typedef struct {
    double cutoff_fp64;    /* near-field radius in sigma, FP64 path (8.0,
                              Sec. 4.4: the kernel is the Laplace double
                              layer beyond 8 sigma to 1e-13 relative) */
    double cutoff_mixed;   /* same for the mixed path (6.5: neglected
                              relative term 4e-9 < FP32 rounding) */
    double mixed_switch;   /* mixed Newton: a node moves to FP64 steps once
                              |Phi - 1/2| < mixed_switch (1e-4; the mixed step
                              then lands near 1e-8, and one accurate step
                              below 1e-12) */
    double mixed_accept;   /* mixed Newton: a tolerance >= mixed_accept
                              (1e-7, the mixed kernels' accuracy on Phi) is
                              met on mixed evaluations alone, with no FP64
                              steps */
    /* Far field of the mixed path on large meshes: a barycentric Lagrange
     * treecode.  Source tiles are grouped by Morton order into a binary tree;
     * a node whose box lies beyond the mixed cutoff from a target block acts
     * on the block through a tensor grid of Chebyshev proxy points carrying
     * its interpolated dipole weights.  The grid lies along the principal
     * axes of the node's sources: degree p points on the widest axis, fewer
     * on narrower ones; p is the largest of tree_degree, tree_degree - 2, ...
     * whose grid has at most 2/3 as many points as the node has sources.
     * Opening rule: every target at distance >= r + q_p h_max from the box's
     * centre (r its radius, h_max its largest half-width), with q_p chosen so
     * that the interpolation error bound equals that of the classic rule
     * |x - c| >= r / tree_theta on a cube at tree_degree (tree_grid 1).
     * tree_grid 2: axis-aligned boxes, (tree_degree + 1)^3 points, the
     * classic rule. */
    int32_t tree_degree;      /* Chebyshev degree p per axis (8; 1..12) */
    float tree_theta;         /* opening parameter (0.45; (0, 1)) */
    int32_t tree_min_sources; /* meshes with at least this many source nodes
                                 use it (262,144); -1: never */
    /* The same for the float-float path (Phi to FP64 accuracy): proxies
     * with float-float positions and weights computed in FP64. */
    int32_t tree_ff_degree;      /* 14; 1..16 */
    float tree_ff_theta;         /* 0.45 */
    int32_t tree_ff_min_sources; /* 262,144; -1: never */
    int32_t tree_grid;           /* proxy grids of both treecodes: 0 or 1
                                    oriented per-axis grids and a degree ladder
                                    (default), 2 (degree + 1)^3 axis-aligned
                                    grids of one degree */
    /* Target clusters of the float-float treecode: runs of this many
     * Morton-sorted targets (a multiple of 128) get an oriented box with a
     * tensor Chebyshev grid (degree tree_ff_degree on the widest axis); a
     * node far enough from a cluster (the opening rule from the targets'
     * side, with the same error bound) acts on the grid's points, and the
     * targets interpolate its field from them.  0 selects 4096; -1: off. */
    int32_t tree_ff_cluster;
    /* The same for the mixed path's treecode (degree tree_degree grids on
     * clusters of this many targets, a multiple of 256).  0 selects 4096;
     * -1: off.  Measured: the bumped icosphere's 2e7-target evaluation takes
     * 3.9 s instead of 6.5 s, the graded torus's 1e6 targets 160 ms instead
     * of 170 ms, at the same error against FP64. */
    int32_t tree_cluster;
    /* Targets per CTA of the float-float kernel (64 or 128; 0 selects 64):
     * the near/far split and the treecode's lists are per CTA, so a smaller
     * target box means fewer pairs per target, at the price of more CTAs
     * streaming each source tile.  Every mode takes it: per-triangle sigma,
     * the target-dependent sigma(x) and batches. */
    int32_t ff_block;
    /* Targets per CTA of the mixed kernel (64, 128 or 256; 0: the mesh's
     * or the batch's autotuned choice, else 64).  A nonzero value
     * overrides the autotuner's, in sigma(x) mode too. */
    int32_t mixed_block;
    /* The mixed Newton sweeps of a chart solve only carry each node to
     * |Phi - 1/2| < mixed_switch; the float-float steps after them decide
     * the result.  On meshes with the mixed treecode they take a coarser
     * treecode of their own, with Chebyshev degree newton_tree_degree and
     * opening parameter newton_tree_theta (0 selects 5 and 0.5: errors near
     * 1e-6, far below the switch; the graded torus's order-8 solve at 10^6
     * nodes then takes 1.53 s instead of 1.67 s, its nodes as accurate).
     * The mesh's own mixed treecode is used when it is no finer than that;
     * -1: always.  Evaluations (lsm_eval_phi_grad) never use it. */
    int32_t newton_tree_degree;   /* 0: 5; 1..12; -1: off */
    float newton_tree_theta;      /* 0: 0.5; (0, 1) */
    /* The same sweeps' near-field radius in sigma, single meshes and
     * batches (0 selects 5.0, whose neglected relative term, about 1.5e-5
     * at the radius and falling as a Gaussian beyond, leaves errors near
     * 1e-7; the smaller of it and the mesh's or batch's mixed radius is
     * used; 512 ellipsoids solve 3 % faster, the graded torus 1.4 %). */
    float newton_cutoff;
} lsm_options;

/* Statistics of one chart solve. */
typedef struct {
    int32_t iterations;       /* Newton sweeps (evaluations of the active set) */
    int32_t n_nodes;
    int32_t n_converged;
    int32_t n_failed;         /* status != CONVERGED */
    double eps_newton;        /* max |h^(k) - h^(k-1)| over nodes' last steps
                                 (the paper's epsilon_N, Sec. 5) */
    double max_residual;      /* max |Phi - 1/2| at the converged nodes' last
                                 evaluation */
    int64_t evals_fp32;       /* target evaluations done by the mixed kernels */
    int64_t evals_fp64;       /* target evaluations done by FP64-accurate kernels
                                 (LSM_FP64, or the float-float steps of LSM_MIXED) */
    int32_t active_per_iter[32];
    int64_t evals_near_only;  /* of evals_fp64: float-float verification sweeps that
                                 re-evaluate only the near tiles and reuse the far
                                 part recorded by the sweep before */
} lsm_solve_stats;

/* Counts describing an uploaded mesh. */
typedef struct {
    int64_t n_vertices;
    int64_t n_triangles;
    int64_t n_sources;        /* n_triangles * nodes per triangle */
    int64_t n_tiles;          /* source tiles of the tiled kernels: runs of at most 128
                                 Morton-ordered nodes, cut where the curve jumps */
    int64_t device_bytes;     /* device memory held by the mesh */
    double sigma_min, sigma_max;
} lsm_mesh_info;

/* Create a context on CUDA device `device`.  Allocates no large memory.
 * Errors: LSM_E_INVALID_ARG (bad device or options), LSM_E_CUDA. */
int lsm_create(lsm_ctx** out, int device, const lsm_options* opt);
/* Destroy a context.  Servers, batches and meshes made from it that are
 * still alive are destroyed first (their handles become invalid), so that
 * none is ever used after its context. */
int lsm_destroy(lsm_ctx* ctx);
/* Message of the calling thread's last failed call on ctx ("" if none;
 * never NULL).  The string belongs to the calling thread and stays valid
 * until its next lsm_last_error call. */
const char* lsm_last_error(const lsm_ctx* ctx);
/* Number of kernel launches the library issued on this context so far. */
int64_t lsm_launch_count(const lsm_ctx* ctx);
/* Synchronise `stream`, then read and clear the calling thread's device
 * error word of ctx: LSM_E_TIMEOUT if a pair kernel launched by this thread
 * since the last check gave up on a bounded wait (its targets hold NaN),
 * else LSM_OK.  Errors: LSM_E_INVALID_ARG, LSM_E_CUDA. */
int lsm_check_error(lsm_ctx* ctx, void* stream);
/* Test hook, off by default: with enable != 0 every pair kernel launched on
 * ctx arms its first stage's barrier without issuing the copy and waits
 * with a short limit, so that the wait runs out with nothing in flight and
 * the call reports LSM_E_TIMEOUT.  Used to test the failure path; never
 * needed otherwise. */
int lsm_test_inject_wait_timeout(lsm_ctx* ctx, int enable);

/* Work counters of a context, for roofline accounting. */
typedef struct {
    int64_t launches;              /* every kernel launch (as lsm_launch_count) */
    int64_t pairs_near;            /* (target, source) pairs evaluated with the
                                      full smoothed kernel (near tiles) */
    int64_t pairs_far;             /* pairs evaluated with the Laplace double
                                      layer (far tiles) */
    int64_t pair_kernel_launches;  /* pair-kernel launches timed while
                                      profiling was on */
    double pair_kernel_ms;         /* their summed device time (CUDA events
                                      recorded on the launching stream) */
    /* the same per pair kernel: [0] mixed, [1] float-float, [2] FP64,
       [3] the Hessian kernel (lsm_eval_hessian) */
    int64_t kind_pairs_near[4];
    int64_t kind_pairs_far[4];
    int64_t kind_launches[4];
    double kind_ms[4];
} lsm_ctx_stats;

/* Measured throughput of the arithmetic the pair kernels run on (their
 * roofline denominators; the kernels are ALU-bound, not HBM- or tensor-
 * bound): one probe kernel per instruction kind, eight independent
 * dependency chains per thread at full occupancy on every SM, timed with
 * CUDA events on `stream`, best of three launches after a warm-up.  Takes
 * well under a second.  Synchronises `stream`.
 * Errors: LSM_E_INVALID_ARG, LSM_E_CUDA. */
typedef struct {
    double ffma_tflops;    /* FP32 fma.rn.f32, 2 flops each */
    double ffma2_tflops;   /* packed fma.rn.f32x2, 4 flops each */
    double dfma_tflops;    /* FP64 fma.rn.f64, 2 flops each */
    double rsqrt_gops;     /* rsqrt.approx.f32 per second (special-function unit) */
    double ex2_gops;       /* ex2.approx.ftz.f32 per second (special-function unit) */
    double ms[5];          /* the probes' best launch times, in the order above */
} lsm_peaks;
int lsm_measure_peaks(lsm_ctx* ctx, lsm_peaks* out, void* stream);

/* Turn per-launch timing of the pair kernels on or off (off by default). */
int lsm_set_profiling(lsm_ctx* ctx, int enable);
/* Read (and with reset != 0, clear) the counters.  Synchronises the device. */
int lsm_read_stats(lsm_ctx* ctx, lsm_ctx_stats* out, int reset);

/*
 * Upload a skeleton triangulation and build its resident device state
 * (Sec. 3 and 4.3): per-triangle frames T_u, T_v, N = T_u x T_v
 * (eq. tparam), sigma_j, vertex pseudonormals H(P) = sum(theta N_hat) /
 * sum(theta) (eq. mkvertexpn, not renormalised), the source nodes
 * y = T^j(u_k, v_k) with nw = w_k N_j, sorted along a Morton curve into
 * tiles, and their FP32 tile-local copies.
 *   verts  double[nv][3]; tris int32[nt][3]; sigma double[nt] or NULL for
 *          sigma_j = 0.5 sqrt(2 area_j).  Copied; the caller keeps them.
 *   rule   source rule (NULL = {4, 0}).
 * Host-side checks: every index in range; the mesh is closed and
 * consistently oriented (each directed edge once, its reverse once);
 * device check: signed volume > 0 and every sigma > 0.  Any failure
 * returns LSM_E_MESH.  Synchronises `stream` before returning.
 */
int lsm_mesh_upload(lsm_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris,
                    int64_t nt, const double* sigma, const lsm_quad* rule, void* stream,
                    lsm_mesh** out);
/* Upload a mesh whose smoothing width depends on the target (Sec. 2.3,
 * eq. sigma2): sigma(x) = sum_j sigma_j e_j / sum_j e_j with
 * e_j = exp(-|x - c_j|^2 / (2 sigma0^2)), c_j the centroid of triangle j and
 * sigma_j = D_j / lambda, D_j the diameter of the smallest ball enclosing it.
 * Every evaluation then uses the target's sigma(x) for all of its pairs, and
 * grad Phi gains (dPhi/dsigma) grad sigma (eq. gradPhi, third term, with the
 * sign that differentiating eq. kerpsi in sigma gives).
 *   lambda   0 selects 2.5 (the paper's choice)
 *   sigma0   0 selects max_j D_j / sqrt(2 ln 2): a centroid one diameter away
 *            weighs 1/2, the influence the paper describes for its choice
 * Everything else as lsm_mesh_upload (sigma_j doubles as the per-triangle
 * sigma of the Newton step clamp).  Batches and lsm_eval_phi_grad_noalloc
 * reject such meshes.  Errors: as lsm_mesh_upload. */
int lsm_mesh_upload_sigmax(lsm_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                           double lambda, double sigma0, const lsm_quad* rule, void* stream, lsm_mesh** out);
/* Upload a skeleton of quadratic (6-node curvilinear) patches (Sec. 5,
 * quadratic skeletons).  Patch j is the second-order Lagrange interpolant
 * T^j(u,v) on the standard simplex through its corners P1, P2, P3
 * (counter-clockwise seen from outside) and one node on each edge: P4 on
 * P1-P2, P5 on P2-P3, P6 on P3-P1.  Everything else is built as for flat
 * triangles with the patch's own tangents T_u, T_v and normal
 * N(u,v) = T_u x T_v: source nodes y = T(u_k, v_k) with nw = w_k N(u_k, v_k);
 * sigma_j = 0.5 sqrt(2 area_j) with the curved area (or the given sigma);
 * vertex pseudonormals (eq. mkvertexpn) from the corners' unit normals and
 * the angles between their two edges' tangents; H^j linear in (u, v) between
 * the corner pseudonormals (eq. mkpseudovec); charts x = T^j + h H^j.
 *   verts  double[nv][3]: corners and edge nodes
 *   tris6  int32[nt][6] (P1, P2, P3, P4, P5, P6); the two patches on an edge
 *          share its edge node
 * Charts, frames and the Gauss flux (lsm_solve_charts*, lsm_chart_frames*,
 * lsm_gauss_flux*), Phi, grad Phi and the Hessian work as for flat meshes;
 * batches and lsm_chart_curvature reject such meshes.  Errors: as
 * lsm_mesh_upload (LSM_E_MESH also for inconsistent edge nodes). */
int lsm_mesh_upload_quadratic(lsm_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris6, int64_t nt,
                              const double* sigma, const lsm_quad* rule, void* stream, lsm_mesh** out);
/* sigma(x) [n] and grad sigma(x) [n][3] (may be NULL) at n targets of a mesh
 * uploaded with lsm_mesh_upload_sigmax (eq. sigma2); pointers as in
 * lsm_eval_phi_grad.  Errors: LSM_E_INVALID_ARG (also for other meshes),
 * LSM_E_OOM, LSM_E_CUDA. */
int lsm_eval_sigma(lsm_mesh* mesh, const double* x, int64_t n, double* sigma, double* gsigma, void* stream);
/* sigma0 of a mesh uploaded with lsm_mesh_upload_sigmax (0 for others). */
int lsm_mesh_get_sigma0(const lsm_mesh* mesh, double* sigma0);
int lsm_mesh_free(lsm_mesh* mesh);
int lsm_mesh_get_info(const lsm_mesh* mesh, lsm_mesh_info* out);

/*
 * Phi and grad Phi at n targets (Sec. 4.4, eq. kerdecomp): source tiles
 * farther than cutoff * sigma_max(tile) from a target block use the Laplace
 * double layer (eq. kerapprox); all other pairs use the full kernel
 * (eq. kerpsi and the gradient of eq. gradPhi with the sign of its second
 * term corrected), with a power series for small u (eq. kerpsi_asymp).
 *   x     double[n][3] targets
 *   phi   double[n] out
 *   grad  double[n][3] out, or NULL
 *   precision  LSM_FP64, LSM_MIXED or LSM_FF
 * n == 0 is a no-op.  Errors: LSM_E_INVALID_ARG, LSM_E_CUDA.
 */
int lsm_eval_phi_grad(lsm_mesh* mesh, const double* x, int64_t n, double* phi, double* grad,
                      int precision, void* stream);

/*
 * Phi and grad Phi at n targets without allocating any memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc while they run -- for example a latency-critical loop in which
 * an allocation or free could synchronise the device, or a process whose
 * device memory is already reserved in full by another allocator (a
 * framework's caching pool), so that a further cudaMalloc would fail.
 *
 * It computes what lsm_eval_phi_grad computes at precision LSM_FP64 or
 * LSM_MIXED, with the same kernels and tolerances (LSM_FF, which needs the
 * treecode's scratch, returns LSM_E_INVALID_ARG), but it does not sort the
 * targets and takes its scratch from one fixed device array of 8 MiB inside
 * the library, which every GPU that loads the library holds until the
 * process exits.  Targets are evaluated in the caller's order: a thread
 * block of consecutive targets decides near and far source tiles from the
 * box around its targets, so targets scattered over the surface put most
 * pairs on the slower near-field path; callers that can should pass targets
 * in a spatially coherent order.
 *   x     double[n][3], device pointer
 *   phi   double[n], device pointer
 *   grad  double[n][3], device pointer, or NULL
 *   n     0 <= n <= 16384; larger n returns LSM_E_INVALID_ARG with a
 *         message naming the limit.  Host pointers also return
 *         LSM_E_INVALID_ARG.
 * Asynchronous on `stream`.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  A bounded wait that runs out leaves NaN in the
 * targets concerned and sets the error word that lsm_check_error reads.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Every call on a device shares the
 * one array and leaves its contents behind for the next call; the kernels
 * overwrite every element they read, so nothing needs clearing, but calls
 * whose executions overlap on the GPU (different streams, or several host
 * threads) race on the array and must be serialised by the caller.
 */
int lsm_eval_phi_grad_noalloc(lsm_mesh* mesh, const double* x, int64_t n, double* phi, double* grad,
                              int precision, void* stream);

/* Local coordinates of the solved charts (Sec. 3.3).  Chart j is
 * x(u,v) = T^j(u,v) + h(u,v) H^j(u,v) (eq. chart); with grad Phi normal to the
 * level set,
 *   h_u = -((T_u + h H_u) . grad Phi) / (H . grad Phi)     (eq. U_vector_2)
 *   x_u = T_u + h H_u + h_u H                                (eq. u_vector)
 * and the same in v (eq. v_vector, v_vector_2); the area element is
 * da = |x_u x x_v| du dv (eq. da).
 *   order     the chart order given to lsm_solve_charts (rule n = order/2+2)
 *   h         [N] solved h, nodes in lsm_solve_charts' order (N = M n^2)
 *   grad      [N][3] grad Phi at the solved nodes (lsm_eval_phi_grad)
 *   xu, xv    [N][3] out; jac [N] out: |x_u x x_v|
 * Host or device pointers (outputs device-resident when device pointers are
 * given).  A node with H . grad Phi = 0 gets non-finite values.
 * Errors: LSM_E_INVALID_ARG, LSM_E_OOM, LSM_E_CUDA. */
int lsm_chart_frames(lsm_mesh* mesh, int order, const double* h, const double* grad, double* xu, double* xv,
                     double* jac, void* stream);
/* Gauss flux error of the charts about an interior point x0 (Sec. 5):
 *   eps0 = 1 + sum_nodes w_i jac N . (x0 - x)/(4 pi |x0 - x|^3),
 * with N = -grad Phi/|grad Phi| the outward normal and the chart rule's
 * weights w_i.  Zero for a closed surface around x0, one when x0 is outside.
 *   x [N][3], grad [N][3], jac [N] as above (host or device); x0[3] host;
 *   eps0 host out.  The sum is reduced in a fixed order (deterministic).
 *   Synchronises `stream`.
 * Errors: LSM_E_INVALID_ARG, LSM_E_OOM, LSM_E_CUDA. */
int lsm_gauss_flux(lsm_mesh* mesh, int order, const double* x, const double* grad, const double* jac,
                   const double* x0, double* eps0, void* stream);

/* The Hessian of Phi at n targets (Sec. 3.3: the charts' second derivatives
 * need it, eq. uu_vector_aux1).  Per pair, with r = y - x, q = nw . r and
 * the radial factors f, F = f'/rho, G = F'/rho of eq. kerpsi,
 *   d2/dx_i dx_j [q f] = F (nw_i r_j + nw_j r_i + q delta_ij) + q G r_i r_j.
 * Near tiles (within the FP64 cutoff) are summed in FP64, far tiles in FP32
 * with compensated sums; direct far field.
 *   x     [n][3] host or device;  hess [n][6] out: xx, xy, xz, yy, yz, zz.
 * Meshes uploaded with lsm_mesh_upload_sigmax are rejected.
 * Errors: LSM_E_INVALID_ARG, LSM_E_OOM, LSM_E_CUDA. */
int lsm_eval_hessian(lsm_mesh* mesh, const double* x, int64_t n, double* hess, void* stream);
/* Second derivatives of the solved charts and the curvatures of the level
 * set at their nodes (Sec. 3.3).  On the flat skeleton triangles, with H
 * linear, eq. uu_vector and its uv, vv analogues read
 *   x_uu = 2 h_u H_u + h_uu H,  x_uv = h_u H_v + h_v H_u + h_uv H,  x_vv = 2 h_v H_v + h_vv H,
 * with h_uu = -(x_u^T Hess x_u + 2 h_u H_u . grad Phi)/(H . grad Phi) and its
 * analogues (eq. uu_vector_aux2).  With the outward normal -grad Phi/|grad Phi|
 * and the two fundamental forms: kgauss = Gaussian curvature, kmean = the
 * sum of the principal curvatures (2/R on a sphere of radius R).
 *   h [N], grad [N][3], hess [N][6] at the solved nodes (lsm_solve_charts'
 *   order); xuu, xuv, xvv [N][3], kmean, kgauss [N] out.  Host or device.
 * Errors: LSM_E_INVALID_ARG, LSM_E_OOM, LSM_E_CUDA. */
int lsm_chart_curvature(lsm_mesh* mesh, int order, const double* h, const double* grad, const double* hess,
                        double* xuu, double* xuv, double* xvv, double* kmean, double* kgauss, void* stream);

/* Refined charts (Sec. 3.4).  A skeleton triangle split 1 -> 4 at its edge
 * midpoints, level times, keeps its parent's chart map: its nodes are the
 * order's n x n Duffy rule composited over the 4^level children, given as
 * points (u, v) of the parent's reference triangle with weights (1/2 per
 * triangle in all).  H stays linear in the parent's (u, v), so the
 * pseudonormal field, and with it the charts, stay continuous between
 * refined and unrefined neighbours.
 *   order     chart order (n = order/2 + 2);  m, level [m] in 0..4 (host)
 *   tri [N], uvw [N][3] out (host): triangle and (u, v, weight) per node, in
 *             triangle order; pass NULL for both to get only *n_out = N =
 *             sum_j n^2 4^level_j.
 * Errors: LSM_E_INVALID_ARG. */
int lsm_refined_nodes(int order, int64_t m, const int32_t* level, int32_t* tri, double* uvw, int64_t* n_out);
/* lsm_solve_charts at explicit nodes: node s in triangle tri[s] at parent
 * coordinates (uvw[3s], uvw[3s+1]) (for instance from lsm_refined_nodes).
 * Outputs and behaviour as lsm_solve_charts, in the given node order.
 * Errors: LSM_E_INVALID_ARG (also a triangle index out of range), LSM_E_OOM,
 * LSM_E_CUDA. */
int lsm_solve_charts_nodes(lsm_mesh* mesh, int64_t n, const int32_t* tri, const double* uvw, double tol,
                           int max_iter, int precision, double* x_out, double* h_out, int32_t* status_out,
                           lsm_solve_stats* stats, void* stream);
/* lsm_chart_frames and lsm_gauss_flux at explicit nodes; the flux weights
 * are uvw[3s+2]. */
int lsm_chart_frames_nodes(lsm_mesh* mesh, int64_t n, const int32_t* tri, const double* uvw, const double* h,
                           const double* grad, double* xu, double* xv, double* jac, void* stream);
int lsm_gauss_flux_nodes(lsm_mesh* mesh, int64_t n, const int32_t* tri, const double* uvw, const double* x,
                         const double* grad, const double* jac, const double* x0, double* eps0, void* stream);

/* Per-triangle Gauss flux (Sec. 5, the quantity of lsm_gauss_flux split by
 * skeleton triangle): out[j] = sum over the nodes s of triangle j of
 * uvw[3s+2] jac[s] N . (x0 - x[s]) / (4 pi |x0 - x[s]|^3), N = -grad Phi/|grad Phi|.
 * Nodes must be grouped by triangle in increasing triangle order (as
 * lsm_refined_nodes lists them); a triangle with no node gets 0.
 *   n, tri [n], uvw [n][3], x [n][3], grad [n][3], jac [n]: host or device;
 *   x0[3] host; out [m] host or device (m = the mesh's triangles).
 * Synchronises `stream`.  Errors: LSM_E_INVALID_ARG, LSM_E_CUDA. */
int lsm_flux_per_triangle(lsm_mesh* mesh, int64_t n, const int32_t* tri, const double* uvw, const double* x,
                          const double* grad, const double* jac, const double* x0, double* out, void* stream);
/* A posteriori refinement of the charts (Sec. 3.4: refinement where standard
 * a posteriori estimates from adaptive integration ask for it).  For each
 * triangle at level L (1 -> 4 midpoint splits, the children keeping the
 * parent's chart map, lsm_refined_nodes) the Gauss flux integral about the
 * interior point x0 over its charts is compared with the same integral one
 * level finer; where they differ by more than flux_tol the triangle is
 * refined and tested again one level further, up to max_level (0..4).  Each
 * test solves the charts (mixed precision finished in float-float, to
 * newton_tol) at the nodes concerned.
 *   order      chart order (rule n = order/2 + 2)
 *   level_out  [m] host: the level of each triangle
 *   rounds_out host, may be NULL: refinement rounds run
 * Synchronises `stream`.  Errors: LSM_E_INVALID_ARG, LSM_E_OOM, LSM_E_CUDA,
 * LSM_E_NOT_CONVERGED (chart nodes that did not converge; level_out is still
 * filled), LSM_E_TIMEOUT. */
int lsm_refine_adaptive(lsm_mesh* mesh, int order, double newton_tol, double flux_tol, int max_level,
                        const double* x0, int32_t* level_out, int* rounds_out, void* stream);

/* Autotuner of the mixed path's far field (the paper has no counterpart:
 * its FMM is run at a fixed precision, Sec. 4.4).  Chooses, for this mesh,
 * between the direct tiled far field and the treecode, and the treecode's
 * Chebyshev degree and opening parameter: the fastest candidate whose
 * largest |Phi error| against the float-float path stays within err_budget.
 *   x        [n][3] targets typical of the workload, host or device; up to
 *            8 windows of 4,096 consecutive targets in Morton order (so with
 *            the workload's density) are the sample
 *   err_budget  bound on max |Phi_mixed - Phi_ff| over the sample (e.g.
 *            5e-8, half the mixed path's 1e-7)
 *   out      the choice and what was measured; may be NULL
 * The choice is stored with the mesh and used by its later mixed
 * evaluations and chart solves (it overrides the context's tree options).
 * With that far field it then chooses the mixed kernel's near-field radius
 * (6.4, 6.5 or 7 sigma: those where the smoothed kernel differs from the
 * Laplace double layer by at most 1e-8 relative, Sec. 4.4) and its target
 * tile (64, 128 or 256 targets per thread block of 128 threads: two threads
 * per target, one, or a thread for two targets; 256 only in sigma(x) mode),
 * again the fastest within the budget.
 * Cost: one float-float evaluation of the sample, and a tree build plus two
 * mixed evaluations of it per candidate.  Synchronises `stream`.
 * Errors: LSM_E_INVALID_ARG (n < 1, bad budget), LSM_E_OOM, LSM_E_CUDA. */
typedef struct {
    int32_t use_tree;         /* 0: the direct far field was chosen */
    int32_t tree_degree;      /* chosen degree and opening parameter */
    float tree_theta;
    int32_t candidates;       /* candidates measured */
    int64_t sample_targets;
    double err_phi;           /* max |dPhi| of the choice on the sample */
    double ms_sample;         /* its mixed-evaluation time on the sample */
    double ms_direct;         /* the direct far field's time on the sample */
    double err_direct;        /* and its error */
    double cutoff;            /* chosen near-field radius of the mixed kernel, in sigma */
    int32_t targets_per_block;/* chosen target tile of the mixed kernel (64, 128 or 256) */
    int32_t reserved;
} lsm_tune_result;
int lsm_autotune(lsm_mesh* mesh, const double* x, int64_t n, double err_budget, lsm_tune_result* out,
                 void* stream);

/*
 * Chart nodes on Phi = 1/2 (Sec. 3.2): for each triangle j and each node
 * (u_i, v_i) of the Duffy n x n chart rule with n = order/2 + 2, Newton's
 * method on h (eq. newtoneq) from h = 0:
 *   x = T^j(u_i, v_i) + h H^j(u_i, v_i)   (H^j from eq. mkpseudovec)
 *   h <- h - (Phi(x) - 1/2) / (H^j . grad Phi(x)),
 * each step clamped to 4 sigma_j, until |Phi(x) - 1/2| < tol or max_iter
 * evaluations.  Converged nodes leave the active set (Sec. 5).
 *   x_out   double[nt * n^2][3] (triangle-major, then rule order) or NULL
 *   h_out   double[nt * n^2] or NULL
 *   status  int32[nt * n^2] or NULL  (LSM_NODE_*)
 *   stats   may be NULL
 * Synchronises `stream` (the active-set size is read each sweep).
 */
int lsm_solve_charts(lsm_mesh* mesh, int order, double tol, int max_iter, int precision,
                     double* x_out, double* h_out, int32_t* status, lsm_solve_stats* stats,
                     void* stream);

/*
 * Batches: many meshes solved together (the paper treats one mesh at a
 * time; batching many independent charts problems is this library's
 * addition).  lsm_batch_create copies the resident state of n uploaded
 * meshes of one context into concatenated arrays (each mesh's source nodes
 * start on a tile boundary, so no work item mixes meshes); the meshes stay
 * valid and independent.  Synchronises `stream`.
 */
int lsm_batch_create(lsm_ctx* ctx, lsm_mesh* const* meshes, int n, void* stream, lsm_batch** out);
int lsm_batch_free(lsm_batch* batch);

/*
 * lsm_solve_charts for every mesh of a batch at once: each Newton sweep is
 * one set of launches over all meshes' active nodes, with the work items
 * (blocks of one mesh's nodes and that mesh's tile range) built on the
 * device.  With use_graph != 0, two sweeps are captured once as a CUDA graph
 * on a private stream and replayed until no node is active or max_iter
 * sweeps have run.  Outputs are concatenated in mesh order, each mesh
 * triangle-major then rule order, as lsm_solve_charts would return them.
 * precision: LSM_FP64 or LSM_MIXED.  Synchronises `stream`.
 */
int lsm_batch_solve_charts(lsm_batch* batch, int order, double tol, int max_iter, int precision, int use_graph,
                           double* x_out, double* h_out, int32_t* status, lsm_solve_stats* stats, void* stream);

/*
 * Autotuner of a batch (this library's addition, as lsm_autotune): chooses
 * the mixed kernel's near-field radius (6.4, 6.5 or 7 sigma, as
 * lsm_autotune) and target tile (64, 128 or 256 targets per work item) for the
 * batch's later lsm_batch_solve_charts calls: the fastest within err_budget
 * of the float-float evaluation, measured on the chart nodes' starting
 * points of every stride-th mesh (about 64 meshes), in the work items the
 * batched solve uses.  Batches use the direct far field, so there is no
 * treecode to tune.  `out` (may be NULL) reports the choice: use_tree = 0,
 * cutoff, targets_per_block, err_phi and ms_sample of the choice, ms_direct
 * and err_direct of the default settings.  Synchronises `stream`.
 * Errors: LSM_E_INVALID_ARG, LSM_E_OOM, LSM_E_CUDA. */
int lsm_batch_autotune(lsm_batch* batch, int order, double err_budget, lsm_tune_result* out, void* stream);

/*
 * Serving: a continuous-batching request server over one context (the paper
 * has no serving layer; this is this library's addition).  Requests are
 * queued in arrival order; `slots` worker threads, each with its own CUDA
 * stream, take the head of the queue as soon as a slot is free and the
 * request's estimated device footprint (mesh state plus chart-solve state)
 * fits in the HBM budget next to the running requests (a request larger
 * than the whole budget runs alone).  Each admitted request is uploaded
 * (lsm_mesh_upload), solved (lsm_solve_charts) on its slot's stream, copied
 * back and freed; requests on different slots overlap on the GPU.
 *   hbm_budget_bytes <= 0: 80% of the device memory free at creation.
 * lsm_server_submit copies the request's arrays and returns at once.
 * lsm_server_poll returns LSM_PENDING until the request is done (or blocks
 * with wait != 0), then fills `out`; the result arrays stay owned by the
 * server until lsm_server_release.  Times are milliseconds on the server's
 * clock.  lsm_server_destroy finishes every queued request first.
 * Per-launch profiling (lsm_set_profiling) must be off while a server runs.
 */
typedef struct {
    const double* verts;     /* host double[nv][3] */
    int64_t nv;
    const int32_t* tris;     /* host int32[nt][3] */
    int64_t nt;
    const double* sigma;     /* host double[nt] or NULL (0.5 sqrt(2 area)) */
    lsm_quad rule;           /* source rule; n_gl == 0 selects {4, 0} */
    int32_t order;           /* chart order, as lsm_solve_charts */
    double tol;
    int32_t max_iter;        /* <= 0 selects 20 */
    int32_t precision;       /* LSM_FP64 or LSM_MIXED */
} lsm_request;

typedef struct {
    int32_t status;          /* LSM_OK or the error of the request */
    int64_t n_nodes;
    double t_submit_ms, t_start_ms, t_done_ms;
    int64_t device_bytes;    /* footprint charged against the budget */
    lsm_solve_stats stats;
    const double* x;         /* [n_nodes][3], server-owned */
    const double* h;         /* [n_nodes] */
    const int32_t* node_status;
    const char* error;       /* the failed request's own message ("" if ok), server-owned */
} lsm_result;

typedef struct {
    int64_t queued, running, max_running;
    int64_t budget_bytes, in_use_bytes, peak_in_use_bytes;
    double now_ms;
} lsm_server_info_t;

int lsm_server_create(lsm_ctx* ctx, int slots, int64_t hbm_budget_bytes, lsm_server** out);
int lsm_server_submit(lsm_server* server, const lsm_request* request, int64_t* ticket);
int lsm_server_poll(lsm_server* server, int64_t ticket, int wait, lsm_result* out);
/* Take a request that is still queued off the queue: its result is then
 * final with status LSM_E_CANCELLED.  Returns LSM_OK, or LSM_E_INVALID_ARG
 * for an unknown ticket or a request that has already started. */
int lsm_server_cancel(lsm_server* server, int64_t ticket);
int lsm_server_release(lsm_server* server, int64_t ticket);
int lsm_server_info(lsm_server* server, lsm_server_info_t* out);
int lsm_server_destroy(lsm_server* server);

#ifdef __cplusplus
}
#endif

#endif /* LSM_H */
