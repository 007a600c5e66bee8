// tree.cu -- far field of the mixed path on large meshes: a barycentric
// Lagrange treecode over the Morton-ordered source tiles.
//
// Beyond the cutoff the smoothed kernel is the Laplace double layer (eq.
// kerapprox, Sec. 4.4); the paper evaluates that part with an FMM.  Here the
// tiles of consecutive Morton-sorted sources are the leaves of a binary tree
// whose node (l, i) holds tiles [i 2^l, (i+1) 2^l) and their tight box.  For
// a node C with box centre c and half-widths h, the double-layer kernel y ->
// K(x, y) interpolated on the tensor Chebyshev grid s_k = c + h * cos(k pi/p)
// (per axis) gives
//     sum_j nw_j . K(x, y_j)  ~  sum_k Q_k . K(x, s_k),   Q_k = sum_j L_k(y_j) nw_j,
// with L_k the tensor-product Lagrange basis of the grid in barycentric form.
// The error falls like a power of (radius of C) / |x - c|, so a node acts
// through its proxies (s_k, Q_k) on a block of targets when
//     |c - block box| >= radius(C) / theta
// and the node's box is beyond the cutoff from the block (every pair is a
// pure double-layer pair).  Proxies are sources of the far-pair kernel like
// any other: each node's proxies fill proxy tiles laid out as source tiles,
// and a target block's interaction list (built per evaluation by a walk of
// the tree) mixes source tiles and proxy tiles.  A node gets proxies only
// when it holds at least twice as many sources as proxies.
//
// Oriented grids.  A node's grid lies in its own frame: the principal axes
// of its sources (mean, covariance, Jacobi eigenvectors) with the extents of
// the sources along them.  Surface patches are thin across the surface in
// that frame, whatever their tilt against the coordinate axes.
//
// Opening rule and points per axis.  As a function of one coordinate along
// axis a (half-width h_a), the kernel has its singularities at distance >= d
// from the node's box when every target is at distance >= d from it; its
// degree-p Chebyshev interpolant then errs like rho(d / h_a)^-p, rho(q) = q +
// sqrt(q^2 - 1) = exp(acosh q), the Bernstein ellipse through the nearest
// singularity (a real one in the worst case).  The widest axis sets the
// error, so a node of degree p acts on a block of targets when
//     |x - c| >= r + q_p h_max,   q_p = cosh(C / p),
// (c, r the centre and radius of the box) for every target x of the block:
// then d >= q_p h_max and the error is ~exp(-C) whatever the box's shape.
// C = p_top acosh(sqrt3 (1/theta - 1)) is the bound of the classic rule
// |x - c| >= r / theta on a cube, so (p_top, theta) keep their meaning.  A
// narrower axis gets the smallest degree whose bound is 1/32 of the widest
// axis's (the tensor interpolant's error sums the axes' errors, each
// amplified by the other axes' Lebesgue constants, about 2.7 each).
//
// Degree ladder.  A node acts through proxies only when it holds 1.5 times
// as many sources as proxies, which at the top degree excludes every small
// node.  So each node takes the largest degree of the ladder p, p - 2, ...
// that it can carry; with the same C, lower degrees act only from farther
// away (larger q_p).
// tree_grid 2 keeps the first design (axis-aligned boxes, (p+1)^3 points,
// one degree, sources >= 2 proxies, |x - c| >= r / theta) through the same
// code with identity frames.
//
// Steps: node boxes bottom-up (k_nodes_leaf, k_nodes_up); node frames
// (k_node_frames); grids and proxy assignment on the host; P2M, the weights
// Q_k summed from the sources in chunks (k_p2m, k_p2m64, k_p2m_reduce); per
// evaluation, target block boxes (k_block_boxes) and two walks (count, then
// write) of the tree per block (k_tree_walk).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr int kP2MThreads = 256;
constexpr int kP2MChunkTiles = 256;      // source tiles per P2M work item
constexpr int kMaxDeg32 = 12;             // FP32 proxies (mixed path): degree at most
constexpr int kMaxN = kMaxDeg32 + 1;      // grid points per axis at most
constexpr int kLStride = 16;              // floats per (axis, source) row of basis values
constexpr int kMaxN64 = kTreeMaxDegree + 1;
constexpr int kP2M64Src = 64;             // sources staged per pass of the FP64 P2M
constexpr int kWalkThreads = 128;
constexpr int kMaxLevels = 32;

inline int blocks_of(int64_t n, int t) { return (int)((n + t - 1) / t); }

__global__ void k_nodes_leaf(const float4* __restrict__ tlo, const float4* __restrict__ thi, int ntiles,
                             float4* __restrict__ nlo, float4* __restrict__ nhi, int4* __restrict__ info)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntiles) return;
    const float4 b = thi[i];
    nlo[i] = tlo[i];
    nhi[i] = make_float4(b.x, b.y, b.z, 0.0f);
    info[i] = make_int4(i, 1, -1, 0);
}

// Node i of a level: the union of children 2i and 2i+1 of the level below.
__global__ void k_nodes_up(const float4* __restrict__ clo, const float4* __restrict__ chi,
                           const int4* __restrict__ cinfo, int nchild, float4* __restrict__ nlo,
                           float4* __restrict__ nhi, int4* __restrict__ info, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = 2 * i, b = 2 * i + 1;
    float4 l = clo[a], h = chi[a];
    int4 f = cinfo[a];
    if (b < nchild) {
        const float4 l2 = clo[b], h2 = chi[b];
        l = make_float4(fminf(l.x, l2.x), fminf(l.y, l2.y), fminf(l.z, l2.z), fmaxf(l.w, l2.w));
        h = make_float4(fmaxf(h.x, h2.x), fmaxf(h.y, h2.y), fmaxf(h.z, h2.z), 0.0f);
        f.y += cinfo[b].y;
    }
    nlo[i] = l;
    nhi[i] = h;
    info[i] = make_int4(f.x, f.y, -1, 0);
}

// Oriented box of a node: centre, orthonormal axes (rows) and half-widths.
struct NodeFrame {
    double c[3];
    double e[3][3];
    double h[3];
};

// Bound exponent C of (degree, theta): the classic rule on a cube (host).
double tree_bound(int degree, double theta)
{
    const double q = std::max(1.05, std::sqrt(3.0) * (1.0 / theta - 1.0));
    return degree * std::acosh(q);
}

// Points per axis of a node's grid of degree p (host only), from its
// half-widths: one on an axis of zero extent; grid 2: p + 1 on every other
// axis; grid 1: p + 1 on the widest axis, and on the others the fewest
// whose bound, at d = q_p h_max, is 1/32 of the widest axis's.
int4 grid_counts(const double h[3], int p, double C, int grid)
{
    double hmax = 0.0;
    for (int a = 0; a < 3; a++) hmax = std::max(hmax, h[a]);
    const double d = std::cosh(C / p) * hmax;
    int n[3];
    for (int a = 0; a < 3; a++) {
        if (!(h[a] > 0.0)) {
            n[a] = 1;
        } else if (grid == 2 || h[a] == hmax) {
            n[a] = p + 1;
        } else {
            const int pa = (int)std::ceil((C + std::log(32.0)) / std::acosh(d / h[a]) - 1e-9);
            n[a] = std::min(p, std::max(1, pa)) + 1;
        }
    }
    return make_int4(n[0], n[1], n[2], 0);
}

// Sum of K doubles over a block of kFrameThreads threads, returned to every
// thread (fixed order: warp shuffles, then the warps in order).
constexpr int kFrameThreads = 256;
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sm)
{
#pragma unroll
    for (int k = 0; k < K; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < K; k++) sm[w * K + k] = v[k];
    __syncthreads();
    for (int k = 0; k < K; k++) {
        double t = 0.0;
        for (int j = 0; j < kFrameThreads / 32; j++) t += sm[j * K + k];
        v[k] = t;
    }
    __syncthreads();
}

// Eigenvectors of a symmetric 3x3 matrix by cyclic Jacobi rotations: the
// columns of v.  The rotations keep v orthonormal, so any stopping point
// gives a valid frame.
__device__ void jacobi3(double a[3][3], double v[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) v[i][j] = i == j ? 1.0 : 0.0;
    const double scale = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
    for (int sweep = 0; sweep < 16; sweep++) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        if (!(off > 1e-18 * scale)) break;
        for (int r = 0; r < 3; r++) {
            const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
            const double apq = a[p][q];
            if (apq == 0.0) continue;
            const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = fabs(th) > 1e150 ? 0.5 / th : (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            const int k = 3 - p - q;
            const double akp = a[k][p], akq = a[k][q];
            a[k][p] = a[p][k] = c * akp - sn * akq;
            a[k][q] = a[q][k] = sn * akp + c * akq;
            for (int i = 0; i < 3; i++) {
                const double vip = v[i][p], viq = v[i][q];
                v[i][p] = c * vip - sn * viq;
                v[i][q] = sn * vip + c * viq;
            }
        }
    }
}

// Frame of each node of levels >= 1 (one CTA per node, nodes node0 ...):
// mean and covariance of its sources in FP64, principal axes, and the
// extents of the sources along them.  Half-widths below 1e-9 of the box's
// radius are raised to it, so that the coordinates of the P2M basis stay in
// [-1, 1] up to rounding.
__global__ void __launch_bounds__(kFrameThreads) k_node_frames(const double4_32a* __restrict__ pos, int64_t ns,
                                                               const int4* __restrict__ info, int64_t node0,
                                                               NodeFrame* __restrict__ fr)
{
    __shared__ double sm[(kFrameThreads / 32) * 6];
    __shared__ double s_e[3][3];
    const int64_t node = node0 + blockIdx.x;
    const int4 f = info[node];
    const int64_t s0 = (int64_t)f.x * kTile, s1 = min(ns, (int64_t)(f.x + f.y) * kTile);
    const double cnt = (double)max((int64_t)1, s1 - s0);
    double m[3] = {0.0, 0.0, 0.0};
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kFrameThreads) {
        const double4_32a p = pos[i];
        m[0] += p.x;
        m[1] += p.y;
        m[2] += p.z;
    }
    block_sum<3>(m, sm);
    for (int k = 0; k < 3; k++) m[k] /= cnt;
    double cv[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kFrameThreads) {
        const double4_32a p = pos[i];
        const double d0 = p.x - m[0], d1 = p.y - m[1], d2 = p.z - m[2];
        cv[0] += d0 * d0;
        cv[1] += d0 * d1;
        cv[2] += d0 * d2;
        cv[3] += d1 * d1;
        cv[4] += d1 * d2;
        cv[5] += d2 * d2;
    }
    block_sum<6>(cv, sm);
    if (threadIdx.x == 0) {
        double a[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}}, v[3][3];
        jacobi3(a, v);
        for (int ax = 0; ax < 3; ax++)
            for (int c = 0; c < 3; c++) s_e[ax][c] = v[c][ax];
    }
    __syncthreads();
    double e[3][3];
    for (int ax = 0; ax < 3; ax++)
        for (int c = 0; c < 3; c++) e[ax][c] = s_e[ax][c];
    double ext[6] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY};   // max, then -min
    for (int64_t i = s0 + threadIdx.x; i < s1; i += kFrameThreads) {
        const double4_32a p = pos[i];
        const double d[3] = {p.x - m[0], p.y - m[1], p.z - m[2]};
        for (int ax = 0; ax < 3; ax++) {
            const double t = d[0] * e[ax][0] + d[1] * e[ax][1] + d[2] * e[ax][2];
            ext[ax] = fmax(ext[ax], t);
            ext[3 + ax] = fmax(ext[3 + ax], -t);
        }
    }
    for (int k = 0; k < 6; k++)
        for (int o = 16; o > 0; o >>= 1) ext[k] = fmax(ext[k], __shfl_xor_sync(0xffffffffu, ext[k], o));
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 6; k++) sm[w * 6 + k] = ext[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; k++)
            for (int j = 1; j < kFrameThreads / 32; j++) ext[k] = fmax(ext[k], sm[j * 6 + k]);
        NodeFrame F;
        double r2 = 0.0;
        for (int ax = 0; ax < 3; ax++) {
            const double hi = ext[ax], lo = -ext[3 + ax];
            F.h[ax] = 0.5 * (hi - lo);
            r2 += F.h[ax] * F.h[ax];
            const double mid = 0.5 * (hi + lo);
            for (int c = 0; c < 3; c++) F.e[ax][c] = e[ax][c];
            m[0] += mid * e[ax][0];
            m[1] += mid * e[ax][1];
            m[2] += mid * e[ax][2];
        }
        const double hmin = 1e-9 * sqrt(r2);
        for (int ax = 0; ax < 3; ax++) F.h[ax] = fmax(F.h[ax], hmin);
        for (int c = 0; c < 3; c++) F.c[c] = m[c];
        fr[node] = F;
    }
}

// Chebyshev points of the second kind on [-1, 1], in FP32.
__device__ __forceinline__ float cheb_point(int k, int degree)
{
    return (float)cospi((double)k / (double)degree);
}

struct P2MArgs {
    const double4_32a* pos;   // (x, y, z, a)
    const double4_32a* nw;    // (nw / 4 pi, 0)
    int64_t ns;               // source slots (tiles x kTile)
    const NodeFrame* fr;      // each node's oriented box
    const int4* ninfo;
    const int4* items;        // node, first tile, end tile, partial offset (in proxies) or -1
    const int4* ngrid;        // points per axis of each node's grid
    float4* p_pos;
    float4* p_nw;
    float4* p_lo;             // FP64 kernel: remainders of the positions
    float4* p_nwlo;           // and of the weights
    double* partial;          // [proxies][3] per chunk
};

// One work item: the weights Q_k of one node summed over a run of its tiles.
// Threads own a pair (k0, k1) of grid indices and every k2; with few pairs,
// groups of threads split the sources of each tile and are summed at the end.
__global__ void __launch_bounds__(kP2MThreads) k_p2m(P2MArgs A)
{
    __shared__ __align__(16) float sL[3][kTile][kLStride];
    __shared__ __align__(16) float sN[kTile][4];
    const int4 it = A.items[blockIdx.x];
    const int node = it.x;
    const int4 info = A.ninfo[node];
    const NodeFrame& F = A.fr[node];
    const int4 gn = A.ngrid[node];
    const int Gn[3] = {gn.x, gn.y, gn.z};
    const int n0 = gn.x, n1 = gn.y, n2 = gn.z;
    const int pairs = n0 * n1;
    const int tid = threadIdx.x;
    const bool fits = (size_t)pairs * n2 * 3 * sizeof(double) <= sizeof(sL);
    const int groups = fits ? max(1, min(3, kP2MThreads / pairs)) : 1;
    const int g = tid / pairs, pr = tid - g * pairs;
    const bool active = g < groups;
    const int k0 = active ? pr / n1 : 0, k1 = active ? pr - (pr / n1) * n1 : 0;

    float acc_h[kMaxN][3], acc_l[kMaxN][3];
#pragma unroll
    for (int k = 0; k < kMaxN; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc_h[k][c] = acc_l[k][c] = 0.0f;

    for (int t = it.y; t < it.z; t++) {
        if (tid < kTile) {
            const int64_t i = (int64_t)t * kTile + tid;
            if (i < A.ns) {
                const double4_32a p = A.pos[i];
                const double4_32a q = A.nw[i];
                const double d[3] = {p.x - F.c[0], p.y - F.c[1], p.z - F.c[2]};
                for (int a = 0; a < 3; a++) {
                    float* L = sL[a][tid];
                    const int na = Gn[a];
                    if (na == 1) {
                        L[0] = 1.0f;
                        continue;
                    }
                    const double pr = d[0] * F.e[a][0] + d[1] * F.e[a][1] + d[2] * F.e[a][2];
                    const float xi = (float)(pr / F.h[a]);
                    // barycentric weights (-1)^k, halved at the two ends
                    int hit = -1;
                    float sum = 0.0f;
                    for (int k = 0; k < na; k++) {
                        const float d = xi - cheb_point(k, na - 1);
                        if (d == 0.0f) hit = k;
                        float w = (k & 1) ? -1.0f : 1.0f;
                        if (k == 0 || k == na - 1) w *= 0.5f;
                        const float tk = d == 0.0f ? 0.0f : w / d;
                        L[k] = tk;
                        sum += tk;
                    }
                    if (hit >= 0) {
                        for (int k = 0; k < na; k++) L[k] = k == hit ? 1.0f : 0.0f;
                    } else {
                        const float inv = 1.0f / sum;
                        for (int k = 0; k < na; k++) L[k] *= inv;
                    }
                }
                sN[tid][0] = (float)q.x;
                sN[tid][1] = (float)q.y;
                sN[tid][2] = (float)q.z;
                sN[tid][3] = 0.0f;
            } else {
                for (int a = 0; a < 3; a++)
                    for (int k = 0; k < Gn[a]; k++) sL[a][tid][k] = 0.0f;
                sN[tid][0] = sN[tid][1] = sN[tid][2] = sN[tid][3] = 0.0f;
            }
        }
        __syncthreads();
        if (active) {
            float ph[kMaxN][3];
#pragma unroll
            for (int k = 0; k < kMaxN; k++) ph[k][0] = ph[k][1] = ph[k][2] = 0.0f;
            for (int s = g; s < kTile; s += groups) {
                const float l01 = sL[0][s][k0] * sL[1][s][k1];
                const float4 nv = *reinterpret_cast<const float4*>(sN[s]);
                const float wx = nv.x * l01, wy = nv.y * l01, wz = nv.z * l01;
                const float4* L2 = reinterpret_cast<const float4*>(sL[2][s]);
#pragma unroll
                for (int q = 0; q < (kMaxN + 3) / 4; q++) {
                    if (4 * q >= n2) break;
                    const float4 l4 = L2[q];
                    const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int k2 = 4 * q + e;
                        if (k2 < kMaxN) {
                            ph[k2][0] = fmaf(lv[e], wx, ph[k2][0]);
                            ph[k2][1] = fmaf(lv[e], wy, ph[k2][1]);
                            ph[k2][2] = fmaf(lv[e], wz, ph[k2][2]);
                        }
                    }
                }
            }
            // fold this tile's FP32 sums into the compensated accumulators
#pragma unroll
            for (int k = 0; k < kMaxN; k++) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const float s = acc_h[k][c] + ph[k][c];
                    const float bp = s - acc_h[k][c];
                    acc_l[k][c] += (acc_h[k][c] - (s - bp)) + (ph[k][c] - bp);
                    acc_h[k][c] = s;
                }
            }
        }
        __syncthreads();
    }

    // sum the groups in order, group 0 writes
    double* buf = reinterpret_cast<double*>(&sL[0][0][0]);
    double Q[kMaxN][3];
#pragma unroll
    for (int k = 0; k < kMaxN; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) Q[k][c] = (double)acc_h[k][c] + (double)acc_l[k][c];
    for (int gg = 1; gg < groups; gg++) {
        if (g == gg) {
            for (int k = 0; k < n2; k++)
                for (int c = 0; c < 3; c++) buf[((size_t)pr * n2 + k) * 3 + c] = Q[k][c];
        }
        __syncthreads();
        if (g == 0) {
            for (int k = 0; k < n2; k++)
                for (int c = 0; c < 3; c++) Q[k][c] += buf[((size_t)pr * n2 + k) * 3 + c];
        }
        __syncthreads();
    }
    if (g != 0 || !active) return;
    const int64_t base = (int64_t)info.z * kTile;
    const bool first_chunk = it.y == info.x;
    for (int k2 = 0; k2 < n2; k2++) {
        const int k = (k0 * n1 + k1) * n2 + k2;
        if (it.w < 0) {
            A.p_nw[base + k] = make_float4((float)Q[k2][0], (float)Q[k2][1], (float)Q[k2][2], 0.0f);
        } else {
            double* dst = A.partial + ((int64_t)it.w + k) * 3;
            dst[0] = Q[k2][0];
            dst[1] = Q[k2][1];
            dst[2] = Q[k2][2];
        }
        if (first_chunk) {
            // the grid point's offset from the frame's centre
            const double t0 = F.h[0] * (double)(n0 > 1 ? cheb_point(k0, n0 - 1) : 0.0f);
            const double t1 = F.h[1] * (double)(n1 > 1 ? cheb_point(k1, n1 - 1) : 0.0f);
            const double t2 = F.h[2] * (double)(n2 > 1 ? cheb_point(k2, n2 - 1) : 0.0f);
            float o[3];
            for (int c = 0; c < 3; c++) o[c] = (float)(t0 * F.e[0][c] + t1 * F.e[1][c] + t2 * F.e[2][c]);
            A.p_pos[base + k] = make_float4(o[0], o[1], o[2], 0.0f);
        }
    }
}

// Chebyshev points of the second kind in FP64 (the float-float proxies).
__device__ __forceinline__ double cheb_point64(int k, int degree) { return cospi((double)k / (double)degree); }

// FP64 P2M for the float-float proxies: thread k of grid row y owns the grid
// pair (k0, k1) = 256 y + k of the item's node and all its k2 points, so the
// tensor factor L0 L1 nw is formed once per source and each proxy costs three
// FP64 FMAs per source.  Summed over the item's tiles, 64 sources at a time
// (their basis values staged in shared memory).
__global__ void __launch_bounds__(kP2MThreads) k_p2m64(P2MArgs A)
{
    __shared__ double sL[3][kP2M64Src][kMaxN64];
    __shared__ double sN[kP2M64Src][3];
    const int4 it = A.items[blockIdx.x];
    const int node = it.x;
    const int4 info = A.ninfo[node];
    const NodeFrame& F = A.fr[node];
    const int4 gn = A.ngrid[node];
    const int Gn[3] = {gn.x, gn.y, gn.z};
    const int n1 = gn.y, n2 = gn.z;
    const int npair = gn.x * n1;
    if ((int)blockIdx.y * kP2MThreads >= npair) return;   // whole CTA, before any barrier
    const int tid = threadIdx.x;
    const int pr = blockIdx.y * kP2MThreads + tid;
    const bool active = pr < npair;
    const int k0 = active ? pr / n1 : 0;
    const int k1 = active ? pr % n1 : 0;
    double q[kMaxN64][3];
#pragma unroll
    for (int m = 0; m < kMaxN64; m++) q[m][0] = q[m][1] = q[m][2] = 0.0;
    for (int t = it.y; t < it.z; t++) {
        for (int half = 0; half < kTile / kP2M64Src; half++) {
            if (tid < kP2M64Src) {
                const int64_t i = (int64_t)t * kTile + half * kP2M64Src + tid;
                if (i < A.ns) {
                    const double4_32a p = A.pos[i];
                    const double4_32a w = A.nw[i];
                    const double d[3] = {p.x - F.c[0], p.y - F.c[1], p.z - F.c[2]};
                    for (int a = 0; a < 3; a++) {
                        double* L = sL[a][tid];
                        const int na = Gn[a];
                        if (na == 1) {
                            L[0] = 1.0;
                            continue;
                        }
                        const double xi = (d[0] * F.e[a][0] + d[1] * F.e[a][1] + d[2] * F.e[a][2]) / F.h[a];
                        int hit = -1;
                        double sum = 0.0;
                        for (int m = 0; m < na; m++) {
                            const double d = xi - cheb_point64(m, na - 1);
                            if (d == 0.0) hit = m;
                            double wm = (m & 1) ? -1.0 : 1.0;
                            if (m == 0 || m == na - 1) wm *= 0.5;
                            const double tm = d == 0.0 ? 0.0 : wm / d;
                            L[m] = tm;
                            sum += tm;
                        }
                        if (hit >= 0) {
                            for (int m = 0; m < na; m++) L[m] = m == hit ? 1.0 : 0.0;
                        } else {
                            const double inv = 1.0 / sum;
                            for (int m = 0; m < na; m++) L[m] *= inv;
                        }
                    }
                    sN[tid][0] = w.x;
                    sN[tid][1] = w.y;
                    sN[tid][2] = w.z;
                } else {
                    for (int a = 0; a < 3; a++)
                        for (int m = 0; m < Gn[a]; m++) sL[a][tid][m] = 0.0;
                    sN[tid][0] = sN[tid][1] = sN[tid][2] = 0.0;
                }
            }
            __syncthreads();
            if (active) {
                for (int s = 0; s < kP2M64Src; s++) {
                    const double l01 = sL[0][s][k0] * sL[1][s][k1];
                    const double wx = l01 * sN[s][0], wy = l01 * sN[s][1], wz = l01 * sN[s][2];
#pragma unroll
                    for (int m = 0; m < kMaxN64; m++) {
                        if (m < n2) {
                            const double l2 = sL[2][s][m];
                            q[m][0] = fma(l2, wx, q[m][0]);
                            q[m][1] = fma(l2, wy, q[m][1]);
                            q[m][2] = fma(l2, wz, q[m][2]);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (!active) return;
#pragma unroll
    for (int k2 = 0; k2 < kMaxN64; k2++) {
        if (k2 >= n2) break;
        const int k = pr * n2 + k2;   // (k0 n1 + k1) n2 + k2
        const int64_t dst = (int64_t)info.z * kTile + k;
        if (it.w < 0) {
            const float h0 = (float)q[k2][0], h1 = (float)q[k2][1], h2 = (float)q[k2][2];
            A.p_nw[dst] = make_float4(h0, h1, h2, 0.0f);
            A.p_nwlo[dst] = make_float4((float)(q[k2][0] - (double)h0), (float)(q[k2][1] - (double)h1),
                                        (float)(q[k2][2] - (double)h2), 0.0f);
        } else {
            double* o = A.partial + ((int64_t)it.w + k) * 3;
            o[0] = q[k2][0];
            o[1] = q[k2][1];
            o[2] = q[k2][2];
        }
        if (it.y == info.x) {
            // the grid point's offset from the frame's centre
            const double t[3] = {Gn[0] > 1 ? F.h[0] * cheb_point64(k0, Gn[0] - 1) : 0.0,
                                 n1 > 1 ? F.h[1] * cheb_point64(k1, n1 - 1) : 0.0,
                                 n2 > 1 ? F.h[2] * cheb_point64(k2, n2 - 1) : 0.0};
            float rh[3], rl[3];
            for (int a = 0; a < 3; a++) {
                const double r = t[0] * F.e[0][a] + t[1] * F.e[1][a] + t[2] * F.e[2][a];
                rh[a] = (float)r;
                rl[a] = (float)(r - (double)rh[a]);
            }
            A.p_pos[dst] = make_float4(rh[0], rh[1], rh[2], 0.0f);
            A.p_lo[dst] = make_float4(rl[0], rl[1], rl[2], 0.0f);
        }
    }
}

// Nodes whose weights were summed in several chunks: add the chunks in order.
// r = node, first partial offset, chunks, proxies.
__global__ void k_p2m_reduce(const int4* __restrict__ red, const int4* __restrict__ ninfo,
                             const double* __restrict__ partial, float4* __restrict__ p_nw,
                             float4* __restrict__ p_nwlo)
{
    const int4 r = red[blockIdx.x];
    const int64_t base = (int64_t)ninfo[r.x].z * kTile;
    for (int k = threadIdx.x; k < r.w; k += blockDim.x) {
        double q[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < r.z; ch++) {
            const double* src = partial + ((int64_t)r.y + (int64_t)ch * r.w + k) * 3;
            q[0] += src[0];
            q[1] += src[1];
            q[2] += src[2];
        }
        const float h0 = (float)q[0], h1 = (float)q[1], h2 = (float)q[2];
        p_nw[base + k] = make_float4(h0, h1, h2, 0.0f);
        if (p_nwlo)
            p_nwlo[base + k] = make_float4((float)(q[0] - (double)h0), (float)(q[1] - (double)h1),
                                           (float)(q[2] - (double)h2), 0.0f);
    }
}

// Box of each block of tpb consecutive sorted targets, FP32 rounded outward
// (the same box the pair kernels compute for the block).
__global__ void __launch_bounds__(kEvalThreads) k_block_boxes(const double* __restrict__ x, int64_t ld, int n,
                                                              int tpb, const double* __restrict__ tsig,
                                                              float4* __restrict__ blo, float4* __restrict__ bhi)
{
    __shared__ float part[6][kEvalThreads / 32];
    __shared__ float psig[kEvalThreads / 32];
    const int b = blockIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float smax = 0.0f;   // sigma(x) mode: the block's largest target sigma
    for (int j = threadIdx.x; j < tpb; j += kEvalThreads) {
        const int64_t i = (int64_t)b * tpb + j;
        if (i >= n) break;
        for (int c = 0; c < 3; c++) {
            const double v = x[c * ld + i];
            lo[c] = fminf(lo[c], __double2float_rd(v));
            hi[c] = fmaxf(hi[c], __double2float_ru(v));
        }
        if (tsig) smax = fmaxf(smax, __double2float_ru(tsig[i]));
    }
    for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    if ((threadIdx.x & 31) == 0) psig[threadIdx.x >> 5] = smax;
    for (int c = 0; c < 3; c++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; c++) {
            part[c][w] = lo[c];
            part[3 + c][w] = hi[c];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < 3; c++)
            for (int k = 1; k < kEvalThreads / 32; k++) {
                part[c][0] = fminf(part[c][0], part[c][k]);
                part[3 + c][0] = fmaxf(part[3 + c][0], part[3 + c][k]);
            }
        float sm = psig[0];
        for (int k = 1; k < kEvalThreads / 32; k++) sm = fmaxf(sm, psig[k]);
        blo[b] = make_float4(part[0][0], part[1][0], part[2][0], sm);
        bhi[b] = make_float4(part[3][0], part[4][0], part[5][0], 0.0f);
    }
}

struct WalkArgs {
    const float4* blo;
    const float4* bhi;
    int nblk;
    const float4* nlo;
    const float4* nhi;
    const float4* acc;     // proxy nodes: centre of the frame, (radius / theta_n)^2
    const int4* info;
    int64_t lev_off[kMaxLevels + 1];
    int top;
    int ntiles;
    int sigx;              // sigma(x) mode: the near width is the block's (blo.w)
    float cut2;
    const uint32_t* off;   // pass 1: list offset of each block
    uint32_t* cnt;         // pass 0: list length of each block
    int* list;             // pass 1
    int2* blist;           // pass 1: (offset, length)
    // target clusters: the nodes block b's cluster (b / bpc) took, a bitmap
    // of cwords words per cluster over the tree's nodes, are left to the
    // cluster's grid (bpc 0: no clusters)
    int bpc = 0;
    const uint32_t* cbits = nullptr;
    int64_t cwords = 0;
    const float4* c_lo = nullptr;   // cluster walk: the clusters' boxes
    const float4* c_hi = nullptr;
    const float4* c_acc = nullptr;
    const float* nr = nullptr;      // node radii
};

// The block rule: node `node` (with proxies) acts on a target box through its
// proxies when its box is beyond the near radius from the target box (sigma
// sw) and the target box satisfies its opening rule.
__device__ __forceinline__ bool box_takes(const WalkArgs& A, int64_t node, float4 bl, float4 bh, float sw)
{
    const float4 lo = A.nlo[node], hi = A.nhi[node];
    const float gx = fmaxf(0.0f, fmaxf(lo.x - bh.x, bl.x - hi.x));
    const float gy = fmaxf(0.0f, fmaxf(lo.y - bh.y, bl.y - hi.y));
    const float gz = fmaxf(0.0f, fmaxf(lo.z - bh.z, bl.z - hi.z));
    if (!(gx * gx + gy * gy + gz * gz > A.cut2 * sw * sw * 1.0001f)) return false;
    const float4 ac = A.acc[node];
    const float dx = fmaxf(0.0f, fmaxf(bl.x - ac.x, ac.x - bh.x));
    const float dy = fmaxf(0.0f, fmaxf(bl.y - ac.y, ac.y - bh.y));
    const float dz = fmaxf(0.0f, fmaxf(bl.z - ac.z, ac.z - bh.z));
    return dx * dx + dy * dy + dz * dz >= ac.w * 1.0001f;
}

// True when cluster c takes node `node` (which has proxies): the node's box is
// beyond the near radius from the cluster's box, the cluster's box satisfies
// the node's opening rule (its proxies represent it there: source side), and
// every point of the node's frame box is at least the cluster's opening radius
// r_C + q h_C from the cluster's centre (the node's field is smooth enough over
// the cluster's box for its grid: target side).  FP32 with a 1e-4 margin.
__device__ __forceinline__ bool cluster_takes(const WalkArgs& A, int64_t node, int c)
{
    if (!box_takes(A, node, A.c_lo[c], A.c_hi[c], A.sigx ? A.c_lo[c].w : A.nlo[node].w)) return false;
    const float4 ac = A.acc[node];
    const float4 cc = A.c_acc[c];
    const float ex = ac.x - cc.x, ey = ac.y - cc.y, ez = ac.z - cc.z;
    const float d = sqrtf(ex * ex + ey * ey + ez * ez) - A.nr[node];
    return d > 0.0f && d * d >= cc.w * 1.0001f;
}

// A warp walks the tree for one target box.  Each round pops up to 32 entries
// from the top of the warp's stack (shared memory), one per lane; a lane's
// node is either emitted (its proxy tiles, or its tile at the leaf level),
// skipped, or opened (its children pushed).  Emitted tiles and pushed
// children are placed by warp prefix sums in lane order, so the walk and its
// list are the same on every call (pass 0 counts, pass 1 writes).  A round
// pops at most kWalkSoft - sp entries, so a round never takes the stack past
// kWalkSoft; at kWalkSoft and above it pops one entry, a plain depth-first
// step, which adds at most one entry per level below the popped node: the
// stack stays within kWalkSoft + kMaxLevels + 1 <= kWalkStack.
constexpr int kWalkSoft = 216;
constexpr int kWalkStack = 256;
static_assert(kWalkSoft + kMaxLevels + 1 <= kWalkStack, "walk stack bound");
enum WalkAct { kSkip = 0, kEmitProxies = 1, kEmitLeaf = 2, kOpen = 3 };

template <class Decide>
__device__ __forceinline__ uint32_t warp_walk(const WalkArgs& A, int* stk, int* list, uint32_t o, int pass,
                                              Decide&& decide)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) stk[0] = A.top << 26;
    __syncwarp();
    int sp = 1;
    uint32_t n = 0;
    while (sp > 0) {
        const int k = min(32, min(sp, max(1, kWalkSoft - sp)));
        int nent = 0, nchild = 0, l = 0, i = 0, act = kSkip;
        int4 f = make_int4(0, 0, -1, 0);
        if (lane < k) {
            const int v = stk[sp - 1 - lane];
            l = v >> 26;
            i = v & ((1 << 26) - 1);
            const int64_t node = A.lev_off[l] + i;
            f = A.info[node];
            act = decide(node, l, f);
            if (act == kEmitProxies) {
                nent = f.w;
            } else if (act == kEmitLeaf) {
                nent = 1;
            } else if (act == kOpen) {
                const int64_t nch = A.lev_off[l] - A.lev_off[l - 1];
                nchild = 2 * i + 1 < nch ? 2 : 1;
            }
        }
        __syncwarp();   // every popped entry is read before children overwrite it
        int pe = nent, pc = nchild;   // inclusive prefix sums over the lanes
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, pe, d), b = __shfl_up_sync(0xffffffffu, pc, d);
            if (lane >= d) {
                pe += a;
                pc += b;
            }
        }
        const int tot_e = __shfl_sync(0xffffffffu, pe, 31), tot_c = __shfl_sync(0xffffffffu, pc, 31);
        if (pass && nent) {
            int* dst = list + o + n + (pe - nent);
            if (act == kEmitLeaf) dst[0] = i;
            else
                for (int q = 0; q < nent; q++) dst[q] = A.ntiles + f.z + q;
        }
        if (nchild) {
            // the odd child below the even one, as a depth-first walk pushes them
            int* dst = stk + (sp - k) + (pc - nchild);
            if (nchild == 2) {
                dst[0] = ((l - 1) << 26) | (2 * i + 1);
                dst[1] = ((l - 1) << 26) | (2 * i);
            } else {
                dst[0] = ((l - 1) << 26) | (2 * i);
            }
        }
        __syncwarp();
        sp = sp - k + tot_c;
        n += (uint32_t)tot_e;
    }
    return n;
}

// The interaction list of each target block, one warp per block: a node with
// proxies that the block's cluster took (bitmap) is skipped, one that the
// block rule accepts is emitted, and the walk descends to the leaf tiles
// otherwise.
__global__ void __launch_bounds__(kWalkThreads) k_tree_walk(WalkArgs A, int pass)
{
    __shared__ int s_stk[kWalkThreads / 32][kWalkStack];
    const int b = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (b >= A.nblk) return;   // whole warps
    const float4 bl = A.blo[b], bh = A.bhi[b];
    const uint32_t o = pass ? A.off[b] : 0u;
    const uint32_t n = warp_walk(A, s_stk[threadIdx.x >> 5], A.list, o, pass, [&](int64_t node, int l, int4 f) {
        if (f.z >= 0) {
            // the cluster's grid has it
            if (A.bpc > 0 && ((A.cbits[(int64_t)(b / A.bpc) * A.cwords + (node >> 5)] >> (node & 31)) & 1u))
                return (int)kSkip;
            // opening rule: the block at distance >= the node's opening radius
            // from the centre of its frame
            if (box_takes(A, node, bl, bh, A.sigx ? bl.w : A.nlo[node].w)) return (int)kEmitProxies;
        }
        return l == 0 ? (int)kEmitLeaf : (int)kOpen;
    });
    if ((threadIdx.x & 31) == 0) {
        if (pass)
            A.blist[b] = make_int2((int)o, (int)n);
        else
            A.cnt[b] = n;
    }
}

// Sort keys that order blocks by decreasing list length (longest first),
// block id as the value.  The key is the length's binary order of magnitude
// only (LSM_ORDER_BUCKETS, the default), so that the stable sort keeps blocks
// of lengths within a factor of two in their Morton order: CTAs resident
// together then share their lists' tiles in L2 (the float-float record sweep on
// the torus read 3.6 GB from DRAM instead of 72 GB, in the same time), while
// the last waves still hold the shortest lists.  0: exact lengths.
#ifndef LSM_ORDER_BUCKETS
#define LSM_ORDER_BUCKETS 1
#endif
__global__ void k_order_keys(const uint32_t* __restrict__ cnt, int n, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ vals)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
#if LSM_ORDER_BUCKETS
    keys[b] = (uint32_t)__clz(cnt[b] | 1u);   // fewer leading zeros: a longer list, earlier
#else
    keys[b] = 0xFFFFFFu - min(cnt[b], 0xFFFFFFu);
#endif
    vals[b] = (uint32_t)b;
}

// ---------------------------------------------------------------- target clusters
// A run of tpc consecutive Morton-sorted targets (a cluster) gets its own
// oriented box: the principal axes of its targets (FP64 mean and covariance,
// Jacobi eigenvectors) and their extents along them, and a tensor Chebyshev
// grid (second kind) on that box with per-axis counts chosen as for the
// source nodes' proxies (the widest axis p + 1 points).  A node far enough
// from the cluster acts on the grid's points instead of on the targets:
// the field of its proxies is smooth over the cluster's box, and its
// degree-p interpolant errs like exp(-C) when the node is at least
// r + q_p h_max from the box's centre (q_p = cosh(C / p), the same bound as
// the source side).  The targets then interpolate the grid's values
// (barycentric Lagrange form, FP64).

__device__ int4 grid_counts_dev(const double h[3], int p, double C)
{
    double hmax = 0.0;
    for (int a = 0; a < 3; a++) hmax = fmax(hmax, h[a]);
    const double d = cosh(C / p) * hmax;
    int n[3];
    for (int a = 0; a < 3; a++) {
        if (!(h[a] > 0.0)) {
            n[a] = 1;
        } else if (h[a] == hmax) {
            n[a] = p + 1;
        } else {
            const int pa = (int)ceil((C + log(32.0)) / acosh(d / h[a]) - 1e-9);
            n[a] = min(p, max(1, pa)) + 1;
        }
    }
    return make_int4(n[0], n[1], n[2], 0);
}

// One CTA per cluster: frame (centre, axes as rows, half-widths) into
// frame[16 c ...], grid counts, the outward box of the oriented box (in
// sigma(x) mode with the cluster's largest target sigma, rounded up, in
// clo.w), and the centre with the squared opening radius (r + q_p h_max)^2.
__global__ void __launch_bounds__(kFrameThreads) k_cluster_frames(const double* __restrict__ x, int64_t ld, int n,
                                                                  int tpc, double C, int p,
                                                                  const double* __restrict__ tsig,
                                                                  double* __restrict__ frame,
                                                                  int4* __restrict__ counts, float4* __restrict__ clo,
                                                                  float4* __restrict__ chi, float4* __restrict__ cacc)
{
    __shared__ double sm[(kFrameThreads / 32) * 7];
    __shared__ double s_e[3][3];
    const int c = blockIdx.x;
    const int64_t i0 = (int64_t)c * tpc, i1 = min((int64_t)n, i0 + tpc);
    const double cnt = (double)max((int64_t)1, i1 - i0);
    double m[3] = {0.0, 0.0, 0.0};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kFrameThreads)
        for (int k = 0; k < 3; k++) m[k] += x[k * ld + i];
    block_sum<3>(m, sm);
    for (int k = 0; k < 3; k++) m[k] /= cnt;
    double cv[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kFrameThreads) {
        const double d0 = x[i] - m[0], d1 = x[ld + i] - m[1], d2 = x[2 * ld + i] - m[2];
        cv[0] += d0 * d0;
        cv[1] += d0 * d1;
        cv[2] += d0 * d2;
        cv[3] += d1 * d1;
        cv[4] += d1 * d2;
        cv[5] += d2 * d2;
    }
    block_sum<6>(cv, sm);
    if (threadIdx.x == 0) {
        double a[3][3] = {{cv[0], cv[1], cv[2]}, {cv[1], cv[3], cv[4]}, {cv[2], cv[4], cv[5]}}, v[3][3];
        jacobi3(a, v);
        for (int ax = 0; ax < 3; ax++)
            for (int k = 0; k < 3; k++) s_e[ax][k] = v[k][ax];
    }
    __syncthreads();
    double e[3][3];
    for (int ax = 0; ax < 3; ax++)
        for (int k = 0; k < 3; k++) e[ax][k] = s_e[ax][k];
    double ext[7] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kFrameThreads) {
        const double d[3] = {x[i] - m[0], x[ld + i] - m[1], x[2 * ld + i] - m[2]};
        for (int ax = 0; ax < 3; ax++) {
            const double t = d[0] * e[ax][0] + d[1] * e[ax][1] + d[2] * e[ax][2];
            ext[ax] = fmax(ext[ax], t);
            ext[3 + ax] = fmax(ext[3 + ax], -t);
        }
        if (tsig) ext[6] = fmax(ext[6], tsig[i]);
    }
    for (int k = 0; k < 7; k++)
        for (int o = 16; o > 0; o >>= 1) ext[k] = fmax(ext[k], __shfl_xor_sync(0xffffffffu, ext[k], o));
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 7; k++) sm[w * 7 + k] = ext[k];
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 0; k < 7; k++)
        for (int j = 1; j < kFrameThreads / 32; j++) ext[k] = fmax(ext[k], sm[j * 7 + k]);
    double h[3], r2 = 0.0;
    for (int ax = 0; ax < 3; ax++) {
        const double hi = ext[ax], lo = -ext[3 + ax];
        h[ax] = 0.5 * (hi - lo);
        r2 += h[ax] * h[ax];
        const double mid = 0.5 * (hi + lo);
        for (int k = 0; k < 3; k++) m[k] += mid * e[ax][k];
    }
    // a small floor keeps the local coordinates of a flat cluster in [-1, 1]
    const double hmin = 1e-9 * sqrt(r2) + 1e-300;
    double hmax = 0.0;
    for (int ax = 0; ax < 3; ax++) {
        h[ax] = fmax(h[ax], hmin);
        hmax = fmax(hmax, h[ax]);
    }
    double* F = frame + 16 * (int64_t)c;
    for (int k = 0; k < 3; k++) F[k] = m[k];
    for (int ax = 0; ax < 3; ax++)
        for (int k = 0; k < 3; k++) F[3 + 3 * ax + k] = e[ax][k];
    for (int ax = 0; ax < 3; ax++) F[12 + ax] = h[ax];
    F[15] = 0.0;
    counts[c] = grid_counts_dev(h, p, C);
    float lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        double ext_k = 0.0;
        for (int ax = 0; ax < 3; ax++) ext_k += h[ax] * fabs(e[ax][k]);
        lo[k] = __double2float_rd(m[k] - ext_k * (1.0 + 1e-12));
        hi[k] = __double2float_ru(m[k] + ext_k * (1.0 + 1e-12));
    }
    clo[c] = make_float4(lo[0], lo[1], lo[2], __double2float_ru(ext[6]));
    chi[c] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    const double R = sqrt(r2) + cosh(C / p) * hmax;
    cacc[c] = make_float4((float)m[0], (float)m[1], (float)m[2], __double2float_ru(R * R));
}

// Grid points of every cluster (one CTA per cluster), SoA with stride ng:
// point g = (k0 n1 + k1) n2 + k2 at centre + sum_a h_a cos(k_a pi / (n_a - 1)) e_a;
// the slots up to the next multiple of the pair kernel's block (tpb) repeat
// the first point.
__global__ void k_cluster_points(const double* __restrict__ frame, const int4* __restrict__ counts, int64_t ng,
                                 int tpb, double* __restrict__ gx)
{
    const int c = blockIdx.x;
    const double* F = frame + 16 * (int64_t)c;
    const int4 nc = counts[c];
    const int np = nc.x * nc.y * nc.z;
    const int npad = (np + tpb - 1) / tpb * tpb;
    for (int g = threadIdx.x; g < npad; g += blockDim.x) {
        const int q = g < np ? g : 0;
        const int k[3] = {q / (nc.y * nc.z), (q / nc.z) % nc.y, q % nc.z};
        const int na[3] = {nc.x, nc.y, nc.z};
        double pt[3] = {F[0], F[1], F[2]};
        for (int ax = 0; ax < 3; ax++) {
            const double t = na[ax] > 1 ? cospi((double)k[ax] / (double)(na[ax] - 1)) : 0.0;
            for (int j = 0; j < 3; j++) pt[j] += F[12 + ax] * t * F[3 + 3 * ax + j];
        }
        for (int j = 0; j < 3; j++) gx[j * ng + nc.w + g] = pt[j];
    }
}

struct ClusterWalkArgs {
    WalkArgs W;            // the tree and the cluster boxes (W.c_lo, ...)
    int ncl;
    int nblk, bpc;         // target blocks, blocks per cluster
    const float4* blo;     // the blocks' boxes
    const float4* bhi;
    uint32_t* cbits;       // pass 1: the bitmap of taken nodes (zeroed)
    const uint32_t* off;   // pass 1: list offset of each cluster
    uint32_t* cnt;         // pass 0: list length of each cluster
    int* list;
    int2* clist;           // pass 1: (offset, length)
};

// Depth-first walk per cluster: the nodes the cluster takes (cluster_takes)
// and their proxy tiles.  The walk does not go below a node that one of the
// cluster's blocks takes itself (the block rule), so every node the cluster
// takes is reached by all of its blocks' walks, which skip it (the bitmap):
// every (target, node) interaction is counted once.
__global__ void __launch_bounds__(kWalkThreads) k_cluster_walk(ClusterWalkArgs A, int pass)
{
    __shared__ int s_stk[kWalkThreads / 32][kWalkStack];
    const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (c >= A.ncl) return;   // whole warps
    const uint32_t o = pass ? A.off[c] : 0u;
    const int b0 = c * A.bpc, b1 = min(A.nblk, b0 + A.bpc);
    const uint32_t n = warp_walk(A.W, s_stk[threadIdx.x >> 5], A.list, o, pass, [&](int64_t node, int l, int4 f) {
        if (f.z >= 0) {
            if (cluster_takes(A.W, node, c)) {
                if (pass) atomicOr(&A.cbits[(int64_t)c * A.W.cwords + (node >> 5)], 1u << (node & 31));
                return (int)kEmitProxies;
            }
            for (int b = b0; b < b1; b++)
                if (box_takes(A.W, node, A.blo[b], A.bhi[b], A.W.sigx ? A.blo[b].w : A.W.nlo[node].w))
                    return (int)kSkip;
        }
        return l == 0 ? (int)kSkip : (int)kOpen;
    });
    if ((threadIdx.x & 31) == 0) {
        if (pass)
            A.clist[c] = make_int2((int)o, (int)n);
        else
            A.cnt[c] = n;
    }
}

// Each block of grid points takes its cluster's list; launch order as given.
__global__ void k_grid_blocks(const int* __restrict__ gb_cluster, int ngblk, const int2* __restrict__ clist,
                              int2* __restrict__ gblist, int* __restrict__ gorder)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ngblk) return;
    gblist[g] = clist[gb_cluster[g]];
    gorder[g] = g;
}

// The targets' share of their clusters' far field: tensor Lagrange
// interpolation (barycentric form on the Chebyshev points of the second kind)
// of the grid values, Phi in FP64, the gradient likewise; added to res [4][n]
// and, when recording, far_io [4][n].
__global__ void k_cluster_l2p(const double* __restrict__ x, int64_t ld, int n, int tpc,
                              const double* __restrict__ frame, const int4* __restrict__ counts,
                              const double* __restrict__ rg, int64_t ng, double* __restrict__ res,
                              double* __restrict__ far_io)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = i / tpc;
    const double* F = frame + 16 * (int64_t)c;
    const int4 nc = counts[c];
    const int na[3] = {nc.x, nc.y, nc.z};
    const double d[3] = {x[i] - F[0], x[ld + i] - F[1], x[2 * ld + i] - F[2]};
    double L[3][kMaxN64];
    for (int ax = 0; ax < 3; ax++) {
        const int m = na[ax];
        if (m == 1) {
            L[ax][0] = 1.0;
            continue;
        }
        double xi = (d[0] * F[3 + 3 * ax] + d[1] * F[4 + 3 * ax] + d[2] * F[5 + 3 * ax]) / F[12 + ax];
        xi = fmin(1.0, fmax(-1.0, xi));
        int hit = -1;
        double den = 0.0;
        for (int k = 0; k < m; k++) {
            const double t = cospi((double)k / (double)(m - 1));
            const double wk = ((k & 1) ? -1.0 : 1.0) * ((k == 0 || k == m - 1) ? 0.5 : 1.0);
            if (xi == t) hit = k;
            L[ax][k] = wk / (xi - t);
            den += L[ax][k];
        }
        for (int k = 0; k < m; k++) L[ax][k] = hit >= 0 ? (k == hit ? 1.0 : 0.0) : L[ax][k] / den;
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t base = nc.w;
    for (int k0 = 0; k0 < na[0]; k0++) {
        double s1[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k1 = 0; k1 < na[1]; k1++) {
            double s2[4] = {0.0, 0.0, 0.0, 0.0};
            const int64_t g0 = base + ((int64_t)k0 * na[1] + k1) * na[2];
            for (int k2 = 0; k2 < na[2]; k2++)
                for (int f = 0; f < 4; f++) s2[f] = fma(L[2][k2], rg[f * ng + g0 + k2], s2[f]);
            for (int f = 0; f < 4; f++) s1[f] = fma(L[1][k1], s2[f], s1[f]);
        }
        for (int f = 0; f < 4; f++) acc[f] = fma(L[0][k0], s1[f], acc[f]);
    }
    for (int f = 0; f < 4; f++) res[(int64_t)f * n + i] += acc[f];
    if (far_io)
        for (int f = 0; f < 4; f++) far_io[(int64_t)f * n + i] += acc[f];
}

}  // namespace

bool tree_wanted(const Ctx* ctx, const Mesh* me, bool ff)
{
    if (me->ntiles < 8) return false;
    if (ff) return ctx->opt.tree_ff_min_sources >= 0 && me->ns >= ctx->opt.tree_ff_min_sources;
    if (me->tune_mode >= 0) return me->tune_mode == 1;
    return ctx->opt.tree_min_sources >= 0 && me->ns >= ctx->opt.tree_min_sources;
}

void tree_free(Tree* t)
{
    if (!t) return;
    void* ps[] = {t->node_lo, t->node_hi, t->node_info, t->node_acc, t->node_r, t->p_pos, t->p_nw, t->p_lo, t->p_nwlo,
                  t->tile_lo,
                  t->tile_hi, t->tile_chi, t->tile_clo};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete t;
}

bool newton_tree_wanted(const Ctx* ctx, const Mesh* me)
{
    if (ctx->opt.newton_tree_degree <= 0) return false;
    const bool tuned = me->tune_mode == 1;
    const int d = tuned ? me->tune_degree : ctx->opt.tree_degree;
    const float th = tuned ? me->tune_theta : ctx->opt.tree_theta;
    const int nd = ctx->opt.newton_tree_degree;
    const float nth = ctx->opt.newton_tree_theta;
    return nd <= d && nth >= th && (nd < d || nth > th);
}

int tree_ensure(Ctx* ctx, Mesh* me, cudaStream_t st, bool ff, bool newton)
{
    const bool tuned = !ff && me->tune_mode == 1;
    int degree = ff ? ctx->opt.tree_ff_degree : (tuned ? me->tune_degree : ctx->opt.tree_degree);
    float theta = ff ? ctx->opt.tree_ff_theta : (tuned ? me->tune_theta : ctx->opt.tree_theta);
    newton = newton && !ff;
    if (newton) {
        degree = ctx->opt.newton_tree_degree;
        theta = ctx->opt.newton_tree_theta;
    }
    const int grid = ctx->opt.tree_grid;
    Tree*& slot = ff ? me->tree_ff : (newton ? me->tree_newton : me->tree);
    if (slot && slot->degree == degree && slot->theta == theta && slot->grid == grid) return LSM_OK;
    if (!ff && degree > kMaxDeg32) {
        ctx->err = "tree: the mixed path's degree is at most 12";
        return LSM_E_INVALID_ARG;
    }
    if (slot) me->bytes -= slot->bytes;
    tree_free(slot);
    slot = nullptr;
    Tree* T = new (std::nothrow) Tree();
    if (!T) return LSM_E_OOM;
    T->ff = ff;
    auto fail = [&](int rc) {
        tree_free(T);
        return rc;
    };
    auto alloc = [&](auto** p, size_t count) -> bool {
        using E = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
        if (cudaMalloc((void**)p, count * sizeof(E) + 16) != cudaSuccess) return false;
        T->bytes += count * sizeof(E);
        return true;
    };
    T->degree = degree;
    T->theta = theta;
    T->grid = grid;
    T->ntiles = (int)me->ntiles;
    // levels: level l has ceil(ntiles / 2^l) nodes, up to a single root
    int64_t n = me->ntiles;
    int lev = 0;
    T->lev_off[0] = 0;
    while (true) {
        T->lev_off[lev + 1] = T->lev_off[lev] + n;
        if (n == 1 || lev == kMaxLevels - 1) break;
        n = (n + 1) / 2;
        lev++;
    }
    if (n != 1) {
        ctx->err = "tree: too many source tiles";
        return fail(LSM_E_INVALID_ARG);
    }
    T->top = lev;
    T->nnodes = T->lev_off[lev + 1];
    if (!alloc(&T->node_lo, T->nnodes) || !alloc(&T->node_hi, T->nnodes) || !alloc(&T->node_info, T->nnodes) ||
        !alloc(&T->node_acc, T->nnodes) || !alloc(&T->node_r, T->nnodes)) {
        cudaGetLastError();
        ctx->err = "tree: out of device memory";
        return fail(LSM_E_OOM);
    }
    k_nodes_leaf<<<blocks_of(me->ntiles, 256), 256, 0, st>>>(me->tile_lo, me->tile_hi, (int)me->ntiles, T->node_lo,
                                                               T->node_hi, T->node_info);
    if (cudaGetLastError() != cudaSuccess) return fail(LSM_E_CUDA);
    ctx->launches++;
    for (int l = 1; l <= T->top; l++) {
        const int64_t c0 = T->lev_off[l - 1], nc = T->lev_off[l] - c0, o = T->lev_off[l],
                      nn = T->lev_off[l + 1] - o;
        k_nodes_up<<<blocks_of(nn, 256), 256, 0, st>>>(T->node_lo + c0, T->node_hi + c0, T->node_info + c0, (int)nc,
                                                       T->node_lo + o, T->node_hi + o, T->node_info + o, (int)nn);
        if (cudaGetLastError() != cudaSuccess) return fail(LSM_E_CUDA);
        ctx->launches++;
    }
    // node frames: principal axes on the device (grid 1), or the axis-aligned
    // boxes (grid 2, filled on the host below)
    Scratch sb(st);
    NodeFrame* d_fr = nullptr;
    const int64_t n_inner = T->nnodes - T->lev_off[1];
    if (sb.get(&d_fr, (size_t)T->nnodes)) {
        ctx->err = "tree: out of device memory";
        return fail(LSM_E_OOM);
    }
    std::vector<NodeFrame> hfr(T->nnodes);
    if (grid != 2 && n_inner > 0) {
        k_node_frames<<<(unsigned)n_inner, kFrameThreads, 0, st>>>(me->s64_pos, me->ntiles * kTile, T->node_info,
                                                                  T->lev_off[1],
                                                                  d_fr);
        if (cudaGetLastError() != cudaSuccess) return fail(LSM_E_CUDA);
        ctx->launches++;
        if (cudaMemcpyAsync(hfr.data() + T->lev_off[1], d_fr + T->lev_off[1], sizeof(NodeFrame) * n_inner,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            ctx->err = "tree: copy of the node frames failed";
            return fail(LSM_E_CUDA);
        }
    }
    // grids and proxy assignment on the host
    std::vector<float4> hlo(T->nnodes), hhi(T->nnodes);
    std::vector<int4> hinfo(T->nnodes);
    if (cudaMemcpyAsync(hlo.data(), T->node_lo, sizeof(float4) * T->nnodes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(hhi.data(), T->node_hi, sizeof(float4) * T->nnodes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(hinfo.data(), T->node_info, sizeof(int4) * T->nnodes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        ctx->err = "tree: copy of the node boxes failed";
        return fail(LSM_E_CUDA);
    }
    if (grid == 2) {
        for (int64_t node = T->lev_off[1]; node < T->nnodes; node++) {
            NodeFrame& F = hfr[node];
            const float l[3] = {hlo[node].x, hlo[node].y, hlo[node].z}, u[3] = {hhi[node].x, hhi[node].y, hhi[node].z};
            for (int a = 0; a < 3; a++) {
                F.c[a] = 0.5 * ((double)l[a] + (double)u[a]);
                F.h[a] = 0.5 * ((double)u[a] - (double)l[a]);
                for (int c = 0; c < 3; c++) F.e[a][c] = a == c ? 1.0 : 0.0;
            }
        }
    }
    // the degree ladder; grid 2: one degree
    const double C = tree_bound(degree, theta);
    std::vector<int> ladder;
    for (int p = degree; p >= (grid == 2 ? degree : std::max(3, degree / 2 - 1)); p -= 2) ladder.push_back(p);
    std::vector<int4> items, reds;
    std::vector<int4> hgrid(T->nnodes, make_int4(1, 1, 1, 0));
    std::vector<float4> hacc(T->nnodes, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    std::vector<float> hrad(T->nnodes, 0.0f);
    std::vector<float4> ptlo, pthi, ptchi, ptclo;
    int64_t nptiles = 0, npartial = 0;
    for (int l = 1; l <= T->top; l++) {
        for (int64_t node = T->lev_off[l]; node < T->lev_off[l + 1]; node++) {
            int4& f = hinfo[node];
            NodeFrame& F = hfr[node];
            const int64_t s0 = (int64_t)f.x * kTile;
            const int64_t s1 = (int64_t)(f.x + f.y) * kTile;   // slots, padding included
            // the largest ladder degree whose grid the node can carry: sources
            // >= 1.5 x proxies (grid 2: >= 2 x)
            int4 gn = make_int4(1, 1, 1, 0);
            int64_t np = 0;
            int pn = 0;
            for (int p : ladder) {
                const int4 g = grid_counts(F.h, p, C, grid);
                const int64_t n3 = (int64_t)g.x * g.y * g.z;
                if (grid == 2 ? 2 * n3 <= s1 - s0 : 3 * n3 <= 2 * (s1 - s0)) {
                    gn = g;
                    np = n3;
                    pn = p;
                    break;
                }
            }
            if (np == 0) continue;
            hgrid[node] = gn;
            // the frame's centre becomes its float pair exactly: the proxies
            // are placed relative to it and the kernels rebuild it from the
            // two floats of the proxy tiles
            for (int a = 0; a < 3; a++) {
                const float h = (float)F.c[a];
                F.c[a] = (double)h + (double)(float)(F.c[a] - (double)h);
            }
            // the opening radius
            const double r = std::sqrt(F.h[0] * F.h[0] + F.h[1] * F.h[1] + F.h[2] * F.h[2]);
            const double hmax = std::max(F.h[0], std::max(F.h[1], F.h[2]));
            const double R = grid == 2 ? r / theta : r + std::cosh(C / pn) * hmax;
            hacc[node] = make_float4((float)F.c[0], (float)F.c[1], (float)F.c[2], (float)(R * R));
            hrad[node] = std::nextafter((float)r, INFINITY);
            const int npt = (int)((np + kTile - 1) / kTile);
            f.z = (int)nptiles;
            f.w = npt;
            for (int j = 0; j < npt; j++) {
                const int cnt = (int)std::min<int64_t>(kTile, np - (int64_t)j * kTile);
                ptlo.push_back(hlo[node]);
                pthi.push_back(make_float4(hhi[node].x, hhi[node].y, hhi[node].z, (float)cnt));
                float ch[3], cl[3];
                for (int a = 0; a < 3; a++) {
                    ch[a] = (float)F.c[a];
                    cl[a] = (float)(F.c[a] - (double)ch[a]);
                }
                ptchi.push_back(make_float4(ch[0], ch[1], ch[2], 0.0f));
                ptclo.push_back(make_float4(cl[0], cl[1], cl[2], 0.0f));
            }
            nptiles += npt;
            const int nch = (f.y + kP2MChunkTiles - 1) / kP2MChunkTiles;
            if (nch == 1) {
                items.push_back(make_int4((int)node, f.x, f.x + f.y, -1));
            } else {
                reds.push_back(make_int4((int)node, (int)npartial, nch, (int)np));
                for (int c = 0; c < nch; c++) {
                    const int t0 = f.x + c * kP2MChunkTiles, t1 = std::min(f.x + f.y, t0 + kP2MChunkTiles);
                    items.push_back(make_int4((int)node, t0, t1, (int)(npartial + (int64_t)c * np)));
                }
                npartial += (int64_t)nch * np;
            }
            if (nptiles + me->ntiles >= (int64_t)1 << 30 || npartial >= (int64_t)1 << 30) {
                ctx->err = "tree: too many proxies";
                return fail(LSM_E_INVALID_ARG);
            }
        }
    }
    if (cudaMemcpyAsync(T->node_acc, hacc.data(), sizeof(float4) * T->nnodes, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(T->node_r, hrad.data(), sizeof(float) * T->nnodes, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d_fr, hfr.data(), sizeof(NodeFrame) * T->nnodes, cudaMemcpyHostToDevice, st)) {
        ctx->err = "tree: copy failed";
        return fail(LSM_E_CUDA);
    }
    T->nptiles = (int)nptiles;
    const int64_t nall = me->ntiles + nptiles;
    if (!alloc(&T->tile_lo, nall) || !alloc(&T->tile_hi, nall) || !alloc(&T->tile_chi, nall) ||
        !alloc(&T->tile_clo, nall) || !alloc(&T->p_pos, std::max<int64_t>(1, nptiles) * kTile) ||
        !alloc(&T->p_nw, std::max<int64_t>(1, nptiles) * kTile) ||
        (ff && (!alloc(&T->p_lo, std::max<int64_t>(1, nptiles) * kTile) ||
                !alloc(&T->p_nwlo, std::max<int64_t>(1, nptiles) * kTile)))) {
        cudaGetLastError();
        ctx->err = "tree: out of device memory";
        return fail(LSM_E_OOM);
    }
    const size_t b4 = sizeof(float4);
    const size_t nt = (size_t)me->ntiles;
    if (cudaMemcpyAsync(T->node_info, hinfo.data(), sizeof(int4) * T->nnodes, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(T->tile_lo, me->tile_lo, b4 * nt, cudaMemcpyDeviceToDevice, st) ||
        cudaMemcpyAsync(T->tile_hi, me->tile_hi, b4 * nt, cudaMemcpyDeviceToDevice, st) ||
        cudaMemcpyAsync(T->tile_chi, me->tile_chi, b4 * nt, cudaMemcpyDeviceToDevice, st) ||
        cudaMemcpyAsync(T->tile_clo, me->tile_clo, b4 * nt, cudaMemcpyDeviceToDevice, st)) {
        ctx->err = "tree: copy failed";
        return fail(LSM_E_CUDA);
    }
    if (nptiles > 0 &&
        (cudaMemcpyAsync(T->tile_lo + nt, ptlo.data(), b4 * nptiles, cudaMemcpyHostToDevice, st) ||
         cudaMemcpyAsync(T->tile_hi + nt, pthi.data(), b4 * nptiles, cudaMemcpyHostToDevice, st) ||
         cudaMemcpyAsync(T->tile_chi + nt, ptchi.data(), b4 * nptiles, cudaMemcpyHostToDevice, st) ||
         cudaMemcpyAsync(T->tile_clo + nt, ptclo.data(), b4 * nptiles, cudaMemcpyHostToDevice, st))) {
        ctx->err = "tree: copy failed";
        return fail(LSM_E_CUDA);
    }
    if (!items.empty()) {
        Scratch s(st);
        int4 *d_items = nullptr, *d_reds = nullptr, *d_grid = nullptr;
        double* d_part = nullptr;
        if (s.get(&d_items, items.size()) || s.get(&d_reds, std::max<size_t>(1, reds.size())) ||
            s.get(&d_part, std::max<int64_t>(1, npartial) * 3) || s.get(&d_grid, (size_t)T->nnodes)) {
            ctx->err = "tree: out of device memory";
            return fail(LSM_E_OOM);
        }
        if (cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st) ||
            cudaMemcpyAsync(d_grid, hgrid.data(), sizeof(int4) * hgrid.size(), cudaMemcpyHostToDevice, st) ||
            (!reds.empty() &&
             cudaMemcpyAsync(d_reds, reds.data(), sizeof(int4) * reds.size(), cudaMemcpyHostToDevice, st))) {
            ctx->err = "tree: copy failed";
            return fail(LSM_E_CUDA);
        }
        P2MArgs P;
        P.pos = me->s64_pos;
        P.nw = me->s64_nw;
        P.ns = me->ntiles * kTile;   // slots: padding has zero weight
        P.fr = d_fr;
        P.ninfo = T->node_info;
        P.items = d_items;
        P.ngrid = d_grid;
        P.p_pos = T->p_pos;
        P.p_nw = T->p_nw;
        P.p_lo = T->p_lo;
        P.p_nwlo = T->p_nwlo;
        P.partial = d_part;
        if (ff) {
            int64_t nmax = 0;   // grid pairs (k0, k1) per node at most
            for (const int4& it : items) nmax = std::max<int64_t>(nmax, (int64_t)hgrid[it.x].x * hgrid[it.x].y);
            const dim3 grid((unsigned)items.size(), (unsigned)((nmax + kP2MThreads - 1) / kP2MThreads));
            k_p2m64<<<grid, kP2MThreads, 0, st>>>(P);
        } else {
            k_p2m<<<(unsigned)items.size(), kP2MThreads, 0, st>>>(P);
        }
        if (cudaGetLastError() != cudaSuccess) return fail(LSM_E_CUDA);
        ctx->launches++;
        if (!reds.empty()) {
            k_p2m_reduce<<<(unsigned)reds.size(), 256, 0, st>>>(d_reds, T->node_info, d_part, T->p_nw, T->p_nwlo);
            if (cudaGetLastError() != cudaSuccess) return fail(LSM_E_CUDA);
            ctx->launches++;
        }
        // the host vectors and the scratch must outlive the copies
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            ctx->err = "tree: build failed";
            return fail(LSM_E_CUDA);
        }
    } else if (cudaStreamSynchronize(st) != cudaSuccess) {
        ctx->err = "tree: build failed";
        return fail(LSM_E_CUDA);
    }
    slot = T;
    me->bytes += T->bytes;
    return LSM_OK;
}

static void fill_walk_tree(WalkArgs& W, const Tree* T, double cut)
{
    W.nlo = T->node_lo;
    W.nhi = T->node_hi;
    W.acc = T->node_acc;
    W.info = T->node_info;
    W.nr = T->node_r;
    for (int l = 0; l <= kMaxLevels; l++) W.lev_off[l] = l <= T->top + 1 ? T->lev_off[l] : 0;
    W.top = T->top;
    W.ntiles = T->ntiles;
    W.cut2 = (float)(cut * cut);
}

int cluster_setup(Ctx* ctx, const Tree* T, const Targets& t, int tpc, int tpb, double cut, const double* tsig,
                  Scratch& s, ClusterPlan* P, cudaStream_t st)
{
    ClusterPlan& cp = *P;
    cp.tpc = tpc;
    cp.ncl = (t.n + tpc - 1) / tpc;
    const int ncl = cp.ncl;
    LSM_CUDA_TRY(ctx, s.get(&cp.box_lo, ncl));
    LSM_CUDA_TRY(ctx, s.get(&cp.box_hi, ncl));
    LSM_CUDA_TRY(ctx, s.get(&cp.cacc, ncl));
    LSM_CUDA_TRY(ctx, s.get(&cp.frame, 16 * (size_t)ncl));
    LSM_CUDA_TRY(ctx, s.get(&cp.counts, ncl));
    const double C = tree_bound(T->degree, T->theta);
    k_cluster_frames<<<ncl, kFrameThreads, 0, st>>>(t.x, t.ld, t.n, tpc, C, T->degree, tsig, cp.frame, cp.counts,
                                                    cp.box_lo,
                                                    cp.box_hi, cp.cacc);
    LSM_LAUNCHED(ctx);
    // grid offsets on the host: each cluster's points start on a block boundary
    std::vector<int4> hc(ncl);
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(hc.data(), cp.counts, sizeof(int4) * ncl, cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    std::vector<int> gb_cluster;
    int64_t ng = 0;
    for (int c = 0; c < ncl; c++) {
        const int64_t np = (int64_t)hc[c].x * hc[c].y * hc[c].z;
        const int64_t nb = (np + tpb - 1) / tpb;
        hc[c].w = (int)ng;
        for (int64_t b = 0; b < nb; b++) gb_cluster.push_back(c);
        ng += nb * tpb;
    }
    if (ng >= ((int64_t)1 << 31)) {
        ctx->err = "tree: too many cluster grid points";
        return LSM_E_INVALID_ARG;
    }
    cp.ng = ng;
    cp.ngblk = (int)gb_cluster.size();
    int* d_gbc;
    LSM_CUDA_TRY(ctx, s.get(&d_gbc, gb_cluster.size()));
    LSM_CUDA_TRY(ctx, s.get(&cp.gx, 3 * (size_t)ng));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(cp.counts, hc.data(), sizeof(int4) * ncl, cudaMemcpyHostToDevice, st));
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(d_gbc, gb_cluster.data(), sizeof(int) * gb_cluster.size(),
                                      cudaMemcpyHostToDevice, st));
    k_cluster_points<<<ncl, 128, 0, st>>>(cp.frame, cp.counts, ng, tpb, cp.gx);
    LSM_LAUNCHED(ctx);
    // the target blocks' boxes (as the block walk sees them) and the bitmap
    const int nblk = (t.n + tpb - 1) / tpb;
    LSM_CUDA_TRY(ctx, s.get(&cp.blo, nblk));
    LSM_CUDA_TRY(ctx, s.get(&cp.bhi, nblk));
    k_block_boxes<<<nblk, kEvalThreads, 0, st>>>(t.x, t.ld, t.n, tpb, tsig, cp.blo, cp.bhi);
    LSM_LAUNCHED(ctx);
    cp.cwords = (T->nnodes + 31) / 32;
    LSM_CUDA_TRY(ctx, s.get(&cp.cbits, (size_t)cp.cwords * ncl));
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(cp.cbits, 0, sizeof(uint32_t) * (size_t)cp.cwords * ncl, st));
    // the clusters' lists: count, scan, write
    ClusterWalkArgs A;
    fill_walk_tree(A.W, T, cut);
    A.W.sigx = tsig != nullptr;
    A.W.c_lo = cp.box_lo;
    A.W.c_hi = cp.box_hi;
    A.W.c_acc = cp.cacc;
    A.W.cwords = cp.cwords;
    A.ncl = ncl;
    A.nblk = nblk;
    A.bpc = tpc / tpb;
    A.blo = cp.blo;
    A.bhi = cp.bhi;
    A.cbits = cp.cbits;
    uint32_t* cnt;
    LSM_CUDA_TRY(ctx, s.get(&cnt, (size_t)ncl + 1));
    int2* clist;
    LSM_CUDA_TRY(ctx, s.get(&clist, ncl));
    A.off = cnt;
    A.cnt = cnt;
    A.list = nullptr;
    A.clist = clist;
    k_cluster_walk<<<blocks_of((int64_t)ncl * 32, kWalkThreads), kWalkThreads, 0, st>>>(A, 0);
    LSM_LAUNCHED(ctx);
    int rc = scan_exclusive(ctx, cnt, ncl, cnt + ncl, st);
    if (rc != LSM_OK) return rc;
    uint32_t h_total = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&h_total, cnt + ncl, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (h_total >= (1u << 31)) {
        ctx->err = "tree: cluster lists too long";
        return LSM_E_INVALID_ARG;
    }
    cp.total = h_total;
    LSM_CUDA_TRY(ctx, s.get(&cp.list, std::max<uint32_t>(1u, h_total)));
    A.list = cp.list;
    k_cluster_walk<<<blocks_of((int64_t)ncl * 32, kWalkThreads), kWalkThreads, 0, st>>>(A, 1);
    LSM_LAUNCHED(ctx);
    LSM_CUDA_TRY(ctx, s.get(&cp.gblist, std::max(1, cp.ngblk)));
    LSM_CUDA_TRY(ctx, s.get(&cp.gorder, std::max(1, cp.ngblk)));
    if (cp.ngblk > 0) {
        k_grid_blocks<<<blocks_of(cp.ngblk, 256), 256, 0, st>>>(d_gbc, cp.ngblk, clist, cp.gblist, cp.gorder);
        LSM_LAUNCHED(ctx);
    }
    return LSM_OK;
}

int cluster_l2p(Ctx* ctx, const ClusterPlan& cp, const Targets& t, const double* rg, double* res, double* far_io,
                cudaStream_t st)
{
    if (t.n <= 0 || cp.ncl <= 0) return LSM_OK;
    k_cluster_l2p<<<blocks_of(t.n, 128), 128, 0, st>>>(t.x, t.ld, t.n, cp.tpc, cp.frame, cp.counts, rg, cp.ng, res,
                                                      far_io);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

int tree_lists(Ctx* ctx, const Tree* T, const Targets& t, int tpb, const double* tsig, Scratch& s, int** list,
               int2** blist, int** order, int64_t* total_out, cudaStream_t st, double cut_override,
               const ClusterPlan* clusters)
{
    const int nblk = (t.n + tpb - 1) / tpb;
    float4 *blo = nullptr, *bhi = nullptr;
    uint32_t* cnt = nullptr;
    LSM_CUDA_TRY(ctx, s.get(&blo, nblk));
    LSM_CUDA_TRY(ctx, s.get(&bhi, nblk));
    LSM_CUDA_TRY(ctx, s.get(&cnt, (size_t)nblk + 1));
    LSM_CUDA_TRY(ctx, s.get(blist, nblk));
    k_block_boxes<<<nblk, kEvalThreads, 0, st>>>(t.x, t.ld, t.n, tpb, tsig, blo, bhi);
    LSM_LAUNCHED(ctx);
    WalkArgs W;
    W.blo = blo;
    W.bhi = bhi;
    W.nblk = nblk;
    W.nlo = T->node_lo;
    W.nhi = T->node_hi;
    W.acc = T->node_acc;
    W.info = T->node_info;
    for (int l = 0; l <= kMaxLevels; l++) W.lev_off[l] = l <= T->top + 1 ? T->lev_off[l] : 0;
    W.top = T->top;
    W.ntiles = T->ntiles;
    W.sigx = tsig != nullptr;
    W.nr = T->node_r;
    // the near radius of the pair kernel that evaluates the lists
    const double cut = cut_override > 0 ? cut_override : (T->ff ? ctx->opt.cutoff_fp64 : ctx->opt.cutoff_mixed);
    W.cut2 = (float)(cut * cut);
    if (clusters && clusters->tpc > 0) {
        W.bpc = clusters->tpc / tpb;
        W.cbits = clusters->cbits;
        W.cwords = clusters->cwords;
    }
    W.off = cnt;
    W.cnt = cnt;
    W.list = nullptr;
    W.blist = *blist;
    k_tree_walk<<<blocks_of((int64_t)nblk * 32, kWalkThreads), kWalkThreads, 0, st>>>(W, 0);
    LSM_LAUNCHED(ctx);
    // launch order: longest lists first, so that the last wave is short
    uint32_t* keys = nullptr;
    LSM_CUDA_TRY(ctx, s.get(&keys, nblk));
    LSM_CUDA_TRY(ctx, s.get(order, nblk));
    uint32_t* vals = reinterpret_cast<uint32_t*>(*order);
    k_order_keys<<<blocks_of(nblk, 256), 256, 0, st>>>(cnt, nblk, keys, vals);
    LSM_LAUNCHED(ctx);
    int rc0 = radix_sort_pairs(ctx, keys, vals, nblk, 24, st);
    if (rc0 != LSM_OK) return rc0;
    uint32_t* total = cnt + nblk;
    int rc = scan_exclusive(ctx, cnt, nblk, total, st);
    if (rc != LSM_OK) return rc;
    uint32_t h_total = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&h_total, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (h_total >= (1u << 31)) {
        ctx->err = "tree: interaction lists too long";
        return LSM_E_INVALID_ARG;
    }
    *total_out = h_total;
    LSM_CUDA_TRY(ctx, s.get(list, std::max<uint32_t>(1u, h_total)));
    W.list = *list;
    k_tree_walk<<<blocks_of((int64_t)nblk * 32, kWalkThreads), kWalkThreads, 0, st>>>(W, 1);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace lsm
