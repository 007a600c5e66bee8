// geometry.cu -- resident mesh state built on the device at upload:
// triangle frames and sigma (Sec. 3, eq. tparam), vertex pseudonormals
// (eq. mkvertexpn), source nodes of the discrete sum (eq. discrete_int) in
// Morton order with per-tile bounding boxes and FP32 tile-local copies, and
// chart nodes with their pseudonormal directions (eq. mkpseudovec).
#include <algorithm>
#include <cstring>

#include <type_traits>

#include "lsm_internal.cuh"

namespace lsm {
namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ long long ordered_bits(double v)
{
    long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double from_ordered(long long b)
{
    return __longlong_as_double(b >= 0 ? b : (b ^ 0x7fffffffffffffffLL));
}

// Per-triangle frames, sigma, interior angles accumulated into the vertex
// sums of eq. mkvertexpn, signed volume and the sigma range.
//   vacc [nv][4] = (sum theta * N_hat, sum theta)
//   red  [0] = volume (double), [1] = ordered(min sigma), [2] = ordered(max sigma),
//        [3] = count of triangles with |N| == 0 or sigma <= 0 (as double)
__global__ void k_tri_geometry(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                               int64_t m, const double* __restrict__ sigma_in,
                               double* __restrict__ tri_n, double* __restrict__ tri_sigma,
                               double* __restrict__ vacc, double* __restrict__ red)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double vol = 0.0;
    double smin = 1e300, smax = -1e300, bad = 0.0;
    if (j < m) {
        const int ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
        const double3 p1 = make_double3(verts[3 * ia], verts[3 * ia + 1], verts[3 * ia + 2]);
        const double3 p2 = make_double3(verts[3 * ib], verts[3 * ib + 1], verts[3 * ib + 2]);
        const double3 p3 = make_double3(verts[3 * ic], verts[3 * ic + 1], verts[3 * ic + 2]);
        const double3 tu = make_double3(p2.x - p1.x, p2.y - p1.y, p2.z - p1.z);
        const double3 tv = make_double3(p3.x - p1.x, p3.y - p1.y, p3.z - p1.z);
        const double3 n = make_double3(tu.y * tv.z - tu.z * tv.y, tu.z * tv.x - tu.x * tv.z,
                                       tu.x * tv.y - tu.y * tv.x);
        const double nn = sqrt(n.x * n.x + n.y * n.y + n.z * n.z);
        tri_n[3 * j] = n.x;
        tri_n[3 * j + 1] = n.y;
        tri_n[3 * j + 2] = n.z;
        const double sg = sigma_in ? sigma_in[j] : 0.5 * sqrt(nn);  // 0.5 sqrt(2 area)
        tri_sigma[j] = sg;
        smin = sg;
        smax = sg;
        if (!(nn > 0.0) || !(sg > 0.0)) bad = 1.0;
        // signed volume contribution p1 . (p2 x p3) / 6
        vol = (p1.x * (p2.y * p3.z - p2.z * p3.y) + p1.y * (p2.z * p3.x - p2.x * p3.z) +
               p1.z * (p2.x * p3.y - p2.y * p3.x)) / 6.0;
        if (nn > 0.0) {
            const double3 nh = make_double3(n.x / nn, n.y / nn, n.z / nn);
            const double3 P[3] = {p1, p2, p3};
            const int idx[3] = {ia, ib, ic};
            for (int c = 0; c < 3; c++) {
                const double3 o = P[c], q = P[(c + 1) % 3], s = P[(c + 2) % 3];
                const double3 e1 = make_double3(q.x - o.x, q.y - o.y, q.z - o.z);
                const double3 e2 = make_double3(s.x - o.x, s.y - o.y, s.z - o.z);
                const double cx = e1.y * e2.z - e1.z * e2.y, cy = e1.z * e2.x - e1.x * e2.z,
                             cz = e1.x * e2.y - e1.y * e2.x;
                const double th = atan2(sqrt(cx * cx + cy * cy + cz * cz),
                                        e1.x * e2.x + e1.y * e2.y + e1.z * e2.z);
                double* a = vacc + 4 * (int64_t)idx[c];
                atomicAdd(a + 0, th * nh.x);
                atomicAdd(a + 1, th * nh.y);
                atomicAdd(a + 2, th * nh.z);
                atomicAdd(a + 3, th);
            }
        }
    }
    // block reductions
    for (int o = 16; o > 0; o >>= 1) {
        vol += __shfl_down_sync(0xffffffffu, vol, o);
        smin = fmin(smin, __shfl_down_sync(0xffffffffu, smin, o));
        smax = fmax(smax, __shfl_down_sync(0xffffffffu, smax, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red + 0, vol);
        atomicMin(reinterpret_cast<long long*>(red + 1), ordered_bits(smin));
        atomicMax(reinterpret_cast<long long*>(red + 2), ordered_bits(smax));
        if (bad > 0) atomicAdd(red + 3, bad);
    }
}

// edge_nodes != 0 (quadratic patches): vertices that are no patch's corner
// are edge nodes and carry no pseudonormal (the host checked that every
// vertex is a corner or an edge node)
__global__ void k_vertex_pn(const double* __restrict__ vacc, int64_t nv, double* __restrict__ vpn,
                            double* __restrict__ red, int edge_nodes)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const double A = vacc[4 * i + 3];
    if (A > 0.0) {
        vpn[3 * i] = vacc[4 * i] / A;
        vpn[3 * i + 1] = vacc[4 * i + 1] / A;
        vpn[3 * i + 2] = vacc[4 * i + 2] / A;
    } else {
        vpn[3 * i] = vpn[3 * i + 1] = vpn[3 * i + 2] = 0.0;
        if (!edge_nodes) atomicAdd(red + 4, 1.0);  // unreferenced vertex
    }
}

// Source nodes, triangle-major then rule order:
//   y = P1 + u T_u + v T_v,  nw = w N / (4 pi),  a = 1/(sqrt2 sigma_j).
__global__ void k_sources(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                          const double* __restrict__ tri_n, const double* __restrict__ tri_sigma,
                          int64_t m, const double* __restrict__ rule, int nq,
                          double4_32a* __restrict__ pos, double4_32a* __restrict__ nw)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= m * nq) return;
    const int64_t j = s / nq;
    const int k = (int)(s - j * nq);
    const double u = rule[3 * k], v = rule[3 * k + 1], w = rule[3 * k + 2];
    const int ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
    double y[3];
    for (int c = 0; c < 3; c++) {
        const double p1 = verts[3 * ia + c];
        y[c] = p1 + u * (verts[3 * ib + c] - p1) + v * (verts[3 * ic + c] - p1);
    }
    const double sg = tri_sigma[j];
    const double q = w / (4.0 * kPi);
    pos[s] = make_double4_32a(y[0], y[1], y[2], 1.0 / (sqrt(2.0) * sg));
    nw[s] = make_double4_32a(q * tri_n[3 * j], q * tri_n[3 * j + 1], q * tri_n[3 * j + 2], sqrt(2.0) * sg);
}

// Quadratic patches: the same per-triangle state as k_tri_geometry, with the
// patch's own tangents.  sigma_j = 0.5 sqrt(2 area_j) (or the given one),
// area_j = sum_k w_k |N(u_k, v_k)| over the source rule; the signed volume
// sum_k w_k T . N / 3 by the same rule; each corner adds its vertex angle
// (between the tangents of its two edges there) and its unit normal to the
// vertex sums of eq. mkvertexpn.  tri_n holds N at the patch centroid.
__global__ void k_tri_geometry_quad(const double* __restrict__ verts, const int32_t* __restrict__ tris6,
                                    int64_t m, const double* __restrict__ sigma_in, const double* __restrict__ rule,
                                    int nq, double* __restrict__ tri_n, double* __restrict__ tri_sigma,
                                    double* __restrict__ vacc, double* __restrict__ red)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double vol = 0.0;
    double smin = 1e300, smax = -1e300, bad = 0.0;
    if (j < m) {
        double area = 0.0;
        for (int k = 0; k < nq; k++) {
            double T[3], Tu[3], Tv[3];
            patch_map(verts, nullptr, tris6, j, rule[3 * k], rule[3 * k + 1], T, Tu, Tv);
            const double nx = Tu[1] * Tv[2] - Tu[2] * Tv[1], ny = Tu[2] * Tv[0] - Tu[0] * Tv[2],
                         nz = Tu[0] * Tv[1] - Tu[1] * Tv[0];
            const double nn = sqrt(nx * nx + ny * ny + nz * nz);
            if (!(nn > 0.0)) bad = 1.0;
            area += rule[3 * k + 2] * nn;
            vol += rule[3 * k + 2] * (T[0] * nx + T[1] * ny + T[2] * nz) / 3.0;
        }
        {
            double T[3], Tu[3], Tv[3];
            patch_map(verts, nullptr, tris6, j, 1.0 / 3.0, 1.0 / 3.0, T, Tu, Tv);
            tri_n[3 * j] = Tu[1] * Tv[2] - Tu[2] * Tv[1];
            tri_n[3 * j + 1] = Tu[2] * Tv[0] - Tu[0] * Tv[2];
            tri_n[3 * j + 2] = Tu[0] * Tv[1] - Tu[1] * Tv[0];
        }
        const double sg = sigma_in ? sigma_in[j] : 0.5 * sqrt(2.0 * area);
        tri_sigma[j] = sg;
        smin = sg;
        smax = sg;
        if (!(sg > 0.0)) bad = 1.0;
        const double cu[3] = {0.0, 1.0, 0.0}, cv[3] = {0.0, 0.0, 1.0};
        for (int c = 0; c < 3; c++) {
            double T[3], Tu[3], Tv[3], e1[3], e2[3];
            patch_map(verts, nullptr, tris6, j, cu[c], cv[c], T, Tu, Tv);
            for (int k = 0; k < 3; k++) {
                // the two edges leaving the corner: (u, v) along (1,0),(0,1) at P1;
                // (-1,1),(-1,0) at P2; (0,-1),(1,-1) at P3
                e1[k] = c == 0 ? Tu[k] : (c == 1 ? Tv[k] - Tu[k] : -Tv[k]);
                e2[k] = c == 0 ? Tv[k] : (c == 1 ? -Tu[k] : Tu[k] - Tv[k]);
            }
            const double nx = Tu[1] * Tv[2] - Tu[2] * Tv[1], ny = Tu[2] * Tv[0] - Tu[0] * Tv[2],
                         nz = Tu[0] * Tv[1] - Tu[1] * Tv[0];
            const double nn = sqrt(nx * nx + ny * ny + nz * nz);
            if (!(nn > 0.0)) {
                bad = 1.0;
                continue;
            }
            const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                         cz = e1[0] * e2[1] - e1[1] * e2[0];
            const double th = atan2(sqrt(cx * cx + cy * cy + cz * cz), e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2]);
            double* a = vacc + 4 * (int64_t)tris6[6 * j + c];
            atomicAdd(a + 0, th * nx / nn);
            atomicAdd(a + 1, th * ny / nn);
            atomicAdd(a + 2, th * nz / nn);
            atomicAdd(a + 3, th);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        vol += __shfl_down_sync(0xffffffffu, vol, o);
        smin = fmin(smin, __shfl_down_sync(0xffffffffu, smin, o));
        smax = fmax(smax, __shfl_down_sync(0xffffffffu, smax, o));
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(red + 0, vol);
        atomicMin(reinterpret_cast<long long*>(red + 1), ordered_bits(smin));
        atomicMax(reinterpret_cast<long long*>(red + 2), ordered_bits(smax));
        if (bad > 0) atomicAdd(red + 3, bad);
    }
}

// Source nodes on quadratic patches: y = T(u, v), nw = w N(u, v) / (4 pi)
// (the area element is in |N|), a = 1/(sqrt2 sigma_j).
__global__ void k_sources_quad(const double* __restrict__ verts, const int32_t* __restrict__ tris6,
                               const double* __restrict__ tri_sigma, int64_t m, const double* __restrict__ rule,
                               int nq, double4_32a* __restrict__ pos, double4_32a* __restrict__ nw)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= m * nq) return;
    const int64_t j = s / nq;
    const int k = (int)(s - j * nq);
    double T[3], Tu[3], Tv[3];
    patch_map(verts, nullptr, tris6, j, rule[3 * k], rule[3 * k + 1], T, Tu, Tv);
    const double sg = tri_sigma[j];
    const double q = rule[3 * k + 2] / (4.0 * kPi);
    pos[s] = make_double4_32a(T[0], T[1], T[2], 1.0 / (sqrt(2.0) * sg));
    nw[s] = make_double4_32a(q * (Tu[1] * Tv[2] - Tu[2] * Tv[1]), q * (Tu[2] * Tv[0] - Tu[0] * Tv[2]),
                             q * (Tu[0] * Tv[1] - Tu[1] * Tv[0]), sqrt(2.0) * sg);
}

// ordered(+DBL_MAX) for the minima, ordered(-DBL_MAX) for the maxima
__global__ void k_bbox_init(long long* bb)
{
    if (threadIdx.x < 3) bb[threadIdx.x] = 0x7fefffffffffffffLL;
    else if (threadIdx.x < 6) bb[threadIdx.x] = (long long)0x8010000000000000ULL;
}

// red[0]=volume, [1]=ordered(+DBL_MAX) (sigma min), [2]=ordered(-DBL_MAX)
// (sigma max), [3..7]=0
__global__ void k_red_init(double* red)
{
    long long* r = reinterpret_cast<long long*>(red);
    if (threadIdx.x < 8) r[threadIdx.x] = 0;
    if (threadIdx.x == 1) r[1] = 0x7fefffffffffffffLL;
    if (threadIdx.x == 2) r[2] = (long long)0x8010000000000000ULL;
}

// Bounding box of n points (AoS with `stride` doubles per point, first three
// are x, y, z) into bb[0..6) as ordered bits: min x,y,z then max x,y,z.
__global__ void k_bbox(const double* __restrict__ p, int stride, int n, long long* __restrict__ bb)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        for (int c = 0; c < 3; c++) {
            const double v = p[(int64_t)i * stride + c];
            lo[c] = fmin(lo[c], v);
            hi[c] = fmax(hi[c], v);
        }
    }
    for (int c = 0; c < 3; c++) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_down_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_down_sync(0xffffffffu, hi[c], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; c++) {
            atomicMin(bb + c, ordered_bits(lo[c]));
            atomicMax(bb + 3 + c, ordered_bits(hi[c]));
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// 30-bit Morton key of each point in the cube spanned by the bounding box.
__global__ void k_morton(const double* __restrict__ p, int stride, int n,
                         const long long* __restrict__ bb, uint32_t* __restrict__ keys,
                         uint32_t* __restrict__ vals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo[3], ext = 0.0;
    for (int c = 0; c < 3; c++) {
        lo[c] = from_ordered(bb[c]);
        ext = fmax(ext, from_ordered(bb[3 + c]) - lo[c]);
    }
    const double sc = ext > 0.0 ? 1023.0 / ext : 0.0;
    uint32_t q[3];
    for (int c = 0; c < 3; c++) {
        double t = (p[(int64_t)i * stride + c] - lo[c]) * sc;
        t = fmin(fmax(t, 0.0), 1023.0);
        q[c] = (uint32_t)t;
    }
    keys[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    vals[i] = (uint32_t)i;
}

__global__ void k_gather_sources(const double4_32a* __restrict__ pin, const double4_32a* __restrict__ nin,
                                 const uint32_t* __restrict__ perm, int n,
                                 double4_32a* __restrict__ pout, double4_32a* __restrict__ nout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = perm[i];
    pout[i] = pin[k];
    nout[i] = nin[k];
}

// Segments of the Morton-ordered sources: a new one starts where two
// consecutive sources lie farther apart than kSegJump times the larger of
// their sigmas.  Tiles never straddle a segment boundary, so a tile does not
// span a jump of the curve (a tile of sources from two far parts of the
// surface would be near too many targets, and its sources' float-pair
// offsets from the tile's centre would lose absolute precision).
constexpr double kSegJump = 8.0;
__global__ void k_seg_flags(const double4_32a* __restrict__ p, int n, uint32_t* __restrict__ flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t f = 1;
    if (i > 0) {
        const double4_32a a = p[i], b = p[i - 1];
        const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        // a = 1/(sqrt2 sigma): the larger sigma has the smaller a
        const double s = 1.0 / (1.41421356237309505 * fmin(a.w, b.w));
        f = dx * dx + dy * dy + dz * dz > kSegJump * kSegJump * s * s ? 1u : 0u;
    }
    flags[i] = f;
}
// First source of each segment (sid: exclusive scan of the flags).
__global__ void k_seg_starts(const uint32_t* __restrict__ flags, const uint32_t* __restrict__ sid, int n,
                             uint32_t* __restrict__ starts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flags[i]) starts[sid[i]] = (uint32_t)i;
}
// Tiles of each segment.
__global__ void k_seg_tiles(const uint32_t* __restrict__ starts, int nseg, int n, uint32_t* __restrict__ ntile)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const uint32_t len = (s + 1 < nseg ? starts[s + 1] : (uint32_t)n) - starts[s];
    ntile[s] = (len + kTile - 1) / kTile;
}
// Each source to its slot: tile tbase[segment] + local / kTile, slot local %
// kTile; the first source of a tile writes the tile's count.
__global__ void k_seg_scatter(const double4_32a* __restrict__ pin, const double4_32a* __restrict__ nin,
                              const uint32_t* __restrict__ flags, const uint32_t* __restrict__ sid,
                              const uint32_t* __restrict__ starts, const uint32_t* __restrict__ tbase, int nseg,
                              int n, double4_32a* __restrict__ pout, double4_32a* __restrict__ nout,
                              int* __restrict__ tcnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int seg = (int)(sid[i] + flags[i]) - 1;
    const uint32_t local = (uint32_t)i - starts[seg];
    const uint32_t tile = tbase[seg] + local / kTile, slot = local % kTile;
    const int64_t dst = (int64_t)tile * kTile + slot;
    pout[dst] = pin[i];
    nout[dst] = nin[i];
    if (slot == 0) {
        const uint32_t len = (seg + 1 < nseg ? starts[seg + 1] : (uint32_t)n) - starts[seg];
        tcnt[tile] = (int)min((uint32_t)kTile, len - local);
    }
}

// One block per tile: bounding box (outward-rounded to FP32), sigma_max,
// centre (split in two floats) and the FP32 tile-local copies of its nodes.
// Slots past the tile's count become padding: a copy of the tile's first
// node with zero weight (every kernel stops at the count; the tree's P2M and
// node frames read whole tiles, where zero weight adds nothing).
__global__ void __launch_bounds__(kTile) k_tile_meta(
    double4_32a* __restrict__ pos, double4_32a* __restrict__ nw, const int* __restrict__ tcnt,
    float4* __restrict__ s32p, float4* __restrict__ s32n, float4* __restrict__ s32l,
    float4* __restrict__ s32nl, float4* __restrict__ tlo,
    float4* __restrict__ thi, float4* __restrict__ tchi, float4* __restrict__ tclo)
{
    __shared__ double red[7][kTile / 32];
    const int t = blockIdx.x;
    const int i = t * kTile + threadIdx.x;
    const int tc = tcnt[t];
    const bool ok = (int)threadIdx.x < tc;
    double4_32a p = ok ? pos[i] : make_double4_32a(0, 0, 0, 0);
    double lo[3], hi[3], sg;
    if (ok) {
        lo[0] = hi[0] = p.x;
        lo[1] = hi[1] = p.y;
        lo[2] = hi[2] = p.z;
        sg = 1.0 / (sqrt(2.0) * p.w);
    } else {
        lo[0] = lo[1] = lo[2] = 1e300;
        hi[0] = hi[1] = hi[2] = -1e300;
        sg = 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int c = 0; c < 3; c++) {
            lo[c] = fmin(lo[c], __shfl_down_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_down_sync(0xffffffffu, hi[c], o));
        }
        sg = fmax(sg, __shfl_down_sync(0xffffffffu, sg, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; c++) {
            red[c][w] = lo[c];
            red[3 + c][w] = hi[c];
        }
        red[6][w] = sg;
    }
    __syncthreads();
    double L[3], Hh[3], S = 0.0;
    for (int c = 0; c < 3; c++) {
        L[c] = red[c][0];
        Hh[c] = red[3 + c][0];
        for (int k = 1; k < kTile / 32; k++) {
            L[c] = fmin(L[c], red[c][k]);
            Hh[c] = fmax(Hh[c], red[3 + c][k]);
        }
    }
    for (int k = 0; k < kTile / 32; k++) S = fmax(S, red[6][k]);
    // the centre is the float pair (ch, cl) itself, exactly: sources are
    // stored relative to it and the kernels rebuild it from the two floats
    // (a centre off by the pair's rounding, ~2^-48 |C|, shifts every source
    // of the tile alike, ~1e-13 of Phi through grad Phi ~ 1/sigma)
    double C[3];
    float ch[3], cl[3];
    for (int c = 0; c < 3; c++) {
        const double mid = 0.5 * (L[c] + Hh[c]);
        ch[c] = __double2float_rn(mid);
        cl[c] = __double2float_rn(mid - (double)ch[c]);
        C[c] = (double)ch[c] + (double)cl[c];
    }
    if (threadIdx.x == 0) {
        tlo[t] = make_float4(__double2float_rd(L[0]), __double2float_rd(L[1]), __double2float_rd(L[2]),
                             __double2float_ru(S));
        thi[t] = make_float4(__double2float_ru(Hh[0]), __double2float_ru(Hh[1]), __double2float_ru(Hh[2]),
                             (float)tc);
        tchi[t] = make_float4(ch[0], ch[1], ch[2], 0.0f);
        tclo[t] = make_float4(cl[0], cl[1], cl[2], 0.0f);
    }
    if (ok) {
        const double4_32a q = nw[i];
        const double lx = p.x - C[0], ly = p.y - C[1], lz = p.z - C[2];
        const float hx = __double2float_rn(lx), hy = __double2float_rn(ly), hz = __double2float_rn(lz);
        const float ah = __double2float_rn(p.w);
        s32p[i] = make_float4(hx, hy, hz, ah);
        s32l[i] = make_float4(__double2float_rn(lx - (double)hx), __double2float_rn(ly - (double)hy),
                              __double2float_rn(lz - (double)hz), __double2float_rn(p.w - (double)ah));
        const float nx = __double2float_rn(q.x), ny = __double2float_rn(q.y), nz = __double2float_rn(q.z);
        s32n[i] = make_float4(nx, ny, nz, __double2float_rn(q.w));
        s32nl[i] = make_float4(__double2float_rn(q.x - (double)nx), __double2float_rn(q.y - (double)ny),
                               __double2float_rn(q.z - (double)nz), 0.0f);
    } else {
        // padding slot: the tile's first node with zero weight
        const double4_32a f = pos[(int64_t)t * kTile];
        pos[i] = f;
        nw[i] = make_double4_32a(0, 0, 0, 0);
        const double lx = f.x - C[0], ly = f.y - C[1], lz = f.z - C[2];
        const float hx = __double2float_rn(lx), hy = __double2float_rn(ly), hz = __double2float_rn(lz);
        const float ah = __double2float_rn(f.w);
        s32p[i] = make_float4(hx, hy, hz, ah);
        s32l[i] = make_float4(__double2float_rn(lx - (double)hx), __double2float_rn(ly - (double)hy),
                              __double2float_rn(lz - (double)hz), __double2float_rn(f.w - (double)ah));
        s32n[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s32nl[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
}

// Chart nodes (Sec. 3.2): x0 = T^j(u_i, v_i), H = H^j(u_i, v_i) (eq. mkpseudovec),
// sloc = sigma_j.  Triangle-major, then rule order.  x0, hdir AoS [n][3].
__global__ void k_chart_nodes(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                              const int32_t* __restrict__ tris6, const double* __restrict__ vpn,
                              const double* __restrict__ tri_sigma, int64_t m, const double* __restrict__ rule,
                              int np, double* __restrict__ x0, double* __restrict__ hdir,
                              double* __restrict__ sloc)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= m * np) return;
    const int64_t j = s / np;
    const int k = (int)(s - j * np);
    const double u = rule[3 * k], v = rule[3 * k + 1];
    const int ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
    double T[3], Tu[3], Tv[3];
    patch_map(verts, tris, tris6, j, u, v, T, Tu, Tv);
    for (int c = 0; c < 3; c++) {
        const double h1 = vpn[3 * ia + c];
        x0[3 * s + c] = T[c];
        hdir[3 * s + c] = h1 + u * (vpn[3 * ib + c] - h1) + v * (vpn[3 * ic + c] - h1);
    }
    sloc[s] = tri_sigma[j];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Chart nodes given explicitly: node s in triangle tri[s] at parent
// coordinates (uvw[3s], uvw[3s+1]) (refined charts keep their parent's map,
// Sec. 3.4).
__global__ void k_chart_nodes_at(const double* __restrict__ verts, const int32_t* __restrict__ tris,
                                 const int32_t* __restrict__ tris6, const double* __restrict__ vpn,
                                 const double* __restrict__ tri_sigma, int64_t n, const int32_t* __restrict__ tri,
                                 const double* __restrict__ uvw, double* __restrict__ x0,
                                 double* __restrict__ hdir, double* __restrict__ sloc)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t j = tri[s];
    const double u = uvw[3 * s], v = uvw[3 * s + 1];
    const int ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
    double T[3], Tu[3], Tv[3];
    patch_map(verts, tris, tris6, j, u, v, T, Tu, Tv);
    for (int c = 0; c < 3; c++) {
        const double h1 = vpn[3 * ia + c];
        x0[3 * s + c] = T[c];
        hdir[3 * s + c] = h1 + u * (vpn[3 * ib + c] - h1) + v * (vpn[3 * ic + c] - h1);
    }
    sloc[s] = tri_sigma[j];
}

}  // namespace

int chart_nodes_at(Ctx* ctx, const Mesh* me, int64_t n, const int32_t* tri, const double* uvw, double* x0,
                   double* hdir, double* sloc, cudaStream_t st)
{
    if (n <= 0) return LSM_OK;
    k_chart_nodes_at<<<blocks_for(n, 256), 256, 0, st>>>(me->verts, me->tris, me->tris6, me->vpn, me->tri_sigma, n,
                                                         tri, uvw, x0, hdir, sloc);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

// Morton permutation of n points (AoS, `stride` doubles per point).
int morton_order_points(Ctx* ctx, const double* pts, int stride, int n, uint32_t* perm,
                        cudaStream_t st)
{
    if (n <= 0) return LSM_OK;
    Scratch s(st);
    long long* bb;
    uint32_t* keys;
    LSM_CUDA_TRY(ctx, s.get(&bb, 6));
    LSM_CUDA_TRY(ctx, s.get(&keys, n));
    k_bbox_init<<<1, 32, 0, st>>>(bb);
    LSM_LAUNCHED(ctx);
    const int nbb = (int)std::min<int64_t>(blocks_for(n, 256), 4 * (int64_t)ctx->num_sms);
    k_bbox<<<nbb, 256, 0, st>>>(pts, stride, n, bb);
    LSM_LAUNCHED(ctx);
    k_morton<<<blocks_for(n, 256), 256, 0, st>>>(pts, stride, n, bb, keys, perm);
    LSM_LAUNCHED(ctx);
    return radix_sort_pairs(ctx, keys, perm, n, 30, st);
}

int build_mesh_device(Ctx* ctx, Mesh* me, const double* sigma_in_dev, const double* rule_dev,
                      double* host_red, cudaStream_t st)
{
    Scratch s(st);
    double *vacc, *red;
    LSM_CUDA_TRY(ctx, s.get(&vacc, 4 * me->nv));
    LSM_CUDA_TRY(ctx, s.get(&red, 8));
    LSM_CUDA_TRY(ctx, cudaMemsetAsync(vacc, 0, sizeof(double) * 4 * me->nv, st));
    k_red_init<<<1, 32, 0, st>>>(red);
    LSM_LAUNCHED(ctx);
    if (me->tris6)
        k_tri_geometry_quad<<<blocks_for(me->m, 256), 256, 0, st>>>(me->verts, me->tris6, me->m, sigma_in_dev,
                                                                  rule_dev, me->nq, me->tri_n, me->tri_sigma, vacc,
                                                                  red);
    else
        k_tri_geometry<<<blocks_for(me->m, 256), 256, 0, st>>>(me->verts, me->tris, me->m, sigma_in_dev,
                                                             me->tri_n, me->tri_sigma, vacc, red);
    LSM_LAUNCHED(ctx);
    k_vertex_pn<<<blocks_for(me->nv, 256), 256, 0, st>>>(vacc, me->nv, me->vpn, red, me->tris6 ? 1 : 0);
    LSM_LAUNCHED(ctx);
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(host_red, red, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int k = 1; k <= 2; k++) {
        long long b;
        memcpy(&b, &host_red[k], 8);
        if (b < 0) b ^= 0x7fffffffffffffffLL;
        memcpy(&host_red[k], &b, 8);
    }
    if (host_red[3] > 0 || host_red[4] > 0 || !(host_red[0] > 0)) return LSM_E_MESH;
    me->sigma_min = host_red[1];
    me->sigma_max = host_red[2];

    // source nodes, unsorted, then Morton order
    const int ns = (int)me->ns;
    double4_32a *p0, *n0;
    uint32_t* perm;
    LSM_CUDA_TRY(ctx, s.get(&p0, ns));
    LSM_CUDA_TRY(ctx, s.get(&n0, ns));
    LSM_CUDA_TRY(ctx, s.get(&perm, ns));
    if (me->tris6)
        k_sources_quad<<<blocks_for(ns, 256), 256, 0, st>>>(me->verts, me->tris6, me->tri_sigma, me->m, rule_dev,
                                                           me->nq, p0, n0);
    else
        k_sources<<<blocks_for(ns, 256), 256, 0, st>>>(me->verts, me->tris, me->tri_n, me->tri_sigma, me->m,
                                                      rule_dev, me->nq, p0, n0);
    LSM_LAUNCHED(ctx);
    int rc = morton_order_points(ctx, reinterpret_cast<const double*>(p0), 4, ns, perm, st);
    if (rc != LSM_OK) return rc;
    double4_32a *p1, *n1;
    LSM_CUDA_TRY(ctx, s.get(&p1, ns));
    LSM_CUDA_TRY(ctx, s.get(&n1, ns));
    k_gather_sources<<<blocks_for(ns, 256), 256, 0, st>>>(p0, n0, perm, ns, p1, n1);
    LSM_LAUNCHED(ctx);

    // segments at jumps of the Morton curve, then tiles within segments
    uint32_t *flags, *sid, *cnt2;
    LSM_CUDA_TRY(ctx, s.get(&flags, ns));
    LSM_CUDA_TRY(ctx, s.get(&sid, ns));
    LSM_CUDA_TRY(ctx, s.get(&cnt2, 2));
    k_seg_flags<<<blocks_for(ns, 256), 256, 0, st>>>(p1, ns, flags);
    LSM_LAUNCHED(ctx);
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(sid, flags, sizeof(uint32_t) * ns, cudaMemcpyDeviceToDevice, st));
    rc = scan_exclusive(ctx, sid, ns, cnt2, st);
    if (rc != LSM_OK) return rc;
    uint32_t nseg = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&nseg, cnt2, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    uint32_t *starts, *tbase;
    LSM_CUDA_TRY(ctx, s.get(&starts, nseg));
    LSM_CUDA_TRY(ctx, s.get(&tbase, nseg));
    k_seg_starts<<<blocks_for(ns, 256), 256, 0, st>>>(flags, sid, ns, starts);
    LSM_LAUNCHED(ctx);
    k_seg_tiles<<<blocks_for(nseg, 256), 256, 0, st>>>(starts, (int)nseg, ns, tbase);
    LSM_LAUNCHED(ctx);
    rc = scan_exclusive(ctx, tbase, nseg, cnt2 + 1, st);
    if (rc != LSM_OK) return rc;
    uint32_t ntiles = 0;
    LSM_CUDA_TRY(ctx, cudaMemcpyAsync(&ntiles, cnt2 + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if ((int64_t)ntiles * kTile >= ((int64_t)1 << 31)) {
        ctx->err = "mesh_upload: too many source tiles";
        return LSM_E_INVALID_ARG;
    }
    me->ntiles = ntiles;
    const size_t nsl = (size_t)ntiles * kTile, ntl = ntiles;
    auto alloc = [&](auto** p, size_t count) -> bool {
        using T = std::remove_pointer_t<std::remove_reference_t<decltype(*p)>>;
        if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) return false;
        me->bytes += count * sizeof(T);
        return true;
    };
    if (!alloc(&me->s64_pos, nsl) || !alloc(&me->s64_nw, nsl) || !alloc(&me->s32_pos, nsl) ||
        !alloc(&me->s32_nw, nsl) || !alloc(&me->s32_lo, nsl) || !alloc(&me->s32_nwlo, nsl) ||
        !alloc(&me->tile_lo, ntl) || !alloc(&me->tile_hi, ntl) || !alloc(&me->tile_chi, ntl) ||
        !alloc(&me->tile_clo, ntl)) {
        cudaGetLastError();
        ctx->err = "mesh_upload: out of device memory";
        return LSM_E_OOM;
    }
    int* tcnt;
    LSM_CUDA_TRY(ctx, s.get(&tcnt, ntl));
    k_seg_scatter<<<blocks_for(ns, 256), 256, 0, st>>>(p1, n1, flags, sid, starts, tbase, (int)nseg, ns,
                                                      me->s64_pos, me->s64_nw, tcnt);
    LSM_LAUNCHED(ctx);
    k_tile_meta<<<(unsigned)ntiles, kTile, 0, st>>>(me->s64_pos, me->s64_nw, tcnt, me->s32_pos, me->s32_nw,
                                                    me->s32_lo, me->s32_nwlo, me->tile_lo, me->tile_hi,
                                                    me->tile_chi, me->tile_clo);
    LSM_LAUNCHED(ctx);
    LSM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return LSM_OK;
}

int chart_nodes_init(Ctx* ctx, const Mesh* me, const double* chart_rule_dev, int np, double* x0,
                     double* hdir, double* sloc, cudaStream_t st)
{
    const int64_t n = me->m * np;
    k_chart_nodes<<<blocks_for(n, 256), 256, 0, st>>>(me->verts, me->tris, me->tris6, me->vpn, me->tri_sigma, me->m,
                                                    chart_rule_dev, np, x0, hdir, sloc);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

int chart_nodes_raw(Ctx* ctx, const double* verts, const int32_t* tris, const double* vpn, const double* tri_sigma,
                    int64_t m, const double* chart_rule_dev, int np, double* x0, double* hdir, double* sloc,
                    cudaStream_t st)
{
    const int64_t n = m * np;
    k_chart_nodes<<<blocks_for(n, 256), 256, 0, st>>>(verts, tris, nullptr, vpn, tri_sigma, m, chart_rule_dev, np, x0,
                                                    hdir, sloc);
    LSM_LAUNCHED(ctx);
    return LSM_OK;
}

}  // namespace lsm
