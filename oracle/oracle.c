/*
 * oracle.c -- plain FP64 CPU oracle for the smoothed level-set function.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this code.  It shares no source,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded input arrays of the synth/ package.
 *
 * Everything here is the plain definition, written for a reader to check
 * against the paper by eye:
 *   - triangle chart T^j(u,v) = P1 + u (P2-P1) + v (P3-P1), T_u, T_v,
 *     N = T_u x T_v                                     (Sec. 3, eq. tparam)
 *   - vertex pseudonormal H(P) = sum(theta * N_hat) / sum(theta), the
 *     angle-weighted mean, not renormalised                 (eq. mkvertexpn)
 *   - pseudonormal field H^j(u,v) by linear interpolation   (eq. mkpseudovec)
 *   - the discrete boundary sum Phi(x) = sum_{j,k} w_k |N_j| psi(x, T^j(u_k,v_k))
 *                                                 (eq. discrete_int, kerpsi)
 *   - grad Phi by differentiating psi in x                   (eq. gradPhi, with
 *     the sign of the second term corrected; see below)
 *   - Newton on h: h <- h - (Phi(T + hH) - 1/2) / (H . grad Phi),  h0 = 0
 *                                                    (eq. newton, newtoneq)
 *   - local coordinates x_u, x_v and da of the charts (eq. u_vector,
 *     U_vector_2, v_vector, v_vector_2, da) and the Gauss flux error eps0
 *     (Sec. 5)
 *   - refined charts: nodes of the 1 -> 4 midpoint children of a triangle in
 *     the parent's chart map (Sec. 3.4)
 *   - the Hessian of Phi and the charts' second derivatives and curvatures
 *     (Sec. 3.3, eq. uu_vector, uu_vector_aux1, uu_vector_aux2)
 *   - the target-dependent width sigma(x), a Gaussian-weighted mean of
 *     sigma_j = D_j / lambda over the triangle centroids (eq. sigma2), and
 *     Phi, grad Phi with it (eq. gradPhi's third term, sign corrected)
 *
 * Notation.  r = y - x (source node minus target), rho = |r|,
 * a = 1/(sqrt(2) sigma), u = rho a,
 * g(u) = erf(u) - (2u/sqrt(pi)) exp(-u^2),  f(rho) = g(u) / (4 pi rho^3),
 * so psi * da = (nw . r) f(rho) with nw = w |N| N_hat  (eq. kerpsi).
 * Gradient in x: -( nw f + (nw . r) F r ) with F = f'(rho)/rho.  The paper's
 * eq. gradPhi prints the second term with a plus sign; its sigma -> 0 limit
 * must be the gradient of the Laplace double layer, -nw/(4 pi rho^3) +
 * 3 (nw.r) r/(4 pi rho^5), which the minus sign gives.  Its F is the same
 * function as ours: F = [sqrt(2/pi)(rho/sigma)^3 e^{-u^2} - 3 g] / (4 pi rho^5).
 *
 * For small u both f and F are written as power series in u (the paper's
 * eq. kerpsi_asymp gives the first five terms of f's series; eq.
 * kerpsi_asymp2 drops the (nw.r) F r term, which we keep).  The series is
 * used for u < 0.5 and summed until the next term is below 1e-18 of the sum;
 * the closed forms with libm erf/exp are used otherwise.
 *
 * sigma belongs to the source triangle (one sigma_j per skeleton triangle),
 * so there is no grad-sigma term.  With a constant sigma this is exactly the
 * paper's Phi (eq. basemodelg).
 *
 * Parity: every function here is pinned by the not-gpu tests in
 * tests/test_oracle_pins.py (closed forms, limits, finite differences,
 * brute-force volume quadrature), except the positions returned by the
 * Newton solve on meshes other than a flat face: those are checked only by
 * Phi(x) = 1/2 re-evaluated, and are marked "parity unpinned" there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* 1-D Gauss-Legendre rule on [0,1] (n points), by Newton's method on the
 * three-term recurrence of the Legendre polynomials.  Nodes ascending. */
int or_gauss_legendre01(int n, double* x, double* w)
{
    if (n < 1) return -1;
    for (int i = 0; i < n; i++) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 200; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        /* z descends with i; map to [0,1] ascending */
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Rule on the standard simplex T0 = {u,v >= 0, u+v <= 1}:
 * the simplex is split `subdiv` times into four midpoint children
 * (Sec. 4.5), and each (sub)triangle (A,B,C) carries the Duffy-collapsed
 * n x n Gauss-Legendre rule
 *     p = A + xi (1-eta) (B-A) + xi eta (C-A),
 *     weight = w_xi w_eta xi |det(B-A, C-A)|,
 * collapsed at A.  Child order of (A,B,C) with edge midpoints
 * mAB, mBC, mCA: (A,mAB,mCA), (mAB,B,mBC), (mCA,mBC,C), (mBC,mCA,mAB).
 * Node order: subtriangle, then xi, then eta.  Sum of weights = 1/2.
 * Returns the node count n*n*4^subdiv. */
int or_simplex_rule(int n, int subdiv, double* u, double* v, double* w)
{
    if (n < 1 || subdiv < 0 || subdiv > 6) return -1;
    int nsub = 1;
    for (int s = 0; s < subdiv; s++) nsub *= 4;
    double* tri = (double*)malloc(sizeof(double) * 6 * nsub);
    double* nxt = (double*)malloc(sizeof(double) * 6 * nsub);
    tri[0] = 0; tri[1] = 0; tri[2] = 1; tri[3] = 0; tri[4] = 0; tri[5] = 1;
    int cnt = 1;
    for (int s = 0; s < subdiv; s++) {
        for (int t = 0; t < cnt; t++) {
            double ax = tri[6*t+0], ay = tri[6*t+1];
            double bx = tri[6*t+2], by = tri[6*t+3];
            double cx = tri[6*t+4], cy = tri[6*t+5];
            double abx = 0.5*(ax+bx), aby = 0.5*(ay+by);
            double bcx = 0.5*(bx+cx), bcy = 0.5*(by+cy);
            double cax = 0.5*(cx+ax), cay = 0.5*(cy+ay);
            double kids[4][6] = {
                {ax, ay, abx, aby, cax, cay},
                {abx, aby, bx, by, bcx, bcy},
                {cax, cay, bcx, bcy, cx, cy},
                {bcx, bcy, cax, cay, abx, aby},
            };
            for (int c = 0; c < 4; c++)
                memcpy(nxt + 6*(4*t + c), kids[c], sizeof(double) * 6);
        }
        cnt *= 4;
        double* tmp = tri; tri = nxt; nxt = tmp;
    }
    double* gx = (double*)malloc(sizeof(double) * n);
    double* gw = (double*)malloc(sizeof(double) * n);
    or_gauss_legendre01(n, gx, gw);
    int m = 0;
    for (int t = 0; t < cnt; t++) {
        double ax = tri[6*t+0], ay = tri[6*t+1];
        double e1x = tri[6*t+2] - ax, e1y = tri[6*t+3] - ay;
        double e2x = tri[6*t+4] - ax, e2y = tri[6*t+5] - ay;
        double jac = fabs(e1x * e2y - e1y * e2x);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                double s = gx[i] * (1.0 - gx[j]);
                double q = gx[i] * gx[j];
                u[m] = ax + s * e1x + q * e2x;
                v[m] = ay + s * e1y + q * e2y;
                w[m] = gw[i] * gw[j] * gx[i] * jac;
                m++;
            }
    }
    free(gx); free(gw); free(tri); free(nxt);
    return m;
}

/* ------------------------------------------------------------------ */
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1]*b[2] - a[2]*b[1];
    c[1] = a[2]*b[0] - a[0]*b[2];
    c[2] = a[0]*b[1] - a[1]*b[0];
}
static double dot3(const double* a, const double* b)
{
    return a[0]*b[0] + a[1]*b[1] + a[2]*b[2];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* interior angle at vertex p between edges to q and s */
static double angle_at(const double* p, const double* q, const double* s)
{
    double a[3] = {q[0]-p[0], q[1]-p[1], q[2]-p[2]};
    double b[3] = {s[0]-p[0], s[1]-p[1], s[2]-p[2]};
    double c[3];
    cross3(a, b, c);
    return atan2(norm3(c), dot3(a, b));
}

/* Per-triangle geometry (eq. tparam) and vertex pseudonormals
 * (eq. mkvertexpn).
 *   verts [nv][3], tris [m][3] (0-based, counter-clockwise seen from outside)
 *   sigma_in [m] or NULL -> sigma_j = 0.5 sqrt(2 area_j)
 * Outputs: tu,tv,nrm [m][3] (nrm = T_u x T_v), sigma [m], vpn [nv][3].
 * Returns 0, or -1 when a vertex has zero total angle. */
int or_geometry(int64_t nv, const double* verts, int64_t m, const int32_t* tris,
                const double* sigma_in, double* tu, double* tv, double* nrm,
                double* sigma, double* vpn)
{
    double* asum = (double*)calloc((size_t)nv, sizeof(double));
    memset(vpn, 0, sizeof(double) * 3 * (size_t)nv);
    for (int64_t j = 0; j < m; j++) {
        const double* p1 = verts + 3 * (int64_t)tris[3*j+0];
        const double* p2 = verts + 3 * (int64_t)tris[3*j+1];
        const double* p3 = verts + 3 * (int64_t)tris[3*j+2];
        double a[3], b[3], n[3];
        for (int k = 0; k < 3; k++) { a[k] = p2[k] - p1[k]; b[k] = p3[k] - p1[k]; }
        cross3(a, b, n);
        double nn = norm3(n);
        for (int k = 0; k < 3; k++) { tu[3*j+k] = a[k]; tv[3*j+k] = b[k]; nrm[3*j+k] = n[k]; }
        sigma[j] = sigma_in ? sigma_in[j] : 0.5 * sqrt(2.0 * 0.5 * nn);
        double th[3] = { angle_at(p1, p2, p3), angle_at(p2, p3, p1), angle_at(p3, p1, p2) };
        for (int c = 0; c < 3; c++) {
            int64_t vi = tris[3*j+c];
            asum[vi] += th[c];
            for (int k = 0; k < 3; k++) vpn[3*vi+k] += th[c] * n[k] / nn;
        }
    }
    int bad = 0;
    for (int64_t i = 0; i < nv; i++) {
        if (asum[i] > 0) {
            for (int k = 0; k < 3; k++) vpn[3*i+k] /= asum[i];
        } else {
            bad = 1;
        }
    }
    free(asum);
    return bad ? -1 : 0;
}

/* Source nodes of the discrete sum (eq. discrete_int):
 * y_jk = T^j(u_k, v_k), nw_jk = w_k |N_j| N_hat_j = w_k N_j, sig_jk = sigma_j.
 * Node order: triangle-major, then rule order.  Outputs [m*nq][3], [m*nq]. */
void or_sources(int64_t nv, const double* verts, int64_t m, const int32_t* tris,
                const double* nrm, const double* sigma, int nq,
                const double* ru, const double* rv, const double* rw,
                double* y, double* nw, double* sig)
{
    (void)nv;
    for (int64_t j = 0; j < m; j++) {
        const double* p1 = verts + 3 * (int64_t)tris[3*j+0];
        const double* p2 = verts + 3 * (int64_t)tris[3*j+1];
        const double* p3 = verts + 3 * (int64_t)tris[3*j+2];
        for (int k = 0; k < nq; k++) {
            int64_t s = j * nq + k;
            for (int c = 0; c < 3; c++) {
                y[3*s+c] = p1[c] + ru[k] * (p2[c] - p1[c]) + rv[k] * (p3[c] - p1[c]);
                nw[3*s+c] = rw[k] * nrm[3*j+c];
            }
            sig[s] = sigma[j];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Radial factors of the pair kernel at rho = u / a, a = 1/(sqrt2 sigma):
 *   f = g(u) / (4 pi rho^3),      F = f'(rho) / rho.
 * Series form: with h(u) = g(u)/u^3 = (2/sqrt pi) sum_{k>=1} c_k u^{2k-2},
 * c_k = (-1)^{k+1} 2k / (k! (2k+1)),
 *   f = h(u) a^3 / (4 pi),   F = (h'(u)/u) a^5 / (4 pi),
 *   h'(u)/u = (2/sqrt pi) sum_{k>=2} c_k (2k-2) u^{2k-4}. */
void or_radial(double rho, double sig, double* f_out, double* F_out)
{
    const double a = 1.0 / (sqrt(2.0) * sig);
    const double u = rho * a;
    const double tsp = 2.0 / sqrt(OR_PI);
    if (u < 0.5) {
        double h = 0.0, hp = 0.0;
        double fact = 1.0;      /* k! */
        double upow = 1.0;      /* u^{2k-2} */
        double upow2 = 1.0;     /* u^{2k-4}, for k >= 2 */
        for (int k = 1; k < 60; k++) {
            fact *= k;
            double ck = ((k & 1) ? 1.0 : -1.0) * (2.0 * k) / (fact * (2.0 * k + 1.0));
            double th = ck * upow;
            h += th;
            if (k >= 2) {
                double tp = ck * (2.0 * k - 2.0) * upow2;
                hp += tp;
                upow2 *= u * u;
                if (fabs(th) < 1e-18 * fabs(h) && fabs(tp) < 1e-18 * fabs(hp)) break;
            }
            upow *= u * u;
        }
        h *= tsp;
        hp *= tsp;
        *f_out = h * a * a * a / (4.0 * OR_PI);
        *F_out = hp * a * a * a * a * a / (4.0 * OR_PI);
    } else {
        double e = exp(-u * u);
        double g = erf(u) - tsp * u * e;
        double r3 = rho * rho * rho;
        double q = rho / sig;
        *f_out = g / (4.0 * OR_PI * r3);
        *F_out = (sqrt(2.0 / OR_PI) * q * q * q * e - 3.0 * g) / (4.0 * OR_PI * r3 * rho * rho);
    }
}

/* One source node's contribution at target x (eq. kerpsi and gradient). */
static void or_pair(const double* y, const double* nw, double sig, const double* x,
                    double* phi, double* gr)
{
    double r[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
    double rho = norm3(r);
    double f, F;
    or_radial(rho, sig, &f, &F);
    double d = dot3(nw, r);
    *phi += d * f;
    for (int c = 0; c < 3; c++) gr[c] -= nw[c] * f + d * F * r[c];
}

/* Phi and grad Phi at nt targets by direct summation over all ns source
 * nodes: full kernel, no cutoff, no far-field approximation.  grad may be
 * NULL.  nthreads <= 0 uses the OpenMP default. */
void or_phi_grad(int64_t ns, const double* y, const double* nw, const double* sig,
                 int64_t nt, const double* x, double* phi, double* grad, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        double p = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int64_t s = 0; s < ns; s++)
            or_pair(y + 3*s, nw + 3*s, sig[s], x + 3*t, &p, g);
        phi[t] = p;
        if (grad) { grad[3*t] = g[0]; grad[3*t+1] = g[1]; grad[3*t+2] = g[2]; }
    }
}

/* ------------------------------------------------------------------ */
/* Chart nodes (Sec. 3.2): x0 = T^j(u_i, v_i), H = H^j(u_i, v_i) by linear
 * interpolation of the vertex pseudonormals (eq. mkpseudovec), sig = sigma_j.
 * Node order: triangle-major, then rule order. */
void or_chart_nodes(const double* verts, int64_t m, const int32_t* tris,
                    const double* vpn, const double* sigma, int np,
                    const double* cu, const double* cv,
                    double* x0, double* hdir, double* sloc)
{
    for (int64_t j = 0; j < m; j++) {
        const double* p1 = verts + 3 * (int64_t)tris[3*j+0];
        const double* p2 = verts + 3 * (int64_t)tris[3*j+1];
        const double* p3 = verts + 3 * (int64_t)tris[3*j+2];
        const double* h1 = vpn + 3 * (int64_t)tris[3*j+0];
        const double* h2 = vpn + 3 * (int64_t)tris[3*j+1];
        const double* h3 = vpn + 3 * (int64_t)tris[3*j+2];
        for (int i = 0; i < np; i++) {
            int64_t s = j * np + i;
            for (int c = 0; c < 3; c++) {
                x0[3*s+c] = p1[c] + cu[i] * (p2[c] - p1[c]) + cv[i] * (p3[c] - p1[c]);
                hdir[3*s+c] = h1[c] + cu[i] * (h2[c] - h1[c]) + cv[i] * (h3[c] - h1[c]);
            }
            sloc[s] = sigma[j];
        }
    }
}

/* Status codes of the Newton solve, one per chart node. */
#define OR_ST_CONVERGED 0
#define OR_ST_MAXITER 1
#define OR_ST_ZERODERIV 2
#define OR_ST_NONFINITE 3

/* Newton's method on h for each chart node (eq. newtoneq), h0 = 0.
 * Iteration: x = x0 + h H; evaluate Phi, grad Phi by or_phi_grad's direct sum;
 * stop when |Phi - 1/2| < tol; else h <- h - (Phi - 1/2)/(H . grad Phi), the
 * step clamped to at most 4 sigma_loc (a clamped step sets bit 8 of the
 * status).  At most max_iter evaluations.
 * Outputs: x [n][3], h [n], status [n], iters [n], last |dh| [n]. */
void or_solve_charts(int64_t ns, const double* y, const double* nw, const double* sig,
                     int64_t n, const double* x0, const double* hdir, const double* sloc,
                     double tol, int max_iter, double* xout, double* hout,
                     int32_t* status, int32_t* iters, double* lastdh, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; i++) {
        const double* H = hdir + 3*i;
        double h = 0.0, dh = 0.0;
        int st = OR_ST_MAXITER, clamped = 0, it = 0;
        double x[3];
        for (it = 0; it < max_iter; it++) {
            for (int c = 0; c < 3; c++) x[c] = x0[3*i+c] + h * H[c];
            double p = 0.0, g[3] = {0.0, 0.0, 0.0};
            for (int64_t s = 0; s < ns; s++)
                or_pair(y + 3*s, nw + 3*s, sig[s], x, &p, g);
            double res = p - 0.5;
            if (!isfinite(res)) { st = OR_ST_NONFINITE; it++; break; }
            const int done = fabs(res) < tol;
            double d = dot3(H, g);
            if (!isfinite(d) || d == 0.0) {
                st = done ? OR_ST_CONVERGED : (isfinite(d) ? OR_ST_ZERODERIV : OR_ST_NONFINITE);
                it++;
                break;
            }
            /* the update of eq. newtoneq is applied before the stopping test
               (Sec. 5), also on the sweep that meets the tolerance */
            double step = -res / d;
            double lim = 4.0 * sloc[i];
            if (step > lim) { step = lim; clamped = 1; }
            if (step < -lim) { step = -lim; clamped = 1; }
            h += step;
            dh = fabs(step);
            if (done) { st = OR_ST_CONVERGED; it++; break; }
        }
        for (int c = 0; c < 3; c++) xout[3*i+c] = x0[3*i+c] + h * H[c];
        hout[i] = h;
        status[i] = st | (clamped ? 256 : 0);
        iters[i] = it;
        lastdh[i] = dh;
    }
}

/* Local coordinates of the chart nodes (Sec. 3.3): the chart is
 * x(u,v) = T(u,v) + h(u,v) H(u,v)                               (eq. chart)
 * with T_u = P2 - P1, T_v = P3 - P1 and, H being linear in (u,v),
 * H_u = H2 - H1, H_v = H3 - H1.  x_u is tangent to the level set and grad Phi
 * normal to it, so x_u . grad Phi = 0 gives
 *   h_u = -((T_u + h H_u) . grad Phi) / (H . grad Phi)      (eq. U_vector_2)
 *   x_u = T_u + h H_u + h_u H                                 (eq. u_vector)
 * and the same in v (eq. v_vector, v_vector_2); the area element is
 * da = |x_u x x_v| du dv                                         (eq. da).
 * Node s = j * np + i sits at the rule point (cu[i], cv[i]) of triangle j;
 * h [n] and grad [n][3] are the solved h and grad Phi at the node.
 * Outputs: xu, xv [n][3], jac [n] = |x_u x x_v|. */
void or_chart_frames(const double* verts, int64_t m, const int32_t* tris, const double* vpn,
                     int np, const double* cu, const double* cv, const double* h,
                     const double* grad, double* xu, double* xv, double* jac)
{
    for (int64_t j = 0; j < m; j++) {
        const double* p1 = verts + 3 * (int64_t)tris[3*j+0];
        const double* p2 = verts + 3 * (int64_t)tris[3*j+1];
        const double* p3 = verts + 3 * (int64_t)tris[3*j+2];
        const double* h1 = vpn + 3 * (int64_t)tris[3*j+0];
        const double* h2 = vpn + 3 * (int64_t)tris[3*j+1];
        const double* h3 = vpn + 3 * (int64_t)tris[3*j+2];
        double tu[3], tv[3], hu[3], hv[3];
        for (int c = 0; c < 3; c++) {
            tu[c] = p2[c] - p1[c];
            tv[c] = p3[c] - p1[c];
            hu[c] = h2[c] - h1[c];
            hv[c] = h3[c] - h1[c];
        }
        for (int i = 0; i < np; i++) {
            const int64_t s = j * np + i;
            const double* g = grad + 3*s;
            double H[3], au[3], av[3];
            for (int c = 0; c < 3; c++) {
                H[c] = h1[c] + cu[i] * hu[c] + cv[i] * hv[c];
                au[c] = tu[c] + h[s] * hu[c];
                av[c] = tv[c] + h[s] * hv[c];
            }
            const double hg = dot3(H, g);
            const double h_u = -dot3(au, g) / hg;
            const double h_v = -dot3(av, g) / hg;
            double a[3], b[3], n[3];
            for (int c = 0; c < 3; c++) {
                a[c] = au[c] + h_u * H[c];
                b[c] = av[c] + h_v * H[c];
                xu[3*s+c] = a[c];
                xv[3*s+c] = b[c];
            }
            cross3(a, b, n);
            jac[s] = norm3(n);
        }
    }
}

/* Gauss flux error of the charts (Sec. 5):
 *   eps0 = 1 + integral over Gamma_1/2 of N_hat . grad_x 1/(4 pi |x0 - x|) da
 * with grad_x 1/(4 pi |x0 - x|) = (x0 - x)/(4 pi |x0 - x|^3), the outward unit
 * normal N_hat = -grad Phi/|grad Phi| (Phi falls from 1 inside to 0
 * outside), and the chart rule as quadrature: node s = j * np + i carries
 * cw[i] * jac[s] (the rule's weights sum to the reference triangle's 1/2).
 * Zero for a closed surface around x0; 1 when x0 is outside. */
double or_gauss_flux(int64_t n, int np, const double* cw, const double* x, const double* grad,
                     const double* jac, const double* x0)
{
    double sum = 0.0;
    for (int64_t s = 0; s < n; s++) {
        const double* g = grad + 3*s;
        const double gn = norm3(g);
        double d[3];
        for (int c = 0; c < 3; c++) d[c] = x0[c] - x[3*s+c];
        const double r = norm3(d);
        const double nd = -dot3(g, d) / gn;
        sum += cw[s % np] * jac[s] * nd / (4.0 * M_PI * r * r * r);
    }
    return 1.0 + sum;
}

/* ------------------------------------------------------------------ */
/* Target-dependent smoothing width (Sec. 2.3, eq. sigma2).
 * sigma_j = D_j / lambda with D_j the diameter of the smallest ball enclosing
 * triangle j: the longest edge when the triangle is right or obtuse (the
 * ball on that edge contains the third vertex), else twice the circumradius,
 * 2R = abc / (2 area).  c_j is the centroid.  Outputs c [m][3], sj [m];
 * returns max_j D_j. */
double or_sigma_sources(const double* verts, int64_t m, const int32_t* tris, double lambda,
                        double* c, double* sj)
{
    double dmax = 0.0;
    for (int64_t j = 0; j < m; j++) {
        const double* p[3] = {verts + 3 * (int64_t)tris[3*j+0], verts + 3 * (int64_t)tris[3*j+1],
                              verts + 3 * (int64_t)tris[3*j+2]};
        double e2[3], ab[3], ac[3], n[3];
        for (int k = 0; k < 3; k++) {
            const double* a = p[(k + 1) % 3];
            const double* b = p[(k + 2) % 3];
            double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
            e2[k] = dot3(d, d);             /* squared edge opposite vertex k */
        }
        for (int k = 0; k < 3; k++) {
            ab[k] = p[1][k] - p[0][k];
            ac[k] = p[2][k] - p[0][k];
            c[3*j+k] = (p[0][k] + p[1][k] + p[2][k]) / 3.0;
        }
        cross3(ab, ac, n);
        const double area = 0.5 * norm3(n);
        int kl = 0;
        if (e2[1] > e2[kl]) kl = 1;
        if (e2[2] > e2[kl]) kl = 2;
        double D;
        if (e2[kl] >= e2[(kl + 1) % 3] + e2[(kl + 2) % 3]) {
            D = sqrt(e2[kl]);
        } else {
            D = sqrt(e2[0]) * sqrt(e2[1]) * sqrt(e2[2]) / (2.0 * area);
        }
        sj[j] = D / lambda;
        if (D > dmax) dmax = D;
    }
    return dmax;
}

/* sigma(x) = sum_j sigma_j e_j / sum_j e_j, e_j = exp(-|x - c_j|^2 / (2 sigma0^2))
 * (eq. sigma2), and its gradient
 *   grad sigma = (S1 sum_j e_j (x - c_j) - S0 sum_j sigma_j e_j (x - c_j)) / (sigma0^2 S0^2)
 * with S0 = sum_j e_j, S1 = sum_j sigma_j e_j; direct sums over all M
 * triangles.  gsig may be NULL. */
static void sigma_x_one(int64_t m, const double* c, const double* sj, double sigma0, const double* x,
                        double* sig, double* gsig)
{
    const double inv2s2 = 1.0 / (2.0 * sigma0 * sigma0);
    double S0 = 0.0, S1 = 0.0, A[3] = {0, 0, 0}, B[3] = {0, 0, 0};
    for (int64_t j = 0; j < m; j++) {
        double d[3] = {x[0] - c[3*j], x[1] - c[3*j+1], x[2] - c[3*j+2]};
        const double e = exp(-dot3(d, d) * inv2s2);
        S0 += e;
        S1 += sj[j] * e;
        for (int k = 0; k < 3; k++) {
            A[k] += e * d[k];
            B[k] += sj[j] * e * d[k];
        }
    }
    *sig = S1 / S0;
    if (gsig)
        for (int k = 0; k < 3; k++) gsig[k] = (S1 * A[k] - S0 * B[k]) / (sigma0 * sigma0 * S0 * S0);
}

void or_sigma_x(int64_t m, const double* c, const double* sj, double sigma0, int64_t n, const double* x,
                double* sig, double* gsig)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < n; t++) sigma_x_one(m, c, sj, sigma0, x + 3*t, sig + t, gsig ? gsig + 3*t : NULL);
}

/* Phi and grad Phi with the target's sigma: every pair of target t takes
 * sigma = sig[t] (eq. kerpsi with sigma(x)), and grad Phi gains
 * (dPhi/dsigma) grad sigma (eq. gradPhi, third term), with
 *   d/dsigma [(nw . r) g(u) / (4 pi rho^3)] = -(nw . r) exp(-u^2) / (2 sqrt2 pi^(3/2) sigma^4),
 * r = y - x, u = rho / (sqrt2 sigma).  (The paper prints this term with the
 * opposite sign; differentiating g(u) = erf(u) - (2u/sqrt pi) exp(-u^2),
 * g'(u) = (4 u^2 / sqrt pi) exp(-u^2), and u in sigma gives the minus.) */
static void phi_grad_sigx_one(int64_t ns, const double* y, const double* nw, const double* x, double s,
                              const double* gsig, double* phi, double* grad)
{
    const double cs = 1.0 / (2.0 * sqrt(2.0) * pow(M_PI, 1.5));
    double p = 0.0, g[3] = {0.0, 0.0, 0.0}, dps = 0.0;
    for (int64_t k = 0; k < ns; k++) {
        or_pair(y + 3*k, nw + 3*k, s, x, &p, g);
        double r[3] = {y[3*k] - x[0], y[3*k+1] - x[1], y[3*k+2] - x[2]};
        const double u2 = dot3(r, r) / (2.0 * s * s);
        dps -= dot3(nw + 3*k, r) * exp(-u2) * cs / (s * s * s * s);
    }
    *phi = p;
    if (grad)
        for (int c = 0; c < 3; c++) grad[c] = g[c] + dps * gsig[c];
}

void or_phi_grad_sigx(int64_t ns, const double* y, const double* nw, int64_t nt, const double* x,
                      const double* sig, const double* gsig, double* phi, double* grad, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++)
        phi_grad_sigx_one(ns, y, nw, x + 3*t, sig[t], gsig + 3*t, phi + t, grad ? grad + 3*t : NULL);
}

/* Newton's method for the charts with sigma(x): as or_solve_charts, with
 * sigma(x) and grad sigma re-evaluated at every iterate. */
void or_solve_charts_sigx(int64_t ns, const double* y, const double* nw, int64_t m, const double* c,
                          const double* sj, double sigma0, int64_t n, const double* x0, const double* hdir,
                          const double* sloc, double tol, int max_iter, double* xout, double* hout,
                          int32_t* status, int32_t* iters, double* lastdh, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; i++) {
        const double* H = hdir + 3*i;
        double h = 0.0, dh = 0.0;
        int st = OR_ST_MAXITER, clamped = 0, it = 0;
        double x[3];
        for (it = 0; it < max_iter; it++) {
            for (int k = 0; k < 3; k++) x[k] = x0[3*i+k] + h * H[k];
            double s, gs[3], p, g[3];
            sigma_x_one(m, c, sj, sigma0, x, &s, gs);
            phi_grad_sigx_one(ns, y, nw, x, s, gs, &p, g);
            double res = p - 0.5;
            if (!isfinite(res)) { st = OR_ST_NONFINITE; it++; break; }
            const int done = fabs(res) < tol;
            double d = dot3(H, g);
            if (!isfinite(d) || d == 0.0) {
                st = done ? OR_ST_CONVERGED : (isfinite(d) ? OR_ST_ZERODERIV : OR_ST_NONFINITE);
                it++;
                break;
            }
            /* the update of eq. newtoneq is applied before the stopping test
               (Sec. 5), also on the sweep that meets the tolerance */
            double step = -res / d;
            double lim = 4.0 * sloc[i];
            if (step > lim) { step = lim; clamped = 1; }
            if (step < -lim) { step = -lim; clamped = 1; }
            h += step;
            dh = fabs(step);
            if (done) { st = OR_ST_CONVERGED; it++; break; }
        }
        for (int k = 0; k < 3; k++) xout[3*i+k] = x0[3*i+k] + h * H[k];
        hout[i] = h;
        status[i] = st | (clamped ? 256 : 0);
        iters[i] = it;
        lastdh[i] = dh;
    }
}

/* ------------------------------------------------------------------ */
/* Second derivatives (Sec. 3.3, higher derivatives of the charts).
 * Third radial factor G = F'(rho) / rho.  With k(u) = h'(u)/u as above,
 * G = (k'(u)/u) a^7 / (4 pi):
 *   series  k'(u)/u = (2/sqrt pi) sum_{k>=3} c_k (2k-2)(2k-4) u^{2k-6}
 *   closed  k'(u)/u = 15 g / u^7 - (4/sqrt pi) e^{-u^2} (2/u^2 + 5/u^4)
 * (g'(u) = (4/sqrt pi) u^2 e^{-u^2} differentiated through h = g/u^3).  The
 * series is used below u = 1, where the closed form cancels. */
double or_radial_G(double rho, double sig)
{
    const double a = 1.0 / (sqrt(2.0) * sig);
    const double u = rho * a;
    const double tsp = 2.0 / sqrt(OR_PI);
    double kp;
    if (u < 1.0) {
        double s = 0.0, fact = 1.0, wp = 1.0;   /* wp = u^{2k-6} for k >= 3 */
        for (int k = 1; k < 80; k++) {
            fact *= k;
            if (k < 3) continue;
            const double ck = ((k & 1) ? 1.0 : -1.0) * (2.0 * k) / (fact * (2.0 * k + 1.0));
            const double t = ck * (2.0 * k - 2.0) * (2.0 * k - 4.0) * wp;
            s += t;
            if (k > 6 && fabs(t) < 1e-18 * fabs(s)) break;
            wp *= u * u;
        }
        kp = tsp * s;
    } else {
        const double e = exp(-u * u);
        const double g = erf(u) - tsp * u * e;
        const double u2 = u * u, u4 = u2 * u2;
        kp = 15.0 * g / (u4 * u2 * u) - 2.0 * tsp * e * (2.0 / u2 + 5.0 / u4);
    }
    const double a2 = a * a;
    return kp * a2 * a2 * a2 * a / (4.0 * OR_PI);
}

/* Phi, grad Phi and the Hessian of Phi (per-triangle sigma), direct sums.
 * For one pair, with r = y - x, q = nw . r:
 *   d2/dx_i dx_j [q f] = F (nw_i r_j + nw_j r_i + q delta_ij) + q G r_i r_j.
 * hess [nt][6] = (xx, xy, xz, yy, yz, zz). */
void or_phi_grad_hess(int64_t ns, const double* y, const double* nw, const double* sig, int64_t nt,
                      const double* x, double* phi, double* grad, double* hess, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        double p = 0.0, g[3] = {0.0, 0.0, 0.0}, H[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t s = 0; s < ns; s++) {
            const double* yy = y + 3*s;
            const double* n = nw + 3*s;
            double r[3] = {yy[0] - x[3*t], yy[1] - x[3*t+1], yy[2] - x[3*t+2]};
            const double rho = norm3(r);
            double f, F;
            or_radial(rho, sig[s], &f, &F);
            const double G = or_radial_G(rho, sig[s]);
            const double q = dot3(n, r);
            p += q * f;
            for (int c = 0; c < 3; c++) g[c] -= n[c] * f + q * F * r[c];
            int k = 0;
            for (int i = 0; i < 3; i++)
                for (int j = i; j < 3; j++)
                    H[k++] += F * (n[i] * r[j] + n[j] * r[i] + (i == j ? q : 0.0)) + q * G * r[i] * r[j];
        }
        phi[t] = p;
        for (int c = 0; c < 3; c++) grad[3*t+c] = g[c];
        for (int c = 0; c < 6; c++) hess[6*t+c] = H[c];
    }
}

/* Second derivatives of the charts and the curvatures of Gamma_1/2 at the
 * chart nodes.  On a flat triangle T_uu = T_uv = T_vv = 0 and the linear H
 * has no second derivatives, so (eq. uu_vector, read with the H_u factor on
 * 2 h_u and h_uu on H, and its v and mixed analogues)
 *   x_uu = 2 h_u H_u + h_uu H,  x_uv = h_u H_v + h_v H_u + h_uv H,  x_vv = 2 h_v H_v + h_vv H,
 * and differentiating x_u . grad Phi(x) = 0 once more (eq. uu_vector_aux1,
 * uu_vector_aux2):
 *   h_uu = -(x_u^T Hess x_u + 2 h_u H_u . grad Phi) / (H . grad Phi)
 *   h_uv = -(x_u^T Hess x_v + (h_u H_v + h_v H_u) . grad Phi) / (H . grad Phi)
 *   h_vv = -(x_v^T Hess x_v + 2 h_v H_v . grad Phi) / (H . grad Phi).
 * With N = -grad Phi/|grad Phi| (outward), E, F, G = x_u.x_u, x_u.x_v, x_v.x_v
 * and L, M, Nn = x_uu.N, x_uv.N, x_vv.N:
 *   kgauss = (L Nn - M^2) / (E G - F^2),
 *   kmean  = -(E Nn - 2 F M + G L) / (E G - F^2)  (sum of the principal
 *            curvatures, 2/R on a sphere of radius R).
 * Inputs as or_chart_frames plus hess [n][6]; outputs xuu, xuv, xvv [n][3],
 * kmean, kgauss [n]. */
void or_chart_second(const double* verts, int64_t m, const int32_t* tris, const double* vpn, int np,
                     const double* cu, const double* cv, const double* h, const double* grad, const double* hess,
                     double* xuu, double* xuv, double* xvv, double* kmean, double* kgauss)
{
    for (int64_t j = 0; j < m; j++) {
        const double* p1 = verts + 3 * (int64_t)tris[3*j+0];
        const double* p2 = verts + 3 * (int64_t)tris[3*j+1];
        const double* p3 = verts + 3 * (int64_t)tris[3*j+2];
        const double* h1 = vpn + 3 * (int64_t)tris[3*j+0];
        const double* h2 = vpn + 3 * (int64_t)tris[3*j+1];
        const double* h3 = vpn + 3 * (int64_t)tris[3*j+2];
        double tu[3], tv[3], hu[3], hv[3];
        for (int c = 0; c < 3; c++) {
            tu[c] = p2[c] - p1[c];
            tv[c] = p3[c] - p1[c];
            hu[c] = h2[c] - h1[c];
            hv[c] = h3[c] - h1[c];
        }
        for (int i = 0; i < np; i++) {
            const int64_t s = j * np + i;
            const double* g = grad + 3*s;
            const double* Hs = hess + 6*s;
            const double S[3][3] = {{Hs[0], Hs[1], Hs[2]}, {Hs[1], Hs[3], Hs[4]}, {Hs[2], Hs[4], Hs[5]}};
            double H[3], a[3], b[3];
            for (int c = 0; c < 3; c++) H[c] = h1[c] + cu[i] * hu[c] + cv[i] * hv[c];
            const double hg = dot3(H, g);
            double au[3], av[3];
            for (int c = 0; c < 3; c++) {
                au[c] = tu[c] + h[s] * hu[c];
                av[c] = tv[c] + h[s] * hv[c];
            }
            const double h_u = -dot3(au, g) / hg, h_v = -dot3(av, g) / hg;
            for (int c = 0; c < 3; c++) {
                a[c] = au[c] + h_u * H[c];
                b[c] = av[c] + h_v * H[c];
            }
            double Sa[3], Sb[3];
            for (int r = 0; r < 3; r++) {
                Sa[r] = S[r][0] * a[0] + S[r][1] * a[1] + S[r][2] * a[2];
                Sb[r] = S[r][0] * b[0] + S[r][1] * b[1] + S[r][2] * b[2];
            }
            const double huu = -(dot3(a, Sa) + 2.0 * h_u * dot3(hu, g)) / hg;
            const double huv = -(dot3(a, Sb) + h_u * dot3(hv, g) + h_v * dot3(hu, g)) / hg;
            const double hvv = -(dot3(b, Sb) + 2.0 * h_v * dot3(hv, g)) / hg;
            double uu[3], uv[3], vv[3];
            for (int c = 0; c < 3; c++) {
                uu[c] = 2.0 * h_u * hu[c] + huu * H[c];
                uv[c] = h_u * hv[c] + h_v * hu[c] + huv * H[c];
                vv[c] = 2.0 * h_v * hv[c] + hvv * H[c];
                xuu[3*s+c] = uu[c];
                xuv[3*s+c] = uv[c];
                xvv[3*s+c] = vv[c];
            }
            const double gn = norm3(g);
            double N[3] = {-g[0] / gn, -g[1] / gn, -g[2] / gn};
            const double E = dot3(a, a), F = dot3(a, b), G = dot3(b, b);
            const double L = dot3(uu, N), M = dot3(uv, N), Nn = dot3(vv, N);
            const double det = E * G - F * F;
            kgauss[s] = (L * Nn - M * M) / det;
            kmean[s] = -(E * Nn - 2.0 * F * M + G * L) / det;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Refinement (Sec. 3.4, surface refinement): a triangle split 1 -> 4 at its
 * edge midpoints, any number of times, keeps the chart map of its parent:
 * nodes of the children are points (u, v) of the parent's reference
 * triangle, x0 = T(u, v) and H(u, v) linear in the parent's (u, v).  Since H
 * is linear along every edge, a midpoint's H equals the mean of the edge's
 * end values whichever neighbour is refined, so the pseudonormal field stays
 * continuous across refined and unrefined neighbours.  Node s lies in
 * triangle tri[s] at (uv[2s], uv[2s+1]). */
void or_chart_nodes_at(const double* verts, const int32_t* tris, const double* vpn, const double* sigma,
                       int64_t n, const int32_t* tri, const double* uv, double* x0, double* hdir, double* sloc)
{
    for (int64_t s = 0; s < n; s++) {
        const int64_t j = tri[s];
        const double u = uv[2*s], v = uv[2*s+1];
        const double* p1 = verts + 3 * (int64_t)tris[3*j+0];
        const double* p2 = verts + 3 * (int64_t)tris[3*j+1];
        const double* p3 = verts + 3 * (int64_t)tris[3*j+2];
        const double* h1 = vpn + 3 * (int64_t)tris[3*j+0];
        const double* h2 = vpn + 3 * (int64_t)tris[3*j+1];
        const double* h3 = vpn + 3 * (int64_t)tris[3*j+2];
        for (int c = 0; c < 3; c++) {
            x0[3*s+c] = p1[c] + u * (p2[c] - p1[c]) + v * (p3[c] - p1[c]);
            hdir[3*s+c] = h1[c] + u * (h2[c] - h1[c]) + v * (h3[c] - h1[c]);
        }
        sloc[s] = sigma[j];
    }
}

/* or_chart_frames at explicit nodes (triangle and parent (u, v) per node). */
void or_chart_frames_at(const double* verts, const int32_t* tris, const double* vpn, int64_t n,
                        const int32_t* tri, const double* uv, const double* h, const double* grad, double* xu,
                        double* xv, double* jac)
{
    for (int64_t s = 0; s < n; s++) {
        const int64_t j = tri[s];
        /* one node of triangle j: reuse the rule form with a one-point rule */
        or_chart_frames(verts, 1, tris + 3 * j, vpn, 1, uv + 2*s, uv + 2*s + 1, h + s, grad + 3*s,
                        xu + 3*s, xv + 3*s, jac + s);
    }
}

/* Gauss flux error with a quadrature weight per node (w[s] in the parent's
 * reference triangle, as the chart rule's weights). */
double or_gauss_flux_w(int64_t n, const double* w, const double* x, const double* grad, const double* jac,
                       const double* x0)
{
    double sum = 0.0;
    for (int64_t s = 0; s < n; s++) {
        const double* g = grad + 3*s;
        const double gn = norm3(g);
        double d[3];
        for (int c = 0; c < 3; c++) d[c] = x0[c] - x[3*s+c];
        const double r = norm3(d);
        const double nd = -dot3(g, d) / gn;
        sum += w[s] * jac[s] * nd / (4.0 * M_PI * r * r * r);
    }
    return 1.0 + sum;
}

/* ------------------------------------------------------------------ */
/* Quadratic (curved) skeleton patches (Sec. 5, quadratic skeletons): each
 * patch is the 6-node curvilinear triangle through its corners P1, P2, P3
 * and one node on each edge, P4 (edge P1-P2), P5 (edge P2-P3), P6 (edge
 * P3-P1):
 *   T(u,v) = sum_k N_k(u,v) P_k  with L1 = 1 - u - v, L2 = u, L3 = v and
 *   N1 = L1 (2 L1 - 1), N2 = L2 (2 L2 - 1), N3 = L3 (2 L3 - 1),
 *   N4 = 4 L1 L2,       N5 = 4 L2 L3,       N6 = 4 L3 L1,
 * the standard second-order Lagrange basis on T0.  With the edge nodes at
 * the edge midpoints the map is the flat chart of eq. tparam.  Everything
 * else follows the flat construction with the patch's own tangents: the
 * normal N(u,v) = T_u x T_v now varies over the patch, a source node
 * carries nw = w N(u_k, v_k), a corner's vertex angle is the angle between
 * the tangents of its two edges there, the vertex pseudonormal is the
 * angle-weighted mean of the corner unit normals (eq. mkvertexpn), and H is
 * linear in (u, v) between the three corner pseudonormals (eq. mkpseudovec),
 * which the paper describes as analogous to the flat case.  Neighbouring
 * patches share an edge's three nodes, so T, and with it the charts, stay
 * continuous across edges.  tris6 [m][6] holds P1..P6's vertex indices. */
static void quad_map(const double* verts, const int32_t* t6, double u, double v, double* T, double* Tu,
                     double* Tv)
{
    const double L1 = 1.0 - u - v, L2 = u, L3 = v;
    const double N[6] = {L1 * (2.0*L1 - 1.0), L2 * (2.0*L2 - 1.0), L3 * (2.0*L3 - 1.0),
                         4.0 * L1 * L2, 4.0 * L2 * L3, 4.0 * L3 * L1};
    /* d/du: dL1 = -1, dL2 = 1, dL3 = 0;  d/dv: dL1 = -1, dL2 = 0, dL3 = 1 */
    const double Nu[6] = {-(4.0*L1 - 1.0), 4.0*L2 - 1.0, 0.0, 4.0 * (L1 - L2), 4.0 * L3, -4.0 * L3};
    const double Nv[6] = {-(4.0*L1 - 1.0), 0.0, 4.0*L3 - 1.0, -4.0 * L2, 4.0 * L2, 4.0 * (L1 - L3)};
    for (int c = 0; c < 3; c++) {
        T[c] = Tu[c] = Tv[c] = 0.0;
        for (int k = 0; k < 6; k++) {
            const double p = verts[3 * (int64_t)t6[k] + c];
            T[c] += N[k] * p;
            Tu[c] += Nu[k] * p;
            Tv[c] += Nv[k] * p;
        }
    }
}

/* Geometry of quadratic patches: sigma_j = 0.5 sqrt(2 area_j) (or sigma_in),
 * area_j = sum_k w_k |N(u_k, v_k)| with the given rule on the patch, and the
 * vertex pseudonormals (eq. mkvertexpn) from the corners' unit normals and
 * vertex angles.  At the corners (0,0), (1,0), (0,1) the two edges leave
 * along (T_u, T_v), (T_v - T_u, -T_u) and (-T_v, T_u - T_v).
 * Returns 0, or -1 when a vertex has zero total angle. */
int or_geometry_quad(int64_t nv, const double* verts, int64_t m, const int32_t* tris6, const double* sigma_in,
                     int nq, const double* ru, const double* rv, const double* rw, double* sigma, double* vpn)
{
    double* asum = (double*)calloc((size_t)nv, sizeof(double));
    memset(vpn, 0, sizeof(double) * 3 * (size_t)nv);
    static const double cuv[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    for (int64_t j = 0; j < m; j++) {
        const int32_t* t6 = tris6 + 6 * j;
        double area = 0.0;
        for (int k = 0; k < nq; k++) {
            double T[3], Tu[3], Tv[3], n[3];
            quad_map(verts, t6, ru[k], rv[k], T, Tu, Tv);
            cross3(Tu, Tv, n);
            area += rw[k] * norm3(n);
        }
        sigma[j] = sigma_in ? sigma_in[j] : 0.5 * sqrt(2.0 * area);
        for (int c = 0; c < 3; c++) {
            double T[3], Tu[3], Tv[3], n[3], e1[3], e2[3], x[3];
            quad_map(verts, t6, cuv[c][0], cuv[c][1], T, Tu, Tv);
            cross3(Tu, Tv, n);
            const double nn = norm3(n);
            for (int d = 0; d < 3; d++) {
                if (c == 0) { e1[d] = Tu[d]; e2[d] = Tv[d]; }
                else if (c == 1) { e1[d] = Tv[d] - Tu[d]; e2[d] = -Tu[d]; }
                else { e1[d] = -Tv[d]; e2[d] = Tu[d] - Tv[d]; }
            }
            cross3(e1, e2, x);
            const double th = atan2(norm3(x), dot3(e1, e2));
            const int64_t vi = t6[c];
            asum[vi] += th;
            for (int d = 0; d < 3; d++) vpn[3*vi+d] += th * n[d] / nn;
        }
    }
    int bad = 0;
    for (int64_t i = 0; i < nv; i++) {
        if (asum[i] > 0) {
            for (int k = 0; k < 3; k++) vpn[3*i+k] /= asum[i];
        }
    }
    /* only corner vertices carry pseudonormals; edge nodes keep zero */
    for (int64_t j = 0; j < m; j++)
        for (int c = 0; c < 3; c++)
            if (!(asum[tris6[6*j+c]] > 0)) bad = 1;
    free(asum);
    return bad ? -1 : 0;
}

/* Source nodes on quadratic patches (eq. discrete_int on the curved
 * skeleton): y = T(u_k, v_k), nw = w_k N(u_k, v_k) (the area element is in
 * |N|), sig = sigma_j.  Triangle-major, then rule order. */
void or_sources_quad(const double* verts, int64_t m, const int32_t* tris6, const double* sigma, int nq,
                     const double* ru, const double* rv, const double* rw, double* y, double* nw, double* sig)
{
    for (int64_t j = 0; j < m; j++) {
        for (int k = 0; k < nq; k++) {
            const int64_t s = j * nq + k;
            double T[3], Tu[3], Tv[3], n[3];
            quad_map(verts, tris6 + 6 * j, ru[k], rv[k], T, Tu, Tv);
            cross3(Tu, Tv, n);
            for (int c = 0; c < 3; c++) {
                y[3*s+c] = T[c];
                nw[3*s+c] = rw[k] * n[c];
            }
            sig[s] = sigma[j];
        }
    }
}

/* Chart nodes on quadratic patches at explicit (triangle, u, v):
 * x0 = T(u, v), H linear in the corner pseudonormals (eq. mkpseudovec). */
void or_chart_nodes_quad_at(const double* verts, const int32_t* tris6, const double* vpn, const double* sigma,
                            int64_t n, const int32_t* tri, const double* uv, double* x0, double* hdir,
                            double* sloc)
{
    for (int64_t s = 0; s < n; s++) {
        const int64_t j = tri[s];
        const double u = uv[2*s], v = uv[2*s+1];
        double T[3], Tu[3], Tv[3];
        quad_map(verts, tris6 + 6 * j, u, v, T, Tu, Tv);
        const double* h1 = vpn + 3 * (int64_t)tris6[6*j+0];
        const double* h2 = vpn + 3 * (int64_t)tris6[6*j+1];
        const double* h3 = vpn + 3 * (int64_t)tris6[6*j+2];
        for (int c = 0; c < 3; c++) {
            x0[3*s+c] = T[c];
            hdir[3*s+c] = h1[c] + u * (h2[c] - h1[c]) + v * (h3[c] - h1[c]);
        }
        sloc[s] = sigma[j];
    }
}

/* Local coordinates of charts on quadratic patches (eq. u_vector,
 * U_vector_2, v_vector, v_vector_2, da) with the patch's tangents at the
 * node: h_u = -((T_u + h H_u) . grad Phi)/(H . grad Phi), x_u = T_u + h H_u
 * + h_u H, and the same in v; jac = |x_u x x_v|. */
void or_chart_frames_quad_at(const double* verts, const int32_t* tris6, const double* vpn, int64_t n,
                             const int32_t* tri, const double* uv, const double* h, const double* grad,
                             double* xu, double* xv, double* jac)
{
    for (int64_t s = 0; s < n; s++) {
        const int64_t j = tri[s];
        const double u = uv[2*s], v = uv[2*s+1];
        double T[3], Tu[3], Tv[3];
        quad_map(verts, tris6 + 6 * j, u, v, T, Tu, Tv);
        const double* h1 = vpn + 3 * (int64_t)tris6[6*j+0];
        const double* h2 = vpn + 3 * (int64_t)tris6[6*j+1];
        const double* h3 = vpn + 3 * (int64_t)tris6[6*j+2];
        const double* g = grad + 3*s;
        double H[3], au[3], av[3];
        for (int c = 0; c < 3; c++) {
            H[c] = h1[c] + u * (h2[c] - h1[c]) + v * (h3[c] - h1[c]);
            au[c] = Tu[c] + h[s] * (h2[c] - h1[c]);
            av[c] = Tv[c] + h[s] * (h3[c] - h1[c]);
        }
        const double hg = dot3(H, g);
        const double h_u = -dot3(au, g) / hg;
        const double h_v = -dot3(av, g) / hg;
        double a[3], b[3], nn[3];
        for (int c = 0; c < 3; c++) {
            a[c] = au[c] + h_u * H[c];
            b[c] = av[c] + h_v * H[c];
            xu[3*s+c] = a[c];
            xv[3*s+c] = b[c];
        }
        cross3(a, b, nn);
        jac[s] = norm3(nn);
    }
}
