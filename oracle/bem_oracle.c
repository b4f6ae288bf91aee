/*
 * bem_oracle.c -- plain, slow, FP64 reference ("oracle") for the collocation
 * boundary element method with Burton-Miller coupling described in
 * Kreuzer, Pollack, Brinkmann, Majdak, "NumCalc: An open-source BEM code for
 * solving acoustic scattering problems" (arXiv 2312.00005).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA implementation in the package;
 * the package must never call it.
 *
 * What it computes (pressure variables, time factor e^{-i w t}, exterior
 * problem tau = +1, constant elements on flat triangles, collocation at the
 * element midpoints):
 *   - geometry of each triangle: normal, area, midpoint (Sec. 2.3, App. A);
 *   - the kernels G, H = dG/dn_y, H' = dG/dn_x, E = d2G/dn_x dn_y (Eq. BIE_I,
 *     Eq. dBIE);
 *   - the element integrals with the paper's rules: Duffy singular rule on
 *     six sub-triangles with 4x4 Gauss points (Sec. 3.1.1), H_ii = H'_ii = 0,
 *     the hypersingular E_ii as an edge integral (4 parts x 3 Gauss points
 *     per edge) plus k^2 G_ii (Sec. 3.1.2), the quasi-singular subdivision
 *     while r~ < 1.3 (Sec. 3.1.3) and the regular rule of order m chosen by
 *     the a-priori error estimates with tolerance 1e-3, m <= 6 (Sec. 3.1.4);
 *   - the dense Burton-Miller system of Eq. SystemI with gamma = i/k, with
 *     per-column coefficients that fold in the boundary conditions;
 *   - a dense O(N^2) matrix-vector product and restarted GMRES;
 *   - the interior problem (tau = -1 in Eq. BIE_I and Eq. SystemI: the sign
 *     of every integral operator) as a parameter, tau = +1 by default;
 *   - the field at exterior points from the representation formula with
 *     lambda = 1 (Eq. BIE_I; interior points when tau = -1), and its gradient (the particle velocity of
 *     Eq. utopandv) from the same formula differentiated under the integral;
 *   - the field-point integrals G(x)_j, H(x)_j as dense matrices, for the
 *     adjoint gradient of a field loss with respect to the admittances (a
 *     derived quantity the paper does not compute; its steps are in the
 *     Python wrapper);
 *   - the pieces of the plane-wave expansion of Eq. FMMBase (spherical Hankel
 *     functions by upward recursion, Legendre polynomials, the unit-sphere
 *     grid of Sec. 3.3.1, the translation D_L and the single-pair expansion)
 *     for unit tests only: the dense oracle never uses the FMM.
 *
 * Readings of the paper where it is silent or garbled (each listed in the
 * design notes): the triangle rule of order m is the m x m conical-product
 * (collapsed Gauss) rule; r~ is the distance from the collocation point to the
 * (sub)element midpoint over the square root of the (sub)element area, both
 * for subdivision and for the order; subdivision deeper than 15 levels is an
 * error; the six Duffy sub-triangles join the midpoint to the three vertices
 * and the three edge midpoints; the FMM prefactor is ik/(16 pi^2).
 *
 * Complex numbers cross the C ABI as interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846

/* Parameters of the quadrature (Sec. 3.1); defaults are the paper's. */
typedef struct {
    double quad_tol;      /* a-priori tolerance for the regular order, 1e-3 */
    int    m_max;         /* cap on the regular order, 6 */
    double rt_subdiv;     /* subdivide while r~ < 1.3 */
    int    max_depth;     /* at most 15 nested subdivisions */
    int    n_duffy;       /* Gauss points per direction in the Duffy rule, 4 */
    int    edge_parts;    /* parts per edge in the hypersingular rule, 4 */
    int    edge_gauss;    /* Gauss points per part, 3 */
    double tau;           /* +1 exterior problem, -1 interior problem (Eq. BIE_I) */
} orc_params;

static void default_params(orc_params *p)
{
    p->quad_tol = 1e-3;
    p->m_max = 6;
    p->rt_subdiv = 1.3;
    p->max_depth = 15;
    p->n_duffy = 4;
    p->edge_parts = 4;
    p->edge_gauss = 3;
    p->tau = 1.0;
}

static int clamp_rule(int n);

/* Fill parameters from an optional array of 7 doubles (NULL = defaults). */
static void read_params(const double *pp, orc_params *p)
{
    default_params(p);
    if (!pp) return;
    p->quad_tol = pp[0];
    p->m_max = (int)pp[1];
    p->rt_subdiv = pp[2];
    p->max_depth = (int)pp[3];
    p->n_duffy = (int)pp[4];
    p->edge_parts = (int)pp[5];
    p->edge_gauss = (int)pp[6];
    p->tau = pp[7] < 0.0 ? -1.0 : 1.0;
    p->m_max = clamp_rule(p->m_max);
    p->n_duffy = clamp_rule(p->n_duffy);
    p->edge_gauss = clamp_rule(p->edge_gauss);
    if (p->edge_parts < 1) p->edge_parts = 1;
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static void vsub(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double vdot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void vcross(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double vnorm(const double *a) { return sqrt(vdot(a, a)); }

/* ------------------------------------------------------------------------ */
/* Gauss rules.  Nodes are found by bracketing sign changes of the          */
/* orthogonal polynomial on a fine grid in theta (t = cos theta), bisection, */
/* then one Newton polish; weights from the classical closed forms.          */
/* ------------------------------------------------------------------------ */

/* Legendre P_n(t) and P_{n-1}(t) by the three-term recurrence. */
static void legendre_pair(int n, double t, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = t;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

/* Jacobi P_n^{(1,0)}(t) and P_{n-1}^{(1,0)}(t) by the three-term recurrence
 * (n+1)(2n-1) P_n = ((2n+1)(2n-1) t + 1) P_{n-1} - (n-1)(2n+1) P_{n-2}. */
static void jacobi10_pair(int n, double t, double *pn, double *pnm1)
{
    double p0 = 1.0, p1 = 0.5 * (1.0 + 3.0 * t);
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int j = 2; j <= n; ++j) {
        double p2 = (((2.0 * j + 1.0) * (2.0 * j - 1.0) * t + 1.0) * p1
                     - (j - 1.0) * (2.0 * j + 1.0) * p0) / ((j + 1.0) * (2.0 * j - 1.0));
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

static double poly_value(int family, int n, double t)
{
    double pn, pm;
    if (family == 0) legendre_pair(n, t, &pn, &pm);
    else jacobi10_pair(n, t, &pn, &pm);
    return pn;
}

/* derivative of P_n (family 0: Legendre, 1: Jacobi(1,0)) at interior t */
static double poly_deriv(int family, int n, double t)
{
    double pn, pm;
    if (family == 0) {
        legendre_pair(n, t, &pn, &pm);
        /* (1 - t^2) P_n' = n (P_{n-1} - t P_n) */
        return n * (pm - t * pn) / (1.0 - t * t);
    }
    jacobi10_pair(n, t, &pn, &pm);
    /* (2n+1)(1 - t^2) P_n' = n (1 - (2n+1) t) P_n + 2 n (n+1) P_{n-1} */
    return (n * (1.0 - (2.0 * n + 1.0) * t) * pn + 2.0 * n * (n + 1.0) * pm)
           / ((2.0 * n + 1.0) * (1.0 - t * t));
}

/* zeros of P_n in (-1, 1), ascending */
static int poly_zeros(int family, int n, double *z)
{
    int found = 0;
    int ngrid = 64 * n + 64;
    double th_prev = ORC_PI, t_prev = cos(th_prev);
    double f_prev = poly_value(family, n, t_prev);
    for (int g = 1; g <= ngrid && found < n; ++g) {
        double th = ORC_PI * (1.0 - (double)g / ngrid);
        double t = cos(th);
        double f = poly_value(family, n, t);
        if (f == 0.0) { z[found++] = t; t_prev = t; f_prev = f; continue; }
        if (f_prev != 0.0 && (f_prev < 0.0) != (f < 0.0)) {
            double lo = t_prev, hi = t, flo = f_prev;
            for (int it = 0; it < 200 && hi - lo > 1e-300; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double fm = poly_value(family, n, mid);
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
                else hi = mid;
            }
            double r = 0.5 * (lo + hi);
            double d = poly_deriv(family, n, r);
            if (d != 0.0) {
                double rn = r - poly_value(family, n, r) / d;
                if (rn > t_prev && rn < t) r = rn;
            }
            z[found++] = r;
        }
        t_prev = t;
        f_prev = f;
    }
    return found == n ? 0 : -1;
}

/* Gauss-Legendre rule with n points on [-1, 1]: integrates degree 2n-1. */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return -1;
    if (poly_zeros(0, n, x)) return -1;
    for (int i = 0; i < n; ++i) {
        double d = poly_deriv(0, n, x[i]);
        w[i] = 2.0 / ((1.0 - x[i] * x[i]) * d * d);
    }
    return 0;
}

/* Gauss-Jacobi rule with n points on [-1, 1] for the weight (1 - t). */
int orc_gauss_jacobi10(int n, double *x, double *w)
{
    if (n < 1) return -1;
    if (poly_zeros(1, n, x)) return -1;
    for (int i = 0; i < n; ++i) {
        double d = poly_deriv(1, n, x[i]);
        w[i] = 4.0 / ((1.0 - x[i] * x[i]) * d * d);
    }
    return 0;
}

/* Triangle rule of order m on the reference triangle {xi, eta >= 0,
 * xi + eta <= 1}: the conical product of an m-point Gauss-Jacobi(1,0) rule
 * in u = xi and an m-point Gauss-Legendre rule in v, with eta = (1 - u) v.
 * m*m points, weights summing to 1/2, exact for polynomials of degree 2m-1.
 * (The paper cites Cowper's tables without printing them; this rule of the
 * same order is our reading.) */
int orc_triangle_rule(int m, double *xi, double *eta, double *w)
{
    double tj[64], wj[64], tl[64], wl[64];
    if (m < 1 || m > 64) return -1;
    if (orc_gauss_jacobi10(m, tj, wj) || orc_gauss_legendre(m, tl, wl)) return -1;
    int q = 0;
    for (int a = 0; a < m; ++a) {
        double u = 0.5 * (tj[a] + 1.0), wu = 0.25 * wj[a];
        for (int b = 0; b < m; ++b) {
            double v = 0.5 * (tl[b] + 1.0), wv = 0.5 * wl[b];
            xi[q] = u;
            eta[q] = (1.0 - u) * v;
            w[q] = wu * wv;
            ++q;
        }
    }
    return 0;
}

/* The rules are computed once and cached (rules up to 32 points per
 * direction); caching changes no arithmetic. */
#define ORC_MAXR 32
static double gl_x[ORC_MAXR + 1][ORC_MAXR], gl_w[ORC_MAXR + 1][ORC_MAXR];
static double tr_xi[ORC_MAXR + 1][ORC_MAXR * ORC_MAXR], tr_eta[ORC_MAXR + 1][ORC_MAXR * ORC_MAXR],
    tr_w[ORC_MAXR + 1][ORC_MAXR * ORC_MAXR];
static int rules_ready = 0;

/* Called at the top of every exported entry point that integrates, before
 * any parallel region. */
static void ensure_rules(void)
{
    if (rules_ready) return;
    for (int n = 1; n <= ORC_MAXR; ++n) {
        orc_gauss_legendre(n, gl_x[n], gl_w[n]);
        orc_triangle_rule(n, tr_xi[n], tr_eta[n], tr_w[n]);
    }
    rules_ready = 1;
}

static int clamp_rule(int n) { return n < 1 ? 1 : (n > ORC_MAXR ? ORC_MAXR : n); }

/* ------------------------------------------------------------------------ */
/* Regular-quadrature order (Sec. 3.1.4): smallest m with all three          */
/* a-priori estimates below the tolerance, capped at m_max.                  */
/* ------------------------------------------------------------------------ */
int orc_quad_order(double rt, double tol, int m_max)
{
    double q = 1.0 / (2.0 * rt);
    for (int m = 1; m <= m_max; ++m) {
        double eG = 32.0 * pow(q, 2.0 * m + 1.0);
        double eH = 64.0 * (2.0 * m + 1.0) * pow(q, 2.0 * m + 2.0);
        double eE = 128.0 * (m + 1.0) * (2.0 * m + 1.0) * pow(q, 2.0 * m + 3.0);
        if (eG < tol && eH < tol && eE < tol) return m;
    }
    return m_max;
}

/* ------------------------------------------------------------------------ */
/* Kernels.  d = y - x, r = |d|.                                             */
/*   G  = e^{ikr} / (4 pi r)                                                 */
/*   H  = dG/dn_y = G (ik - 1/r) (d.n_y)/r                                   */
/*   H' = dG/dn_x = -G (ik - 1/r) (d.n_x)/r                                  */
/*   E  = d2G/dn_x dn_y = G [ (k^2 + 3ik/r - 3/r^2)(d.n_x/r)(d.n_y/r)        */
/*                            - (ik/r - 1/r^2)(n_x.n_y) ]                    */
/* (E follows from differentiating G twice; the paper defines it below       */
/* Eq. dBIE.)                                                                */
/* ------------------------------------------------------------------------ */
static void kernels(const double *x, const double *nx, const double *y, const double *ny,
                    double k, cplx out[4])
{
    double d[3];
    vsub(y, x, d);
    double r = vnorm(d);
    double rx = vdot(d, nx) / r, ry = vdot(d, ny) / r, nn = vdot(nx, ny);
    cplx ik = I * k;
    cplx G = cexp(ik * r) / (4.0 * ORC_PI * r);
    out[0] = G;
    out[1] = G * (ik - 1.0 / r) * ry;
    out[2] = -G * (ik - 1.0 / r) * rx;
    out[3] = G * ((k * k + 3.0 * ik / r - 3.0 / (r * r)) * rx * ry - (ik / r - 1.0 / (r * r)) * nn);
}

void orc_kernels(const double *x, const double *nx, const double *y, const double *ny, double k,
                 double *out8)
{
    cplx o[4];
    kernels(x, nx, y, ny, k, o);
    for (int i = 0; i < 4; ++i) { out8[2 * i] = creal(o[i]); out8[2 * i + 1] = cimag(o[i]); }
}

/* ------------------------------------------------------------------------ */
/* Singular rule (Sec. 3.1.1): the polygon p[0..nv-1] around x is cut into   */
/* nv triangles (x, p[e], p[e+1]); each is mapped from the unit square by    */
/* y = x + u ((p[e] - x) + v (p[e+1] - p[e])), Jacobian 2 A_e u, and         */
/* integrated with n x n Gauss-Legendre points.  Returns the integral of G.  */
/* For a triangle element the polygon is (a, m_ab, b, m_bc, c, m_ca).        */
/* ------------------------------------------------------------------------ */
static cplx duffy_G(const double *x, const double *poly, int nv, double k, int n)
{
    n = clamp_rule(n);
    const double *gt = gl_x[n], *gw = gl_w[n];
    cplx sum = 0.0;
    for (int e = 0; e < nv; ++e) {
        const double *p1 = poly + 3 * e, *p2 = poly + 3 * ((e + 1) % nv);
        double e1[3], e2[3], cr[3];
        vsub(p1, x, e1);
        vsub(p2, p1, e2);
        vcross(e1, e2, cr);
        double twoA = vnorm(cr);
        for (int a = 0; a < n; ++a) {
            double u = 0.5 * (gt[a] + 1.0), wu = 0.5 * gw[a];
            for (int b = 0; b < n; ++b) {
                double v = 0.5 * (gt[b] + 1.0), wv = 0.5 * gw[b];
                double y[3];
                for (int c = 0; c < 3; ++c) y[c] = x[c] + u * (e1[c] + v * e2[c]);
                double d[3];
                vsub(y, x, d);
                double r = vnorm(d);
                cplx G = cexp(I * k * r) / (4.0 * ORC_PI * r);
                sum += wu * wv * twoA * u * G;
            }
        }
    }
    return sum;
}

void orc_duffy_G(const double *x, const double *poly, int nv, double k, int n, double *out2)
{
    ensure_rules();
    cplx g = duffy_G(x, poly, nv, k, n);
    out2[0] = creal(g);
    out2[1] = cimag(g);
}

/* Hypersingular edge part (Sec. 3.1.2): sum over the polygon edges,         */
/* traversed counter-clockwise about n, of                                   */
/*   sum_{l,m,j} n_l eps_{lmj} \oint dG/dy_m dy_j  =  \oint grad_y G . m ds,  */
/* m = t x n the outward in-plane edge normal.  Each edge is cut into        */
/* `parts` equal pieces with `ng` Gauss points each.                         */
static cplx edge_fp(const double *x, const double *n, const double *poly, int nv, double k,
                    int parts, int ng)
{
    ng = clamp_rule(ng);
    const double *gt = gl_x[ng], *gw = gl_w[ng];
    cplx sum = 0.0;
    cplx ik = I * k;
    for (int e = 0; e < nv; ++e) {
        const double *P = poly + 3 * e, *Q = poly + 3 * ((e + 1) % nv);
        double PQ[3], t[3], m[3];
        vsub(Q, P, PQ);
        double len = vnorm(PQ);
        for (int c = 0; c < 3; ++c) t[c] = PQ[c] / len;
        vcross(t, n, m);
        for (int s = 0; s < parts; ++s) {
            double s0 = (double)s / parts, s1 = (double)(s + 1) / parts;
            for (int g = 0; g < ng; ++g) {
                double sg = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * gt[g];
                double wg = 0.5 * (s1 - s0) * gw[g] * len;
                double y[3], d[3];
                for (int c = 0; c < 3; ++c) y[c] = P[c] + sg * PQ[c];
                vsub(y, x, d);
                double r = vnorm(d);
                cplx G = cexp(ik * r) / (4.0 * ORC_PI * r);
                cplx dGdr = G * (ik - 1.0 / r);
                sum += wg * dGdr * vdot(d, m) / r;
            }
        }
    }
    return sum;
}

void orc_edge_fp(const double *x, const double *n, const double *poly, int nv, double k,
                 int parts, int ng, double *out2)
{
    ensure_rules();
    cplx g = edge_fp(x, n, poly, nv, k, parts, ng);
    out2[0] = creal(g);
    out2[1] = cimag(g);
}

/* ------------------------------------------------------------------------ */
/* Element integrals of (G, H, H', E) of element (a, b, c) with normal ny at */
/* point x with normal nx.                                                   */
/* ------------------------------------------------------------------------ */
static void tri_geom(const double *a, const double *b, const double *c, double *cen, double *area)
{
    double ab[3], ac[3], cr[3];
    vsub(b, a, ab);
    vsub(c, a, ac);
    vcross(ab, ac, cr);
    *area = 0.5 * vnorm(cr);
    for (int i = 0; i < 3; ++i) cen[i] = (a[i] + b[i] + c[i]) / 3.0;
}

/* self term, x = midpoint of the element (Sec. 3.1.1, 3.1.2) */
static void self_integrals(const double *x, const double *a, const double *b, const double *c,
                           const double *n, double k, const orc_params *P, cplx out[4])
{
    double hexa[18];
    for (int i = 0; i < 3; ++i) {
        hexa[0 + i] = a[i];
        hexa[3 + i] = 0.5 * (a[i] + b[i]);
        hexa[6 + i] = b[i];
        hexa[9 + i] = 0.5 * (b[i] + c[i]);
        hexa[12 + i] = c[i];
        hexa[15 + i] = 0.5 * (c[i] + a[i]);
    }
    double tri[9];
    for (int i = 0; i < 3; ++i) { tri[i] = a[i]; tri[3 + i] = b[i]; tri[6 + i] = c[i]; }
    cplx G = duffy_G(x, hexa, 6, k, P->n_duffy);
    cplx Ee = edge_fp(x, n, tri, 3, k, P->edge_parts, P->edge_gauss);
    out[0] = G;
    out[1] = 0.0;           /* (y - x) is orthogonal to n on a flat element */
    out[2] = 0.0;
    out[3] = Ee + k * k * G;
}

/* regular and quasi-singular terms (Sec. 3.1.3, 3.1.4); returns 0 or -1 when
 * the subdivision would exceed max_depth levels */
static int regular_integrals(const double *x, const double *nx, const double *a, const double *b,
                             const double *c, const double *ny, double k, int depth,
                             const orc_params *P, cplx acc[4])
{
    double cen[3], area, d[3];
    tri_geom(a, b, c, cen, &area);
    vsub(x, cen, d);
    double rt = vnorm(d) / sqrt(area);
    if (rt < P->rt_subdiv) {
        if (depth >= P->max_depth) return -1;
        double mab[3], mbc[3], mca[3];
        for (int i = 0; i < 3; ++i) {
            mab[i] = 0.5 * (a[i] + b[i]);
            mbc[i] = 0.5 * (b[i] + c[i]);
            mca[i] = 0.5 * (c[i] + a[i]);
        }
        if (regular_integrals(x, nx, a, mab, mca, ny, k, depth + 1, P, acc)) return -1;
        if (regular_integrals(x, nx, mab, b, mbc, ny, k, depth + 1, P, acc)) return -1;
        if (regular_integrals(x, nx, mca, mbc, c, ny, k, depth + 1, P, acc)) return -1;
        if (regular_integrals(x, nx, mab, mbc, mca, ny, k, depth + 1, P, acc)) return -1;
        return 0;
    }
    int m = orc_quad_order(rt, P->quad_tol, P->m_max);
    const double *xi = tr_xi[m], *eta = tr_eta[m], *w = tr_w[m];
    double ab[3], ac[3];
    vsub(b, a, ab);
    vsub(c, a, ac);
    for (int q = 0; q < m * m; ++q) {
        double y[3];
        for (int i = 0; i < 3; ++i) y[i] = a[i] + xi[q] * ab[i] + eta[q] * ac[i];
        cplx kv[4];
        kernels(x, nx, y, ny, k, kv);
        double wq = 2.0 * area * w[q];
        for (int t = 0; t < 4; ++t) acc[t] += wq * kv[t];
    }
    return 0;
}

static int element_integrals(const double *x, const double *nx, const double *a, const double *b,
                             const double *c, const double *ny, int self, double k,
                             const orc_params *P, cplx out[4])
{
    if (self) { self_integrals(x, a, b, c, ny, k, P, out); return 0; }
    for (int t = 0; t < 4; ++t) out[t] = 0.0;
    return regular_integrals(x, nx, a, b, c, ny, k, 0, P, out);
}

/* Integrals of (G, H, H', E) over triangle (a,b,c) at x.  self != 0 means x
 * is the triangle's midpoint (singular rules).  params: NULL or 7 doubles. */
int orc_element_integrals(const double *x, const double *nx, const double *a, const double *b,
                          const double *c, int self, double k, const double *params, double *out8)
{
    ensure_rules();
    orc_params P;
    read_params(params, &P);
    double ab[3], ac[3], cr[3], ny[3];
    vsub(b, a, ab);
    vsub(c, a, ac);
    vcross(ab, ac, cr);
    double l = vnorm(cr);
    for (int i = 0; i < 3; ++i) ny[i] = cr[i] / l;
    cplx o[4];
    int st = element_integrals(x, nx, a, b, c, ny, self, k, &P, o);
    for (int i = 0; i < 4; ++i) { out8[2 * i] = creal(o[i]); out8[2 * i + 1] = cimag(o[i]); }
    return st;
}

/* ------------------------------------------------------------------------ */
/* Mesh geometry (Sec. 2.3, App. A): outward normal from counter-clockwise   */
/* vertex order, area, midpoint = mean of the vertices.                      */
/* ------------------------------------------------------------------------ */
void orc_geometry(const double *nodes, const int *tris, long n, double *cen, double *nrm, double *area)
{
    for (long j = 0; j < n; ++j) {
        const double *a = nodes + 3 * tris[3 * j], *b = nodes + 3 * tris[3 * j + 1],
                     *c = nodes + 3 * tris[3 * j + 2];
        double ab[3], ac[3], cr[3];
        vsub(b, a, ab);
        vsub(c, a, ac);
        vcross(ab, ac, cr);
        double l = vnorm(cr);
        area[j] = 0.5 * l;
        for (int i = 0; i < 3; ++i) {
            nrm[3 * j + i] = cr[i] / l;
            cen[3 * j + i] = (a[i] + b[i] + c[i]) / 3.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One row of the Burton-Miller system (Eq. SystemI, tau = 1):               */
/*   A_ij = cp_j * ( -(H_ij - gamma E_ij) ) + cq_j * ( G_ij - gamma H'_ij )  */
/*        + delta_ij * (cp_i - gamma cq_i) / 2,        gamma = i/k.          */
/* cp_j, cq_j say how the column's unknown enters as surface pressure p and  */
/* as normal derivative q = dp/dn (e.g. a sound-hard or admittance element   */
/* with unknown p has cp = 1, cq = -ik beta; a pressure element with unknown */
/* q has cp = 0, cq = 1).                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *nodes;
    const int *tris;
    long n;
    double *cen, *nrm;
    double k;
    const cplx *cp, *cq;
    orc_params P;
} mesh_ctx;

static int row_entry(const mesh_ctx *M, long i, long j, cplx *aij)
{
    const double *a = M->nodes + 3 * M->tris[3 * j], *b = M->nodes + 3 * M->tris[3 * j + 1],
                 *c = M->nodes + 3 * M->tris[3 * j + 2];
    cplx o[4];
    if (element_integrals(M->cen + 3 * i, M->nrm + 3 * i, a, b, c, M->nrm + 3 * j, i == j, M->k,
                          &M->P, o))
        return -1;
    cplx gamma = I / M->k;
    /* Eq. SystemI: tau on every integral operator, not on the identity halves */
    cplx v = M->P.tau * (M->cp[j] * (-(o[1] - gamma * o[3])) + M->cq[j] * (o[0] - gamma * o[2]));
    if (i == j) v += 0.5 * (M->cp[i] - gamma * M->cq[i]);
    *aij = v;
    return 0;
}

static void ctx_init(mesh_ctx *M, const double *nodes, const int *tris, long n, double k,
                     const double *cp, const double *cq, const double *params)
{
    M->nodes = nodes;
    M->tris = tris;
    M->n = n;
    M->k = k;
    M->cen = (double *)malloc(sizeof(double) * 3 * n);
    M->nrm = (double *)malloc(sizeof(double) * 3 * n);
    double *area = (double *)malloc(sizeof(double) * n);
    orc_geometry(nodes, tris, n, M->cen, M->nrm, area);
    free(area);
    M->cp = (const cplx *)cp;
    M->cq = (const cplx *)cq;
    read_params(params, &M->P);
}

static void ctx_free(mesh_ctx *M)
{
    free(M->cen);
    free(M->nrm);
}

/* Dense assembly of A (row-major, n*n complex).  Returns 0, or -1 with
 * *bad_elem = index of the element whose subdivision exceeded the limit
 * (Sec. 4.1 error message). */
int orc_assemble(const double *nodes, const int *tris, long n, double k, const double *cp,
                 const double *cq, const double *params, double *A, long *bad_elem)
{
    ensure_rules();
    mesh_ctx M;
    ctx_init(&M, nodes, tris, n, k, cp, cq, params);
    long bad = -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; ++i) {
        for (long j = 0; j < n; ++j) {
            cplx v = 0.0;
            if (row_entry(&M, i, j, &v)) {
#pragma omp critical
                { if (bad < 0 || j < bad) bad = j; }
            }
            A[2 * (i * n + j)] = creal(v);
            A[2 * (i * n + j) + 1] = cimag(v);
        }
    }
    ctx_free(&M);
    if (bad_elem) *bad_elem = bad;
    return bad >= 0 ? -1 : 0;
}

/* y_r = sum_j A_{rj} x_j for the listed rows, entries computed on the fly. */
int orc_matvec_rows(const double *nodes, const int *tris, long n, double k, const double *cp,
                    const double *cq, const double *params, const double *x, const long *rows,
                    long nrows, double *y, long *bad_elem)
{
    ensure_rules();
    mesh_ctx M;
    ctx_init(&M, nodes, tris, n, k, cp, cq, params);
    const cplx *xv = (const cplx *)x;
    long bad = -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < nrows; ++r) {
        long i = rows[r];
        cplx s = 0.0;
        for (long j = 0; j < n; ++j) {
            cplx v = 0.0;
            if (row_entry(&M, i, j, &v)) {
#pragma omp critical
                { if (bad < 0 || j < bad) bad = j; }
            }
            s += v * xv[j];
        }
        y[2 * r] = creal(s);
        y[2 * r + 1] = cimag(s);
    }
    ctx_free(&M);
    if (bad_elem) *bad_elem = bad;
    return bad >= 0 ? -1 : 0;
}

/* y = A x for a dense row-major complex A */
void orc_matvec_dense(const double *A, long n, const double *x, double *y)
{
    const cplx *Av = (const cplx *)A, *xv = (const cplx *)x;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        cplx s = 0.0;
        for (long j = 0; j < n; ++j) s += Av[i * n + j] * xv[j];
        y[2 * i] = creal(s);
        y[2 * i + 1] = cimag(s);
    }
}

/* y = A x for a dense row-major complex block A of `rows` x n */
void orc_matvec_block(const double *A, long rows, long n, const double *x, double *y)
{
    const cplx *Av = (const cplx *)A, *xv = (const cplx *)x;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < rows; ++i) {
        cplx s = 0.0;
        for (long j = 0; j < n; ++j) s += Av[i * n + j] * xv[j];
        y[2 * i] = creal(s);
        y[2 * i + 1] = cimag(s);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES(restart) on a dense complex system, x0 = 0, Arnoldi with  */
/* modified Gram-Schmidt and complex Givens rotations.  Stops when           */
/* ||b - A x|| / ||b|| <= tol (estimated from the Givens residual) or after  */
/* maxit matrix-vector products.  Returns 0 converged, 1 not converged.      */
/* ------------------------------------------------------------------------ */
int orc_gmres(const double *A, long n, const double *b, double *x, double tol, int maxit,
              int restart, int *iters, double *relres)
{
    const cplx *bv = (const cplx *)b;
    cplx *xv = (cplx *)x;
    int m = restart;
    cplx *V = (cplx *)malloc(sizeof(cplx) * (size_t)n * (m + 1));
    cplx *Hm = (cplx *)calloc((size_t)(m + 1) * m, sizeof(cplx));
    cplx *cs = (cplx *)malloc(sizeof(cplx) * m), *sn = (cplx *)malloc(sizeof(cplx) * m);
    cplx *g = (cplx *)malloc(sizeof(cplx) * (m + 1));
    cplx *w = (cplx *)malloc(sizeof(cplx) * n), *yv = (cplx *)malloc(sizeof(cplx) * m);
    double bn = 0.0;
    for (long i = 0; i < n; ++i) { xv[i] = 0.0; bn += creal(bv[i] * conj(bv[i])); }
    bn = sqrt(bn);
    int it = 0, status = 1;
    double rr = 1.0;
    if (bn == 0.0) { *iters = 0; *relres = 0.0; status = 0; goto done; }
    while (it < maxit) {
        /* r = b - A x */
        orc_matvec_dense(A, n, x, (double *)w);
        double beta = 0.0;
        for (long i = 0; i < n; ++i) { w[i] = bv[i] - w[i]; beta += creal(w[i] * conj(w[i])); }
        beta = sqrt(beta);
        rr = beta / bn;
        if (rr <= tol) { status = 0; break; }
        for (long i = 0; i < n; ++i) V[i] = w[i] / beta;
        memset(g, 0, sizeof(cplx) * (m + 1));
        g[0] = beta;
        int j;
        for (j = 0; j < m && it < maxit; ++j) {
            ++it;
            orc_matvec_dense(A, n, (const double *)(V + (size_t)j * n), (double *)w);
            for (int l = 0; l <= j; ++l) {
                cplx h = 0.0;
                const cplx *vl = V + (size_t)l * n;
                for (long i = 0; i < n; ++i) h += conj(vl[i]) * w[i];
                for (long i = 0; i < n; ++i) w[i] -= h * vl[i];
                Hm[l * m + j] = h;
            }
            double hn = 0.0;
            for (long i = 0; i < n; ++i) hn += creal(w[i] * conj(w[i]));
            hn = sqrt(hn);
            Hm[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (long i = 0; i < n; ++i) V[(size_t)(j + 1) * n + i] = w[i] / hn;
            /* apply previous rotations to column j */
            for (int l = 0; l < j; ++l) {
                cplx h0 = Hm[l * m + j], h1 = Hm[(l + 1) * m + j];
                Hm[l * m + j] = conj(cs[l]) * h0 + conj(sn[l]) * h1;
                Hm[(l + 1) * m + j] = -sn[l] * h0 + cs[l] * h1;
            }
            /* new rotation zeroing H[j+1][j] */
            cplx h0 = Hm[j * m + j], h1 = Hm[(j + 1) * m + j];
            double den = sqrt(creal(h0 * conj(h0)) + creal(h1 * conj(h1)));
            if (den == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = h0 / den; sn[j] = h1 / den; }
            Hm[j * m + j] = conj(cs[j]) * h0 + conj(sn[j]) * h1;
            Hm[(j + 1) * m + j] = 0.0;
            cplx g0 = g[j];
            g[j] = conj(cs[j]) * g0;
            g[j + 1] = -sn[j] * g0;
            rr = cabs(g[j + 1]) / bn;
            if (rr <= tol || hn == 0.0) { ++j; break; }
        }
        /* back substitution and update x */
        for (int l = j - 1; l >= 0; --l) {
            cplx s = g[l];
            for (int c = l + 1; c < j; ++c) s -= Hm[l * m + c] * yv[c];
            yv[l] = s / Hm[l * m + l];
        }
        for (int l = 0; l < j; ++l)
            for (long i = 0; i < n; ++i) xv[i] += yv[l] * V[(size_t)l * n + i];
        /* the loop head recomputes the true residual and decides */
    }
    if (status != 0) {
        orc_matvec_dense(A, n, x, (double *)w);
        double t = 0.0;
        for (long i = 0; i < n; ++i) { cplx d = bv[i] - w[i]; t += creal(d * conj(d)); }
        rr = sqrt(t) / bn;
        if (rr <= tol) status = 0;
    }
    *iters = it;
    *relres = rr;
done:
    free(V); free(Hm); free(cs); free(sn); free(g); free(w); free(yv);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Incident fields (Sec. 2.4, App. C.4), in pressure: plane wave            */
/* p = P0 e^{ik d.x}; point source p = P0 e^{ik R} / (4 pi R), R = |x - x0|. */
/* Writes p and dp/dn at x with normals nx (nx may be NULL: dp/dn skipped).  */
/* kind 0 = plane wave (v = direction), 1 = point source (v = position).     */
/* ------------------------------------------------------------------------ */
void orc_incident(const double *x, const double *nx, long npts, double k, int kind,
                  const double *v, const double *amp, double *p_out, double *dp_out)
{
    cplx P0 = amp[0] + I * amp[1];
    for (long i = 0; i < npts; ++i) {
        const double *xi = x + 3 * i;
        cplx p, dp = 0.0;
        if (kind == 0) {
            p = P0 * cexp(I * k * vdot(v, xi));
            if (nx) dp = I * k * vdot(v, nx + 3 * i) * p;
        } else {
            double d[3];
            vsub(xi, v, d);
            double R = vnorm(d);
            p = P0 * cexp(I * k * R) / (4.0 * ORC_PI * R);
            if (nx) dp = p * (I * k - 1.0 / R) * vdot(d, nx + 3 * i) / R;
        }
        p_out[2 * i] = creal(p);
        p_out[2 * i + 1] = cimag(p);
        if (nx && dp_out) { dp_out[2 * i] = creal(dp); dp_out[2 * i + 1] = cimag(dp); }
    }
}

/* ------------------------------------------------------------------------ */
/* Scattered field at exterior points (Eq. BIE_I with lambda = 1, tau = 1):  */
/*   p_s(x) = sum_j [ H(x)_j p_j - G(x)_j q_j ],                             */
/* element integrals with the regular / quasi-singular rules, r~ measured    */
/* from x.  Returns 0 or -1 (subdivision limit) with *bad_elem.              */
/* ------------------------------------------------------------------------ */
int orc_field(const double *nodes, const int *tris, long n, double k, const double *p,
              const double *q, const double *params, const double *pts, long npts, double *out,
              long *bad_elem)
{
    ensure_rules();
    orc_params P;
    read_params(params, &P);
    double *cen = (double *)malloc(sizeof(double) * 3 * n), *nrm = (double *)malloc(sizeof(double) * 3 * n),
           *area = (double *)malloc(sizeof(double) * n);
    orc_geometry(nodes, tris, n, cen, nrm, area);
    const cplx *pv = (const cplx *)p, *qv = (const cplx *)q;
    long bad = -1;
    double nx0[3] = {0.0, 0.0, 1.0}; /* H' and E are not used here */
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < npts; ++r) {
        cplx s = 0.0;
        for (long j = 0; j < n; ++j) {
            const double *a = nodes + 3 * tris[3 * j], *b = nodes + 3 * tris[3 * j + 1],
                         *c = nodes + 3 * tris[3 * j + 2];
            cplx o[4] = {0.0, 0.0, 0.0, 0.0};
            if (regular_integrals(pts + 3 * r, nx0, a, b, c, nrm + 3 * j, k, 0, &P, o)) {
#pragma omp critical
                { if (bad < 0 || j < bad) bad = j; }
            }
            s += o[1] * pv[j] - o[0] * qv[j];
        }
        s *= P.tau;
        out[2 * r] = creal(s);
        out[2 * r + 1] = cimag(s);
    }
    free(cen); free(nrm); free(area);
    if (bad_elem) *bad_elem = bad;
    return bad >= 0 ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* The element integrals of the representation formula (Eq. BIE_I with      */
/* lambda = 1) as dense matrices, Gm[r][j] = G(x_r)_j and Hm[r][j] = H(x_r)_j */
/* (row-major [npts][n] complex), without the tau sign: the field is         */
/* p_inc + tau (Hm p - Gm q).  Same rules as orc_field.  Used by the adjoint  */
/* gradient, which needs the transposed field operator.  Returns 0 or -1     */
/* (subdivision limit) with *bad_elem.                                       */
/* ------------------------------------------------------------------------ */
int orc_field_mats(const double *nodes, const int *tris, long n, double k, const double *params,
                   const double *pts, long npts, double *Gm, double *Hm, long *bad_elem)
{
    ensure_rules();
    orc_params P;
    read_params(params, &P);
    double *cen = (double *)malloc(sizeof(double) * 3 * n), *nrm = (double *)malloc(sizeof(double) * 3 * n),
           *area = (double *)malloc(sizeof(double) * n);
    orc_geometry(nodes, tris, n, cen, nrm, area);
    long bad = -1;
    double nx0[3] = {0.0, 0.0, 1.0}; /* H' and E are not used here */
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < npts; ++r) {
        for (long j = 0; j < n; ++j) {
            const double *a = nodes + 3 * tris[3 * j], *b = nodes + 3 * tris[3 * j + 1],
                         *c = nodes + 3 * tris[3 * j + 2];
            cplx o[4] = {0.0, 0.0, 0.0, 0.0};
            if (regular_integrals(pts + 3 * r, nx0, a, b, c, nrm + 3 * j, k, 0, &P, o)) {
#pragma omp critical
                { if (bad < 0 || j < bad) bad = j; }
            }
            size_t e = 2 * ((size_t)r * n + j);
            Gm[e] = creal(o[0]);
            Gm[e + 1] = cimag(o[0]);
            Hm[e] = creal(o[1]);
            Hm[e + 1] = cimag(o[1]);
        }
    }
    free(cen); free(nrm); free(area);
    if (bad_elem) *bad_elem = bad;
    return bad >= 0 ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient of the scattered field at exterior points, for the particle     */
/* velocity of Eq. utopandv (v = grad p / (i w rho)) that the paper writes   */
/* per field point (appendix Output): differentiating Eq. BIE_I (lambda = 1) */
/* under the integral (x is off the surface), the component along a unit     */
/* vector e is                                                               */
/*   e . grad p_s(x) = sum_j [ E(x)_j p_j - H'(x)_j q_j ],                   */
/* where H' = dG/dn_x and E = d2G/dn_x dn_y are the kernels of Eq. dBIE with */
/* n_x = e.  Same element rules as orc_field.  out: [npts][3] complex (the   */
/* x, y, z components).  Returns 0 or -1 (subdivision limit).                */
/* ------------------------------------------------------------------------ */
int orc_field_grad(const double *nodes, const int *tris, long n, double k, const double *p,
                   const double *q, const double *params, const double *pts, long npts, double *out,
                   long *bad_elem)
{
    ensure_rules();
    orc_params P;
    read_params(params, &P);
    double *cen = (double *)malloc(sizeof(double) * 3 * n), *nrm = (double *)malloc(sizeof(double) * 3 * n),
           *area = (double *)malloc(sizeof(double) * n);
    orc_geometry(nodes, tris, n, cen, nrm, area);
    const cplx *pv = (const cplx *)p, *qv = (const cplx *)q;
    long bad = -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < npts; ++r) {
        for (int ax = 0; ax < 3; ++ax) {
            double e[3] = {0.0, 0.0, 0.0};
            e[ax] = 1.0;
            cplx s = 0.0;
            for (long j = 0; j < n; ++j) {
                const double *a = nodes + 3 * tris[3 * j], *b = nodes + 3 * tris[3 * j + 1],
                             *c = nodes + 3 * tris[3 * j + 2];
                cplx o[4] = {0.0, 0.0, 0.0, 0.0};
                if (regular_integrals(pts + 3 * r, e, a, b, c, nrm + 3 * j, k, 0, &P, o)) {
#pragma omp critical
                    { if (bad < 0 || j < bad) bad = j; }
                }
                s += o[3] * pv[j] - o[2] * qv[j];
            }
            s *= P.tau;
            out[6 * r + 2 * ax] = creal(s);
            out[6 * r + 2 * ax + 1] = cimag(s);
        }
    }
    free(cen); free(nrm); free(area);
    if (bad_elem) *bad_elem = bad;
    return bad >= 0 ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Pieces of the plane-wave expansion (Sec. 3.3.1, Eq. FMMBase) -- used by   */
/* unit tests only.                                                          */
/* ------------------------------------------------------------------------ */

/* h_n^{(1)}(x), n = 0..nmax, by upward recursion h_{n+1} = (2n+1)/x h_n - h_{n-1}
 * from h_0 = -i e^{ix}/x and h_1 = -e^{ix}(x + i)/x^2 (Sec. 4.2). */
void orc_sph_hankel(int nmax, double x, double *out)
{
    cplx e = cexp(I * x);
    cplx h0 = -I * e / x, h1 = -e * (x + I) / (x * x);
    out[0] = creal(h0); out[1] = cimag(h0);
    if (nmax >= 1) { out[2] = creal(h1); out[3] = cimag(h1); }
    for (int n = 1; n < nmax; ++n) {
        cplx h2 = (2.0 * n + 1.0) / x * h1 - h0;
        out[2 * (n + 1)] = creal(h2);
        out[2 * (n + 1) + 1] = cimag(h2);
        h0 = h1;
        h1 = h2;
    }
}

/* Unit-sphere grid: L Gauss-Legendre nodes in cos(theta) times 2L equally
 * spaced azimuths phi_b = pi b / L; weights w = w_GL * pi / L (sum 4 pi).
 * s: 2L^2 x 3, w: 2L^2. */
int orc_sphere_grid(int L, double *s, double *w)
{
    double t[256], wt[256];
    if (L < 1 || L > 256) return -1;
    if (orc_gauss_legendre(L, t, wt)) return -1;
    int q = 0;
    for (int a = 0; a < L; ++a) {
        double st = sqrt(1.0 - t[a] * t[a]);
        for (int b = 0; b < 2 * L; ++b) {
            double ph = ORC_PI * b / L;
            s[3 * q] = st * cos(ph);
            s[3 * q + 1] = st * sin(ph);
            s[3 * q + 2] = t[a];
            w[q] = wt[a] * ORC_PI / L;
            ++q;
        }
    }
    return 0;
}

/* D_L(X, s) = sum_{n=0}^{L} i^n (2n+1) h_n(k|X|) P_n(X.s/|X|) for ns directions */
void orc_translation(int L, double k, const double *X, const double *s, int ns, double *out)
{
    double h[2 * 512];
    double R = vnorm(X);
    orc_sph_hankel(L, k * R, h);
    for (int v = 0; v < ns; ++v) {
        double t = vdot(X, s + 3 * v) / R;
        double p0 = 1.0, p1 = t;
        cplx in = 1.0, sum = 0.0;
        for (int n = 0; n <= L; ++n) {
            double pn = (n == 0) ? 1.0 : (n == 1 ? t : 0.0);
            if (n >= 2) {
                pn = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = pn;
            }
            sum += in * (2.0 * n + 1.0) * (h[2 * n] + I * h[2 * n + 1]) * pn;
            in *= I;
        }
        out[2 * v] = creal(sum);
        out[2 * v + 1] = cimag(sum);
    }
}

/* Single-pair expansion (Eq. FMMBase) of G(x, y) through the cluster
 * midpoints z1 (around x) and z2 (around y):
 *   G ~ (ik / 16 pi^2) sum_nu w_nu e^{ik (x - z1).s} D_L(z1 - z2, s) e^{ik (z2 - y).s}. */
int orc_fmm_pair(const double *x, const double *y, const double *z1, const double *z2, double k,
                 int L, double *out2)
{
    int ns = 2 * L * L;
    double *s = (double *)malloc(sizeof(double) * 3 * ns), *w = (double *)malloc(sizeof(double) * ns),
           *D = (double *)malloc(sizeof(double) * 2 * ns);
    if (orc_sphere_grid(L, s, w)) { free(s); free(w); free(D); return -1; }
    double X[3], dx[3], dy[3];
    vsub(z1, z2, X);
    vsub(x, z1, dx);
    vsub(z2, y, dy);
    orc_translation(L, k, X, s, ns, D);
    cplx sum = 0.0;
    for (int v = 0; v < ns; ++v) {
        cplx Sv = cexp(I * k * vdot(dx, s + 3 * v));
        cplx Tv = cexp(I * k * vdot(dy, s + 3 * v));
        sum += w[v] * Sv * (D[2 * v] + I * D[2 * v + 1]) * Tv;
    }
    sum *= I * k / (16.0 * ORC_PI * ORC_PI);
    out2[0] = creal(sum);
    out2[1] = cimag(sum);
    free(s); free(w); free(D);
    return 0;
}
