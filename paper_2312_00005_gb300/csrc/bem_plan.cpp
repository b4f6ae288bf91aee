// bem_plan.cpp -- host-side geometry, quadrature tables and cluster plan.
// See bem_plan.hpp for the paper sections each part follows.
#include "bem_plan.hpp"

#include <algorithm>
#include <cmath>
#include <complex>
#include <exception>
#include <functional>
#include <thread>
#include <unordered_map>
#include <cstdio>
#include <numeric>
#include <tuple>

namespace bem {

namespace {
// Runs fn(q) for q = 0 .. n - 1, on n threads when n > 1, and once every one
// has finished rethrows the first exception any of them raised, so that a
// failure in a worker (a host allocation) reaches the caller as it would from
// a serial run.  A thread that cannot be started runs its share, and the
// rest, on the calling thread.
template <typename F>
void run_parallel(int n, F &&fn)
{
    if (n <= 1) {
        fn(0);
        return;
    }
    std::vector<std::exception_ptr> err(n);
    auto body = [&](int q) {
        try {
            fn(q);
        } catch (...) {
            err[q] = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    th.reserve(n);
    for (int q = 0; q < n; ++q) {
        try {
            th.emplace_back(body, q);
        } catch (...) {
            for (int r = q; r < n; ++r) body(r);
            break;
        }
    }
    for (auto &t : th) t.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
}

inline void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
inline double norm3(const double *a) { return std::sqrt(dot3(a, a)); }
}  // namespace

// ------------------------------------------------------------------ geometry
std::string compute_geometry(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n,
                             Geometry &g)
{
    g.n = n;
    g.cen.assign(3 * n, 0.0);
    g.nrm.assign(3 * n, 0.0);
    g.area.assign(n, 0.0);
    g.va.assign(3 * n, 0.0);
    g.e1.assign(3 * n, 0.0);
    g.e2.assign(3 * n, 0.0);
    g.vrad.assign(n, 0.0);
    g.vmin.assign(3, 1e300);
    g.vmax.assign(3, -1e300);
    double edge_sum = 0.0;
    g.max_area = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        int32_t ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= n_nodes || ib >= n_nodes || ic >= n_nodes) {
            char buf[128];
            snprintf(buf, sizeof buf, "element %lld has a node index out of range", (long long)j);
            return buf;
        }
        const double *a = nodes + 3 * ia, *b = nodes + 3 * ib, *c = nodes + 3 * ic;
        double ab[3], ac[3], bc[3], cr[3];
        sub3(b, a, ab);
        sub3(c, a, ac);
        sub3(c, b, bc);
        cross3(ab, ac, cr);
        double l = norm3(cr);
        if (!(l > 0.0) || !std::isfinite(l)) {
            char buf[128];
            snprintf(buf, sizeof buf, "element %lld is degenerate (zero area)", (long long)j);
            return buf;
        }
        g.area[j] = 0.5 * l;
        g.max_area = std::max(g.max_area, g.area[j]);
        for (int i = 0; i < 3; ++i) {
            g.nrm[3 * j + i] = cr[i] / l;
            g.cen[3 * j + i] = (a[i] + b[i] + c[i]) / 3.0;
            g.e1[3 * j + i] = ab[i];
            g.e2[3 * j + i] = ac[i];
        }
        for (int i = 0; i < 3; ++i) g.va[3 * j + i] = a[i] - g.cen[3 * j + i];
        const double *vs[3] = {a, b, c};
        double vr = 0.0;
        for (int v = 0; v < 3; ++v) {
            double d[3];
            sub3(vs[v], &g.cen[3 * j], d);
            vr = std::max(vr, norm3(d));
            for (int i = 0; i < 3; ++i) {
                g.vmin[i] = std::min(g.vmin[i], vs[v][i]);
                g.vmax[i] = std::max(g.vmax[i], vs[v][i]);
            }
        }
        g.vrad[j] = vr;
        edge_sum += norm3(ab) + norm3(ac) + norm3(bc);
    }
    g.mean_edge = n ? edge_sum / (3.0 * n) : 0.0;
    return "";
}

// ------------------------------------------------------------------ Golub-Welsch
// Eigen-decomposition of a small symmetric matrix by cyclic Jacobi rotations.
static void sym_eig(int n, std::vector<double> &A, std::vector<double> &V)
{
    V.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-34) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double theta = 0.5 * (aqq - app) / apq;
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
}

// Nodes/weights on [-1,1] from recurrence coefficients (diag a_k, offdiag b_k)
// and the moment mu0 of the weight.
static void golub_welsch(int n, const std::vector<double> &a, const std::vector<double> &b, double mu0,
                         std::vector<double> &x, std::vector<double> &w)
{
    std::vector<double> J(n * n, 0.0), V;
    for (int i = 0; i < n; ++i) J[i * n + i] = a[i];
    for (int i = 0; i + 1 < n; ++i) J[i * n + i + 1] = J[(i + 1) * n + i] = b[i];
    sym_eig(n, J, V);
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int p, int q) { return J[p * n + p] < J[q * n + q]; });
    x.resize(n);
    w.resize(n);
    for (int r = 0; r < n; ++r) {
        int c = idx[r];
        x[r] = J[c * n + c];
        w[r] = mu0 * V[0 * n + c] * V[0 * n + c];
    }
}

void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w)
{
    std::vector<double> a(n, 0.0), b(n > 1 ? n - 1 : 0);
    for (int k = 1; k < n; ++k) b[k - 1] = k / std::sqrt(4.0 * k * k - 1.0);
    golub_welsch(n, a, b, 2.0, x, w);
    for (int i = 0; i < n; ++i) { x[i] = 0.5 * (x[i] + 1.0); w[i] *= 0.5; }
}

void gauss_jacobi10_01(int n, std::vector<double> &x, std::vector<double> &w)
{
    // Jacobi alpha = 1, beta = 0 on [-1,1] (weight 1 - t):
    //   a_k = (beta^2 - alpha^2) / ((2k+s)(2k+s+2)), s = alpha + beta
    //   b_k = sqrt(4k(k+alpha)(k+beta)(k+s) / ((2k+s)^2 (2k+s+1)(2k+s-1)))
    const double al = 1.0, be = 0.0, s = al + be;
    std::vector<double> a(n), b(n > 1 ? n - 1 : 0);
    for (int k = 0; k < n; ++k) a[k] = (be * be - al * al) / ((2.0 * k + s) * (2.0 * k + s + 2.0));
    for (int k = 1; k < n; ++k) {
        double t = 2.0 * k + s;
        b[k - 1] = std::sqrt(4.0 * k * (k + al) * (k + be) * (k + s) / (t * t * (t + 1.0) * (t - 1.0)));
    }
    golub_welsch(n, a, b, 2.0, x, w);
    // u = (t + 1)/2, (1 - u) = (1 - t)/2, du = dt/2  =>  w_u = w_t / 4
    for (int i = 0; i < n; ++i) { x[i] = 0.5 * (x[i] + 1.0); w[i] *= 0.25; }
}

void conical_rule(int m, std::vector<double> &xi, std::vector<double> &eta, std::vector<double> &w)
{
    std::vector<double> uj, wj, vl, wl;
    gauss_jacobi10_01(m, uj, wj);
    gauss_legendre01(m, vl, wl);
    xi.clear(); eta.clear(); w.clear();
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            xi.push_back(uj[a]);
            eta.push_back((1.0 - uj[a]) * vl[b]);
            w.push_back(wj[a] * wl[b]);
        }
}

void order_thresholds(double tol, int m_max, double *R)
{
    // eps_G = 32 q^(2m+1), eps_H = 64 (2m+1) q^(2m+2),
    // eps_E = 128 (m+1)(2m+1) q^(2m+3), q = 1 / (2 r~): each is below tol
    // exactly when r~ exceeds 1 / (2 q*), q* the root of eps = tol.
    for (int m = 1; m < m_max; ++m) {
        double qG = std::pow(tol / 32.0, 1.0 / (2.0 * m + 1.0));
        double qH = std::pow(tol / (64.0 * (2.0 * m + 1.0)), 1.0 / (2.0 * m + 2.0));
        double qE = std::pow(tol / (128.0 * (m + 1.0) * (2.0 * m + 1.0)), 1.0 / (2.0 * m + 3.0));
        double q = std::min(qG, std::min(qH, qE));
        R[m] = 0.5 / q;
    }
}

void sphere_grid(int L, std::vector<double> &s, std::vector<double> &w)
{
    std::vector<double> t, wt;
    gauss_legendre01(L, t, wt);      // on [0,1]: cos(theta) = 2t - 1, weight 2 wt
    // cos(theta) nodes and weights made exactly symmetric about 0
    std::vector<double> ct(L), wc(L);
    for (int a = 0; a < L; ++a) {
        ct[a] = 2.0 * t[a] - 1.0;
        wc[a] = 2.0 * wt[a];
    }
    for (int a = 0; a < L / 2; ++a) {
        const int b = L - 1 - a;
        const double m = 0.5 * (ct[b] - ct[a]), v = 0.5 * (wc[a] + wc[b]);
        ct[a] = -m;
        ct[b] = m;
        wc[a] = wc[b] = v;
    }
    if (L % 2) ct[L / 2] = 0.0;
    const int half = L * L;
    s.resize(3 * 2 * half);
    w.resize(2 * half);
    int q = 0;
    auto put = [&](int a, int b) {
        const double st = std::sqrt(std::max(0.0, 1.0 - ct[a] * ct[a]));
        const double ph = M_PI * b / L;
        s[3 * q] = st * std::cos(ph);
        s[3 * q + 1] = st * std::sin(ph);
        s[3 * q + 2] = ct[a];
        w[q] = wc[a] * M_PI / L;
        // the antipode -s_q (theta -> pi - theta, phi -> phi + pi)
        for (int c = 0; c < 3; ++c) s[3 * (q + half) + c] = -s[3 * q + c];
        w[q + half] = w[q];
        ++q;
    };
    for (int a = 0; a < L / 2; ++a)
        for (int b = 0; b < 2 * L; ++b) put(a, b);
    if (L % 2)
        for (int b = 0; b < L; ++b) put(L / 2, b);
}

double hankel_growth(double x, int L)
{
    std::complex<double> I(0.0, 1.0), e = std::exp(I * x);
    std::complex<double> h0 = -I * e / x, h1 = -e * (x + I) / (x * x);
    double a0 = std::abs(h0), sum = a0;
    if (L >= 1) sum += 3.0 * std::abs(h1);
    for (int n = 1; n < L; ++n) {
        std::complex<double> h2 = (2.0 * n + 1.0) / x * h1 - h0;
        sum += (2.0 * n + 3.0) * std::abs(h2);
        h0 = h1;
        h1 = h2;
        if (!std::isfinite(sum)) return 1e300;
    }
    return sum / a0;
}

// ------------------------------------------------------------------ tree
static inline uint64_t spread3(uint64_t v)
{
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

double auto_leaf_edge(const Geometry &g, const bem_params &p)
{
    // Far pairs must keep every element pair at the regular order m = 1
    // (the centroid rule of the far field), i.e. midpoint distances above
    // R_1 sqrt(A_max).  Leaves a fifth of that radius keep the near field
    // close to its minimum without crowding the interaction lists.
    double R[kMaxRule + 1] = {0};
    order_thresholds(p.quad_tol, std::max(2, p.m_max), R);
    double r1 = R[1] * std::sqrt(g.max_area);
    return std::max(r1 / 5.0, 2.0 * g.mean_edge);
}

void build_tree(const Geometry &g, double leaf_edge, Tree &t)
{
    const int64_t n = g.n;
    double ext = 0.0;
    for (int i = 0; i < 3; ++i) ext = std::max(ext, g.vmax[i] - g.vmin[i]);
    ext *= 1.0 + 1e-9;
    if (ext <= 0) ext = 1.0;
    for (int i = 0; i < 3; ++i) t.origin[i] = 0.5 * (g.vmin[i] + g.vmax[i]) - 0.5 * ext;
    t.edge = ext;
    int depth = 0;
    if (leaf_edge > 0) depth = (int)std::lround(std::log2(ext / leaf_edge));
    depth = std::max(0, std::min(depth, 20));
    t.leaf_depth = depth;
    const int64_t side = (int64_t)1 << depth;
    const double box = ext / side;
    std::vector<uint64_t> code(n);
    std::vector<int32_t> bx(3 * n);
    for (int64_t j = 0; j < n; ++j) {
        for (int i = 0; i < 3; ++i) {
            int64_t b = (int64_t)std::floor((g.cen[3 * j + i] - t.origin[i]) / box);
            b = std::max<int64_t>(0, std::min<int64_t>(side - 1, b));
            bx[3 * j + i] = (int32_t)b;
        }
        code[j] = spread3(bx[3 * j]) | (spread3(bx[3 * j + 1]) << 1) | (spread3(bx[3 * j + 2]) << 2);
    }
    t.perm.resize(n);
    std::iota(t.perm.begin(), t.perm.end(), 0);
    std::stable_sort(t.perm.begin(), t.perm.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
    t.lv.assign(depth + 1, Level());
    for (int d = 0; d <= depth; ++d) {
        Level &L = t.lv[d];
        L.depth = d;
        L.box = ext / (double)((int64_t)1 << d);
        L.elem_cluster.assign(n, -1);
        int shift = 3 * (depth - d);
        int64_t i = 0;
        while (i < n) {
            uint64_t key = code[t.perm[i]] >> shift;
            int64_t j = i;
            while (j < n && (code[t.perm[j]] >> shift) == key) ++j;
            int32_t c = (int32_t)L.start.size();
            L.start.push_back(i);
            L.count.push_back(j - i);
            int64_t e0 = t.perm[i];
            int sh = depth - d;
            L.ix.push_back(bx[3 * e0] >> sh);
            L.iy.push_back(bx[3 * e0 + 1] >> sh);
            L.iz.push_back(bx[3 * e0 + 2] >> sh);
            double z[3] = {t.origin[0] + (L.ix.back() + 0.5) * L.box, t.origin[1] + (L.iy.back() + 0.5) * L.box,
                           t.origin[2] + (L.iz.back() + 0.5) * L.box};
            double rad = 0.0, crad = 0.0, amax = 0.0;
            for (int64_t q = i; q < j; ++q) {
                int64_t e = t.perm[q];
                L.elem_cluster[q] = c;
                double d3[3];
                sub3(&g.cen[3 * e], z, d3);
                double dc = norm3(d3);
                crad = std::max(crad, dc);
                rad = std::max(rad, dc + g.vrad[e]);
                amax = std::max(amax, g.area[e]);
            }
            // vertex radius: exact maximum over the three vertices
            rad = 0.0;
            for (int64_t q = i; q < j; ++q) {
                int64_t e = t.perm[q];
                for (int v = 0; v < 3; ++v) {
                    double vx[3];
                    for (int k = 0; k < 3; ++k) {
                        double base = g.cen[3 * e + k] + g.va[3 * e + k];
                        if (v == 1) base += g.e1[3 * e + k];
                        if (v == 2) base += g.e2[3 * e + k];
                        vx[k] = base - z[k];
                    }
                    rad = std::max(rad, norm3(vx));
                }
            }
            for (int k = 0; k < 3; ++k) L.z.push_back(z[k]);
            L.rad.push_back(rad);
            L.crad.push_back(crad);
            L.amax.push_back(amax);
            L.rmax = std::max(L.rmax, rad);
            i = j;
        }
    }
    // parent / children links (clusters are nested runs of the Morton order)
    for (int d = 0; d <= depth; ++d) {
        Level &L = t.lv[d];
        int nc = (int)L.start.size();
        L.parent.assign(nc, -1);
        L.child0.assign(nc, 0);
        L.nchild.assign(nc, 0);
        if (d > 0) {
            const Level &P = t.lv[d - 1];
            for (int c = 0; c < nc; ++c) L.parent[c] = P.elem_cluster[L.start[c]];
        }
    }
    for (int d = 0; d < depth; ++d) {
        Level &L = t.lv[d];
        const Level &C = t.lv[d + 1];
        int nc = (int)L.start.size();
        for (int c = 0; c < nc; ++c) { L.child0[c] = -1; L.nchild[c] = 0; }
        for (int c = 0; c < (int)C.start.size(); ++c) {
            int p = C.parent[c];
            if (L.child0[p] < 0) L.child0[p] = c;
            L.nchild[p]++;
        }
    }
}

// ------------------------------------------------------------------ plan
// Near and interaction lists by the recursion of Sec. 3.3.4 (stability_max
// >= 1e300 skips the Hankel-growth test: purely geometric lists): the candidates
// of a cluster at depth d are the children of its parent's near clusters;
// far candidates form its interaction list, the others its near list.  The
// far test depends on the pair only through the box offset (distance,
// Hankel growth) and the clusters' radii, so the offset-only parts are
// cached in a dense table per depth.
void build_plan(const Geometry &g, const Tree &t, const bem_params &p, double k, FreqPlan &fp, int leaf_depth)
{
    fp = FreqPlan();
    fp.k = k;
    fp.direct = (p.mode == BEM_MODE_DIRECT);
    const int D = (leaf_depth < 0 || leaf_depth > t.leaf_depth) ? t.leaf_depth : leaf_depth;
    fp.leaf_depth = D;
    double R[kMaxRule + 1] = {0};
    order_thresholds(p.quad_tol, std::max(2, p.m_max), R);
    const double r1 = R[1] * (1.0 + 1e-9);
    std::vector<int> Ld(D + 1, 0);
    for (int d = 0; d <= D; ++d) {
        double x = 2.0 * t.lv[d].rmax * k;
        double L = x + p.trunc_factor * std::log10(x + M_PI);
        Ld[d] = std::max(p.L_min, (int)std::ceil(L - 1e-12));
    }
    fp.Ld = Ld;
    // near lists of the previous depth in CSR form
    std::vector<int32_t> nprev_ptr{0, 1}, nprev{0};
    int rnear_prev = 0;                 // largest |offset component| among near pairs
    std::vector<FarLevel> far_all(D + 1);
    for (int d = 1; d <= D; ++d) {
        const Level &L = t.lv[d];
        const Level &P = t.lv[d - 1];
        const int nc = (int)L.start.size();
        FarLevel &F = far_all[d];
        F.depth = d;
        F.L = Ld[d];
        F.nc = nc;
        F.il_ptr.assign(nc + 1, 0);
        std::vector<double> r1sq(nc);
        for (int c = 0; c < nc; ++c) r1sq[c] = r1 * std::sqrt(L.amax[c]);
        const int Rb = 2 * rnear_prev + 1;           // candidate offsets lie in [-Rb, Rb]^3
        const int W = 2 * Rb + 1;
        // The clusters in contiguous ranges, scanned in parallel; each range
        // keeps its lists with far entries tagged by offset key, and the keys
        // in the order it first met them.  The merge below visits the ranges
        // in order, so offset rows and verdicts come out in the order of a
        // scan of the clusters one by one.
        struct Part {
            std::vector<int32_t> il_src, ncur, il_cnt, n_cnt;
            std::vector<int64_t> il_key;
            std::vector<int64_t> met;           // keys in the order first met
            std::vector<char> met_ok;           // their stability verdicts
            std::vector<int64_t> first_far;     // keys in the order of their first far use
            int rnear = 0;
        };
        const int nthr = nc >= 2048 ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
        std::vector<Part> parts(nthr);
        auto scan = [&](int c0, int c1, Part &pt) {
            // per offset: -2 unknown, -1 not far by offset (unstable), -3 far-capable
            std::vector<int8_t> st_loc((size_t)W * W * W, -2);
            std::vector<char> used_loc((size_t)W * W * W, 0);
            pt.il_cnt.assign(c1 - c0, 0);
            pt.n_cnt.assign(c1 - c0, 0);
            for (int c = c0; c < c1; ++c) {
                const int par = L.parent[c];
                int nfar = 0, nnear = 0;
                for (int q = nprev_ptr[par]; q < nprev_ptr[par + 1]; ++q) {
                    const int sp = nprev[q];
                    for (int s = P.child0[sp]; s < P.child0[sp] + P.nchild[sp]; ++s) {
                        const int dx = L.ix[c] - L.ix[s], dy = L.iy[c] - L.iy[s], dz = L.iz[c] - L.iz[s];
                        bool far = false;
                        int64_t key = -1;
                        if (!fp.direct && (dx | dy | dz) != 0) {
                            key = ((int64_t)(dx + Rb) * W + (dy + Rb)) * W + (dz + Rb);
                            int8_t &stl = st_loc[(size_t)key];
                            const double X[3] = {dx * L.box, dy * L.box, dz * L.box};
                            const double dist = norm3(X);
                            if (stl == -2) {
                                const bool ok = p.stability_max >= 1e300 || hankel_growth(k * dist, F.L) <= p.stability_max;
                                stl = ok ? -3 : -1;
                                pt.met.push_back(key);
                                pt.met_ok.push_back(ok ? 1 : 0);
                            }
                            if (stl != -1) {
                                // r~ of every element pair above R_1: bounded with the
                                // source cluster's largest area, or with the larger
                                // of both clusters' (symmetric_far: the same verdict
                                // both ways, so the lists have mirrors)
                                const double rb = p.symmetric_far ? std::max(r1sq[c], r1sq[s]) : r1sq[s];
                                far = dist > p.admissibility * (L.rad[c] + L.rad[s]) &&
                                      dist - L.crad[c] - L.crad[s] > rb;
                            }
                        }
                        if (far) {
                            pt.il_src.push_back(s);
                            pt.il_key.push_back(key);
                            if (!used_loc[(size_t)key]) {
                                used_loc[(size_t)key] = 1;
                                pt.first_far.push_back(key);
                            }
                            ++nfar;
                        } else {
                            pt.ncur.push_back(s);
                            pt.rnear = std::max(pt.rnear, std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))));
                            ++nnear;
                        }
                    }
                }
                pt.il_cnt[c - c0] = nfar;
                pt.n_cnt[c - c0] = nnear;
            }
        };
        std::vector<int> cut(nthr + 1);
        for (int q = 0; q <= nthr; ++q) cut[q] = (int)((int64_t)nc * q / nthr);
        run_parallel(nthr, [&](int q) { scan(cut[q], cut[q + 1], parts[q]); });
        // merge in cluster order: verdicts at the first meeting of each
        // offset and translation rows at its first far use (short lists,
        // serial), then every range's entries copied to their places
        std::vector<int32_t> off_row((size_t)W * W * W, -1);
        std::vector<char> seen((size_t)W * W * W, 0);
        int rnear = 0;
        std::vector<size_t> far_base(nthr + 1, 0), near_base(nthr + 1, 0);
        for (int q = 0; q < nthr; ++q) {
            const Part &pt = parts[q];
            rnear = std::max(rnear, pt.rnear);
            far_base[q + 1] = far_base[q] + pt.il_src.size();
            near_base[q + 1] = near_base[q] + pt.ncur.size();
            if (p.stability_max < 1e300)
                for (size_t u = 0; u < pt.met.size(); ++u) {
                    const int64_t key = pt.met[u];
                    if (seen[(size_t)key]) continue;
                    seen[(size_t)key] = 1;
                    const int ddz = (int)(key % W) - Rb, ddy = (int)((key / W) % W) - Rb,
                              ddx = (int)(key / ((int64_t)W * W)) - Rb;
                    fp.verdicts.push_back(Verdict{d, ddx, ddy, ddz, F.L, pt.met_ok[u] != 0});
                }
            for (const int64_t key : pt.first_far) {
                int32_t &row = off_row[(size_t)key];
                if (row >= 0) continue;
                const int ddz = (int)(key % W) - Rb, ddy = (int)((key / W) % W) - Rb,
                          ddx = (int)(key / ((int64_t)W * W)) - Rb;
                row = (int32_t)(F.offsets.size() / 3);
                F.offsets.push_back(ddx * L.box);
                F.offsets.push_back(ddy * L.box);
                F.offsets.push_back(ddz * L.box);
            }
        }
        std::vector<int32_t> ncur_ptr(nc + 1, 0), ncur(near_base[nthr]);
        std::vector<int32_t> il_src(far_base[nthr]), il_off(far_base[nthr]);
        auto place = [&](int q) {
            const Part &pt = parts[q];
            size_t fe = 0, ne = 0;
            for (int c = cut[q]; c < cut[q + 1]; ++c) {
                for (int u = 0; u < pt.il_cnt[c - cut[q]]; ++u, ++fe) {
                    il_src[far_base[q] + fe] = pt.il_src[fe];
                    il_off[far_base[q] + fe] = off_row[(size_t)pt.il_key[fe]];
                }
                for (int u = 0; u < pt.n_cnt[c - cut[q]]; ++u, ++ne) ncur[near_base[q] + ne] = pt.ncur[ne];
                F.il_ptr[c + 1] = (int32_t)(far_base[q] + fe);
                ncur_ptr[c + 1] = (int32_t)(near_base[q] + ne);
            }
        };
        run_parallel(nthr, place);
        F.il_src.swap(il_src);
        F.il_off.swap(il_off);
        F.n_inter = (int64_t)F.il_src.size();
        nprev_ptr.swap(ncur_ptr);
        nprev.swap(ncur);
        rnear_prev = rnear;
    }
    // leaf near lists (sorted source leaves): each leaf's sorted list takes
    // the places of its unsorted one, so the leaves sort in parallel
    const Level &Lf = t.lv[D];
    const int nl = (int)Lf.start.size();
    fp.near_ptr = nprev_ptr;
    fp.near_src = nprev;
    const int nthl = nl >= 2048 ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
    std::vector<int64_t> nnz_part(nthl, 0);
    auto sort_leaves = [&](int q) {
        const int c0 = (int)((int64_t)nl * q / nthl), c1 = (int)((int64_t)nl * (q + 1) / nthl);
        int64_t z = 0;
        for (int c = c0; c < c1; ++c) {
            const int b0 = fp.near_ptr[c], b1 = fp.near_ptr[c + 1];
            std::sort(fp.near_src.begin() + b0, fp.near_src.begin() + b1);
            int64_t cols = 0;
            for (int u = b0; u < b1; ++u) cols += Lf.count[fp.near_src[u]];
            z += cols * Lf.count[c];
        }
        nnz_part[q] = z;
    };
    run_parallel(nthl, sort_leaves);
    fp.nnz = 0;
    for (int64_t z : nnz_part) fp.nnz += z;
    for (int d = 1; d <= D; ++d)
        if (far_all[d].n_inter > 0) {
            fp.far.push_back(std::move(far_all[d]));
            fp.max_L = std::max(fp.max_L, fp.far.back().L);
        }
}

std::string validate_plan(const Tree &t, const FreqPlan &fp)
{
    if (fp.leaf_depth < 0 || fp.leaf_depth >= (int)t.lv.size()) return "leaf depth out of range";
    const Level &Lf = t.lv[fp.leaf_depth];
    const int nl = (int)Lf.start.size();
    if ((int)fp.near_ptr.size() != nl + 1 || fp.near_ptr[0] != 0) return "near list pointers of the wrong length";
    if ((size_t)fp.near_ptr[nl] != fp.near_src.size()) return "near list pointers do not end at the entries";
    int64_t nnz = 0;
    for (int c = 0; c < nl; ++c) {
        if (fp.near_ptr[c + 1] < fp.near_ptr[c]) return "near list pointers not monotone at leaf " + std::to_string(c);
        bool self = Lf.count[c] == 0;
        int64_t cols = 0;
        for (int q = fp.near_ptr[c]; q < fp.near_ptr[c + 1]; ++q) {
            const int s2 = fp.near_src[q];
            if (s2 < 0 || s2 >= nl) return "near list of leaf " + std::to_string(c) + " names leaf " + std::to_string(s2);
            self = self || s2 == c;
            cols += Lf.count[s2];
        }
        if (!self) return "leaf " + std::to_string(c) + " is not in its own near list";
        nnz += cols * Lf.count[c];
    }
    if (nnz != fp.nnz) return "near-field entry count disagrees with the lists";
    for (const FarLevel &F : fp.far) {
        if (F.depth < 1 || F.depth >= (int)t.lv.size()) return "far level depth out of range";
        const int nc = (int)t.lv[F.depth].start.size();
        if (F.nc != nc || (int)F.il_ptr.size() != nc + 1 || F.il_ptr[0] != 0)
            return "interaction list pointers of the wrong length at depth " + std::to_string(F.depth);
        if ((size_t)F.il_ptr[nc] != F.il_src.size() || F.il_src.size() != F.il_off.size())
            return "interaction list pointers do not end at the entries at depth " + std::to_string(F.depth);
        const int64_t noff = (int64_t)(F.offsets.size() / 3);
        if (F.offsets.size() % 3 != 0) return "translation offsets not in triples";
        for (int c = 0; c < nc; ++c)
            if (F.il_ptr[c + 1] < F.il_ptr[c]) return "interaction list pointers not monotone";
        for (size_t q = 0; q < F.il_src.size(); ++q) {
            if (F.il_src[q] < 0 || F.il_src[q] >= nc) return "interaction list names a cluster out of range";
            if (F.il_off[q] < 0 || F.il_off[q] >= noff) return "interaction list names a translation row out of range";
        }
    }
    return "";
}

namespace {
struct OffKey {
    int64_t x, y, z;
    bool operator==(const OffKey &o) const { return x == o.x && y == o.y && z == o.z; }
};
struct OffKeyHash {
    size_t operator()(const OffKey &k) const
    {
        uint64_t h = (uint64_t)k.x * 0x9E3779B97F4A7C15ULL;
        h ^= (uint64_t)k.y * 0xC2B2AE3D27D4EB4FULL + (h << 6) + (h >> 2);
        h ^= (uint64_t)k.z * 0x165667B19E3779F9ULL + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};
}  // namespace

std::string build_eval_plan(const Geometry &g, const Tree &t, const bem_params &p, double k, int leaf_depth,
                            const double *pts, int64_t m, int max_L, EvalPlan &ep)
{
    ep = EvalPlan();
    const int n_threads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int D = (leaf_depth < 0 || leaf_depth > t.leaf_depth) ? t.leaf_depth : leaf_depth;
    ep.leaf_depth = D;
    const double boxD = t.edge / (double)((int64_t)1 << D);
    // integer box coordinates at the leaf depth, shifted by B so that every
    // coarser depth's coordinate is a right shift (B divisible by 2^D)
    const int64_t B = (int64_t)1 << 20;
    std::vector<int64_t> U(3 * (size_t)m);
    std::vector<uint64_t> code(m);
    for (int64_t j = 0; j < m; ++j) {
        for (int i = 0; i < 3; ++i) {
            const double v = std::floor((pts[3 * j + i] - t.origin[i]) / boxD);
            if (!(v > (double)-B && v < (double)B))
                return "field point " + std::to_string(j) + " lies more than 2^20 leaf boxes from the mesh";
            U[3 * j + i] = (int64_t)v + B;
        }
        code[j] = spread3((uint64_t)U[3 * j]) | (spread3((uint64_t)U[3 * j + 1]) << 1) |
                  (spread3((uint64_t)U[3 * j + 2]) << 2);
    }
    {
        std::vector<std::pair<uint64_t, int64_t>> ci(m);
        for (int64_t j = 0; j < m; ++j) ci[j] = {code[j], j};
        std::sort(ci.begin(), ci.end());   // by code, then by caller index
        ep.perm.resize(m);
        for (int64_t j = 0; j < m; ++j) ep.perm[j] = ci[j].second;
    }
    // codes, coordinates and points in the sorted order (sequential access below)
    std::vector<uint64_t> scode(m);
    std::vector<int64_t> sU(3 * (size_t)m);
    std::vector<double> sp(3 * (size_t)m);
    for (int64_t i = 0; i < m; ++i) {
        const int64_t e = ep.perm[i];
        scode[i] = code[e];
        for (int a = 0; a < 3; ++a) {
            sU[3 * i + a] = U[3 * e + a];
            sp[3 * i + a] = pts[3 * e + a];
        }
    }
    // point clusters of every depth: runs of equal code prefixes
    struct PDepth {
        std::vector<int64_t> start;
        std::vector<int64_t> ix, iy, iz;
        std::vector<double> rad;
        std::vector<int32_t> parent, pcl;
    };
    std::vector<PDepth> pd(D + 1);
    for (int d = 0; d <= D; ++d) {
        PDepth &P = pd[d];
        const int sh = D - d;
        const double box = t.edge / (double)((int64_t)1 << d);
        P.pcl.assign(m, -1);
        int64_t i = 0;
        while (i < m) {
            const uint64_t key = scode[i] >> (3 * sh);
            int64_t j = i;
            while (j < m && (scode[j] >> (3 * sh)) == key) ++j;
            const int32_t c = (int32_t)P.start.size();
            P.start.push_back(i);
            P.ix.push_back((sU[3 * i] >> sh) - (B >> sh));
            P.iy.push_back((sU[3 * i + 1] >> sh) - (B >> sh));
            P.iz.push_back((sU[3 * i + 2] >> sh) - (B >> sh));
            const double z[3] = {t.origin[0] + (P.ix.back() + 0.5) * box, t.origin[1] + (P.iy.back() + 0.5) * box,
                                 t.origin[2] + (P.iz.back() + 0.5) * box};
            double rad = 0.0;
            for (int64_t q = i; q < j; ++q) {
                P.pcl[q] = c;
                double d3[3];
                sub3(&sp[3 * q], z, d3);
                rad = std::max(rad, norm3(d3));
            }
            P.rad.push_back(rad);
            P.parent.push_back(d > 0 ? pd[d - 1].pcl[i] : -1);
            i = j;
        }
        P.start.push_back(m);
    }
    double R[kMaxRule + 1] = {0};
    order_thresholds(p.quad_tol, std::max(2, p.m_max), R);
    const double r1 = R[1] * (1.0 + 1e-9);
    const bool direct = p.mode == BEM_MODE_DIRECT;
    // near element clusters of each point cluster at the previous depth (CSR)
    std::vector<int32_t> nprev_ptr(pd[0].parent.size() + 1), nprev;
    int64_t rnear_prev = 0;   // largest |offset component| among the previous depth's near pairs
    for (size_t c = 0; c < pd[0].parent.size(); ++c) {
        nprev.push_back(0);   // the root element cluster
        nprev_ptr[c + 1] = (int32_t)nprev.size();
        rnear_prev = std::max(rnear_prev, std::max(std::abs(pd[0].ix[c] - t.lv[0].ix[0]),
                                                   std::max(std::abs(pd[0].iy[c] - t.lv[0].iy[0]),
                                                            std::abs(pd[0].iz[c] - t.lv[0].iz[0]))));
    }
    for (int d = 1; d <= D; ++d) {
        const Level &E = t.lv[d], &Ep = t.lv[d - 1];
        const PDepth &P = pd[d];
        const int npc = (int)P.parent.size();
        const double xL = 2.0 * E.rmax * k;
        const int L = std::max(p.L_min, (int)std::ceil(xL + p.trunc_factor * std::log10(xL + M_PI) - 1e-12));
        const bool stab_on = p.stability_max < 1e300;
        const bool allowed = !direct && L <= max_L && (!stab_on || (double)(L + 1) * (L + 1) <= p.stability_max);
        // the growth sum decreases with x, so an offset is stable when k |X|
        // reaches the root x* of growth = stability_max (bisection, once per
        // level)
        double xstar = 0.0;
        if (allowed && stab_on) {
            double lo = 1e-9, hi = 1.0;
            for (int it = 0; it < 64 && !(hankel_growth(hi, L) <= p.stability_max); ++it) hi *= 2.0;
            for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (hankel_growth(mid, L) <= p.stability_max) hi = mid;
                else lo = mid;
            }
            xstar = hi;
        }
        EvalLevel F;
        F.depth = d;
        F.L = L;
        F.npc = npc;
        F.il_ptr.assign(npc + 1, 0);
        // the point clusters in contiguous chunks, one per thread; each chunk
        // numbers its stable far offsets itself, and the chunks' numbers are
        // merged in chunk order afterwards (the plan does not depend on the
        // thread count's timing)
        struct Chunk {
            std::vector<int32_t> il_src, il_off, ncur, nil, nnear;   // nil / nnear: per cluster
            std::vector<OffKey> keys;                                 // local offset index -> key
            std::vector<double> X;                                    // 3 per local offset
            int64_t far_pairs = 0;
            int64_t rnear = 0;                                        // largest |offset component| of near pairs
        };
        // candidates are children of the previous depth's near pairs, so their
        // offsets lie in [-Rb, Rb]^3: a dense table of offset states when that
        // window is small, else a hash map
        const int64_t Rb = 2 * rnear_prev + 1, W = 2 * Rb + 1;
        const bool dense = W * W * W <= ((int64_t)1 << 21);
        const int64_t work = (int64_t)nprev.size() * 8;
        const int nth = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)n_threads, work / 20000, (int64_t)npc}));
        std::vector<Chunk> ch(nth);
        auto run = [&](int ti) {
            Chunk &C = ch[ti];
            const int c0 = (int)((int64_t)npc * ti / nth), c1 = (int)((int64_t)npc * (ti + 1) / nth);
            std::unordered_map<OffKey, int32_t, OffKeyHash> off_index;   // local index, -1: unstable
            std::vector<int32_t> off_state(dense ? (size_t)(W * W * W) : 0, -2);   // -2: not seen yet
            C.nil.assign(c1 - c0, 0);
            C.nnear.assign(c1 - c0, 0);
            for (int c = c0; c < c1; ++c) {
                const int par = P.parent[c];
                const int64_t cnt = P.start[c + 1] - P.start[c];
                const size_t il0 = C.il_src.size(), nn0 = C.ncur.size();
                for (int q = nprev_ptr[par]; q < nprev_ptr[par + 1]; ++q) {
                    const int sp = nprev[q];
                    for (int s = Ep.child0[sp]; s < Ep.child0[sp] + Ep.nchild[sp]; ++s) {
                        const int64_t dx = P.ix[c] - E.ix[s], dy = P.iy[c] - E.iy[s], dz = P.iz[c] - E.iz[s];
                        const double X[3] = {dx * E.box, dy * E.box, dz * E.box};
                        const double dist = norm3(X);
                        bool far = allowed && P.rad[c] <= E.rmax && dist > p.admissibility * (P.rad[c] + E.rad[s]) &&
                                   dist - P.rad[c] - E.crad[s] > r1 * std::sqrt(E.amax[s]);
                        int32_t oi = -1;
                        if (far) {
                            auto local_index = [&]() {
                                if (stab_on && !(k * dist >= xstar)) return -1;
                                C.keys.push_back(OffKey{dx, dy, dz});
                                C.X.insert(C.X.end(), X, X + 3);
                                return (int)C.keys.size() - 1;
                            };
                            if (dense) {
                                int32_t &st = off_state[(size_t)(((dx + Rb) * W + (dy + Rb)) * W + (dz + Rb))];
                                if (st == -2) st = local_index();
                                oi = st;
                            } else {
                                const OffKey key{dx, dy, dz};
                                auto it = off_index.find(key);
                                if (it == off_index.end()) it = off_index.emplace(key, local_index()).first;
                                oi = it->second;
                            }
                            far = oi >= 0;
                        }
                        if (far) {
                            C.il_src.push_back(s);
                            C.il_off.push_back(oi);
                            C.far_pairs += cnt * E.count[s];
                        } else {
                            C.ncur.push_back(s);
                            C.rnear = std::max(C.rnear, std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))));
                        }
                    }
                }
                C.nil[c - c0] = (int32_t)(C.il_src.size() - il0);
                C.nnear[c - c0] = (int32_t)(C.ncur.size() - nn0);
            }
        };
        run_parallel(nth, run);
        std::unordered_map<OffKey, int32_t, OffKeyHash> off_index;   // global index
        std::vector<int32_t> ncur_ptr(npc + 1, 0), ncur;
        int64_t rnear = 0;
        for (int ti = 0; ti < nth; ++ti) {
            Chunk &C = ch[ti];
            std::vector<int32_t> remap(C.keys.size());
            for (size_t u = 0; u < C.keys.size(); ++u) {
                auto it = off_index.find(C.keys[u]);
                if (it == off_index.end()) {
                    it = off_index.emplace(C.keys[u], (int32_t)(F.offsets.size() / 3)).first;
                    F.offsets.insert(F.offsets.end(), &C.X[3 * u], &C.X[3 * u] + 3);
                }
                remap[u] = it->second;
            }
            const int c0 = (int)((int64_t)npc * ti / nth);
            for (size_t u = 0; u < C.nil.size(); ++u) {
                F.il_ptr[c0 + u + 1] = F.il_ptr[c0 + u] + C.nil[u];
                ncur_ptr[c0 + u + 1] = ncur_ptr[c0 + u] + C.nnear[u];
            }
            F.il_src.insert(F.il_src.end(), C.il_src.begin(), C.il_src.end());
            for (int32_t oi : C.il_off) F.il_off.push_back(remap[oi]);
            ncur.insert(ncur.end(), C.ncur.begin(), C.ncur.end());
            ep.far_pairs += C.far_pairs;
            rnear = std::max(rnear, C.rnear);
            Chunk().il_src.swap(C.il_src);
        }
        F.n_inter = (int64_t)F.il_src.size();
        if (F.n_inter > 0) {
            F.pcl = P.pcl;
            F.zp.resize(3 * (size_t)npc);
            for (int c = 0; c < npc; ++c) {
                F.zp[3 * c] = t.origin[0] + (P.ix[c] + 0.5) * E.box;
                F.zp[3 * c + 1] = t.origin[1] + (P.iy[c] + 0.5) * E.box;
                F.zp[3 * c + 2] = t.origin[2] + (P.iz[c] + 0.5) * E.box;
            }
            ep.far.push_back(std::move(F));
        }
        nprev_ptr.swap(ncur_ptr);
        nprev.swap(ncur);
        rnear_prev = rnear;
    }
    // leaf near lists (sorted element leaves)
    const PDepth &PL = pd[D];
    const int npl = (int)PL.parent.size();
    ep.leaf_start = PL.start;
    ep.near_ptr.assign(npl + 1, 0);
    const Level &EL = t.lv[D];
    for (int c = 0; c < npl; ++c) {
        std::vector<int32_t> v(nprev.begin() + nprev_ptr[c], nprev.begin() + nprev_ptr[c + 1]);
        std::sort(v.begin(), v.end());
        for (int32_t s2 : v) {
            ep.near_src.push_back(s2);
            ep.near_pairs += (PL.start[c + 1] - PL.start[c]) * EL.count[s2];
        }
        ep.near_ptr[c + 1] = (int32_t)ep.near_src.size();
    }
    return "";
}

// Kernel evaluations of one near pair (row element at x, column element e):
// the whole element under one regular rule, or the subdivision of Sec. 3.1.3
// into four children (midpoint, vertex, edge midpoints) while r~ < rt_sub.
static int64_t pair_points(const Geometry &g, const double *x, int64_t e, const double *R, const bem_params &p)
{
    auto order = [&](double rt) {
        for (int m = 1; m < p.m_max; ++m)
            if (rt > R[m]) return m;
        return p.m_max;
    };
    struct Sub { double x0, y0, x1, y1, x2, y2; int depth; };
    std::vector<Sub> st{{0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0}};
    int64_t pts = 0;
    while (!st.empty()) {
        const Sub s = st.back();
        st.pop_back();
        const double cx = (s.x0 + s.x1 + s.x2) / 3.0, cy = (s.y0 + s.y1 + s.y2) / 3.0;
        double d[3];
        for (int q = 0; q < 3; ++q)
            d[q] = g.cen[3 * e + q] + g.va[3 * e + q] + cx * g.e1[3 * e + q] + cy * g.e2[3 * e + q] - x[q];
        const double rt = norm3(d) / std::sqrt(g.area[e] * std::ldexp(1.0, -2 * s.depth));
        if (rt >= p.rt_subdiv || s.depth >= p.max_depth) {
            const int m = order(rt);
            pts += (int64_t)m * m;
            continue;
        }
        const double mx01 = 0.5 * (s.x0 + s.x1), my01 = 0.5 * (s.y0 + s.y1);
        const double mx12 = 0.5 * (s.x1 + s.x2), my12 = 0.5 * (s.y1 + s.y2);
        const double mx20 = 0.5 * (s.x2 + s.x0), my20 = 0.5 * (s.y2 + s.y0);
        const int dd = s.depth + 1;
        st.push_back({mx01, my01, mx12, my12, mx20, my20, dd});
        st.push_back({mx20, my20, mx12, my12, s.x2, s.y2, dd});
        st.push_back({mx01, my01, s.x1, s.y1, mx12, my12, dd});
        st.push_back({s.x0, s.y0, mx01, my01, mx20, my20, dd});
    }
    return pts;
}

NearCount count_near_points(const Geometry &g, const Tree &t, const FreqPlan &fp, const bem_params &p)
{
    NearCount c;
    double R[kMaxRule + 1] = {0};
    order_thresholds(p.quad_tol, std::max(2, p.m_max), R);
    // the light / heavy split of the entry kernels: light when r~ is above
    // R_3 (1 + 1e-5), so that one rule of order 1..3 covers the element
    const double heavy_rt2 = p.m_max > 3 ? (R[3] * (1.0 + 1e-5)) * (R[3] * (1.0 + 1e-5)) : 0.0;
    const Level &Lf = t.lv[fp.leaf_depth];
    const int nl = (int)Lf.start.size();
    for (int a = 0; a < nl; ++a) {
        for (int64_t ii = Lf.start[a]; ii < Lf.start[a] + Lf.count[a]; ++ii) {
            const int64_t ei = t.perm[ii];
            const double *x = &g.cen[3 * ei];
            for (int q = fp.near_ptr[a]; q < fp.near_ptr[a + 1]; ++q) {
                const int b = fp.near_src[q];
                for (int64_t jj = Lf.start[b]; jj < Lf.start[b] + Lf.count[b]; ++jj) {
                    const int64_t ej = t.perm[jj];
                    if (ej == ei) {
                        c.heavy_entries += 1;
                        c.heavy_points += 6 * 16 + 3 * 4 * 3;
                        continue;
                    }
                    double d[3];
                    sub3(&g.cen[3 * ej], x, d);
                    const double rt2 = dot3(d, d) / g.area[ej];
                    if (p.m_max > 3 && !(rt2 > heavy_rt2)) {
                        c.heavy_entries += 1;
                        c.heavy_points += pair_points(g, x, ej, R, p);
                    } else {
                        const int m = rt2 > R[1] * R[1] ? 1 : (rt2 > R[2] * R[2] ? 2 : 3);
                        c.light_entries += 1;
                        c.light_points += (int64_t)m * m;
                    }
                }
            }
        }
    }
    return c;
}

MeshCheck check_mesh(const Geometry &g, const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n)
{
    MeshCheck r;
    // weld coincident vertices: id[v] = first vertex with the same rounded position
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) ext = std::max(ext, g.vmax[d] - g.vmin[d]);
    const double q = ext > 0 ? 1e-9 * ext : 1.0;
    std::vector<std::tuple<int64_t, int64_t, int64_t, int32_t>> key((size_t)n_nodes);
    for (int64_t v = 0; v < n_nodes; ++v)
        key[v] = std::make_tuple((int64_t)std::llround((nodes[3 * v] - g.vmin[0]) / q),
                                 (int64_t)std::llround((nodes[3 * v + 1] - g.vmin[1]) / q),
                                 (int64_t)std::llround((nodes[3 * v + 2] - g.vmin[2]) / q), (int32_t)v);
    std::sort(key.begin(), key.end());
    std::vector<int32_t> id((size_t)n_nodes);
    for (size_t i = 0; i < key.size(); ++i) {
        const bool same = i > 0 && std::get<0>(key[i]) == std::get<0>(key[i - 1]) &&
                          std::get<1>(key[i]) == std::get<1>(key[i - 1]) && std::get<2>(key[i]) == std::get<2>(key[i - 1]);
        id[std::get<3>(key[i])] = same ? id[std::get<3>(key[i - 1])] : std::get<3>(key[i]);
    }
    for (int64_t j = 0; j < n; ++j)
        r.volume += g.area[j] * (g.cen[3 * j] * g.nrm[3 * j] + g.cen[3 * j + 1] * g.nrm[3 * j + 1] +
                                 g.cen[3 * j + 2] * g.nrm[3 * j + 2]) / 3.0;
    // undirected edge (lo, hi) -> traversals lo -> hi and hi -> lo
    std::vector<std::tuple<int32_t, int32_t, int>> ed;
    ed.reserve(3 * n);
    for (int64_t j = 0; j < n; ++j)
        for (int e = 0; e < 3; ++e) {
            const int32_t a = id[tris[3 * j + e]], b = id[tris[3 * j + (e + 1) % 3]];
            ed.emplace_back(std::min(a, b), std::max(a, b), a < b ? 1 : 0);
        }
    std::sort(ed.begin(), ed.end());
    for (size_t i = 0; i < ed.size();) {
        size_t k = i;
        int fwd = 0;
        while (k < ed.size() && std::get<0>(ed[k]) == std::get<0>(ed[i]) && std::get<1>(ed[k]) == std::get<1>(ed[i])) {
            fwd += std::get<2>(ed[k]);
            ++k;
        }
        const size_t cnt = k - i;
        if (cnt != 2) ++r.open_edges;
        else if (fwd != 1) ++r.misoriented_edges;
        i = k;
    }
    return r;
}

}  // namespace bem
