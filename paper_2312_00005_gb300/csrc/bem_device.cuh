// bem_device.cuh -- device data structures and the element-integral routines
// (quadrature of Sec. 3.1 of arXiv 2312.00005) shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bem {

constexpr int kRules = 7;                 // conical rules for m = 1..6 (index m)
constexpr float kInv4Pi = 0.0795774715459476679f;

struct QuadTables {
    float tri_xi[kRules][36], tri_eta[kRules][36], tri_w[kRules][36];
    float gl4_x[4], gl4_w[4];             // Duffy rule, [0,1]
    float gl3_x[3], gl3_w[3];             // edge rule per part, [0,1]
    float R[kRules];                      // order thresholds R[1..m_max-1]
    double Rd[kRules];
    float rt_sub;
    double rt_sub_d;
    // squared thresholds of the light / heavy split: a pair is light when
    // r~^2 > heavy_rt2 = (R_3 (1 + 1e-5))^2; R2[m] = R_m^2
    float R2[kRules];
    float heavy_rt2;
    int m_max;
    int max_depth;
    int edge_parts;
};

// Element data in the internal (cluster-sorted) order.
struct ElemDev {
    int64_t n;
    const float4 *chi;   // midpoint, high part; .w = area
    const float4 *clo;   // midpoint, low part (x - float(x))
    const float4 *nrm;   // unit normal
    const float4 *va;    // vertex a - midpoint
    const float4 *e1;    // b - a
    const float4 *e2;    // c - a
    const double *cd;    // 3n midpoints (FP64, for rule decisions near thresholds)
    const double *vad;   // 3n
    const double *e1d;   // 3n
    const double *e2d;   // 3n
    const double *ad;    // n areas
};

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c)
{   // a * b + c
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub3f(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mad3(float s, float3 a, float3 b)
{
    return make_float3(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y), fmaf(s, a.z, b.z));
}

// sin and cos of 2 pi t, t in turns: t - round(t) is exact, so the
// reduction adds no error; then the SFU approximations on [-pi, pi]
// (absolute error about 2^-21).  Used for the phases e^{ikr} of the regular
// quadrature points and of the far field.  The unit tests compare it with
// CUDA's sincospif.
__device__ __forceinline__ void sincos_turns(float t, float *s, float *c)
{
    // round to the nearest integer by adding and removing 1.5 2^23 (exact
    // for |t| < 2^22; the phases stay far below)
    const float r = t - __fsub_rn(__fadd_rn(t, 12582912.f), 12582912.f);
    __sincosf(r * 6.28318548f, s, c);
}

// ------------------------------------------------------------------ kernels
// Burton-Miller column kernels at one quadrature point (Eq. SystemI, tau = 1,
// gamma = i/k), with d = y - x, weight w:
//   Kp = -(H - gamma E)    (multiplies the column's pressure)
//   Kq =  G - gamma H'     (multiplies the column's q = dp/dn)
// G = e^{ikr}/(4 pi r), H = G (ik - 1/r) (d.ny)/r, H' = -G (ik - 1/r) (d.nx)/r,
// E = G [(k^2 + 3ik/r - 3/r^2)(d.nx/r)(d.ny/r) - (ik/r - 1/r^2)(nx.ny)].
// With ir = 1/r, rx = d.nx/r, ry = d.ny/r, nn = nx.ny this is
//   Kp = G [ ir (ry - 3 rx ry + nn) + i ( -k ry + (k - 3 ir^2/k) rx ry + (ir^2/k) nn ) ]
//   Kq = G [ 1 - rx - i (ir/k) rx ].
__device__ __forceinline__ void bm_point(float3 d, float3 nx, float3 ny, float k, float ik_inv, float w,
                                         float2 &Kp, float2 &Kq)
{
    float r2 = dot3f(d, d);
    float ir = rsqrtf(r2);
    float r = r2 * ir;
    float s, c;
    sincos_turns(k * r * 0.15915494309189535f, &s, &c);
    float g = w * ir * kInv4Pi;
    float2 G = make_float2(c * g, s * g);
    float rx = dot3f(d, nx) * ir, ry = dot3f(d, ny) * ir, nn = dot3f(nx, ny);
    float ir2k = ir * ir * ik_inv;
    float rxry = rx * ry;
    float2 P = make_float2(ir * (ry - 3.0f * rxry + nn), -k * ry + (k - 3.0f * ir2k) * rxry + ir2k * nn);
    float2 Q = make_float2(1.0f - rx, -(ir * ik_inv) * rx);
    Kp = cfma(G, P, Kp);
    Kq = cfma(G, Q, Kq);
}

// G and H only (field evaluation, Eq. BIE_I with lambda = 1).
__device__ __forceinline__ void gh_point(float3 d, float3 ny, float k, float w, float2 &G, float2 &H)
{
    float r2 = dot3f(d, d);
    float ir = rsqrtf(r2);
    float r = r2 * ir;
    float s, c;
    sincos_turns(k * r * 0.15915494309189535f, &s, &c);
    float g = w * ir * kInv4Pi;
    float2 Gp = make_float2(c * g, s * g);
    float ry = dot3f(d, ny) * ir;
    G = cadd(G, Gp);
    // H = G (ik - 1/r) ry
    H = cfma(Gp, make_float2(-ir * ry, k * ry), H);
}


// grad_x G and grad_x H (H = dG/dn_y) at one quadrature point, d = y - x,
// for the particle velocity at field points (Eq. utopandv, with Eq. BIE_I
// differentiated under the integral).  With f = G (ik - 1/r) / r:
//   grad_x G = -f d,
//   grad_x H = -f'(r) (d.ny / r) d - f ny,
//   f'(r) = G (-k^2 / r - 3ik / r^2 + 3 / r^3);
// their components along a unit vector e are the kernels H' and E of
// Eq. dBIE with n_x = e.
__device__ __forceinline__ void grad_point(float3 d, float3 ny, float k, float w, float2 *gG, float2 *gH)
{
    const float r2 = dot3f(d, d);
    const float ir = rsqrtf(r2);
    const float r = r2 * ir;
    float s, c;
    sincos_turns(k * r * 0.15915494309189535f, &s, &c);
    const float g = w * ir * kInv4Pi;
    const float2 G = make_float2(c * g, s * g);
    const float2 Ga = cmul(G, make_float2(-ir, k));          // G (ik - 1/r)
    const float2 f = make_float2(Ga.x * ir, Ga.y * ir);
    const float ir2 = ir * ir;
    const float2 fp = cmul(G, make_float2(-k * k * ir + 3.0f * ir2 * ir, -3.0f * k * ir2));
    const float dn = dot3f(d, ny) * ir;
    const float2 cd = make_float2(-fp.x * dn, -fp.y * dn);   // grad_x H = cd d - f ny
    const float dv[3] = {d.x, d.y, d.z}, nv[3] = {ny.x, ny.y, ny.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gG[a].x = fmaf(-f.x, dv[a], gG[a].x);
        gG[a].y = fmaf(-f.y, dv[a], gG[a].y);
        gH[a].x = fmaf(cd.x, dv[a], fmaf(-f.x, nv[a], gH[a].x));
        gH[a].y = fmaf(cd.y, dv[a], fmaf(-f.y, nv[a], gH[a].y));
    }
}

// Rule code for a (sub)element: 0 = subdivide, m >= 1 = regular order m.
__device__ __forceinline__ int rule_from_rt(float rt, const QuadTables &Q)
{
    if (rt < Q.rt_sub) return 0;
    for (int m = 1; m < Q.m_max; ++m)
        if (rt > Q.R[m]) return m;
    return Q.m_max;
}
__device__ __forceinline__ int rule_from_rt_d(double rt, const QuadTables &Q)
{
    if (rt < Q.rt_sub_d) return 0;
    for (int m = 1; m < Q.m_max; ++m)
        if (rt > Q.Rd[m]) return m;
    return Q.m_max;
}
__device__ __forceinline__ bool rt_ambiguous(float rt, const QuadTables &Q)
{
    const float g = 1e-5f;
    if (fabsf(rt - Q.rt_sub) <= g * Q.rt_sub) return true;
    for (int m = 1; m < Q.m_max; ++m)
        if (fabsf(rt - Q.R[m]) <= g * Q.R[m]) return true;
    return false;
}

// r~^2 of the whole element j seen from x (x_j - x from high / low parts,
// 1/area_j given), with every rounding spelled out so that the classifier
// and the light-entry kernel derive the same bits.
__device__ __forceinline__ float pair_rt2(float3 xj_hi, float3 xj_lo, float3 xi_hi, float3 xi_lo, float inv_area,
                                          float3 &D0)
{
    D0 = make_float3(__fadd_rn(__fsub_rn(xj_hi.x, xi_hi.x), __fsub_rn(xj_lo.x, xi_lo.x)),
                     __fadd_rn(__fsub_rn(xj_hi.y, xi_hi.y), __fsub_rn(xj_lo.y, xi_lo.y)),
                     __fadd_rn(__fsub_rn(xj_hi.z, xi_hi.z), __fsub_rn(xj_lo.z, xi_lo.z)));
    return __fmul_rn(__fmaf_rn(D0.x, D0.x, __fmaf_rn(D0.y, D0.y, __fmul_rn(D0.z, D0.z))), inv_area);
}
// Expensive pair: the self term, or an element whose r~ (whole element) is
// not clearly above R_3, i.e. that may need subdivision or a rule of order
// >= 4.  The cheap pairs take 1 to 9 quadrature points.
__device__ __forceinline__ bool heavy_rt2(int64_t i, int64_t j, float rt2, const QuadTables &Q)
{
    if (i == j) return true;
    if (Q.m_max <= 3) return false;
    return !(rt2 > Q.heavy_rt2);
}

// Sub-triangle in the reference coordinates (xi, eta) of its element.
struct SubTri {
    float x0, y0, x1, y1, x2, y2;
    int depth;
};

// Integrate kernels over element j from point x (high/low parts xhi, xlo;
// FP64 copy xd), with the subdivision of Sec. 3.1.3 and the regular rule of
// Sec. 3.1.4: acc.point(d, ny, w) adds the kernels at each quadrature point
// (d = y - x, weight w).  Quadrature points are y = a + xi (b - a) +
// eta (c - a); every distance is formed from local offsets so FP32 keeps its
// relative accuracy.  Returns false if the subdivision limit is exceeded.
template <class Acc>
__device__ bool integrate_regular_acc(const ElemDev &E, int64_t j, float3 xhi, float3 xlo, const double *xd,
                                      const QuadTables &Q, Acc &acc)
{
    const float4 ch = E.chi[j], cl = E.clo[j];
    const float3 D0 = add3(sub3f(f3(ch), xhi), sub3f(f3(cl), xlo));   // x_j - x
    const float3 va = f3(E.va[j]), e1 = f3(E.e1[j]), e2 = f3(E.e2[j]), ny = f3(E.nrm[j]);
    const float3 base = add3(D0, va);                                   // a - x
    const float area = ch.w;
    // Fast path: r~ of the whole element clearly above R_1 (order m = 1, no
    // subdivision).  The 1 x 1 conical rule is the centroid rule (node
    // (1/3, 1/3), weight 1/2), so the integral is A_j K(x, x_j).
    if (Q.m_max > 1) {
        const float rt0 = sqrtf(dot3f(D0, D0) / area);
        if (rt0 > Q.R[1] * (1.0f + 1e-5f)) {
            acc.point(D0, ny, area);
            return true;
        }
    }
    // Whole element under one regular rule (no subdivision): the common
    // case, handled without the subdivision stack.  Same decision as the
    // first step of the loop below (the unit triangle's centroid is x_j).
    {
        const float rt = sqrtf(dot3f(D0, D0) / area);
        int code;
        if (!rt_ambiguous(rt, Q)) {
            code = rule_from_rt(rt, Q);
        } else {
            double d[3];
            for (int q = 0; q < 3; ++q)
                d[q] = (xd[q] - E.cd[3 * j + q]) -
                       (E.vad[3 * j + q] + (1.0 / 3.0) * E.e1d[3 * j + q] + (1.0 / 3.0) * E.e2d[3 * j + q]);
            code = rule_from_rt_d(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / sqrt(E.ad[j]), Q);
        }
        if (code > 0) {
            const int nq = code * code;
            for (int q = 0; q < nq; ++q) {
                const float3 d = mad3(Q.tri_eta[code][q], e2, mad3(Q.tri_xi[code][q], e1, base));
                const float w = 2.0f * area * Q.tri_w[code][q];
                acc.point(d, ny, w);
            }
            return true;
        }
    }
    SubTri stack[3 * 15 + 4];
    int top = 0;
    stack[top++] = SubTri{0.f, 0.f, 1.f, 0.f, 0.f, 1.f, 0};
    bool ok = true;
    while (top > 0) {
        SubTri s = stack[--top];
        const float cx = (s.x0 + s.x1 + s.x2) * (1.0f / 3.0f), cy = (s.y0 + s.y1 + s.y2) * (1.0f / 3.0f);
        const float3 dc = mad3(cy, e2, mad3(cx, e1, base));              // centroid - x
        const float sa = area * exp2f(-2.0f * (float)s.depth);           // area / 4^depth
        const float rt = sqrtf(dot3f(dc, dc) / sa);
        int code;
        if (!rt_ambiguous(rt, Q)) {
            code = rule_from_rt(rt, Q);
        } else {
            // FP64 decision (same formula as in FP32, exact coordinates)
            double d[3];
            const double cxd = ((double)s.x0 + (double)s.x1 + (double)s.x2) / 3.0;
            const double cyd = ((double)s.y0 + (double)s.y1 + (double)s.y2) / 3.0;
            for (int q = 0; q < 3; ++q)
                d[q] = (xd[q] - E.cd[3 * j + q]) - (E.vad[3 * j + q] + cxd * E.e1d[3 * j + q] + cyd * E.e2d[3 * j + q]);
            const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double rtd = dist / sqrt(E.ad[j] * exp2(-2.0 * s.depth));
            code = rule_from_rt_d(rtd, Q);
        }
        if (code == 0) {
            if (s.depth >= Q.max_depth) { ok = false; break; }
            const float mx01 = 0.5f * (s.x0 + s.x1), my01 = 0.5f * (s.y0 + s.y1);
            const float mx12 = 0.5f * (s.x1 + s.x2), my12 = 0.5f * (s.y1 + s.y2);
            const float mx20 = 0.5f * (s.x2 + s.x0), my20 = 0.5f * (s.y2 + s.y0);
            const int dd = s.depth + 1;
            // children in the vertex order (a, m_ab, m_ca), (m_ab, b, m_bc),
            // (m_ca, m_bc, c), (m_ab, m_bc, m_ca)
            stack[top++] = SubTri{mx01, my01, mx12, my12, mx20, my20, dd};
            stack[top++] = SubTri{mx20, my20, mx12, my12, s.x2, s.y2, dd};
            stack[top++] = SubTri{mx01, my01, s.x1, s.y1, mx12, my12, dd};
            stack[top++] = SubTri{s.x0, s.y0, mx01, my01, mx20, my20, dd};
            continue;
        }
        const int nq = code * code;
        const float sx1 = s.x1 - s.x0, sy1 = s.y1 - s.y0, sx2 = s.x2 - s.x0, sy2 = s.y2 - s.y0;
        for (int q = 0; q < nq; ++q) {
            const float u = Q.tri_xi[code][q], v = Q.tri_eta[code][q];
            const float px = s.x0 + u * sx1 + v * sx2, py = s.y0 + u * sy1 + v * sy2;
            const float3 d = mad3(py, e2, mad3(px, e1, base));
            const float w = 2.0f * sa * Q.tri_w[code][q];
            acc.point(d, ny, w);
        }
    }
    return ok;
}

// Point accumulators for integrate_regular_acc.
struct BmAcc {        // Burton-Miller column kernels Kp, Kq (bm_point)
    float3 nx;
    float k, ik_inv;
    float2 A0, A1;
    __device__ __forceinline__ void point(float3 d, float3 ny, float w) { bm_point(d, nx, ny, k, ik_inv, w, A0, A1); }
};
struct GhAcc {        // G and H of a field point (gh_point)
    float k;
    float2 A0, A1;
    __device__ __forceinline__ void point(float3 d, float3 ny, float w) { gh_point(d, ny, k, w, A0, A1); }
};
struct GradAcc {      // grad_x G and grad_x H of a field point (grad_point)
    float k;
    float2 gG[3], gH[3];
    __device__ __forceinline__ void point(float3 d, float3 ny, float w) { grad_point(d, ny, k, w, gG, gH); }
};

// The Burton-Miller kernels (kField false) or G and H of a field point
// (kField true) integrated over element j; see integrate_regular_acc.
template <bool kField>
__device__ __forceinline__ bool integrate_regular(const ElemDev &E, int64_t j, float3 xhi, float3 xlo,
                                                  const double *xd, float3 nx, float k, float ik_inv,
                                                  const QuadTables &Q, float2 &A0, float2 &A1)
{
    if (kField) {
        GhAcc a{k, A0, A1};
        const bool ok = integrate_regular_acc(E, j, xhi, xlo, xd, Q, a);
        A0 = a.A0;
        A1 = a.A1;
        return ok;
    }
    BmAcc a{nx, k, ik_inv, A0, A1};
    const bool ok = integrate_regular_acc(E, j, xhi, xlo, xd, Q, a);
    A0 = a.A0;
    A1 = a.A1;
    return ok;
}

// Self term (x = midpoint of element j): Duffy rule on the six sub-triangles
// (midpoint, vertex, edge midpoint) with 4 x 4 Gauss points for G
// (Sec. 3.1.1), H = H' = 0, and E = edge integral + k^2 G with 4 parts x 3
// Gauss points per edge (Sec. 3.1.2).  Returns G_ii and E_ii.
__device__ __forceinline__ void self_term(const ElemDev &E, int64_t j, float k, const QuadTables &Q,
                                          float2 &Gii, float2 &Eii)
{
    const float3 va = f3(E.va[j]), e1 = f3(E.e1[j]), e2 = f3(E.e2[j]), n = f3(E.nrm[j]);
    float3 P[6];
    P[0] = va;                                  // a - x
    P[2] = add3(va, e1);                        // b - x
    P[4] = add3(va, e2);                        // c - x
    P[1] = make_float3(0.5f * (P[0].x + P[2].x), 0.5f * (P[0].y + P[2].y), 0.5f * (P[0].z + P[2].z));
    P[3] = make_float3(0.5f * (P[2].x + P[4].x), 0.5f * (P[2].y + P[4].y), 0.5f * (P[2].z + P[4].z));
    P[5] = make_float3(0.5f * (P[4].x + P[0].x), 0.5f * (P[4].y + P[0].y), 0.5f * (P[4].z + P[0].z));
    float2 G = make_float2(0.f, 0.f);
    for (int e = 0; e < 6; ++e) {
        const float3 p1 = P[e], dp = sub3f(P[(e + 1) % 6], P[e]);
        const float3 cr = make_float3(p1.y * dp.z - p1.z * dp.y, p1.z * dp.x - p1.x * dp.z, p1.x * dp.y - p1.y * dp.x);
        const float twoA = sqrtf(dot3f(cr, cr));
        for (int a = 0; a < 4; ++a) {
            const float u = Q.gl4_x[a];
            for (int b = 0; b < 4; ++b) {
                const float v = Q.gl4_x[b];
                const float3 d = make_float3(u * (p1.x + v * dp.x), u * (p1.y + v * dp.y), u * (p1.z + v * dp.z));
                const float r2 = dot3f(d, d);
                const float ir = rsqrtf(r2);
                float s, c;
                sincosf(k * r2 * ir, &s, &c);
                const float g = Q.gl4_w[a] * Q.gl4_w[b] * twoA * u * ir * kInv4Pi;
                G.x = fmaf(c, g, G.x);
                G.y = fmaf(s, g, G.y);
            }
        }
    }
    // hypersingular edge part: sum over edges (a->b, b->c, c->a) of
    // integral of dG/dr (d.m)/r ds, m = t x n the outward edge normal
    float2 Ee = make_float2(0.f, 0.f);
    const float3 V[3] = {P[0], P[2], P[4]};
    const int parts = Q.edge_parts;
    for (int e = 0; e < 3; ++e) {
        const float3 p = V[e], pq = sub3f(V[(e + 1) % 3], V[e]);
        const float len = sqrtf(dot3f(pq, pq));
        const float3 t = make_float3(pq.x / len, pq.y / len, pq.z / len);
        const float3 m = make_float3(t.y * n.z - t.z * n.y, t.z * n.x - t.x * n.z, t.x * n.y - t.y * n.x);
        const float hm = dot3f(p, m);            // (y - x).m, constant on the edge
        for (int sp = 0; sp < parts; ++sp) {
            for (int g3 = 0; g3 < 3; ++g3) {
                const float sg = ((float)sp + Q.gl3_x[g3]) / (float)parts;
                const float wg = Q.gl3_w[g3] * len / (float)parts;
                const float3 d = mad3(sg, pq, p);
                const float r2 = dot3f(d, d);
                const float ir = rsqrtf(r2);
                float s, c;
                sincosf(k * r2 * ir, &s, &c);
                const float g = wg * ir * kInv4Pi * hm * ir;   // G (d.m)/r without the (ik - 1/r) factor
                const float2 Gp = make_float2(c * g, s * g);
                Ee = cfma(Gp, make_float2(-ir, k), Ee);
            }
        }
    }
    Gii = G;
    Eii = make_float2(Ee.x + k * k * G.x, Ee.y + k * k * G.y);
}

// Entry A_ij of the Burton-Miller matrix for columns with coefficients
// (cp_j, cq_j) that already carry tau (Eq. SystemI: +1 exterior, -1
// interior, on every integral operator): A_ij = cp_j Kp_ij + cq_j Kq_ij +
// delta_ij tau (cp_i - gamma cq_i)/2, the identity half without tau.
__device__ __forceinline__ bool bm_entry(const ElemDev &E, int64_t i, int64_t j, float3 xhi, float3 xlo,
                                         const double *xd, float3 nx, float k, float ik_inv, float tau,
                                         const QuadTables &Q, float2 cpj, float2 cqj, float2 &out)
{
    if (i == j) {
        float2 Gii, Eii;
        self_term(E, j, k, Q, Gii, Eii);
        // Kp = gamma E_ii (H_ii = 0), Kq = G_ii (H'_ii = 0); gamma = i/k
        const float2 gE = make_float2(-Eii.y * ik_inv, Eii.x * ik_inv);
        float2 v = cadd(cmul(cpj, gE), cmul(cqj, Gii));
        // (cp - gamma cq)/2 of the coefficients without tau
        const float2 gcq = make_float2(-cqj.y * ik_inv, cqj.x * ik_inv);
        v = cadd(v, cscale(csub(cpj, gcq), 0.5f * tau));
        out = v;
        return true;
    }
    float2 Kp = make_float2(0.f, 0.f), Kq = make_float2(0.f, 0.f);
    const bool ok = integrate_regular<false>(E, j, xhi, xlo, xd, nx, k, ik_inv, Q, Kp, Kq);
    out = cadd(cmul(cpj, Kp), cmul(cqj, Kq));
    return ok;
}

}  // namespace bem
