// bem_plan.hpp -- host-side (C++, FP64) geometry, quadrature tables and the
// cluster tree / per-frequency plan of the BEM + FMM operator.
//
// Method: arXiv 2312.00005 (NumCalc).  Geometry Sec. 2.3 / App. A;
// quadrature Sec. 3.1; clustering and lists Sec. 3.3.2-3.3.4; truncation
// Eq. FMMTruncation; admissibility Eq. Farfieldcond.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bemfmm.h"

namespace bem {

constexpr int kMaxRule = 6;          // regular order cap supported on the device
constexpr int kMaxLevels = 16;

// ---------------------------------------------------------------- geometry
struct Geometry {
    int64_t n = 0;
    std::vector<double> cen;   // 3n midpoints (mean of the vertices)
    std::vector<double> nrm;   // 3n unit normals, (b - a) x (c - a) / |.|
    std::vector<double> area;  // n
    std::vector<double> va;    // 3n vertex a relative to the midpoint
    std::vector<double> e1;    // 3n b - a
    std::vector<double> e2;    // 3n c - a
    std::vector<double> vmin, vmax;  // bounding box of all vertices
    std::vector<double> vrad;  // per element: max distance of its vertices to its midpoint
    double mean_edge = 0.0;
    double max_area = 0.0;
};

// Returns an empty string or an error message (degenerate triangle, bad index).
std::string compute_geometry(const double *nodes, int64_t n_nodes, const int32_t *tris,
                             int64_t n, Geometry &g);

// Orientation diagnostics of a closed triangle surface (Sec. 2.1: the normals
// must point away from the scatterer): the signed enclosed volume
// (1/3) sum_j A_j (x_j . n_j) by the divergence theorem, positive when every
// normal points out of the enclosed volume; the edges not shared by exactly
// two triangles; the shared edges that both triangles traverse in the same
// direction (inconsistent winding).  Vertices closer than 1e-9 of the
// bounding box are one vertex for the edge count (node lists may repeat a
// point).
struct MeshCheck {
    double volume = 0.0;
    int64_t open_edges = 0, misoriented_edges = 0;
};
MeshCheck check_mesh(const Geometry &g, const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n);

// ---------------------------------------------------------------- quadrature tables
// Gauss rules by the Golub-Welsch eigenvalue method (Jacobi rotations on the
// symmetric tridiagonal Jacobi matrix of the three-term recurrence).
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w);  // on [0,1]
void gauss_jacobi10_01(int n, std::vector<double> &x, std::vector<double> &w); // weight (1-u) on [0,1]
// m x m conical-product triangle rule on {xi, eta >= 0, xi + eta <= 1}:
// xi = u (Gauss-Jacobi(1,0)), eta = (1 - u) v (Gauss-Legendre); weights sum 1/2.
void conical_rule(int m, std::vector<double> &xi, std::vector<double> &eta, std::vector<double> &w);
// R[m] for m = 1..m_max-1: the regular order is the smallest m with r~ > R[m]
// (all three a-priori estimates of Sec. 3.1.4 below tol), else m_max.
void order_thresholds(double tol, int m_max, double *R);
// unit-sphere grid: L Gauss-Legendre nodes in cos(theta) x 2L azimuths
// phi = pi b / L; weights w_GL * pi / L (sum 4 pi).  s: 3 * 2L^2, ordered in
// antipodal halves: for q < L^2, s_{q + L^2} = -s_q exactly (same weight),
// so a phase e^{ik d.s} serves both (the second is the conjugate).
void sphere_grid(int L, std::vector<double> &s, std::vector<double> &w);
// sum_{n<=L} (2n+1) |h_n(x)| / |h_0(x)| (h_n by upward recursion)
double hankel_growth(double x, int L);

// ---------------------------------------------------------------- tree
struct Level {
    int depth = 0;
    double box = 0.0;                 // box edge at this depth
    std::vector<int64_t> start, count;  // element ranges (internal order)
    std::vector<int32_t> ix, iy, iz;  // integer box coordinates
    std::vector<double> z;            // 3 * nc box centres
    std::vector<double> rad;          // max |vertex - z| (admissibility radius, Sec. 3.3.1)
    std::vector<double> crad;         // max |midpoint - z|
    std::vector<double> amax;         // max element area
    std::vector<int32_t> parent;      // cluster index at depth - 1
    std::vector<int32_t> child0, nchild;  // children range at depth + 1
    std::vector<int32_t> elem_cluster;    // per element (internal order)
    double rmax = 0.0;
};

struct Tree {
    double origin[3] = {0, 0, 0};
    double edge = 0.0;
    int leaf_depth = 0;
    std::vector<int64_t> perm;        // internal -> caller index
    std::vector<Level> lv;            // depth 0 .. leaf_depth
};

void build_tree(const Geometry &g, double leaf_edge, Tree &t);
double auto_leaf_edge(const Geometry &g, const bem_params &p);

// ---------------------------------------------------------------- per-frequency plan
struct FarLevel {
    int depth = 0;
    int L = 0;
    int nc = 0;                          // clusters at this depth
    std::vector<int32_t> il_ptr;         // nc + 1
    std::vector<int32_t> il_src, il_off; // interaction list entries
    std::vector<double> offsets;         // 3 * noff translation vectors z_t - z_s
    int64_t n_inter = 0;
};

// A Hankel-growth verdict the list builder evaluated: depth, box offset,
// expansion length, and whether the offset passed.
struct Verdict {
    int depth, dx, dy, dz, L;
    bool stable;
};

struct FreqPlan {
    double k = 0.0;
    bool direct = false;
    int leaf_depth = 0;                  // depth of the leaves these lists end at
    std::vector<Verdict> verdicts;       // every stability test the build evaluated
    std::vector<int> Ld;                 // expansion length per depth used by the build
    std::vector<FarLevel> far;           // used levels, coarse to fine
    // near field at the leaf depth: per leaf a list of source leaves
    std::vector<int32_t> near_ptr, near_src;
    int64_t nnz = 0;
    int max_L = 0;
};

// Quadrature work of the near field of a plan (the rules of Sec. 3.1 as the
// entry kernels apply them): entries under one regular rule of order 1..3
// over the whole element ("light") and the rest (self terms, subdivided
// pairs, orders 4..6: "heavy"), with their kernel evaluations.  Rule
// decisions in FP64 (the device decides in FP32 with an FP64 fallback within
// 1e-5 of a threshold, so both agree).
struct NearCount {
    int64_t light_entries = 0, light_points = 0, heavy_entries = 0, heavy_points = 0;
};
NearCount count_near_points(const Geometry &g, const Tree &t, const FreqPlan &fp, const bem_params &p);

// Field-point plan: the representation formula (Eq. BIE with lambda = 1) at
// points off the surface through the same plane-wave expansions (Sec. 3.3):
// the points are clustered on the element tree's box grid (boxes outside the
// root cube included), and a point cluster P and an element cluster s of the
// same depth interact in the far field when the element pair test of
// build_plan holds for them (Eq. Farfieldcond with the points' radius, the
// stability test, every point-element distance above R_1 times the square
// root of the largest element area, so the one-point rule of the
// aggregation is the element rule of the field) and the point radius stays
// within the depth's element radius (which sets L); pairs still near at the
// leaf depth are summed directly.
struct EvalLevel {
    int depth = 0, L = 0;
    int npc = 0;                          // point clusters at this depth
    std::vector<int32_t> il_ptr;          // npc + 1
    std::vector<int32_t> il_src, il_off;  // element clusters of this depth, translation rows
    std::vector<double> offsets;          // 3 * noff vectors z_P - z_s
    std::vector<int32_t> pcl;             // per point (internal order): cluster at this depth
    std::vector<double> zp;               // 3 * npc box centres
    int64_t n_inter = 0;
};
struct EvalPlan {
    int leaf_depth = 0;
    std::vector<int64_t> perm;            // internal -> caller point index
    std::vector<int64_t> leaf_start;      // point clusters at leaf_depth: internal ranges (+ end)
    std::vector<EvalLevel> far;           // levels with interactions, coarse to fine
    std::vector<int32_t> near_ptr, near_src;  // per point leaf: element leaves at leaf_depth
    int64_t near_pairs = 0, far_pairs = 0;    // point-element pairs
};
// Returns an empty string or an error message.  max_L: the largest expansion
// length the translation tables support.
std::string build_eval_plan(const Geometry &g, const Tree &t, const bem_params &p, double k, int leaf_depth,
                            const double *pts, int64_t m, int max_L, EvalPlan &ep);

// Sets the calling thread's message returned by bem_last_error.
void set_last_error(const std::string &msg);

// Builds near and interaction lists (Sec. 3.3.4) for wavenumber k.
// leaf_depth < 0: the tree's own leaf depth; otherwise any depth 0..leaf_depth
// (clusters at every depth are runs of the same element order).
// Structural check of a plan before the device kernels index with it: every
// list's pointer array monotone and of the right length, every leaf, cluster
// and translation-row index in range, every leaf near itself, and nnz the
// sum of its near blocks.  Returns an empty string or what is wrong.
std::string validate_plan(const Tree &t, const FreqPlan &fp);

void build_plan(const Geometry &g, const Tree &t, const bem_params &p, double k, FreqPlan &fp,
                int leaf_depth = -1);

}  // namespace bem
