/*
 * bemfmm.h -- C ABI of the GB300 (sm_103a) collocation BEM + fast multipole
 * matrix-vector product for the 3D Helmholtz equation.
 *
 * Method: Kreuzer, Pollack, Brinkmann, Majdak, "NumCalc: An open-source BEM
 * code for solving acoustic scattering problems", arXiv 2312.00005.
 *   - constant elements on flat triangles, collocation at the element
 *     midpoints (Sec. 2.2, 2.3);
 *   - exterior (tau = +1) or interior (tau = -1, bem_params.tau) problem
 *     with Burton-Miller coupling gamma = i/k, Eq. SystemI;
 *   - near field by the quadrature of Sec. 3.1 (Duffy singular rule,
 *     edge-integral hypersingular rule, subdivision while r~ < 1.3, regular
 *     order from the a-priori estimates, m <= 6);
 *   - far field by the plane-wave expansion of Eq. FMMBase with the
 *     truncation of Eq. FMMTruncation and the admissibility of
 *     Eq. Farfieldcond, per level (Sec. 3.3.4: operator
 *     N + sum_l S(l) D(l) T(l));
 *   - restarted GMRES on the device, optionally row-scaled or block-Jacobi
 *     preconditioned (Sec. 3.2);
 *   - beyond the paper: the transposed product and the adjoint gradient of a
 *     field loss with respect to the region admittances
 *     (bem_matvec_transpose, bem_admittance_gradient), and an opt-in check
 *     of the normals' orientation (bem_mesh_check_host).
 *
 * Variables are pressures: p on the surface and q = dp/dn = i w rho v, with
 * n the outward normal (pointing away from the enclosed volume: into the
 * fluid for the exterior problem, App. A, out of it for the interior problem
 * of bem_params.tau = -1) and time factor e^{-i w t}.  Complex numbers are
 * interleaved (re, im): float2 ("cf32") on the device, double[2] on the
 * host.
 *
 * Ownership: every entry point copies what it needs from host arrays before
 * it returns.  Device buffers passed in belong to the caller and must hold the
 * stated number of elements; the library never frees them.  Work is
 * enqueued on the caller's CUDA stream (a cudaStream_t passed as void*;
 * NULL = the legacy default stream) and is stream-ordered.  bem_solve,
 * bem_solve_sweep, bem_admittance_gradient, bem_matvec_host and
 * bem_mesh_stats synchronise the stream before they return;
 * bem_matvec_transpose, bem_evaluate and bem_evaluate_velocity wait for
 * their own work (they read the quadrature's error flag) but leave the
 * caller's stream to its own order; bem_matvec does not wait.
 *
 * Errors: every function returns BEM_OK (0), a negative error code, or a
 * positive warning code with all outputs written.  bem_last_error() gives a
 * message for the calling thread's last non-zero status.  A mesh handle is
 * not thread-safe: one thread at a time per mesh.
 */
#ifndef BEMFMM_H
#define BEMFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BEM_OK                 0
#define BEM_E_ARG             -1  /* invalid argument */
#define BEM_E_SUBDIV_LIMIT    -2  /* more than max_depth nested subdivisions (Sec. 4.1); the
                                     message names the element */
#define BEM_E_CUDA            -3  /* a CUDA call failed */
#define BEM_E_OOM             -4  /* device allocation failed */
#define BEM_E_TIMEOUT         -5  /* a bounded device wait gave up: the tensor-core aggregation's
                                      wait for its own MMAs (far_precision 1); no device code of
                                      this library waits on another block or launch */
#define BEM_E_INTERNAL        -6
#define BEM_W_NOT_CONVERGED    1  /* GMRES stopped at max_iter above tol (cf. Sec. 3.2 warning) */
#define BEM_W_UNDERRESOLVED    2  /* mean edge longer than a sixth of the wavelength (Sec. 2.2) */

/* boundary condition per element (App. A, App. C.3); VELO with v = 0 is
 * sound hard and is the default */
#define BEM_VELO 0  /* normal particle velocity v given            */
#define BEM_PRES 1  /* pressure p given                             */
#define BEM_ADMI 2  /* admittance Y of the element's region (velocity into the wall = Y p),
                       plus an optional extra normal velocity        */

#define BEM_MODE_FMM    0  /* near field by quadrature + plane-wave FMM far field */
#define BEM_MODE_DIRECT 1  /* every pair by quadrature (conventional BEM)          */

#define BEM_SRC_PLANE 0    /* p = P0 e^{ik d.x}, d a unit direction (App. C.4)     */
#define BEM_SRC_POINT 1    /* p = P0 e^{ikR}/(4 pi R), R = |x - x0| (Eq. PointSrc) */

typedef struct bem_params {
    int32_t mode;           /* BEM_MODE_FMM (default) or BEM_MODE_DIRECT                      */
    double  quad_tol;       /* a-priori quadrature tolerance, 1e-3 (Sec. 3.1.4)                */
    int32_t m_max;          /* cap on the regular order, 6 (Sec. 3.1.4), 1..6                  */
    double  rt_subdiv;      /* subdivide while r~ < rt_subdiv, 1.3 (Sec. 3.1.3)                */
    int32_t max_depth;      /* subdivision limit, 15 (Sec. 4.1)                                */
    double  trunc_factor;   /* factor of Eq. FMMTruncation, 1.8                                */
    int32_t L_min;          /* lower bound of the expansion length, 8 (Eq. FMMTruncation)      */
    double  admissibility;  /* far if |z_i - z_j| > admissibility (r_i + r_j); 2/sqrt(3)        */
    double  leaf_edge;      /* leaf box edge in metres; 0 = chosen from the mesh               */
    double  stability_max;  /* far only if sum_n (2n+1)|h_n(kX)| / |h_0(kX)| <= this, 1e3     */
    int32_t near_store;     /* 1: store near-field entries per frequency (default);
                               0: recompute them inside every product                         */
    int32_t restart;        /* GMRES restart length, 100 (2..1024)                             */
    int32_t autotune;       /* 1: choose the leaf size by timing candidates on the GPU at the
                               mesh's first plan (when leaf_edge is 0; default); 0: off       */
    double  tau;            /* +1: exterior problem (default); -1: interior problem, the field
                               inside the closed surface (Eq. BIE_I, Eq. SystemI: the sign of
                               every integral operator).  Normals point away from the enclosed
                               volume in both cases (Sec. 2.1).  Other values: BEM_E_ARG.    */
    int32_t row_scaling;    /* 1: row-scaling preconditioner of the iterative solver (Sec. 3.2):
                               bem_solve / bem_solve_sweep run GMRES on D^-1 A u = D^-1 b with
                               D = diag(A) (the self entries), and tol and relres refer to
                               that scaled residual; the solution is that of A u = b.
                               0: off (default).  Other values: BEM_E_ARG.                    */
    int32_t check_orientation; /* 1: bem_mesh_create rejects (BEM_E_ARG, before any device work)
                               a mesh that is not closed and consistently wound or whose normals
                               point into the enclosed volume (bem_mesh_check_host); the paper
                               leaves this to the user (Sec. 2.1).  0: off (default).         */
    int32_t symmetric_far;  /* 1: a cluster pair is far only if r~ > R_1 holds with the larger
                               of the two clusters' element areas, so its verdict is the same
                               both ways and bem_matvec_transpose is the exact transpose of
                               bem_matvec (asymmetric_pairs = 0) at the cost of a few more
                               near pairs; 0 (default): the source cluster's area, the bound
                               r~ of Sec. 3.1.4 needs.  Other values: BEM_E_ARG.              */
    int32_t block_jacobi;   /* 1: block-Jacobi preconditioner, the block form of the row scaling
                               of Sec. 3.2: bem_solve / bem_solve_sweep run GMRES on
                               P A u = P b with P the inverse of A's block diagonal over the
                               leaf boxes of the plan (each split into runs of at most 64
                               elements; bem_mesh_blocks lists them), and tol and relres refer
                               to that preconditioned residual; the solution is that of
                               A u = b.  0: off (default).  Not together with row_scaling;
                               other values: BEM_E_ARG.                                        */
    int32_t far_precision;  /* arithmetic of the aggregation T(l) (Sec. 3.3.3) in the forward
                               products: 0 (default) FP32 on the CUDA cores; 1 split BF16 on
                               the tensor cores (every operand as a sum of two BF16 parts,
                               three products accumulated in FP32; a few 1e-6 relative, see
                               bem_solve_multi for the refinement that recovers the FP32
                               form's accuracy).  Other values: BEM_E_ARG.                     */
    int32_t near_chunk;     /* stored near-field product: columns of a leaf's near list staged
                               in shared memory per pass.  0 (default): the library's choice
                               (every column at once for one right-hand side, 512 for
                               several); an even number in 64..4096: that many for any
                               number of right-hand sides.  Results agree to rounding order
                               of the row sums.  Other values: BEM_E_ARG.                     */
    int32_t gs_rows;        /* GMRES Gram-Schmidt step: rows of the basis per block (its sums
                               are FP64 atomic additions of the blocks' partials, one per
                               basis column and block).  0 (default): 128, or more to keep the
                               blocks at most 1024; 64..1024 otherwise.  Results agree to the
                               summation order.  Other values: BEM_E_ARG.                     */
    int32_t field_mode;     /* bem_evaluate: 1 the direct sum over every element with the rules
                               of Sec. 3.1 at each point; 2 (FMM meshes) near elements by the
                               same rules and the rest through the plane-wave expansions of
                               Sec. 3.3 (the points clustered on the element tree's grid, the
                               far test of the lists with the points as targets, the
                               one-point rule beyond R_1; the point plan is kept for the next
                               call with the same points and frequency); 0 (default): 2 on an
                               FMM mesh from 1e9 point-element pairs, else 1.  Other values:
                               BEM_E_ARG.                                                      */
    int32_t far_table;      /* phases e^{ik (z_c - x_j).s} of the aggregation T(l) and, conjugated,
                               of the disaggregation S(l) (Sec. 3.3.3) in products with one
                               right-hand side (and the transposed product): 0 (default)
                               regenerated in every product (one sine and cosine per element
                               and antipodal direction pair); 1 computed once per frequency
                               for every level, element and pair and stored, 8 bytes each
                               (64 MB for 20,480 elements and 389 pairs over three levels), as
                               the paper stores T and S, unless that would exceed 4 GiB; the
                               products then read them instead.  The stored values are those
                               the products regenerate, so the results are the same.
                               Products with several right-hand sides always regenerate them
                               (one phase serves all their planes).  Other values: BEM_E_ARG. */
    int32_t graphs;         /* GMRES launches: 1 (default) each restart cycle is one CUDA graph
                               launch (a conditional WHILE node over bodies of four Arnoldi
                               steps, the condition set on the device); 0 the steps are launched
                               one at a time with a status read after each (for profilers that
                               do not see into conditional graph nodes).  Same kernels, same
                               results.  Other values: BEM_E_ARG.                             */
    int32_t near_transpose; /* transposed product (bem_matvec_transpose, the adjoint solve of
                               bem_admittance_gradient) with the stored near field: 1 (default)
                               A^T is stored once per frequency in the layout of A (8 bytes
                               per stored value more, made from A's values when the near lists
                               are symmetric) and streamed like A; 0 A's values are read by
                               column.  Results agree to the rounding of the sums.  Other
                               values: BEM_E_ARG.                                             */
} bem_params;

typedef struct bem_medium {
    double c;    /* speed of sound, m/s (343 if <= 0) */
    double rho;  /* density, kg/m^3 (1.21 if <= 0)    */
} bem_medium;

typedef struct bem_source {
    int32_t kind;    /* BEM_SRC_PLANE or BEM_SRC_POINT                    */
    double  vec[3];  /* unit direction (plane) or position in m (point)   */
    double  amp[2];  /* complex amplitude P0 in Pa (re, im)               */
} bem_source;

typedef struct bem_solve_info {
    int32_t iterations;       /* matrix-vector products in GMRES              */
    int32_t restarts;
    double  relres;           /* final ||b - A u|| / ||b|| (GMRES estimate; of the
                                 row-scaled system when row_scaling is on)     */
    double  seconds;          /* wall time of the call                         */
    int32_t levels;           /* FMM levels with interaction lists             */
    int32_t L[16];            /* expansion length per used level, finest last  */
    int64_t near_nnz;         /* stored near-field entries                     */
    int32_t status;           /* same as the return value                      */
    double  setup_seconds;    /* plan, coefficients and near-field entries     */
    double  rhs_seconds;      /* incident field and known boundary data        */
    double  gmres_seconds;    /* GMRES iterations (graph build included)       */
} bem_solve_info;

typedef struct bem_plan_stats {
    int64_t n_elements;
    int32_t leaf_level;         /* octree depth of the leaves                          */
    int32_t levels;             /* levels with interaction lists                       */
    int32_t level_depth[16];    /* octree depth of each used level, coarse to fine     */
    int32_t L[16];              /* expansion length per used level                     */
    int32_t n_clusters[16];     /* clusters per used level                             */
    int64_t n_interactions[16]; /* interaction-list entries per used level             */
    int32_t n_offsets[16];      /* distinct translation offsets per used level         */
    int32_t n_leaves;
    int64_t near_nnz;           /* near-field element pairs (with the diagonal)        */
    int64_t near_quad_points;   /* quadrature points summed over the near pairs        */
    double  leaf_edge;          /* metres                                              */
    double  mean_edge;          /* mean element edge length, metres                    */
    int64_t device_bytes;       /* device memory held by the mesh and this plan        */
    int64_t far_pairs;          /* element pairs covered by the interaction lists;
                                   near_nnz + far_pairs = n_elements^2                  */
    int32_t n_tuned;            /* leaf depths the autotuner timed (0: not run)        */
    int32_t tuned_depth[4];     /* ... their octree depths                             */
    double  tuned_seconds[4];   /* ... estimated seconds per solve (entries + 40 products) */
    int64_t asymmetric_pairs;   /* element pairs of list entries without a mirror: near leaf
                                   pairs (a, b) without (b, a) plus interaction entries
                                   (t, s) without (s, t), each weighted by its clusters'
                                   sizes.  The far test bounds r~ with the source cluster's
                                   largest element area (Sec. 3.1.4 measures r~ against the
                                   source element), so a pair can be far one way and near
                                   the other; bem_matvec_transpose reads the lists backwards
                                   and applies, on these pairs, the other direction's rule */
    double  order_R[8];         /* the order thresholds of Sec. 3.1.4 the plan uses: the
                                   regular order is m when r~ > order_R[m] (m = 1 .. m_max - 1,
                                   smallest such m), else m_max; order_R[0] = rt_subdiv      */
    int64_t near_light_entries; /* near pairs under one regular rule of order 1..3 over the
                                   whole element (the light entry kernel) ...               */
    int64_t near_light_points;  /* ... and their quadrature points (m^2 each)              */
    int64_t near_heavy_entries; /* self terms, subdivided pairs and orders 4..6 ...         */
    int64_t near_heavy_points;  /* ... and their kernel evaluations: a self term takes
                                   6 x 16 Duffy points and 3 x 4 x 3 edge points, a
                                   subdivided pair m^2 points per leaf subelement;
                                   near_quad_points = near_light_points + near_heavy_points */
    int64_t n_src_elements[16]; /* per used level: elements of the clusters that are
                                   interaction sources (aggregated: L^2 antipodal direction
                                   pairs each, Sec. 3.3.3 T(l))                             */
    int64_t n_tgt_elements[16]; /* per used level: elements of the clusters with an
                                   interaction list (disaggregated, S(l))                   */
    int64_t asymmetric_near_pairs; /* the part of asymmetric_pairs from near leaf pairs: 0
                                   lets bem_matvec_transpose read the stored values      */
} bem_plan_stats;

/* Paper defaults (Sec. 3.1, Eq. FMMTruncation, Eq. Farfieldcond). */
void bem_params_default(bem_params *p);

/* Create a mesh (App. A): nodes [n_nodes][3] in metres, tris [n_tris][3]
 * 0-based node indices in counter-clockwise order seen from outside the
 * enclosed volume (outward normal: into the fluid for the exterior problem,
 * out of it for the interior one; not checked, Sec. 2.1).  bc_type [n_tris] (NULL = all
 * BEM_VELO), bc_value [n_tris][2] complex (NULL = 0): p for PRES, v for
 * VELO, the extra velocity for ADMI.  region [n_tris] (NULL = 0) selects the
 * admittance entry of ADMI elements.  params NULL = defaults.  Geometry,
 * clustering and the frequency-independent plan are built here, and the
 * mesh is copied to the current CUDA device.  *out receives the handle. */
int bem_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris,
                    const int32_t *bc_type, const double *bc_value, const int32_t *region,
                    const bem_params *params, void **out);

int bem_mesh_destroy(void *mesh);

/* y = A x for n_rhs right-hand sides (Eq. SystemI with the mesh's tau), where A is the
 * Burton-Miller matrix in the unknowns u (p on VELO / ADMI elements, q on
 * PRES elements) with the boundary conditions folded in: column j enters as
 * p_j = c^p_j u_j and q_j = c^q_j u_j with (c^p, c^q) = (1, 0) for VELO,
 * (1, -tau ik rho c Y) for ADMI (Y = velocity into the wall / p) and (0, 1)
 * for PRES.
 * x_dev, y_dev: device cf32 [n_rhs][n_tris] in the caller's element order.
 * admittance: host double [n_regions][2] (Y in m/(Pa s)); may be NULL when
 * no element is ADMI.  Builds (or reuses) the plan for this frequency. */
int bem_matvec(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
               int32_t n_regions, const void *x_dev, void *y_dev, int32_t n_rhs, void *stream);

/* y = A^T x (the transpose of bem_matvec's A, one right-hand side), the
 * product of the adjoint solve in bem_admittance_gradient.  It reads the near
 * and interaction lists backwards: exact where the near/far verdict of a
 * pair is the same both ways; on the pairs counted by
 * bem_plan_stats.asymmetric_pairs it takes the other direction's rule (the
 * plane-wave expansion where A used quadrature of a higher order, or the
 * reverse), which agree within the quadrature tolerance and the truncation.
 * Near part: the same entries as A: from the stored values (near_store = 1)
 * when every near leaf pair of the plan has its mirror (A^T stored once per
 * frequency in A's layout and streamed like A, near_transpose = 1, or A read
 * by column, near_transpose = 0 or no room for A^T), else recomputed by
 * quadrature in every call.  Far part (FMM mode): the antipodal symmetry of the sphere grid of
 * Sec. 3.3.3 and D(-X, s) = D(X, -s) in Eq. FMMBase make it the forward
 * aggregation of x with the source factor 1 - s.n, the forward transfer and
 * a disaggregation with A's column factor A_j (c^q_j - ik c^p_j s.n_j) as
 * its row factor.  x_dev, y_dev: device cf32 [n_tris], caller order.
 * Arguments and errors as bem_matvec. */
int bem_matvec_transpose(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                         int32_t n_regions, const void *x_dev, void *y_dev, void *stream);

/* As bem_matvec with host buffers x_host, y_host (cf32 [n_rhs][n_tris]):
 * copies in, multiplies, copies out, synchronises. */
int bem_matvec_host(void *mesh, double freq_hz, const bem_medium *medium,
                    const double *admittance, int32_t n_regions, const void *x_host,
                    void *y_host, int32_t n_rhs, void *stream);

/* Solve Eq. SystemI at one frequency for the incident field of n_src
 * sources and the mesh's boundary data, with restarted GMRES on the device
 * (classical Gram-Schmidt with a second pass when the first cancels more
 * than half of the vector, its sums FP64 additions of FP32 block partials;
 * FP64 Hessenberg matrix and Givens rotations; FP32 products and basis;
 * each restart cycle one CUDA graph launch, see bem_params.graphs).  Writes the
 * surface pressure p_dev and q_dev = dp/dn (device cf32 [n_tris] each, caller
 * order; q_dev may be NULL).  tol: relative residual target (e.g. 1e-6).
 * max_iter: cap on products.  info may be NULL.  Returns BEM_OK,
 * BEM_W_NOT_CONVERGED (outputs hold the last iterate), or an error. */
int bem_solve(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
              int32_t n_regions, const bem_source *srcs, int32_t n_src, double tol,
              int32_t max_iter, void *p_dev, void *q_dev, bem_solve_info *info, void *stream);

/* Several right-hand sides at one frequency (the paper's input can list
 * several plane waves and point sources, App. C.4; here each source is its
 * own right-hand side instead of one summed incident field): solves
 * Eq. SystemI for n_rhs (1..4) systems A u_r = b_r that share the matrix, as
 * n_rhs calls of bem_solve with srcs + r would, with GMRES on the device for
 * all of them in lockstep: every product takes the n_rhs basis vectors in
 * one pass (the stored near field streamed once, one phase per element and
 * direction pair for all of them), while each system keeps its own Krylov
 * basis, Hessenberg matrix and convergence test.
 *   srcs: host [n_rhs], source r makes right-hand side r (the mesh's
 *   boundary data enter every one); p_dev, q_dev: device cf32
 *   [n_rhs][n_tris] (q_dev may be NULL); infos: host [n_rhs] or NULL.
 * Returns BEM_OK, BEM_W_NOT_CONVERGED (some system stopped at max_iter; its
 * info says which), BEM_W_UNDERRESOLVED or an error. */
int bem_solve_multi(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                    int32_t n_regions, const bem_source *srcs, int32_t n_rhs, double tol, int32_t max_iter,
                    void *p_dev, void *q_dev, bem_solve_info *infos, void *stream);

/* Frequency sweep (the paper solves the frequencies of a sweep
 * independently and splits sweeps into frequency ranges, appendix
 * "Command-line parameters", subsection Parallelization; the overlap below
 * is this library's own): solves Eq. SystemI at n_freq frequencies freqs_hz
 * (host) in order, as n_freq calls of bem_solve would, with the same
 * arguments per frequency and the same results.  While the GMRES of
 * frequency i runs, a host thread prepares frequency i + 1 (its plan,
 * translation tables and near-field entries) on a second stream and set of
 * buffers, so that work overlaps the solve.
 *   p_dev, q_dev: device cf32 [n_freq][n_tris] (q_dev may be NULL when
 *   n_pts = 0); pts: host double [n_pts][3] field points (may be NULL with
 *   n_pts = 0); field_dev: device cf32 [n_freq][n_pts], the field (Eq. BIE_I
 *   with lambda = 1, as bem_evaluate) at each frequency; infos: host
 *   [n_freq] or NULL.
 * Returns on the first error (the outputs of earlier frequencies are
 * written); otherwise BEM_OK or the first warning met (its message in
 * bem_last_error).  The caller's stream is joined and synchronised. */
int bem_solve_sweep(void *mesh, const double *freqs_hz, int32_t n_freq, const bem_medium *medium,
                    const double *admittance, int32_t n_regions, const bem_source *srcs, int32_t n_src,
                    double tol, int32_t max_iter, void *p_dev, void *q_dev, const double *pts,
                    int64_t n_pts, void *field_dev, bem_solve_info *infos, void *stream);

/* Total pressure at M field points (Eq. BIE_I with lambda = 1), outside the
 * surface for the exterior problem, inside it for the interior one:
 * p(x) = p_inc(x) + tau sum_j [H(x)_j p_j - G(x)_j q_j], element integrals by
 * the regular / quasi-singular rules measured from x.  p_dev, q_dev: device
 * cf32 [n_tris] (caller order, as written by bem_solve).  pts: host double
 * [M][3].  out_dev: device cf32 [M].  M = 0 returns BEM_OK at once (pts and
 * out_dev may then be NULL). */
int bem_evaluate(void *mesh, double freq_hz, const bem_medium *medium, const bem_source *srcs,
                 int32_t n_src, const void *p_dev, const void *q_dev, const double *pts,
                 int64_t M, void *out_dev, void *stream);

/* Particle velocity at M field points (Eq. utopandv: v = grad p / (i w
 * rho); the paper writes its x, y and z components per evaluation point,
 * appendix Output, file vEvalGrid): grad p(x) = grad p_inc(x) +
 * tau sum_j [grad H(x)_j p_j - grad G(x)_j q_j], i.e. Eq. BIE_I (lambda = 1)
 * differentiated under the integral, with the element rules of
 * bem_evaluate.  rho from medium.  p_dev, q_dev: device cf32 [n_tris]
 * (caller order, as written by bem_solve).  pts: host double [M][3].
 * v_out_dev: device cf32 [M][3] (x, y, z components of each point).
 * Errors as for bem_evaluate. */
int bem_evaluate_velocity(void *mesh, double freq_hz, const bem_medium *medium, const bem_source *srcs,
                          int32_t n_src, const void *p_dev, const void *q_dev, const double *pts, int64_t M,
                          void *v_out_dev, void *stream);

/* Gradient of a field loss with respect to the region admittances, by the
 * adjoint of the discrete system (a derived quantity: the paper solves the
 * forward problem of Eq. SystemI only).  L = sum_m |p(x_m)|^2 with p the
 * total pressure of Eq. BIE_I (lambda = 1, as bem_evaluate) at the n_pts
 * points pts (host double [n_pts][3]); the parameters are the admittances
 * Y_r of the regions (admittance: host double [n_regions][2], as for
 * bem_solve), entering column j of an ADMI element as c^q_j = -tau ik rho c
 * Y_r.  Steps: the forward solve (as bem_solve: p_dev, q_dev receive p and
 * q, device cf32 [n_tris], caller order; info its statistics), the field
 * f at the points, one adjoint GMRES solve A^T lambda = F^T conj(f) (F the
 * map from the unknowns to the field), and per element of region r the term
 * d u_j (-tau (G_f^T conj f)_j - (A_q^T lambda)_j), d = -tau ik rho c, A_q
 * the operator on q-unknowns.  Writes *loss = L and grad (host double
 * [n_regions][2]) = dL/dRe Y_r + i dL/dIm Y_r.
 * The adjoint solve uses the transposed product of bem_matvec_transpose
 * (FMM or direct, as the mesh's mode).  Returns BEM_OK, BEM_W_NOT_CONVERGED
 * (either solve; outputs filled from the last iterates) or an error. */
int bem_admittance_gradient(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                            int32_t n_regions, const bem_source *srcs, int32_t n_src, const double *pts,
                            int64_t n_pts, double tol, int32_t max_iter, void *p_dev, void *q_dev, double *loss,
                            double *grad, bem_solve_info *info, void *stream);

/* Orientation diagnostics of a closed triangle surface, host only (no
 * device work).  The paper requires the normals to point away from the
 * scatterer, into the fluid of an exterior problem, and leaves the check to
 * the user (Sec. 2.1: inward normals swap the interior and exterior
 * problems; App. A).  volume: the signed enclosed volume
 * (1/3) sum_j A_j (x_j . n_j), x_j the midpoint, n_j = (b - a) x (c - a) / |.|
 * (divergence theorem; positive when every normal points out of the
 * enclosed volume); open_edges: edges not shared by exactly two triangles;
 * misoriented_edges: shared edges that both triangles traverse in the same
 * direction.  Any output may be NULL.  Errors: BEM_E_ARG (bad index,
 * degenerate triangle), BEM_E_OOM. */
int bem_mesh_check_host(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris, double *volume,
                        int64_t *open_edges, int64_t *misoriented_edges);

/* Plan statistics for a frequency (builds the plan if needed). */
int bem_mesh_stats(void *mesh, double freq_hz, const bem_medium *medium, bem_plan_stats *out);

/* The sub-blocks of the block-Jacobi preconditioner (bem_params.block_jacobi)
 * in the plan for a frequency: block_of (host int32 [n_tris], caller order)
 * receives each element's sub-block index.  Sub-blocks are the leaf boxes of
 * the plan's octree, each split into runs of at most 64 elements of its
 * Morton-ordered element list.  Builds the plan if needed. */
int bem_mesh_blocks(void *mesh, double freq_hz, const bem_medium *medium, int32_t *block_of);

/* The field-point plan of bem_evaluate's FMM path (field_mode 2), computed on
 * the host only (no CUDA call) with the tree of bem_plan_stats_host: pts is
 * host double [n_pts][3] in metres. */
typedef struct bem_field_stats {
    int32_t leaf_level;          /* depth of the point leaves                           */
    int32_t levels;              /* depths with point-cluster interactions               */
    int32_t level_depth[16];
    int32_t L[16];               /* expansion length per level (Eq. FMMTruncation)       */
    int32_t n_point_clusters[16];
    int64_t n_interactions[16];  /* (point cluster, element cluster) list entries        */
    int32_t n_offsets[16];       /* distinct translation vectors                         */
    int64_t near_pairs;          /* point-element pairs summed by the element rules ...  */
    int64_t far_pairs;           /* ... and through the expansions: together
                                    n_pts x n_tris                                       */
    int64_t n_point_leaves;
} bem_field_stats;
int bem_field_plan_stats_host(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris,
                              const double *pts, int64_t n_pts, const bem_params *params, double freq_hz,
                              double c, bem_field_stats *out);

/* The same statistics computed on the host only (no CUDA call): geometry,
 * clustering and the near / interaction lists of Sec. 3.3.4 for the given
 * frequency and speed of sound.  device_bytes is 0. */
int bem_plan_stats_host(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris,
                        const bem_params *params, double freq_hz, double c, bem_plan_stats *out);

/* Free the per-frequency plan of a mesh (lists, translation tables, stored
 * near-field entries); the next call at any frequency rebuilds it. */
int bem_mesh_release_plan(void *mesh);

/* Kernel timing with CUDA events recorded on the library's own stream around
 * every kernel it launches (the GMRES step is then launched kernel by kernel
 * instead of as a CUDA graph).  enable = 1 starts (and clears) the record,
 * 0 stops it.  bem_timing_get returns, for the kernel named `name` (e.g.
 * "k_near_spmv"), the summed milliseconds and the number of launches
 * resolved so far; it returns BEM_E_ARG for a name never timed. */
int bem_timing_enable(int enable);
int bem_timing_get(const char *name, double *total_ms, int64_t *launches);

/* Self-test of the far-field sine/cosine of 2 pi t, t in turns (an exact
 * reduction to [-1/2, 1/2] turn followed by the SFU approximations; no
 * counterpart in the paper): for n device floats x_dev (= t) writes device
 * float4 out_dev[i] = (sin, cos by the library's routine, sin, cos by CUDA's
 * sincospif(2 t)).  Stream-ordered, no synchronisation. */
int bem_selftest_sincos(const void *x_dev, int64_t n, void *out_dev, void *stream);

/* Direct product without device allocation (the paper has no counterpart;
 * it exists for callers that must not call cudaMalloc while running, such
 * as real-time or embedded pipelines that reserve all device memory at
 * start-up, or hosts whose own allocator owns the device, and that therefore
 * cannot create a mesh handle).  Computes y = A x, A the conventional dense
 * Burton-Miller matrix (every pair by the quadrature of Sec. 3.1, no FMM) of
 * a sound-hard surface (all elements VELO with v = 0, unknown p) for the
 * exterior problem (tau = +1).
 *   nodes_dev: device double [n_nodes][3]; tris_dev: device int32 [n_tris][3]
 *   (counter-clockwise); x_dev, y_dev: device cf32 [n_tris]; medium may be
 *   NULL (c = 343 m/s).
 * Everything it derives from the mesh lives in one fixed 8 MiB array
 * compiled into the library (held on every GPU that loads the library until
 * the process exits), so n_tris is limited to 32768; larger meshes are
 * rejected with BEM_E_ARG and a message.  It calls no allocating routine.
 * The first call on a device (and the first after that device's CUDA
 * context was replaced, e.g. by cudaDeviceReset) looks up that array's
 * device address in the current context; later calls reuse it.  All calls on
 * a device share the array and each call overwrites it: calls that overlap on
 * the GPU race.  Work is enqueued on `stream`; the call synchronises that
 * stream before it returns (to report degenerate elements or the subdivision
 * limit), so it must not be called while that stream is being captured into
 * a CUDA graph.  medium as for the mesh entry points (NULL, or c <= 0: 343
 * m/s). */
int bem_matvec_direct_noalloc(const double *nodes_dev, int64_t n_nodes, const int32_t *tris_dev, int64_t n_tris,
                              double freq_hz, const bem_medium *medium, const void *x_dev, void *y_dev,
                              void *stream);

/* Test hook for the library's own allocation-failure path (no counterpart
 * in the paper), so that tests reach it without exhausting the device.
 * Process-wide.
 *   alloc_fail_after >= 0: that many further device allocations succeed and
 *     the next one is refused without calling cudaMalloc (the entry point
 *     returns BEM_E_OOM and frees what it had allocated); < 0: off.
 *   live_device_bytes (may be NULL): bytes the library holds in device
 *     allocations (every mesh's buffers) at the time of the call. */
int bem_test_hooks(int64_t alloc_fail_after, int64_t *live_device_bytes);

/* The Krylov basis of the last GMRES cycle of the mesh's last solve (no
 * counterpart in the paper; for measuring the orthogonality of the FP32
 * basis): right-hand side `plane` (0 for bem_solve), its ncols normalised
 * basis vectors V_0 .. V_{ncols-1} (Arnoldi step ncols - 1 was the last),
 * each n_tris complex float32 values in the library's internal element
 * order (one permutation for all, so V^H V is unchanged).  v_dev: device
 * buffer of max_cols * n_tris cf32, receives min(ncols, max_cols) vectors
 * one after the other; *n_cols receives ncols.  Waits for the copy.  Errors:
 * BEM_E_ARG (bad argument, plane out of range or no solve yet). */
int bem_krylov_basis(void *mesh, int32_t plane, void *v_dev, int32_t max_cols, int32_t *n_cols);

/* Number of kernels this library has launched in this process. */
uint64_t bem_launch_count(void);

/* Message of the calling thread's last non-zero status ("" if none). */
const char *bem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BEMFMM_H */
