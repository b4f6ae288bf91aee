// bem_kernels.cuh -- kernel argument blocks and kernel declarations.
#pragma once

#include "../../include/bemfmm.h"
#include "bem_device.cuh"

namespace bem {

constexpr int kMaxRestart = 1024;
constexpr int kMaxFarLevels = 16;

// Near columns of a leaf: runs of consecutive elements (the elements of
// consecutive near leaves in Morton order are contiguous); run r covers the
// row positions [runs[r].y, runs[r + 1].y) starting at element runs[r].x.
struct NearDev {
    const int *leaf_of;      // per element: leaf cluster
    const int *run_ptr;      // per leaf (+1): offsets into runs
    const int2 *runs;        // {first element, first row position}
    const int *ncol;         // per leaf: near columns
    const int64_t *row_ptr;  // per element (+1): offsets into the stored values
    const int64_t *leaf_start;  // per leaf (+1): first element (rows of a leaf are contiguous)
};

// Column of row position p for a lane that walks positions upwards; r is the
// lane's current run (advanced monotonically).
__device__ __forceinline__ int near_col(const NearDev &N, int r_end, int &r, int p)
{
    while (r + 1 < r_end && N.runs[r + 1].y <= p) ++r;
    const int2 rr = N.runs[r];
    return rr.x + (p - rr.y);
}

struct NearArgs {
    ElemDev E;
    NearDev N;
    const QuadTables *Q;
    float k, ik_inv;
    float tau;               // +1 exterior, -1 interior problem; cp, cq below already carry it
    const float2 *cp, *cq;   // column coefficients (internal order)
};

struct GmresState {
    int j, done, converged, iters, ncols, maxit;
    double bnorm, beta, resid, tol, hn;
    int reorth;              // second Gram-Schmidt pass needed for the current column
    int n_reorth;            // columns that needed it
    int fault;               // unused (kept zero)
    double nn;               // ||w||^2 after orthogonalisation (k_gs_finish -> k_gm_givens)
    // Skip flag of the product kernels: a copy of done taken by k_gs_dots
    // (in stream order before the next product).  done itself is set by
    // k_gm_givens on a side stream while that product runs, so reading it
    // there could differ between the threads of one block.
    int skip_prod;
    // With several right-hand sides (plane 0's state only): the product
    // kernels skip once every plane's skip_prod is set (k_gm_skip_all).
    int skip_all;
    // Bodies of the device-driven Arnoldi loop run in the current cycle
    // (plane 0's state; k_gm_continue counts, k_gm_start resets).
    int bodies;
};

struct PrepArgs {
    int64_t n;
    const float2 *x;         // input vector (caller order if perm, else internal)
    const int *jidx;         // optional: x += (*jidx) * n
    const int64_t *perm;     // optional: internal -> caller
    float2 *xint;
    float4 *wts;             // far-field weights (alpha, c) per element; may be null
    const float4 *chi, *nrm;
    const float2 *cp, *cq;
    float k;
    int64_t plane;           // element stride between the right-hand sides of xint and wts
    int64_t xplane;          // ... and of x (launch grid.y = number of right-hand sides)
};

// Aggregation work item: `ne` (at most kAggChunk) elements from e0 of
// cluster c and the antipodal direction pairs [p0, p0 + kAggThreads),
// written to row `row` of the multipole buffer (row c when the cluster is
// one element chunk).
constexpr int kAggThreads = 128;
constexpr int kAggChunk = 64;
struct AggTask {
    int c, row;
    int64_t e0;
    int ne;
    int lev;                 // index of the level (in LevelsArgs) the task belongs to
    int red;                 // split cluster: index of its partial-row range (in FarArgs), else -1
    int gred;                // split cluster: index of its arrival counter, else -1
    int p0;                  // first direction pair
};

// Disaggregation work item: elements [x, y) of one leaf, at most kDisTask,
// one block of kDisThreads threads each.
constexpr int kDisTask = 16;
constexpr int kDisThreads = 128;
constexpr int kDisTabChunk = 128;   // direction pairs per staged chunk when the phases are stored

struct FarArgs {
    int nd;                  // 2 L^2 directions
    float k;
    const AggTask *tasks;    // aggregation tasks
    int ntasks;
    const int *red_ptr;      // clusters with several tasks: rows [red_ptr[q], red_ptr[q+1]) ...
    const int *red_c;        // ... are summed into row red_c[q]
    int nred;
    const float4 *dirs;      // (s, w)
    const int *il_ptr, *il_src, *il_off;
    const float2 *D;         // [noff][nd]
    float2 *M, *Lam;         // [nc][nd]
    const int64_t *cstart;   // [nc + 1] element ranges
    const int *is_src;       // [nc]
    const float4 *dz;        // per element: z_c - x_j
    const int *elem_cl;      // per element: cluster at this level
    int64_t mplane, lplane;  // stride (in float2) between the right-hand sides' M and Lam planes
    // stored phases of this level (null when the products regenerate them):
    // ph[j * phs + p] = (cos, sin) of k (z_c - x_j).s_p for every element j
    // and antipodal pair p < nd / 2, rows padded to the even length phs
    const float2 *ph;
    int phs;
};

// Stored far-field phases of every level of a plan, built in one launch
// (k_phase_table): block b fills kPhaseElems elements of level l, where
// start[l] <= b < start[l + 1].
constexpr int kPhaseElems = 16;
struct PhaseLevel {
    const float4 *dz;        // z_c - x_j per element
    const float4 *dirs;      // (s, w) per direction
    float2 *ph;              // [n][phs]
    int h, phs;              // antipodal pairs, row length (h rounded up to even)
};
struct PhaseTableArgs {
    int64_t n;
    float k;
    int nlev;
    PhaseLevel lev[kMaxFarLevels];
    int start[kMaxFarLevels + 1];
};
__global__ void k_phase_table(PhaseTableArgs a);

// All far levels of a plan, for the kernels that run every level in one launch.
struct LevelsArgs {
    int nlev;
    const AggTask *tasks;    // aggregation tasks of every level
    int ntasks;
    const int2 *reds;        // (level, split-cluster index) pairs to sum
    int nreds;
    const int2 *targets;     // (level, target cluster) pairs with interaction lists
    int ntargets;
    const int4 *tgroups;     // transfer blocks: (level, target cluster, first direction, 0)
    int ntgroups;
    unsigned int *red_cnt;   // arrival counters of the split clusters (zero between uses)
    FarArgs lev[kMaxFarLevels];
};

struct DisaggArgs {
    int64_t n;
    const float4 *nrm;
    const int64_t *perm;     // optional
    float k;
    int nlev;
    const int2 *tasks;       // element ranges [x, y) within one leaf, one per block
    const float4 *rowf;      // k_disaggregate_t: per-element row factor (a, b); else unused
    FarArgs lev[kMaxFarLevels];
};

struct SourceDev {
    int kind;
    double v[3];
    double amp[2];
};

constexpr int kHeavyKinds = 8;          // self, subdivided, orders 2 .. 6 (see k_near_classify)
__global__ void k_near_classify(NearArgs a, int2 *heavy, unsigned long long *count, const unsigned long long *off);
__global__ void k_near_store_light(NearArgs a, float2 *val, int *err);
__global__ void k_near_store_heavy(NearArgs a, const int2 *heavy, int64_t nheavy, float2 *val, int *err);
__global__ void k_near_spmv(NearArgs a, const float2 *val, const float2 *x, float2 *y, const int *skip);
// Stored near-field product over work items (leaf, first row, end row),
// one block per item.
constexpr int kSpmvThreads = 128;
constexpr int kSpmvMaxItemRows = 32;
__global__ void k_near_spmv_items(NearArgs a, const int4 *items, const float2 *val, const float2 *x, float2 *y,
                                  const int *skip);
// Transposed product from the stored values: one block per leaf t, the
// rows of its near leaves listed in [trow_ptr[t], trow_ptr[t + 1]) with the
// row element trow_i and the position trow_off of its value at t's first
// element.
constexpr int kSpmvTThreads = 256;
__global__ void k_near_spmv_t(const int64_t *leaf_start, const int *trow_ptr, const int *trow_i,
                              const int64_t *trow_off, const float2 *val, const float2 *x, float2 *y, const int *skip);
// A^T in the layout of A (the near relation of the leaves being symmetric,
// row j of leaf t has the same near columns in both): column c of t's rows
// takes A_i,j for the c-th transposed row i of t (trow_*); pad columns 0.
// One block per leaf; the forward product k_near_spmv_items then streams
// valT as it streams val.
__global__ void k_near_transpose(const int64_t *leaf_start, const int *trow_ptr, const int64_t *trow_off,
                                 const int64_t *row_ptr, const float2 *val, float2 *valT);
// The same for nr <= kMaxPlanes right-hand sides (planes `plane` elements
// apart in x and y): the stored values are streamed once for all of them.
// The leaf's columns are staged in chunks of cw (even) columns: dynamic
// shared memory nr * cw * 8 bytes, small enough for several blocks per SM.
constexpr int kSpmvMultiChunk = 512;
__global__ void k_near_spmv_items_multi(NearArgs a, const int4 *items, const float2 *val, const float2 *x, float2 *y,
                                        int nr, int64_t plane, int cw, const int *skip);
__global__ void k_near_fused(NearArgs a, const float2 *x, float2 *y, int *err, const int *skip);
__global__ void k_prep(PrepArgs a, const int *skip);
// True when the product kernels of a finished GMRES cycle should skip.
__device__ __forceinline__ bool skip_now(const int *skip) { return skip != nullptr && *(volatile const int *)skip != 0; }

// Split cluster (T.red >= 0) of an aggregation launch whose blocks take ppb
// direction pairs each: its blocks are (element chunks) x (pair ranges), and
// the last one to finish sums the partial rows in row order into row T.c of
// every plane (nplanes right-hand sides).  Called by every thread of the
// block after its own rows are written.
__device__ __forceinline__ void aggregate_reduce(const LevelsArgs *A, const AggTask &T, const FarArgs &f, int ppb,
                                                 int nplanes)
{
    if (T.red < 0) return;
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int h = f.nd / 2;
        const int npb = (h + ppb - 1) / ppb;
        const int ntask = (f.red_ptr[T.red + 1] - f.red_ptr[T.red]) * npb;
        last = atomicAdd(&A->red_cnt[T.gred], 1u) == (unsigned)(ntask - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int r0 = f.red_ptr[T.red], r1 = f.red_ptr[T.red + 1];
    const int nd = f.nd;
    const int nt = blockDim.x;
    for (int pl = 0; pl < nplanes; ++pl) {
        const float2 *__restrict__ Mp = f.M + pl * f.mplane;
        float2 *__restrict__ dst = f.M + pl * f.mplane + (int64_t)T.c * nd;
        // each thread sums kRedDirs directions at a time and loads kRedRows
        // rows of them together (L2 loads of other blocks' rows, all in
        // flight at once); every direction still adds its rows in row order
        constexpr int kRedDirs = 4, kRedRows = 4;
        for (int nb = threadIdx.x; nb < nd; nb += nt * kRedDirs) {
            float2 acc[kRedDirs];
#pragma unroll
            for (int b = 0; b < kRedDirs; ++b) acc[b] = make_float2(0.f, 0.f);
            for (int rr = r0; rr < r1; rr += kRedRows) {
                float2 v[kRedRows][kRedDirs];
#pragma unroll
                for (int a = 0; a < kRedRows; ++a)
#pragma unroll
                    for (int b = 0; b < kRedDirs; ++b) {
                        const int nu = nb + b * nt;
                        v[a][b] = (rr + a < r1 && nu < nd) ? __ldcg(Mp + (int64_t)(rr + a) * nd + nu)
                                                           : make_float2(0.f, 0.f);
                    }
#pragma unroll
                for (int a = 0; a < kRedRows; ++a)
#pragma unroll
                    for (int b = 0; b < kRedDirs; ++b) {
                        acc[b].x += v[a][b].x;
                        acc[b].y += v[a][b].y;
                    }
            }
#pragma unroll
            for (int b = 0; b < kRedDirs; ++b)
                if (nb + b * nt < nd) dst[nb + b * nt] = acc[b];
        }
    }
    if (threadIdx.x == 0) A->red_cnt[T.gred] = 0;
}

// Aggregation of NR right-hand sides at once (one phase per element and
// direction pair serves all of them); wts holds NR planes of n elements.
__global__ void k_aggregate_1(const LevelsArgs *A, const float4 *wts, int64_t wplane, const float4 *nrm, const int *skip);
__global__ void k_aggregate_2(const LevelsArgs *A, const float4 *wts, int64_t wplane, const float4 *nrm, const int *skip);
__global__ void k_aggregate_3(const LevelsArgs *A, const float4 *wts, int64_t wplane, const float4 *nrm, const int *skip);
__global__ void k_aggregate_4(const LevelsArgs *A, const float4 *wts, int64_t wplane, const float4 *nrm, const int *skip);
// One right-hand side, with the level's stored phases (FarArgs::ph).
__global__ void k_aggregate_1t(const LevelsArgs *A, const float4 *wts, int64_t wplane, const float4 *nrm, const int *skip);
constexpr int kMaxPlanes = 4;            // right-hand sides per multi-plane launch
// Aggregation on the tensor cores (bem_tc.cu): tasks of one element chunk
// and kTcPairs direction pairs, split-BF16 operands, FP32 accumulation;
// fault is set when the wait for the tensor cores runs out.
constexpr int kTcThreads = 256;
constexpr int kTcPairs = 128;
constexpr int kTcSub = 16;               // elements per pass of the MMAs (a chunk takes up to four)
constexpr size_t kTcSmemBytes = 2 * (size_t)kTcPairs * 4 * kTcSub * 2 + 2 * (size_t)4 * kMaxPlanes * 4 * kTcSub * 2 +
                                1024;
__global__ void k_aggregate_tc(const LevelsArgs *A, const AggTask *tasks, const float4 *wts, int64_t wplane,
                               const float4 *nrm, int nr, int *fault, const int *skip);
__global__ void k_selftest_sincos(const float *x, int64_t n, float4 *out);
// Transfer with the interaction list of one target split among
// kTransferWarps warps: one block per (target, kTransferDirs directions).
constexpr int kTransferDirs = 32;
constexpr int kTransferWarps = 2;          // warps sharing one target's list
constexpr int kTransferUnroll = 8;         // list entries per warp in flight
constexpr int kTransferEntries = 512;     // interaction-list entries staged per pass
__global__ void k_transfer_split(const LevelsArgs *A, const int *skip);
// The same for 2 or 4 right-hand sides (M and Lambda planes mplane and
// lplane apart): each D value is loaded once for all of them.
__global__ void k_transfer_m2(const LevelsArgs *A, const int *skip);
__global__ void k_transfer_m4(const LevelsArgs *A, const int *skip);
// 1, 2 or 4 right-hand sides at once (one phase per element and pair for
// all), element-major with the directions staged in chunks (no dynamic
// shared memory)
__global__ void k_disaggregate_m1(DisaggArgs a, const float2 *ynear, float2 *y, const int *skip);
__global__ void k_disaggregate_m2(DisaggArgs a, const float2 *ynear, float2 *y, const int *skip);
__global__ void k_disaggregate_m4(DisaggArgs a, const float2 *ynear, float2 *y, const int *skip);
__global__ void k_disaggregate_t(DisaggArgs a, const float2 *ynear, float2 *y, const int *skip);
// One right-hand side (m1t) and the transposed product (tt) with the levels'
// stored phases (FarArgs::ph), staged per chunk of kDisTabChunk pairs.
__global__ void k_disaggregate_m1t(DisaggArgs a, const float2 *ynear, float2 *y, const int *skip);
__global__ void k_disaggregate_tt(DisaggArgs a, const float2 *ynear, float2 *y, const int *skip);
// largest expansion length of the translation tables (shared-memory rows)
constexpr int kMaxTableL = 255;
// Translation tables of every far level: block b serves offset
// b - start[l] of the level l with start[l] <= b < start[l + 1].
struct DTableLevel {
    const double *offs;      // [noff][3] offsets z_t - z_s
    const double *dirs;      // [nd][3] directions (first half: one of each antipodal pair)
    float2 *D;               // [noff][nd]
    int nd, L;
};
struct DTableArgs {
    int nlev;
    double k;
    int start[kMaxFarLevels + 1];
    DTableLevel lev[kMaxFarLevels];
};
__global__ void k_dtable(DTableArgs a);
__global__ void k_rhs(const double *cd, const float4 *nrm, int64_t n, double k, const SourceDev *src, int nsrc,
                      float2 *b);
__global__ void k_field(ElemDev E, const QuadTables *Q, const double *pts, int64_t M, float k, float tau,
                        const float2 *p, const float2 *q, const SourceDev *src, int nsrc, float2 *part, float2 *out,
                        int *err);
__global__ void k_field_finish(const double *pts, int64_t M, int S, float k, const SourceDev *src, int nsrc,
                               const float2 *part, float2 *out);
__global__ void k_field_velocity(ElemDev E, const QuadTables *Q, const double *pts, int64_t M, float k, float tau,
                                 float inv_omega_rho, const float2 *p, const float2 *q, const SourceDev *src, int nsrc,
                                 float2 *part, float2 *out, int *err);
__global__ void k_field_velocity_finish(const double *pts, int64_t M, int S, float k, float inv_omega_rho,
                                        const SourceDev *src, int nsrc, const float2 *part, float2 *out);
__global__ void k_gather(const float2 *x, const int64_t *perm, int64_t n, float2 *y);
// FMM evaluation of the field at points (see the definitions)
__global__ void k_field_weights(int64_t n, const float2 *p, const float2 *q, const float4 *chi, float k, float4 *wts);
__global__ void k_field_near(ElemDev E, const QuadTables *Q, const double *pts, int64_t M, float k, const float2 *p,
                             const float2 *q, const int *pleaf, const int *nptr, const int2 *nruns, float2 *v,
                             int *err);
__global__ void k_field_eval_finish(const double *pts, int64_t M, float k, float tau, const SourceDev *src, int nsrc,
                                    const float2 *v, const int64_t *perm, float2 *out);

__global__ void k_near_fused_t(NearArgs a, const float2 *x, float2 *y, float2 *zero, int *err, const int *skip);
__global__ void k_prep_t(int64_t n, const float2 *x, float2 *xint, float4 *wts, float4 *rowf, const float4 *chi,
                         const float2 *cp, const float2 *cq, float k, const int *skip);
__global__ void k_field_t(ElemDev E, const QuadTables *Qp, const double *pts, int64_t M, float k, const float2 *f,
                          const float2 *cp, const float2 *cq, float2 *g_out, float2 *r_out, int *err);
__global__ void k_adjoint_reduce(const float2 *u, const float2 *g, const float2 *aq, const int *region, int64_t n,
                                 float tau, double dre, double dim, const float2 *f, int64_t M, int nreg,
                                 double *acc);
// block-Jacobi sub-blocks: at most kBjMax consecutive elements of one leaf
constexpr int kBjMax = 64;
__global__ void k_bj_factor(NearArgs a, const int4 *blocks, float2 *binv, int *err);
__global__ void k_bj_apply(const int4 *blocks, const float2 *binv, float2 *w, float2 *wnear, const int *skip);
__global__ void k_row_scale_init(NearArgs a, float2 *dinv, int *err);
__global__ void k_row_scale(float2 *y, float2 *y2, const float2 *dinv, int64_t n, const int *skip);
__global__ void k_sub(float2 *b, const float2 *y, int64_t n);
__global__ void k_refine_residual(const float2 *b, const float2 *y, float2 *r, int64_t n, double *part);
__global__ void k_refine_update(double2 *x64, const float2 *d, float2 *x, int64_t n);
__global__ void k_rsub(float2 *w, const float2 *b, int64_t n);
__global__ void k_pq(const float2 *u, const float2 *z, const float2 *aq, const int *type, const int64_t *perm,
                     int64_t n, float2 *p, float2 *q);
struct GmresArgs {
    float2 *V, *w;
    int64_t n;
    GmresState *st;
    int nblk;
    double2 *H, *cs, *sn, *g;
    double *normpart;        // [nblk] norm partials
    int m;
    const double *gs_acc;    // the Gram-Schmidt sums [2][4] (k_gm_givens reads ||v_{j+1}||^2 there)
};

// One Gram-Schmidt step of the Arnoldi process in three launches
// (k_gs_dots, k_gs_update, k_gs_finish) with no waits between blocks: sums
// are FP64 atomic additions of the blocks' partials, read by the next
// launch.  v_{j+1} is stored unnormalised with its squared norm in the sums;
// k_gm_givens takes the norm (h_{j+1,j}) from there, and the next step's
// k_gs_dots scales its rows of v_{j+1} and of the product A v_{j+1} (formed
// from the unnormalised vector; the product is linear).
struct GsArgs {
    GmresArgs g;             // g.nblk = gridDim.x
    PrepArgs next;           // inputs of the next product, formed from V_{j+1}
    const float2 *wnear;     // near-field part of the product (g.w holds the far part)
    double *acc;             // [2][4] per parity of j: ||w||^2, ||w_1||^2, ||w_2||^2, arrival counter
    double2 *h2;             // [2][m + 1] per parity of j: second-pass dots V^H w_1
    int rows;                // rows of the basis per block
};
constexpr int kGsThreads = 256;
constexpr int kGsMaxRows = 1024;    // rows per block staged in shared memory
__global__ void k_gs_dots(GsArgs a);
__global__ void k_gs_update(GsArgs a);
__global__ void k_gs_finish(GsArgs a);
__global__ void k_gm_givens(GmresArgs a);
__global__ void k_gm_skip_all(GmresState *st, int nr);
// Loop condition of the WHILE node of a device-driven Arnoldi cycle: one
// more body while some plane is not done and fewer than max_bodies have run.
__global__ void k_gm_continue(cudaGraphConditionalHandle h, GmresState *st, int nr, int max_bodies);
__global__ void k_gm_backsolve(const GmresState *st, const double2 *H, const double2 *g, double2 *y, int m,
                               int smem_cols);
__global__ void k_gm_xupdate(float2 *x, const float2 *V, int64_t n, const GmresState *st, const double2 *y);
__global__ void k_gm_start(GmresState *st, float2 *V, const float2 *r, int64_t n, const double *normpart, int nblk,
                           double2 *g, int m, int first, double *gs_acc, double2 *gs_h2);
__global__ void k_norm_part(const float2 *r, int64_t n, double *part);

// Host helpers shared by the translation units (bem_capi.cu): the
// quadrature tables of a parameter set (conical rules m = 1..6, the Duffy and
// edge rules, the order thresholds of Sec. 3.1.4) and the medium defaults.
QuadTables make_tables(const bem_params &p);
void medium_of(const bem_medium *m, double &c, double &rho);

}  // namespace bem
