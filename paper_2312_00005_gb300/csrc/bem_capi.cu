// bem_capi.cu -- implementation of the C ABI declared in include/bemfmm.h:
// mesh set-up, per-frequency plans, the FMM matrix-vector product, the
// device-resident GMRES driver and the field evaluation.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/bemfmm.h"
#include "bem_kernels.cuh"
#include "bem_plan.hpp"

using namespace bem;

// Largest stored far-field phase table of a plan (far_table); above it the
// products regenerate the phases.
constexpr double kPhaseTableMaxBytes = 4.0 * 1024 * 1024 * 1024;
// bem_evaluate with field_mode 0 takes the FMM path from this many
// point-element pairs (below it the direct sum takes about as long as the
// host build of the point plan)
constexpr double kFieldFmmMinPairs = 1e9;
// Arnoldi steps captured in one CUDA graph (one status read per graph)
constexpr int kStepsPerGraph = 4;
// values per work item of the stored near-field product
constexpr int64_t kSpmvItemEntries = 65536;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};

// optional per-kernel event timing (see bem_timing_enable)
#include <map>
#include <mutex>
static bool g_timing = false;
static std::mutex g_tmu;
struct TimingRec {
    const char *name;
    cudaEvent_t a, b;
};
static std::vector<TimingRec> g_pending;
static std::vector<cudaEvent_t> g_pool;
static std::map<std::string, std::pair<double, int64_t>> g_tacc;

namespace bem {
// Sets the calling thread's message returned by bem_last_error.
void set_last_error(const std::string &msg) { g_err = msg; }

// ------------------------------------------------------------------ tables
QuadTables make_tables(const bem_params &p)
{
    QuadTables Q;
    memset(&Q, 0, sizeof Q);
    for (int m = 1; m <= kMaxRule; ++m) {
        std::vector<double> xi, eta, w;
        conical_rule(m, xi, eta, w);
        for (int q = 0; q < m * m; ++q) {
            Q.tri_xi[m][q] = (float)xi[q];
            Q.tri_eta[m][q] = (float)eta[q];
            Q.tri_w[m][q] = (float)w[q];
        }
    }
    std::vector<double> x, w;
    gauss_legendre01(4, x, w);
    for (int i = 0; i < 4; ++i) { Q.gl4_x[i] = (float)x[i]; Q.gl4_w[i] = (float)w[i]; }
    gauss_legendre01(3, x, w);
    for (int i = 0; i < 3; ++i) { Q.gl3_x[i] = (float)x[i]; Q.gl3_w[i] = (float)w[i]; }
    double R[kMaxRule + 1] = {0};
    order_thresholds(p.quad_tol, p.m_max, R);
    for (int m = 1; m < p.m_max; ++m) {
        Q.R[m] = (float)R[m];
        Q.Rd[m] = R[m];
        Q.R2[m] = (float)(R[m] * R[m]);
    }
    Q.heavy_rt2 = p.m_max > 3 ? (float)((R[3] * (1.0 + 1e-5)) * (R[3] * (1.0 + 1e-5))) : 0.f;
    Q.rt_sub = (float)p.rt_subdiv;
    Q.rt_sub_d = p.rt_subdiv;
    Q.m_max = p.m_max;
    Q.max_depth = p.max_depth;
    Q.edge_parts = 4;
    return Q;
}

// c and rho of a medium (NULL or non-positive values: 343 m/s, 1.21 kg/m^3)
void medium_of(const bem_medium *m, double &c, double &rho)
{
    c = (m && m->c > 0) ? m->c : 343.0;
    rho = (m && m->rho > 0) ? m->rho : 1.21;
}
}  // namespace bem

namespace {

struct Fail {
    int code;
};

int set_err(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

void ck(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        g_err = std::string(what) + ": " + cudaGetErrorString(e);
        throw Fail{e == cudaErrorMemoryAllocation ? BEM_E_OOM : BEM_E_CUDA};
    }
}

void ck_launch(const char *what)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ck(cudaGetLastError(), what);
}

cudaEvent_t pool_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    ck(cudaEventCreate(&e), "cudaEventCreate");
    return e;
}

// Records an event pair around the kernel launched in its scope when timing
// is on and the stream is not being captured.
// NVTX range over a scope, so that profilers show the library's calls and
// phases by name (without a tool attached a push or pop only checks a
// function pointer).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct KTimer {
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    KTimer(const char *n, cudaStream_t st) : name(n), s(st)
    {
        if (!g_timing) return;
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        std::lock_guard<std::mutex> lk(g_tmu);
        a = pool_event();
        cudaEventRecord(a, s);
    }
    ~KTimer()
    {
        if (!a) return;
        std::lock_guard<std::mutex> lk(g_tmu);
        cudaEvent_t b = pool_event();
        cudaEventRecord(b, s);
        g_pending.push_back({name, a, b});
    }
};

// Accumulates the elapsed times of completed event pairs.
void resolve_timing()
{
    std::lock_guard<std::mutex> lk(g_tmu);
    std::vector<TimingRec> keep;
    for (auto &r : g_pending) {
        if (cudaEventQuery(r.b) != cudaSuccess) { keep.push_back(r); continue; }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto &acc = g_tacc[r.name];
            acc.first += ms;
            acc.second += 1;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_pending.swap(keep);
}

// Device array with grow-only capacity: alloc() reuses the allocation when
// it is large enough, so buffers handed from one plan to the next are not
// reallocated.
// Test hooks (bem_test_hooks): the number of device allocations still
// allowed before one is reported as failed (-1: no limit), and the bytes the
// library holds in device allocations.
std::atomic<int64_t> g_alloc_budget{-1};
std::atomic<int64_t> g_live_bytes{0};

void dev_malloc(void **p, size_t bytes)
{
    for (;;) {
        int64_t b = g_alloc_budget.load();
        if (b < 0) break;
        if (b == 0) {
            g_err = "device allocation of " + std::to_string(bytes) + " bytes refused by the test hook";
            throw Fail{BEM_E_OOM};
        }
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    ck(cudaMalloc(p, bytes), "cudaMalloc");
    g_live_bytes += (int64_t)bytes;
}

template <typename T>
struct DevArr {
    T *p = nullptr;
    size_t n = 0, cap = 0;
    DevArr() = default;
    DevArr(const DevArr &) = delete;
    DevArr &operator=(const DevArr &) = delete;
    ~DevArr() { release(); }
    void release()
    {
        if (p) {
            cudaFree(p);
            g_live_bytes -= (int64_t)(cap * sizeof(T));
        }
        p = nullptr;
        n = cap = 0;
    }
    void alloc(size_t count)
    {
        if (count <= cap && p) { n = count; return; }
        release();
        if (count == 0) return;
        dev_malloc((void **)&p, count * sizeof(T));
        n = cap = count;
    }
    void swap(DevArr &o)
    {
        std::swap(p, o.p);
        std::swap(n, o.n);
        std::swap(cap, o.cap);
    }
    void upload(const std::vector<T> &v, cudaStream_t s)
    {
        alloc(v.size());
        if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s), "H2D");
    }
    size_t bytes() const { return n * sizeof(T); }
};

inline unsigned nblocks(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

// Near / interaction lists (host copy + device copy).  The purely geometric
// lists of a mesh are reused at every frequency whose Hankel-growth test
// admits all of their far offsets; otherwise a frequency gets its own.
struct ListsLevelDev {
    DevArr<int> il_ptr, il_src, il_off, is_src;
    DevArr<double> offs;
    DevArr<AggTask> tasks;        // aggregation work items (element chunks)
    DevArr<int> red_ptr, red_c;   // split clusters: partial rows to sum
    int ntasks = 0, nred = 0, nextra = 0;
};

struct Lists {
    FreqPlan fp;
    int max_ncol = 0;
    DevArr<int64_t> leaf_start;
    DevArr<int2> dis_tasks;       // disaggregation work items (element ranges)
    int n_dis_tasks = 0;
    DevArr<int> leaf_of, run_ptr, ncol;
    DevArr<int2> runs;
    DevArr<int64_t> row_ptr;
    DevArr<int4> spmv_items;      // (leaf, first row, end row) work items of the product
    int n_spmv_items = 0;
    int64_t nnz = 0;
    std::vector<std::unique_ptr<ListsLevelDev>> lev;
    // all levels together, for the one-launch far-field kernels
    std::vector<AggTask> h_tasks;    // aggregation element chunks of every level (host)
    DevArr<int2> all_reds, all_targets;
    std::vector<int2> h_targets;   // host copy of all_targets
    DevArr<unsigned int> red_cnt;
    int n_tasks = 0, n_reds = 0, n_targets = 0;
    // expensive near pairs (row, position), listed on first use
    DevArr<int2> heavy;
    int64_t n_heavy = -1;
    // transposed near product from the stored values: per leaf t, the rows i
    // of the leaves s in its near list, each with the position of A_i,t0 (t's
    // first element) in the stored values; usable when every near pair has
    // its mirror (tsym)
    DevArr<int> trow_ptr, trow_i;
    DevArr<int64_t> trow_off;
    bool tsym = false, trow_checked = false, trow_ready = false;
    std::vector<int64_t> h_row_ptr;
    std::vector<int> h_trow_ptr;  // host copy of trow_ptr
    // block-Jacobi sub-blocks (first element, size, offset of the inverse)
    std::vector<int4> h_bj;
    DevArr<int4> bj;
    int64_t bj_entries = 0;
};

// Per-depth element data (frequency independent).
struct DepthDev {
    int nc = 0;
    DevArr<float4> dz;        // z_c - x_j per element
    DevArr<int> elem_cl;
    DevArr<int64_t> cstart;
};

struct LevelDev {
    int depth = 0, L = 0, nd = 0, nc = 0, noff = 0;
    const ListsLevelDev *ll = nullptr;
    const DepthDev *dd = nullptr;
    DevArr<float4> dirs;
    DevArr<double> dirs_d;
    DevArr<float2> D, M, Lam;
    DevArr<float2> ph;            // stored phases [n][phs] (far_table), else empty
    int phs = 0;
    FarArgs args() const
    {
        FarArgs f;
        memset(&f, 0, sizeof f);
        f.nd = nd;
        f.k = 0.f;
        f.dirs = dirs.p;
        f.il_ptr = ll->il_ptr.p;
        f.il_src = ll->il_src.p;
        f.il_off = ll->il_off.p;
        f.D = D.p;
        f.M = M.p;
        f.Lam = Lam.p;
        f.cstart = dd->cstart.p;
        f.is_src = ll->is_src.p;
        f.tasks = ll->tasks.p;
        f.ntasks = ll->ntasks;
        f.red_ptr = ll->red_ptr.p;
        f.red_c = ll->red_c.p;
        f.nred = ll->nred;
        f.dz = dd->dz.p;
        f.elem_cl = dd->elem_cl.p;
        f.ph = ph.p;
        f.phs = phs;
        return f;
    }
};

struct Plan {
    int planes = 1;               // right-hand sides the M and Lambda buffers hold
    DevArr<int4> tgroups;         // transfer blocks (level, target, first direction)
    DevArr<AggTask> agg_tasks;    // aggregation blocks (element chunk, first direction pair)
    DevArr<AggTask> agg_tasks_tc; // the same with kTcPairs pairs per block (tensor-core aggregation)
    int n_tc_tasks = 0;
    double freq = -1.0, c = -1.0, k = 0.0;
    std::shared_ptr<Lists> lists;
    bool shared_lists = false;
    std::vector<std::unique_ptr<LevelDev>> lev;
    DevArr<LevelsArgs> largs;     // device copy of the per-level arguments
    LevelsArgs hargs;
    DevArr<float2> val;
    DevArr<float2> valT;          // A^T in A's layout (near_transpose), made from val
    bool valT_valid = false;
    bool has_phases = false;      // every level's stored phases built (far_table)
    std::vector<float> val_key;   // host copy of the coefficients the stored values were made with
    bool val_valid = false;
    int64_t nnz() const { return lists->nnz; }
    const FreqPlan &fp() const { return lists->fp; }
};

struct Coeffs {
    std::vector<float2> cp, cq, cp0, cq0, z, aq;   // internal order
    bool known_nonzero = false;
};

}  // namespace

// The state of one frequency: plan, column coefficients, error flag.
struct Frame {
    std::unique_ptr<Plan> plan;
    DevArr<float2> cp, cq, cp0, cq0, z, aq;    // column coefficients, known data (internal order)
    DevArr<int> err;                           // first element whose subdivision failed
    DevArr<float2> vtmp, vout;                 // scratch of the fused validation pass
    cudaStream_t s = nullptr;                  // stream of this frame's setup work
    bool known_nonzero = false;
};

// Device data of the FMM field evaluation at points (one call's plan).
struct EvalLevelDev {
    int L = 0, nd = 0, noff = 0, npc = 0, nc = 0, nextra = 0;
    DevArr<int> il_ptr, il_src, il_off, pcl, red_ptr, red_c;
    DevArr<double> offs, dirs_d;
    DevArr<float4> dirs, dzp;
    DevArr<float2> D, Mx, Lam;
};
struct EvalDev {
    // the plan below serves calls with the same points, wavenumber, tree depth
    // and expansion parameters (key), so repeated evaluations skip the host
    // build, the uploads and the translation tables
    bool valid = false;
    std::vector<double> key_pts;
    double key_k = 0.0, key_trunc = 0.0;
    int key_depth = -1;
    int64_t np = 0;
    int npl = 0, n_dtasks = 0;
    bool far = false;
    LevelsArgs A;
    DisaggArgs da;
    std::vector<std::unique_ptr<EvalLevelDev>> lev;
    DevArr<AggTask> tasks;
    DevArr<int2> reds, dtasks, nruns;
    DevArr<unsigned int> red_cnt;
    DevArr<int4> tgroups;
    DevArr<LevelsArgs> largs;
    DevArr<int> pleaf, nptr;
    DevArr<double> pts;
    DevArr<int64_t> perm;
    DevArr<float4> wts, zeros;
    DevArr<float2> vnear, vall;
};

struct bem_mesh_impl {
    int device = 0;
    bem_params prm;
    Geometry g;
    Tree t;
    int64_t n = 0;
    std::vector<int32_t> bct, region, type_int;
    std::vector<double> bcv;
    DevArr<float4> chi, clo, nrm, va, e1, e2;
    DevArr<double> cd, vad, e1d, e2d, ad;
    DevArr<int64_t> perm;
    DevArr<QuadTables> Q;
    DevArr<int> type;
    DevArr<float2> xint, ynear, tmp, tmp2, bvec, uvec;
    DevArr<float2> dinv;         // row scaling 1 / A_ii (internal order) when row_scaling is on
    DevArr<float2> bjinv;        // block-Jacobi inverses of the diagonal sub-blocks when block_jacobi is on
    // admittance gradient: forward u, field at the points, G_f^T conj(f),
    // coefficients of the q-operator, region per element, accumulators
    DevArr<float2> uadj, fadj, gadj, adj_cp, adj_cq;
    DevArr<float4> rowf;         // transposed product: row factor (a, b) per element
    DevArr<int> adjreg;
    DevArr<double> adjacc;
    DevArr<float4> wts;          // far-field weights (alpha, c) per element
    DevArr<int> tc_fault;        // set when a tensor-core aggregation's wait ran out
    bool force_fp32 = false;     // products with the FP32 aggregation (the refinement's residuals)
    DevArr<float2> bsave, xcur, rtmp;   // refinement: right-hand side, current solution, A x
    DevArr<double2> x64;         // refinement: solution in FP64
    // GMRES workspace
    DevArr<float2> V, w;
    DevArr<double2> H, cs, sn, g_, yv;
    DevArr<double> normpart;
    DevArr<double> gsacc;        // Gram-Schmidt norm sums [2][4] (per parity of the column)
    DevArr<double2> gsh2;        // Gram-Schmidt second-pass dots [2][m + 1]
    DevArr<GmresState> st;
    // frequency state: cur serves the products and the solve; next is filled
    // by the setup thread of a frequency sweep for the following frequency
    // (its work on s_setup) while cur's GMRES runs
    Frame cur, next;
    cudaStream_t s_setup = nullptr;
    std::shared_ptr<Lists> geo_lists;                  // frequency-independent lists
    std::vector<std::shared_ptr<Lists>> freq_lists;    // recent frequency-specific builds (newest last)
    int leaf_depth = 0;                                // leaf depth of the lists (autotuned)
    bool tuned = false;
    std::vector<std::pair<int, double>> tune_log;      // (leaf depth, estimated seconds per solve)
    // buffers kept from the previous plan (reused by the next frequency's plan)
    DevArr<float2> spare_val;
    std::vector<std::unique_ptr<DevArr<float2>>> spare_bufs;
    DevArr<SourceDev> srcbuf;
    DevArr<float2> fieldpart;     // per-point partial sums of the field (point-major)
    std::unique_ptr<EvalDev> eval;  // FMM field evaluation
    DevArr<double> ptsbuf;
    std::map<int, std::unique_ptr<DepthDev>> depth_dev;
    std::map<int, double> growth_root;                 // x*(L) of the Hankel stability test
    cudaStream_t s = nullptr;
    // side stream for the far-field upward pass, which runs beside the
    // near-field product (fork after k_prep, join before k_disaggregate)
    cudaStream_t s_far = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // side stream and events of the GMRES Givens steps inside one graph
    cudaStream_t s_giv = nullptr;
    cudaEvent_t ev_orth[kStepsPerGraph] = {}, ev_giv[kStepsPerGraph] = {};
    // GMRES status after each Arnoldi cycle (or step, with event timing):
    // pinned host copies of every plane's state (room for two copies)
    GmresState *h_st = nullptr;
    int h_st_planes = 0;                       // planes h_st holds per copy (two copies)
    std::vector<float> coef_key;

    ElemDev elem() const
    {
        ElemDev E;
        E.n = n;
        E.chi = chi.p; E.clo = clo.p; E.nrm = nrm.p; E.va = va.p; E.e1 = e1.p; E.e2 = e2.p;
        E.cd = cd.p; E.vad = vad.p; E.e1d = e1d.p; E.e2d = e2d.p; E.ad = ad.p;
        return E;
    }
    ~bem_mesh_impl()
    {
        for (int t = 0; t < kStepsPerGraph; ++t) {
            if (ev_orth[t]) cudaEventDestroy(ev_orth[t]);
            if (ev_giv[t]) cudaEventDestroy(ev_giv[t]);
        }
        if (h_st) cudaFreeHost(h_st);
        if (s_giv) cudaStreamDestroy(s_giv);
        if (s_setup) cudaStreamDestroy(s_setup);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (s_far) cudaStreamDestroy(s_far);
        if (s) cudaStreamDestroy(s);
    }
};

// The frame the calling thread works on: a sweep's setup thread points this
// at the mesh's next frame; every other caller uses cur.
static thread_local Frame *t_frame = nullptr;
static inline Frame &fr(bem_mesh_impl &M) { return t_frame ? *t_frame : M.cur; }

namespace {

double wavenumber(double f, double c) { return 2.0 * M_PI * f / c; }

// ------------------------------------------------------------------ plan
std::shared_ptr<Lists> upload_lists(bem_mesh_impl &M, FreqPlan &&fp)
{
    {
        // the kernels index with these lists: check them on the host first
        const std::string bad = validate_plan(M.t, fp);
        if (!bad.empty()) throw Fail{set_err(BEM_E_INTERNAL, "plan check: " + bad)};
    }
    auto Ls = std::make_shared<Lists>();
    Ls->fp = std::move(fp);
    const FreqPlan &F = Ls->fp;
    const Level &Lf = M.t.lv[F.leaf_depth];
    const int nl = (int)Lf.start.size();
    cudaStream_t s = fr(M).s;
    // near columns of each leaf as runs of consecutive leaves
    std::vector<int> run_ptr(nl + 1, 0), ncol(nl, 0);
    std::vector<int2> runs;
    for (int t = 0; t < nl; ++t) {
        int pos = 0, prev = -2;
        for (int q = F.near_ptr[t]; q < F.near_ptr[t + 1]; ++q) {
            const int sl = F.near_src[q];
            if (sl != prev + 1) runs.push_back(make_int2((int)Lf.start[sl], pos));
            pos += (int)Lf.count[sl];
            prev = sl;
        }
        ncol[t] = pos;
        run_ptr[t + 1] = (int)runs.size();
    }
    std::vector<int> leaf_of(M.n);
    std::vector<int64_t> row_ptr(M.n + 1, 0), leaf_start(nl + 1, M.n);
    // rows padded to an even length: every row (and every leaf's block of
    // rows) starts on a 16-byte boundary for the TMA product
    for (int64_t i = 0; i < M.n; ++i) {
        leaf_of[i] = Lf.elem_cluster[i];
        row_ptr[i + 1] = row_ptr[i] + ((ncol[leaf_of[i]] + 1) & ~1);
    }
    for (int t = 0; t < nl; ++t) {
        leaf_start[t] = Lf.start[t];
        Ls->max_ncol = std::max(Ls->max_ncol, ncol[t]);
    }
    Ls->leaf_start.upload(leaf_start, s);
    {
        // disaggregation tasks: each leaf split into ranges of at most
        // kDisTask elements of nearly equal size, largest first
        std::vector<int2> dt;
        for (int t = 0; t < nl; ++t) {
            const int64_t a = leaf_start[t], cnt = leaf_start[t + 1] - a;
            const int64_t nch = (cnt + kDisTask - 1) / kDisTask;
            for (int64_t q = 0; q < nch; ++q)
                dt.push_back(make_int2((int)(a + cnt * q / nch), (int)(a + cnt * (q + 1) / nch)));
        }
        std::stable_sort(dt.begin(), dt.end(), [](int2 u, int2 v) { return u.y - u.x > v.y - v.x; });
        Ls->n_dis_tasks = (int)dt.size();
        Ls->dis_tasks.upload(dt, s);
    }
    {
        // block-Jacobi sub-blocks: each leaf split into ceil(count / kBjMax)
        // runs of consecutive elements of nearly equal size
        int64_t off = 0;
        for (int t = 0; t < nl; ++t) {
            const int64_t a = leaf_start[t], cnt = leaf_start[t + 1] - a;
            const int64_t nsub = (cnt + kBjMax - 1) / kBjMax;
            for (int64_t q = 0; q < nsub; ++q) {
                const int64_t b0 = a + cnt * q / nsub, b1 = a + cnt * (q + 1) / nsub;
                const int nb = (int)(b1 - b0);
                Ls->h_bj.push_back(make_int4((int)b0, nb, (int)off, 0));
                off += (int64_t)nb * nb;
            }
        }
        if (off > INT_MAX) throw Fail{set_err(BEM_E_ARG, "block-Jacobi blocks exceed the 32-bit offset range")};
        Ls->bj_entries = off;
        Ls->bj.upload(Ls->h_bj, s);
    }
    Ls->nnz = row_ptr[M.n];
    Ls->h_row_ptr = row_ptr;   // for the transposed product's rows, built when first needed
    Ls->leaf_of.upload(leaf_of, s);
    Ls->run_ptr.upload(run_ptr, s);
    Ls->ncol.upload(ncol, s);
    Ls->runs.upload(runs, s);
    Ls->row_ptr.upload(row_ptr, s);
    {
        // about kSpmvItemEntries values per item (at most kSpmvMaxItemRows
        // rows), a leaf's rows split evenly
        std::vector<int4> items;
        for (int t = 0; t < nl; ++t) {
            const int rows = (int)Lf.count[t];
            if (rows == 0) continue;
            const int rpi = (int)std::max<int64_t>(1, std::min<int64_t>(kSpmvMaxItemRows,
                                                                        kSpmvItemEntries / std::max(1, ncol[t])));
            const int nit = (rows + rpi - 1) / rpi;
            for (int q = 0; q < nit; ++q)
                items.push_back(make_int4(t, (int)((int64_t)rows * q / nit), (int)((int64_t)rows * (q + 1) / nit), 0));
        }
        Ls->n_spmv_items = (int)items.size();
        Ls->spmv_items.upload(items, s);
    }
    std::vector<AggTask> all_tasks;
    std::vector<int2> all_reds, all_targets;
    for (const FarLevel &FL : F.far) {
        const int lev_index = (int)Ls->lev.size();
        auto D = std::make_unique<ListsLevelDev>();
        D->il_ptr.upload(FL.il_ptr, s);
        D->il_src.upload(FL.il_src, s);
        D->il_off.upload(FL.il_off, s);
        D->offs.upload(FL.offsets, s);
        std::vector<int> is_src(FL.nc, 0);
        for (int v : FL.il_src) is_src[v] = 1;
        D->is_src.upload(is_src, s);
        // aggregation tasks: chunks of at most kAggChunk elements of each
        // source cluster, of nearly equal size (each plan expands them into
        // ranges of direction pairs for its expansion lengths)
        const Level &L = M.t.lv[FL.depth];
        std::vector<AggTask> tasks;
        std::vector<int> red_ptr{FL.nc}, red_c;
        int extra = 0;
        for (int c = 0; c < FL.nc; ++c) {
            if (!is_src[c]) continue;
            const int64_t cnt = L.count[c];
            const int64_t nch = std::max<int64_t>(1, (cnt + kAggChunk - 1) / kAggChunk);
            if (nch == 1) {
                tasks.push_back(AggTask{c, c, L.start[c], (int)cnt, lev_index, -1, -1, 0});
                continue;
            }
            const int red = (int)red_c.size();
            const int gred = (int)all_reds.size() + red;
            for (int64_t q = 0; q < nch; ++q) {
                const int64_t a = cnt * q / nch, b = cnt * (q + 1) / nch;
                tasks.push_back(AggTask{c, FL.nc + extra, L.start[c] + a, (int)(b - a), lev_index, red, gred, 0});
                ++extra;
            }
            red_c.push_back(c);
            red_ptr.push_back(FL.nc + extra);
        }
        D->ntasks = (int)tasks.size();
        D->nred = (int)red_c.size();
        D->nextra = extra;
        D->tasks.upload(tasks, s);
        D->red_ptr.upload(red_ptr, s);
        D->red_c.upload(red_c, s);
        all_tasks.insert(all_tasks.end(), tasks.begin(), tasks.end());
        for (int q = 0; q < D->nred; ++q) all_reds.push_back(make_int2(lev_index, q));
        for (int c = 0; c < FL.nc; ++c)
            if (FL.il_ptr[c + 1] > FL.il_ptr[c]) all_targets.push_back(make_int2(lev_index, c));
        Ls->lev.push_back(std::move(D));
    }
    Ls->n_tasks = (int)all_tasks.size();
    Ls->n_reds = (int)all_reds.size();
    Ls->n_targets = (int)all_targets.size();
    Ls->h_tasks = all_tasks;
    Ls->all_reds.upload(all_reds, s);
    Ls->all_targets.upload(all_targets, s);
    Ls->h_targets = all_targets;
    Ls->red_cnt.alloc(std::max(1, Ls->n_reds));
    ck(cudaMemsetAsync(Ls->red_cnt.p, 0, std::max(1, Ls->n_reds) * sizeof(unsigned int), s), "memset");
    ck(cudaStreamSynchronize(s), "sync");
    return Ls;
}

const DepthDev *depth_data(bem_mesh_impl &M, int depth)
{
    auto it = M.depth_dev.find(depth);
    if (it != M.depth_dev.end()) return it->second.get();
    auto D = std::make_unique<DepthDev>();
    const Level &L = M.t.lv[depth];
    D->nc = (int)L.start.size();
    std::vector<int64_t> cst(D->nc + 1);
    for (int cc = 0; cc < D->nc; ++cc) cst[cc] = L.start[cc];
    cst[D->nc] = M.n;
    std::vector<float4> dz(M.n);
    std::vector<int> ecl(M.n);
    for (int64_t i = 0; i < M.n; ++i) {
        const int cc = L.elem_cluster[i];
        ecl[i] = cc;
        const int64_t e = M.t.perm[i];
        dz[i] = make_float4((float)(L.z[3 * cc] - M.g.cen[3 * e]), (float)(L.z[3 * cc + 1] - M.g.cen[3 * e + 1]),
                            (float)(L.z[3 * cc + 2] - M.g.cen[3 * e + 2]), 0.f);
    }
    D->cstart.upload(cst, fr(M).s);
    D->dz.upload(dz, fr(M).s);
    D->elem_cl.upload(ecl, fr(M).s);
    ck(cudaStreamSynchronize(fr(M).s), "sync");
    const DepthDev *r = D.get();
    M.depth_dev[depth] = std::move(D);
    return r;
}

// expansion length of a depth (Eq. FMMTruncation, largest radius of the depth)
int level_L(const bem_mesh_impl &M, int depth, double k)
{
    const double x = 2.0 * M.t.lv[depth].rmax * k;
    const double L = x + M.prm.trunc_factor * std::log10(x + M_PI);
    return std::max(M.prm.L_min, (int)std::ceil(L - 1e-12));
}

// Moves the large buffers of the current plan into the mesh's spares.
void recycle_plan(bem_mesh_impl &M)
{
    if (!fr(M).plan) return;
    ck(cudaStreamSynchronize(fr(M).s), "sync");
    M.spare_val.swap(fr(M).plan->val);
    for (auto &L : fr(M).plan->lev) {
        for (DevArr<float2> *b : {&L->D, &L->M, &L->Lam, &L->ph}) {
            if (!b->p) continue;
            auto d = std::make_unique<DevArr<float2>>();
            d->swap(*b);
            M.spare_bufs.push_back(std::move(d));
        }
    }
    fr(M).plan.reset();
}

// Takes the spare buffer with the smallest sufficient capacity (or any).
void take_spare(bem_mesh_impl &M, DevArr<float2> &dst, size_t count)
{
    int best = -1;
    for (int i = 0; i < (int)M.spare_bufs.size(); ++i) {
        const size_t c = M.spare_bufs[i]->cap;
        if (c >= count && (best < 0 || c < M.spare_bufs[best]->cap)) best = i;
    }
    if (best >= 0) {
        dst.swap(*M.spare_bufs[best]);
        M.spare_bufs.erase(M.spare_bufs.begin() + best);
    }
    dst.alloc(count);
}

// Per-frequency part of a plan on given lists: expansion lengths, sphere
// grids, translation tables (GPU), buffers and the kernel argument block.
void finish_plan(bem_mesh_impl &M, Plan &Pl)
{
    NvtxRange nvtx_("plan: expansions and translation tables");
    Plan *P = &Pl;
    const double k = P->k;
    cudaStream_t s = fr(M).s;
    const FreqPlan &fp = P->fp();
    for (size_t l = 0; l < fp.far.size(); ++l) {
        const FarLevel &F = fp.far[l];
        auto D = std::make_unique<LevelDev>();
        D->depth = F.depth;
        D->L = level_L(M, F.depth, k);
        D->nd = 2 * D->L * D->L;
        D->nc = F.nc;
        D->noff = (int)(F.offsets.size() / 3);
        D->ll = P->lists->lev[l].get();
        D->dd = depth_data(M, F.depth);
        std::vector<double> sd, sw;
        sphere_grid(D->L, sd, sw);
        std::vector<float4> dirs(D->nd);
        for (int q = 0; q < D->nd; ++q)
            dirs[q] = make_float4((float)sd[3 * q], (float)sd[3 * q + 1], (float)sd[3 * q + 2], (float)sw[q]);
        D->dirs.upload(dirs, s);
        D->dirs_d.upload(sd, s);
        take_spare(M, D->D, (size_t)D->noff * D->nd);
        take_spare(M, D->M, (size_t)(D->nc + D->ll->nextra) * D->nd);
        take_spare(M, D->Lam, (size_t)D->nc * D->nd);
        if ((int64_t)D->noff * D->nd > 0 && D->L > kMaxTableL)
            throw Fail{set_err(BEM_E_ARG, "far field: expansion length " + std::to_string(D->L) +
                                              " exceeds the translation-table limit " + std::to_string(kMaxTableL))};
        P->lev.push_back(std::move(D));
    }
    {
        // translation tables of every level in one launch
        DTableArgs ta;
        memset(&ta, 0, sizeof ta);
        ta.k = k;
        int nb = 0;
        for (const auto &D : P->lev) {
            if ((int64_t)D->noff * D->nd == 0) continue;
            ta.start[ta.nlev] = nb;
            ta.lev[ta.nlev] = DTableLevel{D->ll->offs.p, D->dirs_d.p, D->D.p, D->nd, D->L};
            nb += D->noff;
            ++ta.nlev;
        }
        ta.start[ta.nlev] = nb;
        if (nb > 0) {
            {
                KTimer kt_("k_dtable", s);
                k_dtable<<<nb, 128, 0, s>>>(ta);
            }
            ck_launch("k_dtable");
        }
    }
    {
        // the phases of the aggregation and (conjugated) of the
        // disaggregation, once per frequency for every level, element and
        // antipodal pair (far_table; single-right-hand-side products read
        // them), unless they would take more than kPhaseTableMaxBytes
        P->has_phases = false;
        const int64_t n = M.n;
        double bytes = 0.0;
        for (const auto &D : P->lev) bytes += (double)n * (double)((D->nd / 2 + 1) & ~1) * sizeof(float2);
        if (M.prm.far_table == 1 && !P->lev.empty() && bytes <= kPhaseTableMaxBytes) {
            PhaseTableArgs pa;
            memset(&pa, 0, sizeof pa);
            pa.n = n;
            pa.k = (float)k;
            const int per = (int)((n + kPhaseElems - 1) / kPhaseElems);
            int nb = 0;
            for (const auto &D : P->lev) {
                D->phs = (D->nd / 2 + 1) & ~1;
                take_spare(M, D->ph, (size_t)n * D->phs);
                pa.start[pa.nlev] = nb;
                pa.lev[pa.nlev] = PhaseLevel{D->dd->dz.p, D->dirs.p, D->ph.p, D->nd / 2, D->phs};
                nb += per;
                ++pa.nlev;
            }
            pa.start[pa.nlev] = nb;
            {
                KTimer kt_("k_phase_table", s);
                k_phase_table<<<nb, 128, 0, s>>>(pa);
            }
            ck_launch("k_phase_table");
            P->has_phases = true;
        }
    }
    LevelsArgs &A = P->hargs;
    memset(&A, 0, sizeof A);
    A.nlev = (int)P->lev.size();
    {
        // aggregation blocks for this plan's expansion lengths: every
        // element chunk times the ranges of kAggThreads direction pairs
        std::vector<AggTask> at;
        for (const AggTask &t : P->lists->h_tasks)
            for (int p0 = 0; p0 < P->lev[t.lev]->nd / 2; p0 += kAggThreads) {
                AggTask u = t;
                u.p0 = p0;
                at.push_back(u);
            }
        P->agg_tasks.upload(at, s);
        A.tasks = P->agg_tasks.p;
        A.ntasks = (int)at.size();
        if (M.prm.far_precision == 1) {
            std::vector<AggTask> tt;
            for (const AggTask &t : P->lists->h_tasks)
                for (int p0 = 0; p0 < P->lev[t.lev]->nd / 2; p0 += kTcPairs) {
                    AggTask u = t;
                    u.p0 = p0;
                    tt.push_back(u);
                }
            P->agg_tasks_tc.upload(tt, s);
            P->n_tc_tasks = (int)tt.size();
        }
    }
    A.reds = P->lists->all_reds.p;
    A.nreds = P->lists->n_reds;
    A.targets = P->lists->all_targets.p;
    A.ntargets = P->lists->n_targets;
    {
        // transfer blocks for this plan's expansion lengths: (level, target,
        // first direction)
        std::vector<int4> tg;
        for (const int2 &lt : P->lists->h_targets)
            for (int nu0 = 0; nu0 < P->lev[lt.x]->nd; nu0 += kTransferDirs) tg.push_back(make_int4(lt.x, lt.y, nu0, 0));
        P->tgroups.upload(tg, s);
        A.tgroups = P->tgroups.p;
        A.ntgroups = (int)tg.size();
    }
    A.red_cnt = P->lists->red_cnt.p;
    for (size_t l = 0; l < P->lev.size(); ++l) {
        A.lev[l] = P->lev[l]->args();
        A.lev[l].k = (float)k;
        A.lev[l].mplane = (int64_t)(P->lev[l]->nc + P->lev[l]->ll->nextra) * P->lev[l]->nd;
        A.lev[l].lplane = (int64_t)P->lev[l]->nc * P->lev[l]->nd;
    }
    std::vector<LevelsArgs> hv(1, A);
    P->largs.upload(hv, s);
    ck(cudaStreamSynchronize(s), "sync");
}

void autotune_leaf_depth(bem_mesh_impl &M, double k);

void build_plan_dev(bem_mesh_impl &M, double freq, double c)
{
    if (fr(M).plan && fr(M).plan->freq == freq && fr(M).plan->c == c) return;
    recycle_plan(M);
    auto P = std::make_unique<Plan>();
    P->freq = freq;
    P->c = c;
    P->k = wavenumber(freq, c);
    const double k = P->k;
    if (!M.geo_lists) {
        if (!M.tuned) autotune_leaf_depth(M, k);
        if (!M.geo_lists) {
            bem_params gp = M.prm;
            gp.stability_max = 1e308;
            FreqPlan fp;
            build_plan(M.g, M.t, gp, k, fp, M.leaf_depth);
            M.geo_lists = upload_lists(M, std::move(fp));
        }
    }
    // The Hankel growth sum_{n<=L}(2n+1)|h_n(x)|/|h_0(x)| decreases with x,
    // so "stable" is x >= x*(L), the root of growth = stability_max, found
    // once per L by bisection; the per-frequency reuse tests below then need
    // no Hankel evaluations.
    auto stable_from = [&](int L) {
        auto it = M.growth_root.find(L);
        if (it != M.growth_root.end()) return it->second;
        // as x grows every |h_n(x)| tends to 1/x, so the growth tends to
        // sum_{n<=L} (2n+1) = (L+1)^2 from above: beyond the bound no offset
        // is ever stable
        if ((double)(L + 1) * (L + 1) > M.prm.stability_max) {
            M.growth_root[L] = HUGE_VAL;
            return HUGE_VAL;
        }
        double lo = 1e-9, hi = 1.0;
        for (int it2 = 0; it2 < 64 && !(hankel_growth(hi, L) <= M.prm.stability_max); ++it2) hi *= 2.0;
        for (int it2 = 0; it2 < 200 && hi - lo > 1e-13 * hi; ++it2) {
            const double mid = 0.5 * (lo + hi);
            if (hankel_growth(mid, L) <= M.prm.stability_max) hi = mid;
            else lo = mid;
        }
        M.growth_root[L] = hi;
        return hi;
    };
    // reuse the geometric lists when every far offset passes the Hankel test
    // (the shortest offset of each level decides)
    bool ok = true;
    for (const FarLevel &FL : M.geo_lists->fp.far) {
        double xmin = 1e300;
        for (size_t o = 0; o < FL.offsets.size() / 3; ++o)
            xmin = std::min(xmin, FL.offsets[3 * o] * FL.offsets[3 * o] + FL.offsets[3 * o + 1] * FL.offsets[3 * o + 1] +
                                      FL.offsets[3 * o + 2] * FL.offsets[3 * o + 2]);
        if (FL.offsets.empty()) continue;
        if (!(k * std::sqrt(xmin) >= stable_from(level_L(M, FL.depth, k)))) { ok = false; break; }
    }
    // else reuse a recent frequency-specific build when every stability
    // verdict it evaluated (and the expansion length per depth) is unchanged:
    // the recursion then makes the same decisions
    std::shared_ptr<Lists> reuse;
    if (!ok) {
        for (auto it = M.freq_lists.rbegin(); it != M.freq_lists.rend() && !reuse; ++it) {
            const FreqPlan &lf = (*it)->fp;
            bool same = true;
            for (size_t d = 0; same && d < lf.Ld.size(); ++d)
                if (level_L(M, (int)d, k) != lf.Ld[d]) same = false;
            for (size_t q = 0; same && q < lf.verdicts.size(); ++q) {
                const Verdict &v = lf.verdicts[q];
                const double b = M.t.lv[v.depth].box;
                const double X = b * std::sqrt((double)v.dx * v.dx + (double)v.dy * v.dy + (double)v.dz * v.dz);
                if ((k * X >= stable_from(v.L)) != v.stable) same = false;
            }
            if (same) reuse = *it;
        }
    }
    if (ok) {
        P->lists = M.geo_lists;
        P->shared_lists = true;
    } else if (reuse) {
        P->lists = reuse;
        P->shared_lists = true;
    } else {
        FreqPlan fp;
        build_plan(M.g, M.t, M.prm, k, fp, M.leaf_depth);
        P->lists = upload_lists(M, std::move(fp));
        M.freq_lists.push_back(P->lists);
        if (M.freq_lists.size() > 4) M.freq_lists.erase(M.freq_lists.begin());
    }
    finish_plan(M, *P);
    fr(M).plan = std::move(P);
}

NearArgs near_args(const bem_mesh_impl &M, const Plan &P, const float2 *cp, const float2 *cq)
{
    NearArgs a;
    a.E = M.elem();
    a.N.leaf_of = P.lists->leaf_of.p;
    a.N.run_ptr = P.lists->run_ptr.p;
    a.N.runs = P.lists->runs.p;
    a.N.ncol = P.lists->ncol.p;
    a.N.row_ptr = P.lists->row_ptr.p;
    a.N.leaf_start = P.lists->leaf_start.p;
    a.Q = M.Q.p;
    a.k = (float)P.k;
    a.ik_inv = (float)(1.0 / P.k);
    a.tau = M.prm.tau < 0 ? -1.f : 1.f;
    a.cp = cp;
    a.cq = cq;
    return a;
}

// coefficient sets (Eq. SystemI with the boundary conditions folded in)
void make_coeffs(bem_mesh_impl &M, double k, double omega, double c, double rho, const double *adm, int nreg, Coeffs &C)
{
    const int64_t n = M.n;
    C.cp.assign(n, make_float2(0.f, 0.f));
    C.cq = C.cp0 = C.cq0 = C.z = C.aq = C.cp;
    C.known_nonzero = false;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t e = M.t.perm[i];
        const int ty = M.bct[e];
        const double vr = M.bcv[2 * e], vi = M.bcv[2 * e + 1];
        if (ty == BEM_PRES) {
            C.cq[i] = make_float2(1.f, 0.f);
            C.cp0[i] = make_float2(1.f, 0.f);
            C.z[i] = make_float2((float)vr, (float)vi);
        } else {
            C.cp[i] = make_float2(1.f, 0.f);
            C.cq0[i] = make_float2(1.f, 0.f);
            // g = i w rho v
            C.z[i] = make_float2((float)(-omega * rho * vi), (float)(omega * rho * vr));
            if (ty == BEM_ADMI) {
                const int r = M.region[e];
                const double yr = adm[2 * r], yi = adm[2 * r + 1];
                // a = -tau i k beta, beta = rho c Y, Y = velocity into the
                // wall / p (the wall lies along the normal for the interior
                // problem, against it for the exterior problem)
                const double t = M.prm.tau < 0 ? -1.0 : 1.0;
                const double br = t * rho * c * yr, bi = t * rho * c * yi;
                C.cq[i] = make_float2((float)(k * bi), (float)(-k * br));
                C.aq[i] = C.cq[i];
            }
        }
        if (C.z[i].x != 0.f || C.z[i].y != 0.f) C.known_nonzero = true;
    }
    // tau (Eq. SystemI: +1 exterior, -1 interior) multiplies every integral
    // operator: it is folded into the column coefficients of the unknowns
    // and of the known data (the self entry takes it out of its identity
    // half again); aq, the physical relation q = a p, keeps its sign
    if (M.prm.tau < 0)
        for (int64_t i = 0; i < n; ++i) {
            C.cp[i] = make_float2(-C.cp[i].x, -C.cp[i].y);
            C.cq[i] = make_float2(-C.cq[i].x, -C.cq[i].y);
            C.cp0[i] = make_float2(-C.cp0[i].x, -C.cp0[i].y);
            C.cq0[i] = make_float2(-C.cq0[i].x, -C.cq0[i].y);
        }
}

void upload_coeffs(bem_mesh_impl &M, const Coeffs &C)
{
    fr(M).cp.upload(C.cp, fr(M).s);
    fr(M).cq.upload(C.cq, fr(M).s);
    fr(M).cp0.upload(C.cp0, fr(M).s);
    fr(M).cq0.upload(C.cq0, fr(M).s);
    fr(M).z.upload(C.z, fr(M).s);
    fr(M).aq.upload(C.aq, fr(M).s);
    fr(M).known_nonzero = C.known_nonzero;
}

void check_err(bem_mesh_impl &M)
{
    int e = INT_MAX;
    ck(cudaMemcpyAsync(&e, fr(M).err.p, sizeof(int), cudaMemcpyDeviceToHost, fr(M).s), "D2H err");
    ck(cudaStreamSynchronize(fr(M).s), "sync");
    if (e != INT_MAX) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "number of subelements which are subdivided in a loop exceeds %d at element %lld",
                 M.prm.max_depth, (long long)M.t.perm[e]);
        g_err = buf;
        throw Fail{BEM_E_SUBDIV_LIMIT};
    }
}

// Reports (BEM_E_TIMEOUT) a tensor-core aggregation whose wait for the
// tensor cores ran out since the last check; waits for the mesh's stream.
void check_tc_fault(bem_mesh_impl &M)
{
    if (M.prm.far_precision != 1) return;
    int f = 0;
    ck(cudaMemcpyAsync(&f, M.tc_fault.p, sizeof(int), cudaMemcpyDeviceToHost, M.s), "D2H fault");
    ck(cudaStreamSynchronize(M.s), "sync");
    if (f) {
        ck(cudaMemsetAsync(M.tc_fault.p, 0, sizeof(int), M.s), "memset");
        g_err = "tensor-core aggregation: the wait for the tensor cores gave up";
        throw Fail{BEM_E_TIMEOUT};
    }
}

void reset_err(bem_mesh_impl &M)
{
    const int v = INT_MAX;
    ck(cudaMemcpyAsync(fr(M).err.p, &v, sizeof(int), cudaMemcpyHostToDevice, fr(M).s), "H2D err");
}

// Stored near-field entries of plan P for the column coefficients (cp, cq):
// the expensive pairs are listed once per set of lists, then computed by
// their own kernel.
void store_near(bem_mesh_impl &M, Plan &P, const float2 *cp, const float2 *cq)
{
    NvtxRange nvtx_("near-field entries");
    if (!P.val.p) P.val.swap(M.spare_val);
    P.val.alloc((size_t)P.nnz());
    reset_err(M);
    NearArgs a = near_args(M, P, cp, cq);
    Lists &Ls = *P.lists;
    if (Ls.n_heavy < 0) {
        // count, then list, the expensive pairs of these lists (geometry
        // only), grouped by kind
        DevArr<unsigned long long> cnt, off;
        cnt.alloc(kHeavyKinds);
        off.alloc(kHeavyKinds);
        ck(cudaMemsetAsync(cnt.p, 0, kHeavyKinds * sizeof(unsigned long long), fr(M).s), "memset");
        {
            KTimer kt_("k_near_classify", fr(M).s);
            k_near_classify<<<nblocks(M.n, 8), 256, 0, fr(M).s>>>(a, nullptr, cnt.p, nullptr);
        }
        ck_launch("k_near_classify");
        unsigned long long hk[kHeavyKinds], ho[kHeavyKinds];
        ck(cudaMemcpyAsync(hk, cnt.p, sizeof hk, cudaMemcpyDeviceToHost, fr(M).s), "D2H");
        ck(cudaStreamSynchronize(fr(M).s), "sync");
        unsigned long long h = 0;
        for (int q = 0; q < kHeavyKinds; ++q) {
            ho[q] = h;
            h += hk[q];
        }
        Ls.heavy.alloc(std::max<unsigned long long>(h, 1));
        ck(cudaMemcpyAsync(off.p, ho, sizeof ho, cudaMemcpyHostToDevice, fr(M).s), "H2D");
        ck(cudaMemsetAsync(cnt.p, 0, kHeavyKinds * sizeof(unsigned long long), fr(M).s), "memset");
        {
            KTimer kt_("k_near_classify", fr(M).s);
            k_near_classify<<<nblocks(M.n, 8), 256, 0, fr(M).s>>>(a, Ls.heavy.p, cnt.p, off.p);
        }
        ck_launch("k_near_classify");
        ck(cudaStreamSynchronize(fr(M).s), "sync");
        Ls.n_heavy = (int64_t)h;
    }
    {
        KTimer kt_("k_near_store", fr(M).s);
        const int nleaf = (int)(P.lists->leaf_start.n - 1);
        const dim3 grid(nleaf, nblocks(std::max(1, P.lists->max_ncol), 256));
        k_near_store_light<<<grid, 256, 0, fr(M).s>>>(a, P.val.p, fr(M).err.p);
    }
    ck_launch("k_near_store");
    if (Ls.n_heavy > 0) {
        {
            KTimer kt_("k_near_store_heavy", fr(M).s);
            k_near_store_heavy<<<nblocks(Ls.n_heavy, 128), 128, 0, fr(M).s>>>(a, Ls.heavy.p, Ls.n_heavy, P.val.p,
                                                                          fr(M).err.p);
        }
        ck_launch("k_near_store_heavy");
    }
    check_err(M);
}

// Make sure the stored near-field values match the current unknowns' coefficients.
void ensure_near_values(bem_mesh_impl &M, const Coeffs &C)
{
    Plan &P = *fr(M).plan;
    std::vector<float> key;
    key.reserve(4 * M.n);
    for (int64_t i = 0; i < M.n; ++i) {
        key.push_back(C.cp[i].x); key.push_back(C.cp[i].y);
        key.push_back(C.cq[i].x); key.push_back(C.cq[i].y);
    }
    if (!M.prm.near_store || P.fp().direct) {
        if (!P.val_valid) {
            // one fused pass validates the subdivision limit for this plan
            reset_err(M);
            Frame &F = fr(M);
            F.vtmp.alloc(M.n);
            F.vout.alloc(M.n);
            ck(cudaMemsetAsync(F.vtmp.p, 0, M.n * sizeof(float2), F.s), "memset");
            NearArgs a = near_args(M, P, F.cp.p, F.cq.p);
            {
                KTimer kt_("k_near_fused", F.s);
                k_near_fused<<<nblocks(M.n, 8), 256, 0, F.s>>>(a, F.vtmp.p, F.vout.p, F.err.p, nullptr);
            }
            ck_launch("k_near_fused");
            check_err(M);
            P.val_valid = true;
        }
        return;
    }
    if (P.val_valid && key == P.val_key) return;
    P.valT_valid = false;
    store_near(M, P, fr(M).cp.p, fr(M).cq.p);
    P.val_key.swap(key);
    P.val_valid = true;
}

// y = A x with the given column coefficients.  x: caller order when
// perm_in, else internal (optionally x + (*jidx) n).  y: caller order when
// perm_out.  use_store: use the stored near-field values.
PrepArgs prep_args(bem_mesh_impl &M, const float2 *cp, const float2 *cq, const float2 *x)
{
    const bool far = !fr(M).plan->lev.empty();
    PrepArgs pa;
    pa.n = M.n;
    pa.x = x;
    pa.jidx = nullptr;
    pa.perm = nullptr;
    pa.xint = M.xint.p;
    pa.wts = far ? M.wts.p : nullptr;
    pa.chi = M.chi.p;
    pa.nrm = M.nrm.p;
    pa.cp = cp;
    pa.cq = cq;
    pa.k = (float)fr(M).plan->k;
    pa.plane = 0;
    pa.xplane = 0;
    return pa;
}

// Room for nr right-hand sides in the current plan's M and Lambda buffers
// and in the product's work vectors (xint, ynear, wts: nr planes of n).
void ensure_planes(bem_mesh_impl &M, int nr)
{
    Plan &P = *fr(M).plan;
    if (M.xint.cap < (size_t)M.n * nr) {
        M.xint.alloc((size_t)M.n * nr);
        M.ynear.alloc((size_t)M.n * nr);
        M.wts.alloc((size_t)M.n * nr);
    }
    if (P.planes >= nr) return;
    LevelsArgs &A = P.hargs;
    for (size_t l = 0; l < P.lev.size(); ++l) {
        LevelDev &D = *P.lev[l];
        D.M.alloc((size_t)(D.nc + D.ll->nextra) * D.nd * nr);
        D.Lam.alloc((size_t)D.nc * D.nd * nr);
        A.lev[l].M = D.M.p;
        A.lev[l].Lam = D.Lam.p;
    }
    std::vector<LevelsArgs> hv(1, A);
    P.largs.upload(hv, fr(M).s);
    ck(cudaStreamSynchronize(fr(M).s), "sync");
    P.planes = nr;
}

// y = A x with the given column coefficients.  x: caller order when
// perm_in, else internal (optionally x + (*jidx) n).  y: caller order when
// perm_out.  use_store: use the stored near-field values.  prepared: the
// product inputs (x_int and the far-field weights) are already formed and x
// is unused.  far_only: y receives the far-field part alone and the
// near-field part stays in M.ynear (the caller adds them); the whole far
// chain (aggregation, transfer, disaggregation) then runs on the side
// stream beside the near-field product.
void matvec_internal(bem_mesh_impl &M, const float2 *cp, const float2 *cq, bool use_store, const float2 *x,
                     const int *jidx, bool perm_in, float2 *y, bool perm_out, const int *skip, cudaStream_t s,
                     bool prepared = false, bool far_only = false, int nr = 1)
{
    Plan &P = *fr(M).plan;
    const int64_t n = M.n;
    if (nr > 1) ensure_planes(M, nr);
    if (!prepared) {
        PrepArgs pa = prep_args(M, cp, cq, x);
        pa.jidx = jidx;
        pa.perm = perm_in ? M.perm.p : nullptr;
        pa.plane = n;
        pa.xplane = n;
        {
            KTimer kt_("k_prep", s);
            k_prep<<<dim3(nblocks(n, 256), nr), 256, 0, s>>>(pa, skip);
        }
        ck_launch("k_prep");
    }
    // The far-field upward pass (aggregation, transfer) depends only on
    // k_prep and runs on the high-priority side stream beside the near-field
    // product; k_disaggregate joins both.  With kernel timing on, everything
    // stays on one stream so each kernel is timed alone.
    const LevelsArgs &A = P.hargs;
    const bool fork = !g_timing && (A.ntasks > 0 || A.ntargets > 0);
    cudaStream_t sf = fork ? M.s_far : s;
    if (fork) {
        ck(cudaEventRecord(M.ev_fork, s), "record fork");
        ck(cudaStreamWaitEvent(sf, M.ev_fork, 0), "wait fork");
    }
    if (A.ntasks > 0 && M.prm.far_precision == 1 && !M.force_fp32) {
        {
            KTimer kt_("k_aggregate_tc", sf);
            if (P.n_tc_tasks > 0)
                k_aggregate_tc<<<P.n_tc_tasks, kTcThreads, kTcSmemBytes, sf>>>(P.largs.p, P.agg_tasks_tc.p, M.wts.p, n,
                                                                               M.nrm.p, nr, M.tc_fault.p, skip);
        }
        ck_launch("k_aggregate_tc");
    } else if (A.ntasks > 0) {
        {
            KTimer kt_("k_aggregate", sf);
            switch (nr) {
                case 1:
                    if (P.has_phases) k_aggregate_1t<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip);
                    else k_aggregate_1<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip);
                    break;
                case 2: k_aggregate_2<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip); break;
                case 3: k_aggregate_3<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip); break;
                default: k_aggregate_4<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip); break;
            }
        }
        ck_launch("k_aggregate");
    }
    if (A.ntargets > 0) {
        if (A.ntgroups > 0) {
            KTimer kt_("k_transfer", sf);
            if (nr == 4) k_transfer_m4<<<A.ntgroups, 32 * kTransferWarps, 0, sf>>>(P.largs.p, skip);
            else if (nr == 2) k_transfer_m2<<<A.ntgroups, 32 * kTransferWarps, 0, sf>>>(P.largs.p, skip);
            else k_transfer_split<<<dim3(A.ntgroups, nr), 32 * kTransferWarps, 0, sf>>>(P.largs.p, skip);
        }
        ck_launch("k_transfer");
    }
    NearArgs na = near_args(M, P, cp, cq);
    if ((nr > 1 || M.prm.near_chunk > 0) && use_store && M.prm.near_store && !P.fp().direct) {
        // all right-hand sides in one pass over the stored values, the leaf's
        // columns staged in chunks
        const int ncp = (P.lists->max_ncol + 1) & ~1;
        const int cw = std::max(2, std::min(ncp, M.prm.near_chunk > 0 ? M.prm.near_chunk : kSpmvMultiChunk));
        if (P.lists->n_spmv_items > 0) {
            KTimer kt_("k_near_spmv", s);
            k_near_spmv_items_multi<<<P.lists->n_spmv_items, kSpmvThreads, (size_t)nr * cw * sizeof(float2), s>>>(
                na, P.lists->spmv_items.p, P.val.p, M.xint.p, M.ynear.p, nr, n, cw, skip);
        }
        ck_launch("k_near_spmv");
    } else if (nr > 1) {
        // one right-hand side at a time (the values are streamed nr times)
        for (int r = 0; r < nr; ++r) {
            if (use_store && M.prm.near_store && !P.fp().direct &&
                (size_t)P.lists->max_ncol * sizeof(float2) <= 160 * 1024) {
                if (P.lists->n_spmv_items > 0) {
                    KTimer kt_("k_near_spmv", s);
                    k_near_spmv_items<<<P.lists->n_spmv_items, kSpmvThreads,
                                        (size_t)P.lists->max_ncol * sizeof(float2), s>>>(
                        na, P.lists->spmv_items.p, P.val.p, M.xint.p + r * n, M.ynear.p + r * n, skip);
                }
                ck_launch("k_near_spmv");
            } else if (use_store && M.prm.near_store && !P.fp().direct) {
                {
                    KTimer kt_("k_near_spmv", s);
                    k_near_spmv<<<nblocks(n, 8), 256, 0, s>>>(na, P.val.p, M.xint.p + r * n, M.ynear.p + r * n, skip);
                }
                ck_launch("k_near_spmv");
            } else {
                {
                    KTimer kt_("k_near_fused", s);
                    k_near_fused<<<nblocks(n, 8), 256, 0, s>>>(na, M.xint.p + r * n, M.ynear.p + r * n, fr(M).err.p,
                                                                skip);
                }
                ck_launch("k_near_fused");
            }
        }
    } else if (use_store && M.prm.near_store && !P.fp().direct) {
        const size_t xs_bytes = (size_t)P.lists->max_ncol * sizeof(float2);
        if (xs_bytes <= 160 * 1024) {
            if (P.lists->n_spmv_items > 0) {
                KTimer kt_("k_near_spmv", s);
                k_near_spmv_items<<<P.lists->n_spmv_items, kSpmvThreads, xs_bytes, s>>>(
                    na, P.lists->spmv_items.p, P.val.p, M.xint.p, M.ynear.p, skip);
            }
            ck_launch("k_near_spmv");
        } else {
            {
                KTimer kt_("k_near_spmv", s);
                k_near_spmv<<<nblocks(n, 8), 256, 0, s>>>(na, P.val.p, M.xint.p, M.ynear.p, skip);
            }
            ck_launch("k_near_spmv");
        }
    } else {
        {
            KTimer kt_("k_near_fused", s);
            k_near_fused<<<nblocks(n, 8), 256, 0, s>>>(na, M.xint.p, M.ynear.p, fr(M).err.p, skip);
        }
        ck_launch("k_near_fused");
    }
    DisaggArgs da;
    da.n = n;
    da.nrm = M.nrm.p;
    da.perm = perm_out ? M.perm.p : nullptr;
    da.k = (float)P.k;
    da.nlev = (int)P.lev.size();
    da.rowf = nullptr;
    if (fork && !far_only) {
        ck(cudaEventRecord(M.ev_join, sf), "record join");
        ck(cudaStreamWaitEvent(s, M.ev_join, 0), "wait join");
    }
    cudaStream_t sd = far_only ? sf : s;
    for (int l = 0; l < A.nlev; ++l) da.lev[l] = A.lev[l];
    da.tasks = P.lists->dis_tasks.p;
    {
        KTimer kt_("k_disaggregate", sd);
        if (P.lists->n_dis_tasks > 0) {
            if (nr == 1) {
                const float2 *yn = far_only ? nullptr : M.ynear.p;
                if (P.has_phases) k_disaggregate_m1t<<<P.lists->n_dis_tasks, kDisThreads, 0, sd>>>(da, yn, y, skip);
                else k_disaggregate_m1<<<P.lists->n_dis_tasks, kDisThreads, 0, sd>>>(da, yn, y, skip);
            } else {
                // the planes in groups of four (or two): one phase per element
                // and direction pair serves a whole group
                for (int r0 = 0; r0 < nr;) {
                    const int g = nr - r0 >= 4 ? 4 : (nr - r0 >= 2 ? 2 : 1);
                    DisaggArgs dg = da;
                    for (int l = 0; l < A.nlev; ++l) dg.lev[l].Lam = A.lev[l].Lam + r0 * A.lev[l].lplane;
                    const float2 *yn = far_only ? nullptr : M.ynear.p + r0 * n;
                    float2 *yo = y + r0 * n;
                    if (g == 4) k_disaggregate_m4<<<P.lists->n_dis_tasks, kDisThreads, 0, sd>>>(dg, yn, yo, skip);
                    else if (g == 2) k_disaggregate_m2<<<P.lists->n_dis_tasks, kDisThreads, 0, sd>>>(dg, yn, yo, skip);
                    else k_disaggregate_m1<<<P.lists->n_dis_tasks, kDisThreads, 0, sd>>>(dg, yn, yo, skip);
                    r0 += g;
                }
            }
        }
    }
    ck_launch("k_disaggregate");
    if (fork && far_only) {
        ck(cudaEventRecord(M.ev_join, sf), "record join");
        ck(cudaStreamWaitEvent(s, M.ev_join, 0), "wait join");
    }
}

// The rows of the transposed product from the stored values (per leaf t,
// every row i of its near leaves with the position of A_i,t0 in the stored
// values), built on the first transposed product of a plan's lists: outside
// any graph capture (the callers of the transposed products run it first).
void ensure_transposed_rows(bem_mesh_impl &M)
{
    Lists &Ls = *fr(M).plan->lists;
    if (Ls.trow_checked || !M.prm.near_store || Ls.fp.direct) return;
    Ls.trow_checked = true;
    const FreqPlan &F = Ls.fp;
    const Level &Lf = M.t.lv[F.leaf_depth];
    const int nl = (int)Lf.start.size();
    // the column of each near entry's first element in its row leaf's list,
    // and per (row leaf s, listed leaf) that column, sorted for lookups
    std::vector<std::pair<int64_t, int>> key;
    key.reserve(F.near_src.size());
    for (int s2 = 0; s2 < nl; ++s2) {
        int pos = 0;
        for (int q = F.near_ptr[s2]; q < F.near_ptr[s2 + 1]; ++q) {
            key.emplace_back((int64_t)s2 * nl + F.near_src[q], pos);
            pos += (int)Lf.count[F.near_src[q]];
        }
    }
    std::sort(key.begin(), key.end());
    // per leaf t, every row i of its near leaves with the position of A_i,t0
    // (row_ptr[i] + the column of t in i's row); every near pair must have
    // its mirror, else the transposed product recomputes its entries
    std::vector<int> rptr(nl + 1, 0), ri;
    std::vector<int64_t> roff;
    for (int t = 0; t < nl; ++t) {
        for (int q = F.near_ptr[t]; q < F.near_ptr[t + 1]; ++q) {
            const int sl = F.near_src[q];
            if (Lf.count[sl] == 0 || Lf.count[t] == 0) continue;
            const auto it = std::lower_bound(key.begin(), key.end(), std::make_pair((int64_t)sl * nl + t, INT_MIN));
            if (it == key.end() || it->first != (int64_t)sl * nl + t) return;   // tsym stays false
            for (int64_t i = Lf.start[sl]; i < Lf.start[sl] + Lf.count[sl]; ++i) {
                ri.push_back((int)i);
                roff.push_back(Ls.h_row_ptr[i] + it->second);
            }
        }
        if (ri.size() > (size_t)INT_MAX) throw Fail{set_err(BEM_E_ARG, "transposed near rows exceed 2^31")};
        rptr[t + 1] = (int)ri.size();
    }
    cudaStream_t s = fr(M).s;
    Ls.trow_ptr.upload(rptr, s);
    Ls.h_trow_ptr = rptr;
    Ls.trow_i.upload(ri, s);
    Ls.trow_off.upload(roff, s);
    ck(cudaStreamSynchronize(s), "sync");
    Ls.tsym = true;
    Ls.trow_ready = true;
}

// A^T stored in A's layout (near_transpose), made from the stored values of
// A once they exist and the transposed rows are listed: the transposed
// product then streams it with the forward kernel instead of reading A's
// columns.  Each leaf's transposed rows must fill exactly the stride of its
// forward rows (they do when the near lists are symmetric); else nothing is
// made and the product reads by column, as it does when the device has no
// room for A^T.  Not inside a graph capture (it allocates).
void ensure_transposed_values(bem_mesh_impl &M)
{
    ensure_transposed_rows(M);
    Plan &P = *fr(M).plan;
    const Lists &Ls = *P.lists;
    if (M.prm.near_transpose != 1 || !Ls.trow_ready || !P.val_valid || P.valT_valid) return;
    const Level &Lf = M.t.lv[Ls.fp.leaf_depth];
    const int nl = (int)Lf.start.size();
    if ((int)Ls.h_trow_ptr.size() != nl + 1) return;
    for (int t = 0; t < nl; ++t) {
        if (Lf.count[t] == 0) continue;
        const int nk = Ls.h_trow_ptr[t + 1] - Ls.h_trow_ptr[t];
        const int64_t i0 = Lf.start[t];
        if ((int64_t)((nk + 1) & ~1) != Ls.h_row_ptr[i0 + 1] - Ls.h_row_ptr[i0]) return;
    }
    cudaStream_t s = fr(M).s;
    try {
        P.valT.alloc(P.val.n);
    } catch (Fail &) {
        // no room for A^T (8 bytes per stored value): the transposed
        // product reads A by column instead
        P.valT.release();
        (void)cudaGetLastError();
        g_err.clear();
        return;
    }
    {
        KTimer kt_("k_near_transpose", s);
        k_near_transpose<<<nl, 256, 0, s>>>(Ls.leaf_start.p, Ls.trow_ptr.p, Ls.trow_off.p, Ls.row_ptr.p, P.val.p,
                                            P.valT.p);
    }
    ck_launch("k_near_transpose");
    ck(cudaStreamSynchronize(s), "sync");
    P.valT_valid = true;
}

// y = A^T x with the given column coefficients (the adjoint solve): the
// near part by k_near_spmv_t (the stored values, when they were made with
// these coefficients and the near lists are symmetric) or k_near_fused_t
// (entries recomputed), the far part by the
// forward aggregation and transfer kernels on the weights k_prep_t forms
// and k_disaggregate_t.  x: internal order, or null when x_int already
// holds x (formed by k_gs_finish).  y: caller order when perm_out, else
// internal.  far_only: y receives the far part alone and the near part
// stays in M.ynear (the Gram-Schmidt step adds them).
void matvec_t_internal(bem_mesh_impl &M, const float2 *cp, const float2 *cq, const float2 *x, float2 *y,
                       bool perm_out, bool far_only, const int *skip, cudaStream_t s)
{
    Plan &P = *fr(M).plan;
    const int64_t n = M.n;
    const bool far = !P.lev.empty();
    M.rowf.alloc(n);   // no-op when run_gmres allocated it before a graph capture
    {
        KTimer kt_("k_prep_t", s);
        k_prep_t<<<nblocks(n, 256), 256, 0, s>>>(n, x, M.xint.p, far ? M.wts.p : nullptr, M.rowf.p, M.chi.p, cp, cq,
                                                 (float)P.k, skip);
    }
    ck_launch("k_prep_t");
    const LevelsArgs &A = P.hargs;
    const bool fork = !g_timing && (A.ntasks > 0 || A.ntargets > 0);
    cudaStream_t sf = fork ? M.s_far : s;
    if (fork) {
        ck(cudaEventRecord(M.ev_fork, s), "record fork");
        ck(cudaStreamWaitEvent(sf, M.ev_fork, 0), "wait fork");
    }
    if (A.ntasks > 0) {
        {
            KTimer kt_("k_aggregate", sf);
            if (P.has_phases) k_aggregate_1t<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip);
            else k_aggregate_1<<<A.ntasks, kAggThreads, 0, sf>>>(P.largs.p, M.wts.p, n, M.nrm.p, skip);
        }
        ck_launch("k_aggregate");
    }
    if (A.ntargets > 0 && A.ntgroups > 0) {
        {
            KTimer kt_("k_transfer", sf);
            k_transfer_split<<<A.ntgroups, 32 * kTransferWarps, 0, sf>>>(P.largs.p, skip);
        }
        ck_launch("k_transfer");
    }
    const Lists &Ls = *P.lists;
    const bool stored = cp == fr(M).cp.p && cq == fr(M).cq.p && P.val_valid && M.prm.near_store && !P.fp().direct;
    const size_t xs_bytes = (size_t)Ls.max_ncol * sizeof(float2);
    if (stored && P.valT_valid && xs_bytes <= 160 * 1024) {
        // A^T stored in A's layout, streamed by the forward product's kernel
        NearArgs na = near_args(M, P, cp, cq);
        {
            KTimer kt_("k_near_spmv_t", s);
            if (Ls.n_spmv_items > 0)
                k_near_spmv_items<<<Ls.n_spmv_items, kSpmvThreads, xs_bytes, s>>>(na, Ls.spmv_items.p, P.valT.p,
                                                                                  M.xint.p, M.ynear.p, skip);
        }
        ck_launch("k_near_spmv_t");
    } else if (stored && Ls.trow_ready) {
        // the stored values of A (made with these coefficients), read by column
        {
            KTimer kt_("k_near_spmv_t", s);
            const int nl = (int)Ls.fp.near_ptr.size() - 1;
            if (nl > 0)
                k_near_spmv_t<<<nl, kSpmvTThreads, 0, s>>>(Ls.leaf_start.p, Ls.trow_ptr.p, Ls.trow_i.p,
                                                            Ls.trow_off.p, P.val.p, M.xint.p, M.ynear.p, skip);
        }
        ck_launch("k_near_spmv_t");
    } else {
        NearArgs na = near_args(M, P, cp, cq);
        {
            KTimer kt_("k_near_fused_t", s);
            k_near_fused_t<<<nblocks(n, 8), 256, 0, s>>>(na, M.xint.p, M.ynear.p, nullptr, fr(M).err.p, skip);
        }
        ck_launch("k_near_fused_t");
    }
    if (fork) {
        ck(cudaEventRecord(M.ev_join, sf), "record join");
        ck(cudaStreamWaitEvent(s, M.ev_join, 0), "wait join");
    }
    DisaggArgs da;
    da.n = n;
    da.nrm = M.nrm.p;
    da.perm = perm_out ? M.perm.p : nullptr;
    da.k = (float)P.k;
    da.nlev = (int)P.lev.size();
    da.rowf = M.rowf.p;
    for (int l = 0; l < A.nlev; ++l) da.lev[l] = A.lev[l];
    da.tasks = P.lists->dis_tasks.p;
    {
        KTimer kt_("k_disaggregate_t", s);
        const float2 *yn = far_only ? nullptr : M.ynear.p;
        if (P.lists->n_dis_tasks > 0) {
            if (P.has_phases) k_disaggregate_tt<<<P.lists->n_dis_tasks, kDisThreads, 0, s>>>(da, yn, y, skip);
            else k_disaggregate_t<<<P.lists->n_dis_tasks, kDisThreads, 0, s>>>(da, yn, y, skip);
        }
    }
    ck_launch("k_disaggregate_t");
}

// Leaf-size autotuner: builds the geometric lists for the automatic leaf
// depth and its neighbours, times the near-field entries and a few FMA
// products of each on this GPU, and keeps the depth with the smallest
// estimated solve time (entries + 40 products).  Runs once per mesh.
void autotune_leaf_depth(bem_mesh_impl &M, double k)
{
    NvtxRange nvtx_("leaf-depth autotuner");
    M.tuned = true;
    if (!M.prm.autotune || M.prm.mode == BEM_MODE_DIRECT || M.prm.leaf_edge > 0 || M.n < 4096) return;
    const int64_t n = M.n;
    DevArr<float2> tcp, tcq, tx, ty;
    std::vector<float2> h1(n, make_float2(1.f, 0.f)), h0(n, make_float2(0.f, 0.f)), hx(n);
    for (int64_t i = 0; i < n; ++i) hx[i] = make_float2(std::cos(0.37 * i), std::sin(0.11 * i));
    tcp.upload(h1, M.s);
    tcq.upload(h0, M.s);
    tx.upload(hx, M.s);
    ty.alloc(n);
    // events destroyed on every exit (a failed allocation throws from here)
    struct Events {
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        ~Events()
        {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (cudaEvent_t &x : ev.e) ck(cudaEventCreate(&x), "event");
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1], e2 = ev.e[2];
    std::vector<std::tuple<int, double, std::shared_ptr<Lists>>> cand;
    for (int d = M.leaf_depth - 1; d <= M.leaf_depth + 1; ++d) {
        if (d < 1 || d > M.t.leaf_depth) continue;
        // a deeper candidate whose leaves average under 8 elements is not
        // tried: its lists (tens of millions of leaf pairs on large meshes)
        // take longer to build than the tuner can gain
        if (d > M.leaf_depth && (double)n < 8.0 * (double)M.t.lv[d].start.size()) continue;
        bem_params gp = M.prm;
        gp.stability_max = 1e308;
        FreqPlan fp;
        build_plan(M.g, M.t, gp, k, fp, d);
        if (fp.far.empty() && d != M.leaf_depth) continue;
        auto lists = upload_lists(M, std::move(fp));
        auto P = std::make_unique<Plan>();
        P->k = k;
        P->lists = lists;
        finish_plan(M, *P);
        // the frame's plan is the candidate while it is timed; the guard
        // puts the previous one back on every exit
        struct Restore {
            std::unique_ptr<Plan> &slot;
            std::unique_ptr<Plan> keep;
            ~Restore() { slot.swap(keep); }
        } restore{fr(M).plan, nullptr};
        restore.keep.swap(fr(M).plan);
        fr(M).plan = std::move(P);
        fr(M).plan->val.alloc((size_t)fr(M).plan->nnz());
        ck(cudaEventRecord(e0, M.s), "record");
        store_near(M, *fr(M).plan, tcp.p, tcq.p);
        ck(cudaEventRecord(e1, M.s), "record");
        ck(cudaEventSynchronize(e1), "sync");
        float ms_store = 0.f, ms_mv = 0.f;
        ck(cudaEventElapsedTime(&ms_store, e0, e1), "elapsed");
        matvec_internal(M, tcp.p, tcq.p, true, tx.p, nullptr, false, ty.p, false, nullptr, M.s);   // warm-up
        // the fastest of three rounds of three products
        ms_mv = 1e30f;
        for (int round = 0; round < 3; ++round) {
            float ms = 0.f;
            ck(cudaEventRecord(e1, M.s), "record");
            for (int r = 0; r < 3; ++r)
                matvec_internal(M, tcp.p, tcq.p, true, tx.p, nullptr, false, ty.p, false, nullptr, M.s);
            ck(cudaEventRecord(e2, M.s), "record");
            ck(cudaEventSynchronize(e2), "sync");
            ck(cudaEventElapsedTime(&ms, e1, e2), "elapsed");
            ms_mv = std::min(ms_mv, ms);
        }
        const double cost = 1e-3 * (ms_store + 40.0 * ms_mv / 3.0);
        M.tune_log.push_back({d, cost});
        cand.emplace_back(d, cost, lists);
    }
    // Another depth replaces the automatic one only when it is at least 3%
    // faster, so that near ties do not flip between runs.
    std::shared_ptr<Lists> best;
    int best_d = M.leaf_depth;
    double best_cost = 1e300, auto_cost = 1e300;
    for (auto &c : cand)
        if (std::get<0>(c) == M.leaf_depth) {
            auto_cost = std::get<1>(c);
            best = std::get<2>(c);
            best_cost = 0.97 * auto_cost;
        }
    for (auto &c : cand)
        if (std::get<0>(c) != M.leaf_depth && std::get<1>(c) < best_cost) {
            best_cost = std::get<1>(c);
            best_d = std::get<0>(c);
            best = std::get<2>(c);
        }
    if (best) {
        M.leaf_depth = best_d;
        M.geo_lists = best;
    }
}

void ensure_work(bem_mesh_impl &M)
{
    // (ensure_planes may have given xint, ynear and wts room for several
    // right-hand sides; alloc keeps a larger capacity)
    M.xint.alloc(std::max<size_t>(M.xint.n, M.n));
    M.ynear.alloc(std::max<size_t>(M.ynear.n, M.n));
    M.wts.alloc(std::max<size_t>(M.wts.n, M.n));
    M.tmp.alloc(M.n);
    M.tmp2.alloc(M.n);
}

void prepare(bem_mesh_impl &M, double freq, const bem_medium *med, const double *adm, int nreg, Coeffs &C)
{
    double c, rho;
    medium_of(med, c, rho);
    if (!(freq > 0) || !std::isfinite(freq)) { g_err = "frequency must be positive"; throw Fail{BEM_E_ARG}; }
    for (int64_t e = 0; e < M.n; ++e)
        if (M.bct[e] == BEM_ADMI) {
            if (!adm || M.region[e] >= nreg) {
                g_err = "admittance missing for an ADMI element's region";
                throw Fail{BEM_E_ARG};
            }
        }
    ck(cudaSetDevice(M.device), "cudaSetDevice");
    ensure_work(M);
    build_plan_dev(M, freq, c);
    make_coeffs(M, fr(M).plan->k, 2.0 * M_PI * freq, c, rho, adm, nreg, C);
    upload_coeffs(M, C);
    ensure_near_values(M, C);
}

int resolution_warning(const bem_mesh_impl &M, double freq, const bem_medium *med)
{
    double c, rho;
    medium_of(med, c, rho);
    const double lambda = c / freq;
    if (M.g.mean_edge > lambda / 6.0) {
        char buf[160];
        snprintf(buf, sizeof buf, "mean element edge %.4g m exceeds a sixth of the wavelength (%.4g m)",
                 M.g.mean_edge, lambda / 6.0);
        g_err = buf;
        return BEM_W_UNDERRESOLVED;
    }
    return BEM_OK;
}

std::vector<SourceDev> sources_of(const bem_source *srcs, int n)
{
    std::vector<SourceDev> v(n);
    for (int i = 0; i < n; ++i) {
        if (srcs[i].kind != BEM_SRC_PLANE && srcs[i].kind != BEM_SRC_POINT) {
            g_err = "unknown source kind";
            throw Fail{BEM_E_ARG};
        }
        v[i].kind = srcs[i].kind;
        for (int q = 0; q < 3; ++q) v[i].v[q] = srcs[i].vec[q];
        v[i].amp[0] = srcs[i].amp[0];
        v[i].amp[1] = srcs[i].amp[1];
    }
    return v;
}

void join_streams(cudaStream_t from, cudaStream_t to)
{
    cudaEvent_t ev;
    ck(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    ck(cudaEventRecord(ev, from), "record");
    ck(cudaStreamWaitEvent(to, ev, 0), "wait");
    cudaEventDestroy(ev);
}


void fill_stats(const Geometry &g, const Tree &t, const FreqPlan &fp, const bem_params &p, bem_plan_stats *out)
{
    memset(out, 0, sizeof *out);
    {
        double R[kMaxRule + 1] = {0};
        order_thresholds(p.quad_tol, std::max(2, p.m_max), R);
        out->order_R[0] = p.rt_subdiv;
        for (int m = 1; m < p.m_max && m < 8; ++m) out->order_R[m] = R[m];
    }
    out->n_elements = g.n;
    out->leaf_level = fp.leaf_depth;
    out->levels = (int)fp.far.size();
    int64_t far_pairs = 0;
    for (size_t l = 0; l < fp.far.size() && l < 16; ++l) {
        const FarLevel &F = fp.far[l];
        const Level &L = t.lv[F.depth];
        out->level_depth[l] = F.depth;
        out->L[l] = F.L;
        out->n_clusters[l] = F.nc;
        out->n_interactions[l] = F.n_inter;
        out->n_offsets[l] = (int)(F.offsets.size() / 3);
        std::vector<char> src(F.nc, 0);
        for (int c = 0; c < F.nc; ++c) {
            for (int q = F.il_ptr[c]; q < F.il_ptr[c + 1]; ++q) {
                far_pairs += L.count[c] * L.count[F.il_src[q]];
                src[F.il_src[q]] = 1;
            }
            if (F.il_ptr[c + 1] > F.il_ptr[c]) out->n_tgt_elements[l] += L.count[c];
        }
        for (int c = 0; c < F.nc; ++c)
            if (src[c]) out->n_src_elements[l] += L.count[c];
    }
    out->far_pairs = far_pairs;
    // symmetry of the lists (the transposed product reads them backwards):
    // near leaf pairs (a, b) without (b, a), interaction entries (c, s)
    // without (s, c) at the same level
    int64_t asym = 0;   // element pairs
    auto count_asym = [&asym](std::vector<int64_t> &keys, int64_t m, const std::vector<int64_t> &cnt) {
        std::sort(keys.begin(), keys.end());
        for (int64_t key : keys)
            if (!std::binary_search(keys.begin(), keys.end(), (key % m) * m + key / m))
                asym += cnt[key / m] * cnt[key % m];
    };
    {
        const int64_t nl = (int64_t)fp.near_ptr.size() - 1;
        std::vector<int64_t> keys;
        for (int64_t a = 0; a < nl; ++a)
            for (int q = fp.near_ptr[a]; q < fp.near_ptr[a + 1]; ++q) keys.push_back(a * nl + fp.near_src[q]);
        if (nl > 0) count_asym(keys, nl, t.lv[fp.leaf_depth].count);
    }
    out->asymmetric_near_pairs = asym;
    for (const FarLevel &F : fp.far) {
        std::vector<int64_t> keys;
        for (int c = 0; c < F.nc; ++c)
            for (int q = F.il_ptr[c]; q < F.il_ptr[c + 1]; ++q) keys.push_back((int64_t)c * F.nc + F.il_src[q]);
        if (F.nc > 0) count_asym(keys, F.nc, t.lv[F.depth].count);
    }
    out->asymmetric_pairs = asym;
    out->n_leaves = (int)t.lv[fp.leaf_depth].start.size();
    out->near_nnz = fp.nnz;
    const NearCount nc = count_near_points(g, t, fp, p);
    out->near_light_entries = nc.light_entries;
    out->near_light_points = nc.light_points;
    out->near_heavy_entries = nc.heavy_entries;
    out->near_heavy_points = nc.heavy_points;
    out->near_quad_points = nc.light_points + nc.heavy_points;
    out->leaf_edge = t.lv[fp.leaf_depth].box;
    out->mean_edge = g.mean_edge;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

void bem_params_default(bem_params *p)
{
    if (!p) return;
    p->mode = BEM_MODE_FMM;
    p->quad_tol = 1e-3;
    p->m_max = 6;
    p->rt_subdiv = 1.3;
    p->max_depth = 15;
    p->trunc_factor = 1.8;
    p->L_min = 8;
    p->admissibility = 2.0 / std::sqrt(3.0);
    p->leaf_edge = 0.0;
    p->stability_max = 1e3;
    p->near_store = 1;
    p->restart = 100;
    p->autotune = 1;
    p->tau = 1.0;
    p->row_scaling = 0;
    p->check_orientation = 0;
    p->symmetric_far = 0;
    p->block_jacobi = 0;
    p->far_precision = 0;
    p->near_chunk = 0;
    p->gs_rows = 0;
    p->field_mode = 0;
    p->far_table = 0;
    p->graphs = 1;
    p->near_transpose = 1;
}

const char *bem_last_error(void) { return g_err.c_str(); }

uint64_t bem_launch_count(void) { return g_launches.load(); }

int bem_mesh_create(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris,
                    const int32_t *bc_type, const double *bc_value, const int32_t *region,
                    const bem_params *params, void **out)
{
    NvtxRange nvtx_("bem_mesh_create");
    if (!out) return set_err(BEM_E_ARG, "out is NULL");
    *out = nullptr;
    if (!nodes || !tris || n_nodes < 3 || n_tris < 1) return set_err(BEM_E_ARG, "empty mesh");
    if (n_tris > INT_MAX / 2) return set_err(BEM_E_ARG, "too many elements");
    bem_params p;
    bem_params_default(&p);
    if (params) p = *params;
    if (p.m_max < 1 || p.m_max > kMaxRule) return set_err(BEM_E_ARG, "m_max must be in 1..6");
    if (p.max_depth < 0 || p.max_depth > 15) return set_err(BEM_E_ARG, "max_depth must be in 0..15");
    if (p.restart < 2 || p.restart > kMaxRestart) return set_err(BEM_E_ARG, "restart must be in 2..1024");
    if (!(p.tau == 1.0 || p.tau == -1.0)) return set_err(BEM_E_ARG, "tau must be +1 (exterior) or -1 (interior)");
    if (p.row_scaling != 0 && p.row_scaling != 1) return set_err(BEM_E_ARG, "row_scaling must be 0 or 1");
    if (p.check_orientation != 0 && p.check_orientation != 1)
        return set_err(BEM_E_ARG, "check_orientation must be 0 or 1");
    if (p.symmetric_far != 0 && p.symmetric_far != 1) return set_err(BEM_E_ARG, "symmetric_far must be 0 or 1");
    if (p.block_jacobi != 0 && p.block_jacobi != 1) return set_err(BEM_E_ARG, "block_jacobi must be 0 or 1");
    if (p.far_precision != 0 && p.far_precision != 1) return set_err(BEM_E_ARG, "far_precision must be 0 or 1");
    if (p.near_chunk != 0 && (p.near_chunk < 64 || p.near_chunk > 4096 || (p.near_chunk & 1)))
        return set_err(BEM_E_ARG, "near_chunk must be 0 or an even number in 64..4096");
    if (p.field_mode < 0 || p.field_mode > 2) return set_err(BEM_E_ARG, "field_mode must be 0, 1 or 2");
    if (p.far_table != 0 && p.far_table != 1) return set_err(BEM_E_ARG, "far_table must be 0 or 1");
    if (p.graphs != 0 && p.graphs != 1) return set_err(BEM_E_ARG, "graphs must be 0 or 1");
    if (p.near_transpose != 0 && p.near_transpose != 1) return set_err(BEM_E_ARG, "near_transpose must be 0 or 1");
    if (p.gs_rows != 0 && (p.gs_rows < 64 || p.gs_rows > kGsMaxRows))
        return set_err(BEM_E_ARG, "gs_rows must be 0 or in 64..1024");
    if (p.block_jacobi && p.row_scaling)
        return set_err(BEM_E_ARG, "row_scaling and block_jacobi are alternatives: set at most one");
    if (!(p.quad_tol > 0) || !(p.rt_subdiv > 0) || !(p.admissibility > 0) || p.L_min < 1 || p.L_min > 200)
        return set_err(BEM_E_ARG, "invalid parameter");
    if (p.check_orientation) {
        // host only, before any device work
        try {
            Geometry g;
            std::string e = compute_geometry(nodes, n_nodes, tris, n_tris, g);
            if (!e.empty()) return set_err(BEM_E_ARG, e);
            const MeshCheck mc = check_mesh(g, nodes, n_nodes, tris, n_tris);
            char buf[200];
            if (mc.open_edges || mc.misoriented_edges) {
                snprintf(buf, sizeof buf, "orientation check: %lld edges not shared by two triangles, %lld shared "
                                          "edges wound the same way by both",
                         (long long)mc.open_edges, (long long)mc.misoriented_edges);
                return set_err(BEM_E_ARG, buf);
            }
            if (!(mc.volume > 0)) {
                snprintf(buf, sizeof buf, "orientation check: the normals point into the enclosed volume (signed "
                                          "volume %.6g m^3); reverse the winding of every triangle",
                         mc.volume);
                return set_err(BEM_E_ARG, buf);
            }
        } catch (std::bad_alloc &) {
            return set_err(BEM_E_OOM, "host allocation failed");
        }
    }
    try {
        auto M = std::make_unique<bem_mesh_impl>();
        M->prm = p;
        M->n = n_tris;
        std::string e = compute_geometry(nodes, n_nodes, tris, n_tris, M->g);
        if (!e.empty()) return set_err(BEM_E_ARG, e);
        M->bct.assign(n_tris, BEM_VELO);
        M->bcv.assign(2 * n_tris, 0.0);
        M->region.assign(n_tris, 0);
        for (int64_t j = 0; j < n_tris; ++j) {
            if (bc_type) {
                if (bc_type[j] < 0 || bc_type[j] > 2) return set_err(BEM_E_ARG, "bad boundary type");
                M->bct[j] = bc_type[j];
            }
            if (bc_value) { M->bcv[2 * j] = bc_value[2 * j]; M->bcv[2 * j + 1] = bc_value[2 * j + 1]; }
            if (region) {
                if (region[j] < 0) return set_err(BEM_E_ARG, "negative region");
                M->region[j] = region[j];
            }
        }
        const double leaf = p.mode == BEM_MODE_DIRECT ? 0.0
                            : (p.leaf_edge > 0 ? p.leaf_edge : auto_leaf_edge(M->g, p));
        const bool tune = p.autotune && p.mode != BEM_MODE_DIRECT && !(p.leaf_edge > 0) && n_tris >= 4096;
        // one level deeper than the automatic leaves so the tuner can try a
        // finer leaf size; the lists use M->leaf_depth
        build_tree(M->g, tune ? 0.5 * leaf : leaf, M->t);
        M->leaf_depth = tune ? std::max(0, M->t.leaf_depth - 1) : M->t.leaf_depth;
        M->tuned = !tune;
        ck(cudaGetDevice(&M->device), "cudaGetDevice");
        ck(cudaStreamCreateWithFlags(&M->s, cudaStreamNonBlocking), "stream");
        ck(cudaStreamCreateWithFlags(&M->s_setup, cudaStreamNonBlocking), "stream");
        M->cur.s = M->s;
        M->next.s = M->s_setup;
        {
            int lo = 0, hi = 0;
            ck(cudaDeviceGetStreamPriorityRange(&lo, &hi), "stream priorities");
            ck(cudaStreamCreateWithPriority(&M->s_far, cudaStreamNonBlocking, hi), "stream");
            ck(cudaEventCreateWithFlags(&M->ev_fork, cudaEventDisableTiming), "event");
            ck(cudaEventCreateWithFlags(&M->ev_join, cudaEventDisableTiming), "event");
            ck(cudaStreamCreateWithFlags(&M->s_giv, cudaStreamNonBlocking), "stream");
            for (int t = 0; t < kStepsPerGraph; ++t) {
                ck(cudaEventCreateWithFlags(&M->ev_orth[t], cudaEventDisableTiming), "event");
                ck(cudaEventCreateWithFlags(&M->ev_giv[t], cudaEventDisableTiming), "event");
            }
            ck(cudaMallocHost(&M->h_st, 2 * sizeof(GmresState)), "cudaMallocHost");
            M->h_st_planes = 1;
        }
        const int64_t n = n_tris;
        std::vector<float4> chi(n), clo(n), nr(n), va(n), e1(n), e2(n);
        std::vector<double> cd(3 * n), vad(3 * n), e1d(3 * n), e2d(3 * n), ad(n);
        std::vector<int> ty(n);
        M->type_int.resize(n);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t j = M->t.perm[i];
            const double *c = &M->g.cen[3 * j];
            const float h0 = (float)c[0], h1 = (float)c[1], h2 = (float)c[2];
            chi[i] = make_float4(h0, h1, h2, (float)M->g.area[j]);
            clo[i] = make_float4((float)(c[0] - h0), (float)(c[1] - h1), (float)(c[2] - h2), 0.f);
            nr[i] = make_float4((float)M->g.nrm[3 * j], (float)M->g.nrm[3 * j + 1], (float)M->g.nrm[3 * j + 2], 0.f);
            va[i] = make_float4((float)M->g.va[3 * j], (float)M->g.va[3 * j + 1], (float)M->g.va[3 * j + 2], 0.f);
            e1[i] = make_float4((float)M->g.e1[3 * j], (float)M->g.e1[3 * j + 1], (float)M->g.e1[3 * j + 2], 0.f);
            e2[i] = make_float4((float)M->g.e2[3 * j], (float)M->g.e2[3 * j + 1], (float)M->g.e2[3 * j + 2], 0.f);
            for (int q = 0; q < 3; ++q) {
                cd[3 * i + q] = c[q];
                vad[3 * i + q] = M->g.va[3 * j + q];
                e1d[3 * i + q] = M->g.e1[3 * j + q];
                e2d[3 * i + q] = M->g.e2[3 * j + q];
            }
            ad[i] = M->g.area[j];
            ty[i] = M->bct[j];
        }
        cudaStream_t s = M->s;
        M->chi.upload(chi, s); M->clo.upload(clo, s); M->nrm.upload(nr, s);
        M->va.upload(va, s); M->e1.upload(e1, s); M->e2.upload(e2, s);
        M->cd.upload(cd, s); M->vad.upload(vad, s); M->e1d.upload(e1d, s); M->e2d.upload(e2d, s);
        M->ad.upload(ad, s);
        M->perm.upload(M->t.perm, s);
        M->type.upload(ty, s);
        ck(cudaFuncSetAttribute(k_near_spmv_items, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024),
           "cudaFuncSetAttribute");
        ck(cudaFuncSetAttribute(k_near_spmv_items_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kMaxPlanes * 4096 * sizeof(float2))),
           "cudaFuncSetAttribute");

        ck(cudaFuncSetAttribute(k_gm_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 100 * 16),
           "cudaFuncSetAttribute");
        if (p.far_precision == 1) {
            ck(cudaFuncSetAttribute(k_aggregate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes),
               "cudaFuncSetAttribute");
        }
        M->tc_fault.alloc(1);
        ck(cudaMemsetAsync(M->tc_fault.p, 0, sizeof(int), s), "memset");

        std::vector<QuadTables> qt(1, make_tables(p));
        M->Q.upload(qt, s);
        {
            const int none = INT_MAX;
            for (Frame *F : {&M->cur, &M->next}) {
                F->err.alloc(1);
                ck(cudaMemcpyAsync(F->err.p, &none, sizeof none, cudaMemcpyHostToDevice, s), "H2D err");
            }
        }
        ck(cudaStreamSynchronize(s), "sync");
        *out = M.release();
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    } catch (std::bad_alloc &) {
        return set_err(BEM_E_OOM, "host allocation failed");
    }
}

int bem_mesh_destroy(void *mesh)
{
    if (!mesh) return set_err(BEM_E_ARG, "mesh is NULL");
    auto *M = (bem_mesh_impl *)mesh;
    cudaSetDevice(M->device);
    if (M->s) cudaStreamSynchronize(M->s);
    delete M;
    return BEM_OK;
}

int bem_matvec(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
               int32_t n_regions, const void *x_dev, void *y_dev, int32_t n_rhs, void *stream)
{
    NvtxRange nvtx_("bem_matvec");
    if (!mesh || !x_dev || !y_dev || n_rhs < 1) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        cudaStream_t us = (cudaStream_t)stream;
        Coeffs C;
        join_streams(us, M.s);
        prepare(M, freq_hz, medium, admittance, n_regions, C);
        // up to kMaxPlanes right-hand sides per pass: one stream of the stored
        // near field and one phase per element and direction for all of them
        for (int r = 0; r < n_rhs; r += kMaxPlanes) {
            const int nr = std::min(kMaxPlanes, n_rhs - r);
            const float2 *x = (const float2 *)x_dev + (int64_t)r * M.n;
            float2 *y = (float2 *)y_dev + (int64_t)r * M.n;
            matvec_internal(M, fr(M).cp.p, fr(M).cq.p, true, x, nullptr, true, y, true, nullptr, M.s, false, false,
                            nr);
        }
        check_tc_fault(M);
        join_streams(M.s, us);
        return resolution_warning(M, freq_hz, medium);
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_matvec_transpose(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                         int32_t n_regions, const void *x_dev, void *y_dev, void *stream)
{
    NvtxRange nvtx_("bem_matvec_transpose");
    if (!mesh || !x_dev || !y_dev) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        cudaStream_t us = (cudaStream_t)stream;
        Coeffs C;
        join_streams(us, M.s);
        prepare(M, freq_hz, medium, admittance, n_regions, C);
        reset_err(M);
        M.tmp.alloc(M.n);
        {
            KTimer kt_("k_gather", M.s);
            k_gather<<<nblocks(M.n, 256), 256, 0, M.s>>>((const float2 *)x_dev, M.perm.p, M.n, M.tmp.p);
        }
        ck_launch("k_gather");
        ensure_transposed_values(M);
        matvec_t_internal(M, fr(M).cp.p, fr(M).cq.p, M.tmp.p, (float2 *)y_dev, true, false, nullptr, M.s);
        check_err(M);
        join_streams(M.s, us);
        return resolution_warning(M, freq_hz, medium);
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_matvec_host(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                    int32_t n_regions, const void *x_host, void *y_host, int32_t n_rhs, void *stream)
{
    NvtxRange nvtx_("bem_matvec_host");
    if (!mesh || !x_host || !y_host || n_rhs < 1) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        ck(cudaSetDevice(M.device), "cudaSetDevice");
        M.bvec.alloc((size_t)M.n * n_rhs);
        M.uvec.alloc((size_t)M.n * n_rhs);
        cudaStream_t us = (cudaStream_t)stream;
        const size_t bytes = (size_t)M.n * n_rhs * sizeof(float2);
        ck(cudaMemcpyAsync(M.bvec.p, x_host, bytes, cudaMemcpyHostToDevice, us), "H2D x");
        int st = bem_matvec(mesh, freq_hz, medium, admittance, n_regions, M.bvec.p, M.uvec.p, n_rhs, stream);
        if (st < 0) return st;
        ck(cudaMemcpyAsync(y_host, M.uvec.p, bytes, cudaMemcpyDeviceToHost, us), "D2H y");
        ck(cudaStreamSynchronize(us), "sync");
        resolve_timing();
        return st;
    } catch (Fail &f) {
        return f.code;
    }
}

namespace {

struct GmresResult {
    int total_iters = 0, restarts = 0;   // plane 0 (the only one unless nr > 1)
    bool converged = false;
    GmresState h;
    std::vector<GmresState> hp;          // final state of every plane
    std::vector<int> iters;              // products of every plane
    std::vector<char> conv;              // convergence of every plane
};

// Restarted GMRES on A u = b, or on A^T u = b when transposed (the adjoint
// solve; matvec_t_internal), for nr right-hand sides at once (nr systems in
// lockstep, each with its own Krylov basis, Hessenberg matrix and state,
// sharing every product: the product takes all planes in one pass), with b
// in M.bvec and u in M.uvec (nr planes of n, internal order), for the
// current frame's plan and column coefficients.  Preconditioned (row scaling
// or block-Jacobi) when the mesh asks for it (the forward system only; the
// caller has preconditioned b).  Throws Fail.
GmresResult run_gmres(bem_mesh_impl &M, double tol, int32_t max_iter, bool transposed, int nr = 1)
{
    cudaStream_t s = M.s;
    const int64_t n = M.n;
    const int m = M.prm.restart;
    const bool rscale = M.prm.row_scaling != 0 && !transposed;
    const bool bjac = M.prm.block_jacobi != 0 && !transposed;
    const Lists &Lb = *fr(M).plan->lists;
    GmresResult R;
    if (transposed) M.rowf.alloc(n);   // before the Arnoldi steps are captured (no allocation in a capture)
    if (nr > 1) ensure_planes(M, nr);
    // GMRES workspace, nr planes of each
    const int64_t vplane = (int64_t)(m + 1) * n, hplane = (int64_t)(m + 1) * m;
    M.V.alloc((size_t)nr * vplane);
    M.w.alloc((size_t)nr * n);
    M.H.alloc((size_t)nr * hplane);
    M.cs.alloc((size_t)nr * m);
    M.sn.alloc((size_t)nr * m);
    M.g_.alloc((size_t)nr * (m + 1));
    M.yv.alloc((size_t)nr * (m + 1));
    // the Gram-Schmidt step: block b owns rows [b R, b R + R), R <= kGsMaxRows
    // (staged in shared memory); 128 rows per block (measured against 64,
    // 256 and 512: 64 made twice the atomic additions, the larger ones kept
    // fewer loads of the basis in flight), and more when that would exceed
    // about 1024 blocks
    int nblk = 0;
    {
        const int64_t rows = M.prm.gs_rows > 0 ? (int64_t)M.prm.gs_rows : std::max<int64_t>(128, (n + 1023) / 1024);
        nblk = (int)std::max<int64_t>(1, (n + rows - 1) / rows);
    }
    const int orows = (int)((n + nblk - 1) / nblk);
    M.gsacc.alloc((size_t)8 * nr);
    M.gsh2.alloc((size_t)2 * (m + 1) * nr);
    const int nnorm = (int)nblocks(n, 256);
    const int npart = std::max(nnorm, nblk);
    M.normpart.alloc((size_t)npart * nr);
    M.st.alloc(nr);
    if (M.h_st_planes < nr) {
        if (M.h_st) cudaFreeHost(M.h_st);
        M.h_st = nullptr;
        M.h_st_planes = 0;
        ck(cudaMallocHost(&M.h_st, 2 * nr * sizeof(GmresState)), "cudaMallocHost");
        M.h_st_planes = nr;
    }
    {
        std::vector<GmresState> hs(nr);
        memset(hs.data(), 0, nr * sizeof(GmresState));
        for (auto &h : hs) {
            h.tol = tol;
            h.maxit = max_iter;
        }
        ck(cudaMemcpyAsync(M.st.p, hs.data(), nr * sizeof(GmresState), cudaMemcpyHostToDevice, s), "H2D st");
    }
    ck(cudaMemsetAsync(M.uvec.p, 0, (size_t)nr * n * sizeof(float2), s), "memset x");
    ck(cudaMemsetAsync(M.H.p, 0, M.H.bytes(), s), "memset H");
    // per-plane pointers of the Gram-Schmidt and Givens kernels
    std::vector<GsArgs> oa(nr);
    for (int r = 0; r < nr; ++r) {
        GmresArgs &ga = oa[r].g;
        ga.V = M.V.p + r * vplane;
        ga.w = M.w.p + r * n;
        ga.n = n;
        ga.st = M.st.p + r;
        ga.nblk = nblk;
        ga.H = M.H.p + r * hplane;
        ga.cs = M.cs.p + (int64_t)r * m;
        ga.sn = M.sn.p + (int64_t)r * m;
        ga.g = M.g_.p + (int64_t)r * (m + 1);
        ga.normpart = M.normpart.p + (int64_t)r * npart;
        ga.m = m;
        oa[r].next = prep_args(M, fr(M).cp.p, fr(M).cq.p, nullptr);
        oa[r].next.xint = M.xint.p + r * n;
        if (oa[r].next.wts) oa[r].next.wts = M.wts.p + r * n;
        oa[r].wnear = M.ynear.p + r * n;
        oa[r].acc = M.gsacc.p + 8 * r;
        oa[r].g.gs_acc = oa[r].acc;
        oa[r].h2 = M.gsh2.p + (int64_t)2 * (m + 1) * r;
        oa[r].rows = orows;
    }
    // the product inputs of every plane's v_0 (later basis vectors get
    // theirs from k_gs_finish)
    auto prep_v0 = [&]() {
        PrepArgs pa = prep_args(M, fr(M).cp.p, fr(M).cq.p, M.V.p);
        pa.plane = n;
        pa.xplane = vplane;
        {
            KTimer kt_("k_prep", s);
            k_prep<<<dim3(nblocks(n, 256), nr), 256, 0, s>>>(pa, nullptr);
        }
        ck_launch("k_prep");
    };
    // r0 = b, V_0 = r0 / ||r0||, cycle state reset (every plane)
    auto start = [&](const float2 *r0, int first) {
        for (int r = 0; r < nr; ++r) {
            {
                KTimer kt_("k_norm_part", s);
                k_norm_part<<<nnorm, 256, 0, s>>>(r0 + r * n, n, oa[r].g.normpart);
            }
            ck_launch("k_norm_part");
            {
                KTimer kt_("k_gm_start", s);
                k_gm_start<<<nblocks(n, 256), 256, 0, s>>>(oa[r].g.st, oa[r].g.V, r0 + r * n, n, oa[r].g.normpart,
                                                           nnorm, oa[r].g.g, m, first, oa[r].acc, oa[r].h2);
            }
            ck_launch("k_gm_start");
        }
        prep_v0();
    };
    start(M.bvec.p, 1);
    // skip flag of the product kernels: uniform within every launch; with
    // several planes the product runs until every plane is done
    const int *done = nr == 1 ? &M.st.p->skip_prod : &M.st.p->skip_all;
    // one Arnoldi step: product of v_j (inputs already formed), then the
    // Gram-Schmidt / Givens step, which also forms v_{j+1}
    const bool use_graph = !g_timing && M.prm.graphs != 0;
    // Arnoldi steps per graph (and per status read).  With event timing
    // on, one step per read and every kernel on one stream, so that each
    // kernel is timed alone and no timed launch is a skipped one.
    const int batch = use_graph ? kStepsPerGraph : 1;
    auto ortho = [&]() {
        for (int r = 0; r < nr; ++r) {
            {
                KTimer kt_("k_gs_dots", s);
                k_gs_dots<<<nblk, kGsThreads, 0, s>>>(oa[r]);
            }
            ck_launch("k_gs_dots");
            {
                KTimer kt_("k_gs_update", s);
                k_gs_update<<<nblk, kGsThreads, 0, s>>>(oa[r]);
            }
            ck_launch("k_gs_update");
            {
                KTimer kt_("k_gs_finish", s);
                k_gs_finish<<<nblk, kGsThreads, 0, s>>>(oa[r]);
            }
            ck_launch("k_gs_finish");

        }
        if (nr > 1) {
            k_gm_skip_all<<<1, 32, 0, s>>>(M.st.p, nr);
            ck_launch("k_gm_skip_all");
        }
    };
    auto givens = [&](cudaStream_t gs) {
        for (int r = 0; r < nr; ++r) {
            {
                KTimer kt_("k_gm_givens", gs);
                k_gm_givens<<<1, 32, 0, gs>>>(oa[r].g);
            }
            ck_launch("k_gm_givens");
        }
    };
    // the preconditioner on every plane of w (and of the near part, which
    // the Gram-Schmidt step would add, when wnear is given)
    auto precond = [&](float2 *w, float2 *wnear, const int *skip) {
        for (int r = 0; r < nr; ++r) {
            if (rscale) {
                {
                    KTimer kt_("k_row_scale", s);
                    k_row_scale<<<nblocks(n, 256), 256, 0, s>>>(w + r * n, wnear ? wnear + r * n : nullptr, M.dinv.p,
                                                                n, skip);
                }
                ck_launch("k_row_scale");
            }
            if (bjac) {
                // w <- P (w + wnear), the near part cleared
                {
                    KTimer kt_("k_bj_apply", s);
                    k_bj_apply<<<(unsigned)Lb.h_bj.size(), kBjMax, 0, s>>>(Lb.bj.p, M.bjinv.p, w + r * n,
                                                                           wnear ? wnear + r * n : nullptr, skip);
                }
                ck_launch("k_bj_apply");
            }
        }
    };
    // the product of the current basis vectors (their inputs already
    // formed), preconditioned when the mesh asks for it
    auto product = [&]() {
        if (transposed) {
            matvec_t_internal(M, fr(M).cp.p, fr(M).cq.p, nullptr, M.w.p, false, true, done, s);
            return;
        }
        matvec_internal(M, fr(M).cp.p, fr(M).cq.p, true, nullptr, nullptr, false, M.w.p, false, done, s, true, true,
                        nr);
        precond(M.w.p, M.ynear.p, done);
    };
    // nsteps Arnoldi steps, each the Gram-Schmidt step of column j
    // (which also forms v_{j+1}'s product inputs), the Givens step and
    // the product of v_{j+1}; a cycle's first product runs before its
    // first steps.  In the graph the Givens step runs on a side stream
    // beside the product, which does not need it, and the next
    // Gram-Schmidt step waits for it; the last Givens step of a graph
    // ends beside its last product, so it does not delay the next graph.
    auto arnoldi_steps = [&](int nsteps) {
        const bool side = use_graph;
        for (int t = 0; t < nsteps; ++t) {
            if (side && t > 0) ck(cudaStreamWaitEvent(s, M.ev_giv[t - 1], 0), "wait givens");
            ortho();
            if (side) {
                ck(cudaEventRecord(M.ev_orth[t], s), "record ortho");
                ck(cudaStreamWaitEvent(M.s_giv, M.ev_orth[t], 0), "wait ortho");
                givens(M.s_giv);
                ck(cudaEventRecord(M.ev_giv[t], M.s_giv), "record givens");
            } else {
                givens(s);
            }
            product();
        }
        if (side) ck(cudaStreamWaitEvent(s, M.ev_giv[nsteps - 1], 0), "join givens");
    };
    // Bodies of `batch` Arnoldi steps per cycle at most (the cycle's m
    // steps and one body of skipped steps to spare).
    const int max_graphs = (m + batch + batch - 1) / batch;
    // With graphs, one Arnoldi cycle is one graph launch: a WHILE node whose
    // body is `batch` Arnoldi steps and k_gm_continue, which sets the loop
    // condition on the device (some plane not done, fewer than max_graphs
    // bodies run), so the host waits once per cycle and no body is queued
    // after the cycle has ended.
    uint64_t per_graph = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (use_graph) {
        ck(cudaGraphCreate(&graph, 0), "graph create");
        cudaGraphConditionalHandle loop;
        ck(cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault), "conditional handle");
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};   // the rest zero
        np.conditional.handle = loop;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t wnode;
        ck(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &np), "conditional node");
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const uint64_t before = g_launches.load();
        ck(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal), "capture");
        arnoldi_steps(batch);
        k_gm_continue<<<1, 32, 0, s>>>(loop, M.st.p, nr, max_graphs);
        ck_launch("k_gm_continue");
        ck(cudaStreamEndCapture(s, &body), "end capture");
        per_graph = g_launches.load() - before;
        g_launches.fetch_sub(per_graph);   // captured, not launched
        ck(cudaGraphInstantiate(&gexec, graph, 0), "instantiate");
    }
    R.hp.assign(nr, GmresState());
    for (;;) {
        product();
        if (use_graph) {
            ck(cudaGraphLaunch(gexec, s), "graph launch");
            ck(cudaMemcpyAsync(M.h_st, M.st.p, nr * sizeof(GmresState), cudaMemcpyDeviceToHost, s), "D2H st");
            ck(cudaStreamSynchronize(s), "sync st");
            g_launches.fetch_add(per_graph * (uint64_t)std::max(0, M.h_st[0].bodies));
            for (int r = 0; r < nr; ++r) R.hp[r] = M.h_st[r];
        } else {
            // one step per status read (event timing: every kernel on one
            // stream, timed alone)
            for (int launched = 0; launched < max_graphs; ++launched) {
                arnoldi_steps(1);
                ck(cudaMemcpyAsync(M.h_st, M.st.p, nr * sizeof(GmresState), cudaMemcpyDeviceToHost, s), "D2H st");
                ck(cudaStreamSynchronize(s), "sync st");
                bool all_done = true;
                for (int r = 0; r < nr; ++r) {
                    R.hp[r] = M.h_st[r];
                    all_done = all_done && R.hp[r].done;
                }
                if (all_done) break;
            }
        }
        for (int r = 0; r < nr; ++r) {
            {
                KTimer kt_("k_gm_backsolve", s);
                const int tri_cols = std::min(m, 100);
                k_gm_backsolve<<<1, 256, (size_t)tri_cols * tri_cols * sizeof(double2), s>>>(
                    oa[r].g.st, oa[r].g.H, oa[r].g.g, M.yv.p + (int64_t)r * (m + 1), m, tri_cols);
            }
            ck_launch("k_gm_backsolve");
            {
                KTimer kt_("k_gm_xupdate", s);
                k_gm_xupdate<<<nblocks(n, 256), 256, 0, s>>>(M.uvec.p + r * n, oa[r].g.V, n, oa[r].g.st,
                                                             M.yv.p + (int64_t)r * (m + 1));
            }
            ck_launch("k_gm_xupdate");
        }
        bool all_conv = true, at_max = false;
        for (int r = 0; r < nr; ++r) {
            all_conv = all_conv && R.hp[r].converged;
            at_max = at_max || R.hp[r].iters >= max_iter;
        }
        if (all_conv || at_max) break;
        // restart (every plane): r = b - A x
        ++R.restarts;
        if (transposed) {
            matvec_t_internal(M, fr(M).cp.p, fr(M).cq.p, M.uvec.p, M.w.p, false, false, nullptr, s);
        } else {
            matvec_internal(M, fr(M).cp.p, fr(M).cq.p, true, M.uvec.p, nullptr, false, M.w.p, false, nullptr, s, false,
                            false, nr);
        }
        precond(M.w.p, nullptr, nullptr);
        k_rsub<<<nblocks((int64_t)nr * n, 256), 256, 0, s>>>(M.w.p, M.bvec.p, (int64_t)nr * n);   // w = P (b - A x)
        ck_launch("k_rsub");
        start(M.w.p, 0);
        ck(cudaMemsetAsync(M.H.p, 0, M.H.bytes(), s), "memset H");
        ck(cudaMemcpyAsync(M.h_st, M.st.p, nr * sizeof(GmresState), cudaMemcpyDeviceToHost, s), "D2H st");
        ck(cudaStreamSynchronize(s), "sync");
        bool all_done = true;
        for (int r = 0; r < nr; ++r) all_done = all_done && M.h_st[r].done;
        if (all_done) {
            for (int r = 0; r < nr; ++r) R.hp[r] = M.h_st[r];
            break;
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    R.iters.resize(nr);
    R.conv.resize(nr);
    for (int r = 0; r < nr; ++r) {
        R.iters[r] = R.hp[r].iters;
        R.conv[r] = R.hp[r].converged;
    }
    R.h = R.hp[0];
    R.total_iters = R.hp[0].iters;
    R.converged = R.hp[0].converged;
    return R;
}

// The solver's preconditioner (row scaling or block-Jacobi, when the mesh
// asks for one) applied to nr planes of b in place.
void precondition_rhs(bem_mesh_impl &M, float2 *b, int nr)
{
    cudaStream_t s = M.s;
    const int64_t n = M.n;
    const Lists &Lb = *fr(M).plan->lists;
    for (int r = 0; r < nr; ++r) {
        if (M.prm.row_scaling) {
            {
                KTimer kt_("k_row_scale", s);
                k_row_scale<<<nblocks(n, 256), 256, 0, s>>>(b + r * n, nullptr, M.dinv.p, n, nullptr);
            }
            ck_launch("k_row_scale");
        }
        if (M.prm.block_jacobi) {
            {
                KTimer kt_("k_bj_apply", s);
                k_bj_apply<<<(unsigned)Lb.h_bj.size(), kBjMax, 0, s>>>(Lb.bj.p, M.bjinv.p, b + r * n, nullptr, nullptr);
            }
            ck_launch("k_bj_apply");
        }
    }
}

// Iterative refinement of a solve whose products aggregate in split BF16 on
// the tensor cores (far_precision 1): the solution is kept in FP64 (x64), the
// residual r = b - A x is formed with the FP32 products and differenced in
// FP64, and each inner GMRES (the mixed-precision products, preconditioned
// as the mesh asks) solves A d = r to half the remaining target, x64 += d,
// until ||r|| <= tol ||b|| for every plane (the true residual of the FP32
// operator, not the GMRES estimate of the mixed-precision one).  b:
// M.bvec (nr planes, not preconditioned); the solution ends in M.uvec.
// Products: inner products plus one FP32 product per outer step.
GmresResult run_refined(bem_mesh_impl &M, double tol, int32_t max_iter, int nr)
{
    cudaStream_t s = M.s;
    const int64_t n = M.n;
    const size_t pn = (size_t)nr * n;
    M.bsave.alloc(pn);
    M.xcur.alloc(pn);
    M.rtmp.alloc(pn);
    M.x64.alloc(pn);
    ck(cudaMemcpyAsync(M.bsave.p, M.bvec.p, pn * sizeof(float2), cudaMemcpyDeviceToDevice, s), "D2D b");
    ck(cudaMemsetAsync(M.x64.p, 0, pn * sizeof(double2), s), "memset x64");
    ck(cudaMemsetAsync(M.xcur.p, 0, pn * sizeof(float2), s), "memset x");
    const int nparts = 152;
    DevArr<double> part;
    part.alloc((size_t)nparts * nr);
    std::vector<double> hp((size_t)nparts * nr), bn(nr, 0.0), rn(nr, 0.0);
    // out[r] = ||b_r - y_r|| for y = A x (FP32 products); M.bvec receives b - y
    auto norms = [&](const float2 *y, std::vector<double> &out) {
        for (int r = 0; r < nr; ++r) {
            k_refine_residual<<<nparts, 256, 0, s>>>(M.bsave.p + r * n, y + r * n, M.bvec.p + r * n, n,
                                                     part.p + (int64_t)r * nparts);
            ck_launch("k_refine_residual");
        }
        ck(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H norms");
        ck(cudaStreamSynchronize(s), "sync");
        for (int r = 0; r < nr; ++r) {
            double v = 0.0;
            for (int q = 0; q < nparts; ++q) v += hp[(size_t)r * nparts + q];
            out[r] = std::sqrt(v);
        }
    };
    norms(M.xcur.p, bn);        // x = 0: the residual is b
    GmresResult R;
    R.hp.assign(nr, GmresState());
    R.iters.assign(nr, 0);
    R.conv.assign(nr, 0);
    int total = 0;
    rn = bn;
    for (int outer = 0; outer < 30; ++outer) {
        if (outer > 0) {
            // r = b - A x with the FP32 products, differenced in FP64
            M.force_fp32 = true;
            try {
                matvec_internal(M, fr(M).cp.p, fr(M).cq.p, true, M.xcur.p, nullptr, false, M.rtmp.p, false, nullptr,
                                s, false, false, nr);
            } catch (...) {
                M.force_fp32 = false;
                throw;
            }
            M.force_fp32 = false;
            total += 1;
            norms(M.rtmp.p, rn);
        }
        bool all = true;
        double worst = 0.0;
        for (int r = 0; r < nr; ++r) {
            const double rel = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
            R.hp[r].resid = rel;
            R.conv[r] = rel <= tol;
            all = all && R.conv[r];
            worst = std::max(worst, rel);
        }
        if (all || total >= max_iter) break;
        // inner solve of A d = r with the mixed-precision products, aimed at
        // the target (with a margin of two): the split-BF16 products carry
        // errors near the FP32 products' own, so one inner solve usually
        // suffices and the FP32 residual only confirms it
        precondition_rhs(M, M.bvec.p, nr);
        const double inner = std::min(0.5, 0.5 * tol / std::max(worst, 1e-300));
        GmresResult G = run_gmres(M, inner, std::max(1, max_iter - total), false, nr);
        int most = 0;
        for (int r = 0; r < nr; ++r) most = std::max(most, G.iters[r]);
        total += most;
        R.restarts += G.restarts + 1;
        for (int r = 0; r < nr; ++r) {
            k_refine_update<<<nblocks(n, 256), 256, 0, s>>>(M.x64.p + r * n, M.uvec.p + r * n, M.xcur.p + r * n, n);
            ck_launch("k_refine_update");
        }
    }
    ck(cudaMemcpyAsync(M.uvec.p, M.xcur.p, pn * sizeof(float2), cudaMemcpyDeviceToDevice, s), "D2D x");
    for (int r = 0; r < nr; ++r) {
        R.iters[r] = total;
        R.hp[r].iters = total;
        R.hp[r].converged = R.conv[r];
    }
    R.h = R.hp[0];
    R.total_iters = total;
    R.converged = R.conv[0];
    return R;
}

// Solve with the current frame's plan (prepared for freq_hz): right-hand
// side, GMRES, p and q in the caller's order.  nr = 1: one right-hand side,
// the incident field of all n_src sources; nr > 1 (= n_src): one system per
// source, solved together (planes of p_dev, q_dev and info).  Throws Fail.
int solve_frame(bem_mesh_impl &M, double freq_hz, const bem_medium *medium, const bem_source *srcs, int32_t n_src,
                double tol, int32_t max_iter, void *p_dev, void *q_dev, bem_solve_info *info, cudaStream_t us,
                std::chrono::steady_clock::time_point t0, std::chrono::steady_clock::time_point t_setup, int nr = 1)
{
    {
        Plan &P = *fr(M).plan;
        cudaStream_t s = M.s;
        const int64_t n = M.n;
        // right-hand side: incident field minus the known boundary data
        std::vector<SourceDev> sv = sources_of(srcs, n_src);
        DevArr<SourceDev> &sdev = M.srcbuf;
        sdev.upload(sv, s);
        M.bvec.alloc((size_t)nr * n);
        M.uvec.alloc((size_t)nr * n);
        if (nr > 1) {
            // one source per right-hand side
            for (int r = 0; r < nr; ++r) {
                {
                    KTimer kt_("k_rhs", s);
                    k_rhs<<<nblocks(n, 256), 256, 0, s>>>(M.cd.p, M.nrm.p, n, P.k, sdev.p + r, 1, M.bvec.p + r * n);
                }
                ck_launch("k_rhs");
            }
        } else if (n_src > 0) {
            {
                KTimer kt_("k_rhs", s);
                k_rhs<<<nblocks(n, 256), 256, 0, s>>>(M.cd.p, M.nrm.p, n, P.k, sdev.p, n_src, M.bvec.p);
            }
            ck_launch("k_rhs");
        } else {
            ck(cudaMemsetAsync(M.bvec.p, 0, n * sizeof(float2), s), "memset");
        }
        if (fr(M).known_nonzero) {
            reset_err(M);
            matvec_internal(M, fr(M).cp0.p, fr(M).cq0.p, false, fr(M).z.p, nullptr, false, M.tmp2.p, false, nullptr, s);
            check_err(M);
            for (int r = 0; r < nr; ++r) {
                {
                    KTimer kt_("k_sub", s);
                    k_sub<<<nblocks(n, 256), 256, 0, s>>>(M.bvec.p + r * n, M.tmp2.p, n);
                }
                ck_launch("k_sub");
            }
        }
        // row scaling (Sec. 3.2): GMRES on D^-1 A u = D^-1 b, D = diag(A)
        const bool rscale = M.prm.row_scaling != 0;
        if (rscale) {
            M.dinv.alloc(n);
            NearArgs na = near_args(M, P, fr(M).cp.p, fr(M).cq.p);
            {
                KTimer kt_("k_row_scale_init", s);
                k_row_scale_init<<<nblocks(n, 128), 128, 0, s>>>(na, M.dinv.p, fr(M).err.p);
            }
            ck_launch("k_row_scale_init");
        }
        // block-Jacobi (the block form of the row scaling of Sec. 3.2):
        // GMRES on P A u = P b, P the inverse of A's block diagonal
        if (M.prm.block_jacobi) {
            const Lists &Lb = *P.lists;
            M.bjinv.alloc((size_t)std::max<int64_t>(1, Lb.bj_entries));
            reset_err(M);
            NearArgs na = near_args(M, P, fr(M).cp.p, fr(M).cq.p);
            {
                KTimer kt_("k_bj_factor", s);
                k_bj_factor<<<(unsigned)Lb.h_bj.size(), 256, 0, s>>>(na, Lb.bj.p, M.bjinv.p, fr(M).err.p);
            }
            ck_launch("k_bj_factor");
            check_err(M);
        }
        // the preconditioned right-hand side (the refinement of a
        // mixed-precision solve preconditions each inner residual instead)
        if (M.prm.far_precision != 1) precondition_rhs(M, M.bvec.p, nr);
        ck(cudaStreamSynchronize(s), "sync");
        auto t_rhs = std::chrono::steady_clock::now();
        GmresResult R;
        {
            NvtxRange nvtx_(M.prm.far_precision == 1 ? "refined GMRES" : "GMRES");
            R = M.prm.far_precision == 1 ? run_refined(M, tol, max_iter, nr) : run_gmres(M, tol, max_iter, false, nr);
        }
        check_tc_fault(M);
        auto t_gmres = std::chrono::steady_clock::now();
        // p and q in the caller's order
        for (int r = 0; r < nr; ++r) {
            {
                KTimer kt_("k_pq", s);
                k_pq<<<nblocks(n, 256), 256, 0, s>>>(M.uvec.p + r * n, fr(M).z.p, fr(M).aq.p, M.type.p, M.perm.p, n,
                                                     (float2 *)p_dev + r * n, q_dev ? (float2 *)q_dev + r * n : nullptr);
            }
            ck_launch("k_pq");
        }
        check_err(M);
        join_streams(s, us);
        ck(cudaStreamSynchronize(us), "sync");
        resolve_timing();
        bool all_conv = true;
        for (int r = 0; r < nr; ++r) all_conv = all_conv && R.conv[r];
        int status = all_conv ? BEM_OK : BEM_W_NOT_CONVERGED;
        if (!all_conv) {
            char buf[200];
            for (int r = 0; r < nr; ++r)
                if (!R.conv[r]) {
                    snprintf(buf, sizeof buf, "GMRES: relative residual %.3g after %d products (tol %.3g)%s",
                             R.hp[r].resid, R.iters[r], tol, nr > 1 ? " for a right-hand side" : "");
                    break;
                }
            g_err = buf;
        } else if (resolution_warning(M, freq_hz, medium) != BEM_OK) {
            status = BEM_W_UNDERRESOLVED;
        }
        for (int r = 0; info && r < nr; ++r) {
            bem_solve_info *ir = info + r;
            memset(ir, 0, sizeof *ir);
            ir->iterations = R.iters[r];
            ir->restarts = R.restarts;
            ir->relres = R.hp[r].resid;
            ir->levels = (int)P.lev.size();
            for (size_t l = 0; l < P.lev.size() && l < 16; ++l) ir->L[l] = P.lev[l]->L;
            ir->near_nnz = P.nnz();
            ir->status = R.conv[r] ? (status == BEM_W_NOT_CONVERGED ? BEM_OK : status) : BEM_W_NOT_CONVERGED;
            ir->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            ir->setup_seconds = std::chrono::duration<double>(t_setup - t0).count();
            ir->rhs_seconds = std::chrono::duration<double>(t_rhs - t_setup).count();
            ir->gmres_seconds = std::chrono::duration<double>(t_gmres - t_rhs).count();
        }
        return status;
    }
}

// Ends a stream capture that a failure left open.
void abandon_capture(bem_mesh_impl &M)
{
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(M.s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g;
        cudaStreamEndCapture(M.s, &g);
        if (g) cudaGraphDestroy(g);
    }
}

// Exchanges the frequency state of two frames (not their streams).
void swap_frames(Frame &a, Frame &b)
{
    std::swap(a.plan, b.plan);
    a.cp.swap(b.cp);
    a.cq.swap(b.cq);
    a.cp0.swap(b.cp0);
    a.cq0.swap(b.cq0);
    a.z.swap(b.z);
    a.aq.swap(b.aq);
    a.err.swap(b.err);
    a.vtmp.swap(b.vtmp);
    a.vout.swap(b.vout);
    std::swap(a.known_nonzero, b.known_nonzero);
}

}  // namespace

int bem_solve(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
              int32_t n_regions, const bem_source *srcs, int32_t n_src, double tol, int32_t max_iter,
              void *p_dev, void *q_dev, bem_solve_info *info, void *stream)
{
    NvtxRange nvtx_("bem_solve");
    auto t0 = std::chrono::steady_clock::now();
    if (!mesh || !p_dev || n_src < 0 || (n_src > 0 && !srcs) || !(tol > 0) || max_iter < 1)
        return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        cudaStream_t us = (cudaStream_t)stream;
        Coeffs C;
        join_streams(us, M.s);
        prepare(M, freq_hz, medium, admittance, n_regions, C);
        ck(cudaStreamSynchronize(M.s), "sync");
        return solve_frame(M, freq_hz, medium, srcs, n_src, tol, max_iter, p_dev, q_dev, info, us, t0,
                           std::chrono::steady_clock::now());
    } catch (Fail &f) {
        abandon_capture(M);
        return f.code;
    }
}

int bem_solve_multi(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                    int32_t n_regions, const bem_source *srcs, int32_t n_rhs, double tol, int32_t max_iter,
                    void *p_dev, void *q_dev, bem_solve_info *infos, void *stream)
{
    NvtxRange nvtx_("bem_solve_multi");
    auto t0 = std::chrono::steady_clock::now();
    if (!mesh || !p_dev || n_rhs < 1 || n_rhs > kMaxPlanes || !srcs || !(tol > 0) || max_iter < 1)
        return set_err(BEM_E_ARG, "bad argument (n_rhs must be in 1..4)");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        cudaStream_t us = (cudaStream_t)stream;
        Coeffs C;
        join_streams(us, M.s);
        prepare(M, freq_hz, medium, admittance, n_regions, C);
        ck(cudaStreamSynchronize(M.s), "sync");
        return solve_frame(M, freq_hz, medium, srcs, n_rhs, tol, max_iter, p_dev, q_dev, infos, us, t0,
                           std::chrono::steady_clock::now(), n_rhs);
    } catch (Fail &f) {
        abandon_capture(M);
        return f.code;
    }
}

int bem_solve_sweep(void *mesh, const double *freqs_hz, int32_t n_freq, const bem_medium *medium,
                    const double *admittance, int32_t n_regions, const bem_source *srcs, int32_t n_src, double tol,
                    int32_t max_iter, void *p_dev, void *q_dev, const double *pts, int64_t n_pts, void *field_dev,
                    bem_solve_info *infos, void *stream)
{
    NvtxRange nvtx_("bem_solve_sweep");
    if (!mesh || !freqs_hz || n_freq < 1 || !p_dev || n_src < 0 || (n_src > 0 && !srcs) || !(tol > 0) ||
        max_iter < 1 || n_pts < 0 || (n_pts > 0 && (!pts || !field_dev || !q_dev)))
        return set_err(BEM_E_ARG, "bad argument");
    for (int32_t i = 0; i < n_freq; ++i)
        if (!(freqs_hz[i] > 0) || !std::isfinite(freqs_hz[i])) return set_err(BEM_E_ARG, "frequency must be positive");
    auto &M = *(bem_mesh_impl *)mesh;
    const int64_t n = M.n;
    int worst = BEM_OK;
    std::string worst_msg;
    try {
        cudaStream_t us = (cudaStream_t)stream;
        join_streams(us, M.s);
        auto t0 = std::chrono::steady_clock::now();
        {
            Coeffs C;
            prepare(M, freqs_hz[0], medium, admittance, n_regions, C);
            ck(cudaStreamSynchronize(M.s), "sync");
        }
        for (int32_t i = 0; i < n_freq; ++i) {
            auto t_setup = std::chrono::steady_clock::now();
            // the next frequency's plan and near-field entries, on the setup
            // thread and stream, while this frequency's GMRES runs
            std::thread ahead;
            int next_code = BEM_OK;
            std::string next_msg;
            if (i + 1 < n_freq) {
                const double fn = freqs_hz[i + 1];
                ahead = std::thread([&M, &next_code, &next_msg, fn, medium, admittance, n_regions]() {
                    t_frame = &M.next;
                    try {
                        ck(cudaSetDevice(M.device), "cudaSetDevice");
                        Coeffs Cn;
                        prepare(M, fn, medium, admittance, n_regions, Cn);
                        ck(cudaStreamSynchronize(M.s_setup), "sync");
                    } catch (Fail &f) {
                        next_code = f.code;
                        next_msg = g_err;
                    } catch (std::exception &e) {
                        next_code = BEM_E_INTERNAL;
                        next_msg = e.what();
                    }
                    t_frame = nullptr;
                });
            }
            int st = BEM_OK;
            try {
                bem_solve_info *info = infos ? infos + i : nullptr;
                float2 *p = (float2 *)p_dev + (int64_t)i * n;
                float2 *q = q_dev ? (float2 *)q_dev + (int64_t)i * n : nullptr;
                st = solve_frame(M, freqs_hz[i], medium, srcs, n_src, tol, max_iter, p, q, info, us, t0, t_setup);
                if (n_pts > 0) {
                    const int se = bem_evaluate(mesh, freqs_hz[i], medium, srcs, n_src, p, q, pts, n_pts,
                                                (float2 *)field_dev + (int64_t)i * n_pts, stream);
                    if (se < 0) throw Fail{se};
                }
                ck(cudaStreamSynchronize(us), "sync");
            } catch (Fail &f) {
                abandon_capture(M);
                const std::string msg = g_err;
                if (ahead.joinable()) ahead.join();
                g_err = msg;
                return f.code;
            }
            if (st > 0 && worst == BEM_OK) {
                worst = st;
                worst_msg = g_err;
            }
            t0 = std::chrono::steady_clock::now();
            if (ahead.joinable()) {
                ahead.join();
                if (next_code != BEM_OK) {
                    g_err = next_msg;
                    return next_code;
                }
                swap_frames(M.cur, M.next);
                t_frame = &M.next;      // the finished frequency's buffers become spares
                recycle_plan(M);
                t_frame = nullptr;
            }
        }
        if (worst != BEM_OK) g_err = worst_msg;
        return worst;
    } catch (Fail &f) {
        abandon_capture(M);
        return f.code;
    }
}

// The field at points through the plane-wave expansions (build_eval_plan):
// near pairs by the element rules of k_field over the point leaves' near
// lists; far pairs by an aggregation of the weights (-A q, -ik A p) at every
// level the plan uses, translation tables for the point-cluster offsets, the
// transfer onto the point clusters and the disaggregation onto the points
// (no normal factor).  p, q: internal element order; out: caller point order.
void field_fmm_plan(bem_mesh_impl &M, double k, const double *pts, int64_t np, cudaStream_t s)
{
    if (!M.eval) M.eval = std::make_unique<EvalDev>();
    EvalDev &V = *M.eval;
    if (V.valid && V.np == np && V.key_k == k && V.key_depth == M.leaf_depth && V.key_trunc == M.prm.trunc_factor &&
        std::equal(pts, pts + 3 * np, V.key_pts.begin()))
        return;
    V.valid = false;
    EvalPlan ep;
    const std::string msg = build_eval_plan(M.g, M.t, M.prm, k, M.leaf_depth, pts, np, kMaxTableL, ep);
    if (!msg.empty()) throw Fail{set_err(BEM_E_ARG, msg)};
    if ((int)ep.far.size() > kMaxFarLevels)
        throw Fail{set_err(BEM_E_ARG, "field evaluation: more far levels than the kernels take")};
    // the points in internal order, their leaf clusters and near element runs
    std::vector<double> hp(3 * (size_t)np);
    for (int64_t i = 0; i < np; ++i)
        for (int a = 0; a < 3; ++a) hp[3 * i + a] = pts[3 * ep.perm[i] + a];
    V.pts.upload(hp, s);
    V.perm.upload(ep.perm, s);
    const int npl = (int)ep.leaf_start.size() - 1;
    std::vector<int> pleaf((size_t)np);
    for (int c = 0; c < npl; ++c)
        for (int64_t i = ep.leaf_start[c]; i < ep.leaf_start[c + 1]; ++i) pleaf[i] = c;
    V.pleaf.upload(pleaf, s);
    const Level &EL = M.t.lv[ep.leaf_depth];
    std::vector<int> nptr(npl + 1, 0);
    std::vector<int2> nruns;
    for (int c = 0; c < npl; ++c) {
        int prev = -2;
        for (int q2 = ep.near_ptr[c]; q2 < ep.near_ptr[c + 1]; ++q2) {
            const int sl = ep.near_src[q2];
            if (EL.count[sl] == 0) continue;
            if (sl == prev + 1) nruns.back().y += (int)EL.count[sl];   // consecutive leaves: one run
            else nruns.push_back(make_int2((int)EL.start[sl], (int)EL.count[sl]));
            prev = sl;
        }
        nptr[c + 1] = (int)nruns.size();
    }
    V.nptr.upload(nptr, s);
    V.nruns.upload(nruns, s);
    V.vnear.alloc(np);
    V.vall.alloc(np);
    V.np = np;
    V.npl = npl;
    V.far = !ep.far.empty();
    V.n_dtasks = 0;
    if (V.far) {
        while (V.lev.size() < ep.far.size()) V.lev.push_back(std::make_unique<EvalLevelDev>());
        std::vector<AggTask> tasks;
        std::vector<int2> reds;
        std::vector<int4> tg;
        DTableArgs ta;
        memset(&ta, 0, sizeof ta);
        ta.k = k;
        int nb = 0;
        LevelsArgs &A = V.A;
        memset(&A, 0, sizeof A);
        DisaggArgs &da = V.da;
        memset(&da, 0, sizeof da);
        for (size_t l = 0; l < ep.far.size(); ++l) {
            const EvalLevel &F = ep.far[l];
            EvalLevelDev &Ld = *V.lev[l];
            const Level &E = M.t.lv[F.depth];
            Ld.L = F.L;
            Ld.nd = 2 * F.L * F.L;
            Ld.noff = (int)(F.offsets.size() / 3);
            Ld.npc = F.npc;
            Ld.nc = (int)E.start.size();
            const int nd = Ld.nd;
            std::vector<double> sd, sw;
            sphere_grid(F.L, sd, sw);
            std::vector<float4> dirs(nd);
            for (int q2 = 0; q2 < nd; ++q2)
                dirs[q2] = make_float4((float)sd[3 * q2], (float)sd[3 * q2 + 1], (float)sd[3 * q2 + 2], (float)sw[q2]);
            Ld.dirs.upload(dirs, s);
            Ld.dirs_d.upload(sd, s);
            Ld.il_ptr.upload(F.il_ptr, s);
            Ld.il_src.upload(F.il_src, s);
            Ld.il_off.upload(F.il_off, s);
            Ld.offs.upload(F.offsets, s);
            Ld.pcl.upload(F.pcl, s);
            std::vector<float4> dzp((size_t)np);
            for (int64_t i = 0; i < np; ++i) {
                const int c = F.pcl[i];
                dzp[i] = make_float4((float)(F.zp[3 * c] - hp[3 * i]), (float)(F.zp[3 * c + 1] - hp[3 * i + 1]),
                                     (float)(F.zp[3 * c + 2] - hp[3 * i + 2]), 0.f);
            }
            Ld.dzp.upload(dzp, s);
            // aggregation tasks over this level's source clusters: element
            // chunks of at most kAggChunk (split clusters summed by the last
            // block) times ranges of kAggThreads direction pairs
            std::vector<char> is_src(Ld.nc, 0);
            for (int v : F.il_src) is_src[v] = 1;
            std::vector<int> red_ptr{Ld.nc}, red_c;
            int extra = 0;
            for (int c = 0; c < Ld.nc; ++c) {
                if (!is_src[c]) continue;
                const int64_t cnt = E.count[c];
                const int64_t nch = std::max<int64_t>(1, (cnt + kAggChunk - 1) / kAggChunk);
                if (nch == 1) {
                    for (int p0 = 0; p0 < nd / 2; p0 += kAggThreads)
                        tasks.push_back(AggTask{c, c, E.start[c], (int)cnt, (int)l, -1, -1, p0});
                    continue;
                }
                const int red = (int)red_c.size();
                const int gred = (int)reds.size() + red;
                for (int64_t q2 = 0; q2 < nch; ++q2) {
                    const int64_t a = cnt * q2 / nch, b = cnt * (q2 + 1) / nch;
                    for (int p0 = 0; p0 < nd / 2; p0 += kAggThreads)
                        tasks.push_back(AggTask{c, Ld.nc + extra, E.start[c] + a, (int)(b - a), (int)l, red, gred, p0});
                    ++extra;
                }
                red_c.push_back(c);
                red_ptr.push_back(Ld.nc + extra);
            }
            for (size_t q2 = 0; q2 < red_c.size(); ++q2) reds.push_back(make_int2((int)l, (int)q2));
            Ld.nextra = extra;
            Ld.red_ptr.upload(red_ptr, s);
            Ld.red_c.upload(red_c, s);
            Ld.Mx.alloc((size_t)(Ld.nc + extra) * nd);
            Ld.Lam.alloc((size_t)Ld.npc * nd);
            Ld.D.alloc((size_t)Ld.noff * nd);
            if (Ld.noff > 0) {
                ta.start[ta.nlev] = nb;
                ta.lev[ta.nlev] = DTableLevel{Ld.offs.p, Ld.dirs_d.p, Ld.D.p, nd, F.L};
                nb += Ld.noff;
                ++ta.nlev;
            }
            for (int c = 0; c < F.npc; ++c)
                if (F.il_ptr[c + 1] > F.il_ptr[c])
                    for (int nu0 = 0; nu0 < nd; nu0 += kTransferDirs) tg.push_back(make_int4((int)l, c, nu0, 0));
            const DepthDev *dd = depth_data(M, F.depth);
            FarArgs f;
            memset(&f, 0, sizeof f);
            f.nd = nd;
            f.k = (float)k;
            f.red_ptr = Ld.red_ptr.p;
            f.red_c = Ld.red_c.p;
            f.nred = (int)red_c.size();
            f.dirs = Ld.dirs.p;
            f.il_ptr = Ld.il_ptr.p;
            f.il_src = Ld.il_src.p;
            f.il_off = Ld.il_off.p;
            f.D = Ld.D.p;
            f.M = Ld.Mx.p;
            f.Lam = Ld.Lam.p;
            f.cstart = dd->cstart.p;
            f.dz = dd->dz.p;
            f.elem_cl = dd->elem_cl.p;
            f.mplane = (int64_t)(Ld.nc + extra) * nd;
            f.lplane = (int64_t)Ld.npc * nd;
            A.lev[l] = f;
            // the disaggregation sees the points: their clusters and z_P - x_m
            f.dz = Ld.dzp.p;
            f.elem_cl = Ld.pcl.p;
            da.lev[l] = f;
        }
        ta.start[ta.nlev] = nb;
        A.nlev = (int)ep.far.size();
        V.tasks.upload(tasks, s);
        A.tasks = V.tasks.p;
        A.ntasks = (int)tasks.size();
        V.reds.upload(reds, s);
        A.reds = V.reds.p;
        A.nreds = (int)reds.size();
        V.red_cnt.alloc(std::max<size_t>(1, reds.size()));
        ck(cudaMemsetAsync(V.red_cnt.p, 0, std::max<size_t>(1, reds.size()) * sizeof(unsigned int), s), "memset");
        A.red_cnt = V.red_cnt.p;
        V.tgroups.upload(tg, s);
        A.tgroups = V.tgroups.p;
        A.ntgroups = (int)tg.size();
        std::vector<LevelsArgs> hv(1, A);
        V.largs.upload(hv, s);
        if (nb > 0) {
            {
                KTimer kt_("k_dtable", s);
                k_dtable<<<nb, 128, 0, s>>>(ta);
            }
            ck_launch("k_dtable");
        }
        // disaggregation onto the points: tasks of at most kDisTask points of
        // one point leaf (zero normals: no row factor)
        std::vector<int2> dt;
        for (int c = 0; c < npl; ++c) {
            const int64_t a = ep.leaf_start[c], cnt = ep.leaf_start[c + 1] - a;
            const int64_t nch = (cnt + kDisTask - 1) / kDisTask;
            for (int64_t q2 = 0; q2 < nch; ++q2)
                dt.push_back(make_int2((int)(a + cnt * q2 / nch), (int)(a + cnt * (q2 + 1) / nch)));
        }
        V.dtasks.upload(dt, s);
        V.n_dtasks = (int)dt.size();
        V.zeros.alloc(np);
        ck(cudaMemsetAsync(V.zeros.p, 0, np * sizeof(float4), s), "memset");
        da.n = np;
        da.nrm = V.zeros.p;
        da.perm = nullptr;
        da.k = (float)k;
        da.nlev = A.nlev;
        da.tasks = V.dtasks.p;
        da.rowf = nullptr;
    }
    ck(cudaStreamSynchronize(s), "sync");   // the host vectors above are uploaded before they go
    V.key_pts.assign(pts, pts + 3 * np);
    V.key_k = k;
    V.key_depth = M.leaf_depth;
    V.key_trunc = M.prm.trunc_factor;
    V.valid = true;
}

// The field at points through the plane-wave expansions (build_eval_plan):
// near pairs by the element rules of k_field over the point leaves' near
// lists; far pairs by an aggregation of the weights (-A q, -ik A p) at every
// level the plan uses, translation tables for the point-cluster offsets, the
// transfer onto the point clusters and the disaggregation onto the points
// (no normal factor).  p, q: internal element order; out: caller point order.
void field_fmm(bem_mesh_impl &M, double k, const double *pts, int64_t np, const float2 *p, const float2 *q,
               const SourceDev *src, int nsrc, float2 *out, cudaStream_t s)
{
    field_fmm_plan(M, k, pts, np, s);
    EvalDev &V = *M.eval;
    const int64_t n = M.n;
    {
        KTimer kt_("k_field_near", s);
        k_field_near<<<nblocks(np, 8), 256, 0, s>>>(M.elem(), M.Q.p, V.pts.p, np, (float)k, p, q, V.pleaf.p,
                                                   V.nptr.p, V.nruns.p, V.vnear.p, fr(M).err.p);
    }
    ck_launch("k_field_near");
    const float2 *vres = V.vnear.p;
    if (V.far) {
        V.wts.alloc(n);
        {
            KTimer kt_("k_field_weights", s);
            k_field_weights<<<nblocks(n, 256), 256, 0, s>>>(n, p, q, M.chi.p, (float)k, V.wts.p);
        }
        ck_launch("k_field_weights");
        if (V.A.ntasks > 0) {
            {
                KTimer kt_("k_aggregate", s);
                k_aggregate_1<<<V.A.ntasks, kAggThreads, 0, s>>>(V.largs.p, V.wts.p, n, M.nrm.p, nullptr);
            }
            ck_launch("k_aggregate");
        }
        if (V.A.ntgroups > 0) {
            {
                KTimer kt_("k_transfer", s);
                k_transfer_split<<<V.A.ntgroups, 32 * kTransferWarps, 0, s>>>(V.largs.p, nullptr);
            }
            ck_launch("k_transfer");
        }
        if (V.n_dtasks > 0) {
            {
                KTimer kt_("k_disaggregate", s);
                k_disaggregate_m1<<<(unsigned)V.n_dtasks, kDisThreads, 0, s>>>(V.da, V.vnear.p, V.vall.p, nullptr);
            }
            ck_launch("k_disaggregate");
        }
        vres = V.vall.p;
    }
    {
        KTimer kt_("k_field_eval_finish", s);
        k_field_eval_finish<<<nblocks(np, 128), 128, 0, s>>>(V.pts.p, np, (float)k, (float)M.prm.tau, src, nsrc, vres,
                                                             V.perm.p, out);
    }
    ck_launch("k_field_eval_finish");
}

int bem_evaluate(void *mesh, double freq_hz, const bem_medium *medium, const bem_source *srcs, int32_t n_src,
                 const void *p_dev, const void *q_dev, const double *pts, int64_t M_pts, void *out_dev,
                 void *stream)
{
    NvtxRange nvtx_("bem_evaluate");
    if (!mesh || !p_dev || !q_dev || M_pts < 0 || n_src < 0 || (n_src > 0 && !srcs))
        return set_err(BEM_E_ARG, "bad argument");
    if (M_pts == 0) return BEM_OK;   // nothing to evaluate (pts and out_dev may be NULL)
    if (!pts || !out_dev) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        double c, rho;
        medium_of(medium, c, rho);
        if (!(freq_hz > 0)) return set_err(BEM_E_ARG, "frequency must be positive");
        ck(cudaSetDevice(M.device), "cudaSetDevice");
        ensure_work(M);
        cudaStream_t us = (cudaStream_t)stream;
        join_streams(us, M.s);
        cudaStream_t s = M.s;
        const int64_t n = M.n;
        {
            KTimer kt_("k_gather", s);
            k_gather<<<nblocks(n, 256), 256, 0, s>>>((const float2 *)p_dev, M.perm.p, n, M.tmp.p);
        }
        ck_launch("k_gather");
        {
            KTimer kt_("k_gather", s);
            k_gather<<<nblocks(n, 256), 256, 0, s>>>((const float2 *)q_dev, M.perm.p, n, M.tmp2.p);
        }
        ck_launch("k_gather");
        std::vector<double> hp(pts, pts + 3 * M_pts);
        DevArr<double> &dp = M.ptsbuf;
        dp.upload(hp, s);
        std::vector<SourceDev> sv = sources_of(srcs, n_src);
        DevArr<SourceDev> &sdev = M.srcbuf;
        sdev.upload(sv, s);
        reset_err(M);
        const double k = wavenumber(freq_hz, c);
        if (M.prm.mode == BEM_MODE_FMM &&
            (M.prm.field_mode == 2 || (M.prm.field_mode == 0 && (double)M_pts * (double)n >= kFieldFmmMinPairs))) {
            field_fmm(M, k, pts, M_pts, M.tmp.p, M.tmp2.p, sdev.p, n_src, (float2 *)out_dev, s);
            check_err(M);
            join_streams(s, us);
            resolve_timing();
            return BEM_OK;
        }
        // each point's element sum split over S blocks when the points alone
        // would leave SMs idle (partials added in slice order)
        int nsm = 0;
        ck(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, M.device), "attribute");
        const int64_t want = 8 * (int64_t)nsm;
        const int S = (int)std::max<int64_t>(1, std::min<int64_t>({16, (want + M_pts - 1) / M_pts,
                                                                   (n + 255) / 256}));
        if (S > 1) M.fieldpart.alloc((size_t)M_pts * S);
        {
            KTimer kt_("k_field", s);
            k_field<<<dim3((unsigned)M_pts, (unsigned)S), 256, 0, s>>>(M.elem(), M.Q.p, dp.p, M_pts, (float)k,
                                                                      (float)M.prm.tau, M.tmp.p, M.tmp2.p,
                                                                      sdev.p, n_src,
                                                                      M.fieldpart.p, (float2 *)out_dev,
                                                                      fr(M).err.p);
        }
        ck_launch("k_field");
        if (S > 1) {
            {
                KTimer kt_("k_field", s);
                k_field_finish<<<nblocks(M_pts, 128), 128, 0, s>>>(dp.p, M_pts, S, (float)k, sdev.p, n_src,
                                                                  M.fieldpart.p, (float2 *)out_dev);
            }
            ck_launch("k_field_finish");
        }
        check_err(M);
        join_streams(s, us);
        resolve_timing();
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_evaluate_velocity(void *mesh, double freq_hz, const bem_medium *medium, const bem_source *srcs,
                          int32_t n_src, const void *p_dev, const void *q_dev, const double *pts, int64_t M_pts,
                          void *v_out_dev, void *stream)
{
    NvtxRange nvtx_("bem_evaluate_velocity");
    if (!mesh || !p_dev || !q_dev || M_pts < 0 || n_src < 0 || (n_src > 0 && !srcs))
        return set_err(BEM_E_ARG, "bad argument");
    if (M_pts == 0) return BEM_OK;   // nothing to evaluate (pts and v_out_dev may be NULL)
    if (!pts || !v_out_dev) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        double c, rho;
        medium_of(medium, c, rho);
        if (!(freq_hz > 0)) return set_err(BEM_E_ARG, "frequency must be positive");
        ck(cudaSetDevice(M.device), "cudaSetDevice");
        ensure_work(M);
        cudaStream_t us = (cudaStream_t)stream;
        join_streams(us, M.s);
        cudaStream_t s = M.s;
        const int64_t n = M.n;
        {
            KTimer kt_("k_gather", s);
            k_gather<<<nblocks(n, 256), 256, 0, s>>>((const float2 *)p_dev, M.perm.p, n, M.tmp.p);
        }
        ck_launch("k_gather");
        {
            KTimer kt_("k_gather", s);
            k_gather<<<nblocks(n, 256), 256, 0, s>>>((const float2 *)q_dev, M.perm.p, n, M.tmp2.p);
        }
        ck_launch("k_gather");
        std::vector<double> hp(pts, pts + 3 * M_pts);
        DevArr<double> &dp = M.ptsbuf;
        dp.upload(hp, s);
        std::vector<SourceDev> sv = sources_of(srcs, n_src);
        DevArr<SourceDev> &sdev = M.srcbuf;
        sdev.upload(sv, s);
        reset_err(M);
        const double k = wavenumber(freq_hz, c);
        const float inv_omega_rho = (float)(1.0 / (2.0 * 3.14159265358979323846 * freq_hz * rho));
        // blocks per point as for the field (partials added in slice order)
        int nsm = 0;
        ck(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, M.device), "attribute");
        const int64_t want = 8 * (int64_t)nsm;
        const int S = (int)std::max<int64_t>(1, std::min<int64_t>({16, (want + M_pts - 1) / M_pts,
                                                                   (n + 255) / 256}));
        if (S > 1) M.fieldpart.alloc((size_t)M_pts * S * 3);
        {
            KTimer kt_("k_field_velocity", s);
            k_field_velocity<<<dim3((unsigned)M_pts, (unsigned)S), 256, 0, s>>>(
                M.elem(), M.Q.p, dp.p, M_pts, (float)k, (float)M.prm.tau, inv_omega_rho, M.tmp.p, M.tmp2.p,
                sdev.p, n_src,
                M.fieldpart.p, (float2 *)v_out_dev, fr(M).err.p);
        }
        ck_launch("k_field_velocity");
        if (S > 1) {
            {
                KTimer kt_("k_field_velocity", s);
                k_field_velocity_finish<<<nblocks(M_pts, 128), 128, 0, s>>>(
                    dp.p, M_pts, S, (float)k, inv_omega_rho, sdev.p, n_src, M.fieldpart.p, (float2 *)v_out_dev);
            }
            ck_launch("k_field_velocity_finish");
        }
        check_err(M);
        join_streams(s, us);
        resolve_timing();
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_admittance_gradient(void *mesh, double freq_hz, const bem_medium *medium, const double *admittance,
                            int32_t n_regions, const bem_source *srcs, int32_t n_src, const double *pts,
                            int64_t n_pts, double tol, int32_t max_iter, void *p_dev, void *q_dev, double *loss,
                            double *grad, bem_solve_info *info, void *stream)
{
    NvtxRange nvtx_("bem_admittance_gradient");
    if (!mesh || !admittance || n_regions < 1 || n_src < 0 || (n_src > 0 && !srcs) || !pts || n_pts < 1 ||
        !(tol > 0) || max_iter < 1 || !p_dev || !q_dev || !loss || !grad)
        return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    // forward problem: u, p, q (Eq. SystemI) and the field at the points
    const int fwd = bem_solve(mesh, freq_hz, medium, admittance, n_regions, srcs, n_src, tol, max_iter, p_dev,
                              q_dev, info, stream);
    if (fwd < 0) return fwd;
    const std::string fwd_msg = g_err;
    try {
        double c, rho;
        medium_of(medium, c, rho);
        cudaStream_t us = (cudaStream_t)stream;
        cudaStream_t s = M.s;
        const int64_t n = M.n;
        const double k = wavenumber(freq_hz, c);
        const float tau = M.prm.tau < 0 ? -1.f : 1.f;
        M.uadj.alloc(n);
        M.fadj.alloc(n_pts);
        M.gadj.alloc(n);
        join_streams(us, s);
        ck(cudaMemcpyAsync(M.uadj.p, M.uvec.p, n * sizeof(float2), cudaMemcpyDeviceToDevice, s), "D2D u");
        join_streams(s, us);
        const int ev = bem_evaluate(mesh, freq_hz, medium, srcs, n_src, p_dev, q_dev, pts, n_pts, M.fadj.p, stream);
        if (ev < 0) return ev;
        join_streams(us, s);
        reset_err(M);
        // adjoint right-hand side F^T conj(f) into b, and G_f^T conj(f)
        std::vector<double> hp(pts, pts + 3 * n_pts);
        M.ptsbuf.upload(hp, s);
        M.bvec.alloc(n);
        {
            KTimer kt_("k_field_t", s);
            k_field_t<<<nblocks(n, 8), 256, 0, s>>>(M.elem(), M.Q.p, M.ptsbuf.p, n_pts, (float)k, M.fadj.p,
                                                     fr(M).cp.p, fr(M).cq.p, M.gadj.p, M.bvec.p, fr(M).err.p);
        }
        ck_launch("k_field_t");
        // adjoint solve A^T lambda = F^T conj(f) (lambda in uvec)
        ensure_transposed_values(M);
        GmresResult R = run_gmres(M, tol, max_iter, true);
        // aq = A_q^T lambda: the transposed product with c^p = 0 and c^q = 1
        // (tau folded in as for the unknowns' coefficients)
        std::vector<float2> h0((size_t)n, make_float2(0.f, 0.f)), hq((size_t)n, make_float2(tau, 0.f));
        M.adj_cp.upload(h0, s);
        M.adj_cq.upload(hq, s);
        matvec_t_internal(M, M.adj_cp.p, M.adj_cq.p, M.uvec.p, M.w.p, false, false, nullptr, s);
        // per-region sums and the loss
        std::vector<int> reg((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t e = M.t.perm[i];
            reg[i] = M.bct[e] == BEM_ADMI ? M.region[e] : -1;
        }
        M.adjreg.upload(reg, s);
        const int nacc = 2 * n_regions + 1;
        M.adjacc.alloc(nacc);
        ck(cudaMemsetAsync(M.adjacc.p, 0, nacc * sizeof(double), s), "memset acc");
        {
            KTimer kt_("k_adjoint_reduce", s);
            k_adjoint_reduce<<<nblocks(std::max<int64_t>(n, n_pts), 256), 256, 0, s>>>(
                M.uadj.p, M.gadj.p, M.w.p, M.adjreg.p, n, tau, 0.0, -(double)tau * k * rho * c, M.fadj.p, n_pts,
                n_regions, M.adjacc.p);
        }
        ck_launch("k_adjoint_reduce");
        std::vector<double> hacc(nacc);
        ck(cudaMemcpyAsync(hacc.data(), M.adjacc.p, nacc * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H acc");
        check_err(M);
        join_streams(s, us);
        ck(cudaStreamSynchronize(s), "sync");
        resolve_timing();
        *loss = hacc[2 * n_regions];
        for (int r = 0; r < 2 * n_regions; ++r) grad[r] = hacc[r];
        // the adjoint's non-convergence first: it makes the gradient itself
        // approximate; then the forward warning, if any
        if (!R.converged) {
            char buf[160];
            snprintf(buf, sizeof buf, "adjoint GMRES: relative residual %.3g after %d products (tol %.3g)",
                     R.h.resid, R.total_iters, tol);
            g_err = buf;
            return BEM_W_NOT_CONVERGED;
        }
        if (fwd != BEM_OK) g_err = fwd_msg;
        return fwd;
    } catch (Fail &f) {
        abandon_capture(M);
        return f.code;
    }
}

int bem_selftest_sincos(const void *x_dev, int64_t n, void *out_dev, void *stream)
{
    if (!x_dev || !out_dev || n < 0) return set_err(BEM_E_ARG, "bad argument");
    if (n == 0) return BEM_OK;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        {
            KTimer kt_("k_selftest_sincos", s);
            k_selftest_sincos<<<nblocks(n, 256), 256, 0, s>>>((const float *)x_dev, n, (float4 *)out_dev);
        }
        ck_launch("k_selftest_sincos");
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_mesh_release_plan(void *mesh)
{
    if (!mesh) return set_err(BEM_E_ARG, "mesh is NULL");
    auto &M = *(bem_mesh_impl *)mesh;
    cudaSetDevice(M.device);
    if (M.s) cudaStreamSynchronize(M.s);
    fr(M).plan.reset();
    M.freq_lists.clear();
    M.spare_val.release();
    M.spare_bufs.clear();
    return BEM_OK;
}

int bem_timing_enable(int enable)
{
    if (enable) {
        std::lock_guard<std::mutex> lk(g_tmu);
        g_tacc.clear();
    } else {
        resolve_timing();
    }
    g_timing = enable != 0;
    return BEM_OK;
}

int bem_timing_get(const char *name, double *total_ms, int64_t *launches)
{
    if (!name || !total_ms || !launches) return set_err(BEM_E_ARG, "bad argument");
    resolve_timing();
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_tacc.find(name);
    if (it == g_tacc.end()) { *total_ms = 0.0; *launches = 0; return set_err(BEM_E_ARG, "kernel never timed"); }
    *total_ms = it->second.first;
    *launches = it->second.second;
    return BEM_OK;
}

int bem_test_hooks(int64_t alloc_fail_after, int64_t *live_device_bytes)
{
    g_alloc_budget.store(alloc_fail_after < 0 ? -1 : alloc_fail_after);
    if (live_device_bytes) *live_device_bytes = g_live_bytes.load();
    return BEM_OK;
}

int bem_krylov_basis(void *mesh, int32_t plane, void *v_dev, int32_t max_cols, int32_t *n_cols)
{
    if (!mesh || !v_dev || max_cols < 0 || !n_cols) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        if (!M.st.p || !M.V.p || plane < 0 || (size_t)(plane + 1) > M.st.n)
            return set_err(BEM_E_ARG, "no GMRES state for this right-hand side");
        ck(cudaSetDevice(M.device), "cudaSetDevice");
        ck(cudaStreamSynchronize(M.s), "sync");
        GmresState st;
        ck(cudaMemcpy(&st, M.st.p + plane, sizeof st, cudaMemcpyDeviceToHost), "D2H state");
        const int64_t n = M.n;
        const int64_t vplane = (int64_t)(M.V.n / M.st.n);
        const int nc = std::min<int>(st.ncols, max_cols);
        if (nc > 0)
            ck(cudaMemcpy(v_dev, M.V.p + plane * vplane, (size_t)nc * n * sizeof(float2), cudaMemcpyDeviceToDevice),
               "D2D basis");
        *n_cols = st.ncols;
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_mesh_check_host(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris, double *volume,
                        int64_t *open_edges, int64_t *misoriented_edges)
{
    if (!nodes || !tris || n_nodes < 3 || n_tris < 1) return set_err(BEM_E_ARG, "bad argument");
    try {
        Geometry g;
        std::string e = compute_geometry(nodes, n_nodes, tris, n_tris, g);
        if (!e.empty()) return set_err(BEM_E_ARG, e);
        const MeshCheck mc = check_mesh(g, nodes, n_nodes, tris, n_tris);
        if (volume) *volume = mc.volume;
        if (open_edges) *open_edges = mc.open_edges;
        if (misoriented_edges) *misoriented_edges = mc.misoriented_edges;
        return BEM_OK;
    } catch (std::bad_alloc &) {
        return set_err(BEM_E_OOM, "host allocation failed");
    }
}

int bem_plan_stats_host(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris,
                        const bem_params *params, double freq_hz, double c, bem_plan_stats *out)
{
    if (!nodes || !tris || !out || n_nodes < 3 || n_tris < 1 || !(freq_hz > 0)) return set_err(BEM_E_ARG, "bad argument");
    bem_params p;
    bem_params_default(&p);
    if (params) p = *params;
    if (p.m_max < 1 || p.m_max > kMaxRule) return set_err(BEM_E_ARG, "m_max must be in 1..6");
    try {
        Geometry g;
        std::string e = compute_geometry(nodes, n_nodes, tris, n_tris, g);
        if (!e.empty()) return set_err(BEM_E_ARG, e);
        Tree t;
        const double leaf = p.mode == BEM_MODE_DIRECT ? 0.0 : (p.leaf_edge > 0 ? p.leaf_edge : auto_leaf_edge(g, p));
        build_tree(g, leaf, t);
        FreqPlan fp;
        build_plan(g, t, p, wavenumber(freq_hz, c > 0 ? c : 343.0), fp);
        const std::string bad = validate_plan(t, fp);
        if (!bad.empty()) return set_err(BEM_E_INTERNAL, "plan check: " + bad);
        fill_stats(g, t, fp, p, out);
        return BEM_OK;
    } catch (std::bad_alloc &) {
        return set_err(BEM_E_OOM, "host allocation failed");
    }
}

int bem_field_plan_stats_host(const double *nodes, int64_t n_nodes, const int32_t *tris, int64_t n_tris,
                              const double *pts, int64_t n_pts, const bem_params *params, double freq_hz,
                              double c, bem_field_stats *out)
{
    if (!nodes || !tris || !pts || !out || n_nodes < 3 || n_tris < 1 || n_pts < 1 || !(freq_hz > 0))
        return set_err(BEM_E_ARG, "bad argument");
    bem_params p;
    bem_params_default(&p);
    if (params) p = *params;
    if (p.m_max < 1 || p.m_max > kMaxRule) return set_err(BEM_E_ARG, "m_max must be in 1..6");
    try {
        Geometry g;
        std::string e = compute_geometry(nodes, n_nodes, tris, n_tris, g);
        if (!e.empty()) return set_err(BEM_E_ARG, e);
        Tree t;
        const double leaf = p.mode == BEM_MODE_DIRECT ? 0.0 : (p.leaf_edge > 0 ? p.leaf_edge : auto_leaf_edge(g, p));
        build_tree(g, leaf, t);
        EvalPlan ep;
        e = build_eval_plan(g, t, p, wavenumber(freq_hz, c > 0 ? c : 343.0), -1, pts, n_pts, kMaxTableL, ep);
        if (!e.empty()) return set_err(BEM_E_ARG, e);
        memset(out, 0, sizeof *out);
        out->leaf_level = ep.leaf_depth;
        out->levels = (int)std::min<size_t>(16, ep.far.size());
        for (int l = 0; l < out->levels; ++l) {
            const EvalLevel &F = ep.far[l];
            out->level_depth[l] = F.depth;
            out->L[l] = F.L;
            out->n_point_clusters[l] = F.npc;
            out->n_interactions[l] = F.n_inter;
            out->n_offsets[l] = (int)(F.offsets.size() / 3);
        }
        out->near_pairs = ep.near_pairs;
        out->far_pairs = ep.far_pairs;
        out->n_point_leaves = (int64_t)ep.leaf_start.size() - 1;
        return BEM_OK;
    } catch (std::bad_alloc &) {
        return set_err(BEM_E_OOM, "host allocation failed");
    }
}

int bem_mesh_blocks(void *mesh, double freq_hz, const bem_medium *medium, int32_t *block_of)
{
    if (!mesh || !block_of) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        double c, rho;
        medium_of(medium, c, rho);
        if (!(freq_hz > 0)) return set_err(BEM_E_ARG, "frequency must be positive");
        ck(cudaSetDevice(M.device), "cudaSetDevice");
        ensure_work(M);
        build_plan_dev(M, freq_hz, c);
        ck(cudaStreamSynchronize(M.s), "sync");
        const Lists &L = *fr(M).plan->lists;
        for (size_t b = 0; b < L.h_bj.size(); ++b) {
            const int4 B = L.h_bj[b];
            for (int r = 0; r < B.y; ++r) block_of[M.t.perm[B.x + r]] = (int32_t)b;
        }
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    }
}

int bem_mesh_stats(void *mesh, double freq_hz, const bem_medium *medium, bem_plan_stats *out)
{
    if (!mesh || !out) return set_err(BEM_E_ARG, "bad argument");
    auto &M = *(bem_mesh_impl *)mesh;
    try {
        double c, rho;
        medium_of(medium, c, rho);
        if (!(freq_hz > 0)) return set_err(BEM_E_ARG, "frequency must be positive");
        ck(cudaSetDevice(M.device), "cudaSetDevice");
        ensure_work(M);
        build_plan_dev(M, freq_hz, c);
        ck(cudaStreamSynchronize(M.s), "sync");
        Plan &P = *fr(M).plan;
        fill_stats(M.g, M.t, P.fp(), M.prm, out);
        for (size_t l = 0; l < P.lev.size() && l < 16; ++l) out->L[l] = P.lev[l]->L;
        out->n_tuned = (int)std::min<size_t>(4, M.tune_log.size());
        for (int q = 0; q < out->n_tuned; ++q) {
            out->tuned_depth[q] = M.tune_log[q].first;
            out->tuned_seconds[q] = M.tune_log[q].second;
        }
        int64_t bytes = 0;
        bytes += M.chi.bytes() * 6 + M.cd.bytes() * 4 + M.ad.bytes() + M.perm.bytes();
        bytes += P.lists->runs.bytes() + P.lists->row_ptr.bytes() + P.val.bytes();
        for (auto &L : P.lev) bytes += L->D.bytes() + L->M.bytes() + L->Lam.bytes() + L->ph.bytes();
        for (auto &kv : M.depth_dev) bytes += kv.second->dz.bytes() + kv.second->elem_cl.bytes();
        out->device_bytes = bytes;
        return BEM_OK;
    } catch (Fail &f) {
        return f.code;
    }
}

}  // extern "C"
