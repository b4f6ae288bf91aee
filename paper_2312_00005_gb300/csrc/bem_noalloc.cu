// bem_noalloc.cu -- a direct (every pair by quadrature) Burton-Miller product
// for callers that cannot allocate device memory.
//
// Who needs this: programs that are not allowed to call cudaMalloc once they
// are running -- a real-time audio or embedded pipeline that budgets every
// byte of device memory at start-up, or a host application whose own
// allocator owns the whole device.  They cannot create a mesh handle
// (bem_mesh_create allocates), so this entry point takes the mesh straight
// from the caller's device arrays and keeps everything it derives from them
// (element geometry, quadrature tables, the column runs, an error word) in
// one fixed array compiled into the library.
//
// That array, kScratchBytes long, is reserved on every GPU that loads the
// library and stays reserved until the process exits.  All calls on a device
// share it: a call overwrites what the previous call left there, and calls
// that overlap on the GPU (two streams, two threads) race on it.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bemfmm.h"
#include "bem_kernels.cuh"
#include "bem_plan.hpp"

namespace bem {
namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;   // 8 MiB
constexpr int64_t kNoallocMaxTris = 32768;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
// The scratch address of each device, with the id of the CUDA context it
// was looked up in: a context created anew (after cudaDeviceReset, or a
// different primary context) loads the module again, and the symbol may then
// live elsewhere, so the address is looked up again whenever the current
// context's id differs from the cached one.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    bool valid = false;
    void *p = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

// messages go to the library's per-thread error text (bem_last_error)
int fail(int code, const std::string &msg)
{
    set_last_error(msg);
    return code;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Scratch layout for n elements (each piece 256-byte aligned).
struct Layout {
    size_t chi, clo, nrm, va, e1, e2, cd, vad, e1d, e2d, ad, cp, cq, leaf_of, run_ptr, runs, ncol, Q, err, total;
    explicit Layout(int64_t n)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
        chi = take(16 * n); clo = take(16 * n); nrm = take(16 * n);
        va = take(16 * n); e1 = take(16 * n); e2 = take(16 * n);
        cd = take(24 * n); vad = take(24 * n); e1d = take(24 * n); e2d = take(24 * n); ad = take(8 * n);
        cp = take(8 * n); cq = take(8 * n);
        leaf_of = take(4 * n); run_ptr = take(8); runs = take(8); ncol = take(4);
        Q = take(sizeof(QuadTables)); err = take(4);
        total = o;
    }
};

// Element data from the caller's nodes and triangles (FP64, as the mesh set-up
// does on the host), sound-hard column coefficients, a single leaf whose one
// column run covers every element, and a cleared error word.
__global__ void k_noalloc_geometry(const double *__restrict__ nodes, int64_t n_nodes, const int32_t *__restrict__ tris,
                                   int64_t n, unsigned char *__restrict__ base, Layout lay)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int *err = (int *)(base + lay.err);
    if (j == 0) {
        ((int *)(base + lay.run_ptr))[0] = 0;
        ((int *)(base + lay.run_ptr))[1] = 1;
        ((int2 *)(base + lay.runs))[0] = make_int2(0, 0);
        ((int *)(base + lay.ncol))[0] = (int)n;
    }
    if (j >= n) return;
    const int32_t ia = tris[3 * j], ib = tris[3 * j + 1], ic = tris[3 * j + 2];
    if (ia < 0 || ib < 0 || ic < 0 || ia >= n_nodes || ib >= n_nodes || ic >= n_nodes) {
        atomicMin(err, -(int)(j + 1));
        return;
    }
    const double *a = nodes + 3 * ia, *b = nodes + 3 * ib, *c = nodes + 3 * ic;
    double e1[3], e2[3], cen[3], va[3];
    for (int q = 0; q < 3; ++q) {
        e1[q] = b[q] - a[q];
        e2[q] = c[q] - a[q];
        cen[q] = (a[q] + b[q] + c[q]) / 3.0;
        va[q] = a[q] - cen[q];
    }
    const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double l = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    if (!(l > 0.0)) {
        atomicMin(err, -(int)(j + 1));
        return;
    }
    const double area = 0.5 * l;
    const float h0 = (float)cen[0], h1 = (float)cen[1], h2 = (float)cen[2];
    ((float4 *)(base + lay.chi))[j] = make_float4(h0, h1, h2, (float)area);
    ((float4 *)(base + lay.clo))[j] = make_float4((float)(cen[0] - h0), (float)(cen[1] - h1), (float)(cen[2] - h2), 0.f);
    ((float4 *)(base + lay.nrm))[j] = make_float4((float)(cr[0] / l), (float)(cr[1] / l), (float)(cr[2] / l), 0.f);
    ((float4 *)(base + lay.va))[j] = make_float4((float)va[0], (float)va[1], (float)va[2], 0.f);
    ((float4 *)(base + lay.e1))[j] = make_float4((float)e1[0], (float)e1[1], (float)e1[2], 0.f);
    ((float4 *)(base + lay.e2))[j] = make_float4((float)e2[0], (float)e2[1], (float)e2[2], 0.f);
    for (int q = 0; q < 3; ++q) {
        ((double *)(base + lay.cd))[3 * j + q] = cen[q];
        ((double *)(base + lay.vad))[3 * j + q] = va[q];
        ((double *)(base + lay.e1d))[3 * j + q] = e1[q];
        ((double *)(base + lay.e2d))[3 * j + q] = e2[q];
    }
    ((double *)(base + lay.ad))[j] = area;
    ((float2 *)(base + lay.cp))[j] = make_float2(1.f, 0.f);   // unknown p, sound hard: q = 0
    ((float2 *)(base + lay.cq))[j] = make_float2(0.f, 0.f);
    ((int *)(base + lay.leaf_of))[j] = 0;
}

// Clears the error word and stores the quadrature tables (passed by value).
__global__ void k_noalloc_clear(int *err, QuadTables q, QuadTables *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *err = INT_MAX;
        *out = q;
    }
}

// Id of the calling thread's current CUDA context (driver entry points
// queried through the runtime, so the library needs no link to the driver
// library); false when there is none yet or the query is unavailable.
bool current_context_id(unsigned long long *id)
{
    typedef int (*GetCurrentFn)(void **);
    typedef int (*GetIdFn)(void *, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrentFn)f0;
            get_id = (GetIdFn)f1;
        }
    }
    if (!get_current || !get_id) return false;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of the scratch array on the current device (which the
// caller has made current).  Looked up once per device and context: the
// first call on a device, and the first after its context changed, call
// cudaGetSymbolAddress; later calls reuse the address.
int scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(BEM_E_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchAddr &c = g_scratch_addr[dev];
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (!(have_id && c.valid && c.ctx_id == id)) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return fail(BEM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        c.p = p;
        // the lookup made a context current if there was none
        c.valid = current_context_id(&c.ctx_id);
    }
    *out = (unsigned char *)c.p;
    return BEM_OK;
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" int bem_matvec_direct_noalloc(const double *nodes_dev, int64_t n_nodes, const int32_t *tris_dev,
                                         int64_t n_tris, double freq_hz, const bem_medium *medium, const void *x_dev,
                                         void *y_dev, void *stream)
{
    if (!nodes_dev || !tris_dev || !x_dev || !y_dev || n_nodes < 3 || n_tris < 1 || !(freq_hz > 0))
        return fail(BEM_E_ARG, "bem_matvec_direct_noalloc: bad argument");
    if (n_tris > kNoallocMaxTris)
        return fail(BEM_E_ARG, "bem_matvec_direct_noalloc: " + std::to_string((long long)n_tris) +
                                   " triangles exceed the fixed scratch limit of " +
                                   std::to_string((long long)kNoallocMaxTris));
    const Layout lay(n_tris);
    if (lay.total > kScratchBytes) return fail(BEM_E_ARG, "bem_matvec_direct_noalloc: scratch layout too large");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(BEM_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    unsigned char *base = nullptr;
    int st = scratch_address(dev, &base);
    if (st != BEM_OK) return st;
    double c = 343.0, rho = 1.21;
    medium_of(medium, c, rho);
    const double k = 2.0 * M_PI * freq_hz / c;
    bem_params prm;
    bem_params_default(&prm);
    // quadrature tables of the paper's default rules (the mesh set-up's
    // generator), copied into the scratch array by value
    const QuadTables Q = make_tables(prm);
    cudaStream_t s = (cudaStream_t)stream;
    k_noalloc_clear<<<1, 32, 0, s>>>((int *)(base + lay.err), Q, (QuadTables *)(base + lay.Q));
    k_noalloc_geometry<<<(unsigned)((n_tris + 255) / 256), 256, 0, s>>>(nodes_dev, n_nodes, tris_dev, n_tris, base,
                                                                        lay);
    NearArgs a;
    a.E.n = n_tris;
    a.E.chi = (const float4 *)(base + lay.chi);
    a.E.clo = (const float4 *)(base + lay.clo);
    a.E.nrm = (const float4 *)(base + lay.nrm);
    a.E.va = (const float4 *)(base + lay.va);
    a.E.e1 = (const float4 *)(base + lay.e1);
    a.E.e2 = (const float4 *)(base + lay.e2);
    a.E.cd = (const double *)(base + lay.cd);
    a.E.vad = (const double *)(base + lay.vad);
    a.E.e1d = (const double *)(base + lay.e1d);
    a.E.e2d = (const double *)(base + lay.e2d);
    a.E.ad = (const double *)(base + lay.ad);
    a.N.leaf_of = (const int *)(base + lay.leaf_of);
    a.N.run_ptr = (const int *)(base + lay.run_ptr);
    a.N.runs = (const int2 *)(base + lay.runs);
    a.N.ncol = (const int *)(base + lay.ncol);
    a.N.row_ptr = nullptr;
    a.Q = (const QuadTables *)(base + lay.Q);
    a.k = (float)k;
    a.ik_inv = (float)(1.0 / k);
    a.tau = 1.f;             // exterior problem
    a.cp = (const float2 *)(base + lay.cp);
    a.cq = (const float2 *)(base + lay.cq);
    k_near_fused<<<(unsigned)((n_tris + 7) / 8), 256, 0, s>>>(a, (const float2 *)x_dev, (float2 *)y_dev,
                                                               (int *)(base + lay.err), nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BEM_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    int herr = INT_MAX;
    e = cudaMemcpyAsync(&herr, base + lay.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(BEM_E_CUDA, std::string("cuda: ") + cudaGetErrorString(e));
    if (herr < 0)
        return fail(BEM_E_ARG, "element " + std::to_string(-(long long)herr - 1) +
                                   " is degenerate or has a node index out of range");
    if (herr != INT_MAX)
        return fail(BEM_E_SUBDIV_LIMIT,
                    "number of subelements which are subdivided in a loop exceeds the limit at element " +
                        std::to_string((long long)herr));
    return BEM_OK;
}

