// bem_tc.cu -- aggregation (Sec. 3.3.3, T(l)) of several right-hand sides on
// the fifth-generation tensor cores (tcgen05, sm_103a) in split-BF16
// precision.
//
// For a chunk of ne <= 64 elements of one cluster and 128 antipodal direction
// pairs s_p (and -s_p), the sums of the aggregation for R <= 4 right-hand
// sides,
//   M(s_p)  = sum_j E_pj (alpha_j + t_pj c_j),
//   M(-s_p) = sum_j conj(E_pj) (alpha_j - t_pj c_j),
// with the phase E_pj = e^{ik (z_c - x_j).s_p}, t_pj = n_j.s_p and F_pj =
// t_pj E_pj, form one real product D = A B:
//   A [128 x 256]: row p = (Re E_pj, Im E_pj, Re F_pj, Im F_pj) for j = 0..63,
//   B [256 x 16] : for right-hand side r the columns (Re M, Im M, Re M', Im M')
//                  take element j's rows as
//                  Re E: ( a_r,  a_i,  a_r,  a_i)   Im E: (-a_i,  a_r,  a_i, -a_r)
//                  Re F: ( c_r,  c_i, -c_r, -c_i)   Im F: (-c_i,  c_r, -c_i,  c_r)
//                  (alpha = a_r + i a_i, c = c_r + i c_i; M' = M(-s_p)).
// A is generated in shared memory (one sine / cosine per element and pair, as
// the FP32 kernel), B from the weights; both are split into BF16 parts, X =
// X_hi + X_lo, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32
// in tensor memory by 48 tcgen05.mma instructions (M 128, N 16, K 16) issued
// by one thread, then read back with tcgen05.ld.  The dropped term A_lo B_lo
// is below 2^-16 relative.
//
// Shared-memory operands use the canonical no-swizzle K-major layout of
// tcgen05: core matrices of 8 rows x 16 bytes (128 bytes contiguous); the
// core matrices along K are LBO bytes apart, the 8-row groups SBO bytes apart.
// Here a tile is stored K-chunk-major, so each instruction's 16-column slice
// of A (or B) is one contiguous run.
#include <cuda_bf16.h>

#include "bem_kernels.cuh"

namespace bem {
namespace {

constexpr int kTcM = 128;                  // direction pairs per tile (MMA M)
constexpr int kTcK = 4 * kTcSub;           // 64: four reals per element of a sub-chunk (MMA K per pass)
constexpr int kTcN = 4 * kMaxPlanes;       // 16: four reals per right-hand side (MMA N)
constexpr uint32_t kTcSmemA = kTcM * kTcK * 2;          // one BF16 part of A: 16 KB
constexpr uint32_t kTcSmemB = kTcN * kTcK * 2;          // one BF16 part of B: 2 KB
constexpr uint32_t kTcLboA = (kTcM / 8) * 128, kTcSboA = 128;   // 2048, 128
constexpr uint32_t kTcLboB = (kTcN / 8) * 128, kTcSboB = 128;   // 256, 128
constexpr uint32_t kTcStepA = 2 * kTcLboA, kTcStepB = 2 * kTcLboB;   // bytes per K step of 16
constexpr uint32_t kTcCols = 32;           // tensor-memory columns allocated (>= kTcN, power of 2)
constexpr unsigned int kTcSpin = 1u << 22; // polls of the completion barrier before giving up

// Byte offsets of element (row, k) in the K-chunk-major tiles.
__device__ __forceinline__ uint32_t a_off(int p, int k)
{
    return (uint32_t)(((k >> 3) * (kTcM / 8) + (p >> 3)) * 128 + (p & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint32_t b_off(int n, int k)
{
    return (uint32_t)(((k >> 3) * (kTcN / 8) + (n >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05: start address, LBO and SBO (all
// >> 4), the descriptor version (1) at bit 46, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bit 4), BF16 A and
// B (bits 7, 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

// (a, b) = hi + lo, both parts as BF16 pairs (two values per conversion;
// each value rounded to BF16, then its remainder).
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// Stores (v0, v1, v2, v3) as hi and lo parts at one 8-byte place of two tiles.
__device__ __forceinline__ void store_split4(unsigned char *hi_tile, unsigned char *lo_tile, uint32_t off, float v0,
                                             float v1, float v2, float v3)
{
    uint32_t h01, l01, h23, l23;
    split_bf16x2(v0, v1, h01, l01);
    split_bf16x2(v2, v3, h23, l23);
    *reinterpret_cast<uint2 *>(hi_tile + off) = make_uint2(h01, h23);
    *reinterpret_cast<uint2 *>(lo_tile + off) = make_uint2(l01, l23);
}

// Bounded wait for the completion of phase `parity` of the barrier the MMAs
// signal: false when it ran out (the caller sets the fault flag).
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    uint32_t ready = 0;
    for (unsigned int it = 0; it < kTcSpin && !ready; ++it) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(ready) : "r"(addr), "r"(parity) : "memory");
    }
    return ready != 0;
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 4) k_aggregate_tc(const LevelsArgs *__restrict__ A,
                                                                const AggTask *__restrict__ tasks,
                                                                const float4 *__restrict__ wts, int64_t wplane,
                                                                const float4 *__restrict__ nrm, int nr, int *fault,
                                                                const int *skip)
{
    if (skip_now(skip)) return;
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *Ahi = sm, *Alo = sm + kTcSmemA, *Bhi = sm + 2 * kTcSmemA, *Blo = Bhi + kTcSmemB;
    __shared__ float4 sd[kAggChunk];      // (z_c - x_j) k / (2 pi)
    __shared__ float4 sn[kAggChunk];      // n_j
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const AggTask T = tasks[blockIdx.x];
    const FarArgs &f = A->lev[T.lev];
    const int h = f.nd / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // tensor memory for the 128 x 16 FP32 accumulator (warp 0) and the
    // barrier the MMAs signal on completion (thread 0)
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTcCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    const float kt = f.k * 0.15915494309189535f;
    for (int q = threadIdx.x; q < T.ne; q += kTcThreads) {
        const int64_t j = T.e0 + q;
        const float4 d = f.dz[j];
        sd[q] = make_float4(kt * d.x, kt * d.y, kt * d.z, 0.f);
        sn[q] = nrm[j];
    }
    // tcgen05.alloc wrote the tensor-memory address into shared memory
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t mb = smem_u32(&mbar);
    const int p = threadIdx.x & (kTcM - 1);
    const bool pv = T.p0 + p < h;
    const float4 sv = pv ? f.dirs[T.p0 + p] : make_float4(0.f, 0.f, 0.f, 0.f);
    // the chunk in passes of kTcSub elements, the MMAs of every pass adding
    // into the same accumulator; a pass rewrites the operands only after the
    // previous pass's MMAs have completed
    const int npass = (T.ne + kTcSub - 1) / kTcSub;
    bool ok = true;
    for (int ps = 0; ps < npass && ok; ++ps) {
        const int q0 = ps * kTcSub, qn = min(kTcSub, T.ne - q0);
        if (ps > 0) {
            // the same decision in every thread (a wait that ran out in any
            // thread ends the passes for the whole block)
            ok = __syncthreads_and(mbar_wait(mb, (uint32_t)((ps - 1) & 1)) ? 1 : 0) != 0;
            if (!ok) {
                if (threadIdx.x == 0) atomicExch(fault, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        // B: thread (element q, column n) forms element q's four rows (Re E,
        // Im E, Re F, Im F) of column n = 4 r + c (right-hand side r, its
        // (Re M, Im M, Re M', Im M') column c), zero beyond the pass's
        // elements and nr right-hand sides; the four rows are consecutive in
        // K, one 8-byte store per part
        {
            static_assert(kTcThreads == kTcSub * kTcN, "one thread per (element, column) of B");
            const int q = threadIdx.x / kTcN, nn = threadIdx.x % kTcN;
            const int r = nn >> 2, c = nn & 3;
            float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < qn && r < nr) w = wts[r * wplane + T.e0 + q0 + q];
            const float ar = w.x, ai = w.y, cr = w.z, ci = w.w;
            // rows[e][c] = {{ar, ai, ar, ai}, {-ai, ar, ai, -ar}, {cr, ci, -cr, -ci}, {-ci, cr, -ci, cr}}
            const float v0 = (c & 1) ? ai : ar;
            const float v1 = c == 0 ? -ai : (c == 1 ? ar : (c == 2 ? ai : -ar));
            const float v2 = (c & 1) ? ((c == 1) ? ci : -ci) : ((c == 0) ? cr : -cr);
            const float v3 = (c & 1) ? cr : -ci;
            store_split4(Bhi, Blo, b_off(nn, 4 * q), v0, v1, v2, v3);
        }
        // A: thread takes direction pair p (fixed) and every other element
        for (int q = threadIdx.x / kTcM; q < kTcSub; q += kTcThreads / kTcM) {
            float er = 0.f, ei = 0.f, fr = 0.f, fi = 0.f;
            if (pv && q < qn) {
                const float4 d = sd[q0 + q], n = sn[q0 + q];
                sincos_turns(fmaf(d.x, sv.x, fmaf(d.y, sv.y, d.z * sv.z)), &ei, &er);
                const float t = fmaf(n.x, sv.x, fmaf(n.y, sv.y, n.z * sv.z));
                fr = t * er;
                fi = t * ei;
            }
            store_split4(Ahi, Alo, a_off(p, 4 * q), er, ei, fr, fi);
        }
        // the operands written by the threads are read by the tensor cores
        // (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x == 0) {
            // only the K steps that hold elements
            const int ksteps = (4 * qn + 15) / 16;
            const uint32_t aH = smem_u32(Ahi), aL = smem_u32(Alo), bH = smem_u32(Bhi), bL = smem_u32(Blo);
            uint32_t acc = ps > 0 ? 1u : 0u;
            for (int term = 0; term < 3; ++term) {
                const uint32_t a0 = term == 2 ? aL : aH;   // hi hi, hi lo, lo hi
                const uint32_t b0 = term == 1 ? bL : bH;
                for (int st = 0; st < ksteps; ++st) {
                    const uint64_t ad = smem_desc(a0 + st * kTcStepA, kTcLboA, kTcSboA);
                    const uint64_t bd = smem_desc(b0 + st * kTcStepB, kTcLboB, kTcSboB);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                        :: "r"(tmem), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc) : "memory");
                    acc = 1;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mb) : "memory");
        }
    }
    // wait for the last pass's MMAs (bounded: a wait that runs out sets the
    // fault flag, which the host reports, instead of hanging the GPU)
    if (warp < 4) {
        const bool ready = ok && mbar_wait(mb, (uint32_t)((npass - 1) & 1));
        if (!ready && lane == 0) atomicExch(fault, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // row 32 warp + lane of the accumulator: pair p0 + 32 warp + lane
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((uint32_t)(32 * warp) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int pr = T.p0 + 32 * warp + lane;
        if (ready && pr < h) {
            float2 *__restrict__ out = f.M + (int64_t)T.row * f.nd;
            for (int r = 0; r < nr; ++r) {
                out[r * f.mplane + pr] = make_float2(__uint_as_float(v[4 * r]), __uint_as_float(v[4 * r + 1]));
                out[r * f.mplane + pr + h] = make_float2(__uint_as_float(v[4 * r + 2]), __uint_as_float(v[4 * r + 3]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols) : "memory");
    }
    aggregate_reduce(A, T, f, kTcM, nr);
}

}  // namespace bem
