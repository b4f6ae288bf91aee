// bem_kernels.cu -- CUDA kernels (sm_103a) of the BEM + FMM matrix-vector
// product, the incident field, the field evaluation and the device-resident
// GMRES primitives.  Method: arXiv 2312.00005 (NumCalc); each kernel names
// the section or equation it computes.
#include "bem_kernels.cuh"

namespace bem {

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ float2 warp_sum(float2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ double2 warp_sum_d(double2 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}


// ------------------------------------------------------------------ near field
// Expensive pairs (heavy_rt2) of the stored near field, listed by kind so
// that the warps of k_near_store_heavy take pairs of one kind: 0 = self term,
// 1 = subdivided element, 1 + m = regular order m >= 4 (a sorting hint from
// FP32 r~; the heavy kernel decides the rules itself).  Pass 1 (heavy null)
// counts per kind; pass 2 writes each pair at off[kind] + its rank.
__global__ void k_near_classify(NearArgs a, int2 *__restrict__ heavy, unsigned long long *count,
                                const unsigned long long *off)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.E.n) return;
    const QuadTables &Q = *a.Q;
    const float3 xhi = f3(a.E.chi[i]), xlo = f3(a.E.clo[i]);
    const int t = a.N.leaf_of[i];
    const int r_end = a.N.run_ptr[t + 1], nc = a.N.ncol[t];
    int r = a.N.run_ptr[t];
    for (int p = lane; p < nc; p += 32) {
        const int j = near_col(a.N, r_end, r, p);
        const float4 cj = a.E.chi[j];
        float3 D0;
        const float rt2 = pair_rt2(f3(cj), f3(a.E.clo[j]), xhi, xlo, __frcp_rn(cj.w), D0);
        if (!heavy_rt2(i, j, rt2, Q)) continue;
        int kind;
        if (i == j) {
            kind = 0;
        } else if (rt2 < Q.rt_sub * Q.rt_sub) {
            kind = 1;
        } else {
            int m = 1;
            while (m < Q.m_max && !(rt2 > Q.R2[m])) ++m;
            kind = 1 + m;
        }
        const unsigned long long q = atomicAdd(count + kind, 1ull);
        if (heavy) heavy[off[kind] + q] = make_int2((int)i, p);
    }
}

// Near-field entries except the expensive pairs (self, order >= 4 or
// subdivided: k_near_store_heavy).  One block per (leaf, 256 columns): a
// thread holds its column's element data in registers and walks the leaf's
// rows, whose data sit in shared memory (broadcast reads); the 32 columns of
// a warp then write 32 consecutive values of one row.  r~ is compared in
// squared form (FP64 when within 2e-5 of a threshold).  Four blocks per SM
// (64 registers, a few spilled) keep more warps issuing than two blocks
// with every value in registers.
constexpr int kLightRows = 64;
// the general rule out of line, so that the common path keeps few registers
__device__ __noinline__ bool general_entry(const ElemDev &E, int64_t i, int64_t j, float3 xhi, float3 xlo,
                                           const double *xd, float3 nx, float k, float ik_inv, float tau,
                                           const QuadTables &Q, float2 cpj, float2 cqj, float2 *out)
{
    return bm_entry(E, i, j, xhi, xlo, xd, nx, k, ik_inv, tau, Q, cpj, cqj, *out);
}
// Entry A_ij of order 2 or 3 over the whole element j (no subdivision).
__device__ __forceinline__ float2 order23_entry(const ElemDev &E, int j, float3 D0, float3 nx, float k, float ik_inv,
                                                const QuadTables &Q, int code, float2 cpj, float2 cqj)
{
    const float4 cj = E.chi[j];
    const float3 ny = f3(E.nrm[j]), e1 = f3(E.e1[j]), e2 = f3(E.e2[j]);
    const float3 base = add3(D0, f3(E.va[j]));          // a - x
    float2 Kp = make_float2(0.f, 0.f), Kq = Kp;
    const int nq = code * code;
    for (int u = 0; u < nq; ++u) {
        const float3 d = mad3(Q.tri_eta[code][u], e2, mad3(Q.tri_xi[code][u], e1, base));
        bm_point(d, nx, ny, k, ik_inv, 2.0f * cj.w * Q.tri_w[code][u], Kp, Kq);
    }
    return cadd(cmul(cpj, Kp), cmul(cqj, Kq));
}

__global__ void __launch_bounds__(256, 4) k_near_store_light(NearArgs a, float2 *__restrict__ val,
                                                          int *__restrict__ err)
{
    __shared__ float4 s_hi[kLightRows], s_lo[kLightRows], s_n[kLightRows];
    __shared__ double s_xd[kLightRows][3];
    __shared__ int64_t s_rp[kLightRows];
    // per warp: queued order-2 / order-3 entries (row slot, column position, column)
    __shared__ int3 s_q[8][2][64];
    const int t = blockIdx.x;
    const int nc = a.N.ncol[t];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if ((int)(blockIdx.y * blockDim.x) >= nc) return;
    const QuadTables &Q = *a.Q;
    const int64_t e0 = a.N.leaf_start[t], e1 = a.N.leaf_start[t + 1];
    const bool live = p < nc;
    const unsigned lt = (1u << lane) - 1u;
    // this thread's column: binary search of the leaf's runs
    int j = 0;
    float4 cj = make_float4(0.f, 0.f, 0.f, 1.f), lj = cj, nj = cj;
    float2 cpj = make_float2(0.f, 0.f), cqj = cpj;
    if (live) {
        int lo = a.N.run_ptr[t], hi = a.N.run_ptr[t + 1] - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.N.runs[mid].y <= p) lo = mid;
            else hi = mid - 1;
        }
        const int2 rr = a.N.runs[lo];
        j = rr.x + (p - rr.y);
        cj = a.E.chi[j];
        lj = a.E.clo[j];
        nj = a.E.nrm[j];
        cpj = a.cp[j];
        cqj = a.cq[j];
    }
    const float inv_area = __frcp_rn(cj.w);
    int nq2 = 0, nq3 = 0;      // warp-uniform queue lengths
    // computes 32 queued entries of order c (one per lane; fewer on a flush)
    auto run_queue = [&](int c, int cnt) {
        if (lane < cnt) {
            const int3 e = s_q[warp][c - 2][lane];
            const float4 cjq = a.E.chi[e.z];
            float3 D0;
            pair_rt2(f3(cjq), f3(a.E.clo[e.z]), f3(s_hi[e.x]), f3(s_lo[e.x]), __frcp_rn(cjq.w), D0);
            val[s_rp[e.x] + e.y] = order23_entry(a.E, e.z, D0, f3(s_n[e.x]), a.k, a.ik_inv, Q, c, a.cp[e.z], a.cq[e.z]);
        }
        __syncwarp();
        // keep the entries beyond the first 32
        const int rest = cnt > 32 ? cnt - 32 : 0;
        int3 keep = make_int3(0, 0, 0);
        if (lane < rest) keep = s_q[warp][c - 2][32 + lane];
        __syncwarp();
        if (lane < rest) s_q[warp][c - 2][lane] = keep;
        __syncwarp();
        return rest;
    };
    for (int64_t b0 = e0; b0 < e1; b0 += kLightRows) {
        const int nr = (int)min((int64_t)kLightRows, e1 - b0);
        __syncthreads();
        for (int q = threadIdx.x; q < nr; q += blockDim.x) {
            s_hi[q] = a.E.chi[b0 + q];
            s_lo[q] = a.E.clo[b0 + q];
            s_n[q] = a.E.nrm[b0 + q];
            s_xd[q][0] = a.E.cd[3 * (b0 + q)];
            s_xd[q][1] = a.E.cd[3 * (b0 + q) + 1];
            s_xd[q][2] = a.E.cd[3 * (b0 + q) + 2];
            s_rp[q] = a.N.row_ptr[b0 + q];
        }
        __syncthreads();
        for (int q = 0; q < nr; ++q) {
            const int64_t i = b0 + q;
            int code = -1;
            float3 D0 = make_float3(0.f, 0.f, 0.f);
            if (live) {
                const float3 xhi = f3(s_hi[q]), xlo = f3(s_lo[q]);
                const float rt2 = pair_rt2(f3(cj), f3(lj), xhi, xlo, inv_area, D0);
                if (!heavy_rt2(i, j, rt2, Q)) {
                    if (Q.m_max > 3) {
                        const float g = 2e-5f;
                        if (fabsf(rt2 - Q.R2[1]) <= g * Q.R2[1] || fabsf(rt2 - Q.R2[2]) <= g * Q.R2[2]) {
                            double d[3];
                            for (int c = 0; c < 3; ++c)
                                d[c] = (s_xd[q][c] - a.E.cd[3 * j + c]) -
                                       (a.E.vad[3 * j + c] + (1.0 / 3.0) * a.E.e1d[3 * j + c] +
                                        (1.0 / 3.0) * a.E.e2d[3 * j + c]);
                            code = rule_from_rt_d(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) / sqrt(a.E.ad[j]), Q);
                        } else {
                            code = rt2 > Q.R2[1] ? 1 : (rt2 > Q.R2[2] ? 2 : 3);
                        }
                    } else {
                        code = 0;
                    }
                }
            }
            if (code == 1) {
                // the 1 x 1 conical rule is the centroid rule
                float2 Kp = make_float2(0.f, 0.f), Kq = Kp;
                bm_point(D0, f3(s_n[q]), f3(nj), a.k, a.ik_inv, cj.w, Kp, Kq);
                val[s_rp[q] + p] = cadd(cmul(cpj, Kp), cmul(cqj, Kq));
            } else if (code == 0) {
                // subdivision or a high order (only when the heavy split is
                // off, m_max <= 3): the general rule
                const double xd[3] = {s_xd[q][0], s_xd[q][1], s_xd[q][2]};
                float2 v;
                if (!general_entry(a.E, i, j, f3(s_hi[q]), f3(s_lo[q]), xd, f3(s_n[q]), a.k, a.ik_inv, a.tau, Q, cpj,
                                   cqj, &v)) {
                    atomicMin(err, j);
                    v = make_float2(0.f, 0.f);
                }
                val[s_rp[q] + p] = v;
            }
            // queue orders 2 and 3 for batches of one order
            const unsigned m2 = __ballot_sync(0xffffffffu, code == 2), m3 = __ballot_sync(0xffffffffu, code == 3);
            if (code == 2) s_q[warp][0][nq2 + __popc(m2 & lt)] = make_int3(q, p, j);
            if (code == 3) s_q[warp][1][nq3 + __popc(m3 & lt)] = make_int3(q, p, j);
            nq2 += __popc(m2);
            nq3 += __popc(m3);
            __syncwarp();
            if (nq2 >= 32) nq2 = run_queue(2, nq2);
            if (nq3 >= 32) nq3 = run_queue(3, nq3);
        }
        // the rows' data are replaced next: flush
        while (nq2 > 0) nq2 = run_queue(2, nq2);
        while (nq3 > 0) nq3 = run_queue(3, nq3);
    }
}

// Stored near field, expensive pairs: one thread per listed pair.
__global__ void k_near_store_heavy(NearArgs a, const int2 *__restrict__ heavy, int64_t nheavy,
                                   float2 *__restrict__ val, int *__restrict__ err)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nheavy) return;
    const int2 ip = heavy[q];
    const int64_t i = ip.x;
    const QuadTables &Q = *a.Q;
    const float4 ch = a.E.chi[i], cl = a.E.clo[i];
    const float3 xhi = f3(ch), xlo = f3(cl), nx = f3(a.E.nrm[i]);
    const double xd[3] = {a.E.cd[3 * i], a.E.cd[3 * i + 1], a.E.cd[3 * i + 2]};
    const int t = a.N.leaf_of[i];
    int r = a.N.run_ptr[t];
    const int j = near_col(a.N, a.N.run_ptr[t + 1], r, ip.y);
    float2 v;
    if (!bm_entry(a.E, i, j, xhi, xlo, xd, nx, a.k, a.ik_inv, a.tau, Q, a.cp[j], a.cq[j], v)) {
        atomicMin(err, j);
        v = make_float2(0.f, 0.f);
    }
    val[a.N.row_ptr[i] + ip.y] = v;
}

// Near-field product with stored entries: y_i = sum_p val[row_i + p] x[col(p)],
// one warp per row; four independent loads in flight per lane.
__global__ void k_near_spmv(NearArgs a, const float2 *__restrict__ val, const float2 *__restrict__ x,
                            float2 *__restrict__ y, const int *skip)
{
    if (skip_now(skip)) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.E.n) return;
    const int t = a.N.leaf_of[i];
    const int r_end = a.N.run_ptr[t + 1], nc = a.N.ncol[t];
    int r = a.N.run_ptr[t];
    const float2 *__restrict__ v = val + a.N.row_ptr[i];
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    int p = lane;
    for (; p + 96 < nc; p += 128) {
        const float2 v0 = __ldcs(v + p), v1 = __ldcs(v + p + 32), v2 = __ldcs(v + p + 64), v3 = __ldcs(v + p + 96);
        const int j0 = near_col(a.N, r_end, r, p);
        const int j1 = near_col(a.N, r_end, r, p + 32);
        const int j2 = near_col(a.N, r_end, r, p + 64);
        const int j3 = near_col(a.N, r_end, r, p + 96);
        acc0 = cfma(v0, x[j0], acc0);
        acc1 = cfma(v1, x[j1], acc1);
        acc0 = cfma(v2, x[j2], acc0);
        acc1 = cfma(v3, x[j3], acc1);
    }
    for (; p < nc; p += 32) acc0 = cfma(__ldcs(v + p), x[near_col(a.N, r_end, r, p)], acc0);
    float2 acc = warp_sum(cadd(acc0, acc1));
    if (lane == 0) y[i] = acc;
}

// Stored near field (Sec. 3.3.3, matrix N) over work items: an item is a
// range of rows of one leaf; the leaf's near columns x are staged in shared
// memory (kept while consecutive items share the leaf) and the item's values
// (rows x ncol, contiguous) are split evenly among the warps, which stream
// them from HBM (evict-first, 8 loads per lane in flight: enough for
// the bandwidth with 8 blocks per SM, and few registers, which the far-field
// kernels running beside need).  Each warp
// leaves a partial per row it touched; the block sums them in warp order.
// One block per item: items are small, so the block scheduler balances the
// work across SMs (and shares them with the far-field kernels running
// beside) whatever the leaf sizes.
// Streamed 16-byte load of stored values: read-only path, no L1 allocation,
// and an L2 fetch of the surrounding 256 bytes (the next lanes' values).
__device__ __forceinline__ float4 ld_stream4(const float4 *p)
{
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ float2 spmv_segment(const float2 *__restrict__ v, const float2 *__restrict__ xs, int c0,
                                               int c1, int lane)
{
    // sum_{c0 <= c < c1} v[c] xs[c] with c0 even: column pairs per 16-byte
    // load (v and xs 16-byte aligned), the odd last column alone
    const float4 *__restrict__ v4 = reinterpret_cast<const float4 *>(v);
    const float4 *__restrict__ x4 = reinterpret_cast<const float4 *>(xs);
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0, acc2 = acc0, acc3 = acc0;
    int q = (c0 >> 1) + lane;
    const int qe = c1 >> 1;
    for (; q + 224 < qe; q += 256) {
        float4 vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) vv[u] = ld_stream4(v4 + q + 32 * u);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            const float4 xa = x4[q + 32 * u], xb = x4[q + 32 * (u + 1)];
            acc0 = cfma(make_float2(vv[u].x, vv[u].y), make_float2(xa.x, xa.y), acc0);
            acc1 = cfma(make_float2(vv[u].z, vv[u].w), make_float2(xa.z, xa.w), acc1);
            acc2 = cfma(make_float2(vv[u + 1].x, vv[u + 1].y), make_float2(xb.x, xb.y), acc2);
            acc3 = cfma(make_float2(vv[u + 1].z, vv[u + 1].w), make_float2(xb.z, xb.w), acc3);
        }
    }
    for (; q + 96 < qe; q += 128) {
        float4 vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) vv[u] = ld_stream4(v4 + q + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
            const float4 xa = x4[q + 32 * u], xb = x4[q + 32 * (u + 1)];
            acc0 = cfma(make_float2(vv[u].x, vv[u].y), make_float2(xa.x, xa.y), acc0);
            acc1 = cfma(make_float2(vv[u].z, vv[u].w), make_float2(xa.z, xa.w), acc1);
            acc2 = cfma(make_float2(vv[u + 1].x, vv[u + 1].y), make_float2(xb.x, xb.y), acc2);
            acc3 = cfma(make_float2(vv[u + 1].z, vv[u + 1].w), make_float2(xb.z, xb.w), acc3);
        }
    }
    for (; q < qe; q += 32) {
        const float4 vv = ld_stream4(v4 + q), xa = x4[q];
        acc0 = cfma(make_float2(vv.x, vv.y), make_float2(xa.x, xa.y), acc0);
        acc1 = cfma(make_float2(vv.z, vv.w), make_float2(xa.z, xa.w), acc1);
    }
    if ((c1 & 1) && lane == 0) acc2 = cfma(v[c1 - 1], xs[c1 - 1], acc2);
    return warp_sum(cadd(cadd(acc0, acc1), cadd(acc2, acc3)));
}

__global__ void __launch_bounds__(kSpmvThreads) k_near_spmv_items(NearArgs a, const int4 *__restrict__ items,
                                                                  const float2 *__restrict__ val,
                                                                  const float2 *__restrict__ x,
                                                                  float2 *__restrict__ y, const int *skip)
{
    if (skip_now(skip)) return;
    extern __shared__ float2 xs[];
    constexpr int kW = kSpmvThreads / 32;
    static_assert(kSpmvMaxItemRows * kW == kSpmvThreads, "one partial slot per thread");
    __shared__ float2 part[kSpmvMaxItemRows][kW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 W = items[blockIdx.x];
    const int t = W.x;
    const int nc = a.N.ncol[t];
    {
        const int r0 = a.N.run_ptr[t], r1 = a.N.run_ptr[t + 1];
        for (int r = r0 + warp; r < r1; r += kW) {
            const int2 rr = a.N.runs[r];
            const int end = (r + 1 < r1) ? a.N.runs[r + 1].y : nc;
            int p = rr.y + lane;
            for (; p + 224 < end; p += 256) {
                float2 t8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) t8[u] = x[rr.x + (p + 32 * u - rr.y)];
#pragma unroll
                for (int u = 0; u < 8; ++u) xs[p + 32 * u] = t8[u];
            }
            for (; p < end; p += 32) xs[p] = x[rr.x + (p - rr.y)];
        }
    }
    part[threadIdx.x / kW][threadIdx.x % kW] = make_float2(0.f, 0.f);
    __syncthreads();
    const int64_t i0 = a.N.leaf_start[t] + W.y;
    const int nrow = min(W.z - W.y, kSpmvMaxItemRows);   // the host never makes larger items
    // the item's rows (stride ncp, padded to even) split at even positions
    const int ncp = (nc + 1) & ~1;
    const int64_t total = (int64_t)nrow * ncp;
    int64_t qa = (total * warp / kW) & ~(int64_t)1;
    const int64_t qb = warp == kW - 1 ? total : (total * (warp + 1) / kW) & ~(int64_t)1;
    while (qa < qb) {
        const int r = (int)(qa / ncp);
        const int c0 = (int)(qa - (int64_t)r * ncp);
        const int c1 = (int)min((int64_t)ncp, (int64_t)c0 + (qb - qa));
        const int c1r = min(c1, nc);
        if (c0 < c1r) {
            const float2 acc = spmv_segment(val + a.N.row_ptr[i0 + r], xs, c0, c1r, lane);
            if (lane == 0) part[r][warp] = acc;
        }
        qa += c1 - c0;
    }
    __syncthreads();
    if (threadIdx.x < nrow) {
        float2 sum = part[threadIdx.x][0];
#pragma unroll
        for (int w = 1; w < kW; ++w) sum = cadd(sum, part[threadIdx.x][w]);
        y[i0 + threadIdx.x] = sum;
    }
}

// A^T from the stored values of A, in A's layout: the rows j of leaf t, each
// padded to an even length ncp (the stride of t's rows), take at column c
// the value A_i,j of t's c-th transposed row i, which sits at trow_off[k0 +
// c] + (j - t0).  Threads take consecutive columns of a row (coalesced
// writes); the reads are the scattered column segments.
__global__ void k_near_transpose(const int64_t *__restrict__ leaf_start, const int *__restrict__ trow_ptr,
                                 const int64_t *__restrict__ trow_off, const int64_t *__restrict__ row_ptr,
                                 const float2 *__restrict__ val, float2 *__restrict__ valT)
{
    const int t = blockIdx.x;
    const int64_t t0 = leaf_start[t];
    const int nt = (int)(leaf_start[t + 1] - t0);
    const int k0 = trow_ptr[t], nk = trow_ptr[t + 1] - k0;
    const int ncp = (nk + 1) & ~1;
    const int64_t total = (int64_t)nt * ncp;
    for (int64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int jj = (int)(idx / ncp), c = (int)(idx - (int64_t)jj * ncp);
        valT[row_ptr[t0 + jj] + c] = c < nk ? val[trow_off[k0 + c] + jj] : make_float2(0.f, 0.f);
    }
}

// Transposed near-field product from the stored values (the near relation
// of the leaves being symmetric): for the elements j of leaf t = blockIdx.x,
//   y_j = sum_{s in near(t)} sum_{i in s} A_ij x_i,
// where A_ij sits at trow_off[k] + (j - first element of t) for row k of the
// leaf's list.  A warp takes R = 32 / w rows at a time (w the power of two at
// or above the leaf size, at most 32): lane (sub, jj) reads one row's value at
// column jj of a w-wide segment (a coalesced run per row); the sub-rows' and
// then the warps' sums are added in a fixed order.
__global__ void __launch_bounds__(kSpmvTThreads) k_near_spmv_t(const int64_t *__restrict__ leaf_start,
                                                               const int *__restrict__ trow_ptr,
                                                               const int *__restrict__ trow_i,
                                                               const int64_t *__restrict__ trow_off,
                                                               const float2 *__restrict__ val,
                                                               const float2 *__restrict__ x, float2 *__restrict__ y,
                                                               const int *skip)
{
    if (skip_now(skip)) return;
    constexpr int kW = kSpmvTThreads / 32;
    __shared__ float2 part[kW][32];
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j0 = leaf_start[t];
    const int cnt = (int)(leaf_start[t + 1] - j0);
    int w = 1;
    while (w < cnt && w < 32) w <<= 1;
    const int R = 32 / w, sub = lane / w, jj = lane % w;
    const int k0 = trow_ptr[t], k1 = trow_ptr[t + 1];
    for (int c0 = 0; c0 < cnt; c0 += w) {
        const bool live = c0 + jj < cnt;
        float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
        int k = k0 + warp * R + sub;
        const int step = kW * R;
        // kTU rows per warp step: their positions first, then all their
        // values and x in flight together
        constexpr int kTU = 4;
        for (; k + (kTU - 1) * step < k1; k += kTU * step) {
            int iv[kTU];
            int64_t ov[kTU];
#pragma unroll
            for (int u = 0; u < kTU; ++u) {
                iv[u] = trow_i[k + u * step];
                ov[u] = trow_off[k + u * step];
            }
            float2 xv[kTU], vv[kTU];
#pragma unroll
            for (int u = 0; u < kTU; ++u) {
                xv[u] = x[iv[u]];
                vv[u] = live ? __ldcs(val + ov[u] + c0 + jj) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < kTU; u += 2) {
                acc0 = cfma(vv[u], xv[u], acc0);
                acc1 = cfma(vv[u + 1], xv[u + 1], acc1);
            }
        }
        for (; k < k1; k += step)
            if (live) acc0 = cfma(__ldcs(val + trow_off[k] + c0 + jj), x[trow_i[k]], acc0);
        float2 acc = cadd(acc0, acc1);
        // add the R sub-rows (lanes jj, jj + w, ...) in a fixed order
        for (int o = w; o < 32; o <<= 1) {
            acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
        }
        if (sub == 0) part[warp][jj] = acc;
        __syncthreads();
        if (warp == 0 && lane < w && c0 + lane < cnt) {
            float2 sum = part[0][lane];
#pragma unroll
            for (int v = 1; v < kW; ++v) sum = cadd(sum, part[v][lane]);
            y[j0 + c0 + lane] = sum;
        }
        __syncthreads();
    }
}

// sum_{c0 <= c < c1} v[c] xs_r[c] for the planes r < nr of xs (ncp floats2
// apart), as spmv_segment for one plane: each 16-byte load of v serves all
// planes.
__device__ __forceinline__ void spmv_segment_multi(const float2 *__restrict__ v, const float2 *__restrict__ xs, int ncp,
                                                   int c0, int c1, int lane, int nr, float2 out[kMaxPlanes])
{
    const float4 *__restrict__ v4 = reinterpret_cast<const float4 *>(v);
    float2 acc0[kMaxPlanes], acc1[kMaxPlanes];
#pragma unroll
    for (int r = 0; r < kMaxPlanes; ++r) acc0[r] = acc1[r] = make_float2(0.f, 0.f);
    int q = (c0 >> 1) + lane;
    const int qe = c1 >> 1;
    for (; q + 96 < qe; q += 128) {
        float4 vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) vv[u] = ld_stream4(v4 + q + 32 * u);
#pragma unroll
        for (int r = 0; r < kMaxPlanes; ++r) {
            if (r >= nr) break;
            const float4 *__restrict__ x4 = reinterpret_cast<const float4 *>(xs + (int64_t)r * ncp);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 xa = x4[q + 32 * u];
                acc0[r] = cfma(make_float2(vv[u].x, vv[u].y), make_float2(xa.x, xa.y), acc0[r]);
                acc1[r] = cfma(make_float2(vv[u].z, vv[u].w), make_float2(xa.z, xa.w), acc1[r]);
            }
        }
    }
    for (; q < qe; q += 32) {
        const float4 vv = ld_stream4(v4 + q);
#pragma unroll
        for (int r = 0; r < kMaxPlanes; ++r) {
            if (r >= nr) break;
            const float4 xa = reinterpret_cast<const float4 *>(xs + (int64_t)r * ncp)[q];
            acc0[r] = cfma(make_float2(vv.x, vv.y), make_float2(xa.x, xa.y), acc0[r]);
            acc1[r] = cfma(make_float2(vv.z, vv.w), make_float2(xa.z, xa.w), acc1[r]);
        }
    }
    if ((c1 & 1) && lane == 0) {
        const float2 vl = v[c1 - 1];
#pragma unroll
        for (int r = 0; r < kMaxPlanes; ++r)
            if (r < nr) acc0[r] = cfma(vl, xs[(int64_t)r * ncp + c1 - 1], acc0[r]);
    }
#pragma unroll
    for (int r = 0; r < kMaxPlanes; ++r) out[r] = warp_sum(cadd(acc0[r], acc1[r]));
}

__global__ void __launch_bounds__(kSpmvThreads) k_near_spmv_items_multi(NearArgs a, const int4 *__restrict__ items,
                                                                        const float2 *__restrict__ val,
                                                                        const float2 *__restrict__ x,
                                                                        float2 *__restrict__ y, int nr, int64_t plane,
                                                                        int cw, const int *skip)
{
    if (skip_now(skip)) return;
    extern __shared__ float2 xs[];            // [nr][cw]: one chunk of the leaf's columns
    constexpr int kW = kSpmvThreads / 32;
    __shared__ float2 part[kMaxPlanes][kSpmvMaxItemRows][kW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 W = items[blockIdx.x];
    const int t = W.x;
    const int nc = a.N.ncol[t];
    const int ncp = (nc + 1) & ~1;
    const int run0 = a.N.run_ptr[t], run1 = a.N.run_ptr[t + 1];
    for (int q = threadIdx.x; q < kMaxPlanes * kSpmvMaxItemRows * kW; q += kSpmvThreads)
        (&part[0][0][0])[q] = make_float2(0.f, 0.f);
    const int64_t i0 = a.N.leaf_start[t] + W.y;
    const int nrow = min(W.z - W.y, kSpmvMaxItemRows);
    // the columns in chunks of cw (even, so every chunk's rows start on a
    // 16-byte boundary); each warp keeps its partial sums of a row in its
    // own slot of part across the chunks
    for (int cb = 0; cb < ncp; cb += cw) {
        const int cwp = min(cw, ncp - cb);
        const int ce = min(cb + cwp, nc);
        if (cb > 0) __syncthreads();          // the previous chunk's columns are no longer read
        for (int r = run0 + warp; r < run1; r += kW) {
            const int2 rr = a.N.runs[r];
            const int end = (r + 1 < run1) ? a.N.runs[r + 1].y : nc;
            const int lo = max(rr.y, cb), hi = min(end, ce);
            for (int p = lo + lane; p < hi; p += 32)
                for (int pl = 0; pl < nr; ++pl) xs[pl * cw + (p - cb)] = x[pl * plane + rr.x + (p - rr.y)];
        }
        __syncthreads();
        const int64_t total = (int64_t)nrow * cwp;
        int64_t qa = (total * warp / kW) & ~(int64_t)1;
        const int64_t qb = warp == kW - 1 ? total : (total * (warp + 1) / kW) & ~(int64_t)1;
        while (qa < qb) {
            const int r = (int)(qa / cwp);
            const int c0 = (int)(qa - (int64_t)r * cwp);
            const int c1 = (int)min((int64_t)cwp, (int64_t)c0 + (qb - qa));
            const int c1r = min(c1, ce - cb);
            if (c0 < c1r) {
                float2 acc[kMaxPlanes];
                spmv_segment_multi(val + a.N.row_ptr[i0 + r] + cb, xs, cw, c0, c1r, lane, nr, acc);
                if (lane == 0)
#pragma unroll
                    for (int pl = 0; pl < kMaxPlanes; ++pl) part[pl][r][warp] = cadd(part[pl][r][warp], acc[pl]);
            }
            qa += c1 - c0;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nrow * nr; q += kSpmvThreads) {
        const int row = q % nrow, pl = q / nrow;
        float2 sum = part[pl][row][0];
#pragma unroll
        for (int w = 1; w < kW; ++w) sum = cadd(sum, part[pl][row][w]);
        y[pl * plane + i0 + row] = sum;
    }
}

// Near-field product with the entries recomputed on the fly (no storage);
// also the conventional dense BEM product when the near list is everything.
__global__ void k_near_fused(NearArgs a, const float2 *__restrict__ x, float2 *__restrict__ y,
                             int *__restrict__ err, const int *skip)
{
    if (skip_now(skip)) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= a.E.n) return;
    const QuadTables &Q = *a.Q;
    const float4 ch = a.E.chi[i], cl = a.E.clo[i];
    const float3 xhi = f3(ch), xlo = f3(cl), nx = f3(a.E.nrm[i]);
    const double xd[3] = {a.E.cd[3 * i], a.E.cd[3 * i + 1], a.E.cd[3 * i + 2]};
    const int t = a.N.leaf_of[i];
    const int r_end = a.N.run_ptr[t + 1], nc = a.N.ncol[t];
    int r = a.N.run_ptr[t];
    float2 acc = make_float2(0.f, 0.f);
    for (int p = lane; p < nc; p += 32) {
        const int j = near_col(a.N, r_end, r, p);
        const float2 cp = a.cp[j], cq = a.cq[j];
        if (cp.x == 0.f && cp.y == 0.f && cq.x == 0.f && cq.y == 0.f) continue;
        float2 v;
        if (!bm_entry(a.E, i, j, xhi, xlo, xd, nx, a.k, a.ik_inv, a.tau, Q, cp, cq, v)) {
            atomicMin(err, j);
            continue;
        }
        acc = cfma(v, x[j], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) y[i] = acc;
}

// Row scaling of Eq. SystemI (Sec. 3.2, the solver's row-scaling
// preconditioner): dinv_i = 1 / A_ii, the self entry of row i with the
// element's own column coefficients (the value the stored near field holds).
__global__ void k_row_scale_init(NearArgs a, float2 *__restrict__ dinv, int *__restrict__ err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.E.n) return;
    const float4 ch = a.E.chi[i], cl = a.E.clo[i];
    const float3 xhi = f3(ch), xlo = f3(cl), nx = f3(a.E.nrm[i]);
    const double xd[3] = {a.E.cd[3 * i], a.E.cd[3 * i + 1], a.E.cd[3 * i + 2]};
    float2 v;
    if (!bm_entry(a.E, i, i, xhi, xlo, xd, nx, a.k, a.ik_inv, a.tau, *a.Q, a.cp[i], a.cq[i], v)) {
        atomicMin(err, (int)i);
        v = make_float2(1.f, 0.f);
    }
    const float m2 = v.x * v.x + v.y * v.y;
    dinv[i] = m2 > 0.f ? make_float2(v.x / m2, -v.y / m2) : make_float2(1.f, 0.f);
}

// y_i *= dinv_i, and y2_i *= dinv_i when y2 is given (the two parts of a
// product that the Gram-Schmidt step adds): the row scaling of a product or
// of the right-hand side.  Skips with the product kernels.
__global__ void k_row_scale(float2 *__restrict__ y, float2 *__restrict__ y2, const float2 *__restrict__ dinv,
                            int64_t n, const int *skip)
{
    if (skip_now(skip)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 d = dinv[i];
    y[i] = cmul(y[i], d);
    if (y2) y2[i] = cmul(y2[i], d);
}

// Block-Jacobi preconditioner (the block form of the solver's row scaling,
// Sec. 3.2): P = inverse of the block diagonal of A over sub-blocks of at
// most kBjMax consecutive elements of one leaf (blocks[b] = (first element,
// size, offset of its inverse, 0)).  One CUDA block per sub-block: the
// entries A_ij of the sub-block (bm_entry, the stored near field's values),
// then Gauss-Jordan inversion in place with partial pivoting in shared
// memory (FP32 complex).  The inverse is stored column-major so that the
// apply kernel's threads (one per row) read consecutive entries.  A zero
// pivot leaves the sub-block's inverse the identity (no preconditioning
// there); err takes the subdivision limit of the entries, as for the stored
// near field.
__global__ void __launch_bounds__(256) k_bj_factor(NearArgs a, const int4 *__restrict__ blocks, float2 *__restrict__ binv,
                                                   int *__restrict__ err)
{
    __shared__ float2 A[kBjMax][kBjMax + 1];
    __shared__ int piv[kBjMax];
    __shared__ int s_p;
    __shared__ bool s_bad;
    const int4 B = blocks[blockIdx.x];
    const int64_t e0 = B.x;
    const int nb = B.y;
    const QuadTables &Q = *a.Q;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int r = idx / nb, c = idx % nb;
        const int64_t i = e0 + r, j = e0 + c;
        const float4 ch = a.E.chi[i], cl = a.E.clo[i];
        const double xd[3] = {a.E.cd[3 * i], a.E.cd[3 * i + 1], a.E.cd[3 * i + 2]};
        float2 v;
        if (!bm_entry(a.E, i, j, f3(ch), f3(cl), xd, f3(a.E.nrm[i]), a.k, a.ik_inv, a.tau, Q, a.cp[j], a.cq[j], v)) {
            atomicMin(err, (int)j);
            v = make_float2(r == c ? 1.f : 0.f, 0.f);
        }
        A[r][c] = v;
    }
    if (threadIdx.x == 0) s_bad = false;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < nb; ++k) {
        // pivot: the largest |A[i][k]|, i >= k (warp 0)
        if (warp == 0) {
            float best = -1.f;
            int bi = k;
            for (int i = k + lane; i < nb; i += 32) {
                const float m = A[i][k].x * A[i][k].x + A[i][k].y * A[i][k].y;
                if (m > best) { best = m; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) {
                s_p = bi;
                piv[k] = bi;
                if (!(best > 0.f)) s_bad = true;
            }
        }
        __syncthreads();
        if (s_bad) break;
        const int p = s_p;
        if (p != k)
            for (int c = threadIdx.x; c < nb; c += blockDim.x) {
                const float2 t = A[k][c];
                A[k][c] = A[p][c];
                A[p][c] = t;
            }
        __syncthreads();
        const float2 d = A[k][k];
        const float dm = 1.f / (d.x * d.x + d.y * d.y);
        const float2 inv = make_float2(d.x * dm, -d.y * dm);
        __syncthreads();
        // row k /= pivot (the pivot's own place becomes 1 / pivot)
        for (int c = threadIdx.x; c < nb; c += blockDim.x) A[k][c] = c == k ? inv : cmul(A[k][c], inv);
        __syncthreads();
        // eliminate column k from the other rows (their column k becomes -f / pivot)
        for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
            const int i = idx / nb, c = idx % nb;
            if (i == k) continue;
            const float2 f = A[i][k];
            if (c == k) continue;
            A[i][c] = csub(A[i][c], cmul(f, A[k][c]));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            if (i != k) A[i][k] = make_float2(-(A[i][k].x * inv.x - A[i][k].y * inv.y),
                                              -(A[i][k].x * inv.y + A[i][k].y * inv.x));
        __syncthreads();
    }
    if (s_bad) {
        for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x)
            binv[B.z + idx] = make_float2((idx / nb) == (idx % nb) ? 1.f : 0.f, 0.f);
        return;
    }
    // undo the row exchanges as column exchanges, last first
    for (int k = nb - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int r = threadIdx.x; r < nb; r += blockDim.x) {
                const float2 t = A[r][k];
                A[r][k] = A[r][p];
                A[r][p] = t;
            }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int c = idx / nb, r = idx % nb;      // column-major
        binv[B.z + idx] = A[r][c];
    }
}

// w <- P (w + wnear) over the sub-blocks (wnear, when given, is cleared):
// the preconditioner applied to a product whose two parts the Gram-Schmidt
// step would add, or to a right-hand side / residual (wnear null).  One block
// of kBjMax threads per sub-block, one thread per row.  Skips with the
// product kernels.
__global__ void __launch_bounds__(kBjMax) k_bj_apply(const int4 *__restrict__ blocks, const float2 *__restrict__ binv,
                                                     float2 *__restrict__ w, float2 *__restrict__ wnear,
                                                     const int *skip)
{
    if (skip_now(skip)) return;
    __shared__ float2 xs[kBjMax];
    const int4 B = blocks[blockIdx.x];
    const int nb = B.y;
    const int r = threadIdx.x;
    if (r < nb) {
        float2 v = w[B.x + r];
        if (wnear) v = cadd(v, wnear[B.x + r]);
        xs[r] = v;
    }
    __syncthreads();
    if (r >= nb) return;
    const float2 *__restrict__ col = binv + B.z + r;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    int c = 0;
    for (; c + 1 < nb; c += 2) {
        acc0 = cfma(col[(int64_t)c * nb], xs[c], acc0);
        acc1 = cfma(col[(int64_t)(c + 1) * nb], xs[c + 1], acc1);
    }
    if (c < nb) acc0 = cfma(col[(int64_t)c * nb], xs[c], acc0);
    w[B.x + r] = cadd(acc0, acc1);
    if (wnear) wnear[B.x + r] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------------ adjoint
// Near part of the transposed product: y_j = sum_i A_ij x_i over the rows i
// whose leaves are in the near list of j's own leaf (the lists read
// backwards), with the entries recomputed by bm_entry (row i, column j; the
// forward product's entries).  Where a pair's near/far verdict differs by
// direction (the far test uses the source cluster's element areas), the
// pair is taken here or in the far part, the other way than in A.  One warp
// per column j, lanes over those rows.  zero (may be null): also cleared
// at j.
__global__ void k_near_fused_t(NearArgs a, const float2 *__restrict__ x, float2 *__restrict__ y,
                               float2 *__restrict__ zero, int *__restrict__ err, const int *skip)
{
    if (skip_now(skip)) return;
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= a.E.n) return;
    const QuadTables &Q = *a.Q;
    const float2 cp = a.cp[j], cq = a.cq[j];
    float2 acc = make_float2(0.f, 0.f);
    if (cp.x != 0.f || cp.y != 0.f || cq.x != 0.f || cq.y != 0.f) {
        const int t = a.N.leaf_of[j];
        const int r_end = a.N.run_ptr[t + 1], nc = a.N.ncol[t];
        int r = a.N.run_ptr[t];
        for (int p = lane; p < nc; p += 32) {
            const int64_t i = near_col(a.N, r_end, r, p);
            const float4 ch = a.E.chi[i], cl = a.E.clo[i];
            const float3 xhi = f3(ch), xlo = f3(cl), nx = f3(a.E.nrm[i]);
            const double xd[3] = {a.E.cd[3 * i], a.E.cd[3 * i + 1], a.E.cd[3 * i + 2]};
            float2 v;
            if (!bm_entry(a.E, i, j, xhi, xlo, xd, nx, a.k, a.ik_inv, a.tau, Q, cp, cq, v)) {
                atomicMin(err, (int)j);
                continue;
            }
            acc = cfma(v, x[i], acc);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        y[j] = acc;
        if (zero) zero[j] = make_float2(0.f, 0.f);
    }
}

// Inputs of the transposed product's far field.  With the antipodal
// symmetry of the sphere grid and D(-X, s) = D(X, -s) (Eq. FMMBase), the far
// part of A^T x is the forward aggregation of the weights (alpha, c) =
// (x_i, -x_i) (row operator 1 - s.n_i on the source side), the forward
// transfer, and a disaggregation with the row factor A_i (cq_i - ik cp_i
// (s.n_i)) = a_i + b_i (s.n_i) (the column factor of the forward product).
// x: internal order, or null to use x_int as it stands.
__global__ void k_prep_t(int64_t n, const float2 *__restrict__ x, float2 *__restrict__ xint,
                         float4 *__restrict__ wts, float4 *__restrict__ rowf, const float4 *__restrict__ chi,
                         const float2 *__restrict__ cp, const float2 *__restrict__ cq, float k, const int *skip)
{
    if (skip_now(skip)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 xv = x ? x[i] : xint[i];
    if (x) xint[i] = xv;
    if (wts) wts[i] = make_float4(xv.x, xv.y, -xv.x, -xv.y);
    const float A = chi[i].w;
    const float2 av = cscale(cq[i], A), t = cscale(cp[i], A);
    rowf[i] = make_float4(av.x, av.y, k * t.y, -k * t.x);   // (A cq, -ik A cp)
}

// Transposed field operator of the representation formula (Eq. BIE_I with
// lambda = 1, the element rules of k_field): for each element j,
//   g_j = sum_m G(x_m)_j conj(f_m),  h_j = sum_m H(x_m)_j conj(f_m),
// and the adjoint right-hand side r_j = cp_j h_j - cq_j g_j (the column
// coefficients carry tau, so r = F^T conj(f) with F the map from the
// unknowns to the field).  One warp per element, lanes over the points.
__global__ void k_field_t(ElemDev E, const QuadTables *__restrict__ Qp, const double *__restrict__ pts, int64_t M,
                          float k, const float2 *__restrict__ f, const float2 *__restrict__ cp,
                          const float2 *__restrict__ cq, float2 *__restrict__ g_out, float2 *__restrict__ r_out,
                          int *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= E.n) return;
    const QuadTables &Q = *Qp;
    float2 ga = make_float2(0.f, 0.f), ha = make_float2(0.f, 0.f);
    for (int64_t m = lane; m < M; m += 32) {
        const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
        const float3 xhi = make_float3((float)xd[0], (float)xd[1], (float)xd[2]);
        const float3 xlo = make_float3((float)(xd[0] - (double)xhi.x), (float)(xd[1] - (double)xhi.y),
                                       (float)(xd[2] - (double)xhi.z));
        float2 G = make_float2(0.f, 0.f), H = make_float2(0.f, 0.f);
        if (!integrate_regular<true>(E, j, xhi, xlo, xd, make_float3(0.f, 0.f, 1.f), k, 1.0f / k, Q, G, H)) {
            atomicMin(err, (int)j);
            continue;
        }
        const float2 w = make_float2(f[m].x, -f[m].y);
        ga = cfma(G, w, ga);
        ha = cfma(H, w, ha);
    }
    ga = warp_sum(ga);
    ha = warp_sum(ha);
    if (lane == 0) {
        g_out[j] = ga;
        r_out[j] = csub(cmul(cp[j], ha), cmul(cq[j], ga));
    }
}

// Gradient of L = sum_m |f_m|^2 with respect to the region admittances Y_r,
// from the forward solution u, the adjoint solution lambda of
// A^T lambda = F^T conj(f), g = G_f^T conj(f) and aq = A_q^T lambda (A_q the
// operator on q-unknowns, c^p = 0 and c^q = 1): element j of region r adds
//   t_j = d u_j (-tau g_j - aq_j),  d = dc^q_j / dY_r = -tau i k rho c,
// and grad_r = 2 conj(sum_j t_j) = dL/dRe Y_r + i dL/dIm Y_r.  acc
// (zeroed by the caller): [n_regions][2] gradient, then L.  region: per
// element (internal order), -1 when the element is not ADMI.
__global__ void k_adjoint_reduce(const float2 *__restrict__ u, const float2 *__restrict__ g,
                                 const float2 *__restrict__ aq, const int *__restrict__ region, int64_t n,
                                 float tau, double dre, double dim, const float2 *__restrict__ f, int64_t M,
                                 int nreg, double *acc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int r = region[i];
        if (r >= 0 && r < nreg) {
            const double gr = g[i].x, gi = g[i].y, ar = aq[i].x, ai = aq[i].y;
            const double br = -tau * gr - ar, bi = -tau * gi - ai;      // -tau g_j - aq_j
            const double ur = u[i].x, ui = u[i].y;
            const double cr = ur * br - ui * bi, ci = ur * bi + ui * br; // u_j (...)
            const double tr = dre * cr - dim * ci, ti = dre * ci + dim * cr;
            atomicAdd(&acc[2 * r], 2.0 * tr);
            atomicAdd(&acc[2 * r + 1], -2.0 * ti);
        }
    }
    if (i < M) {
        const double fr_ = f[i].x, fi = f[i].y;
        atomicAdd(&acc[2 * nreg], fr_ * fr_ + fi * fi);
    }
}

// ------------------------------------------------------------------ far field
// Per product: gather x into the internal order (x_int[i] = x[perm[i]] or
// x = xbase + jidx * n) and form the aggregation weights of the centroid
// rule, alpha_i = A_i cq_i x_i and c_i = ik A_i cp_i x_i, so that the column
// factor of Sec. 3.3.1 is alpha_i + c_i (n_i . s).
__device__ __forceinline__ void prep_store(const PrepArgs &a, int64_t i, float2 xv)
{
    a.xint[i] = xv;
    if (a.wts) {
        const float A = a.chi[i].w;
        const float2 al = cscale(cmul(a.cq[i], xv), A);
        const float2 t = cscale(cmul(a.cp[i], xv), A);
        // (alpha, c) = (A cq x, ik A cp x)
        a.wts[i] = make_float4(al.x, al.y, -a.k * t.y, a.k * t.x);
    }
}
__global__ void k_prep(PrepArgs a, const int *skip)
{
    if (skip_now(skip)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float2 *xb = a.x;
    if (a.jidx) xb += (int64_t)(*a.jidx) * a.n;
    if (blockIdx.y) {
        // right-hand side blockIdx.y: its planes of x, xint and wts
        const int64_t o = (int64_t)blockIdx.y * a.plane;
        xb += (int64_t)blockIdx.y * a.xplane;
        a.xint += o;
        if (a.wts) a.wts += o;
    }
    prep_store(a, i, a.perm ? xb[a.perm[i]] : xb[i]);
}

// Streamed 8-byte load of a stored phase (read once per product): read-only
// path, no L1 allocation.
__device__ __forceinline__ float2 ld_stream2(const float2 *p)
{
    float2 v;
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}

// Aggregation (Sec. 3.3.3, matrix T(l) with the centroid rule): for every
// source cluster c and direction s_nu,
//   M_c(nu) = sum_{j in c} e^{ik (z_c - x_j).s_nu} (alpha_j + c_j (n_j . s_nu)).
// One block per task: a chunk of at most kAggChunk elements of one cluster
// and kAggThreads antipodal direction pairs, one pair per thread; phases in
// turns, regenerated (kTab false) or read from the level's stored phases
// (kTab, the same values: k_phase_table evaluates the same expression).
// Tasks of equal size keep every block short, so no large cluster sets the
// kernel's length.  For a cluster split into several element chunks, the
// last of its blocks to finish sums the chunks' partial rows in row order.
template <int NR, bool kTab>
__device__ __forceinline__ void aggregate_body(const LevelsArgs *__restrict__ A, const float4 *__restrict__ wts,
                                               int64_t wplane, const float4 *__restrict__ nrm)
{
    const AggTask T = A->tasks[blockIdx.x];
    const FarArgs &f = A->lev[T.lev];
    __shared__ float4 sd[kTab ? 1 : kAggChunk];   // (z_c - x_j) k / (2 pi)
    __shared__ float4 sw[NR][kAggChunk];           // (alpha_j, c_j) per right-hand side
    __shared__ float4 sn[kAggChunk];               // n_j
    const float kt = f.k * 0.15915494309189535f;
    for (int q = threadIdx.x; q < T.ne; q += blockDim.x) {
        const int64_t j = T.e0 + q;
        if (!kTab) {
            const float4 d = f.dz[j];
            sd[q] = make_float4(kt * d.x, kt * d.y, kt * d.z, 0.f);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) sw[r][q] = wts[r * wplane + j];
        sn[q] = nrm[j];
    }
    __syncthreads();
    // directions in antipodal halves: s_{p + h} = -s_p, so one phase serves
    // both, e^{ik d.(-s)} = conj(e^{ik d.s}), and n.(-s) = -(n.s)
    float2 *__restrict__ out = f.M + (int64_t)T.row * f.nd;
    const int h = f.nd / 2;
    const int p = T.p0 + threadIdx.x;
    if (p < h) {
        const float4 sv = f.dirs[p];
        float2 accp[NR], accm[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) accp[r] = accm[r] = make_float2(0.f, 0.f);
        // element q of the chunk with the phase cs0 + i sn0
        auto term = [&](int q, float sn0, float cs0) {
            const float4 n = sn[q];
            const float t = fmaf(n.x, sv.x, fmaf(n.y, sv.y, n.z * sv.z));
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const float4 w = sw[r][q];
                const float2 wp = make_float2(fmaf(w.z, t, w.x), fmaf(w.w, t, w.y));
                const float2 wm = make_float2(fmaf(-w.z, t, w.x), fmaf(-w.w, t, w.y));
                // (cs + i sn) wp and (cs - i sn) wm
                accp[r].x = fmaf(cs0, wp.x, fmaf(-sn0, wp.y, accp[r].x));
                accp[r].y = fmaf(cs0, wp.y, fmaf(sn0, wp.x, accp[r].y));
                accm[r].x = fmaf(cs0, wm.x, fmaf(sn0, wm.y, accm[r].x));
                accm[r].y = fmaf(cs0, wm.y, fmaf(-sn0, wm.x, accm[r].y));
            }
        };
        if (kTab) {
            // the chunk's rows of stored phases, 16 loads per thread in flight
            const float2 *__restrict__ ph = f.ph + (int64_t)T.e0 * f.phs + p;
            int q = 0;
            for (; q + 16 <= T.ne; q += 16) {
                float2 e[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) e[u] = ld_stream2(ph + (int64_t)(q + u) * f.phs);
#pragma unroll
                for (int u = 0; u < 16; ++u) term(q + u, e[u].y, e[u].x);
            }
            for (; q < T.ne; ++q) {
                const float2 e = ld_stream2(ph + (int64_t)q * f.phs);
                term(q, e.y, e.x);
            }
        } else {
            for (int q = 0; q < T.ne; ++q) {
                const float4 d = sd[q];
                float sn0, cs0;
                sincos_turns(fmaf(d.x, sv.x, fmaf(d.y, sv.y, d.z * sv.z)), &sn0, &cs0);
                term(q, sn0, cs0);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            out[r * f.mplane + p] = accp[r];
            out[r * f.mplane + p + h] = accm[r];
        }
    }
    aggregate_reduce(A, T, f, kAggThreads, NR);
}

#define BEM_AGGREGATE_KERNEL(NR, TAB, NAME)                                                                           \
    __global__ void __launch_bounds__(kAggThreads)                                                                   \
        NAME(const LevelsArgs *__restrict__ A, const float4 *__restrict__ wts, int64_t wplane,                       \
             const float4 *__restrict__ nrm, const int *skip)                                                        \
    {                                                                                                                 \
        if (skip_now(skip)) return;                                                                                   \
        aggregate_body<NR, TAB>(A, wts, wplane, nrm);                                                                \
    }
BEM_AGGREGATE_KERNEL(1, false, k_aggregate_1)
BEM_AGGREGATE_KERNEL(2, false, k_aggregate_2)
BEM_AGGREGATE_KERNEL(3, false, k_aggregate_3)
BEM_AGGREGATE_KERNEL(4, false, k_aggregate_4)
BEM_AGGREGATE_KERNEL(1, true, k_aggregate_1t)
#undef BEM_AGGREGATE_KERNEL

// Stored phases of the aggregation (and, conjugated, of the
// disaggregation) for every level, element and antipodal direction pair,
// by the expression the products evaluate when they regenerate them:
// ph[j][p] = (cos, sin) 2 pi t, t = (k / 2 pi)(z_c - x_j).s_p in turns;
// the padding column of odd rows holds zero.
__global__ void k_phase_table(PhaseTableArgs a)
{
    int l = 0;
    while (l + 1 < a.nlev && (int)blockIdx.x >= a.start[l + 1]) ++l;
    const PhaseLevel &L = a.lev[l];
    const int64_t e0 = (int64_t)((int)blockIdx.x - a.start[l]) * kPhaseElems;
    const float kt = a.k * 0.15915494309189535f;
    for (int p = threadIdx.x; p < L.phs; p += blockDim.x) {
        const float4 sv = p < L.h ? L.dirs[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int u = 0; u < kPhaseElems; ++u) {
            const int64_t j = e0 + u;
            if (j >= a.n) break;
            float2 v = make_float2(0.f, 0.f);
            if (p < L.h) {
                const float4 d = L.dz[j];
                const float dx = kt * d.x, dy = kt * d.y, dzz = kt * d.z;
                float sn0, cs0;
                sincos_turns(fmaf(dx, sv.x, fmaf(dy, sv.y, dzz * sv.z)), &sn0, &cs0);
                v = make_float2(cs0, sn0);
            }
            L.ph[j * L.phs + p] = v;
        }
    }
}

// sin / cos of 2 pi x by sincos_turns and by sincospif, for the unit tests.
__global__ void k_selftest_sincos(const float *__restrict__ x, int64_t n, float4 *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s0, c0, s1, c1;
    sincos_turns(x[i], &s0, &c0);
    sincospif(2.f * x[i], &s1, &c1);
    out[i] = make_float4(s0, c0, s1, c1);
}

// Diagonal transfer (Sec. 3.3.3, matrix D(l)): for every target cluster t
// with an interaction list (Sec. 3.3.4),
//   Lambda_t(nu) = sum_{s in I(t)} D_L(z_t - z_s, s_nu) M_s(nu).
// A block takes one target and kTransferDirs directions (lanes); its
// kTransferWarps warps take every kTransferWarps-th list entry, each with
// kTransferUnroll entries (their D and M loads) in flight, and the partial
// sums are added in warp order.  Few warps per target with deep load
// batches hold fewer registers and warps of an SM for the same L2 traffic,
// which leaves room for the near-field product running beside.
__global__ void __launch_bounds__(32 * kTransferWarps) k_transfer_split(const LevelsArgs *__restrict__ A,
                                                                        const int *skip)
{
    if (skip_now(skip)) return;
    __shared__ float2 part[kTransferWarps][kTransferDirs];
    __shared__ int2 s_ent[kTransferEntries];      // (source cluster, offset) of the list entries
    const int4 T = A->tgroups[blockIdx.x];
    const FarArgs &f = A->lev[T.x];
    const int t = T.y, nu0 = T.z, nd = f.nd;
    // right-hand side blockIdx.y: its M and Lambda planes
    const float2 *__restrict__ Mp = f.M + blockIdx.y * f.mplane;
    float2 *__restrict__ Lp = f.Lam + blockIdx.y * f.lplane;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nu = nu0 + lane;
    const bool live = nu < nd;
    const int b = f.il_ptr[t], e = f.il_ptr[t + 1];
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    constexpr int kW = kTransferWarps, kU = kTransferUnroll;
    static_assert(kU % 2 == 0, "entries are added in pairs");
    for (int c0 = b; c0 < e; c0 += kTransferEntries) {
        const int cnt = min(kTransferEntries, e - c0);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += blockDim.x)
            s_ent[q] = make_int2(f.il_src[c0 + q], f.il_off[c0 + q]);
        __syncthreads();
        if (!live) continue;
        int q = warp;
        for (; q + kW * (kU - 1) < cnt; q += kW * kU) {
            float2 dv[kU], mv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int2 en = s_ent[q + kW * u];
                dv[u] = __ldg(f.D + (int64_t)en.y * nd + nu);
                mv[u] = Mp[(int64_t)en.x * nd + nu];
            }
#pragma unroll
            for (int u = 0; u < kU; u += 2) {
                acc0 = cfma(dv[u], mv[u], acc0);
                acc1 = cfma(dv[u + 1], mv[u + 1], acc1);
            }
        }
        for (; q < cnt; q += kW) {
            const int2 en = s_ent[q];
            acc0 = cfma(__ldg(f.D + (int64_t)en.y * nd + nu), Mp[(int64_t)en.x * nd + nu], acc0);
        }
    }
    part[warp][lane] = cadd(acc0, acc1);
    __syncthreads();
    if (warp == 0 && live) {
        float2 sum = part[0][lane];
#pragma unroll
        for (int w = 1; w < kW; ++w) sum = cadd(sum, part[w][lane]);
        Lp[(int64_t)t * nd + nu] = sum;
    }
}

// The transfer for NR right-hand sides at once: the same blocks and list
// order as k_transfer_split, each D value loaded once for all planes (the
// M and Lambda planes are mplane and lplane apart).
template <int NR>
__device__ __forceinline__ void transfer_multi_body(const LevelsArgs *__restrict__ A)
{
    constexpr int kW = kTransferWarps, kU = 8 / NR;
    __shared__ float2 part[NR][kW][kTransferDirs];
    __shared__ int2 s_ent[kTransferEntries];
    const int4 T = A->tgroups[blockIdx.x];
    const FarArgs &f = A->lev[T.x];
    const int t = T.y, nu0 = T.z, nd = f.nd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nu = nu0 + lane;
    const bool live = nu < nd;
    const int b = f.il_ptr[t], e = f.il_ptr[t + 1];
    float2 acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = make_float2(0.f, 0.f);
    for (int c0 = b; c0 < e; c0 += kTransferEntries) {
        const int cnt = min(kTransferEntries, e - c0);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += blockDim.x)
            s_ent[q] = make_int2(f.il_src[c0 + q], f.il_off[c0 + q]);
        __syncthreads();
        if (!live) continue;
        int q = warp;
        for (; q + kW * (kU - 1) < cnt; q += kW * kU) {
            float2 dv[kU], mv[kU][NR];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int2 en = s_ent[q + kW * u];
                dv[u] = __ldg(f.D + (int64_t)en.y * nd + nu);
#pragma unroll
                for (int r = 0; r < NR; ++r) mv[u][r] = f.M[r * f.mplane + (int64_t)en.x * nd + nu];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = cfma(dv[u], mv[u][r], acc[r]);
        }
        for (; q < cnt; q += kW) {
            const int2 en = s_ent[q];
            const float2 dv = __ldg(f.D + (int64_t)en.y * nd + nu);
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[r] = cfma(dv, f.M[r * f.mplane + (int64_t)en.x * nd + nu], acc[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) part[r][warp][lane] = acc[r];
    __syncthreads();
    if (warp == 0 && live) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            float2 sum = part[r][0][lane];
#pragma unroll
            for (int w = 1; w < kW; ++w) sum = cadd(sum, part[r][w][lane]);
            f.Lam[r * f.lplane + (int64_t)t * nd + nu] = sum;
        }
    }
}

#define BEM_TRANSFER_MULTI_KERNEL(NR)                                                                               \
    __global__ void __launch_bounds__(32 * kTransferWarps) k_transfer_m##NR(const LevelsArgs *__restrict__ A,      \
                                                                            const int *skip)                       \
    {                                                                                                               \
        if (skip_now(skip)) return;                                                                                 \
        transfer_multi_body<NR>(A);                                                                                 \
    }
BEM_TRANSFER_MULTI_KERNEL(2)
BEM_TRANSFER_MULTI_KERNEL(4)
#undef BEM_TRANSFER_MULTI_KERNEL

// Disaggregation over all levels (Sec. 3.3.3, matrix S(l), with the
// Burton-Miller row operator 1 + s.n_i) and the sum with the near field
// (when ynear is given; else y receives the far part alone):
//   y_i = near_i + (ik/16 pi^2) sum_l sum_nu w_nu (1 + s_nu.n_i)
//                   e^{ik (x_i - z_t).s_nu} Lambda_t(nu),
// for NR right-hand sides at once (one phase per element and direction serves
// all of them; planes n apart in ynear and y, lplane apart in Lambda).
// One block of kDisThreads per task (at most kDisTask elements of one leaf;
// large leaves are split so that no block is much longer than the others).
// Element-major: thread t takes element t % cnt of the task and every nsl-th
// antipodal direction pair (s_p, -s_p) (one phase and its conjugate; nsl =
// kDisThreads / cnt slices).  The leaf shares its cluster at every level, so
// the direction pairs and the weighted rows (A, B) of every plane are staged
// in shared memory in chunks of kDisPairChunk pairs, level by level, and read
// by all the task's elements at once; each thread keeps its element's sums in
// registers, and the slices' sums are added in slice order.
// kRowF (NR = 1): the row factor a_i + b_i (s.n_i) with per-element (a, b) =
// a.rowf[i] in place of 1 + s.n_i (the transposed product: two sums per
// element, S0 = sum (1-part) and S1 = sum (s.n-part), combined as a S0 + b S1).
constexpr int kDisPairChunk = 256;
template <int NR, bool kRowF, bool kTab>
__device__ __forceinline__ void disaggregate_body(const DisaggArgs &a, const float2 *__restrict__ ynear,
                                                  float2 *__restrict__ y)
{
    static_assert(!kRowF || NR == 1, "the transposed product has one right-hand side");
    constexpr int kS = kRowF ? 2 : 1;           // sums per element and plane
    // pairs per staged chunk; with stored phases the chunk's rows of them
    // are staged too (row stride kChunk + 1: the 16 elements of a half-warp
    // read one pair's phases from distinct banks)
    constexpr int kChunk = kTab ? kDisTabChunk : kDisPairChunk;
    static_assert(!kTab || kDisTabChunk <= kDisThreads, "the phase staging takes one pair per thread");
    __shared__ float4 dir_s[kChunk];
    __shared__ float4 ab_s[NR][kChunk];
    __shared__ float2 ph_s[kTab ? kDisTask : 1][kTab ? kChunk + 1 : 1];
    __shared__ float2 red[kDisThreads][NR * kS];
    const int2 tk = a.tasks[blockIdx.x];
    const int64_t e0 = tk.x, e1 = tk.y;
    const int cnt = (int)min((int64_t)kDisTask, e1 - e0);   // the host makes tasks of 1..kDisTask elements
    if (cnt <= 0) return;
    const int nsl = kDisThreads / cnt;
    const int q = threadIdx.x % cnt, sl = threadIdx.x / cnt;
    const bool act = sl < nsl;
    const float4 n = a.nrm[e0 + q];
    float2 acc[NR * kS];
#pragma unroll
    for (int r = 0; r < NR * kS; ++r) acc[r] = make_float2(0.f, 0.f);
    for (int l = 0; l < a.nlev; ++l) {
        const FarArgs &f = a.lev[l];
        const int c = f.elem_cl[e0];
        if (f.il_ptr[c] == f.il_ptr[c + 1]) continue;   // no interaction list at this level
        const int h = f.nd / 2;
        const float kt = -f.k * 0.15915494309189535f;
        const float4 dz = kTab ? make_float4(0.f, 0.f, 0.f, 0.f) : f.dz[e0 + q];   // z_c - x_i
        const float dx = kt * dz.x, dy = kt * dz.y, dzz = kt * dz.z;
        for (int p0 = 0; p0 < h; p0 += kChunk) {
            const int np = min(kChunk, h - p0);
            __syncthreads();
            // per antipodal pair: s_p and, with lp = w Lambda(s_p), lm =
            // w Lambda(-s_p), A = lp + lm and B = lp - lm, so that
            // (1 + t) lp + (1 - t) lm = A + t B and (1 + t) lp - (1 - t) lm = B + t A
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                const float4 d = f.dirs[p0 + i];
                dir_s[i] = d;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float2 *__restrict__ src = f.Lam + r * f.lplane + (int64_t)c * f.nd;
                    const float2 lp = cscale(src[p0 + i], d.w), lm = cscale(src[p0 + i + h], d.w);
                    ab_s[r][i] = make_float4(lp.x + lm.x, lp.y + lm.y, lp.x - lm.x, lp.y - lm.y);
                }
            }
            if (kTab) {
                // the task's rows of the chunk's phases (coalesced along the pairs)
                const float2 *__restrict__ src = f.ph + e0 * f.phs + p0;
                // (np <= blockDim.x: one pair per thread, every row's load in flight together)
                if (threadIdx.x < np) {
                    float2 v[kDisTask];
#pragma unroll
                    for (int qq = 0; qq < kDisTask; ++qq)
                        if (qq < cnt) v[qq] = ld_stream2(src + (int64_t)qq * f.phs + threadIdx.x);
#pragma unroll
                    for (int qq = 0; qq < kDisTask; ++qq)
                        if (qq < cnt) ph_s[qq][threadIdx.x] = v[qq];
                }
            }
            __syncthreads();
            if (!act) continue;
            for (int i = sl; i < np; i += nsl) {
                const float4 sv = dir_s[i];
                float sn0, cs0;
                if (kTab) {
                    // the phase of (x_i - z_c).s is the conjugate of the stored one
                    const float2 e = ph_s[q][i];
                    cs0 = e.x;
                    sn0 = -e.y;
                } else {
                    sincos_turns(fmaf(dx, sv.x, fmaf(dy, sv.y, dzz * sv.z)), &sn0, &cs0);
                }
                const float tn = fmaf(n.x, sv.x, fmaf(n.y, sv.y, n.z * sv.z));
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const float4 ab = ab_s[r][i];
                    if (kRowF) {
                        // S0 += cs A + i sn B, S1 += t (cs B + i sn A)
                        acc[0].x = fmaf(cs0, ab.x, fmaf(-sn0, ab.w, acc[0].x));
                        acc[0].y = fmaf(cs0, ab.y, fmaf(sn0, ab.z, acc[0].y));
                        acc[kS - 1].x = fmaf(tn, fmaf(cs0, ab.z, -sn0 * ab.y), acc[kS - 1].x);
                        acc[kS - 1].y = fmaf(tn, fmaf(cs0, ab.w, sn0 * ab.x), acc[kS - 1].y);
                    } else {
                        // (cs + i sn)(1 + t) lp + (cs - i sn)(1 - t) lm = cs sp + i sn dm
                        const float spx = fmaf(tn, ab.z, ab.x), spy = fmaf(tn, ab.w, ab.y);
                        const float dmx = fmaf(tn, ab.x, ab.z), dmy = fmaf(tn, ab.y, ab.w);
                        acc[r].x = fmaf(cs0, spx, fmaf(-sn0, dmy, acc[r].x));
                        acc[r].y = fmaf(cs0, spy, fmaf(sn0, dmx, acc[r].y));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < NR * kS; ++r) red[threadIdx.x][r] = acc[r];
    __syncthreads();
    for (int t = threadIdx.x; t < cnt * NR; t += blockDim.x) {
        const int qq = t % cnt, r = t / cnt;
        float2 v = red[qq][r * kS];
        for (int w = 1; w < nsl; ++w) v = cadd(v, red[w * cnt + qq][r * kS]);
        const int64_t i = e0 + qq;
        if (kRowF) {
            float2 v1 = red[qq][kS - 1];
            for (int w = 1; w < nsl; ++w) v1 = cadd(v1, red[w * cnt + qq][kS - 1]);
            const float4 rf = a.rowf[i];
            v = cadd(cmul(make_float2(rf.x, rf.y), v), cmul(make_float2(rf.z, rf.w), v1));
        }
        // (ik / 16 pi^2) v
        const float sc = a.k * 0.00633257397764611f;   // k / (16 pi^2)
        const float2 far = make_float2(-sc * v.y, sc * v.x);
        const float2 out = ynear ? cadd(ynear[r * a.n + i], far) : far;
        if (a.perm) y[r * a.n + a.perm[i]] = out;
        else y[r * a.n + i] = out;
    }
}

#define BEM_DISAGG_KERNEL(NR)                                                                                       \
    __global__ void __launch_bounds__(kDisThreads) k_disaggregate_m##NR(DisaggArgs a, const float2 *__restrict__ ynear, \
                                                                        float2 *__restrict__ y, const int *skip)     \
    {                                                                                                               \
        if (skip_now(skip)) return;                                                                                 \
        disaggregate_body<NR, false, false>(a, ynear, y);                                                           \
    }
BEM_DISAGG_KERNEL(1)
BEM_DISAGG_KERNEL(2)
BEM_DISAGG_KERNEL(4)
#undef BEM_DISAGG_KERNEL

__global__ void __launch_bounds__(kDisThreads) k_disaggregate_m1t(DisaggArgs a, const float2 *__restrict__ ynear,
                                                                  float2 *__restrict__ y, const int *skip)
{
    if (skip_now(skip)) return;
    disaggregate_body<1, false, true>(a, ynear, y);
}

// The disaggregation of the transposed product: row factor a_i + b_i (s.n_i)
// from a.rowf (see k_prep_t).
__global__ void __launch_bounds__(kDisThreads) k_disaggregate_t(DisaggArgs a, const float2 *__restrict__ ynear,
                                                                float2 *__restrict__ y, const int *skip)
{
    if (skip_now(skip)) return;
    disaggregate_body<1, true, false>(a, ynear, y);
}

__global__ void __launch_bounds__(kDisThreads) k_disaggregate_tt(DisaggArgs a, const float2 *__restrict__ ynear,
                                                                 float2 *__restrict__ y, const int *skip)
{
    if (skip_now(skip)) return;
    disaggregate_body<1, true, true>(a, ynear, y);
}

// Translation table per distinct offset X (Eq. FMMBase):
//   D_L(X, s_nu) = sum_{n=0}^{L} i^n (2n+1) h_n(k|X|) P_n(X.s_nu / |X|),
// FP64, spherical Hankel functions by upward recursion (Sec. 4.2).  The
// offsets of every far level in one launch (each block's work is a short
// serial FP64 chain, so the levels' blocks run side by side).
__global__ void k_dtable(DTableArgs a)
{
    // one block per offset X: the coefficients c_n = (2n+1) i^n h_n(k|X|)
    // depend on X only and are formed once (thread 0, upward recursion);
    // threads then take antipodal direction pairs (s, -s): with
    // P_n(-t) = (-1)^n P_n(t), the even and odd partial sums give both
    // D(X, s) = E + O and D(X, -s) = E - O.
    __shared__ double2 cn[kMaxTableL + 1];
    __shared__ double inv[kMaxTableL + 1];
    int lv = 0;
    while (lv + 1 < a.nlev && (int)blockIdx.x >= a.start[lv + 1]) ++lv;
    const DTableLevel &T = a.lev[lv];
    const int o = blockIdx.x - a.start[lv];
    const double *__restrict__ offs = T.offs;
    const double *__restrict__ dirs = T.dirs;
    const int nd = T.nd, L = T.L;
    const double k = a.k;
    float2 *__restrict__ D = T.D;
    const double X0 = offs[3 * o], X1 = offs[3 * o + 1], X2 = offs[3 * o + 2];
    const double R = sqrt(X0 * X0 + X1 * X1 + X2 * X2);
    if (threadIdx.x == 0) {
        const double x = k * R;
        double sx, cx;
        sincos(x, &sx, &cx);
        // h_0 = -i e^{ix}/x, h_1 = -e^{ix}(x + i)/x^2
        double h0r = sx / x, h0i = -cx / x;
        double h1r = -(cx * x - sx) / (x * x), h1i = -(sx * x + cx) / (x * x);
        const double ix = 1.0 / x;
        for (int n = 0; n <= L; ++n) {
            double hr, hi;
            if (n == 0) { hr = h0r; hi = h0i; }
            else if (n == 1) { hr = h1r; hi = h1i; }
            else {
                const double f = (2.0 * n - 1.0) * ix;
                hr = f * h1r - h0r;
                hi = f * h1i - h0i;
                h0r = h1r; h0i = h1i; h1r = hr; h1i = hi;
            }
            // (2n+1) i^n h_n
            const double c = 2.0 * n + 1.0;
            double ar = c * hr, ai = c * hi;
            switch (n & 3) {
                case 0: cn[n] = make_double2(ar, ai); break;
                case 1: cn[n] = make_double2(-ai, ar); break;
                case 2: cn[n] = make_double2(-ar, -ai); break;
                default: cn[n] = make_double2(ai, -ar); break;
            }
            inv[n] = 1.0 / (n + 1.0);
        }
    }
    __syncthreads();
    const double iR = 1.0 / R;
    const int h = nd / 2;
    float2 *__restrict__ Drow = D + (int64_t)o * nd;
    for (int p = threadIdx.x; p < h; p += blockDim.x) {
        const double t = (X0 * dirs[3 * p] + X1 * dirs[3 * p + 1] + X2 * dirs[3 * p + 2]) * iR;
        double p0 = 1.0, p1 = t;
        double er = cn[0].x, ei = cn[0].y, odr = 0.0, odi = 0.0;
        if (L >= 1) {
            odr = cn[1].x * t;
            odi = cn[1].y * t;
        }
        for (int n = 1; n < L; ++n) {
            // P_{n+1} = ((2n+1) t P_n - n P_{n-1}) / (n+1)
            const double p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) * inv[n];
            const double2 c = cn[n + 1];
            if (n & 1) { er = fma(c.x, p2, er); ei = fma(c.y, p2, ei); }
            else { odr = fma(c.x, p2, odr); odi = fma(c.y, p2, odi); }
            p0 = p1;
            p1 = p2;
        }
        Drow[p] = make_float2((float)(er + odr), (float)(ei + odi));
        Drow[p + h] = make_float2((float)(er - odr), (float)(ei - odi));
    }
}

// ------------------------------------------------------------------ incident field
// b_i = sum_src [p_inc(x_i) - gamma dp_inc/dn(x_i)] (right-hand side of
// Eq. SystemI), gamma = i/k; FP64 phases.  Output in the internal order.
__global__ void k_rhs(const double *__restrict__ cd, const float4 *__restrict__ nrm, int64_t n, double k,
                      const SourceDev *__restrict__ src, int nsrc, float2 *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x0 = cd[3 * i], x1 = cd[3 * i + 1], x2 = cd[3 * i + 2];
    const double n0 = nrm[i].x, n1 = nrm[i].y, n2 = nrm[i].z;
    double br = 0.0, bi = 0.0;
    for (int q = 0; q < nsrc; ++q) {
        const SourceDev s = src[q];
        double pr, pi, dr, di;
        if (s.kind == 0) {
            const double ph = k * (s.v[0] * x0 + s.v[1] * x1 + s.v[2] * x2);
            double sn, cs;
            sincos(ph, &sn, &cs);
            pr = s.amp[0] * cs - s.amp[1] * sn;
            pi = s.amp[0] * sn + s.amp[1] * cs;
            const double kd = k * (s.v[0] * n0 + s.v[1] * n1 + s.v[2] * n2);
            dr = -kd * pi;              // ik (d.n) p
            di = kd * pr;
        } else {
            const double d0 = x0 - s.v[0], d1 = x1 - s.v[1], d2 = x2 - s.v[2];
            const double R = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double sn, cs;
            sincos(k * R, &sn, &cs);
            const double g = 1.0 / (4.0 * 3.14159265358979323846 * R);
            const double gr = g * cs, gi = g * sn;
            pr = s.amp[0] * gr - s.amp[1] * gi;
            pi = s.amp[0] * gi + s.amp[1] * gr;
            const double dn = (d0 * n0 + d1 * n1 + d2 * n2) / R;
            // p (ik - 1/R) dn
            const double fr = -dn / R, fi = k * dn;
            dr = pr * fr - pi * fi;
            di = pr * fi + pi * fr;
        }
        // p - (i/k) dp
        br += pr + di / k;
        bi += pi - dr / k;
    }
    b[i] = make_float2((float)br, (float)bi);
}

// ------------------------------------------------------------------ field evaluation
// p(x) = p_inc(x) + tau sum_j [H(x)_j p_j - G(x)_j q_j] (Eq. BIE_I, lambda =
// 1; tau = +1 at exterior points, -1 at interior points).  Block (m, s)
// takes field point m and every S-th slice of blockDim elements from slice
// s, threads over elements.  With S = 1 the block adds
// the incident field and writes p(x_m); otherwise it leaves its partial sum
// in part[m S + s] and k_field_finish adds the S partials in slice order.
__device__ void field_incident(const double *xd, float k, const SourceDev *__restrict__ src, int nsrc, double &br,
                               double &bi)
{
    for (int s = 0; s < nsrc; ++s) {
        const SourceDev S = src[s];
        double sn, cs, gr, gi;
        if (S.kind == 0) {
            sincos((double)k * (S.v[0] * xd[0] + S.v[1] * xd[1] + S.v[2] * xd[2]), &sn, &cs);
            gr = cs; gi = sn;
        } else {
            const double d0 = xd[0] - S.v[0], d1 = xd[1] - S.v[1], d2 = xd[2] - S.v[2];
            const double R = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            sincos((double)k * R, &sn, &cs);
            gr = cs / (4.0 * 3.14159265358979323846 * R);
            gi = sn / (4.0 * 3.14159265358979323846 * R);
        }
        br += S.amp[0] * gr - S.amp[1] * gi;
        bi += S.amp[0] * gi + S.amp[1] * gr;
    }
}

__global__ void k_field(ElemDev E, const QuadTables *__restrict__ Qp, const double *__restrict__ pts, int64_t M,
                        float k, float tau, const float2 *__restrict__ p, const float2 *__restrict__ q,
                        const SourceDev *__restrict__ src, int nsrc, float2 *__restrict__ part,
                        float2 *__restrict__ out, int *err)
{
    const int64_t m = blockIdx.x;
    const int S = gridDim.y, sl = blockIdx.y;
    if (m >= M) return;
    const QuadTables &Q = *Qp;
    const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
    const float3 xhi = make_float3((float)xd[0], (float)xd[1], (float)xd[2]);
    const float3 xlo = make_float3((float)(xd[0] - (double)xhi.x), (float)(xd[1] - (double)xhi.y),
                                   (float)(xd[2] - (double)xhi.z));
    float2 acc = make_float2(0.f, 0.f);
    for (int64_t j = (int64_t)sl * blockDim.x + threadIdx.x; j < E.n; j += (int64_t)S * blockDim.x) {
        float2 G = make_float2(0.f, 0.f), H = make_float2(0.f, 0.f);
        if (!integrate_regular<true>(E, j, xhi, xlo, xd, make_float3(0.f, 0.f, 1.f), k, 1.0f / k, Q, G, H)) {
            atomicMin(err, (int)j);
            continue;
        }
        acc = cadd(acc, csub(cmul(H, p[j]), cmul(G, q[j])));
    }
    __shared__ float2 red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float2 v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : make_float2(0.f, 0.f);
        v = warp_sum(v);
        v = cscale(v, tau);      // tau on the integral part (Eq. BIE_I)
        if (threadIdx.x == 0) {
            if (S > 1) {
                part[m * S + sl] = v;
            } else {
                double br = v.x, bi = v.y;
                field_incident(xd, k, src, nsrc, br, bi);
                out[m] = make_float2((float)br, (float)bi);
            }
        }
    }
}

// The S partial sums of each field point in slice order, plus the incident
// field; one thread per point.
__global__ void k_field_finish(const double *__restrict__ pts, int64_t M, int S, float k,
                               const SourceDev *__restrict__ src, int nsrc, const float2 *__restrict__ part,
                               float2 *__restrict__ out)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float2 v = part[m * S];
    for (int s = 1; s < S; ++s) v = cadd(v, part[m * S + s]);
    const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
    double br = v.x, bi = v.y;
    field_incident(xd, k, src, nsrc, br, bi);
    out[m] = make_float2((float)br, (float)bi);
}

// Far-field weights of the representation formula (Eq. BIE with lambda = 1)
// for the aggregation T(l) (Sec. 3.3.3): with the one-point element rule,
//   H_j p_j - G_j q_j ~ A_j (-q_j - ik (n_j.s) p_j) e^{ik (z_s - y_j).s} (...),
// i.e. (alpha, c) = (-A q, -ik A p) in the form sum_j E_pj (alpha_j + t_pj c_j)
// of the aggregation (internal element order).
__global__ void k_field_weights(int64_t n, const float2 *__restrict__ p, const float2 *__restrict__ q,
                                const float4 *__restrict__ chi, float k, float4 *__restrict__ wts)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float A = chi[i].w;
    const float2 pv = p[i], qv = q[i];
    wts[i] = make_float4(-A * qv.x, -A * qv.y, k * A * pv.y, -k * A * pv.x);
}

// Near part of the field at points (internal point order): the element
// rules of k_field over the element runs (first element, count) of the
// point's leaf near list, one warp per point; v_m = sum_j H_j p_j - G_j q_j.
__global__ void k_field_near(ElemDev E, const QuadTables *__restrict__ Qp, const double *__restrict__ pts, int64_t M,
                             float k, const float2 *__restrict__ p, const float2 *__restrict__ q,
                             const int *__restrict__ pleaf, const int *__restrict__ nptr,
                             const int2 *__restrict__ nruns, float2 *__restrict__ v, int *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t m = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (m >= M) return;
    const QuadTables &Q = *Qp;
    const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
    const float3 xhi = make_float3((float)xd[0], (float)xd[1], (float)xd[2]);
    const float3 xlo = make_float3((float)(xd[0] - (double)xhi.x), (float)(xd[1] - (double)xhi.y),
                                   (float)(xd[2] - (double)xhi.z));
    const int pl = pleaf[m];
    float2 acc = make_float2(0.f, 0.f);
    for (int r = nptr[pl]; r < nptr[pl + 1]; ++r) {
        const int2 run = nruns[r];
        for (int u = lane; u < run.y; u += 32) {
            const int64_t j = run.x + u;
            float2 G = make_float2(0.f, 0.f), H = make_float2(0.f, 0.f);
            if (!integrate_regular<true>(E, j, xhi, xlo, xd, make_float3(0.f, 0.f, 1.f), k, 1.0f / k, Q, G, H)) {
                atomicMin(err, (int)j);
                continue;
            }
            acc = cadd(acc, csub(cmul(H, p[j]), cmul(G, q[j])));
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) v[m] = acc;
}

// The field at the points: tau (near + far) plus the incident field (FP64),
// written in caller order.
__global__ void k_field_eval_finish(const double *__restrict__ pts, int64_t M, float k, float tau,
                                    const SourceDev *__restrict__ src, int nsrc, const float2 *__restrict__ v,
                                    const int64_t *__restrict__ perm, float2 *__restrict__ out)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
    const float2 w = cscale(v[m], tau);
    double br = w.x, bi = w.y;
    field_incident(xd, k, src, nsrc, br, bi);
    out[perm[m]] = make_float2((float)br, (float)bi);
}

// Gradient of the incident fields at x (FP64): plane wave grad p = ik d p,
// point source grad p = p (ik - 1/R) (x - x0) / R.
__device__ void incident_grad(const double *xd, float k, const SourceDev *__restrict__ src, int nsrc, double *gr,
                              double *gi)
{
    for (int s = 0; s < nsrc; ++s) {
        const SourceDev S = src[s];
        double sn, cs;
        if (S.kind == 0) {
            sincos((double)k * (S.v[0] * xd[0] + S.v[1] * xd[1] + S.v[2] * xd[2]), &sn, &cs);
            // p = A e^{i phi}; ik d p = k d (i p): i p = (-p_i, p_r)
            const double pr = S.amp[0] * cs - S.amp[1] * sn, pi = S.amp[0] * sn + S.amp[1] * cs;
            for (int a = 0; a < 3; ++a) {
                gr[a] += -(double)k * S.v[a] * pi;
                gi[a] += (double)k * S.v[a] * pr;
            }
        } else {
            const double d[3] = {xd[0] - S.v[0], xd[1] - S.v[1], xd[2] - S.v[2]};
            const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            sincos((double)k * R, &sn, &cs);
            const double g = 1.0 / (4.0 * 3.14159265358979323846 * R);
            const double pr = (S.amp[0] * cs - S.amp[1] * sn) * g, pi = (S.amp[0] * sn + S.amp[1] * cs) * g;
            // p (ik - 1/R) = (-pr/R - k pi) + i (k pr - pi/R)
            const double fr = -pr / R - (double)k * pi, fi = (double)k * pr - pi / R;
            for (int a = 0; a < 3; ++a) {
                gr[a] += fr * d[a] / R;
                gi[a] += fi * d[a] / R;
            }
        }
    }
}

// Particle velocity at field points, v = grad p / (i w rho) (Eq. utopandv),
// with grad p = grad p_inc + tau sum_j [grad H(x)_j p_j - grad G(x)_j q_j]
// (Eq. BIE_I, lambda = 1, differentiated under the integral; the element
// rules of the field).  Blocks as in k_field: block (m, s) takes field point
// m and every S-th slice of blockDim elements from slice s; with S = 1 it
// writes v(x_m), otherwise its partial gradient part[(m S + s) 3 + a] for
// k_field_velocity_finish.  out: [M][3] (x, y, z components).
__global__ void k_field_velocity(ElemDev E, const QuadTables *__restrict__ Qp, const double *__restrict__ pts,
                                 int64_t M, float k, float tau, float inv_omega_rho, const float2 *__restrict__ p,
                                 const float2 *__restrict__ q, const SourceDev *__restrict__ src, int nsrc,
                                 float2 *__restrict__ part, float2 *__restrict__ out, int *err)
{
    const int64_t m = blockIdx.x;
    const int S = gridDim.y, sl = blockIdx.y;
    if (m >= M) return;
    const QuadTables &Q = *Qp;
    const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
    const float3 xhi = make_float3((float)xd[0], (float)xd[1], (float)xd[2]);
    const float3 xlo = make_float3((float)(xd[0] - (double)xhi.x), (float)(xd[1] - (double)xhi.y),
                                   (float)(xd[2] - (double)xhi.z));
    float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (int64_t j = (int64_t)sl * blockDim.x + threadIdx.x; j < E.n; j += (int64_t)S * blockDim.x) {
        GradAcc g;
        g.k = k;
#pragma unroll
        for (int a = 0; a < 3; ++a) g.gG[a] = g.gH[a] = make_float2(0.f, 0.f);
        if (!integrate_regular_acc(E, j, xhi, xlo, xd, Q, g)) {
            atomicMin(err, (int)j);
            continue;
        }
        const float2 pj = p[j], qj = q[j];
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] = cadd(acc[a], csub(cmul(g.gH[a], pj), cmul(g.gG[a], qj)));
    }
    __shared__ float2 red[3][32];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 v = warp_sum(acc[a]);
        if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double gr[3], gi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 v = threadIdx.x < (blockDim.x >> 5) ? red[a][threadIdx.x] : make_float2(0.f, 0.f);
            v = warp_sum(v);
            gr[a] = tau * v.x;   // tau on the integral part (Eq. BIE_I)
            gi[a] = tau * v.y;
        }
        if (threadIdx.x == 0) {
            if (S > 1) {
                for (int a = 0; a < 3; ++a) part[(m * S + sl) * 3 + a] = make_float2((float)gr[a], (float)gi[a]);
            } else {
                incident_grad(xd, k, src, nsrc, gr, gi);
                // v = grad p / (i w rho) = -i grad p / (w rho)
                for (int a = 0; a < 3; ++a)
                    out[3 * m + a] = make_float2((float)(gi[a] * inv_omega_rho), (float)(-gr[a] * inv_omega_rho));
            }
        }
    }
}

// The S partial gradients of each field point in slice order, the incident
// gradient and the scaling to the velocity; one thread per point.
__global__ void k_field_velocity_finish(const double *__restrict__ pts, int64_t M, int S, float k,
                                        float inv_omega_rho, const SourceDev *__restrict__ src, int nsrc,
                                        const float2 *__restrict__ part, float2 *__restrict__ out)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double gr[3], gi[3];
    for (int a = 0; a < 3; ++a) {
        float2 v = part[(m * S) * 3 + a];
        for (int s = 1; s < S; ++s) v = cadd(v, part[(m * S + s) * 3 + a]);
        gr[a] = v.x;
        gi[a] = v.y;
    }
    const double xd[3] = {pts[3 * m], pts[3 * m + 1], pts[3 * m + 2]};
    incident_grad(xd, k, src, nsrc, gr, gi);
    for (int a = 0; a < 3; ++a)
        out[3 * m + a] = make_float2((float)(gi[a] * inv_omega_rho), (float)(-gr[a] * inv_omega_rho));
}

// ------------------------------------------------------------------ vector helpers
__global__ void k_gather(const float2 *__restrict__ x, const int64_t *__restrict__ perm, int64_t n,
                         float2 *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[perm[i]];
}
// Iterative refinement of a mixed-precision solve: r = b - y in FP64 from the
// FP32 right-hand side and product (y = A x with the FP32 products), stored
// as FP32 in r; part[blockIdx.x] = the block's ||r||^2 in FP64.
__global__ void k_refine_residual(const float2 *__restrict__ b, const float2 *__restrict__ y, float2 *__restrict__ r,
                                  int64_t n, double *__restrict__ part)
{
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double rx = (double)b[i].x - (double)y[i].x, ry = (double)b[i].y - (double)y[i].y;
        r[i] = make_float2((float)rx, (float)ry);
        v += rx * rx + ry * ry;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

// x64 += d (the refinement's FP64 solution) and x = x64 rounded to FP32.
__global__ void k_refine_update(double2 *__restrict__ x64, const float2 *__restrict__ d, float2 *__restrict__ x,
                                int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = make_double2(x64[i].x + (double)d[i].x, x64[i].y + (double)d[i].y);
    x64[i] = v;
    x[i] = make_float2((float)v.x, (float)v.y);
}

// b <- b - y
__global__ void k_sub(float2 *__restrict__ b, const float2 *__restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = csub(b[i], y[i]);
}
// w <- b - w
__global__ void k_rsub(float2 *__restrict__ w, const float2 *__restrict__ b, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = csub(b[i], w[i]);
}
// p, q from the unknowns u and the known data z (internal order), written in
// the caller order: VELO/ADMI: p = u, q = a u + z; PRES: p = z, q = u.
__global__ void k_pq(const float2 *__restrict__ u, const float2 *__restrict__ z, const float2 *__restrict__ aq,
                     const int *__restrict__ type, const int64_t *__restrict__ perm, int64_t n,
                     float2 *__restrict__ p, float2 *__restrict__ q)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 pv, qv;
    if (type[i] == 1) { pv = z[i]; qv = u[i]; }
    else { pv = u[i]; qv = cfma(aq[i], u[i], z[i]); }
    p[perm[i]] = pv;
    if (q) q[perm[i]] = qv;
}


// ------------------------------------------------------------------ GMRES
// Givens step (FP64), run by one warp: h_{j+1,j} = ||w|| (nn = ||w||^2),
// apply the previous rotations to column j, form the new rotation, update g
// and the residual estimate, and decide whether the cycle ends.
//
// Rotation l maps (t_l, h_{l+1}) to (conj(c_l) t_l + s_l h_{l+1},
// -s_l t_l + c_l h_{l+1}) with s_l real, so the running entry obeys the affine
// recurrence t_{l+1} = a_l t_l + b_l, a_l = -s_l, b_l = c_l h_{l+1}.  The warp
// composes these maps with a prefix scan (|a_l| <= 1: no growth) instead of
// applying j rotations one after another in one thread: FP64 issue is scarce
// on this part, and the serial chain costs j times its latency.
__device__ void gm_givens_warp(const GmresArgs &a, double nn, int j)
{
    __shared__ double2 sh[kMaxRestart + 1], shr[kMaxRestart + 1];
    __shared__ double2 s_tj;
    GmresState *st = a.st;
    const int m = a.m;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    for (int l = lane; l <= j; l += 32) sh[l] = __ldcg(a.H + (int64_t)l * m + j);
    __syncwarp();
    const int K = (j + 31) / 32;                 // rotations per lane
    const int l0 = min(j, lane * K), l1 = min(j, l0 + K);
    double A = 1.0;
    double2 B = make_double2(0.0, 0.0);
    for (int l = l0; l < l1; ++l) {
        const double2 c = __ldcg(a.cs + l);
        const double sl = __ldcg(&a.sn[l].x);
        const double2 h1 = sh[l + 1];
        const double bx = c.x * h1.x - c.y * h1.y, by = c.x * h1.y + c.y * h1.x;
        A = -sl * A;
        B = make_double2(fma(-sl, B.x, bx), fma(-sl, B.y, by));
    }
    // inclusive scan: mine o (lane - o)'s
    for (int o = 1; o < 32; o <<= 1) {
        const double Ap = __shfl_up_sync(full, A, o);
        const double Bx = __shfl_up_sync(full, B.x, o), By = __shfl_up_sync(full, B.y, o);
        if (lane >= o) {
            B = make_double2(fma(A, Bx, B.x), fma(A, By, B.y));
            A *= Ap;
        }
    }
    double Ae = __shfl_up_sync(full, A, 1);
    double Bex = __shfl_up_sync(full, B.x, 1), Bey = __shfl_up_sync(full, B.y, 1);
    if (lane == 0) { Ae = 1.0; Bex = 0.0; Bey = 0.0; }
    const double2 h0 = sh[0];
    double2 t = make_double2(fma(Ae, h0.x, Bex), fma(Ae, h0.y, Bey));
    for (int l = l0; l < l1; ++l) {
        const double2 c = __ldcg(a.cs + l);
        const double sl = __ldcg(&a.sn[l].x);
        const double2 h1 = sh[l + 1];
        shr[l] = make_double2(c.x * t.x + c.y * t.y + sl * h1.x, c.x * t.y - c.y * t.x + sl * h1.y);
        t = make_double2(-sl * t.x + c.x * h1.x - c.y * h1.y, -sl * t.y + c.x * h1.y + c.y * h1.x);
    }
    if ((j == 0 && lane == 0) || (l0 < l1 && l1 == j)) s_tj = t;
    __syncwarp();
    if (lane == 0) {
        const double hn = sqrt(nn);
        const double2 hj = s_tj;
        const double den = sqrt(hj.x * hj.x + hj.y * hj.y + hn * hn);
        double2 c, sv;
        if (den == 0.0) { c = make_double2(1.0, 0.0); sv = make_double2(0.0, 0.0); }
        else { c = make_double2(hj.x / den, hj.y / den); sv = make_double2(hn / den, 0.0); }
        a.cs[j] = c;
        a.sn[j] = sv;
        shr[j] = make_double2(den, 0.0);
        shr[j + 1] = make_double2(0.0, 0.0);
        const double2 g0 = a.g[j];
        a.g[j] = make_double2(c.x * g0.x + c.y * g0.y, c.x * g0.y - c.y * g0.x);
        const double2 g1 = make_double2(-(sv.x * g0.x - sv.y * g0.y), -(sv.x * g0.y + sv.y * g0.x));
        a.g[j + 1] = g1;
        const double res = sqrt(g1.x * g1.x + g1.y * g1.y) / st->bnorm;
        st->resid = res;
        st->iters += 1;
        st->hn = hn;
        st->ncols = j + 1;
        if (res <= st->tol || hn <= 1e-300 * st->bnorm || j + 1 >= m || st->iters >= st->maxit) {
            st->done = 1;
            st->converged = res <= st->tol;
        } else {
            st->j = j + 1;
        }
    }
    __syncwarp();
    for (int l = lane; l <= j + 1; l += 32) a.H[(int64_t)l * m + j] = shr[l];
}

// Compensated FP32 ("float-float") sums: s + e holds the running sum to
// about 2^-44 relative.  The reductions below are issued by every block in
// a fixed order, so all blocks derive identical values without FP64, whose
// issue rate and latency on this part would dominate the step.
struct FF {
    float2 hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_add1(float &hi, float &lo, float xh, float xl)
{
    float s, e;
    two_sum(hi, xh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, xl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
__device__ __forceinline__ void ff_add(FF &a, const FF &b)
{
    ff_add1(a.hi.x, a.lo.x, b.hi.x, b.lo.x);
    ff_add1(a.hi.y, a.lo.y, b.hi.y, b.lo.y);
}
// sum of p[0..n), n <= 32 kFFLoads (float2, written by other blocks before
// the reduction: read through L2) by one warp: lane order, then a fixed
// xor tree.  All loads are issued before the first add.
constexpr int kFFLoads = 16;
__device__ __forceinline__ FF warp_sum_ff(const float2 *p, int n)
{
    FF v = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const int lane = threadIdx.x & 31;
    float2 x[kFFLoads];
#pragma unroll
    for (int u = 0; u < kFFLoads; ++u) {
        const int q = lane + 32 * u;
        x[u] = q < n ? __ldcg(p + q) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kFFLoads; ++u) {
        const FF t = {x[u], make_float2(0.f, 0.f)};
        ff_add(v, t);
    }
    for (int o = 16; o > 0; o >>= 1) {
        FF x;
        x.hi.x = __shfl_xor_sync(0xffffffffu, v.hi.x, o);
        x.hi.y = __shfl_xor_sync(0xffffffffu, v.hi.y, o);
        x.lo.x = __shfl_xor_sync(0xffffffffu, v.lo.x, o);
        x.lo.y = __shfl_xor_sync(0xffffffffu, v.lo.y, o);
        // both partners add in the same operand order: identical results
        if ((threadIdx.x & o) == 0) ff_add(v, x);
        else { ff_add(x, v); v = x; }
    }
    return v;
}

// ------------------------------------------------------------------ Gram-Schmidt
// Classical Gram-Schmidt with selective reorthogonalisation (DGKS: a second
// pass when ||w_1|| < 0.1 ||w||) for Arnoldi column j, in three launches with
// no block ever waiting for another:
//   k_gs_dots    w = (far + near part of A v_j); each block adds its partial
//                dots V_l^H w into column j of H and its partial ||w||^2
//                into acc (FP64 atomics);
//   k_gs_update  w_1 = w - V h and its partial ||w_1||^2; the DGKS test on
//                the sums (||w_1||^2 = ||w||^2 - |h|^2 by Pythagoras; exact
//                enough to decide, since the sums are) asks for a second pass
//                rarely, and only then the block adds the dots V_l^H w_1;
//   k_gs_finish  the decision read from the state (k_gs_update's block 0
//                leaves it there); without a second pass v_{j+1} = w_1 /
//                ||w_1|| and the next product's inputs; with one h_2 is
//                added to column j of H, w_2 = w_1 - V h_2 and its partial
//                ||w_2||^2 are formed, and the last block to finish (an
//                arrival counter) forms v_{j+1} = w_2 / ||w_2|| for every
//                row (second passes are rare).
// Every norm is summed from the vector itself, never estimated (when w_1 is
// mostly rounding noise inside span(V), ||w_1||^2 - |h_2|^2 would cancel to
// nothing and fake a breakdown of the Arnoldi process).
// Every block of k_gs_update takes the same decision from the same FP64
// sums.  Block b owns
// rows [b R, b R + R) of every vector (R about 64: the basis comes from HBM,
// since each product streams the stored near field through L2, so many
// blocks keep many loads in flight), with FP32 sums within a block.  The
// FP64 sums of the blocks' FP32 partials are exact whenever the partials span
// fewer than 29 binary orders of magnitude, so they do not depend on the
// order in which the blocks add them.  acc ([4]: ||w||^2, ||w_1||^2,
// ||w_2||^2, arrival counter) and h2 alternate between two copies by the
// parity of j: the normalising block clears the copy of step j + 1
// (k_gm_start clears both at the start of a cycle, where H is cleared too).
// The Givens step (k_gm_givens) follows on a side stream.
__device__ __forceinline__ int gs_rows(const GsArgs &a, int64_t &r0)
{
    r0 = (int64_t)blockIdx.x * a.rows;
    const int64_t rem = a.g.n - r0;
    return rem <= 0 ? 0 : (int)(rem < a.rows ? rem : (int64_t)a.rows);
}

__device__ __forceinline__ void atomic_add_c(double2 *p, float2 v)
{
    atomicAdd(&p->x, (double)v.x);
    atomicAdd(&p->y, (double)v.y);
}

// (The basis is read through L1 here and in gs_update: a block reads only
// its own rows, which k_gs_update reads twice, for the update and then the
// second pass's dots.)
// Partial dots sum_{i in block} conj(V_l[i]) ws[i], l <= j, added into
// dst[l * stride]: warp w takes the columns l = w (mod 8), four at a time,
// its lanes the rows, so that every warp keeps several independent loads in
// flight.
__device__ void gs_dots_part(const GsArgs &a, const float2 *ws, int R, int64_t r0, int j, double2 *dst, int64_t stride)
{
    const GmresArgs &g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarp = kGsThreads / 32;
    constexpr int kC = 8;     // columns per warp at a time (their loads in flight together)
    for (int l0 = warp; l0 <= j; l0 += kC * nwarp) {
        float2 acc[kC];
#pragma unroll
        for (int u = 0; u < kC; ++u) acc[u] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int i = lane; i < R; i += 32) {
            const float2 y = ws[i];
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int l = l0 + u * nwarp;
                if (l <= j) {
                    const float2 x = __ldca(g.V + (int64_t)l * g.n + r0 + i);
                    acc[u].x = fmaf(x.x, y.x, fmaf(x.y, y.y, acc[u].x));
                    acc[u].y = fmaf(x.x, y.y, fmaf(-x.y, y.x, acc[u].y));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kC; ++u) {
            const int l = l0 + u * nwarp;
            const float2 d = warp_sum(acc[u]);
            if (lane == u && l <= j) atomic_add_c(dst + (int64_t)l * stride, d);
        }
    }
}

// The block's sum_{i in block} |ws[i]|^2 added into *nrm.
__device__ void gs_norm_part(const float2 *ws, int R, double *nrm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarp = kGsThreads / 32;
    __shared__ float red[nwarp];
    float v2 = 0.f;
    for (int i = threadIdx.x; i < R; i += kGsThreads) v2 = fmaf(ws[i].x, ws[i].x, fmaf(ws[i].y, ws[i].y, v2));
    for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    if (lane == 0) red[warp] = v2;
    __syncthreads();
    if (warp == 0) {
        float v = lane < nwarp ? red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(nrm, (double)v);
    }
}

// w_1 = ws - V h (h as FP32 in hs), written back into ws: thread (row rr,
// column group cg) sums the columns l = cg (mod kCg) of its row.
__device__ void gs_update(const GsArgs &a, float2 *ws, const float2 *hs, int R, int64_t r0, int j)
{
    const GmresArgs &g = a.g;
    constexpr int kRowsPerPass = 64, kCg = kGsThreads / kRowsPerPass;
    __shared__ float2 cpart[2][kGsThreads];
    const int cg = threadIdx.x / kRowsPerPass, rr = threadIdx.x % kRowsPerPass;
    // two passes of rows at a time, so each thread has the loads of two rows
    // in flight
    for (int i0 = 0; i0 < R; i0 += 2 * kRowsPerPass) {
        const int ia = i0 + rr, ib = i0 + kRowsPerPass + rr;
        const bool va = ia < R, vb = ib < R;
        float2 acca = make_float2(0.f, 0.f), accb = acca;
        const float2 *pa = g.V + r0 + ia, *pb = g.V + r0 + ib;
#pragma unroll 8
        for (int l = cg; l <= j; l += kCg) {
            const float2 h = hs[l];
            const int64_t o = (int64_t)l * g.n;
            const float2 v = va ? __ldca(pa + o) : make_float2(0.f, 0.f);
            const float2 w = vb ? __ldca(pb + o) : make_float2(0.f, 0.f);
            acca.x = fmaf(h.x, v.x, fmaf(-h.y, v.y, acca.x));
            acca.y = fmaf(h.x, v.y, fmaf(h.y, v.x, acca.y));
            accb.x = fmaf(h.x, w.x, fmaf(-h.y, w.y, accb.x));
            accb.y = fmaf(h.x, w.y, fmaf(h.y, w.x, accb.y));
        }
        cpart[0][threadIdx.x] = acca;
        cpart[1][threadIdx.x] = accb;
        __syncthreads();
        if (cg < 2) {
            const int i = cg == 0 ? ia : ib;
            if (i < R) {
                float2 c = cpart[cg][rr];
#pragma unroll
                for (int q = 1; q < kCg; ++q) {
                    c.x += cpart[cg][rr + q * kRowsPerPass].x;
                    c.y += cpart[cg][rr + q * kRowsPerPass].y;
                }
                ws[i] = make_float2(ws[i].x - c.x, ws[i].y - c.y);
            }
        }
        __syncthreads();
    }
}

// h_l (l <= j) of a column sum as FP32 into hs, and sum_l |h_l|^2 (FP64, the
// same order in every block) returned to every thread.
__device__ double gs_load_h(const double2 *src, int64_t stride, float2 *hs, int j)
{
    __shared__ double s_hh;
    for (int l = threadIdx.x; l <= j; l += kGsThreads) {
        const double2 h = __ldcg(src + (int64_t)l * stride);
        hs[l] = make_float2((float)h.x, (float)h.y);
    }
    if (threadIdx.x < 32) {
        double hh = 0.0;
        for (int l = threadIdx.x; l <= j; l += 32) {
            const double2 h = __ldcg(src + (int64_t)l * stride);
            hh += h.x * h.x + h.y * h.y;
        }
        for (int o = 16; o > 0; o >>= 1) hh += __shfl_xor_sync(0xffffffffu, hh, o);
        if (threadIdx.x == 0) s_hh = hh;
    }
    __syncthreads();
    return s_hh;
}

// DGKS test from the FP64 sums with the classical threshold 1/sqrt(2):
// ||w_1||^2 = ||w||^2 - |h|^2 < ||w||^2 / 2.  (A threshold of 0.1 let the
// FP32 basis lose orthogonality roughly as eps / relres over a GMRES cycle:
// 0.02 after 19 steps, 1 after 53.)
__device__ __forceinline__ bool gs_second_pass(double ww, double hh) { return ww - hh < 0.5 * ww; }

__global__ void __launch_bounds__(kGsThreads) k_gs_dots(GsArgs a)
{
    const GmresArgs &g = a.g;
    GmresState *st = g.st;
    int64_t r0;
    const int R = gs_rows(a, r0);
    // w = A v_j (far part g.w + near part) and the state (j, done) are
    // loaded together: one memory round trip before any decision
    constexpr int kWr = kGsMaxRows / kGsThreads;
    float2 wv[kWr];
#pragma unroll
    for (int u = 0; u < kWr; ++u) {
        const int i = threadIdx.x + u * kGsThreads;
        wv[u] = i < R ? cadd(g.w[r0 + i], a.wnear[r0 + i]) : make_float2(0.f, 0.f);
    }
    const int2 jd = __ldcv(reinterpret_cast<const int2 *>(&st->j));   // (j, done)
    const int j = jd.x, done = jd.y;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->skip_prod = done;
    if (done) return;
    // v_j was stored unnormalised (||v_j||^2 = st->nn, set by k_gm_givens of
    // step j - 1, or 1 by k_gm_start): scale the block's rows of v_j and of
    // the product
    const float sc = (float)(1.0 / sqrt(__ldcv(&st->nn)));
    float2 *vj = g.V + (int64_t)j * g.n + r0;
    __shared__ float2 ws[kGsMaxRows];
#pragma unroll
    for (int u = 0; u < kWr; ++u) {
        const int i = threadIdx.x + u * kGsThreads;
        if (i < R) {
            const float2 wsc = cscale(wv[u], sc);
            ws[i] = wsc;
            g.w[r0 + i] = wsc;
            if (j > 0) vj[i] = cscale(vj[i], sc);
        }
    }
    __syncthreads();
    gs_dots_part(a, ws, R, r0, j, g.H + j, g.m);
    gs_norm_part(ws, R, a.acc + 4 * (j & 1));
}

__global__ void __launch_bounds__(kGsThreads) k_gs_update(GsArgs a)
{
    const GmresArgs &g = a.g;
    GmresState *st = g.st;
    const int2 jd = __ldcv(reinterpret_cast<const int2 *>(&st->j));
    const int j = jd.x;
    if (jd.y) return;
    int64_t r0;
    const int R = gs_rows(a, r0);
    __shared__ float2 ws[kGsMaxRows];
    __shared__ float2 hs[kMaxRestart + 1];
    for (int i = threadIdx.x; i < R; i += kGsThreads) ws[i] = g.w[r0 + i];
    const double hh = gs_load_h(g.H + j, g.m, hs, j);
    const double ww = __ldcg(a.acc + 4 * (j & 1));
    gs_update(a, ws, hs, R, r0, j);
    for (int i = threadIdx.x; i < R; i += kGsThreads) g.w[r0 + i] = ws[i];
    gs_norm_part(ws, R, a.acc + 4 * (j & 1) + 1);
    const bool need = gs_second_pass(ww, hh);
    // the decision for k_gs_finish (whose block 0 changes column j of H)
    if (blockIdx.x == 0 && threadIdx.x == 0) st->reorth = need;
    if (need) gs_dots_part(a, ws, R, r0, j, a.h2 + (int64_t)(j & 1) * (g.m + 1), 1);
}

// v_{j+1} = ws (unnormalised; its squared norm is in the sums) over the
// block's rows, with the next product's inputs; block 0 keeps the books of
// step j: H column j takes the second pass's h_2 (when there was one), and
// the other parity's sums are cleared for step j + 1.
__device__ void gs_store(const GsArgs &a, const float2 *ws, int R, int64_t r0, int j, bool need)
{
    const GmresArgs &g = a.g;
    GmresState *st = g.st;
    float2 *vn = g.V + (int64_t)(j + 1) * g.n;
    for (int i = threadIdx.x; i < R; i += kGsThreads) {
        const float2 xv = ws[i];
        vn[r0 + i] = xv;
        prep_store(a.next, r0 + i, xv);
    }
    if (blockIdx.x == 0) {
        const double2 *h2 = a.h2 + (int64_t)(j & 1) * (g.m + 1);
        if (need)
            for (int l = threadIdx.x; l <= j; l += kGsThreads) {
                double2 *hp = g.H + (int64_t)l * g.m + j;
                const double2 h = h2[l], h0 = *hp;
                *hp = make_double2(h0.x + h.x, h0.y + h.y);
            }
        double2 *h2n = a.h2 + (int64_t)((j + 1) & 1) * (g.m + 1);
        for (int l = threadIdx.x; l <= j + 1 && l <= g.m; l += kGsThreads) h2n[l] = make_double2(0.0, 0.0);
        if (threadIdx.x < 4) a.acc[4 * ((j + 1) & 1) + threadIdx.x] = 0.0;
        if (threadIdx.x == 0) st->n_reorth += need;
    }
}

__global__ void __launch_bounds__(kGsThreads) k_gs_finish(GsArgs a)
{
    const GmresArgs &g = a.g;
    GmresState *st = g.st;
    const int2 jd = __ldcv(reinterpret_cast<const int2 *>(&st->j));
    const int j = jd.x;
    if (jd.y) return;
    int64_t r0;
    const int R = gs_rows(a, r0);
    __shared__ float2 ws[kGsMaxRows];
    __shared__ float2 hs[kMaxRestart + 1];
    for (int i = threadIdx.x; i < R; i += kGsThreads) ws[i] = g.w[r0 + i];
    const bool need = __ldcv(&st->reorth) != 0;      // k_gs_update's decision
    if (need) {
        // second pass: w_2 = w_1 - V h_2 and its partial ||w_2||^2 (summed, as
        // every norm here: when w_1 is mostly rounding noise inside span(V),
        // ||w_1||^2 - |h_2|^2 would cancel to nothing)
        gs_load_h(a.h2 + (int64_t)(j & 1) * (g.m + 1), 1, hs, j);
        gs_update(a, ws, hs, R, r0, j);
        gs_norm_part(ws, R, a.acc + 4 * (j & 1) + 2);
    } else {
        __syncthreads();
    }
    gs_store(a, ws, R, r0, j, need);
}

// Givens step of the column the Gram-Schmidt kernels just formed (one warp).
__global__ void k_gm_givens(GmresArgs a)
{
    GmresState *st = a.st;
    if (*(volatile int *)&st->done) return;
    // ||v_{j+1}||^2 from the Gram-Schmidt sums (after the second pass when
    // there was one); k_gs_dots of step j + 1 scales v_{j+1} by it
    const int j = st->j;
    const double nn = __ldcg(a.gs_acc + 4 * (j & 1) + (*(volatile int *)&st->reorth ? 2 : 1));
    if (threadIdx.x == 0) st->nn = nn;
    gm_givens_warp(a, nn, j);
}

// st[0].skip_all = every plane's skip_prod (the product kernels of several
// right-hand sides skip only when all systems are done).
__global__ void k_gm_skip_all(GmresState *st, int nr)
{
    if (threadIdx.x != 0) return;
    int all = 1;
    for (int r = 0; r < nr; ++r) all &= __ldcv(&st[r].skip_prod) != 0;
    st[0].skip_all = all;
}

// The condition of the WHILE node that runs one Arnoldi cycle on the device
// (each body a few Arnoldi steps, then this kernel, after every step of the
// body, the Givens steps included, has finished): set to 1 while some plane
// is not done and fewer than max_bodies bodies have run, so the loop ends
// even if no plane ever reports done.
__global__ void k_gm_continue(cudaGraphConditionalHandle h, GmresState *st, int nr, int max_bodies)
{
    if (threadIdx.x != 0) return;
    int all = 1;
    for (int r = 0; r < nr; ++r) all &= __ldcv(&st[r].done) != 0;
    const int b = st[0].bodies + 1;
    st[0].bodies = b;
    cudaGraphSetConditional(h, (!all && b < max_bodies) ? 1u : 0u);
}

// Back substitution y = R^{-1} g over ncols columns (FP64), one warp:
// column-oriented, each step scales one entry by the reciprocal of its
// diagonal and the lanes update the rest.  The reciprocals 1 / R_ll are
// formed first, all in parallel, so the sequential chain of steps holds no
// division (FP64 division is a long dependent sequence on this part).  The
// triangle is staged in shared memory when it fits (smem_cols columns).
__global__ void k_gm_backsolve(const GmresState *st, const double2 *__restrict__ H, const double2 *__restrict__ g,
                               double2 *__restrict__ y, int m, int smem_cols)
{
    extern __shared__ double2 tri[];       // [nc][nc] when nc <= smem_cols (upper triangle filled)
    __shared__ double2 sv[kMaxRestart + 1];
    __shared__ double2 rinv[kMaxRestart + 1];
    const int nc = st->ncols;
    const int lane = threadIdx.x & 31;
    const bool in_smem = nc <= smem_cols;
    // staging by the whole block (its loads independent of one another),
    // then warp 0 alone runs the sequential steps
    for (int l = threadIdx.x; l < nc; l += blockDim.x) {
        sv[l] = g[l];
        const double2 d = H[(int64_t)l * m + l];
        const double inv = 1.0 / (d.x * d.x + d.y * d.y);
        rinv[l] = make_double2(d.x * inv, -d.y * inv);   // conj(d) / |d|^2
    }
    if (in_smem)
        for (int r = threadIdx.x / 32; r < nc; r += blockDim.x / 32)
            for (int c = r + lane; c < nc; c += 32) tri[r * nc + c] = H[(int64_t)r * m + c];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    for (int l = nc - 1; l >= 0; --l) {
        const double2 ri = rinv[l];
        const double2 sl = sv[l];
        const double2 yl = make_double2(sl.x * ri.x - sl.y * ri.y, sl.x * ri.y + sl.y * ri.x);
        if (lane == 0) y[l] = yl;
        for (int r = lane; r < l; r += 32) {
            const double2 h = in_smem ? tri[r * nc + l] : H[(int64_t)r * m + l];
            sv[r].x -= h.x * yl.x - h.y * yl.y;
            sv[r].y -= h.x * yl.y + h.y * yl.x;
        }
        __syncwarp();
    }
}

// x <- x + sum_l y_l V_l
__global__ void k_gm_xupdate(float2 *__restrict__ x, const float2 *__restrict__ V, int64_t n,
                             const GmresState *st, const double2 *__restrict__ y)
{
    __shared__ float2 ys[kMaxRestart + 1];
    const int nc = st->ncols;
    for (int l = threadIdx.x; l < nc; l += blockDim.x) ys[l] = make_float2((float)y[l].x, (float)y[l].y);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 acc = x[i];
    for (int l = 0; l < nc; ++l) acc = cfma(ys[l], V[(int64_t)l * n + i], acc);
    x[i] = acc;
}

// r = b - A x is formed by the caller; here: V_0 = r / ||r|| with ||r|| from
// normpart, and the cycle state is reset.
__global__ void k_gm_start(GmresState *st, float2 *__restrict__ V, const float2 *__restrict__ r, int64_t n,
                           const double *__restrict__ normpart, int nblk, double2 *__restrict__ g, int m, int first,
                           double *__restrict__ gs_acc, double2 *__restrict__ gs_h2)
{
    if (blockIdx.x == 0) {
        // the Gram-Schmidt sums of both parities (see k_gs_dots)
        for (int l = threadIdx.x; l < 2 * (m + 1); l += blockDim.x) gs_h2[l] = make_double2(0.0, 0.0);
        if (threadIdx.x < 8) gs_acc[threadIdx.x] = 0.0;
    }
    __shared__ double beta_s;
    if (threadIdx.x == 0) {
        double nn = 0.0;
        for (int b = 0; b < nblk; ++b) nn += normpart[b];
        beta_s = sqrt(nn);
    }
    __syncthreads();
    const double beta = beta_s;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) V[i] = beta > 0.0 ? cscale(r[i], (float)(1.0 / beta)) : make_float2(0.f, 0.f);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (first) st->bnorm = beta;
        st->beta = beta;
        st->j = 0;
        st->nn = 1.0;      // v_0 is stored normalised
        st->ncols = 0;
        st->done = 0;
        st->skip_prod = 0;
        st->converged = 0;
        st->bodies = 0;
        st->resid = st->bnorm > 0.0 ? beta / st->bnorm : 0.0;
        for (int l = 0; l <= m; ++l) g[l] = make_double2(0.0, 0.0);
        g[0] = make_double2(beta, 0.0);
        if (st->resid <= st->tol) { st->done = 1; st->converged = 1; }
    }
}

// partial ||r||^2 per block
__global__ void k_norm_part(const float2 *__restrict__ r, int64_t n, double *__restrict__ part)
{
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += (double)r[i].x * r[i].x + (double)r[i].y * r[i].y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

}  // namespace bem
