// Both plane sweeps of a one-box plane-by-plane LU (the coarse problem E of
// the two-level preconditioner, Eq. 2lvl) in ONE persistent cooperative
// launch, complex64.
//
// The multi-launch path spends three launches per plane (preparation, split-K
// product, reduction) on a few megabytes of work each, so on the coarse grid
// of the 112^3 workload (29 planes of 841 unknowns) launch latency and ramp-up
// are most of its time.  Here one CTA per SM walks all 2 bz - 1 steps:
//
//   1. rb = b_k - L_k y_{k-1} (forward) or U_k x_{k+1} (backward), one
//      thread per (node, rhs) over the whole grid;
//   -- grid barrier --
//   2. each CTA owns rpc consecutive rows of G_k = S_k^{-1}: rb is copied to
//      shared memory ([node][16 rhs], asynchronous 16-byte copies issued all
//      at once, so the L2 latency is paid once), the CTA's rows of G_k are
//      already there (odd row pitch: the two row groups a warp reads fall in
//      different banks), the 8 warps split the K range and every lane
//      accumulates 4 rows x 1 rhs; partial sums are added across the warps in
//      a fixed order, so results do not depend on scheduling;
//      y_k = G_k rb (forward) or x_k = y_k - G_k rb (backward);
//   3. cp.async prefetch of the next step's rows of G into shared memory,
//      which overlaps the barrier and the next preparation;
//   -- grid barrier --
//
// Data written inside the launch (rb, the local vector) is read with
// L2-only loads.  The grid barrier is a counter in global memory; its wait is
// bounded (about 0.3 s), checks the launch's error flag and, on expiry,
// records an error code and makes the CTA drain its copies and return, so a
// failure surfaces as HELM_ETIMEOUT instead of a hang.  A cooperative launch
// guarantees that all CTAs are resident at once.
#include <atomic>

#include "internal.h"

namespace {

constexpr int CO_THREADS = 256;
constexpr int CO_WARPS = CO_THREADS / 32;
constexpr int CO_RN = 16;     // right-hand sides per pass of the product
constexpr int CO_ROWS = 8;    // rows per tile: lanes 0-15 take rows 0-3, lanes 16-31 rows 4-7
constexpr uint32_t CO_WAIT_LIMIT = 1u << 22;
constexpr int CO_ERR_BARRIER = 4;

__device__ __forceinline__ c64 ldcg_c(const c64* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return mk<float>(v.x, v.y);
}
__device__ __forceinline__ void stcg_c(c64* p, c64 v) { __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y)); }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
// 16-byte copy through L2 only (the source is written by other CTAs of the same launch)
__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Grid barrier number n (1, 2, ...) over a counter zeroed before the launch; false when the
// bounded wait gave up or another CTA has recorded an error.
__device__ bool grid_sync(unsigned* bar, unsigned n, int* err, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = n * gridDim.x;
        int ok = 1;
        for (uint32_t i = 0;; ++i) {
            if (ld_acquire_u32(bar) >= target) break;
            if (i >= CO_WAIT_LIMIT || *reinterpret_cast<volatile int*>(err) != 0) {
                ok = 0;
                break;
            }
            if (i > 32) __nanosleep(64);
        }
        if (!ok) atomicCAS(err, 0, CO_ERR_BARRIER);
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__global__ void __launch_bounds__(CO_THREADS, 1) coarse_sweeps(const BoxInfo* __restrict__ boxes,
                                                                const c64* __restrict__ G,
                                                                const c64* __restrict__ coef, c64* loc, c64* rb,
                                                                int nrhs, int rpc, int gp, unsigned* bar, int* err) {
    extern __shared__ __align__(16) unsigned char co_smem[];
    __shared__ int s_ok;
    const BoxInfo B = boxes[0];
    const int m = B.m, bx = B.dims[0], by = B.dims[1], bz = B.dims[2];
    c64* rs = reinterpret_cast<c64*>(co_smem);   // [m][CO_RN]
    c64* gsm = rs + (size_t)CO_RN * m;             // [rpc][gp]: this CTA's rows of G_k
    c64* red = gsm + (size_t)rpc * gp;             // [CO_WARPS][CO_ROWS][CO_RN]
    const int row_a = blockIdx.x * rpc;
    const int nrow = max(0, min(m, row_a + rpc) - row_a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int rl = lane & 15, half = lane >> 4;
    const long long gt = (long long)blockIdx.x * CO_THREADS + threadIdx.x;
    const long long gstride = (long long)gridDim.x * CO_THREADS;
    const int ks = (m + CO_WARPS - 1) / CO_WARPS;
    const int q0 = min(m, wid * ks), q1 = min(m, q0 + ks);
    const int nsteps = 2 * bz - 1;
    // step t: forward plane k = t (t < bz), backward plane k = 2 bz - 2 - t
    auto plane_of = [&](int t) { return t < bz ? t : 2 * bz - 2 - t; };
    auto prefetch = [&](int t) {
        const c64* Gk = G + B.fac_off + (long long)plane_of(t) * B.pstride;
        for (int e = threadIdx.x; e < nrow * m; e += CO_THREADS) {
            const int i = e / m, q = e % m;
            cp_async8(gsm + (size_t)i * gp + q, Gk + (size_t)(row_a + i) * B.ld + q);
        }
        cp_async_commit();
    };
    unsigned nb = 0;
    prefetch(0);
    for (int t = 0; t < nsteps; ++t) {
        const bool fwd = t < bz;
        const int k = plane_of(t);
        const long long plane = B.loc_off + (long long)k * m;
        // 1. the prepared right-hand side of this step
        {
            const long long nbr = fwd ? plane - m : plane + m;
            const int off = fwd ? 0 : 18;
            const bool couple = !(fwd && k == 0);
            for (long long e = gt; e < (long long)m * nrhs; e += gstride) {
                const int p = (int)(e / nrhs), r = (int)(e % nrhs);
                c64 acc = fwd ? ldcg_c(loc + (plane + p) * nrhs + r) : mk<float>(0, 0);
                if (couple) {
                    // the 18 loads first (one L2 latency): couplings that leave the grid have zero coefficients,
                    // so their neighbour index is clamped
                    const int px = p % bx, py = p / bx;
                    const c64* cp = coef + (plane + p) * 27 + off;
                    c64 c[9], v[9];
#pragma unroll
                    for (int d = 0; d < 9; ++d) {
                        const int qx = min(max(px + d % 3 - 1, 0), bx - 1), qy = min(max(py + d / 3 - 1, 0), by - 1);
                        c[d] = cp[d];
                        v[d] = ldcg_c(loc + (nbr + qy * bx + qx) * nrhs + r);
                    }
#pragma unroll
                    for (int d = 0; d < 9; ++d) {
                        if (fwd) {
                            acc.x -= c[d].x * v[d].x - c[d].y * v[d].y;
                            acc.y -= c[d].x * v[d].y + c[d].y * v[d].x;
                        } else {
                            cmac(acc, c[d], v[d]);
                        }
                    }
                }
                stcg_c(rb + e, acc);
            }
        }
        if (!grid_sync(bar, ++nb, err, &s_ok)) {
            cp_async_wait_all();
            return;
        }
        // 2. this CTA's rows of y_k = G_k rb (forward) or x_k = y_k - G_k rb (backward)
        cp_async_wait_all();
        __syncthreads();
        for (int r0 = 0; r0 < nrhs; r0 += CO_RN) {
            const int rn = min(CO_RN, nrhs - r0);
            const int npair = rn >> 1;   // nrhs is even: whole column pairs, 16-byte aligned
            for (int e = threadIdx.x; e < m * npair; e += CO_THREADS) {
                const int q = e / npair, pr = e % npair;
                cp_async16_cg(rs + (size_t)q * CO_RN + 2 * pr, rb + (size_t)q * nrhs + r0 + 2 * pr);
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
            for (int i0 = 0; i0 < nrow; i0 += CO_ROWS) {
                c64 acc[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i] = mk<float>(0, 0);
                const int rbase = i0 + half * 4;   // first of this lane's 4 rows (tile-local)
                // lanes rl >= rn accumulate values that are never written out
                const c64* bcol = rs + rl;
                // every lane runs the same loop: rows past the CTA's last are clamped onto it (their sums are
                // never written), so the two half-warps never diverge
                const c64* g[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) g[i] = gsm + (size_t)min(rbase + i, nrow - 1) * gp;
#pragma unroll 4
                for (int q = q0; q < q1; ++q) {
                    const c64 bv = bcol[(size_t)q * CO_RN];
#pragma unroll
                    for (int i = 0; i < 4; ++i) cmac(acc[i], g[i][q], bv);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) red[(wid * CO_ROWS + half * 4 + i) * CO_RN + rl] = acc[i];
                __syncthreads();
                if (threadIdx.x < CO_ROWS * CO_RN) {
                    const int i = threadIdx.x / CO_RN, r = threadIdx.x % CO_RN;
                    if (i0 + i < nrow && r < rn) {
                        c64 sum = mk<float>(0, 0);
                        for (int w = 0; w < CO_WARPS; ++w) sum = sum + red[(w * CO_ROWS + i) * CO_RN + r];
                        c64* dst = loc + (plane + row_a + i0 + i) * nrhs + r0 + r;
                        stcg_c(dst, fwd ? sum : ldcg_c(dst) - sum);
                    }
                }
                __syncthreads();
            }
        }
        // 3. the next step's rows of G, in flight while the grid synchronises
        if (t + 1 < nsteps) prefetch(t + 1);
        if (!grid_sync(bar, ++nb, err, &s_ok)) {
            cp_async_wait_all();
            return;
        }
    }
}

struct CoopPlan {
    bool ok = false;
    int grid = 0, rpc = 0, gp = 0;
    size_t smem = 0;
};

CoopPlan plan_for(helm_ctx ctx, const PlaneSet& P) {
    CoopPlan c;
    if (P.nbox != 1 || P.prec == HELM_PREC_FP64 || P.prec == HELM_PREC_BF16 || P.padded) return c;
    static std::atomic<int> coop_attr{-1};
    if (coop_attr.load(std::memory_order_acquire) < 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, ctx->device);
        coop_attr.store(v, std::memory_order_release);
    }
    if (!coop_attr.load(std::memory_order_acquire) || ctx->sm_count <= 0) return c;
    const int m = P.hbox[0].m;
    c.grid = ctx->sm_count;
    c.rpc = (m + c.grid - 1) / c.grid;
    c.gp = m | 1;
    c.smem = ((size_t)CO_RN * m + (size_t)c.rpc * c.gp + (size_t)CO_WARPS * CO_ROWS * CO_RN) * sizeof(c64);
    if (c.smem > 200 * 1024) return c;
    static std::atomic<bool> attr{false};
    if (!attr.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(coarse_sweeps, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr.store(true, std::memory_order_release);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_sweeps, CO_THREADS, c.smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return c;
    }
    c.ok = true;
    return c;
}

}  // namespace

// Both sweeps of a one-box complex64 plane set in one cooperative launch.  rbuf must hold
// m * nrhs complex64 entries followed by a 4-byte barrier counter (the one-box scratch is
// sized 9 planes deep, far more).  *done = false when the set or the device does not qualify
// (the caller then runs the multi-launch sweeps).
helm_status planeset_solve_coop(helm_ctx ctx, const PlaneSet& P, c64* loc, c64* rbuf, int nrhs, cudaStream_t st,
                                int* err, bool* done) {
    *done = false;
    if (!err || nrhs <= 0 || nrhs % 2) return HELM_OK;   // column pairs: 16-byte copies
    const CoopPlan c = plan_for(ctx, P);
    if (!c.ok) return HELM_OK;
    const BoxInfo& b = P.hbox[0];
    const long long m = b.m;
    unsigned* bar = reinterpret_cast<unsigned*>(rbuf + m * nrhs);
    HELM_CUDA(ctx, cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    const BoxInfo* dbox = P.dbox;
    const c64* G = (const c64*)P.G;
    const c64* coef = (const c64*)P.coef;
    int nr = nrhs, rpc = c.rpc, gp = c.gp;
    void* args[] = {(void*)&dbox, (void*)&G, (void*)&coef, (void*)&loc, (void*)&rbuf, (void*)&nr,
                    (void*)&rpc,  (void*)&gp, (void*)&bar, (void*)&err};
    // algorithmic bytes: every factor once, the local vector read and written per step, the
    // coefficient rows of the couplings
    const double es = sizeof(c64);
    const double bytes = (2.0 * b.dims[2] - 1.0) * ((double)m * m * es + 3.0 * m * nrhs * es + 9.0 * m * es);
    const int tk = prof_begin(ctx, "coarse_sweep");
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)coarse_sweeps, dim3(c.grid), dim3(CO_THREADS), args,
                                                c.smem, st);
    prof_end(ctx, tk, bytes);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cooperative coarse sweeps");
    ctx->launches += 1;
    *done = true;
    return HELM_OK;
}
