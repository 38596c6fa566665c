// Plane sweeps of the ORAS local solves on the 5th-generation tensor cores
// (tcgen05, kind::tf32, FP32 accumulation in TMEM, operands staged by TMA).
//
// Each sweep step multiplies, for every box, the dense plane inverse
// G_k = S_k^{-1} (m x m complex, stored interleaved (re, im) with row pitch
// ld) by the prepared m x nrhs complex block R.  The complex product is one
// real GEMM: row i of G read as 2m floats (re, im, re, im, ...) is a K-major
// A operand with K = 2m, and the B operand is the 2x2 real embedding of R,
// stored transposed (N x K, K contiguous):
//   B^T[2r][2p] = Re R[p][r],  B^T[2r][2p+1] = -Im R[p][r],
//   B^T[2r+1][2p] = Im R[p][r], B^T[2r+1][2p+1] = Re R[p][r],
// so D[i][2r] = Re (G R)[i][r] and D[i][2r+1] = Im (G R)[i][r].
//
// Two operand types: TF32 (complex64 factors read as fp32, kind::tf32, K = 8 per MMA) and
// BF16 (factors stored as bfloat16 pairs, kind::f16, K = 16 per MMA); both accumulate in FP32.
//
// tc_prep builds B^T for the step (FWD: R = b_k - L_k y_{k-1}; BWD:
// R = U_k x_{k+1}).  tc_sweep_gemm: one CTA per (128-row tile, box), four
// warps; warp 0 lane 0 issues the TMA loads of 128 x 32-float A tiles and
// N x 32-float B tiles (128-byte swizzle) into a 5-stage mbarrier ring, warp 1
// lane 0 issues 4 MMAs (M = 128, N = NPAD, K = 8) per stage and commits each
// stage back to the producer, and all four warps read the accumulator from
// TMEM (thread t <-> row t) and write y_k (FWD) or x_k = y_k - D (BWD).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <vector>

#include "internal.h"
#include "tc.cuh"

namespace {

constexpr int TC_BM = 128;

// element traits: operands per 128-byte swizzled row, MMA K, conversion from float
template <typename E> struct Elem;
template <> struct Elem<float> {
    static constexpr int BK = 32;
    static constexpr int MMA_K = 8;
    static __device__ __forceinline__ float from(float v) { return v; }
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr int BK = 64;
    static constexpr int MMA_K = 16;
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};

// Tiles of 32 plane nodes x nrhs: values formed with the rhs index fastest (coalesced reads of
// the [node][rhs] local vectors), transposed through shared memory, written as B^T rows.
constexpr int PREP_TP = 32;

template <typename E>
__global__ void __launch_bounds__(256) tc_prep(const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef,
                                               const c64* __restrict__ lb, const c64* __restrict__ loc,
                                               E* __restrict__ bt, int ld2, int npad, int nrhs, int s, int fwd) {
    __shared__ c64 tile[128 * (PREP_TP + 1)];
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m, bz = B.dims[2], bx = B.dims[0], by = B.dims[1];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz) return;
    if (!fwd && k == bz - 1) return;
    const long long plane = B.loc_off + (long long)k * m;
    const long long nbr = fwd ? plane - m : plane + m;
    const int off = fwd ? 0 : 18;
    E* bb = bt + (size_t)blockIdx.y * npad * ld2;
    for (int p0 = blockIdx.x * PREP_TP; p0 < m; p0 += gridDim.x * PREP_TP) {
        for (int e = threadIdx.x; e < PREP_TP * nrhs; e += blockDim.x) {
            const int pl = e / nrhs, r = e % nrhs, p = p0 + pl;
            c64 acc = mk<float>(0, 0);
            if (p < m) {
                if (fwd) acc = lb[(plane + p) * nrhs + r];
                if (!(fwd && k == 0)) {
                    const int px = p % bx, py = p / bx;
                    const c64* cp = coef + (plane + p) * 27 + off;
#pragma unroll
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int qy = py + dy;
                        if (qy < 0 || qy >= by) continue;
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int qx = px + dx;
                            if (qx < 0 || qx >= bx) continue;
                            const c64 c = cp[(dy + 1) * 3 + (dx + 1)];
                            const c64 v = loc[(nbr + qy * bx + qx) * nrhs + r];
                            if (fwd) {
                                acc.x -= c.x * v.x - c.y * v.y;
                                acc.y -= c.x * v.y + c.y * v.x;
                            } else {
                                cmac(acc, c, v);
                            }
                        }
                    }
                }
            }
            tile[r * (PREP_TP + 1) + pl] = acc;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nrhs * PREP_TP; e += blockDim.x) {
            const int r = e / PREP_TP, pl = e % PREP_TP, p = p0 + pl;
            if (p < m) {
                const c64 a = tile[r * (PREP_TP + 1) + pl];
                E* re_row = bb + (size_t)(2 * r) * ld2 + 2 * p;
                E* im_row = bb + (size_t)(2 * r + 1) * ld2 + 2 * p;
                re_row[0] = Elem<E>::from(a.x);
                re_row[1] = Elem<E>::from(-a.y);
                im_row[0] = Elem<E>::from(a.y);
                im_row[1] = Elem<E>::from(a.x);
            }
        }
        __syncthreads();
    }
}

// Vectorised variant for an even column count: thread per (plane node, column pair), the pair
// fastest, so each neighbour load of a warp is one 16-byte vector per thread over contiguous memory
// (512 threads: one item each at 16 columns, so every thread waits on one round of loads);
// the values of a tile of PREP2_TP nodes are transposed through shared memory ([nrhs][PREP2_TP + 1])
// and written as (re, -im) and (im, re) pairs along rows 2r and 2r+1 of B^T.
constexpr int PREP2_TP = 64;

template <typename E> struct Pair2;
template <> struct Pair2<float> {
    typedef float2 type;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Pair2<__nv_bfloat16> {
    typedef __nv_bfloat162 type;
    static __device__ __forceinline__ __nv_bfloat162 make(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

// One tile of tpn plane nodes of box B (index box) for step s: thread per (node, column pair), any
// block size; tile is [nrhs][tpn + 1] complex64 in shared memory.
template <typename E, bool CG = false>
__device__ __forceinline__ void prep_tile(const BoxInfo& B, int box, int t, int tpn, const c64* __restrict__ coef,
                                          const c64* __restrict__ lb, const c64* __restrict__ loc,
                                          E* __restrict__ bt, int ld2, int npad, int nrhs, int s, int fwd, c64* tile) {
    const int m = B.m, bz = B.dims[2], bx = B.dims[0], by = B.dims[1];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz || (!fwd && k == bz - 1)) return;
    const int p0 = t * tpn;
    if (p0 >= m) return;
    const int npair = nrhs >> 1;
    const long long plane = B.loc_off + (long long)k * m;
    const long long nbr = fwd ? plane - m : plane + m;
    const int off = fwd ? 0 : 18;
    const bool couple = !(fwd && k == 0);
    for (int e = threadIdx.x; e < tpn * npair; e += blockDim.x) {
        const int pr = e % npair, pl = e / npair, p = p0 + pl;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);   // columns 2 pr and 2 pr + 1: (re, im, re, im)
        if (p < m) {
            if (fwd) acc = *reinterpret_cast<const float4*>(lb + (plane + p) * nrhs + 2 * pr);
            if (couple) {
                // all 18 loads first (one memory latency, not nine): a coupling that points out of the box
                // has a zero coefficient (the fold moved it), so its neighbour index is clamped into the box
                const int px = p % bx, py = p / bx;
                const c64* cp = coef + (plane + p) * 27 + off;
                c64 c[9];
                float4 v[9];
#pragma unroll
                for (int d = 0; d < 9; ++d) {
                    const int qx = min(max(px + d % 3 - 1, 0), bx - 1), qy = min(max(py + d / 3 - 1, 0), by - 1);
                    c[d] = cp[d];
                    const float4* src = reinterpret_cast<const float4*>(loc + (nbr + qy * bx + qx) * nrhs + 2 * pr);
                    v[d] = CG ? __ldcg(src) : *src;
                }
#pragma unroll
                for (int d = 0; d < 9; ++d) {
                    // forward: acc -= c v; backward: acc += c v
                    const float sr = fwd ? -c[d].x : c[d].x, si = fwd ? -c[d].y : c[d].y;
                    acc.x = fmaf(sr, v[d].x, fmaf(-si, v[d].y, acc.x));
                    acc.y = fmaf(sr, v[d].y, fmaf(si, v[d].x, acc.y));
                    acc.z = fmaf(sr, v[d].z, fmaf(-si, v[d].w, acc.z));
                    acc.w = fmaf(sr, v[d].w, fmaf(si, v[d].z, acc.w));
                }
            }
        }
        tile[(2 * pr) * (tpn + 1) + pl] = mk<float>(acc.x, acc.y);
        tile[(2 * pr + 1) * (tpn + 1) + pl] = mk<float>(acc.z, acc.w);
    }
    __syncthreads();
    E* bb = bt + (size_t)box * npad * ld2;
    typedef typename Pair2<E>::type P2;
    for (int e = threadIdx.x; e < nrhs * tpn; e += blockDim.x) {
        const int r = e / tpn, pl = e % tpn, p = p0 + pl;
        if (p >= m) continue;
        const c64 a = tile[r * (tpn + 1) + pl];
        *reinterpret_cast<P2*>(bb + (size_t)(2 * r) * ld2 + 2 * p) = Pair2<E>::make(a.x, -a.y);
        *reinterpret_cast<P2*>(bb + (size_t)(2 * r + 1) * ld2 + 2 * p) = Pair2<E>::make(a.y, a.x);
    }
}

// prep_tile for the persistent sweep.  One round of asynchronous copies (all in flight at once) brings into
// shared memory the tile's neighbour rows (a contiguous stretch of the neighbour plane, read from L2),
// its 9 coupling coefficients per node and, forward, its right-hand sides; every value is then formed
// from shared memory with the same operations in the same order as prep_tile, by a thread per
// (node, column pair) with the node fastest, and written straight into its four B^T rows (coalesced
// along the node).  Node rows are padded to one float4 more than a chunk against bank conflicts.  When
// all column pairs do not fit in smem_bytes, they are staged and formed in chunks (the largest halving
// of the pair count that fits; the coefficients are staged once).  Plane 0 of the forward sweep (no
// coupling) and tiles whose data exceed smem_bytes even for one pair use prep_tile.
template <typename E>
__device__ __forceinline__ void prep_tile_staged(const BoxInfo& B, int box, int t, int tpn,
                                                 const c64* __restrict__ coef, const c64* __restrict__ lb,
                                                 const c64* __restrict__ loc, E* __restrict__ bt, int ld2, int npad,
                                                 int nrhs, int s, int fwd, unsigned char* smem, int smem_bytes) {
    const int m = B.m, bz = B.dims[2], bx = B.dims[0], by = B.dims[1];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz || (!fwd && k == bz - 1)) return;
    const int p0 = t * tpn;
    if (p0 >= m) return;
    const int np = min(tpn, m - p0);
    const int r_lo = max(p0 / bx - 1, 0), r_hi = min((p0 + np - 1) / bx + 1, by - 1);
    const int ns = (r_hi - r_lo + 1) * bx;   // staged neighbour nodes
    const int npair = nrhs >> 1;
    const int nl = fwd ? np : 0;              // staged right-hand-side nodes
    auto need = [&](int cp) {
        return ((size_t)ns + nl) * (cp + 1) * sizeof(float4) + (size_t)np * 9 * sizeof(float2);
    };
    int cp = npair;
    while (cp > 1 && need(cp) > (size_t)smem_bytes) cp = (cp + 1) >> 1;
    if ((fwd && k == 0) || need(cp) > (size_t)smem_bytes) {
        prep_tile<E, true>(B, box, t, tpn, coef, lb, loc, bt, ld2, npad, nrhs, s, fwd, reinterpret_cast<c64*>(smem));
        return;
    }
    const int sp = cp + 1;
    const long long plane = B.loc_off + (long long)k * m;
    const long long nbr = fwd ? plane - m : plane + m;
    const int off = fwd ? 0 : 18;
    float4* stg = reinterpret_cast<float4*>(smem);            // [ns][sp]
    float4* lbs = stg + (size_t)ns * sp;                        // [np][sp] (forward)
    float2* cfs = reinterpret_cast<float2*>(lbs + (size_t)nl * sp);   // [np][9]
    const float4* nsrc = reinterpret_cast<const float4*>(loc + (nbr + (long long)r_lo * bx) * nrhs);
    const float4* lsrc = reinterpret_cast<const float4*>(lb + (plane + p0) * nrhs);
    const float2* csrc = reinterpret_cast<const float2*>(coef + (plane + p0) * 27 + off);
    E* bb = bt + (size_t)box * npad * ld2;
    typedef typename Pair2<E>::type P2;
    for (int c0 = 0; c0 < npair; c0 += cp) {
        const int cw = min(cp, npair - c0);
        const int n1 = ns * cw, n2 = nl * cw, n3 = c0 == 0 ? np * 9 : 0;
        if (c0 > 0) __syncthreads();   // the previous chunk's values are read before they are replaced
        for (int e = threadIdx.x; e < n1; e += blockDim.x)
            tc::cp_async16(stg + (e / cw) * sp + e % cw, nsrc + (long long)(e / cw) * npair + c0 + e % cw);
        for (int e = threadIdx.x; e < n2; e += blockDim.x)
            tc::cp_async16(lbs + (e / cw) * sp + e % cw, lsrc + (long long)(e / cw) * npair + c0 + e % cw);
        for (int e = threadIdx.x; e < n3; e += blockDim.x) tc::cp_async8(cfs + e, csrc + (e / 9) * 27 + e % 9);
        tc::cp_async_wait_all();
        __syncthreads();
        for (int e = threadIdx.x; e < np * cw; e += blockDim.x) {
            const int pl = e % np, pc = e / np, pr = c0 + pc, p = p0 + pl;
            float4 acc = fwd ? lbs[pl * sp + pc] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int px = p % bx, py = p / bx;
            float2 c[9];
            float4 v[9];
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                const int qx = min(max(px + d % 3 - 1, 0), bx - 1), qy = min(max(py + d / 3 - 1, 0), by - 1);
                c[d] = cfs[pl * 9 + d];
                v[d] = stg[((qy - r_lo) * bx + qx) * sp + pc];
            }
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                const float sr = fwd ? -c[d].x : c[d].x, si = fwd ? -c[d].y : c[d].y;
                acc.x = fmaf(sr, v[d].x, fmaf(-si, v[d].y, acc.x));
                acc.y = fmaf(sr, v[d].y, fmaf(si, v[d].x, acc.y));
                acc.z = fmaf(sr, v[d].z, fmaf(-si, v[d].w, acc.z));
                acc.w = fmaf(sr, v[d].w, fmaf(si, v[d].z, acc.w));
            }
            // columns 2 pr (acc.x, acc.y) and 2 pr + 1 (acc.z, acc.w): B^T rows 4 pr .. 4 pr + 3 at entries 2p, 2p + 1
            E* row = bb + (size_t)(4 * pr) * ld2 + 2 * p;
            *reinterpret_cast<P2*>(row) = Pair2<E>::make(acc.x, -acc.y);
            *reinterpret_cast<P2*>(row + ld2) = Pair2<E>::make(acc.y, acc.x);
            *reinterpret_cast<P2*>(row + 2 * (size_t)ld2) = Pair2<E>::make(acc.z, -acc.w);
            *reinterpret_cast<P2*>(row + 3 * (size_t)ld2) = Pair2<E>::make(acc.w, acc.z);
        }
    }
}

template <typename E>
__global__ void __launch_bounds__(512) tc_prep2(const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef,
                                                const c64* __restrict__ lb, const c64* __restrict__ loc,
                                                E* __restrict__ bt, int ld2, int npad, int nrhs, int s, int fwd) {
    extern __shared__ __align__(16) unsigned char prep_smem[];
    const BoxInfo B = boxes[blockIdx.y];
    prep_tile<E>(B, blockIdx.y, blockIdx.x, PREP2_TP, coef, lb, loc, bt, ld2, npad, nrhs, s, fwd,
                 reinterpret_cast<c64*>(prep_smem));
}

template <typename E, int NPAD, int NST>
struct TcCfg {
    static constexpr int BK = Elem<E>::BK;
    static constexpr int A_BYTES = TC_BM * 128;
    static constexpr int B_BYTES = NPAD * 128;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = NST;
    static constexpr uint32_t TCOLS = NPAD <= 32 ? 32 : (NPAD <= 64 ? 64 : (NPAD <= 128 ? 128 : 256));
    static constexpr int SMEM = STAGES * STAGE + (2 * STAGES + 1) * 8 + 16 + 1024;
};

// Position of a CTA in its operand ring: chunks issued so far (stage = g mod NST, phase = g / NST)
// and the phase of the accumulator-ready barrier.  Carried across the row tiles a persistent CTA takes.
struct Ring {
    uint32_t g = 0;
    uint32_t dphase = 0;
};

// mbarriers, tensor-map prefetch and the TMEM accumulator of one CTA; returns the TMEM address.
template <typename E, int NPAD, int NST>
__device__ __forceinline__ uint32_t gemm_setup(const CUtensorMap* mapA, const CUtensorMap* mapA32,
                                               const CUtensorMap* mapB, unsigned char* base) {
    using Cfg = TcCfg<E, NPAD, NST>;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + NST * Cfg::STAGE);
    uint64_t* empty = full + NST;
    uint64_t* done = empty + NST;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    if (threadIdx.x == 0) {
        for (int i = 0; i < NST; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::prefetch_tmap(mapA);
        tc::prefetch_tmap(mapA32);
        tc::prefetch_tmap(mapB);
    }
    if ((threadIdx.x >> 5) == 1) {
        tc::tmem_alloc(tmem_slot, Cfg::TCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return *tmem_slot;
}

template <typename E, int NPAD, int NST>
__device__ __forceinline__ void gemm_teardown(uint32_t tmem) {
    using Cfg = TcCfg<E, NPAD, NST>;
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, Cfg::TCOLS);
    }
}

// Row tile t of box (index box) at plane k: y_k rows (forward) or x_k = y_k - G_k R rows (backward).
// base: 1024-aligned dynamic shared memory (NST stages, then the barriers).  All 128 threads call it;
// it ends with a CTA barrier after the accumulator has been read, so the next tile may reuse TMEM and
// the stages.  A wait that gives up leaves an error code in *err.
template <typename E, int NPAD, int NST>
__device__ __forceinline__ void gemm_core(const CUtensorMap* mapA, const CUtensorMap* mapA32, const CUtensorMap* mapB,
                                          const BoxInfo& B, int box, int t, int k, c64* __restrict__ loc, int nrhs,
                                          int fwd, int nkc, int* __restrict__ err, unsigned char* base, uint32_t tmem,
                                          Ring& R) {
    using Cfg = TcCfg<E, NPAD, NST>;
    constexpr int TC_BK = Cfg::BK;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + NST * Cfg::STAGE);
    uint64_t* empty = full + NST;
    uint64_t* done = empty + NST;
    const int m = B.m;
    const int row0 = t * TC_BM;
    const int nK = (2 * m + TC_BK - 1) / TC_BK;
    const int plane = B.plane0 + k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    int issued = 0;   // thread 0: chunks whose loads it issued for this tile
    if (warp == 0 && lane == 0) {
        // TMA producer.  A tile (rows row0.., chunk kc): 16 KB contiguous in the tile layout; the last,
        // partial row tile of a box loads only its 32-row groups that hold rows < m (the rest of the
        // shared tile keeps stale values, which only reach accumulator rows that are never stored)
        const int rows = min(TC_BM, m - row0);
        const int nsub = rows >= TC_BM ? 0 : (rows + 31) / 32;
        const uint32_t a_bytes = nsub ? (uint32_t)nsub * 32 * 128 : (uint32_t)Cfg::A_BYTES;
        for (int kc = 0; kc < nK; ++kc) {
            const uint32_t gi = R.g + kc;
            const int st = gi % NST;
            if (gi >= NST && !tc::mbar_wait(&empty[st], ((gi / NST) - 1) & 1, err, 1)) break;
            unsigned char* sa = base + st * Cfg::STAGE;
            tc::mbar_arrive_expect_tx(&full[st], a_bytes + Cfg::B_BYTES);
            const int line = (t * nkc + kc) * TC_BM;
            if (nsub == 0)
                tc::tma_load_3d(sa, mapA, 0, line, plane, &full[st]);
            else
                for (int q = 0; q < nsub; ++q) tc::tma_load_3d(sa + q * 4096, mapA32, 0, line + 32 * q, plane, &full[st]);
            tc::tma_load_3d(sa + Cfg::A_BYTES, mapB, kc * TC_BK, 0, box, &full[st]);
            ++issued;
        }
        if (issued < nK) {
            // gave up: let the copies already issued land (bounded) before the stages are left
            for (int kc = max(0, issued - NST); kc < issued; ++kc) {
                const uint32_t gi = R.g + kc;
                tc::mbar_drain(&full[gi % NST], (gi / NST) & 1);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr bool BF = sizeof(E) == 2;
        constexpr uint32_t idesc = BF ? tc::idesc_bf16(TC_BM, NPAD) : tc::idesc_tf32(TC_BM, NPAD);
        for (int kc = 0; kc < nK; ++kc) {
            const uint32_t gi = R.g + kc;
            const int st = gi % NST;
            if (!tc::mbar_wait(&full[st], (gi / NST) & 1, err, 2)) break;
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_u32(base + st * Cfg::STAGE);
            const uint32_t sb = sa + Cfg::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / Elem<E>::MMA_K; ++kk) {
                const uint64_t ad = tc::desc_k_sw128(sa + kk * 32), bd = tc::desc_k_sw128(sb + kk * 32);
                if (BF) tc::mma_f16(tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                else tc::mma_tf32(tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(done);
    }
    __syncwarp();

    // epilogue: thread t of warp w owns TMEM lane 32 w + t = output row row0 + 32 w + t
    const bool ok = tc::mbar_wait(done, R.dphase, err, 3);
    // gave up (here or elsewhere): the MMAs already issued still write TMEM and the loads already issued
    // still land in the stages, so wait for both (bounded, ignoring the flag) before TMEM or the stages
    // are reused or freed.  `done` is always committed once the issuer has left its loop.
    if (!ok) tc::mbar_drain(done, R.dphase);
    tc::fence_after_sync();
    if (!ok && threadIdx.x == 0)
        for (int kc = max(0, issued - NST); kc < issued; ++kc) {
            const uint32_t gi = R.g + kc;
            tc::mbar_drain(&full[gi % NST], (gi / NST) & 1);
        }
    if (ok) {
        const int row = row0 + warp * 32 + lane;
        c64* dst = loc + (B.loc_off + (long long)k * m + row) * nrhs;
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 32) {
            uint32_t v[32];
            tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            tc::tmem_ld_wait();
            if (row < m) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int r = c0 / 2 + q;
                    if (r < nrhs) {
                        const float re = __uint_as_float(v[2 * q]), im = __uint_as_float(v[2 * q + 1]);
                        if (fwd) {
                            dst[r] = mk<float>(re, im);
                        } else {
                            // y_k may come from another CTA of a persistent launch: read it from L2
                            const float2 o = __ldcg(reinterpret_cast<const float2*>(dst + r));
                            dst[r] = mk<float>(o.x - re, o.y - im);
                        }
                    }
                }
            }
        }
    }
    R.g += nK;
    R.dphase ^= 1u;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~static_cast<uintptr_t>(1023));
}

template <typename E, int NPAD, int NST>
__global__ void __launch_bounds__(128, 1) tc_sweep_gemm(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapA32,
                                                        const __grid_constant__ CUtensorMap mapB,
                                                        const BoxInfo* __restrict__ boxes, c64* __restrict__ loc,
                                                        int nrhs, int s, int fwd, int nkc, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const BoxInfo B = boxes[blockIdx.y];
    const int bz = B.dims[2];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz || (!fwd && k == bz - 1) || (int)blockIdx.x * TC_BM >= B.m) return;
    unsigned char* base = align1024(smem_raw);
    const uint32_t tmem = gemm_setup<E, NPAD, NST>(&mapA, &mapA32, &mapB, base);
    Ring R;
    gemm_core<E, NPAD, NST>(&mapA, &mapA32, &mapB, B, blockIdx.y, blockIdx.x, k, loc, nrhs, fwd, nkc, err, base, tmem,
                            R);
    gemm_teardown<E, NPAD, NST>(tmem);
}

// ---------------------------------------------------------------- persistent dataflow sweep
//
// Both sweeps of every box in one launch.  Box b runs the chain of operations
//   prep(0), gemm(0), prep(1), gemm(1), ..., prep(2 n_z - 2), gemm(2 n_z - 2)
// (steps 0..n_z-1 forward, then n_z-1 backward steps), each operation split into items: row tiles of
// 128 for a product, tiles of tpn nodes (the queue's tpn, 128) for an operand preparation.  Items wait in a queue: the
// preparations of step 0 are there at the start (init), and the CTA that completes the last item of an
// operation appends the items of the box's next operation.  Each CTA takes the next queue slot, waits
// until that slot has been written, runs the item and counts it done.  A slot is written only after
// everything its item depends on has completed, and a CTA waits only for slots, so as long as one CTA
// runs, work advances (no co-residency is assumed).  Every wait is bounded (HELM_ETIMEOUT).
//
// Ordering across CTAs: an item's global writes (loc, the B operand) are made visible with a gpu-scope
// fence (and a generic-to-async proxy fence, since the next product reads the B operand by TMA) before
// its completion is counted; queue slots are published with release stores and read with acquire loads;
// values other CTAs wrote in this launch are read through L2 (ld.cg), never a stale L1 line.
constexpr int FLOW_TPN_MAX = 128;

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
    int old;
    asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

constexpr int FLOW_QT = 96;   // the thread that handles the queue (warp 3, lane 0)

// A queue item packed in one int: box (11 bits), operation (10 bits), tile (10 bits), stored + 1 so that a
// published slot is never 0 (the flag of a slot is its item).
__device__ __host__ __forceinline__ int flow_pack(int box, int j, int t) { return ((box << 20) | (j << 10) | t) + 1; }

// The item in queue slot `slot` (bounded wait until it has been published); x = -1 when the queue is
// exhausted or a wait anywhere gave up.
// wait_ns bounds the wait (the context's flow_wait_us knob, 2 s by default); 0 gives up at the first
// unpublished poll.
__device__ __forceinline__ int4 flow_fetch(int slot, const int* __restrict__ init, int ninit, const int* flag, int total,
                                           int* err, uint64_t wait_ns) {
    if (slot >= total || *reinterpret_cast<volatile int*>(err) != 0) return make_int4(-1, 0, 0, 0);
    int v = 0;
    if (slot < ninit) {
        v = init[slot];
    } else {
        const int q = slot - ninit;
        const uint64_t t0 = global_ns();
        for (uint32_t i = 0;; ++i) {
            if ((v = ld_acquire_gpu(flag + q)) != 0) break;
            if ((i & 255) == 255 || wait_ns == 0) {
                if (*reinterpret_cast<volatile int*>(err) != 0) return make_int4(-1, 0, 0, 0);
                if (global_ns() - t0 >= wait_ns) {
                    atomicExch(err, 4);
                    return make_int4(-1, 0, 0, 0);
                }
            }
            __nanosleep(32);
        }
    }
    --v;
    return make_int4(v >> 20, (v >> 10) & 1023, v & 1023, 0);
}

// ops in box b's chain, and the items of operation j
__device__ __host__ __forceinline__ int flow_chain(int bz) { return 2 * (2 * bz - 1); }
__device__ __host__ __forceinline__ int flow_tiles(int m, int j, int tpn) {
    return (j & 1) ? (m + TC_BM - 1) / TC_BM : (m + tpn - 1) / tpn;
}

template <typename E, int NPAD, int NST>
__global__ void __launch_bounds__(128, 1) tc_sweep_flow(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapA32,
                                                        const __grid_constant__ CUtensorMap mapB,
                                                        const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef,
                                                        const c64* __restrict__ lb, c64* __restrict__ loc,
                                                        E* __restrict__ bt, int ld2, int nrhs, int nkc,
                                                        const int* __restrict__ init, int ninit, int* flag, int total,
                                                        int* ctl, int* __restrict__ err, uint64_t wait_ns, int tpn) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int4 cur;
    unsigned char* base = align1024(smem_raw);
    int* head = ctl;
    int* tail = ctl + 1;
    int* cnt = ctl + 2;   // per box: items of its current operation completed
    const uint32_t tmem = gemm_setup<E, NPAD, NST>(&mapA, &mapA32, &mapB, base);
    Ring R;
    // Queue work is done by thread FLOW_QT (idle in a product's main loop): it takes the next slot while
    // the current item runs, and after the item counts it done, publishes the box's next operation if
    // the item was the operation's last, and waits for the next slot's item.
    int slot = 0;
    if (threadIdx.x == FLOW_QT) {
        slot = atomicAdd(head, 1);
        cur = flow_fetch(slot, init, ninit, flag, total, err, wait_ns);
    }
    for (;;) {
        __syncthreads();
        const int4 it = cur;
        if (it.x < 0) break;
        // the product's TMA reads the B operand another CTA wrote: generic-to-async proxy order after the
        // acquire that FLOW_QT made before the barrier above
        if (threadIdx.x == 0) fence_proxy_async_global();
        if (threadIdx.x == FLOW_QT) slot = atomicAdd(head, 1);
        const int box = it.x, j = it.y, t = it.z;
        const BoxInfo B = boxes[box];
        const int bz = B.dims[2];
        const int q = j >> 1;
        const int fwd = q < bz;
        const int s = fwd ? q : q - bz + 1;
        if (j & 1) {
            const int k = fwd ? s : bz - 1 - s;
            gemm_core<E, NPAD, NST>(&mapA, &mapA32, &mapB, B, box, t, k, loc, nrhs, fwd, nkc, err, base, tmem, R);
        } else {
            prep_tile_staged<E>(B, box, t, tpn, coef, lb, loc, bt, ld2, NPAD, nrhs, s, fwd, base,
                                NST * TcCfg<E, NPAD, NST>::STAGE);
            tc::fence_proxy_async_smem();   // the stages are TMA destinations again in a later product
            fence_proxy_async_global();     // B operand written here, read by TMA in another CTA
        }
        __syncthreads();
        if (threadIdx.x == FLOW_QT) {
            // acq_rel: releases this CTA's writes (ordered before by the barrier) and, for the operation's
            // last item, acquires the other items' writes so that the publication below carries them
            if (atom_add_acq_rel_gpu(cnt + box, 1) == flow_tiles(B.m, j, tpn) - 1) {
                atomicExch(cnt + box, 0);
                if (j + 1 < flow_chain(bz)) {
                    const int n = flow_tiles(B.m, j + 1, tpn);
                    const int q0 = atomicAdd(tail, n);
                    for (int i = 0; i < n && ninit + q0 + i < total; ++i)
                        st_release_gpu(flag + q0 + i, flow_pack(box, j + 1, i));
                }
            }
            cur = flow_fetch(slot, init, ninit, flag, total, err, wait_ns);
        }
    }
    gemm_teardown<E, NPAD, NST>(tmem);
}

// cuTensorMapEncodeTiled from the driver, looked up through the runtime so that the
// library itself does not link against libcuda (it still loads on machines without a driver).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool encode_3d(CUtensorMap* map, void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1, uint64_t s2,
               uint32_t b0, uint32_t b1, bool bf16) {
    PFN_cuTensorMapEncodeTiled_v12000 cuTensorMapEncodeTiled = encode_fn();
    if (!cuTensorMapEncodeTiled) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {s1, s2};   // bytes
    cuuint32_t box[3] = {b0, b1, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = cuTensorMapEncodeTiled(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                        base, dims, strides, box, es,
                                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename E, int NPAD, int NST>
helm_status run_tc(helm_ctx ctx, const PlaneSet& P, const c64* lb, c64* loc, E* bt, int nrhs, cudaStream_t st,
                   int* err, const TcFlow* flow) {
    using Cfg = TcCfg<E, NPAD, NST>;
    constexpr bool BF = sizeof(E) == 2;
    CUtensorMap mapA, mapA32, mapB;
    const int ld = P.ld;
    const uint64_t eb = BF ? 2 : 4;
    if (!P.packed) return set_error(ctx, HELM_EINVAL, "tensor-core sweep: factors are not in the tile layout");
    // A: the tile layout, one 128-byte line per (tile, chunk, row): lines of 128 bytes, planes pstride apart
    const uint64_t lines = (uint64_t)P.pk_tiles * P.pk_chunks * TC_BM;
    const uint64_t pbytes = (uint64_t)P.hbox[0].pstride * P.esize();
    if (!encode_3d(&mapA, P.G, Cfg::BK, lines, (uint64_t)P.nplanes, 128, pbytes, Cfg::BK, TC_BM, BF) ||
        !encode_3d(&mapA32, P.G, Cfg::BK, lines, (uint64_t)P.nplanes, 128, pbytes, Cfg::BK, 32, BF) ||
        !encode_3d(&mapB, bt, 2ull * ld, (uint64_t)NPAD, (uint64_t)P.nbox, 2ull * ld * eb, 2ull * ld * NPAD * eb,
                   Cfg::BK, NPAD, BF))
        return set_error(ctx, HELM_ECUDA, "cuTensorMapEncodeTiled failed for the tensor-core sweep");
    static std::atomic<bool> attr{false};
    static std::atomic<int> flow_occ{0};
    if (!attr.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(tc_sweep_gemm<E, NPAD, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        cudaFuncSetAttribute(tc_sweep_flow<E, NPAD, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        // all of the unified L1 as shared memory, so that as many persistent CTAs fit per SM as its 228 KB allow
        cudaFuncSetAttribute(tc_sweep_flow<E, NPAD, NST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        // persistent CTAs per SM from the kernel's shared memory, registers and TMEM columns (the
        // occupancy calculator reports 1 for these tcgen05 kernels, while two of them run side by side)
        int dev = 0, smem_sm = 0, regs_sm = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, tc_sweep_flow<E, NPAD, NST>) == cudaSuccess) {
            const int per_block = Cfg::SMEM + (int)fa.sharedSizeBytes + 1024;   // + the 1 KB reserved per block
            const int regs = (fa.numRegs + 7) / 8 * 8 * 128;
            flow_occ.store(std::min(std::min(smem_sm / per_block, regs_sm / std::max(1, regs)),
                                    std::min(512 / (int)Cfg::TCOLS, 8)));
        }
        cudaFuncSetAttribute(tc_prep2<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(128 * (PREP2_TP + 1) * sizeof(c64)));
        attr.store(true, std::memory_order_release);
    }
    const int m = P.m_max;
    const int gtiles = (m + TC_BM - 1) / TC_BM;
    const dim3 ggrid(gtiles, P.nbox);
    const dim3 pgrid((unsigned)((m + PREP_TP - 1) / PREP_TP), P.nbox);
    const dim3 pgrid2((unsigned)((m + PREP2_TP - 1) / PREP2_TP), P.nbox);
    const size_t psmem2 = (size_t)nrhs * (PREP2_TP + 1) * sizeof(c64);
    const bool vec2 = nrhs % 2 == 0 && (((uintptr_t)lb | (uintptr_t)loc) & 15) == 0;
    const c64* coef = (const c64*)P.coef;
    const double es = sizeof(c64);
    const double fs = 2.0 * sizeof(E);   // bytes of one stored complex factor entry
    // algorithmic bytes of the product and of the operand preparation of step (s, fwd) over boxes [b0, b1)
    auto bytes = [&](int s, bool fwd, int b0, int b1, double& gemm, double& prep) {
        gemm = prep = 0;
        for (int i = b0; i < b1; ++i) {
            const auto& b = P.hbox[i];
            const int bz = b.dims[2];
            const bool act = fwd ? s < bz : (s >= 1 && s <= bz - 1);
            if (!act) continue;
            gemm += ((double)b.m * b.m + (double)b.m * NPAD / 2) * fs + (fwd ? 1.0 : 2.0) * b.m * nrhs * es;
            prep += ((double)b.m * 9 + (fwd ? 3.0 : 2.0) * b.m * nrhs) * es;
        }
    };
    double gb, pb;
    if (flow && flow->mem && ctx->tc_flow && vec2 && flow_occ > 0 &&
        (size_t)nrhs * (flow->tpn + 1) * sizeof(c64) <= (size_t)NST * Cfg::STAGE) {
        double all = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int s = pass == 0 ? 0 : 1; s < P.bz_max; ++s) {
                bytes(s, pass == 0, 0, P.nbox, gb, pb);
                all += gb + pb;
            }
        const int grid = std::max(1, std::min(flow->total, flow_occ * std::max(1, ctx->sm_count)));
        HELM_CUDA(ctx, cudaMemsetAsync(flow->mem, 0, flow->reset_bytes, st));
        const int t = prof_begin(ctx, "sweep_flow");
        tc_sweep_flow<E, NPAD, NST><<<grid, 128, Cfg::SMEM, st>>>(mapA, mapA32, mapB, P.dbox, coef, lb, loc, bt, 2 * ld,
                                                                   nrhs, P.pk_chunks, flow->init, flow->ninit,
                                                                   flow->flag, flow->total, flow->ctl, err,
                                                                   (uint64_t)ctx->flow_wait_us * 1000ull, flow->tpn);
        prof_end(ctx, t, all);
        ctx->launches++;
        return cuda_check(ctx, cudaGetLastError(), "tensor-core plane sweeps (persistent)");
    }
    for (int pass = 0; pass < 2; ++pass) {
        const int fwd = pass == 0;
        for (int s = fwd ? 0 : 1; s < P.bz_max; ++s) {
            bytes(s, fwd, 0, P.nbox, gb, pb);
            int t = prof_begin(ctx, "sweep_prep");
            if (vec2)
                tc_prep2<E><<<pgrid2, 512, psmem2, st>>>(P.dbox, coef, lb, loc, bt, 2 * ld, NPAD, nrhs, s, fwd);
            else
                tc_prep<E><<<pgrid, 256, 0, st>>>(P.dbox, coef, lb, loc, bt, 2 * ld, NPAD, nrhs, s, fwd);
            prof_end(ctx, t, pb);
            t = prof_begin(ctx, "sweep_gemm_tc");
            tc_sweep_gemm<E, NPAD, NST><<<ggrid, 128, Cfg::SMEM, st>>>(mapA, mapA32, mapB, P.dbox, loc, nrhs, s,
                                                                        fwd, P.pk_chunks, err);
            prof_end(ctx, t, gb);
            ctx->launches += 2;
        }
    }
    return cuda_check(ctx, cudaGetLastError(), "tensor-core plane sweeps");
}

template <typename E, int NPAD>
helm_status dispatch_stages(helm_ctx ctx, const PlaneSet& P, const c64* lb, void* loc, void* bt, int ns, int nrhs,
                            cudaStream_t st, int* err, const TcFlow* flow) {
    switch (ns) {
        case 2: return run_tc<E, NPAD, 2>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err, flow);
        case 3: return run_tc<E, NPAD, 3>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err, flow);
        case 4: return run_tc<E, NPAD, 4>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err, flow);
        default: return run_tc<E, NPAD, (NPAD >= 256 ? 4 : 5)>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err, flow);
    }
}

template <typename E>
helm_status dispatch_tc(helm_ctx ctx, const PlaneSet& P, const c64* lb, void* loc, void* bt, int npad, int ns,
                        int nrhs, cudaStream_t st, int* err, const TcFlow* flow) {
    switch (npad) {
        case 16: return dispatch_stages<E, 16>(ctx, P, lb, loc, bt, ns, nrhs, st, err, flow);
        case 32: return dispatch_stages<E, 32>(ctx, P, lb, loc, bt, ns, nrhs, st, err, flow);
        case 64: return dispatch_stages<E, 64>(ctx, P, lb, loc, bt, ns, nrhs, st, err, flow);
        case 128: return dispatch_stages<E, 128>(ctx, P, lb, loc, bt, ns, nrhs, st, err, flow);
        default: return dispatch_stages<E, 256>(ctx, P, lb, loc, bt, ns, nrhs, st, err, flow);
    }
}

}  // namespace

namespace {

// packed[((t * chunks + c) * 128 + i) * 128 + b] = row (128 t + i), byte 128 c + b of the row-major
// plane (zero past the row or the plane), in 16-byte pieces
__global__ void pack_tiles(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst, int nplanes,
                           long long pbytes, int rows, long long row_bytes, int tiles, int chunks) {
    const long long lines = (long long)tiles * chunks * 128;
    const long long total = (long long)nplanes * lines * 8;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e % 8);
        const long long L = (e / 8) % lines;
        const int pl = (int)(e / 8 / lines);
        const int t = (int)(L / ((long long)chunks * 128));
        const int c = (int)((L / 128) % chunks);
        const int i = (int)(L % 128);
        const int r = t * 128 + i;
        const long long boff = (long long)c * 128 + q * 16;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r < rows && boff < row_bytes)
            v = *reinterpret_cast<const uint4*>(src + pl * pbytes + (long long)r * row_bytes + boff);
        *reinterpret_cast<uint4*>(dst + pl * pbytes + L * 128 + q * 16) = v;
    }
}

}  // namespace

// Rearrange the padded row-major plane inverses of a tensor-core set into the tile layout, in place,
// a batch of planes at a time through a scratch copy.
helm_status planeset_pack_tc(helm_ctx ctx, PlaneSet& P) {
    if (!P.padded || P.packed) return HELM_OK;
    const long long esz = (long long)P.esize();
    const long long row_bytes = (long long)P.ld * esz;
    const int tiles = (P.ld + TC_BM - 1) / TC_BM;
    const int chunks = (int)((row_bytes + 127) / 128);
    const long long pbytes = P.hbox[0].pstride * esz;
    if ((long long)tiles * chunks * 128 * 128 > pbytes)
        return set_error(ctx, HELM_EINVAL, "planeset_pack_tc: plane slot too small for the tile layout");
    const int batch = (int)std::max<long long>(1, std::min<long long>(P.nplanes, (256ll << 20) / pbytes));
    void* tmp = nullptr;
    HELM_TRY(dev_alloc(ctx, &tmp, (size_t)batch * pbytes, "factor packing scratch"));
    cudaStream_t st = ctx->stream;
    helm_status rc = HELM_OK;
    for (int p0 = 0; p0 < P.nplanes && rc == HELM_OK; p0 += batch) {
        const int nb = std::min(batch, P.nplanes - p0);
        unsigned char* slot = (unsigned char*)P.G + (size_t)p0 * pbytes;
        rc = cuda_check(ctx, cudaMemcpyAsync(tmp, slot, (size_t)nb * pbytes, cudaMemcpyDeviceToDevice, st),
                        "factor packing copy");
        if (rc) break;
        const long long work = (long long)nb * tiles * chunks * 128 * 8;
        const unsigned grid = (unsigned)std::min<long long>((work + 255) / 256, (long long)ctx->sm_count * 32);
        pack_tiles<<<std::max(1u, grid), 256, 0, st>>>((const unsigned char*)tmp, slot, nb, pbytes, P.ld, row_bytes,
                                                       tiles, chunks);
        ctx->launches++;
        rc = cuda_check(ctx, cudaGetLastError(), "pack_tiles");
    }
    if (rc == HELM_OK) rc = cuda_check(ctx, cudaStreamSynchronize(st), "factor packing");
    dev_free(ctx, tmp, (size_t)batch * pbytes);
    if (rc) return rc;
    P.packed = true;
    P.pk_tiles = tiles;
    P.pk_chunks = chunks;
    return HELM_OK;
}

int tc_npad(int nrhs) {
    const int n = 2 * nrhs;
    if (n <= 16) return 16;
    if (n <= 32) return 32;
    if (n <= 64) return 64;
    if (n <= 128) return 128;
    return 256;
}

helm_status planeset_solve_tc(helm_ctx ctx, const PlaneSet& P, const void* lb_, void* loc, void* bt, int npad,
                              int nrhs, cudaStream_t st, int* err, const TcFlow* flow) {
    const c64* lb = (const c64*)lb_;
    if (nrhs > 128 || tc_npad(nrhs) > npad) return set_error(ctx, HELM_EINVAL, "tensor-core sweep: too many rhs");
    // pipeline depth: the context's tuning value, else 4 stages (3 for N = 256); measured at 112^3 x 16 RHS:
    // 2/3/4/5 stages give 4.97/4.92/5.24/5.16 TB/s (TF32)
    int ns = ctx->tc_stages;
    if (ns < 2 || ns > 5) ns = npad >= 256 ? 3 : 4;
    if (npad >= 256 && ns > 4) ns = 4;   // shared memory: 5 x 48 KB does not fit
    if (P.prec == HELM_PREC_BF16)
        return dispatch_tc<__nv_bfloat16>(ctx, P, lb, loc, bt, npad, ns, nrhs, st, err, flow);
    return dispatch_tc<float>(ctx, P, lb, loc, bt, npad, ns, nrhs, st, err, flow);
}

int tc_flow_tpn(int nrhs) {
    // 128 nodes at every column count: smaller tiles at 128 columns (16 nodes) stage about 4.5 times the neighbour
    // rows they use and measured slower (53 vs 42 ms per launch on 160 x 160 x 80 with 128 columns)
    (void)nrhs;
    return FLOW_TPN_MAX;
}

helm_status tc_flow_alloc(helm_ctx ctx, const PlaneSet& P, TcFlow& F, int tpn) {
    tc_flow_free(ctx, F);
    std::vector<int> init;
    long long total = 0;
    // the packed items hold box < 2048, operation < 1024 (n_z <= 256) and tile < 1024; otherwise no queue
    // (the sweep then runs as per-step launches)
    if (P.nbox >= 2048) return HELM_OK;
    for (int b = 0; b < P.nbox; ++b) {
        const BoxInfo& B = P.hbox[b];
        if (flow_chain(B.dims[2]) > 1024 || flow_tiles(B.m, 0, tpn) > 1024 || flow_tiles(B.m, 1, tpn) > 1024)
            return HELM_OK;
        for (int j = 0; j < flow_chain(B.dims[2]); ++j) total += flow_tiles(B.m, j, tpn);
        for (int i = 0; i < flow_tiles(B.m, 0, tpn); ++i) init.push_back(flow_pack(b, 0, i));
    }
    if (total >= (1ll << 30)) return HELM_OK;
    const size_t nctl = ((size_t)P.nbox + 2 + 3) / 4 * 4;   // ints, padded to 16 bytes
    const size_t nflag = ((size_t)total + 3) / 4 * 4;
    F.reset_bytes = (nctl + nflag) * sizeof(int);
    F.bytes = F.reset_bytes + init.size() * sizeof(int);
    HELM_TRY(dev_alloc(ctx, &F.mem, F.bytes, "tensor-core sweep queue"));
    F.ctl = (int*)F.mem;
    F.flag = F.ctl + nctl;
    F.init = F.flag + nflag;
    F.ninit = (int)init.size();
    F.total = (int)total;
    F.tpn = tpn;
    HELM_CUDA(ctx, cudaMemcpyAsync(F.init, init.data(), init.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HELM_OK;
}

void tc_flow_free(helm_ctx ctx, TcFlow& F) {
    if (F.mem) dev_free(ctx, F.mem, F.bytes);
    F = TcFlow{};
}
