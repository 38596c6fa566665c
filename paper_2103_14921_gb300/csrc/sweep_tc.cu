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

template <typename E>
__global__ void __launch_bounds__(512) tc_prep2(const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef,
                                                const c64* __restrict__ lb, const c64* __restrict__ loc,
                                                E* __restrict__ bt, int ld2, int npad, int nrhs, int s, int fwd) {
    extern __shared__ __align__(16) unsigned char prep_smem[];
    c64* tile = reinterpret_cast<c64*>(prep_smem);   // [nrhs][PREP2_TP + 1]
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m, bz = B.dims[2], bx = B.dims[0], by = B.dims[1];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz || (!fwd && k == bz - 1)) return;
    const int p0 = blockIdx.x * PREP2_TP;
    if (p0 >= m) return;
    const int npair = nrhs >> 1;
    const long long plane = B.loc_off + (long long)k * m;
    const long long nbr = fwd ? plane - m : plane + m;
    const int off = fwd ? 0 : 18;
    const bool couple = !(fwd && k == 0);
    for (int e = threadIdx.x; e < PREP2_TP * npair; e += blockDim.x) {
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
                    v[d] = *reinterpret_cast<const float4*>(loc + (nbr + qy * bx + qx) * nrhs + 2 * pr);
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
        tile[(2 * pr) * (PREP2_TP + 1) + pl] = mk<float>(acc.x, acc.y);
        tile[(2 * pr + 1) * (PREP2_TP + 1) + pl] = mk<float>(acc.z, acc.w);
    }
    __syncthreads();
    E* bb = bt + (size_t)blockIdx.y * npad * ld2;
    typedef typename Pair2<E>::type P2;
    for (int e = threadIdx.x; e < nrhs * PREP2_TP; e += blockDim.x) {
        const int r = e / PREP2_TP, pl = e % PREP2_TP, p = p0 + pl;
        if (p >= m) continue;
        const c64 a = tile[r * (PREP2_TP + 1) + pl];
        *reinterpret_cast<P2*>(bb + (size_t)(2 * r) * ld2 + 2 * p) = Pair2<E>::make(a.x, -a.y);
        *reinterpret_cast<P2*>(bb + (size_t)(2 * r + 1) * ld2 + 2 * p) = Pair2<E>::make(a.y, a.x);
    }
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

template <typename E, int NPAD, int NST>
__global__ void __launch_bounds__(128, 1) tc_sweep_gemm(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapA32,
                                                        const __grid_constant__ CUtensorMap mapB,
                                                        const BoxInfo* __restrict__ boxes, c64* __restrict__ loc,
                                                        int nrhs, int s, int fwd, int nkc, int* __restrict__ err) {
    using Cfg = TcCfg<E, NPAD, NST>;
    constexpr int TC_STAGES = Cfg::STAGES;
    constexpr int TC_BK = Cfg::BK;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + TC_STAGES * Cfg::STAGE);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* done = empty + TC_STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m, bz = B.dims[2];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz) return;
    if (!fwd && k == bz - 1) return;
    const int row0 = blockIdx.x * TC_BM;
    if (row0 >= m) return;
    const int nK = (2 * m + TC_BK - 1) / TC_BK;
    const int plane = B.plane0 + k;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mapA);
        tc::prefetch_tmap(&mapA32);
        tc::prefetch_tmap(&mapB);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, Cfg::TCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer.  A tile (rows row0.., chunk kc): 16 KB contiguous in the tile layout; the last,
        // partial row tile of a box loads only its 32-row groups that hold rows < m (the rest of the
        // shared tile keeps stale values, which only reach accumulator rows that are never stored)
        const int rows = min(TC_BM, m - row0);
        const int nsub = rows >= TC_BM ? 0 : (rows + 31) / 32;
        const uint32_t a_bytes = nsub ? (uint32_t)nsub * 32 * 128 : (uint32_t)Cfg::A_BYTES;
        for (int kc = 0; kc < nK; ++kc) {
            const int st = kc % TC_STAGES;
            if (kc >= TC_STAGES && !tc::mbar_wait(&empty[st], ((kc / TC_STAGES) - 1) & 1, err, 1)) break;
            unsigned char* sa = base + st * Cfg::STAGE;
            tc::mbar_arrive_expect_tx(&full[st], a_bytes + Cfg::B_BYTES);
            const int line = (blockIdx.x * nkc + kc) * TC_BM;
            if (nsub == 0)
                tc::tma_load_3d(sa, &mapA, 0, line, plane, &full[st]);
            else
                for (int q = 0; q < nsub; ++q) tc::tma_load_3d(sa + q * 4096, &mapA32, 0, line + 32 * q, plane, &full[st]);
            tc::tma_load_3d(sa + Cfg::A_BYTES, &mapB, kc * TC_BK, 0, blockIdx.y, &full[st]);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr bool BF = sizeof(E) == 2;
        constexpr uint32_t idesc = BF ? tc::idesc_bf16(TC_BM, NPAD) : tc::idesc_tf32(TC_BM, NPAD);
        for (int kc = 0; kc < nK; ++kc) {
            const int st = kc % TC_STAGES;
            if (!tc::mbar_wait(&full[st], (kc / TC_STAGES) & 1, err, 2)) break;
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
    const bool ok = tc::mbar_wait(done, 0, err, 3);
    tc::fence_after_sync();
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
                            const c64 o = dst[r];
                            dst[r] = mk<float>(o.x - re, o.y - im);
                        }
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, Cfg::TCOLS);
    }
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
                   int* err) {
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
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(tc_sweep_gemm<E, NPAD, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        cudaFuncSetAttribute(tc_prep2<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(128 * (PREP2_TP + 1) * sizeof(c64)));
        attr = true;
    }
    const int m = P.m_max;
    const dim3 ggrid((m + TC_BM - 1) / TC_BM, P.nbox);
    const dim3 pgrid((unsigned)((m + PREP_TP - 1) / PREP_TP), P.nbox);
    const dim3 pgrid2((unsigned)((m + PREP2_TP - 1) / PREP2_TP), P.nbox);
    const size_t psmem2 = (size_t)nrhs * (PREP2_TP + 1) * sizeof(c64);
    const bool vec2 = nrhs % 2 == 0 && (((uintptr_t)lb | (uintptr_t)loc) & 15) == 0;
    const c64* coef = (const c64*)P.coef;
    const double es = sizeof(c64);
    const double fs = 2.0 * sizeof(E);   // bytes of one stored complex factor entry
    auto bytes = [&](int s, bool fwd, double& gemm, double& prep) {
        gemm = prep = 0;
        for (const auto& b : P.hbox) {
            const int bz = b.dims[2];
            const bool act = fwd ? s < bz : (s >= 1 && s <= bz - 1);
            if (!act) continue;
            gemm += ((double)b.m * b.m + (double)b.m * NPAD / 2) * fs + (fwd ? 1.0 : 2.0) * b.m * nrhs * es;
            prep += ((double)b.m * 9 + (fwd ? 3.0 : 2.0) * b.m * nrhs) * es;
        }
    };
    double gb, pb;
    for (int pass = 0; pass < 2; ++pass) {
        const int fwd = pass == 0;
        for (int s = fwd ? 0 : 1; s < P.bz_max; ++s) {
            bytes(s, fwd, gb, pb);
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
                            cudaStream_t st, int* err) {
    switch (ns) {
        case 2: return run_tc<E, NPAD, 2>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err);
        case 3: return run_tc<E, NPAD, 3>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err);
        case 4: return run_tc<E, NPAD, 4>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err);
        default: return run_tc<E, NPAD, (NPAD >= 256 ? 4 : 5)>(ctx, P, lb, (c64*)loc, (E*)bt, nrhs, st, err);
    }
}

template <typename E>
helm_status dispatch_tc(helm_ctx ctx, const PlaneSet& P, const c64* lb, void* loc, void* bt, int npad, int ns,
                        int nrhs, cudaStream_t st, int* err) {
    switch (npad) {
        case 16: return dispatch_stages<E, 16>(ctx, P, lb, loc, bt, ns, nrhs, st, err);
        case 32: return dispatch_stages<E, 32>(ctx, P, lb, loc, bt, ns, nrhs, st, err);
        case 64: return dispatch_stages<E, 64>(ctx, P, lb, loc, bt, ns, nrhs, st, err);
        case 128: return dispatch_stages<E, 128>(ctx, P, lb, loc, bt, ns, nrhs, st, err);
        default: return dispatch_stages<E, 256>(ctx, P, lb, loc, bt, ns, nrhs, st, err);
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
                              int nrhs, cudaStream_t st, int* err) {
    const c64* lb = (const c64*)lb_;
    if (nrhs > 128 || tc_npad(nrhs) > npad) return set_error(ctx, HELM_EINVAL, "tensor-core sweep: too many rhs");
    // pipeline depth: the context's tuning value, else 4 stages (3 for N = 256); measured at 112^3 x 16 RHS:
    // 2/3/4/5 stages give 4.97/4.92/5.24/5.16 TB/s (TF32)
    int ns = ctx->tc_stages;
    if (ns < 2 || ns > 5) ns = npad >= 256 ? 3 : 4;
    if (npad >= 256 && ns > 4) ns = 4;   // shared memory: 5 x 48 KB does not fit
    if (P.prec == HELM_PREC_BF16) return dispatch_tc<__nv_bfloat16>(ctx, P, lb, loc, bt, npad, ns, nrhs, st, err);
    return dispatch_tc<float>(ctx, P, lb, loc, bt, npad, ns, nrhs, st, err);
}

