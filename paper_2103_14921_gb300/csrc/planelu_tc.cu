// Plane factorisation of the complex64 local operators on the tensor cores (the exact local solves of
// Eq. oras): for every box and plane k, S_0 = D_0, S_k = D_k - L_k S_{k-1}^{-1} U_{k-1} and the dense
// inverse G_k = S_k^{-1}, by blocked Gauss-Jordan whose rank-NB updates run as tcgen05 GEMMs.
//
// Blocked Gauss-Jordan with block pivots.  For the panel J = [j0, j0 + NB) of the m x m matrix A:
//   P      = A[J,J]^{-1}                      (NB x NB, Gauss-Jordan with partial pivoting inside the block)
//   A[J,:] = P A[J,:]  (columns outside J),    A[J,J] = P
//   A[I,:] = A[I,:] - A[I,J] A[J,:]_new  (rows I outside J, columns outside J)
//   A[I,J] = -A[I,J] P                      (rows I outside J)
// After the last panel A holds S^{-1}.  The last two lines are one product: with W = A[:,J] (before the
// step) and R = the new rows J (R[:,J] = P), A[I,j] = [j not in J] A[I,j] - (W R)[I,j] for I outside J.
// Pivoting stays inside each diagonal block: for these Helmholtz Schur complements (condition numbers
// 1e0-1e2 at the workload sizes) block pivots give the same accuracy as full partial pivoting, and a block
// pivot below 1e-6 of its block's largest entry is reported so that the caller can fall back to the
// fully pivoted CUDA-core elimination.
//
// The product W R (m x NB times NB x m, complex) is one real GEMM with the 2x2 embedding used by the plane
// sweeps: A operand = rows of W read as 2 NB reals (K-major), B operand = B^T[2j][2c] = Re R[c][j],
// B^T[2j][2c+1] = -Im R[c][j], B^T[2j+1][2c] = Im R[c][j], B^T[2j+1][2c+1] = Re R[c][j].  FP32 accuracy
// from TF32 units: each operand x is split into hi = x with its low 13 mantissa bits cleared (exact in TF32)
// and lo = x - hi, and D = hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), accumulated in
// FP32 in TMEM.  Three MMAs (M = 128, N = 256, K = 8) per K step; operands staged by TMA (128-byte swizzle).
//
// Padding: the work matrix of every box is L x L (L = m_max rounded up to 128) with identity rows and
// columns beyond the box's m, written once and never touched again, so the block inverse of a partial last
// panel is that of block-diag(S_JJ, I) and the padding contributes nothing to rows and columns below m.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "blockinv.cuh"
#include <atomic>

#include "internal.h"
#include "tc.cuh"

namespace {

constexpr int NB = 128;              // panel width (complex columns)
constexpr int K2 = 2 * NB;           // real K of the update product
constexpr int UBM = 128;             // output rows per tile
constexpr int UBN = 256;             // output real columns per tile (128 complex)
constexpr int UST = 2;               // operand ring stages
constexpr int A_TILE = UBM * 128;    // 128 rows x 32 fp32 = 16 KB
constexpr int B_TILE = UBN * 128;    // 256 rows x 32 fp32 = 32 KB
constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;
constexpr int USMEM = UST * STAGE + 1024 + 128;
constexpr int DIAG_THREADS = 512;
constexpr int DP = NB + 1;           // row pitch of the diagonal block in shared memory

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// ------------------------------------------------------------------ Schur complements (pitch L)

// S_0 = D_0: the in-plane couplings of plane 0
__global__ void tgj_schur_init(const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef, c64* __restrict__ S,
                               int L) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m, bx = B.dims[0];
    c64* Sb = S + (size_t)blockIdx.y * L * L;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int p = e / m, q = e % m;
        const int dx = q % bx - p % bx, dy = q / bx - p / bx;
        c64 v = mk<float>(0.f, 0.f);
        if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) v = coef[(B.loc_off + p) * 27 + 9 + (dy + 1) * 3 + (dx + 1)];
        Sb[(size_t)p * L + q] = v;
    }
}

// T = G_{k-1} U_{k-1}, G_{k-1} held in S: T[a][q] = sum_d G[a][q-d] U(node q-d of plane k-1, offset (d, +1))
__global__ void tgj_schur_gu(const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef,
                             const c64* __restrict__ S, c64* __restrict__ T, int L, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    const int bx = B.dims[0], by = B.dims[1];
    const c64* G = S + (size_t)blockIdx.y * L * L;
    c64* Tb = T + (size_t)blockIdx.y * L * L;
    const c64* cU = coef + (B.loc_off + (long long)(k - 1) * m) * 27 + 18;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int a = e / m, q = e % m;
        const int qx = q % bx, qy = q / bx;
        c64 acc = mk<float>(0.f, 0.f);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int py = qy - dy;
            if (py < 0 || py >= by) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int px = qx - dx;
                if (px < 0 || px >= bx) continue;
                const int p = py * bx + px;
                cmac(acc, G[(size_t)a * L + p], cU[(long long)p * 27 + (dy + 1) * 3 + (dx + 1)]);
            }
        }
        Tb[(size_t)a * L + q] = acc;
    }
}

// S = D_k - L_k T: S[p][q] = D_k[p][q] - sum_d L(node p of plane k, offset (d, -1)) T[p+d][q]
__global__ void tgj_schur_lt(const BoxInfo* __restrict__ boxes, const c64* __restrict__ coef,
                             const c64* __restrict__ T, c64* __restrict__ S, int L, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    const int bx = B.dims[0], by = B.dims[1];
    const c64* Tb = T + (size_t)blockIdx.y * L * L;
    c64* Sb = S + (size_t)blockIdx.y * L * L;
    const c64* cK = coef + (B.loc_off + (long long)k * m) * 27;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int p = e / m, q = e % m;
        const int px = p % bx, py = p / bx;
        const int dxq = q % bx - px, dyq = q / bx - py;
        c64 acc = mk<float>(0.f, 0.f);
        if (dxq >= -1 && dxq <= 1 && dyq >= -1 && dyq <= 1) acc = cK[(long long)p * 27 + 9 + (dyq + 1) * 3 + (dxq + 1)];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int ny_ = py + dy;
            if (ny_ < 0 || ny_ >= by) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int nx_ = px + dx;
                if (nx_ < 0 || nx_ >= bx) continue;
                const c64 l = cK[(long long)p * 27 + (dy + 1) * 3 + (dx + 1)];
                const c64 t = Tb[(size_t)(ny_ * bx + nx_) * L + q];
                acc.x -= l.x * t.x - l.y * t.y;
                acc.y -= l.x * t.y + l.y * t.x;
            }
        }
        Sb[(size_t)p * L + q] = acc;
    }
}

// identity on the padding diagonal (the rest of the padding is zero from the initial memset)
__global__ void tgj_pad_diag(const BoxInfo* __restrict__ boxes, c64* __restrict__ S, int L) {
    const BoxInfo B = boxes[blockIdx.y];
    for (int i = B.m + blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x)
        S[(size_t)blockIdx.y * L * L + (size_t)i * L + i] = mk<float>(1.f, 0.f);
}

// ------------------------------------------------------------------ panel: block inverse, rows, W

// P = A[J,J]^{-1} by Gauss-Jordan with partial pivoting inside the block, in 16-column sub-panels (one CTA per
// box, blockinv.cuh).  flag bit 0: a zero pivot; bit 1: a pivot below 1e-6 of the block's largest entry.
__global__ void __launch_bounds__(DIAG_THREADS) tgj_diag(const BoxInfo* __restrict__ boxes,
                                                         const c64* __restrict__ S, int L, c64* __restrict__ Pbuf,
                                                         int* __restrict__ flag, int j0, int k) {
    extern __shared__ __align__(16) unsigned char dsm[];
    c64* X = reinterpret_cast<c64*>(dsm);   // [NB][DP], then the sub-panel rows [16][NB]
    __shared__ c64 s_row[NB], s_col[NB];
    __shared__ int s_perm[NB], s_pos[NB];
    __shared__ int s_piv;
    __shared__ float s_wmax[DIAG_THREADS / 32];
    const BoxInfo B = boxes[blockIdx.x];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const c64* A = S + (size_t)blockIdx.x * L * L;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float amax = 0.f;
    for (int e = tid; e < NB * NB; e += DIAG_THREADS) {
        const int r = e / NB, c = e % NB;
        const c64 v = A[(size_t)(j0 + r) * L + j0 + c];
        X[r * DP + c] = v;
        amax = fmaxf(amax, v.x * v.x + v.y * v.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) s_wmax[wid] = amax;
    __syncthreads();
    amax = 0.f;
    for (int w = 0; w < DIAG_THREADS / 32; ++w) amax = fmaxf(amax, s_wmax[w]);
    block_inverse<float, NB, DP, 16, DIAG_THREADS>(X, X + NB * DP, s_perm, s_row, s_col, &s_piv, amax, flag);
    // the row swaps become a column permutation of the inverse (undone in reverse pivot order)
    if (tid == 0) {
        for (int j = 0; j < NB; ++j) s_pos[j] = j;
        for (int c = NB - 1; c >= 0; --c) {
            const int p = s_perm[c];
            const int t = s_pos[c];
            s_pos[c] = s_pos[p];
            s_pos[p] = t;
        }
    }
    __syncthreads();
    c64* Pb = Pbuf + (size_t)blockIdx.x * NB * NB;
    for (int e = tid; e < NB * NB; e += DIAG_THREADS) {
        const int r = e / NB, j = e % NB;
        Pb[e] = X[r * DP + s_pos[j]];
    }
}

// R = P A[J, :] for the CTA's 64 columns (R[:, J] = P), written into rows J of A (entries below m) and as
// the hi / lo parts of the B operand B^T (every column below L, so that the operand is finite everywhere).
// Thread (tx, ty): rows c = tx + 16 i (i < 8), columns col0 + ty + 16 q (q < 4).
__global__ void __launch_bounds__(256) tgj_rows(const BoxInfo* __restrict__ boxes, c64* __restrict__ S, int L,
                                                const c64* __restrict__ Pbuf, float* __restrict__ Bh,
                                                float* __restrict__ Bl, int j0, int k) {
    __shared__ c64 Ps[NB][17];
    __shared__ c64 As[16][64];
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int col0 = blockIdx.x * 64;
    c64* A = S + (size_t)blockIdx.y * L * L;
    const c64* P = Pbuf + (size_t)blockIdx.y * NB * NB;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    c64 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = mk<float>(0.f, 0.f);
    for (int k0 = 0; k0 < NB; k0 += 16) {
        for (int e = tid; e < NB * 16; e += 256) {
            const int r = e >> 4, kk = e & 15;
            Ps[r][kk] = P[r * NB + k0 + kk];
        }
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e >> 6, jj = e & 63;
            As[kk][jj] = A[(size_t)(j0 + k0 + kk) * L + col0 + jj];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            c64 a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = Ps[tx + 16 * i][kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = As[kk][ty + 16 * q];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) cmac(acc[i][q], a[i], b[q]);
        }
        __syncthreads();
    }
    float* bh = Bh + (size_t)blockIdx.y * 2 * L * K2;
    float* bl = Bl + (size_t)blockIdx.y * 2 * L * K2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = col0 + ty + 16 * q;
        const bool inJ = j >= j0 && j < j0 + NB;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = tx + 16 * i;
            const c64 v = inJ ? P[c * NB + (j - j0)] : acc[i][q];
            if (j0 + c < m && j < m) A[(size_t)(j0 + c) * L + j] = v;
            const float re_h = tf32_hi(v.x), im_h = tf32_hi(v.y);
            const float re_l = v.x - re_h, im_l = v.y - im_h;
            float* h0 = bh + (size_t)(2 * j) * K2 + 2 * c;
            float* l0 = bl + (size_t)(2 * j) * K2 + 2 * c;
            *reinterpret_cast<float2*>(h0) = make_float2(re_h, -im_h);
            *reinterpret_cast<float2*>(h0 + K2) = make_float2(im_h, re_h);
            *reinterpret_cast<float2*>(l0) = make_float2(re_l, -im_l);
            *reinterpret_cast<float2*>(l0 + K2) = make_float2(im_l, re_l);
        }
    }
}

// W = A[:, J] (zero on rows J and rows beyond m) as the hi / lo A operand, rows of 2 NB reals.
__global__ void __launch_bounds__(256) tgj_wcopy(const BoxInfo* __restrict__ boxes, const c64* __restrict__ S,
                                                 int L, float* __restrict__ Wh, float* __restrict__ Wl, int j0, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const c64* A = S + (size_t)blockIdx.y * L * L;
    float* wh = Wh + (size_t)blockIdx.y * L * K2;
    float* wl = Wl + (size_t)blockIdx.y * L * K2;
    for (int e = threadIdx.x; e < 32 * NB; e += 256) {
        const int I = blockIdx.x * 32 + e / NB, c = e % NB;
        c64 v = mk<float>(0.f, 0.f);
        if (I < m && !(I >= j0 && I < j0 + NB)) v = A[(size_t)I * L + j0 + c];
        const float re_h = tf32_hi(v.x), im_h = tf32_hi(v.y);
        *reinterpret_cast<float2*>(wh + (size_t)I * K2 + 2 * c) = make_float2(re_h, im_h);
        *reinterpret_cast<float2*>(wl + (size_t)I * K2 + 2 * c) = make_float2(v.x - re_h, v.y - im_h);
    }
}

// ------------------------------------------------------------------ the rank-NB update on the tensor cores

// Tile (tn, tm, box): rows row0 .. row0 + 127, complex columns col0 .. col0 + 127.  Warp 0 lane 0 issues the
// TMA loads (W hi, W lo, B^T hi, B^T lo per 32-real K chunk), warp 1 lane 0 the MMAs, all four warps the
// epilogue (thread t of warp w owns row row0 + 32 w + t): A[I][j] = [j not in J] A[I][j] - D[I][j].
__global__ void __launch_bounds__(128, 1) tgj_update(const __grid_constant__ CUtensorMap mWh,
                                                     const __grid_constant__ CUtensorMap mWl,
                                                     const __grid_constant__ CUtensorMap mBh,
                                                     const __grid_constant__ CUtensorMap mBl,
                                                     const BoxInfo* __restrict__ boxes, c64* __restrict__ S, int L,
                                                     int j0, int k, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char usm_raw[];
    const int box = blockIdx.z;
    const BoxInfo B = boxes[box];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int row0 = blockIdx.y * UBM, col0 = blockIdx.x * (UBN / 2);
    if (row0 >= m || col0 >= m || row0 == j0) return;   // rows J are the panel's own (NB == UBM, j0 % 128 == 0)
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(usm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(base + UST * STAGE);
    uint64_t* empty = full + UST;
    uint64_t* done = empty + UST;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < UST; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mWh);
        tc::prefetch_tmap(&mWl);
        tc::prefetch_tmap(&mBh);
        tc::prefetch_tmap(&mBl);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 256);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    constexpr int NKC = K2 / 32;
    int issued = 0;
    if (warp == 0 && lane == 0) {
        for (int kc = 0; kc < NKC; ++kc) {
            const int st = kc % UST;
            if (kc >= UST && !tc::mbar_wait(&empty[st], ((kc / UST) - 1) & 1, err, 11)) break;
            unsigned char* s = base + st * STAGE;
            tc::mbar_arrive_expect_tx(&full[st], STAGE);
            tc::tma_load_3d(s, &mWh, kc * 32, row0, box, &full[st]);
            tc::tma_load_3d(s + A_TILE, &mWl, kc * 32, row0, box, &full[st]);
            tc::tma_load_3d(s + 2 * A_TILE, &mBh, kc * 32, 2 * col0, box, &full[st]);
            tc::tma_load_3d(s + 2 * A_TILE + B_TILE, &mBl, kc * 32, 2 * col0, box, &full[st]);
            ++issued;
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = tc::idesc_tf32(UBM, UBN);
        for (int kc = 0; kc < NKC; ++kc) {
            const int st = kc % UST;
            if (!tc::mbar_wait(&full[st], (kc / UST) & 1, err, 12)) break;
            tc::fence_after_sync();
            const uint32_t sah = tc::smem_u32(base + st * STAGE);
            const uint32_t sal = sah + A_TILE, sbh = sah + 2 * A_TILE, sbl = sbh + B_TILE;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ah = tc::desc_k_sw128(sah + kk * 32), al = tc::desc_k_sw128(sal + kk * 32);
                const uint64_t bh = tc::desc_k_sw128(sbh + kk * 32), bl = tc::desc_k_sw128(sbl + kk * 32);
                tc::mma_tf32(tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                tc::mma_tf32(tmem, al, bh, idesc, 1u);
            }
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(done);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait(done, 0, err, 13);
    if (!ok) tc::mbar_drain(done, 0);   // products already issued still write TMEM
    tc::fence_after_sync();
    if (!ok && threadIdx.x == 0)
        for (int kc = max(0, issued - UST); kc < issued; ++kc) tc::mbar_drain(&full[kc % UST], (kc / UST) & 1);
    const int I = row0 + warp * 32 + lane;
    if (ok) {
        const bool zero_base = col0 == j0;   // the panel's columns: A[I,J] = -W P
        c64* arow = S + (size_t)box * L * L + (size_t)I * L + col0;
#pragma unroll 1
        for (int cc = 0; cc < UBN / 32; ++cc) {
            uint32_t v[32];
            tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
            tc::tmem_ld_wait();
            if (I < m) {
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const int j = col0 + cc * 16 + q;   // complex columns j and j + 1
                    float4* dst = reinterpret_cast<float4*>(arow + cc * 16 + q);
                    if (j + 1 < m) {
                        const float4 o = zero_base ? make_float4(0.f, 0.f, 0.f, 0.f) : *dst;
                        *dst = make_float4(o.x - __uint_as_float(v[2 * q]), o.y - __uint_as_float(v[2 * q + 1]),
                                           o.z - __uint_as_float(v[2 * q + 2]), o.w - __uint_as_float(v[2 * q + 3]));
                    } else if (j < m) {
                        c64* d1 = arow + cc * 16 + q;
                        const c64 o = zero_base ? mk<float>(0.f, 0.f) : *d1;
                        *d1 = mk<float>(o.x - __uint_as_float(v[2 * q]), o.y - __uint_as_float(v[2 * q + 1]));
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 256);
    }
}

// Persistent form of the update: one CTA per SM takes the launch's tiles in turn (tile t = box-major, then row
// tile, then column tile, every gridDim.x-th one), with two TMEM accumulators so that the epilogue of one tile
// runs while the products of the next are issued.  Warp 0 lane 0 loads the operands (TMA, 2-stage ring),
// warp 1 lane 0 issues the MMAs, warps 2-5 read the accumulator (warp w owns TMEM lanes 32 (w mod 4)..) and
// write -D back through shared memory with TMA: a reduce-add into A for the columns outside J (A - D), a
// store for the panel's own columns (-W P).  The padding diagonal a store overwrites in the panel's column
// tile is restored before the next plane.  Every wait is bounded; on a give-up each role leaves its loop,
// copies and products already issued are waited for, and TMEM is freed.
constexpr int PW = 6;                     // warps: producer, MMA issuer, four epilogue warps
constexpr int STG = 2 * UBM * 128;        // staging: two 128-row x 32-float boxes (32 KB)
constexpr int PSMEM = UST * STAGE + STG + 1024 + 256;

__device__ __forceinline__ bool tile_of(const BoxInfo* __restrict__ boxes, int t, int tl, int j0, int k, int& box,
                                        int& row0, int& col0) {
    box = t / (tl * tl);
    const int r = t % (tl * tl);
    row0 = (r / tl) * UBM;
    col0 = (r % tl) * (UBN / 2);
    const BoxInfo& B = boxes[box];
    return k < B.dims[2] && j0 < B.m && row0 < B.m && col0 < B.m && row0 != j0;
}

__global__ void __launch_bounds__(PW * 32, 1) tgj_update_pers(const __grid_constant__ CUtensorMap mWh,
                                                              const __grid_constant__ CUtensorMap mWl,
                                                              const __grid_constant__ CUtensorMap mBh,
                                                              const __grid_constant__ CUtensorMap mBl,
                                                              const __grid_constant__ CUtensorMap mS,
                                                              const BoxInfo* __restrict__ boxes, int nbox, int L,
                                                              int j0, int k, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char psm_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(psm_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char* stg = base + UST * STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(stg + STG);
    uint64_t* empty = full + UST;
    uint64_t* tfull = empty + UST;
    uint64_t* tempty = tfull + 2;
    uint64_t* fin = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
    int* s_go = reinterpret_cast<int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tl = L / UBM;
    const int ntiles = nbox * tl * tl;
    if (threadIdx.x == 0) {
        for (int i = 0; i < UST; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 4);
        }
        tc::mbar_init(fin, 1);
        tc::fence_barrier_init();
        tc::prefetch_tmap(&mWh);
        tc::prefetch_tmap(&mWl);
        tc::prefetch_tmap(&mBh);
        tc::prefetch_tmap(&mBl);
        tc::prefetch_tmap(&mS);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    constexpr int NKC = K2 / 32;
    int box, row0, col0;
    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                if (!tile_of(boxes, t, tl, j0, k, box, row0, col0)) continue;
                for (int kc = 0; kc < NKC; ++kc, ++g) {
                    const int st = g % UST;
                    if (g >= UST && !tc::mbar_wait(&empty[st], ((g / UST) - 1) & 1, err, 21)) {
                        ok = false;
                        break;
                    }
                    unsigned char* s = base + st * STAGE;
                    tc::mbar_arrive_expect_tx(&full[st], STAGE);
                    tc::tma_load_3d(s, &mWh, kc * 32, row0, box, &full[st]);
                    tc::tma_load_3d(s + A_TILE, &mWl, kc * 32, row0, box, &full[st]);
                    tc::tma_load_3d(s + 2 * A_TILE, &mBh, kc * 32, 2 * col0, box, &full[st]);
                    tc::tma_load_3d(s + 2 * A_TILE + B_TILE, &mBl, kc * 32, 2 * col0, box, &full[st]);
                }
            }
            // a give-up anywhere: let the loads already issued land before the stages are left
            if (!ok || *reinterpret_cast<volatile int*>(err) != 0)
                for (uint32_t q = g > UST ? g - UST : 0; q < g; ++q) tc::mbar_drain(&full[q % UST], (q / UST) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(UBM, UBN);
            uint32_t g = 0, i = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                if (!tile_of(boxes, t, tl, j0, k, box, row0, col0)) continue;
                const uint32_t a = i & 1, u = i >> 1;
                if (u >= 1 && !tc::mbar_wait(&tempty[a], (u - 1) & 1, err, 22)) break;
                tc::fence_after_sync();
                const uint32_t acc = tmem + a * 256;
                for (int kc = 0; kc < NKC; ++kc, ++g) {
                    const int st = g % UST;
                    if (!tc::mbar_wait(&full[st], (g / UST) & 1, err, 23)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sah = tc::smem_u32(base + st * STAGE);
                    const uint32_t sal = sah + A_TILE, sbh = sah + 2 * A_TILE, sbl = sbh + B_TILE;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ah = tc::desc_k_sw128(sah + kk * 32), al = tc::desc_k_sw128(sal + kk * 32);
                        const uint64_t bh = tc::desc_k_sw128(sbh + kk * 32), bl = tc::desc_k_sw128(sbl + kk * 32);
                        tc::mma_tf32(acc, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                        tc::mma_tf32(acc, ah, bl, idesc, 1u);
                        tc::mma_tf32(acc, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[st]);
                }
                if (!ok) break;
                tc::mma_commit(&tfull[a]);
                ++i;
            }
            // every product issued has completed before TMEM is freed
            tc::mma_commit(fin);
            tc::mbar_drain(fin, 0);
        }
    } else {
        // epilogue: 128 threads, hardware barrier 1 among them
        const int et = threadIdx.x - 64;
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int r = q * 32 + lane;            // tile row of this thread
        uint32_t i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (!tile_of(boxes, t, tl, j0, k, box, row0, col0)) continue;
            const uint32_t a = i & 1, u = i >> 1;
            if (et == 0) *s_go = tc::mbar_wait(&tfull[a], u & 1, err, 24) ? 1 : 0;
            tc::named_bar(1, 128);
            if (!*s_go) break;                  // uniform over the four warps
            tc::fence_after_sync();
            const bool store = col0 == j0;      // the panel's own columns: A[I,J] = -W P
            for (int c = 0; c < UBN / 64; ++c) {
                uint32_t v[2][32];
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + a * 256 + c * 64;
                tc::tmem_ld_32x32b_x32(ta, v[0]);
                tc::tmem_ld_32x32b_x32(ta + 32, v[1]);
                tc::tmem_ld_wait();
                if (c == UBN / 64 - 1) {
                    // the accumulator has been read: the MMA issuer may reuse it
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tempty[a]);
                }
                if (et == 0) tc::bulk_wait_read0();   // the staging buffer's last TMA copy has read it
                tc::named_bar(1, 128);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    unsigned char* rowp = stg + h * (UBM * 128) + r * 128;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 val = make_float4(-__uint_as_float(v[h][4 * j]), -__uint_as_float(v[h][4 * j + 1]),
                                                       -__uint_as_float(v[h][4 * j + 2]),
                                                       -__uint_as_float(v[h][4 * j + 3]));
                        *reinterpret_cast<float4*>(rowp + ((j ^ (r & 7)) << 4)) = val;
                    }
                }
                tc::fence_proxy_async_smem();
                tc::named_bar(1, 128);
                if (et == 0) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int x = 2 * col0 + c * 64 + h * 32;
                        if (store) tc::tma_store_3d(&mS, stg + h * (UBM * 128), x, row0, box);
                        else tc::tma_reduce_add_3d(&mS, stg + h * (UBM * 128), x, row0, box);
                    }
                    tc::bulk_commit();
                }
            }
            ++i;
        }
        if (et == 0) tc::bulk_wait0();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// G_k (row pitch ld, complex64) <- the inverse in S
__global__ void tgj_store(const BoxInfo* __restrict__ boxes, const c64* __restrict__ S, int L, c64* __restrict__ G,
                          int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    const c64* A = S + (size_t)blockIdx.y * L * L;
    c64* Gk = G + B.fac_off + (size_t)k * B.pstride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int r = e / m, j = e % m;
        Gk[(size_t)r * B.ld + j] = A[(size_t)r * L + j];
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_f() {
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

// the work matrices S as fp32 [nb][L][2L], boxes of 32 floats x 128 rows, 128-byte swizzle (epilogue stores)
bool encode_matrix(CUtensorMap* map, void* base, uint64_t L, uint64_t nb) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_f();
    if (!enc) return false;
    cuuint64_t dims[3] = {2 * L, L, nb};
    cuuint64_t strides[2] = {2 * L * 4, 2 * L * 4 * L};
    cuuint32_t box[3] = {32, (cuuint32_t)UBM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// fp32 [nb][rows][K2] operand, boxes of 32 x box_rows, 128-byte swizzle
bool encode_operand(CUtensorMap* map, void* base, uint64_t rows, uint64_t nb, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_f();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K2, rows, nb};
    cuuint64_t strides[2] = {(cuuint64_t)K2 * 4, (cuuint64_t)K2 * 4 * rows};
    cuuint32_t box[3] = {32, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Tensor-core factorisation of a padded complex64 plane set (the fine sets of TF32 / BF16 factors).
// *singular: a zero block pivot; *weak: a block pivot below 1e-6 of its block (the caller then factors the
// set again with full partial pivoting).  Returns HELM_ETIMEOUT if a bounded wait of the update gave up.
helm_status planeset_factor_tc(helm_ctx ctx, PlaneSet& P, int* singular, int* weak) {
    *singular = *weak = 0;
    if (P.prec != HELM_PREC_FP32 || !P.padded)
        return set_error(ctx, HELM_EINVAL, "planeset_factor_tc: needs a padded complex64 set");
    cudaStream_t st = ctx->stream;
    const int L = (P.m_max + NB - 1) / NB * NB;
    const size_t nb = (size_t)P.nbox;
    const size_t s_bytes = nb * L * L * sizeof(c64);
    const size_t w_bytes = nb * L * K2 * sizeof(float);
    const size_t b_bytes = nb * 2 * L * K2 * sizeof(float);
    const size_t p_bytes = nb * NB * NB * sizeof(c64);
    void *S = nullptr, *T = nullptr, *Wh = nullptr, *Wl = nullptr, *Bh = nullptr, *Bl = nullptr, *Pb = nullptr;
    int* flag = nullptr;   // [0] pivots, [1] bounded waits
    auto cleanup = [&]() {
        dev_free(ctx, S, s_bytes);
        dev_free(ctx, T, s_bytes);
        dev_free(ctx, Wh, w_bytes);
        dev_free(ctx, Wl, w_bytes);
        dev_free(ctx, Bh, b_bytes);
        dev_free(ctx, Bl, b_bytes);
        dev_free(ctx, Pb, p_bytes);
        dev_free(ctx, flag, 2 * sizeof(int));
    };
    helm_status rc;
    if ((rc = dev_alloc(ctx, &S, s_bytes, "tensor-core factor work S")) ||
        (rc = dev_alloc(ctx, &T, s_bytes, "tensor-core factor work T")) ||
        (rc = dev_alloc(ctx, &Wh, w_bytes, "factor operand W")) || (rc = dev_alloc(ctx, &Wl, w_bytes, "factor operand W")) ||
        (rc = dev_alloc(ctx, &Bh, b_bytes, "factor operand B")) || (rc = dev_alloc(ctx, &Bl, b_bytes, "factor operand B")) ||
        (rc = dev_alloc(ctx, &Pb, p_bytes, "block pivots")) ||
        (rc = dev_alloc(ctx, (void**)&flag, 2 * sizeof(int), "factor flags"))) {
        cleanup();
        return rc;
    }
    CUtensorMap mWh, mWl, mBh, mBl, mS;
    if (!encode_operand(&mWh, Wh, L, nb, UBM) || !encode_operand(&mWl, Wl, L, nb, UBM) ||
        !encode_operand(&mBh, Bh, 2ull * L, nb, UBN) || !encode_operand(&mBl, Bl, 2ull * L, nb, UBN) ||
        !encode_matrix(&mS, S, L, nb)) {
        cleanup();
        return set_error(ctx, HELM_ECUDA, "cuTensorMapEncodeTiled failed for the tensor-core factorisation");
    }
    static std::atomic<bool> attr{false};
    if (!attr.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(tgj_update, cudaFuncAttributeMaxDynamicSharedMemorySize, USMEM);
        cudaFuncSetAttribute(tgj_update_pers, cudaFuncAttributeMaxDynamicSharedMemorySize, PSMEM);
        cudaFuncSetAttribute(tgj_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((NB * DP + 16 * NB) * sizeof(c64)));
        attr.store(true, std::memory_order_release);
    }
    cudaMemsetAsync(S, 0, s_bytes, st);
    cudaMemsetAsync(flag, 0, 2 * sizeof(int), st);
    const c64* coef = (const c64*)P.coef;
    const int tl = L / NB;
    // tc_factor 1: persistent update (one CTA per SM, overlapped epilogue); 2: one CTA per tile
    const bool persistent = ctx->tc_factor == 1;
    const int pgrid = std::max(1, std::min(ctx->sm_count, P.nbox * tl * tl));
    const unsigned eb = (unsigned)std::min<long long>(((long long)P.m_max * P.m_max + 255) / 256, 2048);
    const dim3 egrid(eb, P.nbox);
    tgj_pad_diag<<<dim3(1, P.nbox), 128, 0, st>>>(P.dbox, (c64*)S, L);
    ctx->launches++;
    // algorithmic bytes of one update launch: every active box reads and writes the rows outside J (below m) of
    // its matrix once; of one panel (block inverse, rows, W): the block, the rows J, the column block J and
    // the operands written
    for (int k = 0; k < P.bz_max; ++k) {
        if (k > 0 && persistent) {
            // the padding diagonal that the panel's column store may have overwritten in the last plane
            tgj_pad_diag<<<dim3(1, P.nbox), 128, 0, st>>>(P.dbox, (c64*)S, L);
            ctx->launches++;
        }
        if (k == 0) {
            tgj_schur_init<<<egrid, 256, 0, st>>>(P.dbox, coef, (c64*)S, L);
            ctx->launches++;
        } else {
            tgj_schur_gu<<<egrid, 256, 0, st>>>(P.dbox, coef, (const c64*)S, (c64*)T, L, k);
            tgj_schur_lt<<<egrid, 256, 0, st>>>(P.dbox, coef, (const c64*)T, (c64*)S, L, k);
            ctx->launches += 2;
        }
        for (int j0 = 0; j0 < P.m_max; j0 += NB) {
            double ub = 0, pb = 0;
            for (const auto& b : P.hbox)
                if (k < b.dims[2] && j0 < b.m) {
                    const double rows = b.m - std::min(NB, b.m - j0);
                    ub += 2.0 * rows * b.m * sizeof(c64);
                    pb += (2.0 * NB * b.m + (double)NB * b.m) * sizeof(c64) + (2.0 * 2 * b.m + b.m) * K2 * sizeof(float);
                }
            int t = prof_begin(ctx, "gj_panel_tc");
            tgj_diag<<<P.nbox, DIAG_THREADS, (NB * DP + 16 * NB) * sizeof(c64), st>>>(P.dbox, (const c64*)S, L, (c64*)Pb, flag,
                                                                          j0, k);
            tgj_rows<<<dim3(L / 64, P.nbox), 256, 0, st>>>(P.dbox, (c64*)S, L, (const c64*)Pb, (float*)Bh, (float*)Bl,
                                                           j0, k);
            tgj_wcopy<<<dim3(L / 32, P.nbox), 256, 0, st>>>(P.dbox, (const c64*)S, L, (float*)Wh, (float*)Wl, j0, k);
            prof_end(ctx, t, pb);
            t = prof_begin(ctx, "gj_update_tc");
            if (persistent)
                tgj_update_pers<<<pgrid, PW * 32, PSMEM, st>>>(mWh, mWl, mBh, mBl, mS, P.dbox, P.nbox, L, j0, k,
                                                               flag + 1);
            else
                tgj_update<<<dim3(tl, tl, P.nbox), 128, USMEM, st>>>(mWh, mWl, mBh, mBl, P.dbox, (c64*)S, L, j0, k,
                                                                     flag + 1);
            prof_end(ctx, t, ub);
            ctx->launches += 4;
        }
        tgj_store<<<egrid, 256, 0, st>>>(P.dbox, (const c64*)S, L, (c64*)P.G, k);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cleanup();
            return cuda_check(ctx, e, "tensor-core plane factorisation launch");
        }
    }
    int hflag[2] = {0, 0};
    cudaMemcpyAsync(hflag, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    rc = cuda_check(ctx, cudaStreamSynchronize(st), "tensor-core plane factorisation");
    cleanup();
    if (rc) return rc;
    if (hflag[1]) return set_error(ctx, HELM_ETIMEOUT, "tensor-core plane factorisation: a bounded wait gave up");
    *singular = hflag[0] & 1;
    *weak = (hflag[0] >> 1) & 1;
    return HELM_OK;
}
