// Plane-by-plane block LU of the local operators (the exact local solves
// A_i^{-1} of Eq. oras, and of the coarse operator E of Eq. 2lvl).
//
// A box with nx_l x ny_l x nz_l nodes is ordered plane by plane (z slowest);
// its operator is block tridiagonal with m x m blocks (m = nx_l ny_l): D_k
// (in-plane couplings), L_k (to plane k-1) and U_k (to plane k+1), each a
// 9-point in-plane pattern taken from the 27 stored coefficients of every
// node.  Factorisation, batched over boxes and sequential over planes:
//   S_0 = D_0,  S_k = D_k - L_k S_{k-1}^{-1} U_{k-1},  G_k = S_k^{-1} (dense).
// Solve (forward then backward sweeps):
//   y_k = G_k (b_k - L_k y_{k-1}),   x_k = y_k - G_k (U_k x_{k+1}).
//
// Kernels:
//   schur_gu     T = G_{k-1} U_{k-1}      (9 complex MACs per entry)
//   schur_lt     S = D_k - L_k T          (9 complex MACs per entry)
//   gj_panel     Gauss-Jordan with partial pivoting on an nb-column panel,
//                whole-row swaps applied at once
//   gj_update    rank-nb update of the columns outside the panel
//   gj_store     undo the column permutation, store G_k
//   sweep_prep   b_k - L_k y_{k-1}  or  U_k x_{k+1}
//   sweep_gemv   G_k times the prepared plane, nrhs columns (warp per row)
//
// Blocked in-place Gauss-Jordan: with the pivot-row swaps applied to whole
// rows immediately, after the panel [j0, j1) has been eliminated the panel
// columns hold W[:, j0:j1] of the accumulated elimination transform, and the
// other columns B become W B = B + (W[:, j0:j1] - I[:, j0:j1]) B[j0:j1, :]
// (rows j0..j1 of B are copied out first).  At the end the columns are
// swapped back in reverse pivot order.
#include <cuda_bf16.h>

#include "blockinv.cuh"
#include <atomic>

#include "internal.h"

namespace {

template <typename T> __device__ __forceinline__ T cabs2(cplx<T> a) { return a.x * a.x + a.y * a.y; }
template <typename T> __device__ __forceinline__ cplx<T> cinv(cplx<T> a) {
    const T d = a.x * a.x + a.y * a.y;
    return mk<T>(a.x / d, -a.y / d);
}
template <typename S, typename T> __device__ __forceinline__ cplx<T> ccast(cplx<S> a) { return mk<T>((T)a.x, (T)a.y); }

// ------------------------------------------------------------------ Schur update

template <typename T>
__global__ void schur_init(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ coef, cplx<T>* __restrict__ S,
                           int m_max, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    cplx<T>* Sb = S + (size_t)blockIdx.y * m_max * m_max;
    const int bx = B.dims[0];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * m;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / m), q = (int)(e % m);
        const int dx = q % bx - p % bx, dy = q / bx - p / bx;
        cplx<T> v = mk<T>(0, 0);
        if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1)
            v = coef[(B.loc_off + (long long)k * m + p) * 27 + 9 + (dy + 1) * 3 + (dx + 1)];
        Sb[e] = v;
    }
}

// Tm = G_{k-1} U_{k-1}:  Tm[a][q] = sum_d G[a][q-d] * U(node q-d of plane k-1, offset (d, +1))
template <typename T>
__global__ void schur_gu(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ coef,
                         const cplx<T>* __restrict__ G, cplx<T>* __restrict__ Tm, int m_max, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    const int bx = B.dims[0], by = B.dims[1];
    const cplx<T>* Gp = G + B.fac_off + (size_t)(k - 1) * B.pstride;
    const int ld = B.ld;
    cplx<T>* Tb = Tm + (size_t)blockIdx.y * m_max * m_max;
    const cplx<T>* cU = coef + (B.loc_off + (long long)(k - 1) * m) * 27 + 18;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * m;
         e += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(e / m), q = (int)(e % m);
        const int qx = q % bx, qy = q / bx;
        cplx<T> acc = mk<T>(0, 0);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int py = qy - dy;
            if (py < 0 || py >= by) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int px = qx - dx;
                if (px < 0 || px >= bx) continue;
                const int p = py * bx + px;
                cmac(acc, Gp[(size_t)a * ld + p], cU[(long long)p * 27 + (dy + 1) * 3 + (dx + 1)]);
            }
        }
        Tb[e] = acc;
    }
}

// S = D_k - L_k Tm:  S[p][q] = D_k[p][q] - sum_d L(node p of plane k, offset (d, -1)) * Tm[p+d][q]
template <typename T>
__global__ void schur_lt(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ coef,
                         const cplx<T>* __restrict__ Tm, cplx<T>* __restrict__ S, int m_max, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    const int bx = B.dims[0], by = B.dims[1];
    const cplx<T>* Tb = Tm + (size_t)blockIdx.y * m_max * m_max;
    cplx<T>* Sb = S + (size_t)blockIdx.y * m_max * m_max;
    const cplx<T>* cK = coef + (B.loc_off + (long long)k * m) * 27;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * m;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / m), q = (int)(e % m);
        const int px = p % bx, py = p / bx;
        const int dxq = q % bx - px, dyq = q / bx - py;
        cplx<T> acc = mk<T>(0, 0);
        if (dxq >= -1 && dxq <= 1 && dyq >= -1 && dyq <= 1) acc = cK[(long long)p * 27 + 9 + (dyq + 1) * 3 + (dxq + 1)];
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int ny_ = py + dy;
            if (ny_ < 0 || ny_ >= by) continue;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int nx_ = px + dx;
                if (nx_ < 0 || nx_ >= bx) continue;
                const cplx<T> l = cK[(long long)p * 27 + (dy + 1) * 3 + (dx + 1)];
                const cplx<T> t = Tb[(size_t)(ny_ * bx + nx_) * m + q];
                acc.x -= l.x * t.x - l.y * t.y;
                acc.y -= l.x * t.y + l.y * t.x;
            }
        }
        Sb[e] = acc;
    }
}

// ------------------------------------------------------------------ Gauss-Jordan

constexpr int GJ_THREADS = 512;

// One CTA per box: eliminate panel columns [j0, j1) with partial pivoting.
template <typename T>
__global__ void __launch_bounds__(GJ_THREADS) gj_panel(const BoxInfo* __restrict__ boxes, cplx<T>* __restrict__ S,
                                                       int* __restrict__ perm, cplx<T>* __restrict__ rows,
                                                       int* __restrict__ flag, int m_max, int nb, int j0, int k) {
    const BoxInfo B = boxes[blockIdx.x];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int j1 = min(m, j0 + nb);
    cplx<T>* A = S + (size_t)blockIdx.x * m_max * m_max;
    int* pv = perm + (size_t)blockIdx.x * m_max;
    __shared__ T s_val[GJ_THREADS / 32];
    __shared__ int s_idx[GJ_THREADS / 32];
    __shared__ int s_piv;
    __shared__ cplx<T> s_row[64];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (int c = j0; c < j1; ++c) {
        // pivot search over rows c..m-1 (ties -> smallest index)
        T best = (T)-1;
        int bi = m;
        for (int r = c + tid; r < m; r += GJ_THREADS) {
            const T v = cabs2(A[(size_t)r * m + c]);
            if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            T bv = s_val[0];
            int bidx = s_idx[0];
            for (int w = 1; w < GJ_THREADS / 32; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bidx)) { bv = s_val[w]; bidx = s_idx[w]; }
            if (!(bv > (T)0) || bidx >= m) {
                atomicOr(flag, 1);
                bidx = c;
            }
            s_piv = bidx;
            pv[c] = bidx;
        }
        __syncthreads();
        const int p = s_piv;
        if (p != c) {
            for (int j = tid; j < m; j += GJ_THREADS) {
                const cplx<T> t = A[(size_t)c * m + j];
                A[(size_t)c * m + j] = A[(size_t)p * m + j];
                A[(size_t)p * m + j] = t;
            }
            __syncthreads();
        }
        cplx<T> piv = A[(size_t)c * m + c];
        if (!(cabs2(piv) > (T)0)) piv = mk<T>((T)1, (T)0);   // singular: flagged above, keep going finite
        const cplx<T> inv = cinv(piv);
        if (tid < j1 - j0) {
            const int j = j0 + tid;
            s_row[tid] = (j == c) ? inv : A[(size_t)c * m + j] * inv;
        }
        __syncthreads();
        for (int r = tid; r < m; r += GJ_THREADS) {
            cplx<T>* Ar = A + (size_t)r * m;
            if (r == c) {
                for (int jj = 0; jj < j1 - j0; ++jj) Ar[j0 + jj] = s_row[jj];
                continue;
            }
            const cplx<T> f = Ar[c];
            for (int jj = 0; jj < j1 - j0; ++jj) {
                const int j = j0 + jj;
                if (j == c) {
                    const cplx<T> v = f * inv;
                    Ar[c] = mk<T>(-v.x, -v.y);
                } else {
                    const cplx<T> s = s_row[jj];
                    Ar[j].x -= f.x * s.x - f.y * s.y;
                    Ar[j].y -= f.x * s.y + f.y * s.x;
                }
            }
        }
        __syncthreads();
    }
    // copy rows j0..j1 (all columns) for the trailing update
    cplx<T>* Rb = rows + (size_t)blockIdx.x * 64 * m_max;
    for (long long e = tid; e < (long long)(j1 - j0) * m; e += GJ_THREADS) {
        const int i = (int)(e / m), j = (int)(e % m);
        Rb[(size_t)i * m + j] = A[(size_t)(j0 + i) * m + j];
    }
}

// gj_panel with the panel held in shared memory: NB columns of all m rows (column-major, m * NB complex
// values), 1024 threads.  The same pivots (largest modulus, ties to the smallest row) and the same
// per-entry operations as gj_panel; the row swaps of the columns outside the panel are recorded and
// applied to the matrix, in order, after the panel, which gives the rows gj_panel's whole-row swaps
// leave (nothing else touches those columns in between).
constexpr int GJS_THREADS = 1024;

template <typename T, int NB>
__global__ void __launch_bounds__(GJS_THREADS) gj_panel_smem(const BoxInfo* __restrict__ boxes, cplx<T>* __restrict__ S,
                                                             int* __restrict__ perm, cplx<T>* __restrict__ rows,
                                                             int* __restrict__ flag, int m_max, int j0, int k) {
    extern __shared__ __align__(16) unsigned char gjs_smem[];
    cplx<T>* P = reinterpret_cast<cplx<T>*>(gjs_smem);   // [NB][m]: column-major, a warp reads 32 consecutive rows
    const BoxInfo B = boxes[blockIdx.x];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int nbw = min(NB, m - j0);
    cplx<T>* A = S + (size_t)blockIdx.x * m_max * m_max;
    int* pv = perm + (size_t)blockIdx.x * m_max;
    __shared__ T s_val[GJS_THREADS / 32];
    __shared__ int s_idx[GJS_THREADS / 32];
    __shared__ int s_piv[NB];
    __shared__ cplx<T> s_row[NB];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int e = tid; e < m * NB; e += GJS_THREADS) {
        const int r = e / NB, c = e % NB;
        P[c * m + r] = c < nbw ? A[(size_t)r * m + j0 + c] : mk<T>(0, 0);
    }
    __syncthreads();
    for (int cc = 0; cc < nbw; ++cc) {
        const int c = j0 + cc;
        T best = (T)-1;
        int bi = m;
        for (int r = c + tid; r < m; r += GJS_THREADS) {
            const T v = cabs2(P[cc * m + r]);
            if (v > best) { best = v; bi = r; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            T bv = s_val[0];
            int bidx = s_idx[0];
            for (int w = 1; w < GJS_THREADS / 32; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bidx)) { bv = s_val[w]; bidx = s_idx[w]; }
            if (!(bv > (T)0) || bidx >= m) {
                atomicOr(flag, 1);
                bidx = c;
            }
            s_piv[cc] = bidx;
            pv[c] = bidx;
        }
        __syncthreads();
        const int p = s_piv[cc];
        if (p != c && tid < NB) {
            const cplx<T> t = P[tid * m + c];
            P[tid * m + c] = P[tid * m + p];
            P[tid * m + p] = t;
        }
        __syncthreads();
        cplx<T> piv = P[cc * m + c];
        if (!(cabs2(piv) > (T)0)) piv = mk<T>((T)1, (T)0);   // singular: flagged above, keep going finite
        const cplx<T> inv = cinv(piv);
        if (tid < nbw) s_row[tid] = (tid == cc) ? inv : P[tid * m + c] * inv;
        __syncthreads();
        for (int r = tid; r < m; r += GJS_THREADS) {
            if (r == c) {
                for (int jj = 0; jj < nbw; ++jj) P[jj * m + r] = s_row[jj];
                continue;
            }
            const cplx<T> f = P[cc * m + r];
            for (int jj = 0; jj < nbw; ++jj) {
                cplx<T>& x = P[jj * m + r];
                if (jj == cc) {
                    const cplx<T> v = f * inv;
                    x = mk<T>(-v.x, -v.y);
                } else {
                    const cplx<T> sv = s_row[jj];
                    x.x -= f.x * sv.x - f.y * sv.y;
                    x.y -= f.x * sv.y + f.y * sv.x;
                }
            }
        }
        __syncthreads();
    }
    // the recorded row swaps, in order, on the columns outside the panel
    for (int cc = 0; cc < nbw; ++cc) {
        const int c = j0 + cc, p = s_piv[cc];
        if (p != c)
            for (int j = tid; j < m; j += GJS_THREADS) {
                if (j >= j0 && j < j0 + nbw) continue;
                const cplx<T> t = A[(size_t)c * m + j];
                A[(size_t)c * m + j] = A[(size_t)p * m + j];
                A[(size_t)p * m + j] = t;
            }
        __syncthreads();
    }
    // the panel back, and rows j0..j0+nbw (all columns) for the trailing update
    for (int e = tid; e < m * NB; e += GJS_THREADS) {
        const int r = e / NB, c = e % NB;
        if (c < nbw) A[(size_t)r * m + j0 + c] = P[c * m + r];
    }
    __syncthreads();
    cplx<T>* Rb = rows + (size_t)blockIdx.x * 64 * m_max;
    for (long long e = tid; e < (long long)nbw * m; e += GJS_THREADS) {
        const int i = (int)(e / m), j = (int)(e % m);
        Rb[(size_t)i * m + j] = (j >= j0 && j < j0 + nbw) ? P[(j - j0) * m + j0 + i] : A[(size_t)(j0 + i) * m + j];
    }
}

// Columns outside the panel: A[r][j] = [r not in panel] A[r][j] + sum_c W[r][c] Rows[c][j].
// 64 x 64 output tile per CTA, 16 x 16 threads, 4 x 4 outputs per thread.
template <typename T, int NB>
__global__ void __launch_bounds__(256) gj_update(const BoxInfo* __restrict__ boxes, cplx<T>* __restrict__ S,
                                                 const cplx<T>* __restrict__ rows, int m_max, int j0, int k) {
    const BoxInfo B = boxes[blockIdx.z];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int nbw = min(NB, m - j0);
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    if (r0 >= m || c0 >= m) return;
    if (c0 >= j0 && c0 + 64 <= j0 + nbw) return;   // tile entirely inside the panel
    cplx<T>* A = S + (size_t)blockIdx.z * m_max * m_max;
    const cplx<T>* Rb = rows + (size_t)blockIdx.z * 64 * m_max;
    __shared__ cplx<T> sW[64][NB + 1];
    __shared__ cplx<T> sR[NB][64 + 1];
    const int tid = threadIdx.x;
    for (int e = tid; e < 64 * NB; e += 256) {
        const int r = e / NB, c = e % NB;
        sW[r][c] = (r0 + r < m && c < nbw) ? A[(size_t)(r0 + r) * m + j0 + c] : mk<T>(0, 0);
        const int cc = e / 64, jj = e % 64;
        sR[cc][jj] = (cc < nbw && c0 + jj < m) ? Rb[(size_t)cc * m + c0 + jj] : mk<T>(0, 0);
    }
    __syncthreads();
    const int tx = tid % 16, ty = tid / 16;
    cplx<T> acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk<T>(0, 0);
    for (int c = 0; c < nbw; ++c) {
        cplx<T> w[4], rr[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a] = sW[ty + 16 * a][c];
#pragma unroll
        for (int b = 0; b < 4; ++b) rr[b] = sR[c][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) cmac(acc[a][b], w[a], rr[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = r0 + ty + 16 * a;
        if (r >= m) continue;
        const bool in_panel_row = r >= j0 && r < j0 + nbw;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = c0 + tx + 16 * b;
            if (j >= m || (j >= j0 && j < j0 + nbw)) continue;
            cplx<T>* dst = A + (size_t)r * m + j;
            const cplx<T> base = in_panel_row ? mk<T>(0, 0) : *dst;
            *dst = base + acc[a][b];
        }
    }
}

// Undo the column swaps (reverse pivot order) and write G_k.
template <typename T>
__global__ void gj_store(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ S, const int* __restrict__ perm,
                         cplx<T>* __restrict__ G, int m_max, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    extern __shared__ int s_pos[];
    const int* pv = perm + (size_t)blockIdx.y * m_max;
    if (threadIdx.x == 0) {
        for (int j = 0; j < m; ++j) s_pos[j] = j;
        for (int c = m - 1; c >= 0; --c) {
            const int p = pv[c];
            const int t = s_pos[c];
            s_pos[c] = s_pos[p];
            s_pos[p] = t;
        }
    }
    __syncthreads();
    const cplx<T>* A = S + (size_t)blockIdx.y * m_max * m_max;
    cplx<T>* Gk = G + B.fac_off + (size_t)k * B.pstride;
    const int rows_per = (m + gridDim.x - 1) / gridDim.x;
    const int ra = blockIdx.x * rows_per, rb = min(m, ra + rows_per);
    for (long long e = (long long)ra * m + threadIdx.x; e < (long long)rb * m; e += blockDim.x) {
        const int r = (int)(e / m), j = (int)(e % m);
        Gk[(size_t)r * B.ld + j] = A[(size_t)r * m + s_pos[j]];
    }
}

// ------------------------------------------------------------------ sweeps

// FWD: rb = b_k - L_k y_{k-1} (k > 0) or b_0;  BWD: rb = U_k x_{k+1} (k < bz-1).
template <typename T, bool FWD>
__global__ void sweep_prep(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ coef,
                           const cplx<T>* __restrict__ loc, cplx<T>* __restrict__ rbuf, int m_max, int nrhs, int s) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m, bz = B.dims[2], bx = B.dims[0], by = B.dims[1];
    const int k = FWD ? s : bz - 1 - s;
    if (k < 0 || k >= bz) return;
    if (!FWD && k == bz - 1) return;
    cplx<T>* rb = rbuf + (size_t)blockIdx.y * m_max * nrhs;
    const long long plane = B.loc_off + (long long)k * m;
    const long long nbr = FWD ? plane - m : plane + m;
    const int off = FWD ? 0 : 18;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * nrhs;
         e += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(e / nrhs), r = (int)(e % nrhs);
        cplx<T> acc = mk<T>(0, 0);
        if (FWD) acc = loc[(plane + p) * nrhs + r];
        if (FWD && k == 0) {
            rb[e] = acc;
            continue;
        }
        // all 18 loads first: a coupling that points out of the box has a zero coefficient (the fold moved
        // it), so its neighbour index is clamped into the box
        const int px = p % bx, py = p / bx;
        const cplx<T>* cp = coef + (plane + p) * 27 + off;
        cplx<T> c[9], v[9];
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            const int qx = min(max(px + d % 3 - 1, 0), bx - 1), qy = min(max(py + d / 3 - 1, 0), by - 1);
            c[d] = cp[d];
            v[d] = loc[(nbr + qy * bx + qx) * nrhs + r];
        }
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            if (FWD) {
                acc.x -= c[d].x * v[d].x - c[d].y * v[d].y;
                acc.y -= c[d].x * v[d].y + c[d].y * v[d].x;
            } else {
                cmac(acc, c[d], v[d]);
            }
        }
        rb[e] = acc;
    }
}

// loc[plane k][row][r0 + r] = (FWD ? 0 : loc[...]) +/- sum_kk G_k[row][kk] rb[kk][r0 + r]
// One warp per row; the rhs chunk of rb is staged in shared memory as [RN][m].
template <typename T, int RN, bool FWD>
__global__ void __launch_bounds__(256) sweep_gemv(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ G,
                                                  const cplx<T>* __restrict__ rbuf, cplx<T>* __restrict__ loc,
                                                  int m_max, int nrhs, int s, int rows_per_cta) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m, bz = B.dims[2];
    const int k = FWD ? s : bz - 1 - s;
    if (k < 0 || k >= bz) return;
    if (!FWD && k == bz - 1) return;
    const int row_a = blockIdx.x * rows_per_cta;
    if (row_a >= m) return;
    const int row_b = min(m, row_a + rows_per_cta);
    const int r0 = blockIdx.z * RN;
    const int rn = min(RN, nrhs - r0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);   // [RN][m]
    const cplx<T>* rb = rbuf + (size_t)blockIdx.y * m_max * nrhs;
    // staging with kk fastest: conflict-free shared stores (the rhs block itself is L2-resident)
    for (int e = threadIdx.x; e < m * RN; e += blockDim.x) {
        const int r = e / m, kk = e % m;
        rs[e] = (r < rn) ? rb[(size_t)kk * nrhs + r0 + r] : mk<T>(0, 0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const cplx<T>* Gk = G + B.fac_off + (size_t)k * B.pstride;
    for (int row = row_a + wid; row < row_b; row += nw) {
        cplx<T> acc[RN];
#pragma unroll
        for (int r = 0; r < RN; ++r) acc[r] = mk<T>(0, 0);
        const cplx<T>* g = Gk + (size_t)row * B.ld;
        for (int kk = lane; kk < m; kk += 32) {
            const cplx<T> gv = g[kk];
#pragma unroll
            for (int r = 0; r < RN; ++r) cmac(acc[r], gv, rs[r * m + kk]);
        }
#pragma unroll
        for (int r = 0; r < RN; ++r) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
                acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
            }
        }
        cplx<T>* dst = loc + (B.loc_off + (long long)k * m + row) * nrhs + r0;
#pragma unroll
        for (int r = 0; r < RN; ++r) {
            if (lane == r && r < rn) {
                if (FWD) dst[r] = acc[r];
                else dst[r] = dst[r] - acc[r];
            }
        }
    }
}

// Split-K variant for sets with few boxes (the coarse grid is one box): CTA (row block, K slice)
// writes partial sums part[slice][row][r]; sweep_reduce adds the slices in a fixed order.
constexpr int KSPLIT = 8;

template <typename T, int RN>
__global__ void __launch_bounds__(256) sweep_gemv_splitk(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ G,
                                                         const cplx<T>* __restrict__ rbuf, cplx<T>* __restrict__ part,
                                                         int m_max, int nrhs, int s, int fwd, int rows_per_cta) {
    const BoxInfo B = boxes[0];
    const int m = B.m, bz = B.dims[2];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz || (!fwd && k == bz - 1)) return;
    const int row_a = blockIdx.x * rows_per_cta;
    if (row_a >= m) return;
    const int row_b = min(m, row_a + rows_per_cta);
    const int kw = (m + KSPLIT - 1) / KSPLIT;
    const int k0 = blockIdx.y * kw, k1 = min(m, k0 + kw);
    const int r0 = blockIdx.z * RN;
    const int rn = min(RN, nrhs - r0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* rs = reinterpret_cast<cplx<T>*>(smem_raw);   // [RN][kw]
    for (int e = threadIdx.x; e < kw * RN; e += blockDim.x) {
        const int r = e / kw, kk = e % kw;
        rs[e] = (r < rn && k0 + kk < k1) ? rbuf[(size_t)(k0 + kk) * nrhs + r0 + r] : mk<T>(0, 0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const cplx<T>* Gk = G + B.fac_off + (size_t)k * B.pstride;
    for (int row = row_a + wid; row < row_b; row += nw) {
        cplx<T> acc[RN];
#pragma unroll
        for (int r = 0; r < RN; ++r) acc[r] = mk<T>(0, 0);
        const cplx<T>* g = Gk + (size_t)row * B.ld;
        for (int kk = k0 + lane; kk < k1; kk += 32) {
            const cplx<T> gv = g[kk];
#pragma unroll
            for (int r = 0; r < RN; ++r) cmac(acc[r], gv, rs[r * kw + (kk - k0)]);
        }
#pragma unroll
        for (int r = 0; r < RN; ++r) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, o);
                acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, o);
            }
        }
        cplx<T>* dst = part + ((size_t)blockIdx.y * m_max + row) * nrhs + r0;
#pragma unroll
        for (int r = 0; r < RN; ++r)
            if (lane == r && r < rn) dst[r] = acc[r];
    }
}

template <typename T>
__global__ void sweep_reduce(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ part,
                             cplx<T>* __restrict__ loc, int m_max, int nrhs, int s, int fwd) {
    const BoxInfo B = boxes[0];
    const int m = B.m, bz = B.dims[2];
    const int k = fwd ? s : bz - 1 - s;
    if (k < 0 || k >= bz || (!fwd && k == bz - 1)) return;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * nrhs;
         e += (long long)gridDim.x * blockDim.x) {
        cplx<T> acc = mk<T>(0, 0);
        for (int sl = 0; sl < KSPLIT; ++sl) acc = acc + part[(size_t)sl * m_max * nrhs + e];
        cplx<T>* dst = loc + (B.loc_off + (long long)k * m) * nrhs + e;
        *dst = fwd ? acc : *dst - acc;
    }
}

// ------------------------------------------------------------------ host side

template <typename T>
helm_status factor_t(helm_ctx ctx, PlaneSet& P, int* singular) {
    cudaStream_t st = ctx->stream;
    const int nb = sizeof(T) == 4 ? 32 : 16;
    const size_t mm = (size_t)P.m_max * P.m_max;
    cplx<T>*S = nullptr, *Tm = nullptr, *rows = nullptr;
    int *perm = nullptr, *flag = nullptr;
    helm_status rc = HELM_OK;
    auto cleanup = [&]() {
        dev_free(ctx, S, P.nbox * mm * sizeof(cplx<T>));
        dev_free(ctx, Tm, P.nbox * mm * sizeof(cplx<T>));
        dev_free(ctx, rows, (size_t)P.nbox * 64 * P.m_max * sizeof(cplx<T>));
        dev_free(ctx, perm, (size_t)P.nbox * P.m_max * sizeof(int));
        dev_free(ctx, flag, sizeof(int));
    };
    if ((rc = dev_alloc(ctx, (void**)&S, P.nbox * mm * sizeof(cplx<T>), "factor work S")) ||
        (rc = dev_alloc(ctx, (void**)&Tm, P.nbox * mm * sizeof(cplx<T>), "factor work T")) ||
        (rc = dev_alloc(ctx, (void**)&rows, (size_t)P.nbox * 64 * P.m_max * sizeof(cplx<T>), "factor rows")) ||
        (rc = dev_alloc(ctx, (void**)&perm, (size_t)P.nbox * P.m_max * sizeof(int), "pivots")) ||
        (rc = dev_alloc(ctx, (void**)&flag, sizeof(int), "singular flag"))) {
        cleanup();
        return rc;
    }
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    const cplx<T>* coef = (const cplx<T>*)P.coef;
    cplx<T>* G = (cplx<T>*)P.G;
    const int m = P.m_max;
    const unsigned eblocks = (unsigned)std::min<long long>(((long long)m * m + 255) / 256, 4096);
    const dim3 egrid(eblocks, P.nbox);
    const int tiles = (m + 63) / 64;
    // complex64: 24-column panels held in shared memory while they fit (m * 24 * 8 bytes, m <= 1066);
    // else the global-memory panel of nb columns
    constexpr int NBS = 24;
    const size_t psm = (size_t)m * NBS * sizeof(cplx<T>);
    static std::atomic<bool> psm_attr{false};
    if constexpr (sizeof(T) == 4) {
        if (!psm_attr.load(std::memory_order_acquire)) {
            cudaFuncSetAttribute(gj_panel_smem<T, NBS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            psm_attr.store(true, std::memory_order_release);
        }
    }
    const bool smem_panel = sizeof(T) == 4 && psm <= 200 * 1024;
    const int nbk = smem_panel ? NBS : nb;
    for (int k = 0; k < P.bz_max; ++k) {
        if (k == 0) {
            schur_init<T><<<egrid, 256, 0, st>>>(P.dbox, coef, S, m, k);
            ctx->launches++;
        } else {
            schur_gu<T><<<egrid, 256, 0, st>>>(P.dbox, coef, G, Tm, m, k);
            schur_lt<T><<<egrid, 256, 0, st>>>(P.dbox, coef, Tm, S, m, k);
            ctx->launches += 2;
        }
        double ub = 0;
        for (const auto& b : P.hbox)
            if (k < b.dims[2]) ub += 2.0 * b.m * b.m * sizeof(cplx<T>);
        for (int j0 = 0; j0 < m; j0 += nbk) {
            int t = prof_begin(ctx, "gj_panel");
            if constexpr (sizeof(T) == 4) {
                if (smem_panel)
                    gj_panel_smem<T, NBS><<<P.nbox, GJS_THREADS, psm, st>>>(P.dbox, S, perm, rows, flag, m, j0, k);
                else
                    gj_panel<T><<<P.nbox, GJ_THREADS, 0, st>>>(P.dbox, S, perm, rows, flag, m, nb, j0, k);
            } else {
                gj_panel<T><<<P.nbox, GJ_THREADS, 0, st>>>(P.dbox, S, perm, rows, flag, m, nb, j0, k);
            }
            prof_end(ctx, t, 0.0);
            t = prof_begin(ctx, "gj_update");
            if (sizeof(T) == 4 && smem_panel)
                gj_update<T, NBS><<<dim3(tiles, tiles, P.nbox), 256, 0, st>>>(P.dbox, S, rows, m, j0, k);
            else if (sizeof(T) == 4)
                gj_update<T, 32><<<dim3(tiles, tiles, P.nbox), 256, 0, st>>>(P.dbox, S, rows, m, j0, k);
            else
                gj_update<T, 16><<<dim3(tiles, tiles, P.nbox), 256, 0, st>>>(P.dbox, S, rows, m, j0, k);
            prof_end(ctx, t, ub);
            ctx->launches += 2;
        }
        gj_store<T><<<dim3(std::max(1, std::min(64, m / 16)), P.nbox), 256, m * sizeof(int), st>>>(P.dbox, S, perm,
                                                                                                    G, m, k);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cleanup();
            return cuda_check(ctx, e, "plane factorisation launch");
        }
    }
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    rc = cuda_check(ctx, cudaStreamSynchronize(st), "plane factorisation");
    cleanup();
    *singular = hflag;
    return rc;
}

// ------------------------------------------------------------------ block-pivot Gauss-Jordan (CUDA cores)
//
// The same elimination as the tensor-core factorisation (planelu_tc.cu), for complex128 and complex64 sets
// on the CUDA cores: NB-column panels J (BgjNB), P = A[J,J]^{-1} with partial pivoting inside the block,
// A[J,:] = P A[J,:] (A[J,J] = P), and for the rows outside J A[I,j] = [j not in J] A[I,j] - W[I,:] A[J,j]
// with W = A[:, J] copied before the step.  The rank-NB update is spread over every SM (64 x 64 output
// tiles), where the fully pivoted elimination above eliminates one column at a time in one CTA per box.
// panel width: 64 columns for complex64 sets, 32 for complex128 (the block inverse's cost per panel grows as NB^3
// and runs in one CTA per box on the FP64 pipe; the coarse problem is a single box)
template <typename T> struct BgjNB { static constexpr int v = 64; };
template <> struct BgjNB<double> { static constexpr int v = 32; };

template <typename T>
__global__ void __launch_bounds__(512) bgj_diag(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ S,
                                                int m_max, cplx<T>* __restrict__ Pbuf, int* __restrict__ flag, int j0,
                                                int k) {
    constexpr int NB = BgjNB<T>::v, DP = NB + 1;
    extern __shared__ __align__(16) unsigned char bgj_sm[];
    cplx<T>* X = reinterpret_cast<cplx<T>*>(bgj_sm);   // [NB][DP]
    __shared__ cplx<T> s_row[NB], s_col[NB];
    __shared__ int s_perm[NB], s_pos[NB];
    __shared__ int s_piv;
    __shared__ T s_wmax[16];
    const BoxInfo B = boxes[blockIdx.x];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int nbw = min(NB, m - j0);
    const cplx<T>* A = S + (size_t)blockIdx.x * m_max * m_max;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    T amax = 0;
    for (int e = tid; e < NB * NB; e += 512) {
        const int r = e / NB, c = e % NB;
        cplx<T> v = mk<T>(r == c ? (T)1 : (T)0, (T)0);   // identity beyond a partial panel
        if (r < nbw && c < nbw) v = A[(size_t)(j0 + r) * m + j0 + c];
        X[r * DP + c] = v;
        amax = max(amax, v.x * v.x + v.y * v.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) s_wmax[wid] = amax;
    __syncthreads();
    amax = 0;
    for (int w = 0; w < 16; ++w) amax = max(amax, s_wmax[w]);
    block_inverse<T, NB, DP, 16, 512>(X, X + NB * DP, s_perm, s_row, s_col, &s_piv, amax, flag);
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
    cplx<T>* Pb = Pbuf + (size_t)blockIdx.x * NB * NB;
    for (int e = tid; e < NB * NB; e += 512) Pb[e] = X[(e / NB) * DP + s_pos[e % NB]];
}

// R = P A[J, :] for 64 columns per CTA, written into rows J (R[:, J] = P).  Thread (tx, ty): rows tx + 16 i,
// columns col0 + ty + 16 q.
template <typename T>
__global__ void __launch_bounds__(256) bgj_rows(const BoxInfo* __restrict__ boxes, cplx<T>* __restrict__ S, int m_max,
                                                const cplx<T>* __restrict__ Pbuf, int j0, int k) {
    constexpr int NB = BgjNB<T>::v;
    __shared__ cplx<T> Ps[NB][17];
    __shared__ cplx<T> As[16][64];
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int col0 = blockIdx.x * 64;
    if (col0 >= m) return;
    const int nbw = min(NB, m - j0);
    cplx<T>* A = S + (size_t)blockIdx.y * m_max * m_max;
    const cplx<T>* P = Pbuf + (size_t)blockIdx.y * NB * NB;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    cplx<T> acc[NB / 16][4];
#pragma unroll
    for (int i = 0; i < NB / 16; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = mk<T>(0, 0);
    for (int k0 = 0; k0 < NB; k0 += 16) {
        for (int e = tid; e < NB * 16; e += 256) Ps[e >> 4][e & 15] = P[(e >> 4) * NB + k0 + (e & 15)];
        for (int e = tid; e < 16 * 64; e += 256) {
            const int kk = e >> 6, jj = e & 63;
            As[kk][jj] = (k0 + kk < nbw && col0 + jj < m) ? A[(size_t)(j0 + k0 + kk) * m + col0 + jj] : mk<T>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            cplx<T> a[NB / 16], b[4];
#pragma unroll
            for (int i = 0; i < NB / 16; ++i) a[i] = Ps[tx + 16 * i][kk];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = As[kk][ty + 16 * q];
#pragma unroll
            for (int i = 0; i < NB / 16; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) cmac(acc[i][q], a[i], b[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int j = col0 + ty + 16 * q;
        if (j >= m) continue;
        const bool inJ = j >= j0 && j < j0 + nbw;
#pragma unroll
        for (int i = 0; i < NB / 16; ++i) {
            const int c = tx + 16 * i;
            if (c < nbw) A[(size_t)(j0 + c) * m + j] = inJ ? P[c * NB + (j - j0)] : acc[i][q];
        }
    }
}

// W = A[:, J] (rows J and columns beyond the panel zero), [m_max][NB] per box
template <typename T>
__global__ void bgj_wcopy(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ S, int m_max,
                          cplx<T>* __restrict__ Wbuf, int j0, int k) {
    constexpr int NB = BgjNB<T>::v;
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int nbw = min(NB, m - j0);
    const cplx<T>* A = S + (size_t)blockIdx.y * m_max * m_max;
    cplx<T>* W = Wbuf + (size_t)blockIdx.y * m_max * NB;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * NB; e += gridDim.x * blockDim.x) {
        const int I = e / NB, c = e % NB;
        W[e] = (c < nbw && !(I >= j0 && I < j0 + nbw)) ? A[(size_t)I * m + j0 + c] : mk<T>(0, 0);
    }
}

// A[I, j] = [j not in J] A[I, j] - sum_c W[I, c] A[j0 + c, j] for rows I outside J; 64 x 64 tiles, 4 x 4 per thread
template <typename T>
__global__ void __launch_bounds__(256) bgj_update(const BoxInfo* __restrict__ boxes, cplx<T>* __restrict__ S,
                                                  int m_max, const cplx<T>* __restrict__ Wbuf, int j0, int k) {
    constexpr int NB = BgjNB<T>::v;
    const BoxInfo B = boxes[blockIdx.z];
    const int m = B.m;
    if (k >= B.dims[2] || j0 >= m) return;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int nbw = min(NB, m - j0);
    if (r0 >= m || c0 >= m || (r0 >= j0 && r0 + 64 <= j0 + nbw)) return;   // a tile of rows J only
    cplx<T>* A = S + (size_t)blockIdx.z * m_max * m_max;
    const cplx<T>* W = Wbuf + (size_t)blockIdx.z * m_max * NB;
    __shared__ cplx<T> Ws[64][17];
    __shared__ cplx<T> Rs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    cplx<T> acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk<T>(0, 0);
    for (int k0 = 0; k0 < nbw; k0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            const int r = e >> 4, kk = e & 15;
            Ws[r][kk] = r0 + r < m ? W[(size_t)(r0 + r) * NB + k0 + kk] : mk<T>(0, 0);
            const int kr = e >> 6, jj = e & 63;
            Rs[kr][jj] = (k0 + kr < nbw && c0 + jj < m) ? A[(size_t)(j0 + k0 + kr) * m + c0 + jj] : mk<T>(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            cplx<T> w[4], rr[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) w[a] = Ws[ty + 16 * a][kk];
#pragma unroll
            for (int b = 0; b < 4; ++b) rr[b] = Rs[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) cmac(acc[a][b], w[a], rr[b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = r0 + ty + 16 * a;
        if (r >= m || (r >= j0 && r < j0 + nbw)) continue;   // rows J hold the panel's new rows
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = c0 + tx + 16 * b;
            if (j >= m) continue;
            cplx<T>* dst = A + (size_t)r * m + j;
            const cplx<T> base = (j >= j0 && j < j0 + nbw) ? mk<T>(0, 0) : *dst;
            *dst = base - acc[a][b];
        }
    }
}

template <typename T>
__global__ void bgj_store(const BoxInfo* __restrict__ boxes, const cplx<T>* __restrict__ S, cplx<T>* __restrict__ G,
                          int m_max, int k) {
    const BoxInfo B = boxes[blockIdx.y];
    const int m = B.m;
    if (k >= B.dims[2]) return;
    const cplx<T>* A = S + (size_t)blockIdx.y * m_max * m_max;
    cplx<T>* Gk = G + B.fac_off + (size_t)k * B.pstride;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)m * m;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / m), j = (int)(e % m);
        Gk[(size_t)r * B.ld + j] = A[e];
    }
}

// Block-pivot factorisation of a set on the CUDA cores.  *weak: a block pivot below 1e-6 of its block.
template <typename T>
helm_status factor_block_t(helm_ctx ctx, PlaneSet& P, int* singular, int* weak) {
    *singular = *weak = 0;
    cudaStream_t st = ctx->stream;
    constexpr int NB = BgjNB<T>::v;
    const size_t mm = (size_t)P.m_max * P.m_max;
    cplx<T>*S = nullptr, *Tm = nullptr, *W = nullptr, *Pb = nullptr;
    int* flag = nullptr;
    auto cleanup = [&]() {
        dev_free(ctx, S, P.nbox * mm * sizeof(cplx<T>));
        dev_free(ctx, Tm, P.nbox * mm * sizeof(cplx<T>));
        dev_free(ctx, W, (size_t)P.nbox * P.m_max * NB * sizeof(cplx<T>));
        dev_free(ctx, Pb, (size_t)P.nbox * NB * NB * sizeof(cplx<T>));
        dev_free(ctx, flag, sizeof(int));
    };
    helm_status rc;
    if ((rc = dev_alloc(ctx, (void**)&S, P.nbox * mm * sizeof(cplx<T>), "factor work S")) ||
        (rc = dev_alloc(ctx, (void**)&Tm, P.nbox * mm * sizeof(cplx<T>), "factor work T")) ||
        (rc = dev_alloc(ctx, (void**)&W, (size_t)P.nbox * P.m_max * NB * sizeof(cplx<T>), "factor panel W")) ||
        (rc = dev_alloc(ctx, (void**)&Pb, (size_t)P.nbox * NB * NB * sizeof(cplx<T>), "block pivots")) ||
        (rc = dev_alloc(ctx, (void**)&flag, sizeof(int), "factor flag"))) {
        cleanup();
        return rc;
    }
    static std::atomic<bool> attr{false};
    if (!attr.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(bgj_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((NB * (NB + 1) + 16 * NB) * sizeof(cplx<T>)));
        attr.store(true, std::memory_order_release);
    }
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    const cplx<T>* coef = (const cplx<T>*)P.coef;
    const int m = P.m_max;
    const unsigned eblocks = (unsigned)std::min<long long>(((long long)m * m + 255) / 256, 4096);
    const dim3 egrid(eblocks, P.nbox);
    const int t64 = (m + 63) / 64;
    const unsigned wblocks = (unsigned)std::min<long long>(((long long)m * NB + 255) / 256, 1024);
    for (int k = 0; k < P.bz_max; ++k) {
        if (k == 0) {
            schur_init<T><<<egrid, 256, 0, st>>>(P.dbox, coef, S, m, k);
            ctx->launches++;
        } else {
            schur_gu<T><<<egrid, 256, 0, st>>>(P.dbox, coef, (const cplx<T>*)P.G, Tm, m, k);
            schur_lt<T><<<egrid, 256, 0, st>>>(P.dbox, coef, Tm, S, m, k);
            ctx->launches += 2;
        }
        for (int j0 = 0; j0 < m; j0 += NB) {
            double ub = 0;
            for (const auto& b : P.hbox)
                if (k < b.dims[2] && j0 < b.m) ub += 2.0 * (b.m - std::min(NB, b.m - j0)) * b.m * sizeof(cplx<T>);
            int t = prof_begin(ctx, "gj_diag");
            bgj_diag<T><<<P.nbox, 512, (NB * (NB + 1) + 16 * NB) * sizeof(cplx<T>), st>>>(P.dbox, S, m, Pb, flag, j0, k);
            prof_end(ctx, t, 0.0);
            t = prof_begin(ctx, "gj_panel");
            bgj_rows<T><<<dim3(t64, P.nbox), 256, 0, st>>>(P.dbox, S, m, Pb, j0, k);
            bgj_wcopy<T><<<dim3(wblocks, P.nbox), 256, 0, st>>>(P.dbox, S, m, W, j0, k);
            prof_end(ctx, t, 0.0);
            t = prof_begin(ctx, "gj_update");
            bgj_update<T><<<dim3(t64, t64, P.nbox), 256, 0, st>>>(P.dbox, S, m, W, j0, k);
            prof_end(ctx, t, ub);
            ctx->launches += 4;
        }
        bgj_store<T><<<dim3(std::max(1, std::min(64, m / 16)), P.nbox), 256, 0, st>>>(P.dbox, S, (cplx<T>*)P.G, m, k);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            cleanup();
            return cuda_check(ctx, e, "block plane factorisation launch");
        }
    }
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    rc = cuda_check(ctx, cudaStreamSynchronize(st), "block plane factorisation");
    cleanup();
    *singular = hflag & 1;
    *weak = (hflag >> 1) & 1;
    return rc;
}

template <typename T, int RN>
void launch_sweep_rn(const PlaneSet& P, cplx<T>* loc, cplx<T>* rbuf, int nrhs, cudaStream_t st, helm_ctx ctx) {
    const int m = P.m_max;
    // rows per CTA: at most 64, fewer when there are few boxes, so that the grid covers every SM twice
    const int chunks = (nrhs + RN - 1) / RN;
    const long long want = 2LL * std::max(1, ctx->sm_count);
    int rows_per = (int)std::min<long long>(64, std::max<long long>(8, (long long)m * P.nbox * chunks / want / 8 * 8));
    const dim3 ggrid((m + rows_per - 1) / rows_per, P.nbox, (nrhs + RN - 1) / RN);
    const size_t smem = (size_t)RN * m * sizeof(cplx<T>);
    const unsigned pblocks = (unsigned)std::min<long long>(((long long)m * nrhs + 255) / 256, 1024);
    const dim3 pgrid(pblocks, P.nbox);
    const cplx<T>* coef = (const cplx<T>*)P.coef;
    const cplx<T>* G = (const cplx<T>*)P.G;
    static std::atomic<bool> attr_set{false};
    if (!attr_set.load(std::memory_order_acquire)) {
        cudaFuncSetAttribute(sweep_gemv<T, RN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(sweep_gemv<T, RN, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set.store(true, std::memory_order_release);
    }
    // algorithmic bytes of one step: every active box reads its m x m factor plane once,
    // the prepared plane (m x nrhs) and writes (backward: also reads) its output plane;
    // the preparation reads 1 + 9 planes of coefficients and vectors, writes one plane.
    const double es = sizeof(cplx<T>);
    auto step_bytes = [&](int s, bool fwd, double& gemv, double& prep) {
        gemv = prep = 0;
        for (const auto& b : P.hbox) {
            const int bz = b.dims[2];
            const bool act = fwd ? s < bz : (s >= 1 && s <= bz - 1);
            if (!act) continue;
            gemv += ((double)b.m * b.m + (fwd ? 2.0 : 3.0) * b.m * nrhs) * es;
            prep += ((double)b.m * 9 + (fwd ? 3.0 : 2.0) * b.m * nrhs) * es;
        }
    };
    double gb, pb;
    if (P.nbox == 1) {
        // one box: split K so that the grid still covers the GPU
        const int kw = (m + KSPLIT - 1) / KSPLIT;
        const int rows = 32;
        const dim3 sgrid((m + rows - 1) / rows, KSPLIT, (nrhs + RN - 1) / RN);
        const size_t ssm = (size_t)RN * kw * sizeof(cplx<T>);
        cplx<T>* part = rbuf + (size_t)m * nrhs;   // the caller sizes rbuf (1 + KSPLIT) planes deep
        static std::atomic<bool> sattr{false};
        if (!sattr.load(std::memory_order_acquire)) {
            cudaFuncSetAttribute(sweep_gemv_splitk<T, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            sattr.store(true, std::memory_order_release);
        }
        const unsigned rblocks = (unsigned)std::min<long long>(((long long)m * nrhs + 255) / 256, 512);
        for (int pass = 0; pass < 2; ++pass) {
            const int fwd = pass == 0;
            for (int s = fwd ? 0 : 1; s < P.bz_max; ++s) {
                step_bytes(s, fwd, gb, pb);
                int t = prof_begin(ctx, "coarse_prep");
                if (fwd) sweep_prep<T, true><<<pgrid, 256, 0, st>>>(P.dbox, coef, loc, rbuf, m, nrhs, s);
                else sweep_prep<T, false><<<pgrid, 256, 0, st>>>(P.dbox, coef, loc, rbuf, m, nrhs, s);
                prof_end(ctx, t, pb);
                t = prof_begin(ctx, "coarse_sweep");
                sweep_gemv_splitk<T, RN><<<sgrid, 256, ssm, st>>>(P.dbox, G, rbuf, part, m, nrhs, s, fwd, rows);
                sweep_reduce<T><<<rblocks, 256, 0, st>>>(P.dbox, part, loc, m, nrhs, s, fwd);
                prof_end(ctx, t, gb);
                ctx->launches += 3;
            }
        }
        return;
    }
    for (int s = 0; s < P.bz_max; ++s) {
        step_bytes(s, true, gb, pb);
        int t = prof_begin(ctx, "sweep_prep");
        sweep_prep<T, true><<<pgrid, 256, 0, st>>>(P.dbox, coef, loc, rbuf, m, nrhs, s);
        prof_end(ctx, t, pb);
        t = prof_begin(ctx, "sweep_gemv");
        sweep_gemv<T, RN, true><<<ggrid, 256, smem, st>>>(P.dbox, G, rbuf, loc, m, nrhs, s, rows_per);
        prof_end(ctx, t, gb);
    }
    for (int s = 1; s < P.bz_max; ++s) {
        step_bytes(s, false, gb, pb);
        int t = prof_begin(ctx, "sweep_prep");
        sweep_prep<T, false><<<pgrid, 256, 0, st>>>(P.dbox, coef, loc, rbuf, m, nrhs, s);
        prof_end(ctx, t, pb);
        t = prof_begin(ctx, "sweep_gemv");
        sweep_gemv<T, RN, false><<<ggrid, 256, smem, st>>>(P.dbox, G, rbuf, loc, m, nrhs, s, rows_per);
        prof_end(ctx, t, gb);
    }
    ctx->launches += 4 * P.bz_max - 2;
}

template <typename T>
helm_status solve_t(helm_ctx ctx, const PlaneSet& P, cplx<T>* loc, cplx<T>* rbuf, int nrhs, cudaStream_t st) {
    const size_t per = (size_t)P.m_max * sizeof(cplx<T>);
    const size_t cap = 200 * 1024;
    int rn = 16;
    while (rn > 1 && (rn > nrhs * 2 || rn * per > cap)) rn >>= 1;
    while (rn > 1 && rn >= 2 * nrhs) rn >>= 1;
    if (rn * per > cap) return set_error(ctx, HELM_EINVAL, "plane size %d too large for the sweep kernel", P.m_max);
    switch (rn) {
        case 16: launch_sweep_rn<T, 16>(P, loc, rbuf, nrhs, st, ctx); break;
        case 8: launch_sweep_rn<T, 8>(P, loc, rbuf, nrhs, st, ctx); break;
        case 4: launch_sweep_rn<T, 4>(P, loc, rbuf, nrhs, st, ctx); break;
        case 2: launch_sweep_rn<T, 2>(P, loc, rbuf, nrhs, st, ctx); break;
        default: launch_sweep_rn<T, 1>(P, loc, rbuf, nrhs, st, ctx); break;
    }
    return cuda_check(ctx, cudaGetLastError(), "plane sweeps");
}

}  // namespace

helm_status planeset_alloc(helm_ctx ctx, PlaneSet& P) {
    P.nbox = (int)P.hbox.size();
    P.m_max = 0;
    P.bz_max = 0;
    for (auto& b : P.hbox) {
        b.m = b.dims[0] * b.dims[1];
        P.m_max = std::max(P.m_max, b.m);
        P.bz_max = std::max(P.bz_max, b.dims[2]);
    }
    P.ld = P.padded ? (P.m_max + 15) / 16 * 16 : 0;
    long long loc = 0;
    size_t fac = 0;
    int planes = 0;
    for (auto& b : P.hbox) {
        b.loc_off = loc;
        b.fac_off = (long long)fac;
        b.plane0 = planes;
        b.ld = P.padded ? P.ld : b.m;
        b.pstride = P.padded ? padded_pstride(P.ld) : (long long)b.m * b.m;
        loc += (long long)b.m * b.dims[2];
        fac += (size_t)b.pstride * b.dims[2];
        planes += b.dims[2];
    }
    P.nloc = loc;
    P.fac_entries = fac;
    P.nplanes = planes;
    HELM_TRY(dev_alloc(ctx, (void**)&P.dbox, P.nbox * sizeof(BoxInfo), "box table"));
    HELM_CUDA(ctx, cudaMemcpyAsync(P.dbox, P.hbox.data(), P.nbox * sizeof(BoxInfo), cudaMemcpyHostToDevice,
                                   ctx->stream));
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    HELM_TRY(dev_alloc(ctx, &P.coef, (size_t)P.nloc * 27 * P.cesize(), "local operator coefficients"));
    if (P.coef_only) return HELM_OK;
    HELM_TRY(dev_alloc(ctx, &P.G, P.fac_entries * P.esize(), "plane factors"));
    if (P.padded) HELM_CUDA(ctx, cudaMemsetAsync(P.G, 0, P.fac_entries * P.esize(), ctx->stream));
    return HELM_OK;
}

void planeset_free(helm_ctx ctx, PlaneSet& P) {
    dev_free(ctx, P.dbox, P.nbox * sizeof(BoxInfo));
    dev_free(ctx, P.coef, (size_t)P.nloc * 27 * P.cesize());
    dev_free(ctx, P.G, P.fac_entries * P.esize());
    P.dbox = nullptr;
    P.coef = P.G = nullptr;
}

helm_status planeset_factor(helm_ctx ctx, PlaneSet& P, int* singular) {
    int weak = 0;
    if (P.prec == HELM_PREC_FP32 && P.padded && ctx->tc_factor) {
        HELM_TRY(planeset_factor_tc(ctx, P, singular, &weak));
        if (!weak && !*singular) return HELM_OK;
        ctx->factor_fallbacks++;   // a tiny (or zero) block pivot: factor the set again with full partial pivoting
    } else if (!P.padded && ctx->block_gj) {
        if (P.prec == HELM_PREC_FP64) HELM_TRY(factor_block_t<double>(ctx, P, singular, &weak));
        else HELM_TRY(factor_block_t<float>(ctx, P, singular, &weak));
        if (!weak && !*singular) return HELM_OK;
        ctx->factor_fallbacks++;
    }
    if (P.prec == HELM_PREC_FP64) return factor_t<double>(ctx, P, singular);
    return factor_t<float>(ctx, P, singular);
}

namespace {
__global__ void to_bf16_pairs(const c64* __restrict__ a, __nv_bfloat162* __restrict__ b, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = __floats2bfloat162_rn(a[i].x, a[i].y);
}
}  // namespace

// Replace complex64 factors by bfloat16 pairs (same layout), freeing the complex64 copy.
helm_status planeset_to_bf16(helm_ctx ctx, PlaneSet& P) {
    if (P.prec != HELM_PREC_FP32) return set_error(ctx, HELM_EINVAL, "planeset_to_bf16: factors are not complex64");
    void* g16 = nullptr;
    HELM_TRY(dev_alloc(ctx, &g16, P.fac_entries * 4, "bf16 plane factors"));
    to_bf16_pairs<<<(unsigned)std::min<size_t>((P.fac_entries + 255) / 256, 65535), 256, 0, ctx->stream>>>(
        (const c64*)P.G, (__nv_bfloat162*)g16, P.fac_entries);
    ctx->launches++;
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, P.G, P.fac_entries * sizeof(c64));
    P.G = g16;
    P.prec = HELM_PREC_BF16;
    return HELM_OK;
}

helm_status planeset_solve(helm_ctx ctx, const PlaneSet& P, void* loc, void* rbuf, int nrhs, cudaStream_t st,
                           int* err) {
    if (P.prec == HELM_PREC_FP64) return solve_t<double>(ctx, P, (c128*)loc, (c128*)rbuf, nrhs, st);
    if (err && ctx->coarse_coop) {
        bool done = false;
        HELM_TRY(planeset_solve_coop(ctx, P, (c64*)loc, (c64*)rbuf, nrhs, st, err, &done));
        if (done) return HELM_OK;
    }
    return solve_t<float>(ctx, P, (c64*)loc, (c64*)rbuf, nrhs, st);
}
