// In-place inverse of an NB x NB complex block held in shared memory, for the panel step of the block-pivot
// Gauss-Jordan factorisations (planelu.cu, planelu_tc.cu): Gauss-Jordan with partial pivoting inside the
// block, in sub-panels of SB columns.  Within a sub-panel each column is eliminated on the sub-panel's
// columns only (whole rows are swapped at once); the accumulated transform W of the sub-panel then reaches
// the other columns B in one rank-SB step, B <- [rows outside the sub-panel] B + W[:, sub] B[sub rows, :]
// (the rows of B it reads are copied out first), so the per-column work is NB x SB instead of NB x NB.
// On return X holds the inverse of the row-permuted block; the caller undoes the permutation (s_perm: the
// pivot row chosen at each column).  flag bit 0: a zero pivot (replaced by 1 to stay finite); bit 1: a pivot
// below 1e-6 of the block's largest entry (amax is the largest |x|^2 of the block).
#pragma once
#include "internal.h"

template <typename T, int NB, int DP, int SB, int NT>
__device__ __forceinline__ void block_inverse(cplx<T>* X, cplx<T>* Brow, int* s_perm, cplx<T>* s_row, cplx<T>* s_col,
                                              int* s_piv, T amax, int* flag) {
    static_assert(NB % SB == 0 && NT % 32 == 0 && NT >= NB, "block_inverse: shape");
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int c0 = 0; c0 < NB; c0 += SB) {
        for (int c = c0; c < c0 + SB; ++c) {
            if (wid == 0) {
                T best = -1;
                int bi = NB;
                for (int r = c + lane; r < NB; r += 32) {
                    const cplx<T> v = X[r * DP + c];
                    const T a = v.x * v.x + v.y * v.y;
                    if (a > best) { best = a; bi = r; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (lane == 0) {
                    if (!(best > (T)0) || bi >= NB) {
                        atomicOr(flag, 1);
                        bi = c;
                    } else if (best < (T)1e-12 * amax) {
                        atomicOr(flag, 2);
                    }
                    *s_piv = bi;
                    s_perm[c] = bi;
                }
            }
            __syncthreads();
            const int p = *s_piv;
            if (p != c)
                for (int j = tid; j < NB; j += NT) {
                    const cplx<T> t = X[c * DP + j];
                    X[c * DP + j] = X[p * DP + j];
                    X[p * DP + j] = t;
                }
            __syncthreads();
            cplx<T> piv = X[c * DP + c];
            if (!(piv.x * piv.x + piv.y * piv.y > (T)0)) piv = mk<T>((T)1, (T)0);   // flagged above
            const T d = piv.x * piv.x + piv.y * piv.y;
            const cplx<T> inv = mk<T>(piv.x / d, -piv.y / d);
            if (tid < NB) s_col[tid] = X[tid * DP + c];
            if (tid < SB) s_row[tid] = (c0 + tid == c) ? inv : X[c * DP + c0 + tid] * inv;
            __syncthreads();
            for (int e = tid; e < NB * SB; e += NT) {
                const int r = e / SB, jj = e % SB, j = c0 + jj;
                cplx<T>& x = X[r * DP + j];
                if (r == c) {
                    x = s_row[jj];
                } else if (j == c) {
                    const cplx<T> v = s_col[r] * inv;
                    x = mk<T>(-v.x, -v.y);
                } else {
                    const cplx<T> f = s_col[r], sv = s_row[jj];
                    x.x -= f.x * sv.x - f.y * sv.y;
                    x.y -= f.x * sv.y + f.y * sv.x;
                }
            }
            __syncthreads();
        }
        // the sub-panel's transform on the other columns
        for (int e = tid; e < SB * NB; e += NT) {
            const int c = e / NB, j = e % NB;
            Brow[e] = X[(c0 + c) * DP + j];
        }
        __syncthreads();
        for (int e = tid; e < NB * NB; e += NT) {
            const int r = e / NB, j = e % NB;
            if (j >= c0 && j < c0 + SB) continue;
            cplx<T> acc = (r >= c0 && r < c0 + SB) ? mk<T>((T)0, (T)0) : X[r * DP + j];
#pragma unroll
            for (int c = 0; c < SB; ++c) cmac(acc, X[r * DP + c0 + c], Brow[c * NB + j]);
            X[r * DP + j] = acc;
        }
        __syncthreads();
    }
}
