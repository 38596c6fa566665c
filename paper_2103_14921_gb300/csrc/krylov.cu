// Right-preconditioned restarted GMRES / flexible GMRES (the paper's Krylov
// solver, with M^{-1} of Eq. 2lvl), one independent Krylov space per
// right-hand side, all right-hand sides batched in every kernel.
//
//   x0 = 0, r = b, beta = ||r||, v_0 = r / beta, g = beta e_0
//   for j = 0 .. restart-1:
//     z_j = M^{-1} v_j ; w = A z_j
//     CGS2: h = V^H w, w -= V h, h' = V^H w, w -= V h', h += h' (FP64 sums)
//     h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
//     complex Givens rotations (real cosine) on column j, g updated,
//     |g_{j+1}| / ||b|| <= tol stops that column's cycle
//   y = R^{-1} g ; x += Z y (FGMRES) or x += M^{-1} (V y) (GMRES)
//   true residual ||b - A x|| / ||b|| in FP64; restart the columns above tol.
//
// Vectors (basis V, Z, w) are complex128 or complex64 (basis_prec); x, the
// true residual, the Hessenberg matrix, the rotations and every reduction
// are FP64.  Reductions are two-pass (per-block partials, then a fixed-order
// sum), so results do not depend on scheduling.
#include <math.h>
#include <string.h>

#include "internal.h"

namespace {

constexpr int RED_THREADS = 256;
constexpr int IC = 8;   // basis vectors handled per pass of a dot-product kernel

// Number of reduction blocks: the grid stride (blocks x 256) must be a multiple
// of nrhs so that every thread only ever touches one right-hand side.  At most two
// blocks per SM (the reduction kernels run two resident blocks each): one wave, so
// each block's closing block-wide reduction is amortised over as many elements as
// possible and no partial wave trails.
inline int red_blocks(helm_ctx ctx, long long elems, int nrhs) {
    int a = RED_THREADS, b = nrhs;
    while (b) { const int t = a % b; a = b; b = t; }
    const long long q = nrhs / a;   // nrhs / gcd(256, nrhs)
    long long nb = (elems + RED_THREADS - 1) / RED_THREADS;
    const long long cap = std::max(q, ((long long)std::max(1, ctx->sm_count) * 2 / q) * q);
    nb = ((nb + q - 1) / q) * q;
    return (int)std::min(nb, cap);
}

template <typename T> __device__ __forceinline__ c128 widen(cplx<T> a) { return mk<double>((double)a.x, (double)a.y); }

// Per-thread accumulators of the reductions.  complex64 data: compensated (Kahan) FP32 sums, which
// keep the error of a thread's sum near one rounding of the FP32 inputs without FP64 arithmetic in the
// element loops (FP64 issues far slower than FP32 on this part); the thread totals are then reduced
// in FP64.  complex128 data: plain FP64 sums.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}
template <typename T> struct CAcc;
template <> struct CAcc<float> {
    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
    __device__ __forceinline__ void add(c64 v) {
        kahan_add(sx, cx, v.x);
        kahan_add(sy, cy, v.y);
    }
    __device__ __forceinline__ c128 value() const { return mk<double>((double)sx - (double)cx, (double)sy - (double)cy); }
};
template <> struct CAcc<double> {
    c128 s = {0.0, 0.0};
    __device__ __forceinline__ void add(c128 v) { s = s + v; }
    __device__ __forceinline__ c128 value() const { return s; }
};
template <typename T> struct RAcc;
template <> struct RAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) { kahan_add(s, c, v); }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct RAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

// partial[blk][i][r] = sum over this block's elements of conj(V_i[e]) w[e], i in [i0, i0+ni),
// and with npart also |w|^2.  Runs on the reduction grid (grid stride a multiple of nrhs, so each
// thread keeps one column).  EPT elements per loop trip and IC basis vectors per pass keep EPT * (IC+1)
// independent loads in flight (EPT = 8 for bases of up to 2 vectors, else 2); products in the basis
// precision are summed in groups of up to 8 before they are added to the thread's accumulator (CAcc);
// one FP64 block-wide reduction per pass.
template <typename T, int EPT = 2>
__global__ void __launch_bounds__(RED_THREADS, 2) dots_kernel(const cplx<T>* __restrict__ V, long long vstride,
                                                              const cplx<T>* __restrict__ w, long long n_el, int nrhs,
                                                              int i0, int ni, c128* __restrict__ partial, int ldp,
                                                              double* __restrict__ npart,
                                                              const int* __restrict__ any) {
    __shared__ c128 s[IC][RED_THREADS];
    __shared__ double sn[RED_THREADS];
    if (any && *any == 0) return;
    const long long t = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
    const long long stride = (long long)gridDim.x * RED_THREADS;
    for (int ib = 0; ib < ni; ib += IC) {
        const int nq = min(IC, ni - ib);
        const bool with_norm = npart && ib == 0;
        CAcc<T> acc[IC];
        cplx<T> part[IC];
#pragma unroll
        for (int q = 0; q < IC; ++q) part[q] = mk<T>(0, 0);
        RAcc<T> nrm;
        T pn = (T)0;
        int cnt = 0;
        const cplx<T>* Vb = V + (long long)(i0 + ib) * vstride;
        constexpr int QL = EPT > 2 ? 2 : IC;   // basis vectors loaded per trip (IC, or 2 with 8 elements)
        long long e = t;
        for (; e + (EPT - 1) * stride < n_el; e += EPT * stride) {
            cplx<T> wv[EPT];
            cplx<T> a[EPT][QL];
#pragma unroll
            for (int u = 0; u < EPT; ++u) wv[u] = w[e + u * stride];
#pragma unroll
            for (int u = 0; u < EPT; ++u)
#pragma unroll
                for (int q = 0; q < QL; ++q)
                    if (q < nq) a[u][q] = Vb[(long long)q * vstride + e + u * stride];
#pragma unroll
            for (int u = 0; u < EPT; ++u)
#pragma unroll
                for (int q = 0; q < QL; ++q)
                    if (q < nq) cmac_conj(part[q], a[u][q], wv[u]);
            if (with_norm)
#pragma unroll
                for (int u = 0; u < EPT; ++u) pn += wv[u].x * wv[u].x + wv[u].y * wv[u].y;
            if ((cnt += EPT) >= 8) {
#pragma unroll
                for (int q = 0; q < IC; ++q) {
                    if (q < nq) acc[q].add(part[q]);
                    part[q] = mk<T>(0, 0);
                }
                nrm.add(pn);
                pn = (T)0;
                cnt = 0;
            }
        }
        // the last, partial trip: at most EPT - 1 elements, each product added once
        for (int u = 0; u < (EPT == 2 ? 1 : EPT - 1) && e < n_el; ++u, e += stride) {
            const cplx<T> w0 = w[e];
#pragma unroll
            for (int q = 0; q < QL; ++q)
                if (q < nq) cmac_conj(part[q], Vb[(long long)q * vstride + e], w0);
            if (with_norm) pn += w0.x * w0.x + w0.y * w0.y;
        }
#pragma unroll
        for (int q = 0; q < IC; ++q) {
            acc[q].add(part[q]);
            s[q][threadIdx.x] = acc[q].value();
        }
        nrm.add(pn);
        if (with_norm) sn[threadIdx.x] = nrm.value();
        __syncthreads();
        const int nr = min(nrhs, RED_THREADS);
        for (int o = threadIdx.x; o < nq * nr; o += RED_THREADS) {
            const int q = o / nr, u0 = o % nr;
            c128 sum = mk<double>(0, 0);
            for (int u = u0; u < RED_THREADS; u += nrhs) sum = sum + s[q][u];
            const int r = (int)(((long long)blockIdx.x * RED_THREADS + u0) % nrhs);
            partial[((long long)blockIdx.x * ldp + (i0 + ib + q)) * nrhs + r] = sum;
        }
        if (with_norm && threadIdx.x < nr) {
            double sum = 0.0;
            for (int u = threadIdx.x; u < RED_THREADS; u += nrhs) sum += sn[u];
            const int r = (int)(((long long)blockIdx.x * RED_THREADS + threadIdx.x) % nrhs);
            npart[(long long)blockIdx.x * nrhs + r] = sum;
        }
        __syncthreads();
    }
}

// out[i][r] (+)= sum_blk partial[blk][i][r]: one 128-thread block per (i, r); thread t sums the
// partials t, t+128, ... in order, then a fixed shuffle and shared-memory tree (deterministic).
__device__ __forceinline__ c128 block_sum128(c128 v) {
    __shared__ c128 red[4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return (red[0] + red[1]) + (red[2] + red[3]);
}

__global__ void __launch_bounds__(128) finish_dots(const c128* __restrict__ partial, int nblk, int ldp, int ni,
                                                   int nrhs, c128* __restrict__ H, int ldh_i, int ldh_r, int col,
                                                   int accumulate, const int* __restrict__ colmask,
                                                   const int* __restrict__ any) {
    const int i = blockIdx.x / nrhs, r = blockIdx.x % nrhs;
    if (i >= ni) return;
    if (any && *any == 0) return;
    if (colmask && !colmask[r]) return;
    c128 sum = mk<double>(0, 0);
    for (int b = threadIdx.x; b < nblk; b += 128) sum = sum + partial[((long long)b * ldp + i) * nrhs + r];
    sum = block_sum128(sum);
    if (threadIdx.x == 0) {
        c128* dst = H + (long long)r * ldh_r + (long long)i * ldh_i + col;
        *dst = accumulate ? *dst + sum : sum;
    }
}

// w -= V h for the columns selected by colmask (all when colmask is null; none when *any == 0),
// and npart[blk][r] = |w|^2 of the result over this block's elements.  Runs on the reduction grid
// (grid stride a multiple of nrhs), so each thread keeps one column; the coefficients h are staged
// in shared memory in the basis precision when they fit (ni * nrhs entries).
template <typename T>
__global__ void __launch_bounds__(RED_THREADS, 2) update_norm_kernel(const cplx<T>* __restrict__ V, long long vstride,
                                                                  cplx<T>* __restrict__ w, long long n_el, int nrhs,
                                                                  int ni, const c128* __restrict__ hsrc,
                                                                  const int* __restrict__ colmask,
                                                                  const int* __restrict__ any,
                                                                  double* __restrict__ npart, int hsmem) {
    extern __shared__ __align__(16) unsigned char upd_smem[];
    cplx<T>* hs = reinterpret_cast<cplx<T>*>(upd_smem);
    __shared__ double sn[RED_THREADS];
    const long long t = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
    const long long stride = (long long)gridDim.x * RED_THREADS;
    const int r = (int)(t % nrhs);
    const bool project = (!any || *any != 0) && (!colmask || colmask[r]);
    if (hsmem)
        for (int e = threadIdx.x; e < ni * nrhs; e += RED_THREADS) hs[e] = mk<T>((T)hsrc[e].x, (T)hsrc[e].y);
    __syncthreads();
    RAcc<T> nrm;
    // two elements per trip (e and e + stride, the same column): batches of 2 x 8 independent basis
    // loads, then the multiply-subtracts
    for (long long e = t; e < n_el; e += 2 * stride) {
        const bool two = e + stride < n_el;
        const long long e1 = two ? e + stride : e;
        cplx<T> acc0 = w[e], acc1 = w[e1];
        if (project) {
            for (int i0 = 0; i0 < ni; i0 += 8) {
                cplx<T> v0[8], v1[8];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (i0 + q < ni) {
                        v0[q] = V[(long long)(i0 + q) * vstride + e];
                        v1[q] = V[(long long)(i0 + q) * vstride + e1];
                    }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (i0 + q < ni) {
                        cplx<T> h;
                        if (hsmem) h = hs[(i0 + q) * nrhs + r];
                        else h = mk<T>((T)hsrc[(long long)(i0 + q) * nrhs + r].x, (T)hsrc[(long long)(i0 + q) * nrhs + r].y);
                        acc0.x -= h.x * v0[q].x - h.y * v0[q].y;
                        acc0.y -= h.x * v0[q].y + h.y * v0[q].x;
                        acc1.x -= h.x * v1[q].x - h.y * v1[q].y;
                        acc1.y -= h.x * v1[q].y + h.y * v1[q].x;
                    }
                }
            }
            w[e] = acc0;
            if (two) w[e1] = acc1;
        }
        nrm.add(acc0.x * acc0.x + acc0.y * acc0.y);
        if (two) nrm.add(acc1.x * acc1.x + acc1.y * acc1.y);
    }
    sn[threadIdx.x] = nrm.value();
    __syncthreads();
    if (threadIdx.x < min(nrhs, RED_THREADS)) {
        double sum = 0.0;
        for (int u = threadIdx.x; u < RED_THREADS; u += nrhs) sum += sn[u];
        const int rr = (int)(((long long)blockIdx.x * RED_THREADS + threadIdx.x) % nrhs);
        npart[(long long)blockIdx.x * nrhs + rr] = sum;
    }
}

// Fused first update and second projection of CGS2 (IM >= ni basis vectors): every element's ni basis
// values are loaded once into registers, w' = w - V h1 is written, and the partials of V^H w' (the second
// projection's coefficients, plain FP32 sums per thread: they only correct rounding-level remainders) and of
// |w'|^2 (compensated) are reduced per block.  Runs on the reduction grid (one column per thread), one
// resident block per SM.
// HS: the coefficients h are read from shared memory at every use instead of being held in registers
// (needs ni * nrhs <= 16 IM); the freed registers carry twice as many elements per trip.
template <typename T, int IM, bool HS = false>
__global__ void __launch_bounds__(RED_THREADS, IM <= 4 ? 2 : 1) update_dots_kernel(const cplx<T>* __restrict__ V, long long vstride,
                                                                    cplx<T>* __restrict__ w, long long n_el, int nrhs,
                                                                    int ni, const c128* __restrict__ hsrc,
                                                                    c128* __restrict__ partial, int ldp,
                                                                    double* __restrict__ npart) {
    __shared__ cplx<T> hs[IM * 16];
    __shared__ c128 s[8][RED_THREADS];
    __shared__ double sn[RED_THREADS];
    const long long t = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
    const long long stride = (long long)gridDim.x * RED_THREADS;
    const int r = (int)(t % nrhs);
    const bool hsm = ni * nrhs <= IM * 16;
    if (hsm)
        for (int e = threadIdx.x; e < ni * nrhs; e += RED_THREADS) hs[e] = mk<T>((T)hsrc[e].x, (T)hsrc[e].y);
    __syncthreads();
    cplx<T> h[HS ? 1 : IM];
    if (!HS) {
#pragma unroll
        for (int q = 0; q < IM; ++q)
            if (q < ni) {
                if (hsm) h[q] = hs[q * nrhs + r];
                else h[q] = mk<T>((T)hsrc[(long long)q * nrhs + r].x, (T)hsrc[(long long)q * nrhs + r].y);
            }
    }
    cplx<T> acc[IM];
#pragma unroll
    for (int q = 0; q < IM; ++q) acc[q] = mk<T>(0, 0);
    RAcc<T> nrm;
    // EPT elements per trip (e, e + stride, ...: the same column), so that every trip keeps the same number
    // of basis loads in flight whatever IM is
    // (bases of up to 4 vectors: 8 elements (8 / IM in FP64), two blocks per SM)
    constexpr int EPT0 = IM <= 4 ? (sizeof(T) == 4 ? 8 : 8 / IM)
                                 : ((sizeof(T) == 4 ? 32 : 16) / IM > 0 ? (sizeof(T) == 4 ? 32 : 16) / IM : 1);
    constexpr int EPT = HS ? 2 * EPT0 : EPT0;
    for (long long e0 = t; e0 < n_el; e0 += EPT * stride) {
        cplx<T> v[EPT][IM];
        cplx<T> x[EPT];
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
            const long long e = e0 + u * stride;
            const long long ec = e < n_el ? e : e0;
#pragma unroll
            for (int q = 0; q < IM; ++q)
                if (q < ni) v[u][q] = V[(long long)q * vstride + ec];
            x[u] = w[ec];
        }
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
            const long long e = e0 + u * stride;
            if (e >= n_el) break;
#pragma unroll
            for (int q = 0; q < IM; ++q)
                if (q < ni) {
                    const cplx<T> hq = HS ? hs[q * nrhs + r] : h[HS ? 0 : q];
                    x[u].x -= hq.x * v[u][q].x - hq.y * v[u][q].y;
                    x[u].y -= hq.x * v[u][q].y + hq.y * v[u][q].x;
                }
            w[e] = x[u];
            nrm.add(x[u].x * x[u].x + x[u].y * x[u].y);
#pragma unroll
            for (int q = 0; q < IM; ++q)
                if (q < ni) cmac_conj(acc[q], v[u][q], x[u]);
        }
    }
    sn[threadIdx.x] = nrm.value();
    const int nr = min(nrhs, RED_THREADS);
    // block reduction of the ni coefficients in groups of 8 (fixed order)
#pragma unroll
    for (int q0 = 0; q0 < IM; q0 += 8) {
        if (q0 >= ni) break;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q][threadIdx.x] = q0 + q < IM ? widen(acc[min(q0 + q, IM - 1)]) : mk<double>(0, 0);
        __syncthreads();
        const int nq = min(8, ni - q0);
        for (int o = threadIdx.x; o < nq * nr; o += RED_THREADS) {
            const int q = o / nr, u0 = o % nr;
            c128 sum = mk<double>(0, 0);
            for (int u = u0; u < RED_THREADS; u += nrhs) sum = sum + s[q][u];
            const int rr = (int)(((long long)blockIdx.x * RED_THREADS + u0) % nrhs);
            partial[((long long)blockIdx.x * ldp + q0 + q) * nrhs + rr] = sum;
        }
    }
    __syncthreads();
    if (threadIdx.x < nr) {
        double sum = 0.0;
        for (int u = threadIdx.x; u < RED_THREADS; u += nrhs) sum += sn[u];
        const int rr = (int)(((long long)blockIdx.x * RED_THREADS + threadIdx.x) % nrhs);
        npart[(long long)blockIdx.x * nrhs + rr] = sum;
    }
}

// Second update of CGS2 fused with the normalisation: out = (w' - V h2) * inv[r] (inv = 0 writes zeros, for
// the columns whose cycle has stopped).  EPT elements per trip and batches of QB basis loads (EPT * QB = 16,
// more elements for fewer basis vectors, so that short bases still keep 16 loads in flight per thread).
template <typename T, int EPT, int QB>
__global__ void __launch_bounds__(RED_THREADS, 2) update_scale_kernel(const cplx<T>* __restrict__ V, long long vstride,
                                                                     const cplx<T>* __restrict__ w,
                                                                     cplx<T>* __restrict__ out, long long n_el,
                                                                     int nrhs, int ni, const c128* __restrict__ hsrc,
                                                                     const double* __restrict__ inv) {
    extern __shared__ __align__(16) unsigned char us_smem[];
    cplx<T>* hs = reinterpret_cast<cplx<T>*>(us_smem);
    const long long t = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
    const long long stride = (long long)gridDim.x * RED_THREADS;
    const int r = (int)(t % nrhs);
    for (int e = threadIdx.x; e < ni * nrhs; e += RED_THREADS) hs[e] = mk<T>((T)hsrc[e].x, (T)hsrc[e].y);
    __syncthreads();
    const T sc = (T)inv[r];
    for (long long e0 = t; e0 < n_el; e0 += EPT * stride) {
        cplx<T> acc[EPT];
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
            const long long e = e0 + u * stride;
            acc[u] = w[e < n_el ? e : e0];
        }
        for (int i0 = 0; i0 < ni; i0 += QB) {
            cplx<T> v[EPT][QB];
#pragma unroll
            for (int u = 0; u < EPT; ++u) {
                const long long e = e0 + u * stride;
                const long long ec = e < n_el ? e : e0;
#pragma unroll
                for (int q = 0; q < QB; ++q)
                    if (i0 + q < ni) v[u][q] = V[(long long)(i0 + q) * vstride + ec];
            }
#pragma unroll
            for (int q = 0; q < QB; ++q)
                if (i0 + q < ni) {
                    const cplx<T> h = hs[(i0 + q) * nrhs + r];
#pragma unroll
                    for (int u = 0; u < EPT; ++u) {
                        acc[u].x -= h.x * v[u][q].x - h.y * v[u][q].y;
                        acc[u].y -= h.x * v[u][q].y + h.y * v[u][q].x;
                    }
                }
        }
#pragma unroll
        for (int u = 0; u < EPT; ++u) {
            const long long e = e0 + u * stride;
            if (e < n_el) out[e] = mk<T>(acc[u].x * sc, acc[u].y * sc);
        }
    }
}

// ||w''|| = sqrt(||w'||^2 - ||h2||^2) per column (V orthonormal; h2 is a rounding-level correction, so there
// is no cancellation), as the subdiagonal entry H[j+1][j].
__global__ void second_norm(const double* __restrict__ nw, const c128* __restrict__ h2, int ni, int nrhs,
                            double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    double s = nw[r] * nw[r];
    for (int i = 0; i < ni; ++i) {
        const c128 a = h2[(long long)i * nrhs + r];
        s -= a.x * a.x + a.y * a.y;
    }
    out[r] = sqrt(fmax(s, 0.0));
}

// Re-orthogonalisation test per column: a second projection when ||w'|| < ||w|| / sqrt(2).
__global__ void reorth_flags(const double* __restrict__ before, const double* __restrict__ after, int* __restrict__ flag,
                             int* __restrict__ any, int nrhs) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int a = 0;
    for (int r = 0; r < nrhs; ++r) {
        const int f = after[r] < 0.70710678118654752 * before[r];
        flag[r] = f;
        a |= f;
    }
    *any = a;
}

// partial[blk][r] = sum |v[e]|^2 over this block's elements
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) norm2_kernel(const cplx<T>* __restrict__ v, long long n_el, int nrhs,
                                                            double* __restrict__ partial) {
    __shared__ double s[RED_THREADS];
    const long long t = (long long)blockIdx.x * RED_THREADS + threadIdx.x;
    const long long stride = (long long)gridDim.x * RED_THREADS;
    double acc = 0.0;
    for (long long e = t; e < n_el; e += stride) {
        const c128 a = widen(v[e]);
        acc += a.x * a.x + a.y * a.y;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < min(nrhs, RED_THREADS)) {
        double sum = 0.0;
        for (int u = threadIdx.x; u < RED_THREADS; u += nrhs) sum += s[u];
        const int r = (int)(((long long)blockIdx.x * RED_THREADS + threadIdx.x) % nrhs);
        partial[(long long)blockIdx.x * nrhs + r] = sum;
    }
}

__global__ void __launch_bounds__(128) finish_norm2(const double* __restrict__ partial, int nblk, int nrhs,
                                                    double* __restrict__ out) {
    __shared__ double red[4];
    const int r = blockIdx.x;
    double sum = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 128) sum += partial[(long long)b * nrhs + r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) out[r] = sqrt((red[0] + red[1]) + (red[2] + red[3]));
}

// Column index of a grid-stride loop over [N][nrhs] entries without a 64-bit division per entry:
// one at the start, then the stride's remainder is added each trip.
struct ColumnWalk {
    int r, step, n;
    __device__ ColumnWalk(long long e0, long long stride, int nrhs)
        : r((int)(e0 % nrhs)), step((int)(stride % nrhs)), n(nrhs) {}
    __device__ __forceinline__ void next() {
        r += step;
        if (r >= n) r -= n;
    }
};

// dst[e] = src[e] * scale[r]  (scale = 0 -> zero)
template <typename TS, typename TD>
__global__ void scale_copy(const cplx<TS>* __restrict__ src, cplx<TD>* __restrict__ dst, long long n_el, int nrhs,
                           const double* __restrict__ scale) {
    const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    ColumnWalk cw(e0, stride, nrhs);
    for (long long e = e0; e < n_el; e += stride, cw.next()) {
        const int r = cw.r;
        const cplx<TS> a = src[e];
        if (sizeof(TS) == 4 && sizeof(TD) == 4) {   // complex64 -> complex64: FP32 arithmetic
            const float s = (float)scale[r];
            dst[e] = mk<TD>((TD)(s * (float)a.x), (TD)(s * (float)a.y));
        } else {
            const double s = scale[r];
            dst[e] = mk<TD>((TD)(s * (double)a.x), (TD)(s * (double)a.y));
        }
    }
}


// Start of a cycle: inv[r] = 1/beta for active columns, g = beta e_0.
__global__ void cycle_start(RhsState* __restrict__ S, const double* __restrict__ beta, double* __restrict__ inv,
                            c128* __restrict__ g, int m, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    RhsState& s = S[r];
    s.steps = 0;
    s.active = !s.done && beta[r] > 0.0;
    inv[r] = s.active ? 1.0 / beta[r] : 0.0;
    for (int i = 0; i <= m; ++i) g[(long long)r * (m + 1) + i] = mk<double>(0, 0);
    g[(long long)r * (m + 1)] = mk<double>(s.active ? beta[r] : 0.0, 0.0);
}

// Column j of H for every rhs: apply earlier rotations, make a new one, update g and the estimate.
// H[r][i][j] is (m+1) x m per rhs; hnorm[r] = ||w|| = H[j+1][j]; inv[r] <- 1/hnorm (or 0).
__global__ void givens_step(RhsState* __restrict__ S, c128* __restrict__ H, double* __restrict__ cs,
                            c128* __restrict__ sn, c128* __restrict__ g, const double* __restrict__ hnorm,
                            double* __restrict__ inv, int j, int m, int nrhs, int* __restrict__ running) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    RhsState& s = S[r];
    if (!s.active) {
        inv[r] = 0.0;
        return;
    }
    c128* h = H + (long long)r * (m + 1) * m;
    double* c = cs + (long long)r * m;
    c128* sv = sn + (long long)r * m;
    c128* gg = g + (long long)r * (m + 1);
    const double hn = hnorm[r];
    h[(long long)(j + 1) * m + j] = mk<double>(hn, 0.0);
    for (int i = 0; i < j; ++i) {
        const c128 a = h[(long long)i * m + j], b = h[(long long)(i + 1) * m + j];
        const c128 si = sv[i];
        const c128 sb = si * b;
        const c128 csa = mk<double>(c[i] * a.x, c[i] * a.y);
        h[(long long)i * m + j] = csa + sb;
        // -conj(s) a + c b
        const c128 sca = mk<double>(si.x * a.x + si.y * a.y, si.x * a.y - si.y * a.x);
        h[(long long)(i + 1) * m + j] = mk<double>(c[i] * b.x - sca.x, c[i] * b.y - sca.y);
    }
    const c128 a = h[(long long)j * m + j], b = h[(long long)(j + 1) * m + j];
    const double na = hypot(a.x, a.y), nbv = hypot(b.x, b.y);
    double cc;
    c128 ss;
    if (nbv == 0.0) {
        cc = 1.0;
        ss = mk<double>(0, 0);
    } else if (na == 0.0) {
        cc = 0.0;
        ss = mk<double>(b.x / nbv, -b.y / nbv);
    } else {
        const double t = hypot(na, nbv);
        cc = na / t;
        const c128 ua = mk<double>(a.x / na, a.y / na);
        const c128 cb = mk<double>(b.x / t, -b.y / t);
        ss = ua * cb;
    }
    c[j] = cc;
    sv[j] = ss;
    h[(long long)j * m + j] = mk<double>(cc * a.x, cc * a.y) + ss * b;
    h[(long long)(j + 1) * m + j] = mk<double>(0, 0);
    const c128 gj = gg[j];
    gg[j + 1] = mk<double>(-(ss.x * gj.x + ss.y * gj.y), -(ss.x * gj.y - ss.y * gj.x));
    gg[j] = mk<double>(cc * gj.x, cc * gj.y);
    s.steps = j + 1;
    s.iters += 1;
    s.est = hypot(gg[j + 1].x, gg[j + 1].y) / s.bnorm;
    const bool stop = s.est <= s.tol || hn == 0.0 || s.iters >= s.maxit || j + 1 >= m;
    inv[r] = (hn > 0.0 && !stop) ? 1.0 / hn : 0.0;
    if (stop) s.active = 0;
    else atomicAdd(running, 1);
}

// y = R^{-1} g for the steps taken this cycle (upper-triangular back substitution).
// y32 (when not null) receives y rounded to complex64 for the FP32 combination kernel.
__global__ void back_substitute(const RhsState* __restrict__ S, const c128* __restrict__ H, const c128* __restrict__ g,
                                c128* __restrict__ y, c64* __restrict__ y32, int m, int nrhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    const int nsteps = S[r].steps;
    const c128* h = H + (long long)r * (m + 1) * m;
    const c128* gg = g + (long long)r * (m + 1);
    for (int i = 0; i < m; ++i) y[(long long)i * nrhs + r] = mk<double>(0, 0);
    for (int i = nsteps - 1; i >= 0; --i) {
        c128 acc = gg[i];
        for (int k = i + 1; k < nsteps; ++k) {
            const c128 p = h[(long long)i * m + k] * y[(long long)k * nrhs + r];
            acc = acc - p;
        }
        const c128 d = h[(long long)i * m + i];
        const double den = d.x * d.x + d.y * d.y;
        y[(long long)i * nrhs + r] =
            den > 0 ? mk<double>((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den) : mk<double>(0, 0);
    }
    if (y32)
        for (int i = 0; i < m; ++i) {
            const c128 v = y[(long long)i * nrhs + r];
            y32[(long long)i * nrhs + r] = mk<float>((float)v.x, (float)v.y);
        }
}

// x[e] += sum_i Zb_i[e] y_i[r]  (FP64 accumulation into complex128 x)   -- or u = sum_i Zb_i y_i (into TU)
template <typename T, typename TO, bool ACC>
__global__ void combine_kernel(const cplx<T>* __restrict__ Zb, long long zstride, const c128* __restrict__ y,
                               cplx<TO>* __restrict__ x, long long n_el, int nrhs, int ni) {
    const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    ColumnWalk cw(e0, stride, nrhs);
    for (long long e = e0; e < n_el; e += stride, cw.next()) {
        const int r = cw.r;
        c128 acc = ACC ? widen(x[e]) : mk<double>(0, 0);
        for (int i = 0; i < ni; ++i) cmac(acc, widen(Zb[(long long)i * zstride + e]), y[(long long)i * nrhs + r]);
        x[e] = mk<TO>((TO)acc.x, (TO)acc.y);
    }
}

// The same for a complex64 basis: products and their compensated sum in FP32, then x[e] += sum in
// FP64 (TO = double, FGMRES) or u[e] = sum (TO = float, GMRES).
template <typename TO>
__global__ void combine32(const c64* __restrict__ Zb, long long zstride, const c64* __restrict__ y32,
                          cplx<TO>* __restrict__ x, long long n_el, int nrhs, int ni) {
    const long long e0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    ColumnWalk cw(e0, stride, nrhs);
    for (long long e = e0; e < n_el; e += stride, cw.next()) {
        const int r = cw.r;
        CAcc<float> acc;
        for (int i = 0; i < ni; ++i) acc.add(Zb[(long long)i * zstride + e] * y32[(long long)i * nrhs + r]);
        if (sizeof(TO) == 8) {
            const c128 v = widen(x[e]) + acc.value();
            x[e] = mk<TO>((TO)v.x, (TO)v.y);
        } else {
            x[e] = mk<TO>((TO)(acc.sx - acc.cx), (TO)(acc.sy - acc.cy));
        }
    }
}

// x += u (u widened to FP64)
template <typename T>
__global__ void accum_widen(const cplx<T>* __restrict__ u, c128* __restrict__ x, long long n_el) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (long long)gridDim.x * blockDim.x)
        x[e] = x[e] + widen(u[e]);
}

// column-masked set-up of new columns: x = 0, r = b (mask[r] != 0)
__global__ void start_columns_kernel(const c128* __restrict__ B, c128* __restrict__ X, c128* __restrict__ R,
                                     const int* __restrict__ mask, long long n_el, int nrhs) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (long long)gridDim.x * blockDim.x) {
        if (!mask[e % nrhs]) continue;
        X[e] = mk<double>(0, 0);
        R[e] = B[e];
    }
}

// bad |= 1 when a masked column of v has NaN/Inf
__global__ void finite_check_cols(const c128* __restrict__ v, const int* __restrict__ mask, long long n_el, int nrhs,
                                  int* __restrict__ bad) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (long long)gridDim.x * blockDim.x)
        if (mask[e % nrhs] && (!isfinite(v[e].x) || !isfinite(v[e].y))) atomicOr(bad, 1);
}

// ------------------------------------------------------------------ host driver

// Batched (F)GMRES over S columns: workspaces, per-column state and one restart cycle at a time.
template <typename T>
struct Krylov final : KrylovEngine {
    helm_oras o = nullptr;
    helm_ctx ctx = nullptr;
    cudaStream_t st = nullptr;
    int S = 0, m = 0, wp = 0;
    bool flex = true;
    long long N = 0, nel = 0;
    int nblk = 0, ldp = 0;
    unsigned eg = 0, rg = 0;
    std::vector<std::pair<void*, size_t>> allocs;
    cplx<T>*V = nullptr, *Zb = nullptr, *w = nullptr, *u = nullptr;
    c128 *Bd = nullptr, *Xd = nullptr, *r = nullptr, *H = nullptr, *sn = nullptr, *gv = nullptr, *y = nullptr;
    c128 *part = nullptr, *hpass = nullptr;
    c64* y32 = nullptr;
    double *cs = nullptr, *dpart = nullptr, *beta = nullptr, *inv = nullptr, *hn = nullptr;
    RhsState* Sd = nullptr;
    int *running = nullptr, *mask = nullptr, *rflag = nullptr, *rany = nullptr;
    double *nb = nullptr, *na = nullptr;
    int hsmem_cap = 0;
    std::vector<RhsState> hs;
    std::vector<double> trel;
    // one captured CUDA graph per iteration index j (its kernels depend on j through the basis offsets)
    struct IterGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<ProfRecord> recs;   // external event nodes of profiled families
        uint64_t launches = 0;          // kernels in the graph
        uint64_t ctx_gen = 0, scratch_gen = 0;
        int uses = 0;
        bool failed = false;
    };
    bool graphs = false;
    std::vector<IterGraph> ig;

    helm_status alloc(void** p, size_t bytes, const char* what) {
        helm_status rc = dev_alloc(ctx, p, bytes, what);
        if (!rc && *p) allocs.push_back({*p, bytes});
        return rc;
    }
    ~Krylov() override {
        if (ctx) {
            cudaStreamSynchronize(st);
            for (auto& g : ig) drop(g);
            for (auto& a : allocs) dev_free(ctx, a.first, a.second);
        }
    }
    void drop(IterGraph& g) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        prof_release(ctx, g.recs);
    }
    void rebind(c128* B_ext, c128* X_ext) override {
        Bd = B_ext;
        Xd = X_ext;
    }
    void enable_graphs(bool on) override {
        graphs = on;
        if (!on)
            for (auto& g : ig) drop(g);
    }
    c128* B() override { return Bd; }
    c128* X() override { return Xd; }
    int slots() const override { return S; }
    const RhsState& state(int c) const override { return hs[c]; }
    double true_rel(int c) const override { return trel[c]; }
    size_t bytes() const override {
        size_t b = 0;
        for (auto& a : allocs) b += a.second;
        return b;
    }

    helm_status init(helm_oras o_, int S_, int restart, bool flexible, int basis_prec, c128* B_ext, c128* X_ext) {
        o = o_;
        ctx = o->g->ctx;
        st = ctx->stream;
        S = S_;
        m = restart;
        flex = flexible;
        wp = basis_prec;
        N = o->g->n;
        nel = N * S;
        nblk = red_blocks(ctx, nel, S);
        ldp = m + 1;
        eg = (unsigned)std::min<long long>((nel + 255) / 256, (long long)ctx->sm_count * 16);
        rg = (unsigned)((S + 127) / 128);
        if (B_ext) Bd = B_ext;
        else HELM_TRY(alloc((void**)&Bd, nel * sizeof(c128), "batch right-hand sides"));
        if (X_ext) Xd = X_ext;
        else HELM_TRY(alloc((void**)&Xd, nel * sizeof(c128), "batch solutions"));
        HELM_TRY(alloc((void**)&V, (size_t)(m + 1) * nel * sizeof(cplx<T>), "Krylov basis V"));
        if (flex) HELM_TRY(alloc((void**)&Zb, (size_t)m * nel * sizeof(cplx<T>), "Krylov basis Z"));
        HELM_TRY(alloc((void**)&w, nel * sizeof(cplx<T>), "Arnoldi vector"));
        HELM_TRY(alloc((void**)&u, nel * sizeof(cplx<T>), "preconditioned vector"));
        HELM_TRY(alloc((void**)&r, nel * sizeof(c128), "residual"));
        HELM_TRY(alloc((void**)&H, (size_t)S * (m + 1) * m * sizeof(c128), "Hessenberg"));
        HELM_TRY(alloc((void**)&sn, (size_t)S * m * sizeof(c128), "Givens sines"));
        HELM_TRY(alloc((void**)&cs, (size_t)S * m * sizeof(double), "Givens cosines"));
        HELM_TRY(alloc((void**)&gv, (size_t)S * (m + 1) * sizeof(c128), "Givens rhs"));
        HELM_TRY(alloc((void**)&y, (size_t)S * m * sizeof(c128), "least-squares solution"));
        if (sizeof(T) == 4)
            HELM_TRY(alloc((void**)&y32, (size_t)S * m * sizeof(c64), "least-squares solution (complex64)"));
        HELM_TRY(alloc((void**)&part, (size_t)nblk * ldp * S * sizeof(c128), "dot partials"));
        HELM_TRY(alloc((void**)&hpass, (size_t)ldp * S * sizeof(c128), "dot pass"));
        HELM_TRY(alloc((void**)&dpart, (size_t)nblk * S * sizeof(double), "norm partials"));
        HELM_TRY(alloc((void**)&beta, S * sizeof(double), "norms"));
        HELM_TRY(alloc((void**)&inv, S * sizeof(double), "inverse norms"));
        HELM_TRY(alloc((void**)&hn, S * sizeof(double), "new norms"));
        HELM_TRY(alloc((void**)&Sd, S * sizeof(RhsState), "column state"));
        HELM_TRY(alloc((void**)&running, 2 * sizeof(int), "running flag"));
        HELM_TRY(alloc((void**)&mask, S * sizeof(int), "column mask"));
        HELM_TRY(alloc((void**)&rflag, S * sizeof(int), "re-orthogonalisation flags"));
        HELM_TRY(alloc((void**)&rany, sizeof(int), "re-orthogonalisation any"));
        HELM_TRY(alloc((void**)&nb, S * sizeof(double), "norms before projection"));
        HELM_TRY(alloc((void**)&na, S * sizeof(double), "norms after projection"));
        hsmem_cap = 40 * 1024 / (int)sizeof(cplx<T>);   // coefficient entries kept in shared memory (<= 40 KB)
        ig.resize(m);
        hs.assign(S, RhsState{0.0, 0, 0, 0, 1, 0.0, 0.0, 0});
        trel.assign(S, 0.0);
        HELM_CUDA(ctx, cudaMemcpyAsync(Sd, hs.data(), S * sizeof(RhsState), cudaMemcpyHostToDevice, st));
        if (!X_ext) HELM_CUDA(ctx, cudaMemsetAsync(Xd, 0, nel * sizeof(c128), st));
        if (!B_ext) HELM_CUDA(ctx, cudaMemsetAsync(Bd, 0, nel * sizeof(c128), st));
        HELM_CUDA(ctx, cudaMemsetAsync(r, 0, nel * sizeof(c128), st));
        return HELM_OK;
    }

    template <typename V_t>
    void norms(const V_t* vec, double* out) {
        const int tk = prof_begin(ctx, "krylov_misc");
        norm2_kernel<<<nblk, RED_THREADS, 0, st>>>(vec, nel, S, dpart);
        finish_norm2<<<S, 128, 0, st>>>(dpart, nblk, S, out);
        prof_end(ctx, tk, (double)nel * sizeof(*vec));
        ctx->launches += 2;
    }

    // partials of V^H w (and, with npart, of |w|^2) into `part`; skipped on the device when *any == 0
    // (profiled as "arnoldi", or "arnoldi_reorth" for the conditional second projection, whose
    // kernels return at once when no column needs it, so that the first family's bandwidth is exact)
    void dots_pass(const cplx<T>* Vb, const cplx<T>* vec, int ni, double* npart, const int* anyp) {
        const int tk = prof_begin(ctx, anyp ? "arnoldi_reorth" : "arnoldi");
        if (ni <= 2)
            dots_kernel<T, 8><<<nblk, RED_THREADS, 0, st>>>(Vb, nel, vec, nel, S, 0, ni, part, ldp, npart, anyp);
        else
            dots_kernel<T><<<nblk, RED_THREADS, 0, st>>>(Vb, nel, vec, nel, S, 0, ni, part, ldp, npart, anyp);
        prof_end(ctx, tk, (double)(ni + 1 + (npart ? 1 : 0)) * nel * sizeof(cplx<T>));
        ctx->launches++;
    }
    void finish_into(int ni, c128* dst, int ldh_i, int ldh_r, int col, int accumulate, const int* cm, const int* anyp) {
        finish_dots<<<ni * S, 128, 0, st>>>(part, nblk, ldp, ni, S, dst, ldh_i, ldh_r, col, accumulate, cm, anyp);
        ctx->launches++;
    }
    // w -= V h (masked), |w|^2 partials into dpart, then the norms into out
    void update_pass(int ni, const int* cm, const int* anyp, double* out) {
        const int hs = ni * S <= hsmem_cap ? 1 : 0;
        const size_t smem = hs ? (size_t)ni * S * sizeof(cplx<T>) : 0;
        const int tk = prof_begin(ctx, anyp ? "arnoldi_reorth" : "arnoldi");
        update_norm_kernel<T><<<nblk, RED_THREADS, smem, st>>>(V, nel, w, nel, S, ni, hpass, cm, anyp, dpart, hs);
        prof_end(ctx, tk, (double)(ni + 2) * nel * sizeof(cplx<T>));
        finish_norm2<<<S, 128, 0, st>>>(dpart, nblk, S, out);
        ctx->launches += 2;
    }

    // Start the listed columns (their b already in B()): x = 0, r = b, state reset.
    helm_status begin_columns(const int* cols, int n, const double* tol, const int* maxit, bool warm) override {
        if (warm && n != S) return set_error(ctx, HELM_EINVAL, "gmres_solve: a warm start lists every column");
        std::vector<int> hm(S, 0);
        for (int i = 0; i < n; ++i) hm[cols[i]] = 1;
        HELM_CUDA(ctx, cudaMemcpyAsync(mask, hm.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
        int* bad = running + 1;
        HELM_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), st));
        finite_check_cols<<<eg, 256, 0, st>>>(Bd, mask, nel, S, bad);
        ctx->launches++;
        if (warm) {
            finite_check_cols<<<eg, 256, 0, st>>>(Xd, mask, nel, S, bad);
            ctx->launches++;
        } else {
            start_columns_kernel<<<eg, 256, 0, st>>>(Bd, Xd, r, mask, nel, S);
            ctx->launches++;
        }
        norms(Bd, beta);
        std::vector<double> hb(S);
        int hbad = 0;
        HELM_CUDA(ctx, cudaMemcpyAsync(hb.data(), beta, S * sizeof(double), cudaMemcpyDeviceToHost, st));
        HELM_CUDA(ctx, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
        HELM_CUDA(ctx, cudaStreamSynchronize(st));
        if (hbad) return set_error(ctx, HELM_ENONFINITE, "gmres_solve: right-hand side or initial guess has NaN/Inf");
        if (warm) {
            // columns with b = 0 return x = 0; the others start from r = b - A x0 (FP64)
            std::vector<int> hz(S, 0);
            for (int c = 0; c < S; ++c) hz[c] = hb[c] == 0.0 ? 1 : 0;
            HELM_CUDA(ctx, cudaMemcpyAsync(mask, hz.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
            start_columns_kernel<<<eg, 256, 0, st>>>(Bd, Xd, r, mask, nel, S);
            ctx->launches++;
            HELM_TRY(launch_stencil_sub(o->g, HELM_PREC_FP64, Xd, Bd, r, S, st));
        }
        std::vector<double> hr(S, 0.0);
        if (warm) {
            norms(r, beta);
            HELM_CUDA(ctx, cudaMemcpyAsync(hr.data(), beta, S * sizeof(double), cudaMemcpyDeviceToHost, st));
            HELM_CUDA(ctx, cudaStreamSynchronize(st));
        }
        for (int i = 0; i < n; ++i) {
            const int c = cols[i];
            // a warm start that already meets its tolerance returns x0 with no iterations
            const double rel = hb[c] > 0.0 ? hr[c] / hb[c] : 0.0;
            if (warm && !std::isfinite(rel))
                return set_error(ctx, HELM_ENONFINITE, "gmres_solve: residual of the initial guess is NaN/Inf");
            const int done = hb[c] == 0.0 || (warm && rel <= tol[i]);
            hs[c] = RhsState{hb[c], 0, 0, 0, done, 0.0, tol[i], maxit[i]};
            trel[c] = warm ? rel : 0.0;
        }
        HELM_CUDA(ctx, cudaMemcpyAsync(Sd, hs.data(), S * sizeof(RhsState), cudaMemcpyHostToDevice, st));
        return HELM_OK;
    }

    // Leave column c out of the following cycles.
    void retire(int c) override {
        hs[c].done = 1;
        hs[c].bnorm = 0.0;
    }
    helm_status push_state() override {
        HELM_CUDA(ctx, cudaMemcpyAsync(Sd, hs.data(), S * sizeof(RhsState), cudaMemcpyHostToDevice, st));
        return HELM_OK;
    }

    // CGS2 in three passes over the basis (up to 32 basis vectors): h1 = V^H w; w' = w - V h1 fused with
    // h2 = V^H w' and ||w'||; H[.][j] = h1 + h2, H[j+1][j] = sqrt(||w'||^2 - ||h2||^2); the Givens step; then
    // v_{j+1} = (w' - V h2) / H[j+1][j] fused with the second update.
    helm_status cgs2_fused(int j) {
        const int ni = j + 1;
        // resident blocks per SM for the fused kernel (two for bases of up to 4 vectors, whose smaller register
        // arrays allow it), as the largest multiple of q <= that many blocks
        int a = RED_THREADS, bq = S;
        while (bq) { const int t = a % bq; a = bq; bq = t; }
        const int q = S / a;
        const int per_sm = ni <= 4 ? 2 : 1;
        const int nb1 = std::min(nblk, std::max(q, (per_sm * std::max(1, ctx->sm_count) / q) * q));
        dots_pass(V, w, ni, nullptr, nullptr);
        finish_into(ni, hpass, S, 1, 0, 0, nullptr, nullptr);
        finish_into(ni, H, m, (m + 1) * m, j, 0, nullptr, nullptr);
        {
            const int tk = prof_begin(ctx, "arnoldi");
            if (ni <= 2)
                update_dots_kernel<T, 2><<<nb1, RED_THREADS, 0, st>>>(V, nel, w, nel, S, ni, hpass, part, ldp, dpart);
            else if (ni <= 4)
                update_dots_kernel<T, 4><<<nb1, RED_THREADS, 0, st>>>(V, nel, w, nel, S, ni, hpass, part, ldp, dpart);
            else if (ni <= 8)
                update_dots_kernel<T, 8><<<nb1, RED_THREADS, 0, st>>>(V, nel, w, nel, S, ni, hpass, part, ldp, dpart);
            else if (ni <= 16 || sizeof(T) == 8)
                update_dots_kernel<T, 16><<<nb1, RED_THREADS, 0, st>>>(V, nel, w, nel, S, ni, hpass, part, ldp, dpart);
            else if (S <= 16)
                update_dots_kernel<T, (sizeof(T) == 4 ? 32 : 16), true><<<nb1, RED_THREADS, 0, st>>>(
                    V, nel, w, nel, S, ni, hpass, part, ldp, dpart);
            else
                update_dots_kernel<T, (sizeof(T) == 4 ? 32 : 16)><<<nb1, RED_THREADS, 0, st>>>(V, nel, w, nel, S, ni,
                                                                                           hpass, part, ldp, dpart);
            prof_end(ctx, tk, (double)(ni + 2) * nel * sizeof(cplx<T>));
        }
        finish_dots<<<ni * S, 128, 0, st>>>(part, nb1, ldp, ni, S, hpass, S, 1, 0, 0, nullptr, nullptr);
        finish_dots<<<ni * S, 128, 0, st>>>(part, nb1, ldp, ni, S, H, m, (m + 1) * m, j, 1, nullptr, nullptr);
        finish_norm2<<<S, 128, 0, st>>>(dpart, nb1, S, na);
        second_norm<<<rg, 128, 0, st>>>(na, hpass, ni, S, hn);
        ctx->launches += 5;
        HELM_CUDA(ctx, cudaMemsetAsync(running, 0, sizeof(int), st));
        givens_step<<<rg, 128, 0, st>>>(Sd, H, cs, sn, gv, hn, inv, j, m, S, running);
        {
            const int tk = prof_begin(ctx, "arnoldi");
            const size_t hsm = (size_t)ni * S * sizeof(cplx<T>);
            cplx<T>* vn = V + (long long)(j + 1) * nel;
            if (ni <= 2)
                update_scale_kernel<T, (sizeof(T) == 4 ? 8 : 4), (sizeof(T) == 4 ? 2 : 4)><<<nblk, RED_THREADS, hsm, st>>>(
                    V, nel, w, vn, nel, S, ni, hpass, inv);
            else if (ni <= 4)
                update_scale_kernel<T, 4, 4><<<nblk, RED_THREADS, hsm, st>>>(V, nel, w, vn, nel, S, ni, hpass, inv);
            else
                update_scale_kernel<T, 2, 8><<<nblk, RED_THREADS, hsm, st>>>(V, nel, w, vn, nel, S, ni, hpass, inv);
            prof_end(ctx, tk, (double)(ni + 2) * nel * sizeof(cplx<T>));
        }
        ctx->launches += 2;
        return cuda_check(ctx, cudaGetLastError(), "Krylov iteration");
    }

    // Iteration j of a cycle: z_j = M^{-1} v_j, w = A z_j, CGS with selective re-orthogonalisation,
    // the Givens step and v_{j+1}; no host synchronisation inside, so it can be captured as a graph.
    helm_status iteration_body(int j) {
        cplx<T>* vj = V + (long long)j * nel;
        cplx<T>* zj = flex ? Zb + (long long)j * nel : u;
        HELM_TRY(oras_apply_wp(o, wp, vj, zj, S));
        HELM_TRY(launch_stencil(o->g, wp, zj, w, S, st));
        // (complex128 bases: up to 16 vectors, the register budget of the fused kernel)
        if (j + 1 <= (sizeof(T) == 4 ? 32 : 16) && (size_t)(j + 1) * S * sizeof(cplx<T>) <= 40 * 1024)
            return cgs2_fused(j);
        // Classical Gram-Schmidt for column j of H (H[r][i][j]) with a second projection for the
        // columns whose norm dropped below 1/sqrt(2) of its value (selective re-orthogonalisation)
        dots_pass(V, w, j + 1, dpart, nullptr);
        finish_into(j + 1, hpass, S, 1, 0, 0, nullptr, nullptr);
        finish_into(j + 1, H, m, (m + 1) * m, j, 0, nullptr, nullptr);
        finish_norm2<<<S, 128, 0, st>>>(dpart, nblk, S, nb);
        ctx->launches++;
        update_pass(j + 1, nullptr, nullptr, na);
        reorth_flags<<<1, 32, 0, st>>>(nb, na, rflag, rany, S);
        ctx->launches++;
        dots_pass(V, w, j + 1, nullptr, rany);
        finish_into(j + 1, hpass, S, 1, 0, 0, nullptr, rany);
        finish_into(j + 1, H, m, (m + 1) * m, j, 1, rflag, rany);
        update_pass(j + 1, rflag, rany, hn);
        HELM_CUDA(ctx, cudaMemsetAsync(running, 0, sizeof(int), st));
        {
            const int tk = prof_begin(ctx, "krylov_misc");
            givens_step<<<rg, 128, 0, st>>>(Sd, H, cs, sn, gv, hn, inv, j, m, S, running);
            scale_copy<T, T><<<eg, 256, 0, st>>>(w, V + (long long)(j + 1) * nel, nel, S, inv);
            prof_end(ctx, tk, 2.0 * nel * sizeof(cplx<T>));
        }
        ctx->launches += 2;
        return cuda_check(ctx, cudaGetLastError(), "Krylov iteration");
    }

    // Run iteration j: eagerly on its first use, captured into a CUDA graph on the second, replayed
    // from the graph afterwards.  A graph is dropped when the ORAS scratch is reallocated or a
    // setting it depends on (tuning, profiling) changes; if capture fails the iteration stays eager.
    helm_status run_iteration(int j, IterGraph** replayed) {
        *replayed = nullptr;
        if (!graphs || !ctx->use_graphs) return iteration_body(j);
        IterGraph& G = ig[j];
        if (G.exec && (G.ctx_gen != ctx->graph_gen || G.scratch_gen != o->scratch_gen)) drop(G);
        if (!G.exec) {
            const bool ready = o->cap_nrhs >= S && o->cap_wp == wp;   // no allocation inside the capture
            if (G.failed || G.uses < 1 || !ready) {
                G.uses++;
                return iteration_body(j);
            }
            std::vector<ProfRecord> recs;
            cudaGraph_t g = nullptr;
            if (ctx->prof.on) prof_reserve(ctx, 1024);
            if (!ctx->cap_stream) HELM_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            // capture on the private stream (nothing runs during a capture, so the swap orders nothing);
            // the graph is launched on the context's stream
            cudaStream_t user = st;
            st = ctx->stream = ctx->cap_stream;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                st = ctx->stream = user;
                cudaGetLastError();
                G.failed = true;
                return iteration_body(j);
            }
            ctx->prof.capture = &recs;
            const uint64_t l0 = ctx->launches;
            const helm_status rc = iteration_body(j);
            ctx->prof.capture = nullptr;
            cudaError_t e = cudaStreamEndCapture(st, &g);
            st = ctx->stream = user;
            const uint64_t nl = ctx->launches - l0;
            ctx->launches = l0;
            if (rc == HELM_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&G.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (rc != HELM_OK || e != cudaSuccess || !G.exec) {
                cudaGetLastError();
                if (G.exec) cudaGraphExecDestroy(G.exec);
                G.exec = nullptr;
                prof_release(ctx, recs);
                G.failed = true;
                return iteration_body(j);
            }
            G.recs = std::move(recs);
            G.launches = nl;
            G.ctx_gen = ctx->graph_gen;
            G.scratch_gen = o->scratch_gen;
        }
        HELM_CUDA(ctx, cudaGraphLaunch(G.exec, st));
        ctx->launches += G.launches;
        *replayed = &G;
        return HELM_OK;
    }

    // One restart cycle for every column not done; then the FP64 true residual decides which are done.
    helm_status cycle(bool* any_left) override {
        norms(r, beta);
        cycle_start<<<rg, 128, 0, st>>>(Sd, beta, inv, gv, m, S);
        scale_copy<double, T><<<eg, 256, 0, st>>>(r, V, nel, S, inv);
        ctx->launches += 2;
        int jdone = 0;
        for (int j = 0; j < m; ++j) {
            IterGraph* replayed = nullptr;
            HELM_TRY(run_iteration(j, &replayed));
            int hrun = 0;
            HELM_CUDA(ctx, cudaMemcpyAsync(&hrun, running, sizeof(int), cudaMemcpyDeviceToHost, st));
            HELM_CUDA(ctx, cudaStreamSynchronize(st));
            HELM_CUDA(ctx, cudaGetLastError());
            if (replayed && ctx->prof.on && !replayed->recs.empty()) prof_harvest(ctx, replayed->recs);
            jdone = j + 1;
            if (hrun == 0) break;
        }
        // x update with the steps taken in this cycle
        back_substitute<<<rg, 128, 0, st>>>(Sd, H, gv, y, y32, m, S);
        ctx->launches++;
        if (flex) {
            const int tk = prof_begin(ctx, "krylov_misc");
            if (y32)
                combine32<double><<<eg, 256, 0, st>>>((const c64*)Zb, nel, y32, Xd, nel, S, jdone);
            else
                combine_kernel<T, double, true><<<eg, 256, 0, st>>>(Zb, nel, y, Xd, nel, S, jdone);
            prof_end(ctx, tk, (double)(jdone * sizeof(cplx<T>) + 2 * sizeof(c128)) * nel);
            ctx->launches++;
        } else {
            if (y32)
                combine32<float><<<eg, 256, 0, st>>>((const c64*)V, nel, y32, (c64*)w, nel, S, jdone);
            else
                combine_kernel<T, T, false><<<eg, 256, 0, st>>>(V, nel, y, w, nel, S, jdone);
            ctx->launches++;
            HELM_TRY(oras_apply_wp(o, wp, w, u, S));
            accum_widen<T><<<eg, 256, 0, st>>>(u, Xd, nel);
            ctx->launches++;
        }
        // true residual r = b - A x (FP64)
        HELM_TRY(launch_stencil_sub(o->g, HELM_PREC_FP64, Xd, Bd, r, S, st));
        norms(r, beta);
        std::vector<double> rn(S);
        HELM_CUDA(ctx, cudaMemcpyAsync(hs.data(), Sd, S * sizeof(RhsState), cudaMemcpyDeviceToHost, st));
        HELM_CUDA(ctx, cudaMemcpyAsync(rn.data(), beta, S * sizeof(double), cudaMemcpyDeviceToHost, st));
        HELM_CUDA(ctx, cudaStreamSynchronize(st));
        bool any = false;
        for (int i = 0; i < S; ++i) {
            if (hs[i].done) continue;
            trel[i] = hs[i].bnorm > 0 ? rn[i] / hs[i].bnorm : 0.0;
            if (!std::isfinite(trel[i])) return set_error(ctx, HELM_ENONFINITE, "gmres_solve: residual is NaN/Inf");
            if (trel[i] <= hs[i].tol || hs[i].iters >= hs[i].maxit) hs[i].done = 1;
            else any = true;
        }
        HELM_CUDA(ctx, cudaMemcpyAsync(Sd, hs.data(), S * sizeof(RhsState), cudaMemcpyHostToDevice, st));
        HELM_TRY(oras_check_device_error(o));
        *any_left = any;
        return HELM_OK;
    }
};

}  // namespace

KrylovEngine* make_krylov_engine(helm_oras o, int S, int restart, bool flexible, int basis_prec, c128* B_ext,
                                 c128* X_ext, helm_status* rc) {
    KrylovEngine* e = nullptr;
    if (basis_prec == HELM_PREC_FP64) {
        auto* k = new Krylov<double>();
        *rc = k->init(o, S, restart, flexible, basis_prec, B_ext, X_ext);
        e = k;
    } else {
        auto* k = new Krylov<float>();
        *rc = k->init(o, S, restart, flexible, basis_prec, B_ext, X_ext);
        e = k;
    }
    if (*rc) {
        delete e;
        return nullptr;
    }
    return e;
}

// ------------------------------------------------------------------ inexact coarse solve (inner GMRES)

namespace {

// Column state of the inner solve: tolerance 0 (only an exact zero residual stops a column early),
// iteration cap = the inner iteration count.
__global__ void inner_init(RhsState* __restrict__ S, const double* __restrict__ beta, int nrhs, int iters) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    S[r] = RhsState{beta[r], 0, 0, 0, beta[r] == 0.0 ? 1 : 0, 0.0, 0.0, iters};
}

}  // namespace

// Workspace of the inner GMRES over coarse vectors [nc][S].
struct InnerKrylov {
    int wp = 0, S = 0, m = 0, nblk = 0;
    long long nel = 0;
    std::vector<std::pair<void*, size_t>> allocs;
    void *V = nullptr, *w = nullptr, *u = nullptr;
    c128 *H = nullptr, *sn = nullptr, *gv = nullptr, *y = nullptr, *part = nullptr, *hpass = nullptr;
    c64* y32 = nullptr;
    double *cs = nullptr, *dpart = nullptr, *beta = nullptr, *inv = nullptr, *hn = nullptr, *nb = nullptr, *na = nullptr;
    RhsState* Sd = nullptr;
    int *running = nullptr, *rflag = nullptr, *rany = nullptr;
};

helm_status inner_alloc(helm_oras o, int wp, int nrhs) {
    helm_ctx ctx = o->g->ctx;
    inner_free(o);
    InnerKrylov* K = new InnerKrylov();
    o->inner = K;
    K->wp = wp;
    K->S = nrhs;
    K->m = o->d.coarse_iters;
    K->nel = o->nc * nrhs;
    K->nblk = red_blocks(ctx, K->nel, nrhs);
    const size_t te = wp == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);
    const int S = nrhs, m = K->m, ldp = m + 1;
    auto al = [&](void** p, size_t bytes, const char* what) {
        helm_status rc = dev_alloc(ctx, p, bytes, what);
        if (!rc) K->allocs.push_back({*p, bytes});
        return rc;
    };
    HELM_TRY(al(&K->V, (size_t)(m + 1) * K->nel * te, "inner Krylov basis"));
    HELM_TRY(al(&K->w, K->nel * te, "inner Arnoldi vector"));
    HELM_TRY(al(&K->u, K->nel * te, "inner preconditioned vector"));
    HELM_TRY(al((void**)&K->H, (size_t)S * (m + 1) * m * sizeof(c128), "inner Hessenberg"));
    HELM_TRY(al((void**)&K->sn, (size_t)S * m * sizeof(c128), "inner Givens sines"));
    HELM_TRY(al((void**)&K->cs, (size_t)S * m * sizeof(double), "inner Givens cosines"));
    HELM_TRY(al((void**)&K->gv, (size_t)S * (m + 1) * sizeof(c128), "inner Givens rhs"));
    HELM_TRY(al((void**)&K->y, (size_t)S * m * sizeof(c128), "inner least-squares solution"));
    HELM_TRY(al((void**)&K->y32, (size_t)S * m * sizeof(c64), "inner least-squares solution (complex64)"));
    HELM_TRY(al((void**)&K->part, (size_t)K->nblk * ldp * S * sizeof(c128), "inner dot partials"));
    HELM_TRY(al((void**)&K->hpass, (size_t)ldp * S * sizeof(c128), "inner dot pass"));
    HELM_TRY(al((void**)&K->dpart, (size_t)K->nblk * S * sizeof(double), "inner norm partials"));
    for (double** q : {&K->beta, &K->inv, &K->hn, &K->nb, &K->na})
        HELM_TRY(al((void**)q, S * sizeof(double), "inner norms"));
    HELM_TRY(al((void**)&K->Sd, S * sizeof(RhsState), "inner column state"));
    HELM_TRY(al((void**)&K->running, sizeof(int), "inner running flag"));
    HELM_TRY(al((void**)&K->rflag, S * sizeof(int), "inner re-orthogonalisation flags"));
    HELM_TRY(al((void**)&K->rany, sizeof(int), "inner re-orthogonalisation any"));
    return HELM_OK;
}

void inner_free(helm_oras o) {
    if (!o->inner) return;
    helm_ctx ctx = o->g->ctx;
    for (auto& a : o->inner->allocs) dev_free(ctx, a.first, a.second);
    delete o->inner;
    o->inner = nullptr;
}

namespace {

template <typename T>
helm_status inner_solve_t(helm_oras o, InnerKrylov& K, const cplx<T>* c, cplx<T>* yout) {
    helm_ctx ctx = o->g->ctx;
    cudaStream_t st = ctx->stream;
    const int S = K.S, m = K.m, ldp = m + 1, nblk = K.nblk;
    const long long nel = K.nel;
    const unsigned eg = (unsigned)std::min<long long>((nel + 255) / 256, (long long)ctx->sm_count * 16);
    const unsigned rg = (unsigned)((S + 127) / 128);
    cplx<T>* V = (cplx<T>*)K.V;
    cplx<T>* w = (cplx<T>*)K.w;
    cplx<T>* u = (cplx<T>*)K.u;
    const int hsmem_cap = 40 * 1024 / (int)sizeof(cplx<T>);
    // beta = ||c||, state, v_0 = c / beta
    norm2_kernel<T><<<nblk, RED_THREADS, 0, st>>>(c, nel, S, K.dpart);
    finish_norm2<<<S, 128, 0, st>>>(K.dpart, nblk, S, K.beta);
    inner_init<<<rg, 128, 0, st>>>(K.Sd, K.beta, S, m);
    cycle_start<<<rg, 128, 0, st>>>(K.Sd, K.beta, K.inv, K.gv, m, S);
    scale_copy<T, T><<<eg, 256, 0, st>>>(c, V, nel, S, K.inv);
    ctx->launches += 5;
    auto dots = [&](int ni, double* npart, const int* anyp) {
        dots_kernel<T><<<nblk, RED_THREADS, 0, st>>>(V, nel, w, nel, S, 0, ni, K.part, ldp, npart, anyp);
        finish_dots<<<ni * S, 128, 0, st>>>(K.part, nblk, ldp, ni, S, K.hpass, S, 1, 0, 0, nullptr, anyp);
        ctx->launches += 2;
    };
    auto update = [&](int ni, const int* cm, const int* anyp, double* out) {
        const int hs = ni * S <= hsmem_cap ? 1 : 0;
        const size_t smem = hs ? (size_t)ni * S * sizeof(cplx<T>) : 0;
        update_norm_kernel<T><<<nblk, RED_THREADS, smem, st>>>(V, nel, w, nel, S, ni, K.hpass, cm, anyp, K.dpart, hs);
        finish_norm2<<<S, 128, 0, st>>>(K.dpart, nblk, S, out);
        ctx->launches += 2;
    };
    for (int j = 0; j < m; ++j) {
        HELM_TRY(coarse_dd_apply(o, K.wp, V + (long long)j * nel, u, S));
        HELM_TRY(coarse_E_apply(o, K.wp, u, w, S));
        // classical Gram-Schmidt with selective re-orthogonalisation, as in the outer iteration
        dots(j + 1, K.dpart, nullptr);
        finish_dots<<<(j + 1) * S, 128, 0, st>>>(K.part, nblk, ldp, j + 1, S, K.H, m, (m + 1) * m, j, 0, nullptr,
                                                 nullptr);
        finish_norm2<<<S, 128, 0, st>>>(K.dpart, nblk, S, K.nb);
        ctx->launches += 2;
        update(j + 1, nullptr, nullptr, K.na);
        reorth_flags<<<1, 32, 0, st>>>(K.nb, K.na, K.rflag, K.rany, S);
        ctx->launches++;
        dots(j + 1, nullptr, K.rany);
        finish_dots<<<(j + 1) * S, 128, 0, st>>>(K.part, nblk, ldp, j + 1, S, K.H, m, (m + 1) * m, j, 1, K.rflag,
                                                 K.rany);
        ctx->launches++;
        update(j + 1, K.rflag, K.rany, K.hn);
        HELM_CUDA(ctx, cudaMemsetAsync(K.running, 0, sizeof(int), st));
        givens_step<<<rg, 128, 0, st>>>(K.Sd, K.H, K.cs, K.sn, K.gv, K.hn, K.inv, j, m, S, K.running);
        scale_copy<T, T><<<eg, 256, 0, st>>>(w, V + (long long)(j + 1) * nel, nel, S, K.inv);
        ctx->launches += 2;
    }
    // y = M_c^{-1} (V y_ls): standard right-preconditioned GMRES keeps only V
    back_substitute<<<rg, 128, 0, st>>>(K.Sd, K.H, K.gv, K.y, sizeof(T) == 4 ? K.y32 : nullptr, m, S);
    if (sizeof(T) == 4)
        combine32<float><<<eg, 256, 0, st>>>((const c64*)V, nel, K.y32, (c64*)u, nel, S, m);
    else
        combine_kernel<T, T, false><<<eg, 256, 0, st>>>(V, nel, K.y, u, nel, S, m);
    ctx->launches += 2;
    HELM_TRY(coarse_dd_apply(o, K.wp, u, yout, S));
    return cuda_check(ctx, cudaGetLastError(), "inner coarse GMRES");
}

}  // namespace

helm_status inner_solve(helm_oras o, int wp, const void* c, void* y, int nrhs) {
    helm_ctx ctx = o->g->ctx;
    if (!o->inner || o->inner->wp != wp || o->inner->S != nrhs)
        return set_error(ctx, HELM_EINVAL, "inner coarse solve: workspace not sized for this call");
    const int tk = prof_begin(ctx, "coarse_inner");
    helm_status rc = wp == HELM_PREC_FP64
                         ? inner_solve_t<double>(o, *o->inner, (const c128*)c, (c128*)y)
                         : inner_solve_t<float>(o, *o->inner, (const c64*)c, (c64*)y);
    prof_end(ctx, tk, 0.0);
    return rc;
}

namespace {

helm_status solve_all(helm_oras o, c128* b, c128* x, int nrhs, const helm_gmres_desc& D, helm_rhs_stats* stats) {
    helm_ctx ctx = o->g->ctx;
    helm_status rc = HELM_OK;
    // with graphs on, the workspace (and its captured iteration graphs) stays on the handle
    const bool keep = ctx->use_graphs != 0;
    const int flex = D.flexible != 0;
    KrylovEngine* K = nullptr;
    std::unique_ptr<KrylovEngine> owned;
    if (keep && o->kcache && o->kc_slots == nrhs && o->kc_restart == D.restart && o->kc_flex == flex &&
        o->kc_prec == D.basis_prec) {
        K = o->kcache;
        K->rebind(b, x);
    } else {
        delete o->kcache;
        o->kcache = nullptr;
        K = make_krylov_engine(o, nrhs, D.restart, flex != 0, D.basis_prec, b, x, &rc);
        if (!K) return rc;
        if (keep) {
            o->kcache = K;
            o->kc_slots = nrhs;
            o->kc_restart = D.restart;
            o->kc_flex = flex;
            o->kc_prec = D.basis_prec;
            K->enable_graphs(true);
        } else {
            owned.reset(K);
        }
    }
    std::vector<int> cols(nrhs), maxit(nrhs, D.maxit);
    std::vector<double> tol(nrhs, D.tol);
    for (int i = 0; i < nrhs; ++i) cols[i] = i;
    HELM_TRY(K->begin_columns(cols.data(), nrhs, tol.data(), maxit.data(), D.use_x0 != 0));
    bool any = false;
    for (int i = 0; i < nrhs; ++i) any = any || !K->state(i).done;
    while (any) HELM_TRY(K->cycle(&any));
    bool all = true;
    for (int i = 0; i < nrhs; ++i) {
        const RhsState& s = K->state(i);
        const double tr = K->true_rel(i);
        const bool conv = tr <= D.tol;
        all = all && conv;
        if (stats) stats[i] = helm_rhs_stats{s.iters, conv ? 1 : 0, tr, s.est};
    }
    if (!all) return set_error(ctx, HELM_ENOTCONV, "gmres_solve: some columns did not reach tol within maxit");
    return HELM_OK;
}

}  // namespace

extern "C" helm_status gmres_solve(helm_oras o, const void* b, void* x, int nrhs, const helm_gmres_desc* d,
                                   helm_rhs_stats* stats) {
    if (!o) return HELM_EINVAL;
    helm_ctx ctx = o->g->ctx;
    if (!b || !x || !d || nrhs < 0) return set_error(ctx, HELM_EINVAL, "gmres_solve: invalid argument");
    if (!(d->tol > 0) || d->restart < 1 || d->restart > 200 || d->maxit < 1 ||
        (d->basis_prec != HELM_PREC_FP64 && d->basis_prec != HELM_PREC_FP32) || (d->use_x0 != 0 && d->use_x0 != 1))
        return set_error(ctx, HELM_EINVAL, "gmres_solve: invalid solver description");
    if (nrhs == 0) return HELM_OK;
    if (nrhs > 256) return set_error(ctx, HELM_EINVAL, "gmres_solve: at most 256 right-hand sides per call");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t bytes = (size_t)o->g->n * nrhs * sizeof(c128);
    const bool bdev = is_device_pointer(b), xdev = is_device_pointer(x);
    c128 *bd = (c128*)b, *xd = (c128*)x;
    void* stage_b = nullptr;
    void* stage_x = nullptr;
    if (!bdev) {
        HELM_TRY(dev_alloc(ctx, &stage_b, bytes, "staged b"));
        HELM_CUDA(ctx, cudaMemcpyAsync(stage_b, b, bytes, cudaMemcpyHostToDevice, st));
        bd = (c128*)stage_b;
    }
    if (!xdev) {
        helm_status rc = dev_alloc(ctx, &stage_x, bytes, "staged x");
        if (rc) {
            dev_free(ctx, stage_b, bytes);
            return rc;
        }
        xd = (c128*)stage_x;
        if (d->use_x0 && (rc = cuda_check(ctx, cudaMemcpyAsync(stage_x, x, bytes, cudaMemcpyHostToDevice, st),
                                          "copy x0"))) {
            cudaStreamSynchronize(st);
            dev_free(ctx, stage_b, bytes);
            dev_free(ctx, stage_x, bytes);
            return rc;
        }
    }
    helm_status rc = solve_all(o, bd, xd, nrhs, *d, stats);
    if (!xdev && (rc == HELM_OK || rc == HELM_ENOTCONV)) {
        cudaError_t e = cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_check(ctx, e, "copy x to host");
    }
    cudaStreamSynchronize(st);
    dev_free(ctx, stage_b, bytes);
    dev_free(ctx, stage_x, bytes);
    return rc;
}
