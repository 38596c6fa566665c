// 27-point mixed-grid Helmholtz stencil y = A u (Eq. eq1), matrix-free, multi-RHS.
//
// The mixed-grid stencil (rotated-coordinate Laplacians with weights w1..w3
// plus a consistent mass term with weights wm1..wm4) is applied in its exact
// product form with 1-D second differences:
//   A u = h^-2 [sum D_a + a2 sum_{a<b} D_a D_b + a3 D_x D_y D_z] u
//       + [m0 + m1 sum P_a + m2 sum P_a P_b + m3 P_x P_y P_z] (k^2 u)
// with a2 = w2/6 + w3/2, a3 = w3/4, m0 = wm1+6wm2+12wm3+8wm4,
// m1 = wm2+4wm3+4wm4, m2 = wm3+2wm4, m3 = wm4.  D_a is the 3-point second
// difference stretched by the absorbing layer (coefficients cm, c0, cp per
// node, from the grid's 1-D tables); P_a is the plain (1, -2, 1).  Ghost
// neighbours (outside the grid, including the Dirichlet plane above k = 0)
// contribute zero.
//
// The coefficient of neighbour (dx, dy, dz) is a tensor product of the 1-D
// coefficients; per (dy, dz) pair the two partial sums
//   A = e_y e_z + a2 (Y e_z + e_y Z) + a3 Y Z,  B = Y e_z + e_y Z + a2 Y Z
// give the Laplacian coefficient X_dx A + [dx == 0] B, and likewise for the
// real mass coefficient.  Each thread owns one node and RCH consecutive
// right-hand sides, rhs fastest across threads (complex64: RCH = 2, one
// 16-byte vector per thread, so every neighbour load of a warp covers 512
// contiguous bytes; complex128: RCH up to 4, as the FP64 arithmetic and not
// the loads bounds it).  The coefficient is formed once per neighbour and
// reused for the RCH columns.  The grid is (x-line chunks, y, z), so no
// thread divides 64-bit indices.
#include <atomic>

#include "internal.h"

namespace {

// Rows whose 1-D coefficients are all the plain (1, -2, 1) and whose 26 neighbours exist
// (inside [lo, hi] on every axis) use the four class constants of the stencil: with
// plain differences the Laplacian coefficient of a neighbour depends only on its class
// (centre, face, edge, corner), Lc = {-6+12a2-8a3, 1-4a2+4a3, a2-2a3, a3}, and the mass
// coefficient is Mc = {wm1, wm2, wm3, wm4}; the neighbour's coefficient is Lc/h^2 + Mc k^2_q,
// real when k^2 is real (REALK).
struct Interior {
    int lo[3], hi[3];
    double Lc[4], Mc[4];
};

// RCH consecutive complex values loaded or stored as one aligned vector
template <typename T, int RCH>
struct __align__(2 * sizeof(T) * RCH) CPack {
    cplx<T> v[RCH];
};

// NR > 0: the column count as a compile-time constant (neighbour addresses become immediate offsets)
template <typename T, int RCH, bool SUB, bool REALK, int NR>
__global__ void __launch_bounds__(128) stencil_kernel(const cplx<T>* __restrict__ u, const cplx<T>* __restrict__ b,
                                                      cplx<T>* __restrict__ y,
                                                      const cplx<T>* __restrict__ k2,
                                                      const cplx<T>* __restrict__ tab, int nx, int ny, int nz,
                                                      int nrhs_rt, StencilW w, Interior in,
                                                      const StencilW* __restrict__ wtab,
                                                      const unsigned char* __restrict__ wbin) {
    // grid: (x-line chunks, y, z); a thread owns node (i, j, k) and columns [ch RCH, ch RCH + RCH)
    const int nrhs = NR > 0 ? NR : nrhs_rt;
    const int nch = nrhs / RCH;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx * nch) return;
    const int ch = t % nch, i = t / nch;
    const int j = blockIdx.y, k = blockIdx.z;
    const long long p = ((long long)k * ny + j) * nx + i;
    // neighbour offsets: nodes for k^2, entries for the vectors
    const long long nxy = (long long)nx * ny;
    const cplx<T>* up = u + p * nrhs + (long long)ch * RCH;
    const cplx<T>* kp = k2 + p;

    if (wtab) w = wtab[wbin[p]];   // adaptive weights: this row's bin
    const T ih2 = (T)w.inv_h2;
    const cplx<T> zero = mk<T>(0, 0);
    cplx<T> acc[RCH];
#pragma unroll
    for (int r = 0; r < RCH; ++r) acc[r] = zero;

    if (i >= in.lo[0] && i <= in.hi[0] && j >= in.lo[1] && j <= in.hi[1] && k >= in.lo[2] && k <= in.hi[2]) {
        T L[4], M[4];
        if (wtab) {
            // class constants of this row's weights (the same identities as for the grid's constant weights)
            const double Lr[4] = {-6.0 + 12.0 * w.a2 - 8.0 * w.a3, 1.0 - 4.0 * w.a2 + 4.0 * w.a3, w.a2 - 2.0 * w.a3, w.a3};
            const double Mr[4] = {w.m0 - 6.0 * w.m1 + 12.0 * w.m2 - 8.0 * w.m3, w.m1 - 4.0 * w.m2 + 4.0 * w.m3,
                                  w.m2 - 2.0 * w.m3, w.m3};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                L[c] = (T)(Lr[c] * w.inv_h2);
                M[c] = (T)Mr[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                L[c] = (T)(in.Lc[c] * w.inv_h2);
                M[c] = (T)in.Mc[c];
            }
        }
        // one z-plane of 9 neighbours at a time: its 18 loads are issued together, then the FMAs
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            cplx<T> kq[9];
            CPack<T, RCH> uq[9];
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                const long long dq = dz * nxy + (d / 3 - 1) * nx + (d % 3 - 1);
                kq[d] = kp[dq];
                uq[d] = *reinterpret_cast<const CPack<T, RCH>*>(up + dq * nrhs);
            }
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                const int cls = (d % 3 != 1) + (d / 3 != 1) + (dz != 0);
                if (REALK) {
                    const T cr = L[cls] + M[cls] * kq[d].x;
#pragma unroll
                    for (int r = 0; r < RCH; ++r) {
                        acc[r].x = fma(cr, uq[d].v[r].x, acc[r].x);
                        acc[r].y = fma(cr, uq[d].v[r].y, acc[r].y);
                    }
                } else {
                    const cplx<T> cc = mk<T>(L[cls] + M[cls] * kq[d].x, M[cls] * kq[d].y);
#pragma unroll
                    for (int r = 0; r < RCH; ++r) cmac(acc[r], cc, uq[d].v[r]);
                }
            }
        }
    } else {
    const cplx<T>* tx = tab + 3 * i;
    const cplx<T>* ty = tab + 3 * (nx + j);
    const cplx<T>* tz = tab + 3 * (nx + ny + k);
    cplx<T> X[3], Y[3], Z[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) { X[d] = tx[d]; Y[d] = ty[d]; Z[d] = tz[d]; }

    const T a2 = (T)w.a2, a3 = (T)w.a3, m0 = (T)w.m0, m1 = (T)w.m1, m2 = (T)w.m2, m3 = (T)w.m3;

#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int kk = k + dz;
        if (kk < 0 || kk >= nz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int jj = j + dy;
            if (jj < 0 || jj >= ny) continue;
            const cplx<T> Yd = Y[dy + 1], Zd = Z[dz + 1];
            const cplx<T> yz = Yd * Zd;
            const cplx<T> ye = (dz == 0) ? Yd : zero;       // Y e_z
            const cplx<T> ez = (dy == 0) ? Zd : zero;       // e_y Z
            const T ee = (dy == 0 && dz == 0) ? (T)1 : (T)0;
            cplx<T> Ac = a3 * yz + a2 * (ye + ez);
            Ac.x += ee;
            const cplx<T> Bc = ye + ez + a2 * yz;
            const T Py = (dy == 0) ? (T)-2 : (T)1, Pz = (dz == 0) ? (T)-2 : (T)1;
            const T pe = (dz == 0) ? Py : (T)0;
            const T ep = (dy == 0) ? Pz : (T)0;
            const T pp = Py * Pz;
            const T Am = m1 * ee + m2 * (pe + ep) + m3 * pp;
            const T Bm = m0 * ee + m1 * (pe + ep) + m2 * pp;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int ii = i + dx;
                if (ii < 0 || ii >= nx) continue;
                cplx<T> lap = X[dx + 1] * Ac;
                T mass = ((dx == 0) ? (T)-2 : (T)1) * Am;
                if (dx == 0) { lap = lap + Bc; mass += Bm; }
                const long long dq = dz * nxy + dy * nx + dx;
                const cplx<T> kq = kp[dq];
                cplx<T> coef = mk<T>(lap.x * ih2 + mass * kq.x, lap.y * ih2 + mass * kq.y);
                const CPack<T, RCH> uq = *reinterpret_cast<const CPack<T, RCH>*>(up + dq * nrhs);
#pragma unroll
                for (int r = 0; r < RCH; ++r) cmac(acc[r], coef, uq.v[r]);
            }
        }
    }
    }
    CPack<T, RCH> out;
    if (SUB) {
        const CPack<T, RCH> bp = *reinterpret_cast<const CPack<T, RCH>*>(b + p * nrhs + (long long)ch * RCH);
#pragma unroll
        for (int r = 0; r < RCH; ++r) out.v[r] = bp.v[r] - acc[r];
    } else {
#pragma unroll
        for (int r = 0; r < RCH; ++r) out.v[r] = acc[r];
    }
    *reinterpret_cast<CPack<T, RCH>*>(y + p * nrhs + (long long)ch * RCH) = out;
}

// ---------------------------------------------------------------- z-march (complex64, columns in chunks of 16)
//
// The same operator grouped by z-planes: with D_a the stretched and P_a the plain second differences,
//   A u = h^-2 [S0 + D_z S1] + [T0 + P_z T1],
//   S0 = (D_x + D_y) u + a2 D_x D_y u,   S1 = u + a2 (D_x + D_y) u + a3 D_x D_y u,
//   T0 = m0 v + m1 (P_x + P_y) v + m2 P_x P_y v,   T1 = m1 v + m2 (P_x + P_y) v + m3 P_x P_y v,   v = k^2 u,
// where S0, S1, T0, T1 are in-plane.  A thread owns MN consecutive x-nodes of one row j and one column pair
// and walks a chunk of output planes (a launch parameter): for every plane q it loads the (MN + 2) x 3 in-plane neighbourhood
// once, forms the in-plane terms of its nodes, and adds their contributions to the outputs q - 1 (last
// term, then stored), q and q + 1 (first term).  Each output therefore costs (MN + 2) * 3 / MN vector loads
// instead of 27.  Blocks whose rows all have plain (1, -2, 1) 1-D coefficients take the real-coefficient
// path; the others use the complex table coefficients.  Ghost nodes contribute zero.
constexpr int MN = 4;      // x-nodes per thread
constexpr int MNP = 8;     // column pairs (16 columns)

struct PlainRange {
    int lo[3], hi[3];   // per axis: indices whose stretched coefficients are exactly (1, -2, 1)
};

// Two complex64 values (re0, im0, re1, im1) in a float4, processed as two (re, im) pairs by the packed FP32
// instructions (two lanes per instruction, each lane rounded like the scalar operation).
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 sw2(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return cat4(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    const float2 m = make_float2(-1.f, -1.f);
    return cat4(__ffma2_rn(m, lo2(b), lo2(a)), __ffma2_rn(m, hi2(b), hi2(a)));
}
// s b (s real)
__device__ __forceinline__ float4 scal4(float s, float4 b) {
    const float2 ss = make_float2(s, s);
    return cat4(__fmul2_rn(ss, lo2(b)), __fmul2_rn(ss, hi2(b)));
}
// a + s b (s real)
__device__ __forceinline__ float4 axpy4(float s, float4 b, float4 a) {
    const float2 ss = make_float2(s, s);
    return cat4(__ffma2_rn(ss, lo2(b), lo2(a)), __ffma2_rn(ss, hi2(b), hi2(a)));
}
// a + c b (c complex, b two complex values): per value re = c.x b.re + (-c.y b.im + a.re),
// im = c.x b.im + (c.y b.re + a.im)
__device__ __forceinline__ float4 caxpy4(c64 c, float4 b, float4 a) {
    const float2 cr = make_float2(c.x, c.x), ci = make_float2(-c.y, c.y);
    return cat4(__ffma2_rn(cr, lo2(b), __ffma2_rn(ci, sw2(lo2(b)), lo2(a))),
                __ffma2_rn(cr, hi2(b), __ffma2_rn(ci, sw2(hi2(b)), hi2(a))));
}
// c b (c complex)
__device__ __forceinline__ float4 cmul4(c64 c, float4 b) {
    const float2 cr = make_float2(c.x, c.x), ci = make_float2(-c.y, c.y);
    return cat4(__ffma2_rn(cr, lo2(b), __fmul2_rn(ci, sw2(lo2(b)))),
                __ffma2_rn(cr, hi2(b), __fmul2_rn(ci, sw2(hi2(b)))));
}
// A complex coefficient c as the pairs (c.re, c.re, c.im, c.im) of one float4.
__device__ __forceinline__ float4 cpair(c64 c) { return make_float4(c.x, c.x, c.y, c.y); }
// the 3-point second difference c0 x0 + c1 x1 + c2 x2, plain (1, -2, 1) or with complex coefficients given as
// pairs: per value the real-coefficient sum R = sum re(c_d) x_d and the imaginary one I = sum im(c_d) x_d are
// formed first and combined once, R + i I = (R.re - I.im, R.im + I.re)
template <bool PLAIN>
__device__ __forceinline__ float4 d3(const float4* c, float4 x0, float4 x1, float4 x2) {
    if (PLAIN) return axpy4(-2.f, x1, add4(x0, x2));
    const float2 j = make_float2(-1.f, 1.f);
    float2 r[2], im[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float2 v0 = h ? hi2(x0) : lo2(x0), v1 = h ? hi2(x1) : lo2(x1), v2 = h ? hi2(x2) : lo2(x2);
        r[h] = __ffma2_rn(lo2(c[2]), v2, __ffma2_rn(lo2(c[1]), v1, __fmul2_rn(lo2(c[0]), v0)));
        im[h] = __ffma2_rn(hi2(c[2]), v2, __ffma2_rn(hi2(c[1]), v1, __fmul2_rn(hi2(c[0]), v0)));
    }
    return cat4(__ffma2_rn(j, sw2(im[0]), r[0]), __ffma2_rn(j, sw2(im[1]), r[1]));
}

// The block's planes pass through shared memory: a 128-thread block covers 16 x-nodes x 4 rows x 16
// columns, and plane q's neighbourhood (18 nodes x 6 rows, all columns, and k^2) is copied in with cp.async
// two planes ahead of the one computed (three buffers; ghost nodes are zero-filled by the copy).
constexpr int MTX = (32 / MNP) * MN;       // x-nodes per block (16)
constexpr int MTY = 4;                     // rows per block (one warp each)
constexpr int MBX = MTX + 2, MBY = MTY + 2;
constexpr int MBUF_U = MBX * MBY * MNP;    // float4 entries of one plane buffer
constexpr int MBUF_K = MBX * MBY;          // float2 entries (k^2) of one plane buffer
constexpr int MNBUF = 3;                   // plane buffers: q is computed while q + 1 and q + 2 arrive

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(sdst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// issue the copies of plane q (rows j0-1..j0+MTY, nodes i0-1..i0+MTX); out-of-grid entries become zero
__device__ __forceinline__ void march_stage(float4* su, float2* sk, const float4* __restrict__ u,
                                            const c64* __restrict__ k2, int nx, int ny, int nz, int nrs, int i0,
                                            int j0, int q) {
    const bool qin = q >= 0 && q < nz;
    for (int e = threadIdx.x; e < MBUF_U; e += blockDim.x) {
        const int pc = e % MNP, xn = (e / MNP) % MBX, yr = e / (MNP * MBX);
        const int ii = i0 + xn - 1, jj = j0 + yr - 1;
        const bool ok = qin && ii >= 0 && ii < nx && jj >= 0 && jj < ny;
        const long long node = ok ? ((long long)q * ny + jj) * nx + ii : 0;
        cp_async16(su + e, u + node * nrs + pc, ok);
    }
    for (int e = threadIdx.x; e < MBUF_K; e += blockDim.x) {
        const int xn = e % MBX, yr = e / MBX;
        const int ii = i0 + xn - 1, jj = j0 + yr - 1;
        const bool ok = qin && ii >= 0 && ii < nx && jj >= 0 && jj < ny;
        const long long node = ok ? ((long long)q * ny + jj) * nx + ii : 0;
        cp_async8(sk + e, k2 + node, ok);
    }
}

// march_run in product form for blocks in the absorbing layers; PX, PY, PZ: the block's rows have plain
// (1, -2, 1) coefficients along that axis (a block in one layer only is stretched along one axis), so only the
// stretched axes pay complex products.  The x coefficients of the block's 16 nodes sit in shared memory as
// pairs (sx, filled before the first barrier of the plane loop), the row's y coefficients in registers.
template <bool SUB, bool REALK, bool PX, bool PY, bool PZ>
__device__ __forceinline__ void march_run(const float4* __restrict__ u, const float4* __restrict__ b,
                                          float4* __restrict__ y, const c64* __restrict__ k2,
                                          const c64* __restrict__ tab, int nx, int ny, int nz, int nrs,
                                          const StencilW& w, int i0, int j0, int k0, int k1, float4* su, float2* sk,
                                          float4* sx) {
    const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
    const int pc = lane % MNP, g = lane / MNP;
    const int j = j0 + wr, xb = g * MN, ib = i0 + xb;
    const bool live = j < ny;
    const float ih2 = (float)w.inv_h2, a2 = (float)w.a2, a3 = (float)w.a3;
    const float m0 = (float)w.m0, m1 = (float)w.m1, m2 = (float)w.m2, m3 = (float)w.m3;
    if (!PX && threadIdx.x < MTX * 3) {
        const int n = threadIdx.x / 3, d = threadIdx.x % 3;
        sx[threadIdx.x] = i0 + n < nx ? cpair(tab[3 * (i0 + n) + d]) : f4(0.f);
    }
    float4 Y[3];
    if (!PY) {
#pragma unroll
        for (int d = 0; d < 3; ++d) Y[d] = live ? cpair(tab[3 * (nx + j) + d]) : f4(0.f);
    }
    const c64* tz = tab + 3 * (nx + ny);
    float4 P[MN], N[MN];   // outputs q and q + 1, partial
#pragma unroll
    for (int c = 0; c < MN; ++c) P[c] = N[c] = f4(0.f);
    march_stage(su, sk, u, k2, nx, ny, nz, nrs, i0, j0, k0 - 1);
    cp_async_commit();
    march_stage(su + MBUF_U, sk + MBUF_K, u, k2, nx, ny, nz, nrs, i0, j0, k0);
    cp_async_commit();
    for (int q = k0 - 1, buf = 0; q <= k1; ++q, buf = buf == MNBUF - 1 ? 0 : buf + 1) {
        // prefetch plane q + 2 into the buffer plane q - 1 used (free since the barrier ending the last step)
        const int nb = buf >= 1 ? buf - 1 : MNBUF - 1;
        if (q + 2 <= k1) march_stage(su + nb * MBUF_U, sk + nb * MBUF_K, u, k2, nx, ny, nz, nrs, i0, j0, q + 2);
        cp_async_commit();
        cp_async_wait<2>();
        __syncthreads();
        // b of the output plane q - 1, loaded now so that its latency overlaps this step's arithmetic
        float4 bq[MN];
        if (SUB) {
#pragma unroll
            for (int c = 0; c < MN; ++c) {
                bq[c] = f4(0.f);
                if (live && q - 1 >= k0 && ib + c < nx)
                    bq[c] = __ldg(b + (((long long)(q - 1) * ny + j) * nx + ib + c) * nrs + pc);
            }
        }
        const float4* cu = su + buf * MBUF_U;
        const float2* ck = sk + buf * MBUF_K;
        const bool qin = q >= 0 && q < nz;
        c64 zm = mk<float>(0, 0), zc = mk<float>(0, 0), zp = mk<float>(0, 0);
        if (!PZ) {
            zm = q - 1 >= 0 && q - 1 < nz ? tz[3 * (q - 1) + 2] : mk<float>(0, 0);
            zc = qin ? tz[3 * q + 1] : mk<float>(0, 0);
            zp = q + 1 >= 0 && q + 1 < nz ? tz[3 * (q + 1) + 0] : mk<float>(0, 0);
        }
        // sliding window over the columns n = c, c + 1, c + 2 of node c (column n = block node xb + n - 1):
        // D_y u, P_y v, v and u on row j
        float4 DyU[3], PyV[3], V1[3], U1[3];
        auto column = [&](int n, int slot) {
            float4 Ur[3], V[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int sidx = (wr + r) * MBX + xb + n;
                Ur[r] = cu[sidx * MNP + pc];
                const float2 kk = ck[sidx];
                V[r] = REALK ? scal4(kk.x, Ur[r]) : cmul4(mk<float>(kk.x, kk.y), Ur[r]);
            }
            DyU[slot] = d3<PY>(Y, Ur[0], Ur[1], Ur[2]);
            PyV[slot] = d3<true>(nullptr, V[0], V[1], V[2]);
            V1[slot] = V[1];
            U1[slot] = Ur[1];
        };
        column(0, 0);
        column(1, 1);
#pragma unroll
        for (int c = 0; c < MN; ++c) {
            column(c + 2, (c + 2) % 3);
            const int s0 = c % 3, s1 = (c + 1) % 3, s2 = (c + 2) % 3;
            float4 X[3];
            if (!PX) {
#pragma unroll
                for (int d = 0; d < 3; ++d) X[d] = sx[(xb + c) * 3 + d];
            }
            const float4 u0 = U1[s1];
            const float4 Eu = add4(d3<PX>(X, U1[s0], U1[s1], U1[s2]), DyU[s1]);
            const float4 Fu = d3<PX>(X, DyU[s0], DyU[s1], DyU[s2]);
            const float4 v0 = V1[s1];
            const float4 Ev = add4(d3<true>(nullptr, V1[s0], V1[s1], V1[s2]), PyV[s1]);
            const float4 Fv = d3<true>(nullptr, PyV[s0], PyV[s1], PyV[s2]);
            const float4 S0 = axpy4(a2, Fu, Eu);
            const float4 S1 = axpy4(a3, Fu, axpy4(a2, Eu, u0));
            const float4 T0 = axpy4(m2, Fv, axpy4(m1, Ev, scal4(m0, v0)));
            const float4 T1 = axpy4(m3, Fv, axpy4(m2, Ev, scal4(m1, v0)));
            const float4 hS1 = scal4(ih2, S1);
            // output q - 1: its last term
            const int i = ib + c;
            if (live && q - 1 >= k0 && i < nx) {
                float4 o = add4(PZ ? add4(P[c], hS1) : caxpy4(zm, hS1, P[c]), T1);
                const long long node = ((long long)(q - 1) * ny + j) * nx + i;
                if (SUB) o = sub4(bq[c], o);
                __stcs(y + node * nrs + pc, o);
            }
            // output q: the centre term; output q + 1: its first term
            float4 pn = add4(N[c], axpy4(ih2, S0, axpy4(-2.f, T1, T0)));
            pn = PZ ? axpy4(-2.f, hS1, pn) : caxpy4(zc, hS1, pn);
            N[c] = add4(PZ ? hS1 : cmul4(zp, hS1), T1);
            P[c] = pn;
        }
        __syncthreads();   // buffer buf is refilled by the next step's prefetch
    }
    cp_async_wait<0>();
}

// march_run for blocks whose rows all have plain (1, -2, 1) coefficients, in class-sum form: with plain
// differences the coefficient of a neighbour depends only on its class (centre, face, edge, corner), so per
// plane q and node the in-plane terms of a field w (u for the Laplacian, v = k^2 u for the mass term) are its
// centre value c, its in-plane face sum F = s_x w + s_y w and its in-plane corner sum E = s_x s_y w (s_a: the sum
// of the two neighbours along axis a); plane q then adds Lc0 c + Lc1 F + Lc2 E (u) and Mc0 c + Mc1 F + Mc2 E (v)
// to output q and Lc1 c + Lc2 F + Lc3 E, Mc1 c + Mc2 F + Mc3 E to outputs q - 1 and q + 1, with the class
// constants Lc = {-6 + 12 a2 - 8 a3, 1 - 4 a2 + 4 a3, a2 - 2 a3, a3} / h^2 and Mc = {m0 - 6 m1 + 12 m2 - 8 m3,
// m1 - 4 m2 + 4 m3, m2 - 2 m3, m3}.  The same operator as the product form (expanded), in fewer operations.
template <bool SUB, bool REALK>
__device__ __forceinline__ void march_run_plain(const float4* __restrict__ u, const float4* __restrict__ b,
                                                float4* __restrict__ y, const c64* __restrict__ k2, int nx, int ny,
                                                int nz, int nrs, const StencilW& w, int i0, int j0, int k0, int k1,
                                                float4* su, float2* sk) {
    const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
    const int pc = lane % MNP, g = lane / MNP;
    const int j = j0 + wr, xb = g * MN, ib = i0 + xb;
    const bool live = j < ny;
    const double ih2 = w.inv_h2;
    const float L0 = (float)((-6.0 + 12.0 * w.a2 - 8.0 * w.a3) * ih2), L1 = (float)((1.0 - 4.0 * w.a2 + 4.0 * w.a3) * ih2);
    const float L2 = (float)((w.a2 - 2.0 * w.a3) * ih2), L3 = (float)(w.a3 * ih2);
    const float M0 = (float)(w.m0 - 6.0 * w.m1 + 12.0 * w.m2 - 8.0 * w.m3), M1 = (float)(w.m1 - 4.0 * w.m2 + 4.0 * w.m3);
    const float M2 = (float)(w.m2 - 2.0 * w.m3), M3 = (float)w.m3;
    float4 P[MN], N[MN];
#pragma unroll
    for (int c = 0; c < MN; ++c) P[c] = N[c] = f4(0.f);
    march_stage(su, sk, u, k2, nx, ny, nz, nrs, i0, j0, k0 - 1);
    cp_async_commit();
    march_stage(su + MBUF_U, sk + MBUF_K, u, k2, nx, ny, nz, nrs, i0, j0, k0);
    cp_async_commit();
    for (int q = k0 - 1, buf = 0; q <= k1; ++q, buf = buf == MNBUF - 1 ? 0 : buf + 1) {
        const int nb = buf >= 1 ? buf - 1 : MNBUF - 1;
        if (q + 2 <= k1) march_stage(su + nb * MBUF_U, sk + nb * MBUF_K, u, k2, nx, ny, nz, nrs, i0, j0, q + 2);
        cp_async_commit();
        cp_async_wait<2>();
        __syncthreads();
        float4 bq[MN];
        if (SUB) {
#pragma unroll
            for (int c = 0; c < MN; ++c) {
                bq[c] = f4(0.f);
                if (live && q - 1 >= k0 && ib + c < nx)
                    bq[c] = __ldg(b + (((long long)(q - 1) * ny + j) * nx + ib + c) * nrs + pc);
            }
        }
        const float4* cu = su + buf * MBUF_U;
        const float2* ck = sk + buf * MBUF_K;
        // sliding window over the columns n of the block row: centre values and the sums over rows j - 1, j + 1
        float4 Cu[3], Cv[3], Yu[3], Yv[3];
        auto column = [&](int n, int slot) {
            float4 U[3], V[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const int sidx = (wr + r) * MBX + xb + n;
                U[r] = cu[sidx * MNP + pc];
                const float2 kk = ck[sidx];
                V[r] = REALK ? scal4(kk.x, U[r]) : cmul4(mk<float>(kk.x, kk.y), U[r]);
            }
            Cu[slot] = U[1];
            Cv[slot] = V[1];
            Yu[slot] = add4(U[0], U[2]);
            Yv[slot] = add4(V[0], V[2]);
        };
        column(0, 0);
        column(1, 1);
#pragma unroll
        for (int c = 0; c < MN; ++c) {
            column(c + 2, (c + 2) % 3);
            const int s0 = c % 3, s1 = (c + 1) % 3, s2 = (c + 2) % 3;
            const float4 cU = Cu[s1], cV = Cv[s1];
            const float4 FU = add4(add4(Cu[s0], Cu[s2]), Yu[s1]), EU = add4(Yu[s0], Yu[s2]);
            const float4 FV = add4(add4(Cv[s0], Cv[s2]), Yv[s1]), EV = add4(Yv[s0], Yv[s2]);
            // plane q's contribution to output q (A0) and to outputs q -/+ 1 (A1)
            const float4 A0 = axpy4(M2, EV, axpy4(M1, FV, axpy4(M0, cV, axpy4(L2, EU, axpy4(L1, FU,
                                  scal4(L0, cU))))));
            const float4 A1 = axpy4(M3, EV, axpy4(M2, FV, axpy4(M1, cV, axpy4(L3, EU, axpy4(L2, FU,
                                  scal4(L1, cU))))));
            const int i = ib + c;
            if (live && q - 1 >= k0 && i < nx) {
                float4 o = add4(P[c], A1);
                const long long node = ((long long)(q - 1) * ny + j) * nx + i;
                if (SUB) o = sub4(bq[c], o);
                __stcs(y + node * nrs + pc, o);
            }
            P[c] = add4(N[c], A0);
            N[c] = A1;
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// grid: (x-node blocks, row blocks, plane chunks x column chunks); the column chunk (16 columns) is the
// fastest part of blockIdx.z, so the chunks of one node range run side by side
template <bool SUB, bool REALK>
__global__ void __launch_bounds__(128, 3) stencil_march(const c64* __restrict__ u, const c64* __restrict__ b,
                                                     c64* __restrict__ y, const c64* __restrict__ k2,
                                                     const c64* __restrict__ tab, int nx, int ny, int nz, int nrhs,
                                                     int mzc, StencilW w, PlainRange pl, int axis_variants) {
    __shared__ float4 su[MNBUF * MBUF_U];
    __shared__ float2 sk[MNBUF * MBUF_K];
    __shared__ float4 sx[MTX * 3];
    const int nrs = nrhs >> 1, ncc = nrs / MNP;   // float4 per node, column chunks
    const int cc = blockIdx.z % ncc, zc = blockIdx.z / ncc;
    const int i0 = blockIdx.x * MTX, j0 = blockIdx.y * MTY;
    const int k0 = zc * mzc, k1 = min(k0 + mzc, nz);
    const float4* u4 = reinterpret_cast<const float4*>(u) + cc * MNP;
    const float4* b4 = SUB ? reinterpret_cast<const float4*>(b) + cc * MNP : nullptr;
    float4* y4 = reinterpret_cast<float4*>(y) + cc * MNP;
    // blocks whose rows all have plain coefficients on every axis take the class-sum form
    const bool plain = i0 >= pl.lo[0] && min(i0 + MTX, nx) - 1 <= pl.hi[0] && j0 >= pl.lo[1] &&
                       min(j0 + MTY, ny) - 1 <= pl.hi[1] && k0 >= pl.lo[2] && k1 - 1 <= pl.hi[2];
    if (plain) {
        march_run_plain<SUB, REALK>(u4, b4, y4, k2, nx, ny, nz, nrs, w, i0, j0, k0, k1, su, sk);
        return;
    }
    // per axis: the block's rows are plain along it (with axis_variants; else the general product form,
    // which keeps the kernel's instruction footprint to two loop bodies)
    const bool px = axis_variants && i0 >= pl.lo[0] && min(i0 + MTX, nx) - 1 <= pl.hi[0];
    const bool py = axis_variants && j0 >= pl.lo[1] && min(j0 + MTY, ny) - 1 <= pl.hi[1];
    const bool pz = axis_variants && k0 >= pl.lo[2] && k1 - 1 <= pl.hi[2];
    if (py && pz) march_run<SUB, REALK, false, true, true>(u4, b4, y4, k2, tab, nx, ny, nz, nrs, w, i0, j0, k0, k1, su, sk, sx);
    else if (px && pz) march_run<SUB, REALK, true, false, true>(u4, b4, y4, k2, tab, nx, ny, nz, nrs, w, i0, j0, k0, k1, su, sk, sx);
    else if (px && py) march_run<SUB, REALK, true, true, false>(u4, b4, y4, k2, tab, nx, ny, nz, nrs, w, i0, j0, k0, k1, su, sk, sx);
    else march_run<SUB, REALK, false, false, false>(u4, b4, y4, k2, tab, nx, ny, nz, nrs, w, i0, j0, k0, k1, su, sk, sx);
}

struct RowW {
    const StencilW* wtab;
    const unsigned char* wbin;
};

template <typename T, int RCH, bool SUB, int NR = 0>
void launch_t(const cplx<T>* u, const cplx<T>* b, cplx<T>* y, const cplx<T>* k2, const cplx<T>* tab,
              const helm_grid_desc& d, int nrhs, const StencilW& w, const Interior& in, bool realk, RowW rw,
              cudaStream_t s) {
    const int threads = 128;
    const dim3 grid((unsigned)((d.nx * (nrhs / RCH) + threads - 1) / threads), (unsigned)d.ny, (unsigned)d.nz);
    if (realk)
        stencil_kernel<T, RCH, SUB, true, NR><<<grid, threads, 0, s>>>(u, b, y, k2, tab, d.nx, d.ny, d.nz, nrhs, w, in,
                                                                       rw.wtab, rw.wbin);
    else
        stencil_kernel<T, RCH, SUB, false, NR><<<grid, threads, 0, s>>>(u, b, y, k2, tab, d.nx, d.ny, d.nz, nrhs, w,
                                                                        in, rw.wtab, rw.wbin);
}

template <typename T, bool SUB>
void dispatch(const cplx<T>* u, const cplx<T>* b, cplx<T>* y, const cplx<T>* k2, const cplx<T>* tab,
              const helm_grid_desc& d, int nrhs, const StencilW& w, const Interior& in, bool realk, RowW rw,
              cudaStream_t s) {
    // complex64: one 16-byte vector per thread and neighbour, two columns when the column count is
    // even and every base address is 16-byte aligned, else one.  complex128 (FP64-pipe bound on this
    // part): up to four columns per thread, so each neighbour's coefficient is formed once for four
    // (a pack of RCH values is loaded as one aligned object: every base address must be aligned to it)
    const auto al = [&](uintptr_t a) {
        return ((uintptr_t)u & (a - 1)) == 0 && ((uintptr_t)y & (a - 1)) == 0 && (!SUB || ((uintptr_t)b & (a - 1)) == 0);
    };
    if constexpr (sizeof(T) == 4) {
        if (nrhs == 16 && al(16))
            launch_t<T, 2, SUB, 16>(u, b, y, k2, tab, d, nrhs, w, in, realk, rw, s);
        else if (nrhs % 2 == 0 && al(16))
            launch_t<T, 2, SUB>(u, b, y, k2, tab, d, nrhs, w, in, realk, rw, s);
        else
            launch_t<T, 1, SUB>(u, b, y, k2, tab, d, nrhs, w, in, realk, rw, s);
    } else {
        if (nrhs % 4 == 0 && al(64)) launch_t<T, 4, SUB>(u, b, y, k2, tab, d, nrhs, w, in, realk, rw, s);
        else if (nrhs % 2 == 0 && al(32)) launch_t<T, 2, SUB>(u, b, y, k2, tab, d, nrhs, w, in, realk, rw, s);
        else launch_t<T, 1, SUB>(u, b, y, k2, tab, d, nrhs, w, in, realk, rw, s);
    }
}

Interior interior_of(helm_grid g) {
    const helm_grid_desc& d = g->d;
    Interior in;
    const int n[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a) {
        const bool low = a < 2 || d.top_bc == HELM_TOP_PML;
        in.lo[a] = std::max(1, low && d.npml > 0 ? d.npml + 1 : 1);
        in.hi[a] = n[a] - 2 - (d.npml > 0 ? d.npml : 0);
    }
    const double a2 = g->w.a2, a3 = g->w.a3;
    in.Lc[0] = -6.0 + 12.0 * a2 - 8.0 * a3;
    in.Lc[1] = 1.0 - 4.0 * a2 + 4.0 * a3;
    in.Lc[2] = a2 - 2.0 * a3;
    in.Lc[3] = a3;
    const double m0 = g->w.m0, m1 = g->w.m1, m2 = g->w.m2, m3 = g->w.m3;
    in.Mc[0] = m0 - 6.0 * m1 + 12.0 * m2 - 8.0 * m3;
    in.Mc[1] = m1 - 4.0 * m2 + 4.0 * m3;
    in.Mc[2] = m2 - 2.0 * m3;
    in.Mc[3] = m3;
    return in;
}

// Per axis, the index range whose complex64 stretched coefficients are exactly (1, -2, 1) (the table is
// contiguous-plain in the middle and stretched in the absorbing layers); empty if not contiguous.
PlainRange plain_range(helm_grid g) {
    PlainRange r;
    const int n[3] = {g->d.nx, g->d.ny, g->d.nz};
    int base = 0;
    for (int a = 0; a < 3; ++a) {
        auto plain = [&](int i) {
            const c128* c = &g->htab[3 * (base + i)];
            return (float)c[0].x == 1.f && (float)c[0].y == 0.f && (float)c[1].x == -2.f && (float)c[1].y == 0.f &&
                   (float)c[2].x == 1.f && (float)c[2].y == 0.f;
        };
        int lo = 0, hi = n[a] - 1;
        while (lo < n[a] && !plain(lo)) ++lo;
        while (hi >= 0 && !plain(hi)) --hi;
        for (int i = lo; i <= hi; ++i)
            if (!plain(i)) {
                lo = 1;
                hi = 0;
                break;
            }
        r.lo[a] = lo;
        r.hi[a] = hi;
        base += n[a];
    }
    return r;
}

template <bool SUB>
helm_status launch_any(helm_grid g, int prec, const void* u, const void* b, void* y, int nrhs, cudaStream_t s) {
    if (nrhs <= 0) return HELM_OK;
    // algorithmic bytes: read u (and b), write y, read k^2 once
    const double es = prec == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);
    const double bytes = (double)g->n * es * ((SUB ? 3.0 : 2.0) * nrhs + 1.0);
    const int tok = prof_begin(g->ctx, prec == HELM_PREC_FP64 ? "stencil64" : "stencil");
    const Interior in = interior_of(g);
    const RowW rw{g->wtab, g->wbin};
    const uintptr_t al = (uintptr_t)u | (uintptr_t)y | (SUB ? (uintptr_t)b : 0);
    if (prec == HELM_PREC_FP64) {
        dispatch<double, SUB>((const c128*)u, (const c128*)b, (c128*)y, g->k2, g->tab, g->d, nrhs, g->w, in,
                              g->k2_real, rw, s);
    } else if (g->ctx->stencil_march && nrhs % (2 * MNP) == 0 && !g->wtab && (al & 15) == 0) {
        const PlainRange pl = plain_range(g);
        const int gx = (g->d.nx + MTX - 1) / MTX, gy = (g->d.ny + MTY - 1) / MTY, ncc = nrhs / (2 * MNP);
        int mzc = g->ctx->stencil_planes;
        if (mzc == 0) {
            // the fewest plane chunks (longest walks: less halo per output) of at most 64 planes that still give
            // every resident block slot two blocks or more (measured: fewer blocks than that leave the launch
            // short of latency hiding), chunks of 8 planes at least
            static std::atomic<int> occ{0};
            int per_sm = occ.load(std::memory_order_relaxed);
            if (per_sm == 0) {
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stencil_march<SUB, true>, 128, 0) !=
                    cudaSuccess)
                    per_sm = 0;
                occ.store(per_sm, std::memory_order_relaxed);
            }
            const long long slots = (long long)std::max(per_sm, 1) * std::max(g->ctx->sm_count, 1);
            const long long xy = (long long)gx * gy * ncc;
            const int nz = g->d.nz;
            mzc = std::min(nz, 8);
            for (int nch = 1; nch <= nz; ++nch) {
                const int c = (nz + nch - 1) / nch;
                if (c > 64) continue;
                mzc = std::max(c, std::min(nz, 8));
                if (c <= 8 || xy * ((nz + c - 1) / c) >= 2 * slots) break;
            }
        }
        const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)((g->d.nz + mzc - 1) / mzc * ncc));
        if (g->k2_real)
            stencil_march<SUB, true><<<grid, 128, 0, s>>>((const c64*)u, (const c64*)b, (c64*)y, g->k2f, g->tabf,
                                                          g->d.nx, g->d.ny, g->d.nz, nrhs, mzc, g->w, pl,
                                                          g->ctx->stencil_march == 2 ? 1 : 0);
        else
            stencil_march<SUB, false><<<grid, 128, 0, s>>>((const c64*)u, (const c64*)b, (c64*)y, g->k2f, g->tabf,
                                                           g->d.nx, g->d.ny, g->d.nz, nrhs, mzc, g->w, pl,
                                                          g->ctx->stencil_march == 2 ? 1 : 0);
    } else {
        dispatch<float, SUB>((const c64*)u, (const c64*)b, (c64*)y, g->k2f, g->tabf, g->d, nrhs, g->w, in,
                             g->k2_real, rw, s);
    }
    prof_end(g->ctx, tok, bytes);
    HELM_LAUNCH_CHECK(g->ctx, "stencil_kernel");
    return HELM_OK;
}

}  // namespace

helm_status launch_stencil(helm_grid g, int prec, const void* u, void* y, int nrhs, cudaStream_t s) {
    return launch_any<false>(g, prec, u, nullptr, y, nrhs, s);
}

helm_status launch_stencil_sub(helm_grid g, int prec, const void* u, const void* b, void* y, int nrhs, cudaStream_t s) {
    return launch_any<true>(g, prec, u, b, y, nrhs, s);
}
