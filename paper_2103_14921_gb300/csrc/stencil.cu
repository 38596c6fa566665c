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

template <bool SUB>
helm_status launch_any(helm_grid g, int prec, const void* u, const void* b, void* y, int nrhs, cudaStream_t s) {
    if (nrhs <= 0) return HELM_OK;
    // algorithmic bytes: read u (and b), write y, read k^2 once
    const double es = prec == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);
    const double bytes = (double)g->n * es * ((SUB ? 3.0 : 2.0) * nrhs + 1.0);
    const int tok = prof_begin(g->ctx, prec == HELM_PREC_FP64 ? "stencil64" : "stencil");
    const Interior in = interior_of(g);
    const RowW rw{g->wtab, g->wbin};
    if (prec == HELM_PREC_FP64) {
        dispatch<double, SUB>((const c128*)u, (const c128*)b, (c128*)y, g->k2, g->tab, g->d, nrhs, g->w, in,
                              g->k2_real, rw, s);
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
