// Two-level ORAS preconditioner (Eq. 2lvl, Eq. oras):
//   M^{-1} v = M1^{-1} (v - A Q v) + Q v,  Q = Z E^{-1} Z^T,  E = Z^T A Z,
//   M1^{-1}  = sum_i R_i^T D_i A_i^{-1} R_i.
//
// * Box subdomains: axis a is cut into p_a cores at floor(t n_a / p_a); each
//   box is its core grown by `overlap` nodes on every side that is not a
//   global face.  R_i is the Boolean gather of the box nodes; D_i is the
//   owner partition of unity (1 on the core, 0 on the overlap), so the sum
//   over boxes reduces to a gather from each node's owner box: deterministic,
//   no atomics.
// * A_i: the rows of A for the box nodes; a stencil neighbour outside the box
//   across an interface face is folded onto the clamped in-box node times
//   rho_p = exp(i k_p h) per crossed face (k_p = omega / c at the row node),
//   an absorbing condition exact for waves leaving the box normally.  With
//   interface_bc = 1 the neighbour is dropped instead (RAS).
// * Coarse space: nodes at fine indices r J, trilinear hats; E = Z^T A Z is a
//   27-point operator on the coarse grid, assembled by probing A with Z e_c
//   for the 27 colours c = J mod 3, and factored plane by plane in FP64.
// * Local solves and the coarse solve use the plane-by-plane block LU of
//   planelu.cu.
#include <cuda_runtime.h>
#include <math.h>

#include <cuda_bf16.h>

#include "coef.cuh"
#include "internal.h"

namespace {

// ------------------------------------------------------------------ local operators

// coef_out[(loc_off + l) * 27 + d'] = sum over offsets d folding onto d' of A_row(d) * rho^crossed
template <typename TO>
__global__ void build_local_coef(const BoxInfo* __restrict__ boxes, const c128* __restrict__ tab,
                                 const c128* __restrict__ k2, const c128* __restrict__ c, int nx, int ny, int nz,
                                 StencilW w, const StencilW* __restrict__ wtab, const unsigned char* __restrict__ wbin,
                                 double omega, double h, int dirichlet, cplx<TO>* __restrict__ out) {
    const BoxInfo B = boxes[blockIdx.y];
    const long long nl = (long long)B.m * B.dims[2];
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += (long long)gridDim.x * blockDim.x) {
        const int li = (int)(l % B.dims[0]);
        const int lj = (int)((l / B.dims[0]) % B.dims[1]);
        const int lk = (int)(l / B.m);
        const int gi = B.lo[0] + li, gj = B.lo[1] + lj, gk = B.lo[2] + lk;
        c128 a[27], loc[27];
        const long long gidx = ((long long)gk * ny + gj) * nx + gi;
        global_row_coef27(tab, k2, nx, ny, nz, wtab ? wtab[wbin[gidx]] : w, gi, gj, gk, a);
        for (int d = 0; d < 27; ++d) loc[d] = mk<double>(0, 0);
        const c128 cv = c[((long long)gk * ny + gj) * nx + gi];
        const double den = cv.x * cv.x + cv.y * cv.y;
        const double kr = omega * cv.x / den, ki = -omega * cv.y / den;   // k = omega / c
        const double mag = exp(-ki * h);
        c128 rho = mk<double>(mag * cos(kr * h), mag * sin(kr * h));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const c128 v = a[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
                    if (v.x == 0.0 && v.y == 0.0) continue;
                    const int qi = li + dx, qj = lj + dy, qk = lk + dz;
                    int crossed = 0;
                    int cx = dx, cy = dy, cz = dz;
                    if (qi < 0 || qi >= B.dims[0]) { crossed++; cx = 0; }
                    if (qj < 0 || qj >= B.dims[1]) { crossed++; cy = 0; }
                    if (qk < 0 || qk >= B.dims[2]) { crossed++; cz = 0; }
                    c128 val = v;
                    if (crossed) {
                        if (dirichlet) continue;
                        for (int t = 0; t < crossed; ++t) val = val * rho;
                    }
                    const int dd = (cz + 1) * 9 + (cy + 1) * 3 + (cx + 1);
                    loc[dd] = loc[dd] + val;
                }
        cplx<TO>* o = out + (B.loc_off + l) * 27;
        for (int d = 0; d < 27; ++d) o[d] = mk<TO>((TO)loc[d].x, (TO)loc[d].y);
    }
}

// Local coefficients of the coarse boxes (inexact coarse solve): rows of E (27 per coarse node, E27) with
// the same folding as the fine boxes, rho = exp(i k H) with H = r h the coarse spacing and k = omega / c at
// the coarse node's fine position r J (clamped to the grid).
template <typename TO>
__global__ void build_local_coef27(const BoxInfo* __restrict__ boxes, const c128* __restrict__ E27,
                                   const c128* __restrict__ c, int nx, int ny, int nz, int cx, int cy, int r,
                                   double omega, double H, int dirichlet, cplx<TO>* __restrict__ out) {
    const BoxInfo B = boxes[blockIdx.y];
    const long long nl = (long long)B.m * B.dims[2];
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += (long long)gridDim.x * blockDim.x) {
        const int li = (int)(l % B.dims[0]);
        const int lj = (int)((l / B.dims[0]) % B.dims[1]);
        const int lk = (int)(l / B.m);
        const int gi = B.lo[0] + li, gj = B.lo[1] + lj, gk = B.lo[2] + lk;
        const c128* a = E27 + (((long long)gk * cy + gj) * cx + gi) * 27;
        c128 loc[27];
        for (int q = 0; q < 27; ++q) loc[q] = mk<double>(0, 0);
        const int fi = min(r * gi, nx - 1), fj = min(r * gj, ny - 1), fk = min(r * gk, nz - 1);
        const c128 cv = c[((long long)fk * ny + fj) * nx + fi];
        const double den = cv.x * cv.x + cv.y * cv.y;
        const double kr = omega * cv.x / den, ki = -omega * cv.y / den;   // k = omega / c
        const double mag = exp(-ki * H);
        const c128 rho = mk<double>(mag * cos(kr * H), mag * sin(kr * H));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const c128 v = a[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
                    if (v.x == 0.0 && v.y == 0.0) continue;
                    const int qi = li + dx, qj = lj + dy, qk = lk + dz;
                    int crossed = 0;
                    int ex = dx, ey = dy, ez = dz;
                    if (qi < 0 || qi >= B.dims[0]) { crossed++; ex = 0; }
                    if (qj < 0 || qj >= B.dims[1]) { crossed++; ey = 0; }
                    if (qk < 0 || qk >= B.dims[2]) { crossed++; ez = 0; }
                    c128 val = v;
                    if (crossed) {
                        if (dirichlet) continue;
                        for (int t = 0; t < crossed; ++t) val = val * rho;
                    }
                    const int dd = (ez + 1) * 9 + (ey + 1) * 3 + (ex + 1);
                    loc[dd] = loc[dd] + val;
                }
        cplx<TO>* o = out + (B.loc_off + l) * 27;
        for (int q = 0; q < 27; ++q) o[q] = mk<TO>((TO)loc[q].x, (TO)loc[q].y);
    }
}

// y = E x on the coarse grid from E's 27 coefficients per node; grid (x-line chunks, y, z)
template <typename T>
__global__ void e27_apply(const cplx<T>* __restrict__ E27, const cplx<T>* __restrict__ x, cplx<T>* __restrict__ y,
                          int cx, int cy, int cz, int nrhs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cx * nrhs) return;
    const int i = t / nrhs, r = t % nrhs;
    const int j = blockIdx.y, k = blockIdx.z;
    const long long p = ((long long)k * cy + j) * cx + i;
    const cplx<T>* a = E27 + p * 27;
    cplx<T> acc = mk<T>(0, 0);
    for (int dz = -1; dz <= 1; ++dz) {
        if (k + dz < 0 || k + dz >= cz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            if (j + dy < 0 || j + dy >= cy) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                if (i + dx < 0 || i + dx >= cx) continue;
                const long long q = p + ((long long)dz * cy + dy) * cx + dx;
                cmac(acc, a[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)], x[q * nrhs + r]);
            }
        }
    }
    y[p * nrhs + r] = acc;
}

// ------------------------------------------------------------------ restriction / prolongation

// loc[(loc_off + l) * nrhs + r] = v[g(l) * nrhs + r]   (R_i v for every box)
template <typename TV, typename TL>
__global__ void restrict_boxes(const BoxInfo* __restrict__ boxes, const cplx<TV>* __restrict__ v,
                               cplx<TL>* __restrict__ loc, int nx, int ny, int nrhs) {
    // grid: (x-line chunks, box rows (y, z) strided, box); 32-bit index arithmetic inside a row
    const BoxInfo B = boxes[blockIdx.z];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.dims[0] * nrhs) return;
    const int li = t / nrhs, r = t % nrhs;
    for (int row = blockIdx.y; row < B.dims[1] * B.dims[2]; row += gridDim.y) {
        const int lj = row % B.dims[1], lk = row / B.dims[1];
        const long long g = ((long long)(B.lo[2] + lk) * ny + (B.lo[1] + lj)) * nx + (B.lo[0] + li);
        const long long l = (long long)row * B.dims[0] + li;
        const cplx<TV> x = v[g * nrhs + r];
        loc[(B.loc_off + l) * nrhs + r] = mk<TL>((TL)x.x, (TL)x.y);
    }
}

// out[g] = loc[owner box of g][local index of g] (+ q[g])     (sum_i R_i^T D_i x_i with Boolean owner PU)
template <typename TL, typename TV, bool ADDQ>
__global__ void prolong_owner(const BoxInfo* __restrict__ boxes, const int* __restrict__ owner,
                              const cplx<TL>* __restrict__ loc, const cplx<TV>* __restrict__ q, cplx<TV>* __restrict__ out,
                              int nx, int ny, int nz, int px, int py, int nrhs) {
    // grid: (x-line chunks, y, z)
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx * nrhs) return;
    const int i = t / nrhs, r = t % nrhs;
    const int j = blockIdx.y, k = blockIdx.z;
    const long long e = (((long long)k * ny + j) * nx + i) * nrhs + r;
    const int b = (owner[nx + ny + k] * py + owner[nx + j]) * px + owner[i];
    const BoxInfo& B = boxes[b];
    const long long l = ((long long)(k - B.lo[2]) * B.dims[1] + (j - B.lo[1])) * B.dims[0] + (i - B.lo[0]);
    const cplx<TL> x = loc[(B.loc_off + l) * nrhs + r];
    cplx<TV> y = mk<TV>((TV)x.x, (TV)x.y);
    if (ADDQ) y = y + q[e];
    out[e] = y;
}

// ------------------------------------------------------------------ coarse space

__device__ __forceinline__ double hat(int i, int J, int r) {
    const double t = fabs((double)(i - r * J)) / r;
    return t < 1.0 ? 1.0 - t : 0.0;
}

// cv[J * nrhs + rr] = sum_i Z[i, J] v[i * nrhs + rr]   (Z^T v)
// Hat weights are (r - |d_x|)(r - |d_y|)(r - |d_z|) / r^3 with integer numerators; the sum is
// accumulated in the input's precision and the result stored in complex128.
template <typename TV, typename TC>
__global__ void coarse_restrict(const cplx<TV>* __restrict__ v, cplx<TC>* __restrict__ cv, int nx, int ny, int nz,
                                int cx, int cy, int cz, int r, int nrhs) {
    const long long total = (long long)cx * cy * cz * nrhs;
    const TV inv_r3 = (TV)1 / (TV)(r * r * r);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long J = e / nrhs;
        const int rr = (int)(e % nrhs);
        const int Jx = (int)(J % cx), Jy = (int)((J / cx) % cy), Jz = (int)(J / ((long long)cx * cy));
        cplx<TV> acc = mk<TV>(0, 0);
        const int k0 = max(0, r * Jz - r + 1), k1 = min(nz - 1, r * Jz + r - 1);
        const int j0 = max(0, r * Jy - r + 1), j1 = min(ny - 1, r * Jy + r - 1);
        const int i0 = max(0, r * Jx - r + 1), i1 = min(nx - 1, r * Jx + r - 1);
        for (int k = k0; k <= k1; ++k) {
            const int wz = r - abs(k - r * Jz);
            for (int j = j0; j <= j1; ++j) {
                const int wyz = wz * (r - abs(j - r * Jy));
                const cplx<TV>* row = v + (((long long)k * ny + j) * nx) * nrhs + rr;
                for (int i = i0; i <= i1; ++i) {
                    const TV wt = (TV)(wyz * (r - abs(i - r * Jx)));
                    const cplx<TV> x = row[(long long)i * nrhs];
                    acc.x += wt * x.x;
                    acc.y += wt * x.y;
                }
            }
        }
        cv[e] = mk<TC>((TC)(acc.x * inv_r3), (TC)(acc.y * inv_r3));
    }
}

inline unsigned grid_for(long long n, int threads = 256, long long cap = 152LL * 16) {
    long long b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// One axis of the separable restriction Z^T = Z_z^T (x) Z_y^T (x) Z_x^T on [n2][n1][n0][R] arrays:
// along axis ax (0 = x, 1 = y, 2 = z) the n nodes are replaced by nc coarse nodes,
// out[.., J, ..] = scale * sum_i (r - |i - r J|) in[.., i, ..] over the hat's support.  Three
// passes read each fine value once (the direct 3-D sum reads it (2r - 1)^3 / r^3 times).
template <typename TI, typename TO>
__global__ void restrict_axis(const cplx<TI>* __restrict__ in, cplx<TO>* __restrict__ out, int n0, int n1, int n2,
                              int ax, int nc, int r, int R, TI scale) {
    const int d0 = ax == 0 ? nc : n0, d1 = ax == 1 ? nc : n1, d2 = ax == 2 ? nc : n2;
    const int n = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
    const long long sa = (ax == 0 ? 1LL : (ax == 1 ? (long long)n0 : (long long)n0 * n1)) * R;
    const long long total = (long long)d0 * d1 * d2 * R;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int rr = (int)(e % R);
        long long t = e / R;
        const int o0 = (int)(t % d0);
        t /= d0;
        const int o1 = (int)(t % d1);
        const int o2 = (int)(t / d1);
        const int J = ax == 0 ? o0 : (ax == 1 ? o1 : o2);
        const long long base = ((((long long)(ax == 2 ? 0 : o2) * n1 + (ax == 1 ? 0 : o1)) * n0) + (ax == 0 ? 0 : o0)) * R + rr;
        const int i0 = max(0, r * J - r + 1), i1 = min(n - 1, r * J + r - 1);
        cplx<TI> acc = mk<TI>(0, 0);
        for (int i = i0; i <= i1; ++i) {
            const TI wt = (TI)(r - abs(i - r * J));
            const cplx<TI> x = in[base + (long long)i * sa];
            acc.x += wt * x.x;
            acc.y += wt * x.y;
        }
        out[e] = mk<TO>((TO)(acc.x * scale), (TO)(acc.y * scale));
    }
}

// cv = Z^T v / r^3 by three axis passes (x into t1, y into t2, z into cv)
template <typename TV, typename TC>
void restrict_separable(const cplx<TV>* v, cplx<TV>* t1, cplx<TV>* t2, cplx<TC>* cv, int nx, int ny, int nz, int cx,
                        int cy, int cz, int r, int R, cudaStream_t st) {
    const TV one = (TV)1, s3 = (TV)1 / (TV)(r * r * r);
    restrict_axis<TV, TV><<<grid_for((long long)nz * ny * cx * R), 256, 0, st>>>(v, t1, nx, ny, nz, 0, cx, r, R, one);
    restrict_axis<TV, TV><<<grid_for((long long)nz * cy * cx * R), 256, 0, st>>>(t1, t2, cx, ny, nz, 1, cy, r, R, one);
    restrict_axis<TV, TC><<<grid_for((long long)cz * cy * cx * R), 256, 0, st>>>(t2, cv, cx, cy, nz, 2, cz, r, R, s3);
}

// q[i * nrhs + rr] = sum_J Z[i, J] cv[J * nrhs + rr]   (trilinear interpolation, weights (i mod r)/r,
// exact in binary for r a power of two; accumulated in the output precision)
template <typename TC, typename TV>
__global__ void coarse_prolong(const cplx<TC>* __restrict__ cv, cplx<TV>* __restrict__ q, int nx, int ny, int nz,
                               int cx, int cy, int cz, int r, int nrhs) {
    // grid: (x-line chunks, y, z)
    const TV inv_r = (TV)1 / (TV)r;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx * nrhs) return;
    const int i = t / nrhs, rr = t % nrhs;
    const int j = blockIdx.y, k = blockIdx.z;
    const long long e = (((long long)k * ny + j) * nx + i) * nrhs + rr;
    const int I0 = i / r, J0 = j / r, K0 = k / r;
    const TV wx1 = (TV)(i - r * I0) * inv_r, wy1 = (TV)(j - r * J0) * inv_r, wz1 = (TV)(k - r * K0) * inv_r;
    const TV wx[2] = {(TV)1 - wx1, wx1}, wy[2] = {(TV)1 - wy1, wy1}, wz[2] = {(TV)1 - wz1, wz1};
    cplx<TV> acc = mk<TV>(0, 0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
        const TV wt = wx[a] * wy[b] * wz[d];
        if (wt == (TV)0 || I0 + a >= cx || J0 + b >= cy || K0 + d >= cz) continue;
        const cplx<TC> x = cv[(((long long)(K0 + d) * cy + (J0 + b)) * cx + (I0 + a)) * nrhs + rr];
        acc.x += wt * (TV)x.x;
        acc.y += wt * (TV)x.y;
    }
    q[e] = acc;
}

// The same for complex64 with an even column count: a thread per fine node forms the 8 trilinear weights
// and corner indices once and sweeps the columns in 16-byte pairs (the per-column kernel repeats that
// integer work for every column).  grid: (x-line chunks of 128 nodes, y, z).
__global__ void coarse_prolong_pairs(const c64* __restrict__ cv, c64* __restrict__ q, int nx, int ny, int nz, int cx,
                                     int cy, int cz, int r, int nrhs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int j = blockIdx.y, k = blockIdx.z;
    const float inv_r = 1.0f / (float)r;
    const int I0 = i / r, J0 = j / r, K0 = k / r;
    const float wx1 = (float)(i - r * I0) * inv_r, wy1 = (float)(j - r * J0) * inv_r, wz1 = (float)(k - r * K0) * inv_r;
    const float wx[2] = {1.0f - wx1, wx1}, wy[2] = {1.0f - wy1, wy1}, wz[2] = {1.0f - wz1, wz1};
    float wt[8];
    long long base[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
        const bool in = I0 + a < cx && J0 + b < cy && K0 + d < cz;
        wt[c] = in ? wx[a] * wy[b] * wz[d] : 0.0f;
        // a corner past the coarse grid has weight 0: point it at the base corner
        base[c] = in ? (((long long)(K0 + d) * cy + (J0 + b)) * cx + (I0 + a)) * nrhs
                     : (((long long)K0 * cy + J0) * cx + I0) * nrhs;
    }
    float4* out = reinterpret_cast<float4*>(q + (((long long)k * ny + j) * nx + i) * nrhs);
    for (int p = 0; p < nrhs / 2; ++p) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 x = *reinterpret_cast<const float4*>(cv + base[c] + 2 * p);
            acc.x += wt[c] * x.x;
            acc.y += wt[c] * x.y;
            acc.z += wt[c] * x.z;
            acc.w += wt[c] * x.w;
        }
        out[p] = acc;
    }
}

// Probe vectors: zc[i * 27 + c] = (Z e_c)_i, e_c = indicator of the coarse nodes of colour c = (J mod 3).
__global__ void coarse_probe_vectors(c128* __restrict__ zc, int nx, int ny, int nz, int cx, int cy, int cz, int r) {
    const long long n = (long long)nx * ny * nz;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g % nx), j = (int)((g / nx) % ny), k = (int)(g / ((long long)nx * ny));
        const int idx[3] = {i, j, k};
        const int cdim[3] = {cx, cy, cz};
        double wa[3][3];
        for (int a = 0; a < 3; ++a) {
            wa[a][0] = wa[a][1] = wa[a][2] = 0.0;
            const int J0 = idx[a] / r;
            for (int J = J0; J <= min(J0 + 1, cdim[a] - 1); ++J) wa[a][J % 3] += hat(idx[a], J, r);
        }
        for (int c = 0; c < 27; ++c) {
            const int c0 = c % 3, c1 = (c / 3) % 3, c2 = c / 9;
            zc[g * 27 + c] = mk<double>(wa[0][c0] * wa[1][c1] * wa[2][c2], 0.0);
        }
    }
}

// E27[J * 27 + d] = probe[J][colour(J + d)] for neighbours inside the coarse grid, else 0.
__global__ void coarse_gather_E(const c128* __restrict__ probe, c128* __restrict__ E27, int cx, int cy, int cz) {
    const long long nc = (long long)cx * cy * cz;
    for (long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x; J < nc; J += (long long)gridDim.x * blockDim.x) {
        const int Jx = (int)(J % cx), Jy = (int)((J / cx) % cy), Jz = (int)(J / ((long long)cx * cy));
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    const int X = Jx + dx, Y = Jy + dy, Zc = Jz + dz;
                    c128 v = mk<double>(0, 0);
                    if (X >= 0 && X < cx && Y >= 0 && Y < cy && Zc >= 0 && Zc < cz) {
                        const int col = (X % 3) + 3 * (Y % 3) + 9 * (Zc % 3);
                        v = probe[J * 27 + col];
                    }
                    E27[J * 27 + d] = v;
                }
    }
}

__global__ void narrow_c128(const c128* __restrict__ a, c64* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = mk<float>((float)a[i].x, (float)a[i].y);
}

}  // namespace

// ------------------------------------------------------------------ factor

// The inexact coarse solve's one-level ORAS on the coarse grid: the fine partition carried to the coarse
// nodes (coarse node J goes to the part whose fine core holds r J; the last coarse node, which may lie
// past the fine grid, to the last part), coarse_overlap layers on interior sides, local operators from
// E's rows with the absorbing fold, FP64 plane factors (and complex64 copies with mixed fine factors).
static helm_status setup_coarse_dd(helm_oras o, const std::vector<int>& cuts) {
    helm_grid g = o->g;
    helm_ctx ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const helm_oras_desc& d = o->d;
    const int n[3] = {g->d.nx, g->d.ny, g->d.nz};
    const int p[3] = {d.px, d.py, d.pz};
    const int r = d.coarse_ratio;
    std::vector<int> cc[3];
    std::vector<int> cowner(o->cdims[0] + o->cdims[1] + o->cdims[2]);
    int base = 0, fb = 0;
    for (int a = 0; a < 3; ++a) {
        cc[a].push_back(0);
        for (int t = 1; t < p[a]; ++t) cc[a].push_back((cuts[fb + t] + r - 1) / r);
        cc[a].push_back(o->cdims[a]);
        for (int t = 0; t < p[a]; ++t) {
            if (cc[a][t + 1] <= cc[a][t])
                return set_error(ctx, HELM_EINVAL, "oras_factor: the coarse grid is too small for the partition");
            for (int J = cc[a][t]; J < cc[a][t + 1]; ++J) cowner[base + J] = t;
        }
        base += o->cdims[a];
        fb += p[a] + 1;
        (void)n;
    }
    const int ov = d.coarse_overlap;
    for (int tz = 0; tz < p[2]; ++tz)
        for (int ty = 0; ty < p[1]; ++ty)
            for (int tx = 0; tx < p[0]; ++tx) {
                BoxInfo b{};
                const int t[3] = {tx, ty, tz};
                for (int a = 0; a < 3; ++a) {
                    const int c0 = cc[a][t[a]], c1 = cc[a][t[a] + 1];
                    b.core_lo[a] = c0;
                    b.core_hi[a] = c1;
                    b.lo[a] = c0 > 0 ? std::max(0, c0 - ov) : 0;
                    const int hi = c1 < o->cdims[a] ? std::min(o->cdims[a], c1 + ov) : o->cdims[a];
                    b.dims[a] = hi - b.lo[a];
                }
                o->cdd.hbox.push_back(b);
            }
    o->cdd.prec = HELM_PREC_FP64;
    HELM_TRY(planeset_alloc(ctx, o->cdd));
    HELM_TRY(dev_alloc(ctx, (void**)&o->cowner, cowner.size() * sizeof(int), "coarse owner table"));
    HELM_CUDA(ctx, cudaMemcpyAsync(o->cowner, cowner.data(), cowner.size() * sizeof(int), cudaMemcpyHostToDevice,
                                   ctx->stream));
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    long long mx = 0;
    for (auto& b : o->cdd.hbox) mx = std::max(mx, (long long)b.m * b.dims[2]);
    build_local_coef27<double><<<dim3(grid_for(mx, 128, 4096), o->cdd.nbox), 128, 0, st>>>(
        o->cdd.dbox, (const c128*)o->coarse.coef, g->c, n[0], n[1], n[2], o->cdims[0], o->cdims[1], r, g->omega,
        r * g->d.h, d.interface_bc, (c128*)o->cdd.coef);
    ctx->launches++;
    HELM_CUDA(ctx, cudaGetLastError());
    int singular = 0;
    HELM_TRY(planeset_factor(ctx, o->cdd, &singular));
    if (singular) return set_error(ctx, HELM_ESINGULAR, "oras_factor: zero pivot in a coarse local factor");
    // complex64 copies: E for FP32 work vectors, and the local factors with mixed fine factors
    HELM_TRY(dev_alloc(ctx, &o->Ecoef32, (size_t)o->nc * 27 * sizeof(c64), "coarse operator (complex64)"));
    narrow_c128<<<grid_for(o->nc * 27), 256, 0, st>>>((const c128*)o->coarse.coef, (c64*)o->Ecoef32, o->nc * 27);
    ctx->launches++;
    if (o->fine.prec != HELM_PREC_FP64) {
        o->cdd32.prec = HELM_PREC_FP32;
        o->cdd32.hbox = o->cdd.hbox;
        HELM_TRY(planeset_alloc(ctx, o->cdd32));
        narrow_c128<<<grid_for((long long)o->cdd.nloc * 27), 256, 0, st>>>(
            (const c128*)o->cdd.coef, (c64*)o->cdd32.coef, (long long)o->cdd.nloc * 27);
        narrow_c128<<<grid_for((long long)o->cdd.fac_entries), 256, 0, st>>>(
            (const c128*)o->cdd.G, (c64*)o->cdd32.G, (long long)o->cdd.fac_entries);
        ctx->launches += 2;
    }
    return cuda_check(ctx, cudaGetLastError(), "coarse subdomain set-up");
}

extern "C" helm_status oras_factor(helm_grid g, const helm_oras_desc* d, helm_oras* out) {
    if (!g || !d || !out) return set_error(g ? g->ctx : nullptr, HELM_EINVAL, "oras_factor: NULL argument");
    helm_ctx ctx = g->ctx;
    *out = nullptr;
    const int n[3] = {g->d.nx, g->d.ny, g->d.nz};
    const int p[3] = {d->px, d->py, d->pz};
    for (int a = 0; a < 3; ++a)
        if (p[a] < 1 || p[a] > n[a]) return set_error(ctx, HELM_EINVAL, "oras_factor: bad number of boxes");
    if (d->overlap < 0 || d->coarse_ratio < 0)
        return set_error(ctx, HELM_EINVAL, "oras_factor: bad overlap or coarse ratio");
    if (d->interface_bc != 0 && d->interface_bc != 1) return set_error(ctx, HELM_EINVAL, "oras_factor: bad interface_bc");
    if (d->coarse_iters < 0 || d->coarse_iters > 200 || (d->coarse_iters > 0 && (d->coarse_ratio < 1 || d->coarse_overlap < 0)))
        return set_error(ctx, HELM_EINVAL, "oras_factor: coarse_iters needs 0..200 with a coarse grid and coarse_overlap >= 0");
    if (d->factor_prec < HELM_PREC_FP64 || d->factor_prec > HELM_PREC_BF16)
        return set_error(ctx, HELM_EINVAL, "oras_factor: bad factor_prec");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);

    helm_oras o = new helm_oras_s();
    o->g = g;
    o->d = *d;
    g->refs++;
    helm_status rc = HELM_OK;
    auto fail = [&](helm_status s) {
        oras_destroy(o);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
    };

    // --- box decomposition
    std::vector<int> cuts;
    std::vector<int> owner(n[0] + n[1] + n[2]);
    int base = 0;
    for (int a = 0; a < 3; ++a) {
        for (int t = 0; t <= p[a]; ++t) cuts.push_back((int)((long long)t * n[a] / p[a]));
        for (int t = 0; t < p[a]; ++t) {
            const int c0 = (int)((long long)t * n[a] / p[a]), c1 = (int)((long long)(t + 1) * n[a] / p[a]);
            for (int i = c0; i < c1; ++i) owner[base + i] = t;
        }
        base += n[a];
    }
    if (d->factor_prec == HELM_PREC_TF32X3)
        return fail(set_error(ctx, HELM_EINVAL, "oras_factor: TF32X3 factors are not available"));
    o->fine.prec = d->factor_prec == HELM_PREC_FP64 ? HELM_PREC_FP64 : HELM_PREC_FP32;
    o->fine.padded = d->factor_prec == HELM_PREC_TF32 || d->factor_prec == HELM_PREC_BF16;
    if ((rc = dev_alloc(ctx, (void**)&o->dev_err, sizeof(int), "device error flag"))) return fail(rc);
    if ((rc = cuda_check(ctx, cudaMemsetAsync(o->dev_err, 0, sizeof(int), st), "clear error flag"))) return fail(rc);
    for (int tz = 0; tz < p[2]; ++tz)
        for (int ty = 0; ty < p[1]; ++ty)
            for (int tx = 0; tx < p[0]; ++tx) {
                BoxInfo b{};
                const int t[3] = {tx, ty, tz};
                for (int a = 0; a < 3; ++a) {
                    const int c0 = (int)((long long)t[a] * n[a] / p[a]), c1 = (int)((long long)(t[a] + 1) * n[a] / p[a]);
                    if (c1 <= c0) return fail(set_error(ctx, HELM_EINVAL, "oras_factor: empty box core"));
                    b.core_lo[a] = c0;
                    b.core_hi[a] = c1;
                    b.lo[a] = c0 > 0 ? std::max(0, c0 - d->overlap) : 0;
                    const int hi = c1 < n[a] ? std::min(n[a], c1 + d->overlap) : n[a];
                    b.dims[a] = hi - b.lo[a];
                }
                o->fine.hbox.push_back(b);
            }
    if ((rc = planeset_alloc(ctx, o->fine))) return fail(rc);
    if ((rc = dev_alloc(ctx, (void**)&o->owner, owner.size() * sizeof(int), "owner table"))) return fail(rc);
    if ((rc = cuda_check(ctx, cudaMemcpyAsync(o->owner, owner.data(), owner.size() * sizeof(int),
                                              cudaMemcpyHostToDevice, st), "owner copy")) ||
        (rc = cuda_check(ctx, cudaStreamSynchronize(st), "owner copy")))
        return fail(rc);

    // --- local operators with absorbing interface folding
    {
        long long mx = 0;
        for (auto& b : o->fine.hbox) mx = std::max(mx, (long long)b.m * b.dims[2]);
        const dim3 grid(grid_for(mx, 128, 4096), o->fine.nbox);
        if (o->fine.prec == HELM_PREC_FP64)
            build_local_coef<double><<<grid, 128, 0, st>>>(o->fine.dbox, g->tab, g->k2, g->c, n[0], n[1], n[2], g->w,
                                                           g->wtab, g->wbin, g->omega, g->d.h, d->interface_bc,
                                                           (c128*)o->fine.coef);
        else
            build_local_coef<float><<<grid, 128, 0, st>>>(o->fine.dbox, g->tab, g->k2, g->c, n[0], n[1], n[2], g->w,
                                                          g->wtab, g->wbin, g->omega, g->d.h, d->interface_bc,
                                                          (c64*)o->fine.coef);
        ctx->launches++;
        if ((rc = cuda_check(ctx, cudaGetLastError(), "build_local_coef"))) return fail(rc);
    }
    int singular = 0;
    if ((rc = planeset_factor(ctx, o->fine, &singular))) return fail(rc);
    if (singular) return fail(set_error(ctx, HELM_ESINGULAR, "oras_factor: zero pivot in a local plane factor"));
    if (d->factor_prec == HELM_PREC_BF16 && (rc = planeset_to_bf16(ctx, o->fine))) return fail(rc);
    if (o->fine.padded && (rc = planeset_pack_tc(ctx, o->fine))) return fail(rc);

    // --- coarse level
    if (d->coarse_ratio > 0) {
        const int r = d->coarse_ratio;
        for (int a = 0; a < 3; ++a) o->cdims[a] = (n[a] - 1 + r - 1) / r + 1;
        o->nc = (long long)o->cdims[0] * o->cdims[1] * o->cdims[2];
        const long long N = g->n;
        c128 *zc = nullptr, *az = nullptr, *probe = nullptr;
        auto cfree = [&]() {
            dev_free(ctx, zc, N * 27 * sizeof(c128));
            dev_free(ctx, az, N * 27 * sizeof(c128));
            dev_free(ctx, probe, o->nc * 27 * sizeof(c128));
        };
        if ((rc = dev_alloc(ctx, (void**)&zc, N * 27 * sizeof(c128), "coarse probes")) ||
            (rc = dev_alloc(ctx, (void**)&az, N * 27 * sizeof(c128), "coarse probes A")) ||
            (rc = dev_alloc(ctx, (void**)&probe, o->nc * 27 * sizeof(c128), "coarse probe results"))) {
            cfree();
            return fail(rc);
        }
        coarse_probe_vectors<<<grid_for(N), 256, 0, st>>>(zc, n[0], n[1], n[2], o->cdims[0], o->cdims[1], o->cdims[2],
                                                          r);
        ctx->launches++;
        if ((rc = launch_stencil(g, HELM_PREC_FP64, zc, az, 27, st))) { cfree(); return fail(rc); }
        coarse_restrict<double, double><<<grid_for(o->nc * 27), 256, 0, st>>>(az, probe, n[0], n[1], n[2], o->cdims[0],
                                                                       o->cdims[1], o->cdims[2], r, 27);
        ctx->launches++;
        BoxInfo cb{};
        for (int a = 0; a < 3; ++a) {
            cb.lo[a] = 0;
            cb.dims[a] = o->cdims[a];
            cb.core_lo[a] = 0;
            cb.core_hi[a] = o->cdims[a];
        }
        o->coarse.prec = HELM_PREC_FP64;
        o->coarse.hbox.push_back(cb);
        o->coarse.coef_only = d->coarse_iters > 0;   // the inexact solve applies E, it does not factor it
        if ((rc = planeset_alloc(ctx, o->coarse))) { cfree(); return fail(rc); }
        coarse_gather_E<<<grid_for(o->nc), 256, 0, st>>>(probe, (c128*)o->coarse.coef, o->cdims[0], o->cdims[1],
                                                         o->cdims[2]);
        ctx->launches++;
        rc = cuda_check(ctx, cudaStreamSynchronize(st), "coarse operator");
        cfree();
        if (rc) return fail(rc);
        if (d->coarse_iters > 0) {
            if ((rc = setup_coarse_dd(o, cuts))) return fail(rc);
            cudaEventRecord(e1, st);
            if ((rc = cuda_check(ctx, cudaEventSynchronize(e1), "oras_factor"))) return fail(rc);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            o->setup_s = ms * 1e-3;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            *out = o;
            return HELM_OK;
        }
        if ((rc = planeset_factor(ctx, o->coarse, &singular))) return fail(rc);
        if (singular) return fail(set_error(ctx, HELM_ESINGULAR, "oras_factor: zero pivot in the coarse factor"));
        if (o->fine.prec != HELM_PREC_FP64) {
            // mixed precision: the coarse factors computed in FP64 are applied from a complex64 copy
            o->coarse32.prec = HELM_PREC_FP32;
            o->coarse32.hbox = o->coarse.hbox;
            if ((rc = planeset_alloc(ctx, o->coarse32))) return fail(rc);
            narrow_c128<<<grid_for((long long)o->coarse.nloc * 27), 256, 0, st>>>(
                (const c128*)o->coarse.coef, (c64*)o->coarse32.coef, (long long)o->coarse.nloc * 27);
            narrow_c128<<<grid_for((long long)o->coarse.fac_entries), 256, 0, st>>>(
                (const c128*)o->coarse.G, (c64*)o->coarse32.G, (long long)o->coarse.fac_entries);
            ctx->launches += 2;
            if ((rc = cuda_check(ctx, cudaGetLastError(), "coarse narrow"))) return fail(rc);
        }
    }
    cudaEventRecord(e1, st);
    if ((rc = cuda_check(ctx, cudaEventSynchronize(e1), "oras_factor"))) return fail(rc);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    o->setup_s = ms * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *out = o;
    return HELM_OK;
}

// Planes in the fine sweep buffer: one prepared plane per box; a single box also keeps the
// 8 split-K partial planes of its sweeps there.
static int rbuf_planes(helm_oras o) { return o->fine.nbox == 1 ? 9 : o->fine.nbox; }

static size_t tc_elem(helm_oras o) { return o->fine.prec == HELM_PREC_BF16 ? 2 : sizeof(float); }

static void free_scratch(helm_oras o) {
    helm_ctx ctx = o->g->ctx;
    if (!o->cap_nrhs) return;
    const size_t fe = o->fine.cesize();
    const size_t we = o->cap_wp == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);
    const int R = o->cap_nrhs;
    dev_free(ctx, o->loc, (size_t)o->fine.nloc * R * fe);
    dev_free(ctx, o->rbuf, (size_t)rbuf_planes(o) * o->fine.m_max * R * fe);
    dev_free(ctx, o->cvec, (size_t)o->nc * R * sizeof(c128));
    if (o->d.coarse_iters == 0) dev_free(ctx, o->crbuf, (size_t)9 * o->coarse.m_max * R * sizeof(c128));
    dev_free(ctx, o->qf, (size_t)o->g->n * R * we);
    dev_free(ctx, o->tf, (size_t)o->g->n * R * we);
    dev_free(ctx, o->tcb, (size_t)o->fine.nbox * o->tc_npad * 2 * o->fine.ld * tc_elem(o));
    if (o->fine.padded) dev_free(ctx, o->lb, (size_t)o->fine.nloc * R * fe);
    o->tcb = nullptr;
    o->lb = nullptr;
    o->tc_npad = 0;
    tc_flow_free(ctx, o->flow);
    o->loc = o->rbuf = o->qf = o->tf = nullptr;
    o->cvec = o->crbuf = nullptr;
    dev_free(ctx, o->cy, (size_t)o->nc * R * sizeof(c128));
    dev_free(ctx, o->cloc, (size_t)o->cdd.nloc * R * sizeof(c128));
    dev_free(ctx, o->crb, (size_t)o->cdd.nbox * o->cdd.m_max * R * sizeof(c128));
    o->cy = o->cloc = o->crb = nullptr;
    inner_free(o);
    o->cap_nrhs = 0;
}

static helm_status ensure_scratch(helm_oras o, int wp, int nrhs) {
    if (o->cap_nrhs >= nrhs && o->cap_wp == wp) return HELM_OK;
    helm_ctx ctx = o->g->ctx;
    cudaStreamSynchronize(ctx->stream);
    free_scratch(o);
    o->scratch_gen++;   // graphs captured over the old buffers are stale
    const size_t fe = o->fine.cesize();
    const size_t we = wp == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);
    o->cap_nrhs = nrhs;
    o->cap_wp = wp;
    const int R = nrhs;
    HELM_TRY(dev_alloc(ctx, &o->loc, (size_t)o->fine.nloc * R * fe, "local vectors"));
    HELM_TRY(dev_alloc(ctx, &o->rbuf, (size_t)rbuf_planes(o) * o->fine.m_max * R * fe, "sweep buffer"));
    if (o->fine.padded) {
        o->tc_npad = tc_npad(R);
        const size_t bytes = (size_t)o->fine.nbox * o->tc_npad * 2 * o->fine.ld * tc_elem(o);
        HELM_TRY(dev_alloc(ctx, &o->tcb, bytes, "tensor-core sweep operand"));
        HELM_CUDA(ctx, cudaMemsetAsync(o->tcb, 0, bytes, ctx->stream));
        HELM_TRY(dev_alloc(ctx, &o->lb, (size_t)o->fine.nloc * R * fe, "restricted right-hand sides"));
        if (!o->flow.mem) HELM_TRY(tc_flow_alloc(ctx, o->fine, o->flow, tc_flow_tpn(R)));
    }
    if (o->nc) {
        HELM_TRY(dev_alloc(ctx, (void**)&o->cvec, (size_t)o->nc * R * sizeof(c128), "coarse vector"));
        // coarse sweep buffer: the prepared plane plus 8 split-K partial planes
        if (o->d.coarse_iters == 0)
            HELM_TRY(dev_alloc(ctx, (void**)&o->crbuf, (size_t)9 * o->coarse.m_max * R * sizeof(c128),
                               "coarse sweep buffer"));
        HELM_TRY(dev_alloc(ctx, &o->qf, (size_t)o->g->n * R * we, "coarse correction"));
        HELM_TRY(dev_alloc(ctx, &o->tf, (size_t)o->g->n * R * we, "coarse residual"));
    }
    if (o->d.coarse_iters > 0) {
        HELM_TRY(dev_alloc(ctx, &o->cy, (size_t)o->nc * R * sizeof(c128), "inner coarse solution"));
        HELM_TRY(dev_alloc(ctx, &o->cloc, (size_t)o->cdd.nloc * R * sizeof(c128), "coarse local vectors"));
        HELM_TRY(dev_alloc(ctx, &o->crb, (size_t)o->cdd.nbox * o->cdd.m_max * R * sizeof(c128),
                           "coarse sweep buffer (subdomains)"));
        HELM_TRY(inner_alloc(o, wp, R));
    }
    return HELM_OK;
}

// ------------------------------------------------------------------ apply

namespace {

template <typename TV, typename TL>
helm_status apply_t(helm_oras o, const cplx<TV>* v, cplx<TV>* out, int nrhs) {
    helm_grid g = o->g;
    helm_ctx ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const int wp = sizeof(TV) == 8 ? HELM_PREC_FP64 : HELM_PREC_FP32;
    const long long N = g->n;
    const int nx = g->d.nx, ny = g->d.ny, nz = g->d.nz;
    const cplx<TV>* src = v;
    const cplx<TV>* q = nullptr;
    if (o->nc) {
        const int r = o->d.coarse_ratio;
        const int cx = o->cdims[0], cy = o->cdims[1], cz = o->cdims[2];
        const double vb = (double)N * nrhs * sizeof(cplx<TV>);
        // the restriction's intermediates live in tf and qf, free until the prolongation and t = v - A q
        cplx<TV>* t1 = (cplx<TV>*)o->tf;
        cplx<TV>* t2 = (cplx<TV>*)o->qf;
        int tk = prof_begin(ctx, "coarse_restrict");
        if (o->d.coarse_iters > 0) {
            // the paper's inexact coarse solve: coarse_iters GMRES steps with one-level ORAS on the coarse grid
            restrict_separable<TV, TV>(v, t1, t2, (cplx<TV>*)o->cvec, nx, ny, nz, cx, cy, cz, r, nrhs, st);
            prof_end(ctx, tk, vb);
            HELM_TRY(inner_solve(o, wp, o->cvec, o->cy, nrhs));
            tk = prof_begin(ctx, "coarse_prolong");
            coarse_prolong<TV, TV><<<dim3((unsigned)((nx * nrhs + 255) / 256), (unsigned)ny, (unsigned)nz), 256, 0,
                                     st>>>((const cplx<TV>*)o->cy, (cplx<TV>*)o->qf, nx, ny, nz, cx, cy, cz, r, nrhs);
        } else if (o->coarse32.G) {
            restrict_separable<TV, float>(v, t1, t2, (c64*)o->cvec, nx, ny, nz, cx, cy, cz, r, nrhs, st);
            prof_end(ctx, tk, vb);
            HELM_TRY(planeset_solve(ctx, o->coarse32, o->cvec, o->crbuf, nrhs, st, o->dev_err));
            tk = prof_begin(ctx, "coarse_prolong");
            if (sizeof(TV) == 4 && nrhs % 2 == 0 && (((uintptr_t)o->cvec | (uintptr_t)o->qf) & 15) == 0)
                coarse_prolong_pairs<<<dim3((unsigned)((nx + 127) / 128), (unsigned)ny, (unsigned)nz), 128, 0, st>>>(
                    (const c64*)o->cvec, (c64*)o->qf, nx, ny, nz, cx, cy, cz, r, nrhs);
            else
                coarse_prolong<float, TV><<<dim3((unsigned)((nx * nrhs + 255) / 256), (unsigned)ny, (unsigned)nz), 256,
                                            0, st>>>((const c64*)o->cvec, (cplx<TV>*)o->qf, nx, ny, nz, cx, cy, cz, r,
                                                     nrhs);
        } else {
            restrict_separable<TV, double>(v, t1, t2, o->cvec, nx, ny, nz, cx, cy, cz, r, nrhs, st);
            prof_end(ctx, tk, vb);
            HELM_TRY(planeset_solve(ctx, o->coarse, o->cvec, o->crbuf, nrhs, st));
            tk = prof_begin(ctx, "coarse_prolong");
            coarse_prolong<double, TV><<<dim3((unsigned)((nx * nrhs + 255) / 256), (unsigned)ny, (unsigned)nz), 256, 0,
                                         st>>>(o->cvec, (cplx<TV>*)o->qf, nx, ny, nz, cx, cy, cz, r, nrhs);
        }
        prof_end(ctx, tk, vb);
        ctx->launches += 4;
        HELM_TRY(launch_stencil_sub(g, wp, o->qf, v, o->tf, nrhs, st));   // t = v - A q
        src = (const cplx<TV>*)o->tf;
        q = (const cplx<TV>*)o->qf;
    }
    long long mx = 0;
    for (auto& b : o->fine.hbox) mx = std::max(mx, (long long)b.m * b.dims[2] * nrhs);
    const double lb = (double)o->fine.nloc * nrhs * (sizeof(cplx<TV>) + sizeof(cplx<TL>));
    int tr = prof_begin(ctx, "oras_transfer");
    // the tensor-core sweeps keep b apart (o->lb): their forward step overwrites loc while others read b
    cplx<TL>* rdst = (cplx<TL>*)(o->fine.padded ? o->lb : o->loc);
    int bxm = 0, rows = 0;
    for (auto& b : o->fine.hbox) {
        bxm = std::max(bxm, b.dims[0]);
        rows = std::max(rows, b.dims[1] * b.dims[2]);
    }
    restrict_boxes<TV, TL><<<dim3((unsigned)((bxm * nrhs + 255) / 256), (unsigned)std::min(rows, 65535), o->fine.nbox),
                             256, 0, st>>>(o->fine.dbox, src, rdst, nx, ny, nrhs);
    prof_end(ctx, tr, lb);
    ctx->launches++;
    if (o->fine.padded)
        HELM_TRY(planeset_solve_tc(ctx, o->fine, o->lb, o->loc, o->tcb, o->tc_npad, nrhs, st, o->dev_err, &o->flow));
    else
        HELM_TRY(planeset_solve(ctx, o->fine, o->loc, o->rbuf, nrhs, st));
    tr = prof_begin(ctx, "oras_transfer");
    const dim3 lgrid((unsigned)((nx * nrhs + 255) / 256), (unsigned)ny, (unsigned)nz);   // (x-line chunks, y, z)
    if (q)
        prolong_owner<TL, TV, true><<<lgrid, 256, 0, st>>>(o->fine.dbox, o->owner, (const cplx<TL>*)o->loc, q, out,
                                                           nx, ny, nz, o->d.px, o->d.py, nrhs);
    else
        prolong_owner<TL, TV, false><<<lgrid, 256, 0, st>>>(o->fine.dbox, o->owner, (const cplx<TL>*)o->loc, nullptr,
                                                            out, nx, ny, nz, o->d.px, o->d.py, nrhs);
    prof_end(ctx, tr, (double)N * nrhs * (sizeof(cplx<TL>) + (q ? 2 : 1) * sizeof(cplx<TV>)));
    ctx->launches++;
    return cuda_check(ctx, cudaGetLastError(), "oras apply");
}

}  // namespace

helm_status oras_apply_wp(helm_oras o, int wp, const void* v, void* out, int nrhs) {
    HELM_TRY(ensure_scratch(o, wp, nrhs));
    const bool f64 = o->fine.prec == HELM_PREC_FP64;
    if (wp == HELM_PREC_FP64) {
        if (f64) return apply_t<double, double>(o, (const c128*)v, (c128*)out, nrhs);
        return apply_t<double, float>(o, (const c128*)v, (c128*)out, nrhs);
    }
    if (f64) return apply_t<float, double>(o, (const c64*)v, (c64*)out, nrhs);
    return apply_t<float, float>(o, (const c64*)v, (c64*)out, nrhs);
}

namespace {

template <typename TV, typename TL>
helm_status coarse_dd_t(helm_oras o, const PlaneSet& P, const cplx<TV>* v, cplx<TV>* out, int nrhs) {
    helm_ctx ctx = o->g->ctx;
    cudaStream_t st = ctx->stream;
    const int cx = o->cdims[0], cy = o->cdims[1], cz = o->cdims[2];
    int bxm = 0, rows = 0;
    for (auto& b : P.hbox) {
        bxm = std::max(bxm, b.dims[0]);
        rows = std::max(rows, b.dims[1] * b.dims[2]);
    }
    restrict_boxes<TV, TL><<<dim3((unsigned)((bxm * nrhs + 255) / 256), (unsigned)std::min(rows, 65535), P.nbox), 256, 0,
                             st>>>(P.dbox, v, (cplx<TL>*)o->cloc, cx, cy, nrhs);
    ctx->launches++;
    HELM_TRY(planeset_solve(ctx, P, o->cloc, o->crb, nrhs, st));
    prolong_owner<TL, TV, false><<<dim3((unsigned)((cx * nrhs + 255) / 256), (unsigned)cy, (unsigned)cz), 256, 0, st>>>(
        P.dbox, o->cowner, (const cplx<TL>*)o->cloc, nullptr, out, cx, cy, cz, o->d.px, o->d.py, nrhs);
    ctx->launches++;
    return cuda_check(ctx, cudaGetLastError(), "coarse subdomain solve");
}

}  // namespace

helm_status coarse_dd_apply(helm_oras o, int wp, const void* v, void* out, int nrhs) {
    const PlaneSet& P = o->cdd32.G ? o->cdd32 : o->cdd;
    const bool l64 = P.prec == HELM_PREC_FP64;
    if (wp == HELM_PREC_FP64)
        return l64 ? coarse_dd_t<double, double>(o, P, (const c128*)v, (c128*)out, nrhs)
                   : coarse_dd_t<double, float>(o, P, (const c128*)v, (c128*)out, nrhs);
    return l64 ? coarse_dd_t<float, double>(o, P, (const c64*)v, (c64*)out, nrhs)
               : coarse_dd_t<float, float>(o, P, (const c64*)v, (c64*)out, nrhs);
}

helm_status coarse_E_apply(helm_oras o, int wp, const void* x, void* y, int nrhs) {
    helm_ctx ctx = o->g->ctx;
    const int cx = o->cdims[0], cy = o->cdims[1], cz = o->cdims[2];
    const dim3 grid((unsigned)((cx * nrhs + 255) / 256), (unsigned)cy, (unsigned)cz);
    if (wp == HELM_PREC_FP64)
        e27_apply<double><<<grid, 256, 0, ctx->stream>>>((const c128*)o->coarse.coef, (const c128*)x, (c128*)y, cx, cy,
                                                         cz, nrhs);
    else
        e27_apply<float><<<grid, 256, 0, ctx->stream>>>((const c64*)o->Ecoef32, (const c64*)x, (c64*)y, cx, cy, cz,
                                                        nrhs);
    ctx->launches++;
    return cuda_check(ctx, cudaGetLastError(), "coarse operator apply");
}

extern "C" helm_status oras_apply(helm_oras o, const void* v, void* out, int nrhs) {
    if (!o) return HELM_EINVAL;
    helm_ctx ctx = o->g->ctx;
    if (!v || !out || nrhs < 0) return set_error(ctx, HELM_EINVAL, "oras_apply: invalid argument");
    if (nrhs == 0) return HELM_OK;
    if (v == out) return set_error(ctx, HELM_EINVAL, "oras_apply: v and out must differ");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));
    HELM_TRY(oras_apply_wp(o, HELM_PREC_FP64, v, out, nrhs));
    HELM_TRY(cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "oras_apply"));
    return oras_check_device_error(o);
}

helm_status oras_check_device_error(helm_oras o) {
    helm_ctx ctx = o->g->ctx;
    if (!o->dev_err) return HELM_OK;
    int e = 0;
    HELM_CUDA(ctx, cudaMemcpyAsync(&e, o->dev_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HELM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (e) {
        cudaMemsetAsync(o->dev_err, 0, sizeof(int), ctx->stream);
        return set_error(ctx, HELM_ETIMEOUT, "a bounded device wait gave up (code %d)", e);
    }
    return HELM_OK;
}

extern "C" void oras_destroy(helm_oras o) {
    if (!o) return;
    helm_ctx ctx = o->g->ctx;
    cudaStreamSynchronize(ctx->stream);
    delete o->kcache;
    o->kcache = nullptr;
    free_scratch(o);
    planeset_free(ctx, o->fine);
    planeset_free(ctx, o->coarse);
    planeset_free(ctx, o->coarse32);
    planeset_free(ctx, o->cdd);
    planeset_free(ctx, o->cdd32);
    dev_free(ctx, o->cowner, (size_t)(o->cdims[0] + o->cdims[1] + o->cdims[2]) * sizeof(int));
    dev_free(ctx, o->Ecoef32, (size_t)o->nc * 27 * sizeof(c64));
    const int n = o->g->d.nx + o->g->d.ny + o->g->d.nz;
    dev_free(ctx, o->owner, n * sizeof(int));
    dev_free(ctx, o->dev_err, sizeof(int));
    helm_grid g = o->g;
    delete o;
    if (--g->refs == 0 && g->destroy_pending) helm_destroy_grid(g);
}

extern "C" helm_status oras_box_info(helm_oras o, int box, int* nboxes, int lo[3], int dims[3]) {
    if (!o) return HELM_EINVAL;
    if (nboxes) *nboxes = o->fine.nbox;
    if (box < 0) return HELM_OK;
    if (box >= o->fine.nbox) return set_error(o->g->ctx, HELM_ENOTFOUND, "oras_box_info: box out of range");
    for (int a = 0; a < 3; ++a) {
        if (lo) lo[a] = o->fine.hbox[box].lo[a];
        if (dims) dims[a] = o->fine.hbox[box].dims[a];
    }
    return HELM_OK;
}

namespace {
__global__ void widen_bf16(const __nv_bfloat162* __restrict__ a, c128* __restrict__ b, int m, int ld) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)m * m) return;
    const long long r = i / m, j = i % m;
    const float2 v = __bfloat1622float2(a[r * ld + j]);
    b[i] = mk<double>(v.x, v.y);
}

// b[r * m + j] = a[r * ld + j] widened, for an m x m plane stored with row pitch ld
// entry (r, j) of a plane in the tensor-core tile layout (esz-byte entries, pk_chunks chunks per row)
template <typename T>
__device__ __forceinline__ const T* packed_at(const T* plane, int r, int j, int chunks) {
    const long long off = (long long)j * sizeof(T);
    const long long line = ((long long)(r / 128) * chunks + off / 128) * 128 + (r % 128);
    return reinterpret_cast<const T*>(reinterpret_cast<const unsigned char*>(plane) + line * 128 + off % 128);
}
__global__ void widen_packed_c64(const c64* __restrict__ a, c128* __restrict__ b, int m, int chunks) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)m * m) return;
    const c64 v = *packed_at(a, (int)(i / m), (int)(i % m), chunks);
    b[i] = mk<double>(v.x, v.y);
}
__global__ void widen_packed_bf16(const __nv_bfloat162* __restrict__ a, c128* __restrict__ b, int m, int chunks) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)m * m) return;
    const float2 v = __bfloat1622float2(*packed_at(a, (int)(i / m), (int)(i % m), chunks));
    b[i] = mk<double>(v.x, v.y);
}
__global__ void widen_c64(const c64* __restrict__ a, c128* __restrict__ b, int m, int ld) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)m * m) return;
    const long long r = i / m, j = i % m;
    b[i] = mk<double>(a[r * ld + j].x, a[r * ld + j].y);
}
}  // namespace

extern "C" helm_status oras_plane_inverse(helm_oras o, int box, int plane, void* out) {
    if (!o || !out) return HELM_EINVAL;
    helm_ctx ctx = o->g->ctx;
    if (box < 0 || box >= o->fine.nbox) return set_error(ctx, HELM_ENOTFOUND, "oras_plane_inverse: bad box");
    const BoxInfo& B = o->fine.hbox[box];
    if (plane < 0 || plane >= B.dims[2]) return set_error(ctx, HELM_ENOTFOUND, "oras_plane_inverse: bad plane");
    const long long mm = (long long)B.m * B.m;
    const size_t off = B.fac_off + (size_t)plane * B.pstride;
    const bool dev = is_device_pointer(out);
    c128* tmp = nullptr;
    c128* dst = (c128*)out;
    if (!dev) {
        HELM_TRY(dev_alloc(ctx, (void**)&tmp, mm * sizeof(c128), "plane inverse staging"));
        dst = tmp;
    }
    if (o->fine.prec == HELM_PREC_FP64) {
        cudaMemcpy2DAsync(dst, B.m * sizeof(c128), (c128*)o->fine.G + off, B.ld * sizeof(c128), B.m * sizeof(c128), B.m,
                          cudaMemcpyDeviceToDevice, ctx->stream);
    } else if (o->fine.packed && o->fine.prec == HELM_PREC_BF16) {
        widen_packed_bf16<<<(unsigned)((mm + 255) / 256), 256, 0, ctx->stream>>>(
            (const __nv_bfloat162*)o->fine.G + off, dst, B.m, o->fine.pk_chunks);
        ctx->launches++;
    } else if (o->fine.packed) {
        widen_packed_c64<<<(unsigned)((mm + 255) / 256), 256, 0, ctx->stream>>>((c64*)o->fine.G + off, dst, B.m,
                                                                                o->fine.pk_chunks);
        ctx->launches++;
    } else if (o->fine.prec == HELM_PREC_BF16) {
        widen_bf16<<<(unsigned)((mm + 255) / 256), 256, 0, ctx->stream>>>((const __nv_bfloat162*)o->fine.G + off, dst,
                                                                          B.m, B.ld);
        ctx->launches++;
    } else {
        widen_c64<<<(unsigned)((mm + 255) / 256), 256, 0, ctx->stream>>>((c64*)o->fine.G + off, dst, B.m, B.ld);
        ctx->launches++;
    }
    if (!dev) cudaMemcpyAsync(out, tmp, mm * sizeof(c128), cudaMemcpyDeviceToHost, ctx->stream);
    helm_status rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "oras_plane_inverse");
    if (tmp) dev_free(ctx, tmp, mm * sizeof(c128));
    return rc;
}

extern "C" double oras_setup_seconds(helm_oras o) { return o ? o->setup_s : 0.0; }

// ------------------------------------------------------------------ allocation-free apply
//
// oras_apply_noalloc: the same M^{-1} v as oras_apply, for callers that must
// not have the library allocate device memory during the call -- for example
// an application that has already reserved (almost) all of the GPU's memory
// in its own pool, or a serving loop that cannot afford the device-wide
// synchronisation that cudaMalloc/cudaFree imply.  Its working vectors live
// in one file-scope device array of HELM_NOALLOC_SCRATCH_BYTES (8 MiB), which
// every GPU that loads the library keeps until the process exits.
//
// In host code the array's name only stands for it; its device address is
// looked up with cudaGetSymbolAddress once per device, on that device's first
// call (so make the first call on a device before any stream capture), and
// cached.  All calls share the array and it keeps the last call's contents:
// every working vector is fully written before it is read, so nothing needs
// clearing, but calls whose work overlaps on the GPU (two streams, or two
// threads) race on it.  During the call the handle's working-vector pointers
// point into the array, so no other call may use the same handle (from
// another thread) until this one returns.

#define HELM_NOALLOC_SCRATCH_BYTES (8u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[HELM_NOALLOC_SCRATCH_BYTES];
static void* g_noalloc_ptr[64];

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" helm_status oras_apply_noalloc(helm_oras o, const void* v, void* out, int nrhs) {
    if (!o) return HELM_EINVAL;
    helm_ctx ctx = o->g->ctx;
    if (!v || !out || nrhs < 0) return set_error(ctx, HELM_EINVAL, "oras_apply_noalloc: invalid argument");
    if (nrhs == 0) return HELM_OK;
    if (v == out) return set_error(ctx, HELM_EINVAL, "oras_apply_noalloc: v and out must differ");
    if (ctx->device < 0 || ctx->device >= 64) return set_error(ctx, HELM_EINVAL, "oras_apply_noalloc: device id");
    if (o->d.coarse_iters > 0)
        return set_error(ctx, HELM_EINVAL, "oras_apply_noalloc: not available with the inexact coarse solve");
    HELM_CUDA(ctx, cudaSetDevice(ctx->device));
    // working vectors, carved from the static array (complex128 work precision)
    const size_t fe = o->fine.cesize();
    const size_t R = (size_t)nrhs;
    const size_t s_loc = align256((size_t)o->fine.nloc * R * fe);
    const size_t s_rb = align256((size_t)rbuf_planes(o) * o->fine.m_max * R * fe);
    const size_t s_cv = o->nc ? align256((size_t)o->nc * R * sizeof(c128)) : 0;
    const size_t s_crb = o->nc ? align256((size_t)9 * o->coarse.m_max * R * sizeof(c128)) : 0;
    const size_t s_vec = o->nc ? align256((size_t)o->g->n * R * sizeof(c128)) : 0;
    const int npad = o->fine.padded ? tc_npad(nrhs) : 0;
    const size_t s_tcb = o->fine.padded ? align256((size_t)o->fine.nbox * npad * 2 * o->fine.ld * tc_elem(o)) : 0;
    const size_t s_lb = o->fine.padded ? s_loc : 0;
    const size_t need = s_loc + s_rb + s_cv + s_crb + 2 * s_vec + s_tcb + s_lb;
    if (need > HELM_NOALLOC_SCRATCH_BYTES)
        return set_error(ctx, HELM_EINVAL,
                         "oras_apply_noalloc: needs %zu bytes of scratch for this problem and nrhs = %d, more than "
                         "the fixed %u bytes; use oras_apply or fewer right-hand sides",
                         need, nrhs, HELM_NOALLOC_SCRATCH_BYTES);
    if (!g_noalloc_ptr[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_check(ctx, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                      "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[ctx->device] = p;
    }
    unsigned char* base = (unsigned char*)g_noalloc_ptr[ctx->device];
    // point the handle's working vectors into the static array for this call only
    void *s_loc_p = o->loc, *s_rbuf_p = o->rbuf, *s_qf_p = o->qf, *s_tf_p = o->tf, *s_tcb_p = o->tcb, *s_lb_p = o->lb;
    const int s_npad = o->tc_npad;
    if (o->fine.padded) {
        // the tensor-core operand's padding must read as zero
        unsigned char* t = base + s_loc + s_rb + s_cv + s_crb + 2 * s_vec;
        HELM_CUDA(ctx, cudaMemsetAsync(t, 0, s_tcb, ctx->stream));
        o->tcb = t;
        o->tc_npad = npad;
        o->lb = t + s_tcb;
    }
    c128 *s_cvec_p = o->cvec, *s_crbuf_p = o->crbuf;
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;
    o->loc = base;
    o->rbuf = base + s_loc;
    o->cvec = o->nc ? (c128*)(base + s_loc + s_rb) : nullptr;
    o->crbuf = o->nc ? (c128*)(base + s_loc + s_rb + s_cv) : nullptr;
    o->qf = o->nc ? (void*)(base + s_loc + s_rb + s_cv + s_crb) : nullptr;
    o->tf = o->nc ? (void*)(base + s_loc + s_rb + s_cv + s_crb + s_vec) : nullptr;
    helm_status rc = o->fine.prec == HELM_PREC_FP64 ? apply_t<double, double>(o, (const c128*)v, (c128*)out, nrhs)
                                                    : apply_t<double, float>(o, (const c128*)v, (c128*)out, nrhs);
    if (rc == HELM_OK) rc = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "oras_apply_noalloc");
    o->loc = s_loc_p;
    o->rbuf = s_rbuf_p;
    o->qf = s_qf_p;
    o->tf = s_tf_p;
    o->tcb = s_tcb_p;
    o->lb = s_lb_p;
    o->tc_npad = s_npad;
    o->cvec = s_cvec_p;
    o->crbuf = s_crbuf_p;
    ctx->prof.on = prof_on;
    if (rc) return rc;
    // a bounded device wait that gave up during this call is this call's failure (reading the flag
    // copies one int to host memory and allocates nothing)
    return oras_check_device_error(o);
}

size_t oras_estimate_bytes(const helm_grid_desc& g, const helm_oras_desc& d, int nrhs) {
    const int n[3] = {g.nx, g.ny, g.nz};
    const int p[3] = {std::max(1, d.px), std::max(1, d.py), std::max(1, d.pz)};
    const size_t fe = d.factor_prec == HELM_PREC_FP64 ? sizeof(c128) : sizeof(c64);   // as factorised
    const bool padded = d.factor_prec == HELM_PREC_TF32 || d.factor_prec == HELM_PREC_BF16;
    size_t m_max = 0, nloc = 0, planes = 0, fac = 0;
    std::vector<std::pair<size_t, size_t>> boxes;   // (m, bz)
    for (int tz = 0; tz < p[2]; ++tz)
        for (int ty = 0; ty < p[1]; ++ty)
            for (int tx = 0; tx < p[0]; ++tx) {
                const int t[3] = {tx, ty, tz};
                size_t dims[3];
                for (int a = 0; a < 3; ++a) {
                    const int c0 = (int)((long long)t[a] * n[a] / p[a]), c1 = (int)((long long)(t[a] + 1) * n[a] / p[a]);
                    const int lo = c0 > 0 ? std::max(0, c0 - d.overlap) : 0;
                    const int hi = c1 < n[a] ? std::min(n[a], c1 + d.overlap) : n[a];
                    dims[a] = (size_t)(hi - lo);
                }
                const size_t m = dims[0] * dims[1];
                boxes.push_back({m, dims[2]});
                m_max = std::max(m_max, m);
                nloc += m * dims[2];
                planes += dims[2];
            }
    const size_t ld = padded ? (m_max + 15) / 16 * 16 : 0;
    for (auto& b : boxes) fac += (padded ? (size_t)padded_pstride((int)ld) : b.first * b.first) * b.second;
    size_t bytes = fac * fe + nloc * 27 * fe;
    const size_t N = (size_t)g.nx * g.ny * g.nz;
    const size_t R = (size_t)std::max(1, nrhs);
    bytes += nloc * R * fe + std::max<size_t>(boxes.size(), 9) * m_max * R * fe;   // apply scratch
    if (padded) bytes += boxes.size() * (size_t)tc_npad(nrhs) * 2 * ld * sizeof(float) + nloc * R * fe;
    if (d.coarse_ratio > 0) {
        size_t nc = 1, cm = 1;
        for (int a = 0; a < 3; ++a) {
            const size_t ca = (size_t)((n[a] - 1 + d.coarse_ratio - 1) / d.coarse_ratio + 1);
            nc *= ca;
            if (a < 2) cm *= ca;
        }
        const size_t cz = nc / cm;
        bytes += 2 * N * 27 * sizeof(c128);                                  // probing vectors during set-up
        bytes += nc * R * sizeof(c128) + 2 * N * R * sizeof(c128);
        if (d.coarse_iters == 0) {
            bytes += (cm * cm * cz + nc * 27) * (sizeof(c128) + sizeof(c64));   // FP64 factors and the complex64 copy
            bytes += 9 * cm * R * sizeof(c128);
        } else {
            // E (FP64 and complex64), the coarse subdomain factors (FP64 and copy), their scratch, the inner basis
            size_t cfac = 0, cloc = 0, cmx = 0;
            const int r = d.coarse_ratio;
            for (int tz = 0; tz < p[2]; ++tz)
                for (int ty = 0; ty < p[1]; ++ty)
                    for (int tx = 0; tx < p[0]; ++tx) {
                        const int t[3] = {tx, ty, tz};
                        size_t dims[3];
                        for (int a = 0; a < 3; ++a) {
                            const int ca = (n[a] - 1 + r - 1) / r + 1;
                            auto cut = [&](int q) {
                                return q == 0 ? 0 : (q == p[a] ? ca : (int)(((long long)q * n[a] / p[a] + r - 1) / r));
                            };
                            const int c0 = cut(t[a]), c1 = cut(t[a] + 1);
                            const int lo = c0 > 0 ? std::max(0, c0 - d.coarse_overlap) : 0;
                            const int hi = c1 < ca ? std::min(ca, c1 + d.coarse_overlap) : ca;
                            dims[a] = (size_t)std::max(0, hi - lo);
                        }
                        const size_t m = dims[0] * dims[1];
                        cfac += m * m * dims[2];
                        cloc += m * dims[2];
                        cmx = std::max(cmx, m);
                    }
            bytes += nc * 27 * (sizeof(c128) + sizeof(c64)) + (cfac + cloc * 27) * (sizeof(c128) + sizeof(c64));
            bytes += (nc + cloc + boxes.size() * cmx) * R * sizeof(c128);
            bytes += ((size_t)d.coarse_iters + 3) * nc * R * sizeof(c128);
        }
    }
    return bytes + bytes / 16;
}

extern "C" helm_status oras_estimate_bytes_c(const helm_grid_desc* g, const helm_oras_desc* d, int nrhs, size_t* bytes) {
    if (!g || !d || !bytes || nrhs < 0 || g->nx < 2 || g->ny < 2 || g->nz < 2 || d->px < 1 || d->py < 1 || d->pz < 1)
        return HELM_EINVAL;
    *bytes = oras_estimate_bytes(*g, *d, nrhs);
    return HELM_OK;
}
