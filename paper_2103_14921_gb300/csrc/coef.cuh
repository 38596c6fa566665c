// The 27 coefficients of one row of the global operator A (Eq. eq1) in the
// product form of the mixed-grid stencil (see stencil.cu for the identity).
// Used by the setup kernels that assemble local operators and the coarse
// operator; the hot stencil kernel forms the same coefficients inline.
#pragma once
#include "internal.h"

// coef[(dz+1)*9 + (dy+1)*3 + (dx+1)] multiplies u at (i+dx, j+dy, k+dz); entries
// whose neighbour is a ghost (outside the grid) are zero.
__device__ __forceinline__ void global_row_coef27(const c128* __restrict__ tab, const c128* __restrict__ k2, int nx,
                                                  int ny, int nz, const StencilW& w, int i, int j, int k,
                                                  c128* coef) {
    const c128* tx = tab + 3 * i;
    const c128* ty = tab + 3 * (nx + j);
    const c128* tz = tab + 3 * (nx + ny + k);
    const c128 zero = mk<double>(0, 0);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int ii = i + dx, jj = j + dy, kk = k + dz;
                c128 c = zero;
                if (ii >= 0 && ii < nx && jj >= 0 && jj < ny && kk >= 0 && kk < nz) {
                    const c128 X = tx[dx + 1], Y = ty[dy + 1], Z = tz[dz + 1];
                    const double ex = dx == 0, ey = dy == 0, ez = dz == 0;
                    const c128 XY = X * Y, XZ = X * Z, YZ = Y * Z, XYZ = XY * Z;
                    c128 lap = (ey * ez) * X + (ex * ez) * Y + (ex * ey) * Z;
                    lap = lap + w.a2 * (ez * XY + ey * XZ + ex * YZ) + w.a3 * XYZ;
                    const double Px = dx == 0 ? -2.0 : 1.0, Py = dy == 0 ? -2.0 : 1.0, Pz = dz == 0 ? -2.0 : 1.0;
                    const double mass = w.m0 * ex * ey * ez + w.m1 * (Px * ey * ez + ex * Py * ez + ex * ey * Pz) +
                                        w.m2 * (Px * Py * ez + Px * ey * Pz + ex * Py * Pz) + w.m3 * Px * Py * Pz;
                    const c128 kq = k2[((long long)kk * ny + jj) * nx + ii];
                    c = mk<double>(lap.x * w.inv_h2 + mass * kq.x, lap.y * w.inv_h2 + mass * kq.y);
                }
                coef[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = c;
            }
}
