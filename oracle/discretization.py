"""Grid, absorbing layers and the 27-point mixed-grid Helmholtz operator (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

What the paper fixes (section "Tetrahedral finite elements versus 27-point
finite-differences", Eq. eqh and Eq. eq1):

* ``(Delta + k^2(x)) u = b`` with ``k = omega / c(x)``; ``c`` is complex in
  viscous media.
* Absorbing conditions on the four vertical faces and on the bottom, a
  homogeneous Dirichlet condition on the top face.
* A 27-point stencil mixing second-order Laplacians written in rotated
  coordinate systems (Cartesian, three one-axis rotations, the body-diagonal
  system) with a consistent mass term spread over the 27 points; the weights
  come from a least-squares fit of the numerical dispersion.

Readings taken where the paper is silent:

* Time convention ``exp(-i omega t)``: outgoing waves are ``exp(+i k r)`` and
  attenuation ``c (1 - i/(2Q))`` gives ``Im k > 0``.
* Nodes ``(i, j, k)`` at ``x = i h``, ``y = j h``, depth ``z = (k + 1) h``; the
  Dirichlet plane is the ghost ``k = -1``; every ghost beyond the outer faces
  is zero.
* Absorbing layers are a separable stretched-coordinate PML of ``npml`` nodes:
  in the Laplacian each 3-point second difference becomes
  ``(1/xi_i) [ (u_{i+1}-u_i)/xi_{i+1/2} - (u_i-u_{i-1})/xi_{i-1/2} ]`` with
  ``xi = 1 + i gamma(d)/omega``, ``gamma = gamma0 (d/L)^2``, ``L = npml h``,
  ``gamma0 = 3 c_ref / (2 L) ln(1/R)``, ``c_ref = max Re c``.  The mass term is
  not stretched.
* The mass term acts on ``k^2 u`` sampled at each neighbour.
* Written with 1-D second differences ``D_a`` (stretched) and ``P_a`` (plain),
  the mixed-grid stencil is exactly
  ``A u = h^-2 [sum D_a + a2 sum_{a<b} D_a D_b + a3 D_x D_y D_z] u
          + [m0 + m1 sum P_a + m2 sum P_a P_b + m3 P_x P_y P_z] (k^2 u)``
  with ``a2 = w2/6 + w3/2``, ``a3 = w3/4``, ``m0 = wm1+6wm2+12wm3+8wm4``,
  ``m1 = wm2+4wm3+4wm4``, ``m2 = wm3+2wm4``, ``m3 = wm4``.
  ``tests/test_oracle_operator.py`` pins this identity against the stencil
  written point by point in its rotated-system form.

Pins: 7-point special case vs a textbook Kronecker-sum Laplacian; the
plane-wave symbol on interior nodes; rotated-system form vs product form;
assembled matrix vs matrix-free apply.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# The 7-point stencil: w1 = 1 (Cartesian Laplacian only), wm1 = 1 (lumped mass).
WEIGHTS_7PT = (1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@dataclass
class Problem:
    """One Helmholtz problem: grid, medium, frequency and boundary setup."""

    nx: int
    ny: int
    nz: int
    h: float
    freq: float
    c: np.ndarray                     # complex128 [nz, ny, nx] wave speed
    npml: int = 8
    top_pml: bool = False             # False: Dirichlet top (paper); True: PML top
    pml_R: float = 1e-3
    weights: tuple = WEIGHTS_7PT      # (w1, w2, w3, wm1, wm2, wm3, wm4)
    row_weights: np.ndarray = None    # optional [nz, ny, nx, 7]: weights of each row (adaptive stencil)
    _cache: dict = field(default_factory=dict, repr=False, compare=False)

    @property
    def omega(self) -> float:
        return 2.0 * np.pi * self.freq

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def k2(self) -> np.ndarray:
        """``k^2 = (omega / c)^2`` at every node, complex128 ``[nz, ny, nx]``."""
        c = np.asarray(self.c, dtype=np.complex128)
        return (self.omega / c) ** 2


def stencil_coefficients(weights):
    """Map the mixed-grid weights to the product-form coefficients.

    Returns ``(a2, a3, m0, m1, m2, m3)`` (identities stated in the module
    docstring).
    """
    w1, w2, w3, wm1, wm2, wm3, wm4 = [float(v) for v in weights]
    a2 = w2 / 6.0 + w3 / 2.0
    a3 = w3 / 4.0
    m0 = wm1 + 6.0 * wm2 + 12.0 * wm3 + 8.0 * wm4
    m1 = wm2 + 4.0 * wm3 + 4.0 * wm4
    m2 = wm3 + 2.0 * wm4
    m3 = wm4
    return a2, a3, m0, m1, m2, m3


def row_coefficients(prob: Problem):
    """``(a2, a3, m0, m1, m2, m3)`` of every row: scalars for constant weights, ``[nz, ny, nx]`` arrays
    when ``prob.row_weights`` gives each row its own weights (the adaptive stencil, whose row ``p`` is
    the constant-weight row built with the weights of ``p``)."""
    if prob.row_weights is None:
        return stencil_coefficients(prob.weights)
    w = np.asarray(prob.row_weights, dtype=np.float64)
    w1, w2, w3, wm1, wm2, wm3, wm4 = (w[..., q] for q in range(7))
    return (w2 / 6.0 + w3 / 2.0, w3 / 4.0, wm1 + 6.0 * wm2 + 12.0 * wm3 + 8.0 * wm4, wm2 + 4.0 * wm3 + 4.0 * wm4,
            wm3 + 2.0 * wm4, wm4)


def pml_xi(n: int, h: float, npml: int, low: bool, high: bool, omega: float, c_ref: float, R: float):
    """Stretching factors ``xi`` at nodes ``s = 0..n-1`` and half nodes.

    Returns ``(xi_node[n], xi_half[n+1])`` where ``xi_half[i]`` sits at
    ``s = i - 1/2``.  Depth into a layer: ``d = (npml - s) h`` on the low side,
    ``d = (s - (n - 1 - npml)) h`` on the high side, zero elsewhere; the last
    unstretched node on each side has ``d = 0``.
    """
    L = npml * h
    gamma0 = 0.0 if npml == 0 else 1.5 * c_ref / L * np.log(1.0 / R)

    def xi(s):
        s = np.asarray(s, dtype=np.float64)
        d = np.zeros_like(s)
        if low and npml > 0:
            d = np.where(s < npml, (npml - s) * h, d)
        if high and npml > 0:
            d = np.where(s > n - 1 - npml, (s - (n - 1 - npml)) * h, d)
        gamma = gamma0 * (d / L) ** 2 if npml > 0 else np.zeros_like(s)
        return 1.0 + 1j * gamma / omega

    nodes = np.arange(n, dtype=np.float64)
    halves = np.arange(n + 1, dtype=np.float64) - 0.5
    return xi(nodes), xi(halves)


def second_difference_1d(n: int, xi_node=None, xi_half=None):
    """Coefficients ``(cm, c0, cp)`` of the 1-D second difference at each node.

    Without ``xi`` this is the plain ``(1, -2, 1)``; with it, the stretched
    form ``cm = 1/(xi_i xi_{i-1/2})``, ``cp = 1/(xi_i xi_{i+1/2})``,
    ``c0 = -(cm + cp)``.  The ghost neighbours beyond the ends are zero, so the
    first ``cm`` and last ``cp`` multiply nothing.
    """
    if xi_node is None:
        cm = np.ones(n, dtype=np.complex128)
        cp = np.ones(n, dtype=np.complex128)
    else:
        cm = 1.0 / (xi_node * xi_half[:-1])
        cp = 1.0 / (xi_node * xi_half[1:])
    return cm, -(cm + cp), cp


def axis_tables(prob: Problem):
    """Stretched 1-D coefficient tables ``(cm, c0, cp)`` for the x, y, z axes."""
    key = "axis_tables"
    if key in prob._cache:
        return prob._cache[key]
    c_ref = float(np.max(np.real(prob.c)))
    tx = second_difference_1d(prob.nx, *pml_xi(prob.nx, prob.h, prob.npml, True, True, prob.omega, c_ref, prob.pml_R))
    ty = second_difference_1d(prob.ny, *pml_xi(prob.ny, prob.h, prob.npml, True, True, prob.omega, c_ref, prob.pml_R))
    tz = second_difference_1d(prob.nz, *pml_xi(prob.nz, prob.h, prob.npml, prob.top_pml, True, prob.omega, c_ref,
                                                prob.pml_R))
    prob._cache[key] = (tx, ty, tz)
    return tx, ty, tz


def _d2_along(u: np.ndarray, axis: int, table) -> np.ndarray:
    """Apply a 1-D three-point operator with per-node coefficients along one axis.

    ``u`` has shape ``[nz, ny, nx, ...]``; array axis 0 is z, 1 is y, 2 is x.
    Zero ghosts beyond both ends.
    """
    cm, c0, cp = table
    n = u.shape[axis]
    shape = [1] * u.ndim
    shape[axis] = n
    cm = cm.reshape(shape)
    c0 = c0.reshape(shape)
    cp = cp.reshape(shape)
    out = c0 * u
    lo = [slice(None)] * u.ndim
    hi = [slice(None)] * u.ndim
    # out[i] += cm[i] * u[i-1]  for i >= 1
    lo[axis] = slice(1, None)
    hi[axis] = slice(0, n - 1)
    out[tuple(lo)] += cm[tuple(lo)] * u[tuple(hi)]
    # out[i] += cp[i] * u[i+1]  for i <= n-2
    out[tuple(hi)] += cp[tuple(hi)] * u[tuple(lo)]
    return out


def apply_A(prob: Problem, u: np.ndarray) -> np.ndarray:
    """Matrix-free ``A u`` (Eq. eq1) in FP64.

    ``u`` is ``[nz, ny, nx]`` or ``[nz, ny, nx, nrhs]`` complex.  The Laplacian
    and mass parts are applied as sums of products of 1-D operators
    (module docstring).
    """
    u = np.asarray(u, dtype=np.complex128)
    extra = u.ndim - 3
    a2, a3, m0, m1, m2, m3 = (np.reshape(q, np.shape(q) + (1,) * extra) for q in row_coefficients(prob))
    tx, ty, tz = axis_tables(prob)
    # axis 0 = z, axis 1 = y, axis 2 = x
    Dx = lambda v: _d2_along(v, 2, tx)
    Dy = lambda v: _d2_along(v, 1, ty)
    Dz = lambda v: _d2_along(v, 0, tz)
    ux, uy, uz = Dx(u), Dy(u), Dz(u)
    uxy = Dy(ux)
    lap = ux + uy + uz + a2 * (uxy + Dz(ux) + Dz(uy)) + a3 * Dz(uxy)

    plain = lambda n: second_difference_1d(n)
    px, py, pz = plain(prob.nx), plain(prob.ny), plain(prob.nz)
    k2 = prob.k2().reshape(prob.shape + (1,) * extra)
    w = k2 * u
    wx = _d2_along(w, 2, px)
    wy = _d2_along(w, 1, py)
    wz = _d2_along(w, 0, pz)
    wxy = _d2_along(wx, 1, py)
    mass = (m0 * w + m1 * (wx + wy + wz)
            + m2 * (wxy + _d2_along(wx, 0, pz) + _d2_along(wy, 0, pz))
            + m3 * _d2_along(wxy, 0, pz))
    return lap / prob.h ** 2 + mass


def neighbour_coefficients(prob: Problem) -> np.ndarray:
    """The 27 stencil coefficients of every row, complex128 ``[3, 3, 3, nz, ny, nx]``.

    ``coef[dz+1, dy+1, dx+1, k, j, i]`` multiplies ``u`` at ``(i+dx, j+dy, k+dz)``
    in row ``(i, j, k)``; it includes ``k^2`` of that neighbour in the mass
    part.  Entries that point at a ghost are set to zero.  Built from the same
    product form as :func:`apply_A` but one matrix entry at a time, as the
    tensor product of the 1-D coefficient tables.
    """
    a2, a3, m0, m1, m2, m3 = row_coefficients(prob)
    tx, ty, tz = axis_tables(prob)
    nz, ny, nx = prob.shape
    k2 = prob.k2()
    # 1-D coefficient of offset d at node index: table[d+1][index]
    X = np.stack([tx[0], tx[1], tx[2]])          # [3, nx]
    Y = np.stack([ty[0], ty[1], ty[2]])          # [3, ny]
    Z = np.stack([tz[0], tz[1], tz[2]])          # [3, nz]
    P = np.array([1.0, -2.0, 1.0])
    E = np.array([0.0, 1.0, 0.0])                # identity (offset 0 only)
    coef = np.zeros((3, 3, 3, nz, ny, nx), dtype=np.complex128)
    kpad = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.complex128)
    kpad[1:-1, 1:-1, 1:-1] = k2
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                x = X[dx][None, None, :]
                y = Y[dy][None, :, None]
                z = Z[dz][:, None, None]
                ex, ey, ez = E[dx], E[dy], E[dz]
                lap = (x * ey * ez + ex * y * ez + ex * ey * z
                       + a2 * (x * y * ez + x * ey * z + ex * y * z)
                       + a3 * x * y * z) / prob.h ** 2
                px, py, pz = P[dx], P[dy], P[dz]
                mass = (m0 * ex * ey * ez + m1 * (px * ey * ez + ex * py * ez + ex * ey * pz)
                        + m2 * (px * py * ez + px * ey * pz + ex * py * pz) + m3 * px * py * pz)
                kn = kpad[dz:dz + nz, dy:dy + ny, dx:dx + nx]
                coef[dz, dy, dx] = lap + mass * kn
    # zero the entries whose neighbour is a ghost
    coef[:, :, 0, :, :, 0] = 0.0
    coef[:, :, 2, :, :, nx - 1] = 0.0
    coef[:, 0, :, :, 0, :] = 0.0
    coef[:, 2, :, :, ny - 1, :] = 0.0
    coef[0, :, :, 0, :, :] = 0.0
    coef[2, :, :, nz - 1, :, :] = 0.0
    return coef


def assemble_A(prob: Problem) -> sp.csr_matrix:
    """Assembled sparse ``A`` (CSR, complex128), row/column index ``(k*ny + j)*nx + i``."""
    coef = neighbour_coefficients(prob)
    nz, ny, nx = prob.shape
    idx = np.arange(prob.n).reshape(prob.shape)
    rows, cols, vals = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                c = coef[dz + 1, dy + 1, dx + 1]
                ks = slice(max(0, -dz), nz - max(0, dz))
                js = slice(max(0, -dy), ny - max(0, dy))
                is_ = slice(max(0, -dx), nx - max(0, dx))
                r = idx[ks, js, is_]
                q = idx[ks.start + dz:ks.stop + dz, js.start + dy:js.stop + dy, is_.start + dx:is_.stop + dx]
                rows.append(r.ravel())
                cols.append(q.ravel())
                vals.append(c[ks, js, is_].ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(prob.n, prob.n))


def symbol(prob: Problem, kappa, k2: complex) -> complex:
    """Closed-form plane-wave symbol on interior unstretched nodes at constant ``k^2``.

    With ``s_a = 2 (cos(kappa_a h) - 1)``:
    ``A_hat = h^-2 [sum s + a2 sum s_a s_b + a3 s_x s_y s_z]
              + k^2 [m0 + m1 sum s + m2 sum s_a s_b + m3 s_x s_y s_z]``.
    """
    a2, a3, m0, m1, m2, m3 = stencil_coefficients(prob.weights)
    s = [2.0 * (np.cos(kk * prob.h) - 1.0) for kk in kappa]
    s1 = s[0] + s[1] + s[2]
    s2 = s[0] * s[1] + s[0] * s[2] + s[1] * s[2]
    s3 = s[0] * s[1] * s[2]
    return (s1 + a2 * s2 + a3 * s3) / prob.h ** 2 + k2 * (m0 + m1 * s1 + m2 * s2 + m3 * s3)
