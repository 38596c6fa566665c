"""Closed-form point-source solutions used to check the discretisation (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

With the time convention ``exp(-i omega t)`` and ``(Delta + k^2) u = delta``
(Eq. eqh with a unit point source on the right-hand side), ``u = -G`` where
``G`` is the outgoing Green's function of ``-(Delta + k^2)``.

* Homogeneous medium: ``G = exp(i k r) / (4 pi r)``.
* Dirichlet top at depth 0: ``G(x, s) - G(x, s*)`` with ``s*`` the mirror
  image of the source in the plane ``z = 0``.
* Linear velocity gradient ``c(z) = c0 + alpha z`` (the paper's validation
  medium; it cites Kuvshinov 2006 for the solution but prints no formula).
  Written here from the substitution ``u = zeta^{-1/2} w`` with
  ``zeta = c(z)/alpha``, which maps ``Delta + omega^2/c^2`` to the Helmholtz
  operator of hyperbolic 3-space:
  ``G = exp(i mu d) / (4 pi sqrt(zeta zeta_s) sinh d)``,
  ``cosh d = 1 + |x - x_s|^2 / (2 zeta zeta_s)``,
  ``mu = sqrt(omega^2/alpha^2 - 1/4)``.
  Pinned in the tests by a fine-step finite-difference PDE residual, by
  ``4 pi r G -> 1`` at the source and by the ``alpha -> 0`` limit.
"""
from __future__ import annotations

import numpy as np


def green_homogeneous(x, y, z, src, k):
    r = np.sqrt((x - src[0]) ** 2 + (y - src[1]) ** 2 + (z - src[2]) ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):      # r = 0 at the source node itself
        return np.exp(1j * k * r) / (4.0 * np.pi * r)


def green_homogeneous_dirichlet_top(x, y, z, src, k):
    img = (src[0], src[1], -src[2])
    return green_homogeneous(x, y, z, src, k) - green_homogeneous(x, y, z, img, k)


def green_linear_gradient(x, y, z, src, omega, c0, alpha):
    zeta = (c0 + alpha * z) / alpha
    zeta_s = (c0 + alpha * src[2]) / alpha
    r2 = (x - src[0]) ** 2 + (y - src[1]) ** 2 + (z - src[2]) ** 2
    # cosh d = 1 + r^2/(2 zeta zeta_s), i.e. sinh(d/2) = r / (2 sqrt(zeta zeta_s)) (no cancellation)
    d = 2.0 * np.arcsinh(np.sqrt(r2) / (2.0 * np.sqrt(zeta * zeta_s)))
    mu = np.sqrt(omega ** 2 / alpha ** 2 - 0.25 + 0j)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.exp(1j * mu * d) / (4.0 * np.pi * np.sqrt(zeta * zeta_s) * np.sinh(d))


def node_coordinates(nx, ny, nz, h):
    """Physical coordinates of the unknown nodes: ``x = i h``, ``y = j h``, ``z = (k+1) h``."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i * h, j * h, (k + 1) * h


def relative_l2_misfit(u_num, u_ref, mask):
    """``||u_num - u_ref|| / ||u_ref||`` over the nodes where ``mask`` is true."""
    d = (u_num - u_ref)[mask]
    return float(np.linalg.norm(d) / np.linalg.norm(u_ref[mask]))


def comparison_mask(nx, ny, nz, npml, top_pml, src_idx, min_dist):
    """Non-PML nodes at least ``min_dist`` nodes away from the source."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = (i >= npml) & (i < nx - npml) & (j >= npml) & (j < ny - npml) & (k < nz - npml)
    if top_pml:
        m &= k >= npml
    si, sj, sk = src_idx
    dist = np.sqrt((i - si) ** 2 + (j - sj) ** 2 + (k - sk) ** 2)
    return m & (dist >= min_dist)
