"""Least-squares fit of the 27-point mixed-grid stencil weights (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

The paper fits the stiffness and consistent-mass weights by least squares against
the stencil's phase-velocity and direction errors (section on finite elements versus
the 27-point stencil),
but prints no values.  Reading taken: minimise the normalised phase-velocity
error ``1 - sqrt(-L_hat(kappa)/M_hat(kappa)) / |kappa|`` of plane waves over
``G`` = 4..30 grid points per wavelength and propagation directions in one
octant, with ``w1 = 1 - w2 - w3`` and ``wm1 = 1 - 6 wm2 - 12 wm3 - 8 wm4`` so
both weight sets sum to one, and every weight kept non-negative (each set is
a convex combination of stencils; the unconstrained minimum has negative
weights and no smaller error).  ``L_hat``/``M_hat`` are the Laplacian and mass
parts of the symbol in :func:`oracle.discretization.symbol`.

Parity: the fitted values themselves are unpinned (the paper prints none);
what is pinned is that the fit reduces the maximum phase-velocity error far
below the 7-point stencil's over the fitted range.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import least_squares

from .discretization import stencil_coefficients


def _sample_directions(n_theta=7, n_phi=7):
    th = np.linspace(0.0, np.pi / 2, n_theta)
    ph = np.linspace(0.0, np.pi / 2, n_phi)
    dirs = []
    for t in th:
        for p in ph:
            dirs.append((np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)))
    return np.array(dirs)


def phase_velocity_ratio(weights, G, direction) -> float:
    """``v_phase / c`` of a plane wave with ``G`` points per wavelength (h = 1)."""
    a2, a3, m0, m1, m2, m3 = stencil_coefficients(weights)
    kap = 2.0 * np.pi / G
    s = [2.0 * (np.cos(kap * d) - 1.0) for d in direction]
    s1 = s[0] + s[1] + s[2]
    s2 = s[0] * s[1] + s[0] * s[2] + s[1] * s[2]
    s3 = s[0] * s[1] * s[2]
    L = s1 + a2 * s2 + a3 * s3
    M = m0 + m1 * s1 + m2 * s2 + m3 * s3
    return np.sqrt(max(-L / M, 0.0)) / kap


def full_weights(p):
    w2, w3, wm2, wm3, wm4 = p
    return (1.0 - w2 - w3, w2, w3, 1.0 - 6.0 * wm2 - 12.0 * wm3 - 8.0 * wm4, wm2, wm3, wm4)


def dispersion_residuals(weights, G_values=None, directions=None):
    if G_values is None:
        G_values = 1.0 / np.linspace(1.0 / 30.0, 1.0 / 4.0, 24)
    if directions is None:
        directions = _sample_directions()
    return np.array([1.0 - phase_velocity_ratio(weights, G, d) for G in G_values for d in directions])


def fit_weights(G_min=4.0, G_max=30.0):
    """Fit ``(w1, w2, w3, wm1, wm2, wm3, wm4)``; returns a 7-tuple of floats."""
    G_values = 1.0 / np.linspace(1.0 / G_max, 1.0 / G_min, 24)
    directions = _sample_directions()
    p0 = np.array([0.5, 0.1, 0.08, 0.005, 0.001])
    lower = [0.0, 0.0, 0.0, 0.0, 0.0]
    upper = [1.0, 1.0, 1.0 / 6.0, 1.0 / 12.0, 1.0 / 8.0]
    res = least_squares(lambda p: dispersion_residuals(full_weights(p), G_values, directions), p0,
                        bounds=(lower, upper), xtol=1e-14, ftol=1e-14, gtol=1e-14, max_nfev=4000)
    return tuple(float(v) for v in full_weights(res.x))


# ---------------------------------------------------------------------------
# Adaptive weights (weights matched to the local wave speed, row by row)
# ---------------------------------------------------------------------------
#
# The paper uses coefficients matched to the local wave speed in each row of A
# (it cites Turkel et al. 2013) but gives no construction.  Reading taken: the
# points-per-wavelength range of the model, G = Re c / (f h) from its minimum to
# its maximum, is cut into ``nbins`` geometric bins; each bin gets the weights of
# the least-squares fit above restricted to the bin's G interval, and each row
# uses the weights of the bin that holds its own G.

def adaptive_bin_edges(G_lo: float, G_hi: float, nbins: int) -> np.ndarray:
    """``nbins + 1`` geometric edges from ``G_lo`` to ``G_hi`` (edge b = G_lo * ratio**b)."""
    if nbins < 1:
        raise ValueError("nbins must be >= 1")
    ratio = (G_hi / G_lo) ** (1.0 / nbins)
    return np.array([G_lo * ratio ** b for b in range(nbins + 1)])


def row_weight_bins(c, freq: float, h: float, edges) -> np.ndarray:
    """Bin of every node: the number of interior edges at or below its ``G = Re c / (f h)``."""
    G = np.real(np.asarray(c, dtype=np.complex128)) / (freq * h)
    b = np.zeros(G.shape, dtype=np.int64)
    for e in np.asarray(edges)[1:-1]:
        b += (G >= e)
    return b


def adaptive_row_weights(c, freq: float, h: float, nbins: int, fit=fit_weights):
    """``(table[nbins, 7], bins[nz, ny, nx], row_weights[nz, ny, nx, 7])`` for a model; ``fit(G_min, G_max)``
    supplies each bin's weights (this module's fit by default; a test may pass another fitter's values)."""
    G = np.real(np.asarray(c, dtype=np.complex128)) / (freq * h)
    edges = adaptive_bin_edges(float(G.min()), float(G.max()), nbins)
    table = np.array([fit(edges[b], edges[b + 1]) for b in range(nbins)])
    bins = row_weight_bins(c, freq, h, edges)
    return table, bins, table[bins]
