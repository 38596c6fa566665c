"""Seeded synthetic inputs: velocity models, source positions, right-hand sides.

This module holds input generation only (no part of the solver's
arithmetic); both the GPU library's tests/bench and the CPU oracle's tests
draw their inputs from it.  Node depth convention of the grid: node
``(i, j, k)`` sits at ``x = i h``, ``y = j h``, depth ``z = (k + 1) h`` (the
Dirichlet surface is the ghost plane at depth 0).

Workloads (all seeded; base seed 2103, workload ``c`` uses ``2103*100 + c``):

* linear gradient ``c(z) = c0 + alpha z`` -- the paper's validation medium;
* the same with attenuation ``c (1 - i/(2Q))``;
* a thrust-fold model standing in for SEG/EAGE Overthrust (dataset absent):
  folded layers 2000..6000 m/s with two dipping faults of +-15 % contrast;
* small layered models for the request-stream workload.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2103


def workload_seed(c: int) -> int:
    return BASE_SEED * 100 + c


def node_depths(nz: int, h: float) -> np.ndarray:
    return (np.arange(nz) + 1) * h


def linear_gradient(nx, ny, nz, h, c0=1500.0, alpha=0.6, Q=None) -> np.ndarray:
    """complex128 ``[nz, ny, nx]`` velocity ``c0 + alpha z`` (times ``1 - i/(2Q)`` if Q)."""
    z = node_depths(nz, h)
    c = np.broadcast_to((c0 + alpha * z)[:, None, None], (nz, ny, nx)).astype(np.complex128)
    if Q is not None:
        c = c * (1.0 - 0.5j / Q)
    return np.ascontiguousarray(c)


def homogeneous(nx, ny, nz, c0=1500.0) -> np.ndarray:
    return np.full((nz, ny, nx), c0, dtype=np.complex128)


def layered(nx, ny, nz, h, seed, n_layers=None, vmin=1500.0, vmax=4500.0) -> np.ndarray:
    """Flat layers with seeded interface depths and velocities increasing with depth."""
    rng = np.random.default_rng(seed)
    if n_layers is None:
        n_layers = int(rng.integers(3, 7))
    zmax = nz * h
    depths = np.sort(rng.uniform(0.1 * zmax, 0.9 * zmax, n_layers - 1))
    vel = np.sort(rng.uniform(vmin, vmax, n_layers))
    z = node_depths(nz, h)
    lay = np.searchsorted(depths, z)
    c = vel[lay]
    return np.ascontiguousarray(np.broadcast_to(c[:, None, None], (nz, ny, nx)).astype(np.complex128))


def thrust_fold(nx, ny, nz, h, seed) -> np.ndarray:
    """Folded, faulted layered model (8 layers, 2000..6000 m/s, two dipping faults)."""
    rng = np.random.default_rng(seed)
    n_layers = 8
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    z = node_depths(nz, h)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    tops = np.linspace(150.0, 2300.0, n_layers - 1)
    vel = np.linspace(2000.0, 6000.0, n_layers)
    amp = rng.uniform(50.0, 200.0)
    lx, ly = rng.uniform(1500.0, 4000.0, 2)
    phx, phy = rng.uniform(0.0, 2 * np.pi, 2)
    fold = amp * np.sin(2 * np.pi * X / lx + phx) * np.cos(2 * np.pi * Y / ly + phy)
    Zf = Z - fold
    lay = np.zeros(Z.shape, dtype=np.int64)
    for t in tops:
        lay += (Zf > t)
    c = vel[lay]
    for scale in (1.15, 0.85):
        strike = rng.uniform(0.0, np.pi)
        dip = np.deg2rad(rng.uniform(30.0, 60.0))
        x0 = rng.uniform(0.3, 0.7) * nx * h
        y0 = rng.uniform(0.3, 0.7) * ny * h
        nrm = np.array([np.sin(dip) * np.cos(strike), np.sin(dip) * np.sin(strike), np.cos(dip)])
        side = nrm[0] * (X - x0) + nrm[1] * (Y - y0) + nrm[2] * (Z - 0.5 * nz * h)
        c = np.where(side > 0, c * scale, c)
    c = np.clip(c, 1700.0, 6900.0)
    return np.ascontiguousarray(c.astype(np.complex128))


def source_plane_positions(nx, ny, npml, k_index, count, seed):
    """``count`` distinct seeded source nodes ``(i, j, k)`` on plane ``k_index``, inside the non-PML area."""
    rng = np.random.default_rng(seed)
    lo_i, hi_i = npml, nx - npml
    lo_j, hi_j = npml, ny - npml
    flat = rng.choice((hi_i - lo_i) * (hi_j - lo_j), size=count, replace=False)
    return [(int(lo_i + f % (hi_i - lo_i)), int(lo_j + f // (hi_i - lo_i)), int(k_index)) for f in flat]


def source_array_positions(nx, ny, npml, k_index, per_side):
    """A regular ``per_side x per_side`` node array evenly spread over the non-PML area."""
    ii = np.linspace(npml, nx - npml - 1, per_side + 2)[1:-1].round().astype(int)
    jj = np.linspace(npml, ny - npml - 1, per_side + 2)[1:-1].round().astype(int)
    return [(int(i), int(j), int(k_index)) for j in jj for i in ii]


def point_sources(nx, ny, nz, h, positions) -> np.ndarray:
    """complex128 ``[nz, ny, nx, nrhs]``: column r is a unit point source ``1/h^3`` at ``positions[r]``."""
    b = np.zeros((nz, ny, nx, len(positions)), dtype=np.complex128)
    for r, (i, j, k) in enumerate(positions):
        b[k, j, i, r] = 1.0 / h ** 3
    return b


def random_complex(shape, seed) -> np.ndarray:
    """Seeded standard complex normal array (complex128)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex128)


def random_weights(seed):
    """Random positive stencil weights with both sets summing to one (for operator parity)."""
    rng = np.random.default_rng(seed)
    w = rng.dirichlet([1.0, 1.0, 1.0])
    wm = rng.dirichlet([1.0, 1.0, 1.0, 1.0]) / np.array([1.0, 6.0, 12.0, 8.0])
    wm = wm / (wm[0] + 6 * wm[1] + 12 * wm[2] + 8 * wm[3])
    return (float(w[0]), float(w[1]), float(w[2]), float(wm[0]), float(wm[1]), float(wm[2]), float(wm[3]))
