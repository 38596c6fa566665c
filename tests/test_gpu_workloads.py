"""Workload-scale GPU checks through the C ABI.

* The timed workload exactly as bench.py runs it (112^3 linear gradient, 5 Hz, 16 sources on the plane
  z = 100 m, two-level ORAS 4x4x4 overlap 2, coarse ratio 4, TF32 factors, FGMRES(30), tol 1e-6):
  the oracle's FP64 matrix-free A gives the relative residual of sampled columns (<= tol); two columns
  are compared with an oracle reference solution x_ref = x + e, where the oracle solves A e = b - A x
  with its own FP64 two-level ORAS-FGMRES (splu local solves) until its residual drops by 1e-3, so
  x_ref has an oracle residual <= 1e-3 x tol and ||x - x_ref|| is the error of x to within 1e-3 of
  itself; ||x - x_ref|| / ||x_ref|| <= 10 x tol.  The same two columns solved by the plain FP64 GPU
  path also agree with the mixed solution within 10 x tol.
* Attenuating medium c (1 - i/(2Q)), Q = 100, at three frequencies (the multi-frequency workload,
  reduced to 160 x 160 x 80 with 16 sources per frequency): every column converges and its oracle
  residual is <= tol.
* The thrust-fold model (folded layers and two faults, the Overthrust stand-in) on 128 x 128 x 64 with
  a regular 4 x 4 node array at z = 50 m and BF16 factors: converged, oracle residual <= tol.
"""
import os

import numpy as np
import pytest

from oracle.discretization import Problem, apply_A
from oracle.krylov import gmres
from oracle.schwarz import ORAS
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _oracle_residuals(prob, x, b, cols):
    out = []
    for r in cols:
        out.append(np.linalg.norm(apply_A(prob, x[..., r]) - b[..., r]) / np.linalg.norm(b[..., r]))
    return out


def test_timed_workload_full_size(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    n, h, f, tol = 112, 25.0, 5.0, 1e-6
    c = synth.linear_gradient(n, n, n, h, 1500.0, 0.6)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, n, n, n, h, f, c, npml=8, weights=w)
    pos = synth.source_plane_positions(n, n, 8, 3, 16, synth.workload_seed(2))
    b = synth.point_sources(n, n, n, h, pos)
    bt = torch.from_numpy(b).cuda()
    o = helm.Oras(grid, (4, 4, 4), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
    x, stats = o.solve(bt, tol=tol, restart=30, flexible=True, basis_prec=helm.PREC_FP32)
    assert all(s["converged"] for s in stats)
    xm = x.cpu().numpy()
    del o
    prob = Problem(n, n, n, h, f, c, npml=8, weights=w)
    for res in _oracle_residuals(prob, xm, b, [0, 5, 10, 15]):
        assert res <= tol
    # oracle reference solutions of two columns by defect correction (the oracle's own method, FP64)
    # (the 64 local factorisations and solves run in a pool of worker processes: the same splu arithmetic)
    M = ORAS(prob, (4, 4, 4), 2, coarse_ratio=4, local="splu", workers=min(16, os.cpu_count() or 1))
    try:
        aA = lambda u: apply_A(prob, u.reshape(n, n, n)).ravel()
        for r in (0, 15):
            xr = xm[..., r].ravel()
            res = b[..., r].ravel() - aA(xr)
            e, info = gmres(aA, res, M.apply, tol=1e-3, restart=30, maxit=200, flexible=True)
            assert info["converged"]
            xref = xr + e
            assert np.linalg.norm(b[..., r].ravel() - aA(xref)) <= 1e-3 * tol * np.linalg.norm(b[..., r])
            assert np.linalg.norm(xr - xref) <= 10 * tol * np.linalg.norm(xref), r
    finally:
        M.close()
    del M
    o64 = helm.Oras(grid, (4, 4, 4), 2, coarse_ratio=4, factor_prec=helm.PREC_FP64)
    x64, s64 = o64.solve(bt[..., [0, 15]].contiguous(), tol=tol, restart=30, basis_prec=helm.PREC_FP64)
    x64 = x64.cpu().numpy()
    for k, r in enumerate([0, 15]):
        assert s64[k]["converged"]
        assert np.linalg.norm(xm[..., r] - x64[..., k]) <= 10 * tol * np.linalg.norm(x64[..., k])


def test_attenuating_three_frequencies(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz, h, tol = 160, 160, 80, 25.0, 1e-6
    c = synth.linear_gradient(nx, ny, nz, h, 1500.0, 0.6, Q=100.0)
    w = helm.fit_weights()
    pos = synth.source_plane_positions(nx, ny, 8, 3, 16, synth.workload_seed(4))
    b = synth.point_sources(nx, ny, nz, h, pos)
    bt = torch.from_numpy(b).cuda()
    for f in (3.0, 4.0, 6.0):
        grid = helm.Grid(ctx, nx, ny, nz, h, f, c, npml=8, weights=w)
        o = helm.Oras(grid, (8, 8, 4), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
        x, stats = o.solve(bt, tol=tol, restart=30, basis_prec=helm.PREC_FP32)
        assert all(s["converged"] for s in stats), f
        prob = Problem(nx, ny, nz, h, f, c, npml=8, weights=w)
        for res in _oracle_residuals(prob, x.cpu().numpy(), b, [0, 7]):
            assert res <= tol
        del o, grid


def test_thrust_fold_bf16(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz, h, f, tol = 128, 128, 64, 25.0, 5.0, 1e-6
    c = synth.thrust_fold(nx, ny, nz, h, synth.workload_seed(3))
    assert 1700.0 <= c.real.min() and c.real.max() <= 6900.0
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, h, f, c, npml=8, weights=w)
    pos = synth.source_array_positions(nx, ny, 8, 1, 4)
    b = synth.point_sources(nx, ny, nz, h, pos)
    o = helm.Oras(grid, (6, 6, 3), 3, coarse_ratio=4, factor_prec=helm.PREC_BF16)
    x, stats = o.solve(torch.from_numpy(b).cuda(), tol=tol, restart=30, basis_prec=helm.PREC_FP32)
    assert all(s["converged"] for s in stats)
    prob = Problem(nx, ny, nz, h, f, c, npml=8, weights=w)
    for res in _oracle_residuals(prob, x.cpu().numpy(), b, [0, 9]):
        assert res <= tol
