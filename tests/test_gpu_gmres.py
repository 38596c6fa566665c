"""GPU (F)GMRES with ORAS against the FP64 oracle, through the C ABI.

Bars: converged solutions within 10 x tol (relative L2) of the oracle's
direct solution, and the oracle-evaluated FP64 relative residual of the GPU
solution <= tol (reported together, as the two can differ by the condition
number).
"""
import numpy as np
import pytest

from oracle.discretization import Problem, apply_A, assemble_A
from oracle.schwarz import ORAS, direct_solve_planes
from oracle.krylov import gmres
from oracle.analytic import green_linear_gradient, node_coordinates, relative_l2_misfit, comparison_mask
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _problem(ctx, dims, f=5.0, npml=4, Q=None, top=False):
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 0.6, Q=Q)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, f, c, npml=npml, top_bc=helm.TOP_PML if top else helm.TOP_DIRICHLET,
                     weights=w)
    prob = Problem(nx, ny, nz, 25.0, f, c, npml=npml, top_pml=top, weights=w)
    return grid, prob


def _residual(prob, x, b):
    return np.linalg.norm(apply_A(prob, x) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("flexible", [True, False])
def test_fp64_gmres_matches_oracle_solution_and_iterations(ctx, flexible):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (24, 22, 20)
    grid, prob = _problem(ctx, dims)
    pos = [(12, 11, 3), (5, 17, 9)]
    b = synth.point_sources(*dims, 25.0, pos)
    tol = 1e-8
    o = helm.Oras(grid, (2, 2, 2), 2)
    x, stats = o.solve(torch.from_numpy(b).cuda(), tol=tol, restart=30, flexible=flexible)
    x = x.cpu().numpy()
    xs = direct_solve_planes(prob, b.reshape(-1, 2)).reshape(b.shape)
    M = ORAS(prob, (2, 2, 2), 2)
    A = assemble_A(prob)
    for r in range(2):
        assert stats[r]["converged"]
        assert _rel(x[..., r], xs[..., r]) <= 10 * tol
        assert _residual(prob, x[..., r], b[..., r]) <= tol
        _, info = gmres(lambda v: A @ v, b[..., r].ravel(), M.apply, tol=tol, restart=30, flexible=flexible)
        assert abs(stats[r]["iterations"] - info["iterations"]) <= 1


def test_two_level_fgmres_restarts_and_mixed_precision(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (28, 26, 24)
    grid, prob = _problem(ctx, dims, f=6.0, Q=100.0)
    rng_pos = synth.source_plane_positions(28, 26, 4, 3, 4, 7)
    b = synth.point_sources(*dims, 25.0, rng_pos)
    xs = direct_solve_planes(prob, b.reshape(-1, 4)).reshape(b.shape)
    tol = 1e-6
    for fprec, bprec in [(helm.PREC_FP64, helm.PREC_FP64), (helm.PREC_FP32, helm.PREC_FP32)]:
        o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=fprec)
        x, stats = o.solve(torch.from_numpy(b).cuda(), tol=tol, restart=8, basis_prec=bprec)
        x = x.cpu().numpy()
        for r in range(4):
            assert stats[r]["converged"], stats[r]
            assert _residual(prob, x[..., r], b[..., r]) <= tol
            assert _rel(x[..., r], xs[..., r]) <= 10 * tol


def test_host_buffers_and_zero_rhs(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (16, 16, 14)
    grid, prob = _problem(ctx, dims, npml=3)
    b = synth.point_sources(*dims, 25.0, [(8, 8, 4), (3, 4, 5), (9, 9, 9)])
    b[..., 1] = 0.0                                # a zero column gives x = 0 with no iterations
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    o = helm.Oras(grid, (2, 1, 2), 1, coarse_ratio=3)
    _, stats = o.solve(bh, xh, tol=1e-7, restart=20)
    x = xh.numpy()
    assert stats[1]["iterations"] == 0 and np.all(x[..., 1] == 0)
    for r in (0, 2):
        assert _residual(prob, x[..., r], b[..., r]) <= 1e-7


def test_notconv_and_nonfinite_are_reported(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (16, 16, 14)
    grid, prob = _problem(ctx, dims, npml=3)
    b = synth.point_sources(*dims, 25.0, [(8, 8, 4)])
    o = helm.Oras(grid, (2, 2, 2), 1)
    x, stats = o.solve(torch.from_numpy(b).cuda(), tol=1e-12, restart=3, maxit=4, allow_notconv=True)
    assert not stats[0]["converged"] and stats[0]["iterations"] == 4
    assert np.isfinite(stats[0]["true_relres"]) and stats[0]["true_relres"] < 1
    bad = b.copy()
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(helm.HelmError) as e:
        o.solve(torch.from_numpy(bad).cuda())
    assert e.value.status == helm.ENONFINITE


def test_linear_gradient_one_level_matches_closed_form(ctx):
    """48^3, c = 1500 + 0.6 z, 3 Hz, one-level ORAS 2x2x2 overlap 2, FP64 GMRES(30) to 1e-6, PML top."""
    import torch
    from paper_2103_14921_gb300 import helm
    n, h, f = 48, 25.0, 3.0
    grid, prob = _problem(ctx, (n, n, n), f=f, npml=8, top=True)
    s = (24, 24, 24)
    b = synth.point_sources(n, n, n, h, [s])
    o = helm.Oras(grid, (2, 2, 2), 2)
    x, stats = o.solve(torch.from_numpy(b).cuda(), tol=1e-6, restart=30, flexible=False)
    assert stats[0]["converged"]
    u = x.cpu().numpy()[..., 0]
    X, Y, Z = node_coordinates(n, n, n, h)
    G = green_linear_gradient(X, Y, Z, (s[0] * h, s[1] * h, (s[2] + 1) * h), 2 * np.pi * f, 1500.0, 0.6)
    mask = comparison_mask(n, n, n, 8, True, s, 4)
    assert relative_l2_misfit(u, -G, mask) <= 0.05


def test_graph_replayed_iterations_equal_eager_launches(ctx):
    """Krylov iterations replayed from captured CUDA graphs run the same kernels with the same
    arguments as host launches, and every reduction has a fixed order, so the solutions are
    bit-identical; the launch count and the profiler's per-family records agree too (the profiled
    kernels are timed through event nodes inside the graphs).  Restart 8 with about twice as many
    iterations makes the second cycle and the next solves replay graphs captured earlier."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (28, 26, 24)
    grid, prob = _problem(ctx, dims, f=6.0, Q=100.0)
    pos = synth.source_plane_positions(28, 26, 4, 3, 6, 11)
    b = torch.from_numpy(synth.point_sources(*dims, 25.0, pos)).cuda()
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
    kw = dict(tol=1e-6, restart=8, basis_prec=helm.PREC_FP32)

    def run():
        ctx.profile(True, only=["sweep_flow", "coarse_sweep"])
        l0 = ctx.launches
        x, st = o.solve(b, **kw)
        n = ctx.launches - l0
        prof = {f: ctx.profile_query(f) for f in ("sweep_flow", "coarse_sweep")}
        ctx.profile(False)
        return x, [s["iterations"] for s in st], n, prof

    ctx.set_tuning(helm.TUNE_GRAPHS, 0)
    x0, it0, n0, p0 = run()
    assert max(it0) > 8
    ctx.set_tuning(helm.TUNE_GRAPHS, 1)
    for _ in range(3):                       # capture on second use, then replays
        x1, it1, n1, p1 = run()
        assert it1 == it0
        assert torch.equal(x1, x0)
        assert n1 == n0
        for f in p0:
            assert p1[f][0] == p0[f][0] and p1[f][1] > 0
    assert _residual(prob, x1.cpu().numpy()[..., 0], b.cpu().numpy()[..., 0]) <= 1e-6


def test_inexact_coarse_fgmres_mixed_precision(ctx):
    """FGMRES with the paper's inexact coarse solve (10 inner GMRES steps, coarse ORAS) and TF32 local
    factors converges; the oracle's FP64 residual of the result is <= tol and the solution is within
    10 x tol of the direct solution.  A second solve replays the captured iteration graphs (the inner
    solve runs without host synchronisation inside them) and gives the same iterate."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (28, 26, 24)
    grid, prob = _problem(ctx, dims, f=6.0, Q=100.0)
    pos = synth.source_plane_positions(28, 26, 4, 3, 4, 9)
    b = synth.point_sources(*dims, 25.0, pos)
    xs = direct_solve_planes(prob, b.reshape(-1, 4)).reshape(b.shape)
    tol = 1e-6
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32, coarse_iters=10)
    bt = torch.from_numpy(b).cuda()
    x1, st1 = o.solve(bt, tol=tol, restart=30, flexible=True, basis_prec=helm.PREC_FP32)
    x2, st2 = o.solve(bt, tol=tol, restart=30, flexible=True, basis_prec=helm.PREC_FP32)
    assert torch.equal(x1, x2) and [s["iterations"] for s in st1] == [s["iterations"] for s in st2]
    x = x1.cpu().numpy()
    for r in range(4):
        assert st1[r]["converged"], st1[r]
        assert _residual(prob, x[..., r], b[..., r]) <= tol
        assert _rel(x[..., r], xs[..., r]) <= 10 * tol


def test_adaptive_weights_two_level_solve(ctx):
    """The two-level FGMRES solve with adaptive stencil weights (TF32 local factors): converged, the oracle's
    FP64 residual of its own row-weighted operator <= tol, and within 10 x tol of its direct solution."""
    import torch
    from paper_2103_14921_gb300 import helm
    from oracle.weights import row_weight_bins
    nx, ny, nz = 26, 24, 28
    h, f = 25.0, 7.0
    c = synth.linear_gradient(nx, ny, nz, h, 1000.0, 2.0)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, h, f, c, npml=4, weights=w, weight_bins=4)
    edges, table = grid.row_weights()
    prob = Problem(nx, ny, nz, h, f, c, npml=4, weights=w, row_weights=table[row_weight_bins(c, f, h, edges)])
    pos = synth.source_plane_positions(nx, ny, 4, 3, 3, 13)
    b = synth.point_sources(nx, ny, nz, h, pos)
    xs = direct_solve_planes(prob, b.reshape(-1, 3)).reshape(b.shape)
    tol = 1e-6
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
    x, st = o.solve(torch.from_numpy(b).cuda(), tol=tol, restart=30, basis_prec=helm.PREC_FP32)
    x = x.cpu().numpy()
    for r in range(3):
        assert st[r]["converged"]
        assert _residual(prob, x[..., r], b[..., r]) <= tol
        assert _rel(x[..., r], xs[..., r]) <= 10 * tol


def test_warm_start_from_neighbouring_frequency(ctx):
    """Warm starts (use_x0): the solution at 5.0 Hz as the initial guess at 5.2 Hz.  The GPU FP64 GMRES
    from that guess converges with the oracle's FP64 residual <= tol, within 10 x tol of the direct
    solution, in the oracle's iteration count (+-1) from the same guess; restarting from its own result
    takes no iteration and returns it unchanged; a b = 0 column returns 0 whatever the guess."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (24, 22, 20)
    pos = [(12, 11, 3), (5, 17, 9), (18, 6, 4)]
    b = synth.point_sources(*dims, 25.0, pos)
    b[..., 2] = 0.0
    tol = 1e-8
    grid0, _ = _problem(ctx, dims, f=5.0)
    x0, _ = helm.Oras(grid0, (2, 2, 2), 2).solve(torch.from_numpy(b).cuda(), tol=tol, restart=30)
    x0[..., 2] = 1.0 + 1.0j                        # a guess for the zero column that must be ignored
    grid, prob = _problem(ctx, dims, f=5.2)
    o = helm.Oras(grid, (2, 2, 2), 2)
    _, cold = o.solve(torch.from_numpy(b).cuda(), tol=tol, restart=30)
    x = x0.clone()
    _, st = o.solve(torch.from_numpy(b).cuda(), x, tol=tol, restart=30, warm=True)
    xh = x.cpu().numpy()
    xs = direct_solve_planes(prob, b.reshape(-1, 3)).reshape(b.shape)
    M = ORAS(prob, (2, 2, 2), 2)
    A = assemble_A(prob)
    x0h = x0.cpu().numpy()
    for r in range(2):
        assert st[r]["converged"]
        assert _residual(prob, xh[..., r], b[..., r]) <= tol
        assert _rel(xh[..., r], xs[..., r]) <= 10 * tol
        _, info = gmres(lambda v: A @ v, b[..., r].ravel(), M.apply, tol=tol, restart=30,
                        x0=x0h[..., r].ravel())
        assert abs(st[r]["iterations"] - info["iterations"]) <= 1
        assert st[r]["iterations"] < cold[r]["iterations"]
    assert st[2]["iterations"] == 0 and torch.all(x[..., 2] == 0)
    x2 = x.clone()
    _, st2 = o.solve(torch.from_numpy(b).cuda(), x2, tol=tol, restart=30, warm=True)
    assert all(s["iterations"] == 0 and s["converged"] for s in st2)
    assert torch.equal(x2, x)
    with pytest.raises(helm.HelmError) as e:           # nonfinite guess
        x3 = x.clone()
        x3[0, 0, 0, 0] = complex("nan")
        o.solve(torch.from_numpy(b).cuda(), x3, tol=tol, warm=True)
    assert e.value.status == helm.ENONFINITE
