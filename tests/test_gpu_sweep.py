"""Frequency sweeps (helm_frequency_sweep) through the C ABI: one model and one set of sources at several
frequencies, warm starts from the previous frequency, the next frequency's factorisation overlapped with the
current solve on a second context.

Bars: overlap on and off give bit-identical solutions and statistics (each frequency runs the same kernels
in the same order on its own context); every frequency's solution has an oracle FP64 residual <= tol and is
within 10 x tol of an independent cold solve at that frequency; warm starts take no more iterations than
cold ones in total."""
import numpy as np
import pytest

from oracle.discretization import Problem, apply_A
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_sweep_overlap_warm_and_parity(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz, h, tol = 28, 26, 24, 25.0, 1e-6
    freqs = [5.6, 5.8, 6.0]
    c = synth.linear_gradient(nx, ny, nz, h, 1500.0, 0.6, Q=100.0)
    w = helm.fit_weights()
    b = synth.point_sources(nx, ny, nz, h, synth.source_plane_positions(nx, ny, 4, 3, 4, 21))
    bt = torch.from_numpy(b).cuda()
    kw = dict(npml=4, weights=w, coarse_ratio=4, factor_prec=helm.PREC_TF32, tol=tol, restart=30,
              basis_prec=helm.PREC_FP32)
    xo, so, to = helm.frequency_sweep(ctx, nx, ny, nz, h, freqs, c, bt, (2, 2, 2), 2, overlap_factor=True, **kw)
    xs, ss, ts = helm.frequency_sweep(ctx, nx, ny, nz, h, freqs, c, bt, (2, 2, 2), 2, overlap_factor=False, **kw)
    assert torch.equal(xo, xs) and so == ss
    assert all(t > 0 for t in to + ts)
    xc, sc, _ = helm.frequency_sweep(ctx, nx, ny, nz, h, freqs, c, bt, (2, 2, 2), 2, warm=False, **kw)
    warm_its = sum(s["iterations"] for f in so[1:] for s in f)
    cold_its = sum(s["iterations"] for f in sc[1:] for s in f)
    assert warm_its <= cold_its, (warm_its, cold_its)
    assert [s["iterations"] for s in so[0]] == [s["iterations"] for s in sc[0]]   # frequency 0 starts from 0
    x = xo.cpu().numpy()
    for i, f in enumerate(freqs):
        prob = Problem(nx, ny, nz, h, f, c, npml=4, weights=w)
        grid = helm.Grid(ctx, nx, ny, nz, h, f, c, npml=4, weights=w)
        o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
        xi, _ = o.solve(bt, tol=tol, restart=30, basis_prec=helm.PREC_FP32)
        xi = xi.cpu().numpy()
        for r in range(4):
            assert so[i][r]["converged"]
            res = np.linalg.norm(apply_A(prob, x[i][..., r]) - b[..., r]) / np.linalg.norm(b[..., r])
            assert res <= tol
            assert _rel(x[i][..., r], xi[..., r]) <= 10 * tol
        del o, grid


def test_sweep_host_buffers_and_errors(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz, h = 16, 16, 14, 25.0
    c = synth.linear_gradient(nx, ny, nz, h, 1500.0, 0.6)
    b = synth.point_sources(nx, ny, nz, h, [(8, 8, 4), (3, 4, 5)])
    kw = dict(npml=3, coarse_ratio=3, tol=1e-7, restart=20)
    xd, sd, _ = helm.frequency_sweep(ctx, nx, ny, nz, h, [4.0, 4.5], c, torch.from_numpy(b).cuda(), (2, 1, 2), 1,
                                     **kw)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.empty((2,) + tuple(b.shape), dtype=torch.complex128).pin_memory()
    _, sh, _ = helm.frequency_sweep(ctx, nx, ny, nz, h, [4.0, 4.5], c, bh, (2, 1, 2), 1, x=xh, **kw)
    assert torch.equal(xh, xd.cpu()) and sh == sd
    with pytest.raises(helm.HelmError) as e:
        helm.frequency_sweep(ctx, nx, ny, nz, h, [4.0, 0.0], c, torch.from_numpy(b).cuda(), (2, 1, 2), 1, **kw)
    assert e.value.status == helm.EINVAL
    with pytest.raises(helm.HelmError) as e:      # a box decomposition the grid cannot hold fails at frequency 0
        helm.frequency_sweep(ctx, nx, ny, nz, h, [4.0, 4.5], c, torch.from_numpy(b).cuda(), (64, 1, 1), 1, **kw)
    assert e.value.status == helm.EINVAL
    assert ctx.bytes_in_use == 0
