"""GPU parity of the ORAS preconditioner (Eq. oras, Eq. 2lvl) against the FP64 oracle, through the C ABI.

Bars (derived from the arithmetic): FP64 local factors reproduce the oracle's
plane inverses and preconditioner to 1e-9 relative (pivoted Gauss-Jordan
versus LAPACK inverse, condition numbers of the plane Schur complements up to
~1e4 at these sizes); FP32 factors to 1e-3 (the same condition numbers times
FP32 rounding accumulated over the planes).
"""
import numpy as np
import pytest

from oracle.discretization import Problem
from oracle.schwarz import ORAS, decompose, local_operator, plane_blocks, plane_factor
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _setup(ctx, dims, npml=3, f=5.0, Q=None, top=False, weights=None):
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.5, Q=Q)
    w = weights if weights is not None else helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, f, c, npml=npml, top_bc=helm.TOP_PML if top else helm.TOP_DIRICHLET,
                     weights=w)
    prob = Problem(nx, ny, nz, 25.0, f, c, npml=npml, top_pml=top, weights=w)
    return grid, prob


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-3)])
def test_plane_inverses_match_oracle(ctx, prec, tol):
    from paper_2103_14921_gb300 import helm
    dims = (14, 12, 10)
    grid, prob = _setup(ctx, dims, Q=80.0)
    parts, ov = (2, 2, 1), 2
    o = helm.Oras(grid, parts, ov, factor_prec=prec)
    boxes = decompose(dims, parts, ov)
    nb, lo, bdims = o.box_info(1)
    assert nb == len(boxes) and lo == boxes[1].lo and bdims == boxes[1].dims
    for bi in (0, 3):
        b = boxes[bi]
        Ai = local_operator(prob, b, "oras")
        m = b.dims[0] * b.dims[1]
        D, L, U = plane_blocks(Ai, m, b.dims[2])
        G = plane_factor(D, L, U)
        for k in (0, 1, b.dims[2] - 1):
            got = o.plane_inverse(bi, k).cpu().numpy()
            assert _rel(got, G[k]) <= tol, (bi, k)


@pytest.mark.parametrize("coarse", [0, 4])
@pytest.mark.parametrize("mode", [0, 1])
def test_oras_apply_matches_oracle(ctx, coarse, mode):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (21, 18, 17)                        # ragged boxes and a ragged coarse grid
    grid, prob = _setup(ctx, dims, npml=3)
    parts, ov = (3, 2, 2), 2
    o = helm.Oras(grid, parts, ov, coarse_ratio=coarse, interface_bc=mode)
    M = ORAS(prob, parts, ov, coarse_ratio=coarse, mode="oras" if mode == 0 else "ras")
    v = synth.random_complex((dims[2], dims[1], dims[0], 3), 31)
    want = M.apply(v.reshape(-1, 3)).reshape(v.shape)
    got = o.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(got, want) <= 1e-9


def test_oras_apply_fp32_factors(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (20, 20, 16)
    grid, prob = _setup(ctx, dims, npml=3)
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_FP32)
    M = ORAS(prob, (2, 2, 2), 2, coarse_ratio=4)
    v = synth.random_complex((dims[2], dims[1], dims[0], 2), 32)
    want = M.apply(v.reshape(-1, 2)).reshape(v.shape)
    got = o.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(got, want) <= 1e-3


@pytest.mark.parametrize("nrhs", [4, 20, 3])
def test_cooperative_coarse_sweeps_match_per_plane_launches(ctx, nrhs):
    """The complex64 coarse solve in one cooperative launch against the per-plane launches (the
    tuning switch selects the path): the same arithmetic in FP32 summed in another order, so the two
    agree to FP32 rounding (1e-5), and both match the FP64 oracle to the FP32-factor bar (1e-3).
    20 columns take two passes of the 16-column product; the ragged grid gives a ragged coarse plane;
    an odd column count keeps the per-plane launches (the cooperative copies move column pairs)."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (23, 21, 18)
    grid, prob = _setup(ctx, dims, npml=3, Q=90.0)
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=3, factor_prec=helm.PREC_FP32)
    M = ORAS(prob, (2, 2, 2), 2, coarse_ratio=3)
    v = synth.random_complex((dims[2], dims[1], dims[0], nrhs), 35)
    want = M.apply(v.reshape(-1, nrhs)).reshape(v.shape)
    vt = torch.from_numpy(v).cuda()
    got = {}
    for coop in (1, 0):
        ctx.set_tuning(helm.TUNE_COARSE_COOP, coop)
        ctx.profile(True, only=["coarse_sweep"])
        got[coop] = o.apply(vt).cpu().numpy()
        launches = ctx.profile_query("coarse_sweep")[0]
        ctx.profile(False)
        cz = -(-(dims[2] - 1) // 3) + 1
        assert launches == (1 if coop and nrhs % 2 == 0 else 2 * cz - 1), (coop, launches)
    ctx.set_tuning(helm.TUNE_COARSE_COOP, 1)
    assert _rel(got[1], got[0]) <= 1e-5
    for coop in (1, 0):
        assert _rel(got[coop], want) <= 1e-3


@pytest.mark.parametrize("mode", [0, 1])
def test_inexact_coarse_apply_matches_oracle(ctx, mode):
    """The paper's coarse solve (10 GMRES steps with one-level ORAS on the coarse grid, same partition):
    the FP64 preconditioner against the oracle's, on a ragged grid whose coarse partition is ragged too.
    Ten GMRES steps are a smooth function of the data away from breakdown; CGS with re-orthogonalisation
    (GPU) and MGS (oracle) differ by rounding only, so the bar is 1e-8."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (21, 18, 17)
    grid, prob = _setup(ctx, dims, npml=3)
    parts, ov = (3, 2, 2), 2
    o = helm.Oras(grid, parts, ov, coarse_ratio=4, interface_bc=mode, coarse_iters=10, coarse_overlap=1)
    M = ORAS(prob, parts, ov, coarse_ratio=4, mode="oras" if mode == 0 else "ras", coarse_solve="gmres",
             coarse_iters=10, coarse_overlap=1)
    v = synth.random_complex((dims[2], dims[1], dims[0], 3), 36)
    want = M.apply(v.reshape(-1, 3)).reshape(v.shape)
    got = o.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    assert _rel(got, want) <= 1e-8


def test_inexact_coarse_rejects_too_small_coarse_grid(ctx):
    from paper_2103_14921_gb300 import helm
    grid, _ = _setup(ctx, (9, 9, 9), npml=2)
    with pytest.raises(helm.HelmError) as e:
        helm.Oras(grid, (4, 1, 1), 1, coarse_ratio=4, coarse_iters=10)   # 3 coarse nodes, 4 parts
    assert e.value.status == helm.EINVAL
    with pytest.raises(helm.HelmError):
        helm.Oras(grid, (2, 1, 1), 1, coarse_ratio=0, coarse_iters=10)   # no coarse grid


def test_one_box_is_the_exact_inverse(ctx):
    """One box: M^{-1} = A^{-1}, so A M^{-1} v = v (GPU stencil times GPU preconditioner)."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (16, 15, 12)
    grid, prob = _setup(ctx, dims, npml=3, Q=50.0)
    o = helm.Oras(grid, (1, 1, 1), 0)
    v = torch.from_numpy(synth.random_complex((12, 15, 16, 2), 33)).cuda()
    z = o.apply(v)
    back = grid.apply(z)
    assert _rel(back.cpu().numpy(), v.cpu().numpy()) <= 1e-10


def test_coarse_ratio_one_is_the_exact_inverse(ctx):
    """Z = I: Q = A^{-1} and M^{-1} = A^{-1} whatever the boxes."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (12, 11, 10)
    grid, prob = _setup(ctx, dims, npml=2)
    o = helm.Oras(grid, (2, 2, 2), 1, coarse_ratio=1)
    v = torch.from_numpy(synth.random_complex((10, 11, 12, 1), 34)).cuda()
    back = grid.apply(o.apply(v))
    assert _rel(back.cpu().numpy(), v.cpu().numpy()) <= 1e-9


def test_factor_rejects_bad_descriptions(ctx):
    from paper_2103_14921_gb300 import helm
    grid, _ = _setup(ctx, (10, 10, 10), npml=2)
    with pytest.raises(helm.HelmError) as e:
        helm.Oras(grid, (0, 1, 1), 1)
    assert e.value.status == helm.EINVAL
    with pytest.raises(helm.HelmError):
        helm.Oras(grid, (11, 1, 1), 1)


def test_destroy_order_and_profiler(ctx):
    """A grid destroyed before its ORAS handle stays valid until the handle goes; profiling counts launches."""
    import torch
    from paper_2103_14921_gb300 import helm
    grid, _ = _setup(ctx, (12, 12, 10), npml=2)
    o = helm.Oras(grid, (2, 2, 1), 1, coarse_ratio=3)
    grid.close()                                   # deferred: o still uses it
    ctx.profile(True)
    v = torch.from_numpy(synth.random_complex((10, 12, 12, 2), 40)).cuda()
    o.apply(v)
    g = ctx.profile_query("sweep_gemv")
    s = ctx.profile_query("stencil64")            # the FP64 apply: t = v - A q in FP64
    ctx.profile(False)
    assert g is not None and g[0] > 0 and g[1] > 0 and g[2] > 0
    assert s is not None and s[0] == 1
    assert ctx.profile_query("no_such_kernel") is None
    o.close()                                      # frees the grid too
