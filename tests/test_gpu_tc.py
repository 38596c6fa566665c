"""Tensor-core (tcgen05 kind::tf32) plane sweeps, through the C ABI.

Single-plane boxes make every local solve exactly one tensor-core GEMM
y = G_0 (R_i v); the result must equal the same product computed in FP64
from TF32-rounded operands up to FP32 accumulation (2e-5 relative), and the
exact FP64 product up to TF32 input rounding (2e-3).  Multi-plane TF32 local
solves are checked through converged FGMRES solutions.
"""
import numpy as np
import pytest

from oracle.discretization import Problem, apply_A
from oracle.schwarz import direct_solve_planes
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _tf32(a, mode):
    """Round float32 values to TF32 (10 explicit mantissa bits): truncation or nearest-even."""
    import torch
    x = a.contiguous().view(torch.int32)
    if mode == "rn":
        lsb = (x >> 13) & 1
        x = x + 0x0FFF + lsb
    return (x & ~0x1FFF).view(torch.float32)


def _emulate(G, R, mode):
    import torch
    Gr = torch.complex(_tf32(G.real.float(), mode), _tf32(G.imag.float(), mode)).to(torch.complex128)
    Rr = torch.complex(_tf32(R.real.float(), mode), _tf32(R.imag.float(), mode)).to(torch.complex128)
    return Gr @ Rr


@pytest.mark.parametrize("dims,nrhs", [((24, 20, 2), 16), ((37, 29, 2), 3), ((12, 40, 2), 40)])
def test_single_plane_boxes_equal_emulated_tf32_gemm(ctx, dims, nrhs):
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=1, weights=helm.fit_weights())
    parts = (2, 2, 2)
    o = helm.Oras(grid, parts, 0, factor_prec=helm.PREC_TF32)
    v = torch.from_numpy(synth.random_complex((nz, ny, nx, nrhs), 61)).cuda()
    got = o.apply(v)
    nb = o.box_info(0)[0]
    for b in range(nb):
        _, lo, bd = o.box_info(b)
        assert bd[2] == 1
        G = o.plane_inverse(b, 0)                                 # stored complex64 values, widened
        vb = v[lo[2], lo[1]:lo[1] + bd[1], lo[0]:lo[0] + bd[0], :].reshape(-1, nrhs)
        vb32 = vb.to(torch.complex64).to(torch.complex128)
        y = got[lo[2], lo[1]:lo[1] + bd[1], lo[0]:lo[0] + bd[0], :].reshape(-1, nrhs)
        exact = G @ vb32
        errs = [float(torch.linalg.norm(y - _emulate(G, vb32, mode)) / torch.linalg.norm(exact))
                for mode in ("trunc", "rn")]
        assert min(errs) <= 2e-5, (b, errs)
        assert float(torch.linalg.norm(y - exact) / torch.linalg.norm(exact)) <= 2e-3


@pytest.mark.parametrize("dims,nrhs", [((24, 20, 2), 16), ((37, 29, 2), 5)])
def test_single_plane_boxes_bf16_factors(ctx, dims, nrhs):
    """BF16-stored factors (kind::f16): equal to the FP64 product of the bf16-rounded operands (products of
    bf16 values are exact in FP32, so only the FP32 accumulation differs: 2e-5), and within bf16 rounding
    (2e-2) of the product with the complex64 operands."""
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=1, weights=helm.fit_weights())
    o = helm.Oras(grid, (2, 2, 2), 0, factor_prec=helm.PREC_BF16)
    v = torch.from_numpy(synth.random_complex((nz, ny, nx, nrhs), 62)).cuda()
    got = o.apply(v)
    for b in range(o.box_info(0)[0]):
        _, lo, bd = o.box_info(b)
        G = o.plane_inverse(b, 0)                                  # the stored bf16 values, widened
        vb = v[lo[2], lo[1]:lo[1] + bd[1], lo[0]:lo[0] + bd[0], :].reshape(-1, nrhs).to(torch.complex64)
        vr = torch.complex(vb.real.to(torch.bfloat16).double(), vb.imag.to(torch.bfloat16).double())
        y = got[lo[2], lo[1]:lo[1] + bd[1], lo[0]:lo[0] + bd[0], :].reshape(-1, nrhs)
        want = G @ vr
        assert float(torch.linalg.norm(y - want) / torch.linalg.norm(want)) <= 2e-5, b
        exact = G @ vb.to(torch.complex128)
        assert float(torch.linalg.norm(y - exact) / torch.linalg.norm(exact)) <= 2e-2


def test_bf16_fgmres_converges(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (30, 28, 26)
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 0.6)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 6.0, c, npml=4, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 6.0, c, npml=4, weights=w)
    b = synth.point_sources(nx, ny, nz, 25.0, synth.source_plane_positions(nx, ny, 4, 3, 4, 10))
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_BF16)
    x, stats = o.solve(torch.from_numpy(b).cuda(), tol=1e-6, restart=30, basis_prec=helm.PREC_FP32)
    x = x.cpu().numpy()
    for r in range(4):
        assert stats[r]["converged"]
        res = np.linalg.norm(apply_A(prob, x[..., r]) - b[..., r]) / np.linalg.norm(b[..., r])
        assert res <= 1e-6


def test_tf32_fgmres_converges_to_the_direct_solution(ctx):
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (30, 28, 26)
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 0.6)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 6.0, c, npml=4, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 6.0, c, npml=4, weights=w)
    pos = synth.source_plane_positions(nx, ny, 4, 3, 6, 9)
    b = synth.point_sources(nx, ny, nz, 25.0, pos)
    xs = direct_solve_planes(prob, b.reshape(-1, 6)).reshape(b.shape)
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
    x, stats = o.solve(torch.from_numpy(b).cuda(), tol=1e-6, restart=30, basis_prec=helm.PREC_FP32)
    x = x.cpu().numpy()
    for r in range(6):
        assert stats[r]["converged"]
        res = np.linalg.norm(apply_A(prob, x[..., r]) - b[..., r]) / np.linalg.norm(b[..., r])
        assert res <= 1e-6
        assert np.linalg.norm(x[..., r] - xs[..., r]) <= 1e-5 * np.linalg.norm(xs[..., r])


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("parts,nrhs", [((3, 2, 2), 16), ((3, 1, 1), 2), ((2, 2, 2), 40), ((2, 2, 2), 128),
                                        ((2, 1, 2), 3)])
def test_persistent_sweep_equals_per_step_launches(ctx, prec, parts, nrhs):
    """Both sweeps of every box as one persistent launch fed by a device work queue, against one
    preparation and one product launch per plane step: the same arithmetic on every element, so the
    preconditioner outputs are bit-identical.  Ragged boxes with unequal plane counts, a single-box
    row, 40 columns (N = 128), 128 columns (N = 256: the persistent launch stages its preparation tiles in
    column chunks) and an odd column count (which keeps the per-step launches).  Launches:
    one persistent (family sweep_flow), or 2 n_z - 1 of each kind; repeated applies reuse the queue."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (21, 18, 17)
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=3, weights=helm.fit_weights())
    fp = helm.PREC_TF32 if prec == "tf32" else helm.PREC_BF16
    o = helm.Oras(grid, parts, 2, factor_prec=fp)
    v = torch.from_numpy(synth.random_complex((nz, ny, nx, nrhs), 63)).cuda()
    bz = max(o.box_info(b)[2][2] for b in range(o.box_info(0)[0]))
    steps = 2 * bz - 1
    got, counts = {}, {}
    fams = ("sweep_prep", "sweep_gemm_tc", "sweep_flow")
    for flow in (1, 0):
        ctx.set_tuning(helm.TUNE_TC_FLOW, flow)
        ctx.profile(True, only=list(fams))
        got[flow] = o.apply(v)
        counts[flow] = tuple((ctx.profile_query(f) or (0,))[0] for f in fams)
        ctx.profile(False)
    ctx.set_tuning(helm.TUNE_TC_FLOW, 1)
    again = o.apply(v)
    assert torch.equal(got[1], got[0])
    assert torch.equal(again, got[1])
    assert torch.isfinite(torch.view_as_real(got[1])).all()
    assert counts[0] == (steps, steps, 0)
    assert counts[1] == ((0, 0, 1) if nrhs % 2 == 0 else (steps, steps, 0))
