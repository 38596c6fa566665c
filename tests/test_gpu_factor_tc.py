"""The plane factorisation on the tensor cores (blocked Gauss-Jordan, 128-column panels, block pivots,
rank-128 updates as tcgen05 products with the three-product TF32 split) against the oracle.

The oracle's inverses S_k^{-1} (Eq. oras local solves: S_0 = D_0, S_k = D_k - L_k S_{k-1}^{-1} U_{k-1},
numpy.linalg.inv in FP64) are the reference.  Bar: the stored complex64 inverses within 1e-4 relative
(Frobenius) of the oracle's -- FP32 elimination error (2^-24 per operation) grown by the planes'
condition numbers (1e0-1e2 here) and the 3-product split (each product within 2^-20 of FP32's), far
inside 1e-4; the fully pivoted CUDA-core elimination (the tuning switch) lands within the same bar of both.
BF16-stored inverses: the same values rounded to bfloat16 (2^-9 relative per entry): 1e-2.
Boxes of 22 x 36 = 792 nodes per plane (six full 128-column panels and a partial one), and 34 x 34 = 1156
(nine and a partial one), so every kernel of the panel step and the product's partial tiles run.
"""
import numpy as np
import pytest

from oracle.discretization import Problem
from oracle.schwarz import decompose, local_operator, plane_blocks, plane_factor
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("dims,parts,Q", [((40, 36, 6), (2, 1, 1), None), ((64, 64, 5), (2, 2, 1), 60.0)])
def test_tc_factor_inverses_match_oracle(ctx, dims, parts, Q):
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0, Q=Q)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=4, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 5.0, c, npml=4, weights=w)
    ov = 2
    boxes = decompose(dims, parts, ov)
    got = {}
    for mode in (1, 0):
        ctx.set_tuning(helm.TUNE_TC_FACTOR, mode)
        ctx.profile(True, only=["gj_update_tc", "gj_update"])
        o = helm.Oras(grid, parts, ov, factor_prec=helm.PREC_TF32)
        tc_runs = (ctx.profile_query("gj_update_tc") or (0,))[0]
        cc_runs = (ctx.profile_query("gj_update") or (0,))[0]
        ctx.profile(False)
        assert (tc_runs > 0) == (mode == 1) and (cc_runs > 0) == (mode == 0), (mode, tc_runs, cc_runs)
        got[mode] = {(bi, k): o.plane_inverse(bi, k).cpu().numpy() for bi in (0, len(boxes) - 1)
                     for k in (0, 1, nz - 1)}
        o.close()
    ctx.set_tuning(helm.TUNE_TC_FACTOR, 1)
    worst = 0.0
    for bi in (0, len(boxes) - 1):
        b = boxes[bi]
        m = b.dims[0] * b.dims[1]
        assert m > 128
        D, L, U = plane_blocks(local_operator(prob, b, "oras"), m, b.dims[2])
        G = plane_factor(D, L, U)
        for k in (0, 1, nz - 1):
            e_tc = _rel(got[1][bi, k], G[k])
            worst = max(worst, e_tc)
            assert e_tc <= 1e-4, (bi, k, e_tc)
            assert _rel(got[0][bi, k], G[k]) <= 1e-4, (bi, k)
            assert _rel(got[1][bi, k], got[0][bi, k]) <= 1e-4, (bi, k)
    print(f"tensor-core factorisation, dims {dims}: worst relative error vs oracle {worst:.2e}")


def test_tc_factor_bf16_storage(ctx):
    from paper_2103_14921_gb300 import helm
    dims, parts = (40, 36, 6), (2, 1, 1)
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=4, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 5.0, c, npml=4, weights=w)
    o = helm.Oras(grid, parts, 2, factor_prec=helm.PREC_BF16)
    b = decompose(dims, parts, 2)[1]
    m = b.dims[0] * b.dims[1]
    D, L, U = plane_blocks(local_operator(prob, b, "oras"), m, b.dims[2])
    G = plane_factor(D, L, U)
    for k in (0, 3, nz - 1):
        assert _rel(o.plane_inverse(1, k).cpu().numpy(), G[k]) <= 1e-2, k


def test_tc_factor_solves_the_two_level_problem(ctx):
    """A two-level TF32 solve with tensor-core factors converges in the same iteration counts (+-1) as with
    the CUDA-core factors, to the same tolerance."""
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = 48, 44, 30
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 0.6)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=6, weights=helm.fit_weights())
    b = torch.from_numpy(synth.point_sources(nx, ny, nz, 25.0, synth.source_plane_positions(nx, ny, 6, 3, 4, 5)))
    its = {}
    for mode in (1, 0):
        ctx.set_tuning(helm.TUNE_TC_FACTOR, mode)
        o = helm.Oras(grid, (2, 2, 1), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
        x, st = o.solve(b.cuda(), tol=1e-6, basis_prec=helm.PREC_FP32)
        assert all(s["converged"] and s["true_relres"] <= 1e-6 for s in st)
        its[mode] = [s["iterations"] for s in st]
        o.close()
    ctx.set_tuning(helm.TUNE_TC_FACTOR, 1)
    assert all(abs(a - b_) <= 1 for a, b_ in zip(its[1], its[0])), its


@pytest.mark.parametrize("prec,bar", [(0, 1e-9), (1, 1e-4)])
def test_block_pivot_cuda_core_factor_matches_oracle(ctx, prec, bar):
    """FP64 and FP32 sets by the block-pivot elimination on the CUDA cores (64-column panels, rank-64 updates
    over all SMs): planes of 792 nodes (twelve full panels and a partial one) against the oracle's inverses,
    and against the fully pivoted elimination (the tuning switch).  FP64: LAPACK-level agreement (1e-9);
    FP32: the same bar as the tensor-core factors (1e-4)."""
    from paper_2103_14921_gb300 import helm
    dims, parts = (40, 36, 6), (2, 1, 1)
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0, Q=80.0)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=4, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 5.0, c, npml=4, weights=w)
    b = decompose(dims, parts, 2)[0]
    m = b.dims[0] * b.dims[1]
    D, L, U = plane_blocks(local_operator(prob, b, "oras"), m, b.dims[2])
    G = plane_factor(D, L, U)
    got = {}
    for mode in (1, 0):
        ctx.set_tuning(helm.TUNE_BLOCK_GJ, mode)
        ctx.profile(True, only=["gj_update"])
        o = helm.Oras(grid, parts, 2, coarse_ratio=4, factor_prec=prec)
        n_upd = ctx.profile_query("gj_update")[0]
        ctx.profile(False)
        got[mode] = [o.plane_inverse(0, k).cpu().numpy() for k in range(nz)]
        if mode == 1:   # one rank-64 update per panel and plane of the fine set, plus the coarse set's
            assert n_upd >= nz * ((m + 63) // 64)
        o.close()
    ctx.set_tuning(helm.TUNE_BLOCK_GJ, 1)
    for k in range(nz):
        assert _rel(got[1][k], G[k]) <= bar, k
        assert _rel(got[1][k], got[0][k]) <= bar, k
