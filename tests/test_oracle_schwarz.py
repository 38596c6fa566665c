"""Pins of the oracle's ORAS preconditioner (Eq. oras, Eq. 2lvl) and local solves."""
import numpy as np
import scipy.sparse.linalg as spla
import pytest

from oracle.discretization import Problem, assemble_A, apply_A
from oracle.schwarz import (ORAS, decompose, restriction, partition_of_unity, local_operator, plane_blocks,
                            plane_factor, plane_solve, coarse_basis, coarse_dims, box_global_indices,
                            direct_solve_planes)
from oracle.krylov import gmres
from paper_2103_14921_gb300 import synth


def _prob(nx, ny, nz, c=None, npml=3, f=6.0, weights=None, top_pml=False):
    if c is None:
        c = synth.linear_gradient(nx, ny, nz, 25.0)
    if weights is None:
        weights = synth.random_weights(21)
    return Problem(nx, ny, nz, 25.0, f, c, npml=npml, top_pml=top_pml, weights=weights)


def test_partition_of_unity_sums_to_identity():
    dims = (13, 11, 9)
    boxes = decompose(dims, (3, 2, 2), 2)
    n = np.prod(dims)
    S = sum(restriction(b, dims).T @ (partition_of_unity(b)[:, None] * restriction(b, dims).toarray())
            for b in boxes)
    assert np.array_equal(S, np.eye(n))


def test_boxes_overlap_and_clip():
    boxes = decompose((48, 48, 48), (2, 2, 2), 2)
    assert len(boxes) == 8
    assert boxes[0].lo == (0, 0, 0) and boxes[0].hi == (26, 26, 26)
    assert boxes[-1].lo == (22, 22, 22) and boxes[-1].hi == (48, 48, 48)
    boxes = decompose((112, 112, 112), (4, 4, 4), 2)
    assert max(b.dims[0] for b in boxes) == 32 and min(b.dims[0] for b in boxes) == 30


def test_ras_local_operator_is_the_restricted_global_operator():
    prob = _prob(12, 11, 10)
    A = assemble_A(prob)
    for b in decompose((12, 11, 10), (2, 2, 2), 2):
        R = restriction(b, (12, 11, 10))
        Ai = local_operator(prob, b, "ras")
        assert abs(Ai - R @ A @ R.T).max() == 0


def test_oras_differs_only_on_interface_rows():
    prob = _prob(12, 11, 10)
    A = assemble_A(prob)
    dims = (12, 11, 10)
    for b in decompose(dims, (2, 2, 2), 2):
        R = restriction(b, dims)
        diff = (local_operator(prob, b, "oras") - R @ A @ R.T).tocsr()
        rows = np.unique(diff.nonzero()[0])
        bx, by, bz = b.dims
        k, j, i = np.unravel_index(rows, (bz, by, bx))
        gi, gj, gk = i + b.lo[0], j + b.lo[1], k + b.lo[2]
        on_iface = (((i == 0) & (b.lo[0] > 0)) | ((i == bx - 1) & (b.hi[0] < dims[0]))
                    | ((j == 0) & (b.lo[1] > 0)) | ((j == by - 1) & (b.hi[1] < dims[1]))
                    | ((k == 0) & (b.lo[2] > 0)) | ((k == bz - 1) & (b.hi[2] < dims[2])))
        assert on_iface.all()
        assert len(rows) > 0


def test_absorbing_fold_is_exact_for_outgoing_waves():
    """Homogeneous box: ``A_i R_i u = R_i A u`` for ``u = prod_a exp(i k |x_a - mid_a|)``."""
    dims = (14, 13, 12)
    c = synth.homogeneous(*dims, 1800.0) * (1 - 0.01j)
    prob = _prob(*dims, c=c, npml=3)
    A = assemble_A(prob)
    kk = prob.omega / complex(c[0, 0, 0])
    for b in decompose(dims, (2, 2, 2), 2):
        mid = [(b.lo[a] + b.hi[a] - 1) / 2.0 for a in range(3)]
        k, j, i = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
        u = (np.exp(1j * kk * prob.h * np.abs(i - mid[0])) * np.exp(1j * kk * prob.h * np.abs(j - mid[1]))
             * np.exp(1j * kk * prob.h * np.abs(k - mid[2]))).ravel()
        R = restriction(b, dims)
        lhs = local_operator(prob, b, "oras") @ (R @ u)
        rhs = R @ (A @ u)
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
        # the Dirichlet (RAS) operator does not satisfy it
        lhs_ras = local_operator(prob, b, "ras") @ (R @ u)
        assert np.linalg.norm(lhs_ras - rhs) > 1e-3 * np.linalg.norm(rhs)


def test_plane_lu_equals_dense_solve():
    prob = _prob(10, 9, 11, c=synth.linear_gradient(10, 9, 11, 25.0, Q=80.0))
    dims = (10, 9, 11)
    for b in decompose(dims, (2, 1, 2), 2)[:2]:
        Ai = local_operator(prob, b, "oras")
        m = b.dims[0] * b.dims[1]
        D, L, U = plane_blocks(Ai, m, b.dims[2])
        G = plane_factor(D, L, U)
        rhs = synth.random_complex((b.size, 3), 8)
        x = plane_solve(G, L, U, rhs)
        want = np.linalg.solve(Ai.toarray(), rhs)
        assert np.linalg.norm(x - want) <= 1e-11 * np.linalg.norm(want)
        # and the first Schur complement inverse is the inverse of the first diagonal block
        assert np.allclose(G[0] @ D[0], np.eye(m), atol=1e-10)


def test_direct_solve_planes_matches_splu():
    prob = _prob(12, 10, 9, npml=3)
    b = synth.random_complex((prob.n, 2), 12)
    x = direct_solve_planes(prob, b)
    want = spla.splu(assemble_A(prob).tocsc()).solve(b)
    assert np.linalg.norm(x - want) <= 1e-11 * np.linalg.norm(want)


def test_one_subdomain_is_the_direct_solve():
    """One box: ``M^{-1} = A^{-1}`` so GMRES converges in one iteration."""
    prob = _prob(11, 10, 9)
    M = ORAS(prob, (1, 1, 1), 2)
    A = assemble_A(prob)
    b = synth.random_complex((prob.n,), 13)
    x, info = gmres(lambda v: A @ v, b, M.apply, tol=1e-10, restart=10)
    assert info["iterations"] == 1 and info["converged"]


def test_coarse_ratio_one_is_the_direct_solve():
    """``Z = I`` makes ``Q = A^{-1}`` and ``M^{-1} = A^{-1}``."""
    prob = _prob(10, 9, 8)
    M = ORAS(prob, (2, 2, 1), 1, coarse_ratio=1)
    A = assemble_A(prob)
    b = synth.random_complex((prob.n,), 14)
    x, info = gmres(lambda v: A @ v, b, M.apply, tol=1e-10, restart=10)
    assert info["iterations"] == 1


def test_coarse_basis_properties():
    dims = (13, 10, 9)
    r = 4
    Z = coarse_basis(dims, r)
    nc = coarse_dims(dims, r)
    assert Z.shape == (np.prod(dims), np.prod(nc))
    assert np.allclose(Z @ np.ones(Z.shape[1]), 1.0)           # hats sum to one
    # trilinear interpolation reproduces linear functions exactly
    K, J, I = np.meshgrid(np.arange(nc[2]), np.arange(nc[1]), np.arange(nc[0]), indexing="ij")
    k, j, i = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    lin = lambda a, b_, c: 0.3 + 1.7 * a - 0.4 * b_ + 2.2 * c
    assert np.allclose(Z @ lin(r * I, r * J, r * K).ravel(), lin(i, j, k).ravel())
    # E = Z^T A Z couples coarse nodes at most one step apart (27-point)
    prob = _prob(*dims, npml=2)
    E = (Z.T @ assemble_A(prob) @ Z).tocoo()
    Jr = np.array(np.unravel_index(E.row, nc[::-1]))
    Jc = np.array(np.unravel_index(E.col, nc[::-1]))
    assert np.abs(Jr - Jc).max() <= 1
    assert coarse_dims((112, 112, 112), 4) == (29, 29, 29)


def test_two_level_oras_fgmres_reaches_direct_solution():
    prob = _prob(20, 20, 20, npml=4, weights=None, f=5.0)
    A = assemble_A(prob)
    b = synth.point_sources(20, 20, 20, 25.0, [(10, 10, 3)])[..., 0].ravel()
    xs = direct_solve_planes(prob, b)
    for coarse in (0, 4):
        M = ORAS(prob, (2, 2, 2), 2, coarse_ratio=coarse)
        x, info = gmres(lambda v: A @ v, b, M.apply, tol=1e-8, restart=30)
        assert info["converged"]
        assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)


def test_oras_converges_faster_than_ras():
    prob = _prob(20, 20, 20, npml=4, f=5.0)
    A = assemble_A(prob)
    b = synth.point_sources(20, 20, 20, 25.0, [(10, 10, 3)])[..., 0].ravel()
    its = {}
    for mode in ("oras", "ras"):
        M = ORAS(prob, (2, 2, 2), 2, mode=mode)
        _, info = gmres(lambda v: A @ v, b, M.apply, tol=1e-8, restart=50)
        its[mode] = info["iterations"]
    assert its["oras"] < its["ras"]


def test_plane_local_route_equals_splu_route():
    prob = _prob(14, 12, 10, npml=3)
    v = synth.random_complex((prob.n, 2), 15)
    a = ORAS(prob, (2, 2, 1), 2, coarse_ratio=4, local="splu").apply(v)
    b = ORAS(prob, (2, 2, 1), 2, coarse_ratio=4, local="planes").apply(v)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)


# --- the paper's inexact coarse solve (10 inner GMRES iterations, one-level ORAS on the coarse grid) ---

def test_stencil_diagonals_reassemble_the_operator():
    """The 27 diagonals read off the assembled matrix equal the oracle's own coefficient array."""
    from oracle.discretization import neighbour_coefficients
    from oracle.schwarz import stencil_coefficients_of
    prob = _prob(9, 8, 7, npml=2)
    got = stencil_coefficients_of(assemble_A(prob), (9, 8, 7))
    assert np.array_equal(got, neighbour_coefficients(prob))


def test_coarse_partition_follows_the_fine_cuts_and_sums_to_identity():
    from oracle.schwarz import coarse_decompose
    dims, parts, r = (21, 18, 17), (3, 2, 2), 4
    cd = coarse_dims(dims, r)
    boxes = coarse_decompose(dims, parts, r, 1)
    fine = decompose(dims, parts, 0)
    n = int(np.prod(cd))
    S = np.zeros((n, n))
    for b, fb in zip(boxes, fine):
        R = restriction(b, cd).toarray()
        S += R.T @ (partition_of_unity(b)[:, None] * R)
        # every core node's fine position r J (clamped) lies in the matching fine core
        for a in range(3):
            for J in range(b.core_lo[a], b.core_hi[a]):
                assert fb.core_lo[a] <= min(r * J, dims[a] - 1) < fb.core_hi[a]
    assert np.array_equal(S, np.eye(n))
    with pytest.raises(ValueError):
        coarse_decompose((9, 9, 9), (4, 1, 1), 4, 1)          # 3 coarse nodes cannot hold 4 parts


def test_coarse_gmres_with_one_box_is_the_exact_coarse_solve():
    """One coarse box: the coarse ORAS is E^{-1} itself, one GMRES step solves exactly."""
    from oracle.schwarz import CoarseGMRES
    prob = _prob(17, 15, 13, npml=3)
    Z = coarse_basis((17, 15, 13), 4)
    E = (Z.T @ assemble_A(prob) @ Z).tocsc()
    cg = CoarseGMRES(prob, E, (1, 1, 1), 4, overlap=1, iters=10)
    c = synth.random_complex((E.shape[0], 2), 16)
    want = spla.spsolve(E, c)
    assert np.linalg.norm(cg.solve(c) - want) <= 1e-10 * np.linalg.norm(want)


def test_coarse_gmres_finite_termination_and_monotone_residual():
    """GMRES on n coarse unknowns is exact after n steps whatever the preconditioner; with fewer
    steps the residual of E y = c decreases with the number of steps."""
    from oracle.schwarz import CoarseGMRES
    dims = (9, 9, 9)                                          # 3 x 3 x 3 coarse nodes
    prob = _prob(*dims, npml=2)
    Z = coarse_basis(dims, 4)
    E = (Z.T @ assemble_A(prob) @ Z).tocsc()
    c = synth.random_complex((E.shape[0],), 17)
    exact = CoarseGMRES(prob, E, (2, 2, 1), 4, overlap=1, iters=E.shape[0]).solve(c)
    want = spla.spsolve(E, c)
    assert np.linalg.norm(exact - want) <= 1e-9 * np.linalg.norm(want)
    dims = (29, 25, 21)
    prob = _prob(*dims, npml=4, f=5.0)
    Z = coarse_basis(dims, 4)
    E = (Z.T @ assemble_A(prob) @ Z).tocsc()
    c = synth.random_complex((E.shape[0],), 18)
    res = [np.linalg.norm(c - E @ CoarseGMRES(prob, E, (2, 2, 2), 4, overlap=1, iters=k).solve(c))
           for k in (1, 3, 10)]
    assert res[0] < np.linalg.norm(c) and res[1] < res[0] and res[2] < res[1]


def test_inexact_two_level_fgmres_reaches_direct_solution():
    """The paper's two-level method (coarse E by 10 ORAS-preconditioned GMRES steps) inside FGMRES
    converges to the direct solution; the inner iteration makes the preconditioner nonlinear, which
    FGMRES tolerates."""
    prob = _prob(20, 20, 20, npml=4, f=5.0)
    A = assemble_A(prob)
    b = synth.point_sources(20, 20, 20, 25.0, [(10, 10, 3)])[..., 0].ravel()
    xs = direct_solve_planes(prob, b)
    M = ORAS(prob, (2, 2, 2), 2, coarse_ratio=4, coarse_solve="gmres", coarse_iters=10)
    x, info = gmres(lambda v: A @ v, b, M.apply, tol=1e-8, restart=30, flexible=True)
    assert info["converged"]
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)


def test_worker_pool_local_solves_equal_the_serial_route():
    """Local solves farmed to spawned worker processes (splu in each worker) give the same preconditioner
    as the serial splu route: the same factorisations of the same local operators, up to the summation
    order of the BLAS inside SuperLU (single-threaded in the workers), so to 1e-13 relative."""
    prob = _prob(15, 13, 12)
    v = synth.random_complex((prob.n, 2), 17)
    serial = ORAS(prob, (2, 2, 2), 2, coarse_ratio=4)
    pooled = ORAS(prob, (2, 2, 2), 2, coarse_ratio=4, workers=3)
    try:
        assert len(pooled.pool.pids()) == 3
        for a, b in ((pooled.apply(v), serial.apply(v)), (pooled.apply(v[:, 0]), serial.apply(v[:, 0]))):
            assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    finally:
        pooled.close()
