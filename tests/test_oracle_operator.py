"""Pins of the oracle's discretisation (Eq. eq1, the 27-point mixed-grid stencil)."""
import numpy as np
import scipy.sparse as sp
import pytest

from oracle.discretization import (Problem, WEIGHTS_7PT, apply_A, assemble_A, neighbour_coefficients, symbol,
                                   stencil_coefficients, pml_xi)
from oracle.weights import fit_weights, dispersion_residuals, phase_velocity_ratio
from paper_2103_14921_gb300 import synth


def _prob(n=(9, 8, 7), weights=WEIGHTS_7PT, npml=0, c=None, top_pml=False, f=5.0, h=25.0):
    nx, ny, nz = n
    if c is None:
        c = synth.homogeneous(nx, ny, nz, 1500.0)
    return Problem(nx, ny, nz, h, f, c, npml=npml, top_pml=top_pml, weights=weights)


def test_seven_point_equals_textbook_laplacian():
    """w1 = 1, wm1 = 1 without PML: the Kronecker-sum Laplacian plus diag(k^2)."""
    nx, ny, nz = 9, 8, 7
    c = synth.linear_gradient(nx, ny, nz, 25.0) * (1 - 0.01j)
    prob = _prob((nx, ny, nz), c=c)
    h = prob.h

    def lap1(n):
        return sp.diags([np.ones(n - 1), -2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / h ** 2

    I = lambda n: sp.identity(n)
    L = (sp.kron(I(nz), sp.kron(I(ny), lap1(nx))) + sp.kron(I(nz), sp.kron(lap1(ny), I(nx)))
         + sp.kron(lap1(nz), sp.kron(I(ny), I(nx))))
    A_text = (L + sp.diags(prob.k2().ravel())).toarray()
    A = assemble_A(prob).toarray()
    assert np.allclose(A, A_text, rtol=0, atol=1e-14 * np.abs(A_text).max())
    u = synth.random_complex((nz, ny, nx), 4)
    assert np.allclose(apply_A(prob, u).ravel(), A_text @ u.ravel(), rtol=1e-13, atol=0)


def test_rotated_system_form_equals_product_form():
    """Interior rows: the stencil written per rotated coordinate system (Operto et al. form)."""
    w = synth.random_weights(11)
    w1, w2, w3, wm1, wm2, wm3, wm4 = w
    nx, ny, nz = 8, 7, 6
    c = synth.linear_gradient(nx, ny, nz, 25.0, c0=1500.0, alpha=3.0) * (1 - 0.02j)
    prob = _prob((nx, ny, nz), weights=w, c=c)
    u = synth.random_complex((nz, ny, nx), 5)
    k2 = prob.k2()
    h = prob.h
    got = apply_A(prob, u)
    upad = np.pad(u, 1)
    wpad = np.pad(k2 * u, 1)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                F = E = C = 0
                Fw = Ew = Cw = 0
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            nnz = abs(dx) + abs(dy) + abs(dz)
                            v = upad[k + 1 + dz, j + 1 + dy, i + 1 + dx]
                            vw = wpad[k + 1 + dz, j + 1 + dy, i + 1 + dx]
                            if nnz == 1:
                                F += v; Fw += vw
                            elif nnz == 2:
                                E += v; Ew += vw
                            elif nnz == 3:
                                C += v; Cw += vw
                u0 = u[k, j, i]
                lap = (w1 * (F - 6 * u0) + (w2 / 3) * ((F - 6 * u0) + (E - 12 * u0) / 2)
                       + w3 * (C - 8 * u0) / 4) / h ** 2
                mass = wm1 * k2[k, j, i] * u0 + wm2 * Fw + wm3 * Ew + wm4 * Cw
                assert abs(got[k, j, i] - (lap + mass)) <= 1e-12 * (abs(lap) + abs(mass))


def test_plane_wave_symbol_interior():
    """``A exp(i kappa.x) = A_hat(kappa) exp(i kappa.x)`` on interior unstretched nodes."""
    w = fit_weights()
    prob = _prob((10, 9, 8), weights=w)
    k2 = complex(prob.k2()[0, 0, 0])
    rng = np.random.default_rng(7)
    for _ in range(5):
        kappa = rng.uniform(-np.pi / prob.h, np.pi / prob.h, 3)
        k, j, i = np.meshgrid(np.arange(8), np.arange(9), np.arange(10), indexing="ij")
        u = np.exp(1j * (kappa[0] * i * prob.h + kappa[1] * j * prob.h + kappa[2] * (k + 1) * prob.h))
        got = apply_A(prob, u)[1:-1, 1:-1, 1:-1]
        want = symbol(prob, kappa, k2) * u[1:-1, 1:-1, 1:-1]
        assert np.allclose(got, want, rtol=1e-11, atol=1e-11 * np.abs(want).max())


def test_assembled_equals_matrix_free_with_pml_and_attenuation():
    nx, ny, nz = 14, 13, 12
    c = synth.linear_gradient(nx, ny, nz, 25.0, Q=50.0)
    for top in (False, True):
        prob = _prob((nx, ny, nz), weights=synth.random_weights(2), npml=4, c=c, top_pml=top)
        A = assemble_A(prob)
        U = synth.random_complex((nz, ny, nx, 3), 6)
        got = apply_A(prob, U).reshape(-1, 3)
        want = A @ U.reshape(-1, 3)
        assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.norm(want)
        # 27 nonzeros per interior row
        assert A.getnnz(axis=1).max() == 27


def test_neighbour_coefficients_zero_at_ghosts_and_dirichlet_top():
    prob = _prob((6, 5, 4), weights=synth.random_weights(3), npml=2)
    coef = neighbour_coefficients(prob)
    assert np.all(coef[0, :, :, 0] == 0)       # no coupling to the Dirichlet ghost plane
    assert np.all(coef[:, :, 2, :, :, -1] == 0)
    assert np.abs(coef[1, 1, 1]).min() > 0


def test_pml_stretching_profile():
    """xi = 1 inside, 1 + i gamma0 (d/L)^2 / omega in the layers, symmetric, growing outwards."""
    n, h, npml, omega, cref, R = 30, 25.0, 8, 2 * np.pi * 5, 2000.0, 1e-3
    xn, xh = pml_xi(n, h, npml, True, True, omega, cref, R)
    L = npml * h
    g0 = 1.5 * cref / L * np.log(1 / R)
    assert np.allclose(xn[npml:n - npml], 1.0)
    assert np.isclose(xn[0], 1 + 1j * g0 / omega)            # d = L at the outermost node
    assert np.allclose(xn, xn[::-1])
    assert np.allclose(xh, xh[::-1])
    assert np.all(np.diff(xn[:npml + 1].imag) < 0)
    # no high layer requested -> no stretch there
    xn2, _ = pml_xi(n, h, npml, False, True, omega, cref, R)
    assert np.allclose(xn2[:n - npml], 1.0)


def test_fitted_weights_reduce_dispersion():
    """The fitted stencil keeps |1 - v_ph/c| small over 4..30 points per wavelength."""
    w = fit_weights()
    assert abs(sum(w[:3]) - 1) < 1e-12
    assert abs(w[3] + 6 * w[4] + 12 * w[5] + 8 * w[6] - 1) < 1e-12
    assert min(w) >= 0
    err_fit = np.abs(dispersion_residuals(w)).max()
    err_7 = np.abs(dispersion_residuals(WEIGHTS_7PT)).max()
    assert err_fit < 0.006
    assert err_7 > 0.05
    # consistency: v_ph / c -> 1 for well-resolved waves in any direction
    for d in [(1, 0, 0), (0.6, 0.8, 0), (0.48, 0.6, 0.64)]:
        assert abs(1 - phase_velocity_ratio(w, 200.0, d)) < 1e-4


def test_stencil_coefficient_identities():
    # the mass weights summing to one give m0 = 1
    w = synth.random_weights(9)
    a2, a3, m0, m1, m2, m3 = stencil_coefficients(w)
    assert abs(m0 - 1) < 1e-12
    assert a2 >= 0 and a3 >= 0


def test_interior_row_depends_only_on_the_neighbour_class():
    """Away from the absorbing layers the expanded 27-point row (Eq. eq1 in the product form of reading 2) gives
    every neighbour a coefficient that depends only on its class (centre, face, edge, corner): the mass part is
    exactly the paper's per-neighbour mass weight wm1..wm4 times k^2, and the Laplacian part is a consistent
    second-order Laplacian whatever the weights -- zero on constants, exactly 2 on x^2 (and on y^2, z^2), zero
    on xy -- with class values (-6 + 12 a2 - 8 a3, 1 - 4 a2 + 4 a3, a2 - 2 a3, a3) / h^2."""
    w = synth.random_weights(31)
    h = 25.0
    rows = []
    for f in (3.0, 7.0):
        prob = _prob(n=(7, 7, 7), weights=w, npml=0, f=f, h=h)
        rows.append((neighbour_coefficients(prob)[:, :, :, 3, 3, 3], prob.k2()[3, 3, 3]))
    (c1, k1), (c2, k2) = rows
    mass = (c1 - c2) / (k1 - k2)
    lap = c1 - mass * k1
    off = np.array([-1, 0, 1])
    dz, dy, dx = np.meshgrid(off, off, off, indexing="ij")
    cls = np.abs(dx) + np.abs(dy) + np.abs(dz)
    a2, a3 = stencil_coefficients(w)[:2]
    want_lap = np.array([-6 + 12 * a2 - 8 * a3, 1 - 4 * a2 + 4 * a3, a2 - 2 * a3, a3]) / h ** 2
    want_mass = np.array(w[3:7])
    for c in range(4):
        assert np.allclose(mass[cls == c], want_mass[c], rtol=1e-12, atol=1e-15)
        assert np.allclose(lap[cls == c], want_lap[c], rtol=1e-12, atol=1e-18)
    # consistency of the Laplacian part, independently of the class formula
    assert abs(lap.sum()) * h ** 2 < 1e-12
    for d in (dx, dy, dz):
        assert abs((lap * d ** 2).sum() * h ** 2 - 2.0) < 1e-12
    assert abs((lap * dx * dy).sum()) * h ** 2 < 1e-12
    assert abs(mass.sum() - 1.0) < 1e-12     # the mass weights of one row sum to one


# --- adaptive stencil weights (each row with the weights matched to its own points per wavelength) ---

def test_row_weights_rows_equal_their_constant_weight_rows():
    """Row p of the adaptive operator is row p of the constant-weight operator built with p's weights
    (so per-row weights act on the right rows and nothing mixes across rows); matrix-free = assembled."""
    nx, ny, nz = 9, 8, 7
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 3.0, Q=80.0)
    sets = [synth.random_weights(s) for s in (31, 32, 33)]
    rng = np.random.default_rng(4)
    pick = rng.integers(0, 3, size=(nz, ny, nx))
    rw = np.array(sets)[pick]
    prob = Problem(nx, ny, nz, 25.0, 5.0, c, npml=2, weights=sets[0], row_weights=rw)
    A = assemble_A(prob).toarray()
    for q in range(3):
        Aq = assemble_A(Problem(nx, ny, nz, 25.0, 5.0, c, npml=2, weights=sets[q])).toarray()
        rows = np.flatnonzero(pick.ravel() == q)
        assert np.allclose(A[rows], Aq[rows], rtol=0, atol=1e-12 * np.abs(Aq).max())
    u = synth.random_complex((nz, ny, nx, 2), 5)
    Au = apply_A(prob, u)
    want = (A @ u.reshape(-1, 2)).reshape(u.shape)
    assert np.linalg.norm(Au - want) <= 1e-12 * np.linalg.norm(want)


def test_one_bin_of_row_weights_is_the_constant_stencil():
    nx, ny, nz = 8, 7, 6
    c = synth.linear_gradient(nx, ny, nz, 25.0)
    w = synth.random_weights(34)
    rw = np.broadcast_to(np.array(w), (nz, ny, nx, 7))
    u = synth.random_complex((nz, ny, nx), 6)
    a = apply_A(Problem(nx, ny, nz, 25.0, 5.0, c, npml=2, weights=w, row_weights=rw), u)
    b = apply_A(Problem(nx, ny, nz, 25.0, 5.0, c, npml=2, weights=w), u)
    assert np.array_equal(a, b)


def test_adaptive_bins_cover_the_model_and_beat_the_broadband_fit_in_their_range():
    from oracle.weights import adaptive_bin_edges, row_weight_bins, adaptive_row_weights
    c = synth.linear_gradient(10, 9, 24, 25.0, 1000.0, 2.0)
    f, h = 8.0, 25.0
    G = np.real(c) / (f * h)
    edges = adaptive_bin_edges(G.min(), G.max(), 4)
    assert np.isclose(edges[0], G.min()) and np.isclose(edges[-1], G.max())
    bins = row_weight_bins(c, f, h, edges)
    assert bins.min() == 0 and bins.max() == 3
    for b in range(4):                           # every node lies in its bin's interval
        g = G[bins == b]
        assert g.min() >= edges[b] * (1 - 1e-12) and g.max() <= edges[b + 1] * (1 + 1e-12)
    table, bins2, rw = adaptive_row_weights(c, f, h, 4)
    assert np.array_equal(bins, bins2) and np.array_equal(rw, table[bins])
    broad = fit_weights()
    for b in range(4):
        Gs = 1.0 / np.linspace(1.0 / edges[b + 1], 1.0 / edges[b], 8)
        err_bin = np.abs(dispersion_residuals(tuple(table[b]), Gs)).max()
        err_broad = np.abs(dispersion_residuals(broad, Gs)).max()
        assert err_bin < err_broad


def test_adaptive_weights_are_closer_to_the_linear_gradient_closed_form():
    """In the paper's validation medium the row-adapted stencil is more accurate than the broadband one
    against the closed-form solution (the purpose the paper gives for adaptive coefficients)."""
    from oracle.analytic import green_linear_gradient, node_coordinates, relative_l2_misfit, comparison_mask
    from oracle.schwarz import direct_solve_planes
    from oracle.weights import adaptive_row_weights
    n, h, f, c0, alpha = 32, 25.0, 5.0, 1500.0, 0.6
    c = synth.linear_gradient(n, n, n, h, c0, alpha)
    s = (16, 16, 16)
    X, Y, Z = node_coordinates(n, n, n, h)
    G = green_linear_gradient(X, Y, Z, (s[0] * h, s[1] * h, (s[2] + 1) * h), 2 * np.pi * f, c0, alpha)
    mask = comparison_mask(n, n, n, 8, True, s, 4)
    b = synth.point_sources(n, n, n, h, [s])[..., 0].ravel()
    w = fit_weights()
    _, _, rw = adaptive_row_weights(c, f, h, 4)
    mis = []
    for row_weights in (None, rw):
        prob = Problem(n, n, n, h, f, c, npml=8, top_pml=True, weights=w, row_weights=row_weights)
        mis.append(relative_l2_misfit(direct_solve_planes(prob, b).reshape(prob.shape), -G, mask))
    assert mis[1] < mis[0] < 0.05
