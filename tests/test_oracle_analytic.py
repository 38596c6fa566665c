"""Pins of the closed-form solutions and of the discrete solution against them."""
import numpy as np
import pytest

from oracle.analytic import (green_homogeneous, green_homogeneous_dirichlet_top, green_linear_gradient,
                             node_coordinates, relative_l2_misfit, comparison_mask)
from oracle.discretization import Problem
from oracle.schwarz import direct_solve_planes
from oracle.weights import fit_weights
from paper_2103_14921_gb300 import synth


def _laplacian_fd(f, x, y, z, s):
    return (f(x + s, y, z) + f(x - s, y, z) + f(x, y + s, z) + f(x, y - s, z) + f(x, y, z + s)
            + f(x, y, z - s) - 6 * f(x, y, z)) / s ** 2


def test_linear_gradient_green_solves_the_pde():
    """``(Delta + omega^2/c(z)^2) G = 0`` away from the source (fine-step finite differences)."""
    c0, alpha, omega = 1000.0, 0.8, 2 * np.pi * 3.0
    src = (0.0, 0.0, 500.0)
    G = lambda x, y, z: green_linear_gradient(x, y, z, src, omega, c0, alpha)
    rng = np.random.default_rng(1)
    for _ in range(6):
        p = rng.uniform([-600, -600, 100], [600, 600, 1500])
        s = 0.5
        k2 = (omega / (c0 + alpha * p[2])) ** 2
        res = _laplacian_fd(G, *p, s) + k2 * G(*p)
        scale = k2 * abs(G(*p))
        assert abs(res) < 1e-4 * scale


def test_linear_gradient_green_limits():
    c0, omega = 1500.0, 2 * np.pi * 4.0
    src = (100.0, 200.0, 700.0)
    # near the source it behaves like 1/(4 pi r)
    r = 0.01
    g = green_linear_gradient(src[0] + r, src[1], src[2], src, omega, c0, 0.6)
    assert abs(4 * np.pi * r * g - 1) < 1e-3
    # alpha -> 0 recovers exp(ikr)/(4 pi r) with k = omega/c(z_s)
    x, y, z = 400.0, -100.0, 900.0
    cz = c0 + 1e-6 * src[2]
    g0 = green_homogeneous(x, y, z, src, omega / cz)
    g1 = green_linear_gradient(x, y, z, src, omega, c0, 1e-6)
    assert abs(g1 - g0) < 1e-5 * abs(g0)


def _solve_point(prob, s):
    b = synth.point_sources(prob.nx, prob.ny, prob.nz, prob.h, [s])[..., 0]
    return direct_solve_planes(prob, b.ravel()).reshape(prob.shape)


@pytest.fixture(scope="module")
def weights():
    return fit_weights()


def test_homogeneous_pml_all_sides_matches_free_space(weights):
    n, h, f, c0 = 32, 25.0, 6.0, 1500.0             # 10 points per wavelength
    prob = Problem(n, n, n, h, f, synth.homogeneous(n, n, n, c0), npml=8, top_pml=True, weights=weights)
    s = (16, 16, 16)
    u = _solve_point(prob, s)
    X, Y, Z = node_coordinates(n, n, n, h)
    G = green_homogeneous(X, Y, Z, (s[0] * h, s[1] * h, (s[2] + 1) * h), 2 * np.pi * f / c0)
    mask = comparison_mask(n, n, n, 8, True, s, 4)
    assert relative_l2_misfit(u, -G, mask) < 0.05
    # the 7-point stencil at the same sampling is far less accurate (pins the weights' use)
    prob7 = Problem(n, n, n, h, f, synth.homogeneous(n, n, n, c0), npml=8, top_pml=True)
    u7 = _solve_point(prob7, s)
    mis, mis7 = relative_l2_misfit(u, -G, mask), relative_l2_misfit(u7, -G, mask)
    assert mis7 > 0.05 and mis7 > 1.5 * mis


def test_homogeneous_dirichlet_top_matches_image_source(weights):
    n, h, f, c0 = 32, 25.0, 6.0, 1500.0
    prob = Problem(n, n, n, h, f, synth.homogeneous(n, n, n, c0), npml=8, top_pml=False, weights=weights)
    s = (16, 16, 6)
    u = _solve_point(prob, s)
    X, Y, Z = node_coordinates(n, n, n, h)
    G = green_homogeneous_dirichlet_top(X, Y, Z, (s[0] * h, s[1] * h, (s[2] + 1) * h), 2 * np.pi * f / c0)
    mask = comparison_mask(n, n, n, 8, False, s, 4)
    assert relative_l2_misfit(u, -G, mask) < 0.05


def test_linear_gradient_matches_closed_form(weights):
    """The paper's validation medium, c(z) = c0 + alpha z, PML top (whole-space solution)."""
    n, h, f, c0, alpha = 32, 25.0, 5.0, 1500.0, 0.6     # 12..16 points per wavelength
    c = synth.linear_gradient(n, n, n, h, c0, alpha)
    prob = Problem(n, n, n, h, f, c, npml=8, top_pml=True, weights=weights)
    s = (16, 16, 16)
    u = _solve_point(prob, s)
    X, Y, Z = node_coordinates(n, n, n, h)
    G = green_linear_gradient(X, Y, Z, (s[0] * h, s[1] * h, (s[2] + 1) * h), 2 * np.pi * f, c0, alpha)
    mask = comparison_mask(n, n, n, 8, True, s, 4)
    mis = relative_l2_misfit(u, -G, mask)
    assert mis < 0.05
    # a homogeneous Green's function with the source velocity is clearly worse: the gradient matters
    Gh = green_homogeneous(X, Y, Z, (s[0] * h, s[1] * h, (s[2] + 1) * h), 2 * np.pi * f / (c0 + alpha * (s[2] + 1) * h))
    assert relative_l2_misfit(u, -Gh, mask) > 1.5 * mis
