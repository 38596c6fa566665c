"""Pins of the oracle's GMRES / FGMRES."""
import numpy as np
import pytest

from oracle.krylov import gmres, gmres_multi, givens, arnoldi_record
from paper_2103_14921_gb300 import synth


def _rand_matrix(n, seed, shift=0.0):
    M = synth.random_complex((n, n), seed) / np.sqrt(n)
    return M + shift * np.eye(n)


def test_givens_is_unitary_and_zeroes():
    rng = np.random.default_rng(0)
    for a, b in [(1 + 2j, 3 - 1j), (0, 2j), (1.5, 0), (-2j, 1e-9)]:
        c, s = givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        assert np.allclose(G @ G.conj().T, np.eye(2))
        out = G @ np.array([a, b])
        assert abs(out[1]) < 1e-14 * max(abs(a), abs(b))
        assert np.isclose(abs(out[0]), np.hypot(abs(a), abs(b)))


@pytest.mark.parametrize("flexible", [True, False])
def test_full_gmres_converges_in_at_most_n_steps(flexible):
    for n in (5, 17, 27):
        A = _rand_matrix(n, n)
        b = synth.random_complex((n,), n + 100)
        x, info = gmres(lambda v: A @ v, b, tol=1e-12, restart=n, flexible=flexible)
        assert info["iterations"] <= n
        assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-8, atol=1e-8 * np.linalg.norm(x))


def test_residual_estimate_monotone_and_matches_true_residual():
    n = 60
    A = _rand_matrix(n, 3, shift=2.0)
    b = synth.random_complex((n,), 4)
    x, info = gmres(lambda v: A @ v, b, tol=1e-10, restart=40)
    est = np.array(info["estimates"])
    assert np.all(np.diff(est) <= 1e-15)
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(true - info["true_residual"]) < 1e-14
    assert true <= 1e-10 * 10
    assert abs(est[-1] - true) < 1e-9


def test_arnoldi_relation_and_orthonormality():
    n, m = 40, 12
    A = _rand_matrix(n, 5, shift=1.0)
    Minv = np.diag(1.0 / (1.0 + np.arange(n) / n))
    b = synth.random_complex((n,), 6)
    V, Z, H = arnoldi_record(lambda v: A @ v, b, lambda v: Minv @ v, m)
    assert np.allclose(V.conj() @ V.T, np.eye(m + 1), atol=1e-12)
    assert np.allclose(A @ Z.T, V.T @ H, atol=1e-12)


def test_restarted_and_flexible_agree_with_direct_solve():
    n = 80
    A = _rand_matrix(n, 7, shift=3.0)
    Minv = np.linalg.inv(A + 0.3 * _rand_matrix(n, 8))
    B = synth.random_complex((n, 3), 9)
    X, infos = gmres_multi(lambda v: A @ v, B, lambda v: Minv @ v, tol=1e-9, restart=5)
    assert all(i["converged"] for i in infos)
    assert np.allclose(X, np.linalg.solve(A, B), rtol=0, atol=1e-7 * np.abs(X).max())
    assert all(i["cycles"] >= 1 for i in infos)


def test_zero_rhs_gives_zero():
    x, info = gmres(lambda v: v, np.zeros(4, complex))
    assert np.all(x == 0) and info["iterations"] == 0


def test_initial_guess():
    """From x0 = the solution: no iteration, x0 returned; from a restarted iterate: the method continues the
    same solve (one restart cycle of GMRES(m) from x_m is the next cycle of the restarted run); b = 0 gives
    x = 0 whatever x0."""
    n = 60
    A = _rand_matrix(n, 21, shift=2.5)
    b = synth.random_complex((n,), 22)
    xs = np.linalg.solve(A, b)
    x, info = gmres(lambda v: A @ v, b, tol=1e-10, restart=10, x0=xs)
    assert info["iterations"] == 0 and np.array_equal(x, xs)
    x1, i1 = gmres(lambda v: A @ v, b, tol=1e-14, restart=8, maxit=8)          # one cycle, not converged
    x2, i2 = gmres(lambda v: A @ v, b, tol=1e-14, restart=8, maxit=8, x0=x1)   # the second cycle
    x12, i12 = gmres(lambda v: A @ v, b, tol=1e-14, restart=8, maxit=16)       # both cycles at once
    assert np.allclose(x2, x12, rtol=0, atol=1e-12 * np.linalg.norm(x12))
    assert np.isclose(i2["true_residual"], i12["true_residual"], rtol=1e-6)
    x0, _ = gmres(lambda v: A @ v, np.zeros(n, complex), x0=xs)
    assert not np.any(x0)
