"""Right-preconditioned restarted GMRES and flexible GMRES (FP64, complex).

Test infrastructure only (see ``oracle/__init__.py``).

The paper solves Eq. (eq1) with GMRES (Saad 2003) preconditioned by Eq. (2lvl)
(section "Domain decomposition preconditioner"); because its coarse solve is
itself an inner iteration the preconditioner varies, which calls for the
flexible variant.  Readings taken where the paper is silent:

* Right preconditioning; the tolerance applies to the unpreconditioned
  relative residual ``||b - A x||_2 / ||b||_2``.
* Independent Krylov spaces per right-hand side (no block GMRES); ``x0 = 0``.
* Modified Gram-Schmidt Arnoldi, complex Givens rotations with real cosine,
  stop when ``|g_{j+1}| / ||b|| <= tol``; at the end of each cycle the true
  residual is recomputed and the method restarts when it is above ``tol``.
* ``||b|| = 0`` gives ``x = 0``.

GMRES keeps only ``V`` and forms ``x += M^{-1} (V y)``; FGMRES keeps
``Z_j = M^{-1} v_j`` and forms ``x += Z y``.  Pinned by: full GMRES on n
unknowns converges in at most n steps to ``numpy.linalg.solve``; the
residual estimate is monotone in a cycle; the Arnoldi relation and
orthonormality hold; estimate and true residual agree.
"""
from __future__ import annotations

import numpy as np


def givens(a: complex, b: complex):
    """Rotation ``[[c, s], [-conj(s), c]]`` (c real) that zeroes ``b`` under ``a``."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    return abs(a) / t, (a / abs(a)) * np.conj(b) / t


def gmres(apply_A, b, apply_M=None, tol=1e-6, restart=30, maxit=1000, flexible=True, record=None, x0=None):
    """Solve ``A x = b`` for one right-hand side ``b`` (complex vector), from ``x0`` (zero by default;
    ``b = 0`` gives ``x = 0`` whatever ``x0``).

    Returns ``(x, info)``; ``info`` holds ``iterations``, ``converged``,
    ``estimates`` (relative residual estimate after each iteration) and
    ``true_residual`` (relative, at exit).  When ``record`` is a dict, the
    last cycle's ``V``, ``Z`` and ``H`` are stored in it.
    """
    b = np.asarray(b, dtype=np.complex128)
    if apply_M is None:
        apply_M = lambda v: v
    n = b.size
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, dtype=np.complex128)
    info = {"iterations": 0, "converged": True, "estimates": [], "true_residual": 0.0, "cycles": 0}
    if bnorm == 0.0:
        return x, info
    total = 0
    r = b.copy()
    if x0 is not None:
        x = np.array(x0, dtype=np.complex128)
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            info.update(true_residual=float(rel))
            return x, info
    while True:
        info["cycles"] += 1
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        Zs = np.zeros((restart, n), dtype=np.complex128) if flexible else None
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            z = apply_M(V[j])
            if flexible:
                Zs[j] = z
            w = apply_A(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            est = abs(g[j + 1]) / bnorm
            info["estimates"].append(est)
            if est <= tol or total >= maxit:
                break
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:j_done]) / H[i, i]
        if flexible:
            x = x + y @ Zs[:j_done]
        else:
            x = x + apply_M(y @ V[:j_done])
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        if record is not None:
            record.update(V=V[:j_done + 1], Z=None if Zs is None else Zs[:j_done], H=H, j=j_done)
        if rel <= tol or total >= maxit:
            info.update(iterations=total, converged=bool(rel <= tol), true_residual=float(rel))
            return x, info


def gmres_multi(apply_A, B, apply_M=None, **kw):
    """Independent GMRES per column of ``B`` (``[N, nrhs]``); returns ``(X, infos)``."""
    B = np.asarray(B, dtype=np.complex128)
    X = np.zeros_like(B)
    infos = []
    for r in range(B.shape[1]):
        X[:, r], inf = gmres(apply_A, B[:, r], apply_M, **kw)
        infos.append(inf)
    return X, infos


def arnoldi_record(apply_A, b, apply_M, steps):
    """Run ``steps`` flexible Arnoldi steps without rotations; returns ``(V, Z, Hbar)``.

    Used to pin the Arnoldi relation ``A Z_m = V_{m+1} Hbar_m``.
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    V = np.zeros((steps + 1, n), dtype=np.complex128)
    Zs = np.zeros((steps, n), dtype=np.complex128)
    H = np.zeros((steps + 1, steps), dtype=np.complex128)
    V[0] = b / np.linalg.norm(b)
    for j in range(steps):
        Zs[j] = apply_M(V[j])
        w = apply_A(Zs[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    return V, Zs, H
