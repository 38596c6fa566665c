"""Two-level ORAS preconditioner (Eq. 2lvl, Eq. oras) in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

What the paper fixes (section "Domain decomposition preconditioner"):

* ``M1^{-1} = sum_i R_i^T D_i A_i^{-1} R_i`` (Eq. oras) over an overlapping
  decomposition, ``R_i`` Boolean restrictions, ``D_i`` diagonal partition of
  unity, ``A_i`` local Helmholtz operators with absorbing conditions on the
  subdomain interfaces (the "optimized" in ORAS; RAS uses Dirichlet).
* ``M^{-1} = M1^{-1} (I - A Q) + Q``, ``Q = Z E^{-1} Z^T``, ``E = Z^T A Z``
  (Eq. 2lvl), ``Z^T`` the interpolation from the fine space to a coarse space.
* Local problems are solved exactly by a direct solver.

Readings taken where the paper is silent:

* Box subdomains on the grid: axis ``a`` is cut into ``p_a`` cores at
  ``floor(t n_a / p_a)``; each box is its core grown by ``overlap`` nodes on
  every side that is not a global face.
* ``D_i`` is the Boolean owner partition of unity: 1 on the core, 0 on the
  overlap, so ``sum_i R_i^T D_i R_i = I``.
* Absorbing interface condition: a stencil neighbour ``q`` of row ``p`` that
  lies outside the box across an interface face is replaced by the clamped
  in-box node times ``rho_p = exp(i k_p h)`` per crossed face, ``k_p`` at the
  row node.  This is exact for waves ``exp(i k |x_a - x_mid|)`` leaving the
  box along each axis; the tests pin it by that identity.  ``mode="ras"``
  drops those neighbours instead (Dirichlet).
* Coarse space: nodes at fine indices ``r J_a``, ``J_a = 0..ceil((n_a-1)/r)``,
  trilinear hats ``Z[i, J] = prod_a max(0, 1 - |i_a - r J_a| / r)``; ``E`` is
  solved exactly (``coarse_solve="exact"``), or as in the paper by 10 GMRES
  iterations preconditioned by one-level ORAS on the coarse grid over the same
  spatial partition (``coarse_solve="gmres"``, :class:`CoarseGMRES`).

Local solves have two independent routes: ``scipy.sparse.linalg.splu`` (the
paper's sparse direct solver) and the plane-by-plane block-tridiagonal LU
with dense Schur-complement inverses
``S_0 = D_0, S_k = D_k - L_k S_{k-1}^{-1} U_{k-1}`` and the sweeps
``y_k = S_k^{-1}(b_k - L_k y_{k-1})``, ``x_k = y_k - S_k^{-1} U_k x_{k+1}``.
Pinned against ``numpy.linalg.solve`` of the dense ``A_i``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .discretization import Problem, neighbour_coefficients, assemble_A


@dataclass
class Box:
    """One subdomain; all triples are in (x, y, z) order, half-open ranges."""

    core_lo: tuple
    core_hi: tuple
    lo: tuple
    hi: tuple

    @property
    def dims(self):
        return tuple(self.hi[a] - self.lo[a] for a in range(3))

    @property
    def size(self):
        d = self.dims
        return d[0] * d[1] * d[2]


def decompose(dims, parts, overlap):
    """Box decomposition of a grid ``dims = (nx, ny, nz)`` into ``parts = (px, py, pz)``."""
    cuts = [[(t * dims[a]) // parts[a] for t in range(parts[a] + 1)] for a in range(3)]
    boxes = []
    for tz in range(parts[2]):
        for ty in range(parts[1]):
            for tx in range(parts[0]):
                t = (tx, ty, tz)
                clo = tuple(cuts[a][t[a]] for a in range(3))
                chi = tuple(cuts[a][t[a] + 1] for a in range(3))
                lo = tuple(max(0, clo[a] - overlap) if clo[a] > 0 else 0 for a in range(3))
                hi = tuple(min(dims[a], chi[a] + overlap) if chi[a] < dims[a] else dims[a] for a in range(3))
                boxes.append(Box(clo, chi, lo, hi))
    return boxes


def box_global_indices(box: Box, dims):
    """Global flat indices of the box nodes, local order ``(k, j, i)`` with i fastest."""
    nx, ny, _ = dims
    k, j, i = np.meshgrid(np.arange(box.lo[2], box.hi[2]), np.arange(box.lo[1], box.hi[1]),
                          np.arange(box.lo[0], box.hi[0]), indexing="ij")
    return ((k * ny + j) * nx + i).ravel()


def restriction(box: Box, dims) -> sp.csr_matrix:
    """Boolean ``R_i`` (local size x global size)."""
    g = box_global_indices(box, dims)
    n = dims[0] * dims[1] * dims[2]
    return sp.csr_matrix((np.ones(g.size), (np.arange(g.size), g)), shape=(g.size, n))


def partition_of_unity(box: Box) -> np.ndarray:
    """Boolean owner weights ``diag(D_i)``: 1 on core nodes, 0 on overlap nodes."""
    k, j, i = np.meshgrid(np.arange(box.lo[2], box.hi[2]), np.arange(box.lo[1], box.hi[1]),
                          np.arange(box.lo[0], box.hi[0]), indexing="ij")
    own = ((i >= box.core_lo[0]) & (i < box.core_hi[0]) & (j >= box.core_lo[1]) & (j < box.core_hi[1])
           & (k >= box.core_lo[2]) & (k < box.core_hi[2]))
    return own.ravel().astype(np.float64)


def local_operator(prob: Problem, box: Box, mode: str = "oras", coef=None) -> sp.csr_matrix:
    """``A_i``: the rows of A for the box nodes with absorbing (or Dirichlet) interface folding."""
    if coef is None:
        coef = neighbour_coefficients(prob)
    rho = np.exp(1j * (prob.omega / np.asarray(prob.c, dtype=np.complex128)) * prob.h)
    return fold_operator(coef, rho, box, mode)


def fold_operator(coef, rho, box: Box, mode: str = "oras") -> sp.csr_matrix:
    """Rows of a 27-point grid operator (coefficients ``coef[3, 3, 3, nz, ny, nx]``) for the box nodes,
    a neighbour outside the box folded onto the clamped in-box node times ``rho`` of the row node per
    crossed face (``mode="oras"``) or dropped (``mode="ras"``).  ``rho`` is ``[nz, ny, nx]``."""
    bx, by, bz = box.dims
    k, j, i = np.meshgrid(np.arange(bz), np.arange(by), np.arange(bx), indexing="ij")
    gi, gj, gk = i + box.lo[0], j + box.lo[1], k + box.lo[2]
    rho = np.asarray(rho)[gk, gj, gi]
    row = ((k * by + j) * bx + i)
    rows, cols, vals = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                c = coef[dz + 1, dy + 1, dx + 1][gk, gj, gi]
                qi, qj, qk = i + dx, j + dy, k + dz
                crossed = ((qi < 0) | (qi >= bx)).astype(int) + ((qj < 0) | (qj >= by)).astype(int) \
                    + ((qk < 0) | (qk >= bz)).astype(int)
                # neighbours outside the global grid already carry a zero coefficient
                ci, cj, ck = np.clip(qi, 0, bx - 1), np.clip(qj, 0, by - 1), np.clip(qk, 0, bz - 1)
                if mode == "oras":
                    v = c * rho ** crossed
                elif mode == "ras":
                    v = np.where(crossed > 0, 0.0, c)
                else:
                    raise ValueError(mode)
                rows.append(row.ravel())
                cols.append(((ck * by + cj) * bx + ci).ravel())
                vals.append(v.ravel())
    n = bx * by * bz
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.eliminate_zeros()
    return A


# ---------------------------------------------------------------------------
# Plane-by-plane block-tridiagonal LU (second route for the local solves)
# ---------------------------------------------------------------------------

def plane_blocks(Ai: sp.spmatrix, m: int, nplanes: int):
    """Dense ``(D_k, L_k, U_k)`` of a local operator ordered plane by plane."""
    A = Ai.tocsr()
    D, L, U = [], [], []
    for kk in range(nplanes):
        s = slice(kk * m, (kk + 1) * m)
        D.append(A[s, s].toarray())
        L.append(A[s, (kk - 1) * m:kk * m].toarray() if kk > 0 else None)
        U.append(A[s, (kk + 1) * m:(kk + 2) * m].toarray() if kk < nplanes - 1 else None)
    return D, L, U


def plane_factor(D, L, U):
    """Dense Schur-complement inverses ``G_k = S_k^{-1}``."""
    G = []
    for kk in range(len(D)):
        S = D[kk] if kk == 0 else D[kk] - L[kk] @ G[kk - 1] @ U[kk - 1]
        G.append(np.linalg.inv(S))
    return G


def plane_solve(G, L, U, b):
    """Forward and backward plane sweeps; ``b`` is ``[nplanes*m]`` or ``[nplanes*m, nrhs]``."""
    nplanes = len(G)
    m = G[0].shape[0]
    bb = b.reshape((nplanes, m) + b.shape[1:])
    y = np.empty_like(bb, dtype=np.complex128)
    for kk in range(nplanes):
        rhs = bb[kk] if kk == 0 else bb[kk] - L[kk] @ y[kk - 1]
        y[kk] = G[kk] @ rhs
    x = np.empty_like(y)
    x[-1] = y[-1]
    for kk in range(nplanes - 2, -1, -1):
        x[kk] = y[kk] - G[kk] @ (U[kk] @ x[kk + 1])
    return x.reshape(b.shape)


# ---------------------------------------------------------------------------
# Coarse space
# ---------------------------------------------------------------------------

def coarse_dims(dims, r):
    return tuple(-(-(dims[a] - 1) // r) + 1 for a in range(3))


def hat_1d(n: int, r: int) -> sp.csr_matrix:
    nc = -(-(n - 1) // r) + 1
    i = np.arange(n)[:, None]
    J = np.arange(nc)[None, :]
    w = np.maximum(0.0, 1.0 - np.abs(i - r * J) / r)
    return sp.csr_matrix(w)


def coarse_basis(dims, r) -> sp.csr_matrix:
    """``Z`` (fine size x coarse size), trilinear hats; index ``(k*ny + j)*nx + i`` on both grids."""
    Zx, Zy, Zz = hat_1d(dims[0], r), hat_1d(dims[1], r), hat_1d(dims[2], r)
    return sp.kron(Zz, sp.kron(Zy, Zx, format="csr"), format="csr")


def stencil_coefficients_of(M: sp.spmatrix, dims) -> np.ndarray:
    """The 27 diagonals of a grid operator with a 27-point pattern, as ``coef[3, 3, 3, nz, ny, nx]``
    (``coef[dz+1, dy+1, dx+1, k, j, i] = M[(k, j, i), (k+dz, j+dy, i+dx)]``, zero past the grid)."""
    nx, ny, nz = dims
    M = M.tocsr()
    coef = np.zeros((3, 3, 3, nz, ny, nx), dtype=np.complex128)
    rows, cols = M.nonzero()
    vals = np.asarray(M[rows, cols]).ravel()
    ri, rj, rk = rows % nx, (rows // nx) % ny, rows // (nx * ny)
    ci, cj, ck = cols % nx, (cols // nx) % ny, cols // (nx * ny)
    dx, dy, dz = ci - ri, cj - rj, ck - rk
    if np.any(np.abs(dx) > 1) or np.any(np.abs(dy) > 1) or np.any(np.abs(dz) > 1):
        raise ValueError("operator couples nodes more than one step apart")
    coef[dz + 1, dy + 1, dx + 1, rk, rj, ri] = vals
    return coef


def coarse_decompose(dims, parts, r, overlap):
    """The fine partition carried to the coarse grid: coarse node ``J`` (at fine index ``r J``) belongs
    to the part whose fine core holds ``r J`` (the last coarse node, which may lie past the fine grid,
    to the last part); boxes grow by ``overlap`` coarse layers on interior sides."""
    cd = coarse_dims(dims, r)
    cuts = []
    for a in range(3):
        fine = [(t * dims[a]) // parts[a] for t in range(parts[a] + 1)]
        c = [0] + [-(-fine[t] // r) for t in range(1, parts[a])] + [cd[a]]
        if any(c[t + 1] <= c[t] for t in range(parts[a])):
            raise ValueError("the coarse grid is too small for this partition")
        cuts.append(c)
    boxes = []
    for tz in range(parts[2]):
        for ty in range(parts[1]):
            for tx in range(parts[0]):
                t = (tx, ty, tz)
                clo = tuple(cuts[a][t[a]] for a in range(3))
                chi = tuple(cuts[a][t[a] + 1] for a in range(3))
                lo = tuple(max(0, clo[a] - overlap) if clo[a] > 0 else 0 for a in range(3))
                hi = tuple(min(cd[a], chi[a] + overlap) if chi[a] < cd[a] else cd[a] for a in range(3))
                boxes.append(Box(clo, chi, lo, hi))
    return boxes


class CoarseGMRES:
    """The inexact coarse solve of the paper's two-level method: ``iters`` right-preconditioned GMRES
    iterations on ``E y = c`` (``x0 = 0``, no restart) with the one-level ORAS preconditioner of the
    coarse grid over the same spatial partition, local problems solved exactly.

    Readings: the coarse boxes are the fine partition carried to the coarse nodes
    (:func:`coarse_decompose`) with ``overlap`` coarse layers; the absorbing fold uses
    ``rho = exp(i k H)``, ``H = r h`` the coarse spacing, ``k`` at the coarse node's fine position
    (clamped to the grid); the partition of unity is the Boolean owner one."""

    def __init__(self, prob: Problem, E, parts, r, overlap=1, iters=10, mode="oras"):
        self.E = E.tocsr()
        self.iters = iters
        dims = (prob.nx, prob.ny, prob.nz)
        self.cdims = coarse_dims(dims, r)
        self.boxes = coarse_decompose(dims, parts, r, overlap)
        coef = stencil_coefficients_of(self.E, self.cdims)
        cx, cy, cz = self.cdims
        K, J, I = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
        c = np.asarray(prob.c, dtype=np.complex128)
        cf = c[np.minimum(r * K, prob.nz - 1), np.minimum(r * J, prob.ny - 1), np.minimum(r * I, prob.nx - 1)]
        rho = np.exp(1j * (prob.omega / cf) * (r * prob.h))
        self.idx, self.pu, self.lu = [], [], []
        for box in self.boxes:
            self.idx.append(box_global_indices(box, self.cdims))
            self.pu.append(partition_of_unity(box))
            self.lu.append(spla.splu(fold_operator(coef, rho, box, mode).tocsc()))

    def apply_M(self, v):
        """One-level ORAS on the coarse grid: ``sum_i R_i^T D_i E_i^{-1} R_i v``."""
        out = np.zeros(v.shape, dtype=np.complex128)
        for i in range(len(self.boxes)):
            out[self.idx[i]] += self.pu[i] * self.lu[i].solve(np.ascontiguousarray(v[self.idx[i]]))
        return out

    def solve(self, c):
        """The inner GMRES approximation of ``E^{-1} c`` (``c`` is ``[nc]`` or ``[nc, nrhs]``)."""
        from .krylov import gmres
        c = np.asarray(c, dtype=np.complex128)
        if c.ndim == 2:
            return np.stack([self.solve(c[:, q]) for q in range(c.shape[1])], axis=1)
        y, _ = gmres(lambda v: self.E @ v, c, self.apply_M, tol=0.0, restart=self.iters, maxit=self.iters,
                     flexible=False)
        return y


# ---------------------------------------------------------------------------
# The preconditioner
# ---------------------------------------------------------------------------

def _local_solve_worker(conn, prob, boxes, mode):
    """Worker process of :class:`LocalSolvePool`: factor its boxes' ``A_i`` with ``splu`` and answer solve
    requests ``{box index: right-hand side}`` until it receives ``None``."""
    coef = neighbour_coefficients(prob)
    lus = {i: spla.splu(local_operator(prob, box, mode, coef).tocsc()) for i, box in boxes}
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        conn.send({i: lus[i].solve(r) for i, r in msg.items()})
    conn.close()


class LocalSolvePool:
    """The exact local solves ``A_i^{-1}`` of Eq. (oras) by ``splu``, as ``ORAS(local="splu")`` computes them,
    with the boxes shared out over spawned worker processes (each builds and keeps the factors of its own
    boxes; single-threaded BLAS in the workers).  Only where the work runs differs: every box's solve is the
    same ``splu`` factorisation and solve."""

    def __init__(self, prob: Problem, boxes, mode, workers):
        import dataclasses
        import multiprocessing as mp
        import os
        order = sorted(range(len(boxes)), key=lambda i: -boxes[i].size)
        share = [[] for _ in range(workers)]
        load = [0] * workers
        for i in order:                       # largest boxes first, each to the least-loaded worker
            w = load.index(min(load))
            share[w].append((i, boxes[i]))
            load[w] += boxes[i].size
        lean = dataclasses.replace(prob, _cache={})
        ctx = mp.get_context("spawn")
        saved = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        self.procs, self.conns = [], []
        try:
            for w in range(workers):
                if not share[w]:
                    continue
                a, b = ctx.Pipe()
                pr = ctx.Process(target=_local_solve_worker, args=(b, lean, share[w], mode), daemon=True)
                pr.start()
                self.procs.append(pr)
                self.conns.append((a, [i for i, _ in share[w]]))
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        for a, _ in self.conns:
            if a.recv() != "ready":
                raise RuntimeError("local solve worker failed")

    def solve(self, rhs):
        """``{box index: A_i^{-1} r}`` for ``rhs = {box index: r}``."""
        for a, idx in self.conns:
            a.send({i: rhs[i] for i in idx})
        out = {}
        for a, _ in self.conns:
            out.update(a.recv())
        return out

    def pids(self):
        return [p.pid for p in self.procs]

    def close(self):
        for a, _ in self.conns:
            try:
                a.send(None)
            except (OSError, BrokenPipeError):
                pass
        for p in self.procs:
            p.join(timeout=10)
            if p.is_alive():
                p.terminate()
        self.procs, self.conns = [], []


class ORAS:
    """``M^{-1}`` of Eq. (2lvl) (or Eq. (oras) alone when ``coarse_ratio == 0``).

    ``workers = k > 1`` (with ``local="splu"``) runs the local solves in a :class:`LocalSolvePool` of k
    processes; the result is the same."""

    def __init__(self, prob: Problem, parts, overlap, coarse_ratio=0, mode="oras", local="splu",
                 coarse_solve="exact", coarse_iters=10, coarse_overlap=1, workers=0):
        self.prob = prob
        self.dims = (prob.nx, prob.ny, prob.nz)
        self.boxes = decompose(self.dims, parts, overlap)
        coef = neighbour_coefficients(prob)
        self.A = assemble_A(prob)
        self.local = local
        self.pool = None
        if workers and workers > 1:
            if local != "splu":
                raise ValueError("a worker pool runs splu local solves")
            self.pool = LocalSolvePool(prob, self.boxes, mode, min(workers, len(self.boxes)))
        self.idx, self.pu, self.Ai, self.solvers = [], [], [], []
        for box in self.boxes:
            self.idx.append(box_global_indices(box, self.dims))
            self.pu.append(partition_of_unity(box))
            if self.pool is not None:
                continue
            Ai = local_operator(prob, box, mode, coef)
            self.Ai.append(Ai)
            if local == "splu":
                self.solvers.append(spla.splu(Ai.tocsc()))
            elif local == "planes":
                m = box.dims[0] * box.dims[1]
                D, L, U = plane_blocks(Ai, m, box.dims[2])
                self.solvers.append((plane_factor(D, L, U), L, U))
            else:
                raise ValueError(local)
        self.coarse_ratio = coarse_ratio
        if coarse_ratio:
            self.Z = coarse_basis(self.dims, coarse_ratio)
            self.E = (self.Z.T @ self.A @ self.Z).tocsc()
            if coarse_solve == "exact":
                self.E_lu = spla.splu(self.E)
                self.coarse = None
            elif coarse_solve == "gmres":
                self.coarse = CoarseGMRES(prob, self.E, parts, coarse_ratio, coarse_overlap, coarse_iters, mode)
            else:
                raise ValueError(coarse_solve)

    def local_solve(self, i, r):
        if self.local == "splu":
            return self.solvers[i].solve(r)
        G, L, U = self.solvers[i]
        return plane_solve(G, L, U, r)

    def apply_one_level(self, v):
        """``sum_i R_i^T D_i A_i^{-1} R_i v`` for ``v`` of shape ``[N]`` or ``[N, nrhs]``."""
        out = np.zeros(v.shape, dtype=np.complex128)
        if self.pool is not None:
            xs = self.pool.solve({i: np.ascontiguousarray(v[self.idx[i]]) for i in range(len(self.boxes))})
        for i in range(len(self.boxes)):
            xi = xs[i] if self.pool is not None else self.local_solve(i, np.ascontiguousarray(v[self.idx[i]]))
            d = self.pu[i] if v.ndim == 1 else self.pu[i][:, None]
            out[self.idx[i]] += d * xi
        return out

    def close(self):
        """Stop the worker pool, if any."""
        if self.pool is not None:
            self.pool.close()
            self.pool = None

    def coarse_correction(self, v):
        """``Q v = Z E^{-1} Z^T v`` (the inner GMRES approximation of ``E^{-1}`` with ``coarse_solve="gmres"``,
        which makes the preconditioner depend on ``v`` nonlinearly: the outer method must be FGMRES)."""
        c = np.asarray(self.Z.T @ v)
        if self.coarse is not None:
            return self.Z @ self.coarse.solve(c)
        return self.Z @ self.E_lu.solve(c)

    def apply(self, v):
        v = np.asarray(v, dtype=np.complex128)
        if not self.coarse_ratio:
            return self.apply_one_level(v)
        q = self.coarse_correction(v)
        return self.apply_one_level(v - self.A @ q) + q


def direct_solve_planes(prob: Problem, B):
    """Exact ``A^{-1} B`` by the plane-by-plane block LU of the whole grid (one box, no folding).

    ``B`` is ``[N]`` or ``[N, nrhs]``.  Used as the reference solution of
    small problems; pinned against ``splu`` and ``numpy.linalg.solve``.
    """
    A = assemble_A(prob)
    m = prob.nx * prob.ny
    D, L, U = plane_blocks(A, m, prob.nz)
    G = plane_factor(D, L, U)
    return plane_solve(G, L, U, np.asarray(B, dtype=np.complex128))
