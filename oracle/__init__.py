"""FP64 CPU oracle for the ORAS-GMRES Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the GPU library computes, written from the paper
(Dolean, Jolivet, Tournier, Combe, Operto, Riffo, EAGE 2021, arXiv 2103.14921):

* Eq. (eqh) / Eq. (eq1): the Helmholtz equation ``(Delta + k^2) u = b`` and its
  discrete form ``A u = b`` with absorbing layers on the vertical and bottom
  faces and a homogeneous Dirichlet top (section "Tetrahedral finite elements
  versus 27-point finite-differences").
* The 27-point mixed-grid stencil (same section; Operto et al. 2007 cited
  there): rotated-coordinate Laplacians and a consistent mass term whose
  weights are fitted by least squares on the numerical dispersion.
* Eq. (2lvl) and Eq. (oras): the two-level ORAS preconditioner with Boolean
  restrictions, a partition of unity and absorbing interface conditions in the
  local operators, and a coarse space ``Q = Z E^{-1} Z^T``.
* GMRES (section "Domain decomposition preconditioner").

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with ``paper_2103_14921_gb300`` and imports nothing from it.

Parity status of each function is stated in its module docstring; every
function here is pinned by a ``-m "not gpu"`` test against something other
than itself (a closed form, a textbook special case, a library routine or an
invariant), except where a module says "parity unpinned".
"""
