"""Tensor-core local solves against the FP64 oracle at the level of one preconditioner apply.

``oras_apply`` with TF32 or BF16 factors on multi-plane boxes, so that both
sweeps of the plane-by-plane block LU run (Eq. oras; forward
``y_k = G_k (b_k - L_k y_{k-1})``, backward ``x_k = y_k - G_k U_k x_{k+1}``),
through the persistent queue (even column counts) and the per-step launches
(odd), compared element by element with the oracle's FP64 apply (exact plane
inverses from the oracle's own block LU).

The bar is the error that TF32 / BF16 operands cause by themselves: the oracle
runs the same sweeps with its exact inverses and every tensor-core operand
rounded as the hardware rounds it (TF32: the low 13 mantissa bits of each
FP32 operand dropped -- the GPU's error matches truncation, not rounding to
nearest, which would be 3-9 times smaller; BF16: factors and right-hand sides
rounded to nearest bfloat16), exactly otherwise.  Per column, the GPU's
relative L2 error must stay within 1.5 times that emulated rounding error, and
its largest element error within 2 times the emulation's largest.

A second check pins the kernels' arithmetic: the same emulation built from the
library's own stored inverses (read back exactly) must be closer to the GPU
result than half the rounding error itself (what remains is the tensor core's
FP32 accumulation and the FP32 operand preparation, carried through the later
planes like the rounding error).

Cases: ragged boxes with 9-11 planes (3 x 2 x 2 boxes of a 21 x 18 x 17
grid), full-size planes (a 64 x 64 x 12 grid in 2 x 2 x 1 boxes of
34 x 34 x 12 nodes, m = 1156 = 9 full 128-row tiles and a partial tile of 4
rows), and the two-level preconditioner (Eq. 2lvl).
"""
import numpy as np
import pytest

from oracle.discretization import Problem
from oracle.schwarz import ORAS
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.Context(0)


def _round_tf32(a, mode):
    """Complex values rounded to TF32 through FP32: 'trunc' keeps the top 10 mantissa bits, 'rn' rounds to
    nearest even."""
    def r(x):
        u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        if mode == "rn":
            u = u + 0x0FFF + ((u >> 13) & 1)
        return (u & 0xFFFFE000).astype(np.uint32).view(np.float32).astype(np.float64)
    return r(a.real) + 1j * r(a.imag)


def _round_bf16(a):
    """Complex values rounded to nearest-even bfloat16 through FP32."""
    def r(x):
        u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        u = u + 0x7FFF + ((u >> 16) & 1)
        return (u & 0xFFFF0000).astype(np.uint32).view(np.float32).astype(np.float64)
    return r(a.real) + 1j * r(a.imag)


def _f32(a):
    return a.astype(np.complex64).astype(np.complex128)


def _emulated_sweep(G, L, U, b, rnd):
    """The two plane sweeps with stored inverses G (exact values), tensor-core operands rounded by `rnd`,
    FP32 results (local vectors are complex64 on the device)."""
    nz = len(G)
    y = [None] * nz
    for k in range(nz):
        r = b[k] if k == 0 else _f32(b[k] - L[k] @ y[k - 1])
        y[k] = _f32(G[k] @ rnd(r))
    x = [None] * nz
    x[-1] = y[-1]
    for k in range(nz - 2, -1, -1):
        x[k] = _f32(y[k] - G[k] @ rnd(_f32(U[k] @ x[k + 1])))
    return np.concatenate(x, axis=0)


def _rounders(prec):
    """(factor rounding, operand rounding) of the tensor-core sweep in this precision."""
    if prec == "tf32":
        return (lambda g: _round_tf32(g, "trunc")), (lambda a: _round_tf32(a, "trunc"))
    return (lambda g: _round_bf16(_f32(g))), _round_bf16


def _one_level_emulated(M, vf, factors, rnd_g, rnd):
    """sum_i R_i^T D_i (emulated sweeps of box i) R_i v with the given inverses per box."""
    out = np.zeros(vf.shape, dtype=np.complex128)
    for i, box in enumerate(M.boxes):
        _, L, U = M.solvers[i]
        m = box.dims[0] * box.dims[1]
        bi = vf[M.idx[i]]
        bk = [_f32(bi[k * m:(k + 1) * m]) for k in range(box.dims[2])]
        out[M.idx[i]] += M.pu[i][:, None] * _emulated_sweep([rnd_g(g) for g in factors[i]], L, U, bk, rnd)
    return out


def _check(prec, got, want, emu_oracle, emu_own, label):
    worst = []
    for r in range(want.shape[1]):
        g, w_, eo, ew = got[:, r], want[:, r], emu_oracle[:, r], emu_own[:, r]
        nw = np.linalg.norm(w_)
        rel = np.linalg.norm(g - w_) / nw
        bar = 1.5 * np.linalg.norm(eo - w_) / nw
        mx, mx_bar = np.abs(g - w_).max(), 2.0 * np.abs(eo - w_).max()
        own = np.linalg.norm(g - ew) / nw
        worst.append((rel, bar, mx / np.abs(w_).max(), mx / mx_bar, own, bar / 1.5))
        assert rel <= bar, (label, r, rel, bar)
        assert mx <= mx_bar, (label, r, mx, mx_bar)
        assert own <= 0.5 * bar / 1.5, (label, r, own, bar / 1.5)
    w = max(worst, key=lambda t: t[0] / t[1])
    print(f"{label}: rel L2 {w[0]:.3e} (emulated rounding {w[5]:.3e}, bar {w[1]:.3e}), max per column "
          f"{w[2]:.3e} (max-error ratio to bar {max(t[3] for t in worst):.2f}), vs own-factor emulation "
          f"{max(t[4] for t in worst):.3e}")


def _case(ctx, dims, parts, ov, npml, prec, nrhs, seed):
    import torch
    from paper_2103_14921_gb300 import helm
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=npml, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 5.0, c, npml=npml, weights=w)
    fp = helm.PREC_TF32 if prec == "tf32" else helm.PREC_BF16
    o = helm.Oras(grid, parts, ov, factor_prec=fp)
    M = ORAS(prob, parts, ov, local="planes")
    v = synth.random_complex((nz, ny, nx, nrhs), seed)
    got = o.apply(torch.from_numpy(v).cuda()).cpu().numpy().reshape(-1, nrhs)
    vf = v.reshape(-1, nrhs)
    want = M.apply(vf)
    nb = o.box_info(-1)[0]
    assert nb == len(M.boxes)
    own = []
    for i in range(nb):
        _, lo, bd = o.box_info(i)
        assert lo == M.boxes[i].lo and bd == M.boxes[i].dims
        own.append([o.plane_inverse(i, k).cpu().numpy() for k in range(bd[2])])   # the library's stored inverses
    rnd_g, rnd = _rounders(prec)
    emu_oracle = _one_level_emulated(M, vf, [M.solvers[i][0] for i in range(nb)], rnd_g, rnd)
    # the stored inverses are already in the operand format (TF32 reads the stored FP32 values truncated)
    emu_own = _one_level_emulated(M, vf, own, rnd_g if prec == "tf32" else (lambda g: g), rnd)
    _check(prec, got, want, emu_oracle, emu_own, f"{prec} dims={dims} parts={parts} nrhs={nrhs}")


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("nrhs", [16, 3, 128])
def test_multiplane_tc_apply_matches_oracle(ctx, prec, nrhs):
    """Ragged boxes of 9-11 planes; 16 columns take the persistent queue, 3 the per-step launches, 128 the
    persistent queue with the preparation staged in column chunks (N = 256, one CTA per SM)."""
    _case(ctx, (21, 18, 17), (3, 2, 2), 2, 3, prec, nrhs, 71 + nrhs)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_full_size_planes_tc_apply_matches_oracle(ctx, prec):
    """Planes of 34 x 34 = 1156 nodes (9 full row tiles and a partial one), 12 planes per box."""
    _case(ctx, (64, 64, 12), (2, 2, 1), 2, 4, prec, 4, 81)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_two_level_tc_apply_matches_oracle(ctx, prec):
    """Two-level ORAS (Eq. 2lvl) with tensor-core local solves and the complex64 copy of the FP64 coarse
    factors; the emulation applies the rounded sweeps to t = v - A q with the oracle's exact coarse term q."""
    import torch
    from paper_2103_14921_gb300 import helm
    dims = (21, 18, 17)
    nx, ny, nz = dims
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    w = helm.fit_weights()
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=3, weights=w)
    prob = Problem(nx, ny, nz, 25.0, 5.0, c, npml=3, weights=w)
    fp = helm.PREC_TF32 if prec == "tf32" else helm.PREC_BF16
    o = helm.Oras(grid, (3, 2, 2), 2, coarse_ratio=4, factor_prec=fp)
    M = ORAS(prob, (3, 2, 2), 2, coarse_ratio=4, local="planes")
    v = synth.random_complex((nz, ny, nx, 8), 91)
    vf = v.reshape(-1, 8)
    got = o.apply(torch.from_numpy(v).cuda()).cpu().numpy().reshape(-1, 8)
    want = M.apply(vf)
    q = M.coarse_correction(vf)
    t = vf - M.A @ q
    rnd_g, rnd = _rounders(prec)
    nb = len(M.boxes)
    emu_oracle = _one_level_emulated(M, t, [M.solvers[i][0] for i in range(nb)], rnd_g, rnd) + q
    own = [[o.plane_inverse(i, k).cpu().numpy() for k in range(M.boxes[i].dims[2])] for i in range(nb)]
    emu_own = _one_level_emulated(M, t, own, rnd_g if prec == "tf32" else (lambda g: g), rnd) + q
    _check(prec, got, want, emu_oracle, emu_own, f"{prec} two-level")
