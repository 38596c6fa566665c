"""The allocation-free preconditioner apply gives the same result as oras_apply.

``oras_apply_noalloc`` exists for callers that cannot let the library allocate
device memory during a call (an application holding the GPU's memory in its
own pool, or a loop that must avoid the device-wide synchronisation of
cudaMalloc/cudaFree).  It keeps its working vectors in a fixed 8 MiB device
array.  This file is collected last on purpose: a failure here comes after
every other test has run.
"""
import numpy as np
import pytest

from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _noalloc(helm, ctx, o, v):
    import torch
    got = torch.empty_like(v)
    before = ctx.bytes_in_use
    st = helm.lib().oras_apply_noalloc(o._h, helm._ptr(v), helm._ptr(got), v.shape[-1])
    assert st == helm.OK, helm.lib().helm_last_error(ctx._h)
    assert ctx.bytes_in_use == before          # nothing allocated through the library
    return got


def test_noalloc_apply_matches_oras_apply_twice_in_a_row():
    """FP64 and FP32 (CUDA-core sweeps), TF32 and BF16 (tensor-core sweeps) factors; two calls in a row
    with different inputs.  The tensor-core sweeps give the same values whichever launch form runs them
    (the persistent queue or per-step launches), so the two entry points agree to rounding."""
    import torch
    from paper_2103_14921_gb300 import build, helm
    build.build()
    ctx = helm.Context(0)
    nx, ny, nz = 20, 18, 14
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=3, weights=helm.fit_weights())
    for prec in (helm.PREC_FP64, helm.PREC_FP32, helm.PREC_TF32, helm.PREC_BF16):
        o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=prec)
        for call, seed in enumerate((51, 52)):       # two calls in a row, different inputs
            v = torch.from_numpy(synth.random_complex((nz, ny, nx, 4), seed)).cuda()
            want = o.apply(v)
            got = _noalloc(helm, ctx, o, v)
            assert _rel(got.cpu().numpy(), want.cpu().numpy()) <= 1e-12, (prec, call)
        # a request whose working vectors exceed the fixed array is rejected with a clear message
        big = torch.zeros((nz, ny, nx, 200), dtype=torch.complex128, device="cuda")
        out = torch.empty_like(big)
        st = helm.lib().oras_apply_noalloc(o._h, helm._ptr(big), helm._ptr(out), 200)
        assert st == helm.EINVAL
        assert b"scratch" in helm.lib().helm_last_error(ctx._h)
        o.close()


def test_noalloc_apply_first_call_on_a_new_handle():
    """The allocation-free apply as the very first call on a fresh handle (no apply scratch or sweep queue
    allocated yet), then twice more, each checked against oras_apply afterwards."""
    import torch
    from paper_2103_14921_gb300 import build, helm
    build.build()
    ctx = helm.Context(0)
    nx, ny, nz = 18, 20, 12
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 4.0, c, npml=3, weights=helm.fit_weights())
    for prec in (helm.PREC_TF32, helm.PREC_FP64):
        o = helm.Oras(grid, (2, 2, 1), 2, coarse_ratio=4, factor_prec=prec)
        vs = [torch.from_numpy(synth.random_complex((nz, ny, nx, 2), s)).cuda() for s in (53, 54, 55)]
        got = [_noalloc(helm, ctx, o, v) for v in vs]
        for v, g in zip(vs, got):
            assert _rel(g.cpu().numpy(), o.apply(v).cpu().numpy()) <= 1e-12, prec
        o.close()
