"""The allocation-free preconditioner apply gives the same result as oras_apply.

``oras_apply_noalloc`` exists for callers that cannot let the library allocate
device memory during a call (an application holding the GPU's memory in its
own pool, or a loop that must avoid the device-wide synchronisation of
cudaMalloc/cudaFree).  It keeps its working vectors in a fixed 8 MiB device
array.  This file is collected last on purpose: a failure here comes after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_noalloc_apply_matches_oras_apply_twice_in_a_row():
    import torch
    from paper_2103_14921_gb300 import build, helm
    build.build()
    ctx = helm.Context(0)
    nx, ny, nz = 20, 18, 14
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=3, weights=helm.fit_weights())
    for prec in (helm.PREC_FP64, helm.PREC_FP32):
        o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=prec)
        for call, seed in enumerate((51, 52)):       # two calls in a row, different inputs
            v = torch.from_numpy(synth.random_complex((nz, ny, nx, 3), seed)).cuda()
            want = o.apply(v)
            got = torch.empty_like(v)
            before = ctx.bytes_in_use
            st = helm.lib().oras_apply_noalloc(o._h, helm._ptr(v), helm._ptr(got), 3)
            assert st == helm.OK, helm.lib().helm_last_error(ctx._h)
            assert ctx.bytes_in_use == before          # nothing allocated through the library
            assert _rel(got.cpu().numpy(), want.cpu().numpy()) <= 1e-12, (prec, call)
        # a request whose working vectors exceed the fixed array is rejected with a clear message
        big = torch.zeros((nz, ny, nx, 200), dtype=torch.complex128, device="cuda")
        out = torch.empty_like(big)
        st = helm.lib().oras_apply_noalloc(o._h, helm._ptr(big), helm._ptr(out), 200)
        assert st == helm.EINVAL
        assert b"scratch" in helm.lib().helm_last_error(ctx._h)
        o.close()
