"""A bounded device wait that gives up is reported, and the handle stays usable.

The persistent tensor-core sweep waits (bounded) for each queue slot to be
published.  The test-only knob HELM_TUNE_FLOW_WAIT_US = 0 makes a CTA give up
at its first poll of a slot that is not yet published (every launch has such
a poll: the queue starts with only the first operation of each box).  The
launch then drains -- the copies and tensor-core products already issued
complete, TMEM is freed -- and oras_apply returns HELM_ETIMEOUT.  Nothing
hangs or faults: the wait is a poll loop with a time limit, not an endless
spin.  With the knob restored the same handle gives the result it gave before.
"""
import pytest

from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


def test_flow_wait_timeout_returns_etimeout_and_recovers():
    import torch
    from paper_2103_14921_gb300 import build, helm
    build.build()
    ctx = helm.Context(0)
    nx, ny, nz = 24, 22, 20
    c = synth.linear_gradient(nx, ny, nz, 25.0, 1500.0, 1.0)
    grid = helm.Grid(ctx, nx, ny, nz, 25.0, 5.0, c, npml=3, weights=helm.fit_weights())
    o = helm.Oras(grid, (2, 2, 2), 2, coarse_ratio=4, factor_prec=helm.PREC_TF32)
    v = torch.from_numpy(synth.random_complex((nz, ny, nx, 16), 41)).cuda()
    ctx.profile(True, only=["sweep_flow"])
    want = o.apply(v)
    assert ctx.profile_query("sweep_flow")[0] == 1        # the persistent sweep ran
    ctx.profile(False)
    ctx.set_tuning(helm.TUNE_FLOW_WAIT_US, 0)
    with pytest.raises(helm.HelmError) as ei:
        o.apply(v)
    assert ei.value.status == helm.ETIMEOUT
    assert "bounded device wait" in str(ei.value)
    ctx.set_tuning(helm.TUNE_FLOW_WAIT_US, 2000000)
    again = o.apply(v)
    assert torch.equal(again, want)
    # a solve on the same context afterwards is unaffected
    b = torch.from_numpy(synth.point_sources(nx, ny, nz, 25.0, [(12, 11, 3), (8, 9, 4)])).cuda()
    x, stats = o.solve(b, tol=1e-6, basis_prec=helm.PREC_FP32)
    assert all(s["converged"] for s in stats)
    o.close()
    grid.close()
    ctx.close()
