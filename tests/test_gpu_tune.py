"""The autotuner times real solves through the library and caches its choice."""
import pytest

from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu


def test_tuner_picks_a_converging_decomposition_and_caches_it(tmp_path):
    import torch
    from paper_2103_14921_gb300 import build, helm, tune
    build.build()
    ctx = helm.Context(0)
    n, h, f = 48, 25.0, 4.0
    grid = helm.Grid(ctx, n, n, n, h, f, synth.linear_gradient(n, n, n, h), npml=8, weights=helm.fit_weights())
    b = torch.from_numpy(synth.point_sources(n, n, n, h, synth.source_plane_positions(n, n, 8, 3, 2, 1))).cuda()
    path = str(tmp_path / "tune.json")
    cands = [((2, 2, 2), 2), ((3, 3, 2), 2), ((2, 2, 2), 4)]
    r = tune.tune(ctx, grid, b, cands=cands, cache_path=path, nrhs=16)
    assert not r["cached"] and tuple(r["parts"]) in {c[0] for c in cands}
    assert r["rhs_per_s"] > 0 and len(r["trials"]) == 3
    assert all(t["converged"] for t in r["trials"])
    again = tune.tune(ctx, grid, b, cands=cands, cache_path=path, nrhs=16)
    assert again["cached"] and again["parts"] == r["parts"]
    o = helm.Oras(grid, tuple(r["parts"]), r["overlap"], coarse_ratio=4, factor_prec=helm.PREC_TF32)
    _, st = o.solve(b)
    assert all(s["converged"] for s in st)
    # the plane-sweep knobs on the chosen factors: every setting timed, the fastest kept and cached
    k = tune.tune_knobs(ctx, o, b)
    assert len(k["trials"]) == len(tune.KNOB_GRID) and k["best"] in tune.KNOB_GRID
    r2 = tune.tune(ctx, grid, b, cands=cands[:1], cache_path=str(tmp_path / "tune2.json"), nrhs=16, knobs=True)
    assert r2["knobs"] in tune.KNOB_GRID and len(r2["knob_trials"]) == len(tune.KNOB_GRID)
    assert tune.tune(ctx, grid, b, cands=cands[:1], cache_path=str(tmp_path / "tune2.json"), nrhs=16,
                     knobs=True)["cached"]
    tune.apply_knobs(ctx, {"tc_stages": 0, "tc_flow": 1})
