"""Serving loop: continuous batching, factor cache, admission under an HBM budget (through the C ABI).

Each request's result must be the same alone and in a mix with other requests
(same factors and other models), within 10 x tol; with a fixed number of
column slots the per-column arithmetic does not depend on the other columns,
so the results are expected to be bit-identical, which is checked too.
"""
import numpy as np
import pytest

from oracle.discretization import Problem, apply_A
from paper_2103_14921_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (24, 22, 20)
H, F, NPML = 25.0, 5.0, 4


def _descs(helm, w, factor_prec):
    nx, ny, nz = DIMS
    gd = helm.GridDesc(nx, ny, nz, H, F, NPML, 1e-3, helm.TOP_DIRICHLET, (__import__("ctypes").c_double * 7)(*w))
    od = helm.OrasDesc(2, 2, 2, 2, 4, 0, factor_prec)
    return gd, od


def _rhs(positions):
    nx, ny, nz = DIMS
    return synth.point_sources(nx, ny, nz, H, positions)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2103_14921_gb300 import build, helm
    build.build()
    ctx = helm.Context(0)
    w = helm.fit_weights()
    nx, ny, nz = DIMS
    cA = torch.from_numpy(synth.linear_gradient(nx, ny, nz, H))
    cB = torch.from_numpy(synth.layered(nx, ny, nz, H, seed=5))
    return helm, ctx, w, cA, cB


@pytest.mark.parametrize("factor_prec", [2, 0])   # TF32 tensor-core factors, FP64 factors
def test_same_alone_and_in_the_mix(env, factor_prec):
    import torch
    helm, ctx, w, cA, cB = env
    gd, od = _descs(helm, w, factor_prec)
    basis = helm.PREC_FP32 if factor_prec != helm.PREC_FP64 else helm.PREC_FP64
    tol = 1e-6
    bA = torch.from_numpy(_rhs([(12, 11, 3), (5, 6, 7), (18, 15, 9)])).cuda()
    bC = torch.from_numpy(_rhs([(3, 3, 3), (20, 18, 12), (10, 10, 10), (7, 16, 4)])).cuda()
    bB = torch.from_numpy(_rhs([(11, 11, 5), (6, 17, 8)]))                     # host buffers for model B
    with helm.Server(ctx, slots_per_batch=12) as sv:
        xA = torch.empty_like(bA)
        s0 = sv.wait(sv.submit(1, gd, cA, od, bA, xA, tol=tol, basis_prec=basis))
        assert s0["status"] == helm.OK and not s0["factors_reused"]
        x_alone = xA.clone()
        # the mix: B (other model, host buffers), A again and C (same factors) submitted together
        xA2, xC = torch.empty_like(bA), torch.empty_like(bC)
        xB = torch.empty_like(bB)
        tB = sv.submit(2, gd, cB, od, bB, xB, tol=tol, basis_prec=basis)
        tA = sv.submit(1, gd, cA, od, bA, xA2, tol=tol, basis_prec=basis)
        tC = sv.submit(1, gd, cA, od, bC, xC, tol=tol, basis_prec=basis)
        sA, sB, sC = sv.wait(tA), sv.wait(tB), sv.wait(tC)
        for s in (sA, sB, sC):
            assert s["status"] == helm.OK and s["true_relres_max"] <= tol
        assert sA["factors_reused"] and sC["factors_reused"] and not sB["factors_reused"]
    a, b = x_alone.cpu().numpy(), xA2.cpu().numpy()
    assert np.linalg.norm(a - b) <= 10 * tol * np.linalg.norm(a)
    assert np.array_equal(a, b), "columns are expected to be bit-identical alone and in the mix"
    # every result solves its own problem (oracle FP64 residual)
    nx, ny, nz = DIMS
    for c, bb, xx in ((cA, bC, xC), (cB, bB, xB)):
        prob = Problem(nx, ny, nz, H, F, c.numpy(), npml=NPML, weights=w)
        X = xx.cpu().numpy()
        Bn = bb.cpu().numpy()
        for r in range(Bn.shape[-1]):
            res = np.linalg.norm(apply_A(prob, X[..., r]) - Bn[..., r]) / np.linalg.norm(Bn[..., r])
            assert res <= tol


def test_budget_admission_and_latency_stats(env):
    import torch
    helm, _, w, cA, _ = env
    small = helm.Context(0, budget_bytes=16 << 20)         # far too small for the factors
    gd, od = _descs(helm, w, helm.PREC_TF32)
    b = torch.from_numpy(_rhs([(12, 11, 3)])).cuda()
    x = torch.empty_like(b)
    with helm.Server(small, slots_per_batch=4) as sv:
        s = sv.wait(sv.submit(7, gd, cA, od, b, x))
        assert s["done"] and s["status"] == helm.ENOMEM
    # a sequence of requests on a roomy context reports queue and end-to-end latency
    ctx = helm.Context(0)
    lat = []
    with helm.Server(ctx, slots_per_batch=4) as sv:
        tickets = []
        for i in range(6):
            bi = torch.from_numpy(_rhs([(4 + 2 * i, 5 + i, 3 + i)])).cuda()
            tickets.append((sv.submit(3, gd, cA, od, bi, torch.empty_like(bi)), bi))
        for t, _ in tickets:
            s = sv.wait(t)
            assert s["status"] == helm.OK
            lat.append(s["latency_ms"])
            assert s["queue_ms"] <= s["latency_ms"]
    assert len(lat) == 6 and min(lat) > 0
    with pytest.raises(helm.HelmError):
        helm.Server(ctx, 0)


def test_new_factor_set_joins_while_another_batch_runs(env):
    """A request on a new model arrives while a batch on cached factors is cycling: its factors are built on
    the builder thread meanwhile and it joins the running loop; both results are bit-identical to the same
    requests served alone."""
    import torch
    helm, ctx, w, cA, cB = env
    gd, od = _descs(helm, w, helm.PREC_TF32)
    tol = 1e-6
    bA = torch.from_numpy(_rhs([(12, 11, 3), (5, 6, 7), (18, 15, 9), (9, 4, 12)])).cuda()
    bB = torch.from_numpy(_rhs([(11, 11, 5), (6, 17, 8)])).cuda()
    alone = {}
    for key, c, bb in (("A", cA, bA), ("B", cB, bB)):
        with helm.Server(ctx, slots_per_batch=8) as sv:
            xx = torch.empty_like(bb)
            s = sv.wait(sv.submit(10 if key == "A" else 20, gd, c, od, bb, xx, tol=tol))
            assert s["status"] == helm.OK
            alone[key] = xx.cpu().numpy()
    with helm.Server(ctx, slots_per_batch=8) as sv:
        warm = torch.from_numpy(_rhs([(4, 4, 4)])).cuda()
        assert sv.wait(sv.submit(10, gd, cA, od, warm, torch.empty_like(warm), tol=tol))["status"] == helm.OK
        xA, xB = torch.empty_like(bA), torch.empty_like(bB)
        tA = sv.submit(10, gd, cA, od, bA, xA, tol=tol)          # cached factors: admitted at once
        tB = sv.submit(20, gd, cB, od, bB, xB, tol=tol)          # new model: built while A's batch cycles
        sA, sB = sv.wait(tA), sv.wait(tB)
    assert sA["status"] == helm.OK and sB["status"] == helm.OK
    assert sA["factors_reused"] and not sB["factors_reused"]
    assert np.array_equal(xA.cpu().numpy(), alone["A"])
    assert np.array_equal(xB.cpu().numpy(), alone["B"])


def test_burst_of_new_sets_under_a_tight_budget_all_complete(env):
    """Four requests on four new models submitted at once under a budget that holds about two factor sets
    with their solver workspace: the later ones wait for room (sets built for waiting requests are not
    evicted for another's room, and each set's estimate stays reserved until its first cycle has allocated
    its scratch), so every request completes with status OK and the tolerance, none with ENOMEM."""
    import torch
    helm, _, w, cA, _ = env
    gd, od = _descs(helm, w, helm.PREC_TF32)
    nx, ny, nz = DIMS
    restart = 30
    engine = nx * ny * nz * 16 * ((2 * restart + 3) * 8 + 3 * 16) + nx * ny * nz * 48   # FP32 basis, 16 slots
    need = helm.estimate_bytes(gd, od, 16) + engine
    tight = helm.Context(0, budget_bytes=int(2.5 * need))
    tol = 1e-6
    with helm.Server(tight, slots_per_batch=16) as sv:
        jobs = []
        for i in range(4):
            bi = torch.from_numpy(_rhs([(6 + 3 * i, 7 + 2 * i, 4 + i), (15, 12, 9 + i)])).cuda()
            jobs.append((sv.submit(100 + i, gd, cA, od, bi, torch.empty_like(bi), tol=tol, restart=restart), bi))
        stats = [sv.wait(t) for t, _ in jobs]
    for s in stats:
        assert s["status"] == helm.OK, s
        assert s["true_relres_max"] <= tol
        assert not s["factors_reused"]
