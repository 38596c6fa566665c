"""Autotuner for the box decomposition of the ORAS local solves.

For a problem (grid, medium, frequency, number of right-hand sides, factor
precision) the tuner enumerates box decompositions whose cores are
``core_xy`` nodes in x and y and ``core_z`` in z with ``overlap`` nodes added
on interior sides, drops those whose estimated device memory (factors,
apply scratch and the Krylov basis) exceeds a cap, orders the rest by that
estimate, times a short sample solve for up to ``max_trials`` of them and
keeps the fastest in right-hand sides per second.  On the chosen factors it
then times the plane-sweep knobs (pipeline depth of the tensor-core sweep,
persistent queue or per-step launches) and keeps the fastest setting.
Choices are cached in a JSON file keyed by the problem class, so a later run
reuses them without timing.  All work runs through the C library; the tuner
only orchestrates.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import helm


def problem_key(nx, ny, nz, freq_hz, nrhs, factor_prec):
    """Cache key: grid, frequency, right-hand sides rounded up to a power of two, precision."""
    r = 1 << max(0, math.ceil(math.log2(max(1, nrhs))))
    return f"{nx}x{ny}x{nz}_f{freq_hz:g}_r{r}_p{factor_prec}"


def candidates(nx, ny, nz, core_xy=(16, 20, 24), core_z=(16, 20, 24), overlaps=(2, 3, 4)):
    """Distinct ``(parts, overlap)`` decompositions; parts = round(n / core) per axis (at least 1)."""
    seen, out = set(), []
    for s in core_xy:
        for sz in core_z:
            for ov in overlaps:
                parts = (max(1, round(nx / s)), max(1, round(ny / s)), max(1, round(nz / sz)))
                key = (parts, ov)
                if key not in seen:
                    seen.add(key)
                    out.append(key)
    return out


def krylov_bytes(n_points, nrhs, restart, basis_bytes=8):
    """Bytes of the flexible GMRES basis (V and Z) and the complex128 right-hand side, solution, residual."""
    return n_points * nrhs * ((2 * restart + 3) * basis_bytes + 3 * 16)


def load_cache(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_cache(path, cache):
    if path:
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def tune(ctx, grid, b_sample, factor_prec=helm.PREC_TF32, coarse_ratio=4, restart=30, tol=1e-6, nrhs=None,
         mem_cap_bytes=None, max_trials=6, cache_path=None, cands=None, knobs=False, coarse_opts=None):
    """Pick the decomposition with the most right-hand sides per second for this problem.

    ``grid`` is a :class:`helm.Grid`; ``b_sample`` a CUDA tensor of right-hand sides used for the
    timing (a few columns of the real workload); ``nrhs`` the batch size the choice is for (memory
    estimate and cache key; default the sample's).  Returns a dict with ``parts``, ``overlap``,
    ``rhs_per_s``, ``iterations`` and ``trials`` (every timed candidate); with ``knobs=True`` also
    ``knobs`` (the fastest plane-sweep setting, left set on the context) and ``knob_trials``; with
    ``coarse_opts`` (a list of ``(coarse_ratio, coarse_iters)``, ``coarse_iters = 0`` for the exact coarse
    solve) the coarse level of the chosen decomposition is timed for each option as well, and the result
    carries ``coarse_ratio`` and ``coarse_iters``.
    """
    d = grid.desc
    nrhs = nrhs or b_sample.shape[-1]
    key = problem_key(d.nx, d.ny, d.nz, d.freq_hz, nrhs, factor_prec)
    cache = load_cache(cache_path)
    if key in cache and (not knobs or "knobs" in cache[key]):
        if "knobs" in cache[key]:
            apply_knobs(ctx, cache[key]["knobs"])
        return dict(cache[key], cached=True)
    if mem_cap_bytes is None:
        mem_cap_bytes = 200 << 30
    npts = d.nx * d.ny * d.nz
    scored = []
    for parts, ov in (cands or candidates(d.nx, d.ny, d.nz)):
        od = helm.OrasDesc(parts[0], parts[1], parts[2], ov, coarse_ratio, 0, factor_prec)
        est = helm.estimate_bytes(d, od, nrhs) + krylov_bytes(npts, nrhs, restart)
        if est <= mem_cap_bytes:
            scored.append((est, parts, ov))
    scored.sort()
    trials = []
    for est, parts, ov in scored[:max_trials]:
        try:
            o = helm.Oras(grid, parts, ov, coarse_ratio=coarse_ratio, factor_prec=factor_prec)
        except helm.HelmError as e:
            trials.append(dict(parts=parts, overlap=ov, error=str(e)))
            continue
        import torch
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, stats = o.solve(b_sample, tol=tol, restart=restart, basis_prec=helm.PREC_FP32, allow_notconv=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        conv = all(s["converged"] for s in stats)
        trials.append(dict(parts=list(parts), overlap=ov, est_bytes=est, solve_s=dt, converged=conv,
                           rhs_per_s=b_sample.shape[-1] / dt if conv else 0.0,
                           iterations=max(s["iterations"] for s in stats), setup_s=o.setup_seconds))
        o.close()
    good = [t for t in trials if t.get("converged")]
    if not good:
        raise RuntimeError(f"no decomposition converged or fitted the memory cap: {trials}")
    best = max(good, key=lambda t: t["rhs_per_s"])
    out = dict(parts=list(best["parts"]), overlap=best["overlap"], rhs_per_s=best["rhs_per_s"],
               iterations=best["iterations"], trials=trials, key=key)
    out.update(coarse_ratio=coarse_ratio, coarse_iters=0)
    if coarse_opts:
        ctrials = []
        for cr, ci in coarse_opts:
            import torch
            t0 = time.perf_counter()
            o = helm.Oras(grid, tuple(best["parts"]), best["overlap"], coarse_ratio=cr, factor_prec=factor_prec,
                          coarse_iters=ci)
            torch.cuda.synchronize()
            su = time.perf_counter() - t0
            t0 = time.perf_counter()
            _, stats = o.solve(b_sample, tol=tol, restart=restart, basis_prec=helm.PREC_FP32, allow_notconv=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            o.close()
            conv = all(s_["converged"] for s_ in stats)
            ctrials.append(dict(coarse_ratio=cr, coarse_iters=ci, setup_s=su, solve_s=dt, converged=conv,
                                iterations=max(s_["iterations"] for s_ in stats)))
        cbest = min((t for t in ctrials if t["converged"]), key=lambda t: t["solve_s"])
        out.update(coarse_ratio=cbest["coarse_ratio"], coarse_iters=cbest["coarse_iters"], coarse_trials=ctrials)
    if knobs:
        o = helm.Oras(grid, tuple(best["parts"]), best["overlap"], coarse_ratio=out["coarse_ratio"],
                      factor_prec=factor_prec, coarse_iters=out["coarse_iters"])
        kn = tune_knobs(ctx, o, b_sample, restart, tol)
        o.close()
        out.update(knobs=kn["best"], knob_trials=kn["trials"])
    cache[key] = out
    save_cache(cache_path, cache)
    return dict(out, cached=False)


KNOB_GRID = [{"tc_stages": st, "tc_flow": fl} for fl in (1, 0) for st in (3, 4, 5)]


def apply_knobs(ctx, knobs):
    """Set the plane-sweep knobs of a tuning result on the context."""
    ctx.set_tuning(helm.TUNE_TC_STAGES, int(knobs.get("tc_stages", 0)))
    ctx.set_tuning(helm.TUNE_TC_FLOW, int(knobs.get("tc_flow", 1)))


def tune_knobs(ctx, oras, b_sample, restart=30, tol=1e-6, grid_=None):
    """Time a sample solve under every plane-sweep setting of ``grid_`` (default :data:`KNOB_GRID`) on the
    given factors (each setting solved twice, the second solve timed, so that captured iteration graphs
    are not charged); leaves the fastest setting on the context and returns it with the trials."""
    import torch
    trials = []
    for kn in (grid_ or KNOB_GRID):
        apply_knobs(ctx, kn)
        oras.solve(b_sample, tol=tol, restart=restart, basis_prec=helm.PREC_FP32, allow_notconv=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, stats = oras.solve(b_sample, tol=tol, restart=restart, basis_prec=helm.PREC_FP32, allow_notconv=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        trials.append(dict(kn, solve_s=dt, converged=all(s["converged"] for s in stats)))
    best = min((t for t in trials if t["converged"]), key=lambda t: t["solve_s"])
    kn = {k: best[k] for k in ("tc_stages", "tc_flow")}
    apply_knobs(ctx, kn)
    return {"best": kn, "trials": trials}
