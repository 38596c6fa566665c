#!/usr/bin/env python
"""Throughput benchmark: right-hand sides solved per second to relative residual 1e-6.

Workload (default): the linear-gradient model c(z) = 1500 + 0.6 z m/s on a
112^3 grid (h = 25 m, 8-node absorbing layers on the sides and bottom,
Dirichlet top), f = 5 Hz, 16 unit point sources at seeded distinct positions
on the plane z = 100 m, two-level ORAS with 4 x 4 x 4 boxes, overlap 2,
coarse grid 4x coarser (29^3), flexible GMRES(30) to 1e-6.

One step = one batched solve of the 16 right-hand sides with the ORAS factors
resident (the paper's T_GM; setup is reported separately).  The timed path
is the mixed-precision batched solver: complex64 local factors, sweeps and
Krylov basis, FP64 Hessenberg least squares, FP64 coarse factors and FP64
true residual.  The plain FP64 single-right-hand-side solve on the GPU is
measured beside it.  Every factor plane is read twice per preconditioner
application and the factors (~15 GB) are far larger than L2, so no L2 flush
is needed between steps.

``--impl reference`` solves the same workload with the FP64 CPU oracle on
the host cores instead (right-hand sides solved in full; one step = one
oracle FGMRES iteration).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if "reference" in sys.argv or "--impl=reference" in sys.argv:
    # the oracle arm: single-threaded BLAS in this process (set before numpy loads); its parallelism is the
    # process pool of local solves
    for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(_v, "1")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_14921_gb300 import synth  # noqa: E402

# the headline metric, the same on the library's line and the reference (oracle) line
METRIC = "RHS solved/s to rel-res 1e-6 (mixed batched vs FP64 plain GPU)"
# DRAM bytes per launch over algorithmic bytes, per kernel family (ncu, TF32 factors)
TRAFFIC_RATIO = {"sweep_flow": 0.994, "sweep_gemm_tc": 1.037}
# the autotuner's cache of tuned problem classes (decomposition, coarse level, sweep knobs)
TUNE_CACHE = os.path.join(ROOT, "paper_2103_14921_gb300", "tuned.json")

WORKLOADS = {
    "lg112": dict(desc="linear-gradient 112^3, 5 Hz, 16 RHS, two-level ORAS 4x4x4 ov2 r4, FGMRES(30) tol 1e-6",
                  n=112, h=25.0, f=5.0, c0=1500.0, alpha=0.6, npml=8, parts=(4, 4, 4), overlap=2, coarse=4,
                  nrhs=16, src_k=3, seed=synth.workload_seed(2), restart=30, tol=1e-6),
    "lg64": dict(desc="linear-gradient 64^3, 5 Hz, 16 RHS, two-level ORAS 2x2x2 ov2 r4, FGMRES(30) tol 1e-6",
                 n=64, h=25.0, f=5.0, c0=1500.0, alpha=0.6, npml=8, parts=(2, 2, 2), overlap=2, coarse=4,
                 nrhs=16, src_k=3, seed=synth.workload_seed(2), restart=30, tol=1e-6),
    # same plane sizes as lg112 (1024-node fine planes, 841-node coarse planes) on a 24-plane slab: a few GB
    # of factors, the size ncu full-section captures of single kernels are taken on
    "slab112": dict(desc="linear-gradient 112x112x24 slab, 5 Hz, 16 RHS, two-level ORAS 4x4x1 ov2 r4, FGMRES(30)",
                    n=112, nz=24, h=25.0, f=5.0, c0=1500.0, alpha=0.6, npml=8, parts=(4, 4, 1), overlap=2, coarse=4,
                    nrhs=16, src_k=3, seed=synth.workload_seed(2), restart=30, tol=1e-6),
    "lg48": dict(desc="linear-gradient 48^3, 3 Hz, 1 RHS, one-level ORAS 2x2x2 ov2, GMRES(30) tol 1e-6",
                 n=48, h=25.0, f=3.0, c0=1500.0, alpha=0.6, npml=8, parts=(2, 2, 2), overlap=2, coarse=0,
                 nrhs=1, src_k=None, seed=synth.workload_seed(1), restart=30, tol=1e-6),
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def sources(W):
    n = W["n"]
    if W["src_k"] is None:
        return [(n // 2, n // 2, n // 2)]
    return synth.source_plane_positions(n, n, W["npml"], W["src_k"], W["nrhs"], W["seed"])


def velocity(W):
    return synth.linear_gradient(W["n"], W["n"], W.get("nz", W["n"]), W["h"], W["c0"], W["alpha"])


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- CPU oracle sample

def oracle_sample(W, iters_per_rhs, weights, repeats=1):
    """Time the FP64 oracle's per-iteration work on this workload and scale it to RHS/s.

    Sample: one matrix-free A u on the full grid (two per iteration: A z_j and
    v - A q), one ORAS local solve (``splu`` of the largest box, as the oracle's
    ORAS class builds it) scaled by the number of boxes, and one Arnoldi pass
    (dot + axpy over the full grid) scaled by the mean Krylov dimension.  The
    coarse solve is left out (it is small next to the local solves).
    """
    import numpy as np
    import scipy.sparse.linalg as spla
    from oracle.discretization import Problem, apply_A, neighbour_coefficients
    from oracle.schwarz import decompose, local_operator

    n, nz = W["n"], W.get("nz", W["n"])
    prob = Problem(n, n, nz, W["h"], W["f"], velocity(W), npml=W["npml"], weights=weights)
    boxes = decompose((n, n, nz), W["parts"], W["overlap"])
    big = max(boxes, key=lambda b: b.size)
    t0 = time.perf_counter()
    coef = neighbour_coefficients(prob)
    Ai = local_operator(prob, big, "oras", coef)
    lu = spla.splu(Ai.tocsc())
    setup_box = time.perf_counter() - t0
    u = synth.random_complex((nz, n, n), 1)
    rb = synth.random_complex((big.size,), 2)
    out = []
    jbar = W["restart"] / 2.0
    # cores actually used by the timed work (numpy / scipy may run BLAS threads): process CPU time over wall time
    cpu0, wall0 = time.process_time(), time.perf_counter()
    for _ in range(repeats):
        t = time.perf_counter()
        apply_A(prob, u)
        t_mv = time.perf_counter() - t
        t = time.perf_counter()
        lu.solve(rb)
        t_ls = time.perf_counter() - t
        v = u.ravel()
        t = time.perf_counter()
        h = np.vdot(v, v)
        v2 = v - h * v
        t_ar = time.perf_counter() - t
        t_it = 2 * t_mv + len(boxes) * t_ls + 2 * (jbar + 1) * t_ar
        out.append(t_it)
    cores = max(1, round((time.process_time() - cpu0) / max(time.perf_counter() - wall0, 1e-9)))
    t_it = statistics.median(out)
    rhs_per_s = 1.0 / (iters_per_rhs * t_it)
    return {
        "value": rhs_per_s, "unit": "RHS/s", "cores": cores, "kind": "oracle",
        "sample": (f"oracle FP64 per-iteration work on the {n}^3 grid (2 matrix-free A u, {len(boxes)} x one splu "
                   f"local solve of a {big.dims[0]}x{big.dims[1]}x{big.dims[2]} box, Arnoldi at mean Krylov dim "
                   f"{jbar:.0f}; coarse solve left out) = {t_it:.3f} s/iteration, times {iters_per_rhs:.1f} "
                   f"iterations per RHS; box factorisation {setup_box:.1f} s not counted"),
        "t_iteration_s": t_it, "host_cpus": os.cpu_count(),
    }


# FGMRES restart of the request stream: the flexible basis of a 160^3 set with 64 columns then takes about 80 GB,
# so that the largest requests fit beside others in the 150 GB budget
SERVE_RESTART = 15
# the request stream's coarse problem is solved as in the paper, by 10 GMRES iterations with one-level ORAS on the
# coarse grid: a new factor set then needs no FP64 factorisation of the whole coarse grid (2.6 s of the 3.3 s set-up
# at 160^3), and nearly every request of the stream builds a new set
SERVE_COARSE_ITERS = 10
# a serving phase gives up waiting after this long (the requests still open are reported as timed out)
SERVE_PHASE_LIMIT_S = 240.0


class RequestMix:
    """The serving workload: seeded requests over cubic grids n in {48, 64, ..., 160} (h = 25 m, 8-node
    absorbing layers), 4 seeded layered models per size (3-6 layers, 1500-4500 m/s), f in {2, 3, 4, 5, 6} Hz,
    1-64 point sources each at seeded interior nodes; two-level ORAS with boxes of about 24 nodes per axis, coarse
    ratio 4 with the paper's inexact coarse solve (10 inner GMRES iterations), TF32 factors, FGMRES(15) to 1e-6.  Right-hand sides are made on the device when a request is submitted
    and released when it is done."""

    SIZES = (48, 64, 80, 96, 112, 128, 144, 160)

    def __init__(self, seed, count):
        import numpy as np
        rng = np.random.default_rng(seed)
        self.items = []
        for _ in range(count):
            n = int(rng.choice(self.SIZES))
            nr = int(rng.integers(1, 65))
            pos = rng.integers(8, n - 8, size=(nr, 3))
            pos[:, 2] = np.minimum(pos[:, 2], n - 9)
            self.items.append(dict(n=n, mid=int(rng.integers(0, 4)), f=float(rng.choice([2.0, 3.0, 4.0, 5.0, 6.0])),
                                   pos=[tuple(int(v) for v in p) for p in pos]))
        self.models = {}

    def model(self, n, mid):
        import torch
        key = (n, mid)
        if key not in self.models:
            self.models[key] = torch.from_numpy(synth.layered(n, n, n, 25.0, seed=synth.workload_seed(5) * 10 + 7 * n + mid,
                                                              vmin=1500.0, vmax=4500.0))
        return self.models[key]


def log(msg):
    """Progress on stderr (the JSON line is the only stdout output)."""
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def serve_phase(helm, sv, mix, items, weights, arrivals=None):
    """Submit `items` (at the given arrival offsets in seconds, or all at once), wait for all; returns the
    per-request stats and the wall time."""
    import ctypes as C
    import torch
    t0 = time.perf_counter()
    deadline = t0 + SERVE_PHASE_LIMIT_S
    live = {}
    out = []

    def reap(block):
        for tk in list(live):
            if block:
                try:
                    s = sv.wait(tk, timeout_s=max(1.0, deadline - time.perf_counter()))
                except TimeoutError:   # reported as not done; the phase ends
                    s = dict(sv.poll(tk)[1], done=False)
                    out.append(dict(s, **live.pop(tk), timed_out=True))
                    continue
            else:
                s = sv.poll(tk)[1]
            if s["done"]:
                out.append(dict(s, **live.pop(tk)))

    for i, it in enumerate(items):
        if arrivals is not None:
            while time.perf_counter() - t0 < arrivals[i]:
                reap(False)
                time.sleep(0.0005)
        n = it["n"]
        b = torch.zeros((n, n, n, len(it["pos"])), dtype=torch.complex128, device="cuda")
        for r, (ii, jj, kk) in enumerate(it["pos"]):
            b[kk, jj, ii, r] = 1.0 / 25.0 ** 3
        gd = helm.GridDesc(n, n, n, 25.0, it["f"], 8, 1e-3, helm.TOP_DIRICHLET, (C.c_double * 7)(*weights))
        p = max(2, round(n / 24))
        od = helm.OrasDesc(p, p, p, 2, 4, 0, helm.PREC_TF32, SERVE_COARSE_ITERS, 1)
        tk = sv.submit(1000 * n + it["mid"], gd, mix.model(n, it["mid"]), od, b, torch.empty_like(b), tol=1e-6,
                       restart=SERVE_RESTART, basis_prec=helm.PREC_FP32)
        live[tk] = dict(nrhs=len(it["pos"]), n=n, f=it["f"], model=it["mid"])
        del b
    reap(True)
    return out, time.perf_counter() - t0


def run_serving(helm, device, stream, weights, args):
    """The request stream through helm_submit/helm_poll under a 150 GB HBM budget with 64 column slots per
    factor set: first the saturated request rate (a burst of requests submitted at once), then Poisson
    arrivals at 0.8 x that rate (the main figure: RHS/s, p50/p99 latency) and a short sweep of rates."""
    import numpy as np
    mix = RequestMix(synth.workload_seed(5), args.serve_requests + args.serve_burst + 2 * args.serve_sweep)
    ctx = helm.Context(device, stream=stream.cuda_stream, budget_bytes=150 << 30)
    items = mix.items
    res = {"mix": RequestMix.__doc__.split("\n\n")[0].replace("\n", " "), "budget_gb": 150, "slots_per_batch": 64}

    def summary(st, wall, rate=None):
        done = [s_ for s_ in st if not s_.get("timed_out")]
        lat = [s_["latency_ms"] for s_ in done] or [float("nan")]
        rhs = sum(s_["nrhs"] for s_ in done if s_["status"] == helm.OK)
        ok = sum(1 for s_ in done if s_["status"] == helm.OK)
        return {"requests": len(st), "ok": ok, "timed_out": sum(1 for s_ in st if s_.get("timed_out")),
                "rhs": rhs, "wall_s": wall, "rhs_per_s": rhs / wall,
                "requests_per_s": len(done) / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "arrival_rate_per_s": rate,
                "factors_reused": sum(1 for s_ in st if s_["factors_reused"]),
                "not_ok": [{k: s_[k] for k in ("n", "f", "model", "nrhs", "status", "iterations_max",
                                               "true_relres_max", "latency_ms")}
                           for s_ in done if s_["status"] != helm.OK]}

    with helm.Server(ctx, slots_per_batch=64) as sv:
        pos = 0
        burst = items[pos:pos + args.serve_burst]
        pos += args.serve_burst
        log(f"serving: burst of {len(burst)} requests")
        st, wall = serve_phase(helm, sv, mix, burst, weights)
        sat = max(1e-3, sum(1 for s_ in st if not s_.get("timed_out")) / wall)
        res["saturated"] = summary(st, wall)
        log(f"serving: saturated {sat:.2f} requests/s ({res['saturated']['rhs_per_s']:.1f} RHS/s) in {wall:.1f} s")
        rng = np.random.default_rng(synth.workload_seed(5) + 1)
        lam = 0.8 * sat
        main = items[pos:pos + args.serve_requests]
        pos += args.serve_requests
        arr = np.cumsum(rng.exponential(1.0 / lam, len(main)))
        log(f"serving: {len(main)} requests at {lam:.2f} requests/s")
        st, wall = serve_phase(helm, sv, mix, main, weights, arr)
        res["main"] = summary(st, wall, lam)
        log(f"serving: main phase {wall:.1f} s, p50 {res['main']['p50_ms']:.0f} ms, p99 {res['main']['p99_ms']:.0f} ms")
        sweep = []
        for frac in (0.5, 1.2):
            part = items[pos:pos + args.serve_sweep]
            pos += args.serve_sweep
            if not part:
                break
            arr = np.cumsum(rng.exponential(1.0 / (frac * sat), len(part)))
            st, wall = serve_phase(helm, sv, mix, part, weights, arr)
            sweep.append(dict(summary(st, wall, frac * sat), rate_fraction_of_saturated=frac))
        res["rate_sweep"] = sweep
    res.update({k: res["main"][k] for k in ("requests", "ok", "rhs", "wall_s", "rhs_per_s", "p50_ms", "p99_ms",
                                             "arrival_rate_per_s")})
    ctx.close()
    return res


def factor_roofline(ctx, o, peaks):
    """Tensor-pipe roofline of the plane factorisation's rank-128 updates (family gj_update_tc) from the
    profile of a factorisation of ``o``: algorithmic flops = for every box, plane and 128-column panel,
    8 (rows outside the panel) x m x (panel columns below m) real flops per complex product, times 3 for the
    three-product TF32 split; peak = the measured dense BF16 rate halved (TF32 runs at half the BF16 rate)."""
    q = ctx.profile_query("gj_update_tc")
    if not q:
        return None
    nl, ms, by = q
    fl = 0.0
    nb = o.box_info(-1)[0]
    for b in range(nb):
        _, _, d = o.box_info(b)
        m = d[0] * d[1]
        for j0 in range(0, m, 128):
            w = min(128, m - j0)
            fl += d[2] * 3 * 8.0 * (m - w) * m * w
    tf32 = float(peaks.get("bf16_tflops", 1900.0)) / 2.0
    ach = fl / (ms / 1e3) / 1e12
    out = {"kernel": "gj_update_tc", "bound": "tensor", "launches": nl, "ms_total": ms,
           "achieved_tflops": ach, "peak_tflops": tf32, "peak_source": "measured bf16 / 2 (TF32)",
           "frac": ach / tf32, "flops": fl, "GBps": by / (ms / 1e3) / 1e9}
    # the rest of the set-up: tensor-core panel steps (fine planes), block-pivot panels and updates of the
    # FP64 coarse problem on the CUDA cores
    for fam in ("gj_panel_tc", "gj_diag", "gj_panel", "gj_update"):
        q = ctx.profile_query(fam)
        out[fam + "_ms"] = q[1] if q else None
    return out


def _sweep_roofline(ctx, fam, hbm, tf32_peak, nrhs, W_planes):
    """Roofline figures of a profiled persistent-sweep family: HBM bytes and TF32 flops per second."""
    q = ctx.profile_query(fam)
    if not q:
        return None
    nl, ms, by = q
    fl = W_planes * nrhs * 8.0     # complex multiply-adds of the plane products, 8 real flops each, per launch
    return {"kernel": fam, "launches": nl, "avg_launch_us": 1000.0 * ms / nl, "GBps": by / (ms / 1e3) / 1e9,
            "hbm_frac": by / (ms / 1e3) / 1e9 / hbm, "tflops": fl * nl / (ms / 1e3) / 1e12,
            "tensor_frac_tf32": fl * nl / (ms / 1e3) / 1e12 / tf32_peak}


def _plane_entries(o):
    """Sum over the fine boxes and both sweeps of m^2 per plane step (the entries one apply multiplies)."""
    tot = 0
    for b in range(o.box_info(-1)[0]):
        _, _, d = o.box_info(b)
        tot += (d[0] * d[1]) ** 2 * (2 * d[2] - 1)
    return tot


def run_thrust_fold(helm, ctx, stream, weights, peaks, retune=False):
    """The Overthrust stand-in: thrust-fold model 256 x 256 x 96 (h = 25 m, 8 folded layers 2000-6000 m/s, two
    dipping faults), 5 Hz, 64 sources on an 8 x 8 node array at z = 50 m, decomposition and sweep knobs picked
    by the autotuner (in-plane cores 16-24, overlap 2-4), TF32 tensor-core local solves, two-level ORAS
    (the coarse level chosen by the tuner between ratio 8 solved exactly and ratio 4 solved as in the paper by
    10 inner GMRES iterations: the exact FP64 coarse plane LU of ratio 4 would cost ~1.5e13 FP64 flops), FGMRES(30)
    to 1e-6, the 64 right-hand sides solved as two batches of 32 (the flexible basis of all 64 at once would
    not fit next to the factors)."""
    import numpy as np
    import torch
    from paper_2103_14921_gb300 import tune
    nx, ny, nz, h, f = 256, 256, 96, 25.0, 5.0
    c = synth.thrust_fold(nx, ny, nz, h, synth.workload_seed(3))
    grid = helm.Grid(ctx, nx, ny, nz, h, f, c, npml=8, weights=weights)
    pos = synth.source_array_positions(nx, ny, 8, 1, 8)
    b = torch.from_numpy(synth.point_sources(nx, ny, nz, h, pos)).cuda()
    chunk = 32
    t = time.perf_counter()
    # the autotuner's choice for this problem class is kept in the package's tuning cache (written by the
    # tuner itself on a GB300); --retune times every candidate again
    tr = tune.tune(ctx, grid, b[..., :8].contiguous(), factor_prec=helm.PREC_TF32, coarse_ratio=8, nrhs=chunk,
                   max_trials=4, knobs=True, coarse_opts=[(8, 0), (4, 10)],
                   cache_path=None if retune else TUNE_CACHE)
    tune_s = time.perf_counter() - t
    t = time.perf_counter()
    o = helm.Oras(grid, tuple(tr["parts"]), tr["overlap"], coarse_ratio=tr.get("coarse_ratio", 8),
                  factor_prec=helm.PREC_TF32, coarse_iters=tr.get("coarse_iters", 0))
    setup_s = time.perf_counter() - t
    kw = dict(tol=1e-6, restart=30, flexible=True, basis_prec=helm.PREC_FP32)
    x = torch.empty_like(b)
    b0 = b[..., :chunk].contiguous()
    x0 = torch.empty_like(b0)
    o.solve(b0, x0, **kw)                        # warm-up: workspace and iteration graphs
    ctx.profile(True, only=["sweep_flow"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record(stream)
    for c0 in range(0, b.shape[-1], chunk):
        bc = b[..., c0:c0 + chunk].contiguous()
        xc = torch.empty_like(bc)
        _, st = o.solve(bc, xc, **kw)
        x[..., c0:c0 + chunk] = xc
        stats += st
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    tf32 = float(peaks.get("bf16_tflops", 1900.0)) / 2.0
    roof = _sweep_roofline(ctx, "sweep_flow", hbm, tf32, chunk, _plane_entries(o))
    ctx.profile(False)
    tune.apply_knobs(ctx, {"tc_stages": 0, "tc_flow": 1})
    out = {"workload": "thrust-fold 256x256x96, 5 Hz, 64 RHS (8x8 node array, z = 50 m), autotuned ORAS "
                       "(boxes, overlap, coarse level, sweep knobs), TF32 factors, FGMRES(30) tol 1e-6, 2 batches of 32",
           "value": b.shape[-1] / (ms / 1e3), "unit": "RHS/s", "solve_s": ms / 1e3, "setup_s": setup_s,
           "tune_s": tune_s, "parts": tr["parts"], "overlap": tr["overlap"], "knobs": tr.get("knobs"),
           "coarse_ratio": tr.get("coarse_ratio"), "coarse_iters": tr.get("coarse_iters"),
           "tune_cached": tr.get("cached", False), "tune_trials": tr.get("trials"),
           "iterations_max": max(s_["iterations"] for s_ in stats),
           "iterations_mean": float(np.mean([s_["iterations"] for s_ in stats])),
           "max_true_relres": max(s_["true_relres"] for s_ in stats),
           "converged": all(s_["converged"] for s_ in stats), "sweep_roofline": roof}
    del o, x, b, b0, x0, grid
    torch.cuda.synchronize()
    return out


# box decompositions the attenuating workload's autotuner times (overlap 2): cores of 20, 27, 32 and 40 nodes
# in x and y, 20, 40 or all 80 planes in z
ATTEN_CANDS = [((8, 8, 4), 2), ((6, 6, 4), 2), ((5, 5, 4), 2), ((4, 4, 4), 2), ((4, 4, 2), 2), ((4, 4, 1), 2)]


def run_attenuating(helm, ctx, stream, weights, peaks, retune=False):
    """The attenuating workload: linear gradient with c (1 - i/(2Q)), Q = 100, on 160 x 160 x 80, frequencies
    3, 4 and 6 Hz, 128 sources on the plane z = 100 m (seeded), two-level ORAS with overlap 2 and coarse ratio
    4, the box decomposition picked by the autotuner at the hardest frequency (6 Hz, 8 sample columns, the
    decompositions of ATTEN_CANDS; the choice is cached), TF32 factors, all 128 right-hand sides in one batch
    (one persistent sweep launch per preconditioner apply, graph-replayed FGMRES(30) iterations), tol 1e-6.
    Per frequency: set-up and solve time, every column's FP64 true residual; at 6 Hz two columns are also
    solved by the plain FP64 path (8 x 8 x 4 boxes) and the mixed solution's relative difference from it is
    reported."""
    import torch
    from paper_2103_14921_gb300 import tune
    nx, ny, nz, h = 160, 160, 80, 25.0
    c = synth.linear_gradient(nx, ny, nz, h, 1500.0, 0.6, Q=100.0)
    pos = synth.source_plane_positions(nx, ny, 8, 3, 128, synth.workload_seed(4))
    b = torch.from_numpy(synth.point_sources(nx, ny, nz, h, pos)).cuda()
    kw = dict(tol=1e-6, restart=30, flexible=True, basis_prec=helm.PREC_FP32)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    tf32 = float(peaks.get("bf16_tflops", 1900.0)) / 2.0
    t = time.perf_counter()
    grid = helm.Grid(ctx, nx, ny, nz, h, 6.0, c, npml=8, weights=weights)
    tr = tune.tune(ctx, grid, b[..., :8].contiguous(), factor_prec=helm.PREC_TF32, coarse_ratio=4,
                   nrhs=b.shape[-1], cands=ATTEN_CANDS, max_trials=len(ATTEN_CANDS),
                   cache_path=None if retune else TUNE_CACHE)
    tune_s = time.perf_counter() - t
    parts, ov = tuple(tr["parts"]), tr["overlap"]
    del grid
    freqs = {}
    tot_ms = 0.0
    for f in (3.0, 4.0, 6.0):
        grid = helm.Grid(ctx, nx, ny, nz, h, f, c, npml=8, weights=weights)
        torch.cuda.synchronize()
        t = time.perf_counter()
        o = helm.Oras(grid, parts, ov, coarse_ratio=4, factor_prec=helm.PREC_TF32)
        setup_s = time.perf_counter() - t
        x = torch.empty_like(b)
        ctx.profile(True, only=["sweep_flow"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = o.solve(b, x, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        tot_ms += ms
        roof = _sweep_roofline(ctx, "sweep_flow", hbm, tf32, b.shape[-1], _plane_entries(o))
        ctx.profile(False)
        rec = {"setup_s": setup_s, "solve_s": ms / 1e3, "rhs_per_s": b.shape[-1] / (ms / 1e3),
               "iterations": [s_["iterations"] for s_ in st], "true_relres": [s_["true_relres"] for s_ in st],
               "converged": all(s_["converged"] for s_ in st), "sweep_roofline": roof}
        if f == 6.0:
            del o
            torch.cuda.synchronize()
            # the FP64 reference solves the same system with the smaller 8 x 8 x 4 boxes: FP64 factors of the
            # tuned boxes would take ~10x the CUDA-core factor time, and any decomposition converges to the
            # same solution within the tolerance
            o64 = helm.Oras(grid, (8, 8, 4), 2, coarse_ratio=4, factor_prec=helm.PREC_FP64)
            cols = [0, 127]
            x64, s64 = o64.solve(b[..., cols].contiguous(), tol=1e-6, restart=30, basis_prec=helm.PREC_FP64)
            rec["fp64_vs_mixed"] = {str(cc): float(torch.linalg.vector_norm(x[..., cc] - x64[..., k]) /
                                                   torch.linalg.vector_norm(x64[..., k]))
                                    for k, cc in enumerate(cols)}
            rec["fp64_setup_s"] = o64.setup_seconds
            del o64, x64
        freqs[f"{f:g}Hz"] = rec
        del x, grid
        torch.cuda.synchronize()
    n_all = 3 * b.shape[-1]
    return {"workload": "attenuating linear gradient (Q = 100) 160x160x80, 3/4/6 Hz x 128 RHS, two-level ORAS "
                        "autotuned boxes, ov2 r4, TF32 factors, FGMRES(30) tol 1e-6, one batch of 128 per frequency",
            "value": n_all / (tot_ms / 1e3), "unit": "RHS/s", "solve_s": tot_ms / 1e3, "parts": list(parts),
            "overlap": ov, "tune_s": tune_s, "tune_cached": tr.get("cached", False), "tune_trials": tr.get("trials"),
            "per_frequency": freqs}


def _host_info():
    """Host CPU description: logical CPUs, the ones this process may run on, and the model name."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "affinity_cpus": len(os.sched_getaffinity(0)), "cpu_model": model}


def _threads(pids):
    out = []
    for pid in pids:
        try:
            out += [int(t) for t in os.listdir(f"/proc/{pid}/task")]
        except OSError:
            pass
    return out


def _pin_all_threads(cpus, pids=()):
    """Restrict every thread of this process and of the processes `pids` to `cpus`; returns the previous
    sets."""
    prev = {}
    for tid in _threads(["self", *pids]):
        try:
            prev[tid] = os.sched_getaffinity(tid)
            os.sched_setaffinity(tid, cpus)
        except OSError:
            pass
    return prev


def _unpin_all_threads(prev, default):
    for tid, cpus in prev.items():
        try:
            os.sched_setaffinity(tid, cpus or default)
        except OSError:
            pass


def _cpu_seconds(pids):
    """User + system CPU seconds of this process and of the processes `pids` (from /proc)."""
    tot = time.process_time()
    tick = os.sysconf("SC_CLK_TCK")
    for pid in pids:
        try:
            f = open(f"/proc/{pid}/stat").read().rsplit(")", 1)[1].split()
            tot += (int(f[11]) + int(f[12])) / tick
        except (OSError, IndexError, ValueError):
            pass
    return tot


def oracle_timed_solve(prob, M, b, tol, restart, flexible, maxit=1000):
    """One oracle (F)GMRES solve with a timestamp at every preconditioner application: returns the
    solution, the oracle's info, the wall time, the per-iteration times and the cores used (process CPU
    time over wall time)."""
    from oracle.discretization import apply_A
    from oracle.krylov import gmres
    shape = (prob.nz, prob.ny, prob.nx)
    marks = []

    def aM(v):
        marks.append(time.perf_counter())
        return M.apply(v)

    def aA(u):
        return apply_A(prob, u.reshape(shape)).ravel()

    pids = M.pool.pids() if M.pool is not None else []
    cpu0, t0 = _cpu_seconds(pids), time.perf_counter()
    x, info = gmres(aA, b.ravel(), aM, tol=tol, restart=restart, maxit=maxit, flexible=flexible)
    t1 = time.perf_counter()
    cores = (_cpu_seconds(pids) - cpu0) / max(t1 - t0, 1e-9)
    its = [marks[i + 1] - marks[i] for i in range(len(marks) - 1)] + ([t1 - marks[-1]] if marks else [])
    return x, info, t1 - t0, its, cores


def run_reference(args, W):
    """The FP64 CPU oracle solving the workload on the host cores (the reference has no installable
    implementation: it is a paper).  Nothing from the library is imported or loaded here: weights, operator,
    ORAS set-up (splu local solves, exact coarse solve) and FGMRES are all the oracle's.

    One step = one oracle FGMRES iteration of a real solve of the workload (one two-level preconditioner
    application with its coarse solve, one matrix-free A u, the Arnoldi and Givens work); the warm-up and
    timed steps are consecutive iterations of solves of the workload's right-hand sides, each run to
    convergence.  value = right-hand sides solved / their total solve wall time (set-up reported apart).
    Beside it: the same solve's iterations on one core, and the plain-method workload (48^3, FP64,
    one-level ORAS 2x2x2, GMRES(30)) solved in full on all cores and on one core."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle.discretization import Problem, apply_A
    from oracle.schwarz import ORAS
    from oracle.weights import fit_weights

    host = _host_info()
    all_cpus = os.sched_getaffinity(0)
    weights = fit_weights()
    n, nz = W["n"], W.get("nz", W["n"])
    prob = Problem(n, n, nz, W["h"], W["f"], velocity(W), npml=W["npml"], weights=weights)
    b_all = synth.point_sources(n, n, nz, W["h"], sources(W))
    nrhs = b_all.shape[-1]
    workers = len(all_cpus)
    t = time.perf_counter()
    M = ORAS(prob, W["parts"], W["overlap"], coarse_ratio=W["coarse"], local="splu", workers=workers)
    setup_s = time.perf_counter() - t
    flexible = W["coarse"] > 0
    need = args.warmup + args.steps
    its_all, solves = [], []
    col = 0
    while col < nrhs and (len(its_all) < need or not solves):
        x, info, wall, its, cores = oracle_timed_solve(prob, M, b_all[..., col], W["tol"], W["restart"], flexible)
        solves.append({"column": col, "wall_s": wall, "iterations": info["iterations"],
                       "true_relres": info["true_residual"], "converged": info["converged"], "cores": cores})
        its_all += its
        col += 1
    timed = its_all[args.warmup:need] or its_all[-args.steps:]
    value = len(solves) / sum(s_["wall_s"] for s_ in solves)
    cores_used = max(1, round(statistics.median(s_["cores"] for s_ in solves)))
    # the same iterations with every thread of the process on one CPU
    one = None
    try:
        prev = _pin_all_threads({min(all_cpus)}, M.pool.pids() if M.pool is not None else ())
        try:
            _, _, _, its1, _ = oracle_timed_solve(prob, M, b_all[..., col % nrhs], W["tol"], W["restart"],
                                                  flexible, maxit=3)
        finally:
            _unpin_all_threads(prev, all_cpus)
        it1 = statistics.median(its1)
        one = {"cores": 1, "s_per_iteration": it1, "iterations_timed": len(its1),
               "rhs_per_s_at_all_core_iteration_count": 1.0 / (it1 * statistics.mean(s_["iterations"] for s_ in solves))}
    except Exception as exc:
        one = {"error": repr(exc)}
    M.close()
    del M
    # the plain-method workload in full (48^3, FP64, one-level ORAS 2x2x2, GMRES(30)), all cores and one core
    plain = None
    try:
        W1 = WORKLOADS["lg48"]
        if W1 is W:
            raise LookupError("the plain-method workload is the timed workload itself")
        p1 = Problem(W1["n"], W1["n"], W1["n"], W1["h"], W1["f"], velocity(W1), npml=W1["npml"], weights=weights)
        b1 = synth.point_sources(W1["n"], W1["n"], W1["n"], W1["h"], sources(W1))[..., 0]
        t = time.perf_counter()
        M1 = ORAS(p1, W1["parts"], W1["overlap"], coarse_ratio=0, local="splu", workers=workers)
        su1 = time.perf_counter() - t
        _, inf1, wall1, _, c1 = oracle_timed_solve(p1, M1, b1, W1["tol"], W1["restart"], False)
        prev = _pin_all_threads({min(all_cpus)}, M1.pool.pids() if M1.pool is not None else ())
        try:
            _, inf1b, wall1b, _, _ = oracle_timed_solve(p1, M1, b1, W1["tol"], W1["restart"], False)
        finally:
            _unpin_all_threads(prev, all_cpus)
            M1.close()
        plain = {"workload": W1["desc"], "setup_s": su1, "solve_s": wall1, "iterations": inf1["iterations"],
                 "true_relres": inf1["true_residual"], "rhs_per_s": 1.0 / wall1, "cores": max(1, round(c1)),
                 "one_core": {"solve_s": wall1b, "iterations": inf1b["iterations"], "rhs_per_s": 1.0 / wall1b}}
    except Exception as exc:
        plain = {"error": repr(exc)}
    sample = (f"oracle FP64 two-level ORAS-FGMRES (splu local solves in {workers} worker processes, exact "
              f"coarse solve) solving "
              f"{len(solves)} of the workload's right-hand sides in full on the host cores: "
              f"{sum(s_['iterations'] for s_ in solves)} iterations in {sum(s_['wall_s'] for s_ in solves):.1f} s "
              f"(set-up {setup_s:.1f} s apart); a step is one of those iterations")
    try:
        maps = open("/proc/self/maps").read()
    except OSError:
        maps = ""
    cb = {"value": value, "unit": "RHS/s", "cores": cores_used, "kind": "oracle", "sample": sample, "workers": workers,
          "setup_s": setup_s, "solves": solves, "one_core": one, "plain_method_48": plain, "host": host,
          "product_library_loaded": "libhelm" in maps}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": W["desc"], "grid": [n, n, nz], "nrhs": W["nrhs"]},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU arm

def run_gpu(args, W):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2103_14921_gb300 import build, helm
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    stream = torch.cuda.current_stream()
    ctx = helm.Context(local, stream=stream.cuda_stream)
    n, nz = W["n"], W.get("nz", W["n"])
    weights = helm.fit_weights()
    grid = helm.Grid(ctx, n, n, nz, W["h"], W["f"], velocity(W), npml=W["npml"], weights=weights)
    pos = sources(W)
    nrhs = len(pos)
    b_host = synth.point_sources(n, n, nz, W["h"], pos)
    b = torch.from_numpy(b_host).cuda()
    x = torch.empty_like(b)
    mixed_prec = helm.PREC_NAMES[args.factor_prec]
    t = time.perf_counter()
    oras = helm.Oras(grid, W["parts"], W["overlap"], coarse_ratio=W["coarse"], factor_prec=mixed_prec)
    setup_wall = time.perf_counter() - t
    setup_device = oras.setup_seconds
    log(f"headline: set-up {setup_wall:.2f} s")
    # the plane factorisation's kernels, from a second, instrumented factorisation of the same problem
    factor = None
    if mixed_prec in (helm.PREC_TF32, helm.PREC_BF16):
        ctx.profile(True, only=["gj_update_tc", "gj_panel_tc", "gj_diag", "gj_panel", "gj_update"])
        of = helm.Oras(grid, W["parts"], W["overlap"], coarse_ratio=W["coarse"], factor_prec=mixed_prec)
        factor = factor_roofline(ctx, of, load_peaks()[0])
        ctx.profile(False)
        del of
        torch.cuda.synchronize()
    solve_kw = dict(tol=W["tol"], restart=W["restart"], flexible=True, basis_prec=helm.PREC_FP32)

    # the persistent tensor-core sweep (both sweeps, products and operand preparation, one launch per apply)
    roof_fam = "sweep_flow" if args.factor_prec in ("tf32", "bf16") else "sweep_gemv"
    # events around the roofline kernel only; enabled before the warm-up so that the iteration graphs
    # captured there already carry the event nodes the timed region reads
    ctx.profile(True, only=[roof_fam])
    for _ in range(args.warmup):
        oras.solve(b, x, **solve_kw)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True, only=[roof_fam])          # clears the totals; same selection, graphs stay valid
    l0 = ctx.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats_all = []
    for _ in range(args.steps):
        _, st = oras.solve(b, x, **solve_kw)
        stats_all.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = ctx.launches - l0
    elapsed_ms = e0.elapsed_time(e1)
    roof_meas = ctx.profile_query(roof_fam)
    ctx.profile(False)
    # per-family breakdown from one more, fully instrumented solve (outside the timed region)
    families = ("sweep_flow", "sweep_gemm_tc", "sweep_gemv", "sweep_prep", "coarse_sweep", "coarse_prep", "stencil",
                "stencil64", "arnoldi", "arnoldi_reorth", "oras_transfer", "coarse_restrict", "coarse_prolong",
                "krylov_misc")
    ctx.profile(True)
    oras.solve(b, x, **solve_kw)                # captures the iteration graphs with every family's events
    ctx.profile(True)                           # clears the totals
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    oras.solve(b, x, **solve_kw)
    b1.record(stream)
    torch.cuda.synchronize()
    breakdown_ms = b0.elapsed_time(b1)
    prof = {fam: ctx.profile_query(fam) for fam in families}
    ctx.profile(False)
    from paper_2103_14921_gb300 import replicas
    dev = torch.device("cuda", local)
    value, t_max_s = replicas.job_throughput(nrhs * args.steps, elapsed_ms / 1000.0, dev)
    t_max = 1000.0 * t_max_s
    iters = [s["iterations"] for s in stats_all[-1]]
    relres = max(s["true_relres"] for s in stats_all[-1])
    x_mixed = x.clone()

    log(f"headline: {args.steps} timed solves, {elapsed_ms / args.steps:.1f} ms each")
    # variant: bfloat16-stored local factors (the same solve, reported beside the headline path)
    variants = {}
    if args.factor_prec == "tf32" and not args.no_variants:
        ob = helm.Oras(grid, W["parts"], W["overlap"], coarse_ratio=W["coarse"], factor_prec=helm.PREC_BF16)
        xb = torch.empty_like(b)
        for _ in range(2):                      # first use runs eagerly, the second captures the graphs
            ob.solve(b, xb, **solve_kw)
        torch.cuda.synchronize()
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        kv = max(1, min(args.steps, 3))
        for _ in range(kv):
            _, stb = ob.solve(b, xb, **solve_kw)
        v1.record(stream)
        torch.cuda.synchronize()
        vb, _ = replicas.job_throughput(nrhs * kv, v0.elapsed_time(v1) / 1000.0, dev)
        err = float(torch.linalg.vector_norm(xb - x) / torch.linalg.vector_norm(x))
        variants["bf16_factors"] = {"value": vb, "unit": "RHS/s", "steps": kv,
                                    "iterations": [s_["iterations"] for s_ in stb],
                                    "max_true_relres": max(s_["true_relres"] for s_ in stb),
                                    "rel_l2_vs_tf32_solution": err}
        del ob, xb
        if W["coarse"]:
            # variant: the paper's own coarse solve (10 GMRES steps with one-level ORAS on the coarse grid)
            oi = helm.Oras(grid, W["parts"], W["overlap"], coarse_ratio=W["coarse"], factor_prec=mixed_prec,
                           coarse_iters=10, coarse_overlap=1)
            xi = torch.empty_like(b)
            for _ in range(2):
                oi.solve(b, xi, **solve_kw)
            torch.cuda.synchronize()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            kv = max(1, min(args.steps, 3))
            for _ in range(kv):
                _, sti = oi.solve(b, xi, **solve_kw)
            v1.record(stream)
            torch.cuda.synchronize()
            vi, _ = replicas.job_throughput(nrhs * kv, v0.elapsed_time(v1) / 1000.0, dev)
            err = float(torch.linalg.vector_norm(xi - x) / torch.linalg.vector_norm(x))
            variants["coarse_gmres10"] = {"value": vi, "unit": "RHS/s", "steps": kv, "setup_s": oi.setup_seconds,
                                          "iterations": [s_["iterations"] for s_ in sti],
                                          "max_true_relres": max(s_["true_relres"] for s_ in sti),
                                          "rel_l2_vs_exact_coarse_solution": err}
            del oi, xi
        # a frequency sweep of the same model and sources (three neighbouring frequencies): warm starts from
        # the previous frequency, and the next frequency's grid and factors built on a second context while
        # the current one is solved; wall time includes every set-up
        fs = [W["f"] - 0.1, W["f"], W["f"] + 0.1]
        sweep_kw = dict(npml=W["npml"], weights=weights, coarse_ratio=W["coarse"], factor_prec=helm.PREC_TF32,
                        tol=W["tol"], restart=W["restart"], basis_prec=helm.PREC_FP32)
        sweep = {"freqs_hz": fs}
        for name, warm, ov in (("overlap_warm", True, True), ("sequential_warm", True, False),
                               ("overlap_cold", False, True)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            xs_, st_, su_ = helm.frequency_sweep(ctx, n, n, nz, W["h"], fs, velocity(W), b, W["parts"],
                                                 W["overlap"], warm=warm, overlap_factor=ov, **sweep_kw)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t
            sweep[name] = {"wall_s": wall, "rhs_per_s_incl_setup": len(fs) * nrhs / wall, "setup_s": su_,
                           "iterations_max": [max(s_["iterations"] for s_ in f_) for f_ in st_],
                           "iterations_total": [sum(s_["iterations"] for s_ in f_) for f_ in st_]}
            del xs_
        variants["freq_sweep"] = sweep

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    bh = torch.from_numpy(b_host).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(e2e_steps):
        oras.solve(bh, xh, **solve_kw)
    e2e_value, _ = replicas.job_throughput(nrhs * e2e_steps, time.perf_counter() - t, dev)

    # plain FP64 single-RHS path on the GPU (same preconditioner structure, FP64 everywhere)
    plain = None
    if not args.no_plain:
        del oras
        torch.cuda.synchronize()
        t = time.perf_counter()
        o64 = helm.Oras(grid, W["parts"], W["overlap"], coarse_ratio=W["coarse"], factor_prec=helm.PREC_FP64)
        setup64 = time.perf_counter() - t
        b1 = b[..., :1].contiguous()
        x1 = torch.empty_like(b1)
        for _ in range(2):                      # eager first use, then graph capture
            o64.solve(b1, x1, tol=W["tol"], restart=W["restart"], flexible=True, basis_prec=helm.PREC_FP64)
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        _, st64 = o64.solve(b1, x1, tol=W["tol"], restart=W["restart"], flexible=True, basis_prec=helm.PREC_FP64)
        p1.record(stream)
        torch.cuda.synchronize()
        t64 = p0.elapsed_time(p1) / 1000.0
        err = float(torch.linalg.vector_norm(x_mixed[..., 0] - x1[..., 0]) / torch.linalg.vector_norm(x1[..., 0]))
        plain = {"value": 1.0 / t64, "unit": "RHS/s", "setup_s": setup64, "iterations": st64[0]["iterations"],
                 "true_relres": st64[0]["true_relres"], "mixed_vs_fp64_rel_l2": err,
                 "speedup_mixed_batched_vs_plain": value / (ws / t64)}
        del o64

    peaks, src = load_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # DRAM traffic per launch relative to the algorithmic bytes (dram__bytes_read.sum + dram__bytes_write.sum
    # over the kernel's own byte count), measured by ncu on a 112 x 112 x 24 slab of the same kernels
    traffic_ratio = TRAFFIC_RATIO.get(roof_fam) if args.factor_prec == "tf32" else None
    roof = None
    fam = roof_fam
    g = roof_meas
    if g:
        nl, ms, by = g
        ach = by / (ms / 1000.0) / 1e9
        roof = {"kernel": fam, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": (traffic_ratio * by / nl) if traffic_ratio else None,
                "traffic_source": ("ncu 112x112x24 slab capture of the same kernel, scaled by algorithmic bytes"
                                   if traffic_ratio else None),
                "peak_source": src, "launches": nl,
                "avg_launch_us": 1000.0 * ms / nl, "algorithmic_bytes_per_launch": by / nl}
    kernels = {}
    for fam, v in prof.items():
        if v:
            nl, ms, by = v
            kernels[fam] = {"launches": nl, "ms_total": ms, "share_of_step": ms / breakdown_ms,
                            "GBps": by / (ms / 1000.0) / 1e9}
    serving = None
    if not args.no_serve:
        del grid
        torch.cuda.synchronize()
        serving = run_serving(helm, local, stream, weights, args)
    # the other workloads of the paper's method at their full sizes (each line's own RHS/s and sweep roofline)
    more = {}
    if not args.no_workloads and args.workload == "lg112":
        torch.cuda.synchronize()
        for name, fn in (("thrust_fold_256x256x96_64rhs", run_thrust_fold),
                         ("attenuating_160x160x80_3freq_128rhs", run_attenuating)):
            log(f"workload {name}")
            try:
                more[name] = fn(helm, ctx, stream, weights, peaks, retune=args.retune)
            except Exception as exc:   # report the failure; the headline line stands
                more[name] = {"error": repr(exc)}
            torch.cuda.synchronize()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        try:
            from oracle.weights import fit_weights as oracle_fit_weights
            cpu = oracle_sample(W, float(np.mean(iters)), oracle_fit_weights())
        except Exception as exc:  # keep the GPU line even if the oracle leg fails
            cpu = {"error": repr(exc)}
    line = {
        "metric": METRIC,
        "value": value, "unit": "RHS/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic (seeded linear-gradient model, seeded point sources)",
        "config": {"workload": W["desc"], "grid": [n, n, nz], "nrhs": nrhs, "factor_prec": args.factor_prec,
                   "basis_prec": "fp32", "parallelism": f"replicas x{ws}",
                   "l2": "factors (>10 GB) and Krylov basis exceed L2; no flush"},
        "setup_s": setup_wall, "setup_device_s": setup_device, "factorisation": factor,
        "iterations": iters, "max_true_relres": relres,
        "e2e": {"value": e2e_value, "unit": "RHS/s", "h2d_bytes_per_step": int(b_host.nbytes),
                "d2h_bytes_per_step": int(b_host.nbytes)},
        "gpu_launches": int(launches),
        "launches_before_timed": int(l0),   # the library's launches up to the timed region (ncu -s for a launch list)
        "roofline": roof, "kernels": kernels, "plain_fp64_gpu": plain,
        "cpu_baseline": cpu, "clocks": clk, "serving": serving, "variants": variants, "workloads": more,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="lg112")
    ap.add_argument("--factor-prec", choices=["fp32", "tf32", "bf16"], default="tf32",
                    help="fine local factors: tf32 = complex64 factors, tensor-core sweeps; bf16 = bfloat16-stored "
                         "factors, tensor-core sweeps; fp32 = CUDA-core sweeps")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 single-RHS measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-stream (serving) measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the bf16-factor variant measurement")
    ap.add_argument("--retune", action="store_true", help="ignore the tuning cache (time every candidate again)")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the thrust-fold (256x256x96, 64 RHS) and attenuating (160x160x80, 3 x 128 RHS) lines")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the main serving phase (the full request-stream workload: 500)")
    ap.add_argument("--serve-burst", type=int, default=10, help="requests of the saturated-rate burst")
    ap.add_argument("--serve-sweep", type=int, default=6, help="requests per point of the arrival-rate sweep")
    args = ap.parse_args()
    W = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, W)
    else:
        run_gpu(args, W)


if __name__ == "__main__":
    main()
