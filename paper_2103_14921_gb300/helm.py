"""ctypes binding of ``libhelm.so`` (argument marshalling only).

Names follow ``include/helm.h``.  Arrays are torch tensors; the binding
passes their data pointers and the current CUDA stream.  All computation
happens in the CUDA library; if the library is missing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libhelm.so")
_lib = None
_finalizing = False


def _mark_finalizing():
    global _finalizing
    _finalizing = True


import atexit as _atexit
_atexit.register(_mark_finalizing)   # handles still alive at exit are left to process teardown

OK, EINVAL, ENOMEM, ENOTCONV, ESINGULAR, ENONFINITE, ETIMEOUT, EBUSY, ECUDA, ENOTFOUND = range(10)
TOP_DIRICHLET, TOP_PML = 0, 1
TUNE_TC_STAGES = 1
TUNE_COARSE_COOP = 2
TUNE_GRAPHS = 3
TUNE_TC_FLOW = 4
TUNE_STENCIL_MARCH = 5
TUNE_FLOW_WAIT_US = 6
TUNE_TC_FACTOR = 7
TUNE_BLOCK_GJ = 8
TUNE_STENCIL_PLANES = 9
PREC_FP64, PREC_FP32, PREC_TF32, PREC_TF32X3, PREC_BF16 = 0, 1, 2, 3, 4
PREC_NAMES = {"fp64": PREC_FP64, "fp32": PREC_FP32, "tf32": PREC_TF32, "tf32x3": PREC_TF32X3, "bf16": PREC_BF16}


class HelmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"helm status {status}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double), ("freq_hz", C.c_double),
                ("npml", C.c_int), ("pml_R", C.c_double), ("top_bc", C.c_int), ("weights", C.c_double * 7),
                ("weight_bins", C.c_int)]


class OrasDesc(C.Structure):
    _fields_ = [("px", C.c_int), ("py", C.c_int), ("pz", C.c_int), ("overlap", C.c_int), ("coarse_ratio", C.c_int),
                ("interface_bc", C.c_int), ("factor_prec", C.c_int), ("coarse_iters", C.c_int),
                ("coarse_overlap", C.c_int)]


class GmresDesc(C.Structure):
    _fields_ = [("tol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int), ("flexible", C.c_int),
                ("basis_prec", C.c_int), ("use_x0", C.c_int)]


class RhsStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("true_relres", C.c_double),
                ("est_relres", C.c_double)]


class SweepDesc(C.Structure):
    _fields_ = [("grid", GridDesc), ("oras", OrasDesc), ("gmres", GmresDesc), ("nfreq", C.c_int),
                ("freqs", C.POINTER(C.c_double)), ("warm", C.c_int), ("overlap", C.c_int)]


class Request(C.Structure):
    _fields_ = [("model_id", C.c_uint64), ("grid", GridDesc), ("c", C.c_void_p), ("oras", OrasDesc),
                ("gmres", GmresDesc), ("nrhs", C.c_int), ("b", C.c_void_p), ("x", C.c_void_p)]


class RequestStats(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("iterations_max", C.c_int), ("true_relres_max", C.c_double),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double), ("factors_reused", C.c_int)]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2103_14921_gb300.build.build()")
    L = C.CDLL(_LIB_PATH)
    vp, i32, st = C.c_void_p, C.c_int, C.c_int
    sig = {
        "helm_create": (st, [C.POINTER(vp), i32, vp, C.c_size_t]),
        "helm_destroy": (None, [vp]),
        "helm_last_error": (C.c_char_p, [vp]),
        "helm_bytes_in_use": (C.c_size_t, [vp]),
        "helm_launch_count": (C.c_uint64, [vp]),
        "helm_profile_enable": (st, [vp, i32]),
        "helm_set_tuning": (st, [vp, i32, i32]),
        "helm_profile_select": (st, [vp, C.c_char_p]),
        "helm_profile_query": (st, [vp, C.c_char_p, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
        "helm_fit_weights": (st, [C.c_double, C.c_double, C.POINTER(C.c_double)]),
        "helm_setup_grid": (st, [vp, C.POINTER(GridDesc), vp, C.POINTER(vp)]),
        "helm_destroy_grid": (None, [vp]),
        "helm_grid_row_weights": (st, [vp, C.POINTER(C.c_int), vp, vp]),
        "helm_apply": (st, [vp, i32, vp, vp, i32]),
        "oras_factor": (st, [vp, C.POINTER(OrasDesc), C.POINTER(vp)]),
        "oras_destroy": (None, [vp]),
        "oras_apply": (st, [vp, vp, vp, i32]),
        "oras_apply_noalloc": (st, [vp, vp, vp, i32]),
        "oras_box_info": (st, [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
        "oras_plane_inverse": (st, [vp, i32, i32, vp]),
        "oras_setup_seconds": (C.c_double, [vp]),
        "oras_estimate_bytes_c": (st, [C.POINTER(GridDesc), C.POINTER(OrasDesc), i32, C.POINTER(C.c_size_t)]),
        "gmres_solve": (st, [vp, vp, vp, i32, C.POINTER(GmresDesc), C.POINTER(RhsStats)]),
        "helm_frequency_sweep": (st, [vp, C.POINTER(SweepDesc), vp, vp, vp, i32, C.POINTER(RhsStats),
                                      C.POINTER(C.c_double)]),
        "helm_serve_start": (st, [vp, i32]),
        "helm_submit": (st, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "helm_poll": (st, [vp, C.c_uint64, C.POINTER(i32), C.POINTER(RequestStats)]),
        "helm_serve_stop": (st, [vp]),
    }
    for name, (res, args) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    _lib = L
    return L


def fit_weights(G_min=4.0, G_max=30.0):
    """Stencil weights fitted by the library (host computation)."""
    out = (C.c_double * 7)()
    st = lib().helm_fit_weights(G_min, G_max, out)
    if st:
        raise HelmError(st, "helm_fit_weights")
    return tuple(out)


def estimate_bytes(grid_desc, oras_desc, nrhs):
    """Library estimate of the device bytes of an ORAS handle plus apply scratch (host computation)."""
    out = C.c_size_t()
    st = lib().oras_estimate_bytes_c(C.byref(grid_desc), C.byref(oras_desc), nrhs, C.byref(out))
    if st:
        raise HelmError(st, "oras_estimate_bytes_c")
    return out.value


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Context:
    def __init__(self, device=0, stream=None, budget_bytes=0):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self._h = C.c_void_p()
        st = lib().helm_create(C.byref(self._h), device, C.c_void_p(stream), budget_bytes)
        if st:
            raise HelmError(st, lib().helm_last_error(None).decode())
        self.device = device

    def check(self, st, what=""):
        if st:
            raise HelmError(st, f"{what}: {lib().helm_last_error(self._h).decode()}")

    @property
    def bytes_in_use(self):
        return lib().helm_bytes_in_use(self._h)

    @property
    def launches(self):
        return lib().helm_launch_count(self._h)

    def set_tuning(self, key, value):
        """``helm_set_tuning`` (e.g. ``TUNE_TC_STAGES``)."""
        self.check(lib().helm_set_tuning(self._h, key, value), "helm_set_tuning")

    def profile(self, on=True, only=None):
        """Enable (and clear) or disable per-kernel-family event timing; ``only`` = list of families."""
        self.check(lib().helm_profile_select(self._h, ",".join(only).encode() if only else None),
                   "helm_profile_select")
        self.check(lib().helm_profile_enable(self._h, 1 if on else 0), "helm_profile_enable")

    def profile_query(self, family):
        """``(launches, total_ms, total_algorithmic_bytes)`` of a kernel family, or None."""
        n, ms, b = C.c_uint64(), C.c_double(), C.c_double()
        st = lib().helm_profile_query(self._h, family.encode(), C.byref(n), C.byref(ms), C.byref(b))
        if st == ENOTFOUND:
            return None
        self.check(st, "helm_profile_query")
        return n.value, ms.value, b.value

    def close(self):
        if self._h:
            lib().helm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        if _finalizing:
            return
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """``helm_setup_grid``: one problem (grid, medium, frequency)."""

    def __init__(self, ctx: Context, nx, ny, nz, h, freq_hz, c, npml=8, top_bc=TOP_DIRICHLET, pml_R=1e-3,
                 weights=None, weight_bins=0):
        """``weight_bins > 0``: adaptive weights matched to the local wave speed (``row_weights()``)."""
        import torch
        if weights is None:
            weights = fit_weights()
        d = GridDesc(nx, ny, nz, h, freq_hz, npml, pml_R, top_bc, (C.c_double * 7)(*weights), weight_bins)
        self.ctx = ctx
        self.desc = d
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz
        if isinstance(c, np.ndarray):
            c = torch.from_numpy(np.ascontiguousarray(c, dtype=np.complex128))
        c = c.contiguous()
        assert c.dtype == torch.complex128 and c.numel() == self.n
        self._h = C.c_void_p()
        ctx.check(lib().helm_setup_grid(ctx._h, C.byref(d), _ptr(c), C.byref(self._h)), "helm_setup_grid")

    def apply(self, u, y=None, prec=PREC_FP64):
        """``y = A u``; u is a CUDA tensor ``[nz, ny, nx, nrhs]`` complex128 (FP64) or complex64 (FP32)."""
        import torch
        want = torch.complex128 if prec == PREC_FP64 else torch.complex64
        assert u.is_cuda and u.dtype == want and u.is_contiguous()
        nrhs = u.numel() // self.n
        if y is None:
            y = torch.empty_like(u)
        self.ctx.check(lib().helm_apply(self._h, prec, _ptr(u), _ptr(y), nrhs), "helm_apply")
        return y

    def row_weights(self):
        """``(edges[nbins + 1], table[nbins, 7])`` of the adaptive weights (``None`` for constant weights)."""
        nb = C.c_int()
        self.ctx.check(lib().helm_grid_row_weights(self._h, C.byref(nb), None, None), "helm_grid_row_weights")
        if nb.value == 0:
            return None
        edges = (C.c_double * (nb.value + 1))()
        table = (C.c_double * (nb.value * 7))()
        self.ctx.check(lib().helm_grid_row_weights(self._h, C.byref(nb), edges, table), "helm_grid_row_weights")
        return np.array(edges[:]), np.array(table[:]).reshape(nb.value, 7)

    def close(self):
        if self._h:
            lib().helm_destroy_grid(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        if _finalizing:
            return
        try:
            self.close()
        except Exception:
            pass


class Oras:
    """``oras_factor``: the two-level ORAS preconditioner with resident plane factors."""

    def __init__(self, grid: Grid, parts, overlap, coarse_ratio=0, interface_bc=0, factor_prec=PREC_FP64,
                 coarse_iters=0, coarse_overlap=1):
        """``coarse_iters = k >= 1`` solves the coarse problem as the paper does (k GMRES iterations with
        one-level ORAS on the coarse grid, ``coarse_overlap`` coarse layers); 0 solves it exactly."""
        d = OrasDesc(parts[0], parts[1], parts[2], overlap, coarse_ratio, interface_bc, factor_prec, coarse_iters,
                     coarse_overlap)
        self.grid = grid
        self.ctx = grid.ctx
        self.desc = d
        self._h = C.c_void_p()
        self.ctx.check(lib().oras_factor(grid._h, C.byref(d), C.byref(self._h)), "oras_factor")

    @property
    def setup_seconds(self):
        return lib().oras_setup_seconds(self._h)

    def box_info(self, box):
        nb = C.c_int()
        lo = (C.c_int * 3)()
        dims = (C.c_int * 3)()
        self.ctx.check(lib().oras_box_info(self._h, box, C.byref(nb), lo, dims), "oras_box_info")
        return nb.value, tuple(lo), tuple(dims)

    def plane_inverse(self, box, plane):
        import torch
        _, _, dims = self.box_info(box)
        m = dims[0] * dims[1]
        out = torch.empty((m, m), dtype=torch.complex128, device="cuda")
        self.ctx.check(lib().oras_plane_inverse(self._h, box, plane, _ptr(out)), "oras_plane_inverse")
        return out

    def apply(self, v, out=None):
        import torch
        assert v.is_cuda and v.dtype == torch.complex128 and v.is_contiguous()
        nrhs = v.numel() // self.grid.n
        if out is None:
            out = torch.empty_like(v)
        self.ctx.check(lib().oras_apply(self._h, _ptr(v), _ptr(out), nrhs), "oras_apply")
        return out

    def solve(self, b, x=None, tol=1e-6, restart=30, maxit=1000, flexible=True, basis_prec=PREC_FP64,
              allow_notconv=False, warm=False):
        """``gmres_solve``; b is complex128 ``[nz, ny, nx, nrhs]`` (CUDA or pinned/pageable CPU tensor).
        ``warm=True``: ``x`` (required) holds the initial guess on entry."""
        import torch
        assert b.dtype == torch.complex128 and b.is_contiguous()
        nrhs = b.numel() // self.grid.n
        if x is None:
            assert not warm, "a warm start needs x"
            x = torch.empty_like(b)
        d = GmresDesc(tol, restart, maxit, 1 if flexible else 0, basis_prec, 1 if warm else 0)
        stats = (RhsStats * max(nrhs, 1))()
        st = lib().gmres_solve(self._h, _ptr(b), _ptr(x), nrhs, C.byref(d), stats)
        if st and not (allow_notconv and st == ENOTCONV):
            self.ctx.check(st, "gmres_solve")
        return x, [dict(iterations=s.iterations, converged=bool(s.converged), true_relres=s.true_relres,
                        est_relres=s.est_relres) for s in stats[:nrhs]]

    def close(self):
        if self._h:
            lib().oras_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        if _finalizing:
            return
        try:
            self.close()
        except Exception:
            pass


class Server:
    """``helm_serve_start`` .. ``helm_serve_stop``: request loop with continuous batching on a context.

    While serving, the context must not be used for other calls.  Buffers
    passed to :meth:`submit` are kept referenced until the request is done.
    """

    def __init__(self, ctx: Context, slots_per_batch=16):
        self.ctx = ctx
        self._keep = {}
        ctx.check(lib().helm_serve_start(ctx._h, slots_per_batch), "helm_serve_start")
        self.running = True

    def submit(self, model_id, grid_desc, c, oras_desc, b, x, tol=1e-6, restart=30, maxit=1000, flexible=True,
               basis_prec=PREC_FP32):
        """Queue a solve; c, b, x are contiguous complex128 tensors (CUDA or CPU); returns a ticket."""
        nrhs = b.shape[-1]
        req = Request(model_id, grid_desc, C.c_void_p(c.data_ptr()), oras_desc,
                      GmresDesc(tol, restart, maxit, 1 if flexible else 0, basis_prec), nrhs,
                      C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()))
        t = C.c_uint64()
        self.ctx.check(lib().helm_submit(self.ctx._h, C.byref(req), C.byref(t)), "helm_submit")
        self._keep[t.value] = (c, b, x)
        return t.value

    def poll(self, ticket):
        """``(done, stats dict)``."""
        done = C.c_int()
        s = RequestStats()
        self.ctx.check(lib().helm_poll(self.ctx._h, ticket, C.byref(done), C.byref(s)), "helm_poll")
        out = dict(done=bool(done.value), status=s.status, iterations_max=s.iterations_max,
                   true_relres_max=s.true_relres_max, queue_ms=s.queue_ms, latency_ms=s.latency_ms,
                   factors_reused=bool(s.factors_reused))
        if done.value:
            self._keep.pop(ticket, None)
        return out["done"], out

    def wait(self, ticket, timeout_s=600.0, interval_s=0.002):
        import time
        t0 = time.time()
        while True:
            d, s = self.poll(ticket)
            if d:
                return s
            if time.time() - t0 > timeout_s:
                raise TimeoutError(f"ticket {ticket} not done after {timeout_s} s")
            time.sleep(interval_s)

    def stop(self):
        if self.running:
            self.ctx.check(lib().helm_serve_stop(self.ctx._h), "helm_serve_stop")
            self.running = False
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.stop()

    def __del__(self):
        if _finalizing:
            return
        try:
            self.stop()
        except Exception:
            pass


def frequency_sweep(ctx: Context, nx, ny, nz, h, freqs, c, b, parts, overlap, x=None, npml=8,
                    top_bc=TOP_DIRICHLET, pml_R=1e-3, weights=None, weight_bins=0, coarse_ratio=0, interface_bc=0,
                    factor_prec=PREC_FP64, coarse_iters=0, coarse_overlap=1, tol=1e-6, restart=30, maxit=1000,
                    flexible=True, basis_prec=PREC_FP64, warm=True, overlap_factor=True, allow_notconv=False):
    """``helm_frequency_sweep``: b complex128 ``[nz, ny, nx, nrhs]`` (the sources of every frequency);
    returns x ``[nfreq, nz, ny, nx, nrhs]``, per-frequency stats and set-up seconds."""
    import torch
    if weights is None:
        weights = fit_weights()
    nf = len(freqs)
    gd = GridDesc(nx, ny, nz, h, 0.0, npml, pml_R, top_bc, (C.c_double * 7)(*weights), weight_bins)
    od = OrasDesc(parts[0], parts[1], parts[2], overlap, coarse_ratio, interface_bc, factor_prec, coarse_iters,
                  coarse_overlap)
    gm = GmresDesc(tol, restart, maxit, 1 if flexible else 0, basis_prec, 0)
    fa = (C.c_double * nf)(*freqs)
    d = SweepDesc(gd, od, gm, nf, fa, 1 if warm else 0, 1 if overlap_factor else 0)
    if isinstance(c, np.ndarray):
        c = torch.from_numpy(np.ascontiguousarray(c, dtype=np.complex128))
    c = c.contiguous()
    assert b.dtype == torch.complex128 and b.is_contiguous()
    n = nx * ny * nz
    nrhs = b.numel() // n
    if x is None:
        x = torch.empty((nf,) + tuple(b.shape), dtype=b.dtype, device=b.device)
    stats = (RhsStats * (nf * nrhs))()
    setup = (C.c_double * nf)()
    st = lib().helm_frequency_sweep(ctx._h, C.byref(d), _ptr(c), _ptr(b), _ptr(x), nrhs, stats, setup)
    if st and not (allow_notconv and st == ENOTCONV):
        ctx.check(st, "helm_frequency_sweep")
    out = [[dict(iterations=stats[f * nrhs + r].iterations, converged=bool(stats[f * nrhs + r].converged),
                 true_relres=stats[f * nrhs + r].true_relres) for r in range(nrhs)] for f in range(nf)]
    return x, out, list(setup)
