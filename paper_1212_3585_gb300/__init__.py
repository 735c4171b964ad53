"""GB300-native ADER-WENO finite volume solver on space-time adaptive meshes.

The solver (WENO reconstruction, space-time DG predictor, Rusanov fluxes, one-step update,
local time stepping, AMR bookkeeping) lives in the CUDA library ``lib/libaderweno.so`` behind
the C ABI of ``include/aderweno.h``; this package only binds it.  ``Solver`` mirrors the C
calls one to one.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import (AwSrvInfo, AwSrvSummary, AW_BATCH_MAX, AW_BC_INFLOW, AW_BC_PERIODIC, AW_BC_REFLECTIVE, AW_BC_TRANSMISSIVE, AW_FLUX_OSHER, AW_FLUX_RUSANOV, AW_IC_CONST, AW_IC_EXPLOSION,  # noqa: F401
                   AW_IC_FOURIER, AW_IC_OT, AW_IC_RP4, AW_IC_VORTEX, AW_INTERNAL_CHI, AW_INTERNAL_FLUX,
                   AW_INTERNAL_PREDICTOR, AW_INTERNAL_WENO, AW_PDE_EULER, AW_PDE_LINADV, AW_PDE_MHD_GLM,
                   AwCell, AwConfig, AwError, AwStats)


def make_config(dim=2, pde=AW_PDE_EULER, M=2, n=(16, 16, 1), gamma=1.4, c_h=2.0, lo=(0.0, 0.0, 0.0),
                hi=(1.0, 1.0, 1.0), bc=AW_BC_PERIODIC, r=3, lmax=0, chi_ref=0.2, chi_rec=0.1, eps_ind=0.01,
                cfl=0.9, picard=0, auto_regrid=1, adv=(1.0, 1.0, 1.0), flux=AW_FLUX_RUSANOV, inflow=()) -> AwConfig:
    c = AwConfig()
    c.dim, c.pde, c.M = dim, pde, M
    c.nx, c.ny, c.nz = n[0], n[1], (n[2] if dim == 3 else 1)
    c.gamma, c.c_h = gamma, c_h
    for a in range(3):
        c.lo[a], c.hi[a], c.adv[a] = lo[a], hi[a], adv[a]
    bcs = bc if isinstance(bc, (list, tuple)) else [bc] * 6
    for i in range(6):
        c.bc[i] = bcs[i]
    c.refine_factor, c.lmax = r, lmax
    c.chi_ref, c.chi_rec, c.eps_ind, c.cfl = chi_ref, chi_rec, eps_ind, cfl
    c.picard_iters, c.flux, c.auto_regrid = picard, flux, auto_regrid
    for v, q in enumerate(inflow):
        c.inflow[v] = q
    return c


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Solver:
    """One solver on the current CUDA device, ordered on `stream` (an integer cudaStream_t)."""

    def __init__(self, cfg: AwConfig, stream: int = 0):
        self.L = _lib.load()
        self.cfg = cfg
        h = C.c_void_p()
        _lib.check(self.L.aw_create(C.byref(cfg), stream, C.byref(h)))
        self.h = h
        self.V = self.L.aw_num_vars(h)
        self.d = cfg.dim
        self.N = cfg.M + 1

    def close(self):
        if getattr(self, "h", None):
            self.L.aw_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_initial(self, ic, params, nrefine=-1):
        p = np.ascontiguousarray(params, dtype=np.float64)
        _lib.check(self.L.aw_set_initial(self.h, ic, _dp(p), len(p), nrefine))

    def set_cell_averages(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        _lib.check(self.L.aw_set_cell_averages(self.h, _dp(u), u.shape[0]))

    def step(self, t_end=1e300):
        st = AwStats()
        _lib.check(self.L.aw_step(self.h, t_end, C.byref(st)))
        return st

    def step_dt(self, dt0):
        st = AwStats()
        _lib.check(self.L.aw_step_dt(self.h, dt0, C.byref(st)))
        return st

    def advance_to(self, t_end):
        st = AwStats()
        _lib.check(self.L.aw_advance_to(self.h, t_end, C.byref(st)))
        return st

    def advance_graph(self, t_end, chunk=16):
        """aw_advance_graph: uniform meshes, device-side time step, graph replay."""
        st = AwStats()
        _lib.check(self.L.aw_advance_graph(self.h, t_end, chunk, C.byref(st)))
        return st

    def compute_dt(self):
        d = C.c_double()
        _lib.check(self.L.aw_compute_dt(self.h, C.byref(d)))
        return d.value

    def regrid(self, init_mode=0):
        _lib.check(self.L.aw_regrid(self.h, init_mode))

    def regrid_with_flags(self, flags, init_mode=0):
        f = np.ascontiguousarray(flags, dtype=np.int8)
        _lib.check(self.L.aw_regrid_with_flags(self.h, f.ctypes.data_as(C.POINTER(C.c_int8)), len(f), init_mode))

    def compute_flags(self, init_mode=0):
        n, _ = self.counts()[:2]
        f = np.zeros(max(n, 1), dtype=np.int8)
        got = C.c_int64()
        _lib.check(self.L.aw_compute_flags(self.h, init_mode, f.ctypes.data_as(C.POINTER(C.c_int8)), len(f),
                                           C.byref(got)))
        return f[: got.value]

    def counts(self):
        nc, na = C.c_int64(), C.c_int64()
        cpl, apl = (C.c_int64 * 8)(), (C.c_int64 * 8)()
        _lib.check(self.L.aw_get_counts(self.h, C.byref(nc), C.byref(na), cpl, apl))
        lm = self.cfg.lmax + 1
        return nc.value, na.value, list(cpl)[:lm], list(apl)[:lm]

    def cells(self):
        n = self.counts()[0]
        meta = (AwCell * max(n, 1))()
        u = np.zeros((max(n, 1), self.V))
        got = C.c_int64()
        _lib.check(self.L.aw_read_cells(self.h, meta, _dp(u), n, C.byref(got)))
        m = np.frombuffer(meta, dtype=np.int32).reshape(-1, 5)[:n].copy()
        return m, u[:n]

    def cells_into(self, meta, u):
        """aw_read_cells into caller-owned buffers (for example pinned host memory): meta is a
        C-contiguous int32 array of shape (cap, 5) (level, status, i, j, k), u a C-contiguous
        float64 array of shape (cap, V); returns the number of cells written"""
        assert meta.dtype == np.int32 and meta.flags.c_contiguous and meta.shape[1:] == (5,)
        assert u.dtype == np.float64 and u.flags.c_contiguous and u.shape[1:] == (self.V,)
        assert meta.shape[0] == u.shape[0]
        got = C.c_int64()
        _lib.check(self.L.aw_read_cells(self.h, meta.ctypes.data_as(C.POINTER(AwCell)), _dp(u), meta.shape[0],
                                        C.byref(got)))
        return got.value

    def internal(self, what, level=0):
        got = C.c_int64()
        rc = self.L.aw_read_internal(self.h, what, level, None, 0, C.byref(got))
        if rc not in (0, _lib.AW_EINVAL):
            _lib.check(rc)
        buf = np.zeros(max(got.value, 1))
        _lib.check(self.L.aw_read_internal(self.h, what, level, _dp(buf), len(buf), C.byref(got)))
        return buf[: got.value]

    @property
    def t(self):
        d = C.c_double()
        _lib.check(self.L.aw_get_time(self.h, C.byref(d)))
        return d.value

    def totals(self):
        out = np.zeros(self.V)
        _lib.check(self.L.aw_totals(self.h, _dp(out)))
        return out

    def reset(self):
        _lib.check(self.L.aw_reset(self.h))

    def set_profiling(self, on=True):
        _lib.check(self.L.aw_set_profiling(self.h, 1 if on else 0))

    def kernel_times(self):
        """(ms, launches) per kind: WENO, predictor, face flux, update, projection"""
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        _lib.check(self.L.aw_kernel_times(self.h, _dp(ms), n.ctypes.data_as(C.POINTER(C.c_int64))))
        return ms[:5], n[:5]

    def sync(self):
        _lib.check(self.L.aw_sync(self.h))

    def set_memory_limit(self, nbytes):
        """aw_set_memory_limit: refuse allocations above nbytes of live device memory (0: none)"""
        _lib.check(self.L.aw_set_memory_limit(self.h, int(nbytes)))

    def memory(self):
        """aw_get_memory: (live, peak, refused) device bytes of this solver"""
        v = [C.c_int64(), C.c_int64(), C.c_int64()]
        _lib.check(self.L.aw_get_memory(self.h, C.byref(v[0]), C.byref(v[1]), C.byref(v[2])))
        return tuple(x.value for x in v)

    def graph_stats(self):
        """aw_graph_stats: (reuses, in-place updates, instantiations) of this solver's step graphs"""
        v = [C.c_int64(), C.c_int64(), C.c_int64()]
        _lib.check(self.L.aw_graph_stats(self.h, C.byref(v[0]), C.byref(v[1]), C.byref(v[2])))
        return tuple(x.value for x in v)

    def kernel_launches(self):
        return self.L.aw_kernel_launches(self.h)


def get_launch_params() -> dict:
    """aw_get_launch_params: the process-wide launch-shape rules."""
    p = _lib.AwLaunchParams()
    _lib.check(_lib.load().aw_get_launch_params(C.byref(p)))
    return {"pass_min_cells": p.pass_min_cells, "tile8_min_cells": p.tile8_min_cells,
            "small_ctas_per_sm": p.small_ctas_per_sm, "fuse_flux_update": p.fuse_flux_update,
            "autotune": p.autotune, "persistent": p.persistent, "graph_steps": p.graph_steps}


def set_launch_params(pass_min_cells=None, tile8_min_cells=None, small_ctas_per_sm=None, fuse_flux_update=None,
                      autotune=None, persistent=None, graph_steps=None):
    """aw_set_launch_params: change some of the launch-shape rules (speed only, never results)."""
    cur = get_launch_params()
    p = _lib.AwLaunchParams()
    p.pass_min_cells = cur["pass_min_cells"] if pass_min_cells is None else int(pass_min_cells)
    p.tile8_min_cells = cur["tile8_min_cells"] if tile8_min_cells is None else int(tile8_min_cells)
    p.small_ctas_per_sm = cur["small_ctas_per_sm"] if small_ctas_per_sm is None else int(small_ctas_per_sm)
    p.fuse_flux_update = cur["fuse_flux_update"] if fuse_flux_update is None else int(fuse_flux_update)
    p.autotune = cur["autotune"] if autotune is None else int(autotune)
    p.persistent = cur["persistent"] if persistent is None else int(persistent)
    p.graph_steps = cur["graph_steps"] if graph_steps is None else int(graph_steps)
    _lib.check(_lib.load().aw_set_launch_params(C.byref(p)))


def get_tuning() -> list:
    """aw_get_tuning: one dict per (configuration, kernel, level size class) the autotuner has seen"""
    L = _lib.load()
    n = C.c_int32()
    _lib.check(L.aw_get_tuning(None, 0, C.byref(n)))
    buf = (_lib.AwTuneEntry * max(n.value, 1))()
    _lib.check(L.aw_get_tuning(buf, n.value, C.byref(n)))
    return [{"dim": e.dim, "M": e.M, "pde": e.pde, "flux": e.flux, "kernel": e.kernel, "size_class": e.size_class,
             "choice": e.choice, "trials": list(e.trials), "inherited": e.inherited,
             "ns_per_cell": list(e.ns_per_cell)}
            for e in buf[: n.value]]


def reset_tuning():
    """aw_reset_tuning: forget every decision of the autotuner"""
    _lib.check(_lib.load().aw_reset_tuning())


def tables_host(M: int, r: int) -> dict:
    """aw_tables_host: the reference-element tables the kernels use, unpacked into arrays."""
    L = _lib.load()
    n = C.c_int64(0)
    L.aw_tables_host(M, r, None, 0, C.byref(n))
    buf = np.zeros(n.value)
    _lib.check(L.aw_tables_host(M, r, buf.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)))
    N, ns = int(buf[0]), int(buf[1])
    sizes = [("x", (N,)), ("w", (N,)), ("SL", (4,)), ("lam", (4,)), ("Ainv", (4, N, N)), ("Sig", (N, N)),
             ("Dm", (N, N)), ("G", (N, N)), ("psi0", (N,)), ("psi1", (N,)), ("Wc", (r, N)), ("Pf", (r, N, N)),
             ("Pt", (r, N)), ("gsum", (N,)), ("Bq", (4, N - 1, N - 1))]
    out, k = {"N": N, "Ns": ns, "r": int(buf[2])}, 3
    for name, shape in sizes:
        m = int(np.prod(shape))
        out[name] = buf[k:k + m].reshape(shape)
        k += m
    out["SL"] = out["SL"][:ns].astype(int)
    out["lam"], out["Ainv"], out["Bq"] = out["lam"][:ns], out["Ainv"][:ns], out["Bq"][:ns]
    return out


def advance_batch(solvers, t_end, stream: int = 0):
    """aw_advance_batch: advance independent solvers of one kernel configuration to t_end with
    their hot kernels batched per level and sub-step.  Returns (stats, rc) per solver; raises
    AwError with the first failure."""
    n = len(solvers)
    arr = (C.c_void_p * n)(*[s.h.value for s in solvers])
    st = (AwStats * n)()
    rc = (C.c_int32 * n)()
    code = _lib.load().aw_advance_batch(arr, n, t_end, stream, st, rc)
    out = list(st), list(rc)
    _lib.check(code)
    return out


def step_batch(solvers, t_ends, stream: int = 0):
    """aw_step_batch: one lockstep level-0 step of every solver not yet at its own end time, the
    hot kernels batched.  Returns (stats, rc) per solver; raises AwError with the first failure."""
    n = len(solvers)
    if len(t_ends) != n:
        raise ValueError("one end time per solver")
    arr = (C.c_void_p * n)(*[s.h.value for s in solvers])
    te = (C.c_double * n)(*[float(t) for t in t_ends])
    st = (AwStats * n)()
    rc = (C.c_int32 * n)()
    code = _lib.load().aw_step_batch(arr, n, te, stream, st, rc)
    out = list(st), list(rc)
    _lib.check(code)
    return out


class Server:
    """Request loop of independent solves (aw_srv_*): continuous admission under a device-memory
    budget, concurrent requests on their own streams, reservations that grow in place; with
    max_batch > 1, continuous batching: compatible requests share batched launches, leave their
    group when they finish and join a running group between steps (aw_srv_set_batching)."""

    def __init__(self, hbm_budget_bytes: int, max_concurrent: int = 4, max_batch: int = 1):
        self.L = _lib.load()
        h = C.c_void_p()
        rc = self.L.aw_srv_create(int(hbm_budget_bytes), max_concurrent, C.byref(h))
        if rc:
            raise AwError(rc, self.L.aw_srv_last_error().decode())
        self.h = h
        if max_batch != 1:
            self._check(self.L.aw_srv_set_batching(self.h, max_batch))

    def _check(self, rc):
        if rc:
            raise AwError(rc, self.L.aw_srv_last_error().decode())

    def submit(self, cfg: AwConfig, ic, params, t_end) -> int:
        p = np.ascontiguousarray(params, dtype=np.float64)
        rid = C.c_int64()
        self._check(self.L.aw_srv_submit(self.h, C.byref(cfg), ic, _dp(p), len(p), t_end, C.byref(rid)))
        return rid.value

    def poll(self, rid) -> int:
        st = C.c_int32()
        self._check(self.L.aw_srv_poll(self.h, rid, C.byref(st)))
        return st.value

    def wait_all(self):
        self._check(self.L.aw_srv_wait_all(self.h))

    def result(self, rid, V):
        n = C.c_int64()
        info = AwSrvInfo()
        rc = self.L.aw_srv_result(self.h, rid, None, None, 0, C.byref(n), C.byref(info))
        if rc not in (0, _lib.AW_EINVAL):
            self._check(rc)
        meta = (AwCell * max(n.value, 1))()
        u = np.zeros((max(n.value, 1), V))
        self._check(self.L.aw_srv_result(self.h, rid, meta, _dp(u), n.value, C.byref(n), C.byref(info)))
        m = np.frombuffer(meta, dtype=np.int32).reshape(-1, 5)[: n.value].copy()
        return m, u[: n.value], info

    def stats(self) -> AwSrvSummary:
        s = AwSrvSummary()
        self._check(self.L.aw_srv_stats(self.h, C.byref(s)))
        return s

    def close(self):
        if getattr(self, "h", None):
            self.L.aw_srv_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
