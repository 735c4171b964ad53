"""FP64 CPU oracle of the ADER-WENO space-time AMR scheme -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import this package.  The product path (``paper_1212_3585_gb300``)
never imports it and shares no code with it.

This module is a thin ctypes binding of ``aw_oracle.c``; all arithmetic lives there.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PDE_EULER, PDE_MHD, PDE_LINADV = 0, 1, 2
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_INFLOW = 0, 1, 2, 3
IC_CONST, IC_VORTEX, IC_EXPLOSION, IC_OT, IC_RP4, IC_FOURIER = 0, 1, 2, 3, 4, 5
ST_NONE = -2


class OrcCfg(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("pde", C.c_int), ("M", C.c_int),
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("gamma", C.c_double), ("c_h", C.c_double),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("bc", C.c_int * 6),
        ("r", C.c_int), ("lmax", C.c_int),
        ("chi_ref", C.c_double), ("chi_rec", C.c_double), ("eps_ind", C.c_double), ("cfl", C.c_double),
        ("picard", C.c_int), ("auto_regrid", C.c_int),
        ("adv", C.c_double * 3),
        ("flux", C.c_int),
        ("inflow", C.c_double * 9),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        i8 = C.POINTER(C.c_int8)
        i32 = C.POINTER(C.c_int32)
        i64 = C.POINTER(C.c_int64)
        lp = C.POINTER(C.c_long)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcCfg)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_last_error.restype = C.c_char_p
        L.orc_set_threads.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_initial.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, C.c_int]
        L.orc_num_cells.restype = C.c_long
        L.orc_num_cells.argtypes = [C.c_void_p, lp, lp]
        L.orc_read_cells.restype = C.c_long
        L.orc_read_cells.argtypes = [C.c_void_p, i32, dp, C.c_long]
        L.orc_set_cell_averages.argtypes = [C.c_void_p, dp, C.c_long]
        L.orc_compute_dt.restype = C.c_double
        L.orc_compute_dt.argtypes = [C.c_void_p]
        L.orc_advance_dt.argtypes = [C.c_void_p, C.c_double]
        L.orc_step.argtypes = [C.c_void_p, C.c_double, dp]
        L.orc_time.restype = C.c_double
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_set_time.argtypes = [C.c_void_p, C.c_double]
        L.orc_updates.restype = C.c_int64
        L.orc_updates.argtypes = [C.c_void_p, i64]
        L.orc_compute_flags.restype = C.c_long
        L.orc_compute_flags.argtypes = [C.c_void_p, C.c_int, i8, C.c_long]
        L.orc_regrid_with_flags.argtypes = [C.c_void_p, i8, C.c_long, C.c_int]
        L.orc_regrid.argtypes = [C.c_void_p, C.c_int]
        L.orc_read_internal.restype = C.c_long
        L.orc_read_internal.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_long]
        L.orc_weno_level.argtypes = [C.c_void_p, C.c_int]
        L.orc_tables.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, ip, ip, dp]
        L.orc_st_matrices.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.orc_weno1d.argtypes = [C.c_int, dp, dp]
        L.orc_predictor.argtypes = [C.c_void_p, dp, C.c_double, dp, dp]
        L.orc_flux.argtypes = [C.c_void_p, dp, C.c_int, dp]
        L.orc_max_speed.restype = C.c_double
        L.orc_max_speed.argtypes = [C.c_void_p, dp, C.c_int]
        L.orc_rusanov.argtypes = [C.c_void_p, dp, dp, C.c_int, dp]
        L.orc_osher.argtypes = [C.c_void_p, dp, dp, C.c_int, dp]
        L.orc_abs_jacobian_apply.argtypes = [C.c_void_p, dp, C.c_int, dp, dp]
        L.orc_eval_st.argtypes = [C.c_void_p, dp, dp, C.c_double, dp]
        L.orc_eval_sp.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_project_st.argtypes = [C.c_void_p, dp, ip, C.c_double, dp]
        L.orc_project_sp.argtypes = [C.c_void_p, dp, ip, dp]
        L.orc_indicator_at.restype = C.c_double
        L.orc_indicator_at.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_ic_average.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, dp]
        L.orc_nvars.argtypes = [C.c_void_p]
        L.orc_radial_explosion.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_int, C.c_double, C.c_double, C.c_double, dp, dp, dp]
        L.orc_totals.argtypes = [C.c_void_p, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_cfg(dim=2, pde=PDE_EULER, M=2, n=(16, 16, 1), gamma=1.4, c_h=2.0, lo=(0.0, 0.0, 0.0),
             hi=(1.0, 1.0, 1.0), bc=BC_PERIODIC, r=3, lmax=0, chi_ref=0.2, chi_rec=0.1, eps_ind=0.01,
             cfl=0.9, picard=0, auto_regrid=1, adv=(1.0, 1.0, 1.0), flux=0, inflow=()):
    c = OrcCfg()
    c.dim, c.pde, c.M = dim, pde, M
    c.nx, c.ny, c.nz = n[0], n[1], (n[2] if dim == 3 else 1)
    c.gamma, c.c_h = gamma, c_h
    for a in range(3):
        c.lo[a], c.hi[a], c.adv[a] = lo[a], hi[a], adv[a]
    bcs = bc if isinstance(bc, (list, tuple)) else [bc] * 6
    for i in range(6):
        c.bc[i] = bcs[i]
    c.r, c.lmax = r, lmax
    c.chi_ref, c.chi_rec, c.eps_ind, c.cfl = chi_ref, chi_rec, eps_ind, cfl
    c.picard, c.auto_regrid = picard, auto_regrid
    c.flux = flux
    for v, q in enumerate(inflow):
        c.inflow[v] = q
    return c


class Oracle:
    """One oracle solver instance (CPU, FP64)."""

    def __init__(self, cfg: OrcCfg, threads: int = 1):
        self.cfg = cfg
        self.L = lib()
        self.h = self.L.orc_create(C.byref(cfg))
        if not self.h:
            raise ValueError(self.L.orc_last_error().decode())
        self.V = self.L.orc_nvars(self.h)
        self.d = cfg.dim
        self.N = cfg.M + 1
        self.nsp = self.N ** self.d
        self.nst = self.nsp * self.N
        self.L.orc_set_threads(self.h, threads)

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_destroy(self.h)
            self.h = None

    def set_initial(self, ic, params, nrefine=None):
        p = np.ascontiguousarray(params, dtype=np.float64)
        if nrefine is None:
            nrefine = self.cfg.lmax
        self.L.orc_set_initial(self.h, ic, _dp(p), len(p), nrefine)

    def counts(self):
        pl = (C.c_long * 8)()
        al = (C.c_long * 8)()
        n = self.L.orc_num_cells(self.h, pl, al)
        return n, list(pl)[: self.cfg.lmax + 1], list(al)[: self.cfg.lmax + 1]

    def cells(self):
        n = self.L.orc_num_cells(self.h, None, None)
        meta = np.zeros((n, 5), dtype=np.int32)
        u = np.zeros((n, self.V))
        self.L.orc_read_cells(self.h, meta.ctypes.data_as(C.POINTER(C.c_int32)), _dp(u), n)
        return meta, u

    def set_cell_averages(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        rc = self.L.orc_set_cell_averages(self.h, _dp(u), u.shape[0])
        if rc:
            raise ValueError(self.L.orc_last_error().decode())

    def compute_dt(self):
        return self.L.orc_compute_dt(self.h)

    def advance_dt(self, dt0):
        return self.L.orc_advance_dt(self.h, dt0)

    def step(self, t_end=1e300):
        dt = C.c_double(0.0)
        rc = self.L.orc_step(self.h, t_end, C.byref(dt))
        return rc, dt.value

    @property
    def t(self):
        return self.L.orc_time(self.h)

    def updates(self):
        pl = (C.c_int64 * 8)()
        n = self.L.orc_updates(self.h, pl)
        return n, list(pl)[: self.cfg.lmax + 1]

    def compute_flags(self, init_mode=0):
        n = self.L.orc_num_cells(self.h, None, None)
        f = np.zeros(max(n, 1), dtype=np.int8)
        self.L.orc_compute_flags(self.h, init_mode, f.ctypes.data_as(C.POINTER(C.c_int8)), n)
        return f[:n]

    def regrid_with_flags(self, flags, init_mode=0):
        f = np.ascontiguousarray(flags, dtype=np.int8)
        rc = self.L.orc_regrid_with_flags(self.h, f.ctypes.data_as(C.POINTER(C.c_int8)), len(f), init_mode)
        if rc:
            raise ValueError(self.L.orc_last_error().decode())

    def regrid(self, init_mode=0):
        self.L.orc_regrid(self.h, init_mode)

    def internal(self, what, lv=0):
        n = self.L.orc_read_internal(self.h, what, lv, None, 0)
        buf = np.zeros(max(n, 1))
        self.L.orc_read_internal(self.h, what, lv, _dp(buf), n)
        return buf[:n]

    def weno_level(self, lv=0):
        self.L.orc_weno_level(self.h, lv)

    def predictor(self, wh, dt, dx):
        wh = np.ascontiguousarray(wh, dtype=np.float64)
        dxa = np.ascontiguousarray(list(dx) + [1.0] * (3 - len(dx)), dtype=np.float64)
        qh = np.zeros(self.V * self.nst)
        self.L.orc_predictor(self.h, _dp(wh), dt, _dp(dxa), _dp(qh))
        return qh

    def flux(self, q, n):
        q = np.ascontiguousarray(q, dtype=np.float64)
        f = np.zeros(self.V)
        self.L.orc_flux(self.h, _dp(q), n, _dp(f))
        return f

    def max_speed(self, q, n):
        q = np.ascontiguousarray(q, dtype=np.float64)
        return self.L.orc_max_speed(self.h, _dp(q), n)

    def rusanov(self, qm, qp, n):
        qm = np.ascontiguousarray(qm, dtype=np.float64)
        qp = np.ascontiguousarray(qp, dtype=np.float64)
        f = np.zeros(self.V)
        self.L.orc_rusanov(self.h, _dp(qm), _dp(qp), n, _dp(f))
        return f

    def osher(self, qm, qp, n):
        qm = np.ascontiguousarray(qm, dtype=np.float64)
        qp = np.ascontiguousarray(qp, dtype=np.float64)
        f = np.zeros(self.V)
        self.L.orc_osher(self.h, _dp(qm), _dp(qp), n, _dp(f))
        return f

    def abs_jacobian(self, q, n):
        """the matrix |A(q)| (columns = |A| applied to unit vectors)"""
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((self.V, self.V))
        for j in range(self.V):
            e = np.zeros(self.V)
            e[j] = 1.0
            col = np.zeros(self.V)
            self.L.orc_abs_jacobian_apply(self.h, _dp(q), n, _dp(e), _dp(col))
            out[:, j] = col
        return out

    def eval_st(self, qh, xi, tau):
        qh = np.ascontiguousarray(qh, dtype=np.float64)
        x = np.ascontiguousarray(list(xi) + [0.0] * (3 - len(xi)), dtype=np.float64)
        out = np.zeros(self.V)
        self.L.orc_eval_st(self.h, _dp(qh), _dp(x), tau, _dp(out))
        return out

    def eval_sp(self, wh, xi):
        wh = np.ascontiguousarray(wh, dtype=np.float64)
        x = np.ascontiguousarray(list(xi) + [0.0] * (3 - len(xi)), dtype=np.float64)
        out = np.zeros(self.V)
        self.L.orc_eval_sp(self.h, _dp(wh), _dp(x), _dp(out))
        return out

    def project_st(self, qh, ch, tau):
        qh = np.ascontiguousarray(qh, dtype=np.float64)
        c = (C.c_int * 3)(*(list(ch) + [0] * (3 - len(ch))))
        out = np.zeros(self.V)
        self.L.orc_project_st(self.h, _dp(qh), c, tau, _dp(out))
        return out

    def project_sp(self, wh, ch):
        wh = np.ascontiguousarray(wh, dtype=np.float64)
        c = (C.c_int * 3)(*(list(ch) + [0] * (3 - len(ch))))
        out = np.zeros(self.V)
        self.L.orc_project_sp(self.h, _dp(wh), c, _dp(out))
        return out

    def indicator_at(self, lv, i, j, k=0):
        return self.L.orc_indicator_at(self.h, lv, i, j, k)

    def ic_average(self, lv, i, j, k=0):
        out = np.zeros(self.V)
        self.L.orc_ic_average(self.h, lv, i, j, k, _dp(out))
        return out

    def totals(self):
        out = np.zeros(self.V)
        self.L.orc_totals(self.h, _dp(out))
        return out


def tables(M, d=2):
    """GL nodes/weights on [0,1], Lagrange coefficients (of (xi-1/2)^k), stencil inverses, Sigma."""
    N = M + 1
    x, w = np.zeros(N), np.zeros(N)
    psi = np.zeros((N, N))
    ainv = np.zeros((4, N, N))
    sig = np.zeros((N, N))
    sl = (C.c_int * 4)()
    sr = (C.c_int * 4)()
    lam = np.zeros(4)
    ns = lib().orc_tables(M, d, _dp(x), _dp(w), _dp(psi), _dp(ainv), _dp(sig), sl, sr, _dp(lam))
    return dict(x=x, w=w, psi=psi, ainv=ainv[:ns], sig=sig, SL=list(sl)[:ns], SR=list(sr)[:ns], lam=lam[:ns], Ns=ns)


def st_matrices(M, d=2):
    N = M + 1
    nsp = N ** d
    nst = nsp * N
    k1inv = np.zeros((nst, nst))
    kd = np.zeros((d, nst, nst))
    f0 = np.zeros((nst, nsp))
    lib().orc_st_matrices(M, d, _dp(k1inv), _dp(kd), _dp(f0))
    return k1inv, kd, f0


def weno1d(M, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(M + 1)
    lib().orc_weno1d(M, _dp(v), _dp(out))
    return out


def radial_explosion(d, R=0.5, rho_in=1.0, p_in=1.0, rho_out=0.125, p_out=0.1, gamma=1.4, n=10000, rmax=1.5,
                     t_end=0.25, cfl=0.4):
    """1D radial reference of the explosion problems (Eq. eq.1D): zone centres and (rho, u, p)"""
    rho, u, p = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().orc_radial_explosion(d, R, rho_in, p_in, rho_out, p_out, gamma, n, rmax, t_end, cfl, _dp(rho), _dp(u),
                               _dp(p))
    r = (np.arange(n) + 0.5) * rmax / n
    return r, rho, u, p
