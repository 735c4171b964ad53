"""Drive the CUDA solver and the FP64 oracle side by side on the same seeded inputs.

In ``Pair.step`` the oracle decides every refinement flag (its own indicator); the CUDA solver
receives the same flags through aw_regrid_with_flags, so both meshes must be bit-identical and
the cell averages are compared within the FP64 tolerance.  ``Pair.solve_step`` instead runs
each side's own product path (CFL step, own indicator, own regrid: ``aw_step`` on the device,
``orc_step`` on the oracle) and requires the same trees and averages.
"""
import numpy as np

import oracle
import paper_1212_3585_gb300 as pg

# tolerance of the normwise relative error per step, taken per variable: for every variable v,
# max over cells |gpu_v - oracle_v| divided by max(max over cells |oracle_v|, FLOOR * S), where S
# is the largest |oracle| over all variables and cells; the worst variable must stay below RTOL.
# The floor only matters for a variable that is zero in exact arithmetic and holds rounding
# noise only: the transverse momentum of a planar shock tube grows to 9e-14 S over 39 steps on
# both sides, with different noise.  Its differences are rounding errors of O(S) quantities, so
# it is measured against 1e-2 S (an absolute bound of 1e-12 S) rather than against its own
# noise.  Every variable above 1e-2 S is measured against its own largest magnitude.
RTOL = 1e-10
FLOOR = 1e-2
# The CFL time step (and the time a side reaches by its own steps) is a function of the state
# with relative sensitivity of order one, so it is held to the bar of the state, RTOL, not to
# the rounding of a single evaluation.
DT_RTOL = RTOL

PDE_MAP = {"euler": (oracle.PDE_EULER, pg.AW_PDE_EULER), "mhd": (oracle.PDE_MHD, pg.AW_PDE_MHD_GLM),
           "linadv": (oracle.PDE_LINADV, pg.AW_PDE_LINADV)}
IC_MAP = {"const": (oracle.IC_CONST, pg.AW_IC_CONST), "vortex": (oracle.IC_VORTEX, pg.AW_IC_VORTEX),
          "explosion": (oracle.IC_EXPLOSION, pg.AW_IC_EXPLOSION), "ot": (oracle.IC_OT, pg.AW_IC_OT),
          "rp4": (oracle.IC_RP4, pg.AW_IC_RP4), "fourier": (oracle.IC_FOURIER, pg.AW_IC_FOURIER)}


def rel_err(a, b):
    """worst per-variable normwise relative error of a against b; the last axis indexes the
    variables (a 1D array is one variable)"""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.size == 0:
        return 0.0
    a2 = a.reshape(-1, 1) if a.ndim == 1 else a.reshape(-1, a.shape[-1])
    b2 = b.reshape(-1, 1) if b.ndim == 1 else b.reshape(-1, b.shape[-1])
    if not (np.all(np.isfinite(a2)) and np.all(np.isfinite(b2))):
        return float("inf")
    S = max(float(np.max(np.abs(b2))), 1e-300)
    scale = np.maximum(np.max(np.abs(b2), axis=0), FLOOR * S)
    return float(np.max(np.max(np.abs(a2 - b2), axis=0) / scale))


class Pair:
    def __init__(self, dim=2, pde="euler", M=2, n=(16, 16, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc="periodic",
                 r=3, lmax=0, gamma=1.4, c_h=2.0, chi_ref=0.2, chi_rec=0.1, cfl=0.9, adv=(1.0, 0.5, 0.25),
                 threads=8, flux=0, inflow=(), auto_regrid=0):
        op, gp = PDE_MAP[pde]
        if isinstance(bc, (list, tuple)):
            obc = gbc = list(bc)   # per-face codes, identical numbering on both sides
        else:
            obc = oracle.BC_PERIODIC if bc == "periodic" else oracle.BC_TRANSMISSIVE
            gbc = pg.AW_BC_PERIODIC if bc == "periodic" else pg.AW_BC_TRANSMISSIVE
        kw = dict(dim=dim, M=M, n=n, lo=lo, hi=hi, r=r, lmax=lmax, gamma=gamma, c_h=c_h, chi_ref=chi_ref,
                  chi_rec=chi_rec, cfl=cfl, auto_regrid=auto_regrid, adv=adv, inflow=inflow)
        self.o = oracle.Oracle(oracle.make_cfg(pde=op, bc=obc, flux=flux, **kw), threads=threads)
        self.g = pg.Solver(pg.make_config(pde=gp, bc=gbc, flux=flux, **kw))
        self.lmax = lmax

    def init(self, ic, params, passes=None):
        oi, gi = IC_MAP[ic]
        self.o.set_initial(oi, params, nrefine=0)
        self.g.set_initial(gi, params, nrefine=0)
        self.check_cells(tol=1e-12)
        for _ in range(self.lmax if passes is None else passes):
            f = self.o.compute_flags(init_mode=1)
            self.o.regrid_with_flags(f, init_mode=1)
            self.g.regrid_with_flags(f, init_mode=1)
            self.check_cells(tol=1e-12)

    def set_state(self, u):
        self.o.set_cell_averages(u)
        self.g.set_cell_averages(u)

    def check_cells(self, tol=RTOL):
        mo, uo = self.o.cells()
        mg, ug = self.g.cells()
        assert np.array_equal(mo, mg), "meshes differ"
        e = rel_err(ug[mo[:, 1] <= 0], uo[mo[:, 1] <= 0])
        assert e <= tol, f"cell averages differ: {e:.3e} > {tol:.1e}"
        return e

    def step(self, dt=None, regrid=True, tol=RTOL):
        if dt is None:
            dt = self.o.compute_dt()
            dg = self.g.compute_dt()
            assert abs(dg - dt) <= DT_RTOL * dt, (dg, dt)
        rc = self.o.advance_dt(dt)
        assert rc == 0
        self.g.step_dt(dt)
        e = self.check_cells(tol)
        if regrid and self.lmax > 0:
            f = self.o.compute_flags(init_mode=0)
            self.o.regrid_with_flags(f, init_mode=0)
            self.g.regrid_with_flags(f, init_mode=0)
            e = max(e, self.check_cells(tol))
        return e

    def solve_step(self, t_end, tol=RTOL):
        """one level-0 step of each side's own product path: CFL dt clipped at t_end, the step,
        then (auto_regrid) each side's own indicator, flags and regrid"""
        assert self.o.cfg.auto_regrid == 1 and self.g.cfg.auto_regrid == 1
        rc, dto = self.o.step(t_end)
        assert rc == 0
        st = self.g.step(t_end)
        assert abs(self.g.t - self.o.t) <= DT_RTOL * max(1.0, abs(self.o.t)), (self.g.t, self.o.t, dto)
        return self.check_cells(tol), st
