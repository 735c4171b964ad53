"""Drive the CUDA solver and the FP64 oracle side by side on the same seeded inputs.

The oracle decides every refinement flag (its own indicator); the CUDA solver receives the
same flags through aw_regrid_with_flags, so both meshes must be bit-identical and the cell
averages are compared within the FP64 tolerance.
"""
import numpy as np

import oracle
import paper_1212_3585_gb300 as pg

# tolerance of the normwise relative error per step: max |gpu - oracle| over cells and
# variables, divided by the largest |oracle| over the whole field (variables that stay near zero,
# such as the GLM cleaning variable psi, are measured against the state's magnitude)
RTOL = 1e-10

PDE_MAP = {"euler": (oracle.PDE_EULER, pg.AW_PDE_EULER), "mhd": (oracle.PDE_MHD, pg.AW_PDE_MHD_GLM),
           "linadv": (oracle.PDE_LINADV, pg.AW_PDE_LINADV)}
IC_MAP = {"const": (oracle.IC_CONST, pg.AW_IC_CONST), "vortex": (oracle.IC_VORTEX, pg.AW_IC_VORTEX),
          "explosion": (oracle.IC_EXPLOSION, pg.AW_IC_EXPLOSION), "ot": (oracle.IC_OT, pg.AW_IC_OT),
          "rp4": (oracle.IC_RP4, pg.AW_IC_RP4), "fourier": (oracle.IC_FOURIER, pg.AW_IC_FOURIER)}


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0 and b.size == 0:
        return 0.0
    scale = max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b)) / scale)


class Pair:
    def __init__(self, dim=2, pde="euler", M=2, n=(16, 16, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc="periodic",
                 r=3, lmax=0, gamma=1.4, c_h=2.0, chi_ref=0.2, chi_rec=0.1, cfl=0.9, adv=(1.0, 0.5, 0.25),
                 threads=8, flux=0, inflow=()):
        op, gp = PDE_MAP[pde]
        if isinstance(bc, (list, tuple)):
            obc = gbc = list(bc)   # per-face codes, identical numbering on both sides
        else:
            obc = oracle.BC_PERIODIC if bc == "periodic" else oracle.BC_TRANSMISSIVE
            gbc = pg.AW_BC_PERIODIC if bc == "periodic" else pg.AW_BC_TRANSMISSIVE
        kw = dict(dim=dim, M=M, n=n, lo=lo, hi=hi, r=r, lmax=lmax, gamma=gamma, c_h=c_h, chi_ref=chi_ref,
                  chi_rec=chi_rec, cfl=cfl, auto_regrid=0, adv=adv, inflow=inflow)
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
            assert abs(dg - dt) <= 1e-12 * dt, (dg, dt)
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
