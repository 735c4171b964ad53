"""Parity of the CUDA path with the FP64 oracle, element by element on the same seeded inputs.

Tolerance: 1e-10 relative per step for cell averages and kernel outputs, per variable (each
variable's largest difference over the largest magnitude of that variable, floored at 1e-2 of
the largest magnitude of the state for variables that hold rounding noise only; see
``tests/pairs.py``); the mesh (levels, statuses, indices) must be identical given identical
refinement flags.  Sizes span
several WENO tiles (8x8 in 2D, 4x4x4 in 3D) and a ragged tail.  The product path's own regrid
(device indicator, flags and regrid inside ``aw_step`` / ``aw_advance_to``) is held to the
oracle's own regrid over whole solves, with identical trees at every level-0 step.
"""
import numpy as np
import pytest

import aw_inputs
import oracle
import paper_1212_3585_gb300 as pg
from tests.pairs import IC_MAP, RTOL, Pair, rel_err

IC_MAP_G = {k: v[1] for k, v in IC_MAP.items()}

pytestmark = pytest.mark.gpu

EXPL = [0.5, 1.0, 1.0, 0.125, 0.1]


def by_var(buf, what, V, per=None):
    """internal dump -> (points, V): WENO/predictor dumps are [cell][v][dof]; for face fluxes
    ([cell][axis][side][v]) the low face of every axis, the face each cell always computes"""
    if what == 3:
        return buf.reshape(-1, 2, V)[:, 0, :]
    return buf.reshape(-1, V, per).transpose(0, 2, 1).reshape(-1, V)


VORTEX = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("bc", ["periodic", "transmissive"])
def test_uniform_euler_kernels(M, bc):
    """WENO dofs, predictor dofs, face fluxes and averages after one step of a uniform grid."""
    p = Pair(dim=2, M=M, n=(22, 17, 1), bc=bc)
    params = aw_inputs.fourier_params(seed=1, dim=2, pde="euler", nmodes=4)
    p.init("fourier", params)
    dt = 0.5 * p.o.compute_dt()
    p.o.advance_dt(dt)
    p.g.step_dt(dt)
    for what in (0, 1, 3):
        a = p.g.internal(what, 0)
        b = p.o.internal(what, 0)
        assert a.shape == b.shape
        per = {0: (M + 1) ** 2, 1: (M + 1) ** 3, 3: None}[what]
        assert rel_err(by_var(a, what, 4, per), by_var(b, what, 4, per)) <= RTOL, what
    p.check_cells()


def test_vortex_config_full_size_20_steps():
    """2D Euler M=2 vortex on the periodic 32x32 grid of [0,10]^2, CFL 0.9, 20 steps."""
    p = Pair(dim=2, M=2, n=(32, 32, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc="periodic")
    p.init("vortex", VORTEX)
    for _ in range(20):
        p.step()


@pytest.mark.parametrize("pde,M,dim", [("linadv", 1, 2), ("linadv", 2, 2), ("linadv", 3, 2), ("linadv", 2, 3), ("euler", 2, 3)])
def test_uniform_other_systems(pde, M, dim):
    n = (9, 7, 6) if dim == 3 else (13, 10, 1)
    p = Pair(dim=dim, pde=pde, M=M, n=n, bc="periodic")
    p.init("fourier", aw_inputs.fourier_params(seed=2, dim=dim, pde=pde, nmodes=3))
    for _ in range(2):
        p.step()


@pytest.mark.parametrize("M,lmax", [(3, 2), (2, 1), (1, 2)])
def test_amr_explosion_lts(M, lmax):
    """Explosion shaped like the 2D AMR configuration at a small base grid: tree bit-exact,
    averages within tolerance after each level-0 step with local time stepping and regrids."""
    p = Pair(dim=2, M=M, n=(14, 14, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc="transmissive", r=3, lmax=lmax, cfl=0.6)
    p.init("explosion", EXPL)
    n, na, cpl, apl = p.g.counts()
    assert all(a > 0 for a in apl)
    for _ in range(3):
        p.step()


def test_vortex_amr_lts():
    """the smooth vortex with one level of refinement around its core (chi_ref = 0.02) and local
    time stepping: the case of the oracle's AMR convergence pin"""
    p = Pair(dim=2, M=3, n=(16, 16, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc="periodic", r=3, lmax=1, chi_ref=0.02,
             chi_rec=0.01)
    p.init("vortex", VORTEX)
    n, na, cpl, apl = p.g.counts()
    assert apl[1] > 0
    for _ in range(4):
        p.step()


@pytest.mark.parametrize("M,r,lmax,n", [(3, 4, 2, 10), (2, 2, 3, 16), (1, 4, 2, 10)])
def test_amr_deep_and_wide_refinement(M, r, lmax, n):
    """refinement factor 4 (the paper's efficiency-table setting) and a four-level hierarchy with
    r = 2: local time stepping over r^l_max sub-steps, memory variables on every interface"""
    p = Pair(dim=2, M=M, n=(n, n, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc="transmissive", r=r, lmax=lmax, cfl=0.6)
    p.init("explosion", EXPL)
    n_, na, cpl, apl = p.g.counts()
    assert all(a > 0 for a in apl)
    for _ in range(2):
        p.step()


def test_amr_periodic_conservation_gpu():
    p = Pair(dim=2, M=3, n=(12, 12, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc="periodic", r=3, lmax=2, chi_ref=0.1,
             chi_rec=0.01)
    p.init("vortex", VORTEX)
    t0 = p.g.totals()
    for _ in range(2):
        p.step()
    t1 = p.g.totals()
    assert np.allclose(t1, t0, rtol=1e-13, atol=1e-13 * np.abs(t0).max())


def test_mhd_orszag_tang_amr():
    p = Pair(dim=2, pde="mhd", M=3, n=(12, 12, 1), lo=(0, 0, 0), hi=(2 * np.pi, 2 * np.pi, 1), bc="periodic",
             r=3, lmax=1, gamma=5 / 3, c_h=2.0, chi_ref=0.05, chi_rec=0.02)
    p.init("ot", [])
    for _ in range(2):
        p.step()


@pytest.mark.parametrize("lmax", [0, 1])
def test_mhd_osher_orszag_tang(lmax):
    """Osher-Solomon flux for MHD-GLM (Eq. eqn.osher, Sec. 4.2): |A| of the 9 x 9 Jacobian along the
    path, uniform and with AMR and local time stepping (the Orszag-Tang density is constant at
    t = 0, so the indicator refines nothing yet: random refinement flags make the coarse/fine
    faces)"""
    p = Pair(dim=2, pde="mhd", M=3, n=(12, 12, 1), lo=(0, 0, 0), hi=(2 * np.pi, 2 * np.pi, 1), bc="periodic",
             r=3, lmax=lmax, gamma=5 / 3, c_h=2.0, flux=1)
    p.init("ot", [], passes=0)
    if lmax:
        meta, _ = p.o.cells()
        flags = aw_inputs.random_flags(np.random.default_rng(11), meta, p_refine=0.3, p_coarsen=0.0)
        p.o.regrid_with_flags(flags, init_mode=1)
        p.g.regrid_with_flags(flags, init_mode=1)
        p.check_cells(tol=1e-12)
        assert p.g.counts()[3][1] > 0
    for _ in range(2):
        p.step(regrid=False)


def test_3d_explosion_amr():
    p = Pair(dim=3, M=2, n=(6, 6, 6), lo=(-1, -1, -1), hi=(1, 1, 1), bc="transmissive", r=3, lmax=1, cfl=0.6)
    p.init("explosion", EXPL)
    p.step()


def test_indicator_matches_oracle():
    p = Pair(dim=2, M=3, n=(14, 14, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc="transmissive", r=3, lmax=2, cfl=0.6)
    p.init("explosion", EXPL)
    p.step(regrid=False)
    fo = p.o.compute_flags(0)
    fg = p.g.compute_flags(0)
    chi_o = {}
    for lv in range(2):
        co = p.o.internal(2, lv)
        cg = p.g.internal(2, lv)
        assert rel_err(cg, co) <= 1e-9
        chi_o[lv] = co
    # flags may only differ where the indicator sits on a threshold: every mismatched cell's
    # neighbourhood maximum of chi (reading R14) is within 1e-9 of chi_ref or chi_rec
    meta, _ = p.o.cells()
    bad = np.nonzero(fo != fg)[0]
    if bad.size:
        hat = chi_hat(meta, chi_o, (14, 14, 1), 3, periodic=False)
        for c in bad:
            h = hat[c]
            assert min(abs(h - 0.2) / 0.2, abs(h - 0.1) / 0.1) <= 1e-9, (c, meta[c], h, fo[c], fg[c])


def chi_hat(meta, chi, n, r, periodic):
    """the neighbourhood maximum of the indicator (reading R14) per existing cell in canonical
    order: over the cell and its same-level Voronoi neighbours of status 0 or -1 (out-of-domain
    neighbours skipped unless periodic), for cells of status 0 or -1; NaN elsewhere"""
    out = np.full(len(meta), np.nan)
    dim = 3 if n[2] > 1 else 2
    for lv, cl in chi.items():
        sel = np.nonzero(meta[:, 0] == lv)[0]
        L = [n[a] * r ** lv for a in range(3)] if dim == 3 else [n[0] * r ** lv, n[1] * r ** lv, 1]
        st = np.full((L[2], L[1], L[0]), -9, dtype=np.int64)
        cv = np.full((L[2], L[1], L[0]), -np.inf)
        m = meta[sel]
        st[m[:, 4], m[:, 3], m[:, 2]] = m[:, 1]
        cv[m[:, 4], m[:, 3], m[:, 2]] = cl
        offs = [(di, dj, dk) for dk in ((-1, 0, 1) if dim == 3 else (0,)) for dj in (-1, 0, 1) for di in (-1, 0, 1)]
        for idx, (lv_, s_, i, j, k) in zip(sel, m):
            if s_ not in (0, -1):
                continue
            h = cv[k, j, i]
            for di, dj, dk in offs:
                ii, jj, kk = i + di, j + dj, k + dk
                if periodic:
                    ii, jj, kk = ii % L[0], jj % L[1], kk % L[2]
                elif not (0 <= ii < L[0] and 0 <= jj < L[1] and 0 <= kk < L[2]):
                    continue
                if st[kk, jj, ii] in (0, -1):
                    h = max(h, cv[kk, jj, ii])
            out[idx] = h
    return out


def _own_refinement(p, ic, params):
    """each side's own initial refinement (its indicator, l_max passes at t = 0); trees must agree"""
    oi, gi = IC_MAP[ic]
    p.o.set_initial(oi, params, nrefine=p.lmax)
    p.g.set_initial(gi, params, nrefine=-1)
    return p.check_cells(tol=1e-12)


@pytest.mark.parametrize("case", ["vortex", "explosion"])
def test_product_path_own_regrid_whole_solve(case):
    """The path the bench and the request loop run: every level-0 step is the CFL step of aw_step
    followed by the device's own indicator, flags, closure and regrid (auto_regrid = 1), against
    the oracle's own orc_step with its own regrid. Trees identical and averages within the
    per-variable tolerance after every level-0 step, the last step clipped at t_end; then the
    same solve through the one call aw_advance_to on a fresh solver gives the same tree and
    averages. Vortex: the smooth AMR vortex of the oracle's AMR convergence pin (Sec. 4.1) with
    refinement around its core; explosion: the 2D AMR explosion at a small base (two levels)."""
    if case == "vortex":
        kw = dict(dim=2, M=3, n=(16, 16, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc="periodic", r=3, lmax=1,
                  chi_ref=0.02, chi_rec=0.01, cfl=0.9)
        ic, params, t_end = "vortex", VORTEX, 0.6
    else:
        kw = dict(dim=2, M=3, n=(14, 14, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc="transmissive", r=3, lmax=2,
                  cfl=0.6)
        ic, params, t_end = "explosion", EXPL, 0.12
    p = Pair(auto_regrid=1, **kw)
    _own_refinement(p, ic, params)
    assert p.g.counts()[3][1] > 0
    steps, trees_changed, prev = 0, 0, p.o.cells()[0]
    while p.o.t < t_end:
        p.solve_step(t_end)
        steps += 1
        cur = p.o.cells()[0]
        trees_changed += int(cur.shape != prev.shape or not np.array_equal(cur, prev))
        prev = cur
    assert steps >= 5 and p.g.t == t_end
    assert trees_changed >= 1          # the regrid did change the tree along the way
    mo, uo = p.o.cells()
    q = Pair(auto_regrid=1, **kw)
    q.o = None
    g2 = q.g
    g2.set_initial(IC_MAP_G[ic], params, nrefine=-1)
    st = g2.advance_to(t_end)
    assert st.level0_steps == steps
    mg, ug = g2.cells()
    assert np.array_equal(mg, mo), "aw_advance_to's tree differs from the oracle's"
    assert rel_err(ug[mo[:, 1] <= 0], uo[mo[:, 1] <= 0]) <= RTOL


def test_3d_explosion_r3_two_levels():
    """The 3D explosion configuration's hierarchy on a small base: r = 3, l_max = 2 (nine fine
    sub-steps per level-0 step, two coarse/fine interface levels), M = 2, transmissive, CFL 0.6;
    trees identical and averages within the per-variable tolerance after every level-0 step and
    every regrid."""
    p = Pair(dim=3, M=2, n=(5, 5, 5), lo=(-1, -1, -1), hi=(1, 1, 1), bc="transmissive", r=3, lmax=2, cfl=0.6,
             threads=16)
    p.init("explosion", EXPL)
    n, na, cpl, apl = p.g.counts()
    assert apl[1] > 0 and apl[2] > 0
    for _ in range(2):
        p.step()


def test_random_flags_tree_parity():
    """random refine/coarsen flags: identical trees and values, also for flags the oracle's
    indicator would never produce"""
    p = Pair(dim=2, M=3, n=(10, 9, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc="periodic", r=3, lmax=3)
    p.init("fourier", aw_inputs.fourier_params(seed=4, dim=2, pde="euler", nmodes=3), passes=0)
    rng = np.random.default_rng(5)
    for it in range(4):
        meta, _ = p.o.cells()
        flags = aw_inputs.random_flags(rng, meta, p_refine=0.1 if it < 3 else 0.02, p_coarsen=0.5)
        p.o.regrid_with_flags(flags, init_mode=0)
        p.g.regrid_with_flags(flags, init_mode=0)
        p.check_cells(tol=RTOL)
    p.step(regrid=False)


def test_empty_levels_and_errors():
    g = pg.Solver(pg.make_config(dim=2, M=2, n=(8, 8, 1), lmax=2, r=3))
    g.set_initial(pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], nrefine=2)
    n, na, cpl, apl = g.counts()
    assert cpl == [64, 0, 0] and apl == [64, 0, 0]
    g.step()
    with pytest.raises(pg.AwError):
        g.set_cell_averages(np.zeros((3, 4)))
    with pytest.raises(pg.AwError):
        pg.Solver(pg.make_config(dim=2, M=5))
    # a negative density is reported as a non-physical state
    m, u = g.cells()
    u[5, 0] = -1.0
    g.set_cell_averages(u)
    with pytest.raises(pg.AwError) as ei:
        g.step_dt(1e-3)
    assert ei.value.code == pg._lib.AW_ENONPHYSICAL


@pytest.mark.parametrize("dim,M,lmax", [(2, 3, 0), (2, 3, 2), (3, 2, 1), (2, 1, 2)])
def test_osher_flux_explosion(dim, M, lmax):
    """Osher-Solomon flux (Eq. eqn.osher), uniform and AMR with local time stepping"""
    n = (16, 16, 1) if dim == 2 else (6, 6, 6)
    p = Pair(dim=dim, M=M, n=n, lo=(-1, -1, -1), hi=(1, 1, 1), bc="transmissive", r=3, lmax=lmax, cfl=0.6,
             flux=1)
    p.init("explosion", EXPL)
    for _ in range(2):
        p.step()


@pytest.mark.parametrize("dim,M,lmax,flux,n3", [(2, 3, 1, 0, 5), (2, 2, 2, 1, 5), (3, 2, 1, 0, 5), (2, 1, 1, 1, 5),
                                                 (3, 2, 1, 1, 8)])
def test_reflective_walls(dim, M, lmax, flux, n3):
    """walls on the low faces, transmissive high faces: the quadrant of the centred explosion (the
    8^3 case's level 1 is large enough for the WENO by passes, the 5^3 one keeps the tiles)"""
    R, T = pg.AW_BC_REFLECTIVE, pg.AW_BC_TRANSMISSIVE
    n = (10, 10, 1) if dim == 2 else (n3, n3, n3)
    p = Pair(dim=dim, M=M, n=n, lo=(0, 0, 0), hi=(1, 1, 1), bc=[R, T, R, T, R, T], r=3, lmax=lmax, cfl=0.6,
             flux=flux)
    p.init("explosion", EXPL)
    for _ in range(2):
        p.step()


@pytest.mark.parametrize("dim,M,lmax,flux", [(2, 3, 2, 0), (2, 2, 1, 1), (3, 2, 1, 0)])
def test_inflow_boundary(dim, M, lmax, flux):
    """a Mach-3 shock entering through an inflow face into gas at rest (the post-shock state is the
    inflow state), transmissive elsewhere, with AMR and local time stepping"""
    g = 1.4
    # Rankine-Hugoniot post-shock state of a Mach-3 shock running into rho = 1.4, p = 1, u = 0
    rho1, p1, ms = 1.4, 1.0, 3.0
    rho2 = rho1 * (g + 1) * ms ** 2 / ((g - 1) * ms ** 2 + 2)
    p2 = p1 * (2 * g * ms ** 2 - (g - 1)) / (g + 1)
    u2 = ms * (1 - rho1 / rho2)                      # sound speed 1 ahead of the shock
    E2 = p2 / (g - 1) + 0.5 * rho2 * u2 ** 2
    qin = [rho2, rho2 * u2] + [0.0] * (dim - 1) + [E2]
    I, T = pg.AW_BC_INFLOW, pg.AW_BC_TRANSMISSIVE
    n = (16, 12, 1) if dim == 2 else (8, 6, 6)
    p = Pair(dim=dim, M=M, n=n, lo=(0, 0, 0), hi=(1, 0.75, 0.75), bc=[I, T, T, T, T, T], r=3, lmax=lmax,
             cfl=0.5, flux=flux, inflow=qin)
    p.init("const", [rho1, 0.0] + [0.0] * (dim - 1) + [p1])
    for _ in range(3):
        p.step()
    m, u = p.g.cells()
    assert np.max(u[:, 0]) > 1.5 * rho1          # the shock has entered
