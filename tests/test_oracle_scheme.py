"""Pins of the oracle's whole scheme (Secs. 2-3 of the paper).

  * Free stream: a constant state stays constant through WENO, predictor, fluxes and update,
    on a uniform grid and on an AMR grid with local time stepping.
  * Conservation (Eq. eq:finite_vol with the memory variables of Eq. eqn.memory.sum): on a
    periodic domain the totals sum(vol * u) over active cells are conserved to round-off
    across refinement levels with local time stepping.
  * Local time stepping (Eq. eqn.update.criterion): a level-0 grid that is refined
    everywhere (l_max = 1) advanced by dt_0 equals a uniform r-times finer grid advanced
    r times by dt_0 / r.
  * Projection and averaging (Sec. 3.1.3, Eq. eqn.average): the average of the r^d child
    projections of a mother polynomial is the mother's average.
  * Design order of accuracy on the isentropic vortex of Sec. 4.1 with its exact solution
    (advection by (1,1)): observed L2 order of rho close to M+1.
  * Design order in the max norm of linear advection across a fixed refined patch, where the
    errors of coarse/fine faces (Sec. 3.1.3) concentrate: in 2D on square and on anisotropic
    cells, and in 3D with conservation of the total.
  * Local time stepping leaves the level-0 step of a refined constant state unchanged.
  * The errors the paper prints for the vortex on its coarse uniform grids (Table tab.conv2,
    tests/golden/tab_conv2_uniform.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle
from tests.polyref import gl01

VORTEX = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]


def vortex_prim(x, y, t, gamma=1.4, eps=5.0):
    # exact solution: the initial vortex advected with velocity (1, 1), period 10
    xc = (x - t - 5.0 + 5.0) % 10.0 - 5.0
    yc = (y - t - 5.0 + 5.0) % 10.0 - 5.0
    r2 = xc * xc + yc * yc
    dT = -eps * eps * (gamma - 1) / (8 * gamma * math.pi ** 2) * np.exp(1 - r2)
    rho = (1 + dT) ** (1 / (gamma - 1))
    return rho


def exact_rho_averages(n, L, t, nq=8):
    x, w = gl01(nq)
    h = L / n
    out = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            X = (i + x[:, None]) * h
            Y = (j + x[None, :]) * h
            out[j, i] = np.sum(w[:, None] * w[None, :] * vortex_prim(X, Y, t))
    return out


def test_free_stream_uniform_and_amr():
    q = [1.1, 0.4, -0.3, 0.9]
    for lmax in (0, 1):
        cfg = oracle.make_cfg(dim=2, M=3, n=(9, 9, 1), lo=(0, 0, 0), hi=(1, 1, 1), lmax=lmax, r=3,
                              auto_regrid=0)
        o = oracle.Oracle(cfg)
        o.set_initial(oracle.IC_CONST, q, nrefine=0)
        if lmax:
            _, u = o.cells()
            flags = np.zeros(len(u), dtype=np.int8)
            flags[[10, 11, 40]] = 1
            o.regrid_with_flags(flags, init_mode=1)
        meta0, u0 = o.cells()
        for _ in range(2):
            o.advance_dt(0.5 * o.compute_dt())
        meta1, u1 = o.cells()
        assert np.array_equal(meta0, meta1)
        act = meta1[:, 1] <= 0
        cons = np.array([1.1, 1.1 * 0.4, 1.1 * -0.3, 0.9 / 0.4 + 0.5 * 1.1 * (0.16 + 0.09)])
        assert np.allclose(u1[act], cons, rtol=1e-13, atol=1e-13)


def test_lts_level0_step_not_limited_by_refinement():
    """level l takes r^l steps per level-0 step, so refining cells of a constant state (cells
    r^l times smaller) leaves the level-0 time step unchanged (Eq. eqn.update.criterion)"""
    q = [1.1, 0.4, -0.3, 0.9]
    for lmax in (1, 2):
        cfg = oracle.make_cfg(dim=2, M=2, n=(9, 9, 1), lo=(0, 0, 0), hi=(1, 1.5, 1), lmax=lmax, r=3,
                              auto_regrid=0)
        o = oracle.Oracle(cfg)
        o.set_initial(oracle.IC_CONST, q, nrefine=0)
        dt_uniform = o.compute_dt()
        for lv in range(lmax):
            meta, _ = o.cells()
            act = np.flatnonzero((meta[:, 0] == lv) & (meta[:, 1] == 0))
            flags = np.zeros(len(meta), dtype=np.int8)
            flags[act[len(act) // 2:len(act) // 2 + 3]] = 1
            o.regrid_with_flags(flags, init_mode=1)
        _, _, act = o.counts()
        assert all(a > 0 for a in act)
        assert o.compute_dt() == pytest.approx(dt_uniform, rel=1e-14)


@pytest.mark.parametrize("M,lmax", [(1, 1), (2, 1), (3, 2)])
def test_conservation_amr_lts_periodic(M, lmax):
    cfg = oracle.make_cfg(dim=2, M=M, n=(12, 12, 1), lo=(0, 0, 0), hi=(10, 10, 1), lmax=lmax, r=3,
                          chi_ref=0.1, chi_rec=0.01, auto_regrid=1)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_VORTEX, VORTEX)
    n, per, act = o.counts()
    assert all(a > 0 for a in act), "every level must hold active cells for this test"
    tot0 = o.totals()
    for _ in range(2):
        rc, _ = o.step()
        assert rc == 0
    tot1 = o.totals()
    assert np.allclose(tot1, tot0, rtol=1e-13, atol=1e-13 * np.abs(tot0).max())


def test_conservation_amr_lts_mhd():
    """all nine totals of MHD-GLM (psi included) on a periodic AMR mesh with local time stepping:
    the Orszag-Tang data (constant density, so the density indicator refines nothing) with a
    refined block of cells kept fixed"""
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, M=3, n=(12, 12, 1), lo=(0, 0, 0), hi=(2 * math.pi, 2 * math.pi, 1),
                          lmax=1, r=3, gamma=5.0 / 3.0, c_h=2.0, cfl=0.6, auto_regrid=0)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_OT, [], nrefine=0)
    meta, _ = o.cells()
    o.regrid_with_flags(((meta[:, 2] >= 2) & (meta[:, 2] < 7) & (meta[:, 3] >= 4) & (meta[:, 3] < 9)).astype(np.int8),
                        init_mode=1)
    _, _, act = o.counts()
    assert act[1] == 25 * 9
    tot0 = o.totals()
    for _ in range(2):
        rc, _ = o.step()
        assert rc == 0
    assert np.allclose(o.totals(), tot0, rtol=0, atol=1e-13 * np.abs(tot0).max())


def test_conservation_amr_lts_3d():
    """all five totals of the 3D explosion in a periodic box with one AMR level: a refined block
    of 3^3 base cells, kept fixed, cuts through the jump, so coarse/fine faces of every
    orientation carry the flow (the indicator would refine the whole of this coarse grid)"""
    cfg = oracle.make_cfg(dim=3, M=2, n=(6, 6, 6), lo=(-1, -1, -1), hi=(1, 1, 1), bc=oracle.BC_PERIODIC, lmax=1,
                          r=3, cfl=0.6, auto_regrid=0)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_EXPLOSION, [0.5, 1.0, 1.0, 0.125, 0.1], nrefine=0)
    meta, _ = o.cells()
    blk = lambda c: (c >= 1) & (c < 4)
    o.regrid_with_flags((blk(meta[:, 2]) & blk(meta[:, 3]) & blk(meta[:, 4])).astype(np.int8), init_mode=1)
    _, _, act = o.counts()
    assert act == [216 - 27, 27 * 27]
    tot0 = o.totals()
    for _ in range(2):
        rc, _ = o.step()
        assert rc == 0
    assert np.allclose(o.totals(), tot0, rtol=0, atol=1e-13 * np.abs(tot0).max())


@pytest.mark.parametrize("M", [2, 3])
def test_fully_refined_equals_uniform_fine(M):
    n, r = 6, 3
    params = [1.0, 0.5, -0.2, 1.0, 2, 0, 1, 1, 0, 0.1, 0.3, 3, 2, 1, 0, 0.05, 1.1]
    a = oracle.Oracle(oracle.make_cfg(dim=2, M=M, n=(n, n, 1), lmax=1, r=r, auto_regrid=0))
    a.set_initial(oracle.IC_FOURIER, params, nrefine=0)
    _, u = a.cells()
    a.regrid_with_flags(np.ones(len(u), dtype=np.int8), init_mode=1)
    b = oracle.Oracle(oracle.make_cfg(dim=2, M=M, n=(n * r, n * r, 1), lmax=0))
    b.set_initial(oracle.IC_FOURIER, params, nrefine=0)
    meta, ua = a.cells()
    fine = meta[:, 0] == 1
    assert np.all(meta[fine, 1] == 0) and np.all(meta[~fine, 1] == -1)
    _, ub = b.cells()
    assert np.allclose(ua[fine], ub, rtol=0, atol=1e-15)
    dt0 = 0.5 * a.compute_dt()
    a.advance_dt(dt0)
    for _ in range(r):
        b.advance_dt(dt0 / r)
    meta, ua = a.cells()
    _, ub = b.cells()
    assert np.allclose(ua[fine], ub, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_projection_then_average_is_identity(d):
    M, r = 3 if d == 2 else 2, 3
    o = oracle.Oracle(oracle.make_cfg(dim=d, M=M, n=(4, 4, 4), r=r))
    rng = np.random.default_rng(12)
    wh = rng.normal(size=o.V * o.nsp)
    qh = rng.normal(size=o.V * o.nst)
    mother_avg_sp = np.zeros(o.V)
    x, w = gl01(M + 1)
    # mother's own averages by Gauss quadrature of the nodal polynomial = weighted nodal sum
    W = np.ones(1)
    for _a in range(d):
        W = np.kron(w, W)
    mother_avg_sp = wh.reshape(o.V, o.nsp) @ W
    kids = []
    kids_st = []
    tau = 0.37
    for c in np.ndindex(*([r] * d)):
        ch = list(c[::-1])
        kids.append(o.project_sp(wh, ch))
        kids_st.append(o.project_st(qh, ch, tau))
    assert np.allclose(np.mean(kids, axis=0), mother_avg_sp, rtol=1e-13, atol=1e-13)
    # space-time: the mother's average at tau, from its own nodal dofs
    x, _ = gl01(M + 1)
    from tests.polyref import lagrange_values
    bt = lagrange_values(x, [tau])[0]
    q = qh.reshape(o.V, M + 1, o.nsp)        # [v][s][spatial]
    avg_tau = np.einsum("vsp,s,p->v", q, bt, W)
    assert np.allclose(np.mean(kids_st, axis=0), avg_tau, rtol=1e-13, atol=1e-13)


def _vortex_l2(M, n, t_end):
    cfg = oracle.make_cfg(dim=2, M=M, n=(n, n, 1), lo=(0, 0, 0), hi=(10, 10, 1))
    o = oracle.Oracle(cfg, threads=4)
    o.set_initial(oracle.IC_VORTEX, VORTEX)
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    meta, u = o.cells()
    rho = u[:, 0].reshape(n, n)
    ex = exact_rho_averages(n, 10.0, t_end)
    return math.sqrt(np.sum((rho - ex) ** 2) * (10.0 / n) ** 2)


@pytest.mark.parametrize("M,grids,lo_order", [(2, (48, 96), 2.6), (3, (20, 40), 3.2)])
def test_vortex_design_order(M, grids, lo_order):
    e = [_vortex_l2(M, n, 1.0) for n in grids]
    order = math.log(e[0] / e[1]) / math.log(grids[1] / grids[0])
    assert order > lo_order, (e, order)


def test_vortex_coarse_errors_match_the_paper():
    """the L2 density errors the paper prints for the coarse uniform grids of Table tab.conv2
    (tests/golden/tab_conv2_uniform.txt), reproduced within 10 %: the whole scheme (WENO,
    predictor, fluxes, update) over 10 time units; the paper states neither the CFL number nor
    the discrete form of its norm (measured: 0.535 against 0.501, 0.504 against 0.515)"""
    path = os.path.join(os.path.dirname(__file__), "golden", "tab_conv2_uniform.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for M, n, eps in rows:
        e = _vortex_l2(int(M), int(n), 10.0)
        assert abs(e - float(eps)) < 0.1 * float(eps), (M, n, e, eps)


def _vortex_amr_l2(M, n, t_end):
    """L2 error of rho over the active cells of both levels (each against the exact averages of
    its own level) of the vortex with one level of refinement around its core (chi_ref = 0.02)"""
    cfg = oracle.make_cfg(dim=2, M=M, n=(n, n, 1), lo=(0, 0, 0), hi=(10, 10, 1), r=3, lmax=1, chi_ref=0.02,
                          chi_rec=0.01, auto_regrid=1)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_VORTEX, VORTEX)
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    meta, u = o.cells()
    e2, counts = 0.0, []
    for lv in range(2):
        sel = (meta[:, 0] == lv) & (meta[:, 1] == 0)
        nn = n * 3 ** lv
        ex = exact_rho_averages(nn, 10.0, t_end)
        m = meta[sel]
        e2 += np.sum((u[sel, 0] - ex[m[:, 3], m[:, 2]]) ** 2) * (10.0 / nn) ** 2
        counts.append(int(sel.sum()))
    assert min(counts) > 0    # both levels carry active cells
    return math.sqrt(e2)


@pytest.mark.parametrize("M,grids,lo_order", [(2, (24, 48), 2.5), (3, (16, 32), 3.2)])
def test_vortex_design_order_with_amr(M, grids, lo_order):
    """the design order survives local time stepping and coarse/fine faces (measured: 2.73, 3.49)"""
    e = [_vortex_amr_l2(M, n, 1.0) for n in grids]
    order = math.log(e[0] / e[1]) / math.log(grids[1] / grids[0])
    assert order > lo_order, (e, order)


def _patch_errors(M, n, t_end, ly=1.0):
    """linear advection of sin 2 pi (x + 2y / ly) by (1, 1/2) on a periodic base grid of n^2
    cells over [0, 1] x [0, ly] whose middle [1/4, 3/4)^2 (in units of the sides) is refined once
    (r = 3) and kept fixed: the wave crosses coarse/fine faces on all four sides, with local time
    stepping.  Returns the L2 and max-norm errors over the active cells against the exact
    averages."""
    a = (1.0, 0.5)
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_LINADV, M=M, n=(n, n, 1), lo=(0, 0, 0), hi=(1, ly, 1),
                          adv=(a[0], a[1], 0.0), lmax=1, r=3, auto_regrid=0, cfl=0.9)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_FOURIER, [0.0, 1, 0, 1, 2, 0, 1.0, 0.0], nrefine=0)
    meta, _ = o.cells()
    i, j = meta[:, 2], meta[:, 3]
    o.regrid_with_flags(((i >= n // 4) & (i < 3 * n // 4) & (j >= n // 4) & (j < 3 * n // 4)).astype(np.int8),
                        init_mode=1)
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    meta, u = o.cells()
    act = meta[:, 1] == 0
    assert np.count_nonzero(meta[act, 0] == 1) == (3 * n // 2) ** 2
    h = (1.0 / n) / 3.0 ** meta[act, 0]
    x, w = gl01(8)
    X = (meta[act, 2] * h)[:, None, None] + x[None, :, None] * h[:, None, None] - a[0] * t_end
    Y = (meta[act, 3] * h * ly)[:, None, None] + x[None, None, :] * h[:, None, None] * ly - a[1] * t_end
    ex = np.sum(w[None, :, None] * w[None, None, :] * np.sin(2 * np.pi * (X + 2 * Y / ly)), axis=(1, 2))
    err = u[act, 0] - ex
    return math.sqrt(np.sum(err ** 2 * h * h * ly)), np.max(np.abs(err))


@pytest.mark.parametrize("M,lo_order,ly", [(2, 2.7, 1.0), (3, 3.6, 1.0), (3, 3.6, 2.0)])
def test_coarse_fine_patch_design_order(M, lo_order, ly):
    """the max-norm error keeps the design order M+1 in the cells along the coarse/fine faces
    (measured from 12 to 48 cells: 2.98, 3.05 for M=2; 4.39, 5.30 for M=3).  Errors confined to
    those faces hide in the L2 norm: the coarse polynomial taken at the centre of each fine face
    instead of at its Gauss points gives 3.37 from 24 to 48 cells (M=3), the coarse time of the
    sub-step or of the virtual children's projection taken at its start about 1.  With ly = 2 the
    cells are twice as high as wide, which every other whole-scheme pin leaves square (measured
    4.65, 5.38); an update that divides by dx for every axis fails only there."""
    e = [_patch_errors(M, n, 0.25, ly) for n in (12, 24, 48)]
    for norm in (0, 1):
        orders = [math.log(e[k][norm] / e[k + 1][norm], 2) for k in range(2)]
        assert min(orders) > lo_order, (norm, e, orders)


def _patch3_errors(n, t_end):
    """3D counterpart of _patch_errors: sin 2 pi (x + y + z) advected by (1, 1/2, 1/4) on a
    periodic n^3 base grid whose middle cube [1/4, 3/4)^3 is refined once (r = 3, M = 2, local
    time stepping).  Returns the L2 and max-norm errors over the active cells and the change of
    the total."""
    a = (1.0, 0.5, 0.25)
    cfg = oracle.make_cfg(dim=3, pde=oracle.PDE_LINADV, M=2, n=(n, n, n), lo=(0, 0, 0), hi=(1, 1, 1), adv=a,
                          lmax=1, r=3, auto_regrid=0, cfl=0.9)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_FOURIER, [0.0, 1, 0, 1, 1, 1, 1.0, 0.0], nrefine=0)
    meta, _ = o.cells()
    mid = lambda c: (c >= n // 4) & (c < 3 * n // 4)
    o.regrid_with_flags((mid(meta[:, 2]) & mid(meta[:, 3]) & mid(meta[:, 4])).astype(np.int8), init_mode=1)
    tot0 = o.totals()[0]
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    meta, u = o.cells()
    act = meta[:, 1] == 0
    assert np.count_nonzero(meta[act, 0] == 1) == (3 * n // 2) ** 3
    h = (1.0 / n) / 3.0 ** meta[act, 0]
    x, w = gl01(6)
    # the box average of sin 2 pi (x + y + z) is the imaginary part of the product over the axes
    # of the averages of exp(2 pi i x_a)
    ex = np.ones(np.count_nonzero(act), dtype=complex)
    for b in range(3):
        xa = (meta[act, 2 + b] * h)[:, None] + x[None, :] * h[:, None] - a[b] * t_end
        ex *= np.sum(w[None, :] * np.exp(2j * np.pi * xa), axis=1)
    err = u[act, 0] - ex.imag
    return math.sqrt(np.sum(err ** 2 * h ** 3)), np.max(np.abs(err)), o.totals()[0] - tot0


def test_coarse_fine_patch_3d():
    """coarse/fine faces with two transverse directions, 3D memory variables, projection and
    averaging over r^3 children: the total is conserved and both norms keep the design order 3
    (measured from 8^3 to 16^3: 3.03 in L2, 3.24 in the max norm)"""
    e = [_patch3_errors(n, 0.25) for n in (8, 16)]
    for norm in (0, 1):
        order = math.log(e[0][norm] / e[1][norm], 2)
        assert order > 2.7, (norm, e, order)
    assert max(abs(e[0][2]), abs(e[1][2])) < 1e-13


def _linadv_err(M, n, t_end):
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_LINADV, M=M, n=(n, n, 1), lo=(0, 0, 0), hi=(1, 1, 1),
                          adv=(1.0, 1.0, 0.0))
    o = oracle.Oracle(cfg, threads=4)
    o.set_initial(oracle.IC_FOURIER, [0.0, 1, 0, 1, 1, 0, 1.0, 0.0])
    while o.t < t_end:
        o.step(t_end)
    _, u = o.cells()
    x, w = gl01(8)
    h = 1.0 / n
    ex = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            X = (i + x[:, None]) * h - t_end
            Y = (j + x[None, :]) * h - t_end
            ex[j, i] = np.sum(w[:, None] * w[None, :] * np.sin(2 * np.pi * (X + Y)))
    return math.sqrt(np.mean((u[:, 0].reshape(n, n) - ex) ** 2))


# M = 1: the two-cell stencils' weights (exponent 8) switch near the extrema of the sine wave, so
# the second order is reached only slowly (1.67, 1.69, 1.81 from 20 to 160 cells)
@pytest.mark.parametrize("M,grids,lo_order", [(1, (40, 80, 160), 1.65), (2, (10, 20, 40), 2.85), (3, (10, 20, 40), 3.8)])
def test_linear_advection_design_order(M, grids, lo_order):
    e = [_linadv_err(M, n, 0.5) for n in grids]
    orders = [math.log(e[i] / e[i + 1], 2) for i in range(2)]
    assert min(orders) > lo_order, (e, orders)


def _wave3_averages(n, shift):
    """cell averages of sin(2 pi (x + y + z - shift)) on an n^3 grid of the unit cube (closed form:
    the average of exp(i k (x + y + z)) is the product of three one-dimensional averages)"""
    k = 2 * np.pi
    x0 = np.arange(n) / n
    f = (np.exp(1j * k * (x0 + 1.0 / n)) - np.exp(1j * k * x0)) / (1j * k / n)
    return (f[None, None, :] * f[None, :, None] * f[:, None, None] * np.exp(-1j * k * shift)).imag.reshape(-1)


def _wave3_error(pde, M, n, t_end):
    a, p, g = (1.0, 0.5, 0.25), 1.0, 1.4
    cfg = oracle.make_cfg(dim=3, pde=pde, M=M, n=(n, n, n), lo=(0, 0, 0), hi=(1, 1, 1), adv=a, cfl=0.9, gamma=g)
    o = oracle.Oracle(cfg, threads=8)

    def state(shift):
        w = _wave3_averages(n, shift)
        if pde == oracle.PDE_LINADV:
            return w.reshape(-1, 1)
        rho = 1.0 + 0.2 * w     # a density wave carried at constant velocity and pressure
        return np.stack([rho] + [a[d] * rho for d in range(3)] + [p / (g - 1) + 0.5 * sum(x * x for x in a) * rho], 1)

    o.set_initial(oracle.IC_CONST, [0.0] if pde == oracle.PDE_LINADV else [1.0, *a, p], nrefine=0)
    o.set_cell_averages(state(0.0))
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    _, u = o.cells()
    return math.sqrt(np.mean((u - state(sum(a) * t_end)) ** 2))


@pytest.mark.parametrize("pde,lo_order", [(oracle.PDE_LINADV, 2.85), (oracle.PDE_EULER, 2.4)])
def test_3d_design_order(pde, lo_order):
    """the 3D scheme (x, y and z sweeps, 3D predictor and fluxes) on a wave along the diagonal with
    an exact translated solution, M = 2, 8^3 -> 16^3 (measured: 3.00 linear advection, 2.68 Euler)"""
    e = [_wave3_error(pde, 2, n, 0.2) for n in (8, 16)]
    order = math.log(e[0] / e[1], 2)
    assert order > lo_order, (e, order)
