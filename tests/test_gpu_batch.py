"""Cross-request batching (aw_advance_batch): independent solves of one kernel configuration
advanced with their hot kernels batched per level and sub-step.  Each member must compute exactly
what the same solve computes alone (identical meshes and cell averages), uniform members agree
with the oracle, mismatched members are rejected, and one member's failure stops only that one."""
import numpy as np
import pytest

import aw_inputs
import oracle
import paper_1212_3585_gb300 as pg
from tests.pairs import RTOL, rel_err

pytestmark = pytest.mark.gpu

EXPL = [0.5, 1.0, 1.0, 0.125, 0.1]


def member_specs(M):
    """four members of different sizes, depths, domains, boundaries and data (2D Euler, r = 3)"""
    T, P = pg.AW_BC_TRANSMISSIVE, pg.AW_BC_PERIODIC
    return [
        (pg.make_config(dim=2, M=M, n=(14, 14, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6,
                        auto_regrid=1), pg.AW_IC_EXPLOSION, EXPL),
        (pg.make_config(dim=2, M=M, n=(20, 12, 1), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1), bc=T, r=3, lmax=1,
                        cfl=0.5, auto_regrid=1), pg.AW_IC_RP4, aw_inputs.rp4_params(7)),
        (pg.make_config(dim=2, M=M, n=(9, 23, 1), bc=P, r=3, lmax=0, cfl=0.9),
         pg.AW_IC_FOURIER, aw_inputs.fourier_params(seed=3, dim=2, pde="euler", nmodes=3)),
        (pg.make_config(dim=2, M=M, n=(17, 17, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6,
                        auto_regrid=1), pg.AW_IC_EXPLOSION, [0.3, 2.0, 3.0, 0.2, 0.15]),
    ]


def solo(cfg, ic, p, t_end):
    s = pg.Solver(cfg)
    s.set_initial(ic, p, -1)
    st = s.advance_to(t_end)
    m, u = s.cells()
    s.close()
    return m, u, st


@pytest.mark.parametrize("M", [3, 2])
def test_batch_equals_solo_solves(M):
    t_end = 0.04
    specs = member_specs(M)
    ref = [solo(cfg, ic, p, t_end) for cfg, ic, p in specs]
    sol = []
    for cfg, ic, p in specs:
        s = pg.Solver(cfg)
        s.set_initial(ic, p, -1)
        sol.append(s)
    stats, rc = pg.advance_batch(sol, t_end)
    assert rc == [0] * len(sol)
    for s, st, (m0, u0, st0) in zip(sol, stats, ref):
        m, u = s.cells()
        assert np.array_equal(m, m0), "meshes differ"
        assert np.array_equal(u, u0), f"averages differ by {np.max(np.abs(u - u0)):.3e}"
        assert st.level0_steps == st0.level0_steps and st.cell_updates == st0.cell_updates
        assert st.t == pytest.approx(t_end, abs=0.0)
        s.close()


def test_batch_uniform_members_match_oracle():
    """uniform members of different grids against the oracle after several steps"""
    t_end = 0.05
    grids = [(13, 10), (24, 8), (16, 16)]
    sol, orc = [], []
    for k, (nx, ny) in enumerate(grids):
        kw = dict(dim=2, M=3, n=(nx, ny, 1), cfl=0.9)
        prm = aw_inputs.fourier_params(seed=10 + k, dim=2, pde="euler", nmodes=3)
        s = pg.Solver(pg.make_config(bc=pg.AW_BC_PERIODIC, **kw))
        s.set_initial(pg.AW_IC_FOURIER, prm, -1)
        o = oracle.Oracle(oracle.make_cfg(bc=oracle.BC_PERIODIC, **kw), threads=8)
        o.set_initial(oracle.IC_FOURIER, prm, nrefine=0)
        sol.append(s)
        orc.append(o)
    _, rc = pg.advance_batch(sol, t_end)
    assert rc == [0, 0, 0]
    for s, o in zip(sol, orc):
        while o.t < t_end:
            r, _ = o.step(t_end)
            assert r == 0
        mg, ug = s.cells()
        mo, uo = o.cells()
        assert np.array_equal(mg, mo)
        assert rel_err(ug, uo) <= 10 * RTOL
        s.close()


def test_batch_rejects_mismatched_members():
    a = pg.Solver(pg.make_config(dim=2, M=2, n=(8, 8, 1)))
    b = pg.Solver(pg.make_config(dim=2, M=3, n=(8, 8, 1)))
    for s in (a, b):
        s.set_initial(pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], -1)
    with pytest.raises(pg.AwError) as ei:
        pg.advance_batch([a, b], 0.01)
    assert ei.value.code == pg._lib.AW_EINVAL
    with pytest.raises(pg.AwError):
        pg.advance_batch([a, a], 0.01)
    with pytest.raises(pg.AwError):
        pg.advance_batch([a] * (pg.AW_BATCH_MAX + 1), 0.01)
    a.close()
    b.close()


def test_failing_member_stops_alone():
    """a member whose density is negative everywhere (a uniform state: the update keeps it) fails
    at its first update; the others finish and equal their solo solves"""
    t_end = 0.03
    specs = member_specs(3)[:3]
    ref = [solo(cfg, ic, p, t_end) for cfg, ic, p in specs]
    sol = []
    for cfg, ic, p in specs:
        s = pg.Solver(cfg)
        s.set_initial(ic, p, -1)
        sol.append(s)
    bad = pg.Solver(pg.make_config(dim=2, M=3, n=(8, 8, 1), bc=pg.AW_BC_PERIODIC))
    bad.set_initial(pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], -1)
    m, u = bad.cells()
    u[:, 0] = -1.0
    bad.set_cell_averages(u)
    members = sol[:1] + [bad] + sol[1:]
    with pytest.raises(pg.AwError) as ei:
        pg.advance_batch(members, t_end)
    assert ei.value.code == pg._lib.AW_ENONPHYSICAL
    for s, (m0, u0, _) in zip(sol, ref):
        m, u = s.cells()
        assert np.array_equal(m, m0) and np.array_equal(u, u0)
        s.close()
    bad.close()


def other_specs(kind):
    T, P, I = pg.AW_BC_TRANSMISSIVE, pg.AW_BC_PERIODIC, pg.AW_BC_INFLOW
    if kind == "3d":
        return [(pg.make_config(dim=3, M=2, n=(8, 8, 8), lo=(-1, -1, -1), hi=(1, 1, 1), bc=T, r=3, lmax=1, cfl=0.6,
                                auto_regrid=1), pg.AW_IC_EXPLOSION, EXPL),
                (pg.make_config(dim=3, M=2, n=(7, 6, 5), bc=P, cfl=0.9), pg.AW_IC_FOURIER,
                 aw_inputs.fourier_params(seed=8, dim=3, pde="euler", nmodes=3))]
    if kind == "mhd":
        return [(pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=3, n=(n, n, 1), lo=(0, 0, 0),
                                hi=(2 * np.pi, 2 * np.pi, 1), bc=P, r=3, lmax=lm, gamma=5 / 3, c_h=2.0, cfl=0.6,
                                auto_regrid=1), pg.AW_IC_OT, []) for n, lm in ((16, 1), (12, 0))]
    # second order, Osher flux, inflow and reflective boundaries
    qin = [2.0, 1.0, 0.0, 4.0]
    return [(pg.make_config(dim=2, M=1, n=(20, 16, 1), lo=(0, 0, 0), hi=(1, 0.8, 1),
                            bc=[I, T, pg.AW_BC_REFLECTIVE, T, T, T], r=3, lmax=2, cfl=0.6, flux=pg.AW_FLUX_OSHER,
                            auto_regrid=1, inflow=qin), pg.AW_IC_CONST, [1.0, 0.0, 0.0, 1.0]),
            (pg.make_config(dim=2, M=1, n=(14, 14, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T, r=3, lmax=1, cfl=0.6,
                            flux=pg.AW_FLUX_OSHER, auto_regrid=1), pg.AW_IC_EXPLOSION, EXPL)]


@pytest.mark.parametrize("kind", ["3d", "mhd", "m1_osher_inflow"])
def test_batch_other_configurations(kind):
    t_end = 0.02
    specs = other_specs(kind)
    ref = [solo(cfg, ic, p, t_end) for cfg, ic, p in specs]
    sol = []
    for cfg, ic, p in specs:
        s = pg.Solver(cfg)
        s.set_initial(ic, p, -1)
        sol.append(s)
    stats, rc = pg.advance_batch(sol, t_end)
    assert rc == [0] * len(sol)
    for s, st, (m0, u0, st0) in zip(sol, stats, ref):
        m, u = s.cells()
        assert np.array_equal(m, m0) and np.array_equal(u, u0)
        assert st.cell_updates == st0.cell_updates
        s.close()


@pytest.mark.parametrize("M", [3, 2])
def test_persistent_level_kernel_equals_separate_launches(M):
    """aw_set_launch_params.persistent: one cooperative launch per level and sub-step for the
    projection, WENO and predictor of every member (with the fused face flux and update on a level
    where no member has a finer one) gives bitwise the averages of the separate launches, with
    fewer launches; members of different depths, WENO tiles and passes"""
    t_end = 0.03
    specs = member_specs(M)
    specs.append((pg.make_config(dim=2, M=M, n=(70, 64, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=pg.AW_BC_TRANSMISSIVE,
                                 r=3, lmax=1, cfl=0.6), pg.AW_IC_EXPLOSION, EXPL))   # level 0 by passes
    out, launches = {}, {}
    saved = pg.get_launch_params()
    try:
        for persistent in (1, 0):
            pg.set_launch_params(persistent=persistent)
            sol = []
            for cfg, ic, p in specs:
                s = pg.Solver(cfg)
                s.set_initial(ic, p, -1)
                sol.append(s)
            n0 = sum(s.kernel_launches() for s in sol)
            _, rc = pg.advance_batch(sol, t_end)
            assert rc == [0] * len(sol)
            launches[persistent] = sum(s.kernel_launches() for s in sol) - n0
            out[persistent] = [s.cells() for s in sol]
            for s in sol:
                s.close()
    finally:
        pg.set_launch_params(**saved)
    for (m1, u1), (m0, u0) in zip(out[1], out[0]):
        assert np.array_equal(m1, m0)
        assert np.array_equal(u1, u0), f"differ by {np.max(np.abs(u1 - u0)):.3e}"
    assert launches[1] < launches[0], launches
