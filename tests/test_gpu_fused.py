"""The fused face flux and update (one launch of k_flux_update per level and sub-step: the face
integrals of Eqs. eqn.rusanov / eqn.osher with the memory variables of Eq. eqn.memory.sum, then
the one-step update of Eq. eq:finite_vol) against the two-kernel path (k_flux, then k_update).

The two must give bitwise the same meshes and cell averages over whole solves: uniform periodic
grids (whose wrap-around high faces the fused kernel takes from the high side), AMR with local
time stepping in 2D and 3D (coarse and fine sides of the interfaces), reflective and inflow walls,
the Osher flux, MHD-GLM, and the batched and graph paths."""
import numpy as np
import pytest

import aw_inputs
import paper_1212_3585_gb300 as pg

pytestmark = pytest.mark.gpu

EXPL = [0.5, 1.0, 1.0, 0.125, 0.1]
VORTEX = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]
T, P, R, I = pg.AW_BC_TRANSMISSIVE, pg.AW_BC_PERIODIC, pg.AW_BC_REFLECTIVE, pg.AW_BC_INFLOW


def cases():
    return {
        "vortex 32^2 M=2 periodic": (pg.make_config(dim=2, M=2, n=(32, 32, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc=P,
                                                    cfl=0.9), pg.AW_IC_VORTEX, VORTEX, 0.5),
        "explosion 2D M=3 r=3 l_max=2": (pg.make_config(dim=2, M=3, n=(14, 14, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T,
                                                        r=3, lmax=2, cfl=0.6), pg.AW_IC_EXPLOSION, EXPL, 0.05),
        "explosion 2D M=2 r=2 l_max=3 periodic": (pg.make_config(dim=2, M=2, n=(12, 10, 1), lo=(-1, -1, 0),
                                                                 hi=(1, 1, 1), bc=P, r=2, lmax=3, cfl=0.6),
                                                  pg.AW_IC_EXPLOSION, EXPL, 0.12),
        "explosion 3D M=2 r=3 l_max=2": (pg.make_config(dim=3, M=2, n=(5, 5, 5), lo=(-1, -1, -1), hi=(1, 1, 1), bc=T,
                                                        r=3, lmax=2, cfl=0.6), pg.AW_IC_EXPLOSION, EXPL, 0.15),
        "fourier 3D M=2 periodic": (pg.make_config(dim=3, M=2, n=(9, 7, 6), bc=P, cfl=0.9), pg.AW_IC_FOURIER,
                                    aw_inputs.fourier_params(seed=4, dim=3, pde="euler", nmodes=3), 0.1),
        "reflective + inflow, Osher": (pg.make_config(dim=2, M=3, n=(16, 12, 1), lo=(-1, -1, 0), hi=(1, 1, 1),
                                                      bc=[I, T, R, R, P, P], r=3, lmax=1, cfl=0.6,
                                                      flux=pg.AW_FLUX_OSHER, inflow=[1.2, 0.3, 0.0, 2.0]),
                                       pg.AW_IC_EXPLOSION, EXPL, 0.08),
        "MHD-GLM Orszag-Tang r=3 l_max=1": (pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=3, n=(16, 16, 1),
                                                           lo=(0, 0, 0), hi=(2 * np.pi, 2 * np.pi, 1), bc=P,
                                                           gamma=5.0 / 3.0, r=3, lmax=1, cfl=0.6, c_h=2.0),
                                            pg.AW_IC_OT, [], 0.15),
        "MHD-GLM Orszag-Tang Osher": (pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=2, n=(12, 12, 1), lo=(0, 0, 0),
                                                     hi=(2 * np.pi, 2 * np.pi, 1), bc=P, gamma=5.0 / 3.0, r=3, lmax=1,
                                                     cfl=0.6, c_h=2.0, flux=pg.AW_FLUX_OSHER),
                                      pg.AW_IC_OT, [], 0.15),
        "linear advection M=1": (pg.make_config(dim=2, pde=pg.AW_PDE_LINADV, M=1, n=(19, 13, 1), bc=P, cfl=0.9),
                                 pg.AW_IC_FOURIER, aw_inputs.fourier_params(seed=5, dim=2, pde="linadv", nmodes=3),
                                 0.3),
    }


def solve(cfg, ic, params, t_end, fused, path="host"):
    saved = pg.get_launch_params()
    pg.set_launch_params(fuse_flux_update=fused)
    try:
        s = pg.Solver(cfg)
        s.set_initial(ic, params, -1)
        if path == "graph":
            st = s.advance_graph(t_end, 8)
        else:
            st = s.advance_to(t_end)
        m, u = s.cells()
        s.close()
    finally:
        pg.set_launch_params(**saved)
    return m, u, st


@pytest.mark.parametrize("name", list(cases()))
def test_fused_equals_two_kernels(name):
    cfg, ic, params, t_end = cases()[name]
    m1, u1, s1 = solve(cfg, ic, params, t_end, 1)
    m0, u0, s0 = solve(cfg, ic, params, t_end, 0)
    assert s1.level0_steps == s0.level0_steps and s1.level0_steps >= 2
    assert np.array_equal(m1, m0), "meshes differ"
    assert np.array_equal(u1, u0), f"{name}: averages differ by {np.max(np.abs(u1 - u0)):.3e}"


@pytest.mark.parametrize("name", ["vortex 32^2 M=2 periodic", "fourier 3D M=2 periodic"])
def test_fused_graph_path(name):
    cfg, ic, params, t_end = cases()[name]
    m1, u1, _ = solve(cfg, ic, params, t_end, 1, path="graph")
    m0, u0, _ = solve(cfg, ic, params, t_end, 0, path="host")
    assert np.array_equal(m1, m0)
    assert np.array_equal(u1, u0)


def test_fused_batch_path():
    specs = [cases()[k] for k in ("explosion 2D M=3 r=3 l_max=2",)]
    cfg, ic, params, t_end = specs[0]
    cfg2 = pg.make_config(dim=2, M=3, n=(20, 12, 1), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1), bc=T, r=3, lmax=1,
                          cfl=0.5)
    members = [(cfg, ic, params), (cfg2, pg.AW_IC_RP4, aw_inputs.rp4_params(7))]
    out = {}
    saved = pg.get_launch_params()
    try:
        for fused in (1, 0):
            pg.set_launch_params(fuse_flux_update=fused)
            sol = []
            for c, i, p in members:
                s = pg.Solver(c)
                s.set_initial(i, p, -1)
                sol.append(s)
            _, rc = pg.advance_batch(sol, t_end)
            assert rc == [0, 0]
            out[fused] = [s.cells() for s in sol]
            for s in sol:
                s.close()
    finally:
        pg.set_launch_params(**saved)
    for (m1, u1), (m0, u0) in zip(out[1], out[0]):
        assert np.array_equal(m1, m0)
        assert np.array_equal(u1, u0)


def test_fused_launch_list():
    """the fused path launches no update kernel: one flux-and-update launch per level and sub-step"""
    cfg, ic, params, t_end = cases()["vortex 32^2 M=2 periodic"]
    counts = {}
    saved = pg.get_launch_params()
    try:
        for fused in (1, 0):
            pg.set_launch_params(fuse_flux_update=fused)
            s = pg.Solver(cfg)
            s.set_initial(ic, params, -1)
            n0 = s.kernel_launches()
            st = s.step()
            counts[fused] = (s.kernel_launches() - n0, st.level0_steps)
            s.close()
    finally:
        pg.set_launch_params(**saved)
    assert counts[1][1] == counts[0][1] == 1
    assert counts[0][0] - counts[1][0] == 1
