"""aw_advance_graph: uniform meshes advanced with the time step computed on the device and the
level-0 steps replayed from a CUDA graph.  It must compute exactly what aw_advance_to computes
(bitwise: the same kernels and the same time steps), for any chunk size, and report the same
errors."""
import numpy as np
import pytest

import aw_inputs
import paper_1212_3585_gb300 as pg

pytestmark = pytest.mark.gpu

VORTEX = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]


def cases():
    P = pg.AW_BC_PERIODIC
    return [
        ("vortex 32^2 M=2", pg.make_config(dim=2, M=2, n=(32, 32, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc=P, cfl=0.9),
         pg.AW_IC_VORTEX, VORTEX, 0.7),
        ("euler 3D M=2", pg.make_config(dim=3, M=2, n=(9, 7, 6), bc=P, cfl=0.9), pg.AW_IC_FOURIER,
         aw_inputs.fourier_params(seed=4, dim=3, pde="euler", nmodes=3), 0.05),
        ("linadv M=1", pg.make_config(dim=2, pde=pg.AW_PDE_LINADV, M=1, n=(19, 13, 1), bc=P, cfl=0.9),
         pg.AW_IC_FOURIER, aw_inputs.fourier_params(seed=5, dim=2, pde="linadv", nmodes=3), 0.3),
        ("explosion M=3 transmissive", pg.make_config(dim=2, M=3, n=(24, 24, 1), lo=(-1, -1, 0), hi=(1, 1, 1),
                                                      bc=pg.AW_BC_TRANSMISSIVE, cfl=0.6),
         pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, 0.1),
    ]


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("chunk", [1, 7, 64])
def test_graph_path_equals_host_path(k, chunk):
    name, cfg, ic, params, t_end = cases()[k]
    a = pg.Solver(cfg)
    a.set_initial(ic, params, -1)
    sa = a.advance_to(t_end)
    b = pg.Solver(cfg)
    b.set_initial(ic, params, -1)
    sb = b.advance_graph(t_end, chunk)
    ma, ua = a.cells()
    mb, ub = b.cells()
    assert np.array_equal(ma, mb)
    assert np.array_equal(ua, ub), f"{name}: differs by {np.max(np.abs(ua - ub)):.3e}"
    assert (sa.level0_steps, sa.cell_updates, sa.t) == (sb.level0_steps, sb.cell_updates, sb.t)
    assert sb.last_dt0 == sa.last_dt0
    # continuing from an intermediate time, and nothing to do once t_end is reached
    sc = b.advance_graph(t_end, chunk)
    assert sc.level0_steps == 0 and b.t == t_end
    a.close()
    b.close()


def test_graph_path_errors():
    with pytest.raises(pg.AwError) as ei:
        s = pg.Solver(pg.make_config(dim=2, M=2, n=(8, 8, 1), lmax=1, r=3))
        s.set_initial(pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], -1)
        s.advance_graph(0.1, 4)
    assert ei.value.code == pg._lib.AW_EINVAL
    res = []
    for path in ("host", "graph"):
        s = pg.Solver(pg.make_config(dim=2, M=2, n=(8, 8, 1), bc=pg.AW_BC_PERIODIC))
        s.set_initial(pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], -1)
        m, u = s.cells()
        u[:, 0] = -1.0
        s.set_cell_averages(u)
        with pytest.raises(pg.AwError) as ei:
            s.advance_to(1.0) if path == "host" else s.advance_graph(1.0, 8)
        assert ei.value.code == pg._lib.AW_ENONPHYSICAL
        res.append((s.t, s.cells()[1]))
        s.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1], equal_nan=True)


def amr_cases():
    T = pg.AW_BC_TRANSMISSIVE
    return [
        (pg.make_config(dim=2, M=3, n=(24, 24, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6),
         pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, 0.08),
        (pg.make_config(dim=3, M=2, n=(6, 6, 6), lo=(-1, -1, -1), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6),
         pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, 0.3),
        (pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=2, n=(12, 12, 1), lo=(0, 0, 0), hi=(2 * np.pi, 2 * np.pi, 1),
                        bc=pg.AW_BC_PERIODIC, gamma=5.0 / 3.0, r=3, lmax=1, cfl=0.6, c_h=2.0, flux=pg.AW_FLUX_OSHER),
         pg.AW_IC_OT, [], 0.3),
    ]


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("prof", [0, 1])
def test_amr_steps_replayed_from_graphs(k, prof):
    """graph_steps = 1: every level-0 step of an AMR solve (all levels and sub-steps with local
    time stepping, the regrid between steps) runs from a captured graph.  The solve is bitwise the
    one launched kernel by kernel.  Without timing events (tuner off, no profiling) the steps after
    the first update the executable graph in place or relaunch it; with profiling and the
    autotuner's timed trials, their events are captured as event-record nodes that record when
    the graph runs, and such graphs are never relaunched unchanged."""
    cfg, ic, params, t_end = amr_cases()[k]
    out = {}
    saved = pg.get_launch_params()
    try:
        for g in (1, 0):
            pg.set_launch_params(graph_steps=g, autotune=prof)
            s = pg.Solver(cfg)
            s.set_profiling(bool(prof))
            s.set_initial(ic, params, -1)
            st = s.advance_to(t_end)
            out[g] = (s.cells(), st.level0_steps, s.graph_stats(), s.kernel_times() if prof else None)
            s.close()
    finally:
        pg.set_launch_params(**saved)
    (m1, u1), n1, (reuse, upd, inst), kt1 = out[1]
    (m0, u0), n0, stats0, kt0 = out[0]
    assert n1 == n0 >= 3, (n1, n0)
    assert np.array_equal(m1, m0), "meshes differ"
    assert np.array_equal(u1, u0), f"averages differ by {np.max(np.abs(u1 - u0)):.3e}"
    assert stats0 == (0, 0, 0)
    assert reuse + upd + inst == n1 and inst >= 1, (reuse, upd, inst, n1)
    if not prof:
        assert reuse + upd >= 1, (reuse, upd, inst, n1)
    if prof:
        assert reuse == 0                    # a graph with timing events is captured anew each step
        # the timing events of the captured launches record when the graph runs
        ms1, n_1 = kt1
        ms0, n_0 = kt0
        assert list(n_1) == list(n_0)
        assert all(t > 0 for t, c in zip(ms1, n_1) if c > 0)


def test_batched_amr_steps_replayed_from_graphs():
    """graph_steps = 1 in aw_advance_batch (on the legacy default stream, which cannot be captured:
    the capture runs on the first member's own stream): bitwise the directly launched batch, and
    with the persistent level kernel requested the captured steps fall back to separate launches"""
    specs = [amr_cases()[0][:3],
             (pg.make_config(dim=2, M=3, n=(16, 20, 1), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1),
                             bc=pg.AW_BC_TRANSMISSIVE, r=3, lmax=1, cfl=0.5), pg.AW_IC_RP4, aw_inputs.rp4_params(3))]
    out = {}
    saved = pg.get_launch_params()
    try:
        for g, pers in ((1, 0), (1, 1), (0, 0)):
            pg.set_launch_params(graph_steps=g, persistent=pers)
            sol = []
            for cfg, ic, p in specs:
                s = pg.Solver(cfg)
                s.set_initial(ic, p, -1)
                sol.append(s)
            st, rc = pg.advance_batch(sol, 0.08)
            assert rc == [0, 0]
            out[(g, pers)] = ([s.cells() for s in sol], sol[0].graph_stats(), max(x.level0_steps for x in st))
            for s in sol:
                s.close()
    finally:
        pg.set_launch_params(**saved)
    ref = out[(0, 0)]
    assert ref[1] == (0, 0, 0) and ref[2] >= 3, ref[1:]
    for key in ((1, 0), (1, 1)):
        for (m1, u1), (m0, u0) in zip(out[key][0], ref[0]):
            assert np.array_equal(m1, m0) and np.array_equal(u1, u0)
        reuse, upd, inst = out[key][1]
        assert inst >= 1 and reuse + upd + inst == out[key][2], (key, out[key][1], out[key][2])


def test_unchanged_mesh_relaunches_the_step_graph():
    """a mesh that the regrids leave as it is (a constant state refines nowhere): after the first
    captured step every level-0 step launches the same graph again, without a capture, and the
    solve is bitwise the directly launched one"""
    cfg = pg.make_config(dim=2, M=3, n=(20, 16, 1), bc=pg.AW_BC_PERIODIC, r=3, lmax=1, cfl=0.9)
    out = {}
    saved = pg.get_launch_params()
    try:
        for g in (1, 0):
            pg.set_launch_params(graph_steps=g, autotune=0)
            s = pg.Solver(cfg)
            s.set_initial(pg.AW_IC_CONST, [1.0, 0.3, -0.2, 1.0], -1)
            n_before = s.kernel_launches()
            st = s.advance_to(0.2)
            out[g] = (s.cells(), st.level0_steps, s.graph_stats(), s.kernel_launches() - n_before)
            s.close()
    finally:
        pg.set_launch_params(**saved)
    (m1, u1), n1, (reuse, upd, inst), l1 = out[1]
    (m0, u0), n0, _, l0 = out[0]
    assert n1 == n0 >= 4
    assert np.array_equal(m1, m0) and np.array_equal(u1, u0)
    assert (reuse, upd, inst) == (n1 - 1, 0, 1)
    assert l1 == l0                          # the relaunched graphs count their kernels
