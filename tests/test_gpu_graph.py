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
