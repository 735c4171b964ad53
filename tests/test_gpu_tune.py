"""The launch-shape autotuner (aw_set_launch_params.autotune, aw_get_tuning): the predictor's and
the face flux's full- and quarter-size CTAs compute bitwise the same averages, so the tuner may
pick either per level size class; a solve with the tuner on equals the same solve with it off,
and the tuner decides every class it has timed often enough."""
import numpy as np
import pytest

import aw_inputs
import paper_1212_3585_gb300 as pg

pytestmark = pytest.mark.gpu

EXPL = [0.5, 1.0, 1.0, 0.125, 0.1]


def configs():
    T = pg.AW_BC_TRANSMISSIVE
    return [
        (pg.make_config(dim=2, M=3, n=(40, 40, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6),
         pg.AW_IC_EXPLOSION, EXPL, 0.06),
        (pg.make_config(dim=3, M=2, n=(8, 8, 8), lo=(-1, -1, -1), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6),
         pg.AW_IC_EXPLOSION, EXPL, 0.12),
        (pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=3, n=(24, 24, 1), lo=(0, 0, 0), hi=(2 * np.pi, 2 * np.pi, 1),
                        bc=pg.AW_BC_PERIODIC, gamma=5.0 / 3.0, r=3, lmax=1, cfl=0.6, c_h=2.0, chi_ref=0.05,
                        chi_rec=0.02), pg.AW_IC_OT, [], 0.1),
    ]


def solve(cfg, ic, params, t_end, **launch):
    saved = pg.get_launch_params()
    pg.set_launch_params(**launch)
    try:
        s = pg.Solver(cfg)
        s.set_initial(ic, params, -1)
        st = s.advance_to(t_end)
        m, u = s.cells()
        s.close()
    finally:
        pg.set_launch_params(**saved)
    return m, u, st


@pytest.mark.parametrize("k", range(3))
def test_full_and_quarter_size_ctas_agree_bitwise(k):
    cfg, ic, params, t_end = configs()[k]
    m1, u1, s1 = solve(cfg, ic, params, t_end, autotune=0, small_ctas_per_sm=0)    # always full size
    m4, u4, s4 = solve(cfg, ic, params, t_end, autotune=0, small_ctas_per_sm=64)   # always quarter size
    assert s1.level0_steps == s4.level0_steps >= 2
    assert np.array_equal(m1, m4)
    assert np.array_equal(u1, u4)


def test_autotuner_decides_and_leaves_results_unchanged():
    pg.reset_tuning()
    cfg, ic, params, t_end = configs()[0]
    m0, u0, _ = solve(cfg, ic, params, t_end, autotune=0)
    m1, u1, _ = solve(cfg, ic, params, t_end, autotune=1)
    assert np.array_equal(m0, m1) and np.array_equal(u0, u1)
    tun = pg.get_tuning()
    kernels = {e["kernel"] for e in tun}
    assert kernels == {pg._lib.AW_TUNE_PREDICTOR, pg._lib.AW_TUNE_FLUX}
    for e in tun:
        assert (e["dim"], e["M"], e["pde"]) == (2, 3, pg.AW_PDE_EULER)
        if e["choice"] >= 0 and not e["inherited"]:
            assert min(e["trials"]) >= pg._lib.AW_TUNE_TRIALS
            assert e["ns_per_cell"][e["choice"]] <= e["ns_per_cell"][1 - e["choice"]]
            assert min(e["ns_per_cell"]) > 0
    timed = [e for e in tun if e["choice"] >= 0 and not e["inherited"]]
    assert {e["kernel"] for e in timed} == kernels
    # an inherited decision follows a timed one of the same kernel: full size above a class that
    # kept full size, quarter size below one that kept quarter size
    for e in tun:
        if e["inherited"]:
            same = [f for f in timed if f["kernel"] == e["kernel"]]
            assert any((f["size_class"] < e["size_class"] and f["choice"] == e["choice"] == 0) or
                       (f["size_class"] > e["size_class"] and f["choice"] == e["choice"] == 1) for f in same)
    # a second solve runs on the decisions, with the same result
    m2, u2, _ = solve(cfg, ic, params, t_end, autotune=1)
    assert np.array_equal(m0, m2) and np.array_equal(u0, u2)
    pg.reset_tuning()
    assert pg.get_tuning() == []
