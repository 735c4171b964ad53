"""Pins of the oracle's level-0 time step (reading R11 of the CFL condition, which the paper does
not state): dt_0 = min over active cells of r^l * CFL / sum_d (s_d / dx_d), with s_d the largest
|eigenvalue| of the flux Jacobian along axis d (Euler |v_d| + c; MHD-GLM the fast speed, at least
c_h; linear advection |a_d|) from the cell average.

Every expected value is a literal worked out by hand from the state, the grid and the CFL number
(the arithmetic is written beside it), on grids with unequal spacings and states with unequal
speeds per axis, so that the sum over axes cannot pass for the largest term
(CFL / max_d(s_d / dx_d)) or for CFL * min_d dx_d / max_d s_d, and the minimum over cells
cannot pass for the value of one cell.
"""
import numpy as np
import pytest

import oracle


def _euler2d(n=(10, 20, 1), lmax=0, r=3, cfl=0.9):
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_EULER, M=2, n=n, lo=(0, 0, 0), hi=(2, 1, 1),
                          bc=oracle.BC_PERIODIC, lmax=lmax, r=r, cfl=cfl, auto_regrid=0)
    return oracle.Oracle(cfg)


def test_dt_euler_2d_constant_state():
    # rho = 1, (u, v) = (0.5, -1), p = 1, gamma = 1.4 on [0,2]x[0,1] with 10 x 20 cells:
    # dx = 0.2, dy = 0.05, c = sqrt(1.4) = 1.1832159566199232
    # s_x = 1.6832159566199232, s_y = 2.1832159566199232
    # sum = 8.416079783099616 + 43.664319132398464 = 52.08039891549808
    # dt = 0.9 / 52.08039891549808 = 0.0172809736242665
    # (the largest term alone would give 0.02061179511974136)
    o = _euler2d()
    o.set_initial(oracle.IC_CONST, [1.0, 0.5, -1.0, 1.0], nrefine=0)
    assert o.compute_dt() == pytest.approx(0.0172809736242665, rel=1e-13)


def test_dt_euler_2d_scales_with_cfl_and_takes_the_slowest_cell():
    o = _euler2d(cfl=0.45)
    o.set_initial(oracle.IC_CONST, [1.0, 0.5, -1.0, 1.0], nrefine=0)
    assert o.compute_dt() == pytest.approx(0.5 * 0.0172809736242665, rel=1e-13)
    # one cell at rest with p = 1 has s_x = s_y = c and a larger dt; one cell moving at
    # (u, v) = (3, 0) with rho = 1, p = 1 has s_x = 3 + c = 4.183215956619923, s_y = c:
    # sum = 20.916079783099616 + 23.664319132398464 = 44.58039891549808, dt = 0.45 / that
    # = 0.010094122326114: its sum 44.58 is below the other cells' 52.08, so the minimum stays
    # 0.45 / 52.08...
    meta, u = o.cells()
    E_rest = 1.0 / 0.4
    u[3] = [1.0, 0.0, 0.0, E_rest]
    u[7] = [1.0, 3.0, 0.0, E_rest + 4.5]
    o.set_cell_averages(u)
    assert o.compute_dt() == pytest.approx(0.5 * 0.0172809736242665, rel=1e-13)
    # ... until the fast cell moves along y as well, (u, v) = (3, -2):
    # s_y = 2 + c = 3.183215956619923, sum = 20.916079783099616 + 63.66431913239846
    # = 84.58039891549808, dt = 0.45 / 84.58039891549808 = 0.005320381622338
    u[7] = [1.0, 3.0, -2.0, E_rest + 6.5]
    o.set_cell_averages(u)
    assert o.compute_dt() == pytest.approx(0.005320381622337611, rel=1e-13)


def test_dt_euler_3d_constant_state():
    # rho = 2, (u, v, w) = (0.3, -0.2, 1.5), p = 0.8 on [0,2]x[0,1]x[0,3] with 10 x 20 x 5 cells:
    # dx = 0.2, dy = 0.05, dz = 0.6, c = sqrt(1.4 * 0.8 / 2) = sqrt(0.56) = 0.7483314773547883
    # s = (1.0483314773547883, 0.9483314773547883, 2.2483314773547883)
    # sum = 5.241657386773941 + 18.966629547095766 + 3.7472191289246473 = 27.955506062794356
    # dt = 0.6 / 27.955506062794356 = 0.021462677107410077
    cfg = oracle.make_cfg(dim=3, pde=oracle.PDE_EULER, M=2, n=(10, 20, 5), lo=(0, 0, 0), hi=(2, 1, 3),
                          bc=oracle.BC_PERIODIC, cfl=0.6, auto_regrid=0)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [2.0, 0.3, -0.2, 1.5, 0.8], nrefine=0)
    assert o.compute_dt() == pytest.approx(0.021462677107410077, rel=1e-13)


@pytest.mark.parametrize("c_h,expected", [
    # rho = 1, v = 0, p = 0.6, gamma = 5/3: a^2 = 1; B = (0.5, 0, 0): b^2 = 0.25
    # along x (B_n = B): c_f^2 = (1.25 + sqrt(1.25^2 - 4 * 0.25)) / 2 = (1.25 + 0.75) / 2 = 1
    # along y (B_n = 0): c_f^2 = (1.25 + 1.25) / 2 = 1.25, c_f = 1.118033988749895
    # c_h = 0.5 (below both): dt = 0.9 / (1 / 0.2 + 1.118033988749895 / 0.05)
    #                            = 0.9 / (5 + 22.3606797749979) = 0.03289391957368022
    (0.5, 0.03289391957368022),
    # c_h = 2 (above both): dt = 0.9 / (2 / 0.2 + 2 / 0.05) = 0.9 / 50 = 0.018
    (2.0, 0.018),
])
def test_dt_mhd_glm_fast_speed_and_cleaning_speed(c_h, expected):
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, M=2, n=(10, 20, 1), lo=(0, 0, 0), hi=(2, 1, 1),
                          bc=oracle.BC_PERIODIC, gamma=5.0 / 3.0, c_h=c_h, cfl=0.9, auto_regrid=0)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [1.0, 0.0, 0.0, 0.0, 0.6, 0.5, 0.0, 0.0, 0.0], nrefine=0)
    assert o.compute_dt() == pytest.approx(expected, rel=1e-13)


def test_dt_linear_advection():
    # a = (1, -0.5): dt = 0.9 / (1 / 0.2 + 0.5 / 0.05) = 0.9 / 15 = 0.06
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_LINADV, M=2, n=(10, 20, 1), lo=(0, 0, 0), hi=(2, 1, 1),
                          bc=oracle.BC_PERIODIC, adv=(1.0, -0.5, 0.0), cfl=0.9, auto_regrid=0)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [1.0], nrefine=0)
    assert o.compute_dt() == pytest.approx(0.06, rel=1e-13)


def test_dt_refined_cells_carry_the_factor_r():
    """a fast state only on the active cells of level 1 (r = 3): their own step is
    CFL / sum_d(s_d / dx_{d,1}) = CFL / (3 sum_d(s_d / dx_{d,0})), and local time stepping makes
    dt_0 = 3 times that, the value a level-0 cell with that state would have"""
    o = _euler2d(n=(10, 20, 1), lmax=1, r=3)
    o.set_initial(oracle.IC_CONST, [1.0, 0.5, -1.0, 1.0], nrefine=0)
    meta, _ = o.cells()
    flags = np.zeros(len(meta), dtype=np.int8)
    flags[(meta[:, 2] >= 3) & (meta[:, 2] < 6) & (meta[:, 3] >= 8) & (meta[:, 3] < 12)] = 1
    o.regrid_with_flags(flags, init_mode=0)
    meta, u = o.cells()
    assert np.any(meta[:, 0] == 1)
    # level 1 active cells moving at (u, v) = (1, -3), rho = 1, p = 1, E = 2.5 + 5:
    # s_x = 1 + c = 2.183215956619923, s_y = 3 + c = 4.183215956619923
    # on level 0 spacings: sum = 10.916079783099616 + 83.66431913239846 = 94.58039891549808
    # dt_0 = 0.9 / 94.58039891549808 = 0.009515713724195
    fast = (meta[:, 0] == 1) & (meta[:, 1] == 0)
    u[fast] = [1.0, 1.0, -3.0, 2.5 + 5.0]
    o.set_cell_averages(u)
    assert o.compute_dt() == pytest.approx(0.009515713724194547, rel=1e-13)
