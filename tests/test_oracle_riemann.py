"""Pins of the oracle's shocked flows against an exact solution: Sod's shock tube (left state
rho = 1, p = 1; right state rho = 0.125, p = 0.1; at rest, gamma = 1.4) set up as a planar
four-quadrant problem on a 2D strip, with the exact Riemann solution (Toro's pressure iteration,
written independently in `test_oracle_radial.py`) averaged over every cell.

  * the whole 2D scheme (WENO, predictor, Rusanov and Osher fluxes) converges in L1 towards it;
  * one level of refinement with local time stepping (the Loehner indicator marks the three
    waves) lowers the error of the base grid;
  * while no wave has reached the ends, mass and energy are conserved and the x momentum grows by
    (p_left - p_right) L_y t (the two boundary faces see the constant states, up to the
    exponentially small precursor of the high-order stencils: 1e-10 relative);
  * the strip along y gives the strip along x with the axes exchanged, and every row of a strip
    stays the same up to rounding (the problem is planar).

Measured L1 density errors at t = 0.2 (Rusanov): M=2 1.03e-2, 5.56e-3, 3.07e-3 (50, 100, 200
cells); M=3 9.29e-3, 5.34e-3, 2.93e-3; one AMR level (r = 3) on 50 cells, M=3: 3.54e-3 over the
active cells; Osher, M=3, 100 cells: 3.86e-3.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_radial import exact_riemann

LEFT, RIGHT = (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1)
T_END, NY = 0.2, 4


def rp4_params(axis):
    """the RP4 parameters (x0, y0, quadrants 1..4) of Sod's problem with its jump at 1/2 along axis"""
    if axis == 0:       # quadrants 1, 4 (x > x0) right; 2, 3 left; y0 below the strip
        return [0.5, -1.0] + list(RIGHT) + list(LEFT) + list(LEFT) + list(RIGHT)
    sw = lambda s: (s[0], s[2], s[1], s[3])
    return [-1.0, 0.5] + list(sw(RIGHT)) + list(sw(RIGHT)) + list(sw(LEFT)) + list(sw(LEFT))


def exact_density_averages(xl, h, ns=400):
    """averages over [xl, xl + h] of the exact density, by the midpoint rule on ns points"""
    xs = xl[:, None] + (np.arange(ns) + 0.5) / ns * h[:, None]
    ex = exact_riemann(*LEFT[:2], LEFT[3], *RIGHT[:2], RIGHT[3], 1.4, (xs.ravel() - 0.5) / T_END)
    return ex[:, 0].reshape(xs.shape).mean(axis=1)


def run_sod(n, M, lmax=0, flux=0, axis=0):
    """Sod's problem on an n x NY strip (NY x n for axis 1); returns (meta, u, total change, L1)"""
    ext = (n, NY, 1) if axis == 0 else (NY, n, 1)
    hi = (1.0, NY / n, 1) if axis == 0 else (NY / n, 1.0, 1)
    cfg = oracle.make_cfg(dim=2, M=M, n=ext, lo=(0, 0, 0), hi=hi, bc=oracle.BC_TRANSMISSIVE, cfl=0.9,
                          lmax=lmax, r=3, flux=flux)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_RP4, rp4_params(axis))
    tot0 = o.totals()
    while o.t < T_END:
        rc, _ = o.step(T_END)
        assert rc == 0
    assert o.t == T_END
    meta, u = o.cells()
    act = meta[:, 1] == 0                       # meta = (level, status, i, j, k); status 0 = active
    h = (1.0 / n) / 3.0 ** meta[act, 0]
    err = np.abs(u[act, 0] - exact_density_averages(meta[act, 2 + axis] * h, h))
    l1 = np.sum(err * h * h) / (NY / n)         # per unit length of the strip
    return meta, u, o.totals() - tot0, l1


@pytest.mark.parametrize("M", [2, 3])
def test_sod_converges_to_exact_solution(M):
    """error ratio about 0.55 per halving of h; a scheme converging to another solution (energy
    flux v (E + 0.9 p), say) saturates: 0.81 from 100 to 200 cells"""
    e = [run_sod(n, M)[3] for n in (50, 100, 200)]
    assert e[2] < 3.4e-3 and e[1] < 0.65 * e[0] and e[2] < 0.65 * e[1], e


@pytest.mark.parametrize("M", [2, 3])
def test_sod_boundary_fluxes_and_conservation(M):
    n = 50
    meta, u, dtot, _ = run_sod(n, M)
    Ly = NY / n
    assert dtot[1] == pytest.approx((LEFT[3] - RIGHT[3]) * Ly * T_END, rel=1e-9, abs=0)
    assert abs(dtot[0]) < 1e-12 and abs(dtot[2]) < 1e-14 and abs(dtot[3]) < 1e-11
    rows = u.reshape(NY, n, 4)
    assert np.max(np.abs(rows - rows[0])) < 1e-12 * np.max(np.abs(u))   # rounding only
    assert np.max(np.abs(u[:, 2])) < 1e-12         # no transverse momentum appears


def test_sod_amr_with_local_time_stepping_beats_its_base_grid():
    meta, u, dtot, l1_amr = run_sod(50, 3, lmax=1)
    assert np.count_nonzero(meta[:, 0] == 1) > 0
    l1_base = run_sod(50, 3)[3]
    assert l1_amr < 0.5 * l1_base, (l1_amr, l1_base)
    assert l1_amr < 3.9e-3
    assert dtot[1] == pytest.approx((LEFT[3] - RIGHT[3]) * NY / 50 * T_END, rel=1e-9, abs=0)
    assert abs(dtot[0]) < 1e-13 and abs(dtot[3]) < 1e-12


def test_sod_osher_converges_and_is_less_dissipative():
    e_osher = [run_sod(n, 3, flux=1)[3] for n in (50, 100)]
    e_rus = run_sod(100, 3)[3]
    assert e_osher[1] < 0.65 * e_osher[0], e_osher
    assert e_osher[1] < 0.85 * e_rus, (e_osher, e_rus)


def test_sod_along_y_equals_sod_along_x():
    n = 50
    _, ux, _, lx = run_sod(n, 3)
    _, uy, _, ly = run_sod(n, 3, axis=1)
    ux = ux.reshape(NY, n, 4)
    uy = uy.reshape(n, NY, 4).transpose(1, 0, 2)[..., [0, 2, 1, 3]]
    assert np.max(np.abs(ux - uy)) < 1e-12
    assert abs(lx - ly) < 1e-12
