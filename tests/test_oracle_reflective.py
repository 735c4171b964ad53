"""Pin of the reflecting walls: the centred explosion on the quadrant [0,1]^2 with walls on x = 0
and y = 0 equals the full-domain solution on [-1,1]^2 restricted to that quadrant (mirror
symmetry), cell by cell, with and without AMR, and likewise the octant of the 3D explosion; a
closed box conserves every total."""
import numpy as np
import pytest

import oracle

EXPL = [0.5, 1.0, 1.0, 0.125, 0.1]
R, T = oracle.BC_REFLECTIVE, oracle.BC_TRANSMISSIVE


@pytest.mark.parametrize("M,lmax,flux", [(3, 0, 0), (2, 1, 0), (3, 1, 1)])
def test_quadrant_with_walls_equals_full_domain(M, lmax, flux):
    n = 10
    full = oracle.Oracle(oracle.make_cfg(dim=2, M=M, n=(2 * n, 2 * n, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=T, r=3,
                                         lmax=lmax, cfl=0.6, flux=flux), threads=8)
    quad = oracle.Oracle(oracle.make_cfg(dim=2, M=M, n=(n, n, 1), lo=(0, 0, 0), hi=(1, 1, 1), bc=[R, T, R, T, T, T],
                                         r=3, lmax=lmax, cfl=0.6, flux=flux), threads=8)
    full.set_initial(oracle.IC_EXPLOSION, EXPL)
    quad.set_initial(oracle.IC_EXPLOSION, EXPL)
    for _ in range(3):
        dt = full.compute_dt()
        assert quad.compute_dt() == pytest.approx(dt, rel=1e-14)
        full.advance_dt(dt)
        quad.advance_dt(dt)
        if lmax:
            full.regrid()
            quad.regrid()
    mf, uf = full.cells()
    mq, uq = quad.cells()
    lookup = {(lv, i, j): (st, u) for (lv, st, i, j, _), u in zip(mf, uf)}
    for (lv, st, i, j, _), u in zip(mq, uq):
        off = n * 3 ** lv
        st2, u2 = lookup[(lv, i + off, j + off)]
        assert st2 == st
        if st <= 0:
            assert np.allclose(u, u2, rtol=0, atol=1e-12), (lv, i, j, u, u2)


def test_closed_box_conserves_totals():
    o = oracle.Oracle(oracle.make_cfg(dim=2, M=3, n=(12, 12, 1), lo=(-1, -1, 0), hi=(1, 1, 1), bc=R, r=3, lmax=1,
                                      cfl=0.6), threads=8)
    o.set_initial(oracle.IC_EXPLOSION, [0.5, 1.0, 1.0, 0.125, 0.1])
    t0 = o.totals()
    while o.t < 0.6:          # long enough for the shock to hit the walls
        rc, _ = o.step(0.6)
        assert rc == 0
    t1 = o.totals()
    assert abs(t1[0] - t0[0]) < 1e-13 * t0[0] and abs(t1[3] - t0[3]) < 1e-13 * t0[3]


def test_octant_with_walls_equals_full_domain_3d():
    """the spherical explosion on the octant [0,1]^3 with walls on x = 0, y = 0 and z = 0 equals
    the full-domain solution on [-1,1]^3 restricted to it, cell by cell (uniform, M = 2)"""
    n = 6
    full = oracle.Oracle(oracle.make_cfg(dim=3, M=2, n=(2 * n, 2 * n, 2 * n), lo=(-1, -1, -1), hi=(1, 1, 1), bc=T,
                                         cfl=0.6), threads=8)
    octant = oracle.Oracle(oracle.make_cfg(dim=3, M=2, n=(n, n, n), lo=(0, 0, 0), hi=(1, 1, 1),
                                           bc=[R, T, R, T, R, T], cfl=0.6), threads=8)
    full.set_initial(oracle.IC_EXPLOSION, EXPL)
    octant.set_initial(oracle.IC_EXPLOSION, EXPL)
    for _ in range(3):
        dt = full.compute_dt()
        assert octant.compute_dt() == pytest.approx(dt, rel=1e-14)
        full.advance_dt(dt)
        octant.advance_dt(dt)
    _, uf = full.cells()
    _, uo = octant.cells()
    uf = uf.reshape(2 * n, 2 * n, 2 * n, 5)[n:, n:, n:]
    assert np.allclose(uo.reshape(n, n, n, 5), uf, rtol=0, atol=1e-12)
    assert np.max(np.abs(uo[:, 1:4])) > 1e-3              # the flow has started
