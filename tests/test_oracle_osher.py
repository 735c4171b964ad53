"""Pins of the oracle's Osher-Solomon flux (Eq. eqn.osher, Dumbser-Toro path integral).

  * |A(q)| against numpy: eigen-decomposition of the finite-difference Jacobian,
    V |Lambda| V^-1 (2D and 3D Euler, every direction);
  * consistency f~(q, q) = f(q);
  * linear advection: the Osher flux is the upwind flux;
  * supersonic states (all eigenvalues of one sign along the path): the flux approaches the
    upwind physical flux, f~ -> f(q-) for flow to the right.
"""
import numpy as np
import pytest

import oracle


def _euler(d, flux=1):
    return oracle.Oracle(oracle.make_cfg(dim=d, pde=oracle.PDE_EULER, gamma=1.4, flux=flux))


def _cons(rho, vel, p, g=1.4):
    vel = np.asarray(vel, dtype=float)
    return np.concatenate([[rho], rho * vel, [p / (g - 1) + 0.5 * rho * vel @ vel]])


def _num_jac(o, q, n):
    V = len(q)
    J = np.zeros((V, V))
    for j in range(V):
        h = 1e-6 * max(1.0, abs(q[j]))
        a, b = q.copy(), q.copy()
        a[j] += h
        b[j] -= h
        J[:, j] = (o.flux(a, n) - o.flux(b, n)) / (2 * h)
    return J


@pytest.mark.parametrize("d", [2, 3])
def test_abs_jacobian_matches_numpy(d):
    o = _euler(d)
    rng = np.random.default_rng(21)
    for _ in range(5):
        q = _cons(rng.uniform(0.3, 2), rng.uniform(-1, 1, d), rng.uniform(0.3, 2))
        for n in range(d):
            lam, Vv = np.linalg.eig(_num_jac(o, q, n))
            ref = (Vv @ np.diag(np.abs(lam)) @ np.linalg.inv(Vv)).real
            assert np.allclose(o.abs_jacobian(q, n), ref, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("d", [2, 3])
def test_osher_consistency_and_supersonic_upwinding(d):
    o = _euler(d)
    q = _cons(1.2, [0.3] + [0.1] * (d - 1), 0.8)
    for n in range(d):
        assert np.allclose(o.osher(q, q, n), o.flux(q, n), rtol=0, atol=1e-15)
    # supersonic to the right along x: u - c > 0 on the whole path
    qm = _cons(1.0, [3.0] + [0.2] * (d - 1), 1.0)
    qp = _cons(1.01, [3.02] + [0.21] * (d - 1), 1.01)
    f = o.osher(qm, qp, 0)
    assert np.allclose(f, o.flux(qm, 0), rtol=1e-6)


def test_osher_linear_advection_is_upwind():
    o = oracle.Oracle(oracle.make_cfg(dim=2, pde=oracle.PDE_LINADV, adv=(0.7, -0.4, 0.0), flux=1))
    qm, qp = np.array([1.3]), np.array([-0.2])
    assert o.osher(qm, qp, 0)[0] == pytest.approx(0.7 * 1.3)
    assert o.osher(qm, qp, 1)[0] == pytest.approx(-0.4 * -0.2)


def test_explosion_with_osher_is_symmetric_and_conservative():
    o = oracle.Oracle(oracle.make_cfg(dim=2, M=3, n=(20, 20, 1), lo=(-1, -1, 0), hi=(1, 1, 1),
                                      bc=oracle.BC_TRANSMISSIVE, r=3, lmax=1, cfl=0.6, flux=1), threads=8)
    o.set_initial(oracle.IC_EXPLOSION, [0.5, 1.0, 1.0, 0.125, 0.1])
    t0 = o.totals()
    for _ in range(3):
        rc, _ = o.step(0.25)
        assert rc == 0
    assert np.allclose(o.totals()[[0, 3]], t0[[0, 3]], rtol=1e-13)
    meta, u = o.cells()
    d = {(m[0], m[2], m[3]): (m[1], uu) for m, uu in zip(meta, u)}
    for (lv, i, j), (st, uu) in d.items():
        if st > 0:
            continue
        n = 20 * 3 ** lv
        st2, u2 = d[(lv, n - 1 - i, j)]
        assert st2 == st
        assert abs(uu[0] - u2[0]) < 1e-11 and abs(uu[1] + u2[1]) < 1e-11
