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


# ---- MHD-GLM (Sec. 4.2): |A| of the 9 x 9 Jacobian by the matrix sign function ----

G53, CH = 5.0 / 3.0, 2.0


def _mhd(flux=1):
    return oracle.Oracle(oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, gamma=G53, c_h=CH, flux=flux))


def _mhd_state(rng, bscale=1.5):
    rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
    v, B = rng.uniform(-1, 1, 3), rng.uniform(-bscale, bscale, 3)
    E = p / (G53 - 1) + 0.5 * rho * v @ v + 0.5 * B @ B
    return np.concatenate([[rho], rho * v, [E], B, [rng.uniform(-0.1, 0.1)]])


def _mhd_eigenvalues(q, n):
    """closed forms: v_n, v_n +- c_a, v_n +- c_s, v_n +- c_f (ideal MHD with B_n given) and +-c_h
    (the GLM cleaning pair)"""
    rho, v, B = q[0], q[1:4] / q[0], q[5:8]
    p = (G53 - 1) * (q[4] - 0.5 * rho * v @ v - 0.5 * B @ B)
    a2, b2, bn2 = G53 * p / rho, B @ B / rho, B[n] ** 2 / rho
    disc = np.sqrt((a2 + b2) ** 2 - 4 * a2 * bn2)
    cf, cs, ca = np.sqrt(0.5 * (a2 + b2 + disc)), np.sqrt(max(0.5 * (a2 + b2 - disc), 0.0)), np.sqrt(bn2)
    vn = v[n]
    return np.sort([vn, vn - ca, vn + ca, vn - cs, vn + cs, vn - cf, vn + cf, -CH, CH])


def test_mhd_jacobian_spectrum_and_abs_jacobian_match_numpy():
    """the finite-difference Jacobian of the oracle's MHD-GLM flux has the closed-form
    eigenvalues, and the oracle's |A| equals V |Lambda| V^-1 from numpy's eigen-decomposition of
    that Jacobian"""
    o = _mhd()
    rng = np.random.default_rng(23)
    for _ in range(6):
        q = _mhd_state(rng)
        for n in range(2):
            J = _num_jac(o, q, n)
            lam, Vv = np.linalg.eig(J)
            assert np.max(np.abs(lam.imag)) < 1e-6
            assert np.allclose(np.sort(lam.real), _mhd_eigenvalues(q, n), atol=1e-6)
            ref = (Vv @ np.diag(np.abs(lam)) @ np.linalg.inv(Vv)).real
            got = o.abs_jacobian(q, n)
            assert np.allclose(got, ref, atol=1e-6 * np.abs(ref).max()), np.abs(got - ref).max()
            # |A| has the moduli of the eigenvalues as its spectrum
            assert np.allclose(np.sort(np.linalg.eigvals(got).real), np.sort(np.abs(_mhd_eigenvalues(q, n))),
                               atol=1e-8)


def test_mhd_osher_cleaning_part_is_the_exact_linear_riemann_flux():
    """B_n and psi obey the linear system dB_n/dt + dpsi/dn = 0, dpsi/dt + c_h^2 dB_n/dn = 0 on
    their own (the other fluxes do not depend on psi, B_n's and psi's fluxes on nothing else), so
    their rows of |A| are c_h times the identity there: the Osher flux of B_n and psi is the exact
    Riemann flux of that system for any two states"""
    o = _mhd()
    rng = np.random.default_rng(5)
    for _ in range(4):
        qm, qp = _mhd_state(rng), _mhd_state(rng)
        for n in range(2):
            f = o.osher(qm, qp, n)
            bm, bp, pm, pp = qm[5 + n], qp[5 + n], qm[8], qp[8]
            assert f[5 + n] == pytest.approx(0.5 * (pm + pp) - 0.5 * CH * (bp - bm), rel=1e-12, abs=1e-13)
            assert f[8] == pytest.approx(0.5 * CH ** 2 * (bm + bp) - 0.5 * CH * (pp - pm), rel=1e-12, abs=1e-13)
            assert np.allclose(o.osher(qm, qm, n), o.flux(qm, n), rtol=0, atol=1e-14)


def test_mhd_abs_jacobian_without_field_is_the_euler_one():
    """with B = 0 and psi = 0 the hydrodynamic block of the MHD-GLM |A| is the 3D Euler |A|, whose
    eigenvectors the oracle writes out in closed form"""
    o = _mhd()
    e3 = oracle.Oracle(oracle.make_cfg(dim=3, pde=oracle.PDE_EULER, gamma=G53, flux=1))
    rng = np.random.default_rng(9)
    for _ in range(4):
        rho, p, v = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0), rng.uniform(-1, 1, 3)
        qe = _cons(rho, v, p, g=G53)
        q = np.concatenate([qe, np.zeros(4)])
        for n in range(2):
            assert np.allclose(o.abs_jacobian(q, n)[:5, :5], e3.abs_jacobian(qe, n), rtol=0, atol=1e-11)


@pytest.mark.parametrize("M,lo_order", [(2, 2.7)])
def test_mhd_osher_alfven_wave_order(M, lo_order):
    """the circularly polarised Alfven wave (exact nonlinear solution; tests/test_oracle_mhd.py)
    with the Osher flux converges at the design order"""
    from tests.test_oracle_mhd import alfven_error
    e = [alfven_error(M, n, 0.25, flux=1) for n in (16, 32)]
    order = np.log2(e[0] / e[1])
    assert order > lo_order, (e, order)
    assert e[1] < 2e-4
