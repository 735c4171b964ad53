"""Pins of the oracle's space-time predictor, fluxes and multi-D WENO (Secs. 2.1-2.3).

  * K1, K_xi, F0 (defined before Eq. eqn.pde.weak4) against an independent numpy quadrature
    of their defining integrals, using integration by parts for K1.
  * Predictor (Eq. eqn.stdg.final): a constant state is a fixed point; for a linear flux
    (linear advection, and the Euler contact wave whose flux is linear in rho) and data of
    total degree <= M, M+1 Picard iterations reproduce the exact space-time solution
    w(xi - a tau dt/dx), because each iteration lowers the spatial degree of the error.
  * Picard iteration converges to the solution of Eq. eqn.pde.weak4 (residual check).
  * Fluxes: the largest |eigenvalue| of the finite-difference Jacobian equals max_speed
    (Euler, MHD-GLM); Rusanov consistency f~(q,q) = f(q) (Eq. eqn.rusanov); axis-swap
    invariance of the MHD-GLM flux; stationary-gas flux.
  * Multi-D WENO (Eqs. eqn.weno.y, eqn.weno.z) reproduces tensor polynomials of degree <= M
    per direction from their exact cell averages.
"""
import itertools
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.polyref import gl01, lagrange_derivs, lagrange_values, mono_cell_average


def nodal_index_points(N, d):
    """reference coordinates of the space-time nodes in the oracle's order (p fastest, time last)"""
    x, _ = gl01(N)
    pts = []
    for idx in range(N ** (d + 1)):
        t = idx
        c = []
        for _a in range(d + 1):
            c.append(x[t % N])
            t //= N
        pts.append(c)
    return np.array(pts)


@pytest.mark.parametrize("M,d", [(1, 2), (2, 2), (3, 2), (2, 3)])
def test_space_time_matrices_against_quadrature(M, d):
    N = M + 1
    nst = N ** (d + 1)
    nsp = N ** d
    k1inv, kd, f0 = oracle.st_matrices(M, d)
    x, _ = gl01(N)
    qx, qw = gl01(N + 2)
    B = lagrange_values(x, qx)       # (nq, N)
    DB = lagrange_derivs(x, qx)
    B0 = lagrange_values(x, [0.0])[0]

    def theta(idx):
        t = idx
        out = []
        for _a in range(d + 1):
            out.append(t % N)
            t //= N
        return out

    rng = np.random.default_rng(1)
    g = rng.normal(size=nst)          # nodal values of a space-time polynomial
    w = rng.normal(size=nsp)
    nq = len(qx)
    # integrals over all quadrature points (d+1 nested)
    K1g = np.zeros(nst)
    Kg = np.zeros((d, nst))
    F0w = np.zeros(nst)
    grids = list(itertools.product(range(nq), repeat=d + 1))
    # precompute g and its derivatives at quadrature points
    gval = {}
    for gp in grids:
        val = 0.0
        dt = 0.0
        dsp = np.zeros(d)
        for p in range(nst):
            ip = theta(p)
            bv = np.prod([B[gp[a], ip[a]] for a in range(d + 1)])
            val += g[p] * bv
            dt += g[p] * np.prod([B[gp[a], ip[a]] for a in range(d)]) * DB[gp[d], ip[d]]
            for a in range(d):
                dsp[a] += g[p] * np.prod([(DB if b == a else B)[gp[b], ip[b]] for b in range(d + 1)])
        gval[gp] = (val, dt, dsp)
    for q in range(nst):
        iq = theta(q)
        s1 = 0.0
        sk = np.zeros(d)
        for gp in grids:
            wt = np.prod([qw[gp[a]] for a in range(d + 1)])
            th = np.prod([B[gp[a], iq[a]] for a in range(d + 1)])
            val, dt, dsp = gval[gp]
            s1 += wt * th * dt
            sk += wt * th * dsp
        # + int theta_q(xi,0) g(xi,0)  and  int theta_q(xi,0) w(xi)
        s0 = 0.0
        sf = 0.0
        for gs in itertools.product(range(nq), repeat=d):
            wt = np.prod([qw[gs[a]] for a in range(d)])
            thq = np.prod([B[gs[a], iq[a]] for a in range(d)]) * B0[iq[d]]
            g0 = 0.0
            for p in range(nst):
                ip = theta(p)
                g0 += g[p] * np.prod([B[gs[a], ip[a]] for a in range(d)]) * B0[ip[d]]
            w0 = 0.0
            for m in range(nsp):
                im = theta(m)
                w0 += w[m] * np.prod([B[gs[a], im[a]] for a in range(d)])
            s0 += wt * thq * g0
            sf += wt * thq * w0
        K1g[q] = s1 + s0
        Kg[:, q] = sk
        F0w[q] = sf
    assert np.allclose(np.linalg.solve(k1inv, g), K1g, rtol=1e-11, atol=1e-11)
    for a in range(d):
        assert np.allclose(kd[a] @ g, Kg[a], rtol=1e-11, atol=1e-11)
    assert np.allclose(f0 @ w, F0w, rtol=1e-11, atol=1e-11)


def _st_nodal(f, N, d):
    pts = nodal_index_points(N, d)
    return np.array([f(p) for p in pts])


def _sp_nodal(f, N, d):
    x, _ = gl01(N)
    out = []
    for idx in range(N ** d):
        t = idx
        c = []
        for _a in range(d):
            c.append(x[t % N])
            t //= N
        out.append(f(c))
    return np.array(out)


def _random_total_degree_poly(M, d, rng):
    terms = [e for e in itertools.product(range(M + 1), repeat=d) if sum(e) <= M]
    coef = {e: rng.normal() for e in terms}
    return lambda x: sum(c * np.prod([x[a] ** e[a] for a in range(d)]) for e, c in coef.items())


@pytest.mark.parametrize("M,d", [(1, 2), (2, 2), (3, 2), (2, 3)])
def test_predictor_linear_advection_exact(M, d):
    adv = (0.7, -0.4, 0.3)
    cfg = oracle.make_cfg(dim=d, pde=oracle.PDE_LINADV, M=M, n=(8, 8, 8), adv=adv)
    o = oracle.Oracle(cfg)
    rng = np.random.default_rng(2)
    P = _random_total_degree_poly(M, d, rng)
    N = M + 1
    dt = 0.3
    dx = (0.5, 0.8, 0.6)[:d]
    wh = _sp_nodal(P, N, d)
    qh = o.predictor(wh, dt, dx)
    exact = _st_nodal(lambda p: P([p[a] - adv[a] * p[d] * dt / dx[a] for a in range(d)]), N, d)
    assert np.allclose(qh, exact, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("M,d", [(1, 2), (2, 2), (3, 2), (2, 3)])
def test_picard_iteration_beyond_m_plus_1_changes_nothing(M, d):
    """for a linear flux the Picard iteration is exact after M+1 steps (the spatial derivative is
    nilpotent on degree-M data): one more step changes the result by round-off only"""
    adv = (0.7, -0.4, 0.3)
    rng = np.random.default_rng(12)
    P = _random_total_degree_poly(M, d, rng)
    N = M + 1
    wh = _sp_nodal(P, N, d)
    dx = (0.5, 0.8, 0.6)[:d]
    out = []
    for picard in (M + 1, M + 2):
        cfg = oracle.make_cfg(dim=d, pde=oracle.PDE_LINADV, M=M, n=(8, 8, 8), adv=adv, picard=picard)
        out.append(oracle.Oracle(cfg).predictor(wh, 0.3, dx))
    assert np.allclose(out[0], out[1], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_predictor_euler_contact_wave_exact(M):
    d = 2
    gamma = 1.4
    cfg = oracle.make_cfg(dim=d, pde=oracle.PDE_EULER, M=M, gamma=gamma)
    o = oracle.Oracle(cfg)
    rng = np.random.default_rng(3)
    P = _random_total_degree_poly(M, d, rng)
    rho = lambda x: 2.0 + 0.1 * P(x)
    u, v, p = 0.6, -0.35, 1.3
    N = M + 1
    dt, dx = 0.05, (0.1, 0.08)
    r = _sp_nodal(rho, N, d)
    wh = np.concatenate([r, u * r, v * r, p / (gamma - 1) + 0.5 * (u * u + v * v) * r])
    qh = o.predictor(wh, dt, dx)
    re = _st_nodal(lambda q: rho([q[0] - u * q[d] * dt / dx[0], q[1] - v * q[d] * dt / dx[1]]), N, d)
    exact = np.concatenate([re, u * re, v * re, p / (gamma - 1) + 0.5 * (u * u + v * v) * re])
    assert np.allclose(qh, exact, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("pde,M", [(oracle.PDE_EULER, 2), (oracle.PDE_MHD, 3)])
def test_predictor_constant_state_fixed_point(pde, M):
    cfg = oracle.make_cfg(dim=2, pde=pde, M=M, gamma=5 / 3 if pde == oracle.PDE_MHD else 1.4)
    o = oracle.Oracle(cfg)
    V = o.V
    if pde == oracle.PDE_EULER:
        q = np.array([1.2, 0.3, -0.2, 2.5])
    else:
        q = np.array([1.2, 0.3, -0.2, 0.1, 3.0, 0.4, -0.3, 0.2, 0.05])
    wh = np.repeat(q, o.nsp)
    qh = o.predictor(wh, 0.01, (0.1, 0.1))
    assert np.allclose(qh, np.repeat(q, o.nst), rtol=1e-13, atol=1e-13)


def test_picard_solves_the_weak_form():
    """many iterations at a small CFL: residual of Eq. eqn.pde.weak4 -> 0"""
    M, d = 2, 2
    cfg = oracle.make_cfg(dim=d, pde=oracle.PDE_EULER, M=M, picard=40)
    o = oracle.Oracle(cfg)
    k1inv, kd, f0 = oracle.st_matrices(M, d)
    rng = np.random.default_rng(4)
    N = M + 1
    base = np.array([1.0, 0.2, -0.1, 2.5])
    wh = np.concatenate([base[v] + 0.05 * rng.normal(size=o.nsp) for v in range(4)])
    dt, dx = 0.01, (0.1, 0.1)
    qh = o.predictor(wh, dt, dx).reshape(4, o.nst)
    K1 = np.linalg.inv(k1inv)
    fs = np.zeros((d, 4, o.nst))
    for p in range(o.nst):
        for a in range(d):
            fs[a, :, p] = dt / dx[a] * o.flux(qh[:, p], a)
    for v in range(4):
        res = K1 @ qh[v] + sum(kd[a] @ fs[a, v] for a in range(d)) - f0 @ wh.reshape(4, o.nsp)[v]
        assert np.max(np.abs(res)) < 1e-12


def _num_jacobian(o, q, n):
    V = len(q)
    J = np.zeros((V, V))
    for j in range(V):
        h = 1e-6 * max(1.0, abs(q[j]))
        qp, qm = q.copy(), q.copy()
        qp[j] += h
        qm[j] -= h
        J[:, j] = (o.flux(qp, n) - o.flux(qm, n)) / (2 * h)
    return J


@pytest.mark.parametrize("d", [2, 3])
def test_euler_eigenvalues_and_flux(d):
    o = oracle.Oracle(oracle.make_cfg(dim=d, pde=oracle.PDE_EULER, gamma=1.4))
    rng = np.random.default_rng(6)
    for _ in range(5):
        rho, p = rng.uniform(0.2, 2.0), rng.uniform(0.2, 2.0)
        vel = rng.uniform(-1, 1, size=d)
        q = np.concatenate([[rho], rho * vel, [p / 0.4 + 0.5 * rho * vel @ vel]])
        for n in range(d):
            ev = np.linalg.eigvals(_num_jacobian(o, q, n))
            c = np.sqrt(1.4 * p / rho)
            assert np.allclose(np.sort(ev.real), np.sort([vel[n] - c, vel[n] + c] + [vel[n]] * d), atol=1e-6)
            assert o.max_speed(q, n) == pytest.approx(np.max(np.abs(ev)), rel=1e-6)
            assert np.allclose(o.rusanov(q, q, n), o.flux(q, n), rtol=0, atol=0)
    q = np.concatenate([[1.3], np.zeros(d), [0.7 / 0.4]])
    f = o.flux(q, 0)
    assert np.allclose(f, np.concatenate([[0.0, 0.7], np.zeros(d - 1), [0.0]]))


def test_mhd_glm_eigenvalues_and_symmetry():
    ch = 2.0
    o = oracle.Oracle(oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, gamma=5 / 3, c_h=ch))
    rng = np.random.default_rng(8)
    g = 5 / 3
    for _ in range(5):
        rho, p = rng.uniform(0.5, 2.0), rng.uniform(0.5, 2.0)
        v = rng.uniform(-1, 1, size=3)
        B = rng.uniform(-1, 1, size=3)
        psi = rng.uniform(-0.1, 0.1)
        q = np.array([rho, *(rho * v), p / (g - 1) + 0.5 * rho * v @ v + 0.5 * B @ B, *B, psi])
        for n in range(2):
            ev = np.linalg.eigvals(_num_jacobian(o, q, n))
            assert o.max_speed(q, n) == pytest.approx(max(np.max(np.abs(ev.real)), ch), rel=1e-5)
            # the GLM subsystem contributes the eigenvalues +-c_h
            assert np.min(np.abs(np.abs(ev.real) - ch)) < 1e-6
            assert np.allclose(o.rusanov(q, q, n), o.flux(q, n), rtol=0, atol=0)
        # swapping the x and y axes maps the x flux onto the y flux
        perm = [0, 2, 1, 3, 4, 6, 5, 7, 8]
        qs = q[perm]
        assert np.allclose(o.flux(qs, 1)[perm], o.flux(q, 0), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("M,d", [(1, 2), (2, 2), (3, 2), (2, 3)])
def test_multid_weno_reproduces_tensor_polynomials(M, d):
    n = 2 * M + 3
    cfg = oracle.make_cfg(dim=d, pde=oracle.PDE_LINADV, M=M, n=(n, n, n), lo=(0, 0, 0), hi=(n, n, n),
                          bc=oracle.BC_TRANSMISSIVE)
    o = oracle.Oracle(cfg)
    rng = random.Random(9)
    # separable tensor polynomial of degree M in each direction
    coefs = [[Fraction(rng.randint(-9, 9), rng.randint(1, 4)) for _ in range(M + 1)] for _a in range(d)]
    avgs1 = [[mono_cell_average(coefs[a], i, i + 1) for i in range(n)] for a in range(d)]
    u = []
    for k in range(n if d == 3 else 1):
        for j in range(n):
            for i in range(n):
                v = avgs1[0][i] * avgs1[1][j] * (avgs1[2][k] if d == 3 else 1)
                u.append([float(v)])
    o.set_cell_averages(np.array(u))
    o.weno_level(0)
    wh = o.internal(0, 0).reshape(-1, o.nsp)
    x, _ = gl01(M + 1)
    ncell = 0
    for k in range(n if d == 3 else 1):
        for j in range(n):
            for i in range(n):
                ijk = (i, j, k)
                inner = all(M <= ijk[a] < n - M for a in range(d))
                if inner:
                    def f(c, ijk=ijk):
                        val = 1.0
                        for a in range(d):
                            val *= sum(float(cf) * (ijk[a] + c[a]) ** e for e, cf in enumerate(coefs[a]))
                        return val
                    expect = _sp_nodal(f, M + 1, d)
                    assert np.allclose(wh[ncell], expect, rtol=1e-10, atol=1e-10)
                ncell += 1
