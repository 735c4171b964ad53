"""Pins of the oracle's reference-element tables and 1D WENO (Sec. 2.2 of the paper).

Each check compares the oracle with something it does not compute itself:
  * Gauss-Legendre rule: closed forms for 3 and 4 points and numpy's leggauss.
  * Nodal basis psi_l: Kronecker property psi_l(x_k) = delta_lk.
  * Stencil inverses (Eq. eqn.rec.x): the reconstruction polynomial of each stencil is the
    unique degree-M polynomial with the given cell averages; it is solved here exactly in
    the monomial basis with Fractions and compared at the Gauss nodes.
  * Oscillation matrix (Eq. eqn.sigmas): w^T Sigma w equals sum_alpha int_0^1 (P^(alpha))^2
    computed exactly for the monomial-basis polynomial P.
  * 1D WENO (Eqs. eqn.weno, eqn.omegas): reproduces polynomials of degree <= M for any
    weights, mirror symmetry, constant data, and selection of the smooth stencil at a jump.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.polyref import gl01, lagrange_values, mono_cell_average, poly_deriv, poly_eval, solve_exact


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_gauss_legendre_matches_numpy(M):
    t = oracle.tables(M)
    x, w = gl01(M + 1)
    assert np.allclose(t["x"], x, atol=1e-15, rtol=0)
    assert np.allclose(t["w"], w, atol=1e-15, rtol=0)


def test_gauss_legendre_closed_forms():
    # 3 points on [-1,1]: 0, +-sqrt(3/5), weights 8/9, 5/9; 4 points: +-sqrt(3/7 -+ 2/7 sqrt(6/5))
    t = oracle.tables(2)
    assert np.allclose(t["x"], 0.5 * (1 + np.array([-math.sqrt(0.6), 0.0, math.sqrt(0.6)])), atol=1e-15)
    assert np.allclose(t["w"], 0.5 * np.array([5 / 9, 8 / 9, 5 / 9]), atol=1e-15)
    t = oracle.tables(3)
    a = math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5))
    b = math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))
    wa = (18 + math.sqrt(30)) / 36
    wb = (18 - math.sqrt(30)) / 36
    assert np.allclose(t["x"], 0.5 * (1 + np.array([-b, -a, a, b])), atol=1e-15)
    assert np.allclose(t["w"], 0.5 * np.array([wb, wa, wa, wb]), atol=1e-15)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_lagrange_kronecker(M):
    t = oracle.tables(M)
    N = M + 1
    for l in range(N):
        vals = [np.polyval(t["psi"][l][::-1], xk - 0.5) for xk in t["x"]]
        assert np.allclose(vals, np.eye(N)[l], atol=1e-13)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_stencils_match_paper(M):
    t = oracle.tables(M)
    if M % 2 == 0:
        assert t["Ns"] == 3
        assert list(zip(t["SL"], t["SR"])) == [(M // 2, M // 2), (M, 0), (0, M)]
        assert list(t["lam"]) == [1e5, 1.0, 1.0]
    else:
        assert t["Ns"] == 4
        f = M // 2
        assert list(zip(t["SL"], t["SR"])) == [(f + 1, f), (f, f + 1), (M, 0), (0, M)]
        assert list(t["lam"]) == [1e5, 1e5, 1.0, 1.0]


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_stencil_inverse_exact(M):
    t = oracle.tables(M)
    N = M + 1
    rng = random.Random(7 + M)
    for s in range(t["Ns"]):
        L = t["SL"][s]
        offs = [-L + e for e in range(N)]
        for _ in range(3):
            avg = [Fraction(rng.randint(-50, 50), rng.randint(1, 9)) for _ in range(N)]
            A = [[mono_cell_average([0] * k + [1], o, o + 1) for k in range(N)] for o in offs]
            coef = solve_exact(A, avg)
            expect = [poly_eval(coef, xk) for xk in t["x"]]
            got = t["ainv"][s] @ np.array([float(a) for a in avg])
            assert np.allclose(got, expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_sigma_closed_form(M):
    t = oracle.tables(M)
    rng = random.Random(11 + M)
    for _ in range(5):
        coef = [Fraction(rng.randint(-9, 9), rng.randint(1, 5)) for _ in range(M + 1)]
        exact = Fraction(0)
        c = coef
        for _a in range(M):
            c = poly_deriv(c)
            sq = [Fraction(0)] * (2 * len(c))
            for i, ci in enumerate(c):
                for j, cj in enumerate(c):
                    sq[i + j] += ci * cj
            exact += sum(sq[k] / (k + 1) for k in range(len(sq)))
        w = np.array([poly_eval(coef, xk) for xk in t["x"]])
        assert w @ t["sig"] @ w == pytest.approx(float(exact), rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_weno1d_reproduces_polynomials(M):
    t = oracle.tables(M)
    rng = random.Random(3 + M)
    for deg in range(M + 1):
        coef = [Fraction(rng.randint(-20, 20), rng.randint(1, 7)) for _ in range(deg + 1)]
        avg = np.array([float(mono_cell_average(coef, e, e + 1)) for e in range(-M, M + 1)])
        got = oracle.weno1d(M, avg)
        expect = [poly_eval(coef, xk) for xk in t["x"]]
        assert np.allclose(got, expect, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_weno1d_mirror_and_constant(M):
    rng = np.random.default_rng(5)
    for _ in range(20):
        v = rng.normal(size=2 * M + 1)
        a = oracle.weno1d(M, v)
        b = oracle.weno1d(M, v[::-1])
        assert np.allclose(a, b[::-1], rtol=1e-10, atol=1e-10)
    c = oracle.weno1d(M, np.full(2 * M + 1, 3.25))
    assert np.allclose(c, 3.25, atol=1e-14)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_weno1d_picks_smooth_stencil_at_jump(M):
    # jump just right of the cell: the fully left-sided stencil sees constant data
    v = np.zeros(2 * M + 1)
    v[M + 1:] = 1.0
    out = oracle.weno1d(M, v)
    assert np.all(np.abs(out) < 1e-6)
    # the reconstruction is always a convex combination of the stencil polynomials
    v = np.arange(2 * M + 1.0) ** 3 - 7 * np.arange(2 * M + 1.0)
    out = oracle.weno1d(M, v)
    t = oracle.tables(M)
    polys = [t["ainv"][s] @ v[M - t["SL"][s]: M - t["SL"][s] + M + 1] for s in range(t["Ns"])]
    lo = np.min(polys, axis=0)
    hi = np.max(polys, axis=0)
    assert np.all(out >= lo - 1e-12) and np.all(out <= hi + 1e-12)
