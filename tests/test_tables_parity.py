"""Parity of the reference-element tables of the CUDA path (computed on the host by the library,
aw_tables_host, in long double) with the oracle's own tables (built independently in double):
no GPU is needed.  The oracle's basis is given by its coefficients in powers of (xi - 1/2), so the
derivative matrix, end values, child averages and fine-point values are evaluated here from those
polynomials; the predictor's time block G is read off the oracle's full space-time matrix K1^-1,
which in the nodal tensor basis is diag(1 / (w x w)) (x) K_t^-1 (Sec. 2.3)."""
import numpy as np
import pytest

import oracle
import paper_1212_3585_gb300 as pg


def poly(coef, xi):
    return sum(c * (xi - 0.5) ** k for k, c in enumerate(coef))


def dpoly(coef, xi):
    return sum(k * c * (xi - 0.5) ** (k - 1) for k, c in enumerate(coef) if k > 0)


def ipoly(coef, a, b):
    """exact integral over [a, b]"""
    return sum(c * ((b - 0.5) ** (k + 1) - (a - 0.5) ** (k + 1)) / (k + 1) for k, c in enumerate(coef))


def close(a, b, tol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("r", [2, 3, 4])
def test_tables_match_the_oracle(M, r):
    if r < M:
        pytest.skip("the configurations use r >= M")
    g = pg.tables_host(M, r)
    o = oracle.tables(M)
    N = M + 1
    assert (g["N"], g["Ns"], g["r"]) == (N, o["Ns"], r)
    assert close(g["x"], o["x"], 1e-15) and close(g["w"], o["w"], 1e-15)
    assert list(g["SL"]) == list(o["SL"]) and list(g["lam"]) == list(o["lam"])
    assert close(g["Ainv"], o["ainv"], 1e-12)
    assert close(g["Sig"], o["sig"], 1e-12)
    psi = o["psi"]                     # psi[l][k]: coefficient of (xi - 1/2)^k in psi_l
    x = o["x"]
    assert close(g["psi0"], [poly(psi[l], 0.0) for l in range(N)], 1e-13)
    assert close(g["psi1"], [poly(psi[l], 1.0) for l in range(N)], 1e-13)
    assert close(g["Dm"], [[dpoly(psi[l], x[i]) for l in range(N)] for i in range(N)], 1e-12)
    assert close(g["Wc"], [[r * ipoly(psi[l], c / r, (c + 1) / r) for l in range(N)] for c in range(r)], 1e-13)
    assert close(g["Pf"], [[[poly(psi[l], (c + x[i]) / r) for l in range(N)] for i in range(N)] for c in range(r)],
                 1e-13)
    assert close(g["Pt"], [[poly(psi[l], c / r) for l in range(N)] for c in range(r)], 1e-13)
    k1inv, _, _ = oracle.st_matrices(M, 2)
    nsp = N * N
    w = o["w"]
    G = np.array([[k1inv[nsp * a, nsp * b] * w[0] * w[0] * w[b] for b in range(N)] for a in range(N)])
    assert close(g["G"], G, 1e-12)
    assert close(g["gsum"], G.sum(axis=1), 1e-12)
    # sigma of each stencil as a quadratic form of the differences to the centre cell's average
    for s, sl in enumerate(o["SL"]):
        B = o["ainv"][s].T @ o["sig"] @ o["ainv"][s]
        keep = [e for e in range(N) if e != sl]
        Bq = np.array([[0.0 if j < i else (1.0 if i == j else 2.0) * B[keep[i], keep[j]] for j in range(N - 1)]
                       for i in range(N - 1)])
        assert close(g["Bq"][s], Bq, 1e-10)
        # and it gives the oracle's sigma: stencil values v, differences d = v - v_centre
        v = np.random.default_rng(s).uniform(-1, 1, N)
        v[sl] = 0.3
        c = o["ainv"][s] @ v
        d = np.array([v[e] - v[sl] for e in keep])
        assert abs(d @ g["Bq"][s] @ d - c @ o["sig"] @ c) <= 1e-11 * max(1.0, abs(c @ o["sig"] @ c))


def test_tables_host_rejects_bad_arguments():
    L = pg._lib.load()
    import ctypes as C
    n = C.c_int64(0)
    for M, r in ((0, 3), (4, 3), (2, 1), (2, 5)):
        assert L.aw_tables_host(M, r, None, 0, C.byref(n)) == pg._lib.AW_EINVAL
    assert L.aw_tables_host(2, 3, None, 0, None) == pg._lib.AW_EINVAL
    N, r = 3, 3
    need = 11 + 5 * N + 7 * N * N + 2 * r * N + r * N * N + 4 * (N - 1) ** 2
    assert L.aw_tables_host(2, 3, None, 0, C.byref(n)) == pg._lib.AW_EINVAL and n.value == need


@pytest.mark.parametrize("M", [1, 2, 3])
def test_predictor_time_block_carries_the_initial_data(M):
    """the factorised predictor adds the reconstruction w_h(node) itself in place of the
    K1^-1 F0 w term: that needs K_t^-1 psi(0) = 1, i.e. G (psi(0) / w) = 1 for G = K_t^-1 diag(w)
    (a function constant in time solves the time block with unit data at tau = 0)"""
    g = pg.tables_host(M, 3)
    assert np.allclose(g["G"] @ (g["psi0"] / g["w"]), 1.0, rtol=0, atol=1e-13)
