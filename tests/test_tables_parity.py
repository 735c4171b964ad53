"""Parity of the reference-element tables of the CUDA path (computed on the host by the library,
aw_tables_host, in long double) with the oracle's own tables (built independently in double),
and of the factorised predictor form the kernels implement with the oracle's full Picard
iteration: no GPU is needed.  The oracle's basis is given by its coefficients in powers of (xi - 1/2), so the
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


def factorised_predictor(o, g, wh, dt, dx, d, P):
    """the predictor in the factorised nodal form the kernels use, written with numpy and the
    library's tables: with the nodal tensor basis,
      q(node, s) = w_h(node) - sum_s' G[s][s'] sum_a (dt / dx_a) sum_k Dm[i_a][k] f_a(q(node_{i_a -> k}, s'))
    iterated P times from q = w_h (constant in time)"""
    N, V = g["N"], o.V
    shape = (V,) + (N,) * d                   # [v][i_z][i_y][i_x] in C order of the oracle's p + N q + N^2 r
    w = wh.reshape(shape)
    q = np.repeat(w[..., None], N, axis=-1)   # [..., s]
    for _ in range(P):
        flat = q.reshape(V, -1)
        F = np.stack([np.array([o.flux(flat[:, m], a) for m in range(flat.shape[1])]).T.reshape(q.shape) * dt / dx[a]
                      for a in range(d)])     # [a][v][...nodes][s]
        rhs = np.zeros_like(q)
        for a in range(d):
            axis = 1 + (d - 1 - a)              # the array axis of coordinate a
            rhs += np.moveaxis(np.tensordot(g["Dm"], np.moveaxis(F[a], axis, 0), axes=(1, 0)), 0, axis)
        q = w[..., None] - np.einsum("st,...t->...s", g["G"], rhs)
    # back to the oracle's layout [v][node + nsp * s]
    return np.moveaxis(q, -1, 1).reshape(V, -1)


@pytest.mark.parametrize("d,pde,M", [(2, oracle.PDE_EULER, 3), (2, oracle.PDE_EULER, 2), (3, oracle.PDE_EULER, 2),
                                     (2, oracle.PDE_MHD, 3), (2, oracle.PDE_LINADV, 1)])
def test_factorised_predictor_equals_the_full_picard_iteration(d, pde, M):
    """the kernels' factorised form computes exactly the Picard iteration of Eq. eqn.stdg.final
    with the full space-time matrices (the oracle), up to rounding"""
    cfg = oracle.make_cfg(dim=d, pde=pde, M=M, n=(4, 4, 4), adv=(1.0, -0.5, 0.25))
    o = oracle.Oracle(cfg)
    g = pg.tables_host(M, 3)
    rng = np.random.default_rng(40 + 10 * d + M)
    base = {oracle.PDE_EULER: [1.0, 0.3, -0.2, 0.1, 2.5][:d + 2], oracle.PDE_LINADV: [1.0],
            oracle.PDE_MHD: [1.0, 0.3, -0.2, 0.1, 2.5, 0.4, 0.3, -0.2, 0.05]}[pde]
    wh = (np.array(base)[:, None] * (1.0 + 0.05 * rng.standard_normal((o.V, o.nsp)))).ravel()
    dt, dx = 0.02, (0.1, 0.08, 0.12)[:d]
    ref = o.predictor(wh, dt, dx).reshape(o.V, o.nst)
    got = factorised_predictor(o, g, wh, dt, dx, d, M + 1)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_difference_form_identities(M):
    """the kernels reconstruct from the differences to the cell's own average and drop the centre
    cell's column (reading R4b): exact because every stencil reproduces constants (each row of
    Ainv sums to 1) and Sigma annihilates them (a constant has equal nodal values)"""
    g = pg.tables_host(M, 3)
    N = g["N"]
    assert np.allclose(g["Ainv"].sum(axis=2), 1.0, rtol=0, atol=1e-13)
    assert np.allclose(g["Sig"] @ np.ones(N), 0.0, rtol=0, atol=1e-12 * np.abs(g["Sig"]).max())
    assert np.allclose(g["Dm"] @ np.ones(N), 0.0, rtol=0, atol=1e-12 * np.abs(g["Dm"]).max())


def weno1d_difference_form(g, v):
    """one-dimensional WENO as the kernels form it: the N-1 differences to the centre average,
    stencil polynomials from the other columns of Ainv, sigma from the quadratic form Bq, weights
    lambda / (sigma + 1e-14)^8"""
    N = g["N"]
    M = N - 1
    c = v[M]
    out, om = np.zeros(N), []
    polys = []
    for s in range(g["Ns"]):
        sl = g["SL"][s]
        keep = [e for e in range(N) if e != sl]
        d = np.array([v[M - sl + e] - c for e in keep])
        polys.append(g["Ainv"][s][:, keep] @ d)
        sigma = d @ g["Bq"][s] @ d
        om.append(g["lam"][s] / (sigma + 1e-14) ** 8)
    om = np.array(om) / sum(om)
    for s in range(g["Ns"]):
        out += om[s] * polys[s]
    return out + c


@pytest.mark.parametrize("M", [1, 2, 3])
def test_weno_difference_form_equals_the_oracle(M):
    g = pg.tables_host(M, 3)
    rng = np.random.default_rng(50 + M)
    x = np.arange(2 * M + 1) - M
    cases = [rng.uniform(0.5, 1.5, 2 * M + 1) for _ in range(20)]
    cases += [1.0 + 0.1 * np.sin(0.7 * x + p) for p in rng.uniform(0, 6, 10)]          # smooth
    cases += [np.where(x >= k, 2.0, 1.0) for k in range(-M, M + 1)]                    # jumps
    cases += [1e5 + 1e-3 * rng.standard_normal(2 * M + 1)]                              # large constant part
    for v in cases:
        ref = oracle.weno1d(M, v)
        got = weno1d_difference_form(g, v)
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), (v, got, ref)


@pytest.mark.parametrize("d,M,r", [(2, 3, 3), (2, 2, 2), (3, 2, 3), (2, 1, 4)])
def test_projection_with_the_tables_equals_the_oracle(d, M, r):
    """virtual children as the kernels form them (Sec. 3.1.3): the average over child box c of the
    mother's q_h at tau = k/r is sum over nodes of prod_a Wc[c_a][i_a] times Pt[k][s] times the
    node's value; likewise for w_h without the time factor.  The oracle integrates by quadrature."""
    o = oracle.Oracle(oracle.make_cfg(dim=d, pde=oracle.PDE_EULER, M=M, n=(4, 4, 4), r=r, lmax=1))
    g = pg.tables_host(M, r)
    N, V = M + 1, o.V
    rng = np.random.default_rng(60 + 10 * d + M)
    qh = rng.standard_normal(V * o.nst)
    wh = rng.standard_normal(V * o.nsp)
    q = qh.reshape((V, N) + (N,) * d)          # [v][s][i_z][i_y][i_x]
    w = wh.reshape((V,) + (N,) * d)
    for c in [tuple(int(v) for v in rng.integers(0, r, d)) for _ in range(4)]:
        u = w
        for a in range(d):                      # axes (v, [z], y, x): x is last, then y, then z
            u = np.tensordot(u, g["Wc"][c[a]], axes=([u.ndim - 1], [0]))
        assert np.allclose(u, o.project_sp(wh, c), rtol=0, atol=1e-13 * np.abs(wh).max())
        for k in range(r):
            t = np.tensordot(q, g["Pt"][k], axes=([1], [0]))     # the time axis
            for a in range(d):
                t = np.tensordot(t, g["Wc"][c[a]], axes=([t.ndim - 1], [0]))
            assert np.allclose(t, o.project_st(qh, c, k / r), rtol=0, atol=1e-13 * np.abs(qh).max())


@pytest.mark.parametrize("d,M,r", [(2, 3, 3), (3, 2, 3), (2, 2, 4)])
def test_coarse_trace_at_fine_points_with_the_tables(d, M, r):
    """the fine side of a coarse/fine face (Eq. eqn.memory.sum, reading R18): the coarse q_h at
    the fine face's Gauss point jt (transverse offset c_b = fine index - r * coarse index) and time
    node s of sub-step k, as the kernels form it from psi0/psi1 along the normal and Pf in the
    transverse directions and in time, equals the oracle's direct evaluation at
    ((c_b + x_jt) / r, (k + x_s) / r)"""
    o = oracle.Oracle(oracle.make_cfg(dim=d, pde=oracle.PDE_LINADV, M=M, n=(4, 4, 4), r=r, lmax=1))
    g = pg.tables_host(M, r)
    N = M + 1
    rng = np.random.default_rng(70 + 10 * d + M)
    qh = rng.standard_normal(o.nst)
    q = qh.reshape((N,) + (N,) * d)            # [s][i_z][i_y][i_x]
    x = g["x"]
    for _ in range(6):
        a = int(rng.integers(0, d))            # normal axis
        side = int(rng.integers(0, 2))         # the coarse cell's face: low (0) or high (1)
        c = [int(v) for v in rng.integers(0, r, d)]
        jt = [int(v) for v in rng.integers(0, N, d)]
        k, s = int(rng.integers(0, r)), int(rng.integers(0, N))
        t = np.tensordot(q, g["Pf"][k][s], axes=([0], [0]))
        xi = []
        for b in range(d):
            basis = (g["psi1"] if side else g["psi0"]) if b == a else g["Pf"][c[b]][jt[b]]
            t = np.tensordot(t, basis, axes=([t.ndim - 1], [0]))
            xi.append(float(side) if b == a else (c[b] + x[jt[b]]) / r)
        ref = o.eval_st(qh, xi, (k + x[s]) / r)[0]
        assert abs(float(t) - ref) <= 1e-13 * np.abs(qh).max(), (a, side, c, jt, k, s)
