"""Pins of the oracle's inflow boundaries (reading: the ghost cells beyond an inflow face hold the
prescribed conserved state, and the face flux is the numerical flux between that state and the
interior trace).

* Linear advection entering a constant state: the total changes at exactly a (c_in - c_0) L_y per
  unit time while the front is inside the domain (the inflow face flux of the upwind scheme is
  a c_in, the outflow face still sees c_0).
* A supersonic channel: a contact discontinuity enters with the inflow state and leaves the
  channel filled with it (a transmissive boundary would keep the initial state).
* An inflow state equal to the adjacent constant state gives the transmissive solution.
* The reconstruction next to an inflow (transmissive) face is the 1D WENO of the stencil line
  extended by the inflow state (the nearest cell).  The tests above cannot see which ghost
  state a cell's stencil holds: WENO puts all weight on the stencil inside the constant state.
"""
import numpy as np
import pytest

import aw_inputs
import oracle


@pytest.mark.parametrize("M", [2, 3])
def test_linear_advection_inflow_balance(M):
    c0, c1, a, Ly = 0.3, 1.0, 1.0, 0.25
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_LINADV, M=M, n=(64, 4, 1), lo=(0, 0, 0), hi=(1.0, Ly, 1),
                          bc=[oracle.BC_INFLOW, oracle.BC_TRANSMISSIVE, oracle.BC_PERIODIC, oracle.BC_PERIODIC,
                              oracle.BC_PERIODIC, oracle.BC_PERIODIC],
                          adv=(a, 0.0, 0.0), inflow=(c1,), cfl=0.9)
    o = oracle.Oracle(cfg, threads=4)
    o.set_initial(oracle.IC_CONST, [c0], nrefine=0)
    tot0 = o.totals()[0]
    t_end = 0.15
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    assert abs(o.totals()[0] - (tot0 + a * (c1 - c0) * Ly * t_end)) < 1e-13
    _, u = o.cells()
    assert np.max(np.abs(u[:, 0].reshape(4, 64)[:, -8:] - c0)) < 1e-15   # the outflow end untouched


def test_supersonic_channel_fills_with_inflow_state():
    g = 1.4
    rho0, rho1, u, p = 0.5, 1.0, 3.0, 1.0
    cons = lambda rho: [rho, rho * u, 0.0, p / (g - 1) + 0.5 * rho * u * u]
    cfg = oracle.make_cfg(dim=2, M=3, n=(24, 4, 1), lo=(0, 0, 0), hi=(1.0, 1.0 / 6, 1),
                          bc=[oracle.BC_INFLOW, oracle.BC_TRANSMISSIVE, oracle.BC_PERIODIC, oracle.BC_PERIODIC,
                              oracle.BC_PERIODIC, oracle.BC_PERIODIC],
                          inflow=cons(rho1), cfl=0.9, gamma=g)
    o = oracle.Oracle(cfg, threads=4)
    o.set_initial(oracle.IC_CONST, [rho0, u, 0.0, p], nrefine=0)   # primitive variables
    t_end = 1.0     # the contact (speed u) has left by t = 1/3; u - c = 1.8 flushes the rest
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    _, q = o.cells()
    assert np.max(np.abs(q - np.array(cons(rho1)))) < 1e-9 * cons(rho1)[3]


def test_inflow_of_the_boundary_state_equals_transmissive():
    """the explosion on [-1.5, 1.5]^2 for three steps, while even its numerical precursor is far
    from the boundary: an inflow face holding the outer state changes nothing"""
    E = aw_inputs.EXPLOSION
    outer = [E[3], 0.0, 0.0, E[4] / 0.4]
    runs = []
    for left in (oracle.BC_TRANSMISSIVE, oracle.BC_INFLOW):
        cfg = oracle.make_cfg(dim=2, M=3, n=(30, 30, 1), lo=(-1.5, -1.5, 0), hi=(1.5, 1.5, 1),
                              bc=[left] + [oracle.BC_TRANSMISSIVE] * 5, inflow=outer, cfl=0.6, r=3, lmax=1)
        o = oracle.Oracle(cfg, threads=4)
        o.set_initial(oracle.IC_EXPLOSION, E)
        for _ in range(3):
            assert o.step(1.0)[0] == 0
        runs.append(o.cells())
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.max(np.abs(runs[0][1] - runs[1][1])) < 1e-14


@pytest.mark.parametrize("M", [2, 3])
@pytest.mark.parametrize("axis", [0, 1])
def test_boundary_reconstruction_sees_the_ghost_states(M, axis):
    """the WENO polynomial of a cell within M of a boundary is the 1D WENO of its stencil line
    with the ghost states of the reading: the inflow state beyond an inflow face, the nearest
    cell (clamp) beyond a transmissive one.  The data vary only along `axis`, so the sweep along
    the other axis returns its constant line exactly."""
    n, nt, c_in = 9, 3, 2.5
    I, T, P = oracle.BC_INFLOW, oracle.BC_TRANSMISSIVE, oracle.BC_PERIODIC
    bc = [I, T, P, P, P, P] if axis == 0 else [P, P, I, T, P, P]
    ext = (n, nt, 1) if axis == 0 else (nt, n, 1)
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_LINADV, M=M, n=ext, lo=(0, 0, 0), hi=(ext[0], ext[1], 1), bc=bc,
                          adv=(1.0, 1.0, 0.0), inflow=(c_in,))
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [0.0], nrefine=0)
    prof = np.random.default_rng(20 + M).uniform(0.5, 1.5, n)
    u = np.tile(prof, (nt, 1)) if axis == 0 else np.tile(prof[:, None], (1, nt))
    o.set_cell_averages(u.reshape(-1, 1))
    o.weno_level(0)
    N = M + 1
    wh = o.internal(0, 0).reshape(ext[1], ext[0], N, N)      # [j][i][q][p], nodal
    line = np.concatenate([np.full(M, c_in), prof, np.full(M, prof[-1])])
    for c in list(range(M)) + list(range(n - M, n)):
        expect = oracle.weno1d(M, line[c:c + 2 * M + 1])
        for t in range(nt):
            w = wh[t, c] if axis == 0 else wh[c, t].T        # rows: the other axis' nodes
            assert np.array_equal(w, np.tile(expect, (N, 1))), (c, t)


@pytest.mark.parametrize("M", [2])
def test_boundary_reconstruction_sees_the_ghost_states_3d(M):
    """the same along z in 3D: data varying only with z, an inflow face at z = 0 and a
    transmissive one at the top; the x and y sweeps return their constant lines exactly"""
    n, nt, c_in = 9, 3, 2.5
    I, T, P = oracle.BC_INFLOW, oracle.BC_TRANSMISSIVE, oracle.BC_PERIODIC
    cfg = oracle.make_cfg(dim=3, pde=oracle.PDE_LINADV, M=M, n=(nt, nt, n), lo=(0, 0, 0), hi=(nt, nt, n),
                          bc=[P, P, P, P, I, T], adv=(0.0, 0.0, 1.0), inflow=(c_in,))
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [0.0], nrefine=0)
    prof = np.random.default_rng(30 + M).uniform(0.5, 1.5, n)
    o.set_cell_averages(np.repeat(prof, nt * nt).reshape(-1, 1))     # canonical order (k, j, i)
    o.weno_level(0)
    N = M + 1
    wh = o.internal(0, 0).reshape(n, nt, nt, N, N, N)                 # [k][j][i][r][q][p], nodal
    line = np.concatenate([np.full(M, c_in), prof, np.full(M, prof[-1])])
    for c in list(range(M)) + list(range(n - M, n)):
        expect = oracle.weno1d(M, line[c:c + 2 * M + 1])
        for j in range(nt):
            for i in range(nt):
                assert np.array_equal(wh[c, j, i], np.broadcast_to(expect[:, None, None], (N, N, N))), (c, j, i)
