"""Pins of the oracle's MHD-GLM scheme.  First, an exact nonlinear solution of ideal MHD: the
circularly polarised Alfven wave (constant density 1, pressure 0.1 and normal field B_x = 1;
v_perp = B_perp = 0.1 (sin, cos) of 2 pi x).  With v_perp = +B_perp / sqrt(rho) and B_x > 0 it
travels towards -x at the Alfven speed B_x / sqrt(rho) = 1 without changing shape; the field
stays divergence free, so the GLM cleaning variable psi stays zero.  The cell averages of the
initial data and of the exact solution are computed here in closed form.  Second, the linear
wave of the GLM divergence cleaning (B_x and psi), with d'Alembert's exact solution.
"""
import math

import numpy as np
import pytest

import oracle

GAMMA = 5.0 / 3.0


def alfven_averages(n, ny, shift):
    """cell averages of the wave translated by `shift` (conserved variables, canonical order)"""
    x0, x1 = np.arange(n) / n, (np.arange(n) + 1) / n
    k = 2 * np.pi
    s = (np.cos(k * (x0 - shift)) - np.cos(k * (x1 - shift))) / (k / n)
    c = (np.sin(k * (x1 - shift)) - np.sin(k * (x0 - shift))) / (k / n)
    u = np.zeros((ny, n, 9))
    u[..., 0] = 1.0
    u[..., 2], u[..., 3] = 0.1 * s, 0.1 * c
    u[..., 5] = 1.0
    u[..., 6], u[..., 7] = 0.1 * s, 0.1 * c
    # |v|^2 = |B_perp|^2 = 0.01 at every point, so the energy density is constant
    u[..., 4] = 0.1 / (GAMMA - 1) + 0.5 * 0.01 + 0.5 * (1.0 + 0.01)
    return u.reshape(-1, 9)


def alfven_error(M, n, t_end, flux=0):
    ny = 4
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, M=M, n=(n, ny, 1), lo=(0, 0, 0), hi=(1, ny / n, 1),
                          gamma=GAMMA, c_h=2.0, cfl=0.9, flux=flux)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_CONST, [1.0, 0.0, 0.0, 0.0, 0.1, 1.0, 0.0, 0.0, 0.0], nrefine=0)
    o.set_cell_averages(alfven_averages(n, ny, 0.0))
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    _, u = o.cells()
    ex = alfven_averages(n, ny, -t_end)
    assert np.max(np.abs(u[:, 8])) < 1e-10          # psi stays zero
    return math.sqrt(np.mean((u - ex) ** 2))


@pytest.mark.parametrize("M,lo_order", [(2, 2.7), (3, 3.5)])
def test_circularly_polarised_alfven_wave(M, lo_order):
    """measured orders from 16 to 32 cells at t = 1/4: 2.96 (M=2) and above 5 (M=3)"""
    e = [alfven_error(M, n, 0.25) for n in (16, 32)]
    order = math.log(e[0] / e[1], 2)
    assert order > lo_order, (e, order)
    assert e[1] < 2e-4


CH, DELTA = 2.0, 1e-6


def glm_averages(n, ny, t):
    """cell averages of the linear GLM wave: rho = 1, v = 0, p = 1, B_perp = 0, and
    B_x = DELTA/2 (s(x - c_h t) + s(x + c_h t)), psi = c_h DELTA/2 (s(x - c_h t) - s(x + c_h t))
    with s = sin 2 pi x: d'Alembert's solution of dB_x/dt + dpsi/dx = 0, dpsi/dt + c_h^2 dB_x/dx = 0.
    B_x enters momentum and energy only quadratically (B_x(0) = 0), so they keep their values up
    to DELTA^2."""
    def s(shift):
        x0, x1 = np.arange(n) / n, (np.arange(n) + 1) / n
        k = 2 * np.pi
        return (np.cos(k * (x0 - shift)) - np.cos(k * (x1 - shift))) / (k / n)
    a, b = s(CH * t), s(-CH * t)
    u = np.zeros((ny, n, 9))
    u[..., 0] = 1.0
    u[..., 4] = 1.0 / (GAMMA - 1)
    u[..., 5] = 0.5 * DELTA * (a + b)
    u[..., 8] = 0.5 * CH * DELTA * (a - b)
    return u.reshape(-1, 9)


def glm_errors(M, n, t_end):
    ny = 4
    cfg = oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, M=M, n=(n, ny, 1), lo=(0, 0, 0), hi=(1, ny / n, 1),
                          gamma=GAMMA, c_h=CH, cfl=0.9)
    o = oracle.Oracle(cfg, threads=8)
    o.set_initial(oracle.IC_CONST, [1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0], nrefine=0)
    o.set_cell_averages(glm_averages(n, ny, 0.0))
    while o.t < t_end:
        rc, _ = o.step(t_end)
        assert rc == 0
    _, u = o.cells()
    e = u - glm_averages(n, ny, t_end)
    assert np.max(np.abs(e[:, [0, 1, 2, 3, 4, 6, 7]])) < 1e-11
    return [math.sqrt(np.mean(e[:, v] ** 2)) / DELTA for v in (5, 8)]


@pytest.mark.parametrize("M,lo_order", [(2, 2.7), (3, 3.5)])
def test_glm_cleaning_wave(M, lo_order):
    """the divergence-cleaning part of the MHD-GLM flux, which the Alfven wave (psi = 0,
    div B = 0) leaves untouched: B_x and psi converge to the exact wave at speed c_h (measured
    orders from 16 to 32 cells: 2.98, 4.00 for M=2; 5.38, 4.17 for M=3)"""
    e = [glm_errors(M, n, 0.25) for n in (16, 32)]
    for v in range(2):
        order = math.log(e[0][v] / e[1][v], 2)
        assert order > lo_order, (e, order)
