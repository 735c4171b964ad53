"""Pins of the 1D radial reference of the explosion problems (Eq. eq.1D) and, through it, of
the oracle's shocked 2D explosion.

  * planar geometry (d = 1): before the waves reach the centre the solution near r = R is the
    Riemann problem inner|outer, whose exact solution (Toro's pressure iteration, written here
    independently) the second-order TVD scheme must approach at first order in L1;
  * cylindrical/spherical geometry: the radial mass integral is conserved while the shock is
    inside the domain;
  * the 2D ADER-WENO explosion (M=3, Rusanov) on uniform grids converges towards the radial
    reference along the x axis at t = 0.25 (the comparison the paper makes in Sec. 4.1).
"""
import math

import numpy as np
import pytest

import oracle
from tests.polyref import gl01


def exact_riemann(rl, ul, pl, rr, ur, pr, g, xi):
    """Exact solution of the 1D Euler Riemann problem at x/t = xi (Toro, ch. 4)."""
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)

    def f(p, rk, pk, ck):
        if p > pk:
            A, B = 2 / ((g + 1) * rk), (g - 1) / (g + 1) * pk
            return (p - pk) * math.sqrt(A / (p + B)), math.sqrt(A / (p + B)) * (1 - (p - pk) / (2 * (B + p)))
        return 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1), (p / pk) ** (-(g + 1) / (2 * g)) / (rk * ck)

    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dl = f(p, rl, pl, cl)
        fr, dr = f(p, rr, pr, cr)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-14 * p:
            break
    fl, _ = f(p, rl, pl, cl)
    fr, _ = f(p, rr, pr, cr)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    out = np.zeros((len(xi), 3))
    for i, s in enumerate(xi):
        if s <= u:   # left of the contact
            if p > pl:
                sh = ul - cl * math.sqrt((g + 1) / (2 * g) * p / pl + (g - 1) / (2 * g))
                st = (rl * ((p / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pl + 1)), u, p) if s > sh else (rl, ul, pl)
            else:
                cs = cl * (p / pl) ** ((g - 1) / (2 * g))
                if s <= ul - cl:
                    st = (rl, ul, pl)
                elif s >= u - cs:
                    st = (rl * (p / pl) ** (1 / g), u, p)
                else:
                    uu = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    cc = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    st = (rl * (cc / cl) ** (2 / (g - 1)), uu, pl * (cc / cl) ** (2 * g / (g - 1)))
        else:
            if p > pr:
                sh = ur + cr * math.sqrt((g + 1) / (2 * g) * p / pr + (g - 1) / (2 * g))
                st = (rr * ((p / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pr + 1)), u, p) if s < sh else (rr, ur, pr)
            else:
                cs = cr * (p / pr) ** ((g - 1) / (2 * g))
                if s >= ur + cr:
                    st = (rr, ur, pr)
                elif s <= u + cs:
                    st = (rr * (p / pr) ** (1 / g), u, p)
                else:
                    uu = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    cc = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    st = (rr * (cc / cr) ** (2 / (g - 1)), uu, pr * (cc / cr) ** (2 * g / (g - 1)))
        out[i] = st
    return out


def test_planar_reference_approaches_exact_riemann_solution():
    t, R = 0.2, 0.5
    errs = []
    for n in (500, 2000):
        r, rho, u, p = oracle.radial_explosion(1, R=R, n=n, rmax=1.5, t_end=t)
        ex = exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, (r - R) / t)
        errs.append(np.mean(np.abs(rho - ex[:, 0])) * 1.5)
    assert errs[1] < 0.012 and errs[1] < 0.45 * errs[0], errs


@pytest.mark.parametrize("d", [2, 3])
def test_radial_mass_conserved(d):
    n, rmax = 2000, 1.5
    r0, rho0, _, _ = oracle.radial_explosion(d, n=n, rmax=rmax, t_end=1e-12)
    r1, rho1, _, _ = oracle.radial_explosion(d, n=n, rmax=rmax, t_end=0.25)
    dr = rmax / n
    vol = ((r0 + dr / 2) ** d - (r0 - dr / 2) ** d)
    assert np.sum(rho1 * vol) == pytest.approx(np.sum(rho0 * vol), rel=2e-3)


def _explosion_2d_cut(n):
    o = oracle.Oracle(oracle.make_cfg(dim=2, M=3, n=(n, n, 1), lo=(-1, -1, 0), hi=(1, 1, 1),
                                      bc=oracle.BC_TRANSMISSIVE, cfl=0.6), threads=8)
    o.set_initial(oracle.IC_EXPLOSION, [0.5, 1.0, 1.0, 0.125, 0.1])
    while o.t < 0.25:
        rc, _ = o.step(0.25)
        assert rc == 0
    _, u = o.cells()
    rho = u[:, 0].reshape(n, n)
    j = n // 2            # the row just above the x axis
    x = -1 + (np.arange(n) + 0.5) * 2 / n
    y = -1 + (j + 0.5) * 2 / n
    return np.hypot(x, y)[n // 2:], rho[j, n // 2:]


def test_2d_explosion_converges_to_radial_reference():
    r, rho_ref, _, _ = oracle.radial_explosion(2, n=10000, rmax=1.5, t_end=0.25)
    errs = []
    for n in (40, 80):
        rc, rho = _explosion_2d_cut(n)
        ref = np.interp(rc, r, rho_ref)
        errs.append(np.mean(np.abs(rho - ref)))
    assert errs[1] < 0.02 and errs[1] < 0.8 * errs[0], errs
