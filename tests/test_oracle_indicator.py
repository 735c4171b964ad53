"""Pins of the oracle's refinement indicator (Sec. 3.1.1, Eq. eqn.indicator: Loehner's normalised
second derivative of Phi = the first conserved variable, with the noise filter eps = 0.01) by
properties that any correct form of it has, not by its formula:

  * it vanishes on data that are linear in the cell indices (second differences are zero);
  * it depends on Phi only up to a factor (homogeneous of degree 0) and lies in [0, 1]
    (a second difference is bounded by the sum of the first differences);
  * at a jump it is of order one on every grid, on smooth data it falls at least like h;
  * the filter: ripples far below the background level stay below chi_ref, the same ripples
    around zero reach 1;
  * mixed second derivatives count: Phi = i j (no pure second difference) gives chi > 0;
  * it is invariant under exchanging the axes and under mirroring;
  * the flags refine exactly the cells whose 3^d neighbourhood holds a cell above chi_ref.
"""
import numpy as np
import pytest

import oracle

EPS = 0.01


def chi_field(phi, dim=2, bc=oracle.BC_PERIODIC, eps=EPS, lmax=0):
    """indicator of every cell of a uniform grid whose first variable is phi (shape (nz,) ny, nx)"""
    shape = phi.shape
    n = (shape[-1], shape[-2], shape[0] if dim == 3 else 1)
    cfg = oracle.make_cfg(dim=dim, pde=oracle.PDE_LINADV, M=2, n=n, bc=bc, eps_ind=eps, lmax=lmax, r=3,
                          auto_regrid=0)
    o = oracle.Oracle(cfg)
    o.set_initial(oracle.IC_CONST, [0.0], nrefine=0)
    o.set_cell_averages(phi.reshape(-1, 1))
    chi = np.zeros(shape)
    for idx in np.ndindex(*shape):
        if dim == 2:
            chi[idx] = o.indicator_at(0, idx[1], idx[0])
        else:
            chi[idx] = o.indicator_at(0, idx[2], idx[1], idx[0])
    return chi, o


def test_linear_data_give_zero():
    j, i = np.mgrid[0:12, 0:14].astype(float)
    chi, _ = chi_field(3.0 + i / 8 - j / 16, bc=oracle.BC_TRANSMISSIVE)
    assert np.all(chi[1:-1, 1:-1] == 0.0)
    k, j, i = np.mgrid[0:6, 0:7, 0:8].astype(float)
    chi3, _ = chi_field(1.0 + i / 4 + j / 8 - k / 2, dim=3, bc=oracle.BC_TRANSMISSIVE)
    assert np.all(chi3[1:-1, 1:-1, 1:-1] == 0.0)


def test_homogeneous_and_bounded():
    rng = np.random.default_rng(11)
    phi = rng.standard_normal((10, 12))
    chi, _ = chi_field(phi)
    chi7, _ = chi_field(-7.3 * phi)
    assert np.all(chi >= 0.0) and np.all(chi <= 1.0)
    assert np.allclose(chi7, chi, rtol=1e-14, atol=0)
    chi0, _ = chi_field(phi, eps=0.0)
    assert np.all(chi0 <= 1.0 + 1e-15) and np.all(chi0 >= chi)


def test_jump_order_one_smooth_order_h():
    """peaks at the jump stay put; on the sine wave the largest value falls by 0.36 and 0.28 per
    halving of h here (like h where G dominates eps A, like h^2 once eps A does)"""
    peaks, smooth = [], []
    for n in (32, 64, 128):
        x = (np.arange(n) + 0.5) / n
        step = np.tile(np.where(x > 0.5, 2.0, 1.0), (4, 1))
        peaks.append(chi_field(step, bc=oracle.BC_TRANSMISSIVE)[0].max())
        wave = np.tile(2.0 + np.sin(2 * np.pi * x), (4, 1))
        smooth.append(chi_field(wave)[0].max())
    assert min(peaks) > 0.5 and max(peaks) - min(peaks) < 1e-12, peaks
    assert smooth[2] < 0.05 and smooth[1] < 0.6 * smooth[0] and smooth[2] < 0.6 * smooth[1], smooth


def test_noise_filter():
    i = np.arange(16)
    ripple = np.tile(1e-3 * (-1.0) ** i, (4, 1))
    on_background, _ = chi_field(100.0 + ripple)
    around_zero, _ = chi_field(ripple)
    assert on_background.max() < 0.2
    assert around_zero.max() > 0.9


def test_mixed_derivative_counts():
    j, i = np.mgrid[0:10, 0:10].astype(float)
    chi, _ = chi_field(i * j, bc=oracle.BC_TRANSMISSIVE)
    assert np.all(chi[1:-1, 1:-1] > 0.0)


def test_axis_exchange_and_mirror():
    rng = np.random.default_rng(12)
    phi = rng.uniform(0.5, 1.5, (9, 11))
    chi, _ = chi_field(phi, bc=oracle.BC_TRANSMISSIVE)
    chi_t, _ = chi_field(phi.T.copy(), bc=oracle.BC_TRANSMISSIVE)
    chi_m, _ = chi_field(phi[:, ::-1].copy(), bc=oracle.BC_TRANSMISSIVE)
    assert np.allclose(chi_t.T, chi, rtol=1e-14, atol=0)
    assert np.allclose(chi_m[:, ::-1], chi, rtol=1e-14, atol=0)
    phi3 = rng.uniform(0.5, 1.5, (5, 6, 7))
    c3, _ = chi_field(phi3, dim=3, bc=oracle.BC_TRANSMISSIVE)
    c3t, _ = chi_field(phi3.transpose(2, 1, 0).copy(), dim=3, bc=oracle.BC_TRANSMISSIVE)
    assert np.allclose(c3t.transpose(2, 1, 0), c3, rtol=1e-14, atol=0)


def test_flags_are_the_neighbourhood_maximum_above_chi_ref():
    rng = np.random.default_rng(13)
    phi = 1.0 + (rng.uniform(size=(12, 12)) < 0.08)         # isolated jumps on a flat field
    chi, o = chi_field(phi, lmax=1)
    flags = o.compute_flags().reshape(12, 12)
    pad = np.pad(chi, 1, mode="wrap")                       # periodic neighbourhoods
    hat = np.max([pad[1 + dj:13 + dj, 1 + di:13 + di] for dj in (-1, 0, 1) for di in (-1, 0, 1)], axis=0)
    assert np.array_equal(flags, (hat > 0.2).astype(np.int8))
    assert 0 < np.count_nonzero(flags) < 144
