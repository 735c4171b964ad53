"""Numerical building blocks of the kernels checked against CUDA's own results."""
import numpy as np
import pytest

from paper_1212_3585_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_newton_reciprocal_matches_ieee_division():
    import torch
    L = _lib.load()
    rng = np.random.default_rng(0)
    # densities, sigma + eps of the WENO weights, sums of WENO weights, values near powers of two,
    # and the rest of the normal double range
    x = np.concatenate([rng.uniform(1e-3, 1e3, 200000), 10.0 ** rng.uniform(-14, 6, 200000),
                        10.0 ** rng.uniform(-6, 120, 100000), 2.0 ** np.arange(-40, 40),
                        10.0 ** rng.uniform(-300, 300, 100000), -rng.uniform(1e-3, 1e3, 1000)])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(2 * len(x), dtype=torch.float64, device="cuda")
    _lib.check(L.aw_selftest_reciprocal(xd.data_ptr(), len(x), out.data_ptr(), torch.cuda.current_stream().cuda_stream))
    o = out.cpu().numpy()
    nr, ieee = o[: len(x)], o[len(x):]
    rel = np.abs(nr - ieee) / np.abs(ieee)
    assert rel.max() <= 4 * np.finfo(np.float64).eps, rel.max()


def test_one_step_reciprocal_and_square_root_of_the_face_fluxes():
    """the face fluxes' one-step Newton reciprocal and square root stay within 2^-38 (relative) of
    IEEE division and CUDA's sqrt over the range of densities and squared sound speeds, and the
    square root of zero is (nearly) zero, not NaN"""
    import torch
    L = _lib.load()
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(1e-3, 1e3, 200000), 10.0 ** rng.uniform(-14, 6, 200000),
                        10.0 ** rng.uniform(-200, 200, 200000), 2.0 ** np.arange(-60, 60),
                        1.0 + np.arange(1, 2000) * np.finfo(np.float64).eps])
    xd = torch.from_numpy(x).cuda()
    n = len(x)
    out = torch.empty(4 * n, dtype=torch.float64, device="cuda")
    _lib.check(L.aw_selftest_flux_math(xd.data_ptr(), n, out.data_ptr(), torch.cuda.current_stream().cuda_stream))
    o = out.cpu().numpy()
    rcp1, ieee, sq1, sq = o[:n], o[n:2 * n], o[2 * n:3 * n], o[3 * n:]
    assert np.max(np.abs(rcp1 - ieee) / np.abs(ieee)) <= 2.0 ** -38
    assert np.max(np.abs(sq1 - sq) / sq) <= 2.0 ** -38
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    _lib.check(L.aw_selftest_flux_math(z.data_ptr(), 4, out.data_ptr(), torch.cuda.current_stream().cuda_stream))
    o = out.cpu().numpy()
    assert np.all(np.isfinite(o[8:12])) and np.all(o[8:12] <= 1e-149)
