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
