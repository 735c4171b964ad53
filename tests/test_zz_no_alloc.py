"""aw_cfl_dt_noalloc: the CFL time step for callers that cannot allocate device memory when they
need it.  Its result must equal the solver's aw_compute_dt on the same averages, on two calls
in a row with different data (the shared scratch array keeps the first call's contents).
Collected last on purpose so that a stop-at-first-failure run has run everything else first."""
import ctypes as C

import numpy as np
import pytest

import aw_inputs
import paper_1212_3585_gb300 as pg
from paper_1212_3585_gb300 import _lib

pytestmark = pytest.mark.gpu


def _solver_dt_and_soa(cfg, params):
    s = pg.Solver(cfg)
    s.set_initial(pg.AW_IC_FOURIER, params, 0)
    dt = s.compute_dt()
    _, u = s.cells()            # level 0 only: canonical order = (k, j, i)
    s.close()
    return dt, np.ascontiguousarray(u.T)


@pytest.mark.parametrize("dim,n", [(2, (61, 47, 1)), (3, (13, 11, 9))])
def test_noalloc_dt_matches_solver_twice(dim, n):
    import torch
    L = _lib.load()
    cfg = pg.make_config(dim=dim, M=2, n=n, lo=(0, 0, 0), hi=(1.0, 2.0, 1.5), bc=pg.AW_BC_PERIODIC, cfl=0.9)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (3, 4):          # two calls in a row on different data
        params = aw_inputs.fourier_params(seed=seed, dim=dim, pde="euler", nmodes=4, amp=0.2)
        dt_ref, soa = _solver_dt_and_soa(cfg, params)
        u = torch.from_numpy(soa).cuda()
        out.fill_(-1.0)
        _lib.check(L.aw_cfl_dt_noalloc(C.byref(cfg), u.data_ptr(), u.shape[1], out.data_ptr(), stream.cuda_stream))
        torch.cuda.synchronize()
        assert abs(out.item() - dt_ref) <= 1e-10 * dt_ref, (out.item(), dt_ref)


def test_noalloc_rejects_oversized_grid():
    L = _lib.load()
    cfg = pg.make_config(dim=2, M=2, n=(2048, 1025, 1))
    rc = L.aw_cfl_dt_noalloc(C.byref(cfg), C.c_void_p(1), 2048 * 1025, C.c_void_p(1), 0)
    assert rc == _lib.AW_EINVAL and b"at most" in L.aw_last_error()
