"""aw_cfl_dt_noalloc: the CFL time step for callers that cannot allocate device memory when they
need it.  Its result must equal the solver's aw_compute_dt on the same averages, on two calls
in a row with different data (the shared scratch array keeps the first call's contents), for the
Euler equations in 2D and 3D, MHD-GLM and linear advection; and it must write the documented
values where aw_compute_dt reports a state it cannot step (0 for NaN averages, at least 1e300 when
no speed limits the step).  Collected last on purpose so that a stop-at-first-failure run has run
everything else first."""
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


def _noalloc(L, cfg, soa, out, stream):
    import torch
    u = torch.from_numpy(np.ascontiguousarray(soa)).cuda()
    out.fill_(-1.0)
    _lib.check(L.aw_cfl_dt_noalloc(C.byref(cfg), u.data_ptr(), u.shape[1], out.data_ptr(), stream.cuda_stream))
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("dim,pde,n", [(2, "euler", (61, 47, 1)), (3, "euler", (13, 11, 9)),
                                       (2, "mhd", (37, 29, 1)), (2, "linadv", (40, 33, 1)),
                                       (3, "linadv", (9, 10, 11))])
def test_noalloc_dt_matches_solver_twice(dim, pde, n):
    import torch
    L = _lib.load()
    code = {"euler": pg.AW_PDE_EULER, "mhd": pg.AW_PDE_MHD_GLM, "linadv": pg.AW_PDE_LINADV}[pde]
    extra = dict(gamma=5.0 / 3.0, c_h=0.5) if pde == "mhd" else {}
    cfg = pg.make_config(dim=dim, pde=code, M=2, n=n, lo=(0, 0, 0), hi=(1.0, 2.0, 1.5), bc=pg.AW_BC_PERIODIC,
                         cfl=0.9, adv=(0.7, -1.3, 0.4), **extra)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (3, 4):          # two calls in a row on different data
        params = aw_inputs.fourier_params(seed=seed, dim=dim, pde=pde, nmodes=4, amp=0.2)
        dt_ref, soa = _solver_dt_and_soa(cfg, params)
        got = _noalloc(L, cfg, soa, out, stream)
        assert abs(got - dt_ref) <= 1e-10 * dt_ref, (got, dt_ref)


def test_noalloc_values_where_the_solver_rejects_the_state():
    import torch
    L = _lib.load()
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    cfg = pg.make_config(dim=2, M=2, n=(20, 18, 1), bc=pg.AW_BC_PERIODIC, cfl=0.9)
    _, soa = _solver_dt_and_soa(cfg, aw_inputs.fourier_params(seed=5, dim=2, pde="euler", nmodes=3, amp=0.2))
    soa[:, 17] = np.nan                       # one cell with NaN averages: 0
    assert _noalloc(L, cfg, soa, out, stream) == 0.0
    # linear advection with a = 0: no speed limits the step
    cfg0 = pg.make_config(dim=2, pde=pg.AW_PDE_LINADV, M=2, n=(16, 16, 1), bc=pg.AW_BC_PERIODIC,
                          adv=(0.0, 0.0, 0.0))
    assert _noalloc(L, cfg0, np.ones((1, 256)), out, stream) >= 1e300
    # and a valid call right after both gives the solver's value again
    params = aw_inputs.fourier_params(seed=6, dim=2, pde="euler", nmodes=3, amp=0.2)
    dt_ref, soa = _solver_dt_and_soa(cfg, params)
    assert abs(_noalloc(L, cfg, soa, out, stream) - dt_ref) <= 1e-10 * dt_ref


def test_noalloc_rejects_oversized_grid():
    L = _lib.load()
    cfg = pg.make_config(dim=2, M=2, n=(2048, 1025, 1))
    rc = L.aw_cfl_dt_noalloc(C.byref(cfg), C.c_void_p(1), 2048 * 1025, C.c_void_p(1), 0)
    assert rc == _lib.AW_EINVAL and b"at most" in L.aw_last_error()
