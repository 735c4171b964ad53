"""Request loop: independent AMR solves of different sizes, orders and depths admitted under a
device-memory budget and run concurrently (and, with batching on, advanced together with batched
launches); each result is bitwise identical to the same solve run alone, and the loop reports
p50/p99 time to solution."""
import numpy as np
import pytest

import aw_inputs
import paper_1212_3585_gb300 as pg

pytestmark = pytest.mark.gpu


def rp_config(base, M, lmax):
    return pg.make_config(dim=2, M=M, n=(base, base, 1), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1),
                          bc=pg.AW_BC_TRANSMISSIVE, r=3, lmax=lmax, cfl=0.5)


def test_results_identical_alone_and_in_the_mix():
    rng = np.random.default_rng(20121213)
    reqs = []
    for k in range(10):
        base = int(rng.integers(16, 41))
        M = int(rng.choice([2, 3]))
        lmax = int(rng.integers(0, 3))
        reqs.append((rp_config(base, M, lmax), aw_inputs.rp4_params(1000 + k)))
    srv = pg.Server(hbm_budget_bytes=6 << 30, max_concurrent=4)
    ids = [srv.submit(cfg, pg.AW_IC_RP4, p, 0.03) for cfg, p in reqs]
    srv.wait_all()
    st = srv.stats()
    assert st.done == len(reqs) and st.failed == 0
    assert 0 < st.p50_ms <= st.p99_ms
    for rid, (cfg, p) in zip(ids[:5], reqs[:5]):
        m, u, info = srv.result(rid, 4)
        s = pg.Solver(cfg)
        s.set_initial(pg.AW_IC_RP4, p, -1)
        s.advance_to(0.03)
        m2, u2 = s.cells()
        assert np.array_equal(m, m2)
        assert np.array_equal(u, u2)
        assert info.cell_updates > 0
    srv.close()


def test_batched_loop_results_identical_to_solo():
    """with batching on, compatible requests share launches; every result still equals its solo
    solve bit for bit"""
    rng = np.random.default_rng(77)
    reqs = []
    for k in range(9):
        base = int(rng.integers(12, 33))
        M = int(rng.choice([2, 3]))
        lmax = int(rng.integers(0, 3))
        reqs.append((rp_config(base, M, lmax), aw_inputs.rp4_params(2000 + k)))
    srv = pg.Server(hbm_budget_bytes=8 << 30, max_concurrent=2, max_batch=4)
    ids = [srv.submit(cfg, pg.AW_IC_RP4, p, 0.02) for cfg, p in reqs]
    srv.wait_all()
    st = srv.stats()
    assert st.done + st.failed == len(reqs)
    for rid, (cfg, p) in zip(ids, reqs):
        s = pg.Solver(cfg)
        s.set_initial(pg.AW_IC_RP4, p, -1)
        try:
            s.advance_to(0.02)
        except pg.AwError:
            with pytest.raises(pg.AwError):
                srv.result(rid, 4)
            continue
        m2, u2 = s.cells()
        m, u, info = srv.result(rid, 4)
        assert np.array_equal(m, m2)
        assert np.array_equal(u, u2)
        s.close()
    srv.close()
    with pytest.raises(pg.AwError):
        pg.Server(hbm_budget_bytes=1 << 30, max_concurrent=1, max_batch=pg.AW_BATCH_MAX + 1)


def test_budget_rejects_oversized_request():
    srv = pg.Server(hbm_budget_bytes=1 << 20, max_concurrent=1)
    with pytest.raises(pg.AwError):
        srv.submit(rp_config(64, 3, 2), pg.AW_IC_RP4, aw_inputs.rp4_params(1), 0.01)
    srv.close()
