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


def ot_config(base, lmax):
    """MHD-GLM Orszag-Tang type data on the periodic [0, 2 pi]^2 (gamma 5/3, M = 3)"""
    return pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=3, n=(base, base, 1), lo=(0, 0, 0),
                          hi=(2 * np.pi, 2 * np.pi, 1), bc=pg.AW_BC_PERIODIC, gamma=5.0 / 3.0, r=3, lmax=lmax,
                          cfl=0.6, c_h=2.0, chi_ref=0.05, chi_rec=0.02)


def solo(cfg, ic, p, t_end):
    s = pg.Solver(cfg)
    s.set_initial(ic, p, -1)
    s.advance_to(t_end)
    out = s.cells()
    s.close()
    return out


def test_results_identical_alone_and_in_the_mix():
    """Euler and MHD-GLM requests of different sizes, orders and depths"""
    rng = np.random.default_rng(20121213)
    reqs = []
    for k in range(10):
        base = int(rng.integers(16, 41))
        M = int(rng.choice([2, 3]))
        lmax = int(rng.integers(0, 3))
        reqs.append((rp_config(base, M, lmax), pg.AW_IC_RP4, aw_inputs.rp4_params(1000 + k)))
    for base, lmax in ((16, 1), (20, 0), (24, 1)):
        reqs.append((ot_config(base, lmax), pg.AW_IC_OT, []))
    order = rng.permutation(len(reqs))
    reqs = [reqs[i] for i in order]
    srv = pg.Server(hbm_budget_bytes=6 << 30, max_concurrent=4)
    ids = [srv.submit(cfg, ic, p, 0.03) for cfg, ic, p in reqs]
    srv.wait_all()
    st = srv.stats()
    assert st.done == len(reqs) and st.failed == 0
    assert 0 < st.p50_ms <= st.p99_ms
    assert st.peak_reserved_bytes <= st.budget_bytes == 6 << 30
    checked_mhd = 0
    for k, (rid, (cfg, ic, p)) in enumerate(zip(ids, reqs)):
        if k >= 5 and ic != pg.AW_IC_OT:
            continue
        V = 9 if ic == pg.AW_IC_OT else 4
        m, u, info = srv.result(rid, V)
        m2, u2 = solo(cfg, ic, p, 0.03)
        assert np.array_equal(m, m2)
        assert np.array_equal(u, u2)
        assert info.cell_updates > 0
        checked_mhd += ic == pg.AW_IC_OT
    assert checked_mhd == 3
    srv.close()


VORTEX = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]


def full_refinement_config(base=24):
    """the vortex refined everywhere to l_max = 2 (every indicator value is above chi_ref = -1):
    its finest level is fully active, four times what a first reservation allows for"""
    return pg.make_config(dim=2, M=2, n=(base, base, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc=pg.AW_BC_PERIODIC,
                          r=3, lmax=2, cfl=0.9, chi_ref=-1.0, chi_rec=-2.0)


def test_solver_memory_limit():
    cfg = full_refinement_config()
    ref = pg.Solver(cfg)
    ref.set_initial(pg.AW_IC_VORTEX, VORTEX, -1)
    ref.advance_to(0.1)
    m0, u0 = ref.cells()
    live, peak, refused = ref.memory()
    assert refused == 0 and 0 < live <= peak
    assert m0[:, 0].max() == 2 and np.all(m0[m0[:, 1] == 0, 0] == 2)   # every active cell on level 2
    ref.close()
    s = pg.Solver(cfg)
    s.set_memory_limit(peak // 2)
    with pytest.raises(pg.AwError) as ei:
        s.set_initial(pg.AW_IC_VORTEX, VORTEX, -1)
        s.advance_to(0.1)
    assert ei.value.code == pg._lib.AW_ELIMIT
    live2, peak2, refused2 = s.memory()
    assert peak2 <= peak // 2 < refused2
    # the solve restarts from its initial condition once the limit is lifted
    s.reset()
    s.set_memory_limit(0)
    assert s.memory()[2] == 0
    s.set_initial(pg.AW_IC_VORTEX, VORTEX, -1)
    s.advance_to(0.1)
    m, u = s.cells()
    assert np.array_equal(m, m0) and np.array_equal(u, u0)
    with pytest.raises(pg.AwError) as ei:
        s.set_memory_limit(-1)
    assert ei.value.code == pg._lib.AW_EINVAL
    s.close()


@pytest.mark.parametrize("max_batch", [1, 2])
def test_request_outgrowing_its_reservation_waits_and_completes(max_batch):
    """Two requests whose meshes refine everywhere (four times the first reservation) under a
    budget that holds one grown reservation but not two: a refused one goes back to the head of the
    queue with a larger reservation, waits for the other, and completes with the result of its solo
    solve; the reservations of running requests never exceed the budget.  A request of the same
    kind submitted afterwards starts with the share of the finest level the loop has learned and
    runs without a requeue."""
    cfg = full_refinement_config()
    ref = pg.Solver(cfg)
    ref.set_initial(pg.AW_IC_VORTEX, VORTEX, -1)
    ref.advance_to(0.1)
    m0, u0 = ref.cells()
    peak = ref.memory()[1]
    ref.close()
    small = rp_config(16, 2, 1)
    ps = aw_inputs.rp4_params(31)
    m1, u1 = solo(small, pg.AW_IC_RP4, ps, 0.1)
    budget = int(1.6 * (peak + (64 << 20)))
    srv = pg.Server(hbm_budget_bytes=budget, max_concurrent=3, max_batch=max_batch)
    ids = [srv.submit(cfg, pg.AW_IC_VORTEX, VORTEX, 0.1), srv.submit(small, pg.AW_IC_RP4, ps, 0.1),
           srv.submit(cfg, pg.AW_IC_VORTEX, VORTEX, 0.1)]
    srv.wait_all()
    st = srv.stats()
    assert st.done == 3 and st.failed == 0
    assert st.requeues >= 1
    assert st.peak_reserved_bytes <= budget
    for rid in (ids[0], ids[2]):
        m, u, info = srv.result(rid, 4)
        assert np.array_equal(m, m0) and np.array_equal(u, u0)
        assert info.peak_bytes + (64 << 20) <= info.footprint_bytes <= budget
    assert srv.result(ids[0], 4)[2].requeues + srv.result(ids[2], 4)[2].requeues >= 1
    m, u, info = srv.result(ids[1], 4)
    assert np.array_equal(m, m1) and np.array_equal(u, u1)
    late = srv.submit(cfg, pg.AW_IC_VORTEX, VORTEX, 0.1)
    srv.wait_all()
    m, u, info = srv.result(late, 4)
    assert np.array_equal(m, m0) and np.array_equal(u, u0)
    assert info.requeues == 0 and srv.stats().peak_reserved_bytes <= budget
    srv.close()


@pytest.mark.parametrize("max_batch", [1, 2])
def test_request_outgrowing_its_reservation_grows_in_place(max_batch):
    """Requests whose meshes refine everywhere (four times the first reservation) under a budget
    with room for their growth: each reservation grows in place while the solve runs, nothing is
    queued again, the reservations held never exceed the budget, and the results are the solo
    solve's."""
    cfg = full_refinement_config()
    m0, u0 = solo(cfg, pg.AW_IC_VORTEX, VORTEX, 0.1)
    srv = pg.Server(hbm_budget_bytes=16 << 30, max_concurrent=2, max_batch=max_batch)
    ids = [srv.submit(cfg, pg.AW_IC_VORTEX, VORTEX, 0.1) for _ in range(2)]
    srv.wait_all()
    st = srv.stats()
    assert st.done == 2 and st.failed == 0
    assert st.requeues == 0 and st.grows >= 2
    assert st.peak_reserved_bytes <= st.budget_bytes
    for rid in ids:
        m, u, info = srv.result(rid, 4)
        assert np.array_equal(m, m0) and np.array_equal(u, u0)
        assert info.requeues == 0 and info.grows >= 1
        assert info.peak_bytes + (64 << 20) <= info.footprint_bytes
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


def test_continuous_batching_members_leave_and_join():
    """continuous batching on one worker: requests of one kernel configuration with different end
    times and grids share a group, each leaves it when it reaches its own end time (so the earlier
    ones are done before the group ends), a request submitted while the group runs joins it at a
    step boundary instead of waiting for the group to end, and every result equals its solo solve
    bit for bit"""
    import time
    reqs = [(rp_config(40, 2, 1), aw_inputs.rp4_params(501), 0.03),
            (rp_config(24, 2, 1), aw_inputs.rp4_params(502), 0.12),
            (rp_config(32, 2, 1), aw_inputs.rp4_params(503), 0.25)]
    late = (rp_config(20, 2, 1), aw_inputs.rp4_params(504), 0.05)
    # the solo solves first (they also load every kernel the loop will launch)
    ref = [solo(c, pg.AW_IC_RP4, p, te) for c, p, te in reqs + [late]]
    srv = pg.Server(hbm_budget_bytes=8 << 30, max_concurrent=1, max_batch=4)
    t0 = time.monotonic()
    ids = [srv.submit(c, pg.AW_IC_RP4, p, te) for c, p, te in reqs]
    time.sleep(0.05)
    t_late = time.monotonic() - t0
    lid = srv.submit(late[0], pg.AW_IC_RP4, late[1], late[2])
    srv.wait_all()
    st = srv.stats()
    assert st.done == 4 and st.failed == 0
    infos = []
    for rid, (m0, u0) in zip(ids + [lid], ref):
        m, u, info = srv.result(rid, 4)
        assert np.array_equal(m, m0) and np.array_equal(u, u0)
        infos.append(info)
    done = [i.total_ms for i in infos[:3]]          # the first three were submitted together
    assert done[0] < done[2] and done[1] < done[2]
    # the late request started before the group's last member finished: it joined the group
    assert t_late * 1e3 + infos[3].queue_ms < done[2]
    assert infos[3].queue_ms < 0.5 * (done[2] - t_late * 1e3)
    srv.close()


def test_step_batch_equals_solo_steps():
    """aw_step_batch: one lockstep level-0 step of each member not yet at its own end time, each
    member's step exactly its own aw_step; members at their end time are left as they are"""
    cfgs = [rp_config(20, 3, 2), rp_config(28, 3, 1), rp_config(16, 3, 0)]
    ps = [aw_inputs.rp4_params(600 + k) for k in range(3)]
    ends = [0.02, 0.05, 0.08]
    sol, ref = [], []
    for c, p in zip(cfgs, ps):
        for lst in (sol, ref):
            s = pg.Solver(c)
            s.set_initial(pg.AW_IC_RP4, p, -1)
            lst.append(s)
    steps = 0
    while any(s.t < te for s, te in zip(sol, ends)):
        before = [s.t for s in sol]
        st, rc = pg.step_batch(sol, ends)
        assert rc == [0, 0, 0]
        for k in range(3):
            if before[k] < ends[k]:
                one = ref[k].step(ends[k])
                assert st[k].level0_steps == 1 and st[k].cell_updates == one.cell_updates
                assert st[k].t == ref[k].t
            else:
                assert st[k].level0_steps == 0 and sol[k].t == before[k]
        steps += 1
    assert steps >= 3
    for a, b in zip(sol, ref):
        ma, ua = a.cells()
        mb, ub = b.cells()
        assert np.array_equal(ma, mb) and np.array_equal(ua, ub)
        a.close()
        b.close()


def test_budget_rejects_oversized_request():
    srv = pg.Server(hbm_budget_bytes=1 << 20, max_concurrent=1)
    with pytest.raises(pg.AwError):
        srv.submit(rp_config(64, 3, 2), pg.AW_IC_RP4, aw_inputs.rp4_params(1), 0.01)
    srv.close()
