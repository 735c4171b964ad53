"""The C ABI's argument checks, on the CPU: every call below is rejected with AW_EINVAL and a
message naming the problem before it touches the device (no GPU is needed)."""
import ctypes as C

import pytest

import paper_1212_3585_gb300 as pg
from paper_1212_3585_gb300 import _lib

P, T, R = pg.AW_BC_PERIODIC, pg.AW_BC_TRANSMISSIVE, pg.AW_BC_REFLECTIVE


def create_error(cfg):
    L = _lib.load()
    h = C.c_void_p()
    rc = L.aw_create(C.byref(cfg), 0, C.byref(h))
    return rc, L.aw_last_error().decode(), h.value


BAD_CONFIGS = [
    (dict(dim=1), "dim"),
    (dict(dim=4), "dim"),
    (dict(M=0), "M must"),
    (dict(M=4), "M must"),
    (dict(pde=3), "unknown pde"),
    (dict(pde=-1), "unknown pde"),
    (dict(lmax=-1), "lmax"),
    (dict(lmax=99), "lmax"),
    (dict(lmax=1, r=1), "refine_factor"),
    (dict(lmax=1, M=3, r=2), "refine_factor"),        # r >= M (the child box holds a stencil)
    (dict(lmax=1, r=99), "refine_factor"),
    (dict(n=(0, 8, 1)), "grid size"),
    (dict(n=(8, -1, 1)), "grid size"),
    (dict(dim=3, n=(8, 8, 0)), "grid size"),
    (dict(lo=(0, 1, 0), hi=(1, 1, 1)), "empty domain on axis 1"),
    (dict(lo=(2, 0, 0), hi=(1, 1, 1)), "empty domain on axis 0"),
    (dict(bc=[P, T, P, P, P, P]), "pair up on axis 0"),
    (dict(bc=[T, T, T, P, T, T]), "pair up on axis 1"),
    (dict(bc=[T, T, T, T, 7, T], dim=3, n=(8, 8, 8)), "unknown boundary condition 7"),
    (dict(bc=[R, T, P, P, P, P], pde=pg.AW_PDE_MHD_GLM), "reflective"),
    (dict(cfl=0.0), "cfl"),
    (dict(cfl=float("nan")), "cfl"),
    (dict(flux=5), "unknown numerical flux"),
    (dict(flux=7), "numerical flux"),
    (dict(dim=3, M=3, n=(8, 8, 8)), "not compiled in"),
    (dict(dim=3, pde=pg.AW_PDE_MHD_GLM, n=(8, 8, 8)), "not compiled in"),
    (dict(dim=3, M=1, n=(8, 8, 8)), "not compiled in"),
]


@pytest.mark.parametrize("kw,msg", BAD_CONFIGS, ids=[m + str(i) for i, (_, m) in enumerate(BAD_CONFIGS)])
def test_create_rejects(kw, msg):
    rc, err, h = create_error(pg.make_config(**kw))
    assert rc == _lib.AW_EINVAL and msg in err, (rc, err)
    assert not h                                          # no solver is handed out


def test_create_rejects_null_arguments():
    L = _lib.load()
    h = C.c_void_p()
    assert L.aw_create(None, 0, C.byref(h)) == _lib.AW_EINVAL
    cfg = pg.make_config()
    assert L.aw_create(C.byref(cfg), 0, None) == _lib.AW_EINVAL
    assert "null argument" in L.aw_last_error().decode()


def test_calls_on_a_null_solver():
    L = _lib.load()
    st = pg.AwStats()
    d = C.c_double(0.0)
    checks = [
        L.aw_step(None, 1.0, C.byref(st)),
        L.aw_step_dt(None, 0.1, C.byref(st)),
        L.aw_advance_to(None, 1.0, C.byref(st)),
        L.aw_advance_graph(None, 1.0, 4, C.byref(st)),
        L.aw_compute_dt(None, C.byref(d)),
        L.aw_set_initial(None, pg.AW_IC_CONST, None, 0, 0),
        L.aw_set_cell_averages(None, None, 0),
    ]
    assert all(rc == _lib.AW_EINVAL for rc in checks), checks


def test_batch_rejects_bad_member_lists():
    L = _lib.load()
    st = (pg.AwStats * 1)()
    rc = (C.c_int32 * 1)()
    none = (C.c_void_p * 1)(None)
    assert L.aw_advance_batch(none, 0, 1.0, 0, st, rc) == _lib.AW_EINVAL
    assert L.aw_advance_batch(none, pg.AW_BATCH_MAX + 1, 1.0, 0, st, rc) == _lib.AW_EINVAL
    assert L.aw_advance_batch(none, 1, 1.0, 0, st, rc) == _lib.AW_EINVAL
    assert "null solver 0" in L.aw_last_error().decode()


def test_step_batch_and_graph_stats_reject_bad_arguments():
    L = _lib.load()
    st = (pg.AwStats * 1)()
    rc = (C.c_int32 * 1)()
    none = (C.c_void_p * 1)(None)
    te = (C.c_double * 1)(1.0)
    assert L.aw_step_batch(none, 1, None, 0, st, rc) == _lib.AW_EINVAL
    assert "null end times" in L.aw_last_error().decode()
    assert L.aw_step_batch(none, 0, te, 0, st, rc) == _lib.AW_EINVAL
    assert L.aw_step_batch(none, 1, te, 0, st, rc) == _lib.AW_EINVAL
    assert "null solver 0" in L.aw_last_error().decode()
    v = C.c_int64()
    assert L.aw_graph_stats(None, C.byref(v), None, None) == _lib.AW_EINVAL
    with pytest.raises(ValueError):
        pg.step_batch([], [1.0])


def test_server_rejects_bad_arguments():
    L = _lib.load()
    h = C.c_void_p()
    for budget, workers in ((0, 1), (-5, 1), (1 << 30, 0), (1 << 30, 257)):
        assert L.aw_srv_create(budget, workers, C.byref(h)) == _lib.AW_EINVAL
    assert L.aw_srv_create(1 << 30, 1, None) == _lib.AW_EINVAL
    assert "bad server arguments" in L.aw_srv_last_error().decode()
    assert L.aw_srv_set_batching(None, 2) == _lib.AW_EINVAL
    assert "max_batch" in L.aw_srv_last_error().decode()


def test_noalloc_step_rejects_before_the_device():
    L = _lib.load()
    buf = (C.c_double * 4)()
    cfg = pg.make_config(n=(16, 16, 1))
    # cell count that does not match the grid
    assert L.aw_cfl_dt_noalloc(C.byref(cfg), buf, 100, buf, 0) == _lib.AW_EINVAL
    assert "does not match" in L.aw_last_error().decode()
    # a grid beyond the static scratch (8192 blocks of 256 cells)
    big = pg.make_config(n=(2048, 1025, 1))
    assert L.aw_cfl_dt_noalloc(C.byref(big), buf, 2048 * 1025, buf, 0) == _lib.AW_EINVAL
    assert "at most 2097152 cells" in L.aw_last_error().decode()
    assert L.aw_cfl_dt_noalloc(C.byref(cfg), None, 256, buf, 0) == _lib.AW_EINVAL
    bad = pg.make_config(n=(16, 16, 1), cfl=-1.0)
    assert L.aw_cfl_dt_noalloc(C.byref(bad), buf, 256, buf, 0) == _lib.AW_EINVAL


def test_request_loop_reports_failures_without_a_device():
    """host logic of the request loop on a machine without a usable GPU: an oversized request is
    refused at submission, admitted requests fail alone with AW_ECUDA and a message naming the
    CUDA error, the statistics count them, unknown ids are refused and the loop shuts down"""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: the requests would run")
    except ImportError:
        pass
    import aw_inputs
    srv = pg.Server(hbm_budget_bytes=1 << 20, max_concurrent=2)
    with pytest.raises(pg.AwError) as ei:
        srv.submit(pg.make_config(M=3, n=(64, 64, 1), lmax=2, bc=T), pg.AW_IC_RP4, aw_inputs.rp4_params(1), 0.01)
    assert ei.value.code == _lib.AW_EINVAL and "budget" in str(ei.value)
    srv.close()
    srv = pg.Server(hbm_budget_bytes=1 << 30, max_concurrent=2)
    ids = [srv.submit(pg.make_config(n=(8, 8, 1)), pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], 0.01) for _ in range(3)]
    srv.wait_all()
    assert [srv.poll(i) for i in ids] == [3] * 3                # AW_REQ_FAILED
    with pytest.raises(pg.AwError) as ei:
        srv.result(ids[0], 4)
    assert ei.value.code == _lib.AW_ECUDA and "stream creation failed" in str(ei.value)
    s = srv.stats()
    assert (s.done, s.failed, s.queued, s.running) == (0, 3, 0, 0)
    with pytest.raises(pg.AwError):
        srv.poll(10 ** 6)
    srv.close()


def test_request_loop_under_concurrent_submission_without_a_device():
    """the loop's locking, on the CPU: four threads submit 50 requests each while four workers
    take them (each fails at its stream for want of a device); ids are unique, every request ends
    FAILED, the statistics add up and the loop shuts down"""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: the requests would run")
    except ImportError:
        pass
    import threading
    srv = pg.Server(hbm_budget_bytes=1 << 30, max_concurrent=4)
    ids, lock = [], threading.Lock()

    def submit():
        mine = [srv.submit(pg.make_config(n=(8, 8, 1)), pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], 0.01)
                for _ in range(50)]
        with lock:
            ids.extend(mine)

    threads = [threading.Thread(target=submit) for _ in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    srv.wait_all()
    assert len(ids) == 200 and len(set(ids)) == 200
    assert all(srv.poll(i) == 3 for i in ids)                      # AW_REQ_FAILED
    s = srv.stats()
    assert (s.done, s.failed, s.queued, s.running) == (0, 200, 0, 0)
    srv.close()


def test_batched_request_loop_reports_failures_without_a_device():
    """with batching on, queued requests of one configuration are taken together: without a
    device every member fails with the stream's CUDA error, and all are accounted for"""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: the requests would run")
    except ImportError:
        pass
    srv = pg.Server(hbm_budget_bytes=1 << 30, max_concurrent=2, max_batch=4)
    ids = [srv.submit(pg.make_config(n=(8, 8, 1)), pg.AW_IC_CONST, [1.0, 0.1, 0.2, 1.0], 0.01) for _ in range(9)]
    srv.wait_all()
    assert all(srv.poll(i) == 3 for i in ids)                      # AW_REQ_FAILED
    for i in ids:
        with pytest.raises(pg.AwError) as ei:
            srv.result(i, 4)
        assert ei.value.code == _lib.AW_ECUDA and "stream creation failed" in str(ei.value)
    s = srv.stats()
    assert (s.done, s.failed) == (0, 9)
    srv.close()
