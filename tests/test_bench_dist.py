"""bench.py on the CPU: the N>1 path (independent replicas, job time = slowest rank; gloo, 2 ranks),
the reference arm's JSON line and the oracle leg of --configs."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)

    def max_reduce(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms = 100.0 + 50.0 * rank        # rank 1 is slower
    value, job_ms = bench.combine_replicas(1_000_000, ms, ws, max_reduce)
    dist.barrier()
    q.put((rank, value, job_ms))
    dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, value, job_ms in res:
        assert job_ms == 150.0
        assert value == pytest.approx(2 * 1_000_000 / 0.150)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0


@pytest.mark.parametrize("workload", ["explosion2d", "explosion3d"])
def test_reference_arm_line(monkeypatch, capsys, workload):
    """rank 0 of the reference arm prints one JSON line with the contract's keys (the 2D oracle on
    a reduced base grid, the 3D one on its 3^3 sample, one step each, to keep the CPU suite short)"""
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", workload]
    if workload == "explosion2d":
        argv += ["--base", "24", "--t-end", "0.01"]
    monkeypatch.setattr("sys.argv", argv)
    # main() rewrites these for a custom base grid and end time: restored after the test
    monkeypatch.setitem(bench.CFG, "n", bench.CFG["n"])
    monkeypatch.setattr(bench, "T_END", bench.T_END)
    monkeypatch.setattr(bench, "WORKLOAD", bench.WORKLOAD)
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["workload"].startswith("3D" if workload == "explosion3d" else "2D")
    if workload == "explosion2d":
        assert "base 24x24" in line["config"]["workload"]


def test_oracle_sample_of_a_configuration():
    """the oracle leg of `bench.py --configs`: cell updates per second over a bounded number of
    level-0 steps, on all host cores"""
    import oracle
    out = bench.oracle_sample(oracle.make_cfg(dim=2, M=2, n=(8, 8, 1), lo=(0, 0, 0), hi=(10, 10, 1), cfl=0.9),
                              oracle.IC_VORTEX, [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0], 3, "three steps")
    assert out["kind"] == "oracle" and out["sample"] == "three steps" and out["cores"] >= 1
    assert out["cell_updates"] == 3 * 64 and out["value"] > 0
