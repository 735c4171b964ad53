#!/usr/bin/env python
"""Benchmark: ADER-WENO cell-updates/s on the 2D AMR explosion workload.

Workload (one "step" = one complete solve): 2D Euler, gamma 1.4, FP64, ADER-WENO M=3 (fourth
order), base grid 100x100 on [-1,1]^2, refinement factor 3, l_max = 2, local time stepping,
Loehner density indicator, cylindrical explosion (rho=1, p=1 inside r=0.5; rho=0.125, p=0.1
outside), transmissive boundaries, Rusanov flux, CFL 0.6, from t=0 to t=0.25.  Each solve
re-initialises the mesh on the device (aw_reset + initial condition + l_max refinement passes)
and advances to t_end with a regrid after every level-0 step.

value   = cell updates (active cell advanced by its level's dt) per second, device-resident
e2e     = the same through the C ABI with host buffers: level-0 averages uploaded from pinned
          host memory, data-driven refinement, solve, all cell averages read back
roofline= the dominant kernel's algorithmic FP64 FLOP rate against the FP64 peak
cpu_baseline = the FP64 CPU oracle on all host cores, on the first four level-0 steps of the same
          solve (and on one core, on the first level-0 step)

Multi-GPU: one independent replica per rank (the path has no exchange step), weak scaling.

Other modes (one JSON line each, not the benchmark line): --serve (request loop, with and without
cross-request batching, against one-at-a-time solves), --efficiency (cost per cell update of
orders 2-4, uniform against AMR), --configs (throughput of the other configurations), --tune (the
launch-shape rules timed one at a time).
"""
import argparse
import ctypes as C
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADER-WENO cell-updates/s vs roofline; batched solves/s + p99 latency vs plain"
UNIT = "cell-updates/s"
WORKLOAD = ("2D Euler FP64, ADER-WENO M=3, base 100x100 on [-1,1]^2, r=3, l_max=2, local time stepping, "
            "cylindrical explosion (R=0.5; rho,p = 1,1 inside; 0.125,0.1 outside), transmissive, "
            "Rusanov, CFL 0.6, t_end=0.25")
CFG = dict(dim=2, M=3, n=(100, 100, 1), lo=(-1.0, -1.0, 0.0), hi=(1.0, 1.0, 1.0), r=3, lmax=2, gamma=1.4,
           chi_ref=0.2, chi_rec=0.1, cfl=0.6)
T_END = 0.25
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2      # sm_103a: measured 0.598 T DFMA/s at ~1.97 GHz on 152 SMs
SM_MAX_MHZ = 2070.0
HBM_GBS = 6792.1                 # measured copy bandwidth of this GB300 pool
# DRAM bytes per cell of k_predict<2,3,Euler> from one ncu capture of a full-size level-2 launch
# of this workload (6264 CTAs x 16 cells: dram__bytes_read.sum 51.36 MB + dram__bytes_write.sum
# 141.52 MB); scaled by the cells of an average launch.  Must be re-captured whenever k_predict
# changes.
PREDICTOR_DRAM_BYTES_PER_CELL = (51356416 + 141521408) / (6264 * 16)


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return HBM_GBS
FP64_PEAK_TFLOPS = 2 * FP64_FMA_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12   # 1.2586


def predictor_flops_per_cell(D, M, V, P, flux_flops):
    """Algorithmic FP64 FLOPs of the space-time predictor per cell update in its factorised form
    (FMA = 2): flux evaluations at the nodes, spatial derivative contractions, time contraction;
    the first Picard iteration starts from a state constant in time."""
    N = M + 1
    nsp, nst = N ** D, N ** (D + 1)
    first = nsp * flux_flops + nsp * V * D * N * 2 + nst * V * 2
    later = nst * flux_flops + nst * V * D * N * 2 + nst * V * N * 2
    return first + (P - 1) * later


# FP64 operations of the Euler fluxes in all D directions at one state (1/rho, velocities,
# kinetic energy, pressure, E+p, then D*(D+2) components)
EULER_FLUX_FLOPS = {2: 18, 3: 25}
# MHD-GLM fluxes in both 2D directions at one state: shared primitives 1/rho, v, |B|^2, rho|v|^2, p,
# v.B, p + |B|^2/2, c_h^2 (28), then per direction momentum (10), energy (4), induction (6) and
# cleaning (1) components (21)
MHD_FLUX_FLOPS_2D = 28 + 2 * 21


def weno_flops_per_cell(D, M, V):
    """Algorithmic FP64 FLOPs of the dimension-by-dimension WENO per cell: one 1D reconstruction
    per variable on each of the N^(a) lines of sweep a (1 in x, N in y, N^2 in z), each with
    N_s stencils of N-1 differences (stencil product, sigma as a quadratic form, weight) and
    the normalised combination.  Halo sweeps a tile recomputes are overhead, not counted."""
    N = M + 1
    ns = 3 if M % 2 == 0 else 4
    per_stencil = 2 * (N - 1) * N + 2 * ((N - 1) * N // 2 + (N - 1)) + 5 + 2 * N
    per_recon = ns * per_stencil + ns + 1 + 2 * N
    lines = sum(N ** a for a in range(D))
    return per_recon * lines * V


def flux_flops_per_cell(D, M, V):
    """Algorithmic FP64 FLOPs of the face fluxes per cell: D owned faces of N^D space-time Gauss
    points; two traces (N-term contractions), the Euler flux and spectral radius of both states,
    the Rusanov combination and the quadrature weight."""
    N = M + 1
    per_state = 1 + 2 * D + 6 + 2 * D + 4 + 1 + 2
    per_point = 2 * V * N * 2 + 2 * per_state + 3 * V + V
    return D * N ** D * per_point


def bytes_per_cell(D, M, V):
    """Algorithmic HBM bytes per cell update of each kernel (every array read or written once)."""
    N = M + 1
    wh, qh, fl = V * N ** D * 8, V * N ** (D + 1) * 8, 2 * D * V * 8
    return {"weno": V * 8 + wh, "predictor": wh + qh, "face_flux": qh + fl}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()

    def summary(self):
        self.f.seek(0)
        rows = [ln.strip().split(", ") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def combine_replicas(updates, ms, world_size, max_reduce):
    """Whole-job throughput of independent replicas: every rank did `updates` cell updates in
    `ms`; the job time is the slowest rank's."""
    job_ms = max_reduce(ms)
    return world_size * updates / (job_ms * 1e-3), job_ms


def serve_requests(n, base_max, seed=20121213, base_min=32, lmax_max=2):
    """Seeded stream shaped like the serving workload: 2D Euler four-quadrant Riemann problems on
    [-0.5, 0.5]^2, base grid uniform in base_min..base_max, M in {2, 3}, l_max in 0..lmax_max,
    r = 3, per-quadrant rho, p ~ U[0.1, 1.5], u, v ~ U[-1, 1] (aw_inputs.rp4_params)."""
    import numpy as np
    import aw_inputs
    import paper_1212_3585_gb300 as pg
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        base = int(rng.integers(base_min, base_max + 1))
        M = int(rng.choice([2, 3]))
        lmax = int(rng.integers(0, lmax_max + 1))
        cfg = pg.make_config(dim=2, M=M, n=(base, base, 1), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1),
                             bc=pg.AW_BC_TRANSMISSIVE, r=3, lmax=lmax, cfl=0.5)
        out.append((cfg, aw_inputs.rp4_params(seed + k)))
    return out


def run_serve(args):
    """Continuous admission (aw_srv_*, concurrent requests on their own streams), with and without
    cross-request batching, against one-at-a-time plain solves, on the same seeded requests and
    arrival times."""
    import threading
    import numpy as np
    import torch
    import paper_1212_3585_gb300 as pg
    torch.cuda.set_device(0)
    reqs = serve_requests(args.requests, args.serve_base_max, base_min=args.serve_base_min,
                          lmax_max=args.serve_lmax_max)
    t_end = args.serve_t_end

    def plain(arrivals):
        t0 = time.perf_counter()
        tts, done, upd, failed = [], 0.0, 0, 0
        for (cfg, p), a in zip(reqs, arrivals):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            s = pg.Solver(cfg)
            try:
                s.set_initial(pg.AW_IC_RP4, p, -1)
                st = s.advance_to(t_end)
                s.cells()
                upd += st.cell_updates
                ok = True
            except pg.AwError:
                ok = False    # a request whose solution leaves the physical states fails, as in the loop
            s.close()
            done = time.perf_counter() - t0
            if ok:
                tts.append(1e3 * (done - a))
            else:
                failed += 1
        return {"solves_per_s": len(tts) / done, "p50_ms": float(np.percentile(tts, 50)),
                "p99_ms": float(np.percentile(tts, 99)), "cell_updates_per_s": upd / done, "failed": failed}

    def loop(arrivals, max_batch=1):
        srv = pg.Server(hbm_budget_bytes=int(args.serve_budget_gb * (1 << 30)), max_concurrent=args.concurrency,
                        max_batch=max_batch)
        t0 = time.perf_counter()
        ids = []
        for (cfg, p), a in zip(reqs, arrivals):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            ids.append(srv.submit(cfg, pg.AW_IC_RP4, p, t_end))
        srv.wait_all()
        st = srv.stats()
        out = {"solves_per_s": st.solves_per_s, "p50_ms": st.p50_ms, "p99_ms": st.p99_ms,
               "cell_updates_per_s": st.cell_updates_per_s, "failed": int(st.failed)}
        srv.close()
        return out

    burst = [0.0] * len(reqs)
    B = args.serve_batch
    res = {"burst": {"plain": plain(burst), "loop": loop(burst), f"loop_batch{B}": loop(burst, B)}}
    lam = 0.8 * max(res["burst"]["loop"]["solves_per_s"], res["burst"][f"loop_batch{B}"]["solves_per_s"])
    rng = np.random.default_rng(7)
    arr = list(np.cumsum(rng.exponential(1.0 / lam, len(reqs))))
    res["poisson"] = {"rate_per_s": lam, "plain": plain(arr), "loop": loop(arr), f"loop_batch{B}": loop(arr, B)}
    print(json.dumps({"metric": "request-loop solves/s + p50/p99 time to solution vs plain", "unit": "solves/s",
                      "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"{len(reqs)} 2D Euler four-quadrant Riemann AMR solves, "
                                             f"base {args.serve_base_min}..{args.serve_base_max}, M in {{2,3}}, "
                                             f"l_max in 0..{args.serve_lmax_max}, r=3, CFL 0.5, t_end={t_end}",
                                 "concurrency": args.concurrency, "budget_gb": args.serve_budget_gb, "batch": args.serve_batch},
                      **res}))
    return 0


def run_efficiency(args):
    """Cost per cell update of the second- to fourth-order schemes (M = 1, 2, 3) on a uniform
    grid and on the AMR grid (r = 4, l_max = 2) of the 2D explosion, normalised by the
    second-order scheme on the uniform grid: the measurement of the paper's Sec. 3.2 efficiency
    table (whole solve, ghost projection, averaging and regrid included) on this GPU."""
    import torch
    import aw_inputs
    import paper_1212_3585_gb300 as pg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    B, r, lmax = args.eff_base, 4, 2
    rows = []
    for M in (1, 2, 3):
        for grid in ("uniform", "amr"):
            n = B * r ** lmax if grid == "uniform" else B
            cfg = pg.make_config(dim=2, M=M, n=(n, n, 1), lo=(-1.0, -1.0, 0.0), hi=(1.0, 1.0, 1.0),
                                 bc=pg.AW_BC_TRANSMISSIVE, r=r, lmax=0 if grid == "uniform" else lmax,
                                 cfl=0.6, auto_regrid=1)
            s = pg.Solver(cfg, stream.cuda_stream)
            times, upd = [], 0
            for i in range(args.warmup + args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                s.reset()
                s.set_initial(pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, -1)
                st = s.advance_to(args.eff_t_end)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    times.append(e0.elapsed_time(e1))
                    upd += st.cell_updates
            s.close()
            ns = 1e6 * sum(times) / upd
            rows.append({"order": M + 1, "M": M, "grid": grid, "ns_per_cell_update": ns,
                         "cell_updates_per_solve": upd // args.steps, "ms_per_solve": sum(times) / len(times)})
    ref = rows[0]["ns_per_cell_update"]
    table = {}
    for M in (1, 2, 3):
        u = next(x for x in rows if x["M"] == M and x["grid"] == "uniform")["ns_per_cell_update"]
        a = next(x for x in rows if x["M"] == M and x["grid"] == "amr")["ns_per_cell_update"]
        table[f"O{M + 1}"] = {"uniform": u / ref, "amr": a / ref, "amr_overhead_pct": 100 * (a / u - 1)}
    print(json.dumps({"metric": "normalised time per cell update (second-order uniform = 1)", "unit": "ratio",
                      "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"2D Euler explosion, [-1,1]^2, CFL 0.6, t_end={args.eff_t_end}; "
                                             f"AMR: base {B}x{B}, r={r}, l_max={lmax}; uniform: {B * r ** lmax}^2",
                                 "steps": args.steps, "warmup": args.warmup},
                      "table": table, "rows": rows}))
    return 0


def oracle_sample(ocfg, ic, params, steps, sample):
    """The FP64 CPU oracle as it stands on all host cores: cell updates per second over `steps`
    level-0 steps after the initial condition and its refinement passes"""
    import oracle
    threads = os.cpu_count() or 1
    o = oracle.Oracle(ocfg, threads=threads)
    o.set_initial(ic, params)
    n0 = o.updates()[0]
    t0 = time.perf_counter()
    for _ in range(steps):
        rc, _ = o.step()
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")
    el = time.perf_counter() - t0
    n = o.updates()[0] - n0
    return {"value": n / el, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
            "cell_updates": int(n), "seconds": el}


def run_configs(args):
    """Throughput of the other configurations (one JSON line each, device time with CUDA events on
    the solver's stream, after a warm-up solve): the vortex at 32^2 (20 steps) and its labelled
    scaled variants at 1024^2 and 2048^2, the 3D explosion (64^3 base, l_max = 2) on a time-boxed
    sample of level-0 steps after the initial refinement, and the MHD Orszag-Tang run to t = 0.5.
    Unless --no-cpu-baseline, each line is followed by the oracle's rate on a bounded sample of the
    same configuration (host cores, stated in the line)."""
    import numpy as np
    import torch
    import aw_inputs
    import oracle
    import paper_1212_3585_gb300 as pg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    names = ["weno", "predictor", "face_flux", "update", "projection"]

    def cpu(name, ocfg, ic, params, steps, sample):
        if args.no_cpu_baseline:
            return
        print(json.dumps({"config": name, "cpu_baseline": oracle_sample(ocfg, ic, params, steps, sample)}),
              flush=True)

    def measure(name, cfg, ic, params, steps=None, t_end=None, flops=None):
        s = pg.Solver(cfg, stream.cuda_stream)
        s.set_initial(ic, params, -1)      # warm-up: module loading, first launches
        s.step(1e300)
        s.reset()
        s.set_initial(ic, params, -1)
        torch.cuda.synchronize()
        s.set_profiling(True)
        s.kernel_times()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        upd, l0 = 0, 0
        with ClockSampler(0) as clk:
            e0.record(stream)
            if steps is not None:
                for _ in range(steps):
                    st = s.step(1e300)
                    upd += st.cell_updates
                    l0 += st.level0_steps
            else:
                st = s.advance_to(t_end)
                upd, l0 = st.cell_updates, st.level0_steps
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms, kn = s.kernel_times()
        n, na, cpl, apl = s.counts()
        s.close()
        line = {"config": name, "metric": "cell-updates/s", "value": upd / (ms * 1e-3), "cell_updates": int(upd),
                "level0_steps": int(l0), "ms": ms, "active_cells_per_level": [int(a) for a in apl],
                "kernel_share": {k: float(kms[i] / max(kms.sum(), 1e-9)) for i, k in enumerate(names)},
                "clocks": clk.summary()}
        if flops is not None and kn[1] > 0:
            ach = flops * upd / (kms[1] * 1e-3) / 1e12
            line["predictor"] = {"fp64_tflops": ach, "frac": ach / FP64_PEAK_TFLOPS,
                                 "flops_per_cell_update": flops}
        print(json.dumps(line), flush=True)

    T, P = pg.AW_BC_TRANSMISSIVE, pg.AW_BC_PERIODIC
    vortex = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]
    f2 = predictor_flops_per_cell(2, 2, 4, 3, EULER_FLUX_FLOPS[2])
    for n, label in ((32, "vortex 32^2 (configuration)"), (1024, "vortex 1024^2 (scaled variant)"),
                     (2048, "vortex 2048^2 (scaled variant)")):
        cfg = pg.make_config(dim=2, M=2, n=(n, n, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc=P, cfl=0.9)
        name = f"{label}: 2D Euler M=2 periodic [0,10]^2, CFL 0.9, 20 steps"
        measure(name, cfg, pg.AW_IC_VORTEX, vortex, steps=20, flops=f2)
        m = min(n, 1024)
        cpu(name, oracle.make_cfg(dim=2, M=2, n=(m, m, 1), lo=(0, 0, 0), hi=(10, 10, 1), cfl=0.9), oracle.IC_VORTEX,
            vortex, 20 if n == 32 else 1,
            "all 20 steps" if n == 32 else f"one level-0 step of the same vortex on {m}^2 (a uniform grid costs "
                                          "the same per cell update at any size)")
    # configuration 1 again through the latency path (device-side dt, CUDA graph of 20 steps):
    # the end time is the host path's time after 20 steps, so exactly the same 20 steps are taken
    cfg = pg.make_config(dim=2, M=2, n=(32, 32, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc=P, cfl=0.9)
    s = pg.Solver(cfg, stream.cuda_stream)
    s.set_initial(pg.AW_IC_VORTEX, vortex, -1)
    for _ in range(20):
        s.step(1e300)
    t20 = s.t
    s.set_initial(pg.AW_IC_VORTEX, vortex, -1)
    s.advance_graph(t20, 20)                     # warm-up (capture, module loading)
    times = []
    for _ in range(5):
        s.set_initial(pg.AW_IC_VORTEX, vortex, -1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = s.advance_graph(t20, 20)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        assert st.level0_steps == 20
    ms = statistics.median(times)
    print(json.dumps({"config": "vortex 32^2 (configuration), latency path: aw_advance_graph, device-side dt, "
                                "one CUDA graph of 20 steps", "metric": "cell-updates/s",
                      "value": st.cell_updates / (ms * 1e-3), "cell_updates": int(st.cell_updates),
                      "level0_steps": int(st.level0_steps), "ms": ms, "ms_runs": times}), flush=True)
    s.close()
    cfg = pg.make_config(dim=2, pde=pg.AW_PDE_MHD_GLM, M=3, n=(128, 128, 1), lo=(0, 0, 0),
                         hi=(2 * np.pi, 2 * np.pi, 1), bc=P, r=3, lmax=1, gamma=5.0 / 3.0, c_h=2.0, cfl=0.6,
                         auto_regrid=1)
    name = "MHD-GLM Orszag-Tang type: M=3, base 128^2 on [0,2pi]^2, r=3, l_max=1, CFL 0.6, t_end=0.5"
    measure(name, cfg, pg.AW_IC_OT, [], t_end=0.5, flops=predictor_flops_per_cell(2, 3, 9, 4, MHD_FLUX_FLOPS_2D))
    cpu(name, oracle.make_cfg(dim=2, pde=oracle.PDE_MHD, M=3, n=(128, 128, 1), lo=(0, 0, 0),
                              hi=(2 * np.pi, 2 * np.pi, 1), r=3, lmax=1, gamma=5.0 / 3.0, c_h=2.0, cfl=0.6),
        oracle.IC_OT, [], 2, "the first 2 level-0 steps")
    cfg = pg.make_config(dim=3, M=2, n=(64, 64, 64), lo=(-1, -1, -1), hi=(1, 1, 1), bc=T, r=3, lmax=2, cfl=0.6,
                         auto_regrid=1)
    f3 = predictor_flops_per_cell(3, 2, 5, 3, EULER_FLUX_FLOPS[3])
    name = (f"3D explosion: Euler M=2, base 64^3 on [-1,1]^3, r=3, l_max=2, CFL 0.6; sample: the first "
            f"{args.cfg3_steps} level-0 steps after the initial refinement")
    measure(name, cfg, pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, steps=args.cfg3_steps, flops=f3)
    # the oracle cannot hold the 576^3 finest level on the host: the same depth, r, M and CFL on a
    # 4^3 base (per cell update the oracle's cost does not depend on the base)
    cpu(name, oracle.make_cfg(dim=3, M=2, n=(4, 4, 4), lo=(-1, -1, -1), hi=(1, 1, 1), bc=oracle.BC_TRANSMISSIVE,
                              r=3, lmax=2, cfl=0.6),
        oracle.IC_EXPLOSION, aw_inputs.EXPLOSION, 1,
        "the first level-0 step after the initial refinement of the same explosion on a 4^3 base (same r, l_max, "
        "M, CFL)")
    return 0


def run_tune(args):
    """The launch-shape rules (aw_set_launch_params) tuned by measurement: device time per cell
    update of the explosion workload (to t = 0.05) and of the 32^2 vortex (20 steps) for each
    setting of one rule at a time, the others at their defaults.  Results never depend on these
    rules; the library's defaults are the values this sweep selects."""
    import torch
    import aw_inputs
    import paper_1212_3585_gb300 as pg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    default = pg.get_launch_params()

    def ns_per_update(cfg, ic, params, steps=None, t_end=None, reps=2):
        s = pg.Solver(cfg, stream.cuda_stream)
        s.set_initial(ic, params, -1)
        s.step(1e300)                     # warm-up
        best = float("inf")
        for _ in range(reps):
            s.reset()
            s.set_initial(ic, params, -1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            upd = 0
            if steps:
                for _ in range(steps):
                    upd += s.step(1e300).cell_updates
            else:
                upd = s.advance_to(t_end).cell_updates
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, 1e6 * e0.elapsed_time(e1) / upd)
        s.close()
        return best

    expl = pg.make_config(bc=pg.AW_BC_TRANSMISSIVE, auto_regrid=1, **CFG)
    vort = pg.make_config(dim=2, M=2, n=(32, 32, 1), lo=(0, 0, 0), hi=(10, 10, 1), bc=pg.AW_BC_PERIODIC, cfl=0.9)
    vortex = [5.0, 5.0, 5.0, 1.0, 1.0, 1.0, 1.0]

    def measure(**kw):
        pg.set_launch_params(**{**default, **kw})
        r = {"explosion_ns": ns_per_update(expl, pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, t_end=0.05),
             "vortex32_ns": ns_per_update(vort, pg.AW_IC_VORTEX, vortex, steps=20)}
        return {**kw, **r}

    sweeps = {"pass_min_cells": [0, 4096, 65536, 10 ** 12], "tile8_min_cells": [0, 20000, 10 ** 12],
              "small_ctas_per_sm": [0, 1, 2, 4]}
    out = {}
    for knob, values in sweeps.items():
        out[knob] = [measure(**{knob: v}) for v in values]
    pg.set_launch_params(**default)
    print(json.dumps({"metric": "device ns per cell update by launch-shape rule", "unit": "ns",
                      "higher_is_better": False, "dtype": "f64", "data": "synthetic", "defaults": default,
                      "config": {"workload": "explosion (bench workload to t=0.05) and vortex 32^2 (20 steps)"},
                      "sweeps": out}))
    return 0


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The FP64 CPU oracle as it stands, timed on the host cores; each step = the first level-0
    step of the workload (setup untimed)."""
    import oracle
    import aw_inputs
    threads = os.cpu_count() or 1
    times, updates = [], []
    for i in range(args.warmup + args.steps):
        o = oracle.Oracle(oracle.make_cfg(dim=2, M=3, n=CFG["n"], lo=CFG["lo"], hi=CFG["hi"],
                                          bc=oracle.BC_TRANSMISSIVE, r=3, lmax=2, cfl=0.6, auto_regrid=1),
                          threads=threads)
        o.set_initial(oracle.IC_EXPLOSION, aw_inputs.EXPLOSION)
        u0 = o.updates()[0]
        t0 = time.perf_counter()
        o.step(T_END)
        el = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(el)
            updates.append(o.updates()[0] - u0)
        del o
    value = sum(updates) / sum(times)
    sample = "first level-0 step (all 3 levels, LTS, regrid) of the workload, per step"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)", "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_sample(level0_steps=4):
    """The oracle as it stands on all host cores (OpenMP over cells), timed on the first
    level-0 steps of the workload (about 10 s of CPU work); setup untimed."""
    import oracle
    import aw_inputs
    threads = os.cpu_count() or 1
    o = oracle.Oracle(oracle.make_cfg(dim=2, M=3, n=CFG["n"], lo=CFG["lo"], hi=CFG["hi"],
                                      bc=oracle.BC_TRANSMISSIVE, r=3, lmax=2, cfl=0.6, auto_regrid=1),
                      threads=threads)
    o.set_initial(oracle.IC_EXPLOSION, aw_inputs.EXPLOSION)
    u0 = o.updates()[0]
    t0 = time.perf_counter()
    for _ in range(level0_steps):
        o.step(T_END)
    el = time.perf_counter() - t0
    n = o.updates()[0] - u0
    out = {"value": n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {level0_steps} level-0 steps of the workload ({n} cell updates, {el:.1f} s)"}
    # the same oracle on one core, on the first level-0 step
    o1 = oracle.Oracle(oracle.make_cfg(dim=2, M=3, n=CFG["n"], lo=CFG["lo"], hi=CFG["hi"],
                                       bc=oracle.BC_TRANSMISSIVE, r=3, lmax=2, cfl=0.6, auto_regrid=1), threads=1)
    o1.set_initial(oracle.IC_EXPLOSION, aw_inputs.EXPLOSION)
    u1 = o1.updates()[0]
    t1 = time.perf_counter()
    o1.step(T_END)
    el1 = time.perf_counter() - t1
    n1 = o1.updates()[0] - u1
    out["single_core"] = {"value": n1 / el1, "unit": UNIT, "cores": 1,
                          "sample": f"first level-0 step of the workload ({n1} cell updates, {el1:.1f} s)"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--base", type=int, default=100, help="level-0 cells per direction (workload: 100)")
    ap.add_argument("--serve", action="store_true", help="request-stream benchmark of the serving loop")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--serve-base-max", type=int, default=96)
    ap.add_argument("--serve-base-min", type=int, default=32)
    ap.add_argument("--serve-lmax-max", type=int, default=2)
    ap.add_argument("--serve-t-end", type=float, default=0.05)
    ap.add_argument("--concurrency", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=160.0)
    ap.add_argument("--serve-batch", type=int, default=8, help="batch size of the batched request loop")
    ap.add_argument("--t-end", type=float, default=T_END, help="end time (workload: 0.25)")
    ap.add_argument("--efficiency", action="store_true",
                    help="cost per cell update of orders 2-4, uniform vs AMR (r=4, l_max=2)")
    ap.add_argument("--eff-base", type=int, default=25)
    ap.add_argument("--configs", action="store_true", help="throughput of the other configurations")
    ap.add_argument("--tune", action="store_true", help="time the launch-shape rules (aw_set_launch_params)")
    ap.add_argument("--cfg3-steps", type=int, default=2)
    ap.add_argument("--eff-t-end", type=float, default=0.1)
    args = ap.parse_args()
    if args.base != 100 or args.t_end != T_END:
        CFG["n"] = (args.base, args.base, 1)
        globals()["T_END"] = args.t_end
        globals()["WORKLOAD"] = WORKLOAD.replace("base 100x100", f"base {args.base}x{args.base}").replace(
            "t_end=0.25", f"t_end={args.t_end}")
    ws, rank, local = dist_setup()
    if args.serve:
        return run_serve(args) if rank == 0 else 0
    if args.efficiency:
        return run_efficiency(args) if rank == 0 else 0
    if args.configs:
        return run_configs(args) if rank == 0 else 0
    if args.tune:
        return run_tune(args) if rank == 0 else 0
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0

    import numpy as np
    import torch
    import aw_inputs
    import paper_1212_3585_gb300 as pg
    torch.cuda.set_device(local)
    pgroup = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pgroup = dist

    def barrier():
        if pgroup:
            pgroup.barrier()

    stream = torch.cuda.current_stream()
    cfg = pg.make_config(bc=pg.AW_BC_TRANSMISSIVE, auto_regrid=1, **CFG)
    s = pg.Solver(cfg, stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB of L2

    def solve():
        s.reset()
        s.set_initial(pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, -1)
        st = s.advance_to(T_END)
        return st.cell_updates, st.level0_steps

    for _ in range(args.warmup):
        solve()
        flush.fill_(1)
    torch.cuda.synchronize()
    s.set_profiling(True)
    s.kernel_times()
    launches0 = s.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    upd, l0 = 0, 0
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            evs[i][0].record(stream)
            u, n0 = solve()
            evs[i][1].record(stream)
            upd += u
            l0 += n0
            flush.fill_(1)
        torch.cuda.synchronize()
    barrier()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    launches = s.kernel_launches() - launches0
    kms, kn = s.kernel_times()
    s.set_profiling(False)
    def max_reduce(x):
        if not pgroup:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        pgroup.all_reduce(t, op=pgroup.ReduceOp.MAX)
        return float(t.item())

    value, ms = combine_replicas(upd, ms, ws, max_reduce)

    # dominant kernel and its algorithmic FP64 rate
    names = ["weno", "predictor", "face_flux", "update", "projection"]
    dom = int(np.argmax(kms))
    upd_per_step = upd / args.steps
    V = 4
    pf = predictor_flops_per_cell(2, 3, V, 4, EULER_FLUX_FLOPS[2])
    roofline = None
    if names[dom] == "predictor" and kn[dom] > 0:
        ach = pf * upd / (kms[dom] * 1e-3) / 1e12
        cells_per_launch = upd / kn[dom]
        roofline = {"bound": "alu", "kernel": "k_predict<2,3,Euler>", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                    "traffic": PREDICTOR_DRAM_BYTES_PER_CELL * cells_per_launch,
                    "traffic_note": "bytes per average launch: ncu dram read+write of a full-size launch per cell x cells per launch",
                    "cells_per_launch": cells_per_launch,
                    "flops_per_cell_update": pf, "launches": int(kn[dom]),
                    "avg_launch_ms": float(kms[dom] / kn[dom]),
                    "peak_note": "FP64 FMA pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (derived; 1.195 measured)"}
    else:
        roofline = {"bound": "alu", "kernel": names[dom], "achieved": None, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": None, "traffic": None}
    kernel_share = {n: float(kms[i] / max(kms.sum(), 1e-9)) for i, n in enumerate(names)}
    flops = {"weno": weno_flops_per_cell(2, 3, V), "predictor": pf, "face_flux": flux_flops_per_cell(2, 3, V)}
    hbm = _measured_hbm()
    bpc = bytes_per_cell(2, 3, V)
    kernels = {}
    for i, n in enumerate(names[:3]):
        if kms[i] <= 0:
            continue
        t = kms[i] * 1e-3
        kernels[n] = {"ms_total": float(kms[i]), "launches": int(kn[i]), "share": kernel_share[n],
                      "fp64_tflops": flops[n] * upd / t / 1e12,
                      "fp64_frac": flops[n] * upd / t / 1e12 / FP64_PEAK_TFLOPS,
                      "hbm_gbs_algorithmic": bpc[n] * upd / t / 1e9,
                      "hbm_frac": bpc[n] * upd / t / 1e9 / hbm,
                      "flops_per_cell_update": flops[n], "bytes_per_cell_update": bpc[n]}

    # the whole step: algorithmic FP64 work of WENO, predictor and face flux per cell update over
    # the timed device time of the solve (bookkeeping, projection and host gaps included)
    step_flops = sum(flops.values()) * upd / args.steps
    step_tf = step_flops / (ms / args.steps * 1e-3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cell_updates_per_solve": upd_per_step, "level0_steps_per_solve": l0 / args.steps,
                   "l2": "flushed between timed solves (256 MB write)", "parallelism": f"replicas x{ws}"},
        "roofline": roofline,
        "step_fp64": {"achieved": step_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": step_tf / FP64_PEAK_TFLOPS,
                      "flops_per_cell_update": sum(flops.values())},
        "kernel_time_share": kernel_share, "kernels": kernels, "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }

    if not args.no_e2e:
        # end to end through the C ABI with host buffers
        s.reset()
        s.set_initial(pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, 0)
        _, u0 = s.cells()
        h_u0 = torch.from_numpy(u0).pin_memory()
        n_out = 0
        t_e2e, upd_e2e = 0.0, 0
        ncell_out = 0
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.reset()
            s.set_cell_averages(h_u0.numpy())
            for _ in range(cfg.lmax):
                s.regrid(0)
            st = s.advance_to(T_END)
            meta, u = s.cells()
            el = time.perf_counter() - t0
            if i >= args.warmup:
                t_e2e += el
                upd_e2e += st.cell_updates
                ncell_out = len(u)
        e2e_val = ws * upd_e2e / t_e2e
        out["e2e"] = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(u0.nbytes),
                      "d2h_bytes_per_step": int(ncell_out * (V * 8 + 20)),
                      "note": "level-0 averages uploaded from pinned host memory, data-driven refinement "
                              "(projection mode), solve, every cell read back"}
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(out))
    s.close()
    if pgroup:
        pgroup.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
