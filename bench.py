#!/usr/bin/env python
"""Benchmark: ADER-WENO cell-updates/s on the 3D AMR explosion (the headline) or the 2D one.

Headline workload (--workload explosion3d, the default): 3D Euler, gamma 1.4, FP64, ADER-WENO M=2
(third order), base grid 64^3 on [-1,1]^3, refinement factor 3, l_max = 2 (576^3 effective),
local time stepping, Loehner density indicator, spherical explosion (rho=1, p=1 inside r=0.5;
rho=0.125, p=0.1 outside), transmissive boundaries, Rusanov flux, CFL 0.6, to t=0.25.  A whole
solve is a hundred level-0 steps of several seconds each, so one "step" is one level-0 step of
the solve as the library runs it (aw_step: CFL time step, the nine level-2 sub-steps with their
coarse levels, the regrid after it), taken after the initial condition, its refinement passes and
the W warm-up level-0 steps: the timed steps are level-0 steps W+1 .. W+K of the solve.
Secondary workload (--workload explosion2d): the 2D explosion (M=3, base 100^2, r=3, l_max=2,
t=0.25), one step = one complete solve from aw_reset.

Three passes run the same steps from the same start (every pass computes the same bits):
value   = cell updates (active cell advanced by its level's dt) per second, device time of the timed
          steps with CUDA events on the solver's stream, no per-kernel events; L2 flushed (256 MB
          write) between steps
kernels = a second pass with the library's per-kernel CUDA events on (aw_set_profiling): each
          kernel's share and the dominant kernel's average launch duration, for the roofline
e2e     = a third pass through the C ABI with host buffers: every step uploads the state from
          pinned host memory (aw_set_cell_averages), steps, and reads every cell back into pinned
          host memory (aw_read_cells); wall time with the copies
roofline= the dominant kernel's algorithmic FP64 FLOP rate against the FP64 peak
cpu_baseline = the FP64 CPU oracle on all host cores, on a bounded sample of the same workload

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
WORKLOADS = {
    "explosion3d": {
        "desc": ("3D Euler FP64, ADER-WENO M=2, base 64x64x64 on [-1,1]^3, r=3, l_max=2, local time stepping, "
                 "spherical explosion (R=0.5; rho,p = 1,1 inside; 0.125,0.1 outside), transmissive, Rusanov, "
                 "CFL 0.6, t_end=0.25"),
        "cfg": dict(dim=3, M=2, n=(64, 64, 64), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), r=3, lmax=2, gamma=1.4,
                    chi_ref=0.2, chi_rec=0.1, cfl=0.6),
        "t_end": 0.25, "step": "level0",
        # the host cannot hold the oracle's 576^3 finest level: its samples run the same r, l_max,
        # M and CFL on a small base (the oracle's cost per cell update does not depend on the base)
        "oracle_base": 5, "reference_base": 3,
    },
    "explosion2d": {"desc": WORKLOAD, "cfg": CFG, "t_end": T_END, "step": "solve", "oracle_base": None,
                    "reference_base": None},
}
SM_COUNT = 152
FP64_FMA_PER_CLK_PER_SM = 2      # sm_103a: measured 0.598 T DFMA/s at ~1.97 GHz on 152 SMs
SM_MAX_MHZ = 2070.0
HBM_GBS = 6792.1                 # measured copy bandwidth of this GB300 pool
# DRAM bytes per cell of the predictor from one ncu capture of a launch of the kernel's current
# build, scaled by the cells of an average launch of the timed steps.  3D (k_predict<3,2,Euler>):
# a level-2 launch of the same explosion on a 20^3 base (72792 CTAs x 7 cells, 2.2 GB of
# predictor data, far above the 129 MB L2): dram__bytes_read.sum 552.00 MB +
# dram__bytes_write.sum 1590.03 MB.  2D (k_predict<2,3,Euler>): a level-2 launch of the 100x100
# explosion (6264 CTAs x 16 cells): 51.63 MB + 140.97 MB.  Must be re-captured whenever k_predict
# changes.
PREDICTOR_DRAM_BYTES_PER_CELL = (51634944 + 140974592) / (6264 * 16)
PREDICTOR_DRAM_BYTES_PER_CELL_3D = {"predictor": (552003328 + 1590025000) / (72792 * 7)}


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
                "p99_ms": float(np.percentile(tts, 99)), "cell_updates_per_s": upd / done, "failed": failed,
                "failure_rate": failed / len(reqs)}

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
               "cell_updates_per_s": st.cell_updates_per_s, "failed": int(st.failed),
               "failure_rate": int(st.failed) / len(reqs), "requeues": int(st.requeues), "grows": int(st.grows),
               "peak_reserved_gb": st.peak_reserved_bytes / 2 ** 30}
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
                                 "sample": (f"the first {len(reqs)} requests of the seeded stream (seed 20121213), "
                                            f"end time {t_end} instead of the stream's 0.2"
                                            if t_end != 0.2 else f"the first {len(reqs)} requests of the seeded stream"),
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


def _oracle_cfg(wl, base=None):
    """the oracle's configuration of workload wl (optionally on a smaller base grid)"""
    import oracle
    c = dict(wl["cfg"])
    if base is not None:
        c["n"] = (base, base, base) if c["dim"] == 3 else (base, base, 1)
    return oracle.make_cfg(dim=c["dim"], M=c["M"], n=c["n"], lo=c["lo"], hi=c["hi"], bc=oracle.BC_TRANSMISSIVE,
                           r=c["r"], lmax=c["lmax"], gamma=c["gamma"], chi_ref=c["chi_ref"], chi_rec=c["chi_rec"],
                           cfl=c["cfl"], auto_regrid=1)


def _oracle_first_step(wl, base, threads):
    """the oracle as it stands: initial condition and refinement passes (untimed), then the first
    level-0 step of the workload (timed); returns (cell updates, seconds)"""
    import oracle
    import aw_inputs
    o = oracle.Oracle(_oracle_cfg(wl, base), threads=threads)
    o.set_initial(oracle.IC_EXPLOSION, aw_inputs.EXPLOSION)
    u0 = o.updates()[0]
    t0 = time.perf_counter()
    rc, _ = o.step(wl["t_end"])
    el = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError(f"oracle step failed ({rc})")
    return o.updates()[0] - u0, el


def run_reference(args, wl):
    """The FP64 CPU oracle as it stands, timed on the host cores; each step = the first level-0
    step of the workload (setup untimed): on the workload's own grid for the 2D explosion, on a
    3^3 base with the same r, l_max, M and CFL for the 3D one (the 576^3 finest level does not fit
    the host, and the oracle's cost per cell update does not depend on the base)."""
    threads = os.cpu_count() or 1
    times, updates = [], []
    for i in range(args.warmup + args.steps):
        n, el = _oracle_first_step(wl, wl["reference_base"], threads)
        if i >= args.warmup:
            times.append(el)
            updates.append(n)
    value = sum(updates) / sum(times)
    if wl["reference_base"]:
        b = wl["reference_base"]
        sample = (f"first level-0 step (all 3 levels, LTS, regrid) of the same explosion on a {b}^3 base "
                  f"(same r, l_max, M, CFL; {updates[0]} cell updates), per step")
    else:
        sample = "first level-0 step (all 3 levels, LTS, regrid) of the workload, per step"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "l2": "n/a (CPU)", "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_sample(wl, level0_steps=4):
    """The oracle as it stands on all host cores (OpenMP over cells), about 10-30 s of CPU work,
    setup untimed: the 2D explosion's first level-0 steps on its own grid (and its first step on
    one core); the 3D explosion's first level-0 step on a 5^3 base with the same r, l_max, M and
    CFL (the 576^3 finest level does not fit the host)."""
    import oracle
    import aw_inputs
    threads = os.cpu_count() or 1
    if wl["oracle_base"]:
        b = wl["oracle_base"]
        n, el = _oracle_first_step(wl, b, threads)
        return {"value": n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": (f"first level-0 step after the initial refinement of the same explosion on a {b}^3 base "
                           f"(same r, l_max, M, CFL; {n} cell updates, {el:.1f} s)")}
    o = oracle.Oracle(_oracle_cfg(wl), threads=threads)
    o.set_initial(oracle.IC_EXPLOSION, aw_inputs.EXPLOSION)
    u0 = o.updates()[0]
    t0 = time.perf_counter()
    for _ in range(level0_steps):
        o.step(wl["t_end"])
    el = time.perf_counter() - t0
    n = o.updates()[0] - u0
    out = {"value": n / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"first {level0_steps} level-0 steps of the workload ({n} cell updates, {el:.1f} s)"}
    n1, el1 = _oracle_first_step(wl, None, 1)
    out["single_core"] = {"value": n1 / el1, "unit": UNIT, "cores": 1,
                          "sample": f"first level-0 step of the workload ({n1} cell updates, {el1:.1f} s)"}
    return out


def kernel_flops(D, M, V):
    """algorithmic FP64 FLOP per cell update of the three hot kernels (Euler)"""
    P = M + 1
    return {"weno": weno_flops_per_cell(D, M, V), "predictor": predictor_flops_per_cell(D, M, V, P, EULER_FLUX_FLOPS[D]),
            "face_flux": flux_flops_per_cell(D, M, V)}


KERNEL_NAMES = ["weno", "predictor", "face_flux", "update", "projection"]
KERNEL_SYMBOLS = {"weno": "k_weno*", "predictor": "k_predict", "face_flux": "k_flux", "update": "k_update",
                  "projection": "k_project"}


def roofline_entry(kms, kn, upd, flops, D, M, traffic_per_cell):
    """the dominant kernel of a profiled pass: algorithmic FP64 FLOP per launch over its average
    launch duration, against the FP64 peak"""
    import numpy as np
    dom = int(np.argmax(kms))
    name = KERNEL_NAMES[dom]
    if name not in flops or kn[dom] <= 0:
        return {"bound": "alu", "kernel": name, "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "traffic": None}
    cells_per_launch = upd / kn[dom] if name == "predictor" else None
    ach = flops[name] * upd / (kms[dom] * 1e-3) / 1e12
    tr = traffic_per_cell.get(name)
    return {"bound": "alu", "kernel": f"{KERNEL_SYMBOLS[name]}<{D},{M},Euler>", "achieved": ach,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
            "traffic": (tr * upd / kn[dom]) if tr is not None else None,
            "traffic_note": ("DRAM read+write bytes per launch: ncu bytes per cell of a captured launch x cells per "
                             "average launch" if tr is not None else "no ncu capture of this kernel's current build"),
            "flops_per_cell_update": flops[name], "launches": int(kn[dom]), "cell_updates": int(upd),
            "avg_launch_ms": float(kms[dom] / kn[dom]), "cells_per_launch": cells_per_launch,
            "peak_note": "FP64 FMA pipe: 2 DFMA/clk/SM x 152 SMs x 2070 MHz (derived; 1.195 measured)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="explosion3d", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps of the profiled pass: the first timed steps again (0: all of them)")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="steps of the end-to-end pass: the first timed steps again (0: all of them)")
    ap.add_argument("--base", type=int, default=0, help="level-0 cells per direction (workload: 64 in 3D, 100 in 2D)")
    ap.add_argument("--serve", action="store_true", help="request-stream benchmark of the serving loop")
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--serve-base-max", type=int, default=96)
    ap.add_argument("--serve-base-min", type=int, default=32)
    ap.add_argument("--serve-lmax-max", type=int, default=2)
    ap.add_argument("--serve-t-end", type=float, default=0.05)
    ap.add_argument("--concurrency", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=160.0)
    ap.add_argument("--serve-batch", type=int, default=8, help="batch size of the batched request loop")
    ap.add_argument("--t-end", type=float, default=0.0, help="end time (workloads: 0.25)")
    ap.add_argument("--efficiency", action="store_true",
                    help="cost per cell update of orders 2-4, uniform vs AMR (r=4, l_max=2)")
    ap.add_argument("--eff-base", type=int, default=25)
    ap.add_argument("--configs", action="store_true", help="throughput of the other configurations")
    ap.add_argument("--tune", action="store_true", help="time the launch-shape rules (aw_set_launch_params)")
    ap.add_argument("--cfg3-steps", type=int, default=2)
    ap.add_argument("--eff-t-end", type=float, default=0.1)
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    wl["cfg"] = dict(wl["cfg"])
    D = wl["cfg"]["dim"]
    if args.base:
        b0 = wl["cfg"]["n"][0]
        wl["cfg"]["n"] = (args.base, args.base, args.base if D == 3 else 1)
        dims = "x".join([str(b0)] * D)
        wl["desc"] = wl["desc"].replace(f"base {dims}", "base " + "x".join([str(args.base)] * D))
    if args.t_end:
        wl["desc"] = wl["desc"].replace(f"t_end={wl['t_end']}", f"t_end={args.t_end}")
        wl["t_end"] = args.t_end
    if args.workload == "explosion2d":       # --configs/--tune use the 2D workload's globals
        CFG["n"] = wl["cfg"]["n"]
        globals()["T_END"] = wl["t_end"]
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
        print(json.dumps(run_reference(args, wl)))
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

    def max_reduce(x):
        if not pgroup:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        pgroup.all_reduce(t, op=pgroup.ReduceOp.MAX)
        return float(t.item())

    t_end = wl["t_end"]
    per_solve = wl["step"] == "solve"
    M, V = wl["cfg"]["M"], D + 2
    stream = torch.cuda.current_stream()
    cfg = pg.make_config(bc=pg.AW_BC_TRANSMISSIVE, auto_regrid=1, **wl["cfg"])
    s = pg.Solver(cfg, stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB of L2

    def start():
        """initial condition and its l_max refinement passes on the device"""
        s.reset()
        s.set_initial(pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, -1)

    def one_step():
        """one benchmark step: a whole solve, or the next level-0 step of the running solve"""
        if per_solve:
            start()
            st = s.advance_to(t_end)
        else:
            if not s.t < t_end:
                raise RuntimeError(f"the solve reached t_end = {t_end} before the last timed step")
            st = s.step(t_end)
        return st.cell_updates, st.level0_steps

    def warm():
        if not per_solve:
            start()
        for _ in range(args.warmup):
            one_step()
            flush.fill_(1)
        torch.cuda.synchronize()

    # ---- pass 1: the value (device time, no per-kernel events) ----
    warm()
    t_first = s.t
    launches0 = s.kernel_launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    upd, l0, step_updates, max_cells = 0, 0, [], 0
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            evs[i][0].record(stream)
            u, n0 = one_step()
            evs[i][1].record(stream)
            upd += u
            l0 += n0
            step_updates.append(int(u))
            flush.fill_(1)
            max_cells = max(max_cells, s.counts()[0])
        torch.cuda.synchronize()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms)
    launches = s.kernel_launches() - launches0
    t_last = s.t
    counts_last = s.counts()
    value, ms = combine_replicas(upd, ms, ws, max_reduce)

    # ---- pass 2: the same steps with the library's per-kernel events (shares, roofline) ----
    kprof = min(args.profile_steps or args.steps, args.steps)
    ke2e = min(args.e2e_steps or args.steps, args.steps)
    warm()
    s.set_profiling(True)
    s.kernel_times()
    upd_p = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(kprof):
        u, _ = one_step()
        upd_p += u
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = e0.elapsed_time(e1)
    kms, kn = s.kernel_times()
    s.set_profiling(False)
    if upd_p != sum(step_updates[:kprof]):
        raise RuntimeError("the profiled pass did not repeat the timed steps")

    flops = kernel_flops(D, M, V)
    traffic = PREDICTOR_DRAM_BYTES_PER_CELL_3D if D == 3 else (
        {"predictor": PREDICTOR_DRAM_BYTES_PER_CELL} if PREDICTOR_DRAM_BYTES_PER_CELL else {})
    roofline = roofline_entry(kms, kn, upd_p, flops, D, M, traffic)
    kernel_share = {n: float(kms[i] / max(kms.sum(), 1e-9)) for i, n in enumerate(KERNEL_NAMES)}
    hbm = _measured_hbm()
    bpc = bytes_per_cell(D, M, V)
    kernels = {}
    for i, n in enumerate(KERNEL_NAMES[:3]):
        if kms[i] <= 0:
            continue
        t = kms[i] * 1e-3
        kernels[n] = {"ms_total": float(kms[i]), "launches": int(kn[i]), "share": kernel_share[n],
                      "fp64_tflops": flops[n] * upd_p / t / 1e12,
                      "fp64_frac": flops[n] * upd_p / t / 1e12 / FP64_PEAK_TFLOPS,
                      "hbm_gbs_algorithmic": bpc[n] * upd_p / t / 1e9,
                      "hbm_frac": bpc[n] * upd_p / t / 1e9 / hbm,
                      "flops_per_cell_update": flops[n], "bytes_per_cell_update": bpc[n]}
    # the whole step: algorithmic FP64 work of WENO, predictor and face flux per cell update over
    # the timed device time (bookkeeping, projection and host gaps included)
    step_tf = sum(flops.values()) * upd / (ms * 1e-3) / 1e12
    unit_desc = ("one complete solve from aw_reset (initial condition, refinement passes, solve to t_end)"
                 if per_solve else
                 f"one level-0 step (aw_step: CFL dt, r^l_max sub-steps, regrid); timed: level-0 steps "
                 f"{args.warmup + 1}..{args.warmup + args.steps} of the solve, t = {t_first:.5f} .. {t_last:.5f}")
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "step": unit_desc, "cell_updates_per_step": upd / args.steps,
                   "level0_steps_per_step": l0 / args.steps, "cell_updates_by_step": step_updates,
                   "ms_by_step": step_ms,
                   "cells_after_last_step": int(counts_last[0]), "active_per_level_after_last_step":
                       [int(a) for a in counts_last[3]],
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"},
        "roofline": roofline,
        "step_fp64": {"achieved": step_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                      "frac": step_tf / FP64_PEAK_TFLOPS, "flops_per_cell_update": sum(flops.values())},
        "kernel_time_share": kernel_share, "kernels": kernels,
        "profiled_pass": {"steps": kprof, "ms": ms_p, "ms_unprofiled_same_steps": float(sum(step_ms[:kprof])),
                          "hot_kernels_share_of_step": float(kms.sum() / ms_p),
                          "note": "the same steps again with a CUDA event pair around every hot launch; "
                                  "the rest of the step is regrid, compaction, dt, averaging and host gaps"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        # the autotuner's CTA sizes for this configuration's level size classes (floor(log2 active
        # cells)): full- or reduced-size CTAs, with the device ns per cell of each variant's trials
        "tuning": [{"kernel": ("predictor", "face_flux")[e["kernel"]], "size_class": e["size_class"],
                    "cta": {-1: "trying", 0: "full", 1: "reduced"}[e["choice"]], "inherited": bool(e["inherited"]),
                    "ns_per_cell": [round(x, 3) for x in e["ns_per_cell"]]}
                   for e in pg.get_tuning() if (e["dim"], e["M"], e["pde"]) == (cfg.dim, cfg.M, cfg.pde)],
    }

    if not args.no_e2e:
        # ---- pass 3: end to end through the C ABI with pinned host buffers ----
        if per_solve:
            s.reset()
            s.set_initial(pg.AW_IC_EXPLOSION, aw_inputs.EXPLOSION, 0)
            _, u0 = s.cells()                       # the level-0 initial averages: the solve's input
            h_u = torch.empty((max_cells, V), dtype=torch.float64).pin_memory().numpy()
            h_m = torch.empty((max_cells, 5), dtype=torch.int32).pin_memory().numpy()
            h_u0 = torch.from_numpy(u0).pin_memory().numpy()
            t_e2e, upd_e2e, h2d, d2h = 0.0, 0, 0, 0
            for i in range(args.warmup + ke2e):
                flush.fill_(1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.reset()
                s.set_cell_averages(h_u0)          # H2D: the initial level-0 averages
                for _ in range(cfg.lmax):
                    s.regrid(1)                     # the initial refinement passes of set_initial
                st = s.advance_to(t_end)
                n = s.cells_into(h_m, h_u)          # D2H: every cell of the result
                el = time.perf_counter() - t0
                if i >= args.warmup:
                    t_e2e += el
                    upd_e2e += st.cell_updates
                    h2d += h_u0.nbytes
                    d2h += n * (V * 8 + 20)
            note = ("every step: level-0 initial averages uploaded from pinned host memory, the initial "
                    "refinement passes, the solve, every cell read back into pinned host memory")
        else:
            warm()
            cap = int(max_cells * 1.05) + 64
            h_u = torch.empty((cap, V), dtype=torch.float64).pin_memory().numpy()
            h_m = torch.empty((cap, 5), dtype=torch.int32).pin_memory().numpy()
            n = s.cells_into(h_m, h_u)              # the state the first timed step starts from
            t_e2e, upd_e2e, h2d, d2h = 0.0, 0, 0, 0
            for i in range(ke2e):
                flush.fill_(1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.set_cell_averages(h_u[:n])        # H2D: the step's input state
                h2d += n * V * 8
                u, _ = one_step()
                n = s.cells_into(h_m, h_u)          # D2H: the step's result, every cell
                d2h += n * (V * 8 + 20)
                t_e2e += time.perf_counter() - t0
                upd_e2e += u
            note = ("every step: the whole state uploaded from pinned host memory (aw_set_cell_averages), "
                    "the level-0 step, every cell read back into pinned host memory (aw_read_cells)")
        if upd_e2e != sum(step_updates[:ke2e]):
            raise RuntimeError("the end-to-end pass did not repeat the timed steps")
        t_job = max_reduce(t_e2e)
        same = combine_replicas(sum(step_updates[:ke2e]), sum(step_ms[:ke2e]), ws, max_reduce)[0]
        out["e2e"] = {"value": ws * upd_e2e / t_job, "unit": UNIT, "h2d_bytes_per_step": int(h2d // ke2e),
                      "d2h_bytes_per_step": int(d2h // ke2e), "ms_per_step": 1e3 * t_job / ke2e, "steps": ke2e,
                      "value_same_steps": same,
                      "note": note + f"; the first {ke2e} timed steps again (value_same_steps: the device-timed "
                                     "value over those steps); L2 flushed between steps, host wall time"}
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline_sample(wl)
        print(json.dumps(out))
    s.close()
    if pgroup:
        pgroup.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
