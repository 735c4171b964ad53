/*
 * aderweno.h -- C ABI of the GB300 (sm_103a) ADER-WENO finite volume solver on space-time
 * adaptive Cartesian meshes (Dumbser, Zanotti, Hidalgo, Balsara, arXiv:1212.3585).
 *
 * The library advances the cell averages of a hyperbolic conservation law
 * (Sec. 2.1, Eq. eq:governingPDE, source zero) on a cell-by-cell AMR mesh (Sec. 3.1) with
 * time-accurate local time stepping (Sec. 3.1.2), one level-0 step at a time.  Every step
 * of the method runs in CUDA kernels on the caller's stream:
 *   - dimension-by-dimension WENO reconstruction (Sec. 2.2),
 *   - element-local space-time DG predictor by Picard iteration (Sec. 2.3, Eq. eqn.stdg.final),
 *   - Rusanov fluxes integrated over space-time faces (Eqs. flux:F..flux:H, eqn.rusanov),
 *   - the one-step finite volume update (Eq. eq:finite_vol) with memory variables at
 *     coarse/fine faces (Eq. eqn.memory.sum),
 *   - projection (Sec. 3.1.3) and averaging (Eq. eqn.average) of virtual cells,
 *   - the refinement indicator (Eq. eqn.indicator) and the regrid under rules 1-7 of Sec. 3.1.
 *
 * Conventions
 *   - Every call returns an int status: AW_OK (0) or a negative AW_E* code; aw_last_error()
 *     returns a message for the last failing call on this thread.
 *   - The library owns every device buffer.  The caller owns every host pointer it passes;
 *     host buffers are only read/written during the call.
 *   - A call given a capacity smaller than needed returns AW_EINVAL and writes the needed
 *     size through its size pointer.
 *   - `stream` is a cudaStream_t passed as an integer (0 = the legacy default stream).  All
 *     device work of a solver is ordered on that stream; calls that return host data
 *     synchronise it.
 *   - Canonical cell order: level ascending, then k, j, i ascending (z slowest).
 *   - Cell status (Sec. 3.1 rule 2): 0 active, 1 virtual child, -1 virtual mother.
 *   - Conserved variables: Euler (rho, rho u, rho v[, rho w], E) with 2+d components;
 *     MHD-GLM (rho, rho u, rho v, rho w, E, Bx, By, Bz, psi) in rationalised units;
 *     linear advection (u).
 */
#ifndef ADERWENO_H
#define ADERWENO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AW_OK 0
#define AW_EINVAL (-1)       /* bad argument, size mismatch or capacity too small */
#define AW_ENOMEM (-2)       /* device allocation failed */
#define AW_ECUDA (-3)        /* a CUDA call failed (message has the CUDA error string) */
#define AW_ENONPHYSICAL (-4) /* rho <= 0, p <= 0 or NaN appeared in an updated cell average */
#define AW_ETIMEOUT (-5)     /* a bounded device-side wait gave up */
#define AW_ESTATE (-6)       /* call not valid in the solver's current state */
#define AW_ELIMIT (-7)       /* the solver's own device-memory limit (aw_set_memory_limit) refused an allocation */

#define AW_PDE_EULER 0
#define AW_PDE_MHD_GLM 1
#define AW_PDE_LINADV 2

#define AW_BC_PERIODIC 0
#define AW_BC_TRANSMISSIVE 1
#define AW_BC_REFLECTIVE 2   /* wall: mirror image with the normal momentum negated (Euler, linear advection) */
#define AW_BC_INFLOW 3       /* ghost cells hold the constant conserved state inflow[]; face flux against it */

#define AW_FLUX_RUSANOV 0  /* Eq. eqn.rusanov */
#define AW_FLUX_OSHER 1    /* Eq. eqn.osher, 3-point Gauss-Legendre path quadrature (Euler, MHD-GLM, linear advection) */

/* initial conditions of Sec. 4; parameter layouts:
 *  AW_IC_CONST:     primitive state (Euler: rho, v_1..v_d, p; MHD: rho, vx, vy, vz, p, Bx, By,
 *                   Bz, psi; linear advection: u)
 *  AW_IC_VORTEX:    eps, xc, yc, rho0, u0, v0, p0 (isentropic vortex of Sec. 4.1)
 *  AW_IC_EXPLOSION: R, rho_in, p_in, rho_out, p_out (explosion problems of Sec. 4.1)
 *  AW_IC_OT:        none (Orszag-Tang data of Sec. 4.2, rationalised units)
 *  AW_IC_RP4:       x0, y0, then (rho, u, v, p) of quadrants 1..4 (x>x0,y>y0; x<x0,y>y0;
 *                   x<x0,y<y0; x>x0,y<y0), the 2D Riemann problems of Sec. 4.1
 *  AW_IC_FOURIER:   base primitive state (V values), nmodes, then per mode
 *                   (var, kx, ky, kz, amp, phase) adding amp*sin(2 pi k.(x-lo)/(hi-lo) + phase)
 * Cell averages are taken with the (M+1)^d-point tensor Gauss rule. */
#define AW_IC_CONST 0
#define AW_IC_VORTEX 1
#define AW_IC_EXPLOSION 2
#define AW_IC_OT 3
#define AW_IC_RP4 4
#define AW_IC_FOURIER 5

/* aw_read_internal selectors */
#define AW_INTERNAL_WENO 0      /* WENO dofs of active cells of a level: V*N^d each, [v][p + N q + N^2 r] */
#define AW_INTERNAL_PREDICTOR 1 /* predictor dofs of active cells: V*N^(d+1) each, [v][spatial + N^d s] */
#define AW_INTERNAL_CHI 2       /* indicator of every existing cell of a level (0 where not computed) */
#define AW_INTERNAL_FLUX 3      /* face fluxes of active cells from the last update: 2d*V each, [axis][side][v] */

typedef struct aw_config {
  int32_t dim;          /* 2 or 3 */
  int32_t pde;          /* AW_PDE_* */
  int32_t M;            /* polynomial degree of the reconstruction, 1, 2 or 3 (order M+1); M = 1 for 2D Euler and linear advection only */
  int32_t nx, ny, nz;   /* level-0 cells per direction (nz ignored when dim == 2) */
  double gamma;         /* ratio of specific heats */
  double c_h;           /* GLM cleaning speed (MHD) */
  double lo[3], hi[3];  /* domain box */
  int32_t bc[6];        /* AW_BC_* for faces x-, x+, y-, y+, z-, z+; periodic must pair up */
  int32_t refine_factor;/* r of Eq. refine-factor; r >= max(2, M) when lmax > 0 */
  int32_t lmax;         /* finest level, 0..4 */
  double chi_ref;       /* refine when chi > chi_ref (Sec. 3.1.1) */
  double chi_rec;       /* recoarsen when chi < chi_rec */
  double eps_ind;       /* filter epsilon of Eq. eqn.indicator */
  double cfl;           /* CFL number */
  int32_t picard_iters; /* Picard iterations of the predictor, 0 -> M+1 */
  int32_t flux;         /* AW_FLUX_RUSANOV or AW_FLUX_OSHER */
  int32_t auto_regrid;  /* 1: regrid after every level-0 step (aw_step / aw_advance_to) */
  int32_t reserved;
  double adv[3];        /* advection velocity of AW_PDE_LINADV */
  double inflow[9];     /* conserved state beyond AW_BC_INFLOW faces (first V entries used) */
} aw_config;

typedef struct aw_stats {
  int64_t level0_steps;          /* level-0 steps taken by this call */
  int64_t cell_updates;          /* active-cell updates (one cell advanced by its level's dt) */
  int64_t updates_per_level[8];
  double last_dt0;               /* last level-0 time step */
  double t;                      /* solver time after the call */
} aw_stats;

typedef struct aw_cell {
  int32_t level, status, i, j, k;
} aw_cell;

typedef struct aw_solver aw_solver;

/* Create a solver on the current CUDA device.  Allocates the dense per-level grids (Sec. 3.1:
 * level l has n*r^l cells per direction) and installs a uniform level-0 mesh of active cells
 * with zero averages.  All device work and device memory of the solver are ordered on `stream`
 * (memory from the device's default pool, allocated and freed in stream order, so creating and
 * destroying solvers does not synchronise the device); the stream must outlive the solver.
 * Errors: AW_EINVAL (bad config), AW_ENOMEM, AW_ECUDA. */
int aw_create(const aw_config* cfg, uintptr_t stream, aw_solver** out);

/* Wait for the solver's stream, then release every buffer of the solver.  Safe on NULL. */
void aw_destroy(aw_solver* s);

/* Message of the last failing call on this thread (never NULL). */
const char* aw_last_error(void);

/* Set the averages of every existing cell from an analytic initial condition (see AW_IC_*),
 * then apply `nrefine` passes of indicator + regrid in initial-condition mode, in which new
 * cells take the initial condition's averages (Sec. 3.1: the refinement criterion is applied
 * to the initial condition up to l_max).  nrefine < 0 means lmax passes.  Resets t to 0. */
int aw_set_initial(aw_solver* s, int32_t ic_kind, const double* params, int32_t nparams, int32_t nrefine);

/* Set the averages of every existing cell (canonical order, V doubles per cell, host memory).
 * Virtual mothers are then re-averaged from their children (Eq. eqn.average).
 * n must equal the current cell count (AW_EINVAL otherwise). */
int aw_set_cell_averages(aw_solver* s, const double* u_host, int64_t n);

/* One level-0 step: dt_0 from the CFL condition (clipped at t_end), the recursive local time
 * stepping of all levels (Eq. eqn.update.criterion), then, if auto_regrid, one regrid.
 * Returns AW_ENONPHYSICAL if a non-physical state appeared. */
int aw_step(aw_solver* s, double t_end, aw_stats* stats);

/* One level-0 step of a given size dt0 (no CFL, no clipping, no regrid); for tests. */
int aw_step_dt(aw_solver* s, double dt0, aw_stats* stats);

/* Level-0 steps (with regrids if auto_regrid) until t reaches t_end. */
int aw_advance_to(aw_solver* s, double t_end, aw_stats* stats);

/* Cross-request batching (no counterpart in the paper, which advances one mesh): advances the n
 * independent solvers (1 <= n <= AW_BATCH_MAX) each to t_end, as aw_advance_to does, in lockstep
 * level-0 steps whose hot kernels (WENO, predictor, face flux, update, projection of virtual
 * children) of one level and sub-step run as ONE launch over the cells of all members.  Each
 * member keeps its own mesh, state, CFL time step, regrids and errors, and computes exactly what
 * aw_advance_to would.  The members must agree in dim, pde, M, flux and refine_factor (grid,
 * domain, lmax, boundaries, physics and data may differ) and be distinct.  All device work of the
 * call is ordered on `stream` (the members' own streams are synchronised first and restored on
 * return).  stats and rc (arrays of n entries, either may be NULL) receive each member's
 * statistics and status.  A member that fails (AW_ENONPHYSICAL, ...) stops; the others go on.
 * Returns AW_OK when every member reached t_end, else the first member's failure, or a failure of
 * the batch as a whole (AW_ECUDA).  Kernel timing (aw_set_profiling) does not cover batched
 * launches; they are counted in aw_kernel_launches of the first live member. */
#define AW_BATCH_MAX 8
int aw_advance_batch(aw_solver* const* solvers, int32_t n, double t_end, uintptr_t stream, aw_stats* stats,
                     int32_t* rc);

/* One lockstep level-0 step of a batch (no counterpart in the paper; the request loop's
 * continuous batching is built on it): every member m with t < t_end[m] takes the one level-0
 * step that aw_step(solvers[m], t_end[m]) takes (its CFL dt clipped at its own end time, all
 * levels and sub-steps, its regrid), with the hot kernels batched as in aw_advance_batch; members
 * already at their end time are left as they are.  So members may have different end times, and
 * the set of members may change from one call to the next: the step of each member is exactly
 * its own.  t_end: n end times (AW_EINVAL for NULL or NaN).  stats receive each member's
 * statistics of this step, rc each member's status; the return value, the members' requirements
 * and the stream as in aw_advance_batch. */
int aw_step_batch(aw_solver* const* solvers, int32_t n, const double* t_end, uintptr_t stream, aw_stats* stats,
                  int32_t* rc);

/* Latency path for a uniform mesh (lmax = 0; no counterpart in the paper): advances to t_end as
 * aw_advance_to does, with the CFL time step reduced, clipped at t_end and turned into the level
 * time steps on the device, so that `chunk` (1..256) level-0 steps run between two host
 * synchronisations; the steps are captured into a CUDA graph (on a stream of the solver's own,
 * ordered after `stream`), kept by the solver while its launch arguments stay the same, and
 * replayed.  Steps past t_end within the last chunk have
 * dt = 0 and change nothing.  Computes exactly what aw_advance_to computes (same kernels, same
 * time steps).  AW_EINVAL if lmax > 0 or chunk is out of range; AW_ENONPHYSICAL as aw_step. */
int aw_advance_graph(aw_solver* s, double t_end, int32_t chunk, aw_stats* stats);

/* Launch shapes (no counterpart in the paper; they change the speed, never a result):
 * WENO by passes (x, then y, then z sweeps over compact lists) on levels of at least
 * pass_min_cells cells (default 4096; tiles below), 2D WENO tiles of 8x8 cells on levels of at
 * least tile8_min_cells cells (default 20000; 4x4 below), and reduced-size predictor and flux
 * CTAs when the full-size ones would give fewer than small_ctas_per_sm CTAs per SM (default 2;
 * 0 never), fuse_flux_update: 1 (default) runs the face fluxes and the update of Eq.
 * eq:finite_vol as one kernel (the face CTA that delivers the last face flux a chunk of cells
 * needs updates that chunk; nothing waits), 0 as two kernels; and autotune: 1 (default) lets the
 * library's autotuner pick the CTA size (cells, or faces, per block: full or reduced size) of the
 * predictor and of the face flux per configuration and level size class, from CUDA-event timings
 * of the first launches of each (aw_get_tuning), in place of the small_ctas_per_sm rule; 0 the
 * rule alone; and persistent: 1 advances every level and sub-step of a batch (aw_advance_batch)
 * with one persistent cooperative launch for the projection, WENO and predictor of all members,
 * which also runs the fused face flux and update on a level with no finer level, with grid-wide
 * barriers between the phases (2D configurations, where the predictor and the face flux share
 * their CTA shape, with fuse_flux_update = 1); 0 (default: measured faster) the separate
 * launches; and graph_steps: 1 captures the launches of every level-0 step of aw_step,
 * aw_advance_to and aw_advance_batch (all levels and sub-steps) into a CUDA graph on a stream
 * of the solver's own (of the first member's, for a batch), ordered after the caller's stream,
 * and launches it: the executable graph of the previous step is updated in place when the new
 * step has the same launch sequence (the sizes and arguments may differ), else built anew; a
 * step whose launch arguments are those of the previous graph (the regrid left every level's
 * lists and sizes as they were) launches that graph again without a capture, unless it holds
 * timing events (aw_set_profiling, trials of the autotuner) (aw_graph_stats); the persistent
 * level kernel is not used in a captured step; 0 (default) launches the kernels directly.
 * The averages are bitwise the same for every setting.  Process-wide.  The first two are fixed
 * per level when a solver is created, the others apply to every launch.  AW_EINVAL for negative
 * values, small_ctas_per_sm > 64, or fuse_flux_update, autotune, persistent or graph_steps not
 * 0 or 1.
 * bench.py --tune times the workload over these parameters. */
typedef struct aw_launch_params {
  int64_t pass_min_cells;
  int64_t tile8_min_cells;
  int32_t small_ctas_per_sm;
  int32_t fuse_flux_update;
  int32_t autotune;
  int32_t persistent;
  int32_t graph_steps;
  int32_t reserved;        /* set to 0 */
} aw_launch_params;
int aw_get_launch_params(aw_launch_params* out);
int aw_set_launch_params(const aw_launch_params* in);

/* The autotuner's state (no counterpart in the paper).  For every configuration (dim, M, pde,
 * numerical flux), kernel (AW_TUNE_PREDICTOR, AW_TUNE_FLUX) and level size class (floor(log2) of
 * the level's active cells) that solvers of this process have launched, the first launches try
 * the full-size (variant 0) and reduced-size (variant 1: about a quarter, filling whole warps) CTAs
 * in turn, each timed with a pair of CUDA events on the solver's stream; once each variant has
 * AW_TUNE_TRIALS timings, the one with
 * the least device time per active cell (the least over its timings) is used for every later
 * launch of that class, by every solver.  A new class larger than a class that kept full-size
 * CTAs, or smaller than one that kept reduced-size CTAs, takes that decision without trials
 * (inherited = 1).  Single-solver steps only (also when replayed from graphs, graph_steps): the
 * batched path and aw_advance_graph use the rules.  aw_get_tuning copies up to `cap` entries (in
 * key order) into `out` and sets *n to the number of entries; aw_reset_tuning forgets them all.
 * AW_EINVAL for a null n or cap < 0. */
#define AW_TUNE_PREDICTOR 0
#define AW_TUNE_FLUX 1
#define AW_TUNE_TRIALS 2
typedef struct aw_tune_entry {
  int32_t dim, M, pde, flux, kernel, size_class;
  int32_t choice;          /* the variant kept, -1 while still trying */
  int32_t trials[2];       /* timings taken of variants 0 and 1 */
  int32_t inherited;       /* 1: decided from a neighbouring class, without trials */
  double ns_per_cell[2];   /* least device time per active cell of variants 0 and 1 */
} aw_tune_entry;
int aw_get_tuning(aw_tune_entry* out, int32_t cap, int32_t* n);
int aw_reset_tuning(void);

/* Stable level-0 time step of the current state (CFL condition over all active cells). */
int aw_compute_dt(aw_solver* s, double* dt0);

/* Regrid from the refinement indicator (Eq. eqn.indicator, Phi = rho) under rules 1-7 of
 * Sec. 3.1.  init_mode = 1 takes new cells from the initial condition, 0 projects the
 * mothers' WENO polynomials. */
int aw_regrid(aw_solver* s, int32_t init_mode);

/* Regrid with caller-supplied flags, one per existing cell in canonical order:
 * +1 refine (honoured on active cells below lmax), -1 recoarsen (honoured on virtual mothers
 * whose children are all active leaves), 0 keep.  The tree that results is a function of the
 * flags alone; this is the hook for bit-exact tree parity. */
int aw_regrid_with_flags(aw_solver* s, const int8_t* flags, int64_t n, int32_t init_mode);

/* Flags the indicator gives for the current state (canonical order), without regridding. */
int aw_compute_flags(aw_solver* s, int32_t init_mode, int8_t* flags, int64_t cap, int64_t* n);

/* Cell counts: all existing cells, active cells, and per level (arrays of 8, may be NULL). */
int aw_get_counts(aw_solver* s, int64_t* n_cells, int64_t* n_active, int64_t* cells_per_level,
                  int64_t* active_per_level);

/* Canonical export of every existing cell: meta (may be NULL) and V averages per cell. */
int aw_read_cells(aw_solver* s, aw_cell* meta, double* u, int64_t cap, int64_t* n);

/* Internal per-level arrays for kernel-level parity (AW_INTERNAL_*), in the level's
 * canonical order.  *n receives the number of doubles. */
int aw_read_internal(aw_solver* s, int32_t what, int32_t level, double* buf, int64_t cap, int64_t* n);

/* Solver time, and total sum(volume * u) over active cells (V doubles). */
int aw_get_time(aw_solver* s, double* t);
int aw_totals(aw_solver* s, double* tot);

/* Number of conserved variables of the configured PDE. */
int aw_num_vars(const aw_solver* s);

/* Reset the mesh to the uniform level-0 grid of active cells with zero averages, t = 0
 * (re-uses the solver's device memory for a new problem). */
int aw_reset(aw_solver* s);

/* Device-memory limit of one solver (no counterpart in the paper; the request loop admits
 * requests by their device bytes with it): an allocation that would take the solver's live
 * device bytes above `bytes` is refused, and the call that needed it returns AW_ELIMIT.  0 (the
 * default) removes the limit.  A call that failed with AW_ELIMIT leaves the solve part way
 * through a step or a regrid: restart it (aw_reset and a new initial condition) or destroy the
 * solver.  aw_reset also clears the record of the refusal.  AW_EINVAL for bytes < 0. */
int aw_set_memory_limit(aw_solver* s, int64_t bytes);

/* Device bytes the solver holds (its own allocations, not the CUDA context): live now, peak
 * since creation, and refused: the live total that the largest refused allocation would have
 * reached (0 if none).  NULL outputs are skipped. */
int aw_get_memory(const aw_solver* s, int64_t* live, int64_t* peak, int64_t* refused);

/* Graph replay of level-0 steps (aw_launch_params.graph_steps; no counterpart in the paper): of
 * the steps of this solver (as a solver, or as the first member of a batch) that ran from a
 * graph, how many launched the previous graph again unchanged (the same launch arguments at every
 * level: the mesh did not change in the regrid before), how many were captured and updated the
 * previous executable graph in place, and how many built one anew.  NULL outputs are skipped. */
int aw_graph_stats(const aw_solver* s, int64_t* reuses, int64_t* updates, int64_t* instantiations);

/* Per-kernel timing: when on, every launch of the hot kernels is bracketed by CUDA events on the
 * solver's stream.  aw_kernel_times() synchronises, returns the accumulated device time (ms) and
 * launch count per kind since the previous call, and restarts the accumulation.
 * Kinds: 0 WENO, 1 predictor, 2 face flux, 3 update, 4 projection of virtual cells (arrays of 8). */
int aw_set_profiling(aw_solver* s, int32_t on);
int aw_kernel_times(aw_solver* s, double* ms, int64_t* launches);

/* Wait for all work of the solver on its stream. */
int aw_sync(aw_solver* s);

/* Kernel launches issued by this solver since creation (device work the library ran). */
int64_t aw_kernel_launches(const aw_solver* s);

/* ------------------------------------------------------------------------------------------
 * Request loop: independent solves (each a full aw_create / aw_set_initial / aw_advance_to of
 * its own configuration) admitted as device memory and worker slots free up; concurrent
 * requests run on their own CUDA streams, so their kernels overlap on the GPU.  Admission is
 * in arrival order against a device-memory budget using an estimate of each solve's footprint
 * (the dense per-level grids plus per-active arrays for a quarter of the finest level).  A
 * finished request's cell averages are kept in host memory and its device memory is released.
 * Results do not depend on the mix: every request runs the same kernels as a solve alone.
 * (Not a passage of the paper: a serving layer around the method.)
 * ------------------------------------------------------------------------------------------ */
typedef struct aw_server aw_server;

#define AW_REQ_QUEUED 0
#define AW_REQ_RUNNING 1
#define AW_REQ_DONE 2
#define AW_REQ_FAILED 3

typedef struct aw_srv_info {
  int64_t cell_updates, level0_steps;
  int64_t footprint_bytes;             /* the device bytes reserved for the run that finished it */
  double queue_ms, run_ms, total_ms;   /* submit -> start of the last run, its start -> done, submit -> done */
  int64_t requeues;                    /* runs restarted because the solve outgrew its reservation */
  int64_t peak_bytes;                  /* the solver's own peak device bytes in the last run */
  int64_t grows;                       /* times its reservation grew in place while it ran */
} aw_srv_info;

typedef struct aw_srv_summary {
  int64_t done, failed, queued, running;
  double p50_ms, p99_ms;               /* time to solution (submit -> done) of finished requests */
  double solves_per_s, cell_updates_per_s;   /* over first submit -> last completion */
  int64_t requeues;                    /* restarts of outgrown runs, all requests */
  int64_t budget_bytes;                /* the loop's device-memory budget */
  int64_t peak_reserved_bytes;         /* the most bytes the admitted runs ever held reserved together */
  int64_t grows;                       /* in-place growths of running requests' reservations */
} aw_srv_summary;

/* Start `max_concurrent` worker threads on the current device with a device-memory budget.
 * Admission by bytes: a request is admitted (oldest first) when its reservation fits what the
 * running requests leave of the budget; its solver runs under that reservation as its memory
 * limit (aw_set_memory_limit, less 64 MiB for the CUDA context and staging).  The first
 * reservation is an estimate: the dense per-level grids exactly, per-active arrays for a quarter
 * of the finest level, or for 1.25 times the largest share of it that finished or refused runs of
 * the same dim, pde, M, lmax and refine_factor held (the loop learns it from their device
 * bytes).  A solve whose mesh refines more than its reservation allows has the reservation grown
 * in place, while it runs, when the budget has room for the growth beside the other running
 * requests (to the bytes it asked for and half again, or just those bytes; aw_srv_info.grows).
 * Otherwise (AW_ELIMIT) it gives its memory back and goes back to the head of the queue with a
 * larger reservation (at least the bytes it was refused, at least twice the old one, at most what
 * every cell of every level active would take), and waits there until the budget has room for
 * it; it then runs again from its initial condition.  So the reservations of running requests
 * never exceed the budget, and a request fails for memory only if it needs more than the whole
 * budget. */
int aw_srv_create(int64_t hbm_budget_bytes, int32_t max_concurrent, aw_server** out);

/* Continuous cross-request batching in the loop (no counterpart in the paper): a worker that
 * admits the oldest queued request also admits up to max_batch - 1 further queued requests (in
 * arrival order) that agree with it in dim, pde, M, flux and refine_factor and fit the remaining
 * budget (end times, grids and depths may differ), and advances the group one lockstep level-0
 * step at a time with aw_step_batch.  A member leaves the group as soon as it reaches its end time
 * or fails: its results are kept and its solver and reservation released.  Between steps the
 * worker admits further such requests into the running group, up to max_batch members, when
 * their reservations fit the budget beside the running requests and the oldest queued request.
 * Every member computes exactly what it computes alone.  1 (the default) turns batching off.
 * Applies to requests admitted after the call.  AW_EINVAL unless 1 <= max_batch <=
 * AW_BATCH_MAX. */
int aw_srv_set_batching(aw_server* srv, int32_t max_batch);
/* Queue one solve (configuration copied; params copied).  AW_EINVAL if its footprint exceeds
 * the whole budget. */
int aw_srv_submit(aw_server* s, const aw_config* cfg, int32_t ic_kind, const double* params, int32_t nparams,
                  double t_end, int64_t* id);
/* State of a request: AW_REQ_*. */
int aw_srv_poll(aw_server* s, int64_t id, int32_t* state);
/* Block until the queue is empty and no request is running. */
int aw_srv_wait_all(aw_server* s);
/* Cells of a finished request in canonical order (as aw_read_cells), and its timings; returns
 * the request's own error code if it failed, AW_ESTATE if it has not finished. */
int aw_srv_result(aw_server* s, int64_t id, aw_cell* meta, double* u, int64_t cap, int64_t* n, aw_srv_info* info);
/* p50/p99 time to solution and throughput of the finished requests. */
int aw_srv_stats(aw_server* s, aw_srv_summary* out);
/* Message of the last failing aw_srv_* call on this thread. */
const char* aw_srv_last_error(void);
/* Drop queued requests, wait for running ones, stop the workers. */
void aw_srv_destroy(aw_server* s);

/* Self-test of the Newton-Raphson reciprocal the kernels use in place of IEEE division
 * (y <- y + y(1 - x y) twice from the hardware's approximate reciprocal): out_dev[k] = that
 * reciprocal of x_dev[k], out_dev[n + k] = 1.0 / x_dev[k] by IEEE division, for k < n (device
 * buffers owned by the caller; out_dev holds 2n doubles).  Asynchronous on `stream`.
 * AW_EINVAL for null pointers or n < 0. */
int aw_selftest_reciprocal(const double* x_dev, int64_t n, double* out_dev, uintptr_t stream);

/* Self-test of the one-step reciprocal and square root of the face fluxes (no counterpart in
 * the paper; both are Newton steps from the hardware's approximations, relative error below
 * 2^-38): out_dev[k] = the one-step reciprocal of x_dev[k], out_dev[n + k] = 1.0 / x_dev[k],
 * out_dev[2n + k] = the one-step square root, out_dev[3n + k] = sqrt(x_dev[k]) (CUDA), for
 * k < n (device buffers owned by the caller; out_dev holds 4n doubles; the square roots want
 * x >= 0).  Asynchronous on `stream`.  AW_EINVAL for null pointers or n < 0. */
int aw_selftest_flux_math(const double* x_dev, int64_t n, double* out_dev, uintptr_t stream);

/* Allocation-free CFL time step of a uniform grid (the paper has no counterpart; this is a
 * convenience for callers that cannot allocate device memory when they need it, such as code
 * inside a framework that owns every device allocation through its own pool, or a time loop
 * that must not pay the implicit synchronisation of cudaMalloc/cudaFree).
 * Computes min over the cells of CFL / sum_d(s_d / dx_d) (the same formula as aw_compute_dt)
 * for the level-0 grid of `cfg` (nx*ny[*nz] cells, spacing from lo/hi) and writes it to the
 * device double `dt_dev`, asynchronously on `stream`.
 *   u_dev:   device pointer, cell averages as a structure of arrays u[v * n_cells + c], cells in
 *            canonical order (k, j, i); read only.
 *   n_cells: must equal the grid's cell count and be at most 8192 * 256 = 2,097,152
 *            (AW_EINVAL otherwise, before any device work).
 * Result values that aw_compute_dt rejects: the result is only known on the device, so where
 * aw_compute_dt returns AW_ENONPHYSICAL this call still returns AW_OK and writes the rejected
 * value to dt_dev: 0 when some cell's step is NaN or not positive (NaN averages, for example),
 * and a value of at least 1e300 (1e300 or +inf) when no wave speed limits the step (every speed
 * zero).  Like aw_compute_dt it does not test rho > 0 or p > 0: a cell with c^2 < 0 gets the
 * modulus of its complex wave speeds.  The caller checks the value before stepping with it.
 * Scratch: a fixed 64 KiB array in the library's device memory, which every GPU that loads the
 * library holds until the process exits.  The first call on a device looks up its address
 * (make that call before any stream capture).  The array is shared: calls whose device work
 * overlaps (different streams, or threads) race on it and must be serialised by the caller.
 * Nothing is allocated or freed. */
int aw_cfl_dt_noalloc(const aw_config* cfg, const double* u_dev, int64_t n_cells, double* dt_dev, uintptr_t stream);

/* Reference-element tables the kernels use for order M (1..3) and refinement factor r (2..4),
 * computed on the host in long double and rounded to double; no device work, no solver needed.
 * They are the Gauss-Legendre rule on [0,1] and the nodal Lagrange basis through it (Sec. 2.2);
 * the WENO stencils of Eq. eqn.stencildef with their reconstruction matrices (the inverse of
 * the integral-conservation system of Eq. eqn.rec.x) and the oscillation-indicator matrix of
 * Eq. eqn.sigmas; the time block of the predictor matrix K1 of Sec. 2.3 in its factorised
 * form; and the child-box averages and fine-point values of the basis used by the projection
 * of Sec. 3.1.3.  With N = M + 1, out[] receives, in this order:
 *   N, Ns (number of stencils), r;
 *   x[N], w[N]                 nodes and weights;
 *   SL[4], lam[4]              left extent and linear weight of stencil s (unused entries 0);
 *   Ainv[4][N][N]              Ainv[s][p][e]: nodal value p of the polynomial of stencil s from
 *                              the averages of its cells e = 0..N-1 (leftmost first);
 *   Sig[N][N]                  sigma = c^T Sig c for nodal coefficients c;
 *   Dm[N][N]                   Dm[i][l] = psi_l'(x_i);
 *   G[N][N]                    K_t^{-1} diag(w), K_t[a][b] = psi_a(1) psi_b(1) - w_b Dm[b][a];
 *   psi0[N], psi1[N]           psi_l(0), psi_l(1);
 *   Wc[r][N]                   Wc[c][l]: average of psi_l over [c/r, (c+1)/r];
 *   Pf[r][N][N]                Pf[c][i][l] = psi_l((c + x_i)/r);
 *   Pt[r][N]                   Pt[k][l] = psi_l(k/r);
 *   gsum[N]                    row sums of G;
 *   Bq[4][N-1][N-1]            sigma of stencil s as a quadratic form of the differences d of its
 *                              other cells' averages to the centre cell's: sigma = sum_{i<=j}
 *                              Bq[s][i][j] d_i d_j (the upper triangle of Ainv^T Sig Ainv, with
 *                              the centre cell's row and column removed, off-diagonal doubled);
 * 11 + 5N + 7N^2 + 2rN + rN^2 + 4(N-1)^2 doubles, written to *n.  AW_EINVAL for M or r out of
 * range, a null n, or cap < *n (out untouched). */
int aw_tables_host(int32_t M, int32_t r, double* out, int64_t cap, int64_t* n);

#ifdef __cplusplus
}
#endif
#endif
