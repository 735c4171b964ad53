// aw_ops.h -- launch table of the templated hot kernels for one (D, M, PDE) configuration.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

struct aw_solver;

namespace aw {
struct HotArgs;
struct HotBatch;

struct HotOps {
  int D, M, PDE, V;
  // WENO tile edge of a level of n cells (8x8 tiles in 2D unless the level is small, 4x4x4 in 3D)
  int (*weno_tile)(long long n);
  // each launcher returns the number of kernels it launched (0 when there was no work)
  int (*weno)(const HotArgs&, cudaStream_t);
  int (*predict)(const HotArgs&, cudaStream_t);
  int (*flux)(const HotArgs&, cudaStream_t);
  int (*update)(const HotArgs&, cudaStream_t);
  // the face flux and the update in one launch (k_flux_update), bitwise what flux + update give
  int (*flux_update)(const HotArgs&, cudaStream_t);
  // project virtual cells (vlist, nv) from mother dofs `src` (space-time if spacetime != 0,
  // else spatial WENO dofs), into the dense averages (dense != 0) or into out[k*V + v]
  int (*project)(const HotArgs&, const int32_t* vlist, int nv, const double* src, int spacetime,
                 double* out, int dense, cudaStream_t);
  // the same kernels over all members of a batch (b.n and b.a[] set by the caller; the launcher
  // fills b.start); the projection takes each member's vlist/nv and mother predictor qhm
  int (*weno_b)(HotBatch&, cudaStream_t);
  int (*predict_b)(HotBatch&, cudaStream_t);
  int (*flux_b)(HotBatch&, cudaStream_t);
  int (*update_b)(HotBatch&, cudaStream_t);
  int (*flux_update_b)(HotBatch&, cudaStream_t);
  // the persistent level kernel of a batch (k_level_batch): projection, WENO, predictor and (with
  // with_flux) the fused face flux and update in one cooperative launch; -1 when it cannot be
  // launched (the separate launches then run), NULL for configurations where the predictor and
  // the face flux differ in CTA shape
  int (*level_b)(HotBatch&, int with_flux, cudaStream_t);
  int (*project_b)(HotBatch&, cudaStream_t);
};

// returns false when the configuration is not compiled in
bool get_ops(int D, int M, int PDE, HotOps* out);

// launch-shape rules (aw_set_launch_params): WENO by passes from pass_min_cells cells per level,
// 2D WENO tiles of 8x8 from tile8_min_cells, reduced-size predictor/flux CTAs when the full-size
// ones give fewer than small_ctas_per_sm CTAs per SM, the face flux and the update fused into one
// launch (fuse_flux_update != 0) or two, the autotuner of the predictor's and the face flux's CTA
// sizes (autotune != 0; it replaces the small_ctas_per_sm rule where it has decided), the
// persistent level kernel of batches (persistent != 0), and level-0 steps of AMR solves and of
// batches replayed from captured CUDA graphs (graph_steps != 0).
// Process-wide; the results never depend on them, only the speed.
struct LaunchParams {
  long long pass_min_cells, tile8_min_cells;
  int small_ctas_per_sm;
  int fuse_flux_update;
  int autotune;
  int persistent;
  int graph_steps;
};
LaunchParams launch_params();
void set_launch_params(const LaunchParams& p);

// The request loop's hook on a solver's memory limit: called when an allocation would take the
// solver's live device bytes to `need`, above its limit; returns the new limit (>= need) when the
// loop has grown the solve's reservation by that much, or 0 to refuse (the allocation then fails
// and the call returns AW_ELIMIT).  Called on the thread that advances the solver.
typedef int64_t (*GrowFn)(void* ctx, int64_t need);
void set_grow_hook(aw_solver* s, GrowFn fn, void* ctx);
}  // namespace aw
