// aw_ops.cu -- selects the compiled hot-kernel instantiation for a configuration; holds the
// process-wide launch-shape rules.
#include <atomic>

#include "aw_ops.h"

namespace aw {
HotOps ops_2_1_0();
HotOps ops_2_1_2();
HotOps ops_2_2_0();
HotOps ops_2_3_0();
HotOps ops_3_2_0();
HotOps ops_2_2_1();
HotOps ops_2_3_1();
HotOps ops_2_2_2();
HotOps ops_2_3_2();
HotOps ops_3_2_2();

static std::atomic<long long> g_pass_min_cells{4096}, g_tile8_min_cells{20000};
static std::atomic<int> g_small_ctas_per_sm{2};
static std::atomic<int> g_fuse_flux_update{1};
static std::atomic<int> g_autotune{1};
static std::atomic<int> g_persistent{0};
static std::atomic<int> g_graph_steps{0};

LaunchParams launch_params() {
  LaunchParams p;
  p.pass_min_cells = g_pass_min_cells.load();
  p.tile8_min_cells = g_tile8_min_cells.load();
  p.small_ctas_per_sm = g_small_ctas_per_sm.load();
  p.fuse_flux_update = g_fuse_flux_update.load();
  p.autotune = g_autotune.load();
  p.persistent = g_persistent.load();
  p.graph_steps = g_graph_steps.load();
  return p;
}

void set_launch_params(const LaunchParams& p) {
  g_pass_min_cells.store(p.pass_min_cells);
  g_tile8_min_cells.store(p.tile8_min_cells);
  g_small_ctas_per_sm.store(p.small_ctas_per_sm);
  g_fuse_flux_update.store(p.fuse_flux_update);
  g_autotune.store(p.autotune);
  g_persistent.store(p.persistent);
  g_graph_steps.store(p.graph_steps);
}

bool get_ops(int D, int M, int PDE, HotOps* out) {
  int key = D * 100 + M * 10 + PDE;
  switch (key) {
    case 210: *out = ops_2_1_0(); return true;
    case 212: *out = ops_2_1_2(); return true;
    case 220: *out = ops_2_2_0(); return true;
    case 230: *out = ops_2_3_0(); return true;
    case 320: *out = ops_3_2_0(); return true;
    case 221: *out = ops_2_2_1(); return true;
    case 231: *out = ops_2_3_1(); return true;
    case 222: *out = ops_2_2_2(); return true;
    case 232: *out = ops_2_3_2(); return true;
    case 322: *out = ops_3_2_2(); return true;
  }
  return false;
}
}  // namespace aw
