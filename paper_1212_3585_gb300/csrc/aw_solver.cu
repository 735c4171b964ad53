// aw_solver.cu -- solver state, local time stepping scheduler, AMR bookkeeping kernels and the
// C ABI of include/aderweno.h.
//
// Data layout (GB300-first; one GPU holds the whole mesh): every level l is a dense grid of
// n*r^l cells per direction (Sec. 3.1: Delta x_l = r Delta x_{l+1}) with a status byte per cell
// (ST_NONE where no cell exists), the cell averages as a structure of arrays, and an active-id
// map.  Compact per-level lists (active, virtual child, virtual mother, existing cells, tiles)
// are rebuilt after every regrid by an order-preserving stream compaction, so every list is in
// canonical order (k, j, i) and every result is deterministic.  The per-active FP64 arrays
// (WENO dofs, predictor dofs, face fluxes, memory variables) are indexed by the active id.
//
// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the solver's stream, from
// the device's default pool, which keeps freed blocks for reuse): creating or destroying a solver
// does not synchronise the device, so the solves of a request loop keep running while others
// start and finish.  The two small pinned host buffers of a solver come from a process-wide free
// list for the same reason.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>
#include <string>
#include <vector>

#include "aderweno.h"
#include "aw_device.cuh"
#include "aw_ops.h"

namespace aw {
bool build_tables(int M, int r, Tables* T);
}
using namespace aw;

static thread_local std::string g_err = "";

#define AW_FAIL(code, ...)                        \
  do {                                            \
    char b_[600];                                 \
    snprintf(b_, sizeof b_, __VA_ARGS__);         \
    g_err = b_;                                   \
    return code;                                  \
  } while (0)
#define CK(x)                                                                                          \
  do {                                                                                                 \
    cudaError_t e_ = (x);                                                                              \
    if (e_ != cudaSuccess) AW_FAIL(AW_ECUDA, "%s: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)
#define TRY(x)                \
  do {                        \
    int rc_ = (x);            \
    if (rc_ != AW_OK) return rc_; \
  } while (0)

static const int CHUNK = 4096;
// device count slots per level (active, virtual child, virtual mother, existing, tiles, high
// faces, x-sweep rows, y-sweep cells); the error word follows the last level's slots
static const int NSLOT = 8;

// stream-ordered device allocation on the solver's stream

// the default pool of a device keeps freed memory for reuse instead of returning it at every
// synchronisation (set once per device)
static std::mutex g_pool_mu;
static bool g_pool_ready[64];
static void keep_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (dev < 0 || dev >= 64 || g_pool_ready[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  g_pool_ready[dev] = true;
}

// 256-byte pinned host blocks, allocated once per process and recycled
static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;
static void* pinned_block() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (!g_pin_free.empty()) {
    void* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
  }
  void* p = nullptr;
  return cudaMallocHost(&p, 256) == cudaSuccess ? p : nullptr;
}
static void pinned_release(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

struct Level {
  int L[3] = {1, 1, 1};
  long long n = 0;
  double dx[3] = {1, 1, 1};
  int8_t *st = nullptr, *R = nullptr, *nst = nullptr, *flag = nullptr;
  double *u = nullptr, *chi = nullptr;
  int32_t *aid = nullptr, *alist = nullptr, *vlist = nullptr, *mlist = nullptr, *clist = nullptr;
  int na = 0, nv = 0, nm = 0, nc = 0;
  int ts = 4;                  // WENO tile edge
  int tdim[3] = {1, 1, 1};
  long long ntd = 0;
  int8_t* tflag = nullptr;
  int32_t* tiles = nullptr;
  int ntiles = 0;
  double *wh = nullptr, *qh = nullptr, *fl = nullptr, *mem = nullptr;
  int8_t* xmark = nullptr;     // WENO by passes: rows whose x sweep feeds an active cell (dense)
  int32_t* xslot = nullptr;    // dense cell -> position in xlist, -1 elsewhere
  int32_t* xlist = nullptr;    // those rows (dense indices), canonical order
  double* xs = nullptr;        // their x sweeps [slot][V][N]
  int nx = 0;
  long long xlcap = 0, xcap = 0;  // capacities of xlist and xs (rows)
  int8_t* ymark = nullptr;     // 3D: cells whose y sweeps feed an active cell (dense)
  int32_t* yslot = nullptr;
  int32_t* ylist = nullptr;
  double* ys = nullptr;        // their y sweeps [slot][V][N][N]
  int ny = 0;
  long long ylcap = 0, ycap = 0;
  int8_t* hflag = nullptr;     // per (axis, active id): the high face needs computing
  int32_t* hflist = nullptr;   // compacted high faces, axis * na + active id
  int nh = 0;
  int32_t* fsync = nullptr;    // arrival counters of the fused face flux and update, per chunk
  long long cap = 0;
};

// device-side time stepping state of aw_advance_graph (see k_dt_commit)
struct GState {
  double t, t_end, last_dt0;
  long long nsteps;
  int stop;
};

// An executable graph of one level-0 step (graph_steps) and what it was captured from: the
// launch arguments of every level (a step with the same arguments launches the same kernels with
// the same parameters: the time steps and the mesh live in device memory), whether it can run
// again as it is (it holds no timing events: no profiling, no trial of the autotuner), and the
// kernel launches it holds.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<char> sig;
  bool reusable = false;
  int64_t launches = 0;
};

struct aw_solver {
  aw_config cfg;
  int D, V, N, M, r, lmax, NSP, NST, P;
  cudaStream_t stream;
  Tables T;
  Phys phys;
  HotOps ops;
  Level lev[MAXL];
  double t = 0.0;
  int ic = -1;
  std::vector<double> icp;
  double* d_dtl = nullptr;
  unsigned long long* d_dtmin = nullptr;
  GState* d_gs = nullptr;           // device-side time stepping of aw_advance_graph
  GState* h_gs = nullptr;
  cudaStream_t gstream = nullptr;   // capture and replay stream of aw_advance_graph
  cudaGraphExec_t gexec = nullptr;  // its instantiated graph, reused while the arguments match
  HotArgs gargs;
  int gchunk = 0;
  bool gfused = false;
  // level-0 steps of AMR solves and batches replayed from CUDA graphs (aw_launch_params.graph_steps):
  // the graphs of the last single-solver and batched step (captured on gstream), an event that
  // orders the capture stream after the caller's stream and back, flags set while a step is
  // being captured and when the capture took timing events, and the counts of aw_graph_stats
  StepGraph sgraph, bgraph;
  cudaEvent_t gev = nullptr;
  bool capturing = false, captured_events = false;
  int64_t graph_reuses = 0, graph_updates = 0, graph_instantiations = 0;
  int* d_err = nullptr;
  int* d_cnt = nullptr;
  int* h_cnt = nullptr;
  double* h_dtl = nullptr;
  int* d_bcnt = nullptr;
  long long bcnt_cap = 0;
  double* d_buf = nullptr;
  long long buf_cap = 0;
  int64_t launches = 0;
  // optional per-kernel timing with CUDA events on the solver's stream
  int prof = 0;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  double kind_ms[8] = {0};
  int64_t kind_n[8] = {0};
  // device memory of the solver: bytes of every live allocation, their sum and its maximum, an
  // optional limit (aw_set_memory_limit; 0: none) and the largest total a refused allocation
  // would have reached
  std::unordered_map<void*, size_t> alloc_bytes;
  int64_t mem_live = 0, mem_peak = 0, mem_limit = 0, mem_refused = 0;
  // the request loop's hook that may raise the limit instead of refusing (aw::set_grow_hook)
  aw::GrowFn grow = nullptr;
  void* grow_ctx = nullptr;
  // the autotuner's timed trial launches of this solver, read after the next synchronisation
  struct TunePending {
    int key[6];
    int var;
    long long na;
    cudaEvent_t a, b;
  };
  std::vector<TunePending> tune_used;
};

// Stream-ordered device allocation on the solver's stream, counted against the solver's memory
// limit: an allocation that would take the live total above the limit is refused (the caller
// then fails with AW_ELIMIT, see oom_code).
static cudaError_t dalloc(aw_solver* s, void** p, size_t bytes) {
  if (!bytes) bytes = 1;
  if (s->mem_limit > 0 && s->mem_live + (int64_t)bytes > s->mem_limit) {
    const int64_t need = s->mem_live + (int64_t)bytes;
    const int64_t grown = s->grow ? s->grow(s->grow_ctx, need) : 0;
    if (grown >= need) {
      s->mem_limit = grown;
    } else {
      s->mem_refused = std::max(s->mem_refused, need);
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, s->stream);
  if (e != cudaSuccess) return e;
  s->alloc_bytes[*p] = bytes;
  s->mem_live += (int64_t)bytes;
  s->mem_peak = std::max(s->mem_peak, s->mem_live);
  return cudaSuccess;
}

static void dfree(aw_solver* s, void* p) {
  if (!p) return;
  auto it = s->alloc_bytes.find(p);
  if (it != s->alloc_bytes.end()) {
    s->mem_live -= (int64_t)it->second;
    s->alloc_bytes.erase(it);
  }
  cudaFreeAsync(p, s->stream);
}

// the status of a failed device allocation: AW_ELIMIT once the solver's own limit refused one
static int oom_code(const aw_solver* s) { return s->mem_refused ? AW_ELIMIT : AW_ENOMEM; }

enum { KIND_WENO = 0, KIND_PREDICT = 1, KIND_FLUX = 2, KIND_UPDATE = 3, KIND_PROJECT = 4 };

static cudaEvent_t take_event(aw_solver* s) {
  if (!s->ev_free.empty()) {
    cudaEvent_t e = s->ev_free.back();
    s->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// record a timing event on the solver's stream; inside a captured step as an event-record node,
// which records when the graph runs
static void record(aw_solver* s, cudaEvent_t e) {
  if (s->capturing) {
    cudaEventRecordWithFlags(e, s->stream, cudaEventRecordExternal);
    s->captured_events = true;
  } else {
    cudaEventRecord(e, s->stream);
  }
}

// run one hot launcher, bracketed by events when profiling
template <class F>
static int timed(aw_solver* s, int kind, F&& launch) {
  if (!s->prof) return launch();
  cudaEvent_t a = take_event(s), b = take_event(s);
  record(s, a);
  int n = launch();
  record(s, b);
  if (n > 0) s->ev_used.push_back({kind, {a, b}});
  else { s->ev_free.push_back(a); s->ev_free.push_back(b); }
  s->kind_n[kind] += n;
  return n;
}

// ---- autotuner of the CTA sizes of the predictor and the face flux (aw_get_tuning) ----
// Both kernels have a full-size and a reduced-size CTA variant (about a quarter of the cells or
// faces, as many as fill whole warps) that compute bitwise the same results.  Per (dim, M, pde,
// numerical flux, kernel, level size class) the first launches
// alternate the two, each timed with an event pair on the solver's stream; once each has
// AW_TUNE_TRIALS timings, the variant with the least device time per active cell (the least over
// its timings, which leaves out a first launch's one-off costs) is used for that class by every
// solver of the process.  A class larger than one that kept full-size CTAs keeps them too, and a
// class smaller than one that kept reduced-size CTAs keeps those, without trials (more cells give
// more CTAs, which only favours the larger CTAs): so trials run only between the two.
struct TuneState {
  int issued[2] = {0, 0}, trials[2] = {0, 0};
  double ns_per_cell[2] = {0.0, 0.0};
  int choice = -1;
  int inherited = 0;
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int, int, int>, TuneState> g_tune;

static std::tuple<int, int, int, int, int, int> tune_key(const int* k) {
  return std::make_tuple(k[0], k[1], k[2], k[3], k[4], k[5]);
}

static int size_class(long long n) {
  int c = 0;
  while (n > 1) {
    n >>= 1;
    c++;
  }
  return c;
}

// The variant of a launch of `kernel` over `na` active cells: the kept one (0 or 1), or while the
// class is being tried the one launched fewer times so far, with bit 1 set (a timed trial);
// -1 when the tuner is off.
static int tune_pick(const aw_solver* s, int kernel, long long na, int* key) {
  if (!launch_params().autotune || na <= 0) return -1;
  key[0] = s->D;
  key[1] = s->M;
  key[2] = s->cfg.pde;
  key[3] = s->cfg.flux;
  key[4] = kernel;
  key[5] = size_class(na);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneState& t = g_tune[tune_key(key)];
  if (t.choice >= 0) return t.choice;
  if (t.issued[0] + t.issued[1] == 0) {
    // a new class: decided by a smaller class that kept full-size CTAs or a larger one that kept
    // reduced-size CTAs
    for (const auto& kv : g_tune) {
      const auto& k2 = kv.first;
      if (std::get<0>(k2) != key[0] || std::get<1>(k2) != key[1] || std::get<2>(k2) != key[2] ||
          std::get<3>(k2) != key[3] || std::get<4>(k2) != key[4] || kv.second.choice < 0)
        continue;
      const int c2 = std::get<5>(k2);
      if ((c2 < key[5] && kv.second.choice == 0) || (c2 > key[5] && kv.second.choice == 1)) {
        t.choice = kv.second.choice;
        t.inherited = 1;
        return t.choice;
      }
    }
  }
  const int v = t.issued[1] < t.issued[0] ? 1 : 0;
  t.issued[v]++;
  return v | 2;
}

// the CTA size of a launch for the tuner's variant (0: the launch rules)
static int tune_div(int v) { return v < 0 ? 0 : ((v & 1) ? 4 : 1); }

// run a launch; time it with an event pair when it is a trial of the tuner
template <class F>
static int tuned(aw_solver* s, int v, const int* key, long long na, F&& launch) {
  if (v < 0 || !(v & 2)) return launch();
  cudaEvent_t a = take_event(s), b = take_event(s);
  record(s, a);
  const int n = launch();
  record(s, b);
  if (n > 0) {
    aw_solver::TunePending p;
    for (int i = 0; i < 6; i++) p.key[i] = key[i];
    p.var = v & 1;
    p.na = na;
    p.a = a;
    p.b = b;
    s->tune_used.push_back(p);
  } else {
    s->ev_free.push_back(a);
    s->ev_free.push_back(b);
  }
  return n;
}

// read the solver's finished trials (after a synchronisation of its stream) into the tuner
static void tune_harvest(aw_solver* s) {
  if (s->tune_used.empty()) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& p : s->tune_used) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      TuneState& t = g_tune[tune_key(p.key)];
      const double ns = 1e6 * (double)ms / (double)p.na;
      if (t.choice < 0) {
        t.ns_per_cell[p.var] = t.trials[p.var] ? std::min(t.ns_per_cell[p.var], ns) : ns;
        t.trials[p.var]++;
        if (t.trials[0] >= AW_TUNE_TRIALS && t.trials[1] >= AW_TUNE_TRIALS)
          t.choice = t.ns_per_cell[1] < t.ns_per_cell[0] ? 1 : 0;
      }
    }
    s->ev_free.push_back(p.a);
    s->ev_free.push_back(p.b);
  }
  s->tune_used.clear();
}

static void harvest_events(aw_solver* s) {
  for (auto& e : s->ev_used) {
    float ms = 0.f;
    cudaEventSynchronize(e.second.second);
    cudaEventElapsedTime(&ms, e.second.first, e.second.second);
    s->kind_ms[e.first] += ms;
    s->ev_free.push_back(e.second.first);
    s->ev_free.push_back(e.second.second);
  }
  s->ev_used.clear();
}

// ------------------------------------------------------------------------------------------
// runtime-generic device helpers for the bookkeeping kernels
// ------------------------------------------------------------------------------------------
struct RtPhys {
  int pde, D, V;
  Phys P;
};

__device__ double rt_pressure(const RtPhys& R, const double* q) {
  double g = R.P.gamma;
  if (R.pde == PDE_EULER) {
    double m2 = 0.0;
    for (int a = 0; a < R.D; a++) m2 += q[1 + a] * q[1 + a];
    return (g - 1.0) * (q[R.D + 1] - 0.5 * m2 / q[0]);
  }
  if (R.pde == PDE_MHD) {
    double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    return (g - 1.0) * (q[4] - 0.5 * m2 / q[0] - 0.5 * B2);
  }
  return 1.0;
}

__device__ double rt_speed(const RtPhys& R, const double* q, int n) {
  if (R.pde == PDE_LINADV) return fabs(R.P.adv[n]);
  double p = rt_pressure(R, q);
  double vn = fabs(q[1 + n] / q[0]);
  if (R.pde == PDE_EULER) {
    double c2 = R.P.gamma * p / q[0];
    return c2 >= 0.0 ? vn + sqrt(c2) : sqrt(vn * vn - c2);
  }
  double a2 = R.P.gamma * p / q[0];
  double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  double b2 = B2 / q[0], bn2 = q[5 + n] * q[5 + n] / q[0];
  double s = a2 + b2;
  double c = vn + sqrt(0.5 * (s + sqrt(s * s - 4.0 * a2 * bn2)));
  return c > R.P.c_h ? c : R.P.c_h;
}

__device__ __forceinline__ void cell_coords(const LevelView& L, long long di, int* ijk) {
  ijk[0] = (int)(di % L.L[0]);
  ijk[1] = (int)((di / L.L[0]) % L.L[1]);
  ijk[2] = (int)(di / ((long long)L.L[0] * L.L[1]));
}

// ---- initial conditions (Sec. 4) ----
struct IcArgs {
  int kind, np;
  double p[128];
  RtPhys R;
  double lo[3], hi[3];
  double x[MAXN], w[MAXN];
  int N;
};

__device__ void ic_point(const IcArgs& I, const double* x, double* q) {
  const int D = I.R.D, V = I.R.V;
  double w[MAXV];
  for (int v = 0; v < MAXV; v++) w[v] = 0.0;
  const double* p = I.p;
  const double g = I.R.P.gamma;
  const int ip = (I.R.pde == PDE_EULER) ? D + 1 : 4;  // index of the pressure in the primitive state
  switch (I.kind) {
    case AW_IC_CONST:
      for (int v = 0; v < V; v++) w[v] = p[v];
      break;
    case AW_IC_VORTEX: {
      double dx = x[0] - p[1], dy = x[1] - p[2], r2 = dx * dx + dy * dy;
      double dT = -p[0] * p[0] * (g - 1.0) / (8.0 * g * M_PI * M_PI) * exp(1.0 - r2);
      double e = p[0] / (2.0 * M_PI) * exp(0.5 * (1.0 - r2));
      w[0] = p[3] * pow(1.0 + dT, 1.0 / (g - 1.0));
      w[1] = p[4] - dy * e;
      w[2] = p[5] + dx * e;
      w[ip] = p[6] * pow(1.0 + dT, g / (g - 1.0));
      break;
    }
    case AW_IC_EXPLOSION: {
      double r2 = 0.0;
      for (int a = 0; a < D; a++) r2 += x[a] * x[a];
      bool in = sqrt(r2) <= p[0];
      w[0] = in ? p[1] : p[3];
      w[ip] = in ? p[2] : p[4];
      break;
    }
    case AW_IC_OT:
      w[0] = g * g; w[1] = -sin(x[1]); w[2] = sin(x[0]); w[3] = 0.0; w[4] = g;
      w[5] = -sin(x[1]); w[6] = sin(2.0 * x[0]); w[7] = 0.0; w[8] = 0.0;
      break;
    case AW_IC_RP4: {
      int qd = (x[0] > p[0]) ? ((x[1] > p[1]) ? 0 : 3) : ((x[1] > p[1]) ? 1 : 2);
      const double* s = p + 2 + 4 * qd;
      w[0] = s[0]; w[1] = s[1]; w[2] = s[2]; w[ip] = s[3];
      break;
    }
    case AW_IC_FOURIER: {
      for (int v = 0; v < V; v++) w[v] = p[v];
      int nm = (int)p[V];
      for (int m = 0; m < nm; m++) {
        const double* md = p + V + 1 + 6 * m;
        double ph = md[5];
        for (int a = 0; a < D; a++) ph += 2.0 * M_PI * md[1 + a] * (x[a] - I.lo[a]) / (I.hi[a] - I.lo[a]);
        w[(int)md[0]] += md[4] * sin(ph);
      }
      break;
    }
  }
  // primitive -> conserved
  if (I.R.pde == PDE_LINADV) { q[0] = w[0]; return; }
  if (I.R.pde == PDE_EULER) {
    double ke = 0.0;
    q[0] = w[0];
    for (int a = 0; a < D; a++) { q[1 + a] = w[0] * w[1 + a]; ke += w[1 + a] * w[1 + a]; }
    q[D + 1] = w[D + 1] / (g - 1.0) + 0.5 * w[0] * ke;
    return;
  }
  double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  double B2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
  q[0] = w[0]; q[1] = w[0] * w[1]; q[2] = w[0] * w[2]; q[3] = w[0] * w[3];
  q[4] = w[4] / (g - 1.0) + 0.5 * w[0] * v2 + 0.5 * B2;
  q[5] = w[5]; q[6] = w[6]; q[7] = w[7]; q[8] = w[8];
}

// IC cell averages by the (M+1)^d-point Gauss rule.  mode 0: every existing cell; mode 1: cells
// that exist in `stn` but not in `sto` (new cells of an initial-condition regrid).
__global__ void k_ic(LevelView L, IcArgs I, const int8_t* sto, const int8_t* stn, int mode) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  if (mode == 0 && L.st[c] == ST_NONE) return;
  if (mode == 1 && !(sto[c] == ST_NONE && stn[c] != ST_NONE)) return;
  int ijk[3];
  cell_coords(L, c, ijk);
  const int D = I.R.D, V = I.R.V, N = I.N;
  double acc[MAXV];
  for (int v = 0; v < V; v++) acc[v] = 0.0;
  int nq = 1;
  for (int a = 0; a < D; a++) nq *= N;
  for (int g = 0; g < nq; g++) {
    int t = g;
    double x[3] = {0, 0, 0}, wt = 1.0, q[MAXV];
    for (int a = 0; a < D; a++) {
      int gi = t % N;
      t /= N;
      x[a] = I.lo[a] + (ijk[a] + I.x[gi]) * L.dx[a];
      wt *= I.w[gi];
    }
    ic_point(I, x, q);
    for (int v = 0; v < V; v++) acc[v] += wt * q[v];
  }
  for (int v = 0; v < V; v++) L.u[v * L.n + c] = acc[v];
}

// ---- CFL time step: min over active cells of r^l * CFL / sum_d(s_d / dx_d) ----
__global__ void k_dt(LevelView L, const int32_t* alist, int na, RtPhys R, double cfl, double rl,
                     unsigned long long* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  double dt = 1e300;
  if (k < na) {
    long long di = alist[k];
    double q[MAXV];
    for (int v = 0; v < R.V; v++) q[v] = L.u[v * L.n + di];
    double den = 0.0;
    for (int a = 0; a < R.D; a++) den += rt_speed(R, q, a) / L.dx[a];
    dt = rl * cfl / den;
    if (!(dt > 0.0)) dt = 0.0;  // NaN or negative: report a zero step
  }
  for (int o = 16; o > 0; o >>= 1) dt = fmin(dt, __shfl_xor_sync(0xffffffffu, dt, o));
  if ((threadIdx.x & 31) == 0 && dt < 1e300) atomicMin(out, (unsigned long long)__double_as_longlong(dt));
}

// ---- device-side time step of a uniform mesh (aw_advance_graph): the host logic of step_cfl on
// one thread -- dt0 from the CFL reduction, clipped at t_end, the time advanced, the level time
// steps dt0 / r^l written -- so that level-0 steps need no host synchronisation.  A step after
// t_end, after a non-physical update or without a stable time step gets dt = 0 (the update leaves
// the averages unchanged) ----
__global__ void k_dt_commit(unsigned long long* dtmin, GState* g, double* dtl, int r, int* err) {
  const double h = __longlong_as_double((long long)*dtmin);
  *dtmin = (unsigned long long)__double_as_longlong(1e300);
  double dt = 0.0;
  if (!g->stop && (*err & 1)) g->stop = 1;
  if (!g->stop && g->t < g->t_end) {
    if (!(h > 0.0) || h >= 1e300) {
      atomicOr(err, 8);
      g->stop = 1;
    } else {
      const double t = g->t;
      const bool clip = t + h >= g->t_end;
      dt = clip ? g->t_end - t : h;
      g->t = clip ? g->t_end : t + dt;
      g->nsteps++;
      g->last_dt0 = dt;
    }
  }
  for (int l = 0; l < MAXL; l++) {
    dtl[l] = dt;
    dt /= r;
  }
}

// ---- averaging (Eq. eqn.average): virtual mothers of level l from level l+1, children summed in
// canonical order ----
__global__ void k_average(LevelView L, LevelView Lc, const int32_t* mlist, int nm, int V, int D, int r) {
  int it = blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= nm * V) return;
  int k = it / V, v = it % V;
  long long di = mlist[k];
  int ijk[3];
  cell_coords(L, di, ijk);
  double s = 0.0;
  int rz = D == 3 ? r : 1;
  for (int kk = 0; kk < rz; kk++)
    for (int jj = 0; jj < r; jj++)
      for (int ii = 0; ii < r; ii++)
        s += Lc.u[v * Lc.n + didx(Lc, r * ijk[0] + ii, r * ijk[1] + jj, D == 3 ? r * ijk[2] + kk : 0)];
  double rd = 1.0;
  for (int a = 0; a < D; a++) rd *= r;
  L.u[v * L.n + di] = s / rd;
}

// ---- refinement indicator (Eq. eqn.indicator), Phi = rho, undivided differences on the 3^d
// same-level box; see the solver documentation for the discrete form ----
__device__ __forceinline__ double phi(const LevelView& L, const Bc6& bc6, const int* ijk, int D, int a, int sa, int b,
                                      int sb) {
  int c[3] = {ijk[0], ijk[1], ijk[2]};
  c[a] += sa;
  c[b] += sb;
  int m[3] = {0, 0, 0};
  for (int e = 0; e < D; e++) {
    if (beyond_inflow(L.L, bc6.v, e, c[e])) return bc6.inflow_rho;
    bcmap(L.L, bc6.v, e, c[e], &m[e]);
  }
  return L.u[didx(L, m[0], m[1], m[2])];
}

__global__ void k_indicator(LevelView L, Bc6 bc6, int D, double eps, double* chi) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int8_t s = L.st[c];
  if (s != 0 && s != -1) { chi[c] = 0.0; return; }
  int ijk[3];
  cell_coords(L, c, ijk);
  double P0 = L.u[c], num = 0.0, den = 0.0;
  for (int k = 0; k < D; k++)
    for (int l = 0; l < D; l++) {
      double d2, g, a;
      if (k == l) {
        double Pp = phi(L, bc6, ijk, D, k, 1, k, 0), Pm = phi(L, bc6, ijk, D, k, -1, k, 0);
        d2 = Pp - 2.0 * P0 + Pm;
        g = fabs(Pp - P0) + fabs(P0 - Pm);
        a = fabs(Pp) + 2.0 * fabs(P0) + fabs(Pm);
      } else {
        double Ppp = phi(L, bc6, ijk, D, k, 1, l, 1), Ppm = phi(L, bc6, ijk, D, k, 1, l, -1);
        double Pmp = phi(L, bc6, ijk, D, k, -1, l, 1), Pmm = phi(L, bc6, ijk, D, k, -1, l, -1);
        d2 = (Ppp - Ppm - Pmp + Pmm) / 4.0;
        g = (fabs(Ppp - Pmp) + fabs(Ppm - Pmm)) / 4.0;
        a = (fabs(Ppp) + fabs(Ppm) + fabs(Pmp) + fabs(Pmm)) / 4.0;
      }
      num += d2 * d2;
      double e = g + eps * a;
      den += e * e;
    }
  chi[c] = den > 0.0 ? sqrt(num / den) : 0.0;
}

// flags from the indicator: +1 refine (active, below lmax, chi^ > chi_ref), -1 recoarsen (virtual
// mother, chi^ < chi_rec); chi^ = the largest indicator over the cell and its same-level Voronoi
// neighbours of status <= 0 (the second difference vanishes in the middle of a smeared jump and
// peaks on both sides of it, so the criterion is applied to neighbourhoods)
__global__ void k_flags_from_chi(LevelView L, Bc6 bc6, int D, const double* chi, int is_below_lmax, double chi_ref,
                                 double chi_rec, int8_t* flag) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int8_t f = 0;
  const int8_t s = L.st[c];
  if (is_below_lmax && (s == 0 || s == -1)) {
    int ijk[3];
    cell_coords(L, c, ijk);
    double m = chi[c];
    const int kz0 = D == 3 ? -1 : 0, kz1 = D == 3 ? 1 : 0;
    for (int oz = kz0; oz <= kz1; oz++)
      for (int oy = -1; oy <= 1; oy++)
        for (int ox = -1; ox <= 1; ox++) {
          if (!ox && !oy && !oz) continue;
          int nb[3] = {ijk[0] + ox, ijk[1] + oy, ijk[2] + oz};
          bool in = true;
          for (int a = 0; a < D; a++) in &= bcmap(L.L, bc6.v, a, nb[a], &nb[a]);
          if (!in) continue;
          long long nd = didx(L, nb[0], nb[1], nb[2]);
          const int8_t sn = L.st[nd];
          if ((sn == 0 || sn == -1) && chi[nd] > m) m = chi[nd];
        }
    if (s == 0 && m > chi_ref) f = 1;
    if (s == -1 && m < chi_rec) f = -1;
  }
  flag[c] = f;
}

// R (cells with children of status <= 0) after the flags: refine active cells flagged +1
// below lmax; drop virtual mothers flagged -1 whose children are all active, none flagged +1,
// with no grandchildren of any status (rule 7).
__global__ void k_rinit(LevelView L, LevelView Lc, LevelView Lg, const int8_t* flag, const int8_t* cflag,
                        int below_lmax, int has_grand, int D, int r, int8_t* R) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int8_t s = L.st[c];
  int8_t v = (s == -1);
  if (below_lmax) {
    if (flag[c] == 1 && s == 0) v = 1;
    if (flag[c] == -1 && s == -1) {
      int ijk[3];
      cell_coords(L, c, ijk);
      bool ok = true;
      int rz = D == 3 ? r : 1;
      for (int kk = 0; kk < rz && ok; kk++)
        for (int jj = 0; jj < r && ok; jj++)
          for (int ii = 0; ii < r && ok; ii++) {
            int cc[3] = {r * ijk[0] + ii, r * ijk[1] + jj, D == 3 ? r * ijk[2] + kk : 0};
            long long cd = didx(Lc, cc[0], cc[1], cc[2]);
            if (Lc.st[cd] != 0 || cflag[cd] == 1) ok = false;
            else if (has_grand &&
                     Lg.st[didx(Lg, r * cc[0], r * cc[1], D == 3 ? r * cc[2] : 0)] != ST_NONE)
              ok = false;
          }
      if (ok) v = 0;
    }
  } else {
    v = 0;
  }
  R[c] = v;
}

// closure under rules 4-5: every Voronoi neighbour of a cell in R (level l >= 1) gets its mother
// into R (level l-1)
__global__ void k_closure(LevelView L, LevelView Lm, Bc6 bc6, const int8_t* R, int8_t* Rm, int D, int r) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n || !R[c]) return;
  int ijk[3];
  cell_coords(L, c, ijk);
  int kz0 = D == 3 ? -1 : 0, kz1 = D == 3 ? 1 : 0;
  for (int oz = kz0; oz <= kz1; oz++)
    for (int oy = -1; oy <= 1; oy++)
      for (int ox = -1; ox <= 1; ox++) {
        if (!ox && !oy && !oz) continue;
        int nb[3] = {ijk[0] + ox, ijk[1] + oy, ijk[2] + oz};
        bool in = true;
        for (int a = 0; a < D; a++) in &= bcmap(L.L, bc6.v, a, nb[a], &nb[a]);
        if (!in) continue;
        Rm[didx(Lm, nb[0] / r, nb[1] / r, D == 3 ? nb[2] / r : 0)] = 1;
      }
}

// new statuses: -1 in R; 0 if the mother is in R (or level 0); 1 if the mother is active and
// has a Voronoi neighbour in R; otherwise no cell
__global__ void k_newstatus(LevelView L, LevelView Lm, Bc6 bc6, const int8_t* R, const int8_t* Rm,
                            const int8_t* nstm, int level, int D, int r, int8_t* nst) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  if (level == 0) { nst[c] = R[c] ? -1 : 0; return; }
  int ijk[3];
  cell_coords(L, c, ijk);
  int mi[3] = {ijk[0] / r, ijk[1] / r, D == 3 ? ijk[2] / r : 0};
  long long m = didx(Lm, mi[0], mi[1], mi[2]);
  int8_t s = ST_NONE;
  if (Rm[m]) s = R[c] ? -1 : 0;
  else if (nstm[m] == 0) {
    bool has = false;
    int kz0 = D == 3 ? -1 : 0, kz1 = D == 3 ? 1 : 0;
    for (int oz = kz0; oz <= kz1 && !has; oz++)
      for (int oy = -1; oy <= 1 && !has; oy++)
        for (int ox = -1; ox <= 1 && !has; ox++) {
          if (!ox && !oy && !oz) continue;
          int nb[3] = {mi[0] + ox, mi[1] + oy, mi[2] + oz};
          bool in = true;
          for (int a = 0; a < D; a++) in &= bcmap(Lm.L, bc6.v, a, nb[a], &nb[a]);
          if (in && Rm[didx(Lm, nb[0], nb[1], nb[2])]) has = true;
        }
    if (has) s = 1;
  }
  nst[c] = s;
}

// newly active cells (new, or virtual before the edit) take the child-box average of the
// mother's WENO polynomial (mother active before the edit; its pre-edit active id is used)
__global__ void k_newvalues(LevelView L, LevelView Lm, const int8_t* nst, const double* whm, Tables T, int D, int V,
                            int* err) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  int8_t o = L.st[c], n = nst[c];
  if (!(n == 0 || n == -1) || !(o == ST_NONE || o == 1)) return;
  int r = T.r, N = T.N;
  int ijk[3];
  cell_coords(L, c, ijk);
  int mi[3] = {ijk[0] / r, ijk[1] / r, D == 3 ? ijk[2] / r : 0};
  int ch[3] = {ijk[0] - r * mi[0], ijk[1] - r * mi[1], D == 3 ? ijk[2] - r * mi[2] : 0};
  int ma = Lm.aid[didx(Lm, mi[0], mi[1], mi[2])];
  if (ma < 0) { atomicOr(err, 8); return; }
  int nsp = 1;
  for (int a = 0; a < D; a++) nsp *= N;
  for (int v = 0; v < V; v++) {
    const double* q = whm + ((long long)ma * V + v) * nsp;
    double acc = 0.0;
    for (int nn = 0; nn < nsp; nn++) {
      int t = nn;
      double th = 1.0;
      for (int b = 0; b < D; b++) { th *= T.Wc[ch[b]][t % N]; t /= N; }
      acc = fma(th, q[nn], acc);
    }
    L.u[v * L.n + c] = acc;
  }
}

__global__ void k_commit(LevelView L, const int8_t* nst, int8_t* st, int V) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n) return;
  st[c] = nst[c];
  if (nst[c] == ST_NONE)
    for (int v = 0; v < V; v++) L.u[v * L.n + c] = 0.0;
}

// virtual children hold their mother's average until the next projection
__global__ void k_virtual_from_mother(LevelView L, LevelView Lm, int D, int V, int r) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L.n || L.st[c] != 1) return;
  int ijk[3];
  cell_coords(L, c, ijk);
  long long m = didx(Lm, ijk[0] / r, ijk[1] / r, D == 3 ? ijk[2] / r : 0);
  for (int v = 0; v < V; v++) L.u[v * L.n + c] = Lm.u[v * Lm.n + m];
}

// ---- order-preserving stream compaction of a dense int8 array ----
// mode 0: a == val; mode 1: a != ST_NONE; mode 2: a != 0
__device__ __forceinline__ bool cpred(int8_t x, int mode, int val) {
  return mode == 0 ? x == val : (mode == 1 ? x != ST_NONE : x != 0);
}

__global__ void k_ccount(const int8_t* a, long long n, int mode, int val, int* bcnt) {
  long long base = (long long)blockIdx.x * CHUNK;
  int c = 0;
  for (int i = threadIdx.x; i < CHUNK; i += blockDim.x) {
    long long k = base + i;
    if (k < n && cpred(a[k], mode, val)) c++;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += ws[w];
    bcnt[blockIdx.x] = s;
  }
}

__global__ void k_cscan(int* b, int nb, int* total) {
  __shared__ int s[1024];
  int carry = 0;
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < nb ? b[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int t = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) b[i] = carry + s[threadIdx.x] - v;
    int tot = s[1023];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_cscatter(const int8_t* a, long long n, int mode, int val, const int* boff, int32_t* list,
                           int32_t* idmap) {
  __shared__ int ws[32];
  __shared__ int wo[32];
  long long base = (long long)blockIdx.x * CHUNK;
  int off = boff[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < CHUNK; i0 += blockDim.x) {
    long long k = base + i0 + threadIdx.x;
    bool f = k < n && cpred(a[k], mode, val);
    unsigned b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) ws[wid] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int w = 0; w < nw; w++) { wo[w] = s; s += ws[w]; }
      ws[31] = s;
    }
    __syncthreads();
    int pos = off + wo[wid] + __popc(b & ((1u << lane) - 1u));
    if (f) {
      list[pos] = (int32_t)k;
      if (idmap) idmap[k] = pos;
    } else if (idmap && k < n) {
      idmap[k] = -1;
    }
    off += ws[31];
    __syncthreads();
  }
}

// 2D WENO in two passes: the rows (i, j + dj), |dj| <= M, of every active cell (i, j), mapped
// through the y boundary (wrapped, clamped or mirrored into the level; none beyond an inflow face)
__global__ void k_xmark(LevelView L, Bc6 bc6, const int32_t* alist, int na, int M, int8_t* xmark) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= na) return;
  int ijk[3];
  cell_coords(L, alist[k], ijk);
  for (int dj = -M; dj <= M; dj++) {
    const int j = ijk[1] + dj;
    if (beyond_inflow(L.L, bc6.v, 1, j)) continue;
    int jm = j;
    bcmap(L.L, bc6.v, 1, j, &jm);
    xmark[didx(L, ijk[0], jm, 0)] = 1;
  }
}

// 3D WENO in three passes: the cells (i, j, k + dk) whose y sweeps, and the rows (i, j + dj, k + dk)
// whose x sweeps feed the active cell (i, j, k), |dj|, |dk| <= M, mapped through the boundaries
__global__ void k_mark3(LevelView L, Bc6 bc6, const int32_t* alist, int na, int M, int8_t* xmark, int8_t* ymark) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= na) return;
  int ijk[3];
  cell_coords(L, alist[k], ijk);
  for (int dk = -M; dk <= M; dk++) {
    const int kk = ijk[2] + dk;
    if (beyond_inflow(L.L, bc6.v, 2, kk)) continue;
    int km = kk;
    bcmap(L.L, bc6.v, 2, kk, &km);
    ymark[didx(L, ijk[0], ijk[1], km)] = 1;
    for (int dj = -M; dj <= M; dj++) {
      const int jj = ijk[1] + dj;
      if (beyond_inflow(L.L, bc6.v, 1, jj)) continue;
      int jm = jj;
      bcmap(L.L, bc6.v, 1, jj, &jm);
      xmark[didx(L, ijk[0], jm, km)] = 1;
    }
  }
}

__global__ void k_tmark(LevelView L, const int32_t* alist, int na, int TS, int t0, int t1, int8_t* tflag) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= na) return;
  int ijk[3];
  cell_coords(L, alist[k], ijk);
  long long t = ((long long)(ijk[2] / TS) * t1 + ijk[1] / TS) * t0 + ijk[0] / TS;
  tflag[t] = 1;
}

// high faces that need their own flux: the +axis neighbour is outside a transmissive boundary, a
// virtual child or a virtual mother (an active neighbour computes the face as its low face)
__global__ void k_hmark(LevelView L, Bc6 bc6, const int32_t* alist, int na, int D, int8_t* hflag) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= na) return;
  int ijk[3];
  cell_coords(L, alist[k], ijk);
  for (int d = 0; d < D; d++) {
    int nb[3] = {ijk[0], ijk[1], ijk[2]};
    bool in = bcmap(L.L, bc6.v, d, ijk[d] + 1, &nb[d]);
    bool need = !in || L.st[didx(L, nb[0], nb[1], nb[2])] != 0;
    hflag[(long long)d * na + k] = need ? 1 : 0;
  }
}

// canonical gather / scatter of cell averages and metadata
__global__ void k_gather(LevelView L, const int32_t* clist, int nc, int V, double* out, aw_cell* meta, int level) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  long long di = clist[k];
  for (int v = 0; v < V; v++) out[(long long)k * V + v] = L.u[v * L.n + di];
  if (meta) {
    int ijk[3];
    cell_coords(L, di, ijk);
    meta[k].level = level;
    meta[k].status = L.st[di];
    meta[k].i = ijk[0];
    meta[k].j = ijk[1];
    meta[k].k = ijk[2];
  }
}
__global__ void k_scatter(LevelView L, const int32_t* clist, int nc, int V, const double* in) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc) return;
  long long di = clist[k];
  for (int v = 0; v < V; v++) L.u[v * L.n + di] = in[(long long)k * V + v];
}
__global__ void k_gather_d(const double* src, const int32_t* clist, int nc, double* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nc) out[k] = src[clist[k]];
}
__global__ void k_gather_i8(const int8_t* src, const int32_t* clist, int nc, int8_t* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nc) out[k] = src[clist[k]];
}
__global__ void k_scatter_i8(int8_t* dst, const int32_t* clist, int nc, const int8_t* in) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nc) dst[clist[k]] = in[k];
}
// per-block partial sums of the active cells' averages (fixed reduction order)
__global__ void k_partial(LevelView L, const int32_t* alist, int na, int V, double* part) {
  __shared__ double sh[256];
  for (int v = 0; v < V; v++) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    sh[threadIdx.x] = k < na ? L.u[v * L.n + alist[k]] : 0.0;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)blockIdx.x * V + v] = sh[0];
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------------
static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

static LevelView view(const aw_solver* s, int l) {
  LevelView v;
  const Level& L = s->lev[l];
  for (int a = 0; a < 3; a++) { v.L[a] = L.L[a]; v.dx[a] = L.dx[a]; }
  v.n = L.n;
  v.st = L.st;
  v.u = L.u;
  v.aid = L.aid;
  return v;
}

static Bc6 bc6_of(const aw_solver* s) {
  Bc6 b;
  for (int i = 0; i < 6; i++) b.v[i] = s->cfg.bc[i];
  b.inflow_rho = s->cfg.inflow[0];
  return b;
}

static RtPhys rtphys(const aw_solver* s) {
  RtPhys R;
  R.pde = s->cfg.pde;
  R.D = s->D;
  R.V = s->V;
  R.P = s->phys;
  return R;
}

static int ensure_buf(aw_solver* s, long long ndouble) {
  if (ndouble <= s->buf_cap) return AW_OK;
  dfree(s, s->d_buf);
  s->d_buf = nullptr;
  long long cap = std::max(ndouble, (long long)1024);
  if (dalloc(s, (void**)&s->d_buf, cap * sizeof(double)) != cudaSuccess)
    AW_FAIL(oom_code(s), "staging buffer of %lld doubles", cap);
  s->buf_cap = cap;
  return AW_OK;
}

// compact a dense int8 array into list (+ idmap); the count lands in d_cnt[slot]
static int compact(aw_solver* s, const int8_t* a, long long n, int mode, int val, int32_t* list, int32_t* idmap,
                   int slot) {
  long long nb = (n + CHUNK - 1) / CHUNK;
  if (nb > s->bcnt_cap) {
    dfree(s, s->d_bcnt);
    s->d_bcnt = nullptr;
    if (dalloc(s, (void**)&s->d_bcnt, nb * sizeof(int)) != cudaSuccess) AW_FAIL(oom_code(s), "scan scratch");
    s->bcnt_cap = nb;
  }
  k_ccount<<<(unsigned)nb, 256, 0, s->stream>>>(a, n, mode, val, s->d_bcnt);
  k_cscan<<<1, 1024, 0, s->stream>>>(s->d_bcnt, (int)nb, s->d_cnt + slot);
  k_cscatter<<<(unsigned)nb, 256, 0, s->stream>>>(a, n, mode, val, s->d_bcnt, list, idmap);
  s->launches += 3;
  CK(cudaGetLastError());
  return AW_OK;
}

// WENO by passes: a row (cell) list of at least `need` entries, allocated before the compaction
// that fills it (need: a bound from the active count), and a sweep buffer of `count` rows times
// `per` doubles, allocated once the count is known
static int ensure_list(aw_solver* s, int32_t** list, long long* cap, long long need, int l) {
  if (need <= *cap) return AW_OK;
  long long c = std::max(need + need / 2, (long long)64);
  c = std::min(c, s->lev[l].n);
  dfree(s, *list);
  *list = nullptr;
  *cap = 0;
  if (dalloc(s, (void**)list, c * sizeof(int32_t)) != cudaSuccess)
    AW_FAIL(oom_code(s), "sweep list of level %d (%lld entries)", l, c);
  *cap = c;
  return AW_OK;
}

static int ensure_sweeps(aw_solver* s, double** buf, long long* cap, long long count, long long per, int l) {
  if (count <= *cap) return AW_OK;
  long long c = std::max(count + count / 4, (long long)64);
  dfree(s, *buf);
  *buf = nullptr;
  *cap = 0;
  if (dalloc(s, (void**)buf, c * per * sizeof(double)) != cudaSuccess)
    AW_FAIL(oom_code(s), "sweep buffer of level %d (%lld entries)", l, c);
  *cap = c;
  return AW_OK;
}

// WENO by passes (one sweep direction after the other over compact lists) applies unless an
// inflow face on one axis meets a reflective face on a later axis: the mirrored ghost lines of
// the later axis would need the inflow values of the earlier sweep unmirrored
static bool weno_by_passes(const aw_solver* s) {
  const int* b = s->cfg.bc;
  for (int a = 0; a < s->D; a++)
    for (int c = a + 1; c < s->D; c++) {
      bool inflow_a = b[2 * a] == AW_BC_INFLOW || b[2 * a + 1] == AW_BC_INFLOW;
      bool reflective_c = b[2 * c] == AW_BC_REFLECTIVE || b[2 * c + 1] == AW_BC_REFLECTIVE;
      if (inflow_a && reflective_c) return false;
    }
  return true;
}

static int ensure_active_cap(aw_solver* s, int l, long long need) {
  Level& L = s->lev[l];
  if (need <= L.cap) return AW_OK;
  long long cap = std::max(need + need / 2, (long long)64);
  for (void* p : {(void*)L.wh, (void*)L.qh, (void*)L.fl, (void*)L.mem, (void*)L.hflag, (void*)L.hflist,
                  (void*)L.fsync})
    dfree(s, p);
  L.wh = L.qh = L.fl = L.mem = nullptr;
  L.hflag = nullptr;
  L.hflist = nullptr;
  L.fsync = nullptr;
  L.cap = 0;
  size_t V = s->V;
  if (dalloc(s, (void**)&L.hflag, cap * s->D) != cudaSuccess ||
      dalloc(s, (void**)&L.hflist, cap * s->D * sizeof(int32_t)) != cudaSuccess ||
      dalloc(s, (void**)&L.wh, cap * V * s->NSP * sizeof(double)) != cudaSuccess ||
      dalloc(s, (void**)&L.qh, cap * V * s->NST * sizeof(double)) != cudaSuccess ||
      dalloc(s, (void**)&L.fl, cap * 2 * s->D * V * sizeof(double)) != cudaSuccess ||
      dalloc(s, (void**)&L.mem, cap * 2 * s->D * V * sizeof(double)) != cudaSuccess ||
      dalloc(s, (void**)&L.fsync, cap * sizeof(int32_t)) != cudaSuccess)
    AW_FAIL(oom_code(s), "per-active arrays of level %d (%lld cells)", l, cap);
  L.cap = cap;
  CK(cudaMemsetAsync(L.fsync, 0, cap * sizeof(int32_t), s->stream));
  return AW_OK;
}

// Rebuild every per-level list and read the counts back, in three phases around two host
// synchronisations (lists_issue; sync; lists_mid; sync; lists_finish), so that a batch of solvers
// can share the synchronisations.
static int lists_issue(aw_solver* s) {
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    TRY(compact(s, L.st, L.n, 0, 0, L.alist, L.aid, NSLOT * l + 0));
    TRY(compact(s, L.st, L.n, 0, 1, L.vlist, nullptr, NSLOT * l + 1));
    TRY(compact(s, L.st, L.n, 0, -1, L.mlist, nullptr, NSLOT * l + 2));
    TRY(compact(s, L.st, L.n, 1, 0, L.clist, nullptr, NSLOT * l + 3));
  }
  CK(cudaMemcpyAsync(s->h_cnt, s->d_cnt, sizeof(int) * NSLOT * MAXL, cudaMemcpyDeviceToHost, s->stream));
  return AW_OK;
}

static int lists_mid(aw_solver* s) {
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    L.na = s->h_cnt[NSLOT * l + 0];
    L.nv = s->h_cnt[NSLOT * l + 1];
    L.nm = s->h_cnt[NSLOT * l + 2];
    L.nc = s->h_cnt[NSLOT * l + 3];
    CK(cudaMemsetAsync(L.tflag, 0, L.ntd, s->stream));
    if (L.na > 0) {
      k_tmark<<<nblk(L.na, 256), 256, 0, s->stream>>>(view(s, l), L.alist, L.na, L.ts, L.tdim[0], L.tdim[1],
                                                      L.tflag);
      s->launches++;
    }
    TRY(compact(s, L.tflag, L.ntd, 2, 0, L.tiles, nullptr, NSLOT * l + 4));
    TRY(ensure_active_cap(s, l, L.na));
    if (L.na > 0) {
      k_hmark<<<nblk(L.na, 256), 256, 0, s->stream>>>(view(s, l), bc6_of(s), L.alist, L.na, s->D, L.hflag);
      s->launches++;
      TRY(compact(s, L.hflag, (long long)s->D * L.na, 2, 0, L.hflist, nullptr, NSLOT * l + 5));
    } else {
      CK(cudaMemsetAsync(s->d_cnt + NSLOT * l + 5, 0, sizeof(int), s->stream));
    }
    CK(cudaMemsetAsync(L.mem, 0, (size_t)L.cap * 2 * s->D * s->V * sizeof(double), s->stream));
    const long long w = 2 * s->M + 1;
    if (L.xmark && L.na > 0 && s->D == 2) {
      // rows whose x sweep feeds an active cell (through the y boundary map)
      TRY(ensure_list(s, &L.xlist, &L.xlcap, std::min(L.n, w * L.na), l));
      CK(cudaMemsetAsync(L.xmark, 0, L.n, s->stream));
      k_xmark<<<nblk(L.na, 256), 256, 0, s->stream>>>(view(s, l), bc6_of(s), L.alist, L.na, s->M, L.xmark);
      s->launches++;
      TRY(compact(s, L.xmark, L.n, 2, 0, L.xlist, L.xslot, NSLOT * l + 6));
      CK(cudaMemsetAsync(s->d_cnt + NSLOT * l + 7, 0, sizeof(int), s->stream));
    } else if (L.xmark && L.na > 0) {
      // 3D: rows of the x sweeps and cells of the y sweeps that feed the active cells
      TRY(ensure_list(s, &L.xlist, &L.xlcap, std::min(L.n, w * w * L.na), l));
      TRY(ensure_list(s, &L.ylist, &L.ylcap, std::min(L.n, w * L.na), l));
      CK(cudaMemsetAsync(L.xmark, 0, L.n, s->stream));
      CK(cudaMemsetAsync(L.ymark, 0, L.n, s->stream));
      k_mark3<<<nblk(L.na, 256), 256, 0, s->stream>>>(view(s, l), bc6_of(s), L.alist, L.na, s->M, L.xmark, L.ymark);
      s->launches++;
      TRY(compact(s, L.xmark, L.n, 2, 0, L.xlist, L.xslot, NSLOT * l + 6));
      TRY(compact(s, L.ymark, L.n, 2, 0, L.ylist, L.yslot, NSLOT * l + 7));
    } else {
      CK(cudaMemsetAsync(s->d_cnt + NSLOT * l + 6, 0, 2 * sizeof(int), s->stream));
    }
  }
  CK(cudaMemcpyAsync(s->h_cnt, s->d_cnt, sizeof(int) * NSLOT * MAXL, cudaMemcpyDeviceToHost, s->stream));
  return AW_OK;
}

static int lists_finish(aw_solver* s) {
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    // the fused flux-and-update kernel leaves its arrival counters at zero; zeroed here too, so
    // that a step that found an inconsistent mesh cannot leave counts behind for the next one
    if (L.fsync && L.cap > 0) CK(cudaMemsetAsync(L.fsync, 0, L.cap * sizeof(int32_t), s->stream));
    L.ntiles = s->h_cnt[NSLOT * l + 4];
    L.nh = s->h_cnt[NSLOT * l + 5];
    L.nx = s->h_cnt[NSLOT * l + 6];
    L.ny = s->h_cnt[NSLOT * l + 7];
    if (L.xmark) TRY(ensure_sweeps(s, &L.xs, &L.xcap, L.nx, (long long)s->V * s->N, l));
    if (L.ymark) TRY(ensure_sweeps(s, &L.ys, &L.ycap, L.ny, (long long)s->V * s->N * s->N, l));
  }
  return AW_OK;
}

static int rebuild_lists(aw_solver* s) {
  TRY(lists_issue(s));
  CK(cudaStreamSynchronize(s->stream));
  TRY(lists_mid(s));
  CK(cudaStreamSynchronize(s->stream));
  return lists_finish(s);
}

static HotArgs make_args(const aw_solver* s, int l, int sub) {
  HotArgs a;
  memset(&a, 0, sizeof a);
  a.T = s->T;
  a.P = s->phys;
  for (int i = 0; i < 6; i++) a.bc[i] = s->cfg.bc[i];
  a.level = l;
  a.sub = sub;
  a.picard = s->P;
  a.flux = s->cfg.flux;
  a.lv = view(s, l);
  if (l >= 1) a.lvm = view(s, l - 1);
  if (l < s->lmax) a.lvc = view(s, l + 1);
  const Level& L = s->lev[l];
  a.alist = L.alist;
  a.na = L.na;
  a.hflist = L.hflist;
  a.nh = L.nh;
  a.tiles = L.tiles;
  a.ntiles = L.ntiles;
  for (int i = 0; i < 3; i++) a.tdim[i] = L.tdim[i];
  a.wh = L.wh;
  a.qh = L.qh;
  a.fl = L.fl;
  a.mem = L.mem;
  if (l >= 1) a.qhm = s->lev[l - 1].qh;
  if (l < s->lmax) a.memc = s->lev[l + 1].mem;
  a.dtl = s->d_dtl;
  a.err = s->d_err;
  a.vlist = L.vlist;
  a.nv = L.nv;
  a.ts = L.ts;
  if (L.xmark) {
    a.xlist = L.xlist;
    a.xslot = L.xslot;
    a.xs = L.xs;
    a.nxs = L.nx;
  }
  if (L.ymark) {
    a.ylist = L.ylist;
    a.yslot = L.yslot;
    a.ys = L.ys;
    a.nys = L.ny;
  }
  a.fsync = L.fsync;
  return a;
}

static int average_into(aw_solver* s, int l) {
  Level& L = s->lev[l];
  if (L.nm == 0) return AW_OK;
  k_average<<<nblk((long long)L.nm * s->V, 128), 128, 0, s->stream>>>(view(s, l), view(s, l + 1), L.mlist, L.nm, s->V,
                                                                   s->D, s->r);
  s->launches++;
  CK(cudaGetLastError());
  return AW_OK;
}

static int average_all(aw_solver* s) {
  for (int l = s->lmax - 1; l >= 0; l--) TRY(average_into(s, l));
  return AW_OK;
}

// one step of level l (Eq. eqn.update.criterion by recursion): reconstruction and prediction of
// level l, then r sub-steps of level l+1, then the fluxes and update of level l
static int advance(aw_solver* s, int l, int sub) {
  HotArgs a = make_args(s, l, sub);
  const Level& L = s->lev[l];
  cudaStream_t st = s->stream;
  if (l >= 1)
    s->launches += timed(s, KIND_PROJECT, [&] { return s->ops.project(a, L.vlist, L.nv, s->lev[l - 1].qh, 1, nullptr, 1, st); });
  s->launches += timed(s, KIND_WENO, [&] { return s->ops.weno(a, st); });
  int key[6];
  const int vp = tune_pick(s, AW_TUNE_PREDICTOR, a.na, key);
  a.cta_div = tune_div(vp);
  s->launches += tuned(s, vp, key, a.na, [&] { return timed(s, KIND_PREDICT, [&] { return s->ops.predict(a, st); }); });
  CK(cudaGetLastError());
  if (l < s->lmax)
    for (int k = 0; k < s->r; k++) TRY(advance(s, l + 1, k));
  const int vf = tune_pick(s, AW_TUNE_FLUX, a.na, key);
  a.cta_div = tune_div(vf);
  if (launch_params().fuse_flux_update) {
    s->launches += tuned(s, vf, key, a.na, [&] { return timed(s, KIND_FLUX, [&] { return s->ops.flux_update(a, st); }); });
  } else {
    s->launches += tuned(s, vf, key, a.na, [&] { return timed(s, KIND_FLUX, [&] { return s->ops.flux(a, st); }); });
    s->launches += timed(s, KIND_UPDATE, [&] { return s->ops.update(a, st); });
  }
  CK(cudaGetLastError());
  if (l >= 1 && sub == s->r - 1) TRY(average_into(s, l - 1));
  return AW_OK;
}

// dt0 (reading R11): issue the reduction and the copy of its result to host slot h_dtl[MAXL]
static int dt_issue(aw_solver* s) {
  double big = 1e300;
  CK(cudaMemcpyAsync(s->d_dtmin, &big, sizeof(double), cudaMemcpyHostToDevice, s->stream));
  double rl = 1.0;
  for (int l = 0; l <= s->lmax; l++) {
    const Level& L = s->lev[l];
    if (L.na > 0) {
      k_dt<<<nblk(L.na, 256), 256, 0, s->stream>>>(view(s, l), L.alist, L.na, rtphys(s), s->cfg.cfl, rl, s->d_dtmin);
      s->launches++;
    }
    rl *= s->r;
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(s->h_dtl + MAXL, s->d_dtmin, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  return AW_OK;
}

// after the stream has reached the copy of dt_issue
static int dt_finish(aw_solver* s, double* dt) {
  double h = s->h_dtl[MAXL];
  if (!(h > 0.0) || h >= 1e300) AW_FAIL(AW_ENONPHYSICAL, "no positive stable time step (dt = %g)", h);
  *dt = h;
  return AW_OK;
}

static int compute_dt(aw_solver* s, double* dt) {
  TRY(dt_issue(s));
  CK(cudaStreamSynchronize(s->stream));
  return dt_finish(s, dt);
}

// level time steps dt0 / r^l to the device and a cleared error word
static int step_begin(aw_solver* s, double dt0) {
  double dt = dt0;
  for (int l = 0; l < MAXL; l++) {
    s->h_dtl[l] = dt;
    dt /= s->r;
  }
  CK(cudaMemcpyAsync(s->d_dtl, s->h_dtl, sizeof(double) * MAXL, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
  return AW_OK;
}

// after the stream has reached the copy of the error word to h_cnt[NSLOT * MAXL]: statistics, errors
static int step_finish(aw_solver* s, double dt0, aw_stats* st) {
  tune_harvest(s);
  const int err = s->h_cnt[NSLOT * MAXL];
  int64_t rl = 1;
  for (int l = 0; l <= s->lmax; l++) {
    int64_t u = (int64_t)s->lev[l].na * rl;
    if (st) { st->cell_updates += u; st->updates_per_level[l] += u; }
    rl *= s->r;
  }
  if (st) { st->level0_steps++; st->last_dt0 = dt0; }
  if (err & 1) AW_FAIL(AW_ENONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN) after the update");
  if (err) AW_FAIL(AW_ESTATE, "inconsistent mesh detected on the device (error word %d)", err);
  return AW_OK;
}

// The launch arguments of a level-0 step of solver s: per level, the hot kernels' arguments and
// the averaging list (every pointer and size of the mesh; the time steps are read from device
// memory).  The autotuner's decisions and the launch-shape rules are added by step_signature.
static void put_solver_signature(const aw_solver* s, std::vector<char>* sig) {
  auto put = [&](const void* p, size_t n) { sig->insert(sig->end(), (const char*)p, (const char*)p + n); };
  put(&s, sizeof s);
  for (int l = 0; l <= s->lmax; l++) {
    const HotArgs a = make_args(s, l, 0);   // zero-filled, padding included
    put(&a, sizeof a);
    put(&s->lev[l].mlist, sizeof s->lev[l].mlist);
    put(&s->lev[l].nm, sizeof s->lev[l].nm);
  }
}

static std::atomic<int64_t> g_tune_epoch{0};   // advanced by aw_reset_tuning

static void step_signature(aw_solver* const* S, int n, const bool* live, std::vector<char>* sig) {
  sig->clear();
  const LaunchParams lp = launch_params();
  const int64_t v[] = {lp.pass_min_cells, lp.tile8_min_cells, lp.small_ctas_per_sm, lp.fuse_flux_update,
                       lp.autotune, lp.persistent, g_tune_epoch.load()};
  sig->insert(sig->end(), (const char*)v, (const char*)v + sizeof v);
  for (int m = 0; m < n; m++) {
    const char on = live ? (char)live[m] : 1;
    sig->push_back(on);
    if (on) put_solver_signature(S[m], sig);
  }
}

// Run a level-0 step from a CUDA graph.  issue(stream) issues the step's launches on the given
// stream, through solvers S[0..n-1], and adds their number to *launches.  The graph runs on S[0]'s
// own stream gstream (the caller's stream may be one that cannot be captured, the legacy default
// stream), ordered after the caller's stream `st` and joined back to it.  When the last graph of
// this slot was captured from the same launch arguments (signature `sig`) and holds no timing
// events, it is launched again as it is; otherwise the step is captured, with the members'
// streams pointed at gstream meanwhile, and the executable graph is updated in place when the new
// capture has its shape (the same kinds of nodes in the same order) or built anew.  Every launch,
// memset and timing event is captured as it is issued, so the device does exactly what the
// direct launches do.
template <class F>
static int graph_replay(aw_solver* const* S, int n, cudaStream_t st, StepGraph* g, const std::vector<char>& sig,
                        int64_t* launches, F&& issue) {
  aw_solver* s = S[0];
  if (!s->gstream) CK(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
  if (!s->gev) CK(cudaEventCreateWithFlags(&s->gev, cudaEventDisableTiming));
  cudaStream_t gs = s->gstream;
  CK(cudaEventRecord(s->gev, st));
  CK(cudaStreamWaitEvent(gs, s->gev, 0));
  if (g->exec && g->reusable && g->sig == sig) {
    CK(cudaGraphLaunch(g->exec, gs));
    *launches += g->launches;
    s->graph_reuses++;
  } else {
    for (int m = 0; m < n; m++) {
      S[m]->stream = gs;
      S[m]->capturing = true;
      S[m]->captured_events = false;
    }
    const int64_t before = *launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal);
    int rc = AW_OK;
    if (e == cudaSuccess) {
      rc = issue(gs);
      e = cudaStreamEndCapture(gs, &graph);
    }
    bool events = false;
    for (int m = 0; m < n; m++) {
      S[m]->stream = st;
      S[m]->capturing = false;
      events = events || S[m]->captured_events;
    }
    if (rc != AW_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      g->reusable = false;
      if (rc != AW_OK) return rc;
      AW_FAIL(AW_ECUDA, "step capture: %s", cudaGetErrorString(e));
    }
    if (g->exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(g->exec, graph, &info) == cudaSuccess) {
        s->graph_updates++;
      } else {
        cudaGetLastError();   // not a sticky error: the graph is built anew
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
      }
    }
    if (!g->exec) {
      e = cudaGraphInstantiate(&g->exec, graph, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        g->exec = nullptr;
        g->reusable = false;
        AW_FAIL(AW_ECUDA, "step graph instantiation: %s", cudaGetErrorString(e));
      }
      s->graph_instantiations++;
    }
    cudaGraphDestroy(graph);
    g->sig = sig;
    g->reusable = !events;
    g->launches = *launches - before;
    CK(cudaGraphLaunch(g->exec, gs));
  }
  CK(cudaEventRecord(s->gev, gs));
  CK(cudaStreamWaitEvent(st, s->gev, 0));
  return AW_OK;
}

static int step_dt(aw_solver* s, double dt0, aw_stats* st) {
  TRY(step_begin(s, dt0));
  if (launch_params().graph_steps) {
    std::vector<char> sig;
    step_signature(&s, 1, nullptr, &sig);
    TRY(graph_replay(&s, 1, s->stream, &s->sgraph, sig, &s->launches,
                     [&](cudaStream_t) { return advance(s, 0, 0); }));
  } else
    TRY(advance(s, 0, 0));
  CK(cudaMemcpyAsync(s->h_cnt + NSLOT * MAXL, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return step_finish(s, dt0, st);
}

// regrid pre-pass (at a synchronisation time): WENO polynomials of the active cells of levels
// 0..lmax-1 top-down, virtual children of levels 1..lmax-1 filled from their mothers' WENO
// polynomials; then the indicator on levels 0..lmax-1
static int regrid_prepass(aw_solver* s, int init_mode) {
  if (!init_mode) {
    for (int l = 0; l < s->lmax; l++) {
      HotArgs a = make_args(s, l, 0);
      s->launches += s->ops.weno(a, s->stream);
      if (l + 1 < s->lmax) {
        HotArgs b = make_args(s, l + 1, 0);
        s->launches += s->ops.project(b, s->lev[l + 1].vlist, s->lev[l + 1].nv, s->lev[l].wh, 0, nullptr, 1, s->stream);
      }
    }
  }
  for (int l = 0; l < s->lmax; l++) {
    Level& L = s->lev[l];
    k_indicator<<<nblk(L.n, 256), 256, 0, s->stream>>>(view(s, l), bc6_of(s), s->D, s->cfg.eps_ind, L.chi);
    s->launches++;
  }
  CK(cudaGetLastError());
  return AW_OK;
}

static IcArgs ic_args(const aw_solver* s) {
  IcArgs I;
  memset(&I, 0, sizeof I);
  I.kind = s->ic;
  I.np = (int)std::min<size_t>(s->icp.size(), 128);
  for (int i = 0; i < I.np; i++) I.p[i] = s->icp[i];
  I.R = rtphys(s);
  for (int a = 0; a < 3; a++) { I.lo[a] = s->cfg.lo[a]; I.hi[a] = s->cfg.hi[a]; }
  for (int i = 0; i < s->N; i++) { I.x[i] = s->T.x[i]; I.w[i] = s->T.w[i]; }
  I.N = s->N;
  return I;
}

// apply the dense flags of every level (L.flag) and rebuild the tree
// the tree edit of the flags on the device, up to (not including) the list rebuild
static int apply_flags_issue(aw_solver* s, int init_mode) {
  const int lmax = s->lmax;
  Bc6 bc = bc6_of(s);
  for (int l = 0; l <= lmax; l++) {
    Level& L = s->lev[l];
    LevelView Lc = l < lmax ? view(s, l + 1) : view(s, l);
    LevelView Lg = l + 2 <= lmax ? view(s, l + 2) : view(s, l);
    const int8_t* cflag = l < lmax ? s->lev[l + 1].flag : L.flag;
    k_rinit<<<nblk(L.n, 256), 256, 0, s->stream>>>(view(s, l), Lc, Lg, L.flag, cflag, l < lmax, l + 2 <= lmax, s->D,
                                                   s->r, L.R);
    s->launches++;
  }
  for (int l = lmax - 1; l >= 1; l--) {
    k_closure<<<nblk(s->lev[l].n, 256), 256, 0, s->stream>>>(view(s, l), view(s, l - 1), bc, s->lev[l].R,
                                                             s->lev[l - 1].R, s->D, s->r);
    s->launches++;
  }
  for (int l = 0; l <= lmax; l++) {
    Level& L = s->lev[l];
    const Level& Lm = s->lev[l > 0 ? l - 1 : 0];
    k_newstatus<<<nblk(L.n, 256), 256, 0, s->stream>>>(view(s, l), view(s, l > 0 ? l - 1 : 0), bc, L.R, Lm.R, Lm.nst,
                                                       l, s->D, s->r, L.nst);
    s->launches++;
  }
  CK(cudaGetLastError());
  // values of cells that change role (the pre-edit statuses and active ids are still in place)
  IcArgs I = ic_args(s);
  for (int l = 1; l <= lmax; l++) {
    Level& L = s->lev[l];
    if (init_mode) k_ic<<<nblk(L.n, 128), 128, 0, s->stream>>>(view(s, l), I, L.st, L.nst, 1);
    else
      k_newvalues<<<nblk(L.n, 128), 128, 0, s->stream>>>(view(s, l), view(s, l - 1), L.nst, s->lev[l - 1].wh, s->T,
                                                         s->D, s->V, s->d_err);
    s->launches++;
  }
  for (int l = 0; l <= lmax; l++) {
    Level& L = s->lev[l];
    k_commit<<<nblk(L.n, 256), 256, 0, s->stream>>>(view(s, l), L.nst, L.st, s->V);
    s->launches++;
  }
  if (!init_mode)
    for (int l = 1; l <= lmax; l++) {
      k_virtual_from_mother<<<nblk(s->lev[l].n, 256), 256, 0, s->stream>>>(view(s, l), view(s, l - 1), s->D, s->V,
                                                                           s->r);
      s->launches++;
    }
  CK(cudaGetLastError());
  return AW_OK;
}

static int apply_flags(aw_solver* s, int init_mode) {
  if (s->lmax == 0) return AW_OK;
  TRY(apply_flags_issue(s, init_mode));
  TRY(rebuild_lists(s));
  TRY(average_all(s));
  return AW_OK;
}

static int flags_from_chi(aw_solver* s) {
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    k_flags_from_chi<<<nblk(L.n, 256), 256, 0, s->stream>>>(view(s, l), bc6_of(s), s->D, L.chi, l < s->lmax,
                                                            s->cfg.chi_ref, s->cfg.chi_rec, L.flag);
    s->launches++;
  }
  CK(cudaGetLastError());
  return AW_OK;
}

static int regrid(aw_solver* s, int init_mode) {
  if (s->lmax == 0) return AW_OK;
  TRY(regrid_prepass(s, init_mode));
  TRY(flags_from_chi(s));
  return apply_flags(s, init_mode);
}

static int64_t total_cells(const aw_solver* s) {
  int64_t n = 0;
  for (int l = 0; l <= s->lmax; l++) n += s->lev[l].nc;
  return n;
}

static void free_solver(aw_solver* s) {
  harvest_events(s);
  tune_harvest(s);
  for (auto e : s->ev_free) cudaEventDestroy(e);
  s->ev_free.clear();
  // stream-ordered: after the solver's last work on its stream
  cudaStream_t st = s->stream;
  for (int l = 0; l < MAXL; l++) {
    Level& L = s->lev[l];
    for (void* p : {(void*)L.st, (void*)L.R, (void*)L.nst, (void*)L.flag, (void*)L.u, (void*)L.chi, (void*)L.aid,
                    (void*)L.alist, (void*)L.vlist, (void*)L.mlist, (void*)L.clist, (void*)L.tflag, (void*)L.tiles,
                    (void*)L.wh, (void*)L.qh, (void*)L.fl, (void*)L.mem, (void*)L.hflag, (void*)L.hflist,
                    (void*)L.xmark, (void*)L.xslot, (void*)L.xlist, (void*)L.xs, (void*)L.ymark, (void*)L.yslot,
                    (void*)L.ylist, (void*)L.ys, (void*)L.fsync})
      dfree(s, p);
  }
  for (void* p : {(void*)s->d_dtl, (void*)s->d_dtmin, (void*)s->d_err, (void*)s->d_cnt, (void*)s->d_bcnt,
                  (void*)s->d_buf, (void*)s->d_gs})
    dfree(s, p);
  // the host blocks may still be the target of copies in flight
  cudaStreamSynchronize(st);
  if (s->gstream) {
    cudaStreamSynchronize(s->gstream);
    cudaStreamDestroy(s->gstream);
  }
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->sgraph.exec) cudaGraphExecDestroy(s->sgraph.exec);
  if (s->bgraph.exec) cudaGraphExecDestroy(s->bgraph.exec);
  if (s->gev) cudaEventDestroy(s->gev);
  pinned_release(s->h_cnt);
  pinned_release(s->h_dtl);
  pinned_release(s->h_gs);
}

// ------------------------------------------------------------------------------------------
// Allocation-free CFL time step (aw_cfl_dt_noalloc).  Some callers cannot allocate device
// memory at the moment they need a stable time step: code running inside a host framework that
// owns every device allocation through its own pool, or a time loop that must not pay the
// implicit device synchronisation of cudaMalloc/cudaFree.  This variant of the CFL reduction
// keeps its per-block partial minima in a fixed file-scope device array instead of solver
// memory.  The array is shared by every call in the process and keeps the last call's contents;
// each call overwrites every slot it later reads, so nothing has to start at zero.
// ------------------------------------------------------------------------------------------
#define AW_NOALLOC_BLOCK 256
#define AW_NOALLOC_SLOTS 8192  // partial minima: up to 8192 * 256 cells (64 KiB of device memory)
static __device__ __align__(256) double g_noalloc_dt_scratch[AW_NOALLOC_SLOTS];
static double* g_noalloc_ptr[64];  // device address of the array, per device, from set-up
static bool g_noalloc_ready[64];
static std::mutex g_noalloc_mu;

__global__ void k_dt_blockmin(const double* u, long long n, RtPhys R, double dx0, double dx1, double dx2, double cfl,
                              double* partial) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double dt = 1e300;
  if (k < n) {
    double q[MAXV];
    for (int v = 0; v < R.V; v++) q[v] = u[v * n + k];
    double dx[3] = {dx0, dx1, dx2};
    double den = 0.0;
    for (int a = 0; a < R.D; a++) den += rt_speed(R, q, a) / dx[a];
    dt = cfl / den;
    if (!(dt > 0.0)) dt = 0.0;
  }
  for (int o = 16; o > 0; o >>= 1) dt = fmin(dt, __shfl_xor_sync(0xffffffffu, dt, o));
  __shared__ double wmin[AW_NOALLOC_BLOCK / 32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = dt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = wmin[0];
    for (int w = 1; w < AW_NOALLOC_BLOCK / 32; w++) m = fmin(m, wmin[w]);
    partial[blockIdx.x] = m;
  }
}

__global__ void k_dt_final(const double* partial, int nb, double* out) {
  double m = 1e300;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = fmin(m, partial[b]);
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wmin[32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = wmin[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) r = fmin(r, wmin[w]);
    *out = r;
  }
}

__global__ void k_selftest_rcp(const double* x, long long n, double* out) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = rcp_nr(x[k]);
  out[n + k] = 1.0 / x[k];
}

__global__ void k_selftest_flux_math(const double* x, long long n, double* out) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = rcp_nr1(x[k]);
  out[n + k] = 1.0 / x[k];
  out[2 * n + k] = sqrt_nr1(x[k]);
  out[3 * n + k] = sqrt(x[k]);
}

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

const char* aw_last_error(void) { return g_err.c_str(); }

int aw_num_vars(const aw_solver* s) { return s ? s->V : 0; }

int64_t aw_kernel_launches(const aw_solver* s) { return s ? s->launches : 0; }

int aw_create(const aw_config* cfg, uintptr_t stream, aw_solver** out) {
  if (!cfg || !out) AW_FAIL(AW_EINVAL, "null argument");
  *out = nullptr;
  const aw_config& c = *cfg;
  if (c.dim != 2 && c.dim != 3) AW_FAIL(AW_EINVAL, "dim must be 2 or 3");
  if (c.M < 1 || c.M > 3) AW_FAIL(AW_EINVAL, "M must be 1, 2 or 3");
  if (c.pde < 0 || c.pde > 2) AW_FAIL(AW_EINVAL, "unknown pde %d", c.pde);
  if (c.lmax < 0 || c.lmax >= MAXL) AW_FAIL(AW_EINVAL, "lmax must be in 0..%d", MAXL - 1);
  int r = c.lmax > 0 ? c.refine_factor : (c.refine_factor > 0 ? c.refine_factor : 2);
  if (c.lmax > 0 && (r < 2 || r < c.M || r > MAXR)) AW_FAIL(AW_EINVAL, "refine_factor must satisfy max(2, M) <= r <= %d", MAXR);
  if (r > MAXR) r = MAXR;
  if (c.nx < 1 || c.ny < 1 || (c.dim == 3 && c.nz < 1)) AW_FAIL(AW_EINVAL, "grid size must be positive");
  for (int a = 0; a < c.dim; a++) {
    if (!(c.hi[a] > c.lo[a])) AW_FAIL(AW_EINVAL, "empty domain on axis %d", a);
    if ((c.bc[2 * a] == AW_BC_PERIODIC) != (c.bc[2 * a + 1] == AW_BC_PERIODIC))
      AW_FAIL(AW_EINVAL, "periodic boundaries must pair up on axis %d", a);
    for (int sd = 0; sd < 2; sd++) {
      int b = c.bc[2 * a + sd];
      if (b != AW_BC_PERIODIC && b != AW_BC_TRANSMISSIVE && b != AW_BC_REFLECTIVE && b != AW_BC_INFLOW)
        AW_FAIL(AW_EINVAL, "unknown boundary condition %d", b);
      if (b == AW_BC_REFLECTIVE && c.pde == AW_PDE_MHD_GLM)
        AW_FAIL(AW_EINVAL, "reflective walls are available for the Euler equations and linear advection");
    }
  }
  if (!(c.cfl > 0.0)) AW_FAIL(AW_EINVAL, "cfl must be positive");
  if (c.flux != AW_FLUX_RUSANOV && c.flux != AW_FLUX_OSHER) AW_FAIL(AW_EINVAL, "unknown numerical flux %d", c.flux);
  aw_solver* s = new aw_solver();
  s->cfg = c;
  s->D = c.dim;
  s->M = c.M;
  s->N = c.M + 1;
  s->r = r;
  s->lmax = c.lmax;
  s->V = nvars(c.dim, c.pde);
  s->NSP = ipow(s->N, s->D);
  s->NST = s->NSP * s->N;
  s->P = c.picard_iters > 0 ? c.picard_iters : c.M + 1;
  s->stream = (cudaStream_t)stream;
  s->phys.gamma = c.gamma;
  s->phys.c_h = c.c_h;
  for (int a = 0; a < 3; a++) s->phys.adv[a] = c.adv[a];
  for (int v = 0; v < 9; v++) s->phys.inflow[v] = c.inflow[v];
  if (!get_ops(c.dim, c.M, c.pde, &s->ops)) {
    delete s;
    AW_FAIL(AW_EINVAL, "configuration dim=%d M=%d pde=%d is not compiled in", c.dim, c.M, c.pde);
  }
  if (!build_tables(c.M, r, &s->T)) {
    delete s;
    AW_FAIL(AW_EINVAL, "table construction failed");
  }
  int rc = AW_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  keep_pool(dev);
  auto alloc = [&](void** p, size_t bytes) {
    if (rc != AW_OK) return;
    if (dalloc(s, p, bytes) != cudaSuccess) {
      rc = AW_ENOMEM;
      char b[200];
      snprintf(b, sizeof b, "device allocation of %zu bytes failed", bytes);
      g_err = b;
    }
  };
  long long rr = 1;
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    L.L[0] = (int)(c.nx * rr);
    L.L[1] = (int)(c.ny * rr);
    L.L[2] = s->D == 3 ? (int)(c.nz * rr) : 1;
    L.n = (long long)L.L[0] * L.L[1] * L.L[2];
    L.dx[0] = (c.hi[0] - c.lo[0]) / c.nx;
    L.dx[1] = (c.hi[1] - c.lo[1]) / c.ny;
    L.dx[2] = s->D == 3 ? (c.hi[2] - c.lo[2]) / c.nz : 1.0;
    for (int k = 0; k < l; k++)
      for (int a = 0; a < s->D; a++) L.dx[a] /= s->r;
    L.ts = s->ops.weno_tile(L.n);
    int TS = L.ts;
    for (int a = 0; a < 3; a++) L.tdim[a] = a < s->D ? (L.L[a] + TS - 1) / TS : 1;
    L.ntd = (long long)L.tdim[0] * L.tdim[1] * L.tdim[2];
    alloc((void**)&L.st, L.n);
    alloc((void**)&L.R, L.n);
    alloc((void**)&L.nst, L.n);
    alloc((void**)&L.flag, L.n);
    alloc((void**)&L.u, L.n * s->V * sizeof(double));
    alloc((void**)&L.chi, L.n * sizeof(double));
    alloc((void**)&L.aid, L.n * sizeof(int32_t));
    alloc((void**)&L.alist, L.n * sizeof(int32_t));
    alloc((void**)&L.vlist, L.n * sizeof(int32_t));
    alloc((void**)&L.mlist, L.n * sizeof(int32_t));
    alloc((void**)&L.clist, L.n * sizeof(int32_t));
    alloc((void**)&L.tflag, L.ntd);
    alloc((void**)&L.tiles, L.ntd * sizeof(int32_t));
    // WENO by passes from 4096 cells by default (on tinier levels the tiles' single launch is
    // quicker)
    if (weno_by_passes(s) && L.n >= launch_params().pass_min_cells) {
      alloc((void**)&L.xmark, L.n);
      alloc((void**)&L.xslot, L.n * sizeof(int32_t));
      if (s->D == 3) {
        alloc((void**)&L.ymark, L.n);
        alloc((void**)&L.yslot, L.n * sizeof(int32_t));
      }
    }
    rr *= s->r;
  }
  alloc((void**)&s->d_dtl, sizeof(double) * MAXL);
  alloc((void**)&s->d_dtmin, sizeof(double));
  alloc((void**)&s->d_err, sizeof(int));
  alloc((void**)&s->d_cnt, sizeof(int) * (NSLOT * MAXL + 8));
  static_assert(sizeof(int) * (NSLOT * MAXL + 8) <= 256 && sizeof(double) * (MAXL + 1) <= 256, "pinned blocks");
  if (rc == AW_OK) {
    s->h_cnt = (int*)pinned_block();
    s->h_dtl = (double*)pinned_block();
    if (!s->h_cnt || !s->h_dtl) {
      rc = AW_ENOMEM;
      g_err = "pinned host allocation failed";
    }
  }
  if (rc != AW_OK) {
    free_solver(s);
    delete s;
    return rc;
  }
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    cudaMemsetAsync(L.st, l == 0 ? 0 : ST_NONE, L.n, s->stream);
    cudaMemsetAsync(L.u, 0, L.n * s->V * sizeof(double), s->stream);
    cudaMemsetAsync(L.chi, 0, L.n * sizeof(double), s->stream);
    cudaMemsetAsync(L.flag, 0, L.n, s->stream);
    cudaMemsetAsync(L.nst, ST_NONE, L.n, s->stream);
  }
  cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
  rc = rebuild_lists(s);
  if (rc != AW_OK) {
    free_solver(s);
    delete s;
    return rc;
  }
  *out = s;
  return AW_OK;
}

void aw_destroy(aw_solver* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  free_solver(s);
  delete s;
}

int aw_reset(aw_solver* s) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  s->mem_refused = 0;
  for (int l = 0; l <= s->lmax; l++) {
    Level& L = s->lev[l];
    CK(cudaMemsetAsync(L.st, l == 0 ? 0 : ST_NONE, L.n, s->stream));
    CK(cudaMemsetAsync(L.u, 0, L.n * s->V * sizeof(double), s->stream));
  }
  TRY(rebuild_lists(s));
  s->t = 0.0;
  return AW_OK;
}

int aw_set_memory_limit(aw_solver* s, int64_t bytes) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (bytes < 0) AW_FAIL(AW_EINVAL, "the memory limit must be >= 0 (0: none)");
  s->mem_limit = bytes;
  s->mem_refused = 0;
  return AW_OK;
}

}  // extern "C"

void aw::set_grow_hook(aw_solver* s, aw::GrowFn fn, void* ctx) {
  s->grow = fn;
  s->grow_ctx = ctx;
}

extern "C" {

int aw_get_memory(const aw_solver* s, int64_t* live, int64_t* peak, int64_t* refused) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (live) *live = s->mem_live;
  if (peak) *peak = s->mem_peak;
  if (refused) *refused = s->mem_refused;
  return AW_OK;
}

int aw_graph_stats(const aw_solver* s, int64_t* reuses, int64_t* updates, int64_t* instantiations) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (reuses) *reuses = s->graph_reuses;
  if (updates) *updates = s->graph_updates;
  if (instantiations) *instantiations = s->graph_instantiations;
  return AW_OK;
}

int aw_set_profiling(aw_solver* s, int32_t on) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  s->prof = on ? 1 : 0;
  return AW_OK;
}

int aw_kernel_times(aw_solver* s, double* ms, int64_t* launches) {
  if (!s || !ms || !launches) AW_FAIL(AW_EINVAL, "null argument");
  CK(cudaStreamSynchronize(s->stream));
  harvest_events(s);
  for (int k = 0; k < 8; k++) {
    ms[k] = s->kind_ms[k];
    launches[k] = s->kind_n[k];
    s->kind_ms[k] = 0.0;
    s->kind_n[k] = 0;
  }
  return AW_OK;
}

int aw_sync(aw_solver* s) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_set_initial(aw_solver* s, int32_t ic_kind, const double* params, int32_t nparams, int32_t nrefine) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (ic_kind < AW_IC_CONST || ic_kind > AW_IC_FOURIER) AW_FAIL(AW_EINVAL, "unknown initial condition %d", ic_kind);
  if (nparams < 0 || nparams > 128 || (nparams > 0 && !params)) AW_FAIL(AW_EINVAL, "bad parameter array");
  if ((ic_kind == AW_IC_VORTEX || ic_kind == AW_IC_RP4) && s->D != 2) AW_FAIL(AW_EINVAL, "initial condition is 2D");
  if (ic_kind == AW_IC_OT && s->cfg.pde != AW_PDE_MHD_GLM) AW_FAIL(AW_EINVAL, "Orszag-Tang data needs the MHD system");
  s->ic = ic_kind;
  s->icp.assign(params, params + nparams);
  s->icp.resize(128, 0.0);
  IcArgs I = ic_args(s);
  for (int l = 0; l <= s->lmax; l++) {
    k_ic<<<nblk(s->lev[l].n, 128), 128, 0, s->stream>>>(view(s, l), I, nullptr, nullptr, 0);
    s->launches++;
  }
  CK(cudaGetLastError());
  TRY(average_all(s));
  s->t = 0.0;
  int passes = nrefine < 0 ? s->lmax : nrefine;
  for (int p = 0; p < passes; p++) TRY(regrid(s, 1));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_set_cell_averages(aw_solver* s, const double* u_host, int64_t n) {
  if (!s || (!u_host && n > 0)) AW_FAIL(AW_EINVAL, "null argument");
  int64_t nc = total_cells(s);
  if (n != nc) AW_FAIL(AW_EINVAL, "expected %lld cells, got %lld", (long long)nc, (long long)n);
  TRY(ensure_buf(s, nc * s->V));
  CK(cudaMemcpyAsync(s->d_buf, u_host, sizeof(double) * nc * s->V, cudaMemcpyHostToDevice, s->stream));
  long long off = 0;
  for (int l = 0; l <= s->lmax; l++) {
    const Level& L = s->lev[l];
    if (L.nc > 0) {
      k_scatter<<<nblk(L.nc, 256), 256, 0, s->stream>>>(view(s, l), L.clist, L.nc, s->V, s->d_buf + off * s->V);
      s->launches++;
    }
    off += L.nc;
  }
  CK(cudaGetLastError());
  TRY(average_all(s));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_compute_dt(aw_solver* s, double* dt0) {
  if (!s || !dt0) AW_FAIL(AW_EINVAL, "null argument");
  return compute_dt(s, dt0);
}

int aw_step_dt(aw_solver* s, double dt0, aw_stats* st) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (!(dt0 > 0.0)) AW_FAIL(AW_EINVAL, "dt0 must be positive");
  if (st) memset(st, 0, sizeof *st);
  int rc = step_dt(s, dt0, st);
  s->t += dt0;
  if (st) st->t = s->t;
  return rc;
}

static int step_cfl(aw_solver* s, double t_end, aw_stats* st) {
  double dt;
  TRY(compute_dt(s, &dt));
  bool clip = s->t + dt >= t_end;
  if (clip) dt = t_end - s->t;
  int rc = step_dt(s, dt, st);
  s->t = clip ? t_end : s->t + dt;
  if (rc != AW_OK) return rc;
  if (s->cfg.auto_regrid && s->lmax > 0) TRY(regrid(s, 0));
  return AW_OK;
}

int aw_step(aw_solver* s, double t_end, aw_stats* st) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (st) memset(st, 0, sizeof *st);
  if (!(t_end > s->t)) AW_FAIL(AW_EINVAL, "t_end %g is not after t %g", t_end, s->t);
  int rc = step_cfl(s, t_end, st);
  if (st) st->t = s->t;
  return rc;
}

int aw_advance_to(aw_solver* s, double t_end, aw_stats* st) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (st) memset(st, 0, sizeof *st);
  while (s->t < t_end) {
    int rc = step_cfl(s, t_end, st);
    if (rc != AW_OK) {
      if (st) st->t = s->t;
      return rc;
    }
  }
  if (st) st->t = s->t;
  return AW_OK;
}

// ------------------------------------------------------------------------------------------
// Cross-request batching: independent solves of one kernel configuration advanced in lockstep
// level-0 steps; every hot kernel of a (level, sub-step) runs once for all members.
// ------------------------------------------------------------------------------------------
}  // extern "C"

static_assert(AW_BATCH_MAX <= MAXB, "a batch fits one kernel parameter block");

// one step of level l (the recursion of advance()) for every live member whose finest level is
// at least l; *launches counts the batched launches
static int advance_batch(aw_solver* const* S, int n, const bool* live, int l, int sub, cudaStream_t st,
                         int64_t* launches) {
  HotBatch b;
  b.n = 0;
  int idx[MAXB];
  bool deeper = false;
  for (int m = 0; m < n; m++) {
    if (!live[m] || S[m]->lmax < l) continue;
    idx[b.n] = m;
    b.a[b.n++] = make_args(S[m], l, sub);
    if (S[m]->lmax > l) deeper = true;
  }
  if (b.n == 0) return AW_OK;
  const HotOps& ops = S[idx[0]]->ops;
  const int r = S[idx[0]]->r;
  // the persistent level kernel: projection, WENO and predictor of every member in one launch, and
  // the fused face flux and update too when no member has a finer level to step in between
  const LaunchParams lp = launch_params();
  const bool capturing = S[idx[0]]->capturing;
  const int lk = (ops.level_b && lp.persistent && lp.fuse_flux_update && !capturing)
                     ? ops.level_b(b, deeper ? 0 : 1, st)
                     : -1;
  if (lk >= 0) {
    *launches += lk;
  } else {
    if (l >= 1) *launches += ops.project_b(b, st);
    *launches += ops.weno_b(b, st);
    *launches += ops.predict_b(b, st);
  }
  CK(cudaGetLastError());
  if (deeper)
    for (int k = 0; k < r; k++) TRY(advance_batch(S, n, live, l + 1, k, st, launches));
  if (lk >= 0 && !deeper) {
    // done in the persistent kernel
  } else if (lp.fuse_flux_update) {
    *launches += ops.flux_update_b(b, st);
  } else {
    *launches += ops.flux_b(b, st);
    *launches += ops.update_b(b, st);
  }
  CK(cudaGetLastError());
  if (l >= 1 && sub == r - 1)
    for (int k = 0; k < b.n; k++) TRY(average_into(S[idx[k]], l - 1));
  return AW_OK;
}

// Returns a failure of the batch as a whole (CUDA errors); a member's own failure (non-physical
// state, no stable time step) stops that member only and is reported through rcs[m], *first and
// *first_err.
static int batch_run(aw_solver* const* S, int n, const double* tend, bool one_step, cudaStream_t st,
                     aw_stats* stats, int32_t* rcs, int* first, std::string* first_err) {
  bool live[MAXB];
  auto fail = [&](int m, int rc) {
    live[m] = false;
    rcs[m] = rc;
    if (*first == AW_OK) {
      *first = rc;
      *first_err = g_err;
    }
  };
  for (int m = 0; m < n; m++) {
    live[m] = S[m]->t < tend[m];
    rcs[m] = AW_OK;
  }
  double dt[MAXB];
  bool clip[MAXB];
  std::vector<char> sig;
  for (int iter = 0;; iter++) {
    int nlive = 0;
    for (int m = 0; m < n; m++) nlive += live[m];
    if (!nlive || (one_step && iter == 1)) break;
    // the time step of every member, one synchronisation
    for (int m = 0; m < n; m++) if (live[m]) TRY(dt_issue(S[m]));
    CK(cudaStreamSynchronize(st));
    for (int m = 0; m < n; m++) {
      if (!live[m]) continue;
      int rc = dt_finish(S[m], &dt[m]);
      if (rc != AW_OK) { fail(m, rc); continue; }
      clip[m] = S[m]->t + dt[m] >= tend[m];
      if (clip[m]) dt[m] = tend[m] - S[m]->t;
      rc = step_begin(S[m], dt[m]);
      if (rc != AW_OK) fail(m, rc);
    }
    // the step of every member, the hot kernels batched
    int64_t nl = 0;
    int rc;
    if (launch_params().graph_steps) {
      step_signature(S, n, live, &sig);
      rc = graph_replay(S, n, st, &S[0]->bgraph, sig, &nl,
                        [&](cudaStream_t gs) { return advance_batch(S, n, live, 0, 0, gs, &nl); });
    } else {
      rc = advance_batch(S, n, live, 0, 0, st, &nl);
    }
    for (int m = 0; m < n; m++)
      if (live[m]) { S[m]->launches += nl; break; }
    TRY(rc);
    for (int m = 0; m < n; m++)
      if (live[m]) CK(cudaMemcpyAsync(S[m]->h_cnt + NSLOT * MAXL, S[m]->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int m = 0; m < n; m++) {
      if (!live[m]) continue;
      aw_stats one;
      memset(&one, 0, sizeof one);
      rc = step_finish(S[m], dt[m], &one);
      S[m]->t = clip[m] ? tend[m] : S[m]->t + dt[m];
      if (stats) {
        stats[m].level0_steps += one.level0_steps;
        stats[m].cell_updates += one.cell_updates;
        for (int l = 0; l < 8; l++) stats[m].updates_per_level[l] += one.updates_per_level[l];
        stats[m].last_dt0 = one.last_dt0;
        stats[m].t = S[m]->t;
      }
      if (rc != AW_OK) { fail(m, rc); continue; }
    }
    // regrids of the live members (the same device work as regrid(), the two host
    // synchronisations of the list rebuild shared by all members)
    bool rg[MAXB];
    int nrg = 0;
    for (int m = 0; m < n; m++) {
      rg[m] = live[m] && S[m]->cfg.auto_regrid && S[m]->lmax > 0;
      if (!rg[m]) continue;
      // a member whose regrid cannot be issued (its memory limit, say) stops alone
      rc = regrid_prepass(S[m], 0);
      if (rc == AW_OK) rc = flags_from_chi(S[m]);
      if (rc == AW_OK) rc = apply_flags_issue(S[m], 0);
      if (rc == AW_OK) rc = lists_issue(S[m]);
      if (rc != AW_OK) {
        fail(m, rc);
        rg[m] = false;
        continue;
      }
      nrg++;
    }
    if (nrg) {
      CK(cudaStreamSynchronize(st));
      for (int m = 0; m < n; m++) {
        if (!rg[m]) continue;
        rc = lists_mid(S[m]);
        if (rc != AW_OK) { fail(m, rc); rg[m] = false; }
      }
      CK(cudaStreamSynchronize(st));
      for (int m = 0; m < n; m++) {
        if (!rg[m]) continue;
        rc = lists_finish(S[m]);
        if (rc != AW_OK) { fail(m, rc); continue; }
        TRY(average_all(S[m]));
      }
    }
    for (int m = 0; m < n; m++)
      if (live[m] && !(S[m]->t < tend[m])) live[m] = false;
  }
  return AW_OK;
}

extern "C" {

}  // extern "C"

// aw_advance_batch (one_step false) and aw_step_batch (one_step true): member m advances to tend[m]
static int batch_call(aw_solver* const* solvers, int32_t n, const double* tend, bool one_step, uintptr_t stream,
                      aw_stats* stats, int32_t* rc_out) {
  if (!solvers || n < 1 || n > AW_BATCH_MAX) AW_FAIL(AW_EINVAL, "need 1 <= n <= %d solvers", AW_BATCH_MAX);
  for (int m = 0; m < n; m++) {
    const aw_solver* a = solvers[m];
    if (!a) AW_FAIL(AW_EINVAL, "null solver %d", m);
    const aw_solver* z = solvers[0];
    if (a->D != z->D || a->cfg.pde != z->cfg.pde || a->M != z->M || a->cfg.flux != z->cfg.flux || a->r != z->r)
      AW_FAIL(AW_EINVAL, "solver %d differs from solver 0 in dim, pde, M, flux or refine_factor", m);
    for (int k = 0; k < m; k++)
      if (solvers[k] == a) AW_FAIL(AW_EINVAL, "solver %d appears twice", m);
    if (std::isnan(tend[m])) AW_FAIL(AW_EINVAL, "end time of solver %d is NaN", m);
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaStream_t own[MAXB];
  for (int m = 0; m < n; m++) {
    CK(cudaStreamSynchronize(solvers[m]->stream));
    own[m] = solvers[m]->stream;
    solvers[m]->stream = st;
  }
  if (stats) memset(stats, 0, sizeof(aw_stats) * n);
  int32_t rcs[MAXB];
  for (int m = 0; m < n; m++) rcs[m] = AW_OK;
  int first = AW_OK;
  std::string first_err;
  int fatal = batch_run(solvers, n, tend, one_step, st, stats, rcs, &first, &first_err);
  std::string fatal_err = g_err;
  cudaError_t e = cudaStreamSynchronize(st);
  if (fatal == AW_OK && e != cudaSuccess) {
    fatal = AW_ECUDA;
    fatal_err = std::string("batched advance: ") + cudaGetErrorString(e);
  }
  for (int m = 0; m < n; m++) {
    solvers[m]->stream = own[m];
    if (stats) stats[m].t = solvers[m]->t;
    if (fatal != AW_OK && rcs[m] == AW_OK && solvers[m]->t < tend[m]) rcs[m] = fatal;
    if (rc_out) rc_out[m] = rcs[m];
  }
  if (fatal != AW_OK) {
    g_err = fatal_err;
    return fatal;
  }
  if (first != AW_OK) g_err = first_err;
  return first;
}

extern "C" {

int aw_advance_batch(aw_solver* const* solvers, int32_t n, double t_end, uintptr_t stream, aw_stats* stats,
                     int32_t* rc_out) {
  double tend[MAXB];
  for (int m = 0; m < MAXB; m++) tend[m] = t_end;
  return batch_call(solvers, n, tend, false, stream, stats, rc_out);
}

int aw_step_batch(aw_solver* const* solvers, int32_t n, const double* t_end, uintptr_t stream, aw_stats* stats,
                  int32_t* rc_out) {
  if (!t_end) AW_FAIL(AW_EINVAL, "null end times");
  return batch_call(solvers, n, t_end, true, stream, stats, rc_out);
}

int aw_advance_graph(aw_solver* s, double t_end, int32_t chunk, aw_stats* st) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (st) memset(st, 0, sizeof *st);
  if (s->lmax != 0) AW_FAIL(AW_EINVAL, "the graph path needs a uniform mesh (lmax = 0)");
  if (chunk < 1 || chunk > 256) AW_FAIL(AW_EINVAL, "chunk must be 1..256 level-0 steps");
  if (!(t_end > s->t)) {
    if (st) st->t = s->t;
    return AW_OK;
  }
  if (!s->d_gs) {
    if (dalloc(s, (void**)&s->d_gs, sizeof(GState)) != cudaSuccess) AW_FAIL(oom_code(s), "graph state");
    s->h_gs = (GState*)pinned_block();
    if (!s->h_gs) AW_FAIL(AW_ENOMEM, "pinned host allocation failed");
    static_assert(sizeof(GState) <= 256, "pinned block");
  }
  if (!s->gstream) CK(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
  cudaStream_t gs = s->gstream;
  // the state on the device, after everything already ordered on the solver's stream
  memset(s->h_gs, 0, sizeof(GState));
  s->h_gs->t = s->t;
  s->h_gs->t_end = t_end;
  s->h_dtl[MAXL] = 1e300;
  CK(cudaMemcpyAsync(s->d_gs, s->h_gs, sizeof(GState), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(s->d_dtmin, s->h_dtl + MAXL, sizeof(double), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
  struct EventHolder {
    cudaEvent_t e = nullptr;
    ~EventHolder() {
      if (e) cudaEventDestroy(e);
    }
  } evh;
  CK(cudaEventCreateWithFlags(&evh.e, cudaEventDisableTiming));
  cudaEvent_t ev = evh.e;
  CK(cudaEventRecord(ev, s->stream));
  CK(cudaStreamWaitEvent(gs, ev, 0));
  // `chunk` level-0 steps: CFL reduction, device-side dt, the four hot kernels; captured once and
  // kept while the launch arguments (every pointer and size of the level) stay the same
  const Level& L = s->lev[0];
  HotArgs a = make_args(s, 0, 0);
  const bool fused = launch_params().fuse_flux_update != 0;
  const int per_step = 2 + (L.ntiles > 0 ? (a.xs ? s->D : 1) : 0) + (fused ? 2 : 3);
  cudaError_t ce = cudaSuccess;
  if (!s->gexec || s->gchunk != chunk || s->gfused != fused || memcmp(&s->gargs, &a, sizeof a) != 0) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
    cudaGraph_t graph = nullptr;
    ce = cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
      for (int k = 0; k < chunk; k++) {
        k_dt<<<nblk(L.na, 256), 256, 0, gs>>>(view(s, 0), L.alist, L.na, rtphys(s), s->cfg.cfl, 1.0, s->d_dtmin);
        k_dt_commit<<<1, 1, 0, gs>>>(s->d_dtmin, s->d_gs, s->d_dtl, s->r, s->d_err);
        s->ops.weno(a, gs);
        s->ops.predict(a, gs);
        if (fused) {
          s->ops.flux_update(a, gs);
        } else {
          s->ops.flux(a, gs);
          s->ops.update(a, gs);
        }
      }
      ce = cudaStreamEndCapture(gs, &graph);
    }
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&s->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      s->gexec = nullptr;
      AW_FAIL(AW_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    }
    memcpy(&s->gargs, &a, sizeof a);   // every byte, padding included, for the memcmp above
    s->gchunk = chunk;
    s->gfused = fused;
  }
  cudaGraphExec_t exec = s->gexec;
  // replay until the device time reaches t_end, one host synchronisation per chunk
  int rc = AW_OK, err = 0;
  for (;;) {
    ce = cudaGraphLaunch(exec, gs);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->h_gs, s->d_gs, sizeof(GState), cudaMemcpyDeviceToHost, gs);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(s->h_cnt + NSLOT * MAXL, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, gs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(gs);
    if (ce != cudaSuccess) {
      rc = AW_ECUDA;
      g_err = std::string("graph replay: ") + cudaGetErrorString(ce);
      break;
    }
    s->launches += (int64_t)per_step * chunk;
    err = s->h_cnt[NSLOT * MAXL];
    if (s->h_gs->stop || !(s->h_gs->t < t_end)) break;
  }
  cudaEventRecord(ev, gs);
  cudaStreamWaitEvent(s->stream, ev, 0);
  if (rc != AW_OK) return rc;
  s->t = s->h_gs->t;
  if (st) {
    st->level0_steps = s->h_gs->nsteps;
    st->cell_updates = s->h_gs->nsteps * (int64_t)L.na;
    st->updates_per_level[0] = st->cell_updates;
    st->last_dt0 = s->h_gs->last_dt0;
    st->t = s->t;
  }
  if (err & 1) AW_FAIL(AW_ENONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN) after the update");
  if (err & 8) AW_FAIL(AW_ENONPHYSICAL, "no positive stable time step");
  if (err) AW_FAIL(AW_ESTATE, "inconsistent mesh detected on the device (error word %d)", err);
  return AW_OK;
}

int aw_regrid(aw_solver* s, int32_t init_mode) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  if (init_mode && s->ic < 0) AW_FAIL(AW_ESTATE, "initial-condition regrid before aw_set_initial");
  TRY(regrid(s, init_mode));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_compute_flags(aw_solver* s, int32_t init_mode, int8_t* flags, int64_t cap, int64_t* n) {
  if (!s || !n) AW_FAIL(AW_EINVAL, "null argument");
  int64_t nc = total_cells(s);
  *n = nc;
  if (cap < nc) AW_FAIL(AW_EINVAL, "capacity %lld < %lld cells", (long long)cap, (long long)nc);
  if (s->lmax == 0) {
    memset(flags, 0, nc);
    return AW_OK;
  }
  TRY(regrid_prepass(s, init_mode));
  TRY(flags_from_chi(s));
  TRY(ensure_buf(s, nc / 8 + 1));
  int8_t* d = (int8_t*)s->d_buf;
  long long off = 0;
  for (int l = 0; l <= s->lmax; l++) {
    const Level& L = s->lev[l];
    if (L.nc > 0) {
      k_gather_i8<<<nblk(L.nc, 256), 256, 0, s->stream>>>(L.flag, L.clist, L.nc, d + off);
      s->launches++;
    }
    off += L.nc;
  }
  CK(cudaMemcpyAsync(flags, d, nc, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_regrid_with_flags(aw_solver* s, const int8_t* flags, int64_t n, int32_t init_mode) {
  if (!s || (!flags && n > 0)) AW_FAIL(AW_EINVAL, "null argument");
  int64_t nc = total_cells(s);
  if (n != nc) AW_FAIL(AW_EINVAL, "expected %lld flags, got %lld", (long long)nc, (long long)n);
  if (init_mode && s->ic < 0) AW_FAIL(AW_ESTATE, "initial-condition regrid before aw_set_initial");
  if (s->lmax == 0) return AW_OK;
  TRY(regrid_prepass(s, init_mode));
  TRY(ensure_buf(s, nc / 8 + 1));
  int8_t* d = (int8_t*)s->d_buf;
  CK(cudaMemcpyAsync(d, flags, nc, cudaMemcpyHostToDevice, s->stream));
  long long off = 0;
  for (int l = 0; l <= s->lmax; l++) {
    const Level& L = s->lev[l];
    CK(cudaMemsetAsync(L.flag, 0, L.n, s->stream));
    if (L.nc > 0) {
      k_scatter_i8<<<nblk(L.nc, 256), 256, 0, s->stream>>>(L.flag, L.clist, L.nc, d + off);
      s->launches++;
    }
    off += L.nc;
  }
  CK(cudaGetLastError());
  TRY(apply_flags(s, init_mode));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_get_counts(aw_solver* s, int64_t* n_cells, int64_t* n_active, int64_t* cpl, int64_t* apl) {
  if (!s) AW_FAIL(AW_EINVAL, "null solver");
  int64_t nc = 0, na = 0;
  for (int l = 0; l < 8; l++) {
    int64_t c = l <= s->lmax ? s->lev[l].nc : 0, a = l <= s->lmax ? s->lev[l].na : 0;
    if (cpl) cpl[l] = c;
    if (apl) apl[l] = a;
    nc += c;
    na += a;
  }
  if (n_cells) *n_cells = nc;
  if (n_active) *n_active = na;
  return AW_OK;
}

int aw_read_cells(aw_solver* s, aw_cell* meta, double* u, int64_t cap, int64_t* n) {
  if (!s || !n) AW_FAIL(AW_EINVAL, "null argument");
  int64_t nc = total_cells(s);
  *n = nc;
  if (cap < nc) AW_FAIL(AW_EINVAL, "capacity %lld < %lld cells", (long long)cap, (long long)nc);
  long long words = nc * s->V + (nc * (long long)sizeof(aw_cell) + 7) / 8;
  TRY(ensure_buf(s, words + 1));
  double* du = s->d_buf;
  aw_cell* dm = (aw_cell*)(s->d_buf + nc * s->V);
  long long off = 0;
  for (int l = 0; l <= s->lmax; l++) {
    const Level& L = s->lev[l];
    if (L.nc > 0) {
      k_gather<<<nblk(L.nc, 256), 256, 0, s->stream>>>(view(s, l), L.clist, L.nc, s->V, du + off * s->V, dm + off, l);
      s->launches++;
    }
    off += L.nc;
  }
  CK(cudaGetLastError());
  if (u) CK(cudaMemcpyAsync(u, du, sizeof(double) * nc * s->V, cudaMemcpyDeviceToHost, s->stream));
  if (meta) CK(cudaMemcpyAsync(meta, dm, sizeof(aw_cell) * nc, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_read_internal(aw_solver* s, int32_t what, int32_t level, double* buf, int64_t cap, int64_t* n) {
  if (!s || !n) AW_FAIL(AW_EINVAL, "null argument");
  if (level < 0 || level > s->lmax) AW_FAIL(AW_EINVAL, "level out of range");
  const Level& L = s->lev[level];
  int64_t cnt;
  const double* src = nullptr;
  switch (what) {
    case AW_INTERNAL_WENO: cnt = (int64_t)L.na * s->V * s->NSP; src = L.wh; break;
    case AW_INTERNAL_PREDICTOR: cnt = (int64_t)L.na * s->V * s->NST; src = L.qh; break;
    case AW_INTERNAL_FLUX: cnt = (int64_t)L.na * 2 * s->D * s->V; src = L.fl; break;
    case AW_INTERNAL_CHI: cnt = L.nc; break;
    default: AW_FAIL(AW_EINVAL, "unknown selector %d", what);
  }
  *n = cnt;
  if (cap < cnt) AW_FAIL(AW_EINVAL, "capacity %lld < %lld", (long long)cap, (long long)cnt);
  if (cnt == 0) return AW_OK;
  if (what == AW_INTERNAL_CHI) {
    TRY(ensure_buf(s, cnt));
    k_gather_d<<<nblk(cnt, 256), 256, 0, s->stream>>>(L.chi, L.clist, L.nc, s->d_buf);
    s->launches++;
    src = s->d_buf;
  }
  CK(cudaMemcpyAsync(buf, src, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return AW_OK;
}

int aw_get_time(aw_solver* s, double* t) {
  if (!s || !t) AW_FAIL(AW_EINVAL, "null argument");
  *t = s->t;
  return AW_OK;
}

int aw_totals(aw_solver* s, double* tot) {
  if (!s || !tot) AW_FAIL(AW_EINVAL, "null argument");
  for (int v = 0; v < s->V; v++) tot[v] = 0.0;
  for (int l = 0; l <= s->lmax; l++) {
    const Level& L = s->lev[l];
    if (L.na == 0) continue;
    int nb = (int)nblk(L.na, 256);
    TRY(ensure_buf(s, (long long)nb * s->V));
    k_partial<<<nb, 256, 0, s->stream>>>(view(s, l), L.alist, L.na, s->V, s->d_buf);
    s->launches++;
    std::vector<double> h((size_t)nb * s->V);
    CK(cudaMemcpyAsync(h.data(), s->d_buf, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    double vol = 1.0;
    for (int a = 0; a < s->D; a++) vol *= L.dx[a];
    for (int v = 0; v < s->V; v++) {
      double acc = 0.0;
      for (int b = 0; b < nb; b++) acc += h[(size_t)b * s->V + v];
      tot[v] += vol * acc;
    }
  }
  return AW_OK;
}

int aw_get_launch_params(aw_launch_params* out) {
  if (!out) AW_FAIL(AW_EINVAL, "null argument");
  LaunchParams p = launch_params();
  memset(out, 0, sizeof *out);
  out->pass_min_cells = p.pass_min_cells;
  out->tile8_min_cells = p.tile8_min_cells;
  out->small_ctas_per_sm = p.small_ctas_per_sm;
  out->fuse_flux_update = p.fuse_flux_update;
  out->autotune = p.autotune;
  out->persistent = p.persistent;
  out->graph_steps = p.graph_steps;
  return AW_OK;
}

int aw_set_launch_params(const aw_launch_params* in) {
  if (!in) AW_FAIL(AW_EINVAL, "null argument");
  if (in->pass_min_cells < 0 || in->tile8_min_cells < 0 || in->small_ctas_per_sm < 0 || in->small_ctas_per_sm > 64 ||
      (in->fuse_flux_update != 0 && in->fuse_flux_update != 1) || (in->autotune != 0 && in->autotune != 1) ||
      (in->persistent != 0 && in->persistent != 1) || (in->graph_steps != 0 && in->graph_steps != 1))
    AW_FAIL(AW_EINVAL, "launch parameters out of range");
  LaunchParams p;
  p.pass_min_cells = in->pass_min_cells;
  p.tile8_min_cells = in->tile8_min_cells;
  p.small_ctas_per_sm = in->small_ctas_per_sm;
  p.fuse_flux_update = in->fuse_flux_update;
  p.autotune = in->autotune;
  p.persistent = in->persistent;
  p.graph_steps = in->graph_steps;
  set_launch_params(p);
  return AW_OK;
}

int aw_get_tuning(aw_tune_entry* out, int32_t cap, int32_t* n) {
  if (!n || cap < 0 || (cap > 0 && !out)) AW_FAIL(AW_EINVAL, "null argument or negative capacity");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *n = (int32_t)g_tune.size();
  int32_t i = 0;
  for (const auto& kv : g_tune) {
    if (i >= cap) break;
    aw_tune_entry& e = out[i++];
    memset(&e, 0, sizeof e);
    std::tie(e.dim, e.M, e.pde, e.flux, e.kernel, e.size_class) = kv.first;
    e.choice = kv.second.choice;
    e.inherited = kv.second.inherited;
    for (int v = 0; v < 2; v++) {
      e.trials[v] = kv.second.trials[v];
      e.ns_per_cell[v] = kv.second.ns_per_cell[v];
    }
  }
  return AW_OK;
}

int aw_reset_tuning(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  g_tune_epoch++;
  return AW_OK;
}

int aw_tables_host(int32_t M, int32_t r, double* out, int64_t cap, int64_t* n) {
  if (!n) AW_FAIL(AW_EINVAL, "null argument");
  if (M < 1 || M > 3) AW_FAIL(AW_EINVAL, "M must be 1, 2 or 3");
  if (r < 2 || r > MAXR) AW_FAIL(AW_EINVAL, "r must be in 2..%d", MAXR);
  const int N = M + 1;
  const int64_t need = 11 + 5 * N + 7 * N * N + 2 * r * N + r * N * N + 4 * (N - 1) * (N - 1);
  *n = need;
  if (!out || cap < need) AW_FAIL(AW_EINVAL, "need room for %lld doubles", (long long)need);
  Tables T;
  if (!build_tables(M, r, &T)) AW_FAIL(AW_EINVAL, "table construction failed");
  int64_t k = 0;
  out[k++] = N;
  out[k++] = T.Ns;
  out[k++] = r;
  for (int i = 0; i < N; i++) out[k++] = T.x[i];
  for (int i = 0; i < N; i++) out[k++] = T.w[i];
  for (int s = 0; s < 4; s++) out[k++] = s < T.Ns ? T.SL[s] : 0.0;
  for (int s = 0; s < 4; s++) out[k++] = s < T.Ns ? T.lam[s] : 0.0;
  for (int s = 0; s < 4; s++)
    for (int p = 0; p < N; p++)
      for (int e = 0; e < N; e++) out[k++] = s < T.Ns ? T.Ainv[s][p][e] : 0.0;
  for (int p = 0; p < N; p++)
    for (int m = 0; m < N; m++) out[k++] = T.Sig[p][m];
  for (int i = 0; i < N; i++)
    for (int l = 0; l < N; l++) out[k++] = T.Dm[i][l];
  for (int a = 0; a < N; a++)
    for (int b = 0; b < N; b++) out[k++] = T.G[a][b];
  for (int l = 0; l < N; l++) out[k++] = T.psi0[l];
  for (int l = 0; l < N; l++) out[k++] = T.psi1[l];
  for (int c = 0; c < r; c++)
    for (int l = 0; l < N; l++) out[k++] = T.Wc[c][l];
  for (int c = 0; c < r; c++)
    for (int i = 0; i < N; i++)
      for (int l = 0; l < N; l++) out[k++] = T.Pf[c][i][l];
  for (int c = 0; c < r; c++)
    for (int l = 0; l < N; l++) out[k++] = T.Pt[c][l];
  for (int a = 0; a < N; a++) out[k++] = T.gsum[a];
  for (int s = 0; s < 4; s++)
    for (int i = 0; i < N - 1; i++)
      for (int j = 0; j < N - 1; j++) out[k++] = s < T.Ns ? T.Bq[s][i][j] : 0.0;
  return k == need ? AW_OK : AW_EINVAL;
}

int aw_cfl_dt_noalloc(const aw_config* cfg, const double* u_dev, int64_t n_cells, double* dt_dev, uintptr_t stream) {
  if (!cfg || !u_dev || !dt_dev) AW_FAIL(AW_EINVAL, "null argument");
  const aw_config& c = *cfg;
  if (c.dim != 2 && c.dim != 3) AW_FAIL(AW_EINVAL, "dim must be 2 or 3");
  if (c.pde < 0 || c.pde > 2) AW_FAIL(AW_EINVAL, "unknown pde %d", c.pde);
  if (c.nx < 1 || c.ny < 1 || (c.dim == 3 && c.nz < 1)) AW_FAIL(AW_EINVAL, "grid size must be positive");
  long long n = (long long)c.nx * c.ny * (c.dim == 3 ? c.nz : 1);
  if (n_cells != n) AW_FAIL(AW_EINVAL, "n_cells %lld does not match the %lld cells of the grid", (long long)n_cells, n);
  long long nb = (n + AW_NOALLOC_BLOCK - 1) / AW_NOALLOC_BLOCK;
  if (nb > AW_NOALLOC_SLOTS)
    AW_FAIL(AW_EINVAL, "aw_cfl_dt_noalloc handles at most %d cells (got %lld)", AW_NOALLOC_SLOTS * AW_NOALLOC_BLOCK, n);
  if (!(c.cfl > 0.0)) AW_FAIL(AW_EINVAL, "cfl must be positive");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) AW_FAIL(AW_EINVAL, "device ordinal %d out of range", dev);
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ready[dev]) {
      // once per device, with that device current: the host-side name of the array is not a
      // device address, so take the address from the runtime
      double* p = nullptr;
      CK(cudaGetSymbolAddress((void**)&p, g_noalloc_dt_scratch));
      g_noalloc_ptr[dev] = p;
      g_noalloc_ready[dev] = true;
    }
    scratch = g_noalloc_ptr[dev];
  }
  RtPhys R;
  R.pde = c.pde;
  R.D = c.dim;
  R.V = nvars(c.dim, c.pde);
  R.P.gamma = c.gamma;
  R.P.c_h = c.c_h;
  for (int a = 0; a < 3; a++) R.P.adv[a] = c.adv[a];
  double dx0 = (c.hi[0] - c.lo[0]) / c.nx, dx1 = (c.hi[1] - c.lo[1]) / c.ny;
  double dx2 = c.dim == 3 ? (c.hi[2] - c.lo[2]) / c.nz : 1.0;
  cudaStream_t st = (cudaStream_t)stream;
  k_dt_blockmin<<<(unsigned)nb, AW_NOALLOC_BLOCK, 0, st>>>(u_dev, n, R, dx0, dx1, dx2, c.cfl, scratch);
  k_dt_final<<<1, 1024, 0, st>>>(scratch, (int)nb, dt_dev);
  CK(cudaGetLastError());
  return AW_OK;
}

int aw_selftest_reciprocal(const double* x_dev, int64_t n, double* out_dev, uintptr_t stream) {
  if (!x_dev || !out_dev || n < 0) AW_FAIL(AW_EINVAL, "bad argument");
  if (n == 0) return AW_OK;
  k_selftest_rcp<<<nblk(n, 256), 256, 0, (cudaStream_t)stream>>>(x_dev, n, out_dev);
  CK(cudaGetLastError());
  return AW_OK;
}

int aw_selftest_flux_math(const double* x_dev, int64_t n, double* out_dev, uintptr_t stream) {
  if (!x_dev || !out_dev || n < 0) AW_FAIL(AW_EINVAL, "bad argument");
  if (n == 0) return AW_OK;
  k_selftest_flux_math<<<nblk(n, 256), 256, 0, (cudaStream_t)stream>>>(x_dev, n, out_dev);
  CK(cudaGetLastError());
  return AW_OK;
}

}  // extern "C"
