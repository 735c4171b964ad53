// aw_serve.cu -- request loop for independent AMR solves (continuous admission).
//
// Requests (a configuration, an initial condition and an end time) are queued by aw_srv_submit.
// Worker threads admit them in arrival order as soon as their device-memory reservation fits the
// remaining budget and a worker is free; each admitted request gets its own CUDA stream and
// solver, so the kernels of concurrent requests overlap on the GPU.  The solver runs with its
// reservation as its memory limit: a solve whose mesh outgrows the reservation has it grown in
// place while the budget has room beside the other running requests; otherwise it is refused the
// allocation (AW_ELIMIT), gives its memory back and is queued again at the head with a larger
// reservation, to run again from its initial condition once the budget has room.  A finished
// request's cell averages are copied to host memory and its device memory is released at once,
// which admits the next request.  Every request runs exactly the same kernels as a solve on its
// own, so its result does not depend on what else is running.
//
// With batching on (aw_srv_set_batching), a worker that admits the oldest request also admits
// queued requests of the same kernel configuration (up to the batch size, in arrival order, while
// the budget allows) and advances the group in lockstep level-0 steps with aw_step_batch: one
// launch per hot kernel, level and sub-step for the whole group.  Members leave the group when
// they finish and compatible requests join it between steps (run_continuous).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <tuple>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "aderweno.h"
#include "aw_device.cuh"
#include "aw_ops.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
  int64_t id;
  aw_config cfg;
  int32_t ic;
  std::vector<double> params;
  double t_end;
  int64_t footprint;
  int32_t state = AW_REQ_QUEUED;
  int32_t rc = AW_OK;
  std::string err;
  clk::time_point t_submit, t_start, t_done;
  int64_t cell_updates = 0, level0_steps = 0;
  int64_t requeues = 0, grows = 0, peak_bytes = 0, refused_bytes = 0;
  std::vector<aw_cell> meta;
  std::vector<double> u;
};

}  // namespace

struct aw_server {
  int device = 0;
  int64_t budget = 0, in_use = 0, peak_in_use = 0, requeues = 0, grows = 0;
  // per (dim, pde, M, lmax, r): the largest share of its finest level a run of that kind has held
  // per-active arrays for, learned from the runs' device bytes (first reservations use it)
  std::map<std::tuple<int, int, int, int, int>, double> active_share;
  int nworkers = 1;
  int max_batch = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<int64_t> queue;
  std::map<int64_t, Request> req;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_id = 1;
  int running = 0;
  clk::time_point t_first_submit;
  bool any_submitted = false;
};

// the part of a reservation that is not the solver's own allocations: the CUDA context's share
// and staging buffers
static const int64_t kAllowance = (int64_t)64 << 20;

// Device bytes of the dense per-level grids of `c` (exact, with the row marks and slot maps of the
// WENO by passes), of per-active arrays per active cell (the WENO sweep buffers counted at two rows
// per active cell), and the finest level's cell count.
static void footprint_parts(const aw_config& c, int64_t* dense, int64_t* per_active, int64_t* finest_cells,
                            int64_t* all_cells) {
  int V = aw::nvars(c.dim, c.pde), N = c.M + 1;
  int64_t nsp = 1;
  for (int a = 0; a < c.dim; a++) nsp *= N;
  int64_t nst = nsp * N;
  int64_t dense_per_cell = 8 * V + 4 + 8 + 4 * 5 + 5 * (c.dim == 3 ? 2 : 1);
  int64_t sweeps = 2 * 8 * V * N * (c.dim == 3 ? 1 + N : 1);
  *per_active = 8 * (V * nsp + V * nst + 4 * c.dim * V) + sweeps;
  int64_t total = 0, finest = 0, all = 0, rr = 1;
  int r = c.lmax > 0 ? c.refine_factor : 1;
  for (int l = 0; l <= c.lmax; l++) {
    int64_t n = (int64_t)c.nx * rr * c.ny * rr * (c.dim == 3 ? c.nz * rr : 1);
    total += n * dense_per_cell;
    finest = n;
    all += n;
    rr *= r;
  }
  *dense = total;
  *finest_cells = finest;
  *all_cells = all;
}

// Device bytes one solve of `c` is reserved with per-active arrays for `active_frac` of the finest
// level's cells (a quarter for a first reservation, unless the loop has learned more for this
// kind of run) plus the dense grids and the allowance.
static int64_t footprint_bytes(const aw_config& c, double active_frac = 0.25) {
  int64_t dense, per_active, finest, all;
  footprint_parts(c, &dense, &per_active, &finest, &all);
  if (active_frac > 1.0)   // every cell of every level active, with the arrays' growth headroom
    return dense + (int64_t)(1.5 * (double)all * (double)per_active) + kAllowance;
  return dense + (int64_t)(active_frac * (double)finest) * per_active + kAllowance;
}

// the bound on any reservation of `c`: every cell of every level active
static int64_t footprint_max(const aw_config& c) { return footprint_bytes(c, 2.0); }

static std::tuple<int, int, int, int, int> run_kind(const aw_config& c) {
  return std::make_tuple(c.dim, c.pde, c.M, c.lmax, c.refine_factor);
}

// A first reservation: per-active arrays for a quarter of the finest level, or for 1.25 times the
// largest share of it that runs of the same kind held so far, at most footprint_max.
static int64_t first_reservation(const aw_server* S, const aw_config& c) {
  double share = 0.25;
  auto it = S->active_share.find(run_kind(c));
  if (it != S->active_share.end()) share = std::max(share, 1.25 * it->second);
  if (share >= 1.0) return footprint_max(c);
  return std::min(footprint_bytes(c, share), footprint_max(c));
}

// what a finished or refused run of R tells about its kind: the share of the finest level its
// per-active arrays (and everything else above the dense grids) came to
static void learn_share(aw_server* S, const Request& R) {
  int64_t dense, per_active, finest, all;
  footprint_parts(R.cfg, &dense, &per_active, &finest, &all);
  const int64_t held = std::max(R.peak_bytes, R.refused_bytes) - dense;
  if (held <= 0 || finest <= 0 || per_active <= 0) return;
  const double share = (double)held / ((double)finest * (double)per_active);
  double& s = S->active_share[run_kind(R.cfg)];
  s = std::max(s, share);
}

// After a run that the solver's memory limit stopped (AW_ELIMIT): the next reservation, at least
// the bytes it was refused with half again as headroom and at least twice the old one, at most
// footprint_max and the budget; 0 if even the refused bytes exceed the budget.
static int64_t next_reservation(const aw_server* S, const Request& R) {
  const int64_t refused = R.refused_bytes + kAllowance;
  int64_t want = std::max(2 * R.footprint, refused + refused / 2);
  want = std::min(want, std::max(footprint_max(R.cfg), refused));
  if (want > S->budget) want = refused <= S->budget ? S->budget : 0;
  return want;
}

// A running solve that outgrows its reservation asks the loop for more (aw::set_grow_hook): the
// reservation grows in place, to the bytes asked for and half again (at most what every cell of
// every level active would take), or to just the bytes asked for, when the budget has room for the
// growth beside the other running requests' reservations; else the allocation is refused and the
// solve is queued again (AW_ELIMIT).  The growth is added to the worker's total, which it gives
// back when the run ends.
struct GrowCtx {
  aw_server* S;
  Request* R;
  int64_t* held;   // the worker's reserved bytes (all requests of its batch)
};

static int64_t grow_reservation(void* ctx, int64_t need) {
  GrowCtx* g = (GrowCtx*)ctx;
  aw_server* S = g->S;
  Request& R = *g->R;
  std::lock_guard<std::mutex> lk(S->mu);
  const int64_t have = R.footprint - kAllowance;
  if (need <= have) return have;
  const int64_t cap = std::max(footprint_max(R.cfg) - kAllowance, need);
  for (int64_t limit : {std::min(need + need / 2, cap), need}) {
    const int64_t extra = limit - have;
    if (S->in_use + extra > S->budget) continue;
    S->in_use += extra;
    S->peak_in_use = std::max(S->peak_in_use, S->in_use);
    *g->held += extra;
    R.footprint += extra;
    R.grows++;
    S->grows++;
    return limit;
  }
  return 0;
}

// the request's own stream; on failure the CUDA error goes into the request's message
static int create_stream(cudaStream_t* st, std::string* err) {
  cudaError_t e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
  if (e == cudaSuccess) return AW_OK;
  *st = nullptr;
  *err = std::string("stream creation failed: ") + cudaGetErrorString(e);
  return AW_ECUDA;
}

static void run_request(aw_server* S, Request& R, int64_t* held) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  aw_solver* sol = nullptr;
  std::string err0;
  GrowCtx gc{S, &R, held};
  int rc = create_stream(&st, &err0);
  if (rc == AW_OK) rc = aw_create(&R.cfg, (uintptr_t)st, &sol);
  if (rc == AW_OK) rc = aw_set_memory_limit(sol, std::max<int64_t>(R.footprint - kAllowance, 1));
  if (rc == AW_OK) aw::set_grow_hook(sol, grow_reservation, &gc);
  if (rc == AW_OK)
    rc = aw_set_initial(sol, R.ic, R.params.empty() ? nullptr : R.params.data(), (int32_t)R.params.size(), -1);
  aw_stats stats;
  memset(&stats, 0, sizeof stats);
  if (rc == AW_OK) rc = aw_advance_to(sol, R.t_end, &stats);
  if (rc == AW_OK) {
    int64_t n = 0;
    aw_get_counts(sol, &n, nullptr, nullptr, nullptr);
    R.meta.resize(n);
    R.u.resize((size_t)n * aw::nvars(R.cfg.dim, R.cfg.pde));
    rc = aw_read_cells(sol, R.meta.data(), R.u.data(), n, &n);
  }
  if (rc != AW_OK) R.err = err0.empty() ? aw_last_error() : err0;
  R.cell_updates = stats.cell_updates;
  R.level0_steps = stats.level0_steps;
  if (sol) aw_get_memory(sol, nullptr, &R.peak_bytes, &R.refused_bytes);
  aw_destroy(sol);
  if (st) cudaStreamDestroy(st);
  R.rc = rc;
}

// requests that can share batched launches with R (end times may differ: continuous batching
// steps each member to its own)
static bool batchable(const Request& R, const Request& Q) {
  return R.cfg.dim == Q.cfg.dim && R.cfg.pde == Q.cfg.pde && R.cfg.M == Q.cfg.M && R.cfg.flux == Q.cfg.flux &&
         R.cfg.refine_factor == Q.cfg.refine_factor;
}

// The end of a run of R, under the lock, after its reservation has been given back: the loop
// learns from its device bytes; an outgrown run (AW_ELIMIT) goes into `again` with a larger
// reservation, to be queued at the head; else the request is DONE or FAILED.
static void finish_locked(aw_server* S, Request* R, std::vector<int64_t>* again) {
  learn_share(S, *R);
  if (R->rc == AW_ELIMIT) {
    const int64_t next = next_reservation(S, *R);
    if (next > 0) {
      R->footprint = next;
      R->requeues++;
      S->requeues++;
      R->state = AW_REQ_QUEUED;
      R->rc = AW_OK;
      R->err.clear();
      R->refused_bytes = 0;
      again->push_back(R->id);
      return;
    }
    R->rc = AW_ENOMEM;
    R->err = "the solve needs more device memory than the whole budget of the loop";
  }
  R->state = R->rc == AW_OK ? AW_REQ_DONE : AW_REQ_FAILED;
}

// Continuous batching (max_batch > 1): the worker advances its group in lockstep level-0 steps
// (aw_step_batch), each member to its own end time.  A member that finishes or fails leaves the
// group at once: its cell averages go to host memory, its solver and reservation are released and
// waiting callers are woken.  Between steps the worker admits queued requests that can share the
// group's launches (in arrival order, up to the batch size) when their reservations fit the
// budget beside the other running requests and the oldest queued request.  The group ends when it
// has no members left.
struct Member {
  Request* R = nullptr;
  aw_solver* sol = nullptr;
  GrowCtx gc{};
};

static void run_continuous(aw_server* S, std::vector<Request*> G, int64_t* held) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  std::string err0;
  const int rc0 = create_stream(&st, &err0);
  const Request proto = *G[0];   // the kernel configuration of the group
  std::vector<std::unique_ptr<Member>> mem;
  // a member's end: results, solver, reservation, state
  auto leave = [&](Member& m, int rc, const std::string& err) {
    Request& R = *m.R;
    if (rc == AW_OK) {
      int64_t nc = 0;
      aw_get_counts(m.sol, &nc, nullptr, nullptr, nullptr);
      R.meta.resize(nc);
      R.u.resize((size_t)nc * aw::nvars(R.cfg.dim, R.cfg.pde));
      rc = aw_read_cells(m.sol, R.meta.data(), R.u.data(), nc, &nc);
      if (rc != AW_OK) R.err = aw_last_error();
    } else {
      R.err = err;
    }
    R.rc = rc;
    if (m.sol) aw_get_memory(m.sol, nullptr, &R.peak_bytes, &R.refused_bytes);
    aw_destroy(m.sol);
    m.sol = nullptr;
    std::vector<int64_t> again;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      R.t_done = clk::now();
      S->in_use -= R.footprint;
      *held -= R.footprint;
      S->running--;
      finish_locked(S, &R, &again);
      for (auto it = again.rbegin(); it != again.rend(); ++it) S->queue.push_front(*it);
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  };
  // a new member: solver, memory limit and growth hook, initial condition
  auto join = [&](Request* R) {
    auto m = std::make_unique<Member>();
    m->R = R;
    m->gc = GrowCtx{S, R, held};
    int rc = rc0;
    if (rc == AW_OK) rc = aw_create(&R->cfg, (uintptr_t)st, &m->sol);
    if (rc == AW_OK) rc = aw_set_memory_limit(m->sol, std::max<int64_t>(R->footprint - kAllowance, 1));
    if (rc == AW_OK) aw::set_grow_hook(m->sol, grow_reservation, &m->gc);
    if (rc == AW_OK)
      rc = aw_set_initial(m->sol, R->ic, R->params.empty() ? nullptr : R->params.data(), (int32_t)R->params.size(), -1);
    if (rc != AW_OK) {
      leave(*m, rc, rc0 == AW_OK ? std::string(aw_last_error()) : err0);
      return;
    }
    mem.push_back(std::move(m));
  };
  for (Request* R : G) join(R);
  std::vector<aw_solver*> sol;
  std::vector<double> tend;
  std::vector<aw_stats> stats;
  std::vector<int32_t> rcs;
  while (!mem.empty()) {
    const int n = (int)mem.size();
    sol.resize(n);
    tend.resize(n);
    stats.assign(n, aw_stats{});
    rcs.assign(n, AW_OK);
    for (int k = 0; k < n; k++) {
      sol[k] = mem[k]->sol;
      tend[k] = mem[k]->R->t_end;
    }
    const int rc = aw_step_batch(sol.data(), n, tend.data(), (uintptr_t)st, stats.data(), rcs.data());
    const std::string msg = rc != AW_OK ? aw_last_error() : "";
    std::vector<std::unique_ptr<Member>> keep;
    for (int k = 0; k < n; k++) {
      Member& m = *mem[k];
      m.R->cell_updates += stats[k].cell_updates;
      m.R->level0_steps += stats[k].level0_steps;
      if (rcs[k] != AW_OK)
        leave(m, rcs[k], msg.empty() ? "failed in a batch" : "failed in a batch (first failure of the step: " + msg + ")");
      else if (!(stats[k].t < m.R->t_end))
        leave(m, AW_OK, "");
      else
        keep.push_back(std::move(mem[k]));
    }
    mem = std::move(keep);
    // admit queued requests that can share the launches
    std::vector<Request*> add;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto it = S->queue.begin(); it != S->queue.end() && (int)(mem.size() + add.size()) < S->max_batch;) {
        Request& Q = S->req[*it];
        if (Q.requeues == 0) Q.footprint = std::min(first_reservation(S, Q.cfg), S->budget);
        const Request& head = S->req[S->queue.front()];
        const int64_t keep_free = *it == S->queue.front() ? 0 : head.footprint;
        if (S->stop || !batchable(proto, Q) || S->in_use + Q.footprint + keep_free > S->budget) {
          ++it;
          continue;
        }
        S->in_use += Q.footprint;
        S->peak_in_use = std::max(S->peak_in_use, S->in_use);
        *held += Q.footprint;
        S->running++;
        Q.state = AW_REQ_RUNNING;
        Q.t_start = clk::now();
        add.push_back(&Q);
        it = S->queue.erase(it);
      }
    }
    for (Request* R : add) join(R);
  }
  if (st) cudaStreamDestroy(st);
}

static void worker_main(aw_server* S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // the oldest queued request that fits the remaining budget (arrival order)
    int64_t pick = -1;
    S->cv_work.wait(lk, [&] {
      if (S->stop) return true;
      pick = -1;
      if (!S->queue.empty()) {
        int64_t id = S->queue.front();
        Request& Q = S->req[id];
        if (Q.requeues == 0) Q.footprint = std::min(first_reservation(S, Q.cfg), S->budget);
        if (S->in_use + Q.footprint <= S->budget) pick = id;
      }
      return pick >= 0;
    });
    if (S->stop) return;
    S->queue.pop_front();
    std::vector<Request*> G{&S->req[pick]};
    int64_t need = G[0]->footprint;
    // batching: compatible queued requests, in arrival order, while the budget allows
    for (auto it = S->queue.begin(); it != S->queue.end() && (int)G.size() < S->max_batch;) {
      Request& Q = S->req[*it];
      if (Q.requeues == 0) Q.footprint = std::min(first_reservation(S, Q.cfg), S->budget);
      if (batchable(*G[0], Q) && S->in_use + need + Q.footprint <= S->budget) {
        G.push_back(&Q);
        need += Q.footprint;
        it = S->queue.erase(it);
      } else {
        ++it;
      }
    }
    S->in_use += need;
    S->peak_in_use = std::max(S->peak_in_use, S->in_use);
    S->running += (int)G.size();
    const clk::time_point t0 = clk::now();
    for (Request* R : G) {
      R->state = AW_REQ_RUNNING;
      R->t_start = t0;
    }
    lk.unlock();
    if (S->max_batch > 1) {
      // every member releases its own reservation when it leaves the group
      run_continuous(S, G, &need);
      lk.lock();
      continue;
    }
    run_request(S, *G[0], &need);
    lk.lock();
    Request* R = G[0];
    R->t_done = clk::now();
    S->in_use -= need;
    S->running--;
    std::vector<int64_t> again;   // an outgrown run, back to the head of the queue
    finish_locked(S, R, &again);
    for (auto it = again.rbegin(); it != again.rend(); ++it) S->queue.push_front(*it);
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

static thread_local std::string g_srv_err;
#define SRV_FAIL(code, msg) \
  do {                      \
    g_srv_err = msg;        \
    return code;            \
  } while (0)

extern "C" {

const char* aw_srv_last_error(void) { return g_srv_err.c_str(); }

int aw_srv_create(int64_t hbm_budget_bytes, int32_t max_concurrent, aw_server** out) {
  if (!out || hbm_budget_bytes <= 0 || max_concurrent < 1 || max_concurrent > 256)
    SRV_FAIL(AW_EINVAL, "bad server arguments");
  aw_server* S = new aw_server();
  cudaGetDevice(&S->device);
  S->budget = hbm_budget_bytes;
  S->nworkers = max_concurrent;
  for (int i = 0; i < max_concurrent; i++) S->workers.emplace_back(worker_main, S);
  *out = S;
  return AW_OK;
}

int aw_srv_set_batching(aw_server* S, int32_t max_batch) {
  if (!S || max_batch < 1 || max_batch > AW_BATCH_MAX) SRV_FAIL(AW_EINVAL, "max_batch must be 1..AW_BATCH_MAX");
  std::lock_guard<std::mutex> lk(S->mu);
  S->max_batch = max_batch;
  return AW_OK;
}

int aw_srv_submit(aw_server* S, const aw_config* cfg, int32_t ic_kind, const double* params, int32_t nparams,
                  double t_end, int64_t* id) {
  if (!S || !cfg || !id || nparams < 0 || (nparams > 0 && !params)) SRV_FAIL(AW_EINVAL, "null argument");
  Request R;
  R.cfg = *cfg;
  R.ic = ic_kind;
  R.params.assign(params, params + nparams);
  R.t_end = t_end;
  R.footprint = footprint_bytes(*cfg);
  if (R.footprint > S->budget) SRV_FAIL(AW_EINVAL, "request needs more device memory than the whole budget");
  std::lock_guard<std::mutex> lk(S->mu);
  R.id = S->next_id++;
  R.t_submit = clk::now();
  if (!S->any_submitted) {
    S->any_submitted = true;
    S->t_first_submit = R.t_submit;
  }
  S->req[R.id] = std::move(R);
  S->queue.push_back(S->req.rbegin()->first);
  *id = S->req.rbegin()->first;
  S->cv_work.notify_all();
  return AW_OK;
}

int aw_srv_poll(aw_server* S, int64_t id, int32_t* state) {
  if (!S || !state) SRV_FAIL(AW_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->req.find(id);
  if (it == S->req.end()) SRV_FAIL(AW_EINVAL, "unknown request id");
  *state = it->second.state;
  return AW_OK;
}

int aw_srv_wait_all(aw_server* S) {
  if (!S) SRV_FAIL(AW_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_done.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
  return AW_OK;
}

int aw_srv_result(aw_server* S, int64_t id, aw_cell* meta, double* u, int64_t cap, int64_t* n, aw_srv_info* info) {
  if (!S || !n) SRV_FAIL(AW_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->req.find(id);
  if (it == S->req.end()) SRV_FAIL(AW_EINVAL, "unknown request id");
  Request& R = it->second;
  if (R.state == AW_REQ_FAILED) {
    g_srv_err = R.err;
    return R.rc;
  }
  if (R.state != AW_REQ_DONE) SRV_FAIL(AW_ESTATE, "request not finished");
  *n = (int64_t)R.meta.size();
  if (info) {
    info->cell_updates = R.cell_updates;
    info->level0_steps = R.level0_steps;
    info->queue_ms = std::chrono::duration<double, std::milli>(R.t_start - R.t_submit).count();
    info->run_ms = std::chrono::duration<double, std::milli>(R.t_done - R.t_start).count();
    info->total_ms = std::chrono::duration<double, std::milli>(R.t_done - R.t_submit).count();
    info->footprint_bytes = R.footprint;
    info->requeues = R.requeues;
    info->peak_bytes = R.peak_bytes;
    info->grows = R.grows;
  }
  if (cap < *n) SRV_FAIL(AW_EINVAL, "capacity too small");
  if (meta) memcpy(meta, R.meta.data(), sizeof(aw_cell) * R.meta.size());
  if (u) memcpy(u, R.u.data(), sizeof(double) * R.u.size());
  return AW_OK;
}

int aw_srv_stats(aw_server* S, aw_srv_summary* out) {
  if (!S || !out) SRV_FAIL(AW_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> tts;
  int64_t upd = 0, failed = 0;
  clk::time_point last = S->t_first_submit;
  for (auto& kv : S->req) {
    const Request& R = kv.second;
    if (R.state == AW_REQ_DONE) {
      tts.push_back(std::chrono::duration<double, std::milli>(R.t_done - R.t_submit).count());
      upd += R.cell_updates;
      last = std::max(last, R.t_done);
    } else if (R.state == AW_REQ_FAILED) {
      failed++;
    }
  }
  memset(out, 0, sizeof *out);
  out->done = (int64_t)tts.size();
  out->failed = failed;
  out->queued = (int64_t)S->queue.size();
  out->running = S->running;
  if (!tts.empty()) {
    std::sort(tts.begin(), tts.end());
    auto pct = [&](double p) {
      size_t k = (size_t)std::min<double>(tts.size() - 1, std::ceil(p * tts.size()) - 1);
      return tts[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double span = std::chrono::duration<double>(last - S->t_first_submit).count();
    out->solves_per_s = span > 0 ? tts.size() / span : 0.0;
    out->cell_updates_per_s = span > 0 ? upd / span : 0.0;
  }
  out->requeues = S->requeues;
  out->grows = S->grows;
  out->budget_bytes = S->budget;
  out->peak_reserved_bytes = S->peak_in_use;
  return AW_OK;
}

void aw_srv_destroy(aw_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->queue.clear();
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  // give the memory the solves kept in the device's pool back
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
  }
  delete S;
}

}  // extern "C"
