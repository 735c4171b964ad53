// aw_inst.cuh -- launchers of the hot kernels for one configuration; included by aw_inst_*.cu.
#pragma once
#include <mutex>

#include "aw_hot.cuh"

namespace aw {

// SMs of the current device (launch shapes for small levels)
inline int sm_count() {
  static std::once_flag once;
  static int n = 152;
  std::call_once(once, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
  });
  return n;
}

template <int D, int M, int PDE>
struct Launch {
  // WENO tiles, for levels below the passes threshold (4096 cells by default; larger levels run the
  // WENO by passes, k_weno_x/y and k_weno3_x/y/z, batched or not): 8x8 cells in 2D (6 sweep passes of 256
  // threads per 64 cells, against 2 per 16 with 4x4 tiles, whose x pass fills 160 of 256 lanes),
  // 4x4 on levels below 20,000 cells so that their tiles still spread over the SMs; 4x4x4 in 3D
  // (shared memory)
  static int weno_tile(long long n) { return (D == 2 && n >= launch_params().tile8_min_cells) ? 8 : 4; }
  using CP = PredCfg<D, M, PDE>;
  using CF = FluxCfg<D, M, PDE>;
  // about a quarter of the cells (face items) per CTA, filling whole warps, when the full-size CTAs
  // would give fewer than two CTAs per SM; every cell and face computes exactly the same either way
  static constexpr int SMALL = 4;
  using CPs = PredCfg<D, M, PDE, SMALL>;
  using CFs = FluxCfg<D, M, PDE, SMALL>;
  static constexpr int V = nvars(D, PDE);

  // CTAs of each kernel for one solve's level (0 when there is no work)
  static int weno_ctas(const HotArgs& a) { return a.ntiles > 0 ? a.ntiles : 0; }
  template <class C>
  static int predict_ctas_of(const HotArgs& a) { return a.na > 0 ? (a.na + C::CPB - 1) / C::CPB : 0; }
  static int predict_ctas(const HotArgs& a) { return predict_ctas_of<CP>(a); }
  template <class C>
  static int flux_ctas_of(const HotArgs& a) {
    if (a.na <= 0) return 0;
    long long lo = (long long)D * ((a.na + C::CPB - 1) / C::CPB);
    return (int)(lo + (a.nh + C::CPB - 1) / C::CPB);
  }
  static int flux_ctas(const HotArgs& a) { return flux_ctas_of<CF>(a); }
  static int update_ctas(const HotArgs& a) { return a.na > 0 ? (a.na + 127) / 128 : 0; }
  static int project_ctas(int nv) { return nv > 0 ? (int)(((long long)nv * V + 127) / 128) : 0; }
  static bool small(int ctas) { return ctas < launch_params().small_ctas_per_sm * sm_count(); }
  // reduced-size CTAs: the autotuner's choice for this launch, else the rule above
  static bool use_small(const HotArgs& a, int ctas) { return a.cta_div == 4 || (a.cta_div != 1 && small(ctas)); }

  // the dynamic shared memory attribute, once per kernel (request-loop workers launch concurrently)
  template <class K>
  static void smem_attr(K kernel, int bytes, std::once_flag& once) {
    std::call_once(once, [&] { cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
  }

  template <int TS>
  static void weno_launch(const HotArgs& a, int blocks, cudaStream_t st) {
    using C = WenoCfg<D, M, PDE, TS>;
    static std::once_flag init;
    smem_attr(k_weno<D, M, PDE, TS>, C::SMEM, init);
    k_weno<D, M, PDE, TS><<<blocks, 256, C::SMEM, st>>>(a);
  }
  static int weno(const HotArgs& a, cudaStream_t st) {
    const int blocks = weno_ctas(a);
    if (!blocks) return 0;
    constexpr int N = M + 1;
    if constexpr (D == 3) {
      if (a.xs && a.ys) {   // three passes: x sweeps of the feeding rows, y sweeps, z sweeps
        const long long nx = (long long)a.nxs * V, ny = (long long)a.nys * V, nz = (long long)a.na * N * V;
        k_weno3_x<M, PDE><<<(unsigned)((nx + 127) / 128), 128, 0, st>>>(a);
        k_weno3_y<M, PDE><<<(unsigned)((ny + 127) / 128), 128, 0, st>>>(a);
        k_weno3_z<M, PDE><<<(unsigned)((nz + 127) / 128), 128, 0, st>>>(a);
        return 3;
      }
    }
    if constexpr (D == 2) {
      if (a.xs) {   // two passes: the x sweeps of the feeding rows, then the y sweeps
        const long long nx = (long long)a.nxs * V, ny = (long long)a.na * N * V;
        k_weno_x<M, PDE><<<(unsigned)((nx + 127) / 128), 128, 0, st>>>(a);
        k_weno_y<M, PDE><<<(unsigned)((ny + 127) / 128), 128, 0, st>>>(a);
        return 2;
      }
      if (a.ts == 8) {
        weno_launch<8>(a, blocks, st);
        return 1;
      }
    }
    weno_launch<4>(a, blocks, st);
    return 1;
  }
  static int predict(const HotArgs& a, cudaStream_t st) {
    int blocks = predict_ctas_of<CP>(a);
    if (!blocks) return 0;
    if (use_small(a, blocks)) {
      static std::once_flag init;
      smem_attr(k_predict<D, M, PDE, SMALL>, CPs::SMEM, init);
      k_predict<D, M, PDE, SMALL><<<predict_ctas_of<CPs>(a), CPs::THREADS, CPs::SMEM, st>>>(a);
    } else {
      static std::once_flag init;
      smem_attr(k_predict<D, M, PDE, 1>, CP::SMEM, init);
      k_predict<D, M, PDE, 1><<<blocks, CP::THREADS, CP::SMEM, st>>>(a);
    }
    return 1;
  }
  // the face flux kernels of one numerical flux (FL: 0 Rusanov, 1 Osher-Solomon; Euler and MHD-GLM)
  template <int FL>
  static int flux_fl(const HotArgs& a, cudaStream_t st) {
    int blocks = flux_ctas_of<CF>(a);
    if (!blocks) return 0;
    if (use_small(a, blocks)) {
      static std::once_flag init;
      smem_attr(k_flux<D, M, PDE, SMALL, FL>, CFs::SMEM, init);
      k_flux<D, M, PDE, SMALL, FL><<<flux_ctas_of<CFs>(a), CFs::THREADS, CFs::SMEM, st>>>(a);
    } else {
      static std::once_flag init;
      smem_attr(k_flux<D, M, PDE, 1, FL>, CF::SMEM, init);
      k_flux<D, M, PDE, 1, FL><<<blocks, CF::THREADS, CF::SMEM, st>>>(a);
    }
    return 1;
  }
  static int flux(const HotArgs& a, cudaStream_t st) {
    if constexpr (PDE == PDE_EULER || PDE == PDE_MHD) {
      if (a.flux == 1) return flux_fl<1>(a, st);
    }
    return flux_fl<0>(a, st);
  }
  // fused face flux and update: one launch (the per-chunk arrival counters are zero between launches)
  template <int FL>
  static int flux_update_fl(const HotArgs& a, cudaStream_t st) {
    int blocks = flux_ctas_of<CF>(a);
    if (!blocks) return 0;
    if (use_small(a, blocks)) {
      static std::once_flag init;
      smem_attr(k_flux_update<D, M, PDE, SMALL, FL>, CFs::SMEM, init);
      k_flux_update<D, M, PDE, SMALL, FL><<<flux_ctas_of<CFs>(a), CFs::THREADS, CFs::SMEM, st>>>(a);
    } else {
      static std::once_flag init;
      smem_attr(k_flux_update<D, M, PDE, 1, FL>, CF::SMEM, init);
      k_flux_update<D, M, PDE, 1, FL><<<blocks, CF::THREADS, CF::SMEM, st>>>(a);
    }
    return 1;
  }
  static int flux_update(const HotArgs& a, cudaStream_t st) {
    if constexpr (PDE == PDE_EULER || PDE == PDE_MHD) {
      if (a.flux == 1) return flux_update_fl<1>(a, st);
    }
    return flux_update_fl<0>(a, st);
  }
  static int update(const HotArgs& a, cudaStream_t st) {
    const int blocks = update_ctas(a);
    if (!blocks) return 0;
    k_update<D, M, PDE><<<blocks, 128, 0, st>>>(a);
    return 1;
  }
  static int project(const HotArgs& a, const int32_t* vlist, int nv, const double* src, int spacetime,
                     double* out, int dense, cudaStream_t st) {
    const int blocks = project_ctas(nv);
    if (!blocks) return 0;
    k_project<D, M, PDE><<<blocks, 128, 0, st>>>(a, vlist, nv, src, spacetime, out, dense);
    return 1;
  }

  // batched launches: member m gets CTAs start[m] .. start[m+1]-1
  template <class F>
  static int fill_starts(HotBatch& b, F ctas) {
    int tot = 0;
    for (int m = 0; m < b.n; m++) {
      b.start[m] = tot;
      tot += ctas(b.a[m]);
    }
    b.start[b.n] = tot;
    return tot;
  }
  template <int TS>
  static int weno_b_ts(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, weno_ctas);
    if (!blocks) return 0;
    using C = WenoCfg<D, M, PDE, TS>;
    static std::once_flag init;
    smem_attr(k_weno_batch<D, M, PDE, TS>, C::SMEM, init);
    k_weno_batch<D, M, PDE, TS><<<blocks, 256, C::SMEM, st>>>(b);
    return 1;
  }
  // members whose level has 8x8 tiles and members with 4x4 tiles run as two launches
  // WENO by passes for the members whose level has them (one launch per pass over those members)
  template <class K>
  static int pass_b(HotBatch& b, K kernel, long long (*items)(const HotArgs&), cudaStream_t st) {
    const int blocks = fill_starts(b, [&](const HotArgs& a) { return (int)((items(a) + 127) / 128); });
    if (!blocks) return 0;
    kernel<<<blocks, 128, 0, st>>>(b);
    return 1;
  }
  static int weno_passes_b(HotBatch& b, cudaStream_t st) {
    constexpr int N = M + 1;
    if constexpr (D == 2) {
      int n = pass_b(b, k_weno_x_batch<M, PDE>, [](const HotArgs& a) { return (long long)a.nxs * V; }, st);
      return n + pass_b(b, k_weno_y_batch<M, PDE>, [](const HotArgs& a) { return (long long)a.na * N * V; }, st);
    } else {
      int n = pass_b(b, k_weno3_x_batch<M, PDE>, [](const HotArgs& a) { return (long long)a.nxs * V; }, st);
      n += pass_b(b, k_weno3_y_batch<M, PDE>, [](const HotArgs& a) { return (long long)a.nys * V; }, st);
      return n + pass_b(b, k_weno3_z_batch<M, PDE>, [](const HotArgs& a) { return (long long)a.na * N * V; }, st);
    }
  }
  static bool has_passes(const HotArgs& a) { return a.xs && (D == 2 || a.ys); }
  static int weno_b(HotBatch& b, cudaStream_t st) {
    int np = 0;
    for (int m = 0; m < b.n; m++) np += has_passes(b.a[m]);
    if (np == b.n) return weno_passes_b(b, st);
    if (np > 0) {
      HotBatch p, t;
      p.n = t.n = 0;
      for (int m = 0; m < b.n; m++) {
        if (has_passes(b.a[m])) p.a[p.n++] = b.a[m];
        else t.a[t.n++] = b.a[m];
      }
      return weno_passes_b(p, st) + weno_tiles_b(t, st);
    }
    return weno_tiles_b(b, st);
  }
  static int weno_tiles_b(HotBatch& b, cudaStream_t st) {
    if constexpr (D == 2) {
      bool mixed = false;
      for (int m = 1; m < b.n; m++) mixed |= b.a[m].ts != b.a[0].ts;
      if (!mixed) return b.a[0].ts == 8 ? weno_b_ts<8>(b, st) : weno_b_ts<4>(b, st);
      int n = 0;
      for (int ts : {8, 4}) {
        HotBatch g;
        g.n = 0;
        for (int m = 0; m < b.n; m++)
          if (b.a[m].ts == ts) g.a[g.n++] = b.a[m];
        if (g.n) n += ts == 8 ? weno_b_ts<8>(g, st) : weno_b_ts<4>(g, st);
      }
      return n;
    } else {
      return weno_b_ts<4>(b, st);
    }
  }
  static int predict_b(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, predict_ctas);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_predict_batch<D, M, PDE>, CP::SMEM, init);
    k_predict_batch<D, M, PDE><<<blocks, CP::THREADS, CP::SMEM, st>>>(b);
    return 1;
  }
  template <int FL>
  static int flux_b_fl(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, flux_ctas);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_flux_batch<D, M, PDE, FL>, CF::SMEM, init);
    k_flux_batch<D, M, PDE, FL><<<blocks, CF::THREADS, CF::SMEM, st>>>(b);
    return 1;
  }
  // every member of a batch has the same numerical flux
  static int flux_b(HotBatch& b, cudaStream_t st) {
    if constexpr (PDE == PDE_EULER || PDE == PDE_MHD) {
      if (b.n > 0 && b.a[0].flux == 1) return flux_b_fl<1>(b, st);
    }
    return flux_b_fl<0>(b, st);
  }
  template <int FL>
  static int flux_update_b_fl(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, flux_ctas);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_flux_update_batch<D, M, PDE, FL>, CF::SMEM, init);
    k_flux_update_batch<D, M, PDE, FL><<<blocks, CF::THREADS, CF::SMEM, st>>>(b);
    return 1;
  }
  static int flux_update_b(HotBatch& b, cudaStream_t st) {
    if constexpr (PDE == PDE_EULER || PDE == PDE_MHD) {
      if (b.n > 0 && b.a[0].flux == 1) return flux_update_b_fl<1>(b, st);
    }
    return flux_update_b_fl<0>(b, st);
  }
  static int update_b(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, update_ctas);
    if (!blocks) return 0;
    k_update_batch<D, M, PDE><<<blocks, 128, 0, st>>>(b);
    return 1;
  }
  static int project_b(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, [](const HotArgs& a) { return project_ctas(a.nv); });
    if (!blocks) return 0;
    k_project_batch<D, M, PDE><<<blocks, 128, 0, st>>>(b);
    return 1;
  }

  // The persistent level kernel (k_level_batch) of one level and sub-step of a batch: the work of
  // every phase per member, then one cooperative launch with as many CTAs as the GPU holds at
  // once (at most the largest phase's work).  Available where the predictor and the face flux
  // share their CTA shape.
  static constexpr bool kLevelKernel = PredCfg<D, M, PDE>::THREADS == FluxCfg<D, M, PDE>::THREADS;
  template <int FL>
  static int level_b_fl(HotBatch& b, int with_flux, cudaStream_t st) {
    constexpr int T = PredCfg<D, M, PDE>::THREADS, N = M + 1;
    constexpr int SMEM0 = PredCfg<D, M, PDE>::SMEM > FluxCfg<D, M, PDE>::SMEM ? PredCfg<D, M, PDE>::SMEM
                                                                                : FluxCfg<D, M, PDE>::SMEM;
    constexpr int SMEMW = (D == 2) ? WenoCfg<D, M, PDE, 8>::SMEM : WenoCfg<D, M, PDE, 4>::SMEM;
    constexpr int SMEM = SMEM0 > SMEMW ? SMEM0 : SMEMW;
    static LevelBatch lb;   // the 21 KB parameter block, built on the host (one batch at a time per process)
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    lb.b = b;
    lb.with_flux = with_flux;
    auto cdiv = [](long long x, long long y) { return (int)((x + y - 1) / y); };
    int most = 0;
    for (int p = 0; p < NPHASE; p++) {
      int tot = 0;
      for (int m = 0; m < b.n; m++) {
        const HotArgs& a = b.a[m];
        const bool passes = has_passes(a);
        int w = 0;
        switch (p) {
          case PH_PROJECT: w = a.level >= 1 ? cdiv((long long)a.nv * V, T) : 0; break;
          case PH_WENO4: w = (!passes && (D == 3 || a.ts != 8)) ? weno_ctas(a) : 0; break;
          case PH_WENO8: w = (!passes && D == 2 && a.ts == 8) ? weno_ctas(a) : 0; break;
          case PH_WENO_X: w = passes ? cdiv((long long)a.nxs * V, T) : 0; break;
          case PH_WENO_Y: w = passes ? cdiv((D == 2 ? (long long)a.na * N : (long long)a.nys) * V, T) : 0; break;
          case PH_WENO_Z: w = (passes && D == 3) ? cdiv((long long)a.na * N * V, T) : 0; break;
          case PH_PREDICT: w = predict_ctas(a); break;
          case PH_FLUX: w = with_flux ? flux_ctas(a) : 0; break;
        }
        lb.start[p][m] = tot;
        tot += w;
      }
      lb.start[p][b.n] = tot;
      most = std::max(most, tot);
    }
    if (!most) return 0;
    auto kernel = k_level_batch<D, M, PDE, FL>;
    static std::once_flag init;
    static int per_sm = 0;
    std::call_once(init, [&] {
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, T, SMEM) != cudaSuccess) per_sm = 0;
    });
    if (per_sm < 1) return -1;
    const int grid = std::min(most, per_sm * sm_count());
    void* args[] = {(void*)&lb};
    if (cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(T), args, SMEM, st) != cudaSuccess) {
      cudaGetLastError();   // a launch that could not start leaves no sticky error; the caller falls back
      return -1;
    }
    return 1;
  }
  static int level_b(HotBatch& b, int with_flux, cudaStream_t st) {
    if constexpr (!kLevelKernel) {
      return -1;
    } else {
      if constexpr (PDE == PDE_EULER || PDE == PDE_MHD) {
        if (b.n > 0 && b.a[0].flux == 1) return level_b_fl<1>(b, with_flux, st);
      }
      return level_b_fl<0>(b, with_flux, st);
    }
  }

  static HotOps ops() {
    HotOps o;
    o.D = D; o.M = M; o.PDE = PDE; o.V = V;
    o.weno_tile = &weno_tile;
    o.weno = &weno; o.predict = &predict; o.flux = &flux; o.update = &update; o.project = &project;
    o.flux_update = &flux_update;
    o.weno_b = &weno_b; o.predict_b = &predict_b; o.flux_b = &flux_b; o.update_b = &update_b;
    o.flux_update_b = &flux_update_b;
    o.project_b = &project_b;
    o.level_b = kLevelKernel ? &level_b : nullptr;
    return o;
  }
};

}  // namespace aw

#define AW_INSTANTIATE(D, M, P) \
  namespace aw { HotOps ops_##D##_##M##_##P() { return Launch<D, M, P>::ops(); } }
