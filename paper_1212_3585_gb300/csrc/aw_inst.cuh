// aw_inst.cuh -- launchers of the hot kernels for one configuration; included by aw_inst_*.cu.
#pragma once
#include "aw_hot.cuh"

namespace aw {

template <int D, int M, int PDE>
struct Launch {
  static constexpr int TS = 4;
  static int weno(const HotArgs& a, cudaStream_t st) {
    if (a.ntiles <= 0) return 0;
    using C = WenoCfg<D, M, PDE, TS>;
    static bool init = false;
    if (!init) {
      cudaFuncSetAttribute(k_weno<D, M, PDE, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
      init = true;
    }
    k_weno<D, M, PDE, TS><<<a.ntiles, 256, C::SMEM, st>>>(a);
    return 1;
  }
  static int predict(const HotArgs& a, cudaStream_t st) {
    if (a.na <= 0) return 0;
    using C = PredCfg<D, M, PDE>;
    static bool init = false;
    if (!init) {
      cudaFuncSetAttribute(k_predict<D, M, PDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
      init = true;
    }
    int blocks = (a.na + C::CPB - 1) / C::CPB;
    k_predict<D, M, PDE><<<blocks, C::THREADS, C::SMEM, st>>>(a);
    return 1;
  }
  static int flux(const HotArgs& a, cudaStream_t st) {
    if (a.na <= 0) return 0;
    using C = FluxCfg<D, M, PDE>;
    static bool init = false;
    if (!init) {
      cudaFuncSetAttribute(k_flux<D, M, PDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
      init = true;
    }
    long long blocks_lo = (long long)D * ((a.na + C::CPB - 1) / C::CPB);
    int blocks = (int)(blocks_lo + (a.nh + C::CPB - 1) / C::CPB);
    k_flux<D, M, PDE><<<blocks, C::THREADS, C::SMEM, st>>>(a);
    return 1;
  }
  static int update(const HotArgs& a, cudaStream_t st) {
    if (a.na <= 0) return 0;
    k_update<D, M, PDE><<<(a.na + 127) / 128, 128, 0, st>>>(a);
    return 1;
  }
  static int project(const HotArgs& a, const int32_t* vlist, int nv, const double* src, int spacetime,
                     double* out, int dense, cudaStream_t st) {
    if (nv <= 0) return 0;
    constexpr int V = nvars(D, PDE);
    long long n = (long long)nv * V;
    k_project<D, M, PDE><<<(int)((n + 127) / 128), 128, 0, st>>>(a, vlist, nv, src, spacetime, out, dense);
    return 1;
  }
  static HotOps ops() {
    HotOps o;
    o.D = D; o.M = M; o.PDE = PDE; o.V = nvars(D, PDE); o.wenoTS = TS;
    o.weno = &weno; o.predict = &predict; o.flux = &flux; o.update = &update; o.project = &project;
    return o;
  }
};

}  // namespace aw

#define AW_INSTANTIATE(D, M, P) \
  namespace aw { HotOps ops_##D##_##M##_##P() { return Launch<D, M, P>::ops(); } }
