// aw_inst.cuh -- launchers of the hot kernels for one configuration; included by aw_inst_*.cu.
#pragma once
#include <mutex>

#include "aw_hot.cuh"

namespace aw {

template <int D, int M, int PDE>
struct Launch {
  // WENO tile edge: 8x8 cells in 2D (6 sweep passes of 256 threads per 64 cells, against 2 per 16
  // with 4x4 tiles, whose x pass fills 160 of 256 lanes), 4x4x4 in 3D (shared memory)
  static constexpr int TS = (D == 2) ? 8 : 4;
  using CW = WenoCfg<D, M, PDE, TS>;
  using CP = PredCfg<D, M, PDE>;
  using CF = FluxCfg<D, M, PDE>;
  static constexpr int V = nvars(D, PDE);

  // CTAs of each kernel for one solve's level (0 when there is no work)
  static int weno_ctas(const HotArgs& a) { return a.ntiles > 0 ? a.ntiles : 0; }
  static int predict_ctas(const HotArgs& a) { return a.na > 0 ? (a.na + CP::CPB - 1) / CP::CPB : 0; }
  static int flux_ctas(const HotArgs& a) {
    if (a.na <= 0) return 0;
    long long lo = (long long)D * ((a.na + CF::CPB - 1) / CF::CPB);
    return (int)(lo + (a.nh + CF::CPB - 1) / CF::CPB);
  }
  static int update_ctas(const HotArgs& a) { return a.na > 0 ? (a.na + 127) / 128 : 0; }
  static int project_ctas(int nv) { return nv > 0 ? (int)(((long long)nv * V + 127) / 128) : 0; }

  // the dynamic shared memory attribute, once per kernel (request-loop workers launch concurrently)
  template <class K>
  static void smem_attr(K kernel, int bytes, std::once_flag& once) {
    std::call_once(once, [&] { cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
  }

  static int weno(const HotArgs& a, cudaStream_t st) {
    const int blocks = weno_ctas(a);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_weno<D, M, PDE, TS>, CW::SMEM, init);
    k_weno<D, M, PDE, TS><<<blocks, 256, CW::SMEM, st>>>(a);
    return 1;
  }
  static int predict(const HotArgs& a, cudaStream_t st) {
    const int blocks = predict_ctas(a);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_predict<D, M, PDE>, CP::SMEM, init);
    k_predict<D, M, PDE><<<blocks, CP::THREADS, CP::SMEM, st>>>(a);
    return 1;
  }
  static int flux(const HotArgs& a, cudaStream_t st) {
    const int blocks = flux_ctas(a);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_flux<D, M, PDE>, CF::SMEM, init);
    k_flux<D, M, PDE><<<blocks, CF::THREADS, CF::SMEM, st>>>(a);
    return 1;
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
  static int weno_b(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, weno_ctas);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_weno_batch<D, M, PDE, TS>, CW::SMEM, init);
    k_weno_batch<D, M, PDE, TS><<<blocks, 256, CW::SMEM, st>>>(b);
    return 1;
  }
  static int predict_b(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, predict_ctas);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_predict_batch<D, M, PDE>, CP::SMEM, init);
    k_predict_batch<D, M, PDE><<<blocks, CP::THREADS, CP::SMEM, st>>>(b);
    return 1;
  }
  static int flux_b(HotBatch& b, cudaStream_t st) {
    const int blocks = fill_starts(b, flux_ctas);
    if (!blocks) return 0;
    static std::once_flag init;
    smem_attr(k_flux_batch<D, M, PDE>, CF::SMEM, init);
    k_flux_batch<D, M, PDE><<<blocks, CF::THREADS, CF::SMEM, st>>>(b);
    return 1;
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

  static HotOps ops() {
    HotOps o;
    o.D = D; o.M = M; o.PDE = PDE; o.V = V; o.wenoTS = TS;
    o.weno = &weno; o.predict = &predict; o.flux = &flux; o.update = &update; o.project = &project;
    o.weno_b = &weno_b; o.predict_b = &predict_b; o.flux_b = &flux_b; o.update_b = &update_b;
    o.project_b = &project_b;
    return o;
  }
};

}  // namespace aw

#define AW_INSTANTIATE(D, M, P) \
  namespace aw { HotOps ops_##D##_##M##_##P() { return Launch<D, M, P>::ops(); } }
