// aw_hot.cuh -- the per-level hot kernels of the ADER-WENO update, templated on the space
// dimension D, the polynomial degree M and the PDE system.  Instantiated per configuration in
// aw_inst_*.cu.  Everything here is FP64: the scheme is bound by the FP64 pipe on sm_103a, so
// the kernels are laid out to keep every lane of every issued FP64 instruction busy (compacted
// work lists, one thread per cell x spatial node) rather than for memory traffic.
#pragma once
#include <cooperative_groups.h>

#include "aw_device.cuh"
#include "aw_ops.h"

namespace aw {

template <int M>
struct Sten {
  static constexpr int NS = (M % 2 == 0) ? 3 : 4;
  __host__ __device__ static constexpr int SL(int s) {
    return (M % 2 == 0) ? (s == 0 ? M / 2 : (s == 1 ? M : 0))
                        : (s == 0 ? M / 2 + 1 : (s == 1 ? M / 2 : (s == 2 ? M : 0)));
  }
};

// One-dimensional WENO reconstruction (Sec. 2.2, Eqs. eqn.rec.x, eqn.weno, eqn.omegas,
// eqn.sigmas): values at offsets -M..M (stride apart) -> N nodal coefficients.  The stencil
// polynomials and oscillation indicators are formed from the differences to the cell's own value
// (exact: stencils reproduce constants and Sigma annihilates them), so that the rounding of a
// large constant part does not reach sigma, whose 8th power sets the weights.
template <int M>
__device__ __forceinline__ void weno1d(const Tables& T, const double* v, int stride, double* out) {
  constexpr int N = M + 1, W = 2 * M + 1, NS = Sten<M>::NS;
  double val[W];
  const double c = v[M * stride];
#pragma unroll
  for (int e = 0; e < W; e++) val[e] = (e == M) ? 0.0 : v[e * stride] - c;
  double acc[N], sum = 0.0;
#pragma unroll
  for (int p = 0; p < N; p++) acc[p] = 0.0;
#pragma unroll
  for (int s = 0; s < NS; s++) {
    const int o = M - Sten<M>::SL(s);   // stencil cells o..o+M, the centre cell at e = SL(s)
    // the N-1 nonzero differences of this stencil
    double d[N - 1];
#pragma unroll
    for (int e = 0, k = 0; e < N; e++)
      if (e != Sten<M>::SL(s)) d[k++] = val[o + e];
    double ws[N];
#pragma unroll
    for (int p = 0; p < N; p++) {
      double t = 0.0;
#pragma unroll
      for (int e = 0, k = 0; e < N; e++)
        if (e != Sten<M>::SL(s)) t = fma(T.Ainv[s][p][e], d[k++], t);
      ws[p] = t;
    }
    // sigma + eps, the quadratic form accumulated onto eps (one addition fewer)
    double sig = 1e-14;
#pragma unroll
    for (int i = 0; i < N - 1; i++) {
      double t = T.Bq[s][i][i] * d[i];
#pragma unroll
      for (int j = i + 1; j < N - 1; j++) t = fma(T.Bq[s][i][j], d[j], t);
      sig = fma(t, d[i], sig);
    }
    // lambda_s / (sigma + eps)^8 from the reciprocal of sigma + eps (>= 1e-14)
    double y = rcp_nr1(sig), y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    double om = (s < (M % 2 == 0 ? 1 : 2)) ? 1e5 * y8 : y8;
    sum = s == 0 ? om : sum + om;
#pragma unroll
    for (int p = 0; p < N; p++) acc[p] = fma(om, ws[p], acc[p]);
  }
  // sum >= lambda_s / (sigma_s + eps)^8 of the smoothest stencil: a normal double unless every
  // sigma exceeds ~1e38 (IEEE division there)
  double is = sum >= 1e-300 ? rcp_nr1(sum) : 1.0 / sum;
#pragma unroll
  for (int p = 0; p < N; p++) out[p] = fma(acc[p], is, c);
}

// Warp 0 compacts the candidates 0..ncand-1 for which pred(c) holds into list[], count into *cnt.
template <class Pred>
__device__ __forceinline__ void warp0_compact(int ncand, Pred pred, int16_t* list, int* cnt) {
  if (threadIdx.x >= 32) return;
  int lane = threadIdx.x, base = 0;
  for (int c0 = 0; c0 < ncand; c0 += 32) {
    int c = c0 + lane;
    bool f = c < ncand && pred(c);
    unsigned b = __ballot_sync(0xffffffffu, f);
    if (f) list[base + __popc(b & ((1u << lane) - 1u))] = (int16_t)c;
    base += __popc(b);
  }
  if (lane == 0) *cnt = base;
}

// ------------------------------------------------------------------------------------------
// WENO kernel: one CTA per tile of TS^D cells of one level.  The (TS+2M)^D box of averages is
// staged in shared memory through the boundary map; x sweeps run on every box line that feeds
// an active cell of the tile, then y (and z) sweeps on the active cells only (compacted work
// lists, Eqs. eqn.weno, eqn.weno.y, eqn.weno.z).  Output: WENO dofs per active cell.  Used for
// levels below 4096 cells (by default); larger levels run the same reconstructions by passes
// (k_weno_x/y, k_weno3_x/y/z below, and their batched forms), without the halo recomputation.
// ------------------------------------------------------------------------------------------
template <int D, int M, int PDE, int TS>
struct WenoCfg {
  static constexpr int N = M + 1, V = nvars(D, PDE), B = TS + 2 * M;
  static constexpr int NB = ipow(B, D);
  static constexpr int NXS = (D == 2) ? V * B * TS * N : V * B * B * TS * N;
  static constexpr int NYS = (D == 2) ? 0 : V * B * TS * TS * N * N;
  static constexpr int SMEM = (V * NB + NXS + NYS) * 8;
  static constexpr int NC = ipow(TS, D);
  static constexpr int NXC = (D == 2) ? B * TS : B * B * TS;
  static constexpr int NYC = (D == 2) ? 0 : B * TS * TS;
};

template <int D, int M, int PDE, int TS>
__device__ __forceinline__ void weno_body(const HotArgs& a, const int bid) {
  using C = WenoCfg<D, M, PDE, TS>;
  constexpr int N = C::N, V = C::V, B = C::B, NB = C::NB, NSP = ipow(N, D);
  extern __shared__ double smem[];
  double* box = smem;
  double* xs = box + V * NB;
  double* ys = xs + C::NXS;
  __shared__ int taid[C::NC];
  __shared__ int16_t lx[C::NXC];
  __shared__ int16_t ly[(C::NYC > 0) ? C::NYC : 1];
  __shared__ int16_t lc[C::NC];
  __shared__ int nx_, ny_, nc_;
  __shared__ uint8_t needxy[(C::NYC > 0) ? C::NYC : 1];

  const LevelView& L = a.lv;
  const int tile = a.tiles[bid];
  int org[3] = {0, 0, 0};
  {
    int t = tile;
    for (int d = 0; d < D; d++) { org[d] = (t % a.tdim[d]) * TS; t /= a.tdim[d]; }
  }
  // stage the box (reflective walls: mirror image with the normal momentum negated; beyond an
  // inflow face: the inflow state)
  for (int idx = threadIdx.x; idx < NB; idx += blockDim.x) {
    int t = idx, c[3] = {0, 0, 0};
    unsigned flip = 0;
    bool inflow = false;
    for (int d = 0; d < D; d++) {
      int b = t % B;
      t /= B;
      if (reflected(L.L, a.bc, d, org[d] - M + b)) flip |= 1u << d;
      inflow |= beyond_inflow(L.L, a.bc, d, org[d] - M + b);
      bcmap(L.L, a.bc, d, org[d] - M + b, &c[d]);
    }
    if (inflow) {
#pragma unroll
      for (int v = 0; v < V; v++) box[v * NB + idx] = a.P.inflow[v];
      continue;
    }
    long long di = didx(L, c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < V; v++) {
      double x = L.u[v * L.n + di];
      if (PDE == PDE_EULER && v >= 1 && v <= D && (flip >> (v - 1) & 1u)) x = -x;
      box[v * NB + idx] = x;
    }
  }
  for (int idx = threadIdx.x; idx < C::NC; idx += blockDim.x) {
    int t = idx, c[3] = {0, 0, 0};
    bool in = true;
    for (int d = 0; d < D; d++) {
      c[d] = org[d] + t % TS;
      t /= TS;
      in &= c[d] < L.L[d];
    }
    taid[idx] = in ? L.aid[didx(L, c[0], c[1], c[2])] : -1;
  }
  __syncthreads();

  if (D == 2) {
    // x sweeps needed at box row y, tile column cx: an active cell (cx, ty) with |y - ty - M| <= M
    warp0_compact(C::NXC, [&](int c) {
      int y = c / TS, cx = c % TS;
      for (int ty = 0; ty < TS; ty++)
        if (taid[ty * TS + cx] >= 0 && abs(y - ty - M) <= M) return true;
      return false;
    }, lx, &nx_);
    warp0_compact(C::NC, [&](int c) { return taid[c] >= 0; }, lc, &nc_);
    __syncthreads();
    const int nx = nx_ * V;
    for (int it = threadIdx.x; it < nx; it += blockDim.x) {
      int pos = lx[it / V], v = it % V;
      int y = pos / TS, cx = pos % TS;
      double o[N];
      weno1d<M>(a.T, box + v * NB + y * B + cx, 1, o);
#pragma unroll
      for (int p = 0; p < N; p++) xs[((v * B + y) * TS + cx) * N + p] = o[p];
    }
    __syncthreads();
    const int nyi = nc_ * N * V;
    for (int it = threadIdx.x; it < nyi; it += blockDim.x) {
      int k = it / (N * V), rem = it % (N * V), p = rem / V, v = rem % V;
      int c = lc[k], cx = c % TS, cy = c / TS;
      double o[N];
      weno1d<M>(a.T, xs + ((v * B + cy) * TS + cx) * N + p, TS * N, o);
      double* dst = a.wh + ((long long)taid[c] * V + v) * NSP;
#pragma unroll
      for (int q = 0; q < N; q++) dst[p + N * q] = o[q];
    }
  } else {
    // z sweeps at active cells; y sweeps where an active cell within M in z needs them; x sweeps
    // where a needed y sweep within M in y needs them.
    for (int c = threadIdx.x; c < C::NYC; c += blockDim.x) {
      int z = c / (TS * TS), cy = (c / TS) % TS, cx = c % TS;
      bool f = false;
      for (int tz = 0; tz < TS; tz++)
        f |= taid[(tz * TS + cy) * TS + cx] >= 0 && abs(z - tz - M) <= M;
      needxy[c] = f;
    }
    __syncthreads();
    warp0_compact(C::NXC, [&](int c) {
      int z = c / (B * TS), y = (c / TS) % B, cx = c % TS;
      for (int cy = 0; cy < TS; cy++)
        if (needxy[(z * TS + cy) * TS + cx] && abs(y - cy - M) <= M) return true;
      return false;
    }, lx, &nx_);
    warp0_compact(C::NYC, [&](int c) { return needxy[c] != 0; }, ly, &ny_);
    warp0_compact(C::NC, [&](int c) { return taid[c] >= 0; }, lc, &nc_);
    __syncthreads();
    const int nx = nx_ * V;
    for (int it = threadIdx.x; it < nx; it += blockDim.x) {
      int pos = lx[it / V], v = it % V;
      int z = pos / (B * TS), y = (pos / TS) % B, cx = pos % TS;
      double o[N];
      weno1d<M>(a.T, box + v * NB + (z * B + y) * B + cx, 1, o);
#pragma unroll
      for (int p = 0; p < N; p++) xs[(((v * B + z) * B + y) * TS + cx) * N + p] = o[p];
    }
    __syncthreads();
    const int nyi = ny_ * N * V;
    for (int it = threadIdx.x; it < nyi; it += blockDim.x) {
      int k = it / (N * V), rem = it % (N * V), p = rem / V, v = rem % V;
      int pos = ly[k];
      int z = pos / (TS * TS), cy = (pos / TS) % TS, cx = pos % TS;
      double o[N];
      weno1d<M>(a.T, xs + (((v * B + z) * B + cy) * TS + cx) * N + p, TS * N, o);
#pragma unroll
      for (int q = 0; q < N; q++) ys[((((v * B + z) * TS + cy) * TS + cx) * N + p) * N + q] = o[q];
    }
    __syncthreads();
    const int nzi = nc_ * N * N * V;
    for (int it = threadIdx.x; it < nzi; it += blockDim.x) {
      int k = it / (N * N * V), rem = it % (N * N * V), pq = rem / V, v = rem % V;
      int p = pq % N, q = pq / N;
      int c = lc[k], cx = c % TS, cy = (c / TS) % TS, cz = c / (TS * TS);
      double o[N];
      weno1d<M>(a.T, ys + ((((v * B + cz) * TS + cy) * TS + cx) * N + p) * N + q, TS * TS * N * N, o);
      double* dst = a.wh + ((long long)taid[c] * V + v) * NSP;
#pragma unroll
      for (int r = 0; r < N; r++) dst[p + N * q + N * N * r] = o[r];
    }
  }
}

template <int D, int M, int PDE, int TS>
__global__ void __launch_bounds__(256) k_weno(const __grid_constant__ HotArgs a) {
  weno_body<D, M, PDE, TS>(a, blockIdx.x);
}

// ------------------------------------------------------------------------------------------
// 2D WENO in two passes (the same reconstructions as the tiles, Eqs. eqn.weno, eqn.weno.y):
// first the x sweep of every row that feeds an active cell, once, into a buffer that stays in
// L2; then the y sweeps of the active cells over the x sweeps of their column.  A tile instead
// recomputes the x sweeps of its 2M halo rows.  Ghost rows map exactly: periodic and
// transmissive rows are interior rows, a mirrored row's sweep is the sweep of its image with the
// normal momentum negated (WENO commutes with negation), and a row beyond an inflow face is the
// inflow state.
// ------------------------------------------------------------------------------------------
template <int M, int PDE>
__device__ __forceinline__ void weno_x_body(const HotArgs& a, const int bid) {
  constexpr int D = 2, N = M + 1, V = nvars(D, PDE), W = 2 * M + 1;
  const long long it = (long long)bid * blockDim.x + threadIdx.x;
  if (it >= (long long)a.nxs * V) return;
  const int slot = (int)(it / V), v = (int)(it % V);
  const LevelView& L = a.lv;
  const long long di = a.xlist[slot];
  const int i = (int)(di % L.L[0]), j = (int)(di / L.L[0]);
  double val[W];
#pragma unroll
  for (int e = 0; e < W; e++) {
    const int ii = i - M + e;
    if (beyond_inflow(L.L, a.bc, 0, ii)) {
      val[e] = a.P.inflow[v];
      continue;
    }
    int im = ii;
    bcmap(L.L, a.bc, 0, ii, &im);
    double x = L.u[v * L.n + didx(L, im, j, 0)];
    if (PDE == PDE_EULER && v == 1 && reflected(L.L, a.bc, 0, ii)) x = -x;
    val[e] = x;
  }
  double o[N];
  weno1d<M>(a.T, val, 1, o);
  double* dst = a.xs + ((long long)slot * V + v) * N;
#pragma unroll
  for (int p = 0; p < N; p++) dst[p] = o[p];
}

template <int M, int PDE>
__global__ void __launch_bounds__(128) k_weno_x(const __grid_constant__ HotArgs a) {
  weno_x_body<M, PDE>(a, blockIdx.x);
}

// 3D: the same by three passes -- x sweeps of the rows feeding the y sweeps, y sweeps of the
// cells feeding the z sweeps, z sweeps of the active cells -- with the same exact ghost mapping
template <int M, int PDE>
__device__ __forceinline__ void weno3_x_body(const HotArgs& a, const int bid) {
  constexpr int D = 3, N = M + 1, V = nvars(D, PDE), W = 2 * M + 1;
  const long long it = (long long)bid * blockDim.x + threadIdx.x;
  if (it >= (long long)a.nxs * V) return;
  const int slot = (int)(it / V), v = (int)(it % V);
  const LevelView& L = a.lv;
  int c[3];
  cell_ijk(L, a.xlist[slot], c);
  double val[W];
#pragma unroll
  for (int e = 0; e < W; e++) {
    const int ii = c[0] - M + e;
    if (beyond_inflow(L.L, a.bc, 0, ii)) {
      val[e] = a.P.inflow[v];
      continue;
    }
    int im = ii;
    bcmap(L.L, a.bc, 0, ii, &im);
    double x = L.u[v * L.n + didx(L, im, c[1], c[2])];
    if (PDE == PDE_EULER && v == 1 && reflected(L.L, a.bc, 0, ii)) x = -x;
    val[e] = x;
  }
  double o[N];
  weno1d<M>(a.T, val, 1, o);
  double* dst = a.xs + ((long long)slot * V + v) * N;
#pragma unroll
  for (int p = 0; p < N; p++) dst[p] = o[p];
}

template <int M, int PDE>
__global__ void __launch_bounds__(128) k_weno3_x(const __grid_constant__ HotArgs a) {
  weno3_x_body<M, PDE>(a, blockIdx.x);
}

// y sweeps: one thread per (cell of the y list, variable), looping over the x dofs p, so that
// the stencil's slots are looked up once for the N reconstructions
template <int M, int PDE>
__device__ __forceinline__ void weno3_y_body(const HotArgs& a, const int bid) {
  constexpr int D = 3, N = M + 1, V = nvars(D, PDE), W = 2 * M + 1;
  const long long it = (long long)bid * blockDim.x + threadIdx.x;
  if (it >= (long long)a.nys * V) return;
  const int ysl = (int)(it / V), v = (int)(it % V);
  const LevelView& L = a.lv;
  int c[3];
  cell_ijk(L, a.ylist[ysl], c);
  long long base[W];   // x sweeps of the stencil's cells (-1: the inflow state)
  bool neg[W];
#pragma unroll
  for (int e = 0; e < W; e++) {
    const int jj = c[1] - M + e;
    neg[e] = false;
    if (beyond_inflow(L.L, a.bc, 1, jj)) {
      base[e] = -1;
      continue;
    }
    int jm = jj;
    bcmap(L.L, a.bc, 1, jj, &jm);
    int slot = a.xslot[didx(L, c[0], jm, c[2])];
    if (slot < 0) {   // not marked: an inconsistent list (reported, read in bounds)
      atomicOr(a.err, 4);
      slot = 0;
    }
    base[e] = ((long long)slot * V + v) * N;
    neg[e] = PDE == PDE_EULER && v == 2 && reflected(L.L, a.bc, 1, jj);
  }
#pragma unroll 1
  for (int p = 0; p < N; p++) {
    double val[W];
#pragma unroll
    for (int e = 0; e < W; e++) {
      double x = base[e] < 0 ? a.P.inflow[v] : a.xs[base[e] + p];
      val[e] = neg[e] ? -x : x;
    }
    double o[N];
    weno1d<M>(a.T, val, 1, o);
    double* dst = a.ys + (((long long)ysl * V + v) * N + p) * N;
#pragma unroll
    for (int q = 0; q < N; q++) dst[q] = o[q];
  }
}

template <int M, int PDE>
__global__ void __launch_bounds__(128) k_weno3_y(const __grid_constant__ HotArgs a) {
  weno3_y_body<M, PDE>(a, blockIdx.x);
}

// z sweeps: one thread per (active cell, x dof p, variable), looping over the y dofs q, so that
// the stencil's slots are looked up once for the N reconstructions
template <int M, int PDE>
__device__ __forceinline__ void weno3_z_body(const HotArgs& a, const int bid) {
  constexpr int D = 3, N = M + 1, V = nvars(D, PDE), W = 2 * M + 1, NSP = N * N * N;
  const long long it = (long long)bid * blockDim.x + threadIdx.x;
  if (it >= (long long)a.na * N * V) return;
  const int k = (int)(it / (N * V)), rem = (int)(it % (N * V)), p = rem / V, v = rem % V;
  const LevelView& L = a.lv;
  int c[3];
  cell_ijk(L, a.alist[k], c);
  long long base[W];   // y sweeps of the stencil's cells (-1: the inflow state)
  bool neg[W];
#pragma unroll
  for (int e = 0; e < W; e++) {
    const int kk = c[2] - M + e;
    neg[e] = false;
    if (beyond_inflow(L.L, a.bc, 2, kk)) {
      base[e] = -1;
      continue;
    }
    int km = kk;
    bcmap(L.L, a.bc, 2, kk, &km);
    int slot = a.yslot[didx(L, c[0], c[1], km)];
    if (slot < 0) {
      atomicOr(a.err, 4);
      slot = 0;
    }
    base[e] = (((long long)slot * V + v) * N + p) * N;
    neg[e] = PDE == PDE_EULER && v == 3 && reflected(L.L, a.bc, 2, kk);
  }
  double* dst = a.wh + ((long long)k * V + v) * NSP;
#pragma unroll 1
  for (int q = 0; q < N; q++) {
    double val[W];
#pragma unroll
    for (int e = 0; e < W; e++) {
      double x = base[e] < 0 ? a.P.inflow[v] : a.ys[base[e] + q];
      val[e] = neg[e] ? -x : x;
    }
    double o[N];
    weno1d<M>(a.T, val, 1, o);
#pragma unroll
    for (int r = 0; r < N; r++) dst[p + N * q + N * N * r] = o[r];
  }
}

template <int M, int PDE>
__global__ void __launch_bounds__(128) k_weno3_z(const __grid_constant__ HotArgs a) {
  weno3_z_body<M, PDE>(a, blockIdx.x);
}

template <int M, int PDE>
__device__ __forceinline__ void weno_y_body(const HotArgs& a, const int bid) {
  constexpr int D = 2, N = M + 1, V = nvars(D, PDE), W = 2 * M + 1, NSP = N * N;
  const long long it = (long long)bid * blockDim.x + threadIdx.x;
  if (it >= (long long)a.na * N * V) return;
  const int k = (int)(it / (N * V)), rem = (int)(it % (N * V)), p = rem / V, v = rem % V;
  const LevelView& L = a.lv;
  const long long di = a.alist[k];
  const int i = (int)(di % L.L[0]), j = (int)(di / L.L[0]);
  double val[W];
#pragma unroll
  for (int e = 0; e < W; e++) {
    const int jj = j - M + e;
    if (beyond_inflow(L.L, a.bc, 1, jj)) {
      val[e] = a.P.inflow[v];
      continue;
    }
    int jm = jj;
    bcmap(L.L, a.bc, 1, jj, &jm);
    int slot = a.xslot[didx(L, i, jm, 0)];
    if (slot < 0) {   // not marked: an inconsistent list (reported, read in bounds)
      atomicOr(a.err, 4);
      slot = 0;
    }
    double x = a.xs[((long long)slot * V + v) * N + p];
    if (PDE == PDE_EULER && v == 2 && reflected(L.L, a.bc, 1, jj)) x = -x;
    val[e] = x;
  }
  double o[N];
  weno1d<M>(a.T, val, 1, o);
  double* dst = a.wh + ((long long)k * V + v) * NSP;
#pragma unroll
  for (int q = 0; q < N; q++) dst[p + N * q] = o[q];
}

template <int M, int PDE>
__global__ void __launch_bounds__(128) k_weno_y(const __grid_constant__ HotArgs a) {
  weno_y_body<M, PDE>(a, blockIdx.x);
}

// ------------------------------------------------------------------------------------------
// Predictor kernel (Sec. 2.3, Eq. eqn.stdg.final).  One thread per (active cell, spatial node);
// the thread holds the time column of q_h at its node for all variables.  With the nodal
// tensor basis the Picard step reads
//     q(node, s) = w(node) - sum_s' G[s][s'] R(node, s'),
//     R(node, s') = sum_d (dt/dx_d) sum_k Dm[i_d][k] f_d(q(node with i_d = k, s')),
// where G = K_t^{-1} diag(w) is the inverted time block of K1 and K_t^{-1} psi(0) = 1.  The
// spatial derivative contractions read the neighbouring nodes' fluxes from shared memory.
// The first iteration starts from q = w, constant in time, so it needs one flux evaluation per
// node and R is constant in time.
// ------------------------------------------------------------------------------------------
// DIV > 1: a CTA of CPB / DIV cells, for levels too small to give every SM work otherwise
template <int D, int M, int PDE, int DIV = 1>
struct PredCfg {
  static constexpr int N = M + 1, NSP = ipow(N, D), NST = NSP * N, V = nvars(D, PDE);
  // cells per CTA: 256 threads where the fluxes of all nodes (D V N^(d+1) doubles per cell) leave
  // room for two CTAs per SM; halved where one CTA would fill the shared memory (MHD); 3D Euler
  // M=2: 7 cells (189 threads, 68 KB), so that three CTAs fit an SM's shared memory (8 cells,
  // 77.8 KB, fit two)
  static constexpr int CPB1 = (NSP == 4) ? 64 : (NSP == 9) ? 32 : (NSP == 16 ? 16 : (NSP == 27 ? 14 : 4));
  static constexpr int CPB0 = (CPB1 * D * V * NST * 8 > 113 * 1024 && CPB1 > 1) ? CPB1 / 2 : CPB1;
  static constexpr int CPB = DIV == 1 ? CPB0 : warp_fill_units(CPB0 / DIV > 0 ? CPB0 / DIV : 1, NSP);
  static constexpr int THREADS = CPB * NSP;
  static constexpr int SMEM = CPB * D * V * NST * 8;   // fluxes at every space-time node
};

template <int D, int M, int PDE, int DIV = 1>
__device__ __forceinline__ void predict_body(const HotArgs& a, const int bid) {
  using C = PredCfg<D, M, PDE, DIV>;
  using Q = Pde<PDE, D>;
  constexpr int N = C::N, NSP = C::NSP, NST = C::NST, V = C::V;
  extern __shared__ double sh[];  // [CPB][D][V][NST]
  const int lc = threadIdx.x / NSP, node = threadIdx.x % NSP;
  const int cell = bid * C::CPB + lc;
  const bool ok = cell < a.na;
  int ix[D];
  {
    int t = node;
#pragma unroll
    for (int d = 0; d < D; d++) { ix[d] = t % N; t /= N; }
  }
  const double dt = a.dtl[a.level];
  double Dr[D][N];
#pragma unroll
  for (int d = 0; d < D; d++) {
    double lam = dt / a.lv.dx[d];
#pragma unroll
    for (int k = 0; k < N; k++) Dr[d][k] = lam * a.T.Dm[ix[d]][k];
  }
  double w[V];
  const double* wsrc = a.wh + (long long)(ok ? cell : 0) * V * NSP;
#pragma unroll
  for (int v = 0; v < V; v++) w[v] = wsrc[v * NSP + node];
  double* shc = sh + lc * D * V * NST;
  double q[V][N], R[V][N];
  // first Picard iteration from q = w, constant in time: one flux evaluation per node
  {
    double F[D][V];
    Q::fluxes(w, F, a.P);
#pragma unroll
    for (int d = 0; d < D; d++)
#pragma unroll
      for (int v = 0; v < V; v++) shc[(d * V + v) * NST + node] = F[d][v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V; v++) {
      double r = 0.0;
#pragma unroll
      for (int d = 0; d < D; d++) {
        const int st = (d == 0 ? 1 : (d == 1 ? N : N * N));
        const int base = node - ix[d] * st;
#pragma unroll
        for (int k = 0; k < N; k++) r = fma(Dr[d][k], shc[(d * V + v) * NST + base + k * st], r);
      }
#pragma unroll
      for (int s = 0; s < N; s++) q[v][s] = fma(-a.T.gsum[s], r, w[v]);
    }
    __syncthreads();
  }
  for (int it = 1; it < a.picard; it++) {
    // fluxes at all N time nodes of this thread's spatial node
#pragma unroll
    for (int s = 0; s < N; s++) {
      double qs[V], F[D][V];
#pragma unroll
      for (int v = 0; v < V; v++) qs[v] = q[v][s];
      Q::fluxes(qs, F, a.P);
#pragma unroll
      for (int d = 0; d < D; d++)
#pragma unroll
        for (int v = 0; v < V; v++) shc[(d * V + v) * NST + node + NSP * s] = F[d][v];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < N; s++)
#pragma unroll
      for (int v = 0; v < V; v++) {
        double r = 0.0;
#pragma unroll
        for (int d = 0; d < D; d++) {
          const int st = (d == 0 ? 1 : (d == 1 ? N : N * N));
          const int base = node - ix[d] * st + NSP * s;
#pragma unroll
          for (int k = 0; k < N; k++) r = fma(Dr[d][k], shc[(d * V + v) * NST + base + k * st], r);
        }
        R[v][s] = r;
      }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
      for (int s = 0; s < N; s++) {
        double t = w[v];
#pragma unroll
        for (int s2 = 0; s2 < N; s2++) t = fma(-a.T.G[s][s2], R[v][s2], t);
        q[v][s] = t;
      }
  }
  if (ok) {
    double* dst = a.qh + (long long)cell * V * NST;
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
      for (int s = 0; s < N; s++) dst[v * NST + node + NSP * s] = q[v][s];
  }
}

template <int D, int M, int PDE, int DIV>
__global__ void __launch_bounds__(PredCfg<D, M, PDE, DIV>::THREADS) k_predict(const __grid_constant__ HotArgs a) {
  predict_body<D, M, PDE, DIV>(a, blockIdx.x);
}

// Face flux configuration: CPB face items per CTA (a chunk of CPB active cells for the low faces),
// one thread per (face item, spatial quadrature point of the face), each thread looping over the
// N time nodes; CPB is a multiple of 32, so every warp is full (reduced CTAs: nearly full).
template <int D, int M, int PDE, int DIV = 1>
struct FluxCfg {
  static constexpr int N = M + 1, NF = ipow(N, D - 1), V = nvars(D, PDE);
  // threads of a full-size CTA: the predictor's CTA size where a whole number of warps of face
  // items fills it (so that the persistent level kernel k_level_batch runs both bodies in one CTA
  // shape), else about 256 (128 for the 9 MHD-GLM variables)
  static constexpr int PT = PredCfg<D, M, PDE, 1>::THREADS;
  static constexpr int TARGET = PT % (32 * NF) == 0 ? PT : (PDE == PDE_MHD ? 128 : 256);
  static constexpr int FULL = 32 * (TARGET / (32 * NF) > 0 ? TARGET / (32 * NF) : 1);
  // face items per CTA (reduced CTAs: about FULL / DIV items, filling their warps)
  static constexpr int CPB = DIV == 1 ? FULL : warp_fill_units(FULL / DIV > 0 ? FULL / DIV : 1, NF);
  static constexpr int THREADS = CPB * NF;
  // CTAs per SM the register allocation must allow (at least 16 warps per SM)
  static constexpr int MINB = (THREADS <= 288 / DIV) ? 3 : 2;
  // shared memory per thread: the coarse mother's polynomial contracted along the normal (V*N per
  // thread, V*N*NF per item; fine sides of coarse/fine faces), later this thread's share of the
  // face integral (V), and the mother's values at its face point and the N time nodes (V*N)
  static constexpr int SMEM = THREADS * V * 2 * N * 8;
};

enum { FK_SAME = 0, FK_FINE = 1, FK_COARSE = 2, FK_BOUNDARY = 3, FK_SKIP = 4 };

// per-item data of a flux CTA, shared by its threads
template <int CPB>
struct FluxShm {
  int kind[CPB];
  int item[3 * CPB];   // cell, axis, side
  int nb[3 * CPB];     // the neighbour across the face (through the boundary conditions)
  int nbaid[CPB];      // its active id when it is an active cell of this level (FK_SAME), else -1
};

// N-term trace of a nodal polynomial along the normal: sum_k p[k] q[k * STR]
template <int N, int STR>
__device__ __forceinline__ double trace_n(const double* p, const double* q) {
  double t = p[0] * q[0];
#pragma unroll
  for (int k = 1; k < N; k++) t = fma(p[k], q[k * STR], t);
  return t;
}

// Euler Rusanov flux times two (Eq. eqn.rusanov without its factor 1/2, which the caller folds
// into the quadrature weight): F(q-) + F(q+) - s_max (q+ - q-)
template <int D>
__device__ __forceinline__ void rusanov_euler_x2(const double* qm, const double* qp, int n, double* out,
                                                 const Phys& P) {
  constexpr int V = D + 2;
  double fm[V], fp[V];
  const double sm = euler_flux_speed<D>(qm, n, fm, P), sp = euler_flux_speed<D>(qp, n, fp, P);
  const double s = sm > sp ? sm : sp;
#pragma unroll
  for (int v = 0; v < V; v++) out[v] = fma(-s, qp[v] - qm[v], fm[v] + fp[v]);
}

// The kind of a face (axis d, side) of an active cell, the neighbour across it (through the
// boundary conditions), that neighbour's active id when it is an active cell of this level, and,
// on the fine side of a coarse/fine face, the active id of the virtual neighbour's coarse mother.
template <int D>
__device__ __forceinline__ int face_kind(const HotArgs& a, bool ok, const int* ijk, int d, int side, int* nb,
                                         int* aidb, int* maid) {
  const LevelView& L = a.lv;
  nb[0] = ijk[0]; nb[1] = ijk[1]; nb[2] = ijk[2];
  *aidb = -1;
  *maid = -1;
  if (!ok) return FK_SKIP;
  int o;
  const int c = (d == 0 ? ijk[0] : (d == 1 ? ijk[1] : ijk[2])) + (side ? 1 : -1);
  const bool inside = bcmap(L.L, a.bc, d, c, &o);
  if (d == 0) nb[0] = o;
  else if (d == 1) nb[1] = o;
  else nb[2] = o;
  if (!inside) return FK_BOUNDARY;
  const long long nbd = didx(L, nb[0], nb[1], nb[2]);
  const int8_t sn = L.st[nbd];
  if (sn == 0) {
    if (side) return FK_SKIP;
    *aidb = L.aid[nbd];
    return FK_SAME;
  }
  if (sn != 1) return FK_COARSE;
  const LevelView& Lm = a.lvm;
  const int r = a.T.r;
  *maid = Lm.aid[didx(Lm, nb[0] / r, nb[1] / r, D == 3 ? nb[2] / r : 0)];
  return FK_FINE;
}

// Fine side of a coarse/fine face, first stage: the coarse mother's space-time polynomial
// contracted along the normal at its face toward this cell.  Thread g of the item takes the
// transverse basis index g: R[(v*N + lt)*NF + g] for every variable v and time basis lt.
template <int D, int M, int PDE, int d>
__device__ __forceinline__ void fine_normal(const HotArgs& a, int side, const double* qC, int g, double* R) {
  constexpr int N = M + 1, V = nvars(D, PDE), NSP = ipow(N, D), NST = NSP * N, NF = ipow(N, D - 1);
  const double* pm = side ? a.T.psi0 : a.T.psi1;
  int off = 0;
  {
    int t = g;
#pragma unroll
    for (int b = 0; b < D; b++) {
      if (b == d) continue;
      off += (t % N) * ipow(N, b);
      t /= N;
    }
  }
#pragma unroll 1
  for (int v = 0; v < V; v++)
#pragma unroll
    for (int lt = 0; lt < N; lt++) R[(v * N + lt) * NF + g] = trace_n<N, ipow(N, d)>(pm, qC + v * NST + off + lt * NSP);
}

// second stage: at this thread's face point (transverse nodes of face point g of the fine cell,
// mapped into the mother by the child offsets) and every time node of the sub-step,
// qf[v*N + s], from the item's normal contractions R.
template <int D, int M, int PDE, int d>
__device__ __forceinline__ void fine_transverse(const HotArgs& a, const int* ijk, int g, const double* R, double* qf) {
  constexpr int N = M + 1, V = nvars(D, PDE), NF = ipow(N, D - 1);
  const int r = a.T.r;
  int jt[3] = {0, 0, 0}, ch[3] = {0, 0, 0};
  {
    int t = g;
#pragma unroll
    for (int b = 0; b < D; b++) {
      if (b == d) continue;
      jt[b] = t % N;
      t /= N;
      ch[b] = ijk[b] % r;   // transverse axes: the fine cell and its virtual neighbour share the mother's slab
    }
  }
  double qsp[V][N];
#pragma unroll
  for (int v = 0; v < V; v++)
#pragma unroll
    for (int lt = 0; lt < N; lt++) qsp[v][lt] = 0.0;
#pragma unroll
  for (int tg = 0; tg < NF; tg++) {
    int t = tg;
    double th = 1.0;
#pragma unroll
    for (int b = 0; b < D; b++) {
      if (b == d) continue;
      th *= a.T.Pf[ch[b]][jt[b]][t % N];
      t /= N;
    }
#pragma unroll
    for (int v = 0; v < V; v++)
#pragma unroll
      for (int lt = 0; lt < N; lt++) qsp[v][lt] = fma(th, R[(v * N + lt) * NF + tg], qsp[v][lt]);
  }
#pragma unroll
  for (int v = 0; v < V; v++)
#pragma unroll
    for (int s = 0; s < N; s++) {
      const double* bt = a.T.Pf[a.sub][s];
      double t = bt[0] * qsp[v][0];
#pragma unroll
      for (int lt = 1; lt < N; lt++) t = fma(bt[lt], qsp[v][lt], t);
      qf[v * N + s] = t;
    }
}

// One face (axis d, side) of an active cell at spatial face point g: this thread's share of the
// face integral, summed over the N time nodes into acc (quadrature weights included).  qf holds
// the virtual neighbour's values on the fine side of a coarse/fine face.  FL: the numerical flux
// (0 Rusanov, 1 Osher-Solomon; Euler and MHD-GLM), a template parameter so that the Rusanov
// kernels do not carry the Osher flux's registers.
template <int D, int M, int PDE, int d, int FL>
__device__ __forceinline__ void flux_face(const HotArgs& a, int kind, const double* qA, const double* qB,
                                          const double* qf, int g, int side, double* acc) {
  constexpr int N = M + 1, V = nvars(D, PDE), NSP = ipow(N, D), NST = NSP * N;
  constexpr int dstr = ipow(N, d);
  int sbase = 0;
  double ws = 1.0;
  {
    int t = g;
#pragma unroll
    for (int b = 0; b < D; b++) {
      if (b == d) continue;
      const int j = t % N;
      t /= N;
      sbase += j * ipow(N, b);
      ws *= a.T.w[j];
    }
  }
#pragma unroll
  for (int v = 0; v < V; v++) acc[v] = 0.0;
  if (kind != FK_SAME && kind != FK_FINE && kind != FK_BOUNDARY) return;
  const double* pa = side ? a.T.psi1 : a.T.psi0;
  const double* pb = side ? a.T.psi0 : a.T.psi1;
  const int bck = kind == FK_BOUNDARY ? a.bc[2 * d + side] : -1;
  // a transmissive boundary face takes the flux of the trace itself
  const bool plain = kind == FK_BOUNDARY && bck != BC_INFLOW && bck != BC_REFLECTIVE;
  const bool x2 = PDE == PDE_EULER && FL == 0 && !plain;   // rusanov_euler_x2
  const double wsp = x2 ? 0.5 * ws : ws;
#pragma unroll 1
  for (int s = 0; s < N; s++) {
    const int nbase = sbase + NSP * s;
    double qa[V], ql[V], qr[V], f[V];
#pragma unroll
    for (int v = 0; v < V; v++) qa[v] = trace_n<N, dstr>(pa, qA + v * NST + nbase);
#pragma unroll
    for (int v = 0; v < V; v++) {
      double qo;   // the state across the face
      if (kind == FK_SAME) qo = trace_n<N, dstr>(pb, qB + v * NST + nbase);
      else if (kind == FK_FINE) qo = qf[v * N + s];
      else if (bck == BC_INFLOW) qo = a.P.inflow[v];
      else if (bck == BC_REFLECTIVE && PDE == PDE_EULER && v == 1 + d) qo = -qa[v];
      else qo = qa[v];
      ql[v] = side ? qa[v] : qo;
      qr[v] = side ? qo : qa[v];
    }
    if (plain) {
      Pde<PDE, D>::flux(qa, d, f, a.P);
    } else if constexpr (PDE == PDE_EULER && FL == 1) {
      osher_euler<D>(ql, qr, d, f, a.P);
    } else if constexpr (PDE == PDE_MHD && FL == 1) {
      osher_mhd<D>(ql, qr, d, f, a.P);
    } else if constexpr (PDE == PDE_EULER) {
      rusanov_euler_x2<D>(ql, qr, d, f, a.P);
    } else {
      rusanov<PDE, D>(ql, qr, d, f, a.P);
    }
    const double wgt = wsp * a.T.w[s];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = fma(wgt, f[v], acc[v]);
  }
}

// reduce the face points' shares of every (face item, variable) of the CTA and finish the face
template <int D, int M, int PDE, int DIV>
__device__ __forceinline__ void flux_finish(const HotArgs& a, const double* sh,
                                            const FluxShm<FluxCfg<D, M, PDE, DIV>::CPB>& fs) {
  using C = FluxCfg<D, M, PDE, DIV>;
  constexpr int NF = C::NF, V = C::V, CPB = C::CPB;
  const LevelView& L = a.lv;
  for (int t = threadIdx.x; t < CPB * V; t += C::THREADS) {
    const int li = t / V, v = t - (t / V) * V;
    const int kind = fs.kind[li];
    if (kind == FK_SKIP) continue;
    const int cell = fs.item[3 * li], d = fs.item[3 * li + 1], side = fs.item[3 * li + 2];
    const double dt = a.dtl[a.level];
    double area = 1.0;
#pragma unroll
    for (int b = 0; b < D; b++)
      if (b != d) area *= L.dx[b];
    double F;
    if (kind == FK_COARSE) {
      // fine cells of the refined neighbour that touch this face; their memory slot faces this cell
      const LevelView& Lc = a.lvc;
      const int r = a.T.r;
      int ci[3];
      cell_ijk(L, a.alist[cell], ci);
      const int* nb = fs.nb + 3 * li;
      const int t0 = d == 0 ? 1 : 0;
      const int t1 = d == 2 ? 1 : 2;
      double acc = 0.0;
      const int nr2 = (D == 3) ? r : 1;
      for (int c1 = 0; c1 < nr2; c1++)
        for (int c0 = 0; c0 < r; c0++) {
          // fine cell (axis by axis, so that nothing is indexed at run time): across the face on
          // axis d, offsets c0, c1 on the transverse axes t0, t1
          int fc[3];
#pragma unroll
          for (int b = 0; b < 3; b++)
            fc[b] = b == d ? (side ? r * nb[b] : r * nb[b] + r - 1)
                           : (b == t0 ? r * ci[b] + c0 : ((D == 3 && b == t1) ? r * ci[b] + c1 : 0));
          const int fa = Lc.aid[didx(Lc, fc[0], fc[1], fc[2])];
          if (fa < 0) { atomicOr(a.err, 2); continue; }
          double* m = a.memc + ((long long)fa * 2 * D + 2 * d + (1 - side)) * V + v;
          acc += *m;
          *m = 0.0;
        }
      F = acc / (dt * area);
    } else {
      double acc = 0.0;
      const double* src = sh + (li * NF) * V + v;
#pragma unroll
      for (int g = 0; g < NF; g++) acc += src[g * V];
      F = acc;
    }
    a.fl[((long long)cell * 2 * D + 2 * d + side) * V + v] = F;
    // a low face between two active cells of this level is also the -d neighbour's high face: a
    // copy in its high slot, so that the update reads only its own cell's 2*D slots
    if (kind == FK_SAME) a.fl[((long long)fs.nbaid[li] * 2 * D + 2 * d + 1) * V + v] = F;
    if (kind == FK_FINE) a.mem[((long long)cell * 2 * D + 2 * d + side) * V + v] += F * dt * area;
  }
}

// ------------------------------------------------------------------------------------------
// Face flux kernel (Eqs. flux:F..flux:H, eqn.rusanov, eqn.osher, eqn.memory.sum).  Work items are
// faces: the listed high faces whose neighbour is not an active cell of this level (boundary,
// coarse or fine neighbour), then the low face of every active cell on every axis (by chunks of
// CPB cells, the axes of a chunk in turn).  One thread per (face, spatial quadrature point), looping
// over the N time nodes; the N^(d-1) x N space-time Gauss points of a face coincide with the
// nodal points, so a trace is one N-term contraction along the normal.  Faces toward a virtual
// child are fine sides of a coarse/fine face: the coarse predictor is evaluated at this cell's
// points and sub-step (contracted along the normal by the item's threads together, then across
// the face by each thread for its point), and the face integral is added to this cell's memory
// variable.  Faces toward a virtual mother are coarse sides: the flux is the sum of the fine
// cells' memory variables over the r sub-steps, normalised by dt * area of this level.
// ------------------------------------------------------------------------------------------
template <int D, int M, int PDE, int DIV, int FL>
__device__ __forceinline__ void flux_body(const HotArgs& a, const int bid,
                                          FluxShm<FluxCfg<D, M, PDE, DIV>::CPB>& fs) {
  using C = FluxCfg<D, M, PDE, DIV>;
  constexpr int N = M + 1, NF = C::NF, V = C::V, CPB = C::CPB;
  constexpr int NST = ipow(N, D + 1);
  extern __shared__ double sh[];
  const int li = threadIdx.x / NF, g = threadIdx.x - (threadIdx.x / NF) * NF;
  // The first CTAs take the listed high faces (item e = d * na + cell), the others the low faces:
  // chunk c of CPB active cells, the chunks from the last to the first, axis d = CTA mod D, so the
  // D passes over a chunk run back to back and share its predictor data in L2 (and, in the fused
  // kernel, the faces a chunk needs from later chunks are mostly done when its own are).
  const long long nchunk = (a.na + CPB - 1) / CPB;
  const long long nhb = (a.nh + CPB - 1) / CPB;
  bool ok;
  int cell = 0, d = 0, side = 0;
  if (bid >= nhb) {
    const long long q = bid - nhb;
    const long long chunk = nchunk - 1 - q / D;
    d = (int)(q - (q / D) * D);
    const long long c = chunk * CPB + li;
    ok = c < a.na;
    cell = ok ? (int)c : 0;
  } else {
    const long long h = bid * CPB + li;
    ok = h < a.nh;
    if (ok) {
      const long long e = a.hflist[h];
      d = (int)(e / a.na);
      cell = (int)(e - (long long)d * a.na);
      side = 1;
    }
  }
  const LevelView& L = a.lv;
  int ijk[3] = {0, 0, 0};
  if (ok) cell_ijk(L, a.alist[cell], ijk);
  int nb[3], aidb, maid;
  const int kind = face_kind<D>(a, ok, ijk, d, side, nb, &aidb, &maid);
  double* R = sh + li * NF * V * N;
  double* qf = sh + C::THREADS * V * N + threadIdx.x * V * N;
  if (__syncthreads_or(kind == FK_FINE)) {
    // fine sides of coarse/fine faces: the virtual neighbour's values from its coarse mother
    const double* qC = a.qhm + (long long)(maid < 0 ? 0 : maid) * V * NST;
    if (kind == FK_FINE) {
      if (d == 0) fine_normal<D, M, PDE, 0>(a, side, qC, g, R);
      else if (D == 2 || d == 1) fine_normal<D, M, PDE, 1>(a, side, qC, g, R);
      else fine_normal<D, M, PDE, (D == 3 ? 2 : 1)>(a, side, qC, g, R);
    }
    __syncthreads();
    if (kind == FK_FINE) {
      if (d == 0) fine_transverse<D, M, PDE, 0>(a, ijk, g, R, qf);
      else if (D == 2 || d == 1) fine_transverse<D, M, PDE, 1>(a, ijk, g, R, qf);
      else fine_transverse<D, M, PDE, (D == 3 ? 2 : 1)>(a, ijk, g, R, qf);
    }
    __syncthreads();   // R is read no more: its space takes the face points' shares below
  }
  const double* qA = a.qh + (long long)cell * V * NST;
  const double* qB = a.qh + (long long)(aidb < 0 ? 0 : aidb) * V * NST;
  double acc[V];
  if (d == 0) flux_face<D, M, PDE, 0, FL>(a, kind, qA, qB, qf, g, side, acc);
  else if (D == 2 || d == 1) flux_face<D, M, PDE, 1, FL>(a, kind, qA, qB, qf, g, side, acc);
  else flux_face<D, M, PDE, (D == 3 ? 2 : 1), FL>(a, kind, qA, qB, qf, g, side, acc);
#pragma unroll
  for (int v = 0; v < V; v++) sh[threadIdx.x * V + v] = acc[v];
  if (g == 0) {
    fs.kind[li] = kind;
    fs.nb[3 * li] = nb[0]; fs.nb[3 * li + 1] = nb[1]; fs.nb[3 * li + 2] = nb[2];
    fs.item[3 * li] = cell; fs.item[3 * li + 1] = d; fs.item[3 * li + 2] = side;
    fs.nbaid[li] = aidb;
  }
  __syncthreads();
  flux_finish<D, M, PDE, DIV>(a, sh, fs);
}

template <int D, int M, int PDE, int DIV, int FL>
__global__ void __launch_bounds__(FluxCfg<D, M, PDE, DIV>::THREADS, FluxCfg<D, M, PDE, DIV>::MINB) k_flux(const __grid_constant__ HotArgs a) {
  __shared__ FluxShm<FluxCfg<D, M, PDE, DIV>::CPB> fs;
  flux_body<D, M, PDE, DIV, FL>(a, blockIdx.x, fs);
}

// Eq. eq:finite_vol (source zero) for active cell `cell`: u -= dt/dx_d (F_high - F_low) per axis.
// The high face of every axis is in the cell's own high slot (the flux kernel copies a +d
// neighbour's low face there), so the cell reads only its 2*D contiguous slots.
template <int D, int M, int PDE>
__device__ __forceinline__ void update_cell(const HotArgs& a, int cell, double dt) {
  constexpr int V = nvars(D, PDE);
  const LevelView& L = a.lv;
  const long long di = a.alist[cell];
  const double* fc = a.fl + (long long)cell * 2 * D * V;
  double u[V];
#pragma unroll
  for (int v = 0; v < V; v++) u[v] = L.u[v * L.n + di];
#pragma unroll
  for (int d = 0; d < D; d++) {
    const double c = dt / L.dx[d];
#pragma unroll
    for (int v = 0; v < V; v++) {
      const double* lo = fc + 2 * d * V + v;
      const double fhi = lo[V], flo = lo[0];
      u[v] -= c * (fhi - flo);
    }
  }
#pragma unroll
  for (int v = 0; v < V; v++) L.u[v * L.n + di] = u[v];
  if (!Pde<PDE, D>::physical(u, a.P)) atomicOr(a.err, 1);
}

// ------------------------------------------------------------------------------------------
// Fused face flux and update (Eq. eq:finite_vol with Eqs. eqn.rusanov / eqn.osher /
// eqn.memory.sum), without any wait.  The CTAs of k_flux; chunk c holds the active cells
// c*CPB .. c*CPB+CPB-1.  Each of a chunk's cells needs 2*D face fluxes (a low and a high face per
// axis), and every face item a CTA finishes is an arrival at the chunks that read it: a low face
// at its own cell's chunk, and, when the -d neighbour is an active cell of this level, at that
// neighbour's chunk too (it is the neighbour's high face); a listed high face at its cell's
// chunk.  So every cell receives exactly 2*D arrivals.  A CTA publishes its fluxes, then adds its
// arrivals to the per-chunk counters; the CTA whose addition brings a chunk's counter to 2*D times
// its cells applies the one-step update to that chunk.  The update does the arithmetic of
// k_update in the same order, so the averages are bitwise those of the two-kernel path.  The CTA
// that completes a chunk also sets its counter back to zero, so the counters are zero at the start
// of every launch without a memset (they are zeroed when allocated and at every list rebuild).
// ------------------------------------------------------------------------------------------
template <int D, int M, int PDE, int DIV, int FL>
__device__ __forceinline__ void flux_update_body(const HotArgs& a, const int bid,
                                                 FluxShm<FluxCfg<D, M, PDE, DIV>::CPB>& fs) {
  using C = FluxCfg<D, M, PDE, DIV>;
  constexpr int V = C::V, CPB = C::CPB;
  flux_body<D, M, PDE, DIV, FL>(a, bid, fs);
  __shared__ int s_nfull;
  __shared__ int s_full[CPB + 1];   // chunks this CTA completed
  const int t = threadIdx.x;
  if (t == 0) s_nfull = 0;
  // publish this CTA's fluxes before any arrival is counted
  if (t < CPB * V) __threadfence();
  __syncthreads();
  const long long nhb = (a.nh + CPB - 1) / CPB;
  auto arrive = [&](int chunk, int n) {
    const int cells = min(CPB, a.na - chunk * CPB);
    if (atomicAdd(a.fsync + chunk, n) + n == 2 * D * cells) {
      __threadfence();
      a.fsync[chunk] = 0;   // complete: no other arrival comes; the counter is ready for the next launch
      s_full[atomicAdd(&s_nfull, 1)] = chunk;
    }
  };
  if (t < CPB) {
    if (bid >= nhb) {
      // low faces: the chunk's own cells, and the -d neighbours that are active cells of this level
      const int chunk = (int)((a.na + CPB - 1) / CPB - 1 - (bid - nhb) / D);
      if (t == 0) arrive(chunk, min(CPB, a.na - chunk * CPB));
      if (chunk * CPB + t < a.na && fs.nbaid[t] >= 0) arrive(fs.nbaid[t] / CPB, 1);
    } else {
      const long long h = bid * CPB + t;
      if (h < a.nh) arrive(fs.item[3 * t] / CPB, 1);
    }
  }
  __syncthreads();
  const int nfull = s_nfull;
  if (nfull == 0) return;
  const double dt = a.dtl[a.level];
  if (dt == 0.0) return;   // a step of length zero leaves the averages as they are
  // Eq. eq:finite_vol for the cells of the completed chunks, one thread per (cell, variable) with
  // the arithmetic of update_cell (the fluxes come from L2: other CTAs wrote them); then one
  // thread per cell checks the new state
  __shared__ double s_u[CPB * V];
  const LevelView& L = a.lv;
  for (int j = 0; j < nfull; j++) {
    const int c0 = s_full[j] * CPB, ncell = min(CPB, a.na - c0);
    for (int k = t; k < ncell * V; k += C::THREADS) {
      const int lc = k / V, v = k - lc * V, cell = c0 + lc;
      const long long di = a.alist[cell];
      const double* fc = a.fl + (long long)cell * 2 * D * V + v;
      double u = L.u[v * L.n + di];
#pragma unroll
      for (int d = 0; d < D; d++) {
        const double c = dt / L.dx[d];
        const double fhi = __ldcg(fc + 2 * d * V + V), flo = __ldcg(fc + 2 * d * V);
        u -= c * (fhi - flo);
      }
      L.u[v * L.n + di] = u;
      s_u[k] = u;
    }
    __syncthreads();
    if (t < ncell) {
      double u[V];
#pragma unroll
      for (int v = 0; v < V; v++) u[v] = s_u[t * V + v];
      if (!Pde<PDE, D>::physical(u, a.P)) atomicOr(a.err, 1);
    }
    __syncthreads();
  }
}

template <int D, int M, int PDE, int DIV, int FL>
__global__ void __launch_bounds__(FluxCfg<D, M, PDE, DIV>::THREADS, FluxCfg<D, M, PDE, DIV>::MINB) k_flux_update(const __grid_constant__ HotArgs a) {
  __shared__ FluxShm<FluxCfg<D, M, PDE, DIV>::CPB> fs;
  flux_update_body<D, M, PDE, DIV, FL>(a, blockIdx.x, fs);
}

// ------------------------------------------------------------------------------------------
// Update kernel, Eq. eq:finite_vol (source zero): one thread per active cell (update_cell).
// ------------------------------------------------------------------------------------------
template <int D, int M, int PDE>
__device__ __forceinline__ void update_body(const HotArgs& a, const int bid) {
  const int cell = bid * blockDim.x + threadIdx.x;
  if (cell >= a.na) return;
  const double dt = a.dtl[a.level];
  if (dt == 0.0) return;   // a step of length zero leaves the averages as they are
  update_cell<D, M, PDE>(a, cell, dt);
}

template <int D, int M, int PDE>
__global__ void k_update(const __grid_constant__ HotArgs a) {
  update_body<D, M, PDE>(a, blockIdx.x);
}

// ------------------------------------------------------------------------------------------
// Projection of virtual children (Sec. 3.1.3): child-box average of the mother's space-time
// polynomial at mother time tau = sub / r; one thread per (virtual cell, variable).
// With spatial dofs only (predictor == false) the mother's WENO polynomial is projected.
// ------------------------------------------------------------------------------------------
template <int D, int M, int PDE>
__device__ __forceinline__ void project_body(const HotArgs& a, const int32_t* vlist, int nv, const double* src,
                                             int spacetime, double* out_u, int write_dense, const int bid) {
  constexpr int N = M + 1, V = nvars(D, PDE), NSP = ipow(N, D), NST = NSP * N;
  const int it = bid * blockDim.x + threadIdx.x;
  if (it >= nv * V) return;
  const int k = it / V, v = it % V;
  const LevelView& L = a.lv;
  const LevelView& Lm = a.lvm;
  const int r = a.T.r;
  long long di = vlist[k];
  int ijk[3] = {(int)(di % L.L[0]), (int)((di / L.L[0]) % L.L[1]), (int)(di / ((long long)L.L[0] * L.L[1]))};
  int cm[3] = {ijk[0] / r, ijk[1] / r, D == 3 ? ijk[2] / r : 0};
  int ch[3] = {ijk[0] - r * cm[0], ijk[1] - r * cm[1], D == 3 ? ijk[2] - r * cm[2] : 0};
  int ma = Lm.aid[didx(Lm, cm[0], cm[1], cm[2])];
  if (ma < 0) { atomicOr(a.err, 4); return; }
  double acc = 0.0;
  if (spacetime) {
    const double* q = src + ((long long)ma * V + v) * NST;
    for (int nn = 0; nn < NST; nn++) {
      int t = nn;
      double th = 1.0;
      for (int b = 0; b < D; b++) { th *= a.T.Wc[ch[b]][t % N]; t /= N; }
      th *= a.T.Pt[a.sub][t];
      acc = fma(th, q[nn], acc);
    }
  } else {
    const double* q = src + ((long long)ma * V + v) * NSP;
    for (int nn = 0; nn < NSP; nn++) {
      int t = nn;
      double th = 1.0;
      for (int b = 0; b < D; b++) { th *= a.T.Wc[ch[b]][t % N]; t /= N; }
      acc = fma(th, q[nn], acc);
    }
  }
  if (write_dense) L.u[v * L.n + di] = acc;
  else out_u[(long long)k * V + v] = acc;
}

template <int D, int M, int PDE>
__global__ void k_project(const __grid_constant__ HotArgs a, const int32_t* vlist, int nv, const double* src,
                          int spacetime, double* out_u, int write_dense) {
  project_body<D, M, PDE>(a, vlist, nv, src, spacetime, out_u, write_dense, blockIdx.x);
}

// ------------------------------------------------------------------------------------------
// Batched launches: the same bodies over the CTAs of several solves (cross-request batching).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int batch_member(const HotBatch& b, int blk) {
  int m = 0;
  while (m + 1 < b.n && blk >= b.start[m + 1]) m++;
  return m;
}

template <int D, int M, int PDE, int TS>
__global__ void __launch_bounds__(256) k_weno_batch(const __grid_constant__ HotBatch b) {
  const int m = batch_member(b, blockIdx.x);
  weno_body<D, M, PDE, TS>(b.a[m], blockIdx.x - b.start[m]);
}

template <int D, int M, int PDE>
__global__ void __launch_bounds__(PredCfg<D, M, PDE>::THREADS) k_predict_batch(const __grid_constant__ HotBatch b) {
  const int m = batch_member(b, blockIdx.x);
  predict_body<D, M, PDE>(b.a[m], blockIdx.x - b.start[m]);
}

template <int D, int M, int PDE, int FL>
__global__ void __launch_bounds__(FluxCfg<D, M, PDE>::THREADS, FluxCfg<D, M, PDE>::MINB) k_flux_batch(const __grid_constant__ HotBatch b) {
  const int m = batch_member(b, blockIdx.x);
  __shared__ FluxShm<FluxCfg<D, M, PDE>::CPB> fs;
  flux_body<D, M, PDE, 1, FL>(b.a[m], blockIdx.x - b.start[m], fs);
}

// fused face flux and update of every member (each member counts the arrivals of its own chunks)
template <int D, int M, int PDE, int FL>
__global__ void __launch_bounds__(FluxCfg<D, M, PDE>::THREADS, FluxCfg<D, M, PDE>::MINB) k_flux_update_batch(const __grid_constant__ HotBatch b) {
  const int m = batch_member(b, blockIdx.x);
  __shared__ FluxShm<FluxCfg<D, M, PDE>::CPB> fs;
  flux_update_body<D, M, PDE, 1, FL>(b.a[m], blockIdx.x - b.start[m], fs);
}

template <int D, int M, int PDE>
__global__ void k_update_batch(const __grid_constant__ HotBatch b) {
  const int m = batch_member(b, blockIdx.x);
  update_body<D, M, PDE>(b.a[m], blockIdx.x - b.start[m]);
}

// WENO by passes over the members whose level has them (the same bodies)
#define AW_BATCHED_PASS(kname, bname)                                              \
  template <int M, int PDE>                                                        \
  __global__ void __launch_bounds__(128) kname(const __grid_constant__ HotBatch b) { \
    const int m = batch_member(b, blockIdx.x);                                     \
    bname<M, PDE>(b.a[m], blockIdx.x - b.start[m]);                                \
  }
AW_BATCHED_PASS(k_weno_x_batch, weno_x_body)
AW_BATCHED_PASS(k_weno_y_batch, weno_y_body)
AW_BATCHED_PASS(k_weno3_x_batch, weno3_x_body)
AW_BATCHED_PASS(k_weno3_y_batch, weno3_y_body)
AW_BATCHED_PASS(k_weno3_z_batch, weno3_z_body)
#undef AW_BATCHED_PASS

// virtual children of every member from their mothers' predictor at tau = sub / r
template <int D, int M, int PDE>
__global__ void k_project_batch(const __grid_constant__ HotBatch b) {
  const int m = batch_member(b, blockIdx.x);
  const HotArgs& a = b.a[m];
  project_body<D, M, PDE>(a, a.vlist, a.nv, a.qhm, 1, nullptr, 1, blockIdx.x - b.start[m]);
}

// ------------------------------------------------------------------------------------------
// Persistent level kernel of a batch (cross-request batching): one cooperative launch per level
// and sub-step runs, for every member, the projection of its virtual children, its WENO
// reconstruction (tiles or passes), its predictor and, when no member has a finer level (whose
// sub-steps must come in between), its fused face flux and update, one phase after another with
// a grid-wide barrier between dependent phases.  Every CTA is resident (cooperative launch), so
// the barriers end.  In each phase the CTAs loop over that phase's work items, the work items of
// the separate launches with the same bodies, so the results are bitwise those of the separate
// launches.  The CTA has the predictor's shape, which the face flux shares (FluxCfg), and the
// WENO and projection bodies take any CTA size.
// ------------------------------------------------------------------------------------------
enum { PH_PROJECT = 0, PH_WENO4, PH_WENO8, PH_WENO_X, PH_WENO_Y, PH_WENO_Z, PH_PREDICT, PH_FLUX, NPHASE };

struct LevelBatch {
  HotBatch b;
  int start[NPHASE][MAXB + 1];   // work of each phase: member m owns items start[p][m] .. start[p][m+1]-1
  int with_flux;                 // run the fused face flux and update too
};

template <int D, int M, int PDE, int FL>
__global__ void __launch_bounds__(PredCfg<D, M, PDE>::THREADS) k_level_batch(const __grid_constant__ LevelBatch lb) {
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  __shared__ FluxShm<FluxCfg<D, M, PDE>::CPB> fs;
  const HotBatch& b = lb.b;
  auto run = [&](int ph, auto&& body) {
    const int* st = lb.start[ph];
    for (int w = blockIdx.x; w < st[b.n]; w += gridDim.x) {
      int m = 0;
      while (m + 1 < b.n && w >= st[m + 1]) m++;
      body(b.a[m], w - st[m]);
      __syncthreads();   // the next item's body reuses the shared memory
    }
  };
  // (the fused flux's arrival counters are zero between launches: flux_update_body resets them)
  run(PH_PROJECT, [&](const HotArgs& a, int w) { project_body<D, M, PDE>(a, a.vlist, a.nv, a.qhm, 1, nullptr, 1, w); });
  grid.sync();
  run(PH_WENO4, [&](const HotArgs& a, int w) { weno_body<D, M, PDE, 4>(a, w); });
  if constexpr (D == 2) {
    run(PH_WENO8, [&](const HotArgs& a, int w) { weno_body<D, M, PDE, 8>(a, w); });
    run(PH_WENO_X, [&](const HotArgs& a, int w) { weno_x_body<M, PDE>(a, w); });
    grid.sync();
    run(PH_WENO_Y, [&](const HotArgs& a, int w) { weno_y_body<M, PDE>(a, w); });
  } else {
    run(PH_WENO_X, [&](const HotArgs& a, int w) { weno3_x_body<M, PDE>(a, w); });
    grid.sync();
    run(PH_WENO_Y, [&](const HotArgs& a, int w) { weno3_y_body<M, PDE>(a, w); });
    grid.sync();
    run(PH_WENO_Z, [&](const HotArgs& a, int w) { weno3_z_body<M, PDE>(a, w); });
  }
  grid.sync();
  run(PH_PREDICT, [&](const HotArgs& a, int w) { predict_body<D, M, PDE, 1>(a, w); });
  if (lb.with_flux) {
    grid.sync();
    run(PH_FLUX, [&](const HotArgs& a, int w) { flux_update_body<D, M, PDE, 1, FL>(a, w, fs); });
  }
}

template <int D, int M, int PDE>
HotOps make_ops();

}  // namespace aw
