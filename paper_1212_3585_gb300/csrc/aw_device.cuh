// aw_device.cuh -- device-side definitions shared by the kernels of the ADER-WENO solver:
// reference-element tables, PDE systems, per-level views and kernel arguments.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace aw {

constexpr int MAXN = 4;   // N = M + 1 <= 4 (M in {2, 3})
constexpr int MAXR = 4;   // refinement factor r <= 4
constexpr int MAXL = 5;   // levels 0..4
constexpr int MAXV = 9;
constexpr int8_t ST_NONE = -2;

enum { PDE_EULER = 0, PDE_MHD = 1, PDE_LINADV = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3 };

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Units (cells or face items of `per` threads each) of a reduced CTA of about `want` units: `want`
// itself, or the most units that fit in the whole warps `want` units fill, whichever leaves the
// smaller share of the last warp's lanes idle (idle lanes waste FP64 issue slots: a warp
// instruction occupies the pipe whatever its active lanes).
__host__ __device__ constexpr int warp_fill_units(int want, int per) {
  return (((want * per) / 32) * 32 / per > 0 &&
          (long long)(((want * per) / 32) * 32 / per) * per * (((want * per + 31) / 32) * 32) >
              (long long)want * per * (((((want * per) / 32) * 32 / per) * per + 31) / 32 * 32))
             ? ((want * per) / 32) * 32 / per
             : want;
}
static_assert(warp_fill_units(8, 9) == 7 && warp_fill_units(24, 3) == 21 && warp_fill_units(2, 27) == 2 &&
                  warp_fill_units(16, 4) == 16 && warp_fill_units(8, 4) == 8,
              "reduced CTAs fill their warps");
__host__ __device__ constexpr int nvars(int D, int PDE) {
  return PDE == PDE_LINADV ? 1 : (PDE == PDE_EULER ? D + 2 : 9);
}

// Reference-element tables (Sec. 2.2-2.3 and 3.1.3), computed on the host and passed by value
// in the kernel parameter space (read through the constant cache).
struct Tables {
  int N, M, Ns, r;
  double x[MAXN], w[MAXN];        // Gauss-Legendre nodes/weights on [0,1]
  double psi0[MAXN], psi1[MAXN];  // psi_l(0), psi_l(1)
  double Dm[MAXN][MAXN];          // Dm[i][l] = psi_l'(x_i): nodal derivative matrix
  int SL[4];                      // left extent of WENO stencil s
  double lam[4];                  // linear weight lambda_s
  double Ainv[4][MAXN][MAXN];     // Ainv[s][p][e]: stencil reconstruction matrix
  double Sig[MAXN][MAXN];         // oscillation indicator matrix
  // sigma_s as a quadratic form of the N-1 stencil differences to the cell value (the centre
  // cell's difference is zero): Bq[s][i][j] = B_ii on the diagonal, 2 B_ij above it, where
  // B = Ainv_s^T Sigma Ainv_s without the centre row and column
  double Bq[4][MAXN - 1][MAXN - 1];
  double G[MAXN][MAXN];           // K_t^{-1} diag(w): time block of the predictor
  double gsum[MAXN];              // row sums of G
  double Wc[MAXR][MAXN];          // Wc[c][l] = r * int_{c/r}^{(c+1)/r} psi_l (child averages)
  double Pf[MAXR][MAXN][MAXN];    // Pf[c][i][l] = psi_l((c + x_i)/r) (fine points in coarse frame)
  double Pt[MAXR][MAXN];          // Pt[k][l] = psi_l(k/r)
};

struct Phys {
  double gamma, c_h;
  double adv[3];
  double inflow[9];   // conserved state of the ghost cells beyond inflow faces
};

struct Bc6 {
  int v[6];           // boundary condition of faces x-, x+, y-, y+, z-, z+
  double inflow_rho;  // density of the inflow state (refinement indicator)
};

// One level of the mesh: dense status/average/active-id grids over the whole level box.
struct LevelView {
  int L[3];
  long long n;         // L[0]*L[1]*L[2]
  const int8_t* st;    // status per dense cell (ST_NONE, -1, 0, 1)
  double* u;           // averages, structure of arrays: u[v * n + c]
  const int32_t* aid;  // active id per dense cell or -1
  double dx[3];
};

__host__ __device__ inline long long didx(const LevelView& L, int i, int j, int k) {
  return ((long long)k * L.L[1] + j) * L.L[0] + i;
}

// coordinates of dense index di
__device__ __forceinline__ void cell_ijk(const LevelView& L, long long di, int* c) {
  c[0] = (int)(di % L.L[0]);
  c[1] = (int)((di / L.L[0]) % L.L[1]);
  c[2] = (int)(di / ((long long)L.L[0] * L.L[1]));
}

// Map coordinate c of axis a through the boundary conditions.  Returns true inside (possibly
// wrapped), false outside a transmissive boundary, where *out is clamped (ghost layers copy the
// adjacent interior cell of the same level), or outside a reflective wall, where *out is the
// mirror image (the caller negates the normal momentum).
__device__ __forceinline__ bool bcmap(const int* L, const int* bc, int a, int c, int* out) {
  int n = L[a];
  if (c >= 0 && c < n) { *out = c; return true; }
  int b = bc[2 * a + (c < 0 ? 0 : 1)];
  if (b == BC_PERIODIC) {
    int m = c % n;
    *out = m < 0 ? m + n : m;
    return true;
  }
  if (b == BC_REFLECTIVE) { *out = c < 0 ? -1 - c : 2 * n - 1 - c; return false; }
  *out = c < 0 ? 0 : n - 1;
  return false;
}

__device__ __forceinline__ bool reflected(const int* L, const int* bc, int a, int c) {
  return (c < 0 || c >= L[a]) && bc[2 * a + (c < 0 ? 0 : 1)] == BC_REFLECTIVE;
}

// beyond an inflow face: the ghost cell holds the inflow state, whatever the other directions
__device__ __forceinline__ bool beyond_inflow(const int* L, const int* bc, int a, int c) {
  return (c < 0 || c >= L[a]) && bc[2 * a + (c < 0 ? 0 : 1)] == BC_INFLOW;
}

// Reciprocal by the Newton-Raphson iteration y <- y + y (1 - x y) (quadratic convergence),
// seeded with the hardware's approximate double-precision reciprocal (PTX rcp.approx.ftz.f64,
// no conversions to and from single precision); two steps reach double precision (error a few
// ulp, tested against IEEE division).  Valid for normal |x| (subnormal inputs are flushed).
// On sm_103a the FP64 pipe is the bottleneck and this costs 4 FP64 FMAs instead of the ~10
// FP64 operations of an IEEE double division.
__device__ __forceinline__ double rcp_approx(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return y;
}

__device__ __forceinline__ double rcp_nr(double x) {
  double y = rcp_approx(x);
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// The same with one Newton-Raphson step: the seed's relative error (about 2^-20) squared, below
// 2^-38 (tested against IEEE division), for 2 FP64 FMAs less.  Used for 1/rho in the Euler
// fluxes of the predictor and of the face fluxes, and in the WENO weights; an error of 2^-38
// there changes a cell average by about 1e-12 of its size per step, far below the 1e-10 the
// solver is held to.
__device__ __forceinline__ double rcp_nr1(double x) {
  const double y = rcp_approx(x);
  return fma(y, fma(-x, y, 1.0), y);
}

// Square root of x >= 0 from the hardware's approximate reciprocal square root z ~ x^(-1/2)
// (PTX rsqrt.approx.ftz.f64, relative error about 2^-20) and one Newton step for the root of
// s^2 = x written with z: s = x z, s <- s + (x - s^2) z / 2.  Relative error below 2^-38 (tested
// against CUDA's sqrt), for about half the FP64 operations of a correctly rounded root.  Used
// for the sound speed in the face fluxes' spectral radius.  Arguments below 1e-300 (zero and
// subnormals, which the approximation flushes to zero) are taken as 1e-300.
__device__ __forceinline__ double sqrt_nr1(double x) {
  x = fmax(x, 1e-300);
  double z;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(z) : "d"(x));
  const double s = x * z;
  return fma(fma(-s, s, x), 0.5 * z, s);
}

// ------------------------------------------------------------------------------------------
// PDE systems.  Euler (Eq. eq:Euler-system), ideal MHD with hyperbolic GLM cleaning (Sec. 4.2,
// rationalised units) and linear advection.  All in FP64.
// ------------------------------------------------------------------------------------------
template <int PDE, int D>
struct Pde;

template <int D>
struct Pde<PDE_EULER, D> {
  static constexpr int V = D + 2;
  // fluxes in every direction at one state, sharing the primitive variables
  __device__ __forceinline__ static void fluxes(const double* q, double (*F)[V], const Phys& P) {
    double ir = rcp_nr1(q[0]);
    double v[D];
#pragma unroll
    for (int a = 0; a < D; a++) v[a] = q[1 + a] * ir;
    double ke = q[1] * v[0];
#pragma unroll
    for (int a = 1; a < D; a++) ke = fma(q[1 + a], v[a], ke);
    const double gm1 = P.gamma - 1.0;
    double p = gm1 * (q[D + 1] - 0.5 * ke);
    double Ep = q[D + 1] + p;
    // the off-diagonal momentum fluxes rho v_a v_n are symmetric in (a, n): computed once
    double mv[D][D];
#pragma unroll
    for (int n = 0; n < D; n++)
#pragma unroll
      for (int a = 0; a <= n; a++) mv[n][a] = mv[a][n] = (a == n) ? fma(q[1 + a], v[n], p) : q[1 + a] * v[n];
#pragma unroll
    for (int n = 0; n < D; n++) {
      F[n][0] = q[1 + n];
#pragma unroll
      for (int a = 0; a < D; a++) F[n][1 + a] = mv[n][a];
      F[n][D + 1] = v[n] * Ep;
    }
  }
  __device__ __forceinline__ static void flux(const double* q, int n, double* f, const Phys& P) {
    double ir = 1.0 / q[0];
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) ke += q[1 + a] * q[1 + a];
    double p = (P.gamma - 1.0) * (q[D + 1] - 0.5 * ke * ir);
    double vn = q[1 + n] * ir;
    f[0] = q[1 + n];
#pragma unroll
    for (int a = 0; a < D; a++) f[1 + a] = q[1 + a] * vn + (a == n ? p : 0.0);
    f[D + 1] = vn * (q[D + 1] + p);
  }
  __device__ __forceinline__ static double pressure(const double* q, const Phys& P) {
    double ke = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) ke += q[1 + a] * q[1 + a];
    return (P.gamma - 1.0) * (q[D + 1] - 0.5 * ke / q[0]);
  }
  // spectral radius of the flux Jacobian: eigenvalues v_n, v_n +- c with c^2 = gamma p / rho;
  // for a face state with c^2 < 0 the pair v_n +- c is complex with modulus sqrt(v_n^2 - c^2)
  __device__ __forceinline__ static double speed(const double* q, int n, const Phys& P) {
    double p = pressure(q, P);
    double vn = q[1 + n] / q[0], c2 = P.gamma * p / q[0];
    return c2 >= 0.0 ? fabs(vn) + sqrt(c2) : sqrt(vn * vn - c2);
  }
  __device__ __forceinline__ static bool physical(const double* q, const Phys& P) {
#pragma unroll
    for (int v = 0; v < V; v++)
      if (!(q[v] == q[v])) return false;
    return q[0] > 0.0 && pressure(q, P) > 0.0;
  }
};

template <int D>
struct Pde<PDE_MHD, D> {
  static constexpr int V = 9;
  // x/y/z fluxes of the MHD-GLM system for the directions n < ND, sharing the primitives
  template <int ND>
  __device__ __forceinline__ static void flux_dirs(const double* q, double (*F)[V], const Phys& P, int n0) {
    const double ir = rcp_nr(q[0]);
    const double vv[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
    const double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    const double mv = q[1] * vv[0] + q[2] * vv[1] + q[3] * vv[2];
    const double p = (P.gamma - 1.0) * (q[4] - 0.5 * mv - 0.5 * B2);
    const double vB = vv[0] * q[5] + vv[1] * q[6] + vv[2] * q[7];
    const double pt = p + 0.5 * B2;
    const double ch2 = P.c_h * P.c_h;
#pragma unroll
    for (int k = 0; k < ND; k++) {
      const int n = ND == 1 ? n0 : k;
      const double vn = vv[n], Bn = q[5 + n];
      double* f = F[k];
      f[0] = q[1 + n];
#pragma unroll
      for (int a = 0; a < 3; a++) f[1 + a] = q[1 + a] * vn + (a == n ? pt : 0.0) - q[5 + a] * Bn;
      f[4] = vn * (q[4] + pt) - Bn * vB;
#pragma unroll
      for (int a = 0; a < 3; a++) f[5 + a] = (a == n) ? q[8] : (vn * q[5 + a] - Bn * vv[a]);
      f[8] = ch2 * Bn;
    }
  }
  __device__ __forceinline__ static void flux(const double* q, int n, double* f, const Phys& P) {
    flux_dirs<1>(q, (double(*)[V])f, P, n);
  }
  __device__ __forceinline__ static void fluxes(const double* q, double (*F)[V], const Phys& P) {
    flux_dirs<D>(q, F, P, 0);
  }
  __device__ __forceinline__ static double pressure(const double* q, const Phys& P) {
    double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    return (P.gamma - 1.0) * (q[4] - 0.5 * m2 / q[0] - 0.5 * B2);
  }
  __device__ __forceinline__ static double speed(const double* q, int n, const Phys& P) {
    const double ir = rcp_nr(q[0]);
    double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    double p = (P.gamma - 1.0) * (q[4] - 0.5 * m2 * ir - 0.5 * B2);
    double a2 = P.gamma * p * ir;
    double b2 = B2 * ir, bn2 = q[5 + n] * q[5 + n] * ir;
    double s = a2 + b2;
    double cf = sqrt(0.5 * (s + sqrt(s * s - 4.0 * a2 * bn2)));
    double c = fabs(q[1 + n] * ir) + cf;
    return c > P.c_h ? c : P.c_h;
  }
  __device__ __forceinline__ static bool physical(const double* q, const Phys& P) {
#pragma unroll
    for (int v = 0; v < V; v++)
      if (!(q[v] == q[v])) return false;
    return q[0] > 0.0 && pressure(q, P) > 0.0;
  }
};

template <int D>
struct Pde<PDE_LINADV, D> {
  static constexpr int V = 1;
  __device__ __forceinline__ static void flux(const double* q, int n, double* f, const Phys& P) {
    f[0] = P.adv[n] * q[0];
  }
  __device__ __forceinline__ static void fluxes(const double* q, double (*F)[V], const Phys& P) {
#pragma unroll
    for (int n = 0; n < D; n++) F[n][0] = P.adv[n] * q[0];
  }
  __device__ __forceinline__ static double speed(const double*, int n, const Phys& P) { return fabs(P.adv[n]); }
  __device__ __forceinline__ static bool physical(const double* q, const Phys&) { return q[0] == q[0]; }
};

// Euler flux in direction n and the spectral radius of its Jacobian at one state, sharing 1/rho
// (face fluxes: one-step reciprocal and square root).
template <int D>
__device__ __forceinline__ double euler_flux_speed(const double* q, int n, double* f, const Phys& P) {
  const double ir = rcp_nr1(q[0]);
  const double vn = q[1 + n] * ir;
  double ke = q[1] * q[1];
#pragma unroll
  for (int a = 1; a < D; a++) ke = fma(q[1 + a], q[1 + a], ke);
  const double p = (P.gamma - 1.0) * fma(-0.5 * ir, ke, q[D + 1]);
  f[0] = q[1 + n];
#pragma unroll
  for (int a = 0; a < D; a++) f[1 + a] = (a == n) ? fma(q[1 + a], vn, p) : q[1 + a] * vn;
  f[D + 1] = vn * (q[D + 1] + p);
  const double c2 = P.gamma * p * ir;
  return c2 >= 0.0 ? fabs(vn) + sqrt_nr1(c2) : sqrt(fma(vn, vn, -c2));
}

// |A(q)| dq for the Euler flux in direction n, from the characteristic decomposition: wave
// amplitudes alpha = L dq (acoustic -, entropy, shears, acoustic +), scaled by |u_n - c|, |u_n|,
// |u_n + c|, and recombined with the right eigenvectors.  Where c^2 <= 0 the eigenvalues are
// complex and |A| dq is replaced by the spectral radius times dq.
template <int D>
__device__ __forceinline__ void euler_abs_jacobian_apply(const double* q, int n, const double* dq, double* out,
                                                         const Phys& P) {
  constexpr int V = D + 2;
  const double ir = rcp_nr(q[0]);
  double v[D], v2 = 0.0, vdm = 0.0;
#pragma unroll
  for (int a = 0; a < D; a++) { v[a] = q[1 + a] * ir; v2 = fma(v[a], v[a], v2); vdm = fma(v[a], dq[1 + a], vdm); }
  const double p = (P.gamma - 1.0) * fma(-0.5 * q[0], v2, q[D + 1]);
  const double c2 = P.gamma * p * ir;
  const double un = v[n];
  if (!(c2 > 0.0)) {
    const double sr = sqrt(fma(un, un, -c2));
#pragma unroll
    for (int k = 0; k < V; k++) out[k] = sr * dq[k];
    return;
  }
  const double c = sqrt(c2), icv = rcp_nr(c), H = (q[D + 1] + p) * ir;
  const double b1 = (P.gamma - 1.0) * rcp_nr(c2);
  const double b2 = 0.5 * v2 * b1;
  const double Pq = b1 * (vdm - dq[D + 1]);
  const double A = (un * dq[0] - dq[1 + n]) * icv;
  double a0 = 0.5 * (b2 * dq[0] - Pq + A);
  double a1 = (1.0 - b2) * dq[0] + Pq;
  double a4 = 0.5 * (b2 * dq[0] - Pq - A);
  a0 *= fabs(un - c);
  a1 *= fabs(un);
  a4 *= fabs(un + c);
  const double s04 = a0 + a4, d40 = a4 - a0, sum = s04 + a1;
  double eshear = 0.0;
  out[0] = sum;
#pragma unroll
  for (int a = 0; a < D; a++) {
    double o = v[a] * sum;
    if (a == n) o = fma(c, d40, o);
    else {
      double as = fabs(un) * fma(-v[a], dq[0], dq[1 + a]);
      o += as;
      eshear = fma(v[a], as, eshear);
    }
    out[1 + a] = o;
  }
  out[D + 1] = H * s04 + un * c * d40 + 0.5 * v2 * a1 + eshear;
}

// Osher-Solomon flux of Dumbser and Toro, Eq. eqn.osher: straight path between the states,
// |A| integrated by the 3-point Gauss-Legendre rule on [0,1].
template <int D>
__device__ __forceinline__ void osher_euler(const double* qm, const double* qp, int n, double* out, const Phys& P) {
  constexpr int V = D + 2;
  const double gs[3] = {0.5 - 0.3872983346207417, 0.5, 0.5 + 0.3872983346207417};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double fm[V], fp[V], dq[V], acc[V];
  euler_flux_speed<D>(qm, n, fm, P);
  euler_flux_speed<D>(qp, n, fp, P);
#pragma unroll
  for (int k = 0; k < V; k++) { dq[k] = qp[k] - qm[k]; acc[k] = 0.0; }
#pragma unroll
  for (int j = 0; j < 3; j++) {
    double q[V], t[V];
#pragma unroll
    for (int k = 0; k < V; k++) q[k] = fma(gs[j], dq[k], qm[k]);
    euler_abs_jacobian_apply<D>(q, n, dq, t, P);
#pragma unroll
    for (int k = 0; k < V; k++) acc[k] = fma(gw[j], t[k], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < V; k++) out[k] = fma(-0.5, acc[k], 0.5 * (fm[k] + fp[k]));
}

// Jacobian of the MHD-GLM flux in direction n with respect to the conserved variables, by the
// chain rule through the primitive variables W = (rho, v_x, v_y, v_z, p, B_x, B_y, B_z, psi):
// A = (dF/dW)(dW/dQ), both factors written out from the flux and the equation of state
// (rationalised units).  A[i * 9 + j] = dF_i / dQ_j.
__device__ __forceinline__ void mhd_jacobian(const double* q, int n, double* A, const Phys& P) {
  const double g = P.gamma, g1 = g - 1.0, rho = q[0], ir = 1.0 / rho;
  double v[3], B[3];
#pragma unroll
  for (int a = 0; a < 3; a++) { v[a] = q[1 + a] * ir; B[a] = q[5 + a]; }
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  const double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  const double p = g1 * (q[4] - 0.5 * rho * v2 - 0.5 * B2);
  const double Ept = g * p / g1 + 0.5 * rho * v2 + B2;   // E + p_t
  const double vn = v[n], Bn = B[n];
  // dF/dW, rows F, columns W
  double FW[81];
  for (int k = 0; k < 81; k++) FW[k] = 0.0;
  FW[0 * 9 + 0] = vn;
  FW[0 * 9 + 1 + n] = rho;
  for (int a = 0; a < 3; a++) {
    double* r = FW + (1 + a) * 9;
    r[0] = v[a] * vn;
    r[1 + a] += rho * vn;
    r[1 + n] += rho * v[a];
    if (a == n) r[4] = 1.0;
    for (int b = 0; b < 3; b++) r[5 + b] = (a == n ? B[b] : 0.0) - (a == b ? Bn : 0.0) - (b == n ? B[a] : 0.0);
  }
  {
    double* r = FW + 4 * 9;
    r[0] = 0.5 * vn * v2;
    for (int b = 0; b < 3; b++) {
      r[1 + b] = (b == n ? Ept : 0.0) + vn * rho * v[b] - Bn * B[b];
      r[5 + b] = 2.0 * vn * B[b] - (b == n ? vB : 0.0) - Bn * v[b];
    }
    r[4] = vn * g / g1;
  }
  for (int a = 0; a < 3; a++) {
    double* r = FW + (5 + a) * 9;
    if (a == n) { r[8] = 1.0; continue; }
    r[1 + n] = B[a];
    r[1 + a] -= Bn;
    r[5 + a] = vn;
    r[5 + n] -= v[a];
  }
  FW[8 * 9 + 5 + n] = P.c_h * P.c_h;
  // dW/dQ
  double WQ[81];
  for (int k = 0; k < 81; k++) WQ[k] = 0.0;
  WQ[0] = 1.0;
  for (int a = 0; a < 3; a++) {
    WQ[(1 + a) * 9 + 0] = -v[a] * ir;
    WQ[(1 + a) * 9 + 1 + a] = ir;
    WQ[4 * 9 + 1 + a] = -g1 * v[a];
    WQ[4 * 9 + 5 + a] = -g1 * B[a];
    WQ[(5 + a) * 9 + 5 + a] = 1.0;
  }
  WQ[4 * 9 + 0] = 0.5 * g1 * v2;
  WQ[4 * 9 + 4] = g1;
  WQ[8 * 9 + 8] = 1.0;
  for (int i = 0; i < 9; i++)
    for (int j = 0; j < 9; j++) {
      double t = 0.0;
      for (int k = 0; k < 9; k++) t = fma(FW[i * 9 + k], WQ[k * 9 + j], t);
      A[i * 9 + j] = t;
    }
}

// |A(q)| dq for the MHD-GLM flux in direction n: |A| = A sign(A), the sign by the Newton-Schulz
// iteration S <- S (3 I - S^2) / 2 from S = A / s, s = max(|v_n| + c_f, c_h) the spectral radius
// (each eigenvalue x / s in [-1, 1] goes to its sign, 0 stays 0; 80 steps bring every eigenvalue
// above 1e-14 s to +-1).  Where gamma p / rho <= 0 the fast speed is not real and |A| dq is
// s dq with s = max(|v_n| + |B| / sqrt(rho), c_h).  The matrices live in local memory.
template <int D>
__device__ __noinline__ void mhd_abs_jacobian_apply(const double* q, int n, const double* dq, double* out,
                                                    const Phys& P) {
  const double rho = q[0];
  const double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  const double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const double p = (P.gamma - 1.0) * (q[4] - 0.5 * m2 / rho - 0.5 * B2);
  if (!(P.gamma * p / rho > 0.0)) {
    double s = fabs(q[1 + n] / rho) + sqrt(B2 / rho);
    if (s < P.c_h) s = P.c_h;
    for (int v = 0; v < 9; v++) out[v] = s * dq[v];
    return;
  }
  double A[81], S[81], T[81];
  mhd_jacobian(q, n, A, P);
  const double is = 1.0 / Pde<PDE_MHD, D>::speed(q, n, P);
  for (int k = 0; k < 81; k++) S[k] = A[k] * is;
  for (int it = 0; it < 80; it++) {
    // T = 3 I - S^2
    for (int i = 0; i < 9; i++)
      for (int j = 0; j < 9; j++) {
        double t = 0.0;
        for (int k = 0; k < 9; k++) t = fma(S[i * 9 + k], S[k * 9 + j], t);
        T[i * 9 + j] = (i == j ? 3.0 : 0.0) - t;
      }
    // S <- S T / 2, a row at a time (row i of the product needs row i of S only)
    for (int i = 0; i < 9; i++) {
      double row[9];
#pragma unroll
      for (int j = 0; j < 9; j++) {
        double t = 0.0;
        for (int k = 0; k < 9; k++) t = fma(S[i * 9 + k], T[k * 9 + j], t);
        row[j] = 0.5 * t;
      }
#pragma unroll
      for (int j = 0; j < 9; j++) S[i * 9 + j] = row[j];
    }
  }
  double w[9];
  for (int i = 0; i < 9; i++) {
    double t = 0.0;
    for (int k = 0; k < 9; k++) t = fma(S[i * 9 + k], dq[k], t);
    w[i] = t;
  }
  for (int i = 0; i < 9; i++) {
    double t = 0.0;
    for (int k = 0; k < 9; k++) t = fma(A[i * 9 + k], w[k], t);
    out[i] = t;
  }
}

// Osher-Solomon flux of Dumbser and Toro for MHD-GLM, Eq. eqn.osher: the straight path between
// the states, |A| integrated by the 3-point Gauss-Legendre rule on [0,1].
template <int D>
__device__ __forceinline__ void osher_mhd(const double* qm, const double* qp, int n, double* out, const Phys& P) {
  constexpr int V = 9;
  const double gs[3] = {0.5 - 0.3872983346207417, 0.5, 0.5 + 0.3872983346207417};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  double fm[V], fp[V], dq[V], acc[V];
  Pde<PDE_MHD, D>::flux(qm, n, fm, P);
  Pde<PDE_MHD, D>::flux(qp, n, fp, P);
#pragma unroll
  for (int k = 0; k < V; k++) { dq[k] = qp[k] - qm[k]; acc[k] = 0.0; }
  for (int j = 0; j < 3; j++) {
    double q[V], t[V];
#pragma unroll
    for (int k = 0; k < V; k++) q[k] = fma(gs[j], dq[k], qm[k]);
    mhd_abs_jacobian_apply<D>(q, n, dq, t, P);
#pragma unroll
    for (int k = 0; k < V; k++) acc[k] = fma(gw[j], t[k], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < V; k++) out[k] = fma(-0.5, acc[k], 0.5 * (fm[k] + fp[k]));
}

// Rusanov flux, Eq. eqn.rusanov: s_max is the larger of the two states' largest |eigenvalue|.
template <int PDE, int D>
__device__ __forceinline__ void rusanov(const double* qm, const double* qp, int n, double* out, const Phys& P) {
  if constexpr (PDE == PDE_EULER) {
    constexpr int V = D + 2;
    double fm[V], fp[V];
    double sm = euler_flux_speed<D>(qm, n, fm, P), sp = euler_flux_speed<D>(qp, n, fp, P);
    double hs = 0.5 * (sm > sp ? sm : sp);
#pragma unroll
    for (int v = 0; v < V; v++) out[v] = fma(-hs, qp[v] - qm[v], 0.5 * (fm[v] + fp[v]));
    return;
  }
  using Q = Pde<PDE, D>;
  constexpr int V = Q::V;
  double fm[V], fp[V];
  Q::flux(qm, n, fm, P);
  Q::flux(qp, n, fp, P);
  double sm = Q::speed(qm, n, P), sp = Q::speed(qp, n, P);
  double s = sm > sp ? sm : sp;
#pragma unroll
  for (int v = 0; v < V; v++) out[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * s * (qp[v] - qm[v]);
}

// Arguments of the per-level hot kernels.
struct HotArgs {
  Tables T;
  Phys P;
  int bc[6];
  int flux;             // 0 Rusanov, 1 Osher-Solomon (Euler)
  int level, sub, picard;
  LevelView lv;         // this level
  LevelView lvm;        // mother level (level-1), valid when level >= 1
  LevelView lvc;        // child level (level+1), valid when level < lmax
  const int32_t* alist; // active cells of this level (dense indices), canonical order
  int na;
  const int32_t* hflist; // high faces to compute: axis * na + active id, axis-major, where the +axis
  int nh;                // neighbour is not an active cell of this level
  const int32_t* tiles; // tile origins (tile linear index on the level's tile grid)
  int ntiles;
  int tdim[3];          // tiles per direction
  double* wh;           // WENO dofs per active cell [aid][V][N^d]
  double* qh;           // predictor dofs per active cell [aid][V][N^(d+1)]
  const double* qhm;    // predictor dofs of the mother level
  double* fl;           // face fluxes per active cell [aid][2d][V]
  double* mem;          // memory variables per active cell of this level [aid][2d][V]
  double* memc;         // memory variables of the child level
  const double* dtl;    // device array: dt of each level
  int* err;             // device error word
  const int32_t* vlist; // virtual children of this level (dense indices), projected from qhm
  int nv;
  int ts;               // WENO tile edge of this level
  // WENO by passes (null xs: tiles): rows whose x sweep feeds an active cell, the dense
  // cell -> row slot map and the x sweeps [slot][V][N]; in 3D also the cells whose y sweeps feed
  // an active cell, their slot map and the y sweeps [slot][V][N][N]
  const int32_t* xlist;
  const int32_t* xslot;
  double* xs;
  int nxs;
  const int32_t* ylist;
  const int32_t* yslot;
  double* ys;
  int nys;
  // fused face flux and update (k_flux_update): face arrivals per chunk of active cells, zeroed
  // before each launch
  int* fsync;
  // CTA size of the predictor and face-flux launches: 0 the launch rules, 1 full-size, 4
  // reduced size (the autotuner's choice; the results are the same either way)
  int cta_div;
};

// Several independent solves of the same kernel configuration in one launch: member m owns CTAs
// start[m] .. start[m+1]-1 and runs them with its own arguments (passed as one grid-constant
// kernel parameter, 20.8 KB for 8 members).
constexpr int MAXB = 8;
struct HotBatch {
  int n;
  int start[MAXB + 1];
  HotArgs a[MAXB];
};

}  // namespace aw
