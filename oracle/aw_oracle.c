/*
 * aw_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 reference implementation ("oracle") of the one-step ADER-WENO finite
 * volume scheme on space-time adaptive Cartesian meshes of Dumbser, Zanotti, Hidalgo and
 * Balsara (arXiv:1212.3585).  Only tests/, __graft_entry__.smoke() and bench.py (its
 * cpu_baseline leg and its --impl reference arm) may load it.  It shares no code, header,
 * table or helper with the CUDA path; it computes its own Gauss-Legendre nodes, Lagrange
 * basis, stencil inverses, oscillation matrix and space-time matrices from their definitions.
 *
 * It is written for checking by eye against the paper, not for speed:
 *   - WENO: every cell reconstructs its own (2M+1)^d box, one 1D reconstruction at a time
 *     (Sec. 2.2, Eqs. eqn.rec.x .. eqn.weno.z).
 *   - Predictor: full (N^{d+1})^2 space-time matrices K1, K_xi, F0 built by quadrature,
 *     K1 inverted by Gauss-Jordan, Picard iteration of Eq. eqn.stdg.final (Sec. 2.3).
 *   - Fluxes: q_h evaluated as a full space-time polynomial at every Gauss point of every
 *     face; every cell computes all of its faces itself (Eqs. flux:F..flux:H, eqn.rusanov).
 *   - AMR: per-level dense grids of cells with status sigma in {-1,0,1} (Sec. 3.1 rules
 *     1-7), local time stepping by recursion on the update criterion (Sec. 3.1.2,
 *     Eq. eqn.update.criterion), memory variables (Eq. eqn.memory.sum), projection
 *     (Sec. 3.1.3) and averaging (Eq. eqn.average).
 * Readings of points where the paper is silent are stated where they are used.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_*.py against closed
 * forms, exact rationals, invariants or brute force; see the test module docstrings.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 5            /* N = M+1 <= 5 */
#define MAXL 6            /* levels 0..5 */
#define MAXV 9
#define ST_NONE ((int8_t)-2)

enum { PDE_EULER = 0, PDE_MHD = 1, PDE_LINADV = 2 };
enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1, BC_REFLECTIVE = 2, BC_INFLOW = 3 };
enum { IC_CONST = 0, IC_VORTEX = 1, IC_EXPLOSION = 2, IC_OT = 3, IC_RP4 = 4, IC_FOURIER = 5 };

typedef struct {
  int dim, pde, M, nx, ny, nz;
  double gamma, c_h;
  double lo[3], hi[3];
  int bc[6];
  int r, lmax;
  double chi_ref, chi_rec, eps_ind, cfl;
  int picard;
  int auto_regrid;
  double adv[3];
  int flux; /* 0 Rusanov, 1 Osher-Solomon (Dumbser-Toro) */
  double inflow[MAXV]; /* conserved state held by the ghost cells beyond BC_INFLOW faces */
} orc_cfg;

static char g_err[512];
static void seterr(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char *orc_last_error(void) { return g_err; }

/* ===================================================================================
 * 1. One-dimensional polynomials, Gauss-Legendre rule, nodal basis (Sec. 2.2)
 * =================================================================================== */

/* Gauss-Legendre nodes/weights on [0,1], ascending (reading: node order ascending).
 * Newton iteration on the Legendre polynomial P_n from the classical cosine guesses. */
static void gauss_legendre01(int n, double *x, double *w) {
  for (int i = 0; i < n; i++) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 200; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[n - 1 - i] = 0.5 * (1.0 + z);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* polynomial with coefficients c[0..n-1]; c[k] multiplies (x - 1/2)^k (monomials centred
 * on the reference interval keep the coefficients small) */
static double poly_eval(const double *c, int n, double x) {
  double s = 0.0, y = x - 0.5;
  for (int k = n - 1; k >= 0; k--) s = s * y + c[k];
  return s;
}
static void poly_deriv(const double *c, int n, double *out) {
  for (int k = 0; k < n; k++) out[k] = (k + 1 < n) ? (k + 1) * c[k + 1] : 0.0;
}
static double poly_integral(const double *c, int n, double a, double b) {
  double s = 0.0;
  for (int k = 0; k < n; k++) s += c[k] * (pow(b - 0.5, k + 1) - pow(a - 0.5, k + 1)) / (k + 1);
  return s;
}

/* Lagrange basis psi_l through the GL nodes: coefficient table coef[l][k] of (xi-1/2)^k. */
static void lagrange_coeffs(int N, const double *x, double coef[MAXN][MAXN]) {
  for (int l = 0; l < N; l++) {
    double c[MAXN] = {1.0};
    int deg = 0;
    for (int k = 0; k < N; k++) {
      if (k == l) continue;
      double den = x[l] - x[k];
      double nc[MAXN] = {0};
      /* multiply by (xi - x_k)/den = ((xi - 1/2) - (x_k - 1/2))/den */
      for (int j = 0; j <= deg; j++) {
        nc[j + 1] += c[j] / den;
        nc[j] -= c[j] * (x[k] - 0.5) / den;
      }
      deg++;
      memcpy(c, nc, sizeof c);
    }
    for (int k = 0; k < N; k++) coef[l][k] = c[k];
  }
}

/* Gauss-Jordan inverse with partial pivoting, n x n row-major. Returns 0 on success. */
static int invert(int n, const double *A, double *Ainv) {
  double *a = malloc(sizeof(double) * n * 2 * n);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < 2 * n; j++) a[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i);
  for (int c = 0; c < n; c++) {
    int piv = c;
    for (int i = c + 1; i < n; i++)
      if (fabs(a[i * 2 * n + c]) > fabs(a[piv * 2 * n + c])) piv = i;
    if (fabs(a[piv * 2 * n + c]) < 1e-300) { free(a); return -1; }
    if (piv != c)
      for (int j = 0; j < 2 * n; j++) {
        double t = a[c * 2 * n + j];
        a[c * 2 * n + j] = a[piv * 2 * n + j];
        a[piv * 2 * n + j] = t;
      }
    double d = a[c * 2 * n + c];
    for (int j = 0; j < 2 * n; j++) a[c * 2 * n + j] /= d;
    for (int i = 0; i < n; i++) {
      if (i == c) continue;
      double f = a[i * 2 * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; j++) a[i * 2 * n + j] -= f * a[c * 2 * n + j];
    }
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) Ainv[i * n + j] = a[i * 2 * n + n + j];
  free(a);
  return 0;
}

/* ===================================================================================
 * 2. Reference-element tables: WENO stencils (Eq. eqn.stencildef), stencil inverses
 *    (Eq. eqn.rec.x), oscillation matrix (Eq. eqn.sigmas), space-time matrices
 *    K1, K_xi, F0 (Sec. 2.3, before Eq. eqn.pde.weak4).
 * =================================================================================== */
typedef struct {
  int M, N, Ns, d, nsp, nst;
  double x[MAXN], w[MAXN];
  double psi[MAXN][MAXN]; /* psi[l][k] coefficient of (xi - 1/2)^k */
  int SL[4], SR[4];
  double lam[4];
  double Ainv[4][MAXN][MAXN]; /* Ainv[s][p][e]: coefficient p from the e-th stencil cell */
  double Sig[MAXN][MAXN];
  double *K1inv; /* nst x nst */
  double *Kd[3]; /* nst x nst */
  double *F0;    /* nst x nsp */
} tables;

/* stencil extents (reading: M even -> 3 stencils, M odd -> 4 stencils, centrals first) */
static void stencils(int M, int *Ns, int *SL, int *SR, double *lam) {
  if (M % 2 == 0) {
    *Ns = 3;
    SL[0] = M / 2; SR[0] = M / 2; lam[0] = 1e5;
    SL[1] = M;     SR[1] = 0;     lam[1] = 1.0;
    SL[2] = 0;     SR[2] = M;     lam[2] = 1.0;
  } else {
    *Ns = 4;
    SL[0] = M / 2 + 1; SR[0] = M / 2;     lam[0] = 1e5;
    SL[1] = M / 2;     SR[1] = M / 2 + 1; lam[1] = 1e5;
    SL[2] = M;         SR[2] = 0;         lam[2] = 1.0;
    SL[3] = 0;         SR[3] = M;         lam[3] = 1.0;
  }
}

/* value of the 1D basis function psi_l (or its first derivative) at xi */
static double psi_val(const tables *T, int l, double xi) { return poly_eval(T->psi[l], T->N, xi); }
static double psi_der(const tables *T, int l, double xi) {
  double dc[MAXN];
  poly_deriv(T->psi[l], T->N, dc);
  return poly_eval(dc, T->N, xi);
}

static void build_tables(tables *T, int M, int d) {
  memset(T, 0, sizeof *T);
  T->M = M; T->N = M + 1; T->d = d;
  int N = T->N;
  gauss_legendre01(N, T->x, T->w);
  lagrange_coeffs(N, T->x, T->psi);
  stencils(M, &T->Ns, T->SL, T->SR, T->lam);
  /* integral conservation matrix per stencil: A[e][p] = int_{o_e}^{o_e+1} psi_p */
  for (int s = 0; s < T->Ns; s++) {
    double A[MAXN * MAXN] = {0}, Ai[MAXN * MAXN] = {0};
    for (int e = 0; e < N; e++) {
      double o = -T->SL[s] + e;
      for (int p = 0; p < N; p++) A[e * N + p] = poly_integral(T->psi[p], N, o, o + 1.0);
    }
    invert(N, A, Ai);
    for (int p = 0; p < N; p++)
      for (int e = 0; e < N; e++) T->Ainv[s][p][e] = Ai[p * N + e];
  }
  /* Sigma_pm = sum_{alpha=1..M} int_0^1 psi_p^(alpha) psi_m^(alpha); the integrand has
   * degree <= 2M-2, so the N-point Gauss rule is exact */
  {
    double der[MAXN][MAXN][MAXN]; /* der[alpha-1][l][gauss point] */
    for (int l = 0; l < N; l++) {
      double c[MAXN];
      memcpy(c, T->psi[l], sizeof c);
      for (int a = 1; a <= M; a++) {
        double t[MAXN];
        poly_deriv(c, N, t);
        memcpy(c, t, sizeof t);
        for (int g = 0; g < N; g++) der[a - 1][l][g] = poly_eval(c, N, T->x[g]);
      }
    }
    for (int p = 0; p < N; p++)
      for (int m = 0; m < N; m++) {
        double s = 0.0;
        for (int a = 1; a <= M; a++)
          for (int g = 0; g < N; g++) s += T->w[g] * der[a - 1][p][g] * der[a - 1][m][g];
        T->Sig[p][m] = s;
      }
  }
  /* space-time matrices by (N+1)-point Gauss quadrature in each of the d+1 directions,
   * which integrates the polynomial integrands (degree <= 2M+1 per direction) exactly */
  int nsp = 1;
  for (int a = 0; a < d; a++) nsp *= N;
  int nst = nsp * N;
  T->nsp = nsp; T->nst = nst;
  int Q = N + 1;
  double qx[MAXN + 1], qw[MAXN + 1];
  gauss_legendre01(Q, qx, qw);
  /* basis values at quadrature points */
  double B[MAXN][MAXN + 1], DB[MAXN][MAXN + 1], B1[MAXN], B0[MAXN];
  for (int l = 0; l < N; l++) {
    for (int i = 0; i < Q; i++) { B[l][i] = psi_val(T, l, qx[i]); DB[l][i] = psi_der(T, l, qx[i]); }
    B1[l] = psi_val(T, l, 1.0);
    B0[l] = psi_val(T, l, 0.0);
  }
  double *K1 = calloc((size_t)nst * nst, sizeof(double));
  for (int a = 0; a < d; a++) T->Kd[a] = calloc((size_t)nst * nst, sizeof(double));
  T->F0 = calloc((size_t)nst * nsp, sizeof(double));
  T->K1inv = calloc((size_t)nst * nst, sizeof(double));
  int nqs = 1;
  for (int a = 0; a < d; a++) nqs *= Q;
  for (int iq = 0; iq < nst; iq++)
    for (int ip = 0; ip < nst; ip++) {
      int qi[4], pi[4];
      int t1 = iq, t2 = ip;
      for (int a = 0; a < d; a++) { qi[a] = t1 % N; t1 /= N; pi[a] = t2 % N; t2 /= N; }
      int qs = t1, ps = t2;
      double k1 = 0.0, kd[3] = {0, 0, 0};
      for (int g = 0; g < nqs; g++) {
        int gi[3], tg = g;
        double wsp = 1.0, thq = 1.0, thp = 1.0;
        for (int a = 0; a < d; a++) {
          gi[a] = tg % Q; tg /= Q;
          wsp *= qw[gi[a]];
          thq *= B[qi[a]][gi[a]];
          thp *= B[pi[a]][gi[a]];
        }
        /* boundary term at tau = 1 */
        k1 += wsp * thq * B1[qs] * thp * B1[ps];
        for (int gt = 0; gt < Q; gt++) {
          double wt = wsp * qw[gt];
          /* - int (d/dtau theta_q) theta_p */
          k1 -= wt * thq * DB[qs][gt] * thp * B[ps][gt];
          /* K_a = int theta_q d/dxi_a theta_p */
          for (int a = 0; a < d; a++) {
            double dthp = 1.0;
            for (int b = 0; b < d; b++) dthp *= (b == a) ? DB[pi[b]][gi[b]] : B[pi[b]][gi[b]];
            kd[a] += wt * thq * B[qs][gt] * dthp * B[ps][gt];
          }
        }
      }
      K1[iq * nst + ip] = k1;
      for (int a = 0; a < d; a++) T->Kd[a][iq * nst + ip] = kd[a];
    }
  /* F0_{q m} = int theta_q(xi,0) psi_m(xi) dxi */
  for (int iq = 0; iq < nst; iq++)
    for (int im = 0; im < nsp; im++) {
      int qi[4], mi[4], t1 = iq, t2 = im;
      for (int a = 0; a < d; a++) { qi[a] = t1 % N; t1 /= N; mi[a] = t2 % N; t2 /= N; }
      int qs = t1;
      double s = 0.0;
      for (int g = 0; g < nqs; g++) {
        int tg = g;
        double v = 1.0;
        for (int a = 0; a < d; a++) {
          int gi = tg % Q; tg /= Q;
          v *= qw[gi] * B[qi[a]][gi] * B[mi[a]][gi];
        }
        s += v * B0[qs];
      }
      T->F0[iq * nsp + im] = s;
    }
  invert(nst, K1, T->K1inv);
  free(K1);
}

static void free_tables(tables *T) {
  free(T->K1inv); free(T->F0);
  for (int a = 0; a < 3; a++) free(T->Kd[a]);
}

/* ===================================================================================
 * 3. PDE systems: Euler (Eq. eq:Euler-system) and ideal MHD with hyperbolic GLM
 *    cleaning (Sec. 4.2) in rationalised units (reading: the 4*pi factors dropped),
 *    plus linear advection as a test system.
 * =================================================================================== */
typedef struct { int pde, d, V, flux; double gamma, c_h, adv[3]; } phys;

static void flux(const phys *P, const double *q, int n, double *f) {
  if (P->pde == PDE_LINADV) { f[0] = P->adv[n] * q[0]; return; }
  double g = P->gamma;
  if (P->pde == PDE_EULER) {
    int d = P->d;
    double rho = q[0], E = q[d + 1], ke = 0.0;
    for (int a = 0; a < d; a++) ke += q[1 + a] * q[1 + a];
    ke = 0.5 * ke / rho;
    double p = (g - 1.0) * (E - ke);
    double vn = q[1 + n] / rho;
    f[0] = q[1 + n];
    for (int a = 0; a < d; a++) f[1 + a] = q[1 + a] * vn + (a == n ? p : 0.0);
    f[d + 1] = vn * (E + p);
    return;
  }
  /* MHD-GLM: q = (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi) */
  double rho = q[0], E = q[4], psi = q[8];
  double v[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  const double *B = q + 5;
  double B2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double p = (g - 1.0) * (E - 0.5 * rho * v2 - 0.5 * B2);
  double vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  double pt = p + 0.5 * B2;
  f[0] = q[1 + n];
  for (int a = 0; a < 3; a++) f[1 + a] = q[1 + a] * v[n] + (a == n ? pt : 0.0) - B[a] * B[n];
  f[4] = v[n] * (E + pt) - B[n] * vB;
  for (int a = 0; a < 3; a++) f[5 + a] = (a == n) ? psi : (v[n] * B[a] - B[n] * v[a]);
  f[8] = P->c_h * P->c_h * B[n];
}

static double pressure(const phys *P, const double *q) {
  double g = P->gamma;
  if (P->pde == PDE_EULER) {
    int d = P->d;
    double ke = 0.0;
    for (int a = 0; a < d; a++) ke += q[1 + a] * q[1 + a];
    return (g - 1.0) * (q[d + 1] - 0.5 * ke / q[0]);
  }
  if (P->pde == PDE_MHD) {
    double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
    return (g - 1.0) * (q[4] - 0.5 * m2 / q[0] - 0.5 * B2);
  }
  return 1.0;
}

/* largest |eigenvalue| of the flux Jacobian in direction n (used by Rusanov, Eq. eqn.rusanov,
 * and by the CFL condition) */
static double max_speed(const phys *P, const double *q, int n) {
  if (P->pde == PDE_LINADV) return fabs(P->adv[n]);
  double rho = q[0], p = pressure(P, q);
  double vn = q[1 + n] / rho;
  if (P->pde == PDE_EULER) {
    /* eigenvalues v_n, v_n +- c with c^2 = gamma p / rho; a state extrapolated to a face can
     * have c^2 < 0, where v_n +- c are complex and the largest modulus is sqrt(v_n^2 - c^2)
     * (reading of Eq. eqn.rusanov: the spectral radius, taken literally) */
    double c2 = P->gamma * p / rho;
    return c2 >= 0.0 ? fabs(vn) + sqrt(c2) : sqrt(vn * vn - c2);
  }
  double a2 = P->gamma * p / rho;
  double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
  double b2 = B2 / rho, bn2 = q[5 + n] * q[5 + n] / rho;
  double s = a2 + b2;
  double cf = sqrt(0.5 * (s + sqrt(s * s - 4.0 * a2 * bn2)));
  double c = fabs(vn) + cf;
  return c > P->c_h ? c : P->c_h;
}

/* Rusanov flux, Eq. eqn.rusanov */
static void rusanov(const phys *P, const double *qm, const double *qp, int n, double *out) {
  double fm[MAXV], fp[MAXV];
  flux(P, qm, n, fm);
  flux(P, qp, n, fp);
  double sm = max_speed(P, qm, n), sp = max_speed(P, qp, n);
  double s = sm > sp ? sm : sp;
  for (int v = 0; v < P->V; v++) out[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * s * (qp[v] - qm[v]);
}

/* Jacobian A[i][j] = dF_i/dQ_j of the MHD-GLM flux in direction n (the flux above, rationalised
 * units) with respect to the conserved variables Q = (rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi),
 * written out term by term from F with v = m / rho, p = (gamma - 1)(E - rho |v|^2 / 2 - |B|^2 / 2)
 * and p_t = p + |B|^2 / 2. */
static void mhd_jacobian(const phys *P, const double *q, int n, double A[9][9]) {
  const double g1 = P->gamma - 1.0, rho = q[0], E = q[4];
  double v[3], B[3], v2 = 0.0, B2 = 0.0, vB = 0.0;
  for (int a = 0; a < 3; a++) {
    v[a] = q[1 + a] / rho;
    B[a] = q[5 + a];
    v2 += v[a] * v[a];
    B2 += B[a] * B[a];
    vB += v[a] * B[a];
  }
  const double p = g1 * (E - 0.5 * rho * v2 - 0.5 * B2), pt = p + 0.5 * B2;
  /* dp/dQ and dp_t/dQ */
  double dp[9] = {0.5 * g1 * v2, -g1 * v[0], -g1 * v[1], -g1 * v[2], g1, -g1 * B[0], -g1 * B[1], -g1 * B[2], 0.0};
  double dpt[9];
  for (int j = 0; j < 9; j++) dpt[j] = dp[j];
  for (int a = 0; a < 3; a++) dpt[5 + a] += B[a];
  for (int i = 0; i < 9; i++)
    for (int j = 0; j < 9; j++) A[i][j] = 0.0;
  /* F_rho = m_n */
  A[0][1 + n] = 1.0;
  /* F_m_a = m_a v_n + p_t delta_an - B_a B_n; d(v_n)/d(rho) = -v_n / rho, d(v_n)/d(m_n) = 1 / rho */
  for (int a = 0; a < 3; a++) {
    A[1 + a][0] += -v[a] * v[n];
    A[1 + a][1 + a] += v[n];
    A[1 + a][1 + n] += v[a];
    if (a == n)
      for (int j = 0; j < 9; j++) A[1 + a][j] += dpt[j];
    A[1 + a][5 + a] -= B[n];
    A[1 + a][5 + n] -= B[a];
  }
  /* F_E = v_n (E + p_t) - B_n (v . B) */
  A[4][0] += -(E + pt) * v[n] / rho + B[n] * vB / rho;
  A[4][1 + n] += (E + pt) / rho;
  A[4][4] += v[n];
  for (int j = 0; j < 9; j++) A[4][j] += v[n] * dpt[j];
  A[4][5 + n] -= vB;
  for (int b = 0; b < 3; b++) {
    A[4][1 + b] -= B[n] * B[b] / rho;
    A[4][5 + b] -= B[n] * v[b];
  }
  /* F_B_a = v_n B_a - B_n v_a (a != n), F_B_n = psi */
  for (int a = 0; a < 3; a++) {
    if (a == n) continue;
    A[5 + a][0] += (B[n] * v[a] - B[a] * v[n]) / rho;
    A[5 + a][1 + n] += B[a] / rho;
    A[5 + a][1 + a] -= B[n] / rho;
    A[5 + a][5 + a] += v[n];
    A[5 + a][5 + n] -= v[a];
  }
  A[5 + n][8] = 1.0;
  /* F_psi = c_h^2 B_n */
  A[8][5 + n] = P->c_h * P->c_h;
}

/* |A| = A sign(A) for a real V x V matrix with real eigenvalues of modulus at most s (A
 * diagonalisable: |A| = R |Lambda| R^-1).  sign(A) by the Newton-Schulz iteration for the matrix
 * sign function, S <- S (3 I - S^2) / 2 from S = A / s: every eigenvalue x of S moves by the
 * scalar map x (3 - x^2) / 2, which takes x in (0, 1] to 1 and x in [-1, 0) to -1 (quadratically
 * near +-1, by a factor 1.5 per step while small) and keeps x = 0 at 0, as |A| needs.  80 steps
 * take every eigenvalue above 1e-14 s to its sign; below that its share of |A| is below 1e-14 s. */
static void abs_matrix(int V, const double *A, double s, double *out) {
  double S[MAXV * MAXV], T[MAXV * MAXV], U[MAXV * MAXV];
  for (int i = 0; i < V * V; i++) S[i] = A[i] / s;
  for (int it = 0; it < 80; it++) {
    for (int i = 0; i < V; i++)
      for (int j = 0; j < V; j++) {
        double t = 0.0;
        for (int k = 0; k < V; k++) t += S[i * V + k] * S[k * V + j];
        T[i * V + j] = (i == j ? 3.0 : 0.0) - t;
      }
    for (int i = 0; i < V; i++)
      for (int j = 0; j < V; j++) {
        double t = 0.0;
        for (int k = 0; k < V; k++) t += S[i * V + k] * T[k * V + j];
        U[i * V + j] = 0.5 * t;
      }
    memcpy(S, U, sizeof(double) * V * V);
  }
  for (int i = 0; i < V; i++)
    for (int j = 0; j < V; j++) {
      double t = 0.0;
      for (int k = 0; k < V; k++) t += A[i * V + k] * S[k * V + j];
      out[i * V + j] = t;
    }
}

/* |A(q)| applied to dq for the Euler flux in direction n: R |Lambda| L dq with the right and left
 * eigenvectors of the Jacobian written out (eigenvalues u_n - c, u_n (d times), u_n + c).  A state
 * with c^2 <= 0 has complex eigenvalues; there |A| dq is replaced by s dq with s the spectral
 * radius (reading).  Linear advection: |a_n| dq.  MHD-GLM: |A| of the Jacobian above by
 * abs_matrix, with s = max(|v_n| + c_f, c_h) its spectral radius (eigenvalues v_n, v_n +- c_a,
 * v_n +- c_s, v_n +- c_f and +-c_h); where gamma p / rho <= 0 the fast speed is not real and
 * |A| dq is replaced by s dq with s = max(|v_n| + sqrt(|B|^2 / rho), c_h) (reading). */
static void abs_jacobian_apply(const phys *P, const double *q, int n, const double *dq, double *out) {
  int V = P->V, d = P->d;
  if (P->pde == PDE_LINADV) { out[0] = fabs(P->adv[n]) * dq[0]; return; }
  if (P->pde == PDE_MHD) {
    const double rho = q[0], a2 = P->gamma * pressure(P, q) / rho;
    if (!(a2 > 0.0)) {
      double B2 = q[5] * q[5] + q[6] * q[6] + q[7] * q[7];
      double s = fabs(q[1 + n] / rho) + sqrt(B2 / rho);
      if (s < P->c_h) s = P->c_h;
      for (int v = 0; v < 9; v++) out[v] = s * dq[v];
      return;
    }
    double A[9][9], Aa[81];
    mhd_jacobian(P, q, n, A);
    abs_matrix(9, &A[0][0], max_speed(P, q, n), Aa);
    for (int i = 0; i < 9; i++) {
      double t = 0.0;
      for (int j = 0; j < 9; j++) t += Aa[i * 9 + j] * dq[j];
      out[i] = t;
    }
    return;
  }
  double rho = q[0], vel[3] = {0, 0, 0}, v2 = 0.0;
  for (int a = 0; a < d; a++) { vel[a] = q[1 + a] / rho; v2 += vel[a] * vel[a]; }
  double p = pressure(P, q), c2 = P->gamma * p / rho;
  if (!(c2 > 0.0)) {
    double s = max_speed(P, q, n);
    for (int v = 0; v < V; v++) out[v] = s * dq[v];
    return;
  }
  double c = sqrt(c2), H = (q[d + 1] + p) / rho, un = vel[n];
  double R[5][5] = {{0}}, L[5][5] = {{0}}, lam[5];
  /* columns: acoustic -, entropy, shear (transverse axes), acoustic + */
  R[0][0] = 1.0; R[d + 1][0] = H - un * c;
  R[0][1] = 1.0; R[d + 1][1] = 0.5 * v2;
  R[0][V - 1] = 1.0; R[d + 1][V - 1] = H + un * c;
  for (int a = 0; a < d; a++) {
    R[1 + a][0] = vel[a] - (a == n ? c : 0.0);
    R[1 + a][1] = vel[a];
    R[1 + a][V - 1] = vel[a] + (a == n ? c : 0.0);
  }
  double b1 = (P->gamma - 1.0) / c2, b2 = 0.5 * v2 * b1;
  L[0][0] = 0.5 * (b2 + un / c); L[0][d + 1] = 0.5 * b1;
  L[1][0] = 1.0 - b2; L[1][d + 1] = -b1;
  L[V - 1][0] = 0.5 * (b2 - un / c); L[V - 1][d + 1] = 0.5 * b1;
  for (int a = 0; a < d; a++) {
    L[0][1 + a] = 0.5 * (-b1 * vel[a] - (a == n ? 1.0 / c : 0.0));
    L[1][1 + a] = b1 * vel[a];
    L[V - 1][1 + a] = 0.5 * (-b1 * vel[a] + (a == n ? 1.0 / c : 0.0));
  }
  lam[0] = un - c; lam[1] = un; lam[V - 1] = un + c;
  int k = 2;
  for (int a = 0; a < d; a++) {
    if (a == n) continue;
    R[1 + a][k] = 1.0; R[d + 1][k] = vel[a];
    L[k][0] = -vel[a]; L[k][1 + a] = 1.0;
    lam[k] = un;
    k++;
  }
  double al[5];
  for (int i = 0; i < V; i++) {
    double t = 0.0;
    for (int j = 0; j < V; j++) t += L[i][j] * dq[j];
    al[i] = fabs(lam[i]) * t;
  }
  for (int i = 0; i < V; i++) {
    double t = 0.0;
    for (int j = 0; j < V; j++) t += R[i][j] * al[j];
    out[i] = t;
  }
}

/* Osher-Solomon flux of Dumbser and Toro, Eq. eqn.osher: the path integral of |A| along the
 * straight segment between the states by 3-point Gauss-Legendre quadrature (reading: the paper
 * asks for at least two points). */
static void osher(const phys *P, const double *qm, const double *qp, int n, double *out) {
  double fm[MAXV], fp[MAXV], dq[MAXV], acc[MAXV] = {0};
  flux(P, qm, n, fm);
  flux(P, qp, n, fp);
  for (int v = 0; v < P->V; v++) dq[v] = qp[v] - qm[v];
  double s[3], w[3];
  gauss_legendre01(3, s, w);
  for (int j = 0; j < 3; j++) {
    double q[MAXV] = {0}, t[MAXV];
    for (int v = 0; v < P->V; v++) q[v] = qm[v] + s[j] * dq[v];
    abs_jacobian_apply(P, q, n, dq, t);
    for (int v = 0; v < P->V; v++) acc[v] += w[j] * t[v];
  }
  for (int v = 0; v < P->V; v++) out[v] = 0.5 * (fm[v] + fp[v]) - 0.5 * acc[v];
}

static void numflux(const phys *P, const double *qm, const double *qp, int n, double *out) {
  if (P->flux == 1) osher(P, qm, qp, n, out);
  else rusanov(P, qm, qp, n, out);
}

static int physical(const phys *P, const double *q) {
  for (int v = 0; v < P->V; v++)
    if (!(q[v] == q[v])) return 0;
  if (P->pde == PDE_LINADV) return 1;
  return q[0] > 0.0 && pressure(P, q) > 0.0;
}

/* ===================================================================================
 * 4. Solver state: per-level dense grids (Sec. 3.1).  Level l has L = n*r^l cells per
 *    direction; a cell exists iff status != ST_NONE.  Children of (i,j,k) at level l are
 *    (r i + a, r j + b, r k + c) at level l+1; the mother is the integer quotient by r.
 * =================================================================================== */
typedef struct {
  int L[3];
  long n;
  int8_t *st;
  double *u;    /* V per dense cell */
  double *mem;  /* 2d*V per dense cell (memory variables, used on virtual children) */
  double *chi;  /* indicator per dense cell */
  int32_t *aid; /* active id per dense cell or -1 */
  int na;
  int32_t *alist;
  double *wh, *qh, *fl; /* per active: V*nsp, V*nst, 2d*V */
} olev;

typedef struct {
  orc_cfg c;
  phys P;
  tables T;
  int d, V, N, nsp, nst, P_iters;
  double dx0[3];
  olev lev[MAXL];
  double t;
  int ic;
  double icp[128];
  int icn;
  int64_t updates, level_updates[MAXL];
  int nthreads;
} osolver;

static long didx(const olev *L, int i, int j, int k) { return ((long)k * L->L[1] + j) * L->L[0] + i; }

/* map coordinate c in direction a at level lv through the boundary conditions.
 * Returns 1 if inside (possibly wrapped periodically), 0 if outside a non-periodic boundary;
 * *out is then the clamped coordinate (reading: transmissive ghost layers copy the adjacent
 * interior cell of the same level), or the mirror image beyond a reflective wall.  Beyond an
 * inflow face uget replaces the value by the inflow state. */
static int bcmap(const osolver *S, int lv, int a, int c, int *out) {
  int n = S->lev[lv].L[a];
  if (c >= 0 && c < n) { *out = c; return 1; }
  int bc = S->c.bc[2 * a + (c < 0 ? 0 : 1)];
  if (bc == BC_PERIODIC) { *out = ((c % n) + n) % n; return 1; }
  if (bc == BC_REFLECTIVE) { *out = c < 0 ? -1 - c : 2 * n - 1 - c; return 0; }  /* mirror image */
  *out = c < 0 ? 0 : n - 1;
  return 0;
}

/* is coordinate c of axis a beyond a reflective boundary? */
static int reflected(const osolver *S, int lv, int a, int c) {
  int n = S->lev[lv].L[a];
  if (c >= 0 && c < n) return 0;
  return S->c.bc[2 * a + (c < 0 ? 0 : 1)] == BC_REFLECTIVE;
}

static double dxl(const osolver *S, int lv, int a) {
  double dx = S->dx0[a];
  for (int l = 0; l < lv; l++) dx /= S->c.r;
  return dx;
}

static void lev_alloc(osolver *S, int lv) {
  olev *L = &S->lev[lv];
  int rr = 1;
  for (int l = 0; l < lv; l++) rr *= S->c.r;
  L->L[0] = S->c.nx * rr;
  L->L[1] = S->c.ny * rr;
  L->L[2] = S->d == 3 ? S->c.nz * rr : 1;
  L->n = (long)L->L[0] * L->L[1] * L->L[2];
  L->st = malloc(L->n);
  memset(L->st, ST_NONE, L->n);
  L->u = calloc((size_t)L->n * S->V, sizeof(double));
  L->mem = calloc((size_t)L->n * 2 * S->d * S->V, sizeof(double));
  L->chi = calloc((size_t)L->n, sizeof(double));
  L->aid = malloc(sizeof(int32_t) * L->n);
  for (long i = 0; i < L->n; i++) L->aid[i] = -1;
  L->na = 0;
  L->alist = NULL; L->wh = L->qh = L->fl = NULL;
}

/* rebuild the active lists (canonical order: k, j, i ascending) */
static void build_active(osolver *S) {
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    int na = 0;
    for (long c = 0; c < L->n; c++) {
      L->aid[c] = -1;
      if (L->st[c] == 0) L->aid[c] = na++;
    }
    free(L->alist); free(L->wh); free(L->qh); free(L->fl);
    L->na = na;
    L->alist = malloc(sizeof(int32_t) * (na + 1));
    for (long c = 0; c < L->n; c++)
      if (L->st[c] == 0) L->alist[L->aid[c]] = (int32_t)c;
    L->wh = calloc((size_t)(na + 1) * S->V * S->nsp, sizeof(double));
    L->qh = calloc((size_t)(na + 1) * S->V * S->nst, sizeof(double));
    L->fl = calloc((size_t)(na + 1) * 2 * S->d * S->V, sizeof(double));
  }
}

static void coords(const olev *L, long c, int *ijk) {
  ijk[0] = (int)(c % L->L[0]);
  ijk[1] = (int)((c / L->L[0]) % L->L[1]);
  ijk[2] = (int)(c / ((long)L->L[0] * L->L[1]));
}

/* ===================================================================================
 * 5. Initial conditions (Sec. 4): point values, then cell averages by (M+1)^d-point
 *    tensor Gauss quadrature (reading: the same rule for smooth and discontinuous data).
 * =================================================================================== */
static void prim2cons(const phys *P, const double *w, double *q) {
  /* primitive layout: Euler (rho, v_1..v_d, p); MHD (rho, vx, vy, vz, p, Bx, By, Bz, psi) */
  if (P->pde == PDE_LINADV) { q[0] = w[0]; return; }
  double g = P->gamma;
  if (P->pde == PDE_EULER) {
    int d = P->d;
    double rho = w[0], ke = 0.0;
    q[0] = rho;
    for (int a = 0; a < d; a++) { q[1 + a] = rho * w[1 + a]; ke += w[1 + a] * w[1 + a]; }
    q[d + 1] = w[d + 1] / (g - 1.0) + 0.5 * rho * ke;
    return;
  }
  double rho = w[0];
  double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
  double B2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
  q[0] = rho; q[1] = rho * w[1]; q[2] = rho * w[2]; q[3] = rho * w[3];
  q[4] = w[4] / (g - 1.0) + 0.5 * rho * v2 + 0.5 * B2;
  q[5] = w[5]; q[6] = w[6]; q[7] = w[7]; q[8] = w[8];
}

/* Primitive state of an IC at point x.  Parameter layouts (params[]):
 *  IC_CONST:     primitive state (V values)
 *  IC_VORTEX:    eps, xc, yc, background rho, u, v, p (isentropic vortex, Sec. 4.1)
 *  IC_EXPLOSION: R, rho_in, p_in, rho_out, p_out (explosion, Sec. 4.1)
 *  IC_OT:        (none) Orszag-Tang data of Sec. 4.2 in rationalised units
 *  IC_RP4:       x0, y0, then (rho, u, v, p) for quadrants 1..4 (x>x0,y>y0; x<x0,y>y0;
 *                x<x0,y<y0; x>x0,y<y0)
 *  IC_FOURIER:   base primitive state (V values), then nmodes, then per mode
 *                (var, kx, ky, kz, amp, phase): w_var += amp*sin(2 pi k.(x-lo)/(hi-lo) + phase)
 */
static void ic_prim(const osolver *S, const double *x, double *w) {
  const phys *P = &S->P;
  const double *p = S->icp;
  int V = S->V, d = S->d;
  for (int v = 0; v < MAXV; v++) w[v] = 0.0;
  switch (S->ic) {
  case IC_CONST:
    for (int v = 0; v < V; v++) w[v] = p[v];
    break;
  case IC_VORTEX: {
    double eps = p[0], dxv = x[0] - p[1], dyv = x[1] - p[2], r2 = dxv * dxv + dyv * dyv;
    double g = P->gamma;
    double dT = -eps * eps * (g - 1.0) / (8.0 * g * M_PI * M_PI) * exp(1.0 - r2);
    double e = eps / (2.0 * M_PI) * exp(0.5 * (1.0 - r2));
    w[0] = p[3] * pow(1.0 + dT, 1.0 / (g - 1.0));
    w[1] = p[4] - dyv * e;
    w[2] = p[5] + dxv * e;
    w[d + 1] = p[6] * pow(1.0 + dT, g / (g - 1.0));
    break;
  }
  case IC_EXPLOSION: {
    double r2 = 0.0;
    for (int a = 0; a < d; a++) r2 += x[a] * x[a];
    int in = sqrt(r2) <= p[0];
    w[0] = in ? p[1] : p[3];
    if (P->pde == PDE_EULER) w[d + 1] = in ? p[2] : p[4];
    else w[4] = in ? p[2] : p[4];
    break;
  }
  case IC_OT: {
    double g = P->gamma;
    w[0] = g * g; w[1] = -sin(x[1]); w[2] = sin(x[0]); w[3] = 0.0; w[4] = g;
    w[5] = -sin(x[1]); w[6] = sin(2.0 * x[0]); w[7] = 0.0; w[8] = 0.0;
    break;
  }
  case IC_RP4: {
    int qd;
    if (x[0] > p[0]) qd = (x[1] > p[1]) ? 0 : 3;
    else qd = (x[1] > p[1]) ? 1 : 2;
    const double *s = p + 2 + 4 * qd;
    w[0] = s[0]; w[1] = s[1]; w[2] = s[2]; w[d + 1] = s[3];
    break;
  }
  case IC_FOURIER: {
    for (int v = 0; v < V; v++) w[v] = p[v];
    int nm = (int)p[V];
    for (int m = 0; m < nm; m++) {
      const double *md = p + V + 1 + 6 * m;
      int var = (int)md[0];
      double ph = md[5];
      for (int a = 0; a < d; a++) ph += 2.0 * M_PI * md[1 + a] * (x[a] - S->c.lo[a]) / (S->c.hi[a] - S->c.lo[a]);
      w[var] += md[4] * sin(ph);
    }
    break;
  }
  }
}

/* cell average of the IC over cell (ijk) of level lv */
static void ic_average(const osolver *S, int lv, const int *ijk, double *out) {
  int N = S->N, d = S->d, V = S->V;
  double acc[MAXV] = {0};
  int nq = 1;
  for (int a = 0; a < d; a++) nq *= N;
  for (int g = 0; g < nq; g++) {
    int t = g;
    double x[3] = {0, 0, 0}, wt = 1.0;
    for (int a = 0; a < d; a++) {
      int gi = t % N; t /= N;
      double h = dxl(S, lv, a);
      x[a] = S->c.lo[a] + (ijk[a] + S->T.x[gi]) * h;
      wt *= S->T.w[gi];
    }
    double w[MAXV], q[MAXV];
    ic_prim(S, x, w);
    prim2cons(&S->P, w, q);
    for (int v = 0; v < V; v++) acc[v] += wt * q[v];
  }
  for (int v = 0; v < V; v++) out[v] = acc[v];
}

/* ===================================================================================
 * 6. WENO reconstruction, dimension by dimension (Sec. 2.2)
 * =================================================================================== */

/* One-dimensional WENO: v[0..2M] are the values at offsets -M..M (cell averages, or
 * degrees of freedom of a previous sweep); out[0..M] the nodal coefficients of the
 * reconstruction polynomial (Eqs. eqn.rec.x, eqn.weno, eqn.omegas, eqn.sigmas).
 * Reading: the stencil polynomials and the oscillation indicators are evaluated on the
 * differences v - v[M] from the cell's own value.  This is exact (every stencil reproduces
 * constants, and Sigma annihilates them because it only involves derivatives), and it keeps
 * the rounding of a large constant part out of sigma, which the exponent r = 8 would
 * otherwise amplify into the weights. */
static void weno1d(const tables *T, const double *v, double *out) {
  int N = T->N, M = T->M;
  double ws[4][MAXN], om[4], sum = 0.0, c = v[M];
  for (int s = 0; s < T->Ns; s++) {
    for (int p = 0; p < N; p++) {
      double a = 0.0;
      for (int e = 0; e < N; e++) a += T->Ainv[s][p][e] * (v[M - T->SL[s] + e] - c);
      ws[s][p] = a;
    }
    double sig = 0.0;
    for (int p = 0; p < N; p++)
      for (int m = 0; m < N; m++) sig += T->Sig[p][m] * ws[s][p] * ws[s][m];
    /* (sigma + eps)^r with r = 8 by three squarings (reading: eps = 1e-14, r = 8) */
    double x = sig + 1e-14, x2 = x * x, x4 = x2 * x2, x8 = x4 * x4;
    om[s] = T->lam[s] / x8;
    sum += om[s];
  }
  for (int p = 0; p < N; p++) out[p] = 0.0;
  for (int s = 0; s < T->Ns; s++) {
    double w = om[s] / sum;
    for (int p = 0; p < N; p++) out[p] += w * ws[s][p];
  }
  for (int p = 0; p < N; p++) out[p] += c;
}

/* averages at level lv of the cell at integer coordinates c[], through the BCs: periodic wrap,
 * transmissive clamp, reflective mirror image with the normal momentum negated (reading: a
 * reflecting wall is the mirror image of the interior, for the Euler equations) */
/* is coordinate c of axis a beyond an inflow boundary? */
static int beyond_inflow(const osolver *S, int lv, int a, int c) {
  int n = S->lev[lv].L[a];
  if (c >= 0 && c < n) return 0;
  return S->c.bc[2 * a + (c < 0 ? 0 : 1)] == BC_INFLOW;
}

/* average of cell c of level lv through the boundary conditions (reading: a ghost cell beyond
 * an inflow face, in any direction, holds the inflow state) */
static void uget(const osolver *S, int lv, const int *c, double *out) {
  const olev *L = &S->lev[lv];
  for (int a = 0; a < S->d; a++)
    if (beyond_inflow(S, lv, a, c[a])) {
      for (int v = 0; v < S->V; v++) out[v] = S->c.inflow[v];
      return;
    }
  int m[3] = {0, 0, 0};
  for (int a = 0; a < S->d; a++) bcmap(S, lv, a, c[a], &m[a]);
  const double *u = L->u + didx(L, m[0], m[1], m[2]) * S->V;
  for (int v = 0; v < S->V; v++) out[v] = u[v];
  if (S->P.pde == PDE_EULER)
    for (int a = 0; a < S->d; a++)
      if (reflected(S, lv, a, c[a])) out[1 + a] = -out[1 + a];
}

/* WENO polynomial of cell ijk at level lv: wh[v*nsp + (p + N q + N^2 r)] */
static void weno_cell(const osolver *S, int lv, const int *ijk, double *wh) {
  int N = S->N, M = S->T.M, d = S->d, V = S->V, W = 2 * M + 1;
  if (d == 2) {
    /* x sweep on every row of the box, then y sweep on every x degree of freedom */
    double wx[2 * MAXN + 1][MAXV][MAXN];
    for (int e = -M; e <= M; e++) {
      for (int v = 0; v < V; v++) {
        double line[2 * MAXN + 1];
        for (int f = -M; f <= M; f++) {
          int c[3] = {ijk[0] + f, ijk[1] + e, 0};
          double tmp[MAXV];
          uget(S, lv, c, tmp);
          line[f + M] = tmp[v];
        }
        weno1d(&S->T, line, wx[e + M][v]);
      }
    }
    for (int v = 0; v < V; v++)
      for (int p = 0; p < N; p++) {
        double line[2 * MAXN + 1], o[MAXN];
        for (int e = 0; e < W; e++) line[e] = wx[e][v][p];
        weno1d(&S->T, line, o);
        for (int q = 0; q < N; q++) wh[v * S->nsp + p + N * q] = o[q];
      }
    return;
  }
  /* d == 3: x sweep on every (y,z) line of the box, y sweep per x dof, z sweep per (x,y) dof */
  static __thread double wx[2 * MAXN + 1][2 * MAXN + 1][MAXV][MAXN];
  static __thread double wxy[2 * MAXN + 1][MAXV][MAXN][MAXN];
  for (int ez = -M; ez <= M; ez++)
    for (int ey = -M; ey <= M; ey++)
      for (int v = 0; v < V; v++) {
        double line[2 * MAXN + 1];
        for (int f = -M; f <= M; f++) {
          int c[3] = {ijk[0] + f, ijk[1] + ey, ijk[2] + ez};
          double tmp[MAXV];
          uget(S, lv, c, tmp);
          line[f + M] = tmp[v];
        }
        weno1d(&S->T, line, wx[ez + M][ey + M][v]);
      }
  for (int ez = 0; ez < W; ez++)
    for (int v = 0; v < V; v++)
      for (int p = 0; p < N; p++) {
        double line[2 * MAXN + 1], o[MAXN];
        for (int ey = 0; ey < W; ey++) line[ey] = wx[ez][ey][v][p];
        weno1d(&S->T, line, o);
        for (int q = 0; q < N; q++) wxy[ez][v][p][q] = o[q];
      }
  for (int v = 0; v < V; v++)
    for (int p = 0; p < N; p++)
      for (int q = 0; q < N; q++) {
        double line[2 * MAXN + 1], o[MAXN];
        for (int ez = 0; ez < W; ez++) line[ez] = wxy[ez][v][p][q];
        weno1d(&S->T, line, o);
        for (int r = 0; r < N; r++) wh[v * S->nsp + p + N * q + N * N * r] = o[r];
      }
}

/* ===================================================================================
 * 7. Local space-time DG predictor (Sec. 2.3): Picard iteration of Eq. eqn.stdg.final,
 *    K1 q^{k+1} = F0 w - sum_a K_a f*_a(q^k), with f*_a = dt/dx_a f_a (Eq. eqn.pde.ref),
 *    source zero.  Reading: initial guess q^0 = w (constant in time), a fixed number
 *    P of iterations (default M+1).
 * =================================================================================== */
static void predictor(const osolver *S, const double *wh, double dt, const double *dx, double *qh) {
  int nsp = S->nsp, nst = S->nst, V = S->V, d = S->d;
  double *rhs0 = malloc(sizeof(double) * V * nst);
  double *fs = malloc(sizeof(double) * 3 * V * nst);
  double *rhs = malloc(sizeof(double) * nst);
  for (int v = 0; v < V; v++)
    for (int ip = 0; ip < nst; ip++) qh[v * nst + ip] = wh[v * nsp + ip % nsp];
  for (int v = 0; v < V; v++)
    for (int iq = 0; iq < nst; iq++) {
      double s = 0.0;
      for (int im = 0; im < nsp; im++) s += S->T.F0[iq * nsp + im] * wh[v * nsp + im];
      rhs0[v * nst + iq] = s;
    }
  for (int it = 0; it < S->P_iters; it++) {
    for (int ip = 0; ip < nst; ip++) {
      double q[MAXV], f[MAXV];
      for (int v = 0; v < V; v++) q[v] = qh[v * nst + ip];
      for (int a = 0; a < d; a++) {
        flux(&S->P, q, a, f);
        for (int v = 0; v < V; v++) fs[(a * V + v) * nst + ip] = dt / dx[a] * f[v];
      }
    }
    for (int v = 0; v < V; v++) {
      for (int iq = 0; iq < nst; iq++) {
        double s = rhs0[v * nst + iq];
        for (int a = 0; a < d; a++)
          for (int ip = 0; ip < nst; ip++) s -= S->T.Kd[a][iq * nst + ip] * fs[(a * V + v) * nst + ip];
        rhs[iq] = s;
      }
      for (int iq = 0; iq < nst; iq++) {
        double s = 0.0;
        for (int ip = 0; ip < nst; ip++) s += S->T.K1inv[iq * nst + ip] * rhs[ip];
        qh[v * nst + iq] = s;
      }
    }
  }
  free(rhs0); free(fs); free(rhs);
}

/* evaluate the space-time polynomial q_h (nodal dofs qh) at reference point (xi[], tau) */
static void eval_st(const osolver *S, const double *qh, const double *xi, double tau, double *out) {
  int N = S->N, d = S->d, V = S->V, nst = S->nst;
  double bx[3][MAXN], bt[MAXN];
  for (int a = 0; a < d; a++)
    for (int l = 0; l < N; l++) bx[a][l] = psi_val(&S->T, l, xi[a]);
  for (int l = 0; l < N; l++) bt[l] = psi_val(&S->T, l, tau);
  for (int v = 0; v < V; v++) out[v] = 0.0;
  for (int ip = 0; ip < nst; ip++) {
    int t = ip;
    double th = 1.0;
    for (int a = 0; a < d; a++) { th *= bx[a][t % N]; t /= N; }
    th *= bt[t];
    for (int v = 0; v < V; v++) out[v] += th * qh[v * nst + ip];
  }
}

/* evaluate the spatial polynomial w_h at reference point xi[] */
static void eval_sp(const osolver *S, const double *wh, const double *xi, double *out) {
  int N = S->N, d = S->d, V = S->V, nsp = S->nsp;
  double bx[3][MAXN];
  for (int a = 0; a < d; a++)
    for (int l = 0; l < N; l++) bx[a][l] = psi_val(&S->T, l, xi[a]);
  for (int v = 0; v < V; v++) out[v] = 0.0;
  for (int ip = 0; ip < nsp; ip++) {
    int t = ip;
    double th = 1.0;
    for (int a = 0; a < d; a++) { th *= bx[a][t % N]; t /= N; }
    for (int v = 0; v < V; v++) out[v] += th * wh[v * nsp + ip];
  }
}

/* ===================================================================================
 * 8. Ghost values: projection (Sec. 3.1.3) and averaging (Eq. eqn.average)
 * =================================================================================== */

/* child-box average of the mother's space-time polynomial at mother time tau:
 * the child occupies [ch_a/r, (ch_a+1)/r] of the mother's reference interval in each
 * direction; N-point Gauss rule per direction (exact for degree M). */
static void project_st(const osolver *S, const double *qh_m, const int *ch, double tau, double *out) {
  int N = S->N, d = S->d, V = S->V, r = S->c.r;
  int nq = 1;
  for (int a = 0; a < d; a++) nq *= N;
  for (int v = 0; v < V; v++) out[v] = 0.0;
  for (int g = 0; g < nq; g++) {
    int t = g;
    double xi[3] = {0, 0, 0}, wt = 1.0, q[MAXV];
    for (int a = 0; a < d; a++) {
      int gi = t % N; t /= N;
      xi[a] = (ch[a] + S->T.x[gi]) / r;
      wt *= S->T.w[gi];
    }
    eval_st(S, qh_m, xi, tau, q);
    for (int v = 0; v < V; v++) out[v] += wt * q[v];
  }
}

/* child-box average of the mother's spatial WENO polynomial (reading: new children of a
 * regrid take this value, which is conservative) */
static void project_sp(const osolver *S, const double *wh_m, const int *ch, double *out) {
  int N = S->N, d = S->d, V = S->V, r = S->c.r;
  int nq = 1;
  for (int a = 0; a < d; a++) nq *= N;
  for (int v = 0; v < V; v++) out[v] = 0.0;
  for (int g = 0; g < nq; g++) {
    int t = g;
    double xi[3] = {0, 0, 0}, wt = 1.0, q[MAXV];
    for (int a = 0; a < d; a++) {
      int gi = t % N; t /= N;
      xi[a] = (ch[a] + S->T.x[gi]) / r;
      wt *= S->T.w[gi];
    }
    eval_sp(S, wh_m, xi, q);
    for (int v = 0; v < V; v++) out[v] += wt * q[v];
  }
}

/* mother index and child offsets of cell ijk at level lv >= 1 */
static long mother_of(const osolver *S, int lv, const int *ijk, int *ch) {
  int r = S->c.r, m[3] = {0, 0, 0};
  for (int a = 0; a < 3; a++) { m[a] = ijk[a] / r; ch[a] = ijk[a] - r * m[a]; }
  if (S->d == 2) { m[2] = 0; ch[2] = 0; }
  return didx(&S->lev[lv - 1], m[0], m[1], m[2]);
}

/* project all virtual children (status 1) of level lv from their active mothers' q_h at
 * mother time tau (Sec. 3.1.3) */
static void project_level(osolver *S, int lv, double tau) {
  olev *L = &S->lev[lv], *Lm = &S->lev[lv - 1];
#pragma omp parallel for schedule(dynamic, 64) num_threads(S->nthreads)
  for (long c = 0; c < L->n; c++) {
    if (L->st[c] != 1) continue;
    int ijk[3], ch[3];
    coords(L, c, ijk);
    long m = mother_of(S, lv, ijk, ch);
    int ma = Lm->aid[m];
    project_st(S, Lm->qh + (size_t)ma * S->V * S->nst, ch, tau, L->u + c * S->V);
  }
}

/* average level lv+1 into the virtual mothers (status -1) of level lv (Eq. eqn.average);
 * children summed in canonical order (k, j, i) */
static void average_into(osolver *S, int lv) {
  olev *L = &S->lev[lv], *Lc = &S->lev[lv + 1];
  int r = S->c.r, d = S->d, V = S->V, rz = d == 3 ? r : 1;
  double rd = 1.0;
  for (int a = 0; a < d; a++) rd *= r;
  for (long c = 0; c < L->n; c++) {
    if (L->st[c] != -1) continue;
    int ijk[3];
    coords(L, c, ijk);
    double s[MAXV] = {0};
    for (int kk = 0; kk < rz; kk++)
      for (int jj = 0; jj < r; jj++)
        for (int ii = 0; ii < r; ii++) {
          long cc = didx(Lc, r * ijk[0] + ii, r * ijk[1] + jj, d == 3 ? r * ijk[2] + kk : 0);
          for (int v = 0; v < V; v++) s[v] += Lc->u[cc * V + v];
        }
    for (int v = 0; v < V; v++) L->u[c * V + v] = s[v] / rd;
  }
}

static void average_all(osolver *S) {
  for (int lv = S->c.lmax - 1; lv >= 0; lv--) average_into(S, lv);
}

/* ===================================================================================
 * 9. Face fluxes and the finite volume update (Eqs. eq:finite_vol, flux:F..flux:H,
 *    eqn.rusanov), with local time stepping (Eq. eqn.update.criterion) and memory
 *    variables at coarse/fine faces (Eq. eqn.memory.sum).
 * =================================================================================== */

/* face-averaged numerical flux on face (a, side) of active cell ijk of level lv, during
 * the sub-step sub (0..r-1) of the mother level's step.  Writes F[V].  Fine-side faces
 * at a virtual neighbour add their space-time integral to that neighbour's memory
 * variable (when addmem). */
static void face_flux(osolver *S, int lv, const int *ijk, int ia, int a, int side, int sub, double dt,
                      double *F, int addmem) {
  int N = S->N, d = S->d, V = S->V, r = S->c.r, nst = S->nst;
  olev *L = &S->lev[lv];
  const double *qA = L->qh + (size_t)ia * V * nst;
  int nb[3] = {ijk[0], ijk[1], ijk[2]}, nbm[3] = {ijk[0], ijk[1], ijk[2]};
  nb[a] += side ? 1 : -1;
  int inside = bcmap(S, lv, a, nb[a], &nbm[a]);
  for (int v = 0; v < V; v++) F[v] = 0.0;
  /* transverse directions */
  int tdir[2], nt = 0;
  for (int b = 0; b < d; b++)
    if (b != a) tdir[nt++] = b;
  int npt = 1;
  for (int b = 0; b < nt; b++) npt *= N;
  if (!inside && S->c.bc[2 * a + side] == BC_INFLOW) {
    /* inflow face: the outer state is the prescribed inflow state (reading) */
    const double *qi = S->c.inflow;
    for (int g = 0; g < npt * N; g++) {
      int t = g;
      double xi[3], wt = 1.0, q[MAXV], f[MAXV];
      xi[a] = side ? 1.0 : 0.0;
      for (int b = 0; b < nt; b++) { int gi = t % N; t /= N; xi[tdir[b]] = S->T.x[gi]; wt *= S->T.w[gi]; }
      int gs = t;
      wt *= S->T.w[gs];
      eval_st(S, qA, xi, S->T.x[gs], q);
      if (side) numflux(&S->P, q, qi, a, f);
      else numflux(&S->P, qi, q, a, f);
      for (int v = 0; v < V; v++) F[v] += wt * f[v];
    }
    return;
  }
  if (!inside && S->c.bc[2 * a + side] == BC_REFLECTIVE) {
    /* reflecting wall: the outer state is the mirror image of the inner trace */
    for (int g = 0; g < npt * N; g++) {
      int t = g;
      double xi[3], wt = 1.0, q[MAXV], qm[MAXV], f[MAXV];
      xi[a] = side ? 1.0 : 0.0;
      for (int b = 0; b < nt; b++) { int gi = t % N; t /= N; xi[tdir[b]] = S->T.x[gi]; wt *= S->T.w[gi]; }
      int gs = t;
      wt *= S->T.w[gs];
      eval_st(S, qA, xi, S->T.x[gs], q);
      for (int v = 0; v < V; v++) qm[v] = q[v];
      if (S->P.pde == PDE_EULER) qm[1 + a] = -qm[1 + a];
      if (side) numflux(&S->P, q, qm, a, f);
      else numflux(&S->P, qm, q, a, f);
      for (int v = 0; v < V; v++) F[v] += wt * f[v];
    }
    return;
  }
  if (!inside) {
    /* transmissive boundary face: q+ = q- (reading), Rusanov reduces to f(q-) */
    for (int g = 0; g < npt * N; g++) {
      int t = g;
      double xi[3], wt = 1.0, q[MAXV], f[MAXV];
      xi[a] = side ? 1.0 : 0.0;
      for (int b = 0; b < nt; b++) { int gi = t % N; t /= N; xi[tdir[b]] = S->T.x[gi]; wt *= S->T.w[gi]; }
      int gs = t;
      wt *= S->T.w[gs];
      eval_st(S, qA, xi, S->T.x[gs], q);
      numflux(&S->P, q, q, a, f);
      for (int v = 0; v < V; v++) F[v] += wt * f[v];
    }
    return;
  }
  long nc = didx(L, nbm[0], nbm[1], nbm[2]);
  int8_t nst_ = L->st[nc];
  if (nst_ == 0) {
    /* same-level face */
    const double *qB = L->qh + (size_t)L->aid[nc] * V * nst;
    for (int g = 0; g < npt * N; g++) {
      int t = g;
      double xiA[3], xiB[3], wt = 1.0, qa[MAXV], qb[MAXV], f[MAXV];
      xiA[a] = side ? 1.0 : 0.0;
      xiB[a] = side ? 0.0 : 1.0;
      for (int b = 0; b < nt; b++) {
        int gi = t % N; t /= N;
        xiA[tdir[b]] = xiB[tdir[b]] = S->T.x[gi];
        wt *= S->T.w[gi];
      }
      int gs = t;
      wt *= S->T.w[gs];
      eval_st(S, qA, xiA, S->T.x[gs], qa);
      eval_st(S, qB, xiB, S->T.x[gs], qb);
      if (side) numflux(&S->P, qa, qb, a, f);
      else numflux(&S->P, qb, qa, a, f);
      for (int v = 0; v < V; v++) F[v] += wt * f[v];
    }
    return;
  }
  if (nst_ == 1) {
    /* fine side of a coarse/fine face: the neighbour is a virtual child of an active
     * coarse cell C; q_h of C evaluated at this cell's face points and sub-step
     * (reading: the coarse polynomial is evaluated directly at the fine points). */
    int ch[3];
    long mc = mother_of(S, lv, nbm, ch);
    olev *Lm = &S->lev[lv - 1];
    const double *qC = Lm->qh + (size_t)Lm->aid[mc] * V * nst;
    int cm[3];
    coords(Lm, mc, cm);
    for (int g = 0; g < npt * N; g++) {
      int t = g;
      double xiA[3], xiC[3], wt = 1.0, qa[MAXV], qc[MAXV], f[MAXV];
      xiA[a] = side ? 1.0 : 0.0;
      xiC[a] = side ? 0.0 : 1.0;
      for (int b = 0; b < nt; b++) {
        int gi = t % N; t /= N;
        int tb = tdir[b];
        xiA[tb] = S->T.x[gi];
        xiC[tb] = (ijk[tb] - r * cm[tb] + S->T.x[gi]) / r;
        wt *= S->T.w[gi];
      }
      int gs = t;
      wt *= S->T.w[gs];
      eval_st(S, qA, xiA, S->T.x[gs], qa);
      eval_st(S, qC, xiC, (sub + S->T.x[gs]) / r, qc);
      if (side) numflux(&S->P, qa, qc, a, f);
      else numflux(&S->P, qc, qa, a, f);
      for (int v = 0; v < V; v++) F[v] += wt * f[v];
    }
    if (addmem) {
      double dA = 1.0;
      for (int b = 0; b < nt; b++) dA *= dxl(S, lv, tdir[b]);
      /* the neighbour's face that touches this cell: its low face if side=+, else high */
      double *m = L->mem + ((size_t)nc * 2 * d + 2 * a + (side ? 0 : 1)) * V;
      for (int v = 0; v < V; v++) m[v] += F[v] * dt * dA;
    }
    return;
  }
  /* nst_ == -1: coarse side; the flux is the sum of the memory variables of this cell's
   * virtual children along the face, normalised by dt_l * dA_l (Eq. eqn.memory.sum). */
  olev *Lc = &S->lev[lv + 1];
  double dA = 1.0;
  for (int b = 0; b < nt; b++) dA *= dxl(S, lv, tdir[b]);
  int rz = d == 3 ? r : 1;
  double s[MAXV] = {0};
  for (int kk = 0; kk < rz; kk++)
    for (int jj = 0; jj < r; jj++)
      for (int ii = 0; ii < r; ii++) {
        int o[3] = {ii, jj, kk};
        if (o[a] != (side ? r - 1 : 0)) continue;
        long cc = didx(Lc, r * ijk[0] + ii, r * ijk[1] + jj, d == 3 ? r * ijk[2] + kk : 0);
        double *m = Lc->mem + ((size_t)cc * 2 * d + 2 * a + side) * V;
        for (int v = 0; v < V; v++) s[v] += m[v];
        if (addmem)
          for (int v = 0; v < V; v++) m[v] = 0.0;
      }
  for (int v = 0; v < V; v++) F[v] = s[v] / (dt * dA);
}

static int g_nonphysical;

/* one step of level lv by its own dt (dt0 / r^lv); sub = index of this sub-step within
 * the mother level's step.  Recursion order = update criterion: coarse reconstruction and
 * prediction first, then r sub-steps of the finer level, then the coarse update. */
static void advance(osolver *S, int lv, int sub, double dt0) {
  olev *L = &S->lev[lv];
  int V = S->V, d = S->d;
  double dt = dt0;
  for (int l = 0; l < lv; l++) dt /= S->c.r;
  double dx[3] = {dxl(S, lv, 0), dxl(S, lv, 1), d == 3 ? dxl(S, lv, 2) : 1.0};
  /* 1. ghost values: virtual children projected from the mothers' q_h at tau = sub/r */
  if (lv >= 1) project_level(S, lv, (double)sub / S->c.r);
  /* 2. reconstruction and local predictor on every active cell of this level */
#pragma omp parallel for schedule(dynamic, 16) num_threads(S->nthreads)
  for (int ia = 0; ia < L->na; ia++) {
    int ijk[3];
    coords(L, L->alist[ia], ijk);
    double *wh = L->wh + (size_t)ia * V * S->nsp;
    weno_cell(S, lv, ijk, wh);
    predictor(S, wh, dt, dx, L->qh + (size_t)ia * V * S->nst);
  }
  /* 3. finer level: r sub-steps */
  if (lv < S->c.lmax)
    for (int k = 0; k < S->c.r; k++) advance(S, lv + 1, k, dt0);
  /* 4. fluxes of every face of every active cell (each cell computes its own faces) */
#pragma omp parallel for schedule(dynamic, 16) num_threads(S->nthreads)
  for (int ia = 0; ia < L->na; ia++) {
    int ijk[3];
    coords(L, L->alist[ia], ijk);
    for (int a = 0; a < d; a++)
      for (int side = 0; side < 2; side++)
        face_flux(S, lv, ijk, ia, a, side, sub, dt, L->fl + ((size_t)ia * 2 * d + 2 * a + side) * V, 1);
  }
  /* 5. update (Eq. eq:finite_vol, source zero) */
  int bad = 0;
  for (int ia = 0; ia < L->na; ia++) {
    double *u = L->u + (size_t)L->alist[ia] * V;
    const double *F = L->fl + (size_t)ia * 2 * d * V;
    for (int a = 0; a < d; a++)
      for (int v = 0; v < V; v++) u[v] -= dt / dx[a] * (F[(2 * a + 1) * V + v] - F[(2 * a) * V + v]);
    if (!physical(&S->P, u)) bad = 1;
  }
  if (bad) g_nonphysical = 1;
  S->updates += L->na;
  S->level_updates[lv] += L->na;
  /* 6. at the end of the mother's step, average this level into the virtual mothers */
  if (lv >= 1 && sub == S->c.r - 1) average_into(S, lv - 1);
}

/* stable dt_0: min over active cells of r^l * CFL / sum_a(s_a / dx_a) (reading) */
static double compute_dt(const osolver *S) {
  double best = 1e300;
  double rl = 1.0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    const olev *L = &S->lev[lv];
    double dx[3] = {dxl(S, lv, 0), dxl(S, lv, 1), S->d == 3 ? dxl(S, lv, 2) : 1.0};
    for (int ia = 0; ia < L->na; ia++) {
      const double *u = L->u + (size_t)L->alist[ia] * S->V;
      double den = 0.0;
      for (int a = 0; a < S->d; a++) den += max_speed(&S->P, u, a) / dx[a];
      double dt = rl * S->c.cfl / den;
      if (dt < best) best = dt;
    }
    rl *= S->c.r;
  }
  return best;
}

/* ===================================================================================
 * 10. Refinement indicator (Eq. eqn.indicator) and regrid (rules 1-7 of Sec. 3.1)
 * =================================================================================== */

/* Loehner indicator of cell ijk at level lv, Phi = rho (first conserved variable), with
 * undivided differences on the 3^d same-level box (reading of the garbled formula):
 *   num = sum_{k,l} D2_kl^2
 *   den = sum_{k,l} (G_kl + eps * A_kl)^2
 * k = l: D2 = P+ - 2 P0 + P-, G = |P+ - P0| + |P0 - P-|, A = |P+| + 2|P0| + |P-|
 * k != l: D2 = (P++ - P+- - P-+ + P--)/4, G = (|P++ - P-+| + |P+- - P--|)/4,
 *         A = (|P++| + |P+-| + |P-+| + |P--|)/4   (P_{s_k s_l}: offsets s_k e_k + s_l e_l)
 * chi = sqrt(num / den). */
static double phi_at(const osolver *S, int lv, const int *ijk, int a, int sa, int b, int sb) {
  int c[3] = {ijk[0], ijk[1], ijk[2]};
  c[a] += sa;
  c[b] += sb;
  double tmp[MAXV];
  uget(S, lv, c, tmp);
  return tmp[0];
}
static double indicator(const osolver *S, int lv, const int *ijk) {
  int d = S->d;
  double eps = S->c.eps_ind, num = 0.0, den = 0.0;
  double P0 = phi_at(S, lv, ijk, 0, 0, 0, 0);
  for (int k = 0; k < d; k++)
    for (int l = 0; l < d; l++) {
      double D2, G, A;
      if (k == l) {
        double Pp = phi_at(S, lv, ijk, k, 1, k, 0), Pm = phi_at(S, lv, ijk, k, -1, k, 0);
        D2 = Pp - 2.0 * P0 + Pm;
        G = fabs(Pp - P0) + fabs(P0 - Pm);
        A = fabs(Pp) + 2.0 * fabs(P0) + fabs(Pm);
      } else {
        double Ppp = phi_at(S, lv, ijk, k, 1, l, 1), Ppm = phi_at(S, lv, ijk, k, 1, l, -1);
        double Pmp = phi_at(S, lv, ijk, k, -1, l, 1), Pmm = phi_at(S, lv, ijk, k, -1, l, -1);
        D2 = (Ppp - Ppm - Pmp + Pmm) / 4.0;
        G = (fabs(Ppp - Pmp) + fabs(Ppm - Pmm)) / 4.0;
        A = (fabs(Ppp) + fabs(Ppm) + fabs(Pmp) + fabs(Pmm)) / 4.0;
      }
      num += D2 * D2;
      den += (G + eps * A) * (G + eps * A);
    }
  if (den <= 0.0) return 0.0;
  return sqrt(num / den);
}

/* Voronoi neighbour offsets (3^d - 1) */
static int voronoi(int d, int off[26][3]) {
  int n = 0;
  for (int k = (d == 3 ? -1 : 0); k <= (d == 3 ? 1 : 0); k++)
    for (int j = -1; j <= 1; j++)
      for (int i = -1; i <= 1; i++) {
        if (!i && !j && !k) continue;
        off[n][0] = i; off[n][1] = j; off[n][2] = k;
        n++;
      }
  return n;
}

/* Regrid pre-pass at a synchronisation time: WENO polynomial of every active cell of
 * levels 0..lmax-1, top-down, and the virtual children of levels 1..lmax-1 filled with
 * the child-box averages of their mothers' WENO polynomials, so that the indicator sees
 * current same-level neighbours (reading). In initial-condition mode the IC averages are
 * used instead and nothing is filled. */
static void regrid_prepass(osolver *S, int init_mode) {
  int V = S->V;
  for (int lv = 0; lv < S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    if (!init_mode) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(S->nthreads)
      for (int ia = 0; ia < L->na; ia++) {
        int ijk[3];
        coords(L, L->alist[ia], ijk);
        weno_cell(S, lv, ijk, L->wh + (size_t)ia * V * S->nsp);
      }
      if (lv + 1 < S->c.lmax) {
        olev *Lc = &S->lev[lv + 1];
        for (long c = 0; c < Lc->n; c++) {
          if (Lc->st[c] != 1) continue;
          int ijk[3], ch[3];
          coords(Lc, c, ijk);
          long m = mother_of(S, lv + 1, ijk, ch);
          project_sp(S, L->wh + (size_t)L->aid[m] * V * S->nsp, ch, Lc->u + c * V);
        }
      }
    }
  }
  /* indicator on cells of status <= 0 of levels 0..lmax-1 */
  for (int lv = 0; lv < S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      L->chi[c] = 0.0;
      if (L->st[c] == 0 || L->st[c] == -1) {
        int ijk[3];
        coords(L, c, ijk);
        L->chi[c] = indicator(S, lv, ijk);
      }
    }
  }
}

/* flags from the indicator: +1 refine (active, l < lmax, chi^ > chi_ref), -1 coarsen
 * (virtual mother, chi^ < chi_rec), 0 otherwise; dense per level.  chi^ is the largest indicator
 * over the cell and its same-level Voronoi neighbours of status <= 0 (reading: the second
 * difference vanishes in the middle of a jump smeared over a few cells and peaks on both sides
 * of it, so Loehner's criterion is applied to neighbourhoods, as in the block-based codes the
 * paper cites; a cell cut by a discontinuity is thereby refined with its neighbours). */
static void flags_from_chi(const osolver *S, int8_t **fl) {
  int off[26][3];
  int nv = voronoi(S->d, off);
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    const olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      int8_t f = 0;
      if (lv < S->c.lmax && (L->st[c] == 0 || L->st[c] == -1)) {
        int ijk[3];
        coords(L, c, ijk);
        double chi = L->chi[c];
        for (int o = 0; o < nv; o++) {
          int nb[3] = {ijk[0] + off[o][0], ijk[1] + off[o][1], ijk[2] + off[o][2]}, in = 1;
          for (int a = 0; a < S->d; a++) in &= bcmap(S, lv, a, nb[a], &nb[a]);
          if (!in) continue;
          long nc = didx(L, nb[0], nb[1], nb[2]);
          if ((L->st[nc] == 0 || L->st[nc] == -1) && L->chi[nc] > chi) chi = L->chi[nc];
        }
        if (L->st[c] == 0 && chi > S->c.chi_ref) f = 1;
        if (L->st[c] == -1 && chi < S->c.chi_rec) f = -1;
      }
      fl[lv][c] = f;
    }
  }
}

/* can virtual mother c (level lv) be recoarsened? (rule 7: all children active with no
 * children of any status, and no child flagged for refinement) */
static int coarsen_ok(const osolver *S, int lv, long c, int8_t **fl) {
  const olev *L = &S->lev[lv], *Lc = &S->lev[lv + 1];
  int r = S->c.r, d = S->d, rz = d == 3 ? r : 1, ijk[3];
  coords(L, c, ijk);
  for (int kk = 0; kk < rz; kk++)
    for (int jj = 0; jj < r; jj++)
      for (int ii = 0; ii < r; ii++) {
        int cc3[3] = {r * ijk[0] + ii, r * ijk[1] + jj, d == 3 ? r * ijk[2] + kk : 0};
        long cc = didx(Lc, cc3[0], cc3[1], cc3[2]);
        if (Lc->st[cc] != 0) return 0;
        if (fl[lv + 1][cc] == 1) return 0;
        if (lv + 1 < S->c.lmax) {
          const olev *Lg = &S->lev[lv + 2];
          /* any grandchild of any status forbids destruction */
          long g = didx(Lg, r * cc3[0], r * cc3[1], d == 3 ? r * cc3[2] : 0);
          if (Lg->st[g] != ST_NONE) return 0;
        }
      }
  return 1;
}

/* Apply flags (dense per level) and rebuild the tree.  R = set of cells with children of
 * status <= 0 (virtual mothers).  R1 = R - {eligible coarsen} + {refine}; closure under
 * rules 4-5: for m in R at level l >= 1, every Voronoi neighbour n of m must have its
 * mother in R (fine to coarse, one pass per level reaches the least fixed point).  Then
 * statuses follow from R: sigma=-1 in R; sigma=0 if the mother is in R (or l = 0);
 * sigma=1 if the mother is active and has a Voronoi neighbour in R; otherwise no cell. */
static int apply_flags(osolver *S, int8_t **fl, int init_mode) {
  int lmax = S->c.lmax, d = S->d, V = S->V, r = S->c.r;
  if (lmax == 0) return 0;
  int off[26][3];
  int nv = voronoi(d, off);
  int8_t *R[MAXL], *nstat[MAXL];
  for (int lv = 0; lv <= lmax; lv++) {
    olev *L = &S->lev[lv];
    R[lv] = calloc(L->n, 1);
    nstat[lv] = malloc(L->n);
    for (long c = 0; c < L->n; c++) R[lv][c] = (L->st[c] == -1);
  }
  for (int lv = 0; lv < lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      if (fl[lv][c] == 1 && L->st[c] == 0) R[lv][c] = 1;
      if (fl[lv][c] == -1 && L->st[c] == -1 && coarsen_ok(S, lv, c, fl)) R[lv][c] = 0;
    }
  }
  for (int lv = lmax - 1; lv >= 1; lv--) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      if (!R[lv][c]) continue;
      int ijk[3];
      coords(L, c, ijk);
      for (int o = 0; o < nv; o++) {
        int nb[3] = {ijk[0] + off[o][0], ijk[1] + off[o][1], ijk[2] + off[o][2]}, in = 1;
        for (int a = 0; a < d; a++) in &= bcmap(S, lv, a, nb[a], &nb[a]);
        if (!in) continue;
        int m[3] = {nb[0] / r, nb[1] / r, d == 3 ? nb[2] / r : 0};
        R[lv - 1][didx(&S->lev[lv - 1], m[0], m[1], m[2])] = 1;
      }
    }
  }
  /* statuses, top-down */
  for (int lv = 0; lv <= lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      int8_t s = ST_NONE;
      if (lv == 0) s = R[0][c] ? -1 : 0;
      else {
        int ijk[3], ch[3];
        coords(L, c, ijk);
        long m = mother_of(S, lv, ijk, ch);
        if (R[lv - 1][m]) s = R[lv][c] ? -1 : 0;
        else if (nstat[lv - 1][m] == 0) {
          int mi[3];
          coords(&S->lev[lv - 1], m, mi);
          int has = 0;
          for (int o = 0; o < nv && !has; o++) {
            int nb[3] = {mi[0] + off[o][0], mi[1] + off[o][1], mi[2] + off[o][2]}, in = 1;
            for (int a = 0; a < d; a++) in &= bcmap(S, lv - 1, a, nb[a], &nb[a]);
            if (in && R[lv - 1][didx(&S->lev[lv - 1], nb[0], nb[1], nb[2])]) has = 1;
          }
          if (has) s = 1;
        }
      }
      nstat[lv][c] = s;
    }
  }
  /* values of cells that change role */
  for (int lv = 1; lv <= lmax; lv++) {
    olev *L = &S->lev[lv], *Lm = &S->lev[lv - 1];
    for (long c = 0; c < L->n; c++) {
      int8_t o = L->st[c], n = nstat[lv][c];
      if (n == ST_NONE) continue;
      int ijk[3], ch[3];
      coords(L, c, ijk);
      long m = mother_of(S, lv, ijk, ch);
      if (init_mode) {
        if (o == ST_NONE) ic_average(S, lv, ijk, L->u + c * V);
        continue;
      }
      if (n <= 0 && (o == ST_NONE || o == 1)) {
        /* newly active (or new virtual mother, re-averaged below): project the mother's
         * WENO polynomial; the mother was active before the edit */
        project_sp(S, Lm->wh + (size_t)Lm->aid[m] * V * S->nsp, ch, L->u + c * V);
      }
    }
  }
  for (int lv = 0; lv <= lmax; lv++) {
    memcpy(S->lev[lv].st, nstat[lv], S->lev[lv].n);
    free(R[lv]); free(nstat[lv]);
  }
  /* virtual children hold their mother's average until the next projection (reading) */
  if (!init_mode)
    for (int lv = 1; lv <= lmax; lv++) {
      olev *L = &S->lev[lv], *Lm = &S->lev[lv - 1];
      for (long c = 0; c < L->n; c++) {
        if (L->st[c] != 1) continue;
        int ijk[3], ch[3];
        coords(L, c, ijk);
        long m = mother_of(S, lv, ijk, ch);
        for (int v = 0; v < V; v++) L->u[c * V + v] = Lm->u[m * V + v];
      }
    }
  /* cells that no longer exist are cleared */
  for (int lv = 0; lv <= lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++)
      if (L->st[c] == ST_NONE) {
        for (int v = 0; v < V; v++) L->u[c * V + v] = 0.0;
      }
  }
  average_all(S);
  build_active(S);
  return 0;
}

/* ===================================================================================
 * 11. Public (ctypes) interface
 * =================================================================================== */
void *orc_create(const orc_cfg *c) {
  if (c->dim != 2 && c->dim != 3) { seterr("dim must be 2 or 3"); return NULL; }
  if (c->M < 1 || c->M + 1 > MAXN) { seterr("M out of range"); return NULL; }
  if (c->lmax < 0 || c->lmax >= MAXL) { seterr("lmax out of range"); return NULL; }
  if (c->lmax > 0 && (c->r < 2 || c->r < c->M)) { seterr("need r >= max(2, M)"); return NULL; }
  osolver *S = calloc(1, sizeof *S);
  S->c = *c;
  S->d = c->dim;
  S->N = c->M + 1;
  S->P.pde = c->pde; S->P.d = c->dim; S->P.gamma = c->gamma; S->P.c_h = c->c_h; S->P.flux = c->flux;
  for (int i = 0; i < 6; i++)
    if (c->bc[i] == BC_REFLECTIVE && c->pde == PDE_MHD) {
      seterr("reflective walls are available for Euler and linear advection");
      free(S);
      return NULL;
    }
  for (int a = 0; a < 3; a++) S->P.adv[a] = c->adv[a];
  S->V = c->pde == PDE_LINADV ? 1 : (c->pde == PDE_EULER ? c->dim + 2 : 9);
  S->P.V = S->V;
  S->P_iters = c->picard > 0 ? c->picard : c->M + 1;
  build_tables(&S->T, c->M, c->dim);
  S->nsp = S->T.nsp; S->nst = S->T.nst;
  S->dx0[0] = (c->hi[0] - c->lo[0]) / c->nx;
  S->dx0[1] = (c->hi[1] - c->lo[1]) / c->ny;
  S->dx0[2] = c->dim == 3 ? (c->hi[2] - c->lo[2]) / c->nz : 1.0;
  S->nthreads = 1;
  for (int lv = 0; lv <= c->lmax; lv++) lev_alloc(S, lv);
  memset(S->lev[0].st, 0, S->lev[0].n);
  build_active(S);
  return S;
}

void orc_destroy(void *h) {
  osolver *S = h;
  if (!S) return;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    free(L->st); free(L->u); free(L->mem); free(L->chi); free(L->aid); free(L->alist);
    free(L->wh); free(L->qh); free(L->fl);
  }
  free_tables(&S->T);
  free(S);
}

void orc_set_threads(void *h, int n) { ((osolver *)h)->nthreads = n > 0 ? n : 1; }

/* set the IC on every existing cell; then nrefine passes of indicator + regrid in
 * initial-condition mode (new cells take IC averages) */
int orc_regrid(void *h, int init_mode);
int orc_set_initial(void *h, int ic, const double *params, int np, int nrefine) {
  osolver *S = h;
  S->ic = ic;
  S->icn = np < 128 ? np : 128;
  for (int i = 0; i < S->icn; i++) S->icp[i] = params[i];
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      if (L->st[c] == ST_NONE) continue;
      int ijk[3];
      coords(L, c, ijk);
      ic_average(S, lv, ijk, L->u + c * S->V);
    }
  }
  average_all(S);
  S->t = 0.0;
  for (int p = 0; p < nrefine; p++) orc_regrid(h, 1);
  return 0;
}

long orc_num_cells(void *h, long *per_level, long *active_per_level) {
  osolver *S = h;
  long n = 0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    long k = 0;
    for (long c = 0; c < L->n; c++) k += L->st[c] != ST_NONE;
    if (per_level) per_level[lv] = k;
    if (active_per_level) active_per_level[lv] = L->na;
    n += k;
  }
  return n;
}

/* canonical export: levels ascending, then (k, j, i); meta = (level, status, i, j, k) */
long orc_read_cells(void *h, int32_t *meta, double *u, long cap) {
  osolver *S = h;
  long n = 0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      if (L->st[c] == ST_NONE) continue;
      if (n < cap) {
        int ijk[3];
        coords(L, c, ijk);
        if (meta) { meta[5 * n] = lv; meta[5 * n + 1] = L->st[c]; meta[5 * n + 2] = ijk[0]; meta[5 * n + 3] = ijk[1]; meta[5 * n + 4] = ijk[2]; }
        if (u) memcpy(u + n * S->V, L->u + c * S->V, sizeof(double) * S->V);
      }
      n++;
    }
  }
  return n;
}

/* set values of every existing cell in canonical order; virtual mothers re-averaged */
int orc_set_cell_averages(void *h, const double *u, long n) {
  osolver *S = h;
  long k = 0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      if (L->st[c] == ST_NONE) continue;
      if (k >= n) { seterr("too few values"); return -1; }
      memcpy(L->u + c * S->V, u + k * S->V, sizeof(double) * S->V);
      k++;
    }
  }
  if (k != n) { seterr("value count does not match the cell count"); return -1; }
  average_all(S);
  return 0;
}

double orc_compute_dt(void *h) { return compute_dt(h); }

/* one level-0 step of size dt0 (all levels, local time stepping); returns 0, or -4 if a
 * non-physical state appeared */
int orc_advance_dt(void *h, double dt0) {
  osolver *S = h;
  g_nonphysical = 0;
  advance(S, 0, 0, dt0);
  S->t += dt0;
  return g_nonphysical ? -4 : 0;
}

/* one level-0 step with CFL dt clipped at t_end, followed by a regrid if auto_regrid */
int orc_step(void *h, double t_end, double *dt_out) {
  osolver *S = h;
  if (!(t_end > S->t)) { seterr("t_end is not after t"); return -1; }
  double dt = compute_dt(S);
  int clipped = 0;
  if (S->t + dt >= t_end) { dt = t_end - S->t; clipped = 1; }
  g_nonphysical = 0;
  advance(S, 0, 0, dt);
  if (clipped) S->t = t_end;
  else S->t += dt;
  if (dt_out) *dt_out = dt;
  if (S->c.auto_regrid && S->c.lmax > 0) orc_regrid(h, 0);
  return g_nonphysical ? -4 : 0;
}

double orc_time(void *h) { return ((osolver *)h)->t; }
void orc_set_time(void *h, double t) { ((osolver *)h)->t = t; }
int64_t orc_updates(void *h, int64_t *per_level) {
  osolver *S = h;
  if (per_level)
    for (int lv = 0; lv <= S->c.lmax; lv++) per_level[lv] = S->level_updates[lv];
  return S->updates;
}

/* flags of every existing cell in canonical order (from the indicator) */
long orc_compute_flags(void *h, int init_mode, int8_t *out, long cap) {
  osolver *S = h;
  if (S->c.lmax == 0) return 0;
  regrid_prepass(S, init_mode);
  int8_t *fl[MAXL];
  for (int lv = 0; lv <= S->c.lmax; lv++) fl[lv] = malloc(S->lev[lv].n);
  flags_from_chi(S, fl);
  long n = 0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    for (long c = 0; c < L->n; c++) {
      if (L->st[c] == ST_NONE) continue;
      if (n < cap) out[n] = fl[lv][c];
      n++;
    }
  }
  for (int lv = 0; lv <= S->c.lmax; lv++) free(fl[lv]);
  return n;
}

/* regrid with given flags (canonical order, one per existing cell) */
int orc_regrid_with_flags(void *h, const int8_t *flags, long n, int init_mode) {
  osolver *S = h;
  if (S->c.lmax == 0) return 0;
  regrid_prepass(S, init_mode);
  int8_t *fl[MAXL];
  long k = 0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    fl[lv] = calloc(L->n, 1);
    for (long c = 0; c < L->n; c++) {
      if (L->st[c] == ST_NONE) continue;
      if (k < n) fl[lv][c] = flags[k];
      k++;
    }
  }
  int rc = 0;
  if (k != n) { seterr("flag count does not match the cell count"); rc = -1; }
  else rc = apply_flags(S, fl, init_mode);
  for (int lv = 0; lv <= S->c.lmax; lv++) free(fl[lv]);
  return rc;
}

int orc_regrid(void *h, int init_mode) {
  osolver *S = h;
  if (S->c.lmax == 0) return 0;
  regrid_prepass(S, init_mode);
  int8_t *fl[MAXL];
  for (int lv = 0; lv <= S->c.lmax; lv++) fl[lv] = malloc(S->lev[lv].n);
  flags_from_chi(S, fl);
  int rc = apply_flags(S, fl, init_mode);
  for (int lv = 0; lv <= S->c.lmax; lv++) free(fl[lv]);
  return rc;
}

/* internal dumps of level lv, in the canonical order of that level:
 * what=0: WENO dofs of active cells (V*nsp each, [v][p + N q + N^2 r])
 * what=1: predictor dofs of active cells (V*nst each, [v][p + N q (+ N^2 r) + nsp s])
 * what=2: indicator of every existing cell
 * what=3: face fluxes of active cells (2d*V each, [a][side][v]) from the last update */
long orc_read_internal(void *h, int what, int lv, double *buf, long cap) {
  osolver *S = h;
  olev *L = &S->lev[lv];
  long per = what == 0 ? S->V * S->nsp : what == 1 ? S->V * S->nst : what == 3 ? 2 * S->d * S->V : 1;
  long n = 0;
  if (what == 2) {
    for (long c = 0; c < L->n; c++) {
      if (L->st[c] == ST_NONE) continue;
      if (n < cap) buf[n] = L->chi[c];
      n++;
    }
    return n;
  }
  const double *src = what == 0 ? L->wh : what == 1 ? L->qh : L->fl;
  for (int ia = 0; ia < L->na; ia++) {
    if ((ia + 1) * per <= cap) memcpy(buf + ia * per, src + (size_t)ia * per, sizeof(double) * per);
    n += per;
  }
  return n;
}

/* compute (without stepping) the WENO polynomials of all active cells of level lv from the
 * current cell averages (virtual children must hold valid values) */
int orc_weno_level(void *h, int lv) {
  osolver *S = h;
  olev *L = &S->lev[lv];
  for (int ia = 0; ia < L->na; ia++) {
    int ijk[3];
    coords(L, L->alist[ia], ijk);
    weno_cell(S, lv, ijk, L->wh + (size_t)ia * S->V * S->nsp);
  }
  return 0;
}

/* ---------- stand-alone building blocks for the pins ---------- */
int orc_tables(int M, int d, double *x, double *w, double *psi, double *ainv, double *sig, int *sl, int *sr,
               double *lam) {
  tables T;
  build_tables(&T, M, d);
  int N = M + 1;
  for (int i = 0; i < N; i++) { x[i] = T.x[i]; w[i] = T.w[i]; }
  for (int l = 0; l < N; l++)
    for (int k = 0; k < N; k++) psi[l * N + k] = T.psi[l][k];
  for (int s = 0; s < T.Ns; s++) {
    sl[s] = T.SL[s]; sr[s] = T.SR[s]; lam[s] = T.lam[s];
    for (int p = 0; p < N; p++)
      for (int e = 0; e < N; e++) ainv[(s * N + p) * N + e] = T.Ainv[s][p][e];
  }
  for (int p = 0; p < N; p++)
    for (int m = 0; m < N; m++) sig[p * N + m] = T.Sig[p][m];
  int ns = T.Ns;
  free_tables(&T);
  return ns;
}

/* space-time matrices: K1inv (nst^2), Kd (d*nst^2), F0 (nst*nsp) */
int orc_st_matrices(int M, int d, double *k1inv, double *kd, double *f0) {
  tables T;
  build_tables(&T, M, d);
  int nst = T.nst, nsp = T.nsp;
  memcpy(k1inv, T.K1inv, sizeof(double) * nst * nst);
  for (int a = 0; a < d; a++) memcpy(kd + (size_t)a * nst * nst, T.Kd[a], sizeof(double) * nst * nst);
  memcpy(f0, T.F0, sizeof(double) * nst * nsp);
  free_tables(&T);
  return nst;
}

void orc_weno1d(int M, const double *v, double *out) {
  tables T;
  build_tables(&T, M, 2);
  weno1d(&T, v, out);
  free_tables(&T);
}

/* predictor on one cell: wh (V*nsp) -> qh (V*nst) */
int orc_predictor(void *h, const double *wh, double dt, const double *dx, double *qh) {
  predictor(h, wh, dt, dx, qh);
  return 0;
}

void orc_flux(void *h, const double *q, int n, double *f) { flux(&((osolver *)h)->P, q, n, f); }
double orc_max_speed(void *h, const double *q, int n) { return max_speed(&((osolver *)h)->P, q, n); }
void orc_rusanov(void *h, const double *qm, const double *qp, int n, double *f) { rusanov(&((osolver *)h)->P, qm, qp, n, f); }
void orc_osher(void *h, const double *qm, const double *qp, int n, double *f) { osher(&((osolver *)h)->P, qm, qp, n, f); }
void orc_abs_jacobian_apply(void *h, const double *q, int n, const double *dq, double *out) { abs_jacobian_apply(&((osolver *)h)->P, q, n, dq, out); }
void orc_eval_st(void *h, const double *qh, const double *xi, double tau, double *out) { eval_st(h, qh, xi, tau, out); }
void orc_eval_sp(void *h, const double *wh, const double *xi, double *out) { eval_sp(h, wh, xi, out); }
void orc_project_st(void *h, const double *qh, const int *ch, double tau, double *out) { project_st(h, qh, ch, tau, out); }
void orc_project_sp(void *h, const double *wh, const int *ch, double *out) { project_sp(h, wh, ch, out); }
double orc_indicator_at(void *h, int lv, int i, int j, int k) { int ijk[3] = {i, j, k}; return indicator(h, lv, ijk); }
void orc_ic_average(void *h, int lv, int i, int j, int k, double *out) { int ijk[3] = {i, j, k}; ic_average(h, lv, ijk, out); }
int orc_nvars(void *h) { return ((osolver *)h)->V; }
/* total of vol * u over active cells (conservation check) */
void orc_totals(void *h, double *tot) {
  osolver *S = h;
  for (int v = 0; v < S->V; v++) tot[v] = 0.0;
  for (int lv = 0; lv <= S->c.lmax; lv++) {
    olev *L = &S->lev[lv];
    double vol = 1.0;
    for (int a = 0; a < S->d; a++) vol *= dxl(S, lv, a);
    for (int ia = 0; ia < L->na; ia++)
      for (int v = 0; v < S->V; v++) tot[v] += vol * L->u[(size_t)L->alist[ia] * S->V + v];
  }
}

/* ===================================================================================
 * 12. One-dimensional radial reference solution of the explosion problems (Eq. eq.1D):
 *     the Euler equations in the radial coordinate with the geometric source
 *     -(d-1)/r (rho u, rho u^2, u (E + p)), solved by a second-order TVD finite volume
 *     scheme (minmod-limited linear reconstruction of the primitive variables, Rusanov
 *     flux, two-stage SSP Runge-Kutta) on n zones of [0, rmax]; reflection at r = 0,
 *     transmissive at rmax.  Returns the primitive state (rho, u, p) at the zone centres.
 *     (The paper's reference used 10000 zones and the Osher flux.)
 * =================================================================================== */
static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

static void radial_rhs(int d, int n, double dr, double g, const double *U, double *L) {
  /* U: 3 per zone (rho, m, E) */
  double *W = malloc(sizeof(double) * 3 * (n + 4));
  for (int i = 0; i < n + 4; i++) {
    int j = i - 2;
    int src = j < 0 ? -j - 1 : (j >= n ? n - 1 : j); /* mirror at 0, copy at rmax */
    double rho = U[3 * src], m = U[3 * src + 1], E = U[3 * src + 2];
    double u = m / rho, p = (g - 1.0) * (E - 0.5 * rho * u * u);
    W[3 * i] = rho;
    W[3 * i + 1] = j < 0 ? -u : u;
    W[3 * i + 2] = p;
  }
  double *F = malloc(sizeof(double) * 3 * (n + 1));
  for (int f = 0; f <= n; f++) {
    /* face between zones f-1 and f: ghost-padded indices i = f+1 and f+2 */
    int il = f + 1, ir = f + 2;
    double wl[3], wr[3];
    for (int k = 0; k < 3; k++) {
      double sl = minmod(W[3 * il + k] - W[3 * (il - 1) + k], W[3 * (il + 1) + k] - W[3 * il + k]);
      double sr = minmod(W[3 * ir + k] - W[3 * (ir - 1) + k], W[3 * (ir + 1) + k] - W[3 * ir + k]);
      wl[k] = W[3 * il + k] + 0.5 * sl;
      wr[k] = W[3 * ir + k] - 0.5 * sr;
    }
    double ql[3] = {wl[0], wl[0] * wl[1], wl[2] / (g - 1.0) + 0.5 * wl[0] * wl[1] * wl[1]};
    double qr[3] = {wr[0], wr[0] * wr[1], wr[2] / (g - 1.0) + 0.5 * wr[0] * wr[1] * wr[1]};
    double fl[3] = {ql[1], ql[1] * wl[1] + wl[2], wl[1] * (ql[2] + wl[2])};
    double fr[3] = {qr[1], qr[1] * wr[1] + wr[2], wr[1] * (qr[2] + wr[2])};
    double cl = fabs(wl[1]) + sqrt(g * fabs(wl[2] / wl[0])), cr = fabs(wr[1]) + sqrt(g * fabs(wr[2] / wr[0]));
    double sm = cl > cr ? cl : cr;
    for (int k = 0; k < 3; k++) F[3 * f + k] = 0.5 * (fl[k] + fr[k]) - 0.5 * sm * (qr[k] - ql[k]);
  }
  for (int i = 0; i < n; i++) {
    double r = (i + 0.5) * dr;
    double rho = U[3 * i], m = U[3 * i + 1], E = U[3 * i + 2], u = m / rho, p = (g - 1.0) * (E - 0.5 * rho * u * u);
    double geo = (d - 1) / r;
    L[3 * i] = -(F[3 * (i + 1)] - F[3 * i]) / dr - geo * m;
    L[3 * i + 1] = -(F[3 * (i + 1) + 1] - F[3 * i + 1]) / dr - geo * m * u;
    L[3 * i + 2] = -(F[3 * (i + 1) + 2] - F[3 * i + 2]) / dr - geo * u * (E + p);
  }
  free(W);
  free(F);
}

int orc_radial_explosion(int d, double R, double rho_in, double p_in, double rho_out, double p_out, double gamma,
                         int n, double rmax, double t_end, double cfl, double *rho_o, double *u_o, double *p_o) {
  double dr = rmax / n, g = gamma;
  double *U = malloc(sizeof(double) * 3 * n), *U1 = malloc(sizeof(double) * 3 * n), *L = malloc(sizeof(double) * 3 * n);
  for (int i = 0; i < n; i++) {
    /* exact zone averages of the piecewise constant data (the jump at R may cut a zone) */
    double a = i * dr, b = (i + 1) * dr, f = (R <= a) ? 0.0 : (R >= b ? 1.0 : (R - a) / dr);
    double rho = f * rho_in + (1 - f) * rho_out, p = f * p_in + (1 - f) * p_out;
    U[3 * i] = rho; U[3 * i + 1] = 0.0; U[3 * i + 2] = p / (g - 1.0);
  }
  double t = 0.0;
  while (t < t_end) {
    double smax = 0.0;
    for (int i = 0; i < n; i++) {
      double rho = U[3 * i], u = U[3 * i + 1] / rho, p = (g - 1.0) * (U[3 * i + 2] - 0.5 * rho * u * u);
      double s = fabs(u) + sqrt(g * p / rho);
      if (s > smax) smax = s;
    }
    double dt = cfl * dr / smax;
    if (t + dt > t_end) dt = t_end - t;
    radial_rhs(d, n, dr, g, U, L);
    for (int k = 0; k < 3 * n; k++) U1[k] = U[k] + dt * L[k];
    radial_rhs(d, n, dr, g, U1, L);
    for (int k = 0; k < 3 * n; k++) U[k] = 0.5 * (U[k] + U1[k] + dt * L[k]);
    t += dt;
  }
  for (int i = 0; i < n; i++) {
    double rho = U[3 * i], u = U[3 * i + 1] / rho;
    rho_o[i] = rho;
    u_o[i] = u;
    p_o[i] = (g - 1.0) * (U[3 * i + 2] - 0.5 * rho * u * u);
  }
  free(U); free(U1); free(L);
  return 0;
}
