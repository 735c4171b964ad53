// aw_tables.cu -- reference-element tables of the ADER-WENO scheme, computed on the host in
// long double (aw_tables_host exports them):
//   * Gauss-Legendre nodes/weights on [0,1] (bracketing of the sign changes of P_N, then Newton),
//   * nodal Lagrange basis psi_l through those nodes (Sec. 2.2) in product form, its derivative
//     matrix Dm[i][l] = psi_l'(x_i) from the barycentric weights,
//   * WENO stencil reconstruction matrices, the inverse of the integral-conservation system
//     of Eq. eqn.rec.x for each stencil of Eq. eqn.stencildef,
//   * the oscillation indicator matrix of Eq. eqn.sigmas, from the nodal values of the
//     derivatives (powers of Dm) and the Gauss rule, which is exact for these degrees,
//   * the time block of the predictor matrix K1 (Sec. 2.3): with the nodal tensor basis
//     K1 = diag(w x w ...) (x) K_t, K_t[s'][s] = psi_s'(1) psi_s(1) - w_s Dm[s][s'], and
//     G = K_t^{-1} diag(w),
//   * projection tables of Sec. 3.1.3 for the r^d children of a cell.
#include <cmath>
#include <cstring>
#include <vector>

#include "aw_device.cuh"

namespace aw {

typedef long double LD;

static LD legendre(int n, LD z, LD* dp) {
  LD p0 = 1.0L, p1 = z;
  if (n == 0) { *dp = 0; return 1; }
  for (int k = 2; k <= n; k++) {
    LD p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *dp = n * (p0 - z * p1) / (1.0L - z * z);
  return p1;
}

// nodes ascending on [0,1]
static void gauss01(int n, LD* x, LD* w) {
  const int NS = 2000;
  int found = 0;
  LD dp;
  LD a = -1.0L, fa = legendre(n, a + 1e-12L, &dp);
  for (int i = 1; i <= NS && found < n; i++) {
    LD b = -1.0L + 2.0L * i / NS, fb = legendre(n, b, &dp);
    if (i == NS) b -= 1e-12L, fb = legendre(n, b, &dp);
    if ((fa < 0) != (fb < 0)) {
      LD lo = a, hi = b;
      for (int it = 0; it < 100; it++) {
        LD m = 0.5L * (lo + hi), fm = legendre(n, m, &dp);
        if ((fm < 0) == (fa < 0)) lo = m; else hi = m;
      }
      LD z = 0.5L * (lo + hi);
      for (int it = 0; it < 5; it++) {
        LD f = legendre(n, z, &dp);
        z -= f / dp;
      }
      legendre(n, z, &dp);
      x[found] = 0.5L * (z + 1.0L);
      w[found] = 1.0L / ((1.0L - z * z) * dp * dp);
      found++;
    }
    a = b;
    fa = fb;
  }
}

static LD lag(const LD* x, int n, int l, LD t) {
  LD v = 1.0L;
  for (int k = 0; k < n; k++)
    if (k != l) v *= (t - x[k]) / (x[l] - x[k]);
  return v;
}

static bool invert(int n, std::vector<LD>& A, std::vector<LD>& Ai) {
  std::vector<LD> a(A);
  Ai.assign(n * n, 0.0L);
  for (int i = 0; i < n; i++) Ai[i * n + i] = 1.0L;
  for (int c = 0; c < n; c++) {
    int p = c;
    for (int i = c + 1; i < n; i++)
      if (fabsl(a[i * n + c]) > fabsl(a[p * n + c])) p = i;
    if (fabsl(a[p * n + c]) == 0.0L) return false;
    for (int j = 0; j < n; j++) { std::swap(a[c * n + j], a[p * n + j]); std::swap(Ai[c * n + j], Ai[p * n + j]); }
    LD d = a[c * n + c];
    for (int j = 0; j < n; j++) { a[c * n + j] /= d; Ai[c * n + j] /= d; }
    for (int i = 0; i < n; i++) {
      if (i == c) continue;
      LD f = a[i * n + c];
      for (int j = 0; j < n; j++) { a[i * n + j] -= f * a[c * n + j]; Ai[i * n + j] -= f * Ai[c * n + j]; }
    }
  }
  return true;
}

bool build_tables(int M, int r, Tables* T) {
  if (M < 1 || M + 1 > MAXN || r < 1 || r > MAXR) return false;
  std::memset(T, 0, sizeof *T);
  const int N = M + 1;
  T->N = N; T->M = M; T->r = r;
  LD x[MAXN], w[MAXN];
  gauss01(N, x, w);
  for (int i = 0; i < N; i++) { T->x[i] = (double)x[i]; T->w[i] = (double)w[i]; }
  for (int l = 0; l < N; l++) { T->psi0[l] = (double)lag(x, N, l, 0.0L); T->psi1[l] = (double)lag(x, N, l, 1.0L); }
  // barycentric weights and derivative matrix
  LD bw[MAXN], Dm[MAXN][MAXN];
  for (int j = 0; j < N; j++) {
    bw[j] = 1.0L;
    for (int k = 0; k < N; k++)
      if (k != j) bw[j] /= (x[j] - x[k]);
  }
  for (int i = 0; i < N; i++) {
    LD diag = 0.0L;
    for (int j = 0; j < N; j++) {
      if (j == i) continue;
      Dm[i][j] = (bw[j] / bw[i]) / (x[i] - x[j]);
      diag -= Dm[i][j];
    }
    Dm[i][i] = diag;
  }
  for (int i = 0; i < N; i++)
    for (int j = 0; j < N; j++) T->Dm[i][j] = (double)Dm[i][j];
  // stencils: M even: central, fully left, fully right; M odd: two central, left, right
  int NS = (M % 2 == 0) ? 3 : 4;
  T->Ns = NS;
  int SL[4];
  if (M % 2 == 0) { SL[0] = M / 2; SL[1] = M; SL[2] = 0; T->lam[0] = 1e5; T->lam[1] = 1.0; T->lam[2] = 1.0; }
  else { SL[0] = M / 2 + 1; SL[1] = M / 2; SL[2] = M; SL[3] = 0; T->lam[0] = 1e5; T->lam[1] = 1e5; T->lam[2] = 1.0; T->lam[3] = 1.0; }
  for (int s = 0; s < NS; s++) {
    T->SL[s] = SL[s];
    std::vector<LD> A(N * N), Ai;
    for (int e = 0; e < N; e++) {
      LD o = -SL[s] + e;
      for (int p = 0; p < N; p++) {
        LD acc = 0.0L;  // exact N-point Gauss rule on [o, o+1]
        for (int g = 0; g < N; g++) acc += w[g] * lag(x, N, p, o + x[g]);
        A[e * N + p] = acc;
      }
    }
    if (!invert(N, A, Ai)) return false;
    for (int p = 0; p < N; p++)
      for (int e = 0; e < N; e++) T->Ainv[s][p][e] = (double)Ai[p * N + e];
  }
  // oscillation indicator: nodal values of psi^(alpha) are the columns of Dm^alpha
  {
    LD P[MAXN][MAXN], Q[MAXN][MAXN], S[MAXN][MAXN];
    for (int i = 0; i < N; i++)
      for (int j = 0; j < N; j++) { P[i][j] = Dm[i][j]; S[i][j] = 0.0L; }
    for (int al = 1; al <= M; al++) {
      for (int p = 0; p < N; p++)
        for (int m = 0; m < N; m++) {
          LD acc = 0.0L;
          for (int i = 0; i < N; i++) acc += w[i] * P[i][p] * P[i][m];
          S[p][m] += acc;
        }
      for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
          LD acc = 0.0L;
          for (int k = 0; k < N; k++) acc += Dm[i][k] * P[k][j];
          Q[i][j] = acc;
        }
      for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) P[i][j] = Q[i][j];
    }
    for (int p = 0; p < N; p++)
      for (int m = 0; m < N; m++) T->Sig[p][m] = (double)S[p][m];
  }
  // sigma_s as a quadratic form of the stencil differences
  for (int s = 0; s < NS; s++) {
    LD B[MAXN][MAXN];
    for (int e = 0; e < N; e++)
      for (int f = 0; f < N; f++) {
        LD acc = 0.0L;
        for (int p = 0; p < N; p++)
          for (int m = 0; m < N; m++) acc += (LD)T->Ainv[s][p][e] * (LD)T->Sig[p][m] * (LD)T->Ainv[s][m][f];
        B[e][f] = acc;
      }
    int idx[MAXN], k = 0;
    for (int e = 0; e < N; e++)
      if (e != SL[s]) idx[k++] = e;
    for (int i = 0; i < N - 1; i++)
      for (int j = 0; j < N - 1; j++)
        T->Bq[s][i][j] = j < i ? 0.0 : (double)((j == i ? 1.0L : 2.0L) * B[idx[i]][idx[j]]);
  }
  // time block of K1 and G = K_t^{-1} diag(w)
  {
    std::vector<LD> Kt(N * N), Ki;
    for (int a = 0; a < N; a++)
      for (int b = 0; b < N; b++) Kt[a * N + b] = lag(x, N, a, 1.0L) * lag(x, N, b, 1.0L) - w[b] * Dm[b][a];
    if (!invert(N, Kt, Ki)) return false;
    for (int a = 0; a < N; a++) {
      LD gs = 0.0L;
      for (int b = 0; b < N; b++) { LD g = Ki[a * N + b] * w[b]; T->G[a][b] = (double)g; gs += g; }
      T->gsum[a] = (double)gs;
    }
  }
  // projection tables
  for (int c = 0; c < r; c++) {
    for (int l = 0; l < N; l++) {
      LD acc = 0.0L;
      for (int g = 0; g < N; g++) acc += w[g] * lag(x, N, l, (c + x[g]) / r);
      T->Wc[c][l] = (double)acc;
      T->Pt[c][l] = (double)lag(x, N, l, (LD)c / r);
      for (int i = 0; i < N; i++) T->Pf[c][i][l] = (double)lag(x, N, l, (c + x[i]) / r);
    }
  }
  return true;
}

}  // namespace aw
