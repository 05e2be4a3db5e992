// Host-side collocation setup in extended precision (paper Section 2.1):
// right-Radau nodes, the collocation matrix Q (Eq. 2.3-2.4), the
// eigen-decomposition Q = V diag(lambda) V^{-1} used to decouple the slab
// solves, the DG matrix K (Eq. 2.9) and the slab-bisection transfers, and the
// SDC lower-triangular preconditioners.
#include "st_setup.h"

#include <cmath>
#include <complex>

namespace st {

typedef long double LD;
typedef std::complex<LD> CLD;

// Legendre P_k(x) and P_k'(x) by the three-term recurrences.
static void legendre(int k, LD x, LD& p, LD& dp) {
  LD p0 = 1, p1 = x, d0 = 0, d1 = 1;
  if (k == 0) { p = 1; dp = 0; return; }
  for (int j = 1; j < k; ++j) {
    const LD p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
    const LD d2 = d0 + (2 * j + 1) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  p = p1;
  dp = d1;
}

static LD radau_f(int M, LD x, LD* df) {
  LD a, da, b, db;
  legendre(M - 1, x, a, da);
  legendre(M, x, b, db);
  if (df) *df = da - db;
  return a - b;
}

// Real Gauss-Jordan inverse with partial pivoting (n <= 2*MAXM).
static bool invert(int n, LD A[][2 * MAXM], LD Ai[][2 * MAXM]) {
  LD W[2 * MAXM][4 * MAXM];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) W[r][c] = (c < n) ? A[r][c] : (c - n == r ? 1 : 0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabsl(W[r][col]) > fabsl(W[piv][col])) piv = r;
    if (W[piv][col] == 0) return false;
    for (int c = 0; c < 2 * n; ++c) std::swap(W[col][c], W[piv][c]);
    const LD inv = 1 / W[col][col];
    for (int c = 0; c < 2 * n; ++c) W[col][c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const LD f = W[r][col];
      for (int c = 0; c < 2 * n; ++c) W[r][c] -= f * W[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ai[r][c] = W[r][c + n];
  return true;
}

static bool cinvert(int n, CLD A[][MAXM], CLD Ai[][MAXM]) {
  CLD W[MAXM][2 * MAXM];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) W[r][c] = (c < n) ? A[r][c] : CLD(c - n == r ? 1 : 0, 0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::abs(W[r][col]) > std::abs(W[piv][col])) piv = r;
    if (std::abs(W[piv][col]) == 0) return false;
    for (int c = 0; c < 2 * n; ++c) std::swap(W[col][c], W[piv][c]);
    const CLD inv = CLD(1, 0) / W[col][col];
    for (int c = 0; c < 2 * n; ++c) W[col][c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const CLD f = W[r][col];
      for (int c = 0; c < 2 * n; ++c) W[r][c] -= f * W[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ai[r][c] = W[r][c + n];
  return true;
}

static LD lagrange(const LD* tau, int M, int j, LD s) {
  LD v = 1;
  for (int k = 0; k < M; ++k)
    if (k != j) v *= (s - tau[k]) / (tau[j] - tau[k]);
  return v;
}

int colloc_setup(int M, Colloc* out) {
  if (M < 1 || M > MAXM) return -1;
  Colloc c;
  c.M = M;
  LD tau[MAXM];
  // 1. nodes: x = 1 and the M-1 sign changes of P_{M-1} - P_M inside (-1, 1)
  {
    int found = 0;
    const int NS = 20000;
    LD xa = -1, fa = radau_f(M, xa, nullptr);
    for (int i = 1; i <= NS && found < M - 1; ++i) {
      const LD xb = -1 + (LD)2 * i / NS * (1 - 1e-7L);
      const LD fb = radau_f(M, xb, nullptr);
      if ((fa < 0) != (fb < 0) || fb == 0) {
        LD lo = xa, hi = xb, flo = fa;
        for (int it = 0; it < 200; ++it) {
          const LD mid = (lo + hi) / 2;
          const LD fm = radau_f(M, mid, nullptr);
          if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
        }
        LD x = (lo + hi) / 2;
        for (int it = 0; it < 3; ++it) {
          LD d;
          const LD f = radau_f(M, x, &d);
          if (d != 0) x -= f / d;
        }
        tau[found++] = (x + 1) / 2;
      }
      xa = xb;
      fa = fb;
    }
    if (found != M - 1) return -2;
    tau[M - 1] = 1;
  }
  // 2. Q = C Vand^{-1}, Vand[m][k] = tau_m^k, C[m][k] = tau_m^{k+1}/(k+1)
  LD Vd[2 * MAXM][2 * MAXM], Vi[2 * MAXM][2 * MAXM];
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < M; ++k) Vd[m][k] = powl(tau[m], k);
  if (!invert(M, Vd, Vi)) return -3;  // Vi[k][j]: coefficient of s^k in l_j
  LD Q[MAXM][MAXM];
  for (int m = 0; m < M; ++m)
    for (int j = 0; j < M; ++j) {
      LD acc = 0;
      for (int k = 0; k < M; ++k) acc += powl(tau[m], k + 1) / (k + 1) * Vi[k][j];
      Q[m][j] = acc;
    }
  // 3. eigenvalues: reciprocals of the roots of det(I - zQ), the denominator
  //    of the Pade (M-1, M) approximant of exp: sum_j (-1)^j (2M-1-j)! M! /
  //    ((2M-1)! j! (M-j)!) z^j.  Roots by the Weierstrass (Durand-Kerner)
  //    iteration, polished by Newton.
  LD coef[MAXM + 1];
  for (int j = 0; j <= M; ++j) {
    LD v = tgammal(2 * M - j) * tgammal(M + 1) / (tgammal(2 * M) * tgammal(j + 1) * tgammal(M - j + 1));
    coef[j] = (j & 1) ? -v : v;
  }
  auto poly = [&](CLD z, CLD* dz) {
    CLD p = coef[M], d = 0;
    for (int j = M - 1; j >= 0; --j) {
      d = d * z + p;
      p = p * z + coef[j];
    }
    if (dz) *dz = d;
    return p;
  };
  CLD roots[MAXM];
  {
    LD bound = 0;
    for (int j = 0; j < M; ++j) bound = std::max(bound, fabsl(coef[j] / coef[M]));
    bound += 1;
    const CLD seed(0.4L, 0.9L);
    CLD pw(1, 0);
    for (int k = 0; k < M; ++k) {
      pw *= seed;
      roots[k] = pw * bound;
    }
    for (int it = 0; it < 2000; ++it) {
      LD change = 0;
      for (int k = 0; k < M; ++k) {
        CLD den = coef[M];
        for (int j = 0; j < M; ++j)
          if (j != k) den *= (roots[k] - roots[j]);
        const CLD step = poly(roots[k], nullptr) / den;
        roots[k] -= step;
        change = std::max(change, std::abs(step) / std::max(std::abs(roots[k]), (LD)1));
      }
      if (change < 1e-18L) break;
    }
    for (int k = 0; k < M; ++k)
      for (int it = 0; it < 3; ++it) {
        CLD d;
        const CLD f = poly(roots[k], &d);
        if (std::abs(d) > 0) roots[k] -= f / d;
      }
  }
  // order: real first (ascending), then complex with Im > 0 (ascending real
  // part) each followed by its exact conjugate
  CLD lam[MAXM];
  int nl = 0;
  {
    CLD ev[MAXM];
    for (int k = 0; k < M; ++k) ev[k] = CLD(1, 0) / roots[k];
    const LD tol = 1e-12L;
    bool used[MAXM] = {false};
    for (int pass = 0; pass < M; ++pass) {  // reals ascending
      int best = -1;
      for (int k = 0; k < M; ++k)
        if (!used[k] && fabsl(ev[k].imag()) <= tol && (best < 0 || ev[k].real() < ev[best].real())) best = k;
      if (best < 0) break;
      used[best] = true;
      lam[nl++] = CLD(ev[best].real(), 0);
    }
    for (int pass = 0; pass < M; ++pass) {
      int best = -1;
      for (int k = 0; k < M; ++k)
        if (!used[k] && ev[k].imag() > tol && (best < 0 || ev[k].real() < ev[best].real())) best = k;
      if (best < 0) break;
      used[best] = true;
      // its conjugate partner
      int cj = -1;
      for (int k = 0; k < M; ++k)
        if (!used[k] && ev[k].imag() < -tol &&
            (cj < 0 || std::abs(ev[k] - std::conj(ev[best])) < std::abs(ev[cj] - std::conj(ev[best]))))
          cj = k;
      if (cj < 0) return -4;
      used[cj] = true;
      lam[nl++] = ev[best];
      lam[nl++] = std::conj(ev[best]);
    }
    if (nl != M) return -4;
  }
  // eigenvectors by inverse iteration (real for real lambda; conjugate pairs)
  CLD V[MAXM][MAXM], Vinv[MAXM][MAXM];
  for (int p = 0; p < M; ++p) {
    if (p > 0 && lam[p].imag() < 0) {
      for (int r = 0; r < M; ++r) V[r][p] = std::conj(V[r][p - 1]);
      continue;
    }
    const CLD sigma = lam[p] * (LD)(1 + 1e-12L) + (LD)1e-14L;
    CLD A[MAXM][MAXM], Ai[MAXM][MAXM];
    for (int r = 0; r < M; ++r)
      for (int cc = 0; cc < M; ++cc) A[r][cc] = CLD(Q[r][cc], 0) - (r == cc ? sigma : CLD(0, 0));
    if (!cinvert(M, A, Ai)) return -5;
    CLD v[MAXM];
    for (int r = 0; r < M; ++r) v[r] = CLD(1 + 0.1L * r, 0);
    for (int it = 0; it < 4; ++it) {
      CLD w[MAXM];
      LD big = 0;
      int bi = 0;
      for (int r = 0; r < M; ++r) {
        w[r] = 0;
        for (int cc = 0; cc < M; ++cc) w[r] += Ai[r][cc] * v[cc];
        if (std::abs(w[r]) > big) { big = std::abs(w[r]); bi = r; }
      }
      const CLD nrm = w[bi];
      for (int r = 0; r < M; ++r) v[r] = w[r] / nrm;
    }
    if (lam[p].imag() == 0)
      for (int r = 0; r < M; ++r) v[r] = CLD(v[r].real(), 0);
    for (int r = 0; r < M; ++r) V[r][p] = v[r];
  }
  if (!cinvert(M, V, Vinv)) return -6;
  // 4. DG matrix K(i,j) = -int l_i' l_j + l_i(1) l_j(1) from the monomial
  //    coefficients Vi[k][j] of l_j, and the slab-bisection transfers
  LD Kd[2 * MAXM][2 * MAXM], Kinv[2 * MAXM][2 * MAXM];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      LD integ = 0, li1 = 0, lj1 = 0;
      for (int k = 1; k < M; ++k)
        for (int l = 0; l < M; ++l) integ += k * Vi[k][i] * Vi[l][j] / (LD)(k + l);
      for (int k = 0; k < M; ++k) { li1 += Vi[k][i]; lj1 += Vi[k][j]; }
      Kd[i][j] = -integ + li1 * lj1;
    }
  if (!invert(M, Kd, Kinv)) return -7;
  LD P[2 * MAXM][MAXM];
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < M; ++j)
      for (int m = 0; m < M; ++m) P[a * M + j][m] = lagrange(tau, M, m, (a + tau[j]) / 2);
  // R = K^{-1} P^T blockdiag(K, K)
  for (int m = 0; m < M; ++m)
    for (int kk = 0; kk < 2 * M; ++kk) {
      const int a = kk / M, j = kk % M;
      LD acc = 0;
      for (int i = 0; i < M; ++i) {
        LD t = 0;  // (P^T blockdiag(K,K))[i][kk] = sum_l P[a M + l][i] K[l][j]
        for (int l = 0; l < M; ++l) t += P[a * M + l][i] * Kd[l][j];
        acc += Kinv[m][i] * t;
      }
      c.Rt[m][kk] = (double)acc;
    }
  for (int kk = 0; kk < 2 * M; ++kk)
    for (int m = 0; m < M; ++m) c.Pt[kk][m] = (double)P[kk][m];
  for (int m = 0; m < M; ++m) {
    c.tau[m] = (double)tau[m];
    c.lam[m] = std::complex<double>((double)lam[m].real(), (double)lam[m].imag());
    for (int j = 0; j < M; ++j) {
      c.Q[m][j] = (double)Q[m][j];
      c.K[m][j] = (double)Kd[m][j];
      c.V[m][j] = std::complex<double>((double)V[m][j].real(), (double)V[m][j].imag());
      c.Vinv[m][j] = std::complex<double>((double)Vinv[m][j].real(), (double)Vinv[m][j].imag());
    }
  }
  // 5. SDC preconditioners
  for (int m = 0; m < MAXM; ++m)
    for (int j = 0; j < MAXM; ++j) { c.QI_ie[m][j] = 0; c.QI_lu[m][j] = 0; c.QE[m][j] = 0; }
  for (int m = 0; m < M; ++m)
    for (int j = 0; j < M; ++j) {
      const LD dj = tau[j] - (j ? tau[j - 1] : 0);
      if (j <= m) c.QI_ie[m][j] = (double)dj;
      if (j < m) c.QE[m][j] = (double)(tau[j + 1] - tau[j]);
    }
  {
    // Doolittle Q^T = L U (unit lower L), QI = U^T
    LD A[MAXM][MAXM], L[MAXM][MAXM], U[MAXM][MAXM];
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) { A[i][j] = Q[j][i]; L[i][j] = (i == j); U[i][j] = 0; }
    for (int k = 0; k < M; ++k) {
      for (int j = k; j < M; ++j) {
        LD s = A[k][j];
        for (int t = 0; t < k; ++t) s -= L[k][t] * U[t][j];
        U[k][j] = s;
      }
      for (int i = k + 1; i < M; ++i) {
        LD s = A[i][k];
        for (int t = 0; t < k; ++t) s -= L[i][t] * U[t][k];
        L[i][k] = s / U[k][k];
      }
    }
    for (int m = 0; m < M; ++m)
      for (int j = 0; j < M; ++j) c.QI_lu[m][j] = (double)U[j][m];
  }
  *out = c;
  return 0;
}

int node_transfer_setup(int Mf, int Mc, double P[MAXM][MAXM], double R[MAXM][MAXM]) {
  if (Mf < 1 || Mc < 1 || Mf > MAXM || Mc > Mf) return -1;
  Colloc cf, cc;
  if (colloc_setup(Mf, &cf) != 0 || colloc_setup(Mc, &cc) != 0) return -2;
  LD tc[MAXM];
  for (int m = 0; m < Mc; ++m) tc[m] = cc.tau[m];
  LD Pl[MAXM][MAXM];
  for (int j = 0; j < Mf; ++j)
    for (int m = 0; m < Mc; ++m) Pl[j][m] = lagrange(tc, Mc, m, (LD)cf.tau[j]);
  LD Kc[2 * MAXM][2 * MAXM], Kci[2 * MAXM][2 * MAXM];
  for (int a = 0; a < Mc; ++a)
    for (int b = 0; b < Mc; ++b) Kc[a][b] = cc.K[a][b];
  if (!invert(Mc, Kc, Kci)) return -3;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) P[a][b] = R[a][b] = 0.0;
  for (int j = 0; j < Mf; ++j)
    for (int m = 0; m < Mc; ++m) P[j][m] = (double)Pl[j][m];
  // R = Kc^{-1} (P^T Kf)
  for (int m = 0; m < Mc; ++m)
    for (int j = 0; j < Mf; ++j) {
      LD acc = 0;
      for (int i = 0; i < Mc; ++i) {
        LD t = 0;
        for (int l = 0; l < Mf; ++l) t += Pl[l][i] * (LD)cf.K[l][j];
        acc += Kci[m][i] * t;
      }
      R[m][j] = (double)acc;
    }
  return 0;
}

int node_eval_setup(int Mfrom, int Mto, double X[MAXM][MAXM]) {
  if (Mfrom < 1 || Mto < 1 || Mfrom > MAXM || Mto > MAXM) return -1;
  Colloc cf, ct;
  if (colloc_setup(Mfrom, &cf) != 0 || colloc_setup(Mto, &ct) != 0) return -2;
  LD tf[MAXM];
  for (int m = 0; m < Mfrom; ++m) tf[m] = cf.tau[m];
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) X[a][b] = 0.0;
  for (int i = 0; i < Mto; ++i)
    for (int j = 0; j < Mfrom; ++j) X[i][j] = (double)lagrange(tf, Mfrom, j, (LD)ct.tau[i]);
  return 0;
}

}  // namespace st
