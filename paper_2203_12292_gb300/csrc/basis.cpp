// One-dimensional finite-element tables for Q_k (k = 1..4), computed once on
// the host in fp64.
//
// * Support points: Gauss-Lobatto-Legendre points (the end points and the
//   roots of P_k'), the support points of the paper's continuous Lagrange
//   elements (Sec. 5 set-up: tensor products of 1D elements of degree k).
// * Quadrature: Gauss-Legendre with k+1 points per direction (Sec. 5).
// * M, K: the 1D mass and stiffness matrices by that quadrature (exact for the
//   degree-2k and 2k-2 integrands).
// * B, lam: the generalised eigen-decomposition S^T M S = I, S^T K S = diag(lam)
//   with B = S^{-1}.  For an axis-parallel cube of edge h the cell operator
//   S_e^T Q_e S_e of Eq. 2 equals h (K x M x M + M x K x M + M x M x K) and
//   therefore h B'^{(x)3} diag(lam_i + lam_j + lam_l) B^{(x)3} (fast
//   diagonalisation, Lynch, Rice & Thomas, Numer. Math. 6, 1964).
// * I[p]: interpolation from a coarse edge onto the half p of that edge, used
//   for hanging-node constraints (Sec. 3.2, in-place interpolation on
//   hanging faces and edges).
// * Ph, p_prolongation: element prolongation matrices of Sec. 3.5; for nested
//   spaces M_f^{-1}(phi_f, phi_c) is interpolation at the fine support points.
#include <cmath>
#include <cstring>
#include <mutex>
#include <stdexcept>

#include "internal.h"

namespace gcmg {

namespace {

// Legendre P_n and P_n' at x (three-term recurrence)
void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int m = 2; m <= n; ++m) {
    double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_lobatto(int k, double* xi) {
  // interior points: roots of P_k', Newton with P_k'' from Legendre's equation
  xi[0] = -1.0;
  xi[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double x = -std::cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, x, p, dp);
      double d2p = (2.0 * x * dp - k * (k + 1.0) * p) / (1.0 - x * x);
      double dx = dp / d2p;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    xi[i] = x;
  }
  for (int i = 0; i <= k; ++i) xi[i] = 0.5 * (xi[i] + 1.0);
  double tmp[NMAX];
  for (int i = 0; i <= k; ++i) tmp[i] = 0.5 * (xi[i] + 1.0 - xi[k - i]);
  for (int i = 0; i <= k; ++i) xi[i] = tmp[i];
  xi[0] = 0.0;
  xi[k] = 1.0;
  if (k % 2 == 0) xi[k / 2] = 0.5;
}

void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double p = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, p, dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    legendre(n, t, p, dp);
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/(..) on [-1,1], halved
  }
}

double lagrange_deriv(const double* nodes, int n, int a, double t) {
  double s = 0.0;
  for (int c = 0; c < n; ++c) {
    if (c == a) continue;
    double term = 1.0 / (nodes[a] - nodes[c]);
    for (int b = 0; b < n; ++b)
      if (b != a && b != c) term *= (t - nodes[b]) / (nodes[a] - nodes[b]);
    s += term;
  }
  return s;
}

// cyclic Jacobi eigenvalue iteration for a symmetric n x n matrix
void jacobi_eigen(int n, double A[NMAX][NMAX], double V[NMAX][NMAX], double* ev) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i][j] * A[i][j];
    if (off < 1e-60) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (std::fabs(A[p][q]) < 1e-300) continue;
        double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {  // A <- A J
          double arp = A[r][p], arq = A[r][q];
          A[r][p] = c * arp - s * arq;
          A[r][q] = s * arp + c * arq;
        }
        for (int r = 0; r < n; ++r) {  // A <- J^T A
          double apr = A[p][r], aqr = A[q][r];
          A[p][r] = c * apr - s * aqr;
          A[q][r] = s * apr + c * aqr;
        }
        for (int r = 0; r < n; ++r) {
          double vrp = V[r][p], vrq = V[r][q];
          V[r][p] = c * vrp - s * vrq;
          V[r][q] = s * vrp + c * vrq;
        }
      }
  }
  for (int i = 0; i < n; ++i) ev[i] = A[i][i];
}

Basis1D make_basis(int k) {
  Basis1D b{};
  b.k = k;
  const int n = k + 1;
  gauss_lobatto(k, b.xi);
  gauss_legendre(n, b.gq, b.gw);
  for (int q = 0; q < n; ++q)
    for (int a = 0; a < n; ++a) b.Pq[q][a] = lagrange(b.xi, n, a, b.gq[q]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double m = 0.0, s = 0.0;
      for (int q = 0; q < n; ++q) {
        m += b.gw[q] * lagrange(b.xi, n, i, b.gq[q]) * lagrange(b.xi, n, j, b.gq[q]);
        s += b.gw[q] * lagrange_deriv(b.xi, n, i, b.gq[q]) * lagrange_deriv(b.xi, n, j, b.gq[q]);
      }
      b.M[i][j] = m;
      b.K[i][j] = s;
    }
  // generalised eigenproblem via M = L L^T, C = L^{-1} K L^{-T}
  double L[NMAX][NMAX] = {};
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = b.M[i][j];
      for (int m = 0; m < j; ++m) s -= L[i][m] * L[j][m];
      L[i][j] = (i == j) ? std::sqrt(s) : s / L[j][j];
    }
  double Li[NMAX][NMAX] = {};  // L^{-1}
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int m = 0; m < i; ++m) s -= L[i][m] * Li[m][c];
      Li[i][c] = s / L[i][i];
    }
  double C[NMAX][NMAX] = {}, T[NMAX][NMAX] = {};
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int m = 0; m < n; ++m) s += Li[i][m] * b.K[m][j];
      T[i][j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int m = 0; m < n; ++m) s += T[i][m] * Li[j][m];
      C[i][j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) C[i][j] = C[j][i] = 0.5 * (C[i][j] + C[j][i]);
  double Q[NMAX][NMAX], ev[NMAX];
  jacobi_eigen(n, C, Q, ev);
  // sort ascending, deterministic sign (largest-magnitude entry positive)
  int order[NMAX];
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (ev[order[j]] < ev[order[i]]) std::swap(order[i], order[j]);
  for (int r = 0; r < n; ++r) {
    int c = order[r];
    int big = 0;
    for (int m = 1; m < n; ++m)
      if (std::fabs(Q[m][c]) > std::fabs(Q[big][c]) + 1e-12) big = m;
    double sg = Q[big][c] < 0 ? -1.0 : 1.0;
    b.lam[r] = ev[c] < 0 && ev[c] > -1e-12 ? 0.0 : ev[c];
    // B = Q^T L^T: row r = (Q[:,c])^T L^T
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int m = 0; m < n; ++m) s += Q[m][c] * L[j][m];
      b.B[r][j] = sg * s;
    }
  }
  for (int p = 0; p < 2; ++p)
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) b.I[p][a][c] = lagrange(b.xi, n, c, 0.5 * (p + b.xi[a]));
  for (int i = 0; i <= 2 * k; ++i) {
    double t = (i <= k) ? 0.5 * b.xi[i] : 0.5 * (1.0 + b.xi[i - k]);
    for (int a = 0; a < n; ++a) b.Ph[i][a] = lagrange(b.xi, n, a, t);
  }
  return b;
}

std::once_flag g_once;
Basis1D g_basis[KMAX + 1];

}  // namespace

double lagrange(const double* nodes, int n, int a, double t) {
  double v = 1.0;
  for (int b = 0; b < n; ++b)
    if (b != a) v *= (t - nodes[b]) / (nodes[a] - nodes[b]);
  return v;
}

const Basis1D& basis(int k) {
  if (k < 1 || k > KMAX) throw std::runtime_error("degree out of range 1..4");
  std::call_once(g_once, [] {
    for (int kk = 1; kk <= KMAX; ++kk) g_basis[kk] = make_basis(kk);
  });
  return g_basis[k];
}

void p_prolongation(int kf, int kc, double P[NMAX][NMAX]) {
  const Basis1D& f = basis(kf);
  const Basis1D& c = basis(kc);
  for (int i = 0; i < NMAX; ++i)
    for (int a = 0; a < NMAX; ++a) P[i][a] = 0.0;
  for (int i = 0; i <= kf; ++i)
    for (int a = 0; a <= kc; ++a) P[i][a] = lagrange(c.xi, kc + 1, a, f.xi[i]);
}

}  // namespace gcmg
