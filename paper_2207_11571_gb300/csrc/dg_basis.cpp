// Host construction of the 1D Gauss-Lobatto basis (nodal DGSEM, Sec. 2.6) and of
// the modal filter G (Eq. 2, Sec. 2.6), in FP64.
#include <cmath>
#include <cstring>

#include "dg_common.h"

namespace dgnn {

namespace {

// Legendre polynomial L_P(x) and its derivative by the three-term recurrence.
template <typename R>
void legendre(int P, R x, R* L, R* dL) {
  R l0 = 1, l1 = x, d0 = 0, d1 = 1;
  if (P == 0) { *L = 1; *dL = 0; return; }
  for (int k = 1; k < P; ++k) {
    R l2 = ((2 * k + 1) * x * l1 - k * l0) / (k + 1);
    R d2 = d0 + (2 * k + 1) * l1;
    l0 = l1; l1 = l2; d0 = d1; d1 = d2;
  }
  *L = l1;
  *dL = d1;
}

// Solve A X = B in place by Gauss-Jordan with partial pivoting (A n x n, B n x m).
bool gauss_jordan(int n, double* A, int m, double* B) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (std::fabs(A[piv * n + c]) < 1e-300) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      for (int k = 0; k < m; ++k) std::swap(B[c * m + k], B[piv * m + k]);
    }
    double inv = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) A[c * n + k] *= inv;
    for (int k = 0; k < m; ++k) B[c * m + k] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
    }
  }
  return true;
}

}  // namespace

int build_basis(int P, Basis1D* b) {
  if (P < 1 || P > kMaxP) return fail(DG_ERR_INVALID_ARG, "polynomial order must be in [1, 8]");
  // Everything in extended precision (long double), rounded once to FP64 at the end,
  // so that the FP64 tables are (nearly always) the correctly rounded values.
  using R = long double;
  const int n = P + 1;
  R xi[kMaxN1], w[kMaxN1];
  // Nodes: x_0 = -1, x_P = 1, interior roots of L_P' found by Newton on
  // f(x) = (1 - x^2) L_P'(x), whose derivative is -P (P+1) L_P(x) (Legendre's ODE).
  const R pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j < n; ++j) {
    R x = -std::cos(pi * j / P);
    if (j > 0 && j < P) {
      for (int it = 0; it < 200; ++it) {
        R L, dL;
        legendre<R>(P, x, &L, &dL);
        R dx = (1 - x * x) * dL / (-(R)P * (P + 1) * L);
        x -= dx;
        if (std::fabs((double)dx) < 1e-30) break;
      }
    }
    xi[j] = x;
  }
  // symmetrise against round-off
  for (int j = 0; j < n / 2; ++j) {
    R a = (xi[P - j] - xi[j]) / 2;
    xi[j] = -a;
    xi[P - j] = a;
  }
  if (n % 2) xi[P / 2] = 0;
  for (int j = 0; j < n; ++j) {
    R L, dL;
    legendre<R>(P, xi[j], &L, &dL);
    w[j] = 2 / ((R)P * (P + 1) * L * L);
  }
  // Derivative matrix by barycentric weights: D_ij = (lam_j / lam_i) / (x_i - x_j),
  // D_ii = -sum_{j != i} D_ij.
  R lam[kMaxN1];
  for (int j = 0; j < n; ++j) {
    R p = 1;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (xi[j] - xi[k]);
    lam[j] = 1 / p;
  }
  b->P = P;
  for (int i = 0; i < n; ++i) {
    R diag = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      R v = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      b->D[i * n + j] = (double)v;
      diag -= v;
    }
    b->D[i * n + i] = (double)diag;
    b->xi[i] = (double)xi[i];
    b->w[i] = (double)w[i];
  }
  return DG_OK;
}

int build_filter(int P_hi, int P_lo, double* G) {
  if (P_lo < 1 || P_lo > P_hi || P_hi > kMaxP)
    return fail(DG_ERR_INVALID_ARG, "filter needs 1 <= P_lo <= P_hi <= 8");
  Basis1D hi, lo;
  int st = build_basis(P_hi, &hi);
  if (st) return st;
  st = build_basis(P_lo, &lo);
  if (st) return st;
  const int nh = P_hi + 1, nl = P_lo + 1;
  // Vandermonde V[j][m] = L_m(xi_j); modal coefficients = V^{-1} nodal.
  double V[kMaxN1 * kMaxN1], Vinv[kMaxN1 * kMaxN1];
  for (int j = 0; j < nh; ++j)
    for (int m = 0; m < nh; ++m) {
      double L, dL;
      legendre<double>(m, hi.xi[j], &L, &dL);
      V[j * nh + m] = L;
      Vinv[j * nh + m] = (j == m) ? 1.0 : 0.0;
    }
  if (!gauss_jordan(nh, V, nh, Vinv)) return fail(DG_ERR_INVALID_ARG, "singular Vandermonde");
  // G[a][j] = sum_{m <= P_lo} L_m(xi_lo_a) Vinv[m][j]
  for (int a = 0; a < nl; ++a)
    for (int j = 0; j < nh; ++j) {
      double s = 0.0;
      for (int m = 0; m < nl; ++m) {
        double L, dL;
        legendre<double>(m, lo.xi[a], &L, &dL);
        s += L * Vinv[m * nh + j];
      }
      G[a * nh + j] = s;
    }
  return DG_OK;
}

int build_prolongation(int P_lo, int P_hi, double* I) {
  if (P_lo < 1 || P_lo > P_hi || P_hi > kMaxP)
    return fail(DG_ERR_INVALID_ARG, "prolongation needs 1 <= P_lo <= P_hi <= 8");
  Basis1D hi, lo;
  int st = build_basis(P_hi, &hi);
  if (st) return st;
  st = build_basis(P_lo, &lo);
  if (st) return st;
  const int nh = P_hi + 1, nl = P_lo + 1;
  for (int a = 0; a < nh; ++a)
    for (int j = 0; j < nl; ++j) {
      long double l = 1.0L;
      for (int k = 0; k < nl; ++k)
        if (k != j) l *= ((long double)hi.xi[a] - lo.xi[k]) / ((long double)lo.xi[j] - lo.xi[k]);
      I[a * nl + j] = (double)l;
    }
  return DG_OK;
}

}  // namespace dgnn
