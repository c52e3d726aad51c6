// Gauss-Lobatto-Legendre tables and Lagrange operators on the host (FP64).
//
// Reading of Sec. 2 ("DG spatial discretization"): nodal Lagrange basis on the
// n = r+1 GLL points per direction, quadrature collocated on the same points,
// so the mass matrix is diagonal (w_i J_i).  On 2:1 faces the coarse trace is
// the coarse polynomial evaluated at the fine face's GLL points.
#include <cmath>
#include <stdexcept>

#include "dg_internal.h"

namespace dg {

namespace {

// P_r(x) and P_{r-1}(x) by the three-term recurrence.
void legendre_pair(int r, double x, double* pr, double* prm1) {
  double a = 1.0, b = x;
  if (r == 0) {
    *pr = 1.0;
    *prm1 = 0.0;
    return;
  }
  for (int k = 2; k <= r; ++k) {
    double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  *pr = b;
  *prm1 = a;
}

}  // namespace

// Barycentric Lagrange evaluation: l_j(x) = (lam_j / (x - x_j)) / sum_k lam_k / (x - x_k).
void lagrange_eval(const std::vector<double>& nodes, double x, double* out) {
  const int n = (int)nodes.size();
  for (int j = 0; j < n; ++j) {
    if (x == nodes[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0 : 0.0;
      return;
    }
  }
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (nodes[j] - nodes[k]);
  double den = 0.0;
  for (int j = 0; j < n; ++j) den += lam[j] / (x - nodes[j]);
  for (int j = 0; j < n; ++j) out[j] = lam[j] / (x - nodes[j]) / den;
}

Tables1D make_tables(int r) {
  if (r < 1 || r > kMaxDegree) throw std::invalid_argument("degree out of range");
  const int n = r + 1;
  Tables1D t;
  t.degree = r;
  t.xi.assign(n, 0.0);
  t.w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  t.xi[0] = -1.0;
  t.xi[r] = 1.0;
  // interior nodes: roots of P_r'(x); Newton with P_r'' from Legendre's ODE
  for (int k = 1; k < r; ++k) {
    double x = -std::cos(pi * k / r);
    for (int it = 0; it < 100; ++it) {
      double p, q;
      legendre_pair(r, x, &p, &q);
      double dp = r * (q - x * p) / (1.0 - x * x);
      double d2p = (2.0 * x * dp - r * (r + 1.0) * p) / (1.0 - x * x);
      double step = dp / d2p;
      x -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    t.xi[k] = x;
  }
  for (int k = 0; k < n; ++k) {
    double p, q;
    legendre_pair(r, t.xi[k], &p, &q);
    t.w[k] = 2.0 / (r * (r + 1.0) * p * p);
  }
  // barycentric weights and the nodal derivative matrix
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) lam[j] /= (t.xi[j] - t.xi[k]);
  t.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      double v = (lam[k] / lam[i]) / (t.xi[i] - t.xi[k]);
      t.D[i * n + k] = v;
      diag -= v;
    }
    t.D[i * n + i] = diag;
  }
  t.Dw.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) t.Dw[i * n + k] = t.w[k] * t.D[k * n + i] / t.w[i];
  t.I.assign(2 * n * n, 0.0);
  t.It.assign(2 * n * n, 0.0);
  std::vector<double> row(n);
  for (int s = 0; s < 2; ++s) {
    for (int f = 0; f < n; ++f) {
      lagrange_eval(t.xi, 0.5 * (t.xi[f] + (2.0 * s - 1.0)), row.data());
      for (int j = 0; j < n; ++j) t.I[s * n * n + f * n + j] = row[j];
    }
    for (int i = 0; i < n; ++i)
      for (int f = 0; f < n; ++f) t.It[s * n * n + i * n + f] = (t.w[f] / t.w[i]) * t.I[s * n * n + f * n + i];
  }
  return t;
}

std::vector<double> Tables1D::packed() const {
  std::vector<double> out;
  out.insert(out.end(), D.begin(), D.end());
  out.insert(out.end(), Dw.begin(), Dw.end());
  out.insert(out.end(), I.begin(), I.end());
  out.insert(out.end(), It.begin(), It.end());
  out.insert(out.end(), w.begin(), w.end());
  out.push_back(1.0 / w[0]);
  out.insert(out.end(), xi.begin(), xi.end());
  return out;
}

}  // namespace dg
