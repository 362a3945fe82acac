// Host-side setup of the 1D operator data (Sec. 2 and Sec. 2.1, Eq. (9)).
//
// Gauss-Lobatto nodes (roots of P_k' plus the end points) and Gauss-Legendre
// points are found by Newton iteration on the three-term Legendre recurrence;
// the Lagrange basis is evaluated in barycentric form. Mass and stiffness use
// (k+1)-point Gauss-Legendre quadrature, which is exact for both integrands.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <stdexcept>

#include "tp_internal.h"

namespace tp {

namespace {

// P_m(t) and P_m'(t) on [-1, 1] by the Bonnet recurrence.
void legendre(int m, double t, double& p, double& dp) {
  double p0 = 1.0, p1 = t;
  if (m == 0) { p = 1.0; dp = 0.0; return; }
  for (int j = 2; j <= m; ++j) {
    double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
    p0 = p1; p1 = p2;
  }
  p = p1;
  dp = (std::fabs(t) < 1.0) ? m * (t * p1 - p0) / (t * t - 1.0) : 0.5 * m * (m + 1) * std::pow(t, m + 1);
}

}  // namespace

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));  // ascending initial guess
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(q, t, p, dp);
      double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double p, dp;
    legendre(q, t, p, dp);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2)P'^2) on [-1,1], halved for [0,1]
  }
}

static std::vector<double> gauss_lobatto(int k) {
  // interior points: roots of P_k'(t); Newton on f = P_k', f' from the Legendre ODE:
  // (1-t^2) P'' = 2t P' - k(k+1) P.
  std::vector<double> x(k + 1);
  x[0] = 0.0; x[k] = 1.0;
  for (int i = 1; i < k; ++i) {
    double t = -std::cos(M_PI * i / k);  // Chebyshev-Lobatto guess, ascending
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, t, p, dp);
      double d2p = (2.0 * t * dp - k * (k + 1.0) * p) / (1.0 - t * t);
      double dt = dp / d2p;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
  return x;
}

std::vector<double> lagrange_eval(const std::vector<double>& nodes, const std::vector<double>& x) {
  const int n = (int)nodes.size();
  std::vector<double> bw(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) bw[j] /= nodes[j] - nodes[m];
  std::vector<double> out(x.size() * n, 0.0);
  for (size_t p = 0; p < x.size(); ++p) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (x[p] == nodes[j]) hit = j;
    if (hit >= 0) { out[p * n + hit] = 1.0; continue; }
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += bw[j] / (x[p] - nodes[j]);
    for (int j = 0; j < n; ++j) out[p * n + j] = bw[j] / (x[p] - nodes[j]) / s;
  }
  return out;
}

// derivative of every basis function at points x: phi_j'(x) = sum_i D_ij phi_i(x)
static std::vector<double> lagrange_deriv(const std::vector<double>& nodes, const std::vector<double>& x) {
  const int n = (int)nodes.size();
  std::vector<double> bw(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) bw[j] /= nodes[j] - nodes[m];
  std::vector<double> D(n * n, 0.0);  // D[i*n+j] = phi_j'(x_i)
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) { D[i * n + j] = (bw[j] / bw[i]) / (nodes[i] - nodes[j]); diag -= D[i * n + j]; }
    D[i * n + i] = diag;
  }
  std::vector<double> V = lagrange_eval(nodes, x);
  std::vector<double> out(x.size() * n, 0.0);
  for (size_t p = 0; p < x.size(); ++p)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += V[p * n + i] * D[i * n + j];
      out[p * n + j] = s;
    }
  return out;
}

Ref1D make_ref1d(int k) {
  Ref1D r;
  r.k = k; r.n = k + 1;
  const int n = r.n;
  r.nodes = gauss_lobatto(k);
  std::vector<double> xq, wq;
  gauss_legendre(n, xq, wq);
  std::vector<double> V = lagrange_eval(r.nodes, xq), dV = lagrange_deriv(r.nodes, xq);
  r.Mhat.assign(n * n, 0.0);
  r.Khat.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double m = 0.0, s = 0.0;
      for (int q = 0; q < n; ++q) {
        m += wq[q] * V[q * n + i] * V[q * n + j];
        s += wq[q] * dV[q * n + i] * dV[q * n + j];
      }
      r.Mhat[i * n + j] = m;
      r.Khat[i * n + j] = s;
    }
  std::vector<double> ends = {0.0, 1.0};
  std::vector<double> dE = lagrange_deriv(r.nodes, ends);
  r.d0.assign(dE.begin(), dE.begin() + n);
  r.d1.assign(dE.begin() + n, dE.end());
  return r;
}

Dir1D make_dir1d(const Ref1D& r, double h, int penalty_mode) {
  const int n = r.n, k = r.k;
  Dir1D d;
  d.h = h;
  d.gamma = (penalty_mode == TP_PENALTY_PAPER) ? k * (k + 1.0) * (2.0 / h) : (k + 1.0) * (k + 1.0) / h;
  d.M.assign(n * n, 0.0);
  d.L.assign(n * n, 0.0);
  // Gauss-Lobatto nodes contain the end points, so the value traces are unit vectors.
  auto v0 = [&](int i) { return i == 0 ? 1.0 : 0.0; };
  auto v1 = [&](int i) { return i == n - 1 ? 1.0 : 0.0; };
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      d.M[i * n + j] = h * r.Mhat[i * n + j];
      double l = r.Khat[i * n + j] / h;
      l += d.gamma * (v1(i) * v1(j) + v0(i) * v0(j));
      l -= 0.5 * (v1(i) * r.d1[j] + r.d1[i] * v1(j)) / h;
      l += 0.5 * (v0(i) * r.d0[j] + r.d0[i] * v0(j)) / h;
      d.L[i * n + j] = l;
    }
  return d;
}

}  // namespace tp
