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

namespace tp {

// Global 1D DG mass M and SIPG stiffness L on nc cells of width h (dense,
// N = nc*n square, row-major): the 1D factors of Eq. (9). L = interior
// diagonal blocks, rank-2 neighbour blocks
//   L^{c,c+1} = -g v1 v0^T - v1 d0^T/(2h) + d1 v0^T/(2h),  L^{c+1,c} = its transpose,
// and boundary corrections (v0 d0^T + d0 v0^T)/(2h) at the low end,
// -(v1 d1^T + d1 v1^T)/(2h) at the high end.
void global_1d(const Ref1D& r, const Dir1D& d, int nc, std::vector<double>& M, std::vector<double>& L) {
  const int n = r.n, N = nc * n;
  M.assign((size_t)N * N, 0.0);
  L.assign((size_t)N * N, 0.0);
  const double hh = 0.5 / d.h;
  for (int c = 0; c < nc; ++c)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        M[(size_t)(c * n + i) * N + c * n + j] = d.M[i * n + j];
        L[(size_t)(c * n + i) * N + c * n + j] = d.L[i * n + j];
      }
  for (int c = 0; c + 1 < nc; ++c)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v1i = i == n - 1, v0j = j == 0;
        const double val = -d.gamma * v1i * v0j - v1i * r.d0[j] * hh + r.d1[i] * v0j * hh;
        L[(size_t)(c * n + i) * N + (c + 1) * n + j] = val;
        L[(size_t)((c + 1) * n + j) * N + c * n + i] = val;
      }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double v0i = i == 0, v0j = j == 0, v1i = i == n - 1, v1j = j == n - 1;
      L[(size_t)i * N + j] += (v0i * r.d0[j] + r.d0[i] * v0j) * hh;
      const size_t o = (size_t)(N - n);
      L[(o + i) * N + o + j] -= (v1i * r.d1[j] + r.d1[i] * v1j) * hh;
    }
}

// Generalized symmetric-definite eigenproblem L V = M V diag(lam), V^T M V = I,
// by Cholesky M = C C^T and cyclic Jacobi rotations on C^{-1} L C^{-T}.
// Returns false if M is not positive definite. V is row-major N x N with
// eigenvector k in column k.
bool gen_eig(int N, const std::vector<double>& M, const std::vector<double>& L, std::vector<double>& lam,
             std::vector<double>& V) {
  std::vector<double> C((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = M[(size_t)i * N + j];
      for (int k = 0; k < j; ++k) s -= C[(size_t)i * N + k] * C[(size_t)j * N + k];
      if (i == j) {
        if (!(s > 0)) return false;
        C[(size_t)i * N + i] = std::sqrt(s);
      } else {
        C[(size_t)i * N + j] = s / C[(size_t)j * N + j];
      }
    }
  // S = C^{-1} L C^{-T}: first X = C^{-1} L (forward substitution per column), then S = C^{-1} X^T
  std::vector<double> X((size_t)N * N), S((size_t)N * N);
  auto fwd = [&](const std::vector<double>& B, std::vector<double>& out) {  // out = C^{-1} B
    for (int col = 0; col < N; ++col)
      for (int i = 0; i < N; ++i) {
        double s = B[(size_t)i * N + col];
        for (int k = 0; k < i; ++k) s -= C[(size_t)i * N + k] * out[(size_t)k * N + col];
        out[(size_t)i * N + col] = s / C[(size_t)i * N + i];
      }
  };
  fwd(L, X);
  std::vector<double> Xt((size_t)N * N);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) Xt[(size_t)i * N + j] = X[(size_t)j * N + i];
  fwd(Xt, S);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = 0.5 * (S[(size_t)i * N + j] + S[(size_t)j * N + i]);
      S[(size_t)i * N + j] = S[(size_t)j * N + i] = a;
    }
  std::vector<double> Q((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i) Q[(size_t)i * N + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        (i == j ? diag : off) += S[(size_t)i * N + j] * S[(size_t)i * N + j];
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < N; ++p)
      for (int q = p + 1; q < N; ++q) {
        const double apq = S[(size_t)p * N + q];
        if (apq == 0.0) continue;
        const double app = S[(size_t)p * N + p], aqq = S[(size_t)q * N + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < N; ++k) {  // rows p, q
          const double skp = S[(size_t)k * N + p], skq = S[(size_t)k * N + q];
          S[(size_t)k * N + p] = c * skp - s * skq;
          S[(size_t)k * N + q] = s * skp + c * skq;
        }
        for (int k = 0; k < N; ++k) {  // columns p, q
          const double spk = S[(size_t)p * N + k], sqk = S[(size_t)q * N + k];
          S[(size_t)p * N + k] = c * spk - s * sqk;
          S[(size_t)q * N + k] = s * spk + c * sqk;
        }
        for (int k = 0; k < N; ++k) {
          const double qkp = Q[(size_t)k * N + p], qkq = Q[(size_t)k * N + q];
          Q[(size_t)k * N + p] = c * qkp - s * qkq;
          Q[(size_t)k * N + q] = s * qkp + c * qkq;
        }
      }
  }
  lam.assign(N, 0.0);
  for (int i = 0; i < N; ++i) lam[i] = S[(size_t)i * N + i];
  // V = C^{-T} Q (back substitution per column)
  V.assign((size_t)N * N, 0.0);
  for (int col = 0; col < N; ++col)
    for (int i = N - 1; i >= 0; --i) {
      double s = Q[(size_t)i * N + col];
      for (int k = i + 1; k < N; ++k) s -= C[(size_t)k * N + i] * V[(size_t)k * N + col];
      V[(size_t)i * N + col] = s / C[(size_t)i * N + i];
    }
  return true;
}

}  // namespace tp

namespace tp {

std::vector<double> invert(int n, const std::vector<double>& A) {
  std::vector<double> a(A), inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)c * n + k], a[(size_t)piv * n + k]);
        std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
      }
    const double d = a[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      a[(size_t)c * n + k] /= d;
      inv[(size_t)c * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
      }
    }
  }
  return inv;
}

}  // namespace tp
