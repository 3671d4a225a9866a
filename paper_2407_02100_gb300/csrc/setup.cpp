// Host-side set-up math; see setup.h.  Written for FP64 accuracy: the
// Legendre roots are Newton-polished, the eigen solver is cyclic Jacobi run
// to convergence, so T and lambda are accurate to a few ulps.
#include "setup.h"

#include <cmath>
#include <stdexcept>

namespace gmg {

// Legendre P_n and its first two derivatives at x in [-1, 1].
static void legendre(int n, double x, double& p, double& dp, double& ddp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { p = 1.0; dp = 0.0; ddp = 0.0; return; }
  for (int j = 2; j <= n; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  // derivative from (1 - x^2) P_n' = n (P_{n-1} - x P_n), valid off +-1
  dp = n * (p0 - x * p1) / (1.0 - x * x);
  // Legendre ODE: (1 - x^2) P'' - 2 x P' + n (n + 1) P = 0
  ddp = (2.0 * x * dp - n * (n + 1.0) * p1) / (1.0 - x * x);
}

std::vector<double> gauss_lobatto(int k) {
  std::vector<double> x(k + 1);
  x[0] = 0.0;
  x[k] = 1.0;
  // interior points: roots of P_k' on (-1, 1); Newton from Chebyshev-Gauss-
  // Lobatto guesses with f = P_k', f' = P_k''.
  for (int i = 1; i < k; ++i) {
    double t = -std::cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp, ddp;
      legendre(k, t, p, dp, ddp);
      double step = dp / ddp;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
  // symmetrise exactly around 1/2
  for (int i = 1; i < k; ++i) {
    double a = x[i], b = 1.0 - x[k - i];
    x[i] = 0.5 * (a + b);
  }
  if (k % 2 == 0) x[k / 2] = 0.5;
  return x;
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double p = 0, dp = 0, ddp = 0;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, p, dp, ddp);
      double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    legendre(n, t, p, dp, ddp);
    x[i] = 0.5 * (t + 1.0);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);  // 2/((1-t^2)P'^2) scaled to [0,1]
  }
}

double lagrange(const std::vector<double>& nodes, int p, double t, int deriv) {
  const int n = (int)nodes.size();
  if (deriv == 0) {
    double v = 1.0;
    for (int r = 0; r < n; ++r)
      if (r != p) v *= (t - nodes[r]) / (nodes[p] - nodes[r]);
    return v;
  }
  double s = 0.0;
  for (int q = 0; q < n; ++q) {
    if (q == p) continue;
    double v = 1.0 / (nodes[p] - nodes[q]);
    for (int r = 0; r < n; ++r)
      if (r != p && r != q) v *= (t - nodes[r]) / (nodes[p] - nodes[r]);
    s += v;
  }
  return s;
}

void cell_matrices_1d(int k, std::vector<double>& M, std::vector<double>& K) {
  const int n = k + 1;
  std::vector<double> nodes = gauss_lobatto(k), xq, wq;
  gauss_legendre(k + 1, xq, wq);  // exact for degree 2k integrands
  M.assign(n * n, 0.0);
  K.assign(n * n, 0.0);
  for (int q = 0; q < k + 1; ++q) {
    std::vector<double> v(n), d(n);
    for (int i = 0; i < n; ++i) {
      v[i] = lagrange(nodes, i, xq[q], 0);
      d[i] = lagrange(nodes, i, xq[q], 1);
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        M[i * n + j] += wq[q] * v[i] * v[j];
        K[i * n + j] += wq[q] * d[i] * d[j];
      }
  }
}

void assembled_1d(int k, int ncells, int r0, int nr, int c0, int nc,
                  std::vector<double>& M, std::vector<double>& K) {
  std::vector<double> Mc, Kc;
  cell_matrices_1d(k, Mc, Kc);
  M.assign((size_t)nr * nc, 0.0);
  K.assign((size_t)nr * nc, 0.0);
  for (int c = 0; c < ncells; ++c)
    for (int i = 0; i <= k; ++i)
      for (int j = 0; j <= k; ++j) {
        int gi = c * k + i - r0, gj = c * k + j - c0;
        if (gi < 0 || gi >= nr || gj < 0 || gj >= nc) continue;
        M[(size_t)gi * nc + gj] += Mc[i * (k + 1) + j];
        K[(size_t)gi * nc + gj] += Kc[i * (k + 1) + j];
      }
}

bool generalized_eigen(int n, const std::vector<double>& M, const std::vector<double>& K,
                       std::vector<double>& T, std::vector<double>& lambda) {
  // Cholesky M = L L^T
  std::vector<double> L(n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int p = 0; p < j; ++p) s -= L[j * n + p] * L[j * n + p];
    if (!(s > 0.0)) return false;
    L[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int p = 0; p < j; ++p) t -= L[i * n + p] * L[j * n + p];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  // Linv = L^{-1} (lower triangular) by forward substitution
  std::vector<double> Li(n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int p = 0; p < i; ++p) s -= L[i * n + p] * Li[p * n + c];
      Li[i * n + c] = s / L[i * n + i];
    }
  }
  // C = Linv K Linv^T (symmetric)
  std::vector<double> tmp(n * n, 0.0), C(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int p = 0; p < n; ++p) s += Li[i * n + p] * K[p * n + j];
      tmp[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int p = 0; p < n; ++p) s += tmp[i * n + p] * Li[j * n + p];
      C[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) C[i * n + j] = C[j * n + i] = 0.5 * (C[i * n + j] + C[j * n + i]);
  // cyclic Jacobi: C = Q diag Q^T
  std::vector<double> Q(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += C[i * n + i] * C[i * n + i];
      for (int j = i + 1; j < n; ++j) off += C[i * n + j] * C[i * n + j];
    }
    if (off <= 1e-34 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = C[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (C[q * n + q] - C[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {  // columns p, q
          double crp = C[r * n + p], crq = C[r * n + q];
          C[r * n + p] = c * crp - s * crq;
          C[r * n + q] = s * crp + c * crq;
        }
        for (int r = 0; r < n; ++r) {  // rows p, q
          double cpr = C[p * n + r], cqr = C[q * n + r];
          C[p * n + r] = c * cpr - s * cqr;
          C[q * n + r] = s * cpr + c * cqr;
        }
        for (int r = 0; r < n; ++r) {
          double qrp = Q[r * n + p], qrq = Q[r * n + q];
          Q[r * n + p] = c * qrp - s * qrq;
          Q[r * n + q] = s * qrp + c * qrq;
        }
      }
  }
  lambda.assign(n, 0.0);
  for (int i = 0; i < n; ++i) lambda[i] = C[i * n + i];
  // T = L^{-T} Q  (T[i][j] = sum_p Linv[p][i] Q[p][j])
  T.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int p = 0; p < n; ++p) s += Li[p * n + i] * Q[p * n + j];
      T[i * n + j] = s;
    }
  return true;
}

bool generalized_eigen_mirror(int n, const std::vector<double>& M, const std::vector<double>& K,
                              std::vector<double>& T, std::vector<double>& lambda) {
  if (n % 2 == 0) return false;
  const int c = (n - 1) / 2, ne = c + 1, no = c;
  const double r = 1.0 / std::sqrt(2.0);
  // orthonormal mirror bases: E (n x ne), O (n x no)
  std::vector<double> E(n * ne, 0.0), O(n * no, 0.0);
  for (int j = 0; j < c; ++j) {
    E[j * ne + j] = r;
    E[(n - 1 - j) * ne + j] = r;
    O[j * no + j] = r;
    O[(n - 1 - j) * no + j] = -r;
  }
  E[c * ne + c] = 1.0;
  auto project = [&](const std::vector<double>& B, const std::vector<double>& A, int nb) {
    std::vector<double> out(nb * nb, 0.0);  // B^T A B
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        double s2 = 0.0;
        for (int p = 0; p < n; ++p)
          for (int q = 0; q < n; ++q) s2 += B[p * nb + i] * A[p * n + q] * B[q * nb + j];
        out[i * nb + j] = s2;
      }
    return out;
  };
  std::vector<double> Te, le, To, lo;
  if (!generalized_eigen(ne, project(E, M, ne), project(E, K, ne), Te, le)) return false;
  if (no > 0 && !generalized_eigen(no, project(O, M, no), project(O, K, no), To, lo)) return false;
  T.assign(n * n, 0.0);
  lambda.assign(n, 0.0);
  for (int i = 0; i < ne; ++i) {
    lambda[i] = le[i];
    for (int j = 0; j < n; ++j) {
      double s2 = 0.0;
      for (int p = 0; p < ne; ++p) s2 += E[j * ne + p] * Te[p * ne + i];
      T[j * n + i] = s2;
    }
  }
  for (int i = 0; i < no; ++i) {
    lambda[ne + i] = lo[i];
    for (int j = 0; j < n; ++j) {
      double s2 = 0.0;
      for (int p = 0; p < no; ++p) s2 += O[j * no + p] * To[p * no + i];
      T[j * n + ne + i] = s2;
    }
  }
  return true;
}

void assemble_dense_var(int dim, int k, int n, const double* coef, std::vector<double>& A) {
  std::vector<double> Mc, Kc;
  cell_matrices_1d(k, Mc, Kc);
  const int N = n * k + 1, m = N - 2, E = k + 1;
  const long long ni = dim == 3 ? (long long)m * m * m : (long long)m * m;
  const double hs = dim == 3 ? 1.0 / n : 1.0;  // h^{d-2}
  A.assign(ni * ni, 0.0);
  const int nloc = dim == 3 ? E * E * E : E * E;
  const long long ncell = dim == 3 ? (long long)n * n * n : (long long)n * n;
  for (long long c = 0; c < ncell; ++c) {
    const int cc[3] = {(int)(c % n), (int)((c / n) % n), dim == 3 ? (int)(c / ((long long)n * n)) : 0};
    const double a = coef[c] * hs;
    for (int pi = 0; pi < nloc; ++pi) {
      const int li[3] = {pi % E, (pi / E) % E, dim == 3 ? pi / (E * E) : 0};
      long long I = 0, stride = 1;
      bool ok = true;
      for (int d = 0; d < dim; ++d) {
        const int g = cc[d] * k + li[d];
        if (g < 1 || g > m) ok = false;
        I += (g - 1) * stride;
        stride *= m;
      }
      if (!ok) continue;
      for (int pj = 0; pj < nloc; ++pj) {
        const int lj[3] = {pj % E, (pj / E) % E, dim == 3 ? pj / (E * E) : 0};
        long long J = 0, st2 = 1;
        bool ok2 = true;
        for (int d = 0; d < dim; ++d) {
          const int g = cc[d] * k + lj[d];
          if (g < 1 || g > m) ok2 = false;
          J += (g - 1) * st2;
          st2 *= m;
        }
        if (!ok2) continue;
        double v = 0.0;
        for (int al = 0; al < dim; ++al) {
          double prod = 1.0;
          for (int be = 0; be < dim; ++be) {
            const std::vector<double>& Ed = (al == be) ? Kc : Mc;
            prod *= Ed[li[be] * E + lj[be]];
          }
          v += prod;
        }
        A[I * ni + J] += a * v;
      }
    }
  }
}

bool spd_inverse(int n, const std::vector<double>& A, std::vector<double>& Ainv) {
  std::vector<double> L(A);
  for (int j = 0; j < n; ++j) {
    double d = L[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) d -= L[(size_t)j * n + p] * L[(size_t)j * n + p];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    L[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = L[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) t -= L[(size_t)i * n + p] * L[(size_t)j * n + p];
      L[(size_t)i * n + j] = t / d;
    }
  }
  Ainv.assign((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int c = 0; c < n; ++c) {  // solve L L^T x = e_c
    for (int i = 0; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int p = 0; p < i; ++p) t -= L[(size_t)i * n + p] * y[p];
      y[i] = t / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = y[i];
      for (int p = i + 1; p < n; ++p) t -= L[(size_t)p * n + i] * Ainv[(size_t)p * n + c];
      Ainv[(size_t)i * n + c] = t / L[(size_t)i * n + i];
    }
  }
  return true;
}

void prolongation_cell_1d(int k, std::vector<double>& P) {
  std::vector<double> xi = gauss_lobatto(k);
  P.assign((2 * k + 1) * (k + 1), 0.0);
  for (int r = 0; r <= 2 * k; ++r) {
    // fine node r of the coarse cell: fine cell r / k (0 or 1), local r % k
    double x = (r <= k) ? 0.5 * xi[r] : 0.5 + 0.5 * xi[r - k];
    for (int p = 0; p <= k; ++p) {
      P[r * (k + 1) + p] = lagrange(xi, p, x, 0);
    }
  }
}

}  // namespace gmg
