// 1D spectral-difference point sets and Lagrange operators (paper Section 3, Eqs. 13-16),
// computed on the host in double precision for one order N = p + 1.
#pragma once
#include <cmath>
#include <vector>

namespace chorus {

struct Tables1D {
  int N = 0;
  std::vector<double> Xs;    // N solution points (Eq. 13)
  std::vector<double> Xf;    // N+1 flux points: 0, roots of P_{N-1}, 1 (Eq. 14)
  std::vector<double> I;     // [N+1][N]  h_s(Xf_f)
  std::vector<double> D;     // [N][N+1]  l'_f(X_s)
  std::vector<double> Dsol;  // [N][N]    d/dX of the solution polynomial at the solution points (= D I)
  std::vector<double> Lfs;   // [N][N+1]  l_a(X_s)
  std::vector<double> Dfs;   // [N][N+1]  l'_a(X_s)
  std::vector<double> Dff;   // [N+1][N+1] l'_b(Xf_a)
  std::vector<double> w;     // N quadrature weights, integral of h_s over [0,1]
};

// Legendre polynomial L_n(t) on [-1,1] and its derivative; the shifted P_n(x) = L_n(2x-1)
// satisfies the recurrence of Eq. 14.
inline void legendre(int n, double t, double* val, double* der) {
  double l0 = 1.0, l1 = t;
  if (n == 0) { *val = 1.0; *der = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double l2 = ((2.0 * k - 1.0) * t * l1 - (k - 1.0) * l0) / k;
    l0 = l1;
    l1 = l2;
  }
  *val = l1;
  *der = n * (t * l1 - l0) / (t * t - 1.0);
}

// Lagrange cardinal polynomial of node j at x (product definition, Eqs. 15-16).
inline double lag(const std::vector<double>& x, int j, double t) {
  double r = 1.0;
  for (size_t k = 0; k < x.size(); ++k)
    if ((int)k != j) r *= (t - x[k]) / (x[j] - x[k]);
  return r;
}

// Derivative of the cardinal polynomial: l_j(t) * sum_{k != j} 1/(t - x_k) away from the nodes,
// and the barycentric node formula at a node.
inline double lag_deriv(const std::vector<double>& x, int j, double t) {
  const int n = (int)x.size();
  int at = -1;
  for (int k = 0; k < n; ++k)
    if (t == x[k]) at = k;
  if (at < 0) {
    double s = 0.0;
    for (int k = 0; k < n; ++k)
      if (k != j) s += 1.0 / (t - x[k]);
    return lag(x, j, t) * s;
  }
  auto bw = [&](int i) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != i) p *= (x[i] - x[k]);
    return 1.0 / p;
  };
  if (at != j) return (bw(j) / bw(at)) / (x[at] - x[j]);
  double s = 0.0;
  for (int k = 0; k < n; ++k)
    if (k != j) s += 1.0 / (x[j] - x[k]);
  return s;
}

inline Tables1D make_tables(int N) {
  Tables1D T;
  T.N = N;
  const double pi = 3.14159265358979323846;
  for (int s = 1; s <= N; ++s) T.Xs.push_back(0.5 * (1.0 - std::cos((2.0 * s - 1.0) / (2.0 * N) * pi)));
  // roots of L_{N-1} by Newton from the Chebyshev-like first guesses
  const int n = N - 1;
  std::vector<double> roots;
  std::vector<double> gw;
  for (int k = 1; k <= n; ++k) {
    double t = std::cos(pi * (k - 0.25) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double v, d;
      legendre(n, t, &v, &d);
      double dt = v / d;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    double v, d;
    legendre(n, t, &v, &d);
    roots.push_back(0.5 * (t + 1.0));
    gw.push_back(1.0 / ((1.0 - t * t) * d * d));  // Gauss-Legendre weight on [0,1]
  }
  // sort ascending
  for (size_t a = 0; a < roots.size(); ++a)
    for (size_t b = a + 1; b < roots.size(); ++b)
      if (roots[b] < roots[a]) { std::swap(roots[a], roots[b]); std::swap(gw[a], gw[b]); }
  T.Xf.push_back(0.0);
  for (double r : roots) T.Xf.push_back(r);
  T.Xf.push_back(1.0);
  T.I.assign((N + 1) * N, 0.0);
  T.D.assign(N * (N + 1), 0.0);
  T.Dsol.assign(N * N, 0.0);
  T.Lfs.assign(N * (N + 1), 0.0);
  T.Dfs.assign(N * (N + 1), 0.0);
  T.Dff.assign((N + 1) * (N + 1), 0.0);
  T.w.assign(N, 0.0);
  for (int f = 0; f <= N; ++f)
    for (int s = 0; s < N; ++s) T.I[f * N + s] = lag(T.Xs, s, T.Xf[f]);
  for (int s = 0; s < N; ++s)
    for (int f = 0; f <= N; ++f) {
      T.D[s * (N + 1) + f] = lag_deriv(T.Xf, f, T.Xs[s]);
      T.Lfs[s * (N + 1) + f] = lag(T.Xf, f, T.Xs[s]);
      T.Dfs[s * (N + 1) + f] = T.D[s * (N + 1) + f];
    }
  for (int a = 0; a <= N; ++a)
    for (int b = 0; b <= N; ++b) T.Dff[a * (N + 1) + b] = lag_deriv(T.Xf, b, T.Xf[a]);
  for (int i = 0; i < N; ++i)
    for (int s = 0; s < N; ++s) T.Dsol[i * N + s] = lag_deriv(T.Xs, s, T.Xs[i]);
  // weights: Gauss-Legendre rule with N-1 points is exact for the degree N-1 integrand (N >= 2)
  for (int s = 0; s < N; ++s) {
    double acc = 0.0;
    for (size_t g = 0; g < roots.size(); ++g) acc += gw[g] * lag(T.Xs, s, roots[g]);
    T.w[s] = acc;
  }
  return T;
}

}  // namespace chorus
