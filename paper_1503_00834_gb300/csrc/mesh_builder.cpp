// Host mesh builder (see mesh_builder.h).
#include "mesh_builder.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

namespace chorus {
namespace {

// natural coordinates (-1, 0, 1) of the 20 nodes in the documented local order
const int kNat[20][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {1, 1, 1},
                         {-1, 1, 1},   {0, -1, -1}, {1, 0, -1}, {0, 1, -1},  {-1, 0, -1}, {0, -1, 1}, {1, 0, 1},
                         {0, 1, 1},    {-1, 0, 1},  {-1, -1, 0}, {1, -1, 0}, {1, 1, 0},   {-1, 1, 0}};

// corner number from reference-cube corner coordinates (0/1 per axis)
int corner_of(int x, int y, int z) {
  static const int t[2][2][2] = {{{0, 4}, {3, 7}}, {{1, 5}, {2, 6}}};  // t[x][y][z]
  return t[x][y][z];
}

// serendipity shape functions and d/dxi on [0,1]^3
void shape20(double xi, double eta, double zeta, double Nv[20], double dN[20][3]) {
  const double a = 2.0 * xi - 1.0, b = 2.0 * eta - 1.0, c = 2.0 * zeta - 1.0;
  for (int i = 0; i < 20; ++i) {
    const int ai = kNat[i][0], bi = kNat[i][1], ci = kNat[i][2];
    double v, da, db, dc;
    if (ai && bi && ci) {
      const double A = 1 + a * ai, B = 1 + b * bi, C = 1 + c * ci, S = a * ai + b * bi + c * ci - 2.0;
      v = 0.125 * A * B * C * S;
      da = 0.125 * (ai * B * C * S + A * B * C * ai);
      db = 0.125 * (A * bi * C * S + A * B * C * bi);
      dc = 0.125 * (A * B * ci * S + A * B * C * ci);
    } else if (!ai) {
      const double B = 1 + b * bi, C = 1 + c * ci;
      v = 0.25 * (1 - a * a) * B * C;
      da = -0.5 * a * B * C;
      db = 0.25 * (1 - a * a) * bi * C;
      dc = 0.25 * (1 - a * a) * B * ci;
    } else if (!bi) {
      const double A = 1 + a * ai, C = 1 + c * ci;
      v = 0.25 * (1 - b * b) * A * C;
      da = 0.25 * (1 - b * b) * ai * C;
      db = -0.5 * b * A * C;
      dc = 0.25 * (1 - b * b) * A * ci;
    } else {
      const double A = 1 + a * ai, B = 1 + b * bi;
      v = 0.25 * (1 - c * c) * A * B;
      da = 0.25 * (1 - c * c) * ai * B;
      db = 0.25 * (1 - c * c) * A * bi;
      dc = -0.5 * c * A * B;
    }
    Nv[i] = v;
    dN[i][0] = 2.0 * da;
    dN[i][1] = 2.0 * db;
    dN[i][2] = 2.0 * dc;
  }
}

struct FaceKey {
  int64_t k[4];
  int64_t id;  // e * 6 + F
};

// tangential axes of a face normal to direction d, in increasing axis order
void tangential(int d, int* t1, int* t2) {
  *t1 = d == 0 ? 1 : 0;
  *t2 = d == 2 ? 1 : 2;
}

int face_corner(int F, int s, int t) {
  const int d = F / 2, side = F % 2;
  int t1, t2;
  tangential(d, &t1, &t2);
  int c[3];
  c[d] = side;
  c[t1] = s;
  c[t2] = t;
  return corner_of(c[0], c[1], c[2]);
}

}  // namespace

int build_mesh(int64_t n_nodes, const double* node_xyz, int64_t n_elem, const int64_t* hex20, int p,
               double r_inner, double r_outer, int metric_mode, const Tables1D& tab, HostMesh* out,
               const char** why) {
  if (n_nodes <= 0 || n_elem <= 0 || !node_xyz || !hex20 || p < 2 || p > 5 || !(r_inner > 0) ||
      !(r_outer > r_inner) || (metric_mode != 0 && metric_mode != 1) || n_elem > (int64_t)1 << 28) {
    *why = "invalid argument";
    return 1;
  }
  const int N = p + 1, N2 = N * N, N3 = N * N * N, NF = N + 1;
  HostMesh& M = *out;
  M.p = p;
  M.N = N;
  M.E = n_elem;
  const int64_t E = n_elem;
  for (int64_t i = 0; i < E * 20; ++i)
    if (hex20[i] < 0 || hex20[i] >= n_nodes) {
      *why = "node index out of range";
      return 4;
    }
  for (int64_t e = 0; e < E; ++e) {
    std::array<int64_t, 20> v;
    for (int a = 0; a < 20; ++a) v[a] = hex20[e * 20 + a];
    std::sort(v.begin(), v.end());
    if (std::adjacent_find(v.begin(), v.end()) != v.end()) {
      *why = "repeated node in an element";
      return 4;
    }
  }

  // ---- face pairing by sorted corner quadruples
  std::vector<FaceKey> keys((size_t)E * 6);
  for (int64_t e = 0; e < E; ++e)
    for (int F = 0; F < 6; ++F) {
      FaceKey& k = keys[e * 6 + F];
      for (int c = 0; c < 4; ++c) k.k[c] = hex20[e * 20 + face_corner(F, c & 1, c >> 1)];
      std::sort(k.k, k.k + 4);
      k.id = e * 6 + F;
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey& x, const FaceKey& y) {
    for (int c = 0; c < 4; ++c)
      if (x.k[c] != y.k[c]) return x.k[c] < y.k[c];
    return x.id < y.id;
  });
  M.nbr.assign(E * 6, -3);
  M.code.assign(E * 6, 0);
  auto same = [](const FaceKey& x, const FaceKey& y) { return std::memcmp(x.k, y.k, sizeof(x.k)) == 0; };
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && same(keys[i], keys[j])) ++j;
    if (j - i > 2) {
      *why = "face shared by more than two elements";
      return 4;
    }
    if (j - i == 2) {
      const int64_t a = keys[i].id, b = keys[i + 1].id;
      const int64_t ea = a / 6, eb = b / 6;
      const int Fa = (int)(a % 6), Fb = (int)(b % 6);
      if (ea == eb) {
        *why = "element glued to itself";
        return 4;
      }
      // orientation: where each own corner (s,t) lands on the neighbour face
      auto locate = [&](int64_t eo, int Fo, int64_t en, int Fn, int code[1]) -> bool {
        int pos[2][2][2];
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) {
            const int64_t node = hex20[eo * 20 + face_corner(Fo, s, t)];
            bool found = false;
            for (int s2 = 0; s2 < 2 && !found; ++s2)
              for (int t2 = 0; t2 < 2 && !found; ++t2)
                if (hex20[en * 20 + face_corner(Fn, s2, t2)] == node) {
                  pos[s][t][0] = s2;
                  pos[s][t][1] = t2;
                  found = true;
                }
            if (!found) return false;
          }
        const bool swap = pos[1][0][0] == pos[0][0][0];
        const int f1 = pos[0][0][0], f2 = pos[0][0][1];
        for (int s = 0; s < 2; ++s)
          for (int t = 0; t < 2; ++t) {
            int a1 = swap ? t : s, b1 = swap ? s : t;
            if (f1) a1 = 1 - a1;
            if (f2) b1 = 1 - b1;
            if (pos[s][t][0] != a1 || pos[s][t][1] != b1) return false;
          }
        code[0] = Fn * 8 + (swap ? 4 : 0) + (f1 ? 2 : 0) + (f2 ? 1 : 0);
        return true;
      };
      int ca, cb;
      if (!locate(ea, Fa, eb, Fb, &ca) || !locate(eb, Fb, ea, Fa, &cb)) {
        *why = "inconsistent face orientation";
        return 4;
      }
      M.nbr[ea * 6 + Fa] = (int)eb;
      M.code[ea * 6 + Fa] = ca;
      M.nbr[eb * 6 + Fb] = (int)ea;
      M.code[eb * 6 + Fb] = cb;
      ++M.n_interior_faces;
    }
    i = j;
  }
  // ---- walls by corner radius
  const double tol = 1e-6 * (r_outer - r_inner);
  for (int64_t e = 0; e < E; ++e)
    for (int F = 0; F < 6; ++F) {
      if (M.nbr[e * 6 + F] != -3) continue;
      bool in = true, outw = true;
      for (int c = 0; c < 4; ++c) {
        const double* X = node_xyz + 3 * hex20[e * 20 + face_corner(F, c & 1, c >> 1)];
        const double r = std::sqrt(X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
        in = in && std::fabs(r - r_inner) < tol;
        outw = outw && std::fabs(r - r_outer) < tol;
      }
      if (!in && !outw) {
        *why = "boundary face on neither shell wall";
        return 4;
      }
      M.nbr[e * 6 + F] = in ? -1 : -2;
      ++M.n_wall_faces;
    }

  // ---- per-order shape-function tables
  const auto& Xs = tab.Xs;
  const auto& Xf = tab.Xf;
  std::vector<double> Nsol(N3 * 20), dNsol(N3 * 60), Ngrid(NF * NF * NF * 20);
  for (int k = 0; k < N; ++k)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        double Nv[20], dN[20][3];
        shape20(Xs[i], Xs[j], Xs[k], Nv, dN);
        const int pt = i + N * j + N2 * k;
        for (int a = 0; a < 20; ++a) {
          Nsol[pt * 20 + a] = Nv[a];
          for (int d = 0; d < 3; ++d) dNsol[(pt * 20 + a) * 3 + d] = dN[a][d];
        }
      }
  for (int c = 0; c < NF; ++c)
    for (int b = 0; b < NF; ++b)
      for (int a = 0; a < NF; ++a) {
        double Nv[20], dN[20][3];
        shape20(Xf[a], Xf[b], Xf[c], Nv, dN);
        for (int q = 0; q < 20; ++q) Ngrid[((c * NF + b) * NF + a) * 20 + q] = Nv[q];
      }
  // derivatives at the d-flux points for the analytic-cofactor variant
  std::vector<double> dNfl(3 * NF * N2 * 60);
  for (int d = 0; d < 3; ++d)
    for (int f = 0; f < NF; ++f)
      for (int ln = 0; ln < N2; ++ln) {
        const int t1 = ln % N, t2 = ln / N;
        double r[3];
        r[d] = Xf[f];
        int a1, a2;
        tangential(d, &a1, &a2);
        r[a1] = Xs[t1];
        r[a2] = Xs[t2];
        double Nv[20], dN[20][3];
        shape20(r[0], r[1], r[2], Nv, dN);
        for (int a = 0; a < 20; ++a)
          for (int c = 0; c < 3; ++c) dNfl[(((d * NF + f) * N2 + ln) * 20 + a) * 3 + c] = dN[a][c];
      }

  M.Sf.assign((size_t)E * 9 * NF * N2, 0.0);
  M.x.assign((size_t)E * 3 * N3, 0.0);
  M.detJ.assign((size_t)E * N3, 0.0);
  int bad = 0;
  const auto& Dff = tab.Dff;
  const auto& Dfs = tab.Dfs;
  const auto& Lfs = tab.Lfs;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t e = 0; e < E; ++e) {
    // node coordinates, and the same measured from the element's node centroid: the Jacobian and
    // the metrics are invariant under that translation (Eqs. 10-12), and with centred coordinates
    // their sums do not cancel from O(|x|) down to O(h), which keeps them accurate to a few ulp
    double X[20][3], Xc[20][3], cen[3] = {0, 0, 0};
    for (int a = 0; a < 20; ++a)
      for (int c = 0; c < 3; ++c) {
        X[a][c] = node_xyz[3 * hex20[e * 20 + a] + c];
        cen[c] += X[a][c];
      }
    for (int a = 0; a < 20; ++a)
      for (int c = 0; c < 3; ++c) Xc[a][c] = X[a][c] - cen[c] / 20.0;
    // solution-point coordinates and |J|
    for (int pt = 0; pt < N3; ++pt) {
      double xx[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      for (int a = 0; a < 20; ++a) {
        for (int c = 0; c < 3; ++c) {
          xx[c] += Nsol[pt * 20 + a] * X[a][c];
          for (int d = 0; d < 3; ++d) J[c][d] += dNsol[(pt * 20 + a) * 3 + d] * Xc[a][c];
        }
      }
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      if (!(det > 0.0)) bad = 1;
      M.detJ[e * N3 + pt] = det;
      for (int c = 0; c < 3; ++c) M.x[(e * 3 + c) * N3 + pt] = xx[c];
    }
    double* Se = &M.Sf[(size_t)e * 9 * NF * N2];
    auto Sat = [&](int d, int n, int f, int ln) -> double& { return Se[((d * 3 + n) * NF + f) * N2 + ln]; };
    // For N >= 4 the curl form's interpolation of X_l grad X_m is exact (the 20-node map has degree
    // <= 2 in each reference variable, so the products have degree <= 4), and its exact curl equals
    // the cofactor rows grad X_m x grad X_l: the same metrics, evaluated with far less rounding.
    if (metric_mode == 1 || N >= 4) {
      // analytic cofactor rows: S^0 = a_1 x a_2, S^1 = a_2 x a_0, S^2 = a_0 x a_1 with a_d = dx/dxi_d
      for (int d = 0; d < 3; ++d)
        for (int f = 0; f < NF; ++f)
          for (int ln = 0; ln < N2; ++ln) {
            double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int a = 0; a < 20; ++a)
              for (int c = 0; c < 3; ++c)
                for (int dd = 0; dd < 3; ++dd) J[c][dd] += dNfl[(((d * NF + f) * N2 + ln) * 20 + a) * 3 + dd] * Xc[a][c];
            const int u = (d + 1) % 3, w = (d + 2) % 3;
            for (int n = 0; n < 3; ++n) {
              const int n1 = (n + 1) % 3, n2 = (n + 2) % 3;
              Sat(d, n, f, ln) = J[n1][u] * J[n2][w] - J[n2][u] * J[n1][w];
            }
          }
      continue;
    }
    // conservative curl form on the (N+1)^3 flux-point grid
    const int G = NF * NF * NF;
    std::vector<double> Xg(G * 3), dX(G * 9), V(G * 3);
    for (int g = 0; g < G; ++g)
      for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int a = 0; a < 20; ++a) s += Ngrid[g * 20 + a] * Xc[a][c];
        Xg[g * 3 + c] = s;
      }
    auto gid = [&](int a, int b, int c) { return (c * NF + b) * NF + a; };
    for (int c = 0; c < NF; ++c)
      for (int b = 0; b < NF; ++b)
        for (int a = 0; a < NF; ++a)
          for (int m = 0; m < 3; ++m) {
            double d0 = 0, d1 = 0, d2 = 0;
            for (int t = 0; t < NF; ++t) {
              d0 += Dff[a * NF + t] * Xg[gid(t, b, c) * 3 + m];
              d1 += Dff[b * NF + t] * Xg[gid(a, t, c) * 3 + m];
              d2 += Dff[c * NF + t] * Xg[gid(a, b, t) * 3 + m];
            }
            dX[(gid(a, b, c) * 3 + m) * 3 + 0] = d0;
            dX[(gid(a, b, c) * 3 + m) * 3 + 1] = d1;
            dX[(gid(a, b, c) * 3 + m) * 3 + 2] = d2;
          }
    for (int n = 0; n < 3; ++n) {
      const int m = (n + 1) % 3, l = (n + 2) % 3;
      for (int g = 0; g < G; ++g)
        for (int dir = 0; dir < 3; ++dir) V[g * 3 + dir] = Xg[g * 3 + l] * dX[(g * 3 + m) * 3 + dir];
      for (int f = 0; f < NF; ++f)
        for (int t2 = 0; t2 < N; ++t2)
          for (int t1 = 0; t1 < N; ++t1) {
            const int ln = t1 + N * t2;
            double s0 = 0, s1 = 0, s2 = 0;
            for (int u = 0; u < NF; ++u)
              for (int v = 0; v < NF; ++v) {
                // xi-flux point (f, j=t1, k=t2): -(d_eta V_zeta - d_zeta V_eta)
                s0 += V[gid(f, u, v) * 3 + 2] * Dfs[t1 * NF + u] * Lfs[t2 * NF + v] -
                      V[gid(f, u, v) * 3 + 1] * Lfs[t1 * NF + u] * Dfs[t2 * NF + v];
                // eta-flux point (i=t1, f, k=t2): -(d_zeta V_xi - d_xi V_zeta)
                s1 += V[gid(u, f, v) * 3 + 0] * Lfs[t1 * NF + u] * Dfs[t2 * NF + v] -
                      V[gid(u, f, v) * 3 + 2] * Dfs[t1 * NF + u] * Lfs[t2 * NF + v];
                // zeta-flux point (i=t1, j=t2, f): -(d_xi V_eta - d_eta V_xi)
                s2 += V[gid(u, v, f) * 3 + 1] * Dfs[t1 * NF + u] * Lfs[t2 * NF + v] -
                      V[gid(u, v, f) * 3 + 0] * Lfs[t1 * NF + u] * Dfs[t2 * NF + v];
              }
            Sat(0, n, f, ln) = -s0;
            Sat(1, n, f, ln) = -s1;
            Sat(2, n, f, ln) = -s2;
          }
    }
  }
  if (bad) {
    *why = "non-positive Jacobian";
    return 4;
  }
  // ---- h_min and volume
  static const int edges[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                                   {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
  double hmin = 1e300, vol = 0.0;
  for (int64_t e = 0; e < E; ++e) {
    for (auto& ed : edges) {
      const double* A = node_xyz + 3 * hex20[e * 20 + ed[0]];
      const double* B = node_xyz + 3 * hex20[e * 20 + ed[1]];
      const double h = std::sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) +
                                 (A[2] - B[2]) * (A[2] - B[2]));
      hmin = std::min(hmin, h);
    }
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) vol += tab.w[i] * tab.w[j] * tab.w[k] * M.detJ[e * N3 + i + N * j + N2 * k];
  }
  M.h_min = hmin;
  M.volume = vol;
  return 0;
}

}  // namespace chorus
