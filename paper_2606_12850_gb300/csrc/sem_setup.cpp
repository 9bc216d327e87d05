// Host-side set-up of libsemgb: GLL basis, trilinear geometry, element colouring and
// node location. Plain C++17, float64, deterministic; runs once per mesh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "sem_internal.h"

namespace semgb {

namespace {

// P_N(x) and P_{N-1}(x) by the three-term recurrence.
void legendre_pair(int N, double x, double* pN, double* pNm1) {
  double pm1 = 1.0, p = x;
  if (N == 0) {
    *pN = 1.0;
    *pNm1 = 0.0;
    return;
  }
  for (int k = 1; k < N; ++k) {
    const double next = ((2.0 * k + 1.0) * x * p - k * pm1) / (k + 1.0);
    pm1 = p;
    p = next;
  }
  *pN = p;
  *pNm1 = pm1;
}

}  // namespace

// GLL nodes are the zeros of q(x) = (1 - x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)), whose
// derivative is q'(x) = -N (N+1) P_N(x) (Legendre's equation). Interior zeros by Newton on
// q from the Chebyshev-Gauss-Lobatto points; weights 2 / (N (N+1) P_N(x_i)^2); derivative
// matrix by its closed form D_il = P_N(x_i) / (P_N(x_l) (x_i - x_l)), D_00 = -N(N+1)/4,
// D_NN = N(N+1)/4, other diagonal entries 0 (Sec. II-B defines the basis; the closed form
// is the standard one for Lobatto nodes).
int gll_basis(int ngll, double* xi_out, double* w_out, double* h_out, std::string* err) {
  if (ngll < kMinNgll || ngll > kMaxNgll) {
    if (err) *err = "ngll must be in [2, 10], got " + std::to_string(ngll);
    return -1;
  }
  const int N = ngll - 1;
  std::vector<double> x(ngll), pN(ngll);
  for (int i = 0; i < ngll; ++i) x[i] = -std::cos(M_PI * i / N);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    for (int it = 0; it < 64; ++it) {
      double p, pm1;
      legendre_pair(N, x[i], &p, &pm1);
      const double q = N * (pm1 - x[i] * p);
      const double dq = -N * (N + 1.0) * p;
      const double step = q / dq;
      x[i] -= step;
      if (std::fabs(step) < 1e-17) break;
    }
  }
  // symmetrise: the nodes are symmetric about 0 in exact arithmetic
  for (int i = 0; i <= N / 2; ++i) {
    const double s = 0.5 * (x[N - i] - x[i]);
    x[i] = -s;
    x[N - i] = s;
  }
  if (ngll % 2 == 1) x[N / 2] = 0.0;
  for (int i = 0; i < ngll; ++i) {
    double pm1;
    legendre_pair(N, x[i], &pN[i], &pm1);
  }
  if (xi_out) std::memcpy(xi_out, x.data(), sizeof(double) * ngll);
  if (w_out)
    for (int i = 0; i < ngll; ++i) w_out[i] = 2.0 / (N * (N + 1.0) * pN[i] * pN[i]);
  if (h_out) {
    for (int i = 0; i < ngll; ++i)
      for (int l = 0; l < ngll; ++l)
        h_out[i * ngll + l] = (i == l) ? 0.0 : pN[i] / (pN[l] * (x[i] - x[l]));
    h_out[0] = -N * (N + 1.0) / 4.0;
    h_out[N * ngll + N] = N * (N + 1.0) / 4.0;
  }
  return 0;
}

// GLL positions from the trilinear map of the 8 corners, then the geometry from those
// positions (geometry_from_positions; exact for the trilinear map, of degree 1 <= N per
// direction).
bool element_geometry(int n, const double* xi, const double* h, const double* ctrl,
                      double* xyz, double* G, double* J) {
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int p = i + n * (j + n * k);
        double pos[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 8; ++c) {
          const double sa = (c & 1) ? 1.0 : -1.0, sb = (c & 2) ? 1.0 : -1.0, sd = (c & 4) ? 1.0 : -1.0;
          const double Nc = 0.125 * (1.0 + sa * xi[i]) * (1.0 + sb * xi[j]) * (1.0 + sd * xi[k]);
          for (int d = 0; d < 3; ++d) pos[d] += Nc * ctrl[3 * c + d];
        }
        for (int d = 0; d < 3; ++d) xyz[3 * p + d] = pos[d];
      }
  return geometry_from_positions(n, h, xyz, G, J);
}

// dx/dxi at every GLL point by differentiating the positions with the 1D derivative matrix
// along each reference direction (exact for any map of degree <= N per direction, such as
// the trilinear one, and the isoparametric geometry otherwise), then the inverse by
// cofactors and the determinant.
bool geometry_from_positions(int n, const double* h, const double* xyz, double* G, double* J) {
  bool ok = true;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int p = i + n * (j + n * k);
        double A[3][3] = {{0}};  // A[d][r] = dx_d / dxi_r
        for (int l = 0; l < n; ++l) {
          const double hi = h[i * n + l], hj = h[j * n + l], hk = h[k * n + l];
          const int pxi = l + n * (j + n * k), peta = i + n * (l + n * k), pzeta = i + n * (j + n * l);
          for (int d = 0; d < 3; ++d) {
            A[d][0] += hi * xyz[3 * pxi + d];
            A[d][1] += hj * xyz[3 * peta + d];
            A[d][2] += hk * xyz[3 * pzeta + d];
          }
        }
        const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
        const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
        const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
        const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
        J[p] = det;
        if (!(det > 0.0)) ok = false;
        const double inv = 1.0 / det;
        // inverse of A: (A^-1)[r][d] = dxi_r / dx_d = cofactor(A)[d][r] / det
        double* g = G + 9 * p;
        g[0] = c00 * inv;
        g[1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * inv;
        g[2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * inv;
        g[3] = c01 * inv;
        g[4] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * inv;
        g[5] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * inv;
        g[6] = c02 * inv;
        g[7] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * inv;
        g[8] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * inv;
      }
  return ok;
}

// Sec. IV-C: element-to-corner-vertex incidence from ibool, adjacency = elements sharing a
// corner vertex (the pattern of incidence x incidence^T), greedy colouring in element
// order, then an exhaustive check that no two elements of one colour share any node.
int color_elements(int nspec, int n, int nglob, const int32_t* ibool,
                   std::vector<int32_t>* color_out, int* ncolors_out, std::string* err) {
  const int np = n * n * n;
  const int N = n - 1;
  const int corner_p[8] = {0, N, N * n, N + N * n, N * n * n, N + N * n * n, N * n + N * n * n,
                           N + N * n + N * n * n};
  // vertex -> elements (CSR over global ids of corner nodes)
  std::vector<int> count(static_cast<size_t>(nglob) + 1, 0);
  for (int e = 0; e < nspec; ++e)
    for (int c = 0; c < 8; ++c) count[ibool[static_cast<size_t>(e) * np + corner_p[c]] + 1]++;
  for (int g = 0; g < nglob; ++g) count[g + 1] += count[g];
  std::vector<int> elems(static_cast<size_t>(count[nglob]));
  std::vector<int> fill(count.begin(), count.end() - 1);
  for (int e = 0; e < nspec; ++e)
    for (int c = 0; c < 8; ++c) elems[fill[ibool[static_cast<size_t>(e) * np + corner_p[c]]]++] = e;

  std::vector<int32_t>& color = *color_out;
  color.assign(nspec, -1);
  std::vector<int> mark;  // mark[c] == e: colour c used by a neighbour of e
  int ncolors = 0;
  for (int e = 0; e < nspec; ++e) {
    for (int c = 0; c < 8; ++c) {
      const int g = ibool[static_cast<size_t>(e) * np + corner_p[c]];
      for (int q = count[g]; q < count[g + 1]; ++q) {
        const int o = elems[q];
        if (o != e && color[o] >= 0) {
          if (static_cast<int>(mark.size()) <= color[o]) mark.resize(color[o] + 1, -1);
          mark[color[o]] = e;
        }
      }
    }
    int c = 0;
    while (c < static_cast<int>(mark.size()) && mark[c] == e) ++c;
    color[e] = c;
    ncolors = std::max(ncolors, c + 1);
  }
  // exhaustive validity check over all ibool entries
  std::vector<int> owner(nglob, -1), owner_color(nglob, -1);
  std::vector<std::vector<int>> by_color(ncolors);
  for (int e = 0; e < nspec; ++e) by_color[color[e]].push_back(e);
  for (int c = 0; c < ncolors; ++c) {
    for (int e : by_color[c]) {
      for (int p = 0; p < np; ++p) {
        const int g = ibool[static_cast<size_t>(e) * np + p];
        if (owner_color[g] == c) {
          if (err) {
            *err = (owner[g] == e) ? "element " + std::to_string(e) + " repeats node " + std::to_string(g)
                                   : "colouring failed: elements " + std::to_string(owner[g]) + " and " +
                                         std::to_string(e) + " share node " + std::to_string(g) +
                                         " but no corner vertex (non-conforming mesh?)";
          }
          return -1;
        }
        owner_color[g] = c;
        owner[g] = e;
      }
    }
  }
  *ncolors_out = ncolors;
  return 0;
}

// Brute-force nearest node (O(npts * nglob)); ties go to the lowest index.
int locate_nodes(int nglob, const double* X, int npts, const double* xyz, const double* surface_z,
                 int32_t* out) {
  std::vector<int> cand;
  if (surface_z) {
    const double zs = *surface_z;
    const double tol = 1e-9 * std::max(1.0, std::fabs(zs));
    for (int g = 0; g < nglob; ++g)
      if (std::fabs(X[3 * g + 2] - zs) <= tol) cand.push_back(g);
    if (cand.empty()) return -1;
  }
  for (int r = 0; r < npts; ++r) {
    const double px = xyz[3 * r], py = xyz[3 * r + 1], pz = xyz[3 * r + 2];
    double best = std::numeric_limits<double>::infinity();
    int arg = -1;
    const int m = surface_z ? static_cast<int>(cand.size()) : nglob;
    for (int q = 0; q < m; ++q) {
      const int g = surface_z ? cand[q] : q;
      const double dx = X[3 * g] - px, dy = X[3 * g + 1] - py, dz = X[3 * g + 2] - pz;
      const double d2 = dx * dx + dy * dy + dz * dz;
      if (d2 < best) {
        best = d2;
        arg = g;
      }
    }
    out[r] = arg;
  }
  return 0;
}

}  // namespace semgb
