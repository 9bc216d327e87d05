// Sources between GLL nodes: a point source at x_s is tested against the Lagrange basis of
// the element that holds it (Sec. II-B basis psi_(i,j,k) = l_i(xi) l_j(eta) l_k(zeta)):
// a point force F gives the nodal forces F psi_p(x_s), a moment tensor M (the body force
// -M . grad delta) gives M grad psi_p(x_s).
#include "sem_sources.h"

#include <algorithm>
#include <cmath>
#include <vector>

#include "sem_internal.h"

namespace semgb {

namespace {

// x(ref) = sum_c N_c(ref) X_c of a trilinear hexahedron (corner c = a + 2b + 4d at reference
// (2a-1, 2b-1, 2d-1)) and its Jacobian A[d][q] = dx_d / dref_q.
void trilinear_map(const double* X, const double* r, double* x, double A[3][3]) {
  for (int d = 0; d < 3; ++d) {
    x[d] = 0.0;
    for (int q = 0; q < 3; ++q) A[d][q] = 0.0;
  }
  for (int c = 0; c < 8; ++c) {
    const double s[3] = {(c & 1) ? 1.0 : -1.0, (c & 2) ? 1.0 : -1.0, (c & 4) ? 1.0 : -1.0};
    const double f[3] = {1.0 + s[0] * r[0], 1.0 + s[1] * r[1], 1.0 + s[2] * r[2]};
    const double N = 0.125 * f[0] * f[1] * f[2];
    const double dN[3] = {0.125 * s[0] * f[1] * f[2], 0.125 * f[0] * s[1] * f[2], 0.125 * f[0] * f[1] * s[2]};
    for (int d = 0; d < 3; ++d) {
      x[d] += N * X[3 * c + d];
      for (int q = 0; q < 3; ++q) A[d][q] += dN[q] * X[3 * c + d];
    }
  }
}

// Inverse by cofactors; false for a singular or non-finite matrix.
bool invert3(const double A[3][3], double B[3][3]) {
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
  const double inv = 1.0 / det;
  B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) * inv;
  B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * inv;
  B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * inv;
  B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) * inv;
  B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * inv;
  B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * inv;
  B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) * inv;
  B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * inv;
  B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * inv;
  return true;
}

}  // namespace

// Values by the barycentric formula with weights 1 / prod_{j != i} (xi_i - xi_j) (exact
// Kronecker values at a node); derivatives from the nodal derivative matrix, exact because
// l_i' has degree N - 1 and is therefore reproduced by its own nodal values:
// l_i'(x) = sum_j l_i'(xi_j) l_j(x).
void lagrange_at(int n, const double* xi, const double* h, double x, double* l, double* dl) {
  int hit = -1;
  for (int i = 0; i < n; ++i)
    if (x == xi[i]) hit = i;
  if (hit >= 0) {
    for (int i = 0; i < n; ++i) l[i] = (i == hit) ? 1.0 : 0.0;
  } else {
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
      double prod = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != i) prod *= xi[i] - xi[j];
      l[i] = 1.0 / (prod * (x - xi[i]));
      sum += l[i];
    }
    for (int i = 0; i < n; ++i) l[i] /= sum;
  }
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int j = 0; j < n; ++j) d += h[j * n + i] * l[j];
    dl[i] = d;
  }
}

namespace {

constexpr double kInsideTol = 1e-9;

// Corner bounding box of element X[8][3], widened by kInsideTol of its largest side.
void padded_box(const double* X, double* lo, double* hi) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = hi[d] = X[d];
    for (int c = 1; c < 8; ++c) {
      lo[d] = std::min(lo[d], X[3 * c + d]);
      hi[d] = std::max(hi[d], X[3 * c + d]);
    }
  }
  const double pad = kInsideTol * std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  for (int d = 0; d < 3; ++d) {
    lo[d] -= pad;
    hi[d] += pad;
  }
}

// Whether element X holds x: its padded box does, and Newton's method on the trilinear map
// from the element centre (at most 60 iterations) ends within kInsideTol of the reference
// cube; then ref = the solution clipped to [-1, 1].
bool element_holds(const double* X, const double* x, double* ref) {
  double lo[3], hi[3];
  padded_box(X, lo, hi);
  for (int d = 0; d < 3; ++d)
    if (!(x[d] >= lo[d] && x[d] <= hi[d])) return false;
  double r[3] = {0.0, 0.0, 0.0};
  for (int it = 0; it < 60; ++it) {
    double p[3], A[3][3], B[3][3];
    trilinear_map(X, r, p, A);
    if (!invert3(A, B)) return false;
    double big = 0.0, rmax = 0.0;
    for (int q = 0; q < 3; ++q) {
      const double step = B[q][0] * (p[0] - x[0]) + B[q][1] * (p[1] - x[1]) + B[q][2] * (p[2] - x[2]);
      r[q] -= step;
      big = std::max(big, std::fabs(step));
    }
    for (int q = 0; q < 3; ++q) rmax = std::max(rmax, std::fabs(r[q]));
    if (big < 1e-15 || rmax > 10.0) break;
  }
  if (!(std::fabs(r[0]) <= 1.0 + kInsideTol && std::fabs(r[1]) <= 1.0 + kInsideTol &&
        std::fabs(r[2]) <= 1.0 + kInsideTol))
    return false;
  for (int q = 0; q < 3; ++q) ref[q] = std::min(1.0, std::max(-1.0, r[q]));
  return true;
}

}  // namespace

// Elements in index order; the first that holds x.
int locate_point(int nspec, const double* ctrl, const double* x, double* ref) {
  for (int e = 0; e < nspec; ++e)
    if (element_holds(ctrl + 24 * static_cast<size_t>(e), x, ref)) return e;
  return -1;
}

// Buckets: a uniform grid of about nspec cells over the union of the padded boxes; every
// element is listed, in increasing index, in each cell its padded box overlaps. An element
// that holds x has x in its padded box, so it is listed in x's cell, and the first element
// of that list that holds x is the lowest-numbered one.
void locate_points(int nspec, const double* ctrl, int npts, const double* xyz, int32_t* elem, double* ref) {
  if (npts <= 8 || nspec <= 64) {
    for (int s = 0; s < npts; ++s) {
      ref[3 * s] = ref[3 * s + 1] = ref[3 * s + 2] = 0.0;
      elem[s] = locate_point(nspec, ctrl, xyz + 3 * static_cast<size_t>(s), ref + 3 * static_cast<size_t>(s));
    }
    return;
  }
  std::vector<double> box(6 * static_cast<size_t>(nspec));
  double gmin[3] = {0.0, 0.0, 0.0}, gmax[3] = {0.0, 0.0, 0.0};
  for (int e = 0; e < nspec; ++e) {
    double* b = box.data() + 6 * static_cast<size_t>(e);
    padded_box(ctrl + 24 * static_cast<size_t>(e), b, b + 3);
    for (int d = 0; d < 3; ++d) {
      gmin[d] = e ? std::min(gmin[d], b[d]) : b[d];
      gmax[d] = e ? std::max(gmax[d], b[3 + d]) : b[3 + d];
    }
  }
  const int m = std::max(1, static_cast<int>(std::cbrt(static_cast<double>(nspec))));
  double cell[3];
  for (int d = 0; d < 3; ++d) cell[d] = std::max((gmax[d] - gmin[d]) / m, 1e-300);
  auto index = [&](double v, int d) {
    const double t = std::floor((v - gmin[d]) / cell[d]);
    return static_cast<int>(std::min(static_cast<double>(m - 1), std::max(0.0, t)));
  };
  std::vector<std::vector<int32_t>> bucket(static_cast<size_t>(m) * m * m);
  for (int e = 0; e < nspec; ++e) {
    const double* b = box.data() + 6 * static_cast<size_t>(e);
    int c0[3], c1[3];
    for (int d = 0; d < 3; ++d) {
      c0[d] = index(b[d], d);
      c1[d] = index(b[3 + d], d);
    }
    for (int k = c0[2]; k <= c1[2]; ++k)
      for (int j = c0[1]; j <= c1[1]; ++j)
        for (int i = c0[0]; i <= c1[0]; ++i) bucket[(static_cast<size_t>(k) * m + j) * m + i].push_back(e);
  }
  for (int s = 0; s < npts; ++s) {
    const double* x = xyz + 3 * static_cast<size_t>(s);
    double* r = ref + 3 * static_cast<size_t>(s);
    r[0] = r[1] = r[2] = 0.0;
    elem[s] = -1;
    bool inside = true;
    for (int d = 0; d < 3; ++d) inside = inside && x[d] >= gmin[d] && x[d] <= gmax[d];
    if (!inside) continue;
    const auto& list = bucket[(static_cast<size_t>(index(x[2], 2)) * m + index(x[1], 1)) * m + index(x[0], 0)];
    for (const int32_t e : list)
      if (element_holds(ctrl + 24 * static_cast<size_t>(e), x, r)) {
        elem[s] = e;
        break;
      }
    if (elem[s] < 0) r[0] = r[1] = r[2] = 0.0;
  }
}

void point_source_forces(int n, const double* xi, const double* h, const double* ctrl_e, const double* ref,
                         const double* force, const double* moment, double* f) {
  double l[3][kMaxNgll], dl[3][kMaxNgll];
  for (int q = 0; q < 3; ++q) lagrange_at(n, xi, h, ref[q], l[q], dl[q]);
  double x[3], A[3][3], D[3][3];  // D[r][d] = dxi_r / dx_d at the source
  trilinear_map(ctrl_e, ref, x, A);
  invert3(A, D);
  double M[3][3] = {{0.0}};
  if (moment) {
    const double* m = moment;  // Mxx Myy Mzz Mxy Mxz Myz
    const double full[3][3] = {{m[0], m[3], m[4]}, {m[3], m[1], m[5]}, {m[4], m[5], m[2]}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) M[a][b] = full[a][b];
  }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double* fp = f + 3 * (i + n * (j + n * k));
        if (force) {
          const double psi = l[0][i] * l[1][j] * l[2][k];
          for (int a = 0; a < 3; ++a) fp[a] = force[a] * psi;
        } else {
          const double g[3] = {dl[0][i] * l[1][j] * l[2][k], l[0][i] * dl[1][j] * l[2][k], l[0][i] * l[1][j] * dl[2][k]};
          double grad[3];
          for (int d = 0; d < 3; ++d) grad[d] = g[0] * D[0][d] + g[1] * D[1][d] + g[2] * D[2][d];
          for (int a = 0; a < 3; ++a) fp[a] = M[a][0] * grad[0] + M[a][1] * grad[1] + M[a][2] * grad[2];
        }
      }
}

}  // namespace semgb
