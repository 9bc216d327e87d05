/*
 * Compiled FP64 CPU baseline of the spectral-element time step (test infrastructure: only
 * tests/ and the cpu_baseline / --impl reference legs of bench.py load it; it shares no code
 * with the CUDA library).
 *
 * The same arithmetic as oracle/sem_oracle.py, written as plain loops so that it can be
 * timed as a CPU program: per element (Sec. II-B) the reference derivatives along xi, eta
 * and zeta with the 1D derivative matrix, the chain rule, the isotropic Hooke stress, the
 * fluxes and the weighted transposed products; the element forces are added into the
 * global nodes; explicit Newmark (beta = 0, gamma = 1/2) with the diagonal mass and a
 * Ricker point force at t_{n+1} (Sec. I, V-C). With several threads the elements are taken
 * colour by colour (Sec. IV-C: elements of one colour share no node), the elements of one
 * colour split over OpenMP threads, so the result does not depend on the thread count.
 *
 * Array layouts (float64 unless stated; p = i + n j + n^2 k is the local point index):
 *   ibool   int32 [nspec][np]
 *   dxi_dx  [nspec][3 (r)][3 (d)][np]   d xi_r / d x_d
 *   jac, kappa, mu  [nspec][np]
 *   hprime  [n][n] with hprime[i][l] = l_l'(xi_i);  w [n]
 *   u, v, a, f  [nglob][3];  minv [nglob]
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 10

/* f += -K_e u_e for one element e (f is the global array). */
static void element_force(int e, int n, const int* ibool, const double* hprime, const double* w,
                          const double* dxi_dx, const double* jac, const double* kappa, const double* mu,
                          const double* u, double* f) {
  const int np = n * n * n;
  double ue[3][MAXN * MAXN * MAXN];
  double t[3][3][MAXN * MAXN * MAXN]; /* fluxes t[r][c][p] */
  const int* ib = ibool + (size_t)e * np;
  for (int p = 0; p < np; ++p)
    for (int c = 0; c < 3; ++c) ue[c][p] = u[3 * (size_t)ib[p] + c];
  const double* G = dxi_dx + (size_t)e * 9 * np;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int p = i + n * (j + n * k);
        double du[3][3]; /* du[c][r] = d u_c / d xi_r */
        for (int c = 0; c < 3; ++c) {
          double s0 = 0.0, s1 = 0.0, s2 = 0.0;
          for (int l = 0; l < n; ++l) {
            s0 += hprime[i * n + l] * ue[c][l + n * (j + n * k)];
            s1 += hprime[j * n + l] * ue[c][i + n * (l + n * k)];
            s2 += hprime[k * n + l] * ue[c][i + n * (j + n * l)];
          }
          du[c][0] = s0;
          du[c][1] = s1;
          du[c][2] = s2;
        }
        double grad[3][3]; /* grad[c][d] = d u_c / d x_d */
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) {
            double s = 0.0;
            for (int r = 0; r < 3; ++r) s += du[c][r] * G[(3 * r + d) * np + p];
            grad[c][d] = s;
          }
        const double km = kappa[(size_t)e * np + p], m = mu[(size_t)e * np + p];
        const double lam = km - 2.0 * m / 3.0;
        const double tr = grad[0][0] + grad[1][1] + grad[2][2];
        double sig[3][3];
        for (int c = 0; c < 3; ++c)
          for (int d = 0; d < 3; ++d) sig[c][d] = m * (grad[c][d] + grad[d][c]) + (c == d ? lam * tr : 0.0);
        const double J = jac[(size_t)e * np + p];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += sig[c][d] * G[(3 * r + d) * np + p];
            t[r][c][p] = J * s;
          }
      }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int p = i + n * (j + n * k);
        double F[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; ++c) {
          double s = 0.0;
          for (int l = 0; l < n; ++l) {
            s += w[j] * w[k] * w[l] * hprime[l * n + i] * t[0][c][l + n * (j + n * k)];
            s += w[i] * w[k] * w[l] * hprime[l * n + j] * t[1][c][i + n * (l + n * k)];
            s += w[i] * w[j] * w[l] * hprime[l * n + k] * t[2][c][i + n * (j + n * l)];
          }
          F[c] = -s;
        }
        const size_t g = (size_t)ib[p];
        for (int c = 0; c < 3; ++c) f[3 * g + c] += F[c];
      }
}

/* Greedy colouring of the elements over shared nodes (own implementation); fills
 * order[nspec] (elements colour by colour) and color_off[ncolors + 1]; returns ncolors or -1. */
int sem_cpu_color(int nspec, int n, int nglob, const int* ibool, int* order, int* color_off, int max_colors) {
  const int np = n * n * n;
  int* color = (int*)malloc(sizeof(int) * (size_t)nspec);
  /* node -> elements */
  int* cnt = (int*)calloc((size_t)nglob + 1, sizeof(int));
  for (size_t q = 0; q < (size_t)nspec * np; ++q) cnt[ibool[q] + 1]++;
  for (int g = 0; g < nglob; ++g) cnt[g + 1] += cnt[g];
  int* elems = (int*)malloc(sizeof(int) * (size_t)cnt[nglob]);
  int* fill = (int*)malloc(sizeof(int) * (size_t)nglob);
  memcpy(fill, cnt, sizeof(int) * (size_t)nglob);
  for (int e = 0; e < nspec; ++e)
    for (int p = 0; p < np; ++p) elems[fill[ibool[(size_t)e * np + p]]++] = e;
  int* used = (int*)malloc(sizeof(int) * (size_t)max_colors);
  for (int c = 0; c < max_colors; ++c) used[c] = -1;
  int ncolors = 0, ok = 1;
  for (int e = 0; e < nspec && ok; ++e) {
    for (int p = 0; p < np; ++p) {
      const int g = ibool[(size_t)e * np + p];
      for (int q = cnt[g]; q < cnt[g + 1]; ++q) {
        const int o = elems[q];
        if (o < e) used[color[o]] = e;
      }
    }
    int c = 0;
    while (c < max_colors && used[c] == e) ++c;
    if (c == max_colors) ok = 0;
    color[e] = c;
    if (c + 1 > ncolors) ncolors = c + 1;
  }
  if (ok) {
    for (int c = 0; c <= ncolors; ++c) color_off[c] = 0;
    for (int e = 0; e < nspec; ++e) color_off[color[e] + 1]++;
    for (int c = 0; c < ncolors; ++c) color_off[c + 1] += color_off[c];
    int* pos = (int*)malloc(sizeof(int) * (size_t)(ncolors + 1));
    memcpy(pos, color_off, sizeof(int) * (size_t)(ncolors + 1));
    for (int e = 0; e < nspec; ++e) order[pos[color[e]]++] = e;
    free(pos);
  }
  free(used);
  free(fill);
  free(elems);
  free(cnt);
  free(color);
  return ok ? ncolors : -1;
}

/* f = -K u: every element, colour by colour, the elements of a colour over nthreads. */
void sem_cpu_forces(int nspec, int n, int nglob, const int* ibool, const double* hprime, const double* w,
                    const double* dxi_dx, const double* jac, const double* kappa, const double* mu,
                    const int* order, const int* color_off, int ncolors, const double* u, double* f, int nthreads) {
  memset(f, 0, sizeof(double) * 3 * (size_t)nglob);
  for (int c = 0; c < ncolors; ++c) {
    const int e0 = color_off[c], e1 = color_off[c + 1];
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (int s = e0; s < e1; ++s)
      element_force(order[s], n, ibool, hprime, w, dxi_dx, jac, kappa, mu, u, f);
  }
  (void)nspec;
}

/* nsteps explicit Newmark steps from (u, v, a) in place, a point force F R(t_{n+1} - t0) at
 * src_node (src_node < 0: none). f is scratch [nglob][3]. */
void sem_cpu_run(int nspec, int n, int nglob, const int* ibool, const double* hprime, const double* w,
                 const double* dxi_dx, const double* jac, const double* kappa, const double* mu, const double* minv,
                 const int* order, const int* color_off, int ncolors, int nsteps, double dt, int src_node,
                 const double* src_force, double f0, double t0, double* u, double* v, double* a, double* f,
                 int nthreads) {
  const size_t n3 = 3 * (size_t)nglob;
  const double pi = 3.14159265358979323846;
  for (int step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (size_t q = 0; q < n3; ++q) {
      u[q] += dt * v[q] + 0.5 * dt * dt * a[q];
      v[q] += 0.5 * dt * a[q];
    }
    sem_cpu_forces(nspec, n, nglob, ibool, hprime, w, dxi_dx, jac, kappa, mu, order, color_off, ncolors, u, f,
                   nthreads);
    if (src_node >= 0) {
      const double tau = (step + 1) * dt - t0;
      const double x = pi * f0 * tau;
      const double R = (1.0 - 2.0 * x * x) * exp(-x * x);
      for (int c = 0; c < 3; ++c) f[3 * (size_t)src_node + c] += src_force[c] * R;
    }
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (size_t q = 0; q < n3; ++q) {
      a[q] = f[q] * minv[q / 3];
      v[q] += 0.5 * dt * a[q];
    }
  }
}

int sem_cpu_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
