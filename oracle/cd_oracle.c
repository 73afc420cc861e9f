/*
 * Plain FP64 CPU oracle for one implicit Euler step of nonlinear complex
 * diffusion (Sec. 4, Eq. 2 and the diffusivity below it), solved by
 * cell-centred multigrid V-cycles.
 *
 * TEST INFRASTRUCTURE ONLY, like mg_oracle.c and cc_oracle.c: it shares no
 * code, header, table or helper with the CUDA path; only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load it. Build flags: -O2
 * -ffp-contract=off. Complex numbers are C99 double complex (interleaved
 * re, im, as numpy complex128).
 *
 * Model (Sec. 4): u_t = div(g(Im u) grad u) on the unit square with Neumann
 * boundaries, g(s) = e^{i theta} / (1 + (s / (kappa theta))^2), a small
 * angle theta and kappa > 0. Discretisation: n = 2^m cells per dimension,
 * h = 1/n, finite volumes ("averaged finite differences"): the coefficient
 * of the face between cells p and q is the mean (g_p + g_q)/2 of the cell
 * values; implicit Euler with step tau, the diffusivity lagged to the
 * previous time level (computed once from u^n), so each step solves the
 * linear complex system
 *   (A u)_p = u_p + tau h^-2 sum_{faces f of p} g_f (u_p - u_q) = u^n_p,
 * boundary faces carrying no flux. For a linear system the full
 * approximation scheme and the correction scheme give the same iterates,
 * so the V-cycle here is the correction scheme of Algorithm 1 with
 * cell-centred restriction (mean of the 4 fine cells), constant
 * interpolation, and coarse face coefficients rediscretised from the fine
 * ones: a coarse face spans two fine faces and takes their mean, with
 * h_H = 2h. The coarsest grid is one cell, where A u = u.
 *
 * Face arrays: gx[j*n + i] is the face between cells (i, j) and (i+1, j)
 * (i < n-1), gy[j*n + i] the face between (i, j) and (i, j+1) (j < n-1);
 * the last column of gx and the last row of gy are unused (zero).
 */
#include <complex.h>
#undef I /* coarse indices are I, J below; the imaginary unit is _Complex_I */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

void cd_diffusivity(int n, const cplx *u, double theta, double kappa, cplx *g) {
  cplx e = cexp(_Complex_I * theta);
  for (long p = 0; p < (long)n * n; p++) {
    double s = cimag(u[p]) / (kappa * theta);
    g[p] = e / (1.0 + s * s);
  }
}

void cd_faces(int n, const cplx *g, cplx *gx, cplx *gy) {
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) {
      long p = (long)j * n + i;
      gx[p] = i + 1 < n ? 0.5 * (g[p] + g[p + 1]) : 0.0;
      gy[p] = j + 1 < n ? 0.5 * (g[p] + g[p + n]) : 0.0;
    }
}

/* Coarse x-face (I, J) | (I+1, J) covers the fine faces (2I+1, 2J+b) |
 * (2I+2, 2J+b), b = 0, 1; coarse y-faces likewise. */
void cd_coarsen_faces(int nf, const cplx *gxf, const cplx *gyf, cplx *gxc, cplx *gyc) {
  int nc = nf / 2;
  for (int J = 0; J < nc; J++)
    for (int I = 0; I < nc; I++) {
      long P = (long)J * nc + I;
      gxc[P] = I + 1 < nc ? 0.5 * (gxf[(long)(2 * J) * nf + 2 * I + 1] + gxf[(long)(2 * J + 1) * nf + 2 * I + 1]) : 0.0;
      gyc[P] = J + 1 < nc ? 0.5 * (gyf[(long)(2 * J + 1) * nf + 2 * I] + gyf[(long)(2 * J + 1) * nf + 2 * I + 1]) : 0.0;
    }
}

/* Flux sum of cell (i, j): sum over its interior faces of g_f (u_p - u_q). */
static cplx cd_flux(int n, const cplx *gx, const cplx *gy, const cplx *u, int i, int j) {
  long p = (long)j * n + i;
  cplx acc = 0.0;
  if (i > 0) acc += gx[p - 1] * (u[p] - u[p - 1]);
  if (i + 1 < n) acc += gx[p] * (u[p] - u[p + 1]);
  if (j > 0) acc += gy[p - n] * (u[p] - u[p - n]);
  if (j + 1 < n) acc += gy[p] * (u[p] - u[p + n]);
  return acc;
}

static cplx cd_diag(int n, const cplx *gx, const cplx *gy, double tau, int i, int j) {
  long p = (long)j * n + i;
  cplx acc = 0.0;
  if (i > 0) acc += gx[p - 1];
  if (i + 1 < n) acc += gx[p];
  if (j > 0) acc += gy[p - n];
  if (j + 1 < n) acc += gy[p];
  return 1.0 + tau * (double)n * (double)n * acc;
}

void cd_apply(int n, double tau, const cplx *gx, const cplx *gy, const cplx *u, cplx *out) {
  double s = tau * (double)n * (double)n;
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) out[(long)j * n + i] = u[(long)j * n + i] + s * cd_flux(n, gx, gy, u, i, j);
}

void cd_residual(int n, double tau, const cplx *gx, const cplx *gy, const cplx *u, const cplx *f, cplx *r) {
  double s = tau * (double)n * (double)n;
  for (int j = 0; j < n; j++)
    for (int i = 0; i < n; i++) {
      long p = (long)j * n + i;
      r[p] = f[p] - (u[p] + s * cd_flux(n, gx, gy, u, i, j));
    }
}

/* smoother 0: red-black Gauss-Seidel (red = i+j even first), 1: Jacobi;
 * u_p += omega (f_p - (A u)_p) / diag_p. */
void cd_smooth(int n, double tau, const cplx *gx, const cplx *gy, int smoother, double omega, int sweeps, cplx *u,
               const cplx *f) {
  double s = tau * (double)n * (double)n;
  long N = (long)n * n;
  cplx *tmp = (cplx *)malloc(sizeof(cplx) * N);
  for (int it = 0; it < sweeps; it++) {
    if (smoother == 0) {
      for (int color = 0; color < 2; color++)
        for (int j = 0; j < n; j++)
          for (int i = 0; i < n; i++) {
            if (((i + j) & 1) != color) continue;
            long p = (long)j * n + i;
            cplx Au = u[p] + s * cd_flux(n, gx, gy, u, i, j);
            u[p] += omega * (f[p] - Au) / cd_diag(n, gx, gy, tau, i, j);
          }
    } else {
      memcpy(tmp, u, sizeof(cplx) * N);
      for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
          long p = (long)j * n + i;
          cplx Au = tmp[p] + s * cd_flux(n, gx, gy, tmp, i, j);
          u[p] = tmp[p] + omega * (f[p] - Au) / cd_diag(n, gx, gy, tau, i, j);
        }
    }
  }
  free(tmp);
}

void cd_restrict(int nf, const cplx *r, cplx *fc) {
  int nc = nf / 2;
  for (int J = 0; J < nc; J++)
    for (int I = 0; I < nc; I++) {
      cplx acc = 0.0;
      for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) acc += r[(long)(2 * J + b) * nf + 2 * I + a];
      fc[(long)J * nc + I] = 0.25 * acc;
    }
}

void cd_prolong_add(int nc, const cplx *e, cplx *u) {
  int nf = 2 * nc;
  for (int j = 0; j < nf; j++)
    for (int i = 0; i < nf; i++) u[(long)j * nf + i] += e[(long)(j / 2) * nc + i / 2];
}

static double cd_pairwise(const double *x, long m) {
  if (m <= 8) {
    double s = 0.0;
    for (long i = 0; i < m; i++) s += x[i];
    return s;
  }
  long h = m / 2;
  return cd_pairwise(x, h) + cd_pairwise(x + h, m - h);
}

/* sqrt(sum_p |r_p|^2), summed pairwise in index order. */
double cd_norm(int n, const cplx *r) {
  long N = (long)n * n;
  double *sq = (double *)malloc(sizeof(double) * N);
  for (long p = 0; p < N; p++) sq[p] = creal(r[p]) * creal(r[p]) + cimag(r[p]) * cimag(r[p]);
  double s = cd_pairwise(sq, N);
  free(sq);
  return sqrt(s);
}

/* ---------------- hierarchy and time step ---------------- */

#define CD_MAXL 20

typedef struct {
  int nl, smoother, nu1, nu2;
  double tau, omega, theta, kappa;
  int n[CD_MAXL];
  cplx *u[CD_MAXL], *f[CD_MAXL], *r[CD_MAXL], *gx[CD_MAXL], *gy[CD_MAXL];
} CdHier;

void *cd_create(int n, double tau, double theta, double kappa, int smoother, double omega, int nu1, int nu2) {
  if (n < 1 || (n & (n - 1)) || !(tau > 0) || !(kappa > 0) || theta == 0.0) return NULL;
  CdHier *H = (CdHier *)calloc(1, sizeof(CdHier));
  H->tau = tau;
  H->theta = theta;
  H->kappa = kappa;
  H->smoother = smoother;
  H->omega = omega;
  H->nu1 = nu1;
  H->nu2 = nu2;
  for (int nn = n; nn >= 1 && H->nl < CD_MAXL; nn /= 2) {
    int l = H->nl++;
    long N = (long)nn * nn;
    H->n[l] = nn;
    H->u[l] = (cplx *)calloc((size_t)N, sizeof(cplx));
    H->f[l] = (cplx *)calloc((size_t)N, sizeof(cplx));
    H->r[l] = (cplx *)calloc((size_t)N, sizeof(cplx));
    H->gx[l] = (cplx *)calloc((size_t)N, sizeof(cplx));
    H->gy[l] = (cplx *)calloc((size_t)N, sizeof(cplx));
    if (nn == 1) break;
  }
  return H;
}

void cd_destroy(void *h) {
  CdHier *H = (CdHier *)h;
  if (!H) return;
  for (int l = 0; l < H->nl; l++) {
    free(H->u[l]);
    free(H->f[l]);
    free(H->r[l]);
    free(H->gx[l]);
    free(H->gy[l]);
  }
  free(H);
}

int cd_levels(void *h) { return ((CdHier *)h)->nl; }

void cd_get_u(void *h, cplx *u) {
  CdHier *H = (CdHier *)h;
  memcpy(u, H->u[0], sizeof(cplx) * (size_t)H->n[0] * H->n[0]);
}

void cd_get_faces(void *h, int l, cplx *gx, cplx *gy) {
  CdHier *H = (CdHier *)h;
  memcpy(gx, H->gx[l], sizeof(cplx) * (size_t)H->n[l] * H->n[l]);
  memcpy(gy, H->gy[l], sizeof(cplx) * (size_t)H->n[l] * H->n[l]);
}

/* The coefficients of the step from u^n: cell diffusivity, fine faces, then
 * every coarser level's faces; f = u^n and the start u = u^n. */
void cd_begin_step(void *h, const cplx *un) {
  CdHier *H = (CdHier *)h;
  int n = H->n[0];
  long N = (long)n * n;
  cplx *g = (cplx *)malloc(sizeof(cplx) * N);
  cd_diffusivity(n, un, H->theta, H->kappa, g);
  cd_faces(n, g, H->gx[0], H->gy[0]);
  free(g);
  for (int l = 1; l < H->nl; l++) cd_coarsen_faces(H->n[l - 1], H->gx[l - 1], H->gy[l - 1], H->gx[l], H->gy[l]);
  memcpy(H->f[0], un, sizeof(cplx) * N);
  memcpy(H->u[0], un, sizeof(cplx) * N);
}

static void cd_vcycle_rec(CdHier *H, int l) {
  int n = H->n[l];
  if (l == H->nl - 1) {
    /* one cell: no interior faces, A u = u */
    H->u[l][0] = H->f[l][0];
    return;
  }
  cd_smooth(n, H->tau, H->gx[l], H->gy[l], H->smoother, H->omega, H->nu1, H->u[l], H->f[l]);
  cd_residual(n, H->tau, H->gx[l], H->gy[l], H->u[l], H->f[l], H->r[l]);
  cd_restrict(n, H->r[l], H->f[l + 1]);
  memset(H->u[l + 1], 0, sizeof(cplx) * (size_t)H->n[l + 1] * H->n[l + 1]);
  cd_vcycle_rec(H, l + 1);
  cd_prolong_add(H->n[l + 1], H->u[l + 1], H->u[l]);
  cd_smooth(n, H->tau, H->gx[l], H->gy[l], H->smoother, H->omega, H->nu2, H->u[l], H->f[l]);
}

void cd_vcycle(void *h) { cd_vcycle_rec((CdHier *)h, 0); }

double cd_residual_norm(void *h) {
  CdHier *H = (CdHier *)h;
  cd_residual(H->n[0], H->tau, H->gx[0], H->gy[0], H->u[0], H->f[0], H->r[0]);
  return cd_norm(H->n[0], H->r[0]);
}

/* One time step from un: V-cycles until ||r_k|| / ||r_0|| <= tol or maxit;
 * rho[0..k] receives the history. Returns k. */
int cd_time_step(void *h, const cplx *un, double tol, int maxit, double *rho) {
  cd_begin_step(h, un);
  double r0 = cd_residual_norm(h);
  rho[0] = 1.0;
  int k = 0;
  double q = 1.0;
  while (r0 > 0.0 && q > tol && k < maxit) {
    cd_vcycle(h);
    q = cd_residual_norm(h) / r0;
    rho[++k] = q;
  }
  return k;
}
