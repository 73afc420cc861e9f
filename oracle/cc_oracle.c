/*
 * Plain FP64 CPU oracle for the cell-centred multigrid V-cycle: the second
 * grid type of the paper's feature model (Table 1: "cell-centered" location
 * of grid points, Neumann or Dirichlet boundaries, constant interpolation
 * and cell-centred restriction, finite volumes), the setting Sec. 4 uses for
 * its complex-diffusion runs. The operator here is the real, constant-
 * coefficient part of that setting: sigma u - sum_d c_d d^2u/dx_d^2 on the
 * unit square/cube, sigma >= 0 (sigma = 1/dt is one implicit Euler step of
 * the diffusion equation, Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY, like mg_oracle.c: it shares no code, header,
 * table or helper with the CUDA path; only tests/, the smoke check and the
 * benchmark's CPU-baseline leg may load it. Build flags: -O2
 * -ffp-contract=off.
 *
 * Conventions: n = 2^m cells per dimension (m >= 0), h = 1/n, cell centres
 * x_i = (i + 1/2) h, cell p = i + n*(j + n*k), x fastest; no ghost cells are
 * stored. Finite-volume operator:
 *   (A u)_p = sigma u_p + h^-2 sum_d c_d (F_{p,d,-} + F_{p,d,+}),
 *   F = u_p - u_q for the neighbour cell q across an interior face,
 *     = 0 across a Neumann (zero-flux) boundary face,
 *     = 2 u_p across a homogeneous Dirichlet boundary face (ghost value
 *       -u_p, so that the linear interpolant is zero on the face).
 * Transfers (Sec. 4): restriction = mean of the 2^dim fine cells of a coarse
 * cell; interpolation = constant (every fine cell takes its parent's value).
 * Coarse operators are rediscretised (Table 1, "direct (re-discretization)")
 * with h_H = 2h, the same sigma and the same boundary kind.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int dim, n;
  double h, c[3], sigma;
  int neumann;
} CcOp;

static long cc_count(int dim, int n) { return dim == 2 ? (long)n * n : (long)n * n * n; }

static CcOp cc_op(int dim, int n, const double *c, double sigma, int neumann) {
  CcOp op;
  op.dim = dim;
  op.n = n;
  op.h = 1.0 / (double)n;
  for (int d = 0; d < 3; d++) op.c[d] = c ? c[d] : 1.0;
  op.sigma = sigma;
  op.neumann = neumann;
  return op;
}

/* Cell (i, j, k) -> index, and the coordinate of cell p along axis d. */
static long cc_idx(int n, int i, int j, int k) { return i + (long)n * (j + (long)n * k); }
static int cc_coord(int n, long p, int d) {
  if (d == 0) return (int)(p % n);
  if (d == 1) return (int)((p / n) % n);
  return (int)(p / ((long)n * n));
}
static long cc_stride(int n, int d) { return d == 0 ? 1 : (d == 1 ? (long)n : (long)n * n); }

/* Flux sum of cell p along axis d, side s (-1 or +1), as defined above. */
static double cc_face(const CcOp *op, const double *u, long p, int d, int s) {
  int x = cc_coord(op->n, p, d) + s;
  if (x >= 0 && x < op->n) return u[p] - u[p + s * cc_stride(op->n, d)];
  return op->neumann ? 0.0 : 2.0 * u[p];
}

static double cc_apply_at(const CcOp *op, const double *u, long p) {
  double acc = 0.0;
  for (int d = 0; d < op->dim; d++) acc += op->c[d] * (cc_face(op, u, p, d, -1) + cc_face(op, u, p, d, +1));
  return op->sigma * u[p] + acc / (op->h * op->h);
}

/* The coefficient of u_p in (A u)_p. */
static double cc_diag_at(const CcOp *op, long p) {
  double acc = 0.0;
  for (int d = 0; d < op->dim; d++)
    for (int s = -1; s <= 1; s += 2) {
      int x = cc_coord(op->n, p, d) + s;
      if (x >= 0 && x < op->n) acc += op->c[d];
      else if (!op->neumann) acc += 2.0 * op->c[d];
    }
  return op->sigma + acc / (op->h * op->h);
}

void cc_apply(int dim, int n, const double *c, double sigma, int neumann, const double *u, double *out) {
  CcOp op = cc_op(dim, n, c, sigma, neumann);
  for (long p = 0; p < cc_count(dim, n); p++) out[p] = cc_apply_at(&op, u, p);
}

void cc_diag(int dim, int n, const double *c, double sigma, int neumann, double *out) {
  CcOp op = cc_op(dim, n, c, sigma, neumann);
  for (long p = 0; p < cc_count(dim, n); p++) out[p] = cc_diag_at(&op, p);
}

void cc_residual(int dim, int n, const double *c, double sigma, int neumann, const double *u, const double *f,
                 double *r) {
  CcOp op = cc_op(dim, n, c, sigma, neumann);
  for (long p = 0; p < cc_count(dim, n); p++) r[p] = f[p] - cc_apply_at(&op, u, p);
}

/* Red-black Gauss-Seidel: red cells ((i+j[+k]) even) first, then black, each
 * cell relaxed in natural order: u_p += omega (f_p - (A u)_p) / diag_p. */
static void cc_rbgs_sweep(const CcOp *op, double omega, double *u, const double *f) {
  for (int color = 0; color < 2; color++)
    for (long p = 0; p < cc_count(op->dim, op->n); p++) {
      int par = 0;
      for (int d = 0; d < op->dim; d++) par += cc_coord(op->n, p, d);
      if ((par & 1) != color) continue;
      u[p] += omega * (f[p] - cc_apply_at(op, u, p)) / cc_diag_at(op, p);
    }
}

/* Weighted Jacobi: every cell from the previous iterate. */
static void cc_jacobi_sweep(const CcOp *op, double omega, double *u, const double *f, double *tmp) {
  long N = cc_count(op->dim, op->n);
  memcpy(tmp, u, sizeof(double) * N);
  for (long p = 0; p < N; p++) u[p] = tmp[p] + omega * (f[p] - cc_apply_at(op, tmp, p)) / cc_diag_at(op, p);
}

void cc_smooth(int dim, int n, const double *c, double sigma, int neumann, int smoother, double omega, int sweeps,
               double *u, const double *f) {
  CcOp op = cc_op(dim, n, c, sigma, neumann);
  double *tmp = (double *)malloc(sizeof(double) * cc_count(dim, n));
  for (int s = 0; s < sweeps; s++) {
    if (smoother == 0) cc_rbgs_sweep(&op, omega, u, f);
    else cc_jacobi_sweep(&op, omega, u, f, tmp);
  }
  free(tmp);
}

/* Coarse cell P = (I, J, K) of a grid with nc = nf/2 cells gets the mean of
 * the fine cells (2I + a, 2J + b, 2K + e), a, b, e in {0, 1}. */
void cc_restrict(int dim, int nf, const double *r, double *fc) {
  int nc = nf / 2;
  double w = dim == 2 ? 0.25 : 0.125;
  for (long P = 0; P < cc_count(dim, nc); P++) {
    int I = cc_coord(nc, P, 0), J = cc_coord(nc, P, 1), K = dim == 3 ? cc_coord(nc, P, 2) : 0;
    double acc = 0.0;
    for (int e = 0; e < (dim == 3 ? 2 : 1); e++)
      for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) acc += r[cc_idx(nf, 2 * I + a, 2 * J + b, dim == 3 ? 2 * K + e : 0)];
    fc[P] = w * acc;
  }
}

/* Constant interpolation and correction: u_p += e_{parent(p)}. */
void cc_prolong_add(int dim, int nc, const double *e, double *u) {
  int nf = 2 * nc;
  for (long p = 0; p < cc_count(dim, nf); p++) {
    int i = cc_coord(nf, p, 0), j = cc_coord(nf, p, 1), k = dim == 3 ? cc_coord(nf, p, 2) : 0;
    u[p] += e[cc_idx(nc, i / 2, j / 2, k / 2)];
  }
}

/* Euclidean norm over all cells, summed pairwise in index order. */
static double cc_pairwise(const double *x, long m) {
  if (m <= 8) {
    double s = 0.0;
    for (long i = 0; i < m; i++) s += x[i];
    return s;
  }
  long h = m / 2;
  return cc_pairwise(x, h) + cc_pairwise(x + h, m - h);
}

double cc_norm(int dim, int n, const double *r) {
  long N = cc_count(dim, n);
  double *sq = (double *)malloc(sizeof(double) * N);
  for (long p = 0; p < N; p++) sq[p] = r[p] * r[p];
  double s = cc_pairwise(sq, N);
  free(sq);
  return sqrt(s);
}

/* Exact solve of A u = f: the matrix is assembled column by column (A applied
 * to unit vectors) and solved by Gaussian elimination with partial pivoting.
 * Returns 0, or -1 for a singular matrix. */
int cc_dense_solve(int dim, int n, const double *c, double sigma, int neumann, const double *f, double *u) {
  CcOp op = cc_op(dim, n, c, sigma, neumann);
  long N = cc_count(dim, n);
  double *a = (double *)calloc((size_t)(N * N), sizeof(double));
  double *b = (double *)malloc(sizeof(double) * N);
  double *e = (double *)calloc((size_t)N, sizeof(double));
  for (long col = 0; col < N; col++) {
    e[col] = 1.0;
    for (long row = 0; row < N; row++) a[row * N + col] = cc_apply_at(&op, e, row);
    e[col] = 0.0;
  }
  memcpy(b, f, sizeof(double) * N);
  int rc = 0;
  for (long k = 0; k < N && rc == 0; k++) {
    long piv = k;
    for (long i = k + 1; i < N; i++)
      if (fabs(a[i * N + k]) > fabs(a[piv * N + k])) piv = i;
    if (a[piv * N + k] == 0.0) {
      rc = -1;
      break;
    }
    if (piv != k) {
      for (long j = 0; j < N; j++) {
        double t = a[k * N + j];
        a[k * N + j] = a[piv * N + j];
        a[piv * N + j] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (long i = k + 1; i < N; i++) {
      double l = a[i * N + k] / a[k * N + k];
      for (long j = k; j < N; j++) a[i * N + j] -= l * a[k * N + j];
      b[i] -= l * b[k];
    }
  }
  if (rc == 0)
    for (long i = N - 1; i >= 0; i--) {
      double s = b[i];
      for (long j = i + 1; j < N; j++) s -= a[i * N + j] * u[j];
      u[i] = s / a[i * N + i];
    }
  free(a);
  free(b);
  free(e);
  return rc;
}

/* ---------------- hierarchy, V-cycle (Algorithm 1) and solve loop ---------------- */

#define CC_MAXL 24

typedef struct {
  int dim, nl, smoother, nu1, nu2, neumann;
  double c[3], sigma, omega;
  int n[CC_MAXL];
  double *u[CC_MAXL], *f[CC_MAXL], *r[CC_MAXL];
} CcHier;

void *cc_create(int dim, int n, const double *c, double sigma, int neumann, int coarsest_n, int smoother,
                double omega, int nu1, int nu2) {
  if (dim != 2 && dim != 3) return NULL;
  if (n < 1 || (n & (n - 1)) || coarsest_n < 1 || (coarsest_n & (coarsest_n - 1)) || coarsest_n > n) return NULL;
  CcHier *H = (CcHier *)calloc(1, sizeof(CcHier));
  H->dim = dim;
  for (int d = 0; d < 3; d++) H->c[d] = c ? c[d] : 1.0;
  H->sigma = sigma;
  H->neumann = neumann;
  H->smoother = smoother;
  H->omega = omega;
  H->nu1 = nu1;
  H->nu2 = nu2;
  for (int nn = n; nn >= coarsest_n && H->nl < CC_MAXL; nn /= 2) {
    int l = H->nl++;
    H->n[l] = nn;
    long N = cc_count(dim, nn);
    H->u[l] = (double *)calloc((size_t)N, sizeof(double));
    H->f[l] = (double *)calloc((size_t)N, sizeof(double));
    H->r[l] = (double *)calloc((size_t)N, sizeof(double));
    if (nn == coarsest_n) break;
  }
  return H;
}

void cc_destroy(void *h) {
  CcHier *H = (CcHier *)h;
  if (!H) return;
  for (int l = 0; l < H->nl; l++) {
    free(H->u[l]);
    free(H->f[l]);
    free(H->r[l]);
  }
  free(H);
}

int cc_levels(void *h) { return ((CcHier *)h)->nl; }
int cc_level_n(void *h, int l) { return ((CcHier *)h)->n[l]; }
void cc_set_rhs(void *h, const double *f) {
  CcHier *H = (CcHier *)h;
  memcpy(H->f[0], f, sizeof(double) * cc_count(H->dim, H->n[0]));
}
void cc_set_u(void *h, const double *u) {
  CcHier *H = (CcHier *)h;
  memcpy(H->u[0], u, sizeof(double) * cc_count(H->dim, H->n[0]));
}
void cc_get_u(void *h, double *u) {
  CcHier *H = (CcHier *)h;
  memcpy(u, H->u[0], sizeof(double) * cc_count(H->dim, H->n[0]));
}

/* Algorithm 1: presmooth, residual, restrict, zero the coarse solution,
 * recurse, interpolate and correct, postsmooth; exact solve on the coarsest
 * level. */
static void cc_vcycle_rec(CcHier *H, int l) {
  int n = H->n[l];
  if (l == H->nl - 1) {
    cc_dense_solve(H->dim, n, H->c, H->sigma, H->neumann, H->f[l], H->u[l]);
    return;
  }
  cc_smooth(H->dim, n, H->c, H->sigma, H->neumann, H->smoother, H->omega, H->nu1, H->u[l], H->f[l]);
  cc_residual(H->dim, n, H->c, H->sigma, H->neumann, H->u[l], H->f[l], H->r[l]);
  cc_restrict(H->dim, n, H->r[l], H->f[l + 1]);
  memset(H->u[l + 1], 0, sizeof(double) * cc_count(H->dim, H->n[l + 1]));
  cc_vcycle_rec(H, l + 1);
  cc_prolong_add(H->dim, H->n[l + 1], H->u[l + 1], H->u[l]);
  cc_smooth(H->dim, n, H->c, H->sigma, H->neumann, H->smoother, H->omega, H->nu2, H->u[l], H->f[l]);
}

void cc_vcycle(void *h) { cc_vcycle_rec((CcHier *)h, 0); }

double cc_residual_norm(void *h) {
  CcHier *H = (CcHier *)h;
  cc_residual(H->dim, H->n[0], H->c, H->sigma, H->neumann, H->u[0], H->f[0], H->r[0]);
  return cc_norm(H->dim, H->n[0], H->r[0]);
}

/* rho[0..k] = ||r_k|| / ||r_0||; V-cycles until rho <= tol or maxit. */
int cc_solve(void *h, double tol, int maxit, double *rho) {
  double r0 = cc_residual_norm(h);
  rho[0] = 1.0;
  int k = 0;
  double q = 1.0;
  while (r0 > 0.0 && q > tol && k < maxit) {
    cc_vcycle(h);
    q = cc_residual_norm(h) / r0;
    rho[++k] = q;
  }
  return k;
}
