/*
 * Plain FP64 CPU oracle for the geometric multigrid V-cycle
 * (Koestler et al., "A Scala Prototype to Generate Multigrid Solver
 * Implementations for Different Problems and Target Multi-Core Platforms").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * reference that the CUDA library is checked against. It shares no code,
 * header, table or helper with the CUDA path; only tests/, the smoke check
 * and the benchmark's CPU-baseline leg may load it. Build flags:
 * -O2 -ffp-contract=off (no FMA contraction, no fast-math).
 *
 * Conventions (node-based grid, Sec. 2.2 "field@nodes"):
 *   n = 2^m + 1 nodes per dimension including the boundary, h = 1/(n-1),
 *   node p = i + n*(j + n*k), x fastest. Interior nodes are 1..n-2 in every
 *   dimension; boundary nodes carry Dirichlet values (Eq. 1b).
 *   The operator is -sum_d c_d d^2/dx_d^2 (SPD sign; Eq. 1a is written with
 *   the opposite sign) or, with face coefficients, -div(k grad u).
 *   Face array kf[d][p] holds the coefficient of the face between node p and
 *   node p + e_d.
 *
 * Every routine loops over the points in natural order and follows the
 * definitions of Sec. 2.3 (Algorithm 1 and the component list beneath it)
 * and the Layer-4 pseudo code of Sec. 2.4 (VCycle, GaussSeidel, Restrict,
 * interpolatecorr). Parity pins for each routine live in tests/.
 *
 * Timing build. Compiled a second time with -fopenmp (liboracle_mt.so), the
 * loops marked PAR_FOR_INTERIOR run over all host cores: only loops whose
 * points are independent (one colour of a red-black sweep - a 5-/7-point
 * stencil couples a node only to the other colour -, a Jacobi sweep, the
 * residual, the transfers, fills), and the pairwise norm sum evaluates the
 * same tree with its subtrees as tasks. So both builds compute bitwise the
 * same numbers (tests/ checks this); without -fopenmp the pragmas are
 * ignored and every loop is the plain serial loop.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int dim, n;
  double h;
  double c[3];         /* constant stencil coefficients (used if kf[d] == NULL) */
  const double *kf[3]; /* face coefficients or NULL */
} Op;

static long npts(int dim, int n) { return dim == 2 ? (long)n * n : (long)n * n * n; }
static long stride(int n, int d) { return d == 0 ? 1 : (d == 1 ? (long)n : (long)n * n); }

static Op make_op(int dim, int n, const double *c, const double *kx, const double *ky,
                  const double *kz) {
  Op op;
  op.dim = dim;
  op.n = n;
  op.h = 1.0 / (double)(n - 1);
  for (int d = 0; d < 3; d++) op.c[d] = c ? c[d] : 1.0;
  op.kf[0] = kx;
  op.kf[1] = ky;
  op.kf[2] = kz;
  return op;
}

/* (A u)_p = h^-2 sum_d [ k_{p+e_d/2} (u_p - u_{p+e_d}) + k_{p-e_d/2} (u_p - u_{p-e_d}) ]
 * (second-order finite differences, Sec. 2.2). */
static double apply_at(const Op *op, const double *u, long p) {
  double acc = 0.0;
  for (int d = 0; d < op->dim; d++) {
    long s = stride(op->n, d);
    double kp = op->kf[d] ? op->kf[d][p] : op->c[d];
    double km = op->kf[d] ? op->kf[d][p - s] : op->c[d];
    acc += kp * (u[p] - u[p + s]) + km * (u[p] - u[p - s]);
  }
  return acc / (op->h * op->h);
}

/* diag(A)_p = h^-2 sum_d (k_{p+e_d/2} + k_{p-e_d/2}). */
static double diag_at(const Op *op, long p) {
  double acc = 0.0;
  for (int d = 0; d < op->dim; d++) {
    long s = stride(op->n, d);
    double kp = op->kf[d] ? op->kf[d][p] : op->c[d];
    double km = op->kf[d] ? op->kf[d][p - s] : op->c[d];
    acc += kp + km;
  }
  return acc / (op->h * op->h);
}

/* Interior loop in natural order; the body sees i, j, k and p. */
#define FOR_INTERIOR(dim, n, ...)                                     \
  for (int k = ((dim) == 3 ? 1 : 0); k < ((dim) == 3 ? (n)-1 : 1); k++) \
    for (int j = 1; j < (n)-1; j++)                                   \
      for (int i = 1; i < (n)-1; i++) {                               \
        long p = i + (long)(n) * (j + (long)(n) * k);                 \
        __VA_ARGS__                                                   \
      }

/* The same loop, its (k, j) iterations shared out over threads in the
 * OpenMP build; only for loops whose iterations are independent. */
#define PAR_FOR_INTERIOR(dim, n, ...)                        \
  _Pragma("omp parallel for collapse(2) schedule(static)") \
  FOR_INTERIOR(dim, n, __VA_ARGS__)

static void fill0(double *a, long N) {
#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; q++) a[q] = 0.0;
}

static void copy_to(double *dst, const double *src, long N) {
#pragma omp parallel for schedule(static)
  for (long q = 0; q < N; q++) dst[q] = src[q];
}

/* Threads of the OpenMP build (1 in the serial build). */
void or_set_threads(int nt) {
#ifdef _OPENMP
  if (nt > 0) omp_set_num_threads(nt);
#else
  (void)nt;
#endif
}

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------- stateless level operators ---------------- */

void or_apply(int dim, int n, const double *c, const double *kx, const double *ky,
              const double *kz, const double *u, double *out) {
  Op op = make_op(dim, n, c, kx, ky, kz);
  fill0(out, npts(dim, n));
  PAR_FOR_INTERIOR(dim, n, { out[p] = apply_at(&op, u, p); })
}

void or_diag(int dim, int n, const double *c, const double *kx, const double *ky,
             const double *kz, double *out) {
  Op op = make_op(dim, n, c, kx, ky, kz);
  memset(out, 0, sizeof(double) * npts(dim, n));
  FOR_INTERIOR(dim, n, { out[p] = diag_at(&op, p); })
}

/* r = f - A u at interior nodes, 0 on the boundary (Algorithm 1, residual step). */
void or_residual(int dim, int n, const double *c, const double *kx, const double *ky,
                 const double *kz, const double *u, const double *f, double *r) {
  Op op = make_op(dim, n, c, kx, ky, kz);
  fill0(r, npts(dim, n));
  PAR_FOR_INTERIOR(dim, n, { r[p] = f[p] - apply_at(&op, u, p); })
}

/* One omega red-black Gauss-Seidel sweep (Sec. 2.4 GaussSeidel, "order rb"):
 * u_p += omega * (f_p - (A u)_p) / diag_p, first over red nodes
 * (i+j[+k] even), then over black nodes. */
static void rbgs_sweep(const Op *op, double omega, double *u, const double *f) {
  for (int color = 0; color < 2; color++) {
    PAR_FOR_INTERIOR(op->dim, op->n, {
      if (((i + j + k) & 1) == color)
        u[p] += omega * (f[p] - apply_at(op, u, p)) / diag_at(op, p);
    })
  }
}

/* One omega-Jacobi sweep: every interior node is updated from the old iterate. */
static void jacobi_sweep(const Op *op, double omega, double *u, const double *f, double *tmp) {
  copy_to(tmp, u, npts(op->dim, op->n));
  PAR_FOR_INTERIOR(op->dim, op->n, {
    u[p] = tmp[p] + omega * (f[p] - apply_at(op, tmp, p)) / diag_at(op, p);
  })
}

void or_rbgs(int dim, int n, const double *c, const double *kx, const double *ky,
             const double *kz, double omega, int sweeps, double *u, const double *f) {
  Op op = make_op(dim, n, c, kx, ky, kz);
  for (int s = 0; s < sweeps; s++) rbgs_sweep(&op, omega, u, f);
}

void or_jacobi(int dim, int n, const double *c, const double *kx, const double *ky,
               const double *kz, double omega, int sweeps, double *u, const double *f) {
  Op op = make_op(dim, n, c, kx, ky, kz);
  double *tmp = (double *)malloc(sizeof(double) * npts(dim, n));
  for (int s = 0; s < sweeps; s++) jacobi_sweep(&op, omega, u, f, tmp);
  free(tmp);
}

/* 1D full-weighting weights (1, 2, 1)/4 at offsets -1, 0, +1. */
static double fw_w(int a) { return a == 0 ? 0.5 : 0.25; }

/* Full-weighting restriction (Sec. 2.3: restriction = transpose of the
 * bilinear/trilinear interpolation, order 2): the tensor product of
 * (1,2,1)/4 in every dimension, evaluated at coarse interior nodes; the
 * coarse boundary is 0. */
void or_restrict(int dim, int nf, const double *r, double *fc) {
  int nc = (nf - 1) / 2 + 1;
  fill0(fc, npts(dim, nc));
  PAR_FOR_INTERIOR(dim, nc, {
    double acc = 0.0;
    int cmin = dim == 3 ? -1 : 0, cmax = dim == 3 ? 1 : 0;
    for (int cz = cmin; cz <= cmax; cz++)
      for (int cy = -1; cy <= 1; cy++)
        for (int cx = -1; cx <= 1; cx++) {
          long q = (2 * i + cx) + (long)nf * ((2 * j + cy) + (long)nf * (dim == 3 ? 2 * k + cz : 0));
          double w = fw_w(cx) * fw_w(cy) * (dim == 3 ? fw_w(cz) : 1.0);
          acc += w * r[q];
        }
    fc[p] = acc;
  })
}

/* Bilinear/trilinear prolongation with correction (Sec. 2.4 interpolatecorr):
 * u_h += P e_H at fine interior nodes. Along each dimension an even fine
 * index 2I takes coarse node I with weight 1, an odd index 2I+1 takes coarse
 * nodes I and I+1 with weight 1/2 each; the weights multiply across
 * dimensions. */
void or_prolong_add(int dim, int nc, const double *e, double *u) {
  int nf = 2 * (nc - 1) + 1;
  PAR_FOR_INTERIOR(dim, nf, {
    int idx[3] = {i, j, k};
    int lo[3], cnt[3];
    for (int d = 0; d < 3; d++) {
      if (d >= dim) { lo[d] = 0; cnt[d] = 1; continue; }
      lo[d] = idx[d] / 2;
      cnt[d] = (idx[d] & 1) ? 2 : 1;
    }
    double acc = 0.0;
    for (int a = 0; a < cnt[2]; a++)
      for (int b = 0; b < cnt[1]; b++)
        for (int cc = 0; cc < cnt[0]; cc++) {
          double w = (cnt[0] == 2 ? 0.5 : 1.0) * (cnt[1] == 2 ? 0.5 : 1.0) * (cnt[2] == 2 ? 0.5 : 1.0);
          long q = (lo[0] + cc) + (long)nc * ((lo[1] + b) + (long)nc * (lo[2] + a));
          acc += w * e[q];
        }
    u[p] += acc;
  })
}

/* Face coefficients from node (dual-cell) coefficients: the harmonic mean of
 * the two nodes a face joins, times c_d. Faces past the last node are 0. */
void or_node_faces(int dim, int n, const double *c, const double *knode, double *kx,
                   double *ky, double *kz) {
  double *kf[3] = {kx, ky, kz};
  long N = npts(dim, n);
  for (int d = 0; d < dim; d++) {
    long s = stride(n, d);
    for (long p = 0; p < N; p++) {
      long coord = (p / s) % n;
      if (coord >= n - 1) { kf[d][p] = 0.0; continue; }
      double a = knode[p], b = knode[p + s];
      kf[d][p] = (c ? c[d] : 1.0) * (2.0 * a * b / (a + b));
    }
  }
}

/* Coarse faces by rediscretisation (Table 1, "direct" coarsening). A coarse
 * face along dimension d spans two collinear fine faces in series,
 * 2 / (1/k_a + 1/k_b) = 2 k_a k_b / (k_a + k_b); across the face, the series
 * values of the fine lines at offsets -1, 0, +1 (in each other dimension)
 * are averaged in parallel with the full-weighting weights (1/4, 1/2, 1/4).
 * Faces on coarse boundary lines, which no interior stencil uses, take the
 * centre line only. */
void or_coarsen_faces(int dim, int nf, const double *kxf, const double *kyf, const double *kzf,
                      double *kxc, double *kyc, double *kzc) {
  const double *ff[3] = {kxf, kyf, kzf};
  double *fc[3] = {kxc, kyc, kzc};
  int nc = (nf - 1) / 2 + 1;
  long Nc = npts(dim, nc);
  for (int d = 0; d < dim; d++) {
    long sc = stride(nc, d), sf = stride(nf, d);
    for (long P = 0; P < Nc; P++) {
      long C3[3] = {P % nc, (P / nc) % nc, dim == 3 ? P / ((long)nc * nc) : 0};
      long coord = (P / sc) % nc;
      if (coord >= nc - 1) { fc[d][P] = 0.0; continue; }
      double acc = 0.0;
      for (int oz = -1; oz <= 1; oz++)
        for (int oy = -1; oy <= 1; oy++)
          for (int ox = -1; ox <= 1; ox++) {
            int off[3] = {ox, oy, oz};
            double w = 1.0;
            int skip = 0;
            for (int e = 0; e < 3; e++) {
              int interior_line = e < dim && e != d && C3[e] >= 1 && C3[e] <= nc - 2;
              if (e == d || e >= dim || !interior_line) {
                if (off[e] != 0) skip = 1;
              } else {
                w *= off[e] == 0 ? 0.5 : 0.25;
              }
            }
            if (skip) continue;
            long q = (2 * C3[0] + off[0]) + (long)nf * ((2 * C3[1] + off[1]) + (long)nf * (2 * C3[2] + off[2]));
            double a = ff[d][q], b = ff[d][q + sf];
            acc += w * (2.0 * a * b / (a + b));
          }
      fc[d][P] = acc;
    }
  }
}

/* Euclidean norm over interior nodes; squares summed pairwise. */
static double pairwise(const double *x, long m) {
  if (m <= 8) {
    double s = 0.0;
    for (long q = 0; q < m; q++) s += x[q];
    return s;
  }
  long h = m / 2;
  return pairwise(x, h) + pairwise(x + h, m - h);
}

#ifdef _OPENMP
/* The pairwise tree of pairwise(), its upper `depth` levels split into tasks. */
static double pairwise_tasks(const double *x, long m, int depth) {
  if (depth <= 0 || m <= 8) return pairwise(x, m);
  long h = m / 2;
  double a = 0.0, b;
#pragma omp task shared(a)
  a = pairwise_tasks(x, h, depth - 1);
  b = pairwise_tasks(x + h, m - h, depth - 1);
#pragma omp taskwait
  return a + b;
}
#endif

static double sum_pairwise(const double *x, long m) {
#ifdef _OPENMP
  double s = 0.0;
#pragma omp parallel
#pragma omp single
  s = pairwise_tasks(x, m, 8);
  return s;
#else
  return pairwise(x, m);
#endif
}

double or_norm(int dim, int n, const double *r) {
  long m = (long)(n - 2) * (n - 2) * (dim == 3 ? (n - 2) : 1);
  double *sq = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
  /* sq in natural order: interior node (i, j, k) at its lexicographic index */
  PAR_FOR_INTERIOR(dim, n, {
    long q = (i - 1) + (long)(n - 2) * ((j - 1) + (long)(n - 2) * (dim == 3 ? k - 1 : 0));
    sq[q] = r[p] * r[p];
  })
  double s = sum_pairwise(sq, m);
  free(sq);
  return sqrt(s);
}

/* ---------------- dense direct solve (coarsest level) ---------------- */

typedef struct {
  int m;        /* interior unknowns */
  double *lu;   /* m*m, row-major, LU factors with partial pivoting */
  int *piv;
} Dense;

/* Assembles the interior matrix column by column (A applied to unit
 * vectors) and factors it by Gaussian elimination with partial pivoting. */
static int dense_factor(const Op *op, Dense *D) {
  int dim = op->dim, n = op->n;
  long N = npts(dim, n);
  long m = (long)(n - 2) * (n - 2) * (dim == 3 ? (n - 2) : 1);
  D->m = (int)m;
  D->lu = (double *)calloc((size_t)(m * m), sizeof(double));
  D->piv = (int *)malloc(sizeof(int) * (m > 0 ? m : 1));
  long *pos = (long *)malloc(sizeof(long) * (m > 0 ? m : 1));
  double *e = (double *)calloc((size_t)N, sizeof(double));
  long q = 0;
  FOR_INTERIOR(dim, n, { pos[q++] = p; })
  for (long col = 0; col < m; col++) {
    e[pos[col]] = 1.0;
    for (long row = 0; row < m; row++) D->lu[row * m + col] = apply_at(op, e, pos[row]);
    e[pos[col]] = 0.0;
  }
  free(e);
  free(pos);
  double *a = D->lu;
  for (long kk = 0; kk < m; kk++) {
    long pr = kk;
    for (long r = kk + 1; r < m; r++)
      if (fabs(a[r * m + kk]) > fabs(a[pr * m + kk])) pr = r;
    D->piv[kk] = (int)pr;
    if (a[pr * m + kk] == 0.0) return -1;
    if (pr != kk)
      for (long cc = 0; cc < m; cc++) {
        double t = a[kk * m + cc];
        a[kk * m + cc] = a[pr * m + cc];
        a[pr * m + cc] = t;
      }
    for (long r = kk + 1; r < m; r++) {
      double l = a[r * m + kk] / a[kk * m + kk];
      a[r * m + kk] = l;
      for (long cc = kk + 1; cc < m; cc++) a[r * m + cc] -= l * a[kk * m + cc];
    }
  }
  return 0;
}

/* Solves A u = f on the interior; boundary values of u are kept and moved
 * to the right-hand side. */
static void dense_solve(const Op *op, const Dense *D, double *u, const double *f) {
  int dim = op->dim, n = op->n;
  long m = D->m, q = 0;
  long N = npts(dim, n);
  double *b = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
  double *ub = (double *)malloc(sizeof(double) * N);
  memcpy(ub, u, sizeof(double) * N);
  FOR_INTERIOR(dim, n, { ub[p] = 0.0; })
  FOR_INTERIOR(dim, n, { b[q++] = f[p] - apply_at(op, ub, p); })
  const double *a = D->lu;
  for (long kk = 0; kk < m; kk++) {
    long pr = D->piv[kk];
    if (pr != kk) { double t = b[kk]; b[kk] = b[pr]; b[pr] = t; }
    for (long r = kk + 1; r < m; r++) b[r] -= a[r * m + kk] * b[kk];
  }
  for (long r = m - 1; r >= 0; r--) {
    double s = b[r];
    for (long cc = r + 1; cc < m; cc++) s -= a[r * m + cc] * b[cc];
    b[r] = s / a[r * m + r];
  }
  q = 0;
  FOR_INTERIOR(dim, n, { u[p] = b[q++]; })
  free(b);
  free(ub);
}

int or_dense_solve(int dim, int n, const double *c, const double *kx, const double *ky,
                   const double *kz, double *u, const double *f) {
  Op op = make_op(dim, n, c, kx, ky, kz);
  Dense D;
  int rc = dense_factor(&op, &D);
  if (rc == 0) dense_solve(&op, &D, u, f);
  free(D.lu);
  free(D.piv);
  return rc;
}

/* ---------------- hierarchy, V-cycle, solve ---------------- */

typedef struct {
  int n;
  double *u, *f, *r;
  double *kf[3];
} Level;

typedef struct {
  int dim, nl, smoother, nu1, nu2;
  double omega, c[3];
  int variable;
  Level lv[32];
  Dense coarse;
  double *uo, *fo; /* defect correction: outer FP64 solution and right-hand side */
} Hier;

static Op level_op(const Hier *H, int l) {
  const Level *L = &H->lv[l];
  return make_op(H->dim, L->n, H->c, L->kf[0], L->kf[1], L->kf[2]);
}

/* smoother: 0 = red-black Gauss-Seidel, 1 = omega-Jacobi. */
void *or_create(int dim, int n, const double *c, const double *knode, int coarsest_n,
                int smoother, double omega, int nu1, int nu2) {
  if (dim != 2 && dim != 3) return NULL;
  if (coarsest_n < 3 || coarsest_n > n) return NULL;
  Hier *H = (Hier *)calloc(1, sizeof(Hier));
  H->dim = dim;
  H->smoother = smoother;
  H->omega = omega;
  H->nu1 = nu1;
  H->nu2 = nu2;
  H->variable = knode != NULL;
  for (int d = 0; d < 3; d++) H->c[d] = c ? c[d] : 1.0;
  int nl = 0;
  for (int nn = n; nn >= coarsest_n; nn = (nn - 1) / 2 + 1) {
    Level *L = &H->lv[nl++];
    long N = npts(dim, nn);
    L->n = nn;
    L->u = (double *)calloc((size_t)N, sizeof(double));
    L->f = (double *)calloc((size_t)N, sizeof(double));
    L->r = (double *)calloc((size_t)N, sizeof(double));
    if (H->variable)
      for (int d = 0; d < dim; d++) L->kf[d] = (double *)calloc((size_t)N, sizeof(double));
    if (nn == coarsest_n || nn == 3) break;
  }
  H->nl = nl;
  if (H->lv[nl - 1].n != coarsest_n) { /* n and coarsest_n must share 2^m+1 form */
    for (int l = 0; l < nl; l++) {
      free(H->lv[l].u); free(H->lv[l].f); free(H->lv[l].r);
      for (int d = 0; d < 3; d++) free(H->lv[l].kf[d]);
    }
    free(H);
    return NULL;
  }
  if (H->variable) {
    Level *L0 = &H->lv[0];
    or_node_faces(dim, L0->n, H->c, knode, L0->kf[0], L0->kf[1], L0->kf[2]);
    for (int l = 1; l < nl; l++) {
      Level *F = &H->lv[l - 1], *C = &H->lv[l];
      or_coarsen_faces(dim, F->n, F->kf[0], F->kf[1], F->kf[2], C->kf[0], C->kf[1], C->kf[2]);
    }
  }
  Op op = level_op(H, nl - 1);
  dense_factor(&op, &H->coarse);
  long N0 = npts(dim, n);
  H->uo = (double *)calloc((size_t)N0, sizeof(double));
  H->fo = (double *)calloc((size_t)N0, sizeof(double));
  return H;
}

void or_destroy(void *h) {
  Hier *H = (Hier *)h;
  if (!H) return;
  for (int l = 0; l < H->nl; l++) {
    free(H->lv[l].u); free(H->lv[l].f); free(H->lv[l].r);
    for (int d = 0; d < 3; d++) free(H->lv[l].kf[d]);
  }
  free(H->coarse.lu);
  free(H->coarse.piv);
  free(H->uo);
  free(H->fo);
  free(H);
}

int or_levels(void *h) { return ((Hier *)h)->nl; }
int or_level_n(void *h, int l) { return ((Hier *)h)->lv[l].n; }

void or_get_faces(void *h, int l, double *kx, double *ky, double *kz) {
  Hier *H = (Hier *)h;
  long N = npts(H->dim, H->lv[l].n);
  double *out[3] = {kx, ky, kz};
  for (int d = 0; d < H->dim; d++)
    if (out[d]) memcpy(out[d], H->lv[l].kf[d], sizeof(double) * N);
}

void or_set_rhs(void *h, const double *f) {
  Hier *H = (Hier *)h;
  memcpy(H->lv[0].f, f, sizeof(double) * npts(H->dim, H->lv[0].n));
}
void or_set_u(void *h, const double *u) {
  Hier *H = (Hier *)h;
  memcpy(H->lv[0].u, u, sizeof(double) * npts(H->dim, H->lv[0].n));
}
void or_get_u(void *h, double *u) {
  Hier *H = (Hier *)h;
  memcpy(u, H->lv[0].u, sizeof(double) * npts(H->dim, H->lv[0].n));
}

static void smooth(Hier *H, int l, int sweeps) {
  Op op = level_op(H, l);
  Level *L = &H->lv[l];
  for (int s = 0; s < sweeps; s++) {
    if (H->smoother == 0) rbgs_sweep(&op, H->omega, L->u, L->f);
    else jacobi_sweep(&op, H->omega, L->u, L->f, L->r);
  }
}

/* Algorithm 1 (recursive V-cycle, correction scheme) with the Layer-4
 * VCycle structure: presmooth, residual, restrict, zero the coarse
 * solution, recurse, interpolate-and-correct, postsmooth; exact solve on
 * the coarsest level. */
static void vcycle(Hier *H, int l) {
  Level *L = &H->lv[l];
  if (l == H->nl - 1) {
    Op op = level_op(H, l);
    dense_solve(&op, &H->coarse, L->u, L->f);
    return;
  }
  Level *C = &H->lv[l + 1];
  Op op = level_op(H, l);
  smooth(H, l, H->nu1);
  fill0(L->r, npts(H->dim, L->n));
  PAR_FOR_INTERIOR(H->dim, L->n, { L->r[p] = L->f[p] - apply_at(&op, L->u, p); })
  or_restrict(H->dim, L->n, L->r, C->f);
  fill0(C->u, npts(H->dim, C->n));
  vcycle(H, l + 1);
  or_prolong_add(H->dim, C->n, C->u, L->u);
  smooth(H, l, H->nu2);
}

void or_vcycle(void *h) { vcycle((Hier *)h, 0); }

double or_residual_norm(void *h) {
  Hier *H = (Hier *)h;
  Level *L = &H->lv[0];
  Op op = level_op(H, 0);
  fill0(L->r, npts(H->dim, L->n));
  PAR_FOR_INTERIOR(H->dim, L->n, { L->r[p] = L->f[p] - apply_at(&op, L->u, p); })
  return or_norm(H->dim, L->n, L->r);
}

/* Driver loop of the Layer-4 Application: residual norm, then V-cycles until
 * rho_k = ||r_k|| / ||r_0|| <= tol or maxit cycles. rho[0..k] is filled;
 * returns the number of cycles done. */
int or_solve(void *h, double tol, int maxit, double *rho) {
  Hier *H = (Hier *)h;
  double r0 = or_residual_norm(H);
  rho[0] = 1.0;
  if (r0 == 0.0) return 0;
  for (int k = 1; k <= maxit; k++) {
    vcycle(H, 0);
    rho[k] = or_residual_norm(H) / r0;
    if (!(rho[k] > tol)) return k;
  }
  return maxit;
}

/* Defect correction with an FP64 inner V-cycle: r = f - A u, s = ||r||,
 * d = r / s, e = V(0, d), u += s e. Uses lv[0].u, lv[0].f as the inner
 * (e, d) and keeps the outer (u, f) in uo, fo; or_set_rhs / or_set_u /
 * or_get_u address lv[0], so the outer arrays are loaded from there. */
int or_dc_solve(void *h, double tol, int maxit, double *rho) {
  Hier *H = (Hier *)h;
  int dim = H->dim, n = H->lv[0].n;
  long N = npts(dim, n);
  Level *L = &H->lv[0];
  memcpy(H->uo, L->u, sizeof(double) * N);
  memcpy(H->fo, L->f, sizeof(double) * N);
  Op op = level_op(H, 0);
  double r0 = -1.0;
  int it = 0;
  for (;; it++) {
    fill0(L->r, N);
    PAR_FOR_INTERIOR(dim, n, { L->r[p] = H->fo[p] - apply_at(&op, H->uo, p); })
    double s = or_norm(dim, n, L->r);
    if (r0 < 0.0) r0 = s;
    rho[it] = r0 > 0.0 ? s / r0 : 0.0;
    if (it >= maxit || !(rho[it] > tol) || s == 0.0) break;
    fill0(L->f, N);
    PAR_FOR_INTERIOR(dim, n, { L->f[p] = L->r[p] / s; })
    fill0(L->u, N);
    vcycle(H, 0);
    PAR_FOR_INTERIOR(dim, n, { H->uo[p] += s * L->u[p]; })
  }
  memcpy(L->u, H->uo, sizeof(double) * N);
  memcpy(L->f, H->fo, sizeof(double) * N);
  return it;
}
