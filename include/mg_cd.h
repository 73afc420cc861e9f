/* Implicit Euler steps of nonlinear complex diffusion on one GPU: C ABI of
 * libmg.so.
 *
 * Sec. 4 of the paper solves the complex diffusion equation
 *     u_t = div(g(Im u) grad u),   g(s) = e^{i theta} / (1 + (s / (kappa theta))^2),
 * on the unit square with Neumann boundaries (a small angle theta, kappa > 0),
 * discretised by averaged finite differences (finite volumes) on a
 * cell-centred grid and implicit Euler in time, each step solved by
 * multigrid with cell-centred restriction and constant interpolation. Here:
 *   grid      n = 2^m cells per dimension, h = 1/n, complex FP64 values;
 *   faces     the coefficient of the face between cells p and q is the mean
 *             (g_p + g_q) / 2 of the cell diffusivities; boundary faces carry
 *             no flux;
 *   step      the diffusivity is lagged to the previous time level (computed
 *             once from u^n), so a step solves the linear complex system
 *             (A u)_p = u_p + tau h^-2 sum_{faces f of p} g_f (u_p - u_q) = u^n_p;
 *             for a linear system the full approximation scheme and the
 *             correction scheme give the same iterates, and the V-cycle is
 *             the correction scheme of Algorithm 1;
 *   smoother  complex red-black Gauss-Seidel (red: i+j even, first) or
 *             omega-Jacobi, u += omega (f - A u) / diag;
 *   transfers restriction = mean of the 4 fine cells; constant interpolation;
 *             coarse faces = mean of the two fine faces each spans, h_H = 2h;
 *             the coarsest grid is one cell (A u = u there).
 *
 * Conventions are those of include/mg.h (status codes, mg_last_error, a
 * caller-owned 256-byte-aligned device arena, asynchronous calls except the
 * ones that return host values). Complex fields are n*n pairs of doubles
 * (real, imaginary interleaved, as C99 double complex or numpy complex128),
 * x fastest, in host or device memory.
 */
#ifndef MG_CD_H
#define MG_CD_H

#include <stddef.h>

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* n: cells per dimension, 2^m, 1 <= n <= 8192. tau > 0: time step. theta
 * != 0 (radians, small), kappa > 0: diffusivity parameters. smoother, omega
 * (0, 2), nu1, nu2 (0..8, sum > 0) as in mg_options. maxit: V-cycles allowed
 * per step. stream: cudaStream_t, NULL = default stream. */
typedef struct {
  int n;
  double tau, theta, kappa;
  int smoother;
  double omega;
  int nu1, nu2;
  int maxit;
  void *stream;
} mg_cd_params;

typedef struct mg_cd_ctx mg_cd_ctx;

/* Fields of mg_cd_set_field / mg_cd_get_field. gx: face between cells
 * (i, j) and (i+1, j) at index j*n + i (i < n-1); gy: face between (i, j)
 * and (i, j+1) (j < n-1); the last column of gx and row of gy are zero. */
enum { MG_CD_U = 0, MG_CD_F = 1, MG_CD_R = 2, MG_CD_GX = 3, MG_CD_GY = 4 };

/* n = 2, tau = 1e-3, theta = pi/30, kappa = 0.1, RBGS omega 1, V(2,2),
 * maxit 50, default stream. */
void mg_cd_default_params(mg_cd_params *p);
size_t mg_cd_workspace_bytes(const mg_cd_params *p);
mg_status mg_cd_create(const mg_cd_params *p, void *arena, size_t arena_bytes, mg_cd_ctx **out);
mg_status mg_cd_destroy(mg_cd_ctx *ctx);
int mg_cd_num_levels(const mg_cd_ctx *ctx);
int mg_cd_level_size(const mg_cd_ctx *ctx, int level);

/* Setting gx or gy also re-forms the level's omega / diag, which the smoothers use. */
mg_status mg_cd_set_field(mg_cd_ctx *ctx, int level, int field, const double *src);
/* Synchronises the stream. */
mg_status mg_cd_get_field(mg_cd_ctx *ctx, int level, int field, double *dst);

/* Starts a step from u^n: cell diffusivities from Im u^n, the fine faces,
 * every coarser level's faces, f = u^n and the start u = u^n. */
mg_status mg_cd_begin_step(mg_cd_ctx *ctx, const double *un);

/* Algorithm 1 steps on one level with the current faces (as in mg_cc.h). */
mg_status mg_cd_smooth(mg_cd_ctx *ctx, int level, int sweeps);
mg_status mg_cd_residual(mg_cd_ctx *ctx, int level);
mg_status mg_cd_restrict(mg_cd_ctx *ctx, int level);
mg_status mg_cd_prolongate(mg_cd_ctx *ctx, int level);
mg_status mg_cd_coarse_solve(mg_cd_ctx *ctx);
mg_status mg_cd_vcycle(mg_cd_ctx *ctx);

/* sqrt(sum |f - A u|^2) over the cells of a level (fixed summation order). */
mg_status mg_cd_residual_norm(mg_cd_ctx *ctx, int level, double *out);

/* V-cycles from the current u until ||r_k|| / ||r_0|| <= tol or maxit;
 * history: NULL or maxit + 1 doubles. MG_ENOCONV if tol is not reached. */
mg_status mg_cd_solve(mg_cd_ctx *ctx, double tol, int *iters, double *relres, double *history);

/* mg_cd_begin_step(un) followed by mg_cd_solve; u^{n+1} is level 0's u. */
mg_status mg_cd_time_step(mg_cd_ctx *ctx, const double *un, double tol, int *iters, double *relres,
                          double *history);

#ifdef __cplusplus
}
#endif

#endif
