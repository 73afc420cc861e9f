/* Cell-centred geometric multigrid on one GPU: C ABI of libmg.so.
 *
 * The paper's feature model (Table 1) has two locations of grid points,
 * node-based (include/mg.h) and cell-centred, and Neumann as well as
 * Dirichlet boundaries; its complex-diffusion runs (Sec. 4) use cell-centred
 * grids with Neumann boundaries, finite volumes, cell-centred restriction and
 * constant interpolation. This interface solves the real, constant-
 * coefficient operator of that setting,
 *     sigma u - sum_d c_d d^2u/dx_d^2 = f   on the unit square / cube,
 * sigma >= 0 (sigma = 1/dt is one implicit Euler step of the diffusion
 * equation), by V-cycles of Algorithm 1:
 *   grid      n = 2^m cells per dimension, h = 1/n, cell centres
 *             x_i = (i + 1/2) h; no ghost cells are stored;
 *   operator  (A u)_p = sigma u_p + h^-2 sum_d c_d (F_- + F_+) with
 *             F = u_p - u_q across an interior face (neighbour q),
 *             F = 0 across a Neumann (zero-flux) boundary face,
 *             F = 2 u_p across a homogeneous Dirichlet face (ghost -u_p);
 *   smoother  red-black Gauss-Seidel (red: i+j[+k] even, first) or
 *             omega-Jacobi, u += omega (f - A u) / diag;
 *   restrict  f_H = mean of the 2^dim fine residuals of each coarse cell;
 *   prolong   constant interpolation, u_h += u_H of the parent cell;
 *   coarse    operators rediscretised with h_H = 2h (Table 1, "direct
 *             (re-discretization)"); the coarsest grid (1, 2 or 4 cells per
 *             dimension) is solved exactly in FP64 with its inverse, formed
 *             at creation.
 * Everything runs in FP64.
 *
 * Conventions are those of include/mg.h: status codes (mg_status) and
 * mg_last_error() for the message; the caller owns the arena (device memory,
 * 256-byte aligned, at least mg_cc_workspace_bytes) and the library never
 * allocates device memory after creation; calls are asynchronous on the
 * stream except mg_cc_get_field, mg_cc_residual_norm and mg_cc_solve.
 * Dense fields are n^dim FP64 values, x fastest, in host or device memory.
 */
#ifndef MG_CC_H
#define MG_CC_H

#include <stddef.h>

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { MG_CC_NEUMANN = 0, MG_CC_DIRICHLET = 1 } mg_cc_bc;

/* Problem and method. dim: 2 or 3. n: cells per dimension, 2^m with
 * 1 <= n <= 16384 (2D) or 1024 (3D). c: axis coefficients, > 0 (c[2] unused
 * in 2D). sigma >= 0, and > 0 with Neumann faces (otherwise the constants
 * are a null space). bc: mg_cc_bc, on every face. smoother, omega (0, 2),
 * nu1, nu2 (0..8, sum > 0) as in mg_options. coarsest_n: cells per
 * dimension of the coarsest grid, 1, 2 or 4, <= n. maxit: V-cycles allowed
 * in mg_cc_solve. stream: cudaStream_t, NULL = default stream. */
typedef struct {
  int dim, n;
  double c[3];
  double sigma;
  int bc;
  int smoother;
  double omega;
  int nu1, nu2;
  int coarsest_n;
  int maxit;
  void *stream;
} mg_cc_params;

typedef struct mg_cc_ctx mg_cc_ctx;

/* 2D, n = 2, c = 1, sigma = 1, Neumann, RBGS omega 1, V(2,1), coarsest 1,
 * maxit 50, default stream. */
void mg_cc_default_params(mg_cc_params *p);

/* Arena bytes for these parameters; 0 if they are invalid (mg_last_error). */
size_t mg_cc_workspace_bytes(const mg_cc_params *p);

/* Lays out the hierarchy n, n/2, ..., coarsest_n in the arena, zeroes it
 * and forms the coarsest grid's inverse. Synchronises the stream.
 * MG_EINVAL for invalid parameters, MG_ENOMEM for a short arena. */
mg_status mg_cc_create(const mg_cc_params *p, void *arena, size_t arena_bytes, mg_cc_ctx **out);
mg_status mg_cc_destroy(mg_cc_ctx *ctx);

/* Levels (0 finest) and cells per dimension of one level (-1 if invalid). */
int mg_cc_num_levels(const mg_cc_ctx *ctx);
int mg_cc_level_size(const mg_cc_ctx *ctx, int level);

/* Dense copies of a level's field: 0 = u, 1 = f, 2 = r. */
mg_status mg_cc_set_field(mg_cc_ctx *ctx, int level, int field, const double *src);
mg_status mg_cc_get_field(mg_cc_ctx *ctx, int level, int field, double *dst);

/* Algorithm 1 steps on one level: `sweeps` smoothing sweeps; r = f - A u;
 * f_{level+1} = R r_level; u_level += P u_{level+1}; the exact solve of the
 * coarsest level (u += A^{-1}(f - A u)). MG_EINVAL for a level out of range
 * (restrict / prolongate: the coarsest level too). */
mg_status mg_cc_smooth(mg_cc_ctx *ctx, int level, int sweeps);
mg_status mg_cc_residual(mg_cc_ctx *ctx, int level);
mg_status mg_cc_restrict(mg_cc_ctx *ctx, int level);
mg_status mg_cc_prolongate(mg_cc_ctx *ctx, int level);
mg_status mg_cc_coarse_solve(mg_cc_ctx *ctx);

/* One V(nu1, nu2)-cycle from level 0 (coarse levels start from zero). */
mg_status mg_cc_vcycle(mg_cc_ctx *ctx);

/* ||f - A u||_2 over the cells of a level, FP64, summed in a fixed order. */
mg_status mg_cc_residual_norm(mg_cc_ctx *ctx, int level, double *out);

/* V-cycles from the current u until ||r_k|| / ||r_0|| <= tol or maxit;
 * history (NULL or maxit + 1 doubles) receives rho_0 = 1, rho_1, ...
 * MG_ENOCONV if tol was not reached or the residual is not finite. */
mg_status mg_cc_solve(mg_cc_ctx *ctx, double tol, int *iters, double *relres, double *history);

#ifdef __cplusplus
}
#endif

#endif
