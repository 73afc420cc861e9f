/*
 * mg.h - C ABI of the GB300 geometric multigrid library (libmg.so).
 *
 * The library solves the node-based finite-difference problems of
 * Koestler et al., "A Scala Prototype to Generate Multigrid Solver
 * Implementations for Different Problems and Target Multi-Core Platforms"
 * (arXiv:1406.5369):
 *
 *   -sum_d c_d d^2u/dx_d^2 = f  in [0,1]^dim,  u = g on the boundary   (Eq. 1,
 *   written there with the opposite sign; this library uses the SPD sign), or
 *   -div(k grad u) = f with a node-wise diffusivity k (harmonic-mean faces),
 *
 * with the recursive V-cycle of Algorithm 1 (Sec. 2.3): red-black
 * Gauss-Seidel or omega-Jacobi smoothing, residual, full-weighting
 * restriction, bi-/trilinear interpolation with correction and a direct
 * solve on the coarsest grid; coarse operators are rediscretised (Table 1).
 *
 * Grid layout seen by callers: a grid has n = 2^m + 1 nodes per dimension
 * including boundary nodes (h = 1/(n-1)); arrays are dense FP64 with x
 * fastest: element (i, j[, k]) at i + n*(j + n*k). Inside the arena each
 * level is stored with rows padded to 128 bytes.
 *
 * Pointers: every `const double *` input and `double *` output may be host
 * or device memory (the library copies with cudaMemcpyDefault); it is
 * borrowed for the duration of the call only. The arena is device memory
 * owned by the caller and must outlive the context. The library never
 * allocates device memory; it allocates only the small host-side context.
 *
 * Errors: every call returns an mg_status; no call aborts or throws. The
 * message of the last failure on the calling thread is mg_last_error().
 *
 * Streams: calls are asynchronous on options.stream (a cudaStream_t, NULL
 * = the legacy default stream) except mg_residual_norm, mg_solve,
 * mg_get_solution and mg_get_field, which synchronise that stream before
 * returning.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,   /* bad argument: size not 2^m+1, level out of range, NULL ... */
  MG_ENOMEM = 2,   /* arena smaller than mg_workspace_bytes() */
  MG_ECUDA = 3,    /* a CUDA runtime call failed (message in mg_last_error) */
  MG_ENOCONV = 4,  /* residual became NaN/Inf or maxit reached above tol */
  MG_ETIMEOUT = 5  /* reserved for a bounded device-side wait that gives up; no kernel of
                      this library waits on a flag, so no call returns it */
} mg_status;

/* Smoothers of the feature model (Table 1): omega red-black Gauss-Seidel
 * (Sec. 2.4 GaussSeidel, "order rb": red = i+j[+k] even, updated first) and
 * omega-Jacobi (Sec. 4, Table 2 uses omega = 0.8). */
typedef enum { MG_RBGS = 0, MG_JACOBI = 1 } mg_smoother;

/* Data type of the V-cycle (Table 1 "single/double accuracy"; Sec. 5).
 * MG_FP64: every level stored and computed in FP64.
 * MG_FP32_DC / MG_BF16_DC: defect correction - an FP64 outer loop
 * (residual, solution update) around inner V-cycles stored in FP32 or BF16
 * and computed in FP32; the coarsest direct solve stays FP64. */
typedef enum { MG_FP64 = 0, MG_FP32_DC = 1, MG_BF16_DC = 2 } mg_precision;

/* Per-level fields addressable by mg_set_field / mg_get_field. */
typedef enum { MG_FIELD_U = 0, MG_FIELD_F = 1, MG_FIELD_R = 2 } mg_field;

/* Constant stencil -sum_d c_d d^2/dx_d^2 (Sec. 2.2: a constant 5-/7-point
 * stencil stored matrix-free). Poisson: cx = cy = cz = 1. cz is ignored in 2D. */
typedef struct { double cx, cy, cz; } mg_const_stencil;

/* Boundary condition (Eq. 1b). kind 0 = Dirichlet. dirichlet_values: NULL
 * for homogeneous, else a dense n^dim FP64 array of which only boundary
 * nodes are read. */
typedef struct { int kind; const double *dirichlet_values; } mg_boundary;

/* Layer-3 parameters (Sec. 2.3 mgparameter) plus implementation choices.
 * smoother, omega       : smoother and its relaxation weight
 * nu1, nu2              : pre- and post-smoothing sweeps (0..8)
 * coarsest_n            : nodes per dimension of the coarsest grid: 3 (one
 *                         unknown), 5 or 9 ((coarsest_n-2)^dim unknowns);
 *                         n >= coarsest_n. The coarsest grid is solved
 *                         exactly in FP64; for 5 and 9 mg_create forms the
 *                         inverse of its operator (Gauss-Jordan, N x N FP64
 *                         in the arena) and each solve applies it to the
 *                         residual. MG_EINVAL for any other value
 * maxit                 : V-cycles (outer steps for *_DC) allowed in mg_solve
 * precision             : see mg_precision
 * stream                : cudaStream_t for every launch, NULL = default stream
 * fuse                  : 1 = fused fine-level kernels where available,
 *                         0 = one kernel per operator (same results up to
 *                         rounding order of FMA contraction)
 * use_graph             : 1 = replay each V-cycle from a captured CUDA graph
 * inner_cycles          : *_DC only: inner V-cycles per outer FP64 step (1..8, 0 = 1);
 *                         the first starts from e = 0, the others continue
 *                         from the current e. 1 = classic defect correction.
 * exact_outer           : *_DC only: 1 = when every axis coefficient c_d/h^2 of
 *                         the constant stencil is the same power of two
 *                         (Poisson with n = 2^m+1), the outer residual is
 *                         evaluated exactly in 64-bit fixed-point integers and
 *                         rounded once (at least FP64 accuracy, no FP64
 *                         instruction); 0 = FP64 arithmetic. The update
 *                         u += e is an FP64 addition either way.
 * Tile shape and sweep fusion of the 2D fine-level kernels (performance
 * only; every setting computes the same iteration up to FP32 rounding order
 * in the inner cycles, and the library's autotuner searches them):
 * tile_rows             : rows each warp of the streaming fused kernels walks
 *                         (rounded up to a multiple of 8); 0 = automatic (one
 *                         wave of resident warps)
 * tile_max_n            : largest level size (nodes per dimension) that runs on
 *                         the shared-memory block-tile kernels instead of the
 *                         streaming ones; 0 = 257, values below 33 = none
 * fuse_depth            : sweeps fused into each pre-/post-smoothing pass
 *                         (0 = all nu1 / nu2); with 0 < fuse_depth < nu the
 *                         other nu - fuse_depth sweeps run as separate passes
 * join_cycles           : *_DC with inner_cycles > 1 only: 1 = between two inner
 *                         V-cycles, the finest inner level's post-smoothing
 *                         pass and the next cycle's pre-smoothing pass run as
 *                         one pass (packed FP32 2D streaming levels,
 *                         nu1 + nu2 <= 3; the same operations in the same
 *                         order, so the same results), 0 = two passes
 * cluster_max_n         : *_DC, 2D constant stencil, RBGS only: the largest
 *                         inner level (129 or 257) from which the V-cycle of
 *                         every coarser level runs as one kernel on a cluster
 *                         of 16 thread blocks (8 where 16 cannot be placed)
 *                         holding the levels in their shared memory (levels
 *                         33 and below in one of them); 0 = 257, values
 *                         below 129 = never (per-level kernels and the
 *                         single-block cycle below 65)
 * canary                : 1 = debug layout: every buffer the context lays out
 *                         in the arena is followed by a 256-byte guard zone
 *                         filled with the byte 0xA5 at mg_create and checked
 *                         by mg_check_canaries (a write past the end of a
 *                         buffer changes it); mg_workspace_bytes counts the
 *                         zones; 0 = no guard zones (the packed layout) */
typedef struct {
  mg_smoother smoother;
  double omega;
  int nu1, nu2;
  int coarsest_n;
  int maxit;
  mg_precision precision;
  void *stream;
  int fuse;
  int use_graph;
  int inner_cycles;
  int exact_outer;
  int tile_rows;
  int tile_max_n;
  int fuse_depth;
  int join_cycles;
  int cluster_max_n;
  int canary;
} mg_options;

typedef struct mg_ctx mg_ctx;

/* Fills *opt with RBGS, omega 1, V(2,1), coarsest 3, maxit 50, FP64,
 * default stream, fuse 1, use_graph 1, inner_cycles 1, exact_outer 1,
 * tile_rows 0, tile_max_n 0, fuse_depth 0, join_cycles 1, cluster_max_n 0,
 * canary 0 (the Layer-3 defaults of Sec. 2.3 and automatic tiling). */
void mg_default_options(mg_options *opt);

/* Bytes of device arena mg_create needs for this problem (0 if the
 * arguments are invalid). variable_k != 0 reserves face coefficients. */
size_t mg_workspace_bytes(int dim, int n, int variable_k, const mg_options *opt);

/* Builds the grid hierarchy n, (n-1)/2+1, ..., coarsest_n inside the
 * caller's arena (Sec. 2.2 Discrete_Domain ... levels, coarsefac = 2).
 * stencil: NULL = Poisson. k: NULL for the constant stencil, else a dense
 * n^dim FP64 array of node diffusivities (> 0); face coefficients are the
 * harmonic means of the two nodes times c_d, and coarse faces combine the
 * two collinear fine faces in series, 2/(1/k_a + 1/k_b) (rediscretisation,
 * Table 1). bc: NULL = homogeneous Dirichlet. The solution starts at zero
 * (plus boundary values), the right-hand side at zero.
 * Returns MG_EINVAL for dim not 2/3, n not 2^m+1 with m >= 1, bad options;
 * MG_ENOMEM if arena_bytes < mg_workspace_bytes. On success *out owns a
 * host-side context released by mg_destroy. The set-up is queued on
 * options.stream; the call waits for it only when k or boundary values are
 * given (those arrays may be released when it returns). */
mg_status mg_create(int dim, int n, const mg_const_stencil *stencil, const double *k,
                    const mg_boundary *bc, const mg_options *opt, void *arena,
                    size_t arena_bytes, mg_ctx **out);

/* Releases the host context (the arena stays the caller's). NULL is a no-op. */
mg_status mg_destroy(mg_ctx *ctx);

/* Debug check of the arena of a context created with options.canary = 1:
 * waits for the context's stream, copies every guard zone to the host and
 * sets *damaged to the number of zones holding a byte other than 0xA5 (a
 * kernel or copy wrote past the end of the buffer before that zone). When
 * *damaged > 0, mg_last_error names the first damaged zone's buffer and the
 * offset of its first changed byte. Buffers keep their 256-byte alignment
 * with zones between them, so every kernel runs its normal code. Returns MG_EINVAL for a NULL argument or a context created
 * with canary = 0, MG_ECUDA if a copy fails; MG_OK otherwise, damaged or
 * not. Not for a stream under capture (it synchronizes). */
mg_status mg_check_canaries(mg_ctx *ctx, int *damaged);

/* Number of levels L (level 0 finest, L-1 coarsest) and nodes per dimension
 * of a level (-1 if out of range). */
int mg_num_levels(const mg_ctx *ctx);
int mg_level_size(const mg_ctx *ctx, int level);

/* Finest-level right-hand side f (dense n^dim FP64; boundary entries ignored). */
mg_status mg_set_rhs(mg_ctx *ctx, const double *f);

/* Finest-level initial guess (Sec. 2.1 "Unknown solution = init...");
 * u0 == NULL sets zero. Boundary nodes always keep the Dirichlet values. */
mg_status mg_set_solution(mg_ctx *ctx, const double *u0);

/* Copies the finest-level solution (dense n^dim FP64, boundary included).
 * A host destination is staged through the context's FP64 scratch field
 * (the level-0 residual field R of an MG_FP64 context is overwritten). */
mg_status mg_get_solution(mg_ctx *ctx, double *u);

/* Per-level access used by operator-level tests and tools: level ell's
 * solution U, right-hand side F or residual R, as dense n_ell^dim FP64
 * (converted from/to the level's storage type). In the *_DC precisions
 * the levels are the inner hierarchy (U = correction e, F = defect d). */
mg_status mg_set_field(mg_ctx *ctx, int level, mg_field field, const double *src);
mg_status mg_get_field(mg_ctx *ctx, int level, mg_field field, double *dst);

/* `sweeps` smoothing steps on `level` (Algorithm 1 presmoothing /
 * postsmoothing; Sec. 2.4 GaussSeidel). MG_EINVAL if level is out of range
 * or sweeps < 0. */
mg_status mg_smooth(mg_ctx *ctx, int level, int sweeps);

/* r_level = f_level - A_level u_level at interior nodes (Algorithm 1,
 * "compute residual"; Sec. 2.4 Residual). */
mg_status mg_residual(mg_ctx *ctx, int level);

/* f_{level+1} = R r_level with full weighting (Algorithm 1 "restrict
 * residual"; Sec. 2.4 Restrict, ToCoarse). MG_EINVAL on the coarsest level. */
mg_status mg_restrict(mg_ctx *ctx, int level);

/* u_level += P u_{level+1} with bi-/trilinear interpolation at interior
 * nodes (Algorithm 1 "prolongate error and do coarse grid correction";
 * Sec. 2.4 interpolatecorr, ToFine). MG_EINVAL on the coarsest level. */
mg_status mg_prolongate(mg_ctx *ctx, int level);

/* Exact solve on the coarsest level, in FP64 (Algorithm 1, coarsest level):
 * u += A^{-1} (f - A u) over its interior unknowns, so the result does not
 * depend on the starting u; A^{-1} is 1/diag for a 3^dim grid and the dense
 * inverse formed at creation for 5^dim and 9^dim grids. */
mg_status mg_coarse_solve(mg_ctx *ctx);

/* One V(nu1,nu2)-cycle on the finest level (Algorithm 1; Sec. 2.4 VCycle).
 * In the *_DC precisions: one defect-correction step - FP64 residual of
 * the outer problem, inner_cycles inner V-cycles (the first from zero) on
 * it, FP64 update. */
mg_status mg_vcycle(mg_ctx *ctx);

/* Euclidean norm of f - A u over the interior of `level` (Sec. 2.4
 * L2Residual), accumulated in FP64; synchronises the stream. In the *_DC
 * precisions level 0 means the outer FP64 problem. */
mg_status mg_residual_norm(mg_ctx *ctx, int level, double *out);

/* Driver loop of the Layer-4 Application (Sec. 2.4): r0 = ||f - A u||,
 * then V-cycles (defect-correction steps for *_DC) until
 * ||r_k||/r0 <= tol or maxit. *iters = cycles done, *relres = last ratio;
 * history (may be NULL) receives maxit+1 doubles, rho_0 = 1 .. rho_iters.
 * When the solution was last set to zero (mg_set_solution(ctx, NULL), or
 * the context is new) and the Dirichlet data are homogeneous, the initial
 * residual is f itself and is formed without applying the stencil.
 * Returns MG_ENOCONV if the residual is not finite or tol was not reached. */
mg_status mg_solve(mg_ctx *ctx, double tol, int *iters, double *relres, double *history);

/* A stream of independent problems with the same operator (the paper solves
 * one problem per program run; this call keeps the GPU busy while data moves
 * between host and device). Solves count right-hand sides f[i] (dense n^dim
 * FP64, host or device memory; pinned host memory lets the copies overlap
 * the solves), each from u = 0 with mg_solve to tol, and writes solution i to
 * u[i] (dense n^dim FP64, host or device). Contexts a and b must share dim,
 * n, precision and stencil kind and should have been created with the same
 * stencil, coefficients, boundary data and options; each needs its own
 * stream (options.stream), and copy_stream a third one. They take the
 * problems in turn: while one solves problem i, the other receives f[i+1]
 * on its stream and solution i-1 returns on copy_stream, so that every
 * problem's host-to-device and device-to-host copies run beside another
 * problem's solve. iters[i] and relres[i] (may be NULL) receive each solve's
 * cycles and final ratio. All three streams are synchronised before the
 * call returns; f[i] and u[i] are borrowed until then. Returns MG_EINVAL for
 * mismatched contexts, shared streams or NULL arrays, MG_ENOCONV if some
 * problem did not reach tol (the others are still solved and copied), and
 * the first other error of a solve or copy (the sequence stops there). */
mg_status mg_solve_sequence(mg_ctx *a, mg_ctx *b, void *copy_stream, int count, const double *const *f,
                            double *const *u, double tol, int *iters, double *relres);

/* Diagnostic with no counterpart in the paper: the number of CUDA kernels
 * this context has launched so far, counting each kernel node of a
 * replayed graph (memset/copy operations are not counted). */
unsigned long long mg_kernel_launches(const mg_ctx *ctx);

/* Kernel classes for mg_get_timing: presmoothing + residual + restriction,
 * interpolation + postsmoothing, the coarse-level cycle / 3^d solve, the
 * FP64 outer step of defect correction, residual norms, anything else, and
 * the joined postsmoothing + presmoothing pass of two inner cycles
 * (join_cycles). */
typedef enum {
  MG_KERNEL_PRESMOOTH = 0,
  MG_KERNEL_POSTSMOOTH = 1,
  MG_KERNEL_COARSE = 2,
  MG_KERNEL_OUTER = 3,
  MG_KERNEL_NORM = 4,
  MG_KERNEL_OTHER = 5,
  MG_KERNEL_POSTPRE = 6
} mg_kernel_kind;

/* Diagnostics with no counterpart in the paper. mg_set_timing(ctx, 1)
 * brackets every kernel the context launches with CUDA events (inside
 * captured graphs too; graphs are recaptured when the setting changes);
 * mg_set_timing(ctx, 2) only the kernels of level 0 (and the outer step and
 * finest norms), which keeps the event nodes' own cost (a few microseconds
 * each) off the other levels; mg_set_timing(ctx, 3) only the outer step of
 * defect correction; 0 switches timing off; other values give MG_EINVAL.
 * Durations are added up at synchronising calls (mg_solve,
 * mg_residual_norm, mg_get_timing); a graph replayed twice between two of
 * them contributes its last replay only. mg_get_timing returns the total
 * milliseconds and the number of timed launches of one kernel class on one
 * level (level 0 for the outer step and the finest norm); it synchronises
 * the stream. mg_reset_timing clears the totals. */
mg_status mg_set_timing(mg_ctx *ctx, int on);
mg_status mg_get_timing(mg_ctx *ctx, int kind, int level, double *total_ms, unsigned long long *count);
mg_status mg_reset_timing(mg_ctx *ctx);

/* Largest number of per-block partial sums mg_residual_norm_noalloc keeps in
 * its static device scratch. Each block covers 2048 interior nodes, so grids
 * with at most MG_NOALLOC_MAX_PARTIALS * 2048 = 67,108,864 interior nodes are
 * accepted: 2D up to n = 8193, 3D up to n = 257. */
#define MG_NOALLOC_MAX_PARTIALS 32768

/* The paper has no counterpart of this call. It returns in *out the norm
 * ||f - A u||_2 over the interior nodes (FP64 accumulation) for the constant
 * stencil (NULL = Poisson), like mg_residual_norm, for callers that may not
 * allocate device memory at all: code embedded in a framework that owns
 * every device allocation through its own pool, or a latency-critical loop
 * where cudaMalloc (which can synchronise the device) is forbidden. Such
 * callers cannot provide an arena, so this call needs no context: u and f
 * are the caller's dense n^dim FP64 device arrays (x fastest, boundary
 * nodes hold the Dirichlet values); out may be host or device memory.
 * Scratch: the reduction's partial sums live in one static device array of
 * MG_NOALLOC_MAX_PARTIALS + 32 doubles (about 256 KB) that every GPU which
 * loads the library keeps until the process exits; nothing is allocated.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress). The call cannot be made on a stream that is being
 * captured into a graph: it ends by synchronising the stream, which a
 * capturing stream refuses. All calls share the array and it keeps the last call's contents (every
 * call overwrites the slots it reads), so calls that overlap on the GPU -
 * on different streams, or from several host threads - race and must be
 * serialised by the caller. The call runs on `stream` (a cudaStream_t,
 * NULL = default stream) and synchronises it before returning.
 * Returns MG_EINVAL for dim not 2/3, n < 3, NULL pointers or a grid above the
 * limit (message in mg_last_error), MG_ECUDA if a launch fails. */
mg_status mg_residual_norm_noalloc(int dim, int n, const mg_const_stencil *stencil, const double *u,
                                   const double *f, double *out, void *stream);

/* ---- Batches of independent problems (the batching and serving patterns;
 * the paper solves one problem at a time). A batch holds contexts
 * created with mg_create that share smoother, omega, nu1, nu2, precision and
 * inner_cycles (and dim); each keeps its own arena, right-hand side,
 * solution and tolerance. A batch step runs one solve step - a V-cycle, or
 * a defect-correction step - for every listed problem at once: each fine
 * level size is one launch per operator over all problems that have it,
 * the small coarse levels of all problems run in one launch (one block per
 * problem), and the outer step and the norms run once for all. A problem's
 * arithmetic does not depend on the other problems in the batch, so its
 * result is the same alone and in any mix. ---- */
typedef struct mg_batch mg_batch;

/* Device workspace (descriptor arrays, norm partial sums, the state and
 * descriptors of captured solve steps) for at most max_problems problems;
 * 0 if max_problems < 1. */
size_t mg_batch_workspace_bytes(int max_problems);

/* Creates an empty batch using the caller's device workspace (256-byte
 * aligned, at least mg_batch_workspace_bytes bytes) and stream (NULL =
 * default). The batch allocates pinned host staging for descriptors, a
 * private stream to capture steps on and two events. */
mg_status mg_batch_create(int max_problems, void *workspace, size_t bytes, void *stream, mg_batch **out);
mg_status mg_batch_destroy(mg_batch *batch);

/* Adds a context (borrowed; it must outlive its membership) and returns its
 * id. MG_EINVAL if its options differ from the batch's, or for Jacobi with
 * an odd nu1 + nu2; MG_ENOMEM if the batch is full. The problem's initial
 * residual is taken at its first step. Work already queued on the context's
 * own stream (mg_set_rhs, mg_set_solution) is ordered before the batch's
 * later steps through an event, without waiting on the host. */
mg_status mg_batch_add(mg_batch *batch, mg_ctx *ctx, int *id);
mg_status mg_batch_remove(mg_batch *batch, int id);

/* One solve step for the `count` problems in ids (all constant or all
 * variable stencil). rho (may be NULL) receives each problem's relative
 * residual ||r|| / ||r_0|| after the step. Synchronises the batch stream. */
mg_status mg_batch_step(mg_batch *batch, const int *ids, int count, double *rho);

/* The same step in two halves, so that the host can work (and another
 * batch's step run on its own stream) while it runs: mg_batch_step_async
 * enqueues the step on the batch stream, with copies of the norms into
 * pinned host memory and an event after them, and returns; ids is copied.
 * mg_batch_step_wait waits for that event and fills rho (count entries, in
 * the order of ids; may be NULL). One step may be in flight per batch:
 * mg_batch_step_async, mg_batch_step and mg_batch_solve refuse with
 * MG_EINVAL while one is, and mg_batch_step_wait refuses when none is.
 * Problems may be added while a step is in flight (they join the next one);
 * contexts must not be removed or destroyed until it has been waited for. */
mg_status mg_batch_step_async(mg_batch *batch, const int *ids, int count);
mg_status mg_batch_step_wait(mg_batch *batch, double *rho);

/* Steps every problem in the batch until its relative residual is at most
 * tol[id] or maxit steps; iters[id] and relres[id] (arrays indexed by id,
 * may be NULL) receive the steps taken and the final ratio. MG_ENOCONV if
 * some problem did not reach its tolerance or a residual was not finite.
 * By default (mg_batch_set_capture on) two solve steps of all problems are
 * captured once into a CUDA graph and replayed: the stopping test runs on
 * the device after every step (a problem that has reached its tolerance, or
 * maxit, is skipped by every later kernel), and the host reads only a count
 * of the problems still stepping, one replay behind, so the steps run back
 * to back without waiting for the host. The iterates are the same as with
 * mg_batch_step (each problem still stops after the step that meets its
 * tolerance). Synchronises the batch stream. */
mg_status mg_batch_solve(mg_batch *batch, const double *tol, int maxit, int *iters, double *relres);

/* on = 1 (the default): mg_batch_solve replays captured steps as described
 * there; on = 0: it calls mg_batch_step once per step (the host reads every
 * problem's norm after each step). Batches whose steps do not fit the
 * captured-descriptor area of mg_batch_workspace_bytes fall back to the
 * latter by themselves. MG_EINVAL for other values. */
mg_status mg_batch_set_capture(mg_batch *batch, int on);

/* Inner V-cycles per outer step for the batch's defect-correction steps
 * (1..8), overriding the value taken from its first problem. */
mg_status mg_batch_set_inner_cycles(mg_batch *batch, int inner_cycles);

/* Rows each warp of the batch's fused 2D list launches walks per chunk
 * (rounded up to a multiple of 8; 0 = 256, the default): a tile-shape knob
 * for the autotuner. The chunking depends on this value and the level size
 * only, so a problem's results do not depend on the rest of the batch.
 * Any time, before or after problems are added; MG_EINVAL outside 0..65536. */
mg_status mg_batch_set_tile_rows(mg_batch *batch, int rows);

/* Kernels the batch has launched so far (diagnostic). */
unsigned long long mg_batch_launches(const mg_batch *batch);

/* Diagnostics with no counterpart in the paper: CUDA-event timing of the
 * batch's launch groups by kind - presmoothing + residual + restriction of
 * one level size, interpolation + postsmoothing, the coarse cycles, the outer
 * step of defect correction (its residual, or the whole fused step), the
 * separate FP64 update of the generic outer path, norms. mg_batch_set_timing
 * (1 on, 0 off; others MG_EINVAL) applies to steps run by mg_batch_step (and
 * mg_batch_solve with capture off); captured steps are not timed.
 * mg_batch_get_timing returns a kind's total milliseconds, its timed launch
 * groups and their algorithmic bytes (the compulsory traffic of the kernels'
 * operator model: each array read or written once per pass); it synchronises
 * the batch stream. mg_batch_reset_timing clears the totals. */
typedef enum {
  MG_BATCH_PRE = 0,
  MG_BATCH_POST = 1,
  MG_BATCH_COARSE = 2,
  MG_BATCH_OUTER = 3,
  MG_BATCH_UPDATE = 4,
  MG_BATCH_NORM = 5
} mg_batch_kernel;
mg_status mg_batch_set_timing(mg_batch *batch, int on);
mg_status mg_batch_get_timing(mg_batch *batch, int kind, double *total_ms, unsigned long long *launches,
                              double *bytes);
mg_status mg_batch_reset_timing(mg_batch *batch);

/* Diagnostic of the last mg_batch_solve that replayed captured steps: out[0]
 * = host milliseconds of its set-up (initial norms, state snapshots), out[1]
 * = capturing and instantiating the two-step graph, out[2] = the replays
 * until the last problem stopped (with the final synchronisation), out[3] =
 * the replays launched, out[4] = kernel nodes per replay. Zeros before any
 * such solve. */
mg_status mg_batch_solve_profile(const mg_batch *batch, double *out);

/* Message of the last failing call on this thread ("" if none). */
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MG_H */
