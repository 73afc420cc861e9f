// Internal declarations shared by the translation units of libmg.so.
// Nothing here is part of the public C ABI (include/mg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

enum DType { F64 = 0, F32 = 1, BF16 = 2 };

inline int dtype_size(int t) { return t == F64 ? 8 : (t == F32 ? 4 : 2); }
// Face coefficients are stored in the compute type of the level.
inline int face_size(int t) { return t == F64 ? 8 : 4; }

// One grid level as the kernels see it. Sizes are in elements of the
// level's storage type.
struct Level {
  int dim;          // 2 or 3
  int n;            // nodes per dimension, boundary included
  int pitch;        // row stride (elements); every row starts 128-byte aligned
  long long plane;  // plane stride (elements) = pitch * n
  long long count;  // elements per field = plane * (dim == 3 ? n : 1)
  int dtype;        // DType of u, f, r
  void *u[2];       // solution, ping-pong pair; cur selects the live one
  void *f;          // right-hand side
  void *r;          // residual / scratch
  void *kf[3];      // face coefficients (NULL for the constant stencil); kf[d][p] is
                    // the face between node p and p + e_d, same indexing as u
  double c[3];      // constant stencil coefficients
  double inv_h2;    // 1/h^2
  int cur;          // index of the live solution buffer
  double *dense;    // coarsest level with more than one unknown: the FP64
                    // inverse of its operator, N x N row-major over the N
                    // interior nodes in lexicographic order (x fastest);
                    // NULL on every other level and for a 3^dim coarsest grid
};

// Interior unknowns of the largest coarsest grid with a dense solve (9^3).
constexpr int kDenseMax = 343;

constexpr int kNormBlocks = 1024;
constexpr int kMaxPartials = 16384;  // per-warp partial sums of the streaming norms

// Exponent k when every axis coefficient of L's constant stencil, c_d / h^2,
// equals the same power of two 2^k (the exact fixed-point outer step needs
// it, fixed.cuh); kNoPow2 otherwise (and for variable stencils).
constexpr int kNoPow2 = -100000;
int pow2_stencil(const Level &L);

// Per-dimension kernel launchers; all asynchronous on `s`.
#define MG_DIM_OPS                                                                                \
  cudaError_t rbgs_half(const Level &L, void *u, const void *f, int color, double omega,         \
                        cudaStream_t s);                                                          \
  cudaError_t jacobi(const Level &L, const void *uin, void *uout, const void *f, double omega,   \
                     cudaStream_t s);                                                             \
  cudaError_t residual(const Level &L, const void *u, const void *f, void *r, cudaStream_t s);   \
  cudaError_t restrict_fw(const Level &F, const void *rf, const Level &C, void *fc,              \
                          cudaStream_t s);                                                        \
  cudaError_t prolong(const Level &C, const void *ec, const Level &F, void *uf, cudaStream_t s); \
  cudaError_t norm_partials(const Level &L, const void *u, const void *f, double *partials,       \
                            int nblocks, cudaStream_t s);                                         \
  cudaError_t coarse3(const Level &L, void *u, const void *f, cudaStream_t s);                   \
  cudaError_t dense_inverse(const Level &L, cudaStream_t s);                                     \
  cudaError_t coarse_dense(const Level &L, void *u, const void *f, cudaStream_t s);              \
  cudaError_t dc_residual(const Level &O, const void *u, const void *f, const Level &I, void *d, \
                          double *partials, int nblocks, cudaStream_t s);                         \
  cudaError_t dc_update(const Level &O, void *u, const Level &I, const void *e, cudaStream_t s); \
  cudaError_t from_dense(const Level &L, const double *src, void *dst, cudaStream_t s);          \
  cudaError_t to_dense(const Level &L, const void *src, double *dst, cudaStream_t s);            \
  cudaError_t zero_interior(const Level &L, void *field, cudaStream_t s);                        \
  cudaError_t copy_boundary(const Level &L, const void *src, void *dst, cudaStream_t s);         \
  cudaError_t node_faces(const Level &K, const double *knode, const Level &Lout, cudaStream_t s); \
  cudaError_t coarsen_faces(const Level &F, const Level &C, cudaStream_t s);                     \
  cudaError_t convert_faces(const Level &src, const Level &dst, cudaStream_t s);

namespace d2 {
MG_DIM_OPS
}
namespace d3 {
MG_DIM_OPS
}

// Fused 2D fine-level kernels (constant stencil, RBGS): nu sweeps +
// residual + restriction into fc, and interpolation/correction + nu sweeps.
// R = rows per chunk of the streaming kernels (0 = automatic); levels up to
// tile_max_n nodes per dimension run on the block-tile kernels (0 = the
// default size, below 33 = none).
namespace d2 {
bool fused_ok(const Level &L, const Level &Cl, int nu);
cudaError_t pre_fused(const Level &L, const void *uin, void *uout, const Level &Cl, void *fc, bool zero, int nu,
                      double omega, int R, int tile_max_n, cudaStream_t s);
cudaError_t post_fused(const Level &L, const void *uin, void *uout, const Level &Cl, const void *ec, int nu,
                       double omega, int R, int tile_max_n, cudaStream_t s);
// Post-smoothing (nu2 sweeps) of one V-cycle and pre-smoothing (nu1 sweeps,
// residual, restriction into fc) of the next in one pass, on a packed-FP32
// constant-stencil streaming level (postpre_ok): u_out = the u the two
// separate passes would leave, fc = their restricted residual.
bool postpre_ok(const Level &L, const Level &Cl, int nu2, int nu1, int tile_max_n);
cudaError_t postpre_fused(const Level &L, const void *uin, void *uout, const Level &Cl, const void *ec, void *fc,
                          int nu2, int nu1, double omega, int R, int tile_max_n, cudaStream_t s);
}  // namespace d2

// Streaming 2D finest-level kernels (constant stencil). dc_step: FP64 outer
// step of defect correction (optional update u_out = u_in + e, residual ->
// defect d, per-warp partial sums); norm_stream: per-warp partial sums of
// the level residual squared. *nparts receives the number of partials.
namespace d2 {
// exact: take the fixed-point kernel (k_dcx2d) when the step updates and the
// stencil is one power of two (pow2_stencil).
bool outer_ok(const Level &O, const Level &I);
cudaError_t dc_step(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d,
                    double *partials, int *nparts, const float *scale, bool update, bool acc64, bool exact,
                    cudaStream_t s);
bool norm_ok(const Level &L);
cudaError_t norm_stream(const Level &L, const void *u, const void *f, double *partials, int *nparts, cudaStream_t s);
}  // namespace d2

// Plane-marching 3D kernels for constant-stencil levels (stencil3d.cuh):
// z_ok says whether a level takes them; transfer_ok whether a fine/coarse
// pair does (same storage type). dc_step, norm_ok and norm_stream have the
// meaning of their 2D namespaces' counterparts; partial sums are per block.
namespace d3 {
bool z_ok(const Level &L);
bool transfer_ok(const Level &F, const Level &C);
cudaError_t z_sweep(const Level &L, const void *uin, void *uout, const void *f, int color, double omega,
                    cudaStream_t s);
// two omega-Jacobi sweeps from u = 0 in one pass: uout = J(J(0)) = J(alpha f)
// (f must be zero on the boundary; kJZ in stencil3d.cuh)
cudaError_t z_jacobi_zero2(const Level &L, const void *f, void *uout, double omega, cudaStream_t s);
cudaError_t z_residual(const Level &L, const void *u, const void *f, void *r, cudaStream_t s);
cudaError_t z_restrict(const Level &F, const void *rf, const Level &C, void *fc, cudaStream_t s);
cudaError_t z_prolong(const Level &C, const void *ec, const Level &F, void *uf, cudaStream_t s);
bool outer_ok(const Level &O, const Level &I);
cudaError_t dc_step(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d,
                    double *partials, int *nparts, const float *scale, bool update, bool acc64, bool exact,
                    cudaStream_t s);
bool norm_ok(const Level &L);
cudaError_t norm_stream(const Level &L, const void *u, const void *f, double *partials, int *nparts, cudaStream_t s);
}  // namespace d3

// Residual of u = 0 under homogeneous Dirichlet data (= f, exactly) on the
// FP64 level O: kNormBlocks partial sums of f^2 over the interior and, when
// I is given (defect correction), f written as I's right-hand side.
cudaError_t first_defect(const Level &O, const Level *I, double *partials, cudaStream_t s);
// The same over a list of problems in device memory (the batch engine): the
// FP64 outer level's f, the inner level-0 defect, `blocks` partial sums per
// problem into its own slots; grid (blocks, count).
struct FirstRec {
  const double *f;
  void *d;
  int n;
  long long sy, sz, syi, szi;  // outer and inner row / plane strides (elements)
  double *partials;
  const int *live;             // NULL: always live
};
FirstRec first_record(const Level &O, const Level &I, double *partials, const int *live);
cudaError_t first_defect_list(int dim, int inner_dtype, const FirstRec *list, int count, int blocks,
                              cudaStream_t s);

// Deterministic sum of nb partials (any nb): out[0] = sqrt(sum) / *scale_in
// (scale_in may be NULL), out[1] = sum; scale_out (may be NULL) receives the
// power of two for the next scaled pass.
cudaError_t norm_finalize_ex(const double *partials, int nb, double *out, const float *scale_in, float *scale_out,
                             double nint, cudaStream_t s);

// Single-block V-cycle of levels first..nl-1 (coarse.cuh); the levels below
// `first` are not written back. coarse_top_n: largest level size it takes.
int coarse_top_n(int dim, bool fp64);
cudaError_t coarse_cycle(const Level *lv, int first, int nl, bool zero_top, int smoother, double omega, int nu1,
                         int nu2, bool fp64, cudaStream_t s);
// Fills the kernel arguments of one problem's coarse cycle into args_out
// (coarse_args_bytes() bytes); returns the shared memory it needs, 0 if the
// levels do not fit. coarse_cycle_batched runs `count` such argument
// records (device memory) with one block each.
size_t coarse_args(const Level *lv, int first, int nl, bool zero_top, int smoother, double omega, int nu1, int nu2,
                   bool fp64, void *args_out);
size_t coarse_args_bytes();
// V-cycle of levels first..nl-1 on one cluster of thread blocks (2D,
// constant stencil, RBGS, FP32 arithmetic; cluster.cuh). cluster_ok: level
// l takes it (size within cluster_max_n, the hierarchy's shape, and a
// cluster of that size fits the device).
bool cluster_ok(const Level *lv, int l, int nl, int smoother, bool fp64, int cluster_max_n);
// Asks the device once whether the cluster fits (outside any stream capture:
// mg_create calls it); cluster_ok answers no until it has run.
void cluster_probe();
cudaError_t cluster_cycle(const Level *lv, int first, int nl, bool zero_top, double omega, int nu1, int nu2,
                          cudaStream_t s);
// Points a filled argument record at its problem's live flag (captured batch steps).
void coarse_args_set_live(void *args, const int *live);
cudaError_t coarse_cycle_batched(const void *list_dev, int count, int dim, bool var, bool fp64, size_t smem,
                                 cudaStream_t s);

// Sets the message mg_last_error() returns on the calling thread.
void set_error_message(const char *msg);

// out[0] = sqrt(sum of partials), out[1] = the sum; fixed summation order.
cudaError_t norm_finalize(const double *partials, int nblocks, double *out, cudaStream_t s);

}  // namespace mg
