// Cell-centred multigrid (include/mg_cc.h): the cell-centred grid type of
// the paper's feature model (Table 1) with Neumann or Dirichlet boundary
// faces, cell-centred restriction and constant interpolation (Sec. 4), on
// the FP64 operator sigma u - sum_d c_d d^2u/dx_d^2 (finite volumes).
//
// Layout: level l has n_l = n / 2^l cells per dimension, four FP64 fields
// u[0], u[1] (Jacobi ping-pong), f, r with rows padded to 128 bytes (pitch =
// n_l rounded up to 16 doubles), x fastest, no ghost cells: the kernels read
// a neighbour only across an interior face and apply the boundary rule
// (zero flux, or the ghost -u_p of a homogeneous Dirichlet face) in
// registers. One thread per cell (per cell of the swept colour for
// red-black Gauss-Seidel), rows on blockIdx.y, planes on blockIdx.z, so a
// warp reads consecutive doubles of one row.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "mg_cc.h"
#include "mg_internal.h"

namespace mg {
namespace cc {

constexpr int kMaxLev = 16;
constexpr int kCoarseMax = 64;  // unknowns of the largest coarsest grid (4^3)
constexpr int kThreads = 256;
constexpr int kNormBlocks = 4096;  // enough blocks to hide FP64 latency on every level

struct Geo {
  int n;
  long long sy, sz;  // row and plane strides (elements)
};

// FP64 runs at 1/64 of the FP32 rate on this GPU, so the kernels are bound
// by FP64 issue, not by memory: the operator is written to need few FP64
// instructions per cell. A boundary face uses a ghost value (u_p for a
// Neumann face, -u_p for a Dirichlet one), so every face is one subtraction
// u_p - u_q (exactly 0 or 2 u_p at the boundary, as the operator defines),
// and the smoothers multiply by omega / diag_p from a table instead of
// dividing: diag_p depends only on which faces of the cell are boundary
// faces, class a_d = [x_d == 0] + [x_d == n-1] per axis, 3^dim classes.
struct Coef {
  double k[3];        // c_d / h^2 = c_d n^2 (exact scaling: n is a power of two)
  double sigma, ih2;  // ih2 = 1/h^2 = n^2
  int neumann;        // ghost value u_p (Neumann) or -u_p (Dirichlet)
  double wd[27];      // omega / diag by boundary class a_0 + 3 a_1 + 9 a_2
};

// (A u)_p of cell (i, j, k) at index p (the operator of mg_cc.h); cls gets
// the cell's boundary class.
template <int DIM>
__device__ __forceinline__ double apply(const double *__restrict__ u, long long p, int i, int j, int k,
                                        const Geo &g, const Coef &s, int &cls) {
  const double u0 = u[p], gh = s.neumann ? u0 : -u0;
  const int x[3] = {i, j, k};
  const long long st[3] = {1, g.sy, g.sz};
  const int mul[3] = {1, 3, 9};
  double acc = 0.0;
  cls = 0;
#pragma unroll
  for (int d = 0; d < DIM; d++) {
    const bool lo = x[d] == 0, hi = x[d] == g.n - 1;
    const double um = lo ? gh : u[p - st[d]];
    const double up = hi ? gh : u[p + st[d]];
    acc += s.k[d] * ((u0 - um) + (u0 - up));
    cls += mul[d] * ((int)lo + (int)hi);
  }
  return s.sigma * u0 + acc;
}

struct Cell {
  int i, j, k;
  long long p;
  bool ok;
};

template <int DIM> __device__ __forceinline__ Cell cell_of(const Geo &g, int i) {
  Cell c;
  c.i = i;
  c.j = blockIdx.y;
  c.k = DIM == 3 ? (int)blockIdx.z : 0;
  c.p = (long long)c.k * g.sz + (long long)c.j * g.sy + i;
  c.ok = i < g.n;
  return c;
}

// Half-sweep of red-black Gauss-Seidel: thread t of a row takes the t-th
// cell of the colour ((i + j + k) % 2 == color) in that row.
template <int DIM>
__global__ void k_rbgs_half(double *__restrict__ u, const double *__restrict__ f, Geo g, Coef s, int color) {
  const int j = blockIdx.y, k = DIM == 3 ? (int)blockIdx.z : 0;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  Cell c = cell_of<DIM>(g, 2 * t + ((color + j + k) & 1));
  if (!c.ok) return;
  int cls;
  const double Au = apply<DIM>(u, c.p, c.i, c.j, c.k, g, s, cls);
  u[c.p] = u[c.p] + s.wd[cls] * (f[c.p] - Au);
}

template <int DIM>
__global__ void k_jacobi(const double *__restrict__ uin, double *__restrict__ uout, const double *__restrict__ f,
                         Geo g, Coef s) {
  Cell c = cell_of<DIM>(g, blockIdx.x * blockDim.x + threadIdx.x);
  if (!c.ok) return;
  int cls;
  const double Au = apply<DIM>(uin, c.p, c.i, c.j, c.k, g, s, cls);
  uout[c.p] = uin[c.p] + s.wd[cls] * (f[c.p] - Au);
}

template <int DIM>
__global__ void k_residual(const double *__restrict__ u, const double *__restrict__ f, double *__restrict__ r,
                           Geo g, Coef s) {
  Cell c = cell_of<DIM>(g, blockIdx.x * blockDim.x + threadIdx.x);
  if (!c.ok) return;
  int cls;
  r[c.p] = f[c.p] - apply<DIM>(u, c.p, c.i, c.j, c.k, g, s, cls);
}

// Coarse cell (I, J, K): mean of its 2^DIM fine cells (2I+a, 2J+b, 2K+e).
template <int DIM>
__global__ void k_restrict(const double *__restrict__ rf, Geo gf, double *__restrict__ fc, Geo gc) {
  Cell c = cell_of<DIM>(gc, blockIdx.x * blockDim.x + threadIdx.x);
  if (!c.ok) return;
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < (DIM == 3 ? 2 : 1); e++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const double *row = rf + (long long)(2 * c.k + e) * gf.sz + (long long)(2 * c.j + b) * gf.sy + 2 * c.i;
      acc += row[0];
      acc += row[1];
    }
  fc[c.p] = (DIM == 3 ? 0.125 : 0.25) * acc;
}

// Constant interpolation and correction: u_p += e_{parent(p)}.
template <int DIM>
__global__ void k_prolong(const double *__restrict__ ec, Geo gc, double *__restrict__ uf, Geo gf) {
  Cell c = cell_of<DIM>(gf, blockIdx.x * blockDim.x + threadIdx.x);
  if (!c.ok) return;
  uf[c.p] += ec[(long long)(c.k >> 1) * gc.sz + (long long)(c.j >> 1) * gc.sy + (c.i >> 1)];
}

// Fixed-order norm: block b sums r^2 over rows b, b + gridDim, ... (thread t
// over cells t, t + 256, ... of each row), then a fixed-shape tree; no 64-bit
// index division per cell.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double buf[kThreads];
  buf[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) buf[threadIdx.x] += buf[threadIdx.x + s];
    __syncthreads();
  }
  return buf[0];
}

template <int DIM>
__global__ void k_norm_partials(const double *__restrict__ u, const double *__restrict__ f, Geo g, Coef s,
                                double *__restrict__ partials) {
  const int n = g.n, rows = DIM == 3 ? n * n : n;
  double acc = 0.0;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = row % n, k = DIM == 3 ? row / n : 0;
    const long long base = (long long)k * g.sz + (long long)j * g.sy;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      int cls;
      const double r = f[base + i] - apply<DIM>(u, base + i, i, j, k, g, s, cls);
      acc += r * r;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_norm_final(const double *__restrict__ partials, int count, double *__restrict__ out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < count; i += kThreads) a += partials[i];
  a = block_sum(a);
  if (threadIdx.x == 0) out[0] = sqrt(a);
}

// Cell t of the coarsest grid in lexicographic order (x fastest).
template <int DIM> __device__ __forceinline__ void coarse_cell(int t, int n, int &i, int &j, int &k) {
  i = t % n;
  j = DIM == 3 ? (t / n) % n : t / n;
  k = DIM == 3 ? t / (n * n) : 0;
}

// One block: assembles the coarsest operator over its N = n^DIM cells
// (row t: diag_t, and -c_d/h^2 for each neighbour across an interior face)
// and inverts it in place by Gauss-Jordan elimination without pivoting (A
// is symmetric positive definite: sigma > 0 or Dirichlet faces). A
// Dirichlet face adds 2 c_d/h^2 to the diagonal, a Neumann face nothing.
template <int DIM>
__global__ void k_dense_inverse(double *a, Geo g, Coef s) {
  __shared__ double colk[kCoarseMax];
  __shared__ double rpiv;
  const int n = g.n, N = DIM == 3 ? n * n * n : n * n;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) a[e] = 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    int x[3];
    coarse_cell<DIM>(t, n, x[0], x[1], x[2]);
    const int ts[3] = {1, n, n * n};
    double w = 0.0;
    for (int d = 0; d < DIM; d++) {
      if (x[d] > 0) {
        a[t * N + t - ts[d]] = -s.k[d];
        w += s.k[d];
      } else if (!s.neumann) {
        w += 2.0 * s.k[d];
      }
      if (x[d] < n - 1) {
        a[t * N + t + ts[d]] = -s.k[d];
        w += s.k[d];
      } else if (!s.neumann) {
        w += 2.0 * s.k[d];
      }
    }
    a[t * N + t] = s.sigma + w;
  }
  __syncthreads();
  for (int k = 0; k < N; k++) {
    if (threadIdx.x == 0) rpiv = 1.0 / a[k * N + k];
    for (int i = threadIdx.x; i < N; i += blockDim.x) colk[i] = a[i * N + k];
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) a[k * N + j] = (j == k ? 1.0 : a[k * N + j]) * rpiv;
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int i = e / N, j = e % N;
      if (i == k) continue;
      a[e] = (j == k ? 0.0 : a[e]) - colk[i] * a[k * N + j];
    }
    __syncthreads();
  }
}

// One block: u += A^{-1} (f - A u) on the coarsest grid.
template <int DIM>
__global__ void k_coarse_solve(double *__restrict__ u, const double *__restrict__ f, Geo g, Coef s,
                               const double *__restrict__ ainv) {
  __shared__ double r[kCoarseMax];
  const int n = g.n, N = DIM == 3 ? n * n * n : n * n;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    int i, j, k;
    coarse_cell<DIM>(t, n, i, j, k);
    const long long p = (long long)k * g.sz + (long long)j * g.sy + i;
    int cls;
    r[t] = f[p] - apply<DIM>(u, p, i, j, k, g, s, cls);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < N; q++) acc += ainv[q * N + t] * r[q];
    int i, j, k;
    coarse_cell<DIM>(t, n, i, j, k);
    u[(long long)k * g.sz + (long long)j * g.sy + i] += acc;
  }
}

struct Lev {
  int n, pitch;
  long long plane, count;
  double *u[2], *f, *r;
  int cur;
};

}  // namespace cc
}  // namespace mg

using namespace mg::cc;

struct mg_cc_ctx {
  mg_cc_params p;
  int nl;
  Lev lv[kMaxLev];
  double *ainv;      // coarsest grid inverse, N x N
  double *partials;  // kNormBlocks norm partial sums
  double *norm_out;  // one double
  cudaStream_t s;
};

namespace {

thread_local char g_cc_err[256];

mg_status ccfail(mg_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_cc_err, sizeof g_cc_err, fmt, ap);
  va_end(ap);
  mg::set_error_message(g_cc_err);
  return st;
}

#define CCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return ccfail(MG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

mg_status check_params(const mg_cc_params *p) {
  if (!p) return ccfail(MG_EINVAL, "params are NULL");
  if (p->dim != 2 && p->dim != 3) return ccfail(MG_EINVAL, "dim must be 2 or 3 (got %d)", p->dim);
  if (!pow2(p->n) || p->n > (p->dim == 2 ? 16384 : 1024))
    return ccfail(MG_EINVAL, "n must be a power of two, at most %d in %dD (got %d)", p->dim == 2 ? 16384 : 1024,
                  p->dim, p->n);
  for (int d = 0; d < p->dim; d++)
    if (!(p->c[d] > 0.0)) return ccfail(MG_EINVAL, "axis coefficients must be > 0");
  if (p->bc != MG_CC_NEUMANN && p->bc != MG_CC_DIRICHLET) return ccfail(MG_EINVAL, "unknown boundary kind");
  if (!(p->sigma >= 0.0) || !isfinite(p->sigma)) return ccfail(MG_EINVAL, "sigma must be finite and >= 0");
  if (p->bc == MG_CC_NEUMANN && !(p->sigma > 0.0))
    return ccfail(MG_EINVAL, "sigma must be > 0 with Neumann faces (constants are a null space otherwise)");
  if (p->smoother != MG_RBGS && p->smoother != MG_JACOBI) return ccfail(MG_EINVAL, "unknown smoother");
  if (!(p->omega > 0.0 && p->omega < 2.0)) return ccfail(MG_EINVAL, "omega must lie in (0, 2)");
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 > 8 || p->nu2 > 8 || p->nu1 + p->nu2 == 0)
    return ccfail(MG_EINVAL, "nu1, nu2 must lie in 0..8 with a positive sum");
  if (p->coarsest_n != 1 && p->coarsest_n != 2 && p->coarsest_n != 4)
    return ccfail(MG_EINVAL, "coarsest_n must be 1, 2 or 4 (got %d)", p->coarsest_n);
  if (p->coarsest_n > p->n) return ccfail(MG_EINVAL, "coarsest_n (%d) exceeds n (%d)", p->coarsest_n, p->n);
  if (p->maxit < 0) return ccfail(MG_EINVAL, "maxit must be >= 0");
  return MG_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Lays out the context's buffers from `base` (NULL: sizing only).
size_t layout(mg_cc_ctx *c, char *base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align256(off);
    void *q = base ? base + off : nullptr;
    off += bytes;
    return (double *)q;
  };
  const int dim = c->p.dim;
  c->nl = 0;
  for (int n = c->p.n; n >= c->p.coarsest_n; n /= 2) {
    Lev &L = c->lv[c->nl++];
    L.n = n;
    L.pitch = (n + 15) / 16 * 16;
    L.plane = (long long)L.pitch * n;
    L.count = L.plane * (dim == 3 ? n : 1);
    L.cur = 0;
    size_t bytes = (size_t)L.count * sizeof(double);
    L.u[0] = take(bytes);
    L.u[1] = take(bytes);
    L.f = take(bytes);
    L.r = take(bytes);
    if (n == c->p.coarsest_n) break;
  }
  const int nc = c->lv[c->nl - 1].n;
  const size_t N = (size_t)nc * nc * (dim == 3 ? nc : 1);
  c->ainv = take(N * N * sizeof(double));
  c->partials = take(kNormBlocks * sizeof(double));
  c->norm_out = take(sizeof(double));
  return align256(off);
}

Geo geo_of(const Lev &L) { return Geo{L.n, (long long)L.pitch, L.plane}; }

Coef coef_of(const mg_cc_ctx *c, const Lev &L) {
  Coef s;
  memset(&s, 0, sizeof s);
  s.sigma = c->p.sigma;
  s.ih2 = (double)L.n * (double)L.n;
  for (int d = 0; d < 3; d++) s.k[d] = c->p.c[d] * s.ih2;
  const bool neumann = c->p.bc == MG_CC_NEUMANN;
  s.neumann = neumann;
  // diag of each boundary class: per axis, a_d boundary faces (a_d = 2 only
  // for a single cell) weigh 0 (Neumann) or 2 (Dirichlet), interior faces 1
  const int dim = c->p.dim;
  for (int cls = 0; cls < 27; cls++) {
    int a[3] = {cls % 3, (cls / 3) % 3, cls / 9};
    bool valid = true;
    double w = 0.0;
    for (int d = 0; d < 3; d++) {
      if (d >= dim) {
        valid = valid && a[d] == 0;
        continue;
      }
      if (a[d] == 2 && L.n != 1) valid = false;
      w += c->p.c[d] * ((2 - a[d]) + (neumann ? 0 : 2 * a[d]));
    }
    s.wd[cls] = valid ? c->p.omega / (s.sigma + w * s.ih2) : 0.0;
  }
  return s;
}

dim3 grid_of(const Lev &L, int cells_per_row) {
  return dim3((unsigned)((cells_per_row + kThreads - 1) / kThreads), (unsigned)L.n,
              L.count > L.plane ? (unsigned)L.n : 1u);
}

#define DIMCALL(dim, kern, grid, block, ...)                                    \
  do {                                                                          \
    if ((dim) == 2) kern<2><<<grid, block, 0, c->s>>>(__VA_ARGS__);             \
    else kern<3><<<grid, block, 0, c->s>>>(__VA_ARGS__);                        \
    CCK(cudaGetLastError());                                                    \
  } while (0)

mg_status op_smooth(mg_cc_ctx *c, int l, int sweeps) {
  Lev &L = c->lv[l];
  const Geo g = geo_of(L);
  const Coef s = coef_of(c, L);
  for (int it = 0; it < sweeps; it++) {
    if (c->p.smoother == MG_RBGS) {
      for (int color = 0; color < 2; color++)
        DIMCALL(c->p.dim, k_rbgs_half, grid_of(L, (L.n + 1) / 2), kThreads, L.u[L.cur], L.f, g, s, color);
    } else {
      DIMCALL(c->p.dim, k_jacobi, grid_of(L, L.n), kThreads, L.u[L.cur], L.u[L.cur ^ 1], L.f, g, s);
      L.cur ^= 1;
    }
  }
  return MG_OK;
}

mg_status op_residual(mg_cc_ctx *c, int l) {
  Lev &L = c->lv[l];
  DIMCALL(c->p.dim, k_residual, grid_of(L, L.n), kThreads, L.u[L.cur], L.f, L.r, geo_of(L), coef_of(c, L));
  return MG_OK;
}

mg_status op_restrict(mg_cc_ctx *c, int l) {
  Lev &F = c->lv[l], &C = c->lv[l + 1];
  DIMCALL(c->p.dim, k_restrict, grid_of(C, C.n), kThreads, F.r, geo_of(F), C.f, geo_of(C));
  return MG_OK;
}

mg_status op_prolong(mg_cc_ctx *c, int l) {
  Lev &F = c->lv[l], &C = c->lv[l + 1];
  DIMCALL(c->p.dim, k_prolong, grid_of(F, F.n), kThreads, C.u[C.cur], geo_of(C), F.u[F.cur], geo_of(F));
  return MG_OK;
}

mg_status op_coarse(mg_cc_ctx *c) {
  Lev &L = c->lv[c->nl - 1];
  DIMCALL(c->p.dim, k_coarse_solve, 1, 64, L.u[L.cur], L.f, geo_of(L), coef_of(c, L), c->ainv);
  return MG_OK;
}

mg_status op_norm(mg_cc_ctx *c, int l) {
  Lev &L = c->lv[l];
  DIMCALL(c->p.dim, k_norm_partials, kNormBlocks, kThreads, L.u[L.cur], L.f, geo_of(L), coef_of(c, L),
          c->partials);
  k_norm_final<<<1, kThreads, 0, c->s>>>(c->partials, kNormBlocks, c->norm_out);
  CCK(cudaGetLastError());
  return MG_OK;
}

mg_status read_norm(mg_cc_ctx *c, double *out) {
  CCK(cudaMemcpyAsync(out, c->norm_out, sizeof(double), cudaMemcpyDeviceToHost, c->s));
  CCK(cudaStreamSynchronize(c->s));
  return MG_OK;
}

// Algorithm 1 from level l down; coarse levels start from zero.
mg_status vcycle_rec(mg_cc_ctx *c, int l) {
  mg_status st;
  if (l == c->nl - 1) return op_coarse(c);
  if ((st = op_smooth(c, l, c->p.nu1))) return st;
  if ((st = op_residual(c, l))) return st;
  if ((st = op_restrict(c, l))) return st;
  Lev &C = c->lv[l + 1];
  CCK(cudaMemsetAsync(C.u[C.cur], 0, (size_t)C.count * sizeof(double), c->s));
  if ((st = vcycle_rec(c, l + 1))) return st;
  if ((st = op_prolong(c, l))) return st;
  return op_smooth(c, l, c->p.nu2);
}

mg_status level_ok(const mg_cc_ctx *c, int level, bool need_coarser) {
  if (!c) return ccfail(MG_EINVAL, "NULL context");
  if (level < 0 || level >= c->nl - (need_coarser ? 1 : 0))
    return ccfail(MG_EINVAL, "level %d out of range", level);
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_cc_default_params(mg_cc_params *p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->dim = 2;
  p->n = 2;
  p->c[0] = p->c[1] = p->c[2] = 1.0;
  p->sigma = 1.0;
  p->bc = MG_CC_NEUMANN;
  p->smoother = MG_RBGS;
  p->omega = 1.0;
  p->nu1 = 2;
  p->nu2 = 1;
  p->coarsest_n = 1;
  p->maxit = 50;
}

size_t mg_cc_workspace_bytes(const mg_cc_params *p) {
  if (check_params(p)) return 0;
  mg_cc_ctx tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.p = *p;
  return layout(&tmp, nullptr);
}

mg_status mg_cc_create(const mg_cc_params *p, void *arena, size_t arena_bytes, mg_cc_ctx **out) {
  if (!out) return ccfail(MG_EINVAL, "out is NULL");
  *out = nullptr;
  mg_status st = check_params(p);
  if (st) return st;
  if (!arena) return ccfail(MG_EINVAL, "arena is NULL");
  if ((uintptr_t)arena % 256) return ccfail(MG_EINVAL, "arena must be 256-byte aligned");
  mg_cc_ctx *c = (mg_cc_ctx *)calloc(1, sizeof(mg_cc_ctx));
  if (!c) return ccfail(MG_ENOMEM, "host allocation of the context failed");
  c->p = *p;
  c->s = (cudaStream_t)p->stream;
  size_t need = layout(c, nullptr);
  if (arena_bytes < need) {
    free(c);
    return ccfail(MG_ENOMEM, "arena has %zu bytes, %zu needed", arena_bytes, need);
  }
  layout(c, (char *)arena);
  cudaError_t e = cudaMemsetAsync(arena, 0, need, c->s);
  if (e == cudaSuccess) {
    Lev &Z = c->lv[c->nl - 1];
    if (p->dim == 2) k_dense_inverse<2><<<1, kThreads, 0, c->s>>>(c->ainv, geo_of(Z), coef_of(c, Z));
    else k_dense_inverse<3><<<1, kThreads, 0, c->s>>>(c->ainv, geo_of(Z), coef_of(c, Z));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) {
    free(c);
    return ccfail(MG_ECUDA, "creation: %s", cudaGetErrorString(e));
  }
  *out = c;
  return MG_OK;
}

mg_status mg_cc_destroy(mg_cc_ctx *c) {
  free(c);
  return MG_OK;
}

int mg_cc_num_levels(const mg_cc_ctx *c) { return c ? c->nl : -1; }

int mg_cc_level_size(const mg_cc_ctx *c, int level) {
  if (!c || level < 0 || level >= c->nl) return -1;
  return c->lv[level].n;
}

mg_status mg_cc_set_field(mg_cc_ctx *c, int level, int field, const double *src) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (!src) return ccfail(MG_EINVAL, "src is NULL");
  if (field < 0 || field > 2) return ccfail(MG_EINVAL, "field must be 0 (u), 1 (f) or 2 (r)");
  Lev &L = c->lv[level];
  double *dst = field == 0 ? L.u[L.cur] : (field == 1 ? L.f : L.r);
  const size_t rows = (size_t)L.n * (c->p.dim == 3 ? L.n : 1);
  CCK(cudaMemcpy2DAsync(dst, (size_t)L.pitch * 8, src, (size_t)L.n * 8, (size_t)L.n * 8, rows, cudaMemcpyDefault,
                        c->s));
  return MG_OK;
}

mg_status mg_cc_get_field(mg_cc_ctx *c, int level, int field, double *dst) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (!dst) return ccfail(MG_EINVAL, "dst is NULL");
  if (field < 0 || field > 2) return ccfail(MG_EINVAL, "field must be 0 (u), 1 (f) or 2 (r)");
  Lev &L = c->lv[level];
  const double *src = field == 0 ? L.u[L.cur] : (field == 1 ? L.f : L.r);
  const size_t rows = (size_t)L.n * (c->p.dim == 3 ? L.n : 1);
  CCK(cudaMemcpy2DAsync(dst, (size_t)L.n * 8, src, (size_t)L.pitch * 8, (size_t)L.n * 8, rows, cudaMemcpyDefault,
                        c->s));
  CCK(cudaStreamSynchronize(c->s));
  return MG_OK;
}

mg_status mg_cc_smooth(mg_cc_ctx *c, int level, int sweeps) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (sweeps < 0) return ccfail(MG_EINVAL, "sweeps must be >= 0");
  return op_smooth(c, level, sweeps);
}

mg_status mg_cc_residual(mg_cc_ctx *c, int level) {
  mg_status st = level_ok(c, level, false);
  return st ? st : op_residual(c, level);
}

mg_status mg_cc_restrict(mg_cc_ctx *c, int level) {
  mg_status st = level_ok(c, level, true);
  return st ? st : op_restrict(c, level);
}

mg_status mg_cc_prolongate(mg_cc_ctx *c, int level) {
  mg_status st = level_ok(c, level, true);
  return st ? st : op_prolong(c, level);
}

mg_status mg_cc_coarse_solve(mg_cc_ctx *c) {
  if (!c) return ccfail(MG_EINVAL, "NULL context");
  return op_coarse(c);
}

mg_status mg_cc_vcycle(mg_cc_ctx *c) {
  if (!c) return ccfail(MG_EINVAL, "NULL context");
  return vcycle_rec(c, 0);
}

mg_status mg_cc_residual_norm(mg_cc_ctx *c, int level, double *out) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (!out) return ccfail(MG_EINVAL, "out is NULL");
  if ((st = op_norm(c, level))) return st;
  return read_norm(c, out);
}

mg_status mg_cc_solve(mg_cc_ctx *c, double tol, int *iters, double *relres, double *history) {
  if (!c) return ccfail(MG_EINVAL, "NULL context");
  if (!(tol >= 0.0)) return ccfail(MG_EINVAL, "tol must be >= 0");
  mg_status st;
  double r0;
  if ((st = op_norm(c, 0)) || (st = read_norm(c, &r0))) return st;
  if (history) history[0] = 1.0;
  if (!isfinite(r0)) return ccfail(MG_ENOCONV, "initial residual is not finite");
  int k = 0;
  double rho = r0 > 0.0 ? 1.0 : 0.0;
  while (r0 > 0.0 && rho > tol && k < c->p.maxit) {
    if ((st = vcycle_rec(c, 0)) || (st = op_norm(c, 0))) return st;
    double rk;
    if ((st = read_norm(c, &rk))) return st;
    rho = rk / r0;
    k++;
    if (history) history[k] = rho;
    if (!isfinite(rho)) break;
  }
  if (iters) *iters = k;
  if (relres) *relres = rho;
  if (!isfinite(rho)) return ccfail(MG_ENOCONV, "residual is not finite after %d cycles", k);
  if (rho > tol) return ccfail(MG_ENOCONV, "relative residual %.3e above tol %.3e after %d cycles", rho, tol, k);
  return MG_OK;
}

}  // extern "C"
