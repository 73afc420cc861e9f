// Implicit Euler steps of nonlinear complex diffusion (include/mg_cd.h):
// Sec. 4's second test problem on cell-centred grids, complex FP64.
//
// Layout: level l has n_l = n / 2^l cells per dimension and seven complex
// fields (double2: real, imaginary) u[0], u[1] (Jacobi ping-pong), f, r, the
// face coefficients gx, gy and wd = omega / diag per cell, rows padded to 128
// bytes (pitch = n_l rounded up to 8 complex values), x fastest, no ghost
// cells. One thread per cell (per cell of the swept colour for red-black
// Gauss-Seidel), rows on blockIdx.y. The arithmetic is FP64 throughout and
// bound by FP64 issue, so the smoothers take omega / diag from wd (formed
// whenever the faces change) instead of summing faces and dividing per sweep.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "mg_cd.h"
#include "mg_internal.h"

namespace mg {
namespace cd {

constexpr int kMaxLev = 16;
constexpr int kThreads = 256;
constexpr int kNormBlocks = 4096;  // enough blocks to hide FP64 latency on every level

struct Geo {
  int n;
  long long sy;  // row stride (complex elements)
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// a / d = a conj(d) / |d|^2
__device__ __forceinline__ double2 cdiv(double2 a, double2 d) {
  const double q = 1.0 / (d.x * d.x + d.y * d.y);
  return make_double2((a.x * d.x + a.y * d.y) * q, (a.y * d.x - a.x * d.y) * q);
}

// (A u)_p = u_p + s sum_f g_f (u_p - u_q), s = tau / h^2; diag_p = 1 + s sum_f g_f.
__device__ __forceinline__ double2 apply(const double2 *__restrict__ u, const double2 *__restrict__ gx,
                                         const double2 *__restrict__ gy, long long p, int i, int j, const Geo &g,
                                         double s, double2 &diag) {
  const double2 u0 = u[p];
  double2 acc = make_double2(0.0, 0.0), gs = make_double2(0.0, 0.0);
  if (i > 0) {
    const double2 f = gx[p - 1];
    acc = cadd(acc, cmul(f, csub(u0, u[p - 1])));
    gs = cadd(gs, f);
  }
  if (i + 1 < g.n) {
    const double2 f = gx[p];
    acc = cadd(acc, cmul(f, csub(u0, u[p + 1])));
    gs = cadd(gs, f);
  }
  if (j > 0) {
    const double2 f = gy[p - g.sy];
    acc = cadd(acc, cmul(f, csub(u0, u[p - g.sy])));
    gs = cadd(gs, f);
  }
  if (j + 1 < g.n) {
    const double2 f = gy[p];
    acc = cadd(acc, cmul(f, csub(u0, u[p + g.sy])));
    gs = cadd(gs, f);
  }
  diag = make_double2(1.0 + s * gs.x, s * gs.y);
  return cadd(u0, cscale(s, acc));
}

// Cell diffusivity g(Im u) = e^{i theta} w, w = 1 / (1 + (Im u / (kappa theta))^2).
__device__ __forceinline__ double2 diffusivity(double2 u, double er, double ei, double inv_kt) {
  const double t = u.y * inv_kt;
  const double w = 1.0 / (1.0 + t * t);
  return make_double2(er * w, ei * w);
}

__global__ void k_faces(const double2 *__restrict__ u, double2 *__restrict__ gx, double2 *__restrict__ gy, Geo g,
                        double er, double ei, double inv_kt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= g.n) return;
  const long long p = (long long)j * g.sy + i;
  const double2 gp = diffusivity(u[p], er, ei, inv_kt);
  double2 fx = make_double2(0.0, 0.0), fy = make_double2(0.0, 0.0);
  if (i + 1 < g.n) fx = cscale(0.5, cadd(gp, diffusivity(u[p + 1], er, ei, inv_kt)));
  if (j + 1 < g.n) fy = cscale(0.5, cadd(gp, diffusivity(u[p + g.sy], er, ei, inv_kt)));
  gx[p] = fx;
  gy[p] = fy;
}

// Coarse x-face (I, J) | (I+1, J): mean of the fine faces at x index 2I+1,
// rows 2J and 2J+1; coarse y-face (I, J) | (I, J+1): mean of the fine faces
// at row 2J+1, columns 2I and 2I+1.
__global__ void k_coarsen_faces(const double2 *__restrict__ gxf, const double2 *__restrict__ gyf, Geo gf,
                                double2 *__restrict__ gxc, double2 *__restrict__ gyc, Geo gc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
  if (I >= gc.n) return;
  const long long P = (long long)J * gc.sy + I;
  double2 fx = make_double2(0.0, 0.0), fy = make_double2(0.0, 0.0);
  if (I + 1 < gc.n)
    fx = cscale(0.5, cadd(gxf[(long long)(2 * J) * gf.sy + 2 * I + 1], gxf[(long long)(2 * J + 1) * gf.sy + 2 * I + 1]));
  if (J + 1 < gc.n)
    fy = cscale(0.5, cadd(gyf[(long long)(2 * J + 1) * gf.sy + 2 * I], gyf[(long long)(2 * J + 1) * gf.sy + 2 * I + 1]));
  gxc[P] = fx;
  gyc[P] = fy;
}

// omega / diag_p of every cell (diag as in apply).
__global__ void k_wdiag(const double2 *__restrict__ gx, const double2 *__restrict__ gy, double2 *__restrict__ wd,
                        Geo g, double s, double omega) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= g.n) return;
  const long long p = (long long)j * g.sy + i;
  double2 gs = make_double2(0.0, 0.0);
  if (i > 0) gs = cadd(gs, gx[p - 1]);
  if (i + 1 < g.n) gs = cadd(gs, gx[p]);
  if (j > 0) gs = cadd(gs, gy[p - g.sy]);
  if (j + 1 < g.n) gs = cadd(gs, gy[p]);
  wd[p] = cdiv(make_double2(omega, 0.0), make_double2(1.0 + s * gs.x, s * gs.y));
}

__global__ void k_rbgs_half(double2 *__restrict__ u, const double2 *__restrict__ f, const double2 *__restrict__ gx,
                            const double2 *__restrict__ gy, const double2 *__restrict__ wd, Geo g, double s,
                            int color) {
  const int j = blockIdx.y;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((color + j) & 1);
  if (i >= g.n) return;
  const long long p = (long long)j * g.sy + i;
  double2 dg;
  const double2 Au = apply(u, gx, gy, p, i, j, g, s, dg);
  u[p] = cadd(u[p], cmul(wd[p], csub(f[p], Au)));
}

__global__ void k_jacobi(const double2 *__restrict__ uin, double2 *__restrict__ uout, const double2 *__restrict__ f,
                         const double2 *__restrict__ gx, const double2 *__restrict__ gy,
                         const double2 *__restrict__ wd, Geo g, double s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= g.n) return;
  const long long p = (long long)j * g.sy + i;
  double2 dg;
  const double2 Au = apply(uin, gx, gy, p, i, j, g, s, dg);
  uout[p] = cadd(uin[p], cmul(wd[p], csub(f[p], Au)));
}

__global__ void k_residual(const double2 *__restrict__ u, const double2 *__restrict__ f, double2 *__restrict__ r,
                           const double2 *__restrict__ gx, const double2 *__restrict__ gy, Geo g, double s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= g.n) return;
  const long long p = (long long)j * g.sy + i;
  double2 dg;
  r[p] = csub(f[p], apply(u, gx, gy, p, i, j, g, s, dg));
}

__global__ void k_restrict(const double2 *__restrict__ rf, Geo gf, double2 *__restrict__ fc, Geo gc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
  if (I >= gc.n) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < 2; b++) {
    const double2 *row = rf + (long long)(2 * J + b) * gf.sy + 2 * I;
    acc = cadd(acc, row[0]);
    acc = cadd(acc, row[1]);
  }
  fc[(long long)J * gc.sy + I] = cscale(0.25, acc);
}

__global__ void k_prolong(const double2 *__restrict__ ec, Geo gc, double2 *__restrict__ uf, Geo gf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= gf.n) return;
  const long long p = (long long)j * gf.sy + i;
  uf[p] = cadd(uf[p], ec[(long long)(j >> 1) * gc.sy + (i >> 1)]);
}

// The coarsest grid is one cell with no interior face: A u = u, so u = f.
__global__ void k_coarse_solve(double2 *__restrict__ u, const double2 *__restrict__ f) { u[0] = f[0]; }

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double buf[kThreads];
  buf[threadIdx.x] = v;
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) buf[threadIdx.x] += buf[threadIdx.x + st];
    __syncthreads();
  }
  return buf[0];
}

// Fixed-order norm: block b takes rows b, b + gridDim, ...; thread t cells
// t, t + 256, ... of a row; then a fixed-shape tree and a one-block final sum.
__global__ void k_norm_partials(const double2 *__restrict__ u, const double2 *__restrict__ f,
                                const double2 *__restrict__ gx, const double2 *__restrict__ gy, Geo g, double s,
                                double *__restrict__ partials) {
  double acc = 0.0;
  for (int j = blockIdx.x; j < g.n; j += gridDim.x)
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
      const long long p = (long long)j * g.sy + i;
      double2 dg;
      const double2 r = csub(f[p], apply(u, gx, gy, p, i, j, g, s, dg));
      acc += r.x * r.x + r.y * r.y;
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

struct Lev {
  int n, pitch;
  long long count;
  double2 *u[2], *f, *r, *gx, *gy, *wd;
  int cur;
};

}  // namespace cd
}  // namespace mg

using namespace mg::cd;

struct mg_cd_ctx {
  mg_cd_params p;
  int nl;
  Lev lv[kMaxLev];
  double *partials, *norm_out;
  cudaStream_t s;
};

namespace {

thread_local char g_cd_err[256];

mg_status cdfail(mg_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_cd_err, sizeof g_cd_err, fmt, ap);
  va_end(ap);
  mg::set_error_message(g_cd_err);
  return st;
}

#define CDK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return cdfail(MG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

mg_status check_params(const mg_cd_params *p) {
  if (!p) return cdfail(MG_EINVAL, "params are NULL");
  if (p->n < 1 || (p->n & (p->n - 1)) || p->n > 8192)
    return cdfail(MG_EINVAL, "n must be a power of two in 1..8192 (got %d)", p->n);
  if (!(p->tau > 0.0) || !isfinite(p->tau)) return cdfail(MG_EINVAL, "tau must be finite and > 0");
  if (!(p->theta != 0.0) || !isfinite(p->theta)) return cdfail(MG_EINVAL, "theta must be finite and nonzero");
  if (!(p->kappa > 0.0) || !isfinite(p->kappa)) return cdfail(MG_EINVAL, "kappa must be finite and > 0");
  if (p->smoother != MG_RBGS && p->smoother != MG_JACOBI) return cdfail(MG_EINVAL, "unknown smoother");
  if (!(p->omega > 0.0 && p->omega < 2.0)) return cdfail(MG_EINVAL, "omega must lie in (0, 2)");
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 > 8 || p->nu2 > 8 || p->nu1 + p->nu2 == 0)
    return cdfail(MG_EINVAL, "nu1, nu2 must lie in 0..8 with a positive sum");
  if (p->maxit < 0) return cdfail(MG_EINVAL, "maxit must be >= 0");
  return MG_OK;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

size_t layout(mg_cd_ctx *c, char *base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align256(off);
    void *q = base ? base + off : nullptr;
    off += bytes;
    return q;
  };
  c->nl = 0;
  for (int n = c->p.n; n >= 1; n /= 2) {
    Lev &L = c->lv[c->nl++];
    L.n = n;
    L.pitch = (n + 7) / 8 * 8;
    L.count = (long long)L.pitch * n;
    L.cur = 0;
    const size_t bytes = (size_t)L.count * sizeof(double2);
    L.u[0] = (double2 *)take(bytes);
    L.u[1] = (double2 *)take(bytes);
    L.f = (double2 *)take(bytes);
    L.r = (double2 *)take(bytes);
    L.gx = (double2 *)take(bytes);
    L.gy = (double2 *)take(bytes);
    L.wd = (double2 *)take(bytes);
    if (n == 1) break;
  }
  c->partials = (double *)take(kNormBlocks * sizeof(double));
  c->norm_out = (double *)take(sizeof(double));
  return align256(off);
}

Geo geo_of(const Lev &L) { return Geo{L.n, (long long)L.pitch}; }
double s_of(const mg_cd_ctx *c, const Lev &L) { return c->p.tau * (double)L.n * (double)L.n; }
dim3 grid_of(const Lev &L, int cells) { return dim3((unsigned)((cells + kThreads - 1) / kThreads), (unsigned)L.n); }

#define LAUNCH(kern, grid, ...)                               \
  do {                                                        \
    kern<<<grid, kThreads, 0, c->s>>>(__VA_ARGS__);           \
    CDK(cudaGetLastError());                                  \
  } while (0)

mg_status op_smooth(mg_cd_ctx *c, int l, int sweeps) {
  Lev &L = c->lv[l];
  const Geo g = geo_of(L);
  const double s = s_of(c, L);
  for (int it = 0; it < sweeps; it++) {
    if (c->p.smoother == MG_RBGS) {
      for (int color = 0; color < 2; color++)
        LAUNCH(k_rbgs_half, grid_of(L, (L.n + 1) / 2), L.u[L.cur], L.f, L.gx, L.gy, L.wd, g, s, color);
    } else {
      LAUNCH(k_jacobi, grid_of(L, L.n), L.u[L.cur], L.u[L.cur ^ 1], L.f, L.gx, L.gy, L.wd, g, s);
      L.cur ^= 1;
    }
  }
  return MG_OK;
}

mg_status op_residual(mg_cd_ctx *c, int l) {
  Lev &L = c->lv[l];
  LAUNCH(k_residual, grid_of(L, L.n), L.u[L.cur], L.f, L.r, L.gx, L.gy, geo_of(L), s_of(c, L));
  return MG_OK;
}

mg_status op_restrict(mg_cd_ctx *c, int l) {
  Lev &F = c->lv[l], &C = c->lv[l + 1];
  LAUNCH(k_restrict, grid_of(C, C.n), F.r, geo_of(F), C.f, geo_of(C));
  return MG_OK;
}

mg_status op_prolong(mg_cd_ctx *c, int l) {
  Lev &F = c->lv[l], &C = c->lv[l + 1];
  LAUNCH(k_prolong, grid_of(F, F.n), C.u[C.cur], geo_of(C), F.u[F.cur], geo_of(F));
  return MG_OK;
}

mg_status op_coarse(mg_cd_ctx *c) {
  Lev &L = c->lv[c->nl - 1];
  k_coarse_solve<<<1, 1, 0, c->s>>>(L.u[L.cur], L.f);
  CDK(cudaGetLastError());
  return MG_OK;
}

mg_status op_norm(mg_cd_ctx *c, int l) {
  Lev &L = c->lv[l];
  k_norm_partials<<<kNormBlocks, kThreads, 0, c->s>>>(L.u[L.cur], L.f, L.gx, L.gy, geo_of(L), s_of(c, L),
                                                       c->partials);
  CDK(cudaGetLastError());
  k_norm_final<<<1, kThreads, 0, c->s>>>(c->partials, kNormBlocks, c->norm_out);
  CDK(cudaGetLastError());
  return MG_OK;
}

mg_status read_norm(mg_cd_ctx *c, double *out) {
  CDK(cudaMemcpyAsync(out, c->norm_out, sizeof(double), cudaMemcpyDeviceToHost, c->s));
  CDK(cudaStreamSynchronize(c->s));
  return MG_OK;
}

mg_status vcycle_rec(mg_cd_ctx *c, int l) {
  mg_status st;
  if (l == c->nl - 1) return op_coarse(c);
  if ((st = op_smooth(c, l, c->p.nu1))) return st;
  if ((st = op_residual(c, l))) return st;
  if ((st = op_restrict(c, l))) return st;
  Lev &C = c->lv[l + 1];
  CDK(cudaMemsetAsync(C.u[C.cur], 0, (size_t)C.count * sizeof(double2), c->s));
  if ((st = vcycle_rec(c, l + 1))) return st;
  if ((st = op_prolong(c, l))) return st;
  return op_smooth(c, l, c->p.nu2);
}

mg_status level_ok(const mg_cd_ctx *c, int level, bool need_coarser) {
  if (!c) return cdfail(MG_EINVAL, "NULL context");
  if (level < 0 || level >= c->nl - (need_coarser ? 1 : 0)) return cdfail(MG_EINVAL, "level %d out of range", level);
  return MG_OK;
}

double2 *field_ptr(Lev &L, int field) {
  switch (field) {
    case MG_CD_U: return L.u[L.cur];
    case MG_CD_F: return L.f;
    case MG_CD_R: return L.r;
    case MG_CD_GX: return L.gx;
    case MG_CD_GY: return L.gy;
    default: return nullptr;
  }
}

mg_status op_wdiag(mg_cd_ctx *c, int l) {
  Lev &L = c->lv[l];
  LAUNCH(k_wdiag, grid_of(L, L.n), L.gx, L.gy, L.wd, geo_of(L), s_of(c, L), c->p.omega);
  return MG_OK;
}

mg_status copy_in(mg_cd_ctx *c, Lev &L, double2 *dst, const double *src) {
  CDK(cudaMemcpy2DAsync(dst, (size_t)L.pitch * 16, src, (size_t)L.n * 16, (size_t)L.n * 16, (size_t)L.n,
                        cudaMemcpyDefault, c->s));
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_cd_default_params(mg_cd_params *p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->n = 2;
  p->tau = 1e-3;
  p->theta = M_PI / 30.0;
  p->kappa = 0.1;
  p->smoother = MG_RBGS;
  p->omega = 1.0;
  p->nu1 = 2;
  p->nu2 = 2;
  p->maxit = 50;
}

size_t mg_cd_workspace_bytes(const mg_cd_params *p) {
  if (check_params(p)) return 0;
  mg_cd_ctx tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.p = *p;
  return layout(&tmp, nullptr);
}

mg_status mg_cd_create(const mg_cd_params *p, void *arena, size_t arena_bytes, mg_cd_ctx **out) {
  if (!out) return cdfail(MG_EINVAL, "out is NULL");
  *out = nullptr;
  mg_status st = check_params(p);
  if (st) return st;
  if (!arena) return cdfail(MG_EINVAL, "arena is NULL");
  if ((uintptr_t)arena % 256) return cdfail(MG_EINVAL, "arena must be 256-byte aligned");
  mg_cd_ctx *c = (mg_cd_ctx *)calloc(1, sizeof(mg_cd_ctx));
  if (!c) return cdfail(MG_ENOMEM, "host allocation of the context failed");
  c->p = *p;
  c->s = (cudaStream_t)p->stream;
  const size_t need = layout(c, nullptr);
  if (arena_bytes < need) {
    free(c);
    return cdfail(MG_ENOMEM, "arena has %zu bytes, %zu needed", arena_bytes, need);
  }
  layout(c, (char *)arena);
  cudaError_t e = cudaMemsetAsync(arena, 0, need, c->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) {
    free(c);
    return cdfail(MG_ECUDA, "creation: %s", cudaGetErrorString(e));
  }
  *out = c;
  return MG_OK;
}

mg_status mg_cd_destroy(mg_cd_ctx *c) {
  free(c);
  return MG_OK;
}

int mg_cd_num_levels(const mg_cd_ctx *c) { return c ? c->nl : -1; }

int mg_cd_level_size(const mg_cd_ctx *c, int level) {
  if (!c || level < 0 || level >= c->nl) return -1;
  return c->lv[level].n;
}

mg_status mg_cd_set_field(mg_cd_ctx *c, int level, int field, const double *src) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (!src) return cdfail(MG_EINVAL, "src is NULL");
  double2 *dst = field_ptr(c->lv[level], field);
  if (!dst) return cdfail(MG_EINVAL, "unknown field %d", field);
  if ((st = copy_in(c, c->lv[level], dst, src))) return st;
  return (field == MG_CD_GX || field == MG_CD_GY) ? op_wdiag(c, level) : MG_OK;
}

mg_status mg_cd_get_field(mg_cd_ctx *c, int level, int field, double *dst) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (!dst) return cdfail(MG_EINVAL, "dst is NULL");
  Lev &L = c->lv[level];
  const double2 *src = field_ptr(L, field);
  if (!src) return cdfail(MG_EINVAL, "unknown field %d", field);
  CDK(cudaMemcpy2DAsync(dst, (size_t)L.n * 16, src, (size_t)L.pitch * 16, (size_t)L.n * 16, (size_t)L.n,
                        cudaMemcpyDefault, c->s));
  CDK(cudaStreamSynchronize(c->s));
  return MG_OK;
}

mg_status mg_cd_begin_step(mg_cd_ctx *c, const double *un) {
  if (!c || !un) return cdfail(MG_EINVAL, "NULL argument");
  mg_status st;
  Lev &L = c->lv[0];
  L.cur = 0;
  if ((st = copy_in(c, L, L.f, un))) return st;
  CDK(cudaMemcpyAsync(L.u[0], L.f, (size_t)L.count * sizeof(double2), cudaMemcpyDeviceToDevice, c->s));
  LAUNCH(k_faces, grid_of(L, L.n), L.f, L.gx, L.gy, geo_of(L), cos(c->p.theta), sin(c->p.theta),
         1.0 / (c->p.kappa * c->p.theta));
  for (int l = 1; l < c->nl; l++) {
    Lev &F = c->lv[l - 1], &C = c->lv[l];
    LAUNCH(k_coarsen_faces, grid_of(C, C.n), F.gx, F.gy, geo_of(F), C.gx, C.gy, geo_of(C));
  }
  for (int l = 0; l < c->nl; l++)
    if ((st = op_wdiag(c, l))) return st;
  return MG_OK;
}

mg_status mg_cd_smooth(mg_cd_ctx *c, int level, int sweeps) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (sweeps < 0) return cdfail(MG_EINVAL, "sweeps must be >= 0");
  return op_smooth(c, level, sweeps);
}

mg_status mg_cd_residual(mg_cd_ctx *c, int level) {
  mg_status st = level_ok(c, level, false);
  return st ? st : op_residual(c, level);
}

mg_status mg_cd_restrict(mg_cd_ctx *c, int level) {
  mg_status st = level_ok(c, level, true);
  return st ? st : op_restrict(c, level);
}

mg_status mg_cd_prolongate(mg_cd_ctx *c, int level) {
  mg_status st = level_ok(c, level, true);
  return st ? st : op_prolong(c, level);
}

mg_status mg_cd_coarse_solve(mg_cd_ctx *c) {
  if (!c) return cdfail(MG_EINVAL, "NULL context");
  return op_coarse(c);
}

mg_status mg_cd_vcycle(mg_cd_ctx *c) {
  if (!c) return cdfail(MG_EINVAL, "NULL context");
  return vcycle_rec(c, 0);
}

mg_status mg_cd_residual_norm(mg_cd_ctx *c, int level, double *out) {
  mg_status st = level_ok(c, level, false);
  if (st) return st;
  if (!out) return cdfail(MG_EINVAL, "out is NULL");
  if ((st = op_norm(c, level))) return st;
  return read_norm(c, out);
}

mg_status mg_cd_solve(mg_cd_ctx *c, double tol, int *iters, double *relres, double *history) {
  if (!c) return cdfail(MG_EINVAL, "NULL context");
  if (!(tol >= 0.0)) return cdfail(MG_EINVAL, "tol must be >= 0");
  mg_status st;
  double r0;
  if ((st = op_norm(c, 0)) || (st = read_norm(c, &r0))) return st;
  if (history) history[0] = 1.0;
  if (!isfinite(r0)) return cdfail(MG_ENOCONV, "initial residual is not finite");
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
  if (!isfinite(rho)) return cdfail(MG_ENOCONV, "residual is not finite after %d cycles", k);
  if (rho > tol) return cdfail(MG_ENOCONV, "relative residual %.3e above tol %.3e after %d cycles", rho, tol, k);
  return MG_OK;
}

mg_status mg_cd_time_step(mg_cd_ctx *c, const double *un, double tol, int *iters, double *relres, double *history) {
  mg_status st = mg_cd_begin_step(c, un);
  if (st) return st;
  return mg_cd_solve(c, tol, iters, relres, history);
}

}  // extern "C"
