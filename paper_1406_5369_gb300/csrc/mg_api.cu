// C ABI of libmg.so (declared in include/mg.h): context, arena layout,
// V-cycle orchestration (Algorithm 1), solve loop (Layer-4 Application),
// defect correction and CUDA-graph replay.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mg.h"
#include "mg_internal.h"

using mg::Level;

namespace {

thread_local char g_err[512] = "";

mg_status fail(mg_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(MG_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                  \
  } while (0)

// Launches one kernel through a dispatcher and counts it. With timing on,
// CUDA events bracket the launch (kernel class `kind`, grid level `lvl`).
#define TLAUNCH(c, kind, lvl, s, call)                                                        \
  do {                                                                                        \
    int ev_ = timing_begin((c), (kind), (lvl), (s));                                          \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(MG_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                   \
    (c)->launches++;                                                                          \
    timing_end((c), ev_, (s));                                                                \
  } while (0)
#define LAUNCH(c, call) TLAUNCH(c, MG_KERNEL_OTHER, 0, s, call)


// Dimension dispatch of the level kernels.
#define DISPATCH(L, fn, ...) ((L).dim == 2 ? mg::d2::fn(__VA_ARGS__) : mg::d3::fn(__VA_ARGS__))

}  // namespace

#include "ctx.h"

namespace {

int alloc_pair(mg_ctx *c) {
  if (c->nfree > 0) return c->free_pairs[--c->nfree];
  if (c->npairs >= kMaxPairs) return -1;
  TimingPair &p = c->pairs[c->npairs];
  if (cudaEventCreate(&p.a) != cudaSuccess) return -1;
  if (cudaEventCreate(&p.b) != cudaSuccess) {
    cudaEventDestroy(p.a);
    return -1;
  }
  return c->npairs++;
}

// Records the start event of a timed launch; returns the pair or -1.
int timing_begin(mg_ctx *c, int kind, int level, cudaStream_t s) {
  if (!c->timing || (c->timing >= 2 && level != 0) || (c->timing == 3 && kind != MG_KERNEL_OUTER)) return -1;
  int slot = c->capturing_slot;
  if (slot >= 0 && c->graphs[slot].npairs >= kSlotPairs) return -1;
  int i = alloc_pair(c);
  if (i < 0) return -1;
  TimingPair &p = c->pairs[i];
  p.kind = kind;
  p.level = level;
  p.owner = slot;
  p.pending = false;
  if (slot >= 0) {
    cudaEventRecordWithFlags(p.a, s, cudaEventRecordExternal);
    c->graphs[slot].pairs[c->graphs[slot].npairs++] = i;
  } else {
    cudaEventRecord(p.a, s);
  }
  return i;
}

void timing_end(mg_ctx *c, int i, cudaStream_t s) {
  if (i < 0) return;
  TimingPair &p = c->pairs[i];
  if (p.owner >= 0) {
    cudaEventRecordWithFlags(p.b, s, cudaEventRecordExternal);
  } else {
    cudaEventRecord(p.b, s);
    p.pending = true;
  }
}

// Adds the durations of every recorded pair (the stream has been synchronised).
void timing_harvest(mg_ctx *c) {
  for (int i = 0; i < c->npairs; i++) {
    TimingPair &p = c->pairs[i];
    if (!p.pending) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess && p.kind >= 0 && p.kind < kKinds &&
        p.level >= 0 && p.level < kMaxLevels) {
      c->t_ms[p.kind][p.level] += ms;
      c->t_n[p.kind][p.level] += 1;
    }
    p.pending = false;
    if (p.owner < 0) c->free_pairs[c->nfree++] = i;
  }
  cudaGetLastError();  // a pair whose events never completed is simply skipped
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Hands out 256-byte aligned slices of the arena. With a guard context
// (options.canary) each slice is followed by kGuardBytes bytes whose offset
// and owner are recorded there when laying out for real (base != NULL).
struct Bump {
  char *base;
  size_t off;
  mg_ctx *guards;
  void *take(size_t bytes, const char *tag = "buffer", int level = -1) {
    off = align_up(off, 256);
    void *p = base ? base + off : nullptr;
    off += bytes;
    if (guards) {
      if (base && guards->nguards < kMaxGuards) {
        int g = guards->nguards++;
        guards->guard_off[g] = off;
        if (level >= 0) snprintf(guards->guard_tag[g], sizeof guards->guard_tag[g], "l%d.%s", level, tag);
        else snprintf(guards->guard_tag[g], sizeof guards->guard_tag[g], "%s", tag);
      }
      off += kGuardBytes;
    }
    return p;
  }
};

bool valid_n(int n, int *m_out) {
  if (n < 3) return false;
  int m = 0;
  while ((1 << (m + 1)) + 1 <= n) m++;
  if ((1 << m) + 1 != n) return false;
  if (m_out) *m_out = m;
  return true;
}

mg_status check_args(int dim, int n, const mg_options *opt) {
  if (dim != 2 && dim != 3) return fail(MG_EINVAL, "dim must be 2 or 3 (got %d)", dim);
  int m;
  if (!valid_n(n, &m)) return fail(MG_EINVAL, "n must be 2^m+1 with m >= 1 (got %d)", n);
  if (dim == 3 && n > 2049) return fail(MG_EINVAL, "3D grids are limited to n <= 2049");
  if (!opt) return fail(MG_EINVAL, "options are NULL");
  if (opt->smoother != MG_RBGS && opt->smoother != MG_JACOBI) return fail(MG_EINVAL, "unknown smoother");
  if (!(opt->omega > 0.0 && opt->omega < 2.0)) return fail(MG_EINVAL, "omega must lie in (0, 2)");
  if (opt->nu1 < 0 || opt->nu2 < 0 || opt->nu1 > 8 || opt->nu2 > 8) return fail(MG_EINVAL, "nu1, nu2 must lie in 0..8");
  if (opt->nu1 + opt->nu2 == 0) return fail(MG_EINVAL, "nu1 + nu2 must be positive");
  if (opt->coarsest_n != 3 && opt->coarsest_n != 5 && opt->coarsest_n != 9)
    return fail(MG_EINVAL, "coarsest_n must be 3, 5 or 9 (got %d)", opt->coarsest_n);
  if (n < opt->coarsest_n) return fail(MG_EINVAL, "n (%d) is below coarsest_n (%d)", n, opt->coarsest_n);
  if (opt->maxit < 0) return fail(MG_EINVAL, "maxit must be >= 0");
  if (opt->inner_cycles < 0 || opt->inner_cycles > 8) return fail(MG_EINVAL, "inner_cycles must lie in 0..8 (0 = 1)");
  if (opt->precision != MG_FP64 && opt->precision != MG_FP32_DC && opt->precision != MG_BF16_DC)
    return fail(MG_EINVAL, "unknown precision");
  if (opt->exact_outer != 0 && opt->exact_outer != 1) return fail(MG_EINVAL, "exact_outer must be 0 or 1");
  if (opt->tile_rows < 0 || opt->tile_rows > (1 << 20)) return fail(MG_EINVAL, "tile_rows must lie in 0..2^20");
  if (opt->tile_max_n < 0) return fail(MG_EINVAL, "tile_max_n must be >= 0");
  if (opt->fuse_depth < 0 || opt->fuse_depth > 8) return fail(MG_EINVAL, "fuse_depth must lie in 0..8");
  if (opt->join_cycles != 0 && opt->join_cycles != 1) return fail(MG_EINVAL, "join_cycles must be 0 or 1");
  if (opt->canary != 0 && opt->canary != 1) return fail(MG_EINVAL, "canary must be 0 or 1");
  return MG_OK;
}

// Levels n, (n-1)/2+1, ..., nc (both of the form 2^m+1, nc <= n).
int level_count(int n, int nc) {
  int L = 0;
  for (int nn = n; nn >= nc; nn = (nn - 1) / 2 + 1) {
    L++;
    if (nn == nc) break;
  }
  return L;
}

void init_level(Level &L, int dim, int n, int dtype, const double c[3]) {
  memset(&L, 0, sizeof L);
  L.dim = dim;
  L.n = n;
  L.dtype = dtype;
  int per128 = 128 / mg::dtype_size(dtype);
  L.pitch = (int)align_up((size_t)n, (size_t)per128);
  L.plane = (long long)L.pitch * n;
  L.count = L.plane * (dim == 3 ? n : 1);
  for (int d = 0; d < 3; d++) L.c[d] = c[d];
  double h = 1.0 / (double)(n - 1);
  L.inv_h2 = 1.0 / (h * h);
}

void take_level(Level &L, Bump &b, bool variable, int l) {
  static const char *face[3] = {"kx", "ky", "kz"};
  size_t bytes = (size_t)L.count * mg::dtype_size(L.dtype);
  L.u[0] = b.take(bytes, "u0", l);
  L.u[1] = b.take(bytes, "u1", l);
  L.f = b.take(bytes, "f", l);
  L.r = b.take(bytes, "r", l);
  if (variable) {
    size_t fb = (size_t)L.count * mg::face_size(L.dtype);
    for (int d = 0; d < L.dim; d++) L.kf[d] = b.take(fb, face[d], l);
  }
}

// Lays out every buffer of the context in the arena (base == NULL: sizing).
size_t layout(mg_ctx *c, char *base) {
  Bump b{base, 0, c->opt.canary ? c : nullptr};
  c->nguards = 0;
  int inner = c->opt.precision == MG_FP32_DC ? mg::F32 : (c->opt.precision == MG_BF16_DC ? mg::BF16 : mg::F64);
  double cc[3] = {c->lv[0].c[0], c->lv[0].c[1], c->lv[0].c[2]};
  int nn = c->n;
  for (int l = 0; l < c->nl; l++) {
    int dt = (l == c->nl - 1) ? mg::F64 : inner;
    init_level(c->lv[l], c->dim, nn, dt, cc);
    take_level(c->lv[l], b, c->variable, l);
    nn = (nn - 1) / 2 + 1;
  }
  {
    Level &Z = c->lv[c->nl - 1];
    if (Z.n > 3) {
      size_t m = (size_t)Z.n - 2, N = c->dim == 3 ? m * m * m : m * m;
      Z.dense = (double *)b.take(N * N * sizeof(double), "dense");
    }
  }
  if (c->dc) {
    init_level(c->outer, c->dim, c->n, mg::F64, cc);
    size_t bytes = (size_t)c->outer.count * 8;
    c->outer.u[0] = b.take(bytes, "outer.u0");
    c->outer.u[1] = b.take(bytes, "outer.u1");
    c->outer.f = b.take(bytes, "outer.f");
    c->outer.r = b.take(bytes, "outer.r");
    if (c->variable)
      for (int d = 0; d < c->dim; d++) c->outer.kf[d] = b.take(bytes, d == 0 ? "outer.kx" : d == 1 ? "outer.ky" : "outer.kz");
  }
  c->partials = (double *)b.take(sizeof(double) * mg::kMaxPartials, "partials");
  c->norm_out = (double *)b.take(sizeof(double) * 4, "norm_out");
  c->dc_scale = (float *)b.take(sizeof(float) * 4, "dc_scale");
  return align_up(b.off, 256);
}

// The FP64 level whose u/f the user's finest-level calls address.
Level &user_level(mg_ctx *c) { return c->dc ? c->outer : c->lv[0]; }
void *user_u(mg_ctx *c) { return c->dc ? c->outer.u[c->outer.cur] : c->lv[0].u[c->lv[0].cur]; }

double interior_count(const Level &L) {
  double m = (double)(L.n - 2);
  return L.dim == 3 ? m * m * m : m * m;
}

// Dense n^dim FP64 (host or device) <-> pitched FP64 field, whole array.
cudaError_t copy_dense_to_pitched(const Level &L, const double *src, void *dst, cudaStream_t s) {
  size_t rows = (size_t)L.n * (L.dim == 3 ? L.n : 1);
  return cudaMemcpy2DAsync(dst, (size_t)L.pitch * 8, src, (size_t)L.n * 8, (size_t)L.n * 8, rows,
                           cudaMemcpyDefault, s);
}
cudaError_t copy_pitched_to_dense(const Level &L, const void *src, double *dst, cudaStream_t s) {
  size_t rows = (size_t)L.n * (L.dim == 3 ? L.n : 1);
  return cudaMemcpy2DAsync(dst, (size_t)L.n * 8, src, (size_t)L.pitch * 8, (size_t)L.n * 8, rows,
                           cudaMemcpyDefault, s);
}
// Interior box only (boundary of dst untouched).
cudaError_t copy_dense_interior(const Level &L, const double *src, void *dst, cudaStream_t s) {
  size_t n = (size_t)L.n, m = n - 2;
  if (L.dim == 2) {
    return cudaMemcpy2DAsync((char *)dst + ((size_t)L.pitch + 1) * 8, (size_t)L.pitch * 8, src + n + 1, n * 8,
                             m * 8, m, cudaMemcpyDefault, s);
  }
  cudaMemcpy3DParms p;
  memset(&p, 0, sizeof p);
  p.srcPtr = make_cudaPitchedPtr((void *)src, n * 8, n, n);
  p.srcPos = make_cudaPos(8, 1, 1);
  p.dstPtr = make_cudaPitchedPtr(dst, (size_t)L.pitch * 8, n, n);
  p.dstPos = make_cudaPos(8, 1, 1);
  p.extent = make_cudaExtent(m * 8, m, m);
  p.kind = cudaMemcpyDefault;
  return cudaMemcpy3DAsync(&p, s);
}


// ---------------------------------------------------------------- level ops

mg_status op_smooth(mg_ctx *c, int l, int sweeps, cudaStream_t s, int kind = MG_KERNEL_OTHER) {
  Level &L = c->lv[l];
  for (int k = 0; k < sweeps; k++) {
    if (c->opt.smoother == MG_RBGS) {
      TLAUNCH(c, kind, l, s, DISPATCH(L, rbgs_half, L, L.u[L.cur], L.f, 0, c->opt.omega, s));
      TLAUNCH(c, kind, l, s, DISPATCH(L, rbgs_half, L, L.u[L.cur], L.f, 1, c->opt.omega, s));
    } else {
      TLAUNCH(c, kind, l, s, DISPATCH(L, jacobi, L, L.u[L.cur], L.u[L.cur ^ 1], L.f, c->opt.omega, s));
      L.cur ^= 1;
    }
  }
  return MG_OK;
}

mg_status op_residual(mg_ctx *c, int l, cudaStream_t s, int kind = MG_KERNEL_OTHER) {
  Level &L = c->lv[l];
  TLAUNCH(c, kind, l, s, DISPATCH(L, residual, L, L.u[L.cur], L.f, L.r, s));
  return MG_OK;
}

mg_status op_restrict(mg_ctx *c, int l, cudaStream_t s, int kind = MG_KERNEL_OTHER) {
  Level &F = c->lv[l], &C = c->lv[l + 1];
  TLAUNCH(c, kind, l, s, DISPATCH(F, restrict_fw, F, F.r, C, C.f, s));
  return MG_OK;
}

mg_status op_prolong(mg_ctx *c, int l, cudaStream_t s, int kind = MG_KERNEL_OTHER) {
  Level &F = c->lv[l], &C = c->lv[l + 1];
  TLAUNCH(c, kind, l, s, DISPATCH(F, prolong, C, C.u[C.cur], F, F.u[F.cur], s));
  return MG_OK;
}

mg_status op_coarse(mg_ctx *c, cudaStream_t s, int kind = MG_KERNEL_OTHER) {
  Level &L = c->lv[c->nl - 1];
  if (L.dense) TLAUNCH(c, kind, c->nl - 1, s, DISPATCH(L, coarse_dense, L, L.u[L.cur], L.f, s));
  else TLAUNCH(c, kind, c->nl - 1, s, DISPATCH(L, coarse3, L, L.u[L.cur], L.f, s));
  return MG_OK;
}

mg_status op_zero_u(mg_ctx *c, int l, cudaStream_t s) {
  Level &L = c->lv[l];
  CK(cudaMemsetAsync(L.u[L.cur], 0, (size_t)L.count * mg::dtype_size(L.dtype), s));
  return MG_OK;
}

// True when level l's pre- and post-smoothing run as fused 2D kernels.
// Sweeps a fused 2D pass takes of nu (fuse_depth; 0 = all of them).
int fused_sweeps(const mg_ctx *c, int nu) {
  return c->opt.fuse_depth > 0 && c->opt.fuse_depth < nu ? c->opt.fuse_depth : nu;
}

bool level_fused(mg_ctx *c, int l) {
  if (!c->opt.fuse || c->opt.smoother != MG_RBGS || l + 1 >= c->nl) return false;
  return mg::d2::fused_ok(c->lv[l], c->lv[l + 1], fused_sweeps(c, c->opt.nu1)) &&
         mg::d2::fused_ok(c->lv[l], c->lv[l + 1], fused_sweeps(c, c->opt.nu2));
}

// Algorithm 1 from level l down: presmooth, residual, restrict, zero the
// coarse solution, recurse, interpolate and correct, postsmooth. `zero`
// says that u_l is zero on entry (every coarse level, and the finest level
// of a defect-correction step), which lets the fused kernels skip reading it.
mg_status vcycle_rec(mg_ctx *c, int l, bool zero, cudaStream_t s) {
  NvtxRange range(c->level_name[l]);
  mg_status st;
  if (c->opt.fuse && c->dim == 2 && c->lv[l].n > mg::coarse_top_n(c->dim, !c->dc) &&
      mg::cluster_ok(c->lv, l, c->nl, (int)c->opt.smoother, !c->dc, c->opt.cluster_max_n)) {
    TLAUNCH(c, MG_KERNEL_COARSE, l, s,
            mg::cluster_cycle(c->lv, l, c->nl, zero, c->opt.omega, c->opt.nu1, c->opt.nu2, s));
    return MG_OK;
  }
  if (c->opt.fuse && c->lv[l].n <= mg::coarse_top_n(c->dim, !c->dc)) {
    TLAUNCH(c, MG_KERNEL_COARSE, l, s,
            mg::coarse_cycle(c->lv, l, c->nl, zero, c->opt.smoother, c->opt.omega, c->opt.nu1, c->opt.nu2, !c->dc, s));
    return MG_OK;
  }
  if (l == c->nl - 1) {
    if (zero && (st = op_zero_u(c, l, s))) return st;
    return op_coarse(c, s, MG_KERNEL_COARSE);
  }
  Level &L = c->lv[l], &C = c->lv[l + 1];
  if (level_fused(c, l)) {
      // fuse_depth d < nu: nu - d separate sweeps before the fused pre-smoothing
    // pass and after the fused post-smoothing pass
    const int d1 = fused_sweeps(c, c->opt.nu1), d2 = fused_sweeps(c, c->opt.nu2);
    if (d1 < c->opt.nu1) {
      if (zero && (st = op_zero_u(c, l, s))) return st;
      if ((st = op_smooth(c, l, c->opt.nu1 - d1, s, MG_KERNEL_PRESMOOTH))) return st;
      zero = false;
    }
    TLAUNCH(c, MG_KERNEL_PRESMOOTH, l, s,
            mg::d2::pre_fused(L, L.u[L.cur], L.u[L.cur ^ 1], C, C.f, zero, d1, c->opt.omega, c->opt.tile_rows,
                              c->opt.tile_max_n, s));
    L.cur ^= 1;
    if ((st = vcycle_rec(c, l + 1, true, s))) return st;
    TLAUNCH(c, MG_KERNEL_POSTSMOOTH, l, s,
            mg::d2::post_fused(L, L.u[L.cur], L.u[L.cur ^ 1], C, C.u[C.cur], d2, c->opt.omega, c->opt.tile_rows,
                               c->opt.tile_max_n, s));
    L.cur ^= 1;
    if (d2 < c->opt.nu2) return op_smooth(c, l, c->opt.nu2 - d2, s, MG_KERNEL_POSTSMOOTH);
    return MG_OK;
  }
  if (zero && c->opt.fuse && c->opt.smoother == MG_JACOBI && c->opt.nu1 >= 2 && c->dim == 3 && mg::d3::z_ok(L)) {
    // the first two sweeps from zero in one pass that reads f only (no zeroing pass)
    TLAUNCH(c, MG_KERNEL_PRESMOOTH, l, s, mg::d3::z_jacobi_zero2(L, L.f, L.u[L.cur ^ 1], c->opt.omega, s));
    L.cur ^= 1;
    if ((st = op_smooth(c, l, c->opt.nu1 - 2, s, MG_KERNEL_PRESMOOTH))) return st;
  } else {
    if (zero && (st = op_zero_u(c, l, s))) return st;
    if ((st = op_smooth(c, l, c->opt.nu1, s, MG_KERNEL_PRESMOOTH))) return st;
  }
  if ((st = op_residual(c, l, s, MG_KERNEL_PRESMOOTH))) return st;
  if ((st = op_restrict(c, l, s, MG_KERNEL_PRESMOOTH))) return st;
  if ((st = vcycle_rec(c, l + 1, true, s))) return st;
  if ((st = op_prolong(c, l, s, MG_KERNEL_POSTSMOOTH))) return st;
  return op_smooth(c, l, c->opt.nu2, s, MG_KERNEL_POSTSMOOTH);
}

// Streaming finest-level kernels of either dimension (constant stencil).
bool outer_fast(const Level &O, const Level &I) {
  return O.dim == 2 ? mg::d2::outer_ok(O, I) : mg::d3::outer_ok(O, I);
}
cudaError_t outer_step(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d,
                       double *partials, int *nparts, const float *scale, bool update, bool acc64, bool exact,
                       cudaStream_t s) {
  return O.dim == 2 ? mg::d2::dc_step(O, uin, uout, I, e, d, partials, nparts, scale, update, acc64, exact, s)
                    : mg::d3::dc_step(O, uin, uout, I, e, d, partials, nparts, scale, update, acc64, exact, s);
}
bool norm_fast(const Level &L) { return L.dim == 2 ? mg::d2::norm_ok(L) : mg::d3::norm_ok(L); }
cudaError_t norm_fast_partials(const Level &L, const void *u, const void *f, double *partials, int *nparts,
                               cudaStream_t s) {
  return L.dim == 2 ? mg::d2::norm_stream(L, u, f, partials, nparts, s) : mg::d3::norm_stream(L, u, f, partials, nparts, s);
}

// Residual norm of level l into norm_out[0]. In defect-correction contexts
// level 0 is the outer FP64 problem; that pass also leaves the defect in the
// inner level 0's right-hand side and resets the norm scale.
mg_status op_norm(mg_ctx *c, int l, cudaStream_t s) {
  int np = 0;
  if (c->dc && l == 0) {
    Level &O = c->outer, &I = c->lv[0];
    if (outer_fast(O, I)) {
      TLAUNCH(c, MG_KERNEL_OUTER, 0, s, outer_step(O, (const double *)O.u[O.cur], nullptr, I, nullptr, I.f,
                                                        c->partials, &np, c->dc_scale, false, true, false, s));
      TLAUNCH(c, MG_KERNEL_NORM, 0, s,
              mg::norm_finalize_ex(c->partials, np, c->norm_out, nullptr, c->dc_scale, interior_count(O), s));
      return MG_OK;
    }
    TLAUNCH(c, MG_KERNEL_OUTER, 0, s, DISPATCH(O, dc_residual, O, O.u[O.cur], O.f, I, I.f, c->partials, mg::kNormBlocks, s));
  } else {
    Level &L = c->lv[l];
    if (norm_fast(L)) {
      TLAUNCH(c, MG_KERNEL_NORM, l, s, norm_fast_partials(L, L.u[L.cur], L.f, c->partials, &np, s));
      TLAUNCH(c, MG_KERNEL_NORM, l, s,
              mg::norm_finalize_ex(c->partials, np, c->norm_out, nullptr, nullptr, interior_count(L), s));
      return MG_OK;
    }
    TLAUNCH(c, MG_KERNEL_NORM, l, s, DISPATCH(L, norm_partials, L, L.u[L.cur], L.f, c->partials, mg::kNormBlocks, s));
  }
  TLAUNCH(c, MG_KERNEL_NORM, l, s, mg::norm_finalize(c->partials, mg::kNormBlocks, c->norm_out, s));
  return MG_OK;
}

// op_norm(c, 0) when the finest interior u is zero and the Dirichlet data
// are homogeneous: the residual is f itself (same norm, same defect).
mg_status op_first_norm(mg_ctx *c, cudaStream_t s) {
  Level &O = c->dc ? c->outer : c->lv[0];
  TLAUNCH(c, MG_KERNEL_NORM, 0, s, mg::first_defect(O, c->dc ? &c->lv[0] : nullptr, c->partials, s));
  TLAUNCH(c, MG_KERNEL_NORM, 0, s,
          mg::norm_finalize_ex(c->partials, mg::kNormBlocks, c->norm_out, nullptr, c->dc ? c->dc_scale : nullptr,
                               interior_count(O), s));
  return MG_OK;
}

// One defect-correction step with the defect d already in lv[0].f:
// e = V(0, d), then inner_cycles - 1 further cycles e = V(e, d); u += e. With `norm`, the residual of the updated u is
// computed in the same pass (new defect in lv[0].f, norm in norm_out).
// True when level 0 of the inner hierarchy joins the post-smoothing pass of
// one inner cycle with the pre-smoothing pass of the next (join_cycles).
bool can_join(mg_ctx *c) {
  if (!c->opt.join_cycles || c->nl < 2 || !level_fused(c, 0)) return false;
  if (fused_sweeps(c, c->opt.nu1) != c->opt.nu1 || fused_sweeps(c, c->opt.nu2) != c->opt.nu2) return false;
  if (c->lv[0].n <= mg::coarse_top_n(c->dim, !c->dc)) return false;
  return mg::d2::postpre_ok(c->lv[0], c->lv[1], c->opt.nu2, c->opt.nu1, c->opt.tile_max_n);
}

mg_status dc_inner_and_update(mg_ctx *c, bool norm, cudaStream_t s) {
  mg_status st;
  const int inner = c->opt.inner_cycles > 1 ? c->opt.inner_cycles : 1;
  if (inner > 1 && can_join(c)) {
    // level 0: pre-smoothing from zero, then between consecutive cycles one
    // pass of post-smoothing + the next pre-smoothing, post-smoothing last;
    // levels 1.. as in vcycle_rec
    Level &L = c->lv[0], &C = c->lv[1];
    const double om = c->opt.omega;
    TLAUNCH(c, MG_KERNEL_PRESMOOTH, 0, s,
            mg::d2::pre_fused(L, L.u[L.cur], L.u[L.cur ^ 1], C, C.f, true, c->opt.nu1, om, c->opt.tile_rows,
                              c->opt.tile_max_n, s));
    L.cur ^= 1;
    if ((st = vcycle_rec(c, 1, true, s))) return st;
    for (int k = 1; k < inner; k++) {
      TLAUNCH(c, MG_KERNEL_POSTPRE, 0, s,
              mg::d2::postpre_fused(L, L.u[L.cur], L.u[L.cur ^ 1], C, C.u[C.cur], C.f, c->opt.nu2, c->opt.nu1, om,
                                    c->opt.tile_rows, c->opt.tile_max_n, s));
      L.cur ^= 1;
      if ((st = vcycle_rec(c, 1, true, s))) return st;
    }
    TLAUNCH(c, MG_KERNEL_POSTSMOOTH, 0, s,
            mg::d2::post_fused(L, L.u[L.cur], L.u[L.cur ^ 1], C, C.u[C.cur], c->opt.nu2, om, c->opt.tile_rows,
                               c->opt.tile_max_n, s));
    L.cur ^= 1;
  } else {
    if ((st = vcycle_rec(c, 0, true, s))) return st;
    for (int k = 1; k < inner; k++)
      if ((st = vcycle_rec(c, 0, false, s))) return st;
  }
  Level &O = c->outer, &I = c->lv[0];
  if (outer_fast(O, I)) {
    int np = 0;
    TLAUNCH(c, MG_KERNEL_OUTER, 0, s,
            outer_step(O, (const double *)O.u[O.cur], (double *)O.u[O.cur ^ 1], I, I.u[I.cur],
                            norm ? I.f : nullptr, c->partials, &np, c->dc_scale, true, false,
                            c->opt.exact_outer != 0, s));
    O.cur ^= 1;
    if (norm)
      TLAUNCH(c, MG_KERNEL_NORM, 0, s,
              mg::norm_finalize_ex(c->partials, np, c->norm_out, c->dc_scale, c->dc_scale, interior_count(O), s));
    return MG_OK;
  }
  TLAUNCH(c, MG_KERNEL_OUTER, 0, s, DISPATCH(O, dc_update, O, O.u[O.cur], I, I.u[I.cur], s));
  if (norm) return op_norm(c, 0, s);
  return MG_OK;
}

// kind 0: one cycle as mg_vcycle defines it; kind 1: one solve step
// (cycle followed by the finest-level residual norm into norm_out).
mg_status record(mg_ctx *c, int kind, cudaStream_t s) {
  mg_status st;
  if (!c->dc) {
    if ((st = vcycle_rec(c, 0, false, s))) return st;
    if (kind == 1) return op_norm(c, 0, s);
    return MG_OK;
  }
  if (kind == 0) {
    if ((st = op_norm(c, 0, s))) return st;  // leaves the defect in lv[0].f
    return dc_inner_and_update(c, false, s);
  }
  return dc_inner_and_update(c, true, s);
}

unsigned cur_key(mg_ctx *c) {
  unsigned k = 0;
  for (int l = 0; l < c->nl; l++) k |= (unsigned)c->lv[l].cur << l;
  return k | ((unsigned)c->outer.cur << 31);
}
void set_cur(mg_ctx *c, unsigned k) {
  for (int l = 0; l < c->nl; l++) c->lv[l].cur = (k >> l) & 1u;
  c->outer.cur = (k >> 31) & 1u;
}

void release_slot_pairs(mg_ctx *c, GraphSlot &g) {
  for (int i = 0; i < g.npairs; i++) {
    c->pairs[g.pairs[i]].pending = false;
    c->free_pairs[c->nfree++] = g.pairs[i];
  }
  g.npairs = 0;
}

// After a replay the graph's event pairs hold that replay's times.
void mark_slot_pending(mg_ctx *c, GraphSlot &g) {
  for (int i = 0; i < g.npairs; i++) c->pairs[g.pairs[i]].pending = true;
}

void drop_graphs(mg_ctx *c) {
  for (int i = 0; i < kGraphSlots; i++) {
    if (c->graphs[i].valid) cudaGraphExecDestroy(c->graphs[i].exec);
    c->graphs[i].valid = false;
    release_slot_pairs(c, c->graphs[i]);
  }
}

// Runs one cycle or solve step, replaying a captured graph when enabled.
// A graph is keyed by the live-buffer state it was captured in and stores
// the state it leaves behind (Jacobi sweeps flip a level's live buffer).
mg_status run(mg_ctx *c, int kind) {
  NvtxRange range(kind ? "mg solve step" : "mg V-cycle");
  if (!c->opt.use_graph) return record(c, kind, c->stream);
  unsigned key = cur_key(c);
  for (int i = 0; i < kGraphSlots; i++) {
    GraphSlot &g = c->graphs[i];
    if (g.valid && g.kind == kind && g.key == key) {
      CK(cudaGraphLaunch(g.exec, c->stream));
      c->launches += g.kernels;
      mark_slot_pending(c, g);
      set_cur(c, g.post);
      return MG_OK;
    }
  }
  // Capture on the private stream (created on first use), ordered after the user stream.
  if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  cudaEvent_t ev;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CK(cudaEventRecord(ev, c->stream));
  CK(cudaStreamWaitEvent(c->cap, ev, 0));
  CK(cudaEventDestroy(ev));
  GraphSlot &g = c->graphs[c->next_slot];
  c->next_slot = (c->next_slot + 1) % kGraphSlots;
  if (g.valid) cudaGraphExecDestroy(g.exec);
  g.valid = false;
  release_slot_pairs(c, g);
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  unsigned long long before = c->launches;
  c->capturing_slot = (int)(&g - c->graphs);
  mg_status st = record(c, kind, c->cap);
  c->capturing_slot = -1;
  unsigned long long kernels = c->launches - before;
  c->launches = before;
  unsigned post = cur_key(c);
  set_cur(c, key);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap, &graph);
  if (st) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ee != cudaSuccess) return fail(MG_ECUDA, "graph capture: %s", cudaGetErrorString(ee));
  cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(MG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  g.valid = true;
  g.kind = kind;
  g.key = key;
  g.post = post;
  g.kernels = kernels;
  CK(cudaGraphLaunch(g.exec, c->stream));
  c->launches += kernels;
  mark_slot_pending(c, g);
  set_cur(c, post);
  return MG_OK;
}

mg_status read_norm(mg_ctx *c, double *out) {
  if (!c->host_norm) CK(cudaMallocHost((void **)&c->host_norm, 4 * sizeof(double)));
  CK(cudaMemcpyAsync(c->host_norm, c->norm_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (c->timing) timing_harvest(c);
  *out = c->host_norm[0];
  return MG_OK;
}

}  // namespace

// ---------------------------------------------------------------- ABI

namespace {
// The norm scale of a new context: four FP32 ones (no host upload).
__global__ void k_ones4(float *p) { p[threadIdx.x] = 1.0f; }
}  // namespace

extern "C" {

void mg_default_options(mg_options *o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->smoother = MG_RBGS;
  o->omega = 1.0;
  o->nu1 = 2;
  o->nu2 = 1;
  o->coarsest_n = 3;
  o->maxit = 50;
  o->precision = MG_FP64;
  o->stream = nullptr;
  o->fuse = 1;
  o->use_graph = 1;
  o->inner_cycles = 1;
  o->exact_outer = 1;
  o->join_cycles = 1;
  o->cluster_max_n = 0;
  o->canary = 0;
}

size_t mg_workspace_bytes(int dim, int n, int variable_k, const mg_options *opt) {
  if (check_args(dim, n, opt) != MG_OK) return 0;
  mg_ctx tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.dim = dim;
  tmp.n = n;
  tmp.nl = level_count(n, opt->coarsest_n);
  tmp.variable = variable_k != 0;
  tmp.opt = *opt;
  tmp.dc = opt->precision != MG_FP64;
  tmp.lv[0].c[0] = tmp.lv[0].c[1] = tmp.lv[0].c[2] = 1.0;
  return layout(&tmp, nullptr);
}

mg_status mg_create(int dim, int n, const mg_const_stencil *stencil, const double *k, const mg_boundary *bc,
                    const mg_options *opt, void *arena, size_t arena_bytes, mg_ctx **out) {
  g_err[0] = 0;
  if (!out) return fail(MG_EINVAL, "out is NULL");
  *out = nullptr;
  mg_status st = check_args(dim, n, opt);
  if (st) return st;
  if (!arena) return fail(MG_EINVAL, "arena is NULL");
  if ((uintptr_t)arena % 256) return fail(MG_EINVAL, "arena must be 256-byte aligned");
  if (bc && bc->kind != 0) return fail(MG_EINVAL, "only Dirichlet boundaries (kind 0) are supported");
  double c3[3] = {1.0, 1.0, 1.0};
  if (stencil) {
    c3[0] = stencil->cx;
    c3[1] = stencil->cy;
    c3[2] = dim == 3 ? stencil->cz : 1.0;
    if (!(c3[0] > 0 && c3[1] > 0 && c3[2] > 0)) return fail(MG_EINVAL, "stencil coefficients must be > 0");
  }
  mg_ctx *c = (mg_ctx *)calloc(1, sizeof(mg_ctx));
  if (!c) return fail(MG_ENOMEM, "host allocation of the context failed");
  c->dim = dim;
  c->n = n;
  c->nl = level_count(n, opt->coarsest_n);
  c->variable = k != nullptr;
  c->opt = *opt;
  c->bc_zero = !(bc && bc->dirichlet_values);
  c->u_zero = true;  // the arena is zeroed below
  c->dc = opt->precision != MG_FP64;
  c->stream = (cudaStream_t)opt->stream;
  c->capturing_slot = -1;
  // the device check of the cluster cycle runs here, never inside a capture
  if (dim == 2 && c->dc && opt->fuse && opt->smoother == MG_RBGS) mg::cluster_probe();
  for (int d = 0; d < 3; d++) c->lv[0].c[d] = c3[d];
  size_t need = layout(c, nullptr);
  if (arena_bytes < need) {
    free(c);
    return fail(MG_ENOMEM, "arena has %zu bytes, %zu needed", arena_bytes, need);
  }
  layout(c, (char *)arena);
  c->arena = (char *)arena;
  for (int l = 0; l < c->nl; l++)
    snprintf(c->level_name[l], sizeof c->level_name[l], "level %d n=%d", l, c->lv[l].n);
  c->used_bytes = need;
  cudaError_t e;
#define CKC(call)                                                                  \
  do {                                                                             \
    e = (call);                                                                    \
    if (e != cudaSuccess) {                                                        \
      st = fail(MG_ECUDA, "%s: %s", #call, cudaGetErrorString(e));                 \
      goto bad;                                                                    \
    }                                                                              \
  } while (0)
  CKC(cudaMemsetAsync(arena, 0, need, c->stream));
  for (int g = 0; g < c->nguards; g++)
    CKC(cudaMemsetAsync(c->arena + c->guard_off[g], kGuardByte, kGuardBytes, c->stream));
  if (c->variable) {
    // Node coefficients -> FP64 staging with the finest FP64 layout -> faces.
    Level &K = c->dc ? c->outer : c->lv[0];
    void *stage = K.r;
    CKC(copy_dense_to_pitched(K, k, stage, c->stream));
    Level &F0 = c->dc ? c->outer : c->lv[0];
    CKC(DISPATCH(F0, node_faces, K, (const double *)stage, F0, c->stream));
    c->launches++;
    if (c->dc) {
      CKC(DISPATCH(F0, convert_faces, c->outer, c->lv[0], c->stream));
      if (c->nl > 1) CKC(DISPATCH(F0, coarsen_faces, c->outer, c->lv[1], c->stream));
      for (int l = 2; l < c->nl; l++) CKC(DISPATCH(F0, coarsen_faces, c->lv[l - 1], c->lv[l], c->stream));
      c->launches += c->nl;
    } else {
      for (int l = 1; l < c->nl; l++) CKC(DISPATCH(F0, coarsen_faces, c->lv[l - 1], c->lv[l], c->stream));
      c->launches += c->nl - 1;
    }
    CKC(cudaMemsetAsync(stage, 0, (size_t)K.count * 8, c->stream));
  }
  if (c->lv[c->nl - 1].dense) {
    // the coarsest operator's inverse (after its faces, for variable k)
    Level &Z = c->lv[c->nl - 1];
    CKC(DISPATCH(Z, dense_inverse, Z, c->stream));
    c->launches++;
  }
  if (bc && bc->dirichlet_values) {
    Level &U = user_level(c);
    CKC(copy_dense_to_pitched(U, bc->dirichlet_values, U.u[0], c->stream));
    CKC(DISPATCH(U, zero_interior, U, U.u[0], c->stream));
    c->launches++;
    CKC(cudaMemcpyAsync(U.u[1], U.u[0], (size_t)U.count * 8, cudaMemcpyDeviceToDevice, c->stream));
  }
  k_ones4<<<1, 4, 0, c->stream>>>(c->dc_scale);
  CKC(cudaGetLastError());
  // The caller's k and boundary arrays are borrowed for this call only: wait
  // until their copies have run. Without them nothing needs waiting for; the
  // set-up stays queued on the stream ahead of the context's later work.
  if (k || (bc && bc->dirichlet_values)) CKC(cudaStreamSynchronize(c->stream));
#undef CKC
  *out = c;
  return MG_OK;
bad:
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->host_norm) cudaFreeHost(c->host_norm);
  free(c);
  return st;
}

mg_status mg_destroy(mg_ctx *c) {
  if (!c) return MG_OK;
  drop_graphs(c);
  for (int i = 0; i < c->npairs; i++) {
    cudaEventDestroy(c->pairs[i].a);
    cudaEventDestroy(c->pairs[i].b);
  }
  free(c->pairs);
  free(c->free_pairs);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->host_norm) cudaFreeHost(c->host_norm);
  free(c);
  return MG_OK;
}

mg_status mg_check_canaries(mg_ctx *c, int *damaged) {
  g_err[0] = 0;
  if (!c || !damaged) return fail(MG_EINVAL, "NULL argument");
  *damaged = 0;
  if (!c->opt.canary) return fail(MG_EINVAL, "the context was created with canary = 0");
  size_t bytes = (size_t)c->nguards * kGuardBytes;
  unsigned char *h = (unsigned char *)malloc(bytes ? bytes : 1);
  if (!h) return fail(MG_ENOMEM, "host buffer for the guard zones");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  for (int g = 0; g < c->nguards && e == cudaSuccess; g++)
    e = cudaMemcpy(h + (size_t)g * kGuardBytes, c->arena + c->guard_off[g], kGuardBytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    free(h);
    return fail(MG_ECUDA, "reading the guard zones: %s", cudaGetErrorString(e));
  }
  int first = -1, first_byte = 0;
  for (int g = 0; g < c->nguards; g++) {
    const unsigned char *z = h + (size_t)g * kGuardBytes;
    for (size_t i = 0; i < kGuardBytes; i++) {
      if (z[i] != kGuardByte) {
        if (first < 0) {
          first = g;
          first_byte = (int)i;
        }
        ++*damaged;
        break;
      }
    }
  }
  free(h);
  if (first >= 0)
    snprintf(g_err, sizeof g_err, "%d guard zone(s) damaged; first: after %s, byte %d past its end",
             *damaged, c->guard_tag[first], first_byte);
  return MG_OK;
}

int mg_num_levels(const mg_ctx *c) { return c ? c->nl : -1; }

int mg_level_size(const mg_ctx *c, int level) {
  if (!c || level < 0 || level >= c->nl) return -1;
  return c->lv[level].n;
}

// Rows of a dense FP64 array that the device reaches directly (pinned host
// memory) written into a pitched field: the interior box (interior != 0) or
// every node. Each block takes rows in turn, its threads stream one row with
// 8-byte loads (rows of an odd n start only 8-byte aligned), four in flight
// per thread: host reads cross the chip-to-chip link with microseconds of
// latency.
__global__ void __launch_bounds__(1024) k_rows_in(const double *__restrict__ src, double *__restrict__ dst,
                                                  long long pitch, long long plane, int n, int dim, int interior) {
  const int lo = interior ? 1 : 0, m = n - 2 * lo;
  const long long rows = (long long)m * (dim == 3 ? m : 1);
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = lo + (int)(r % m), k = dim == 3 ? lo + (int)(r / m) : 0;
    const double *a = src + ((long long)k * n + j) * n + lo;
    double *b = dst + (long long)k * plane + (long long)j * pitch + lo;
    const int B = (int)blockDim.x;
    for (int i = threadIdx.x; i < m; i += 4 * B) {
      double v[4];
#pragma unroll
      for (int h = 0; h < 4; h++) v[h] = i + h * B < m ? __ldg(a + i + h * B) : 0.0;
#pragma unroll
      for (int h = 0; h < 4; h++)
        if (i + h * B < m) b[i + h * B] = v[h];
    }
  }
}

// Copies a dense FP64 host or device array into the user level's pitched
// field dst (the interior box, or every node). Pinned host memory is read by
// a small kernel through its device mapping: the copy engines' host reads
// measured slow while the other context of a solve sequence kept HBM busy.
static cudaError_t copy_field_in(mg_ctx *c, const double *src, void *dst, bool interior, cudaStream_t s) {
  Level &U = user_level(c);
  cudaPointerAttributes at;
  bool pinned = false;
  if (cudaPointerGetAttributes(&at, src) == cudaSuccess) {
    pinned = at.type == cudaMemoryTypeHost && at.devicePointer != nullptr;
  } else {
    cudaGetLastError();  // an unknown host pointer: clear the error
  }
  if (pinned) {
    // 16 blocks of 1024 threads, as for the solution's way back
    k_rows_in<<<16, 1024, 0, s>>>((const double *)at.devicePointer, (double *)dst, U.pitch, U.plane, U.n, U.dim,
                                  interior ? 1 : 0);
    c->launches++;
    return cudaGetLastError();
  }
  return interior ? copy_dense_interior(U, src, dst, s) : copy_dense_to_pitched(U, src, dst, s);
}

mg_status mg_set_rhs(mg_ctx *c, const double *f) {
  if (!c || !f) return fail(MG_EINVAL, "NULL argument");
  Level &U = user_level(c);
  // Defect correction: interior only, so the outer right-hand side stays
  // zero on the boundary (the exact outer step takes every value of a row
  // into its exponent).
  CK(copy_field_in(c, f, U.f, c->dc, c->stream));
  return MG_OK;
}

mg_status mg_set_solution(mg_ctx *c, const double *u0) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  Level &U = user_level(c);
  void *dst = user_u(c);
  if (!u0) {
    // Homogeneous Dirichlet data: the whole field (boundary and row padding
    // included) is zero, one contiguous memset. Otherwise a kernel zeroes the
    // interior. (A 2D/3D memset of the interior box cost ~0.6 ms of host time
    // per call; the serving loop sets up thousands of solves a second.)
    if (c->bc_zero) {
      CK(cudaMemsetAsync(dst, 0, (size_t)U.count * 8, c->stream));
    } else {
      CK(DISPATCH(U, zero_interior, U, dst, c->stream));
      c->launches++;
    }
  } else {
    CK(copy_field_in(c, u0, dst, true, c->stream));
  }
  c->u_zero = u0 == nullptr;
  return MG_OK;
}

// Rows of a pitched FP64 field written to a dense array that the device
// reaches directly (pinned host memory): each block takes rows in turn, its
// threads stream one row with 8-byte loads and stores.
__global__ void __launch_bounds__(1024) k_rows_out(const double *__restrict__ src, long long pitch, double *__restrict__ dst, int n,
                           long long rows) {
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const double *a = src + r * pitch;
    double *b = dst + r * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = __ldg(a + i);
  }
}

// Copies the finest (user-level) solution to the dense array dst on stream
// s. Pinned host memory is written by a small kernel through its device
// mapping (the copy engines' device-to-host reads measured slow while the
// other context's kernels kept HBM busy); other host memory goes through the
// context's FP64 staging field - the outer level's r in defect-correction
// contexts, level 0's r (scratch of the residual passes) otherwise: a
// device-side 2D copy into dense layout, then one contiguous copy.
static cudaError_t copy_solution_out(mg_ctx *c, double *dst, cudaStream_t s) {
  Level &U = user_level(c);
  cudaPointerAttributes at;
  bool device = false, pinned = false;
  if (cudaPointerGetAttributes(&at, dst) == cudaSuccess) {
    device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    pinned = at.type == cudaMemoryTypeHost && at.devicePointer != nullptr;
  } else {
    cudaGetLastError();  // an unknown host pointer: clear the error
  }
  if (device) return copy_pitched_to_dense(U, user_u(c), dst, s);
  if (pinned) {
    const long long rows = (long long)U.n * (U.dim == 3 ? U.n : 1);
    // 16 blocks of 1024 threads: fast enough to hide behind a concurrent
    // solve, few enough not to slow it (measured over 16..152 blocks)
    k_rows_out<<<16, 1024, 0, s>>>((const double *)user_u(c), U.pitch, (double *)at.devicePointer, U.n, rows);
    c->launches++;
    return cudaGetLastError();
  }
  double *stage = (double *)(c->dc ? c->outer.r : c->lv[0].r);
  const size_t cnt = (size_t)U.n * U.n * (U.dim == 3 ? U.n : 1);
  cudaError_t e = copy_pitched_to_dense(U, user_u(c), stage, s);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(dst, stage, cnt * 8, cudaMemcpyDeviceToHost, s);
}

mg_status mg_get_solution(mg_ctx *c, double *u) {
  if (!c || !u) return fail(MG_EINVAL, "NULL argument");
  CK(copy_solution_out(c, u, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

static void *field_ptr(Level &L, mg_field f) {
  return f == MG_FIELD_U ? L.u[L.cur] : (f == MG_FIELD_F ? L.f : L.r);
}

mg_status mg_set_field(mg_ctx *c, int level, mg_field field, const double *src) {
  if (!c || !src) return fail(MG_EINVAL, "NULL argument");
  if (level < 0 || level >= c->nl) return fail(MG_EINVAL, "level %d out of range", level);
  if (field < MG_FIELD_U || field > MG_FIELD_R) return fail(MG_EINVAL, "unknown field");
  Level &L = c->lv[level];
  void *dst = field_ptr(L, field);
  if (field == MG_FIELD_U && level == 0 && !c->dc) c->u_zero = false;
  if (L.dtype == mg::F64) {
    CK(copy_dense_to_pitched(L, src, dst, c->stream));
  } else {
    double *stage = (double *)c->outer.r;  // DC contexts only have non-FP64 levels
    size_t cnt = (size_t)L.n * L.n * (L.dim == 3 ? L.n : 1);
    CK(cudaMemcpyAsync(stage, src, cnt * 8, cudaMemcpyDefault, c->stream));
    TLAUNCH(c, MG_KERNEL_OTHER, level, c->stream, DISPATCH(L, from_dense, L, stage, dst, c->stream));
  }
  return MG_OK;
}

mg_status mg_get_field(mg_ctx *c, int level, mg_field field, double *dst) {
  if (!c || !dst) return fail(MG_EINVAL, "NULL argument");
  if (level < 0 || level >= c->nl) return fail(MG_EINVAL, "level %d out of range", level);
  if (field < MG_FIELD_U || field > MG_FIELD_R) return fail(MG_EINVAL, "unknown field");
  Level &L = c->lv[level];
  void *src = field_ptr(L, field);
  if (L.dtype == mg::F64) {
    CK(copy_pitched_to_dense(L, src, dst, c->stream));
  } else {
    double *stage = (double *)c->outer.r;
    size_t cnt = (size_t)L.n * L.n * (L.dim == 3 ? L.n : 1);
    TLAUNCH(c, MG_KERNEL_OTHER, level, c->stream, DISPATCH(L, to_dense, L, src, stage, c->stream));
    CK(cudaMemcpyAsync(dst, stage, cnt * 8, cudaMemcpyDefault, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

mg_status mg_smooth(mg_ctx *c, int level, int sweeps) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (level < 0 || level >= c->nl) return fail(MG_EINVAL, "level %d out of range", level);
  if (sweeps < 0) return fail(MG_EINVAL, "sweeps must be >= 0");
  if (level == 0 && !c->dc) c->u_zero = false;
  return op_smooth(c, level, sweeps, c->stream);
}

mg_status mg_residual(mg_ctx *c, int level) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (level < 0 || level >= c->nl) return fail(MG_EINVAL, "level %d out of range", level);
  return op_residual(c, level, c->stream);
}

mg_status mg_restrict(mg_ctx *c, int level) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (level < 0 || level >= c->nl - 1) return fail(MG_EINVAL, "level %d has no coarser level", level);
  return op_restrict(c, level, c->stream);
}

mg_status mg_prolongate(mg_ctx *c, int level) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (level < 0 || level >= c->nl - 1) return fail(MG_EINVAL, "level %d has no coarser level", level);
  if (level == 0 && !c->dc) c->u_zero = false;
  return op_prolong(c, level, c->stream);
}

mg_status mg_coarse_solve(mg_ctx *c) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (c->nl == 1 && !c->dc) c->u_zero = false;
  return op_coarse(c, c->stream);
}

mg_status mg_vcycle(mg_ctx *c) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  c->u_zero = false;
  return run(c, 0);
}

mg_status mg_residual_norm(mg_ctx *c, int level, double *out) {
  if (!c || !out) return fail(MG_EINVAL, "NULL argument");
  if (level < 0 || level >= c->nl) return fail(MG_EINVAL, "level %d out of range", level);
  mg_status st = op_norm(c, level, c->stream);
  if (st) return st;
  return read_norm(c, out);
}

mg_status mg_solve(mg_ctx *c, double tol, int *iters, double *relres, double *history) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  NvtxRange range("mg_solve");
  if (!(tol >= 0.0)) return fail(MG_EINVAL, "tol must be >= 0");
  double r0;
  mg_status st = c->u_zero && c->bc_zero ? op_first_norm(c, c->stream) : op_norm(c, 0, c->stream);
  if (st) return st;
  if ((st = read_norm(c, &r0))) return st;
  if (history) history[0] = 1.0;
  int k = 0;
  double rho = r0 > 0 ? 1.0 : 0.0;
  if (!isfinite(r0)) return fail(MG_ENOCONV, "initial residual is not finite");
  while (r0 > 0.0 && rho > tol && k < c->opt.maxit) {
    c->u_zero = false;
    if ((st = run(c, 1))) return st;
    double rk;
    if ((st = read_norm(c, &rk))) return st;
    k++;
    rho = rk / r0;
    if (history) history[k] = rho;
    if (!isfinite(rho)) {
      if (iters) *iters = k;
      if (relres) *relres = rho;
      return fail(MG_ENOCONV, "residual is not finite after %d cycles", k);
    }
  }
  if (iters) *iters = k;
  if (relres) *relres = rho;
  if (rho > tol) return fail(MG_ENOCONV, "relative residual %.3e above tol %.3e after %d cycles", rho, tol, k);
  return MG_OK;
}

mg_status mg_solve_sequence(mg_ctx *a, mg_ctx *b, void *copy_stream, int count, const double *const *f,
                            double *const *u, double tol, int *iters, double *relres) {
  g_err[0] = 0;
  if (!a || !b || a == b) return fail(MG_EINVAL, "two distinct contexts are needed");
  if (count < 0 || (count > 0 && (!f || !u))) return fail(MG_EINVAL, "bad count or NULL arrays");
  if (a->dim != b->dim || a->n != b->n || a->dc != b->dc || a->variable != b->variable)
    return fail(MG_EINVAL, "the two contexts differ in dimension, size, precision or stencil kind");
  if (a->stream == b->stream || (cudaStream_t)copy_stream == a->stream || (cudaStream_t)copy_stream == b->stream)
    return fail(MG_EINVAL, "the two contexts and the copy stream need three different streams");
  if (!(tol >= 0.0)) return fail(MG_EINVAL, "tol must be >= 0");
  for (int i = 0; i < count; i++)
    if (!f[i] || !u[i]) return fail(MG_EINVAL, "NULL right-hand side or solution %d", i);
  if (count == 0) return MG_OK;
  NvtxRange range("mg_solve_sequence");
  cudaStream_t cs = (cudaStream_t)copy_stream;
  mg_ctx *cx[2] = {a, b};
  cudaEvent_t solved[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
  bool pending[2] = {false, false};  // a copy-back of the context's solution is queued
  mg_status st = MG_OK, worst = MG_OK;
  for (int k = 0; k < 2 && st == MG_OK; k++) {
    if (cudaEventCreateWithFlags(&solved[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied[k], cudaEventDisableTiming) != cudaSuccess)
      st = fail(MG_ECUDA, "event creation failed");
  }
  auto load = [&](int i) -> mg_status {
    mg_ctx *X = cx[i & 1];
    // f travels at once (the copy-back of the context's previous solution
    // reads u only); u is reset once that copy-back has finished
    mg_status s1 = mg_set_rhs(X, f[i]);
    if (s1) return s1;
    if (pending[i & 1] && cudaStreamWaitEvent(X->stream, copied[i & 1], 0) != cudaSuccess)
      return fail(MG_ECUDA, "stream wait");
    return mg_set_solution(X, nullptr);
  };
  if (st == MG_OK) st = load(0);
  for (int i = 0; i < count && st == MG_OK; i++) {
    mg_ctx *X = cx[i & 1];
    // the next problem's right-hand side travels while this one is solved
    if (i + 1 < count && (st = load(i + 1))) break;
    int it = 0;
    double rr = 0.0;
    mg_status s1 = mg_solve(X, tol, &it, &rr, nullptr);
    if (iters) iters[i] = it;
    if (relres) relres[i] = rr;
    if (s1 == MG_ENOCONV) worst = MG_ENOCONV;
    else if (s1) {
      st = s1;
      break;
    }
    // this solution travels back on the copy stream while the next one is solved
    if (cudaEventRecord(solved[i & 1], X->stream) != cudaSuccess ||
        cudaStreamWaitEvent(cs, solved[i & 1], 0) != cudaSuccess ||
        copy_solution_out(X, u[i], cs) != cudaSuccess ||
        cudaEventRecord(copied[i & 1], cs) != cudaSuccess) {
      st = fail(MG_ECUDA, "copy of solution %d", i);
      break;
    }
    pending[i & 1] = true;
  }
  cudaError_t e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; k++) {
    if (solved[k]) cudaEventDestroy(solved[k]);
    if (copied[k]) cudaEventDestroy(copied[k]);
  }
  if (st == MG_OK && e != cudaSuccess) st = fail(MG_ECUDA, "synchronize: %s", cudaGetErrorString(e));
  if (st) return st;
  if (worst) return fail(MG_ENOCONV, "some problems did not reach tol");
  return MG_OK;
}

unsigned long long mg_kernel_launches(const mg_ctx *c) { return c ? c->launches : 0ull; }

mg_status mg_set_timing(mg_ctx *c, int on) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (on && !c->pairs) {
    c->pairs = (TimingPair *)calloc(kMaxPairs, sizeof(TimingPair));
    c->free_pairs = (int *)calloc(kMaxPairs, sizeof(int));
    if (!c->pairs || !c->free_pairs) {
      free(c->pairs);
      free(c->free_pairs);
      c->pairs = nullptr;
      c->free_pairs = nullptr;
      return fail(MG_ENOMEM, "host allocation of timing events failed");
    }
  }
  if (on < 0 || on > 3) return fail(MG_EINVAL, "timing mode must be 0, 1, 2 or 3");
  if (on != c->timing) {
    CK(cudaStreamSynchronize(c->stream));
    if (c->timing) timing_harvest(c);
    drop_graphs(c);  // graphs are recaptured with (or without) event nodes
    c->timing = on;
  }
  return MG_OK;
}

mg_status mg_get_timing(mg_ctx *c, int kind, int level, double *total_ms, unsigned long long *count) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  if (kind < 0 || kind >= kKinds || level < 0 || level >= kMaxLevels) return fail(MG_EINVAL, "bad kind or level");
  CK(cudaStreamSynchronize(c->stream));
  if (c->timing) timing_harvest(c);
  if (total_ms) *total_ms = c->t_ms[kind][level];
  if (count) *count = c->t_n[kind][level];
  return MG_OK;
}

mg_status mg_reset_timing(mg_ctx *c) {
  if (!c) return fail(MG_EINVAL, "NULL context");
  CK(cudaStreamSynchronize(c->stream));
  if (c->timing) timing_harvest(c);
  memset(c->t_ms, 0, sizeof c->t_ms);
  memset(c->t_n, 0, sizeof c->t_n);
  return MG_OK;
}

const char *mg_last_error(void) { return g_err; }

}  // extern "C"

// ---------------------------------------------------------------- norm finalize

namespace mg {

void set_error_message(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

// Sums kNormBlocks partials in a fixed tree order (deterministic).
__global__ void k_norm_finalize(const double *__restrict__ partials, int nb, double *__restrict__ out) {
  __shared__ double buf[1024];
  int t = threadIdx.x;
  buf[t] = t < nb ? partials[t] : 0.0;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (t < s) buf[t] += buf[t + s];
    __syncthreads();
  }
  if (t == 0) {
    out[0] = sqrt(buf[0]);
    out[1] = buf[0];
  }
}

int pow2_stencil(const Level &L) {
  if (L.kf[0]) return kNoPow2;
  const double c = L.c[0] * L.inv_h2;
  for (int d = 1; d < L.dim; d++)
    if (L.c[d] * L.inv_h2 != c) return kNoPow2;
  int e = 0;
  if (!(c > 0.0) || frexp(c, &e) != 0.5) return kNoPow2;
  return e - 1;  // c = 0.5 * 2^e
}

cudaError_t norm_finalize(const double *partials, int nblocks, double *out, cudaStream_t s) {
  if (nblocks > 1024) return cudaErrorInvalidValue;
  k_norm_finalize<<<1, 1024, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

}  // namespace mg
