// Host-side dispatch from a Level (runtime dim/dtype/stencil kind) to the
// templated kernels. Included once per dimension with MG_DIM and MG_NS set.
#include "kernels.cuh"

namespace mg {
namespace MG_NS {

static const int kDim = MG_DIM;

static dim3 node_grid(int n, int bx) {
  return dim3((unsigned)((n + bx - 1) / bx), (unsigned)n, kDim == 3 ? (unsigned)n : 1u);
}

#define MG_DISPATCH_T(dtype, ...)                         \
  switch (dtype) {                                        \
    case F64: { typedef double T; __VA_ARGS__; } break;   \
    case F32: { typedef float T; __VA_ARGS__; } break;    \
    default: { typedef bf16 T; __VA_ARGS__; } break;      \
  }

cudaError_t rbgs_half(const Level &L, void *u, const void *f, int color, double omega, cudaStream_t s) {
  if (kDim == 3 && d3::z_ok(L)) return d3::z_sweep(L, u, u, f, color, omega, s);
  dim3 b(128), gr = node_grid(L.n, 128);
  bool var = L.kf[0] != nullptr;
  MG_DISPATCH_T(L.dtype, {
    typedef typename CT<T>::type C;
    if (var) k_rbgs_half<kDim, T, true><<<gr, b, 0, s>>>((T *)u, (const T *)f, geo_of(L), sten_of<C>(L), color, (C)omega);
    else k_rbgs_half<kDim, T, false><<<gr, b, 0, s>>>((T *)u, (const T *)f, geo_of(L), sten_of<C>(L), color, (C)omega);
  })
  return cudaGetLastError();
}

cudaError_t jacobi(const Level &L, const void *uin, void *uout, const void *f, double omega, cudaStream_t s) {
  if (kDim == 3 && d3::z_ok(L)) return d3::z_sweep(L, uin, uout, f, -1, omega, s);
  dim3 b(128), gr = node_grid(L.n, 128);
  bool var = L.kf[0] != nullptr;
  MG_DISPATCH_T(L.dtype, {
    typedef typename CT<T>::type C;
    if (var) k_jacobi<kDim, T, true><<<gr, b, 0, s>>>((const T *)uin, (T *)uout, (const T *)f, geo_of(L), sten_of<C>(L), (C)omega);
    else k_jacobi<kDim, T, false><<<gr, b, 0, s>>>((const T *)uin, (T *)uout, (const T *)f, geo_of(L), sten_of<C>(L), (C)omega);
  })
  return cudaGetLastError();
}

cudaError_t residual(const Level &L, const void *u, const void *f, void *r, cudaStream_t s) {
  if (kDim == 3 && d3::z_ok(L)) return d3::z_residual(L, u, f, r, s);
  dim3 b(128), gr = node_grid(L.n, 128);
  bool var = L.kf[0] != nullptr;
  MG_DISPATCH_T(L.dtype, {
    typedef typename CT<T>::type C;
    if (var) k_residual<kDim, T, true><<<gr, b, 0, s>>>((const T *)u, (const T *)f, (T *)r, geo_of(L), sten_of<C>(L));
    else k_residual<kDim, T, false><<<gr, b, 0, s>>>((const T *)u, (const T *)f, (T *)r, geo_of(L), sten_of<C>(L));
  })
  return cudaGetLastError();
}

cudaError_t restrict_fw(const Level &F, const void *rf, const Level &C, void *fc, cudaStream_t s) {
  if (kDim == 3 && d3::transfer_ok(F, C)) return d3::z_restrict(F, rf, C, fc, s);
  dim3 b(128), gr = node_grid(C.n, 128);
  switch (F.dtype) {
    case F64:
      k_restrict<kDim, double, double><<<gr, b, 0, s>>>((const double *)rf, geo_of(F), (double *)fc, geo_of(C));
      break;
    case F32:
      if (C.dtype == F64) k_restrict<kDim, float, double><<<gr, b, 0, s>>>((const float *)rf, geo_of(F), (double *)fc, geo_of(C));
      else k_restrict<kDim, float, float><<<gr, b, 0, s>>>((const float *)rf, geo_of(F), (float *)fc, geo_of(C));
      break;
    default:
      if (C.dtype == F64) k_restrict<kDim, bf16, double><<<gr, b, 0, s>>>((const bf16 *)rf, geo_of(F), (double *)fc, geo_of(C));
      else k_restrict<kDim, bf16, bf16><<<gr, b, 0, s>>>((const bf16 *)rf, geo_of(F), (bf16 *)fc, geo_of(C));
      break;
  }
  return cudaGetLastError();
}

cudaError_t prolong(const Level &C, const void *ec, const Level &F, void *uf, cudaStream_t s) {
  if (kDim == 3 && d3::transfer_ok(F, C)) return d3::z_prolong(C, ec, F, uf, s);
  dim3 b(128), gr = node_grid(F.n, 128);
  switch (F.dtype) {
    case F64:
      k_prolong<kDim, double, double><<<gr, b, 0, s>>>((const double *)ec, geo_of(C), (double *)uf, geo_of(F));
      break;
    case F32:
      if (C.dtype == F64) k_prolong<kDim, double, float><<<gr, b, 0, s>>>((const double *)ec, geo_of(C), (float *)uf, geo_of(F));
      else k_prolong<kDim, float, float><<<gr, b, 0, s>>>((const float *)ec, geo_of(C), (float *)uf, geo_of(F));
      break;
    default:
      if (C.dtype == F64) k_prolong<kDim, double, bf16><<<gr, b, 0, s>>>((const double *)ec, geo_of(C), (bf16 *)uf, geo_of(F));
      else k_prolong<kDim, bf16, bf16><<<gr, b, 0, s>>>((const bf16 *)ec, geo_of(C), (bf16 *)uf, geo_of(F));
      break;
  }
  return cudaGetLastError();
}

cudaError_t norm_partials(const Level &L, const void *u, const void *f, double *partials, int nblocks,
                          cudaStream_t s) {
  bool var = L.kf[0] != nullptr;
  MG_DISPATCH_T(L.dtype, {
    typedef typename CT<T>::type C;
    if (var) k_norm_partials<kDim, T, true><<<nblocks, 256, 0, s>>>((const T *)u, (const T *)f, geo_of(L), sten_of<C>(L), partials);
    else k_norm_partials<kDim, T, false><<<nblocks, 256, 0, s>>>((const T *)u, (const T *)f, geo_of(L), sten_of<C>(L), partials);
  })
  return cudaGetLastError();
}

cudaError_t coarse3(const Level &L, void *u, const void *f, cudaStream_t s) {
  if (L.dtype != F64 || L.n != 3) return cudaErrorInvalidValue;
  if (L.kf[0]) k_coarse3<kDim, true><<<1, 1, 0, s>>>((double *)u, (const double *)f, geo_of(L), sten_of<double>(L));
  else k_coarse3<kDim, false><<<1, 1, 0, s>>>((double *)u, (const double *)f, geo_of(L), sten_of<double>(L));
  return cudaGetLastError();
}

// Dense coarsest grids (n - 2)^dim <= kDenseMax unknowns, FP64 only.
static bool dense_ok(const Level &L) {
  long long m = L.n - 2, N = kDim == 3 ? m * m * m : m * m;
  return L.dtype == F64 && L.dense && L.n >= 5 && N <= kDenseMax;
}

cudaError_t dense_inverse(const Level &L, cudaStream_t s) {
  if (!dense_ok(L)) return cudaErrorInvalidValue;
  if (L.kf[0]) k_dense_inverse<kDim, true><<<1, 1024, 0, s>>>(L.dense, geo_of(L), sten_of<double>(L));
  else k_dense_inverse<kDim, false><<<1, 1024, 0, s>>>(L.dense, geo_of(L), sten_of<double>(L));
  return cudaGetLastError();
}

cudaError_t coarse_dense(const Level &L, void *u, const void *f, cudaStream_t s) {
  if (!dense_ok(L)) return cudaErrorInvalidValue;
  if (L.kf[0]) k_coarse_dense<kDim, true><<<1, 352, 0, s>>>((double *)u, (const double *)f, geo_of(L), sten_of<double>(L), L.dense);
  else k_coarse_dense<kDim, false><<<1, 352, 0, s>>>((double *)u, (const double *)f, geo_of(L), sten_of<double>(L), L.dense);
  return cudaGetLastError();
}

cudaError_t dc_residual(const Level &O, const void *u, const void *f, const Level &I, void *d, double *partials,
                        int nblocks, cudaStream_t s) {
  bool var = O.kf[0] != nullptr;
  Sten<double> st = sten_of<double>(O);
  switch (I.dtype) {
    case F32:
      if (var) k_dc_residual<kDim, float, true><<<nblocks, 256, 0, s>>>((const double *)u, (const double *)f, geo_of(O), st, (float *)d, geo_of(I), partials);
      else k_dc_residual<kDim, float, false><<<nblocks, 256, 0, s>>>((const double *)u, (const double *)f, geo_of(O), st, (float *)d, geo_of(I), partials);
      break;
    case BF16:
      if (var) k_dc_residual<kDim, bf16, true><<<nblocks, 256, 0, s>>>((const double *)u, (const double *)f, geo_of(O), st, (bf16 *)d, geo_of(I), partials);
      else k_dc_residual<kDim, bf16, false><<<nblocks, 256, 0, s>>>((const double *)u, (const double *)f, geo_of(O), st, (bf16 *)d, geo_of(I), partials);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t dc_update(const Level &O, void *u, const Level &I, const void *e, cudaStream_t s) {
  dim3 b(128), gr = node_grid(O.n, 128);
  switch (I.dtype) {
    case F32: k_dc_update<kDim, float><<<gr, b, 0, s>>>((double *)u, geo_of(O), (const float *)e, geo_of(I)); break;
    case BF16: k_dc_update<kDim, bf16><<<gr, b, 0, s>>>((double *)u, geo_of(O), (const bf16 *)e, geo_of(I)); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t from_dense(const Level &L, const double *src, void *dst, cudaStream_t s) {
  dim3 b(128), gr = node_grid(L.n, 128);
  MG_DISPATCH_T(L.dtype, { k_from_dense<kDim, T><<<gr, b, 0, s>>>(src, (T *)dst, geo_of(L)); })
  return cudaGetLastError();
}

cudaError_t to_dense(const Level &L, const void *src, double *dst, cudaStream_t s) {
  dim3 b(128), gr = node_grid(L.n, 128);
  MG_DISPATCH_T(L.dtype, { k_to_dense<kDim, T><<<gr, b, 0, s>>>((const T *)src, dst, geo_of(L)); })
  return cudaGetLastError();
}

cudaError_t zero_interior(const Level &L, void *field, cudaStream_t s) {
  dim3 b(128), gr = node_grid(L.n, 128);
  MG_DISPATCH_T(L.dtype, { k_zero_interior<kDim, T><<<gr, b, 0, s>>>((T *)field, geo_of(L)); })
  return cudaGetLastError();
}

cudaError_t copy_boundary(const Level &L, const void *src, void *dst, cudaStream_t s) {
  dim3 b(128), gr = node_grid(L.n, 128);
  MG_DISPATCH_T(L.dtype, { k_copy_boundary<kDim, T><<<gr, b, 0, s>>>((const T *)src, (T *)dst, geo_of(L)); })
  return cudaGetLastError();
}

cudaError_t node_faces(const Level &K, const double *knode, const Level &Lo, cudaStream_t s) {
  dim3 b(128), gr = node_grid(Lo.n, 128);
  if (Lo.dtype == F64)
    k_node_faces<kDim, double><<<gr, b, 0, s>>>(knode, geo_of(K), (double *)Lo.kf[0], (double *)Lo.kf[1],
                                                (double *)Lo.kf[2], geo_of(Lo), Lo.c[0], Lo.c[1], Lo.c[2]);
  else
    k_node_faces<kDim, float><<<gr, b, 0, s>>>(knode, geo_of(K), (float *)Lo.kf[0], (float *)Lo.kf[1],
                                               (float *)Lo.kf[2], geo_of(Lo), Lo.c[0], Lo.c[1], Lo.c[2]);
  return cudaGetLastError();
}

cudaError_t coarsen_faces(const Level &F, const Level &C, cudaStream_t s) {
  dim3 b(128), gr = node_grid(C.n, 128);
  bool f64 = F.dtype == F64, c64 = C.dtype == F64;
  if (f64 && c64)
    k_coarsen_faces<kDim, double, double><<<gr, b, 0, s>>>((const double *)F.kf[0], (const double *)F.kf[1], (const double *)F.kf[2], geo_of(F), (double *)C.kf[0], (double *)C.kf[1], (double *)C.kf[2], geo_of(C));
  else if (!f64 && c64)
    k_coarsen_faces<kDim, float, double><<<gr, b, 0, s>>>((const float *)F.kf[0], (const float *)F.kf[1], (const float *)F.kf[2], geo_of(F), (double *)C.kf[0], (double *)C.kf[1], (double *)C.kf[2], geo_of(C));
  else if (f64 && !c64)
    k_coarsen_faces<kDim, double, float><<<gr, b, 0, s>>>((const double *)F.kf[0], (const double *)F.kf[1], (const double *)F.kf[2], geo_of(F), (float *)C.kf[0], (float *)C.kf[1], (float *)C.kf[2], geo_of(C));
  else
    k_coarsen_faces<kDim, float, float><<<gr, b, 0, s>>>((const float *)F.kf[0], (const float *)F.kf[1], (const float *)F.kf[2], geo_of(F), (float *)C.kf[0], (float *)C.kf[1], (float *)C.kf[2], geo_of(C));
  return cudaGetLastError();
}

cudaError_t convert_faces(const Level &S, const Level &D, cudaStream_t s) {
  dim3 b(128), gr = node_grid(D.n, 128);
  bool s64 = S.dtype == F64, d64 = D.dtype == F64;
  if (s64 && !d64)
    k_convert_faces<kDim, double, float><<<gr, b, 0, s>>>((const double *)S.kf[0], (const double *)S.kf[1], (const double *)S.kf[2], geo_of(S), (float *)D.kf[0], (float *)D.kf[1], (float *)D.kf[2], geo_of(D));
  else if (s64 && d64)
    k_convert_faces<kDim, double, double><<<gr, b, 0, s>>>((const double *)S.kf[0], (const double *)S.kf[1], (const double *)S.kf[2], geo_of(S), (double *)D.kf[0], (double *)D.kf[1], (double *)D.kf[2], geo_of(D));
  else
    k_convert_faces<kDim, float, float><<<gr, b, 0, s>>>((const float *)S.kf[0], (const float *)S.kf[1], (const float *)S.kf[2], geo_of(S), (float *)D.kf[0], (float *)D.kf[1], (float *)D.kf[2], geo_of(D));
  return cudaGetLastError();
}

}  // namespace MG_NS
}  // namespace mg
