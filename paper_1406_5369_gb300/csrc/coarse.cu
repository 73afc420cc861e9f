// Launcher of the single-block coarse-level V-cycle (coarse.cuh).
#include <string.h>

#include "coarse.cuh"

namespace mg {

namespace {

template <int DIM, bool VAR, typename C>
cudaError_t launch(const cz::CoarseArgs &a, size_t smem, cudaStream_t s) {
  static size_t opted = 0;
  if (smem > opted) {
    cudaError_t e = cudaFuncSetAttribute(cz::k_coarse_cycle<DIM, VAR, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    opted = smem;
  }
  cz::k_coarse_cycle<DIM, VAR, C><<<1, cz::kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int coarse_top_n(int dim, bool fp64) {
  // Largest level handed to the single-block cycle: one SM's FP64 rate is
  // 1/64 of its FP32 rate, so FP64 contexts stop one level lower.
  if (dim == 2) return fp64 ? 33 : 65;
  return fp64 ? 9 : 17;
}

cudaError_t coarse_cycle(const Level *lv, int first, int nl, bool zero_top, int smoother, double omega, int nu1,
                         int nu2, bool fp64, cudaStream_t s) {
  cz::CoarseArgs a;
  memset(&a, 0, sizeof a);
  const Level &T = lv[first];
  a.dim = T.dim;
  a.nlev = nl - first;
  if (a.nlev > cz::kMaxLev || a.nlev < 1) return cudaErrorInvalidValue;
  a.var = T.kf[0] != nullptr;
  for (int d = 0; d < 3; d++) a.c[d] = T.c[d];
  size_t elems = 0;
  for (int i = 0; i < a.nlev; i++) {
    const Level &L = lv[first + i];
    a.n[i] = L.n;
    a.inv_h2[i] = L.inv_h2;
    a.pitch[i] = L.pitch;
    a.plane[i] = L.plane;
    a.kf64[i] = L.dtype == F64;
    for (int d = 0; d < 3; d++) a.kf[i][d] = L.kf[d];
    size_t N = (size_t)L.n * L.n * (L.dim == 3 ? L.n : 1);
    a.off_u[i] = (int)elems;
    a.off_f[i] = (int)(elems + N);
    a.off_k[i] = (int)(elems + 2 * N);
    elems += N * (2 + (a.var ? L.dim : 0));
  }
  a.off_tmp = (int)elems;
  elems += (size_t)T.n * T.n * (T.dim == 3 ? T.n : 1);
  a.total = (int)elems;
  a.f_top = T.f;
  a.u_top = T.u[T.cur];
  a.top_dtype = T.dtype;
  a.zero_top = zero_top;
  a.smoother = smoother;
  a.omega = omega;
  a.nu1 = nu1;
  a.nu2 = nu2;
  size_t smem = elems * (fp64 ? 8 : 4);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (T.dim == 2) {
    if (fp64) return a.var ? launch<2, true, double>(a, smem, s) : launch<2, false, double>(a, smem, s);
    return a.var ? launch<2, true, float>(a, smem, s) : launch<2, false, float>(a, smem, s);
  }
  if (fp64) return a.var ? launch<3, true, double>(a, smem, s) : launch<3, false, double>(a, smem, s);
  return a.var ? launch<3, true, float>(a, smem, s) : launch<3, false, float>(a, smem, s);
}

}  // namespace mg
