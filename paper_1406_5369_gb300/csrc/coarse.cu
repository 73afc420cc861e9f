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

size_t coarse_args(const Level *lv, int first, int nl, bool zero_top, int smoother, double omega, int nu1, int nu2,
                   bool fp64, void *args_out) {
  cz::CoarseArgs &a = *(cz::CoarseArgs *)args_out;
  memset(&a, 0, sizeof a);
  const Level &T = lv[first];
  a.dim = T.dim;
  a.nlev = nl - first;
  if (a.nlev > cz::kMaxLev || a.nlev < 1) return 0;
  a.var = T.kf[0] != nullptr;
  for (int d = 0; d < 3; d++) {
    a.c[d] = T.c[d];
    a.cf[d] = (float)T.c[d];
  }
  size_t elems = 0;
  for (int i = 0; i < a.nlev; i++) {
    const Level &L = lv[first + i];
    a.n[i] = L.n;
    a.inv_h2[i] = L.inv_h2;
    a.inv_h2f[i] = (float)L.inv_h2;
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
  const Level &Z = lv[nl - 1];
  if (Z.dense) {
    // N FP64 slots: 2N elements cover them for float cycles, at an even
    // element offset so that they are 8-byte aligned
    size_t m = (size_t)Z.n - 2, N = Z.dim == 3 ? m * m * m : m * m;
    elems = (elems + 1) & ~(size_t)1;
    a.dense = Z.dense;
    a.off_rd = (int)elems;
    elems += 2 * N;
  }
  a.total = (int)elems;
  a.f_top = T.f;
  a.u_top = T.u[T.cur];
  a.top_dtype = T.dtype;
  a.zero_top = zero_top;
  a.smoother = smoother;
  a.omega = omega;
  a.omegaf = (float)omega;
  a.nu1 = nu1;
  a.nu2 = nu2;
  size_t smem = elems * (fp64 ? 8 : 4);
  if (smem > 227 * 1024) return 0;
  return smem;
}

size_t coarse_args_bytes() { return sizeof(cz::CoarseArgs); }

void coarse_args_set_live(void *args, const int *live) { ((cz::CoarseArgs *)args)->live = live; }

cudaError_t coarse_cycle(const Level *lv, int first, int nl, bool zero_top, int smoother, double omega, int nu1,
                         int nu2, bool fp64, cudaStream_t s) {
  cz::CoarseArgs a;
  size_t smem = coarse_args(lv, first, nl, zero_top, smoother, omega, nu1, nu2, fp64, &a);
  if (!smem) return cudaErrorInvalidValue;
  if (a.dim == 2) {
    if (fp64) return a.var ? launch<2, true, double>(a, smem, s) : launch<2, false, double>(a, smem, s);
    return a.var ? launch<2, true, float>(a, smem, s) : launch<2, false, float>(a, smem, s);
  }
  if (fp64) return a.var ? launch<3, true, double>(a, smem, s) : launch<3, false, double>(a, smem, s);
  return a.var ? launch<3, true, float>(a, smem, s) : launch<3, false, float>(a, smem, s);
}

namespace {
template <int DIM, bool VAR, typename C>
cudaError_t launch_batched(const void *list, int count, size_t smem, cudaStream_t s) {
  static size_t opted = 0;
  if (smem > opted) {
    cudaError_t e = cudaFuncSetAttribute(cz::k_coarse_cycle_batched<DIM, VAR, C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    opted = smem;
  }
  cz::k_coarse_cycle_batched<DIM, VAR, C><<<count, cz::kThreads, smem, s>>>((const cz::CoarseArgs *)list);
  return cudaGetLastError();
}
}  // namespace

cudaError_t coarse_cycle_batched(const void *list_dev, int count, int dim, bool var, bool fp64, size_t smem,
                                 cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (dim == 2) {
    if (fp64) return var ? launch_batched<2, true, double>(list_dev, count, smem, s)
                         : launch_batched<2, false, double>(list_dev, count, smem, s);
    return var ? launch_batched<2, true, float>(list_dev, count, smem, s)
               : launch_batched<2, false, float>(list_dev, count, smem, s);
  }
  if (fp64) return var ? launch_batched<3, true, double>(list_dev, count, smem, s)
                       : launch_batched<3, false, double>(list_dev, count, smem, s);
  return var ? launch_batched<3, true, float>(list_dev, count, smem, s)
             : launch_batched<3, false, float>(list_dev, count, smem, s);
}

}  // namespace mg
