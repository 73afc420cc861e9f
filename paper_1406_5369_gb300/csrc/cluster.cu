// Launcher of the thread-block-cluster V-cycle of the small 2D levels
// (cluster.cuh).
#include <string.h>

#include "cluster.cuh"
#include "mg_internal.h"

namespace mg {

namespace {

int log2_exact(int v) {
  int k = 0;
  while ((1 << k) < v) k++;
  return (1 << k) == v ? k : -1;
}

// Fills the kernel arguments for the levels first..nl-1; returns the shared
// memory per block, 0 if the hierarchy does not have the cluster cycle's
// shape (2D, constant stencil, top 129^2 or 257^2, halving down to 33^2
// and below) or does not fit.
size_t cluster_args(const Level *lv, int first, int nl, bool zero_top, double omega, int nu1, int nu2, int nctas,
                    kz::ClusterArgs &a) {
  memset(&a, 0, sizeof a);
  if (nctas < 2 || nctas > kz::kMaxCTAs) return 0;
  a.nctas = nctas;
  const Level &T = lv[first];
  if (T.dim != 2 || T.kf[0] || (T.n != 129 && T.n != 257)) return 0;
  int nd = 0;
  while (first + nd < nl && lv[first + nd].n > kz::kLocalN) nd++;
  if (nd < 1 || nd > kz::kMaxDist || first + nd >= nl || lv[first + nd].n != kz::kLocalN) return 0;
  for (int l = 0; l < nd; l++) {
    const Level &L = lv[first + l];
    if (L.n != ((lv[first + l + 1].n - 1) << 1) + 1 || L.kf[0]) return 0;
  }
  a.nd = nd;
  // bands of the 33^2 level, then each finer level's nested in them
  const int m = kz::kLocalN - 2;
  for (int r = 0; r < nctas; r++) a.band[nd][r] = 1 + r * m / nctas;
  a.band[nd][nctas] = kz::kLocalN - 1;
  for (int l = nd - 1; l >= 0; l--) {
    const int n = lv[first + l].n;
    a.band[l][0] = 1;
    for (int r = 1; r < nctas; r++) a.band[l][r] = 2 * a.band[l + 1][r];
    a.band[l][nctas] = n - 1;
  }
  size_t elems = 0;
  for (int l = 0; l < nd; l++) {
    const Level &L = lv[first + l];
    int rmax = 0;
    for (int r = 0; r < nctas; r++) {
      const int R = a.band[l][r + 1] - a.band[l][r];
      if (R < 1) return 0;
      if (R > rmax) rmax = R;
    }
    a.n[l] = L.n;
    a.lgn[l] = log2_exact(L.n - 1);
    if (a.lgn[l] < 1) return 0;
    a.rmax[l] = rmax;
    a.ih2[l] = (float)L.inv_h2;
    a.off_u[l] = (int)elems;
    elems += (size_t)(rmax + 2) * L.n;
    a.off_f[l] = (int)elems;
    elems += (size_t)rmax * L.n;
    a.off_r[l] = (int)elems;
    elems += (size_t)(rmax + 1) * L.n;
  }
  elems = (elems + 3) & ~(size_t)3;  // the single-block levels start 16-byte aligned
  a.off_local = (int)elems;
  const size_t local = coarse_args(lv, first + nd, nl, true, 0, omega, nu1, nu2, false, &a.local);
  if (!local) return 0;
  elems += (size_t)a.local.total;
  a.total = (int)elems;
  a.cf[0] = (float)T.c[0];
  a.cf[1] = (float)T.c[1];
  a.omegaf = (float)omega;
  a.nu1 = nu1;
  a.nu2 = nu2;
  a.f_top = T.f;
  a.u_top = T.u[T.cur];
  a.top_dtype = T.dtype;
  a.pitch_top = T.pitch;
  a.zero_top = zero_top;
  const size_t smem = elems * sizeof(float);
  return smem <= 227 * 1024 ? smem : 0;
}

// Blocks per cluster the device can place with this kernel's shared memory
// (16 or 8), 0 = neither, -1 = not checked yet.
int g_nctas = -1;
size_t g_opted = 0;

cudaError_t prepare(size_t smem) {
  if (smem > g_opted) {
    cudaError_t e = cudaFuncSetAttribute(kz::k_cluster_cycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    g_opted = smem;
  }
  return cudaSuccess;
}

void config(cudaLaunchConfig_t &cfg, cudaLaunchAttribute &at, size_t smem, int nctas, cudaStream_t s) {
  memset(&cfg, 0, sizeof cfg);
  memset(&at, 0, sizeof at);
  cfg.gridDim = dim3(nctas, 1, 1);
  cfg.blockDim = dim3(kz::kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = nctas;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
}

}  // namespace

void cluster_probe() {
  if (g_nctas >= 0) return;
  // clusters of blocks with the most shared memory a block can have (more
  // than any layout here needs), checked once against the device: 16 blocks
  // (a non-portable size), else 8
  g_nctas = 0;
  if (prepare(227 * 1024) == cudaSuccess) {
    const bool big = cudaFuncSetAttribute(kz::k_cluster_cycle, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                     cudaSuccess;
    for (int nctas : {16, 8}) {
      if (nctas > 8 && !big) continue;
      int clusters = 0;
      cudaLaunchConfig_t cfg;
      cudaLaunchAttribute at;
      config(cfg, at, 227 * 1024, nctas, 0);
      if (cudaOccupancyMaxActiveClusters(&clusters, kz::k_cluster_cycle, &cfg) == cudaSuccess && clusters >= 1) {
        g_nctas = nctas;
        break;
      }
    }
  }
  cudaGetLastError();  // a refused query leaves no sticky error behind
}

bool cluster_ok(const Level *lv, int l, int nl, int smoother, bool fp64, int cluster_max_n) {
  const int top = cluster_max_n > 0 ? cluster_max_n : 257;
  if (g_nctas <= 0 || fp64 || smoother != 0 || lv[l].n > top) return false;
  kz::ClusterArgs a;
  return cluster_args(lv, l, nl, true, 1.0, 1, 1, g_nctas, a) != 0;
}

cudaError_t cluster_cycle(const Level *lv, int first, int nl, bool zero_top, double omega, int nu1, int nu2,
                          cudaStream_t s) {
  kz::ClusterArgs a;
  if (g_nctas <= 0) return cudaErrorInvalidValue;
  const size_t smem = cluster_args(lv, first, nl, zero_top, omega, nu1, nu2, g_nctas, a);
  if (!smem) return cudaErrorInvalidValue;
  cudaError_t e = prepare(smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at;
  config(cfg, at, smem, g_nctas, s);
  e = cudaLaunchKernelEx(&cfg, kz::k_cluster_cycle, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace mg
