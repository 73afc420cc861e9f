// V-cycle of the small 2D levels in one thread-block cluster (Algorithm 1
// below a size threshold, constant stencil, red-black Gauss-Seidel, FP32
// arithmetic: the inner levels of defect correction).
//
// A cluster of 16 blocks (8 where the device cannot place 16) of 1024 threads,
// one per SM, keeps every level from the top one (129^2 or 257^2) down to 65^2
// in distributed shared memory: block r owns a band of interior rows of each
// level plus one halo row above and below. The bands of consecutive levels are
// nested (the fine band of block r starts at twice the first coarse row of its
// coarse band), so that full weighting and bilinear interpolation read only
// the block's own rows and halo rows, apart from one residual row that the
// block above supplies. A red-black half-sweep of colour c updates colour-c
// nodes from colour-(1-c) neighbours only; the thread that updates a node in a
// band's first or last row also stores the new value into the halo row of the
// neighbouring block (a store into that block's shared memory through the
// cluster mapping), and one cluster barrier (release / acquire) ends the
// half-sweep. The neighbour may still be running the same half-sweep while the
// store lands, but it reads only colour-(1-c) values of its halo row and the
// store writes only colour-c values, so the two never touch the same word.
// Levels 33^2 and below run in block 0 alone with the single-block cycle
// (coarse.cuh), between two cluster barriers: the blocks restrict their bands
// of the 65^2 residual straight into block 0's copy of the 33^2 right-hand
// side and later read its 33^2 solution back for the interpolation.
//
// Per V-cycle: 2 nu1 + 1 + 1 + 2 nu2 cluster barriers per distributed level
// and two around block 0's levels, against two kernel launches per level
// (plus the single-block cycle) otherwise. Every node update uses the same
// operations in the same order as the single-block cycle (cz::dense_apply,
// omega / diag once per level, the same full-weighting and interpolation
// sums), so the cycle computes what one block with enough shared memory
// would.
//
// Every block executes the same sequence of cluster barriers (the loop
// bounds are kernel arguments, the same in all blocks), and no block reads
// or writes another block's shared memory after the last barrier.
#pragma once

#include <cooperative_groups.h>

#include "coarse.cuh"

namespace mg {
namespace kz {

constexpr int kMaxCTAs = 16;     // blocks per cluster: 16, or the portable 8
constexpr int kThreads = cz::kThreads;
constexpr int kMaxDist = 3;      // distributed levels: 257^2, 129^2, 65^2
constexpr int kLocalN = 33;      // the largest level block 0 takes alone

struct ClusterArgs {
  int nctas;                          // blocks in the cluster
  int nd;                             // distributed levels (index 0 = top)
  int n[kMaxDist];                    // nodes per dimension (2^m + 1)
  int lgn[kMaxDist];                  // log2(n - 1)
  int band[kMaxDist + 1][kMaxCTAs + 1];  // level l, block r: rows [band[l][r], band[l][r+1]); l = nd: the 33^2 level
  int rmax[kMaxDist];                 // rows of the largest band of the level
  int off_u[kMaxDist];                // elements: (rmax + 2) rows of n (halo, band, halo)
  int off_f[kMaxDist];                // rmax rows of n
  int off_r[kMaxDist];                // residual: (rmax + 1) rows of n (halo above, band)
  float ih2[kMaxDist];
  float cf[2];
  float omegaf;
  int nu1, nu2;
  int off_local;                      // block 0: the single-block levels (offsets in `local` from here)
  int total;                          // elements of shared memory per block
  const void *f_top;                  // top level's right-hand side and solution (global)
  void *u_top;
  int top_dtype, pitch_top, zero_top;
  cz::CoarseArgs local;               // levels 33^2 .. coarsest
};

// The constant-stencil operator at local node p of a band array with row
// pitch n (the single-block cycle's arithmetic).
__device__ __forceinline__ cz::Lev<float> band_level(float *u, float *f, int n, float ih2) {
  cz::Lev<float> L;
  L.u = u;
  L.f = f;
  L.kx = L.ky = L.kz = nullptr;
  L.n = n;
  L.ih2 = ih2;
  return L;
}

// One red-black half-sweep of colour `color` over block r's band of level
// l; band-edge values also go to the neighbours' halo rows. U row q holds
// global row b0 - 1 + q, F row q global row b0 + q.
__device__ __forceinline__ void half_sweep(const ClusterArgs &a, cooperative_groups::cluster_group &cl, int r,
                                           int l, float *sm, int color) {
  const int n = a.n[l], b0 = a.band[l][r], R = a.band[l][r + 1] - b0;
  const int lgm = a.lgn[l] - 1, m = 1 << lgm;  // colour nodes per row, at most
  float *U = sm + a.off_u[l], *F = sm + a.off_f[l];
  const cz::Lev<float> L = band_level(U, F, n, a.ih2[l]);
  const float c[3] = {a.cf[0], a.cf[1], 0.0f};
  const float w = a.omegaf / (2.0f * (c[0] + c[1]) * L.ih2);
  float *up = nullptr, *dn = nullptr;  // the neighbours' halo rows
  if (r > 0) {
    const int Rp = b0 - a.band[l][r - 1];
    up = cl.map_shared_rank(U, r - 1) + (Rp + 1) * n;
  }
  if (r < a.nctas - 1) dn = cl.map_shared_rank(U, r + 1);
  for (int q = threadIdx.x; q < (R << lgm); q += kThreads) {
    const int jl = q >> lgm, k = q & (m - 1);
    const int j = b0 + jl;
    const int i = 2 * k + 1 + ((color + j + 1) & 1);  // (i + j) % 2 == color
    if (i > n - 2) continue;
    const int p = (jl + 1) * n + i;
    float Au, dg;
    cz::dense_apply<2, false, float>(L, U, p, c, Au, dg);
    const float v = U[p] + w * (F[jl * n + i] - Au);
    U[p] = v;
    if (jl == 0 && up) up[i] = v;
    if (jl == R - 1 && dn) dn[i] = v;
  }
  cl.sync();
}

// Residual of block r's band of level l into its residual rows 1..R; the
// band's last row also goes to the halo row of the block below. Ends with a
// cluster barrier.
__device__ __forceinline__ void residual(const ClusterArgs &a, cooperative_groups::cluster_group &cl, int r, int l,
                                         float *sm) {
  const int n = a.n[l], b0 = a.band[l][r], R = a.band[l][r + 1] - b0;
  const int lg = a.lgn[l], nn = 1 << lg;
  float *U = sm + a.off_u[l], *F = sm + a.off_f[l], *T = sm + a.off_r[l];
  const cz::Lev<float> L = band_level(U, F, n, a.ih2[l]);
  const float c[3] = {a.cf[0], a.cf[1], 0.0f};
  float *dn = r < a.nctas - 1 ? cl.map_shared_rank(T, r + 1) : nullptr;
  for (int q = threadIdx.x; q < (R << lg); q += kThreads) {
    const int jl = q >> lg, i = (q & (nn - 1)) + 1;
    if (i > n - 2) continue;
    const int p = (jl + 1) * n + i;
    float Au, dg;
    cz::dense_apply<2, false, float>(L, U, p, c, Au, dg);
    const float v = F[jl * n + i] - Au;
    T[p] = v;
    if (jl == R - 1 && dn) dn[i] = v;
  }
  cl.sync();
}

// Full weighting of level l's residual onto block r's band of level l + 1
// (its right-hand side rows; level nd: block 0's 33^2 array).
__device__ __forceinline__ void restrict_band(const ClusterArgs &a, cooperative_groups::cluster_group &cl, int r,
                                              int l, float *sm) {
  const int n = a.n[l], b0 = a.band[l][r];
  const float *T = sm + a.off_r[l];
  const int B0 = a.band[l + 1][r], RC = a.band[l + 1][r + 1] - B0;
  const int nc = (n + 1) >> 1, lgc = a.lgn[l] - 1, ncm = 1 << lgc;
  float *G;
  int pitch, row0;
  if (l + 1 < a.nd) {  // own rows of the coarse right-hand side
    G = sm + a.off_f[l + 1];
    pitch = nc;
    row0 = B0;
  } else {  // block 0's dense 33^2 right-hand side
    G = cl.map_shared_rank(sm + a.off_local + a.local.off_f[0], 0);
    pitch = nc;
    row0 = 0;
  }
  for (int q = threadIdx.x; q < (RC << lgc); q += kThreads) {
    const int J = B0 + (q >> lgc), I = (q & (ncm - 1)) + 1;
    if (I > nc - 2) continue;
    float acc = 0.0f;
    for (int dy = -1; dy <= 1; dy++) {
      const float *row = T + (2 * J + dy - b0 + 1) * n + 2 * I;  // residual row 2J + dy
      float line = 0.25f * (row[-1] + row[1]) + 0.5f * row[0];
      float wgt = dy == 0 ? 0.5f : 0.25f;
      acc += wgt * line;
    }
    G[(J - row0) * pitch + I] = acc;
  }
}

// Bilinear interpolation of the level-(l + 1) correction added to block r's
// band of level l and to its halo rows (the same sums the owners form, so
// the halo copies stay equal to them). Ends with a cluster barrier: the
// half-sweeps that follow store into the neighbours' halo rows.
__device__ __forceinline__ void prolong_band(const ClusterArgs &a, cooperative_groups::cluster_group &cl, int r,
                                             int l, float *sm) {
  const int n = a.n[l], b0 = a.band[l][r], R = a.band[l][r + 1] - b0;
  const int lg = a.lgn[l], nn = 1 << lg;
  float *U = sm + a.off_u[l];
  const int nc = (n + 1) >> 1;
  const float *E;
  int row0;
  if (l + 1 < a.nd) {  // own coarse rows with their halos: row J at E + (J - B0 + 1) nc
    E = sm + a.off_u[l + 1];
    row0 = a.band[l + 1][r] - 1;
  } else {  // block 0's dense 33^2 solution
    E = cl.map_shared_rank(sm + a.off_local + a.local.off_u[0], 0);
    row0 = 0;
  }
  for (int q = threadIdx.x; q < ((R + 2) << lg); q += kThreads) {
    const int jl = q >> lg, i = (q & (nn - 1)) + 1;
    const int j = b0 - 1 + jl;
    if (i > n - 2 || j < 1 || j > n - 2) continue;
    const int I = i >> 1, J = j >> 1, oi = i & 1, oj = j & 1;
    float acc = 0.0f;
    for (int b = 0; b <= oj; b++) {
      const float *row = E + (J + b - row0) * nc + I;
      acc += oi ? 0.5f * (row[0] + row[1]) : row[0];
    }
    const float wgt = oj ? 0.5f : 1.0f;
    U[jl * n + i] += wgt * acc;
  }
  cl.sync();
}

__global__ void __launch_bounds__(kThreads, 1) k_cluster_cycle(ClusterArgs a) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int r = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sm = (float *)smem_raw;
  for (int p = threadIdx.x; p < a.total; p += kThreads) sm[p] = 0.0f;
  __syncthreads();
  // the top level's band: right-hand side rows, and the solution rows with
  // both halo rows unless it starts from zero
  {
    const int n = a.n[0], b0 = a.band[0][r], R = a.band[0][r + 1] - b0;
    float *U = sm + a.off_u[0], *F = sm + a.off_f[0];
    for (int q = threadIdx.x; q < R * n; q += kThreads) {
      const int jl = q / n, i = q - jl * n;
      F[q] = cz::ldg_as<float>(a.f_top, (long long)(b0 + jl) * a.pitch_top + i, a.top_dtype);
    }
    if (!a.zero_top) {
      for (int q = threadIdx.x; q < (R + 2) * n; q += kThreads) {
        const int jl = q / n, i = q - jl * n;
        U[q] = cz::ldg_as<float>(a.u_top, (long long)(b0 - 1 + jl) * a.pitch_top + i, a.top_dtype);
      }
    }
  }
  // every block has cleared its shared memory before any block stores into it
  cl.sync();
  // descend: pre-smoothing, residual, restriction
  for (int l = 0; l < a.nd; l++) {
    for (int s = 0; s < a.nu1; s++) {
      half_sweep(a, cl, r, l, sm, 0);
      half_sweep(a, cl, r, l, sm, 1);
    }
    residual(a, cl, r, l, sm);
    restrict_band(a, cl, r, l, sm);
    __syncthreads();
  }
  // block 0's levels; the other blocks wait at the barrier
  cl.sync();
  if (r == 0) cz::cycle_in_smem<2, false, float>(a.local, sm + a.off_local);
  cl.sync();
  // ascend: interpolation and correction, post-smoothing
  for (int l = a.nd - 1; l >= 0; l--) {
    prolong_band(a, cl, r, l, sm);
    for (int s = 0; s < a.nu2; s++) {
      half_sweep(a, cl, r, l, sm, 0);
      half_sweep(a, cl, r, l, sm, 1);
    }
  }
  // the band's solution rows back to the top level's global array
  {
    const int n = a.n[0], b0 = a.band[0][r], R = a.band[0][r + 1] - b0;
    const float *U = sm + a.off_u[0];
    for (int q = threadIdx.x; q < R * n; q += kThreads) {
      const int jl = q / n, i = q - jl * n;
      if (i >= 1 && i <= n - 2) cz::stg_as<float>(a.u_top, (long long)(b0 + jl) * a.pitch_top + i, a.top_dtype, U[(jl + 1) * n + i]);
    }
  }
  cl.sync();
}

}  // namespace kz
}  // namespace mg
