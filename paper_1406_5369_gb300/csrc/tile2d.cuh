// Block-tile kernels for the small fine levels of the 2D V-cycle (Algorithm 1,
// constant stencil, red-black Gauss-Seidel): the same two fused passes as
// fused2d.cuh, k_pre2d (nu1 sweeps + residual + full weighting) and k_post2d
// (interpolation and correction + nu2 sweeps), for levels small enough that
// the row-streaming kernels are bound by the latency of their warps' long
// row walks rather than by bandwidth.
//
// A block of 256 threads owns a tile of kTH x kTW output nodes. It loads the
// tile with a halo of H nodes into shared memory in one pass (every load in
// flight at once), runs the red-black half-sweeps there with a block barrier
// between them - half-sweep h updates the nodes of its colour at distance
// >= h from the loaded edge, whose neighbours the previous half-sweep left
// exact, so after 2 nu half-sweeps every node at distance >= 2 nu is exactly
// what a sequential red-then-black sweep of the whole grid gives - and writes
// its output nodes. The pre-smoothing pass also forms the residual on the
// tile plus one node (H = 2 nu + 2) and restricts it by full weighting to the
// coarse nodes whose fine centre lies in the tile. Reads come from the input
// buffer and writes go to the other ping-pong buffer, so neighbouring blocks
// see the unsmoothed values they recompute.
#pragma once

#include "fused2d.cuh"

namespace mg {
namespace tz {

constexpr int kTW = 64;        // output columns per tile (even)
constexpr int kTH = 32;        // output rows per tile (even)
constexpr int kThreads = 256;  // 8 warps

template <int NU> struct PreGeo {
  static constexpr int H = 2 * NU + 2;
  static constexpr int LW = kTW + 2 * H, LH = kTH + 2 * H;
  static constexpr int RW = kTW + 2, RH = kTH + 2;  // residual: tile plus one node
  static constexpr int elems = 2 * LW * LH + RW * RH;
};
template <int NU> struct PostGeo {
  static constexpr int H = 2 * NU;
  static constexpr int LW = kTW + 2 * H, LH = kTH + 2 * H;
  static constexpr int CW = LW / 2 + 2, CH = LH / 2 + 2;  // coarse nodes under the loaded region
  static constexpr int elems = 2 * LW * LH + CW * CH;
};

// Half-sweep h (colour (h - 1) & 1) on the loaded region shrunk by h: warp w
// takes rows h + w, h + w + 8, ...; lane l the colour's nodes 2l, 2l + 64, ...
// of the row. Only interior grid nodes change.
template <typename C, int LW, int LH>
__device__ __forceinline__ void tile_half_sweep(C *su, const C *sf, int h, int gx0, int gy0, int n,
                                                const fz::Coef<C> &k) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int color = (h - 1) & 1;
  for (int ly = h + w; ly < LH - h; ly += kThreads / 32) {
    const int gy = gy0 + ly;
    if (gy < 1 || gy > n - 2) continue;
    const int lx0 = h + ((color - gx0 - gy - h) & 1);  // (gx0 + lx + gy) % 2 == colour
    for (int lx = lx0 + 2 * lane; lx < LW - h; lx += 64) {
      const int gx = gx0 + lx;
      if (gx < 1 || gx > n - 2) continue;
      const int p = ly * LW + lx;
      C v = k.alpha * sf[p] + k.bx * (su[p - 1] + su[p + 1]) + k.by * (su[p - LW] + su[p + LW]);
      if (k.has_gamma) v += k.gamma * su[p];
      su[p] = v;
    }
  }
}

template <typename T, int NU, bool ZERO>
__global__ void __launch_bounds__(kThreads) k_tpre2d(fz::Args2D a) {
  typedef typename CT<T>::type C;
  typedef PreGeo<NU> G;
  constexpr int H = G::H, LW = G::LW, LH = G::LH, RW = G::RW, RH = G::RH;
  extern __shared__ __align__(16) unsigned char smem[];
  C *su = (C *)smem;
  C *sf = su + LW * LH;
  C *sr = sf + LW * LH;
  const int n = a.n;
  const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
  const int gx0 = x0 - H, gy0 = y0 - H;
  const T *uin = (const T *)a.uin;
  const T *f = (const T *)a.f;
  T *uout = (T *)a.uout;
  T *fc = (T *)a.fc;
  const fz::Coef<C> k = fz::coef_of<C>(a);

  for (int i = threadIdx.x; i < LW * LH; i += kThreads) {
    const int ly = i / LW, lx = i - ly * LW;
    const int gx = gx0 + lx, gy = gy0 + ly;
    const bool in = gx >= 0 && gx < n && gy >= 0 && gy < n;
    const long long g = (long long)gy * a.pitch + gx;
    su[i] = (!ZERO && in) ? (C)ld(uin + g) : (C)0;
    sf[i] = in ? (C)ld(f + g) : (C)0;
  }
  __syncthreads();
  for (int h = 1; h <= 2 * NU; h++) {
    tile_half_sweep<C, LW, LH>(su, sf, h, gx0, gy0, n, k);
    __syncthreads();
  }
  // residual on the tile plus one node; smoothed u of the tile
  for (int i = threadIdx.x; i < RW * RH; i += kThreads) {
    const int ry = i / RW, rx = i - ry * RW;
    const int ly = ry + H - 1, lx = rx + H - 1;
    const int gx = gx0 + lx, gy = gy0 + ly;
    C r = (C)0;
    if (gx >= 1 && gx <= n - 2 && gy >= 1 && gy <= n - 2) {
      const int p = ly * LW + lx;
      const C u = su[p], uw = su[p - 1], ue = su[p + 1], us = su[p - LW], un = su[p + LW];
      if (sizeof(C) == 8) r = sf[p] - (k.cx * ((u - uw) + (u - ue)) + k.cy * ((u - us) + (u - un)));
      else r = k.cy * (us + un) + (k.cx * (uw + ue) + (sf[p] - k.cd * u));
      if (rx >= 1 && rx <= kTW && ry >= 1 && ry <= kTH) st(uout + (long long)gy * a.pitch + gx, u);
    }
    sr[i] = r;
  }
  __syncthreads();
  // full weighting to the coarse nodes whose fine centre (2I, 2J) is in the tile
  for (int i = threadIdx.x; i < (kTH / 2) * (kTW / 2); i += kThreads) {
    const int cyi = i / (kTW / 2), cxi = i - cyi * (kTW / 2);
    const int I = (y0 >> 1) + cyi, J = (x0 >> 1) + cxi;
    if (I < 1 || I > a.nc - 2 || J < 1 || J > a.nc - 2) continue;
    const C *r = sr + (2 * cyi + 1) * RW + 2 * cxi + 1;
    const C hA = r[-RW - 1] + (C)2 * r[-RW] + r[-RW + 1];
    const C hB = r[-1] + (C)2 * r[0] + r[1];
    const C hC = r[RW - 1] + (C)2 * r[RW] + r[RW + 1];
    st(fc + (long long)I * a.pitchc + J, (hA + (C)2 * hB + hC) * (C)0.0625);
  }
}

template <typename T, int NU>
__global__ void __launch_bounds__(kThreads) k_tpost2d(fz::Args2D a) {
  typedef typename CT<T>::type C;
  typedef PostGeo<NU> G;
  constexpr int H = G::H, LW = G::LW, LH = G::LH, CW = G::CW, CH = G::CH;
  extern __shared__ __align__(16) unsigned char smem[];
  C *su = (C *)smem;
  C *sf = su + LW * LH;
  C *se = sf + LW * LH;
  const int n = a.n, nc = a.nc;
  const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
  const int gx0 = x0 - H, gy0 = y0 - H;
  const int cx0 = gx0 >> 1, cy0 = gy0 >> 1;  // floor: first coarse column/row under the region
  const T *uin = (const T *)a.uin;
  const T *f = (const T *)a.f;
  const T *ec = (const T *)a.ec;
  T *uout = (T *)a.uout;
  const fz::Coef<C> k = fz::coef_of<C>(a);

  for (int i = threadIdx.x; i < LW * LH; i += kThreads) {
    const int ly = i / LW, lx = i - ly * LW;
    const int gx = gx0 + lx, gy = gy0 + ly;
    const bool in = gx >= 0 && gx < n && gy >= 0 && gy < n;
    const long long g = (long long)gy * a.pitch + gx;
    su[i] = in ? (C)ld(uin + g) : (C)0;
    sf[i] = in ? (C)ld(f + g) : (C)0;
  }
  for (int i = threadIdx.x; i < CW * CH; i += kThreads) {
    const int cyi = i / CW, cxi = i - cyi * CW;
    const int J = cx0 + cxi, I = cy0 + cyi;
    const bool in = J >= 0 && J < nc && I >= 0 && I < nc;
    se[i] = in ? (C)ld(ec + (long long)I * a.pitchc + J) : (C)0;
  }
  __syncthreads();
  // bilinear interpolation and correction at interior nodes of the region
  for (int i = threadIdx.x; i < LW * LH; i += kThreads) {
    const int ly = i / LW, lx = i - ly * LW;
    const int gx = gx0 + lx, gy = gy0 + ly;
    if (gx < 1 || gx > n - 2 || gy < 1 || gy > n - 2) continue;
    const C *e = se + ((gy >> 1) - cy0) * CW + ((gx >> 1) - cx0);
    const bool oj = gy & 1;
    const C e0 = oj ? (C)0.5 * (e[0] + e[CW]) : e[0];
    C v = e0;
    if (gx & 1) {
      const C e1 = oj ? (C)0.5 * (e[1] + e[CW + 1]) : e[1];
      v = (C)0.5 * (e0 + e1);
    }
    su[i] += v;
  }
  __syncthreads();
  for (int h = 1; h <= 2 * NU; h++) {
    tile_half_sweep<C, LW, LH>(su, sf, h, gx0, gy0, n, k);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kTW * kTH; i += kThreads) {
    const int oy = i / kTW, ox = i - oy * kTW;
    const int gx = x0 + ox, gy = y0 + oy;
    if (gx >= 1 && gx <= n - 2 && gy >= 1 && gy <= n - 2)
      st(uout + (long long)gy * a.pitch + gx, su[(oy + H) * LW + ox + H]);
  }
}

}  // namespace tz
}  // namespace mg
