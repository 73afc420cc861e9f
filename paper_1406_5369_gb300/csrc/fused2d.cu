// Launchers of the fused 2D fine-level kernels (fused2d.cuh).
#include <string.h>

#include "fused2d.cuh"
#include "fused2d_x2.cuh"
#include "fused2d_x2v.cuh"
#include "tile2d.cuh"

namespace mg {
namespace d2 {

namespace {

template <typename KernelT>
cudaError_t prepare(KernelT kernel, size_t smem) {
  // Opt in to more than 48 KB of dynamic shared memory once per kernel.
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int sm_count() {
  static int count = 0;
  if (!count) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    if (count <= 0) count = 152;
  }
  return count;
}

// Rows per chunk: as many chunks as fill one wave of resident warps,
// rounded up to a multiple of 8. Small levels get 8-row chunks: each warp
// then walks only 3 blocks of 8 rows, which keeps their latency short.
// Rows per chunk of a list launch (many problems): the problems supply the
// parallelism, so chunks are long (little of the 8-row warm-up is repeated)
// and depend on the level size alone.
constexpr int kListRows = 256;

int pick_rows(int n, int nstrips, int blocks_per_sm, int warps_per_block, int R_override) {
  if (R_override > 0) return (R_override + 7) / 8 * 8;
  long long slots = (long long)sm_count() * blocks_per_sm * warps_per_block;
  long long nchunks = slots / nstrips;
  if (nchunks < 1) nchunks = 1;
  int R = (int)((n + nchunks - 1) / nchunks);
  R = (R + 7) / 8 * 8;
  if (R < 8) R = 8;
  return R;
}

fz::Args2D make_args(const Level &L, const Level &Cl, double omega, int R_override, int blocks_per_sm) {
  fz::Args2D a;
  memset(&a, 0, sizeof a);
  a.n = L.n;
  a.pitch = L.pitch;
  a.nc = Cl.n;
  a.pitchc = Cl.pitch;
  a.nstrips = (L.n + fz::kOut - 1) / fz::kOut;
  a.R = pick_rows(L.n, a.nstrips, blocks_per_sm, 1, R_override);
  a.nchunks = (L.n + a.R - 1) / a.R;
  double cx = L.c[0] * L.inv_h2, cy = L.c[1] * L.inv_h2;
  double diag = 2.0 * (cx + cy);
  a.alpha = omega / diag;
  a.betax = omega * cx / diag;
  a.betay = omega * cy / diag;
  a.gamma = 1.0 - omega;
  a.cx = cx;
  a.cy = cy;
  a.cd = 2.0 * (cx + cy);
  a.alphaf = (float)a.alpha;
  a.betaxf = (float)a.betax;
  a.betayf = (float)a.betay;
  a.gammaf = (float)a.gamma;
  a.cxf = (float)a.cx;
  a.cyf = (float)a.cy;
  a.cdf = (float)a.cd;
  a.has_gamma = a.gamma != 0.0;
  a.kx = L.kf[0];
  a.ky = L.kf[1];
  a.omega = omega;
  a.h2 = 1.0 / L.inv_h2;
  a.ih2 = L.inv_h2;
  a.omegaf = (float)a.omega;
  a.h2f = (float)a.h2;
  a.ih2f = (float)a.ih2;
  return a;
}

template <typename T, int NU, bool ZERO>
cudaError_t launch_pre(fz::Args2D a, int R_override, const Level &L, cudaStream_t s, const fz::Args2D *list = nullptr,
                       int count = 1) {
  constexpr int W = fz::Warps<T>::value;
  constexpr size_t smem = (size_t)W * fz::kRing * 32 * fz::Lane<T>::bytes * (ZERO ? 1 : 2);
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_pre2d<T, NU, ZERO>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_pre2d<T, NU, ZERO>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, list ? kListRows : 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  fz::k_pre2d<T, NU, ZERO><<<dim3(blocks, (unsigned)count), 32 * W, smem, s>>>(a, list);
  return cudaGetLastError();
}

template <typename T, int NU>
cudaError_t launch_post(fz::Args2D a, int R_override, const Level &L, cudaStream_t s, const fz::Args2D *list = nullptr,
                        int count = 1) {
  constexpr int W = fz::Warps<T>::value;
  constexpr size_t smem = (size_t)W * fz::kRing * 32 * (2 * fz::Lane<T>::bytes + 2 * sizeof(T));
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_post2d<T, NU>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_post2d<T, NU>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, list ? kListRows : 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  fz::k_post2d<T, NU><<<dim3(blocks, (unsigned)count), 32 * W, smem, s>>>(a, list);
  return cudaGetLastError();
}

// Block-tile kernels (tile2d.cuh) for constant-stencil levels up to this size
// (mg_options.tile_max_n overrides it): below it the streaming kernels' warps
// walk too few rows in parallel for the grid to be bandwidth-bound, and a
// tile pass costs a handful of barriers. 257 is what the autotuner picks on
// the GB300 for the 8193^2 workload.
constexpr int kTileMaxN = 257;

bool tile_ok(const Level &L, int tile_max_n) {
  return !L.kf[0] && L.n <= (tile_max_n > 0 ? tile_max_n : kTileMaxN);
}

template <typename T, int NU, bool ZERO> cudaError_t launch_tpre(const fz::Args2D &a, const Level &L, cudaStream_t s) {
  constexpr size_t smem = sizeof(typename CT<T>::type) * tz::PreGeo<NU>::elems;
  static bool ready = false;
  if (!ready) {
    cudaError_t e = prepare(tz::k_tpre2d<T, NU, ZERO>, smem);
    if (e != cudaSuccess) return e;
    ready = true;
  }
  const dim3 g((unsigned)((L.n + tz::kTW - 1) / tz::kTW), (unsigned)((L.n + tz::kTH - 1) / tz::kTH));
  tz::k_tpre2d<T, NU, ZERO><<<g, tz::kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int NU> cudaError_t launch_tpost(const fz::Args2D &a, const Level &L, cudaStream_t s) {
  constexpr size_t smem = sizeof(typename CT<T>::type) * tz::PostGeo<NU>::elems;
  static bool ready = false;
  if (!ready) {
    cudaError_t e = prepare(tz::k_tpost2d<T, NU>, smem);
    if (e != cudaSuccess) return e;
    ready = true;
  }
  const dim3 g((unsigned)((L.n + tz::kTW - 1) / tz::kTW), (unsigned)((L.n + tz::kTH - 1) / tz::kTH));
  tz::k_tpost2d<T, NU><<<g, tz::kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t dispatch_tpre(const fz::Args2D &a, const Level &L, cudaStream_t s, bool zero, int nu) {
  if (L.dtype == F32) {
    if (nu == 1) return zero ? launch_tpre<float, 1, true>(a, L, s) : launch_tpre<float, 1, false>(a, L, s);
    return zero ? launch_tpre<float, 2, true>(a, L, s) : launch_tpre<float, 2, false>(a, L, s);
  }
  if (nu == 1) return zero ? launch_tpre<double, 1, true>(a, L, s) : launch_tpre<double, 1, false>(a, L, s);
  return zero ? launch_tpre<double, 2, true>(a, L, s) : launch_tpre<double, 2, false>(a, L, s);
}

cudaError_t dispatch_tpost(const fz::Args2D &a, const Level &L, cudaStream_t s, int nu) {
  if (L.dtype == F32) return nu == 1 ? launch_tpost<float, 1>(a, L, s) : launch_tpost<float, 2>(a, L, s);
  return nu == 1 ? launch_tpost<double, 1>(a, L, s) : launch_tpost<double, 2>(a, L, s);
}

// The packed-FP32 fused kernels (fused2d_x2.cuh), constant stencil; G: the
// relaxation term (1 - omega) u is present (omega != 1).
template <int NU, bool ZERO, bool G>
cudaError_t launch_pre_x2(fz::Args2D a, int R_override, const Level &L, cudaStream_t s, const fz::Args2D *list,
                          int count) {
  constexpr int W = 4;
  constexpr size_t smem = (size_t)W * fz::kRing * 32 * 16 * 2;
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_pre2d_x2<NU, ZERO, false, G>, smem);
    if (e == cudaSuccess) e = prepare(fz::k_pre2d_x2<NU, ZERO, true, G>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_pre2d_x2<NU, ZERO, false, G>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, list ? kListRows : 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  if (list)
    fz::k_pre2d_x2<NU, ZERO, true, G><<<dim3(blocks, (unsigned)count), 32 * W, smem, s>>>(a, list);
  else
    fz::k_pre2d_x2<NU, ZERO, false, G><<<blocks, 32 * W, smem, s>>>(a, nullptr);
  return cudaGetLastError();
}

template <int NU, bool G>
cudaError_t launch_post_x2(fz::Args2D a, int R_override, const Level &L, cudaStream_t s, const fz::Args2D *list,
                           int count) {
  constexpr int W = 4;
  constexpr size_t smem = (size_t)W * fz::kRing * 32 * (16 + 16 + 8);
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_post2d_x2<NU, false, G>, smem);
    if (e == cudaSuccess) e = prepare(fz::k_post2d_x2<NU, true, G>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_post2d_x2<NU, false, G>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, list ? kListRows : 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  if (list)
    fz::k_post2d_x2<NU, true, G><<<dim3(blocks, (unsigned)count), 32 * W, smem, s>>>(a, list);
  else
    fz::k_post2d_x2<NU, false, G><<<blocks, 32 * W, smem, s>>>(a, nullptr);
  return cudaGetLastError();
}

// Post-smoothing of one cycle fused with the pre-smoothing of the next
// (k_postpre2d_x2), single problem.
template <int NUA, int NUB, bool G>
cudaError_t launch_postpre_x2(fz::Args2D a, int R_override, const Level &L, cudaStream_t s) {
  constexpr int W = 4;
  constexpr size_t smem = (size_t)W * fz::kPS * 32 * (16 + 16 + 8);
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_postpre2d_x2<NUA, NUB, G>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_postpre2d_x2<NUA, NUB, G>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  fz::k_postpre2d_x2<NUA, NUB, G><<<blocks, 32 * W, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NUA, int NUB>
cudaError_t postpre_x2(const fz::Args2D &a, int R, const Level &L, cudaStream_t s) {
  return a.has_gamma ? launch_postpre_x2<NUA, NUB, true>(a, R, L, s) : launch_postpre_x2<NUA, NUB, false>(a, R, L, s);
}

// The packed FP32 variable-stencil pre-smoothing pass (fused2d_x2v.cuh).
template <int NU, bool ZERO>
cudaError_t launch_pre_x2v(fz::Args2D a, int R_override, const Level &L, cudaStream_t s, const fz::Args2D *list,
                           int count) {
  constexpr int W = 2;
  constexpr size_t smem = (size_t)W * fz::X2VSmem<ZERO>::WB;
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_pre2d_x2v<NU, ZERO, false>, smem);
    if (e == cudaSuccess) e = prepare(fz::k_pre2d_x2v<NU, ZERO, true>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_pre2d_x2v<NU, ZERO, false>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, list ? kListRows : 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  if (list)
    fz::k_pre2d_x2v<NU, ZERO, true><<<dim3(blocks, (unsigned)count), 32 * W, smem, s>>>(a, list);
  else
    fz::k_pre2d_x2v<NU, ZERO, false><<<blocks, 32 * W, smem, s>>>(a, nullptr);
  return cudaGetLastError();
}

// The packed FP32 variable-stencil post-smoothing pass (fused2d_x2v.cuh).
template <int NU>
cudaError_t launch_post_x2v(fz::Args2D a, int R_override, const Level &L, cudaStream_t s, const fz::Args2D *list,
                            int count) {
  constexpr int W = 2;
  constexpr size_t smem = (size_t)W * fz::kX2VPostWB;
  static bool ready = false;
  static int bps = 1;
  if (!ready) {
    cudaError_t e = prepare(fz::k_post2d_x2v<NU, false>, smem);
    if (e == cudaSuccess) e = prepare(fz::k_post2d_x2v<NU, true>, smem);
    if (e != cudaSuccess) return e;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fz::k_post2d_x2v<NU, false>, 32 * W, smem);
    if (bps < 1) bps = 1;
    ready = true;
  }
  if (R_override <= 0) {
    a.R = pick_rows(L.n, a.nstrips, bps, W, list ? kListRows : 0);
    a.nchunks = (L.n + a.R - 1) / a.R;
  }
  long long warps = (long long)a.nstrips * a.nchunks;
  unsigned blocks = (unsigned)((warps + W - 1) / W);
  if (list)
    fz::k_post2d_x2v<NU, true><<<dim3(blocks, (unsigned)count), 32 * W, smem, s>>>(a, list);
  else
    fz::k_post2d_x2v<NU, false><<<blocks, 32 * W, smem, s>>>(a, nullptr);
  return cudaGetLastError();
}

template <int NU, bool ZERO>
cudaError_t pre_x2(const fz::Args2D &a, int R, const Level &L, cudaStream_t s, const fz::Args2D *list, int count) {
  return a.has_gamma ? launch_pre_x2<NU, ZERO, true>(a, R, L, s, list, count)
                     : launch_pre_x2<NU, ZERO, false>(a, R, L, s, list, count);
}
template <int NU>
cudaError_t post_x2(const fz::Args2D &a, int R, const Level &L, cudaStream_t s, const fz::Args2D *list, int count) {
  return a.has_gamma ? launch_post_x2<NU, true>(a, R, L, s, list, count)
                     : launch_post_x2<NU, false>(a, R, L, s, list, count);
}

// Storage type, sweep count, zero start and stencil kind -> kernel instance.
cudaError_t dispatch_pre(fz::Args2D a, int R, const Level &L, cudaStream_t s, const fz::Args2D *list, int count,
                         bool zero, int nu) {
  const bool var = L.kf[0] != nullptr;
  if (L.dtype == F32 && !var) {
    if (nu == 1) return zero ? pre_x2<1, true>(a, R, L, s, list, count) : pre_x2<1, false>(a, R, L, s, list, count);
    return zero ? pre_x2<2, true>(a, R, L, s, list, count) : pre_x2<2, false>(a, R, L, s, list, count);
  }
  if (L.dtype == F32) {
    // variable stencil: the packed instance
    if (nu == 1) return zero ? launch_pre_x2v<1, true>(a, R, L, s, list, count) : launch_pre_x2v<1, false>(a, R, L, s, list, count);
    return zero ? launch_pre_x2v<2, true>(a, R, L, s, list, count) : launch_pre_x2v<2, false>(a, R, L, s, list, count);
  }
  if (nu == 1) return zero ? launch_pre<double, 1, true>(a, R, L, s, list, count) : launch_pre<double, 1, false>(a, R, L, s, list, count);
  return zero ? launch_pre<double, 2, true>(a, R, L, s, list, count) : launch_pre<double, 2, false>(a, R, L, s, list, count);
}

cudaError_t dispatch_post(fz::Args2D a, int R, const Level &L, cudaStream_t s, const fz::Args2D *list, int count,
                          int nu) {
  const bool var = L.kf[0] != nullptr;
  if (L.dtype == F32 && !var)
    return nu == 1 ? post_x2<1>(a, R, L, s, list, count) : post_x2<2>(a, R, L, s, list, count);
  if (L.dtype == F32) {
    // variable stencil: the packed instance
    return nu == 1 ? launch_post_x2v<1>(a, R, L, s, list, count) : launch_post_x2v<2>(a, R, L, s, list, count);
  }
  return nu == 1 ? launch_post<double, 1>(a, R, L, s, list, count) : launch_post<double, 2>(a, R, L, s, list, count);
}

}  // namespace

// Constant stencil in FP64 or FP32; variable stencil in FP32 (the packed
// kernels of fused2d_x2v.cuh, faces stored in FP32); FP64 variable-stencil
// levels keep the generic kernels.
bool fused_ok(const Level &L, const Level &Cl, int nu) {
  return L.dim == 2 && (L.dtype == F64 || L.dtype == F32) && (!L.kf[0] || L.dtype == F32) && Cl.dtype == L.dtype &&
         (nu == 1 || nu == 2) && L.n >= 33;
}

cudaError_t pre_fused(const Level &L, const void *uin, void *uout, const Level &Cl, void *fc, bool zero, int nu,
                      double omega, int R, int tile_max_n, cudaStream_t s) {
  fz::Args2D a = make_args(L, Cl, omega, R, 1);
  a.uin = uin;
  a.f = L.f;
  a.uout = uout;
  a.fc = fc;
  if (tile_ok(L, tile_max_n)) return dispatch_tpre(a, L, s, zero, nu);
  return dispatch_pre(a, R, L, s, nullptr, 1, zero, nu);
}

bool postpre_ok(const Level &L, const Level &Cl, int nu2, int nu1, int tile_max_n) {
  return L.dim == 2 && L.dtype == F32 && !L.kf[0] && Cl.dtype == F32 && nu2 >= 1 && nu1 >= 1 && nu2 + nu1 <= 3 &&
         L.n >= 33 && !tile_ok(L, tile_max_n);
}

cudaError_t postpre_fused(const Level &L, const void *uin, void *uout, const Level &Cl, const void *ec, void *fc,
                          int nu2, int nu1, double omega, int R, int tile_max_n, cudaStream_t s) {
  if (!postpre_ok(L, Cl, nu2, nu1, tile_max_n)) return cudaErrorInvalidValue;
  fz::Args2D a = make_args(L, Cl, omega, R, 1);
  a.uin = uin;
  a.f = L.f;
  a.uout = uout;
  a.ec = ec;
  a.fc = fc;
  if (nu2 == 1 && nu1 == 2) return postpre_x2<1, 2>(a, R, L, s);
  if (nu2 == 2 && nu1 == 1) return postpre_x2<2, 1>(a, R, L, s);
  return postpre_x2<1, 1>(a, R, L, s);
}

cudaError_t post_fused(const Level &L, const void *uin, void *uout, const Level &Cl, const void *ec, int nu,
                       double omega, int R, int tile_max_n, cudaStream_t s) {
  fz::Args2D a = make_args(L, Cl, omega, R, 1);
  a.uin = uin;
  a.f = L.f;
  a.uout = uout;
  a.ec = ec;
  if (tile_ok(L, tile_max_n)) return dispatch_tpost(a, L, s, nu);
  return dispatch_post(a, R, L, s, nullptr, 1, nu);
}

}  // namespace d2
}  // namespace mg

namespace mg {
namespace d2 {

fz::Args2D fused_record(const Level &L, const Level &Cl, double omega, const void *uin, void *uout, const void *ec,
                        void *fc) {
  fz::Args2D a = make_args(L, Cl, omega, 0, 1);
  a.uin = uin;
  a.f = L.f;
  a.uout = uout;
  a.ec = ec;
  a.fc = fc;
  return a;
}

cudaError_t pre_fused_list(const Level &L, const Level &Cl, const fz::Args2D *list, int count, bool zero, int nu,
                           int rows, cudaStream_t s) {
  fz::Args2D a = make_args(L, Cl, 1.0, rows, 1);
  return dispatch_pre(a, rows, L, s, list, count, zero, nu);
}

cudaError_t post_fused_list(const Level &L, const Level &Cl, const fz::Args2D *list, int count, int nu, int rows,
                            cudaStream_t s) {
  fz::Args2D a = make_args(L, Cl, 1.0, rows, 1);
  return dispatch_post(a, rows, L, s, list, count, nu);
}

}  // namespace d2
}  // namespace mg
