// Launchers of the plane-marching 3D kernels (stencil3d.cuh) for
// constant-stencil levels.
#include <string.h>

#include <algorithm>

#include "stencil3d.cuh"

namespace mg {
namespace d3 {

namespace {

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

// Resident blocks per SM of a kernel (queried once per kernel).
template <typename K> int resident(K kernel, int threads, size_t smem, int *cache) {
  if (*cache == 0) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem);
    *cache = b > 0 ? b : 1;
  }
  return *cache;
}

// Planes per z-chunk of a single-problem launch, for kernels whose blocks
// walk their chunk plus two extra planes: the chunk count that minimises
// (waves of resident blocks) x (planes per block), waves rounded up, so that
// the last wave is not a nearly empty one; chunks of at least 8 planes and no
// more than `max_blocks` blocks.
int pick_zc_waves(int n, long long base_blocks, int per_sm, long long max_blocks) {
  const int planes = n - 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)std::max(sms, 1) * std::max(per_sm, 1);
  long long best_cost = -1;
  int best = planes;
  for (int nz = 1; nz <= 64; nz++) {
    const int zc = (planes + nz - 1) / nz;
    if (nz > 1 && zc < 8) break;
    const int nzr = (planes + zc - 1) / zc;
    if (base_blocks * nzr > max_blocks) break;
    const long long waves = (base_blocks * nzr + slots - 1) / slots;
    const long long cost = waves * (zc + 2);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}

// Planes per z-chunk: enough chunks for about two waves of resident blocks,
// at least 8 planes each, and no more than `max_blocks` blocks in total.
// list: a launch over many problems, which supply the parallelism: chunks of
// about 64 planes, a function of the size alone.
int pick_zc(int n, long long base_blocks, int per_sm, long long max_blocks, bool list = false) {
  const int planes = n - 2;
  long long want = 2LL * sm_count() * per_sm;
  long long nz = list ? (planes + 63) / 64 : (want + base_blocks - 1) / base_blocks;
  if (nz > planes / 8) nz = planes / 8;
  if (nz * base_blocks > max_blocks) nz = max_blocks / base_blocks;
  if (nz < 1) nz = 1;
  return (int)((planes + nz - 1) / nz);
}

z3::Args3 stencil_args(const Level &L, double omega) {
  z3::Args3 a;
  memset(&a, 0, sizeof a);
  a.n = L.n;
  a.pitch = L.pitch;
  a.plane = L.plane;
  double cx = L.c[0] * L.inv_h2, cy = L.c[1] * L.inv_h2, cz = L.c[2] * L.inv_h2;
  double diag = 2.0 * (cx + cy + cz);
  a.alpha = omega / diag;
  a.bx = omega * cx / diag;
  a.by = omega * cy / diag;
  a.bz = omega * cz / diag;
  a.gamma = 1.0 - omega;
  a.cd = diag;
  a.cx = cx;
  a.cy = cy;
  a.cz = cz;
  a.alphaf = (float)a.alpha;
  a.bxf = (float)a.bx;
  a.byf = (float)a.by;
  a.bzf = (float)a.bz;
  a.gammaf = (float)a.gamma;
  a.cdf = (float)a.cd;
  a.cxf = (float)a.cx;
  a.cyf = (float)a.cy;
  a.czf = (float)a.cz;
  a.has_gamma = a.gamma != 0.0;
  a.color = -1;
  return a;
}

template <typename T, int MODE>
cudaError_t launch_stencil(z3::Args3 a, long long max_blocks, int *nblocks, cudaStream_t s,
                           const z3::Args3 *list = nullptr, int count = 1) {
  constexpr int V = z3::VW<T>::V;
  constexpr size_t smem = (size_t)z3::kRingZ * z3::kSlotB;
  static int per_sm = 0;
  int r = resident(z3::k3_stencil<T, MODE>, 32 * z3::kTY, smem, &per_sm);
  a.ntx = (a.n - 1 + 32 * V - 1) / (32 * V);
  a.nty = (a.n - 2 + z3::kTY - 1) / z3::kTY;
  long long base = (long long)a.ntx * a.nty;
  a.zc = pick_zc(a.n, base, r, max_blocks, list != nullptr);
  int nz = (a.n - 2 + a.zc - 1) / a.zc;
  if (nblocks) *nblocks = (int)(base * nz);
  z3::k3_stencil<T, MODE><<<dim3((unsigned)base, (unsigned)nz, (unsigned)count), 32 * z3::kTY, smem, s>>>(a, list);
  return cudaGetLastError();
}

#define Z3_DISPATCH(dtype, ...)                             \
  switch (dtype) {                                          \
    case F64: { typedef double T; __VA_ARGS__; } break;     \
    case F32: { typedef float T; __VA_ARGS__; } break;      \
    default: { typedef bf16 T; __VA_ARGS__; } break;        \
  }

}  // namespace

bool z_ok(const Level &L) { return L.dim == 3 && !L.kf[0] && L.n >= 5; }

cudaError_t z_sweep(const Level &L, const void *uin, void *uout, const void *f, int color, double omega,
                    cudaStream_t s) {
  z3::Args3 a = stencil_args(L, omega);
  a.u = uin;
  a.out = uout;
  a.f = f;
  a.color = color;
  cudaError_t e = cudaSuccess;
  if (color < 0) {
    Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kJacobi>(a, 1LL << 30, nullptr, s)));
  } else {
    Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kRB>(a, 1LL << 30, nullptr, s)));
  }
  return e;
}

cudaError_t z_jacobi_zero2(const Level &L, const void *f, void *uout, double omega, cudaStream_t s) {
  z3::Args3 a = stencil_args(L, omega);
  a.u = f;  // staged in place of u; the kernel scales it by alpha (the first sweep from zero)
  a.out = uout;
  a.f = f;
  cudaError_t e = cudaSuccess;
  Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kJZ>(a, 1LL << 30, nullptr, s)));
  return e;
}

cudaError_t z_residual(const Level &L, const void *u, const void *f, void *r, cudaStream_t s) {
  z3::Args3 a = stencil_args(L, 1.0);
  a.u = u;
  a.out = r;
  a.f = f;
  cudaError_t e = cudaSuccess;
  Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kResid>(a, 1LL << 30, nullptr, s)));
  return e;
}

bool norm_ok(const Level &L) { return z_ok(L); }

cudaError_t norm_stream(const Level &L, const void *u, const void *f, double *partials, int *nparts, cudaStream_t s) {
  z3::Args3 a = stencil_args(L, 1.0);
  a.u = u;
  a.f = f;
  a.partials = partials;
  cudaError_t e = cudaSuccess;
  Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kNorm>(a, kMaxPartials, nparts, s)));
  return e;
}

bool transfer_ok(const Level &F, const Level &C) { return z_ok(F) && C.dtype == F.dtype && C.n >= 3; }

cudaError_t z_restrict(const Level &F, const void *rf, const Level &C, void *fc, cudaStream_t s) {
  z3::ArgsT3 a;
  memset(&a, 0, sizeof a);
  a.src = rf;
  a.dst = fc;
  a.nf = F.n; a.pitchf = F.pitch; a.planef = F.plane;
  a.nc = C.n; a.pitchc = C.pitch; a.planec = C.plane;
  if (C.n < 3) return cudaSuccess;
  const int rows = C.n - 2;
  Z3_DISPATCH(F.dtype, {
    constexpr int V = z3::VW<T>::V;
    a.ntx = (C.n - 1 + 16 * V - 1) / (16 * V);
    dim3 g((unsigned)(a.ntx * ((rows + z3::kTY - 1) / z3::kTY)), (unsigned)rows);
    z3::k3_restrict<T><<<g, 32 * z3::kTY, 0, s>>>(a, nullptr);
  })
  return cudaGetLastError();
}

cudaError_t z_prolong(const Level &C, const void *ec, const Level &F, void *uf, cudaStream_t s) {
  z3::ArgsT3 a;
  memset(&a, 0, sizeof a);
  a.src = ec;
  a.dst = uf;
  a.nf = F.n; a.pitchf = F.pitch; a.planef = F.plane;
  a.nc = C.n; a.pitchc = C.pitch; a.planec = C.plane;
  const int rows = F.n - 2;
  Z3_DISPATCH(F.dtype, {
    constexpr int V = z3::VW<T>::V;
    a.ntx = (F.n - 1 + 32 * V - 1) / (32 * V);
    dim3 g((unsigned)(a.ntx * ((rows + z3::kTY - 1) / z3::kTY)), (unsigned)rows);
    z3::k3_prolong<T><<<g, 32 * z3::kTY, 0, s>>>(a, nullptr);
  })
  return cudaGetLastError();
}

bool outer_ok(const Level &O, const Level &I) {
  return O.dim == 3 && !O.kf[0] && O.dtype == F64 && (I.dtype == F32 || I.dtype == BF16) && I.n == O.n &&
         O.n >= 5;
}

namespace {
template <typename Ti, bool UPDATE, bool ACC64>
cudaError_t launch_dc(z3::ArgsDC3 a, int *nparts, cudaStream_t s, const z3::ArgsDC3 *list = nullptr, int count = 1,
                      int max_parts = kMaxPartials) {
  constexpr size_t smem = (size_t)z3::DCL<Ti>::Smem;
  static int per_sm = 0;
  int r = resident(z3::k3_dc<Ti, UPDATE, ACC64>, 32 * z3::kDCWarps, smem, &per_sm);
  a.ntx = (a.n - 1 + 63) / 64;
  a.nty = (a.n - 2 + z3::kTY - 1) / z3::kTY;
  long long base = (long long)a.ntx * a.nty;
  a.zc = pick_zc(a.n, base, r, max_parts, list != nullptr);
  int nz = (a.n - 2 + a.zc - 1) / a.zc;
  *nparts = (int)(base * nz);
  a.pstride = max_parts;
  z3::k3_dc<Ti, UPDATE, ACC64><<<dim3((unsigned)base, (unsigned)nz, (unsigned)count), 32 * z3::kDCWarps, smem, s>>>(a, list);
  return cudaGetLastError();
}
// The exact outer step (k3_dcx): 8 rows x 128 columns per block, no dynamic
// shared memory; per-block partial sums in the same layout.
template <typename Ti, bool ACC64>
cudaError_t launch_dcx(z3::ArgsDC3 a, int *nparts, cudaStream_t s, const z3::ArgsDC3 *list = nullptr, int count = 1,
                       int max_parts = kMaxPartials) {
  static int per_sm = 0;
  int r = resident(z3::k3_dcx<Ti, ACC64>, 32 * z3::kXW, 0, &per_sm);
  a.ntx = (a.n - 1 + z3::kXC - 1) / z3::kXC;
  a.nty = (a.n - 2 + z3::kXW - 1) / z3::kXW;
  long long base = (long long)a.ntx * a.nty;
  a.zc = list ? pick_zc(a.n, base, r, max_parts, true) : pick_zc_waves(a.n, base, r, max_parts);
  int nz = (a.n - 2 + a.zc - 1) / a.zc;
  *nparts = (int)(base * nz);
  a.pstride = max_parts;
  z3::k3_dcx<Ti, ACC64><<<dim3((unsigned)base, (unsigned)nz, (unsigned)count), 32 * z3::kXW, 0, s>>>(a, list);
  return cudaGetLastError();
}
}  // namespace

cudaError_t dc_step(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d,
                    double *partials, int *nparts, const float *scale, bool update, bool acc64, bool exact,
                    cudaStream_t s) {
  z3::ArgsDC3 a;
  memset(&a, 0, sizeof a);
  a.u = uin;
  a.uout = uout;
  a.f = (const double *)O.f;
  a.e = e;
  a.d = d;
  a.partials = partials;
  a.scale = scale;
  a.n = O.n;
  a.pitch = O.pitch;
  a.pitchi = I.pitch;
  a.plane = O.plane;
  a.planei = I.plane;
  double cx = O.c[0] * O.inv_h2, cy = O.c[1] * O.inv_h2, cz = O.c[2] * O.inv_h2;
  a.cx = cx;
  a.cy = cy;
  a.cz = cz;
  a.cd = 2.0 * (cx + cy + cz);
  const int k2 = pow2_stencil(O);
  if (exact && update && k2 != kNoPow2) {
    a.k2 = k2;
    if (I.dtype == F32) return acc64 ? launch_dcx<float, true>(a, nparts, s) : launch_dcx<float, false>(a, nparts, s);
    return acc64 ? launch_dcx<bf16, true>(a, nparts, s) : launch_dcx<bf16, false>(a, nparts, s);
  }
  if (I.dtype == F32) {
    if (update) return acc64 ? launch_dc<float, true, true>(a, nparts, s) : launch_dc<float, true, false>(a, nparts, s);
    return acc64 ? launch_dc<float, false, true>(a, nparts, s) : launch_dc<float, false, false>(a, nparts, s);
  }
  if (update) return acc64 ? launch_dc<bf16, true, true>(a, nparts, s) : launch_dc<bf16, true, false>(a, nparts, s);
  return acc64 ? launch_dc<bf16, false, true>(a, nparts, s) : launch_dc<bf16, false, false>(a, nparts, s);
}


// ---------------------------------------------------------------- list launches (batch engine)

z3::Args3 stencil_record(const Level &L, double omega, const void *u, void *out, const void *f) {
  z3::Args3 a = stencil_args(L, omega);
  a.u = u;
  a.out = out;
  a.f = f;
  return a;
}

cudaError_t z_sweep_list(const Level &L, const z3::Args3 *list, int count, int color, cudaStream_t s) {
  z3::Args3 a = stencil_args(L, 1.0);
  a.color = color;
  cudaError_t e = cudaSuccess;
  if (color < 0) {
    Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kJacobi>(a, 1LL << 30, nullptr, s, list, count)));
  } else {
    Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kRB>(a, 1LL << 30, nullptr, s, list, count)));
  }
  return e;
}

cudaError_t z_jacobi_zero2_list(const Level &L, const z3::Args3 *list, int count, cudaStream_t s) {
  z3::Args3 a = stencil_args(L, 1.0);
  cudaError_t e = cudaSuccess;
  Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kJZ>(a, 1LL << 30, nullptr, s, list, count)));
  return e;
}

cudaError_t z_residual_list(const Level &L, const z3::Args3 *list, int count, cudaStream_t s) {
  z3::Args3 a = stencil_args(L, 1.0);
  cudaError_t e = cudaSuccess;
  Z3_DISPATCH(L.dtype, e = (launch_stencil<T, z3::kResid>(a, 1LL << 30, nullptr, s, list, count)));
  return e;
}

cudaError_t z_transfer_list(bool restrict_, const Level &F, const Level &C, const z3::ArgsT3 *list, int count,
                            cudaStream_t s) {
  z3::ArgsT3 a;
  memset(&a, 0, sizeof a);
  a.nf = F.n; a.pitchf = F.pitch; a.planef = F.plane;
  a.nc = C.n; a.pitchc = C.pitch; a.planec = C.plane;
  if (restrict_) {
    const int rows = C.n - 2;
    Z3_DISPATCH(F.dtype, {
      constexpr int V = z3::VW<T>::V;
      a.ntx = (C.n - 1 + 16 * V - 1) / (16 * V);
      dim3 g((unsigned)(a.ntx * ((rows + z3::kTY - 1) / z3::kTY)), (unsigned)rows, (unsigned)count);
      z3::k3_restrict<T><<<g, 32 * z3::kTY, 0, s>>>(a, list);
    })
  } else {
    const int rows = F.n - 2;
    Z3_DISPATCH(F.dtype, {
      constexpr int V = z3::VW<T>::V;
      a.ntx = (F.n - 1 + 32 * V - 1) / (32 * V);
      dim3 g((unsigned)(a.ntx * ((rows + z3::kTY - 1) / z3::kTY)), (unsigned)rows, (unsigned)count);
      z3::k3_prolong<T><<<g, 32 * z3::kTY, 0, s>>>(a, list);
    })
  }
  return cudaGetLastError();
}

z3::ArgsDC3 outer_record(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d) {
  z3::ArgsDC3 a;
  memset(&a, 0, sizeof a);
  a.u = uin;
  a.uout = uout;
  a.f = (const double *)O.f;
  a.e = e;
  a.d = d;
  double cx = O.c[0] * O.inv_h2, cy = O.c[1] * O.inv_h2, cz = O.c[2] * O.inv_h2;
  a.cx = cx;
  a.cy = cy;
  a.cz = cz;
  a.cd = 2.0 * (cx + cy + cz);
  return a;
}

cudaError_t dc_step_list(const Level &O, const Level &I, const z3::ArgsDC3 *list, int count, double *partials,
                         int pstride, int *nparts, bool update, bool exact, cudaStream_t s) {
  z3::ArgsDC3 a;
  memset(&a, 0, sizeof a);
  a.partials = partials;
  a.n = O.n;
  a.pitch = O.pitch;
  a.pitchi = I.pitch;
  a.plane = O.plane;
  a.planei = I.plane;
  if (exact && update) {
    return I.dtype == F32 ? launch_dcx<float, true>(a, nparts, s, list, count, pstride)
                          : launch_dcx<bf16, true>(a, nparts, s, list, count, pstride);
  }
  if (I.dtype == F32)
    return update ? launch_dc<float, true, true>(a, nparts, s, list, count, pstride)
                  : launch_dc<float, false, true>(a, nparts, s, list, count, pstride);
  return update ? launch_dc<bf16, true, true>(a, nparts, s, list, count, pstride)
                : launch_dc<bf16, false, true>(a, nparts, s, list, count, pstride);
}

}  // namespace d3
}  // namespace mg
