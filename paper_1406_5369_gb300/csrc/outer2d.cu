// Launchers of the streaming 2D finest-level kernels (outer2d.cuh) and the
// deterministic two-pass norm finalisation.
#include <math.h>
#include <string.h>

#include "outer2d.cuh"

namespace mg {

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

// list: a launch over many problems, which supply the parallelism: chunks of
// 256 rows, a function of the size alone (so is each problem's partition of
// its norm sum, whatever else is in the list).
void chunking(oz::ArgsOuter &a, int n, int bps, int max_parts = kMaxPartials, bool list = false) {
  a.nstrips = (n + oz::kOut - 1) / oz::kOut;
  long long slots = (long long)sm_count() * bps * oz::kWarps;
  long long nchunks = list ? (n + 255) / 256 : slots / a.nstrips;
  if (nchunks < 1) nchunks = 1;
  int R = (int)((n + nchunks - 1) / nchunks);
  R = (R + 7) / 8 * 8;
  if (R < 8) R = 8;
  a.R = R;
  a.nchunks = (n + R - 1) / R;
  if ((long long)a.nstrips * a.nchunks > max_parts) {  // one partial sum per warp must fit
    int nc = max_parts / a.nstrips;
    if (nc < 1) nc = 1;
    a.R = ((n + nc - 1) / nc + 7) / 8 * 8;
    a.nchunks = (n + a.R - 1) / a.R;
  }
}

template <typename KernelT> int occupancy(KernelT k, int threads, size_t smem) {
  int bps = 1;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, threads, smem);
  return bps < 1 ? 1 : bps;
}

template <typename Ti, bool UPDATE, bool ACC64>
cudaError_t launch_dc(oz::ArgsOuter a, int n, int *nparts, cudaStream_t s, const oz::ArgsOuter *list = nullptr,
                      int count = 1, int max_parts = kMaxPartials) {
  constexpr int IB = oz::InnerLane<Ti>::bytes;
  constexpr int IBP = IB < 16 ? 16 : IB;
  constexpr size_t smem = (size_t)oz::kWarps * oz::kRing * 32 * (32 + 32 + IBP);
  static int bps = 0;
  if (!bps) {
    bps = occupancy(oz::k_dc2d<Ti, UPDATE, ACC64, false>, 32 * oz::kWarps, smem);
    occupancy(oz::k_dc2d<Ti, UPDATE, ACC64, true>, 32 * oz::kWarps, smem);  // sets its shared-memory limit
  }
  chunking(a, n, bps, max_parts, list != nullptr);
  long long warps = (long long)a.nstrips * a.nchunks;
  *nparts = (int)warps;
  a.pstride = max_parts;
  unsigned blocks = (unsigned)((warps + oz::kWarps - 1) / oz::kWarps);
  if (list)
    oz::k_dc2d<Ti, UPDATE, ACC64, true><<<dim3(blocks, (unsigned)count), 32 * oz::kWarps, smem, s>>>(a, list);
  else
    oz::k_dc2d<Ti, UPDATE, ACC64, false><<<blocks, 32 * oz::kWarps, smem, s>>>(a, nullptr);
  return cudaGetLastError();
}

template <typename Ti, bool ACC64>
cudaError_t launch_dcx(oz::ArgsOuter a, int n, int *nparts, cudaStream_t s, const oz::ArgsOuter *list = nullptr,
                       int count = 1, int max_parts = kMaxPartials) {
  constexpr int IB = oz::InnerLane<Ti>::bytes;
  constexpr int IBP = IB < 16 ? 16 : IB;
  constexpr size_t smem = (size_t)oz::kWarps * oz::kXRing * 32 * (32 + 32 + IBP);
  static int bps = 0;
  if (!bps) {
    bps = occupancy(oz::k_dcx2d<Ti, ACC64, false>, 32 * oz::kWarps, smem);
    occupancy(oz::k_dcx2d<Ti, ACC64, true>, 32 * oz::kWarps, smem);
  }
  chunking(a, n, bps, max_parts, list != nullptr);
  long long warps = (long long)a.nstrips * a.nchunks;
  *nparts = (int)warps;
  a.pstride = max_parts;
  unsigned blocks = (unsigned)((warps + oz::kWarps - 1) / oz::kWarps);
  if (list)
    oz::k_dcx2d<Ti, ACC64, true><<<dim3(blocks, (unsigned)count), 32 * oz::kWarps, smem, s>>>(a, list);
  else
    oz::k_dcx2d<Ti, ACC64, false><<<blocks, 32 * oz::kWarps, smem, s>>>(a, nullptr);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_norm(oz::ArgsOuter a, int n, int *nparts, cudaStream_t s) {
  constexpr size_t smem = (size_t)oz::kWarps * oz::kRing * 32 * fz::Lane<T>::bytes * 2;
  static int bps = 0;
  if (!bps) bps = occupancy(oz::k_norm2d<T>, 32 * oz::kWarps, smem);
  chunking(a, n, bps);
  long long warps = (long long)a.nstrips * a.nchunks;
  *nparts = (int)warps;
  unsigned blocks = (unsigned)((warps + oz::kWarps - 1) / oz::kWarps);
  oz::k_norm2d<T><<<blocks, 32 * oz::kWarps, smem, s>>>(a);
  return cudaGetLastError();
}

// Sums nb partials: each thread adds a strided subset in order, then a
// fixed tree; the result depends only on nb. out[0] = norm, out[1] = sum.
// With scale_in the partials are sums of (s r)^2 and the norm is divided by
// s; scale_out receives 2^-e with e the exponent of norm / sqrt(nint).
__global__ void k_finalize(const double *__restrict__ partials, int nb, double *__restrict__ out,
                           const float *scale_in, float *scale_out, double nint) {
  __shared__ double buf[1024];
  int t = threadIdx.x;
  double a = 0.0;
  for (int i = t; i < nb; i += 1024) a += partials[i];
  buf[t] = a;
  __syncthreads();
  for (int st = 512; st > 0; st >>= 1) {
    if (t < st) buf[t] += buf[t + st];
    __syncthreads();
  }
  if (t == 0) {
    double sum = buf[0];
    double norm = sqrt(sum);
    if (scale_in) norm /= (double)*scale_in;
    out[0] = norm;
    out[1] = sum;
    if (scale_out && norm > 0.0 && isfinite(norm)) {
      int e = 0;
      frexp(norm / sqrt(nint > 1.0 ? nint : 1.0), &e);
      if (e > 100) e = 100;
      if (e < -100) e = -100;
      *scale_out = (float)ldexp(1.0, -e);
    }
  }
}

}  // namespace

cudaError_t norm_finalize_ex(const double *partials, int nb, double *out, const float *scale_in, float *scale_out,
                             double nint, cudaStream_t s) {
  k_finalize<<<1, 1024, 0, s>>>(partials, nb, out, scale_in, scale_out, nint);
  return cudaGetLastError();
}

namespace d2 {

bool outer_ok(const Level &O, const Level &I) {
  return O.dim == 2 && !O.kf[0] && O.dtype == F64 && (I.dtype == F32 || I.dtype == BF16) && O.n >= 5;
}

cudaError_t dc_step(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d,
                    double *partials, int *nparts, const float *scale, bool update, bool acc64, bool exact,
                    cudaStream_t s) {
  oz::ArgsOuter a;
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
  a.cx = O.c[0] * O.inv_h2;
  a.cy = O.c[1] * O.inv_h2;
  a.cd = 2.0 * (a.cx + a.cy);
  const int k2 = pow2_stencil(O);
  if (exact && update && k2 != kNoPow2) {
    a.k2 = k2;
    if (I.dtype == F32)
      return acc64 ? launch_dcx<float, true>(a, O.n, nparts, s) : launch_dcx<float, false>(a, O.n, nparts, s);
    return acc64 ? launch_dcx<bf16, true>(a, O.n, nparts, s) : launch_dcx<bf16, false>(a, O.n, nparts, s);
  }
  if (I.dtype == F32) {
    if (update) return acc64 ? launch_dc<float, true, true>(a, O.n, nparts, s) : launch_dc<float, true, false>(a, O.n, nparts, s);
    return acc64 ? launch_dc<float, false, true>(a, O.n, nparts, s) : launch_dc<float, false, false>(a, O.n, nparts, s);
  }
  if (update) return acc64 ? launch_dc<bf16, true, true>(a, O.n, nparts, s) : launch_dc<bf16, true, false>(a, O.n, nparts, s);
  return acc64 ? launch_dc<bf16, false, true>(a, O.n, nparts, s) : launch_dc<bf16, false, false>(a, O.n, nparts, s);
}

oz::ArgsOuter outer_record(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d) {
  oz::ArgsOuter a;
  memset(&a, 0, sizeof a);
  a.u = uin;
  a.uout = uout;
  a.f = (const double *)O.f;
  a.e = e;
  a.d = d;
  a.cx = O.c[0] * O.inv_h2;
  a.cy = O.c[1] * O.inv_h2;
  a.cd = 2.0 * (a.cx + a.cy);
  return a;
}

cudaError_t dc_step_list(const Level &O, const Level &I, const oz::ArgsOuter *list, int count, double *partials,
                         int pstride, int *nparts, bool update, bool exact, cudaStream_t s) {
  oz::ArgsOuter a;
  memset(&a, 0, sizeof a);
  a.partials = partials;
  a.n = O.n;
  a.pitch = O.pitch;
  a.pitchi = I.pitch;
  if (exact && update) {
    return I.dtype == F32 ? launch_dcx<float, true>(a, O.n, nparts, s, list, count, pstride)
                          : launch_dcx<bf16, true>(a, O.n, nparts, s, list, count, pstride);
  }
  if (I.dtype == F32) {
    return update ? launch_dc<float, true, true>(a, O.n, nparts, s, list, count, pstride)
                  : launch_dc<float, false, true>(a, O.n, nparts, s, list, count, pstride);
  }
  return update ? launch_dc<bf16, true, true>(a, O.n, nparts, s, list, count, pstride)
                : launch_dc<bf16, false, true>(a, O.n, nparts, s, list, count, pstride);
}

bool norm_ok(const Level &L) { return L.dim == 2 && !L.kf[0] && (L.dtype == F64 || L.dtype == F32) && L.n >= 5; }

cudaError_t norm_stream(const Level &L, const void *u, const void *f, double *partials, int *nparts, cudaStream_t s) {
  oz::ArgsOuter a;
  memset(&a, 0, sizeof a);
  a.u = (const double *)u;  // reinterpreted by the typed kernel
  a.f = (const double *)f;
  a.partials = partials;
  a.n = L.n;
  a.pitch = L.pitch;
  a.cx = L.c[0] * L.inv_h2;
  a.cy = L.c[1] * L.inv_h2;
  if (L.dtype == F64) return launch_norm<double>(a, L.n, nparts, s);
  return launch_norm<float>(a, L.n, nparts, s);
}

}  // namespace d2
}  // namespace mg
