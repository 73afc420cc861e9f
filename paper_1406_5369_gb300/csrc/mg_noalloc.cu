// mg_residual_norm_noalloc: the residual norm ||f - A u||_2 of a constant
// stencil problem for callers that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc: a host framework that owns
// every device allocation through its own pool, or a latency-critical loop
// where an allocation (which may synchronise the whole device) is forbidden.
// They cannot build a context (which needs a caller-provided arena) either.
// This entry point needs nothing but the caller's input and output buffers:
// its only scratch, the per-block partial sums of the two-pass reduction, sits
// in a file-scope static device array that every GPU loading the library
// holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>
#include <stdio.h>

#include "kernels.cuh"
#include "mg.h"

namespace {

// Partial sums (one per block) plus one slot for the finished norm.
constexpr int kMaxPartials = MG_NOALLOC_MAX_PARTIALS;
constexpr int kThreads = 256;
constexpr long long kNodesPerBlock = 2048;  // interior nodes per block (8 per thread)

static __device__ __align__(256) double g_noalloc_scratch[kMaxPartials + 32];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {};

// One block: strided sequential sums per thread, then a fixed tree.
__global__ void k_finalize_dense(const double *__restrict__ partials, int nb, double *__restrict__ result) {
  __shared__ double buf[1024];
  int t = threadIdx.x;
  double a = 0.0;
  for (int i = t; i < nb; i += 1024) a += partials[i];
  buf[t] = a;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (t < s) buf[t] += buf[t + s];
    __syncthreads();
  }
  if (t == 0) result[0] = sqrt(buf[0]);
}

mg_status nfail(mg_status st, const char *msg, cudaError_t e = cudaSuccess) {
  char buf[256];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "%s", msg);
  mg::set_error_message(buf);
  return st;
}

// Device address of the static scratch on the current device, looked up once
// per device (the symbol name is only a host-side handle).
mg_status scratch_ptr(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(MG_ECUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return nfail(MG_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return nfail(MG_ECUDA, "cudaGetSymbolAddress", e);
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return MG_OK;
}

}  // namespace

extern "C" mg_status mg_residual_norm_noalloc(int dim, int n, const mg_const_stencil *stencil, const double *u,
                                              const double *f, double *out, void *stream) {
  mg::set_error_message("");
  if (dim != 2 && dim != 3) return nfail(MG_EINVAL, "dim must be 2 or 3");
  if (n < 3) return nfail(MG_EINVAL, "n must be at least 3");
  if (!u || !f || !out) return nfail(MG_EINVAL, "NULL argument");
  long long m = n - 2;
  long long interior = m * m * (dim == 3 ? m : 1);
  long long nb = (interior + kNodesPerBlock - 1) / kNodesPerBlock;
  if (nb < 1) nb = 1;
  if (nb > kMaxPartials)
    return nfail(MG_EINVAL, "grid too large for the static scratch of mg_residual_norm_noalloc "
                            "(at most MG_NOALLOC_MAX_PARTIALS * 2048 interior nodes)");
  double c[3] = {1.0, 1.0, 1.0};
  if (stencil) {
    c[0] = stencil->cx;
    c[1] = stencil->cy;
    c[2] = dim == 3 ? stencil->cz : 1.0;
    if (!(c[0] > 0 && c[1] > 0 && c[2] > 0)) return nfail(MG_EINVAL, "stencil coefficients must be > 0");
  }
  double *scratch = nullptr;
  mg_status st = scratch_ptr(&scratch);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  mg::Geo g;
  g.n = n;
  g.sy = n;
  g.sz = (long long)n * n;
  mg::Sten<double> sten;
  sten.kf0 = sten.kf1 = sten.kf2 = nullptr;
  sten.c0 = c[0];
  sten.c1 = c[1];
  sten.c2 = c[2];
  double h = 1.0 / (double)(n - 1);
  sten.inv_h2 = 1.0 / (h * h);
  sten.diag = 2.0 * (c[0] + c[1] + (dim == 3 ? c[2] : 0.0)) * sten.inv_h2;
  double *partials = scratch;
  double *result = scratch + kMaxPartials;
  // the library's own partial-sum kernel (one partial per block, fixed
  // per-block order), pointed at the static scratch
  if (dim == 2) mg::k_norm_partials<2, double, false><<<(unsigned)nb, kThreads, 0, s>>>(u, f, g, sten, partials);
  else mg::k_norm_partials<3, double, false><<<(unsigned)nb, kThreads, 0, s>>>(u, f, g, sten, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(MG_ECUDA, "partial-sum kernel launch", e);
  k_finalize_dense<<<1, 1024, 0, s>>>(partials, (int)nb, result);
  e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(MG_ECUDA, "finalize kernel launch", e);
  e = cudaMemcpyAsync(out, result, sizeof(double), cudaMemcpyDefault, s);
  if (e != cudaSuccess) return nfail(MG_ECUDA, "copy of the result", e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return nfail(MG_ECUDA, "stream synchronize", e);
  return MG_OK;
}
