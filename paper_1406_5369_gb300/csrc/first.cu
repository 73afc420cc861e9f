// First residual of a solve that starts from u = 0 with homogeneous Dirichlet
// data: r = f - A 0 = f exactly, so the pass reads f, writes the inner
// defect (defect correction) and sums f^2 over the interior in FP64, with no
// stencil arithmetic.
#include "outer2d.cuh"

namespace mg {
namespace {

// Blocks walk the interior rows (and planes) in a fixed order; each writes
// one partial sum. d: inner defect (interior rows, zeros in the boundary
// columns), skipped when Ti is void.
template <int DIM, typename Ti>
__global__ void __launch_bounds__(256) k_first_defect(const double *__restrict__ f, Geo go, Ti *__restrict__ d,
                                                      Geo gi, double *__restrict__ partials) {
  const int n = go.n, m = n - 2;
  const long long rows = (long long)m * (DIM == 3 ? m : 1);
  double acc = 0.0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = 1 + (int)(r % m), k = DIM == 3 ? 1 + (int)(r / m) : 0;
    const double *fr = f + (long long)k * go.sz + (long long)j * go.sy;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const bool in = i >= 1 && i <= n - 2;
      const double v = in ? fr[i] : 0.0;
      acc = fma(v, v, acc);
      if constexpr (!std::is_void<Ti>::value) {
        st(d + (long long)k * gi.sz + (long long)j * gi.sy + i, oz::d2f_bits(v));
      }
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <int DIM> cudaError_t launch(const Level &O, const Level *I, double *partials, cudaStream_t s) {
  const Geo go = geo_of(O);
  if (!I) {
    k_first_defect<DIM, void><<<kNormBlocks, 256, 0, s>>>((const double *)O.f, go, nullptr, go, partials);
  } else if (I->dtype == F32) {
    k_first_defect<DIM, float><<<kNormBlocks, 256, 0, s>>>((const double *)O.f, go, (float *)I->f, geo_of(*I), partials);
  } else {
    k_first_defect<DIM, bf16><<<kNormBlocks, 256, 0, s>>>((const double *)O.f, go, (bf16 *)I->f, geo_of(*I), partials);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t first_defect(const Level &O, const Level *I, double *partials, cudaStream_t s) {
  if (O.dtype != F64 || (I && I->dtype != F32 && I->dtype != BF16)) return cudaErrorInvalidValue;
  return O.dim == 2 ? launch<2>(O, I, partials, s) : launch<3>(O, I, partials, s);
}

}  // namespace mg
