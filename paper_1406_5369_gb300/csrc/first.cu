// First residual of a solve that starts from u = 0 with homogeneous Dirichlet
// data: r = f - A 0 = f exactly, so the pass reads f, writes the inner
// defect (defect correction) and sums f^2 over the interior in FP64, with no
// stencil arithmetic.
#include "outer2d.cuh"

namespace mg {
namespace {

// Blocks walk the interior rows (and planes) in a fixed order; each writes
// one partial sum. Thread t takes the groups of 4 consecutive nodes t,
// t + 256, ... of each row, two groups per iteration so that four 16-byte
// loads of f are in flight (rows start 128-byte aligned and every row pitch
// is a multiple of 4 elements at least n, so the last group stays inside
// its row). d: inner defect (interior rows, zeros in the boundary columns),
// skipped when Ti is void.
__device__ __forceinline__ void store4(float *p, const float (&v)[4]) {
  *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(bf16 *p, const float (&v)[4]) {
  *(uint2 *)p = make_uint2(bf16_rne_bits(v[0]) | (bf16_rne_bits(v[1]) << 16),
                           bf16_rne_bits(v[2]) | (bf16_rne_bits(v[3]) << 16));
}

// This block's share (rows blockIdx.x, blockIdx.x + gridDim.x, ...) of one
// problem: defect written, sum of squares returned (per thread). SHORT: rows
// of at most blockDim.x groups take the short-row path (3D levels, and the
// batch engine's problems of every size; the single-problem 2D kernel keeps
// its registers without it).
template <int DIM, typename Ti, bool SHORT = (DIM == 3)>
__device__ __forceinline__ double first_rows(const double *__restrict__ f, const Geo &go, Ti *__restrict__ d,
                                             const Geo &gi) {
  const int n = go.n, m = n - 2, ng = (n + 3) >> 2;
  const long long rows = (long long)m * (DIM == 3 ? m : 1);
  double acc = 0.0;
  if (SHORT && ng <= (int)blockDim.x) {
    // short rows: rows r, r + G, r + 2G, r + 3G (G = gridDim.x) per
    // iteration, one group of each per thread, so that eight loads are in
    // flight per thread instead of two
    const int g = threadIdx.x;
    for (long long r0 = blockIdx.x; r0 < rows; r0 += 4LL * gridDim.x) {
      double v[4][4];
#pragma unroll
      for (int h = 0; h < 4; h++) {
        const long long r = r0 + (long long)h * gridDim.x;
        if (r < rows && g < ng) {
          const int j = 1 + (int)(r % m), k = DIM == 3 ? 1 + (int)(r / m) : 0;
          const double *fr = f + (long long)k * go.sz + (long long)j * go.sy + 4 * g;
          const double2 a = __ldg((const double2 *)fr), b = __ldg((const double2 *)(fr + 2));
          v[h][0] = a.x; v[h][1] = a.y; v[h][2] = b.x; v[h][3] = b.y;
        } else {
          v[h][0] = v[h][1] = v[h][2] = v[h][3] = 0.0;
        }
      }
#pragma unroll
      for (int h = 0; h < 4; h++) {
        const long long r = r0 + (long long)h * gridDim.x;
        float out[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int i = 4 * g + q;
          const double x = (i >= 1 && i <= n - 2) ? v[h][q] : 0.0;
          acc = fma(x, x, acc);
          out[q] = oz::d2f_bits(x);
        }
        if constexpr (!std::is_void<Ti>::value) {
          if (r < rows && g < ng) {
            const int j = 1 + (int)(r % m), k = DIM == 3 ? 1 + (int)(r / m) : 0;
            store4(d + (long long)k * gi.sz + (long long)j * gi.sy + 4 * g, out);
          }
        }
      }
    }
    return acc;
  }
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = 1 + (int)(r % m), k = DIM == 3 ? 1 + (int)(r / m) : 0;
    const double *fr = f + (long long)k * go.sz + (long long)j * go.sy;
    for (int g0 = threadIdx.x; g0 < ng; g0 += 2 * blockDim.x) {
      double v[2][4];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int g = g0 + h * (int)blockDim.x;
        if (g < ng) {
          const double2 a = __ldg((const double2 *)(fr + 4 * g)), b = __ldg((const double2 *)(fr + 4 * g + 2));
          v[h][0] = a.x; v[h][1] = a.y; v[h][2] = b.x; v[h][3] = b.y;
        } else {
          v[h][0] = v[h][1] = v[h][2] = v[h][3] = 0.0;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int g = g0 + h * (int)blockDim.x;
        float out[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int i = 4 * g + q;
          const double x = (i >= 1 && i <= n - 2) ? v[h][q] : 0.0;
          acc = fma(x, x, acc);
          out[q] = oz::d2f_bits(x);
        }
        if constexpr (!std::is_void<Ti>::value) {
          if (g < ng) store4(d + (long long)k * gi.sz + (long long)j * gi.sy + 4 * g, out);
        }
      }
    }
  }
  return acc;
}

template <int DIM, typename Ti>
__global__ void __launch_bounds__(256) k_first_defect(const double *__restrict__ f, Geo go, Ti *__restrict__ d,
                                                      Geo gi, double *__restrict__ partials) {
  const double acc = block_sum(first_rows<DIM, Ti>(f, go, d, gi));
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Problem blockIdx.y of a list (the batch engine); a problem no longer live
// is skipped by the whole block.
template <int DIM, typename Ti>
__global__ void __launch_bounds__(256) k_first_defect_list(const FirstRec *__restrict__ list) {
  const FirstRec &rc = list[blockIdx.y];
  if (rc.live && !*rc.live) return;
  Geo go, gi;
  go.n = gi.n = rc.n;
  go.sy = rc.sy;
  go.sz = rc.sz;
  gi.sy = rc.syi;
  gi.sz = rc.szi;
  const double acc = block_sum(first_rows<DIM, Ti, true>(rc.f, go, (Ti *)rc.d, gi));
  if (threadIdx.x == 0) rc.partials[blockIdx.x] = acc;
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

FirstRec first_record(const Level &O, const Level &I, double *partials, const int *live) {
  FirstRec r;
  r.f = (const double *)O.f;
  r.d = I.f;
  r.n = O.n;
  r.sy = O.pitch;
  r.sz = O.plane;
  r.syi = I.pitch;
  r.szi = I.plane;
  r.partials = partials;
  r.live = live;
  return r;
}

cudaError_t first_defect_list(int dim, int inner_dtype, const FirstRec *list, int count, int blocks,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const dim3 g((unsigned)blocks, (unsigned)count);
  if (inner_dtype == F32) {
    if (dim == 2) k_first_defect_list<2, float><<<g, 256, 0, s>>>(list);
    else k_first_defect_list<3, float><<<g, 256, 0, s>>>(list);
  } else if (inner_dtype == BF16) {
    if (dim == 2) k_first_defect_list<2, bf16><<<g, 256, 0, s>>>(list);
    else k_first_defect_list<3, bf16><<<g, 256, 0, s>>>(list);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mg
