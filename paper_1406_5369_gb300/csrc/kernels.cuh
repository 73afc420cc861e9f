// Device kernels of the multigrid V-cycle (Algorithm 1 of the paper,
// Sec. 2.3-2.4), templated on dimension, storage type and stencil kind.
//
// Storage types: double (FP64 levels), float, __nv_bfloat16 (inner levels of
// defect correction). Arithmetic runs in double for double storage and in
// float otherwise. Every kernel touches interior nodes only, so boundary
// nodes keep their Dirichlet values (finest level) or zero (coarse levels).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mg_internal.h"

namespace mg {

typedef __nv_bfloat16 bf16;

template <typename T> struct CT { typedef float type; };
template <> struct CT<double> { typedef double type; };

// A coefficient in the compute type: the double, or its float rounded on the
// host (so that no FP64 -> FP32 conversion, a slow-pipe instruction the
// compiler may repeat inside loops, runs on the device).
template <typename C> __device__ __forceinline__ C pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

__device__ __forceinline__ double ld(const double *p) { return *p; }
__device__ __forceinline__ float ld(const float *p) { return *p; }
__device__ __forceinline__ float ld(const bf16 *p) { return __bfloat162float(*p); }

// FP32 -> BF16 with round to nearest, ties to even, on the integer pipe: add
// 0x7fff plus the lowest kept bit to the float's bits and keep the top 16
// (a carry into the exponent rounds up to the next binade or to infinity,
// as IEEE-754 rounding requires); NaNs keep their sign and get the quiet bit.
// Single values (field copies, the generic kernels) take this path; the
// streaming kernels store pairs with the packed conversion below, which
// measured faster than these integer operations (the 513^3 BF16 Jacobi sweep
// went from 170 to 149 us). Conversions that involve FP64 are different:
// they issue on the slow FP64 pipe, so those are done with bit operations.
__device__ __forceinline__ unsigned bf16_rne_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned r = (b + 0x7fffu + ((b >> 16) & 1u)) >> 16;
  return (b & 0x7fffffffu) > 0x7f800000u ? ((b >> 16) | 0x40u) : r;
}
// Two values packed as a bfloat162 word (a in the low half), rounded to
// nearest even by the packed conversion instruction (one instruction for the
// pair).
__device__ __forceinline__ unsigned bf16x2_rne_bits(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned *>(&v);
}
__device__ __forceinline__ bf16 bf16_rne(float x) { return __ushort_as_bfloat16((unsigned short)bf16_rne_bits(x)); }

__device__ __forceinline__ void st(double *p, double v) { *p = v; }
__device__ __forceinline__ void st(float *p, double v) { *p = (float)v; }
__device__ __forceinline__ void st(bf16 *p, double v) { *p = bf16_rne((float)v); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(bf16 *p, float v) { *p = bf16_rne(v); }
__device__ __forceinline__ void st(double *p, float v) { *p = (double)v; }

// Geometry of a level in kernel form.
struct Geo {
  int n;
  long long sy;  // row stride (pitch)
  long long sz;  // plane stride
};

__host__ __forceinline__ Geo geo_of(const Level &L) {
  Geo g;
  g.n = L.n;
  g.sy = L.pitch;
  g.sz = L.plane;
  return g;
}

// Stencil coefficients in compute type C.
template <typename C> struct Sten {
  const C *kf0, *kf1, *kf2;  // faces (variable stencil)
  C c0, c1, c2;              // constant coefficients
  C inv_h2;
  C diag;                    // constant stencil: 2 (c0+c1[+c2]) / h^2
};

template <typename C> __host__ Sten<C> sten_of(const Level &L) {
  Sten<C> s;
  s.kf0 = (const C *)L.kf[0];
  s.kf1 = (const C *)L.kf[1];
  s.kf2 = (const C *)L.kf[2];
  s.c0 = (C)L.c[0];
  s.c1 = (C)L.c[1];
  s.c2 = (C)L.c[2];
  s.inv_h2 = (C)L.inv_h2;
  double d = 2.0 * (L.c[0] + L.c[1] + (L.dim == 3 ? L.c[2] : 0.0)) * L.inv_h2;
  s.diag = (C)d;
  return s;
}

// (A u)_p and diag_p at node p. Constant stencil:
//   A u = h^-2 sum_d c_d (2 u_p - u_{p-e_d} - u_{p+e_d});
// variable stencil (conservative form):
//   A u = h^-2 sum_d [k_{p+e_d/2} (u_p - u_{p+e_d}) + k_{p-e_d/2} (u_p - u_{p-e_d})].
template <int DIM, bool VAR, typename T, typename C>
__device__ __forceinline__ void apply_at(const T *__restrict__ u, long long p, const Geo &g,
                                         const Sten<C> &s, C &Au, C &diag) {
  C u0 = ld(u + p);
  C uw = ld(u + p - 1), ue = ld(u + p + 1);
  C us = ld(u + p - g.sy), un = ld(u + p + g.sy);
  if (!VAR) {
    C acc = s.c0 * ((u0 + u0) - uw - ue) + s.c1 * ((u0 + u0) - us - un);
    if (DIM == 3) {
      C ud = ld(u + p - g.sz), uu = ld(u + p + g.sz);
      acc += s.c2 * ((u0 + u0) - ud - uu);
    }
    Au = acc * s.inv_h2;
    diag = s.diag;
  } else {
    C kxp = s.kf0[p], kxm = s.kf0[p - 1], kyp = s.kf1[p], kym = s.kf1[p - g.sy];
    C acc = kxp * (u0 - ue) + kxm * (u0 - uw) + kyp * (u0 - un) + kym * (u0 - us);
    C dg = kxp + kxm + kyp + kym;
    if (DIM == 3) {
      C ud = ld(u + p - g.sz), uu = ld(u + p + g.sz);
      C kzp = s.kf2[p], kzm = s.kf2[p - g.sz];
      acc += kzp * (u0 - uu) + kzm * (u0 - ud);
      dg += kzp + kzm;
    }
    Au = acc * s.inv_h2;
    diag = dg * s.inv_h2;
  }
}

// Thread -> node map of the simple kernels: x from the block/thread x index,
// y from blockIdx.y, z from blockIdx.z.
struct Idx {
  int i, j, k;
  long long p;
  bool interior;
};

template <int DIM> __device__ __forceinline__ Idx node_index(const Geo &g) {
  Idx t;
  t.i = blockIdx.x * blockDim.x + threadIdx.x;
  t.j = blockIdx.y;
  t.k = DIM == 3 ? (int)blockIdx.z : 0;
  t.p = (long long)t.k * g.sz + (long long)t.j * g.sy + t.i;
  t.interior = t.i >= 1 && t.i <= g.n - 2 && t.j >= 1 && t.j <= g.n - 2 &&
               (DIM == 2 || (t.k >= 1 && t.k <= g.n - 2));
  return t;
}

// ---------------------------------------------------------------- smoothers

// Half-sweep of omega-RBGS (Sec. 2.4 GaussSeidel, order rb): nodes with
// (i+j[+k]) % 2 == color get u += omega (f - A u) / diag. Same-colour nodes
// do not couple in a 5-/7-point stencil, so all of them update at once.
template <int DIM, typename T, bool VAR>
__global__ void k_rbgs_half(T *__restrict__ u, const T *__restrict__ f, Geo g, Sten<typename CT<T>::type> s,
                            int color, typename CT<T>::type omega) {
  typedef typename CT<T>::type C;
  Idx t = node_index<DIM>(g);
  if (!t.interior || ((t.i + t.j + t.k) & 1) != color) return;
  C Au, dg;
  apply_at<DIM, VAR>(u, t.p, g, s, Au, dg);
  C u0 = ld(u + t.p);
  st(u + t.p, u0 + omega * (ld(f + t.p) - Au) / dg);
}

// omega-Jacobi: uout = uin + omega (f - A uin) / diag.
template <int DIM, typename T, bool VAR>
__global__ void k_jacobi(const T *__restrict__ uin, T *__restrict__ uout, const T *__restrict__ f, Geo g,
                         Sten<typename CT<T>::type> s, typename CT<T>::type omega) {
  typedef typename CT<T>::type C;
  Idx t = node_index<DIM>(g);
  if (!t.interior) return;
  C Au, dg;
  apply_at<DIM, VAR>(uin, t.p, g, s, Au, dg);
  st(uout + t.p, ld(uin + t.p) + omega * (ld(f + t.p) - Au) / dg);
}

// ---------------------------------------------------------------- residual

template <int DIM, typename T, bool VAR>
__global__ void k_residual(const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ r, Geo g,
                           Sten<typename CT<T>::type> s) {
  typedef typename CT<T>::type C;
  Idx t = node_index<DIM>(g);
  if (!t.interior) return;
  C Au, dg;
  apply_at<DIM, VAR>(u, t.p, g, s, Au, dg);
  st(r + t.p, ld(f + t.p) - Au);
}

// ---------------------------------------------------------------- transfers

// Full weighting at coarse interior node (I,J[,K]): tensor product of
// (1,2,1)/4 over the fine neighbourhood of fine node (2I,2J[,2K]).
template <int DIM, typename Tf, typename Tc>
__global__ void k_restrict(const Tf *__restrict__ rf, Geo gf, Tc *__restrict__ fc, Geo gc) {
  typedef typename CT<Tc>::type C;
  Idx t = node_index<DIM>(gc);
  if (!t.interior) return;
  long long q = (long long)(2 * t.k) * gf.sz + (long long)(2 * t.j) * gf.sy + 2 * t.i;
  C acc = 0;
  if (DIM == 2) {
    C a = ld(rf + q - gf.sy - 1) + ld(rf + q - gf.sy + 1) + ld(rf + q + gf.sy - 1) + ld(rf + q + gf.sy + 1);
    C b = ld(rf + q - gf.sy) + ld(rf + q + gf.sy) + ld(rf + q - 1) + ld(rf + q + 1);
    acc = (C)0.0625 * a + (C)0.125 * b + (C)0.25 * ld(rf + q);
  } else {
#pragma unroll
    for (int dz = -1; dz <= 1; dz++) {
      C wz = dz == 0 ? (C)0.5 : (C)0.25;
#pragma unroll
      for (int dy = -1; dy <= 1; dy++) {
        C wy = dy == 0 ? (C)0.5 : (C)0.25;
        const Tf *row = rf + q + dz * gf.sz + dy * gf.sy;
        C line = (C)0.25 * (ld(row - 1) + ld(row + 1)) + (C)0.5 * ld(row);
        acc += wz * wy * line;
      }
    }
  }
  st(fc + t.p, acc);
}

// Bi-/trilinear interpolation and correction at fine interior node (i,j[,k]).
template <int DIM, typename Tc, typename Tf>
__global__ void k_prolong(const Tc *__restrict__ ec, Geo gc, Tf *__restrict__ uf, Geo gf) {
  typedef typename CT<Tf>::type C;
  Idx t = node_index<DIM>(gf);
  if (!t.interior) return;
  int I = t.i >> 1, J = t.j >> 1, K = t.k >> 1;
  int oi = t.i & 1, oj = t.j & 1, ok = DIM == 3 ? (t.k & 1) : 0;
  C acc = 0;
#pragma unroll
  for (int a = 0; a <= 1; a++) {
    if (a && !ok) break;
#pragma unroll
    for (int b = 0; b <= 1; b++) {
      if (b && !oj) break;
      const Tc *row = ec + (long long)(K + a) * gc.sz + (long long)(J + b) * gc.sy + I;
      C v = oi ? (C)0.5 * ((C)ld(row) + (C)ld(row + 1)) : (C)ld(row);
      acc += v;
    }
  }
  C w = (oj ? (C)0.5 : (C)1) * (ok ? (C)0.5 : (C)1);
  st(uf + t.p, (C)ld(uf + t.p) + w * acc);
}

// ---------------------------------------------------------------- norms

// Block sum of a double with warp shuffles, then one value per warp in
// shared memory; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_part[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? warp_part[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Interior node t of a level with m = n-2 interior nodes per dimension.
// Calls body(po, pi) for the interior nodes of block blockIdx.x's share of
// an n^DIM level (m = n - 2 interior nodes per dimension), in a fixed order
// that depends only on the grid size: rows (y, or y and z) blockIdx.x,
// blockIdx.x + gridDim.x, ...; within a row, columns 1 + threadIdx.x,
// 1 + threadIdx.x + blockDim.x, ... po and pi index the same node in the two
// geometries go and gi (an outer level and its inner level). One integer
// division per row, none per node.
template <int DIM, typename Fn>
__device__ __forceinline__ void for_interior_rows(int m, const Geo &go, const Geo &gi, Fn &&body) {
  const int rows = DIM == 3 ? m * m : m;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = 1 + (DIM == 3 ? r % m : r), k = DIM == 3 ? 1 + r / m : 0;
    const long long ro = (long long)k * go.sz + (long long)j * go.sy;
    const long long ri = (long long)k * gi.sz + (long long)j * gi.sy;
    for (int i = 1 + (int)threadIdx.x; i <= m; i += (int)blockDim.x) body(ro + i, ri + i);
  }
}

// Per-block partial sums of (f - A u)^2 in FP64 over a fixed partition of
// the rows, so the summation order depends only on the grid size.
template <int DIM, typename T, bool VAR>
__global__ void k_norm_partials(const T *__restrict__ u, const T *__restrict__ f, Geo g,
                                Sten<typename CT<T>::type> s, double *__restrict__ partials) {
  typedef typename CT<T>::type C;
  double acc = 0.0;
  for_interior_rows<DIM>(g.n - 2, g, g, [&](long long p, long long) {
    C Au, dg;
    apply_at<DIM, VAR>(u, p, g, s, Au, dg);
    double r = (double)(ld(f + p) - Au);
    acc += r * r;
  });
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// ---------------------------------------------------------------- coarsest

// One unknown (3^dim grid): u + (f - A u)/diag is the exact solution.
template <int DIM, bool VAR>
__global__ void k_coarse3(double *u, const double *f, Geo g, Sten<double> s) {
  long long p = (DIM == 3 ? g.sz : 0) + g.sy + 1;
  double Au, dg;
  apply_at<DIM, VAR>(u, p, g, s, Au, dg);
  u[p] = u[p] + (f[p] - Au) / dg;
}

// Coarsest grids of 5^dim or 9^dim nodes are solved directly: the FP64
// inverse of the operator restricted to the interior unknowns is formed once
// (k_dense_inverse) and applied to the residual, u += A^{-1} (f - A u), so a
// nonzero start and Dirichlet values are handled like the 3^dim case.

// Interior node t of the coarsest level, lexicographic order (x fastest).
template <int DIM> __device__ __forceinline__ long long coarse_node(int t, const Geo &g) {
  const int m = g.n - 2;
  const int i = 1 + t % m, r = t / m;
  const int j = 1 + (DIM == 3 ? r % m : r), k = DIM == 3 ? 1 + r / m : 0;
  return (long long)k * g.sz + (long long)j * g.sy + i;
}

// One block. Assembles the interior matrix A (row t: diag at t, -k_f/h^2 at
// each interior neighbour; neighbours on the boundary only enter the
// diagonal) into `a` and inverts it in place by Gauss-Jordan elimination
// without pivoting, which is stable for a symmetric positive definite A.
// Step k divides row k by the pivot (1/a_kk on the diagonal) and subtracts
// a_ik times the new row k from every other row i (-a_ik/a_kk in column k).
template <int DIM, bool VAR>
__global__ void __launch_bounds__(1024) k_dense_inverse(double *a, Geo g, Sten<double> s) {
  __shared__ double colk[kDenseMax];
  __shared__ double rpiv;
  const int m = g.n - 2, N = DIM == 3 ? m * m * m : m * m;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) a[e] = 0.0;
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const long long p = coarse_node<DIM>(t, g);
    const int i = t % m, j = (t / m) % m, k = DIM == 3 ? t / (m * m) : 0;
    const int pos[3] = {i, j, k};
    const long long gs[3] = {1, g.sy, g.sz};
    const int ts[3] = {1, m, m * m};
    const double cc[3] = {s.c0, s.c1, s.c2};
    const double *kf[3] = {s.kf0, s.kf1, s.kf2};
    double diag = 0.0;
    for (int d = 0; d < DIM; d++) {
      const double kp = VAR ? kf[d][p] : cc[d], km = VAR ? kf[d][p - gs[d]] : cc[d];
      diag += kp + km;
      if (pos[d] + 1 < m) a[(long long)t * N + t + ts[d]] = -kp * s.inv_h2;
      if (pos[d] > 0) a[(long long)t * N + t - ts[d]] = -km * s.inv_h2;
    }
    a[(long long)t * N + t] = diag * s.inv_h2;
  }
  __syncthreads();
  for (int k = 0; k < N; k++) {
    if (threadIdx.x == 0) rpiv = 1.0 / a[(long long)k * N + k];
    for (int i = threadIdx.x; i < N; i += blockDim.x) colk[i] = a[(long long)i * N + k];
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x)
      a[(long long)k * N + j] = (j == k ? 1.0 : a[(long long)k * N + j]) * rpiv;
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int i = e / N, j = e % N;
      if (i == k) continue;
      a[e] = (j == k ? 0.0 : a[e]) - colk[i] * a[(long long)k * N + j];
    }
    __syncthreads();
  }
}

// One block: r = f - A u at the N interior nodes (shared memory), then
// u_t += sum_j (A^{-1})_{jt} r_j (A^{-1} is symmetric; reading its column t
// keeps consecutive threads on consecutive addresses).
template <int DIM, bool VAR>
__global__ void __launch_bounds__(352) k_coarse_dense(double *u, const double *f, Geo g, Sten<double> s,
                                                      const double *ainv) {
  __shared__ double r[kDenseMax];
  const int m = g.n - 2, N = DIM == 3 ? m * m * m : m * m;
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    const long long p = coarse_node<DIM>(t, g);
    double Au, dg;
    apply_at<DIM, VAR>(u, p, g, s, Au, dg);
    r[t] = f[p] - Au;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < N; j++) acc += ainv[(long long)j * N + t] * r[j];
    const long long p = coarse_node<DIM>(t, g);
    u[p] += acc;
  }
}

// ---------------------------------------------------------------- defect correction

// d_I = f_O - A_O u_O (FP64 arithmetic, cast to the inner storage type),
// plus per-block partial sums of the FP64 residual squared.
template <int DIM, typename Ti, bool VAR>
__global__ void k_dc_residual(const double *__restrict__ u, const double *__restrict__ f, Geo go,
                              Sten<double> s, Ti *__restrict__ d, Geo gi, double *__restrict__ partials) {
  double acc = 0.0;
  for_interior_rows<DIM>(go.n - 2, go, gi, [&](long long p, long long q) {
    double Au, dg;
    apply_at<DIM, VAR>(u, p, go, s, Au, dg);
    double r = f[p] - Au;
    acc += r * r;
    st(d + q, (float)r);
  });
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// u_O += e_I (FP64 update of the outer solution).
template <int DIM, typename Ti>
__global__ void k_dc_update(double *__restrict__ u, Geo go, const Ti *__restrict__ e, Geo gi) {
  Idx t = node_index<DIM>(go);
  if (!t.interior) return;
  long long q = (long long)t.k * gi.sz + (long long)t.j * gi.sy + t.i;
  u[t.p] += (double)ld(e + q);
}

// ---------------------------------------------------------------- layout helpers

template <int DIM, typename T>
__global__ void k_from_dense(const double *__restrict__ src, T *__restrict__ dst, Geo g) {
  Idx t = node_index<DIM>(g);
  if (t.i >= g.n) return;
  long long q = ((long long)t.k * g.n + t.j) * g.n + t.i;
  st(dst + t.p, src[q]);
}

template <int DIM, typename T>
__global__ void k_to_dense(const T *__restrict__ src, double *__restrict__ dst, Geo g) {
  Idx t = node_index<DIM>(g);
  if (t.i >= g.n) return;
  long long q = ((long long)t.k * g.n + t.j) * g.n + t.i;
  dst[q] = (double)ld(src + t.p);
}

template <int DIM, typename T> __global__ void k_zero_interior(T *__restrict__ a, Geo g) {
  Idx t = node_index<DIM>(g);
  if (t.interior) st(a + t.p, 0.0f);
}

template <int DIM, typename T>
__global__ void k_copy_boundary(const T *__restrict__ src, T *__restrict__ dst, Geo g) {
  Idx t = node_index<DIM>(g);
  if (t.i < g.n && !t.interior) dst[t.p] = src[t.p];
}

// Faces from node coefficients: c_d * 2 a b / (a + b); 0 past the last node.
template <int DIM, typename C>
__global__ void k_node_faces(const double *__restrict__ k, Geo gk, C *kx, C *ky, C *kz, Geo g, double c0,
                             double c1, double c2) {
  Idx t = node_index<DIM>(g);
  if (t.i >= g.n) return;
  long long pk = (long long)t.k * gk.sz + (long long)t.j * gk.sy + t.i;
  double a = k[pk];
  int n = g.n;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  if (t.i < n - 1) { double b = k[pk + 1]; fx = c0 * (2.0 * a * b / (a + b)); }
  if (t.j < n - 1) { double b = k[pk + gk.sy]; fy = c1 * (2.0 * a * b / (a + b)); }
  if (DIM == 3 && t.k < n - 1) { double b = k[pk + gk.sz]; fz = c2 * (2.0 * a * b / (a + b)); }
  kx[t.p] = (C)fx;
  ky[t.p] = (C)fy;
  if (DIM == 3) kz[t.p] = (C)fz;
}

// Coarse faces (rediscretisation): along the face's dimension two collinear
// fine faces in series, 2 a b / (a + b); across it, the series values of the
// fine lines at offsets -1, 0, +1 averaged with weights (1/4, 1/2, 1/4) per
// other dimension (centre line only on coarse boundary lines, which no
// interior stencil uses). Accumulated in FP64.
template <int DIM>
__device__ __forceinline__ double coarse_face(const void *ff, bool f64, Geo gf, int d, int I, int J, int K, int nc) {
  const long long sd = d == 0 ? 1 : (d == 1 ? gf.sy : gf.sz);
  const int C3[3] = {I, J, K};
  int oth[2] = {0, 0}, no = 0;  // the dimensions across the face
  for (int g = 0; g < DIM; g++)
    if (g != d) oth[no++] = g;
  double acc = 0.0;
  for (int o2 = -1; o2 <= 1; o2++)
    for (int o1 = -1; o1 <= 1; o1++) {
      int off[2] = {o1, o2};
      double w = 1.0;
      bool skip = false;
      for (int e = 0; e < 2; e++) {
        bool line = e < no && C3[oth[e]] >= 1 && C3[oth[e]] <= nc - 2;
        if (!line) {
          if (off[e] != 0) skip = true;
        } else {
          w *= off[e] == 0 ? 0.5 : 0.25;
        }
      }
      if (skip) continue;
      int q3[3] = {2 * I, 2 * J, 2 * K};
      for (int e = 0; e < no; e++) q3[oth[e]] += off[e];
      long long q = (long long)q3[2] * gf.sz + (long long)q3[1] * gf.sy + q3[0];
      double a = f64 ? ((const double *)ff)[q] : (double)((const float *)ff)[q];
      double b = f64 ? ((const double *)ff)[q + sd] : (double)((const float *)ff)[q + sd];
      acc += w * (2.0 * a * b / (a + b));
    }
  return acc;
}

template <int DIM, typename Cf, typename Cc>
__global__ void k_coarsen_faces(const Cf *fx, const Cf *fy, const Cf *fz, Geo gf, Cc *cx, Cc *cy, Cc *cz,
                                Geo gc) {
  Idx t = node_index<DIM>(gc);
  if (t.i >= gc.n) return;
  int n = gc.n;
  const bool f64 = sizeof(Cf) == 8;
  double vx = 0.0, vy = 0.0, vz = 0.0;
  if (t.i < n - 1) vx = coarse_face<DIM>(fx, f64, gf, 0, t.i, t.j, t.k, n);
  if (t.j < n - 1) vy = coarse_face<DIM>(fy, f64, gf, 1, t.i, t.j, t.k, n);
  if (DIM == 3 && t.k < n - 1) vz = coarse_face<DIM>(fz, f64, gf, 2, t.i, t.j, t.k, n);
  cx[t.p] = (Cc)vx;
  cy[t.p] = (Cc)vy;
  if (DIM == 3) cz[t.p] = (Cc)vz;
}

template <int DIM, typename Cs, typename Cd>
__global__ void k_convert_faces(const Cs *sx, const Cs *sy, const Cs *sz, Geo gs, Cd *dx, Cd *dy, Cd *dz,
                                Geo gd) {
  Idx t = node_index<DIM>(gd);
  if (t.i >= gd.n) return;
  long long q = (long long)t.k * gs.sz + (long long)t.j * gs.sy + t.i;
  dx[t.p] = (Cd)sx[q];
  dy[t.p] = (Cd)sy[q];
  if (DIM == 3) dz[t.p] = (Cd)sz[q];
}

}  // namespace mg
