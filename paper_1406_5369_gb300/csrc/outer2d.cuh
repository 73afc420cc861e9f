// Streaming 2D kernels of the finest level that only need a 3-row window:
//
//   k_dc2d  : the FP64 outer step of defect correction - optional update
//             u_out = u_in + e (FP64, e from the inner cycle; out of place,
//             since neighbouring warps read halo rows of u_in), then the
//             residual r = f - A u of the updated u one row behind, written
//             as the inner defect d (inner storage type), plus per-warp
//             partial sums of r^2 for the outer norm.
//   k_norm2d: per-warp partial sums of (f - A u)^2 (level norm), FP64.
//
// Layout as in fused2d.cuh: a warp owns 128 columns (4 per lane) of which
// lanes 1..30 are written (lanes 0 and 31 are a one-lane halo), and a chunk
// of rows streamed in blocks of 8 through a cp.async ring.
//
// FP64 work per node of k_dc2d: one add for the update and five operations
// for the residual, f - cd u + cx (uw + ue) + cy (us + un) with
// cd = 2 (cx + cy) (two adds, three fused multiply-adds). Squares for the
// norm are taken in FP32 after multiplying the converted residual by a power
// of two (exact), held on the device and re-chosen from each new norm, so the
// sum neither underflows nor overflows while no further FP64 operation is
// spent; the norm is returned as sqrt(sum) divided by that power of two. The
// first residual of a solve (ACC64) sums FP64 squares instead, so the scale
// always comes from a norm of the right magnitude.
#pragma once

#include "fixed.cuh"
#include "fused2d.cuh"

namespace mg {
namespace oz {

using fz::cp_async16;
using fz::cp_async8;
using fz::cp_async_commit;
using fz::cp_async_wait;
using fz::kSlots;

// These kernels keep 8 rows in shared memory, refilled 4 at a time (rows
// t+4..t+7 land while rows t..t+3 are used): half the footprint of the
// fused kernels' ring, so twice as many FP64 warps fit on an SM.
constexpr int kRing = 8;
using fz::kVec;
using fz::shdn;
using fz::shup;
using fz::static_for;

constexpr int kOut = 120;  // columns written per warp strip
constexpr int kWarps = 2;  // warps per block (FP64 rows)

struct ArgsOuter {
  const double *u;      // outer solution (FP64) read
  double *uout;         // updated outer solution (k_dc2d with UPDATE)
  const double *f;      // outer right-hand side (FP64)
  const void *e;        // inner correction (inner storage type), may be NULL
  void *d;              // inner defect (inner storage type), may be NULL
  double *partials;     // one slot per warp
  const float *scale;   // device: power of two applied before squaring (k_dc2d)
  int n, pitch;         // outer grid (FP64 elements)
  int pitchi;           // inner grid pitch (elements)
  int R, nstrips, nchunks;
  double cx, cy, cd;    // stencil: cx = c0/h^2, cy = c1/h^2, cd = 2 (cx + cy)
  int pstride;          // list launches: partial slots per problem
  int k2;               // k_dcx2d: cx = cy = 2^k2
  // List launches of a captured batch step: the problem's live flag in
  // device memory; a block whose problem is no longer live returns at once
  // (NULL: always live).
  const int *live;
};

// List launches (many problems of one size): record fields of problem
// blockIdx.y, including the address of its partial-sum slots.
__device__ __forceinline__ void take_problem(ArgsOuter &a, const ArgsOuter &p) {
  a.u = p.u; a.uout = p.uout; a.f = p.f; a.e = p.e; a.d = p.d;
  a.cx = p.cx; a.cy = p.cy; a.cd = p.cd; a.k2 = p.k2;
  a.partials = p.partials;  // the problem's own slots (at most pstride of them)
}

template <typename Ti> struct InnerLane { static constexpr int bytes = kVec * (int)sizeof(Ti); };

// FP32 <-> FP64 by bit manipulation on the integer pipe, so that the FP64
// pipe (1/64 of the FP32 rate on this GPU) only executes the outer step's
// real FP64 arithmetic. IEEE-754 layouts: float 1+8+23 bits (bias 127),
// double 1+11+52 bits (bias 1023). Values below 2^-126 in magnitude become
// zero (a correction or defect that small is negligible at any tolerance).
__device__ __forceinline__ double f2d_bits(float x) {
  unsigned b = __float_as_uint(x);
  unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  hi = e == 0xffu ? (sign | 0x7ff00000u | (m >> 3)) : hi;
  hi = e == 0u ? sign : hi;
  unsigned lo = e == 0u ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}
// Truncating FP64 -> FP32 (the defect needs only FP32 relative accuracy).
__device__ __forceinline__ float d2f_bits(double x) {
  unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  unsigned sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7ffu) - 896;
  unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  unsigned b = sign | ((unsigned)e << 23) | m;
  b = e <= 0 ? sign : b;
  b = e >= 255 ? (sign | 0x7f800000u | (((hi & 0xfffffu) | lo) != 0u && e == 2047 - 896 ? 0x400000u : 0u)) : b;
  return __uint_as_float(b);
}

__device__ __forceinline__ void load4d(const unsigned char *src, double (&v)[kVec]) {
  double2 a = *(const double2 *)src, b = *(const double2 *)(src + 16);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename Ti> __device__ __forceinline__ void load4i(const unsigned char *src, double (&v)[kVec]) {
  if (sizeof(Ti) == 4) {
    float4 x = *(const float4 *)src;
    v[0] = f2d_bits(x.x); v[1] = f2d_bits(x.y); v[2] = f2d_bits(x.z); v[3] = f2d_bits(x.w);
  } else {
    const bf16 *b = (const bf16 *)src;
    v[0] = f2d_bits(__bfloat162float(b[0])); v[1] = f2d_bits(__bfloat162float(b[1]));
    v[2] = f2d_bits(__bfloat162float(b[2])); v[3] = f2d_bits(__bfloat162float(b[3]));
  }
}

template <typename Ti> __device__ __forceinline__ void store4i(Ti *dst, const float (&v)[kVec]) {
  if (sizeof(Ti) == 4) {
    *(float4 *)dst = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    *(uint2 *)dst = make_uint2(bf16x2_rne_bits(v[0], v[1]), bf16x2_rne_bits(v[2], v[3]));
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- outer step
// LIST: a launch over many problems (records in `list`); the single-problem
// instance keeps its arguments untouched, as the compiler prefers.
template <typename Ti, bool UPDATE, bool ACC64, bool LIST = false>
__global__ void __launch_bounds__(32 * kWarps) k_dc2d(ArgsOuter a, const ArgsOuter *__restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (LIST) {
    if (list[blockIdx.y].live && !*list[blockIdx.y].live) return;
    take_problem(a, list[blockIdx.y]);
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kWarps + wib;
  if (gw >= (long long)a.nstrips * a.nchunks) return;
  const int s = (int)(gw % a.nstrips), ch = (int)(gw / a.nstrips);
  const int n = a.n;
  const int x0 = s * kOut - kVec;
  const int c0 = x0 + kVec * lane;
  const bool col_ok = c0 >= 0 && c0 < a.pitch;
  const bool out_lane = lane >= 1 && lane <= 30 && col_ok;
  const int r0 = ch * a.R, r1 = min(r0 + a.R, n);
  const int tstart = max(r0 - 8, 0);
  const int tend = r1;  // the residual of row r1 - 1 needs row r1
  constexpr int IB = InnerLane<Ti>::bytes;
  constexpr int IBP = IB < 16 ? 16 : IB;  // staging stride for the inner row piece
  unsigned char *su = smem + (size_t)wib * kRing * 32 * (32 + 32 + IBP);
  unsigned char *sf = su + kRing * 32 * 32;
  unsigned char *se = sf + kRing * 32 * 32;
  const Ti *e = (const Ti *)a.e;
  Ti *d = (Ti *)a.d;
  const float scale = ACC64 ? 1.0f : *a.scale;  // FP64 squares need no scale
  const double cx = a.cx, cy = a.cy, cd = a.cd;

  double U[kSlots][kVec], F[kSlots][kVec];
#pragma unroll
  for (int i = 0; i < kSlots; i++)
#pragma unroll
    for (int q = 0; q < kVec; q++) { U[i][q] = 0.0; F[i][q] = 0.0; }
  float acc = 0.0f;
  double acc64 = 0.0;

  auto issue_half = [&](int hb) {
#pragma unroll
    for (int K = 0; K < 4; K++) {
      int row = hb + K;
      int slot = row & (kRing - 1);
      bool ok = col_ok && row >= 0 && row < n && row <= tend;
      long long off = (long long)row * a.pitch + c0;
      const double *us = ok ? a.u + off : a.u;
      const double *fs = ok ? a.f + off : a.f;
      cp_async16(su + (slot * 32 + lane) * 32, us, ok);
      cp_async16(su + (slot * 32 + lane) * 32 + 16, us + 2, ok);
      cp_async16(sf + (slot * 32 + lane) * 32, fs, ok);
      cp_async16(sf + (slot * 32 + lane) * 32 + 16, fs + 2, ok);
      if (UPDATE) {
        long long offi = (long long)row * a.pitchi + c0;
        const Ti *es = ok ? e + offi : e;
        if (IB == 16) cp_async16(se + (slot * 32 + lane) * IBP, es, ok);
        else cp_async8(se + (slot * 32 + lane) * IBP, es, ok);
      }
    }
    cp_async_commit();
  };

  issue_half(tstart);
  for (int tb = tstart; tb <= tend; tb += kSlots) {
    static_for<0, kSlots>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr ((K & 3) == 0) {
        issue_half(t + 4);
        cp_async_wait<1>();
      }
      load4d(su + (K * 32 + lane) * 32, U[K]);
      load4d(sf + (K * 32 + lane) * 32, F[K]);
      if (UPDATE) {
        double ev[kVec];
        load4i<Ti>(se + (K * 32 + lane) * IBP, ev);
#pragma unroll
        for (int q = 0; q < kVec; q++) U[K][q] += ev[q];  // e is 0 on the boundary
        if (t >= r0 && t < r1 && t < n && out_lane) {
          double *dst = a.uout + (long long)t * a.pitch + c0;
          *(double2 *)dst = make_double2(U[K][0], U[K][1]);
          *(double2 *)(dst + 2) = make_double2(U[K][2], U[K][3]);
        }
      }
      // residual of row t - 1
      {
        const int r = t - 1;
        constexpr int sc = (K - 1) & (kSlots - 1), sa = (K - 2) & (kSlots - 1), sb = K;
        double left = shup(U[sc][3]), right = shdn(U[sc][0]);
        bool rowok = r >= 1 && r <= n - 2;
        float rv[kVec];
#pragma unroll
        for (int q = 0; q < kVec; q++) {
          double uw = q == 0 ? left : U[sc][q - 1];
          double ue = q == kVec - 1 ? right : U[sc][q + 1];
          double rr = fma(cy, U[sa][q] + U[sb][q], fma(cx, uw + ue, fma(-cd, U[sc][q], F[sc][q])));
          int c = c0 + q;
          bool ok = rowok && c >= 1 && c <= n - 2;
          rv[q] = ok ? d2f_bits(rr) : 0.0f;
          if (ACC64 && ok && r >= r0 && r < r1 && out_lane) acc64 = fma(rr, rr, acc64);
        }
        if (r >= r0 && r < r1 && out_lane) {
          if (!ACC64) {
#pragma unroll
            for (int q = 0; q < kVec; q++) {
              float sr = rv[q] * scale;
              acc = fmaf(sr, sr, acc);
            }
          }
          if (d) store4i<Ti>(d + (long long)r * a.pitchi + c0, rv);
        }
      }
    });
  }
  cp_async_wait<0>();
  double w = warp_sum(ACC64 ? acc64 : (double)acc);
  if (lane == 0) a.partials[gw] = w;
}

// ------------------------------------------------ exact outer step (c = 2^k)
// The outer step of k_dc2d<Ti, true, ACC64> for a stencil with cx = cy = 2^k2,
// with the residual evaluated exactly in 64-bit fixed point (fixed.cuh)
// instead of five FP64 operations per node. The update u_out = u_in + e is
// the one FP64 addition per node (IEEE rounding, as in k_dc2d). Each row
// gets the warp-wide largest exponent of its updated u and of f / 2^k2 (the
// outer right-hand side is zero on the boundary, so every f value counts);
// the residual of row r uses the largest of rows r-1..r+1, and rows
// converted at a smaller one are shifted down to it. Rows stream through a
// 4-row ring in two-row cp.async groups (half the staging of k_dc2d, so more
// warps stay resident to cover the integer pipeline's latency).
constexpr int kXRing = 4;
template <typename Ti, bool ACC64, bool LIST = false>
__global__ void __launch_bounds__(32 * kWarps) k_dcx2d(ArgsOuter a, const ArgsOuter *__restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (LIST) {
    if (list[blockIdx.y].live && !*list[blockIdx.y].live) return;
    take_problem(a, list[blockIdx.y]);
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kWarps + wib;
  if (gw >= (long long)a.nstrips * a.nchunks) return;
  const int s = (int)(gw % a.nstrips), ch = (int)(gw / a.nstrips);
  const int n = a.n;
  const int x0 = s * kOut - kVec;
  const int c0 = x0 + kVec * lane;
  const bool col_ok = c0 >= 0 && c0 < a.pitch;
  const bool out_lane = lane >= 1 && lane <= 30 && col_ok;
  const int r0 = ch * a.R, r1 = min(r0 + a.R, n);
  const int tstart = max(r0 - 8, 0);
  const int tend = r1;
  constexpr int IB = InnerLane<Ti>::bytes;
  constexpr int IBP = IB < 16 ? 16 : IB;
  unsigned char *su = smem + (size_t)wib * kXRing * 32 * (32 + 32 + IBP);
  unsigned char *sf = su + kXRing * 32 * 32;
  unsigned char *se = sf + kXRing * 32 * 32;
  const Ti *e = (const Ti *)a.e;
  Ti *d = (Ti *)a.d;
  const float scale = ACC64 ? 1.0f : *a.scale;
  const int k2 = a.k2;
  bool colin[kVec];  // interior column
#pragma unroll
  for (int q = 0; q < kVec; q++) colin[q] = c0 + q >= 1 && c0 + q <= n - 2;

  double F[kXRing][kVec];
  long long X[kXRing][kVec];
  int Bu[kXRing], Bf[kXRing];
#pragma unroll
  for (int i = 0; i < kXRing; i++) {
    Bu[i] = Bf[i] = fx::kHead;
#pragma unroll
    for (int q = 0; q < kVec; q++) { X[i][q] = 0; F[i][q] = 0.0; }
  }
  float acc = 0.0f;
  double acc64 = 0.0;

  auto issue_pair = [&](int hb) {
#pragma unroll
    for (int K = 0; K < 2; K++) {
      int row = hb + K;
      int slot = row & (kXRing - 1);
      bool ok = col_ok && row >= 0 && row < n && row <= tend;
      long long off = (long long)row * a.pitch + c0;
      const double *us = ok ? a.u + off : a.u;
      const double *fs = ok ? a.f + off : a.f;
      cp_async16(su + (slot * 32 + lane) * 32, us, ok);
      cp_async16(su + (slot * 32 + lane) * 32 + 16, us + 2, ok);
      cp_async16(sf + (slot * 32 + lane) * 32, fs, ok);
      cp_async16(sf + (slot * 32 + lane) * 32 + 16, fs + 2, ok);
      long long offi = (long long)row * a.pitchi + c0;
      const Ti *es = ok ? e + offi : e;
      if (IB == 16) cp_async16(se + (slot * 32 + lane) * IBP, es, ok);
      else cp_async8(se + (slot * 32 + lane) * IBP, es, ok);
    }
    cp_async_commit();
  };

  issue_pair(tstart);
  for (int tb = tstart; tb <= tend; tb += kXRing) {
    static_for<0, kXRing>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr ((K & 1) == 0) {
        issue_pair(t + 2);  // its slots held rows t - 2, t - 1, already in registers
        cp_async_wait<1>();
      }
      double u[kVec], ev[kVec];
      load4d(su + (K * 32 + lane) * 32, u);
      load4d(sf + (K * 32 + lane) * 32, F[K]);
      load4i<Ti>(se + (K * 32 + lane) * IBP, ev);
#pragma unroll
      for (int q = 0; q < kVec; q++) u[q] += ev[q];  // e is 0 on the boundary
      if (t >= r0 && t < r1 && t < n && out_lane) {
        double *dst = a.uout + (long long)t * a.pitch + c0;
        *(double2 *)dst = make_double2(u[0], u[1]);
        *(double2 *)(dst + 2) = make_double2(u[2], u[3]);
      }
      // exponents of row t (a maximum of 2047 flags Inf/NaN)
      {
        unsigned mu = 0, mf = 0;
#pragma unroll
        for (int q = 0; q < kVec; q++) {
          mu = max(mu, (unsigned)fx::dexp(u[q]));
          mf = max(mf, (unsigned)fx::dexp(F[K][q]));
        }
        mu = __reduce_max_sync(0xffffffffu, mu);
        mf = __reduce_max_sync(0xffffffffu, mf);
        const bool bad = mu == 0x7ffu || mf == 0x7ffu;
        Bu[K] = (bad ? fx::kNonFinite : (int)mu) + fx::kHead;
        Bf[K] = max((int)mf - k2, 0) + fx::kHead;
#pragma unroll
        for (int q = 0; q < kVec; q++) X[K][q] = fx::to_fixed(u[q], Bu[K]);
      }
      // residual of row t - 1
      {
        const int r = t - 1;
        constexpr int sc = (K - 1) & (kXRing - 1), sa = (K - 2) & (kXRing - 1), sb = K;
        const int B = max(max(Bu[sa], Bu[sb]), max(Bu[sc], Bf[sc]));
        long long xa[kVec], xc[kVec], xb[kVec];
        const int da = B - Bu[sa], dc = B - Bu[sc], db = B - Bu[sb];
#pragma unroll
        for (int q = 0; q < kVec; q++) { xa[q] = X[sa][q]; xc[q] = X[sc][q]; xb[q] = X[sb][q]; }
        if (da) {
#pragma unroll
          for (int q = 0; q < kVec; q++) xa[q] = fx::align_down(xa[q], da);
        }
        if (dc) {
#pragma unroll
          for (int q = 0; q < kVec; q++) xc[q] = fx::align_down(xc[q], dc);
        }
        if (db) {
#pragma unroll
          for (int q = 0; q < kVec; q++) xb[q] = fx::align_down(xb[q], db);
        }
        const long long left = fx::shfl_up64(xc[3]), right = fx::shfl_dn64(xc[0]);
        const bool rowok = r >= 1 && r <= n - 2;
        const bool finite = B < fx::kNonFinite;
        const int E0 = B - 1085 + k2;
        const fx::Pow2f p2 = fx::pow2f(E0);
        const double s64 = ACC64 ? __hiloint2double((min(max(E0, -1022), 1023) + 1023) << 20, 0) : 0.0;
        float rv[kVec];
#pragma unroll
        for (int q = 0; q < kVec; q++) {
          const long long xw = q == 0 ? left : xc[q - 1];
          const long long xe = q == kVec - 1 ? right : xc[q + 1];
          const long long S = 4 * xc[q] - (xw + xe) - (xa[q] + xb[q]);
          const long long R = fx::to_fixed(F[sc][q], B + k2) - S;
          const bool ok = rowok && colin[q];
          const float rf = finite ? fx::fixed_to_float(R, p2) : __int_as_float(0x7fc00000);
          rv[q] = ok ? rf : 0.0f;
          if (ACC64 && ok && r >= r0 && r < r1 && out_lane) {
            const double rr = finite ? fx::fixed_to_double(R, s64) : __longlong_as_double(0x7ff8000000000000ll);
            acc64 = fma(rr, rr, acc64);
          }
        }
        if (r >= r0 && r < r1 && out_lane) {
          if (!ACC64) {
#pragma unroll
            for (int q = 0; q < kVec; q++) {
              float sr = rv[q] * scale;
              acc = fmaf(sr, sr, acc);
            }
          }
          if (d) store4i<Ti>(d + (long long)r * a.pitchi + c0, rv);
        }
      }
    });
  }
  cp_async_wait<0>();
  double w = warp_sum(ACC64 ? acc64 : (double)acc);
  if (lane == 0) a.partials[gw] = w;
}

// ---------------------------------------------------------------- level norm
template <typename T>
__global__ void __launch_bounds__(32 * kWarps) k_norm2d(ArgsOuter a) {
  typedef typename CT<T>::type C;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kWarps + wib;
  if (gw >= (long long)a.nstrips * a.nchunks) return;
  const int s = (int)(gw % a.nstrips), ch = (int)(gw / a.nstrips);
  const int n = a.n;
  const int x0 = s * kOut - kVec;
  const int c0 = x0 + kVec * lane;
  const bool col_ok = c0 >= 0 && c0 < a.pitch;
  const bool out_lane = lane >= 1 && lane <= 30 && col_ok;
  const int r0 = ch * a.R, r1 = min(r0 + a.R, n);
  const int tstart = max(r0 - 8, 0);
  const int tend = r1;
  constexpr int LB = fz::Lane<T>::bytes;
  unsigned char *su = smem + (size_t)wib * kRing * 32 * LB * 2;
  unsigned char *sf = su + kRing * 32 * LB;
  const T *u = (const T *)a.u;
  const T *f = (const T *)a.f;
  const C cx = (C)a.cx, cy = (C)a.cy;

  C U[kSlots][kVec], F[kSlots][kVec];
#pragma unroll
  for (int i = 0; i < kSlots; i++)
#pragma unroll
    for (int q = 0; q < kVec; q++) { U[i][q] = 0; F[i][q] = 0; }
  double acc = 0.0;

  auto issue_half = [&](int hb) {
#pragma unroll
    for (int K = 0; K < 4; K++) {
      int row = hb + K;
      int slot = row & (kRing - 1);
      bool ok = col_ok && row >= 0 && row < n && row <= tend;
      long long off = (long long)row * a.pitch + c0;
      fz::stage_row<T>(su + (slot * 32 + lane) * LB, u, off, ok);
      fz::stage_row<T>(sf + (slot * 32 + lane) * LB, f, off, ok);
    }
    cp_async_commit();
  };

  issue_half(tstart);
  for (int tb = tstart; tb <= tend; tb += kSlots) {
    static_for<0, kSlots>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr ((K & 3) == 0) {
        issue_half(t + 4);
        cp_async_wait<1>();
      }
      fz::load_lane<T, C>(su + (K * 32 + lane) * LB, U[K]);
      fz::load_lane<T, C>(sf + (K * 32 + lane) * LB, F[K]);
      const int r = t - 1;
      constexpr int sc = (K - 1) & (kSlots - 1), sa = (K - 2) & (kSlots - 1), sb = K;
      C left = shup(U[sc][3]), right = shdn(U[sc][0]);
      bool rowok = r >= 1 && r <= n - 2 && r >= r0 && r < r1 && out_lane;
#pragma unroll
      for (int q = 0; q < kVec; q++) {
        C uc = U[sc][q];
        C uw = q == 0 ? left : U[sc][q - 1];
        C ue = q == kVec - 1 ? right : U[sc][q + 1];
        C tt = cx * ((uc - uw) + (uc - ue)) + cy * ((uc - U[sa][q]) + (uc - U[sb][q]));
        int c = c0 + q;
        if (rowok && c >= 1 && c <= n - 2) {
          double rr = (double)(F[sc][q] - tt);
          acc += rr * rr;
        }
      }
    });
  }
  cp_async_wait<0>();
  double w = warp_sum(acc);
  if (lane == 0) a.partials[gw] = w;
}

}  // namespace oz

namespace d2 {
// One problem's record for the outer-step list launch (FP64 squares, no scale).
oz::ArgsOuter outer_record(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d);
// k_dc2d over `count` problems of outer size O.n (inner level I): problem i
// writes its per-warp partial sums to partials[i * pstride ...] (at most
// pstride of them; *nparts receives the count). exact (with update): the
// exact fixed-point step k_dcx2d; every record's k2 must then hold its
// stencil's power-of-two exponent.
cudaError_t dc_step_list(const Level &O, const Level &I, const oz::ArgsOuter *list, int count, double *partials,
                         int pstride, int *nparts, bool update, bool exact, cudaStream_t s);
}  // namespace d2
}  // namespace mg

