// Plane-marching 3D kernels for the constant 7-point stencil (Algorithm 1's
// level operators on 3D grids, Sec. 2.2-2.4):
//
//   k3_stencil<T, kJacobi>: one omega-Jacobi sweep (u_out from u_in);
//   k3_stencil<T, kRB>   : one red-black half-sweep (in place, one colour);
//   k3_stencil<T, kResid>: residual r = f - A u;
//   k3_stencil<T, kNorm> : per-block partial sums of (f - A u)^2;
//   k3_restrict<T>       : full weighting r_h -> f_H;
//   k3_prolong<T>        : trilinear interpolation and correction u_h += P e_H;
//   k3_dc<Ti, ...>       : the FP64 outer step of defect correction (update
//                          u_out = u_in + e, residual of the updated u written
//                          as the inner defect, partial sums of its square).
//
// Decomposition of the marching kernels: a block owns kTY = 8 consecutive
// interior rows y0 .. y0+7 of one x-tile of 32 V columns (V = 16 bytes / element
// size: 8 BF16, 4 FP32 or 2 FP64 values per lane, one 16-byte vector) and a
// chunk of planes z0 .. z1-1, and walks the chunk plane by plane. Each plane
// of the tile, with one halo row above and below and one 16-byte halo chunk
// left and right, is staged by cp.async into a ring of kRingZ plane slots in
// shared memory, kAhead planes ahead of the plane being computed; one
// __syncthreads per plane publishes the staged plane and frees the oldest
// slot. A warp keeps its own row at planes z-1, z, z+1 in registers and reads
// rows y-1, y+1 and the x-halo values of plane z from the staged tile; the
// x-neighbours inside the segment come from warp shuffles. Arithmetic runs in
// float for BF16/FP32 storage and in double for FP64 storage.
#pragma once

#include "fixed.cuh"
#include "fused2d.cuh"
#include "outer2d.cuh"

namespace mg {
namespace z3 {

using fz::cp_async16;
using fz::cp_async_commit;
using fz::cp_async_wait;
using fz::shdn;
using fz::shup;

constexpr int kTY = 8;                     // rows (warps) per block
constexpr int kAhead = 3;                  // planes staged ahead of the computed plane
constexpr int kRingZ = kAhead + 3;         // plane slots: z-1, z, z+1 and the planes in flight
constexpr int kUChunks = 34;               // 16-byte chunks per staged u row: halo, 32 lanes, halo
constexpr int kURowB = kUChunks * 16;
constexpr int kFRowB = 32 * 16;
constexpr int kSlotB = (kTY + 2) * kURowB + kTY * kFRowB;

template <typename T> struct VW { static constexpr int V = 16 / (int)sizeof(T); };

// 16-byte vectors <-> compute type.
__device__ __forceinline__ void vld(const double *p, double (&v)[2]) {
  double2 a = *(const double2 *)p;
  v[0] = a.x; v[1] = a.y;
}
__device__ __forceinline__ void vld(const float *p, float (&v)[4]) {
  float4 a = *(const float4 *)p;
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
// BF16 -> FP32 is exact: the 16 bits are the top half of the float.
__device__ __forceinline__ void vld(const bf16 *p, float (&v)[8]) {
  uint4 a = *(const uint4 *)p;
  unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int k = 0; k < 4; k++) {
    v[2 * k] = __uint_as_float(w[k] << 16);
    v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
  }
}
__device__ __forceinline__ void vst(double *p, const double (&v)[2]) { *(double2 *)p = make_double2(v[0], v[1]); }
__device__ __forceinline__ void vst(float *p, const float (&v)[4]) { *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]); }
__device__ __forceinline__ void vst(bf16 *p, const float (&v)[8]) {
  *(uint4 *)p = make_uint4(bf16x2_rne_bits(v[0], v[1]), bf16x2_rne_bits(v[2], v[3]), bf16x2_rne_bits(v[4], v[5]),
                           bf16x2_rne_bits(v[6], v[7]));
}
template <typename T> __device__ __forceinline__ typename CT<T>::type sld(const unsigned char *p) {
  return (typename CT<T>::type)ld((const T *)p);
}

struct Args3 {
  const void *u;      // solution read (in place for a red-black half-sweep)
  void *out;          // sweep: solution written; residual: r
  const void *f;      // right-hand side
  double *partials;   // norm: one partial sum per block
  int n, pitch;       // nodes per dimension, row stride (elements)
  long long plane;    // plane stride (elements)
  int ntx, nty, zc;   // x-tiles, y-tiles of kTY rows, planes per chunk
  int color;          // red-black half-sweep: colour to update
  double alpha, bx, by, bz, gamma;  // sweep: u' = gamma u + alpha f + bx (uw+ue) + by (us+un) + bz (ud+uu)
  double cd, cx, cy, cz;            // residual: r = f - cd u + cx (uw+ue) + cy (us+un) + cz (ud+uu)
  // The same, rounded to FP32 on the host (read by the FP32-arithmetic kernels).
  float alphaf, bxf, byf, bzf, gammaf, cdf, cxf, cyf, czf;
  int has_gamma;  // gamma != 0 (omega != 1), decided on the host
  // List launches of a captured batch step: the problem's live flag in
  // device memory; a block whose problem is no longer live returns at once
  // (NULL: always live).
  const int *live;
};

// List launches (many problems of one size, the batch engine): blockIdx.z
// is the problem; a block takes its record's fields and coefficients, the
// grid geometry stays that of the launch argument.
__device__ __forceinline__ void take_problem(Args3 &a, const Args3 &p) {
  a.u = p.u; a.out = p.out; a.f = p.f;
  a.alpha = p.alpha; a.bx = p.bx; a.by = p.by; a.bz = p.bz; a.gamma = p.gamma;
  a.cd = p.cd; a.cx = p.cx; a.cy = p.cy; a.cz = p.cz;
  a.alphaf = p.alphaf; a.bxf = p.bxf; a.byf = p.byf; a.bzf = p.bzf; a.gammaf = p.gammaf;
  a.cdf = p.cdf; a.cxf = p.cxf; a.cyf = p.cyf; a.czf = p.czf; a.has_gamma = p.has_gamma;
}

// kJZ: two omega-Jacobi sweeps from u = 0 in one pass. The first sweep of a
// zero start gives alpha f at interior nodes and keeps the (zero) boundary,
// so the pass stages f in place of u, scales every value by alpha as it is
// read (the first sweep's rounding), and applies the second sweep to that.
// Needs f = 0 on the boundary, as on every coarse level and on the inner
// finest level of defect correction.
enum { kJacobi = 0, kRB = 1, kResid = 2, kNorm = 3, kJZ = 4 };

// The 16-byte pieces a thread stages for every plane, fixed for the whole
// march: source address at plane 0, byte stride between planes, shared-memory
// offset inside a slot and whether the piece lies inside its array.
// issue() stages consecutive planes: it is called first with plane `first`
// (start()), then with each following plane, so the source addresses advance
// by one plane stride per call instead of being recomputed. Pieces outside
// their array keep a valid address and a zero stride and copy nothing.
template <int K> struct Pieces {
  const unsigned char *src[K];
  const unsigned char *anchor;  // a valid address handed to zero-filled copies
  long long pstep[K];
  int soff[K];  // -1: no piece
  bool ok[K];
  __device__ __forceinline__ void start(int first) {
#pragma unroll
    for (int k = 0; k < K; k++) src[k] += (long long)first * pstep[k];
  }
  // Stages the current plane into `slot` (zero-fill unless `pok`, which is
  // the same for the whole block), then advances.
  __device__ __forceinline__ void issue(unsigned char *slot, bool pok) {
    if (pok) {
#pragma unroll
      for (int k = 0; k < K; k++)
        if (soff[k] >= 0) cp_async16(slot + soff[k], src[k], ok[k]);
    } else {
#pragma unroll
      for (int k = 0; k < K; k++)
        if (soff[k] >= 0) cp_async16(slot + soff[k], anchor, false);
    }
#pragma unroll
    for (int k = 0; k < K; k++) src[k] += pstep[k];
    cp_async_commit();
  }
};

// The stencil kernels' pieces all advance by the same plane stride, so they
// share one; a piece outside its array issues a zero-filling copy of a valid
// address instead (a per-piece branch, no 64-bit selects).
template <int K> struct Pieces1 {
  const unsigned char *src[K];
  const unsigned char *anchor;
  long long pstep;
  int soff[K];  // -1: no piece
  bool ok[K];
  __device__ __forceinline__ void start(int first) {
#pragma unroll
    for (int k = 0; k < K; k++) src[k] += (long long)first * pstep;
  }
  __device__ __forceinline__ void issue(unsigned char *slot, bool pok) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (soff[k] >= 0) {
        if (ok[k] && pok) cp_async16(slot + soff[k], src[k], true);
        else cp_async16(slot + soff[k], anchor, false);
      }
      src[k] += pstep;
    }
    cp_async_commit();
  }
};

// Pieces of the stencil kernels' tile: u rows y0-1 .. y0+kTY (34 chunks each:
// left halo, 32 lanes, right halo), f rows y0 .. y0+kTY-1 (32 chunks).
constexpr int kStPieces = ((kTY + 2) * kUChunks + kTY * 32 + 32 * kTY - 1) / (32 * kTY);
template <typename T>
__device__ __forceinline__ void stencil_pieces(Pieces1<kStPieces> &pc, const T *u, const T *f, int y0, int x0, int n,
                                               int pitch, long long P) {
  constexpr int V = VW<T>::V;
  constexpr int NU = (kTY + 2) * kUChunks, NF = kTY * 32;
  pc.anchor = (const unsigned char *)u;
  pc.pstep = P * (long long)sizeof(T);
#pragma unroll
  for (int k = 0; k < kStPieces; k++) {
    const int i = threadIdx.x + k * 32 * kTY;
    pc.soff[k] = -1;
    pc.ok[k] = false;
    pc.src[k] = (const unsigned char *)u;
    if (i < NU) {
      const int rr = i / kUChunks, ch = i - rr * kUChunks;
      const int y = y0 - 1 + rr, x = x0 + (ch - 1) * V;
      pc.ok[k] = y >= 0 && y < n && x >= 0 && x + V <= pitch;
      if (pc.ok[k]) pc.src[k] = (const unsigned char *)(u + (long long)y * pitch + x);
      pc.soff[k] = rr * kURowB + ch * 16;
    } else if (i < NU + NF) {
      const int j = i - NU, rr = j >> 5, ch = j & 31;
      const int y = y0 + rr, x = x0 + ch * V;
      pc.ok[k] = y < n && x + V <= pitch;
      pc.src[k] = (const unsigned char *)(pc.ok[k] ? f + (long long)y * pitch + x : f);
      pc.soff[k] = (kTY + 2) * kURowB + rr * kFRowB + ch * 16;
    }
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(32 * kTY, MODE == kResid ? 2 : 3) k3_stencil(Args3 a, const Args3 *__restrict__ list) {
  typedef typename CT<T>::type C;
  constexpr int V = VW<T>::V;
  constexpr int TX = 32 * V;
  constexpr int RB = kRingZ * kSlotB;  // ring bytes
  extern __shared__ __align__(16) unsigned char smem[];
  if (list) {
    if (list[blockIdx.z].live && !*list[blockIdx.z].live) return;
    take_problem(a, list[blockIdx.z]);
  }
  __shared__ double wsum[kTY];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tx = blockIdx.x % a.ntx, ty = blockIdx.x / a.ntx;
  const int n = a.n, pitch = a.pitch;
  const long long P = a.plane;
  const int y0 = 1 + ty * kTY, y = y0 + w;
  const int x0 = tx * TX, cl = x0 + V * lane;
  const int z0 = 1 + blockIdx.y * a.zc, z1 = min(z0 + a.zc, n - 1);
  const bool wact = y <= n - 2;  // warp-uniform
  const C alpha = pick<C>(a.alpha, a.alphaf), bx = pick<C>(a.bx, a.bxf), by = pick<C>(a.by, a.byf);
  const C bz = pick<C>(a.bz, a.bzf), gamma = pick<C>(a.gamma, a.gammaf);
  const C cd = pick<C>(a.cd, a.cdf), cx = pick<C>(a.cx, a.cxf), cy = pick<C>(a.cy, a.cyf), cz = pick<C>(a.cz, a.czf);
  const bool has_gamma = a.has_gamma != 0;
  double acc = 0.0;

  // shared-memory byte offsets inside a slot (32-bit)
  const int own = (w + 1) * kURowB + (lane + 1) * 16;
  const int above = own - kURowB, below = own + kURowB;
  const int frw = (kTY + 2) * kURowB + w * kFRowB + lane * 16;
  const int halo = (w + 1) * kURowB + (lane == 0 ? 16 - (int)sizeof(T) : 33 * 16);

  Pieces1<kStPieces> pc;
  stencil_pieces<T>(pc, (const T *)a.u, (const T *)a.f, y0, x0, n, pitch, P);
  // Planes z0 - 1 .. z0 + kAhead up front; step z then refills with z + kAhead + 1.
  // Ring slot of plane p: p % kRingZ, tracked as byte offsets.
  int so_fill = ((z0 - 1) % kRingZ) * kSlotB;
  auto advance = [](int o) { return o + kSlotB == RB ? 0 : o + kSlotB; };
  pc.start(z0 - 1);
  for (int k = 0; k <= kAhead + 1; k++) {
    pc.issue(smem + so_fill, z0 - 1 + k <= z1);
    so_fill = advance(so_fill);
  }
  // Most lanes have all V columns inside the domain and skip the boundary
  // fix-ups below (the same on every plane).
  const bool lane_in = cl >= 1 && cl + V - 1 <= n - 2;
  T *outp = (T *)a.out + (long long)z0 * P + (long long)y * pitch + cl;
  int so_cur = (z0 % kRingZ) * kSlotB, so_next = advance(so_cur);

  // um, uc: planes z - 1 and z of the own row; up receives plane z + 1.
  C um[V], uc[V], up[V];
  cp_async_wait<kAhead - 1>();
  __syncthreads();
  // kJZ: the staged "u" values are f; the first sweep's result is alpha f at
  // interior nodes and zero on the boundary (bnd: the row or plane is a
  // boundary one; boundary columns of the lane masked here)
  auto first = [&](C (&v)[V], bool bnd) {
    if (MODE == kJZ) {
#pragma unroll
      for (int q = 0; q < V; q++) v[q] = (bnd || cl + q == 0 || cl + q == n - 1) ? (C)0 : alpha * v[q];
    }
  };
  if (wact) {
    vld((const T *)(smem + own + (so_cur == 0 ? RB - kSlotB : so_cur - kSlotB)), um);
    vld((const T *)(smem + own + so_cur), uc);
    first(um, z0 - 1 == 0);
    first(uc, false);
  }
  for (int z = z0; z < z1; z++) {
    cp_async_wait<kAhead - 1>();  // planes up to z + 1 have landed (own copies)
    __syncthreads();              // ... everyone's, and nobody still reads plane z - 2
    C ys[V], yn[V], fc[V];
    C hx = 0;
    if (wact) {
      vld((const T *)(smem + own + so_next), up);
      vld((const T *)(smem + above + so_cur), ys);
      vld((const T *)(smem + below + so_cur), yn);
      vld((const T *)(smem + frw + so_cur), fc);
      if (lane == 0 || lane == 31) hx = sld<T>(smem + halo + so_cur);
      first(up, z + 1 == n - 1);
      first(ys, y - 1 == 0);
      first(yn, y + 1 == n - 1);
      if (MODE == kJZ) {
        const int hc = lane == 0 ? cl - 1 : cl + V;
        hx = (hc <= 0 || hc >= n - 1) ? (C)0 : alpha * hx;
      }
    }
    // the slot of plane z + kAhead + 1 held plane z - 2
    pc.issue(smem + so_fill, z + kAhead + 1 <= z1);
    so_fill = advance(so_fill);
    so_cur = so_next;
    so_next = advance(so_next);
    if (!wact) continue;
    C wl = shup(uc[V - 1]), er = shdn(uc[0]);
    if (lane == 0) wl = hx;
    if (lane == 31) er = hx;
    C res[V];
    auto nbr = [&](int q, C &wv, C &ev) {
      wv = q == 0 ? wl : uc[q - 1];
      ev = q == V - 1 ? er : uc[q + 1];
    };
    if (MODE == kJacobi || MODE == kRB || MODE == kJZ) {
      auto relax = [&](int q) {
        C wv, ev;
        nbr(q, wv, ev);
        C nv = alpha * fc[q] + bx * (wv + ev) + by * (ys[q] + yn[q]) + bz * (um[q] + up[q]);
        if (has_gamma) nv += gamma * uc[q];
        return nv;
      };
      if (MODE == kJacobi || MODE == kJZ) {
#pragma unroll
        for (int q = 0; q < V; q++) res[q] = relax(q);
      } else {
        // cl is even, so column cl + q has this half-sweep's colour iff q has
        // the parity of rbpar (warp-uniform): only those columns are computed
        const int rbpar = (y + z + a.color) & 1;
        if (rbpar == 0) {
#pragma unroll
          for (int q = 0; q < V; q++) res[q] = (q & 1) ? uc[q] : relax(q);
        } else {
#pragma unroll
          for (int q = 0; q < V; q++) res[q] = (q & 1) ? relax(q) : uc[q];
        }
      }
      if (!lane_in) {
#pragma unroll
        for (int q = 0; q < V; q++)
          if (cl + q < 1 || cl + q > n - 2) res[q] = uc[q];
      }
    } else {
      C sq = 0;
#pragma unroll
      for (int q = 0; q < V; q++) {
        C wv, ev;
        nbr(q, wv, ev);
        const C rr = fc[q] - cd * uc[q] + cx * (wv + ev) + cy * (ys[q] + yn[q]) + cz * (um[q] + up[q]);
        const bool in = cl + q >= 1 && cl + q <= n - 2;
        res[q] = in ? rr : (C)0;
        if (MODE == kNorm) sq += res[q] * res[q];
      }
      if (MODE == kNorm) acc += (double)sq;
    }
    if (MODE != kNorm && cl < pitch) vst(outp, res);
    outp += P;
#pragma unroll
    for (int q = 0; q < V; q++) { um[q] = uc[q]; uc[q] = up[q]; }
  }
  cp_async_wait<0>();
  if (MODE == kNorm) {
    double s = oz::warp_sum(acc);
    if (lane == 0) wsum[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < kTY; i++) t += wsum[i];
      a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
  }
}

// ---------------------------------------------------------------- transfers

struct ArgsT3 {
  const void *src;    // restrict: fine residual; prolong: coarse correction
  void *dst;          // restrict: coarse right-hand side; prolong: fine solution (in place)
  int nf, pitchf;     // fine grid
  long long planef;
  int nc, pitchc;     // coarse grid
  long long planec;
  int ntx;            // x-tiles (of the grid the warps run over)
  // List launches of a captured batch step: the problem's live flag in
  // device memory; a block whose problem is no longer live returns at once
  // (NULL: always live).
  const int *live;
};

// Full weighting at coarse interior nodes: a warp covers 16 V coarse columns
// (V / 2 per lane, from one 16-byte vector of V fine values per fine row),
// for one coarse row J and plane K; blocks hold kTY consecutive rows.
template <typename T>
__global__ void __launch_bounds__(32 * kTY) k3_restrict(ArgsT3 a, const ArgsT3 *__restrict__ list) {
  if (list) {
    if (list[blockIdx.z].live && !*list[blockIdx.z].live) return;
    a.src = list[blockIdx.z].src;
    a.dst = list[blockIdx.z].dst;
  }
  typedef typename CT<T>::type C;
  constexpr int V = VW<T>::V, VC = V / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tx = blockIdx.x % a.ntx, jt = blockIdx.x / a.ntx;
  const int J = 1 + jt * kTY + w, K = 1 + blockIdx.y;
  if (J > a.nc - 2) return;
  const int X0 = tx * 16 * V, I0 = X0 + VC * lane;  // first coarse column of this lane
  const int xf = 2 * I0;                              // its fine column
  const bool lact = xf + V <= a.pitchf;
  const T *rf = (const T *)a.src;
  C acc[VC];
#pragma unroll
  for (int q = 0; q < VC; q++) acc[q] = 0;
#pragma unroll
  for (int dz = -1; dz <= 1; dz++) {
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
      const C wyz = (dz == 0 ? (C)0.5 : (C)0.25) * (dy == 0 ? (C)0.5 : (C)0.25);
      const T *row = rf + (long long)(2 * K + dz) * a.planef + (long long)(2 * J + dy) * a.pitchf;
      C v[V];
      if (lact) vld(row + xf, v);
      else {
#pragma unroll
        for (int q = 0; q < V; q++) v[q] = 0;
      }
      C left = shup(v[V - 1]);
      if (lane == 0) left = xf >= 1 ? (C)ld(row + xf - 1) : (C)0;
#pragma unroll
      for (int q = 0; q < VC; q++) {
        const C a0 = q == 0 ? left : v[2 * q - 1];
        acc[q] += wyz * ((C)0.25 * (a0 + v[2 * q + 1]) + (C)0.5 * v[2 * q]);
      }
    }
  }
  T *fc = (T *)a.dst + (long long)K * a.planec + (long long)J * a.pitchc;
#pragma unroll
  for (int q = 0; q < VC; q++) {
    const int I = I0 + q;
    if (I >= 1 && I <= a.nc - 2) st(fc + I, acc[q]);
  }
}

// Trilinear interpolation and correction at fine interior nodes: a warp
// covers 32 V fine columns of one fine row j and plane k.
template <typename T>
__global__ void __launch_bounds__(32 * kTY) k3_prolong(ArgsT3 a, const ArgsT3 *__restrict__ list) {
  if (list) {
    if (list[blockIdx.z].live && !*list[blockIdx.z].live) return;
    a.src = list[blockIdx.z].src;
    a.dst = list[blockIdx.z].dst;
  }
  typedef typename CT<T>::type C;
  constexpr int V = VW<T>::V, VC = V / 2;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tx = blockIdx.x % a.ntx, jt = blockIdx.x / a.ntx;
  const int j = 1 + jt * kTY + w, k = 1 + blockIdx.y;
  if (j > a.nf - 2) return;
  const int cl = tx * 32 * V + V * lane;  // first fine column (even)
  if (cl >= a.pitchf) return;             // whole lane outside the row: no shuffles below read it
  const int Ic = cl >> 1;
  const int J = j >> 1, Kc = k >> 1, oj = j & 1, ok = k & 1;
  const T *ec = (const T *)a.src;
  C e[VC + 1];
#pragma unroll
  for (int q = 0; q <= VC; q++) e[q] = 0;
  const C wgt = (oj ? (C)0.5 : (C)1) * (ok ? (C)0.5 : (C)1);
#pragma unroll
  for (int dk = 0; dk <= 1; dk++) {
    if (dk && !ok) break;
#pragma unroll
    for (int dj = 0; dj <= 1; dj++) {
      if (dj && !oj) break;
      const T *row = ec + (long long)(Kc + dk) * a.planec + (long long)(J + dj) * a.pitchc + Ic;
#pragma unroll
      for (int q = 0; q <= VC; q++) {
        const int I = Ic + q;
        if (I < a.nc) e[q] += (C)ld(row + q);
      }
    }
  }
  T *uf = (T *)a.dst + (long long)k * a.planef + (long long)j * a.pitchf + cl;
  C u[V];
  vld(uf, u);
#pragma unroll
  for (int q = 0; q < V; q++) {
    const int c = cl + q;
    const C ev = (q & 1) ? (C)0.5 * (e[q >> 1] + e[(q >> 1) + 1]) : e[q >> 1];
    if (c >= 1 && c <= a.nf - 2) u[q] += wgt * ev;
  }
  vst(uf, u);
}

// ---------------------------------------------------------------- FP64 outer step

// Block of kTY + 2 warps: rows y0-1 .. y0+kTY (the first and last only update
// their row so that the others see updated y-neighbours). Per plane, staged
// by cp.async kAhead planes ahead: u_in and e for all kTY + 2 rows (with
// 16-byte halo chunks), f for the kTY output rows. Step z updates plane z + 1
// (u_new = u_in + e, FP64; written to u_out and to a 3-slot ring of updated
// rows in shared memory) and, after a barrier, forms the residual of plane z
// from updated values only: FP64 work per node is one add for the update and
// seven operations for the residual f - cd u + cx (uw+ue) + cy (us+un) + cz (ud+uu).
constexpr int kDCWarps = kTY + 2;
constexpr int kDCRing = kAhead + 2;
template <typename Ti> struct DCL {
  static constexpr int ECH = 64 * (int)sizeof(Ti) / 16;  // 16-byte chunks of e per 64-column row
  static constexpr int ERowB = (ECH + 2) * 16;
  static constexpr int SlotB = kDCWarps * kURowB + kDCWarps * ERowB + kTY * kFRowB;
  static constexpr int UNRowB = 64 * 8;
  static constexpr int Smem = kDCRing * SlotB + 3 * kDCWarps * UNRowB;
};

struct ArgsDC3 {
  const double *u;     // outer solution read
  double *uout;        // updated outer solution (UPDATE)
  const double *f;     // outer right-hand side
  const void *e;       // inner correction (inner storage type)
  void *d;             // inner defect (inner storage type), may be NULL
  double *partials;    // one per block
  const float *scale;  // power of two applied before the FP32 squares
  int n, pitch, pitchi;
  long long plane, planei;
  int ntx, nty, zc;
  double cd, cx, cy, cz;
  int pstride;         // list launches: partial slots per problem
  int k2;              // k3_dcx: cx = cy = cz = 2^k2
  // List launches of a captured batch step: the problem's live flag in
  // device memory; a block whose problem is no longer live returns at once
  // (NULL: always live).
  const int *live;
};

// Pieces of the outer step's tile: u and e rows y0-1 .. y0+kTY with halo
// chunks, f rows y0 .. y0+kTY-1.
template <typename Ti, bool UPDATE> struct DCP {
  static constexpr int NU = kDCWarps * kUChunks, NE = UPDATE ? kDCWarps * (DCL<Ti>::ECH + 2) : 0, NF = kTY * 32;
  static constexpr int K = (NU + NE + NF + 32 * kDCWarps - 1) / (32 * kDCWarps);
};
template <typename Ti, bool UPDATE>
__device__ __forceinline__ void dc_pieces(Pieces<DCP<Ti, UPDATE>::K> &pc, const ArgsDC3 &a, int y0, int x0) {
  typedef DCL<Ti> L;
  typedef DCP<Ti, UPDATE> Q;
  constexpr int EV = 16 / (int)sizeof(Ti);  // e values per chunk
  const Ti *e = (const Ti *)a.e;
  pc.anchor = (const unsigned char *)a.u;
#pragma unroll
  for (int k = 0; k < Q::K; k++) {
    const int i = threadIdx.x + k * 32 * kDCWarps;
    pc.soff[k] = -1;
    pc.ok[k] = false;
    pc.src[k] = (const unsigned char *)a.u;
    long long step = a.plane * 8;
    if (i < Q::NU) {
      const int rr = i / kUChunks, ch = i - rr * kUChunks;
      const int y = y0 - 1 + rr, x = x0 + (ch - 1) * 2;
      pc.ok[k] = y >= 0 && y < a.n && x >= 0 && x + 2 <= a.pitch;
      if (pc.ok[k]) pc.src[k] = (const unsigned char *)(a.u + (long long)y * a.pitch + x);
      pc.soff[k] = rr * kURowB + ch * 16;
    } else if (i < Q::NU + Q::NE) {
      const int j = i - Q::NU, rr = j / (L::ECH + 2), ch = j - rr * (L::ECH + 2);
      const int y = y0 - 1 + rr, x = x0 + (ch - 1) * EV;
      pc.ok[k] = y >= 0 && y < a.n && x >= 0 && x + EV <= a.pitchi;
      pc.src[k] = (const unsigned char *)(pc.ok[k] ? e + (long long)y * a.pitchi + x : e);
      step = a.planei * (long long)sizeof(Ti);
      pc.soff[k] = kDCWarps * kURowB + rr * L::ERowB + ch * 16;
    } else if (i < Q::NU + Q::NE + Q::NF) {
      const int j = i - Q::NU - Q::NE, rr = j >> 5, ch = j & 31;
      const int y = y0 + rr, x = x0 + ch * 2;
      pc.ok[k] = y < a.n && x + 2 <= a.pitch;
      pc.src[k] = (const unsigned char *)(pc.ok[k] ? a.f + (long long)y * a.pitch + x : a.f);
      pc.soff[k] = kDCWarps * kURowB + kDCWarps * L::ERowB + rr * kFRowB + ch * 16;
    }
    pc.pstep[k] = pc.ok[k] ? step : 0;
  }
}

template <typename Ti> __device__ __forceinline__ double e_at(const unsigned char *p) {
  return oz::f2d_bits(sizeof(Ti) == 4 ? *(const float *)p : __bfloat162float(*(const bf16 *)p));
}

template <typename Ti, bool UPDATE, bool ACC64>
__global__ void __launch_bounds__(32 * kDCWarps) k3_dc(ArgsDC3 a, const ArgsDC3 *__restrict__ list) {
  typedef DCL<Ti> L;
  extern __shared__ __align__(16) unsigned char smem[];
  if (list) {  // problem blockIdx.z of a list launch
    const ArgsDC3 &p = list[blockIdx.z];
    if (p.live && !*p.live) return;
    a.u = p.u; a.uout = p.uout; a.f = p.f; a.e = p.e; a.d = p.d;
    a.cd = p.cd; a.cx = p.cx; a.cy = p.cy; a.cz = p.cz;
    a.partials = p.partials;  // the problem's own slots (at most pstride of them)
  }
  __shared__ double wsum[kDCWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // w = 0 .. kTY + 1: row y0 - 1 + w
  const int tx = blockIdx.x % a.ntx, ty = blockIdx.x / a.ntx;
  const int n = a.n;
  const int y0 = 1 + ty * kTY, y = y0 - 1 + w;
  const int x0 = tx * 64, cl = x0 + 2 * lane;
  const int z0 = 1 + blockIdx.y * a.zc, z1 = min(z0 + a.zc, n - 1);
  const bool out_warp = w >= 1 && w <= kTY && y <= n - 2;  // residual rows (interior)
  const bool row_ok = y <= n - 1;
  unsigned char *un = smem + kDCRing * L::SlotB;  // 3 slots x kDCWarps rows of updated u
  auto slot = [&](int p) { return smem + (p % kDCRing) * L::SlotB; };
  const float scale = ACC64 ? 1.0f : *a.scale;  // FP64 squares need no scale
  const double cd = a.cd, cx = a.cx, cy = a.cy, cz = a.cz;
  Ti *d = (Ti *)a.d;
  float acc = 0.0f;
  double acc64 = 0.0;

  // Updated u of this warp's row at plane p: own two values and the x-halo
  // value (lane 0: column x0 - 1, lane 31: column x0 + 64).
  auto update_row = [&](int p, double (&v)[2], double &h) {
    const unsigned char *s = slot(p + kDCRing);
    const unsigned char *ur = s + w * kURowB;
    vld((const double *)(ur + (lane + 1) * 16), v);
    h = 0.0;
    if (lane == 0) h = *(const double *)(ur + 8);
    if (lane == 31) h = *(const double *)(ur + 33 * 16);
    if (UPDATE) {
      const unsigned char *er = s + kDCWarps * kURowB + w * L::ERowB;
      const unsigned char *mine = er + 16 + lane * 2 * sizeof(Ti);
      v[0] += e_at<Ti>(mine);
      v[1] += e_at<Ti>(mine + sizeof(Ti));
      if (lane == 0) h += e_at<Ti>(er + 16 - sizeof(Ti));
      if (lane == 31) h += e_at<Ti>(er + 16 + 64 * sizeof(Ti));
    }
  };

  Pieces<DCP<Ti, UPDATE>::K> pc;
  dc_pieces<Ti, UPDATE>(pc, a, y0, x0);
  const int zs = z0 - 2;  // first step: updates plane z0 - 1
  pc.start(zs + 1);
  for (int k = 1; k <= kAhead; k++) {
    const int p = zs + k;
    pc.issue(slot(p + kDCRing), p <= z1);
  }

  double um[2] = {0, 0}, uc[2] = {0, 0}, up[2] = {0, 0};
  double hc = 0, hp = 0;
  for (int z = zs; z < z1; z++) {
    cp_async_wait<kAhead - 1>();  // plane z + 1 staged
    __syncthreads();              // (A) for everyone; plane z - 1's slot is free
    pc.issue(slot(z + kAhead + 1 + kDCRing), z + kAhead + 1 <= z1);
    double nv[2] = {0, 0}, nh = 0;
    if (row_ok) {
      update_row(z + 1, nv, nh);
      *(double2 *)(un + (((z + 1) % 3 + 3) % 3 * kDCWarps + w) * L::UNRowB + lane * 16) = make_double2(nv[0], nv[1]);
      if (UPDATE && out_warp && z + 1 >= z0 && z + 1 < z1 && cl < a.pitch)
        *(double2 *)(a.uout + (long long)(z + 1) * a.plane + (long long)y * a.pitch + cl) = make_double2(nv[0], nv[1]);
    }
    __syncthreads();  // (B) updated rows of plane z + 1 visible
    um[0] = uc[0]; um[1] = uc[1];
    uc[0] = up[0]; uc[1] = up[1];
    up[0] = nv[0]; up[1] = nv[1];
    hc = hp; hp = nh;
    if (z >= z0 && out_warp) {
      const unsigned char *us = un + ((z % 3 + 3) % 3 * kDCWarps + (w - 1)) * L::UNRowB + lane * 16;
      const unsigned char *un_ = un + ((z % 3 + 3) % 3 * kDCWarps + (w + 1)) * L::UNRowB + lane * 16;
      const double2 s2 = *(const double2 *)us, n2 = *(const double2 *)un_;
      const double2 f2 = *(const double2 *)(slot(z + kDCRing) + kDCWarps * kURowB + kDCWarps * L::ERowB +
                                             (w - 1) * kFRowB + lane * 16);
      double wl = shup(uc[1]), er = shdn(uc[0]);
      if (lane == 0) wl = hc;
      if (lane == 31) er = hc;
      const double ysv[2] = {s2.x, s2.y}, ynv[2] = {n2.x, n2.y}, fv[2] = {f2.x, f2.y};
      float rv[2];
#pragma unroll
      for (int q = 0; q < 2; q++) {
        const double uw = q == 0 ? wl : uc[0], ue = q == 1 ? er : uc[1];
        const double rr = fma(cz, um[q] + up[q], fma(cy, ysv[q] + ynv[q], fma(cx, uw + ue, fma(-cd, uc[q], fv[q]))));
        const int c = cl + q;
        const bool in = c >= 1 && c <= n - 2;
        rv[q] = in ? oz::d2f_bits(rr) : 0.0f;
        if (ACC64 && in) acc64 = fma(rr, rr, acc64);
        if (!ACC64) {
          const float sr = rv[q] * scale;
          acc = fmaf(sr, sr, acc);
        }
      }
      if (d && cl < a.pitchi) {
        Ti *dp = d + (long long)z * a.planei + (long long)y * a.pitchi + cl;
        if (sizeof(Ti) == 4) *(float2 *)dp = make_float2(rv[0], rv[1]);
        else *(unsigned *)dp = bf16x2_rne_bits(rv[0], rv[1]);
      }
    }
  }
  cp_async_wait<0>();
  double s = oz::warp_sum(ACC64 ? acc64 : (double)acc);
  if (lane == 0) wsum[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kDCWarps; i++) t += wsum[i];
    a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// ------------------------------------------------ exact outer step (c = 2^k)
// k3_dc<Ti, true, ACC64> for cx = cy = cz = 2^k2, with the residual
// evaluated exactly in 64-bit fixed point (fixed.cuh); the update is the one
// FP64 addition per node.
//
// A block of kXW = 8 warps owns rows y0 .. y0+7 of a 128-column x-tile (four
// columns per lane) and a chunk of planes; warp w owns row y0 + w. At plane
// step z every warp takes its row of u and e at plane z+1 (and of f at plane
// z) from registers that were loaded straight from global memory one step
// earlier, forms u + e (FP64), writes it to u_out, converts it once to fixed
// point at the row's warp-wide exponent and publishes the fixed values and
// that exponent in a 3-slot ring in shared memory. The two halo rows y0-1 and
// y0+8 are updated one value per thread (all 256 threads of the block); their
// row-wide exponent is the largest of four warp maxima, read after the
// plane's one barrier, and their fixed values are published then (they are
// read one step later, after the next barrier). The residual of plane z uses
// the warp's own row at planes z-1, z, z+1 (registers), the neighbour rows of
// plane z from the ring and f/2^k2, all on the grid of the largest exponent B
// among them (rows held at a smaller exponent are shifted down to B).
constexpr int kXW = 8;           // warps (own rows) per block
constexpr int kXC = 128;         // columns per x-tile (four per lane)
constexpr int kXRows = kXW + 2;  // published rows: top halo, the own rows, bottom halo

// Four inner-type values of a lane as FP64 (bit conversions, no FP64 instruction).
__device__ __forceinline__ void e4_to_d(const uint4 &b, double (&v)[4]) {  // float
  v[0] = oz::f2d_bits(__uint_as_float(b.x));
  v[1] = oz::f2d_bits(__uint_as_float(b.y));
  v[2] = oz::f2d_bits(__uint_as_float(b.z));
  v[3] = oz::f2d_bits(__uint_as_float(b.w));
}
__device__ __forceinline__ void e4_to_d(const uint2 &b, double (&v)[4]) {  // bf16 pairs
  v[0] = oz::f2d_bits(__uint_as_float(b.x << 16));
  v[1] = oz::f2d_bits(__uint_as_float(b.x & 0xffff0000u));
  v[2] = oz::f2d_bits(__uint_as_float(b.y << 16));
  v[3] = oz::f2d_bits(__uint_as_float(b.y & 0xffff0000u));
}
template <typename Ti> struct E4 { typedef uint4 V; };
template <> struct E4<bf16> { typedef uint2 V; };

// Non-coherent global loads kept where they are written: the plane step's
// loads for the next plane are issued at its start, ahead of the step's
// arithmetic, so that their latency overlaps it.
__device__ __forceinline__ double2 ldv_d2(const double *p) {
  double2 v;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ldv_e4(const float *p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ldv_e4(const bf16 *p) {
  uint2 v;
  asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ double ldv_d(const double *p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double e1_to_d(const float *p) { return oz::f2d_bits(__ldg(p)); }
__device__ __forceinline__ double e1_to_d(const bf16 *p) {
  return oz::f2d_bits(__uint_as_float((unsigned)__ldg((const unsigned short *)p) << 16));
}

// What one plane step reads from global memory: the lane's four columns of u
// and e at plane p, of f at plane p - 1, its halo-row value (u, e) and, for
// lanes 0 and 31, the x-halo column (u, e) of the row.
template <typename Ti> struct XPlane {
  double u[4], f[4];
  typename E4<Ti>::V e;
  double hu, he, xu, xe;
};

template <typename Ti, bool ACC64>
__global__ void __launch_bounds__(32 * kXW, 2) k3_dcx(ArgsDC3 a, const ArgsDC3 *__restrict__ list) {
  if (list) {  // problem blockIdx.z of a list launch
    const ArgsDC3 &p = list[blockIdx.z];
    if (p.live && !*p.live) return;
    a.u = p.u; a.uout = p.uout; a.f = p.f; a.e = p.e; a.d = p.d;
    a.cd = p.cd; a.cx = p.cx; a.cy = p.cy; a.cz = p.cz; a.k2 = p.k2;
    a.partials = p.partials;
  }
  __shared__ __align__(16) long long pub[3][kXRows][kXC];  // published fixed rows
  __shared__ int pexp[3][kXRows];                           // their exponents
  __shared__ unsigned hmax[3][kXW];                         // halo-row pieces' largest biased exponent
  __shared__ double wsum[kXW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tx = blockIdx.x % a.ntx, ty = blockIdx.x / a.ntx;
  const int n = a.n;
  const long long P = a.plane, Pi = a.planei;
  const int y0 = 1 + ty * kXW, y = y0 + w;
  const int x0 = tx * kXC, c0 = x0 + 4 * lane;
  const int z0 = 1 + blockIdx.y * a.zc, z1 = min(z0 + a.zc, n - 1);
  const bool row_live = y <= n - 1;     // the row exists: updated and published
  const bool out_row = y <= n - 2;      // interior row: written and its residual formed
  const bool cols = c0 < a.pitch;       // the lane's four columns lie inside the row's storage
  const bool lv = row_live && cols;
  // halo: thread t updates column x0 + t % 128 of row y0 - 1 (t < 128) or y0 + 8
  const int t = threadIdx.x, hrow = t >> 7, hcol = x0 + (t & 127);
  const int hy = hrow ? y0 + kXW : y0 - 1;
  const bool hok = hy <= n - 1 && hcol <= n - 1;
  // x-halo columns of the own row: x0 - 1 (lane 0) and x0 + 128 (lane 31)
  const int hx = lane == 0 ? x0 - 1 : x0 + kXC;
  const bool xok = row_live && ((lane == 0 && x0 >= 1) || (lane == 31 && x0 + kXC <= n - 1));
  const int k2 = a.k2;
  const float scale = ACC64 ? 1.0f : *a.scale;
  const Ti *e = (const Ti *)a.e;
  Ti *d = (Ti *)a.d;
  typedef typename E4<Ti>::V EV;

  auto load = [&](int p, XPlane<Ti> &q) {
    if (lv) {
      const double *up = a.u + p * P + (long long)y * a.pitch + c0;
      const double2 u0 = ldv_d2(up), u1 = ldv_d2(up + 2);
      q.u[0] = u0.x; q.u[1] = u0.y; q.u[2] = u1.x; q.u[3] = u1.y;
      q.e = ldv_e4(e + p * Pi + (long long)y * a.pitchi + c0);
    } else {
      q.u[0] = q.u[1] = q.u[2] = q.u[3] = 0.0;
      q.e = EV();
    }
    if (out_row && cols && p - 1 >= z0 && p - 1 < z1) {
      const double *fp = a.f + (p - 1) * P + (long long)y * a.pitch + c0;
      const double2 f0 = ldv_d2(fp), f1 = ldv_d2(fp + 2);
      q.f[0] = f0.x; q.f[1] = f0.y; q.f[2] = f1.x; q.f[3] = f1.y;
    } else {
      q.f[0] = q.f[1] = q.f[2] = q.f[3] = 0.0;
    }
    q.hu = hok ? ldv_d(a.u + p * P + (long long)hy * a.pitch + hcol) : 0.0;
    q.he = hok ? e1_to_d(e + p * Pi + (long long)hy * a.pitchi + hcol) : 0.0;
    q.xu = xok ? ldv_d(a.u + p * P + (long long)y * a.pitch + hx) : 0.0;
    q.xe = xok ? e1_to_d(e + p * Pi + (long long)y * a.pitchi + hx) : 0.0;
  };

  XPlane<Ti> cur, nxt;
  load(z0 - 1, cur);
  long long xm[4] = {0, 0, 0, 0}, xc[4] = {0, 0, 0, 0}, xp[4] = {0, 0, 0, 0};
  long long hxc = 0, hxp = 0;  // x-halo value of the own row (lanes 0 and 31)
  int bm = fx::kHead, bc = fx::kHead, bp = fx::kHead;
  float acc = 0.0f;
  double acc64 = 0.0;
  // step z updates plane z + 1 and, from z0 on, forms the residual of plane z
  for (int z = z0 - 2; z < z1; z++) {
    if (z + 2 <= z1) load(z + 2, nxt);
    const int zp = z + 1, ring = zp % 3;
    // own row at plane z + 1: u + e, written, converted, published
    double ev[4], v[4];
    e4_to_d(cur.e, ev);
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = cur.u[q] + ev[q];
    const double xv = cur.xu + cur.xe;
    if (out_row && cols && zp >= z0 && zp < z1) {
      double *op = a.uout + zp * P + (long long)y * a.pitch + c0;
      *(double2 *)op = make_double2(v[0], v[1]);
      *(double2 *)(op + 2) = make_double2(v[2], v[3]);
    }
    {
      unsigned m = max(max((unsigned)fx::dexp(v[0]), (unsigned)fx::dexp(v[1])),
                       max((unsigned)fx::dexp(v[2]), (unsigned)fx::dexp(v[3])));
      m = max(m, xok ? (unsigned)fx::dexp(xv) : 0u);
      m = __reduce_max_sync(0xffffffffu, m);
      const int bn = (m == 0x7ffu ? fx::kNonFinite : (int)m) + fx::kHead;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        xm[q] = xc[q];
        xc[q] = xp[q];
        xp[q] = fx::to_fixed(v[q], bn);
      }
      hxc = hxp;
      hxp = fx::to_fixed(xv, bn);
      bm = bc;
      bc = bp;
      bp = bn;
      if (row_live) {
        *(longlong2 *)&pub[ring][w + 1][4 * lane] = make_longlong2(xp[0], xp[1]);
        *(longlong2 *)&pub[ring][w + 1][4 * lane + 2] = make_longlong2(xp[2], xp[3]);
        if (lane == 0) pexp[ring][w + 1] = bn;
      }
    }
    // halo rows at plane z + 1, first half: u + e and the pieces' exponents
    const double hv = cur.hu + cur.he;
    {
      unsigned hm = hok ? (unsigned)fx::dexp(hv) : 0u;
      hm = __reduce_max_sync(0xffffffffu, hm);
      if (lane == 0) hmax[ring][w] = hm;
    }
    __syncthreads();  // the only barrier of the step
    // halo rows, second half: the row's exponent and its fixed values
    {
      const unsigned *hp = &hmax[ring][hrow * (kXW / 2)];
      const unsigned mm = max(max(hp[0], hp[1]), max(hp[2], hp[3]));
      const int bh = (mm == 0x7ffu ? fx::kNonFinite : (int)mm) + fx::kHead;
      const int hr = hrow ? kXRows - 1 : 0;
      pub[ring][hr][t & 127] = fx::to_fixed(hv, bh);
      if ((t & 127) == 0) pexp[ring][hr] = bh;
    }
    // residual of plane z
    if (z >= z0 && out_row) {
      const int rc = z % 3;
      const longlong2 s01 = *(const longlong2 *)&pub[rc][w][4 * lane];
      const longlong2 s23 = *(const longlong2 *)&pub[rc][w][4 * lane + 2];
      const longlong2 n01 = *(const longlong2 *)&pub[rc][w + 2][4 * lane];
      const longlong2 n23 = *(const longlong2 *)&pub[rc][w + 2][4 * lane + 2];
      const int bs = pexp[rc][w], bnn = pexp[rc][w + 2];
      unsigned mf = max(max((unsigned)fx::dexp(cur.f[0]), (unsigned)fx::dexp(cur.f[1])),
                        max((unsigned)fx::dexp(cur.f[2]), (unsigned)fx::dexp(cur.f[3])));
      mf = __reduce_max_sync(0xffffffffu, mf);
      int B = max(max(max(bm, bc), max(bp, bs)), max(bnn, max((int)mf - k2, 0) + fx::kHead));
      B = mf == 0x7ffu ? fx::kNonFinite + fx::kHead : B;
      long long um_[4], uc_[4], up_[4], ys[4] = {s01.x, s01.y, s23.x, s23.y}, yn[4] = {n01.x, n01.y, n23.x, n23.y};
      long long h = hxc;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        um_[q] = xm[q];
        uc_[q] = xc[q];
        up_[q] = xp[q];
      }
      if (B != bm) {
#pragma unroll
        for (int q = 0; q < 4; q++) um_[q] = fx::align_down(um_[q], B - bm);
      }
      if (B != bc) {
#pragma unroll
        for (int q = 0; q < 4; q++) uc_[q] = fx::align_down(uc_[q], B - bc);
        h = fx::align_down(h, B - bc);
      }
      if (B != bp) {
#pragma unroll
        for (int q = 0; q < 4; q++) up_[q] = fx::align_down(up_[q], B - bp);
      }
      if (B != bs) {
#pragma unroll
        for (int q = 0; q < 4; q++) ys[q] = fx::align_down(ys[q], B - bs);
      }
      if (B != bnn) {
#pragma unroll
        for (int q = 0; q < 4; q++) yn[q] = fx::align_down(yn[q], B - bnn);
      }
      long long west = fx::shfl_up64(uc_[3]), east = fx::shfl_dn64(uc_[0]);
      if (lane == 0) west = h;
      if (lane == 31) east = h;
      const bool finite = B < fx::kNonFinite;
      const int E0 = B - 1085 + k2;
      const fx::Pow2f p2 = fx::pow2f(E0);
      const double s64 = ACC64 ? __hiloint2double((min(max(E0, -1022), 1023) + 1023) << 20, 0) : 0.0;
      float rv[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const long long xw = q == 0 ? west : uc_[q - 1], xe = q == 3 ? east : uc_[q + 1];
        const long long S = 6 * uc_[q] - (xw + xe) - (ys[q] + yn[q]) - (um_[q] + up_[q]);
        const long long R = fx::to_fixed(cur.f[q], B + k2) - S;
        const int c = c0 + q;
        const bool in = c >= 1 && c <= n - 2;
        const float rf = finite ? fx::fixed_to_float(R, p2) : __int_as_float(0x7fc00000);
        rv[q] = in ? rf : 0.0f;
        if (ACC64 && in) {
          const double rr = finite ? fx::fixed_to_double(R, s64) : __longlong_as_double(0x7ff8000000000000ll);
          acc64 = fma(rr, rr, acc64);
        }
        if (!ACC64) {
          const float sr = rv[q] * scale;
          acc = fmaf(sr, sr, acc);
        }
      }
      if (d && cols) {
        Ti *dp = d + z * Pi + (long long)y * a.pitchi + c0;
        if (sizeof(Ti) == 4) *(float4 *)dp = make_float4(rv[0], rv[1], rv[2], rv[3]);
        else *(uint2 *)dp = make_uint2(bf16x2_rne_bits(rv[0], rv[1]), bf16x2_rne_bits(rv[2], rv[3]));
      }
    }
    cur = nxt;
  }
  double s = oz::warp_sum(ACC64 ? acc64 : (double)acc);
  if (lane == 0) wsum[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int i = 0; i < kXW; i++) tsum += wsum[i];
    a.partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = tsum;
  }
}

}  // namespace z3

// List launches of the 3D kernels over many problems of one level size (the
// batch engine); records in device memory, the grid's z index is the problem.
namespace d3 {
z3::Args3 stencil_record(const Level &L, double omega, const void *u, void *out, const void *f);
cudaError_t z_sweep_list(const Level &L, const z3::Args3 *list, int count, int color, cudaStream_t s);
// kJZ over `count` problems (records as for z_sweep_list, u = f): two Jacobi sweeps from zero.
cudaError_t z_jacobi_zero2_list(const Level &L, const z3::Args3 *list, int count, cudaStream_t s);
cudaError_t z_residual_list(const Level &L, const z3::Args3 *list, int count, cudaStream_t s);
cudaError_t z_transfer_list(bool restrict_, const Level &F, const Level &C, const z3::ArgsT3 *list, int count,
                            cudaStream_t s);
z3::ArgsDC3 outer_record(const Level &O, const double *uin, double *uout, const Level &I, const void *e, void *d);
cudaError_t dc_step_list(const Level &O, const Level &I, const z3::ArgsDC3 *list, int count, double *partials,
                         int pstride, int *nparts, bool update, bool exact, cudaStream_t s);
}  // namespace d3
}  // namespace mg

