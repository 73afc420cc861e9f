// Fused, temporally blocked 2D kernels for the fine levels of the V-cycle
// (Algorithm 1), constant stencil, red-black Gauss-Seidel. These scalar
// instances run the FP64 levels; FP32 levels run the packed FP32x2 instances
// of the same design (fused2d_x2.cuh, and fused2d_x2v.cuh for the variable
// stencil).
//
//   k_pre2d : nu1 RBGS sweeps + residual + full-weighting restriction in one
//             pass: reads f (and u unless the level starts from zero), writes
//             the smoothed u and the coarse right-hand side.
//   k_post2d: bilinear interpolation and correction + nu2 RBGS sweeps in one
//             pass: reads u, the coarse solution and f, writes u.
//
// Work decomposition: one warp owns a strip of 128 columns (lane l holds the
// 4 consecutive columns x0 + 4l .. x0 + 4l + 3) and a chunk of R rows. The
// outer 8 columns on each side are a halo recomputed redundantly, so each
// warp writes 112 columns and needs no barrier. Rows stream in groups of 4
// through an 8-row ring in shared memory filled by cp.async, one commit
// group per 4 rows, issued one group ahead (each lane copies, and later reads
// back, only its own pieces, so a lane's own wait_group is the only
// synchronisation); the small ring keeps 5 blocks of 4 warps resident per
// SM. Rows are processed 8 at a time by straight-line code (the register
// window), which lets the compiler overlap consecutive rows. Warps whose
// rows and columns are all interior run a copy of that code without the
// boundary predicates. Half-sweep h of the stack runs
// on row t - h when row t arrives (red = i+j even first, as in the paper's
// "order rb"), so every update sees exactly the neighbour values a
// sequential red-then-black sweep would; the x-neighbours of a lane's edge
// columns come from warp shuffles. The chunk starts 8 rows early so that
// the rows it writes are exact despite the missing rows above it.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace mg {
namespace fz {

// Calls f(integral_constant<int, I>) for I = B .. E-1 (compile-time phases).
template <int B, int E, typename Fn> __device__ __forceinline__ void static_for(Fn &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

constexpr int kVec = 4;                  // columns per lane
constexpr int kCols = 32 * kVec;         // columns per warp strip (loaded)
constexpr int kHalo = 8;                 // halo columns on each side
constexpr int kOut = kCols - 2 * kHalo;  // columns written per strip
constexpr int kSlots = 8;                // row window in registers
constexpr int kGroup = 4;                // rows per cp.async commit group
constexpr int kRing = 2 * kGroup;        // row ring in shared memory: two groups in flight
// Warps per block: the shared-memory ring of FP64 rows is twice as large.
template <typename T> struct Warps { static constexpr int value = sizeof(T) == 8 ? 2 : 4; };
// Resident blocks asked of the register allocator: 5 blocks of 4 FP32 warps
// (at most 96 registers per thread); FP64 kernels are bound by the FP64 pipe
// and keep their natural register count.
template <typename T> struct MinBlocks { static constexpr int value = sizeof(T) == 8 ? 1 : 5; };

struct Args2D {
  const void *uin;  // level solution (ignored when starting from zero)
  const void *f;    // level right-hand side
  void *uout;       // output solution (the other ping-pong buffer)
  const void *ec;   // post: coarse solution
  void *fc;         // pre: coarse right-hand side
  int n, pitch;     // fine grid
  int nc, pitchc;   // coarse grid
  int R;            // rows per chunk (multiple of 8)
  int nstrips, nchunks;
  double alpha, betax, betay, gamma;  // u_new = gamma u + alpha f + betax (uw+ue) + betay (us+un)
  double cx, cy, cd;                  // residual: f - [cx((u-uw)+(u-ue)) + cy((u-us)+(u-un))], cd = 2 (cx + cy)
  // The same coefficients rounded to FP32 on the host: FP32 kernels read
  // these, so that no FP64 -> FP32 conversion (a slow-pipe instruction the
  // compiler may repeat inside loops) runs on the device.
  float alphaf, betaxf, betayf, gammaf, cxf, cyf, cdf;
  int has_gamma;  // gamma != 0 (omega != 1), decided on the host
  // Variable stencil: faces in the level's type (kx[p]: between p and p + 1,
  // ky[p]: between p and the node one row below), omega, h^2 and 1/h^2.
  const void *kx, *ky;
  double omega, h2, ih2;
  float omegaf, h2f, ih2f;
  // List launches of a captured batch step: the problem's live flag in
  // device memory; a block whose problem is no longer live returns at once
  // (NULL: always live).
  const int *live;
};

// True when a list launch's problem has converged (its blocks do nothing).
template <typename R> __device__ __forceinline__ bool retired(const R &p) { return p.live && !*p.live; }

// Launches over many problems of one level size (the batch engine) pass a
// device list with one record per problem and blockIdx.y as the problem
// index: a block takes the record's fields and coefficients, while the grid
// geometry (sizes, pitches, row chunks) stays that of the launch argument.
__device__ __forceinline__ void take_problem(Args2D &a, const Args2D &p) {
  a.uin = p.uin; a.f = p.f; a.uout = p.uout; a.ec = p.ec; a.fc = p.fc;
  a.alpha = p.alpha; a.betax = p.betax; a.betay = p.betay; a.gamma = p.gamma;
  a.cx = p.cx; a.cy = p.cy; a.cd = p.cd;
  a.alphaf = p.alphaf; a.betaxf = p.betaxf; a.betayf = p.betayf; a.gammaf = p.gammaf;
  a.cxf = p.cxf; a.cyf = p.cyf; a.cdf = p.cdf; a.has_gamma = p.has_gamma;
  a.kx = p.kx; a.ky = p.ky;
  a.omega = p.omega; a.h2 = p.h2; a.ih2 = p.ih2; a.omegaf = p.omegaf; a.h2f = p.h2f; a.ih2f = p.ih2f;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid) {
  unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  int sz = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename C> __device__ __forceinline__ C shup(C v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename C> __device__ __forceinline__ C shdn(C v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Bytes a lane stages per row and array: 4 elements.
template <typename T> struct Lane { static constexpr int bytes = kVec * (int)sizeof(T); };

// Copies this lane's 4 elements of row `row` of `base` into `dst` (zero fill if invalid).
template <typename T>
__device__ __forceinline__ void stage_row(unsigned char *dst, const T *base, long long off, bool valid) {
  const T *src = valid ? base + off : base;
#pragma unroll
  for (int b = 0; b < Lane<T>::bytes; b += 16) cp_async16(dst + b, (const unsigned char *)src + b, valid);
}

template <typename T, typename C>
__device__ __forceinline__ void load_lane(const unsigned char *src, C (&v)[kVec]) {
  if (sizeof(T) == 4) {
    float4 x = *(const float4 *)src;
    v[0] = (C)x.x; v[1] = (C)x.y; v[2] = (C)x.z; v[3] = (C)x.w;
  } else {
    double2 a = *(const double2 *)src, b = *(const double2 *)(src + 16);
    v[0] = (C)a.x; v[1] = (C)a.y; v[2] = (C)b.x; v[3] = (C)b.y;
  }
}

template <typename T, typename C>
__device__ __forceinline__ void store_lane(T *dst, const C (&v)[kVec]) {
  if (sizeof(T) == 4) {
    *(float4 *)dst = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  } else {
    *(double2 *)dst = make_double2((double)v[0], (double)v[1]);
    *(double2 *)(dst + 2) = make_double2((double)v[2], (double)v[3]);
  }
}

template <typename C> struct Coef {
  C alpha, bx, by, gamma, cx, cy, cd;
  bool has_gamma;
};


template <typename C> __device__ __forceinline__ Coef<C> coef_of(const Args2D &a) {
  Coef<C> k;
  k.alpha = pick<C>(a.alpha, a.alphaf);
  k.bx = pick<C>(a.betax, a.betaxf);
  k.by = pick<C>(a.betay, a.betayf);
  k.gamma = pick<C>(a.gamma, a.gammaf);
  k.cx = pick<C>(a.cx, a.cxf);
  k.cy = pick<C>(a.cy, a.cyf);
  k.cd = pick<C>(a.cd, a.cdf);
  k.has_gamma = a.has_gamma != 0;
  return k;
}

// Red-black half-sweep of colour `color` on row r held in uc, with rows r-1
// (ua) and r+1 (ub). Columns c0 + q with (c0 + q + r) % 2 == color update.
// CHECK = false is for warps whose rows and columns are all interior: no
// boundary node can be touched, so the predicates are dropped.
template <bool CHECK, typename C>
__device__ __forceinline__ void half_sweep(C (&uc)[kVec], const C (&ua)[kVec], const C (&ub)[kVec],
                                           const C (&fr)[kVec], int r, int color, int c0, int n,
                                           const Coef<C> &k) {
  bool rowok = !CHECK || (r >= 1 && r <= n - 2);
  int par = (color ^ r) & 1;  // c0 is even, so column parity is q's parity
  if (par == 0) {
    C left = shup(uc[3]);
    C n0 = k.alpha * fr[0] + k.bx * (left + uc[1]) + k.by * (ua[0] + ub[0]);
    C n2 = k.alpha * fr[2] + k.bx * (uc[1] + uc[3]) + k.by * (ua[2] + ub[2]);
    if (k.has_gamma) { n0 += k.gamma * uc[0]; n2 += k.gamma * uc[2]; }
    if (!CHECK) {
      uc[0] = n0;
      uc[2] = n2;
    } else {
      if (rowok && c0 >= 1 && c0 <= n - 2) uc[0] = n0;
      if (rowok && c0 + 2 >= 1 && c0 + 2 <= n - 2) uc[2] = n2;
    }
  } else {
    C right = shdn(uc[0]);
    C n1 = k.alpha * fr[1] + k.bx * (uc[0] + uc[2]) + k.by * (ua[1] + ub[1]);
    C n3 = k.alpha * fr[3] + k.bx * (uc[2] + right) + k.by * (ua[3] + ub[3]);
    if (k.has_gamma) { n1 += k.gamma * uc[1]; n3 += k.gamma * uc[3]; }
    if (!CHECK) {
      uc[1] = n1;
      uc[3] = n3;
    } else {
      if (rowok && c0 + 1 >= 1 && c0 + 1 <= n - 2) uc[1] = n1;
      if (rowok && c0 + 3 >= 1 && c0 + 3 <= n - 2) uc[3] = n3;
    }
  }
}

// Residual of row r. FP64 uses the difference form (u - u_nbr first), which
// keeps the rounding error at the size of A u itself; FP32 inner cycles use
// f - cd u + cx (uw + ue) + cy (us + un) (five operations), whose larger
// rounding error the defect-correction outer loop absorbs.
template <bool CHECK, typename C>
__device__ __forceinline__ void residual_row(C (&rr)[kVec], const C (&uc)[kVec], const C (&ua)[kVec],
                                             const C (&ub)[kVec], const C (&fr)[kVec], int r, int c0, int n,
                                             const Coef<C> &k) {
  C left = shup(uc[3]), right = shdn(uc[0]);
  bool rowok = !CHECK || (r >= 1 && r <= n - 2);
#pragma unroll
  for (int q = 0; q < kVec; q++) {
    C u = uc[q];
    C uw = q == 0 ? left : uc[q - 1];
    C ue = q == kVec - 1 ? right : uc[q + 1];
    C res;
    if (sizeof(C) == 8) {
      C t = k.cx * ((u - uw) + (u - ue)) + k.cy * ((u - ua[q]) + (u - ub[q]));
      res = fr[q] - t;
    } else {
      res = k.cy * (ua[q] + ub[q]) + (k.cx * (uw + ue) + (fr[q] - k.cd * u));
    }
    int c = c0 + q;
    rr[q] = (!CHECK || (rowok && c >= 1 && c <= n - 2)) ? res : (C)0;
  }
}

// Face rows of the variable-stencil kernels (fused2d_x2v.cuh) stay staged
// until the residual 2 NU + 2 rows behind has used them.
constexpr int kFaceRing = 16;

// ------------------------------------------------------------------------
// Pre-smoothing + residual + restriction.
template <typename T, int NU, bool ZERO>
__global__ void __launch_bounds__(32 * Warps<T>::value, MinBlocks<T>::value)
    k_pre2d(Args2D a, const Args2D *__restrict__ list) {
  typedef typename CT<T>::type C;
  extern __shared__ __align__(16) unsigned char smem[];
  if (list) {
    if (retired(list[blockIdx.y])) return;
    take_problem(a, list[blockIdx.y]);
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * Warps<T>::value + wib;
  if (gw >= (long long)a.nstrips * a.nchunks) return;
  const int s = (int)(gw % a.nstrips), ch = (int)(gw / a.nstrips);
  const int n = a.n;
  const int x0 = s * kOut - kHalo;
  const int c0 = x0 + kVec * lane;
  const bool col_ok = c0 >= 0 && c0 < a.pitch;
  const bool out_lane = lane >= kHalo / kVec && lane < 32 - kHalo / kVec && col_ok;
  const int r0 = ch * a.R, r1 = min(r0 + a.R, n);
  const int tstart = max(r0 - 8, 0);
  const int tend = r1 + 2 * NU;  // inclusive: residual of row r1 - 1 needs u up to r1 + 2 NU
  const T *uin = (const T *)a.uin;
  const T *f = (const T *)a.f;
  T *uout = (T *)a.uout;
  T *fc = (T *)a.fc;
  constexpr int LB = Lane<T>::bytes;
  // per-warp rings: u (absent when starting from zero), f
  constexpr size_t UB = ZERO ? 0 : (size_t)kRing * 32 * LB;
  constexpr size_t WB = UB + (size_t)kRing * 32 * LB;
  unsigned char *su = smem + (size_t)wib * WB;
  unsigned char *sf = su + UB;
  const Coef<C> k = coef_of<C>(a);

  C U[kSlots][kVec], F[kSlots][kVec], Rr[kSlots][kVec];
#pragma unroll
  for (int i = 0; i < kSlots; i++)
#pragma unroll
    for (int q = 0; q < kVec; q++) { U[i][q] = 0; F[i][q] = 0; Rr[i][q] = 0; }

  // Stages the kGroup rows starting at tg (one commit group).
  auto issue_group = [&](int tg) {
#pragma unroll
    for (int K = 0; K < kGroup; K++) {
      int row = tg + K;
      int slot = row & (kRing - 1);
      bool ok = col_ok && row >= 0 && row < n && row <= tend;
      long long off = (long long)row * a.pitch + c0;
      if (!ZERO) stage_row<T>(su + (slot * 32 + lane) * LB, uin, off, ok);
      stage_row<T>(sf + (slot * 32 + lane) * LB, f, off, ok);
    }
    cp_async_commit();
  };

  // Rows t of the loop run up to the end of the last block of 8; interior
  // warps (every touched row and column inside the domain) skip predicates.
  const int tlast = tstart + ((tend - tstart) / kSlots + 1) * kSlots - 1;
  const bool interior_warp = x0 >= 1 && x0 + kCols - 1 <= n - 2 && tstart - 2 * NU - 2 >= 1 && tlast <= n - 2;

  // Row t lives in ring slot t % kRing. Group t + kGroup is issued when row
  // t is about to be read: its slots held rows t - kGroup .. t - 1, which are
  // already in registers.
  auto body = [&](auto chk) {
  constexpr bool CHECK = decltype(chk)::value;
  issue_group(tstart);
  for (int tb = tstart; tb <= tend; tb += kSlots) {
    static_for<0, kSlots>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr (K % kGroup == 0) {
        issue_group(t + kGroup);
        cp_async_wait<1>();  // group t has landed; group t + kGroup may be in flight
      }
      {
        constexpr int slot = K % kRing;  // tb is a multiple of kRing
        if (!ZERO) {
          load_lane<T, C>(su + (slot * 32 + lane) * LB, U[K]);
        } else {
#pragma unroll
          for (int q = 0; q < kVec; q++) U[K][q] = (C)0;
        }
        load_lane<T, C>(sf + (slot * 32 + lane) * LB, F[K]);
        // half-sweeps h = 1 .. 2 NU on rows t - h (odd h red, even h black)
#pragma unroll
        for (int h = 1; h <= 2 * NU; h++) {
          const int sc = (K - h) & (kSlots - 1), sa = (K - h - 1) & (kSlots - 1), sb = (K - h + 1) & (kSlots - 1);
          half_sweep<CHECK, C>(U[sc], U[sa], U[sb], F[sc], t - h, (h - 1) & 1, c0, n, k);
        }
        // final u of row t - 2 NU
        {
          const int r = t - 2 * NU;
          const int sc = (K - 2 * NU) & (kSlots - 1);
          if (r >= r0 && r < r1 && out_lane) store_lane<T, C>(uout + (long long)r * a.pitch + c0, U[sc]);
        }
        // residual of row t - 2 NU - 1
        {
          const int r = t - 2 * NU - 1;
          const int sc = (K - 2 * NU - 1) & (kSlots - 1), sa = (K - 2 * NU - 2) & (kSlots - 1),
                    sb = (K - 2 * NU) & (kSlots - 1);
          residual_row<CHECK, C>(Rr[sc], U[sc], U[sa], U[sb], F[sc], r, c0, n, k);
          // restriction once the row below the coarse row is ready (r = 2I + 1);
          // tb is a multiple of 8, so r's parity is known at compile time
          if constexpr (((K - 2 * NU - 1) & 1) != 0) {
            const int I = (r - 1) >> 1;
            const int sA = (K - 2 * NU - 3) & (kSlots - 1), sB = (K - 2 * NU - 2) & (kSlots - 1);
            C lA = shup(Rr[sA][3]), lB = shup(Rr[sB][3]), lC = shup(Rr[sc][3]);
            C h0A = lA + (C)2 * Rr[sA][0] + Rr[sA][1], h1A = Rr[sA][1] + (C)2 * Rr[sA][2] + Rr[sA][3];
            C h0B = lB + (C)2 * Rr[sB][0] + Rr[sB][1], h1B = Rr[sB][1] + (C)2 * Rr[sB][2] + Rr[sB][3];
            C h0C = lC + (C)2 * Rr[sc][0] + Rr[sc][1], h1C = Rr[sc][1] + (C)2 * Rr[sc][2] + Rr[sc][3];
            C v0 = (h0A + (C)2 * h0B + h0C) * (C)0.0625;
            C v1 = (h1A + (C)2 * h1B + h1C) * (C)0.0625;
            const int J0 = c0 >> 1;
            if (out_lane && I >= 1 && I <= a.nc - 2 && 2 * I >= r0 && 2 * I < r1) {
              T *row = fc + (long long)I * a.pitchc;
              if (J0 >= 1 && J0 <= a.nc - 2) st(row + J0, v0);
              if (J0 + 1 >= 1 && J0 + 1 <= a.nc - 2) st(row + J0 + 1, v1);
            }
          }
        }
      }
    });
  }
  };
  if (interior_warp) body(std::false_type{});
  else body(std::true_type{});
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------
// Interpolation + correction + post-smoothing.
template <typename T, int NU>
__global__ void __launch_bounds__(32 * Warps<T>::value, MinBlocks<T>::value)
    k_post2d(Args2D a, const Args2D *__restrict__ list) {
  typedef typename CT<T>::type C;
  extern __shared__ __align__(16) unsigned char smem[];
  if (list) {
    if (retired(list[blockIdx.y])) return;
    take_problem(a, list[blockIdx.y]);
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * Warps<T>::value + wib;
  if (gw >= (long long)a.nstrips * a.nchunks) return;
  const int s = (int)(gw % a.nstrips), ch = (int)(gw / a.nstrips);
  const int n = a.n;
  const int x0 = s * kOut - kHalo;
  const int c0 = x0 + kVec * lane;
  const bool col_ok = c0 >= 0 && c0 < a.pitch;
  const int J0 = c0 >> 1;
  const bool ccol_ok = c0 >= 0 && J0 + 1 < a.pitchc;
  const bool out_lane = lane >= kHalo / kVec && lane < 32 - kHalo / kVec && col_ok;
  const int r0 = ch * a.R, r1 = min(r0 + a.R, n);
  const int tstart = max(r0 - 8, 0);
  const int tend = r1 - 1 + 2 * NU;  // inclusive: final u of row r1 - 1 is ready at t = r1 - 1 + 2 NU
  const T *uin = (const T *)a.uin;
  const T *f = (const T *)a.f;
  const T *ec = (const T *)a.ec;
  T *uout = (T *)a.uout;
  constexpr int LB = Lane<T>::bytes;
  constexpr int CB = 2 * (int)sizeof(T);  // two coarse values per lane
  constexpr size_t WB = (size_t)kRing * 32 * (2 * LB + CB);
  unsigned char *su = smem + (size_t)wib * WB;
  unsigned char *sf = su + kRing * 32 * LB;
  unsigned char *se = sf + kRing * 32 * LB;  // CB bytes per lane and slot
  const Coef<C> k = coef_of<C>(a);

  C U[kSlots][kVec], F[kSlots][kVec];
  // Coarse rows by parity of the coarse row index (values at J0, J0+1). Chunks
  // start at multiples of 8, so every parity below is a compile-time constant.
  C E[2][2];
#pragma unroll
  for (int i = 0; i < kSlots; i++)
#pragma unroll
    for (int q = 0; q < kVec; q++) { U[i][q] = 0; F[i][q] = 0; }
  E[0][0] = E[0][1] = E[1][0] = E[1][1] = 0;

  // With fine row `row` also stage coarse row I = (row + 1) / 2 when row is
  // odd, and coarse row 0 with fine row 0.
  auto issue_group = [&](int tg) {
#pragma unroll
    for (int K = 0; K < kGroup; K++) {
      int row = tg + K;
      int slot = row & (kRing - 1);
      bool ok = col_ok && row >= 0 && row < n && row <= tend;
      long long off = (long long)row * a.pitch + c0;
      stage_row<T>(su + (slot * 32 + lane) * LB, uin, off, ok);
      stage_row<T>(sf + (slot * 32 + lane) * LB, f, off, ok);
      int I = (row & 1) ? (row + 1) >> 1 : (row == 0 ? 0 : -1);
      bool cok = ccol_ok && row >= 0 && row <= tend && I >= 0 && I < a.nc;
      const T *csrc = cok ? ec + (long long)I * a.pitchc + J0 : ec;
      unsigned char *cdst = se + (slot * 32 + lane) * CB;
      if (CB == 16) cp_async16(cdst, csrc, cok);
      else cp_async8(cdst, csrc, cok);
    }
    cp_async_commit();
  };

  const int tlast = tstart + ((tend - tstart) / kSlots + 1) * kSlots - 1;
  const bool interior_warp = x0 >= 1 && x0 + kCols - 1 <= n - 2 && tstart - 2 * NU >= 1 && tlast <= n - 2;

  // Coarse row tstart/2 (even index) precedes the window when the chunk starts inside the grid.
  if (tstart > 0) {
    int I = tstart >> 1;
    if (ccol_ok && I < a.nc) {
      E[0][0] = (C)ld(ec + (long long)I * a.pitchc + J0);
      E[0][1] = (C)ld(ec + (long long)I * a.pitchc + J0 + 1);
    }
  }

  auto body = [&](auto chk) {
  constexpr bool CHECK = decltype(chk)::value;
  issue_group(tstart);
  for (int tb = tstart; tb <= tend; tb += kSlots) {
    static_for<0, kSlots>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr (K % kGroup == 0) {
        issue_group(t + kGroup);
        cp_async_wait<1>();
      }
      {
        constexpr int slot = K % kRing;
        load_lane<T, C>(su + (slot * 32 + lane) * LB, U[K]);
        load_lane<T, C>(sf + (slot * 32 + lane) * LB, F[K]);
        if ((K & 1) || (CHECK && t == 0)) {
          constexpr int PI = ((K + 1) >> 1) & 1;  // parity of I = (t + 1) / 2
          const unsigned char *cs = se + (slot * 32 + lane) * CB;
          if (sizeof(T) == 4) {
            float2 v = *(const float2 *)cs;
            E[PI][0] = (C)v.x; E[PI][1] = (C)v.y;
          } else {
            double2 v = *(const double2 *)cs;
            E[PI][0] = (C)v.x; E[PI][1] = (C)v.y;
          }
        }
        // interpolation and correction of row t
        {
          C e0, e1;
          constexpr int PA = (K >> 1) & 1, PB = PA ^ 1;  // parities of t/2 and t/2 + 1
          if (K & 1) {
            e0 = (C)0.5 * (E[PA][0] + E[PB][0]);
            e1 = (C)0.5 * (E[PA][1] + E[PB][1]);
          } else {
            e0 = E[PA][0];
            e1 = E[PA][1];
          }
          C e2 = shdn(e0);
          C v[kVec] = {e0, (C)0.5 * (e0 + e1), e1, (C)0.5 * (e1 + e2)};
          bool rowok = !CHECK || (t >= 1 && t <= n - 2);
#pragma unroll
          for (int q = 0; q < kVec; q++) {
            int c = c0 + q;
            if (!CHECK || (rowok && c >= 1 && c <= n - 2)) U[K][q] += v[q];
          }
        }
#pragma unroll
        for (int h = 1; h <= 2 * NU; h++) {
          const int sc = (K - h) & (kSlots - 1), sa = (K - h - 1) & (kSlots - 1), sb = (K - h + 1) & (kSlots - 1);
          half_sweep<CHECK, C>(U[sc], U[sa], U[sb], F[sc], t - h, (h - 1) & 1, c0, n, k);
        }
        {
          const int r = t - 2 * NU;
          const int sc = (K - 2 * NU) & (kSlots - 1);
          if (r >= r0 && r < r1 && out_lane) store_lane<T, C>(uout + (long long)r * a.pitch + c0, U[sc]);
        }
      }
    });
  }
  };
  if (interior_warp) body(std::false_type{});
  else body(std::true_type{});
  cp_async_wait<0>();
}

}  // namespace fz

namespace d2 {
// One problem's record for the list launches (pointers and coefficients).
fz::Args2D fused_record(const Level &L, const Level &Cl, double omega, const void *uin, void *uout, const void *ec,
                        void *fc);
// The fused passes over `count` problems of level size L.n (coarse Cl.n),
// records in device memory; the grid's y index is the problem. rows: rows per
// warp chunk (0 = 256), the same for every problem of the size whatever else
// is in the batch.
cudaError_t pre_fused_list(const Level &L, const Level &Cl, const fz::Args2D *list, int count, bool zero, int nu,
                           int rows, cudaStream_t s);
cudaError_t post_fused_list(const Level &L, const Level &Cl, const fz::Args2D *list, int count, int nu, int rows,
                            cudaStream_t s);
}  // namespace d2
}  // namespace mg
