// FP32 variable-stencil instance of k_pre2d (fused2d.cuh) in the packed pair
// layout of fused2d_x2.cuh: nu RBGS sweeps + residual + full weighting in
// one pass, warp strips, row chunks, the cp.async rings of u, f and the two
// face arrays, and the register window, with a lane's four columns held as
// the pairs E = (c0, c0+2) and O = (c0+1, c0+3), so that each red-black
// update of a row is one pair:
//
//   S = kx_c u_{c+1} + kx_{c-1} u_{c-1} + ky_r u_{r+1} + ky_{r-1} u_{r-1},
//   u' = W (F + S) (+ (1 - omega) u),   W = omega / (sum of the four faces),
//   F = h^2 f,
//
// four pair fused multiply-adds and two pair multiplies per pair of nodes
// instead of twelve scalar operations; W and F are formed once per row as it
// arrives (W kept in the register window). The residual is the difference
// form of the scalar kernel, (F + sum_faces k (u_nbr - u)) / h^2, in pairs.
// The colour of every half-sweep is a compile-time constant (chunks start
// on multiples of 8 rows). Rounding differs from the scalar instance only in
// the order of FP32 operations, which the FP64 outer loop of defect
// correction absorbs. Every warp runs the code with boundary predicates (one
// copy of the body: a second, predicate-free copy of the scalar variable
// kernel cost more in instruction-fetch stalls than it saved).
#pragma once

#include "fused2d_x2.cuh"

namespace mg {
namespace fz {

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// A lane's four values of a staged row as the pairs (v0, v2) and (v1, v3).
__device__ __forceinline__ void pairs_of(const unsigned char *src, float2 &e, float2 &o) {
  const float4 v = *(const float4 *)src;
  e = make_float2(v.x, v.z);
  o = make_float2(v.y, v.w);
}

// The faces a row's update uses, as pairs: kx at the nodes' own columns
// (KE = kx(c0, c0+2), KO = kx(c0+1, c0+3)) and at the west neighbours
// (KWE = kx(c0-1, c0+1); the odd nodes' west faces are KE), ky of the row
// (YE, YO) and of the row above (SE, SO).
struct FacesX2 {
  float2 KE, KO, KWE, YE, YO, SE, SO;
};
__device__ __forceinline__ FacesX2 faces_x2(const unsigned char *kxr, const unsigned char *kyr,
                                            const unsigned char *kys) {
  FacesX2 q;
  pairs_of(kxr, q.KE, q.KO);
  q.KWE = make_float2(shup(q.KO.y), q.KO.x);
  pairs_of(kyr, q.YE, q.YO);
  pairs_of(kys, q.SE, q.SO);
  return q;
}

// Half-sweep of row r (pairs E, O) with rows r-1 (A) and r+1 (B); PAR = 0
// updates the even columns, PAR = 1 the odd ones.
template <int PAR>
__device__ __forceinline__ void half_x2v(float2 &E, float2 &O, const float2 &AE, const float2 &AO, const float2 &BE,
                                         const float2 &BO, const float2 &FE, const float2 &FO, const float2 &WE,
                                         const float2 &WO, const FacesX2 &q, bool rowok, const bool (&mE)[2],
                                         const bool (&mO)[2], const float2 &gam, bool has_gamma) {
  if constexpr (PAR == 0) {
    const float2 w = make_float2(shup(O.y), O.x);
    const float2 s = fma2(q.SE, AE, fma2(q.YE, BE, fma2(q.KWE, w, mul2(q.KE, O))));
    float2 v = mul2(WE, add2(FE, s));
    if (has_gamma) v = fma2(gam, E, v);
    E.x = rowok && mE[0] ? v.x : E.x;
    E.y = rowok && mE[1] ? v.y : E.y;
  } else {
    const float2 e = make_float2(E.y, shdn(E.x));
    const float2 s = fma2(q.SO, AO, fma2(q.YO, BO, fma2(q.KE, E, mul2(q.KO, e))));
    float2 v = mul2(WO, add2(FO, s));
    if (has_gamma) v = fma2(gam, O, v);
    O.x = rowok && mO[0] ? v.x : O.x;
    O.y = rowok && mO[1] ? v.y : O.y;
  }
}

// Blocks of 2 warps; per warp the rings of u (absent from zero), f and the
// two face arrays (16 rows: a face row stays staged until the residual
// 2 NU + 2 rows behind has used it, NU <= 3). 4 resident blocks per SM
// (8 warps, up to 256 registers): 5 made the zero-start instance spill and
// measured no faster.
template <bool ZERO> struct X2VSmem {
  static constexpr size_t UB = ZERO ? 0 : (size_t)kRing * 32 * 16;
  static constexpr size_t WB = UB + (size_t)kRing * 32 * 16 + (size_t)kFaceRing * 32 * 16 * 2;
};

template <int NU, bool ZERO, bool LIST>
__global__ void __launch_bounds__(64, 4) k_pre2d_x2v(Args2D a, const Args2D *__restrict__ list) {
  static_assert(2 * NU + 2 + 2 * kGroup <= kFaceRing, "face ring too short for NU");
  extern __shared__ __align__(16) unsigned char smem[];
  if (LIST) {
    if (retired(list[blockIdx.y])) return;
    take_problem(a, list[blockIdx.y]);
  }
  constexpr int W = 2;  // warps per block
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * W + wib;
  if (gw >= (long long)a.nstrips * a.nchunks) return;
  const int s = (int)(gw % a.nstrips), ch = (int)(gw / a.nstrips);
  const int n = a.n;
  const int x0 = s * kOut - kHalo;
  const int c0 = x0 + kVec * lane;
  const bool col_ok = c0 >= 0 && c0 < a.pitch;
  const bool out_lane = lane >= kHalo / kVec && lane < 32 - kHalo / kVec && col_ok;
  const int r0 = ch * a.R, r1 = min(r0 + a.R, n);
  const int tstart = max(r0 - 8, 0);  // a multiple of 8
  const int tend = r1 + 2 * NU;       // inclusive: residual of row r1 - 1 needs u up to r1 + 2 NU
  const int rlim = min(n, tend + 1);  // rows staged: .. rlim - 1
  const long long pitch = a.pitch;
  const float *uin = (const float *)a.uin;
  const float *f = (const float *)a.f;
  const float *kxg = (const float *)a.kx;
  const float *kyg = (const float *)a.ky;
  float *uout = (float *)a.uout;
  float *fc = (float *)a.fc;
  unsigned char *su = smem + (size_t)wib * X2VSmem<ZERO>::WB;
  unsigned char *sf = su + X2VSmem<ZERO>::UB;
  unsigned char *skx = sf + kRing * 32 * 16;
  unsigned char *sky = skx + kFaceRing * 32 * 16;
  const float omega = a.omegaf, ih2 = a.ih2f;
  const float2 h2 = splat2(a.h2f), gam = splat2(a.gammaf);
  const bool has_gamma = a.has_gamma != 0;
  bool mE[2], mO[2];
  mE[0] = c0 >= 1 && c0 <= n - 2;
  mO[0] = c0 + 1 >= 1 && c0 + 1 <= n - 2;
  mE[1] = c0 + 2 >= 1 && c0 + 2 <= n - 2;
  mO[1] = c0 + 3 >= 1 && c0 + 3 <= n - 2;
  const int J0 = c0 >> 1;

  float2 UE[kSlots], UO[kSlots], FE[kSlots], FO[kSlots], WE[kSlots], WO[kSlots], HR[kSlots];
#pragma unroll
  for (int i = 0; i < kSlots; i++) {
    UE[i] = UO[i] = FE[i] = FO[i] = WE[i] = WO[i] = HR[i] = make_float2(0.0f, 0.0f);
  }

  const long long lane_off = col_ok ? c0 : 0;
  // this lane's 16 bytes of face row `row` (zero outside the rows needed)
  auto stage_faces = [&](int row) {
    const bool ok = col_ok && row >= 0 && row < rlim;
    const int fs = row & (kFaceRing - 1);
    const long long off = (long long)(ok ? row : 0) * pitch + lane_off;
    cp_async16(skx + (fs * 32 + lane) * 16, ok ? (const void *)(kxg + off) : (const void *)kxg, ok);
    cp_async16(sky + (fs * 32 + lane) * 16, ok ? (const void *)(kyg + off) : (const void *)kyg, ok);
  };
  auto face_row = [&](const unsigned char *ring, int row) {
    return ring + ((row & (kFaceRing - 1)) * 32 + lane) * 16;
  };
  int tnext = tstart;
  auto issue_group = [&](auto sb) {
    constexpr int SB = decltype(sb)::value;  // ring slot of the group's first row
#pragma unroll
    for (int j = 0; j < kGroup; j++) {
      const int row = tnext + j;
      const bool ok = col_ok && row < rlim;
      const long long off = (long long)(ok ? row : 0) * pitch + lane_off;
      unsigned char *du = su + (((SB + j) & (kRing - 1)) * 32 + lane) * 16;
      unsigned char *df = sf + (((SB + j) & (kRing - 1)) * 32 + lane) * 16;
      if (!ZERO) cp_async16(du, ok ? (const void *)(uin + off) : (const void *)uin, ok);
      cp_async16(df, ok ? (const void *)(f + off) : (const void *)f, ok);
      stage_faces(row);
    }
    cp_async_commit();
    tnext += kGroup;
  };

  // the face rows above the first row (their own commit group)
#pragma unroll
  for (int j = kGroup; j >= 1; j--) stage_faces(tstart - j);
  cp_async_commit();
  issue_group(std::integral_constant<int, 0>{});
  for (int tb = tstart; tb <= tend; tb += kSlots) {
    static_for<0, kSlots>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr (K % kGroup == 0) {
        issue_group(std::integral_constant<int, (K + kGroup) & (kRing - 1)>{});
        cp_async_wait<1>();  // rows up to t + 3 have landed; t + 4 .. t + 7 may be in flight
      }
      // row t arrives: u, F = h^2 f and W = omega / (sum of its four faces)
      if (!ZERO) {
        pairs_of(su + (K * 32 + lane) * 16, UE[K], UO[K]);
      } else {
        UE[K] = UO[K] = make_float2(0.0f, 0.0f);
      }
      {
        float2 fe, fo;
        pairs_of(sf + (K * 32 + lane) * 16, fe, fo);
        FE[K] = mul2(h2, fe);
        FO[K] = mul2(h2, fo);
        const FacesX2 q = faces_x2(face_row(skx, t), face_row(sky, t), face_row(sky, t - 1));
        const float2 dE = add2(add2(q.KE, q.KWE), add2(q.YE, q.SE));
        const float2 dO = add2(add2(q.KO, q.KE), add2(q.YO, q.SO));
        WE[K] = make_float2(__fdividef(omega, dE.x), __fdividef(omega, dE.y));
        WO[K] = make_float2(__fdividef(omega, dO.x), __fdividef(omega, dO.y));
      }
      // half-sweeps h = 1 .. 2 NU on rows t - h (odd h red, even h black)
      static_for<1, 2 * NU + 1>([&](auto hc) {
        constexpr int h = decltype(hc)::value;
        constexpr int sc = (K - h) & (kSlots - 1), sa = (K - h - 1) & (kSlots - 1), sb = (K - h + 1) & (kSlots - 1);
        constexpr int PAR = ((h - 1) ^ (K - h)) & 1;  // colour (h - 1) & 1 on row t - h, t = K mod 2
        const int r = t - h;
        const bool rowok = r >= 1 && r <= n - 2;
        const FacesX2 q = faces_x2(face_row(skx, r), face_row(sky, r), face_row(sky, r - 1));
        half_x2v<PAR>(UE[sc], UO[sc], UE[sa], UO[sa], UE[sb], UO[sb], FE[sc], FO[sc], WE[sc], WO[sc], q, rowok, mE,
                      mO, gam, has_gamma);
      });
      // final u of row t - 2 NU
      {
        const int r = t - 2 * NU;
        constexpr int sc = (K - 2 * NU) & (kSlots - 1);
        if (r >= r0 && r < r1 && out_lane)
          *(float4 *)(uout + (long long)r * pitch + c0) = make_float4(UE[sc].x, UO[sc].x, UE[sc].y, UO[sc].y);
      }
      // residual of row t - 2 NU - 1 and its horizontal full-weighting sums
      {
        const int r = t - 2 * NU - 1;
        constexpr int sc = (K - 2 * NU - 1) & (kSlots - 1), sa = (K - 2 * NU - 2) & (kSlots - 1),
                      sb = (K - 2 * NU) & (kSlots - 1);
        const FacesX2 q = faces_x2(face_row(skx, r), face_row(sky, r), face_row(sky, r - 1));
        const float2 E = UE[sc], O = UO[sc];
        const float2 w = make_float2(shup(O.y), O.x), e = make_float2(E.y, shdn(E.x));
        // (F + sum_faces k (u_nbr - u)) / h^2
        const float2 tE = fma2(q.SE, sub2(UE[sa], E), fma2(q.YE, sub2(UE[sb], E), fma2(q.KWE, sub2(w, E), mul2(q.KE, sub2(O, E)))));
        const float2 tO = fma2(q.SO, sub2(UO[sa], O), fma2(q.YO, sub2(UO[sb], O), fma2(q.KE, sub2(E, O), mul2(q.KO, sub2(e, O)))));
        float2 rE = mul2(add2(FE[sc], tE), splat2(ih2));
        float2 rO = mul2(add2(FO[sc], tO), splat2(ih2));
        const bool rowok = r >= 1 && r <= n - 2;
        rE.x = rowok && mE[0] ? rE.x : 0.0f;
        rE.y = rowok && mE[1] ? rE.y : 0.0f;
        rO.x = rowok && mO[0] ? rO.x : 0.0f;
        rO.y = rowok && mO[1] ? rO.y : 0.0f;
        HR[sc] = add2(add2(rE, rE), add2(make_float2(shup(rO.y), rO.x), rO));
        // restriction once the row below the coarse row is ready (r = 2I + 1)
        if constexpr (((K - 2 * NU - 1) & 1) != 0) {
          constexpr int sA = (K - 2 * NU - 3) & (kSlots - 1), sB = (K - 2 * NU - 2) & (kSlots - 1);
          const float2 t2 = add2(add2(HR[sB], HR[sB]), add2(HR[sA], HR[sc]));
          const float2 v = mul2(t2, splat2(0.0625f));
          const int I = (r - 1) >> 1;
          if (out_lane && I >= 1 && I <= a.nc - 2 && 2 * I >= r0 && 2 * I < r1) {
            float *row = fc + (long long)I * a.pitchc + J0;
            if (J0 >= 1 && J0 <= a.nc - 2) row[0] = v.x;
            if (J0 + 1 >= 1 && J0 + 1 <= a.nc - 2) row[1] = v.y;
          }
        }
      }
    });
  }
  cp_async_wait<0>();
}

// Interpolation + correction + NU RBGS sweeps with the variable stencil
// (k_post2d, FP32) in the pair layout: the coarse correction as in
// k_post2d_x2 (a lane's coarse values at J0 = c0 / 2 and J0 + 1 form one
// pair), the sweeps as in k_pre2d_x2v. Per warp: rings of u, f and the
// coarse rows (8 rows) and of the faces (16 rows).
constexpr size_t kX2VPostWB = (size_t)kRing * 32 * (16 + 16 + 8) + (size_t)kFaceRing * 32 * 16 * 2;

template <int NU, bool LIST>
__global__ void __launch_bounds__(64, 4) k_post2d_x2v(Args2D a, const Args2D *__restrict__ list) {
  static_assert(2 * NU + 1 + 2 * kGroup <= kFaceRing, "face ring too short for NU");
  extern __shared__ __align__(16) unsigned char smem[];
  if (LIST) {
    if (retired(list[blockIdx.y])) return;
    take_problem(a, list[blockIdx.y]);
  }
  constexpr int W = 2;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * W + wib;
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
  const int tstart = max(r0 - 8, 0);  // a multiple of 8
  const int tend = r1 - 1 + 2 * NU;   // inclusive: final u of row r1 - 1 is ready at t = r1 - 1 + 2 NU
  const int rlim = min(n, tend + 1);
  const long long pitch = a.pitch, pitchc = a.pitchc;
  const float *uin = (const float *)a.uin;
  const float *f = (const float *)a.f;
  const float *ec = (const float *)a.ec;
  const float *kxg = (const float *)a.kx;
  const float *kyg = (const float *)a.ky;
  float *uout = (float *)a.uout;
  constexpr int CB = 8;  // two coarse values per lane
  unsigned char *su = smem + (size_t)wib * kX2VPostWB;
  unsigned char *sf = su + kRing * 32 * 16;
  unsigned char *se = sf + kRing * 32 * 16;
  unsigned char *skx = se + kRing * 32 * CB;
  unsigned char *sky = skx + kFaceRing * 32 * 16;
  const float omega = a.omegaf;
  const float2 h2 = splat2(a.h2f), gam = splat2(a.gammaf), half2 = splat2(0.5f);
  const bool has_gamma = a.has_gamma != 0;
  bool mE[2], mO[2];
  mE[0] = c0 >= 1 && c0 <= n - 2;
  mO[0] = c0 + 1 >= 1 && c0 + 1 <= n - 2;
  mE[1] = c0 + 2 >= 1 && c0 + 2 <= n - 2;
  mO[1] = c0 + 3 >= 1 && c0 + 3 <= n - 2;

  float2 UE[kSlots], UO[kSlots], FE[kSlots], FO[kSlots], WE[kSlots], WO[kSlots];
#pragma unroll
  for (int i = 0; i < kSlots; i++) UE[i] = UO[i] = FE[i] = FO[i] = WE[i] = WO[i] = make_float2(0.0f, 0.0f);
  // coarse rows by parity of the coarse row index (values at J0, J0 + 1)
  float2 EC[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};

  const long long lane_off = col_ok ? c0 : 0;
  auto stage_faces = [&](int row) {
    const bool ok = col_ok && row >= 0 && row < rlim;
    const int fs = row & (kFaceRing - 1);
    const long long off = (long long)(ok ? row : 0) * pitch + lane_off;
    cp_async16(skx + (fs * 32 + lane) * 16, ok ? (const void *)(kxg + off) : (const void *)kxg, ok);
    cp_async16(sky + (fs * 32 + lane) * 16, ok ? (const void *)(kyg + off) : (const void *)kyg, ok);
  };
  auto face_row = [&](const unsigned char *ring, int row) {
    return ring + ((row & (kFaceRing - 1)) * 32 + lane) * 16;
  };
  int tnext = tstart;
  // With fine row `row` also stage coarse row (row + 1) / 2 when row is odd,
  // and coarse row 0 with fine row 0.
  auto issue_group = [&](auto sb) {
    constexpr int SB = decltype(sb)::value;
#pragma unroll
    for (int j = 0; j < kGroup; j++) {
      const int row = tnext + j;
      const bool ok = col_ok && row < rlim;
      const long long off = (long long)(ok ? row : 0) * pitch + lane_off;
      const int slot = (SB + j) & (kRing - 1);
      cp_async16(su + (slot * 32 + lane) * 16, ok ? (const void *)(uin + off) : (const void *)uin, ok);
      cp_async16(sf + (slot * 32 + lane) * 16, ok ? (const void *)(f + off) : (const void *)f, ok);
      const int I = (j & 1) ? (row + 1) >> 1 : (row == 0 ? 0 : -1);  // row has the parity of j
      const bool cok = ccol_ok && row <= tend && I >= 0 && I < a.nc;
      cp_async8(se + (slot * 32 + lane) * CB, cok ? (const void *)(ec + (long long)I * pitchc + J0) : (const void *)ec, cok);
      stage_faces(row);
    }
    cp_async_commit();
    tnext += kGroup;
  };

  // coarse row tstart / 2 (even index) precedes the window when the chunk starts inside the grid
  if (tstart > 0) {
    const int I = tstart >> 1;
    if (ccol_ok && I < a.nc) EC[0] = *(const float2 *)(ec + (long long)I * pitchc + J0);
  }
#pragma unroll
  for (int j = kGroup; j >= 1; j--) stage_faces(tstart - j);
  cp_async_commit();
  issue_group(std::integral_constant<int, 0>{});
  for (int tb = tstart; tb <= tend; tb += kSlots) {
    static_for<0, kSlots>([&](auto kc) {
      constexpr int K = decltype(kc)::value;
      const int t = tb + K;
      if constexpr (K % kGroup == 0) {
        issue_group(std::integral_constant<int, (K + kGroup) & (kRing - 1)>{});
        cp_async_wait<1>();
      }
      pairs_of(su + (K * 32 + lane) * 16, UE[K], UO[K]);
      {
        float2 fe, fo;
        pairs_of(sf + (K * 32 + lane) * 16, fe, fo);
        FE[K] = mul2(h2, fe);
        FO[K] = mul2(h2, fo);
        const FacesX2 q = faces_x2(face_row(skx, t), face_row(sky, t), face_row(sky, t - 1));
        const float2 dE = add2(add2(q.KE, q.KWE), add2(q.YE, q.SE));
        const float2 dO = add2(add2(q.KO, q.KE), add2(q.YO, q.SO));
        WE[K] = make_float2(__fdividef(omega, dE.x), __fdividef(omega, dE.y));
        WO[K] = make_float2(__fdividef(omega, dO.x), __fdividef(omega, dO.y));
      }
      constexpr int PI = ((K + 1) >> 1) & 1;  // parity of I = (t + 1) / 2
      if ((K & 1) || t == 0) EC[PI] = *(const float2 *)(se + (K * 32 + lane) * CB);
      // interpolation and correction of row t
      {
        constexpr int PA = (K >> 1) & 1, PB = PA ^ 1;  // parities of t / 2 and t / 2 + 1
        const float2 ce = (K & 1) ? mul2(half2, add2(EC[PA], EC[PB])) : EC[PA];  // (e0, e1)
        const float2 co = mul2(half2, add2(ce, make_float2(ce.y, shdn(ce.x))));   // (e0+e1, e1+e2) / 2
        const bool rowok = t >= 1 && t <= n - 2;
        const float2 vE = add2(UE[K], ce), vO = add2(UO[K], co);
        UE[K].x = rowok && mE[0] ? vE.x : UE[K].x;
        UE[K].y = rowok && mE[1] ? vE.y : UE[K].y;
        UO[K].x = rowok && mO[0] ? vO.x : UO[K].x;
        UO[K].y = rowok && mO[1] ? vO.y : UO[K].y;
      }
      static_for<1, 2 * NU + 1>([&](auto hc) {
        constexpr int h = decltype(hc)::value;
        constexpr int sc = (K - h) & (kSlots - 1), sa = (K - h - 1) & (kSlots - 1), sb = (K - h + 1) & (kSlots - 1);
        constexpr int PAR = ((h - 1) ^ (K - h)) & 1;
        const int r = t - h;
        const bool rowok = r >= 1 && r <= n - 2;
        const FacesX2 q = faces_x2(face_row(skx, r), face_row(sky, r), face_row(sky, r - 1));
        half_x2v<PAR>(UE[sc], UO[sc], UE[sa], UO[sa], UE[sb], UO[sb], FE[sc], FO[sc], WE[sc], WO[sc], q, rowok, mE,
                      mO, gam, has_gamma);
      });
      {
        const int r = t - 2 * NU;
        constexpr int sc = (K - 2 * NU) & (kSlots - 1);
        if (r >= r0 && r < r1 && out_lane)
          *(float4 *)(uout + (long long)r * pitch + c0) = make_float4(UE[sc].x, UO[sc].x, UE[sc].y, UO[sc].y);
      }
    });
  }
  cp_async_wait<0>();
}

}  // namespace fz
}  // namespace mg
