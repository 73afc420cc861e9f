// FP32 constant-stencil instance of k_pre2d (fused2d.cuh) written with the
// packed FP32x2 instructions of this GPU (__ffma2_rn / __fadd2_rn /
// __fmul2_rn): the same pass (nu RBGS sweeps + residual + full weighting),
// warp strips, row chunks, cp.async ring and register window, with
//
//  - a lane's four columns c0..c0+3 held as the pairs E = (c0, c0+2) and
//    O = (c0+1, c0+3): c0 is even, so the nodes one red-black half-sweep
//    updates in a row are exactly one pair, and each update is four pair
//    instructions (two sums of neighbours, two fused multiply-adds);
//  - the right-hand side scaled once per row, F = alpha f with
//    alpha = omega / diag, and the residual formed in the same scaling,
//    alpha r = F - omega u + bx (uw + ue) + by (us + un), which the
//    restriction multiplies back by 1 / (16 alpha) once per coarse node;
//  - the horizontal full-weighting sums (r_w + 2 r + r_e at the lane's two
//    even columns) kept per row instead of the residual rows;
//  - the colour of every half-sweep known at compile time (chunks start on
//    multiples of 8 rows, so the parity of row t - h follows from the
//    window slot).
// Rounding differs from the scalar instance only in the order of FP32
// operations, which the FP64 outer loop of defect correction absorbs.
#pragma once

#include "fused2d.cuh"

namespace mg {
namespace fz {

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// Pair coefficients used on every node; the per-row scale alpha and the
// per-coarse-node scale rsc = 1 / (16 alpha) stay scalars (registers).
struct CoefX2 {
  float2 bx, by, gam, nom;
  float alpha, rsc;
  bool has_gamma;
};

__device__ __forceinline__ CoefX2 coef_x2(const Args2D &a) {
  CoefX2 k;
  k.bx = splat2(a.betaxf);
  k.by = splat2(a.betayf);
  k.gam = splat2(a.gammaf);
  k.nom = splat2(-a.omegaf);
  k.alpha = a.alphaf;
  k.rsc = 0.0625f / a.alphaf;
  k.has_gamma = a.has_gamma != 0;
  return k;
}

// Half-sweep of row r (pairs E, O) with rows r-1 (A) and r+1 (B): PAR = 0
// updates the even columns (E), PAR = 1 the odd ones (O). CHECK: the row and
// the columns may touch the boundary (rowok, masks mE / mO per component).
template <bool CHECK, int PAR, bool G>
__device__ __forceinline__ void half_x2(float2 &E, float2 &O, const float2 &AE, const float2 &AO, const float2 &BE,
                                        const float2 &BO, const float2 &FE, const float2 &FO, bool rowok,
                                        const bool (&mE)[2], const bool (&mO)[2], const CoefX2 &k) {
  if constexpr (PAR == 0) {
    const float2 w = make_float2(shup(O.y), O.x);
    float2 v = fma2(k.bx, add2(w, O), fma2(k.by, add2(AE, BE), FE));
    if (G) v = fma2(k.gam, E, v);
    if (CHECK) {
      E.x = rowok && mE[0] ? v.x : E.x;
      E.y = rowok && mE[1] ? v.y : E.y;
    } else {
      E = v;
    }
  } else {
    const float2 e = make_float2(E.y, shdn(E.x));
    float2 v = fma2(k.bx, add2(E, e), fma2(k.by, add2(AO, BO), FO));
    if (G) v = fma2(k.gam, O, v);
    if (CHECK) {
      O.x = rowok && mO[0] ? v.x : O.x;
      O.y = rowok && mO[1] ? v.y : O.y;
    } else {
      O = v;
    }
  }
}

template <int NU, bool ZERO, bool LIST, bool G>
__global__ void __launch_bounds__(128, 4) k_pre2d_x2(Args2D a, const Args2D *__restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (LIST) {
    if (retired(list[blockIdx.y])) return;
    take_problem(a, list[blockIdx.y]);
  }
  constexpr int W = 4;  // warps per block
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
  const int rlim = min(n, tend + 1);  // rows staged: tstart .. rlim - 1
  const long long pitch = a.pitch;
  const float *uin = (const float *)a.uin;
  const float *f = (const float *)a.f;
  float *uout = (float *)a.uout;
  float *fc = (float *)a.fc;
  unsigned char *su = smem + (size_t)wib * kRing * 32 * 16 * 2;
  unsigned char *sf = su + kRing * 32 * 16;
  const CoefX2 k = coef_x2(a);
  bool mE[2], mO[2];
  mE[0] = c0 >= 1 && c0 <= n - 2;
  mO[0] = c0 + 1 >= 1 && c0 + 1 <= n - 2;
  mE[1] = c0 + 2 >= 1 && c0 + 2 <= n - 2;
  mO[1] = c0 + 3 >= 1 && c0 + 3 <= n - 2;
  const int J0 = c0 >> 1;

  float2 UE[kSlots], UO[kSlots], FE[kSlots], FO[kSlots], HR[kSlots];
#pragma unroll
  for (int i = 0; i < kSlots; i++) {
    UE[i] = UO[i] = FE[i] = FO[i] = HR[i] = make_float2(0.0f, 0.0f);
  }

  // Staging: this lane's 16 bytes of a row; sources advance by rows.
  const long long lane_off = col_ok ? c0 : 0;
  const float *gu = uin + (long long)tstart * pitch + lane_off;
  const float *gf = f + (long long)tstart * pitch + lane_off;
  int tnext = tstart;
  auto issue_group = [&](auto sb) {
    constexpr int SB = decltype(sb)::value;  // ring slot of the group's first row
#pragma unroll
    for (int j = 0; j < kGroup; j++) {
      const bool ok = col_ok && tnext + j < rlim;
      unsigned char *du = su + (((SB + j) & (kRing - 1)) * 32 + lane) * 16;
      unsigned char *df = sf + (((SB + j) & (kRing - 1)) * 32 + lane) * 16;
      if (!ZERO) cp_async16(du, ok ? (const void *)(gu + j * pitch) : (const void *)uin, ok);
      cp_async16(df, ok ? (const void *)(gf + j * pitch) : (const void *)f, ok);
    }
    cp_async_commit();
    tnext += kGroup;
    gu += kGroup * pitch;
    gf += kGroup * pitch;
  };

  const int tlast = tstart + ((tend - tstart) / kSlots + 1) * kSlots - 1;
  const bool interior_warp = x0 >= 1 && x0 + kCols - 1 <= n - 2 && tstart - 2 * NU - 2 >= 1 && tlast <= n - 2;

  auto body = [&](auto chk) {
    constexpr bool CHECK = decltype(chk)::value;
    issue_group(std::integral_constant<int, 0>{});
    for (int tb = tstart; tb <= tend; tb += kSlots) {
      static_for<0, kSlots>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int t = tb + K;
        if constexpr (K % kGroup == 0) {
          issue_group(std::integral_constant<int, (K + kGroup) & (kRing - 1)>{});
          cp_async_wait<1>();
        }
        // row t (ring slot K: tb is a multiple of kRing)
        if (!ZERO) {
          const float4 v = *(const float4 *)(su + (K * 32 + lane) * 16);
          UE[K] = make_float2(v.x, v.z);
          UO[K] = make_float2(v.y, v.w);
        } else {
          UE[K] = UO[K] = make_float2(0.0f, 0.0f);
        }
        {
          const float4 v = *(const float4 *)(sf + (K * 32 + lane) * 16);
          FE[K] = make_float2(k.alpha * v.x, k.alpha * v.z);
          FO[K] = make_float2(k.alpha * v.y, k.alpha * v.w);
        }
        // half-sweeps h = 1 .. 2 NU on rows t - h (odd h red, even h black)
        static_for<1, 2 * NU + 1>([&](auto hc) {
          constexpr int h = decltype(hc)::value;
          constexpr int sc = (K - h) & (kSlots - 1), sa = (K - h - 1) & (kSlots - 1), sb = (K - h + 1) & (kSlots - 1);
          constexpr int PAR = ((h - 1) ^ (K - h)) & 1;  // colour (h - 1) & 1 on row t - h, t = K mod 2
          const int r = t - h;
          const bool rowok = !CHECK || (r >= 1 && r <= n - 2);
          half_x2<CHECK, PAR, G>(UE[sc], UO[sc], UE[sa], UO[sa], UE[sb], UO[sb], FE[sc], FO[sc], rowok, mE, mO, k);
        });
        // final u of row t - 2 NU
        {
          const int r = t - 2 * NU;
          constexpr int sc = (K - 2 * NU) & (kSlots - 1);
          if (r >= r0 && r < r1 && out_lane)
            *(float4 *)(uout + (long long)r * pitch + c0) = make_float4(UE[sc].x, UO[sc].x, UE[sc].y, UO[sc].y);
        }
        // scaled residual of row t - 2 NU - 1 and its horizontal full-weighting sums
        {
          const int r = t - 2 * NU - 1;
          constexpr int sc = (K - 2 * NU - 1) & (kSlots - 1), sa = (K - 2 * NU - 2) & (kSlots - 1),
                        sb = (K - 2 * NU) & (kSlots - 1);
          const float2 E = UE[sc], O = UO[sc];
          const float2 w = make_float2(shup(O.y), O.x), e = make_float2(E.y, shdn(E.x));
          float2 rE = fma2(k.by, add2(UE[sa], UE[sb]), fma2(k.bx, add2(w, O), fma2(k.nom, E, FE[sc])));
          float2 rO = fma2(k.by, add2(UO[sa], UO[sb]), fma2(k.bx, add2(E, e), fma2(k.nom, O, FO[sc])));
          if (CHECK) {
            const bool rowok = r >= 1 && r <= n - 2;
            rE.x = rowok && mE[0] ? rE.x : 0.0f;
            rE.y = rowok && mE[1] ? rE.y : 0.0f;
            rO.x = rowok && mO[0] ? rO.x : 0.0f;
            rO.y = rowok && mO[1] ? rO.y : 0.0f;
          }
          HR[sc] = add2(add2(rE, rE), add2(make_float2(shup(rO.y), rO.x), rO));
          // restriction once the row below the coarse row is ready (r = 2I + 1)
          if constexpr (((K - 2 * NU - 1) & 1) != 0) {
            constexpr int sA = (K - 2 * NU - 3) & (kSlots - 1), sB = (K - 2 * NU - 2) & (kSlots - 1);
            const float2 t2 = add2(add2(HR[sB], HR[sB]), add2(HR[sA], HR[sc]));
            const float2 v = make_float2(k.rsc * t2.x, k.rsc * t2.y);
            const int I = (r - 1) >> 1;
            if (out_lane && I >= 1 && I <= a.nc - 2 && 2 * I >= r0 && 2 * I < r1) {
              float *row = fc + (long long)I * a.pitchc + J0;
              if (!CHECK) {
                *(float2 *)row = v;
              } else {
                if (J0 >= 1 && J0 <= a.nc - 2) row[0] = v.x;
                if (J0 + 1 >= 1 && J0 + 1 <= a.nc - 2) row[1] = v.y;
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

// Interpolation + correction + nu RBGS sweeps (k_post2d, FP32, constant
// stencil) with the same pair layout: a lane's coarse values at J0 = c0 / 2
// and J0 + 1 form one pair, so the correction of a fine row is (e0, e1) on
// the even columns and the averages (e0 + e1, e1 + e2) / 2 on the odd ones.
template <int NU, bool LIST, bool G>
__global__ void __launch_bounds__(128, 4) k_post2d_x2(Args2D a, const Args2D *__restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (LIST) {
    if (retired(list[blockIdx.y])) return;
    take_problem(a, list[blockIdx.y]);
  }
  constexpr int W = 4;
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
  float *uout = (float *)a.uout;
  constexpr int CB = 8;  // two coarse values per lane
  unsigned char *su = smem + (size_t)wib * kRing * 32 * (16 + 16 + CB);
  unsigned char *sf = su + kRing * 32 * 16;
  unsigned char *se = sf + kRing * 32 * 16;
  const CoefX2 k = coef_x2(a);
  bool mE[2], mO[2];
  mE[0] = c0 >= 1 && c0 <= n - 2;
  mO[0] = c0 + 1 >= 1 && c0 + 1 <= n - 2;
  mE[1] = c0 + 2 >= 1 && c0 + 2 <= n - 2;
  mO[1] = c0 + 3 >= 1 && c0 + 3 <= n - 2;
  const float2 half2 = splat2(0.5f);

  float2 UE[kSlots], UO[kSlots], FE[kSlots], FO[kSlots];
#pragma unroll
  for (int i = 0; i < kSlots; i++) UE[i] = UO[i] = FE[i] = FO[i] = make_float2(0.0f, 0.0f);
  // coarse rows by parity of the coarse row index (values at J0, J0 + 1)
  float2 EC[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};

  const long long lane_off = col_ok ? c0 : 0;
  const float *gu = uin + (long long)tstart * pitch + lane_off;
  const float *gf = f + (long long)tstart * pitch + lane_off;
  int tnext = tstart;
  // With fine row `row` also stage coarse row (row + 1) / 2 when row is odd,
  // and coarse row 0 with fine row 0.
  auto issue_group = [&](auto sb) {
    constexpr int SB = decltype(sb)::value;
#pragma unroll
    for (int j = 0; j < kGroup; j++) {
      const int row = tnext + j;
      const bool ok = col_ok && row < rlim;
      const int slot = (SB + j) & (kRing - 1);
      cp_async16(su + (slot * 32 + lane) * 16, ok ? (const void *)(gu + j * pitch) : (const void *)uin, ok);
      cp_async16(sf + (slot * 32 + lane) * 16, ok ? (const void *)(gf + j * pitch) : (const void *)f, ok);
      const int I = (j & 1) ? (row + 1) >> 1 : (row == 0 ? 0 : -1);  // row has the parity of j
      const bool cok = ccol_ok && row <= tend && I >= 0 && I < a.nc;
      cp_async8(se + (slot * 32 + lane) * CB, cok ? (const void *)(ec + (long long)I * pitchc + J0) : (const void *)ec, cok);
    }
    cp_async_commit();
    tnext += kGroup;
    gu += kGroup * pitch;
    gf += kGroup * pitch;
  };

  const int tlast = tstart + ((tend - tstart) / kSlots + 1) * kSlots - 1;
  const bool interior_warp = x0 >= 1 && x0 + kCols - 1 <= n - 2 && tstart - 2 * NU >= 1 && tlast <= n - 2;

  // coarse row tstart / 2 (even index) precedes the window when the chunk starts inside the grid
  if (tstart > 0) {
    const int I = tstart >> 1;
    if (ccol_ok && I < a.nc) EC[0] = *(const float2 *)(ec + (long long)I * pitchc + J0);
  }

  auto body = [&](auto chk) {
    constexpr bool CHECK = decltype(chk)::value;
    issue_group(std::integral_constant<int, 0>{});
    for (int tb = tstart; tb <= tend; tb += kSlots) {
      static_for<0, kSlots>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int t = tb + K;
        if constexpr (K % kGroup == 0) {
          issue_group(std::integral_constant<int, (K + kGroup) & (kRing - 1)>{});
          cp_async_wait<1>();
        }
        {
          const float4 v = *(const float4 *)(su + (K * 32 + lane) * 16);
          UE[K] = make_float2(v.x, v.z);
          UO[K] = make_float2(v.y, v.w);
        }
        {
          const float4 v = *(const float4 *)(sf + (K * 32 + lane) * 16);
          FE[K] = make_float2(k.alpha * v.x, k.alpha * v.z);
          FO[K] = make_float2(k.alpha * v.y, k.alpha * v.w);
        }
        constexpr int PI = ((K + 1) >> 1) & 1;  // parity of I = (t + 1) / 2
        if ((K & 1) || (CHECK && t == 0)) EC[PI] = *(const float2 *)(se + (K * 32 + lane) * CB);
        // interpolation and correction of row t
        {
          constexpr int PA = (K >> 1) & 1, PB = PA ^ 1;  // parities of t / 2 and t / 2 + 1
          const float2 ce = (K & 1) ? mul2(half2, add2(EC[PA], EC[PB])) : EC[PA];  // (e0, e1)
          const float2 co = mul2(half2, add2(ce, make_float2(ce.y, shdn(ce.x))));   // (e0+e1, e1+e2) / 2
          if (!CHECK) {
            UE[K] = add2(UE[K], ce);
            UO[K] = add2(UO[K], co);
          } else {
            const bool rowok = t >= 1 && t <= n - 2;
            const float2 vE = add2(UE[K], ce), vO = add2(UO[K], co);
            UE[K].x = rowok && mE[0] ? vE.x : UE[K].x;
            UE[K].y = rowok && mE[1] ? vE.y : UE[K].y;
            UO[K].x = rowok && mO[0] ? vO.x : UO[K].x;
            UO[K].y = rowok && mO[1] ? vO.y : UO[K].y;
          }
        }
        static_for<1, 2 * NU + 1>([&](auto hc) {
          constexpr int h = decltype(hc)::value;
          constexpr int sc = (K - h) & (kSlots - 1), sa = (K - h - 1) & (kSlots - 1), sb = (K - h + 1) & (kSlots - 1);
          constexpr int PAR = ((h - 1) ^ (K - h)) & 1;
          const int r = t - h;
          const bool rowok = !CHECK || (r >= 1 && r <= n - 2);
          half_x2<CHECK, PAR, G>(UE[sc], UO[sc], UE[sa], UO[sa], UE[sb], UO[sb], FE[sc], FO[sc], rowok, mE, mO, k);
        });
        {
          const int r = t - 2 * NU;
          constexpr int sc = (K - 2 * NU) & (kSlots - 1);
          if (r >= r0 && r < r1 && out_lane)
            *(float4 *)(uout + (long long)r * pitch + c0) = make_float4(UE[sc].x, UO[sc].x, UE[sc].y, UO[sc].y);
        }
      });
    }
  };
  if (interior_warp) body(std::false_type{});
  else body(std::true_type{});
  cp_async_wait<0>();
}

// Post-smoothing of one V-cycle and pre-smoothing of the next on the same
// level in one pass: interpolation and correction of each arriving row,
// then NUA + NUB RBGS sweeps (the NUA post-smoothing sweeps followed by the
// NUB pre-smoothing sweeps, red before black in each), the scaled residual
// and full weighting into the coarse right-hand side - the same operations in
// the same order as k_post2d_x2<NUA> followed by k_pre2d_x2<NUB, false>, but
// u and f are read once and u written once. Between two inner cycles of a
// defect-correction step the finest level does exactly this. The register
// window holds 2 (NUA + NUB) + 3 rows (10 for V(2,1)), so rows stream in
// periods of kPS = 10 through a 10-row cp.async ring filled in groups of 5;
// the window slot of row t is t mod 10 (chunks start on even rows, so the
// colour of every half-sweep is still a compile-time constant), and the
// parity of the coarse row index, which alternates with the period, is taken
// at run time. Every warp runs the code with boundary predicates: the
// unrolled 10-row period is long enough that a second, predicate-free copy
// for interior warps cost more in instruction-fetch stalls than the
// predicates (200 -> 185 us at 8193^2 without it).
constexpr int kPS = 10;      // rows per period (register window and ring)
constexpr int kPGroup = 5;   // rows per cp.async group: two groups in flight

template <int NUA, int NUB, bool G>
__global__ void __launch_bounds__(128, 3) k_postpre2d_x2(Args2D a) {
  constexpr int NU = NUA + NUB;
  static_assert(2 * NU + 3 <= kPS, "the row window must hold 2 (NUA + NUB) + 3 rows");
  static_assert(2 * NU + 2 <= kHalo, "the column halo must cover the sweeps, the residual and the restriction");
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int W = 4;
  constexpr int CB = 8;  // two coarse values per lane
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
  const int tstart = max(r0 - 8, 0);  // even (R is a multiple of 8)
  const int tend = r1 + 2 * NU;       // inclusive: residual of row r1 - 1 needs u up to r1 + 2 NU
  const int rlim = min(n, tend + 1);  // rows staged: tstart .. rlim - 1
  const long long pitch = a.pitch, pitchc = a.pitchc;
  const float *uin = (const float *)a.uin;
  const float *f = (const float *)a.f;
  const float *ec = (const float *)a.ec;
  float *uout = (float *)a.uout;
  float *fc = (float *)a.fc;
  unsigned char *su = smem + (size_t)wib * kPS * 32 * (16 + 16 + CB);
  unsigned char *sf = su + kPS * 32 * 16;
  unsigned char *se = sf + kPS * 32 * 16;
  const CoefX2 k = coef_x2(a);
  bool mE[2], mO[2];
  mE[0] = c0 >= 1 && c0 <= n - 2;
  mO[0] = c0 + 1 >= 1 && c0 + 1 <= n - 2;
  mE[1] = c0 + 2 >= 1 && c0 + 2 <= n - 2;
  mO[1] = c0 + 3 >= 1 && c0 + 3 <= n - 2;
  const float2 half2 = splat2(0.5f);

  float2 UE[kPS], UO[kPS], FE[kPS], FO[kPS], HR[kPS];
#pragma unroll
  for (int i = 0; i < kPS; i++) UE[i] = UO[i] = FE[i] = FO[i] = HR[i] = make_float2(0.0f, 0.0f);
  // coarse rows of even and odd index (values at J0, J0 + 1)
  float2 EC0 = make_float2(0.0f, 0.0f), EC1 = make_float2(0.0f, 0.0f);

  const long long lane_off = col_ok ? c0 : 0;
  const float *gu = uin + (long long)tstart * pitch + lane_off;
  const float *gf = f + (long long)tstart * pitch + lane_off;
  int tnext = tstart;
  // With fine row `row` also stage coarse row (row + 1) / 2 when row is odd,
  // and coarse row 0 with fine row 0.
  auto issue_group = [&](auto sb) {
    constexpr int SB = decltype(sb)::value;
#pragma unroll
    for (int j = 0; j < kPGroup; j++) {
      const int row = tnext + j;
      const bool ok = col_ok && row < rlim;
      const int slot = (SB + j) % kPS;
      cp_async16(su + (slot * 32 + lane) * 16, ok ? (const void *)(gu + j * pitch) : (const void *)uin, ok);
      cp_async16(sf + (slot * 32 + lane) * 16, ok ? (const void *)(gf + j * pitch) : (const void *)f, ok);
      const int I = (row & 1) ? (row + 1) >> 1 : (row == 0 ? 0 : -1);
      const bool cok = ccol_ok && row <= tend && I >= 0 && I < a.nc;
      cp_async8(se + (slot * 32 + lane) * CB, cok ? (const void *)(ec + (long long)I * pitchc + J0) : (const void *)ec, cok);
    }
    cp_async_commit();
    tnext += kPGroup;
    gu += kPGroup * pitch;
    gf += kPGroup * pitch;
  };

  const int tlast = tstart + ((tend - tstart) / kPS + 1) * kPS - 1;
  const bool interior_warp = x0 >= 1 && x0 + kCols - 1 <= n - 2 && tstart - 2 * NU - 2 >= 1 && tlast <= n - 2;

  // coarse row tstart / 2 (even fine row, so no staging brings it) precedes the window
  if (tstart > 0) {
    const int I = tstart >> 1;
    if (ccol_ok && I < a.nc) {
      const float2 v = *(const float2 *)(ec + (long long)I * pitchc + J0);
      if (I & 1) EC1 = v;
      else EC0 = v;
    }
  }

  auto body = [&](auto chk) {
    constexpr bool CHECK = decltype(chk)::value;
    issue_group(std::integral_constant<int, 0>{});
    for (int tb = tstart; tb <= tend; tb += kPS) {
      static_for<0, kPS>([&](auto kc) {
        constexpr int K = decltype(kc)::value;
        const int t = tb + K;  // t and K have the same parity
        if constexpr (K % kPGroup == 0) {
          issue_group(std::integral_constant<int, (K + kPGroup) % kPS>{});
          cp_async_wait<1>();
        }
        {
          const float4 v = *(const float4 *)(su + (K * 32 + lane) * 16);
          UE[K] = make_float2(v.x, v.z);
          UO[K] = make_float2(v.y, v.w);
        }
        {
          const float4 v = *(const float4 *)(sf + (K * 32 + lane) * 16);
          FE[K] = make_float2(k.alpha * v.x, k.alpha * v.z);
          FO[K] = make_float2(k.alpha * v.y, k.alpha * v.w);
        }
        // coarse row (t + 1) / 2 arrives with odd rows (and row 0)
        if ((K & 1) || (CHECK && t == 0)) {
          const float2 v = *(const float2 *)(se + (K * 32 + lane) * CB);
          if (((t + 1) >> 1) & 1) EC1 = v;
          else EC0 = v;
        }
        // interpolation and correction of row t
        {
          const bool pa = (t >> 1) & 1;  // parity of t / 2
          const float2 ca = pa ? EC1 : EC0, cb = pa ? EC0 : EC1;
          const float2 ce = (K & 1) ? mul2(half2, add2(ca, cb)) : ca;                // (e0, e1)
          const float2 co = mul2(half2, add2(ce, make_float2(ce.y, shdn(ce.x))));   // (e0+e1, e1+e2) / 2
          if (!CHECK) {
            UE[K] = add2(UE[K], ce);
            UO[K] = add2(UO[K], co);
          } else {
            const bool rowok = t >= 1 && t <= n - 2;
            const float2 vE = add2(UE[K], ce), vO = add2(UO[K], co);
            UE[K].x = rowok && mE[0] ? vE.x : UE[K].x;
            UE[K].y = rowok && mE[1] ? vE.y : UE[K].y;
            UO[K].x = rowok && mO[0] ? vO.x : UO[K].x;
            UO[K].y = rowok && mO[1] ? vO.y : UO[K].y;
          }
        }
        // half-sweeps h = 1 .. 2 NU on rows t - h (odd h red, even h black)
        static_for<1, 2 * NU + 1>([&](auto hc) {
          constexpr int h = decltype(hc)::value;
          constexpr int sc = (K - h + 2 * kPS) % kPS, sa = (K - h - 1 + 2 * kPS) % kPS, sb = (K - h + 1 + 2 * kPS) % kPS;
          constexpr int PAR = ((h - 1) ^ (K - h + 2 * kPS)) & 1;
          const int r = t - h;
          const bool rowok = !CHECK || (r >= 1 && r <= n - 2);
          half_x2<CHECK, PAR, G>(UE[sc], UO[sc], UE[sa], UO[sa], UE[sb], UO[sb], FE[sc], FO[sc], rowok, mE, mO, k);
        });
        // final u of row t - 2 NU
        {
          const int r = t - 2 * NU;
          constexpr int sc = (K - 2 * NU + 2 * kPS) % kPS;
          if (r >= r0 && r < r1 && out_lane)
            *(float4 *)(uout + (long long)r * pitch + c0) = make_float4(UE[sc].x, UO[sc].x, UE[sc].y, UO[sc].y);
        }
        // scaled residual of row t - 2 NU - 1 and its horizontal full-weighting sums
        {
          const int r = t - 2 * NU - 1;
          constexpr int sc = (K - 2 * NU - 1 + 2 * kPS) % kPS, sa = (K - 2 * NU - 2 + 2 * kPS) % kPS,
                        sb = (K - 2 * NU + 2 * kPS) % kPS;
          const float2 E = UE[sc], O = UO[sc];
          const float2 w = make_float2(shup(O.y), O.x), e = make_float2(E.y, shdn(E.x));
          float2 rE = fma2(k.by, add2(UE[sa], UE[sb]), fma2(k.bx, add2(w, O), fma2(k.nom, E, FE[sc])));
          float2 rO = fma2(k.by, add2(UO[sa], UO[sb]), fma2(k.bx, add2(E, e), fma2(k.nom, O, FO[sc])));
          if (CHECK) {
            const bool rowok = r >= 1 && r <= n - 2;
            rE.x = rowok && mE[0] ? rE.x : 0.0f;
            rE.y = rowok && mE[1] ? rE.y : 0.0f;
            rO.x = rowok && mO[0] ? rO.x : 0.0f;
            rO.y = rowok && mO[1] ? rO.y : 0.0f;
          }
          HR[sc] = add2(add2(rE, rE), add2(make_float2(shup(rO.y), rO.x), rO));
          // restriction once the row below the coarse row is ready (r = 2I + 1)
          if constexpr (((K - 2 * NU - 1 + 2 * kPS) & 1) != 0) {
            constexpr int sA = (K - 2 * NU - 3 + 2 * kPS) % kPS, sB = (K - 2 * NU - 2 + 2 * kPS) % kPS;
            const float2 t2 = add2(add2(HR[sB], HR[sB]), add2(HR[sA], HR[sc]));
            const float2 v = make_float2(k.rsc * t2.x, k.rsc * t2.y);
            const int I = (r - 1) >> 1;
            if (out_lane && I >= 1 && I <= a.nc - 2 && 2 * I >= r0 && 2 * I < r1) {
              float *row = fc + (long long)I * a.pitchc + J0;
              if (!CHECK) {
                *(float2 *)row = v;
              } else {
                if (J0 >= 1 && J0 <= a.nc - 2) row[0] = v.x;
                if (J0 + 1 >= 1 && J0 + 1 <= a.nc - 2) row[1] = v.y;
              }
            }
          }
        }
      });
    }
  };
  (void)interior_warp;
  body(std::true_type{});
  cp_async_wait<0>();
}

}  // namespace fz
}  // namespace mg
