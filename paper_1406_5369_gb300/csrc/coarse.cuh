// Single-block V-cycle on the small coarse levels (Algorithm 1 below a size
// threshold): one block of 1024 threads loads the top level's right-hand
// side (and solution, unless it starts from zero), runs presmoothing,
// residual, full weighting, the exact 3^dim solve, interpolation and
// postsmoothing on every level below in shared memory with block barriers
// between the stages, and writes the top level's solution back. It replaces
// some 10 kernel launches per level, whose latency dominates these levels.
//
// Arithmetic runs in C (double in FP64 contexts, float for the inner levels
// of defect correction); the 3^dim solve runs in FP64 as everywhere else.
// In 2D (n <= 65) each stage maps thread t to row 1 + t/64 (+16 k) and
// column 1 + t%64, or, for a red-black half-sweep, to row 1 + t/32 (+32 k)
// and the (t%32)-th column of the sweep's colour in that row.
#pragma once

#include "kernels.cuh"

namespace mg {
namespace cz {

constexpr int kThreads = 1024;
constexpr int kMaxLev = 8;

struct CoarseArgs {
  int dim, nlev;           // levels handled: top (index 0 here) .. coarsest
  int n[kMaxLev];
  int off_u[kMaxLev], off_f[kMaxLev], off_k[kMaxLev];  // element offsets in shared memory
  int off_tmp, total;
  double inv_h2[kMaxLev];
  double c[3];
  int var;                 // face coefficients present
  const void *kf[kMaxLev][3];
  int kf64[kMaxLev];       // faces stored as double (else float)
  int pitch[kMaxLev];      // element pitch of each level's global arrays
  long long plane[kMaxLev];
  const void *f_top;       // top level right-hand side (global)
  void *u_top;             // top level solution (global, read unless zero_top)
  int top_dtype;           // DType of the top level's fields
  int zero_top;
  int smoother;            // 0 RBGS, 1 Jacobi
  double omega;
  int nu1, nu2;
  // inv_h2, c and omega rounded to FP32 on the host, for FP32 cycles
  float inv_h2f[kMaxLev];
  float cf[3];
  float omegaf;
  // coarsest grid of 5^dim or 9^dim nodes: FP64 inverse of its operator
  // (global, N x N) and the element offset of N FP64 residual slots in
  // shared memory; NULL for a 3^dim coarsest grid
  const double *dense;
  int off_rd;
  // batched cycles of a captured batch step: the problem's live flag in
  // device memory; the block returns at once when it is 0 (NULL: always live)
  const int *live;
};

// Element i of a global field of type dtype, in the cycle's compute type C
// (no round trip through double for float fields).
template <typename C> __device__ __forceinline__ C ldg_as(const void *p, long long i, int dtype) {
  if (dtype == F64) return (C)((const double *)p)[i];
  if (dtype == F32) return (C)((const float *)p)[i];
  return (C)__bfloat162float(((const bf16 *)p)[i]);
}
template <typename C> __device__ __forceinline__ void stg_as(void *p, long long i, int dtype, C v) {
  if (dtype == F64) ((double *)p)[i] = (double)v;
  else if (dtype == F32) ((float *)p)[i] = (float)v;
  else ((bf16 *)p)[i] = bf16_rne((float)v);
}

template <int DIM> __device__ __forceinline__ int npts(int n) { return DIM == 3 ? n * n * n : n * n; }

// Interior node t (0 <= t < (n-2)^DIM) of a dense n^DIM array (3D loops).
template <int DIM> __device__ __forceinline__ int inode(int t, int n, int &i, int &j, int &k) {
  int m = n - 2;
  i = 1 + t % m;
  int rest = t / m;
  j = 1 + (DIM == 3 ? rest % m : rest);
  k = DIM == 3 ? 1 + rest / m : 0;
  return (k * n + j) * n + i;
}

template <typename C> struct Lev {
  C *u, *f, *kx, *ky, *kz;
  int n;
  C ih2;
};

template <int DIM, bool VAR, typename C>
__device__ __forceinline__ Lev<C> level(const CoarseArgs &a, C *sm, int l) {
  Lev<C> L;
  int N = npts<DIM>(a.n[l]);
  L.n = a.n[l];
  L.ih2 = pick<C>(a.inv_h2[l], a.inv_h2f[l]);
  L.u = sm + a.off_u[l];
  L.f = sm + a.off_f[l];
  L.kx = VAR ? sm + a.off_k[l] : nullptr;
  L.ky = VAR ? sm + a.off_k[l] + N : nullptr;
  L.kz = (VAR && DIM == 3) ? sm + a.off_k[l] + 2 * N : nullptr;
  return L;
}

// A u and diag at dense node p.
template <int DIM, bool VAR, typename C>
__device__ __forceinline__ void dense_apply(const Lev<C> &L, const C *u, int p, const C (&c)[3], C &Au, C &dg) {
  int sy = L.n, sz = L.n * L.n;
  C u0 = u[p];
  if (!VAR) {
    C acc = c[0] * ((u0 - u[p - 1]) + (u0 - u[p + 1])) + c[1] * ((u0 - u[p - sy]) + (u0 - u[p + sy]));
    C d = c[0] + c[1];
    if (DIM == 3) {
      acc += c[2] * ((u0 - u[p - sz]) + (u0 - u[p + sz]));
      d += c[2];
    }
    Au = acc * L.ih2;
    dg = (C)2 * d * L.ih2;
  } else {
    C kxp = L.kx[p], kxm = L.kx[p - 1], kyp = L.ky[p], kym = L.ky[p - sy];
    C acc = kxp * (u0 - u[p + 1]) + kxm * (u0 - u[p - 1]) + kyp * (u0 - u[p + sy]) + kym * (u0 - u[p - sy]);
    C d = kxp + kxm + kyp + kym;
    if (DIM == 3) {
      C kzp = L.kz[p], kzm = L.kz[p - sz];
      acc += kzp * (u0 - u[p + sz]) + kzm * (u0 - u[p - sz]);
      d += kzp + kzm;
    }
    Au = acc * L.ih2;
    dg = d * L.ih2;
  }
}

// Calls body(p, i, j, k) for every interior node of an n^DIM level.
template <int DIM, typename Fn> __device__ __forceinline__ void for_interior(int n, Fn &&body) {
  if (DIM == 2) {
    int i = 1 + (threadIdx.x & 63);
    if (i <= n - 2)
      for (int j = 1 + (threadIdx.x >> 6); j <= n - 2; j += kThreads / 64) body(j * n + i, i, j, 0);
  } else {
    int m = n - 2, cnt = m * m * m;
    for (int t = threadIdx.x; t < cnt; t += kThreads) {
      int i, j, k;
      int p = inode<DIM>(t, n, i, j, k);
      body(p, i, j, k);
    }
  }
}

// Calls body(p) for every interior node of colour `color` ((i+j[+k]) % 2).
template <int DIM, typename Fn> __device__ __forceinline__ void for_colour(int n, int color, Fn &&body) {
  if (DIM == 2) {
    int lane = threadIdx.x & 31;
    for (int j = 1 + (threadIdx.x >> 5); j <= n - 2; j += kThreads / 32) {
      int i = 2 * lane + ((color + j) & 1);
      if (i >= 1 && i <= n - 2) body(j * n + i);
    }
  } else {
    int m = n - 2, cnt = m * m * m;
    for (int t = threadIdx.x; t < cnt; t += kThreads) {
      int i, j, k;
      int p = inode<DIM>(t, n, i, j, k);
      if (((i + j + k) & 1) == color) body(p);
    }
  }
}

template <int DIM, bool VAR, typename C>
__device__ void smooth(const Lev<C> &L, C *tmp, const C (&c)[3], int smoother, C omega, int sweeps) {
  // constant stencil: omega / diag once per level instead of a division per node
  const C wconst = omega / ((C)2 * (c[0] + c[1] + (DIM == 3 ? c[2] : (C)0)) * L.ih2);
  for (int s = 0; s < sweeps; s++) {
    if (smoother == 0) {
      for (int color = 0; color < 2; color++) {
        for_colour<DIM>(L.n, color, [&](int p) {
          C Au, dg;
          dense_apply<DIM, VAR>(L, L.u, p, c, Au, dg);
          L.u[p] = L.u[p] + (VAR ? omega / dg : wconst) * (L.f[p] - Au);
        });
        __syncthreads();
      }
    } else {
      int N = npts<DIM>(L.n);
      for (int p = threadIdx.x; p < N; p += kThreads) tmp[p] = L.u[p];
      __syncthreads();
      for_interior<DIM>(L.n, [&](int p, int, int, int) {
        C Au, dg;
        dense_apply<DIM, VAR>(L, tmp, p, c, Au, dg);
        L.u[p] = tmp[p] + (VAR ? omega / dg : wconst) * (L.f[p] - Au);
      });
      __syncthreads();
    }
  }
}

template <int DIM, bool VAR, typename C> __device__ void cycle_in_smem(const CoarseArgs &a, C *sm);

template <int DIM, bool VAR, typename C>
__device__ __forceinline__ void coarse_cycle_body(const CoarseArgs &a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *sm = (C *)smem_raw;
  for (int p = threadIdx.x; p < a.total; p += kThreads) sm[p] = (C)0;
  __syncthreads();
  // load the top level (and the faces of every level)
  {
    Lev<C> T = level<DIM, VAR, C>(a, sm, 0);
    int n = a.n[0], N = npts<DIM>(n);
    for (int p = threadIdx.x; p < N; p += kThreads) {
      int i = p % n, j = (p / n) % n, k = DIM == 3 ? p / (n * n) : 0;
      long long g = (long long)k * a.plane[0] + (long long)j * a.pitch[0] + i;
      T.f[p] = ldg_as<C>(a.f_top, g, a.top_dtype);
      if (!a.zero_top) T.u[p] = ldg_as<C>(a.u_top, g, a.top_dtype);
    }
    if (VAR) {
      for (int l = 0; l < a.nlev; l++) {
        int nl = a.n[l], Nl = npts<DIM>(nl);
        C *dst = sm + a.off_k[l];
        for (int d = 0; d < DIM; d++) {
          for (int p = threadIdx.x; p < Nl; p += kThreads) {
            int i = p % nl, j = (p / nl) % nl, k = DIM == 3 ? p / (nl * nl) : 0;
            long long g = (long long)k * a.plane[l] + (long long)j * a.pitch[l] + i;
            dst[d * Nl + p] = a.kf64[l] ? (C)((const double *)a.kf[l][d])[g] : (C)((const float *)a.kf[l][d])[g];
          }
        }
      }
    }
  }
  __syncthreads();
  cycle_in_smem<DIM, VAR, C>(a, sm);
  // write back the top level's solution
  {
    Lev<C> T = level<DIM, VAR, C>(a, sm, 0);
    for_interior<DIM>(a.n[0], [&](int p, int i, int j, int k) {
      long long g = (long long)k * a.plane[0] + (long long)j * a.pitch[0] + i;
      stg_as<C>(a.u_top, g, a.top_dtype, T.u[p]);
    });
  }
}

// The V-cycle of levels 0 .. a.nlev-1 held in shared memory at sm (offsets
// in a): level 0's right-hand side and solution are in place, every coarser
// solution is zero. Ends with level 0's solution in place (after a block
// barrier).
template <int DIM, bool VAR, typename C> __device__ void cycle_in_smem(const CoarseArgs &a, C *sm) {
  const C c[3] = {pick<C>(a.c[0], a.cf[0]), pick<C>(a.c[1], a.cf[1]), pick<C>(a.c[2], a.cf[2])};
  const C omega = pick<C>(a.omega, a.omegaf);
  C *tmp = sm + a.off_tmp;
  // descend
  for (int l = 0; l + 1 < a.nlev; l++) {
    const Lev<C> F = level<DIM, VAR, C>(a, sm, l);
    const Lev<C> G = level<DIM, VAR, C>(a, sm, l + 1);
    smooth<DIM, VAR, C>(F, tmp, c, a.smoother, omega, a.nu1);
    // residual into tmp at interior nodes (the restriction reads only those)
    for_interior<DIM>(F.n, [&](int p, int, int, int) {
      C Au, dg;
      dense_apply<DIM, VAR>(F, F.u, p, c, Au, dg);
      tmp[p] = F.f[p] - Au;
    });
    __syncthreads();
    // full weighting into the coarse right-hand side; the coarse u is 0
    const int nf = F.n;
    for_interior<DIM>(G.n, [&](int P, int I, int J, int K) {
      C acc = 0;
      for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++)
        for (int dy = -1; dy <= 1; dy++) {
          const C *row = tmp + ((DIM == 3 ? 2 * K + dz : 0) * nf + 2 * J + dy) * nf + 2 * I;
          C line = (C)0.25 * (row[-1] + row[1]) + (C)0.5 * row[0];
          C w = (dy == 0 ? (C)0.5 : (C)0.25) * (DIM == 3 ? (dz == 0 ? (C)0.5 : (C)0.25) : (C)1);
          acc += w * line;
        }
      G.f[P] = acc;
    });
    __syncthreads();
  }
  // coarsest level, solved exactly in FP64: the residual of the coarsest
  // operator at its interior nodes, then one unknown (3^dim) divided by the
  // diagonal or u += A^{-1} r with the dense inverse
  {
    const Lev<C> Z = level<DIM, VAR, C>(a, sm, a.nlev - 1);
    const double ih2 = a.inv_h2[a.nlev - 1];
    const int nz = Z.n, sy = nz, sz = nz * nz;
    // (r_p, diag_p) in FP64 from the stored (C) values
    auto resid = [&](int p, double &dg) {
      double acc;
      const double u0 = (double)Z.u[p];
      if (!VAR) {
        const double d = a.c[0] + a.c[1] + (DIM == 3 ? a.c[2] : 0.0);
        acc = a.c[0] * ((u0 - (double)Z.u[p - 1]) + (u0 - (double)Z.u[p + 1])) +
              a.c[1] * ((u0 - (double)Z.u[p - sy]) + (u0 - (double)Z.u[p + sy]));
        if (DIM == 3) acc += a.c[2] * ((u0 - (double)Z.u[p - sz]) + (u0 - (double)Z.u[p + sz]));
        dg = 2.0 * d * ih2;
      } else {
        const double kxp = Z.kx[p], kxm = Z.kx[p - 1], kyp = Z.ky[p], kym = Z.ky[p - sy];
        acc = kxp * (u0 - (double)Z.u[p + 1]) + kxm * (u0 - (double)Z.u[p - 1]) + kyp * (u0 - (double)Z.u[p + sy]) +
              kym * (u0 - (double)Z.u[p - sy]);
        double d = kxp + kxm + kyp + kym;
        if (DIM == 3) {
          const double kzp = Z.kz[p], kzm = Z.kz[p - sz];
          acc += kzp * (u0 - (double)Z.u[p + sz]) + kzm * (u0 - (double)Z.u[p - sz]);
          d += kzp + kzm;
        }
        dg = d * ih2;
      }
      return (double)Z.f[p] - acc * ih2;
    };
    if (!a.dense) {
      if (threadIdx.x == 0) {
        const int p = DIM == 3 ? 13 : 4;
        double dg;
        const double r = resid(p, dg);
        Z.u[p] = (C)((double)Z.u[p] + r / dg);
      }
    } else {
      double *rd = (double *)(sm + a.off_rd);
      const int m = nz - 2, N = DIM == 3 ? m * m * m : m * m;
      for (int t = threadIdx.x; t < N; t += kThreads) {
        int i, j, k;
        double dg;
        rd[t] = resid(inode<DIM>(t, nz, i, j, k), dg);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < N; t += kThreads) {
        double acc = 0.0;
        for (int q = 0; q < N; q++) acc += a.dense[(long long)q * N + t] * rd[q];
        int i, j, k;
        const int p = inode<DIM>(t, nz, i, j, k);
        Z.u[p] = (C)((double)Z.u[p] + acc);
      }
    }
  }
  __syncthreads();
  // ascend: interpolation and correction, postsmoothing
  for (int l = a.nlev - 2; l >= 0; l--) {
    const Lev<C> F = level<DIM, VAR, C>(a, sm, l);
    const Lev<C> G = level<DIM, VAR, C>(a, sm, l + 1);
    const int nc = G.n;
    for_interior<DIM>(F.n, [&](int p, int i, int j, int k) {
      int I = i >> 1, J = j >> 1, K = k >> 1;
      int oi = i & 1, oj = j & 1, ok = DIM == 3 ? (k & 1) : 0;
      C acc = 0;
      for (int a3 = 0; a3 <= ok; a3++)
        for (int b = 0; b <= oj; b++) {
          const C *row = G.u + ((K + a3) * nc + J + b) * nc + I;
          acc += oi ? (C)0.5 * (row[0] + row[1]) : row[0];
        }
      C w = (oj ? (C)0.5 : (C)1) * (ok ? (C)0.5 : (C)1);
      F.u[p] += w * acc;
    });
    __syncthreads();
    smooth<DIM, VAR, C>(F, tmp, c, a.smoother, omega, a.nu2);
  }
  __syncthreads();
}

template <int DIM, bool VAR, typename C>
__global__ void __launch_bounds__(kThreads) k_coarse_cycle(CoarseArgs a) {
  coarse_cycle_body<DIM, VAR, C>(a);
}

// One block per problem: the coarse cycles of a batch of independent problems.
template <int DIM, bool VAR, typename C>
__global__ void __launch_bounds__(kThreads) k_coarse_cycle_batched(const CoarseArgs *__restrict__ list) {
  if (list[blockIdx.x].live && !*list[blockIdx.x].live) return;
  coarse_cycle_body<DIM, VAR, C>(list[blockIdx.x]);
}

}  // namespace cz
}  // namespace mg
