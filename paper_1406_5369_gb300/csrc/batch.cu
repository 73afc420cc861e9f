// Batched multigrid over many independent problems (mg_batch_* in mg.h).
//
// A batch step runs one solve step (a V-cycle, or a defect-correction step:
// inner_cycles inner V-cycles and the FP64 outer update + residual) for every
// listed problem. Work is grouped by absolute level size across problems:
// each fine level size is one launch per operator over all problems that
// have a level of that size, the levels below the coarse threshold of every
// problem run in one launch of the single-block coarse cycle (one block per
// problem), and the outer step and the norms run once over all problems.
// Kernels read per-problem descriptors from device arrays; each problem's
// arithmetic (and the order of its norm sums) is the same whatever else is
// in the batch, so a problem's result does not depend on its companions.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <new>
#include <map>
#include <unordered_map>
#include <vector>

#include "ctx.h"
#include "kernels.cuh"
#include "outer2d.cuh"
#include "stencil3d.cuh"

namespace mg {
namespace bz {

constexpr int kPartBlocks = 128;   // blocks (one partial sum each) of the generic norm kernels per problem
constexpr int kSlots = 1024;       // partial-sum slots per problem (the streaming kernels write up to this many)

// One level of one problem. The stencil is stored in both compute types,
// converted on the host: FP64 -> FP32 conversions run on the slow FP64 pipe
// of this GPU, so kernels must not redo them per thread.
struct BOp {
  void *u[2];
  void *f;
  void *r;
  Sten<double> sd;
  Sten<float> sf;
  Geo g;
  int cur;  // live solution buffer at the start of the step
  const int *live;  // captured steps: the problem's live flag (NULL = always live)
};

// Fine/coarse pair of one problem (restriction: fine r -> coarse f;
// interpolation: coarse u -> fine u).
struct BXfer {
  const void *src;
  void *dst;
  Geo gf, gc;
  const int *live;
};

// Outer (FP64) finest level and inner level 0 of one problem.
struct BOuter {
  double *u;
  const double *f;
  Sten<double> sd;
  Geo go;
  void *d;        // inner defect (inner f)
  const void *e;  // inner correction (live inner u)
  Geo gi;
  double *partials;  // this problem's partial-sum slots
  const int *live;
};

// A block of a captured batch step whose problem has converged does nothing.
template <typename R> __device__ __forceinline__ bool gone(const R &r) { return r.live && !*r.live; }

template <typename C> __device__ __forceinline__ const Sten<C> &sten_of_op(const BOp &o);
template <> __device__ __forceinline__ const Sten<double> &sten_of_op<double>(const BOp &o) { return o.sd; }
template <> __device__ __forceinline__ const Sten<float> &sten_of_op<float>(const BOp &o) { return o.sf; }

// Generic kernels: a block owns one row (blockIdx.x) of one plane (3D:
// blockIdx.y) of one problem (blockIdx.y in 2D, blockIdx.z in 3D) and its
// threads loop over the columns, so a launch has one block per row and
// problem, not one per 128 nodes. `first` is the index of the first row and
// plane covered (1 when only interior rows/planes are launched).
template <int DIM> struct BRow {
  int j, k, pi;
  long long off;  // element offset of the row
};
template <int DIM> __device__ __forceinline__ BRow<DIM> brow(const Geo &g, int first) {
  BRow<DIM> r;
  r.j = first + (int)blockIdx.x;
  r.k = DIM == 3 ? first + (int)blockIdx.y : 0;
  r.pi = DIM == 3 ? (int)blockIdx.z : (int)blockIdx.y;
  r.off = (long long)r.k * g.sz + (long long)r.j * g.sy;
  return r;
}

template <int DIM, typename T, bool VAR>
__global__ void kb_rbgs_half(const BOp *__restrict__ ops, Geo g, int color, int flip, double omega_d, float omega_f) {
  typedef typename CT<T>::type C;
  BRow<DIM> r = brow<DIM>(g, 1);
  const BOp &o = ops[r.pi];
  if (gone(o)) return;
  T *u = (T *)o.u[o.cur ^ flip];
  const T *f = (const T *)o.f;
  const Sten<C> s = sten_of_op<C>(o);
  const C omega = pick<C>(omega_d, omega_f);
  // columns i with (i + j + k) % 2 == color, from the first interior one
  const int i0 = 1 + ((color + r.j + r.k + 1) & 1);
  for (int i = i0 + 2 * (int)threadIdx.x; i <= g.n - 2; i += 2 * (int)blockDim.x) {
    const long long p = r.off + i;
    C Au, dg;
    apply_at<DIM, VAR>(u, p, g, s, Au, dg);
    st(u + p, ld(u + p) + omega * (ld(f + p) - Au) / dg);
  }
}

template <int DIM, typename T, bool VAR>
__global__ void kb_jacobi(const BOp *__restrict__ ops, Geo g, int flip, double omega_d, float omega_f) {
  typedef typename CT<T>::type C;
  BRow<DIM> r = brow<DIM>(g, 1);
  const BOp &o = ops[r.pi];
  if (gone(o)) return;
  const T *uin = (const T *)o.u[o.cur ^ flip];
  T *uout = (T *)o.u[o.cur ^ flip ^ 1];
  const T *f = (const T *)o.f;
  const Sten<C> s = sten_of_op<C>(o);
  const C omega = pick<C>(omega_d, omega_f);
  for (int i = 1 + (int)threadIdx.x; i <= g.n - 2; i += (int)blockDim.x) {
    const long long p = r.off + i;
    C Au, dg;
    apply_at<DIM, VAR>(uin, p, g, s, Au, dg);
    st(uout + p, ld(uin + p) + omega * (ld(f + p) - Au) / dg);
  }
}

template <int DIM, typename T, bool VAR>
__global__ void kb_residual(const BOp *__restrict__ ops, Geo g, int flip) {
  typedef typename CT<T>::type C;
  BRow<DIM> r = brow<DIM>(g, 1);
  const BOp &o = ops[r.pi];
  if (gone(o)) return;
  const T *u = (const T *)o.u[o.cur ^ flip];
  const T *f = (const T *)o.f;
  T *res = (T *)o.r;
  const Sten<C> s = sten_of_op<C>(o);
  for (int i = 1 + (int)threadIdx.x; i <= g.n - 2; i += (int)blockDim.x) {
    const long long p = r.off + i;
    C Au, dg;
    apply_at<DIM, VAR>(u, p, g, s, Au, dg);
    st(res + p, ld(f + p) - Au);
  }
}

// Zeroes every row (boundary included) of the live solution.
template <int DIM, typename T> __global__ void kb_zero(const BOp *__restrict__ ops, Geo g, int flip) {
  BRow<DIM> r = brow<DIM>(g, 0);
  const BOp &o = ops[r.pi];
  if (gone(o)) return;
  T *u = (T *)o.u[o.cur ^ flip] + r.off;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) st(u + i, 0.0f);
}

// Full weighting: rows/planes of the coarse grid.
template <int DIM, typename Tf, typename Tc>
__global__ void kb_restrict(const BXfer *__restrict__ xs, Geo gf, Geo gc) {
  typedef typename CT<Tc>::type C;
  BRow<DIM> r = brow<DIM>(gc, 1);
  if (gone(xs[r.pi])) return;
  const Tf *rf = (const Tf *)xs[r.pi].src;
  Tc *fc = (Tc *)xs[r.pi].dst;
  const long long qrow = (long long)(2 * r.k) * gf.sz + (long long)(2 * r.j) * gf.sy;
  for (int I = 1 + (int)threadIdx.x; I <= gc.n - 2; I += (int)blockDim.x) {
    const long long q = qrow + 2 * I;
    C acc = 0;
#pragma unroll
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++) {
      C wz = DIM == 3 ? (dz == 0 ? (C)0.5 : (C)0.25) : (C)1;
#pragma unroll
      for (int dy = -1; dy <= 1; dy++) {
        C wy = dy == 0 ? (C)0.5 : (C)0.25;
        const Tf *row = rf + q + dz * gf.sz + dy * gf.sy;
        C line = (C)0.25 * ((C)ld(row - 1) + (C)ld(row + 1)) + (C)0.5 * (C)ld(row);
        acc += wz * wy * line;
      }
    }
    st(fc + r.off + I, acc);
  }
}

// Interpolation and correction: rows/planes of the fine grid.
template <int DIM, typename Tc, typename Tf>
__global__ void kb_prolong(const BXfer *__restrict__ xs, Geo gc, Geo gf) {
  typedef typename CT<Tf>::type C;
  BRow<DIM> r = brow<DIM>(gf, 1);
  if (gone(xs[r.pi])) return;
  const Tc *ec = (const Tc *)xs[r.pi].src;
  Tf *uf = (Tf *)xs[r.pi].dst;
  const int J = r.j >> 1, K = r.k >> 1, oj = r.j & 1, ok = DIM == 3 ? (r.k & 1) : 0;
  const C w = (oj ? (C)0.5 : (C)1) * (ok ? (C)0.5 : (C)1);
  for (int i = 1 + (int)threadIdx.x; i <= gf.n - 2; i += (int)blockDim.x) {
    const int I = i >> 1, oi = i & 1;
    C acc = 0;
    for (int a = 0; a <= ok; a++)
      for (int b = 0; b <= oj; b++) {
        const Tc *row = ec + (long long)(K + a) * gc.sz + (long long)(J + b) * gc.sy + I;
        acc += oi ? (C)0.5 * ((C)ld(row) + (C)ld(row + 1)) : (C)ld(row);
      }
    const long long p = r.off + i;
    st(uf + p, (C)ld(uf + p) + w * acc);
  }
}

// Per-problem partial sums of the FP64 outer residual squared (kPartBlocks
// blocks per problem, fixed partition), writing the inner defect.
template <int DIM, typename Ti, bool VAR>
__global__ void kb_dc_residual(const BOuter *__restrict__ os) {
  const BOuter &o = os[blockIdx.y];
  if (gone(o)) return;
  const Sten<double> s = o.sd;
  double acc = 0.0;
  for_interior_rows<DIM>(o.go.n - 2, o.go, o.gi, [&](long long p, long long q) {
    double Au, dg;
    apply_at<DIM, VAR>(o.u, p, o.go, s, Au, dg);
    double r = o.f[p] - Au;
    acc += r * r;
    if (o.d) st((Ti *)o.d + q, oz::d2f_bits(r));  // truncation to FP32 without the FP64 pipe
  });
  acc = block_sum(acc);
  if (threadIdx.x == 0) o.partials[blockIdx.x] = acc;
}

template <int DIM, typename Ti>
__global__ void kb_dc_update(const BOuter *__restrict__ os) {
  const BOuter &o = os[blockIdx.y];
  if (gone(o)) return;
  for_interior_rows<DIM>(o.go.n - 2, o.go, o.gi,
                         [&](long long p, long long q) { o.u[p] += oz::f2d_bits(ld((const Ti *)o.e + q)); });
}

// Norm partials of level 0 for plain FP64 problems.
template <int DIM, bool VAR>
__global__ void kb_norm(const BOp *__restrict__ ops, double *__restrict__ partials) {
  const BOp &o = ops[blockIdx.y];
  if (gone(o)) return;
  const Sten<double> s = o.sd;
  const double *u = (const double *)o.u[o.cur];
  const double *f = (const double *)o.f;
  double acc = 0.0;
  for_interior_rows<DIM>(o.g.n - 2, o.g, o.g, [&](long long p, long long) {
    double Au, dg;
    apply_at<DIM, VAR>(u, p, o.g, s, Au, dg);
    double r = f[p] - Au;
    acc += r * r;
  });
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[(long long)blockIdx.y * kSlots + blockIdx.x] = acc;
}

// One block per problem: fixed-order sum of its kSlots partial slots
// (unused slots hold zero), norm out.
__global__ void kb_finalize(const double *__restrict__ partials, double *__restrict__ norms) {
  __shared__ double buf[256];
  int t = threadIdx.x;
  const double *p = partials + (long long)blockIdx.x * kSlots;
  double a = 0.0;
  for (int i = t; i < kSlots; i += 256) a += p[i];
  buf[t] = a;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) buf[t] += buf[t + s];
    __syncthreads();
  }
  if (t == 0) norms[blockIdx.x] = sqrt(buf[0]);
}

// Stopping test of a captured batch step (one block): for every problem
// still live, count the step, form rho = ||r|| / ||r_0|| and retire it when
// rho <= tol, rho is not finite or maxit steps are done; *remaining = the
// problems still live. Retired problems' kernels skip them from then on.
__global__ void kb_check(const double *__restrict__ norms, const double *__restrict__ r0,
                         const double *__restrict__ tol, int *__restrict__ live, int *__restrict__ iters,
                         double *__restrict__ rho, int count, int maxit, int *__restrict__ remaining) {
  __shared__ int left;
  if (threadIdx.x == 0) left = 0;
  __syncthreads();
  int mine = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    if (!live[i]) continue;
    const int it = iters[i] + 1;
    iters[i] = it;
    const double a = r0[i];
    const double r = a > 0.0 ? norms[i] / a : (a == 0.0 ? 0.0 : (double)NAN);
    rho[i] = r;
    const int go = (r > tol[i]) && it < maxit;  // a NaN rho fails the comparison and retires
    live[i] = go;
    mine += go;
  }
  atomicAdd(&left, mine);
  __syncthreads();
  if (threadIdx.x == 0) *remaining = left;
}

// Start of a captured solve: every listed problem live, no steps, rho = 1.
__global__ void kb_arm(int *__restrict__ live, int *__restrict__ iters, double *__restrict__ rho, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    live[i] = 1;
    iters[i] = 0;
    rho[i] = 1.0;
  }
}

}  // namespace bz
}  // namespace mg

using namespace mg;
using namespace mg::bz;

namespace {

thread_local char g_berr[256];

mg_status bfail(mg_status st, const char *msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess) snprintf(g_berr, sizeof g_berr, "%s: %s", msg, cudaGetErrorString(e));
  else snprintf(g_berr, sizeof g_berr, "%s", msg);
  set_error_message(g_berr);
  return st;
}

#define BCK(msg, call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return bfail(MG_ECUDA, msg, e_); \
  } while (0)

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct mg_batch {
  int maxp;
  std::vector<mg_ctx *> probs;  // by id; nullptr when free
  std::vector<double> r0;       // initial residual norm per id (< 0: not yet computed)
  char *ws;
  size_t ws_bytes;
  size_t desc_bytes;            // descriptor area at the start of ws
  double *partials;             // maxp * kSlots
  double *norms;                // maxp
  cudaStream_t stream;
  bool have_opts;
  mg_options opt;
  int list_rows;  // rows per chunk of the fused 2D list launches (0 = 256), mg_batch_set_tile_rows
  int dim;
  bool dc, fp64;
  // descriptors: staged in pinned host memory, copied right before the
  // launch that reads them (stream order), reset after each step's sync
  char *pinned;
  size_t dev_off;
  unsigned long long launches;
  // Captured solve (mg_batch_solve): per-position device state of the
  // problems being solved, the descriptor area of the two captured steps and
  // a private stream to capture on.
  int capture;                 // 1: mg_batch_solve replays captured steps
  int *live;                   // maxp flags: problem still stepping
  int *iters_dev;              // maxp steps taken
  double *rho_dev, *r0_dev, *tol_dev;  // maxp each
  int *remaining;              // problems still live after the last check
  char *gdesc;                 // descriptor area of the captured steps (device)
  size_t gdesc_bytes, goff;
  bool gmode;                  // push() stages into gstage for one upload after capture
  std::vector<char> gstage;
  std::unordered_map<const mg_ctx *, int> pos;  // position of each problem in the captured solve
  cudaStream_t cap;
  char *hstage;                // pinned: r0 and tol uploads, remaining-counter reads
  cudaEvent_t ev[2];
  double phase_ms[5];          // last mg_batch_solve: host wall time of its phases
  // a step in flight (mg_batch_step_async): its problems, the fresh ones,
  // the pinned copies of their norms and the event that completes them
  bool step_pending;
  std::vector<int> step_ids, step_fresh;
  double *hstep;               // pinned: maxp step norms, then maxp initial norms
  cudaEvent_t step_ev, add_ev;
  // kernel timing (mg_batch_set_timing): event pairs around launch groups
  // of uncaptured steps, harvested at the step's synchronisation
  int timing;
  struct Pending { cudaEvent_t a, e; int kind; double bytes; };
  std::vector<Pending> tpend;
  std::vector<cudaEvent_t> tpool;
  double t_ms[8], t_bytes[8];
  unsigned long long t_n[8];
};

namespace {

size_t desc_area_bytes(int maxp) {
  // Room for about one V-cycle's records of every problem (12 levels, a few
  // records per level, the coarse record and the outer records); when a step
  // needs more, push() waits for the queued kernels and reuses the area.
  size_t rec = std::max(std::max(sizeof(BOp), sizeof(fz::Args2D)), std::max(sizeof(z3::Args3), sizeof(z3::ArgsDC3)));
  size_t per = (size_t)12 * 6 * rec + coarse_args_bytes() + 2 * sizeof(BOuter) + 1024;
  return align256((size_t)maxp * per);
}

// Device bytes of the captured steps' descriptors per problem: two solve
// steps of up to four inner V-cycles over ten fine levels, the coarse-cycle
// and outer records (a solve whose records need more runs uncaptured).
constexpr size_t kGraphDescPerProblem = 48 * 1024;

size_t graph_area_bytes(int maxp) { return align256((size_t)maxp * kGraphDescPerProblem); }

// Device state of a captured solve: live flags, step counts, rho, r0, tol
// (one each per problem) and the remaining-problems counter.
size_t solve_state_bytes(int maxp) {
  return 2 * align256(sizeof(int) * (size_t)maxp) + 3 * align256(sizeof(double) * (size_t)maxp) + 256;
}

// Stages `bytes` of descriptors and copies them to the next device slot on
// the batch stream (before any kernel launched after this call); returns
// the device address, NULL if the area is exhausted or the copy failed.
// While a solve step is being captured (gmode) the records go to a host
// buffer instead, uploaded once to the captured steps' own area.
void *push(mg_batch *b, const void *src, size_t bytes) {
  if (b->gmode) {
    size_t off = align256(b->goff);
    if (off + bytes > b->gdesc_bytes) return nullptr;
    if (b->gstage.size() < off + bytes) b->gstage.resize(off + bytes);
    memcpy(b->gstage.data() + off, src, bytes);
    b->goff = off + bytes;
    return b->gdesc + off;
  }
  size_t off = align256(b->dev_off);
  if (bytes > b->desc_bytes) return nullptr;
  if (off + bytes > b->desc_bytes) {
    // area full: once the kernels queued so far have read their
    // descriptors, the whole area (and its pinned staging) is free again
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return nullptr;
    off = 0;
  }
  memcpy(b->pinned + off, src, bytes);
  if (cudaMemcpyAsync(b->ws + off, b->pinned + off, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return nullptr;
  b->dev_off = off + bytes;
  return b->ws + off;
}

// Times the launches issued during its lifetime (one launch group of one
// kernel kind) with a pair of events on the batch stream, when timing is on
// and the step is not being captured; `bytes` = the group's algorithmic
// bytes (compulsory traffic of the kernels' operator model).
struct BTimer {
  mg_batch *b;
  int kind;
  double bytes;
  cudaEvent_t a = nullptr;
  static cudaEvent_t take(mg_batch *b) {
    if (!b->tpool.empty()) {
      cudaEvent_t e = b->tpool.back();
      b->tpool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
  }
  BTimer(mg_batch *b_, int kind_, double bytes_) : b(b_), kind(kind_), bytes(bytes_) {
    if (b->timing && !b->gmode && (a = take(b))) cudaEventRecord(a, b->stream);
  }
  ~BTimer() {
    if (!a) return;
    cudaEvent_t e = take(b);
    if (!e) {
      b->tpool.push_back(a);
      return;
    }
    cudaEventRecord(e, b->stream);
    b->tpend.push_back({a, e, kind, bytes});
  }
};

// Adds the finished event pairs to the totals (after a synchronisation).
void harvest(mg_batch *b) {
  for (auto &p : b->tpend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.e) == cudaSuccess) {
      b->t_ms[p.kind] += ms;
      b->t_bytes[p.kind] += p.bytes;
      b->t_n[p.kind]++;
    }
    b->tpool.push_back(p.a);
    b->tpool.push_back(p.e);
  }
  b->tpend.clear();
}

// Nodes of a level (boundary included) and its word size.
double nodes_of(const Level &L) { return (double)L.n * L.n * (L.dim == 3 ? L.n : 1); }

// The live flag a record of problem c points at: its slot while a solve is
// captured, NULL (always live) otherwise.
const int *live_of(const mg_batch *b, const mg_ctx *c) {
  if (!b->gmode) return nullptr;
  auto it = b->pos.find(c);
  return it == b->pos.end() ? nullptr : b->live + it->second;
}

template <typename D> struct Group {
  int n = 0;
  std::vector<D> items;
};

// One block per row (and plane) of one problem: interior rows/planes only
// (`all` = every row and plane, for zeroing).
dim3 bgrid(int dim, int n, int count, bool all = false) {
  unsigned rows = (unsigned)(all ? n : n - 2);
  return dim3(rows, dim == 3 ? rows : (unsigned)count, dim == 3 ? (unsigned)count : 1u);
}
unsigned bthreads(int n) { return n > 129 ? 256u : 128u; }

int chunk_of(int, int) { return 65535; }

BOp make_op(const Level &L) {
  BOp o;
  memset(&o, 0, sizeof o);
  o.u[0] = L.u[0];
  o.u[1] = L.u[1];
  o.f = L.f;
  o.r = L.r;
  o.sd = sten_of<double>(L);
  o.sf = sten_of<float>(L);
  o.g = geo_of(L);
  o.cur = L.cur;
  return o;
}

// ----- launch helpers: dispatch on dim / storage type / variable stencil

#define DISPATCH_T(dtype, ...)                         \
  switch (dtype) {                                     \
    case F64: { typedef double T; __VA_ARGS__; } break; \
    case F32: { typedef float T; __VA_ARGS__; } break;  \
    default: { typedef bf16 T; __VA_ARGS__; } break;    \
  }

}  // namespace

// The batched operator launches need each op's geometry; groups share n and
// storage type, hence pitch and plane, so the group's first op supplies it.
namespace {

cudaError_t launch_group_op(int what, const std::vector<BOp> &items, mg_batch *b, int dim, int dtype, bool var,
                            int color, int flip, double omega) {
  if (items.empty()) return cudaSuccess;
  Geo g = items[0].g;
  int n = g.n;
  int chunk = chunk_of(dim, n);
  for (size_t base = 0; base < items.size(); base += chunk) {
    int count = (int)std::min<size_t>(chunk, items.size() - base);
    const BOp *dev = (const BOp *)push(b, items.data() + base, sizeof(BOp) * count);
    if (!dev) return cudaErrorMemoryAllocation;
    dim3 blk(bthreads(n)), gr = bgrid(dim, n, count, what == 3);
    cudaStream_t s = b->stream;
#define OPK(K, ...)                                                                       \
  if (dim == 2) {                                                                         \
    DISPATCH_T(dtype, if (var) K<2, T, true><<<gr, blk, 0, s>>>(__VA_ARGS__);             \
               else K<2, T, false><<<gr, blk, 0, s>>>(__VA_ARGS__));                      \
  } else {                                                                                \
    DISPATCH_T(dtype, if (var) K<3, T, true><<<gr, blk, 0, s>>>(__VA_ARGS__);             \
               else K<3, T, false><<<gr, blk, 0, s>>>(__VA_ARGS__));                      \
  }
    if (what == 0) { OPK(kb_rbgs_half, dev, g, color, flip, omega, (float)omega) }
    else if (what == 1) { OPK(kb_jacobi, dev, g, flip, omega, (float)omega) }
    else if (what == 2) { OPK(kb_residual, dev, g, flip) }
    else {
      if (dim == 2) { DISPATCH_T(dtype, kb_zero<2, T><<<gr, blk, 0, s>>>(dev, g, flip)) }
      else { DISPATCH_T(dtype, kb_zero<3, T><<<gr, blk, 0, s>>>(dev, g, flip)) }
    }
#undef OPK
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    b->launches++;
  }
  return cudaSuccess;
}

cudaError_t launch_group_xfer(bool restrict_, const std::vector<BXfer> &items, mg_batch *b, int dim, int tf, int tc) {
  if (items.empty()) return cudaSuccess;
  Geo gf = items[0].gf, gc = items[0].gc;
  int n = restrict_ ? gc.n : gf.n;  // grid of the written level
  int chunk = chunk_of(dim, n);
  for (size_t base = 0; base < items.size(); base += chunk) {
    int count = (int)std::min<size_t>(chunk, items.size() - base);
    const BXfer *dev = (const BXfer *)push(b, items.data() + base, sizeof(BXfer) * count);
    if (!dev) return cudaErrorMemoryAllocation;
    dim3 blk(bthreads(n)), gr = bgrid(dim, n, count);
    cudaStream_t s = b->stream;
    // (fine type, coarse type): (T,T) or (T, double) for the FP64 coarsest
    if (restrict_) {
      if (dim == 2) {
        if (tc == F64 && tf != F64) { DISPATCH_T(tf, kb_restrict<2, T, double><<<gr, blk, 0, s>>>(dev, gf, gc)) }
        else { DISPATCH_T(tf, kb_restrict<2, T, T><<<gr, blk, 0, s>>>(dev, gf, gc)) }
      } else {
        if (tc == F64 && tf != F64) { DISPATCH_T(tf, kb_restrict<3, T, double><<<gr, blk, 0, s>>>(dev, gf, gc)) }
        else { DISPATCH_T(tf, kb_restrict<3, T, T><<<gr, blk, 0, s>>>(dev, gf, gc)) }
      }
    } else {
      if (dim == 2) {
        if (tc == F64 && tf != F64) { DISPATCH_T(tf, kb_prolong<2, double, T><<<gr, blk, 0, s>>>(dev, gc, gf)) }
        else { DISPATCH_T(tf, kb_prolong<2, T, T><<<gr, blk, 0, s>>>(dev, gc, gf)) }
      } else {
        if (tc == F64 && tf != F64) { DISPATCH_T(tf, kb_prolong<3, double, T><<<gr, blk, 0, s>>>(dev, gc, gf)) }
        else { DISPATCH_T(tf, kb_prolong<3, T, T><<<gr, blk, 0, s>>>(dev, gc, gf)) }
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    b->launches++;
  }
  return cudaSuccess;
}

#define BLAUNCH(msg, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return bfail(MG_ECUDA, msg, e_);  \
  } while (0)

// One (problem, level) entry of a level-size group. `fast` is decided from
// the problem alone (its stencil, smoother, storage type and sizes), so a
// problem runs the same kernels - and gets the same result - whatever else
// is in the batch. `flip` counts the live-buffer swaps in this cycle.
struct Item {
  mg_ctx *c;
  int l;
  bool fast;
  int flip;
};

bool fast_level(const mg_ctx *c, int l) {
  const Level &L = c->lv[l], &C = c->lv[l + 1];
  const mg_options &o = c->opt;
  if (!o.fuse) return false;
  if (L.dim == 2) return o.smoother == MG_RBGS && d2::fused_ok(L, C, o.nu1) && d2::fused_ok(L, C, o.nu2);
  return d3::z_ok(L) && d3::transfer_ok(L, C);
}

template <typename R> const R *push_list(mg_batch *b, const std::vector<R> &v) {
  return (const R *)push(b, v.data(), sizeof(R) * v.size());
}

// Streaming / fused kernels of the fast items of one group: pre-smoothing,
// residual and restriction (descend) or interpolation and post-smoothing.
mg_status fast_descend(mg_batch *b, std::vector<Item *> &F, bool zero0) {
  if (F.empty()) return MG_OK;
  const mg_options &o = b->opt;
  const Level &L0 = F[0]->c->lv[F[0]->l], &C0 = F[0]->c->lv[F[0]->l + 1];
  cudaStream_t s = b->stream;
  if (L0.dim == 2) {
    for (int zero = 0; zero <= 1; zero++) {
      std::vector<fz::Args2D> recs;
      for (Item *it : F) {
        bool z = it->l > 0 || zero0;
        if (z != (zero != 0)) continue;
        Level &L = it->c->lv[it->l], &C = it->c->lv[it->l + 1];
        recs.push_back(d2::fused_record(L, C, o.omega, L.u[L.cur ^ it->flip], L.u[L.cur ^ it->flip ^ 1], nullptr, C.f));
        recs.back().live = live_of(b, it->c);
      }
      if (recs.empty()) continue;
      const fz::Args2D *dev = push_list(b, recs);
      if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
      // read f (and u), write u and the coarse f; faces (FP32) when variable
      const double w = dtype_size(L0.dtype);
      BTimer tm(b, MG_BATCH_PRE, recs.size() * nodes_of(L0) * ((zero ? 2.25 : 3.25) * w + (L0.kf[0] ? 8.0 : 0.0)));
      BLAUNCH("batched fused pre-smoothing",
              d2::pre_fused_list(L0, C0, dev, (int)recs.size(), zero != 0, o.nu1, b->list_rows, s));
      b->launches++;
    }
    for (Item *it : F) it->flip ^= 1;
    return MG_OK;
  }
  // 3D: levels that start from zero take their first two Jacobi sweeps in one
  // pass that reads f only (kJZ); otherwise they are zeroed first. Then the
  // (remaining) sweeps, residual, restriction.
  const bool jz = o.smoother == MG_JACOBI && o.nu1 >= 2;
  // operator model: nu1 sweeps of 3 words (2 for the f-only first pair),
  // residual 3 words, full weighting 1 + 1/8 words per fine node
  BTimer tm(b, MG_BATCH_PRE, F.size() * nodes_of(L0) * dtype_size(L0.dtype) * (3.0 * o.nu1 + 3.0 + 1.125 - (jz ? 4.0 : 0.0)));
  std::vector<Item *> Zs, Ns;
  for (Item *it : F) ((it->l > 0 || zero0) ? Zs : Ns).push_back(it);
  if (jz && !Zs.empty()) {
    std::vector<z3::Args3> recs;
    for (Item *it : Zs) {
      Level &L = it->c->lv[it->l];
      recs.push_back(d3::stencil_record(L, o.omega, L.f, L.u[L.cur ^ it->flip ^ 1], L.f));
      recs.back().live = live_of(b, it->c);
    }
    const z3::Args3 *dev = push_list(b, recs);
    if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
    BLAUNCH("batched 3D Jacobi from zero", d3::z_jacobi_zero2_list(L0, dev, (int)recs.size(), s));
    b->launches++;
    for (Item *it : Zs) it->flip ^= 1;
  } else {
    std::vector<BOp> zops;
    for (Item *it : Zs) {
      BOp op = make_op(it->c->lv[it->l]);
      op.cur ^= it->flip;
      op.live = live_of(b, it->c);
      zops.push_back(op);
    }
    if (!zops.empty()) BLAUNCH("batched zero", launch_group_op(3, zops, b, 3, L0.dtype, false, 0, 0, 0.0));
  }
  auto sweeps = [&](std::vector<Item *> &F, int nu) -> mg_status {
    for (int k = 0; k < nu; k++) {
      if (F.empty()) break;
      std::vector<z3::Args3> recs;
      for (Item *it : F) {
        Level &L = it->c->lv[it->l];
        void *in = L.u[L.cur ^ it->flip];
        recs.push_back(d3::stencil_record(L, o.omega, in, o.smoother == MG_RBGS ? in : L.u[L.cur ^ it->flip ^ 1], L.f));
        recs.back().live = live_of(b, it->c);
      }
      const z3::Args3 *dev = push_list(b, recs);
      if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
      if (o.smoother == MG_RBGS) {
        BLAUNCH("batched 3D RBGS", d3::z_sweep_list(L0, dev, (int)recs.size(), 0, s));
        BLAUNCH("batched 3D RBGS", d3::z_sweep_list(L0, dev, (int)recs.size(), 1, s));
        b->launches += 2;
      } else {
        BLAUNCH("batched 3D Jacobi", d3::z_sweep_list(L0, dev, (int)recs.size(), -1, s));
        b->launches++;
        for (Item *it : F) it->flip ^= 1;
      }
    }
    return MG_OK;
  };
  mg_status st;
  if (jz) {
    if ((st = sweeps(Zs, o.nu1 - 2))) return st;
    if ((st = sweeps(Ns, o.nu1))) return st;
  } else {
    if ((st = sweeps(F, o.nu1))) return st;
  }
  std::vector<z3::Args3> rrec;
  std::vector<z3::ArgsT3> xrec;
  for (Item *it : F) {
    Level &L = it->c->lv[it->l], &C = it->c->lv[it->l + 1];
    rrec.push_back(d3::stencil_record(L, o.omega, L.u[L.cur ^ it->flip], L.r, L.f));
    rrec.back().live = live_of(b, it->c);
    z3::ArgsT3 x;
    memset(&x, 0, sizeof x);
    x.src = L.r;
    x.dst = C.f;
    x.live = live_of(b, it->c);
    xrec.push_back(x);
  }
  const z3::Args3 *dr = push_list(b, rrec);
  if (!dr) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
  BLAUNCH("batched 3D residual", d3::z_residual_list(L0, dr, (int)rrec.size(), s));
  const z3::ArgsT3 *dx = push_list(b, xrec);
  if (!dx) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
  BLAUNCH("batched 3D restriction", d3::z_transfer_list(true, L0, C0, dx, (int)xrec.size(), s));
  b->launches += 2;
  return MG_OK;
}

mg_status fast_ascend(mg_batch *b, std::vector<Item *> &F, const std::function<int(mg_ctx *, int)> &flip_of) {
  if (F.empty()) return MG_OK;
  const mg_options &o = b->opt;
  const Level &L0 = F[0]->c->lv[F[0]->l], &C0 = F[0]->c->lv[F[0]->l + 1];
  cudaStream_t s = b->stream;
  if (L0.dim == 2) {
    std::vector<fz::Args2D> recs;
    for (Item *it : F) {
      Level &L = it->c->lv[it->l], &C = it->c->lv[it->l + 1];
      const void *ec = C.u[C.cur ^ flip_of(it->c, it->l + 1)];
      recs.push_back(d2::fused_record(L, C, o.omega, L.u[L.cur ^ it->flip], L.u[L.cur ^ it->flip ^ 1], ec, nullptr));
      recs.back().live = live_of(b, it->c);
    }
    const fz::Args2D *dev = push_list(b, recs);
    if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
    // read u, f and the coarse e, write u; faces (FP32) when variable
    BTimer tm(b, MG_BATCH_POST, recs.size() * nodes_of(L0) * (3.25 * dtype_size(L0.dtype) + (L0.kf[0] ? 8.0 : 0.0)));
    BLAUNCH("batched fused post-smoothing", d2::post_fused_list(L0, C0, dev, (int)recs.size(), o.nu2, b->list_rows, s));
    b->launches++;
    for (Item *it : F) it->flip ^= 1;
    return MG_OK;
  }
  // operator model: trilinear correction 2 + 1/8 words, nu2 sweeps of 3 words
  BTimer tm(b, MG_BATCH_POST, F.size() * nodes_of(L0) * dtype_size(L0.dtype) * (2.125 + 3.0 * o.nu2));
  std::vector<z3::ArgsT3> xrec;
  for (Item *it : F) {
    Level &L = it->c->lv[it->l], &C = it->c->lv[it->l + 1];
    z3::ArgsT3 x;
    memset(&x, 0, sizeof x);
    x.src = C.u[C.cur ^ flip_of(it->c, it->l + 1)];
    x.dst = L.u[L.cur ^ it->flip];
    x.live = live_of(b, it->c);
    xrec.push_back(x);
  }
  const z3::ArgsT3 *dx = push_list(b, xrec);
  if (!dx) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
  BLAUNCH("batched 3D interpolation", d3::z_transfer_list(false, L0, C0, dx, (int)xrec.size(), s));
  b->launches++;
  for (int k = 0; k < o.nu2; k++) {
    std::vector<z3::Args3> recs;
    for (Item *it : F) {
      Level &L = it->c->lv[it->l];
      void *in = L.u[L.cur ^ it->flip];
      recs.push_back(d3::stencil_record(L, o.omega, in, o.smoother == MG_RBGS ? in : L.u[L.cur ^ it->flip ^ 1], L.f));
      recs.back().live = live_of(b, it->c);
    }
    const z3::Args3 *dev = push_list(b, recs);
    if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
    if (o.smoother == MG_RBGS) {
      BLAUNCH("batched 3D RBGS", d3::z_sweep_list(L0, dev, (int)recs.size(), 0, s));
      BLAUNCH("batched 3D RBGS", d3::z_sweep_list(L0, dev, (int)recs.size(), 1, s));
      b->launches += 2;
    } else {
      BLAUNCH("batched 3D Jacobi", d3::z_sweep_list(L0, dev, (int)recs.size(), -1, s));
      b->launches++;
      for (Item *it : F) it->flip ^= 1;
    }
  }
  return MG_OK;
}

// One V-cycle of every problem in `ps` (levels grouped by size). zero0:
// level 0 starts from zero (first inner cycle of a defect-correction step).
mg_status batched_vcycle(mg_batch *b, const std::vector<mg_ctx *> &ps, bool zero0) {
  const int dim = b->dim;
  const int top_n = coarse_top_n(dim, b->fp64);
  const mg_options &o = b->opt;
  // level size -> items, for every fine level size (above the coarse threshold)
  std::map<int, std::vector<Item>, std::greater<int>> fine;
  for (mg_ctx *c : ps)
    for (int l = 0; l < c->nl; l++)
      if (c->lv[l].n > top_n) fine[c->lv[l].n].push_back({c, l, fast_level(c, l), 0});
  std::map<std::pair<const mg_ctx *, int>, const Item *> where;
  for (auto &kv : fine)
    for (const Item &it : kv.second) where[{it.c, it.l}] = &it;
  auto flip_of = [&](mg_ctx *c, int l) {
    auto f = where.find({c, l});
    return f == where.end() ? 0 : f->second->flip;
  };
  // generic (one thread per node) kernels for the items that are not fast
  auto ops_of = [&](const std::vector<Item *> &v, bool only_zero) {
    std::vector<BOp> out;
    for (Item *it : v) {
      bool z = it->l > 0 || zero0;
      if (only_zero && !z) continue;
      out.push_back(make_op(it->c->lv[it->l]));
      out.back().live = live_of(b, it->c);
    }
    return out;
  };
  auto smooth = [&](std::vector<Item *> &v, int sweeps) -> mg_status {
    if (v.empty()) return MG_OK;
    std::vector<BOp> ops = ops_of(v, false);
    const Level &L0 = v[0]->c->lv[v[0]->l];
    bool var = L0.kf[0] != nullptr;
    for (int k = 0; k < sweeps; k++) {
      int flip = v[0]->flip;  // equal across the generic items of a group
      if (o.smoother == MG_RBGS) {
        BLAUNCH("batched RBGS", launch_group_op(0, ops, b, dim, L0.dtype, var, 0, flip, o.omega));
        BLAUNCH("batched RBGS", launch_group_op(0, ops, b, dim, L0.dtype, var, 1, flip, o.omega));
      } else {
        BLAUNCH("batched Jacobi", launch_group_op(1, ops, b, dim, L0.dtype, var, 0, flip, o.omega));
        for (Item *it : v) it->flip ^= 1;
      }
    }
    return MG_OK;
  };
  mg_status st;
  std::vector<int> sizes;
  // descend over the fine sizes
  for (auto &kv : fine) {
    sizes.push_back(kv.first);
    std::vector<Item *> G, F;
    for (Item &it : kv.second) (it.fast ? F : G).push_back(&it);
    if ((st = fast_descend(b, F, zero0))) return st;
    if (G.empty()) continue;
    const Level &L0 = G[0]->c->lv[G[0]->l];
    // operator model: nu1 sweeps and the residual of 3 words (+ faces), full
    // weighting 1 + 2^-d words per fine node
    BTimer tm(b, MG_BATCH_PRE, G.size() * nodes_of(L0) * ((3.0 * (o.nu1 + 1) + 1.0 + 1.0 / (1 << dim)) * dtype_size(L0.dtype) +
                                                       (L0.kf[0] ? (o.nu1 + 1) * dim * face_size(L0.dtype) : 0)));
    std::vector<BOp> zops = ops_of(G, true);
    if (!zops.empty()) BLAUNCH("batched zero", launch_group_op(3, zops, b, dim, L0.dtype, false, 0, G[0]->flip, 0.0));
    if ((st = smooth(G, o.nu1))) return st;
    std::vector<BOp> ops = ops_of(G, false);
    BLAUNCH("batched residual", launch_group_op(2, ops, b, dim, L0.dtype, L0.kf[0] != nullptr, 0, G[0]->flip, 0.0));
    std::vector<BXfer> xs;
    int tc = F64;
    for (Item *it : G) {
      const Level &Fl = it->c->lv[it->l];
      const Level &C = it->c->lv[it->l + 1];
      BXfer x;
      x.src = Fl.r;
      x.dst = C.f;
      x.gf = geo_of(Fl);
      x.gc = geo_of(C);
      x.live = live_of(b, it->c);
      xs.push_back(x);
      tc = C.dtype;
    }
    BLAUNCH("batched restriction", launch_group_xfer(true, xs, b, dim, L0.dtype, tc));
  }
  // coarse cycles: one block per problem
  {
    std::vector<char> recs;
    size_t smem = 0, rb = coarse_args_bytes();
    bool var = false;
    for (mg_ctx *c : ps) {
      int t = 0;
      while (t < c->nl && c->lv[t].n > top_n) t++;
      std::vector<char> rec(rb);
      size_t sm = coarse_args(c->lv, t, c->nl, t > 0 || zero0, o.smoother, o.omega, o.nu1, o.nu2, b->fp64,
                              rec.data());
      if (!sm) return bfail(MG_EINVAL, "coarse levels do not fit in shared memory");
      coarse_args_set_live(rec.data(), live_of(b, c));
      smem = std::max(smem, sm);
      var = c->lv[0].kf[0] != nullptr;
      recs.insert(recs.end(), rec.begin(), rec.end());
    }
    const void *dev = push(b, recs.data(), recs.size());
    if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
    BTimer tm(b, MG_BATCH_COARSE, 0.0);  // latency-bound: time only
    BLAUNCH("batched coarse cycle", coarse_cycle_batched(dev, (int)ps.size(), dim, var, b->fp64, smem, b->stream));
    b->launches++;
  }
  // ascend
  std::reverse(sizes.begin(), sizes.end());
  for (int n : sizes) {
    std::vector<Item *> G, F;
    for (Item &it : fine[n]) (it.fast ? F : G).push_back(&it);
    if ((st = fast_ascend(b, F, flip_of))) return st;
    if (G.empty()) continue;
    const Level &L0 = G[0]->c->lv[G[0]->l];
    BTimer tm(b, MG_BATCH_POST, G.size() * nodes_of(L0) * ((2.0 + 1.0 / (1 << dim) + 3.0 * o.nu2) * dtype_size(L0.dtype) +
                                                        (L0.kf[0] ? o.nu2 * dim * face_size(L0.dtype) : 0)));
    std::vector<BXfer> xs;
    int tc = F64;
    for (Item *it : G) {
      Level &Fl = it->c->lv[it->l];
      Level &C = it->c->lv[it->l + 1];
      BXfer x;
      x.src = C.u[C.cur ^ flip_of(it->c, it->l + 1)];
      x.dst = Fl.u[Fl.cur ^ it->flip];
      x.gf = geo_of(Fl);
      x.gc = geo_of(C);
      x.live = live_of(b, it->c);
      xs.push_back(x);
      tc = C.dtype;
    }
    BLAUNCH("batched interpolation", launch_group_xfer(false, xs, b, dim, L0.dtype, tc));
    if ((st = smooth(G, o.nu2))) return st;
  }
  // commit the live-buffer swaps
  for (auto &kv : fine)
    for (Item &it : kv.second)
      if (it.flip & 1) it.c->lv[it.l].cur ^= 1;
  return MG_OK;
}

BOuter make_outer(mg_ctx *c, bool with_d, bool with_e, double *partials) {
  BOuter o;
  memset(&o, 0, sizeof o);
  Level &O = c->dc ? c->outer : c->lv[0];
  Level &I = c->lv[0];
  o.u = (double *)O.u[O.cur];
  o.f = (const double *)O.f;
  o.sd = sten_of<double>(O);
  o.go = geo_of(O);
  o.d = with_d ? I.f : nullptr;
  o.e = with_e ? I.u[I.cur] : nullptr;
  o.gi = geo_of(I);
  o.partials = partials;
  return o;
}

bool fast_outer(const mg_ctx *c) {
  return c->opt.fuse && (c->dim == 2 ? d2::outer_ok(c->outer, c->lv[0]) : d3::outer_ok(c->outer, c->lv[0]));
}

// Defect-correction outer step of every problem in `ps`: with `update`,
// u += e (the live inner solution) first; then the FP64 residual, written as
// the next inner defect, and its norm into b->norms[i] (i = position in ps).
// Fast problems run the fused streaming step (out-of-place update, so their
// outer live buffer swaps); the others the generic update and residual.
mg_status batched_outer(mg_batch *b, const std::vector<mg_ctx *> &ps, bool update) {
  int P = (int)ps.size();
  const int dim = b->dim;
  bool var = ps[0]->variable;
  BCK("clear partials", cudaMemsetAsync(b->partials, 0, sizeof(double) * (size_t)P * kSlots, b->stream));
  std::vector<BOuter> gen;
  std::map<int, std::vector<std::pair<int, mg_ctx *>>> fast;  // outer size -> (position, problem)
  std::vector<FirstRec> first;  // zero start, homogeneous Dirichlet data: the residual is f
  double first_nodes = 0.0;
  int ti = ps[0]->lv[0].dtype;
  for (int i = 0; i < P; i++) {
    mg_ctx *c = ps[i];
    if (!update && c->u_zero && c->bc_zero && (ti == F32 || ti == BF16)) {
      first.push_back(first_record(c->outer, c->lv[0], b->partials + (size_t)i * kSlots, live_of(b, c)));
      first_nodes += nodes_of(c->outer);
    } else if (fast_outer(c)) {
      fast[c->outer.n].push_back({i, c});
    } else {
      gen.push_back(make_outer(c, true, update, b->partials + (size_t)i * kSlots));
      gen.back().live = live_of(b, c);
    }
    // the update makes u non-zero: a later single-context solve must not
    // take the zero-start residual
    if (update) c->u_zero = false;
  }
  cudaStream_t s = b->stream;
  if (!first.empty()) {
    const FirstRec *dev = push_list(b, first);
    if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
    BTimer tm(b, MG_BATCH_OUTER, first_nodes * (8.0 + dtype_size(ti)));  // read f (FP64), write the defect
    BCK("batched first defect", first_defect_list(dim, ti, dev, (int)first.size(), kPartBlocks, s));
    b->launches++;
  }
  if (!gen.empty()) {
    const BOuter *dev = (const BOuter *)push(b, gen.data(), sizeof(BOuter) * gen.size());
    if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
    dim3 gr(kPartBlocks, (unsigned)gen.size());
    double gnodes = 0.0;
    for (const BOuter &g : gen) gnodes += (double)g.go.n * g.go.n * (dim == 3 ? g.go.n : 1);
    const double wi = dtype_size(ti);
    if (update) {
      BTimer tm(b, MG_BATCH_UPDATE, gnodes * (16.0 + wi));  // read u, e; write u
      if (dim == 2) {
        if (ti == F32) kb_dc_update<2, float><<<gr, 256, 0, s>>>(dev);
        else kb_dc_update<2, bf16><<<gr, 256, 0, s>>>(dev);
      } else {
        if (ti == F32) kb_dc_update<3, float><<<gr, 256, 0, s>>>(dev);
        else kb_dc_update<3, bf16><<<gr, 256, 0, s>>>(dev);
      }
      BCK("batched update", cudaGetLastError());
      b->launches++;
    }
    // read u and f (FP64) and the FP64 faces, write the defect
    BTimer tm(b, MG_BATCH_OUTER, gnodes * (16.0 + wi + (var ? 8.0 * dim : 0.0)));
    if (dim == 2) {
      if (ti == F32) { if (var) kb_dc_residual<2, float, true><<<gr, 256, 0, s>>>(dev); else kb_dc_residual<2, float, false><<<gr, 256, 0, s>>>(dev); }
      else { if (var) kb_dc_residual<2, bf16, true><<<gr, 256, 0, s>>>(dev); else kb_dc_residual<2, bf16, false><<<gr, 256, 0, s>>>(dev); }
    } else {
      if (ti == F32) { if (var) kb_dc_residual<3, float, true><<<gr, 256, 0, s>>>(dev); else kb_dc_residual<3, float, false><<<gr, 256, 0, s>>>(dev); }
      else { if (var) kb_dc_residual<3, bf16, true><<<gr, 256, 0, s>>>(dev); else kb_dc_residual<3, bf16, false><<<gr, 256, 0, s>>>(dev); }
    }
    BCK("batched outer residual", cudaGetLastError());
    b->launches++;
  }
  for (auto &kv : fast) {
    auto &v = kv.second;
    const Level &O0 = v[0].second->outer, &I0 = v[0].second->lv[0];
    int np = 0;
    // the exact fixed-point step when every problem of the group asks for it
    // and has a one-power-of-two stencil
    bool exact = update;
    for (auto &pc : v) exact = exact && pc.second->opt.exact_outer && pow2_stencil(pc.second->outer) != kNoPow2;
    if (dim == 2) {
      std::vector<oz::ArgsOuter> recs;
      for (auto &pc : v) {
        mg_ctx *c = pc.second;
        Level &O = c->outer, &I = c->lv[0];
        oz::ArgsOuter r = d2::outer_record(O, (const double *)O.u[O.cur], (double *)O.u[O.cur ^ 1], I,
                                           update ? I.u[I.cur] : nullptr, I.f);
        r.partials = b->partials + (size_t)pc.first * kSlots;
        r.k2 = exact ? pow2_stencil(O) : 0;
        r.live = live_of(b, c);
        recs.push_back(r);
      }
      const oz::ArgsOuter *dev = push_list(b, recs);
      if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
      // read u, f (FP64) and e, write u (FP64) and the defect (no e, no u written without the update)
      BTimer tm(b, MG_BATCH_OUTER, recs.size() * nodes_of(O0) * (update ? 24.0 + 2.0 * dtype_size(I0.dtype) : 16.0 + dtype_size(I0.dtype)));
      BCK("batched outer step", d2::dc_step_list(O0, I0, dev, (int)recs.size(), nullptr, kSlots, &np, update, exact, s));
    } else {
      std::vector<z3::ArgsDC3> recs;
      for (auto &pc : v) {
        mg_ctx *c = pc.second;
        Level &O = c->outer, &I = c->lv[0];
        z3::ArgsDC3 r = d3::outer_record(O, (const double *)O.u[O.cur], (double *)O.u[O.cur ^ 1], I,
                                         update ? I.u[I.cur] : nullptr, I.f);
        r.partials = b->partials + (size_t)pc.first * kSlots;
        r.k2 = exact ? pow2_stencil(O) : 0;
        r.live = live_of(b, c);
        recs.push_back(r);
      }
      const z3::ArgsDC3 *dev = push_list(b, recs);
      if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
      BTimer tm(b, MG_BATCH_OUTER, recs.size() * nodes_of(O0) * (update ? 24.0 + 2.0 * dtype_size(I0.dtype) : 16.0 + dtype_size(I0.dtype)));
      BCK("batched outer step", d3::dc_step_list(O0, I0, dev, (int)recs.size(), nullptr, kSlots, &np, update, exact, s));
    }
    b->launches++;
    if (update)
      for (auto &pc : v) pc.second->outer.cur ^= 1;
  }
  kb_finalize<<<P, 256, 0, s>>>(b->partials, b->norms);
  BCK("batched norm finalize", cudaGetLastError());
  b->launches++;
  return MG_OK;
}

// Residual norms of every problem into b->norms[i] (i = position in ps); in
// defect-correction batches this is the outer FP64 residual, which also
// writes each problem's inner defect.
mg_status batched_norms(mg_batch *b, const std::vector<mg_ctx *> &ps) {
  if (b->dc) return batched_outer(b, ps, false);
  int P = (int)ps.size();
  const int dim = b->dim;
  bool var = ps[0]->variable;
  std::vector<BOp> os;
  for (mg_ctx *c : ps) {
    os.push_back(make_op(c->lv[0]));
    os.back().live = live_of(b, c);
  }
  const BOp *dev = (const BOp *)push(b, os.data(), sizeof(BOp) * P);
  if (!dev) return bfail(MG_ENOMEM, "batch descriptor area exhausted");
  BCK("clear partials", cudaMemsetAsync(b->partials, 0, sizeof(double) * (size_t)P * kSlots, b->stream));
  dim3 gr(kPartBlocks, P);
  if (dim == 2) { if (var) kb_norm<2, true><<<gr, 256, 0, b->stream>>>(dev, b->partials); else kb_norm<2, false><<<gr, 256, 0, b->stream>>>(dev, b->partials); }
  else { if (var) kb_norm<3, true><<<gr, 256, 0, b->stream>>>(dev, b->partials); else kb_norm<3, false><<<gr, 256, 0, b->stream>>>(dev, b->partials); }
  BCK("batched norm partials", cudaGetLastError());
  kb_finalize<<<P, 256, 0, b->stream>>>(b->partials, b->norms);
  BCK("batched norm finalize", cudaGetLastError());
  b->launches += 2;
  return MG_OK;
}

// Live-buffer state of one problem: every level's live solution buffer and
// the outer one.
struct CurSnap {
  int lv[kMaxLevels];
  int outer;
  bool operator==(const CurSnap &o) const { return outer == o.outer && !memcmp(lv, o.lv, sizeof lv); }
};

CurSnap snap(const mg_ctx *c) {
  CurSnap s;
  memset(&s, 0, sizeof s);
  for (int l = 0; l < c->nl; l++) s.lv[l] = c->lv[l].cur;
  s.outer = c->outer.cur;
  return s;
}

void restore(mg_ctx *c, const CurSnap &s) {
  for (int l = 0; l < c->nl; l++) c->lv[l].cur = s.lv[l];
  c->outer.cur = s.outer;
}

// Captures two solve steps of the problems `ps` (positions 0..P-1 of the
// live flags) into one graph: each step's inner V-cycles and outer step (or
// norms), then the stopping test. Two steps, because each step swaps some
// ping-pong buffers (the outer update, Jacobi sweeps) and its records name
// buffers: after two steps every buffer is back where it started, so the
// graph can be replayed. s1 receives each problem's buffer state after one
// step (the state of a problem that stops after an odd number of steps).
// On failure every problem's state is restored and the graph discarded.
mg_status capture_steps(mg_batch *b, const std::vector<mg_ctx *> &ps, int maxit, const std::vector<CurSnap> &s0,
                        std::vector<CurSnap> &s1, cudaGraphExec_t *exec, unsigned long long *kernels) {
  const int P = (int)ps.size();
  b->pos.clear();
  for (int i = 0; i < P; i++) b->pos[ps[i]] = i;
  b->gmode = true;
  b->goff = 0;
  const unsigned long long l0 = b->launches;
  cudaStream_t user = b->stream;
  mg_status st = MG_OK;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    st = bfail(MG_ECUDA, "begin capture of the batch steps", e);
  } else {
    b->stream = b->cap;
    const int inner = b->dc ? std::max(b->opt.inner_cycles, 1) : 1;
    for (int step = 0; step < 2 && st == MG_OK; step++) {
      for (int k = 0; k < inner && st == MG_OK; k++) st = batched_vcycle(b, ps, b->dc && k == 0);
      if (st == MG_OK) st = b->dc ? batched_outer(b, ps, true) : batched_norms(b, ps);
      if (st == MG_OK) {
        kb_check<<<1, 1024, 0, b->cap>>>(b->norms, b->r0_dev, b->tol_dev, b->live, b->iters_dev, b->rho_dev, P,
                                         maxit, b->remaining);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = bfail(MG_ECUDA, "stopping-test kernel", e);
        b->launches++;
      }
      if (step == 0)
        for (int i = 0; i < P; i++) s1[i] = snap(ps[i]);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);  // ends the capture whatever happened inside it
    b->stream = user;
    if (st == MG_OK && e != cudaSuccess) st = bfail(MG_ECUDA, "end capture of the batch steps", e);
    if (st == MG_OK) {
      e = cudaGraphInstantiate(exec, g, 0);
      if (e != cudaSuccess) st = bfail(MG_ECUDA, "instantiate the batch steps", e);
    }
    if (g) cudaGraphDestroy(g);
  }
  b->gmode = false;
  b->pos.clear();
  *kernels = b->launches - l0;
  b->launches = l0;
  for (int i = 0; i < P && st == MG_OK; i++)
    if (!(snap(ps[i]) == s0[i])) st = bfail(MG_EINVAL, "two captured steps do not return the buffers to their start");
  if (st != MG_OK) {
    for (int i = 0; i < P; i++) restore(ps[i], s0[i]);
    return st;
  }
  // the records of both steps, once, to the captured steps' own area
  e = cudaMemcpyAsync(b->gdesc, b->gstage.data(), b->goff, cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) {
    cudaGraphExecDestroy(*exec);
    return bfail(MG_ECUDA, "upload of the captured steps' descriptors", e);
  }
  return MG_OK;
}

// mg_batch_solve by replayed captured steps: the stopping test runs on the
// device, converged problems drop out of every later launch, and the host
// reads one counter per replay (two steps) with one replay queued ahead, so
// no step waits for the host. *used = false (nothing done, states intact)
// when the steps cannot be captured - too many descriptors for the captured
// area, mixed stencil kinds - and the caller steps the batch instead.
mg_status captured_solve(mg_batch *b, const std::vector<int> &ids, const double *tol, int maxit, int *iters,
                         double *relres, bool *used) {
  *used = false;
  typedef std::chrono::steady_clock clk;
  auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
  clk::time_point t0 = clk::now();
  const int P = (int)ids.size();
  std::vector<mg_ctx *> ps;
  for (int id : ids) ps.push_back(b->probs[id]);
  for (mg_ctx *c : ps)
    if ((c->variable != 0) != (ps[0]->variable != 0)) return MG_OK;
  mg_status st;
  cudaStream_t s = b->stream;
  // initial residual norms of problems not stepped before (one synchronisation)
  std::vector<mg_ctx *> fresh;
  std::vector<int> fresh_ids;
  for (int id : ids)
    if (b->r0[id] < 0.0) {
      fresh.push_back(b->probs[id]);
      fresh_ids.push_back(id);
    }
  if (!fresh.empty()) {
    b->dev_off = 0;
    if ((st = batched_norms(b, fresh))) return st;
    std::vector<double> h(fresh.size());
    BCK("read initial norms", cudaMemcpyAsync(h.data(), b->norms, sizeof(double) * fresh.size(),
                                              cudaMemcpyDeviceToHost, s));
    BCK("synchronize", cudaStreamSynchronize(s));
    for (size_t i = 0; i < fresh.size(); i++) b->r0[fresh_ids[i]] = h[i];
    b->dev_off = 0;
  }
  double *h_r0 = (double *)b->hstage, *h_tol = h_r0 + b->maxp;
  int *h_rem = (int *)(h_tol + b->maxp);
  for (int i = 0; i < P; i++) {
    h_r0[i] = b->r0[ids[i]];
    h_tol[i] = tol[ids[i]];
  }
  std::vector<CurSnap> s0(P), s1(P);
  for (int i = 0; i < P; i++) s0[i] = snap(ps[i]);
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
  b->phase_ms[0] = ms_since(t0);
  t0 = clk::now();
  if (capture_steps(b, ps, maxit, s0, s1, &exec, &kernels) != MG_OK) {
    set_error_message("");
    return MG_OK;  // not captured: the caller steps the batch
  }
  *used = true;
  b->phase_ms[1] = ms_since(t0);
  t0 = clk::now();
  BCK("upload r0", cudaMemcpyAsync(b->r0_dev, h_r0, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  BCK("upload tolerances", cudaMemcpyAsync(b->tol_dev, h_tol, sizeof(double) * P, cudaMemcpyHostToDevice, s));
  kb_arm<<<(P + 255) / 256, 256, 0, s>>>(b->live, b->iters_dev, b->rho_dev, P);
  BCK("arm kernel", cudaGetLastError());
  b->launches++;
  const int replays = (maxit + 1) / 2;
  cudaError_t e = cudaSuccess;
  int done_replays = 0;
  for (int r = 0; r < replays && e == cudaSuccess; r++) {
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) break;
    b->launches += kernels;
    done_replays++;
    e = cudaMemcpyAsync(&h_rem[r & 1], b->remaining, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[r & 1], s);
    if (e == cudaSuccess && r >= 1) {
      // the previous replay's count, while this one runs
      e = cudaEventSynchronize(b->ev[(r - 1) & 1]);
      if (e == cudaSuccess && h_rem[(r - 1) & 1] == 0) break;
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  b->phase_ms[2] = ms_since(t0);
  b->phase_ms[3] = (double)done_replays;
  b->phase_ms[4] = (double)kernels;
  cudaGraphExecDestroy(exec);
  if (e == cudaSuccess) e = e2;
  std::vector<int> it(P);
  std::vector<double> rho(P);
  if (e == cudaSuccess) e = cudaMemcpy(it.data(), b->iters_dev, sizeof(int) * P, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(rho.data(), b->rho_dev, sizeof(double) * P, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    for (int i = 0; i < P; i++) restore(ps[i], s0[i]);
    return bfail(MG_ECUDA, "captured batch steps", e);
  }
  bool bad = false, open = false;
  for (int i = 0; i < P; i++) {
    restore(ps[i], (it[i] & 1) ? s1[i] : s0[i]);  // buffers after an odd / even number of steps
    const int id = ids[i];
    if (iters) iters[id] = it[i];
    if (relres) relres[id] = rho[i];
    if (!std::isfinite(rho[i])) bad = true;
    else if (rho[i] > tol[id]) open = true;
  }
  if (bad) return bfail(MG_ENOCONV, "a residual became non-finite");
  if (open) return bfail(MG_ENOCONV, "some problems did not reach their tolerance");
  return MG_OK;
}

bool same_shape(const mg_options &a, const mg_options &b) {
  return a.smoother == b.smoother && a.omega == b.omega && a.nu1 == b.nu1 && a.nu2 == b.nu2 &&
         a.precision == b.precision && std::max(a.inner_cycles, 1) == std::max(b.inner_cycles, 1);
}

}  // namespace

extern "C" {

size_t mg_batch_workspace_bytes(int max_problems) {
  if (max_problems < 1) return 0;
  return desc_area_bytes(max_problems) + align256(sizeof(double) * (size_t)max_problems * kSlots) +
         align256(sizeof(double) * (size_t)max_problems) + solve_state_bytes(max_problems) +
         graph_area_bytes(max_problems);
}

mg_status mg_batch_create(int max_problems, void *workspace, size_t bytes, void *stream, mg_batch **out) {
  if (!out || max_problems < 1 || !workspace) return bfail(MG_EINVAL, "bad batch arguments");
  if ((uintptr_t)workspace % 256) return bfail(MG_EINVAL, "batch workspace must be 256-byte aligned");
  if (bytes < mg_batch_workspace_bytes(max_problems)) return bfail(MG_ENOMEM, "batch workspace too small");
  mg_batch *b = new (std::nothrow) mg_batch();
  if (!b) return bfail(MG_ENOMEM, "host allocation of the batch failed");
  b->maxp = max_problems;
  b->probs.assign(max_problems, nullptr);
  b->r0.assign(max_problems, -1.0);
  b->ws = (char *)workspace;
  b->ws_bytes = bytes;
  b->desc_bytes = desc_area_bytes(max_problems);
  b->partials = (double *)(b->ws + b->desc_bytes);
  b->norms = (double *)(b->ws + b->desc_bytes + align256(sizeof(double) * (size_t)max_problems * kSlots));
  // captured-solve state, then the captured steps' descriptor area
  char *st = (char *)b->norms + align256(sizeof(double) * (size_t)max_problems);
  size_t ib = align256(sizeof(int) * (size_t)max_problems), db = align256(sizeof(double) * (size_t)max_problems);
  b->live = (int *)st;
  b->iters_dev = (int *)(st + ib);
  b->rho_dev = (double *)(st + 2 * ib);
  b->r0_dev = (double *)(st + 2 * ib + db);
  b->tol_dev = (double *)(st + 2 * ib + 2 * db);
  b->remaining = (int *)(st + 2 * ib + 3 * db);
  b->gdesc = st + solve_state_bytes(max_problems);
  b->gdesc_bytes = graph_area_bytes(max_problems);
  b->goff = 0;
  b->gmode = false;
  b->capture = 1;
  b->stream = (cudaStream_t)stream;
  b->have_opts = false;
  b->list_rows = 0;
  b->launches = 0;
  b->dev_off = 0;
  b->pinned = nullptr;
  b->hstage = nullptr;
  b->cap = nullptr;
  b->ev[0] = b->ev[1] = nullptr;
  b->step_pending = false;
  b->hstep = nullptr;
  b->step_ev = b->add_ev = nullptr;
  for (int i = 0; i < 5; i++) b->phase_ms[i] = 0.0;
  b->timing = 0;
  for (int i = 0; i < 8; i++) b->t_ms[i] = b->t_bytes[i] = 0.0, b->t_n[i] = 0;
  if (cudaMallocHost((void **)&b->pinned, b->desc_bytes) != cudaSuccess ||
      cudaMallocHost((void **)&b->hstage, 2 * sizeof(double) * (size_t)max_problems + 64) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void **)&b->hstep, 2 * sizeof(double) * (size_t)max_problems) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->step_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->add_ev, cudaEventDisableTiming) != cudaSuccess) {
    mg_batch_destroy(b);
    return bfail(MG_ENOMEM, "pinned host staging, capture stream or events of the batch failed");
  }
  *out = b;
  return MG_OK;
}

mg_status mg_batch_destroy(mg_batch *b) {
  if (!b) return MG_OK;
  if (b->pinned) cudaFreeHost(b->pinned);
  if (b->hstage) cudaFreeHost(b->hstage);
  if (b->hstep) cudaFreeHost(b->hstep);
  if (b->step_ev) cudaEventDestroy(b->step_ev);
  if (b->add_ev) cudaEventDestroy(b->add_ev);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int i = 0; i < 2; i++)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  for (auto &p : b->tpend) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.e);
  }
  for (cudaEvent_t e : b->tpool) cudaEventDestroy(e);
  delete b;
  return MG_OK;
}

mg_status mg_batch_add(mg_batch *b, mg_ctx *c, int *id) {
  if (!b || !c || !id) return bfail(MG_EINVAL, "NULL argument");
  if (c->opt.smoother == MG_JACOBI && ((c->opt.nu1 + c->opt.nu2) & 1))
    return bfail(MG_EINVAL, "batched Jacobi needs an even number of sweeps per cycle");
  if (b->have_opts && (!same_shape(b->opt, c->opt) || b->dim != c->dim))
    return bfail(MG_EINVAL, "problem options differ from the batch's (smoother, omega, nu, precision, dim)");
  for (int i = 0; i < b->maxp; i++) {
    if (!b->probs[i]) {
      if (!b->have_opts) {
        b->opt = c->opt;
        b->dim = c->dim;
        b->dc = c->dc;
        b->fp64 = !c->dc;
        b->have_opts = true;
      }
      // the batch's kernels read what the context's stream wrote (its
      // right-hand side, a reset solution): order them after it
      if (c->stream != b->stream &&
          (cudaEventRecord(b->add_ev, c->stream) != cudaSuccess ||
           cudaStreamWaitEvent(b->stream, b->add_ev, 0) != cudaSuccess))
        return bfail(MG_ECUDA, "ordering the problem's stream before the batch's");
      b->probs[i] = c;
      b->r0[i] = -1.0;
      *id = i;
      return MG_OK;
    }
  }
  return bfail(MG_ENOMEM, "batch is full");
}

mg_status mg_batch_remove(mg_batch *b, int id) {
  if (!b || id < 0 || id >= b->maxp || !b->probs[id]) return bfail(MG_EINVAL, "unknown problem id");
  b->probs[id] = nullptr;
  b->r0[id] = -1.0;
  return MG_OK;
}

// Builds and enqueues one step of the `count` problems in ids on the batch
// stream: the initial norms of new problems, the step, copies of both into
// pinned host memory and an event after them. step_finish completes it.
static mg_status step_enqueue(mg_batch *b, const int *ids, int count) {
  NvtxRange range("mg_batch step");
  std::vector<mg_ctx *> ps, fresh;
  std::vector<int> fresh_ids;
  for (int i = 0; i < count; i++) {
    int id = ids[i];
    if (id < 0 || id >= b->maxp || !b->probs[id]) return bfail(MG_EINVAL, "unknown problem id");
    ps.push_back(b->probs[id]);
    if (b->r0[id] < 0.0) {
      fresh.push_back(b->probs[id]);
      fresh_ids.push_back(id);
    }
  }
  bool var = ps[0]->variable != 0;
  for (mg_ctx *c : ps)
    if ((c->variable != 0) != var) return bfail(MG_EINVAL, "a step mixes constant and variable stencils");
  mg_status st;
  b->dev_off = 0;
  // initial residual (and, with defect correction, the first defect) of new
  // problems; its norms are copied out before the step overwrites them
  if (!fresh.empty()) {
    if ((st = batched_norms(b, fresh))) return st;
    BCK("copy initial norms", cudaMemcpyAsync(b->hstep + b->maxp, b->norms, sizeof(double) * fresh.size(),
                                              cudaMemcpyDeviceToHost, b->stream));
  }
  int inner = b->dc ? std::max(b->opt.inner_cycles, 1) : 1;
  for (int k = 0; k < inner; k++)
    if ((st = batched_vcycle(b, ps, b->dc && k == 0))) return st;
  if ((st = b->dc ? batched_outer(b, ps, true) : batched_norms(b, ps))) return st;
  BCK("copy norms", cudaMemcpyAsync(b->hstep, b->norms, sizeof(double) * count, cudaMemcpyDeviceToHost, b->stream));
  BCK("step event", cudaEventRecord(b->step_ev, b->stream));
  b->step_ids.assign(ids, ids + count);
  b->step_fresh = fresh_ids;
  b->step_pending = true;
  return MG_OK;
}

// Waits for the step in flight and forms each problem's rho = ||r|| / ||r_0||.
static mg_status step_finish(mg_batch *b, double *rho) {
  NvtxRange range("mg_batch step wait");
  b->step_pending = false;
  BCK("synchronize", cudaEventSynchronize(b->step_ev));
  for (size_t i = 0; i < b->step_fresh.size(); i++) b->r0[b->step_fresh[i]] = b->hstep[b->maxp + i];
  b->dev_off = 0;
  harvest(b);
  if (rho)
    for (size_t i = 0; i < b->step_ids.size(); i++) {
      double r0 = b->r0[b->step_ids[i]];
      rho[i] = r0 > 0.0 ? b->hstep[i] / r0 : 0.0;
    }
  return MG_OK;
}

mg_status mg_batch_step(mg_batch *b, const int *ids, int count, double *rho) {
  if (!b || (count > 0 && !ids)) return bfail(MG_EINVAL, "NULL argument");
  if (b->step_pending) return bfail(MG_EINVAL, "a step started by mg_batch_step_async is still in flight");
  if (count == 0) return MG_OK;
  mg_status st = step_enqueue(b, ids, count);
  if (st) {
    b->step_pending = false;
    return st;
  }
  return step_finish(b, rho);
}

mg_status mg_batch_step_async(mg_batch *b, const int *ids, int count) {
  if (!b || (count > 0 && !ids)) return bfail(MG_EINVAL, "NULL argument");
  if (b->step_pending) return bfail(MG_EINVAL, "a step started by mg_batch_step_async is still in flight");
  if (count == 0) {
    b->step_ids.clear();
    b->step_fresh.clear();
    b->step_pending = true;  // a step of no problems: step_wait returns at once
    return cudaEventRecord(b->step_ev, b->stream) == cudaSuccess ? MG_OK : bfail(MG_ECUDA, "step event");
  }
  mg_status st = step_enqueue(b, ids, count);
  if (st) b->step_pending = false;
  return st;
}

mg_status mg_batch_step_wait(mg_batch *b, double *rho) {
  if (!b) return bfail(MG_EINVAL, "NULL batch");
  if (!b->step_pending) return bfail(MG_EINVAL, "no step in flight");
  return step_finish(b, rho);
}

mg_status mg_batch_solve(mg_batch *b, const double *tol, int maxit, int *iters, double *relres) {
  if (!b || !tol) return bfail(MG_EINVAL, "NULL argument");
  NvtxRange range("mg_batch_solve");
  if (b->step_pending) return bfail(MG_EINVAL, "a step started by mg_batch_step_async is still in flight");
  std::vector<int> active;
  for (int i = 0; i < b->maxp; i++)
    if (b->probs[i]) {
      active.push_back(i);
      if (iters) iters[i] = 0;
      if (relres) relres[i] = 1.0;
    }
  mg_status st;
  if (b->capture && maxit >= 1 && !active.empty()) {
    bool used = false;
    st = captured_solve(b, active, tol, maxit, iters, relres, &used);
    if (used || st != MG_OK) return st;
  }
  bool bad = false;
  for (int k = 1; k <= maxit && !active.empty(); k++) {
    std::vector<double> rho(active.size());
    if ((st = mg_batch_step(b, active.data(), (int)active.size(), rho.data()))) return st;
    std::vector<int> next;
    for (size_t i = 0; i < active.size(); i++) {
      int id = active[i];
      if (iters) iters[id] = k;
      if (relres) relres[id] = rho[i];
      if (!std::isfinite(rho[i])) bad = true;
      else if (rho[i] > tol[id]) next.push_back(id);
    }
    active.swap(next);
  }
  if (bad) return bfail(MG_ENOCONV, "a residual became non-finite");
  if (!active.empty()) return bfail(MG_ENOCONV, "some problems did not reach their tolerance");
  return MG_OK;
}

unsigned long long mg_batch_launches(const mg_batch *b) { return b ? b->launches : 0ull; }

mg_status mg_batch_set_timing(mg_batch *b, int on) {
  if (!b || (on != 0 && on != 1)) return bfail(MG_EINVAL, "timing must be 0 or 1");
  b->timing = on;
  return MG_OK;
}

mg_status mg_batch_get_timing(mg_batch *b, int kind, double *total_ms, unsigned long long *launches, double *bytes) {
  if (!b || kind < 0 || kind > MG_BATCH_NORM) return bfail(MG_EINVAL, "bad batch timing request");
  BCK("synchronize", cudaStreamSynchronize(b->stream));
  harvest(b);
  if (total_ms) *total_ms = b->t_ms[kind];
  if (launches) *launches = b->t_n[kind];
  if (bytes) *bytes = b->t_bytes[kind];
  return MG_OK;
}

mg_status mg_batch_reset_timing(mg_batch *b) {
  if (!b) return bfail(MG_EINVAL, "NULL batch");
  BCK("synchronize", cudaStreamSynchronize(b->stream));
  harvest(b);
  for (int i = 0; i < 8; i++) b->t_ms[i] = b->t_bytes[i] = 0.0, b->t_n[i] = 0;
  return MG_OK;
}

mg_status mg_batch_solve_profile(const mg_batch *b, double *out) {
  if (!b || !out) return bfail(MG_EINVAL, "NULL argument");
  for (int i = 0; i < 5; i++) out[i] = b->phase_ms[i];
  return MG_OK;
}

mg_status mg_batch_set_capture(mg_batch *b, int on) {
  if (!b || (on != 0 && on != 1)) return bfail(MG_EINVAL, "capture must be 0 or 1");
  b->capture = on;
  return MG_OK;
}

mg_status mg_batch_set_tile_rows(mg_batch *b, int rows) {
  if (!b || rows < 0 || rows > 65536) return bfail(MG_EINVAL, "rows must lie in 0..65536");
  b->list_rows = rows;
  return MG_OK;
}

mg_status mg_batch_set_inner_cycles(mg_batch *b, int inner_cycles) {
  if (!b || inner_cycles < 1 || inner_cycles > 8) return bfail(MG_EINVAL, "inner_cycles must lie in 1..8");
  b->opt.inner_cycles = inner_cycles;
  return MG_OK;
}

}  // extern "C"
