// Host-side context of one multigrid problem (shared by the translation
// units that drive kernels: mg_api.cu and batch.cu). Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "mg.h"
#include "mg_internal.h"

using mg::Level;

constexpr int kMaxLevels = 31;
constexpr int kGraphSlots = 4;
constexpr int kMaxPairs = 2048;       // event pairs for kernel timing
constexpr int kSlotPairs = 256;       // timed kernels per captured graph
constexpr int kKinds = 7;             // mg_kernel_kind values
constexpr int kMaxGuards = 256;       // guard zones of a canary layout (31 levels x 7 buffers + 11)
constexpr size_t kGuardBytes = 256;   // bytes per guard zone
constexpr unsigned char kGuardByte = 0xA5;  // finite as FP64, FP32 and BF16 if a kernel ever reads it

// An NVTX range open for the lifetime of the object: per entry point, V-cycle
// or solve step and level, so that a profiler can group kernels by them
// (ncu --nvtx --nvtx-include). Without a tool that reads NVTX attached the
// push and pop return at once. Inside a stream capture the ranges mark the
// capture, not the later replays of the graph.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct TimingPair {
  cudaEvent_t a, b;
  int kind, level;
  int owner;     // -1: direct launch (recycled after harvest), else graph slot
  bool pending;  // recorded, not yet harvested
};

struct GraphSlot {
  bool valid;
  int kind;           // 0 = cycle, 1 = solve step
  unsigned key;       // live-buffer bitmask at capture
  unsigned post;      // live-buffer bitmask after the captured work
  unsigned long long kernels;  // kernel nodes in the graph
  cudaGraphExec_t exec;
  int npairs;                  // timed kernels inside the graph
  int pairs[kSlotPairs];
};

struct mg_ctx {
  int dim, n, nl;
  int variable;
  bool dc;                // defect-correction precision
  bool bc_zero;           // homogeneous Dirichlet data
  bool u_zero;            // the finest (user-level) interior solution is known to be zero
  mg_options opt;
  cudaStream_t stream;    // user stream
  cudaStream_t cap;       // private stream used for graph capture
  Level lv[kMaxLevels];   // working hierarchy (FP64, or the inner DC hierarchy)
  Level outer;            // DC: outer FP64 finest level (u[0..1] ping-pong, f, r = FP64 staging, kf)
  double *partials;       // kMaxPartials doubles
  double *norm_out;       // [0] = norm, [1] = sum of squares
  float *dc_scale;        // power of two applied before squaring in scaled norm passes
  double *host_norm;      // pinned host copy of norm_out
  size_t used_bytes;
  GraphSlot graphs[kGraphSlots];
  int next_slot;
  unsigned long long launches;  // kernels launched (direct or inside replayed graphs)
  // kernel timing (mg_set_timing)
  int timing;
  int capturing_slot;          // graph slot being captured, -1 if none
  TimingPair *pairs;           // kMaxPairs entries, allocated by the first mg_set_timing(ctx, 1)
  int npairs;
  int *free_pairs;             // kMaxPairs entries
  int nfree;
  double t_ms[kKinds][kMaxLevels];
  unsigned long long t_n[kKinds][kMaxLevels];
  // canary layout (options.canary): the zone after each buffer, its owner's name
  char *arena;
  int nguards;
  size_t guard_off[kMaxGuards];
  char guard_tag[kMaxGuards][16];
  // NVTX range names of the levels ("level 3 n=513")
  char level_name[kMaxLevels][24];
};

