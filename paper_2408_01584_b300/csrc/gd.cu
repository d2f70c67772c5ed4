// C-ABI implementation of include/gd.h: scene validation and upload, static
// road / road-edge grids, per-step launches, rollouts and state access.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gd_device.cuh"
#include "observe_kernel.cuh"
#include "step_kernels.cuh"
#include "world_kernel.cuh"
#include "lidar_kernel.cuh"
#include "invert_kernel.cuh"
#include "adjoint_kernel.cuh"

using namespace gd;

namespace {

thread_local std::string g_create_error;

// NVTX range over a host entry point (a marker for profiler timelines; no
// effect unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

constexpr int kObsWarpsDefault = 8;
constexpr int kLidarGroup = 2;    // warps per agent of the stand-alone LiDAR scan (2, 3 or 4 built)
constexpr int kWorldWarps = 8;    // default CTA size of k_world (warps); 4 and 16 also built
constexpr int kAdjWarps = 8;
// Split adjoint's observer kernel: CTA size and shared memory (the
// observation scratch and one slot row per warp).
constexpr int kAdjObsWarps = 8;
constexpr size_t kAdjObsSmem = kAdjObsWarps * (sizeof(ObsWarpSmem) + GD_MAX_AGENTS_PER_WORLD);
constexpr int kTuneSteps = 4;     // consecutive steps timed per tuner window (at least)
constexpr float kTuneTrialMs = 4.f;     // a trial's windows together last about this long (longer windows for
                                       // small batches)
constexpr int kTunePhases = 3;    // points of an episode a tuner trial is timed at
constexpr float kTuneCtaMargin = 0.03f;  // a step CTA of twice the warps must time this much faster to win

// Split form's observation kernel: CTA size and shared memory.
constexpr int kSplitWarps = 8;
constexpr size_t kSplitSmem = kSplitWarps * sizeof(ObsWarpSmem);
// Let `fn` request up to the device's opt-in maximum of dynamic shared
// memory.  The attribute belongs to the kernel, not to an env, so every env
// sets the same value (an env with smaller tiles cannot shrink another's
// limit); occupancy follows the size each launch requests.
inline cudaError_t allow_max_smem(const void* fn) {
  int dev = 0, mx = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);   // the limit excludes static shared memory
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  return e;
}
// Fixed shared memory of the fused and adjoint kernels besides the road tile.
constexpr size_t world_fixed_smem(int warps) { return 128 + sizeof(FusedAgents) + warps * sizeof(ObsWarpSmem); }
constexpr size_t kAdjFixedSmem = 128 + sizeof(AdjAgents) + kAdjWarps * sizeof(ObsWarpSmem);
// Occupancy the layouts are sized for: 228 KB of shared memory per SM, of
// which the hardware keeps 1 KB per resident CTA.  Growing the per-warp
// scratch past these drops a CTA per SM (the adjoint went from 3 to 2 and
// its backward pass slowed by a fifth).
constexpr size_t kSmemPerSM = 228 * 1024, kSmemPerCta = 1024;
static_assert((32 / kSplitWarps) * (kSplitSmem + kSmemPerCta) <= kSmemPerSM, "k_observe_split: 32 warps per SM");
static_assert(3 * (kAdjFixedSmem + 16 + kSmemPerCta) <= kSmemPerSM, "k_adjoint without the tile: 3 CTAs per SM");
static_assert((32 / kAdjObsWarps) * (kAdjObsSmem + kSmemPerCta) <= kSmemPerSM, "k_adj_observer: 32 warps per SM");
// Fixed shared memory of the fused LiDAR kernel besides the road tile.
inline size_t lidar_fixed_smem(int warps, int n) {
  return 128 + sizeof(FusedAgents) + warps * lidar_warp_bytes(n) + lidar_dirs_bytes(n);
}

}  // namespace

// Message for gd_last_error(NULL) from entry points that have no env.
void gd_set_thread_error(const std::string& msg) { g_create_error = msg; }

struct gd_env {
  gd_config cfg{};
  cudaStream_t stream = nullptr;
  int W = 0, A = 0, N = 0, F = 0, amax = 0;
  DevEnv d{};
  std::vector<void*> allocs;
  int64_t bytes = 0;
  std::string err;
  unsigned* h_err = nullptr;   // pinned host copy of the sticky error word
  int obs_warps = kObsWarpsDefault;
  // batched form
  int* order = nullptr;        // [W] world order for the work list
  unsigned* counter = nullptr; // [2] k_world's work counter and exit tally (zero between launches)
  unsigned* acounter = nullptr; // k_adjoint's work counter
  int tile_cap = 0;            // bytes of the shared-memory road tile
  int notile = 0;              // 1: k_world reads every road block from global memory (more CTAs per SM)
  size_t world_smem = 0;       // dynamic shared memory of k_world
  int world_grid = 0;          // persistent CTAs
  size_t step_smem = 0;        // k_world launched without observation: no per-warp observation scratch
  int step_grid = 0;           // its persistent CTAs
  int warps = kWorldWarps;     // CTA size of k_world (4, 8 or 16 warps)
  int split = 1;               // radial observation: 1 = k_world step, then k_observe_split over agents
  int so_grid = 0;             // persistent CTAs of k_observe_split
  unsigned* ocounter = nullptr;  // its agent counters (2 x OBS_STRIPES: the overlapped rollout alternates sets)
  float4* alt_state = nullptr;   // [A] the overlapped rollout's second state buffer
  uint8_t* alt_flags = nullptr;  // [A] and flag buffer
  float road_cell = 8.f;       // road grid cell (m)
  size_t max_block = 16;       // largest road block (bytes)
  // host copy of the road, to rebuild the road blocks for another cell size
  std::vector<int> h_road_off;
  std::vector<float> h_rx, h_ry;
  std::vector<uint8_t> h_rtype;
  std::vector<int32_t> h_rpoly;
  std::vector<float4> h_bbox;
  // captured rollout graph and the arguments it was captured with
  cudaGraphExec_t graph = nullptr;
  const void* g_key[6] = {};
  int g_steps = -1;
  // differentiable rollouts: checkpoints every C steps, one recompute segment
  int C = 0, n_ckpt = 0;
  float4* ckS = nullptr;        // [n_ckpt][A]
  uint8_t* ckF = nullptr;       // [n_ckpt][A]
  int* ckT = nullptr;           // [n_ckpt][W]
  uint8_t* ckWD = nullptr;      // [n_ckpt][W]
  float4* segS = nullptr;       // [C+1][A] states of the segment being differentiated
  uint8_t* segF = nullptr;      // [C+1][A]
  int* segT = nullptr;          // [W]
  uint8_t* segWD = nullptr;     // [W]
  float4* segS2 = nullptr;      // a second segment buffer set: the captured backward recomputes one segment
  uint8_t* segF2 = nullptr;     // while the adjoint of the one after it runs
  int* segT2 = nullptr;
  uint8_t* segWD2 = nullptr;
  float4* lam = nullptr;        // [A] adjoint of the state
  float* rk_hist = nullptr;     // [episode_len][A] K-th road distance of each agent at each objective step
  uint16_t* sel_hist = nullptr; // [episode_len][A][K] road selection of each agent at each objective step, or
                                // nullptr (no room: the backward pass re-selects)
  bool sel_valid = false;       // sel_hist holds the last objective rollout's selections in the current road
                                // layout (block positions; a rebuilt road grid invalidates them)
  uint8_t* fl_hist = nullptr;   // [episode_len][A] post-step flags of each objective step, or nullptr (no room,
                                // or adjoint_recompute = 0: the backward pass recomputes with the step kernel)
  bool rec_valid = false;       // fl_hist holds the last objective rollout's decisions
  unsigned road_epoch = 0;      // number of road layouts built so far (tags the parked agents' selections)
  float* obs_scratch = nullptr; // [A,F] observation rows when the caller passes none
  int adj_tile = 0;
  int adj_notile = 0;           // 1: k_adjoint reads every road block from global memory
  size_t adj_smem = 0;
  int adj_grid = 0;
  int adj_split = 1;            // 1: k_adj_observer + k_adj_dynamics; 0: one fused k_adjoint per step
  int ao_grid = 0;              // persistent CTAs of k_adj_observer
  float4* adj_g = nullptr;      // [C][A] split adjoint: observer-side gradients, one slice per segment step
  float2* adj_cs = nullptr;     // [C][A] split adjoint: observers' (cos, sin)
  uint8_t* adj_slot = nullptr;  // [C][A][GD_MAX_AGENTS_PER_WORLD] split adjoint: partner slot rows
  unsigned* adj_oc = nullptr;   // [ADJ_STRIPES] k_adj_observer's claim counters (zero between launches)
  const float* diff_actions = nullptr;   // actions of the last objective rollout
  int diff_steps = 0;
  // captured differentiable rollouts (batched form) and their arguments
  cudaGraphExec_t ograph = nullptr;      // gd_rollout_objective
  const void* og_key[6] = {};
  int og_steps = -1;
  cudaGraphExec_t bgraph = nullptr;      // gd_rollout_backward
  const void* bg_key[7] = {};
  int bg_steps = -1;
  int og_nodes[2] = {0, 0};              // node counts of the captured objective graph: kernels, others
  int bg_nodes[2] = {0, 0};              // and of the backward graph
  // LiDAR / view cone
  int lidar_n = 0;              // rays per agent (0 = not enabled)
  LidarFan fan{};
  float2* ray_dirs = nullptr;   // [n] (cos, sin) of the ray angles in the sensor frame
  int lidar_groups = 1;         // stand-alone scan: warp groups per CTA of k_lidar_group
  int lo_grid = 0;              // its persistent CTAs
  unsigned* lcounter = nullptr; // its agent counters (two sets of LIDAR_STRIPES, alternating in the
                                // overlapped rollout)
  int lw_split = 0;             // batched form: 1 = k_world step + k_lidar_group, 0 = one fused k_world
  int lw_warps = 8;             // fused LiDAR kernel CTA size (4, 8 or 12 warps)
  int lw_notile = 0;            // 1: no shared-memory road tile (more warps per SM)
  int lw_tile = 0;              // its road tile (bytes)
  size_t lw_smem = 0;
  int lw_grid = 0;
  cudaGraphExec_t lgraph = nullptr;   // captured LiDAR rollout
  // rollout on host buffers: device staging and its captured pipeline
  cudaGraphExec_t hgraph = nullptr;
  const void* hg_key[4] = {};
  int hg_steps = -1;
  float* hs_act = nullptr;      // [steps, A, 2]
  float* hs_rew = nullptr;      // [steps, A]
  uint8_t* hs_done = nullptr;   // [steps, A]
  int hs_cap = 0;               // steps the staging holds
  const void* lg_key[8] = {};
  int lg_steps = -1;
};

namespace {

gd_status fail(gd_env* env, gd_status st, const std::string& msg) {
  if (env) env->err = msg; else g_create_error = msg;
  return st;
}

gd_status cuda_fail(gd_env* env, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(env, e == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA, m);
}

template <typename T>
cudaError_t dev_alloc(gd_env* env, T** p, size_t count) {
  *p = nullptr;
  const size_t b = std::max<size_t>(count, 1) * sizeof(T);
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) return e;
  env->allocs.push_back(q);
  env->bytes += (int64_t)b;
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

template <typename T>
cudaError_t upload(gd_env* env, T** p, const T* host, size_t count) {
  cudaError_t e = dev_alloc(env, p, count);
  if (e != cudaSuccess || count == 0) return e;
  return cudaMemcpyAsync(*p, host, count * sizeof(T), cudaMemcpyHostToDevice, env->stream);
}

bool finite(float v) { return std::isfinite(v); }

// Static uniform grid of one world (host build).  Points are counted per
// cell and placed in row-major cell order (stable: ascending index inside a
// cell), so a run of cells of one row is one contiguous range.
struct HostGrid {
  std::vector<GridDesc> desc;
  std::vector<int> cell_start;
};

void grid_geometry(float minx, float miny, float maxx, float maxy, float cs, GridDesc& g) {
  g.ox = minx;
  g.oy = miny;
  g.cs = cs;
  g.inv_cs = 1.f / cs;
  g.nx = std::max(1, (int)std::floor((maxx - minx) * g.inv_cs) + 1);
  g.ny = std::max(1, (int)std::floor((maxy - miny) * g.inv_cs) + 1);
  g.seg_max = 0.f;
  g.block_bytes = 0;
}

int cell_clamped(float v, float o, float inv, int n) {
  const int c = (int)std::floor((v - o) * inv);
  return std::min(std::max(c, 0), n - 1);
}


// ---- road blocks and kernel shapes (built at create, rebuilt by the tuner) ---

static void dev_free(gd_env* env, void* p) {
  if (!p) return;
  for (size_t k = 0; k < env->allocs.size(); ++k)
    if (env->allocs[k] == p) {
      env->allocs.erase(env->allocs.begin() + (long)k);
      break;
    }
  cudaFree(p);
}

template <int WARPS>
static cudaError_t shape_world(gd_env* env, size_t max_block, int smem_sm, int smem_blk, int nsm) {
  const long fixed = (long)world_fixed_smem(WARPS);
  const long two = ((long)smem_sm / 2 - 2048 - fixed) & ~15L;   // tile bytes, 2 CTAs/SM
  const long one = ((long)smem_blk - 1024 - fixed) & ~15L;      // 1 CTA/SM
  const long cap = ((long)max_block <= two) ? (long)max_block : one;
  env->tile_cap = env->notile ? 16 : (int)std::max(16L, cap);
  env->world_smem = (size_t)fixed + (size_t)env->tile_cap;
  // a launch without observation (the split form's step, gd_step) needs no
  // per-warp observation scratch: the register-capped instantiation with
  // the barrier, the agents and the tile only
  env->step_smem = (size_t)world_fixed_smem(0) + (size_t)env->tile_cap;
  // without the tile: the register-capped instantiation (more CTAs per SM)
  const void* fn = env->notile ? reinterpret_cast<const void*>(k_world<WARPS, false, true>)
                               : reinterpret_cast<const void*>(k_world<WARPS>);
  const void* lean = reinterpret_cast<const void*>(k_world<WARPS, false, true>);
  cudaError_t e = allow_max_smem(fn);
  if (e == cudaSuccess) e = allow_max_smem(lean);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, WARPS * 32, env->world_smem);
  if (e != cudaSuccess) return e;
  env->world_grid = std::max(1, std::min(env->W, std::max(per_sm, 1) * nsm));
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lean, WARPS * 32, env->step_smem);
  if (e != cudaSuccess) return e;
  env->step_grid = std::max(1, std::min(env->W, std::max(per_sm, 1) * nsm));
  return cudaSuccess;
}

template <int WARPS>
static cudaError_t shape_world_lidar(gd_env* env, size_t max_block, int smem_sm, int smem_blk, int nsm) {
  const long fixed = (long)lidar_fixed_smem(WARPS, env->lidar_n);
  const long two = ((long)smem_sm / 2 - 2048 - fixed) & ~15L;
  const long one = ((long)smem_blk - 1024 - fixed) & ~15L;
  const long cap = ((long)max_block <= two) ? (long)max_block : std::min<long>(one, (long)max_block);
  // without a tile every world reads its road from global memory (L1/L2)
  env->lw_tile = env->lw_notile ? 16 : (int)std::max(16L, cap);
  env->lw_smem = (size_t)fixed + (size_t)env->lw_tile;
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(k_world<WARPS, true>));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_world<WARPS, true>, WARPS * 32, env->lw_smem);
  if (e != cudaSuccess) return e;
  env->lw_grid = std::max(1, std::min(env->W, std::max(per_sm, 1) * nsm));
  return cudaSuccess;
}

// Tile sizes, shared memory and grid of the fused (and adjoint) kernel for
// the current road blocks and CTA size.
static cudaError_t shape_kernels(gd_env* env, size_t max_block) {
  int dev = 0, smem_sm = 0, smem_blk = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  switch (env->warps) {
    case 4: e = shape_world<4>(env, max_block, smem_sm, smem_blk, nsm); break;
    case 16: e = shape_world<16>(env, max_block, smem_sm, smem_blk, nsm); break;
    default: env->warps = 8; e = shape_world<8>(env, max_block, smem_sm, smem_blk, nsm); break;
  }
  if (e != cudaSuccess) return e;
  {
    int per_sm = 0;
    e = allow_max_smem(reinterpret_cast<const void*>(k_observe_split<kSplitWarps>));
    if (e == cudaSuccess) e = allow_max_smem(reinterpret_cast<const void*>(k_observe_split<kSplitWarps, true>));
    if (e == cudaSuccess) e = allow_max_smem(reinterpret_cast<const void*>(k_observe_split<kSplitWarps, false, true>));
    if (e == cudaSuccess) e = allow_max_smem(reinterpret_cast<const void*>(k_observe_split<kSplitWarps, true, true>));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_observe_split<kSplitWarps>, kSplitWarps * 32,
                                                        kSplitSmem);
    if (e != cudaSuccess) return e;
    env->so_grid = std::max(1, std::min(std::max(per_sm, 1) * nsm, (env->A + kSplitWarps - 1) / kSplitWarps));
    // warp g draws from claim counter g mod OBS_STRIPES: every counter that
    // holds an agent needs a warp
    env->so_grid = std::max(env->so_grid, (std::min(env->A, (int)OBS_STRIPES) + kSplitWarps - 1) / kSplitWarps);
  }
  if (env->lidar_n > 0) {
    // the tile shrinks first; if even a 16-byte tile does not fit, fewer warps
    while (env->lw_warps > 4 && lidar_fixed_smem(env->lw_warps, env->lidar_n) + 16 + 1024 > (size_t)smem_blk)
      env->lw_warps -= 4;
    switch (env->lw_warps) {
      case 4: e = shape_world_lidar<4>(env, max_block, smem_sm, smem_blk, nsm); break;
      case 12: e = shape_world_lidar<12>(env, max_block, smem_sm, smem_blk, nsm); break;
      default: env->lw_warps = 8; e = shape_world_lidar<8>(env, max_block, smem_sm, smem_blk, nsm); break;
    }
    if (e != cudaSuccess) return e;
  }
  if (env->cfg.flags & GD_DIFFERENTIABLE) {
    const long two = ((long)smem_sm / 2 - 2048 - (long)kAdjFixedSmem) & ~15L;
    const long one = ((long)smem_blk - 1024 - (long)kAdjFixedSmem) & ~15L;
    env->adj_tile = env->adj_notile ? 16 : (int)std::max(16L, ((long)max_block <= two) ? (long)max_block : one);
    env->adj_smem = kAdjFixedSmem + (size_t)env->adj_tile;
    // without the tile: the register-capped instantiation (more CTAs per SM)
    const void* afn = env->adj_notile ? reinterpret_cast<const void*>(k_adjoint<kAdjWarps, true>)
                                      : reinterpret_cast<const void*>(k_adjoint<kAdjWarps>);
    e = allow_max_smem(afn);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, afn, kAdjWarps * 32, env->adj_smem);
    if (e != cudaSuccess) return e;
    env->adj_grid = std::max(1, std::min(env->W, std::max(per_sm, 1) * nsm));
    const void* ofn = reinterpret_cast<const void*>(k_adj_observer<kAdjObsWarps>);
    e = allow_max_smem(ofn);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ofn, kAdjObsWarps * 32, kAdjObsSmem);
    if (e != cudaSuccess) return e;
    env->ao_grid = std::max(1, std::min(std::max(per_sm, 1) * nsm,
                                        (env->C * env->A + kAdjObsWarps - 1) / kAdjObsWarps));
    // every claim counter that holds a task needs a warp (warp g draws from
    // counter g mod ADJ_STRIPES)
    env->ao_grid = std::max(env->ao_grid, (std::min(env->C * env->A, (int)ADJ_STRIPES) + kAdjObsWarps - 1) / kAdjObsWarps);
  }
  return cudaSuccess;
}

// Captured graphs hold kernel shapes and device pointers by value: any
// change of shape or arena drops them (they are captured again on the next
// call).
static void drop_graphs(gd_env* env) {
  for (cudaGraphExec_t* g : {&env->graph, &env->lgraph, &env->hgraph, &env->ograph, &env->bgraph}) {
    if (*g) cudaGraphExecDestroy(*g);
    *g = nullptr;
  }
}

// Road arena for grid cell `cell` (m): per world one 16-byte aligned block of
// cell-sorted points, road_pad(N_w) float2 (x, y), road_pad(N_w) uint16
// (index | type << 15), road_pad(N_w) uint16 next-point-of-the-edge-segment,
// then the uint16 cell starts of the world's road grid.  Replaces any
// earlier arena; synchronises the env's stream.
static cudaError_t build_road(gd_env* env, float cell) {
  const int W = env->W;
  const std::vector<int>& off = env->h_road_off;
  std::vector<GridDesc> rdesc(W);
  std::vector<long long> arena_off(W);
  size_t arena_bytes = 0, max_block = 16;
  for (int w = 0; w < W; ++w) {
    const float4 bb = env->h_bbox[w];
    grid_geometry(bb.x, bb.y, bb.z, bb.w, cell, rdesc[w]);
    rdesc[w].block_bytes = road_block_bytes(off[w + 1] - off[w], rdesc[w].nx * rdesc[w].ny);
    arena_off[w] = (long long)(arena_bytes / 16);
    arena_bytes += (size_t)rdesc[w].block_bytes;
    max_block = std::max(max_block, (size_t)rdesc[w].block_bytes);
  }
  std::vector<unsigned char> arena(std::max<size_t>(arena_bytes, 16), 0);
  std::vector<float4> lsegs;
  std::vector<int> lcell;
  for (int w = 0; w < W; ++w) {
    const int r0 = off[w], r1 = off[w + 1], nr = r1 - r0;
    GridDesc& g = rdesc[w];
    const int nc = g.nx * g.ny;
    std::vector<int> cnt(nc + 1, 0), cellid(nr), pos(nr);
    for (int j = r0; j < r1; ++j) {
      const int cx = cell_clamped(env->h_rx[j], g.ox, g.inv_cs, g.nx), cy = cell_clamped(env->h_ry[j], g.oy, g.inv_cs, g.ny);
      cellid[j - r0] = cy * g.nx + cx;
      cnt[cellid[j - r0] + 1]++;
    }
    for (int c = 0; c < nc; ++c) cnt[c + 1] += cnt[c];
    unsigned char* blk = arena.data() + (size_t)arena_off[w] * 16;
    float2* bxy = reinterpret_cast<float2*>(blk);
    uint16_t* bmeta = reinterpret_cast<uint16_t*>(bxy + road_pad(nr));
    uint16_t* bnext = bmeta + road_pad(nr);
    uint16_t* bcells = bnext + road_pad(nr);
    for (int c = 0; c <= nc; ++c) bcells[c] = (uint16_t)cnt[c];   // positions within the block
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int j = r0; j < r1; ++j) {
      const int dst = fill[cellid[j - r0]]++;
      pos[j - r0] = dst;
      bxy[dst] = make_float2(env->h_rx[j], env->h_ry[j]);
      bmeta[dst] = (uint16_t)((j - r0) | (env->h_rtype[j] << 15));
    }
    // road-edge segments: consecutive ROAD_EDGE points of one polyline
    // (next links inside the block, and the LiDAR list by first-point cell)
    std::vector<int> scnt(nc + 1, 0);
    for (int j = r0; j + 1 < r1; ++j)
      if (env->h_rtype[j] == GD_ROAD_EDGE && env->h_rtype[j + 1] == GD_ROAD_EDGE && env->h_rpoly[j] == env->h_rpoly[j + 1])
        scnt[cellid[j - r0] + 1]++;
    for (int c = 0; c < nc; ++c) scnt[c + 1] += scnt[c];
    g.cell_base = (int)lcell.size();
    const int sbase = (int)lsegs.size();
    for (int c = 0; c <= nc; ++c) lcell.push_back(sbase + scnt[c]);
    lsegs.resize((size_t)sbase + scnt[nc]);
    for (int j = r0; j + 1 < r1; ++j)
      if (env->h_rtype[j] == GD_ROAD_EDGE && env->h_rtype[j + 1] == GD_ROAD_EDGE && env->h_rpoly[j] == env->h_rpoly[j + 1])
        lsegs[(size_t)sbase + scnt[cellid[j - r0]]++] =
            make_float4(env->h_rx[j], env->h_ry[j], env->h_rx[j + 1], env->h_ry[j + 1]);
    float seg_max = 0.f;
    for (int j = r0; j < r1; ++j) {
      const bool seg = j + 1 < r1 && env->h_rtype[j] == GD_ROAD_EDGE && env->h_rtype[j + 1] == GD_ROAD_EDGE &&
                       env->h_rpoly[j] == env->h_rpoly[j + 1];
      bnext[pos[j - r0]] = seg ? (uint16_t)pos[j + 1 - r0] : NO_SEGMENT;
      if (seg) seg_max = std::max(seg_max, std::hypot(env->h_rx[j + 1] - env->h_rx[j], env->h_ry[j + 1] - env->h_ry[j]));
    }
    g.seg_max = seg_max;
  }
  cudaError_t e = cudaStreamSynchronize(env->stream);
  if (e != cudaSuccess) return e;
  dev_free(env, const_cast<GridDesc*>(env->d.rgrid));
  dev_free(env, const_cast<unsigned char*>(env->d.arena));
  dev_free(env, const_cast<float4*>(env->d.lsegs));
  dev_free(env, const_cast<int*>(env->d.lcell));
  env->d.lsegs = nullptr;
  env->d.lcell = nullptr;
  dev_free(env, const_cast<long long*>(env->d.arena_off));
  env->d.rgrid = nullptr;
  env->d.arena = nullptr;
  env->d.arena_off = nullptr;
  GridDesc* p_rg;
  unsigned char* p_arena;
  long long* p_aroff;
  if ((e = upload(env, &p_rg, rdesc.data(), (size_t)W)) != cudaSuccess) return e;
  env->d.rgrid = p_rg;
  if ((e = upload(env, &p_arena, arena.data(), arena.size())) != cudaSuccess) return e;
  env->d.arena = p_arena;
  if ((e = upload(env, &p_aroff, arena_off.data(), (size_t)W)) != cudaSuccess) return e;
  env->d.arena_off = p_aroff;
  float4* p_ls;
  int* p_lc;
  if ((e = upload(env, &p_ls, lsegs.data(), lsegs.size())) != cudaSuccess) return e;
  env->d.lsegs = p_ls;
  if ((e = upload(env, &p_lc, lcell.data(), lcell.size())) != cudaSuccess) return e;
  env->d.lcell = p_lc;
  env->road_cell = cell;
  env->max_block = max_block;
  env->sel_valid = false;    // recorded selections name positions in the old blocks
  env->d.road_epoch = ++env->road_epoch;   // and so do the parked agents' kept selections
  if ((e = shape_kernels(env, max_block)) != cudaSuccess) return e;
  drop_graphs(env);
  return cudaStreamSynchronize(env->stream);
}

}  // namespace

extern "C" {

void gd_default_config(gd_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->k_road = 200;
  c->n_partners = 63;
  c->episode_len = 91;
  c->ckpt_every = 10;
  c->obs_radius = 50.f;
  c->goal_radius = 2.f;
  c->dt = 0.1f;
  c->v_max = 30.f;
  c->collision_penalty = 0.f;
  c->offroad_penalty = 0.f;
  c->smooth_c = 1.f;
  c->flags = 0;
  c->block_size = 0;
  c->road_cell = 0.f;
  c->topk_strategy = 0;
  c->lidar_rays = 0;
  c->lidar_fov = 6.28318530717958647692f;
  c->dynamics = GD_DYN_BICYCLE;
  c->nontrivial_dist = 2.f;
  c->obs_split = 1;
  c->adjoint_split = 1;
  c->adjoint_recompute = 1;
}

const char* gd_last_error(const gd_env* env) { return env ? env->err.c_str() : g_create_error.c_str(); }

gd_status gd_destroy(gd_env* env) {
  if (!env) return GD_OK;
  cudaStreamSynchronize(env->stream);
  drop_graphs(env);
  for (void* p : env->allocs) cudaFree(p);
  if (env->h_err) cudaFreeHost(env->h_err);
  delete env;
  return GD_OK;
}

static inline unsigned blocks_for_host(long n, int per) { return (unsigned)std::max<long>(1, (n + per - 1) / per); }

static gd_status validate(const gd_config* c, const gd_scene_batch* s) {
  if (!c || !s) return fail(nullptr, GD_ERR_INVALID_ARG, "config and scene must not be NULL");
  if (s->num_worlds < 1) return fail(nullptr, GD_ERR_INVALID_ARG, "num_worlds must be >= 1");
  if (!s->agent_off || !s->road_off) return fail(nullptr, GD_ERR_INVALID_ARG, "agent_off / road_off are NULL");
  if (c->k_road < 0 || c->k_road > GD_MAX_K_ROAD) return fail(nullptr, GD_ERR_CAPACITY, "k_road outside 0..GD_MAX_K_ROAD");
  if (c->n_partners < 0 || c->n_partners > GD_MAX_PARTNERS)
    return fail(nullptr, GD_ERR_CAPACITY, "n_partners outside 0..GD_MAX_PARTNERS");
  if (c->episode_len < 1) return fail(nullptr, GD_ERR_INVALID_ARG, "episode_len must be >= 1");
  if (!(c->obs_radius > 0.f) || !finite(c->obs_radius)) return fail(nullptr, GD_ERR_INVALID_ARG, "obs_radius must be > 0");
  if (!(c->goal_radius >= 0.f) || !finite(c->goal_radius)) return fail(nullptr, GD_ERR_INVALID_ARG, "goal_radius must be >= 0");
  if (!(c->dt > 0.f) || !finite(c->dt)) return fail(nullptr, GD_ERR_INVALID_ARG, "dt must be > 0");
  if (!(c->v_max > 0.f) || !finite(c->v_max)) return fail(nullptr, GD_ERR_INVALID_ARG, "v_max must be > 0");
  if (!finite(c->collision_penalty) || !finite(c->offroad_penalty) || !(c->smooth_c > 0.f))
    return fail(nullptr, GD_ERR_INVALID_ARG, "penalties must be finite and smooth_c > 0");
  if (c->road_cell < 0.f || !finite(c->road_cell)) return fail(nullptr, GD_ERR_INVALID_ARG, "road_cell must be >= 0");
  if (c->ckpt_every < 1) return fail(nullptr, GD_ERR_INVALID_ARG, "ckpt_every must be >= 1");
  if (c->block_size != 0 && c->block_size != 128 && c->block_size != 256 && c->block_size != 512)
    return fail(nullptr, GD_ERR_INVALID_ARG, "block_size must be 0, 128, 256 or 512");
  if (c->topk_strategy < 0 || c->topk_strategy > 2) return fail(nullptr, GD_ERR_INVALID_ARG, "topk_strategy must be 0..2");
  if (c->obs_split != 0 && c->obs_split != 1) return fail(nullptr, GD_ERR_INVALID_ARG, "obs_split must be 0 or 1");
  if (c->adjoint_split != 0 && c->adjoint_split != 1)
    return fail(nullptr, GD_ERR_INVALID_ARG, "adjoint_split must be 0 or 1");
  if (c->adjoint_recompute != 0 && c->adjoint_recompute != 1)
    return fail(nullptr, GD_ERR_INVALID_ARG, "adjoint_recompute must be 0 or 1");
  if (c->lidar_rays < 0 || c->lidar_rays > GD_MAX_LIDAR_RAYS)
    return fail(nullptr, GD_ERR_CAPACITY, "lidar_rays outside 0..GD_MAX_LIDAR_RAYS");
  if (!(c->lidar_fov >= 1e-3f) || !(c->lidar_fov <= 6.2831855f))
    return fail(nullptr, GD_ERR_INVALID_ARG, "lidar_fov must be in [1e-3, 2 pi]");
  if (c->lidar_block_size != 0 && c->lidar_block_size != 128 && c->lidar_block_size != 256 &&
      c->lidar_block_size != 384)
    return fail(nullptr, GD_ERR_INVALID_ARG, "lidar_block_size must be 0, 128, 256 or 384");
  if (c->lidar_no_tile != 0 && c->lidar_no_tile != 1) return fail(nullptr, GD_ERR_INVALID_ARG, "lidar_no_tile must be 0 or 1");
  if (c->lidar_split != 0 && c->lidar_split != 1) return fail(nullptr, GD_ERR_INVALID_ARG, "lidar_split must be 0 or 1");
  if (c->road_no_tile != 0 && c->road_no_tile != 1) return fail(nullptr, GD_ERR_INVALID_ARG, "road_no_tile must be 0 or 1");
  if (c->dynamics != GD_DYN_BICYCLE && c->dynamics != GD_DYN_INVERTIBLE)
    return fail(nullptr, GD_ERR_INVALID_ARG, "dynamics must be GD_DYN_BICYCLE or GD_DYN_INVERTIBLE");
  if (!(c->nontrivial_dist >= 0.f) || !finite(c->nontrivial_dist))
    return fail(nullptr, GD_ERR_INVALID_ARG, "nontrivial_dist must be >= 0");
  if ((c->flags & GD_DIFFERENTIABLE) && (c->flags & GD_AUTO_RESET))
    return fail(nullptr, GD_ERR_INVALID_ARG, "GD_DIFFERENTIABLE cannot be combined with GD_AUTO_RESET");
  const int W = s->num_worlds;
  if (s->agent_off[0] != 0 || s->road_off[0] != 0) return fail(nullptr, GD_ERR_INVALID_ARG, "offsets must start at 0");
  for (int w = 0; w < W; ++w) {
    const int na = s->agent_off[w + 1] - s->agent_off[w], nr = s->road_off[w + 1] - s->road_off[w];
    if (na < 0 || nr < 0) return fail(nullptr, GD_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (na > GD_MAX_AGENTS_PER_WORLD)
      return fail(nullptr, GD_ERR_CAPACITY, "world " + std::to_string(w) + " has more than GD_MAX_AGENTS_PER_WORLD agents");
    if (nr > GD_MAX_ROAD_PER_WORLD)
      return fail(nullptr, GD_ERR_CAPACITY, "world " + std::to_string(w) + " has more than GD_MAX_ROAD_PER_WORLD road points");
  }
  const int A = s->agent_off[W], N = s->road_off[W];
  if (A > 0 && (!s->x || !s->y || !s->theta || !s->v || !s->length || !s->width || !s->goal_x || !s->goal_y ||
                !s->agent_type))
    return fail(nullptr, GD_ERR_INVALID_ARG, "agent arrays must not be NULL");
  if (N > 0 && (!s->road_x || !s->road_y || !s->road_type || !s->road_poly))
    return fail(nullptr, GD_ERR_INVALID_ARG, "road arrays must not be NULL");
  for (int i = 0; i < A; ++i) {
    if (!finite(s->x[i]) || !finite(s->y[i]) || !finite(s->theta[i]) || !finite(s->v[i]) || !finite(s->goal_x[i]) ||
        !finite(s->goal_y[i]))
      return fail(nullptr, GD_ERR_INVALID_ARG, "agent " + std::to_string(i) + " has a non-finite value");
    if (!(s->length[i] > 0.f) || !(s->width[i] > 0.f) || !finite(s->length[i]) || !finite(s->width[i]))
      return fail(nullptr, GD_ERR_INVALID_ARG, "agent " + std::to_string(i) + " has a non-positive size");
    if (s->agent_type[i] > GD_AGENT_PEDESTRIAN) return fail(nullptr, GD_ERR_INVALID_ARG, "bad agent_type");
  }
  for (int j = 0; j < N; ++j) {
    if (!finite(s->road_x[j]) || !finite(s->road_y[j]))
      return fail(nullptr, GD_ERR_INVALID_ARG, "road point " + std::to_string(j) + " is not finite");
    if (s->road_type[j] > GD_ROAD_EDGE) return fail(nullptr, GD_ERR_INVALID_ARG, "bad road_type");
  }
  return GD_OK;
}

gd_status gd_create(const gd_config* cfg, const gd_scene_batch* s, void* cuda_stream, gd_env** out) {
  NvtxRange range_("gd_create");
  if (!out) return fail(nullptr, GD_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  gd_status st = validate(cfg, s);
  if (st != GD_OK) return st;
  gd_env* env = new (std::nothrow) gd_env();
  if (!env) return fail(nullptr, GD_ERR_OOM, "host allocation failed");
  env->cfg = *cfg;
  env->stream = static_cast<cudaStream_t>(cuda_stream);
  const int W = s->num_worlds, A = s->agent_off[W], N = s->road_off[W];
  const int K = cfg->k_road, P = cfg->n_partners;
  env->W = W; env->A = A; env->N = N; env->F = 8 + 8 * P + 4 * K;
  for (int w = 0; w < W; ++w) env->amax = std::max(env->amax, s->agent_off[w + 1] - s->agent_off[w]);
  const float R = cfg->obs_radius;
  // road cell: at most MAX_ROWS rows may cross the observation disk
  float rcell = cfg->road_cell > 0.f ? cfg->road_cell : 8.f;
  rcell = std::max(rcell, (2.f * R + 0.01f) / (float)(MAX_ROWS - 2));
  const float ecell = 8.f;

  // ---- host-side preprocessing --------------------------------------------
  std::vector<float4> h_state(A), h_stat(A);
  std::vector<int> h_agent_world(A);
  float max_diag = 0.f;
  for (int w = 0; w < W; ++w)
    for (int i = s->agent_off[w]; i < s->agent_off[w + 1]; ++i) {
      h_state[i] = make_float4(s->x[i], s->y[i], s->theta[i], s->v[i]);
      h_stat[i] = make_float4(s->length[i], s->width[i], s->goal_x[i], s->goal_y[i]);
      h_agent_world[i] = w;
      max_diag = std::max(max_diag, std::sqrt(s->length[i] * s->length[i] + s->width[i] * s->width[i]));
    }
  // keep the road on the host (the tuner rebuilds the road blocks) and
  // build the edge-segment grid of the per-stage form
  env->h_road_off.assign(s->road_off, s->road_off + W + 1);
  env->h_rx.assign(s->road_x, s->road_x + N);
  env->h_ry.assign(s->road_y, s->road_y + N);
  env->h_rtype.assign(s->road_type, s->road_type + N);
  env->h_rpoly.assign(s->road_poly, s->road_poly + N);
  env->h_bbox.resize(W);
  std::vector<GridDesc> edesc(W);
  std::vector<int> ecell_start;
  std::vector<float4> esegs;
  for (int w = 0; w < W; ++w) {
    const int r0 = s->road_off[w], r1 = s->road_off[w + 1];
    float minx = 0.f, miny = 0.f, maxx = 0.f, maxy = 0.f;
    if (r1 > r0) {
      minx = maxx = s->road_x[r0];
      miny = maxy = s->road_y[r0];
      for (int j = r0; j < r1; ++j) {
        minx = std::min(minx, s->road_x[j]); maxx = std::max(maxx, s->road_x[j]);
        miny = std::min(miny, s->road_y[j]); maxy = std::max(maxy, s->road_y[j]);
      }
    }
    env->h_bbox[w] = make_float4(minx, miny, maxx, maxy);
    // road-edge segment grid: a segment is listed under every cell its
    // bounding box (grown by 1 mm) touches
    GridDesc& eg = edesc[w];
    grid_geometry(minx, miny, maxx, maxy, ecell, eg);
    eg.cell_base = (int)ecell_start.size();
    const int enc = eg.nx * eg.ny;
    std::vector<std::vector<float4>> per(enc);
    for (int j = r0; j + 1 < r1; ++j) {
      if (s->road_type[j] != GD_ROAD_EDGE || s->road_type[j + 1] != GD_ROAD_EDGE || s->road_poly[j] != s->road_poly[j + 1])
        continue;
      const float4 sg = make_float4(s->road_x[j], s->road_y[j], s->road_x[j + 1], s->road_y[j + 1]);
      const float m = 1e-3f;
      const int cx0 = cell_clamped(std::min(sg.x, sg.z) - m, eg.ox, eg.inv_cs, eg.nx);
      const int cx1 = cell_clamped(std::max(sg.x, sg.z) + m, eg.ox, eg.inv_cs, eg.nx);
      const int cy0 = cell_clamped(std::min(sg.y, sg.w) - m, eg.oy, eg.inv_cs, eg.ny);
      const int cy1 = cell_clamped(std::max(sg.y, sg.w) + m, eg.oy, eg.inv_cs, eg.ny);
      for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) per[cy * eg.nx + cx].push_back(sg);
    }
    for (int c = 0; c < enc; ++c) {
      ecell_start.push_back((int)esegs.size());
      esegs.insert(esegs.end(), per[c].begin(), per[c].end());
    }
    ecell_start.push_back((int)esegs.size());
  }

  // ---- device upload --------------------------------------------------------
  DevEnv& d = env->d;
  d.W = W; d.A = A; d.N = N; d.K = K; d.P = P; d.F = env->F; d.T = cfg->episode_len;
  d.R = R; d.R2 = R * R; d.goal_r = cfg->goal_radius; d.dt = cfg->dt; d.vmax = cfg->v_max;
  d.cpen = cfg->collision_penalty; d.opn = cfg->offroad_penalty; d.smooth_c = cfg->smooth_c;
  d.agent_cell = max_diag * 1.01f + 0.01f;
  d.cflags = cfg->flags;
  d.dyn = cfg->dynamics;
  std::vector<uint8_t> zeros_a(A, 0);
  std::vector<int> zeros_w(W, 0);
  int* p_aoff; int* p_roff; int* p_aw; float4* p_state; float4* p_init; float4* p_stat; uint8_t* p_type;
  uint8_t* p_flags; uint8_t* p_iflags; int* p_t; uint8_t* p_wd;
  GridDesc* p_eg; int* p_ecs; float4* p_es;
  cudaError_t e = cudaSuccess;
#define GD_TRY(x) do { e = (x); if (e != cudaSuccess) { gd_status r_ = cuda_fail(nullptr, e, #x); gd_destroy(env); return r_; } } while (0)
  GD_TRY(upload(env, &p_aoff, s->agent_off, (size_t)W + 1));
  GD_TRY(upload(env, &p_roff, s->road_off, (size_t)W + 1));
  GD_TRY(upload(env, &p_aw, h_agent_world.data(), (size_t)A));
  GD_TRY(upload(env, &p_state, h_state.data(), (size_t)A));
  GD_TRY(upload(env, &p_init, h_state.data(), (size_t)A));
  GD_TRY(upload(env, &p_stat, h_stat.data(), (size_t)A));
  GD_TRY(upload(env, &p_type, s->agent_type, (size_t)A));
  GD_TRY(upload(env, &p_flags, zeros_a.data(), (size_t)A));
  GD_TRY(upload(env, &p_iflags, zeros_a.data(), (size_t)A));
  GD_TRY(upload(env, &p_t, zeros_w.data(), (size_t)W));
  GD_TRY(dev_alloc(env, &p_wd, (size_t)W));
  GD_TRY(cudaMemsetAsync(p_wd, 0, (size_t)W, env->stream));
  GD_TRY(upload(env, &p_eg, edesc.data(), (size_t)W));
  GD_TRY(upload(env, &p_ecs, ecell_start.data(), ecell_start.size()));
  GD_TRY(upload(env, &p_es, esegs.data(), esegs.size()));
  GD_TRY(dev_alloc(env, &d.agrid_key, (size_t)A));
  GD_TRY(dev_alloc(env, &d.agrid_n, (size_t)W));
  GD_TRY(dev_alloc(env, &d.coll, (size_t)A));
  GD_TRY(dev_alloc(env, &d.off, (size_t)A));
  GD_TRY(dev_alloc(env, &d.err, 1));
  {
    // selection anchors: no earlier selection, so the first one covers the whole radius
    std::vector<float4> anc((size_t)std::max(A, 1), make_float4(0.f, 0.f, INFINITY, 0.f));
    float4* p_anc;
    GD_TRY(upload(env, &p_anc, anc.data(), (size_t)A));
    d.anchor = p_anc;
  }
  // parked agents (the "all nontrivial" initialisation) keep their road
  // selection between steps (K key low words each)
  d.smemo = nullptr;
  if ((cfg->flags & GD_NONTRIVIAL_INIT) && K > 0) GD_TRY(dev_alloc(env, &d.smemo, (size_t)A * K));
  GD_TRY(cudaMemsetAsync(d.err, 0, sizeof(unsigned), env->stream));
  GD_TRY(cudaMallocHost(&env->h_err, sizeof(unsigned)));
  d.agent_off = p_aoff; d.road_off = p_roff; d.agent_world = p_aw; d.state = p_state; d.init_state = p_init;
  d.stat = p_stat; d.type = p_type; d.flags = p_flags; d.init_flags = p_iflags; d.t = p_t; d.world_done = p_wd;
  d.egrid = p_eg; d.ecell_start = p_ecs; d.esegs = p_es;
  if ((cfg->flags & GD_NONTRIVIAL_INIT) && A > 0) {
    k_mark_uncontrolled<<<blocks_for_host(A, 256), 256, 0, env->stream>>>(d, p_iflags, cfg->nontrivial_dist);
    GD_TRY(cudaGetLastError());
  }
  GD_TRY(allow_max_smem(reinterpret_cast<const void*>(k_observe<kObsWarpsDefault>)));
  // batched form: worlds largest first (agents, then road points), a work
  // counter, and a road tile sized for two CTAs per SM when every world fits,
  // else one CTA per SM with the largest tile
  {
    std::vector<int> order(W);
    for (int w = 0; w < W; ++w) order[w] = w;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
      const long cp = (long)(s->agent_off[p + 1] - s->agent_off[p]) * 65536 + (s->road_off[p + 1] - s->road_off[p]);
      const long cq = (long)(s->agent_off[q + 1] - s->agent_off[q]) * 65536 + (s->road_off[q + 1] - s->road_off[q]);
      return cp > cq;
    });
    GD_TRY(upload(env, &env->order, order.data(), (size_t)W));
    // k_world's work counter and exit tally (each launch leaves them at zero), the adjoint's counter
    GD_TRY(dev_alloc(env, &env->counter, 2));
    GD_TRY(cudaMemsetAsync(env->counter, 0, 2 * sizeof(unsigned), env->stream));
    GD_TRY(dev_alloc(env, &env->acounter, 2));
    GD_TRY(cudaMemsetAsync(env->acounter, 0, 2 * sizeof(unsigned), env->stream));
    GD_TRY(dev_alloc(env, &env->ocounter, 2 * OBS_STRIPES));
    if (cfg->flags & GD_BATCHED) {
      GD_TRY(dev_alloc(env, &env->alt_state, (size_t)A));
      GD_TRY(dev_alloc(env, &env->alt_flags, (size_t)A));
    }
  }
  if (cfg->flags & GD_DIFFERENTIABLE) {
    env->C = cfg->ckpt_every;
    env->n_ckpt = (cfg->episode_len + env->C - 1) / env->C;
    GD_TRY(dev_alloc(env, &env->ckS, (size_t)env->n_ckpt * A));
    GD_TRY(dev_alloc(env, &env->ckF, (size_t)env->n_ckpt * A));
    GD_TRY(dev_alloc(env, &env->ckT, (size_t)env->n_ckpt * W));
    GD_TRY(dev_alloc(env, &env->ckWD, (size_t)env->n_ckpt * W));
    GD_TRY(dev_alloc(env, &env->segS, (size_t)(env->C + 1) * A));
    GD_TRY(dev_alloc(env, &env->segF, (size_t)(env->C + 1) * A));
    GD_TRY(dev_alloc(env, &env->segT, (size_t)W));
    GD_TRY(dev_alloc(env, &env->segWD, (size_t)W));
    if (cfg->flags & GD_BATCHED) {
      GD_TRY(dev_alloc(env, &env->segS2, (size_t)(env->C + 1) * A));
      GD_TRY(dev_alloc(env, &env->segF2, (size_t)(env->C + 1) * A));
      GD_TRY(dev_alloc(env, &env->segT2, (size_t)W));
      GD_TRY(dev_alloc(env, &env->segWD2, (size_t)W));
    }
    GD_TRY(dev_alloc(env, &env->lam, (size_t)A));
    GD_TRY(dev_alloc(env, &env->adj_g, (size_t)env->C * A));
    GD_TRY(dev_alloc(env, &env->adj_cs, (size_t)env->C * A));
    GD_TRY(dev_alloc(env, &env->adj_slot, (size_t)env->C * A * GD_MAX_AGENTS_PER_WORLD));
    GD_TRY(dev_alloc(env, &env->adj_oc, ADJ_STRIPES));
    GD_TRY(cudaMemsetAsync(env->adj_oc, 0, ADJ_STRIPES * sizeof(unsigned), env->stream));
    // K-th road distances of the objective rollout; 0x7f7f7f7f (3.4e38) = no bound
    GD_TRY(dev_alloc(env, &env->rk_hist, (size_t)cfg->episode_len * A));
    GD_TRY(cudaMemsetAsync(env->rk_hist, 0x7f, sizeof(float) * (size_t)cfg->episode_len * A, env->stream));
    // the objective rollout's road selections, so that the backward pass
    // reads them instead of selecting again; without room for them it
    // re-selects (the same sets, so the same gradients)
    if (cfg->k_road > 0 && A > 0) {
      if (dev_alloc(env, &env->sel_hist, (size_t)cfg->episode_len * A * cfg->k_road) != cudaSuccess) {
        cudaGetLastError();
        env->sel_hist = nullptr;
      }
    }
    // the objective rollout's decisions (post-step flags), so that the
    // backward pass recomputes a segment's states in one launch instead of a
    // step launch per step; without room for them it runs the steps
    if (A > 0 && cfg->adjoint_recompute) {
      if (dev_alloc(env, &env->fl_hist, (size_t)cfg->episode_len * A) != cudaSuccess) {
        cudaGetLastError();
        env->fl_hist = nullptr;
      }
    }
  }
  if (cfg->block_size) env->warps = cfg->block_size / 32;
  env->split = cfg->obs_split;
  env->notile = cfg->road_no_tile;
  env->adj_notile = cfg->road_no_tile;
  env->adj_split = cfg->adjoint_split ? 1 : 0;
  env->d.topk = cfg->topk_strategy == 2 ? 2 : 1;
  if (cfg->lidar_rays > 0) {
    const int n = cfg->lidar_rays;
    const double fov = (double)cfg->lidar_fov;
    env->lidar_n = n;
    if (cfg->lidar_block_size) env->lw_warps = cfg->lidar_block_size / 32;
    env->lw_notile = cfg->lidar_no_tile;
    env->fan.n = n;
    env->fan.b0 = (float)(-0.5 * fov + 0.5 * fov / n);
    env->fan.inv_step = (float)(n / fov);
    env->fan.wrap_steps = (float)(6.283185307179586 * n / fov);
    GD_TRY(dev_alloc(env, &env->ray_dirs, (size_t)n));
    k_lidar_dirs<<<blocks_for_host(n, 256), 256, 0, env->stream>>>(env->ray_dirs, n, fov);
    GD_TRY(cudaGetLastError());
    int dev = 0, smem_blk = 0;
    GD_TRY(cudaGetDevice(&dev));
    GD_TRY(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    env->lw_split = cfg->lidar_split;
    GD_TRY(dev_alloc(env, &env->lcounter, 2 * LIDAR_STRIPES));
    GD_TRY(cudaMemsetAsync(env->lcounter, 0, 2 * LIDAR_STRIPES * sizeof(unsigned), env->stream));
    // stand-alone scan: groups of kLidarGroup warps, as many as fit one CTA
    constexpr int G = kLidarGroup;
    int groups = std::min(LIDAR_MAX_GROUPS, LidarGroupShape<G>::max_warps / G);
    while (groups > 1 && lidar_groups_smem(G, groups, n) + 1024 > (size_t)smem_blk) --groups;
    if (lidar_groups_smem(G, groups, n) + 1024 > (size_t)smem_blk) {
      gd_destroy(env);
      return fail(nullptr, GD_ERR_INVALID_ARG, "lidar_rays: the scan's keys and ray table do not fit shared memory");
    }
    env->lidar_groups = groups;
    int per_sm = 0, nsm = 0;
    GD_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    GD_TRY(allow_max_smem(reinterpret_cast<const void*>(k_lidar_group<G>)));
    GD_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lidar_group<G>, groups * G * 32,
                                                         lidar_groups_smem(G, groups, n)));
    env->lo_grid = std::max(1, std::min(std::max(per_sm, 1) * nsm, (A + groups - 1) / groups));
    // every claim counter that holds an agent needs a warp group
    env->lo_grid = std::max(env->lo_grid, (std::min(A, (int)LIDAR_STRIPES) + groups - 1) / groups);
  }
  GD_TRY(build_road(env, rcell));
  GD_TRY(cudaStreamSynchronize(env->stream));
#undef GD_TRY
  *out = env;
  return GD_OK;
}

gd_status gd_get_info(const gd_env* env, gd_info* info) {
  if (!env || !info) return GD_ERR_INVALID_ARG;
  info->num_worlds = env->W;
  info->num_agents = env->A;
  info->num_road = env->N;
  info->feat = env->F;
  info->max_agents_per_world = env->amax;
  info->k_road = env->cfg.k_road;
  info->n_partners = env->cfg.n_partners;
  info->episode_len = env->cfg.episode_len;
  info->device_bytes = env->bytes;
  info->block_size = env->warps * 32;
  info->road_tile = env->notile ? 0 : 1;
  info->road_cell = env->road_cell;
  info->topk_strategy = env->d.topk;
  info->lidar_rays = env->lidar_n;
  info->lidar_fov = env->cfg.lidar_fov;
  info->lidar_block_size = env->lw_warps * 32;
  info->lidar_road_tile = env->lw_notile ? 0 : 1;
  info->lidar_split = env->lw_split;
  info->obs_split = env->split;
  info->adjoint_split = env->adj_split;
  info->adjoint_road_tile = env->adj_notile ? 0 : 1;
  info->adjoint_recompute = env->fl_hist ? 1 : 0;
  info->objective_graph_kernels = env->ograph ? env->og_nodes[0] : 0;
  info->objective_graph_other = env->ograph ? env->og_nodes[1] : 0;
  info->backward_graph_kernels = env->bgraph ? env->bg_nodes[0] : 0;
  info->backward_graph_other = env->bgraph ? env->bg_nodes[1] : 0;
  return GD_OK;
}

static gd_status launch_check(gd_env* env, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(env, e, what);
  return GD_OK;
}

static inline unsigned blocks_for(long n, int per) { return (unsigned)std::max<long>(1, (n + per - 1) / per); }

gd_status gd_reset(gd_env* env, const uint8_t* world_mask) {
  NvtxRange range_("gd_reset");
  if (!env) return GD_ERR_INVALID_ARG;
  if (world_mask) {
    k_reset_worlds<<<blocks_for(env->W, 8), 256, 0, env->stream>>>(env->d, world_mask);
  } else {
    // every world: plain copies of the snapshot
    cudaMemcpyAsync(env->d.state, env->d.init_state, sizeof(float4) * env->A, cudaMemcpyDeviceToDevice, env->stream);
    cudaMemcpyAsync(env->d.flags, env->d.init_flags, env->A, cudaMemcpyDeviceToDevice, env->stream);
    cudaMemsetAsync(env->d.t, 0, sizeof(int) * env->W, env->stream);
    cudaMemsetAsync(env->d.world_done, 0, env->W, env->stream);
  }
  return launch_check(env, "gd_reset");
}

// Plain form: one launch per stage.
static void launch_step_plain(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done) {
  const DevEnv& d = env->d;
  cudaStream_t s = env->stream;
  if (d.cflags & GD_AUTO_RESET) k_reset_worlds<<<blocks_for(d.W, 8), 256, 0, s>>>(d, nullptr);
  k_dynamics<<<blocks_for(d.A, 256), 256, 0, s>>>(d, reinterpret_cast<const float2*>(actions));
  k_agent_grid<<<blocks_for(d.W, 8), 256, 0, s>>>(d);
  k_collide<<<blocks_for(d.A, 8), 256, 0, s>>>(d);
  k_offroad<<<blocks_for(d.A, 8), 256, 0, s>>>(d);
  k_finish<<<blocks_for(d.W, 8), 256, 0, s>>>(d, reward, done, world_done);
}

static void launch_observe(gd_env* env, float* obs, int32_t* road_idx, int32_t* partner_idx) {
  const DevEnv& d = env->d;
  constexpr int WARPS = kObsWarpsDefault;
  k_observe<WARPS><<<blocks_for(d.A, WARPS), WARPS * 32, WARPS * sizeof(ObsWarpSmem), env->stream>>>(
      d, obs, road_idx, partner_idx);
}

// Optional instrumentation of a host-issued sequence of launches: CUDA
// events around each launch, tagged with the launch's kind.
struct LaunchTimer {
  cudaStream_t stream = nullptr;
  std::vector<int> kind;
  std::vector<cudaEvent_t> ev;     // two per launch
  cudaError_t err = cudaSuccess;
  void begin(int k) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (err == cudaSuccess) err = cudaEventCreate(&a);
    if (err == cudaSuccess) err = cudaEventCreate(&b);
    if (err != cudaSuccess) return;
    kind.push_back(k);
    ev.push_back(a);
    ev.push_back(b);
    cudaEventRecord(a, stream);
  }
  void end() {
    if (err == cudaSuccess && !ev.empty()) cudaEventRecord(ev.back(), stream);
  }
  // Wait for the stream, then add each launch's time to ms[kind] and count
  // it in n[kind] (kinds below nk).
  cudaError_t collect(float* ms, int32_t* n, int nk) {
    cudaError_t e = err;
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    for (size_t q = 0; q < kind.size() && e == cudaSuccess; ++q) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]);
      if (e == cudaSuccess && kind[q] < nk) {
        ms[kind[q]] += t;
        n[kind[q]] += 1;
      }
    }
    return e;
  }
  ~LaunchTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};
static void tbegin(LaunchTimer* tm, int k) { if (tm) tm->begin(k); }
static void tend(LaunchTimer* tm) { if (tm) tm->end(); }

// The split observation launch: the form that keeps the parked agents' road
// selections between steps when the env has such agents (its own
// instantiation, so that the other form's code is the same without them).
extern "C++" {
template <bool LOSS>
static void launch_observe_split(gd_env* env, const DevEnv& dv, float* obs, int32_t* road_idx, int32_t* partner_idx,
                                 unsigned* counters, const SplitLoss& loss, cudaStream_t stream) {
  if (dv.smemo)
    k_observe_split<kSplitWarps, LOSS, true><<<env->so_grid, kSplitWarps * 32, kSplitSmem, stream>>>(
        dv, obs, road_idx, partner_idx, counters, loss);
  else
    k_observe_split<kSplitWarps, LOSS><<<env->so_grid, kSplitWarps * 32, kSplitSmem, stream>>>(
        dv, obs, road_idx, partner_idx, counters, loss);
}
}  // extern "C++"

// Batched form: one persistent launch (its work counter was left at zero by the previous one).
// With env->split, an observation without the objective is the step launch
// (nothing observed) followed by k_observe_split over all agents.
static void launch_world(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done,
                         float* obs, int32_t* road_idx, int32_t* partner_idx, int do_step,
                         cudaStream_t stream = nullptr, const DevEnv* dv = nullptr, const float* obs_w = nullptr,
                         float reward_w = 0.f, float* ell = nullptr, float* rk_out = nullptr,
                         unsigned* clear = nullptr, int clear_n = (int)OBS_STRIPES, float4* state_out = nullptr,
                         uint8_t* flags_out = nullptr, LaunchTimer* tm = nullptr, uint16_t* sel_out = nullptr,
                         uint8_t* flags_rec = nullptr) {
  if (!stream) stream = env->stream;
  if (!dv) dv = &env->d;
  if (obs && env->split && (!ell || do_step)) {
    // split form: the step over worlds, then the observation over agents
    // (with the objective: the step writes r_s to ell, the observation
    // completes it)
    // the step launch clears the observation counters; without a step, a memset does
    if (do_step)
      launch_world(env, actions, reward, done, world_done, nullptr, nullptr, nullptr, 1, stream, dv, nullptr, 0.f, ell,
                   nullptr, env->ocounter, (int)OBS_STRIPES, nullptr, nullptr, tm, nullptr, flags_rec);
    else
      cudaMemsetAsync(env->ocounter, 0, OBS_STRIPES * sizeof(unsigned), stream);
    const SplitLoss loss{obs_w, reward_w, ell, rk_out, sel_out};
    tbegin(tm, 2);
    if (ell)
      launch_observe_split<true>(env, *dv, obs, road_idx, partner_idx, env->ocounter, loss, stream);
    else
      launch_observe_split<false>(env, *dv, obs, road_idx, partner_idx, env->ocounter, loss, stream);
    tend(tm);
    return;
  }
  FusedArgs a{};
  a.actions = reinterpret_cast<const float2*>(actions);
  a.reward = reward;
  a.done = done;
  a.world_done = world_done;
  a.obs = obs;
  a.road_idx = road_idx;
  a.partner_idx = partner_idx;
  a.counter = env->counter;
  a.order = env->order;
  a.tile_bytes = env->tile_cap;
  a.do_step = do_step;
  a.obs_w = obs_w;
  a.reward_w = reward_w;
  a.ell = ell;
  a.rk_out = (ell && obs) ? rk_out : nullptr;
  a.sel_out = (ell && obs) ? sel_out : nullptr;
  a.clear = clear;
  a.clear_n = clear ? clear_n : 0;
  a.state_out = state_out;
  a.flags_out = flags_out;
  a.flags_rec = do_step ? flags_rec : nullptr;
  const bool step_only = obs == nullptr;
  const dim3 grid(step_only ? env->step_grid : env->world_grid);
  const size_t smem = step_only ? env->step_smem : env->world_smem;
  tbegin(tm, step_only ? 1 : 2);
  struct EndTimer {
    LaunchTimer* t;
    ~EndTimer() { tend(t); }
  } end_timer_{tm};
  if (env->notile || step_only) {
    switch (env->warps) {
      case 4: k_world<4, false, true><<<grid, 4 * 32, smem, stream>>>(*dv, a); break;
      case 16: k_world<16, false, true><<<grid, 16 * 32, smem, stream>>>(*dv, a); break;
      default: k_world<8, false, true><<<grid, 8 * 32, smem, stream>>>(*dv, a); break;
    }
  } else {
    switch (env->warps) {
      case 4: k_world<4><<<grid, 4 * 32, smem, stream>>>(*dv, a); break;
      case 16: k_world<16><<<grid, 16 * 32, smem, stream>>>(*dv, a); break;
      default: k_world<8><<<grid, 8 * 32, smem, stream>>>(*dv, a); break;
    }
  }
}

static LidarArgs lidar_args(const gd_env* env, const float* head, float* depth, uint8_t* cls) {
  LidarArgs la{};
  la.head = head;
  la.depth = depth;
  la.cls = cls;
  la.dirs = env->ray_dirs;
  la.lsegs = env->d.lsegs;
  la.lcell = env->d.lcell;
  la.fan = env->fan;
  la.warp_bytes = (int)lidar_warp_bytes(env->lidar_n);
  return la;
}

// Stand-alone LiDAR scan of every agent: persistent CTAs, warps take agents
// from a counter (cleared first); the scene is read from global memory.
// `cleared`: the launch before it (the split form's step) already cleared
// the agent counter.
static void launch_lidar(gd_env* env, const float* head, float* depth, uint8_t* cls, cudaStream_t stream = nullptr,
                         bool cleared = false) {
  if (!stream) stream = env->stream;
  const LidarArgs la = lidar_args(env, head, depth, cls);
  const int groups = env->lidar_groups;
  if (!cleared) cudaMemsetAsync(env->lcounter, 0, LIDAR_STRIPES * sizeof(unsigned), stream);
  k_lidar_group<kLidarGroup><<<env->lo_grid, groups * kLidarGroup * 32,
                               lidar_groups_smem(kLidarGroup, groups, env->lidar_n), stream>>>(env->d, la, env->lcounter);
}

// Fused LiDAR form: one persistent launch of the step (if do_step) and the
// LiDAR scan of every world.
static void launch_world_lidar(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done,
                               const float* head, float* depth, uint8_t* cls, int do_step,
                               cudaStream_t stream = nullptr) {
  if (!stream) stream = env->stream;
  if (env->lw_split) {
    // split form: the fused step without observation, then the stand-alone scan
    // the step launch clears the scan's agent counter
    if (do_step)
      launch_world(env, actions, reward, done, world_done, nullptr, nullptr, nullptr, 1, stream, nullptr, nullptr, 0.f,
                   nullptr, nullptr, env->lcounter, (int)LIDAR_STRIPES);
    launch_lidar(env, head, depth, cls, stream, do_step != 0);
    return;
  }
  FusedArgs a{};
  a.actions = reinterpret_cast<const float2*>(actions);
  a.reward = reward;
  a.done = done;
  a.world_done = world_done;
  a.counter = env->counter;
  a.order = env->order;
  a.tile_bytes = env->lw_tile;
  a.do_step = do_step;
  a.lidar = lidar_args(env, head, depth, cls);
  switch (env->lw_warps) {
    case 4: k_world<4, true><<<env->lw_grid, 4 * 32, env->lw_smem, stream>>>(env->d, a); break;
    case 12: k_world<12, true><<<env->lw_grid, 12 * 32, env->lw_smem, stream>>>(env->d, a); break;
    default: k_world<8, true><<<env->lw_grid, 8 * 32, env->lw_smem, stream>>>(env->d, a); break;
  }
}

static bool batched(const gd_env* env) { return (env->cfg.flags & GD_BATCHED) != 0; }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

gd_status gd_step(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done) {
  NvtxRange range_("gd_step");
  if (!env) return GD_ERR_INVALID_ARG;
  if (!actions && env->A > 0) return fail(env, GD_ERR_INVALID_ARG, "actions must not be NULL");
  if (!aligned16(actions) && ((uintptr_t)actions & 7u)) return fail(env, GD_ERR_INVALID_ARG, "actions must be 8-byte aligned");
  if (batched(env)) {
    if (env->A > 0 || env->W > 0) launch_world(env, actions, reward, done, world_done, nullptr, nullptr, nullptr, 1);
  } else {
    launch_step_plain(env, actions, reward, done, world_done);
  }
  return launch_check(env, "gd_step");
}

gd_status gd_observe(gd_env* env, float* obs, int32_t* road_idx, int32_t* partner_idx) {
  NvtxRange range_("gd_observe");
  if (!env) return GD_ERR_INVALID_ARG;
  if (!obs && env->A > 0) return fail(env, GD_ERR_INVALID_ARG, "obs must not be NULL");
  if (!aligned16(obs)) return fail(env, GD_ERR_INVALID_ARG, "obs must be 16-byte aligned");
  if (env->A == 0) return GD_OK;
  if (batched(env)) launch_world(env, nullptr, nullptr, nullptr, nullptr, obs, road_idx, partner_idx, 0);
  else launch_observe(env, obs, road_idx, partner_idx);
  return launch_check(env, "gd_observe");
}

gd_status gd_step_observe(gd_env* env, const float* actions, float* reward, uint8_t* done, uint8_t* world_done,
                          float* obs) {
  NvtxRange range_("gd_step_observe");
  if (env && batched(env)) {
    if (!actions && env->A > 0) return fail(env, GD_ERR_INVALID_ARG, "actions must not be NULL");
    if (!obs && env->A > 0) return fail(env, GD_ERR_INVALID_ARG, "obs must not be NULL");
    if (!aligned16(obs)) return fail(env, GD_ERR_INVALID_ARG, "obs must be 16-byte aligned");
    launch_world(env, actions, reward, done, world_done, obs, nullptr, nullptr, 1);
    return launch_check(env, "gd_step_observe");
  }
  gd_status st = gd_step(env, actions, reward, done, world_done);
  if (st != GD_OK) return st;
  return gd_observe(env, obs, nullptr, nullptr);
}

// Copy (state, flags, t, episode-end status) between the env and a slot: one
// launch of k_copy_snapshot.
static void copy_snapshot(gd_env* env, float4* dS, uint8_t* dF, int* dT, uint8_t* dWD, const float4* sS,
                          const uint8_t* sF, const int* sT, const uint8_t* sWD, cudaStream_t stream = nullptr) {
  if (!stream) stream = env->stream;
  const Snapshot dst{dS, dF, dT, dWD};
  const Snapshot src{const_cast<float4*>(sS), const_cast<uint8_t*>(sF), const_cast<int*>(sT),
                     const_cast<uint8_t*>(sWD)};
  const int n = std::max(env->A, env->W);
  k_copy_snapshot<<<std::min(blocks_for(n, 256), 1184u), 256, 0, stream>>>(dst, src, env->A, env->W);
}

#ifndef GD_ROLLOUT_OVERLAP
#define GD_ROLLOUT_OVERLAP 1
#endif

// The step launch of the split form (no observation) on explicit state
// buffers, optionally as a programmatic dependent of the launch before it.
static cudaError_t launch_step_ex(gd_env* env, const DevEnv& dv, const FusedArgs& a, cudaStream_t stream, bool pdl) {
  cudaLaunchConfig_t lc{};
  lc.gridDim = dim3(env->step_grid);
  lc.blockDim = dim3(env->warps * 32);
  lc.dynamicSmemBytes = env->step_smem;
  lc.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = pdl ? 1 : 0;
  switch (env->warps) {
    case 4: return cudaLaunchKernelEx(&lc, k_world<4, false, true>, dv, a);
    case 16: return cudaLaunchKernelEx(&lc, k_world<16, false, true>, dv, a);
    default: return cudaLaunchKernelEx(&lc, k_world<8, false, true>, dv, a);
  }
}

// Overlapped split rollout: the state and flags alternate between the env's
// buffers and a second pair, so that step t + 1 (which reads step t's
// output and writes the other pair) may run beside observation t (which
// reads step t's output); step t + 1 is a programmatic dependent of
// observation t and finishes only after it, and the observation counters
// alternate between two sets.  The last of the rollout's `steps` steps
// writes the env's own buffers.  Issues steps [t0, t1) (t1 <= steps); the
// first of them is an ordinary launch (it may follow other work).
// With obs_w, the objective rollout: step t writes each agent's smooth
// reward into ell[t], observation t completes it and records the K-th road
// distances, and every ckpt_every steps a copy launch saves the state step
// t reads as a checkpoint (the step after a copy is an ordinary launch).
static void issue_rollout_overlapped(gd_env* env, int steps, int t0, int t1, const float* actions, float* obs,
                                     int obs_per_step, float* reward, uint8_t* done, cudaStream_t stream,
                                     const float* obs_w = nullptr, float reward_w = 0.f, float* ell = nullptr) {
  const size_t A = (size_t)env->A, W = (size_t)env->W;
  float4* sbuf[2] = {env->d.state, env->alt_state};
  uint8_t* fbuf[2] = {env->d.flags, env->alt_flags};
  // the buffer step t reads: the env's own before the first step, else the
  // one step t - 1 wrote
  int in = t0 == 0 ? 0 : (((steps - t0) & 1) ? 1 : 0);
  for (int t = t0; t < t1; ++t) {
    const int out = ((steps - 1 - t) & 1) ? 1 : 0;
    unsigned* oc = env->ocounter + (size_t)(t & 1) * OBS_STRIPES;
    const bool ckpt = ell && t % env->C == 0;
    if (ckpt) {
      const int c = t / env->C;
      copy_snapshot(env, env->ckS + c * A, env->ckF + c * A, env->ckT + c * W, env->ckWD + c * W, sbuf[in], fbuf[in],
                    env->d.t, env->d.world_done, stream);
    }
    DevEnv dv = env->d;
    dv.state = sbuf[in];
    dv.flags = fbuf[in];
    FusedArgs a{};
    a.actions = reinterpret_cast<const float2*>(actions + (size_t)t * A * 2);
    a.reward = reward ? reward + (size_t)t * A : nullptr;
    a.done = done ? done + (size_t)t * A : nullptr;
    a.counter = env->counter;
    a.order = env->order;
    a.tile_bytes = env->tile_cap;
    a.do_step = 1;
    a.clear = oc;
    a.clear_n = (int)OBS_STRIPES;
    a.state_out = out == in ? nullptr : sbuf[out];
    a.flags_out = out == in ? nullptr : fbuf[out];
    a.ell = ell ? ell + (size_t)t * A : nullptr;
    // the objective rollout records its decisions for the backward pass
    if (ell && env->fl_hist) a.flags_rec = env->fl_hist + (size_t)t * A;
    launch_step_ex(env, dv, a, stream, t > t0 && !ckpt);
    DevEnv dvo = env->d;
    dvo.state = sbuf[out];
    dvo.flags = fbuf[out];
    float* orow = obs + (obs_per_step ? (size_t)t * A * env->F : 0);
    if (ell) {
      const SplitLoss loss{obs_w, reward_w, ell + (size_t)t * A, env->rk_hist + (size_t)t * A,
                           env->sel_hist ? env->sel_hist + (size_t)t * A * env->d.K : nullptr};
      launch_observe_split<true>(env, dvo, orow, nullptr, nullptr, oc, loss, stream);
    } else {
      const SplitLoss loss{nullptr, 0.f, nullptr, nullptr, nullptr};
      launch_observe_split<false>(env, dvo, orow, nullptr, nullptr, oc, loss, stream);
    }
    in = out;
  }
}

// The split LiDAR rollout overlapped like issue_rollout_overlapped: the
// state and flags alternate between two buffers (the last step leaves them
// in the env's own), the step launch of t + 1 is a programmatic dependent of
// scan t (it starts in that launch's tail and ends only after it), and the
// scan's claim counters alternate between two sets.
static void issue_lidar_overlapped(gd_env* env, int steps, const float* actions, const float* head, float* depth,
                                   uint8_t* cls, int obs_per_step, float* reward, uint8_t* done, cudaStream_t stream) {
  const size_t A = (size_t)env->A, n = (size_t)env->lidar_n;
  float4* sbuf[2] = {env->d.state, env->alt_state};
  uint8_t* fbuf[2] = {env->d.flags, env->alt_flags};
  const int groups = env->lidar_groups;
  int in = 0;
  for (int t = 0; t < steps; ++t) {
    const int out = ((steps - 1 - t) & 1) ? 1 : 0;
    unsigned* lc = env->lcounter + (size_t)(t & 1) * LIDAR_STRIPES;
    DevEnv dv = env->d;
    dv.state = sbuf[in];
    dv.flags = fbuf[in];
    FusedArgs a{};
    a.actions = reinterpret_cast<const float2*>(actions + (size_t)t * A * 2);
    a.reward = reward ? reward + (size_t)t * A : nullptr;
    a.done = done ? done + (size_t)t * A : nullptr;
    a.counter = env->counter;
    a.order = env->order;
    a.tile_bytes = env->tile_cap;
    a.do_step = 1;
    a.clear = lc;
    a.clear_n = (int)LIDAR_STRIPES;
    a.state_out = out == in ? nullptr : sbuf[out];
    a.flags_out = out == in ? nullptr : fbuf[out];
    launch_step_ex(env, dv, a, stream, t > 0);
    DevEnv dvo = env->d;
    dvo.state = sbuf[out];
    dvo.flags = fbuf[out];
    const LidarArgs la = lidar_args(env, head ? head + (size_t)t * A : nullptr,
                                    depth + (obs_per_step ? (size_t)t * A * n : 0),
                                    cls ? cls + (obs_per_step ? (size_t)t * A * n : 0) : nullptr);
    k_lidar_group<kLidarGroup><<<env->lo_grid, groups * kLidarGroup * 32,
                                 lidar_groups_smem(kLidarGroup, groups, env->lidar_n), stream>>>(dvo, la, lc);
    in = out;
  }
}

gd_status gd_rollout(gd_env* env, int32_t steps, const float* actions, float* obs, int32_t obs_per_step, float* reward,
                     uint8_t* done) {
  NvtxRange range_("gd_rollout");
  if (!env) return GD_ERR_INVALID_ARG;
  if (steps < 0) return fail(env, GD_ERR_INVALID_ARG, "steps must be >= 0");
  if (steps == 0 || env->A == 0) return GD_OK;
  if (!actions || !obs) return fail(env, GD_ERR_INVALID_ARG, "actions and obs must not be NULL");
  if (!aligned16(obs)) return fail(env, GD_ERR_INVALID_ARG, "obs must be 16-byte aligned");
  const size_t A = (size_t)env->A;
  if (!batched(env)) {
    // per-stage form: launches issued from the host, one step at a time
    for (int t = 0; t < steps; ++t) {
      gd_status st = gd_step(env, actions + (size_t)t * A * 2, reward ? reward + (size_t)t * A : nullptr,
                             done ? done + (size_t)t * A : nullptr, nullptr);
      if (st != GD_OK) return st;
      st = gd_observe(env, obs + (obs_per_step ? (size_t)t * A * env->F : 0), nullptr, nullptr);
      if (st != GD_OK) return st;
    }
    return GD_OK;
  }
  // batched form: the whole rollout is one CUDA graph (T fused launches),
  // captured on a private stream and re-used while the arguments are the same
  const void* key[6] = {actions, obs, reward, done, (const void*)(intptr_t)(obs_per_step != 0), nullptr};
  bool same = env->graph && env->g_steps == steps;
  for (int k = 0; k < 6 && same; ++k) same = env->g_key[k] == key[k];
  if (!same) {
    if (env->graph) {
      cudaGraphExecDestroy(env->graph);
      env->graph = nullptr;
    }
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout: capture stream");
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(env, e, "gd_rollout: begin capture");
    }
    if (GD_ROLLOUT_OVERLAP && env->split)
      issue_rollout_overlapped(env, steps, 0, steps, actions, obs, obs_per_step, reward, done, cap);
    else
      for (int t = 0; t < steps; ++t)
        launch_world(env, actions + (size_t)t * A * 2, reward ? reward + (size_t)t * A : nullptr,
                     done ? done + (size_t)t * A : nullptr, nullptr,
                     obs + (obs_per_step ? (size_t)t * A * env->F : 0), nullptr, nullptr, 1, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout: end capture");
    e = cudaGraphInstantiate(&env->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      env->graph = nullptr;
      return cuda_fail(env, e, "gd_rollout: instantiate");
    }
    for (int k = 0; k < 6; ++k) env->g_key[k] = key[k];
    env->g_steps = steps;
  }
  cudaError_t e = cudaGraphLaunch(env->graph, env->stream);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout: graph launch");
  return GD_OK;
}

// ---- rollout on host buffers ----------------------------------------------------

static bool page_locked(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

constexpr int kHostChunk = 8;   // steps per copy chunk of gd_rollout_host

gd_status gd_rollout_host(gd_env* env, int32_t steps, const float* actions_host, float* obs, float* reward_host,
                          uint8_t* done_host) {
  NvtxRange range_("gd_rollout_host");
  if (!env) return GD_ERR_INVALID_ARG;
  if (!batched(env)) return fail(env, GD_ERR_STATE, "gd_rollout_host needs GD_BATCHED");
  if (steps < 0) return fail(env, GD_ERR_INVALID_ARG, "steps must be >= 0");
  if (steps == 0 || env->A == 0) return GD_OK;
  if (!actions_host || !obs) return fail(env, GD_ERR_INVALID_ARG, "actions_host and obs must not be NULL");
  if (!aligned16(obs)) return fail(env, GD_ERR_INVALID_ARG, "obs must be 16-byte aligned");
  if (!page_locked(actions_host) || (reward_host && !page_locked(reward_host)) || (done_host && !page_locked(done_host)))
    return fail(env, GD_ERR_INVALID_ARG, "host buffers must be page-locked (cudaHostAlloc / pinned)");
  const size_t A = (size_t)env->A;
  cudaError_t e = cudaSuccess;
  if (env->hs_cap < steps) {
    dev_free(env, env->hs_act);
    dev_free(env, env->hs_rew);
    dev_free(env, env->hs_done);
    env->hs_act = nullptr;
    env->hs_rew = nullptr;
    env->hs_done = nullptr;
    env->hs_cap = 0;
    e = dev_alloc(env, &env->hs_act, (size_t)steps * A * 2);
    if (e == cudaSuccess) e = dev_alloc(env, &env->hs_rew, (size_t)steps * A);
    if (e == cudaSuccess) e = dev_alloc(env, &env->hs_done, (size_t)steps * A);
    if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_host: staging");
    env->hs_cap = steps;
    if (env->hgraph) {
      cudaGraphExecDestroy(env->hgraph);
      env->hgraph = nullptr;
    }
  }
  const void* key[4] = {actions_host, obs, reward_host, done_host};
  bool same = env->hgraph && env->hg_steps == steps;
  for (int k = 0; k < 4 && same; ++k) same = env->hg_key[k] == key[k];
  if (!same) {
    if (env->hgraph) {
      cudaGraphExecDestroy(env->hgraph);
      env->hgraph = nullptr;
    }
    // capture: compute on stream cs, copies in on stream ci (all chunks in
    // order, none waiting for compute), copies out on stream co (chunk c
    // after its steps): the steps of chunk c wait only for its own copy in,
    // and its copy out overlaps the steps of chunk c + 1
    cudaStream_t cs = nullptr, ci = nullptr, co = nullptr;
    std::vector<cudaEvent_t> evs;
    auto event = [&]() {
      cudaEvent_t ev = nullptr;
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) evs.push_back(ev);
      return ev;
    };
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ci, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&co, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
      cudaEvent_t fork = event();
      cudaEventRecord(fork, cs);
      cudaStreamWaitEvent(ci, fork, 0);
      cudaStreamWaitEvent(co, fork, 0);
      std::vector<cudaEvent_t> in_done;
      for (int t0 = 0; t0 < steps; t0 += kHostChunk) {
        const int n = std::min(kHostChunk, steps - t0);
        cudaMemcpyAsync(env->hs_act + (size_t)t0 * A * 2, actions_host + (size_t)t0 * A * 2,
                        sizeof(float) * 2 * A * (size_t)n, cudaMemcpyHostToDevice, ci);
        cudaEvent_t in = event();
        cudaEventRecord(in, ci);
        in_done.push_back(in);
      }
      int c = 0;
      for (int t0 = 0; t0 < steps; t0 += kHostChunk, ++c) {
        const int n = std::min(kHostChunk, steps - t0);
        cudaStreamWaitEvent(cs, in_done[(size_t)c], 0);
        if (GD_ROLLOUT_OVERLAP && env->split)
          issue_rollout_overlapped(env, steps, t0, t0 + n, env->hs_act, obs, 0, env->hs_rew, env->hs_done, cs);
        else
          for (int t = t0; t < t0 + n; ++t)
            launch_world(env, env->hs_act + (size_t)t * A * 2, env->hs_rew + (size_t)t * A,
                         env->hs_done + (size_t)t * A, nullptr, obs, nullptr, nullptr, 1, cs);
        cudaEvent_t out = event();
        cudaEventRecord(out, cs);
        cudaStreamWaitEvent(co, out, 0);
        if (reward_host)
          cudaMemcpyAsync(reward_host + (size_t)t0 * A, env->hs_rew + (size_t)t0 * A, sizeof(float) * A * (size_t)n,
                          cudaMemcpyDeviceToHost, co);
        if (done_host)
          cudaMemcpyAsync(done_host + (size_t)t0 * A, env->hs_done + (size_t)t0 * A, A * (size_t)n,
                          cudaMemcpyDeviceToHost, co);
      }
      cudaEvent_t join_i = event(), join_o = event();
      cudaEventRecord(join_i, ci);
      cudaEventRecord(join_o, co);
      cudaStreamWaitEvent(cs, join_i, 0);
      cudaStreamWaitEvent(cs, join_o, 0);
      e = cudaStreamEndCapture(cs, &g);
    }
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (co) cudaStreamDestroy(co);
    if (ci) cudaStreamDestroy(ci);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(env, e, "gd_rollout_host: capture");
    }
    e = cudaGraphInstantiate(&env->hgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      env->hgraph = nullptr;
      return cuda_fail(env, e, "gd_rollout_host: instantiate");
    }
    for (int k = 0; k < 4; ++k) env->hg_key[k] = key[k];
    env->hg_steps = steps;
  }
  e = cudaGraphLaunch(env->hgraph, env->stream);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_host: graph launch");
  return GD_OK;
}

// ---- LiDAR / view cone -------------------------------------------------------

static gd_status need_lidar(gd_env* env, const char* what) {
  if (env->lidar_n <= 0) return fail(env, GD_ERR_STATE, std::string(what) + ": the env was created with lidar_rays = 0");
  return GD_OK;
}

static bool aligned4(const void* p) { return ((uintptr_t)p & 3u) == 0; }

gd_status gd_observe_lidar(gd_env* env, const float* head, float* depth, uint8_t* cls) {
  NvtxRange range_("gd_observe_lidar");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_lidar(env, "gd_observe_lidar");
  if (st != GD_OK) return st;
  if (!depth && env->A > 0) return fail(env, GD_ERR_INVALID_ARG, "depth must not be NULL");
  if (!aligned4(depth) || !aligned4(head)) return fail(env, GD_ERR_INVALID_ARG, "depth and head must be 4-byte aligned");
  if (env->A == 0) return GD_OK;
  if (batched(env)) launch_world_lidar(env, nullptr, nullptr, nullptr, nullptr, head, depth, cls, 0);
  else launch_lidar(env, head, depth, cls);
  return launch_check(env, "gd_observe_lidar");
}

gd_status gd_step_observe_lidar(gd_env* env, const float* actions, const float* head, float* reward, uint8_t* done,
                                uint8_t* world_done, float* depth, uint8_t* cls) {
  NvtxRange range_("gd_step_observe_lidar");
  if (!env) return GD_ERR_INVALID_ARG;
  if (batched(env)) {
    gd_status st = need_lidar(env, "gd_step_observe_lidar");
    if (st != GD_OK) return st;
    if ((!actions || !depth) && env->A > 0) return fail(env, GD_ERR_INVALID_ARG, "actions and depth must not be NULL");
    if (((uintptr_t)actions & 7u) || !aligned4(depth) || !aligned4(head))
      return fail(env, GD_ERR_INVALID_ARG, "actions must be 8-byte, depth and head 4-byte aligned");
    launch_world_lidar(env, actions, reward, done, world_done, head, depth, cls, 1);
    return launch_check(env, "gd_step_observe_lidar");
  }
  gd_status st = need_lidar(env, "gd_step_observe_lidar");
  if (st != GD_OK) return st;
  st = gd_step(env, actions, reward, done, world_done);
  if (st != GD_OK) return st;
  return gd_observe_lidar(env, head, depth, cls);
}

gd_status gd_rollout_lidar(gd_env* env, int32_t steps, const float* actions, const float* head, float* depth,
                           uint8_t* cls, int32_t obs_per_step, float* reward, uint8_t* done) {
  NvtxRange range_("gd_rollout_lidar");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_lidar(env, "gd_rollout_lidar");
  if (st != GD_OK) return st;
  if (steps < 0) return fail(env, GD_ERR_INVALID_ARG, "steps must be >= 0");
  if (steps == 0 || env->A == 0) return GD_OK;
  if (!actions || !depth) return fail(env, GD_ERR_INVALID_ARG, "actions and depth must not be NULL");
  if (((uintptr_t)actions & 7u) || !aligned4(depth) || !aligned4(head))
    return fail(env, GD_ERR_INVALID_ARG, "actions must be 8-byte, depth and head 4-byte aligned");
  const size_t A = (size_t)env->A, n = (size_t)env->lidar_n;
  auto dstep = [&](int t) { return depth + (obs_per_step ? (size_t)t * A * n : 0); };
  auto cstep = [&](int t) { return cls ? cls + (obs_per_step ? (size_t)t * A * n : 0) : nullptr; };
  auto hstep = [&](int t) { return head ? head + (size_t)t * A : nullptr; };
  if (!batched(env)) {
    for (int t = 0; t < steps; ++t) {
      st = gd_step(env, actions + (size_t)t * A * 2, reward ? reward + (size_t)t * A : nullptr,
                   done ? done + (size_t)t * A : nullptr, nullptr);
      if (st != GD_OK) return st;
      st = gd_observe_lidar(env, hstep(t), dstep(t), cstep(t));
      if (st != GD_OK) return st;
    }
    return GD_OK;
  }
  const void* key[8] = {actions, head, depth, cls, reward, done, (const void*)(intptr_t)(obs_per_step != 0), nullptr};
  bool same = env->lgraph && env->lg_steps == steps;
  for (int k = 0; k < 8 && same; ++k) same = env->lg_key[k] == key[k];
  if (!same) {
    if (env->lgraph) {
      cudaGraphExecDestroy(env->lgraph);
      env->lgraph = nullptr;
    }
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_lidar: capture stream");
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(env, e, "gd_rollout_lidar: begin capture");
    }
    if (GD_ROLLOUT_OVERLAP && env->lw_split)
      issue_lidar_overlapped(env, steps, actions, head, depth, cls, obs_per_step, reward, done, cap);
    else
      for (int t = 0; t < steps; ++t)
        launch_world_lidar(env, actions + (size_t)t * A * 2, reward ? reward + (size_t)t * A : nullptr,
                           done ? done + (size_t)t * A : nullptr, nullptr, hstep(t), dstep(t), cstep(t), 1, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_lidar: end capture");
    e = cudaGraphInstantiate(&env->lgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      env->lgraph = nullptr;
      return cuda_fail(env, e, "gd_rollout_lidar: instantiate");
    }
    for (int k = 0; k < 8; ++k) env->lg_key[k] = key[k];
    env->lg_steps = steps;
  }
  cudaError_t e = cudaGraphLaunch(env->lgraph, env->stream);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_lidar: graph launch");
  return GD_OK;
}

// ---- episode statistics -------------------------------------------------------

// Warp per world: counts of the agents in the scene, the controlled agents in
// the scene, and the agents whose goal, collision and off-road flags are set.
__global__ void k_episode_stats(DevEnv e, int32_t* __restrict__ per_world, unsigned long long* __restrict__ totals) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= e.W) return;
  int c[GD_STATS] = {0, 0, 0, 0, 0};
  for (int i = e.agent_off[w] + lane; i < e.agent_off[w + 1]; i += WARP) {
    const uint8_t f = e.flags[i];
    c[0] += !(f & GD_FLAG_DONE);
    c[1] += !(f & (GD_FLAG_DONE | GD_FLAG_STATIC));
    c[2] += (f & GD_FLAG_GOAL) != 0;
    c[3] += (f & GD_FLAG_COLLIDED) != 0;
    c[4] += (f & GD_FLAG_OFFROAD) != 0;
  }
#pragma unroll
  for (int k = 0; k < GD_STATS; ++k)
    for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
  if (lane < GD_STATS) {
    const int v = c[0] * (lane == 0) + c[1] * (lane == 1) + c[2] * (lane == 2) + c[3] * (lane == 3) + c[4] * (lane == 4);
    if (per_world) per_world[(size_t)w * GD_STATS + lane] = v;
    if (totals && v) atomicAdd(totals + lane, (unsigned long long)v);
  }
}

gd_status gd_episode_stats(gd_env* env, int32_t* per_world, int64_t* totals) {
  if (!env) return GD_ERR_INVALID_ARG;
  if (!per_world && !totals) return fail(env, GD_ERR_INVALID_ARG, "per_world and totals are both NULL");
  if (((uintptr_t)per_world & 3u) || ((uintptr_t)totals & 7u))
    return fail(env, GD_ERR_INVALID_ARG, "per_world must be 4-byte and totals 8-byte aligned");
  if (totals) cudaMemsetAsync(totals, 0, sizeof(int64_t) * GD_STATS, env->stream);
  k_episode_stats<<<blocks_for(env->W, 8), 256, 0, env->stream>>>(env->d, per_world,
                                                                  reinterpret_cast<unsigned long long*>(totals));
  return launch_check(env, "gd_episode_stats");
}

// ---- expert-action inversion -------------------------------------------------

gd_status gd_invert_actions(gd_env* env, int32_t steps, const float* states, float* actions) {
  NvtxRange range_("gd_invert_actions");
  if (!env) return GD_ERR_INVALID_ARG;
  if (steps < 0) return fail(env, GD_ERR_INVALID_ARG, "steps must be >= 0");
  if (steps == 0 || env->A == 0) return GD_OK;
  if (!states || !actions) return fail(env, GD_ERR_INVALID_ARG, "states and actions must not be NULL");
  if (!aligned16(states) || ((uintptr_t)actions & 7u))
    return fail(env, GD_ERR_INVALID_ARG, "states must be 16-byte and actions 8-byte aligned");
  const dim3 grid((unsigned)((env->A + 255) / 256), (unsigned)((steps + INV_CHUNK - 1) / INV_CHUNK));
  k_invert<<<grid, 256, 0, env->stream>>>(env->d, steps, reinterpret_cast<const float4*>(states),
                                         reinterpret_cast<float2*>(actions));
  return launch_check(env, "gd_invert_actions");
}

// ---- differentiable rollouts ------------------------------------------------

static gd_status need_diff(gd_env* env, const char* what) {
  if (!(env->cfg.flags & GD_DIFFERENTIABLE))
    return fail(env, GD_ERR_STATE, std::string(what) + ": the env was not created with GD_DIFFERENTIABLE");
  return GD_OK;
}


// Capture what `issue(stream)` launches on a private stream into *out (an
// existing graph is replaced).
extern "C++" {
namespace {
// Capture what `issue(stream)` launches; nodes[0] / nodes[1] receive the
// graph's kernel nodes / other nodes (copies, memsets, ...) when given.
template <typename Fn>
gd_status capture_graph(gd_env* env, cudaGraphExec_t* out, const char* what, Fn&& issue, int* nodes = nullptr) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  cudaStream_t cap = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(env, e, what);
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    return cuda_fail(env, e, what);
  }
  issue(cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return cuda_fail(env, e, what);
  if (nodes) {
    size_t n = 0;
    nodes[0] = nodes[1] = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess && n > 0) {
      std::vector<cudaGraphNode_t> v(n);
      if (cudaGraphGetNodes(g, v.data(), &n) == cudaSuccess) {
        for (size_t q = 0; q < n; ++q) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(v[q], &t) == cudaSuccess) ++nodes[t == cudaGraphNodeTypeKernel ? 0 : 1];
        }
      }
    }
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(env, e, what);
  }
  return GD_OK;
}
}  // namespace
}  // extern "C++"

// The objective rollout's launches: a checkpoint every C steps (one copy
// launch), then the step (+ observation and objective) launches.
static void issue_objective(gd_env* env, int steps, const float* actions, const float* obs_weight,
                            float reward_weight, float* ell, float* obs, cudaStream_t stream,
                            LaunchTimer* tm = nullptr) {
  const size_t A = (size_t)env->A, W = (size_t)env->W;
  const DevEnv& d = env->d;
  for (int t = 0; t < steps; ++t) {
    if (t % env->C == 0) {
      const int c = t / env->C;
      tbegin(tm, 0);
      copy_snapshot(env, env->ckS + c * A, env->ckF + c * A, env->ckT + c * W, env->ckWD + c * W, d.state, d.flags, d.t,
                    d.world_done, stream);
      tend(tm);
    }
    launch_world(env, actions + (size_t)t * A * 2, nullptr, nullptr, nullptr, obs, nullptr, nullptr, 1, stream, nullptr,
                 obs_weight, reward_weight, ell + (size_t)t * A,
                 env->rk_hist + (size_t)t * A, nullptr, (int)OBS_STRIPES, nullptr, nullptr, tm,
                 env->sel_hist ? env->sel_hist + (size_t)t * A * env->d.K : nullptr,
                 env->fl_hist ? env->fl_hist + (size_t)t * A : nullptr);
  }
}

gd_status gd_rollout_objective(gd_env* env, int32_t steps, const float* actions, const float* obs_weight,
                               float reward_weight, float* ell, float* obs) {
  NvtxRange range_("gd_rollout_objective");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_diff(env, "gd_rollout_objective");
  if (st != GD_OK) return st;
  // the per-step records (K-th distances, selections, decisions) hold episode_len steps
  if (steps < 1 || steps > env->cfg.episode_len)
    return fail(env, GD_ERR_INVALID_ARG, "steps must be in 1..episode_len");
  if (!actions || !obs_weight || !ell) return fail(env, GD_ERR_INVALID_ARG, "actions, obs_weight and ell must not be NULL");
  if (!aligned16(obs_weight) || (obs && !aligned16(obs)))
    return fail(env, GD_ERR_INVALID_ARG, "obs_weight and obs must be 16-byte aligned");
  if (!obs) {
    if (!env->obs_scratch) {
      cudaError_t e = dev_alloc(env, &env->obs_scratch, (size_t)env->A * env->F);
      if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_objective: observation scratch");
    }
    obs = env->obs_scratch;
  }
  if (env->A > 0) {
    if (!batched(env)) {
      // plain form: every launch issued from the host
      issue_objective(env, steps, actions, obs_weight, reward_weight, ell, obs, env->stream);
    } else {
      // batched form: one captured graph, re-used while the arguments are the same
      uint32_t rw_bits;
      std::memcpy(&rw_bits, &reward_weight, sizeof(rw_bits));
      const void* key[6] = {actions, obs_weight, ell, obs, (const void*)(uintptr_t)rw_bits, nullptr};
      bool same = env->ograph && env->og_steps == steps;
      for (int k = 0; k < 6 && same; ++k) same = env->og_key[k] == key[k];
      if (!same) {
        env->og_steps = -1;
        st = capture_graph(
            env, &env->ograph, "gd_rollout_objective: capture",
            [&](cudaStream_t cs) {
              if (GD_ROLLOUT_OVERLAP && env->split)
                issue_rollout_overlapped(env, steps, 0, steps, actions, obs, 0, nullptr, nullptr, cs, obs_weight,
                                         reward_weight, ell);
              else
                issue_objective(env, steps, actions, obs_weight, reward_weight, ell, obs, cs);
            },
            env->og_nodes);
        if (st != GD_OK) return st;
        for (int k = 0; k < 6; ++k) env->og_key[k] = key[k];
        env->og_steps = steps;
      }
      cudaError_t e = cudaGraphLaunch(env->ograph, env->stream);
      if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_objective: graph launch");
    }
  }
  env->diff_actions = actions;
  env->diff_steps = steps;
  env->sel_valid = env->sel_hist != nullptr;
  env->rec_valid = env->fl_hist != nullptr;
  return launch_check(env, "gd_rollout_objective");
}

// Adjoint of `steps` consecutive steps, S[k] -> S[k + 1] under actions[k]
// (S, F: steps + 1 slices of A states / flags; the per-step arrays: steps
// slices of A): the split form's launch pair for the whole segment
// (observer side over (step, agent) tasks, then a thread per agent over the
// steps), or one fused per-world launch per step, last step first.
// lam_zero: the adjoint after the last step is zero; lam_copy: also write
// the adjoint before the first step there.  Neither form needs a memset:
// each leaves its claim counters at zero.
static void launch_adjoint(gd_env* env, const float4* S, const uint8_t* F, const float* actions, int steps,
                           const float* obs_w, long long stride, const float* row_scale, const float* rew_w,
                           float reward_w, float* d_actions, const float* rk = nullptr, cudaStream_t stream = nullptr,
                           int lam_zero = 0, float* lam_copy = nullptr, LaunchTimer* tm = nullptr,
                           const uint16_t* sel = nullptr) {
  if (!stream) stream = env->stream;
  const size_t A = (size_t)env->A;
  AdjArgs a{};
  a.S = S;
  a.F = F;
  a.actions = reinterpret_cast<const float2*>(actions);
  a.obs_w = obs_w;
  a.obs_w_stride = stride;
  a.row_scale = row_scale;
  a.rew_w = rew_w;
  a.reward_w = reward_w;
  a.lam = env->lam;
  a.d_actions = reinterpret_cast<float2*>(d_actions);
  a.rk = rk;
  a.sel = sel;
  a.counter = env->acounter;
  a.order = env->order;
  a.tile_bytes = env->adj_tile;
  a.lam_zero = lam_zero;
  a.lam_copy = reinterpret_cast<float4*>(lam_copy);
  a.steps = steps;
  a.g_obs = env->adj_g;
  a.cs_obs = env->adj_cs;
  a.slot = env->adj_slot;
  a.ocounter = env->adj_oc;
  if (env->adj_split) {
    if (obs_w) {
      tbegin(tm, 2);
      k_adj_observer<kAdjObsWarps><<<env->ao_grid, kAdjObsWarps * 32, kAdjObsSmem, stream>>>(env->d, a);
      tend(tm);
    }
    // 64-thread blocks: a thread's loop is latency-bound, so the blocks are
    // spread over every SM even when there are few agents
    tbegin(tm, 3);
    k_adj_dynamics<<<blocks_for(env->A, 64), 64, 0, stream>>>(env->d, a);
    tend(tm);
    return;
  }
  for (int k = steps - 1; k >= 0; --k) {
    AdjArgs ak = a;
    ak.S = S + (size_t)k * A;
    ak.F = F + (size_t)k * A;
    ak.actions = a.actions + (size_t)k * A;
    ak.row_scale = row_scale ? row_scale + (size_t)k * A : nullptr;
    ak.rk = rk ? rk + (size_t)k * A : nullptr;
    ak.d_actions = a.d_actions + (size_t)k * A;
    ak.steps = 1;
    ak.lam_zero = lam_zero && k == steps - 1;
    ak.lam_copy = k == 0 ? a.lam_copy : nullptr;
    tbegin(tm, 2);
    if (env->adj_notile)
      k_adjoint<kAdjWarps, true><<<env->adj_grid, kAdjWarps * 32, env->adj_smem, stream>>>(env->d, ak);
    else
      k_adjoint<kAdjWarps><<<env->adj_grid, kAdjWarps * 32, env->adj_smem, stream>>>(env->d, ak);
    tend(tm);
  }
}

// Recompute `len` steps of the segment starting from segS[0] / segF[0] /
// segT / segWD, leaving the state after step k in segS[k+1] / segF[k+1]:
// each step reads slot k and writes slot k + 1 (no copy between steps).
// A segment's buffers: states and flags before / after each step, its
// worlds' episode steps and episode-end status.
struct SegBuf {
  float4* S;
  uint8_t* F;
  int* T;
  uint8_t* WD;
};
static SegBuf seg_buf(gd_env* env, int which) {
  return which ? SegBuf{env->segS2, env->segF2, env->segT2, env->segWD2}
               : SegBuf{env->segS, env->segF, env->segT, env->segWD};
}

// With t0 >= 0 (the segment's first step in the last objective rollout) and
// that rollout's record of its decisions, one thread-per-agent launch
// recomputes the states instead (the same states and flags, bit for bit).
static void recompute_segment(gd_env* env, const float* actions0, int len, cudaStream_t stream = nullptr,
                              LaunchTimer* tm = nullptr, int which = 0, int t0 = -1) {
  const size_t A = (size_t)env->A;
  const SegBuf b = seg_buf(env, which);
  if (!stream) stream = env->stream;
  if (t0 >= 0 && env->rec_valid) {
    tbegin(tm, 1);
    k_recompute<<<blocks_for(env->A, 128), 128, 0, stream>>>(
        env->d, reinterpret_cast<const float2*>(actions0), len, b.S, b.F, env->fl_hist + (size_t)t0 * A);
    tend(tm);
    return;
  }
  DevEnv dv = env->d;
  dv.t = b.T;
  dv.world_done = b.WD;
  for (int k = 0; k < len; ++k) {
    dv.state = b.S + k * A;
    dv.flags = b.F + k * A;
    launch_world(env, actions0 + (size_t)k * A * 2, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1, stream, &dv,
                 nullptr, 0.f, nullptr, nullptr, nullptr, 0, b.S + (k + 1) * A, b.F + (k + 1) * A, tm);
  }
}

// The recorded selections the backward pass reads, or nullptr (re-select).
static const uint16_t* rec_sel(const gd_env* env) { return env->sel_valid ? env->sel_hist : nullptr; }

// The backward pass's launches: per checkpoint segment, last first, the
// segment's start copied from its checkpoint, its steps recomputed, then the
// adjoint of each of its steps in reverse.
static void issue_backward(gd_env* env, const float* obs_weight, float reward_weight, const float* d_ell,
                           float* d_actions, float* d_state0, cudaStream_t stream, LaunchTimer* tm = nullptr) {
  const size_t A = (size_t)env->A, W = (size_t)env->W;
  const int T = env->diff_steps, C = env->C;
  for (int seg = (T - 1) / C; seg >= 0; --seg) {
    const int t0 = seg * C, len = std::min(C, T - t0);
    tbegin(tm, 0);
    copy_snapshot(env, env->segS, env->segF, env->segT, env->segWD, env->ckS + seg * A, env->ckF + seg * A,
                  env->ckT + seg * W, env->ckWD + seg * W, stream);
    tend(tm);
    recompute_segment(env, env->diff_actions + (size_t)t0 * A * 2, len, stream, tm, 0, t0);
    launch_adjoint(env, env->segS, env->segF, env->diff_actions + (size_t)t0 * A * 2, len, obs_weight, 0,
                   d_ell ? d_ell + (size_t)t0 * A : nullptr, nullptr, reward_weight, d_actions + (size_t)t0 * A * 2,
                   env->rk_hist + (size_t)t0 * A, stream, t0 + len == T, t0 == 0 ? d_state0 : nullptr, tm,
                   rec_sel(env) ? rec_sel(env) + (size_t)t0 * A * env->d.K : nullptr);
  }
}

// The captured backward pass, pipelined over two segment buffers: on a
// second stream each segment's checkpoint copy and recomputed steps, on the
// capturing stream its adjoint once they are done, so that the recompute of
// a segment runs beside the adjoint of the segment after it; a buffer is
// refilled only after the adjoint that read it.
static void issue_backward_pipelined(gd_env* env, const float* obs_weight, float reward_weight, const float* d_ell,
                                     float* d_actions, float* d_state0, cudaStream_t cap, cudaStream_t sr,
                                     std::vector<cudaEvent_t>& evs) {
  const size_t A = (size_t)env->A, W = (size_t)env->W;
  const int T = env->diff_steps, C = env->C, nseg = (T - 1) / C + 1;
  auto event = [&]() {
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    evs.push_back(e);
    return e;
  };
  cudaEvent_t fork = event();
  cudaEventRecord(fork, cap);
  cudaStreamWaitEvent(sr, fork, 0);
  std::vector<cudaEvent_t> done_adj((size_t)nseg, nullptr);
  for (int j = 0; j < nseg; ++j) {
    const int seg = nseg - 1 - j, t0 = seg * C, len = std::min(C, T - t0), which = j & 1;
    const SegBuf b = seg_buf(env, which);
    if (j >= 2) cudaStreamWaitEvent(sr, done_adj[(size_t)(j - 2)], 0);
    copy_snapshot(env, b.S, b.F, b.T, b.WD, env->ckS + seg * A, env->ckF + seg * A, env->ckT + seg * W,
                  env->ckWD + seg * W, sr);
    recompute_segment(env, env->diff_actions + (size_t)t0 * A * 2, len, sr, nullptr, which, t0);
    cudaEvent_t rec = event();
    cudaEventRecord(rec, sr);
    cudaStreamWaitEvent(cap, rec, 0);
    launch_adjoint(env, b.S, b.F, env->diff_actions + (size_t)t0 * A * 2, len, obs_weight, 0,
                   d_ell ? d_ell + (size_t)t0 * A : nullptr, nullptr, reward_weight, d_actions + (size_t)t0 * A * 2,
                   env->rk_hist + (size_t)t0 * A, cap, t0 + len == T, t0 == 0 ? d_state0 : nullptr, nullptr,
                   rec_sel(env) ? rec_sel(env) + (size_t)t0 * A * env->d.K : nullptr);
    done_adj[(size_t)j] = event();
    cudaEventRecord(done_adj[(size_t)j], cap);
  }
  // the second stream's last work (segment 0's recompute) is already joined
}

gd_status gd_rollout_backward(gd_env* env, const float* obs_weight, float reward_weight, const float* d_ell,
                              float* d_actions, float* d_state0) {
  NvtxRange range_("gd_rollout_backward");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_diff(env, "gd_rollout_backward");
  if (st != GD_OK) return st;
  if (env->diff_steps < 1) return fail(env, GD_ERR_STATE, "gd_rollout_backward: no gd_rollout_objective to differentiate");
  if (!obs_weight || !d_actions) return fail(env, GD_ERR_INVALID_ARG, "obs_weight and d_actions must not be NULL");
  if (!aligned16(obs_weight)) return fail(env, GD_ERR_INVALID_ARG, "obs_weight must be 16-byte aligned");
  if (env->A == 0) return GD_OK;
  if (!batched(env)) {
    // plain form: every launch issued from the host
    issue_backward(env, obs_weight, reward_weight, d_ell, d_actions, d_state0, env->stream);
    return launch_check(env, "gd_rollout_backward");
  }
  uint32_t rw_bits;
  std::memcpy(&rw_bits, &reward_weight, sizeof(rw_bits));
  const void* key[7] = {obs_weight, d_ell, d_actions, d_state0, env->diff_actions, (const void*)(uintptr_t)rw_bits,
                        rec_sel(env)};
  bool same = env->bgraph && env->bg_steps == env->diff_steps;
  for (int k = 0; k < 7 && same; ++k) same = env->bg_key[k] == key[k];
  if (!same) {
    env->bg_steps = -1;
    cudaStream_t sr = nullptr;
    std::vector<cudaEvent_t> evs;
    const bool pipe = cudaStreamCreateWithFlags(&sr, cudaStreamNonBlocking) == cudaSuccess;
    st = capture_graph(
        env, &env->bgraph, "gd_rollout_backward: capture",
        [&](cudaStream_t cs) {
          if (pipe)
            issue_backward_pipelined(env, obs_weight, reward_weight, d_ell, d_actions, d_state0, cs, sr, evs);
          else
            issue_backward(env, obs_weight, reward_weight, d_ell, d_actions, d_state0, cs);
        },
        env->bg_nodes);
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    if (sr) cudaStreamDestroy(sr);
    if (st != GD_OK) return st;
    for (int k = 0; k < 7; ++k) env->bg_key[k] = key[k];
    env->bg_steps = env->diff_steps;
  }
  cudaError_t e = cudaGraphLaunch(env->bgraph, env->stream);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_rollout_backward: graph launch");
  return launch_check(env, "gd_rollout_backward");
}

gd_status gd_time_backward(gd_env* env, const float* obs_weight, float reward_weight, const float* d_ell,
                           float* d_actions, float* d_state0, float* ms, int32_t* launches) {
  NvtxRange range_("gd_time_backward");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_diff(env, "gd_time_backward");
  if (st != GD_OK) return st;
  if (env->diff_steps < 1) return fail(env, GD_ERR_STATE, "gd_time_backward: no gd_rollout_objective to differentiate");
  if (!obs_weight || !d_actions || !ms || !launches)
    return fail(env, GD_ERR_INVALID_ARG, "obs_weight, d_actions, ms and launches must not be NULL");
  if (!aligned16(obs_weight)) return fail(env, GD_ERR_INVALID_ARG, "obs_weight must be 16-byte aligned");
  for (int k = 0; k < GD_BWD_KINDS; ++k) {
    ms[k] = 0.f;
    launches[k] = 0;
  }
  if (env->A == 0) return GD_OK;
  LaunchTimer tm;
  tm.stream = env->stream;
  issue_backward(env, obs_weight, reward_weight, d_ell, d_actions, d_state0, env->stream, &tm);
  cudaError_t e = tm.collect(ms, launches, GD_BWD_KINDS);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_time_backward");
  return launch_check(env, "gd_time_backward");
}

gd_status gd_time_objective(gd_env* env, int32_t steps, const float* actions, const float* obs_weight,
                            float reward_weight, float* ell, float* obs, float* ms, int32_t* launches) {
  NvtxRange range_("gd_time_objective");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_diff(env, "gd_time_objective");
  if (st != GD_OK) return st;
  // the per-step records (K-th distances, selections, decisions) hold episode_len steps
  if (steps < 1 || steps > env->cfg.episode_len)
    return fail(env, GD_ERR_INVALID_ARG, "steps must be in 1..episode_len");
  if (!actions || !obs_weight || !ell || !obs || !ms || !launches)
    return fail(env, GD_ERR_INVALID_ARG, "actions, obs_weight, ell, obs, ms and launches must not be NULL");
  if (!aligned16(obs_weight) || !aligned16(obs))
    return fail(env, GD_ERR_INVALID_ARG, "obs_weight and obs must be 16-byte aligned");
  for (int k = 0; k < GD_OBJ_KINDS; ++k) {
    ms[k] = 0.f;
    launches[k] = 0;
  }
  if (env->A > 0) {
    LaunchTimer tm;
    tm.stream = env->stream;
    issue_objective(env, steps, actions, obs_weight, reward_weight, ell, obs, env->stream, &tm);
    cudaError_t e = tm.collect(ms, launches, GD_OBJ_KINDS);
    if (e != cudaSuccess) return cuda_fail(env, e, "gd_time_objective");
  }
  env->diff_actions = actions;
  env->diff_steps = steps;
  env->sel_valid = env->sel_hist != nullptr;
  env->rec_valid = env->fl_hist != nullptr;
  return launch_check(env, "gd_time_objective");
}

gd_status gd_step_backward(gd_env* env, const float* actions, const float* d_state_next, const float* d_obs,
                           const float* obs_weight, const float* d_reward_s, float* d_state, float* d_actions) {
  NvtxRange range_("gd_step_backward");
  if (!env) return GD_ERR_INVALID_ARG;
  gd_status st = need_diff(env, "gd_step_backward");
  if (st != GD_OK) return st;
  if (!actions || !d_state || !d_actions) return fail(env, GD_ERR_INVALID_ARG, "actions, d_state and d_actions must not be NULL");
  const float* w = d_obs ? d_obs : obs_weight;
  if (w && !aligned16(w)) return fail(env, GD_ERR_INVALID_ARG, "d_obs / obs_weight must be 16-byte aligned");
  const size_t A = (size_t)env->A;
  if (A == 0) return GD_OK;
  copy_snapshot(env, env->segS, env->segF, env->segT, env->segWD, env->d.state, env->d.flags, env->d.t,
                env->d.world_done);
  recompute_segment(env, actions, 1);
  if (d_state_next) cudaMemcpyAsync(env->lam, d_state_next, sizeof(float4) * A, cudaMemcpyDeviceToDevice, env->stream);
  launch_adjoint(env, env->segS, env->segF, actions, 1, w, d_obs ? env->F : 0, nullptr, d_reward_s, 0.f, d_actions,
                 nullptr, nullptr, d_state_next ? 0 : 1, d_state);
  return launch_check(env, "gd_step_backward");
}

gd_status gd_get_state(gd_env* env, float* state, uint8_t* flags, int32_t* t) {
  if (!env) return GD_ERR_INVALID_ARG;
  if (state) cudaMemcpyAsync(state, env->d.state, sizeof(float4) * env->A, cudaMemcpyDeviceToDevice, env->stream);
  if (flags) cudaMemcpyAsync(flags, env->d.flags, env->A, cudaMemcpyDeviceToDevice, env->stream);
  if (t) cudaMemcpyAsync(t, env->d.t, sizeof(int) * env->W, cudaMemcpyDeviceToDevice, env->stream);
  return launch_check(env, "gd_get_state");
}

gd_status gd_set_state(gd_env* env, const float* state, const uint8_t* flags, const int32_t* t) {
  if (!env) return GD_ERR_INVALID_ARG;
  if (state) cudaMemcpyAsync(env->d.state, state, sizeof(float4) * env->A, cudaMemcpyDeviceToDevice, env->stream);
  if (flags) cudaMemcpyAsync(env->d.flags, flags, env->A, cudaMemcpyDeviceToDevice, env->stream);
  if (t) cudaMemcpyAsync(env->d.t, t, sizeof(int) * env->W, cudaMemcpyDeviceToDevice, env->stream);
  k_derive_world_done<<<blocks_for(env->W, 256), 256, 0, env->stream>>>(env->d);
  return launch_check(env, "gd_set_state");
}

// Time the fused step + observation for each (road cell, CTA size, road
// tile, top-K strategy) and keep the fastest.  A step's cost changes over an
// episode (agents leave, the road selections move with their anchors), so a
// trial is timed at kTunePhases points of an episode: the env's current
// state and the states kTunePhases - 1 strides of zero-action steps later
// (stride: a third of the episode, at most 32 steps).  Each phase is saved
// once, with its selection anchors, and restored exactly before each of its
// windows of kTuneSteps steps; a trial's time is the sum over the phases,
// best of three after a warm-up.  The current state is restored at the end.
gd_status gd_autotune(gd_env* env) {
  NvtxRange range_("gd_autotune");
  if (!env) return GD_ERR_INVALID_ARG;
  if (env->A == 0) return GD_OK;
  const size_t A = (size_t)env->A, W = (size_t)env->W;
  const int P = kTunePhases;
  float4* sS = nullptr;
  uint8_t* sF = nullptr;
  int* sT = nullptr;
  uint8_t* sWD = nullptr;
  float4* sAn = nullptr;
  float* act = nullptr;
  cudaError_t e = dev_alloc(env, &sS, P * A);
  if (e == cudaSuccess) e = dev_alloc(env, &sF, P * A);
  if (e == cudaSuccess) e = dev_alloc(env, &sT, P * W);
  if (e == cudaSuccess) e = dev_alloc(env, &sWD, P * W);
  if (e == cudaSuccess) e = dev_alloc(env, &sAn, P * A);
  if (e == cudaSuccess) e = dev_alloc(env, &act, 2 * A);
  if (e == cudaSuccess && !env->obs_scratch) e = dev_alloc(env, &env->obs_scratch, A * (size_t)env->F);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(env, sS); dev_free(env, sF); dev_free(env, sT); dev_free(env, sWD); dev_free(env, sAn);
    dev_free(env, act);
  };
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(env, e, "gd_autotune: scratch");
  }
  DevEnv& d = env->d;
  auto save = [&](int p) {
    copy_snapshot(env, sS + p * A, sF + p * A, sT + p * W, sWD + p * W, d.state, d.flags, d.t, d.world_done);
    cudaMemcpyAsync(sAn + p * A, d.anchor, sizeof(float4) * A, cudaMemcpyDeviceToDevice, env->stream);
  };
  auto restore = [&](int p) {
    copy_snapshot(env, d.state, d.flags, d.t, d.world_done, sS + p * A, sF + p * A, sT + p * W, sWD + p * W);
    cudaMemcpyAsync(d.anchor, sAn + p * A, sizeof(float4) * A, cudaMemcpyDeviceToDevice, env->stream);
  };
  cudaMemsetAsync(act, 0, sizeof(float) * 2 * A, env->stream);
  const int stride = std::min(32, std::max(1, env->cfg.episode_len / P));
  save(0);
  for (int p = 1; p < P; ++p) {
    for (int k = 0; k < stride; ++k)
      launch_world(env, act, nullptr, nullptr, nullptr, env->obs_scratch, nullptr, nullptr, 1);
    save(p);
  }
  // time `launch` (win steps) at every phase: best of three sums after a
  // warm-up
  int win = kTuneSteps;
  auto time_phases = [&](auto&& launch, float& best) -> cudaError_t {
    best = INFINITY;
    for (int rep = 0; rep < 4; ++rep) {
      float sum = 0.f;
      for (int p = 0; p < P; ++p) {
        restore(p);
        cudaEventRecord(e0, env->stream);
        for (int k = 0; k < win; ++k) launch();
        cudaEventRecord(e1, env->stream);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) return err;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        sum += t;
      }
      if (rep > 0) best = std::min(best, sum);
    }
    return cudaSuccess;
  };
  // windows long enough to time: a small batch's steps take tens of
  // microseconds, so its windows grow (up to the stride between the points)
  // until the default shape's trial lasts about kTuneTrialMs
  {
    float probe = INFINITY;
    e = time_phases([&] { launch_world(env, act, nullptr, nullptr, nullptr, env->obs_scratch, nullptr, nullptr, 1); },
                    probe);
    if (e == cudaSuccess && probe > 0.f && probe < kTuneTrialMs)
      win = std::min(std::max(kTuneSteps, stride),
                     std::max(kTuneSteps, (int)std::ceil(kTuneSteps * kTuneTrialMs / probe)));
  }
  const float min_cell = (2.f * env->cfg.obs_radius + 0.01f) / (float)(MAX_ROWS - 2);
  const float cells[] = {6.f, 8.f, 12.f};
  const int warps[] = {4, 8, 16};
  float best_ms = INFINITY, best_cell = env->road_cell;
  int best_w = env->warps, best_st = d.topk, best_nt = env->notile, best_sp = env->split;
  for (float c : cells) {
    if (e != cudaSuccess) break;
    const float cell = std::max(c, min_cell);
    if ((e = build_road(env, cell)) != cudaSuccess) break;
    for (int sp = 0; sp <= 1 && e == cudaSuccess; ++sp) {
      env->split = sp;
      for (int shape = 0; shape < 6; ++shape) {
        const int wp = warps[shape % 3];
        env->warps = wp;
        env->notile = shape / 3;
        if ((e = shape_kernels(env, env->max_block)) != cudaSuccess) break;
        for (int st = 1; st <= 2; ++st) {
          d.topk = st;
          float ms = INFINITY;
          e = time_phases(
              [&] { launch_world(env, act, nullptr, nullptr, nullptr, env->obs_scratch, nullptr, nullptr, 1); }, ms);
          if (e != cudaSuccess) break;
          // the trials issue the launches from the host; in the overlapped
          // rollout the step launch of t + 1 shares the SMs with the tail of
          // observation t, where a larger step CTA finds room later: near
          // ties go to the smaller CTA (a larger one must win by
          // kTuneCtaMargin per doubling of its warps)
          ms *= 1.f + kTuneCtaMargin * (float)(wp == 4 ? 0 : (wp == 8 ? 1 : 2));
          if (ms < best_ms) {
            best_ms = ms;
            best_cell = cell;
            best_w = wp;
            best_st = st;
            best_nt = env->notile;
            best_sp = sp;
          }
        }
        if (e != cudaSuccess) break;
      }
    }
    if (e != cudaSuccess) break;
  }
  env->split = best_sp;
  if (e == cudaSuccess) {
    env->warps = best_w;
    env->notile = best_nt;
    d.topk = best_st;
    e = build_road(env, best_cell);
  }
  // adjoint (differentiable envs): the split form, or the fused form with or
  // without the road tile, timed on one step's adjoint about the current state
  if (e == cudaSuccess && (env->cfg.flags & GD_DIFFERENTIABLE)) {
    float* wts = nullptr;
    float* dact = nullptr;
    e = dev_alloc(env, &wts, (size_t)env->F);
    if (e == cudaSuccess) e = dev_alloc(env, &dact, 2 * A);
    if (e == cudaSuccess) {
      std::vector<float> ones((size_t)env->F, 1.f);
      e = cudaMemcpyAsync(wts, ones.data(), sizeof(float) * env->F, cudaMemcpyHostToDevice, env->stream);
    }
    if (e == cudaSuccess) {
      restore(0);
      copy_snapshot(env, env->segS, env->segF, env->segT, env->segWD, d.state, d.flags, d.t, d.world_done);
      recompute_segment(env, act, 1);
    }
    float abest = INFINITY;
    int abest_nt = env->adj_notile, abest_sp = env->adj_split;
    for (int form = 0; form < 3 && e == cudaSuccess; ++form) {
      env->adj_split = form == 0;
      env->adj_notile = form == 2;
      if ((e = shape_kernels(env, env->max_block)) != cudaSuccess) break;
      float ms = INFINITY;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, env->stream);
        launch_adjoint(env, env->segS, env->segF, act, 1, wts, 0, nullptr, nullptr, 1.f, dact, nullptr, nullptr, 1);
        cudaEventRecord(e1, env->stream);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0) ms = std::min(ms, t);
      }
      if (e == cudaSuccess && ms < abest) {
        abest = ms;
        abest_nt = env->adj_notile;
        abest_sp = env->adj_split;
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(env->stream);
    dev_free(env, wts);
    dev_free(env, dact);
    env->adj_notile = abest_nt;
    env->adj_split = abest_sp;
    if (e == cudaSuccess) e = shape_kernels(env, env->max_block);
  }
  // fused LiDAR kernel: CTA size, on the chosen road grid
  if (e == cudaSuccess && env->lidar_n > 0) {
    float* ldepth = nullptr;
    uint8_t* lcls = nullptr;
    e = dev_alloc(env, &ldepth, A * (size_t)env->lidar_n);
    if (e == cudaSuccess) e = dev_alloc(env, &lcls, A * (size_t)env->lidar_n);
    float lbest = INFINITY;
    int lbest_w = env->lw_warps, lbest_nt = env->lw_notile, lbest_sp = env->lw_split;
    for (int cfg = 0; cfg < 7; ++cfg) {
      if (e != cudaSuccess) break;
      // trials 0..5: fused kernel, 4 / 8 / 12 warps, with and without the
      // road tile; trial 6: step and stand-alone scan as two launches
      const int wp = cfg < 6 ? 4 * (1 + cfg / 2) : 8;
      env->lw_warps = wp;
      env->lw_notile = cfg & 1;
      env->lw_split = cfg == 6;
      if ((e = shape_kernels(env, env->max_block)) != cudaSuccess) break;
      if (env->lw_warps != wp) continue;       // this many warps do not fit with this many rays
      float ms = INFINITY;
      e = time_phases([&] { launch_world_lidar(env, act, nullptr, nullptr, nullptr, nullptr, ldepth, lcls, 1); }, ms);
      if (e == cudaSuccess && ms < lbest) {
        lbest = ms;
        lbest_w = wp;
        lbest_nt = env->lw_notile;
        lbest_sp = env->lw_split;
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(env->stream);
    dev_free(env, ldepth);
    dev_free(env, lcls);
    env->lw_warps = lbest_w;
    env->lw_notile = lbest_nt;
    env->lw_split = lbest_sp;
    if (e == cudaSuccess) e = shape_kernels(env, env->max_block);
  }
  restore(0);
  drop_graphs(env);
  if (e == cudaSuccess) e = cudaStreamSynchronize(env->stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_autotune");
  return launch_check(env, "gd_autotune");
}

// Failure-detection self-test: one CTA waits on an mbarrier phase that
// nothing completes, for at most ~wait_us microseconds of its own clock, then
// records ERR_TIMEOUT in the env's sticky error word and returns.  No copy
// is in flight, so leaving the barrier pending is harmless.
__global__ void k_selftest_wait(unsigned* err, long long limit_cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const long long t0 = clock64();
  bool done = false;
  while (!(done = mbar_try_wait(&bar, 0))) {
    if (clock64() - t0 > limit_cycles) break;
  }
  if (!done && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
}

gd_status gd_selftest_timeout(gd_env* env, int32_t wait_us) {
  if (!env) return GD_ERR_INVALID_ARG;
  if (wait_us < 1 || wait_us > 1000000) return fail(env, GD_ERR_INVALID_ARG, "wait_us must be in 1..1000000");
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  const long long cycles = (long long)std::max(khz, 1000000) * wait_us / 1000;
  k_selftest_wait<<<1, 32, 0, env->stream>>>(env->d.err, cycles);
  return launch_check(env, "gd_selftest_timeout");
}

gd_status gd_sync(gd_env* env) {
  NvtxRange range_("gd_sync");
  if (!env) return GD_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(env->h_err, env->d.err, sizeof(unsigned), cudaMemcpyDeviceToHost, env->stream);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_sync");
  e = cudaStreamSynchronize(env->stream);
  if (e != cudaSuccess) return cuda_fail(env, e, "gd_sync");
  const unsigned w = *env->h_err;
  if (w) {
    cudaMemsetAsync(env->d.err, 0, sizeof(unsigned), env->stream);
    cudaStreamSynchronize(env->stream);
    if (w & ERR_ACTION)
      return fail(env, GD_ERR_INVALID_ARG, "a step saw a non-finite action (or |steer| >= pi/2 for the kinematic bicycle)");
    if (w & ERR_TIMEOUT) return fail(env, GD_ERR_TIMEOUT, "a bounded device wait gave up");
    return fail(env, GD_ERR_CAPACITY, "a device-side capacity was exceeded");
  }
  return GD_OK;
}

}  // extern "C"
