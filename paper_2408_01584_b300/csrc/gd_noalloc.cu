// gd_collide_noalloc: agent/agent collision flags without any allocation.
//
// Who needs this: a caller whose device memory is owned by someone else's
// pool allocator (a training framework that reserves the GPU up front, so a
// cudaMalloc from this library would fail or escape its accounting), or a
// latency-critical loop that cannot afford the device-wide synchronisation
// cudaMalloc / cudaFree may cause.  gd_create allocates the env's buffers,
// so such a caller cannot use the env API; this entry point takes every
// input and output from the caller and keeps its working memory in a fixed
// array compiled into the library.
//
// The computation is the per-stage form's agent grid + box test (the same
// decisions gd_step records in GD_FLAG_COLLIDED): agents are keyed by a
// uniform-grid cell at least as large as the largest box diagonal, sorted
// per world, and each agent tests the boxes in its 3 x 3 neighbouring cells.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "gd_device.cuh"

using namespace gd;

void gd_set_thread_error(const std::string& msg);   // defined in gd.cu

namespace {

constexpr int kMaxAgents = GD_NOALLOC_MAX_AGENTS;
constexpr int kMaxWorlds = GD_NOALLOC_MAX_WORLDS;
// Scratch layout (32-bit words):
//   [kOffOff,   + kMaxWorlds + 1)  world offsets copied from the caller
//   [kOffCount, + kMaxWorlds)      active agents per world (written every call)
//   [kOffKeys,  + kMaxAgents)      sorted grid keys, CSR by world (written every call)
constexpr int kOffOff = 0;
constexpr int kOffCount = ((kMaxWorlds + 1 + 63) / 64) * 64;
constexpr int kOffKeys = kOffCount + kMaxWorlds;
constexpr int kWords = kOffKeys + kMaxAgents;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kWords];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol
// name is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
cudaError_t scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Cell coordinate biased by 2048 cells and clamped to 12 bits (monotone;
// never separates two agents within one cell of each other).
__device__ __forceinline__ int na_cell(float v, float inv) {
  return (int)clampf(floorf(v * inv) + 2048.f, 0.f, 4095.f);
}

// Warp per world: sorted keys of the active agents into the scratch.
__global__ void k_na_grid(int W, uint32_t* __restrict__ scratch, const float4* __restrict__ state,
                          const uint8_t* __restrict__ active, float inv) {
  __shared__ uint32_t keys_s[8][GD_MAX_AGENTS_PER_WORLD];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= W) return;
  const int a0 = (int)scratch[kOffOff + w], a1 = (int)scratch[kOffOff + w + 1];
  uint32_t* keys = keys_s[wib];
  int n = 0;
  for (int j0 = a0; j0 < a1; j0 += WARP) {
    const int j = j0 + lane;
    bool act = false;
    uint32_t key = 0;
    if (j < a1 && (!active || active[j])) {
      const float4 s = state[j];
      key = agent_cell_key(na_cell(s.x, inv), na_cell(s.y, inv), j - a0);
      act = true;
    }
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (act) keys[n + __popc(m & ((1u << lane) - 1u))] = key;
    n += __popc(m);
  }
  __syncwarp();
  for (int k = lane; k < n; k += WARP) {
    const uint32_t key = keys[k];
    int r = 0;
    for (int q = 0; q < n; ++q) r += keys[q] < key;
    scratch[kOffKeys + a0 + r] = key;
  }
  if (lane == 0) scratch[kOffCount + w] = (uint32_t)n;
}

__device__ __forceinline__ int na_bound(const uint32_t* a, int n, uint32_t v, bool upper) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (upper ? (a[mid] <= v) : (a[mid] < v)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Warp per agent: box test against the agents of the 3 x 3 neighbouring cells.
__global__ void k_na_collide(int W, int A, const uint32_t* __restrict__ scratch, const float4* __restrict__ state,
                             const float2* __restrict__ extent, const uint8_t* __restrict__ active, float inv,
                             uint8_t* __restrict__ collided) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= A) return;
  if (active && !active[i]) {
    if (lane == 0) collided[i] = 0;
    return;
  }
  // world of agent i: last w with offset[w] <= i
  int lo = 0, hi = W;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int)scratch[kOffOff + mid] <= i) lo = mid; else hi = mid;
  }
  const int a0 = (int)scratch[kOffOff + lo];
  const int n = (int)scratch[kOffCount + lo];
  const uint32_t* keys = scratch + kOffKeys + a0;
  const float4 s = state[i];
  const float2 ex = extent[i];
  const int cx = na_cell(s.x, inv), cy = na_cell(s.y, inv);
  float sa, ca;
  sincosf(s.z, &sa, &ca);
  bool hit = false;
  for (int dcx = -1; dcx <= 1; ++dcx) {
    const int c = cx + dcx;
    if (c < 0 || c > 4095) continue;
    const int b = na_bound(keys, n, agent_cell_key(c, max(cy - 1, 0), 0), false);
    const int en = na_bound(keys, n, agent_cell_key(c, min(cy + 1, 4095), 255), true);
    for (int k = b + lane; k < en; k += WARP) {
      const int j = a0 + (int)(keys[k] & 0xffu);
      if (j == i) continue;
      const float4 sj = state[j];
      const float2 ej = extent[j];
      float sb, cb;
      sincosf(sj.z, &sb, &cb);
      hit |= box_box_depth(sj.x - s.x, sj.y - s.y, ca, sa, 0.5f * ex.x, 0.5f * ex.y, cb, sb, 0.5f * ej.x,
                           0.5f * ej.y) > 0.f;
    }
  }
  hit = __any_sync(0xffffffffu, hit);
  if (lane == 0) collided[i] = hit ? 1 : 0;
}

gd_status na_fail(gd_status st, const std::string& msg) {
  gd_set_thread_error("gd_collide_noalloc: " + msg);
  return st;
}

}  // namespace

extern "C" gd_status gd_collide_noalloc(int32_t num_worlds, const int32_t* agent_off, const float* state,
                                        const float* extent, const uint8_t* active, float cell, uint8_t* collided,
                                        void* cuda_stream) {
  if (num_worlds < 1) return na_fail(GD_ERR_INVALID_ARG, "num_worlds must be >= 1");
  if (num_worlds > kMaxWorlds)
    return na_fail(GD_ERR_CAPACITY, "num_worlds " + std::to_string(num_worlds) + " exceeds GD_NOALLOC_MAX_WORLDS (" +
                                        std::to_string(kMaxWorlds) + ")");
  if (!agent_off) return na_fail(GD_ERR_INVALID_ARG, "agent_off must not be NULL");
  if (agent_off[0] != 0) return na_fail(GD_ERR_INVALID_ARG, "agent_off[0] must be 0");
  for (int w = 0; w < num_worlds; ++w) {
    const int n = agent_off[w + 1] - agent_off[w];
    if (n < 0) return na_fail(GD_ERR_INVALID_ARG, "agent_off must be non-decreasing");
    if (n > GD_MAX_AGENTS_PER_WORLD)
      return na_fail(GD_ERR_CAPACITY, "world " + std::to_string(w) + " has more than GD_MAX_AGENTS_PER_WORLD agents");
  }
  const int A = agent_off[num_worlds];
  if (A > kMaxAgents)
    return na_fail(GD_ERR_CAPACITY, std::to_string(A) + " agents exceed GD_NOALLOC_MAX_AGENTS (" +
                                        std::to_string(kMaxAgents) + ")");
  if (!(cell > 0.f) || !std::isfinite(cell)) return na_fail(GD_ERR_INVALID_ARG, "cell must be > 0");
  if (A > 0 && (!state || !extent || !collided)) return na_fail(GD_ERR_INVALID_ARG, "state, extent and collided must not be NULL");
  if (((uintptr_t)state & 15u) || ((uintptr_t)extent & 7u))
    return na_fail(GD_ERR_INVALID_ARG, "state must be 16-byte and extent 8-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // a graph would keep the host address of agent_off and read it again at
  // every replay, after the caller may have freed or changed it
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &capture);
  if (e != cudaSuccess) return na_fail(GD_ERR_CUDA, std::string("capture status: ") + cudaGetErrorString(e));
  if (capture != cudaStreamCaptureStatusNone)
    return na_fail(GD_ERR_INVALID_ARG, "the stream is being captured into a CUDA graph; calls are not capturable "
                                       "(each copies agent_off from host memory)");
  uint32_t* scratch = nullptr;
  e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return na_fail(GD_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(scratch + kOffOff, agent_off, sizeof(int32_t) * (num_worlds + 1), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return na_fail(GD_ERR_CUDA, std::string("offset copy: ") + cudaGetErrorString(e));
  if (A == 0) return GD_OK;
  const float inv = 1.f / cell;
  k_na_grid<<<(num_worlds + 7) / 8, 256, 0, s>>>(num_worlds, scratch, reinterpret_cast<const float4*>(state), active, inv);
  k_na_collide<<<(A + 7) / 8, 256, 0, s>>>(num_worlds, A, scratch, reinterpret_cast<const float4*>(state),
                                           reinterpret_cast<const float2*>(extent), active, inv, collided);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(GD_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return GD_OK;
}
