// Per-stage step kernels (the "plain" form: one launch per stage).
//
//   k_reset_worlds  masked world reset (snapshot copy)
//   k_dynamics      bicycle model of App. B (or the simplified invertible model of
//                   Sec. 3.2) for every agent still in the scene
//   k_agent_grid    per world: uniform-grid keys of the active agents, sorted
//   k_collide       per agent: oriented-box test against agents in the 3x3
//                   neighbouring cells (replaces the paper's BVH broad phase, Sec. 3.1)
//   k_offroad       per agent: box against road-edge segments of the edge-grid
//                   cells under its bounding box (Sec. 3.2 "Termination conditions")
//   k_finish        per world: goal, reward, done and end of episode (Sec. 3.2
//                   "Rewards", "Termination conditions")
#pragma once
#include "gd_device.cuh"

namespace gd {

// Warp per world: restore the initial snapshot of worlds selected by mask
// (mask[w] != 0), or, if mask is NULL, of worlds whose episode ended.
__global__ void k_reset_worlds(DevEnv e, const uint8_t* __restrict__ mask) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= e.W) return;
  const bool r = mask ? (mask[w] != 0) : (e.world_done[w] != 0);
  __syncwarp();
  if (!r) return;
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  for (int i = a0 + lane; i < a1; i += WARP) {
    e.state[i] = e.init_state[i];
    e.flags[i] = e.init_flags[i];
  }
  if (lane == 0) {
    e.t[w] = 0;
    e.world_done[w] = 0;
  }
}

// Thread per agent.  Done agents are frozen (removed from the scene) and
// uncontrolled ones (GD_FLAG_STATIC) stay where they are.
__global__ void k_dynamics(DevEnv e, const float2* __restrict__ actions) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.A) return;
  if (e.flags[i] & (GD_FLAG_DONE | GD_FLAG_STATIC)) return;
  const float2 a = actions[i];
  float4 s = e.state[i];
  if (!dynamics_step(e.dyn, s, a.x, a.y, e.stat[i].x, e.dt, e.vmax)) {
    atomicOr(e.err, ERR_ACTION);
    return;
  }
  e.state[i] = s;
}

// The steps k = 0 .. len-1 of a checkpoint segment recomputed for the
// backward pass from S[0] / F[0] (the segment's checkpoint), the steps'
// actions and the forward rollout's record of its decisions, each step's
// post-step flags fl_rec[k].  A thread per agent takes the step kernel's
// state update (the dynamics of an agent neither done nor static, with the
// same arithmetic; a differentiable env never restarts a world inside a
// rollout), so S[k + 1] and F[k + 1] are bit for bit the step kernel's; the
// collision, road-edge and goal decisions come from the record instead of
// the grids.
__global__ void k_recompute(DevEnv e, const float2* __restrict__ actions, int len, float4* __restrict__ S,
                            uint8_t* __restrict__ F, const uint8_t* __restrict__ fl_rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.A) return;
  const float L = e.stat[i].x;
  float4 s = S[i];
  uint8_t f = F[i];
  for (int k = 0; k < len; ++k) {
    const size_t ik = (size_t)k * e.A + i;
    if (!(f & (GD_FLAG_DONE | GD_FLAG_STATIC))) {
      const float2 u = actions[ik];
      if (!dynamics_step(e.dyn, s, u.x, u.y, L, e.dt, e.vmax)) atomicOr(e.err, ERR_ACTION);
    }
    f = fl_rec[ik];
    S[ik + e.A] = s;
    F[ik + e.A] = f;
  }
}

// Cell coordinate clamped to the key's 12-bit range (clamping is monotone
// and never separates two agents that are within one cell of each other).
__device__ __forceinline__ int agent_cell(float v, float o, float inv) {
  return (int)clampf(floorf((v - o) * inv), 0.f, 4095.f);
}

// Warp per world: sort the keys of the active agents (rank by counting, at
// most 128 keys) into agrid_key[agent_off[w] ..], count in agrid_n[w].
__global__ void k_agent_grid(DevEnv e) {
  __shared__ uint32_t keys_s[8][GD_MAX_AGENTS_PER_WORLD];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= e.W) return;
  uint32_t* keys = keys_s[wib];
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  const GridDesc g = e.rgrid[w];
  const float inv = 1.f / e.agent_cell;
  int n = 0;
  for (int j0 = a0; j0 < a1; j0 += WARP) {
    const int j = j0 + lane;
    bool act = false;
    uint32_t key = 0;
    if (j < a1 && !(e.flags[j] & GD_FLAG_DONE)) {
      const float4 s = e.state[j];
      key = agent_cell_key(agent_cell(s.x, g.ox, inv), agent_cell(s.y, g.oy, inv), j - a0);
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
    for (int q = 0; q < n; ++q) r += keys[q] < key;   // keys are distinct (local index in the low bits)
    e.agrid_key[a0 + r] = key;
  }
  if (lane == 0) e.agrid_n[w] = n;
}

// First index with a[k] >= v (lower) / a[k] > v (upper) in a sorted array.
__device__ __forceinline__ int lower_bound_u32(const uint32_t* a, int n, uint32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int upper_bound_u32(const uint32_t* a, int n, uint32_t v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Warp per agent: agent/agent collision through the agent grid.  The cell
// is at least the largest box diagonal, so overlapping boxes sit in the same
// or neighbouring cells; the three cells of one neighbouring column are one
// contiguous key range.  Uncontrolled agents are in the grid (others collide
// with them) but get no test of their own.
__global__ void k_collide(DevEnv e) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= e.A) return;
  if (e.flags[i] & (GD_FLAG_DONE | GD_FLAG_STATIC)) return;
  const int w = e.agent_world[i];
  const int a0 = e.agent_off[w];
  const int n = e.agrid_n[w];
  const uint32_t* keys = e.agrid_key + a0;
  const GridDesc g = e.rgrid[w];
  const float inv = 1.f / e.agent_cell;
  const float4 s = e.state[i];
  const float4 st = e.stat[i];
  const int cx = agent_cell(s.x, g.ox, inv), cy = agent_cell(s.y, g.oy, inv);
  float sa, ca;
  sincosf(s.z, &sa, &ca);
  bool hit = false;
  for (int dcx = -1; dcx <= 1; ++dcx) {
    const int c = cx + dcx;
    if (c < 0 || c > 4095) continue;
    const uint32_t lo = agent_cell_key(c, max(cy - 1, 0), 0), hi = agent_cell_key(c, min(cy + 1, 4095), 255);
    const int b = lower_bound_u32(keys, n, lo);
    const int en = upper_bound_u32(keys, n, hi);
    for (int k = b + lane; k < en; k += WARP) {
      const int j = a0 + (int)(keys[k] & 0xffu);
      if (j == i) continue;
      const float4 sj = e.state[j];
      const float4 tj = e.stat[j];
      float sb, cb;
      sincosf(sj.z, &sb, &cb);
      hit |= box_box_depth(sj.x - s.x, sj.y - s.y, ca, sa, 0.5f * st.x, 0.5f * st.y, cb, sb, 0.5f * tj.x,
                           0.5f * tj.y) > 0.f;
    }
  }
  hit = __any_sync(0xffffffffu, hit);
  if (lane == 0) e.coll[i] = hit ? 1 : 0;
}

// Warp per agent: box against the road-edge segments listed under the
// edge-grid cells touched by the box's bounding box.  Pedestrians may cross
// road edges.
__global__ void k_offroad(DevEnv e) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= e.A) return;
  if (e.flags[i] & (GD_FLAG_DONE | GD_FLAG_STATIC)) return;
  if (e.type[i] == GD_AGENT_PEDESTRIAN) {
    if (lane == 0) e.off[i] = 0;
    return;
  }
  const int w = e.agent_world[i];
  const GridDesc g = e.egrid[w];
  const float4 s = e.state[i];
  const float4 st = e.stat[i];
  float sa, ca;
  sincosf(s.z, &sa, &ca);
  const float hl = 0.5f * st.x, hw = 0.5f * st.y;
  const float ex = hl * fabsf(ca) + hw * fabsf(sa) + 1e-3f, ey = hl * fabsf(sa) + hw * fabsf(ca) + 1e-3f;
  const int cx0 = (int)clampf(floorf((s.x - ex - g.ox) * g.inv_cs), 0.f, (float)(g.nx - 1));
  const int cx1 = (int)clampf(floorf((s.x + ex - g.ox) * g.inv_cs), -1.f, (float)(g.nx - 1));
  const int cy0 = (int)clampf(floorf((s.y - ey - g.oy) * g.inv_cs), 0.f, (float)(g.ny - 1));
  const int cy1 = (int)clampf(floorf((s.y + ey - g.oy) * g.inv_cs), -1.f, (float)(g.ny - 1));
  bool hit = false;
  for (int cy = cy0; cy <= cy1; ++cy) {
    if (cx0 > cx1) break;
    const int b = e.ecell_start[g.cell_base + cy * g.nx + cx0];
    const int en = e.ecell_start[g.cell_base + cy * g.nx + cx1 + 1];
    for (int k = b + lane; k < en; k += WARP) hit |= box_seg_depth(s.x, s.y, ca, sa, hl, hw, e.esegs[k]) > 0.f;
  }
  hit = __any_sync(0xffffffffu, hit);
  if (lane == 0) e.off[i] = hit ? 1 : 0;
}

// Warp per world: goal test, reward, flags, done; then the world's episode
// step count and end-of-episode status: every controlled agent done (a world
// without controlled agents only times out) or t = T.  Uncontrolled agents
// score nothing and report done.
__global__ void k_finish(DevEnv e, float* __restrict__ reward, uint8_t* __restrict__ done,
                         uint8_t* __restrict__ world_done) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= e.W) return;
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  bool all_done = true, any_ctrl = false;
  for (int i = a0 + lane; i < a1; i += WARP) {
    uint8_t f = e.flags[i];
    float r = 0.f;
    if (!(f & (GD_FLAG_DONE | GD_FLAG_STATIC))) {
      const float4 s = e.state[i];
      const float4 st = e.stat[i];
      const float dx = s.x - st.z, dy = s.y - st.w;
      const bool at_goal = sqrtf(fmaf(dx, dx, __fmul_rn(dy, dy))) <= e.goal_r;
      const bool coll = e.coll[i] != 0, offr = e.off[i] != 0;
      const bool first = at_goal && !(f & GD_FLAG_GOAL);
      f &= (uint8_t)~(GD_FLAG_COLLIDED | GD_FLAG_OFFROAD);
      if (at_goal) f |= GD_FLAG_GOAL;
      if (coll) f |= GD_FLAG_COLLIDED;
      if (offr) f |= GD_FLAG_OFFROAD;
      if ((f & GD_FLAG_GOAL) || (coll && (e.cflags & GD_TERM_COLLISION)) || (offr && (e.cflags & GD_TERM_OFFROAD)))
        f |= GD_FLAG_DONE;
      e.flags[i] = f;
      r = (first ? 1.f : 0.f) - (coll ? e.cpen : 0.f) - (offr ? e.opn : 0.f);
    }
    if (reward) reward[i] = r;
    if (done) done[i] = (f & (GD_FLAG_DONE | GD_FLAG_STATIC)) ? 1 : 0;
    if (!(f & GD_FLAG_STATIC)) {
      any_ctrl = true;
      all_done = all_done && (f & GD_FLAG_DONE);
    }
  }
  all_done = __all_sync(0xffffffffu, all_done);
  any_ctrl = __any_sync(0xffffffffu, any_ctrl);
  if (lane == 0) {
    const int t = e.t[w] + 1;
    e.t[w] = t;
    const uint8_t wd = ((any_ctrl && all_done) || t >= e.T) ? 1 : 0;
    e.world_done[w] = wd;
    if (world_done) world_done[w] = wd;
  }
}

// Thread per world: episode-end status from flags and t (after gd_set_state).
__global__ void k_derive_world_done(DevEnv e) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= e.W) return;
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  bool all = true, any_ctrl = false;
  for (int i = a0; i < a1; ++i) {
    if (e.flags[i] & GD_FLAG_STATIC) continue;
    any_ctrl = true;
    all = all && (e.flags[i] & GD_FLAG_DONE);
  }
  e.world_done[w] = ((any_ctrl && all) || e.t[w] >= e.T) ? 1 : 0;
}

// Thread per agent, at create with GD_NONTRIVIAL_INIT ("all nontrivial"
// initialisation, Sec. 3.2 "Simulator sharp-edges"): agents within `dist` of
// their goal are not controlled.
__global__ void k_mark_uncontrolled(DevEnv e, uint8_t* __restrict__ init_flags, float dist) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.A) return;
  const float4 s = e.init_state[i];
  const float4 st = e.stat[i];
  const float dx = s.x - st.z, dy = s.y - st.w;
  if (sqrtf(fmaf(dx, dx, __fmul_rn(dy, dy))) <= dist) {
    init_flags[i] |= GD_FLAG_STATIC;
    e.flags[i] |= GD_FLAG_STATIC;
  }
}

// Grid-stride copy of a state snapshot (state and flags per agent, episode
// step and episode-end status per world) in one launch: the checkpoints of a
// differentiable rollout and the start of each recomputed segment.
struct Snapshot {
  float4* state;
  uint8_t* flags;
  int* t;
  uint8_t* world_done;
};
__global__ void k_copy_snapshot(Snapshot dst, Snapshot src, int A, int W) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A; i += stride) {
    dst.state[i] = src.state[i];
    dst.flags[i] = src.flags[i];
  }
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += stride) {
    dst.t[w] = src.t[w];
    dst.world_done[w] = src.world_done[w];
  }
}

}  // namespace gd
