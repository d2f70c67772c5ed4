// Adjoint (reverse-mode derivative) of one simulator step.  The paper has
// no gradient; this differentiates the step it defines: the bicycle model
// of App. B (or the simplified model of Sec. 3.2 "Agent dynamics"), the
// ego-frame observation of Sec. 3.2 ("Sensor modalities")
// and a smooth goal reward r_s = -(sqrt(d_goal^2 + c^2) - c).  Collision,
// goal, done, selection and clip decisions are held constant (piecewise-
// constant parts of the step): the derivative of clip is 1 on [-v_max,
// v_max] (inclusive) and 0 outside.
//
// Objective of one step for agent i:
//   ell_i = m_i * ( sum_f w_f obs_i[f] + rw_i * r_s(i) * [i in the scene before the step] )
// with weight row w (shared or per agent), per-agent multiplier m_i and
// reward weight rw_i.  The kernel adds d ell / d(post-step state) to the
// incoming adjoint lam (d L / d post-step state from later steps) and maps
// it back through the dynamics:  lam <- J_s^T lam,  d_action = J_a^T lam.
//
// Two forms compute the same sums in the same order, so their gradients are
// bit-identical:
//   split (default), one launch pair per checkpoint segment: k_adj_observer,
//     persistent warps that claim (step, agent) tasks of the whole segment
//     one at a time (no per-world barrier, and every step of the segment in
//     one launch): re-run the forward selection from global memory (same
//     code, same state, so the same sets), accumulate the gradient on the
//     observer's own state (lanes over slots, shuffle-tree reduction) and
//     record which slot each partner sits in; then k_adj_dynamics, a thread
//     per agent that walks the segment's steps backwards with the adjoint in
//     registers: gather the gradient the agent receives as somebody's
//     partner in ascending order of the observer (a fixed order, so the sums
//     are deterministic), add the reward term, apply the dynamics adjoint;
//   fused: k_adjoint, one step per launch, one CTA per world (persistent,
//     work list as in the forward kernel), both parts with the world in
//     shared memory.
#pragma once
#include "gd_device.cuh"
#include "observe_kernel.cuh"
#include "world_kernel.cuh"

namespace gd {

// Adjoint of `steps` consecutive steps (a segment; the fused form takes one
// step, steps = 1).  Step k of the segment goes from S[k] to S[k + 1];
// every per-step array holds one [A] slice per step.
struct AdjArgs {
  const float4* S;          // [steps + 1][A] states: S[k] before step k, S[k + 1] after it
  const uint8_t* F;         // [steps + 1][A] flags, likewise
  const float2* actions;    // [steps][A] actions of the steps
  const float* obs_w;       // weight rows (obs_w + i * obs_w_stride), 16-byte aligned; nullptr = no obs term
  long long obs_w_stride;   // 0 = one row for every agent, F = one row per agent
  const float* row_scale;   // [steps][A] per-agent multiplier m_i, or nullptr (1)
  const float* rew_w;       // [A] per-agent reward weight (steps = 1 only), or nullptr (reward_w)
  float reward_w;
  float4* lam;              // [A] in: dL/d state after the last step; out: dL/d state before the first
  float2* d_actions;        // [steps][A] out: dL/d (accel, steer)
  const float* rk;          // [steps][A] each agent's K-th road distance at the step in the forward
                            // rollout (bounds the re-selection's disk), or nullptr: the full radius
  const uint16_t* sel;      // [steps][A][K] the forward rollout's road selections (split form), or
                            // nullptr: re-selected
  unsigned* counter;        // fused form: [2] work counter and exit tally, left at zero by each launch
  const int* order;
  int tile_bytes;
  int lam_zero;             // 1: the incoming lam is zero (the last step of a rollout); lam is not read
  float4* lam_copy;         // [A] or nullptr: a second copy of the outgoing lam (d_state0 of the first step)
  int steps;
  // split form, one slice per step of the segment
  float4* g_obs;            // [steps][A] observer-side gradient on each agent's own state (agents in the scene)
  float2* cs_obs;           // [steps][A] (cos, sin) of each observer's post-step heading (agents in the scene)
  uint8_t* slot;            // [steps][A][GD_MAX_AGENTS_PER_WORLD] slot of local partner j in observer i's row,
                            // 0xff = none
  unsigned* ocounter;       // [ADJ_STRIPES] task claims of k_adj_observer; k_adj_dynamics leaves them at zero
};

constexpr unsigned ADJ_STRIPES = 256;

struct AdjAgents {
  float4 st[GD_MAX_AGENTS_PER_WORLD];   // post-step state
  float4 sc[GD_MAX_AGENTS_PER_WORLD];
  float4 g[GD_MAX_AGENTS_PER_WORLD];    // observation gradient on the agent's own state
  float2 cs[GD_MAX_AGENTS_PER_WORLD];
  uint8_t fl[GD_MAX_AGENTS_PER_WORLD];  // post-step flags
  uint8_t slot_of[GD_MAX_AGENTS_PER_WORLD][GD_MAX_AGENTS_PER_WORLD];  // [observer][partner], 0xff = none
};

// Bicycle-model adjoint (App. B): lam holds dL/d(x', y', theta', v') and
// becomes dL/d(x, y, theta, v); da = dL/d(accel, steer).  With t = tan(delta):
// d beta/d delta = 2 (1 + t^2) / (4 + t^2) and, for k = cos(beta) tan(delta)
// = 2 t / sqrt(4 + t^2), dk/d delta = 8 (1 + t^2) / (4 + t^2)^(3/2).
__device__ __forceinline__ void bicycle_adjoint(const float4 s, float accel, float steer, float L, float dt, float vmax,
                                                float4& lam, float2& da) {
  const float u = fmaf(__fmul_rn(0.5f, accel), dt, s.w);
  const float m1 = (u >= -vmax && u <= vmax) ? 1.f : 0.f;
  const float vbar = clampf(u, -vmax, vmax);
  const float t = tanf(steer);
  const float beta = atanf(__fmul_rn(0.5f, t));
  float sp, cp;
  sincosf(__fadd_rn(s.z, beta), &sp, &cp);
  const float k = __fmul_rn(cosf(beta), t);
  const float u2 = fmaf(accel, dt, s.w);
  const float m2 = (u2 >= -vmax && u2 <= vmax) ? 1.f : 0.f;
  const float g_vbar = fmaf(fmaf(lam.x, cp, __fmul_rn(lam.y, sp)), dt, __fmul_rn(lam.z, k) * dt / L);
  const float g_phi = fmaf(-lam.x, sp, __fmul_rn(lam.y, cp)) * vbar * dt;
  const float g_k = lam.z * vbar * dt / L;
  const float t2 = t * t, q = 4.f + t2;
  const float dbeta = 2.f * (1.f + t2) / q;
  const float dk = 8.f * (1.f + t2) / (q * sqrtf(q));
  da.x = fmaf(g_vbar * m1, 0.5f * dt, lam.w * m2 * dt);
  da.y = fmaf(g_phi, dbeta, g_k * dk);
  lam.z = lam.z + g_phi;
  lam.w = fmaf(g_vbar, m1, lam.w * m2);
}

// Adjoint of the simplified invertible model (Sec. 3.2 "Agent dynamics"):
// ds = v dt + a dt^2 / 2, x' = x + cos(theta) ds, y' = y + sin(theta) ds,
// theta' = theta + k ds, v' = v + a dt, so with g = dL/d ds =
// lam_x cos + lam_y sin + lam_theta k: dL/d theta = lam_theta + ds (-lam_x
// sin + lam_y cos), dL/dv = lam_v + g dt, dL/da = g dt^2 / 2 + lam_v dt,
// dL/dk = lam_theta ds.
__device__ __forceinline__ void invertible_adjoint(const float4 s, float accel, float curv, float dt, float4& lam,
                                                   float2& da) {
  const float ds = fmaf(__fmul_rn(0.5f, accel), __fmul_rn(dt, dt), __fmul_rn(s.w, dt));
  float sn, cs;
  sincosf(s.z, &sn, &cs);
  const float g = fmaf(lam.x, cs, fmaf(lam.y, sn, __fmul_rn(lam.z, curv)));
  da.x = fmaf(__fmul_rn(g, 0.5f * dt), dt, __fmul_rn(lam.w, dt));
  da.y = __fmul_rn(lam.z, ds);
  lam.z = fmaf(ds, fmaf(-lam.x, sn, __fmul_rn(lam.y, cs)), lam.z);
  lam.w = fmaf(g, dt, lam.w);
}

// ---- arithmetic shared by both forms ---------------------------------------

// Observer side of agent li's row (post-step state st, heading (c, s), weight
// row wrow): d (w . row) / d(own state) as (x, y, theta, v), summed over the
// ego features, the partner slots and the road slots (lanes over slots, then
// a shuffle tree), returned to every lane.  on_partner(r, j) is called once
// per selected partner (slot r, local index j) by the lane that handles it.
// The road selection is re-run (over the disk of radius Rs), or, given
// selrow, read from the forward rollout's record of the same step: the same
// positions in the same slots, so the sums are the same.
template <typename OnPartner>
__device__ __forceinline__ float4 observer_gradient(const DevEnv& e, const WorldView& v, int li, float4 st, float4 sc,
                                                    float c, float s, const float* __restrict__ wrow, float Rs,
                                                    float Rs2, ObsWarpSmem& sm, int lane, OnPartner&& on_partner,
                                                    const uint16_t* __restrict__ selrow = nullptr) {
  float gx = 0.f, gy = 0.f, gt = 0.f, gv = 0.f;
  if (lane == 0) {
    // ego: speed and goal offset in the ego frame
    const float dx = sc.z - st.x, dy = sc.w - st.y;
    const float f3 = rot_x(c, s, dx, dy), f4 = rot_y(c, s, dx, dy);
    const float w3 = __ldg(wrow + 3), w4 = __ldg(wrow + 4);
    gv = __ldg(wrow + 0);
    gx = fmaf(-c, w3, __fmul_rn(s, w4));
    gy = fmaf(-s, w3, -__fmul_rn(c, w4));
    gt = fmaf(w3, f4, -__fmul_rn(w4, f3));
  }
  // partners: the observer side here, the partner side in the gather
  const int np = select_partners(v, li, e.P, e.R2, st.x, st.y, sm, lane);
  for (int r = lane; r < np; r += WARP) {
    const int j = sm.psel[r];
    on_partner(r, j);
    const float4 wa = __ldg(reinterpret_cast<const float4*>(wrow + 8 + 8 * r));
    const float4 q = v.state[j];
    float2 cj;
    if (v.cs) cj = v.cs[j]; else sincosf(q.z, &cj.y, &cj.x);
    const float dx = q.x - st.x, dy = q.y - st.y;
    const float xp = rot_x(c, s, dx, dy), yp = rot_y(c, s, dx, dy);
    const float cd = rot_x(c, s, cj.x, cj.y), sd = rot_y(c, s, cj.x, cj.y);
    gx += fmaf(-c, wa.x, __fmul_rn(s, wa.y));
    gy += fmaf(-s, wa.x, -__fmul_rn(c, wa.y));
    gt += fmaf(wa.x, yp, -__fmul_rn(wa.y, xp)) + fmaf(wa.z, sd, -__fmul_rn(wa.w, cd));
  }
  const float* wroad = wrow + 8 + 8 * e.P;
  auto road_term = [&](int r, unsigned pos) {
    const float2 q = v.xy[pos];
    const float dx = q.x - st.x, dy = q.y - st.y;
    const float xp = rot_x(c, s, dx, dy), yp = rot_y(c, s, dx, dy);
    const float wa = __ldg(wroad + 4 * r), wb = __ldg(wroad + 4 * r + 1);
    gx += fmaf(-c, wa, __fmul_rn(s, wb));
    gy += fmaf(-s, wa, -__fmul_rn(c, wb));
    gt += fmaf(wa, yp, -__fmul_rn(wb, xp));
  };
  if (selrow) {
    // the recorded selection: a lane's slots r = lane, lane + 32, ... in
    // order, their positions loaded four at a time
    constexpr int U = 4;
    for (int r0 = 0; r0 < e.K; r0 += U * WARP) {
      unsigned pos[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u * WARP + lane;
        pos[u] = r < e.K ? (unsigned)selrow[r] : (unsigned)OBS_SEL_NONE;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (pos[u] != OBS_SEL_NONE) road_term(r0 + u * WARP + lane, pos[u]);
    }
  } else {
    // road points: the forward selection's K-th distance bounds the disk
    // that holds the same K points (the full radius when it had fewer than K)
    int nroad = select_road(v, e.K, Rs, Rs2, st.x, st.y, sm, lane, e.topk);
    if (nroad < e.K && Rs < e.R) nroad = select_road(v, e.K, e.R, e.R2, st.x, st.y, sm, lane, e.topk);
    for (int r = lane; r < nroad; r += WARP) road_term(r, sel_pos(sm.sel[r]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
    gt += __shfl_xor_sync(0xffffffffu, gt, o);
  }
  return make_float4(gx, gy, gt, gv);
}

// Radius of the re-selection of agent i at step k: the forward step's K-th
// road distance + 1e-3 m when it is below R, else R.
__device__ __forceinline__ void reselect_radius(const DevEnv& e, const AdjArgs& a, int k, int i, float& Rs,
                                                float& Rs2) {
  Rs = e.R;
  Rs2 = e.R2;
  if (a.rk) {
    const float r = a.rk[(size_t)k * e.A + i] + 1e-3f;
    if (r < e.R) {
      Rs = r;
      Rs2 = r * r;
    }
  }
}

// Partner side: the gradient agent j (heading (cj.x, cj.y)) receives from
// observer i (heading (ci, si), weight row wrow, multiplier m) that holds it
// in slot r.
__device__ __forceinline__ void partner_term(float4& g, float ci, float si, float2 cj, const float* __restrict__ wrow,
                                             int r, float m) {
  const float4 wa = __ldg(reinterpret_cast<const float4*>(wrow + 8 + 8 * r));
  const float we = __ldg(wrow + 8 + 8 * r + 4);
  const float cd = rot_x(ci, si, cj.x, cj.y), sd = rot_y(ci, si, cj.x, cj.y);
  g.x += m * fmaf(ci, wa.x, -__fmul_rn(si, wa.y));
  g.y += m * fmaf(si, wa.x, __fmul_rn(ci, wa.y));
  g.z += m * fmaf(-wa.z, sd, __fmul_rn(wa.w, cd));
  g.w += m * we;
}

// Last part of step k for agent ig: the smooth goal reward term (a
// controlled agent in the scene before the step), lam += g, then the
// dynamics adjoint, which takes lam back to the state before the step;
// writes d_actions of the step.  st, sc: post-step state and extents/goal.
__device__ __forceinline__ void finish_step(const DevEnv& e, const AdjArgs& a, int k, int ig, float4 g, float4 st,
                                            float4 sc, float4& lam) {
  const size_t ik = (size_t)k * e.A + ig;
  const uint8_t f0 = a.F[ik];
  if (!(f0 & (GD_FLAG_DONE | GD_FLAG_STATIC))) {
    const float m = a.row_scale ? a.row_scale[ik] : 1.f;
    const float rw = (a.rew_w ? a.rew_w[ig] : a.reward_w) * m;
    const float dx = st.x - sc.z, dy = st.y - sc.w, c = e.smooth_c;
    const float qn = sqrtf(fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(c, c))));
    g.x -= rw * dx / qn;
    g.y -= rw * dy / qn;
  }
  lam.x += g.x;
  lam.y += g.y;
  lam.z += g.z;
  lam.w += g.w;
  float2 da = make_float2(0.f, 0.f);
  if (!(f0 & (GD_FLAG_DONE | GD_FLAG_STATIC))) {      // done and uncontrolled agents do not move
    const float2 u = a.actions[ik];
    if (e.dyn == 1) invertible_adjoint(a.S[ik], u.x, u.y, e.dt, lam, da);
    else bicycle_adjoint(a.S[ik], u.x, u.y, sc.x, e.dt, e.vmax, lam, da);
  }
  a.d_actions[ik] = da;
}

// ---- fused form --------------------------------------------------------------

// Dynamic shared memory: [mbarrier, 128 B][road tile][AdjAgents][ObsWarpSmem x WARPS]
// LEAN: the instantiation for the form without the road tile, whose shared
// memory leaves room for 32 warps per SM; registers are capped at 64 per
// thread (no spills) so that they can all be resident.  Worlds come from a
// counter that the last CTA out leaves at zero (no memset between launches).
template <int WARPS, bool LEAN = false>
__global__ void __launch_bounds__(WARPS * 32, LEAN ? 32 / WARPS : 1) k_adjoint(DevEnv e, AdjArgs a) {
  extern __shared__ __align__(16) unsigned char asm_[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(asm_);
  unsigned char* tile = asm_ + 128;
  AdjAgents& ag = *reinterpret_cast<AdjAgents*>(asm_ + 128 + (size_t)a.tile_bytes);
  ObsWarpSmem* wsmem = reinterpret_cast<ObsWarpSmem*>(reinterpret_cast<unsigned char*>(&ag) + sizeof(AdjAgents));
  __shared__ int s_w, s_abort, s_next;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  ObsWarpSmem& sm = wsmem[wid];
  if (tid == 0) {
    mbar_init(bar, 1);
    s_abort = 0;
  }
  __syncthreads();
  unsigned phase = 0;
  const bool obs_term = a.obs_w != nullptr;
  for (;;) {
    if (tid == 0) s_w = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int k = s_w;
    if (k >= e.W) break;
    const int w = a.order[k];
    const int a0 = e.agent_off[w], n = e.agent_off[w + 1] - a0;
    const int nr = e.road_off[w + 1] - e.road_off[w];
    const GridDesc g = e.rgrid[w];
    const unsigned block = (unsigned)g.block_bytes;
    const unsigned char* gblock = e.arena + (size_t)e.arena_off[w] * 16;
    const bool use_tile = obs_term && nr > 0 && block <= (unsigned)a.tile_bytes && (unsigned)n * TILE_AGENT_BYTES >= block;
    if (use_tile && tid == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, block);
      tma_load_1d(tile, gblock, block, bar);
    }
    if (tid == 0) s_next = WARPS;
    if (tid < n) {
      const float4 s = a.S[(size_t)e.A + a0 + tid];
      ag.st[tid] = s;
      float sn, cn;
      sincosf(s.z, &sn, &cn);
      ag.cs[tid] = make_float2(cn, sn);
      ag.sc[tid] = e.stat[a0 + tid];
      ag.fl[tid] = a.F[(size_t)e.A + a0 + tid];
      ag.g[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int q = tid; q < n * n; q += WARPS * 32) ag.slot_of[q / n][q % n] = 0xff;
    if (use_tile) {
      if (!mbar_wait_bounded(bar, phase)) s_abort = 1;
      phase ^= 1u;
    }
    __syncthreads();
    if (s_abort) {
      // the copy did not land in time: record it, give the copy one more
      // bounded chance, and leave the world loop (the exit tally below still
      // counts this CTA out)
      if (tid == 0) {
        atomicOr(e.err, ERR_TIMEOUT);
        mbar_wait_bounded(bar, phase ^ 1u);
      }
      __syncthreads();
      break;
    }
    if (obs_term) {
      WorldView v;
      v.state = ag.st;
      v.stat = ag.sc;
      v.cs = ag.cs;
      v.flags = ag.fl;
      v.n = n;
      road_block(use_tile ? tile : gblock, nr, v);
      v.g = g;
      for (int li = wid; li < n;) {
        if (!(ag.fl[li] & GD_FLAG_DONE)) {
          const int i = a0 + li;
          float Rs, Rs2;
          reselect_radius(e, a, 0, i, Rs, Rs2);
          const float4 gr = observer_gradient(e, v, li, ag.st[li], ag.sc[li], ag.cs[li].x, ag.cs[li].y,
                                              a.obs_w + (size_t)i * a.obs_w_stride, Rs, Rs2, sm, lane,
                                              [&](int r, int j) { ag.slot_of[li][j] = (uint8_t)r; });
          if (lane == 0) {
            const float m = a.row_scale ? a.row_scale[i] : 1.f;
            ag.g[li] = make_float4(m * gr.x, m * gr.y, m * gr.z, m * gr.w);
          }
          __syncwarp();
        }
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&s_next, 1);
        li = __shfl_sync(0xffffffffu, nx, 0);
      }
    }
    __syncthreads();
    if (tid < n) {
      const int j = tid, ig = a0 + j;
      float4 gj = ag.g[j];
      if (obs_term) {
        // partner side: every observer i that has j in slot r, ascending i
        const float2 cj = ag.cs[j];
        for (int i = 0; i < n; ++i) {
          const int r = ag.slot_of[i][j];
          if (r == 0xff) continue;
          partner_term(gj, ag.cs[i].x, ag.cs[i].y, cj, a.obs_w + (size_t)(a0 + i) * a.obs_w_stride, r,
                       a.row_scale ? a.row_scale[a0 + i] : 1.f);
        }
      }
      float4 lam = a.lam_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : a.lam[ig];
      finish_step(e, a, 0, ig, gj, ag.st[j], ag.sc[j], lam);
      a.lam[ig] = lam;
      if (a.lam_copy) a.lam_copy[ig] = lam;
    }
    __syncthreads();
  }
  // the last CTA out leaves the work counter and the exit tally at zero for
  // the next launch (every CTA has made its last claim before it counts out)
  __syncthreads();
  if (tid == 0 && atomicAdd(a.counter + 1, 1u) == gridDim.x - 1) {
    a.counter[0] = 0u;
    a.counter[1] = 0u;
  }
}

// ---- split form ----------------------------------------------------------------

// Part 1: persistent warps claim (step, agent) tasks of the segment, step
// major, one at a time from ADJ_STRIPES striped counters (warp g draws tasks
// c, c + ADJ_STRIPES, ... from counter c = g mod ADJ_STRIPES; the counters
// are zero at launch) and, for an agent in the scene after the step,
// re-select its row from global memory (the world's agents and road block
// through L1/L2) and write its observer-side gradient g_obs (times m_i), its
// heading's (cos, sin) and its slot row: slot[i][j] = the slot of local
// partner j, 0xff for every other agent.  A done agent's row is all 0xff.
// Dynamic shared memory: WARPS x (ObsWarpSmem + 128 B).  Registers capped
// for 32 warps per SM.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) k_adj_observer(DevEnv e, AdjArgs a) {
  extern __shared__ __align__(16) unsigned char adj_smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  ObsWarpSmem& sm = reinterpret_cast<ObsWarpSmem*>(adj_smem_raw)[wid];
  uint8_t* srow = adj_smem_raw + WARPS * sizeof(ObsWarpSmem) + wid * GD_MAX_AGENTS_PER_WORLD;
  static_assert(GD_MAX_AGENTS_PER_WORLD == 4 * WARP, "a slot row is one 32-bit word per lane");
  const unsigned c = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) % ADJ_STRIPES;
  const unsigned tasks = (unsigned)a.steps * (unsigned)e.A;
  // the next task is claimed as soon as the current one is known, so the
  // claim's round trip overlaps the task's loads
  unsigned kn = 0;
  if (lane == 0) kn = atomicAdd(a.ocounter + c, 1u);
  for (;;) {
    const unsigned kk = __shfl_sync(0xffffffffu, kn, 0);
    const unsigned q = c + ADJ_STRIPES * kk;
    if (q >= tasks) break;
    if (lane == 0) kn = atomicAdd(a.ocounter + c, 1u);
    const int k = (int)(q / (unsigned)e.A), i = (int)(q - (unsigned)k * (unsigned)e.A);
    const size_t ik = (size_t)k * e.A + i;
    const float4* post = a.S + (size_t)(k + 1) * e.A;
    const uint8_t* fpost = a.F + (size_t)(k + 1) * e.A;
    unsigned* grow = reinterpret_cast<unsigned*>(a.slot + ik * GD_MAX_AGENTS_PER_WORLD);
    if (fpost[i] & GD_FLAG_DONE) {
      grow[lane] = 0xffffffffu;
      continue;
    }
    reinterpret_cast<unsigned*>(srow)[lane] = 0xffffffffu;
    __syncwarp();
    const float4 st = post[i], sc = e.stat[i];
    const int w = e.agent_world[i];
    const int a0 = e.agent_off[w];
    WorldView v;
    v.state = post + a0;
    v.stat = e.stat + a0;
    v.cs = nullptr;
    v.flags = fpost + a0;
    v.n = e.agent_off[w + 1] - a0;
    road_block(e.arena + (size_t)e.arena_off[w] * 16, e.road_off[w + 1] - e.road_off[w], v);
    v.g = e.rgrid[w];
    float sn, cn;
    sincosf(st.z, &sn, &cn);
    float Rs, Rs2;
    reselect_radius(e, a, k, i, Rs, Rs2);
    const float4 gr = observer_gradient(e, v, i - a0, st, sc, cn, sn, a.obs_w + (size_t)i * a.obs_w_stride, Rs,
                                        Rs2, sm, lane, [&](int r, int j) { srow[j] = (uint8_t)r; },
                                        a.sel ? a.sel + ik * e.K : nullptr);
    __syncwarp();
    grow[lane] = reinterpret_cast<const unsigned*>(srow)[lane];
    if (lane == 0) {
      const float m = a.row_scale ? a.row_scale[ik] : 1.f;
      a.g_obs[ik] = make_float4(m * gr.x, m * gr.y, m * gr.z, m * gr.w);
      a.cs_obs[ik] = make_float2(cn, sn);
    }
    __syncwarp();
  }
}

// Part 2: thread per agent j (flat over all agents), the segment's steps
// last to first with the adjoint in registers: per step its own
// observer-side gradient, the partner side from every observer i of its
// world that holds it (ascending i, the fused form's order), the reward term
// and the dynamics adjoint.  Block 0 leaves part 1's claim counters at zero
// for the next part-1 launch.
__global__ void __launch_bounds__(64) k_adj_dynamics(DevEnv e, AdjArgs a) {
  if (blockIdx.x == 0)
    for (unsigned c = threadIdx.x; c < ADJ_STRIPES; c += blockDim.x) a.ocounter[c] = 0u;
  const int ig = blockIdx.x * blockDim.x + threadIdx.x;
  if (ig >= e.A) return;
  const float4 sc = e.stat[ig];
  const int w = e.agent_world[ig];
  const int a0 = e.agent_off[w], n = e.agent_off[w + 1] - a0, j = ig - a0;
  float4 lam = a.lam_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : a.lam[ig];
  for (int k = a.steps - 1; k >= 0; --k) {
    const size_t ik = (size_t)k * e.A + ig;
    const float4 st = a.S[ik + e.A];
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.obs_w) {
      if (!(a.F[ik + e.A] & GD_FLAG_DONE)) g = a.g_obs[ik];
      float2 cj;
      sincosf(st.z, &cj.y, &cj.x);
      const size_t ko = (size_t)k * e.A + a0;       // the world's first agent at step k
      const uint8_t* col = a.slot + ko * GD_MAX_AGENTS_PER_WORLD + j;
      // the column's bytes are read eight at a time, so their loads overlap
      for (int i0 = 0; i0 < n; i0 += 8) {
        uint8_t rr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) rr[u] = i0 + u < n ? col[(size_t)(i0 + u) * GD_MAX_AGENTS_PER_WORLD] : (uint8_t)0xff;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (rr[u] == 0xff) continue;
          const int i = i0 + u;
          const float2 ci = a.cs_obs[ko + i];
          partner_term(g, ci.x, ci.y, cj, a.obs_w + (size_t)(a0 + i) * a.obs_w_stride, rr[u],
                       a.row_scale ? a.row_scale[ko + i] : 1.f);
        }
      }
    }
    finish_step(e, a, k, ig, g, st, sc, lam);
  }
  a.lam[ig] = lam;
  if (a.lam_copy) a.lam_copy[ig] = lam;
}

}  // namespace gd
