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
// One CTA per world (persistent, work list as in the forward kernel).
// Warp per agent: re-run the forward selection (same code, same state, so
// the same sets), accumulate the gradient on its own state (lanes over
// slots, shuffle-tree reduction) and record which slot each partner sits in.
// Thread per agent: gather the gradient it receives as somebody's partner in
// ascending order of the observer (a fixed order, so the sums are
// deterministic), add the reward term, apply the dynamics adjoint.
#pragma once
#include "gd_device.cuh"
#include "observe_kernel.cuh"
#include "world_kernel.cuh"

namespace gd {

struct AdjArgs {
  const float4* pre;        // [A] state before the step
  const uint8_t* fpre;      // [A] flags before the step
  const float4* post;       // [A] state after the step
  const uint8_t* fpost;     // [A] flags after the step
  const float2* actions;    // [A] actions of the step
  const float* obs_w;       // weight rows (obs_w + i * obs_w_stride), 16-byte aligned; nullptr = no obs term
  long long obs_w_stride;   // 0 = one row for every agent, F = one row per agent
  const float* row_scale;   // [A] per-agent multiplier m_i, or nullptr (1)
  const float* rew_w;       // [A] per-agent reward weight, or nullptr (reward_w)
  float reward_w;
  float4* lam;              // [A] in: dL/d post-step state; out: dL/d pre-step state
  float2* d_actions;        // [A] out: dL/d (accel, steer)
  const float* rk;          // [A] each agent's K-th road distance at this step in the forward rollout
                            // (bounds the re-selection's disk), or nullptr: the full radius
  unsigned* counter;
  const int* order;
  int tile_bytes;
};

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

// Dynamic shared memory: [mbarrier, 128 B][road tile][AdjAgents][ObsWarpSmem x WARPS]
// LEAN: the instantiation for the form without the road tile, whose shared
// memory leaves room for 32 warps per SM; registers are capped at 64 per
// thread (no spills) so that they can all be resident.
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
      const float4 s = a.post[a0 + tid];
      ag.st[tid] = s;
      float sn, cn;
      sincosf(s.z, &sn, &cn);
      ag.cs[tid] = make_float2(cn, sn);
      ag.sc[tid] = e.stat[a0 + tid];
      ag.fl[tid] = a.fpost[a0 + tid];
      ag.g[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int q = tid; q < n * n; q += WARPS * 32) ag.slot_of[q / n][q % n] = 0xff;
    if (use_tile) {
      if (!mbar_wait_bounded(bar, phase)) s_abort = 1;
      phase ^= 1u;
    }
    __syncthreads();
    if (s_abort) {
      if (tid == 0) {
        atomicOr(e.err, ERR_TIMEOUT);
        mbar_wait_bounded(bar, phase ^ 1u);
      }
      __syncthreads();
      return;
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
          const float* wrow = a.obs_w + (size_t)i * a.obs_w_stride;
          const float4 st = ag.st[li], sc = ag.sc[li];
          const float c = ag.cs[li].x, s = ag.cs[li].y;
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
          // partners: the observer side here, the partner side in the gather below
          const int np = select_partners(v, li, e.P, e.R2, st.x, st.y, sm, lane);
          for (int r = lane; r < np; r += WARP) {
            const int j = sm.psel[r];
            ag.slot_of[li][j] = (uint8_t)r;
            const float4 wa = __ldg(reinterpret_cast<const float4*>(wrow + 8 + 8 * r));
            const float4 q = ag.st[j];
            const float dx = q.x - st.x, dy = q.y - st.y;
            const float xp = rot_x(c, s, dx, dy), yp = rot_y(c, s, dx, dy);
            const float cd = rot_x(c, s, ag.cs[j].x, ag.cs[j].y), sd = rot_y(c, s, ag.cs[j].x, ag.cs[j].y);
            gx += fmaf(-c, wa.x, __fmul_rn(s, wa.y));
            gy += fmaf(-s, wa.x, -__fmul_rn(c, wa.y));
            gt += fmaf(wa.x, yp, -__fmul_rn(wa.y, xp)) + fmaf(wa.z, sd, -__fmul_rn(wa.w, cd));
          }
          // road points
          // the forward selection's K-th distance bounds the disk that holds
          // the same K points (the full radius when it had fewer than K)
          float Rs = e.R, Rs2 = e.R2;
          if (a.rk) {
            const float r = a.rk[i] + 1e-3f;
            if (r < e.R) {
              Rs = r;
              Rs2 = r * r;
            }
          }
          int nroad = select_road(v, e.K, Rs, Rs2, st.x, st.y, sm, lane, e.topk);
          if (nroad < e.K && Rs < e.R) nroad = select_road(v, e.K, e.R, e.R2, st.x, st.y, sm, lane, e.topk);
          const float* wroad = wrow + 8 + 8 * e.P;
          for (int r = lane; r < nroad; r += WARP) {
            const float2 q = v.xy[sel_pos(sm.sel[r])];
            const float dx = q.x - st.x, dy = q.y - st.y;
            const float xp = rot_x(c, s, dx, dy), yp = rot_y(c, s, dx, dy);
            const float wa = __ldg(wroad + 4 * r), wb = __ldg(wroad + 4 * r + 1);
            gx += fmaf(-c, wa, __fmul_rn(s, wb));
            gy += fmaf(-s, wa, -__fmul_rn(c, wb));
            gt += fmaf(wa, yp, -__fmul_rn(wb, xp));
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gt += __shfl_xor_sync(0xffffffffu, gt, o);
          }
          if (lane == 0) {
            const float m = a.row_scale ? a.row_scale[i] : 1.f;
            ag.g[li] = make_float4(m * gx, m * gy, m * gt, m * gv);
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
      float4 g = ag.g[j];
      if (obs_term) {
        // partner side: every observer i that has j in slot r, ascending i
        const float4 q = ag.st[j];
        const float2 cj = ag.cs[j];
        for (int i = 0; i < n; ++i) {
          const int r = ag.slot_of[i][j];
          if (r == 0xff) continue;
          const float ci = ag.cs[i].x, si = ag.cs[i].y;
          const float* wrow = a.obs_w + (size_t)(a0 + i) * a.obs_w_stride;
          const float4 wa = __ldg(reinterpret_cast<const float4*>(wrow + 8 + 8 * r));
          const float we = __ldg(wrow + 8 + 8 * r + 4);
          const float m = a.row_scale ? a.row_scale[a0 + i] : 1.f;
          const float cd = rot_x(ci, si, cj.x, cj.y), sd = rot_y(ci, si, cj.x, cj.y);
          g.x += m * fmaf(ci, wa.x, -__fmul_rn(si, wa.y));
          g.y += m * fmaf(si, wa.x, __fmul_rn(ci, wa.y));
          g.z += m * fmaf(-wa.z, sd, __fmul_rn(wa.w, cd));
          g.w += m * we;
        }
        (void)q;
      }
      const uint8_t f0 = a.fpre[ig];
      if (!(f0 & (GD_FLAG_DONE | GD_FLAG_STATIC))) {
        // smooth goal reward of a controlled agent in the scene before the step
        const float m = a.row_scale ? a.row_scale[ig] : 1.f;
        const float rw = (a.rew_w ? a.rew_w[ig] : a.reward_w) * m;
        const float4 st = ag.st[j], sc = ag.sc[j];
        const float dx = st.x - sc.z, dy = st.y - sc.w, c = e.smooth_c;
        const float qn = sqrtf(fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(c, c))));
        g.x -= rw * dx / qn;
        g.y -= rw * dy / qn;
      }
      float4 lam = a.lam[ig];
      lam.x += g.x;
      lam.y += g.y;
      lam.z += g.z;
      lam.w += g.w;
      float2 da = make_float2(0.f, 0.f);
      if (!(f0 & (GD_FLAG_DONE | GD_FLAG_STATIC))) {      // done and uncontrolled agents do not move
        const float2 u = a.actions[ig];
        if (e.dyn == 1) invertible_adjoint(a.pre[ig], u.x, u.y, e.dt, lam, da);
        else bicycle_adjoint(a.pre[ig], u.x, u.y, ag.sc[j].x, e.dt, e.vmax, lam, da);
      }
      a.lam[ig] = lam;
      a.d_actions[ig] = da;
    }
    __syncthreads();
  }
}

}  // namespace gd
