// Expert-action inversion (Sec. 3.2 "Agent dynamics": expert actions computed
// from a trajectory and replayed to imitate it; the simplified model is the
// invertible one).
//
// For every agent and step of a trajectory of states (x, y, theta, v):
//   a = (v1 - v0) / dt                                    (both models)
//   simplified model: s = dtheta / ds, ds = v0 dt + a dt^2 / 2
//                     (0 when |ds| <= 1e-6 m)
//   kinematic bicycle: k = dtheta L / (v-bar dt), v-bar = v0 + a dt / 2,
//                     k clamped to +-1.99, delta = atan(k / sqrt(1 - k^2/4))
//                     (0 when |v-bar dt| <= 1e-6 m)
// with dtheta = theta1 - theta0 wrapped to [-pi, pi].  The simplified model
// replays exactly; the bicycle matches heading and speed (not the slip of
// the positions) while no speed is clipped.
//
// One thread per (agent, chunk of INV_CHUNK steps): the chunk's INV_CHUNK + 1
// float4 states are all loaded before any arithmetic (that many loads in
// flight per thread), each state once for two steps, and INV_CHUNK float2
// actions are written; consecutive threads take consecutive agents
// (coalesced).  Memory-bound.
#pragma once
#include "gd_device.cuh"

namespace gd {

__device__ __forceinline__ float2 invert_one(int dyn, float4 s0, float4 s1, float L, float dt) {
  const float a = __fdiv_rn(s1.w - s0.w, dt);
  const float dth = remainderf(s1.z - s0.z, 6.28318530717958648f);
  float steer = 0.f;
  if (dyn == 1) {
    const float ds = fmaf(__fmul_rn(0.5f, a), __fmul_rn(dt, dt), __fmul_rn(s0.w, dt));
    if (fabsf(ds) > 1e-6f) steer = __fdiv_rn(dth, ds);
  } else {
    const float vbdt = __fmul_rn(fmaf(__fmul_rn(0.5f, a), dt, s0.w), dt);
    if (fabsf(vbdt) > 1e-6f) {
      const float k = clampf(__fdiv_rn(__fmul_rn(dth, L), vbdt), -1.99f, 1.99f);
      steer = atanf(__fdiv_rn(k, sqrtf(fmaf(-0.25f * k, k, 1.f))));
    }
  }
  return make_float2(a, steer);
}

constexpr int INV_CHUNK = 8;

// states: [steps + 1, A] float4; actions: [steps, A] float2.  Grid: x over
// agents (blockDim.x each), y over chunks of INV_CHUNK steps.
__global__ void k_invert(DevEnv e, int steps, const float4* __restrict__ states, float2* __restrict__ actions) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.A) return;
  const int t0 = blockIdx.y * INV_CHUNK, t1 = min(t0 + INV_CHUNK, steps);
  const float L = e.stat[i].x;
  const size_t A = (size_t)e.A;
  // all loads of the chunk first (INV_CHUNK + 1 in flight per thread), then the arithmetic
  float4 st[INV_CHUNK + 1];
#pragma unroll
  for (int k = 0; k <= INV_CHUNK; ++k)
    if (t0 + k <= t1) st[k] = states[(size_t)(t0 + k) * A + i];
#pragma unroll
  for (int k = 0; k < INV_CHUNK; ++k)
    if (t0 + k < t1) actions[(size_t)(t0 + k) * A + i] = invert_one(e.dyn, st[k], st[k + 1], L, e.dt);
}

}  // namespace gd
