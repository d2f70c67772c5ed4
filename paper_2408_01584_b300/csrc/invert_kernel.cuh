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
// One thread per (step, agent), grid-stride; reads two float4 states and the
// length, writes one float2: memory-bound.
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

// states: [steps + 1, A] float4; actions: [steps, A] float2.
__global__ void k_invert(DevEnv e, int steps, const float4* __restrict__ states, float2* __restrict__ actions) {
  const long long n = (long long)steps * e.A;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % e.A);
    actions[q] = invert_one(e.dyn, states[q], states[q + e.A], e.stat[i].x, e.dt);
  }
}

}  // namespace gd
