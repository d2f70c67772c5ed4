// Device-side data layout and per-agent arithmetic of the driving step.
//
// Layout in HBM (all arrays in CSR world order, see include/gd.h):
//   state[A]       float4 (x, y, theta, v)        -- 16 B, one coalesced load
//   stat[A]        float4 (length, width, goal_x, goal_y)
//   flags[A]       uint8  GD_FLAG_* bits
//   arena          per world one 16-byte aligned block: road_pad(N_w) float2
//                  (x, y), road_pad(N_w) uint16 (local index | type << 15),
//                  road_pad(N_w) uint16 "next" (block position of the next point
//                  when the two form a road-edge segment, else 0xffff), all
//                  sorted by road-grid cell so that a row of cells is one range,
//                  then the (ny*nx + 1) uint16 cell starts; arena_off[w] is the
//                  block's offset in 16-byte units, rgrid[w].block_bytes its size
//   esegs[]        float4 (x0, y0, x1, y1) road-edge segments listed under every
//                  edge-grid cell their bounding box touches
//   anchor[A]      float4 (x, y, r_K, 0): where each agent last selected its road
//                  points and the distance of the K-th (+inf if fewer than K were
//                  in range); it bounds the next selection's disk
//   lsegs[]        float4 (x0, y0, x1, y1) road-edge segments of each world, each
//                  listed once, under the road-grid cell of its first point, in
//                  cell order; lcell[rgrid[w].cell_base + c] = first segment of
//                  cell c of world w (ny*nx + 1 entries per world)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gd.h"

namespace gd {

constexpr unsigned ERR_ACTION = 1u;     // non-finite action, or |steer| >= pi/2 (kinematic bicycle)
constexpr unsigned ERR_TIMEOUT = 2u;    // a bounded wait gave up
constexpr unsigned ERR_CAPACITY = 4u;   // a device-side capacity was exceeded

constexpr int WARP = 32;

// Points of a world's road block, padded so the block is a multiple of 16 B.
__host__ __device__ __forceinline__ int road_pad(int nr) { return (nr + 7) & ~7; }
// Bytes of a world's road block: points (12 B each, padded) + cell starts.
__host__ __device__ __forceinline__ int road_block_bytes(int nr, int ncells) {
  return road_pad(nr) * 12 + ((2 * (ncells + 1) + 15) & ~15);
}
constexpr unsigned short NO_SEGMENT = 0xffff;
constexpr int MAX_ROWS = 32;            // grid rows spanned by one observation disk

struct GridDesc {      // one per world, for the road-point grid and the edge grid
  float ox, oy;        // lower-left corner of cell (0, 0)
  float cs, inv_cs;    // cell size and its inverse
  int nx, ny;          // cells per row / rows
  int cell_base;       // edge grid: first entry of this world's cell-start table;
                       // road grid: first entry of the world's table in lcell
  float seg_max;       // road grid: longest road-edge segment of the world (m)
  int block_bytes;     // road grid: bytes of the world's road block in the arena
};

// Everything a kernel needs, passed by value (device pointers + sizes).
struct DevEnv {
  int W, A, N, K, P, F, T;
  float R, R2, goal_r, dt, vmax, cpen, opn, smooth_c, agent_cell;
  int topk;              // road top-K: 1 = bucket rank, 2 = bitonic sort when <= 256 points are in range
  unsigned* smemo;       // [A][K] the last road selection (key low words) of each parked agent, or nullptr
  unsigned road_epoch;   // layout number of the road blocks (a rebuild changes it): tags the memo in the anchor
  int dyn;               // 0: kinematic bicycle (App. B); 1: simplified invertible model (Sec. 3.2)
  uint32_t cflags;
  const int* agent_off;
  const int* road_off;
  const int* agent_world;
  float4* state;
  const float4* init_state;
  const float4* stat;
  const uint8_t* type;
  uint8_t* flags;
  const uint8_t* init_flags;
  int* t;
  uint8_t* world_done;
  const GridDesc* rgrid;
  const unsigned char* arena;
  const long long* arena_off;
  const GridDesc* egrid;
  const int* ecell_start;
  const float4* esegs;
  float4* anchor;        // [A] (x, y, r_K, 0) of each agent's last road selection, or nullptr
  const float4* lsegs;   // road-edge segments by road-grid cell of the first point (LiDAR)
  const int* lcell;      // their cell starts
  // scratch of the per-stage form
  uint32_t* agrid_key;   // [A] per world: sorted agent-grid keys of the active agents
  int* agrid_n;          // [W] number of active agents in the agent grid
  uint8_t* coll;         // [A] collision found this step
  uint8_t* off;          // [A] road edge crossed this step
  unsigned* err;         // sticky error word
};

__device__ __forceinline__ float clampf(float a, float lo, float hi) { return fminf(fmaxf(a, lo), hi); }

// Kinematic bicycle model of App. B with l_r = L/2: mid-step clipped speed,
// slip angle beta = atan(tan(delta)/2), explicit Euler with the old heading.
// Every rounding step is spelled out (fmaf / __fmul_rn), so all kernels that
// inline this produce bit-identical states.
__device__ __forceinline__ void bicycle_step(float4& s, float accel, float steer, float L, float dt, float vmax) {
  const float vbar = clampf(fmaf(__fmul_rn(0.5f, accel), dt, s.w), -vmax, vmax);
  const float tn = tanf(steer);
  const float beta = atanf(__fmul_rn(0.5f, tn));
  float sn, cs;
  sincosf(__fadd_rn(s.z, beta), &sn, &cs);
  const float xdot = __fmul_rn(vbar, cs);
  const float ydot = __fmul_rn(vbar, sn);
  const float thdot = __fdiv_rn(__fmul_rn(__fmul_rn(vbar, cosf(beta)), tn), L);
  s.x = fmaf(xdot, dt, s.x);
  s.y = fmaf(ydot, dt, s.y);
  s.z = fmaf(thdot, dt, s.z);
  s.w = clampf(fmaf(accel, dt, s.w), -vmax, vmax);
}

// Simplified invertible model (Sec. 3.2 "Agent dynamics"): the position is a
// double integrator along the heading of the start of the step, the yaw
// turns by the steering curvature `curv` (1/m) times the distance covered,
// ds = v dt + a dt^2 / 2, and the speed is v + a dt (no clip, so the model
// stays invertible).  Independent of the vehicle length.  Rounding spelled
// out as in bicycle_step.
__device__ __forceinline__ void invertible_step(float4& s, float accel, float curv, float dt) {
  const float ds = fmaf(__fmul_rn(0.5f, accel), __fmul_rn(dt, dt), __fmul_rn(s.w, dt));
  float sn, cs;
  sincosf(s.z, &sn, &cs);
  s.x = fmaf(cs, ds, s.x);
  s.y = fmaf(sn, ds, s.y);
  s.z = fmaf(curv, ds, s.z);
  s.w = fmaf(accel, dt, s.w);
}

// One dynamics step of an agent; false when the action is not valid for the
// model (non-finite, or |steer| >= pi/2 for the kinematic bicycle), in
// which case the state is left unchanged.
__device__ __forceinline__ bool dynamics_step(int dyn, float4& s, float accel, float steer, float L, float dt,
                                              float vmax) {
  if (!isfinite(accel) || !isfinite(steer)) return false;
  if (dyn == 1) {
    invertible_step(s, accel, steer, dt);
    return true;
  }
  if (fabsf(steer) >= 1.5707963f) return false;
  bicycle_step(s, accel, steer, L, dt, vmax);
  return true;
}

// Ego-frame rotation by -theta of the offset (dx, dy), given c = cos theta,
// s = sin theta, with a fixed rounding sequence.
__device__ __forceinline__ float rot_x(float c, float s, float dx, float dy) { return fmaf(c, dx, __fmul_rn(s, dy)); }
__device__ __forceinline__ float rot_y(float c, float s, float dx, float dy) { return fmaf(c, dy, -__fmul_rn(s, dx)); }

// Separating-axis depth of two oriented boxes: the minimum over the four box
// axes of (sum of projected half extents - |projected centre offset|).
// > 0 iff the boxes share interior points.  (dx, dy) = centre_b - centre_a;
// (ca, sa), (cb, sb) = heading cos/sin; (la, wa), (lb, wb) = half extents.
__device__ __forceinline__ float box_box_depth(float dx, float dy, float ca, float sa, float la, float wa, float cb,
                                               float sb, float lb, float wb) {
  const float C = fabsf(fmaf(ca, cb, __fmul_rn(sa, sb)));   // |cos(theta_b - theta_a)|
  const float S = fabsf(fmaf(ca, sb, -__fmul_rn(sa, cb)));  // |sin(theta_b - theta_a)|
  const float pa1 = __fadd_rn(la, fmaf(lb, C, __fmul_rn(wb, S))) - fabsf(rot_x(ca, sa, dx, dy));
  const float pa2 = __fadd_rn(wa, fmaf(lb, S, __fmul_rn(wb, C))) - fabsf(rot_y(ca, sa, dx, dy));
  const float pb1 = __fadd_rn(lb, fmaf(la, C, __fmul_rn(wa, S))) - fabsf(rot_x(cb, sb, dx, dy));
  const float pb2 = __fadd_rn(wb, fmaf(la, S, __fmul_rn(wa, C))) - fabsf(rot_y(cb, sb, dx, dy));
  return fminf(fminf(pa1, pa2), fminf(pb1, pb2));
}

// Separating-axis depth of an oriented box (centre c, axes (ca, sa) and
// (-sa, ca), half extents l, w) and a segment: box axes plus the segment
// normal.  > 0 iff the segment passes through the box interior.
__device__ __forceinline__ float box_seg_depth(float cx, float cy, float ca, float sa, float l, float w, float4 seg) {
  const float qx0 = seg.x - cx, qy0 = seg.y - cy, qx1 = seg.z - cx, qy1 = seg.w - cy;
  // box axis 1
  float u0 = rot_x(ca, sa, qx0, qy0), u1 = rot_x(ca, sa, qx1, qy1);
  float d = fminf(fmaxf(u0, u1) + l, l - fminf(u0, u1));
  // box axis 2
  u0 = rot_y(ca, sa, qx0, qy0);
  u1 = rot_y(ca, sa, qx1, qy1);
  d = fminf(d, fminf(fmaxf(u0, u1) + w, w - fminf(u0, u1)));
  // segment normal
  const float ex = seg.z - seg.x, ey = seg.w - seg.y;
  const float el = sqrtf(fmaf(ex, ex, __fmul_rn(ey, ey)));
  if (el > 0.f) {
    const float nx = -ey / el, ny = ex / el;
    const float s = fmaf(qx0, nx, __fmul_rn(qy0, ny));
    const float r = fmaf(l, fabsf(fmaf(nx, ca, __fmul_rn(ny, sa))), __fmul_rn(w, fabsf(fmaf(ny, ca, -__fmul_rn(nx, sa)))));
    d = fminf(d, r - fabsf(s));
  }
  return d;
}

// Agent-grid key: 12-bit column, 12-bit row (clamped, monotone) and the
// 8-bit local agent index, so one column of three cells is one key range.
__device__ __forceinline__ uint32_t agent_cell_key(int cx, int cy, int local) {
  cx = min(max(cx, 0), 4095);
  cy = min(max(cy, 0), 4095);
  return ((uint32_t)cx << 20) | ((uint32_t)cy << 8) | (uint32_t)local;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
  for (int o = 1; o < WARP; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

}  // namespace gd
