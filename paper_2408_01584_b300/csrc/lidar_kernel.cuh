// LiDAR / view-cone observation (Sec. 3.2 "Sensor modalities": rays cast
// from the agent against bounding boxes and road objects, either all around
// or in a narrower cone that a head-rotation action turns; Fig. 1 shows
// 3000 rays over 360 and over 120 degrees).
//
// Ray k of n leaves the agent's centre at angle
//   theta + head - fov/2 + (k + 1/2) fov / n
// and stops at the first point, 0 <= t <= R, in the closed box of another
// agent still in the scene or on a road-edge segment: depth t, class agent
// or road edge (agent first at equal t); depth R, class none when it meets
// nothing.  An agent that is done observes nothing (all zero).
//
// One warp per agent, obstacle-major.  Seen from the ray origin, an obstacle
// that keeps at least LIDAR_NEAR_FULL away subtends an arc shorter than pi:
// the arc between the extreme corner (box) or end point (segment)
// directions.  It maps to one contiguous range of ray indices (two when it
// wraps past the end of a full circle), widened by LIDAR_PAD and one more
// ray at each end to absorb the rounding of atan2f and of the rotations
// (below 1e-6 rad), and only those rays are tested exactly.  A
// closer obstacle is tested on every ray.  Each (obstacle, ray range) is an
// item of a per-warp queue in shared memory; the warp drains the queue one
// (item, ray) pair per lane, balanced by a prefix sum over the range
// lengths, so a near box (hundreds of rays) and a far segment (a few) cost
// the same per ray.
//
// Every warp keeps one 32-bit key per ray in shared memory: the depth's
// bits with the lowest bit replaced by the class (0 agent, 1 road edge),
// folded with atomicMin.  Depths are >= 0, so the bits order like the
// values; the replaced bit moves the depth by at most one unit in the last
// place, and an agent wins a tie.
#pragma once
#include "gd_device.cuh"
#include "observe_kernel.cuh"

namespace gd {

constexpr int LIDAR_ITEMS = 96;              // queue capacity per warp (>= 31 + 2 * 32)
constexpr float LIDAR_NEAR_FULL = 0.1f;      // m: obstacles this close are tested on every ray
constexpr float LIDAR_PAD = 1e-5f;           // rad added at both ends of an arc (atan2f and rotation rounding)
constexpr unsigned LIDAR_EMPTY = 0xffffffffu;
constexpr float LIDAR_PI = 3.14159265358979f;

struct LidarWarpHead {
  float4 ga[LIDAR_ITEMS];        // segment: (w', d') in the sensor frame; box: (o, cos psi, sin psi)
  float2 gb[LIDAR_ITEMS];        // segment: (cross(w', d'), 0); box: half extents
  unsigned range[LIDAR_ITEMS];   // first ray | ray count << 16
  unsigned pre[LIDAR_ITEMS];     // exclusive prefix of the ray counts
  unsigned row_start[MAX_ROWS];
  unsigned row_excl[MAX_ROWS];
};
static_assert(sizeof(LidarWarpHead) % 16 == 0, "per-warp key array must stay 16-byte aligned");

// Shared memory of one warp: the head and one key per ray (rounded up to 4).
__host__ __device__ __forceinline__ size_t lidar_warp_bytes(int n) {
  return sizeof(LidarWarpHead) + 16 * (size_t)((n + 3) / 4);
}

// The ray fan in the sensor frame (x axis = heading turned by the head angle).
struct LidarFan {
  int n;               // rays
  float b0;            // angle of ray 0: -fov/2 + fov/(2n)
  float inv_step;      // n / fov
  float wrap_steps;    // 2 pi n / fov: a full turn in ray units
};

struct LidarArgs {
  const float* head;       // [A] head rotation (rad) or nullptr
  float* depth;            // [A, n] or nullptr (no LiDAR output)
  uint8_t* cls;            // [A, n] or nullptr
  const float2* dirs;      // [n] (cos, sin) of each ray's angle in the sensor frame
  LidarFan fan;
  int warp_bytes;          // lidar_warp_bytes(n)
};

// Ray ranges of the arc [lo, hi] (sensor-frame angles, hi - lo < pi + 2
// rays): the copies of the arc shifted by -2pi, 0, +2pi that meet the fan.
__device__ __forceinline__ int arc_ranges(const LidarFan& f, float lo, float hi, bool full, unsigned& r0,
                                          unsigned& r1) {
  if (full) {
    r0 = (unsigned)f.n << 16;
    return 1;
  }
  int m = 0;
  const float a0 = (lo - LIDAR_PAD - f.b0) * f.inv_step, b0 = (hi + LIDAR_PAD - f.b0) * f.inv_step;
#pragma unroll
  for (int sft = -1; sft <= 1; ++sft) {
    const float a = fmaf((float)sft, f.wrap_steps, a0), b = fmaf((float)sft, f.wrap_steps, b0);
    const int k0 = max((int)ceilf(a) - 1, 0), k1 = min((int)floorf(b) + 1, f.n - 1);
    if (k0 <= k1) {
      const unsigned r = (unsigned)k0 | ((unsigned)(k1 - k0 + 1) << 16);
      if (m == 0) r0 = r; else r1 = r;
      m = min(m + 1, 2);
    }
  }
  return m;
}

// Ray test of a segment item: p + t u = a + s (b - a) in the sensor frame,
// w' = a - p, d' = b - a, C = cross(w', d'); hit iff 0 <= s <= 1, 0 <= t <= R.
__device__ __forceinline__ bool ray_seg_item(float4 g, float C, float cb, float sb, float R, float& t) {
  const float den = fmaf(cb, g.w, -__fmul_rn(sb, g.z));     // cross(u, d')
  const float sn = fmaf(g.x, sb, -__fmul_rn(g.y, cb));      // cross(w', u)
  bool hit = den > 0.f ? (sn >= 0.f && sn <= den) : (den < 0.f && sn <= 0.f && sn >= den);
  t = __fdiv_rn(C, den);
  hit = hit && t >= 0.f && t <= R;
  t = fabsf(t);
  return hit;
}

// Ray test of a box item (slab method in the box frame): o = ray origin in
// the box frame, (cos psi, sin psi) turns the sensor frame into the box
// frame, (hl, hw) = half extents.  t = 0 when the origin is inside.
__device__ __forceinline__ bool ray_box_item(float4 g, float2 h, float cb, float sb, float R, float& t) {
  const float v[2] = {fmaf(g.z, cb, -__fmul_rn(g.w, sb)), fmaf(g.w, cb, __fmul_rn(g.z, sb))};
  const float o[2] = {g.x, g.y};
  const float hh[2] = {h.x, h.y};
  float lo = -INFINITY, hi = INFINITY;
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (v[a] != 0.f) {
      const float inv = __frcp_rn(v[a]);
      const float t1 = __fmul_rn(-hh[a] - o[a], inv), t2 = __fmul_rn(hh[a] - o[a], inv);
      lo = fmaxf(lo, fminf(t1, t2));
      hi = fminf(hi, fmaxf(t1, t2));
    } else {
      ok = ok && fabsf(o[a]) <= hh[a];
    }
  }
  t = lo > 0.f ? lo : 0.f;
  return ok && lo <= hi && hi >= 0.f && t <= R;
}

// Drain the item queue: every (item, ray) pair is tested once, one pair
// per lane per round, and the hits are folded into the per-ray keys.
template <bool SEG>
__device__ __forceinline__ void lidar_drain(LidarWarpHead& h, unsigned* keys, int n_items,
                                            const float2* __restrict__ dirs, float R, int lane) {
  unsigned c[3], sum = 0;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int it = 3 * lane + r;
    c[r] = it < n_items ? (h.range[it] >> 16) : 0u;
    sum += c[r];
  }
  const int incl = warp_incl_scan((int)sum, lane);
  unsigned ex = (unsigned)incl - sum;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int it = 3 * lane + r;
    if (it < n_items) h.pre[it] = ex;
    ex += c[r];
  }
  const unsigned total = (unsigned)__shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  for (unsigned q0 = 0; q0 < total; q0 += WARP) {
    const unsigned q = q0 + lane;
    if (q < total) {
      int lo = 0, hi = n_items - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (h.pre[mid] <= q) lo = mid; else hi = mid - 1;
      }
      const int k = (int)(h.range[lo] & 0xffffu) + (int)(q - h.pre[lo]);
      const float2 u = dirs[k];
      float t;
      const bool hit = SEG ? ray_seg_item(h.ga[lo], h.gb[lo].x, u.x, u.y, R, t)
                           : ray_box_item(h.ga[lo], h.gb[lo], u.x, u.y, R, t);
      if (hit) atomicMin(&keys[k], (__float_as_uint(t) & ~1u) | (SEG ? 1u : 0u));
    }
  }
  __syncwarp();
}

// Append this lane's m (0..2) items to the queue; returns the new length.
__device__ __forceinline__ int lidar_push(LidarWarpHead& h, int nq, int m, unsigned r0, unsigned r1, float4 ga,
                                          float2 gb, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  const unsigned b1 = __ballot_sync(0xffffffffu, m >= 1), b2 = __ballot_sync(0xffffffffu, m >= 2);
  const int slot = nq + __popc(b1 & lt) + __popc(b2 & lt);
  if (m >= 1) {
    h.range[slot] = r0;
    h.ga[slot] = ga;
    h.gb[slot] = gb;
  }
  if (m >= 2) {
    h.range[slot + 1] = r1;
    h.ga[slot + 1] = ga;
    h.gb[slot + 1] = gb;
  }
  __syncwarp();
  return nq + __popc(b1) + __popc(b2);
}

// Rows [row0, row0 + 32) of the grid rows that meet the disk of radius Rr
// about (ex, ey), each clipped to the disk's chord: published in
// h.row_start / h.row_excl like road_rows.  Returns the candidate count of
// the chunk; nrows = rows in it; rows_total = rows of the whole disk.
__device__ __forceinline__ int lidar_rows(const WorldView& v, float Rr, float ex, float ey, int row0,
                                          LidarWarpHead& h, int lane, int& nrows, int& rows_total) {
  const GridDesc& g = v.g;
  const float margin = 1e-3f;
  const int cy0 = (int)clampf(floorf((ey - Rr - margin - g.oy) * g.inv_cs), 0.f, (float)g.ny);
  const int cy1 = (int)clampf(floorf((ey + Rr + margin - g.oy) * g.inv_cs), -1.f, (float)(g.ny - 1));
  rows_total = max(cy1 - cy0 + 1, 0);
  nrows = min(rows_total - row0, MAX_ROWS);
  int len = 0;
  unsigned start = 0;
  if (lane < nrows) {
    const int row = cy0 + row0 + lane;
    const float ylo = g.oy + row * g.cs, yhi = ylo + g.cs;
    const float dy = fmaxf(0.f, fmaxf(ylo - ey, ey - yhi));
    if (dy <= Rr + margin) {
      const float hw = sqrtf(fmaxf(Rr * Rr - dy * dy, 0.f)) + margin;
      const int cx0 = (int)clampf(floorf((ex - hw - g.ox) * g.inv_cs), 0.f, (float)g.nx);
      const int cx1 = (int)clampf(floorf((ex + hw - g.ox) * g.inv_cs), -1.f, (float)(g.nx - 1));
      if (cx0 <= cx1) {
        const uint16_t* cst = v.cell_start + row * g.nx;
        start = cst[cx0];
        len = (int)cst[cx1 + 1] - (int)start;
      }
    }
  }
  const int incl = warp_incl_scan(len, lane);
  h.row_start[lane] = start;
  h.row_excl[lane] = (unsigned)(incl - len);
  __syncwarp();
  return __shfl_sync(0xffffffffu, incl, 31);
}

__device__ __forceinline__ void lidar_decode(unsigned key, float R, float& d, uint8_t& c) {
  if (key == LIDAR_EMPTY) {
    d = R;
    c = 0;
  } else {
    d = __uint_as_float(key & ~1u);
    c = (uint8_t)(1u + (key & 1u));
  }
}

// Write one agent's row from the keys (zeros if `done`).
__device__ __forceinline__ void lidar_write(const unsigned* keys, int n, float R, bool done, float* __restrict__ drow,
                                            uint8_t* __restrict__ crow, int lane) {
  const bool vec = (n & 3) == 0 && ((uintptr_t)drow & 15u) == 0 && (!crow || ((uintptr_t)crow & 3u) == 0);
  if (vec) {
    const uint4* k4 = reinterpret_cast<const uint4*>(keys);
    for (int q = lane; q < (n >> 2); q += WARP) {
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
      uint8_t c[4] = {0, 0, 0, 0};
      if (!done) {
        const uint4 kk = k4[q];
        lidar_decode(kk.x, R, d.x, c[0]);
        lidar_decode(kk.y, R, d.y, c[1]);
        lidar_decode(kk.z, R, d.z, c[2]);
        lidar_decode(kk.w, R, d.w, c[3]);
      }
      reinterpret_cast<float4*>(drow)[q] = d;
      if (crow)
        reinterpret_cast<uint32_t*>(crow)[q] = (uint32_t)c[0] | ((uint32_t)c[1] << 8) | ((uint32_t)c[2] << 16) |
                                               ((uint32_t)c[3] << 24);
    }
  } else {
    for (int k = lane; k < n; k += WARP) {
      float d = 0.f;
      uint8_t c = 0;
      if (!done) lidar_decode(keys[k], R, d, c);
      drow[k] = d;
      if (crow) crow[k] = c;
    }
  }
}

// LiDAR scan of agent li of the world in view v by one warp.
__device__ __forceinline__ void lidar_agent(const WorldView& v, int li, float R, float head, const LidarArgs& la,
                                            float* __restrict__ drow, uint8_t* __restrict__ crow, LidarWarpHead& h,
                                            unsigned* keys, int lane) {
  const int n = la.fan.n;
  if (v.flags[li] & GD_FLAG_DONE) {
    lidar_write(keys, n, R, true, drow, crow, lane);
    return;
  }
  {
    uint4* k4 = reinterpret_cast<uint4*>(keys);
    const uint4 e4 = make_uint4(LIDAR_EMPTY, LIDAR_EMPTY, LIDAR_EMPTY, LIDAR_EMPTY);
    for (int q = lane; q < (n + 3) >> 2; q += WARP) k4[q] = e4;
  }
  __syncwarp();
  const float4 s = v.state[li];
  const float ex = s.x, ey = s.y;
  float ct, st;
  if (v.cs) {
    ct = v.cs[li].x;
    st = v.cs[li].y;
  } else {
    sincosf(s.z, &st, &ct);
  }
  float sh, ch;
  sincosf(head, &sh, &ch);
  // sensor axis: heading turned by the head angle
  const float cs = fmaf(ct, ch, -__fmul_rn(st, sh)), ss = fmaf(st, ch, __fmul_rn(ct, sh));

  // ---- other agents' boxes ------------------------------------------------
  int nq = 0;
  for (int j0 = 0; j0 < v.n; j0 += WARP) {
    const int j = j0 + lane;
    int m = 0;
    unsigned r0 = 0, r1 = 0;
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 gb = make_float2(0.f, 0.f);
    if (j < v.n && j != li && !(v.flags[j] & GD_FLAG_DONE)) {
      const float4 sj = v.state[j];
      const float4 tj = v.stat[j];
      float cj, sjn;
      if (v.cs) {
        cj = v.cs[j].x;
        sjn = v.cs[j].y;
      } else {
        sincosf(sj.z, &sjn, &cj);
      }
      const float hl = 0.5f * tj.x, hw = 0.5f * tj.y;
      const float qx = ex - sj.x, qy = ey - sj.y;               // ray origin relative to the box centre
      const float dc = sqrtf(dist2(qx, qy));
      if (dc <= R + sqrtf(dist2(hl, hw)) + 1e-3f) {
        const float ox = rot_x(cj, sjn, qx, qy), oy = rot_y(cj, sjn, qx, qy);
        const float cp = fmaf(cs, cj, __fmul_rn(ss, sjn)), sp = fmaf(ss, cj, -__fmul_rn(cs, sjn));
        ga = make_float4(ox, oy, cp, sp);
        gb = make_float2(hl, hw);
        bool full = fabsf(ox) <= hl + LIDAR_NEAR_FULL && fabsf(oy) <= hw + LIDAR_NEAR_FULL;
        float lo = 0.f, hi = 0.f;
        if (!full) {
          // box centre and axes in the sensor frame
          const float c1 = rot_x(cs, ss, -qx, -qy), c2 = rot_y(cs, ss, -qx, -qy);
          const float gc = atan2f(c2, c1);
          float dmin = 0.f, dmax = 0.f;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float u = (k & 1) ? hl : -hl, w = (k & 2) ? hw : -hw;
            const float p1 = c1 + fmaf(u, cp, __fmul_rn(w, sp)), p2 = c2 + fmaf(w, cp, -__fmul_rn(u, sp));
            const float dl = atan2f(fmaf(c1, p2, -__fmul_rn(c2, p1)), fmaf(c1, p1, __fmul_rn(c2, p2)));
            dmin = fminf(dmin, dl);
            dmax = fmaxf(dmax, dl);
          }
          lo = gc + dmin;
          hi = gc + dmax;
          full = hi - lo >= LIDAR_PI - 0.01f;
        }
        m = arc_ranges(la.fan, lo, hi, full, r0, r1);
      }
    }
    nq = lidar_push(h, nq, m, r0, r1, ga, gb, lane);
    if (nq >= WARP) {
      lidar_drain<false>(h, keys, nq, la.dirs, R, lane);
      nq = 0;
    }
  }
  if (nq) lidar_drain<false>(h, keys, nq, la.dirs, R, lane);
  nq = 0;

  // ---- road-edge segments: first points within R + longest segment -------
  const float Rr = R + v.g.seg_max + 1e-3f;
  int rows_total = 1;
  for (int row0 = 0; row0 < rows_total; row0 += MAX_ROWS) {
    int nrows = 0;
    const int total = lidar_rows(v, Rr, ex, ey, row0, h, lane, nrows, rows_total);
    walk_rows(h, nrows, total, lane, [&](unsigned p, bool valid) {
      int m = 0;
      unsigned r0 = 0, r1 = 0;
      float4 ga = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 gb = make_float2(0.f, 0.f);
      const unsigned nx = valid ? (unsigned)v.next[p] : (unsigned)NO_SEGMENT;
      if (nx != NO_SEGMENT) {
        const float2 a = v.xy[p], b = v.xy[nx];
        const float wx = a.x - ex, wy = a.y - ey, dx = b.x - a.x, dy = b.y - a.y;
        const float dd = dist2(dx, dy);
        const float tp = dd > 0.f ? clampf(-fmaf(wx, dx, __fmul_rn(wy, dy)) / dd, 0.f, 1.f) : 0.f;
        const float dist = sqrtf(dist2(fmaf(tp, dx, wx), fmaf(tp, dy, wy)));
        if (dist <= R + 1e-3f) {
          const float w1 = rot_x(cs, ss, wx, wy), w2 = rot_y(cs, ss, wx, wy);
          const float d1 = rot_x(cs, ss, dx, dy), d2 = rot_y(cs, ss, dx, dy);
          ga = make_float4(w1, w2, d1, d2);
          gb = make_float2(fmaf(w1, d2, -__fmul_rn(w2, d1)), 0.f);
          bool full = dist < LIDAR_NEAR_FULL;
          float lo = 0.f, hi = 0.f;
          if (!full) {
            const float m1 = fmaf(0.5f, d1, w1), m2 = fmaf(0.5f, d2, w2);   // midpoint
            const float gm = atan2f(m2, m1);
            const float b1 = w1 + d1, b2 = w2 + d2;
            const float da = atan2f(fmaf(m1, w2, -__fmul_rn(m2, w1)), fmaf(m1, w1, __fmul_rn(m2, w2)));
            const float db = atan2f(fmaf(m1, b2, -__fmul_rn(m2, b1)), fmaf(m1, b1, __fmul_rn(m2, b2)));
            lo = gm + fminf(da, db);
            hi = gm + fmaxf(da, db);
            full = hi - lo >= LIDAR_PI - 0.01f;
          }
          m = arc_ranges(la.fan, lo, hi, full, r0, r1);
        }
      }
      nq = lidar_push(h, nq, m, r0, r1, ga, gb, lane);
      if (nq >= WARP) {
        lidar_drain<true>(h, keys, nq, la.dirs, R, lane);
        nq = 0;
      }
    });
  }
  if (nq) lidar_drain<true>(h, keys, nq, la.dirs, R, lane);
  lidar_write(keys, n, R, false, drow, crow, lane);
}

// Per-stage form: one warp per agent over the whole batch, everything read
// from global memory.  Dynamic shared memory: WARPS * warp_bytes.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 1) k_lidar(DevEnv e, LidarArgs la) {
  extern __shared__ __align__(16) unsigned char lidar_smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + wib;
  if (i >= e.A) return;
  unsigned char* base = lidar_smem_raw + (size_t)wib * la.warp_bytes;
  LidarWarpHead& h = *reinterpret_cast<LidarWarpHead*>(base);
  unsigned* keys = reinterpret_cast<unsigned*>(base + sizeof(LidarWarpHead));
  const int w = e.agent_world[i];
  const int a0 = e.agent_off[w];
  WorldView v;
  v.state = e.state + a0;
  v.stat = e.stat + a0;
  v.cs = nullptr;
  v.flags = e.flags + a0;
  v.n = e.agent_off[w + 1] - a0;
  road_block(e.arena + (size_t)e.arena_off[w] * 16, e.road_off[w + 1] - e.road_off[w], v);
  v.g = e.rgrid[w];
  lidar_agent(v, i - a0, e.R, la.head ? la.head[i] : 0.f, la, la.depth + (size_t)i * la.fan.n,
              la.cls ? la.cls + (size_t)i * la.fan.n : nullptr, h, keys, lane);
}

// Ray directions of the fan in the sensor frame, (cos, sin) of
// -fov/2 + (k + 1/2) fov / n, evaluated in double and rounded once.
__global__ void k_lidar_dirs(float2* dirs, int n, double fov) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    double sn, cn;
    sincos(-0.5 * fov + (k + 0.5) * fov / n, &sn, &cn);
    dirs[k] = make_float2((float)cn, (float)sn);
  }
}

}  // namespace gd
