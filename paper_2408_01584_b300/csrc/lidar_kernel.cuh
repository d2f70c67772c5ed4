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
// Obstacle-major, one warp per agent in the fused kernel and a pair of
// warps per agent in the stand-alone scan.  Seen from the ray origin, an obstacle
// that keeps at least LIDAR_NEAR_FULL away subtends an arc shorter than pi:
// the arc between the extreme corner (box) or end point (segment)
// directions.  It maps to one contiguous range of ray indices (two when it
// wraps past the end of a full circle), widened by LIDAR_PAD at each end to
// absorb the error of the arc angles (arc_atan2), of the rotations and of the index
// arithmetic (together below 1e-6 rad), and only those rays are tested
// exactly.  A
// closer obstacle is tested on every ray.  Each (obstacle, ray range) is an
// item of a per-warp queue in shared memory; the warp drains the queue one
// (item, ray) pair per lane, balanced by a prefix sum over the range
// lengths, so a near box (hundreds of rays) and a far segment (a few) cost
// the same per ray.
//
// Every agent being scanned has one 32-bit key per ray in shared memory: the depth's
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
constexpr float LIDAR_PAD = 1e-5f;           // rad added at both ends of an arc (arc_atan2 and rotation rounding)
constexpr unsigned LIDAR_EMPTY = 0xffffffffu;
constexpr float LIDAR_PI = 3.14159265358979f;
constexpr unsigned LIDAR_STRIPES = 16;       // claim counters of the stand-alone scan

struct LidarWarpHead {
  float4 ga[LIDAR_ITEMS];        // segment: (w', d') in the sensor frame; box: (o, cos psi, sin psi)
  float2 gb[LIDAR_ITEMS];        // segment: (cross(w', d'), 0); box: half extents
  unsigned range[LIDAR_ITEMS];   // first ray | ray count << 16
  int kofs[LIDAR_ITEMS];         // first pair index of the item (during a drain)
  unsigned row_start[MAX_ROWS];
  unsigned row_excl[MAX_ROWS];
};
static_assert(sizeof(LidarWarpHead) % 16 == 0, "per-warp key array must stay 16-byte aligned");

// Shared memory of one warp: the head and one key per ray (rounded up to 4).
__host__ __device__ __forceinline__ size_t lidar_warp_bytes(int n) {
  return sizeof(LidarWarpHead) + 16 * (size_t)((n + 3) / 4);
}
// Shared memory of the CTA's copy of the ray directions (float2 per ray).
__host__ __device__ __forceinline__ size_t lidar_dirs_bytes(int n) { return 16 * (size_t)((n + 1) / 2); }

// Copy the ray directions into shared memory (whole CTA; caller syncs).
__device__ __forceinline__ void lidar_stage_dirs(float2* dst, const float2* __restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
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
  const float4* lsegs;     // road-edge segments by road-grid cell of the first point
  const int* lcell;        // their cell starts (world w: from rgrid[w].cell_base)
  LidarFan fan;
  int warp_bytes;          // lidar_warp_bytes(n)
};

// Angle of (x, y) for the arc bounds, within 5e-7 rad of atan2 (far below
// LIDAR_PAD): the octant's ratio a = min / max in [0, 1], atan(a) =
// a P(a^2) with P of degree 6 fitted here to atan(a) / a on [0, 1] by
// weighted least squares (Lawson's iteration toward the minimax fit; the
// float32 evaluation's error, checked on 2e6 points, is 3.5e-7 rad), then
// reflected into the octant.
__device__ __forceinline__ float arc_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
  const float t = a * a;
  float p = 0.006811703089624643f;
  p = fmaf(p, t, -0.033603958785533905f);
  p = fmaf(p, t, 0.07962337881326675f);
  p = fmaf(p, t, -0.13233326375484467f);
  p = fmaf(p, t, 0.19807811081409454f);
  p = fmaf(p, t, -0.3331736624240875f);
  p = fmaf(p, t, 0.9999961256980896f);
  float r = p * a;
  if (ay > ax) r = 1.57079632679489662f - r;
  if (x < 0.f) r = LIDAR_PI - r;
  return copysignf(r, y);
}

// Ray ranges of the arc [lo, hi] (sensor-frame angles, hi - lo < pi): the
// copies of the arc shifted by -2pi, 0, +2pi that meet the fan, each range
// the rays whose angle lies within LIDAR_PAD of the arc.
__device__ __forceinline__ int arc_ranges(const LidarFan& f, float lo, float hi, bool full, unsigned& r0,
                                          unsigned& r1) {
  if (full) {
    r0 = (unsigned)f.n << 16;
    return 1;
  }
  int m = 0;
  const float a0 = (lo - LIDAR_PAD - f.b0) * f.inv_step, b0 = (hi + LIDAR_PAD - f.b0) * f.inv_step;
  if (a0 > 0.f && b0 < (float)(f.n - 1)) {
    // inside the fan: the copies one turn away cannot reach it
    const int k0 = (int)ceilf(a0), k1 = (int)floorf(b0);
    if (k0 > k1) return 0;
    r0 = (unsigned)k0 | ((unsigned)(k1 - k0 + 1) << 16);
    return 1;
  }
#pragma unroll
  for (int sft = -1; sft <= 1; ++sft) {
    const float a = fmaf((float)sft, f.wrap_steps, a0), b = fmaf((float)sft, f.wrap_steps, b0);
    const int k0 = max((int)ceilf(a), 0), k1 = min((int)floorf(b), f.n - 1);
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
// With den = cross(u, d'), s = cross(w', u) / den and t = C / den: both
// conditions are tested on the numerators after flipping their signs by
// den's, and the one division happens for the depth.
__device__ __forceinline__ bool ray_seg_item(float4 g, float C, float cb, float sb, float R, float& t) {
  const float den = fmaf(cb, g.w, -__fmul_rn(sb, g.z));     // cross(u, d')
  const float sn = fmaf(g.x, sb, -__fmul_rn(g.y, cb));      // cross(w', u)
  const unsigned sgn = __float_as_uint(den) & 0x80000000u;
  const float ad = fabsf(den);
  const float sp = __uint_as_float(__float_as_uint(sn) ^ sgn);
  const float cp = __uint_as_float(__float_as_uint(C) ^ sgn);
  t = fminf(fabsf(__fdividef(cp, ad)), R);                   // about 2 ulp; |den| <= segment length
  return ad > 0.f && sp >= 0.f && sp <= ad && cp >= 0.f && cp <= __fmul_rn(R, ad);
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
      const float t1 = __fdividef(-hh[a] - o[a], v[a]), t2 = __fdividef(hh[a] - o[a], v[a]);
      lo = fmaxf(lo, fminf(t1, t2));
      hi = fminf(hi, fmaxf(t1, t2));
    } else {
      ok = ok && fabsf(o[a]) <= hh[a];
    }
  }
  t = lo > 0.f ? lo : 0.f;
  return ok && lo <= hi && hi >= 0.f && t <= R;
}

// Position of a lane in the pair sequence of a drain: the item `it` of pair
// q, the first pair of the next item, the ray index of pair q and the
// item's geometry.
struct LidarCursor {
  unsigned q, end, next;
  int it, k;
  float4 g;
  float2 gb;
};

__device__ __forceinline__ void cursor_load(LidarCursor& c, const LidarWarpHead& h, int n_items, unsigned total) {
  c.next = c.it + 1 < n_items ? (unsigned)h.kofs[c.it + 1] : total;
  c.g = h.ga[c.it];
  c.gb = h.gb[c.it];
}

__device__ __forceinline__ void cursor_start(LidarCursor& c, const LidarWarpHead& h, int n_items, unsigned total,
                                             unsigned q, unsigned end) {
  c.q = q;
  c.end = end;
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)h.kofs[mid] <= q) lo = mid; else hi = mid - 1;
  }
  c.it = lo;
  c.k = (int)(h.range[lo] & 0xffffu) + (int)(q - (unsigned)h.kofs[lo]);
  cursor_load(c, h, n_items, total);
}

template <bool SEG>
__device__ __forceinline__ void cursor_test(LidarCursor& c, const LidarWarpHead& h, unsigned* keys, int n_items,
                                            unsigned total, const float2* __restrict__ dirs, float R) {
  if (c.q < c.end) {
    if (c.q == c.next) {
      ++c.it;
      c.k = (int)(h.range[c.it] & 0xffffu);
      cursor_load(c, h, n_items, total);
    }
    const float2 u = dirs[c.k];
    float t;
    const bool hit = SEG ? ray_seg_item(c.g, c.gb.x, u.x, u.y, R, t) : ray_box_item(c.g, c.gb, u.x, u.y, R, t);
    if (hit) atomicMin(&keys[c.k], (__float_as_uint(t) & ~1u) | (SEG ? 1u : 0u));
    ++c.q;
    ++c.k;
  }
}

// Drain the item queue: every (item, ray) pair is tested once and the hits
// are folded into the per-ray keys.  The pairs, numbered by a prefix sum of
// the range lengths, are cut into 64 contiguous blocks, two per lane: a lane
// finds the item of each block's first pair by bisection and then walks both
// blocks forward side by side (two independent dependency chains), so an
// item's geometry stays in registers while its rays are tested.
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
    if (it < n_items) h.kofs[it] = (int)ex;     // first pair index of the item
    ex += c[r];
  }
  const unsigned total = (unsigned)__shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  const unsigned per = (total + 2 * WARP - 1) / (2 * WARP);
  const unsigned q0 = min(2u * lane * per, total), q1 = min(q0 + per, total), q2 = min(q1 + per, total);
  if (q0 < q2) {
    LidarCursor a, b;
    cursor_start(a, h, n_items, total, q0, q1);
    if (q1 < q2) cursor_start(b, h, n_items, total, q1, q2);
    else b = a, b.q = b.end = q2;
    for (unsigned j = 0; j < per; ++j) {
      cursor_test<SEG>(a, h, keys, n_items, total, dirs, R);
      cursor_test<SEG>(b, h, keys, n_items, total, dirs, R);
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
// about (ex, ey), each clipped to the disk's chord, as ranges of the world's
// road-edge segment list (cell starts `lcell` of the world): published in
// h.row_start / h.row_excl like road_rows.  Returns the candidate count of
// the chunk; nrows = rows in it; rows_total = rows of the whole disk.
__device__ __forceinline__ int lidar_rows(const WorldView& v, const int* __restrict__ lcell, float Rr, float ex,
                                          float ey, int row0, LidarWarpHead& h, int lane, int& nrows,
                                          int& rows_total) {
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
        const int* cst = lcell + g.cell_base + row * g.nx;
        start = (unsigned)cst[cx0];
        len = cst[cx1 + 1] - cst[cx0];
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

// Write one agent's row from the keys (zeros if `done`): thread `lane` of
// the `nt` that share the row (a warp, or a warp pair).
__device__ __forceinline__ void lidar_write(const unsigned* keys, int n, float R, bool done, float* __restrict__ drow,
                                            uint8_t* __restrict__ crow, int lane, int nt = WARP) {
  const bool vec = (n & 3) == 0 && ((uintptr_t)drow & 15u) == 0 && (!crow || ((uintptr_t)crow & 3u) == 0);
  if (vec) {
    const uint4* k4 = reinterpret_cast<const uint4*>(keys);
    for (int q = lane; q < (n >> 2); q += nt) {
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
    for (int k = lane; k < n; k += nt) {
      float d = 0.f;
      uint8_t c = 0;
      if (!done) lidar_decode(keys[k], R, d, c);
      drow[k] = d;
      if (crow) crow[k] = c;
    }
  }
}

// Queue item(s) of the box of agent j (in the scene, not the observer) seen
// from (ex, ey) with sensor axis (cs, ss): returns the number of ray ranges
// (0..2, in r0 / r1) and sets the item geometry ga, gb.
__device__ __forceinline__ int lidar_box_item(const WorldView& v, int j, float ex, float ey, float cs, float ss,
                                              float R, const LidarFan& fan, unsigned& r0, unsigned& r1, float4& ga,
                                              float2& gb) {
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
  if (!(dc <= R + sqrtf(dist2(hl, hw)) + 1e-3f)) return 0;
  const float ox = rot_x(cj, sjn, qx, qy), oy = rot_y(cj, sjn, qx, qy);
  const float cp = fmaf(cs, cj, __fmul_rn(ss, sjn)), sp = fmaf(ss, cj, -__fmul_rn(cs, sjn));
  ga = make_float4(ox, oy, cp, sp);
  gb = make_float2(hl, hw);
  bool full = fabsf(ox) <= hl + LIDAR_NEAR_FULL && fabsf(oy) <= hw + LIDAR_NEAR_FULL;
  float lo = 0.f, hi = 0.f;
  if (!full) {
    // corner directions in the sensor frame; the box subtends less than pi,
    // so offsets from corner 0 need no wrap beyond one turn
    const float c1 = rot_x(cs, ss, -qx, -qy), c2 = rot_y(cs, ss, -qx, -qy);
    float g0 = 0.f, dmin = 0.f, dmax = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float u = (k & 1) ? hl : -hl, w = (k & 2) ? hw : -hw;
      const float p1 = c1 + fmaf(u, cp, __fmul_rn(w, sp)), p2 = c2 + fmaf(w, cp, -__fmul_rn(u, sp));
      const float gk = arc_atan2(p2, p1);
      if (k == 0) {
        g0 = gk;
      } else {
        float dl = gk - g0;
        dl = dl > LIDAR_PI ? dl - 2.f * LIDAR_PI : (dl < -LIDAR_PI ? dl + 2.f * LIDAR_PI : dl);
        dmin = fminf(dmin, dl);
        dmax = fmaxf(dmax, dl);
      }
    }
    lo = g0 + dmin;
    hi = g0 + dmax;
    full = hi - lo >= LIDAR_PI - 0.01f;
  }
  return arc_ranges(fan, lo, hi, full, r0, r1);
}

// Queue item(s) of the road-edge segment sg = (a, b) seen from (ex, ey)
// with sensor axis (cs, ss); as lidar_box_item.
__device__ __forceinline__ int lidar_seg_item(float4 sg, float ex, float ey, float cs, float ss, float R,
                                              const LidarFan& fan, unsigned& r0, unsigned& r1, float4& ga,
                                              float2& gb) {
  const float wx = sg.x - ex, wy = sg.y - ey, dx = sg.z - sg.x, dy = sg.w - sg.y;
  const float dd = dist2(dx, dy);
  const float tp = dd > 0.f ? clampf(__fdividef(-fmaf(wx, dx, __fmul_rn(wy, dy)), dd), 0.f, 1.f) : 0.f;
  const float dist = sqrtf(dist2(fmaf(tp, dx, wx), fmaf(tp, dy, wy)));
  if (!(dist <= R + 1e-3f)) return 0;
  const float w1 = rot_x(cs, ss, wx, wy), w2 = rot_y(cs, ss, wx, wy);
  const float d1 = rot_x(cs, ss, dx, dy), d2 = rot_y(cs, ss, dx, dy);
  ga = make_float4(w1, w2, d1, d2);
  gb = make_float2(fmaf(w1, d2, -__fmul_rn(w2, d1)), 0.f);
  bool full = dist < LIDAR_NEAR_FULL;
  float lo = 0.f, hi = 0.f;
  if (!full) {
    // end point directions; the short way between them is the arc
    const float ga0 = arc_atan2(w2, w1), gb0 = arc_atan2(w2 + d2, w1 + d1);
    float dl = gb0 - ga0;
    dl = dl > LIDAR_PI ? dl - 2.f * LIDAR_PI : (dl < -LIDAR_PI ? dl + 2.f * LIDAR_PI : dl);
    lo = dl >= 0.f ? ga0 : gb0;
    hi = lo + fabsf(dl);
    full = hi - lo >= LIDAR_PI - 0.01f;
  }
  return arc_ranges(fan, lo, hi, full, r0, r1);
}

// Sensor axis of an agent with heading state z (or (cos, sin) from cs) and
// head rotation `head`: the heading turned by the head angle.
__device__ __forceinline__ void lidar_axis(const WorldView& v, int li, float z, float head, float& cs, float& ss) {
  float ct, st;
  if (v.cs) {
    ct = v.cs[li].x;
    st = v.cs[li].y;
  } else {
    sincosf(z, &st, &ct);
  }
  float sh, ch;
  sincosf(head, &sh, &ch);
  cs = fmaf(ct, ch, -__fmul_rn(st, sh));
  ss = fmaf(st, ch, __fmul_rn(ct, sh));
}

// Fold one warp's share of agent li's obstacles into the keys: of the
// rounds of 32 boxes, then of 32 road-edge candidates, those with index
// part, part + parts, ... (all of them when parts = 1).  The warp's queue is
// empty at entry and at exit.
__device__ __forceinline__ void lidar_fold(const WorldView& v, int li, float R, float ex, float ey, float cs, float ss,
                                           const LidarArgs& la, LidarWarpHead& h, unsigned* keys, int lane, int part,
                                           int parts) {
  // ---- other agents' boxes ------------------------------------------------
  int nq = 0;
  for (int j0 = part * WARP; j0 < v.n; j0 += parts * WARP) {
    const int j = j0 + lane;
    int m = 0;
    unsigned r0 = 0, r1 = 0;
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 gb = make_float2(0.f, 0.f);
    if (j < v.n && j != li && !(v.flags[j] & GD_FLAG_DONE))
      m = lidar_box_item(v, j, ex, ey, cs, ss, R, la.fan, r0, r1, ga, gb);
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
    const int total = lidar_rows(v, la.lcell, Rr, ex, ey, row0, h, lane, nrows, rows_total);
    walk_rows(
        h, nrows, total, lane,
        [&](unsigned p, bool valid) {
          int m = 0;
          unsigned r0 = 0, r1 = 0;
          float4 ga = make_float4(0.f, 0.f, 0.f, 0.f);
          float2 gb = make_float2(0.f, 0.f);
          if (valid) m = lidar_seg_item(la.lsegs[p], ex, ey, cs, ss, R, la.fan, r0, r1, ga, gb);
          nq = lidar_push(h, nq, m, r0, r1, ga, gb, lane);
          if (nq >= WARP) {
            lidar_drain<true>(h, keys, nq, la.dirs, R, lane);
            nq = 0;
          }
        },
        part * WARP, parts * WARP);
  }
  if (nq) lidar_drain<true>(h, keys, nq, la.dirs, R, lane);
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
  float cs, ss;
  lidar_axis(v, li, s.z, head, cs, ss);
  lidar_fold(v, li, R, s.x, s.y, cs, ss, la, h, keys, lane, 0, 1);
  lidar_write(keys, n, R, false, drow, crow, lane);
}

// ---- a group of warps per agent ---------------------------------------------
// The stand-alone scan with G warps on each agent: one key array per group
// (the warps fold into it with atomicMin), one item queue per warp.  The
// warps take rounds of 32 boxes and of 32 road-edge candidates in turn, so
// each has its own queue and drains as in the one-warp form; a named
// barrier of the group's 32 G threads (id 1 + group) orders the keys'
// initialisation before the folds and the folds before the row is written.
// A 3000-ray scan's keys then hold more warps per SM than the 12 of one
// warp per agent.  The keys are the same folds of the same tests: the scan
// is bit-identical to the one-warp form.
__device__ __forceinline__ void group_sync(unsigned id, unsigned threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Shared memory of one group: G warp heads, then the keys.
__host__ __device__ __forceinline__ size_t lidar_group_bytes(int G, int n) {
  return (size_t)G * sizeof(LidarWarpHead) + 16 * (size_t)((n + 3) / 4);
}
constexpr int LIDAR_MAX_GROUPS = 15;   // named barriers 1..15
// Shared memory of a CTA of `groups` groups: the groups, the claim slots
// (two per group), the ray directions.
__host__ __device__ __forceinline__ size_t lidar_groups_smem(int G, int groups, int n) {
  return (size_t)groups * lidar_group_bytes(G, n) + 16 * (size_t)((2 * LIDAR_MAX_GROUPS + 3) / 4) +
         lidar_dirs_bytes(n);
}
// CTA size of the group form: at most this many warps.  Measured on the
// 1,024 x 64 workload (3000 rays, 360 degrees, ms per episode): pairs
// with 18, 20 and 22 warps per SM 49.2, 47.0 and 45.7; groups of three
// (24 warps) 48.6 and of four (32 warps, 64 registers) 49.9; one warp per
// agent (12 warps) 59.0.  22 warps of pairs is what shared memory holds
// (11 x 18.2 KB + 23.4 KB of ray directions).
template <int G>
struct LidarGroupShape {
  static constexpr int max_warps = G == 2 ? 22 : (G == 3 ? 24 : 32);
};

// Persistent CTAs of blockDim.x / (32 G) groups; group g of the grid draws
// agents c, c + LIDAR_STRIPES, ... from counter c = g mod LIDAR_STRIPES.  The
// group's first warp claims and publishes the claim in one of two slots,
// alternating, so that a slot is rewritten only after the other warps have
// passed the next barrier (and so read the slot).
template <int G>
__global__ void __launch_bounds__(LidarGroupShape<G>::max_warps * 32, 1)
    k_lidar_group(DevEnv e, LidarArgs la, unsigned* counter) {
  extern __shared__ __align__(16) unsigned char lidar_smem_raw[];
  const int n = la.fan.n;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, grp = wib / G, part = wib - grp * G;
  const int groups = (int)(blockDim.x / (32 * G));
  unsigned char* gbase = lidar_smem_raw + (size_t)grp * lidar_group_bytes(G, n);
  LidarWarpHead& h = *reinterpret_cast<LidarWarpHead*>(gbase + part * sizeof(LidarWarpHead));
  unsigned* keys = reinterpret_cast<unsigned*>(gbase + G * sizeof(LidarWarpHead));
  unsigned* claim = reinterpret_cast<unsigned*>(lidar_smem_raw + (size_t)groups * lidar_group_bytes(G, n));
  float2* sdirs = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(claim) +
                                            16 * (size_t)((2 * LIDAR_MAX_GROUPS + 3) / 4));
  // a step launch queued behind this one as a programmatic dependent (the
  // overlapped rollout) may start as SMs free up at this launch's tail
  asm volatile("griddepcontrol.launch_dependents;");
  lidar_stage_dirs(sdirs, la.dirs, n);
  __syncthreads();
  la.dirs = sdirs;
  const unsigned id = 1u + (unsigned)grp, nthr = 32u * G;
  const int t = part * WARP + lane;     // thread of the group
  const unsigned c = (unsigned)(blockIdx.x * groups + grp) % LIDAR_STRIPES;
  for (int it = 0;; ++it) {
    unsigned* slot = claim + 2 * grp + (it & 1);
    if (t == 0) *slot = atomicAdd(counter + c, 1u);
    group_sync(id, nthr);   // the claim published; the previous agent's row written by every warp
    const unsigned iu = c + LIDAR_STRIPES * *slot;
    if (iu >= (unsigned)e.A) break;
    const int i = (int)iu;
    float* drow = la.depth + (size_t)i * n;
    uint8_t* crow = la.cls ? la.cls + (size_t)i * n : nullptr;
    if (e.flags[i] & GD_FLAG_DONE) {
      // removed from the scene: an all-zero row, no world loads
      lidar_write(keys, n, e.R, true, drow, crow, t, 32 * G);
      continue;
    }
    {
      uint4* k4 = reinterpret_cast<uint4*>(keys);
      const uint4 e4 = make_uint4(LIDAR_EMPTY, LIDAR_EMPTY, LIDAR_EMPTY, LIDAR_EMPTY);
      for (int q = t; q < (n + 3) >> 2; q += 32 * G) k4[q] = e4;
    }
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
    const float4 s = v.state[i - a0];
    float cs, ss;
    lidar_axis(v, i - a0, s.z, la.head ? la.head[i] : 0.f, cs, ss);
    group_sync(id, nthr);   // keys initialised
    lidar_fold(v, i - a0, e.R, s.x, s.y, cs, ss, la, h, keys, lane, part, G);
    group_sync(id, nthr);   // every hit folded
    lidar_write(keys, n, e.R, false, drow, crow, t, 32 * G);
  }
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
