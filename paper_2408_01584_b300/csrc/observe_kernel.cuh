// Ego-frame observation (Sec. 3.2 "Sensor modalities": all road points and
// agents within a fixed radius, in the agent's relative frame; 50 m in
// Fig. 1), truncated to the K nearest road points and P nearest partners,
// sorted by (squared distance, local index).
//
// One warp per agent.  Road candidates come from the rows of the world's
// road grid that meet the observation disk; each row is clipped to the
// disk's chord, so one row is one contiguous range of cell-sorted points and
// the warp walks all rows as one flat list.  A world's road is one block of
// the road arena: x, y as float2 for every point, then one 16-bit word per
// point (local index | type << 15), both in cell order.  The block is read
// from the world's shared-memory tile (fused kernel) or from global memory.
//
// Top-K selection ("bucket rank"): d^2 in [0, R^2] is split into NB equal
// buckets (equal-area annuli).  Pass 1 walks the rows, counts in-radius
// points per bucket and keeps their keys' low words (and the first 256 d^2)
// in a compact list.  An exclusive scan gives each bucket's first rank and
// the bucket b* holding rank K.  Pass 2 walks the compact list in shared
// memory and scatters the keys of buckets
// <= b* into their bucket's slice of shared memory; the rank of a key is its
// bucket's first rank plus the number of smaller keys in its bucket.  If
// buckets <= b* do not fit, the exact K-th key is found by bisection over
// the key space and only keys up to it are kept; if the compact list
// overflows, pass 2 walks the rows again.  Every rank is exact: the output
// equals a full sort.
//
// Key = (d^2 bits << 32) | (local index << 17) | (type << 16) | (position in
// the world's cell-sorted points): d^2 >= 0 so its bits order like the
// value, the local index breaks ties (the type bit below it never decides),
// and the low 32 bits carry everything the row writer needs besides the
// point's coordinates: index, type and the position that locates the point.
#pragma once
#include "gd_device.cuh"

namespace gd {

constexpr int OBS_NB = 256;        // d^2 buckets
constexpr int OBS_CAP = 288;       // keys kept per warp (>= GD_MAX_K_ROAD)
constexpr int OBS_CAND = 448;      // compact list of in-radius points (more: pass 2 walks the rows again);
                                   // its size keeps 3 adjoint CTAs per SM
constexpr int BITONIC_MAX = 256;   // strategy 2 sorts at most this many keys
static_assert(OBS_CAP >= GD_MAX_K_ROAD, "selection capacity must hold K keys");
static_assert(OBS_CAP >= BITONIC_MAX && OBS_CAND >= BITONIC_MAX, "bitonic keys must fit");
static_assert((OBS_NB / WARP) % 2 == 0, "a lane's buckets must fill whole histogram words");
static_assert(GD_MAX_ROAD_PER_WORLD < 65536, "bucket counts and cursors must fit 16 bits");

struct ObsWarpSmem {
  unsigned cur[OBS_NB / 2];        // histogram, then scatter cursor: bucket b in the 16-bit half b & 1 of
                                   // word b / 2 (counts and cursors stay <= GD_MAX_ROAD_PER_WORLD < 2^16)
  unsigned short off[OBS_NB + 2];  // first rank of each bucket
  union {
    unsigned long long keys[OBS_CAP];                     // road keys, bucket order
    unsigned long long pkeys[GD_MAX_AGENTS_PER_WORLD];    // partner keys
  } u;
  unsigned cand[OBS_CAND];         // low key words (index, type, position) of the in-radius points (pass 1)
  unsigned sel[GD_MAX_K_ROAD];     // road: low 32 bits of the key of rank r; during the selection, the d^2
                                   // bits of in-radius point k < GD_MAX_K_ROAD of the compact list
  unsigned char psel[GD_MAX_PARTNERS + 1];                // partner: local index of rank r
  unsigned row_start[MAX_ROWS];
  unsigned row_excl[MAX_ROWS];
};

// View of one world's agents and road for the observation: pointers may be
// shared or global memory.
struct WorldView {
  const float4* state;     // [n] agents of the world
  const float4* stat;      // [n]
  const float2* cs;        // [n] (cos theta, sin theta) of the agents, or nullptr: computed here
  const uint8_t* flags;    // [n]
  int n;                   // agents in the world
  const float2* xy;        // [nr] cell-sorted road points
  const uint16_t* meta;    // [nr] local index | type << 15
  const uint16_t* next;    // [nr] position of the edge segment's second point, or NO_SEGMENT
  const uint16_t* cell_start;  // ny*nx + 1 cell starts (block positions)
  GridDesc g;
};

// Low 32 bits of a road key from meta = local index | type << 15 (the road
// block's 16-bit word) and the block position; the key puts d^2 above them.
__device__ __forceinline__ unsigned road_lo(unsigned meta, unsigned pos) {
  return ((meta & 0x7fffu) << 17) | ((meta >> 15) << 16) | pos;
}
__device__ __forceinline__ unsigned long long road_key(float d2, unsigned lo) {
  return ((unsigned long long)__float_as_uint(d2) << 32) | lo;
}
__device__ __forceinline__ unsigned sel_pos(unsigned k) { return k & 0xffffu; }
__device__ __forceinline__ unsigned sel_type(unsigned k) { return (k >> 16) & 1u; }
__device__ __forceinline__ unsigned sel_index(unsigned k) { return k >> 17; }
// 16-bit bucket counter b of the packed histogram
__device__ __forceinline__ unsigned bucket_shift(int b) { return (unsigned)(b & 1) << 4; }
__device__ __forceinline__ unsigned long long partner_key(float d2, unsigned j) {
  return ((unsigned long long)__float_as_uint(d2) << 32) | j;
}

// Squared distance with a fixed rounding sequence (no contraction choices
// left to the compiler), so every pass computes bit-identical keys.
__device__ __forceinline__ float dist2(float dx, float dy) { return fmaf(dx, dx, __fmul_rn(dy, dy)); }

__device__ __forceinline__ int bucket_of(float d2, float binv) { return min((int)(d2 * binv), OBS_NB - 1); }

// Rows of the observation disk centred at (ex, ey): lane r < nrows
// publishes the point range of row cy0 + r clipped to the chord.  Returns
// the total candidate count; row data lands in sm.row_start / row_excl.
__device__ __forceinline__ int road_rows(const WorldView& v, float R, float R2, float ex, float ey, ObsWarpSmem& sm,
                                         int lane, int& nrows) {
  const GridDesc& g = v.g;
  const float margin = 1e-3f;
  const int cy0 = (int)clampf(floorf((ey - R - margin - g.oy) * g.inv_cs), 0.f, (float)g.ny);
  const int cy1 = (int)clampf(floorf((ey + R + margin - g.oy) * g.inv_cs), -1.f, (float)(g.ny - 1));
  nrows = min(cy1 - cy0 + 1, MAX_ROWS);
  int len = 0;
  unsigned start = 0;
  if (lane < nrows) {
    const int row = cy0 + lane;
    const float ylo = g.oy + row * g.cs, yhi = ylo + g.cs;
    const float dy = fmaxf(0.f, fmaxf(ylo - ey, ey - yhi));
    if (dy <= R + margin) {
      const float hw = sqrtf(fmaxf(R2 - dy * dy, 0.f)) + margin;
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
  sm.row_start[lane] = start;
  sm.row_excl[lane] = (unsigned)(incl - len);
  __syncwarp();
  return __shfl_sync(0xffffffffu, incl, 31);
}

// Warp-uniform walk of the flat candidate list of the rows published in
// sm.row_start / sm.row_excl: fn(pos, valid) is called by every lane in
// every round (valid = this lane has a candidate), so fn may use warp
// collectives.
// Rounds start at entry `first` and step by `stride` (a multiple of 32):
// two warps sharing a list walk alternate rounds.
template <typename SM, typename Fn>
__device__ __forceinline__ void walk_rows(const SM& sm, int nrows, int total, int lane, Fn&& fn, int first = 0,
                                          int stride = WARP) {
  int r = 0;
  unsigned rs = sm.row_start[0], re = nrows > 1 ? sm.row_excl[1] : 0xffffffffu, rx = 0;
  for (int f0 = first; f0 < total; f0 += stride) {
    const int f = f0 + lane;
    const bool valid = f < total;
    if (valid) {
      while ((unsigned)f >= re) {
        ++r;
        rs = sm.row_start[r];
        rx = sm.row_excl[r];
        re = (r + 1 < nrows) ? sm.row_excl[r + 1] : 0xffffffffu;
      }
    }
    fn(valid ? rs + ((unsigned)f - rx) : 0u, valid);
  }
}

// Road selection of one agent at (ex, ey): the low 32 bits of the keys
// (index, type, position) of the n_sel <= K nearest in-radius points, in
// rank order, land in sm.sel; returns n_sel.
__device__ __forceinline__ int select_road(const WorldView& v, int K, float R, float R2, float ex, float ey,
                                           ObsWarpSmem& sm, int lane, int strategy = 1) {
  if (K == 0) return 0;
  const float binv = (float)OBS_NB / R2;
  const float2* __restrict__ xy = v.xy;
  const uint16_t* __restrict__ meta = v.meta;
  int nrows;
  const int total = road_rows(v, R, R2, ex, ey, sm, lane, nrows);

  // pass 1: histogram of d^2 buckets + compact list of the in-radius
  // points' low key words (index, type, position; their d^2 go to the sel
  // array, free until the ranking, for the first GD_MAX_K_ROAD), so that
  // pass 2 reads shared memory only: its reloads of the points missed L1
  // and took 44% of the selection.  The warp walks the flat candidate list
  // U x 32 entries per round, lane l taking entries l, l + 32, ...: each
  // load instruction reads 32 consecutive points (two 128-byte lines when
  // the road is read through L1/L2, no bank conflict in the tile) and their
  // meta words, and the loads are independent.
  // Neighbouring points along a road differ in distance by far more than a
  // bucket's width, so the histogram atomics rarely collide.
  for (int b = lane; b < OBS_NB / 2; b += WARP) sm.cur[b] = 0;
  __syncwarp();
  int n_in = 0;
  const unsigned lt = (1u << lane) - 1u;
  {
    int r = 0;
    unsigned rs = sm.row_start[0], rx = 0;
    unsigned re = (nrows > 1) ? sm.row_excl[1] : 0xffffffffu;
    // U = 3 measured fastest on the 1,024 x 64 workload (2: -2%, 4: -4%,
    // 6 and 8 spill under the 64-register cap)
    constexpr int U = 3;
    for (int f0 = 0; f0 < total; f0 += U * WARP) {
      unsigned pu[U];
      bool vu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int f = f0 + u * WARP + lane;
        vu[u] = f < total;
        if (vu[u]) {
          while ((unsigned)f >= re) {
            ++r;
            rs = sm.row_start[r];
            rx = sm.row_excl[r];
            re = (r + 1 < nrows) ? sm.row_excl[r + 1] : 0xffffffffu;
          }
        }
        pu[u] = vu[u] ? rs + ((unsigned)f - rx) : 0u;
      }
      float2 qu[U];
      unsigned mu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) qu[u] = xy[pu[u]];
#pragma unroll
      for (int u = 0; u < U; ++u) mu[u] = meta[pu[u]];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float d2 = dist2(qu[u].x - ex, qu[u].y - ey);
        const bool in = vu[u] && d2 <= R2;
        if (in) {
          const int bk = bucket_of(d2, binv);
          atomicAdd(&sm.cur[bk >> 1], 1u << bucket_shift(bk));
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        const int slot = n_in + __popc(m & lt);
        if (in && slot < OBS_CAND) {
          sm.cand[slot] = road_lo(mu[u], pu[u]);
          if (slot < GD_MAX_K_ROAD) sm.sel[slot] = __float_as_uint(d2);
        }
        n_in += __popc(m);
      }
    }
  }
  __syncwarp();
  // exclusive scan: lane owns OBS_NB/32 consecutive buckets
  constexpr int PER = OBS_NB / WARP;
  unsigned cnt[PER];
  int mine = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    cnt[k] = (sm.cur[(lane * PER + k) >> 1] >> bucket_shift(k)) & 0xffffu;
    mine += (int)cnt[k];
  }
  const int incl = warp_incl_scan(mine, lane);
  const int n_sel = min(K, n_in);
  int bstar = OBS_NB - 1;    // bucket holding rank n_sel - 1
  {
    unsigned run = (unsigned)(incl - mine);
    int cand = OBS_NB;
    unsigned lo_half = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      sm.off[lane * PER + k] = (unsigned short)run;
      // scatter cursors, two per word
      if (k & 1) sm.cur[(lane * PER + k) >> 1] = lo_half | (run << 16); else lo_half = run;
      if ((int)run < K && (int)(run + cnt[k]) >= K) cand = min(cand, lane * PER + k);
      run += cnt[k];
    }
    if (lane == WARP - 1) sm.off[OBS_NB] = (unsigned short)run;
    if (n_in > K) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
      bstar = cand;
    }
  }
  __syncwarp();
  const bool compact = n_in <= OBS_CAND;
  if (strategy == 2 && n_in <= BITONIC_MAX) {
    // strategy 2: bitonic sort of all in-radius keys (padded to a power of
    // two with ~0), ascending; the first n_sel are the selection
    int m = 1;
    while (m < n_in) m <<= 1;
    for (int k = lane; k < m; k += WARP) {
      unsigned long long key = ~0ull;
      if (k < n_in) key = road_key(__uint_as_float(sm.sel[k]), sm.cand[k]);   // k < BITONIC_MAX <= GD_MAX_K_ROAD
      sm.u.keys[k] = key;
    }
    __syncwarp();
    for (int size = 2; size <= m; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = lane; t < (m >> 1); t += WARP) {
          const int i = (t / stride) * (2 * stride) + (t % stride), j = i + stride;
          const unsigned long long x = sm.u.keys[i], y = sm.u.keys[j];
          if ((x > y) == ((i & size) == 0)) {
            sm.u.keys[i] = y;
            sm.u.keys[j] = x;
          }
        }
        __syncwarp();
      }
    }
    for (int r = lane; r < n_sel; r += WARP) sm.sel[r] = (unsigned)sm.u.keys[r];
    __syncwarp();
    return n_sel;
  }
  // Calls fn(lo, d2) for every in-radius point (lo: the low key word), from
  // the compact list when it holds them all (d^2 from the cache for the
  // first GD_MAX_K_ROAD, else from the point again), else by walking the
  // rows again.
  auto for_each_in_radius = [&](auto&& fn) {
    if (compact) {
      for (int k = lane; k < min(n_in, GD_MAX_K_ROAD); k += WARP) fn(sm.cand[k], __uint_as_float(sm.sel[k]));
      for (int k = GD_MAX_K_ROAD + lane; k < n_in; k += WARP) {
        const unsigned lo = sm.cand[k];
        const float2 q = xy[sel_pos(lo)];
        fn(lo, dist2(q.x - ex, q.y - ey));
      }
    } else {
      walk_rows(sm, nrows, total, lane, [&](unsigned p, bool valid) {
        if (valid) {
          const float2 q = xy[p];
          const float d2 = dist2(q.x - ex, q.y - ey);
          if (d2 <= R2) fn(road_lo(meta[p], p), d2);
        }
      });
    }
  };
  const int keep = (int)sm.off[bstar + 1];   // keys in buckets <= b*
  unsigned long long tau = ~0ull;             // keep keys <= tau in bucket b*
  if (keep > OBS_CAP) {
    // rare overflow: bisect the key space for the n_sel-th smallest key
    const unsigned need = (unsigned)(n_sel - (int)sm.off[bstar]);
    unsigned long long lo = 0, hi = ~0ull;
    while (lo < hi) {
      const unsigned long long mid = lo + ((hi - lo) >> 1);
      unsigned cntle = 0;
      for_each_in_radius([&](unsigned lo, float d2) {
        if (bucket_of(d2, binv) == bstar && road_key(d2, lo) <= mid) ++cntle;
      });
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cntle += __shfl_xor_sync(0xffffffffu, cntle, o);
      if (cntle >= need) hi = mid; else lo = mid + 1;
    }
    tau = lo;
    if (lane == 0) sm.off[bstar + 1] = (unsigned short)n_sel;
    __syncwarp();
  }
  // pass 2: scatter keys of buckets <= b* into their bucket slices
  for_each_in_radius([&](unsigned lo, float d2) {
    const int b = bucket_of(d2, binv);
    if (b <= bstar) {
      const unsigned long long key = road_key(d2, lo);
      if (b < bstar || key <= tau) {
        const unsigned sh = bucket_shift(b);
        const unsigned slot = (atomicAdd(&sm.cur[b >> 1], 1u << sh) >> sh) & 0xffffu;
        if (slot < (unsigned)OBS_CAP) sm.u.keys[slot] = key;
      }
    }
  });
  __syncwarp();
  const int stored = min((int)sm.off[bstar + 1], OBS_CAP);
  // rank inside the bucket
  for (int k = lane; k < stored; k += WARP) {
    const unsigned long long key = sm.u.keys[k];
    const int b = bucket_of(__uint_as_float((unsigned)(key >> 32)), binv);
    const int lo = (int)sm.off[b], hi = min((int)sm.off[b + 1], OBS_CAP);
    int r = lo, q = lo;
    for (; q + 1 < hi; q += 2) r += (int)(sm.u.keys[q] < key) + (int)(sm.u.keys[q + 1] < key);
    if (q < hi) r += sm.u.keys[q] < key;
    if (r < n_sel) sm.sel[r] = (unsigned)key;
  }
  __syncwarp();
  return n_sel;
}

// Road part of one observation row: K float4 slots at out4 (local indices
// to ridx if given).  With LOSS, each lane also adds w . features of its
// slots to acc (w = the row's weights for these slots, 4 per slot).
template <bool LOSS>
__device__ __forceinline__ void write_road(const WorldView& v, int K, int n_sel, float ex, float ey, float c, float s,
                                           const ObsWarpSmem& sm, int lane, float4* __restrict__ out4,
                                           int32_t* __restrict__ ridx, const float* __restrict__ w, float& acc) {
  const float2* __restrict__ xy = v.xy;
  // write K slots, coalesced, streaming (evict-first) stores; index and type
  // come with the selection, so only the coordinates are read, U slots per
  // lane per round with their loads in flight together
  constexpr int U = 4;
  for (int r0 = 0; r0 < K; r0 += U * WARP) {
    unsigned sk[U];
    float2 q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u * WARP + lane;
      sk[u] = r < n_sel ? sm.sel[r] : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      q[u] = (r0 + u * WARP + lane < n_sel) ? xy[sel_pos(sk[u])] : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int r = r0 + u * WARP + lane;
      if (r < K) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        int idx = -1;
        if (r < n_sel) {
          const float dx = q[u].x - ex, dy = q[u].y - ey;
          o = make_float4(rot_x(c, s, dx, dy), rot_y(c, s, dx, dy), (float)sel_type(sk[u]), 1.f);
          idx = (int)sel_index(sk[u]);
        }
        __stcs(out4 + r, o);
        if (ridx) ridx[r] = idx;
        if (LOSS) {
          const float4 wr = __ldg(reinterpret_cast<const float4*>(w) + r);
          acc = fmaf(wr.x, o.x, fmaf(wr.y, o.y, fmaf(wr.z, o.z, fmaf(wr.w, o.w, acc))));
        }
      }
    }
  }
}

// Partner part: other agents of the world still in the scene within R.
// The relative heading uses cos/sin of the difference from the two agents'
// own cos/sin: cos(tj - ti) = cj ci + sj si, sin(tj - ti) = sj ci - cj si.
// Selection: local indices of the n_sel <= P nearest land in sm.psel.
__device__ __forceinline__ int select_partners(const WorldView& v, int li, int P, float R2, float ex, float ey,
                                               ObsWarpSmem& sm, int lane) {
  if (P == 0) return 0;
  int n = 0;
  const unsigned lt = (1u << lane) - 1u;
  // two candidates per lane per round: the flags and states of both go out
  // together, before any test (a done candidate's state is read for
  // nothing, but no load waits for another)
  for (int j0 = 0; j0 < v.n; j0 += 2 * WARP) {
    bool live[2];
    float4 q[2];
    uint8_t fj[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = j0 + u * WARP + lane;
      fj[u] = j < v.n ? v.flags[j] : (uint8_t)GD_FLAG_DONE;
      q[u] = j < v.n ? v.state[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) live[u] = j0 + u * WARP + lane != li && !(fj[u] & GD_FLAG_DONE);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float d2 = dist2(q[u].x - ex, q[u].y - ey);
      const bool ok = live[u] && d2 <= R2;
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) sm.u.pkeys[n + __popc(m & lt)] = partner_key(d2, (unsigned)(j0 + u * WARP + lane));
      n += __popc(m);
    }
  }
  __syncwarp();
  const int n_sel = min(P, n);
  for (int k = lane; k < n; k += WARP) {
    const unsigned long long key = sm.u.pkeys[k];
    int r = 0;
    for (int q = 0; q < n; ++q) r += sm.u.pkeys[q] < key;
    if (r < n_sel) sm.psel[r] = (unsigned char)(key & 0xffu);
  }
  __syncwarp();
  return n_sel;
}

template <bool LOSS>
__device__ __forceinline__ void write_partners(const WorldView& v, int P, int n_sel, float ex, float ey, float c,
                                               float s, const ObsWarpSmem& sm, int lane, float4* __restrict__ out4,
                                               int32_t* __restrict__ pidx, const float* __restrict__ w, float& acc) {
  for (int r = lane; r < P; r += WARP) {
    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
    int idx = -1;
    if (r < n_sel) {
      idx = (int)sm.psel[r];
      const float4 q = v.state[idx];
      const float4 st = v.stat[idx];
      float2 cj;
      if (v.cs) cj = v.cs[idx]; else sincosf(q.z, &cj.y, &cj.x);
      const float dx = q.x - ex, dy = q.y - ey;
      o0 = make_float4(rot_x(c, s, dx, dy), rot_y(c, s, dx, dy), rot_x(c, s, cj.x, cj.y), rot_y(c, s, cj.x, cj.y));
      o1 = make_float4(q.w, st.x, st.y, 1.f);
    }
    __stcs(out4 + 2 * r, o0);
    __stcs(out4 + 2 * r + 1, o1);
    if (pidx) pidx[r] = idx;
    if (LOSS) {
      const float4 w0 = __ldg(reinterpret_cast<const float4*>(w) + 2 * r);
      const float4 w1 = __ldg(reinterpret_cast<const float4*>(w) + 2 * r + 1);
      acc = fmaf(w0.x, o0.x, fmaf(w0.y, o0.y, fmaf(w0.z, o0.z, fmaf(w0.w, o0.w, acc))));
      acc = fmaf(w1.x, o1.x, fmaf(w1.y, o1.y, fmaf(w1.z, o1.z, fmaf(w1.w, o1.w, acc))));
    }
  }
}

// Row of an agent removed from the scene (flags f has GD_FLAG_DONE): all
// zero except the three flags; index lists all -1.  With LOSS, lane 0
// returns w . row (the other lanes 0).
template <bool LOSS>
__device__ __forceinline__ float write_done_row(const DevEnv& e, uint8_t f, float* __restrict__ obs_row,
                                                int32_t* __restrict__ ridx, int32_t* __restrict__ pidx,
                                                const float* __restrict__ w, int lane) {
  float4* row = reinterpret_cast<float4*>(obs_row);
  const float fc = (f & GD_FLAG_COLLIDED) ? 1.f : 0.f, fo = (f & GD_FLAG_OFFROAD) ? 1.f : 0.f,
              fg = (f & GD_FLAG_GOAL) ? 1.f : 0.f;
  const int n4 = e.F >> 2;
  for (int k = lane; k < n4; k += WARP) {
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k == 1) o = make_float4(0.f, fc, fo, fg);
    __stcs(row + k, o);
  }
  if (ridx) for (int k = lane; k < e.K; k += WARP) ridx[k] = -1;
  if (pidx) for (int k = lane; k < e.P; k += WARP) pidx[k] = -1;
  float acc = 0.f;
  if (LOSS && lane == 0) acc = fmaf(__ldg(w + 5), fc, fmaf(__ldg(w + 6), fo, __fmul_rn(__ldg(w + 7), fg)));
  return acc;
}

// Recorded selection (objective rollouts): a slot past the points in range.
constexpr uint16_t OBS_SEL_NONE = 0xffff;
// A parked agent's kept selection: a slot past the points in range (no key
// low word is all ones: a block position is below GD_MAX_ROAD_PER_WORLD).
constexpr unsigned OBS_MEMO_NONE = 0xffffffffu;
static_assert(GD_MAX_ROAD_PER_WORLD <= 0xffff, "block positions must fit a recorded slot below OBS_SEL_NONE");

// One full observation row of local agent li of the world in view v.
// With LOSS, returns (to every lane) w . row for the weight row w (F
// floats); otherwise returns 0.
// MEMO: the form for envs with parked agents, which keeps their road
// selections (memo_row) between steps.
template <bool LOSS, bool MEMO = false>
__device__ __forceinline__ float observe_agent(const DevEnv& e, const WorldView& v, int li, float* __restrict__ obs_row,
                                               int32_t* __restrict__ ridx, int32_t* __restrict__ pidx,
                                               ObsWarpSmem& sm, int lane, float4* anchor,
                                               const float* __restrict__ w = nullptr, float* rk_slot = nullptr,
                                               const float4* own = nullptr, uint16_t* sel_slot = nullptr,
                                               unsigned* memo_row = nullptr) {
  float4* row = reinterpret_cast<float4*>(obs_row);
  const uint8_t f = v.flags[li];
  const float fc = (f & GD_FLAG_COLLIDED) ? 1.f : 0.f, fo = (f & GD_FLAG_OFFROAD) ? 1.f : 0.f,
              fg = (f & GD_FLAG_GOAL) ? 1.f : 0.f;
  float acc = 0.f;
  if (f & GD_FLAG_DONE) {
    acc = write_done_row<LOSS>(e, f, obs_row, ridx, pidx, w, lane);
  } else {
    // the anchor is read here, ahead of the row's stores that it could alias
    const float4 an = anchor ? *anchor : make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
    // own: the agent's state and extents/goal, read by the caller already
    const float4 st = own ? own[0] : v.state[li];
    const float4 sc = own ? own[1] : v.stat[li];
    float c, s;
    if (v.cs) {
      c = v.cs[li].x;
      s = v.cs[li].y;
    } else {
      sincosf(st.z, &s, &c);
    }
    if (lane == 0) {
      const float gx = sc.z - st.x, gy = sc.w - st.y;
      const float4 o0 = make_float4(st.w, sc.x, sc.y, rot_x(c, s, gx, gy));
      const float4 o1 = make_float4(rot_y(c, s, gx, gy), fc, fo, fg);
      __stcs(row + 0, o0);
      __stcs(row + 1, o1);
      if (LOSS) {
        acc = fmaf(__ldg(w + 0), o0.x, fmaf(__ldg(w + 1), o0.y, fmaf(__ldg(w + 2), o0.z, __fmul_rn(__ldg(w + 3), o0.w))));
        acc = fmaf(__ldg(w + 4), o1.x, fmaf(__ldg(w + 5), o1.y, fmaf(__ldg(w + 6), o1.z, fmaf(__ldg(w + 7), o1.w, acc))));
      }
    }
    const int np = select_partners(v, li, e.P, e.R2, st.x, st.y, sm, lane);
    write_partners<LOSS>(v, e.P, np, st.x, st.y, c, s, sm, lane, row + 2, pidx, LOSS ? w + 8 : nullptr, acc);
    // The road does not move, so the disk that held the K nearest points at
    // the last selection, grown by the distance moved since, holds at least
    // K points: the selection over it equals the one over the whole radius.
    float Rs = e.R, Rs2 = e.R2;
    if (anchor) {
      const float r = an.z + sqrtf(dist2(st.x - an.x, st.y - an.y)) + 1e-3f;
      if (r < e.R) {
        Rs = r;
        Rs2 = r * r;
      }
    }
    // A parked agent (GD_FLAG_STATIC) keeps its last selection in memo_row,
    // tagged in its anchor by the road layout: while it is where the anchor
    // says (bit for bit) and the layout is the same, the road and the agent
    // have not moved, so the selection is the same and is read back.
    const bool memo = MEMO && memo_row && anchor && (f & GD_FLAG_STATIC);
    int nroad = 0;
    if (memo && __float_as_uint(an.w) == e.road_epoch && __float_as_uint(an.x) == __float_as_uint(st.x) &&
        __float_as_uint(an.y) == __float_as_uint(st.y)) {
      for (int r0 = 0; r0 < e.K; r0 += WARP) {
        const int r = r0 + lane;
        const unsigned wv = r < e.K ? memo_row[r] : OBS_MEMO_NONE;
        if (r < e.K) sm.sel[r] = wv;
        nroad += __popc(__ballot_sync(0xffffffffu, wv != OBS_MEMO_NONE));
      }
      __syncwarp();
    } else {
      nroad = select_road(v, e.K, Rs, Rs2, st.x, st.y, sm, lane, e.topk);
      if (nroad < e.K && Rs < e.R) nroad = select_road(v, e.K, e.R, e.R2, st.x, st.y, sm, lane, e.topk);
      if (memo)
        for (int r = lane; r < e.K; r += WARP) memo_row[r] = r < nroad ? sm.sel[r] : OBS_MEMO_NONE;
    }
    if ((anchor || rk_slot) && lane == 0) {
      float rk = __int_as_float(0x7f800000);     // +inf: fewer than K in range
      if (nroad == e.K && e.K > 0) {
        const float2 q = v.xy[sel_pos(sm.sel[e.K - 1])];
        rk = sqrtf(dist2(q.x - st.x, q.y - st.y));
      }
      if (anchor) *anchor = make_float4(st.x, st.y, rk, memo ? __uint_as_float(e.road_epoch) : 0.f);
      if (rk_slot) *rk_slot = rk;
    }
    // the selection itself, for the backward pass: block positions in rank
    // order, OBS_SEL_NONE past the points in range
    if (sel_slot)
      for (int r = lane; r < e.K; r += WARP) sel_slot[r] = r < nroad ? (uint16_t)sel_pos(sm.sel[r]) : OBS_SEL_NONE;
    write_road<LOSS>(v, e.K, nroad, st.x, st.y, c, s, sm, lane, row + 2 + 2 * e.P, ridx,
                     LOSS ? w + 8 + 8 * e.P : nullptr, acc);
  }
  if (LOSS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  }
  return acc;
}

// Road block of world w in the arena: (xy, meta, next, cell_start)
// pointers for `base` (global arena or a shared-memory copy of the block).
__device__ __forceinline__ void road_block(const unsigned char* base, int nr, WorldView& v) {
  v.xy = reinterpret_cast<const float2*>(base);
  v.meta = reinterpret_cast<const uint16_t*>(base + (size_t)road_pad(nr) * sizeof(float2));
  v.next = v.meta + road_pad(nr);
  v.cell_start = v.next + road_pad(nr);
}

// Road-edge crossing (Sec. 3.2 "Termination conditions") of a box, from the
// world's road block: a segment that meets the box has its first point
// within (box circumradius + longest segment) of the box centre, so the
// grid cells under that square hold every candidate.  Warp per agent, lanes
// over the candidate points, ballot-OR of the separating-axis tests.
__device__ __forceinline__ bool offroad_from_block(const WorldView& v, float cx, float cy, float ca, float sa, float hl,
                                                   float hw, int lane) {
  const GridDesc& g = v.g;
  const float rq = sqrtf(fmaf(hl, hl, hw * hw)) + g.seg_max + 1e-3f;
  const int cx0 = (int)clampf(floorf((cx - rq - g.ox) * g.inv_cs), 0.f, (float)g.nx);
  const int cx1 = (int)clampf(floorf((cx + rq - g.ox) * g.inv_cs), -1.f, (float)(g.nx - 1));
  const int cy0 = (int)clampf(floorf((cy - rq - g.oy) * g.inv_cs), 0.f, (float)g.ny);
  const int cy1 = (int)clampf(floorf((cy + rq - g.oy) * g.inv_cs), -1.f, (float)(g.ny - 1));
  bool hit = false;
  if (cx0 <= cx1) {
    for (int row = cy0; row <= cy1; ++row) {
      const uint16_t* cst = v.cell_start + row * g.nx;
      const int b = cst[cx0], en = cst[cx1 + 1];
      for (int q = b + lane; q < en; q += WARP) {
        const unsigned nx = v.next[q];
        if (nx != NO_SEGMENT) {
          const float2 p0 = v.xy[q], p1 = v.xy[nx];
          hit |= box_seg_depth(cx, cy, ca, sa, hl, hw, make_float4(p0.x, p0.y, p1.x, p1.y)) > 0.f;
        }
      }
    }
  }
  return __any_sync(0xffffffffu, hit);
}

// Observation row of agent i with everything read from global memory (the
// world's agents and road block through L1/L2).
// With LOSS, returns (to every lane) wrow . row for the weight row wrow,
// and writes the agent's K-th road distance to rk_slot and its road
// selection to sel_slot if given.  MEMO as in observe_agent.
template <bool LOSS = false, bool MEMO = false>
__device__ __forceinline__ float observe_global(const DevEnv& e, int i, float* __restrict__ obs,
                                                int32_t* __restrict__ road_idx, int32_t* __restrict__ partner_idx,
                                                ObsWarpSmem& sm, int lane, const float* __restrict__ wrow = nullptr,
                                                float* rk_slot = nullptr, uint16_t* sel_slot = nullptr) {
  // the agent's own state first: it does not wait for the world's loads
  const float4 own[2] = {e.state[i], e.stat[i]};
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
  return observe_agent<LOSS, MEMO>(e, v, i - a0, obs + (size_t)i * e.F,
                                   road_idx ? road_idx + (size_t)i * e.K : nullptr,
                                   partner_idx ? partner_idx + (size_t)i * e.P : nullptr, sm, lane,
                                   e.anchor ? e.anchor + i : nullptr, wrow, rk_slot, own, sel_slot,
                                   MEMO && e.smemo ? e.smemo + (size_t)i * e.K : nullptr);
}

// Per-stage form: one warp per agent over the whole batch.  Dynamic shared
// memory: WARPS * sizeof(ObsWarpSmem).
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_observe(DevEnv e, float* __restrict__ obs,
                                                       int32_t* __restrict__ road_idx,
                                                       int32_t* __restrict__ partner_idx) {
  extern __shared__ __align__(16) unsigned char obs_smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + wib;
  if (i >= e.A) return;
  observe_global(e, i, obs, road_idx, partner_idx, reinterpret_cast<ObsWarpSmem*>(obs_smem_raw)[wib], lane);
}

// Objective of the split form (LOSS): ell[i] holds the agent's smooth goal
// reward r_s from the step launch and becomes reward_w * r_s + w . row, with
// the same single rounding as the fused kernel; rk[i] gets the K-th road
// distance.
struct SplitLoss {
  const float* w;      // [F] weight row, 16-byte aligned
  float reward_w;
  float* ell;          // [A]
  float* rk;           // [A] or nullptr
  uint16_t* sel;       // [A][K] each observed agent's road selection (block positions), or nullptr
};

// Batched split form, after the step (k_world without observation):
// persistent warps claim agents one at a time until all A are observed.
// The claims are striped over OBS_STRIPES counters (cleared before the
// launch), so that they do not all queue on one address: warp g draws from
// counter c = g mod OBS_STRIPES the agents c, c + OBS_STRIPES, ...  No
// per-world barrier, so a warp that drew a done agent (an all-zero row)
// moves straight on; agents go out in index order, which keeps a world's
// agents, and its road block in L1/L2, together.  Registers are capped for
// 32 warps per SM (its shared memory allows them).
constexpr unsigned OBS_STRIPES = 128;
template <int WARPS, bool LOSS = false, bool MEMO = false>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS) k_observe_split(DevEnv e, float* __restrict__ obs,
                                                                           int32_t* __restrict__ road_idx,
                                                                           int32_t* __restrict__ partner_idx,
                                                                           unsigned* __restrict__ counters,
                                                                           SplitLoss loss) {
  extern __shared__ __align__(16) unsigned char obs_smem_raw[];
  const int lane = threadIdx.x & 31;
  ObsWarpSmem& sm = reinterpret_cast<ObsWarpSmem*>(obs_smem_raw)[threadIdx.x >> 5];
  const unsigned c = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) % OBS_STRIPES;
  // a step launch queued behind this one as a programmatic dependent (the
  // overlapped rollout) may start as SMs free up at this launch's tail
  asm volatile("griddepcontrol.launch_dependents;");
  for (;;) {
    unsigned k = 0;
    if (lane == 0) k = atomicAdd(counters + c, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    const unsigned i = c + OBS_STRIPES * k;
    if (i >= (unsigned)e.A) break;
    // an agent removed from the scene needs only its flags: no world loads
    const uint8_t f = e.flags[i];
    float* orow = obs + (size_t)i * e.F;
    int32_t* ridx = road_idx ? road_idx + (size_t)i * e.K : nullptr;
    int32_t* pidx = partner_idx ? partner_idx + (size_t)i * e.P : nullptr;
    float dot;
    if (f & GD_FLAG_DONE) {
      dot = write_done_row<LOSS>(e, f, orow, ridx, pidx, loss.w, lane);
    } else {
      dot = observe_global<LOSS, MEMO>(e, (int)i, obs, road_idx, partner_idx, sm, lane, loss.w,
                                       LOSS && loss.rk ? loss.rk + i : nullptr,
                                       LOSS && loss.sel ? loss.sel + (size_t)i * e.K : nullptr);
    }
    if (LOSS && lane == 0) loss.ell[i] = fmaf(loss.reward_w, loss.ell[i], dot);
  }
}

}  // namespace gd
