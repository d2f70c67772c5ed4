// Ego-frame observation (Sec. 3.2 "Sensor modalities": all road points and
// agents within a fixed radius, in the agent's relative frame; 50 m in
// Fig. 1), truncated to the K nearest road points and P nearest partners,
// sorted by (squared distance, local index).
//
// One warp per agent.  Road candidates come from the rows of the world's
// road grid that meet the observation disk; each row is clipped to the
// disk's chord, so one row is one contiguous range of cell-sorted points and
// the warp walks all rows as one flat list.
//
// Top-K selection ("bucket rank"): the squared distance d^2 in [0, R^2] is
// split into NB equal buckets (equal-area annuli, so roughly equal counts
// for a uniform point density).  Pass 1 counts candidates per bucket; an
// exclusive scan gives each bucket's first rank and the bucket b* holding
// rank K.  Pass 2 scatters the keys of buckets <= b* to their bucket's
// slice of shared memory; the final rank of a key is its bucket's first
// rank plus the number of smaller keys in its bucket.  If buckets <= b* do
// not fit, the exact K-th key is found by bisection over the key space and
// only keys up to it are kept.  Every rank is exact: the output is the same
// as a full sort.
#pragma once
#include "gd_device.cuh"

namespace gd {

constexpr int OBS_NB = 128;        // d^2 buckets
constexpr int OBS_CAP = 384;       // keys kept per warp (>= GD_MAX_K_ROAD)
static_assert(OBS_CAP >= GD_MAX_K_ROAD, "selection capacity must hold K keys");

struct ObsWarpSmem {
  unsigned off[OBS_NB + 1];        // first rank of each bucket
  unsigned cur[OBS_NB];            // histogram, then scatter cursor
  union {
    struct {
      unsigned long long keys[OBS_CAP];   // (d^2 bits << 32) | local index
      unsigned pos[OBS_CAP];              // position of the key's point in rpts
    } road;
    struct {
      unsigned long long keys[GD_MAX_AGENTS_PER_WORLD];
      unsigned sel[GD_MAX_PARTNERS + 1];
    } partner;
  } u;
  unsigned sel[GD_MAX_K_ROAD];     // rpts position of each selected rank
  unsigned row_start[MAX_ROWS];
  unsigned row_excl[MAX_ROWS];
};

__device__ __forceinline__ unsigned long long make_key(float d2, unsigned idx) {
  return ((unsigned long long)__float_as_uint(d2) << 32) | idx;
}

// Road rows of the observation disk centred at (ex, ey): lane r < nrows
// publishes the point range of row cy0 + r clipped to the chord.  Returns
// the total candidate count; row data lands in sm.row_start / row_excl.
__device__ __forceinline__ int road_rows(const DevEnv& e, const GridDesc& g, float ex, float ey, ObsWarpSmem& sm,
                                         int lane, int& nrows) {
  const float R = e.R;
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
      const float hw = sqrtf(fmaxf(e.R2 - dy * dy, 0.f)) + margin;
      const int cx0 = (int)clampf(floorf((ex - hw - g.ox) * g.inv_cs), 0.f, (float)g.nx);
      const int cx1 = (int)clampf(floorf((ex + hw - g.ox) * g.inv_cs), -1.f, (float)(g.nx - 1));
      if (cx0 <= cx1) {
        const int* cs = e.rcell_start + g.cell_base + row * g.nx;
        start = (unsigned)cs[cx0];
        len = cs[cx1 + 1] - cs[cx0];
      }
    }
  }
  const int incl = warp_incl_scan(len, lane);
  if (lane < MAX_ROWS) {
    sm.row_start[lane] = start;
    sm.row_excl[lane] = (unsigned)(incl - len);
  }
  __syncwarp();
  return __shfl_sync(0xffffffffu, incl, 31);
}

// Walk the flat candidate list; fn(pos) is called for each candidate point.
template <typename Fn>
__device__ __forceinline__ void for_each_candidate(const ObsWarpSmem& sm, int nrows, int total, int lane, Fn&& fn) {
  int r = 0;
  for (int f = lane; f < total; f += WARP) {
    while (r + 1 < nrows && (int)sm.row_excl[r + 1] <= f) ++r;
    fn(sm.row_start[r] + (unsigned)(f - (int)sm.row_excl[r]));
  }
}

__device__ __forceinline__ int bucket_of(float d2, float binv) { return min((int)(d2 * binv), OBS_NB - 1); }

// Squared distance with a fixed rounding sequence (no contraction choices
// left to the compiler), so every pass computes bit-identical keys.
__device__ __forceinline__ float dist2(float dx, float dy) { return fmaf(dx, dx, __fmul_rn(dy, dy)); }

// Road part of one observation row: writes K float4 slots at out4 and the
// optional local indices.
__device__ void observe_road(const DevEnv& e, int w, float ex, float ey, float c, float s, ObsWarpSmem& sm, int lane,
                             float4* __restrict__ out4, int32_t* __restrict__ ridx) {
  const int K = e.K;
  if (K == 0) return;
  const GridDesc g = e.rgrid[w];
  const float R2 = e.R2;
  const float binv = (float)OBS_NB / R2;
  int nrows;
  const int total = road_rows(e, g, ex, ey, sm, lane, nrows);

  // pass 1: histogram of d^2 buckets
  for (int b = lane; b < OBS_NB; b += WARP) sm.cur[b] = 0;
  __syncwarp();
  for_each_candidate(sm, nrows, total, lane, [&](unsigned p) {
    const float4 q = __ldg(e.rpts + p);
    const float dx = q.x - ex, dy = q.y - ey;
    const float d2 = dist2(dx, dy);
    if (d2 <= R2) atomicAdd(&sm.cur[bucket_of(d2, binv)], 1u);
  });
  __syncwarp();
  // exclusive scan: lane owns OBS_NB/32 consecutive buckets
  constexpr int PER = OBS_NB / WARP;
  unsigned cnt[PER];
  int mine = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    cnt[k] = sm.cur[lane * PER + k];
    mine += (int)cnt[k];
  }
  const int incl = warp_incl_scan(mine, lane);
  const int n_in = __shfl_sync(0xffffffffu, incl, 31);
  const int n_sel = min(K, n_in);
  {
    unsigned run = (unsigned)(incl - mine);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      sm.off[lane * PER + k] = run;
      run += cnt[k];
    }
    if (lane == WARP - 1) sm.off[OBS_NB] = run;
  }
  __syncwarp();
  // bucket holding rank n_sel - 1 (the last selected key)
  int bstar = OBS_NB - 1;
  if (n_in > K) {
    int cand = OBS_NB;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int b = lane * PER + k;
      if ((int)sm.off[b] < K && (int)(sm.off[b] + cnt[k]) >= K) cand = min(cand, b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
    bstar = cand;
  }
  const int keep = (int)sm.off[bstar + 1];   // keys in buckets <= b*
  unsigned long long tau = ~0ull;             // keep keys <= tau in bucket b*
  if (keep > OBS_CAP) {
    // rare overflow: bisect the key space for the n_sel-th smallest key of the disk
    const unsigned need = (unsigned)(n_sel - (int)sm.off[bstar]);
    unsigned long long lo = 0, hi = ~0ull;
    while (lo < hi) {
      const unsigned long long mid = lo + ((hi - lo) >> 1);
      unsigned cntle = 0;
      for_each_candidate(sm, nrows, total, lane, [&](unsigned p) {
        const float4 q = __ldg(e.rpts + p);
        const float dx = q.x - ex, dy = q.y - ey;
        const float d2 = dist2(dx, dy);
        if (d2 <= R2 && bucket_of(d2, binv) == bstar && make_key(d2, __float_as_uint(q.z)) <= mid) ++cntle;
      });
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cntle += __shfl_xor_sync(0xffffffffu, cntle, o);
      if (cntle >= need) hi = mid; else lo = mid + 1;
    }
    tau = lo;
    if (lane == 0) sm.off[bstar + 1] = (unsigned)n_sel;
    __syncwarp();
  }
  // pass 2: scatter keys of buckets <= b* into their bucket slices
  for (int b = lane; b <= bstar; b += WARP) sm.cur[b] = sm.off[b];
  __syncwarp();
  for_each_candidate(sm, nrows, total, lane, [&](unsigned p) {
    const float4 q = __ldg(e.rpts + p);
    const float dx = q.x - ex, dy = q.y - ey;
    const float d2 = dist2(dx, dy);
    if (d2 <= R2) {
      const int b = bucket_of(d2, binv);
      const unsigned long long key = make_key(d2, __float_as_uint(q.z));
      if (b < bstar || (b == bstar && key <= tau)) {
        const unsigned slot = atomicAdd(&sm.cur[b], 1u);
        if (slot < (unsigned)OBS_CAP) {
          sm.u.road.keys[slot] = key;
          sm.u.road.pos[slot] = p;
        }
      }
    }
  });
  __syncwarp();
  const int stored = (int)sm.off[bstar + 1];
  // rank inside the bucket
  for (int k = lane; k < stored; k += WARP) {
    const unsigned long long key = sm.u.road.keys[k];
    const int b = bucket_of(__uint_as_float((unsigned)(key >> 32)), binv);
    const int lo = (int)sm.off[b], hi = (int)sm.off[b + 1];
    int r = lo;
    for (int q = lo; q < hi; ++q) r += sm.u.road.keys[q] < key;
    if (r < n_sel) sm.sel[r] = sm.u.road.pos[k];
  }
  __syncwarp();
  // write K slots, coalesced, streaming (evict-first) stores
  for (int r = lane; r < K; r += WARP) {
    float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = -1;
    if (r < n_sel) {
      const float4 q = __ldg(e.rpts + sm.sel[r]);
      const float dx = q.x - ex, dy = q.y - ey;
      o = make_float4(c * dx + s * dy, -s * dx + c * dy, (float)__float_as_int(q.w), 1.f);
      idx = __float_as_int(q.z);
    }
    __stcs(out4 + r, o);
    if (ridx) ridx[r] = idx;
  }
}

// Partner part: other agents of the world still in the scene within R.
__device__ void observe_partners(const DevEnv& e, int i, int a0, int a1, float ex, float ey, float th, float c,
                                 float s, ObsWarpSmem& sm, int lane, float4* __restrict__ out4,
                                 int32_t* __restrict__ pidx) {
  const int P = e.P;
  if (P == 0) return;
  int n = 0;
  for (int j0 = a0; j0 < a1; j0 += WARP) {
    const int j = j0 + lane;
    bool ok = false;
    unsigned long long key = 0;
    if (j < a1 && j != i && !(e.flags[j] & GD_FLAG_DONE)) {
      const float4 q = e.state[j];
      const float dx = q.x - ex, dy = q.y - ey;
      const float d2 = dist2(dx, dy);
      ok = d2 <= e.R2;
      key = make_key(d2, (unsigned)(j - a0));
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (ok) sm.u.partner.keys[n + __popc(m & ((1u << lane) - 1u))] = key;
    n += __popc(m);
  }
  __syncwarp();
  const int n_sel = min(P, n);
  for (int k = lane; k < n; k += WARP) {
    const unsigned long long key = sm.u.partner.keys[k];
    int r = 0;
    for (int q = 0; q < n; ++q) r += sm.u.partner.keys[q] < key;
    if (r < n_sel) sm.u.partner.sel[r] = (unsigned)(key & 0xffffffffu);
  }
  __syncwarp();
  for (int r = lane; r < P; r += WARP) {
    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
    int idx = -1;
    if (r < n_sel) {
      idx = (int)sm.u.partner.sel[r];
      const float4 q = e.state[a0 + idx];
      const float4 st = e.stat[a0 + idx];
      const float dx = q.x - ex, dy = q.y - ey;
      float sd, cd;
      sincosf(q.z - th, &sd, &cd);
      o0 = make_float4(c * dx + s * dy, -s * dx + c * dy, cd, sd);
      o1 = make_float4(q.w, st.x, st.y, 1.f);
    }
    __stcs(out4 + 2 * r, o0);
    __stcs(out4 + 2 * r + 1, o1);
    if (pidx) pidx[r] = idx;
  }
  __syncwarp();
}

// One warp per agent; grid covers all agents in CSR order so that the warps
// of a block mostly share one world's road points in L1.
// Dynamic shared memory: WARPS * sizeof(ObsWarpSmem).
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_observe(DevEnv e, float* __restrict__ obs,
                                                       int32_t* __restrict__ road_idx,
                                                       int32_t* __restrict__ partner_idx) {
  extern __shared__ __align__(16) unsigned char obs_smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + wib;
  if (i >= e.A) return;
  ObsWarpSmem& sm = reinterpret_cast<ObsWarpSmem*>(obs_smem_raw)[wib];
  float4* row = reinterpret_cast<float4*>(obs + (size_t)i * e.F);
  const uint8_t f = e.flags[i];
  const float fc = (f & GD_FLAG_COLLIDED) ? 1.f : 0.f, fo = (f & GD_FLAG_OFFROAD) ? 1.f : 0.f,
              fg = (f & GD_FLAG_GOAL) ? 1.f : 0.f;
  int32_t* ridx = road_idx ? road_idx + (size_t)i * e.K : nullptr;
  int32_t* pidx = partner_idx ? partner_idx + (size_t)i * e.P : nullptr;
  if (f & GD_FLAG_DONE) {
    // removed from the scene: all-zero row except the three flags
    const int n4 = e.F >> 2;
    for (int k = lane; k < n4; k += WARP) {
      float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k == 1) o = make_float4(0.f, fc, fo, fg);
      __stcs(row + k, o);
    }
    if (ridx) for (int k = lane; k < e.K; k += WARP) ridx[k] = -1;
    if (pidx) for (int k = lane; k < e.P; k += WARP) pidx[k] = -1;
    return;
  }
  const int w = e.agent_world[i];
  const int a0 = e.agent_off[w], a1 = e.agent_off[w + 1];
  const float4 st = e.state[i];
  const float4 sc = e.stat[i];
  float s, c;
  sincosf(st.z, &s, &c);
  if (lane == 0) {
    const float gx = sc.z - st.x, gy = sc.w - st.y;
    __stcs(row + 0, make_float4(st.w, sc.x, sc.y, c * gx + s * gy));
    __stcs(row + 1, make_float4(-s * gx + c * gy, fc, fo, fg));
  }
  observe_partners(e, i, a0, a1, st.x, st.y, st.z, c, s, sm, lane, row + 2, pidx);
  observe_road(e, w, st.x, st.y, c, s, sm, lane, row + 2 + 2 * e.P, ridx);
}

}  // namespace gd
