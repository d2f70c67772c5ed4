// Per-world kernel of the batched form: one persistent launch runs the whole
// step -- masked reset, dynamics (App. B or the simplified model of Sec.
// 3.2), agent grid and box collision, road-edge test, goal / reward / done
// (Sec. 3.2) -- of every world, and (the fused form) its observation, taking
// worlds from a work list: each CTA's first world by its index, the rest
// from an atomic counter that the last CTA out leaves at zero for the next
// launch (no grid-wide synchronisation, no memset between launches).  In the
// split form the observation is a second launch, k_observe_split.
//
// Per world the CTA keeps the agents in shared memory and, when it pays,
// copies the world's cell-sorted road points into a shared-memory tile with
// one cp.async.bulk (TMA) copy, issued first so that it overlaps the step
// stages; otherwise the road is read from global memory (the road-edge test
// from the edge grid).  The mbarrier wait is bounded: after ~2 s the CTA
// sets ERR_TIMEOUT, waits once more (bounded) for its copy and leaves the
// world loop; other CTAs keep draining the work list.  Collision and the
// road-edge test (without the tile) run over the world's (agent, candidate)
// pairs laid end to end, so the CTA's threads share a world's tests evenly
// however the candidates fall among its agents.
#pragma once
#include "gd_device.cuh"
#include "observe_kernel.cuh"
#include "lidar_kernel.cuh"

namespace gd {

// Road bytes one agent's observation reads from its world's block (the
// candidates of its disk, about 500 points of 12 B at the default density):
// below n * TILE_AGENT_BYTES a block is read from global memory instead of
// being copied into the tile.
constexpr unsigned TILE_AGENT_BYTES = 6144;

struct FusedArgs {
  const float2* actions;     // [A] (step) or nullptr
  float* reward;             // [A] or nullptr
  uint8_t* done;             // [A] or nullptr
  uint8_t* world_done;       // [W] or nullptr
  float* obs;                // [A,F] or nullptr (no observation)
  int32_t* road_idx;         // [A,K] or nullptr
  int32_t* partner_idx;      // [A,P] or nullptr
  unsigned* counter;         // [2] work counter and exit tally: zero at launch, left at zero by the launch
  const int* order;          // [W] world order (largest first)
  int tile_bytes;            // bytes of the shared-memory road tile
  int do_step;
  // objective terms ell[i] = obs_w . obs row + reward_w * r_s (agents in the
  // scene at the start of the step), written when ell != nullptr; a launch
  // without observation (obs == nullptr) writes r_s alone, for the split
  // observation launch to complete
  const float* obs_w;        // [F], 16-byte aligned
  float reward_w;
  float* ell;                // [A] or nullptr
  float* rk_out;             // [A] with ell: each observed agent's K-th road distance (+inf: fewer), or nullptr
  uint16_t* sel_out;         // [A][K] with ell: each observed agent's road selection (block positions), or nullptr
  unsigned* clear;           // cleared (clear_n words) by the launch, for the launch that follows; or nullptr
  int clear_n;
  // step out of place: the post-step state and flags go here instead of
  // over e.state / e.flags (which the launch then only reads); nullptr = in
  // place.  The backward pass recomputes a checkpoint segment this way, each
  // step's state in its own slot, without a copy per step.
  float4* state_out;
  uint8_t* flags_out;
  uint8_t* flags_rec;        // [A] a second copy of the post-step flags (the objective rollout's record of
                             // its decisions, for the backward pass's recompute), or nullptr
  LidarArgs lidar;           // LiDAR observation (k_world<W, true>); lidar.depth == nullptr: none
};

struct FusedAgents {
  float4 st[GD_MAX_AGENTS_PER_WORLD];
  float4 sc[GD_MAX_AGENTS_PER_WORLD];
  float2 cs[GD_MAX_AGENTS_PER_WORLD];        // (cos theta, sin theta) after the step
  uint32_t key[GD_MAX_AGENTS_PER_WORLD];     // sorted grid keys of the active agents
  uint8_t fl[GD_MAX_AGENTS_PER_WORLD];
  uint8_t ty[GD_MAX_AGENTS_PER_WORLD];
  uint8_t coll[GD_MAX_AGENTS_PER_WORLD];
  uint8_t offr[GD_MAX_AGENTS_PER_WORLD];
  uint8_t act0[GD_MAX_AGENTS_PER_WORLD];     // in the scene at the start of the step
  int poff[GD_MAX_AGENTS_PER_WORLD];         // collision / road-edge test: the agent's first pair
  int2 prow[GD_MAX_AGENTS_PER_WORLD][3];     // collision / road-edge test: (first, count) per range
};

// ---- TMA bulk copy + mbarrier (inline PTX) --------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier: true when it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > 4000000000ll) return false;    // ~2 s at 2 GHz
  }
  return true;
}

// 1-D bulk copy global -> this CTA's shared memory; completion is reported
// to the mbarrier as transferred bytes.  dst, src 16-byte aligned, bytes a
// multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Dynamic shared memory: [mbarrier, 128 B][road tile, tile_bytes][FusedAgents]
// then per warp an ObsWarpSmem (radial observation) or LidarWarpHead + one
// key per ray followed by the CTA's copy of the ray directions (LIDAR).
// LEAN: the instantiation for the form without the road tile and for the
// step alone, both bound by latency (per-world barriers, dependent loads).
// Registers are capped for 40 warps per SM (48 per thread at 4 or 8 warps
// per CTA, a few bytes of spill): the step alone (10 KB of shared memory per
// 4-warp CTA) then holds ten worlds per SM instead of the eight of a
// 64-register cap, which shortens launches that take more than one round of
// worlds (4,096 uneven worlds: 43.7 -> 37.4 us); the form with observation
// stays below that for its shared memory.  The tile form keeps its
// registers (its tile holds it at 2 CTAs per SM anyway).
// Road-edge test without the tile: cell rows per agent read up front (a box
// over more rows walks the rest itself; the pair lists hold 3 ranges per
// agent) and (agent, segment) pairs per thread per round.
constexpr int EDGE_ROWS = 3;
static_assert(EDGE_ROWS == 3, "the pair lists hold three ranges per agent");
constexpr int EDGE_U = 4;

template <int WARPS, bool LIDAR = false, bool LEAN = false>
__global__ void __launch_bounds__(WARPS * 32, LEAN ? 40 / WARPS : 1) k_world(DevEnv e, FusedArgs a) {
  extern __shared__ __align__(16) unsigned char wsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(wsm);
  unsigned char* tile = wsm + 128;
  FusedAgents& ag = *reinterpret_cast<FusedAgents*>(wsm + 128 + (size_t)a.tile_bytes);
  unsigned char* warp_base = reinterpret_cast<unsigned char*>(&ag) + sizeof(FusedAgents);
  __shared__ int s_w;
  __shared__ int s_nact;
  __shared__ int s_abort;
  __shared__ int s_next;
  __shared__ int s_psum[WARPS];  // pair lists: pairs per warp
  __shared__ GridDesc s_eg;   // the world's edge-grid descriptor, read early (used after the collision stage)
  static_assert(WARPS * 32 >= GD_MAX_AGENTS_PER_WORLD, "the step stages take one thread per agent");
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  ObsWarpSmem& osm = reinterpret_cast<ObsWarpSmem*>(warp_base)[wid];
  unsigned char* lbase = warp_base + (size_t)wid * (size_t)a.lidar.warp_bytes;
  LidarWarpHead& lh = *reinterpret_cast<LidarWarpHead*>(lbase);
  unsigned* lkeys = reinterpret_cast<unsigned*>(lbase + sizeof(LidarWarpHead));
  LidarArgs lar = a.lidar;
  if constexpr (LIDAR) {
    float2* sdirs = reinterpret_cast<float2*>(warp_base + (size_t)WARPS * (size_t)a.lidar.warp_bytes);
    lidar_stage_dirs(sdirs, a.lidar.dirs, a.lidar.fan.n);
    lar.dirs = sdirs;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    s_abort = 0;
  }
  // the counters of the observation launch that follows (split forms)
  if (a.clear && blockIdx.x == 0)
    for (int i = tid; i < a.clear_n; i += WARPS * 32) a.clear[i] = 0u;
  __syncthreads();
  unsigned phase = 0;
  const bool observe = LIDAR ? a.lidar.depth != nullptr : a.obs != nullptr;
  // the first world of each CTA is world order[blockIdx.x] (the grid never
  // exceeds W); the rest are claimed from the counter (cleared before the
  // launch), after those
  bool first = true;
  for (;;) {
    if (tid == 0) s_w = first ? (int)blockIdx.x : (int)(gridDim.x + atomicAdd(a.counter, 1u));
    first = false;
    __syncthreads();
    const int k = s_w;
    if (k >= e.W) break;
    const int w = a.order[k];
    const int a0 = e.agent_off[w], n = e.agent_off[w + 1] - a0;
    const int nr = e.road_off[w + 1] - e.road_off[w];
    const GridDesc g = e.rgrid[w];
    const unsigned block = (unsigned)g.block_bytes;
    const unsigned char* gblock = e.arena + (size_t)e.arena_off[w] * 16;
    // the tile pays when the world's agents would read more of the block
    // than its size (each agent reads its disk's candidates, a few KB)
    const bool use_tile = nr > 0 && block <= (unsigned)a.tile_bytes && (unsigned)n * TILE_AGENT_BYTES >= block;
    if (use_tile && tid == 0) {
      fence_proxy_async_smem();     // earlier generic reads of the tile before the async write
      mbar_arrive_expect_tx(bar, block);
      tma_load_1d(tile, gblock, block, bar);
    }
    if (tid == 0) {
      s_next = WARPS;
      if (a.do_step) s_eg = e.egrid[w];
    }
    // Two views of the world: one on the shared-memory tile, one on the
    // global road block.  Each use site picks one with a uniform branch, so
    // the shared path compiles to shared-memory accesses.
    WorldView vt, vg;
    vt.state = vg.state = ag.st;
    vt.stat = vg.stat = ag.sc;
    vt.cs = vg.cs = ag.cs;
    vt.flags = vg.flags = ag.fl;
    vt.n = vg.n = n;
    vt.g = vg.g = g;
    road_block(tile, nr, vt);
    road_block(gblock, nr, vg);
    bool tile_ready = !use_tile;
    // every thread waits for the tile (bounded); false = give up this CTA
    auto wait_tile = [&]() -> bool {
      if (!tile_ready) {
        if (!mbar_wait_bounded(bar, phase)) s_abort = 1;
        phase ^= 1u;
        tile_ready = true;
      }
      __syncthreads();
      if (s_abort) {
        if (tid == 0) {
          atomicOr(e.err, ERR_TIMEOUT);
          mbar_wait_bounded(bar, phase ^ 1u);   // give the copy one more bounded chance to land
        }
        __syncthreads();
        return false;
      }
      return true;
    };
    // Pair lists of the collision and road-edge tests: thread tid < n holds
    // the cnt pairs of agent tid as up to 3 ranges (first, count) in
    // ag.prow[tid].  lay_pairs lays the agents' pairs end to end (ag.poff:
    // exclusive offsets, by a block scan) and returns the world's total;
    // pair_at gives pair f's agent (the last whose pairs start at or before
    // f) and its index in the agent's ranges.
    auto lay_pairs = [&](int cnt) -> int {
      const int incl = warp_incl_scan(cnt, lane);
      if (lane == WARP - 1) s_psum[wid] = incl;
      __syncthreads();
      int total = 0, base = 0;
#pragma unroll
      for (int q = 0; q < WARPS; ++q) {
        const int t = s_psum[q];
        base += q < wid ? t : 0;
        total += t;
      }
      if (tid < n) ag.poff[tid] = base + incl - cnt;
      __syncthreads();
      return total;
    };
    auto pair_at = [&](int f, int& who) -> int {
      int lo = 0, hi = n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ag.poff[mid] <= f) lo = mid; else hi = mid - 1;
      }
      who = lo;
      int rel = f - ag.poff[lo], q = -1;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int2 rr = ag.prow[lo][r];
        if (q < 0 && rel < rr.y) q = rr.x + rel;
        if (q < 0) rel -= rr.y;
      }
      return q;
    };
    if (a.do_step) {
      const bool reset = (e.cflags & GD_AUTO_RESET) && e.world_done[w];
      const float inv = 1.f / e.agent_cell;
      bool act = false;
      uint32_t key = 0;
      if (tid < n) {
        const int i = a0 + tid;
        // every load of the agent goes out at once; a world that restarts
        // (rare) then reads its initial snapshot
        float4 s = e.state[i];
        uint8_t f = e.flags[i];
        const float2 u = a.actions[i];
        const float4 sci = e.stat[i];
        const uint8_t ty = e.type[i];
        if (reset) {
          s = e.init_state[i];
          f = e.init_flags[i];
        }
        ag.act0[tid] = !(f & GD_FLAG_DONE);
        if (!(f & GD_FLAG_DONE)) {
          // uncontrolled agents (GD_FLAG_STATIC) stay in the grid but do not move
          if (!(f & GD_FLAG_STATIC) && !dynamics_step(e.dyn, s, u.x, u.y, sci.x, e.dt, e.vmax))
            atomicOr(e.err, ERR_ACTION);
          act = true;
          key = agent_cell_key((int)clampf(floorf((s.x - g.ox) * inv), 0.f, 4095.f),
                               (int)clampf(floorf((s.y - g.oy) * inv), 0.f, 4095.f), tid);
        }
        ag.st[tid] = s;
        float sn, cn;
        sincosf(s.z, &sn, &cn);
        ag.cs[tid] = make_float2(cn, sn);
        ag.sc[tid] = sci;
        ag.fl[tid] = f;
        ag.ty[tid] = ty;
        // an agent out of the grid (done) and the slots past n hold a key
        // above every cell's, so the rank below counts active keys only
        ag.key[tid] = act ? key : 0xffffffffu;
      } else if (tid < GD_MAX_AGENTS_PER_WORLD) {
        ag.key[tid] = 0xffffffffu;
      }
      const int nact = __syncthreads_count(act);
      // agent grid: rank of each active key among the active keys (keys are
      // distinct: the low byte is the agent's index), four keys per load
      uint32_t rank = 0;
      if (act) {
        const uint4* __restrict__ k4 = reinterpret_cast<const uint4*>(ag.key);
        for (int q = 0; q < (n + 3) >> 2; ++q) {
          const uint4 kq = k4[q];
          rank += (kq.x < key) + (kq.y < key) + (kq.z < key) + (kq.w < key);
        }
      }
      __syncthreads();
      if (act) ag.key[rank] = key;
      if (tid == 0) s_nact = nact;
      __syncthreads();
      // collision over the world's (agent, candidate) pairs: each active
      // agent's thread bounds the three neighbouring columns of the agent
      // grid (rows cy - 1 .. cy + 1 of a column are one run of the sorted
      // keys; six independent binary searches), the pairs are laid end to
      // end and every thread tests one per round
      {
        int cnt = 0;
        if (tid < n) {
          int lo[6], hi[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) lo[k] = hi[k] = 0;
          if (!(ag.fl[tid] & (GD_FLAG_DONE | GD_FLAG_STATIC))) {
            const float4 s = ag.st[tid];
            const int cx = (int)clampf(floorf((s.x - g.ox) * inv), 0.f, 4095.f);
            const int cy = (int)clampf(floorf((s.y - g.oy) * inv), 0.f, 4095.f);
            uint32_t v[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              const int c = cx - 1 + (k >> 1);
              v[k] = (k & 1) ? agent_cell_key(c, min(cy + 1, 4095), 255) : agent_cell_key(c, max(cy - 1, 0), 0);
              // a column off the grid has no candidates
              if (c >= 0 && c <= 4095) hi[k] = s_nact;
            }
            // lower bound (even k) / upper bound (odd k) of each column's run;
            // 8 halvings cover the at most 128 keys
#pragma unroll
            for (int it = 0; it < 8; ++it) {
#pragma unroll
              for (int k = 0; k < 6; ++k) {
                if (lo[k] < hi[k]) {
                  const int m = (lo[k] + hi[k]) >> 1;
                  if ((k & 1) ? (ag.key[m] <= v[k]) : (ag.key[m] < v[k])) lo[k] = m + 1; else hi[k] = m;
                }
              }
            }
          }
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            ag.prow[tid][r] = make_int2(lo[2 * r], lo[2 * r + 1] - lo[2 * r]);
            cnt += lo[2 * r + 1] - lo[2 * r];
          }
          ag.coll[tid] = 0;
        }
        const int total = lay_pairs(cnt);
        for (int f = tid; f < total; f += WARPS * WARP) {
          int li;
          const int j = (int)(ag.key[pair_at(f, li)] & 0xffu);
          if (j == li) continue;
          const float4 s = ag.st[li], sc = ag.sc[li];
          const float2 ci = ag.cs[li];
          const float4 sj = ag.st[j], tj = ag.sc[j];
          const float2 cj = ag.cs[j];
          if (box_box_depth(sj.x - s.x, sj.y - s.y, ci.x, ci.y, 0.5f * sc.x, 0.5f * sc.y, cj.x, cj.y, 0.5f * tj.x,
                            0.5f * tj.y) > 0.f)
            ag.coll[li] = 1;
        }
      }
      // road edges: from the shared-memory tile a warp per agent, ballot-OR
      // over the candidate segments; else from the edge grid (segments under
      // every cell their bounding box touches, so the cells under the box's
      // own bounding box hold every segment it can cross), over the world's
      // (agent, segment) pairs: each agent's thread reads the segment ranges
      // of its cell rows, a block scan lays the agents' pairs end to end, and
      // every thread tests EDGE_U pairs per round, so the whole world's
      // segment loads go out in one or two rounds whatever the agents' counts
      if (!wait_tile()) break;
      if (use_tile) {
        for (int li = wid; li < n; li += WARPS) {
          if ((ag.fl[li] & (GD_FLAG_DONE | GD_FLAG_STATIC)) || ag.ty[li] == GD_AGENT_PEDESTRIAN) {
            if (lane == 0) ag.offr[li] = 0;
            continue;
          }
          const float4 s = ag.st[li];
          const float4 sc = ag.sc[li];
          const bool off = offroad_from_block(vt, s.x, s.y, ag.cs[li].x, ag.cs[li].y, 0.5f * sc.x, 0.5f * sc.y, lane);
          if (lane == 0) ag.offr[li] = off ? 1 : 0;
        }
      } else {
        const GridDesc& eg = s_eg;
        const int* __restrict__ cst = e.ecell_start + eg.cell_base;
        int cnt = 0;
        if (tid < n) {
          bool hit = false;
          int2 rw[EDGE_ROWS];
#pragma unroll
          for (int r = 0; r < EDGE_ROWS; ++r) rw[r] = make_int2(0, 0);
          if (!(ag.fl[tid] & (GD_FLAG_DONE | GD_FLAG_STATIC)) && ag.ty[tid] != GD_AGENT_PEDESTRIAN) {
            const float4 s = ag.st[tid];
            const float4 sc = ag.sc[tid];
            const float2 cs = ag.cs[tid];
            const float hl = 0.5f * sc.x, hw = 0.5f * sc.y;
            const float ex = hl * fabsf(cs.x) + hw * fabsf(cs.y) + 1e-3f, ey = hl * fabsf(cs.y) + hw * fabsf(cs.x) + 1e-3f;
            const int cx0 = (int)clampf(floorf((s.x - ex - eg.ox) * eg.inv_cs), 0.f, (float)(eg.nx - 1));
            const int cx1 = (int)clampf(floorf((s.x + ex - eg.ox) * eg.inv_cs), -1.f, (float)(eg.nx - 1));
            const int cy0 = (int)clampf(floorf((s.y - ey - eg.oy) * eg.inv_cs), 0.f, (float)(eg.ny - 1));
            const int cy1 = (int)clampf(floorf((s.y + ey - eg.oy) * eg.inv_cs), -1.f, (float)(eg.ny - 1));
            if (cx0 <= cx1) {
              int b[EDGE_ROWS], en[EDGE_ROWS];
#pragma unroll
              for (int r = 0; r < EDGE_ROWS; ++r) {
                b[r] = en[r] = 0;
                if (cy0 + r <= cy1) {
                  const int* row = cst + (cy0 + r) * eg.nx;
                  b[r] = row[cx0];
                  en[r] = row[cx1 + 1];
                }
              }
#pragma unroll
              for (int r = 0; r < EDGE_ROWS; ++r) rw[r] = make_int2(b[r], en[r] - b[r]);
              // rows past EDGE_ROWS (boxes over EDGE_ROWS cells high): this thread walks them
              for (int cy = cy0 + EDGE_ROWS; cy <= cy1; ++cy) {
                const int* row = cst + cy * eg.nx;
                for (int q = row[cx0], qe = row[cx1 + 1]; q < qe; ++q)
                  hit |= box_seg_depth(s.x, s.y, cs.x, cs.y, hl, hw, e.esegs[q]) > 0.f;
              }
            }
          }
#pragma unroll
          for (int r = 0; r < EDGE_ROWS; ++r) {
            ag.prow[tid][r] = rw[r];
            cnt += rw[r].y;
          }
          ag.offr[tid] = hit ? 1 : 0;
        }
        const int total = lay_pairs(cnt);
        // EDGE_U pairs per thread per round, their loads in flight together
        for (int f0 = 0; f0 < total; f0 += EDGE_U * WARPS * WARP) {
          int p[EDGE_U], who[EDGE_U];
#pragma unroll
          for (int u = 0; u < EDGE_U; ++u) {
            const int f = f0 + u * WARPS * WARP + tid;
            p[u] = -1;
            who[u] = 0;
            if (f < total) p[u] = pair_at(f, who[u]);
          }
          float4 sg[EDGE_U];
#pragma unroll
          for (int u = 0; u < EDGE_U; ++u) sg[u] = p[u] >= 0 ? e.esegs[p[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < EDGE_U; ++u) {
            if (p[u] < 0) continue;
            const int li = who[u];
            const float4 s = ag.st[li];
            const float4 sc = ag.sc[li];
            const float2 cs = ag.cs[li];
            if (box_seg_depth(s.x, s.y, cs.x, cs.y, 0.5f * sc.x, 0.5f * sc.y, sg[u]) > 0.f) ag.offr[li] = 1;
          }
        }
      }
      __syncthreads();
      // goal, reward, flags, done
      bool dn = true, ctrl = false;
      if (tid < n) {
        const int i = a0 + tid;
        uint8_t f = ag.fl[tid];
        float r = 0.f;
        ctrl = !(f & GD_FLAG_STATIC);
        if (!(f & (GD_FLAG_DONE | GD_FLAG_STATIC))) {
          const float4 s = ag.st[tid];
          const float4 sc = ag.sc[tid];
          const float dx = s.x - sc.z, dy = s.y - sc.w;
          const bool at_goal = sqrtf(fmaf(dx, dx, __fmul_rn(dy, dy))) <= e.goal_r;
          const bool coll = ag.coll[tid] != 0, offr = ag.offr[tid] != 0;
          const bool first = at_goal && !(f & GD_FLAG_GOAL);
          f &= (uint8_t)~(GD_FLAG_COLLIDED | GD_FLAG_OFFROAD);
          if (at_goal) f |= GD_FLAG_GOAL;
          if (coll) f |= GD_FLAG_COLLIDED;
          if (offr) f |= GD_FLAG_OFFROAD;
          if ((f & GD_FLAG_GOAL) || (coll && (e.cflags & GD_TERM_COLLISION)) || (offr && (e.cflags & GD_TERM_OFFROAD)))
            f |= GD_FLAG_DONE;
          r = (first ? 1.f : 0.f) - (coll ? e.cpen : 0.f) - (offr ? e.opn : 0.f);
        }
        ag.fl[tid] = f;
        (a.state_out ? a.state_out : e.state)[i] = ag.st[tid];
        (a.flags_out ? a.flags_out : e.flags)[i] = f;
        if (a.flags_rec) a.flags_rec[i] = f;
        if (a.reward) a.reward[i] = r;
        if (a.done) a.done[i] = (f & (GD_FLAG_DONE | GD_FLAG_STATIC)) ? 1 : 0;
        dn = (f & (GD_FLAG_DONE | GD_FLAG_STATIC)) != 0;
        if (a.ell && !observe) {
          // split objective: the smooth goal reward of an agent in the scene
          // at the start of the step goes to ell[i]; the observation launch
          // that follows folds it in (ell[i] = reward_w * ell[i] + obs term)
          float rs = 0.f;
          if (ag.act0[tid] && !(f & GD_FLAG_STATIC)) {
            const float4 st = ag.st[tid], sc = ag.sc[tid];
            const float dx = st.x - sc.z, dy = st.y - sc.w, c = e.smooth_c;
            rs = c - sqrtf(fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(c, c))));
          }
          a.ell[i] = rs;
        }
      }
      // end of episode: every controlled agent done (a world without
      // controlled agents only times out), or t = T
      const int all_done = __syncthreads_and(dn);
      const int any_ctrl = __syncthreads_or(ctrl);
      if (tid == 0) {
        const int t = (reset ? 0 : e.t[w]) + 1;
        e.t[w] = t;
        const uint8_t wd = ((any_ctrl && all_done) || t >= e.T) ? 1 : 0;
        e.world_done[w] = wd;
        if (a.world_done) a.world_done[w] = wd;
      }
    } else if (observe && tid < n) {
      const float4 s = e.state[a0 + tid];
      ag.st[tid] = s;
      float sn, cn;
      sincosf(s.z, &sn, &cn);
      ag.cs[tid] = make_float2(cn, sn);
      ag.sc[tid] = e.stat[a0 + tid];
      ag.fl[tid] = e.flags[a0 + tid];
    }
    if (observe) {
      if (!wait_tile()) break;
      // warps take the world's agents one at a time (first WARPS statically)
      for (int li = wid; li < n;) {
        const int i = a0 + li;
        if constexpr (LIDAR) {
          const LidarArgs& la = lar;
          const size_t ro = (size_t)i * la.fan.n;
          const float hd = la.head ? la.head[i] : 0.f;
          if (use_tile) lidar_agent(vt, li, e.R, hd, la, la.depth + ro, la.cls ? la.cls + ro : nullptr, lh, lkeys, lane);
          else lidar_agent(vg, li, e.R, hd, la, la.depth + ro, la.cls ? la.cls + ro : nullptr, lh, lkeys, lane);
          int nx = 0;
          if (lane == 0) nx = atomicAdd(&s_next, 1);
          li = __shfl_sync(0xffffffffu, nx, 0);
          continue;
        }
        float* orow = a.obs + (size_t)i * e.F;
        int32_t* ridx = a.road_idx ? a.road_idx + (size_t)i * e.K : nullptr;
        int32_t* pidx = a.partner_idx ? a.partner_idx + (size_t)i * e.P : nullptr;
        if (a.ell) {
          float4* anc = e.anchor ? e.anchor + i : nullptr;
          float* rks = a.rk_out ? a.rk_out + i : nullptr;
          uint16_t* sels = a.sel_out ? a.sel_out + (size_t)i * e.K : nullptr;
          const float dot = use_tile ? observe_agent<true>(e, vt, li, orow, ridx, pidx, osm, lane, anc, a.obs_w, rks,
                                                           nullptr, sels)
                                     : observe_agent<true>(e, vg, li, orow, ridx, pidx, osm, lane, anc, a.obs_w, rks,
                                                           nullptr, sels);
          if (lane == 0) {
            float rs = 0.f;
            if (a.do_step && ag.act0[li] && !(ag.fl[li] & GD_FLAG_STATIC)) {
              const float4 st = ag.st[li], sc = ag.sc[li];
              const float dx = st.x - sc.z, dy = st.y - sc.w, c = e.smooth_c;
              rs = c - sqrtf(fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(c, c))));
            }
            a.ell[i] = fmaf(a.reward_w, rs, dot);
          }
        } else if (use_tile) {
          observe_agent<false>(e, vt, li, orow, ridx, pidx, osm, lane, e.anchor ? e.anchor + i : nullptr);
        } else {
          observe_agent<false>(e, vg, li, orow, ridx, pidx, osm, lane, e.anchor ? e.anchor + i : nullptr);
        }
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&s_next, 1);
        li = __shfl_sync(0xffffffffu, nx, 0);
      }
    }
    __syncthreads();
  }
  // the last CTA out leaves the work counter and the exit tally at zero for
  // the next launch, so no memset separates two launches (every CTA has made
  // its last claim before it counts itself out)
  __syncthreads();
  if (tid == 0 && atomicAdd(a.counter + 1, 1u) == gridDim.x - 1) {
    a.counter[0] = 0u;
    a.counter[1] = 0u;
  }
  // A step launched as a programmatic dependent of the previous observation
  // launch (the overlapped rollout: it reads and writes other state buffers
  // than that launch) ends only once that launch has, so the observation
  // launch after it never overlaps the one before.  Without such a launch
  // this returns at once.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

}  // namespace gd
