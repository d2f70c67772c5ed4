// Polyline decimation at scene load (Sec. 3.1: a Visvalingam-Whyatt pass
// that drops points of straight stretches, 10-15x fewer points).
//
// For every polyline: the interior point of least effective area (the
// triangle it spans with its two current neighbours; ties: lower index) is
// eliminated while that area is below the tolerance; its neighbours' areas
// are recomputed with their new neighbours and raised to the eliminated
// area if smaller.  End points stay.  Points carry 64-bit keys (area bits
// << 32 | local index: areas are >= 0, so the bits order like the values and
// the index breaks ties); the elimination is sequential within a polyline.
// A polyline of up to VW_WARP_CAP points is run by one warp with its keys
// and neighbour links in shared memory: each lane keeps the minimum of its
// own chunk of keys, a shuffle reduction gives the polyline's minimum, and
// after an elimination only the lanes whose chunks changed rescan them.  A
// longer polyline is run by one thread with a binary min-heap of the keys
// and neighbour links in a scratch buffer of 20 bytes per point allocated on
// the stream.  Both take the same decisions.  Areas are float32 with the
// rounding spelled out (no contraction), so every elimination decision is
// reproducible.
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gd.h"

void gd_set_thread_error(const std::string& msg);

namespace {

__device__ __forceinline__ float vw_area(float ax, float ay, float bx, float by, float cx, float cy) {
  const float dx1 = __fsub_rn(bx, ax), dy1 = __fsub_rn(by, ay), dx2 = __fsub_rn(cx, ax), dy2 = __fsub_rn(cy, ay);
  return __fmul_rn(0.5f, fabsf(__fsub_rn(__fmul_rn(dx1, dy2), __fmul_rn(dx2, dy1))));
}

__device__ __forceinline__ unsigned long long vw_key(float area, int i) {
  return ((unsigned long long)__float_as_uint(area) << 32) | (unsigned)i;
}

struct VwHeap {
  unsigned long long* h;   // heap of keys
  int* pos;                // heap position of each local point (-1: not in the heap)
  int n;                   // entries

  __device__ void place(int k, unsigned long long key) {
    h[k] = key;
    pos[(int)(key & 0xffffffffu)] = k;
  }
  __device__ void up(int k) {
    const unsigned long long key = h[k];
    while (k > 0) {
      const int parent = (k - 1) >> 1;
      const unsigned long long pk = h[parent];
      if (pk <= key) break;
      place(k, pk);
      k = parent;
    }
    place(k, key);
  }
  __device__ void down(int k) {
    const unsigned long long key = h[k];
    for (;;) {
      int c = 2 * k + 1;
      if (c >= n) break;
      unsigned long long ck = h[c];
      if (c + 1 < n) {
        const unsigned long long c2 = h[c + 1];
        if (c2 < ck) {
          ck = c2;
          ++c;
        }
      }
      if (key <= ck) break;
      place(k, ck);
      k = c;
    }
    place(k, key);
  }
};

constexpr int VW_WARP_CAP = 1024;     // points of a polyline the warp form holds in shared memory
constexpr int VW_WARPS = 8;            // warps per CTA of the warp form
constexpr size_t VW_WARP_SMEM = (size_t)VW_WARP_CAP * (8 + 2 + 2);   // keys + two 16-bit links per point

// Warp form: one warp per polyline of at most VW_WARP_CAP points (longer
// ones are left to k_vw).  Dynamic shared memory: VW_WARPS x VW_WARP_SMEM.
__global__ void __launch_bounds__(VW_WARPS * 32) k_vw_warp(int num_polylines, const int* __restrict__ poly_off,
                                                         const float* __restrict__ x, const float* __restrict__ y,
                                                         float tol, uint8_t* __restrict__ keep) {
  extern __shared__ __align__(16) unsigned char vw_smem[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(vw_smem + (size_t)wid * VW_WARP_SMEM);
  unsigned short* prv = reinterpret_cast<unsigned short*>(keys + VW_WARP_CAP);
  unsigned short* nxt = prv + VW_WARP_CAP;
  const unsigned long long NONE = ~0ull;     // end points and eliminated points
  for (int p = blockIdx.x * VW_WARPS + wid; p < num_polylines; p += gridDim.x * VW_WARPS) {
    const int o = poly_off[p], n = poly_off[p + 1] - o;
    if (n > VW_WARP_CAP) continue;
    for (int i = lane; i < n; i += 32) keep[o + i] = 1;
    if (n < 3) continue;
    const float* px = x + o;
    const float* py = y + o;
    for (int i = lane; i < n; i += 32) {
      prv[i] = (unsigned short)(i - 1);
      nxt[i] = (unsigned short)(i + 1);
      keys[i] = (i == 0 || i == n - 1) ? NONE
                                       : vw_key(vw_area(px[i - 1], py[i - 1], px[i], py[i], px[i + 1], py[i + 1]), i);
    }
    __syncwarp();
    // lane l owns points [l ch, l ch + ch)
    const int ch = (n + 31) / 32, lo = min(lane * ch, n), hi = min(lo + ch, n);
    // four independent minima, so the chunk's loads overlap
    auto chunk_min = [&]() {
      unsigned long long m0 = NONE, m1 = NONE, m2 = NONE, m3 = NONE;
      int i = lo;
      for (; i + 3 < hi; i += 4) {
        m0 = min(m0, keys[i]);
        m1 = min(m1, keys[i + 1]);
        m2 = min(m2, keys[i + 2]);
        m3 = min(m3, keys[i + 3]);
      }
      for (; i < hi; ++i) m0 = min(m0, keys[i]);
      return min(min(m0, m1), min(m2, m3));
    };
    unsigned long long mine = chunk_min();
    for (;;) {
      // the warp's minimum key: the least area bits, then the least index
      // among the lanes that hold them
      const unsigned hb = __reduce_min_sync(0xffffffffu, (unsigned)(mine >> 32));
      const unsigned lb = __reduce_min_sync(0xffffffffu, (unsigned)(mine >> 32) == hb ? (unsigned)mine : 0xffffffffu);
      const unsigned long long m = ((unsigned long long)hb << 32) | lb;
      const float am = __uint_as_float((unsigned)(m >> 32));
      if (m == NONE || !(am < tol)) break;
      const int i = (int)(m & 0xffffffffu);
      int a = 0, c = 0;
      if (lane == 0) {
        keep[o + i] = 0;
        keys[i] = NONE;
        a = prv[i];
        c = nxt[i];
        nxt[a] = (unsigned short)c;
        prv[c] = (unsigned short)a;
        const int nb[2] = {a, c};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int j = nb[q];
          if (j <= 0 || j >= n - 1) continue;
          const int pj = prv[j], nj = nxt[j];
          const float na = fmaxf(vw_area(px[pj], py[pj], px[j], py[j], px[nj], py[nj]), am);
          keys[j] = vw_key(na, j);
        }
      }
      a = __shfl_sync(0xffffffffu, a, 0);
      c = __shfl_sync(0xffffffffu, c, 0);
      __syncwarp();
      if (lane == i / ch || lane == a / ch || lane == c / ch) mine = chunk_min();
      __syncwarp();
    }
    __syncwarp();
  }
}

// Heap form: one thread per polyline longer than min_len points (grid-
// stride).  Scratch arrays are indexed by the global point index.
__global__ void k_vw(int num_polylines, const int* __restrict__ poly_off, const float* __restrict__ x,
                     const float* __restrict__ y, float tol, uint8_t* __restrict__ keep, unsigned long long* heap,
                     int* hpos, int* prv, int* nxt, int min_len) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < num_polylines; p += gridDim.x * blockDim.x) {
    const int o = poly_off[p], n = poly_off[p + 1] - o;
    if (n <= min_len) continue;
    const float* px = x + o;
    const float* py = y + o;
    for (int i = 0; i < n; ++i) keep[o + i] = 1;
    if (n < 3) continue;
    int* pv = prv + o;
    int* nx = nxt + o;
    VwHeap hp{heap + o, hpos + o, n - 2};
    for (int i = 0; i < n; ++i) {
      pv[i] = i - 1;
      nx[i] = i + 1;
    }
    hp.pos[0] = hp.pos[n - 1] = -1;
    for (int i = 1; i + 1 < n; ++i)
      hp.place(i - 1, vw_key(vw_area(px[i - 1], py[i - 1], px[i], py[i], px[i + 1], py[i + 1]), i));
    for (int k = (hp.n >> 1) - 1; k >= 0; --k) hp.down(k);
    while (hp.n > 0) {
      const unsigned long long m = hp.h[0];
      const float am = __uint_as_float((unsigned)(m >> 32));
      if (!(am < tol)) break;
      const int i = (int)(m & 0xffffffffu);
      keep[o + i] = 0;
      hp.pos[i] = -1;
      if (--hp.n > 0) {
        hp.place(0, hp.h[hp.n]);
        hp.down(0);
      }
      const int a = pv[i], c = nx[i];
      nx[a] = c;
      pv[c] = a;
      const int nb[2] = {a, c};
      for (int q = 0; q < 2; ++q) {
        const int j = nb[q];
        if (j <= 0 || j >= n - 1) continue;
        const float na = fmaxf(vw_area(px[pv[j]], py[pv[j]], px[j], py[j], px[nx[j]], py[nx[j]]), am);
        const unsigned long long key = vw_key(na, j);
        const int k = hp.pos[j];
        const unsigned long long old = hp.h[k];
        hp.h[k] = key;
        if (key < old) hp.up(k); else hp.down(k);
      }
    }
  }
}

}  // namespace

extern "C" gd_status gd_decimate(int32_t num_polylines, int32_t num_points, const int32_t* poly_off, const float* x,
                                 const float* y, float area_tol, uint8_t* keep, void* cuda_stream) {
  if (num_polylines < 0 || num_points < 0) {
    gd_set_thread_error("gd_decimate: num_polylines and num_points must be >= 0");
    return GD_ERR_INVALID_ARG;
  }
  if (!(area_tol >= 0.f) || !(area_tol < 3.0e38f)) {
    gd_set_thread_error("gd_decimate: area_tol must be finite and >= 0");
    return GD_ERR_INVALID_ARG;
  }
  if (num_polylines == 0 || num_points == 0) return GD_OK;
  if (!poly_off || !x || !y || !keep) {
    gd_set_thread_error("gd_decimate: poly_off, x, y and keep must not be NULL");
    return GD_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t n = (size_t)num_points;
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, n * (8 + 4 + 4 + 4), s);
  if (e != cudaSuccess) {
    gd_set_thread_error(std::string("gd_decimate: scratch: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA;
  }
  unsigned long long* heap = static_cast<unsigned long long*>(scratch);
  int* hpos = reinterpret_cast<int*>(heap + n);
  int* prv = hpos + n;
  int* nxt = prv + n;
  // polylines of up to VW_WARP_CAP points: a warp each; longer ones: the heap form
  e = cudaFuncSetAttribute(k_vw_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(VW_WARPS * VW_WARP_SMEM));
  if (e == cudaSuccess) {
    const int wgrid = (num_polylines + VW_WARPS - 1) / VW_WARPS;
    k_vw_warp<<<wgrid, VW_WARPS * 32, VW_WARPS * VW_WARP_SMEM, s>>>(num_polylines, poly_off, x, y, area_tol, keep);
    const int block = 128;
    const int grid = (num_polylines + block - 1) / block;
    k_vw<<<grid, block, 0, s>>>(num_polylines, poly_off, x, y, area_tol, keep, heap, hpos, prv, nxt, VW_WARP_CAP);
    e = cudaGetLastError();
  }
  cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) {
    gd_set_thread_error(std::string("gd_decimate: launch: ") + cudaGetErrorString(e));
    return GD_ERR_CUDA;
  }
  return GD_OK;
}

// Scene-level decimation: the polylines of a host scene batch (maximal runs
// of consecutive road points of one world with one polyline id) decimated on
// the device, then the kept points compacted on the host, world by world.
extern "C" gd_status gd_decimate_scene(const gd_scene_batch* scene, float area_tol, void* cuda_stream, uint8_t* keep,
                                       int32_t* road_off_out, float* road_x_out, float* road_y_out,
                                       uint8_t* road_type_out, int32_t* road_poly_out, int32_t* num_kept) {
  auto bad = [](const char* m) {
    gd_set_thread_error(std::string("gd_decimate_scene: ") + m);
    return GD_ERR_INVALID_ARG;
  };
  if (!scene || !road_off_out || !num_kept) return bad("scene, road_off_out and num_kept must not be NULL");
  const int W = scene->num_worlds;
  if (W < 0) return bad("num_worlds must be >= 0");
  if (W > 0 && !scene->road_off) return bad("road_off must not be NULL");
  if (!(area_tol >= 0.f) || !(area_tol < 3.0e38f)) return bad("area_tol must be finite and >= 0");
  if (W > 0 && scene->road_off[0] != 0) return bad("road_off[0] must be 0");
  for (int w = 0; w < W; ++w)
    if (scene->road_off[w + 1] < scene->road_off[w]) return bad("road_off must be non-decreasing");
  const int N = W > 0 ? scene->road_off[W] : 0;
  if (N > 0 && (!scene->road_x || !scene->road_y || !scene->road_type || !scene->road_poly))
    return bad("road_x, road_y, road_type and road_poly must not be NULL");
  if (N > 0 && (!road_x_out || !road_y_out || !road_type_out || !road_poly_out))
    return bad("road_x_out, road_y_out, road_type_out and road_poly_out must not be NULL");
  // polylines: a new one starts at each world's first point and wherever the id changes
  std::vector<int32_t> off;
  off.reserve(1024);
  for (int w = 0; w < W; ++w)
    for (int p = scene->road_off[w]; p < scene->road_off[w + 1]; ++p)
      if (p == scene->road_off[w] || scene->road_poly[p] != scene->road_poly[p - 1]) off.push_back(p);
  off.push_back(N);
  const int P = (int)off.size() - 1;
  std::vector<uint8_t> k((size_t)N, 1);
  if (N > 0) {
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)N;
    // one device block: polyline offsets, x, y, keep (each part 16-byte aligned)
    const size_t b_off = ((size_t)(P + 1) * 4 + 15) & ~(size_t)15, b_xy = (n * 4 + 15) & ~(size_t)15;
    void* dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, b_off + 2 * b_xy + n, s);
    if (e != cudaSuccess) {
      gd_set_thread_error(std::string("gd_decimate_scene: device buffers: ") + cudaGetErrorString(e));
      return e == cudaErrorMemoryAllocation ? GD_ERR_OOM : GD_ERR_CUDA;
    }
    char* base = static_cast<char*>(dev);
    int32_t* d_off = reinterpret_cast<int32_t*>(base);
    float* d_x = reinterpret_cast<float*>(base + b_off);
    float* d_y = reinterpret_cast<float*>(base + b_off + b_xy);
    uint8_t* d_keep = reinterpret_cast<uint8_t*>(base + b_off + 2 * b_xy);
    e = cudaMemcpyAsync(d_off, off.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, scene->road_x, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_y, scene->road_y, sizeof(float) * n, cudaMemcpyHostToDevice, s);
    gd_status st = GD_OK;
    if (e == cudaSuccess) st = gd_decimate(P, N, d_off, d_x, d_y, area_tol, d_keep, cuda_stream);
    if (e == cudaSuccess && st == GD_OK) e = cudaMemcpyAsync(k.data(), d_keep, n, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st != GD_OK) return st;
    if (e != cudaSuccess) {
      gd_set_thread_error(std::string("gd_decimate_scene: ") + cudaGetErrorString(e));
      return GD_ERR_CUDA;
    }
  }
  // compaction, world by world (kept points keep their order)
  int m = 0;
  road_off_out[0] = 0;
  for (int w = 0; w < W; ++w) {
    for (int p = scene->road_off[w]; p < scene->road_off[w + 1]; ++p) {
      if (!k[(size_t)p]) continue;
      road_x_out[m] = scene->road_x[p];
      road_y_out[m] = scene->road_y[p];
      road_type_out[m] = scene->road_type[p];
      road_poly_out[m] = scene->road_poly[p];
      ++m;
    }
    road_off_out[w + 1] = m;
  }
  if (keep && N > 0) std::memcpy(keep, k.data(), (size_t)N);
  *num_kept = m;
  return GD_OK;
}
