// scene.cu -- voxel-hashed TSDF scene: host-side table build, device lookup, the raycast
// kernel used for query renders, training renders and depth-difference verification.
//
// Sec. 3.3 (a): each agent's sub-scene is an InfiniTAM-style voxel map; Sec. 3.3.1 / Fig. 3:
// relocalisation renders colour + depth of scene b from a frame's pose and verifies a proposed
// pose with a depth render of scene a (Omega_s and mu).  The march below is the library's
// reading of the usual voxel raycast (the paper names it in its appendix on global map
// rendering without giving its steps).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "relo_internal.cuh"

namespace relo {

// ---------------------------------------------------------------------------------------------
// Trilinear sampling with a per-thread cache of the block holding the previous sample.
// ---------------------------------------------------------------------------------------------
struct BlockCache {
  int bx, by, bz, ptr;
};

__device__ __forceinline__ int cached_block(const SceneView& s, BlockCache& c, int bx, int by, int bz, int* err) {
  if (bx != c.bx || by != c.by || bz != c.bz) {
    c.bx = bx;
    c.by = by;
    c.bz = bz;
    c.ptr = s.grid ? grid_block(s, bx, by, bz) : lookup_block(s, bx, by, bz, err);
  }
  return c.ptr;
}

// Per-ray constants for cell exits: reciprocal direction, which face each axis leaves through.
struct RayExit {
  float3 inv;
  int px, py, pz;      // 1 if the ray moves toward +axis
  bool zx, zy, zz;     // the ray is parallel to that axis' faces
};

__device__ __forceinline__ RayExit ray_exit(float3 d) {
  RayExit r;
  r.inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  r.px = d.x > 0.f;
  r.py = d.y > 0.f;
  r.pz = d.z > 0.f;
  r.zx = d.x == 0.f;
  r.zy = d.y == 0.f;
  r.zz = d.z == 0.f;
  return r;
}

// Ray parameter at which the ray leaves the cube of blocks b - (r - 1) ... b + (r - 1) per axis
// (r = 1: block b itself).  Its faces are block faces, (float)(integer) * block size as for a
// single block, so the exit equals that of the last block a block-by-block walk would visit.
__device__ __forceinline__ float cube_exit(float3 C, const RayExit& e, int bx, int by, int bz, int r, float bs) {
  const float lx = e.zx ? INFINITY : ((float)(bx + (e.px ? r : 1 - r)) * bs - C.x) * e.inv.x;
  const float ly = e.zy ? INFINITY : ((float)(by + (e.py ? r : 1 - r)) * bs - C.y) * e.inv.y;
  const float lz = e.zz ? INFINITY : ((float)(bz + (e.pz ? r : 1 - r)) * bs - C.z) * e.inv.z;
  return fminf(lx, fminf(ly, lz));
}

// Blocks holding the 8 corners of the voxel cell at (i, j, k) (corner n = (i + (n & 1),
// j + (n >> 1 & 1), k + (n >> 2))), given b0 = the block of (i, j, k): a corner leaves b0 only
// along the axes where the cell sits on b0's last voxel, so at most 7 further lookups, usually 0
// or 1 (instead of one per corner through a one-entry cache that neighbouring corners evict).
__device__ __forceinline__ void corner_blocks(const SceneView& s, BlockCache& c, int b0, int i, int j, int k,
                                              int (&blk)[8], int* err) {
  const int bx = i >> 3, by = j >> 3, bz = k >> 3;
  const bool ex = (i & 7) == 7, ey = (j & 7) == 7, ez = (k & 7) == 7;
  blk[0] = b0;
  blk[1] = ex ? cached_block(s, c, bx + 1, by, bz, err) : b0;
  blk[2] = ey ? cached_block(s, c, bx, by + 1, bz, err) : b0;
  blk[3] = ex ? (ey ? cached_block(s, c, bx + 1, by + 1, bz, err) : blk[1]) : blk[2];
  if (ez) {
    blk[4] = cached_block(s, c, bx, by, bz + 1, err);
    blk[5] = ex ? cached_block(s, c, bx + 1, by, bz + 1, err) : blk[4];
    blk[6] = ey ? cached_block(s, c, bx, by + 1, bz + 1, err) : blk[4];
    blk[7] = ex ? (ey ? cached_block(s, c, bx + 1, by + 1, bz + 1, err) : blk[5]) : blk[6];
  } else {
    blk[4] = blk[0];
    blk[5] = blk[1];
    blk[6] = blk[2];
    blk[7] = blk[3];
  }
}

// Index inside its block of corner n of the voxel cell at (i, j, k).
__device__ __forceinline__ int corner_voxel(int i, int j, int k, int n) {
  return ((i + (n & 1)) & 7) + 8 * ((j + ((n >> 1) & 1)) & 7) + 64 * ((k + (n >> 2)) & 7);
}

// Trilinear tsdf at voxel-space point q (= p / voxel), given the block b0 holding floor(q);
// corners in unallocated blocks read +1.  kApron: from the scene's apron copy (s.tsdf9, which
// every job of the launch has), where all eight corners lie in block b0 and hold the values the
// neighbour lookups below would read; otherwise from the blocks' own tsdf.
template <bool kApron>
__device__ __forceinline__ float trilinear_tsdf(const SceneView& s, BlockCache& c, int b0, int i, int j, int k,
                                                float fx, float fy, float fz, int* err) {
  float v[8];
  if (!RELO_CHECK(b0 < s.n_blocks)) return 1.0f;
  if (kApron) {
    const float* base = s.tsdf9 + (size_t)b0 * kApronStride + (i & 7) + 9 * (j & 7) + 81 * (k & 7);
    v[0] = __ldg(base);
    v[1] = __ldg(base + 1);
    v[2] = __ldg(base + 9);
    v[3] = __ldg(base + 10);
    v[4] = __ldg(base + 81);
    v[5] = __ldg(base + 82);
    v[6] = __ldg(base + 90);
    v[7] = __ldg(base + 91);
  } else if ((i & 7) != 7 && (j & 7) != 7 && (k & 7) != 7) {
    // all eight corners inside block b0: one contiguous neighbourhood
    const float* base = s.tsdf + (size_t)b0 * kVoxelsPerBlock + (i & 7) + 8 * (j & 7) + 64 * (k & 7);
    v[0] = __ldg(base);
    v[1] = __ldg(base + 1);
    v[2] = __ldg(base + 8);
    v[3] = __ldg(base + 9);
    v[4] = __ldg(base + 64);
    v[5] = __ldg(base + 65);
    v[6] = __ldg(base + 72);
    v[7] = __ldg(base + 73);
  } else {
    int blk[8];
    corner_blocks(s, c, b0, i, j, k, blk, err);
#pragma unroll
    for (int n = 0; n < 8; ++n)
      v[n] = (blk[n] < 0 || !RELO_CHECK(blk[n] < s.n_blocks))
                 ? 1.0f
                 : __ldg(&s.tsdf[(size_t)blk[n] * kVoxelsPerBlock + corner_voxel(i, j, k, n)]);
  }
  const float x00 = v[0] + fx * (v[1] - v[0]);
  const float x10 = v[2] + fx * (v[3] - v[2]);
  const float x01 = v[4] + fx * (v[5] - v[4]);
  const float x11 = v[6] + fx * (v[7] - v[6]);
  const float y0 = x00 + fy * (x10 - x00);
  const float y1 = x01 + fy * (x11 - x01);
  return y0 + fz * (y1 - y0);
}

// Trilinear colour at point p (corners in unallocated blocks read 0), rounded half up.
__device__ __forceinline__ uint32_t trilinear_rgba(const SceneView& s, BlockCache& c, float3 p, int* err) {
  const float qx = p.x * s.inv_voxel, qy = p.y * s.inv_voxel, qz = p.z * s.inv_voxel;
  const float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
  const int i = (int)flx, j = (int)fly, k = (int)flz;
  const float fx = qx - flx, fy = qy - fly, fz = qz - flz;
  int blk[8];
  corner_blocks(s, c, cached_block(s, c, i >> 3, j >> 3, k >> 3, err), i, j, k, blk, err);
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const int dx = n & 1, dy = (n >> 1) & 1, dz = n >> 2;
    const float w = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy) * (dz ? fz : 1.f - fz);
    const uint32_t col = (blk[n] < 0 || !RELO_CHECK(blk[n] < s.n_blocks))
                             ? 0u
                             : __ldg(&s.rgba[(size_t)blk[n] * kVoxelsPerBlock + corner_voxel(i, j, k, n)]);
    acc[0] += w * (float)(col & 0xFF);
    acc[1] += w * (float)((col >> 8) & 0xFF);
    acc[2] += w * (float)((col >> 16) & 0xFF);
  }
  const uint32_t r = (uint32_t)round_half_up_clamp(acc[0], 0, 255);
  const uint32_t g = (uint32_t)round_half_up_clamp(acc[1], 0, 255);
  const uint32_t b = (uint32_t)round_half_up_clamp(acc[2], 0, 255);
  return r | (g << 8) | (b << 16) | (255u << 24);
}

// One ray.  Returns the hit depth parameter (camera z, metres) or a negative value if none.
template <bool kApron>
__device__ __forceinline__ float march_ray(const SceneView& s, float3 C, float3 d, float dmin, float dmax, BlockCache& c,
                                           int* err) {
  const float dn = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  const float inv_dn = 1.0f / dn;
  const RayExit rx = ray_exit(d);
  float lam = dmin, lam_prev = 0.f, f_prev = 0.f;
  bool have_prev = false;
  for (int it = 0; it < kMaxMarchSamples && lam <= dmax; ++it) {
    const float px = fmaf(lam, d.x, C.x), py = fmaf(lam, d.y, C.y), pz = fmaf(lam, d.z, C.z);
    const float qx = px * s.inv_voxel, qy = py * s.inv_voxel, qz = pz * s.inv_voxel;
    const float flx = floorf(qx), fly = floorf(qy), flz = floorf(qz);
    const int i = (int)flx, j = (int)fly, k = (int)flz;
    const int bx = i >> 3, by = j >> 3, bz = k >> 3;
    const int b = cached_block(s, c, bx, by, bz, err);
    if (b < 0) {
      // free space up to the exit of this block -- or, through the grid, of the cube of blocks
      // around it that holds no allocated block (-b = its Chebyshev distance to one, so the
      // cube's half-size is -b - 1 blocks): stepping block by block through that cube ends on
      // the same exit plane, so the skip changes no sample the march evaluates
      const float lexit = cube_exit(C, rx, bx, by, bz, -b, s.block_size);
      lam_prev = fmaxf(lexit, lam);
      f_prev = 1.0f;
      have_prev = true;
      lam = lam_prev + 1e-5f;
      continue;
    }
    const float f = trilinear_tsdf<kApron>(s, c, b, i, j, k, qx - flx, qy - fly, qz - flz, err);
    if (f <= 0.0f) {
      if (!have_prev) return -1.0f;
      return lam_prev + (lam - lam_prev) * f_prev / (f_prev - f);
    }
    lam_prev = lam;
    f_prev = f;
    have_prev = true;
    lam += fmaxf(f * s.mu, s.voxel) * inv_dn;
  }
  return -1.0f;
}

constexpr int kTile = 16;
// CTAs per SM the compiler must fit, depth-only and colour renders: the march is latency-bound,
// so occupancy beats the few registers this spills.  On the house batch: depth-only 12.08 / 11.94
// / 12.99 ms at 5 / 6 / 7, colour 13.53 / 12.86 / 12.40 / 12.57 ms at 4 / 5 / 6 / 7
#ifndef RELO_RAYCAST_MIN_BLOCKS
#define RELO_RAYCAST_MIN_BLOCKS 6
#endif
#ifndef RELO_RAYCAST_COLOUR_MIN_BLOCKS
#define RELO_RAYCAST_COLOUR_MIN_BLOCKS 6
#endif

template <bool kColour, bool kCompare, bool kApron>
__global__ void __launch_bounds__(kTile* kTile, kColour ? RELO_RAYCAST_COLOUR_MIN_BLOCKS : RELO_RAYCAST_MIN_BLOCKS)
    raycast_kernel(const RayJob* __restrict__ jobs, int n_jobs, const RayJob single, int warp_log2w) {
  // locate the job owning this tile (jobs are few; binary search on tile_begin)
  int lo = 0, hi = n_jobs - 1;
  while (jobs && lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  // the CTA's job, staged in shared memory: the march reads its scene fields at every step; a
  // device pose is converted to float once per CTA (double conversions use the FP64 pipe)
  __shared__ __align__(16) RayJob sj;
  __shared__ float s_pose[12];
  __shared__ unsigned s_counts[4], s_arrived;
  if (jobs) {
    const int4* src = reinterpret_cast<const int4*>(jobs + lo);
    int4* dst = reinterpret_cast<int4*>(&sj);
    for (int i = threadIdx.x; i < (int)(sizeof(RayJob) / 16); i += blockDim.x) dst[i] = src[i];
  } else if (threadIdx.x == 0) {
    sj = single;
  }
  if (threadIdx.x < 12) {
    const double* pd = jobs ? jobs[lo].pose_dev : single.pose_dev;
    if (pd) s_pose[threadIdx.x] = (float)pd[threadIdx.x];
  }
  if (kCompare && threadIdx.x < 4) s_counts[threadIdx.x] = 0u;
  if (kCompare && threadIdx.x == 0) s_arrived = 0u;
  __syncthreads();
  const RayJob& job = sj;
  const int tiles_x = (job.W + kTile - 1) / kTile;
  const int tile = (int)blockIdx.x - job.tile_begin;
  // each warp covers a fw x (32 / fw) footprint of the 16 x 16 tile, fw = 1 << warp_log2w in
  // {2, 4, 8, 16} (neighbouring rays march alike); the warps tile it row by row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fw = 1 << warp_log2w, fh = 32 >> warp_log2w, per_row = kTile >> warp_log2w;
  const int u = (tile % tiles_x) * kTile + (warp % per_row) * fw + (lane & (fw - 1));
  const int v = (tile / tiles_x) * kTile + (warp / per_row) * fh + (lane >> warp_log2w);
  const bool active = u < job.W && v < job.H && (job.status_dev == nullptr || *job.status_dev == RELO_OK);

  int err = 0;
  int depth_mm = 0;
  if (active) {
    float R[9], t[3];
    if (job.pose_dev) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int q = 0; q < 3; ++q) R[3 * r + q] = s_pose[4 * r + q];
        t[r] = s_pose[4 * r + 3];
      }
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) R[q] = job.R[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) t[q] = job.t[q];
    }
    const float dcx = ((float)u - job.cx) / job.fx, dcy = ((float)v - job.cy) / job.fy;
    const float3 d = make_float3(R[0] * dcx + R[1] * dcy + R[2], R[3] * dcx + R[4] * dcy + R[5],
                                 R[6] * dcx + R[7] * dcy + R[8]);
    const float3 C = make_float3(t[0], t[1], t[2]);
    BlockCache cache{INT32_MIN, INT32_MIN, INT32_MIN, -1};
    const float lam = march_ray<kApron>(job.scene, C, d, job.dmin, job.dmax, cache, &err);
    const size_t pix = (size_t)v * job.W + u;
    uint32_t col = 0u;
    if (lam >= job.dmin && lam <= job.dmax) {
      float z_mm = lam * 1000.0f;
      if (job.noise) z_mm += 1.5f * lam * lam * __ldg(&job.noise[pix]);
      depth_mm = round_half_up_clamp(z_mm, 1, 65535);
      if (kColour) col = trilinear_rgba(job.scene, cache, make_float3(fmaf(lam, d.x, C.x), fmaf(lam, d.y, C.y),
                                                                      fmaf(lam, d.z, C.z)), &err);
    }
    if (job.depth) job.depth[pix] = (uint16_t)depth_mm;
    if (kColour && job.rgba) job.rgba[pix] = col;
    if (kColour && job.packed) job.packed[pix] = make_uint2((uint32_t)depth_mm | (col & 0xFFFFu) << 16, (col >> 16) & 0xFFu);
    if (err && job.err) atomicExch(job.err, RELO_EDEVICE);
  }
  if (kCompare) {
    // Sec. 3.3.1: |Omega_a|, |Omega_b|, |Omega_ab| and sum over Omega_ab of |D_a - D_b| (integers)
    unsigned oa = 0, ob = 0, oab = 0, sum = 0;
    if (active) {
      const int db = job.depth_ref[(size_t)v * job.W + u];
      oa = depth_mm > 0;
      ob = db > 0;
      oab = oa & ob;
      sum = oab ? (unsigned)abs(depth_mm - db) : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      oa += __shfl_xor_sync(0xffffffffu, oa, o);
      ob += __shfl_xor_sync(0xffffffffu, ob, o);
      oab += __shfl_xor_sync(0xffffffffu, oab, o);
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    // per-warp totals into shared counters; the last warp to arrive adds the CTA's totals to the
    // job's counters (no CTA-wide barrier: warps whose rays ended early do not wait)
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&s_counts[0], oa);
      atomicAdd(&s_counts[1], ob);
      atomicAdd(&s_counts[2], oab);
      atomicAdd(&s_counts[3], sum);
      __threadfence_block();
      if (atomicAdd(&s_arrived, 1u) == kTile * kTile / 32 - 1 &&
          (job.status_dev == nullptr || *job.status_dev == RELO_OK)) {
        __threadfence_block();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const unsigned acc = atomicAdd(&s_counts[q], 0u);
          if (acc) atomicAdd(&job.counts[q], (unsigned long long)acc);
        }
      }
    }
  }
}

template <bool kApron>
void launch_raycast_t(const RayJob* jobs_dev, int n_jobs, const RayJob& one, int total_tiles, bool with_colour,
                      bool compare, cudaStream_t s, int w) {
  const dim3 grid(total_tiles), block(kTile * kTile);
  if (compare) raycast_kernel<false, true, kApron><<<grid, block, 0, s>>>(jobs_dev, n_jobs, one, w);
  else if (with_colour) raycast_kernel<true, false, kApron><<<grid, block, 0, s>>>(jobs_dev, n_jobs, one, w);
  else raycast_kernel<false, false, kApron><<<grid, block, 0, s>>>(jobs_dev, n_jobs, one, w);
}

cudaError_t launch_raycast(const RayJob* jobs_dev, int n_jobs, const RayJob* single, int total_tiles,
                           bool with_colour, bool compare, cudaStream_t s, const Schedule& sched, bool all_apron) {
  if (total_tiles <= 0) return cudaSuccess;
  if (sched.ray_warp_log2w < 1 || sched.ray_warp_log2w > 4) return cudaErrorInvalidValue;
  RayJob one{};
  if (single) one = *single;
  // a single job's own scene decides; a job array's scenes were checked by the caller
  const bool apron = single ? one.scene.tsdf9 != nullptr : all_apron;
  if (apron) launch_raycast_t<true>(jobs_dev, n_jobs, one, total_tiles, with_colour, compare, s, sched.ray_warp_log2w);
  else launch_raycast_t<false>(jobs_dev, n_jobs, one, total_tiles, with_colour, compare, s, sched.ray_warp_log2w);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Global map rendering (Appendix B.2): each scene raycast from its local pose, the nearest depth
// wins per pixel (ties to the lower scene index) and gives the pixel its colour.  A scene's march
// stops past the depth it would have to beat: any hit nearer than best + 1 mm is detected by a
// sample at most one march step (<= mu) beyond it, so the cut changes no winner.
// ---------------------------------------------------------------------------------------------
template <bool kApron>
__global__ void __launch_bounds__(kTile* kTile)
    render_global_kernel(const RayJob* __restrict__ jobs, int n, uint16_t* __restrict__ depth,
                         uint32_t* __restrict__ rgba, int8_t* __restrict__ owner, int32_t* __restrict__ err_flag) {
  extern __shared__ __align__(16) int4 smem_jobs[];
  RayJob* sj = reinterpret_cast<RayJob*>(smem_jobs);
  {
    const int4* src = reinterpret_cast<const int4*>(jobs);
    for (int i = threadIdx.x; i < n * (int)(sizeof(RayJob) / 16); i += blockDim.x) smem_jobs[i] = src[i];
  }
  __syncthreads();
  const int W = sj[0].W, H = sj[0].H;
  const int tiles_x = (W + kTile - 1) / kTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int u = (blockIdx.x % tiles_x) * kTile + (warp & 1) * 8 + (lane & 7);
  const int v = (blockIdx.x / tiles_x) * kTile + (warp >> 1) * 4 + (lane >> 3);
  if (u >= W || v >= H) return;
  int err = 0, best_mm = 0, best = -1;
  float best_lam = 0.f;
  for (int a = 0; a < n; ++a) {
    const RayJob& j = sj[a];
    const float dcx = ((float)u - j.cx) / j.fx, dcy = ((float)v - j.cy) / j.fy;
    const float3 d = make_float3(j.R[0] * dcx + j.R[1] * dcy + j.R[2], j.R[3] * dcx + j.R[4] * dcy + j.R[5],
                                 j.R[6] * dcx + j.R[7] * dcy + j.R[8]);
    const float3 C = make_float3(j.t[0], j.t[1], j.t[2]);
    const float lim = best >= 0 ? fminf(j.dmax, (float)(best_mm + 1) * 0.001f + j.scene.mu + j.scene.voxel) : j.dmax;
    BlockCache cache{INT32_MIN, INT32_MIN, INT32_MIN, -1};
    const float lam = march_ray<kApron>(j.scene, C, d, j.dmin, lim, cache, &err);
    if (lam >= j.dmin && lam <= j.dmax) {
      const int mm = round_half_up_clamp(lam * 1000.0f, 1, 65535);
      if (best < 0 || mm < best_mm) {
        best_mm = mm;
        best = a;
        best_lam = lam;
      }
    }
  }
  uint32_t col = 0u;
  if (best >= 0 && rgba) {
    const RayJob& j = sj[best];
    const float dcx = ((float)u - j.cx) / j.fx, dcy = ((float)v - j.cy) / j.fy;
    const float3 d = make_float3(j.R[0] * dcx + j.R[1] * dcy + j.R[2], j.R[3] * dcx + j.R[4] * dcy + j.R[5],
                                 j.R[6] * dcx + j.R[7] * dcy + j.R[8]);
    BlockCache cache{INT32_MIN, INT32_MIN, INT32_MIN, -1};
    col = trilinear_rgba(j.scene, cache,
                         make_float3(fmaf(best_lam, d.x, j.t[0]), fmaf(best_lam, d.y, j.t[1]), fmaf(best_lam, d.z, j.t[2])),
                         &err);
  }
  const size_t pix = (size_t)v * W + u;
  depth[pix] = (uint16_t)best_mm;
  if (rgba) rgba[pix] = col;
  if (owner) owner[pix] = (int8_t)best;
  if (err && err_flag) atomicExch(err_flag, RELO_EDEVICE);
}

cudaError_t launch_render_global(const RayJob* jobs_dev, int n, int W, int H, uint16_t* depth, uint32_t* rgba,
                                 int8_t* owner, int32_t* err_flag, cudaStream_t s, bool all_apron) {
  if (n < 1 || W < 1 || H < 1) return cudaSuccess;
  const size_t smem = (size_t)n * sizeof(RayJob);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;
  if (all_apron)
    render_global_kernel<true><<<ray_tiles(W, H), kTile * kTile, smem, s>>>(jobs_dev, n, depth, rgba, owner, err_flag);
  else
    render_global_kernel<false><<<ray_tiles(W, H), kTile * kTile, smem, s>>>(jobs_dev, n, depth, rgba, owner, err_flag);
  return cudaGetLastError();
}

// The apron copy (SceneView::tsdf9): CTA per block, thread per apron voxel.  A voxel on the
// last plane along an axis is the first voxel of the neighbouring block along it (the corner a
// trilinear sample on the block's last voxel reads from that block), +1 where it is unallocated.
__global__ void __launch_bounds__(256) build_apron_kernel(SceneView sv, const int32_t* __restrict__ coords,
                                                          float* __restrict__ out) {
  const int64_t b = blockIdx.x;
  const int bx = coords[3 * b], by = coords[3 * b + 1], bz = coords[3 * b + 2];
  for (int q = threadIdx.x; q < kApronStride; q += blockDim.x) {
    float val = 1.0f;
    if (q < 729) {
      const int x = q % 9, y = (q / 9) % 9, z = q / 81;
      int blk = (int)b, err = 0;
      if (x == 8 || y == 8 || z == 8) blk = lookup_block(sv, bx + (x >> 3), by + (y >> 3), bz + (z >> 3), &err);
      if (blk >= 0 && blk < sv.n_blocks)
        val = sv.tsdf[(size_t)blk * kVoxelsPerBlock + (x & 7) + 8 * (y & 7) + 64 * (z & 7)];
    }
    out[b * kApronStride + q] = val;
  }
}

cudaError_t launch_build_apron(const SceneView& sv, const int32_t* coords_dev, int64_t n, float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > INT32_MAX) return cudaErrorInvalidValue;
  build_apron_kernel<<<(unsigned)n, 256, 0, s>>>(sv, coords_dev, out);
  return cudaGetLastError();
}

__global__ void scene_lookup_kernel(SceneView sv, const int32_t* __restrict__ keys, int64_t n,
                                    int64_t* __restrict__ out, int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int e = 0;
  out[i] = lookup_block(sv, keys[3 * i], keys[3 * i + 1], keys[3 * i + 2], &e);
  if (e && err) atomicExch(err, RELO_EDEVICE);
}

cudaError_t launch_scene_lookup(SceneView sv, const int32_t* keys, int64_t n, int64_t* out, int32_t* err,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  scene_lookup_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(sv, keys, n, out, err);
  return cudaGetLastError();
}

RayJob make_ray_job(const SceneView& sv, const relo_intrinsics& in, const double* pose) {
  RayJob j{};
  j.scene = sv;
  if (pose) {
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) j.R[3 * r + q] = (float)pose[4 * r + q];
      j.t[r] = (float)pose[4 * r + 3];
    }
  }
  j.fx = (float)in.fx;
  j.fy = (float)in.fy;
  j.cx = (float)in.cx;
  j.cy = (float)in.cy;
  j.dmin = (float)in.depth_min;
  j.dmax = (float)in.depth_max;
  j.W = in.width;
  j.H = in.height;
  return j;
}

int ray_tiles(int W, int H) { return ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile); }

RELO_DEFINE_CHECK_READER(check_failures_scene)

}  // namespace relo
