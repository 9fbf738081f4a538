// relo_internal.cuh -- device data layouts and helpers shared by the library's translation units.
//
// Everything here belongs to the CUDA path; nothing is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/relo.h"

namespace relo {

// ---------------------------------------------------------------------------------------------
// A launch parameter that depends only on the device (its SM count, a kernel's resident CTAs per
// SM): computed once per device ordinal, with that device current, and shared by every host
// thread.  The lock makes a value and its "ready" mark appear together, so no thread launches
// with a half-published pair.
// ---------------------------------------------------------------------------------------------
struct PerDevice {
  static constexpr int kMaxDevices = 64;
  std::mutex m;
  int value[kMaxDevices] = {};
  bool ready[kMaxDevices] = {};
};

template <class F>
cudaError_t per_device(PerDevice& c, int* out, F&& compute) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= PerDevice::kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(c.m);
  if (!c.ready[dev]) {
    int v = 0;
    e = compute(dev, &v);
    if (e != cudaSuccess) return e;
    c.value[dev] = v;
    c.ready[dev] = true;
  }
  *out = c.value[dev];
  return cudaSuccess;
}

// SMs of the current device.
inline cudaError_t device_sms(int* out) {
  static PerDevice cache;
  return per_device(cache, out, [](int dev, int* v) {
    return cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
  });
}

constexpr int kBlockSide = 8;
constexpr int kVoxelsPerBlock = 512;
constexpr int kMaxTrees = 16;
constexpr int kModeFloats = 12;
constexpr float kLogEps = 69.07755278982137f;  // -log(1e-30): energy of a pixel no mode explains
constexpr int kMaxMarchSamples = 100000;

// ---------------------------------------------------------------------------------------------
// Spatial hash of a voxel scene.  Entry = 16 bytes {int16 x, y, z, pad; int32 block; int32 next},
// loaded as one int4.  Bucket h holds the first block hashing to h; later ones are chained
// through the excess list (next = index into it, -1 ends the chain).
// ---------------------------------------------------------------------------------------------
struct SceneView {
  const int4* buckets;
  const int4* excess;
  const float* tsdf;      // [n_blocks][512]
  const uint32_t* rgba;   // [n_blocks][512] packed r | g << 8 | b << 16 | a << 24
  uint32_t mask;          // n_buckets - 1
  int32_t n_blocks;
  int32_t max_chain;      // longest chain at build time (bounds the walk)
  float voxel, inv_voxel, mu, block_size, inv_block;
  // Dense grid over the blocks' bounding box (null when the box is too large): per block
  // coordinate the block index, or -D for an unallocated block whose nearest allocated block is
  // D >= 1 blocks away in the Chebyshev metric (every block within D - 1 of it is unallocated).
  const int32_t* grid;
  int32_t ox, oy, oz;     // grid origin (block coordinates)
  int32_t gx, gy, gz;     // grid extent in blocks (multiples of 8)
  // Apron copy of the tsdf (null when not built or not in use): per block a 9 x 9 x 9 array
  // (x + 9 y + 81 z, padded to kApronStride floats) whose last plane along each axis repeats the
  // first voxels of the neighbouring block (+1 where that block is unallocated), so the eight
  // corners of every trilinear sample lie in the block holding the sample.
  const float* tsdf9;
  int32_t pad[2];
};
constexpr int kApronStride = 736;  // 729 voxels padded to a multiple of 32 floats (128 bytes)

// Block index, or -D (see SceneView::grid), through the dense grid (caller checks s.grid).
// Outside the box D is the Chebyshev distance to the box, a lower bound of the distance to any
// allocated block.
__device__ __forceinline__ int grid_block(const SceneView& s, int x, int y, int z) {
  const int a = x - s.ox, b = y - s.oy, c = z - s.oz;
  if ((unsigned)a >= (unsigned)s.gx || (unsigned)b >= (unsigned)s.gy || (unsigned)c >= (unsigned)s.gz) {
    const int da = a < 0 ? -a : a - (s.gx - 1);
    const int db = b < 0 ? -b : b - (s.gy - 1);
    const int dc = c < 0 ? -c : c - (s.gz - 1);
    return -max(da, max(db, dc));
  }
  return __ldg(&s.grid[((size_t)c * s.gy + b) * s.gx + a]);
}

__host__ __device__ inline uint32_t block_hash(int x, int y, int z) {
  return ((uint32_t)x * 73856093u) ^ ((uint32_t)y * 19349669u) ^ ((uint32_t)z * 83492791u);
}

__host__ __device__ inline int4 pack_entry(int x, int y, int z, int block, int next) {
  int4 e;
  e.x = (int)((uint32_t)(uint16_t)(int16_t)x | ((uint32_t)(uint16_t)(int16_t)y << 16));
  e.y = (int)((uint32_t)(uint16_t)(int16_t)z);
  e.z = block;
  e.w = next;
  return e;
}

// Block index of block coordinate (x, y, z), -1 if absent; *err set if the chain walk exceeds
// its bound (a corrupted table).
__device__ __forceinline__ int lookup_block(const SceneView& s, int x, int y, int z, int* err) {
  if (x < -32768 || x > 32767 || y < -32768 || y > 32767 || z < -32768 || z > 32767) return -1;
  const int k0 = (int)((uint32_t)(uint16_t)(int16_t)x | ((uint32_t)(uint16_t)(int16_t)y << 16));
  const int k1 = (int)((uint32_t)(uint16_t)(int16_t)z);
  int4 e = __ldg(&s.buckets[block_hash(x, y, z) & s.mask]);
  for (int steps = 0; steps <= s.max_chain; ++steps) {
    if (e.z >= 0 && e.x == k0 && (e.y & 0xFFFF) == k1) return e.z;
    if (e.w < 0) return -1;
    e = __ldg(&s.excess[e.w]);
  }
  *err = 1;
  return -1;
}

// ---------------------------------------------------------------------------------------------
// Forest
// ---------------------------------------------------------------------------------------------
struct ForestView {
  const int4* nodes;        // [T][2^D - 1] split nodes, 16 bytes each
  const float* modes;       // [T][2^D][M][12]
  const uint8_t* n_modes;   // [T][2^D]
  const float4* top;        // [T][2^D]: mode 0 mean xyz, w = number of modes
  int32_t T, D, M;
  int32_t probe_reach;      // 1 + the largest |offset| of any node (0: not known, every probe clamped)
  int32_t offset_shift;     // the device nodes hold offset << offset_shift (7 when every |offset| <= 255, else 0)
};

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): 10 rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85.
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ inline uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ inline uint32_t uniform_below(uint32_t x, uint32_t n) { return mulhi32(x, n); }

// ---------------------------------------------------------------------------------------------
// Poses: 12 doubles, row-major [R | t], camera -> scene.
// ---------------------------------------------------------------------------------------------
struct PoseF {
  float r[9], t[3];
};

__device__ __forceinline__ PoseF pose_to_float(const double* p) {
  PoseF q;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) q.r[3 * i + j] = (float)p[4 * i + j];
    q.t[i] = (float)p[4 * i + 3];
  }
  return q;
}

__device__ __forceinline__ float3 apply(const PoseF& P, float3 c) {
  return make_float3(fmaf(P.r[0], c.x, fmaf(P.r[1], c.y, fmaf(P.r[2], c.z, P.t[0]))),
                     fmaf(P.r[3], c.x, fmaf(P.r[4], c.y, fmaf(P.r[5], c.z, P.t[1]))),
                     fmaf(P.r[6], c.x, fmaf(P.r[7], c.y, fmaf(P.r[8], c.z, P.t[2]))));
}

// Rigid transform from centroids and cross-covariance by Horn's closed form (1987): the rotation is
// the unit quaternion of the largest eigenvalue of the symmetric 4x4 matrix N(S), S = sum of
// (c - cbar)(w - wbar)^T.  The eigenproblem is solved by cyclic Jacobi rotations in FP64, which
// keeps the decomposition stable for near-degenerate point sets.  Writes 12 doubles [R | t].
__device__ inline void horn_pose(const double S[9], const double cbar[3], const double wbar[3], double* out) {
  const double Sxx = S[0], Sxy = S[1], Sxz = S[2], Syx = S[3], Syy = S[4], Syz = S[5], Szx = S[6], Szy = S[7],
               Szz = S[8];
  double A[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                    {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                    {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                    {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
  double V[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  // Cyclic Jacobi in the parallel ordering: each sweep is three stages of two rotations on
  // disjoint index pairs, ((0,1),(2,3)), ((0,2),(1,3)), ((0,3),(1,2)), whose angles are computed
  // independently (two divide / square-root chains in flight instead of one).  Every index is a
  // compile-time constant after unrolling, so A and V stay in registers.
  constexpr int kPairs[3][2][2] = {{{0, 1}, {2, 3}}, {{0, 2}, {1, 3}}, {{0, 3}, {1, 2}}};
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, diag = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      diag += A[p][p] * A[p][p];
#pragma unroll
      for (int q = p + 1; q < 4; ++q) off += A[p][q] * A[p][q];
    }
    if (off <= 1e-30 * (diag + 1e-300)) break;
#pragma unroll
    for (int st = 0; st < 3; ++st) {
      double cs[2], sn[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int p = kPairs[st][r][0], q = kPairs[st][r][1];
        const double apq = A[p][q];
        cs[r] = 1.0;
        sn[r] = 0.0;
        if (fabs(apq) >= 1e-300) {
          const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
          const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          cs[r] = rsqrt(t * t + 1.0);
          sn[r] = t * cs[r];
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int p = kPairs[st][r][0], q = kPairs[st][r][1];
        const double c = cs[r], s = sn[r];
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // A <- J^T A J
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - s * akq;
          A[k][q] = s * akp + c * akq;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - s * aqk;
          A[q][k] = s * apk + c * aqk;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
    }
  }
  double best_d = A[0][0], w = V[0][0], x = V[1][0], y = V[2][0], z = V[3][0];
#pragma unroll
  for (int k = 1; k < 4; ++k)
    if (A[k][k] > best_d) {
      best_d = A[k][k];
      w = V[0][k];
      x = V[1][k];
      y = V[2][k];
      z = V[3][k];
    }
  const double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                       2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 3; ++i) {
    out[4 * i + 0] = R[3 * i + 0];
    out[4 * i + 1] = R[3 * i + 1];
    out[4 * i + 2] = R[3 * i + 2];
    out[4 * i + 3] = wbar[i] - (R[3 * i] * cbar[0] + R[3 * i + 1] * cbar[1] + R[3 * i + 2] * cbar[2]);
  }
}

// Warp-wide sum (all lanes get the result).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Round half up of a non-negative float to an integer in [lo, hi].
__device__ __forceinline__ int round_half_up_clamp(float x, int lo, int hi) {
  float r = floorf(x + 0.5f);
  r = fminf(fmaxf(r, (float)lo), (float)hi);
  return (int)r;
}

// ---------------------------------------------------------------------------------------------
// Raycast jobs (query renders, training renders, verification renders)
// ---------------------------------------------------------------------------------------------
struct RayJob {
  SceneView scene;
  float R[9], t[3];            // camera -> scene (ignored when pose_dev is set)
  const double* pose_dev;      // device pose (12 doubles, row-major R | t) overriding R, t
  const int32_t* status_dev;   // when set, the job is skipped unless *status_dev == RELO_OK
  float fx, fy, cx, cy, dmin, dmax;
  int32_t W, H;
  const float* noise;          // nullable
  uint16_t* depth;             // nullable in compare mode
  uint32_t* rgba;              // nullable
  const uint16_t* depth_ref;   // compare mode: reference depth (D_b)
  unsigned long long* counts;  // compare mode: {omega_a, omega_b, omega_ab, sum |D_a - D_b|}
  int32_t* err;                // device error flag (nullable)
  uint2* packed;               // nullable, colour renders: {depth | r << 16 | g << 24, b} per pixel
  int32_t tile_begin;          // first 16 x 16 tile of this job in the flattened launch
  int32_t pad;                 // size: a multiple of 16 bytes (staged in shared memory)
};
static_assert(sizeof(RayJob) % 16 == 0, "RayJob is staged in shared memory as 16-byte words");

// ---------------------------------------------------------------------------------------------
// Forest jobs (one image through one forest)
// ---------------------------------------------------------------------------------------------
struct ForestJob {
  ForestView forest;
  const uint16_t* depth;
  const uint32_t* rgba;
  const uint2* packed;         // nullable: the same image packed per pixel (see RayJob::packed)
  uint16_t* leaves;            // [T][H][W]
  int32_t W, H;
  int64_t pixel_begin;         // first pixel of this job in the flattened launch (multiple of 256)
  const int32_t* skip;         // when set and non-zero the job does nothing (fallback not needed)
};
static_assert(sizeof(ForestJob) % 8 == 0, "ForestJob is staged in shared memory as 8-byte words");

// ---------------------------------------------------------------------------------------------
// RANSAC jobs (one query view, one forest) and their workspace
// ---------------------------------------------------------------------------------------------
struct RansacJob {
  ForestView forest;
  const uint16_t* depth;
  const uint16_t* leaves;      // [T][H][W]
  int32_t W, H;
  double fx, fy, cx, cy;       // FP64 intrinsics: exact re-checks match the oracle bit for bit
  int32_t K, B, max_tries, n_rounds;
  double rigidity, min_area, inlier_dist;
  uint32_t key0, key1;
  // workspace
  uint4* table;                // [W*H][nv] valid pixels in raster order, packed u16 {u, v, depth, leaf[T]}
  int32_t nv;                  // uint4 words per table entry: ceil((3 + T) / 8)
  int32_t pad1;
  int32_t* chunk_count;        // [n_chunks]
  int32_t* n_valid;            // [1]
  double* poses;               // [K][12]
  int32_t* hyp_ok;             // [K]
  int32_t* tries;              // [K]
  double* energy;              // [K]
  int32_t* alive_a;            // [K]
  int32_t* alive_b;            // [K]
  int32_t* drawn;              // [n_rounds * B] positions in the valid-pixel table
  int32_t* inliers;            // [K]
  float2* refit;               // [K][refit_parts][16] per-survivor inlier sums as compensated (high,
                               // low) FP32 pairs, one block per part of kRefinePixels drawn pixels
                               // (summed in order by the FP64 re-fit)
  float* refit_ref;            // [K][8] reference correspondence of those sums: c_ref (3), w_ref (3)
  int4* pix;                   // [n_rounds * B][hs] drawn pixels: camera point (FP32 bits), then
                               // (first mode, mode count) of the pixel's leaf in each tree, two per word
  int32_t hs;                  // int4 words per drawn-pixel record: 1 + ceil(T / 2)
  int32_t refit_parts;         // blocks per hypothesis in refit: ceil(n_rounds * B / kRefinePixels)
  int32_t* err;                // [1]
  const int32_t* upstream;     // nullable: status of the stage that made this job's input (the
                               // learned path's network); when nonzero it becomes the result's status
  relo_pose_result* result;    // device
  int32_t chunk_begin;         // flattened compaction chunks
  int32_t hyp_begin;           // flattened hypotheses
  int32_t has_pose_b;          // finalise also writes a_T_b = P_a P_b^-1
  int32_t vW, vH;              // size of the view the pose is verified on (the full image)
  int32_t pad2;
  double pose_b[16];           // camera -> scene b pose of the query
  const int32_t* skip;         // when set and non-zero every stage skips the job (fallback not needed)
};

__device__ __forceinline__ bool job_skipped(const int32_t* skip) { return skip != nullptr && *skip != 0; }

constexpr int kCompactChunk = 4096;
constexpr int kRefinePixels = 64;  // drawn pixels per part of the re-fit sums

// Workspace carving helper (256-byte aligned sub-buffers).
struct Carver {
  char* base;
  size_t off;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// ---------------------------------------------------------------------------------------------
// Launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
// Launch schedule of a batch's kernels (relo_schedule): work-to-thread mappings and grid sizes
// only, so every schedule computes the same results.
struct Schedule {
  int ray_warp_log2w = 3;    // raycast: each warp covers a (1 << w) x (32 >> w) footprint of its 16 x 16 tile
  int forest_threads = 256;  // forest: CTA size (128 or 256)
  int forest_tiles = 0;      // forest: 0 = each CTA takes consecutive pixels, 1 = 32 x 8 pixel tiles
  int forest_smem_levels = 0;  // forest: top levels of the trees each CTA copies to shared memory (0: none)
  int search_ctas_per_sm = 0;  // hypothesis search: persistent CTAs per SM (0: occupancy maximum)
  int refit_per = 0;         // re-fit: survivors per one-warp CTA (0: spread over twice the SM count)
  int persistent = 0;        // RANSAC of a batch: 0 = one launch per stage, 1 = one persistent launch
};
constexpr int kMaxSmemLevels = 10;
// Forest slots a job of W x H pixels takes (a multiple of 256 that also holds its 32 x 8 tiles).
inline int64_t forest_slots(int W, int H) {
  const int64_t rows = ((int64_t)W * H + 255) / 256 * 256;
  const int64_t tiles = (int64_t)((W + 31) / 32) * ((H + 7) / 8) * 256;
  return rows > tiles ? rows : tiles;
}

// jobs_dev == nullptr: the single job is passed by value.  all_apron: every job of jobs_dev has
// its scene's apron copy (SceneView::tsdf9), so the launch samples it (a single job's own scene
// decides for itself).
cudaError_t launch_raycast(const RayJob* jobs_dev, int n_jobs, const RayJob* single, int total_tiles,
                           bool with_colour, bool compare, cudaStream_t s, const Schedule& sched = Schedule(),
                           bool all_apron = false);
// max_trees: the largest tree count among the jobs (selects the kernel's unrolled width).  With
// sched.forest_tiles, each job must own forest_slots(W, H) slots from its pixel_begin.
cudaError_t launch_forest(const ForestJob* jobs_dev, int n_jobs, const ForestJob* single, int64_t total_pixels,
                          cudaStream_t s, int max_trees, const Schedule& sched = Schedule());
int ray_tiles(int W, int H);
// Global map rendering over n scene jobs sharing one image size (owner, rgba, err_flag nullable).
cudaError_t launch_render_global(const RayJob* jobs_dev, int n, int W, int H, uint16_t* depth, uint32_t* rgba,
                                 int8_t* owner, int32_t* err_flag, cudaStream_t s, bool all_apron);
cudaError_t launch_verify_decide(const RansacJob* jobs, int n_jobs, cudaStream_t s);
cudaError_t launch_verify_decide_one(relo_pose_result* res, uint64_t omega, cudaStream_t s);
// Learned batches: mark fallback results not run, then pick each attempt's final result.
cudaError_t launch_init_results(relo_pose_result* res, int n, cudaStream_t s);
cudaError_t launch_merge_results(const relo_pose_result* learned, const relo_pose_result* fallback,
                                 const int32_t* kind, int n, relo_pose_result* out, cudaStream_t s);
// Builds SceneView::tsdf9 for n blocks with coordinates coords_dev (n x int32 xyz) from the
// scene's tsdf and hash table.
cudaError_t launch_build_apron(const SceneView& sv, const int32_t* coords_dev, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_scene_lookup(SceneView sv, const int32_t* keys, int64_t n, int64_t* out, int32_t* err,
                                cudaStream_t s);

// RANSAC stages over a device array of jobs.
inline int table_words(int T) { return (3 + T + 7) / 8; }
cudaError_t launch_compact(const RansacJob* jobs, int n_jobs, int total_chunks, cudaStream_t s);
// counter_dev: one int of device scratch the search's warps take hypotheses from (zeroed here)
cudaError_t launch_hypotheses(const RansacJob* jobs, int n_jobs, int total_hyps, int32_t* counter_dev, cudaStream_t s,
                              const Schedule& sched = Schedule());
// round r: prefix[n_jobs + 1] = flattened alive-hypothesis offsets of the jobs still running
cudaError_t launch_round(const RansacJob* jobs, int n_jobs, int round, const int32_t* alive_prefix_dev,
                         int total_alive, int max_alive, const int32_t* surv_prefix_dev, int total_surv, int max_surv,
                         int B, cudaStream_t s, const Schedule& sched = Schedule());
cudaError_t launch_finalise(const RansacJob* jobs, int n_jobs, cudaStream_t s);

// One persistent launch for a pass's search, fit, rounds and finalise (ransac.cu): items in
// dependency order, per-(stage, job) completion counters, bounded waits.
enum PItemKind { kItemFit = 0, kItemDraw, kItemEnergy, kItemSelect, kItemRefine, kItemRefit, kItemFinal };
constexpr int kPersistThreadsHost = 256;  // threads of a persistent CTA (fit and re-fit chunk sizes)
struct PItem {
  int32_t kind, job, sub, part, round;
  int32_t dep, need;  // wait until done[dep] >= need
  int32_t done;       // then add one to done[done]
};
struct PersistArgs {
  const RansacJob* jobs;
  int n_jobs, total_hyps;
  int32_t* ctrl;                  // [0] search counter, [1] item counter, [2] abort flag
  const PItem* items;
  int n_items;
  int32_t* done;                  // completion counters; done[j] = job j's searched hypotheses
  int final_base;                 // done[final_base + j] = job j finalised
  const int32_t* alive_prefix;    // [rounds][n_jobs + 1], as launch_round
  const int32_t* surv_prefix;
  unsigned long long timeout_ns;
};
// ctrl_words: words zeroed from ctrl (ctrl[0..2] and the done counters that follow them)
cudaError_t launch_persistent(const PersistArgs& a, int ctrl_words, cudaStream_t s);
cudaError_t persistent_grid(int* grid);


// Training
cudaError_t launch_scene_coords(const uint16_t* depth, int W, int H, int stride, double fx, double fy, double cx,
                                double cy, const double* P /*16 host values passed by value*/, float* out,
                                cudaStream_t s);
cudaError_t launch_mean_shift(const float* samples, const int32_t* count, int capacity, int n_leaves_total,
                              float bandwidth, float tol, int max_iter, float merge_dist, float cov_floor,
                              int max_modes, float* modes, uint8_t* n_modes, cudaStream_t s);
cudaError_t launch_top_modes(const float* modes, const uint8_t* n_modes, int n_leaves_total, int max_modes,
                             float4* top, cudaStream_t s);

// Helpers for ray jobs
RayJob make_ray_job(const SceneView& sv, const relo_intrinsics& in, const double* pose_host);

// Checked builds (built with RELO_CHECKED=1): guarded accesses first check their index; a failed
// check is counted, once per translation unit, and the access is skipped.  The stand-in for a
// device memory checker.  In normal builds a check is the constant true and costs nothing.
#ifdef RELO_CHECKED
static __device__ unsigned int g_check_failures;
#define RELO_CHECK(cond) ((cond) ? true : (atomicAdd(&g_check_failures, 1u), false))
#define RELO_DEFINE_CHECK_READER(name)                                    \
  unsigned long long name() {                                             \
    unsigned int v = 0;                                                   \
    if (cudaMemcpyFromSymbol(&v, g_check_failures, sizeof v) != cudaSuccess) return ~0ull; \
    return v;                                                             \
  }
#else
#define RELO_CHECK(cond) true
#define RELO_DEFINE_CHECK_READER(name) \
  unsigned long long name() { return 0; }
#endif
unsigned long long check_failures_scene();
unsigned long long check_failures_forest();
unsigned long long check_failures_ransac();
unsigned long long check_failures_fusion();

// Every device allocation of the library goes through here: from cudaMalloc, or from the
// caller's allocator (relo_set_allocator); tests can make the next allocations fail
// (relo_debug_fail_allocations) and check the error paths.  dev_free returns a block to
// whichever of the two gave it (null is ignored).
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);

// TSDF fusion of one frame into a growing scene (fusion.cu).
struct FuseJob {
  int4* buckets;
  int4* excess;
  float* tsdf;
  uint32_t* rgba;
  uint16_t* weight;
  int4* coords;                 // [capacity] block coordinates (w unused)
  int32_t* counters;            // [0] blocks in use, [1] excess entries in use
  int32_t* status;              // RELO_OK, or RELO_ENOMEM once the pool, the chain or the set ran out
  uint32_t bucket_mask;
  int32_t capacity, max_weight;
  const uint16_t* depth;        // frame [H][W] mm
  const uint32_t* frame_rgba;   // frame [H][W] or null
  int32_t W, H;
  float fx, fy, cx, cy, dmin, dmax;
  float R[9], t[3];             // camera -> scene
  float voxel, mu;
  unsigned long long* set;      // per-frame block set, set_mask + 1 slots
  uint32_t set_mask;
  unsigned long long* new_keys; // set_mask + 1
  unsigned long long* keys;     // set_mask + 1: the frame's distinct block keys, in insertion order
  int32_t* visible;             // set_mask + 1 block indices
  int32_t* n_visible;           // n_visible[0], then n_new, then n_keys
  int32_t* n_new;
  int32_t* n_keys;
  unsigned long long* updates;  // the scene's running count of block updates
};
cudaError_t launch_fuse_frame(const FuseJob& j, cudaStream_t s);
cudaError_t launch_fuse_init(float* tsdf, int64_t n, cudaStream_t s);

}  // namespace relo

// Opaque handles (C ABI)
struct relo_scene {
  relo::SceneView view;
  void* d_buckets;
  void* d_excess;
  void* d_tsdf;
  void* d_rgba;
  void* d_grid;
  void* d_tsdf9;       // apron copy of the tsdf (SceneView::tsdf9), static scenes only
  int64_t n_blocks;
  // scenes that grow by fusion (relo_create_fusion_scene): capacity > 0
  int64_t capacity;
  void* d_weight;      // uint16 [capacity][512]
  void* d_coords;      // int4 [capacity]
  void* d_counters;    // int32 [4]: blocks in use, excess entries in use, status, pad; then uint64 block updates
  int32_t max_weight;
  int64_t n_excess;    // excess entries allocated (the chains' storage)
};

struct relo_forest {
  relo::ForestView view;
  void* d_nodes;
  void* d_modes;
  void* d_n_modes;
  void* d_top;
  int32_t T, D, M;
  // training state (host)
  relo_train_params train;
  bool training;
  float* res_samples;   // [T][L][cap][3]
  int32_t* res_count;   // [T][L]
  int64_t* res_seen;    // [T][L]
};
