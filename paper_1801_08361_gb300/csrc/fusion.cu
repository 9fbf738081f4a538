// fusion.cu -- TSDF fusion of a depth (+ colour) frame into a growing voxel-block scene: the
// standard volumetric fusion (Curless and Levoy 1996) in the voxel-hashing form of InfiniTAM,
// which the paper runs for each agent's map (Sec. 3.3 (a)) and, with every frame's pose moved by
// its agent's global pose, for the single global model (Appendix B.3).
//
// One frame is four launches on one stream:
//   mark     : thread per pixel: the band |z - d| <= mu around the pixel's depth d is sampled along
//              its ray every quarter block; each sample's block goes into a per-frame set (open
//              addressing on 64-bit keys, atomicCAS);
//   classify : grid-stride over the set: blocks already in the scene go to the frame's visible
//              list, the others to a list of new keys;
//   insert   : grid-stride over the new keys: a block from the pool (atomic counter), inserted in
//              the scene's chained hash without locks (the bucket head claimed by CAS, or an excess
//              entry appended to the chain by CAS), then appended to the visible list;
//   update   : one CTA per visible block (grid-stride), one thread per voxel: project, compare with
//              the depth, running weighted average of the truncated distance and the colour.
// The arithmetic that decides anything (which block a sample falls in, which pixel a voxel sees,
// whether it is in the band) and the averages are float32 with explicit round-to-nearest
// operations in the order the header states, so no multiply-add contraction changes a bit.
// Block indices depend on the order of the atomics; the blocks' coordinates and contents do not.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "relo_internal.cuh"

namespace relo {

namespace {

constexpr unsigned long long kKeyMark = 1ull << 48;  // set in every stored key (0 = empty slot)

__device__ __forceinline__ unsigned long long block_key(int x, int y, int z) {
  return (unsigned long long)(uint16_t)(int16_t)x | ((unsigned long long)(uint16_t)(int16_t)y << 16) |
         ((unsigned long long)(uint16_t)(int16_t)z << 32) | kKeyMark;
}

__device__ __forceinline__ void key_coords(unsigned long long k, int* x, int* y, int* z) {
  *x = (int)(int16_t)(uint16_t)(k & 0xFFFF);
  *y = (int)(int16_t)(uint16_t)((k >> 16) & 0xFFFF);
  *z = (int)(int16_t)(uint16_t)((k >> 32) & 0xFFFF);
}

__device__ __forceinline__ uint32_t key_slot(unsigned long long k) {
  k ^= k >> 29;
  k *= 0xBF58476D1CE4E5B9ull;
  k ^= k >> 32;
  return (uint32_t)k;
}

// Inserts key into the frame's set; the thread that stores it first also appends it to the
// frame's key list.  False if the set is full.
__device__ __forceinline__ bool set_insert(const FuseJob& j, unsigned long long key) {
  uint32_t i = key_slot(key) & j.set_mask;
  for (uint32_t probe = 0; probe <= j.set_mask; ++probe) {
    const unsigned long long prev = atomicCAS(&j.set[i], 0ull, key);
    if (prev == 0ull) {
      j.keys[atomicAdd(j.n_keys, 1)] = key;
      return true;
    }
    if (prev == key) return true;
    i = (i + 1) & j.set_mask;
  }
  return false;
}

__device__ __forceinline__ void set_status(int32_t* status, int code) { atomicCAS(status, RELO_OK, code); }

__global__ void __launch_bounds__(256) fuse_mark_kernel(const FuseJob j) {
  const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= (int64_t)j.W * j.H) return;
  const int u = (int)(pix % j.W), v = (int)(pix / j.W);
  const uint16_t D = j.depth[pix];
  if (D == 0) return;
  const float z = __fmul_rn((float)D, 0.001f);
  if (!(z >= j.dmin && z <= j.dmax)) return;
  const float dcx = __fdiv_rn(__fsub_rn((float)u, j.cx), j.fx), dcy = __fdiv_rn(__fsub_rn((float)v, j.cy), j.fy);
  float dir[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    dir[r] = __fadd_rn(__fadd_rn(__fmul_rn(j.R[3 * r], dcx), __fmul_rn(j.R[3 * r + 1], dcy)), j.R[3 * r + 2]);
  const float bs = __fmul_rn(j.voxel, 8.0f), h = __fmul_rn(bs, 0.25f);
  const float z0 = __fsub_rn(z, j.mu), z1 = __fadd_rn(z, j.mu);
  const int n = (int)ceilf(__fdiv_rn(__fsub_rn(z1, z0), h));
  unsigned long long last = 0ull;
  for (int k = 0; k <= n; ++k) {
    float zk = __fadd_rn(z0, __fmul_rn((float)k, h));
    if (zk > z1) zk = z1;
    if (!(zk > 0.0f)) continue;
    int b[3];
    bool ok = true;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float p = __fadd_rn(j.t[r], __fmul_rn(zk, dir[r]));
      const float q = floorf(__fdiv_rn(p, bs));
      if (!(q >= -32768.0f && q <= 32767.0f)) ok = false;
      b[r] = ok ? (int)q : 0;
    }
    if (!ok) continue;
    const unsigned long long key = block_key(b[0], b[1], b[2]);
    if (key == last) continue;  // consecutive samples in one block: one insertion
    last = key;
    if (!set_insert(j, key)) set_status(j.status, RELO_ENOMEM);
  }
}

// Block index of (x, y, z) in the scene's hash, -1 if absent (the walk is bounded by the pool).
__device__ __forceinline__ int find_block(const FuseJob& j, int x, int y, int z) {
  const int4 want = pack_entry(x, y, z, 0, 0);
  int4 e = j.buckets[block_hash(x, y, z) & j.bucket_mask];
  for (int steps = 0; steps <= j.capacity; ++steps) {
    if (e.z >= 0 && e.x == want.x && (e.y & 0xFFFF) == (want.y & 0xFFFF)) return e.z;
    if (e.w < 0) return -1;
    e = j.excess[e.w];
  }
  return -1;
}

__global__ void __launch_bounds__(256) fuse_classify_kernel(const FuseJob j) {
  const int n_keys = *j.n_keys;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_keys; i += gridDim.x * blockDim.x) {
    const unsigned long long key = j.keys[i];
    int x, y, z;
    key_coords(key, &x, &y, &z);
    const int b = find_block(j, x, y, z);
    if (b >= 0) j.visible[atomicAdd(j.n_visible, 1)] = b;
    else j.new_keys[atomicAdd(j.n_new, 1)] = key;
  }
}

__global__ void __launch_bounds__(256) fuse_insert_kernel(const FuseJob j) {
  const int n_new = *j.n_new;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_new; i += gridDim.x * blockDim.x) {
    int x, y, z;
    key_coords(j.new_keys[i], &x, &y, &z);
    const int b = atomicAdd(&j.counters[0], 1);
    if (b >= j.capacity) {
      set_status(j.status, RELO_ENOMEM);
      continue;
    }
    j.coords[b] = make_int4(x, y, z, 0);
    const int4 entry = pack_entry(x, y, z, b, -1);
    int4* head = &j.buckets[block_hash(x, y, z) & j.bucket_mask];
    if (atomicCAS(&head->z, -1, b) == -1) {
      // the bucket's head entry is ours: its key words (read by later launches only)
      head->x = entry.x;
      head->y = entry.y;
    } else {
      const int e = atomicAdd(&j.counters[1], 1);
      if (e >= j.capacity) {
        set_status(j.status, RELO_ENOMEM);
        continue;
      }
      j.excess[e] = entry;
      __threadfence();  // the entry is complete before the chain links to it
      int* link = &head->w;
      for (int steps = 0; steps <= j.capacity; ++steps) {
        const int prev = atomicCAS(link, -1, e);
        if (prev == -1) break;
        link = &j.excess[prev].w;
      }
    }
    j.visible[atomicAdd(j.n_visible, 1)] = b;
  }
}

__global__ void __launch_bounds__(512) fuse_update_kernel(const FuseJob j) {
  const int n_vis = *j.n_visible;
  const int vi = threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(j.updates, (unsigned long long)n_vis);
  for (int q = blockIdx.x; q < n_vis; q += gridDim.x) {
    const int b = j.visible[q];
    if (!RELO_CHECK(b >= 0 && b < j.capacity)) continue;
    const int4 bc = j.coords[b];
    const int X = 8 * bc.x + (vi & 7), Y = 8 * bc.y + ((vi >> 3) & 7), Z = 8 * bc.z + (vi >> 6);
    const float dx = __fsub_rn(__fmul_rn((float)X, j.voxel), j.t[0]);
    const float dy = __fsub_rn(__fmul_rn((float)Y, j.voxel), j.t[1]);
    const float dz = __fsub_rn(__fmul_rn((float)Z, j.voxel), j.t[2]);
    const float qx = __fadd_rn(__fadd_rn(__fmul_rn(j.R[0], dx), __fmul_rn(j.R[3], dy)), __fmul_rn(j.R[6], dz));
    const float qy = __fadd_rn(__fadd_rn(__fmul_rn(j.R[1], dx), __fmul_rn(j.R[4], dy)), __fmul_rn(j.R[7], dz));
    const float qz = __fadd_rn(__fadd_rn(__fmul_rn(j.R[2], dx), __fmul_rn(j.R[5], dy)), __fmul_rn(j.R[8], dz));
    if (!(qz > 0.0f)) continue;
    const float uf = __fadd_rn(__fmul_rn(j.fx, __fdiv_rn(qx, qz)), j.cx);
    const float vf = __fadd_rn(__fmul_rn(j.fy, __fdiv_rn(qy, qz)), j.cy);
    const float fu = floorf(__fadd_rn(uf, 0.5f)), fv = floorf(__fadd_rn(vf, 0.5f));
    if (!(fu >= 0.0f && fu < (float)j.W && fv >= 0.0f && fv < (float)j.H)) continue;
    const int pix = (int)fv * j.W + (int)fu;  // 32-bit: 64-bit float conversions run on the FP64 pipe
    if (!RELO_CHECK(pix >= 0 && pix < j.W * j.H)) continue;
    const uint16_t Dm = j.depth[pix];
    if (Dm == 0) continue;
    const float dm = __fmul_rn((float)Dm, 0.001f);
    if (!(dm >= j.dmin && dm <= j.dmax)) continue;
    const float eta = __fsub_rn(dm, qz);
    if (eta < -j.mu) continue;
    const float fn = fminf(1.0f, __fdiv_rn(eta, j.mu));
    const int64_t at = (int64_t)b * kVoxelsPerBlock + vi;
    const uint16_t w0 = j.weight[at];
    const float w = (float)w0, w1 = __fadd_rn(w, 1.0f);
    j.tsdf[at] = __fdiv_rn(__fadd_rn(__fmul_rn(j.tsdf[at], w), fn), w1);
    if (j.frame_rgba) {
      const uint32_t old = j.rgba[at], px = j.frame_rgba[pix];
      uint32_t out = 255u << 24;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float cc = __fdiv_rn(__fadd_rn(__fmul_rn((float)((old >> (8 * c)) & 0xFF), w),
                                             (float)((px >> (8 * c)) & 0xFF)), w1);
        const float r = fminf(255.0f, fmaxf(0.0f, floorf(__fadd_rn(cc, 0.5f))));
        out |= (uint32_t)r << (8 * c);
      }
      j.rgba[at] = out;
    }
    j.weight[at] = (uint16_t)min((int)w0 + 1, j.max_weight);
  }
}

__global__ void fuse_init_kernel(float* tsdf, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    tsdf[i] = 1.0f;
}

int grid_for(int64_t work, int threads) {
  int sms = 0;
  if (device_sms(&sms) != cudaSuccess) sms = 152;
  const int64_t want = (work + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
}

}  // namespace

cudaError_t launch_fuse_init(float* tsdf, int64_t n, cudaStream_t s) {
  fuse_init_kernel<<<grid_for(n, 256), 256, 0, s>>>(tsdf, n);
  return cudaGetLastError();
}

cudaError_t launch_fuse_frame(const FuseJob& j, cudaStream_t s) {
  const int64_t n_pix = (int64_t)j.W * j.H;
  cudaError_t e = cudaMemsetAsync(j.set, 0, ((size_t)j.set_mask + 1) * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(j.n_visible, 0, 3 * sizeof(int32_t), s);  // n_visible, n_new, n_keys
  if (e != cudaSuccess) return e;
  fuse_mark_kernel<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(j);
  fuse_classify_kernel<<<grid_for((int64_t)j.set_mask + 1, 256), 256, 0, s>>>(j);
  fuse_insert_kernel<<<grid_for((int64_t)j.set_mask + 1, 256), 256, 0, s>>>(j);
  fuse_update_kernel<<<grid_for((int64_t)(j.set_mask + 1) * 512, 512) , 512, 0, s>>>(j);
  return cudaGetLastError();
}

RELO_DEFINE_CHECK_READER(check_failures_fusion)

}  // namespace relo
