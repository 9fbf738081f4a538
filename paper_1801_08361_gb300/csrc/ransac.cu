// ransac.cu -- preemptive RANSAC over forest correspondences (the relocaliser's pose solver,
// after Cavallari et al. as used in Sec. 3.3.1; every rule is a stated reading, see relo.h).
//
// Stages, each one launch over all jobs of a batch:
//   compact   : ordered list of valid pixels (two passes: chunk counts, then scatter);
//   hypotheses: one CTA per hypothesis evaluates 256 tries at a time and keeps the first passing
//               try (so the result equals a sequential scan of the tries); the 3-point Kabsch fit
//               runs in FP64 (Horn's quaternion form);
//   per round : draw B pixels; energies (warp per hypothesis, lanes over pixels, FP32 with an FP64
//               running total); halving (CTA per job, bitonic sort of (energy, index)); re-fit
//               (warp per survivor: FP32 centroids and cross-covariance reduced with shuffles,
//               FP64 rotation).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cfloat>
#include <climits>

#include "relo_internal.cuh"

namespace relo {

__device__ __forceinline__ int find_job_by(const int32_t* prefix, int n_jobs, int gid) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= gid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------------
// Valid-pixel compaction
// ---------------------------------------------------------------------------------------------
constexpr int kCompactThreads = 256;
constexpr int kPerThread = kCompactChunk / kCompactThreads;  // 16

__device__ __forceinline__ int chunk_job(const RansacJob* jobs, int n_jobs, int gid) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].chunk_begin <= gid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kCompactThreads) compact_count_kernel(const RansacJob* __restrict__ jobs,
                                                                       int n_jobs) {
  const RansacJob& job = jobs[chunk_job(jobs, n_jobs, blockIdx.x)];
  const int chunk = blockIdx.x - job.chunk_begin;
  const int n_pix = job.W * job.H;
  const int base = chunk * kCompactChunk + threadIdx.x * kPerThread;
  int c = 0;
  for (int k = 0; k < kPerThread; ++k) {
    const int p = base + k;
    if (p < n_pix && job.depth[p] > 0) ++c;
  }
  c = warp_sum_i(c);
  __shared__ int part[kCompactThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) s += part[w];
    job.chunk_count[chunk] = s;
  }
}

__global__ void __launch_bounds__(kCompactThreads) compact_scatter_kernel(const RansacJob* __restrict__ jobs,
                                                                         int n_jobs) {
  const RansacJob& job = jobs[chunk_job(jobs, n_jobs, blockIdx.x)];
  const int chunk = blockIdx.x - job.chunk_begin;
  const int n_pix = job.W * job.H;
  const int n_chunks = (n_pix + kCompactChunk - 1) / kCompactChunk;
  __shared__ int s_off;
  __shared__ int scan[kCompactThreads];
  if (threadIdx.x < 32) {
    int s = 0;
    for (int c = threadIdx.x; c < chunk; c += 32) s += job.chunk_count[c];
    s = warp_sum_i(s);
    if (threadIdx.x == 0) s_off = s;
  }
  const int base = chunk * kCompactChunk + threadIdx.x * kPerThread;
  int mine = 0;
  for (int k = 0; k < kPerThread; ++k) {
    const int p = base + k;
    if (p < n_pix && job.depth[p] > 0) ++mine;
  }
  scan[threadIdx.x] = mine;
  __syncthreads();
  for (int o = 1; o < kCompactThreads; o <<= 1) {  // inclusive Hillis-Steele scan
    const int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  int w = s_off + scan[threadIdx.x] - mine;
  for (int k = 0; k < kPerThread; ++k) {
    const int p = base + k;
    if (p < n_pix && job.depth[p] > 0) job.valid[w++] = p;
  }
  if (chunk == n_chunks - 1 && threadIdx.x == kCompactThreads - 1) *job.n_valid = s_off + scan[threadIdx.x];
}

cudaError_t launch_compact(const RansacJob* jobs, int n_jobs, int total_chunks, cudaStream_t s) {
  if (total_chunks <= 0) return cudaSuccess;
  compact_count_kernel<<<total_chunks, kCompactThreads, 0, s>>>(jobs, n_jobs);
  compact_scatter_kernel<<<total_chunks, kCompactThreads, 0, s>>>(jobs, n_jobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Hypotheses
// ---------------------------------------------------------------------------------------------
constexpr int kHypThreads = 256;
constexpr float kGuardRigid = 1e-4f;  // FP32 error of a distance difference is < 2e-5 m here
constexpr float kGuardArea = 2e-4f;   // and of |cross| < 2e-5 m^2

__device__ __forceinline__ float3 cam_point_f(int pix, int W, int d, float fx, float fy, float cx, float cy) {
  const float z = (float)d * 0.001f;
  const int u = pix % W, v = pix / W;
  return make_float3(z * ((float)u - cx) / fx, z * ((float)v - cy) / fy, z);
}

// FP64 camera point in the oracle's operation order: z = d / 1000; x = (z (u - cx)) / fx.
__device__ __forceinline__ void cam_point_d(int pix, int W, int d, double fx, double fy, double cx, double cy,
                                            double out[3]) {
  const double z = __ddiv_rn((double)d, 1000.0);
  const int u = pix % W, v = pix / W;
  out[0] = __ddiv_rn(__dmul_rn(z, __dsub_rn((double)u, cx)), fx);
  out[1] = __ddiv_rn(__dmul_rn(z, __dsub_rn((double)v, cy)), fy);
  out[2] = z;
}

__device__ __forceinline__ double dist_d(const double* a, const double* b) {
  const double d0 = __dsub_rn(a[0], b[0]), d1 = __dsub_rn(a[1], b[1]), d2 = __dsub_rn(a[2], b[2]);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2)));
}

__device__ __forceinline__ double cross_norm_d(const double* p0, const double* p1, const double* p2) {
  const double e1[3] = {__dsub_rn(p1[0], p0[0]), __dsub_rn(p1[1], p0[1]), __dsub_rn(p1[2], p0[2])};
  const double e2[3] = {__dsub_rn(p2[0], p0[0]), __dsub_rn(p2[1], p0[1]), __dsub_rn(p2[2], p0[2])};
  const double x = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
  const double y = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
  const double z = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
}

__device__ __forceinline__ float dist_f(float3 a, float3 b) {
  const float x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
  return sqrtf(x * x + y * y + z * z);
}

__device__ __forceinline__ float cross_norm_f(float3 p0, float3 p1, float3 p2) {
  const float ax = p1.x - p0.x, ay = p1.y - p0.y, az = p1.z - p0.z;
  const float bx = p2.x - p0.x, by = p2.y - p0.y, bz = p2.z - p0.z;
  const float x = ay * bz - az * by, y = az * bx - ax * bz, z = ax * by - ay * bx;
  return sqrtf(x * x + y * y + z * z);
}

struct TryDraw {
  int pix[3];
  int tree[3];
  int leaf[3];
};

__device__ __forceinline__ TryDraw draw_try(const RansacJob& job, int h, int j, int n_valid) {
  const uint4 x = philox4x32_10(make_uint4(1u, (uint32_t)h, (uint32_t)j, 0u), job.key0, job.key1);
  TryDraw t;
  const uint32_t w[3] = {x.x, x.y, x.z};
  const int n_pix = job.W * job.H;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    t.pix[k] = __ldg(&job.valid[uniform_below(w[k], (uint32_t)n_valid)]);
    t.tree[k] = (int)((((x.w >> (8 * k)) & 0xFFu) * (uint32_t)job.forest.T) >> 8);
    t.leaf[k] = __ldg(&job.leaves[(size_t)t.tree[k] * n_pix + t.pix[k]]);
  }
  return t;
}

// Exact decision of the rigidity and area tests in FP64, in the oracle's operation order.
__device__ bool exact_geometry(const RansacJob& job, const TryDraw& t, const float4* mode) {
  double c[3][3], w[3][3];
  for (int k = 0; k < 3; ++k) {
    cam_point_d(t.pix[k], job.W, job.depth[t.pix[k]], job.fx, job.fy, job.cx, job.cy, c[k]);
    w[k][0] = (double)mode[k].x;
    w[k][1] = (double)mode[k].y;
    w[k][2] = (double)mode[k].z;
  }
  const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  bool ok = true;
  for (int q = 0; q < 3; ++q) {
    const double dc = dist_d(c[pr[q][0]], c[pr[q][1]]), dw = dist_d(w[pr[q][0]], w[pr[q][1]]);
    ok = ok && (fabs(__dsub_rn(dc, dw)) <= job.rigidity);
  }
  ok = ok && (cross_norm_d(c[0], c[1], c[2]) >= job.min_area) && (cross_norm_d(w[0], w[1], w[2]) >= job.min_area);
  return ok;
}

__device__ bool try_passes(const RansacJob& job, int h, int j, int n_valid) {
  const TryDraw t = draw_try(job, h, j, n_valid);
  const int L = 1 << job.forest.D;
  float4 m[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (t.leaf[k] >= L) return false;  // invalid pixel (0xFFFF) or a leaf id outside the forest
    m[k] = __ldg(&job.forest.top[(size_t)t.tree[k] * L + t.leaf[k]]);
    if (m[k].w < 0.5f) return false;  // empty leaf
  }
  if (t.pix[0] == t.pix[1] || t.pix[0] == t.pix[2] || t.pix[1] == t.pix[2]) return false;
  float3 c[3], w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c[k] = cam_point_f(t.pix[k], job.W, job.depth[t.pix[k]], (float)job.fx, (float)job.fy, (float)job.cx,
                       (float)job.cy);
    w[k] = make_float3(m[k].x, m[k].y, m[k].z);
  }
  const float rig = (float)job.rigidity, area = (float)job.min_area;
  bool ambiguous = false;
  const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float diff = fabsf(dist_f(c[pr[q][0]], c[pr[q][1]]) - dist_f(w[pr[q][0]], w[pr[q][1]]));
    if (diff > rig + kGuardRigid) return false;
    if (diff >= rig - kGuardRigid) ambiguous = true;
  }
  const float ac = cross_norm_f(c[0], c[1], c[2]), aw = cross_norm_f(w[0], w[1], w[2]);
  if (ac < area - kGuardArea || aw < area - kGuardArea) return false;
  if (ac <= area + kGuardArea || aw <= area + kGuardArea) ambiguous = true;
  if (!ambiguous) return true;
  return exact_geometry(job, t, m);
}

__global__ void __launch_bounds__(kHypThreads) hypotheses_kernel(const RansacJob* __restrict__ jobs, int n_jobs) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].hyp_begin <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const RansacJob& job = jobs[lo];
  const int h = blockIdx.x - job.hyp_begin;
  if (h >= job.K) return;
  const int n_valid = *job.n_valid;
  __shared__ int s_win;
  if (threadIdx.x == 0) s_win = INT_MAX;
  __syncthreads();
  if (n_valid > 0) {
    for (int base = 0; base < job.max_tries; base += kHypThreads) {
      const int j = base + threadIdx.x;
      if (j < job.max_tries && try_passes(job, h, j, n_valid)) atomicMin(&s_win, j);
      __syncthreads();
      const bool done = s_win != INT_MAX;
      __syncthreads();
      if (done) break;
    }
  }
  if (threadIdx.x == 0) {
    const int win = s_win;
    double* pose = job.poses + 12 * (size_t)h;
    const bool ok = win != INT_MAX;
    if (ok) {
      // FP64 Kabsch (Horn) on the winning try's three correspondences
      const TryDraw t = draw_try(job, h, win, n_valid);
      const int L = 1 << job.forest.D;
      double c[3][3], w[3][3], cb[3] = {0, 0, 0}, wb[3] = {0, 0, 0};
      for (int k = 0; k < 3; ++k) {
        cam_point_d(t.pix[k], job.W, job.depth[t.pix[k]], job.fx, job.fy, job.cx, job.cy, c[k]);
        const float4 m = job.forest.top[(size_t)t.tree[k] * L + t.leaf[k]];
        w[k][0] = m.x;
        w[k][1] = m.y;
        w[k][2] = m.z;
        for (int a = 0; a < 3; ++a) {
          cb[a] += c[k][a] / 3.0;
          wb[a] += w[k][a] / 3.0;
        }
      }
      double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) S[3 * a + b] += (c[k][a] - cb[a]) * (w[k][b] - wb[b]);
      horn_pose(S, cb, wb, pose);
    } else {
      for (int q = 0; q < 12; ++q) pose[q] = (q % 5 == 0) ? 1.0 : 0.0;
    }
    job.hyp_ok[h] = ok ? 1 : 0;
    job.tries[h] = ok ? win : job.max_tries;
    job.energy[h] = ok ? 0.0 : (double)INFINITY;
    job.alive_a[h] = h;
    job.inliers[h] = 0;
  }
}

cudaError_t launch_hypotheses(const RansacJob* jobs, int n_jobs, int total_hyps, cudaStream_t s) {
  if (total_hyps <= 0) return cudaSuccess;
  hypotheses_kernel<<<total_hyps, kHypThreads, 0, s>>>(jobs, n_jobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Rounds
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ const int32_t* alive_in(const RansacJob& j, int r) { return (r & 1) ? j.alive_b : j.alive_a; }
__device__ __forceinline__ int32_t* alive_out(const RansacJob& j, int r) { return (r & 1) ? j.alive_a : j.alive_b; }

// Draw round r's B pixels (one CTA per job).
__global__ void draw_kernel(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ alive_prefix, int r) {
  const int jid = blockIdx.x;
  if (alive_prefix[jid + 1] - alive_prefix[jid] == 0) return;
  const RansacJob& job = jobs[jid];
  const int n_valid = *job.n_valid;
  if (n_valid == 0) return;
  for (int i = threadIdx.x; i < job.B; i += blockDim.x) {
    const uint4 x = philox4x32_10(make_uint4(2u, (uint32_t)r, (uint32_t)i, 0u), job.key0, job.key1);
    job.drawn[(size_t)r * job.B + i] = job.valid[uniform_below(x.x, (uint32_t)n_valid)];
  }
}

// Best mode of pixel pix under x: returns score (-inf if none) and the mode's mean.
__device__ __forceinline__ float best_mode(const RansacJob& job, int pix, float3 x, float3* mu_best) {
  const ForestView& f = job.forest;
  const int n_pix = job.W * job.H, L = 1 << f.D;
  float best = -INFINITY;
  for (int t = 0; t < f.T; ++t) {
    const int leaf = __ldg(&job.leaves[(size_t)t * n_pix + pix]);
    if (leaf >= L) continue;  // invalid pixel (0xFFFF) or a leaf id outside the forest
    const int nm = min((int)__ldg(&f.n_modes[(size_t)t * L + leaf]), f.M);
    const float4* m = reinterpret_cast<const float4*>(f.modes + ((size_t)t * L + leaf) * f.M * kModeFloats);
    for (int k = 0; k < nm; ++k) {
      const float4 a = __ldg(&m[3 * k]), b = __ldg(&m[3 * k + 1]), c = __ldg(&m[3 * k + 2]);
      const float dx = x.x - a.x, dy = x.y - a.y, dz = x.z - a.z;
      // a.w = inv_xx, b = (inv_xy, inv_xz, inv_yy, inv_yz), c = (inv_zz, logw - 0.5 log det, w, pad)
      const float q = dx * (a.w * dx + b.x * dy + b.y * dz) + dy * (b.x * dx + b.z * dy + b.w * dz) +
                      dz * (b.y * dx + b.w * dy + c.x * dz);
      const float sc = c.y - 0.5f * q;
      if (sc > best) {
        best = sc;
        if (mu_best) *mu_best = make_float3(a.x, a.y, a.z);
      }
    }
  }
  return best;
}

__device__ __forceinline__ float3 drawn_cam(const RansacJob& job, int pix) {
  return cam_point_f(pix, job.W, __ldg(&job.depth[pix]), (float)job.fx, (float)job.fy, (float)job.cx, (float)job.cy);
}

// Energies of round r: warp per alive hypothesis.
__global__ void __launch_bounds__(256) energy_kernel(const RansacJob* __restrict__ jobs, int n_jobs,
                                                     const int32_t* __restrict__ alive_prefix, int total, int r) {
  const int gw = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= total) return;
  const int jid = find_job_by(alive_prefix, n_jobs, gw);
  const RansacJob& job = jobs[jid];
  const int h = alive_in(job, r)[gw - alive_prefix[jid]];
  if (!job.hyp_ok[h] || *job.n_valid == 0) return;
  const PoseF P = pose_to_float(job.poses + 12 * (size_t)h);
  float sum = 0.f;
  const int32_t* px = job.drawn + (size_t)r * job.B;
  for (int i = lane; i < job.B; i += 32) {
    const int pix = __ldg(&px[i]);
    const float3 x = apply(P, drawn_cam(job, pix));
    const float best = best_mode(job, pix, x, nullptr);
    sum += fminf(kLogEps, -best);
  }
  sum = warp_sum(sum);
  if (lane == 0) job.energy[h] += (double)sum;
}

__device__ __forceinline__ unsigned long long order_key(double e) {
  unsigned long long b = (unsigned long long)__double_as_longlong(e);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Halving: CTA per job, bitonic sort of (energy key, index) ascending; keep ceil(n/2).
__global__ void __launch_bounds__(1024) select_kernel(const RansacJob* __restrict__ jobs,
                                                      const int32_t* __restrict__ alive_prefix, int r) {
  extern __shared__ unsigned long long skey[];
  const int jid = blockIdx.x;
  const int n = alive_prefix[jid + 1] - alive_prefix[jid];
  if (n == 0) return;
  const RansacJob& job = jobs[jid];
  int npow = 1;
  while (npow < n) npow <<= 1;
  int* sidx = reinterpret_cast<int*>(skey + npow);
  const int32_t* in = alive_in(job, r);
  for (int i = threadIdx.x; i < npow; i += blockDim.x) {
    if (i < n) {
      const int h = in[i];
      skey[i] = order_key(job.energy[h]);
      sidx[i] = h;
    } else {
      skey[i] = ~0ull;
      sidx[i] = INT_MAX;
    }
  }
  __syncthreads();
  for (int k = 2; k <= npow; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        const int l = i ^ jj;
        if (l > i) {
          const bool up = (i & k) == 0;
          const bool gt = skey[i] > skey[l] || (skey[i] == skey[l] && sidx[i] > sidx[l]);
          if (gt == up) {
            const unsigned long long tk = skey[i];
            skey[i] = skey[l];
            skey[l] = tk;
            const int ti = sidx[i];
            sidx[i] = sidx[l];
            sidx[l] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  const int keep = (n + 1) / 2;
  int32_t* out = alive_out(job, r);
  for (int i = threadIdx.x; i < keep; i += blockDim.x) out[i] = sidx[i];
}

// Re-fit: warp per survivor over all pixels drawn in rounds 0..r.
__global__ void __launch_bounds__(256) refine_kernel(const RansacJob* __restrict__ jobs, int n_jobs,
                                                     const int32_t* __restrict__ surv_prefix, int total, int r) {
  const int gw = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= total) return;
  const int jid = find_job_by(surv_prefix, n_jobs, gw);
  const RansacJob& job = jobs[jid];
  const int h = alive_out(job, r)[gw - surv_prefix[jid]];
  if (!job.hyp_ok[h] || *job.n_valid == 0) return;
  const PoseF P = pose_to_float(job.poses + 12 * (size_t)h);
  const int n_drawn = (r + 1) * job.B;
  const float r2 = (float)(job.inlier_dist * job.inlier_dist);
  // pass 1: inlier count and centroids
  int cnt = 0;
  float sc[3] = {0, 0, 0}, sw[3] = {0, 0, 0};
  for (int i = lane; i < n_drawn; i += 32) {
    const int pix = __ldg(&job.drawn[i]);
    const float3 c = drawn_cam(job, pix);
    const float3 x = apply(P, c);
    float3 mu;
    const float best = best_mode(job, pix, x, &mu);
    if (best == -INFINITY) continue;
    const float dx = x.x - mu.x, dy = x.y - mu.y, dz = x.z - mu.z;
    if (dx * dx + dy * dy + dz * dz < r2) {
      ++cnt;
      sc[0] += c.x; sc[1] += c.y; sc[2] += c.z;
      sw[0] += mu.x; sw[1] += mu.y; sw[2] += mu.z;
    }
  }
  cnt = warp_sum_i(cnt);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    sc[a] = warp_sum(sc[a]);
    sw[a] = warp_sum(sw[a]);
  }
  if (lane == 0) job.inliers[h] = cnt;
  if (cnt < 3) return;
  const float inv = 1.0f / (float)cnt;
  const float cb[3] = {sc[0] * inv, sc[1] * inv, sc[2] * inv}, wb[3] = {sw[0] * inv, sw[1] * inv, sw[2] * inv};
  // pass 2: cross-covariance about the centroids
  float S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = lane; i < n_drawn; i += 32) {
    const int pix = __ldg(&job.drawn[i]);
    const float3 c = drawn_cam(job, pix);
    const float3 x = apply(P, c);
    float3 mu;
    const float best = best_mode(job, pix, x, &mu);
    if (best == -INFINITY) continue;
    const float dx = x.x - mu.x, dy = x.y - mu.y, dz = x.z - mu.z;
    if (dx * dx + dy * dy + dz * dz < r2) {
      const float e[3] = {c.x - cb[0], c.y - cb[1], c.z - cb[2]}, g[3] = {mu.x - wb[0], mu.y - wb[1], mu.z - wb[2]};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) S[3 * a + b] = fmaf(e[a], g[b], S[3 * a + b]);
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) S[q] = warp_sum(S[q]);
  if (lane == 0) {
    double Sd[9], cbd[3], wbd[3];
    for (int q = 0; q < 9; ++q) Sd[q] = S[q];
    for (int a = 0; a < 3; ++a) {
      cbd[a] = cb[a];
      wbd[a] = wb[a];
    }
    horn_pose(Sd, cbd, wbd, job.poses + 12 * (size_t)h);
  }
}

cudaError_t launch_round(const RansacJob* jobs, int n_jobs, int round, const int32_t* alive_prefix_dev,
                         int total_alive, const int32_t* surv_prefix_dev, int total_surv, cudaStream_t s) {
  if (total_alive <= 0) return cudaSuccess;
  draw_kernel<<<n_jobs, 256, 0, s>>>(jobs, alive_prefix_dev, round);
  energy_kernel<<<(unsigned)((total_alive * 32 + 255) / 256), 256, 0, s>>>(jobs, n_jobs, alive_prefix_dev,
                                                                           total_alive, round);
  // the largest alive set bounds the shared memory of the sort
  select_kernel<<<n_jobs, 1024, 4096 * (sizeof(unsigned long long) + sizeof(int)), s>>>(jobs, alive_prefix_dev,
                                                                                        round);
  refine_kernel<<<(unsigned)((total_surv * 32 + 255) / 256), 256, 0, s>>>(jobs, n_jobs, surv_prefix_dev,
                                                                          total_surv, round);
  return cudaGetLastError();
}

// Final hypothesis -> result (one thread per job).
__global__ void finalise_kernel(const RansacJob* __restrict__ jobs, int n_jobs) {
  const int jid = blockIdx.x * blockDim.x + threadIdx.x;
  if (jid >= n_jobs) return;
  const RansacJob& job = jobs[jid];
  const int32_t* fin = (job.n_rounds & 1) ? job.alive_b : job.alive_a;
  const int h = fin[0];
  relo_pose_result* res = job.result;
  const double* p = job.poses + 12 * (size_t)h;
  for (int i = 0; i < 3; ++i)
    for (int q = 0; q < 4; ++q) res->pose_c2s[4 * i + q] = p[4 * i + q];
  res->pose_c2s[12] = res->pose_c2s[13] = res->pose_c2s[14] = 0.0;
  res->pose_c2s[15] = 1.0;
  res->energy = job.energy[h];
  res->n_inliers = job.inliers[h];
  res->status = *job.err ? RELO_EDEVICE : (job.hyp_ok[h] ? RELO_OK : RELO_ENOTFOUND);
  res->verified = 0;
  res->n_valid = *job.n_valid;
  res->hypothesis = h;
  res->n_rounds = job.n_rounds;
  res->omega = res->omega_a = res->omega_b = res->omega_ab = res->sum_absdiff_mm = 0;
  for (int q = 0; q < 16; ++q) res->rel_a_b[q] = (q % 5 == 0) ? 1.0 : 0.0;
  if (job.has_pose_b) {
    // a_T_b = P_a P_b^-1 with P_b^-1 = [R_b^T | -R_b^T t_b]
    const double* b = job.pose_b;
    double inv[12];
    for (int i = 0; i < 3; ++i) {
      for (int q = 0; q < 3; ++q) inv[4 * i + q] = b[4 * q + i];
      inv[4 * i + 3] = -(b[i] * b[3] + b[4 + i] * b[7] + b[8 + i] * b[11]);
    }
    for (int i = 0; i < 3; ++i)
      for (int q = 0; q < 4; ++q) {
        double acc = (q == 3) ? p[4 * i + 3] : 0.0;
        for (int k = 0; k < 3; ++k) acc += p[4 * i + k] * inv[4 * k + q];
        res->rel_a_b[4 * i + q] = acc;
      }
  }
}

// Verification decision (Sec. 3.3.1) from the counts the compare raycast accumulated:
// accept iff |Omega_a| / |Omega| > 1/2 and the mean |D_a - D_b| over Omega_ab is below 50 mm
// (an empty Omega_ab rejects), in integers.
__device__ __forceinline__ void decide(relo_pose_result* res, unsigned long long omega) {
  res->omega = omega;
  res->verified = (res->status == RELO_OK && 2 * res->omega_a > res->omega && res->omega_ab > 0 &&
                   res->sum_absdiff_mm < 50ull * res->omega_ab)
                      ? 1
                      : 0;
}

__global__ void verify_decide_kernel(const RansacJob* __restrict__ jobs, int n_jobs) {
  const int jid = blockIdx.x * blockDim.x + threadIdx.x;
  if (jid >= n_jobs) return;
  decide(jobs[jid].result, (unsigned long long)jobs[jid].W * jobs[jid].H);
}

__global__ void verify_decide_one_kernel(relo_pose_result* res, unsigned long long omega) { decide(res, omega); }

cudaError_t launch_verify_decide(const RansacJob* jobs, int n_jobs, cudaStream_t s) {
  verify_decide_kernel<<<(n_jobs + 127) / 128, 128, 0, s>>>(jobs, n_jobs);
  return cudaGetLastError();
}

cudaError_t launch_verify_decide_one(relo_pose_result* res, uint64_t omega, cudaStream_t s) {
  verify_decide_one_kernel<<<1, 1, 0, s>>>(res, (unsigned long long)omega);
  return cudaGetLastError();
}

cudaError_t launch_finalise(const RansacJob* jobs, int n_jobs, cudaStream_t s) {
  finalise_kernel<<<(n_jobs + 127) / 128, 128, 0, s>>>(jobs, n_jobs);
  return cudaGetLastError();
}

}  // namespace relo
