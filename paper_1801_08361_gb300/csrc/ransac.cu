// ransac.cu -- preemptive RANSAC over forest correspondences (the relocaliser's pose solver,
// after Cavallari et al. as used in Sec. 3.3.1; every rule is a stated reading, see relo.h).
//
// Stages, each one launch over all jobs of a batch:
//   compact    : ordered table of valid pixels, each entry packing {u, v, depth, leaf per tree}
//                in 16-byte words so that one load serves a correspondence (two passes: chunk
//                counts, then an ordered scatter with warp ballots);
//   search     : one warp per hypothesis evaluates 32 tries at a time and keeps the first passing
//                try, so the result equals a sequential scan of the tries.  The rigidity / area
//                tests run in FP32 with a guard band; a try inside the band is settled in FP64 in
//                the oracle's operation order;
//   fit        : one thread per hypothesis: 3-point Kabsch in FP64 (Horn's quaternion form);
//   per round  : draw B pixels; energies (warp per hypothesis, lanes over pixels, FP32 with an
//                FP64 running total); halving (CTA per job, bitonic sort of (energy, index));
//                re-fit sums (warp per survivor, one pass of shifted FP32 sums reduced with
//                shuffles); re-fit solve (thread per survivor, FP64 Horn).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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

// u16 number k (0..7) of a 16-byte word
__device__ __forceinline__ uint32_t u16_of(uint4 q, int k) {
  const uint32_t w = (k < 4) ? ((k < 2) ? q.x : q.y) : ((k < 6) ? q.z : q.w);
  return (k & 1) ? (w >> 16) : (w & 0xFFFFu);
}

struct TableEntry {
  int u, v, depth;
  uint4 w0;  // first word (u, v, depth, leaf[0..4])
};

__device__ __forceinline__ TableEntry load_entry(const RansacJob& job, int idx) {
  TableEntry e;
  if (!RELO_CHECK(idx >= 0 && idx < *job.n_valid)) idx = 0;
  e.w0 = __ldg(&job.table[(size_t)idx * job.nv]);
  e.u = (int)(e.w0.x & 0xFFFFu);
  e.v = (int)(e.w0.x >> 16);
  e.depth = (int)(e.w0.y & 0xFFFFu);
  return e;
}

// Leaf of tree t for a table entry (field 3 + t of the packed entry).
__device__ __forceinline__ int entry_leaf(const RansacJob& job, int idx, const TableEntry& e, int t) {
  const int f = 3 + t;
  if (f < 8) return (int)u16_of(e.w0, f);
  return (int)u16_of(__ldg(&job.table[(size_t)idx * job.nv + (f >> 3)]), f & 7);
}

// FP32 camera point with reciprocal focal lengths ifx = 1 / fx, ify = 1 / fy (a few ulp from the
// FP64 point; the FP32 tests and scores that use it tolerate that).
__device__ __forceinline__ float3 cam_point_f(int u, int v, int d, float ifx, float ify, float cx, float cy) {
  const float z = (float)d * 0.001f;
  return make_float3(z * ((float)u - cx) * ifx, z * ((float)v - cy) * ify, z);
}

// FP64 camera point in the oracle's operation order: z = d / 1000; x = (z (u - cx)) / fx.
__device__ __forceinline__ void cam_point_d(int u, int v, int d, double fx, double fy, double cx, double cy,
                                            double out[3]) {
  const double z = __ddiv_rn((double)d, 1000.0);
  out[0] = __ddiv_rn(__dmul_rn(z, __dsub_rn((double)u, cx)), fx);
  out[1] = __ddiv_rn(__dmul_rn(z, __dsub_rn((double)v, cy)), fy);
  out[2] = z;
}

// ---------------------------------------------------------------------------------------------
// Valid-pixel table
// ---------------------------------------------------------------------------------------------
constexpr int kCompactThreads = 256;
constexpr int kIters = kCompactChunk / kCompactThreads;  // 16 coalesced passes of 256 pixels

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
  if (job_skipped(job.skip)) return;
  const int chunk = blockIdx.x - job.chunk_begin;
  const int n_pix = job.W * job.H;
  int c = 0;
  for (int it = 0; it < kIters; ++it) {
    const int p = chunk * kCompactChunk + it * kCompactThreads + threadIdx.x;
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
  if (job_skipped(job.skip)) return;
  const int chunk = blockIdx.x - job.chunk_begin;
  const int n_pix = job.W * job.H;
  const int n_chunks = (n_pix + kCompactChunk - 1) / kCompactChunk;
  const int T = job.forest.T, nv = job.nv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ int s_off;
  __shared__ int s_warp[kCompactThreads / 32];
  if (threadIdx.x < 32) {
    int s = 0;
    for (int c = threadIdx.x; c < chunk; c += 32) s += job.chunk_count[c];
    s = warp_sum_i(s);
    if (threadIdx.x == 0) s_off = s;
  }
  __syncthreads();
  int off = s_off;
  for (int it = 0; it < kIters; ++it) {
    const int p = chunk * kCompactChunk + it * kCompactThreads + threadIdx.x;
    const int d = p < n_pix ? job.depth[p] : 0;
    const unsigned ball = __ballot_sync(0xffffffffu, d > 0);
    if (lane == 0) s_warp[warp] = __popc(ball);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kCompactThreads / 32; ++w) {
      const int c = s_warp[w];
      before += (w < warp) ? c : 0;
      total += c;
    }
    if (d > 0) {
      const int pos = off + before + __popc(ball & ((1u << lane) - 1u));
      uint16_t f[24];
      f[0] = (uint16_t)(p % job.W);
      f[1] = (uint16_t)(p / job.W);
      f[2] = (uint16_t)d;
      for (int t = 0; t < T; ++t) f[3 + t] = job.leaves[(size_t)t * n_pix + p];
      for (int k = 3 + T; k < 8 * nv; ++k) f[k] = 0;
      uint4* dst = job.table + (size_t)pos * nv;
      for (int q = 0; q < nv; ++q)
        dst[q] = make_uint4(f[8 * q] | ((uint32_t)f[8 * q + 1] << 16), f[8 * q + 2] | ((uint32_t)f[8 * q + 3] << 16),
                            f[8 * q + 4] | ((uint32_t)f[8 * q + 5] << 16), f[8 * q + 6] | ((uint32_t)f[8 * q + 7] << 16));
    }
    off += total;
    __syncthreads();
  }
  if (chunk == n_chunks - 1 && threadIdx.x == 0) *job.n_valid = off;
}

cudaError_t launch_compact(const RansacJob* jobs, int n_jobs, int total_chunks, cudaStream_t s) {
  if (total_chunks <= 0) return cudaSuccess;
  compact_count_kernel<<<total_chunks, kCompactThreads, 0, s>>>(jobs, n_jobs);
  compact_scatter_kernel<<<total_chunks, kCompactThreads, 0, s>>>(jobs, n_jobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Hypothesis search
// ---------------------------------------------------------------------------------------------
constexpr float kGuardRigid = 1e-4f;  // FP32 error of a distance difference stays below 2e-5 m here
constexpr float kGuardArea = 2e-4f;   // and that of |cross| below 2e-5 m^2

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

// Distance through the hardware reciprocal square root (relative error about 2^-22, i.e. below
// 1e-5 m on the few-metre distances here and inside the guard band of the tests using it).
__device__ __forceinline__ float dist_f(float3 a, float3 b) {
  const float x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
  const float s = x * x + y * y + z * z;
  return s > 0.f ? s * rsqrtf(s) : 0.f;
}

// |cross(p1 - p0, p2 - p0)|^2 (compared against squared area bounds).
__device__ __forceinline__ float cross_norm2_f(float3 p0, float3 p1, float3 p2) {
  const float ax = p1.x - p0.x, ay = p1.y - p0.y, az = p1.z - p0.z;
  const float bx = p2.x - p0.x, by = p2.y - p0.y, bz = p2.z - p0.z;
  const float x = ay * bz - az * by, y = az * bx - ax * bz, z = ax * by - ay * bx;
  return x * x + y * y + z * z;
}

struct Corr {
  int idx[3], tree[3], leaf[3];
  TableEntry e[3];
};

__device__ __forceinline__ Corr draw_try(const RansacJob& job, int h, int j, int n_valid) {
  const uint4 x = philox4x32_10(make_uint4(1u, (uint32_t)h, (uint32_t)j, 0u), job.key0, job.key1);
  Corr c;
  const uint32_t w[3] = {x.x, x.y, x.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c.idx[k] = (int)uniform_below(w[k], (uint32_t)n_valid);
    c.tree[k] = (int)((((x.w >> (8 * k)) & 0xFFu) * (uint32_t)job.forest.T) >> 8);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) c.e[k] = load_entry(job, c.idx[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k) c.leaf[k] = entry_leaf(job, c.idx[k], c.e[k], c.tree[k]);
  return c;
}

// Exact decision of the rigidity and area tests in FP64, in the oracle's operation order.
__device__ __noinline__ bool exact_geometry(const RansacJob& job, int h, int j, int n_valid) {
  const Corr c = draw_try(job, h, j, n_valid);
  const int L = 1 << job.forest.D;
  double cp[3][3], wp[3][3];
  for (int k = 0; k < 3; ++k) {
    cam_point_d(c.e[k].u, c.e[k].v, c.e[k].depth, job.fx, job.fy, job.cx, job.cy, cp[k]);
    const float4 m = __ldg(&job.forest.top[(size_t)c.tree[k] * L + c.leaf[k]]);
    wp[k][0] = (double)m.x;
    wp[k][1] = (double)m.y;
    wp[k][2] = (double)m.z;
  }
  const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  bool ok = true;
  for (int q = 0; q < 3; ++q) {
    const double dc = dist_d(cp[pr[q][0]], cp[pr[q][1]]), dw = dist_d(wp[pr[q][0]], wp[pr[q][1]]);
    ok = ok && (fabs(__dsub_rn(dc, dw)) <= job.rigidity);
  }
  return ok && (cross_norm_d(cp[0], cp[1], cp[2]) >= job.min_area) &&
         (cross_norm_d(wp[0], wp[1], wp[2]) >= job.min_area);
}

// Mode-0 mean of a correspondence's leaf (w = its count; w < 0.5: empty leaf), or w = -1 when the
// leaf id is outside the forest.
__device__ __forceinline__ float4 corr_mode(const RansacJob& job, int tree, int leaf, int L) {
  return leaf < L ? __ldg(&job.forest.top[(size_t)tree * L + leaf]) : make_float4(0.f, 0.f, 0.f, -1.f);
}

// Rigidity of one pair: 0 fails, 1 passes, 2 inside the guard band.
__device__ __forceinline__ int pair_status(float3 pa, float3 pb, float3 qa, float3 qb, float rig) {
  const float diff = fabsf(dist_f(pa, pb) - dist_f(qa, qb));
  if (diff > rig + kGuardRigid) return 0;
  return diff >= rig - kGuardRigid ? 2 : 1;
}

// The draws of one try: three table positions and three trees.
struct TryDraw {
  int i0, i1, i2, t0, t1, t2;
};

__device__ __forceinline__ TryDraw draw_indices(const RansacJob& job, int h, int j, int n_valid) {
  const uint4 x = philox4x32_10(make_uint4(1u, (uint32_t)h, (uint32_t)j, 0u), job.key0, job.key1);
  const uint32_t T = (uint32_t)job.forest.T;
  TryDraw d;
  d.i0 = (int)uniform_below(x.x, (uint32_t)n_valid);
  d.i1 = (int)uniform_below(x.y, (uint32_t)n_valid);
  d.i2 = (int)uniform_below(x.z, (uint32_t)n_valid);
  d.t0 = (int)(((x.w & 0xFFu) * T) >> 8);
  d.t1 = (int)((((x.w >> 8) & 0xFFu) * T) >> 8);
  d.t2 = (int)((((x.w >> 16) & 0xFFu) * T) >> 8);
  return d;
}

// The first pair of a try, loaded: entries and mode-0 means of correspondences 0 and 1.
struct TryPair {
  TableEntry e0, e1;
  float4 m0, m1;
};

__device__ __forceinline__ TryPair load_pair(const RansacJob& job, const TryDraw& d, int L) {
  TryPair p;
  p.e0 = load_entry(job, d.i0);
  p.e1 = load_entry(job, d.i1);
  p.m0 = corr_mode(job, d.t0, entry_leaf(job, d.i0, p.e0, d.t0), L);
  p.m1 = corr_mode(job, d.t1, entry_leaf(job, d.i1, p.e1, d.t1), L);
  return p;
}

// 0: the try fails; 1: it passes; 2: a test lies inside the FP32 guard band (settle in FP64).
// The tests are a conjunction of pure conditions, so their order does not change the outcome:
// the pair (0, 1) (already loaded) is tested before the third correspondence is loaded, which
// most tries never reach.
__device__ __forceinline__ int try_status(const RansacJob& job, const TryDraw& d, const TryPair& pr, int L, float rig,
                                          float area_lo2, float area_hi2, float ifx, float ify, float cx, float cy) {
  if (d.i0 == d.i1 || d.i0 == d.i2 || d.i1 == d.i2) return 0;
  if (pr.m0.w < 0.5f || pr.m1.w < 0.5f) return 0;
  const float3 p0 = cam_point_f(pr.e0.u, pr.e0.v, pr.e0.depth, ifx, ify, cx, cy);
  const float3 p1 = cam_point_f(pr.e1.u, pr.e1.v, pr.e1.depth, ifx, ify, cx, cy);
  const float3 q0 = make_float3(pr.m0.x, pr.m0.y, pr.m0.z), q1 = make_float3(pr.m1.x, pr.m1.y, pr.m1.z);
  const int s01 = pair_status(p0, p1, q0, q1, rig);
  if (s01 == 0) return 0;
  const TableEntry e2 = load_entry(job, d.i2);
  const float4 m2 = corr_mode(job, d.t2, entry_leaf(job, d.i2, e2, d.t2), L);
  if (m2.w < 0.5f) return 0;
  const float3 p2 = cam_point_f(e2.u, e2.v, e2.depth, ifx, ify, cx, cy);
  const float3 q2 = make_float3(m2.x, m2.y, m2.z);
  const int s02 = pair_status(p0, p2, q0, q2, rig);
  if (s02 == 0) return 0;
  const int s12 = pair_status(p1, p2, q1, q2, rig);
  if (s12 == 0) return 0;
  bool ambiguous = s01 == 2 || s02 == 2 || s12 == 2;
  const float ac2 = cross_norm2_f(p0, p1, p2), aw2 = cross_norm2_f(q0, q1, q2);
  if (ac2 < area_lo2 || aw2 < area_lo2) return 0;
  if (ac2 <= area_hi2 || aw2 <= area_hi2) ambiguous = true;
  return ambiguous ? 2 : 1;
}

// One warp per hypothesis (four per CTA, no block-wide barriers): each step evaluates 64 tries,
// two per lane (tries base + lane and base + 32 + lane, whose loads are issued together), and
// keeps the first one not failing in try order, settling guard-band tries in FP64 in order.
constexpr int kSearchWarps = 4;

// first try of mask (bits = lanes) that passes, settling guard-band statuses in FP64; -1 if none
__device__ __forceinline__ int first_passing(const RansacJob& job, int h, int n_valid, unsigned mask, int st,
                                             int j, int lane) {
  while (mask) {
    const int w = __ffs(mask) - 1;
    const int sw = __shfl_sync(0xffffffffu, st, w);
    int ok = sw == 1;
    if (!ok) {
      int e = 0;
      if (lane == w) e = exact_geometry(job, h, j, n_valid) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, e, w);
    }
    if (ok) return w;
    mask &= mask - 1;  // rejected in FP64: consider the next try of this step
  }
  return -1;
}

// CTAs per SM for the search (5 x 128 threads: 96 registers for the two tries in flight per lane,
// with about 60 bytes spilled): on the house batch the hypotheses stage takes 18.68 ms at 5, 18.98
// at 4 (128 registers, no spills) and 21.89 at 6 (80 registers, 128-byte spills)
#ifndef RELO_SEARCH_MIN_BLOCKS
#define RELO_SEARCH_MIN_BLOCKS 5
#endif
// The search of hypothesis gw (flattened over the jobs) by one warp.
__device__ __forceinline__ int search_one(const RansacJob* __restrict__ jobs, int n_jobs, int gw, int lane) {
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].hyp_begin <= gw) lo = mid;
    else hi = mid - 1;
  }
  const RansacJob& job = jobs[lo];
  const int h = gw - job.hyp_begin;
  if (h >= job.K || job_skipped(job.skip)) return lo;
  const int n_valid = *job.n_valid;
  const float rig = (float)job.rigidity, area = (float)job.min_area;
  // the area test |cross| >= area with its guard band, on squares (both sides non-negative)
  const float area_lo = fmaxf(area - kGuardArea, 0.f), area_hi = area + kGuardArea;
  const float area_lo2 = area_lo * area_lo, area_hi2 = area_hi * area_hi;
  const float ifx = (float)(1.0 / job.fx), ify = (float)(1.0 / job.fy), cx = (float)job.cx, cy = (float)job.cy;
  const int L = 1 << job.forest.D;
  int found = INT_MAX;
  if (n_valid > 0) {
    for (int base = 0; base < job.max_tries && found == INT_MAX; base += 64) {
      const int ja = base + lane, jb = base + 32 + lane;
      const TryDraw da = draw_indices(job, h, ja, n_valid), db = draw_indices(job, h, jb, n_valid);
      const TryPair pa = load_pair(job, da, L), pb = load_pair(job, db, L);
      const int sa = ja < job.max_tries ? try_status(job, da, pa, L, rig, area_lo2, area_hi2, ifx, ify, cx, cy) : 0;
      const int sb = jb < job.max_tries ? try_status(job, db, pb, L, rig, area_lo2, area_hi2, ifx, ify, cx, cy) : 0;
      int w = first_passing(job, h, n_valid, __ballot_sync(0xffffffffu, sa != 0), sa, ja, lane);
      if (w >= 0) {
        found = base + w;
        break;
      }
      w = first_passing(job, h, n_valid, __ballot_sync(0xffffffffu, sb != 0), sb, jb, lane);
      if (w >= 0) found = base + 32 + w;
    }
  }
  if (lane == 0) {
    job.hyp_ok[h] = found != INT_MAX;
    job.tries[h] = found != INT_MAX ? found : job.max_tries;
  }
  return lo;
}

// Persistent: hypotheses need from one try to max_tries, so each warp takes its next hypothesis
// from a counter when it finishes one (which warp computes a hypothesis does not change its result).
__global__ void __launch_bounds__(kSearchWarps * 32, RELO_SEARCH_MIN_BLOCKS)
    search_kernel(const RansacJob* __restrict__ jobs, int n_jobs, int total, int32_t* __restrict__ counter) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int gw = 0;
    if (lane == 0) gw = atomicAdd(counter, 1);
    gw = __shfl_sync(0xffffffffu, gw, 0);
    if (gw >= total) return;
    search_one(jobs, n_jobs, gw, lane);
  }
}

// FP64 Kabsch (Horn) of each hypothesis's kept try; also initialises the round state.
// FP64 Kabsch of hypothesis h's kept try; also initialises its round state.
__device__ __forceinline__ void fit_one(const RansacJob& job, int h) {
  double* pose = job.poses + 12 * (size_t)h;
  const bool ok = job.hyp_ok[h] != 0;
  if (ok) {
    const Corr c = draw_try(job, h, job.tries[h], *job.n_valid);
    const int L = 1 << job.forest.D;
    double cp[3][3], wp[3][3], cb[3] = {0, 0, 0}, wb[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      cam_point_d(c.e[k].u, c.e[k].v, c.e[k].depth, job.fx, job.fy, job.cx, job.cy, cp[k]);
      const float4 m = job.forest.top[(size_t)c.tree[k] * L + c.leaf[k]];
      wp[k][0] = m.x;
      wp[k][1] = m.y;
      wp[k][2] = m.z;
      for (int a = 0; a < 3; ++a) {
        cb[a] += cp[k][a] / 3.0;
        wb[a] += wp[k][a] / 3.0;
      }
    }
    double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] += (cp[k][a] - cb[a]) * (wp[k][b] - wb[b]);
    horn_pose(S, cb, wb, pose);
  } else {
    for (int q = 0; q < 12; ++q) pose[q] = (q % 5 == 0) ? 1.0 : 0.0;
  }
  job.energy[h] = ok ? 0.0 : (double)INFINITY;
  job.alive_a[h] = h;
  job.inliers[h] = 0;
}

__global__ void __launch_bounds__(128) fit_kernel(const RansacJob* __restrict__ jobs, int n_jobs, int total) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  int lo = 0, hi = n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].hyp_begin <= gid) lo = mid;
    else hi = mid - 1;
  }
  const RansacJob& job = jobs[lo];
  const int h = gid - job.hyp_begin;
  if (h >= job.K || job_skipped(job.skip)) return;
  fit_one(job, h);
}

cudaError_t launch_hypotheses(const RansacJob* jobs, int n_jobs, int total_hyps, int32_t* counter, cudaStream_t s,
                              const Schedule& sched) {
  if (total_hyps <= 0) return cudaSuccess;
  static PerDevice resident;  // resident search CTAs per SM on each device
  int sms = 0, per_sm = 0;
  cudaError_t e = device_sms(&sms);
  if (e == cudaSuccess)
    e = per_device(resident, &per_sm, [](int, int* v) {
      cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, search_kernel, kSearchWarps * 32, 0);
      *v = std::max(1, *v);
      return r;
    });
  if (e != cudaSuccess) return e;
  if (sched.search_ctas_per_sm < 0) return cudaErrorInvalidValue;
  const int ctas = sched.search_ctas_per_sm == 0 ? per_sm : std::min(per_sm, sched.search_ctas_per_sm);
  e = cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  const int grid = std::min(sms * ctas, (total_hyps + kSearchWarps - 1) / kSearchWarps);
  search_kernel<<<grid, kSearchWarps * 32, 0, s>>>(jobs, n_jobs, total_hyps, counter);
  fit_kernel<<<(total_hyps + 127) / 128, 128, 0, s>>>(jobs, n_jobs, total_hyps);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Rounds
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ const int32_t* alive_in(const RansacJob& j, int r) { return (r & 1) ? j.alive_b : j.alive_a; }
__device__ __forceinline__ int32_t* alive_out(const RansacJob& j, int r) { return (r & 1) ? j.alive_a : j.alive_b; }

// (first mode, mode count) of an entry's leaf in tree t: its modes are f.modes[first ..
// first + count) in units of kModeFloats; count 0 for a leaf id outside the forest.
__device__ __forceinline__ int2 tree_modes(const RansacJob& job, int idx, const TableEntry& e, int t, int L) {
  const ForestView& f = job.forest;
  const int leaf = entry_leaf(job, idx, e, t);
  if (leaf >= L || !RELO_CHECK(t >= 0 && t < f.T)) return make_int2(0, 0);
  const int node = t * L + leaf;
  return make_int2(node * f.M, min((int)__ldg(&f.n_modes[node]), f.M));
}

// Draw round r's B pixels (positions in the valid table), one CTA per job, and write each drawn
// pixel's record (camera point and where its modes are), which every hypothesis then reads.
__device__ __forceinline__ void draw_block(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ alive_prefix,
                                           int r, int jid) {
  if (alive_prefix[jid + 1] - alive_prefix[jid] == 0) return;
  const RansacJob& job = jobs[jid];
  if (job_skipped(job.skip)) return;
  const int n_valid = *job.n_valid;
  if (n_valid == 0) return;
  const float ifx = (float)(1.0 / job.fx), ify = (float)(1.0 / job.fy), cx = (float)job.cx, cy = (float)job.cy;
  const int T = job.forest.T, L = 1 << job.forest.D;
  for (int i = threadIdx.x; i < job.B; i += blockDim.x) {
    const uint4 x = philox4x32_10(make_uint4(2u, (uint32_t)r, (uint32_t)i, 0u), job.key0, job.key1);
    const int idx = (int)uniform_below(x.x, (uint32_t)n_valid);
    job.drawn[(size_t)r * job.B + i] = idx;
    const TableEntry e = load_entry(job, idx);
    const float3 c = cam_point_f(e.u, e.v, e.depth, ifx, ify, cx, cy);
    int4* rec = job.pix + ((size_t)r * job.B + i) * job.hs;
    rec[0] = make_int4(__float_as_int(c.x), __float_as_int(c.y), __float_as_int(c.z), 0);
    for (int t = 0; t < T; t += 2) {
      const int2 a = tree_modes(job, idx, e, t, L);
      const int2 b = t + 1 < T ? tree_modes(job, idx, e, t + 1, L) : make_int2(0, 0);
      rec[1 + t / 2] = make_int4(a.x, a.y, b.x, b.y);
    }
  }
}

__global__ void draw_kernel(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ alive_prefix, int r) {
  draw_block(jobs, alive_prefix, r, blockIdx.x);
}

// A pixel's modes, staged by its warp in shared memory: the warp copies every mode of the pixel's
// leaves (trees in order, modes in order) with parallel loads, then every lane scores them from
// there, instead of each mode being a dependent global load in turn.
constexpr int kStageModes = 64;  // modes per warp slot; a pixel with more is scored from global memory

struct ModeSlot {
  float4 m[kStageModes * 3];
};

// Copies the modes of record rec into slot (all lanes of the warp take part); returns their
// number, or -1 if they do not fit (then nothing is staged).
__device__ __forceinline__ int stage_modes(const RansacJob& job, const int4* __restrict__ rec, ModeSlot& slot,
                                           int lane) {
  const ForestView& f = job.forest;
  int total = 0;
  for (int t = 0; t < f.T; ++t) {
    const int4 w = __ldg(&rec[1 + t / 2]);
    total += (t & 1) ? w.w : w.y;
  }
  if (total > kStageModes) return -1;
  int off = 0;
  for (int t = 0; t < f.T; ++t) {
    const int4 w = __ldg(&rec[1 + t / 2]);
    const int first = (t & 1) ? w.z : w.x, nm = (t & 1) ? w.w : w.y;
    const float4* src = reinterpret_cast<const float4*>(f.modes + (size_t)first * kModeFloats);
    for (int i = lane; i < 3 * nm; i += 32) slot.m[3 * off + i] = __ldg(&src[i]);
    off += nm;
  }
  __syncwarp();
  return total;
}

// Gaussian score of one mode (a, b, c: its 3 float4) at x.
__device__ __forceinline__ float mode_score(float4 a, float4 b, float4 c, float3 x) {
  const float dx = x.x - a.x, dy = x.y - a.y, dz = x.z - a.z;
  // a.w = inv_xx, b = (inv_xy, inv_xz, inv_yy, inv_yz), c = (inv_zz, logw - 0.5 log det, w, pad)
  const float q = dx * (a.w * dx + b.x * dy + b.y * dz) + dy * (b.x * dx + b.z * dy + b.w * dz) +
                  dz * (b.y * dx + b.w * dy + c.x * dz);
  return c.y - 0.5f * q;
}

// Best mode of a drawn pixel (its record) under x = P c, over trees then modes in order (the first
// of equal scores wins): its score (-inf if none) and mean.  n_staged >= 0: the modes are in slot
// (same order); otherwise they are read from global memory (every lane reads the same mode, so
// each load is one broadcast).
__device__ __forceinline__ float record_best(const RansacJob& job, const int4* __restrict__ rec, const ModeSlot& slot,
                                             int n_staged, float3 x, float3* mu_best) {
  float best = -INFINITY;
  if (n_staged >= 0) {
    for (int k = 0; k < n_staged; ++k) {
      const float4 a = slot.m[3 * k], b = slot.m[3 * k + 1], c = slot.m[3 * k + 2];
      const float sc = mode_score(a, b, c, x);
      if (sc > best) {
        best = sc;
        if (mu_best) *mu_best = make_float3(a.x, a.y, a.z);
      }
    }
    return best;
  }
  const ForestView& f = job.forest;
  for (int t = 0; t < f.T; ++t) {
    const int4 w = __ldg(&rec[1 + t / 2]);
    const int first = (t & 1) ? w.z : w.x, nm = (t & 1) ? w.w : w.y;
    const float4* m = reinterpret_cast<const float4*>(f.modes + (size_t)first * kModeFloats);
    for (int k = 0; k < nm; ++k) {
      const float4 a = __ldg(&m[3 * k]), b = __ldg(&m[3 * k + 1]), c = __ldg(&m[3 * k + 2]);
      const float sc = mode_score(a, b, c, x);
      if (sc > best) {
        best = sc;
        if (mu_best) *mu_best = make_float3(a.x, a.y, a.z);
      }
    }
  }
  return best;
}

__device__ __forceinline__ float3 record_point(const int4* __restrict__ rec) {
  const int4 w = __ldg(&rec[0]);
  return make_float3(__int_as_float(w.x), __int_as_float(w.y), __int_as_float(w.z));
}

// record_best over staged modes with the whole warp on one point x (every lane passes the same x):
// lane l scores modes l, l + 32, ..., then the warp keeps the largest score and, among equal ones,
// the lowest index -- the mode that the scan in order with a strict comparison keeps (a NaN score
// never wins in either).  Returns the score (-inf if none) and, in every lane, the mode's mean.
__device__ __forceinline__ float warp_best_staged(const ModeSlot& slot, int n_staged, float3 x, int lane,
                                                  float3* mu_best) {
  float best = -INFINITY;
  int bi = -1;
  for (int k = lane; k < n_staged; k += 32) {
    const float sc = mode_score(slot.m[3 * k], slot.m[3 * k + 1], slot.m[3 * k + 2], x);
    if (sc > best) {
      best = sc;
      bi = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) {
      best = ob;
      bi = oi;
    }
  }
  if (bi >= 0) {
    const float4 a = slot.m[3 * bi];
    *mu_best = make_float3(a.x, a.y, a.z);
  }
  return best;
}

// Chunks with at most this many hypotheses score each staged pixel with the whole warp per
// hypothesis (warp_best_staged) instead of one lane per hypothesis scanning every mode: the last
// rounds, where a job keeps one or two survivors and the lanes of a chunk would mostly idle.
// Measured on the house batch: faster for 1 and 2 hypotheses (re-fit sums 457 -> 309 us in the
// last round), slower from 4 (the warp pass's shuffle reductions are a dependent chain, while the
// per-lane scan overlaps its independent mode scores).  Both give the same scores and modes.
#ifndef RELO_FEW_HYPS
#define RELO_FEW_HYPS 2
#endif
constexpr int kFewHyps = RELO_FEW_HYPS;

// Round kernels: a CTA takes 32 hypotheses of one job (one per lane) and its warps split the
// pixels, each warp walking every kRoundWarps-th pixel; per-warp partial sums are combined in
// warp order, so the result does not depend on scheduling.
constexpr int kRoundWarps = 8;

// Energies of round r for hypotheses chunk * 32 .. + 31 of job jid.
__device__ __forceinline__ void energy_block(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ alive_prefix,
                                             int r, int chunk, int jid, ModeSlot* slots, float (*part)[32]) {
  const int n_alive = alive_prefix[jid + 1] - alive_prefix[jid];
  if (chunk * 32 >= n_alive) return;
  const RansacJob& job = jobs[jid];
  if (job_skipped(job.skip) || *job.n_valid == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a = chunk * 32 + lane;
  const int h = a < n_alive ? alive_in(job, r)[a] : 0;
  const bool valid = a < n_alive && job.hyp_ok[h];
  const PoseF P = pose_to_float(job.poses + 12 * (size_t)h);
  float sum = 0.f;
  const int4* recs = job.pix + (size_t)r * job.B * job.hs;
  const int n_here = min(32, n_alive - chunk * 32);
  for (int i = warp; i < job.B; i += kRoundWarps) {
    const int4* rec = recs + (size_t)i * job.hs;
    __syncwarp();  // the slot's previous pixel is scored
    const int n_staged = stage_modes(job, rec, slots[warp], lane);
    const float3 x = apply(P, record_point(rec));
    if (n_here <= kFewHyps && n_staged >= 0) {
      for (int j = 0; j < n_here; ++j) {
        const float3 xj = make_float3(__shfl_sync(0xffffffffu, x.x, j), __shfl_sync(0xffffffffu, x.y, j),
                                      __shfl_sync(0xffffffffu, x.z, j));
        float3 mu;
        const float best = warp_best_staged(slots[warp], n_staged, xj, lane, &mu);
        if (lane == j) sum += fminf(kLogEps, -best);
      }
    } else {
      const float best = record_best(job, rec, slots[warp], n_staged, x, nullptr);
      sum += fminf(kLogEps, -best);
    }
  }
  part[warp][lane] = sum;
  __syncthreads();
  if (warp == 0 && valid) {
    float e = 0.f;
#pragma unroll
    for (int w = 0; w < kRoundWarps; ++w) e += part[w][lane];
    job.energy[h] += (double)e;
  }
}

// Energies of round r: grid (hypothesis chunks, jobs).
// CTAs per SM the compiler must fit for the energies, when set (otherwise the compiler's choice:
// 64 registers, four CTAs per SM)
#ifdef RELO_ENERGY_MIN_BLOCKS
#define RELO_ENERGY_BOUNDS __launch_bounds__(kRoundWarps * 32, RELO_ENERGY_MIN_BLOCKS)
#else
#define RELO_ENERGY_BOUNDS __launch_bounds__(kRoundWarps * 32)
#endif
__global__ void RELO_ENERGY_BOUNDS energy_kernel(const RansacJob* __restrict__ jobs,
                                                                  const int32_t* __restrict__ alive_prefix, int r) {
  __shared__ ModeSlot slots[kRoundWarps];
  __shared__ float part[kRoundWarps][32];
  energy_block(jobs, alive_prefix, r, blockIdx.x, blockIdx.y, slots, part);
}
__device__ __forceinline__ unsigned long long order_key(double e) {
  unsigned long long b = (unsigned long long)__double_as_longlong(e);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Halving: CTA per job, bitonic sort of (energy key, index) ascending; keep ceil(n/2).
__device__ __forceinline__ void select_block(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ alive_prefix,
                                             int r, int jid, unsigned long long* skey) {
  const int n = alive_prefix[jid + 1] - alive_prefix[jid];
  if (n == 0) return;
  const RansacJob& job = jobs[jid];
  if (job_skipped(job.skip)) return;
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

__global__ void __launch_bounds__(1024) select_kernel(const RansacJob* __restrict__ jobs,
                                                      const int32_t* __restrict__ alive_prefix, int r) {
  extern __shared__ unsigned long long skey[];
  select_block(jobs, alive_prefix, r, blockIdx.x, skey);
}

// Re-fit sums over all pixels drawn in rounds 0..r: grid (survivor chunks, parts of kRefinePixels
// pixels, jobs).  Sums are taken about a reference correspondence (the first drawn pixel and its
// predicted scene point) so one FP32 pass gives well-conditioned centroids and cross-covariance:
//   refit[h][part] = {n, sum dc (3), sum dw (3), sum dc dw^T (9)},  refit_ref[h] = {c_ref, w_ref}.
// s + e accumulates x: the rounding error of each addition is carried in e (Neumaier 1974), with
// explicitly rounded operations so that no contraction changes the error terms.
__device__ __forceinline__ void comp_add(float& s, float& e, float x) {
  const float t = __fadd_rn(s, x);
  const float err = fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
  e = __fadd_rn(e, err);
  s = t;
}

// Squared distance with explicitly rounded operations, so that every kernel taking the inlier
// decision takes it on the same bits.
__device__ __forceinline__ float dist2_rn(float3 a, float3 b) {
  const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
  return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

__device__ __forceinline__ void refine_block(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ surv_prefix,
                                             int r, int chunk, int part, int jid, ModeSlot* slots,
                                             float (*red)[16][32]) {
  const int n_surv = surv_prefix[jid + 1] - surv_prefix[jid];
  if (chunk * 32 >= n_surv) return;
  const RansacJob& job = jobs[jid];
  const int n_drawn = (r + 1) * job.B;
  const int p0 = part * kRefinePixels;
  if (p0 >= n_drawn || job_skipped(job.skip) || *job.n_valid == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a = chunk * 32 + lane;
  const int h = a < n_surv ? alive_out(job, r)[a] : 0;
  const bool valid = a < n_surv && job.hyp_ok[h];
  const PoseF P = pose_to_float(job.poses + 12 * (size_t)h);
  const float r2 = (float)(job.inlier_dist * job.inlier_dist);
  const float3 cref = record_point(job.pix);
  const float3 wref = apply(P, cref);
  // Each sum is carried as hi + lo in FP32, compensated: products are split exactly into their
  // rounded value and its error (fmaf), and every addition's rounding error is kept (Neumaier's
  // variant of Kahan summation), so the sums hold about twice FP32's precision.  The sums are taken
  // relative to the first drawn pixel; with plain FP32 sums their cancellation against the small
  // spread of a few inliers moved ill-conditioned re-fits by ~1e-4 rad.
  float acc[16], lo[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = lo[q] = 0.f;
  // adds pixel c (its point x under this lane's hypothesis, best mode mean mu) when it is an inlier
  auto add_inlier = [&](float3 c, float3 x, float3 mu) {
    if (dist2_rn(x, mu) < r2) {
      const float u[3] = {c.x - cref.x, c.y - cref.y, c.z - cref.z};
      const float w[3] = {mu.x - wref.x, mu.y - wref.y, mu.z - wref.z};
      acc[0] += 1.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        comp_add(acc[1 + k], lo[1 + k], u[k]);
        comp_add(acc[4 + k], lo[4 + k], w[k]);
      }
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float pr = __fmul_rn(u[p], w[q]);
          comp_add(acc[7 + 3 * p + q], lo[7 + 3 * p + q], pr);
          lo[7 + 3 * p + q] = __fadd_rn(lo[7 + 3 * p + q], __fmaf_rn(u[p], w[q], -pr));
        }
    }
  };
  const int n_here = min(32, n_surv - chunk * 32);
  const int p1 = min(p0 + kRefinePixels, n_drawn);
  for (int i = p0 + warp; i < p1; i += kRoundWarps) {
    const int4* rec = job.pix + (size_t)i * job.hs;
    const float3 c = record_point(rec);
    const float3 x = apply(P, c);
    float3 mu;
    __syncwarp();  // the slot's previous pixel is scored
    const int n_staged = stage_modes(job, rec, slots[warp], lane);
    if (n_here <= kFewHyps && n_staged >= 0) {
      for (int j = 0; j < n_here; ++j) {
        const float3 xj = make_float3(__shfl_sync(0xffffffffu, x.x, j), __shfl_sync(0xffffffffu, x.y, j),
                                      __shfl_sync(0xffffffffu, x.z, j));
        const float best = warp_best_staged(slots[warp], n_staged, xj, lane, &mu);
        if (lane == j && best != -INFINITY) add_inlier(c, x, mu);
      }
    } else {
      const float best = record_best(job, rec, slots[warp], n_staged, x, &mu);
      if (best != -INFINITY) add_inlier(c, x, mu);
    }
  }
  // warps w then write sums q = w, w + kRoundWarps: the kRoundWarps partials added in warp order,
  // compensated as above (first their high parts, then their low parts: one shared buffer, two
  // passes), kept as a (high, low) pair that the re-fit adds in FP64
  constexpr int kPer = (16 + kRoundWarps - 1) / kRoundWarps;
  float sh[kPer], sl[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) sh[i] = sl[i] = 0.f;
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
    for (int q = 0; q < 16; ++q) red[warp][q][lane] = pass ? lo[q] : acc[q];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int q = warp + i * kRoundWarps;
      if (q < 16)
#pragma unroll
        for (int w = 0; w < kRoundWarps; ++w) {
          if (pass == 0) comp_add(sh[i], sl[i], red[w][q][lane]);
          else sl[i] = __fadd_rn(sl[i], red[w][q][lane]);
        }
    }
    __syncthreads();
  }
  if (!valid) return;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int q = warp + i * kRoundWarps;
    if (q < 16) job.refit[((size_t)h * job.refit_parts + part) * 16 + q] = make_float2(sh[i], sl[i]);
  }
  if (part == 0 && warp == 0) {
    float* ref = job.refit_ref + (size_t)h * 8;
    ref[0] = cref.x;
    ref[1] = cref.y;
    ref[2] = cref.z;
    ref[3] = wref.x;
    ref[4] = wref.y;
    ref[5] = wref.z;
  }
}

// CTAs per SM the compiler must fit for the re-fit sums (the 16 compensated sums per lane take
// registers; the fewer a thread holds, the more pixels' loads are in flight per SM)
#ifndef RELO_REFINE_MIN_BLOCKS
#define RELO_REFINE_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(kRoundWarps * 32, RELO_REFINE_MIN_BLOCKS) refine_kernel(const RansacJob* __restrict__ jobs,
                                                                  const int32_t* __restrict__ surv_prefix, int r) {
  __shared__ ModeSlot slots[kRoundWarps];
  __shared__ float red[kRoundWarps][16][32];
  refine_block(jobs, surv_prefix, r, blockIdx.x, blockIdx.y, blockIdx.z, slots, red);
}

// Re-fit sums of rounds whose chunks hold at most kFewHyps hypotheses (the last rounds): the same
// sums as refine_block's, taken with the sixteen sums of hypothesis j spread over lanes 16 j ..
// 16 j + 15 (lane 16 j + q carries sum q) instead of all sixteen in lane j, so a thread holds one
// compensated pair instead of sixteen and more CTAs fit an SM.  Every sum sees the same additions
// in the same order as in refine_block (the pixels of a warp in turn, then the warps in order), so
// the results are identical.
__device__ __forceinline__ void refine_few_block(const RansacJob* __restrict__ jobs,
                                                 const int32_t* __restrict__ surv_prefix, int r, int part, int jid,
                                                 ModeSlot* slots, float (*red)[16][32]) {
  const int n_surv = surv_prefix[jid + 1] - surv_prefix[jid];
  if (n_surv == 0) return;
  const RansacJob& job = jobs[jid];
  const int n_drawn = (r + 1) * job.B;
  const int p0 = part * kRefinePixels;
  if (p0 >= n_drawn || job_skipped(job.skip) || *job.n_valid == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = lane >> 4, q = lane & 15;  // this lane's hypothesis and sum
  const int n_here = min(kFewHyps, n_surv);
  const int h = j < n_here ? alive_out(job, r)[j] : 0;
  const PoseF P = pose_to_float(job.poses + 12 * (size_t)h);
  const float r2 = (float)(job.inlier_dist * job.inlier_dist);
  const float3 cref = record_point(job.pix);
  const float3 wref = apply(P, cref);
  float acc = 0.f, lo = 0.f;
  const int p1 = min(p0 + kRefinePixels, n_drawn);
  for (int i = p0 + warp; i < p1; i += kRoundWarps) {
    const int4* rec = job.pix + (size_t)i * job.hs;
    const float3 c = record_point(rec);
    const float3 x = apply(P, c);  // this lane's hypothesis
    __syncwarp();  // the slot's previous pixel is scored
    const int n_staged = stage_modes(job, rec, slots[warp], lane);
    for (int k = 0; k < n_here; ++k) {
      float best;
      float3 mu = make_float3(0.f, 0.f, 0.f);
      if (n_staged >= 0) {
        const float3 xk = make_float3(__shfl_sync(0xffffffffu, x.x, 16 * k), __shfl_sync(0xffffffffu, x.y, 16 * k),
                                      __shfl_sync(0xffffffffu, x.z, 16 * k));
        best = warp_best_staged(slots[warp], n_staged, xk, lane, &mu);
      } else {
        // more modes than a slot holds: the scan of refine_block's per-lane path, by lane 16 k
        float b = -INFINITY;
        if (lane == 16 * k) b = record_best(job, rec, slots[warp], -1, x, &mu);
        best = __shfl_sync(0xffffffffu, b, 16 * k);
        mu = make_float3(__shfl_sync(0xffffffffu, mu.x, 16 * k), __shfl_sync(0xffffffffu, mu.y, 16 * k),
                         __shfl_sync(0xffffffffu, mu.z, 16 * k));
      }
      if (j == k && best != -INFINITY && dist2_rn(x, mu) < r2) {
        const float u[3] = {c.x - cref.x, c.y - cref.y, c.z - cref.z};
        const float w[3] = {mu.x - wref.x, mu.y - wref.y, mu.z - wref.z};
        if (q == 0) {
          acc += 1.f;
        } else if (q < 4) {
          comp_add(acc, lo, u[q - 1]);
        } else if (q < 7) {
          comp_add(acc, lo, w[q - 4]);
        } else {
          const float a = u[(q - 7) / 3], b = w[(q - 7) % 3];
          const float pr = __fmul_rn(a, b);
          comp_add(acc, lo, pr);
          lo = __fadd_rn(lo, __fmaf_rn(a, b, -pr));
        }
      }
    }
  }
  // the warps' partials combined as in refine_block: sums q = w, w + kRoundWarps of hypothesis
  // `lane` by warp w, added in warp order
  constexpr int kPer = (16 + kRoundWarps - 1) / kRoundWarps;
  float sh[kPer], sl[kPer];
#pragma unroll
  for (int i = 0; i < kPer; ++i) sh[i] = sl[i] = 0.f;
#pragma unroll
  for (int pass = 0; pass < 2; ++pass) {
    if (j < n_here) red[warp][q][j] = pass ? lo : acc;
    __syncthreads();
    if (lane < n_here) {
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int qq = warp + i * kRoundWarps;
        if (qq < 16)
#pragma unroll
          for (int w = 0; w < kRoundWarps; ++w) {
            if (pass == 0) comp_add(sh[i], sl[i], red[w][qq][lane]);
            else sl[i] = __fadd_rn(sl[i], red[w][qq][lane]);
          }
      }
    }
    __syncthreads();
  }
  if (part == 0 && warp == 0 && q == 0 && j < n_here && job.hyp_ok[h]) {
    float* ref = job.refit_ref + (size_t)h * 8;  // written by the hypothesis's first lane
    ref[0] = cref.x;
    ref[1] = cref.y;
    ref[2] = cref.z;
    ref[3] = wref.x;
    ref[4] = wref.y;
    ref[5] = wref.z;
  }
  if (lane >= n_here) return;
  const int hl = alive_out(job, r)[lane];
  if (!job.hyp_ok[hl]) return;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int qq = warp + i * kRoundWarps;
    if (qq < 16) job.refit[((size_t)hl * job.refit_parts + part) * 16 + qq] = make_float2(sh[i], sl[i]);
  }
}

// CTAs per SM for refine_few_kernel (one compensated pair per thread)
#ifndef RELO_REFINE_FEW_MIN_BLOCKS
#define RELO_REFINE_FEW_MIN_BLOCKS 4
#endif
__global__ void __launch_bounds__(kRoundWarps * 32, RELO_REFINE_FEW_MIN_BLOCKS)
    refine_few_kernel(const RansacJob* __restrict__ jobs, const int32_t* __restrict__ surv_prefix, int r) {
  __shared__ ModeSlot slots[kRoundWarps];
  __shared__ float red[kRoundWarps][16][32];
  refine_few_block(jobs, surv_prefix, r, blockIdx.y, blockIdx.z, slots, red);
}

// Re-fit solve: thread per survivor; the parts' sums are added in order in FP64, then FP64 Horn on
// the centroids and cross-covariance (>= 3 inliers, else the pose is kept).  CTAs of one warp take
// `per` survivors each: with few survivors (late rounds) they spread over the SMs, whose FP64 pipes
// would otherwise run one warp's solves in series.
// Re-fit of survivor k of job `job` after round r.
__device__ __forceinline__ void refit_one(const RansacJob& job, int k, int r) {
  if (job_skipped(job.skip)) return;
  const int h = alive_out(job, r)[k];
  if (!job.hyp_ok[h] || *job.n_valid == 0) return;
  const int parts = ((r + 1) * job.B + kRefinePixels - 1) / kRefinePixels;
  double f[16];
  for (int q = 0; q < 16; ++q) f[q] = 0.0;
  for (int p = 0; p < parts; ++p) {
    const float2* src = job.refit + ((size_t)h * job.refit_parts + p) * 16;
    for (int q = 0; q < 16; ++q) f[q] += (double)src[q].x + (double)src[q].y;
  }
  job.inliers[h] = (int)f[0];
  const double n = f[0];
  if (n < 3.0) return;
  const float* ref = job.refit_ref + (size_t)h * 8;
  double mc[3], mw[3], cb[3], wb[3], S[9];
  for (int k = 0; k < 3; ++k) {
    mc[k] = f[1 + k] / n;
    mw[k] = f[4 + k] / n;
    cb[k] = (double)ref[k] + mc[k];
    wb[k] = (double)ref[3 + k] + mw[k];
  }
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) S[3 * p + q] = f[7 + 3 * p + q] - n * mc[p] * mw[q];
  horn_pose(S, cb, wb, job.poses + 12 * (size_t)h);
}

__global__ void __launch_bounds__(32) refit_kernel(const RansacJob* __restrict__ jobs, int n_jobs,
                                                   const int32_t* __restrict__ surv_prefix, int total, int r,
                                                   int per) {
  const int gid = blockIdx.x * per + threadIdx.x;
  if ((int)threadIdx.x >= per || gid >= total) return;
  const int jid = find_job_by(surv_prefix, n_jobs, gid);
  refit_one(jobs[jid], gid - surv_prefix[jid], r);
}

cudaError_t launch_round(const RansacJob* jobs, int n_jobs, int round, const int32_t* alive_prefix_dev,
                         int total_alive, int max_alive, const int32_t* surv_prefix_dev, int total_surv, int max_surv,
                         int B, cudaStream_t s, const Schedule& sched) {
  if (total_alive <= 0) return cudaSuccess;
  if (sched.refit_per < 0 || sched.refit_per > 32) return cudaErrorInvalidValue;
  draw_kernel<<<n_jobs, 256, 0, s>>>(jobs, alive_prefix_dev, round);
  energy_kernel<<<dim3((max_alive + 31) / 32, n_jobs), kRoundWarps * 32, 0, s>>>(jobs, alive_prefix_dev, round);
  // the largest alive set (4096) bounds the shared memory of the sort
  select_kernel<<<n_jobs, 1024, 4096 * (sizeof(unsigned long long) + sizeof(int)), s>>>(jobs, alive_prefix_dev,
                                                                                        round);
  const int parts = ((round + 1) * B + kRefinePixels - 1) / kRefinePixels;
  if (max_surv <= kFewHyps)
    refine_few_kernel<<<dim3(1, parts, n_jobs), kRoundWarps * 32, 0, s>>>(jobs, surv_prefix_dev, round);
  else
    refine_kernel<<<dim3((max_surv + 31) / 32, parts, n_jobs), kRoundWarps * 32, 0, s>>>(jobs, surv_prefix_dev, round);
  int n_sms = 0;
  const cudaError_t e = device_sms(&n_sms);
  if (e != cudaSuccess) return e;
  const int per = sched.refit_per > 0 ? sched.refit_per
                                     : std::max(1, std::min(32, (total_surv + 2 * n_sms - 1) / (2 * n_sms)));
  refit_kernel<<<(unsigned)((total_surv + per - 1) / per), 32, 0, s>>>(jobs, n_jobs, surv_prefix_dev, total_surv,
                                                                       round, per);
  return cudaGetLastError();
}

// Tries of every hypothesis of the job (a kept try j counts j + 1, a failed hypothesis max_tries),
// summed by the 32 lanes of a warp; every lane returns the total.
__device__ __forceinline__ unsigned long long job_tries(const RansacJob& job, int lane) {
  unsigned long long tries = 0;
  for (int q = lane; q < job.K; q += 32)
    tries += job.hyp_ok[q] ? (unsigned long long)job.tries[q] + 1 : job.max_tries;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tries += __shfl_xor_sync(0xffffffffu, tries, o);
  return tries;
}

// Final hypothesis -> result (one thread per job; tries from job_tries).
__device__ __forceinline__ void finalise_one(const RansacJob& job, unsigned long long tries) {
  if (job_skipped(job.skip)) return;
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
  const int32_t up = job.upstream ? *job.upstream : 0;
  res->status = up ? up : (*job.err ? RELO_EDEVICE : (job.hyp_ok[h] ? RELO_OK : RELO_ENOTFOUND));
  res->verified = 0;
  res->n_valid = *job.n_valid;
  res->hypothesis = h;
  res->n_rounds = job.n_rounds;
  res->omega = res->omega_a = res->omega_b = res->omega_ab = res->sum_absdiff_mm = 0;
  res->tries = tries;
  res->path = RELO_PATH_FOREST;
  res->pad = 0;
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

// Warp per job.
__global__ void __launch_bounds__(128) finalise_kernel(const RansacJob* __restrict__ jobs, int n_jobs) {
  const int jid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (jid >= n_jobs) return;
  const RansacJob& job = jobs[jid];
  if (job_skipped(job.skip)) return;
  const unsigned long long tries = job_tries(job, lane);
  if (lane == 0) finalise_one(job, tries);
}

// ---------------------------------------------------------------------------------------------
// One persistent launch for a pass's hypotheses, rounds and results (schedule option).  Warps
// first search hypotheses taken from a counter (as search_kernel); a CTA whose warps find the
// search queue empty then takes items -- (fit | round stage | finalise) x job x chunk -- from a
// host-built list in dependency order.  Before an item runs, one thread waits until the counter of
// the item it depends on (same job) reaches the number of that item's chunks; after it, the CTA
// adds one to its own counter.  An item depends only on items earlier in the list, which threads
// that have started took, so the waits always end -- unless a counter never reaches its target:
// the wait is bounded in time, and one that runs out raises an abort flag that stops every CTA
// (persist_timeout_kernel then reports RELO_ETIMEOUT for the jobs not finalised).  Each item runs
// the same device code as the per-stage kernels, so results are bit-identical.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr int kPersistThreads = kRoundWarps * 32;
static_assert(kPersistThreads == kPersistThreadsHost, "the host's item chunks match the CTA size");
constexpr size_t kPersistSmem = 4096 * (sizeof(unsigned long long) + sizeof(int));  // the largest sort
static_assert(kRoundWarps * sizeof(ModeSlot) + sizeof(float) * kRoundWarps * 16 * 32 <= kPersistSmem,
              "round stages fit the persistent kernel's shared memory");

__global__ void __launch_bounds__(kPersistThreads, 2) persistent_kernel(PersistArgs a) {
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ int s_item, s_go;
  const int lane = threadIdx.x & 31;
  volatile int32_t* abort = a.ctrl + 2;
  // phase 1: hypothesis search, one warp per hypothesis
  for (;;) {
    int gw = 0;
    if (lane == 0) gw = *abort ? a.total_hyps : atomicAdd(a.ctrl + 0, 1);
    gw = __shfl_sync(0xffffffffu, gw, 0);
    if (gw >= a.total_hyps) break;
    const int jid = search_one(a.jobs, a.n_jobs, gw, lane);
    __threadfence();
    __syncwarp();
    if (lane == 0) atomicAdd(a.done + jid, 1);
  }
  __syncthreads();
  // phase 2: CTA items
  ModeSlot* slots = reinterpret_cast<ModeSlot*>(psm);
  float(*part)[32] = reinterpret_cast<float(*)[32]>(psm + kRoundWarps * sizeof(ModeSlot));
  float(*red)[16][32] = reinterpret_cast<float(*)[16][32]>(psm + kRoundWarps * sizeof(ModeSlot));
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(a.ctrl + 1, 1);
      int go = it < a.n_items && !*abort;
      if (go) {
        const PItem pi = a.items[it];
        const unsigned long long t0 = global_ns();
        for (unsigned n = 1; ld_acquire_gpu(a.done + pi.dep) < pi.need; ++n) {
          if ((n & 63) == 0) {
            if (*abort) {
              go = 0;
              break;
            }
            if (global_ns() - t0 > a.timeout_ns) {
              atomicExch(a.ctrl + 2, 1);
              go = 0;
              break;
            }
          }
        }
      }
      s_item = it;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    __threadfence();
    const PItem it = a.items[s_item];
    const RansacJob& job = a.jobs[it.job];
    const int np = a.n_jobs + 1;
    switch (it.kind) {
      case kItemFit: {
        const int h = it.sub * kPersistThreads + threadIdx.x;
        if (h < job.K && !job_skipped(job.skip)) fit_one(job, h);
        break;
      }
      case kItemDraw:
        draw_block(a.jobs, a.alive_prefix + (size_t)it.round * np, it.round, it.job);
        break;
      case kItemEnergy:
        energy_block(a.jobs, a.alive_prefix + (size_t)it.round * np, it.round, it.sub, it.job, slots, part);
        break;
      case kItemSelect:
        select_block(a.jobs, a.alive_prefix + (size_t)it.round * np, it.round, it.job,
                     reinterpret_cast<unsigned long long*>(psm));
        break;
      case kItemRefine:
        refine_block(a.jobs, a.surv_prefix + (size_t)it.round * np, it.round, it.sub, it.part, it.job, slots, red);
        break;
      case kItemRefit: {
        const int32_t* sp = a.surv_prefix + (size_t)it.round * np;
        const int k = it.sub * kPersistThreads + threadIdx.x;
        if (k < sp[it.job + 1] - sp[it.job]) refit_one(job, k, it.round);
        break;
      }
      default:
        if (threadIdx.x < 32 && !job_skipped(job.skip)) {
          const unsigned long long tries = job_tries(job, threadIdx.x);
          if (threadIdx.x == 0) finalise_one(job, tries);
        }
        break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(a.done + it.done, 1);
  }
}

// After an aborted persistent launch: the jobs it did not finalise report RELO_ETIMEOUT.
__global__ void persist_timeout_kernel(const RansacJob* __restrict__ jobs, int n_jobs, const int32_t* __restrict__ ctrl,
                                       const int32_t* __restrict__ final_done) {
  const int jid = blockIdx.x * blockDim.x + threadIdx.x;
  if (jid >= n_jobs || !ctrl[2]) return;
  const RansacJob& job = jobs[jid];
  if (job_skipped(job.skip) || final_done[jid] != 0) return;
  job.result->status = RELO_ETIMEOUT;
  job.result->verified = 0;
}

// The persistent kernel's CTAs: as many as are resident on the device at once (its shared-memory
// limit is raised here, once per device; batches call this when they are prepared, so that a
// launch inside a stream capture finds it done).
cudaError_t persistent_grid(int* grid) {
  static PerDevice resident;  // resident persistent CTAs per SM on each device
  int sms = 0, per_sm = 0;
  cudaError_t e = device_sms(&sms);
  if (e == cudaSuccess)
    e = per_device(resident, &per_sm, [](int, int* v) {
      cudaError_t r = cudaFuncSetAttribute(persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kPersistSmem);
      if (r == cudaSuccess)
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, persistent_kernel, kPersistThreads, kPersistSmem);
      *v = std::max(1, *v);
      return r;
    });
  *grid = sms * per_sm;
  return e;
}

cudaError_t launch_persistent(const PersistArgs& a, int ctrl_words, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.ctrl, 0, (size_t)ctrl_words * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  int grid = 0;
  e = persistent_grid(&grid);
  if (e != cudaSuccess) return e;
  persistent_kernel<<<grid, kPersistThreads, kPersistSmem, s>>>(a);
  persist_timeout_kernel<<<(a.n_jobs + 127) / 128, 128, 0, s>>>(a.jobs, a.n_jobs, a.ctrl, a.done + a.final_base);
  return cudaGetLastError();
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
  if (jid >= n_jobs || job_skipped(jobs[jid].skip)) return;
  // a bound failure in the verification raycast (it reports into the job's word) voids the result
  if (jobs[jid].err && *jobs[jid].err) jobs[jid].result->status = RELO_EDEVICE;
  decide(jobs[jid].result, (unsigned long long)jobs[jid].vW * jobs[jid].vH);
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
  if (n_jobs <= 0) return cudaSuccess;
  finalise_kernel<<<(n_jobs + 3) / 4, 128, 0, s>>>(jobs, n_jobs);
  return cudaGetLastError();
}

// Fallback results start as "not run" (a skipped job writes nothing).
__global__ void init_results_kernel(relo_pose_result* res, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  res[i].status = RELO_ENOTFOUND;
  res[i].verified = 0;
}

cudaError_t launch_init_results(relo_pose_result* res, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  init_results_kernel<<<(n + 127) / 128, 128, 0, s>>>(res, n);
  return cudaGetLastError();
}

// kind[i]: 0 forest only (fallback[i] holds the result), 1 learned without forest, 2 learned with
// a forest fallback.  A learned attempt keeps its learned result when it verified.
__global__ void merge_results_kernel(const relo_pose_result* learned, const relo_pose_result* fallback,
                                     const int32_t* kind, int n, relo_pose_result* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = kind[i];
  if (k == 0) {
    out[i] = fallback[i];
    out[i].path = RELO_PATH_FOREST;
  } else if (k == 1 || learned[i].verified) {
    out[i] = learned[i];
    out[i].path = RELO_PATH_LEARNED;
  } else {
    out[i] = fallback[i];
    out[i].path = RELO_PATH_FALLBACK;
  }
}

cudaError_t launch_merge_results(const relo_pose_result* learned, const relo_pose_result* fallback,
                                 const int32_t* kind, int n, relo_pose_result* out, cudaStream_t s) {
  merge_results_kernel<<<(n + 127) / 128, 128, 0, s>>>(learned, fallback, kind, n, out);
  return cudaGetLastError();
}

RELO_DEFINE_CHECK_READER(check_failures_ransac)

}  // namespace relo
