// forest.cu -- regression-forest evaluation and relocaliser training kernels.
//
// Sec. 3.3 (b): each agent's relocaliser is a scene-coordinate regression forest trained online
// as per Cavallari et al.; Sec. 3.3.1: a query view is evaluated through another agent's forest.
// The split-node features (depth-adaptive pixel-pair differences, integer form), the leaf
// reservoirs and mean-shift modes are the library's readings of that paper-silent relocaliser.
#include <cuda_runtime.h>
#include <stdint.h>

#include "relo_internal.cuh"

namespace relo {

// Offsets are pixel-metres: probe = x + trunc(delta * 1000 / d), integer division toward zero.
// The division by the pixel's depth d uses one multiply-shift per probe: for 0 <= a < 2^25 and
// 1 <= d < 2^16, floor(a / d) = (a * M) >> (25 + l) with l = ceil(log2 d) and
// M = floor(2^(25+l) / d) + 1 (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, round-up method); |delta| * 1000 <= 32768000 < 2^25.  Since
// 2^(l-1) < d, M <= 2^26 + 1 fits in 32 bits and the product is one 32 x 32 -> 64-bit multiply.
struct DepthDivisor {
  uint32_t M;
  int shift;
};

__device__ __forceinline__ DepthDivisor make_divisor(int d) {
  const int l = d > 1 ? 32 - __clz(d - 1) : 0;
  DepthDivisor q;
  q.shift = 25 + l;
  q.M = (uint32_t)((1ull << q.shift) / (unsigned long long)d + 1ull);
  return q;
}

// Offsets stored times 128 (every |delta| <= 255, ForestView::offset_shift = 7) and d >= 16:
// trunc(delta * 1000 / d) = mulhi(128 delta, M7) + [delta < 0] with M7 = floor(2^25 * 1000 / d) + 1,
// the same round-up method with the factor 1000 folded into the multiplier.  With e = M7 -
// 2^25 * 1000 / d in (0, 1], 128 delta M7 / 2^32 = delta * 1000 / d + 128 delta e / 2^32.  Since
// |delta| d <= 255 * 65535 < 2^25, the added term is below 1/d in magnitude, and 1/d is the
// smallest distance from a non-integer delta * 1000 / d to the next integer: for delta >= 0 the
// floor is the quotient; for delta < 0 the term pushes the value just below -q, so the floor is
// one less than the truncation.  d >= 16 keeps M7 below 2^31 (a positive signed multiplier).
// Checked exhaustively for every d in [16, 65535] and |delta| <= 255 (tests/test_probe_division.py).
__device__ __forceinline__ DepthDivisor make_divisor7(int d) {
  DepthDivisor q;
  q.shift = 0;
  q.M = (uint32_t)((1000ull << 25) / (unsigned long long)d + 1ull);
  return q;
}

// kDiv == 1: the shift is >= 32 (every depth d >= 65 mm).  Then trunc(n / d) for a signed n is
// floor(n M / 2^shift) + [n < 0]: the high word of the signed product shifted arithmetically by
// shift - 32, plus the sign bit.  (For n < 0, n M / 2^shift = -(q + r/d + |n| e / 2^shift) with
// 0 < r/d + |n| e / 2^shift < 1, e = M - 2^shift / d, since |n| < 2^25 and 2^-l <= 1/d; checked
// exhaustively for every d in [65, 65535] and every int16 offset.)  Otherwise the full 64-bit
// product of |n| is shifted and the sign restored.
// kClamp = false: the caller has shown that x + q stays in [0, limit] for every node (the pixel is
// at least the forest's probe reach away from the image edges), so no clamp is needed.
// kDiv: 2 = the shifted-offset form above (raw = 128 delta); 1 = kHi, 0 = the 64-bit product
// (raw = delta << oshift).
template <int kDiv, bool kClamp = true>
__device__ __forceinline__ int probe(int x, int raw, const DepthDivisor& dv, int limit, int oshift) {
  if (kDiv == 2) {
    const int q = __mulhi(raw, (int)dv.M) - (raw >> 31);
    return kClamp ? min(max(x + q, 0), limit) : x + q;
  }
  const int n = (raw >> oshift) * 1000;
  int q;
  if (kDiv == 1) {
    q = (__mulhi(n, (int)dv.M) >> (dv.shift - 32)) - (n >> 31);
  } else {
    const unsigned a = (unsigned)(n < 0 ? -n : n);
    const int m = (int)(((unsigned long long)a * (unsigned long long)dv.M) >> dv.shift);
    q = n < 0 ? -m : m;
  }
  return kClamp ? min(max(x + q, 0), limit) : x + q;
}

// Descends pixel (u, v) of depth d through the trees, interleaved level by level so each level
// issues T independent node loads instead of a chain of T * D dependent ones.  In the device copy
// of the forest (relo_create_forest) a node's third word holds the mask of a probe's value (0xFFFF
// for depth, 0xFF for a colour channel) and the bit offsets of its two probes' values in a packed
// pixel (0 for depth, 16 + 8 c for colour channel c), ready to use.
// kPacked: probes read the packed image (one 64-bit load, then a shift and a mask: no branch on
// the node's kind, which differs between neighbouring lanes); otherwise the depth or the colour
// image, by kind.
// The CTA's shared-memory copy of the top levels of its forest's trees ([T][2^levels - 1]).
extern __shared__ int4 s_forest_top[];

// Levels [level_begin, level_end) with nodes from the forest in global memory, or (kShared) from
// s_forest_top, which holds n_nodes of each tree.
template <int MT, int kDiv, bool kPacked, bool kShared, bool kClamp>
__device__ __forceinline__ void descend_levels(const ForestJob& job, int u, int v, const DepthDivisor& dv,
                                               int (&node)[MT], int n_nodes, int level_begin, int level_end) {
  const int T = job.forest.T, W = job.W, H = job.H, os = job.forest.offset_shift;
  for (int level = level_begin; level < level_end; ++level) {
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      if (t < T) {
        int4 nd = make_int4(0, 0, 0, 0);
        if (RELO_CHECK(node[t] >= 0 && node[t] < n_nodes))
          nd = kShared ? s_forest_top[t * n_nodes + node[t]] : __ldg(&job.forest.nodes[(size_t)t * n_nodes + node[t]]);
        const int dx1 = (int)(int16_t)(nd.x & 0xFFFF), dy1 = nd.x >> 16;
        const int dx2 = (int)(int16_t)(nd.y & 0xFFFF), dy2 = nd.y >> 16;
        const int q1 = probe<kDiv, kClamp>(v, dy1, dv, H - 1, os) * W + probe<kDiv, kClamp>(u, dx1, dv, W - 1, os);
        const int q2 = probe<kDiv, kClamp>(v, dy2, dv, H - 1, os) * W + probe<kDiv, kClamp>(u, dx2, dv, W - 1, os);
        int a, b;
        if (!RELO_CHECK((unsigned)q1 < (unsigned)(W * H) && (unsigned)q2 < (unsigned)(W * H))) {
          node[t] = 2 * node[t] + 1;
          continue;
        }
        if (kPacked) {
          const unsigned mask = (unsigned)nd.z & 0xFFFFu, s1 = ((unsigned)nd.z >> 16) & 0xFFu, s2 = (unsigned)nd.z >> 24;
          const uint2 p1 = __ldg(&job.packed[q1]), p2 = __ldg(&job.packed[q2]);
          a = (int)(__funnelshift_rc(p1.x, p1.y, s1) & mask);
          b = (int)(__funnelshift_rc(p2.x, p2.y, s2) & mask);
        } else if ((nd.z & 0xFFFF) == 0xFFFF) {
          a = __ldg(&job.depth[q1]);
          b = __ldg(&job.depth[q2]);
        } else {
          a = (__ldg(&job.rgba[q1]) >> ((((unsigned)nd.z >> 16) & 0xFFu) - 16)) & 0xFF;
          b = (__ldg(&job.rgba[q2]) >> (((unsigned)nd.z >> 24) - 16)) & 0xFF;
        }
        node[t] = 2 * node[t] + ((a - b < nd.w) ? 1 : 2);
      }
    }
  }
}

// The first top_levels levels from s_forest_top, the rest from global memory.
template <int MT, int kDiv, bool kPacked, bool kClamp>
__device__ __forceinline__ void descend(const ForestJob& job, int u, int v, const DepthDivisor& dv, int (&node)[MT],
                                        int top_levels) {
  if (top_levels > 0)
    descend_levels<MT, kDiv, kPacked, true, kClamp>(job, u, v, dv, node, (1 << top_levels) - 1, 0, top_levels);
  descend_levels<MT, kDiv, kPacked, false, kClamp>(job, u, v, dv, node, (1 << job.forest.D) - 1, top_levels,
                                                   job.forest.D);
}

// Descent with or without probe clamping: a warp whose pixels all lie at least the forest's probe
// reach trunc((max |offset|) * 1000 / d) from every image edge takes the clamp-free instance (its
// probes cannot leave the image, so both give the same leaves); any other warp clamps.  Instances
// for more than 6 trees always clamp (a second copy of their descent would spill registers).
template <int MT, int kDiv, bool kPacked>
__device__ __forceinline__ void descend_any(const ForestJob& job, int u, int v, int d, const DepthDivisor& dv,
                                            int (&node)[MT], int top_levels) {
  bool inside = false;
  if (MT <= 6 && job.forest.probe_reach > 0) {
    const int reach = (int)(((long long)(job.forest.probe_reach - 1) * 1000) / d);
    inside = u >= reach && u + reach <= job.W - 1 && v >= reach && v + reach <= job.H - 1;
  }
  if (MT <= 6 && __all_sync(__activemask(), inside)) descend<MT, kDiv, kPacked, false>(job, u, v, dv, node, top_levels);
  else descend<MT, kDiv, kPacked, true>(job, u, v, dv, node, top_levels);
}

// CTAs of 256 threads per SM the compiler must fit: full occupancy (7 and 8 tie, 6 is 10 % slower
// on the house workload)
#ifndef RELO_FOREST_MIN_BLOCKS
#define RELO_FOREST_MIN_BLOCKS 8
#endif

// One thread per pixel.  tiles == 0: a job's slot k is its pixel k (row-major); tiles == 1: its
// slots run over 32 x 8 pixel tiles, 256 slots each, tiles row-major (neighbouring threads
// probe neighbouring pixels in two dimensions).
// levels > 0: the CTA first copies the top min(levels, D) levels of its job's trees into shared
// memory (dynamic, top_trees x (2^levels - 1) nodes), so those node visits read shared memory.
template <int MT>
__global__ void __launch_bounds__(256, RELO_FOREST_MIN_BLOCKS)
    forest_kernel(const ForestJob* __restrict__ jobs, int n_jobs, const ForestJob single, int tiles, int levels,
                  int top_trees) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // jobs start on multiples of the CTA size, so the CTA's first pixel names its job; the job is
  // staged in shared memory (its fields are read at every node visit)
  const int64_t first = (int64_t)blockIdx.x * blockDim.x;
  int lo = 0, hi = n_jobs - 1;
  while (jobs && lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].pixel_begin <= first) lo = mid;
    else hi = mid - 1;
  }
  __shared__ __align__(16) ForestJob sj;
  if (jobs) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(jobs + lo);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sj);
    for (int i = threadIdx.x; i < (int)(sizeof(ForestJob) / 8); i += blockDim.x) dst[i] = src[i];
  } else if (threadIdx.x == 0) {
    sj = single;
  }
  __syncthreads();
  const ForestJob& job = sj;
  if (job_skipped(job.skip)) return;
  // s_forest_top holds top_trees trees of 2^levels - 1 nodes
  const int top_levels = job.forest.T <= top_trees ? min(levels, job.forest.D) : 0;
  if (top_levels > 0) {
    const int n_top = (1 << top_levels) - 1, n_int = (1 << job.forest.D) - 1;
    for (int i = threadIdx.x; i < job.forest.T * n_top; i += blockDim.x) {
      const int t = i / n_top;
      s_forest_top[i] = __ldg(&job.forest.nodes[(size_t)t * n_int + (i - t * n_top)]);
    }
    __syncthreads();
  }
  const int64_t slot = gid - job.pixel_begin;
  const int64_t n_pix = (int64_t)job.W * job.H;
  const int W = job.W, H = job.H;
  int u, v;
  if (tiles) {
    const int64_t t = slot >> 8;
    const int i = (int)(slot & 255), tx = (W + 31) >> 5;
    u = (int)(t % tx) * 32 + (i & 31);
    v = (int)(t / tx) * 8 + (i >> 5);
    if (slot < 0 || u >= W || v >= H) return;
  } else {
    if (slot < 0 || slot >= n_pix) return;
    u = (int)(slot % W);
    v = (int)(slot / W);
  }
  const int64_t pix = (int64_t)v * W + u;
  const ForestView& f = job.forest;
  const int T = f.T;
  const int d = __ldg(&job.depth[pix]);
  if (d == 0) {
    for (int t = 0; t < T; ++t) job.leaves[(size_t)t * n_pix + pix] = 0xFFFF;
    return;
  }
  const int n_int = (1 << f.D) - 1;
  int node[MT];
#pragma unroll
  for (int t = 0; t < MT; ++t) node[t] = 0;
  if (f.offset_shift == 7 && d >= 16) {
    const DepthDivisor dv = make_divisor7(d);
    if (job.packed) descend_any<MT, 2, true>(job, u, v, d, dv, node, top_levels);
    else descend_any<MT, 2, false>(job, u, v, d, dv, node, top_levels);
  } else {
    const DepthDivisor dv = make_divisor(d);
    if (job.packed) {
      if (dv.shift >= 32) descend_any<MT, 1, true>(job, u, v, d, dv, node, top_levels);
      else descend_any<MT, 0, true>(job, u, v, d, dv, node, top_levels);
    } else {
      if (dv.shift >= 32) descend_any<MT, 1, false>(job, u, v, d, dv, node, top_levels);
      else descend_any<MT, 0, false>(job, u, v, d, dv, node, top_levels);
    }
  }
#pragma unroll
  for (int t = 0; t < MT; ++t)
    if (t < T && RELO_CHECK(node[t] >= n_int && node[t] < 2 * n_int + 1))
      job.leaves[(size_t)t * n_pix + pix] = (uint16_t)(node[t] - n_int);
}

RELO_DEFINE_CHECK_READER(check_failures_forest)

cudaError_t launch_forest(const ForestJob* jobs_dev, int n_jobs, const ForestJob* single, int64_t total_pixels,
                          cudaStream_t s, int max_trees, const Schedule& sched) {
  if (total_pixels <= 0) return cudaSuccess;
  const int threads = sched.forest_threads;
  if ((threads != 128 && threads != 256) || (sched.forest_tiles != 0 && sched.forest_tiles != 1) ||
      sched.forest_smem_levels < 0 || sched.forest_smem_levels > kMaxSmemLevels)
    return cudaErrorInvalidValue;
  ForestJob one{};
  if (single) one = *single;
  // total_pixels counts each job's slots, a multiple of 256 (pixel_begin), so no CTA spans two jobs
  const unsigned grid = (unsigned)((total_pixels + threads - 1) / threads);
  const int tiles = sched.forest_tiles;
  // the unrolled width: the smallest instance that holds every job's trees (5, the usual forest
  // size, has its own: no idle unrolled slots, no spills at 32 registers)
  const int mt = max_trees <= 4 ? 4 : max_trees <= 5 ? 5 : max_trees <= 6 ? 6 : max_trees <= 8 ? 8 : kMaxTrees;
  // the staged levels take at most 48 KB of shared memory per CTA (fewer levels for many trees)
  const size_t trees = (size_t)max(1, min(max_trees, mt));
  int levels = sched.forest_smem_levels;
  while (levels > 0 && trees * ((1u << levels) - 1) * sizeof(int4) > 48 * 1024) --levels;
  const size_t smem = levels > 0 ? trees * ((1u << levels) - 1) * sizeof(int4) : 0;
  if (mt == 4) forest_kernel<4><<<grid, threads, smem, s>>>(jobs_dev, n_jobs, one, tiles, levels, (int)trees);
  else if (mt == 5) forest_kernel<5><<<grid, threads, smem, s>>>(jobs_dev, n_jobs, one, tiles, levels, (int)trees);
  else if (mt == 6) forest_kernel<6><<<grid, threads, smem, s>>>(jobs_dev, n_jobs, one, tiles, levels, (int)trees);
  else if (mt == 8) forest_kernel<8><<<grid, threads, smem, s>>>(jobs_dev, n_jobs, one, tiles, levels, (int)trees);
  else forest_kernel<kMaxTrees><<<grid, threads, smem, s>>>(jobs_dev, n_jobs, one, tiles, levels, (int)trees);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Training: scene coordinates of the stride-grid pixels, FP64 rounded to float32 (the values
// the reservoirs store).  out[(v/stride) * ceil(W/stride) + u/stride] = P * backproject(d).
// ---------------------------------------------------------------------------------------------
struct Pose16 {
  double p[16];
};

__global__ void scene_coords_kernel(const uint16_t* __restrict__ depth, int W, int H, int stride, double fx,
                                    double fy, double cx, double cy, Pose16 P, float* __restrict__ out) {
  const int gw = (W + stride - 1) / stride, gh = (H + stride - 1) / stride;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= gw * gh) return;
  const int u = (i % gw) * stride, v = (i / gw) * stride;
  const int d = depth[(size_t)v * W + u];
  float* o = out + 3 * (size_t)i;
  if (d == 0) {
    o[0] = o[1] = o[2] = 0.f;
    return;
  }
  // explicit rounding steps: no contraction, the same operation order as a plain C evaluation
  const double z = __ddiv_rn((double)d, 1000.0);
  const double c0 = __ddiv_rn(__dmul_rn(z, __dsub_rn((double)u, cx)), fx);
  const double c1 = __ddiv_rn(__dmul_rn(z, __dsub_rn((double)v, cy)), fy);
  for (int k = 0; k < 3; ++k) {
    const double w = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(P.p[4 * k], c0), __dmul_rn(P.p[4 * k + 1], c1)),
                                         __dmul_rn(P.p[4 * k + 2], z)),
                               P.p[4 * k + 3]);
    o[k] = (float)w;
  }
}

cudaError_t launch_scene_coords(const uint16_t* depth, int W, int H, int stride, double fx, double fy, double cx,
                                double cy, const double* P, float* out, cudaStream_t s) {
  Pose16 p;
  for (int k = 0; k < 16; ++k) p.p[k] = P[k];
  const int n = ((W + stride - 1) / stride) * ((H + stride - 1) / stride);
  scene_coords_kernel<<<(n + 255) / 256, 256, 0, s>>>(depth, W, H, stride, fx, fy, cx, cy, p, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Mean shift, one CTA per leaf.  Ascents run in FP32 from every sample (one seed per thread
// at a time, samples broadcast from shared memory); the merge, ranking and per-mode statistics
// follow in seed order, the statistics in FP64.
// ---------------------------------------------------------------------------------------------
constexpr int kMsThreads = 128;

__global__ void __launch_bounds__(kMsThreads)
    mean_shift_kernel(const float* __restrict__ samples, const int32_t* __restrict__ count, int capacity,
                      float bandwidth, float tol, int max_iter, float merge_dist, float cov_floor, int max_modes,
                      float* __restrict__ modes, uint8_t* __restrict__ n_modes_out) {
  extern __shared__ float sm[];
  const int leaf = blockIdx.x;
  const int n = count[leaf];
  float* xs = sm;                           // [cap][3]
  float* zs = sm + 3 * capacity;            // [cap][3] converged points
  int* member = (int*)(zs + 3 * capacity);  // [cap]
  int* support = member + capacity;         // [cap]
  int* rank = support + capacity;           // [cap]
  __shared__ int s_modes;
  const float* src = samples + (size_t)leaf * capacity * 3;
  for (int i = threadIdx.x; i < 3 * n; i += blockDim.x) xs[i] = src[i];
  __syncthreads();
  const float inv2h2 = 1.0f / (2.0f * bandwidth * bandwidth);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float y0 = xs[3 * i], y1 = xs[3 * i + 1], y2 = xs[3 * i + 2];
    for (int it = 0; it < max_iter; ++it) {
      float n0 = 0.f, n1 = 0.f, n2 = 0.f, den = 0.f;
      for (int j = 0; j < n; ++j) {
        const float a = y0 - xs[3 * j], b = y1 - xs[3 * j + 1], c = y2 - xs[3 * j + 2];
        const float k = expf(-(a * a + b * b + c * c) * inv2h2);
        n0 += k * xs[3 * j];
        n1 += k * xs[3 * j + 1];
        n2 += k * xs[3 * j + 2];
        den += k;
      }
      const float m0 = n0 / den, m1 = n1 / den, m2 = n2 / den;
      const float sh = sqrtf((m0 - y0) * (m0 - y0) + (m1 - y1) * (m1 - y1) + (m2 - y2) * (m2 - y2));
      y0 = m0;
      y1 = m1;
      y2 = m2;
      if (sh < tol) break;
    }
    zs[3 * i] = y0;
    zs[3 * i + 1] = y1;
    zs[3 * i + 2] = y2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // merge in seed order: a converged point joins the first mode opened within merge_dist
    int nm = 0;
    for (int i = 0; i < n; ++i) {
      int found = -1;
      for (int m = 0; m < nm; ++m) {
        const int o = rank[m];  // rank[] temporarily holds the opening seed of each mode
        const float a = zs[3 * i] - zs[3 * o], b = zs[3 * i + 1] - zs[3 * o + 1], c = zs[3 * i + 2] - zs[3 * o + 2];
        if (sqrtf(a * a + b * b + c * c) < merge_dist) {
          found = m;
          break;
        }
      }
      if (found < 0) {
        found = nm;
        rank[nm] = i;
        support[nm] = 0;
        ++nm;
      }
      member[i] = found;
      support[found]++;
    }
    // rank by support, descending; stable for ties (opening order)
    for (int m = 0; m < nm; ++m) rank[m] = m;
    for (int a = 1; a < nm; ++a) {
      const int v = rank[a];
      int b = a - 1;
      while (b >= 0 && support[rank[b]] < support[v]) {
        rank[b + 1] = rank[b];
        --b;
      }
      rank[b + 1] = v;
    }
    s_modes = nm < max_modes ? nm : max_modes;
    n_modes_out[leaf] = (uint8_t)s_modes;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s_modes; q += blockDim.x) {
    const int m = rank[q];
    double mean[3] = {0, 0, 0};
    int cnt = 0;
    for (int i = 0; i < n; ++i)
      if (member[i] == m) {
        mean[0] += xs[3 * i];
        mean[1] += xs[3 * i + 1];
        mean[2] += xs[3 * i + 2];
        ++cnt;
      }
    for (int k = 0; k < 3; ++k) mean[k] /= cnt;
    double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < n; ++i)
      if (member[i] == m) {
        const double e[3] = {xs[3 * i] - mean[0], xs[3 * i + 1] - mean[1], xs[3 * i + 2] - mean[2]};
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) S[3 * a + b] += e[a] * e[b];
      }
    for (int k = 0; k < 9; ++k) S[k] /= cnt;
    S[0] += cov_floor;
    S[4] += cov_floor;
    S[8] += cov_floor;
    const double det = S[0] * (S[4] * S[8] - S[5] * S[7]) - S[1] * (S[3] * S[8] - S[5] * S[6]) +
                       S[2] * (S[3] * S[7] - S[4] * S[6]);
    const double weight = (double)cnt / n;
    const double two_pi = 6.283185307179586;
    float* o = modes + ((size_t)leaf * max_modes + q) * kModeFloats;
    o[0] = (float)mean[0];
    o[1] = (float)mean[1];
    o[2] = (float)mean[2];
    o[3] = (float)((S[4] * S[8] - S[5] * S[7]) / det);
    o[4] = (float)((S[2] * S[7] - S[1] * S[8]) / det);
    o[5] = (float)((S[1] * S[5] - S[2] * S[4]) / det);
    o[6] = (float)((S[0] * S[8] - S[2] * S[6]) / det);
    o[7] = (float)((S[2] * S[3] - S[0] * S[5]) / det);
    o[8] = (float)((S[0] * S[4] - S[1] * S[3]) / det);
    o[9] = (float)(log(weight) - 0.5 * log(two_pi * two_pi * two_pi * det));
    o[10] = (float)weight;
    o[11] = 0.f;
  }
}

cudaError_t launch_mean_shift(const float* samples, const int32_t* count, int capacity, int n_leaves_total,
                              float bandwidth, float tol, int max_iter, float merge_dist, float cov_floor,
                              int max_modes, float* modes, uint8_t* n_modes, cudaStream_t s) {
  const size_t smem = (size_t)capacity * (6 * sizeof(float) + 3 * sizeof(int));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(mean_shift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  mean_shift_kernel<<<n_leaves_total, kMsThreads, smem, s>>>(samples, count, capacity, bandwidth, tol, max_iter,
                                                            merge_dist, cov_floor, max_modes, modes, n_modes);
  return cudaGetLastError();
}

__global__ void top_modes_kernel(const float* __restrict__ modes, const uint8_t* __restrict__ n_modes, int n,
                                 int max_modes, float4* __restrict__ top) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* m = modes + (size_t)i * max_modes * kModeFloats;
  top[i] = make_float4(m[0], m[1], m[2], (float)n_modes[i]);
}

cudaError_t launch_top_modes(const float* modes, const uint8_t* n_modes, int n_leaves_total, int max_modes,
                             float4* top, cudaStream_t s) {
  top_modes_kernel<<<(n_leaves_total + 255) / 256, 256, 0, s>>>(modes, n_modes, n_leaves_total, max_modes, top);
  return cudaGetLastError();
}

}  // namespace relo
