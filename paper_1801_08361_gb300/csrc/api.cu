// api.cu -- the C ABI (include/relo.h): handle management, argument checks, workspace layout and
// the launch sequence of one relocalisation attempt / a batch of attempts (Sec. 3.3.1, Fig. 3).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "regressor.cuh"
#include "relo_internal.cuh"

using namespace relo;

static_assert(sizeof(relo_pose_result) == 344, "relo_pose_result layout is part of the ABI");
static_assert(sizeof(relo_attempt) == 240, "relo_attempt layout is part of the ABI");
static_assert(sizeof(relo_intrinsics) == 56, "relo_intrinsics layout is part of the ABI");

namespace relo {
std::atomic<int> g_fail_allocations{0};
// test hooks of the tcgen05 convolution (relo_debug_conv_path / relo_debug_conv_stall)
std::atomic<bool> g_conv_tcgen05{true};
std::atomic<int> g_conv_stall_tile{-1};
std::atomic<unsigned long long> g_conv_timeout_ns{2000000000ull};
// test hooks of the persistent RANSAC launch (relo_debug_persistent_stall)
std::atomic<bool> g_persist_stall{false};
std::atomic<unsigned long long> g_persist_timeout_ns{2000000000ull};

// The caller's allocator (relo_set_allocator), and every block it gave the library, with the
// functions that gave it: a block goes back to those even after the allocator has changed.
struct Allocator {
  relo_alloc_fn alloc = nullptr;
  relo_free_fn free = nullptr;
  void* ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;
std::unordered_map<void*, Allocator> g_alloc_owned;

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  int n = g_fail_allocations.load();
  while (n > 0) {
    if (g_fail_allocations.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
  }
  Allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (!a.alloc) return cudaMalloc(p, bytes);
  if (bytes == 0) return cudaSuccess;
  void* q = a.alloc(bytes, a.ctx);
  if (!q) return cudaErrorMemoryAllocation;
  if (((uintptr_t)q & 255) != 0) {
    a.free(q, a.ctx);
    return cudaErrorMemoryAllocation;
  }
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc_owned[q] = a;
  }
  *p = q;
  return cudaSuccess;
}

void dev_free(void* p) {
  if (!p) return;
  Allocator a;
  bool theirs = false;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_alloc_owned.find(p);
    if (it != g_alloc_owned.end()) {
      a = it->second;
      g_alloc_owned.erase(it);
      theirs = true;
    }
  }
  if (!theirs) {
    cudaFree(p);
    return;
  }
  cudaDeviceSynchronize();  // as cudaFree does: no launch may still use the block
  a.free(p, a.ctx);
}
}  // namespace relo

namespace {

thread_local std::string g_error;

relo_status fail(relo_status code, const std::string& msg) {
  g_error = msg;
  return code;
}

relo_status cuda_fail(cudaError_t e, const char* what) {
  return fail(RELO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RELO_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

bool bad_size(int w, int h) { return w < 1 || h < 1 || w > 16384 || h > 16384; }

// A pose whose rotation or translation holds a NaN or an infinity (rays would march nowhere).
bool bad_pose(const double* P) {
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(P[i])) return true;
  return false;
}

relo_status check_intr(const relo_intrinsics* in) {
  if (!in) return fail(RELO_EINVAL, "intrinsics is null");
  if (bad_size(in->width, in->height)) return fail(RELO_EINVAL, "image size outside [1, 16384]");
  if (!(in->fx > 0) || !(in->fy > 0)) return fail(RELO_EINVAL, "focal lengths must be positive");
  if (!(in->depth_min > 0) || !(in->depth_max > in->depth_min)) return fail(RELO_EINVAL, "bad depth range");
  return RELO_OK;
}

relo_status check_params(const relo_ransac_params* p) {
  if (!p) return fail(RELO_EINVAL, "ransac params is null");
  if (p->n_hyps < 1 || p->n_hyps > 4096) return fail(RELO_EINVAL, "n_hyps outside [1, 4096]");
  if (p->batch < 1 || p->batch > 4096) return fail(RELO_EINVAL, "batch outside [1, 4096]");
  if (p->max_tries < 1 || p->max_tries > (1 << 24)) return fail(RELO_EINVAL, "max_tries outside [1, 2^24]");
  if (!(p->rigidity > 0) || !(p->inlier_dist > 0) || !(p->min_area >= 0)) return fail(RELO_EINVAL, "bad thresholds");
  return RELO_OK;
}

int rounds_for(int K) {
  int r = 0;
  while (K > 1) {
    K = (K + 1) / 2;
    ++r;
  }
  return r;
}

// Per-attempt RANSAC scratch, carved from a workspace.
void carve_ransac(Carver& c, RansacJob& j, int W, int H, int K, int B, int n_rounds, int T) {
  const int n_pix = W * H;
  j.nv = table_words(T);
  j.table = c.take<uint4>((size_t)n_pix * j.nv);
  const int R = std::max(n_rounds, 1);
  j.hs = 1 + (T + 1) / 2;
  j.refit_parts = (R * B + kRefinePixels - 1) / kRefinePixels;
  j.refit = c.take<float2>((size_t)K * j.refit_parts * 16);
  j.refit_ref = c.take<float>((size_t)K * 8);
  j.pix = c.take<int4>((size_t)R * B * j.hs);
  j.chunk_count = c.take<int32_t>((n_pix + kCompactChunk - 1) / kCompactChunk);
  j.n_valid = c.take<int32_t>(1);
  j.poses = c.take<double>((size_t)K * 12);
  j.hyp_ok = c.take<int32_t>(K);
  j.tries = c.take<int32_t>(K);
  j.energy = c.take<double>(K);
  j.alive_a = c.take<int32_t>(K);
  j.alive_b = c.take<int32_t>(K);
  j.drawn = c.take<int32_t>((size_t)std::max(n_rounds, 1) * B);
  j.inliers = c.take<int32_t>(K);
  j.err = c.take<int32_t>(1);
}

void fill_ransac_job(RansacJob& j, const ForestView& fv, const uint16_t* depth, const uint16_t* leaves,
                     const relo_intrinsics& in, const relo_ransac_params& p, int K, uint64_t seed) {
  j.forest = fv;
  j.depth = depth;
  j.leaves = leaves;
  j.W = in.width;
  j.H = in.height;
  j.fx = in.fx;
  j.fy = in.fy;
  j.cx = in.cx;
  j.cy = in.cy;
  j.K = K;
  j.B = p.batch;
  j.max_tries = p.max_tries;
  j.n_rounds = rounds_for(K);
  j.rigidity = p.rigidity;
  j.min_area = p.min_area;
  j.inlier_dist = p.inlier_dist;
  j.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
  j.key1 = (uint32_t)(seed >> 32);
  j.vW = in.width;
  j.vH = in.height;
}

// Alive / survivor prefix tables for rounds 0..R-1 (each n_jobs + 1 ints).
// Per round: prefix tables of the jobs' alive and surviving hypothesis counts, their totals and
// their largest per-job values.
void round_tables(const std::vector<int>& K, int R, std::vector<int32_t>& alive, std::vector<int32_t>& surv,
                  std::vector<int>& tot_alive, std::vector<int>& tot_surv, std::vector<int>& max_alive,
                  std::vector<int>& max_surv) {
  const int n = (int)K.size();
  alive.assign((size_t)R * (n + 1), 0);
  surv.assign((size_t)R * (n + 1), 0);
  tot_alive.assign(R, 0);
  tot_surv.assign(R, 0);
  max_alive.assign(R, 0);
  max_surv.assign(R, 0);
  std::vector<int> cur(K);
  for (int r = 0; r < R; ++r) {
    int a = 0, s = 0;
    for (int j = 0; j < n; ++j) {
      alive[(size_t)r * (n + 1) + j] = a;
      surv[(size_t)r * (n + 1) + j] = s;
      if (cur[j] > 1) {
        a += cur[j];
        s += (cur[j] + 1) / 2;
        max_alive[r] = std::max(max_alive[r], cur[j]);
        max_surv[r] = std::max(max_surv[r], (cur[j] + 1) / 2);
        cur[j] = (cur[j] + 1) / 2;
      }
    }
    alive[(size_t)r * (n + 1) + n] = a;
    surv[(size_t)r * (n + 1) + n] = s;
    tot_alive[r] = a;
    tot_surv[r] = s;
  }
}

}  // namespace

// =============================================================================================
// A RANSAC pass: every stage launched once over a set of jobs (one job for the single-view entry
// points, many for batches).
// =============================================================================================
namespace {

struct RansacPass {
  RansacJob* d_jobs = nullptr;
  int n = 0, R = 0, chunks = 0, hyps = 0, B = 0;
  int32_t* d_counter = nullptr;  // the search's hypothesis counter
  int32_t* d_alive_prefix = nullptr;
  int32_t* d_surv_prefix = nullptr;
  std::vector<int> tot_alive, tot_surv, max_alive, max_surv;
  // the persistent schedule (batches): its items, control words + completion counters
  PItem* d_items = nullptr;
  int n_items = 0;
  int32_t* d_ctrl = nullptr;
  int ctrl_words = 0, final_base = 0;
};

// The persistent launch's items for jobs with K[j] hypotheses, B pixels per round, in dependency
// order (every job's fits, then round by round every job's draw, energy chunks, selection, re-fit
// sum parts and re-fits, then the finalisations), and the layout of its completion counters:
// done[g * n + j] for group g of job j -- 0 searched hypotheses, 1 fits, 2 + 5 r + (0 draw,
// 1 energy, 2 select, 3 refine, 4 refit) for round r, then finalisation.  stall (test hook): the
// first selection item waits for one chunk more than exists.
void build_items(const std::vector<int>& K, int B, bool stall, std::vector<PItem>& items, int* n_done,
                 int* final_base) {
  const int n = (int)K.size();
  int R = 0;
  for (int k : K) R = std::max(R, rounds_for(k));
  const int g_final = 2 + 5 * R;
  auto idx = [n](int g, int j) { return g * n + j; };
  items.clear();
  std::vector<int> dep(n), need(n), cur(K);
  for (int j = 0; j < n; ++j) {
    const int nf = (K[j] + kPersistThreadsHost - 1) / kPersistThreadsHost;
    for (int c = 0; c < nf; ++c) items.push_back(PItem{kItemFit, j, c, 0, 0, idx(0, j), K[j], idx(1, j)});
    dep[j] = idx(1, j);
    need[j] = nf;
  }
  for (int r = 0; r < R; ++r) {
    const int gd = 2 + 5 * r;
    const int parts = ((r + 1) * B + kRefinePixels - 1) / kRefinePixels;
    std::vector<int> alive(n, 0);
    for (int j = 0; j < n; ++j) alive[j] = cur[j] > 1 ? cur[j] : 0;
    for (int j = 0; j < n; ++j)
      if (alive[j]) items.push_back(PItem{kItemDraw, j, 0, 0, r, dep[j], need[j], idx(gd, j)});
    for (int j = 0; j < n; ++j)
      for (int c = 0; c < (alive[j] + 31) / 32; ++c)
        items.push_back(PItem{kItemEnergy, j, c, 0, r, idx(gd, j), 1, idx(gd + 1, j)});
    for (int j = 0; j < n; ++j)
      if (alive[j]) items.push_back(PItem{kItemSelect, j, 0, 0, r, idx(gd + 1, j), (alive[j] + 31) / 32, idx(gd + 2, j)});
    for (int j = 0; j < n; ++j)
      for (int c = 0; c < ((alive[j] + 1) / 2 + 31) / 32; ++c)
        for (int q = 0; q < parts; ++q) items.push_back(PItem{kItemRefine, j, c, q, r, idx(gd + 2, j), 1, idx(gd + 3, j)});
    for (int j = 0; j < n; ++j) {
      if (!alive[j]) continue;
      const int surv = (alive[j] + 1) / 2, nref = (surv + 31) / 32 * parts;
      const int nfit = (surv + kPersistThreadsHost - 1) / kPersistThreadsHost;
      for (int c = 0; c < nfit; ++c) items.push_back(PItem{kItemRefit, j, c, 0, r, idx(gd + 3, j), nref, idx(gd + 4, j)});
      dep[j] = idx(gd + 4, j);
      need[j] = nfit;
      cur[j] = surv;
    }
  }
  for (int j = 0; j < n; ++j) items.push_back(PItem{kItemFinal, j, 0, 0, 0, dep[j], need[j], idx(g_final, j)});
  if (stall)
    for (PItem& it : items)
      if (it.kind == kItemSelect) {
        it.need += 1;
        break;
      }
  *n_done = (g_final + 1) * n;
  *final_base = g_final * n;
}

// The size of build_items' list and of its counter block, without building it.
void count_items(const std::vector<int>& K, int B, int* n_items, int* n_done, int* final_base) {
  const int n = (int)K.size();
  int R = 0;
  for (int k : K) R = std::max(R, rounds_for(k));
  long items = 0;
  for (int j = 0; j < n; ++j) {
    items += (K[j] + kPersistThreadsHost - 1) / kPersistThreadsHost + 1;  // fits, finalisation
    int cur = K[j];
    for (int r = 0; r < R && cur > 1; ++r) {
      const int parts = ((r + 1) * B + kRefinePixels - 1) / kRefinePixels, surv = (cur + 1) / 2;
      items += 1 + (cur + 31) / 32 + 1 + (long)(surv + 31) / 32 * parts +
               (surv + kPersistThreadsHost - 1) / kPersistThreadsHost;
      cur = surv;
    }
  }
  *n_items = (int)items;
  *n_done = (2 + 5 * R + 1) * n;
  *final_base = (2 + 5 * R) * n;
}

// Records ev (nullable) on s; external: as an event-record node when s is being captured.
cudaError_t record(cudaEvent_t ev, cudaStream_t s, bool external) {
  if (!ev) return cudaSuccess;
  return external ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
}

// ev_hyp / ev_rounds (nullable) are recorded after the hypotheses and after the rounds.
relo_status run_pass(const RansacPass& p, cudaStream_t s, int* launches, cudaEvent_t ev_hyp, cudaEvent_t ev_rounds,
                     bool external = false, const Schedule& sched = Schedule()) {
  int L = 0;
  if (sched.persistent && p.d_items && p.n > 0) {
    // one launch (plus the compaction before it and the timeout report after it); the stage
    // events bracket the compaction + persistent launch (hypotheses) and the report (rounds)
    RELO_CUDA(launch_compact(p.d_jobs, p.n, p.chunks, s));
    PersistArgs a{};
    a.jobs = p.d_jobs;
    a.n_jobs = p.n;
    a.total_hyps = p.hyps;
    a.ctrl = p.d_ctrl;
    a.items = p.d_items;
    a.n_items = p.n_items;
    a.done = p.d_ctrl + 4;
    a.final_base = p.final_base;
    a.alive_prefix = p.d_alive_prefix;
    a.surv_prefix = p.d_surv_prefix;
    a.timeout_ns = g_persist_timeout_ns.load();
    RELO_CUDA(launch_persistent(a, p.ctrl_words, s));
    RELO_CUDA(record(ev_hyp, s, external));
    RELO_CUDA(record(ev_rounds, s, external));
    *launches += 4;
    return RELO_OK;
  }
  if (p.n > 0) {
    RELO_CUDA(launch_compact(p.d_jobs, p.n, p.chunks, s));
    RELO_CUDA(launch_hypotheses(p.d_jobs, p.n, p.hyps, p.d_counter, s, sched));
    L += 4;
  }
  RELO_CUDA(record(ev_hyp, s, external));
  for (int r = 0; r < p.R; ++r) {
    if (p.tot_alive[r] == 0) continue;
    RELO_CUDA(launch_round(p.d_jobs, p.n, r, p.d_alive_prefix + (size_t)r * (p.n + 1), p.tot_alive[r],
                           p.max_alive[r], p.d_surv_prefix + (size_t)r * (p.n + 1), p.tot_surv[r], p.max_surv[r],
                           p.B, s, sched));
    L += 5;
  }
  if (p.n > 0) {
    RELO_CUDA(launch_finalise(p.d_jobs, p.n, s));
    L += 1;
  }
  RELO_CUDA(record(ev_rounds, s, external));
  *launches += L;
  return RELO_OK;
}

int pass_launches(const RansacPass& p, const Schedule& sched = Schedule()) {
  if (sched.persistent && p.d_items && p.n > 0) return 4;
  int L = p.n > 0 ? 5 : 0;
  for (int r = 0; r < p.R; ++r)
    if (p.tot_alive[r] > 0) L += 5;
  return L;
}

}  // namespace

namespace {

// Free cells of the block grid (value < 0) become -(Chebyshev distance, in blocks, to the nearest
// allocated cell).  The Chebyshev distance is the length of the shortest path through the 26
// neighbours of each cell, which the two raster passes of the unit-weight 3 x 3 x 3 chamfer mask
// compute exactly (Rosenfeld and Pfaltz's sequential distance transform).
void chebyshev_free_distance(std::vector<int32_t>& grid, const int gd[3]) {
  const int X = gd[0], Y = gd[1], Z = gd[2];
  const int32_t kFar = 1 << 24;
  std::vector<int32_t> d(grid.size());
  for (size_t i = 0; i < grid.size(); ++i) d[i] = grid[i] >= 0 ? 0 : kFar;
  auto at = [&](int x, int y, int z) { return ((size_t)z * Y + y) * X + x; };
  for (int pass = 0; pass < 2; ++pass) {
    const int s = pass == 0 ? 1 : -1;  // forward: neighbours earlier in raster order; backward: later
    for (int zi = 0; zi < Z; ++zi)
      for (int yi = 0; yi < Y; ++yi)
        for (int xi = 0; xi < X; ++xi) {
          const int x = s > 0 ? xi : X - 1 - xi, y = s > 0 ? yi : Y - 1 - yi, z = s > 0 ? zi : Z - 1 - zi;
          int32_t& v = d[at(x, y, z)];
          if (v == 0) continue;
          int32_t m = v;
          for (int dz = -1; dz <= 0; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                if (dz == 0 && (dy > 0 || (dy == 0 && dx >= 0))) continue;
                const int xx = x + s * dx, yy = y + s * dy, zz = z + s * dz;
                if (xx < 0 || yy < 0 || zz < 0 || xx >= X || yy >= Y || zz >= Z) continue;
                m = std::min(m, d[at(xx, yy, zz)] + 1);
              }
          v = m;
        }
  }
  for (size_t i = 0; i < grid.size(); ++i)
    if (grid[i] < 0) grid[i] = -d[i];
}

}  // namespace

extern "C" {

const char* relo_last_error(void) { return g_error.c_str(); }

// ---------------------------------------------------------------------------------------------
// Scenes
// ---------------------------------------------------------------------------------------------
relo_status relo_create_scene(const int32_t* coords, const float* tsdf, const uint8_t* rgba, int64_t n,
                              double voxel, double mu, int32_t log2_buckets, relo_scene** out) {
  if (!out) return fail(RELO_EINVAL, "out is null");
  *out = nullptr;
  if (n < 0 || n > (int64_t)INT32_MAX - 1) return fail(RELO_EINVAL, "n_blocks out of range");
  if (n > 0 && (!coords || !tsdf || !rgba)) return fail(RELO_EINVAL, "null block arrays");
  if (log2_buckets < 4 || log2_buckets > 30) return fail(RELO_EINVAL, "log2_buckets outside [4, 30]");
  if (!(voxel > 0) || !(mu > 0)) return fail(RELO_EINVAL, "voxel_size and mu must be positive");
  const uint32_t nb = 1u << log2_buckets, mask = nb - 1;
  std::vector<int4> buckets(nb, pack_entry(0, 0, 0, -1, -1));
  std::vector<int4> excess;
  std::vector<int> chain(nb, 0);
  int max_chain = 0;
  for (int64_t b = 0; b < n; ++b) {
    const int x = coords[3 * b], y = coords[3 * b + 1], z = coords[3 * b + 2];
    if (x < -32768 || x > 32767 || y < -32768 || y > 32767 || z < -32768 || z > 32767)
      return fail(RELO_EINVAL, "block coordinate outside int16 range");
    const uint32_t h = block_hash(x, y, z) & mask;
    const int4 key = pack_entry(x, y, z, (int)b, -1);
    int4* e = &buckets[h];
    if (e->z < 0) {
      *e = key;
      chain[h] = 1;
      max_chain = std::max(max_chain, 1);
      continue;
    }
    bool dup = false;
    int4* last = e;
    while (true) {
      if (last->x == key.x && (last->y & 0xFFFF) == (key.y & 0xFFFF)) {
        dup = true;
        break;
      }
      if (last->w < 0) break;
      last = &excess[last->w];
    }
    if (dup) continue;
    last->w = (int)excess.size();
    excess.push_back(key);  // may reallocate: 'last' is not used after this
    chain[h] += 1;
    max_chain = std::max(max_chain, chain[h]);
  }
  if (excess.empty()) excess.push_back(pack_entry(0, 0, 0, -1, -1));
  // Dense block-index grid over the bounding box (origin and extent on multiples of 8 blocks;
  // skipped when the box exceeds 2^28 blocks), free blocks holding -(Chebyshev distance to the
  // nearest allocated block).
  std::vector<int32_t> grid;
  int g0[3] = {0, 0, 0}, gd[3] = {0, 0, 0};
  if (n > 0) {
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int64_t b = 0; b < n; ++b)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], (int)coords[3 * b + a]);
        hi[a] = std::max(hi[a], (int)coords[3 * b + a]);
      }
    size_t cells = 1;
    for (int a = 0; a < 3; ++a) {
      g0[a] = (int)std::floor(lo[a] / 8.0) * 8;
      gd[a] = ((hi[a] - g0[a]) / 8 + 1) * 8;
      cells *= (size_t)gd[a];
    }
    if (cells <= ((size_t)1 << 28)) {
      grid.assign(cells, -1);
      for (int64_t b = 0; b < n; ++b) {
        const int x = coords[3 * b] - g0[0], y = coords[3 * b + 1] - g0[1], z = coords[3 * b + 2] - g0[2];
        int32_t& cell = grid[((size_t)z * gd[1] + y) * gd[0] + x];
        if (cell < 0) cell = (int32_t)b;  // a repeated coordinate keeps its first block, as in the hash
      }
      chebyshev_free_distance(grid, gd);
    }
  }
  relo_scene* s = new relo_scene();
  s->n_blocks = n;
  s->n_excess = (int64_t)excess.size();
  auto cleanup = [&]() {
    relo::dev_free(s->d_buckets);
    relo::dev_free(s->d_excess);
    relo::dev_free(s->d_tsdf);
    relo::dev_free(s->d_rgba);
    relo::dev_free(s->d_grid);
    delete s;
  };
  if (!grid.empty() && (relo::dev_malloc((void**)&s->d_grid, grid.size() * 4) != cudaSuccess ||
                        cudaMemcpy(s->d_grid, grid.data(), grid.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)) {
    cudaGetLastError();
    cleanup();
    return fail(RELO_ENOMEM, "device allocation for the scene grid failed");
  }
  const size_t nv = (size_t)std::max<int64_t>(n, 1) * kVoxelsPerBlock;
  if (relo::dev_malloc((void**)&s->d_buckets, nb * sizeof(int4)) != cudaSuccess ||
      relo::dev_malloc((void**)&s->d_excess, excess.size() * sizeof(int4)) != cudaSuccess ||
      relo::dev_malloc((void**)&s->d_tsdf, nv * sizeof(float)) != cudaSuccess ||
      relo::dev_malloc((void**)&s->d_rgba, nv * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(RELO_ENOMEM, "device allocation for the scene failed");
  }
  cudaError_t e = cudaMemcpy(s->d_buckets, buckets.data(), nb * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_excess, excess.data(), excess.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(s->d_tsdf, tsdf, (size_t)n * kVoxelsPerBlock * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(s->d_rgba, rgba, (size_t)n * kVoxelsPerBlock * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "scene upload");
  }
  SceneView& v = s->view;
  v.buckets = (const int4*)s->d_buckets;
  v.excess = (const int4*)s->d_excess;
  v.tsdf = (const float*)s->d_tsdf;
  v.rgba = (const uint32_t*)s->d_rgba;
  v.mask = mask;
  v.n_blocks = (int32_t)n;
  v.max_chain = max_chain + 1;
  v.voxel = (float)voxel;
  v.inv_voxel = (float)(1.0 / voxel);
  v.mu = (float)mu;
  v.block_size = (float)(8.0 * voxel);
  v.inv_block = (float)(1.0 / (8.0 * voxel));
  v.grid = (const int32_t*)s->d_grid;
  v.ox = g0[0];
  v.oy = g0[1];
  v.oz = g0[2];
  v.gx = gd[0];
  v.gy = gd[1];
  v.gz = gd[2];
  // the apron copy of the tsdf, built on the device from the uploaded voxels and hash table
  if (n > 0) {
    void* d_coords = nullptr;
    if (relo::dev_malloc(&d_coords, (size_t)n * 3 * sizeof(int32_t)) != cudaSuccess ||
        relo::dev_malloc(&s->d_tsdf9, (size_t)n * kApronStride * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      relo::dev_free(d_coords);
      relo::dev_free(s->d_tsdf9);
      cleanup();
      return fail(RELO_ENOMEM, "device allocation for the scene's apron copy failed");
    }
    e = cudaMemcpy(d_coords, coords, (size_t)n * 3 * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_build_apron(v, (const int32_t*)d_coords, n, (float*)s->d_tsdf9, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    relo::dev_free(d_coords);
    if (e != cudaSuccess) {
      relo::dev_free(s->d_tsdf9);
      cleanup();
      return cuda_fail(e, "scene apron build");
    }
    v.tsdf9 = (const float*)s->d_tsdf9;
  }
  *out = s;
  return RELO_OK;
}

void relo_destroy_scene(relo_scene* s) {
  if (!s) return;
  relo::dev_free(s->d_buckets);
  relo::dev_free(s->d_excess);
  relo::dev_free(s->d_tsdf);
  relo::dev_free(s->d_rgba);
  relo::dev_free(s->d_grid);
  relo::dev_free(s->d_tsdf9);
  relo::dev_free(s->d_weight);
  relo::dev_free(s->d_coords);
  relo::dev_free(s->d_counters);
  delete s;
}

// ---------------------------------------------------------------------------------------------
// Scenes that grow by TSDF fusion (Sec. 3.3 (a); Appendix B.3)
// ---------------------------------------------------------------------------------------------
relo_status relo_create_fusion_scene(int64_t capacity, double voxel, double mu, int32_t log2_buckets,
                                     int32_t max_weight, relo_scene** out) {
  if (!out) return fail(RELO_EINVAL, "out is null");
  *out = nullptr;
  if (capacity < 1 || capacity > ((int64_t)1 << 24)) return fail(RELO_EINVAL, "capacity outside [1, 2^24] blocks");
  if (log2_buckets < 4 || log2_buckets > 30) return fail(RELO_EINVAL, "log2_buckets outside [4, 30]");
  if (!(voxel > 0) || !(mu > 0)) return fail(RELO_EINVAL, "voxel_size and mu must be positive");
  if (max_weight < 1 || max_weight > 65535) return fail(RELO_EINVAL, "max_weight outside [1, 65535]");
  relo_scene* s = new relo_scene();
  s->capacity = capacity;
  s->n_excess = capacity;
  s->max_weight = max_weight;
  const size_t nb = (size_t)1 << log2_buckets, nv = (size_t)capacity * kVoxelsPerBlock;
  cudaError_t e = relo::dev_malloc((void**)&s->d_buckets, nb * sizeof(int4));
  if (e == cudaSuccess) e = relo::dev_malloc((void**)&s->d_excess, (size_t)capacity * sizeof(int4));
  if (e == cudaSuccess) e = relo::dev_malloc((void**)&s->d_tsdf, nv * sizeof(float));
  if (e == cudaSuccess) e = relo::dev_malloc((void**)&s->d_rgba, nv * sizeof(uint32_t));
  if (e == cudaSuccess) e = relo::dev_malloc((void**)&s->d_weight, nv * sizeof(uint16_t));
  if (e == cudaSuccess) e = relo::dev_malloc((void**)&s->d_coords, (size_t)capacity * sizeof(int4));
  if (e == cudaSuccess) e = relo::dev_malloc((void**)&s->d_counters, 4 * sizeof(int32_t) + sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaGetLastError();
    relo_destroy_scene(s);
    return fail(RELO_ENOMEM, "device allocation for the fusion scene failed");
  }
  // empty buckets (0xFF bytes: block -1, next -1; the key words of an empty head are unused),
  // voxels at tsdf +1, weight 0, colour 0
  e = cudaMemset(s->d_buckets, 0xFF, nb * sizeof(int4));
  if (e == cudaSuccess) e = cudaMemset(s->d_excess, 0xFF, (size_t)capacity * sizeof(int4));
  if (e == cudaSuccess) e = cudaMemset(s->d_rgba, 0, nv * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(s->d_weight, 0, nv * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMemset(s->d_counters, 0, 4 * sizeof(int32_t) + sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_fuse_init((float*)s->d_tsdf, (int64_t)nv, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    relo_destroy_scene(s);
    return cuda_fail(e, "fusion scene initialisation");
  }
  SceneView& v = s->view;
  v.buckets = (const int4*)s->d_buckets;
  v.excess = (const int4*)s->d_excess;
  v.tsdf = (const float*)s->d_tsdf;
  v.rgba = (const uint32_t*)s->d_rgba;
  v.mask = (uint32_t)(nb - 1);
  v.n_blocks = (int32_t)capacity;
  v.max_chain = (int32_t)capacity + 1;  // chains grow on the device: bound walks by the pool
  v.voxel = (float)voxel;
  v.inv_voxel = (float)(1.0 / voxel);
  v.mu = (float)mu;
  v.block_size = (float)(8.0 * voxel);
  v.inv_block = (float)(1.0 / (8.0 * voxel));
  v.grid = nullptr;
  v.tsdf9 = nullptr;  // fusion changes the voxels: the raycast reads them directly
  *out = s;
  return RELO_OK;
}

namespace {
size_t fuse_set_slots(int32_t width, int32_t height) {
  size_t s = 1024;
  while (s < 2 * (size_t)width * height) s *= 2;
  return s;
}
}  // namespace

size_t relo_fuse_workspace_size(int32_t width, int32_t height) {
  if (bad_size(width, height)) return 0;
  const size_t S = fuse_set_slots(width, height);
  return S * 8 + 256 + S * 8 + 256 + S * 8 + 256 + S * 4 + 256 + 256;
}

relo_status relo_fuse_frames(relo_scene* scene, const relo_intrinsics* intr, const double* poses, int32_t n,
                             const uint16_t* depth, const uint8_t* rgba, void* ws, size_t ws_bytes,
                             relo_stream stream) {
  if (!poses || n < 1) return fail(RELO_EINVAL, "null poses or n < 1");
  for (int k = 0; k < n; ++k)
    if (bad_pose(poses + 16 * (size_t)k)) return fail(RELO_EINVAL, "a pose is not finite");
  if (!intr || bad_size(intr->width, intr->height)) return fail(RELO_EINVAL, "bad intrinsics");
  const size_t n_pix = (size_t)intr->width * intr->height;
  for (int k = 0; k < n; ++k) {  // in order: each frame sees the blocks of the frames before it
    const relo_status st = relo_fuse_frame(scene, intr, poses + 16 * (size_t)k, depth ? depth + k * n_pix : nullptr,
                                           rgba ? rgba + k * n_pix * 4 : nullptr, ws, ws_bytes, stream);
    if (st) return st;
  }
  return RELO_OK;
}

relo_status relo_fuse_frame(relo_scene* scene, const relo_intrinsics* intr, const double* pose, const uint16_t* depth,
                            const uint8_t* rgba, void* ws, size_t ws_bytes, relo_stream stream) {
  if (!scene || !pose || !depth) return fail(RELO_EINVAL, "null scene, pose or depth");
  if (bad_pose(pose)) return fail(RELO_EINVAL, "pose is not finite");
  if (scene->capacity < 1) return fail(RELO_EINVAL, "scene was not created for fusion");
  relo_status st = check_intr(intr);
  if (st) return st;
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < relo_fuse_workspace_size(intr->width, intr->height))
    return fail(RELO_EINVAL, "workspace missing, misaligned or too small");
  const size_t S = fuse_set_slots(intr->width, intr->height);
  Carver c{(char*)ws, 0};
  FuseJob j{};
  j.set = c.take<unsigned long long>(S);
  j.new_keys = c.take<unsigned long long>(S);
  j.keys = c.take<unsigned long long>(S);
  j.visible = c.take<int32_t>(S);
  j.n_visible = c.take<int32_t>(3);
  j.n_new = j.n_visible + 1;
  j.n_keys = j.n_visible + 2;
  j.set_mask = (uint32_t)(S - 1);
  j.buckets = (int4*)scene->d_buckets;
  j.excess = (int4*)scene->d_excess;
  j.tsdf = (float*)scene->d_tsdf;
  j.rgba = (uint32_t*)scene->d_rgba;
  j.weight = (uint16_t*)scene->d_weight;
  j.coords = (int4*)scene->d_coords;
  j.counters = (int32_t*)scene->d_counters;
  j.status = j.counters + 2;
  j.updates = (unsigned long long*)(j.counters + 4);
  j.bucket_mask = scene->view.mask;
  j.capacity = (int32_t)scene->capacity;
  j.max_weight = scene->max_weight;
  j.depth = depth;
  j.frame_rgba = (const uint32_t*)rgba;
  j.W = intr->width;
  j.H = intr->height;
  j.fx = (float)intr->fx;
  j.fy = (float)intr->fy;
  j.cx = (float)intr->cx;
  j.cy = (float)intr->cy;
  j.dmin = (float)intr->depth_min;
  j.dmax = (float)intr->depth_max;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) j.R[3 * r + q] = (float)pose[4 * r + q];
    j.t[r] = (float)pose[4 * r + 3];
  }
  j.voxel = scene->view.voxel;
  j.mu = scene->view.mu;
  RELO_CUDA(launch_fuse_frame(j, (cudaStream_t)stream));
  return RELO_OK;
}

relo_status relo_fuse_stats(const void* ws, int32_t width, int32_t height, int32_t* visible, int32_t* created) {
  if (!ws || bad_size(width, height)) return fail(RELO_EINVAL, "null workspace or bad size");
  const size_t S = fuse_set_slots(width, height);
  Carver c{(char*)ws, 0};
  c.take<unsigned long long>(S);
  c.take<unsigned long long>(S);
  c.take<unsigned long long>(S);
  c.take<int32_t>(S);
  const int32_t* counts = c.take<int32_t>(3);
  int32_t h[2] = {0, 0};
  RELO_CUDA(cudaDeviceSynchronize());
  RELO_CUDA(cudaMemcpy(h, counts, sizeof(h), cudaMemcpyDeviceToHost));
  if (visible) *visible = h[0];
  if (created) *created = h[1];
  return RELO_OK;
}

relo_status relo_scene_block_count(const relo_scene* scene, int64_t* n_blocks) {
  if (!scene || !n_blocks) return fail(RELO_EINVAL, "null argument");
  if (scene->capacity < 1) {
    *n_blocks = scene->n_blocks;
    return RELO_OK;
  }
  int32_t h[4] = {0, 0, 0, 0};
  RELO_CUDA(cudaDeviceSynchronize());
  RELO_CUDA(cudaMemcpy(h, scene->d_counters, sizeof(h), cudaMemcpyDeviceToHost));
  *n_blocks = std::min<int64_t>(h[0], scene->capacity);
  if (h[2] != RELO_OK) return fail(h[2], "fusion ran out of blocks, chain entries or its per-frame block set");
  return RELO_OK;
}

relo_status relo_scene_fusion_updates(const relo_scene* scene, uint64_t* updates) {
  if (!scene || !updates) return fail(RELO_EINVAL, "null argument");
  if (scene->capacity < 1) return fail(RELO_EINVAL, "scene was not created for fusion");
  RELO_CUDA(cudaDeviceSynchronize());
  RELO_CUDA(cudaMemcpy(updates, (const char*)scene->d_counters + 4 * sizeof(int32_t), sizeof(uint64_t),
                       cudaMemcpyDeviceToHost));
  return RELO_OK;
}

relo_status relo_scene_export(const relo_scene* scene, int32_t* coords, float* tsdf, uint8_t* rgba, uint16_t* weight,
                              int64_t capacity, int64_t* n_out) {
  if (!scene || !n_out) return fail(RELO_EINVAL, "null argument");
  if (scene->capacity < 1) return fail(RELO_EINVAL, "scene was not created for fusion");
  int64_t n = 0;
  relo_status st = relo_scene_block_count(scene, &n);
  if (st != RELO_OK && st != RELO_ENOMEM) return st;
  *n_out = n;
  if (capacity < n) return fail(RELO_EINVAL, "capacity smaller than the block count");
  if (n == 0) return st;
  std::vector<int4> c4((size_t)n);
  RELO_CUDA(cudaMemcpy(c4.data(), scene->d_coords, (size_t)n * sizeof(int4), cudaMemcpyDeviceToHost));
  if (coords)
    for (int64_t b = 0; b < n; ++b) {
      coords[3 * b] = c4[b].x;
      coords[3 * b + 1] = c4[b].y;
      coords[3 * b + 2] = c4[b].z;
    }
  const size_t nv = (size_t)n * kVoxelsPerBlock;
  if (tsdf) RELO_CUDA(cudaMemcpy(tsdf, scene->d_tsdf, nv * sizeof(float), cudaMemcpyDeviceToHost));
  if (rgba) RELO_CUDA(cudaMemcpy(rgba, scene->d_rgba, nv * 4, cudaMemcpyDeviceToHost));
  if (weight) RELO_CUDA(cudaMemcpy(weight, scene->d_weight, nv * sizeof(uint16_t), cudaMemcpyDeviceToHost));
  return st;
}

relo_status relo_set_allocator(relo_alloc_fn alloc, relo_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return fail(RELO_EINVAL, "alloc and free must both be set or both be null");
  std::lock_guard<std::mutex> lk(relo::g_alloc_mu);
  relo::g_alloc.alloc = alloc;
  relo::g_alloc.free = free_fn;
  relo::g_alloc.ctx = alloc ? ctx : nullptr;
  return RELO_OK;
}

void relo_debug_conv_path(int32_t use_tcgen05) { relo::g_conv_tcgen05.store(use_tcgen05 != 0); }

void relo_debug_persistent_stall(int32_t stall, int32_t timeout_ms) {
  relo::g_persist_stall.store(stall != 0);
  relo::g_persist_timeout_ns.store(timeout_ms > 0 ? (unsigned long long)timeout_ms * 1000000ull : 2000000000ull);
}

void relo_debug_conv_stall(int32_t tile, int32_t timeout_ms) {
  relo::g_conv_stall_tile.store(tile);
  relo::g_conv_timeout_ns.store(timeout_ms > 0 ? (unsigned long long)timeout_ms * 1000000ull : 2000000000ull);
}

void relo_debug_fail_allocations(int32_t n) { relo::g_fail_allocations.store(n > 0 ? n : 0); }

int64_t relo_debug_check_failures(void) {
#ifdef RELO_CHECKED
  if (cudaDeviceSynchronize() != cudaSuccess) return -2;
  unsigned long long total = 0;
  for (unsigned long long v : {check_failures_scene(), check_failures_forest(), check_failures_ransac(),
                               check_failures_fusion()}) {
    if (v == ~0ull) return -2;
    total += v;
  }
  return (int64_t)total;
#else
  return -1;
#endif
}

relo_status relo_debug_corrupt_scene(relo_scene* scene) {
  if (!scene || scene->n_excess < 1) return fail(RELO_EINVAL, "null scene");
  const size_t nb = (size_t)scene->view.mask + 1, ne = (size_t)scene->n_excess;
  std::vector<int4> buckets(nb), excess(ne);
  RELO_CUDA(cudaDeviceSynchronize());
  RELO_CUDA(cudaMemcpy(buckets.data(), scene->d_buckets, nb * sizeof(int4), cudaMemcpyDeviceToHost));
  RELO_CUDA(cudaMemcpy(excess.data(), scene->d_excess, ne * sizeof(int4), cudaMemcpyDeviceToHost));
  // every chain ends in a cycle through a self-linked entry (all links stay inside the table)
  for (int4& e : buckets)
    if (e.w < 0) e.w = 0;
  for (size_t i = 0; i < ne; ++i) excess[i].w = (int)i;
  RELO_CUDA(cudaMemcpy(scene->d_buckets, buckets.data(), nb * sizeof(int4), cudaMemcpyHostToDevice));
  RELO_CUDA(cudaMemcpy(scene->d_excess, excess.data(), ne * sizeof(int4), cudaMemcpyHostToDevice));
  return RELO_OK;
}

relo_status relo_scene_use_grid(relo_scene* s, int32_t enable) {
  if (!s) return fail(RELO_EINVAL, "scene is null");
  s->view.grid = enable ? (const int32_t*)s->d_grid : nullptr;
  return RELO_OK;
}

relo_status relo_scene_use_apron(relo_scene* s, int32_t enable) {
  if (!s) return fail(RELO_EINVAL, "scene is null");
  s->view.tsdf9 = enable ? (const float*)s->d_tsdf9 : nullptr;
  return RELO_OK;
}

relo_status relo_scene_lookup(const relo_scene* scene, const int32_t* keys, int64_t n, int64_t* out,
                              relo_stream stream) {
  if (!scene || (n > 0 && (!keys || !out)) || n < 0) return fail(RELO_EINVAL, "bad lookup arguments");
  RELO_CUDA(launch_scene_lookup(scene->view, keys, n, out, nullptr, (cudaStream_t)stream));
  return RELO_OK;
}

// ---------------------------------------------------------------------------------------------
// Raycast
// ---------------------------------------------------------------------------------------------
relo_status relo_raycast_view(const relo_scene* scene, const relo_intrinsics* intr, const double pose[16],
                              const float* noise, uint16_t* depth, uint8_t* rgba, relo_stream stream) {
  if (!scene || !pose || !depth) return fail(RELO_EINVAL, "null scene, pose or depth");
  if (bad_pose(pose)) return fail(RELO_EINVAL, "pose is not finite");
  relo_status st = check_intr(intr);
  if (st) return st;
  RayJob j = make_ray_job(scene->view, *intr, pose);
  j.noise = noise;
  j.depth = depth;
  j.rgba = (uint32_t*)rgba;
  RELO_CUDA(launch_raycast(nullptr, 1, &j, ray_tiles(intr->width, intr->height), rgba != nullptr, false,
                           (cudaStream_t)stream));
  return RELO_OK;
}

constexpr int kMaxGlobalScenes = 64;

size_t relo_raycast_views_workspace_size(int32_t n) { return n < 1 ? 0 : (size_t)n * sizeof(RayJob); }

relo_status relo_raycast_views(const relo_scene* scene, const relo_intrinsics* intr, const double* poses, int32_t n,
                               const float* noise, uint16_t* depth, uint8_t* rgba, void* ws, size_t ws_bytes,
                               relo_stream stream) {
  if (!scene || !poses || !depth || n < 1) return fail(RELO_EINVAL, "null scene, poses or depth, or n < 1");
  for (int k = 0; k < n; ++k)
    if (bad_pose(poses + 16 * (size_t)k)) return fail(RELO_EINVAL, "a pose is not finite");
  relo_status st = check_intr(intr);
  if (st) return st;
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < relo_raycast_views_workspace_size(n))
    return fail(RELO_EINVAL, "workspace missing, misaligned or too small");
  const size_t n_pix = (size_t)intr->width * intr->height;
  const int tiles = ray_tiles(intr->width, intr->height);
  std::vector<RayJob> jobs(n);
  for (int k = 0; k < n; ++k) {
    RayJob& j = jobs[k];
    j = make_ray_job(scene->view, *intr, poses + 16 * (size_t)k);
    j.noise = noise ? noise + k * n_pix : nullptr;
    j.depth = depth + k * n_pix;
    j.rgba = rgba ? (uint32_t*)rgba + k * n_pix : nullptr;
    j.tile_begin = k * tiles;
  }
  cudaStream_t s = (cudaStream_t)stream;
  RELO_CUDA(cudaMemcpyAsync(ws, jobs.data(), n * sizeof(RayJob), cudaMemcpyHostToDevice, s));
  // a copy from pageable memory returns once the host buffer has been staged, so jobs may go
  RELO_CUDA(launch_raycast((const RayJob*)ws, n, nullptr, n * tiles, rgba != nullptr, false, s, Schedule(),
                           scene->view.tsdf9 != nullptr));
  return RELO_OK;
}

size_t relo_render_global_workspace_size(int32_t n_scenes) {
  return (n_scenes < 1 || n_scenes > kMaxGlobalScenes) ? 0 : (size_t)n_scenes * sizeof(RayJob) + 256;
}

relo_status relo_render_global(const relo_scene* const* scenes, const double* global_poses, int32_t n_scenes,
                               const relo_intrinsics* intr, const double* pose_global, uint16_t* depth,
                               uint8_t* rgba, int8_t* owner, int32_t* err_dev, void* ws, size_t ws_bytes,
                               relo_stream stream) {
  if (!scenes || !global_poses || !pose_global || !depth) return fail(RELO_EINVAL, "null argument");
  if (n_scenes < 1 || n_scenes > kMaxGlobalScenes) return fail(RELO_EINVAL, "n_scenes outside [1, 64]");
  if (bad_pose(pose_global)) return fail(RELO_EINVAL, "pose is not finite");
  for (int a = 0; a < n_scenes; ++a)
    if (bad_pose(global_poses + 16 * (size_t)a)) return fail(RELO_EINVAL, "a global pose is not finite");
  relo_status st = check_intr(intr);
  if (st) return st;
  if (!ws || ((uintptr_t)ws & 255) != 0 || ws_bytes < relo_render_global_workspace_size(n_scenes))
    return fail(RELO_EINVAL, "workspace missing, misaligned or too small");
  std::vector<RayJob> jobs(n_scenes);
  bool all_apron = true;
  for (int a = 0; a < n_scenes; ++a) {
    if (!scenes[a]) return fail(RELO_EINVAL, "null scene");
    all_apron = all_apron && scenes[a]->view.tsdf9 != nullptr;
    // local camera -> scene-a pose: (gT_a)^-1 P_g, with gT_a rigid (scene a -> global)
    const double* g = global_poses + 16 * (size_t)a;
    double P[16] = {0};
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int k = 0; k < 3; ++k) acc += g[4 * k + r] * pose_global[4 * k + c];  // R_g^T column r
        if (c == 3)
          for (int k = 0; k < 3; ++k) acc -= g[4 * k + r] * g[4 * k + 3];
        P[4 * r + c] = acc;
      }
    }
    P[15] = 1.0;
    jobs[a] = make_ray_job(scenes[a]->view, *intr, P);
  }
  cudaStream_t s = (cudaStream_t)stream;
  RELO_CUDA(cudaMemcpyAsync(ws, jobs.data(), n_scenes * sizeof(RayJob), cudaMemcpyHostToDevice, s));
  RELO_CUDA(launch_render_global((const RayJob*)ws, n_scenes, intr->width, intr->height, depth, (uint32_t*)rgba,
                                 owner, err_dev, s, all_apron));
  return RELO_OK;
}

// ---------------------------------------------------------------------------------------------
// Forests
// ---------------------------------------------------------------------------------------------
relo_status relo_create_forest(const void* nodes, int32_t T, int32_t D, const float* modes, const uint8_t* n_modes,
                               int32_t M, relo_forest** out) {
  if (!out) return fail(RELO_EINVAL, "out is null");
  *out = nullptr;
  if (T < 1 || T > kMaxTrees) return fail(RELO_EINVAL, "n_trees outside [1, 16]");
  if (D < 1 || D > 16) return fail(RELO_EINVAL, "depth outside [1, 16]");
  if (M < 1 || M > 64) return fail(RELO_EINVAL, "max_modes outside [1, 64]");
  if (!nodes) return fail(RELO_EINVAL, "nodes is null");
  const size_t n_int = ((size_t)1 << D) - 1, L = (size_t)1 << D;
  const int4* in_nodes = (const int4*)nodes;
  for (size_t i = 0; i < (size_t)T * n_int; ++i) {
    const int kind = in_nodes[i].z & 0xFF, c1 = (in_nodes[i].z >> 8) & 0xFF, c2 = (in_nodes[i].z >> 16) & 0xFF;
    if (kind > 1 || (kind == 1 && (c1 > 3 || c2 > 3))) return fail(RELO_EINVAL, "node kind not 0/1 or channel > 3");
  }
  relo_forest* f = new relo_forest();
  f->T = T;
  f->D = D;
  f->M = M;
  const size_t n_modes_bytes = (size_t)T * L, modes_bytes = (size_t)T * L * M * kModeFloats * sizeof(float);
  if (relo::dev_malloc((void**)&f->d_nodes, (size_t)T * n_int * 16) != cudaSuccess ||
      relo::dev_malloc((void**)&f->d_modes, modes_bytes) != cudaSuccess || relo::dev_malloc((void**)&f->d_n_modes, n_modes_bytes) != cudaSuccess ||
      relo::dev_malloc((void**)&f->d_top, (size_t)T * L * sizeof(float4)) != cudaSuccess) {
    cudaGetLastError();
    relo_destroy_forest(f);
    return fail(RELO_ENOMEM, "device allocation for the forest failed");
  }
  // device copy of the nodes: the third word becomes {value mask (16 bits), bit offset of probe 1
  // (8 bits), of probe 2 (8 bits)} in a packed pixel {depth | r << 16 | g << 24 | b << 32}: a depth
  // node's mask 0xFFFF and offsets 0, a colour node's mask 0xFF and offsets 16 + 8 c1, 16 + 8 c2
  std::vector<int4> dev_nodes((size_t)T * n_int);
  std::memcpy(dev_nodes.data(), nodes, dev_nodes.size() * 16);
  int max_offset = 0;  // the largest |offset| of any probe: bounds how far a probe can leave its pixel
  for (int4& nd : dev_nodes) {
    const int kind = nd.z & 0xFF, c1 = (nd.z >> 8) & 0xFF, c2 = (nd.z >> 16) & 0xFF;
    nd.z = kind == 0 ? 0xFFFF : (0xFF | (16 + 8 * c1) << 16 | (16 + 8 * c2) << 24);
    for (const int w : {nd.x, nd.y}) {
      max_offset = std::max(max_offset, std::abs((int)(int16_t)(w & 0xFFFF)));
      max_offset = std::max(max_offset, std::abs((int)(int16_t)((uint32_t)w >> 16)));
    }
  }
  // offsets of at most 255 in magnitude are stored times 128 (still int16), which the evaluation's
  // division by depth takes as they are (forest.cu, probe)
  if (max_offset <= 255)
    for (int4& nd : dev_nodes) {
      int* w[2] = {&nd.x, &nd.y};
      for (int* p : w) {
        const int lo = (int)(int16_t)(*p & 0xFFFF) * 128, hi = (int)(int16_t)((uint32_t)*p >> 16) * 128;
        *p = (int)((uint32_t)(uint16_t)(int16_t)lo | (uint32_t)(uint16_t)(int16_t)hi << 16);
      }
    }
  cudaError_t e = cudaMemcpy(f->d_nodes, dev_nodes.data(), (size_t)T * n_int * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = modes ? cudaMemcpy(f->d_modes, modes, modes_bytes, cudaMemcpyHostToDevice)
                                  : cudaMemset(f->d_modes, 0, modes_bytes);
  if (e == cudaSuccess) e = n_modes ? cudaMemcpy(f->d_n_modes, n_modes, n_modes_bytes, cudaMemcpyHostToDevice)
                                    : cudaMemset(f->d_n_modes, 0, n_modes_bytes);
  if (e == cudaSuccess) e = launch_top_modes((const float*)f->d_modes, (const uint8_t*)f->d_n_modes, (int)(T * L), M,
                                             (float4*)f->d_top, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    relo_destroy_forest(f);
    return cuda_fail(e, "forest upload");
  }
  f->view.nodes = (const int4*)f->d_nodes;
  f->view.modes = (const float*)f->d_modes;
  f->view.n_modes = (const uint8_t*)f->d_n_modes;
  f->view.top = (const float4*)f->d_top;
  f->view.T = T;
  f->view.D = D;
  f->view.M = M;
  f->view.probe_reach = 1 + max_offset;
  f->view.offset_shift = max_offset <= 255 ? 7 : 0;
  *out = f;
  return RELO_OK;
}

void relo_destroy_forest(relo_forest* f) {
  if (!f) return;
  relo::dev_free(f->d_nodes);
  relo::dev_free(f->d_modes);
  relo::dev_free(f->d_n_modes);
  relo::dev_free(f->d_top);
  free(f->res_samples);
  free(f->res_count);
  free(f->res_seen);
  delete f;
}

relo_status relo_forest_get_modes(const relo_forest* f, float* modes, uint8_t* n_modes) {
  if (!f) return fail(RELO_EINVAL, "forest is null");
  const size_t L = (size_t)1 << f->D;
  if (modes) RELO_CUDA(cudaMemcpy(modes, f->d_modes, (size_t)f->T * L * f->M * kModeFloats * 4, cudaMemcpyDeviceToHost));
  if (n_modes) RELO_CUDA(cudaMemcpy(n_modes, f->d_n_modes, (size_t)f->T * L, cudaMemcpyDeviceToHost));
  return RELO_OK;
}

relo_status relo_forest_eval(const relo_forest* f, const uint16_t* depth, const uint8_t* rgba, int32_t W, int32_t H,
                             uint16_t* leaves, relo_stream stream) {
  if (!f || !depth || !rgba || !leaves) return fail(RELO_EINVAL, "null forest or buffer");
  if (bad_size(W, H)) return fail(RELO_EINVAL, "image size outside [1, 16384]");
  ForestJob j{};
  j.forest = f->view;
  j.depth = depth;
  j.rgba = (const uint32_t*)rgba;
  j.leaves = leaves;
  j.W = W;
  j.H = H;
  j.pixel_begin = 0;
  RELO_CUDA(launch_forest(nullptr, 1, &j, (int64_t)W * H, (cudaStream_t)stream, f->T));
  return RELO_OK;
}

// ---------------------------------------------------------------------------------------------
// Relocaliser training
// ---------------------------------------------------------------------------------------------
relo_status relo_forest_train_begin(relo_forest* f, const relo_train_params* p) {
  if (!f || !p) return fail(RELO_EINVAL, "null forest or params");
  if (p->capacity < 1 || p->capacity > 4096) return fail(RELO_EINVAL, "capacity outside [1, 4096]");
  if (p->stride < 1 || p->max_iter < 1 || !(p->bandwidth > 0)) return fail(RELO_EINVAL, "bad training params");
  const size_t L = (size_t)f->T << f->D;
  free(f->res_samples);
  free(f->res_count);
  free(f->res_seen);
  f->res_samples = (float*)calloc(L * p->capacity * 3, sizeof(float));
  f->res_count = (int32_t*)calloc(L, sizeof(int32_t));
  f->res_seen = (int64_t*)calloc(L, sizeof(int64_t));
  if (!f->res_samples || !f->res_count || !f->res_seen) return fail(RELO_ENOMEM, "host reservoirs");
  f->train = *p;
  f->training = true;
  return RELO_OK;
}

relo_status relo_forest_train_frame(relo_forest* f, const relo_intrinsics* intr, const double pose[16],
                                    const uint16_t* depth, const uint8_t* rgba, relo_stream stream) {
  if (!f || !f->training) return fail(RELO_EINVAL, "training not begun");
  if (!pose || !depth || !rgba) return fail(RELO_EINVAL, "null pose or image");
  relo_status st = check_intr(intr);
  if (st) return st;
  const int W = intr->width, H = intr->height, S = f->train.stride, T = f->T;
  const int gw = (W + S - 1) / S, gh = (H + S - 1) / S;
  const size_t n_pix = (size_t)W * H;
  cudaStream_t s = (cudaStream_t)stream;
  uint16_t* d_leaves = nullptr;
  float* d_coords = nullptr;
  RELO_CUDA(relo::dev_malloc((void**)&d_leaves, n_pix * T * sizeof(uint16_t)));
  if (relo::dev_malloc((void**)&d_coords, (size_t)gw * gh * 3 * sizeof(float)) != cudaSuccess) {
    relo::dev_free(d_leaves);
    return fail(RELO_ENOMEM, "training scratch");
  }
  ForestJob j{};
  j.forest = f->view;
  j.depth = depth;
  j.rgba = (const uint32_t*)rgba;
  j.leaves = d_leaves;
  j.W = W;
  j.H = H;
  std::vector<uint16_t> leaves(n_pix * T), dep(n_pix);
  std::vector<float> coords((size_t)gw * gh * 3);
  cudaError_t e = launch_forest(nullptr, 1, &j, (int64_t)n_pix, s, T);
  if (e == cudaSuccess) e = launch_scene_coords(depth, W, H, S, intr->fx, intr->fy, intr->cx, intr->cy, pose, d_coords, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(leaves.data(), d_leaves, leaves.size() * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dep.data(), depth, n_pix * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(coords.data(), d_coords, coords.size() * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  relo::dev_free(d_leaves);
  relo::dev_free(d_coords);
  if (e != cudaSuccess) return cuda_fail(e, "training frame");
  // Algorithm R per leaf, offers in raster order, trees in order (host, sequential by definition)
  const int cap = f->train.capacity;
  const int64_t L = (int64_t)1 << f->D;
  const uint32_t k0 = (uint32_t)(f->train.seed & 0xFFFFFFFFu), k1 = (uint32_t)(f->train.seed >> 32);
  for (int v = 0; v < H; v += S) {
    for (int u = 0; u < W; u += S) {
      const size_t pix = (size_t)v * W + u;
      if (dep[pix] == 0) continue;
      const float* w = &coords[3 * ((size_t)(v / S) * gw + u / S)];
      for (int t = 0; t < T; ++t) {
        const int64_t id = (int64_t)t * L + leaves[(size_t)t * n_pix + pix];
        const int64_t n = f->res_seen[id]++;
        int64_t slot = -1;
        if (n < cap) {
          slot = n;
          f->res_count[id] = (int32_t)(n + 1);
        } else {
          const uint4 x = philox4x32_10(make_uint4(3u, (uint32_t)id, (uint32_t)(n & 0xFFFFFFFF), (uint32_t)(n >> 32)), k0, k1);
          const uint64_t jj = ((uint64_t)x.x * (uint64_t)(n + 1)) >> 32;
          if (jj < (uint64_t)cap) slot = (int64_t)jj;
        }
        if (slot >= 0) std::memcpy(&f->res_samples[((size_t)id * cap + slot) * 3], w, 3 * sizeof(float));
      }
    }
  }
  return RELO_OK;
}

relo_status relo_forest_train_reservoirs(const relo_forest* f, float* samples, int32_t* count) {
  if (!f || !f->training) return fail(RELO_EINVAL, "training not begun");
  const size_t L = (size_t)f->T << f->D;
  if (samples) std::memcpy(samples, f->res_samples, L * f->train.capacity * 3 * sizeof(float));
  if (count) std::memcpy(count, f->res_count, L * sizeof(int32_t));
  return RELO_OK;
}

relo_status relo_forest_train_finish(relo_forest* f, relo_stream stream) {
  if (!f || !f->training) return fail(RELO_EINVAL, "training not begun");
  const size_t L = (size_t)f->T << f->D;
  const int cap = f->train.capacity;
  cudaStream_t s = (cudaStream_t)stream;
  float* d_samples = nullptr;
  int32_t* d_count = nullptr;
  RELO_CUDA(relo::dev_malloc((void**)&d_samples, L * cap * 3 * sizeof(float)));
  if (relo::dev_malloc((void**)&d_count, L * sizeof(int32_t)) != cudaSuccess) {
    relo::dev_free(d_samples);
    return fail(RELO_ENOMEM, "training scratch");
  }
  cudaError_t e = cudaMemcpyAsync(d_samples, f->res_samples, L * cap * 3 * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_count, f->res_count, L * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(f->d_modes, 0, L * f->M * kModeFloats * sizeof(float), s);
  if (e == cudaSuccess)
    e = launch_mean_shift(d_samples, d_count, cap, (int)L, (float)f->train.bandwidth, (float)f->train.tol,
                          f->train.max_iter, (float)f->train.merge_dist, (float)f->train.cov_floor, f->M,
                          (float*)f->d_modes, (uint8_t*)f->d_n_modes, s);
  if (e == cudaSuccess) e = launch_top_modes((const float*)f->d_modes, (const uint8_t*)f->d_n_modes, (int)L, f->M,
                                             (float4*)f->d_top, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  relo::dev_free(d_samples);
  relo::dev_free(d_count);
  if (e != cudaSuccess) return cuda_fail(e, "mean shift");
  return RELO_OK;
}

// ---------------------------------------------------------------------------------------------
// RANSAC on one view
// ---------------------------------------------------------------------------------------------
namespace {

struct Single {
  RansacJob job{};
  RansacJob* d_job = nullptr;
  int32_t* d_counter = nullptr;
  int32_t* d_alive = nullptr;
  int32_t* d_surv = nullptr;
  size_t bytes = 0;
  int chunks = 0;
};

// Workspace of one view: [job | alive prefix tables | surv tables | per-attempt scratch]
void layout_single(char* base, int W, int H, int K, int B, int T, Single& s) {
  Carver c{base, 0};
  s.d_job = c.take<RansacJob>(1);
  s.d_counter = c.take<int32_t>(1);
  const int R = std::max(rounds_for(K), 1);
  s.d_alive = c.take<int32_t>((size_t)R * 2);
  s.d_surv = c.take<int32_t>((size_t)R * 2);
  carve_ransac(c, s.job, W, H, K, B, rounds_for(K), T);
  s.bytes = c.off;
  s.chunks = (W * H + kCompactChunk - 1) / kCompactChunk;
}

relo_status single_setup_view(const ForestView& fv, const uint16_t* depth, const uint16_t* leaves,
                              const relo_intrinsics* intr, const relo_ransac_params* p, void* ws, size_t ws_bytes,
                              Single& s) {
  if (!depth || !leaves || !ws) return fail(RELO_EINVAL, "null image or workspace");
  relo_status st = check_intr(intr);
  if (st) return st;
  st = check_params(p);
  if (st) return st;
  if (((uintptr_t)ws & 255) != 0) return fail(RELO_EINVAL, "workspace must be 256-byte aligned");
  layout_single(nullptr, intr->width, intr->height, p->n_hyps, p->batch, fv.T, s);
  if (s.bytes > ws_bytes) return fail(RELO_EINVAL, "workspace too small");
  layout_single((char*)ws, intr->width, intr->height, p->n_hyps, p->batch, fv.T, s);
  fill_ransac_job(s.job, fv, depth, leaves, *intr, *p, p->n_hyps, p->seed);
  s.job.chunk_begin = 0;
  s.job.hyp_begin = 0;
  return RELO_OK;
}

relo_status single_setup(const relo_forest* f, const uint16_t* depth, const uint16_t* leaves,
                         const relo_intrinsics* intr, const relo_ransac_params* p, void* ws, size_t ws_bytes,
                         Single& s) {
  if (!f) return fail(RELO_EINVAL, "null forest");
  return single_setup_view(f->view, depth, leaves, intr, p, ws, ws_bytes, s);
}

// Runs every RANSAC stage of one prepared single-view job, writing *result.
relo_status single_run(Single& s, const relo_ransac_params* p, relo_pose_result* result, cudaStream_t cs);

}  // namespace

size_t relo_ransac_workspace_size(int32_t W, int32_t H, const relo_ransac_params* p) {
  if (!p || bad_size(W, H) || p->n_hyps < 1 || p->batch < 1) return 0;
  Single s;
  layout_single(nullptr, W, H, p->n_hyps, p->batch, kMaxTrees, s);  // enough for any forest
  return s.bytes;
}

relo_status relo_ransac_relocalise(const relo_forest* f, const uint16_t* depth, const uint16_t* leaves,
                                   const relo_intrinsics* intr, const relo_ransac_params* p, void* ws,
                                   size_t ws_bytes, relo_pose_result* result, relo_stream stream) {
  Single s;
  relo_status st = single_setup(f, depth, leaves, intr, p, ws, ws_bytes, s);
  if (st) return st;
  if (!result) return fail(RELO_EINVAL, "result is null");
  return single_run(s, p, result, (cudaStream_t)stream);
}

}  // extern "C"

namespace {
relo_status single_run(Single& s, const relo_ransac_params* p, relo_pose_result* result, cudaStream_t cs) {
  s.job.result = result;
  std::vector<int> K(1, p->n_hyps);
  std::vector<int32_t> at, su;
  RansacPass b;
  b.n = 1;
  b.R = rounds_for(p->n_hyps);
  round_tables(K, std::max(b.R, 1), at, su, b.tot_alive, b.tot_surv, b.max_alive, b.max_surv);
  b.B = p->batch;
  b.d_jobs = s.d_job;
  b.d_counter = s.d_counter;
  b.d_alive_prefix = s.d_alive;
  b.d_surv_prefix = s.d_surv;
  b.chunks = s.chunks;
  b.hyps = p->n_hyps;
  RELO_CUDA(cudaMemcpyAsync(s.d_job, &s.job, sizeof(RansacJob), cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemcpyAsync(s.d_alive, at.data(), at.size() * 4, cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemcpyAsync(s.d_surv, su.data(), su.size() * 4, cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemsetAsync(s.job.err, 0, sizeof(int32_t), cs));
  int launches = 0;
  return run_pass(b, cs, &launches, nullptr, nullptr);
}
}  // namespace

// ---------------------------------------------------------------------------------------------
// Allocation-free RANSAC: the same stages as relo_ransac_relocalise, with the scratch taken from
// a fixed array compiled into this library instead of a caller-allocated workspace.  Its device
// address is looked up once per device (cudaGetSymbolAddress with that device current) and cached;
// every call on a device reuses the same array.
// ---------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[RELO_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_addr[kMaxDevices] = {};

relo_status static_scratch(void** out) {
  int dev = -1;
  RELO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(RELO_EINVAL, "device ordinal outside [0, 64)");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return RELO_OK;
}
}  // namespace

extern "C" {

relo_status relo_ransac_relocalise_noalloc(const relo_forest* f, const uint16_t* depth, const uint16_t* leaves,
                                           const relo_intrinsics* intr, const relo_ransac_params* p,
                                           relo_pose_result* result, relo_stream stream) {
  if (!f || !intr || !p) return fail(RELO_EINVAL, "null forest, intrinsics or params");
  relo_status st = check_intr(intr);
  if (st) return st;
  st = check_params(p);
  if (st) return st;
  Single need;
  layout_single(nullptr, intr->width, intr->height, p->n_hyps, p->batch, f->T, need);
  if (need.bytes > (size_t)RELO_STATIC_SCRATCH_BYTES)
    return fail(RELO_EINVAL, "view needs " + std::to_string(need.bytes) + " bytes of scratch; the static scratch holds " +
                                 std::to_string((size_t)RELO_STATIC_SCRATCH_BYTES));
  void* scratch = nullptr;
  st = static_scratch(&scratch);
  if (st) return st;
  return relo_ransac_relocalise(f, depth, leaves, intr, p, scratch, (size_t)RELO_STATIC_SCRATCH_BYTES, result, stream);
}

relo_status relo_ransac_hypotheses(const relo_forest* f, const uint16_t* depth, const uint16_t* leaves,
                                   const relo_intrinsics* intr, const relo_ransac_params* p, void* ws,
                                   size_t ws_bytes, double* poses, int32_t* valid, int32_t* tries,
                                   relo_stream stream) {
  Single s;
  relo_status st = single_setup(f, depth, leaves, intr, p, ws, ws_bytes, s);
  if (st) return st;
  if (!poses || !valid || !tries) return fail(RELO_EINVAL, "null output");
  cudaStream_t cs = (cudaStream_t)stream;
  RELO_CUDA(cudaMemcpyAsync(s.d_job, &s.job, sizeof(RansacJob), cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemsetAsync(s.job.err, 0, sizeof(int32_t), cs));
  RELO_CUDA(launch_compact(s.d_job, 1, s.chunks, cs));
  RELO_CUDA(launch_hypotheses(s.d_job, 1, p->n_hyps, s.d_counter, cs));
  RELO_CUDA(cudaMemcpyAsync(poses, s.job.poses, (size_t)p->n_hyps * 12 * 8, cudaMemcpyDeviceToDevice, cs));
  RELO_CUDA(cudaMemcpyAsync(valid, s.job.hyp_ok, (size_t)p->n_hyps * 4, cudaMemcpyDeviceToDevice, cs));
  RELO_CUDA(cudaMemcpyAsync(tries, s.job.tries, (size_t)p->n_hyps * 4, cudaMemcpyDeviceToDevice, cs));
  return RELO_OK;
}

relo_status relo_ransac_round(const relo_forest* f, const uint16_t* depth, const uint16_t* leaves,
                              const relo_intrinsics* intr, const relo_ransac_params* p, int32_t round,
                              const int32_t* alive, int32_t n_alive, const int32_t* valid, double* poses,
                              double* energy, int32_t* drawn, int32_t* survivors, int32_t* inliers, void* ws,
                              size_t ws_bytes, relo_stream stream) {
  Single s;
  relo_status st = single_setup(f, depth, leaves, intr, p, ws, ws_bytes, s);
  if (st) return st;
  if (!alive || !valid || !poses || !energy || !drawn || !survivors || !inliers)
    return fail(RELO_EINVAL, "null buffer");
  if (round < 0 || n_alive < 2 || n_alive > p->n_hyps) return fail(RELO_EINVAL, "bad round or alive count");
  cudaStream_t cs = (cudaStream_t)stream;
  RansacJob j = s.job;
  j.poses = poses;
  j.energy = energy;
  j.hyp_ok = (int32_t*)valid;
  j.drawn = drawn;
  j.inliers = inliers;
  if (round & 1) {
    j.alive_b = (int32_t*)alive;
    j.alive_a = survivors;
  } else {
    j.alive_a = (int32_t*)alive;
    j.alive_b = survivors;
  }
  const int32_t ap[2] = {0, n_alive}, sp[2] = {0, (n_alive + 1) / 2};
  RELO_CUDA(cudaMemcpyAsync(s.d_job, &j, sizeof(RansacJob), cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemcpyAsync(s.d_alive, ap, sizeof(ap), cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemcpyAsync(s.d_surv, sp, sizeof(sp), cudaMemcpyHostToDevice, cs));
  RELO_CUDA(cudaMemsetAsync(j.err, 0, sizeof(int32_t), cs));
  RELO_CUDA(launch_compact(s.d_job, 1, s.chunks, cs));
  RELO_CUDA(launch_round(s.d_job, 1, round, s.d_alive, n_alive, n_alive, s.d_surv, (n_alive + 1) / 2,
                         (n_alive + 1) / 2, p->batch, cs));
  return RELO_OK;
}

// ---------------------------------------------------------------------------------------------
// Verification
// ---------------------------------------------------------------------------------------------
relo_status relo_verify(const relo_scene* scene_a, const relo_intrinsics* intr, const uint16_t* depth_b,
                        relo_pose_result* result, uint16_t* depth_a, relo_stream stream) {
  if (!scene_a || !depth_b || !result) return fail(RELO_EINVAL, "null scene, depth or result");
  relo_status st = check_intr(intr);
  if (st) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  RayJob v = make_ray_job(scene_a->view, *intr, nullptr);
  v.pose_dev = result->pose_c2s;
  v.status_dev = &result->status;
  v.depth_ref = depth_b;
  v.depth = depth_a;
  v.counts = (unsigned long long*)&result->omega_a;
  RELO_CUDA(cudaMemsetAsync(&result->omega, 0, 5 * sizeof(uint64_t), cs));
  RELO_CUDA(launch_raycast(nullptr, 1, &v, ray_tiles(intr->width, intr->height), false, true, cs));
  RELO_CUDA(launch_verify_decide_one(result, (uint64_t)intr->width * intr->height, cs));
  return RELO_OK;
}

}  // extern "C"

// =============================================================================================
// Learned scene-coordinate regressor (the workload's alternative relocaliser; see regressor.cu)
// =============================================================================================
struct relo_regressor {
  float* d_p = nullptr;  // FP32 master parameters, per layer w [3][3][cin][cout] then b [cout]
  float* d_g = nullptr;  // gradients (same layout)
  float* d_m = nullptr;  // Adam moments
  float* d_v = nullptr;
  bf16* d_wk[kRegLayers] = {};    // forward weights [9][cout_pad][cin_pad]
  bf16* d_wt[kRegLayers] = {};    // flipped, transposed weights [9][cin][cout_pad_t] (layers 1..7)
  float* d_bias[kRegLayers] = {}; // biases padded to cout_pad
  int64_t w_off[kRegLayers], b_off[kRegLayers], n_params = 0;
  int t = 0;
  int n_sms = 148;
  double origin[3] = {0, 0, 0};
  int32_t* d_status = nullptr;    // RELO_ETIMEOUT when a tcgen05 convolution's bounded wait ran out
};

namespace {

void reg_offsets(int64_t* w_off, int64_t* b_off, int64_t* total) {
  int64_t off = 0;
  for (int l = 0; l < kRegLayers; ++l) {
    w_off[l] = off;
    off += 9LL * kRegCin[l] * kRegCout[l];
    b_off[l] = off;
    off += kRegCout[l];
  }
  *total = off;
}

int cout_pad_t(int l) { return l == kRegLayers - 1 ? 16 : 64; }

__global__ void pad_bias_kernel(const float* b, int cout, int cout_pad, float* out) {
  const int i = threadIdx.x;
  if (i < cout_pad) out[i] = i < cout ? b[i] : 0.f;
}

relo_status reg_pack(relo_regressor* r, cudaStream_t s) {
  for (int l = 0; l < kRegLayers; ++l) {
    RELO_CUDA(launch_pack(r->d_p + r->w_off[l], kRegCin[l], kRegCout[l], kRegCinPad[l], kRegCoutPad[l], r->d_wk[l],
                          l > 0 ? r->d_wt[l] : nullptr, cout_pad_t(l), s));
    pad_bias_kernel<<<1, 64, 0, s>>>(r->d_p + r->b_off[l], kRegCout[l], kRegCoutPad[l], r->d_bias[l]);
    RELO_CUDA(cudaGetLastError());
  }
  return RELO_OK;
}

// Per-layer grid sizes: H[0] = input, H[l + 1] = output of layer l.
void reg_sizes(int W, int H, int* Hs, int* Ws) {
  Hs[0] = H;
  Ws[0] = W;
  for (int l = 0; l < kRegLayers; ++l) {
    Hs[l + 1] = (Hs[l] - 1) / kRegStride[l] + 1;
    Ws[l + 1] = (Ws[l] - 1) / kRegStride[l] + 1;
  }
}

struct RegBuffers {
  bf16* x = nullptr;                  // [n][H][W][16]
  bf16* act[kRegLayers] = {};         // act[l] = input of layer l (l >= 1): [n][H_l][W_l][64]
  float* head = nullptr;              // [n][Hc][Wc][8]
  float4* tgt = nullptr;              // [n][Hc][Wc]
  bf16* ghead = nullptr;              // [n][Hc][Wc][16]
  bf16* gpre[kRegLayers] = {};        // gpre[l] = gradient of layer l's pre-activation output (l < 7)
  float* partial = nullptr;           // backward-weight chunk sums
  float* bias_scratch = nullptr;
  float* loss = nullptr;
  double* poses = nullptr;            // [n][16]
  size_t bytes = 0;
};

void reg_layout(char* base, int n, int W, int H, bool training, RegBuffers& b, size_t start = 0) {
  Carver c{base, start};
  int Hs[kRegLayers + 1], Ws[kRegLayers + 1];
  reg_sizes(W, H, Hs, Ws);
  b.x = c.take<bf16>((size_t)n * H * W * 16);
  for (int l = 1; l < kRegLayers; ++l) b.act[l] = c.take<bf16>((size_t)n * Hs[l] * Ws[l] * 64);
  const size_t cells = (size_t)n * Hs[kRegLayers] * Ws[kRegLayers];
  b.head = c.take<float>(cells * 8);
  if (training) {
    b.tgt = c.take<float4>(cells);
    b.ghead = c.take<bf16>(cells * 16);
    for (int l = 0; l < kRegLayers - 1; ++l) b.gpre[l] = c.take<bf16>((size_t)n * Hs[l + 1] * Ws[l + 1] * 64);
    size_t part = 0, bias = 0;
    for (int l = 0; l < kRegLayers; ++l) {
      const size_t px = (size_t)n * Hs[l + 1] * Ws[l + 1];
      const size_t chunks = (px + kWgradChunk - 1) / kWgradChunk;
      part = std::max(part, chunks * 9 * kRegCoutPad[l] * kRegCinPad[l]);
      bias = std::max(bias, ((px + 2047) / 2048) * 64);
    }
    b.partial = c.take<float>(part);
    b.bias_scratch = c.take<float>(bias);
    b.loss = c.take<float>(1);
    b.poses = c.take<double>((size_t)n * 16);
  }
  b.bytes = c.off;
}

relo_status reg_forward(relo_regressor* r, const RegBuffers& b, const uint16_t* depth, const uint8_t* rgba, int n,
                        int W, int H, cudaStream_t s) {
  int Hs[kRegLayers + 1], Ws[kRegLayers + 1];
  reg_sizes(W, H, Hs, Ws);
  RELO_CUDA(launch_input(depth, (const uint32_t*)rgba, (long)n * H * W, b.x, s));
  RELO_CUDA(cudaMemsetAsync(r->d_status, 0, sizeof(int32_t), s));
  for (int l = 0; l < kRegLayers; ++l) {
    if (kRegCoutPad[l] == 64 && g_conv_tcgen05.load()) {
      // every layer but the head on the tcgen05 tensor cores (TMA-fed implicit GEMM)
      RELO_CUDA(launch_conv_tc(kRegCinPad[l], l == 0 ? b.x : b.act[l], n, Hs[l], Ws[l], r->d_wk[l], r->d_bias[l],
                               nullptr, b.act[l + 1], Hs[l + 1], Ws[l + 1], kRegStride[l], 1, 1, r->d_status, r->n_sms,
                               s, g_conv_timeout_ns.load(), g_conv_stall_tile.load()));
      continue;
    }
    ConvArgs a{};
    a.in = l == 0 ? b.x : b.act[l];
    a.w = r->d_wk[l];
    a.bias = r->d_bias[l];
    a.out = l < kRegLayers - 1 ? b.act[l + 1] : nullptr;
    a.out_f32 = l == kRegLayers - 1 ? b.head : nullptr;
    a.B = n;
    a.Hi = Hs[l];
    a.Wi = Ws[l];
    a.Ho = Hs[l + 1];
    a.Wo = Ws[l + 1];
    a.stride = kRegStride[l];
    a.relu = l < kRegLayers - 1;
    RELO_CUDA(launch_conv(kRegCinPad[l], kRegCoutPad[l] / 8, a, r->n_sms, s));
  }
  return RELO_OK;
}

relo_status reg_backward(relo_regressor* r, const RegBuffers& b, int n, int W, int H, cudaStream_t s) {
  int Hs[kRegLayers + 1], Ws[kRegLayers + 1];
  reg_sizes(W, H, Hs, Ws);
  const bf16* g = b.ghead;
  int gs = 16;
  for (int l = kRegLayers - 1; l >= 0; --l) {
    WgradArgs wa{};
    wa.in = l == 0 ? b.x : b.act[l];
    wa.g = g;
    wa.partial = b.partial;
    wa.B = n;
    wa.Hi = Hs[l];
    wa.Wi = Ws[l];
    wa.Ho = Hs[l + 1];
    wa.Wo = Ws[l + 1];
    wa.stride = kRegStride[l];
    wa.GS = gs;
    wa.chunk_pix = kWgradChunk;
    RELO_CUDA(launch_wgrad(kRegCinPad[l], kRegCoutPad[l] / 8, wa, s));
    const long px = (long)n * Hs[l + 1] * Ws[l + 1];
    const int chunks = (int)((px + kWgradChunk - 1) / kWgradChunk);
    RELO_CUDA(launch_wgrad_reduce(b.partial, chunks, kRegCoutPad[l], kRegCinPad[l], kRegCin[l], kRegCout[l],
                                  r->d_g + r->w_off[l], s));
    RELO_CUDA(launch_bias_grad(g, px, gs, kRegCout[l], b.bias_scratch, r->d_g + r->b_off[l], s));
    if (l > 0) {
      ConvArgs a{};
      a.in = g;
      a.w = r->d_wt[l];
      a.mask = b.act[l];
      a.out = b.gpre[l - 1];
      a.B = n;
      a.Hi = Hs[l];
      a.Wi = Ws[l];
      a.Hs = Hs[l + 1];
      a.Ws = Ws[l + 1];
      a.Ho = Hs[l];
      a.Wo = Ws[l];
      a.stride = 1;
      a.upsample = kRegStride[l] == 2;
      if (!a.upsample) {
        a.Hi = Hs[l + 1];
        a.Wi = Ws[l + 1];
      }
      if (!a.upsample && g_conv_tcgen05.load()) {
        // a stride-1 layer's backward-data pass is a forward convolution with the flipped,
        // transposed weights, masked by the ReLU of the layer's input: tcgen05 as well
        RELO_CUDA(launch_conv_tc(gs, g, n, a.Hi, a.Wi, r->d_wt[l], nullptr, b.act[l], b.gpre[l - 1], Hs[l], Ws[l], 1,
                                 1, 0, r->d_status, r->n_sms, s, g_conv_timeout_ns.load(), g_conv_stall_tile.load()));
      } else {
        RELO_CUDA(launch_conv(gs, 8, a, r->n_sms, s));
      }
      g = b.gpre[l - 1];
      gs = 64;
    }
  }
  return RELO_OK;
}

relo_status reg_check_size(int n, int W, int H) {
  if (n < 1 || n > 4096) return fail(RELO_EINVAL, "image count outside [1, 4096]");
  if (W < 8 || H < 8 || W % 8 || H % 8 || W > 8192 || H > 8192)
    return fail(RELO_EINVAL, "regressor images must be multiples of 8 in [8, 8192] per side");
  return RELO_OK;
}

relo_status reg_loss_and_grads(relo_regressor* r, const RegBuffers& b, const uint16_t* depth, const uint8_t* rgba,
                               int n, const relo_intrinsics* in, const double* poses, cudaStream_t s) {
  const int W = in->width, H = in->height, Wc = W / 8, Hc = H / 8;
  RELO_CUDA(cudaMemcpyAsync(b.poses, poses, (size_t)n * 16 * sizeof(double), cudaMemcpyHostToDevice, s));
  relo_status st = reg_forward(r, b, depth, rgba, n, W, H, s);
  if (st) return st;
  CellArgs ca{};
  ca.depth = depth;
  ca.poses = b.poses;
  ca.n = n;
  ca.W = W;
  ca.H = H;
  ca.Wc = Wc;
  ca.Hc = Hc;
  ca.fx = in->fx;
  ca.fy = in->fy;
  ca.cx = in->cx;
  ca.cy = in->cy;
  ca.ox = r->origin[0];
  ca.oy = r->origin[1];
  ca.oz = r->origin[2];
  RELO_CUDA(launch_targets(ca, b.tgt, s));
  RELO_CUDA(launch_loss(b.head, b.tgt, n * Wc * Hc, b.ghead, b.loss, s));
  return reg_backward(r, b, n, W, H, s);
}

}  // namespace

extern "C" {

int64_t relo_regressor_param_count(void) {
  int64_t w[kRegLayers], b[kRegLayers], t = 0;
  reg_offsets(w, b, &t);
  return t;
}

relo_status relo_create_regressor(const float* params, uint64_t seed, const double origin[3], relo_regressor** out) {
  if (!out) return fail(RELO_EINVAL, "out is null");
  *out = nullptr;
  relo_regressor* r = new relo_regressor();
  reg_offsets(r->w_off, r->b_off, &r->n_params);
  if (origin)
    for (int k = 0; k < 3; ++k) r->origin[k] = origin[k];
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&r->n_sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<float> host((size_t)r->n_params, 0.f);
  if (params) {
    std::memcpy(host.data(), params, host.size() * sizeof(float));
  } else {
    // He-uniform weights from Philox (counter (4, layer, index)), head scaled by 0.1, zero biases
    const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    for (int l = 0; l < kRegLayers; ++l) {
      const float bound = std::sqrt(6.0f / (9.0f * kRegCin[l])) * (l == kRegLayers - 1 ? 0.1f : 1.0f);
      const int64_t nw = 9LL * kRegCin[l] * kRegCout[l];
      for (int64_t i = 0; i < nw; ++i) {
        const uint4 x = philox4x32_10(make_uint4(4u, (uint32_t)l, (uint32_t)i, 0u), k0, k1);
        host[r->w_off[l] + i] = ((float)(x.x >> 8) * (1.0f / 16777216.0f) * 2.0f - 1.0f) * bound;
      }
    }
  }
  bool ok = relo::dev_malloc((void**)&r->d_p, r->n_params * 4) == cudaSuccess && relo::dev_malloc((void**)&r->d_g, r->n_params * 4) == cudaSuccess &&
            relo::dev_malloc((void**)&r->d_m, r->n_params * 4) == cudaSuccess && relo::dev_malloc((void**)&r->d_v, r->n_params * 4) == cudaSuccess &&
            relo::dev_malloc((void**)&r->d_status, sizeof(int32_t)) == cudaSuccess;
  for (int l = 0; ok && l < kRegLayers; ++l) {
    ok = relo::dev_malloc((void**)&r->d_wk[l], 9LL * kRegCoutPad[l] * kRegCinPad[l] * sizeof(bf16)) == cudaSuccess &&
         relo::dev_malloc((void**)&r->d_bias[l], 64 * sizeof(float)) == cudaSuccess;
    if (ok && l > 0) ok = relo::dev_malloc((void**)&r->d_wt[l], 9LL * kRegCin[l] * cout_pad_t(l) * sizeof(bf16)) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    relo_destroy_regressor(r);
    return fail(RELO_ENOMEM, "device allocation for the regressor failed");
  }
  cudaError_t e = cudaMemcpy(r->d_p, host.data(), r->n_params * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(r->d_m, 0, r->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(r->d_v, 0, r->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(r->d_g, 0, r->n_params * 4);
  if (e == cudaSuccess) e = cudaMemset(r->d_status, 0, sizeof(int32_t));
  if (e != cudaSuccess) {
    relo_destroy_regressor(r);
    return cuda_fail(e, "regressor upload");
  }
  relo_status st = reg_pack(r, 0);
  if (st == RELO_OK && cudaDeviceSynchronize() != cudaSuccess) st = fail(RELO_ECUDA, "regressor packing failed");
  if (st) {
    relo_destroy_regressor(r);
    return st;
  }
  *out = r;
  return RELO_OK;
}

void relo_destroy_regressor(relo_regressor* r) {
  if (!r) return;
  relo::dev_free(r->d_p);
  relo::dev_free(r->d_g);
  relo::dev_free(r->d_m);
  relo::dev_free(r->d_v);
  relo::dev_free(r->d_status);
  for (int l = 0; l < kRegLayers; ++l) {
    relo::dev_free(r->d_wk[l]);
    relo::dev_free(r->d_wt[l]);
    relo::dev_free(r->d_bias[l]);
  }
  delete r;
}

relo_status relo_regressor_get_state(const relo_regressor* r, float* params, float* m, float* v, int64_t* step) {
  if (!r) return fail(RELO_EINVAL, "regressor is null");
  RELO_CUDA(cudaDeviceSynchronize());
  if (params) RELO_CUDA(cudaMemcpy(params, r->d_p, r->n_params * 4, cudaMemcpyDeviceToHost));
  if (m) RELO_CUDA(cudaMemcpy(m, r->d_m, r->n_params * 4, cudaMemcpyDeviceToHost));
  if (v) RELO_CUDA(cudaMemcpy(v, r->d_v, r->n_params * 4, cudaMemcpyDeviceToHost));
  if (step) *step = r->t;
  return RELO_OK;
}

relo_status relo_regressor_set_state(relo_regressor* r, const float* params, const float* m, const float* v,
                                     int64_t step) {
  if (!r || !params || !m || !v) return fail(RELO_EINVAL, "null regressor or state array");
  if (step < 0 || step > INT32_MAX) return fail(RELO_EINVAL, "step outside [0, 2^31)");
  RELO_CUDA(cudaDeviceSynchronize());
  RELO_CUDA(cudaMemcpy(r->d_p, params, r->n_params * 4, cudaMemcpyHostToDevice));
  RELO_CUDA(cudaMemcpy(r->d_m, m, r->n_params * 4, cudaMemcpyHostToDevice));
  RELO_CUDA(cudaMemcpy(r->d_v, v, r->n_params * 4, cudaMemcpyHostToDevice));
  r->t = (int)step;
  relo_status st = reg_pack(r, 0);  // the BF16 copies the kernels multiply
  if (st) return st;
  RELO_CUDA(cudaDeviceSynchronize());
  return RELO_OK;
}

relo_status relo_regressor_get_params(const relo_regressor* r, float* params, float* grads) {
  if (!r) return fail(RELO_EINVAL, "regressor is null");
  if (params) RELO_CUDA(cudaMemcpy(params, r->d_p, r->n_params * 4, cudaMemcpyDeviceToHost));
  if (grads) RELO_CUDA(cudaMemcpy(grads, r->d_g, r->n_params * 4, cudaMemcpyDeviceToHost));
  return RELO_OK;
}

size_t relo_regressor_workspace_size(int32_t n, int32_t W, int32_t H, int32_t training) {
  if (n < 1 || W < 8 || H < 8) return 0;
  RegBuffers b;
  reg_layout(nullptr, n, W, H, training != 0, b);
  return b.bytes;
}

relo_status relo_regressor_forward(relo_regressor* r, const uint16_t* depth, const uint8_t* rgba, int32_t n,
                                   int32_t W, int32_t H, float* out, void* ws, size_t ws_bytes, relo_stream stream) {
  if (!r || !depth || !rgba || !out || !ws) return fail(RELO_EINVAL, "null argument");
  relo_status st = reg_check_size(n, W, H);
  if (st) return st;
  RegBuffers b;
  reg_layout(nullptr, n, W, H, false, b);
  if (b.bytes > ws_bytes || ((uintptr_t)ws & 255)) return fail(RELO_EINVAL, "workspace too small or misaligned");
  reg_layout((char*)ws, n, W, H, false, b);
  cudaStream_t s = (cudaStream_t)stream;
  st = reg_forward(r, b, depth, rgba, n, W, H, s);
  if (st) return st;
  RELO_CUDA(launch_head_copy(b.head, (long)n * (W / 8) * (H / 8), out, s));
  return RELO_OK;
}

relo_status relo_regressor_gradients(relo_regressor* r, const uint16_t* depth, const uint8_t* rgba, int32_t n,
                                     const relo_intrinsics* intr, const double* poses_host, float* loss_dev, void* ws,
                                     size_t ws_bytes, relo_stream stream) {
  if (!r || !depth || !rgba || !intr || !poses_host || !ws) return fail(RELO_EINVAL, "null argument");
  relo_status st = reg_check_size(n, intr->width, intr->height);
  if (st) return st;
  RegBuffers b;
  reg_layout(nullptr, n, intr->width, intr->height, true, b);
  if (b.bytes > ws_bytes || ((uintptr_t)ws & 255)) return fail(RELO_EINVAL, "workspace too small or misaligned");
  reg_layout((char*)ws, n, intr->width, intr->height, true, b);
  cudaStream_t s = (cudaStream_t)stream;
  st = reg_loss_and_grads(r, b, depth, rgba, n, intr, poses_host, s);
  if (st) return st;
  if (loss_dev) RELO_CUDA(cudaMemcpyAsync(loss_dev, b.loss, sizeof(float), cudaMemcpyDeviceToDevice, s));
  return RELO_OK;
}

relo_status relo_regressor_train_step(relo_regressor* r, const uint16_t* depth, const uint8_t* rgba, int32_t n,
                                      const relo_intrinsics* intr, const double* poses_host, float lr,
                                      float* loss_dev, void* ws, size_t ws_bytes, relo_stream stream) {
  relo_status st = relo_regressor_gradients(r, depth, rgba, n, intr, poses_host, loss_dev, ws, ws_bytes, stream);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  r->t += 1;
  RELO_CUDA(launch_adam(r->d_p, r->d_g, r->d_m, r->d_v, r->n_params, lr, r->t, s));
  return reg_pack(r, s);
}


}  // extern "C"

namespace {
// Learned single view: [regressor buffers | cell forest | RANSAC on the cell grid]
struct LearnedLayout {
  RegBuffers reg;
  float* modes;
  uint8_t* n_modes;
  float4* top;
  uint16_t* leaves;
  uint16_t* depth_lr;
  size_t ransac_off;
  Single ransac;
  size_t bytes;
  int L, D;
};

void learned_layout(char* base, int W, int H, const relo_ransac_params& p, LearnedLayout& l) {
  reg_layout(base, 1, W, H, false, l.reg);
  const int Wc = W / 8, Hc = H / 8, n = Wc * Hc;
  l.D = 1;
  while ((1 << l.D) < n) ++l.D;
  l.L = 1 << l.D;
  Carver c{base, l.reg.bytes};
  l.modes = c.take<float>((size_t)l.L * kModeFloats);
  l.n_modes = c.take<uint8_t>(l.L);
  l.top = c.take<float4>(l.L);
  l.leaves = c.take<uint16_t>(n);
  l.depth_lr = c.take<uint16_t>(n);
  l.ransac_off = (c.off + 255) & ~(size_t)255;
  layout_single(base ? base + l.ransac_off : nullptr, Wc, Hc, p.n_hyps, p.batch, 1, l.ransac);
  l.bytes = l.ransac_off + l.ransac.bytes;
}

relo_status learned_ransac(const LearnedLayout& l, const float* cells, int ostride, const double origin[3],
                           const int32_t* upstream, const uint16_t* depth, const relo_intrinsics* intr,
                           const relo_ransac_params* p, void* ws, size_t ws_bytes, relo_pose_result* result,
                           cudaStream_t s);

relo_intrinsics coarse_intrinsics(const relo_intrinsics& in) {
  relo_intrinsics c = in;
  c.width = in.width / 8;
  c.height = in.height / 8;
  c.fx = in.fx / 8.0;
  c.fy = in.fy / 8.0;
  c.cx = (in.cx - 4.0) / 8.0;
  c.cy = (in.cy - 4.0) / 8.0;
  return c;
}
}  // namespace

extern "C" {

size_t relo_regressor_relocalise_workspace_size(int32_t W, int32_t H, const relo_ransac_params* p) {
  if (!p || W < 8 || H < 8 || W % 8 || H % 8) return 0;
  LearnedLayout l;
  learned_layout(nullptr, W, H, *p, l);
  return l.bytes;
}

relo_status relo_regressor_relocalise(relo_regressor* r, const uint16_t* depth, const uint8_t* rgba,
                                      const relo_intrinsics* intr, const relo_ransac_params* p, void* ws,
                                      size_t ws_bytes, relo_pose_result* result, relo_stream stream) {
  if (!r || !depth || !rgba || !intr || !p || !ws || !result) return fail(RELO_EINVAL, "null argument");
  relo_status st = reg_check_size(1, intr->width, intr->height);
  if (st) return st;
  st = check_params(p);
  if (st) return st;
  if (((uintptr_t)ws & 255) != 0) return fail(RELO_EINVAL, "workspace must be 256-byte aligned");
  LearnedLayout l;
  learned_layout(nullptr, intr->width, intr->height, *p, l);
  if (l.bytes > ws_bytes) return fail(RELO_EINVAL, "workspace too small");
  learned_layout((char*)ws, intr->width, intr->height, *p, l);
  cudaStream_t s = (cudaStream_t)stream;
  st = reg_forward(r, l.reg, depth, rgba, 1, intr->width, intr->height, s);
  if (st) return st;
  return learned_ransac(l, l.reg.head, 8, r->origin, r->d_status, depth, intr, p, ws, ws_bytes, result, s);
}

relo_status relo_regressor_relocalise_cells(const float* cells, const double origin[3], const uint16_t* depth,
                                            const relo_intrinsics* intr, const relo_ransac_params* p, void* ws,
                                            size_t ws_bytes, relo_pose_result* result, relo_stream stream) {
  if (!cells || !origin || !depth || !intr || !p || !ws || !result) return fail(RELO_EINVAL, "null argument");
  relo_status st = check_intr(intr);
  if (st) return st;
  if (intr->width < 8 || intr->height < 8 || intr->width % 8 || intr->height % 8)
    return fail(RELO_EINVAL, "width and height must be positive multiples of 8");
  st = check_params(p);
  if (st) return st;
  if (((uintptr_t)ws & 255) != 0) return fail(RELO_EINVAL, "workspace must be 256-byte aligned");
  LearnedLayout l;
  learned_layout(nullptr, intr->width, intr->height, *p, l);
  if (l.bytes > ws_bytes) return fail(RELO_EINVAL, "workspace too small");
  learned_layout((char*)ws, intr->width, intr->height, *p, l);
  return learned_ransac(l, cells, 4, origin, nullptr, depth, intr, p, ws, ws_bytes, result, (cudaStream_t)stream);
}

}  // extern "C"

namespace {
// The learned path's RANSAC from cell outputs (scene coordinate - origin, log-variance; ostride
// floats per cell): the cell forest, the coarse view, then the RANSAC of one view.
relo_status learned_ransac(const LearnedLayout& l, const float* cells, int ostride, const double origin[3],
                           const int32_t* upstream, const uint16_t* depth, const relo_intrinsics* intr,
                           const relo_ransac_params* p, void* ws, size_t ws_bytes, relo_pose_result* result,
                           cudaStream_t s) {
  CellForestArgs ca{};
  ca.out = cells;
  ca.ostride = ostride;
  ca.depth = depth;
  ca.n = 1;
  ca.W = intr->width;
  ca.H = intr->height;
  ca.Wc = intr->width / 8;
  ca.Hc = intr->height / 8;
  ca.L = l.L;
  ca.ox = (float)origin[0];
  ca.oy = (float)origin[1];
  ca.oz = (float)origin[2];
  ca.modes = l.modes;
  ca.n_modes = l.n_modes;
  ca.top = l.top;
  ca.leaves = l.leaves;
  ca.depth_lr = l.depth_lr;
  RELO_CUDA(launch_cell_forest(ca, s));
  ForestView fv{};
  fv.modes = l.modes;
  fv.n_modes = l.n_modes;
  fv.top = l.top;
  fv.T = 1;
  fv.D = l.D;
  fv.M = 1;
  const relo_intrinsics ci = coarse_intrinsics(*intr);
  Single sr;
  const relo_status st =
      single_setup_view(fv, l.depth_lr, l.leaves, &ci, p, (char*)ws + l.ransac_off, ws_bytes - l.ransac_off, sr);
  if (st) return st;
  sr.job.upstream = upstream;
  return single_run(sr, p, result, s);
}
}  // namespace

// =============================================================================================
// Batches of whole attempts (Fig. 3 end to end).  Pass L (learned attempts): regressor forward,
// cell forests, RANSAC on the cell grids, verification.  Pass F (forest attempts and the forest
// fallbacks of learned attempts): forest evaluation, RANSAC, verification -- a fallback job skips
// every stage on the device when its learned pose verified.  A merge kernel writes each attempt's
// final result.  Every stage is one launch over all jobs of its pass.
// =============================================================================================
namespace {
constexpr int kStages = 10;
const char* const kStageNames[kStages] = {"query_raycast",   "learned_forward", "learned_hypotheses",
                                          "learned_rounds",  "learned_verify",  "forest_eval",
                                          "forest_hypotheses", "forest_rounds", "forest_verify",
                                          "merge"};
}  // namespace

struct relo_batch {
  int n = 0, nL = 0, nF = 0;
  RayJob* d_query = nullptr;
  RayJob* d_verify_L = nullptr;
  RayJob* d_verify_F = nullptr;
  ForestJob* d_forest = nullptr;
  RansacPass passL, passF;
  relo_pose_result* d_res_L = nullptr;
  relo_pose_result* d_res_F = nullptr;
  relo_pose_result* d_res = nullptr;
  int32_t* d_kind = nullptr;
  int32_t* d_errs = nullptr;  // nL + nF words
  int query_tiles = 0, verify_L_tiles = 0, verify_F_tiles = 0, max_trees = 1;
  bool query_apron = false, verify_apron = false;  // every query / verification scene has its apron copy
  int64_t forest_pixels = 0;
  // learned pass
  relo_regressor* reg = nullptr;
  int lW = 0, lH = 0;
  uint16_t* depth_L = nullptr;  // learned query images [nL][H][W] (contiguous)
  uint32_t* rgba_L = nullptr;
  RegBuffers regbuf;
  CellForestArgs cells{};
  bool timing = false;
  cudaEvent_t ev[kStages + 1] = {};
  Schedule sched;  // launch schedule (relo_batch_set_schedule / relo_batch_autotune)
  // the persistent schedule's item lists, built and uploaded the first time it is chosen
  std::vector<int> KL, KF;  // hypotheses per job of each pass
  int batch_pixels = 0;
  bool stall_items = false;
  bool items_uploaded = false;
  // per attempt: its query images and forest leaves inside the workspace (for inspection)
  std::vector<uint16_t*> a_depth, a_leaves;
  std::vector<uint32_t*> a_rgba;
  // the captured run (relo_batch_capture)
  cudaGraphExec_t graph = nullptr;
  ~relo_batch() {
    for (cudaEvent_t& e : ev)
      if (e) cudaEventDestroy(e);
    if (graph) cudaGraphExecDestroy(graph);
  }
};

namespace {

relo_status check_attempts(const relo_attempt* at, int n, const relo_ransac_params* p) {
  if (!at || n < 1) return fail(RELO_EINVAL, "need at least one attempt");
  relo_status st = check_params(p);
  if (st) return st;
  const relo_regressor* reg = nullptr;
  int lw = 0, lh = 0;
  for (int i = 0; i < n; ++i) {
    const relo_attempt& a = at[i];
    if (!a.scene_b || !a.scene_a) return fail(RELO_EINVAL, "attempt has a null scene");
    if (!a.forest_a && !a.regressor_a) return fail(RELO_EINVAL, "attempt has neither a forest nor a regressor");
    st = check_intr(&a.intr);
    if (st) return st;
    if (bad_pose(a.pose_b)) return fail(RELO_EINVAL, "attempt pose_b is not finite");
    if (a.n_hyps < 0 || a.n_hyps > 4096) return fail(RELO_EINVAL, "attempt n_hyps outside [0, 4096]");
    if (a.regressor_a) {
      st = reg_check_size(1, a.intr.width, a.intr.height);
      if (st) return st;
      if (reg && (a.regressor_a != reg || a.intr.width != lw || a.intr.height != lh))
        return fail(RELO_EINVAL, "learned attempts of a batch must share one regressor and one image size");
      reg = a.regressor_a;
      lw = a.intr.width;
      lh = a.intr.height;
    }
  }
  return RELO_OK;
}

struct HostJobs {
  std::vector<RayJob> query, verify_L, verify_F;
  std::vector<ForestJob> forest;
  std::vector<RansacJob> ransac_L, ransac_F;
  std::vector<int32_t> alive_L, surv_L, alive_F, surv_F, kind;
};

// Lays out (base == nullptr: sizes only) the workspace of a batch and fills the host job arrays.
void layout_batch(const relo_attempt* at, int n, const relo_ransac_params& p, char* base, size_t* bytes,
                  relo_batch& b, HostJobs& h) {
  // attempt kinds and the learned group
  std::vector<int> kind(n), iL(n, -1), iF(n, -1);
  int nL = 0, nF = 0, lW = 0, lH = 0;
  relo_regressor* reg = nullptr;
  for (int i = 0; i < n; ++i) {
    kind[i] = at[i].regressor_a ? (at[i].forest_a ? 2 : 1) : 0;
    if (kind[i] != 0) {
      iL[i] = nL++;
      reg = const_cast<relo_regressor*>(at[i].regressor_a);
      lW = at[i].intr.width;
      lH = at[i].intr.height;
    }
    if (kind[i] != 1) iF[i] = nF++;
  }
  Carver c{base, 0};
  b.n = n;
  b.nL = nL;
  b.nF = nF;
  b.d_query = c.take<RayJob>(n);
  b.d_verify_L = c.take<RayJob>(std::max(nL, 1));
  b.d_verify_F = c.take<RayJob>(std::max(nF, 1));
  b.d_forest = c.take<ForestJob>(std::max(nF, 1));
  b.passL.d_jobs = c.take<RansacJob>(std::max(nL, 1));
  b.passF.d_jobs = c.take<RansacJob>(std::max(nF, 1));
  b.passL.d_counter = c.take<int32_t>(1);
  b.passF.d_counter = c.take<int32_t>(1);
  b.d_res_L = c.take<relo_pose_result>(n);
  b.d_res_F = c.take<relo_pose_result>(n);
  b.d_res = c.take<relo_pose_result>(n);
  b.d_kind = c.take<int32_t>(n);
  b.d_errs = c.take<int32_t>(nL + nF + 1);
  std::vector<int> KL, KF;
  for (int i = 0; i < n; ++i) {
    const int K = at[i].n_hyps > 0 ? at[i].n_hyps : p.n_hyps;
    if (iL[i] >= 0) KL.push_back(K);
    if (iF[i] >= 0) KF.push_back(K);
  }
  int RL = 0, RF = 0;
  for (int K : KL) RL = std::max(RL, rounds_for(K));
  for (int K : KF) RF = std::max(RF, rounds_for(K));
  b.passL.d_alive_prefix = c.take<int32_t>((size_t)std::max(RL, 1) * (nL + 1));
  b.passL.d_surv_prefix = c.take<int32_t>((size_t)std::max(RL, 1) * (nL + 1));
  b.passF.d_alive_prefix = c.take<int32_t>((size_t)std::max(RF, 1) * (nF + 1));
  b.passF.d_surv_prefix = c.take<int32_t>((size_t)std::max(RF, 1) * (nF + 1));
  // the persistent schedule's items and counters (used when the schedule asks for it)
  // (the lists themselves are built when the persistent schedule is first chosen)
  {
    int nd = 0;
    count_items(KL, p.batch, &b.passL.n_items, &nd, &b.passL.final_base);
    b.passL.ctrl_words = 4 + nd;
    b.passL.d_items = c.take<PItem>(std::max(b.passL.n_items, 1));
    b.passL.d_ctrl = c.take<int32_t>(b.passL.ctrl_words);
    count_items(KF, p.batch, &b.passF.n_items, &nd, &b.passF.final_base);
    b.passF.ctrl_words = 4 + nd;
    b.passF.d_items = c.take<PItem>(std::max(b.passF.n_items, 1));
    b.passF.d_ctrl = c.take<int32_t>(b.passF.ctrl_words);
    b.KL = KL;
    b.KF = KF;
    b.batch_pixels = p.batch;
    b.stall_items = g_persist_stall.load();
  }
  // learned images first (contiguous for the batched forward), then the rest
  uint16_t* depth_L = nullptr;
  uint32_t* rgba_L = nullptr;
  const int Wc = lW / 8, Hc = lH / 8, cells = Wc * Hc;
  int D = 1;
  while ((1 << D) < cells) ++D;
  const int Lv = 1 << D;
  if (nL > 0) {
    depth_L = c.take<uint16_t>((size_t)nL * lW * lH);
    rgba_L = c.take<uint32_t>((size_t)nL * lW * lH);
    b.reg = reg;
    b.lW = lW;
    b.lH = lH;
    b.depth_L = depth_L;
    b.rgba_L = rgba_L;
    RegBuffers rb;
    reg_layout(nullptr, nL, lW, lH, false, rb);
    char* rbase = c.take<char>(rb.bytes);
    reg_layout(rbase, nL, lW, lH, false, b.regbuf);
    CellForestArgs& ca = b.cells;
    ca = CellForestArgs{};
    ca.out = b.regbuf.head;
    ca.depth = depth_L;
    ca.n = nL;
    ca.W = lW;
    ca.H = lH;
    ca.Wc = Wc;
    ca.Hc = Hc;
    ca.L = Lv;
    ca.ox = (float)reg->origin[0];
    ca.oy = (float)reg->origin[1];
    ca.oz = (float)reg->origin[2];
    ca.modes = c.take<float>((size_t)nL * Lv * kModeFloats);
    ca.n_modes = c.take<uint8_t>((size_t)nL * Lv);
    ca.top = c.take<float4>((size_t)nL * Lv);
    ca.leaves = c.take<uint16_t>((size_t)nL * cells);
    ca.depth_lr = c.take<uint16_t>((size_t)nL * cells);
  }
  h = HostJobs{};
  b.a_depth.assign(n, nullptr);
  b.a_rgba.assign(n, nullptr);
  b.a_leaves.assign(n, nullptr);
  h.query.assign(n, RayJob{});
  h.verify_L.assign(nL, RayJob{});
  h.verify_F.assign(nF, RayJob{});
  h.forest.assign(nF, ForestJob{});
  h.ransac_L.assign(nL, RansacJob{});
  h.ransac_F.assign(nF, RansacJob{});
  h.kind.assign(kind.begin(), kind.end());
  int qt = 0, vtL = 0, vtF = 0, chL = 0, chF = 0, hyL = 0, hyF = 0, maxT = 1;
  int64_t fpix = 0;
  for (int i = 0; i < n; ++i) {
    const relo_attempt& a = at[i];
    const int W = a.intr.width, H = a.intr.height, K = a.n_hyps > 0 ? a.n_hyps : p.n_hyps;
    const size_t n_pix = (size_t)W * H;
    uint16_t* depth;
    uint32_t* rgba;
    if (iL[i] >= 0) {
      depth = depth_L ? depth_L + (size_t)iL[i] * n_pix : nullptr;
      rgba = rgba_L ? rgba_L + (size_t)iL[i] * n_pix : nullptr;
    } else {
      depth = c.take<uint16_t>(n_pix);
      rgba = c.take<uint32_t>(n_pix);
    }
    b.a_depth[i] = depth;
    b.a_rgba[i] = rgba;
    RayJob& q = h.query[i];
    q = make_ray_job(a.scene_b->view, a.intr, a.pose_b);
    q.noise = a.noise_dev;
    q.depth = depth;
    q.rgba = rgba;
    q.tile_begin = qt;
    qt += ray_tiles(W, H);
    if (iL[i] >= 0) {
      const int j = iL[i];
      ForestView fv{};
      fv.modes = b.cells.modes ? b.cells.modes + (size_t)j * Lv * kModeFloats : nullptr;
      fv.n_modes = b.cells.n_modes ? b.cells.n_modes + (size_t)j * Lv : nullptr;
      fv.top = b.cells.top ? b.cells.top + (size_t)j * Lv : nullptr;
      fv.T = 1;
      fv.D = D;
      fv.M = 1;
      const relo_intrinsics ci = coarse_intrinsics(a.intr);
      RansacJob& r = h.ransac_L[j];
      fill_ransac_job(r, fv, b.cells.depth_lr ? b.cells.depth_lr + (size_t)j * cells : nullptr,
                      b.cells.leaves ? b.cells.leaves + (size_t)j * cells : nullptr, ci, p, K, a.seed);
      carve_ransac(c, r, Wc, Hc, K, p.batch, r.n_rounds, 1);
      r.vW = W;
      r.vH = H;
      r.err = b.d_errs + j;
      r.upstream = reg->d_status;
      r.result = b.d_res_L + i;
      r.chunk_begin = chL;
      r.hyp_begin = hyL;
      r.has_pose_b = 1;
      for (int k = 0; k < 16; ++k) r.pose_b[k] = a.pose_b[k];
      chL += (cells + kCompactChunk - 1) / kCompactChunk;
      hyL += K;
      RayJob& v = h.verify_L[j];
      v = make_ray_job(a.scene_a->view, a.intr, nullptr);
      v.pose_dev = b.d_res_L[i].pose_c2s;
      v.status_dev = &b.d_res_L[i].status;
      v.depth_ref = depth;
      v.counts = (unsigned long long*)&b.d_res_L[i].omega_a;
      v.err = r.err;
      v.tile_begin = vtL;
      vtL += ray_tiles(W, H);
    }
    if (iF[i] >= 0) {
      const int j = iF[i];
      const int T = a.forest_a->T;
      maxT = std::max(maxT, T);
      uint16_t* leaves = c.take<uint16_t>(n_pix * T);
      b.a_leaves[i] = leaves;
      // the query raycast also writes the image packed per pixel, which the forest reads
      uint2* packed = c.take<uint2>(n_pix);
      h.query[i].packed = packed;
      const int32_t* skip = kind[i] == 2 ? &b.d_res_L[i].verified : nullptr;
      ForestJob& f = h.forest[j];
      f.forest = a.forest_a->view;
      f.depth = depth;
      f.rgba = rgba;
      f.packed = packed;
      f.leaves = leaves;
      f.W = W;
      f.H = H;
      f.pixel_begin = fpix;
      f.skip = skip;
      fpix += forest_slots(W, H);  // a forest CTA never spans two jobs, in any schedule
      RansacJob& r = h.ransac_F[j];
      fill_ransac_job(r, a.forest_a->view, depth, leaves, a.intr, p, K, a.seed);
      carve_ransac(c, r, W, H, K, p.batch, r.n_rounds, T);
      // one error word per attempt: a learned attempt's forest fallback shares the learned word
      r.err = iL[i] >= 0 ? b.d_errs + iL[i] : b.d_errs + nL + j;
      r.result = b.d_res_F + i;
      r.chunk_begin = chF;
      r.hyp_begin = hyF;
      r.has_pose_b = 1;
      r.skip = skip;
      for (int k = 0; k < 16; ++k) r.pose_b[k] = a.pose_b[k];
      chF += (int)((n_pix + kCompactChunk - 1) / kCompactChunk);
      hyF += K;
      RayJob& v = h.verify_F[j];
      v = make_ray_job(a.scene_a->view, a.intr, nullptr);
      v.pose_dev = b.d_res_F[i].pose_c2s;
      v.status_dev = &b.d_res_F[i].status;
      v.depth_ref = depth;
      v.counts = (unsigned long long*)&b.d_res_F[i].omega_a;
      v.err = r.err;
      v.tile_begin = vtF;
      vtF += ray_tiles(W, H);
    }
  }
  for (int i = 0; i < n; ++i)  // the query raycast reports bound failures into the attempt's error word
    h.query[i].err = iL[i] >= 0 ? b.d_errs + iL[i] : (iF[i] >= 0 ? b.d_errs + nL + iF[i] : nullptr);
  b.query_tiles = qt;
  b.verify_L_tiles = vtL;
  b.verify_F_tiles = vtF;
  b.query_apron = b.verify_apron = true;
  for (int i = 0; i < n; ++i) {
    b.query_apron = b.query_apron && h.query[i].scene.tsdf9 != nullptr;
    b.verify_apron = b.verify_apron && at[i].scene_a->view.tsdf9 != nullptr;
  }
  b.forest_pixels = fpix;
  b.max_trees = maxT;
  b.passL.n = nL;
  b.passL.R = RL;
  b.passL.chunks = chL;
  b.passL.hyps = hyL;
  b.passF.n = nF;
  b.passF.R = RF;
  b.passF.chunks = chF;
  b.passF.hyps = hyF;
  round_tables(KL, std::max(RL, 1), h.alive_L, h.surv_L, b.passL.tot_alive, b.passL.tot_surv, b.passL.max_alive,
               b.passL.max_surv);
  round_tables(KF, std::max(RF, 1), h.alive_F, h.surv_F, b.passF.tot_alive, b.passF.tot_surv, b.passF.max_alive,
               b.passF.max_surv);
  b.passL.B = b.passF.B = p.batch;
  for (RansacPass* q : {&b.passL, &b.passF}) {
    q->tot_alive.resize(q->R);
    q->tot_surv.resize(q->R);
    q->max_alive.resize(q->R);
    q->max_surv.resize(q->R);
  }
  *bytes = c.off;
}

template <class T>
cudaError_t upload(T* dst, const std::vector<T>& v) {
  return v.empty() ? cudaSuccess : cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t mark(relo_batch* b, int k, cudaStream_t s, bool capturing) {
  return b->timing ? record(b->ev[k], s, capturing) : cudaSuccess;
}

// Every launch of one run, in stream order, with no host synchronisation (capturable).  While
// capturing, the stage-timing events become event-record nodes of the graph.
relo_status issue_batch(relo_batch* b, relo_pose_result* results, cudaStream_t s, bool capturing) {
  int L = 0;
  RELO_CUDA(cudaMemsetAsync(b->d_errs, 0, (b->nL + b->nF + 1) * sizeof(int32_t), s));
  RELO_CUDA(launch_init_results(b->d_res_F, b->n, s));
  RELO_CUDA(mark(b, 0, s, capturing));
  RELO_CUDA(launch_raycast(b->d_query, b->n, nullptr, b->query_tiles, true, false, s, b->sched, b->query_apron));
  L += 2;
  RELO_CUDA(mark(b, 1, s, capturing));
  // pass L: learned attempts
  if (b->nL > 0) {
    relo_status st = reg_forward(b->reg, b->regbuf, b->depth_L, (const uint8_t*)b->rgba_L, b->nL, b->lW, b->lH, s);
    if (st) return st;
    RELO_CUDA(launch_cell_forest(b->cells, s));
    L += 1 + kRegLayers + 1;
  }
  RELO_CUDA(mark(b, 2, s, capturing));
  const bool ev = b->timing;
  relo_status st = run_pass(b->passL, s, &L, ev ? b->ev[3] : nullptr, ev ? b->ev[4] : nullptr, capturing, b->sched);
  if (st) return st;
  if (b->nL > 0) {
    RELO_CUDA(launch_raycast(b->d_verify_L, b->nL, nullptr, b->verify_L_tiles, false, true, s, b->sched,
                             b->verify_apron));
    RELO_CUDA(launch_verify_decide(b->passL.d_jobs, b->nL, s));
    L += 2;
  }
  RELO_CUDA(mark(b, 5, s, capturing));
  // pass F: forest attempts and fallbacks (skipped on the device where the learned pose verified)
  if (b->nF > 0) {
    RELO_CUDA(launch_forest(b->d_forest, b->nF, nullptr, b->forest_pixels, s, b->max_trees, b->sched));
    L += 1;
  }
  RELO_CUDA(mark(b, 6, s, capturing));
  st = run_pass(b->passF, s, &L, ev ? b->ev[7] : nullptr, ev ? b->ev[8] : nullptr, capturing, b->sched);
  if (st) return st;
  if (b->nF > 0) {
    RELO_CUDA(launch_raycast(b->d_verify_F, b->nF, nullptr, b->verify_F_tiles, false, true, s, b->sched,
                             b->verify_apron));
    RELO_CUDA(launch_verify_decide(b->passF.d_jobs, b->nF, s));
    L += 2;
  }
  RELO_CUDA(mark(b, 9, s, capturing));
  RELO_CUDA(launch_merge_results(b->d_res_L, b->d_res_F, b->d_kind, b->n, b->d_res, s));
  L += 1;
  RELO_CUDA(mark(b, 10, s, capturing));
  if (results && results != b->d_res)
    RELO_CUDA(cudaMemcpyAsync(results, b->d_res, b->n * sizeof(relo_pose_result), cudaMemcpyDeviceToDevice, s));
  return RELO_OK;
}

}  // namespace

extern "C" {

size_t relo_batch_workspace_size(const relo_attempt* at, int32_t n, const relo_ransac_params* p) {
  if (check_attempts(at, n, p) != RELO_OK) return 0;
  relo_batch b;
  HostJobs h;
  size_t bytes = 0;
  layout_batch(at, n, *p, nullptr, &bytes, b, h);
  return bytes;
}

relo_status relo_batch_prepare(const relo_attempt* at, int32_t n, const relo_ransac_params* p, void* ws,
                               size_t ws_bytes, relo_batch** out) {
  if (!out) return fail(RELO_EINVAL, "out is null");
  *out = nullptr;
  relo_status st = check_attempts(at, n, p);
  if (st) return st;
  if (!ws || ((uintptr_t)ws & 255) != 0) return fail(RELO_EINVAL, "workspace must be non-null and 256-byte aligned");
  size_t bytes = 0;
  {
    relo_batch probe;
    HostJobs h;
    layout_batch(at, n, *p, nullptr, &bytes, probe, h);
  }
  if (bytes > ws_bytes) return fail(RELO_EINVAL, "workspace too small");
  int grid = 0;
  RELO_CUDA(persistent_grid(&grid));  // device set-up of the persistent schedule, outside any capture
  relo_batch* b = new relo_batch();
  HostJobs h;
  layout_batch(at, n, *p, (char*)ws, &bytes, *b, h);
  cudaError_t e = upload(b->d_query, h.query);
  if (e == cudaSuccess) e = upload(b->d_verify_L, h.verify_L);
  if (e == cudaSuccess) e = upload(b->d_verify_F, h.verify_F);
  if (e == cudaSuccess) e = upload(b->d_forest, h.forest);
  if (e == cudaSuccess) e = upload(b->passL.d_jobs, h.ransac_L);
  if (e == cudaSuccess) e = upload(b->passF.d_jobs, h.ransac_F);
  if (e == cudaSuccess) e = upload(b->passL.d_alive_prefix, h.alive_L);
  if (e == cudaSuccess) e = upload(b->passL.d_surv_prefix, h.surv_L);
  if (e == cudaSuccess) e = upload(b->passF.d_alive_prefix, h.alive_F);
  if (e == cudaSuccess) e = upload(b->passF.d_surv_prefix, h.surv_F);
  if (e == cudaSuccess) e = upload(b->d_kind, h.kind);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch descriptors");
  }
  *out = b;
  return RELO_OK;
}

relo_status relo_batch_run(relo_batch* b, relo_pose_result* results, relo_stream stream) {
  if (!b) return fail(RELO_EINVAL, "batch not prepared");
  return issue_batch(b, results, (cudaStream_t)stream, false);
}

relo_status relo_batch_capture(relo_batch* b, relo_pose_result* results) {
  if (!b) return fail(RELO_EINVAL, "batch not prepared");
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t cs = nullptr;
  RELO_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  relo_status st = RELO_OK;
  if (e == cudaSuccess) {
    st = issue_batch(b, results, cs, true);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);  // ends the capture even when issuing failed
    if (st == RELO_OK && e2 != cudaSuccess) e = e2;
  }
  if (st == RELO_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (st) return st;
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return cuda_fail(e, "batch graph capture");
  }
  return RELO_OK;
}

relo_status relo_batch_replay(relo_batch* b, relo_stream stream) {
  if (!b || !b->graph) return fail(RELO_EINVAL, "batch has no captured graph");
  RELO_CUDA(cudaGraphLaunch(b->graph, (cudaStream_t)stream));
  return RELO_OK;
}

relo_status relo_batch_attempt_images(const relo_batch* b, int32_t k, const uint16_t** depth_dev,
                                      const uint8_t** rgba_dev, const uint16_t** leaves_dev) {
  if (!b || k < 0 || k >= b->n) return fail(RELO_EINVAL, "attempt index out of range");
  if (depth_dev) *depth_dev = b->a_depth[k];
  if (rgba_dev) *rgba_dev = (const uint8_t*)b->a_rgba[k];
  if (leaves_dev) *leaves_dev = b->a_leaves[k];
  return RELO_OK;
}

int32_t relo_batch_launch_count(const relo_batch* b) {
  if (!b) return 0;
  int L = 2 + 1;  // result init + query raycast, merge
  if (b->nL > 0) L += 1 + kRegLayers + 1 + 2 + pass_launches(b->passL, b->sched);
  if (b->nF > 0) L += 1 + 2 + pass_launches(b->passF, b->sched);
  return L;
}

void relo_batch_destroy(relo_batch* b) { delete b; }

relo_status relo_batch_enable_timing(relo_batch* b, int32_t enable) {
  if (!b) return fail(RELO_EINVAL, "batch is null");
  if (enable) {
    for (cudaEvent_t& e : b->ev)
      if (!e) RELO_CUDA(cudaEventCreate(&e));
  }
  b->timing = enable != 0;
  return RELO_OK;
}

int32_t relo_batch_stage_ms(const relo_batch* b, float* ms, int32_t capacity) {
  if (!b || !b->timing || !ms || capacity < kStages) return 0;
  for (int k = 0; k < kStages; ++k)
    if (cudaEventElapsedTime(&ms[k], b->ev[k], b->ev[k + 1]) != cudaSuccess) return 0;
  return kStages;
}

const char* relo_batch_stage_name(int32_t k) { return (k >= 0 && k < kStages) ? kStageNames[k] : ""; }

// ---- launch schedules and the autotuner ------------------------------------------------------

namespace {
// The persistent schedule's items go to the device the first time a batch may use them.
relo_status ensure_items(relo_batch* b) {
  if (b->items_uploaded) return RELO_OK;
  std::vector<PItem> items_L, items_F;
  int nd = 0, fb = 0;
  build_items(b->KL, b->batch_pixels, b->stall_items, items_L, &nd, &fb);
  build_items(b->KF, b->batch_pixels, b->stall_items, items_F, &nd, &fb);
  if ((int)items_L.size() != b->passL.n_items || (int)items_F.size() != b->passF.n_items)
    return fail(RELO_EINVAL, "persistent schedule: item count mismatch");
  cudaError_t e = upload(b->passL.d_items, items_L);
  if (e == cudaSuccess) e = upload(b->passF.d_items, items_F);
  if (e != cudaSuccess) return cuda_fail(e, "persistent schedule items");
  b->items_uploaded = true;
  return RELO_OK;
}
}  // namespace

relo_status relo_batch_get_schedule(const relo_batch* b, relo_schedule* out) {
  if (!b || !out) return fail(RELO_EINVAL, "null argument");
  out->ray_warp_width = 1 << b->sched.ray_warp_log2w;
  out->forest_threads = b->sched.forest_threads;
  out->forest_tiles = b->sched.forest_tiles;
  out->search_ctas_per_sm = b->sched.search_ctas_per_sm;
  out->refit_per = b->sched.refit_per;
  out->persistent = b->sched.persistent;
  out->forest_smem_levels = b->sched.forest_smem_levels;
  return RELO_OK;
}

relo_status relo_batch_set_schedule(relo_batch* b, const relo_schedule* in) {
  if (!b || !in) return fail(RELO_EINVAL, "null argument");
  Schedule s;
  const int w = in->ray_warp_width;
  if (w != 2 && w != 4 && w != 8 && w != 16) return fail(RELO_EINVAL, "ray_warp_width must be 2, 4, 8 or 16");
  s.ray_warp_log2w = w == 2 ? 1 : w == 4 ? 2 : w == 8 ? 3 : 4;
  if (in->forest_threads != 128 && in->forest_threads != 256) return fail(RELO_EINVAL, "forest_threads must be 128 or 256");
  if (in->forest_tiles != 0 && in->forest_tiles != 1) return fail(RELO_EINVAL, "forest_tiles must be 0 or 1");
  if (in->search_ctas_per_sm < 0 || in->search_ctas_per_sm > 64) return fail(RELO_EINVAL, "search_ctas_per_sm outside [0, 64]");
  if (in->refit_per < 0 || in->refit_per > 32) return fail(RELO_EINVAL, "refit_per outside [0, 32]");
  if (in->persistent != 0 && in->persistent != 1) return fail(RELO_EINVAL, "persistent must be 0 or 1");
  if (in->forest_smem_levels < 0 || in->forest_smem_levels > kMaxSmemLevels)
    return fail(RELO_EINVAL, "forest_smem_levels outside [0, 10]");
  s.persistent = in->persistent;
  if (s.persistent) {
    const relo_status st = ensure_items(b);
    if (st) return st;
  }
  s.forest_threads = in->forest_threads;
  s.forest_tiles = in->forest_tiles;
  s.search_ctas_per_sm = in->search_ctas_per_sm;
  s.refit_per = in->refit_per;
  s.forest_smem_levels = in->forest_smem_levels;
  b->sched = s;
  if (b->graph) {  // the captured launches used the old schedule
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return RELO_OK;
}

// Coordinate descent: each knob in turn takes the candidate whose runs give the smallest total
// time of the stages it affects (the others held at their best so far).  Every candidate
// computes the same results, so the batch may be tuned on its real inputs.
relo_status relo_batch_autotune(relo_batch* b, int32_t repeats, relo_schedule* chosen, relo_stream stream) {
  if (!b || repeats < 1 || repeats > 100) return fail(RELO_EINVAL, "need a batch and repeats in [1, 100]");
  cudaStream_t s = (cudaStream_t)stream;
  const bool had_timing = b->timing;
  relo_status st = ensure_items(b);
  if (st) return st;
  st = relo_batch_enable_timing(b, 1);
  if (st) return st;
  struct Knob {
    int Schedule::*field;
    std::vector<int> values;
    std::vector<int> stages;  // indices into kStageNames whose times the knob changes
  };
  const std::vector<Knob> knobs = {
      {&Schedule::ray_warp_log2w, {3, 4, 2, 1}, {0, 4, 8}},
      {&Schedule::forest_threads, {256, 128}, {5}},
      {&Schedule::forest_tiles, {0, 1}, {5}},
      {&Schedule::forest_smem_levels, {0, 4, 6, 8}, {5}},
      {&Schedule::search_ctas_per_sm, {0, 1, 2, 3}, {2, 6}},
      {&Schedule::refit_per, {0, 1, 4, 16}, {3, 7}},
      {&Schedule::persistent, {0, 1}, {2, 3, 6, 7}},
  };
  Schedule best = b->sched;
  for (const Knob& k : knobs) {
    float best_ms = FLT_MAX;
    int best_v = best.*k.field;
    for (int v : k.values) {
      b->sched = best;
      b->sched.*k.field = v;
      float total = 0.f;
      for (int r = 0; r <= repeats && st == RELO_OK; ++r) {  // run 0 warms up
        st = issue_batch(b, nullptr, s, false);
        if (st == RELO_OK) {
          cudaError_t e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) st = cuda_fail(e, "autotune run");
        }
        if (st == RELO_OK && r > 0) {
          float ms[kStages];
          if (relo_batch_stage_ms(b, ms, kStages) != kStages) st = fail(RELO_ECUDA, "autotune stage times");
          for (int q : k.stages) total += ms[q];
        }
      }
      if (st) break;
      if (total < best_ms) {
        best_ms = total;
        best_v = v;
      }
    }
    if (st) break;
    best.*k.field = best_v;
  }
  b->sched = best;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (!had_timing) b->timing = false;
  if (st) return st;
  return chosen ? relo_batch_get_schedule(b, chosen) : RELO_OK;
}

relo_status relo_relocalise_batch(const relo_attempt* at, int32_t n, const relo_ransac_params* p, void* ws,
                                  size_t ws_bytes, relo_pose_result* results_host, relo_stream stream) {
  if (!results_host) return fail(RELO_EINVAL, "results is null");
  relo_batch* b = nullptr;
  relo_status st = relo_batch_prepare(at, n, p, ws, ws_bytes, &b);
  if (st) return st;
  st = relo_batch_run(b, nullptr, stream);
  if (st == RELO_OK) {
    cudaError_t e = cudaMemcpyAsync(results_host, b->d_res, n * sizeof(relo_pose_result), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) st = cuda_fail(e, "batch results");
  }
  relo_batch_destroy(b);
  return st;
}

}  // extern "C"
