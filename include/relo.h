/*
 * relo.h -- C ABI of the GB300-native inter-agent relocalisation path.
 *
 * Golodetz et al., "Collaborative Large-Scale Dense 3D Reconstruction with
 * Online Inter-Agent Pose Optimisation" (TVCG 2018), Sec. 3.3.1 and Fig. 3:
 * to relate agent b's sub-scene to agent a's, render a synthetic RGB-D view of
 * b's voxel scene from a frame's pose, relocalise that view with a's
 * regression-forest relocaliser (trained as in Cavallari et al., Sec. 3.3 (b)),
 * and accept the proposed pose only if a depth raycast of a's scene from it
 * agrees with b's depth (the Omega_s / mu test of Sec. 3.3.1).  The accepted
 * pose gives the relative transform sample a_T_b of Sec. 3.3.1.
 *
 * Conventions for every entry point:
 *   - Poses are camera->scene, 4x4 row-major double (the inverse of the
 *     paper's f_T_s).  Hence a_T_b = P_a * P_b^-1.
 *   - Images are row-major [H][W]: depth uint16 millimetres (0 = invalid),
 *     colour uint8 RGBA (4 bytes per pixel; alpha 255 where depth is valid).
 *   - "_dev" pointers are CUDA device pointers, "_host" pointers host memory.
 *     The caller owns every buffer it passes and the stream; the library owns
 *     its opaque handles (scene, forest, ...) and the device memory behind them
 *     (from cudaMalloc, or from the caller's allocator: relo_set_allocator).
 *   - Calls are asynchronous on the given stream unless stated otherwise.
 *     Outputs are valid once the stream has synchronised.
 *   - Every call returns RELO_OK (0) or a negative relo_status; on error the
 *     call has launched nothing, and relo_last_error() returns a message
 *     (thread-local).  Kernels never trap: a device-side bounds or wait
 *     failure sets RELO_EDEVICE / RELO_ETIMEOUT in the per-attempt status.
 *   - There is no CPU fallback: every step runs in this library's sm_103a kernels.
 */
#ifndef RELO_H_
#define RELO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* relo_stream; /* same object as cudaStream_t; NULL = legacy default stream */

typedef int relo_status;
#define RELO_OK 0
#define RELO_EINVAL (-1)    /* bad argument (size, pointer, alignment) */
#define RELO_ENOMEM (-2)    /* device allocation failed (creation calls) */
#define RELO_ECUDA (-3)     /* a CUDA runtime call failed */
#define RELO_ETIMEOUT (-4)  /* a bounded device loop gave up */
#define RELO_EDEVICE (-5)   /* a device-side bounds check failed */
#define RELO_ENOTFOUND (-6) /* no valid pose hypothesis */
#define RELO_EBUSY (-7)     /* a serving request was discarded: every request slot is in use */

/* Message for the last failing call on this thread ("" if none). */
const char* relo_last_error(void);

/* Device memory.  By default the library takes the device memory behind its handles (scenes,
 * forests, regressors, batches, servers) and its temporary buffers from cudaMalloc and returns it
 * with cudaFree.  relo_set_allocator routes every later allocation through the caller's functions
 * instead, e.g. a framework's caching allocator, so that one allocator owns and budgets the
 * process's device memory:
 *   alloc(bytes, ctx) returns a device pointer of the current device, aligned to 256 bytes,
 *     usable from any stream, or NULL when it cannot; the library call then fails as it does
 *     when cudaMalloc fails (RELO_ENOMEM from creation calls).  A pointer that is not 256-byte
 *     aligned is handed straight back to free and counts as a failed allocation;
 *   free(ptr, ctx) takes back a pointer that alloc returned.  The library synchronises the
 *     device before it calls free, as cudaFree would, so no launch still uses the block.
 * Each block goes back to the functions that gave it: memory allocated before a change of
 * allocator is still returned to the old one, so the old functions and ctx must stay valid until
 * every handle created under them is destroyed.  alloc and free NULL restore cudaMalloc /
 * cudaFree.  Calls to alloc and free come from the thread of the library call that needs them.
 * Errors: RELO_EINVAL (exactly one of alloc and free is NULL). */
typedef void* (*relo_alloc_fn)(size_t bytes, void* ctx);
typedef void (*relo_free_fn)(void* ptr, void* ctx);
relo_status relo_set_allocator(relo_alloc_fn alloc, relo_free_fn free_fn, void* ctx);

/* Pinhole camera.  The ray through pixel (u, v) is C + lam * R ((u-cx)/fx, (v-cy)/fy, 1),
 * lam = camera-space z, marched over [depth_min, depth_max] metres. */
typedef struct relo_intrinsics {
  int32_t width, height;
  double fx, fy, cx, cy;
  double depth_min, depth_max;
} relo_intrinsics;

/* ---------------------------------------------------------------------------------------
 * Voxel sub-scene (the InfiniTAM-style map of Sec. 3.3 (a); its size, Sec. 4.3.2).
 * Blocks of 8x8x8 voxels: voxel (i,j,k) is the scene point (i,j,k) * voxel_size and lives
 * in block floor((i,j,k) / 8) at local index (i&7) + 8 (j&7) + 64 (k&7).  tsdf is the
 * truncated signed distance / mu in [-1, 1], positive in free space.  Voxels of blocks not
 * in the list read tsdf +1 and colour 0.  Block coordinates must lie in [-32768, 32767];
 * a repeated block coordinate keeps its first occurrence.  The library builds a spatial
 * hash with 2^log2_buckets buckets (chained, entries of 16 bytes) and copies everything to
 * the device (synchronously; about 4 KB per block plus 16 B per bucket, and 2.9 KB per block
 * for the raycast's apron copy of the tsdf, relo_scene_use_apron).
 * Errors: RELO_EINVAL (n_blocks < 0, null arrays with n_blocks > 0, log2_buckets outside
 * [4, 30], voxel_size or mu <= 0, coordinates out of range), RELO_ENOMEM, RELO_ECUDA.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_scene relo_scene;

relo_status relo_create_scene(const int32_t* coords_host /* [n][3] */, const float* tsdf_host /* [n][512] */,
                              const uint8_t* rgba_host /* [n][512][4] */, int64_t n_blocks, double voxel_size,
                              double mu, int32_t log2_buckets, relo_scene** out);
void relo_destroy_scene(relo_scene* scene);

/* Input index of the block holding each block coordinate (n x int32 xyz, device), -1 where
 * unallocated (the hash lookup used by the raycast).  keys_dev and out_dev are device arrays. */
relo_status relo_scene_lookup(const relo_scene* scene, const int32_t* keys_dev, int64_t n, int64_t* out_dev,
                              relo_stream stream);

/* Raycast acceleration (no counterpart in the paper; results are unchanged).  When the blocks'
 * bounding box holds at most 2^28 block coordinates, creation also builds a dense block-index
 * grid over it (4 bytes per coordinate) and one occupancy byte per 8 x 8 x 8 blocks; the raycast
 * then reads block indices from the grid instead of walking the hash, and crosses empty 8^3-block
 * cells in one step.  relo_scene_use_grid(scene, 0) makes later raycasts use the hash alone, 1
 * restores the grid (if one was built).  Errors: RELO_EINVAL (null scene). */
relo_status relo_scene_use_grid(relo_scene* scene, int32_t enable);

/* Raycast acceleration (no counterpart in the paper; results are unchanged).  Creation also
 * builds, on the device, an apron copy of the tsdf: per block 9 x 9 x 9 values (2944 bytes, about
 * 1.44 times the block's own tsdf) whose last plane along each axis repeats the first voxels of
 * the neighbouring block, or +1 where that block is unallocated.  The eight corners of every
 * trilinear sample then lie in one block, so the march never looks up a neighbouring block for a
 * sample on a block's last voxel.  relo_scene_use_apron(scene, 0) makes later raycasts read the
 * blocks' own tsdf (looking neighbours up), 1 restores the copy.  Scenes made by
 * relo_create_fusion_scene have no copy (fusion changes their voxels); the call has no effect on
 * them.  Errors: RELO_EINVAL (null scene). */
relo_status relo_scene_use_apron(relo_scene* scene, int32_t enable);

/* ---------------------------------------------------------------------------------------
 * Synthetic raycast (Sec. 3.3.1, Fig. 3: the query is a colour + depth render of scene b from
 * the frame's pose; the appendix on global map rendering names the usual voxel raycast).
 * March, per ray: start at depth_min; at a sample in an unallocated block the march moves to the
 * block's exit, which becomes the previous sample with f = +1, and samples again 1e-5 (in z)
 * past it; otherwise f = trilinear tsdf, and while f > 0 the next sample is max(f mu, voxel) / |d|
 * further; the first f <= 0 after a positive sample ends the march at the secant root of the last
 * two samples (f <= 0 on the first sample: invalid); the march gives up past depth_max or after
 * 100000 samples.  Depth is the
 * hit's camera z in mm rounded half up, clamped to [1, 65535]; with noise_dev (one standard
 * normal per pixel, float32 [H][W]) 1.5 mm * z^2 * n is added first (the quadratic axial noise
 * model of the appendix on depth sensors).  Colour (rgba_dev may be NULL) is the trilinear
 * voxel colour at the hit, rounded half up.  Computed in FP32.
 * Errors: RELO_EINVAL (null scene/intrinsics/pose/depth, width or height outside [1, 16384], a pose
 * entry that is not finite).
 * ------------------------------------------------------------------------------------- */
relo_status relo_raycast_view(const relo_scene* scene, const relo_intrinsics* intr, const double pose_c2s[16],
                              const float* noise_dev, uint16_t* depth_dev, uint8_t* rgba_dev, relo_stream stream);

/* n views of one scene in one launch (the same raycast as relo_raycast_view for each view):
 * poses_c2s_host [n][16]; noise_dev nullable, [n][H][W]; depth_dev [n][H][W]; rgba_dev nullable,
 * [n][H][W][4].  The per-view descriptors are copied from host memory to workspace_dev (device,
 * 256-byte aligned, at least relo_raycast_views_workspace_size(n) bytes) on the stream, which
 * may wait for the stream's earlier work; the renders themselves are not waited for.
 * Errors: RELO_EINVAL (as relo_raycast_view, n < 1, workspace). */
size_t relo_raycast_views_workspace_size(int32_t n);
relo_status relo_raycast_views(const relo_scene* scene, const relo_intrinsics* intr, const double* poses_c2s_host,
                               int32_t n, const float* noise_dev, uint16_t* depth_dev, uint8_t* rgba_dev,
                               void* workspace_dev, size_t workspace_bytes, relo_stream stream);

/* Global map rendering (Appendix B.2): the n sub-scenes, placed by their global poses
 * global_poses_host [n][16] (gT_a: scene a -> global, rigid, e.g. from relo_pose_graph_optimise),
 * seen by one camera with camera -> global pose pose_global_host.  Each scene a is raycast as
 * relo_raycast_view does (no noise) from its local pose (gT_a)^-1 * pose_global; per pixel the
 * scene with the smallest depth in whole mm wins (ties: the lower index) and gives the pixel its
 * depth (depth_dev u16 mm, 0 where no scene is hit) and colour (rgba_dev, nullable); owner_dev
 * (nullable, int8 [H][W]) receives the winning index or -1.  err_dev (nullable, device int32)
 * is set to RELO_EDEVICE if a hash walk exceeded its bound.  One launch; the descriptors go
 * through workspace_dev (256-byte aligned, relo_render_global_workspace_size(n) bytes) as for
 * relo_raycast_views.  Errors: RELO_EINVAL (null, n outside [1, 64], intrinsics, a pose entry that is
 * not finite, workspace). */
size_t relo_render_global_workspace_size(int32_t n_scenes);
relo_status relo_render_global(const relo_scene* const* scenes, const double* global_poses_host, int32_t n_scenes,
                               const relo_intrinsics* intr, const double pose_global_host[16], uint16_t* depth_dev,
                               uint8_t* rgba_dev, int8_t* owner_dev, int32_t* err_dev, void* workspace_dev,
                               size_t workspace_bytes, relo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Scenes that grow by TSDF fusion: each agent's map is built by fusing its posed RGB-D frames
 * (Sec. 3.3 (a), the InfiniTAM pipeline), and the single global model by fusing every agent's
 * frames with their poses moved by the agent's global pose (Appendix B.3).  The standard
 * volumetric fusion (Curless and Levoy 1996) on voxel blocks; rules, all in float32 with each
 * operation rounded to nearest in the order written:
 *  - depth z = D * 0.001 m, valid in [depth_min, depth_max];
 *  - allocation: along a valid pixel's ray, the points at camera z = z - mu + k h, h = block
 *    size / 4, k = 0 .. ceil(2 mu / h) (the last clamped to z + mu; z <= 0 skipped): every block
 *    holding one is allocated if new and updated this frame;
 *  - update of each voxel of those blocks (centre at its integer coordinates times the voxel
 *    size): q = R^T (p - t), skipped unless q.z > 0; pixel (floor(fx q.x/q.z + cx + 1/2),
 *    floor(fy q.y/q.z + cy + 1/2)) inside the image with a valid depth d; eta = d - q.z, skipped
 *    if eta < -mu; f = min(1, eta / mu); F = (F w + f) / (w + 1); with colour, each channel
 *    c = floor((c w + c_pixel) / (w + 1) + 1/2) and alpha 255; w = min(w + 1, max_weight).
 *    New blocks start at F = +1, w = 0, colour 0.
 * The scene has no dense grid: raycasts walk its hash.  Block indices follow the order in which
 * the device allocates them; coordinates and contents do not depend on it.
 * ------------------------------------------------------------------------------------- */
/* An empty scene with room for capacity_blocks blocks (tsdf f32, colour u8x4 and weight u16 per
 * voxel: 5 KB per block, allocated now) and 2^log2_buckets buckets.
 * Errors: RELO_EINVAL (capacity outside [1, 2^24], log2_buckets outside [4, 30], voxel_size or mu
 * <= 0, max_weight outside [1, 65535]), RELO_ENOMEM, RELO_ECUDA. */
relo_status relo_create_fusion_scene(int64_t capacity_blocks, double voxel_size, double mu, int32_t log2_buckets,
                                     int32_t max_weight, relo_scene** out);
/* Workspace bytes relo_fuse_frame needs for width x height frames (0 for a bad size). */
size_t relo_fuse_workspace_size(int32_t width, int32_t height);
/* Fuses one frame (depth_dev u16 mm [H][W]; rgba_dev u8 [H][W][4] or NULL) seen from pose_c2s
 * (camera -> scene), asynchronously on the stream, in four launches.  If the block pool, the
 * chain entries (capacity_blocks) or the frame's block set (relo_fuse_workspace_size) run out,
 * the frame is fused into what fits and the scene records RELO_ENOMEM (relo_scene_block_count).
 * Errors: RELO_EINVAL (null, a scene not created for fusion, intrinsics, a pose entry that is not
 * finite, workspace). */
relo_status relo_fuse_frame(relo_scene* scene, const relo_intrinsics* intr, const double pose_c2s[16],
                            const uint16_t* depth_dev, const uint8_t* rgba_dev, void* workspace_dev,
                            size_t workspace_bytes, relo_stream stream);
/* n frames fused in order in one call (the host issues every launch, so a frame's launches are not
 * held up by the caller): poses_c2s_host [n][16], depth_dev [n][H][W], rgba_dev [n][H][W][4] or
 * NULL.  Same rules and errors as relo_fuse_frame; stops at the first frame that is rejected. */
relo_status relo_fuse_frames(relo_scene* scene, const relo_intrinsics* intr, const double* poses_c2s_host,
                             int32_t n, const uint16_t* depth_dev, const uint8_t* rgba_dev, void* workspace_dev,
                             size_t workspace_bytes, relo_stream stream);
/* The last frame fused with this workspace (of width x height frames): blocks it updated and blocks
 * it created.  Synchronises the device.  Errors: RELO_EINVAL (null workspace, bad size). */
relo_status relo_fuse_stats(const void* workspace_dev, int32_t width, int32_t height, int32_t* visible,
                            int32_t* created);
/* Block updates (blocks updated, summed over the frames fused so far).  Synchronises the device.
 * Errors: RELO_EINVAL (null, not a fusion scene). */
relo_status relo_scene_fusion_updates(const relo_scene* scene, uint64_t* updates);
/* Blocks in the scene (synchronises the device).  Returns RELO_ENOMEM if a fusion ran out of room. */
relo_status relo_scene_block_count(const relo_scene* scene, int64_t* n_blocks);
/* Copies a fusion scene's blocks to host arrays of at least capacity blocks (any may be NULL):
 * coords [n][3], tsdf [n][512], rgba [n][512][4], weight [n][512]; *n_out = n.  Synchronous.
 * Errors: RELO_EINVAL (null, not a fusion scene, capacity < n); RELO_ENOMEM as above (the copy is
 * still made). */
relo_status relo_scene_export(const relo_scene* scene, int32_t* coords_host, float* tsdf_host, uint8_t* rgba_host,
                              uint16_t* weight_host, int64_t capacity, int64_t* n_out);

/* ---------------------------------------------------------------------------------------
 * Regression forest (the relocaliser of Sec. 3.3 (b), after Cavallari et al.).
 * n_trees complete binary trees of the given depth, stored breadth first (children of node n
 * at 2n+1, 2n+2), 2^depth - 1 split nodes of 16 bytes each:
 *   {int16 dx1, dy1, dx2, dy2; uint8 kind, c1, c2, pad; int32 tau}.
 * At a pixel x with depth d mm > 0 each probe is q = x + trunc(delta * 1000 / d) per axis
 * (integer division toward zero), clamped to the image; kind 0 compares the probes' depths
 * (0 where invalid), kind 1 compares colour channel c1 of q1 with channel c2 of q2; the pixel
 * goes left iff V(q1) - V(q2) < tau.  Leaf = node - (2^depth - 1).
 * Leaves hold up to max_modes modes of 12 floats: mean xyz, inverse covariance (xx, xy, xz,
 * yy, yz, zz), log(weight) - 0.5 log det(2 pi Sigma), weight, pad; modes sorted by support,
 * mode 0 the most supported.  modes_host / n_modes_host may be NULL (empty leaves) and be
 * filled later by training (relo_forest_train_*).  Copies to the device synchronously.
 * Errors: RELO_EINVAL (n_trees outside [1, 16], depth outside [1, 16], max_modes outside
 * [1, 64], null nodes, a node whose kind is not 0 or 1 or whose channel exceeds 3), RELO_ENOMEM,
 * RELO_ECUDA.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_forest relo_forest;

relo_status relo_create_forest(const void* nodes_host, int32_t n_trees, int32_t depth, const float* modes_host,
                               const uint8_t* n_modes_host, int32_t max_modes, relo_forest** out);
void relo_destroy_forest(relo_forest* forest);

/* Copy the forest's modes / mode counts back to host arrays of the layout above (synchronous). */
relo_status relo_forest_get_modes(const relo_forest* forest, float* modes_host, uint8_t* n_modes_host);

/* Leaf index of every pixel in every tree: leaves_dev [T][H][W] uint16, 0xFFFF where d = 0.
 * Integer-exact.  Errors: RELO_EINVAL (null pointers, W or H outside [1, 16384]). */
relo_status relo_forest_eval(const relo_forest* forest, const uint16_t* depth_dev, const uint8_t* rgba_dev,
                             int32_t width, int32_t height, uint16_t* leaves_dev, relo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Relocaliser training (Sec. 3.3 (b): leaves filled online as per Cavallari et al.).
 * relo_forest_train_frame routes the pixels of one posed training frame on the stride grid
 * (u % stride == 0 and v % stride == 0, depth > 0, raster order) through every tree on the
 * device and offers each pixel's scene coordinate P * backproject(depth) to its leaf's
 * reservoir (Algorithm R, capacity per leaf, Philox4x32-10 draws keyed by seed at counter
 * (3, tree * 2^depth + leaf, n_lo, n_hi) for the n-th offer, n from 0; the offer replaces
 * slot floor(word0 * (n+1) / 2^32) if that is below capacity).  Reservoir updates run on the
 * host in frame order (synchronous call).  relo_forest_train_finish runs mean shift on every
 * leaf (Gaussian kernel of the given bandwidth from every sample, until the shift is below
 * tol or max_iter steps; a converged point joins the first mode whose opening point lies
 * within merge_dist; per mode: mean and covariance of its members + cov_floor I; keep the
 * max_modes most supported, ties by opening order) on the device and replaces the modes.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_train_params {
  int32_t capacity, stride, max_iter, pad;
  uint64_t seed;
  double bandwidth, tol, merge_dist, cov_floor;
} relo_train_params;

relo_status relo_forest_train_begin(relo_forest* forest, const relo_train_params* p);
relo_status relo_forest_train_frame(relo_forest* forest, const relo_intrinsics* intr, const double pose_c2s[16],
                                    const uint16_t* depth_dev, const uint8_t* rgba_dev, relo_stream stream);
relo_status relo_forest_train_finish(relo_forest* forest, relo_stream stream);
/* Reservoir contents (host copies, synchronous): samples [T][2^D][capacity][3], count [T][2^D]. */
relo_status relo_forest_train_reservoirs(const relo_forest* forest, float* samples_host, int32_t* count_host);

/* ---------------------------------------------------------------------------------------
 * Preemptive RANSAC (the relocaliser's pose solver, after Cavallari et al.; paper-silent,
 * readings stated here and identically in the CPU oracle).
 * Hypotheses: hypothesis h tries j = 0..max_tries-1; try j is the Philox4x32-10 block at
 * counter (1, h, j, 0) under key (seed_lo, seed_hi): words 0..2 pick three pixels uniformly
 * among the valid pixels (depth > 0, raster order; floor(w * n / 2^32)), byte k of word 3
 * picks the tree of correspondence k as floor(byte * T / 256), each correspondence uses its
 * leaf's mode 0; the first try whose leaves are non-empty, whose pixels differ, whose three
 * camera/scene distance pairs agree within rigidity metres and whose two triangles have
 * |cross| >= min_area is fitted by Kabsch (FP32 covariance, FP64 rotation).
 * Rounds: while more than one hypothesis is alive, draw batch pixels (with replacement) at
 * counters (2, r, i, 0); add to each alive hypothesis's energy the sum over those pixels of
 * min(-log 1e-30, -max over trees and modes of [logw - 0.5 log det 2 pi Sigma - 0.5 (x-mu)^T
 * Sigma^-1 (x-mu)]), x = R c + t; keep the ceil(n/2) lowest (energy, index); re-fit each
 * survivor by Kabsch on its inliers among all pixels drawn so far (best mode within
 * inlier_dist of x; at least 3 inliers, else the pose is kept).
 * ------------------------------------------------------------------------------------- */
typedef struct relo_ransac_params {
  int32_t n_hyps;       /* K, 1 .. 4096 */
  int32_t batch;        /* B pixels added per round, 1 .. 4096 */
  int32_t max_tries;    /* tries per hypothesis, 1 .. 1 << 24 */
  int32_t pad;
  double rigidity;      /* metres */
  double min_area;      /* square metres */
  double inlier_dist;   /* metres */
  uint64_t seed;
} relo_ransac_params;

/* Result of one attempt (device or host copy; 344 bytes). */
typedef struct relo_pose_result {
  double pose_c2s[16];     /* proposed camera -> scene a pose */
  double rel_a_b[16];      /* a_T_b = P_a P_b^-1 (filled by relo_relocalise_batch) */
  double energy;           /* accumulated energy of the final hypothesis */
  int32_t n_inliers;       /* inliers of its last re-fit */
  int32_t status;          /* RELO_OK, RELO_ENOTFOUND, RELO_EDEVICE, RELO_ETIMEOUT */
  int32_t verified;        /* 1 iff 2 |Omega_a| > |Omega| and |Omega_ab| > 0 and sum < 50 |Omega_ab| */
  int32_t n_valid;         /* valid query pixels */
  int32_t hypothesis;      /* index of the final hypothesis */
  int32_t n_rounds;
  uint64_t omega, omega_a, omega_b, omega_ab, sum_absdiff_mm; /* Sec. 3.3.1 verification counts */
  uint64_t tries;          /* hypothesis tries a sequential scan makes: sum over h of (kept try + 1), or
                              max_tries for a hypothesis without a passing try */
  int32_t path;            /* batches: RELO_PATH_FOREST, RELO_PATH_LEARNED or RELO_PATH_FALLBACK */
  int32_t pad;
} relo_pose_result;

#define RELO_PATH_FOREST 0    /* relocalised with the forest */
#define RELO_PATH_LEARNED 1   /* relocalised (and verified, or without a forest) with the regressor */
#define RELO_PATH_FALLBACK 2  /* the regressor's pose failed verification; the forest's result */

/* Bytes of device workspace relo_ransac_relocalise needs for a width x height view. */
size_t relo_ransac_workspace_size(int32_t width, int32_t height, const relo_ransac_params* p);

/* Relocalise one view: depth_dev + leaves_dev (from relo_forest_eval) -> result_dev (device
 * relo_pose_result; the verification fields are zero).  workspace_dev (256-byte aligned, at
 * least relo_ransac_workspace_size bytes) is scratch the call overwrites.  The call uploads its
 * job descriptor and round tables with cudaMemcpyAsync from host memory that lives only for the
 * call, so it is for eager use: a CUDA graph of relocalisation attempts is recorded with
 * relo_batch_capture, whose uploads happen at relo_batch_prepare.
 * Errors: RELO_EINVAL (bad sizes/params/pointers or workspace too small). */
relo_status relo_ransac_relocalise(const relo_forest* forest, const uint16_t* depth_dev, const uint16_t* leaves_dev,
                                   const relo_intrinsics* intr, const relo_ransac_params* p, void* workspace_dev,
                                   size_t workspace_bytes, relo_pose_result* result_dev, relo_stream stream);

/* Allocation-free variant of relo_ransac_relocalise (the paper has no counterpart; this serves
 * callers, not the method).  Some callers may not allocate device memory when they relocalise:
 * a process whose device memory is owned and budgeted by another allocator, or a latency-bound
 * loop where an allocation could block, synchronise the device or fail under memory pressure.
 * This entry point takes no workspace and allocates nothing: its scratch is one array of
 * RELO_STATIC_SCRATCH_BYTES (8 MiB) compiled into the library, which every GPU that loads the
 * library holds until the process exits.  The caller still passes the inputs and the result.
 * The first call on a device looks the array's device address up (with that device current)
 * and caches it; make that first call before any stream capture.  All calls share the one
 * array, which keeps the last call's contents (each call clears what must start at zero): calls
 * that may overlap on the GPU -- on different streams, or from different host threads -- race,
 * so serialise them.  Results equal relo_ransac_relocalise's for the same inputs.
 * Errors: as relo_ransac_relocalise, plus RELO_EINVAL when the view needs more scratch than the
 * array holds, or the device ordinal is 64 or more.  The scratch a view needs, for a forest of
 * T <= 5 trees, K hypotheses, B pixels per round and R = ceil(log2 K) rounds: 16 bytes per pixel,
 * plus 160 + 128 * ceil(R * B / 64) bytes per hypothesis (the re-fit sums take the second term),
 * plus 68 bytes per drawn pixel (R * B of them), each array rounded up to 256 bytes; e.g.
 * 640 x 480 with K = 1024, B = 64 needs about 6.4 MB and fits, 1280 x 960 does not.
 * relo_ransac_workspace_size(width, height, p) is an upper bound for any forest. */
#define RELO_STATIC_SCRATCH_BYTES (8u << 20)
relo_status relo_ransac_relocalise_noalloc(const relo_forest* forest, const uint16_t* depth_dev,
                                           const uint16_t* leaves_dev, const relo_intrinsics* intr,
                                           const relo_ransac_params* p, relo_pose_result* result_dev,
                                           relo_stream stream);

/* Stage-isolated RANSAC steps (the same kernels as relo_ransac_relocalise), for checking each
 * step against the oracle under teacher forcing.  Workspace as above.
 * relo_ransac_hypotheses: poses_dev [K][12] (row-major R | t, camera -> scene), valid_dev [K],
 * tries_dev [K] (index of the kept try, max_tries if none).
 * relo_ransac_round: one round r from the given state: alive_dev [n_alive] hypothesis indices,
 * poses_dev [K][12] and energy_dev [K] updated in place, drawn_dev [(r+1) * batch] positions in
 * the valid-pixel list (depth > 0, raster order) of the pixels drawn in rounds 0..r (only
 * round r's slice is written), survivors_dev [ceil(n_alive/2)] and inliers_dev [K] written. */
relo_status relo_ransac_hypotheses(const relo_forest* forest, const uint16_t* depth_dev, const uint16_t* leaves_dev,
                                   const relo_intrinsics* intr, const relo_ransac_params* p, void* workspace_dev,
                                   size_t workspace_bytes, double* poses_dev, int32_t* valid_dev, int32_t* tries_dev,
                                   relo_stream stream);
relo_status relo_ransac_round(const relo_forest* forest, const uint16_t* depth_dev, const uint16_t* leaves_dev,
                              const relo_intrinsics* intr, const relo_ransac_params* p, int32_t round,
                              const int32_t* alive_dev, int32_t n_alive, const int32_t* valid_dev, double* poses_dev,
                              double* energy_dev, int32_t* drawn_dev, int32_t* survivors_dev, int32_t* inliers_dev,
                              void* workspace_dev, size_t workspace_bytes, relo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Learned scene-coordinate regressor: an alternative relocaliser for one scene, trained online
 * on renders of its own voxel map (the paper uses a forest, Sec. 3.3 (b); this network and its
 * details are readings of the workload, stated identically in the CPU oracle).
 * Input per pixel: (depth in metres - 3) / 2 (depth 0 where invalid) and (R, G, B / 255 - 1/2)
 * x 4.  Eight 3x3 convolutions (zero padding 1, 64 channels; strides 2, 2, 2, 1, 1, 1, 1, 1;
 * ReLU after layers 1-7) give one cell per 8 x 8 pixels with 4 outputs: the scene coordinate of
 * the cell's centre pixel (8 cx + 4, 8 cy + 4) minus `origin`, and a log-variance s.  Loss: mean
 * over cells whose centre pixel has depth of rho(e) + 1/2 e^2 exp(-s) + 3/2 s, e = |y - y_hat|,
 * rho(e) = sqrt(e^2 + 1e-6 m^2); the gradient holds the error of the variance term fixed (the
 * coordinates follow rho alone).  Adam (0.9, 0.999, 1e-8).  Computed with BF16 tensor-core
 * convolutions accumulating in FP32 (FP32 master weights): the 64 -> 64-channel forward layers on
 * tcgen05 (TMA-fed, TMEM accumulators), the rest with mma.sync.
 * Parameters, flat FP32, per layer l: w [3][3][cin][cout] then b [cout], cin = 4, 64, ...,
 * cout = 64, ..., 4 (relo_regressor_param_count() values in all).  Images must have sides that
 * are multiples of 8.  Errors: RELO_EINVAL (sizes, null pointers, workspace), RELO_ENOMEM.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_regressor relo_regressor;

int64_t relo_regressor_param_count(void);
/* params_host NULL: He-uniform weights drawn from Philox4x32-10 (counter (4, layer, index), key
 * = seed), head weights scaled by 0.1, zero biases. */
relo_status relo_create_regressor(const float* params_host, uint64_t seed, const double origin[3],
                                  relo_regressor** out);
void relo_destroy_regressor(relo_regressor* regressor);
/* Training checkpoint (resume mid-run): the master parameters and Adam's moments m and v (each
 * relo_regressor_param_count() floats; NULL skips one) and Adam's step count.  get synchronises
 * the device; set restores all four, re-derives the BF16 weights the kernels multiply and
 * synchronises, so that training continued from a restored state (on a regressor created with the
 * same origin) gives bit for bit the parameters of uninterrupted training.
 * Errors: RELO_EINVAL (null regressor; for set, a null array or step outside [0, 2^31)). */
relo_status relo_regressor_get_state(const relo_regressor* regressor, float* params_host, float* m_host,
                                     float* v_host, int64_t* step);
relo_status relo_regressor_set_state(relo_regressor* regressor, const float* params_host, const float* m_host,
                                     const float* v_host, int64_t step);
/* Copies of the master parameters and of the last computed gradients (either may be NULL). */
relo_status relo_regressor_get_params(const relo_regressor* regressor, float* params_host, float* grads_host);
/* Workspace bytes for n images of width x height (training != 0: with the backward pass). */
size_t relo_regressor_workspace_size(int32_t n_images, int32_t width, int32_t height, int32_t training);
/* Forward pass: out_dev [n][height/8][width/8][4] (scene coordinate - origin, log-variance). */
relo_status relo_regressor_forward(relo_regressor* regressor, const uint16_t* depth_dev, const uint8_t* rgba_dev,
                                   int32_t n_images, int32_t width, int32_t height, float* out_dev,
                                   void* workspace_dev, size_t workspace_bytes, relo_stream stream);
/* Loss (written to loss_dev, nullable) and gradients of n posed views (camera -> scene poses,
 * host [n][16]); the gradients are kept in the regressor (relo_regressor_get_params). */
relo_status relo_regressor_gradients(relo_regressor* regressor, const uint16_t* depth_dev, const uint8_t* rgba_dev,
                                     int32_t n_images, const relo_intrinsics* intr, const double* poses_host,
                                     float* loss_dev, void* workspace_dev, size_t workspace_bytes,
                                     relo_stream stream);
/* relo_regressor_gradients followed by one Adam step with learning rate lr. */
relo_status relo_regressor_train_step(relo_regressor* regressor, const uint16_t* depth_dev, const uint8_t* rgba_dev,
                                      int32_t n_images, const relo_intrinsics* intr, const double* poses_host,
                                      float lr, float* loss_dev, void* workspace_dev, size_t workspace_bytes,
                                      relo_stream stream);
/* Relocalise one view with the regressor: forward pass, then the preemptive RANSAC of
 * relo_ransac_relocalise on the cell grid (one-tree forest whose leaf is the cell and whose one
 * mode is N(y_hat + origin, exp(s) I); the coarse view holds the cells' centre-pixel depths with
 * intrinsics fx / 8, fy / 8, (cx - 4) / 8, (cy - 4) / 8).  The result's pose is camera -> scene;
 * verify with relo_verify at full resolution. */
size_t relo_regressor_relocalise_workspace_size(int32_t width, int32_t height, const relo_ransac_params* p);
relo_status relo_regressor_relocalise(relo_regressor* regressor, const uint16_t* depth_dev, const uint8_t* rgba_dev,
                                      const relo_intrinsics* intr, const relo_ransac_params* p, void* workspace_dev,
                                      size_t workspace_bytes, relo_pose_result* result_dev, relo_stream stream);

/* The second half of relo_regressor_relocalise on cell outputs the caller supplies instead of the
 * network's (stage isolation, for checking the cell-grid RANSAC against a reference):
 * cells_dev [height/8][width/8][4] float (scene coordinate - origin, log-variance s per cell),
 * origin[3] (host), depth_dev [height][width] mm (the full-resolution view whose cell-centre
 * depths form the coarse view).  Workspace: relo_regressor_relocalise_workspace_size.
 * Errors: RELO_EINVAL (null argument, width or height not a positive multiple of 8, bad params,
 * misaligned or small workspace). */
relo_status relo_regressor_relocalise_cells(const float* cells_dev, const double origin[3], const uint16_t* depth_dev,
                                            const relo_intrinsics* intr, const relo_ransac_params* p,
                                            void* workspace_dev, size_t workspace_bytes, relo_pose_result* result_dev,
                                            relo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Depth-difference verification (Sec. 3.3.1): raycast scene a's depth from the proposed pose
 * in result_dev->pose_c2s and compare with depth_b_dev; writes omega (= W H), omega_a,
 * omega_b, omega_ab, sum_absdiff_mm and verified into result_dev (integer-exact).
 * depth_a_dev (nullable) receives scene a's depth.  A result whose status is not RELO_OK is
 * left unverified.
 * ------------------------------------------------------------------------------------- */
relo_status relo_verify(const relo_scene* scene_a, const relo_intrinsics* intr, const uint16_t* depth_b_dev,
                        relo_pose_result* result_dev, uint16_t* depth_a_dev, relo_stream stream);

/* ---------------------------------------------------------------------------------------
 * A batch of whole attempts (Fig. 3 end to end: raycast b, forest of a, RANSAC, verify
 * against a), all stages batched across attempts in one launch per stage.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_attempt {
  const relo_scene* scene_b;
  const relo_forest* forest_a;        /* nullable when regressor_a is set (then no fallback) */
  const relo_scene* scene_a;
  relo_intrinsics intr;
  double pose_b[16];        /* camera -> scene b pose of the query frame */
  const float* noise_dev;   /* nullable: per-pixel standard normals for the query depth */
  int32_t n_hyps;           /* overrides p->n_hyps when > 0 */
  int32_t pad;
  uint64_t seed;            /* Philox key of this attempt's RANSAC */
  const relo_regressor* regressor_a;  /* nullable: relocalise with a's regressor first (learned path) */
} relo_attempt;

/* Learned attempts (regressor_a set): the regressor's RANSAC runs on the cell grid (as in
 * relo_regressor_relocalise) and its pose is verified; when verification fails and forest_a is
 * set, the forest path runs for that attempt in the same launch sequence (each forest stage
 * skips, on the device, the attempts whose learned pose verified) and its result is reported.
 * All learned attempts of a batch must share one regressor and one image size.
 * Workspace bytes for a batch (includes the query images and per-attempt RANSAC scratch). */
size_t relo_batch_workspace_size(const relo_attempt* attempts_host, int32_t n, const relo_ransac_params* p);

/* Run n attempts.  results_host receives n results (the call synchronises the stream).  A bad
 * attempt is one with a null scene, neither forest nor regressor, bad intrinsics, a pose_b entry
 * that is not finite, n_hyps outside [0, 4096], or learned attempts that differ in regressor or
 * image size.  An attempt's status is RELO_EDEVICE when a bounded hash walk of its query or
 * verification raycast, or of its RANSAC, gave up (a corrupted scene table).
 * Errors: RELO_EINVAL (n < 1, bad attempt, workspace too small), RELO_ECUDA. */
relo_status relo_relocalise_batch(const relo_attempt* attempts_host, int32_t n, const relo_ransac_params* p,
                                  void* workspace_dev, size_t workspace_bytes, relo_pose_result* results_host,
                                  relo_stream stream);

/* Device-resident form for timing and graph capture.  relo_batch_prepare lays the batch out in
 * the workspace and copies its descriptors there (synchronous); relo_batch_run launches every
 * stage on the stream with no host synchronisation and no host-side copies, then copies the n
 * results to results_dev; it may be replayed (or captured in a CUDA graph) any number of times
 * while the workspace, scenes and forests live.  relo_batch_launch_count gives the number of
 * kernel launches one run issues.  relo_batch_destroy frees the host-side plan only. */
typedef struct relo_batch relo_batch;
relo_status relo_batch_prepare(const relo_attempt* attempts_host, int32_t n, const relo_ransac_params* p,
                               void* workspace_dev, size_t workspace_bytes, relo_batch** out);
relo_status relo_batch_run(relo_batch* batch, relo_pose_result* results_dev, relo_stream stream);
int32_t relo_batch_launch_count(const relo_batch* batch);
void relo_batch_destroy(relo_batch* batch);

/* One CUDA graph per batch (no counterpart in the paper, whose attempts run one at a time in the
 * background): relo_batch_capture records every launch of one relo_batch_run that writes
 * results_dev (nullable: results stay in the workspace) into a graph owned by the batch,
 * replacing any earlier one; relo_batch_replay launches that graph on a stream, one host call
 * for the whole batch, with the same device work and results as relo_batch_run.  When stage
 * timing was enabled at capture, the graph records the stage events too.  The graph refers to the workspace, scenes, forests, regressor and noise
 * images by address: they must outlive it (relo_batch_destroy frees it).
 * Errors: RELO_EINVAL (null batch, replay before capture), RELO_ECUDA (capture failed). */
relo_status relo_batch_capture(relo_batch* batch, relo_pose_result* results_dev);
relo_status relo_batch_replay(relo_batch* batch, relo_stream stream);

/* Device addresses, inside the workspace, of attempt k's query depth (u16 mm [H][W]), query
 * colour (RGBA u8 [H][W][4]) and forest leaves (u16 [T][H][W]; NULL for an attempt without a
 * forest); their contents are those of the last run (for inspection).  Any output pointer may be
 * NULL.  Errors: RELO_EINVAL (null batch, k outside [0, n)). */
relo_status relo_batch_attempt_images(const relo_batch* batch, int32_t k, const uint16_t** depth_dev,
                                      const uint8_t** rgba_dev, const uint16_t** leaves_dev);

/* Stage timing, for roofline measurements.  Once enabled, relo_batch_run records CUDA events on
 * its stream at the stage boundaries; relo_batch_stage_ms writes the milliseconds each stage of
 * the last run took (call it after that run's stream has synchronised), in this order: query
 * raycast; learned pass: regressor forward and cell forests, compaction + hypotheses, rounds +
 * finalise, verification; forest pass: forest evaluation, compaction + hypotheses, rounds +
 * finalise, verification; merge.  It returns the number of stages written (10), or 0 if timing
 * is off or capacity is too small. */
relo_status relo_batch_enable_timing(relo_batch* batch, int32_t enable);
int32_t relo_batch_stage_ms(const relo_batch* batch, float* ms, int32_t capacity);
/* Name of stage k of relo_batch_stage_ms ("" outside [0, 10)). */
const char* relo_batch_stage_name(int32_t k);

/* Launch schedule of a batch (no counterpart in the paper): how work maps to threads and how
 * large the grids are.  Every schedule computes the same results bit for bit; only the time
 * differs.  A new batch starts with the defaults (8, 256, 0, 0, 0, 0, 0). */
typedef struct relo_schedule {
  int32_t ray_warp_width;     /* raycasts: each warp covers ray_warp_width x (32 / width) pixels of
                                 its CTA's 16 x 16 tile; 2, 4, 8 or 16 */
  int32_t forest_threads;     /* forest evaluation: threads per CTA, 128 or 256 */
  int32_t forest_tiles;       /* forest evaluation: 0 = a CTA takes consecutive row-major pixels,
                                 1 = it takes 32 x 8 pixel tiles */
  int32_t search_ctas_per_sm; /* hypothesis search: persistent CTAs per SM, 0 = as many as fit */
  int32_t refit_per;          /* round re-fits: survivors per one-warp CTA, 1..32; 0 = enough CTAs
                                 for twice the SM count */
  int32_t persistent;         /* RANSAC (search, fits, every round, results) of each pass: 0 = one
                                 launch per stage; 1 = one persistent launch whose CTAs take the
                                 stages of every attempt from a dependency-ordered list, waiting
                                 (bounded in time) on per-attempt counters, so that one attempt's
                                 rounds run while another is still searching.  Same results. */
  int32_t forest_smem_levels; /* forest evaluation: each CTA first copies the top levels of its
                                 forest's trees (up to this many, at most 48 KB) into shared
                                 memory and reads them there; 0..10, 0 = none */
} relo_schedule;
relo_status relo_batch_get_schedule(const relo_batch* batch, relo_schedule* out);
/* Sets the schedule of later runs and drops a captured graph (capture again).
 * Errors: RELO_EINVAL (null, a field outside its values). */
relo_status relo_batch_set_schedule(relo_batch* batch, const relo_schedule* schedule);
/* Autotuner: runs the batch on its own inputs (its results are overwritten by identical ones)
 * 1 + repeats times per candidate value of each field in turn, keeping for each field the value
 * whose runs give the least total time of the stages it affects (stage events, as
 * relo_batch_stage_ms); leaves the batch with the chosen schedule, written to *chosen
 * (nullable), and drops a captured graph.  Synchronises the stream.  Errors: RELO_EINVAL (null
 * batch, repeats outside [1, 100]), RELO_ECUDA. */
relo_status relo_batch_autotune(relo_batch* batch, int32_t repeats, relo_schedule* chosen, relo_stream stream);

/* ---------------------------------------------------------------------------------------
 * Serving: relocalisation attempts submitted one at a time by many agents (threads), run in
 * batches by a worker thread that owns a stream and a workspace.  The paper attempts one
 * relocalisation at a time in the background (Sec. 3.3.1, Sec. 4.3.1); here requests are queued
 * in a fixed pool of slots after the pooled queue of Appendix B.1, with its discard policy: a
 * request that finds every slot in use (queued, running, or finished but not yet collected) is
 * not admitted (RELO_EBUSY).  The worker starts a batch when max_batch requests are queued or
 * the oldest has waited max_wait_us, and takes requests from the front of the queue while the
 * batch's workspace (relo_batch_workspace_size) fits the server's (workspace_bytes, allocated at
 * creation: the HBM budget of one batch).  Latency = collection-ready time - submit time.
 * A request's scenes, forest / regressor and noise image must stay valid until it completes.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_server relo_server;
typedef struct relo_server_params {
  int32_t max_batch;          /* attempts per batch, >= 1 */
  int32_t max_wait_us;        /* a partial batch starts once its oldest request waited this long */
  int32_t slots;              /* request slots (pool size), >= 1 */
  int32_t pad;
  uint64_t workspace_bytes;   /* device workspace of one batch (the HBM budget) */
  relo_ransac_params ransac;  /* for every request (each attempt's n_hyps / seed still apply) */
} relo_server_params;

typedef struct relo_server_stats {
  uint64_t completed, discarded, batches;
  double mean_batch;                     /* requests per batch */
  double p50_ms, p99_ms, max_ms;         /* latency of the completed requests */
} relo_server_stats;

/* Allocates the workspace (cudaMalloc on the current device) and starts the worker.
 * Errors: RELO_EINVAL (params), RELO_ENOMEM, RELO_ECUDA. */
relo_status relo_server_create(const relo_server_params* params, relo_server** out);
/* Queues one attempt (copied); *ticket identifies it.  Errors: RELO_EINVAL (bad attempt: it
 * would be rejected by relo_batch_workspace_size), RELO_EBUSY (discarded, no free slot). */
relo_status relo_server_submit(relo_server* server, const relo_attempt* attempt, uint64_t* ticket);
/* Blocks until the request completes, copies its result (result_host; its status carries any
 * error of the batch it ran in) and latency (nullable), and frees its slot.
 * Errors: RELO_EINVAL (unknown ticket). */
relo_status relo_server_wait(relo_server* server, uint64_t ticket, relo_pose_result* result_host,
                             double* latency_ms);
/* Counters and latency percentiles since creation. */
relo_status relo_server_stats_get(const relo_server* server, relo_server_stats* out);
/* Runs the requests still queued, stops the worker and frees the workspace. */
void relo_server_destroy(relo_server* server);

/* ---------------------------------------------------------------------------------------
 * Pose graph: the host consumer of relative transform samples (Sec. 3.3.2) and the candidate
 * score of Sec. 3.3.1.  Scenes are 0 .. n-1; scene 0 is the first agent's, whose global pose is
 * the identity.  Transforms are row-major 4x4 doubles; aT_b maps scene b's coordinates into
 * scene a's (for a verified attempt, relo_pose_result.rel_a_b).
 * Samples of (a, b) and (b, a) share the unordered pair's clusters.  A sample joins the first
 * cluster holding a sample within 20 degrees and 10 cm of it (Sec. 4.2.4), else opens a new one.
 * A pair is confident once its largest cluster holds N = 2 samples; the pose graph joins the
 * confident pairs of scene 0's connected component, each with the dual-quaternion blend
 * (Kavan et al. 2006, equal weights) of its largest cluster, and Levenberg-Marquardt minimises
 * the squared components of v(gT_b^-1 gT_a aT_b) over its edges (v: imaginary quaternion part,
 * w >= 0, then translation).  Host code; no GPU needed.
 * ------------------------------------------------------------------------------------- */
typedef struct relo_pose_graph relo_pose_graph;
/* Errors: RELO_EINVAL (n_scenes outside [1, 4096], null out). */
relo_status relo_pose_graph_create(int32_t n_scenes, relo_pose_graph** out);
void relo_pose_graph_destroy(relo_pose_graph* graph);
/* Adds sample aT_b; *cluster_size (nullable) receives the size of the cluster it joined (>= 2:
 * the pair has a confident relative transform, a reason to re-optimise).
 * Errors: RELO_EINVAL (null, scene outside [0, n), a == b). */
relo_status relo_pose_graph_add_sample(relo_pose_graph* graph, int32_t a, int32_t b, const double aTb[16],
                                       int32_t* cluster_size);
/* Builds the pose graph and optimises it: global_poses [n][16] receive gT_s for the scenes in
 * it (the identity for the others), in_graph [n] flags them; *epsilon (nullable) receives
 * epsilon(G), the sum over edges of |v(gT_b^-1 gT_a aT_b)|.  Errors: RELO_EINVAL (null). */
relo_status relo_pose_graph_optimise(relo_pose_graph* graph, double* global_poses, int32_t* in_graph,
                                     double* epsilon);
/* Records that a frame of scene b with local pose pose_in_b was tried against scene a. */
relo_status relo_pose_graph_mark_tried(relo_pose_graph* graph, int32_t a, int32_t b, const double pose_in_b[16]);
/* Phi of candidate (a, (b, frame)) (Sec. 3.3.1): phi_new (1 if exactly one of a, b has an optimised
 * global pose after the last relo_pose_graph_optimise) - phi_conf (max(0, largest cluster of the
 * pair - N)) - phi_homog (5 if a frame within 5 cm and 5 degrees of pose_in_b was tried against a). */
relo_status relo_pose_graph_score(const relo_pose_graph* graph, int32_t a, int32_t b, const double pose_in_b[16],
                                  double* score);
/* Dual-quaternion blend of cluster c (creation order) of the pair {a, b}, as aT_b (the inverse
 * of the stored blend when a > b).  Errors: RELO_EINVAL (null, scenes, c outside the clusters). */
relo_status relo_pose_graph_cluster_blend(const relo_pose_graph* graph, int32_t a, int32_t b, int32_t c,
                                          double aTb[16]);
/* Number of clusters of the pair {a, b} (-1 on bad arguments); sizes [capacity] (nullable)
 * receives their sizes in creation order. */
int32_t relo_pose_graph_cluster_count(const relo_pose_graph* graph, int32_t a, int32_t b, int32_t* sizes,
                                      int32_t capacity);

/* ---------------------------------------------------------------------------------------
 * Fault injection, for tests of the error paths (no counterpart in the paper).  Nothing here
 * faults, traps or hangs a GPU: the failures are made on the host, and corrupted data is caught
 * by the kernels' bounded loops, which report RELO_EDEVICE.
 * ------------------------------------------------------------------------------------- */
/* The next n device allocations made by the library fail as if the device were out of memory
 * (creation calls then return RELO_ENOMEM); n <= 0 cancels. */
void relo_debug_fail_allocations(int32_t n);
/* Checked builds (the library built with RELO_CHECKED=1, the stand-in for a device memory
 * checker): the number of guarded accesses whose index check failed (and which were skipped)
 * since the library loaded; -1 in a normal build, -2 if the device could not be read.
 * Synchronises the device. */
int64_t relo_debug_check_failures(void);
/* Makes every hash chain of the scene end in a cycle (each chain entry links to itself; empty
 * links point at entry 0).  A hash walk for a block that is not at its bucket's head then runs into
 * its bound: attempts that raycast the scene through the hash (relo_scene_use_grid(scene, 0))
 * report RELO_EDEVICE.  Synchronous.  Errors: RELO_EINVAL (null scene). */
relo_status relo_debug_corrupt_scene(relo_scene* scene);
/* The regressor's 64 -> 64-channel forward convolutions run on the tcgen05 tensor cores
 * (TMA-fed, TMEM accumulators) by default; use_tcgen05 = 0 switches them to the mma.sync kernel
 * that the other layers use, so that tests can compare the two on the same operands.  Applies to
 * launches issued (or captured) afterwards. */
void relo_debug_conv_path(int32_t use_tcgen05);
/* Makes the tcgen05 convolution's load producer withhold the loads of output tile `tile` of every
 * later launch (tile < 0: none), and sets the limit of its bounded waits to timeout_ms (<= 0: the
 * default of 2 s).  The consumer's wait for the withheld tile then runs out: the launch stops,
 * frees its tensor memory and records RELO_ETIMEOUT, which the learned path reports as the
 * result's status.  The GPU context stays usable. */
void relo_debug_conv_stall(int32_t tile, int32_t timeout_ms);
/* For batches prepared afterwards: stall != 0 makes one item of the persistent RANSAC launch (the
 * first attempt's first selection) wait for a counter that never reaches its target; timeout_ms
 * (<= 0: 2 s) bounds that launch's waits.  With the persistent schedule the wait runs out, the
 * launch stops, and the attempts it did not finish report RELO_ETIMEOUT (unverified).  The GPU
 * context stays usable. */
void relo_debug_persistent_stall(int32_t stall, int32_t timeout_ms);

#ifdef __cplusplus
}
#endif
#endif /* RELO_H_ */
