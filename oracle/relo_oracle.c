/*
 * relo_oracle.c -- plain, slow, FP64 CPU oracle for the inter-agent
 * relocalisation path (Golodetz et al., Sec. 3.3.1, Fig. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file shares no code, header or constant
 * generator with the CUDA library; only tests, the smoke check and the CPU
 * baseline of the benchmark load it.  Every function is the plain definition
 * of one step, written for a reader to check by eye: no blocking, no fusion,
 * no reordering.  Floating point is double throughout; the stored scene and
 * forest values are float32 input data and are widened on read.
 *
 * The paper states only the purpose of the raycast (Sec. 3.3.1 and the
 * appendix "Global Map Rendering": the standard raycasting approach for a
 * voxel scene), the verification test exactly (Sec. 3.3.1, Omega_s, mu), and
 * defers the relocaliser to Cavallari et al.  Every other rule below is a
 * stated reading of that paper-silent step; each reading is named where it is
 * used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",  */
/* SC 2011): ten rounds of the 4x32 Philox S-box with the published multipliers and Weyl key  */
/* increments.                                                                                 */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u; /* golden ratio */
      k1 += 0xBB67AE85u; /* sqrt(3) - 1 */
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* n counters (n x 4) under one key -> n x 4 outputs */
void orc_philox_many(const uint32_t* ctrs, long n, const uint32_t key[2], uint32_t* out) {
  for (long i = 0; i < n; ++i) orc_philox4x32_10(ctrs + 4 * i, key, out + 4 * i);
}

/* ------------------------------------------------------------------------------------------ */
/* Voxel scene (the InfiniTAM-style map of Sec. 3.3): a set of 8^3-voxel blocks.             */
/* The oracle answers "which block holds voxel v" by binary search over the sorted block     */
/* keys -- the definition of set membership -- rather than by hashing.                       */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  long n_blocks;
  const int32_t* coords; /* n x 3 */
  const float* tsdf;     /* n x 512 */
  const uint8_t* rgba;   /* n x 512 x 4 */
  long* order;           /* indices sorted by (bz, by, bx) */
  double voxel, mu;
} orc_scene;

static int key_cmp3(const int32_t* a, int bx, int by, int bz) {
  if (a[2] != bz) return a[2] < bz ? -1 : 1;
  if (a[1] != by) return a[1] < by ? -1 : 1;
  if (a[0] != bx) return a[0] < bx ? -1 : 1;
  return 0;
}

static const int32_t* g_sort_coords;
static int order_cmp(const void* pa, const void* pb) {
  const int32_t* b = g_sort_coords + 3 * (*(const long*)pb);
  int c = key_cmp3(g_sort_coords + 3 * (*(const long*)pa), b[0], b[1], b[2]);
  if (c != 0) return c;
  long x = *(const long*)pa, y = *(const long*)pb;
  return x < y ? -1 : (x > y);
}

orc_scene* orc_scene_create(const int32_t* coords, const float* tsdf, const uint8_t* rgba, long n, double voxel,
                            double mu) {
  orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
  if (!s) return NULL;
  s->n_blocks = n;
  s->coords = coords;
  s->tsdf = tsdf;
  s->rgba = rgba;
  s->voxel = voxel;
  s->mu = mu;
  s->order = (long*)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
  if (!s->order) { free(s); return NULL; }
  for (long i = 0; i < n; ++i) s->order[i] = i;
  g_sort_coords = coords;
  qsort(s->order, (size_t)n, sizeof(long), order_cmp);
  return s;
}

void orc_scene_destroy(orc_scene* s) {
  if (s) { free(s->order); free(s); }
}

/* Index of block (bx,by,bz) in the input block list, or -1 if it is not allocated.
 * Duplicate block coordinates resolve to the lowest input index. */
/* Optional recorder of the distinct data a raycast touches (for the algorithmic-bytes count of
 * the roofline): block keys looked up, and tsdf / colour voxels read.  NULL when not counting. */
typedef struct {
  uint8_t* tsdf_seen;   /* [n_blocks * 512] */
  uint8_t* rgba_seen;   /* [n_blocks * 512] */
  int64_t* keys;        /* open-addressing set of packed block keys, capacity 2^key_bits, 0 = empty */
  int key_bits;
  int64_t n_keys;
} orc_touch;
static orc_touch* g_touch = NULL;

static void touch_key(int bx, int by, int bz) {
  const int64_t k = 1 + (((int64_t)(bx + 32768) << 34) | ((int64_t)(by + 32768) << 17) | (int64_t)(bz + 32768));
  const uint64_t mask = ((uint64_t)1 << g_touch->key_bits) - 1;
  uint64_t h = ((uint64_t)k * 0x9E3779B97F4A7C15ull) >> (64 - g_touch->key_bits);
  while (g_touch->keys[h] != 0 && g_touch->keys[h] != k) h = (h + 1) & mask;
  if (g_touch->keys[h] == 0) {
    g_touch->keys[h] = k;
    g_touch->n_keys++;
  }
}

long orc_scene_find_block(const orc_scene* s, int bx, int by, int bz) {
  if (g_touch) touch_key(bx, by, bz);
  long lo = 0, hi = s->n_blocks; /* first element >= key */
  while (lo < hi) {
    long mid = lo + (hi - lo) / 2;
    if (key_cmp3(s->coords + 3 * s->order[mid], bx, by, bz) < 0) lo = mid + 1;
    else hi = mid;
  }
  if (lo < s->n_blocks && key_cmp3(s->coords + 3 * s->order[lo], bx, by, bz) == 0) return s->order[lo];
  return -1;
}

void orc_scene_find_many(const orc_scene* s, const int32_t* keys, long n, int64_t* out) {
  for (long i = 0; i < n; ++i) out[i] = orc_scene_find_block(s, keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]);
}

static long floor_div8(long v) { return v >= 0 ? v / 8 : -((-v + 7) / 8); }

/* Voxel (i,j,k): tsdf and colour; an unallocated voxel reads tsdf +1 (free space,
 * truncated) and colour 0 (reading).  Returns 1 if allocated. */
static int voxel_at(const orc_scene* s, long i, long j, long k, double* tsdf, double rgb[3]) {
  long bx = floor_div8(i), by = floor_div8(j), bz = floor_div8(k);
  long b = orc_scene_find_block(s, (int)bx, (int)by, (int)bz);
  if (b < 0) {
    *tsdf = 1.0;
    if (rgb) rgb[0] = rgb[1] = rgb[2] = 0.0;
    return 0;
  }
  long li = (i - 8 * bx) + 8 * (j - 8 * by) + 64 * (k - 8 * bz);
  if (g_touch) {
    g_touch->tsdf_seen[b * 512 + li] = 1;
    if (rgb) g_touch->rgba_seen[b * 512 + li] = 1;
  }
  *tsdf = (double)s->tsdf[b * 512 + li];
  if (rgb)
    for (int c = 0; c < 3; ++c) rgb[c] = (double)s->rgba[(b * 512 + li) * 4 + c];
  return 1;
}

/* Trilinear interpolation of tsdf (and colour if rgb != NULL) at scene point p (metres);
 * voxel (i,j,k) sits at (i,j,k) * voxel_size. */
static double trilinear(const orc_scene* s, const double p[3], double rgb[3]) {
  double q[3], f[3];
  long base[3];
  for (int a = 0; a < 3; ++a) {
    q[a] = p[a] / s->voxel;
    base[a] = (long)floor(q[a]);
    f[a] = q[a] - (double)base[a];
  }
  double val = 0.0;
  if (rgb) rgb[0] = rgb[1] = rgb[2] = 0.0;
  for (int c = 0; c < 8; ++c) {
    int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
    double t, col[3];
    voxel_at(s, base[0] + dx, base[1] + dy, base[2] + dz, &t, rgb ? col : NULL);
    val += w * t;
    if (rgb)
      for (int k = 0; k < 3; ++k) rgb[k] += w * col[k];
  }
  return val;
}

static double round_half_up(double x) { return floor(x + 0.5); }

/*
 * Raycast of one pixel.  Sec. 3.3.1 makes the query a synthetic colour + depth
 * image of scene b seen from the frame's pose (Fig. 3); the appendix on global
 * map rendering names the usual voxel-scene raycast as the renderer.
 * Reading of the march:
 *   the ray is p(lam) = C + lam * R * ((u-cx)/fx, (v-cy)/fy, 1), lam = camera z;
 *   start at lam = depth_min; at each sample, if the containing block is
 *   unallocated the march moves to the block's exit lam_exit, which becomes the
 *   previous sample with f = +1 (free space up to there), and the next sample is
 *   1e-5 past it; otherwise f = trilinear tsdf and, while f > 0, the next sample is
 *   max(f * mu, voxel) / |d| further;
 *   the first sample with f <= 0 ends the march: if it is the very first sample
 *   the pixel is invalid, else the surface is the secant root between the last
 *   two samples;
 *   the march gives up (invalid) past depth_max or after 100000 samples.
 * Depth is round-half-up(lam_hit * 1000) mm clamped to [1, 65535]; colour is the
 * trilinear colour at the hit point, rounded half up.  Optional noise adds
 * 1.5 mm * z^2 * n (z in metres) before rounding (Appendix: axial noise
 * quadratic in depth), as the workload's sensor model.
 * Returns depth in mm (0 = invalid) and writes rgba (alpha 255 if valid).
 */
static int raycast_pixel(const orc_scene* s, const double K[4], double dmin, double dmax, const double P[16],
                         int u, int v, const float* noise, uint16_t* depth_out, uint8_t rgba_out[4]) {
  const double fx = K[0], fy = K[1], cx = K[2], cy = K[3];
  double dc[3] = {(u - cx) / fx, (v - cy) / fy, 1.0};
  double d[3], C[3];
  for (int r = 0; r < 3; ++r) {
    d[r] = P[4 * r] * dc[0] + P[4 * r + 1] * dc[1] + P[4 * r + 2] * dc[2];
    C[r] = P[4 * r + 3];
  }
  double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double bsz = 8.0 * s->voxel;
  double lam = dmin, lam_prev = 0.0, f_prev = 0.0;
  int have_prev = 0, hit = 0;
  double lam_hit = 0.0;
  for (int it = 0; it < 100000 && lam <= dmax; ++it) {
    double p[3] = {C[0] + lam * d[0], C[1] + lam * d[1], C[2] + lam * d[2]};
    long b[3] = {(long)floor(p[0] / bsz), (long)floor(p[1] / bsz), (long)floor(p[2] / bsz)};
    if (orc_scene_find_block(s, (int)b[0], (int)b[1], (int)b[2]) < 0) {
      /* free space: jump to the exit of this block along the ray */
      double lam_exit = INFINITY;
      for (int a = 0; a < 3; ++a) {
        if (d[a] > 0.0) {
          double l = ((double)(b[a] + 1) * bsz - C[a]) / d[a];
          if (l < lam_exit) lam_exit = l;
        } else if (d[a] < 0.0) {
          double l = ((double)b[a] * bsz - C[a]) / d[a];
          if (l < lam_exit) lam_exit = l;
        }
      }
      lam_prev = lam_exit > lam ? lam_exit : lam;
      f_prev = 1.0;
      have_prev = 1;
      lam = lam_prev + 1e-5;
      continue;
    }
    double f = trilinear(s, p, NULL);
    if (f <= 0.0) {
      if (have_prev) {
        lam_hit = lam_prev + (lam - lam_prev) * f_prev / (f_prev - f);
        hit = 1;
      }
      break;
    }
    lam_prev = lam;
    f_prev = f;
    have_prev = 1;
    double step = f * s->mu;
    if (step < s->voxel) step = s->voxel;
    lam += step / dn;
  }
  if (!hit || lam_hit < dmin || lam_hit > dmax) {
    *depth_out = 0;
    if (rgba_out) rgba_out[0] = rgba_out[1] = rgba_out[2] = rgba_out[3] = 0;
    return 0;
  }
  double z_mm = lam_hit * 1000.0;
  if (noise) z_mm += 1.5 * lam_hit * lam_hit * (double)noise[0];
  double zr = round_half_up(z_mm);
  if (zr < 1.0) zr = 1.0;
  if (zr > 65535.0) zr = 65535.0;
  *depth_out = (uint16_t)zr;
  if (rgba_out) {
    double p[3] = {C[0] + lam_hit * d[0], C[1] + lam_hit * d[1], C[2] + lam_hit * d[2]}, rgb[3];
    trilinear(s, p, rgb);
    for (int c = 0; c < 3; ++c) {
      double x = round_half_up(rgb[c]);
      if (x < 0.0) x = 0.0;
      if (x > 255.0) x = 255.0;
      rgba_out[c] = (uint8_t)x;
    }
    rgba_out[3] = 255;
  }
  return 1;
}

/* Whole view (pixels == NULL) or a list of pixel indices v*W+u; outputs are indexed
 * like the pixels (full image, or one entry per listed pixel).  K = fx, fy, cx, cy. */
void orc_raycast(const orc_scene* s, int W, int H, const double K[4], double dmin, double dmax, const double P[16],
                 const float* noise, const int64_t* pixels, long n_pixels, uint16_t* depth, uint8_t* rgba) {
  long n = pixels ? n_pixels : (long)W * H;
  for (long k = 0; k < n; ++k) {
    long pix = pixels ? (long)pixels[k] : k;
    int u = (int)(pix % W), v = (int)(pix / W);
    raycast_pixel(s, K, dmin, dmax, P, u, v, noise ? noise + pix : NULL, depth + k, rgba ? rgba + 4 * k : NULL);
  }
}

/* Distinct data one view's raycast touches: out = {tsdf voxels, colour voxels, block keys
 * looked up}.  Colour is counted only when with_colour (the query render; verification renders
 * need depth only).  Returns 0, or -1 if scratch allocation fails. */
int orc_raycast_touched(const orc_scene* s, int W, int H, const double K[4], double dmin, double dmax,
                        const double P[16], int with_colour, int64_t out[3]) {
  orc_touch t;
  t.key_bits = 24;
  t.tsdf_seen = (uint8_t*)calloc((size_t)(s->n_blocks > 0 ? s->n_blocks : 1) * 512, 1);
  t.rgba_seen = (uint8_t*)calloc((size_t)(s->n_blocks > 0 ? s->n_blocks : 1) * 512, 1);
  t.keys = (int64_t*)calloc((size_t)1 << t.key_bits, sizeof(int64_t));
  t.n_keys = 0;
  if (!t.tsdf_seen || !t.rgba_seen || !t.keys) {
    free(t.tsdf_seen); free(t.rgba_seen); free(t.keys);
    return -1;
  }
  uint16_t* depth = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)W * H);
  uint8_t* rgba = with_colour ? (uint8_t*)malloc((size_t)W * H * 4) : NULL;
  g_touch = &t;
  for (long k = 0; k < (long)W * H; ++k)
    raycast_pixel(s, K, dmin, dmax, P, (int)(k % W), (int)(k / W), NULL, depth + k, rgba ? rgba + 4 * k : NULL);
  g_touch = NULL;
  int64_t nt = 0, nc = 0;
  for (long i = 0; i < s->n_blocks * 512; ++i) {
    nt += t.tsdf_seen[i];
    nc += t.rgba_seen[i];
  }
  out[0] = nt; out[1] = nc; out[2] = t.n_keys;
  free(depth); free(rgba); free(t.tsdf_seen); free(t.rgba_seen); free(t.keys);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Regression forest evaluation (the relocaliser of Sec. 3.3, after Cavallari et al.).        */
/* Reading: complete binary trees stored breadth first (children of n at 2n+1 / 2n+2);        */
/* node = {int16 dx1, dy1, dx2, dy2; uint8 kind, c1, c2, pad; int32 tau} (16 bytes).           */
/* At pixel x with depth d mm > 0 each probe is q = x + trunc(delta * 1000 / d) per axis       */
/* (integer division toward zero), clamped to the image; kind 0 compares probe depths          */
/* (an invalid probe reads 0), kind 1 compares colour channel c1 of q1 with c2 of q2;          */
/* go left iff V(q1) - V(q2) < tau.  Leaf = node - (2^D - 1); a pixel with d = 0 gets 0xFFFF.  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int16_t dx1, dy1, dx2, dy2;
  uint8_t kind, c1, c2, pad;
  int32_t tau;
} orc_node;

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

static uint16_t descend(const orc_node* tree, int depth, const uint16_t* dimg, const uint8_t* rgba, int W, int H,
                        int u, int v) {
  int d = dimg[(long)v * W + u];
  if (d == 0) return 0xFFFF;
  long n = 0;
  for (int level = 0; level < depth; ++level) {
    const orc_node* nd = &tree[n];
    int q1x = clampi(u + (int)(((int32_t)nd->dx1 * 1000) / d), 0, W - 1);
    int q1y = clampi(v + (int)(((int32_t)nd->dy1 * 1000) / d), 0, H - 1);
    int q2x = clampi(u + (int)(((int32_t)nd->dx2 * 1000) / d), 0, W - 1);
    int q2y = clampi(v + (int)(((int32_t)nd->dy2 * 1000) / d), 0, H - 1);
    int32_t a, b;
    if (nd->kind == 0) {
      a = dimg[(long)q1y * W + q1x];
      b = dimg[(long)q2y * W + q2x];
    } else {
      a = rgba[((long)q1y * W + q1x) * 4 + nd->c1];
      b = rgba[((long)q2y * W + q2x) * 4 + nd->c2];
    }
    n = (a - b < nd->tau) ? 2 * n + 1 : 2 * n + 2;
  }
  return (uint16_t)(n - ((1L << depth) - 1));
}

/* leaves: [T][H][W] */
void orc_forest_eval(const orc_node* nodes, int T, int depth, const uint16_t* dimg, const uint8_t* rgba, int W,
                     int H, uint16_t* leaves) {
  long n_int = (1L << depth) - 1;
  for (int t = 0; t < T; ++t)
    for (int v = 0; v < H; ++v)
      for (int u = 0; u < W; ++u)
        leaves[((long)t * H + v) * W + u] = descend(nodes + t * n_int, depth, dimg, rgba, W, H, u, v);
}

/* ------------------------------------------------------------------------------------------ */
/* Depth-difference verification (Sec. 3.3.1, equations for Omega_s and mu).                  */
/* out = {|Omega|, |Omega_a|, |Omega_b|, |Omega_ab|, sum over Omega_ab of |D_a - D_b| (mm)}.   */
/* ------------------------------------------------------------------------------------------ */
void orc_verify_counts(const uint16_t* da, const uint16_t* db, long n, uint64_t out[5]) {
  uint64_t oa = 0, ob = 0, oab = 0, sum = 0;
  for (long i = 0; i < n; ++i) {
    if (da[i] > 0) ++oa;
    if (db[i] > 0) ++ob;
    if (da[i] > 0 && db[i] > 0) {
      ++oab;
      sum += (uint64_t)(da[i] > db[i] ? da[i] - db[i] : db[i] - da[i]);
    }
  }
  out[0] = (uint64_t)n; out[1] = oa; out[2] = ob; out[3] = oab; out[4] = sum;
}

/* ------------------------------------------------------------------------------------------ */
/* Leaf filling (relocaliser training as per Cavallari et al., Sec. 3.3 (b)): every sampled    */
/* training pixel's scene coordinate is pushed into a reservoir in the leaf it reaches in each */
/* tree; each leaf's reservoir is then clustered by mean shift into at most max_modes modes.   */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int T, depth, capacity;
  long n_leaves;            /* per tree: 2^depth */
  float* samples;           /* [T][L][capacity][3] */
  int* count;               /* [T][L] samples stored */
  int64_t* seen;            /* [T][L] samples offered */
  uint32_t key[2];
} orc_reservoirs;

orc_reservoirs* orc_reservoirs_create(int T, int depth, int capacity, uint32_t seed_lo, uint32_t seed_hi) {
  orc_reservoirs* r = (orc_reservoirs*)calloc(1, sizeof(orc_reservoirs));
  if (!r) return NULL;
  r->T = T; r->depth = depth; r->capacity = capacity;
  r->n_leaves = 1L << depth;
  r->samples = (float*)calloc((size_t)T * r->n_leaves * capacity * 3, sizeof(float));
  r->count = (int*)calloc((size_t)T * r->n_leaves, sizeof(int));
  r->seen = (int64_t*)calloc((size_t)T * r->n_leaves, sizeof(int64_t));
  r->key[0] = seed_lo; r->key[1] = seed_hi;
  if (!r->samples || !r->count || !r->seen) {
    free(r->samples); free(r->count); free(r->seen); free(r);
    return NULL;
  }
  return r;
}

void orc_reservoirs_destroy(orc_reservoirs* r) {
  if (r) { free(r->samples); free(r->count); free(r->seen); free(r); }
}

/* Algorithm R (Vitter 1985) with Philox draws: the n-th sample offered to leaf l of tree t
 * (n counted from 0) is stored in slot n while n < capacity, else j = U[0, n] is drawn from
 * counter (3, t * 2^D + l, n_lo, n_hi) word 0 and the sample replaces slot j if j < capacity. */
static void reservoir_offer(orc_reservoirs* r, int t, long leaf, const double w[3]) {
  long id = (long)t * r->n_leaves + leaf;
  int64_t n = r->seen[id]++;
  long slot = -1;
  if (n < r->capacity) {
    slot = (long)n;
    r->count[id] = (int)(n + 1);
  } else {
    uint32_t ctr[4] = {3u, (uint32_t)id, (uint32_t)(n & 0xFFFFFFFF), (uint32_t)(n >> 32)}, o[4];
    orc_philox4x32_10(ctr, r->key, o);
    uint64_t j = ((uint64_t)o[0] * (uint64_t)(n + 1)) >> 32;
    if (j < (uint64_t)r->capacity) slot = (long)j;
  }
  if (slot >= 0) {
    float* dst = r->samples + (id * r->capacity + slot) * 3;
    dst[0] = (float)w[0]; dst[1] = (float)w[1]; dst[2] = (float)w[2];
  }
}

/* Offer one training frame: pixels on the stride grid (u % stride == 0 and v % stride == 0)
 * with depth > 0, in raster order; the scene coordinate is P * backproject(depth), stored
 * as float32; each tree routes the pixel with the definition above. */
void orc_reservoirs_add_frame(orc_reservoirs* r, const orc_node* nodes, const uint16_t* dimg, const uint8_t* rgba,
                              int W, int H, const double K[4], const double P[16], int stride) {
  long n_int = (1L << r->depth) - 1;
  for (int v = 0; v < H; v += stride) {
    for (int u = 0; u < W; u += stride) {
      int d = dimg[(long)v * W + u];
      if (d == 0) continue;
      double z = d / 1000.0;
      double c[3] = {z * (u - K[2]) / K[0], z * (v - K[3]) / K[1], z}, w[3];
      for (int k = 0; k < 3; ++k) w[k] = P[4 * k] * c[0] + P[4 * k + 1] * c[1] + P[4 * k + 2] * c[2] + P[4 * k + 3];
      for (int t = 0; t < r->T; ++t) {
        uint16_t leaf = descend(nodes + t * n_int, r->depth, dimg, rgba, W, H, u, v);
        reservoir_offer(r, t, leaf, w);
      }
    }
  }
}

void orc_reservoirs_get(const orc_reservoirs* r, float* samples, int* count) {
  memcpy(samples, r->samples, sizeof(float) * (size_t)r->T * r->n_leaves * r->capacity * 3);
  memcpy(count, r->count, sizeof(int) * (size_t)r->T * r->n_leaves);
}

/*
 * Mean shift over one leaf's n samples (reading; the paper defers to Cavallari et al.):
 *   every sample seeds an ascent y <- sum_j k_j x_j / sum_j k_j with the Gaussian kernel
 *   k_j = exp(-|y - x_j|^2 / (2 h^2)), stopping when the shift is below tol or after
 *   max_iter steps;
 *   seeds are taken in slot order; a converged point joins the first existing mode whose
 *   peak (the converged point that opened it) lies within merge_dist, else opens a new mode;
 *   a mode's mean and covariance are those of the samples whose seeds joined it, plus
 *   cov_floor * I; modes are ranked by support (descending), ties by opening order, and the
 *   first max_modes are kept; weight = support / n.
 * Output per kept mode (float32 x 12): mean[3], inverse covariance (xx, xy, xz, yy, yz, zz),
 * log(weight) - 0.5 * log((2 pi)^3 det), weight, 0.  Returns the number of modes.
 */
int orc_mean_shift_leaf(const float* x, int n, double h, double tol, int max_iter, double merge_dist,
                        double cov_floor, int max_modes, float* modes_out) {
  if (n <= 0) return 0;
  double* peak = (double*)malloc(sizeof(double) * 3 * (size_t)n);
  int* member = (int*)malloc(sizeof(int) * (size_t)n);
  int* support = (int*)calloc((size_t)n, sizeof(int));
  int n_modes = 0;
  for (int i = 0; i < n; ++i) {
    double y[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    for (int it = 0; it < max_iter; ++it) {
      double num[3] = {0, 0, 0}, den = 0.0;
      for (int j = 0; j < n; ++j) {
        double dx = y[0] - x[3 * j], dy = y[1] - x[3 * j + 1], dz = y[2] - x[3 * j + 2];
        double k = exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * h * h));
        num[0] += k * x[3 * j]; num[1] += k * x[3 * j + 1]; num[2] += k * x[3 * j + 2];
        den += k;
      }
      double ny[3] = {num[0] / den, num[1] / den, num[2] / den};
      double sh = sqrt((ny[0] - y[0]) * (ny[0] - y[0]) + (ny[1] - y[1]) * (ny[1] - y[1]) + (ny[2] - y[2]) * (ny[2] - y[2]));
      y[0] = ny[0]; y[1] = ny[1]; y[2] = ny[2];
      if (sh < tol) break;
    }
    int found = -1;
    for (int m = 0; m < n_modes; ++m) {
      double dx = y[0] - peak[3 * m], dy = y[1] - peak[3 * m + 1], dz = y[2] - peak[3 * m + 2];
      if (sqrt(dx * dx + dy * dy + dz * dz) < merge_dist) { found = m; break; }
    }
    if (found < 0) {
      found = n_modes++;
      peak[3 * found] = y[0]; peak[3 * found + 1] = y[1]; peak[3 * found + 2] = y[2];
    }
    member[i] = found;
    support[found]++;
  }
  /* rank modes: support descending, ties by opening order (stable selection) */
  int* rank = (int*)malloc(sizeof(int) * (size_t)n_modes);
  for (int m = 0; m < n_modes; ++m) rank[m] = m;
  for (int a = 1; a < n_modes; ++a) { /* insertion sort, stable */
    int v = rank[a], b = a - 1;
    while (b >= 0 && support[rank[b]] < support[v]) { rank[b + 1] = rank[b]; --b; }
    rank[b + 1] = v;
  }
  int kept = n_modes < max_modes ? n_modes : max_modes;
  for (int q = 0; q < kept; ++q) {
    int m = rank[q];
    double mean[3] = {0, 0, 0};
    int cnt = 0;
    for (int i = 0; i < n; ++i)
      if (member[i] == m) {
        mean[0] += x[3 * i]; mean[1] += x[3 * i + 1]; mean[2] += x[3 * i + 2];
        ++cnt;
      }
    for (int k = 0; k < 3; ++k) mean[k] /= cnt;
    double S[3][3] = {{0}};
    for (int i = 0; i < n; ++i)
      if (member[i] == m) {
        double e[3] = {x[3 * i] - mean[0], x[3 * i + 1] - mean[1], x[3 * i + 2] - mean[2]};
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) S[a][b] += e[a] * e[b];
      }
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) S[a][b] /= cnt;
      S[a][a] += cov_floor;
    }
    /* inverse by the adjugate */
    double det = S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) - S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0]) +
                 S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]);
    double I00 = (S[1][1] * S[2][2] - S[1][2] * S[2][1]) / det;
    double I01 = (S[0][2] * S[2][1] - S[0][1] * S[2][2]) / det;
    double I02 = (S[0][1] * S[1][2] - S[0][2] * S[1][1]) / det;
    double I11 = (S[0][0] * S[2][2] - S[0][2] * S[2][0]) / det;
    double I12 = (S[0][2] * S[1][0] - S[0][0] * S[1][2]) / det;
    double I22 = (S[0][0] * S[1][1] - S[0][1] * S[1][0]) / det;
    double weight = (double)cnt / n;
    const double two_pi = 6.283185307179586;
    double lognorm = log(weight) - 0.5 * log(two_pi * two_pi * two_pi * det);
    float* o = modes_out + 12 * q;
    o[0] = (float)mean[0]; o[1] = (float)mean[1]; o[2] = (float)mean[2];
    o[3] = (float)I00; o[4] = (float)I01; o[5] = (float)I02; o[6] = (float)I11; o[7] = (float)I12; o[8] = (float)I22;
    o[9] = (float)lognorm; o[10] = (float)weight; o[11] = 0.0f;
  }
  free(rank); free(peak); free(member); free(support);
  return kept;
}

/* Leaves [lo, hi) (flat index tree * L + leaf) of a reservoir set: modes [T][L][max_modes][12],
 * n_modes [T][L].  Each leaf is independent of the others, so callers may fill disjoint ranges
 * from several threads. */
void orc_fill_modes_range(const orc_reservoirs* r, long lo, long hi, double h, double tol, int max_iter,
                          double merge_dist, double cov_floor, int max_modes, float* modes, uint8_t* n_modes) {
  for (long id = lo; id < hi; ++id) {
    n_modes[id] = (uint8_t)orc_mean_shift_leaf(r->samples + id * r->capacity * 3, r->count[id], h, tol, max_iter,
                                               merge_dist, cov_floor, max_modes, modes + id * max_modes * 12);
  }
}

/* All leaves of a reservoir set. */
void orc_fill_modes(const orc_reservoirs* r, double h, double tol, int max_iter, double merge_dist, double cov_floor,
                    int max_modes, float* modes, uint8_t* n_modes) {
  orc_fill_modes_range(r, 0, (long)r->T * r->n_leaves, h, tol, max_iter, merge_dist, cov_floor, max_modes, modes,
                       n_modes);
}

/* ------------------------------------------------------------------------------------------ */
/* TSDF fusion of a depth (+ colour) frame into a growing voxel-block scene: the standard       */
/* volumetric fusion (Curless and Levoy 1996) in the voxel-hashing form of InfiniTAM, which the   */
/* paper runs for each agent's map (Sec. 3.3 (a)) and for the single global model (Appendix     */
/* B.3).  Unlike the rest of this file the arithmetic is float32, in the order written (this   */
/* file is compiled without contraction): which block a sample falls in, which pixel a voxel   */
/* projects to and whether it lies in the band are decided in float32 by the library too, so   */
/* both sides must take those decisions in the same precision.                                  */
/* Readings (the paper cites the pipeline, not its rules):                                       */
/*  - depth z = D * 0.001 m, valid in [depth_min, depth_max];                                   */
/*  - allocation: along the ray of a valid pixel, the points at camera z = z - mu + k h,        */
/*    h = block_size / 4, k = 0 .. ceil(2 mu / h) (the last clamped to z + mu, points at z <= 0 */
/*    skipped); every block holding such a point is allocated (if new) and updated this frame; */
/*  - update of a voxel of those blocks (centre at its integer coordinates times the voxel      */
/*    size): camera point q = R^T (p - t), skipped unless q.z > 0; pixel (floor(fx q.x/q.z + cx */
/*    + 1/2), floor(fy q.y/q.z + cy + 1/2)) inside the image with a valid depth d;               */
/*    eta = d - q.z, skipped if eta < -mu; f = min(1, eta / mu); F = (F w + f) / (w + 1),       */
/*    each colour channel c = round_half_up((c w + c_pixel) / (w + 1)), alpha 255,              */
/*    w = min(w + 1, max_weight).  New blocks start at F = 1, w = 0, colour 0.                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  long n, cap;
  int32_t* coords;      /* cap x 3 */
  float* tsdf;          /* cap x 512 */
  uint8_t* rgba;        /* cap x 512 x 4 */
  uint16_t* weight;     /* cap x 512 */
  long* stamp;          /* cap: the last frame that marked the block */
  long* table;          /* open addressing over block coordinates -> index, -1 empty */
  long table_size;
  float voxel, mu;
  int max_weight;
  long frame;
} orc_fusion;

orc_fusion* orc_fusion_create(long cap, double voxel, double mu, int max_weight) {
  orc_fusion* f = (orc_fusion*)calloc(1, sizeof(orc_fusion));
  if (!f || cap < 1) { free(f); return NULL; }
  f->cap = cap;
  f->coords = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)cap);
  f->tsdf = (float*)malloc(sizeof(float) * 512 * (size_t)cap);
  f->rgba = (uint8_t*)calloc((size_t)cap * 512 * 4, 1);
  f->weight = (uint16_t*)calloc((size_t)cap * 512, sizeof(uint16_t));
  f->stamp = (long*)malloc(sizeof(long) * (size_t)cap);
  f->table_size = 1;
  while (f->table_size < 2 * cap) f->table_size *= 2;
  f->table = (long*)malloc(sizeof(long) * (size_t)f->table_size);
  if (!f->coords || !f->tsdf || !f->rgba || !f->weight || !f->stamp || !f->table) {
    free(f->coords); free(f->tsdf); free(f->rgba); free(f->weight); free(f->stamp); free(f->table); free(f);
    return NULL;
  }
  for (long i = 0; i < f->table_size; ++i) f->table[i] = -1;
  f->voxel = (float)voxel;
  f->mu = (float)mu;
  f->max_weight = max_weight;
  return f;
}

void orc_fusion_destroy(orc_fusion* f) {
  if (!f) return;
  free(f->coords); free(f->tsdf); free(f->rgba); free(f->weight); free(f->stamp); free(f->table); free(f);
}

static long fusion_slot(const orc_fusion* f, int bx, int by, int bz) {
  uint64_t h = ((uint64_t)(uint32_t)bx * 2654435761u) ^ ((uint64_t)(uint32_t)by * 40503u) ^
               ((uint64_t)(uint32_t)bz * 2246822519u);
  long i = (long)(h & (uint64_t)(f->table_size - 1));
  for (;;) {
    long b = f->table[i];
    if (b < 0) return i;
    const int32_t* c = f->coords + 3 * b;
    if (c[0] == bx && c[1] == by && c[2] == bz) return i;
    i = (i + 1) & (f->table_size - 1);
  }
}

/* Marks block (bx,by,bz) for this frame, allocating it if new.  Returns -1 when full. */
static int fusion_mark(orc_fusion* f, int bx, int by, int bz) {
  long i = fusion_slot(f, bx, by, bz);
  long b = f->table[i];
  if (b < 0) {
    if (f->n >= f->cap) return -1;
    b = f->n++;
    f->table[i] = b;
    f->coords[3 * b] = bx;
    f->coords[3 * b + 1] = by;
    f->coords[3 * b + 2] = bz;
    for (int v = 0; v < 512; ++v) f->tsdf[512 * b + v] = 1.0f;
  }
  f->stamp[b] = f->frame;
  return 0;
}

/* Fuses one frame.  K = fx, fy, cx, cy; P camera -> scene (row-major 4x4); rgba nullable.
 * Returns 0, or -1 if the block capacity ran out (the frame is then fused into the blocks that
 * fit). */
int orc_fusion_frame(orc_fusion* f, int W, int H, const double K[4], double depth_min, double depth_max,
                     const double P[16], const uint16_t* depth, const uint8_t* rgba) {
  const float fx = (float)K[0], fy = (float)K[1], cx = (float)K[2], cy = (float)K[3];
  const float dmin = (float)depth_min, dmax = (float)depth_max;
  float R[9], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) R[3 * r + c] = (float)P[4 * r + c];
    t[r] = (float)P[4 * r + 3];
  }
  const float mu = f->mu, bs = f->voxel * 8.0f, h = bs * 0.25f;
  int full = 0;
  f->frame += 1;
  /* allocation: the band around every valid pixel's depth */
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      const uint16_t D = depth[(long)v * W + u];
      if (D == 0) continue;
      const float z = (float)D * 0.001f;
      if (!(z >= dmin && z <= dmax)) continue;
      const float dcx = ((float)u - cx) / fx, dcy = ((float)v - cy) / fy;
      float dir[3];
      for (int r = 0; r < 3; ++r) dir[r] = (R[3 * r] * dcx + R[3 * r + 1] * dcy) + R[3 * r + 2];
      const float z0 = z - mu, z1 = z + mu;
      const int n = (int)ceilf((z1 - z0) / h);
      for (int k = 0; k <= n; ++k) {
        float zk = z0 + (float)k * h;
        if (zk > z1) zk = z1;
        if (!(zk > 0.0f)) continue;
        int b[3], ok = 1;
        for (int r = 0; r < 3; ++r) {
          const float p = t[r] + zk * dir[r];
          const float q = floorf(p / bs);
          if (!(q >= -32768.0f && q <= 32767.0f)) ok = 0;
          b[r] = ok ? (int)q : 0;
        }
        if (ok && fusion_mark(f, b[0], b[1], b[2]) != 0) full = 1;
      }
    }
  /* update: every voxel of the blocks marked this frame */
  for (long b = 0; b < f->n; ++b) {
    if (f->stamp[b] != f->frame) continue;
    const int32_t* bc = f->coords + 3 * b;
    for (int vi = 0; vi < 512; ++vi) {
      const int X = 8 * bc[0] + (vi & 7), Y = 8 * bc[1] + ((vi >> 3) & 7), Z = 8 * bc[2] + (vi >> 6);
      const float px = (float)X * f->voxel, py = (float)Y * f->voxel, pz = (float)Z * f->voxel;
      const float dx = px - t[0], dy = py - t[1], dz = pz - t[2];
      const float qx = (R[0] * dx + R[3] * dy) + R[6] * dz;
      const float qy = (R[1] * dx + R[4] * dy) + R[7] * dz;
      const float qz = (R[2] * dx + R[5] * dy) + R[8] * dz;
      if (!(qz > 0.0f)) continue;
      const float uf = fx * (qx / qz) + cx, vf = fy * (qy / qz) + cy;
      const float fu = floorf(uf + 0.5f), fv = floorf(vf + 0.5f);
      if (!(fu >= 0.0f && fu < (float)W && fv >= 0.0f && fv < (float)H)) continue;
      const long pix = (long)fv * W + (long)fu;
      const uint16_t Dm = depth[pix];
      if (Dm == 0) continue;
      const float dm = (float)Dm * 0.001f;
      if (!(dm >= dmin && dm <= dmax)) continue;
      const float eta = dm - qz;
      if (eta < -mu) continue;
      const float fn = fminf(1.0f, eta / mu);
      const long at = 512 * b + vi;
      const float w = (float)f->weight[at];
      f->tsdf[at] = (f->tsdf[at] * w + fn) / (w + 1.0f);
      if (rgba) {
        for (int c = 0; c < 3; ++c) {
          const float cc = ((float)f->rgba[4 * at + c] * w + (float)rgba[4 * pix + c]) / (w + 1.0f);
          float r = floorf(cc + 0.5f);
          if (r < 0.0f) r = 0.0f;
          if (r > 255.0f) r = 255.0f;
          f->rgba[4 * at + c] = (uint8_t)r;
        }
        f->rgba[4 * at + 3] = 255;
      }
      f->weight[at] = (uint16_t)(f->weight[at] + 1 < f->max_weight ? f->weight[at] + 1 : f->max_weight);
    }
  }
  return full ? -1 : 0;
}

long orc_fusion_count(const orc_fusion* f) { return f->n; }

/* Copies the blocks (in allocation order) out. */
void orc_fusion_export(const orc_fusion* f, int32_t* coords, float* tsdf, uint8_t* rgba, uint16_t* weight) {
  memcpy(coords, f->coords, sizeof(int32_t) * 3 * (size_t)f->n);
  memcpy(tsdf, f->tsdf, sizeof(float) * 512 * (size_t)f->n);
  memcpy(rgba, f->rgba, (size_t)f->n * 512 * 4);
  memcpy(weight, f->weight, sizeof(uint16_t) * 512 * (size_t)f->n);
}
