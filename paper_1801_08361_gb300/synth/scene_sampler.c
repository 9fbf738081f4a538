/*
 * Seeded synthetic-scene sampler (input generation only).
 *
 * Stands in for the InfiniTAM fusion that builds each agent's voxel sub-scene
 * (Sec. 3.3): instead of fusing posed RGB-D frames, an analytic signed distance
 * function of a box world (an outer room/house shell, thin walls and furniture
 * boxes) is sampled directly at voxel centres, truncated, and written out as a
 * list of 8x8x8-voxel blocks.  Nothing here is on the relocalisation path; both
 * the CUDA library and the CPU oracle receive the blocks this file produces as
 * plain input data.
 *
 * Conventions shared with the consumers (they are the input format):
 *   voxel (i,j,k) is the scene-frame point (i*s, j*s, k*s);
 *   block (bx,by,bz) holds voxels 8*bx..8*bx+7 (etc.), local index
 *   (i&7) + 8*(j&7) + 64*(k&7);
 *   tsdf = clamp(sdf / mu, -1, 1) as float32, positive in free space;
 *   rgba = texture colour of the nearest surface, alpha 255.
 * A block is emitted when at least one of its voxels has |sdf| < mu and lies
 * inside the crop region.  Blocks come out sorted by (bz, by, bx).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BLK 8
#define VPB 512

typedef struct {
  int kind;        /* 0: free interior of this box (walls enclose it); 1: solid box */
  double lo[3], hi[3];
  double rgb[3];   /* base colour in [0,1] */
  double freq[3];  /* texture frequencies (cycles per metre) */
} comp_t;

/* Signed distance to an axis-aligned box, positive outside. */
static double box_sdf(const double lo[3], const double hi[3], const double p[3]) {
  double q[3], out = 0.0, in = -1e30;
  for (int a = 0; a < 3; ++a) {
    double c = 0.5 * (lo[a] + hi[a]), h = 0.5 * (hi[a] - lo[a]);
    q[a] = fabs(p[a] - c) - h;
    double m = q[a] > 0.0 ? q[a] : 0.0;
    out += m * m;
    if (q[a] > in) in = q[a];
  }
  return sqrt(out) + (in < 0.0 ? in : 0.0);
}

static double comp_sdf(const comp_t* c, const double p[3]) {
  double d = box_sdf(c->lo, c->hi, p);
  return c->kind == 0 ? -d : d;
}

/* Distance from an AABB of points to a component's box (0 if overlapping). */
static double aabb_gap(const comp_t* c, const double lo[3], const double hi[3]) {
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    double g = 0.0;
    if (hi[a] < c->lo[a]) g = c->lo[a] - hi[a];
    else if (lo[a] > c->hi[a]) g = lo[a] - c->hi[a];
    s += g * g;
  }
  return sqrt(s);
}

static void xform(const double* M, const double p[3], double o[3]) {
  for (int r = 0; r < 3; ++r) o[r] = M[4 * r] * p[0] + M[4 * r + 1] * p[1] + M[4 * r + 2] * p[2] + M[4 * r + 3];
}

static uint8_t to_u8(double v) {
  if (v <= 0.0) return 0;
  if (v >= 1.0) return 255;
  return (uint8_t)(v * 255.0 + 0.5);
}

/* Texture of component c at world point p: base colour modulated by a product
 * of sinusoids whose frequencies differ per component. */
static void texture(const comp_t* c, const double p[3], uint8_t out[4]) {
  const double two_pi = 6.283185307179586;
  double t = 0.55 + 0.25 * sin(two_pi * c->freq[0] * (p[0] + 0.37 * p[2])) * sin(two_pi * c->freq[1] * (p[1] - 0.21 * p[2])) +
             0.2 * sin(two_pi * c->freq[2] * (p[0] + p[1] + p[2]));
  for (int k = 0; k < 3; ++k) out[k] = to_u8(c->rgb[k] * t);
  out[3] = 255;
}

typedef struct {
  const comp_t* comps;
  int n_comps;
  double voxel, mu;
  const double* scene_to_world; /* 4x4 row-major */
  double crop_lo[3], crop_hi[3];
} ctx_t;

static int in_crop(const ctx_t* x, const double w[3]) {
  for (int a = 0; a < 3; ++a)
    if (w[a] < x->crop_lo[a] || w[a] > x->crop_hi[a]) return 0;
  return 1;
}

/* Evaluate one block.  Returns 1 if it must be allocated; fills tsdf/rgba when
 * the output pointers are non-null. */
static int eval_block(const ctx_t* x, int bx, int by, int bz, int* near, float* tsdf, uint8_t* rgba) {
  const double s = x->voxel, mu = x->mu;
  /* world-space AABB of the block's voxel centres (transform its 8 corners) */
  double wlo[3] = {1e30, 1e30, 1e30}, whi[3] = {-1e30, -1e30, -1e30};
  for (int c = 0; c < 8; ++c) {
    double ps[3] = {(BLK * bx + ((c & 1) ? BLK - 1 : 0)) * s, (BLK * by + ((c & 2) ? BLK - 1 : 0)) * s,
                    (BLK * bz + ((c & 4) ? BLK - 1 : 0)) * s};
    double pw[3];
    xform(x->scene_to_world, ps, pw);
    for (int a = 0; a < 3; ++a) {
      if (pw[a] < wlo[a]) wlo[a] = pw[a];
      if (pw[a] > whi[a]) whi[a] = pw[a];
    }
  }
  /* components that can bring |sdf| below mu somewhere in the block */
  int n_near = 0;
  for (int i = 0; i < x->n_comps; ++i) {
    const comp_t* c = &x->comps[i];
    if (c->kind == 0) {
      near[n_near++] = i; /* shell: always relevant (negative outside) */
    } else if (aabb_gap(c, wlo, whi) < mu + 1e-9) {
      near[n_near++] = i;
    }
  }
  int alloc = 0;
  for (int v = 0; v < VPB; ++v) {
    int i = BLK * bx + (v & 7), j = BLK * by + ((v >> 3) & 7), k = BLK * bz + (v >> 6);
    double ps[3] = {i * s, j * s, k * s}, pw[3];
    xform(x->scene_to_world, ps, pw);
    double best = 1e30;
    int arg = -1;
    for (int n = 0; n < n_near; ++n) {
      double d = comp_sdf(&x->comps[near[n]], pw);
      if (d < best) { best = d; arg = near[n]; }
    }
    int inside = in_crop(x, pw);
    if (!inside) best = 1e30; /* cropped away: reads as free space */
    if (fabs(best) < mu) alloc = 1;
    if (tsdf) {
      double t = best / mu;
      if (t > 1.0) t = 1.0;
      if (t < -1.0) t = -1.0;
      tsdf[v] = (float)t;
      uint8_t col[4] = {0, 0, 0, 0};
      if (arg >= 0 && inside) texture(&x->comps[arg], pw, col);
      memcpy(rgba + 4 * v, col, 4);
    }
  }
  return alloc;
}

/*
 * Pass 1: flag which blocks of the scene-frame block box [blo, bhi] (inclusive)
 * are allocated.  flags has (bhi-blo+1) entries per axis, x fastest.
 */
int synth_flag_blocks(const double* comps_flat, int n_comps, double voxel, double mu, const double* scene_to_world,
                      const double* crop, const int* blo, const int* bhi, uint8_t* flags) {
  comp_t* comps = (comp_t*)malloc(sizeof(comp_t) * (size_t)(n_comps > 0 ? n_comps : 1));
  if (!comps) return -1;
  for (int i = 0; i < n_comps; ++i) {
    const double* f = comps_flat + 13 * i;
    comps[i].kind = (int)f[0];
    for (int a = 0; a < 3; ++a) {
      comps[i].lo[a] = f[1 + a];
      comps[i].hi[a] = f[4 + a];
      comps[i].rgb[a] = f[7 + a];
      comps[i].freq[a] = f[10 + a];
    }
  }
  ctx_t x = {comps, n_comps, voxel, mu, scene_to_world, {crop[0], crop[1], crop[2]}, {crop[3], crop[4], crop[5]}};
  const int nx = bhi[0] - blo[0] + 1, ny = bhi[1] - blo[1] + 1, nz = bhi[2] - blo[2] + 1;
  const double half_diag = sqrt(3.0) * 0.5 * (BLK - 1) * voxel;
#pragma omp parallel
  {
    int* near = (int*)malloc(sizeof(int) * (size_t)(n_comps > 0 ? n_comps : 1));
#pragma omp for schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z) {
      for (int y = 0; y < ny; ++y) {
        for (int xx = 0; xx < nx; ++xx) {
          int bx = blo[0] + xx, by = blo[1] + y, bz = blo[2] + z;
          size_t idx = ((size_t)z * ny + y) * nx + xx;
          /* cheap reject: the SDF is 1-Lipschitz, so a centre farther than
           * mu + half-diagonal from every surface cannot hold a band voxel */
          double pc[3] = {(BLK * bx + 3.5) * voxel, (BLK * by + 3.5) * voxel, (BLK * bz + 3.5) * voxel}, pw[3];
          xform(scene_to_world, pc, pw);
          double best = 1e30;
          for (int n = 0; n < n_comps; ++n) {
            double d = comp_sdf(&comps[n], pw);
            if (d < best) best = d;
          }
          if (fabs(best) > mu + half_diag + 1e-6) { flags[idx] = 0; continue; }
          flags[idx] = (uint8_t)eval_block(&x, bx, by, bz, near, NULL, NULL);
        }
      }
    }
    free(near);
  }
  free(comps);
  return 0;
}

/* Pass 2: fill tsdf/rgba for the given block coordinates (n x 3). */
int synth_fill_blocks(const double* comps_flat, int n_comps, double voxel, double mu, const double* scene_to_world,
                      const double* crop, const int32_t* coords, long n, float* tsdf, uint8_t* rgba) {
  comp_t* comps = (comp_t*)malloc(sizeof(comp_t) * (size_t)(n_comps > 0 ? n_comps : 1));
  if (!comps) return -1;
  for (int i = 0; i < n_comps; ++i) {
    const double* f = comps_flat + 13 * i;
    comps[i].kind = (int)f[0];
    for (int a = 0; a < 3; ++a) {
      comps[i].lo[a] = f[1 + a];
      comps[i].hi[a] = f[4 + a];
      comps[i].rgb[a] = f[7 + a];
      comps[i].freq[a] = f[10 + a];
    }
  }
  ctx_t x = {comps, n_comps, voxel, mu, scene_to_world, {crop[0], crop[1], crop[2]}, {crop[3], crop[4], crop[5]}};
#pragma omp parallel
  {
    int* near = (int*)malloc(sizeof(int) * (size_t)(n_comps > 0 ? n_comps : 1));
#pragma omp for schedule(dynamic, 64)
    for (long b = 0; b < n; ++b)
      eval_block(&x, coords[3 * b], coords[3 * b + 1], coords[3 * b + 2], near, tsdf + (size_t)b * VPB,
                 rgba + (size_t)b * VPB * 4);
    free(near);
  }
  free(comps);
  return 0;
}

/* Exact analytic signed distance at world points (n x 3): used to pin raycasts. */
void synth_world_sdf(const double* comps_flat, int n_comps, const double* pts, long n, double* out) {
  for (long p = 0; p < n; ++p) {
    double best = 1e30;
    for (int i = 0; i < n_comps; ++i) {
      comp_t c;
      const double* f = comps_flat + 13 * i;
      c.kind = (int)f[0];
      for (int a = 0; a < 3; ++a) { c.lo[a] = f[1 + a]; c.hi[a] = f[4 + a]; }
      double d = comp_sdf(&c, pts + 3 * p);
      if (d < best) best = d;
    }
    out[p] = best;
  }
}
