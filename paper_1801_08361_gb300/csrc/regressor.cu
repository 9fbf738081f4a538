// regressor.cu -- the learned scene-coordinate regressor: BF16 tensor-core 3x3 convolutions
// (forward, backward-data, backward-weight) with FP32 accumulation, the Gaussian-NLL loss, Adam,
// and the cell forest that hands its output to the preemptive RANSAC.
//
// The paper relocalises with a forest (Sec. 3.3 (b)); this network is the workload's alternative
// relocaliser for a scene, trained online on renders of the scene's own voxel map.  Readings
// (identical in the CPU oracle): 4 input channels ((depth m - 3) / 2, (RGB / 255 - 1/2) x 4), eight
// 3x3 convolutions with zero padding, 64 channels, strides 2, 2, 2, 1, 1, 1, 1, 1, ReLU after
// layers 1-7, 4 outputs per 8 x 8-pixel cell (scene coordinate - origin, log-variance s); the
// target of a cell is the scene coordinate of its centre pixel; loss = mean over scored cells of
// rho(e) + 1/2 e^2 exp(-s) + 3/2 s with e = |y - y_hat|, rho(e) = sqrt(e^2 + 1e-6), the error in the
// variance term held fixed for the gradient; Adam (0.9, 0.999, 1e-8).
//
// Layout: activations NHWC in BF16 (channels contiguous); layer 1's input is padded to 16
// channels and the head's output to 8 (its gradient to 16) so every contraction is a multiple
// of the mma.sync m16n8k16 shape.  A convolution is an implicit GEMM: output pixels x output
// channels, contracted over 9 taps x input channels; each CTA (4 warps) keeps all 9 taps of the
// weights in shared memory and loops over 64-pixel tiles, gathering one tap's input rows per
// step.  The backward-data pass of a stride-2 layer is the same kernel reading its input
// through a virtual zero-inserted upsampling, with the weights flipped and transposed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "regressor.cuh"

namespace relo {

// ---------------------------------------------------------------------------------------------
// Tensor-core primitive
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }


constexpr int kConvPix = 64;  // output pixels per backward-weight tile (wgrad_kernel)

// ldmatrix: four (or two) 8 x 8 b16 matrices from shared memory, rows addressed by lanes 8q..8q+7
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

// Forward / backward-data convolution.  A CTA of 8 warps keeps all 9 taps of the weights in shared
// memory and loops over tiles of 128 output pixels (16 per warp, all N output channels per warp).
// Per tap the tile's input rows (one per output pixel) are gathered into shared memory; the next
// tap's rows are loaded into registers while the current tap's MMAs run, so the gathers overlap
// the tensor-core work.  Fragments come from shared memory by ldmatrix; rows are padded to
// CIN + 8 elements, which keeps every ldmatrix phase free of bank conflicts.
constexpr int kConvThreads = 256;
constexpr int kConvTile = 128;

template <int CIN>
struct ConvGather {
  static constexpr int CH = CIN / 8;                              // 16-B chunks per pixel
  static constexpr int PER = kConvTile * CH / kConvThreads;       // chunks per thread per tap
  static_assert(PER >= 1 && kConvTile * CH % kConvThreads == 0, "tile / channel split");
  int b[PER], oy[PER], ox[PER], m[PER], c8[PER];
  bool ok[PER];

  __device__ __forceinline__ void setup(const ConvArgs& a, long m0, long total, int tid) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int v = tid + i * kConvThreads;
      m[i] = v / CH;
      c8[i] = v % CH;
      const long p = m0 + m[i];
      ok[i] = p < total;
      ox[i] = ok[i] ? (int)(p % a.Wo) : 0;
      oy[i] = ok[i] ? (int)((p / a.Wo) % a.Ho) : 0;
      b[i] = ok[i] ? (int)(p / ((long)a.Wo * a.Ho)) : 0;
    }
  }

  __device__ __forceinline__ void load(const ConvArgs& a, int tap, uint4 (&val)[PER]) const {
    const int ky = tap / 3, kx = tap % 3;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      val[i] = make_uint4(0u, 0u, 0u, 0u);
      const int iy = oy[i] * a.stride + ky - 1, ix = ox[i] * a.stride + kx - 1;
      if (ok[i] && iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Wi) {
        if (!a.upsample) {
          val[i] = __ldg(reinterpret_cast<const uint4*>(a.in + (((size_t)b[i] * a.Hi + iy) * a.Wi + ix) * CIN) + c8[i]);
        } else if (!(iy & 1) && !(ix & 1) && (iy >> 1) < a.Hs && (ix >> 1) < a.Ws) {
          val[i] = __ldg(reinterpret_cast<const uint4*>(a.in + (((size_t)b[i] * a.Hs + (iy >> 1)) * a.Ws + (ix >> 1)) *
                                                                  CIN) + c8[i]);
        }
      }
    }
  }
};

template <int CIN, int NT>
__global__ void __launch_bounds__(kConvThreads) conv_kernel(ConvArgs a) {
  constexpr int N = NT * 8;
  constexpr int RS = CIN + 8;  // padded row stride (bf16) of the shared tiles
  using G = ConvGather<CIN>;
  extern __shared__ __align__(16) unsigned char conv_smem[];
  bf16* sW = reinterpret_cast<bf16*>(conv_smem);   // [9][N][RS]
  bf16* sA = sW + 9 * N * RS;                       // [kConvTile][RS]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  for (int v = tid; v < 9 * N * (CIN / 8); v += kConvThreads) {
    const int row = v / (CIN / 8), c8 = v % (CIN / 8);
    *reinterpret_cast<uint4*>(sW + row * RS + c8 * 8) = __ldg(reinterpret_cast<const uint4*>(a.w + (size_t)row * CIN) + c8);
  }
  const long total = (long)a.B * a.Ho * a.Wo;
  const long n_tiles = (total + kConvTile - 1) / kConvTile;
  // ldmatrix row addresses of this lane: A rows warp * 16 + (lane & 7) + 8 * ((lane >> 3) & 1),
  // k half (lane >> 4); B rows (n) (lane & 7) + 8 * (lane >> 4), k half ((lane >> 3) & 1)
  const int a_row = warp * 16 + (lane & 7) + 8 * ((lane >> 3) & 1), a_k = 8 * (lane >> 4);
  const int b_row = (lane & 7) + 8 * (lane >> 4), b_k = 8 * ((lane >> 3) & 1);
  for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long m0 = tile * kConvTile;
    G gat;
    gat.setup(a, m0, total, tid);
    uint4 pre[G::PER];
    gat.load(a, 0, pre);
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int tap = 0; tap < 9; ++tap) {
      __syncthreads();  // readers of the previous tap's rows (and, first, the weight stores) are done
#pragma unroll
      for (int i = 0; i < G::PER; ++i) *reinterpret_cast<uint4*>(sA + gat.m[i] * RS + gat.c8[i] * 8) = pre[i];
      __syncthreads();
      if (tap < 8) gat.load(a, tap + 1, pre);  // in flight during this tap's MMAs
      const bf16* Wt = sW + tap * N * RS;
#pragma unroll
      for (int ks = 0; ks < CIN / 16; ++ks) {
        uint32_t af[4];
        ldsm_x4(af, sA + a_row * RS + ks * 16 + a_k);
#pragma unroll
        for (int j = 0; j + 1 < NT; j += 2) {
          uint32_t bf[4];
          ldsm_x4(bf, Wt + (j * 8 + b_row) * RS + ks * 16 + b_k);
          mma_bf16(acc[j], af, bf[0], bf[1]);
          mma_bf16(acc[j + 1], af, bf[2], bf[3]);
        }
        if (NT & 1) {
          uint32_t b0, b1;
          ldsm_x2(b0, b1, Wt + ((NT - 1) * 8 + (lane & 7)) * RS + ks * 16 + 8 * ((lane >> 3) & 1));
          mma_bf16(acc[NT - 1], af, b0, b1);
        }
      }
    }
    // epilogue: bias, ReLU, mask, stores
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int n0 = j * 8 + 2 * t;
      const float b0 = a.bias ? a.bias[n0] : 0.f, b1 = a.bias ? a.bias[n0 + 1] : 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const long p = m0 + warp * 16 + g + 8 * h;
        if (p >= total) continue;
        float v0 = acc[j][2 * h] + b0, v1 = acc[j][2 * h + 1] + b1;
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.mask) {
          const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(a.mask + (size_t)p * N + n0);
          if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
          if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
        }
        if (a.out) *reinterpret_cast<__nv_bfloat162*>(a.out + (size_t)p * N + n0) = __floats2bfloat162_rn(v0, v1);
        if (a.out_f32) {
          a.out_f32[(size_t)p * N + n0] = v0;
          a.out_f32[(size_t)p * N + n0 + 1] = v1;
        }
      }
    }
  }
}

template <int CIN, int NT>
cudaError_t launch_conv_t(const ConvArgs& a, int n_sms, cudaStream_t s) {
  constexpr int N = NT * 8, RS = CIN + 8;
  const size_t smem = (size_t)(9 * N + kConvTile) * RS * sizeof(bf16);
  static PerDevice resident;  // resident CTAs per SM on each device
  int per_sm = 0;
  const cudaError_t e = per_device(resident, &per_sm, [smem](int, int* v) {
    cudaError_t r = cudaFuncSetAttribute(conv_kernel<CIN, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, conv_kernel<CIN, NT>, kConvThreads, smem);
    if (*v < 1) *v = 1;
    return r;
  });
  if (e != cudaSuccess) return e;
  const long total = (long)a.B * a.Ho * a.Wo;
  const long tiles = (total + kConvTile - 1) / kConvTile;
  const long slots = (long)n_sms * per_sm;
  const long grid = tiles < slots ? tiles : slots;
  if (grid <= 0) return cudaSuccess;
  conv_kernel<CIN, NT><<<(unsigned)grid, kConvThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_conv(int cin, int nt, const ConvArgs& a, int n_sms, cudaStream_t s) {
  if (cin == 16 && nt == 8) return launch_conv_t<16, 8>(a, n_sms, s);
  if (cin == 64 && nt == 8) return launch_conv_t<64, 8>(a, n_sms, s);
  if (cin == 64 && nt == 1) return launch_conv_t<64, 1>(a, n_sms, s);
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------------------------
// Backward-weight: partial[chunk][tap][n][k] = sum over the chunk's output pixels p of
// g[p, n] * in[src(p, tap), k]; a second kernel sums the chunks in a fixed order.
// A CTA (8 warps) owns one tap and one chunk of pixels; per 64-pixel tile it stages the gradient
// rows and the tap's gathered input rows as stored (pixel-major, 16-byte vectors, the next tile
// prefetched into registers) and contracts over the pixels with ldmatrix.trans fragments:
// M = input channels, N = output channels, K = pixels.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

constexpr int kWgradThreads = 256;

template <int CIN, int NT>
__global__ void __launch_bounds__(kWgradThreads) wgrad_kernel(WgradArgs a) {
  constexpr int N = NT * 8;
  constexpr int MT = CIN / 16;                          // m16 tiles over the input channels
  constexpr int WM = (MT >= 2 && MT * NT >= 32) ? 2 : 1;  // m16 tiles per warp
  constexpr int WN = (NT >= 2 && MT * NT >= 32) ? 2 : 1;  // n8 tiles per warp
  constexpr int MG = MT / WM, NG = NT / WN;
  static_assert(MG * NG <= kWgradThreads / 32, "warp split");
  constexpr int RI = CIN + 8;                           // row strides (bf16): conflict-free ldmatrix
  constexpr int RG = (N < 16 ? 16 : N) + 8;
  constexpr int CI = CIN / 8, CG = N / 8;               // 16-B chunks per pixel row
  constexpr int PI = (kConvPix * CI + kWgradThreads - 1) / kWgradThreads;
  constexpr int PG = (kConvPix * CG + kWgradThreads - 1) / kWgradThreads;
  __shared__ __align__(16) bf16 sI[kConvPix][RI];
  __shared__ __align__(16) bf16 sG[kConvPix][RG];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int tap = blockIdx.y, ky = tap / 3, kx = tap % 3;
  const long total = (long)a.B * a.Ho * a.Wo;
  const long p_begin = (long)blockIdx.x * a.chunk_pix;
  const long p_end = min(p_begin + (long)a.chunk_pix, total);
  const int mg = warp % MG, ng = warp / MG;
  const bool mma_warp = warp < MG * NG;
  float acc[WM][WN][4];
#pragma unroll
  for (int i = 0; i < WM; ++i)
#pragma unroll
    for (int j = 0; j < WN; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;

  uint4 vi[PI], vg[PG];
  auto fetch = [&](long p0) {
#pragma unroll
    for (int i = 0; i < PI; ++i) {
      const int v = tid + i * kWgradThreads;
      vi[i] = make_uint4(0u, 0u, 0u, 0u);
      const long p = p0 + v / CI;
      if (v < kConvPix * CI && p < p_end) {
        const int ox = (int)(p % a.Wo), oy = (int)((p / a.Wo) % a.Ho), b = (int)(p / ((long)a.Wo * a.Ho));
        const int iy = oy * a.stride + ky - 1, ix = ox * a.stride + kx - 1;
        if (iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Wi)
          vi[i] = __ldg(reinterpret_cast<const uint4*>(a.in + (((size_t)b * a.Hi + iy) * a.Wi + ix) * CIN) + v % CI);
      }
    }
#pragma unroll
    for (int i = 0; i < PG; ++i) {
      const int v = tid + i * kWgradThreads;
      vg[i] = make_uint4(0u, 0u, 0u, 0u);
      const long p = p0 + v / CG;
      if (v < kConvPix * CG && p < p_end)
        vg[i] = __ldg(reinterpret_cast<const uint4*>(a.g + (size_t)p * a.GS) + v % CG);
    }
  };
  fetch(p_begin);
  for (long p0 = p_begin; p0 < p_end; p0 += kConvPix) {
    __syncthreads();  // the previous tile's fragments are read
#pragma unroll
    for (int i = 0; i < PI; ++i) {
      const int v = tid + i * kWgradThreads;
      if (v < kConvPix * CI) *reinterpret_cast<uint4*>(&sI[v / CI][(v % CI) * 8]) = vi[i];
    }
#pragma unroll
    for (int i = 0; i < PG; ++i) {
      const int v = tid + i * kWgradThreads;
      if (v < kConvPix * CG) *reinterpret_cast<uint4*>(&sG[v / CG][(v % CG) * 8]) = vg[i];
    }
    __syncthreads();
    if (p0 + kConvPix < p_end) fetch(p0 + kConvPix);  // in flight during this tile's MMAs
    if (mma_warp) {
#pragma unroll
      for (int ks = 0; ks < kConvPix / 16; ++ks) {
        const int q = lane >> 3, r = lane & 7;
        uint32_t af[WM][4];
#pragma unroll
        for (int wm = 0; wm < WM; ++wm)
          ldsm_x4_t(af[wm], &sI[ks * 16 + r + 8 * (q >> 1)][(mg * WM + wm) * 16 + 8 * (q & 1)]);
        uint32_t bf[WN][2];
        if (WN == 2) {
          uint32_t b4[4];
          ldsm_x4_t(b4, &sG[ks * 16 + r + 8 * (q & 1)][ng * 16 + 8 * (q >> 1)]);
          bf[0][0] = b4[0];
          bf[0][1] = b4[1];
          bf[WN - 1][0] = b4[2];
          bf[WN - 1][1] = b4[3];
        } else {
          ldsm_x2_t(bf[0][0], bf[0][1], &sG[ks * 16 + r + 8 * (q & 1)][ng * 8]);
        }
#pragma unroll
        for (int wm = 0; wm < WM; ++wm)
#pragma unroll
          for (int wn = 0; wn < WN; ++wn) mma_bf16(acc[wm][wn], af[wm], bf[wn][0], bf[wn][1]);
      }
    }
  }
  if (mma_warp) {
    float* out = a.partial + ((size_t)blockIdx.x * 9 + tap) * N * CIN;
#pragma unroll
    for (int wm = 0; wm < WM; ++wm)
#pragma unroll
      for (int wn = 0; wn < WN; ++wn) {
        const int k = (mg * WM + wm) * 16 + g, n = (ng * WN + wn) * 8 + 2 * t;
        out[(size_t)n * CIN + k] = acc[wm][wn][0];
        out[(size_t)(n + 1) * CIN + k] = acc[wm][wn][1];
        out[(size_t)n * CIN + k + 8] = acc[wm][wn][2];
        out[(size_t)(n + 1) * CIN + k + 8] = acc[wm][wn][3];
      }
  }
}

cudaError_t launch_wgrad(int cin, int nt, const WgradArgs& a, cudaStream_t s) {
  const long total = (long)a.B * a.Ho * a.Wo;
  const unsigned chunks = (unsigned)((total + a.chunk_pix - 1) / a.chunk_pix);
  const dim3 grid(chunks, 9);
  if (cin == 16 && nt == 8) wgrad_kernel<16, 8><<<grid, kWgradThreads, 0, s>>>(a);
  else if (cin == 64 && nt == 8) wgrad_kernel<64, 8><<<grid, kWgradThreads, 0, s>>>(a);
  else if (cin == 64 && nt == 1) wgrad_kernel<64, 1><<<grid, kWgradThreads, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Sum of the chunk partials in chunk order into the master-layout gradient [3][3][cin][cout]
// (only the real channels: cin_real, cout_real), one thread per weight; neighbouring threads take
// neighbouring input channels, which are contiguous in the partials.
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int n_chunks, int N, int CIN, int cin_real,
                                    int cout_real, float* __restrict__ gw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int per_tap = cin_real * cout_real;
  if (i >= 9 * per_tap) return;
  const int tap = i / per_tap, r = i % per_tap, co = r / cin_real, ci = r % cin_real;
  float s = 0.f;
  for (int c = 0; c < n_chunks; ++c) s += partial[(((size_t)c * 9 + tap) * N + co) * CIN + ci];
  gw[(size_t)tap * per_tap + (size_t)ci * cout_real + co] = s;
}

// Bias gradient: sum over pixels of g[p, n] in a fixed order: per chunk, 4 pixel groups x the
// channels (neighbouring threads read neighbouring channels), groups added in order; then the
// chunks in order.
constexpr int kBiasGroups = 4;

__global__ void bias_partial_kernel(const bf16* __restrict__ g, long total, int GS, int n_real, int chunk,
                                    float* __restrict__ partial) {
  __shared__ float part[kBiasGroups][64];
  const int n = threadIdx.x & 63, grp = threadIdx.x >> 6;
  float s = 0.f;
  const long p0 = (long)blockIdx.x * chunk;
  if (n < n_real)
    for (long p = p0 + grp; p < p0 + chunk && p < total; p += kBiasGroups) s += __bfloat162float(g[(size_t)p * GS + n]);
  part[grp][n] = s;
  __syncthreads();
  if (grp == 0 && n < n_real) {
    float v = part[0][n];
    for (int q = 1; q < kBiasGroups; ++q) v += part[q][n];
    partial[(size_t)blockIdx.x * n_real + n] = v;
  }
}

__global__ void bias_reduce_kernel(const float* __restrict__ partial, int n_chunks, int n_real, float* __restrict__ gb) {
  const int n = threadIdx.x;
  if (n >= n_real) return;
  float s = 0.f;
  for (int c = 0; c < n_chunks; ++c) s += partial[(size_t)c * n_real + n];
  gb[n] = s;
}

cudaError_t launch_bias_grad(const bf16* g, long total, int GS, int n_real, float* scratch, float* gb, cudaStream_t s) {
  const int chunk = 2048;
  const int chunks = (int)((total + chunk - 1) / chunk);
  bias_partial_kernel<<<chunks, 64 * kBiasGroups, 0, s>>>(g, total, GS, n_real, chunk, scratch);
  bias_reduce_kernel<<<1, 64, 0, s>>>(scratch, chunks, n_real, gb);
  return cudaGetLastError();
}

cudaError_t launch_wgrad_reduce(const float* partial, int n_chunks, int N, int CIN, int cin_real, int cout_real,
                                float* gw, cudaStream_t s) {
  const int n = 9 * cin_real * cout_real;
  wgrad_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(partial, n_chunks, N, CIN, cin_real, cout_real, gw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Weight packing from the FP32 master layout [3][3][cin][cout]:
//   forward:   wk[tap][n = cout_pad][k = cin_pad]
//   transpose: wt[tap][n = cin][k = cout_pad]  with tap -> 8 - tap (the backward-data kernel)
// ---------------------------------------------------------------------------------------------
__global__ void pack_forward_kernel(const float* __restrict__ w, int cin, int cout, int cin_pad, int cout_pad,
                                    bf16* __restrict__ wk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * cout_pad * cin_pad) return;
  const int tap = i / (cout_pad * cin_pad), r = i % (cout_pad * cin_pad), n = r / cin_pad, k = r % cin_pad;
  const float v = (n < cout && k < cin) ? w[((size_t)tap * cin + k) * cout + n] : 0.f;
  wk[i] = __float2bfloat16(v);
}

__global__ void pack_transpose_kernel(const float* __restrict__ w, int cin, int cout, int cout_pad,
                                      bf16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 9 * cin * cout_pad) return;
  const int tp = i / (cin * cout_pad), r = i % (cin * cout_pad), n = r / cout_pad, k = r % cout_pad;
  const int tap = 8 - tp;
  const float v = k < cout ? w[((size_t)tap * cin + n) * cout + k] : 0.f;
  wt[i] = __float2bfloat16(v);
}

cudaError_t launch_pack(const float* w, int cin, int cout, int cin_pad, int cout_pad, bf16* wk, bf16* wt,
                        int cout_pad_t, cudaStream_t s) {
  const int n1 = 9 * cout_pad * cin_pad;
  pack_forward_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(w, cin, cout, cin_pad, cout_pad, wk);
  if (wt) {
    const int n2 = 9 * cin * cout_pad_t;
    pack_transpose_kernel<<<(n2 + 255) / 256, 256, 0, s>>>(w, cin, cout, cout_pad_t, wt);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Input, targets, loss, Adam
// ---------------------------------------------------------------------------------------------
// [n][H][W] depth + colour -> [n][H][W][16] BF16: (depth m - 3) / 2, (R, G, B / 255 - 1/2) x 4, zeros.
__global__ void input_kernel(const uint16_t* __restrict__ depth, const uint32_t* __restrict__ rgba, long n_pix,
                             bf16* __restrict__ x) {
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  // centred and scaled: (depth m - 3) / 2, (colour / 255 - 1/2) x 4
  const float d = ((float)depth[p] * 0.001f - 3.0f) * 0.5f;
  const uint32_t c = rgba[p];
  __align__(16) bf16 v[16];
  v[0] = __float2bfloat16(d);
  v[1] = __float2bfloat16(((float)(c & 0xFF) / 255.f - 0.5f) * 4.0f);
  v[2] = __float2bfloat16(((float)((c >> 8) & 0xFF) / 255.f - 0.5f) * 4.0f);
  v[3] = __float2bfloat16(((float)((c >> 16) & 0xFF) / 255.f - 0.5f) * 4.0f);
  for (int k = 4; k < 16; ++k) v[k] = __float2bfloat16(0.f);
  uint4* dst = reinterpret_cast<uint4*>(x + (size_t)p * 16);
  dst[0] = *reinterpret_cast<uint4*>(&v[0]);
  dst[1] = *reinterpret_cast<uint4*>(&v[8]);
}

cudaError_t launch_input(const uint16_t* depth, const uint32_t* rgba, long n_pix, bf16* x, cudaStream_t s) {
  input_kernel<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(depth, rgba, n_pix, x);
  return cudaGetLastError();
}



// Targets: scene coordinate of each cell's centre pixel minus the origin; w = 1 if scored.
__global__ void targets_kernel(CellArgs a, float4* __restrict__ tgt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = a.Wc * a.Hc;
  if (i >= a.n * per) return;
  const int img = i / per, c = i % per, cx = c % a.Wc, cy = c / a.Wc;
  const int u = cx * 8 + 4, v = cy * 8 + 4;
  const int d = a.depth[((size_t)img * a.H + v) * a.W + u];
  if (d == 0) {
    tgt[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const double z = d / 1000.0;
  const double c0 = z * (u - a.cx) / a.fx, c1 = z * (v - a.cy) / a.fy;
  const double* P = a.poses + 16 * (size_t)img;
  const double y0 = P[0] * c0 + P[1] * c1 + P[2] * z + P[3] - a.ox;
  const double y1 = P[4] * c0 + P[5] * c1 + P[6] * z + P[7] - a.oy;
  const double y2 = P[8] * c0 + P[9] * c1 + P[10] * z + P[11] - a.oz;
  tgt[i] = make_float4((float)y0, (float)y1, (float)y2, 1.f);
}

cudaError_t launch_targets(const CellArgs& a, float4* tgt, cudaStream_t s) {
  const int n = a.n * a.Wc * a.Hc;
  targets_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, tgt);
  return cudaGetLastError();
}

// Loss and its gradient with respect to the head output (stored [cell][8] FP32), written as the
// BF16 gradient [cell][16] (channels 4..15 zero).  One CTA: scored cells are counted first so
// the mean and the summation order are fixed.
__global__ void __launch_bounds__(1024) loss_kernel(const float* __restrict__ out, const float4* __restrict__ tgt,
                                                     int n_cells, bf16* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float red[32];
  __shared__ int redi[32];
  __shared__ float s_inv;
  int cnt = 0;
  for (int i = threadIdx.x; i < n_cells; i += blockDim.x) cnt += tgt[i].w > 0.5f;
  cnt = warp_sum_i(cnt);
  if ((threadIdx.x & 31) == 0) redi[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c += redi[w];
    s_inv = 1.0f / (float)(c > 0 ? c : 1);
  }
  __syncthreads();
  const float inv = s_inv;
  float acc = 0.f;
  for (int i = threadIdx.x; i < n_cells; i += blockDim.x) {
    const float4 y = tgt[i];
    const float* o = out + (size_t)i * 8;
    __align__(16) bf16 gv[16];
    for (int k = 0; k < 16; ++k) gv[k] = __float2bfloat16(0.f);
    if (y.w > 0.5f) {
      // rho(e) + 1/2 e^2 exp(-s) + 3/2 s, rho(e) = sqrt(e^2 + 1e-6): the coordinates follow d rho,
      // s the NLL's derivative with the error held fixed
      const float e0 = o[0] - y.x, e1 = o[1] - y.y, e2 = o[2] - y.z, s = o[3];
      const float sq = e0 * e0 + e1 * e1 + e2 * e2, es = expf(-s), rho = sqrtf(sq + 1e-6f);
      acc += rho + 0.5f * sq * es + 1.5f * s;
      const float gc = inv / rho;
      gv[0] = __float2bfloat16(e0 * gc);
      gv[1] = __float2bfloat16(e1 * gc);
      gv[2] = __float2bfloat16(e2 * gc);
      gv[3] = __float2bfloat16((-0.5f * sq * es + 1.5f) * inv);
    }
    uint4* dst = reinterpret_cast<uint4*>(grad + (size_t)i * 16);
    dst[0] = *reinterpret_cast<uint4*>(&gv[0]);
    dst[1] = *reinterpret_cast<uint4*>(&gv[8]);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *loss = s * inv;
  }
}

cudaError_t launch_loss(const float* out, const float4* tgt, int n_cells, bf16* grad, float* loss, cudaStream_t s) {
  loss_kernel<<<1, 1024, 0, s>>>(out, tgt, n_cells, grad, loss);
  return cudaGetLastError();
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long n, float lr, int t, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Cell forest: the regressor output as a one-tree forest over the cell grid (leaf = cell, one
// Gaussian of mean y_hat + o and covariance exp(s) I per scored cell) plus the coarse view
// (centre-pixel depths) the RANSAC runs on.
// ---------------------------------------------------------------------------------------------


__global__ void cell_forest_kernel(CellForestArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int img = blockIdx.y;
  if (i >= a.L) return;
  const int n = a.Wc * a.Hc;
  float* m = a.modes + ((size_t)img * a.L + i) * kModeFloats;
  uint8_t* nm = a.n_modes + (size_t)img * a.L;
  float4* top = a.top + (size_t)img * a.L;
  if (i >= n) {
    nm[i] = 0;
    top[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int cx = i % a.Wc, cy = i / a.Wc;
  const int d = a.depth[(size_t)img * a.W * a.H + (size_t)(cy * 8 + 4) * a.W + cx * 8 + 4];
  const float* o = a.out + ((size_t)img * n + i) * a.ostride;
  const float s = o[3], inv = expf(-s);
  const float mx = o[0] + a.ox, my = o[1] + a.oy, mz = o[2] + a.oz;
  m[0] = mx;
  m[1] = my;
  m[2] = mz;
  m[3] = inv;
  m[4] = 0.f;
  m[5] = 0.f;
  m[6] = inv;
  m[7] = 0.f;
  m[8] = inv;
  m[9] = -1.5f * 1.8378770664093453f - 1.5f * s;  // log w - 0.5 log det(2 pi exp(s) I), w = 1
  m[10] = 1.f;
  m[11] = 0.f;
  nm[i] = d > 0 ? 1 : 0;
  top[i] = make_float4(mx, my, mz, d > 0 ? 1.f : 0.f);
  a.leaves[(size_t)img * n + i] = (uint16_t)i;
  a.depth_lr[(size_t)img * n + i] = (uint16_t)d;
}

cudaError_t launch_cell_forest(const CellForestArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  cell_forest_kernel<<<dim3((a.L + 255) / 256, a.n), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// Head output [cell][8] -> [cell][4] (scene coordinate - origin, log-variance).
__global__ void head_copy_kernel(const float* __restrict__ head, long n, float* __restrict__ out4) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  reinterpret_cast<float4*>(out4)[i] = make_float4(head[i * 8], head[i * 8 + 1], head[i * 8 + 2], head[i * 8 + 3]);
}

cudaError_t launch_head_copy(const float* head, long n_cells, float* out4, cudaStream_t s) {
  head_copy_kernel<<<(unsigned)((n_cells + 255) / 256), 256, 0, s>>>(head, n_cells, out4);
  return cudaGetLastError();
}

}  // namespace relo
