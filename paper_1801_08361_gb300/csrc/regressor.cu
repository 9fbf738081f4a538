// regressor.cu -- the learned scene-coordinate regressor: BF16 tensor-core 3x3 convolutions
// (forward, backward-data, backward-weight) with FP32 accumulation, the Gaussian-NLL loss, Adam,
// and the cell forest that hands its output to the preemptive RANSAC.
//
// The paper relocalises with a forest (Sec. 3.3 (b)); this network is the workload's alternative
// relocaliser for a scene, trained online on renders of the scene's own voxel map.  Readings
// (identical in the CPU oracle): 4 input channels (depth in metres, RGB / 255), eight 3x3
// convolutions with zero padding, 64 channels, strides 2, 2, 2, 1, 1, 1, 1, 1, ReLU after
// layers 1-7, 4 outputs per 8 x 8-pixel cell (scene coordinate - origin, log-variance s); the
// target of a cell is the scene coordinate of its centre pixel; loss = mean over scored cells of
// 1/2 |y - y_hat|^2 exp(-s) + 3/2 s; Adam (0.9, 0.999, 1e-8).
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


constexpr int kConvPix = 64;  // output pixels per tile (4 warps x 16)

template <int CIN, int NT>
__global__ void __launch_bounds__(128) conv_kernel(ConvArgs a) {
  constexpr int N = NT * 8;
  constexpr int RS = CIN + 8;  // padded row stride (bf16) of the shared tiles: no bank conflicts
  extern __shared__ __align__(16) unsigned char conv_smem[];
  bf16* sW = reinterpret_cast<bf16*>(conv_smem);   // [9][N][RS]
  bf16* sA = sW + 9 * N * RS;                       // [64][RS]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  for (int v = tid; v < 9 * N * (CIN / 8); v += 128) {
    const int row = v / (CIN / 8), c8 = v % (CIN / 8);
    *reinterpret_cast<uint4*>(sW + row * RS + c8 * 8) = __ldg(reinterpret_cast<const uint4*>(a.w + (size_t)row * CIN) + c8);
  }
  const long total = (long)a.B * a.Ho * a.Wo;
  const long n_tiles = (total + kConvPix - 1) / kConvPix;
  for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long m0 = tile * kConvPix;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap % 3;
      __syncthreads();  // previous readers of sA (and, on the first pass, the weight stores)
      for (int v = tid; v < kConvPix * (CIN / 8); v += 128) {
        const int m = v / (CIN / 8), c8 = v % (CIN / 8);
        const long p = m0 + m;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (p < total) {
          const int ox = (int)(p % a.Wo), oy = (int)((p / a.Wo) % a.Ho), b = (int)(p / ((long)a.Wo * a.Ho));
          const int iy = oy * a.stride + ky - 1, ix = ox * a.stride + kx - 1;
          if (iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Wi) {
            if (!a.upsample) {
              val = __ldg(reinterpret_cast<const uint4*>(a.in + (((size_t)b * a.Hi + iy) * a.Wi + ix) * CIN) + c8);
            } else if (!(iy & 1) && !(ix & 1) && (iy >> 1) < a.Hs && (ix >> 1) < a.Ws) {
              val = __ldg(reinterpret_cast<const uint4*>(a.in + (((size_t)b * a.Hs + (iy >> 1)) * a.Ws + (ix >> 1)) * CIN) + c8);
            }
          }
        }
        *reinterpret_cast<uint4*>(sA + m * RS + c8 * 8) = val;
      }
      __syncthreads();
      const bf16* Ar = sA + (warp * 16 + g) * RS;
      const bf16* Wt = sW + tap * N * RS;
#pragma unroll
      for (int ks = 0; ks < CIN / 16; ++ks) {
        const int k0 = ks * 16 + 2 * t;
        uint32_t af[4] = {ld32(Ar + k0), ld32(Ar + 8 * RS + k0), ld32(Ar + k0 + 8), ld32(Ar + 8 * RS + k0 + 8)};
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          const bf16* Br = Wt + (j * 8 + g) * RS;
          mma_bf16(acc[j], af, ld32(Br + k0), ld32(Br + k0 + 8));
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
  const size_t smem = (size_t)(9 * N + kConvPix) * RS * sizeof(bf16);
  cudaError_t e = cudaFuncSetAttribute(conv_kernel<CIN, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long total = (long)a.B * a.Ho * a.Wo;
  const long tiles = (total + kConvPix - 1) / kConvPix;
  const long grid = tiles < (long)n_sms * 2 ? tiles : (long)n_sms * 2;
  if (grid <= 0) return cudaSuccess;
  conv_kernel<CIN, NT><<<(unsigned)grid, 128, smem, s>>>(a);
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
// ---------------------------------------------------------------------------------------------


template <int CIN, int NT>
__global__ void __launch_bounds__(128) wgrad_kernel(WgradArgs a) {
  constexpr int N = NT * 8;
  constexpr int MT = (N + 15) / 16;   // m16 tiles over the output channels
  constexpr int PS = kConvPix + 8;    // padded pixel stride of the transposed tiles
  __shared__ __align__(16) bf16 sG[MT * 16][PS];  // g^T: [n][pixel]
  __shared__ __align__(16) bf16 sI[CIN][PS];      // in^T: [k][pixel]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int tap = blockIdx.y, ky = tap / 3, kx = tap % 3;
  const long total = (long)a.B * a.Ho * a.Wo;
  const long p_begin = (long)blockIdx.x * a.chunk_pix;
  float acc[CIN / 8][4];
#pragma unroll
  for (int j = 0; j < CIN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (long p0 = p_begin; p0 < p_begin + a.chunk_pix && p0 < total; p0 += kConvPix) {
    __syncthreads();
    // staged transposed; consecutive threads read consecutive channels of a pixel (coalesced)
    for (int v = tid; v < kConvPix * (MT * 16); v += 128) {
      const int n = v % (MT * 16), m = v / (MT * 16);
      const long p = p0 + m;
      bf16 val = __float2bfloat16(0.f);
      if (p < total && n < N) val = a.g[(size_t)p * a.GS + n];
      sG[n][m] = val;
    }
    for (int v = tid; v < kConvPix * CIN; v += 128) {
      const int k = v % CIN, m = v / CIN;
      const long p = p0 + m;
      bf16 val = __float2bfloat16(0.f);
      if (p < total) {
        const int ox = (int)(p % a.Wo), oy = (int)((p / a.Wo) % a.Ho), b = (int)(p / ((long)a.Wo * a.Ho));
        const int iy = oy * a.stride + ky - 1, ix = ox * a.stride + kx - 1;
        if (iy >= 0 && ix >= 0 && iy < a.Hi && ix < a.Wi) val = a.in[(((size_t)b * a.Hi + iy) * a.Wi + ix) * CIN + k];
      }
      sI[k][m] = val;
    }
    __syncthreads();
    if (warp < MT) {
#pragma unroll
      for (int ks = 0; ks < kConvPix / 16; ++ks) {
        const int k0 = ks * 16 + 2 * t;
        const bf16* Ar = &sG[warp * 16 + g][0];
        uint32_t af[4] = {ld32(Ar + k0), ld32(Ar + 8 * PS + k0), ld32(Ar + k0 + 8), ld32(Ar + 8 * PS + k0 + 8)};
#pragma unroll
        for (int j = 0; j < CIN / 8; ++j) {
          const bf16* Br = &sI[j * 8 + g][0];
          mma_bf16(acc[j], af, ld32(Br + k0), ld32(Br + k0 + 8));
        }
      }
    }
  }
  if (warp < MT) {
    float* out = a.partial + ((size_t)blockIdx.x * 9 + tap) * N * CIN;
#pragma unroll
    for (int j = 0; j < CIN / 8; ++j) {
      const int k0 = j * 8 + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int n = warp * 16 + g + 8 * h;
        if (n < N) {
          out[(size_t)n * CIN + k0] = acc[j][2 * h];
          out[(size_t)n * CIN + k0 + 1] = acc[j][2 * h + 1];
        }
      }
    }
  }
}

cudaError_t launch_wgrad(int cin, int nt, const WgradArgs& a, cudaStream_t s) {
  const long total = (long)a.B * a.Ho * a.Wo;
  const unsigned chunks = (unsigned)((total + a.chunk_pix - 1) / a.chunk_pix);
  const dim3 grid(chunks, 9);
  if (cin == 16 && nt == 8) wgrad_kernel<16, 8><<<grid, 128, 0, s>>>(a);
  else if (cin == 64 && nt == 8) wgrad_kernel<64, 8><<<grid, 128, 0, s>>>(a);
  else if (cin == 64 && nt == 1) wgrad_kernel<64, 1><<<grid, 128, 0, s>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// Sum of the chunk partials in chunk order into the master-layout gradient [3][3][cin][cout]
// (only the real channels: cin_real, cout_real), one thread per weight.
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int n_chunks, int N, int CIN, int cin_real,
                                    int cout_real, float* __restrict__ gw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int per_tap = cin_real * cout_real;
  if (i >= 9 * per_tap) return;
  const int tap = i / per_tap, r = i % per_tap, ci = r / cout_real, co = r % cout_real;
  float s = 0.f;
  for (int c = 0; c < n_chunks; ++c) s += partial[(((size_t)c * 9 + tap) * N + co) * CIN + ci];
  gw[i] = s;
}

// Bias gradient: sum over pixels of g[p, n] (two passes for a fixed summation order).
__global__ void bias_partial_kernel(const bf16* __restrict__ g, long total, int GS, int n_real, int chunk,
                                    float* __restrict__ partial) {
  const int n = threadIdx.x;
  if (n >= n_real) return;
  float s = 0.f;
  const long p0 = (long)blockIdx.x * chunk;
  for (long p = p0; p < p0 + chunk && p < total; ++p) s += __bfloat162float(g[(size_t)p * GS + n]);
  partial[(size_t)blockIdx.x * n_real + n] = s;
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
  bias_partial_kernel<<<chunks, 64, 0, s>>>(g, total, GS, n_real, chunk, scratch);
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
// [n][H][W] depth + colour -> [n][H][W][16] BF16: depth in metres, R, G, B / 255, zeros.
__global__ void input_kernel(const uint16_t* __restrict__ depth, const uint32_t* __restrict__ rgba, long n_pix,
                             bf16* __restrict__ x) {
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  const float d = (float)depth[p] * 0.001f;
  const uint32_t c = rgba[p];
  __align__(16) bf16 v[16];
  v[0] = __float2bfloat16(d);
  v[1] = __float2bfloat16((float)(c & 0xFF) / 255.f);
  v[2] = __float2bfloat16((float)((c >> 8) & 0xFF) / 255.f);
  v[3] = __float2bfloat16((float)((c >> 16) & 0xFF) / 255.f);
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
      const float e0 = o[0] - y.x, e1 = o[1] - y.y, e2 = o[2] - y.z, s = o[3];
      const float sq = e0 * e0 + e1 * e1 + e2 * e2, es = expf(-s);
      acc += 0.5f * sq * es + 1.5f * s;
      gv[0] = __float2bfloat16(e0 * es * inv);
      gv[1] = __float2bfloat16(e1 * es * inv);
      gv[2] = __float2bfloat16(e2 * es * inv);
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
  const float* o = a.out + ((size_t)img * n + i) * 8;
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
