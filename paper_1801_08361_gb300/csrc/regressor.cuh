// regressor.cuh -- argument blocks and launchers of the regressor kernels (regressor.cu), used by
// the C ABI in api.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "relo_internal.cuh"

namespace relo {

typedef __nv_bfloat16 bf16;

// Convolution (forward / backward-data): out[p, n] = sum_{tap, k} in[src(p, tap), k] W[tap, n, k]
struct ConvArgs {
  const bf16* in;      // [B][Hi][Wi][CIN] (or the real tensor behind a virtual upsampling)
  const bf16* w;       // [9][N][CIN]
  const float* bias;   // [N] or null
  const bf16* mask;    // [B][Ho][Wo][N]: output multiplied by (mask > 0), or null
  bf16* out;           // [B][Ho][Wo][N] or null
  float* out_f32;      // [B][Ho][Wo][N] or null
  int B, Hi, Wi;       // input grid as the convolution sees it (the upsampled grid when upsample)
  int Hs, Ws;          // real input size when upsample
  int Ho, Wo, stride;
  int relu, upsample;
};

// Backward-weight partial sums (see wgrad_kernel)
struct WgradArgs {
  const bf16* in;     // layer input [B][Hi][Wi][CIN]
  const bf16* g;      // gradient of the pre-activation output [B][Ho][Wo][GS] (first N channels used)
  float* partial;     // [n_chunks][9][N][CIN]
  int B, Hi, Wi, Ho, Wo, stride, GS;
  int chunk_pix;      // multiple of 64
};

// Targets (see targets_kernel)
struct CellArgs {
  const uint16_t* depth;  // [n][H][W]
  const double* poses;    // [n][16] camera -> scene
  int n, W, H, Wc, Hc;
  double fx, fy, cx, cy;
  double ox, oy, oz;      // origin
};

// Cell forest (see cell_forest_kernel)
struct CellForestArgs {
  const float* out;        // [n][Hc][Wc][ostride]: head output (ostride 8) or given cells (4)
  int ostride = 8;
  const uint16_t* depth;   // [n][H][W] full-resolution depth
  int n, W, H, Wc, Hc, L;  // L = leaves per tree (power of two >= Wc Hc)
  float ox, oy, oz;
  float* modes;            // [n][L][1][12]
  uint8_t* n_modes;        // [n][L]
  float4* top;             // [n][L]
  uint16_t* leaves;        // [n][Hc][Wc]
  uint16_t* depth_lr;      // [n][Hc][Wc]
};

constexpr int kRegLayers = 8;
constexpr int kRegStride[kRegLayers] = {2, 2, 2, 1, 1, 1, 1, 1};
constexpr int kRegCin[kRegLayers] = {4, 64, 64, 64, 64, 64, 64, 64};
constexpr int kRegCout[kRegLayers] = {64, 64, 64, 64, 64, 64, 64, 4};
constexpr int kRegCinPad[kRegLayers] = {16, 64, 64, 64, 64, 64, 64, 64};
constexpr int kRegCoutPad[kRegLayers] = {64, 64, 64, 64, 64, 64, 64, 8};
constexpr int kWgradChunk = 1024;  // output pixels per backward-weight CTA (multiple of 64)

cudaError_t launch_conv(int cin, int nt, const ConvArgs& a, int n_sms, cudaStream_t s);
cudaError_t launch_wgrad(int cin, int nt, const WgradArgs& a, cudaStream_t s);
cudaError_t launch_wgrad_reduce(const float* partial, int n_chunks, int N, int CIN, int cin_real, int cout_real,
                                float* gw, cudaStream_t s);
cudaError_t launch_bias_grad(const bf16* g, long total, int GS, int n_real, float* scratch, float* gb, cudaStream_t s);
cudaError_t launch_pack(const float* w, int cin, int cout, int cin_pad, int cout_pad, bf16* wk, bf16* wt,
                        int cout_pad_t, cudaStream_t s);
cudaError_t launch_input(const uint16_t* depth, const uint32_t* rgba, long n_pix, bf16* x, cudaStream_t s);
cudaError_t launch_targets(const CellArgs& a, float4* tgt, cudaStream_t s);
cudaError_t launch_loss(const float* out, const float4* tgt, int n_cells, bf16* grad, float* loss, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long n, float lr, int t, cudaStream_t s);
cudaError_t launch_cell_forest(const CellForestArgs& a, cudaStream_t s);

// Forward 3x3 convolution of a cin -> 64-channel layer (cin 16 or 64) on the tcgen05 tensor cores
// (conv_tc.cu): in [B][Hi][Wi][cin], w [9][64][cin], bias [64] (nullable), mask [B][Ho][Wo][64]
// (nullable: outputs where mask <= 0 become 0), out [B][Ho][Wo][64] BF16 NHWC; stride 1 or 2,
// dilation 1-8, zero padding = dilation.  A bounded wait that runs out sets *status = RELO_ETIMEOUT.
// stall_tile >= 0 (test hook) withholds that tile's loads so that the wait for them runs out.
cudaError_t launch_conv_tc(int cin, const bf16* in, int B, int Hi, int Wi, const bf16* w, const float* bias,
                           const bf16* mask, bf16* out, int Ho, int Wo, int stride, int dil, int relu, int32_t* status,
                           int n_sms, cudaStream_t s, unsigned long long timeout_ns, int stall_tile);
cudaError_t launch_head_copy(const float* head, long n_cells, float* out4, cudaStream_t s);

}  // namespace relo
