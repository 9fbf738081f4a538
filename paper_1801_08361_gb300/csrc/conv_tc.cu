// conv_tc.cu -- forward 3x3 convolution of the regressor's 64 -> 64-channel layers on the
// fifth-generation tensor cores (tcgen05, sm_103a).
//
// Implicit GEMM: the 128 output pixels of a tile (M) times the 64 output channels (N), contracted
// over 9 taps x 64 input channels (K).  For each tap the tile's input rows arrive in one TMA load:
// a 4-D tensor map over the NHWC BF16 activations [B][H][W][64] whose box is 64 channels x Wt x Ht
// pixels (Wt Ht = 128), walked with element strides equal to the layer's stride and started at the
// tap's offset ((ky - 1), (kx - 1)) x dilation.  Rows outside the image are zero-filled by the TMA
// unit: the convolution's zero padding.  A row is 64 channels = 128 B and lands 128-B swizzled,
// which is the canonical K-major layout of the MMA's shared-memory operand (8-row atoms of
// 1024 B).  The 9 taps' weights [9][64 out][64 in] are stored once per CTA in the same layout.
//
// Roles (one persistent CTA per SM, 6 warps): warp 0 issues the TMA loads into a ring of kStages
// buffers; one thread of warp 1 issues the 4 MMAs (K = 16 each) of every tap into one of two TMEM
// accumulators (128 lanes x 64 FP32 columns each) and commits them to mbarriers; warps 2-5 read a
// finished accumulator back (tcgen05.ld: each warp its quarter of the 128 lanes), add the bias,
// apply ReLU and store BF16 NHWC rows while the next tile accumulates into the other buffer.
//
// Every mbarrier wait is bounded by a wall-clock limit (the global nanosecond timer): a wait that
// runs out records RELO_ETIMEOUT in *status, raises the CTA's abort flag (every other wait of the
// CTA then gives up too), the producer waits (bounded) for the loads it still has in flight, and
// the CTA frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "regressor.cuh"

namespace relo {
namespace {

constexpr int kTcThreads = 192;             // 6 warps
constexpr int kTcM = 128, kTcN = 64;
constexpr int kTcAccCols = 64;              // FP32 columns of one accumulator
constexpr int kTcTmemCols = 2 * kTcAccCols;

// Per input-channel count CIN (64: the inner layers; 16: the first layer, its 4 channels padded):
// a pixel row is CIN x 2 bytes, which is also the swizzle span of the operand layout (128 B or 32 B;
// 8-row atoms of 1024 B or 256 B).
template <int CIN>
struct TcShape {
  static constexpr int kRowBytes = CIN * 2;
  static constexpr int kABytes = kTcM * kRowBytes;           // one tap's tile: 16 KB or 4 KB
  static constexpr int kWBytes = 9 * kTcN * kRowBytes;
  static constexpr int kAtomBytes = 8 * kRowBytes;           // stride between 8-row atoms
  static constexpr int kChunks = kRowBytes / 16;             // 16-byte chunks per row
  static constexpr uint64_t kLayout = CIN == 64 ? 2 : 6;     // descriptor swizzle: 128 B / 32 B
  // A-operand ring: 64 KB of tap tiles in flight (4 stages of 16 KB, or 16 of 4 KB)
  static constexpr int kStages = CIN == 64 ? 4 : 16;
  static constexpr size_t kSmem = 1024 + (size_t)kWBytes + (size_t)kStages * kABytes;
  static_assert(CIN == 16 || CIN == 64, "64 -> 64 and 16 -> 64 channels");
};

struct TcArgs {
  const float* bias;      // [64] or null
  const bf16* mask;       // [B][Ho][Wo][64]: outputs where mask <= 0 are zeroed (ReLU derivative), or null
  const bf16* w;          // [9][64 out][64 in]
  bf16* out;              // [B][Ho][Wo][64]
  int32_t* status;        // RELO_ETIMEOUT when a wait ran out (else untouched)
  int B, Ho, Wo, stride, dil, relu;
  int Wt, Ht;             // tile shape in output pixels, Wt * Ht = 128
  int tiles_x, tiles_y, n_tiles;
  unsigned long long timeout_ns;
  int stall_tile;         // test hook: the producer issues no load for this tile (-1: none)
};

// ---- PTX wrappers ------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.  False: the limit ran out or
// another role of the CTA gave up first (abort); the caller then stops its role.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, const TcArgs& a) {
  const unsigned long long t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      if (global_ns() - t0 > a.timeout_ns) {
        *abort = 1;
        atomicExch(a.status, RELO_ETIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in a swizzled layout whose span equals a
// row: start address, stride between 8-row atoms (the leading offset is unused with these
// swizzles), descriptor version 1 (bits 46-47), swizzle mode (bits 61-63: 2 = 128 B, 6 = 32 B).
template <int CIN>
__device__ __forceinline__ uint64_t operand_desc(uint32_t addr) {
  using S = TcShape<CIN>;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(S::kAtomBytes >> 4) << 32) |
         ((uint64_t)1 << 46) | (S::kLayout << 61);
}

// Offset of 16-byte chunk j of row r in the swizzled layout: the chunk index XOR the row's position
// in its 8-row atom (128 B: 3 bits), or its bit 2 (32 B: 1 bit), as the TMA unit writes it.
template <int CIN>
__device__ __forceinline__ int swizzled(int r, int j) {
  using S = TcShape<CIN>;
  const int x = CIN == 64 ? (r & 7) : ((r >> 2) & 1);
  return r * S::kRowBytes + ((j ^ x) << 4);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive FP32 columns: thread i of the warp gets lane (base + i), columns col..col+31
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tile_origin(const TcArgs& a, int t, int& b, int& oy0, int& ox0) {
  const int per = a.tiles_x * a.tiles_y;
  b = t / per;
  const int r = t - b * per;
  oy0 = (r / a.tiles_x) * a.Ht;
  ox0 = (r % a.tiles_x) * a.Wt;
}

template <int CIN>
__global__ void __launch_bounds__(kTcThreads, 1) conv_tc_kernel(const __grid_constant__ CUtensorMap in_map, TcArgs a) {
  using S = TcShape<CIN>;
  constexpr int kTcStages = S::kStages;
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ uint64_t bars[2 * kTcStages + 5];     // full[s], empty[s], acc_full[2], acc_empty[2], drain
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sW = base;                    // [9][64][row] swizzled
  uint8_t* sA = base + S::kWBytes;       // [kStages][128][row] swizzled
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kTcStages]);
  const uint32_t accf0 = smem_u32(&bars[2 * kTcStages]), acce0 = smem_u32(&bars[2 * kTcStages + 2]);
  const uint32_t drain = smem_u32(&bars[2 * kTcStages + 4]);
  volatile int* abort = &abort_sh;

  // weights -> shared memory in the swizzled K-major layout
  for (int v = threadIdx.x; v < 9 * kTcN * S::kChunks; v += kTcThreads) {
    const int row = v / S::kChunks, j = v % S::kChunks;
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(a.w) + v);
    *reinterpret_cast<uint4*>(sW + swizzled<CIN>(row, j)) = x;
  }
  if (threadIdx.x == 0) {
    abort_sh = 0;
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the generic-proxy stores of the weights must be visible to the tensor cores' async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    // ---- producer: one TMA load per (tile, tap) ----
    if (lane == 0) {
      uint32_t q = 0;
      int issued[kTcStages];         // stage s holds a load not yet known to be consumed ...
      uint32_t phase[kTcStages];     // ... which completes the full barrier's phase of this parity
      for (int s = 0; s < kTcStages; ++s) issued[s] = 0, phase[s] = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < a.n_tiles; t += gridDim.x) {
        int b, oy0, ox0;
        tile_origin(a, t, b, oy0, ox0);
        for (int tap = 0; tap < 9; ++tap, ++q) {
          const int s = (int)(q % kTcStages);
          const uint32_t round = q / kTcStages;
          if (round > 0 && !mbar_wait(empty0 + 8 * s, (round - 1) & 1, abort, a)) {
            ok = false;
            break;
          }
          issued[s] = 0;
          if (t == a.stall_tile) continue;   // test hook: the consumer's wait for this stage runs out
          const int ky = tap / 3, kx = tap % 3;
          mbar_expect_tx(full0 + 8 * s, S::kABytes);
          tma_load_4d(smem_u32(sA + s * S::kABytes), &in_map, full0 + 8 * s, 0, ox0 * a.stride + (kx - 1) * a.dil,
                      oy0 * a.stride + (ky - 1) * a.dil, b);
          issued[s] = 1;
          phase[s] = round & 1;
        }
      }
      if (!ok || *abort) {
        // copies still in flight land before the CTA's shared memory is released
        for (int s = 0; s < kTcStages; ++s) {
          if (!issued[s]) continue;
          const unsigned long long t0 = global_ns();
          while (!mbar_test(full0 + 8 * s, phase[s]) && global_ns() - t0 < a.timeout_ns) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      uint32_t q = 0, it = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < a.n_tiles; t += gridDim.x, ++it) {
        const int buf = (int)(it & 1);
        const uint32_t use = it >> 1;
        if (use > 0 && !mbar_wait(acce0 + 8 * buf, (use - 1) & 1, abort, a)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * kTcAccCols);
        for (int tap = 0; tap < 9; ++tap, ++q) {
          const int s = (int)(q % kTcStages);
          if (!mbar_wait(full0 + 8 * s, (q / kTcStages) & 1, abort, a)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + s * S::kABytes), b0 = smem_u32(sW + tap * (kTcN * S::kRowBytes));
#pragma unroll
          for (int kk = 0; kk < CIN / 16; ++kk)
            umma_bf16(d, operand_desc<CIN>(a0 + 32 * kk), operand_desc<CIN>(b0 + 32 * kk), (tap > 0 || kk > 0) ? 1u : 0u);
          umma_commit(empty0 + 8 * s);      // the stage is free once these MMAs have read it
        }
        if (ok) umma_commit(accf0 + 8 * buf);
      }
      if (!ok || *abort) {
        // MMAs still in flight finish before the TMEM is released
        umma_commit(drain);
        const unsigned long long t0 = global_ns();
        while (!mbar_test(drain, 0) && global_ns() - t0 < a.timeout_ns) {
        }
      }
    }
  } else {
    // ---- epilogue: warps 2-5, TMEM lane quarter = warp % 4 ----
    const int quarter = warp & 3;
    uint32_t it = 0;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x, ++it) {
      const int buf = (int)(it & 1);
      // lane 0 waits for the accumulator and tells the warp: tcgen05.ld needs the whole warp
      bool ready = lane == 0 ? mbar_wait(accf0 + 8 * buf, (it >> 1) & 1, abort, a) : false;
      ready = __shfl_sync(0xffffffffu, ready, 0);
      if (!ready) break;
      tc_fence_after();
      const int m = quarter * 32 + lane;
      float v0[32], v1[32];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * kTcAccCols);
      tmem_ld32(taddr, v0);
      tmem_ld32(taddr + 32, v1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * buf);
      int b, oy0, ox0;
      tile_origin(a, t, b, oy0, ox0);
      const int oy = oy0 + m / a.Wt, ox = ox0 + m % a.Wt;
      if (oy < a.Ho && ox < a.Wo) {
        const size_t px = ((size_t)b * a.Ho + oy) * a.Wo + ox;
        uint4* dst = reinterpret_cast<uint4*>(a.out + px * kTcN);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          uint4 mk = make_uint4(0u, 0u, 0u, 0u);
          if (a.mask) mk = __ldg(reinterpret_cast<const uint4*>(a.mask + px * kTcN) + j);
          const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
          uint32_t pk[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int n = 8 * j + 2 * e;
            const float* v = n < 32 ? v0 : v1;
            float x0 = v[n & 31], x1 = v[(n & 31) + 1];
            if (a.bias) {
              x0 += __ldg(&a.bias[n]);
              x1 += __ldg(&a.bias[n + 1]);
            }
            if (a.relu) {
              x0 = fmaxf(x0, 0.f);
              x1 = fmaxf(x1, 0.f);
            }
            if (a.mask) {
              const __nv_bfloat162 mm = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
              if (!(__bfloat162float(mm.x) > 0.f)) x0 = 0.f;
              if (!(__bfloat162float(mm.y) > 0.f)) x1 = 0.f;
            }
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            pk[e] = *reinterpret_cast<const uint32_t*>(&h);
          }
          dst[j] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
}

// ---- host ---------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

int conv_tc_tile_width(int Wo) {
  // output tiles of Wt x (128 / Wt) pixels: the widest of 128, 64, 32, 16 that wastes no column,
  // else 16
  for (int wt : {128, 64, 32, 16})
    if (Wo % wt == 0) return wt;
  return 16;
}

template <int CIN>
cudaError_t launch_conv_tc_t(const bf16* in, int B, int Hi, int Wi, const bf16* w, const float* bias, const bf16* mask,
                             bf16* out, int Ho, int Wo, int stride, int dil, int relu, int32_t* status, int n_sms,
                             cudaStream_t s, unsigned long long timeout_ns, int stall_tile) {
  using S = TcShape<CIN>;
  if (B <= 0 || Ho <= 0 || Wo <= 0) return cudaSuccess;
  if ((stride != 1 && stride != 2) || dil < 1 || dil > 8 || !status) return cudaErrorInvalidValue;
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15) || ((uintptr_t)w & 15)) return cudaErrorMisalignedAddress;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (mask && ((uintptr_t)mask & 15)) return cudaErrorMisalignedAddress;
  TcArgs a{};
  a.bias = bias;
  a.mask = mask;
  a.w = w;
  a.out = out;
  a.status = status;
  a.B = B;
  a.Ho = Ho;
  a.Wo = Wo;
  a.stride = stride;
  a.dil = dil;
  a.relu = relu;
  a.Wt = conv_tc_tile_width(Wo);
  a.Ht = kTcM / a.Wt;
  a.tiles_x = (Wo + a.Wt - 1) / a.Wt;
  a.tiles_y = (Ho + a.Ht - 1) / a.Ht;
  a.n_tiles = B * a.tiles_x * a.tiles_y;
  a.timeout_ns = timeout_ns;
  a.stall_tile = stall_tile;
  // 4-D map: (channel, x, y, image), box CIN x Wt*stride x Ht*stride x 1 walked with element strides
  // (1, stride, stride, 1): Wt x Ht pixel rows of CIN x 2 bytes
  CUtensorMap map;
  const cuuint64_t dims[4] = {(cuuint64_t)CIN, (cuuint64_t)Wi, (cuuint64_t)Hi, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)CIN * 2, (cuuint64_t)Wi * CIN * 2, (cuuint64_t)Hi * Wi * CIN * 2};
  const cuuint32_t box[4] = {(cuuint32_t)CIN, (cuuint32_t)(a.Wt * stride), (cuuint32_t)(a.Ht * stride), 1};
  const cuuint32_t estr[4] = {1, (cuuint32_t)stride, (cuuint32_t)stride, 1};
  if (box[1] > 256 || box[2] > 256) return cudaErrorInvalidValue;
  const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(in), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CIN == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  static PerDevice configured;
  int dummy = 0;
  cudaError_t e = per_device(configured, &dummy, [](int, int* v) {
    *v = 1;
    return cudaFuncSetAttribute(conv_tc_kernel<CIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
  });
  if (e != cudaSuccess) return e;
  const int grid = std::min(a.n_tiles, n_sms);
  conv_tc_kernel<CIN><<<grid, kTcThreads, S::kSmem, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv_tc(int cin, const bf16* in, int B, int Hi, int Wi, const bf16* w, const float* bias,
                           const bf16* mask, bf16* out, int Ho, int Wo, int stride, int dil, int relu, int32_t* status,
                           int n_sms, cudaStream_t s, unsigned long long timeout_ns, int stall_tile) {
  if (cin == 64)
    return launch_conv_tc_t<64>(in, B, Hi, Wi, w, bias, mask, out, Ho, Wo, stride, dil, relu, status, n_sms, s,
                                timeout_ns, stall_tile);
  if (cin == 16)
    return launch_conv_tc_t<16>(in, B, Hi, Wi, w, bias, mask, out, Ho, Wo, stride, dil, relu, status, n_sms, s,
                                timeout_ns, stall_tile);
  return cudaErrorInvalidValue;
}

}  // namespace relo
