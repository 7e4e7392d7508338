// Tensor-core convolutions of the learned warm start (not part of the paper).
//
// 3x3 dilated convolutions with zero padding on 64-wide images, BF16 operands,
// FP32 accumulation, as implicit GEMMs on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory) with every operand tile loaded
// by the Tensor Memory Accelerator (cp.async.bulk.tensor) into 128-byte
// swizzled shared memory.
//
// Layouts: activations NHWC, channels padded to a multiple of 64 (K chunks of
// 64 channels = one 128-byte swizzle row); weights K-major per output row,
// [rows][9 taps][channels].
//
//  forward          y[p][co]  = sum_{tap, ci} Wf[co][tap][ci] x[p + s(tap)][ci]
//                   GEMM M = 128 pixels (two image rows), N = output channels,
//                   K = 9 x channels.  The A tile of tap s = (dy, dx) dil is a
//                   4-D TMA box of x at (c, dx dil, y0 + dy dil, n): the shift
//                   lies on outer dimensions and out-of-image taps read the
//                   TMA's zero fill (zero padding for free).
//  backward (data)  the same kernel on dy with Wb[ci][tap][co] = Wf[co][8 - tap][ci]
//                   (s(8 - tap) = -s(tap)); its epilogue multiplies by the
//                   derivative of the previous layer's leaky ReLU.
//  backward (weight) dW[co][tap][ci] = sum_p dy[p][co] x[p + s(tap)][ci]: a GEMM
//                   with M = 128 output channels, N = input channels, K = pixels,
//                   both operands K-major (pixels contiguous) from transposed
//                   copies dyT[co][n][y][x] and xT[dx][ci][n][y][x] (x-shifted by
//                   dx dil on the copy, so that the TMA's innermost coordinate
//                   stays 0); the y shift is a TMA coordinate.  Split over image
//                   rows into partial sums, reduced by a second kernel.
//
// The forward / data-gradient kernel is persistent (one CTA per SM walks its
// share of the 128-pixel tiles) with warp roles: one thread streams the TMA
// loads into a 6-stage ring, one issues the MMAs (one per 16 K-elements) and
// commits each stage back to the producer, four epilogue warps read the
// accumulator (warp w: tensor-memory lanes 32 (w % 4) ..) while the MMAs of
// the next tile run into the second of two accumulators.  The weight-gradient
// kernel takes one (tap, row range) per CTA with the same producer / MMA
// split.  Every wait on an mbarrier is bounded by the global timer; on expiry
// the CTA sets an error flag, skips its stores, lets the copies and MMAs in
// flight finish (bounded) and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kStages = 4;
constexpr int kTileBytesA = 128 * 128;  // 128 rows x 128 bytes
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s
constexpr float kLeakTc = 0.1f;

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of b: false once *abort is set or the limit
// of the global timer has passed (which sets *abort).
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort) {
  const unsigned long long t0 = gtimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 63) == 63) {
      if (*abort) return false;
      if (gtimer() - t0 > kWaitLimitNs) {
        *abort = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5, %6}], [%7];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (tile 1024-byte aligned).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;             // descriptor version of this architecture
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

struct ConvTcArgs {
  int N, H, W;        // images and image size (W = 64, H even)
  int cin_pad;        // K channels per tap (multiple of 64)
  int nout;           // output channels written (<= BN)
  int ldy;            // channel stride of the BF16 output (>= nout)
  int dil;
  int mode;           // 0: + bias, 1: + bias then leaky ReLU, 2: x leaky-ReLU derivative of ref
  const float* bias;  // [nout] (modes 0, 1)
  const __nv_bfloat16* ref;  // mode 2: [P][ldref] the previous layer's output (sign decides the slope)
  int ldref;
  __nv_bfloat16* y;   // [P][ldy] or NULL
  float* yf;          // [P][nout] or NULL
  int* err;           // set when a bounded wait expired
};

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Bounded wait that ignores the abort flag: used only to let copies and MMAs
// that are already in flight finish before the CTA frees its resources.
__device__ void mbar_drain(uint64_t* b, uint32_t parity) {
  const unsigned long long t0 = gtimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return;
    if ((it & 63) == 63 && gtimer() - t0 > kWaitLimitNs / 10) return;
  }
}

constexpr int kConvStages = 6;  // 6 x (16 KB + BN x 128 B): 192 KB at BN = 128

// Forward / backward-data convolution, persistent: CTA c takes the 128-pixel
// tiles c, c + G, c + 2G, ... (G = grid size, one CTA per SM).  Six warps:
// warp 0 (one thread) streams the TMA loads of all its tiles through a
// 6-stage ring; warp 1 owns tensor memory and (one thread) issues the MMAs;
// warps 2-5 run the epilogue, warp w reading tensor-memory lanes 32 (w % 4)
// .. 32 (w % 4) + 31.  Two accumulators in tensor memory let the epilogue of
// tile i overlap the MMAs of tile i + 1: acc_full[b] (committed by the MMAs)
// hands accumulator b to the epilogue, acc_empty[b] (one arrival per epilogue
// warp) hands it back.
template <int BN>
__global__ void __launch_bounds__(192, 1)
    conv_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ConvTcArgs a) {
  constexpr int kTileBytesB = BN * 128;
  constexpr int kCols = BN < 32 ? 32 : BN;  // columns of one accumulator
  constexpr int kAllocCols = 2 * kCols;     // a power of two >= 32
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kConvStages * kTileBytesA;
  __shared__ __align__(8) uint64_t full[kConvStages], empty[kConvStages], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rows_per_tile = 128 / a.W;
  const int tiles_per_img = a.H / rows_per_tile;
  const int ntiles = a.N * tiles_per_img;
  const int chunks = a.cin_pad / 64;
  const int nk = 9 * chunks;
  if (tid == 0) {
    for (int s = 0; s < kConvStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kAllocCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  volatile int* abort = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // producer: the A (activations) and B (weights) tiles of every K step of every tile
      int k = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int n = t / tiles_per_img, y0 = (t % tiles_per_img) * rows_per_tile;
        for (int kt = 0; kt < nk; ++kt) {
          const int s = k % kConvStages;
          if (k >= kConvStages && !mbar_wait(&empty[s], ((k / kConvStages) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          const int tap = kt / chunks, c = kt % chunks;
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
          mbar_expect_tx(&full[s], kTileBytesA + kTileBytesB);
          tma_load_4d(sA + s * kTileBytesA, &tmA, &full[s], c * 64, dx * a.dil, y0 + dy * a.dil, n);
          tma_load_2d(sB + s * kTileBytesB, &tmB, &full[s], tap * a.cin_pad + c * 64, 0);
          ++k;
        }
      }
      if (!ok) {
        // let the copies in flight land before the CTA's shared memory goes away
        for (int j = (k > kConvStages ? k - kConvStages : 0); j < k; ++j)
          mbar_drain(&full[j % kConvStages], (j / kConvStages) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: 4 MMAs of K = 16 per stage, each stage returned to the producer
      constexpr uint32_t idesc = idesc_bf16(128, BN);
      int k = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int ab = i & 1;
        // accumulator ab is free once the epilogue has read tile i - 2 out of it
        if (i >= 2 && !mbar_wait(&acc_empty[ab], ((i >> 1) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t acc = tmem + (uint32_t)(ab * kCols);
        for (int kt = 0; kt < nk; ++kt, ++k) {
          const int s = k % kConvStages;
          if (!mbar_wait(&full[s], (k / kConvStages) & 1, abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(sA + s * kTileBytesA), b0 = smem_u32(sB + s * kTileBytesB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(acc, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc, (kt | kk) != 0);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[ab]);
      }
      // every MMA issued has completed before tensor memory is freed
      mma_commit(&drain);
      mbar_drain(&drain, 0);
    }
  } else {
    // epilogue: thread (warp w, lane l) = pixel row 32 (w % 4) + l of each tile
    const int q = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int ab = i & 1;
      bool ok = mbar_wait(&acc_full[ab], (i >> 1) & 1, abort);
      ok = __all_sync(0xffffffffu, ok ? 1 : 0) && !*abort;  // warp-uniform before the aligned TMEM loads
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int n = t / tiles_per_img, y0 = (t % tiles_per_img) * rows_per_tile;
      const int row = q * 32 + lane;
      const int64_t p = ((int64_t)n * a.H + y0 + row / a.W) * a.W + row % a.W;
#pragma unroll
      for (int cb = 0; cb < BN; cb += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * kCols + cb), v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int co = cb + k;
          if (a.mode == 2) {
            const float r = (co < a.nout) ? __bfloat162float(a.ref[p * a.ldref + co]) : 0.0f;
            v[k] *= (r < 0.0f) ? kLeakTc : 1.0f;
          } else {
            v[k] += (co < a.nout) ? a.bias[co] : 0.0f;
            if (a.mode == 1 && v[k] < 0.0f) v[k] *= kLeakTc;
          }
          if (co >= a.nout) v[k] = 0.0f;
        }
        if (a.y) {
          // 16 channels = 32 bytes, two 16-byte stores (ldy is a multiple of 16)
          __align__(16) __nv_bfloat162 h[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
          if (cb < a.ldy) {
            uint4* dst = reinterpret_cast<uint4*>(a.y + p * a.ldy + cb);
            dst[0] = *reinterpret_cast<const uint4*>(&h[0]);
            dst[1] = *reinterpret_cast<const uint4*>(&h[4]);
          }
        }
        if (a.yf) {
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (cb + k < a.nout) a.yf[p * a.nout + cb + k] = v[k];
        }
      }
      // accumulator ab read out: hand it back to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort && a.err) atomicExch(a.err, 1);
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAllocCols));
}

// 128-channel layers with the operands swapped: M = 128 output channels (the
// weights are the A operand), N = 256 pixels (four image rows; the activations
// are the B operand), K = 9 taps x 64-channel chunks.  An M = N = 128 MMA reads
// 8 KB of operands from shared memory per 64 tensor-core cycles, which is the
// SM's whole shared-memory bandwidth; at N = 256 the same 4 KB of weights
// serve twice the pixels (12 KB per 128 cycles), and the weights are read from
// L2 once per 256 pixels instead of once per 128.  Accumulator [co][pixel] in
// tensor memory (two of 256 columns: all 512); epilogue thread = one output
// channel (lane 32 (w % 4) + l), walking the tile's pixels, so a warp stores
// 32 consecutive channels of a pixel (64 contiguous bytes).
constexpr int kConvN = 256;                       // pixels per tile
constexpr int kConvNStages = 4;                   // 4 x (16 KB + 32 KB) = 192 KB
constexpr int kTileBytesPix = kConvN * 128;       // 256 rows x 128 bytes

__global__ void __launch_bounds__(192, 1)
    conv_tc_n256(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW, ConvTcArgs a) {
  constexpr int kCols = kConvN;
  constexpr int kAllocCols = 2 * kCols;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sW = smem;                                   // [stage] 128 channels x 64 K (16 KB)
  uint8_t* sX = smem + kConvNStages * kTileBytesA;      // [stage] 256 pixels x 64 K (32 KB)
  __shared__ __align__(8) uint64_t full[kConvNStages], empty[kConvNStages], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rows_per_tile = kConvN / a.W;  // 4
  const int tiles_per_img = a.H / rows_per_tile;
  const int ntiles = a.N * tiles_per_img;
  const int chunks = a.cin_pad / 64;
  const int nk = 9 * chunks;
  if (tid == 0) {
    for (int s = 0; s < kConvNStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kAllocCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  volatile int* abort = &abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      int k = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int n = t / tiles_per_img, y0 = (t % tiles_per_img) * rows_per_tile;
        for (int kt = 0; kt < nk; ++kt) {
          const int s = k % kConvNStages;
          if (k >= kConvNStages && !mbar_wait(&empty[s], ((k / kConvNStages) - 1) & 1, abort)) {
            ok = false;
            break;
          }
          const int tap = kt / chunks, c = kt % chunks;
          const int dy = tap / 3 - 1, dx = tap % 3 - 1;
          mbar_expect_tx(&full[s], kTileBytesA + kTileBytesPix);
          tma_load_2d(sW + s * kTileBytesA, &tmW, &full[s], tap * a.cin_pad + c * 64, 0);
          tma_load_4d(sX + s * kTileBytesPix, &tmX, &full[s], c * 64, dx * a.dil, y0 + dy * a.dil, n);
          ++k;
        }
      }
      if (!ok) {
        for (int j = (k > kConvNStages ? k - kConvNStages : 0); j < k; ++j)
          mbar_drain(&full[j % kConvNStages], (j / kConvNStages) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(128, kConvN);
      int k = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
        const int ab = i & 1;
        if (i >= 2 && !mbar_wait(&acc_empty[ab], ((i >> 1) - 1) & 1, abort)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t acc = tmem + (uint32_t)(ab * kCols);
        for (int kt = 0; kt < nk; ++kt, ++k) {
          const int s = k % kConvNStages;
          if (!mbar_wait(&full[s], (k / kConvNStages) & 1, abort)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t w0 = smem_u32(sW + s * kTileBytesA), x0 = smem_u32(sX + s * kTileBytesPix);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
            mma_bf16(acc, desc_sw128(w0 + kk * 32), desc_sw128(x0 + kk * 32), idesc, (kt | kk) != 0);
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&acc_full[ab]);
      }
      mma_commit(&drain);
      mbar_drain(&drain, 0);
    }
  } else {
    // epilogue: thread (warp w, lane l) = output channel co = 32 (w % 4) + l
    const int q = warp & 3;
    const int co = q * 32 + lane;
    const bool live = co < a.nout;
    const float bco = (a.mode != 2 && live) ? a.bias[co] : 0.0f;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int ab = i & 1;
      bool ok = mbar_wait(&acc_full[ab], (i >> 1) & 1, abort);
      ok = __all_sync(0xffffffffu, ok ? 1 : 0) && !*abort;  // warp-uniform before the aligned TMEM loads
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int n = t / tiles_per_img, y0 = (t % tiles_per_img) * rows_per_tile;
      const int64_t p0 = ((int64_t)n * a.H + y0) * a.W;  // the tile's pixels are p0 .. p0 + 255
#pragma unroll 1
      for (int cb = 0; cb < kConvN; cb += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * kCols + cb), v);
        // the 16 loads of the previous activation first: y may alias ref as far
        // as the compiler knows, so a load placed after a store would wait for it
        float rv[16];
        if (a.mode == 2) {
#pragma unroll
          for (int k = 0; k < 16; ++k)
            rv[k] = live ? __bfloat162float(a.ref[(p0 + cb + k) * a.ldref + co]) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int64_t p = p0 + cb + k;
          float x = v[k];
          if (a.mode == 2) {
            x *= (rv[k] < 0.0f) ? kLeakTc : 1.0f;
          } else {
            x += bco;
            if (a.mode == 1 && x < 0.0f) x *= kLeakTc;
          }
          if (!live) x = 0.0f;
          if (a.y && co < a.ldy) a.y[p * a.ldy + co] = __float2bfloat16_rn(x);
          if (a.yf && live) a.yf[p * a.nout + co] = x;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort && a.err) atomicExch(a.err, 1);
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAllocCols));
}

struct WgradTcArgs {
  int N, H, W;
  int dil;
  int rows_per_split;  // image rows (n, y) per CTA
  int cin_pad;         // N of the GEMM (64 or 128)
  float* part;         // [splits][9][128][cin_pad]
  int* err;
};

// Weight gradient of one tap over a range of image rows: D[co][ci] (128 x BN).
template <int BN>
__global__ void __launch_bounds__(128, 1)
    wgrad_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, WgradTcArgs a) {
  constexpr int kTileBytesB = BN * 128;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint8_t* sA = smem;
  uint8_t* sB = smem + kStages * kTileBytesA;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tap = blockIdx.x, split = blockIdx.y;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int total_rows = a.N * a.H;
  const int r0 = split * a.rows_per_split;
  const int nk = max(0, min(a.rows_per_split, total_rows - r0));
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  volatile int* abort = &abort_flag;
  if (tid == 0) {
    for (int k = 0; k < nk; ++k) {
      const int s = k % kStages;
      if (k >= kStages && !mbar_wait(&empty[s], ((k / kStages) - 1) & 1, abort)) break;
      const int r = r0 + k, n = r / a.H, y = r % a.H;
      mbar_expect_tx(&full[s], kTileBytesA + kTileBytesB);
      tma_load_4d(sA + s * kTileBytesA, &tmA, &full[s], 0, y, n, 0);               // dyT rows (co), 64 x
      tma_load_5d(sB + s * kTileBytesB, &tmB, &full[s], 0, y + dy * a.dil, n, 0, dx + 1);  // xT copy (ci), 64 x
    }
  } else if (tid == 32) {
    constexpr uint32_t idesc = idesc_bf16(128, BN);
    bool ok = true;
    for (int k = 0; k < nk && ok; ++k) {
      const int s = k % kStages;
      ok = mbar_wait(&full[s], (k / kStages) & 1, abort);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA + s * kTileBytesA), b0 = smem_u32(sB + s * kTileBytesB);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma_bf16(tmem, desc_sw128(a0 + kk * 32), desc_sw128(b0 + kk * 32), idesc, (k | kk) != 0);
      mma_commit(&empty[s]);
    }
    if (ok) mma_commit(&done);
  }
  bool ok = true;
  if (nk > 0) ok = mbar_wait(&done, 0, abort);
  ok = __all_sync(0xffffffffu, ok ? 1 : 0) && !*abort;
  asm volatile("tcgen05.fence::after_thread_sync;");
  const int co = warp * 32 + lane;
  float* dst = a.part + (((int64_t)split * 9 + tap) * 128 + co) * a.cin_pad;
  if (ok) {
#pragma unroll
    for (int cb = 0; cb < BN; cb += 16) {
      float v[16];
      if (nk > 0) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
      } else {
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.0f;
      }
#pragma unroll
      for (int k = 0; k < 16; k += 4)
        *reinterpret_cast<float4*>(dst + cb + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    }
  } else if (tid == 0 && a.err) {
    atomicExch(a.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// ---- layout helpers ----

// xT[d][c][n][y][x] = x[n][y][x + (d - 1) dil][c] (0 outside the image), d = 0, 1, 2.
__global__ void k_nhwc_to_shifted_cnhw(const __nv_bfloat16* __restrict__ x, int N, int H, int W, int C, int dil,
                                       __nv_bfloat16* __restrict__ xT) {
  __shared__ __nv_bfloat16 tile[64][65];  // [x][c]
  const int c0 = blockIdx.x * 64, row = blockIdx.y;  // row = n H + y
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 256 threads: 64 x 4
  const int64_t P = (int64_t)N * H * W;
  for (int xx = ty; xx < W; xx += 4) tile[xx][tx] = (c0 + tx < C) ? x[((int64_t)row * W + xx) * C + c0 + tx]
                                                                  : __float2bfloat16(0.0f);
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    const int sh = (d - 1) * dil;
    for (int cc = ty; cc < 64; cc += 4) {
      if (c0 + cc >= C) continue;
      const int xs = tx + sh;
      const __nv_bfloat16 v = (tx < W && xs >= 0 && xs < W) ? tile[xs][cc] : __float2bfloat16(0.0f);
      if (tx < W) xT[(((int64_t)d * C + c0 + cc) * P) + (int64_t)row * W + tx] = v;
    }
  }
}

// yT[c][p] = y[p][c] for c < C (rows of yT beyond C are not written)
__global__ void k_nhwc_to_cnhw(const __nv_bfloat16* __restrict__ y, int64_t P, int C, __nv_bfloat16* __restrict__ yT) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t p = p0 + r;
    tile[r][tx] = (p < P && c0 + tx < C) ? y[p * C + c0 + tx] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t p = p0 + tx;
    if (c < C && p < P) yT[(int64_t)c * P + p] = tile[tx][r];
  }
}

// dW[co][ci][3][3] (FP32, the layer's shape) = sum over splits of part[s][tap][co][ci]
__global__ void k_wgrad_reduce(const float* __restrict__ part, int splits, int cin_pad, int Cout, int Cin,
                               float* __restrict__ dw) {
  const int64_t n = (int64_t)Cout * Cin * 9;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int tap = (int)(t % 9);
    const int ci = (int)((t / 9) % Cin);
    const int co = (int)(t / (9 * (int64_t)Cin));
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(((int64_t)k * 9 + tap) * 128 + co) * cin_pad + ci];
    dw[t] = s;
  }
}

// db[c] = sum_p dy[p][c] (FP32 accumulation of the BF16 gradient), one block per channel
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dy, int64_t P, int ld, int C, float* __restrict__ db) {
  const int c = blockIdx.x;
  float s = 0.0f;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(dy[p * ld + c]);
  __shared__ float red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && c < C) db[c] = red[0];
}

// FP32 weights [Cout][Cin][3][3] -> wf [cout_pad][9][cin_pad] and
// wb [cin_rows][9][cout_kpad] with wb[ci][t][co] = w[co][ci][8 - t] (BF16, zero padding)
__global__ void k_weights_bf16(const float* __restrict__ w, int Cout, int Cin, int cout_pad, int cin_pad,
                               int cin_rows, int cout_kpad, __nv_bfloat16* __restrict__ wf,
                               __nv_bfloat16* __restrict__ wb) {
  const int64_t nf = (int64_t)cout_pad * 9 * cin_pad, nb = (int64_t)cin_rows * 9 * cout_kpad;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nf + nb; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nf) {
      const int ci = (int)(t % cin_pad), tap = (int)((t / cin_pad) % 9), co = (int)(t / (9 * (int64_t)cin_pad));
      const float v = (co < Cout && ci < Cin) ? w[((int64_t)co * Cin + ci) * 9 + tap] : 0.0f;
      wf[t] = __float2bfloat16(v);
    } else if (wb) {
      const int64_t u = t - nf;
      const int co = (int)(u % cout_kpad), tap = (int)((u / cout_kpad) % 9), ci = (int)(u / (9 * (int64_t)cout_kpad));
      const float v = (co < Cout && ci < Cin) ? w[((int64_t)co * Cin + ci) * 9 + (8 - tap)] : 0.0f;
      wb[u] = __float2bfloat16(v);
    }
  }
}

// ---- host side: tensor maps through the driver entry point ----

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// BF16 tensor of `rank` dims (dims[0] innermost, contiguous), box `box`, 128-byte swizzle, zero fill.
bool make_map(CUtensorMap* m, const void* base, int rank, const uint64_t* dims, const uint32_t* box) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)base & 15)) return false;
  cuuint64_t gd[5], gs[4];
  cuuint32_t bx[5], es[5];
  uint64_t stride = 2;
  for (int k = 0; k < rank; ++k) {
    gd[k] = dims[k];
    bx[k] = box[k];
    es[k] = 1;
    if (k > 0) gs[k - 1] = stride;
    stride *= dims[k];
  }
  for (int k = 0; k + 1 < rank; ++k)
    if (gs[k] % 16) return false;
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), gd, gs, bx, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t smem_bytes(int bn) { return 1024 + (size_t)kStages * (kTileBytesA + bn * 128); }
size_t conv_smem_bytes(int bn) { return 1024 + (size_t)kConvStages * (kTileBytesA + bn * 128); }

}  // namespace

// x [N][H][W][ldx] (channels beyond ldx, up to cin_pad, read as zero),
// wk [bn][9][cin_pad] (rows >= nout zero), outputs as ConvTcArgs.
cudaError_t launch_conv_tc(const void* x, const void* wk, int bn, const ConvTcLaunch& L, cudaStream_t s) {
  if (L.W != 64 || L.H % 2 || L.cin_pad % 64 || L.ldx % 8 || L.ldx < 1 || L.ldx > L.cin_pad ||
      (bn != 16 && bn != 64 && bn != 128) || L.nout > bn || L.nout < 1 || (L.y && (L.ldy % 16 || L.ldy < L.nout)) ||
      (L.mode == 2 && (!L.ref || L.ldref < L.nout)) || (L.mode != 2 && !L.bias))
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  // 128-channel layers on images of a multiple of 4 rows: the swapped-operand
  // kernel (256-pixel tiles); others: 128-pixel tiles
  const bool n256 = bn == 128 && L.H % 4 == 0;
  const uint64_t da[4] = {(uint64_t)L.ldx, (uint64_t)L.W, (uint64_t)L.H, (uint64_t)L.N};
  const uint32_t ba[4] = {64, (uint32_t)L.W, n256 ? 4u : 2u, 1};
  const uint64_t db[2] = {(uint64_t)9 * L.cin_pad, (uint64_t)bn};
  const uint32_t bb[2] = {64, (uint32_t)bn};
  if (!make_map(&ma, x, 4, da, ba) || !make_map(&mb, wk, 2, db, bb)) return cudaErrorInvalidValue;
  ConvTcArgs a;
  a.N = L.N;
  a.H = L.H;
  a.W = L.W;
  a.cin_pad = L.cin_pad;
  a.nout = L.nout;
  a.ldy = L.ldy;
  a.dil = L.dil;
  a.mode = L.mode;
  a.bias = L.bias;
  a.ref = reinterpret_cast<const __nv_bfloat16*>(L.ref);
  a.ldref = L.ldref;
  a.y = reinterpret_cast<__nv_bfloat16*>(L.y);
  a.yf = L.yf;
  a.err = L.err;
  const size_t smem = conv_smem_bytes(bn);
  // persistent: one CTA per SM (the stage ring takes most of its shared memory)
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int64_t ntiles = (int64_t)L.N * L.H / (n256 ? 4 : 2);
  const dim3 grid((unsigned)std::min<int64_t>(ntiles, std::max(1, sms)));
  count_launches(1);
  if (n256) {
    const size_t sm256 = 1024 + (size_t)kConvNStages * (kTileBytesA + kTileBytesPix);
    if ((e = smem_at_least(conv_tc_n256, sm256))) return e;
    conv_tc_n256<<<grid, 192, sm256, s>>>(ma, mb, a);
    return cudaGetLastError();
  }
  switch (bn) {
    case 16:
      if ((e = smem_at_least(conv_tc<16>, smem)))
        return e;
      conv_tc<16><<<grid, 192, smem, s>>>(ma, mb, a);
      break;
    case 64:
      if ((e = smem_at_least(conv_tc<64>, smem)))
        return e;
      conv_tc<64><<<grid, 192, smem, s>>>(ma, mb, a);
      break;
    default:
      if ((e = smem_at_least(conv_tc<128>, smem)))
        return e;
      conv_tc<128><<<grid, 192, smem, s>>>(ma, mb, a);
  }
  return cudaGetLastError();
}

// dyT [cout_rows][N][H][W] (cout_rows >= 1; rows beyond are read as zero up to 128),
// xT [3][cin_pad][N][H][W]; dw [Cout][Cin][3][3] FP32; part scratch [splits][9][128][cin_pad].
cudaError_t launch_wgrad_tc(const void* dyT, int cout_rows, const void* xT, int cin_pad, int N, int H, int W, int dil,
                            int Cout, int Cin, float* part, int splits, float* dw, int* err, cudaStream_t s) {
  if (W != 64 || (cin_pad != 64 && cin_pad != 128) || Cout > 128 || Cout > cout_rows || Cin > cin_pad ||
      splits < 1 || splits > N * H)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  const uint64_t da[4] = {(uint64_t)W, (uint64_t)H, (uint64_t)N, (uint64_t)cout_rows};
  const uint32_t ba[4] = {64, 1, 1, 128};
  const uint64_t db[5] = {(uint64_t)W, (uint64_t)H, (uint64_t)N, (uint64_t)cin_pad, 3};
  const uint32_t bb[5] = {64, 1, 1, (uint32_t)cin_pad, 1};
  if (!make_map(&ma, dyT, 4, da, ba) || !make_map(&mb, xT, 5, db, bb)) return cudaErrorInvalidValue;
  WgradTcArgs a;
  a.N = N;
  a.H = H;
  a.W = W;
  a.dil = dil;
  a.rows_per_split = (N * H + splits - 1) / splits;
  a.cin_pad = cin_pad;
  a.part = part;
  a.err = err;
  const size_t smem = smem_bytes(cin_pad);
  const dim3 grid(9, splits);
  cudaError_t e;
  count_launches(2);
  if (cin_pad == 64) {
    if ((e = smem_at_least(wgrad_tc<64>, smem))) return e;
    wgrad_tc<64><<<grid, 128, smem, s>>>(ma, mb, a);
  } else {
    if ((e = smem_at_least(wgrad_tc<128>, smem))) return e;
    wgrad_tc<128><<<grid, 128, smem, s>>>(ma, mb, a);
  }
  if ((e = cudaGetLastError())) return e;
  k_wgrad_reduce<<<(int)std::min<int64_t>(1024, ((int64_t)Cout * Cin * 9 + 255) / 256), 256, 0, s>>>(
      part, splits, cin_pad, Cout, Cin, dw);
  return cudaGetLastError();
}

cudaError_t launch_nhwc_to_shifted_cnhw(const void* x, int N, int H, int W, int C, int dil, void* xT,
                                        cudaStream_t s) {
  if (W > 64) return cudaErrorInvalidValue;
  count_launches(1);
  k_nhwc_to_shifted_cnhw<<<dim3((C + 63) / 64, N * H), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(x), N,
                                                                      H, W, C, dil, reinterpret_cast<__nv_bfloat16*>(xT));
  return cudaGetLastError();
}

cudaError_t launch_nhwc_to_cnhw(const void* y, int64_t P, int C, void* yT, cudaStream_t s) {
  count_launches(1);
  k_nhwc_to_cnhw<<<dim3((unsigned)((P + 31) / 32), (C + 31) / 32), 256, 0, s>>>(
      reinterpret_cast<const __nv_bfloat16*>(y), P, C, reinterpret_cast<__nv_bfloat16*>(yT));
  return cudaGetLastError();
}

cudaError_t launch_bias_grad(const void* dy, int64_t P, int ld, int C, float* db, cudaStream_t s) {
  count_launches(1);
  k_bias_grad<<<C, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(dy), P, ld, C, db);
  return cudaGetLastError();
}

cudaError_t launch_weights_bf16(const float* w, int Cout, int Cin, int cout_pad, int cin_pad, int cin_rows,
                                int cout_kpad, void* wf, void* wb, cudaStream_t s) {
  count_launches(1);
  const int64_t n = (int64_t)cout_pad * 9 * cin_pad + (wb ? (int64_t)cin_rows * 9 * cout_kpad : 0);
  k_weights_bf16<<<(int)std::min<int64_t>(2048, (n + 255) / 256), 256, 0, s>>>(
      w, Cout, Cin, cout_pad, cin_pad, cin_rows, cout_kpad, reinterpret_cast<__nv_bfloat16*>(wf),
      reinterpret_cast<__nv_bfloat16*>(wb));
  return cudaGetLastError();
}

int conv_tc_available() { return encode_fn() != nullptr; }

namespace {

// out[p][c] (BF16, 64 channels): (max(log p, -30), max(log q, -30), log eps, log lambda) / 4, then zeros
__global__ void k_features_nhwc(const float* __restrict__ P, const float* __restrict__ Q,
                                const float* __restrict__ le, const float* __restrict__ ll, int64_t HW, int64_t total,
                                __nv_bfloat16* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = t / HW;
    const float p = P[t], q = Q[t];
    const float f0 = 0.25f * fmaxf(p > 0.0f ? logf(p) : -INFINITY, -30.0f);
    const float f1 = 0.25f * fmaxf(q > 0.0f ? logf(q) : -INFINITY, -30.0f);
    __align__(16) __nv_bfloat162 h[32];
    h[0] = __floats2bfloat162_rn(f0, f1);
    h[1] = __floats2bfloat162_rn(0.25f * le[n], 0.25f * ll[n]);
#pragma unroll
    for (int k = 2; k < 32; ++k) h[k] = __floats2bfloat162_rn(0.0f, 0.0f);
    uint4* dst = reinterpret_cast<uint4*>(out + t * 64);
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[k] = reinterpret_cast<const uint4*>(h)[k];
  }
}

// grad[p][c] (BF16, stride 16) = 2 (pred[p][c] - t_c[p] s[n]) / (2 P) for c < 2, 0 beyond;
// *loss += mean squared difference.  t_0 = U, t_1 = V ([N][HW]), s = per-instance scale.
__global__ void k_mse_nhwc(const float* __restrict__ pred, const float* __restrict__ U, const float* __restrict__ V,
                           const float* __restrict__ scale, int64_t HW, int64_t P, __nv_bfloat16* __restrict__ grad,
                           double* loss) {
  float acc = 0.0f;
  const float inv = 1.0f / (float)(2 * P);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float s = scale[p / HW];
    const float d0 = pred[2 * p] - U[p] * s, d1 = pred[2 * p + 1] - V[p] * s;
    acc += d0 * d0 + d1 * d1;
    __align__(16) __nv_bfloat162 h[8];
    h[0] = __floats2bfloat162_rn(2.0f * d0 * inv, 2.0f * d1 * inv);
#pragma unroll
    for (int k = 1; k < 8; ++k) h[k] = __floats2bfloat162_rn(0.0f, 0.0f);
    uint4* dst = reinterpret_cast<uint4*>(grad + p * 16);
    dst[0] = reinterpret_cast<const uint4*>(h)[0];
    dst[1] = reinterpret_cast<const uint4*>(h)[1];
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, (double)red[0] * (double)inv);
}

// U0[n][hw] = pred[p][0] s[n], V0[n][hw] = pred[p][1] s[n]
__global__ void k_pred_to_potentials(const float* __restrict__ pred, const float* __restrict__ scale, int64_t HW,
                                     int64_t P, float* __restrict__ U0, float* __restrict__ V0) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const float s = scale[p / HW];
    U0[p] = pred[2 * p] * s;
    V0[p] = pred[2 * p + 1] * s;
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (n + 255) / 256)); }

uot_status ck(cudaError_t e) {
  if (e == cudaSuccess) return UOT_OK;
  return e == cudaErrorInvalidValue ? UOT_EINVAL : UOT_ECUDA;
}

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

uot_status uot_conv_tc_forward(const void* x, int ldx, const void* wk, int bn, int N, int H, int W, int cin_pad,
                               int nout, int dil, int mode, const float* bias, const void* ref, int ldref, void* y,
                               int ldy, float* yf, int* err, void* stream) {
  if (!x || !wk || N < 1 || H < 2 || dil < 1 || mode < 0 || mode > 2 || (!y && !yf)) return UOT_EINVAL;
  if (!conv_tc_available()) return UOT_EUNSUPPORTED;
  ConvTcLaunch L;
  L.N = N;
  L.H = H;
  L.W = W;
  L.ldx = ldx;
  L.cin_pad = cin_pad;
  L.nout = nout;
  L.ldy = ldy;
  L.dil = dil;
  L.mode = mode;
  L.bias = bias;
  L.ref = ref;
  L.ldref = ldref;
  L.y = y;
  L.yf = yf;
  L.err = err;
  return ck(launch_conv_tc(x, wk, bn, L, (cudaStream_t)stream));
}

uot_status uot_conv_tc_wgrad(const void* dyT, int cout_rows, const void* xT, int cin_pad, int N, int H, int W,
                             int dil, int Cout, int Cin, float* part, int splits, float* dw, int* err, void* stream) {
  if (!dyT || !xT || !part || !dw || N < 1 || H < 1 || dil < 1 || Cout < 1 || Cin < 1) return UOT_EINVAL;
  if (!conv_tc_available()) return UOT_EUNSUPPORTED;
  return ck(launch_wgrad_tc(dyT, cout_rows, xT, cin_pad, N, H, W, dil, Cout, Cin, part, splits, dw, err,
                            (cudaStream_t)stream));
}

uot_status uot_nhwc_shift_transpose(const void* x, int N, int H, int W, int C, int dil, void* xT, void* stream) {
  if (!x || !xT || N < 1 || H < 1 || W < 1 || C < 1 || dil < 1) return UOT_EINVAL;
  return ck(launch_nhwc_to_shifted_cnhw(x, N, H, W, C, dil, xT, (cudaStream_t)stream));
}

uot_status uot_nhwc_transpose(const void* y, long long P, int C, void* yT, void* stream) {
  if (!y || !yT || P < 1 || C < 1) return UOT_EINVAL;
  return ck(launch_nhwc_to_cnhw(y, P, C, yT, (cudaStream_t)stream));
}

uot_status uot_bias_grad_bf16(const void* dy, long long P, int ld, int C, float* db, void* stream) {
  if (!dy || !db || P < 1 || C < 1 || ld < C) return UOT_EINVAL;
  return ck(launch_bias_grad(dy, P, ld, C, db, (cudaStream_t)stream));
}

uot_status uot_conv_weights_bf16(const float* w, int Cout, int Cin, int cout_pad, int cin_pad, int cin_rows,
                                 int cout_kpad, void* wf, void* wb, void* stream) {
  if (!w || !wf || Cout < 1 || Cin < 1 || cout_pad < Cout || cin_pad < Cin || (wb && (cin_rows < Cin || cout_kpad < Cout)))
    return UOT_EINVAL;
  return ck(launch_weights_bf16(w, Cout, Cin, cout_pad, cin_pad, cin_rows, cout_kpad, wf, wb, (cudaStream_t)stream));
}

uot_status uot_warmstart_features_nhwc(const float* p, const float* q, const float* log_eps, const float* log_lam,
                                       void* out, int N, int H, int W, void* stream) {
  if (!p || !q || !log_eps || !log_lam || !out || N < 1 || H < 1 || W < 1) return UOT_EINVAL;
  const int64_t total = (int64_t)N * H * W;
  count_launches(1);
  k_features_nhwc<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(p, q, log_eps, log_lam, (int64_t)H * W, total,
                                                                     reinterpret_cast<__nv_bfloat16*>(out));
  return ck(cudaGetLastError());
}

uot_status uot_mse_grad_nhwc(const float* pred, const float* U, const float* V, const float* scale, int N, int HW,
                             void* grad, double* loss_dev, void* stream) {
  if (!pred || !U || !V || !scale || !grad || !loss_dev || N < 1 || HW < 1) return UOT_EINVAL;
  const int64_t P = (int64_t)N * HW;
  count_launches(1);
  k_mse_nhwc<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>(pred, U, V, scale, HW, P,
                                                            reinterpret_cast<__nv_bfloat16*>(grad), loss_dev);
  return ck(cudaGetLastError());
}

uot_status uot_pred_to_potentials(const float* pred, const float* scale, int N, int HW, float* U0, float* V0,
                                  void* stream) {
  if (!pred || !scale || !U0 || !V0 || N < 1 || HW < 1) return UOT_EINVAL;
  const int64_t P = (int64_t)N * HW;
  count_launches(1);
  k_pred_to_potentials<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>(pred, scale, HW, P, U0, V0);
  return ck(cudaGetLastError());
}

}  // extern "C"
