// BF16 GEMM on the 5th-generation tensor cores (tcgen05) for the warm-start
// network:  C[M][N] = A[M][K] * B[N][K]^T  (+ bias[N], optional ReLU),
// A and B K-major BF16, FP32 accumulation in tensor memory (TMEM).
//
// Two kernels share the tensor-core step:
//
// gemm_bf16_tn_tma_kernel (default): persistent, one CTA of 320 threads per
// SM walking 128 x BN tiles of C (BN = 64, 128 or 256, chosen per shape),
// roles split by warp:
//   * one thread of warp 0 is the producer: for each K step of 64 it arms
//     a stage's "full" mbarrier with the byte count and issues two TMA tile
//     loads (cp.async.bulk.tensor, 128-byte swizzle, zero fill outside M, N,
//     K) of the A (128 x 64) and B (BN x 64) tiles into a ring of stages
//     that runs on across tiles; it refills a stage once its "empty"
//     mbarrier reports that the MMAs reading it have completed;
//   * one thread of warp 1 issues the MMAs: per K step it waits for the
//     stage's "full" barrier, issues four tcgen05.mma (K = 16 each,
//     128-byte-swizzle K-major descriptors) and commits them to the stage's
//     "empty" barrier.  Tiles alternate between two TMEM accumulators
//     (2 BN columns), so the MMAs of tile i + 1 run while tile i is being
//     stored; a tile's last commit goes to its accumulator's "full" barrier;
//   * warps 2-9 are the epilogue: warp w reads TMEM lanes 32 (w % 4)..+31
//     (rows of the tile), the two warps of a lane quadrant taking alternate
//     32-column blocks; each 32 x 32 block is transposed through a swizzled
//     shared-memory buffer so that every 16-byte store writes consecutive
//     columns of a row (whole row segments per instruction), with bias,
//     ReLU, FP32 and/or BF16 output; then the accumulator is released.
// The operands are viewed as 3-D tensors {K slice, slice, rows} so the
// split-K form (slice z covers K columns [z Kslice, (z+1) Kslice)) reads
// zeros past the end of its own slice.
//
// The same kernel also runs 3x3 convolutions as an implicit GEMM
// (launch_conv3x3_bf16): the A tiles come straight from the NHWC activations
// through an im2col tensor map (TMA im2col mode, one load per 8-channel chunk
// of K, filter offsets per load), so no im2col matrix is written or read.
//
// gemm_bf16_tn_kernel (fallback when no tensor map can be made, or
// CMG_GEMM_TMA=0): a 128 x 64 tile, every thread copying with cp.async into
// the no-swizzle core-matrix layout, kStages - 1 K steps in flight, one
// thread issuing the MMAs after a CTA barrier.
//
// Its epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile)
// with tcgen05.ld, adds bias, applies ReLU, and stores FP32 and/or BF16 with
// 16-byte stores where alignment allows.
//
// Every wait has an iteration limit; on expiry the kernel records an error
// code, stops issuing work, waits (again bounded) for the copies it has in
// flight, frees its TMEM columns and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <cstdlib>
#include <mutex>

#include "cmg_internal.h"

namespace cmg {
namespace nn {

constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kThreads = 128;
constexpr int kStages = 4;
constexpr uint32_t kTmemCols = 64;                 // FP32 accumulator columns (= kBN)
constexpr long kSpinLimit = 1L << 22;              // mbarrier polls before giving up
constexpr int kSmemBytes = kStages * (kBM + kBN) * kBK * 2;   // 96 KiB of operand tiles

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor: start address, leading (K
// direction) and stride (M/N direction) byte offsets, descriptor version 1,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// K-major tile written by TMA with the 64-byte swizzle: rows of 64 bytes
// (32 BF16 of K), 8-row groups 512 bytes apart, layout type 4 (64-byte
// swizzle); the tile base is 512-byte aligned, so a K step of 16 inside the
// 64-byte row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// The same descriptor for a K-major tile written by TMA with the 128-byte
// swizzle: rows of 128 bytes (64 BF16 of K), 8-row groups 1024 bytes apart
// (stride byte offset), layout type 2 (128-byte swizzle) in bits 61-63; the
// leading byte offset is unused for this layout.  The tile base is 1024-byte
// aligned, so a K step of 16 inside the 128-byte row advances the start
// address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B BF16, both
// K-major, N and M of the MMA.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Wait for phase `parity` of the mbarrier; false if the poll limit expires
// or, when `abort` is given, once another thread has set it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* abort = nullptr,
                                          long long limit = kSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
  }
  return false;
}

// Arrive on the barrier and add `bytes` to the transaction count its phase
// waits for (the TMA loads of one stage).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// TMA load of one box of a 3-D tensor map at coordinates (c0, c1, c2),
// completing on `bar` with the box's byte count.  c0 (the K coordinate) is
// always a multiple of 64 elements, which keeps the copy 16-byte aligned.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// TMA load in im2col mode of an NHWC tensor map: from the pixel at
// coordinates (w, h, n) of the map's bounding box on, pixelsPerColumn pixels
// in W, H, N order, each the box's channels from channel c at input pixel
// (w + ow, h + oh); outside the tensor reads as zero.  c is a multiple of 8
// BF16 (16-byte aligned).
__device__ __forceinline__ void tma_load_im2col(void* dst, const CUtensorMap* map, int c, int w, int h, int n,
                                                uint16_t ow, uint16_t oh, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.im2col.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6], {%7, %8};" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(w), "r"(h), "r"(n), "r"(smem_u32(bar)), "h"(ow), "h"(oh)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Asynchronous copy of a rows x 64 BF16 tile (row stride ld elements) into
// the core-matrix layout; rows beyond `valid` and columns beyond K are
// zero-filled (K % 8 == 0).  The source of a zero-filled chunk is the
// (valid) tile base, read with size 0.
__device__ __forceinline__ void load_tile_async(__nv_bfloat16* dst, const __nv_bfloat16* src, int rows, long ld,
                                                int valid, int k0, int K) {
  for (int c = threadIdx.x; c < rows * 8; c += kThreads) {
    const int row = c >> 3, k8 = c & 7;
    const bool ok = row < valid && k0 + k8 * 8 < K;
    const __nv_bfloat16* g = ok ? src + (size_t)row * ld + k0 + k8 * 8 : src;
    const int core = (row >> 3) * 8 + k8;            // core matrices: 8 per 8-row group along K
    const uint32_t d = smem_u32(reinterpret_cast<char*>(dst) + core * 128 + (row & 7) * 16);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(ok ? 16 : 0) : "memory");
  }
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Epilogue of one warp: rows m0 + 32 warp + lane of C, `chunks` blocks of
// 32 accumulator columns (TMEM columns 32c.., C columns n0 + 32c..), bias,
// ReLU, FP32 and/or BF16 stores.  Called by all 32 lanes together.
__device__ __forceinline__ void store_tile(uint32_t tmem, int chunks, int warp, int lane, int m0, int n0, int M, int N,
                                           const float* __restrict__ bias, int relu, float* __restrict__ C32,
                                           __nv_bfloat16* __restrict__ C16, int ldc, int vec16, int vec32) {
  const int row = m0 + warp * 32 + lane;
#pragma unroll 1
  for (int ch = 0; ch < chunks; ++ch) {
    if (n0 + ch * 32 >= N) break;   // uniform over the warp
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (row < M) {
      const int c0 = n0 + ch * 32;
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        v[j] = __uint_as_float(r[j]);
        if (bias && c0 + j < N) v[j] += bias[c0 + j];
        if (relu) v[j] = fmaxf(v[j], 0.f);
      }
      // 16-byte stores of consecutive columns of this thread's row (a
      // scalar store per element only at a ragged right edge or when the
      // row stride does not keep 16-byte alignment)
#pragma unroll
      for (int q = 0; q < 32; q += 8) {
        const int col = c0 + q;
        if (C16) {
          __nv_bfloat16* dst = C16 + (size_t)row * ldc + col;
          if (vec16 && col + 8 <= N) {
            uint4 pk;
            uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[q + 2 * t], v[q + 2 * t + 1]);
              w[t] = *reinterpret_cast<const uint32_t*>(&b2);
            }
            *reinterpret_cast<uint4*>(dst) = pk;
          } else {
            for (int t = 0; t < 8; ++t)
              if (col + t < N) dst[t] = __float2bfloat16_rn(v[q + t]);
          }
        }
        if (C32) {
          float* dst = C32 + (size_t)row * ldc + col;
#pragma unroll
          for (int t = 0; t < 8; t += 4) {
            if (vec32 && col + t + 4 <= N) {
              *reinterpret_cast<float4*>(dst + t) = make_float4(v[q + t], v[q + t + 1], v[q + t + 2], v[q + t + 3]);
            } else {
              for (int u = 0; u < 4; ++u)
                if (col + t + u < N) dst[t + u] = v[q + t + u];
            }
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) gemm_bf16_tn_kernel(const __nv_bfloat16* __restrict__ A, long lda,
                                                                const __nv_bfloat16* __restrict__ B, long ldb, int M,
                                                                int N, int K, const float* __restrict__ bias, int relu,
                                                                float* __restrict__ C32, __nv_bfloat16* __restrict__ C16,
                                                                int ldc, int* __restrict__ status, int vec16, int vec32) {
  extern __shared__ __align__(1024) unsigned char dyn_smem[];   // kSmemBytes: A and B tiles of both stages
  __nv_bfloat16* sA[kStages];
  __nv_bfloat16* sB[kStages];
  for (int s = 0; s < kStages; ++s) {
    sA[s] = reinterpret_cast<__nv_bfloat16*>(dyn_smem + s * (kBM + kBN) * kBK * 2);
    sB[s] = sA[s] + kBM * kBK;
  }
  __shared__ __align__(8) uint64_t bar[kStages];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  // split-K: slice z covers K columns [z*K, (z+1)*K) of the full operands and
  // writes its own FP32 partial matrix
  A += (size_t)blockIdx.z * K;
  B += (size_t)blockIdx.z * K;
  if (C32) C32 += (size_t)blockIdx.z * M * ldc;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc(kBM, kBN);
  const int ksteps = (K + kBK - 1) / kBK;
  const __nv_bfloat16* Ablk = A + (size_t)m0 * lda;
  const __nv_bfloat16* Bblk = B + (size_t)n0 * ldb;
  uint32_t phase[kStages] = {0, 0, 0, 0};
  int commits[kStages] = {0, 0, 0, 0};   // MMA commits made on each stage's barrier

  // prologue: K steps 0 .. kStages-2 in flight (one copy group each, empty past the end)
  for (int p = 0; p < kStages - 1; ++p) {
    if (p < ksteps) {
      load_tile_async(sA[p], Ablk, kBM, lda, M - m0, p * kBK, K);
      load_tile_async(sB[p], Bblk, kBN, ldb, N - n0, p * kBK, K);
    }
    cp_commit();
  }
  for (int ks = 0; ks < ksteps; ++ks) {
    const int s = ks % kStages;
    cp_wait<kStages - 2>();                              // this thread's copies of step ks have landed
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
    __syncthreads();                                     // ... everyone's
    if (failed) break;
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA[s]), b0 = smem_u32(sB[s]);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        // K = 16 covers two core matrices along K: advance 2 * 128 bytes per step
        const uint64_t ad = smem_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = smem_desc(b0 + kk * 256, 128, 1024);
        mma_bf16(tmem, ad, bd, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bar[s]);
    }
    ++commits[s];
    // refill the stage read by step ks-1 with step ks+kStages-1, once those MMAs are done
    const int nxt = ks + kStages - 1;
    if (nxt < ksteps) {
      const int sn = nxt % kStages;
      if (commits[sn] > 0) {
        if (!mbar_wait(&bar[sn], phase[sn])) {
          if (threadIdx.x == 0) failed = 1;
        }
        phase[sn] ^= 1;
      }
      load_tile_async(sA[sn], Ablk, kBM, lda, M - m0, nxt * kBK, K);
      load_tile_async(sB[sn], Bblk, kBN, ldb, N - n0, nxt * kBK, K);
    }
    cp_commit();
  }
  cp_wait<0>();
  // Each stage has exactly one commit not yet waited for (its last one); the
  // i-th commit on a barrier completes phase i, so the last of `uses`
  // commits has parity (uses - 1) & 1.
  if (!failed) {
    for (int s = 0; s < kStages; ++s) {
      const int uses = (ksteps - s + kStages - 1) / kStages;   // commits made on stage s
      if (uses > 0 && !mbar_wait(&bar[s], (uint32_t)((uses - 1) & 1))) failed = 1;
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();

  if (!failed) store_tile(tmem, kBN / 32, warp, lane, m0, n0, M, N, bias, relu, C32, C16, ldc, vec16, vec32);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (failed && threadIdx.x == 0) atomicExch(status, 1);
}


// ---- TMA-fed, warp-specialised, persistent kernel ---------------------------

constexpr int kEpiWarps = 8;                            // two per TMEM lane quadrant
constexpr int kTmaThreads = 64 + 32 * kEpiWarps;        // warp 0 producer, warp 1 MMA, warps 2-9 epilogue

template <int BN, int S>
struct TmaTile {
  static constexpr uint32_t kABytes = kBM * kBK * 2;              // 16 KiB
  static constexpr uint32_t kBBytes = BN * kBK * 2;
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;      // multiple of 1024
  static constexpr uint32_t kEpiBytes = kEpiWarps * 32 * 32 * 4;   // one 32 x 32 FP32 block per warp
  static constexpr int kSmem = S * kStageBytes + kEpiBytes + 1024;   // + slack to align the ring to 1024 bytes
  static constexpr uint32_t kTmemCols = 2 * BN;                   // two accumulators
  static_assert(BN == 64 || BN == 128 || BN == 256, "MMA N and TMEM allocation");
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

// Tile t of the persistent walk: N tile fastest, then M tile, then split-K
// slice.  CTAs running at the same time then share the A block of their
// rows (read once from memory) and together write whole rows of C.
struct TileIdx {
  int m0, n0, z;
};
__device__ __forceinline__ TileIdx tile_of(int t, int mtiles, int ntiles, int bn) {
  const int per = mtiles * ntiles;
  const int z = t / per, r = t - z * per;
  return {(r / ntiles) * kBM, (r % ntiles) * bn, z};
}

// A operand of a 3x3 convolution read straight from the NHWC activations
// (implicit GEMM): row p of A is output pixel p, column t C + c is channel c
// of input pixel (y + t / 3 - 1, x + t % 3 - 1).  H, W: image size; cpt = C / 8
// chunks of 8 channels per tap; kchunks = 9 cpt.
struct ConvGeom {
  int H, W, cpt, kchunks;
};

// AM = 0: A through a tiled map (128-byte swizzle); AM = 1: A through an
// im2col map of the activations (ConvGeom), one load per 8-channel chunk of
// K into the no-swizzle core-matrix layout: chunk q of a K step fills bytes
// q * 2048 .. + 2047 of the A tile (128 pixels x 16 bytes, eight 8 x 16-byte
// core matrices along M), so the descriptor's K stride is 2048 bytes and its
// M stride 128; AM = 2 (C a multiple of 64): one im2col load of 64 channels
// of one tap per K step, with the 128-byte swizzle of the tiled layout;
// AM = 3 (C a multiple of 32): two loads of 32 channels per K step, each a
// 128 x 64-byte half of the tile with the 64-byte swizzle.
template <int BN, int S, int AM>
__global__ void __launch_bounds__(kTmaThreads, 1)
    gemm_bf16_tn_tma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M,
                            int N, int K, const float* __restrict__ bias, int relu, float* __restrict__ C32,
                            __nv_bfloat16* __restrict__ C16, int ldc, int* __restrict__ status, int vec16,
                            int vec32, int mtiles, int ntiles, int tiles, long long wlimit, ConvGeom geo) {
  // wlimit bounds the waits for work (operands, accumulators); the waits
  // that drain MMAs and copies already in flight keep the fixed limit, so a
  // CTA that gives up never leaves an asynchronous operation behind
  using T = TmaTile<BN, S>;
  extern __shared__ __align__(1024) unsigned char dyn_smem[];
  __shared__ __align__(8) uint64_t full[S], empty[S], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int failed;
  __shared__ int issued, consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // the 128-byte swizzle pattern repeats every 1024 bytes: align the ring
  const uint32_t raw = smem_u32(dyn_smem);
  unsigned char* ring = dyn_smem + ((1024u - (raw & 1023u)) & 1023u);
  float* epi = reinterpret_cast<float*>(ring + S * T::kStageBytes);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(T::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(&drain, 1);
    failed = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int ksteps = (K + kBK - 1) / kBK;

  if (warp == 0) {
    if (lane == 0) {
      // producer: the it-th K step overall (across this CTA's tiles) goes to
      // stage it % S; its (it / S)-th use of the stage waits for completion
      // it / S - 1 of the stage's "empty" barrier
      int it = 0;
      for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
        const TileIdx ti = tile_of(t, mtiles, ntiles, BN);
        for (int kt = 0; kt < ksteps; ++kt, ++it) {
          const int s = it % S;
          if (it >= S && !mbar_wait(&empty[s], (uint32_t)((it / S - 1) & 1), &failed, wlimit)) {
            failed = 1;
            break;
          }
          unsigned char* sa = ring + s * T::kStageBytes;
          mbar_expect_tx(&full[s], T::kStageBytes);
          if constexpr (AM == 0) {
            tma_load_3d(sa, &mapA, kt * kBK, ti.z, ti.m0, &full[s]);
          } else if constexpr (AM == 3) {
            // 32 channels of a tap per half K step (C % 32 == 0): two loads of 128 pixels x 64 bytes, 64-byte swizzle
            const int hw = geo.H * geo.W;
            const int b0 = ti.m0 / hw, rem = ti.m0 - b0 * hw, h0 = rem / geo.W, w0 = rem - h0 * geo.W;
            const int C = geo.cpt * 8;
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
              const int k0 = kt * kBK + j * 32;
              int cc = C, tap = 0;   // past K: a channel past the end, zero filled
              if (k0 < 9 * C) {
                tap = k0 / C;
                cc = k0 - tap * C;
              }
              tma_load_im2col(sa + j * 8192, &mapA, cc, w0 - 1, h0 - 1, b0, (uint16_t)(tap % 3), (uint16_t)(tap / 3),
                              &full[s]);
            }
          } else if constexpr (AM == 2) {
            // 64 channels of one tap per K step (C % 64 == 0): one load, 128-byte swizzle
            const int hw = geo.H * geo.W;
            const int b0 = ti.m0 / hw, rem = ti.m0 - b0 * hw, h0 = rem / geo.W, w0 = rem - h0 * geo.W;
            const int k0 = kt * kBK, C = geo.cpt * 8, tap = k0 / C;
            tma_load_im2col(sa, &mapA, k0 - tap * C, w0 - 1, h0 - 1, b0, (uint16_t)(tap % 3), (uint16_t)(tap / 3),
                            &full[s]);
          } else {
            // the tile's first output pixel (b0, h0, w0) is bounding-box pixel (w0 - 1, h0 - 1)
            const int hw = geo.H * geo.W;
            const int b0 = ti.m0 / hw, rem = ti.m0 - b0 * hw, h0 = rem / geo.W, w0 = rem - h0 * geo.W;
#pragma unroll 1
            for (int q = 0; q < kBK / 8; ++q) {
              const int g = kt * (kBK / 8) + q;
              int cc = geo.cpt * 8, tap = 0;   // past the last chunk: a channel past the end, zero filled
              if (g < geo.kchunks) {
                tap = g / geo.cpt;
                cc = (g - tap * geo.cpt) * 8;
              }
              tma_load_im2col(sa + q * 2048, &mapA, cc, w0 - 1, h0 - 1, b0, (uint16_t)(tap % 3), (uint16_t)(tap / 3),
                              &full[s]);
            }
          }
          tma_load_3d(sa + T::kABytes, &mapB, kt * kBK, ti.z, ti.n0, &full[s]);
        }
      }
      issued = it;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: tile number tc of this CTA accumulates into TMEM columns
      // (tc % 2) * BN, after the epilogue has drained that buffer's previous
      // tile (completion tc / 2 - 1 of acc_empty)
      const uint32_t idesc = instr_desc(kBM, BN);
      int it = 0, tc = 0;
      for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x, ++tc) {
        const int b = tc & 1;
        if (tc >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)((tc / 2 - 1) & 1), &failed, wlimit)) {
          failed = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(b * BN);
        bool ok = true;
        for (int kt = 0; kt < ksteps; ++kt, ++it) {
          const int s = it % S;
          if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), &failed, wlimit)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(ring + s * T::kStageBytes), b0 = a0 + T::kABytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            // K = 16: 32 bytes into the swizzled 128-byte rows, or two 2048-byte chunks of the im2col tile
            const uint64_t ad = AM == 1   ? smem_desc(a0 + kk * 4096, 2048, 128)
                                : AM == 3 ? smem_desc_sw64(a0 + (kk >> 1) * 8192 + (kk & 1) * 32)
                                          : smem_desc_sw128(a0 + kk * 32);
            mma_bf16(acc, ad, smem_desc_sw128(b0 + kk * 32), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) {
          failed = 1;
          break;
        }
        mma_commit(&acc_full[b]);
      }
      consumed = it;
      mma_commit(&drain);   // completes once every MMA issued above has completed
      if (!mbar_wait(&drain, 0)) failed = 1;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. rows
    // 32 (w % 4) .. of the tile; the two warps of a quadrant take alternate
    // 32-column blocks.  A block goes through this warp's transpose buffer
    // (rows of 128 bytes, 16-byte slot j of row r stored at slot j ^ (r % 8),
    // so that both the row-per-lane writes and the row-segment reads are
    // free of bank conflicts); each store instruction then writes whole row
    // segments of C.
    const int q = warp & 3, half = (warp - 2) >> 2;
    float* st = epi + (warp - 2) * 32 * 32;
    int tc = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++tc) {
      const int b = tc & 1;
      // every lane waits; the outcome is made uniform over the warp before the
      // warp-collective TMEM loads
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)((tc / 2) & 1), &failed, wlimit))) {
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const TileIdx ti = tile_of(t, mtiles, ntiles, BN);
      float* c32 = C32 ? C32 + (size_t)ti.z * M * ldc : nullptr;
      const int rbase = ti.m0 + q * 32;
      for (int ch = half; ch < BN / 32; ch += 2) {
        const int c0 = ti.n0 + ch * 32;
        if (c0 >= N) break;   // uniform over the warp
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + ch * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        __syncwarp();   // the previous block's reads of the buffer are done
        {
          float4* row = reinterpret_cast<float4*>(st + lane * 32);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            row[j ^ (lane & 7)] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                              __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
        }
        __syncwarp();
        const bool full_rows = rbase + 32 <= M, full_cols = c0 + 32 <= N;
        if (c32) {
          // lane l: columns c0 + 4 (l % 8) .. + 3 of rows 4 i + l / 8
          const int j = lane & 7, cc = c0 + 4 * j;
          float bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) bv[u] = (bias && cc + u < N) ? bias[cc + u] : 0.f;
          const bool fast = full_rows && full_cols && vec32;
#pragma unroll 2
          for (int i = 0; i < 8; ++i) {
            const int rr = 4 * i + (lane >> 3), row = rbase + rr;
            float4 v = reinterpret_cast<const float4*>(st + rr * 32)[j ^ (rr & 7)];
            float* e = &v.x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              e[u] += bv[u];
              if (relu) e[u] = fmaxf(e[u], 0.f);
            }
            float* dst = c32 + (size_t)row * ldc + cc;
            if (fast) {
              *reinterpret_cast<float4*>(dst) = v;
            } else if (row < M) {
              for (int u = 0; u < 4; ++u)
                if (cc + u < N) dst[u] = e[u];
            }
          }
        }
        if (C16) {
          // lane l: columns c0 + 8 (l % 4) .. + 7 of rows 8 i + l / 4
          const int p = lane & 3, cc = c0 + 8 * p;
          float bv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) bv[u] = (bias && cc + u < N) ? bias[cc + u] : 0.f;
          const bool fast = full_rows && full_cols && vec16;
#pragma unroll 2
          for (int i = 0; i < 4; ++i) {
            const int rr = 8 * i + (lane >> 2), row = rbase + rr;
            const float4* srow = reinterpret_cast<const float4*>(st + rr * 32);
            const float4 v0 = srow[(2 * p) ^ (rr & 7)], v1 = srow[(2 * p + 1) ^ (rr & 7)];
            float e[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              e[u] += bv[u];
              if (relu) e[u] = fmaxf(e[u], 0.f);
            }
            __nv_bfloat16* dst = C16 + (size_t)row * ldc + cc;
            if (fast) {
              uint4 pk;
              uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(e[2 * u], e[2 * u + 1]);
                w[u] = *reinterpret_cast<const uint32_t*>(&b2);
              }
              *reinterpret_cast<uint4*>(dst) = pk;
            } else if (row < M) {
              for (int u = 0; u < 8; ++u)
                if (cc + u < N) dst[u] = __float2bfloat16_rn(e[u]);
            }
          }
        }
      }
      // this warp's reads of accumulator b are complete
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
    }
  }
  __syncwarp();
  __syncthreads();
  if (failed && threadIdx.x == 0) {
    // loads issued but never consumed are still landing in the ring
    for (int it = consumed; it < issued; ++it) (void)mbar_wait(&full[it % S], (uint32_t)((it / S) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T::kTmemCols) : "memory");
  }
  if (failed && threadIdx.x == 0) atomicExch(status, 1);
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    (void)cudaGetLastError();
  });
  return fn;
}

// Tensor map of a K-major BF16 operand [rows][ld] read as `ksplit` slices of
// `kslice` columns: dimensions {kslice, ksplit, rows}, strides {kslice, ld}
// elements (both multiples of 8, i.e. of 16 bytes), box {64, 1, box_rows},
// 128-byte swizzle, zero fill outside.
bool operand_map(CUtensorMap* map, const void* base, long ld, int rows, int kslice, int ksplit, int box_rows) {
  const EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)kslice, (cuuint64_t)ksplit, (cuuint64_t)rows};
  const cuuint64_t strides[2] = {(cuuint64_t)kslice * 2, (cuuint64_t)ld * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kBK, 1, (cuuint32_t)box_rows};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// cuTensorMapEncodeIm2col from the driver, looked up once.
using EncodeIm2col = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const int*, const int*, cuuint32_t, cuuint32_t, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeIm2col encoder_im2col() {
  static std::once_flag once;
  static EncodeIm2col fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeIm2col", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeIm2col>(p);
    (void)cudaGetLastError();
  });
  return fn;
}

// im2col map of NHWC BF16 activations [B][H][W][C] for a 3x3 convolution with
// zero padding 1: dimensions {C, W, H, B}; the starting pixels of the filter
// window run over the bounding box [-1, W - 2] x [-1, H - 2] (both corners
// -1), the filter offsets (0 .. 2) are added per load; cpp channels per
// pixel (8: one K chunk, no swizzle; 32: half a K step, 64-byte swizzle; 64:
// one K step, 128-byte swizzle) and
// 128 pixels per load (one 128-row A tile), zero outside the tensor.
bool im2col_map(CUtensorMap* map, const void* X, int B, int H, int W, int C, int cpp) {
  const EncodeIm2col fn = encoder_im2col();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const int lower[2] = {-1, -1}, upper[2] = {-1, -1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(X), dims, strides, lower, upper,
            (cuuint32_t)cpp, (cuuint32_t)kBM, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            cpp == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
            : cpp == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                        : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static std::once_flag once;
  static int sms = 0;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 0;
    (void)cudaGetLastError();
  });
  return sms;
}

// Tile width: the widest of 256, 128 that pads N no more than 64 does and
// still gives every SM a tile; else 64.
int pick_bn(int M, int N) {
  const long mt = (M + kBM - 1) / kBM;
  const long pad64 = (N + 63L) / 64 * 64;
  for (int bn : {256, 128}) {
    const long nt = (N + bn - 1) / bn;
    if (nt * bn == pad64 && mt * nt >= sm_count()) return bn;
  }
  return 64;
}

// Poll limit of the TMA kernel's work waits (0: kSpinLimit); see
// cmg_nn_set_wait_limit.
std::atomic<long long> g_wait_limit{0};

template <int BN, int S, int AM = 0>
cudaError_t launch_tma(const CUtensorMap& mA, const CUtensorMap& mB, int M, int N, int K, const float* bias, int relu,
                       float* C32, __nv_bfloat16* C16, int ldc, int* status, cudaStream_t s, int ksplit, int vec16,
                       int vec32, ConvGeom geo = ConvGeom{0, 0, 0, 0}) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(gemm_bf16_tn_tma_kernel<BN, S, AM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TmaTile<BN, S>::kSmem);
  });
  if (attr != cudaSuccess) return attr;
  const int mtiles = (M + kBM - 1) / kBM, ntiles = (N + BN - 1) / BN;
  const long tiles = (long)mtiles * ntiles * ksplit;
  if (tiles > 0x7fffffffL) return cudaErrorInvalidValue;
  const int sms = sm_count();
  const unsigned grid = (unsigned)(tiles < sms ? tiles : (sms > 0 ? sms : 1));   // persistent: one CTA per SM
  const long long wl = g_wait_limit.load(std::memory_order_relaxed);
  gemm_bf16_tn_tma_kernel<BN, S, AM><<<grid, kTmaThreads, TmaTile<BN, S>::kSmem, s>>>(
      mA, mB, M, N, K, bias, relu, C32, C16, ldc, status, vec16, vec32, mtiles, ntiles, (int)tiles,
      wl > 0 ? wl : (long long)kSpinLimit, geo);
  return cudaGetLastError();
}

}  // namespace nn

void set_gemm_wait_limit(long long polls) { nn::g_wait_limit.store(polls, std::memory_order_relaxed); }

cudaError_t launch_conv3x3_bf16(const void* X, int B, int H, int W, int C, const void* Wt, int Cout,
                                const float* bias, int relu, void* Y16, int* status, cudaStream_t s) {
  const char* env = std::getenv("CMG_GEMM_TMA");
  if (env && env[0] == '0') return cudaErrorNotSupported;
  const long P = (long)B * H * W;
  // loads per K step of 64: one (C a multiple of 64), two (of 32) or eight
  // (C = 8, 16, 24: one per 8-channel chunk of a tap)
  const int cpp = C % 64 == 0 ? 64 : C % 32 == 0 ? 32 : (C % 8 == 0 && C < 32) ? 8 : 0;
  if (!cpp || Cout < 1 || Cout > 64 || P < 1 || P > 0x7fffffffL || 9L * C > 0x7fffffffL)
    return cudaErrorNotSupported;
  const int K = 9 * C;
  CUtensorMap mA, mB;
  if (!nn::im2col_map(&mA, X, B, H, W, C, cpp) || !nn::operand_map(&mB, Wt, K, Cout, K, 1, 64))
    return cudaErrorNotSupported;
  const int vec16 = (Cout % 8 == 0) && ((reinterpret_cast<uintptr_t>(Y16) & 15) == 0);
  const nn::ConvGeom geo{H, W, C / 8, 9 * (C / 8)};
  __nv_bfloat16* y16 = static_cast<__nv_bfloat16*>(Y16);
  cudaError_t e;
  if (cpp == 64)
    e = nn::launch_tma<64, 7, 2>(mA, mB, (int)P, Cout, K, bias, relu, nullptr, y16, Cout, status, s, 1, vec16, 0, geo);
  else if (cpp == 32)
    e = nn::launch_tma<64, 7, 3>(mA, mB, (int)P, Cout, K, bias, relu, nullptr, y16, Cout, status, s, 1, vec16, 0, geo);
  else
    e = nn::launch_tma<64, 7, 1>(mA, mB, (int)P, Cout, K, bias, relu, nullptr, y16, Cout, status, s, 1, vec16, 0, geo);
  count_launches(1);
  return e;
}

cudaError_t launch_gemm_bf16_tn(const void* A, long lda, const void* B, long ldb, int M, int N, int K,
                                const float* bias, int relu, float* C32, void* C16, int ldc, int* status,
                                cudaStream_t s, int ksplit) {
  // 16-byte epilogue stores need every row start 16-byte aligned
  const int vec16 = C16 && (ldc % 8 == 0) && ((reinterpret_cast<uintptr_t>(C16) & 15) == 0);
  const int vec32 = C32 && (ldc % 4 == 0) && ((reinterpret_cast<uintptr_t>(C32) & 15) == 0) &&
                    (ksplit == 1 || ((size_t)M * ldc) % 4 == 0);
  __nv_bfloat16* c16 = static_cast<__nv_bfloat16*>(C16);
  const char* env = std::getenv("CMG_GEMM_TMA");
  if (!(env && env[0] == '0')) {
    const int bn = nn::pick_bn(M, N);
    CUtensorMap mA, mB;
    if (nn::operand_map(&mA, A, lda, M, K, ksplit, nn::kBM) && nn::operand_map(&mB, B, ldb, N, K, ksplit, bn)) {
      cudaError_t e;
      // persistent, one CTA per SM: as many stages as fit beside the epilogue buffers
      if (bn == 256)
        e = nn::launch_tma<256, 3>(mA, mB, M, N, K, bias, relu, C32, c16, ldc, status, s, ksplit, vec16, vec32);
      else if (bn == 128)
        e = nn::launch_tma<128, 5>(mA, mB, M, N, K, bias, relu, C32, c16, ldc, status, s, ksplit, vec16, vec32);
      else
        e = nn::launch_tma<64, 7>(mA, mB, M, N, K, bias, relu, C32, c16, ldc, status, s, ksplit, vec16, vec32);
      count_launches(1);
      return e;
    }
  }
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(nn::gemm_bf16_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               nn::kSmemBytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((M + nn::kBM - 1) / nn::kBM, (N + nn::kBN - 1) / nn::kBN, ksplit);
  nn::gemm_bf16_tn_kernel<<<grid, nn::kThreads, nn::kSmemBytes, s>>>(
      static_cast<const __nv_bfloat16*>(A), lda, static_cast<const __nv_bfloat16*>(B), ldb, M, N, K, bias, relu, C32,
      c16, ldc, status, vec16, vec32);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cmg
