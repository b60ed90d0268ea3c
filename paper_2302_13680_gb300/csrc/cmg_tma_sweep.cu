// FP32 red-black half-sweep (the GS variant named after Eq. (11), Eq. (13)
// at every node of one colour) with its operands brought into shared memory
// by TMA tensor loads that gather every other node of a grid row.
//
// The direct-load sweep (rbgs_item) keeps a node group's loads in
// registers, so the bytes a warp has in flight are capped by its register
// budget and the sweep waits on memory latency.  Here a task is a segment
// of W consecutive nodes of one colour in one grid row (x = ix0, ix0 + 2,
// ...).  One producer thread per CTA loads, per task, eleven boxes with a
// traversal stride of 2 nodes -- f_y, f_p, the rows above and below of y
// and p, the W + 1 left/right neighbours of y and p, the south and north
// faces -- and one of 2W consecutive x-faces, each completing on the
// stage's mbarrier, into a ring of shared-memory stages; neighbours outside
// the grid arrive as the loads' zero fill.  The consumer warps update the
// segment's nodes from the stage and store y, p, u to global memory, then
// free the stage.
//
// Per node the arithmetic, its operand order and the sample map (lanes per
// node, chunks per lane, 16-byte vectors) are those of rbgs_node, so the
// result equals the direct half-sweep's bit for bit.  Covered: the plain
// half-sweep (control updated, a read iterate) with N % 4 == 0, N <= 256
// and 16-byte aligned arrays; elsewhere the launcher returns
// cudaErrorNotSupported and the caller takes the direct kernel.
//
// Every wait is bounded: a wait that runs out adds one to a counter
// (cmg_sweep_wait_timeouts) and makes the CTA's later waits return at
// once; the producer ends by waiting for the loads of the last use of every
// stage, so no copy is in flight when the CTA exits.
#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "cmg_items.cuh"

namespace cmg {

static_assert(kTuneTma == CMG_TUNE_TMA, "tuning flag of the C ABI");

namespace {

constexpr int kTmaSeg = 4;               // nodes of one colour per task (W)
constexpr int kTmaMaxStages = 8;
constexpr size_t kTmaRingBytes = 200 * 1024;
constexpr size_t kTmaSmemMax = 224 * 1024;   // dynamic shared memory of a CTA, ring and margins
constexpr long long kTmaSpin = 1LL << 20;   // polls of one wait before it gives up

// Regions of a stage, in node rows of N floats (each region starts on a
// 128-byte boundary): W f_y, W f_p, W + 1 y and p left/right neighbours
// (slot k = left of node k, slot k + 1 = its right), W each of y and p
// below and above, 2W x-faces (slot 2k west, 2k + 1 east of node k), W
// south and W north y-faces.
enum { kRegFY = 0, kRegFP, kRegYWE, kRegPWE, kRegYS, kRegYN, kRegPS, kRegPN, kRegKX, kRegKS, kRegKN, kRegCount };

__host__ __device__ inline int region_rows(int r, int W) {
  return (r == kRegYWE || r == kRegPWE) ? W + 1 : (r == kRegKX ? 2 * W : W);
}

struct SweepMaps {
  CUtensorMap fy, fp;   // {N, n, n}, box {N, 2W, 1}, node stride 2
  CUtensorMap yA, pA;   // the same shape over y and p
  CUtensorMap yB, pB;   // box {N, 2(W + 1), 1}, node stride 2
  CUtensorMap kx;       // {N, n + 1, n}, box {N, 2W, 1}, stride 1
  CUtensorMap ky;       // {N, n, n + 1}, box {N, 2W, 1}, node stride 2
};

__device__ unsigned int g_tma_timeouts;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__device__ __forceinline__ void bar_arrive_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

// Wait (acquire) for the completion of the phase with this parity; bounded.
// With `abort` (the CTA's flag): a wait that runs out raises it, and every
// later such wait of the CTA returns at once.
__device__ __forceinline__ void bar_wait(uint64_t* b, uint32_t parity, volatile int* abort = nullptr) {
  const uint32_t a = saddr(b);
  for (long long i = 0; i < kTmaSpin; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return;
    if (abort && *abort) return;
  }
  if (abort) *abort = 1;
  atomicAdd(&g_tma_timeouts, 1u);
}

// One box of a 3-D tensor map at (0, c1, c2) into shared memory, completing
// on `b`.  The innermost coordinate is 0 (16-byte aligned); c1, c2 may lie
// outside the tensor (zero fill).
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, int c1, int c2, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(saddr(b))
      : "memory");
}

constexpr int kTmaMaxConsumers = 4;

// One CTA per SM: warp 0 (one thread) produces, warps 1 .. consumers update
// the nodes.  Task t is segment t % segs of grid row t / segs; the CTA's
// k-th task goes to stage k % stages and every consumer warp takes npw of
// its W nodes (warp w: nodes w npw .. w npw + npw - 1).
template <int SPL>
__global__ void __launch_bounds__((1 + kTmaMaxConsumers) * 32, 1)
    rbgs_tma_kernel(const __grid_constant__ SweepMaps M, LevelView<float> L, Vec3<float> x, Vec3c<float> f,
                    int colour, int lpn, int W, int segs, long tasks, int stages, int consumers) {
  constexpr int V = 4;
  extern __shared__ __align__(128) float ring_raw[];
  // the ring starts on a 128-byte boundary (the launch adds 128 bytes)
  float* ring = ring_raw + ((128u - (saddr(ring_raw) & 127u)) & 127u) / sizeof(float);
  __shared__ uint64_t full[kTmaMaxStages], empty[kTmaMaxStages];
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = L.n, N = L.N;
  // region offsets within a stage (floats, 128-byte aligned) and the bytes
  // the loads of one task deliver
  int off[kRegCount];
  int stage_floats = 0;
  uint32_t task_bytes = 0;
#pragma unroll
  for (int r = 0; r < kRegCount; ++r) {
    off[r] = stage_floats;
    const int bytes = region_rows(r, W) * N * (int)sizeof(float);
    task_bytes += (uint32_t)bytes;
    stage_floats += ((bytes + 127) / 128) * 32;
  }
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < stages; ++s) {
      bar_init(&full[s], 1);            // the producer's arrive (with the loads' bytes)
      bar_init(&empty[s], consumers);   // one arrive per consumer warp
    }
  }
  __syncthreads();
  pdl_enter();

  if (warp == 0) {
    if (lane == 0) {
      long k = 0;
      for (long t = blockIdx.x; t < tasks; t += gridDim.x, ++k) {
        const int s = (int)(k % stages);
        const long use = k / stages;
        if (use > 0) bar_wait(&empty[s], (uint32_t)((use - 1) & 1), &abort_flag);   // its last use is consumed
        const int iy = (int)(t / segs), sg = (int)(t - (long)iy * segs);
        const int p = (iy + colour) & 1, m_row = (n - p + 1) >> 1;
        if (sg * W >= m_row) {
          bar_arrive(&full[s]);   // an empty segment: nothing to load
          continue;
        }
        const int ix0 = p + 2 * sg * W;
        float* st = ring + (size_t)s * stage_floats;
        uint64_t* b = &full[s];
        bar_arrive_tx(b, task_bytes);
        tma_box(st + off[kRegFY], &M.fy, ix0, iy, b);
        tma_box(st + off[kRegFP], &M.fp, ix0, iy, b);
        tma_box(st + off[kRegYWE], &M.yB, ix0 - 1, iy, b);
        tma_box(st + off[kRegPWE], &M.pB, ix0 - 1, iy, b);
        tma_box(st + off[kRegYS], &M.yA, ix0, iy - 1, b);
        tma_box(st + off[kRegYN], &M.yA, ix0, iy + 1, b);
        tma_box(st + off[kRegPS], &M.pA, ix0, iy - 1, b);
        tma_box(st + off[kRegPN], &M.pA, ix0, iy + 1, b);
        tma_box(st + off[kRegKX], &M.kx, ix0, iy, b);
        tma_box(st + off[kRegKS], &M.ky, ix0, iy, b);
        tma_box(st + off[kRegKN], &M.ky, ix0, iy + 1, b);
      }
      // no copy may be in flight when the CTA exits: wait for the last use
      // of every stage (complete already unless a consumer gave up waiting;
      // these waits ignore the abort flag)
      for (int s = 0; s < stages && s < k; ++s) bar_wait(&full[s], (uint32_t)(((k - 1 - s) / stages) & 1));
    }
    return;
  }

  const int cw = warp - 1;
  if (cw >= consumers) return;
  const int npw = 32 / lpn;
  const int slot = cw * npw + lane / lpn, li = lane & (lpn - 1);
  const float cf = (float)L.c, ef = (float)L.e;
  long k = 0;
  for (long t = blockIdx.x; t < tasks; t += gridDim.x, ++k) {
    const int s = (int)(k % stages);
    const int iy = (int)(t / segs), sg = (int)(t - (long)iy * segs);
    const int p = (iy + colour) & 1, m_row = (n - p + 1) >> 1;
    const int kk = sg * W + slot;   // the node's index among the row's nodes of this colour
    const bool valid = slot < W && kk < m_row;
    const int ix = valid ? p + 2 * kk : 0;
    const long node = (long)iy * n + ix;
    const bool ctl = L.ctl.inside(iy, ix);
    // the node's scalars do not depend on the stage: loaded before the wait
    double bu = 0.0, isg = 0.0, dwv = 1.0;
    if (valid) {
      bu = (double)f.u[node];
      isg = isigma_of<float>(L, node);
      if (L.dw) dwv = (double)L.dw[node];
    }
    bar_wait(&full[s], (uint32_t)((k / stages) & 1), &abort_flag);
    const float* st = ring + (size_t)s * stage_floats;
    vec<float, V> bp[SPL], by[SPL], ia[SPL];
    float tacc = 0.f;
    if (valid) {
#pragma unroll
      for (int q = 0; q < SPL; ++q) {
        const int j = (li + q * lpn) * V;
        if (j < N) {
          const auto row = [&](int r, int i) { return ldv<float, V>(st + off[r] + (size_t)i * N + j); };
          const vec<float, V> kW = row(kRegKX, 2 * slot), kE = row(kRegKX, 2 * slot + 1), kS = row(kRegKS, slot),
                              kN = row(kRegKN, slot);
          bp[q] = row(kRegFY, slot);   // first block row: c y + A p = f_y
          by[q] = row(kRegFP, slot);   // last block row:  A y + e u = f_p
          // neighbours outside the grid hold the loads' zero fill, as the
          // direct sweep's absent neighbours are zero
          fma_faces<float, V>(bp[q], kW, row(kRegPWE, slot), kE, row(kRegPWE, slot + 1), kS, row(kRegPS, slot), kN,
                              row(kRegPN, slot));
          fma_faces<float, V>(by[q], kW, row(kRegYWE, slot), kE, row(kRegYWE, slot + 1), kS, row(kRegYS, slot), kN,
                              row(kRegYN, slot));
          ia[q] = inv_diag<float, V, false>(L, 0, kW, kE, kS, kN);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float iak = ia[q].v[v];
            tacc += (cf * iak) * (iak * by[q].v[v]) - iak * bp[q].v[v];
          }
        }
      }
    }
    // the stage is not read again: hand it back before the group sum
    __syncwarp();
    if (lane == 0) bar_arrive(&empty[s]);
    const double su = schur_u<float>(L, tacc, lpn, bu, L.d * dwv, isg);
    if (valid) {
      const double uu = ctl ? su : 0.0;
      if (li == 0) x.u[node] = (float)uu;
      const float uT = (float)uu;
      const size_t o = (size_t)node * N;
#pragma unroll
      for (int q = 0; q < SPL; ++q) {
        const int j = (li + q * lpn) * V;
        if (j < N) {
          vec<float, V> yn, pn;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            yn.v[v] = ia[q].v[v] * (by[q].v[v] - ef * uT);
            pn.v[v] = ia[q].v[v] * (bp[q].v[v] - cf * yn.v[v]);
          }
          stv<float, V>(x.y + o + j, yn);
          stv<float, V>(x.p + o + j, pn);
        }
      }
    }
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
EncodeTiledFn tiled_encoder() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    (void)cudaGetLastError();
  });
  return fn;
}

// A 3-D FP32 map {N, d1, d2} (row strides N and N d1 elements) with box
// {N, box1, 1} and traversal stride `stride1` along dimension 1; zero fill
// outside.
bool map3(CUtensorMap* m, const float* base, int N, int d1, int d2, int box1, int stride1) {
  const EncodeTiledFn fn = tiled_encoder();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)d1, (cuuint64_t)d2};
  const cuuint64_t strides[2] = {(cuuint64_t)N * sizeof(float), (cuuint64_t)N * d1 * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)N, (cuuint32_t)box1, 1};
  const cuuint32_t estr[3] = {1, (cuuint32_t)stride1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps per (arrays, n, N, W): made once (a sweep is launched with
// the same arrays many times, inside captured graphs too).
using MapKey = std::tuple<const void*, const void*, const void*, const void*, const void*, const void*, int, int, int>;
std::mutex g_map_mu;
std::map<MapKey, SweepMaps> g_maps;

bool sweep_maps(const LevelView<float>& L, Vec3<float> x, Vec3c<float> f, int W, SweepMaps* out) {
  const MapKey key{L.kx, L.ky, x.y, x.p, f.y, f.p, L.n, L.N, W};
  {
    std::lock_guard<std::mutex> g(g_map_mu);
    const auto it = g_maps.find(key);
    if (it != g_maps.end()) {
      *out = it->second;
      return true;
    }
  }
  const int n = L.n, N = L.N;
  SweepMaps M;
  const bool ok = map3(&M.fy, f.y, N, n, n, 2 * W, 2) && map3(&M.fp, f.p, N, n, n, 2 * W, 2) &&
                  map3(&M.yA, x.y, N, n, n, 2 * W, 2) && map3(&M.pA, x.p, N, n, n, 2 * W, 2) &&
                  map3(&M.yB, x.y, N, n, n, 2 * (W + 1), 2) && map3(&M.pB, x.p, N, n, n, 2 * (W + 1), 2) &&
                  map3(&M.kx, L.kx, N, n + 1, n, 2 * W, 1) && map3(&M.ky, L.ky, N, n, n + 1, 2 * W, 2);
  if (!ok) return false;
  std::lock_guard<std::mutex> g(g_map_mu);
  if (g_maps.size() > 4096) g_maps.clear();
  g_maps[key] = M;
  *out = M;
  return true;
}

int sm_total() {
  static std::once_flag once;
  static int sms = 0;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      sms = 0;
    (void)cudaGetLastError();
  });
  return sms;
}

template <int SPL>
bool tma_attr() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] {
    ok = cudaFuncSetAttribute(rbgs_tma_kernel<SPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kTmaSmemMax) == cudaSuccess;
    (void)cudaGetLastError();
  });
  return ok;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

cudaError_t launch_rbgs_half_tma(const LevelView<float>& L, Vec3<float> x, Vec3c<float> f, int colour,
                                 const SampleMap& m, cudaStream_t st) {
  if (m.V != 4 || (m.spl != 1 && m.spl != 2 && m.spl != 4) || L.freeze_u || L.ld != L.N || L.N % 4 != 0 ||
      L.N > 256 || L.n < 2)
    return cudaErrorNotSupported;
  if (L.ctl32 ? !L.isigma32 : !L.isigma) return cudaErrorNotSupported;
  if (!aligned16(x.y) || !aligned16(x.p) || !aligned16(f.y) || !aligned16(f.p) || !aligned16(L.kx) ||
      !aligned16(L.ky))
    return cudaErrorNotSupported;
  const int npw = 32 / m.lpn;
  const int W = std::max(kTmaSeg, npw);
  const int consumers = (W + npw - 1) / npw;
  if (consumers > kTmaMaxConsumers || 2 * (W + 1) > 256) return cudaErrorNotSupported;
  size_t stage_bytes = 0;
  for (int r = 0; r < kRegCount; ++r) stage_bytes += ((size_t)region_rows(r, W) * L.N * sizeof(float) + 127) / 128 * 128;
  const int stages = (int)std::min<size_t>(kTmaMaxStages, kTmaRingBytes / stage_bytes);
  if (stages < 2) return cudaErrorNotSupported;
  const int n = L.n;
  const int segs = ((n + 1) / 2 + W - 1) / W;
  const long tasks = (long)n * segs;
  const int sms = sm_total();
  if (sms <= 0) return cudaErrorNotSupported;
  SweepMaps M;
  if (!sweep_maps(L, x, f, W, &M)) return cudaErrorNotSupported;
  const unsigned grid = (unsigned)std::min<long>(tasks, sms);
  // + 128 bytes to align the ring, + one more region of the largest size
  // after it (room that no load is meant to reach)
  const size_t smem = (size_t)stages * stage_bytes + 128 + (size_t)2 * (W + 1) * L.N * sizeof(float);
  if (smem > kTmaSmemMax) return cudaErrorNotSupported;
  const dim3 block((1 + consumers) * 32);
  cudaError_t e = cudaErrorNotSupported;
  if (m.spl == 1 && tma_attr<1>())
    e = launch_k(rbgs_tma_kernel<1>, dim3(grid), block, smem, st, M, L, x, f, colour, m.lpn, W, segs, tasks, stages,
                 consumers);
  else if (m.spl == 2 && tma_attr<2>())
    e = launch_k(rbgs_tma_kernel<2>, dim3(grid), block, smem, st, M, L, x, f, colour, m.lpn, W, segs, tasks, stages,
                 consumers);
  else if (m.spl == 4 && tma_attr<4>())
    e = launch_k(rbgs_tma_kernel<4>, dim3(grid), block, smem, st, M, L, x, f, colour, m.lpn, W, segs, tasks, stages,
                 consumers);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cmg

extern "C" cmg_status cmg_sweep_wait_timeouts(unsigned int* count) {
  if (!count) return CMG_ERR_INVALID_ARG;
  if (cudaMemcpyFromSymbol(count, cmg::g_tma_timeouts, sizeof(unsigned int)) != cudaSuccess) {
    (void)cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  return CMG_OK;
}
