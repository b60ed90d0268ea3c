// FP32 red-black half-sweep with its loads staged through shared memory.
//
// The direct-load sweep (rbgs_item in cmg_items.cuh) is bound by global-
// memory latency: a lane holds its 14 vectors per sample chunk (right sides
// f_y, f_p, the four faces, four y and four p neighbours) in registers, so
// the number of loads a warp can keep in flight is capped by its register
// budget.  Here each warp is persistent and double-buffered: while it
// computes node group i from one shared-memory buffer, the asynchronous
// copies (cp.async, 16 bytes each, zero-filled at the boundary) of its next
// group are already landing in the other, costing no registers.  Every lane
// copies and later reads only its own vectors, so no barrier is needed
// beyond the copy-group wait.  The arithmetic is that of rbgs_item (same
// operand order), with Eq. (13) for u (its Schur scalar in FP64).
#include <cstdint>
#include <mutex>

#include "cmg_common.cuh"

namespace cmg {

namespace {

constexpr int kStageWarps = 4;   // warps per CTA
constexpr int kStageVecs = 14;   // 16-byte vectors per lane and sample chunk

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool full) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  // src-size 0 writes 16 zero bytes (a neighbour outside the grid)
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(full ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <int SPL>
constexpr size_t staged_smem_bytes() {
  return (size_t)kStageWarps * (2 * SPL * kStageVecs * 32 * sizeof(float4) + 2 * 32 * sizeof(double) +
                                2 * 2 * 32 * sizeof(float));
}

template <int SPL>
__global__ void __launch_bounds__(kStageWarps * 32) rbgs_staged_kernel(LevelView<float> L, Vec3<float> x,
                                                                       Vec3c<float> f, int colour, int lpn,
                                                                       long groups) {
  pdl_enter();
  extern __shared__ __align__(16) float4 sbuf[];
  constexpr int VEC = SPL * kStageVecs;   // vectors per lane per buffer
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* wv = sbuf + (size_t)warp * 2 * VEC * 32;   // [2][VEC][32]
  // per warp: 1/sigma_i in FP64 [2][32], then the control right side and
  // the FP32 1/sigma_i (all-FP32 option) [2][2][32]
  double* wd = reinterpret_cast<double*>(sbuf + (size_t)kStageWarps * 2 * VEC * 32) + warp * 2 * 32;
  float* ws = reinterpret_cast<float*>(reinterpret_cast<double*>(sbuf + (size_t)kStageWarps * 2 * VEC * 32) +
                                       kStageWarps * 2 * 32) + warp * 2 * 2 * 32;
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const int gpw = 32 / lpn, sub = lane / lpn, ln = lane & (lpn - 1);
  const long items = (groups + gpw - 1) / gpw;
  const long stride = (long)gridDim.x * kStageWarps;
  long item = (long)blockIdx.x * kStageWarps + warp;
  if (item >= items) return;   // uniform over the warp

  auto issue = [&](long it, int b) {
    const long g = it * gpw + sub;
    const bool valid = g < groups;
    int iy = 0, ix = 0;
    if (valid) colour_node(g, n, colour, iy, ix);
    const size_t node = (size_t)iy * n + ix, o = node * ld;
    const float* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const float* kSp = L.ky + ((size_t)iy * n + ix) * ld;
    const bool hW = ix > 0, hE = ix < n - 1, hS = iy > 0, hN = iy < n - 1;
    float4* d = wv + (size_t)b * VEC * 32 + lane;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (ln + s * lpn) * 4;
      const bool ok = valid && j < N;
      const size_t jj = ok ? (size_t)j : 0;
      const float* safe = f.y + o + jj;   // in bounds; read with size 0 when the vector is not needed
      const float* src[kStageVecs] = {f.y + o + jj,        f.p + o + jj,         kWp + jj,
                                      kWp + ld + jj,       kSp + jj,             kSp + (size_t)n * ld + jj,
                                      x.y + o - ld + jj,   x.y + o + ld + jj,    x.y + o - (size_t)n * ld + jj,
                                      x.y + o + (size_t)n * ld + jj,             x.p + o - ld + jj,
                                      x.p + o + ld + jj,   x.p + o - (size_t)n * ld + jj,
                                      x.p + o + (size_t)n * ld + jj};
      const bool use[kStageVecs] = {ok, ok, ok, ok, ok, ok, ok && hW, ok && hE, ok && hS, ok && hN,
                                    ok && hW, ok && hE, ok && hS, ok && hN};
#pragma unroll
      for (int t = 0; t < kStageVecs; ++t) cp_async16(d + (s * kStageVecs + t) * 32, use[t] ? src[t] : safe, use[t]);
    }
    cp_async4(ws + (b * 2 + 0) * 32 + lane, (L.freeze_u ? x.u : f.u) + node);
    if (L.ctl32) cp_async4(ws + (b * 2 + 1) * 32 + lane, L.isigma32 + node);
    else cp_async8(wd + b * 32 + lane, L.isigma + node);
    cp_async_commit();
  };

  auto compute = [&](long it, int b) {
    const long g = it * gpw + sub;
    const bool valid = g < groups;
    int iy = 0, ix = 0;
    if (valid) colour_node(g, n, colour, iy, ix);
    const size_t node = (size_t)iy * n + ix, o = node * ld;
    const bool ctl = L.ctl.inside(iy, ix);
    const float4* d = wv + (size_t)b * VEC * 32 + lane;
    const float c = (float)L.c, e = (float)L.e;
    float bp[SPL][4], by[SPL][4], ia[SPL][4];
    float tacc = 0.f;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (ln + s * lpn) * 4;
      if (valid && j < N) {
        float4 v[kStageVecs];
#pragma unroll
        for (int t = 0; t < kStageVecs; ++t) v[t] = d[(s * kStageVecs + t) * 32];
        const float* fy = &v[0].x;
        const float* fp = &v[1].x;
        const float* kW = &v[2].x;
        const float* kE = &v[3].x;
        const float* kS = &v[4].x;
        const float* kN = &v[5].x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float a = fy[k];   // first block row: c y + A p = f_y
          a = fmaf(kW[k], (&v[10].x)[k], a);
          a = fmaf(kE[k], (&v[11].x)[k], a);
          a = fmaf(kS[k], (&v[12].x)[k], a);
          a = fmaf(kN[k], (&v[13].x)[k], a);
          bp[s][k] = a;
          float q = fp[k];   // last block row: A y + e u = f_p
          q = fmaf(kW[k], (&v[6].x)[k], q);
          q = fmaf(kE[k], (&v[7].x)[k], q);
          q = fmaf(kS[k], (&v[8].x)[k], q);
          q = fmaf(kN[k], (&v[9].x)[k], q);
          by[s][k] = q;
          ia[s][k] = __frcp_rn((kW[k] + kE[k]) + (kS[k] + kN[k]));
          tacc += (c * ia[s][k]) * (ia[s][k] * by[s][k]) - ia[s][k] * bp[s][k];
        }
      }
    }
    // Eq. (13)'s Schur scalar for u in FP64 (schur_u); every lane takes part
    const float bu = valid ? ws[(b * 2 + 0) * 32 + lane] : 0.f;
    const double isg = !valid ? 0.0 : (L.ctl32 ? (double)ws[(b * 2 + 1) * 32 + lane] : wd[b * 32 + lane]);
    const double su = schur_u<float>(L, tacc, lpn, (double)bu, valid ? d_of(L, (long)node) : 0.0, isg);
    if (!valid) return;
    const float uu = L.freeze_u ? bu : (ctl ? (float)su : 0.f);
    if (ln == 0 && !L.freeze_u) x.u[node] = uu;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (ln + s * lpn) * 4;
      if (j < N) {
        float4 yn, pn;
        float* yv = &yn.x;
        float* pv = &pn.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          yv[k] = ia[s][k] * (by[s][k] - e * uu);
          pv[k] = ia[s][k] * (bp[s][k] - c * yv[k]);
        }
        *reinterpret_cast<float4*>(x.y + o + j) = yn;
        *reinterpret_cast<float4*>(x.p + o + j) = pn;
      }
    }
  };

  issue(item, 0);
  int b = 0;
  for (; item < items; item += stride) {
    const long next = item + stride;
    if (next < items) issue(next, b ^ 1);
    else cp_async_commit();   // empty group keeps the wait count uniform
    cp_async_wait_prev();     // the group of `item` has landed
    compute(item, b);
    b ^= 1;
  }
}

// Resident CTAs per SM times the SM count, queried once per instantiation.
template <int SPL>
int staged_grid_cap() {
  static std::once_flag once;
  static int cap = 0;
  std::call_once(once, [] {
    auto kern = rbgs_staged_kernel<SPL>;
    int dev = 0, sms = 0, per = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged_smem_bytes<SPL>()) ==
            cudaSuccess &&
        cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kStageWarps * 32, staged_smem_bytes<SPL>()) ==
            cudaSuccess)
      cap = sms * per;
    (void)cudaGetLastError();
  });
  return cap;
}

}  // namespace

bool staged_supported(int N, int spl) { return N % 4 == 0 && (spl == 1 || spl == 2); }

cudaError_t launch_rbgs_half_staged(const LevelView<float>& L, Vec3<float> x, Vec3c<float> f, int colour,
                                    const SampleMap& m, cudaStream_t st) {
  if (m.V != 4 || !staged_supported(L.N, m.spl) || (L.ctl32 ? !L.isigma32 : !L.isigma)) return cudaErrorNotSupported;
  const long groups = colour_count(L.n, colour);
  const long items = (groups + (32 / m.lpn) - 1) / (32 / m.lpn);
  const long need = (items + kStageWarps - 1) / kStageWarps;
  if (m.spl == 1) {
    const int cap = staged_grid_cap<1>();
    if (cap <= 0) return cudaErrorNotSupported;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    const cudaError_t e = launch_k(rbgs_staged_kernel<1>, dim3(grid), dim3(kStageWarps * 32), staged_smem_bytes<1>(),
                                   st, L, x, f, colour, m.lpn, groups);
    if (e != cudaSuccess) return e;
  } else {
    const int cap = staged_grid_cap<2>();
    if (cap <= 0) return cudaErrorNotSupported;
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    const cudaError_t e = launch_k(rbgs_staged_kernel<2>, dim3(grid), dim3(kStageWarps * 32), staged_smem_bytes<2>(),
                                   st, L, x, f, colour, m.lpn, groups);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = cudaGetLastError();
  count_launches(1);
  return e;
}

}  // namespace cmg
