// Batched persistent form: the node kernels of the FP32 refinement loop for
// many independent instances at once (declarations and the schedule in
// cmg_internal.h, "batched persistent form").  Each instance still runs
// Algorithm 1 (V-cycle, red-black collective Gauss-Seidel, Eq. (13) per
// node) and the single-instance refinement; only the launches are shared.
//
// Work list: for a grid depth d and a kind of phase (colour-0 nodes,
// colour-1 nodes, coarse nodes of a restriction, all nodes) the items are
// (instance, warp of nodes) pairs numbered through per-instance prefix counts;
// a warp finds its instance by binary search, skips it when the instance has
// stopped iterating, and runs the same per-node items as the single-instance
// kernels (cmg_items.cuh) with that instance's sample map.  The maps take
// 16-byte vectors where N % 4 == 0, 8-byte where N % 2 == 0, else scalars,
// 16 samples per lane on depths run one launch per phase and map class (each
// variant compiled on its own: many independent loads per lane), four
// samples per lane in the persistent kernels, whose map is chosen at run
// time.
//
// The down- and up-leg kernels are persistent: every phase (half-sweep,
// residual, restriction) is separated by a grid-wide barrier, so all CTAs
// must be resident at once (cooperative launch).  A barrier wait polls a
// bounded number of times; when a wait runs out the kernel sets the batch's
// error flag and every CTA returns (the host reports CMG_ERR_TIMEOUT), and
// every later batched kernel returns at once while the flag is set.  Loads
// of values written earlier in the same launch bypass L1 (the CG items).
#include <mutex>

#include "cmg_items.cuh"

namespace cmg {

namespace {

constexpr int kBThreads = 256;              // threads per CTA of the batched node kernels
constexpr int kBWarps = kBThreads / 32;

template <int V_, int S_>
struct Map {
  static constexpr int V = V_;
  static constexpr int S = S_;
};

// (V, chunks per lane) by map rule R: kBatchMapPhase (4, 4), (2, 8), (1, 16);
// kBatchMapCoop (4, 1), (2, 2), (1, 4).  VF = 0 chooses at run time (the
// instance's V); VF = 4, 2 or 1 compiles one variant only (a launch per map
// class: the registers of one variant).
template <int V, int R>
constexpr int chunks_of() { return R == kBatchMapPhase ? 16 / V : 4 / V; }
template <int VF, int R, class F>
__device__ __forceinline__ void with_map(int V, F&& f) {
  if constexpr (VF == 4) f(Map<4, chunks_of<4, R>()>{});
  else if constexpr (VF == 2) f(Map<2, chunks_of<2, R>()>{});
  else if constexpr (VF == 1) f(Map<1, chunks_of<1, R>()>{});
  else {
    if (V == 4) f(Map<4, chunks_of<4, R>()>{});
    else if (V == 2) f(Map<2, chunks_of<2, R>()>{});
    else f(Map<1, chunks_of<1, R>()>{});
  }
}

// Map class of a table: 0 = every instance, 1 / 2 / 3 = the instances with
// V = 4 / 2 / 1.
constexpr int vclass(int VF) { return VF == 4 ? 1 : VF == 2 ? 2 : VF == 1 ? 3 : 0; }

__device__ __forceinline__ bool aborted(const BatchTables& T) { return *(volatile const int*)T.err != 0; }

// Grid-wide barrier of a cooperative launch (generation counter; the last
// CTA to arrive resets the count and advances the generation).  A CTA waits
// at most T.limit polls; if the wait runs out it sets the error flag.
// Returns false when the batch has been aborted.
__device__ bool grid_barrier(const BatchTables& T) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = T.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(T.bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(T.bar, 0u);
      __threadfence();
      atomicAdd(T.bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*gen == g) {
        if (aborted(T)) break;
        if (++polls > T.limit) {
          atomicExch(T.err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !aborted(T);
}

__device__ __forceinline__ const int* prefix(const BatchTables& T, int depth, int kind, int cls) {
  return batch_prefix(T, depth, kind, cls);
}

// Every warp of the grid walks the items of (depth, kind, map class) in
// chunks of CH consecutive items (grid-stride over chunks); fn(i, item,
// item index within instance i, lane) runs for items of iterating instances.
// The instance of a chunk's first item is found by binary search over the
// prefix counts and then advanced item by item, so a warp searches once per
// chunk.  Warp-uniform: a warp's lanes share the item.  The persistent
// kernels (few CTAs) walk chunks of 8; the per-phase launches give every
// warp one item (CH = 1, a grid of items / 8 CTAs).
template <int CH = 8, class F>
__device__ __forceinline__ void walk(const BatchTables& T, int depth, int kind, int cls, F&& fn) {
  constexpr int kChunk = CH;
  const int* pre = prefix(T, depth, kind, cls);
  const int total = pre[T.count];
  const int wtot = gridDim.x * kBWarps;
  const int lane = threadIdx.x & 31;
  for (int c0 = (blockIdx.x * kBWarps + (threadIdx.x >> 5)) * kChunk; c0 < total; c0 += wtot * kChunk) {
    int lo = 0, hi = T.count;   // pre[lo] <= c0 < pre[hi]
    if (kChunk == 1 && c0 / kBWarps < T.items[depth][kind][cls] / kBWarps + 1) {
      // one item per warp: start from the instance of the CTA's first item
      // (host table) and step forward; a CTA's items span few instances
      lo = T.first[T.first_off[depth][kind][cls] + c0 / kBWarps];
      while (pre[lo + 1] <= c0) ++lo;
      hi = lo + 1;
    }
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= c0) lo = mid;
      else hi = mid;
    }
    int next = pre[lo + 1];
    const int c1 = min(c0 + kChunk, total);
    for (int it = c0; it < c1; ++it) {
      while (it >= next) {   // the next instance with items
        ++lo;
        next = pre[lo + 1];
      }
      if (!T.act[lo]) continue;
      fn(lo, it, it - pre[lo], lane);
    }
  }
}

// ---- phases: one pass of every iterating instance's items ----------------

// Half-sweep of `colour` on the grids at `depth` (zero: the colour-0
// half-sweep of a cycle from the zero iterate, which does not read x).
template <bool CG, int VF, int CH, int R>
__device__ __forceinline__ void phase_sweep(const BatchTables& T, int depth, int colour, bool zero) {
  walk<CH>(T, depth, colour == 0 ? kBkColour0 : kBkColour1, vclass(VF), [&](int i, int, int w, int lane) {
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels + depth];
    const long g = (long)w * (32 / B.lpn) + lane / B.lpn;
    const int ln = lane & (B.lpn - 1);
    with_map<VF, R>(B.V, [&](auto m) {
      using M = decltype(m);
      if (zero) rbgs_item<float, M::V, M::S, CG, false, true>(B.L, B.x, cview(B.f), 0, g, ln, B.lpn);
      else rbgs_item<float, M::V, M::S, CG>(B.L, B.x, cview(B.f), colour, g, ln, B.lpn);
    });
  });
}

// Residual at the colour-0 nodes (it vanishes at colour 1 after the sweep).
template <bool CG, int VF, int CH, int R>
__device__ __forceinline__ void phase_residual_c0(const BatchTables& T, int depth) {
  walk<CH>(T, depth, kBkColour0, vclass(VF), [&](int i, int, int w, int lane) {
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels + depth];
    const long g = (long)w * (32 / B.lpn) + lane / B.lpn;
    const int n = B.L.n;
    long node = (long)n * n;
    if (g < colour_count(n, 0)) {
      int iy, ix;
      colour_node(g, n, 0, iy, ix);
      node = (long)iy * n + ix;
    }
    with_map<VF, R>(B.V, [&](auto m) {
      using M = decltype(m);
      residual_item<float, M::V, M::S, CG>(B.L, cview(B.x), cview(B.f), B.r, node, lane & (B.lpn - 1), B.lpn, 1.0f);
    });
  });
}

// Restriction P^T from the colour-0 points to the next grid's right side.
template <bool CG, int VF, int CH, int R>
__device__ __forceinline__ void phase_restrict(const BatchTables& T, int depth) {
  walk<CH>(T, depth, kBkCoarse, vclass(VF), [&](int i, int, int w, int lane) {
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels + depth];
    const BatchLevel& C = T.lev[(size_t)i * kMaxLevels + depth + 1];
    const long g = (long)w * (32 / B.lpn) + lane / B.lpn;
    with_map<VF, R>(B.V, [&](auto m) {
      using M = decltype(m);
      restrict_item<float, M::V, M::S, CG>(B.L.n, B.L.N, cview(B.r), C.f, Vec3<float>{nullptr, nullptr, nullptr}, g,
                                           lane & (B.lpn - 1), B.lpn, true);
    });
  });
}

// First post-smoothing half-sweep: the neighbours are read as x + P e (e =
// the next grid's iterate, the coarse correction).
template <bool CG, int VF, int CH, int R>
__device__ __forceinline__ void phase_prolong_sweep(const BatchTables& T, int depth) {
  walk<CH>(T, depth, kBkColour0, vclass(VF), [&](int i, int, int w, int lane) {
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels + depth];
    const BatchLevel& C = T.lev[(size_t)i * kMaxLevels + depth + 1];
    const long g = (long)w * (32 / B.lpn) + lane / B.lpn;
    with_map<VF, R>(B.V, [&](auto m) {
      using M = decltype(m);
      rbgs_item<float, M::V, M::S, CG, true>(B.L, B.x, cview(B.f), 0, g, lane & (B.lpn - 1), B.lpn, cview(C.x), C.L.n);
    });
  });
}

// Prolongation as its own pass: x += P e on every node of the grids at
// `depth` (e = the next grid's iterate).
template <bool CG, int VF, int CH, int R>
__device__ __forceinline__ void phase_prolong_add(const BatchTables& T, int depth) {
  walk<CH>(T, depth, kBkAll32, vclass(VF), [&](int i, int, int w, int lane) {
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels + depth];
    const BatchLevel& C = T.lev[(size_t)i * kMaxLevels + depth + 1];
    const long node = (long)w * (32 / B.lpn) + lane / B.lpn;
    with_map<VF, R>(B.V, [&](auto m) {
      using M = decltype(m);
      prolong_item<float, M::V, M::S, CG>(B.L.n, B.L.N, cview(C.x), B.x, node, lane & (B.lpn - 1), B.lpn, B.L.ctl);
    });
  });
}

// ---- the persistent per-depth kernels ----------------------------------------

// Down-leg of Algorithm 1 on the grids at `depth` (pre-smoothing from the
// zero iterate, residual at colour 0, restriction to the next grid), phase
// after phase with a grid-wide barrier between them.  Loads bypass L1.
__global__ void __launch_bounds__(kBThreads, 2) batch_down_kernel(BatchTables T, int depth) {
  if (aborted(T)) return;
  phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 0, true);
  if (!grid_barrier(T)) return;
  phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 1, false);
  for (int s = 1; s < T.n1; ++s) {
    if (!grid_barrier(T)) return;
    phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 0, false);
    if (!grid_barrier(T)) return;
    phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 1, false);
  }
  if (!grid_barrier(T)) return;
  phase_residual_c0<true, 0, 8, kBatchMapCoop>(T, depth);
  if (!grid_barrier(T)) return;
  phase_restrict<true, 0, 8, kBatchMapCoop>(T, depth);
}

// Up-leg on the grids at `depth`: prolongation fused into the first
// post-smoothing half-sweep, then the rest of the post-smoothing.
__global__ void __launch_bounds__(kBThreads, 2) batch_up_kernel(BatchTables T, int depth) {
  if (aborted(T)) return;
  phase_prolong_sweep<true, 0, 8, kBatchMapCoop>(T, depth);
  if (!grid_barrier(T)) return;
  phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 1, false);
  for (int s = 1; s < T.n2; ++s) {
    if (!grid_barrier(T)) return;
    phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 0, false);
    if (!grid_barrier(T)) return;
    phase_sweep<true, 0, 8, kBatchMapCoop>(T, depth, 1, false);
  }
}

// ---- one launch per phase (grids with much work: no barrier, the
// registers of one phase only, programmatic dependent launch) -------------

enum BatchPhase { kPhZero = 0, kPhSweep = 1, kPhResidual = 2, kPhRestrict = 3, kPhProlong = 4, kPhProlongAdd = 5 };

template <int PH, int VF>
__global__ void __launch_bounds__(kBThreads, 2) batch_phase_kernel(BatchTables T, int depth, int colour) {
  pdl_enter();
  if (aborted(T)) return;
  if constexpr (PH == kPhZero) phase_sweep<false, VF, 1, kBatchMapPhase>(T, depth, 0, true);
  else if constexpr (PH == kPhSweep) phase_sweep<false, VF, 1, kBatchMapPhase>(T, depth, colour, false);
  else if constexpr (PH == kPhResidual) phase_residual_c0<false, VF, 1, kBatchMapPhase>(T, depth);
  else if constexpr (PH == kPhRestrict) phase_restrict<false, VF, 1, kBatchMapPhase>(T, depth);
  else if constexpr (PH == kPhProlongAdd) phase_prolong_add<false, VF, 1, kBatchMapPhase>(T, depth);
  else phase_prolong_sweep<false, VF, 1, kBatchMapPhase>(T, depth);
}

// Warp sum of a lane value (every lane of the warp calls it).
__device__ __forceinline__ double warp_total(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Refinement between anchors on the finest grids: r^ <- r^ - S e, d += e,
// and per-item partial sums of ||W r^||^2 (partial[item]).
template <int VF, int R>
__global__ void __launch_bounds__(kBThreads) batch_recur_kernel(BatchTables T) {
  if (aborted(T)) return;
  const int* pre0 = prefix(T, 0, kBkAll32, 0);
  walk<1>(T, 0, kBkAll32, vclass(VF), [&](int i, int it, int w, int lane) {
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels];
    const BatchInst& I = T.inst[i];
    const long node = (long)w * (32 / B.lpn) + lane / B.lpn;
    it = pre0[i] + w;   // the item's slot in the all-instance numbering (the control kernel's partials)
    float sq = 0.f;
    with_map<VF, R>(B.V, [&](auto m) {
      using M = decltype(m);
      sq = recur_item<M::V, M::S>(B.L, cview(B.x), B.f, I.d32, node, lane & (B.lpn - 1), B.lpn, I.wy2);
    });
    const double t = warp_total((double)sq);
    if (lane == 0) T.partial[it] = t;
  });
}

// Anchor, first half: x += d / sc (sc = the scale of the current right side),
// d = 0, on instances whose anchor is due.
__global__ void __launch_bounds__(kBThreads) batch_fold_kernel(BatchTables T) {
  if (aborted(T)) return;
  walk<1>(T, 0, kBkAll64, 0, [&](int i, int, int w, int lane) {
    const BatchInst& I = T.inst[i];
    if (I.state[kAnchor] == 0.0) return;
    const double a = I.state[kInvSc];
    const int N = I.L64.N, n = I.L64.n;
    const long node = (long)w * (32 / I.lpn64) + lane / I.lpn64;
    if (node >= (long)n * n) return;
    const int ln = lane & (I.lpn64 - 1);
    const size_t o = (size_t)node * N;
    for (int j = ln; j < N; j += I.lpn64) {
      I.x64.y[o + j] = fma(a, (double)I.d32.y[o + j], I.x64.y[o + j]);
      I.x64.p[o + j] = fma(a, (double)I.d32.p[o + j], I.x64.p[o + j]);
      I.d32.y[o + j] = 0.f;
      I.d32.p[o + j] = 0.f;
    }
    if (ln == 0) {
      I.x64.u[node] = fma(a, (double)I.d32.u[node], I.x64.u[node]);
      I.d32.u[node] = 0.f;
    }
  });
}

// Anchor, second half: r^ = sc (f - S x) in FP64 on the finest grid (written
// in FP32 as the next cycle's right side) with per-item partial sums of
// ||W r^||^2, on instances whose anchor is due.
__global__ void __launch_bounds__(kBThreads) batch_cast_kernel(BatchTables T) {
  if (aborted(T)) return;
  walk<1>(T, 0, kBkAll64, 0, [&](int i, int it, int w, int lane) {
    const BatchInst& I = T.inst[i];
    if (I.state[kAnchor] == 0.0) return;   // uniform over the warp
    const BatchLevel& B = T.lev[(size_t)i * kMaxLevels];
    const long node = (long)w * (32 / I.lpn64) + lane / I.lpn64;
    const double sc = I.state[kSc];
    float sq = 0.f;
    const int ln = lane & (I.lpn64 - 1);
    if (I.V64 == 2) sq = residual_cast_item<2, 2>(I.L64, cview(I.x64), I.f64, B.f, node, ln, I.lpn64, sc, I.wy2);
    else sq = residual_cast_item<1, 4>(I.L64, cview(I.x64), I.f64, B.f, node, ln, I.lpn64, sc, I.wy2);
    const double t = warp_total((double)sq);
    if (lane == 0) T.partial[it] = t;
  });
}

template <typename K>
int grid_cap(K kern) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBThreads, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return sms * per;
}

int g_caps[2] = {0, 0};
int g_sms = 0;
std::once_flag g_caps_once;

void init_caps() {
  std::call_once(g_caps_once, [] {
    g_caps[0] = grid_cap(batch_down_kernel);
    g_caps[1] = grid_cap(batch_up_kernel);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      g_sms = 0;
    (void)cudaGetLastError();
  });
}

cudaError_t launch_coop(void (*kern)(BatchTables, int), const BatchTables& T, int depth, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, T, depth);
  count_launches(1);
  return e;
}

}  // namespace

// which: 0 = down-leg kernel, 1 = up-leg kernel.  per_sm > 0 caps the CTAs
// per SM below what fits.
int batch_grid(int which, int per_sm) {
  init_caps();
  const int cap = g_caps[which & 1];
  if (per_sm > 0 && g_sms > 0) return std::min(cap, per_sm * g_sms);
  return cap;
}

cudaError_t launch_batch_down(const BatchTables& T, int depth, int grid, cudaStream_t s) {
  if (grid < 1 || grid > batch_grid(0, 0)) return cudaErrorInvalidValue;
  return launch_coop(batch_down_kernel, T, depth, grid, s);
}

cudaError_t launch_batch_up(const BatchTables& T, int depth, int grid, cudaStream_t s) {
  if (grid < 1 || grid > batch_grid(1, 0)) return cudaErrorInvalidValue;
  return launch_coop(batch_up_kernel, T, depth, grid, s);
}

namespace {
// CTAs for one warp per item of (depth, kind, class).
int class_grid(const BatchTables& T, int depth, int kind, int cls) {
  return std::max(1, std::min((T.items[depth][kind][cls] + kBWarps - 1) / kBWarps, 1 << 20));
}

// The items a phase walks.
constexpr int phase_kind(int ph, int colour) {
  return ph == kPhRestrict ? kBkCoarse : ph == kPhProlongAdd ? kBkAll32 : (ph == kPhSweep && colour) ? kBkColour1
                                                                                                      : kBkColour0;
}

// One launch per map class present at this depth (cls_mask bit c-1 = class
// c), each sized to that class's items.
template <int PH>
cudaError_t launch_phase(const BatchTables& T, int depth, int colour, cudaStream_t s) {
  const int mask = T.cls_mask[depth], kind = phase_kind(PH, colour);
  cudaError_t e = cudaSuccess;
  if (mask & 1)
    e = launch_k(batch_phase_kernel<PH, 4>, dim3(class_grid(T, depth, kind, 1)), dim3(kBThreads), 0, s, T, depth,
                 colour);
  if (e == cudaSuccess && (mask & 2))
    e = launch_k(batch_phase_kernel<PH, 2>, dim3(class_grid(T, depth, kind, 2)), dim3(kBThreads), 0, s, T, depth,
                 colour);
  if (e == cudaSuccess && (mask & 4))
    e = launch_k(batch_phase_kernel<PH, 1>, dim3(class_grid(T, depth, kind, 3)), dim3(kBThreads), 0, s, T, depth,
                 colour);
  count_launches(__builtin_popcount(mask));
  return e;
}
}  // namespace

cudaError_t launch_batch_down_phases(const BatchTables& T, int depth, cudaStream_t s) {
  cudaError_t e = launch_phase<kPhZero>(T, depth, 0, s);
  if (e == cudaSuccess) e = launch_phase<kPhSweep>(T, depth, 1, s);
  for (int k = 1; k < T.n1 && e == cudaSuccess; ++k) {
    e = launch_phase<kPhSweep>(T, depth, 0, s);
    if (e == cudaSuccess) e = launch_phase<kPhSweep>(T, depth, 1, s);
  }
  if (e == cudaSuccess) e = launch_phase<kPhResidual>(T, depth, 0, s);
  if (e == cudaSuccess) e = launch_phase<kPhRestrict>(T, depth, 0, s);
  return e;
}

cudaError_t launch_batch_up_phases(const BatchTables& T, int depth, cudaStream_t s) {
  // the prolongation in its own pass, then the plain post-smoothing (on the
  // grids with much work the fused sweep's extra coarse loads cost more)
  cudaError_t e = launch_phase<kPhProlongAdd>(T, depth, 0, s);
  if (e == cudaSuccess) e = launch_phase<kPhSweep>(T, depth, 0, s);
  if (e == cudaSuccess) e = launch_phase<kPhSweep>(T, depth, 1, s);
  for (int k = 1; k < T.n2 && e == cudaSuccess; ++k) {
    e = launch_phase<kPhSweep>(T, depth, 0, s);
    if (e == cudaSuccess) e = launch_phase<kPhSweep>(T, depth, 1, s);
  }
  return e;
}

namespace {
template <int R>
void recur_classes(const BatchTables& T, cudaStream_t s) {
  const int mask = T.cls_mask[0];
  if (mask & 1) batch_recur_kernel<4, R><<<class_grid(T, 0, kBkAll32, 1), kBThreads, 0, s>>>(T);
  if (mask & 2) batch_recur_kernel<2, R><<<class_grid(T, 0, kBkAll32, 2), kBThreads, 0, s>>>(T);
  if (mask & 4) batch_recur_kernel<1, R><<<class_grid(T, 0, kBkAll32, 3), kBThreads, 0, s>>>(T);
  count_launches(__builtin_popcount(mask));
}
}  // namespace

// The finest grids' maps follow the rule T.maps[0].
cudaError_t launch_batch_recur(const BatchTables& T, cudaStream_t s) {
  if (T.maps[0] == kBatchMapPhase) recur_classes<kBatchMapPhase>(T, s);
  else if (T.maps[0] == kBatchMapCoop) recur_classes<kBatchMapCoop>(T, s);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_batch_anchor(const BatchTables& T, cudaStream_t s) {
  const int grid = class_grid(T, 0, kBkAll64, 0);
  batch_fold_kernel<<<grid, kBThreads, 0, s>>>(T);
  batch_cast_kernel<<<grid, kBThreads, 0, s>>>(T);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace cmg
