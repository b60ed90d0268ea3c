// Node-sample kernels of the collective multigrid cycle:
//   residual r = f - S x (Eq. (2) blocks), red-black collective Gauss-Seidel
//   half-sweep (reduced node systems Eq. (12) solved by Eq. (13)), damped
//   collective Jacobi update (Eq. (11)), restriction P^T and prolongation P
//   (Algorithm 1).
//
// One kernel per step; the per-node work is in cmg_items.cuh.
// Layout: node arrays [n*n][ld] with the sample index fastest.  The lpn
// lanes of a node group read that node's samples as contiguous V-element
// vectors (coalesced 128-bit loads); neighbour rows are re-read from L2 by
// the CTAs of adjacent rows, which run close together in launch order.
// The sum over samples in the control row (u) is a shuffle reduction over
// the node group, carried in the cycle's precision (FP32 or FP64).
#include <cstdlib>

#include "cmg_items.cuh"

namespace cmg {

namespace {

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) residual_kernel(LevelView<T> L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r,
                                                          int lpn, T wy) {
  pdl_enter();
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  residual_item<T, V, SPL, false>(L, x, f, r, node, threadIdx.x & (lpn - 1), lpn, wy);
}

// r = f - S x at the colour-0 nodes only (the g-th node of colour 0).
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) residual_c0_kernel(LevelView<T> L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r,
                                                             int lpn) {
  pdl_enter();
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  long node = (long)L.n * L.n;   // out of range: the item does nothing but its shuffles
  if (g < colour_count(L.n, 0)) {
    int iy, ix;
    colour_node(g, L.n, 0, iy, ix);
    node = (long)iy * L.n + ix;
  }
  residual_item<T, V, SPL, false>(L, x, f, r, node, threadIdx.x & (lpn - 1), lpn, T(1));
}

// The widest FP32 variants (16 samples per lane) at more CTAs per SM than
// their registers would allow: more warps in flight to cover the load latency
// (a few spilled registers cost less).
template <typename T, int V, int SPL>
constexpr int wide_ctas(int k) { return (sizeof(T) == 4 && V * SPL == 16) ? k : 1; }

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock, wide_ctas<T, V, SPL>(3))
    rbgs_half_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> f, int colour, int lpn) {
  pdl_enter();
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  rbgs_item<T, V, SPL, false>(L, x, f, colour, g, threadIdx.x & (lpn - 1), lpn);
}

// Colour-0 half-sweep from a zero iterate (see rbgs_item, ZG).
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock, wide_ctas<T, V, SPL>(3))
    rbgs_zero_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> f, int lpn) {
  pdl_enter();
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  rbgs_item<T, V, SPL, false, false, true>(L, x, f, 0, g, threadIdx.x & (lpn - 1), lpn);
}

// Colour-0 half-sweep that reads its neighbours as x + P e (prolongation of
// the coarse correction e fused in; see rbgs_item).
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) rbgs_prolong_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> f, Vec3c<T> e,
                                                              int nc, int lpn) {
  pdl_enter();
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  rbgs_item<T, V, SPL, false, true>(L, x, f, 0, g, threadIdx.x & (lpn - 1), lpn, e, nc);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) jacobi_update_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> r,
                                                               double theta, int lpn) {
  pdl_enter();
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  jacobi_item<T, V, SPL, false>(L, x, r, theta, node, threadIdx.x & (lpn - 1), lpn);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) restrict_kernel(int nf, int N, Vec3c<T> r, Vec3<T> cv, Vec3<T> zx,
                                                          int lpn, int colour0) {
  pdl_enter();
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  restrict_item<T, V, SPL, false>(nf, N, r, cv, zx, node, threadIdx.x & (lpn - 1), lpn, colour0 != 0);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) prolong_add_kernel(int nf, int N, Vec3c<T> e, Vec3<T> x, int lpn,
                                                             CtlBox ctl) {
  pdl_enter();
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  prolong_item<T, V, SPL, false>(nf, N, e, x, node, threadIdx.x & (lpn - 1), lpn, ctl);
}

// One pass of FP64 refinement: r32 = s (f - S x) and per-CTA partial sums
// of ||W r32||^2 (squares in FP32, CTA sum in FP64).
template <int V, int SPL>
__global__ void __launch_bounds__(kBlock) residual_cast_kernel(LevelView<double> L, Vec3c<double> x,
                                                              Vec3c<double> f, Vec3<float> r, int lpn, double s,
                                                              const double* __restrict__ sdev, float wy2,
                                                              double* __restrict__ partial,
                                                              const double* __restrict__ gate) {
  pdl_enter();
  __shared__ double sh[kBlock / 32];
  if (gate && *gate == 0.0) return;   // refinement anchor not due (residual replacement)
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  const double sc = sdev ? *sdev : s;
  double v = (double)residual_cast_item<V, SPL>(L, x, f, r, node, threadIdx.x & (lpn - 1), lpn, sc, wy2);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// FP32 refinement between FP64 anchors (residual replacement): the scaled
// residual r (the cycle's right side) is updated in place, r <- r - S e (A e
// from neighbour differences, see residual_item), the
// running correction d += e, and per-CTA partial sums of ||W r||^2 are
// written (squares in FP32, CTA sum in FP64).  Each lane reads its own f
// entries before writing r at the same place, so the update in place is safe.
template <int V, int SPL>
__global__ void __launch_bounds__(kBlock, wide_ctas<float, V, SPL>(3)) recur_kernel(LevelView<float> L, Vec3c<float> e, Vec3<float> r,
                                                       Vec3<float> d, int lpn, float wy2,
                                                       double* __restrict__ partial) {
  pdl_enter();
  __shared__ double sh[kBlock / 32];
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  const int lane = threadIdx.x & (lpn - 1);
  const float sq = recur_item<V, SPL>(L, e, r, d, node, lane, lpn, wy2);
  double v = (double)sq;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// Anchor of residual replacement: x += a d (a = *adev) and d = 0, when
// *gate is nonzero.  The y and p blocks move as pairs (16-byte FP64 and
// 8-byte FP32 vectors; the blocks start 16-byte aligned), one odd tail
// element and the u block singly.
__global__ void fold_kernel(const double* __restrict__ adev, const double* __restrict__ gate, Vec3<float> d,
                            Vec3<double> x, size_t ny, size_t nu) {
  pdl_enter();
  if (*gate == 0.0) return;
  const double a = *adev;
  const size_t np = ny / 2;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (size_t i = t0; i < 2 * np; i += stride) {
    const bool isp = i >= np;
    const size_t k = isp ? i - np : i;
    double2* xv = reinterpret_cast<double2*>(isp ? x.p : x.y) + k;
    float2* dv = reinterpret_cast<float2*>(isp ? d.p : d.y) + k;
    double2 xx = *xv;
    const float2 dd = *dv;
    xx.x = fma(a, (double)dd.x, xx.x);
    xx.y = fma(a, (double)dd.y, xx.y);
    *xv = xx;
    *dv = make_float2(0.f, 0.f);
  }
  for (size_t i = t0; i < nu; i += stride) {
    x.u[i] = fma(a, (double)d.u[i], x.u[i]);
    d.u[i] = 0.f;
  }
  if (t0 == 0 && (ny & 1)) {
    const size_t k = ny - 1;
    x.y[k] = fma(a, (double)d.y[k], x.y[k]);
    d.y[k] = 0.f;
    x.p[k] = fma(a, (double)d.p[k], x.p[k]);
    d.p[k] = 0.f;
  }
}

// (y, u, p) = 0 for an FP32 level vector (a kernel, so that it can be a
// programmatic dependent of the kernels around it).
__global__ void zero3_kernel(Vec3<float> v, size_t ny, size_t nu) {
  pdl_enter();
  const size_t total = 2 * ny + nu;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    if (i < ny) v.y[i] = 0.f;
    else if (i < ny + nu) v.u[i - ny] = 0.f;
    else v.p[i - ny - nu] = 0.f;
  }
}

// x += a * e for the three blocks (FP64 iterate, FP32 correction); a read
// from adev when given.
__global__ void axpy3_kernel(double a0, const double* __restrict__ adev, Vec3c<float> e, Vec3<double> x, size_t ny,
                             size_t nu) {
  pdl_enter();
  const double a = adev ? *adev : a0;
  const size_t total = 2 * ny + nu;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    if (i < ny) x.y[i] = fma(a, (double)e.y[i], x.y[i]);
    else if (i < ny + nu) x.u[i - ny] = fma(a, (double)e.u[i - ny], x.u[i - ny]);
    else x.p[i - ny - nu] = fma(a, (double)e.p[i - ny - nu], x.p[i - ny - nu]);
  }
}

inline unsigned grid_for(long groups, int lpn) {
  const long threads = groups * lpn;
  return (unsigned)((threads + kBlock - 1) / kBlock);
}

}  // namespace

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("CMG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

SampleMap choose_map(int N, int elem_bytes, long items, int spl_target) {
  SampleMap m;
  if ((spl_target & kTuneWide) && elem_bytes == 4 && wide_supported(N)) {
    m.V = 2;
    m.spl = 1;
    m.lpn = 1;
    while (m.lpn < N / 2) m.lpn <<= 1;
    return m;
  }
  const int vmax = 16 / elem_bytes;     // 2 for double, 4 for float
  m.V = (N % vmax == 0) ? vmax : 1;
  const int chunks = (N + m.V - 1) / m.V;
  int target = 4;
  while (target > 1 && items * chunks / target < kMinLanes) target >>= 1;
  if ((spl_target & 15) > 0) target = spl_target & 15;   // the staged and wide flags are not part of it
  const int want = (chunks + target - 1) / target;   // lanes needed at `target` chunks each
  int lpn = 1;
  while (lpn < want && lpn < 32) lpn <<= 1;
  m.lpn = lpn;
  int spl = (chunks + lpn - 1) / lpn;
  int p2 = 1;
  while (p2 < spl) p2 <<= 1;
  m.spl = p2;
  return m;
}



template <typename T>
cudaError_t launch_residual(const LevelView<T>& L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r, cudaStream_t st, double wy) {
  const SampleMap m = choose_map(L.N, sizeof(T), (long)L.n * L.n, L.spl_target);
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(residual_kernel<T, V, SPL>, grid, kBlock, 0, st, L, x, f, r, m.lpn, (T)wy)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_c0(const LevelView<T>& L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r, cudaStream_t st) {
  const long groups = colour_count(L.n, 0);
  const SampleMap m = choose_map(L.N, sizeof(T), groups, L.spl_target);
  const unsigned grid = grid_for(groups, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(residual_c0_kernel<T, V, SPL>, grid, kBlock, 0, st, L, x, f, r, m.lpn)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_rbgs_half(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, int colour, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, sizeof(T), colour_count(L.n, colour), L.spl_target);
  if constexpr (sizeof(T) == 4) {
    if (L.spl_target & kTuneStaged) {
      const cudaError_t e = launch_rbgs_half_staged(L, x, f, colour, m, st);
      if (e != cudaErrorNotSupported) return e;
    }
    if (L.spl_target & kTuneTma) {
      const cudaError_t e = launch_rbgs_half_tma(L, x, f, colour, m, st);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  const unsigned grid = grid_for(colour_count(L.n, colour), m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(rbgs_half_kernel<T, V, SPL>, grid, kBlock, 0, st, L, x, f, colour, m.lpn)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_rbgs_zero(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, cudaStream_t st) {
  const long groups = colour_count(L.n, 0);
  const SampleMap m = choose_map(L.N, sizeof(T), groups, L.spl_target);
  const unsigned grid = grid_for(groups, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(rbgs_zero_kernel<T, V, SPL>, grid, kBlock, 0, st, L, x, f, m.lpn)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_rbgs_prolong(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, Vec3c<T> e, int nc, cudaStream_t st) {
  const long groups = colour_count(L.n, 0);
  const SampleMap m = choose_map(L.N, sizeof(T), groups, L.spl_target);
  const unsigned grid = grid_for(groups, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(rbgs_prolong_kernel<T, V, SPL>, grid, kBlock, 0, st, L, x, f, e, nc, m.lpn)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi_update(const LevelView<T>& L, Vec3<T> x, Vec3c<T> r, double theta, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, sizeof(T), (long)L.n * L.n, L.spl_target);
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(jacobi_update_kernel<T, V, SPL>, grid, kBlock, 0, st, L, x, r, theta, m.lpn)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(int nf, int N, Vec3c<T> r, Vec3<T> c, cudaStream_t st, Vec3<T> zx, int colour0) {
  const int nc = (nf - 1) / 2;
  const SampleMap m = choose_map(N, sizeof(T), (long)nc * nc);
  const unsigned grid = grid_for((long)nc * nc, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(restrict_kernel<T, V, SPL>, grid, kBlock, 0, st, nf, N, r, c, zx, m.lpn, colour0)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(int nf, int N, Vec3c<T> e, Vec3<T> x, cudaStream_t st, CtlBox ctl) {
  const SampleMap m = choose_map(N, sizeof(T), (long)nf * nf);
  const unsigned grid = grid_for((long)nf * nf, m.lpn);
  cudaError_t e_ = cudaSuccess;
  CMG_DISPATCH(T, m, (e_ = launch_k(prolong_add_kernel<T, V, SPL>, grid, kBlock, 0, st, nf, N, e, x, m.lpn, ctl)));
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

int launch_residual_cast(const LevelView<double>& L, Vec3c<double> x, Vec3c<double> f, Vec3<float> r, double s,
                         const double* sdev, double wy, double* partial, int max_partials, cudaStream_t st,
                         const double* gate) {
  const SampleMap m = choose_map(L.N, 8, (long)L.n * L.n);
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  if ((int)grid > max_partials) return -1;
  const float wy2 = (float)(wy * wy);
  using T = double;
  auto go = [&]() -> cudaError_t {
    cudaError_t e_ = cudaSuccess;
    CMG_DISPATCH(T, m, (e_ = launch_k(residual_cast_kernel<V, SPL>, grid, kBlock, 0, st, L, x, f, r, m.lpn, s, sdev,
                                                   wy2, partial, gate)));
    return e_ != cudaSuccess ? e_ : cudaGetLastError();
  };
  if (go() != cudaSuccess) return -1;
  count_launches(1);
  return (int)grid;
}

int launch_recur(const LevelView<float>& L, Vec3c<float> e, Vec3<float> r, Vec3<float> d, double wy, double* partial,
                 int max_partials, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, 4, (long)L.n * L.n, L.spl_target);
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  if ((int)grid > max_partials) return -1;
  const float wy2 = (float)(wy * wy);
  using T = float;
  auto go = [&]() -> cudaError_t {
    cudaError_t e_ = cudaSuccess;
    CMG_DISPATCH(T, m, (e_ = launch_k(recur_kernel<V, SPL>, grid, kBlock, 0, st, L, e, r, d, m.lpn, wy2, partial)));
    return e_ != cudaSuccess ? e_ : cudaGetLastError();
  };
  if (go() != cudaSuccess) return -1;
  count_launches(1);
  return (int)grid;
}

cudaError_t launch_fold(const double* adev, const double* gate, Vec3<float> d, Vec3<double> x, size_t ny, size_t nu,
                        cudaStream_t st) {
  const size_t total = ny + nu;
  size_t blocks = (total + kBlock - 1) / kBlock;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const cudaError_t e_ = launch_k(fold_kernel, dim3((unsigned)blocks), dim3(kBlock), 0, st, adev, gate, d, x, ny, nu);
  if (e_ != cudaSuccess) return e_;
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

cudaError_t launch_zero3(Vec3<float> v, size_t ny, size_t nu, cudaStream_t st) {
  const size_t total = 2 * ny + nu;
  size_t blocks = (total + kBlock - 1) / kBlock;
  if (blocks > 152 * 8) blocks = 152 * 8;
  const cudaError_t e_ = launch_k(zero3_kernel, dim3((unsigned)blocks), dim3(kBlock), 0, st, v, ny, nu);
  count_launches(1);
  return e_;
}

cudaError_t launch_axpy3(double a, const double* adev, Vec3c<float> e, Vec3<double> x, size_t ny, size_t nu,
                         cudaStream_t st) {
  const size_t total = 2 * ny + nu;
  size_t blocks = (total + kBlock - 1) / kBlock;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const cudaError_t e_ = launch_k(axpy3_kernel, dim3((unsigned)blocks), dim3(kBlock), 0, st, a, adev, e, x, ny, nu);
  if (e_ != cudaSuccess) return e_;
  count_launches(1);
  return e_ != cudaSuccess ? e_ : cudaGetLastError();
}

#define CMG_INST(T)                                                                                   \
  template cudaError_t launch_residual<T>(const LevelView<T>&, Vec3c<T>, Vec3c<T>, Vec3<T>, cudaStream_t, double); \
  template cudaError_t launch_rbgs_half<T>(const LevelView<T>&, Vec3<T>, Vec3c<T>, int, cudaStream_t);    \
  template cudaError_t launch_rbgs_zero<T>(const LevelView<T>&, Vec3<T>, Vec3c<T>, cudaStream_t);         \
  template cudaError_t launch_jacobi_update<T>(const LevelView<T>&, Vec3<T>, Vec3c<T>, double, cudaStream_t); \
  template cudaError_t launch_restrict<T>(int, int, Vec3c<T>, Vec3<T>, cudaStream_t, Vec3<T>, int);         \
  template cudaError_t launch_residual_c0<T>(const LevelView<T>&, Vec3c<T>, Vec3c<T>, Vec3<T>, cudaStream_t);       \
  template cudaError_t launch_rbgs_prolong<T>(const LevelView<T>&, Vec3<T>, Vec3c<T>, Vec3c<T>, int, cudaStream_t);                     \
  template cudaError_t launch_prolong_add<T>(int, int, Vec3c<T>, Vec3<T>, cudaStream_t, CtlBox);

CMG_INST(double)
CMG_INST(float)

}  // namespace cmg
