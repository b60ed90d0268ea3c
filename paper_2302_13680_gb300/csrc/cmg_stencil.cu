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
// the node group, carried in FP64 in both precisions.
#include "cmg_items.cuh"

namespace cmg {

namespace {

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) residual_kernel(LevelView<T> L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r,
                                                          int lpn, T wy) {
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  residual_item<T, V, SPL, false>(L, x, f, r, node, threadIdx.x & (lpn - 1), lpn, wy);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) rbgs_half_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> f, int colour,
                                                           int lpn) {
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  rbgs_item<T, V, SPL, false>(L, x, f, colour, g, threadIdx.x & (lpn - 1), lpn);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) jacobi_update_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> r,
                                                               double theta, int lpn) {
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  jacobi_item<T, V, SPL, false>(L, x, r, theta, node, threadIdx.x & (lpn - 1), lpn);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) restrict_kernel(int nf, int N, Vec3c<T> r, Vec3<T> cv, int lpn) {
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  restrict_item<T, V, SPL, false>(nf, N, r, cv, Vec3<T>{nullptr, nullptr, nullptr}, node, threadIdx.x & (lpn - 1),
                                  lpn);
}

template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) prolong_add_kernel(int nf, int N, Vec3c<T> e, Vec3<T> x, int lpn) {
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  prolong_item<T, V, SPL, false>(nf, N, e, x, node, threadIdx.x & (lpn - 1), lpn);
}

inline unsigned grid_for(long groups, int lpn) {
  const long threads = groups * lpn;
  return (unsigned)((threads + kBlock - 1) / kBlock);
}

}  // namespace

SampleMap choose_map(int N, int elem_bytes, long items) {
  SampleMap m;
  const int vmax = 16 / elem_bytes;     // 2 for double, 4 for float
  m.V = (N % vmax == 0) ? vmax : 1;
  const int chunks = (N + m.V - 1) / m.V;
  int target = 4;
  while (target > 1 && items * chunks / target < kMinLanes) target >>= 1;
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
  const SampleMap m = choose_map(L.N, sizeof(T), (long)L.n * L.n);
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  CMG_DISPATCH(T, m, (residual_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(L, x, f, r, m.lpn, (T)wy)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rbgs_half(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, int colour, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, sizeof(T), colour_count(L.n, colour));
  const unsigned grid = grid_for(colour_count(L.n, colour), m.lpn);
  CMG_DISPATCH(T, m, (rbgs_half_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(L, x, f, colour, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi_update(const LevelView<T>& L, Vec3<T> x, Vec3c<T> r, double theta, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, sizeof(T), (long)L.n * L.n);
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  CMG_DISPATCH(T, m, (jacobi_update_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(L, x, r, theta, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(int nf, int N, Vec3c<T> r, Vec3<T> c, cudaStream_t st) {
  const int nc = (nf - 1) / 2;
  const SampleMap m = choose_map(N, sizeof(T), (long)nc * nc);
  const unsigned grid = grid_for((long)nc * nc, m.lpn);
  CMG_DISPATCH(T, m, (restrict_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(nf, N, r, c, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(int nf, int N, Vec3c<T> e, Vec3<T> x, cudaStream_t st) {
  const SampleMap m = choose_map(N, sizeof(T), (long)nf * nf);
  const unsigned grid = grid_for((long)nf * nf, m.lpn);
  CMG_DISPATCH(T, m, (prolong_add_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(nf, N, e, x, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

#define CMG_INST(T)                                                                                   \
  template cudaError_t launch_residual<T>(const LevelView<T>&, Vec3c<T>, Vec3c<T>, Vec3<T>, cudaStream_t, double); \
  template cudaError_t launch_rbgs_half<T>(const LevelView<T>&, Vec3<T>, Vec3c<T>, int, cudaStream_t);    \
  template cudaError_t launch_jacobi_update<T>(const LevelView<T>&, Vec3<T>, Vec3c<T>, double, cudaStream_t); \
  template cudaError_t launch_restrict<T>(int, int, Vec3c<T>, Vec3<T>, cudaStream_t);                     \
  template cudaError_t launch_prolong_add<T>(int, int, Vec3c<T>, Vec3<T>, cudaStream_t);

CMG_INST(double)
CMG_INST(float)

}  // namespace cmg
