// Per-node operations of the globalised semismooth Newton method for the
// L1 + box constrained problem (Sec. 4, Algorithm 2).  In the symmetric
// scaling used here the paper's adjoint is N times ours, so its E[p] is the
// plain sum of our adjoint over the samples.
#include "cmg_common.cuh"

namespace cmg {

namespace {

constexpr int kSsnBlock = 256;

// out[i] = sum_j p[i][j]: one warp per node, lanes over samples, then a
// fixed-order shuffle reduction.
__global__ void sum_samples_kernel(long nodes, int N, const double* __restrict__ p, double* __restrict__ out) {
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (node >= nodes) return;   // whole warp
  double s = 0.0;
  for (int j = lane; j < N; j += 32) s += p[(size_t)node * N + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[node] = s;
}

__device__ __forceinline__ double ssn_map(double u, double t, double nu, double beta, double a, double b) {
  // F(u) = u - (max(0, t - beta) + min(0, t + beta) - max(0, t - beta - nu b) - min(0, t + beta - nu a)) / nu
  const double v = fmax(0.0, t - beta) + fmin(0.0, t + beta) - fmax(0.0, t - beta - nu * b) -
                   fmin(0.0, t + beta - nu * a);
  return u - v / nu;
}

// F at (u + g du, Tu + g Tdp) (du, Tdp may be null: g = 0), the active-set
// indicator I+ u I- there (chi, may be null) and per-CTA partial sums of F^2
// (fixed order).
__global__ void __launch_bounds__(kSsnBlock) ssn_map_kernel(long nodes, const double* __restrict__ u,
                                                            const double* __restrict__ du,
                                                            const double* __restrict__ Tu,
                                                            const double* __restrict__ Tdp, double g, double nu,
                                                            double beta, double a, double b, double* __restrict__ F,
                                                            float* __restrict__ chi, double* __restrict__ partial) {
  __shared__ double sh[kSsnBlock / 32];
  double sq = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += (long)gridDim.x * blockDim.x) {
    const double ui = du ? fma(g, du[i], u[i]) : u[i];
    const double ti = Tdp ? fma(g, Tdp[i], Tu[i]) : Tu[i];
    const double fi = ssn_map(ui, ti, nu, beta, a, b);
    if (F) F[i] = fi;
    if (chi) {
      const bool ip = ti - beta >= 0.0 && ti - beta <= nu * b;
      const bool im = ti + beta <= 0.0 && ti + beta >= nu * a;
      chi[i] = (ip || im) ? 1.f : 0.f;
    }
    sq = fma(fi, fi, sq);
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSsnBlock / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void axpy64_kernel(long n, double g, const double* __restrict__ x, double* __restrict__ y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = fma(g, x[i], y[i]);
}

__global__ void scale64_kernel(long n, double s, const double* __restrict__ x, double* __restrict__ y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] = s * x[i];
}

// fy[i][j] = c yd[i] (the state rows' right side (h^2/N) y_d for every sample)
__global__ void spread_kernel(long nodes, int N, double c, const double* __restrict__ yd, double* __restrict__ fy) {
  const long total = nodes * N;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x)
    fy[t] = c * yd[t / N];
}

__global__ void scale32_kernel(long n, float sc, const float* __restrict__ x, float* __restrict__ y) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) y[i] = sc * x[i];
}

__global__ void fill32_kernel(long n, float v, float* __restrict__ x) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = v;
}

// coarse[J][I] = fine[2J+1][2I+1]: the value at the coinciding fine node
__global__ void inject32_kernel(int nf, const float* __restrict__ fine, float* __restrict__ coarse) {
  const int nc = (nf - 1) / 2;
  const long total = (long)nc * nc;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int J = (int)(t / nc), I = (int)(t - (long)J * nc);
    coarse[t] = fine[(size_t)(2 * J + 1) * nf + 2 * I + 1];
  }
}

inline unsigned grid_of(long n) {
  long g = (n + kSsnBlock - 1) / kSsnBlock;
  if (g > 152 * 8) g = 152 * 8;
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_sum_samples(long nodes, int N, const double* p, double* out, cudaStream_t s) {
  const long threads = nodes * 32;
  sum_samples_kernel<<<(unsigned)((threads + kSsnBlock - 1) / kSsnBlock), kSsnBlock, 0, s>>>(nodes, N, p, out);
  count_launches(1);
  return cudaGetLastError();
}

int launch_ssn_map(long nodes, const double* u, const double* du, const double* Tu, const double* Tdp, double g,
                   double nu, double beta, double a, double b, double* F, float* chi, double* partial,
                   int max_partials, cudaStream_t s) {
  unsigned grid = grid_of(nodes);
  if ((int)grid > max_partials) grid = (unsigned)max_partials;
  ssn_map_kernel<<<grid, kSsnBlock, 0, s>>>(nodes, u, du, Tu, Tdp, g, nu, beta, a, b, F, chi, partial);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? (int)grid : -1;
}

cudaError_t launch_axpy64(long n, double g, const double* x, double* y, cudaStream_t s) {
  axpy64_kernel<<<grid_of(n), kSsnBlock, 0, s>>>(n, g, x, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale64(long n, double sc, const double* x, double* y, cudaStream_t s) {
  scale64_kernel<<<grid_of(n), kSsnBlock, 0, s>>>(n, sc, x, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_spread(long nodes, int N, double c, const double* yd, double* fy, cudaStream_t s) {
  spread_kernel<<<grid_of(nodes * N), kSsnBlock, 0, s>>>(nodes, N, c, yd, fy);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale32(long n, float sc, const float* x, float* y, cudaStream_t s) {
  scale32_kernel<<<grid_of(n), kSsnBlock, 0, s>>>(n, sc, x, y);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill32(long n, float v, float* x, cudaStream_t s) {
  fill32_kernel<<<grid_of(n), kSsnBlock, 0, s>>>(n, v, x);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_inject32(int nf, const float* fine, float* coarse, cudaStream_t s) {
  const long nc = (nf - 1) / 2;
  inject32_kernel<<<grid_of(nc * nc), kSsnBlock, 0, s>>>(nf, fine, coarse);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cmg
