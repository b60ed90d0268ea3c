// FP64 vector kernels for norms, the Krylov outer loop and precision
// conversion.  Reductions use a fixed grid (kRedBlocks partials) and a
// fixed-order final sum, so results do not depend on scheduling.
#include "cmg_common.cuh"

namespace cmg {

namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

__global__ void __launch_bounds__(kRedThreads) sumsq_kernel(const double* __restrict__ a, size_t n,
                                                            double* __restrict__ partial, int accumulate,
                                                            double w2) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = a[i];
    s = fma(v, v, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = accumulate ? partial[blockIdx.x] + w2 * s : w2 * s;
}

__global__ void finish_sum_kernel(const double* __restrict__ partial, int count, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// Dots of up to 8 basis vectors with w per pass: w is read once per group.
constexpr int kDotGroup = 8;
__global__ void __launch_bounds__(kRedThreads) mdot_kernel(const double* __restrict__ V, size_t stride, int nv,
                                                           const double* __restrict__ w, size_t n,
                                                           double* __restrict__ partial) {
  __shared__ double sh[32];
  const int g0 = blockIdx.y * kDotGroup;
  const int cnt = min(kDotGroup, nv - g0);
  double acc[kDotGroup];
#pragma unroll
  for (int k = 0; k < kDotGroup; ++k) acc[k] = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < kDotGroup; ++k)
      if (k < cnt) acc[k] = fma(V[(size_t)(g0 + k) * stride + i], wi, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < kDotGroup; ++k) {
    if (k < cnt) {
      const double s = block_sum(acc[k], sh);
      if (threadIdx.x == 0) partial[(size_t)(g0 + k) * gridDim.x + blockIdx.x] = s;
    }
  }
}

__global__ void mdot_finish_kernel(const double* __restrict__ partial, int count, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) s += partial[(size_t)blockIdx.x * count + i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads) maxpy_kernel(const double* __restrict__ V, size_t stride, int nv,
                                                            const double* __restrict__ coef, double sign,
                                                            double* __restrict__ w, size_t n) {
  __shared__ double cs[128];
  for (int k = threadIdx.x; k < nv; k += blockDim.x) cs[k] = sign * coef[k];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int k = 0; k < nv; ++k) acc = fma(cs[k], V[(size_t)k * stride + i], acc);
    w[i] = acc;
  }
}

__global__ void scale_by_kernel(const double* __restrict__ x, const double* __restrict__ den,
                                double* __restrict__ y, size_t n) {
  const double s = 1.0 / sqrt(*den);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}

template <typename Tx, typename Ty>
__global__ void axpy_kernel(double a, const Tx* __restrict__ x, Ty* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (Ty)((double)y[i] + a * (double)x[i]);
}

template <typename Tx, typename Ty>
__global__ void scale_cast_kernel(double a, const Tx* __restrict__ x, Ty* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (Ty)(a * (double)x[i]);
}

__global__ void rhs_kernel(int n, int N, double h, const double* __restrict__ yd, const double* __restrict__ fsrc,
                           double* __restrict__ fy, double* __restrict__ fu, double* __restrict__ fp) {
  const size_t total = (size_t)n * n * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t node = i / N;
    fy[i] = h * h / N * yd[node];
    fp[i] = fsrc ? h * h * fsrc[node] : 0.0;
    if (i % N == 0) fu[node] = 0.0;
  }
}

inline unsigned stream_blocks(size_t n) {
  const size_t b = (n + kRedThreads - 1) / kRedThreads;
  return (unsigned)(b < 152 * 16 ? (b == 0 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t launch_sumsq(const double* a, size_t n, double* partial, int accumulate, double w2, cudaStream_t s) {
  sumsq_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a, n, partial, accumulate, w2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_finish_sum(const double* partial, int count, double* out, cudaStream_t s) {
  finish_sum_kernel<<<1, kRedThreads, 0, s>>>(partial, count, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mdot(const double* V, size_t stride, int nv, const double* w, size_t n, double* partial,
                        double* out, cudaStream_t s) {
  dim3 grid(kRedBlocks, (nv + kDotGroup - 1) / kDotGroup);
  mdot_kernel<<<grid, kRedThreads, 0, s>>>(V, stride, nv, w, n, partial);
  mdot_finish_kernel<<<nv, kRedThreads, 0, s>>>(partial, kRedBlocks, out);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_maxpy(const double* V, size_t stride, int nv, const double* coef, double sign, double* w,
                         size_t n, cudaStream_t s) {
  if (nv > 128) return cudaErrorInvalidValue;
  maxpy_kernel<<<stream_blocks(n), kRedThreads, 0, s>>>(V, stride, nv, coef, sign, w, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_by(const double* x, const double* den, double* y, size_t n, cudaStream_t s) {
  scale_by_kernel<<<stream_blocks(n), kRedThreads, 0, s>>>(x, den, y, n);
  count_launches(1);
  return cudaGetLastError();
}

template <typename Tx, typename Ty>
cudaError_t launch_axpy(double a, const Tx* x, Ty* y, size_t n, cudaStream_t s) {
  axpy_kernel<Tx, Ty><<<stream_blocks(n), kRedThreads, 0, s>>>(a, x, y, n);
  count_launches(1);
  return cudaGetLastError();
}

template <typename Tx, typename Ty>
cudaError_t launch_scale_cast(double a, const Tx* x, Ty* y, size_t n, cudaStream_t s) {
  scale_cast_kernel<Tx, Ty><<<stream_blocks(n), kRedThreads, 0, s>>>(a, x, y, n);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rhs(int n, int N, double h, const double* yd, const double* fsrc, double* fy, double* fu,
                       double* fp, cudaStream_t s) {
  rhs_kernel<<<stream_blocks((size_t)n * n * N), kRedThreads, 0, s>>>(n, N, h, yd, fsrc, fy, fu, fp);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_axpy<double, double>(double, const double*, double*, size_t, cudaStream_t);
template cudaError_t launch_axpy<float, double>(double, const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_scale_cast<double, float>(double, const double*, float*, size_t, cudaStream_t);
template cudaError_t launch_scale_cast<float, double>(double, const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_scale_cast<double, double>(double, const double*, double*, size_t, cudaStream_t);

}  // namespace cmg
