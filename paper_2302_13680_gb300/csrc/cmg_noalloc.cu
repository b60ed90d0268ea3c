// Allocation-free norm of a full-space vector.
//
// Some callers cannot call cudaMalloc at the point where they need a norm:
// code that runs while another component owns every device allocation
// (an embedding application with its own memory pool or a fixed memory
// budget), or a loop that must not allocate between its steps.  For them
// cmg_norm_noalloc computes the same quantity as cmg_norm without a
// handle and without allocating: its per-block partial sums live in a
// file-scope device array that every GPU loading this library holds until
// the process exits.
//
// The array's name is only a host-side stand-in in host code, so the
// device address is looked up once per device with cudaGetSymbolAddress
// (on the first call made while that device is current) and then passed
// to the kernels.
#include <cmath>
#include <mutex>

#include "cmg_common.cuh"

namespace {

constexpr int kNAThreads = 256;
constexpr int kNAPerThread = 16;
constexpr long long kNAPerBlock = (long long)kNAThreads * kNAPerThread;   // 4096 elements per partial
constexpr int kNAMaxBlocks = 65536;                                       // partials per segment
constexpr long long kNAMaxLen = (long long)kNAMaxBlocks * kNAPerBlock;   // 2^28 elements per segment
constexpr int kNAMaxDevices = 64;

// Partial sums of the three segments (y, u, p): 3 x 65536 doubles = 1.5 MiB.
static __device__ __align__(256) double g_noalloc_partial[3 * kNAMaxBlocks];

std::mutex g_na_mutex;
double* g_na_scratch[kNAMaxDevices] = {};

// Block b writes w2 * sum of squares of a[b*4096, (b+1)*4096) to partial[b].
__global__ void __launch_bounds__(kNAThreads) na_sumsq_kernel(const double* __restrict__ a, long long n,
                                                             double w2, double* __restrict__ partial) {
  __shared__ double sh[kNAThreads / 32];
  const long long base = (long long)blockIdx.x * kNAPerBlock;
  double s = 0.0;
#pragma unroll 4
  for (int k = 0; k < kNAPerThread; ++k) {
    const long long i = base + (long long)k * kNAThreads + threadIdx.x;
    if (i < n) s = fma(a[i], a[i], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNAThreads / 32; ++w) t += sh[w];
    partial[blockIdx.x] = w2 * t;
  }
}

// out[0] = sqrt(sum of partial[0 .. count)), fixed summation order.
__global__ void __launch_bounds__(kNAThreads) na_finish_kernel(const double* __restrict__ partial, int count,
                                                              double* __restrict__ out) {
  __shared__ double sh[kNAThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < count; i += kNAThreads) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNAThreads / 32; ++w) t += sh[w];
    out[0] = sqrt(t);
  }
}

// Device address of the scratch array on the current device (set-up on
// the first call per device, under a lock).
cmg_status na_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNAMaxDevices) return CMG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_scratch[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return CMG_ERR_CUDA;
    }
    g_na_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_na_scratch[dev];
  return CMG_OK;
}

inline int na_blocks(long long n) { return (int)((n + kNAPerBlock - 1) / kNAPerBlock); }

}  // namespace

extern "C" cmg_status cmg_norm_noalloc(const double* y, const double* u, const double* p, long long ny,
                                       long long nu, double wy, double* out, void* stream) {
  if (!y || !u || !p || !out || ny < 0 || nu < 0 || !std::isfinite(wy) || wy < 0.0) return CMG_ERR_INVALID_ARG;
  if (ny > kNAMaxLen || nu > kNAMaxLen) return CMG_ERR_UNSUPPORTED;
  double* partial = nullptr;
  const cmg_status st = na_scratch(&partial);
  if (st != CMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int by = na_blocks(ny), bu = na_blocks(nu), bp = na_blocks(ny);
  // Every partial read by the finish kernel is written by this call, so no
  // part of the array has to be cleared first.
  if (by) na_sumsq_kernel<<<by, kNAThreads, 0, s>>>(y, ny, wy * wy, partial);
  if (bu) na_sumsq_kernel<<<bu, kNAThreads, 0, s>>>(u, nu, 1.0, partial + by);
  if (bp) na_sumsq_kernel<<<bp, kNAThreads, 0, s>>>(p, ny, 1.0, partial + by + bu);
  na_finish_kernel<<<1, kNAThreads, 0, s>>>(partial, by + bu + bp, out);
  cmg::count_launches((by ? 1 : 0) + (bu ? 1 : 0) + (bp ? 1 : 0) + 1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CMG_OK : CMG_ERR_CUDA;
}
