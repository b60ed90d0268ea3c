// Device helpers shared by the node-sample kernels.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "cmg_internal.h"

namespace cmg {

// V contiguous elements moved with one vector load/store (16 bytes for
// double2 / float4).
template <typename T, int V>
struct alignas(sizeof(T) * V) vec {
  T v[V];
};

template <typename T, int V>
__device__ __forceinline__ vec<T, V> ldv(const T* p) {
  return *reinterpret_cast<const vec<T, V>*>(p);
}
template <typename T, int V>
__device__ __forceinline__ void stv(T* p, const vec<T, V>& x) {
  *reinterpret_cast<vec<T, V>*>(p) = x;
}
template <typename T, int V>
__device__ __forceinline__ vec<T, V> vzero() {
  vec<T, V> r;
#pragma unroll
  for (int k = 0; k < V; ++k) r.v[k] = T(0);
  return r;
}
template <typename T, int V>
__device__ __forceinline__ vec<T, V> ldv_if(bool ok, const T* p) {
  return ok ? ldv<T, V>(p) : vzero<T, V>();
}

// Programmatic dependent launch: a kernel launched with launch_k may start
// while its predecessor in the stream drains; it waits here, before touching
// any memory, until the predecessor has completed and its writes are
// visible, and at once allows its own successor to be scheduled (which in
// turn waits).  Both are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Sum over the lpn lanes that share a node (aligned groups inside a warp).
// Every lane of the warp must call this.
template <typename A>
__device__ __forceinline__ A group_sum(A v, int lpn) {
  for (int o = lpn >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Arithmetic of the control row of a residual (G u_i + d_i sum_j p_j): the
// vector's own precision.
template <typename T>
using acc_t = typename std::conditional<sizeof(T) == 4, float, double>::type;

// 1/sigma_i of Eq. (13): FP64, except in an FP32 view with the all-FP32
// option (ctl32), which reads the FP32 copy.
template <typename T>
__device__ __forceinline__ double isigma_of(const LevelView<T>& L, long node) {
  if constexpr (sizeof(T) == 4) {
    if (L.ctl32) return (double)L.isigma32[node];
  }
  return L.isigma[node];
}

// The per-node Schur scalar of Eq. (13): u_i = (b_u + d_i sum_j t_j) / sigma_i
// with t_j = c b_y,j / a_j^2 - b_p,j / a_j, from this lane's part `tacc` of
// the sum over samples (accumulated in the vector's precision).  The lane
// parts are converted to FP64 once, then the group sum, the product with
// 1/sigma_i and u_i are FP64: a few FP64 operations per node, not per
// node-sample.  The all-FP32 option (ctl32, FP32 views) keeps all of it in
// FP32.  Every lane of the warp must call this (shuffle reduction).
template <typename T>
__device__ __forceinline__ double schur_u(const LevelView<T>& L, T tacc, int lpn, double bu, double di, double isg) {
  if constexpr (sizeof(T) == 4) {
    if (L.ctl32) {
      const float ts = group_sum(tacc, lpn);
      return (double)(((float)bu + (float)di * ts) * (float)isg);
    }
  }
  const double ts = group_sum((double)tacc, lpn);
  return (bu + di * ts) * isg;
}

// Red-black ordering: map the g-th node of colour `colour` (red = (ix+iy)
// even = 0) to (iy, ix).  Rows are paired: row 2P holds the first count0
// nodes of pair P, row 2P+1 the remaining n - count0.
// 32-bit arithmetic: grids have n <= 4095, so g < n^2 < 2^31.
__device__ __forceinline__ void colour_node(long g, int n, int colour, int& iy, int& ix) {
  const int gi = (int)g;
  const int P = gi / n;
  const int q = gi - P * n;
  const int s0 = colour & 1;
  const int count0 = (n - s0 + 1) >> 1;
  if (q < count0) {
    iy = (int)(2 * P);
    ix = s0 + 2 * q;
  } else {
    iy = (int)(2 * P + 1);
    ix = (1 - s0) + 2 * (q - count0);
  }
}

__host__ __device__ inline long colour_count(int n, int colour) {
  const long nn = (long)n * n;
  return colour == 0 ? (nn + 1) / 2 : nn / 2;
}

}  // namespace cmg
