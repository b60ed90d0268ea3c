// Coarse-grid part of Algorithm 1 as ONE kernel launched as a thread-block
// cluster: every grid with n <= tail_n, down to and including the coarsest
// direct solve, runs inside a single launch whose phases are separated by
// cluster barriers.  On these small grids a separate launch per step costs
// several microseconds of GPU latency while the work itself is a fraction
// of that; inside the cluster a phase costs one pass over L2-resident data
// plus one hardware barrier.
//
// Phases use the same per-node items as the one-kernel-per-step path
// (cmg_items.cuh), with loads that bypass L1 because the data was written by
// other CTAs of the cluster in an earlier phase.  The recursion of the
// cycle (gamma = 1 or 2 calls per grid) is unrolled into an explicit loop
// with a per-grid call counter, so every thread follows the same phase
// sequence.
#pragma once

#include <cooperative_groups.h>

#include "cmg_items.cuh"

namespace cmg {

namespace tail {

namespace cg = cooperative_groups;

// Cluster barrier: arrive has release and wait has acquire semantics at
// cluster scope, which orders every thread's earlier global-memory writes
// before any thread's later reads in the cluster (reads bypass L1, see ldx).
__device__ __forceinline__ void barrier(const cg::cluster_group& cl) { cl.sync(); }

// Coarsest direct solve by one CTA (block elimination, as cmg_coarse.cu):
// thread per sample for the products with A_j^{-1}, block reduction of the
// control right side, control solve with the precomputed inverse, back
// substitution.
template <typename T, int MM>
__device__ void coarse_cta(const TailParams<T>& P, const Vec3<T>& x, const Vec3<T>& f) {
  __shared__ double red[kTailThreads / 32][MM];
  __shared__ double rhs[MM], us[MM];
  const int m = P.cm, N = P.cN;
  const double c = P.cc, d = P.cd, e = P.ce;
  double q[MM];
#pragma unroll
  for (int r = 0; r < MM; ++r) q[r] = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* A = P.Ainv + (size_t)j * m * m;
    double by[MM], bp[MM], z[MM];
#pragma unroll
    for (int r = 0; r < MM; ++r) {
      by[r] = r < m ? (double)ld1<T, true>(f.y + (size_t)r * N + j) : 0.0;
      bp[r] = r < m ? (double)ld1<T, true>(f.p + (size_t)r * N + j) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < MM; ++r) {
      double sw = 0.0, sz = 0.0;
      if (r < m) {
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < m) {
            sw += A[r * m + k] * by[k];
            sz += A[r * m + k] * bp[k];
          }
        P.wz[(size_t)j * m + r] = sw;
        P.wz[(size_t)N * m + (size_t)j * m + r] = sz;
      }
      q[r] += sw;
      z[r] = sz;
    }
#pragma unroll
    for (int r = 0; r < MM; ++r) {
      if (r < m) {
        double sv = 0.0;
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < m) sv += A[r * m + k] * z[k];
        q[r] -= c * sv;
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < MM; ++r) {
    double v = q[r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][r] = v;
  }
  __syncthreads();
  const LevelView<T>& cl = P.lev[P.nlev - 1].L;   // coarsest grid: control rows only at its control nodes
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][r];
    const double dr = cl.dw ? d * (double)cl.dw[r] : d;   // d_i of the coarsest grid's row r
    rhs[r] = cl.ctl.inside(r / cl.n, r % cl.n) ? (double)ld1<T, true>(f.u + r) - dr * s : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    if (!P.freeze_u)
      for (int k = 0; k < m; ++k) s += P.Minv[r * m + k] * rhs[k];
    us[r] = s;
    x.u[r] = (T)s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* A = P.Ainv + (size_t)j * m * m;
    double yv[MM];
#pragma unroll
    for (int r = 0; r < MM; ++r) {
      yv[r] = 0.0;
      if (r < m) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < m) t += A[r * m + k] * us[k];
        yv[r] = P.wz[(size_t)N * m + (size_t)j * m + r] - e * t;
        x.y[(size_t)r * N + j] = (T)yv[r];
      }
    }
#pragma unroll
    for (int r = 0; r < MM; ++r) {
      if (r < m) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < MM; ++k)
          if (k < m) t += A[r * m + k] * yv[k];
        x.p[(size_t)r * N + j] = (T)(P.wz[(size_t)j * m + r] - c * t);
      }
    }
  }
}

// Loop of one phase: the warp's groups step through [0, count) with the
// cluster-wide stride; the trip count is the same for all lanes of a warp.
#define CMG_TAIL_FOR(COUNT, ITEM)                                              \
  for (long g0_ = wfirst; g0_ < (long)(COUNT); g0_ += stride) {               \
    const long g = g0_ + lgroup;                                               \
    ITEM;                                                                      \
  }

template <typename T, int V, int SPL, int MM>
__global__ void __launch_bounds__(kTailThreads) tail_cycle_kernel(const __grid_constant__ TailParams<T> P) {
  pdl_enter();
  const cg::cluster_group cl = cg::this_cluster();
  const int lpn = P.lpn;
  const long ctid = (long)cl.block_rank() * blockDim.x + threadIdx.x;
  const long nthr = (long)cl.num_blocks() * blockDim.x;
  const long wfirst = (ctid & ~31L) / lpn;          // first group of this warp
  const long lgroup = (threadIdx.x & 31) / lpn;     // this lane's group within the warp
  const long stride = nthr / lpn;
  const int lane = threadIdx.x & (lpn - 1);
  const int N = P.lev[0].L.N;

  auto smooth = [&](int k, int sweeps) {
    const TailLevel<T>& lv = P.lev[k];
    const Vec3c<T> f = cview(lv.f);
    for (int s = 0; s < sweeps; ++s) {
      if (P.smoother == CMG_SMOOTH_RBGS) {
        for (int colour = 0; colour < 2; ++colour) {
          CMG_TAIL_FOR(colour_count(lv.L.n, colour),
                       (rbgs_item<T, V, SPL, true>(lv.L, lv.x, f, colour, g, lane, lpn)));
          barrier(cl);
        }
      } else {
        const long nn = (long)lv.L.n * lv.L.n;
        CMG_TAIL_FOR(nn, (residual_item<T, V, SPL, true>(lv.L, cview(lv.x), f, lv.r, g, lane, lpn, T(1))));
        barrier(cl);
        CMG_TAIL_FOR(nn, (jacobi_item<T, V, SPL, true>(lv.L, lv.x, cview(lv.r), P.theta, g, lane, lpn)));
        barrier(cl);
      }
    }
  };

  int calls[kTailMax];
  int k = 0;
  bool down = true;
  while (true) {
    const TailLevel<T>& lv = P.lev[k];
    if (down) {
      if (k == P.nlev - 1) {
        if (cl.block_rank() == 0) coarse_cta<T, MM>(P, lv.x, lv.f);
        barrier(cl);
        down = false;
        if (--k < 0) break;
        continue;
      }
      const TailLevel<T>& cv = P.lev[k + 1];
      smooth(k, P.n1);
      const long nn = (long)lv.L.n * lv.L.n;
      CMG_TAIL_FOR(nn, (residual_item<T, V, SPL, true>(lv.L, cview(lv.x), cview(lv.f), lv.r, g, lane, lpn, T(1))));
      barrier(cl);
      const long nc2 = (long)cv.L.n * cv.L.n;
      CMG_TAIL_FOR(nc2, (restrict_item<T, V, SPL, true>(lv.L.n, N, cview(lv.r), cv.f, cv.x, g, lane, lpn)));
      barrier(cl);
      calls[k] = P.gamma;
      ++k;
    } else {
      if (--calls[k] > 0) {   // W-cycle: visit the coarser grid again from its current iterate
        ++k;
        down = true;
        continue;
      }
      const TailLevel<T>& cv = P.lev[k + 1];
      const long nn = (long)lv.L.n * lv.L.n;
      CMG_TAIL_FOR(nn, (prolong_item<T, V, SPL, true>(lv.L.n, N, cview(cv.x), lv.x, g, lane, lpn, lv.L.ctl)));
      barrier(cl);
      smooth(k, P.n2);
      if (--k < 0) break;
    }
  }
}

#undef CMG_TAIL_FOR

}  // namespace tail

}  // namespace cmg
