// Node-sample kernels of the collective multigrid cycle:
//   residual r = f - S x (Eq. (2) blocks), red-black collective Gauss-Seidel
//   half-sweep (reduced node systems Eq. (12) solved by Eq. (13)), damped
//   collective Jacobi update (Eq. (11)), restriction P^T and prolongation P
//   (Algorithm 1).
//
// Layout: node arrays [n*n][ld] with the sample index fastest.  The lpn
// lanes of a node group read that node's samples as contiguous V-element
// vectors (coalesced 128-bit loads); neighbour rows are re-read from L2 by
// the CTAs of adjacent rows, which run close together in launch order.
// The sum over samples in the control row (u) is a shuffle reduction over
// the node group, carried in FP64 in both precisions.
#include "cmg_common.cuh"

namespace cmg {

namespace {

template <typename T, int V>
__device__ __forceinline__ void fma_faces(vec<T, V>& acc, const vec<T, V>& kW, const vec<T, V>& vW,
                                          const vec<T, V>& kE, const vec<T, V>& vE,
                                          const vec<T, V>& kS, const vec<T, V>& vS,
                                          const vec<T, V>& kN, const vec<T, V>& vN) {
#pragma unroll
  for (int k = 0; k < V; ++k) {
    T a = acc.v[k];
    a = fma(kW.v[k], vW.v[k], a);
    a = fma(kE.v[k], vE.v[k], a);
    a = fma(kS.v[k], vS.v[k], a);
    a = fma(kN.v[k], vN.v[k], a);
    acc.v[k] = a;
  }
}

template <typename T>
__device__ __forceinline__ T recip(T a);
template <>
__device__ __forceinline__ float recip<float>(float a) { return __frcp_rn(a); }

// ---------------------------------------------------------------------------
// r = f - S x on all nodes; with f == nullptr (all three) r = S x instead
// (operator apply, used for the Krylov basis).
// ---------------------------------------------------------------------------
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) residual_kernel(LevelView<T> L, Vec3c<T> x, Vec3c<T> f,
                                                          Vec3<T> r, int lpn, T wy) {
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const int lane = threadIdx.x & (lpn - 1);
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  const bool valid = node < (long)n * n;
  const T c = (T)L.c, e = (T)L.e;
  const bool apply = f.y == nullptr;
  double psum = 0.0;
  if (valid) {
    const int iy = (int)(node / n), ix = (int)(node - (long)iy * n);
    const size_t o = (size_t)node * ld;
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
    const bool hW = ix > 0, hE = ix < n - 1, hS = iy > 0, hN = iy < n - 1;
    const T uu = x.u[node];
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        const vec<T, V> kW = ldv<T, V>(kWp + j), kE = ldv<T, V>(kWp + ld + j);
        const vec<T, V> kS = ldv<T, V>(kSp + j), kN = ldv<T, V>(kSp + (size_t)n * ld + j);
        const vec<T, V> y = ldv<T, V>(x.y + o + j), p = ldv<T, V>(x.p + o + j);
        vec<T, V> offy = vzero<T, V>(), offp = vzero<T, V>();
        fma_faces<T, V>(offy, kW, ldv_if<T, V>(hW, x.y + o - ld + j), kE, ldv_if<T, V>(hE, x.y + o + ld + j),
                        kS, ldv_if<T, V>(hS, x.y + o - (size_t)n * ld + j), kN,
                        ldv_if<T, V>(hN, x.y + o + (size_t)n * ld + j));
        fma_faces<T, V>(offp, kW, ldv_if<T, V>(hW, x.p + o - ld + j), kE, ldv_if<T, V>(hE, x.p + o + ld + j),
                        kS, ldv_if<T, V>(hS, x.p + o - (size_t)n * ld + j), kN,
                        ldv_if<T, V>(hN, x.p + o + (size_t)n * ld + j));
        vec<T, V> ry, rp;
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T a = (kW.v[k] + kE.v[k]) + (kS.v[k] + kN.v[k]);
          // state rows: c y + A p ; adjoint rows: A y + e u
          ry.v[k] = c * y.v[k] + (a * p.v[k] - offp.v[k]);
          rp.v[k] = (a * y.v[k] - offy.v[k]) + e * uu;
          psum += (double)p.v[k];
        }
        if (!apply) {
          const vec<T, V> fy = ldv<T, V>(f.y + o + j), fp = ldv<T, V>(f.p + o + j);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            ry.v[k] = fy.v[k] - ry.v[k];
            rp.v[k] = fp.v[k] - rp.v[k];
          }
        }
        if (wy != T(1)) {
#pragma unroll
          for (int k = 0; k < V; ++k) ry.v[k] *= wy;
        }
        stv<T, V>(r.y + o + j, ry);
        stv<T, V>(r.p + o + j, rp);
      }
    }
  }
  psum = group_sum(psum, lpn);
  if (valid && lane == 0) {
    const double su = L.G * (double)x.u[node] + L.d * psum;   // control row: G u + d sum_j p_j
    r.u[node] = (T)(apply ? su : (double)f.u[node] - su);
  }
}

// ---------------------------------------------------------------------------
// Local solve, Eq. (13), shared by GS and Jacobi.  With b_p the rhs of the
// first block row, b_y of the last, b_u of the control row:
//   u = (b_u + d sum_j (c b_y,j / a_j^2 - b_p,j / a_j)) / sigma
//   y_j = (b_y,j - e u) / a_j,   p_j = (b_p,j - c y_j) / a_j
// ---------------------------------------------------------------------------

template <typename T, int V>
__device__ __forceinline__ vec<T, V> inv_diag(const LevelView<T>& L, size_t off, const vec<T, V>& kW,
                                              const vec<T, V>& kE, const vec<T, V>& kS,
                                              const vec<T, V>& kN) {
  vec<T, V> ia;
  if constexpr (sizeof(T) == 8) {
    ia = ldv<T, V>(reinterpret_cast<const T*>(L.inva) + off);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) ia.v[k] = recip<T>((kW.v[k] + kE.v[k]) + (kS.v[k] + kN.v[k]));
  }
  return ia;
}

// One red-black half-sweep: every node of `colour` is replaced by the
// solution of its reduced system with the current neighbour values.
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) rbgs_half_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> f,
                                                           int colour, int lpn) {
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const int lane = threadIdx.x & (lpn - 1);
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  const bool valid = g < colour_count(n, colour);
  const T c = (T)L.c;
  int iy = 0, ix = 0;
  if (valid) colour_node(g, n, colour, iy, ix);
  const long node = (long)iy * n + ix;
  const size_t o = (size_t)node * ld;
  vec<T, V> bp[SPL], by[SPL], ia[SPL];
  double tsum = 0.0;
  if (valid) {
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
    const bool hW = ix > 0, hE = ix < n - 1, hS = iy > 0, hN = iy < n - 1;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        const vec<T, V> kW = ldv<T, V>(kWp + j), kE = ldv<T, V>(kWp + ld + j);
        const vec<T, V> kS = ldv<T, V>(kSp + j), kN = ldv<T, V>(kSp + (size_t)n * ld + j);
        bp[s] = ldv<T, V>(f.y + o + j);   // first block row: c y + A p = f_y
        by[s] = ldv<T, V>(f.p + o + j);   // last block row:  A y + e u = f_p
        fma_faces<T, V>(bp[s], kW, ldv_if<T, V>(hW, x.p + o - ld + j), kE, ldv_if<T, V>(hE, x.p + o + ld + j),
                        kS, ldv_if<T, V>(hS, x.p + o - (size_t)n * ld + j), kN,
                        ldv_if<T, V>(hN, x.p + o + (size_t)n * ld + j));
        fma_faces<T, V>(by[s], kW, ldv_if<T, V>(hW, x.y + o - ld + j), kE, ldv_if<T, V>(hE, x.y + o + ld + j),
                        kS, ldv_if<T, V>(hS, x.y + o - (size_t)n * ld + j), kN,
                        ldv_if<T, V>(hN, x.y + o + (size_t)n * ld + j));
        ia[s] = inv_diag<T, V>(L, o + j, kW, kE, kS, kN);
        T t = T(0);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T iak = ia[s].v[k];
          t += (c * iak) * (iak * by[s].v[k]) - iak * bp[s].v[k];
        }
        tsum += (double)t;
      }
    }
  }
  tsum = group_sum(tsum, lpn);
  if (valid) {
    const double uu = ((double)f.u[node] + L.d * tsum) / L.sigma[node];
    if (lane == 0) x.u[node] = (T)uu;
    const T uT = (T)uu, e = (T)L.e;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        vec<T, V> yn, pn;
#pragma unroll
        for (int k = 0; k < V; ++k) {
          yn.v[k] = ia[s].v[k] * (by[s].v[k] - e * uT);
          pn.v[k] = ia[s].v[k] * (bp[s].v[k] - c * yn.v[k]);
        }
        stv<T, V>(x.y + o + j, yn);
        stv<T, V>(x.p + o + j, pn);
      }
    }
  }
}

// Damped collective Jacobi, Eq. (11): x_i += theta S~_i^{-1} r_i, r = f - S x
// computed beforehand for all nodes.
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) jacobi_update_kernel(LevelView<T> L, Vec3<T> x, Vec3c<T> r,
                                                               double theta, int lpn) {
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const int lane = threadIdx.x & (lpn - 1);
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  const bool valid = node < (long)n * n;
  const T c = (T)L.c;
  const size_t o = (size_t)(valid ? node : 0) * ld;
  vec<T, V> bp[SPL], by[SPL], ia[SPL];
  double tsum = 0.0;
  if (valid) {
    const int iy = (int)(node / n), ix = (int)(node - (long)iy * n);
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        bp[s] = ldv<T, V>(r.y + o + j);
        by[s] = ldv<T, V>(r.p + o + j);
        ia[s] = inv_diag<T, V>(L, o + j, ldv<T, V>(kWp + j), ldv<T, V>(kWp + ld + j), ldv<T, V>(kSp + j),
                               ldv<T, V>(kSp + (size_t)n * ld + j));
        T t = T(0);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T iak = ia[s].v[k];
          t += (c * iak) * (iak * by[s].v[k]) - iak * bp[s].v[k];
        }
        tsum += (double)t;
      }
    }
  }
  tsum = group_sum(tsum, lpn);
  if (valid) {
    const double du = ((double)r.u[node] + L.d * tsum) / L.sigma[node];
    if (lane == 0) x.u[node] = (T)((double)x.u[node] + theta * du);
    const T duT = (T)du, e = (T)L.e, th = (T)theta;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        vec<T, V> yv = ldv<T, V>(x.y + o + j), pv = ldv<T, V>(x.p + o + j);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T dy = ia[s].v[k] * (by[s].v[k] - e * duT);
          const T dp = ia[s].v[k] * (bp[s].v[k] - c * dy);
          yv.v[k] += th * dy;
          pv.v[k] += th * dp;
        }
        stv<T, V>(x.y + o + j, yv);
        stv<T, V>(x.p + o + j, pv);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Transfers.  Coarse node (J, I) sits on fine node (2J+1, 2I+1).
// ---------------------------------------------------------------------------

// c = P^T r: weights 1 (centre), 1/2 (edge neighbours), 1/4 (corners).
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) restrict_kernel(int nf, int N, Vec3c<T> r, Vec3<T> cv, int lpn) {
  const int nc = (nf - 1) / 2;
  const int lane = threadIdx.x & (lpn - 1);
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  if (node >= (long)nc * nc) return;
  const int J = (int)(node / nc), I = (int)(node - (long)J * nc);
  const size_t ld = (size_t)N;
  const long fc = (long)(2 * J + 1) * nf + (2 * I + 1);
  const T w[3] = {T(0.5), T(1), T(0.5)};
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    const int j = (lane + s * lpn) * V;
    if (j < N) {
      vec<T, V> ay = vzero<T, V>(), ap = vzero<T, V>();
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const T wt = w[dy + 1] * w[dx + 1];
          const size_t o = (size_t)(fc + (long)dy * nf + dx) * ld + j;
          const vec<T, V> vy = ldv<T, V>(r.y + o), vp = ldv<T, V>(r.p + o);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            ay.v[k] = fma(wt, vy.v[k], ay.v[k]);
            ap.v[k] = fma(wt, vp.v[k], ap.v[k]);
          }
        }
      stv<T, V>(cv.y + (size_t)node * ld + j, ay);
      stv<T, V>(cv.p + (size_t)node * ld + j, ap);
    }
  }
  if (lane == 0) {
    T au = T(0);
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) au = fma(w[dy + 1] * w[dx + 1], r.u[fc + (long)dy * nf + dx], au);
    cv.u[node] = au;
  }
}

// x += P e: fine node gets 1 x coinciding coarse node, 1/2 x each of two
// edge neighbours, 1/4 x each of four cell corners (zero outside the grid).
template <typename T, int V, int SPL>
__global__ void __launch_bounds__(kBlock) prolong_add_kernel(int nf, int N, Vec3c<T> e, Vec3<T> x, int lpn) {
  const int nc = (nf - 1) / 2;
  const int lane = threadIdx.x & (lpn - 1);
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) / lpn;
  if (node >= (long)nf * nf) return;
  const int iy = (int)(node / nf), ix = (int)(node - (long)iy * nf);
  int Jr[2], Ir[2];
  T wy[2], wx[2];
  int ny, nx;
  if (iy & 1) { Jr[0] = (iy - 1) >> 1; wy[0] = T(1); ny = 1; }
  else { Jr[0] = (iy >> 1) - 1; Jr[1] = iy >> 1; wy[0] = wy[1] = T(0.5); ny = 2; }
  if (ix & 1) { Ir[0] = (ix - 1) >> 1; wx[0] = T(1); nx = 1; }
  else { Ir[0] = (ix >> 1) - 1; Ir[1] = ix >> 1; wx[0] = wx[1] = T(0.5); nx = 2; }
  const size_t ld = (size_t)N;
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    const int j = (lane + s * lpn) * V;
    if (j < N) {
      vec<T, V> vy = ldv<T, V>(x.y + (size_t)node * ld + j), vp = ldv<T, V>(x.p + (size_t)node * ld + j);
      for (int a = 0; a < ny; ++a) {
        if (Jr[a] < 0 || Jr[a] >= nc) continue;
        for (int b = 0; b < nx; ++b) {
          if (Ir[b] < 0 || Ir[b] >= nc) continue;
          const T wt = wy[a] * wx[b];
          const size_t o = ((size_t)Jr[a] * nc + Ir[b]) * ld + j;
          const vec<T, V> ey = ldv<T, V>(e.y + o), ep = ldv<T, V>(e.p + o);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            vy.v[k] = fma(wt, ey.v[k], vy.v[k]);
            vp.v[k] = fma(wt, ep.v[k], vp.v[k]);
          }
        }
      }
      stv<T, V>(x.y + (size_t)node * ld + j, vy);
      stv<T, V>(x.p + (size_t)node * ld + j, vp);
    }
  }
  if (lane == 0) {
    T vu = x.u[node];
    for (int a = 0; a < ny; ++a) {
      if (Jr[a] < 0 || Jr[a] >= nc) continue;
      for (int b = 0; b < nx; ++b) {
        if (Ir[b] < 0 || Ir[b] >= nc) continue;
        vu = fma(wy[a] * wx[b], e.u[(size_t)Jr[a] * nc + Ir[b]], vu);
      }
    }
    x.u[node] = vu;
  }
}

inline unsigned grid_for(long groups, int lpn) {
  const long threads = groups * lpn;
  return (unsigned)((threads + kBlock - 1) / kBlock);
}

}  // namespace

SampleMap choose_map(int N, int elem_bytes) {
  SampleMap m;
  const int vmax = 16 / elem_bytes;     // 2 for double, 4 for float
  m.V = (N % vmax == 0) ? vmax : 1;
  const int chunks = (N + m.V - 1) / m.V;
  int lpn = 1;
  while (lpn < chunks && lpn < 32) lpn <<= 1;
  m.lpn = lpn;
  int spl = (chunks + lpn - 1) / lpn;
  int p2 = 1;
  while (p2 < spl) p2 <<= 1;
  m.spl = p2;
  return m;
}

#define CMG_SPL_SWITCH(SPLV, V_, ...)                                           \
  switch (SPLV) {                                                              \
    case 1: { constexpr int V = V_, SPL = 1; __VA_ARGS__; } break;             \
    case 2: { constexpr int V = V_, SPL = 2; __VA_ARGS__; } break;             \
    case 4: { constexpr int V = V_, SPL = 4; __VA_ARGS__; } break;             \
    case 8: { constexpr int V = V_, SPL = 8; __VA_ARGS__; } break;             \
    default: return cudaErrorInvalidValue;                                     \
  }

#define CMG_DISPATCH(T, MAP, ...)                                              \
  do {                                                                         \
    if ((MAP).V == 1) { CMG_SPL_SWITCH((MAP).spl, 1, __VA_ARGS__) }            \
    else if constexpr (sizeof(T) == 8) { CMG_SPL_SWITCH((MAP).spl, 2, __VA_ARGS__) } \
    else { CMG_SPL_SWITCH((MAP).spl, 4, __VA_ARGS__) }                         \
  } while (0)

template <typename T>
cudaError_t launch_residual(const LevelView<T>& L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r, cudaStream_t st, double wy) {
  const SampleMap m = choose_map(L.N, sizeof(T));
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  CMG_DISPATCH(T, m, (residual_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(L, x, f, r, m.lpn, (T)wy)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rbgs_half(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, int colour, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, sizeof(T));
  const unsigned grid = grid_for(colour_count(L.n, colour), m.lpn);
  CMG_DISPATCH(T, m, (rbgs_half_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(L, x, f, colour, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi_update(const LevelView<T>& L, Vec3<T> x, Vec3c<T> r, double theta, cudaStream_t st) {
  const SampleMap m = choose_map(L.N, sizeof(T));
  const unsigned grid = grid_for((long)L.n * L.n, m.lpn);
  CMG_DISPATCH(T, m, (jacobi_update_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(L, x, r, theta, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(int nf, int N, Vec3c<T> r, Vec3<T> c, cudaStream_t st) {
  const SampleMap m = choose_map(N, sizeof(T));
  const int nc = (nf - 1) / 2;
  const unsigned grid = grid_for((long)nc * nc, m.lpn);
  CMG_DISPATCH(T, m, (restrict_kernel<T, V, SPL><<<grid, kBlock, 0, st>>>(nf, N, r, c, m.lpn)));
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(int nf, int N, Vec3c<T> e, Vec3<T> x, cudaStream_t st) {
  const SampleMap m = choose_map(N, sizeof(T));
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
