// Coarsest-grid direct solve (Algorithm 1, "direct solver"), FP64.
//
// Block elimination of the saddle system on the coarsest grid (m = n_c^2
// nodes): with the per-sample stiffness inverses A_j^{-1}
//     y_j = A_j^{-1} (f_p,j - e u),   p_j = A_j^{-1} (f_y,j - c y_j),
// and the control row becomes the m x m system
//     (G I + d c e sum_j A_j^{-2}) u = f_u - d sum_j (A_j^{-1} f_y,j - c A_j^{-2} f_p,j).
// Setup inverts every A_j (Gauss-Jordan, SPD so no pivoting) and the control
// Schur matrix once per hierarchy; each solve is two launches: per-sample
// products with a fixed-order reduction of the control right side, then the
// control solve and per-sample back substitution.
#include <algorithm>
#include <type_traits>

#include "cmg_common.cuh"

namespace cmg {

namespace {

// Gauss-Jordan inverse of the m x m matrix in aug[:, 0:m] into aug[:, m:2m].
__device__ void gauss_jordan(double* aug, double* fac, int m) {
  const int w = 2 * m;
  for (int col = 0; col < m; ++col) {
    __syncthreads();
    const double piv = aug[col * w + col];
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) aug[col * w + c] /= piv;
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) fac[r] = aug[r * w + col];
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * w; idx += blockDim.x) {
      const int r = idx / w, c = idx - r * w;
      if (r != col) aug[idx] -= fac[r] * aug[col * w + c];
    }
  }
  __syncthreads();
}

// One CTA per sample: assemble A_j from the face coefficients and invert it.
__global__ void coarse_inv_kernel(int n, int N, const double* __restrict__ kx, const double* __restrict__ ky,
                                  double* __restrict__ Ainv) {
  __shared__ double aug[kMaxCoarseM * 2 * kMaxCoarseM];
  __shared__ double fac[kMaxCoarseM];
  const int j = blockIdx.x;
  const int m = n * n, w = 2 * m;
  for (int idx = threadIdx.x; idx < m * w; idx += blockDim.x) {
    const int r = idx / w, c = idx - r * w;
    double v = 0.0;
    if (c >= m) {
      v = (c - m == r) ? 1.0 : 0.0;
    } else {
      const int iy = r / n, ix = r - iy * n;
      const double kW = kx[((size_t)iy * (n + 1) + ix) * N + j];
      const double kE = kx[((size_t)iy * (n + 1) + ix + 1) * N + j];
      const double kS = ky[((size_t)iy * n + ix) * N + j];
      const double kN = ky[((size_t)(iy + 1) * n + ix) * N + j];
      if (c == r) v = (kW + kE) + (kS + kN);
      else if (ix > 0 && c == r - 1) v = -kW;
      else if (ix < n - 1 && c == r + 1) v = -kE;
      else if (iy > 0 && c == r - n) v = -kS;
      else if (iy < n - 1 && c == r + n) v = -kN;
    }
    aug[idx] = v;
  }
  gauss_jordan(aug, fac, m);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    Ainv[(size_t)j * m * m + idx] = aug[r * w + m + c];
  }
}

// One CTA per entry (r, c) of the control Schur matrix:
// M[r][c] = G delta_rc + d c e sum_j (A_j^{-1} A_j^{-1})[r][c], fixed-order reduction.
// With local control the system is posed on the control nodes only: rows
// and columns of the other nodes are those of the identity (their right
// sides are zero, so their u is zero).
__global__ void coarse_schur_kernel(int m, int N, const double* __restrict__ Ainv, double G, double dce,
                                    double* __restrict__ M, int n, CtlBox ctl, const float* __restrict__ dw) {
  __shared__ double red[128];
  const int r = blockIdx.x / m, c = blockIdx.x - (blockIdx.x / m) * m;
  double s = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* A = Ainv + (size_t)j * m * m;
    double t = 0.0;
    for (int k = 0; k < m; ++k) t += A[r * m + k] * A[k * m + c];
    s += t;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const bool on = ctl.inside(r / n, r % n) && ctl.inside(c / n, c % n);
    const double dcer = dw ? dce * (double)dw[r] : dce;   // row r couples through d_r
    M[blockIdx.x] = on ? (r == c ? G : 0.0) + dcer * red[0] : (r == c ? 1.0 : 0.0);
  }
}

__global__ void invert_kernel(int m, const double* __restrict__ M, double* __restrict__ Minv) {
  __shared__ double aug[kMaxCoarseM * 2 * kMaxCoarseM];
  __shared__ double fac[kMaxCoarseM];
  const int w = 2 * m;
  for (int idx = threadIdx.x; idx < m * w; idx += blockDim.x) {
    const int r = idx / w, c = idx - r * w;
    aug[idx] = c < m ? M[r * m + c] : (c - m == r ? 1.0 : 0.0);
  }
  gauss_jordan(aug, fac, m);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    Minv[idx] = aug[r * w + m + c];
  }
}

constexpr int kCoarseThreads = 32;   // one warp per CTA: samples spread over SMs

// Per sample j: w = A_j^{-1} f_y,j, z = A_j^{-1} f_p,j, v = A_j^{-1} z;
// per-warp partial sums of q = w - c v for the control right side.
template <typename T, int MM>
__global__ void __launch_bounds__(kCoarseThreads) coarse_solve_a(int m, int N, const double* __restrict__ Ainv,
                                                                double c, const T* __restrict__ fy,
                                                                const T* __restrict__ fp, double* __restrict__ wz,
                                                                double* __restrict__ partial) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = j < N;
  double q[MM];
#pragma unroll
  for (int r = 0; r < MM; ++r) q[r] = 0.0;
  if (valid) {
    const double* A = Ainv + (size_t)j * m * m;
    double by[MM], bp[MM], z[MM];
#pragma unroll
    for (int r = 0; r < MM; ++r) {
      by[r] = r < m ? (double)fy[(size_t)r * N + j] : 0.0;
      bp[r] = r < m ? (double)fp[(size_t)r * N + j] : 0.0;
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
        wz[(size_t)j * m + r] = sw;
        wz[(size_t)N * m + (size_t)j * m + r] = sz;
      }
      q[r] = sw;
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
#pragma unroll
  for (int r = 0; r < MM; ++r) {
    double v = q[r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && r < m) partial[(size_t)blockIdx.x * m + r] = v;
  }
}

// Control solve (every CTA redundantly, fixed order) and back substitution.
template <typename T, int MM>
__global__ void __launch_bounds__(kCoarseThreads) coarse_solve_b(int m, int N, int nblk,
                                                                const double* __restrict__ Ainv,
                                                                const double* __restrict__ Minv, double c, double d,
                                                                double e, const T* __restrict__ fu,
                                                                const double* __restrict__ wz,
                                                                const double* __restrict__ partial, T* __restrict__ y,
                                                                T* __restrict__ u, T* __restrict__ p, int freeze_u,
                                                                int n, CtlBox ctl, const float* __restrict__ dw) {
  __shared__ double rhs[MM], us[MM];
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * m + r];
    const double dr = dw ? d * (double)dw[r] : d;
    rhs[r] = ctl.inside(r / n, r % n) ? (double)fu[r] - dr * s : 0.0;   // control rows only at control nodes
  }
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    if (!freeze_u)   // frozen control: zero correction of u, state and adjoint solved for it
      for (int k = 0; k < m; ++k) s += Minv[r * m + k] * rhs[k];
    us[r] = s;
    if (blockIdx.x == 0) u[r] = (T)s;
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double* A = Ainv + (size_t)j * m * m;
  double yv[MM];
#pragma unroll
  for (int r = 0; r < MM; ++r) {
    if (r < m) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < MM; ++k)
        if (k < m) t += A[r * m + k] * us[k];
      yv[r] = wz[(size_t)N * m + (size_t)j * m + r] - e * t;
      y[(size_t)r * N + j] = (T)yv[r];
    } else {
      yv[r] = 0.0;
    }
  }
#pragma unroll
  for (int r = 0; r < MM; ++r) {
    if (r < m) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < MM; ++k)
        if (k < m) t += A[r * m + k] * yv[k];
      p[(size_t)r * N + j] = (T)(wz[(size_t)j * m + r] - c * t);
    }
  }
}

// The whole coarsest solve in one CTA, with every A_j^{-1} and the right
// sides staged in shared memory by coalesced loads and one thread per
// (sample j, row r) for the products.  The two-kernel form above gives each
// thread a whole sample (81 strided loads of A_j^{-1} per product) and is
// latency-bound.  Same block elimination; the control right side is summed
// over the samples in sample order, in FP64, and the m x m control solve is
// FP64.  The per-sample products run in the cycle's precision C: FP64 for
// FP64 cycles, FP32 for FP32 cycles (GB300's FP64 pipe made them ~6 us of
// the FP32 cycle's single-CTA critical path).
constexpr int kCoarseCtaThreads = 512;

template <typename C>
size_t coarse_cta_smem(int N, int m) {
  return 2 * 64 * sizeof(double) + ((size_t)N * m * m + 4 * (size_t)N * m) * sizeof(C);
}

// The coarsest solve by one CTA (the body shared by the single-instance
// kernel and the batched one, which runs one CTA per instance).
template <typename T, typename C>
__device__ __forceinline__ void coarse_cta_body(int m, int N, const C* __restrict__ Ainv,
                                                const double* __restrict__ Minv, double c, double d, double e,
                                                Vec3c<T> f, Vec3<T> x, int freeze_u, int nside, CtlBox ctl,
                                                const float* __restrict__ dw) {
  extern __shared__ __align__(16) double sm[];
  const int mm = m * m, nm = N * m;
  double* rhs = sm;                  // [m] control right side
  double* us = rhs + 64;             // [m] control
  C* A = reinterpret_cast<C*>(us + 64);   // [N][m][m]
  C* by = A + (size_t)N * mm;        // [N][m] f_y, later y
  C* bp = by + nm;                   // [N][m] f_p, later w - c A^{-1} z
  C* w = bp + nm;                    // [N][m] A^{-1} f_y
  C* z = w + nm;                     // [N][m] A^{-1} f_p
  const C cc = (C)c, ec = (C)e;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N * mm; i += nt) A[i] = Ainv[i];
  for (int i = tid; i < nm; i += nt) {   // f.y, f.p are [node r][sample j]
    const int r = i / N, j = i - r * N;
    by[j * m + r] = (C)f.y[i];
    bp[j * m + r] = (C)f.p[i];
  }
  __syncthreads();
  for (int i = tid; i < nm; i += nt) {
    const int j = i / m, r = i - j * m;
    const C* Ar = A + (size_t)j * mm + r * m;
    C sw = 0, sz = 0;
    for (int k = 0; k < m; ++k) {
      sw += Ar[k] * by[j * m + k];
      sz += Ar[k] * bp[j * m + k];
    }
    w[i] = sw;
    z[i] = sz;
  }
  __syncthreads();
  for (int i = tid; i < nm; i += nt) {   // w - c A^{-1} z, into bp (f_p no longer needed)
    const int j = i / m, r = i - j * m;
    const C* Ar = A + (size_t)j * mm + r * m;
    C v = 0;
    for (int k = 0; k < m; ++k) v += Ar[k] * z[j * m + k];
    bp[i] = w[i] - cc * v;
  }
  __syncthreads();
  for (int r = tid; r < m; r += nt) {
    double q = 0.0;
    for (int j = 0; j < N; ++j) q += (double)bp[j * m + r];
    const double dr = dw ? d * (double)dw[r] : d;   // d_r (active-set factor)
    rhs[r] = ctl.inside(r / nside, r % nside) ? (double)f.u[r] - dr * q : 0.0;   // control rows only at control nodes
  }
  __syncthreads();
  for (int r = tid; r < m; r += nt) {
    double u = 0.0;
    if (!freeze_u)   // frozen control: zero correction of u, state and adjoint solved for it
      for (int k = 0; k < m; ++k) u += Minv[r * m + k] * rhs[k];
    us[r] = u;
    x.u[r] = (T)u;
  }
  __syncthreads();
  for (int i = tid; i < nm; i += nt) {   // y = z - e A^{-1} u, into by
    const int j = i / m, r = i - j * m;
    const C* Ar = A + (size_t)j * mm + r * m;
    C t = 0;
    for (int k = 0; k < m; ++k) t += Ar[k] * (C)us[k];
    const C yv = z[i] - ec * t;
    by[i] = yv;
    x.y[(size_t)r * N + j] = (T)yv;
  }
  __syncthreads();
  for (int i = tid; i < nm; i += nt) {   // p = w - c A^{-1} y
    const int j = i / m, r = i - j * m;
    const C* Ar = A + (size_t)j * mm + r * m;
    C t = 0;
    for (int k = 0; k < m; ++k) t += Ar[k] * by[j * m + k];
    x.p[(size_t)r * N + j] = (T)(w[i] - cc * t);
  }
}

template <typename T, typename C>
__global__ void __launch_bounds__(kCoarseCtaThreads) coarse_solve_cta(int m, int N, const C* __restrict__ Ainv,
                                                                     const double* __restrict__ Minv, double c,
                                                                     double d, double e, Vec3c<T> f, Vec3<T> x,
                                                                     int freeze_u, int nside, CtlBox ctl,
                                                                     const float* __restrict__ dw) {
  pdl_enter();
  coarse_cta_body<T, C>(m, N, Ainv, Minv, c, d, e, f, x, freeze_u, nside, ctl, dw);
}

// The coarsest solves of a batch of instances (FP32 cycles), CTA b for
// instance b; instances whose flag act[b] is zero, or whose abort flag is
// set, are skipped.
__global__ void __launch_bounds__(kCoarseCtaThreads) batch_coarse_kernel(const BatchCoarse* __restrict__ bc,
                                                                        const int* __restrict__ act,
                                                                        const int* __restrict__ err) {
  if (*err || !act[blockIdx.x]) return;
  const BatchCoarse& q = bc[blockIdx.x];
  coarse_cta_body<float, float>(q.m, q.N, q.Ainv32, q.Minv, q.c, q.d, q.e, q.f, q.x, 0, q.nside, q.ctl, q.dw);
}

// FP32 copy of the A_j^{-1} for the FP32 coarse solve.
__global__ void cast_ainv_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

template <typename T, int MM>
cudaError_t coarse_solve_mm(const CoarseData& C, double c, double d, double e, Vec3c<T> f, Vec3<T> x,
                            cudaStream_t s, int freeze_u) {
  using Cm = std::conditional_t<sizeof(T) == 4, float, double>;   // precision of the per-sample products
  const Cm* ainv = nullptr;
  if constexpr (sizeof(T) == 4) ainv = C.Ainv32;
  else ainv = C.Ainv;
  if (MM <= 9 && ainv && coarse_cta_smem<Cm>(C.N, C.m) <= 200 * 1024) {
    static bool attr = false;
    if (!attr) {
      const cudaError_t ea = cudaFuncSetAttribute(coarse_solve_cta<T, Cm>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (ea != cudaSuccess) return ea;
      attr = true;
    }
    const cudaError_t ek = launch_k(coarse_solve_cta<T, Cm>, dim3(1), dim3(kCoarseCtaThreads),
                                    coarse_cta_smem<Cm>(C.N, C.m), s, C.m, C.N, ainv, (const double*)C.Minv, c, d, e,
                                    f, x, freeze_u, C.n, C.ctl, C.dw);
    count_launches(1);
    return ek != cudaSuccess ? ek : cudaGetLastError();
  }
  const int nblk = (C.N + kCoarseThreads - 1) / kCoarseThreads;
  coarse_solve_a<T, MM><<<nblk, kCoarseThreads, 0, s>>>(C.m, C.N, C.Ainv, c, f.y, f.p, C.wz, C.partial);
  coarse_solve_b<T, MM><<<nblk, kCoarseThreads, 0, s>>>(C.m, C.N, nblk, C.Ainv, C.Minv, c, d, e, f.u, C.wz,
                                                         C.partial, x.y, x.u, x.p, freeze_u, C.n, C.ctl, C.dw);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_coarse_solve(const CoarseData& C, double c, double d, double e, Vec3c<T> f, Vec3<T> x,
                                cudaStream_t s, int freeze_u) {
  if (C.m == 1) return coarse_solve_mm<T, 1>(C, c, d, e, f, x, s, freeze_u);
  if (C.m == 9) return coarse_solve_mm<T, 9>(C, c, d, e, f, x, s, freeze_u);
  if (C.m == 49) return coarse_solve_mm<T, 49>(C, c, d, e, f, x, s, freeze_u);
  return cudaErrorInvalidValue;
}

size_t batch_coarse_smem(int N_max, int m) { return coarse_cta_smem<float>(N_max, m); }

cudaError_t launch_batch_coarse(const BatchCoarse* bc, int count, int N_max, int m, const int* act, const int* err,
                                cudaStream_t s) {
  const size_t smem = coarse_cta_smem<float>(N_max, m);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    const cudaError_t ea = cudaFuncSetAttribute(batch_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                200 * 1024);
    if (ea != cudaSuccess) return ea;
    attr = true;
  }
  batch_coarse_kernel<<<count, kCoarseCtaThreads, smem, s>>>(bc, act, err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_setup(const CoarseData& C, const double* kx, const double* ky, double c, double G,
                                double d, double e, cudaStream_t s) {
  coarse_inv_kernel<<<C.N, 64, 0, s>>>(C.n, C.N, kx, ky, C.Ainv);
  // M is staged in the wz scratch (2 N m >= m^2 is not guaranteed, so use partial-free space):
  double* M = C.wz;   // wz holds at least max(2 N m, m m) doubles (allocated so)
  coarse_schur_kernel<<<C.m * C.m, 128, 0, s>>>(C.m, C.N, C.Ainv, G, d * c * e, M, C.n, C.ctl, C.dw);
  invert_kernel<<<1, 256, 0, s>>>(C.m, M, C.Minv);
  count_launches(3);
  if (C.Ainv32) {
    const size_t cnt = (size_t)C.N * C.m * C.m;
    cast_ainv_kernel<<<(unsigned)std::min<size_t>((cnt + 255) / 256, 1024), 256, 0, s>>>(C.Ainv, C.Ainv32, cnt);
    count_launches(1);
  }
  return cudaGetLastError();
}

// ---- Galerkin coarsest grid ------------------------------------------------
// With the non-diagonal mass M (9-point, constant) the elimination reads
//     y_j = A_j^{-1} (f_p,j - e M u),   p_j = A_j^{-1} (f_y,j - c M y_j),
//     (G M + d c e M Q M) u = f_u - d M sum_j z_j,   Q = sum_j A_j^{-1} M A_j^{-1},
// with w_j = A_j^{-1} f_p,j and z_j = A_j^{-1} (f_y,j - c M w_j).
namespace {

// (M v)_r on the n x n grid (zero outside).
__device__ __forceinline__ double mass_apply(const Stencil9& M, const double* v, int n, int r) {
  const int ry = r / n, rx = r - (r / n) * n;
  double s = 0.0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int y = ry + dy, x = rx + dx;
      if (y < 0 || y >= n || x < 0 || x >= n) continue;
      s = fma(M.w[(dy + 1) * 3 + dx + 1], v[y * n + x], s);
    }
  return s;
}

// M[r][c] of the n x n grid.
__device__ __forceinline__ double mass_entry(const Stencil9& M, int n, int r, int c) {
  const int dy = c / n - r / n, dx = c % n - r % n;
  return (dy < -1 || dy > 1 || dx < -1 || dx > 1) ? 0.0 : M.w[(dy + 1) * 3 + dx + 1];
}

// One CTA per sample: A_j from its 9-point stencil, inverted.
__global__ void galerkin_coarse_inv_kernel(int n, int N, const double* __restrict__ a9, double* __restrict__ Ainv) {
  __shared__ double aug[kMaxCoarseM * 2 * kMaxCoarseM];
  __shared__ double fac[kMaxCoarseM];
  const int j = blockIdx.x;
  const int m = n * n, w = 2 * m;
  for (int idx = threadIdx.x; idx < m * w; idx += blockDim.x) {
    const int r = idx / w, c = idx - r * w;
    double v = 0.0;
    if (c >= m) {
      v = (c - m == r) ? 1.0 : 0.0;
    } else {
      const int dy = c / n - r / n, dx = c % n - r % n;
      if (dy >= -1 && dy <= 1 && dx >= -1 && dx <= 1)
        v = a9[((size_t)((dy + 1) * 3 + dx + 1) * m + r) * N + j];
    }
    aug[idx] = v;
  }
  gauss_jordan(aug, fac, m);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    Ainv[(size_t)j * m * m + idx] = aug[r * w + m + c];
  }
}

// One CTA per entry (r, c): Q[r][c] = sum_j sum_k A_j^{-1}[r][k] (M A_j^{-1})[k][c],
// fixed-order reduction over the samples.
__global__ void galerkin_q_kernel(int n, int N, const double* __restrict__ Ainv, Stencil9 M, double* __restrict__ Q) {
  __shared__ double red[128];
  const int m = n * n;
  const int r = blockIdx.x / m, c = blockIdx.x - (blockIdx.x / m) * m;
  double s = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* A = Ainv + (size_t)j * m * m;
    double t = 0.0;
    for (int k = 0; k < m; ++k) {
      const int ky = k / n, kx = k - (k / n) * n;
      double mk = 0.0;   // (M A^{-1})[k][c]
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int y = ky + dy, x = kx + dx;
          if (y < 0 || y >= n || x < 0 || x >= n) continue;
          mk = fma(M.w[(dy + 1) * 3 + dx + 1], A[(y * n + x) * m + c], mk);
        }
      t = fma(A[r * m + k], mk, t);
    }
    s += t;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) Q[blockIdx.x] = red[0];
}

// One CTA: S_u = G M + dce M Q M, inverted into Minv.
__global__ void galerkin_schur_inv_kernel(int n, const double* __restrict__ Q, Stencil9 M, double G, double dce,
                                          double* __restrict__ Minv) {
  __shared__ double aug[kMaxCoarseM * 2 * kMaxCoarseM];
  __shared__ double fac[kMaxCoarseM];
  const int m = n * n, w = 2 * m;
  // right half: T = Q M
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    double t = 0.0;
    for (int k = 0; k < m; ++k) t = fma(Q[r * m + k], mass_entry(M, n, k, c), t);
    aug[r * w + m + c] = t;
  }
  __syncthreads();
  // left half: G M + dce M T
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    double t = 0.0;
    for (int k = 0; k < m; ++k) t = fma(mass_entry(M, n, r, k), aug[k * w + m + c], t);
    aug[r * w + c] = G * mass_entry(M, n, r, c) + dce * t;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    aug[r * w + m + c] = (r == c) ? 1.0 : 0.0;
  }
  gauss_jordan(aug, fac, m);
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    Minv[idx] = aug[r * w + m + c];
  }
}

// One CTA, a thread per sample for the per-sample products and a thread per
// node for the control system.  wz: [2][N][m] scratch (w_j, then y_j; z_j).
// f and x in the cycle's precision T; the elimination itself runs in FP64.
template <typename T>
__global__ void galerkin_coarse_solve_kernel(int n, int N, const double* __restrict__ Ainv,
                                             const double* __restrict__ Minv, Stencil9 M, double c, double d,
                                             double e, Vec3c<T> f, Vec3<T> x, double* __restrict__ wz) {
  __shared__ double s_sum[kMaxCoarseM], s_rhs[kMaxCoarseM], s_u[kMaxCoarseM];
  const int m = n * n;
  double* W = wz;
  double* Z = wz + (size_t)N * m;
  double t[kMaxCoarseM];
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* A = Ainv + (size_t)j * m * m;
    double* w = W + (size_t)j * m;
    double* z = Z + (size_t)j * m;
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(A[r * m + k], (double)f.p[(size_t)k * N + j], s);
      w[r] = s;
    }
    for (int r = 0; r < m; ++r) t[r] = (double)f.y[(size_t)r * N + j] - c * mass_apply(M, w, n, r);
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(A[r * m + k], t[k], s);
      z[r] = s;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < N; ++j) s += Z[(size_t)j * m + r];
    s_sum[r] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) s_rhs[r] = (double)f.u[r] - d * mass_apply(M, s_sum, n, r);
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = fma(Minv[r * m + k], s_rhs[k], s);
    s_u[r] = s;
    x.u[r] = (T)s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) s_rhs[r] = mass_apply(M, s_u, n, r);   // M u
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* A = Ainv + (size_t)j * m * m;
    double* w = W + (size_t)j * m;   // becomes y_j
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(A[r * m + k], s_rhs[k], s);
      w[r] -= e * s;
      x.y[(size_t)r * N + j] = (T)w[r];
    }
    for (int r = 0; r < m; ++r) t[r] = (double)f.y[(size_t)r * N + j] - c * mass_apply(M, w, n, r);
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s = fma(A[r * m + k], t[k], s);
      x.p[(size_t)r * N + j] = (T)s;
    }
  }
}

}  // namespace

cudaError_t launch_galerkin_coarse_setup(const CoarseData& C, const double* a9, const Stencil9& M, double c,
                                         double G, double d, double e, cudaStream_t s) {
  if (C.m > kMaxCoarseM) return cudaErrorInvalidValue;
  galerkin_coarse_inv_kernel<<<C.N, 64, 0, s>>>(C.n, C.N, a9, C.Ainv);
  double* Q = C.wz;   // at least m^2 doubles
  galerkin_q_kernel<<<C.m * C.m, 128, 0, s>>>(C.n, C.N, C.Ainv, M, Q);
  galerkin_schur_inv_kernel<<<1, 256, 0, s>>>(C.n, Q, M, G, d * c * e, C.Minv);
  count_launches(3);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_galerkin_coarse_solve(const CoarseData& C, const Stencil9& M, double c, double d, double e,
                                         Vec3c<T> f, Vec3<T> x, cudaStream_t s) {
  if (C.m > kMaxCoarseM || C.N > 1024) return cudaErrorInvalidValue;
  const int threads = std::max(32, std::min(1024, (std::max(C.N, C.m) + 31) / 32 * 32));
  galerkin_coarse_solve_kernel<T><<<1, threads, 0, s>>>(C.n, C.N, C.Ainv, C.Minv, M, c, d, e, f, x, C.wz);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_galerkin_coarse_solve<double>(const CoarseData&, const Stencil9&, double, double, double,
                                                          Vec3c<double>, Vec3<double>, cudaStream_t);
template cudaError_t launch_galerkin_coarse_solve<float>(const CoarseData&, const Stencil9&, double, double, double,
                                                         Vec3c<float>, Vec3<float>, cudaStream_t);

template cudaError_t launch_coarse_solve<double>(const CoarseData&, double, double, double, Vec3c<double>,
                                                 Vec3<double>, cudaStream_t, int);
template cudaError_t launch_coarse_solve<float>(const CoarseData&, double, double, double, Vec3c<float>,
                                                Vec3<float>, cudaStream_t, int);

}  // namespace cmg
