// Galerkin coarse operators (Sec. 3: S_l = P^T S_{l-1} P with the bilinear
// prolongation P and R = P^T), the operator the paper's experiments use.
//
// With P bilinear, the product of a 5- or 9-point stencil is a 9-point
// stencil on the coarse grid, so every coarse grid stores A_j as nine planes
// [9][n*n][N] (offset k = (dy+1)*3 + (dx+1), sample index fastest).  The
// mass blocks (fine: the identity times the scalars c, G, d, e) become
// c M_l, G M_l, d M_l, e M_l with one constant 9-point stencil M_l per grid:
// both the fine and the coarse nodes that enter an entry (C, D) of the
// product are interior, so the constant fine stencil gives a constant coarse
// one.
#include "cmg_common.cuh"

namespace cmg {

namespace {

constexpr int kGBlock = 256;
// grids up to this side take the one-launch residual (FP32, FP64: the
// one-launch form's extra FMAs per node-sample cost more in the FP64 pipe)
constexpr int kResidual9OnePass32 = 63, kResidual9OnePass64 = 31;
constexpr int kGsMaxR = 8;   // four-colour sweep: samples per lane held in registers (N <= 256)
constexpr long kGsHalfWarpNodes = 2048;   // FP32 grids from this many nodes per colour: 16 lanes per node

// The coarse nodes that a fine node 2C+1+g (one axis, g in [-2, 2]) takes
// its bilinear interpolant from, as offsets from C, with their weights: g
// even sits on the coarse node C + g/2 (weight 1); g odd lies halfway
// between C + (g-1)/2 and C + (g+1)/2 (1/2 each).
__host__ __device__ inline int coarse_targets(int g, int* off, double* wt) {
  if ((g & 1) == 0) {
    off[0] = g / 2;
    wt[0] = 1.0;
    return 1;
  }
  off[0] = (g - 1) / 2;
  off[1] = (g + 1) / 2;
  wt[0] = wt[1] = 0.5;
  return 2;
}

// One thread per (coarse node C, sample j): entry (C, C+o) of P^T A P is
// the sum over the fine nodes f of C's interpolation stencil (weight
// P(f, C)) and the fine neighbours g of f (operator entry A(f, g)) of
// P(f, C) A(f, g) P(g, C + o).  Fine nodes outside the grid are Dirichlet
// (no entry); coarse nodes outside the grid receive nothing.
__global__ void galerkin_setup_kernel(int nf, int N, const double* __restrict__ kx, const double* __restrict__ ky,
                                      const double* __restrict__ in9, double* __restrict__ out9) {
  const int nc = (nf - 1) / 2;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nc * nc * N) return;
  const int j = (int)(t % N);
  const long C = t / N;
  const int cy = (int)(C / nc), cx = (int)(C - (long)cy * nc);
  const size_t fnodes = (size_t)nf * nf, cnodes = (size_t)nc * nc;
  const double w1[3] = {0.5, 1.0, 0.5};
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b) {
      const int fy = 2 * cy + 1 + a, fx = 2 * cx + 1 + b;   // in [0, nf): nf = 2 nc + 1
      const double wf = w1[a + 1] * w1[b + 1];
      const long fnode = (long)fy * nf + fx;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int gy = fy + dy, gx = fx + dx;
          if (gy < 0 || gy >= nf || gx < 0 || gx >= nf) continue;
          double v;
          if (in9) {
            v = in9[((size_t)((dy + 1) * 3 + dx + 1) * fnodes + fnode) * N + j];
          } else {
            // the finest grid's 5-point stencil from its face coefficients
            const double kW = kx[((size_t)fy * (nf + 1) + fx) * N + j];
            const double kE = kx[((size_t)fy * (nf + 1) + fx + 1) * N + j];
            const double kS = ky[((size_t)fy * nf + fx) * N + j];
            const double kN = ky[((size_t)(fy + 1) * nf + fx) * N + j];
            if (dy == 0 && dx == 0) v = (kW + kE) + (kS + kN);
            else if (dy == 0) v = dx < 0 ? -kW : -kE;
            else if (dx == 0) v = dy < 0 ? -kS : -kN;
            else continue;   // corners: no entry
          }
          int oy[2], ox[2];
          double wy[2], wx[2];
          const int ny = coarse_targets(a + dy, oy, wy), nx = coarse_targets(b + dx, ox, wx);
          for (int p = 0; p < ny; ++p)
            for (int q = 0; q < nx; ++q) {
              const int Dy = cy + oy[p], Dx = cx + ox[q];
              if (Dy < 0 || Dy >= nc || Dx < 0 || Dx >= nc) continue;
              acc[(oy[p] + 1) * 3 + (ox[q] + 1)] += wf * v * (wy[p] * wx[q]);
            }
        }
    }
#pragma unroll
  for (int k = 0; k < 9; ++k) out9[((size_t)k * cnodes + C) * N + j] = acc[k];
}

// One warp per node, lanes over samples: inva = 1 / (A_j)_ii and
// isigma = 1 / (G + dce sum_j inva^2) (fixed-order shuffle reduction).
__global__ void galerkin_diag_kernel(long nodes, int N, const double* __restrict__ a9, double* __restrict__ inva,
                                     double* __restrict__ isigma, double dce, double G) {
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (node >= nodes) return;   // whole warp
  const double* centre = a9 + (size_t)4 * nodes * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) {
    const double ia = 1.0 / centre[(size_t)node * N + j];
    inva[(size_t)node * N + j] = ia;
    s += ia * ia;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) isigma[node] = 1.0 / (G + dce * s);
}

// T is the vectors' and the per-sample arithmetic's precision (FP64, or
// FP32 for the FP32 cycle on FP32 copies of the planes); the sums over
// samples and the control row are FP64 in both (for FP32: the lanes' partial
// sums over their own samples in FP32, converted once).

// The neighbours of node (iy, ix) in stencil order k = (dy+1)*3 + (dx+1);
// ok[k] false off the grid (Dirichlet: no entry), nb[k] then the node itself.
__device__ __forceinline__ void nine_neighbours(int n, int iy, int ix, bool* ok, int* nb) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ny = iy + k / 3 - 1, nx = ix + k % 3 - 1;
    ok[k] = ny >= 0 && ny < n && nx >= 0 && nx < n;
    nb[k] = ok[k] ? ny * n + nx : iy * n + ix;
  }
}

// psum[i] = sum_j p[i][j]: the lanes' parts in T, then a fixed-order FP64
// shuffle reduction; one warp per node (the three-launch residual and the
// four-colour sweep above 32 kGsMaxR samples).
template <typename T>
__global__ void galerkin_psum_kernel(long nodes, int N, const T* __restrict__ p, double* __restrict__ psum) {
  pdl_enter();
  const long node = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (node >= nodes) return;   // whole warp
  T sl = 0;   // this lane's part in T (FP32: converted once, as the sweeps' sums)
  for (int j = lane; j < N; j += 32) sl += p[(size_t)node * N + j];
  double s = (double)sl;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) psum[node] = s;
}

// Large grids: the residual as three launches in a programmatic-dependent
// chain (the per-node sums of p; the control row, which leaves (M u)_i in
// mu; the state and adjoint rows), one thread per (node, sample) for the
// last, whose FP64 pipe (27 FMAs per node-sample) sets the time there.
// State and adjoint rows, one thread per (node, sample):
//   r_y = f_y - (c (M y_j)_i + (A_j p_j)_i),  r_p = f_p - ((A_j y_j)_i + e (M u)_i),
// with (M u)_i from the control-row kernel (mu).
template <typename T>
__global__ void residual9_yp_kernel(int n, int N, const T* __restrict__ a9, Stencil9 M, double c, double e,
                                    const double* __restrict__ mu, Vec3c<T> x, Vec3c<T> f, Vec3<T> r) {
  pdl_enter();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nodes = (size_t)n * n;
  if (t >= (long)nodes * N) return;
  const int j = (int)(t % N);
  const long i = t / N;
  const int iy = (int)(i / n), ix = (int)(i - (long)iy * n);
  T Ap = 0, Ay = 0, My = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ny = iy + k / 3 - 1, nx = ix + k % 3 - 1;
    if (ny < 0 || ny >= n || nx < 0 || nx >= n) continue;
    const size_t nb = (size_t)ny * n + nx;
    const T a = a9[((size_t)k * nodes + i) * N + j];
    const T yv = x.y[nb * N + j], pv = x.p[nb * N + j];
    Ap = fma(a, pv, Ap);
    Ay = fma(a, yv, Ay);
    My = fma((T)M.w[k], yv, My);
  }
  const T sy = (T)c * My + Ap, sp = Ay + (T)e * (T)mu[i];
  const size_t o = (size_t)i * N + j;
  r.y[o] = f.y ? f.y[o] - sy : sy;
  r.p[o] = f.y ? f.p[o] - sp : sp;
}

// Control row, one thread per node (FP64): r_u = f_u - (G (M u)_i + d (M sum_j p_j)_i);
// (M u)_i is also left in mu.
template <typename T>
__global__ void residual9_u_kernel(int n, const double* __restrict__ psum, Stencil9 M, double G, double d,
                                   Vec3c<T> x, Vec3c<T> f, Vec3<T> r, double* __restrict__ mu) {
  pdl_enter();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)n * n) return;
  const int iy = (int)(i / n), ix = (int)(i - (long)iy * n);
  double Mu = 0.0, Mp = 0.0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int ny = iy + dy, nx = ix + dx;
      if (ny < 0 || ny >= n || nx < 0 || nx >= n) continue;
      const int k = (dy + 1) * 3 + (dx + 1);
      const size_t nb = (size_t)ny * n + nx;
      Mu = fma(M.w[k], (double)x.u[nb], Mu);
      Mp = fma(M.w[k], psum[nb], Mp);
    }
  const double su = G * Mu + d * Mp;
  r.u[i] = f.y ? (T)((double)f.u[i] - su) : (T)su;
  mu[i] = Mu;
}

// Small grids (launch-bound): the 9-point residual in one pass, one warp
// per node, lanes over samples:
//   r_y = f_y - (c (M y_j)_i + (A_j p_j)_i),
//   r_p = f_p - ((A_j y_j)_i + e (M u)_i),
//   r_u = f_u - (G (M u)_i + d sum_j (M p_j)_i).
// (M u)_i in FP64 by every lane (the same nine loads); the control row's
// sum over samples is formed from the p values the state rows load.
// r = S x when f.y == nullptr.
template <typename T>
__global__ void residual9_kernel(int n, int N, const T* __restrict__ a9, Stencil9 M, double c, double G, double d,
                                 double e, Vec3c<T> x, Vec3c<T> f, Vec3<T> r) {
  pdl_enter();
  const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const size_t nodes = (size_t)n * n;
  if (i >= (long)nodes) return;   // whole warp
  const int iy = (int)(i / n), ix = (int)(i - (long)iy * n);
  bool ok[9];
  int nb[9];
  nine_neighbours(n, iy, ix, ok, nb);
  double Mu = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (ok[k]) Mu = fma(M.w[k], (double)x.u[nb[k]], Mu);
  const T eMu = (T)(e * Mu), cT = (T)c;
  T pm = 0;   // this lane's share of sum_j (M p_j)_i
#pragma unroll 1
  for (int j = lane; j < N; j += 32) {
    T Ap = 0, Ay = 0, My = 0, Mp = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (!ok[k]) continue;
      const T a = a9[((size_t)k * nodes + i) * N + j];
      const T yv = x.y[(size_t)nb[k] * N + j], pv = x.p[(size_t)nb[k] * N + j];
      const T m = (T)M.w[k];
      Ap = fma(a, pv, Ap);
      Ay = fma(a, yv, Ay);
      My = fma(m, yv, My);
      Mp = fma(m, pv, Mp);
    }
    const T sy = cT * My + Ap, sp = Ay + eMu;
    const size_t o = (size_t)i * N + j;
    r.y[o] = f.y ? f.y[o] - sy : sy;
    r.p[o] = f.y ? f.p[o] - sp : sp;
    pm += Mp;
  }
  double ps = (double)pm;
  for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
  if (lane == 0) {
    const double su = G * Mu + d * ps;
    r.u[i] = f.y ? (T)((double)f.u[i] - su) : (T)su;
  }
}

// Collective Gauss-Seidel on a 9-point grid, one colour (iy mod 2, ix mod 2)
// = (cy, cx): no two nodes of a colour are coupled, so each node's block
// row is solved with its neighbours' current values (Eq. (13) with the
// diagonal entries of the Galerkin blocks; the variant named after Eq. (11)).
// One warp per node, lanes over samples.  Pass 1 forms the local right sides
//   B_y = f_y - sum_{k != centre} (c m_k y_k + A_k p_k),
//   B_p = f_p - sum_{k != centre} (A_k y_k + e m_k u_k),
//   B_u = f_u - sum_{k != centre} m_k (G u_k + d psum_k)
// and parks B_p, B_y in the node's own y, p slots (read by no other thread
// during this colour); pass 2 writes the solution and the node's new sum
// over samples of p.  c, G, d, e: the finest grid's; the diagonal entries are
// these times m_centre, a = (A_j)_ii; inva, isigma from galerkin_diag_kernel.
// The per-sample work is in T; B_u, the sum over samples for u (the lanes'
// partial sums converted once), 1/sigma and u are FP64.
template <typename T>
__global__ void gs4_colour_kernel(int n, int N, int cy, int cx, const T* __restrict__ a9, Stencil9 M, double c,
                                  double G, double d, double e, const T* __restrict__ inva,
                                  const double* __restrict__ isigma, Vec3<T> x, Vec3c<T> f,
                                  double* __restrict__ psum) {
  pdl_enter();
  const int nbx = (n - cx + 1) / 2, nby = (n - cy + 1) / 2;
  const long g = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (g >= (long)nbx * nby) return;   // whole warp
  const int iy = cy + 2 * (int)(g / nbx), ix = cx + 2 * (int)(g % nbx);
  const size_t nodes = (size_t)n * n;
  const size_t i = (size_t)iy * n + ix;
  const double mc = M.w[4];
  const T cd = (T)(c * mc), ed = (T)(e * mc);   // diagonal entries of the mass blocks
  const double dd = d * mc;
  // the eight neighbours (unrolled, predicated: all loads of a sample issue together)
  bool ok[9];
  size_t nbr[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ny = iy + k / 3 - 1, nx = ix + k % 3 - 1;
    ok[k] = k != 4 && ny >= 0 && ny < n && nx >= 0 && nx < n;
    nbr[k] = ok[k] ? (size_t)ny * n + nx : i;
  }
  double Bu = 0.0;
  if (lane == 0) {
    double s = (double)f.u[i];
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (ok[k]) s -= M.w[k] * (G * (double)x.u[nbr[k]] + d * psum[nbr[k]]);
    Bu = s;
  }
  double eMu = 0.0;   // e (M u)_i off the centre: the same for every sample
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (ok[k]) eMu += e * M.w[k] * (double)x.u[nbr[k]];
  const T eMuT = (T)eMu, cT = (T)c;
  T tacc = 0;
  for (int j = lane; j < N; j += 32) {
    T By = f.y[i * N + j], Bp = f.p[i * N + j] - eMuT;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (!ok[k]) continue;
      const T a = a9[((size_t)k * nodes + i) * N + j];
      const T yv = x.y[nbr[k] * N + j], pv = x.p[nbr[k] * N + j];
      By -= cT * (T)M.w[k] * yv + a * pv;
      Bp -= a * yv;
    }
    const T ia = inva[i * N + j];
    tacc += (cd * ia) * (ia * Bp) - ia * By;
    x.y[i * N + j] = Bp;   // parked until pass 2
    x.p[i * N + j] = By;
  }
  double ts = (double)tacc;
  for (int o = 16; o > 0; o >>= 1) ts += __shfl_xor_sync(0xffffffffu, ts, o);
  Bu = __shfl_sync(0xffffffffu, Bu, 0);
  const double u = (Bu + dd * ts) * isigma[i];
  const T uT = (T)u;
  double ps = 0.0;
  for (int j = lane; j < N; j += 32) {
    const T ia = inva[i * N + j];
    const T Bp = x.y[i * N + j], By = x.p[i * N + j];
    const T y = ia * (Bp - ed * uT);
    const T p = ia * (By - cd * y);
    x.y[i * N + j] = y;
    x.p[i * N + j] = p;
    ps += (double)p;
  }
  for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
  if (lane == 0) {
    x.u[i] = uT;
    psum[i] = ps;
  }
}

// The same colour sweep with each node's samples spread over LPN lanes
// (j = l + LPN q, q < R, N <= LPN R) and held in registers between the two
// passes, and the control row's sum over samples of the neighbours' (M p_j)
// formed from the p values the state rows load (no per-node sums kept
// between launches):
//   B_u = f_u - G (M u)_i - d sum_j (M p_j)_i   (off-centre entries, FP64).
// A warp takes 32 / LPN nodes, so each warp instruction of the node's FP64
// work (the off-centre (M u)_i, the two group sums, u_i) serves as many
// nodes: on this GPU the FP64 pipe, not memory, bounds a warp per node.
template <typename T, int R, int LPN>
__global__ void __launch_bounds__(kGBlock) gs4_colour_reg_kernel(int n, int N, int cy, int cx,
                                                                 const T* __restrict__ a9, Stencil9 M, double c,
                                                                 double G, double d, double e,
                                                                 const T* __restrict__ inva,
                                                                 const double* __restrict__ isigma, Vec3<T> x,
                                                                 Vec3c<T> f) {
  pdl_enter();
  const int nbx = (n - cx + 1) / 2, nby = (n - cy + 1) / 2;
  const long count = (long)nbx * nby;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~31L) / LPN >= count) return;   // the warp's first node is past the end: whole warp
  const long g = t / LPN;
  const int l = (int)(threadIdx.x & (LPN - 1));
  const bool valid = g < count;
  const int iy = valid ? cy + 2 * (int)(g / nbx) : 0, ix = valid ? cx + 2 * (int)(g % nbx) : 0;
  const size_t nodes = (size_t)n * n;
  const size_t i = (size_t)iy * n + ix;
  const double mc = M.w[4];
  const T cd = (T)(c * mc), ed = (T)(e * mc);   // diagonal entries of the mass blocks
  bool ok[9];
  int nb[9];
  nine_neighbours(n, iy, ix, ok, nb);
  ok[4] = false;
  double Mu = 0.0;   // off-centre (M u)_i
  if (valid) {
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (ok[k]) Mu = fma(M.w[k], (double)x.u[nb[k]], Mu);
  }
  const T eMu = (T)(e * Mu), cT = (T)c;
  T By[R], Bp[R], ia[R];
  T tacc = 0, pm = 0;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = l + LPN * q;
    By[q] = Bp[q] = ia[q] = 0;
    if (valid && j < N) {
      T by = f.y[i * N + j], bp = f.p[i * N + j] - eMu, mp = 0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        if (!ok[k]) continue;
        const T a = a9[((size_t)k * nodes + i) * N + j];
        const T yv = x.y[(size_t)nb[k] * N + j], pv = x.p[(size_t)nb[k] * N + j];
        const T m = (T)M.w[k];
        by -= cT * m * yv + a * pv;
        bp -= a * yv;
        mp = fma(m, pv, mp);
      }
      const T iq = inva[i * N + j];
      tacc += (cd * iq) * (iq * bp) - iq * by;
      pm += mp;
      By[q] = by;
      Bp[q] = bp;
      ia[q] = iq;
    }
  }
  double ts = (double)tacc, ps = (double)pm;
  for (int o = LPN / 2; o > 0; o >>= 1) {
    ts += __shfl_xor_sync(0xffffffffu, ts, o);
    ps += __shfl_xor_sync(0xffffffffu, ps, o);
  }
  if (!valid) return;
  const double Bu = (double)f.u[i] - G * Mu - d * ps;
  const double u = (Bu + d * mc * ts) * isigma[i];
  const T uT = (T)u;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = l + LPN * q;
    if (j < N) {
      const T y = ia[q] * (Bp[q] - ed * uT);
      x.y[i * N + j] = y;
      x.p[i * N + j] = ia[q] * (By[q] - cd * y);
    }
  }
  if (l == 0) x.u[i] = uT;
}

// Damped collective Jacobi on a 9-point grid: x_i += theta S~_i^{-1} r_i with
// S~_i the node's block with the Galerkin diagonal entries (Eq. (11), Eq. (13)
// on the residual).  LPN lanes per node (32, or 16 on large FP32 grids, as
// the colour kernel), lanes over samples; per-sample work in T, the sum over
// samples and the u correction in FP64.
template <typename T, int LPN>
__global__ void galerkin_jacobi_kernel(long nodes, int N, Stencil9 M, double c, double d, double e, double theta,
                                       const T* __restrict__ inva, const double* __restrict__ isigma, Vec3<T> x,
                                       Vec3c<T> r) {
  pdl_enter();
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if ((t & ~31L) / LPN >= nodes) return;   // the warp's first node is past the end: whole warp
  const long i = t / LPN;
  const int l = (int)(threadIdx.x & (LPN - 1));
  const bool valid = i < nodes;
  const double mc = M.w[4];
  const T cd = (T)(c * mc), ed = (T)(e * mc);
  T tacc = 0;
  if (valid) {
    for (int j = l; j < N; j += LPN) {
      const T ia = inva[(size_t)i * N + j];
      tacc += (cd * ia) * (ia * r.p[(size_t)i * N + j]) - ia * r.y[(size_t)i * N + j];
    }
  }
  double ts = (double)tacc;
  for (int o = LPN / 2; o > 0; o >>= 1) ts += __shfl_xor_sync(0xffffffffu, ts, o);
  if (!valid) return;
  const double du = ((double)r.u[i] + d * mc * ts) * isigma[i];
  const T duT = (T)du, th = (T)theta;
  for (int j = l; j < N; j += LPN) {
    const size_t o = (size_t)i * N + j;
    const T ia = inva[o];
    const T dy = ia * (r.p[o] - ed * duT);
    const T dp = ia * (r.y[o] - cd * dy);
    x.y[o] += th * dy;
    x.p[o] += th * dp;
  }
  if (l == 0) x.u[i] += (T)(theta * du);
}

unsigned blocks_for(long threads) { return (unsigned)((threads + kGBlock - 1) / kGBlock); }

}  // namespace

Stencil9 galerkin_mass(const Stencil9& fine) {
  // the setup kernel's triple product with a constant stencil and no grid
  // boundary (every node entering an interior entry is interior)
  Stencil9 out{};
  const double w1[3] = {0.5, 1.0, 0.5};
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const double v = fine.w[(dy + 1) * 3 + dx + 1];
          if (v == 0.0) continue;
          int oy[2], ox[2];
          double wy[2], wx[2];
          const int ny = coarse_targets(a + dy, oy, wy), nx = coarse_targets(b + dx, ox, wx);
          for (int p = 0; p < ny; ++p)
            for (int q = 0; q < nx; ++q)
              out.w[(oy[p] + 1) * 3 + (ox[q] + 1)] += w1[a + 1] * w1[b + 1] * v * (wy[p] * wx[q]);
        }
  return out;
}

cudaError_t launch_galerkin_setup(int nf, int N, const double* kx, const double* ky, const double* in9, double* out9,
                                  cudaStream_t s) {
  const int nc = (nf - 1) / 2;
  const long threads = (long)nc * nc * N;
  if (threads == 0) return cudaSuccess;
  galerkin_setup_kernel<<<blocks_for(threads), kGBlock, 0, s>>>(nf, N, kx, ky, in9, out9);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_galerkin_diag(int n, int N, const double* a9, double* inva, double* isigma, double dce, double G,
                                 cudaStream_t s) {
  const long nodes = (long)n * n;
  galerkin_diag_kernel<<<blocks_for(nodes * 32), kGBlock, 0, s>>>(nodes, N, a9, inva, isigma, dce, G);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual9(int n, int N, const T* a9, const Stencil9& M, double c, double G, double d, double e,
                             Vec3c<T> x, Vec3c<T> f, Vec3<T> r, double* psum, cudaStream_t s) {
  const long nodes = (long)n * n;
  if (n <= (sizeof(T) == 4 ? kResidual9OnePass32 : kResidual9OnePass64)) {
    const cudaError_t err =
        launch_k(residual9_kernel<T>, blocks_for(nodes * 32), kGBlock, 0, s, n, N, a9, M, c, G, d, e, x, f, r);
    count_launches(1);
    return err != cudaSuccess ? err : cudaGetLastError();
  }
  double* mu = psum + nodes;
  cudaError_t err = launch_k(galerkin_psum_kernel<T>, blocks_for(nodes * 32), kGBlock, 0, s, nodes, N, x.p, psum);
  if (err == cudaSuccess)
    err = launch_k(residual9_u_kernel<T>, blocks_for(nodes), kGBlock, 0, s, n, (const double*)psum, M, G, d, x, f, r,
                   mu);
  if (err == cudaSuccess)
    err = launch_k(residual9_yp_kernel<T>, blocks_for(nodes * N), kGBlock, 0, s, n, N, a9, M, c, e,
                   (const double*)mu, x, f, r);
  count_launches(3);
  return err != cudaSuccess ? err : cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs4_sweep(int n, int N, const T* a9, const Stencil9& M, double c, double G, double d, double e,
                             const T* inva, const double* isigma, Vec3<T> x, Vec3c<T> f, double* psum,
                             cudaStream_t s) {
  const long nodes = (long)n * n;
  if (N <= 32 * kGsMaxR) {
    // samples in registers: four launches, nothing kept between them.  FP32
    // on grids of at least kGsHalfWarpNodes nodes per colour, up to 64
    // samples: 16 lanes per node (two nodes per warp share the FP64 work);
    // elsewhere a warp per node (smaller grids want the warps, and in FP64
    // the per-sample work outweighs the per-node)
    const long colour_nodes = (long)((n + 1) / 2) * ((n + 1) / 2);
    const int lpn = (sizeof(T) == 4 && N <= 64 && colour_nodes >= kGsHalfWarpNodes) ? 16 : 32;
    const int need = (N + lpn - 1) / lpn;
    const int R = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : 8;
    cudaError_t err = cudaSuccess;
    for (int col = 0; col < 4 && err == cudaSuccess; ++col) {
      const int cy = col >> 1, cx = col & 1;
      const long groups = (long)((n - cx + 1) / 2) * ((n - cy + 1) / 2);
      if (groups == 0) continue;
      const unsigned grid = blocks_for(groups * lpn);
#define CMG_GS4(RR, LL)                                                                                         \
  err = launch_k(gs4_colour_reg_kernel<T, RR, LL>, grid, kGBlock, 0, s, n, N, cy, cx, a9, M, c, G, d, e, inva, \
                 isigma, x, f)
      if (lpn == 16) {
        if (R == 1) CMG_GS4(1, 16);
        else if (R == 2) CMG_GS4(2, 16);
        else CMG_GS4(4, 16);
      } else {
        if (R == 1) CMG_GS4(1, 32);
        else if (R == 2) CMG_GS4(2, 32);
        else if (R == 4) CMG_GS4(4, 32);
        else CMG_GS4(8, 32);
      }
#undef CMG_GS4
    }
    count_launches(4);
    return err != cudaSuccess ? err : cudaGetLastError();
  }
  // more samples: park the local right sides in x between the two passes,
  // with the per-node sums over samples of p in psum
  cudaError_t err = launch_k(galerkin_psum_kernel<T>, blocks_for(nodes * 32), kGBlock, 0, s, nodes, N,
                             (const T*)x.p, psum);
  for (int col = 0; col < 4 && err == cudaSuccess; ++col) {
    const int cy = col >> 1, cx = col & 1;
    const long groups = (long)((n - cx + 1) / 2) * ((n - cy + 1) / 2);
    if (groups == 0) continue;
    err = launch_k(gs4_colour_kernel<T>, blocks_for(groups * 32), kGBlock, 0, s, n, N, cy, cx, a9, M, c, G, d, e,
                   inva, isigma, x, f, psum);
  }
  count_launches(5);
  return err != cudaSuccess ? err : cudaGetLastError();
}

template <typename T>
cudaError_t launch_galerkin_jacobi(int n, int N, const Stencil9& M, double c, double d, double e, double theta,
                                   const T* inva, const double* isigma, Vec3<T> x, Vec3c<T> r, cudaStream_t s) {
  const long nodes = (long)n * n;
  // two nodes per warp where the colour kernel takes them (its node count
  // per colour is a quarter of the grid's)
  const int lpn = (sizeof(T) == 4 && N <= 64 && nodes >= 4 * kGsHalfWarpNodes) ? 16 : 32;
  const cudaError_t err =
      lpn == 16 ? launch_k(galerkin_jacobi_kernel<T, 16>, blocks_for(nodes * 16), kGBlock, 0, s, nodes, N, M, c, d, e,
                           theta, inva, isigma, x, r)
                : launch_k(galerkin_jacobi_kernel<T, 32>, blocks_for(nodes * 32), kGBlock, 0, s, nodes, N, M, c, d, e,
                           theta, inva, isigma, x, r);
  count_launches(1);
  return err != cudaSuccess ? err : cudaGetLastError();
}

template cudaError_t launch_residual9<double>(int, int, const double*, const Stencil9&, double, double, double,
                                              double, Vec3c<double>, Vec3c<double>, Vec3<double>, double*,
                                              cudaStream_t);
template cudaError_t launch_residual9<float>(int, int, const float*, const Stencil9&, double, double, double, double,
                                             Vec3c<float>, Vec3c<float>, Vec3<float>, double*, cudaStream_t);
template cudaError_t launch_gs4_sweep<double>(int, int, const double*, const Stencil9&, double, double, double,
                                              double, const double*, const double*, Vec3<double>, Vec3c<double>,
                                              double*, cudaStream_t);
template cudaError_t launch_gs4_sweep<float>(int, int, const float*, const Stencil9&, double, double, double, double,
                                             const float*, const double*, Vec3<float>, Vec3c<float>, double*,
                                             cudaStream_t);
template cudaError_t launch_galerkin_jacobi<float>(int, int, const Stencil9&, double, double, double, double,
                                                   const float*, const double*, Vec3<float>, Vec3c<float>,
                                                   cudaStream_t);

}  // namespace cmg
