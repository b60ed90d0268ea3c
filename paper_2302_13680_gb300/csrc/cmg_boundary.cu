// Neumann boundary control on Gamma = (0,1) x {0} (Sec. 2's control operator
// B as a Neumann condition; the boundary-control test case of Sec. 3.2),
// solved by collective multigrid with Galerkin coarse operators (Sec. 3).
//
// Grids: n interior columns (x = (ix+1) h, Dirichlet at x = 0 and 1) and
// n + 1 rows (y = r h, r = 0..n; row 0 on Gamma, Dirichlet at y = 1); node
// r n + ix.  Every block of the optimality system is a 9-point stencil per
// node: A_j as nine planes [9][nodes][N] (offset k = (dy+1)*3 + (dx+1)), the
// mass M as nine planes [9][nodes]; the control lives on the n row-0 nodes,
// where G (the control mass) and B (the control-to-adjoint coupling) are
// 3-point stencils along Gamma.  System (the symmetric scaling of Sec. 2):
//     (M/N) y_j + A_j p_j     = f_y,j
//     G u       - B^T sum_j p_j = f_u
//     A_j y_j   - B u          = f_p,j
// Finest grid: A_j the dual-cell 5-point stencil with harmonic-mean faces,
// the x-faces of row 0 halved and no south face there (its flux is the
// control); lumped M = h^2 (h^2 / 2 on row 0); G = nu h I, B = h I on Gamma.
// Coarse grids: S_{l+1} = P^T S_l P with P = P_y (x) P_x for y and p (row 0
// stays on Gamma: fine row 2R is coarse row R, odd fine rows interpolate,
// the top one against the Dirichlet value) and P_x for u, so A_j and M stay
// 9-point and G, B 3-point.  Smoother: damped collective Jacobi, Eq. (11),
// each node's block solved by Eq. (13) on Gamma (2N+1 unknowns) and by
// Eq. (14) elsewhere (u_i = 0); coarsest grid: block elimination.  All FP64.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cmg_common.cuh"

using namespace cmg;

namespace {

constexpr int kBT = 256;
constexpr int kBndMaxLevels = 12;

inline unsigned bblocks(long threads) { return (unsigned)((threads + kBT - 1) / kBT); }

struct BLev {
  int n = 0;                 // interior columns; n + 1 rows
  size_t nodes = 0;          // (n + 1) n
  double* a9 = nullptr;      // [9][nodes][N]
  double* m9 = nullptr;      // [9][nodes]
  double* inva = nullptr;    // [nodes][N] 1 / (A_j)_ii
  double* isigma = nullptr;  // [n] 1 / Schur denominator of Eq. (13) on Gamma
  double* psum = nullptr;    // [n] scratch: sum_j p_j on row 0
  double g3[3] = {0, 0, 0};  // G along Gamma (offsets -1, 0, +1)
  double b3[3] = {0, 0, 0};  // B along Gamma
  double* x[3] = {nullptr, nullptr, nullptr};
  double* f[3] = {nullptr, nullptr, nullptr};
  double* r[3] = {nullptr, nullptr, nullptr};
};

// One thread per (point, sample) of the (n+2) x (n+2) points x = f h,
// y = r h (f, r = 0..n+1): kappa_j = exp(amp sum_k xi_jk sin(k pi x) sin(pi y) / k).
__global__ void bnd_field_kernel(int n, int N, int K, double amp, const double* __restrict__ xi,
                                 double* __restrict__ kap) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long pts = (long)(n + 2) * (n + 2);
  if (t >= pts * N) return;
  const int j = (int)(t % N);
  const long q = t / N;
  const int r = (int)(q / (n + 2)), fx = (int)(q % (n + 2));
  const double h = 1.0 / (n + 1);
  const double x = fx * h, y = r * h;
  const double sy = sin(M_PI * y);
  double g = 0.0;
  for (int k = 1; k <= K; ++k) g += xi[(size_t)j * K + (k - 1)] * sin(k * M_PI * x) / k;
  kap[t] = exp(amp * g * sy);
}

__device__ __forceinline__ double hmean(double a, double b) { return 2.0 * a * b / (a + b); }

// Finest-grid planes from the field: one thread per (node, sample).
__global__ void bnd_finest_kernel(int n, int N, double h, const double* __restrict__ kap, double* __restrict__ a9,
                                  double* __restrict__ m9) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nodes = (size_t)(n + 1) * n;
  if (t >= (long)nodes * N) return;
  const int j = (int)(t % N);
  const long i = t / N;
  const int r = (int)(i / n), ix = (int)(i % n);
  const auto K = [&](int rr, int ff) { return kap[((size_t)rr * (n + 2) + ff) * N + j]; };   // point (x = ff h, y = rr h)
  const double s = r == 0 ? 0.5 : 1.0;
  // node (r, ix) sits at point (r, ix + 1)
  const double kW = s * hmean(K(r, ix), K(r, ix + 1));
  const double kE = s * hmean(K(r, ix + 1), K(r, ix + 2));
  const double kN = hmean(K(r, ix + 1), K(r + 1, ix + 1));
  const double kS = r > 0 ? hmean(K(r - 1, ix + 1), K(r, ix + 1)) : 0.0;
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  v[4] = (kW + kE) + (kS + kN);
  if (ix > 0) v[3] = -kW;
  if (ix < n - 1) v[5] = -kE;
  if (r > 0) v[1] = -kS;
  if (r < n) v[7] = -kN;
#pragma unroll
  for (int k = 0; k < 9; ++k) a9[((size_t)k * nodes + i) * N + j] = v[k];
  if (j == 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) m9[(size_t)k * nodes + i] = 0.0;
    m9[(size_t)4 * nodes + i] = r == 0 ? 0.5 * h * h : h * h;
  }
}

// Weights of the boundary-grid prolongation.  Rows: fine row 2R is coarse
// row R; fine row 2R+1 takes half of rows R and R+1 (R+1 <= nc).  Columns:
// coarse column I sits on fine column 2I+1 (interior rule).
__device__ __forceinline__ double py(int fy, int R) {
  const int d = fy - 2 * R;
  return d == 0 ? 1.0 : (d == 1 || d == -1) ? 0.5 : 0.0;
}
__device__ __forceinline__ double px(int fx, int I) {
  const int d = fx - (2 * I + 1);
  return d == 0 ? 1.0 : (d == 1 || d == -1) ? 0.5 : 0.0;
}

// Galerkin product P^T A P for one 9-point operator with S samples (S = N for
// A_j, S = 1 for the mass): one thread per (coarse node C, sample j); entry
// (C, C+o) = sum over the fine nodes f of C's interpolation stencil and f's
// neighbours g of P(f, C) A(f, g) P(g, C+o).
__global__ void bnd_galerkin_kernel(int nf, int S, const double* __restrict__ in9, double* __restrict__ out9) {
  const int nc = (nf - 1) / 2;
  const size_t fnodes = (size_t)(nf + 1) * nf, cnodes = (size_t)(nc + 1) * nc;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)cnodes * S) return;
  const int j = (int)(t % S);
  const long C = t / S;
  const int R = (int)(C / nc), I = (int)(C % nc);
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (int fy = 2 * R - 1; fy <= 2 * R + 1; ++fy) {
    if (fy < 0 || fy > nf) continue;
    const double wy = py(fy, R);
    for (int fx = 2 * I; fx <= 2 * I + 2; ++fx) {
      const double wf = wy * px(fx, I);
      const size_t fn = (size_t)fy * nf + fx;
      for (int k = 0; k < 9; ++k) {
        const int gy = fy + k / 3 - 1, gx = fx + k % 3 - 1;
        if (gy < 0 || gy > nf || gx < 0 || gx >= nf) continue;
        const double a = in9[((size_t)k * fnodes + fn) * S + j];
        if (a == 0.0) continue;
        for (int oy = -1; oy <= 1; ++oy) {
          const int Dy = R + oy;
          if (Dy < 0 || Dy > nc) continue;
          const double wgy = py(gy, Dy);
          if (wgy == 0.0) continue;
          for (int ox = -1; ox <= 1; ++ox) {
            const int Dx = I + ox;
            if (Dx < 0 || Dx >= nc) continue;
            const double wgx = px(gx, Dx);
            if (wgx == 0.0) continue;
            acc[(oy + 1) * 3 + (ox + 1)] += wf * a * (wgy * wgx);
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) out9[((size_t)k * cnodes + C) * S + j] = acc[k];
}

// One warp per node: inva = 1 / (A_j)_ii; on Gamma also
// isigma = 1 / (G_ii + dce_i sum_j inva^2), dce_i = B_ii^2 M_ii / N.
__global__ void bnd_diag_kernel(int n, int N, const double* __restrict__ a9, const double* __restrict__ m9,
                                double g0, double b0, double* __restrict__ inva, double* __restrict__ isigma) {
  const size_t nodes = (size_t)(n + 1) * n;
  const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (long)nodes) return;   // whole warp
  const double* centre = a9 + (size_t)4 * nodes * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) {
    const double ia = 1.0 / centre[(size_t)i * N + j];
    inva[(size_t)i * N + j] = ia;
    s += ia * ia;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0 && i < n) {
    const double dce = b0 * b0 * m9[(size_t)4 * nodes + i] / N;
    isigma[i] = 1.0 / (g0 + dce * s);
  }
}

// psum[ix] = sum_j p[(0, ix)][j] on Gamma: one warp per row-0 node.
__global__ void bnd_psum_kernel(int n, int N, const double* __restrict__ p, double* __restrict__ psum) {
  const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) s += p[(size_t)i * N + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) psum[i] = s;
}

struct St3 {
  double w[3];
};

// State and adjoint rows, one thread per (node, sample):
//   r_y = f_y - ((M y_j)_i / N + (A_j p_j)_i),   r_p = f_p - ((A_j y_j)_i - (B u)_i)
// (r = S x when f is null).
__global__ void bnd_residual_yp_kernel(int n, int N, const double* __restrict__ a9, const double* __restrict__ m9,
                                       St3 b3, Vec3c<double> x, Vec3c<double> f, Vec3<double> r) {
  const size_t nodes = (size_t)(n + 1) * n;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)nodes * N) return;
  const int j = (int)(t % N);
  const long i = t / N;
  const int ry = (int)(i / n), rx = (int)(i % n);
  double Ap = 0.0, Ay = 0.0, My = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int gy = ry + k / 3 - 1, gx = rx + k % 3 - 1;
    if (gy < 0 || gy > n || gx < 0 || gx >= n) continue;
    const size_t g = (size_t)gy * n + gx;
    const double a = a9[((size_t)k * nodes + i) * N + j];
    const double yv = x.y[g * N + j], pv = x.p[g * N + j];
    Ap = fma(a, pv, Ap);
    Ay = fma(a, yv, Ay);
    My = fma(m9[(size_t)k * nodes + i], yv, My);
  }
  double Bu = 0.0;
  if (ry == 0)
    for (int d = -1; d <= 1; ++d)
      if (rx + d >= 0 && rx + d < n) Bu = fma(b3.w[d + 1], x.u[rx + d], Bu);
  const double sy = My / N + Ap, sp = Ay - Bu;
  const size_t o = (size_t)i * N + j;
  r.y[o] = f.y ? f.y[o] - sy : sy;
  r.p[o] = f.y ? f.p[o] - sp : sp;
}

// Control rows on Gamma: r_u = f_u - ((G u)_k - (B^T psum)_k).
__global__ void bnd_residual_u_kernel(int n, St3 g3, St3 b3, const double* __restrict__ psum, Vec3c<double> x,
                                      Vec3c<double> f, Vec3<double> r) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double Gu = 0.0, Bp = 0.0;
  for (int d = -1; d <= 1; ++d) {
    if (k + d < 0 || k + d >= n) continue;
    Gu = fma(g3.w[d + 1], x.u[k + d], Gu);
    Bp = fma(b3.w[1 - d], psum[k + d], Bp);   // (B^T)_{k, k+d} = B_{k+d, k}
  }
  const double su = Gu - Bp;
  r.u[k] = f.y ? f.u[k] - su : su;
}

// Damped collective Jacobi, Eq. (11): x_i += theta S~_i^{-1} r_i, one warp
// per node.  On Gamma the node block is Eq. (12)'s arrow system with
// c = M_ii / N, a_j = (A_j)_ii, d = e = -B_ii, G = G_ii, solved by Eq. (13);
// elsewhere u_i is absent (Eq. (14)).
__global__ void bnd_jacobi_kernel(int n, int N, const double* __restrict__ m9, const double* __restrict__ inva,
                                  const double* __restrict__ isigma, double b0, double theta, Vec3<double> x,
                                  Vec3c<double> r) {
  const size_t nodes = (size_t)(n + 1) * n;
  const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= (long)nodes) return;   // whole warp
  const double c = m9[(size_t)4 * nodes + i] / N;
  const bool gam = i < n;
  const double d = -b0, e = -b0;
  double du = 0.0;
  if (gam) {
    double t = 0.0;
    for (int j = lane; j < N; j += 32) {
      const double ia = inva[(size_t)i * N + j];
      t += (c * ia) * (ia * r.p[(size_t)i * N + j]) - ia * r.y[(size_t)i * N + j];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    du = (r.u[i] + d * t) * isigma[i];
  }
  for (int j = lane; j < N; j += 32) {
    const size_t o = (size_t)i * N + j;
    const double ia = inva[o];
    const double dy = ia * (r.p[o] - e * du);
    const double dp = ia * (r.y[o] - c * dy);
    x.y[o] += theta * dy;
    x.p[o] += theta * dp;
  }
  if (gam && lane == 0) x.u[i] += theta * du;
}

// c = P^T r from the nf grid to the (nf-1)/2 grid, one thread per (coarse
// node, sample); the control block (sample slot 0 of row-0 nodes) by P_x^T.
__global__ void bnd_restrict_kernel(int nf, int N, Vec3c<double> rf, Vec3<double> cc) {
  const int nc = (nf - 1) / 2;
  const size_t cnodes = (size_t)(nc + 1) * nc;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)cnodes * N) return;
  const int j = (int)(t % N);
  const long C = t / N;
  const int R = (int)(C / nc), I = (int)(C % nc);
  double ay = 0.0, ap = 0.0;
  for (int fy = 2 * R - 1; fy <= 2 * R + 1; ++fy) {
    if (fy < 0 || fy > nf) continue;
    for (int fx = 2 * I; fx <= 2 * I + 2; ++fx) {
      const double w = py(fy, R) * px(fx, I);
      const size_t o = ((size_t)fy * nf + fx) * N + j;
      ay = fma(w, rf.y[o], ay);
      ap = fma(w, rf.p[o], ap);
    }
  }
  cc.y[(size_t)C * N + j] = ay;
  cc.p[(size_t)C * N + j] = ap;
  if (j == 0 && R == 0) {
    double au = 0.0;
    for (int fx = 2 * I; fx <= 2 * I + 2; ++fx) au = fma(px(fx, I), rf.u[fx], au);
    cc.u[I] = au;
  }
}

// x_f += P e_c, one thread per (fine node, sample); u by P_x.
__global__ void bnd_prolong_kernel(int nf, int N, Vec3c<double> ec, Vec3<double> xf) {
  const int nc = (nf - 1) / 2;
  const size_t fnodes = (size_t)(nf + 1) * nf;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)fnodes * N) return;
  const int j = (int)(t % N);
  const long F = t / N;
  const int fy = (int)(F / nf), fx = (int)(F % nf);
  const int R0 = fy / 2, R1 = (fy + 1) / 2;   // the coarse rows (equal when fy is even)
  const int I0 = (fx - 1) / 2, I1 = fx / 2;    // the coarse columns (equal when fx is odd)
  double vy = 0.0, vp = 0.0;
  for (int R = R0; R <= R1; ++R) {
    if (R > nc) continue;
    for (int I = (fx - 1 < 0 ? 0 : I0); I <= I1; ++I) {
      if (I < 0 || I >= nc) continue;
      const double w = py(fy, R) * px(fx, I);
      if (w == 0.0) continue;
      const size_t o = ((size_t)R * nc + I) * N + j;
      vy = fma(w, ec.y[o], vy);
      vp = fma(w, ec.p[o], vp);
    }
  }
  xf.y[(size_t)F * N + j] += vy;
  xf.p[(size_t)F * N + j] += vp;
  if (j == 0 && fy == 0) {
    double vu = 0.0;
    for (int I = I0; I <= I1; ++I)
      if (I >= 0 && I < nc) vu = fma(px(fx, I), ec.u[I], vu);
    xf.u[fx] += vu;
  }
}

// ---- coarsest grid: block elimination --------------------------------------
// y_j = A_j^{-1} (f_p,j + B u), p_j = A_j^{-1} (f_y,j - (M/N) y_j), and the
// control from (G + B^T Q B) u = f_u + B^T sum_j (w_j - A_j^{-1} (M/N) z_j)
// with Q = sum_j A_j^{-1} (M/N) A_j^{-1}, w_j = A_j^{-1} f_y,j, z_j = A_j^{-1} f_p,j.

// Dense A_j (m x m) of the coarsest grid and its inverse by Gauss-Jordan with
// partial pivoting, one CTA per sample.
__global__ void bnd_coarse_inv_kernel(int n, int N, const double* __restrict__ a9, double* __restrict__ Ainv) {
  const int m = (n + 1) * n;
  const int j = blockIdx.x;
  extern __shared__ double sm[];
  double* A = sm;            // [m][m]
  double* X = sm + m * m;    // [m][m]
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    A[t] = 0.0;
    X[t] = (t / m == t % m) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int ry = i / n, rx = i % n;
    for (int k = 0; k < 9; ++k) {
      const int gy = ry + k / 3 - 1, gx = rx + k % 3 - 1;
      if (gy < 0 || gy > n || gx < 0 || gx >= n) continue;
      A[i * m + gy * n + gx] = a9[((size_t)k * m + i) * N + j];
    }
  }
  __syncthreads();
  __shared__ int piv;
  for (int col = 0; col < m; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double best = fabs(A[col * m + col]);
      for (int rr = col + 1; rr < m; ++rr)
        if (fabs(A[rr * m + col]) > best) {
          best = fabs(A[rr * m + col]);
          p = rr;
        }
      piv = p;
    }
    __syncthreads();
    if (piv != col)
      for (int t = threadIdx.x; t < m; t += blockDim.x) {
        double a = A[col * m + t];
        A[col * m + t] = A[piv * m + t];
        A[piv * m + t] = a;
        a = X[col * m + t];
        X[col * m + t] = X[piv * m + t];
        X[piv * m + t] = a;
      }
    __syncthreads();
    const double inv = 1.0 / A[col * m + col];
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      A[col * m + t] *= inv;
      X[col * m + t] *= inv;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int rr = t / m, cc = t % m;
      if (rr == col) continue;
      const double fct = A[rr * m + col];
      if (cc != col) A[rr * m + cc] -= fct * A[col * m + cc];
      X[rr * m + cc] -= fct * X[col * m + cc];
    }
    __syncthreads();
    for (int rr = threadIdx.x; rr < m; rr += blockDim.x)
      if (rr != col) A[rr * m + col] = 0.0;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) Ainv[(size_t)j * m * m + t] = X[t];
}

// The control Schur matrix Z = G + B^T Q B (nc x nc, nc = n controls) and
// its inverse, one CTA (small: n <= 7).
__global__ void bnd_coarse_schur_kernel(int n, int N, const double* __restrict__ Ainv, const double* __restrict__ m9,
                                        St3 g3, St3 b3, double* __restrict__ Zinv) {
  const int m = (n + 1) * n;
  extern __shared__ double sm[];
  double* Q = sm;                 // [m][m]
  double* Mm = Q + m * m;         // [m][m] dense mass / N
  double* T = Mm + m * m;         // [m][m] scratch
  double* Z = T + m * m;          // [n][n]
  double* Zi = Z + n * n;         // [n][n]
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    Q[t] = 0.0;
    Mm[t] = 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int ry = i / n, rx = i % n;
    for (int k = 0; k < 9; ++k) {
      const int gy = ry + k / 3 - 1, gx = rx + k % 3 - 1;
      if (gy < 0 || gy > n || gx < 0 || gx >= n) continue;
      Mm[i * m + gy * n + gx] = m9[(size_t)k * m + i] / N;
    }
  }
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    const double* Ai = Ainv + (size_t)j * m * m;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {   // T = (M/N) A_j^{-1}
      const int rr = t / m, cc = t % m;
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += Mm[rr * m + k] * Ai[k * m + cc];
      T[t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {   // Q += A_j^{-1} T
      const int rr = t / m, cc = t % m;
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += Ai[rr * m + k] * T[k * m + cc];
      Q[t] += s;
    }
    __syncthreads();
  }
  // Z = G + B^T Q B, B [m][n]: B[(0, ix)][k] = b3[k - ix + 1]
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int a = t / n, b = t % n;
    double s = (b - a >= -1 && b - a <= 1) ? g3.w[b - a + 1] : 0.0;
    for (int p = 0; p < n; ++p) {
      const double Bpa = (a - p >= -1 && a - p <= 1) ? b3.w[a - p + 1] : 0.0;
      if (Bpa == 0.0) continue;
      for (int q = 0; q < n; ++q) {
        const double Bqb = (b - q >= -1 && b - q <= 1) ? b3.w[b - q + 1] : 0.0;
        if (Bqb != 0.0) s += Bpa * Q[p * m + q] * Bqb;
      }
    }
    Z[t] = s;
    Zi[t] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // Gauss-Jordan with partial pivoting on the n x n Schur matrix
    for (int col = 0; col < n; ++col) {
      int p = col;
      for (int rr = col + 1; rr < n; ++rr)
        if (fabs(Z[rr * n + col]) > fabs(Z[p * n + col])) p = rr;
      for (int t = 0; t < n; ++t) {
        double v = Z[col * n + t];
        Z[col * n + t] = Z[p * n + t];
        Z[p * n + t] = v;
        v = Zi[col * n + t];
        Zi[col * n + t] = Zi[p * n + t];
        Zi[p * n + t] = v;
      }
      const double inv = 1.0 / Z[col * n + col];
      for (int t = 0; t < n; ++t) {
        Z[col * n + t] *= inv;
        Zi[col * n + t] *= inv;
      }
      for (int rr = 0; rr < n; ++rr) {
        if (rr == col) continue;
        const double fct = Z[rr * n + col];
        for (int t = 0; t < n; ++t) {
          Z[rr * n + t] -= fct * Z[col * n + t];
          Zi[rr * n + t] -= fct * Zi[col * n + t];
        }
      }
    }
    for (int t = 0; t < n * n; ++t) Zinv[t] = Zi[t];
  }
}

// x = S^{-1} f on the coarsest grid, one CTA; work: [4][N][m] doubles.
__global__ void bnd_coarse_solve_kernel(int n, int N, const double* __restrict__ Ainv,
                                        const double* __restrict__ m9, const double* __restrict__ Zinv, St3 b3,
                                        Vec3c<double> f, Vec3<double> x, double* __restrict__ work) {
  const int m = (n + 1) * n;
  double* w = work;                  // [N][m] A^{-1} f_y
  double* z = w + (size_t)N * m;     // [N][m] A^{-1} f_p, later y
  double* t = z + (size_t)N * m;     // [N][m] scratch
  double* q = t + (size_t)N * m;     // [N][m] scratch
  __shared__ double rhs[64], us[64];
  const auto Mv = [&](const double* v, int i) {   // ((M / N) v)_i on the coarsest grid
    const int ry = i / n, rx = i % n;
    double s = 0.0;
    for (int k = 0; k < 9; ++k) {
      const int gy = ry + k / 3 - 1, gx = rx + k % 3 - 1;
      if (gy < 0 || gy > n || gx < 0 || gx >= n) continue;
      s += m9[(size_t)k * m + i] * v[gy * n + gx];
    }
    return s / N;
  };
  for (int s = threadIdx.x; s < N * m; s += blockDim.x) {
    const int j = s / m, i = s % m;
    const double* Ai = Ainv + (size_t)j * m * m + (size_t)i * m;
    double sw = 0.0, sz = 0.0;
    for (int k = 0; k < m; ++k) {
      sw += Ai[k] * f.y[(size_t)k * N + j];
      sz += Ai[k] * f.p[(size_t)k * N + j];
    }
    w[s] = sw;
    z[s] = sz;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < N * m; s += blockDim.x) t[s] = Mv(z + (size_t)(s / m) * m, s % m);
  __syncthreads();
  for (int s = threadIdx.x; s < N * m; s += blockDim.x) {   // q = w - A^{-1} (M/N) z
    const int j = s / m, i = s % m;
    const double* Ai = Ainv + (size_t)j * m * m + (size_t)i * m;
    double v = 0.0;
    for (int k = 0; k < m; ++k) v += Ai[k] * t[(size_t)j * m + k];
    q[s] = w[s] - v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {   // rhs = f_u + B^T sum_j q_j (row-0 nodes)
    double s = f.u[k];
    for (int d = -1; d <= 1; ++d) {
      const int ix = k + d;
      if (ix < 0 || ix >= n) continue;
      double sq = 0.0;
      for (int j = 0; j < N; ++j) sq += q[(size_t)j * m + ix];
      s += b3.w[1 - d] * sq;   // (B^T)_{k, ix} = B_{ix, k}
    }
    rhs[k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double u = 0.0;
    for (int c = 0; c < n; ++c) u += Zinv[k * n + c] * rhs[c];
    us[k] = u;
    x.u[k] = u;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < N * m; s += blockDim.x) {   // y = z + A^{-1} B u
    const int j = s / m, i = s % m;
    const double* Ai = Ainv + (size_t)j * m * m + (size_t)i * m;
    double v = 0.0;
    for (int ix = 0; ix < n; ++ix) {   // (B u) lives on row 0
      double bu = 0.0;
      for (int d = -1; d <= 1; ++d)
        if (ix + d >= 0 && ix + d < n) bu += b3.w[d + 1] * us[ix + d];
      v += Ai[ix] * bu;
    }
    t[s] = z[s] + v;   // y_j
  }
  __syncthreads();
  for (int s = threadIdx.x; s < N * m; s += blockDim.x) {
    const int j = s / m, i = s % m;
    x.y[(size_t)i * N + j] = t[s];
    q[s] = Mv(t + (size_t)j * m, i);   // (M/N) y_j
  }
  __syncthreads();
  for (int s = threadIdx.x; s < N * m; s += blockDim.x) {   // p = w - A^{-1} (M/N) y
    const int j = s / m, i = s % m;
    const double* Ai = Ainv + (size_t)j * m * m + (size_t)i * m;
    double v = 0.0;
    for (int k = 0; k < m; ++k) v += Ai[k] * q[(size_t)j * m + k];
    x.p[(size_t)i * N + j] = w[s] - v;
  }
}

// Sum of squares with the state block weighted by wy^2, fixed-order per block.
__global__ void bnd_sumsq_kernel(const double* __restrict__ a, size_t n, double w2, double* __restrict__ partial) {
  __shared__ double sh[kBT / 32];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(a[i], a[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kBT / 32; ++k) t += sh[k];
    partial[blockIdx.x] = t * w2;
  }
}

}  // namespace

struct cmg_bnd {
  int n = 0, N = 0, K = 0, L = 0;
  double nu = 0, amp = 0;
  cudaStream_t stream = nullptr;
  BLev lv[kBndMaxLevels];
  double* xi = nullptr;
  double* Ainv = nullptr;     // coarsest [N][m][m]
  double* Zinv = nullptr;     // coarsest control Schur inverse [nc][nc]
  double* work = nullptr;     // coarsest solve scratch [4][N][m]
  double* part = nullptr;     // norm partials
  double* hpart = nullptr;    // pinned host copy
  std::vector<void*> allocs;
  std::string err;
};

namespace {

constexpr int kNormBlocks = 152;

cmg_status bfail(cmg_bnd* h, cmg_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

cmg_status bcuda(cmg_bnd* h, cudaError_t e, const char* what) {
  const cmg_status st = e == cudaErrorMemoryAllocation ? CMG_ERR_OOM : CMG_ERR_CUDA;
  (void)cudaGetLastError();
  return bfail(h, st, std::string(what) + ": " + cudaGetErrorString(e));
}

#define BK(call)                                           \
  do {                                                     \
    const cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return bcuda(h, e_, #call);     \
  } while (0)

template <typename T>
cudaError_t balloc(cmg_bnd* h, T** p, size_t count) {
  void* q = nullptr;
  const cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

// 3-point stencil of P_x^T S P_x along Gamma from a fine 3-point stencil S
// (constant along the line; exact at the Dirichlet ends, whose dropped
// terms map outside the coarse line).
void line_galerkin(const double* fine, double* coarse) {
  const double w[3] = {0.5, 1.0, 0.5};
  for (int o = 0; o < 3; ++o) coarse[o] = 0.0;
  for (int a = -1; a <= 1; ++a)        // fine node 2C+1+a of coarse node C's stencil
    for (int d = -1; d <= 1; ++d) {    // its neighbour g = 2C+1+a+d
      const double v = fine[d + 1];
      if (v == 0.0) continue;
      const int gg = a + d;             // g relative to 2C+1
      // coarse nodes C+o with P(g, C+o) != 0: 2(C+o)+1 within one of g
      for (int o = -1; o <= 1; ++o) {
        const int dd = gg - 2 * o;
        const double pw = dd == 0 ? 1.0 : (dd == 1 || dd == -1) ? 0.5 : 0.0;
        if (pw != 0.0) coarse[o + 1] += w[a + 1] * v * pw;
      }
    }
}

Vec3<double> vx(const BLev& v, double* const* a) { return {a[0], a[1], a[2]}; }

cmg_status vec_ok3(const double* y, const double* u, const double* p) {
  const auto a16 = [](const void* q) { return q && (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  return (a16(y) && a16(u) && a16(p)) ? CMG_OK : CMG_ERR_INVALID_ARG;
}

cudaError_t residual(cmg_bnd* h, int l, Vec3c<double> x, Vec3c<double> f, Vec3<double> r) {
  const BLev& v = h->lv[l];
  const int N = h->N;
  St3 g3{{v.g3[0], v.g3[1], v.g3[2]}}, b3{{v.b3[0], v.b3[1], v.b3[2]}};
  bnd_psum_kernel<<<bblocks((long)v.n * 32), kBT, 0, h->stream>>>(v.n, N, x.p, v.psum);
  bnd_residual_yp_kernel<<<bblocks((long)v.nodes * N), kBT, 0, h->stream>>>(v.n, N, v.a9, v.m9, b3, x, f, r);
  bnd_residual_u_kernel<<<bblocks(v.n), kBT, 0, h->stream>>>(v.n, g3, b3, v.psum, x, f, r);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t smooth(cmg_bnd* h, int l, double theta, int sweeps, Vec3<double> x, Vec3c<double> f) {
  BLev& v = h->lv[l];
  const Vec3<double> r = vx(v, v.r);
  for (int s = 0; s < sweeps; ++s) {
    cudaError_t e = residual(h, l, cview(x), f, r);
    if (e != cudaSuccess) return e;
    bnd_jacobi_kernel<<<bblocks((long)v.nodes * 32), kBT, 0, h->stream>>>(v.n, h->N, v.m9, v.inva, v.isigma, v.b3[1],
                                                                          theta, x, cview(r));
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t restrict_to(cmg_bnd* h, int l, Vec3c<double> r, Vec3<double> c) {
  const BLev& v = h->lv[l + 1];
  bnd_restrict_kernel<<<bblocks((long)v.nodes * h->N), kBT, 0, h->stream>>>(h->lv[l].n, h->N, r, c);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t prolong_add(cmg_bnd* h, int l, Vec3c<double> e, Vec3<double> x) {
  const BLev& v = h->lv[l];
  bnd_prolong_kernel<<<bblocks((long)v.nodes * h->N), kBT, 0, h->stream>>>(v.n, h->N, e, x);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t coarse_solve(cmg_bnd* h, Vec3c<double> f, Vec3<double> x) {
  const BLev& v = h->lv[h->L - 1];
  St3 b3{{v.b3[0], v.b3[1], v.b3[2]}};
  bnd_coarse_solve_kernel<<<1, kBT, 0, h->stream>>>(v.n, h->N, h->Ainv, v.m9, h->Zinv, b3, f, x, h->work);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t zero3(cmg_bnd* h, int l, Vec3<double> x) {
  const BLev& v = h->lv[l];
  cudaError_t e = cudaMemsetAsync(x.y, 0, v.nodes * h->N * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x.u, 0, v.n * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x.p, 0, v.nodes * h->N * sizeof(double), h->stream);
  return e;
}

// Algorithm 1 on grid l (gamma = 1: V-cycle, 2: W-cycle) with damped
// collective Jacobi and the direct solve on the coarsest grid.
cudaError_t cycle(cmg_bnd* h, int l, double theta, int n1, int n2, int gamma, Vec3<double> x, Vec3c<double> f) {
  if (l == h->L - 1) return coarse_solve(h, f, x);
  BLev& v = h->lv[l];
  BLev& c = h->lv[l + 1];
  cudaError_t e = smooth(h, l, theta, n1, x, f);
  const Vec3<double> r = vx(v, v.r), fc = vx(c, c.f), xc = vx(c, c.x);
  if (e == cudaSuccess) e = residual(h, l, cview(x), f, r);
  if (e == cudaSuccess) e = restrict_to(h, l, cview(r), fc);
  if (e == cudaSuccess) e = zero3(h, l + 1, xc);
  for (int g = 0; g < gamma && e == cudaSuccess; ++g) e = cycle(h, l + 1, theta, n1, n2, gamma, xc, cview(fc));
  if (e == cudaSuccess) e = prolong_add(h, l, cview(xc), x);
  if (e == cudaSuccess) e = smooth(h, l, theta, n2, x, f);
  return e;
}

// ||W v|| of a finest-grid vector, W = diag(N I, 1, 1) (the paper's row
// scaling); synchronises.
cmg_status paper_norm(cmg_bnd* h, Vec3c<double> v, double* out) {
  const BLev& l0 = h->lv[0];
  const size_t ny = l0.nodes * h->N;
  const double wy2 = (double)h->N * h->N;
  bnd_sumsq_kernel<<<kNormBlocks, kBT, 0, h->stream>>>(v.y, ny, wy2, h->part);
  bnd_sumsq_kernel<<<kNormBlocks, kBT, 0, h->stream>>>(v.u, (size_t)l0.n, 1.0, h->part + kNormBlocks);
  bnd_sumsq_kernel<<<kNormBlocks, kBT, 0, h->stream>>>(v.p, ny, 1.0, h->part + 2 * kNormBlocks);
  count_launches(3);
  BK(cudaGetLastError());
  BK(cudaMemcpyAsync(h->hpart, h->part, 3 * kNormBlocks * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  BK(cudaStreamSynchronize(h->stream));
  double s = 0.0;
  for (int k = 0; k < 3 * kNormBlocks; ++k) s += h->hpart[k];
  *out = std::sqrt(s);
  return CMG_OK;
}

bool lev_ok(const cmg_bnd* h, int l) { return h && l >= 0 && l < h->L; }

}  // namespace

extern "C" {

cmg_status cmg_bnd_create(int n, int N, int K, double nu, double amp, int coarsest_n, const double* xi_host,
                          void* stream, cmg_bnd** out) {
  if (!out) return CMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || n > 4095 || ((n + 1) & n) != 0 || N < 1 || N > 1024 || K < 0 || K > 64 || !(nu > 0.0) ||
      !std::isfinite(amp) || (K > 0 && !xi_host))
    return CMG_ERR_INVALID_ARG;
  if (coarsest_n != 1 && coarsest_n != 3 && coarsest_n != 7) return CMG_ERR_INVALID_ARG;
  if (coarsest_n > n) return CMG_ERR_INVALID_ARG;
  cmg_bnd* h = new (std::nothrow) cmg_bnd;
  if (!h) return CMG_ERR_OOM;
  h->n = n;
  h->N = N;
  h->K = K;
  h->nu = nu;
  h->amp = amp;
  h->stream = static_cast<cudaStream_t>(stream);
  int L = 0;
  for (int m = n;; m = (m - 1) / 2) {
    if (L >= kBndMaxLevels) {
      delete h;
      return CMG_ERR_INVALID_ARG;
    }
    h->lv[L].n = m;
    h->lv[L].nodes = (size_t)(m + 1) * m;
    ++L;
    if (m == coarsest_n) break;
  }
  h->L = L;
  cudaError_t e = cudaSuccess;
  const auto fin = [&](cudaError_t err) {
    const cmg_status st = err == cudaErrorMemoryAllocation ? CMG_ERR_OOM : CMG_ERR_CUDA;
    (void)cudaGetLastError();
    cmg_bnd_destroy(h);
    return st;
  };
  for (int l = 0; l < L && e == cudaSuccess; ++l) {
    BLev& v = h->lv[l];
    e = balloc(h, &v.a9, 9 * v.nodes * N);
    if (e == cudaSuccess) e = balloc(h, &v.m9, 9 * v.nodes);
    if (e == cudaSuccess) e = balloc(h, &v.inva, v.nodes * N);
    if (e == cudaSuccess) e = balloc(h, &v.isigma, (size_t)v.n);
    if (e == cudaSuccess) e = balloc(h, &v.psum, (size_t)v.n);
    for (int b = 0; b < 3 && e == cudaSuccess; ++b) {
      const size_t cnt = b == 1 ? (size_t)v.n : v.nodes * N;
      e = balloc(h, &v.x[b], cnt);
      if (e == cudaSuccess) e = balloc(h, &v.f[b], cnt);
      if (e == cudaSuccess) e = balloc(h, &v.r[b], cnt);
    }
  }
  const BLev& cl = h->lv[L - 1];
  const int m = (int)cl.nodes;
  double* kap = nullptr;
  if (e == cudaSuccess) e = balloc(h, &h->xi, (size_t)N * (K > 0 ? K : 1));
  if (e == cudaSuccess) e = balloc(h, &kap, (size_t)(n + 2) * (n + 2) * N);
  if (e == cudaSuccess) e = balloc(h, &h->Ainv, (size_t)N * m * m);
  if (e == cudaSuccess) e = balloc(h, &h->Zinv, (size_t)cl.n * cl.n);
  if (e == cudaSuccess) e = balloc(h, &h->work, (size_t)4 * N * m);
  if (e == cudaSuccess) e = balloc(h, &h->part, 3 * kNormBlocks);
  if (e == cudaSuccess) e = cudaMallocHost(&h->hpart, 3 * kNormBlocks * sizeof(double));
  if (e != cudaSuccess) return fin(e);
  if (K > 0) e = cudaMemcpy(h->xi, xi_host, (size_t)N * K * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fin(e);
  // finest grid
  const double hh = 1.0 / (n + 1);
  bnd_field_kernel<<<bblocks((long)(n + 2) * (n + 2) * N), kBT, 0, h->stream>>>(n, N, K, amp, h->xi, kap);
  bnd_finest_kernel<<<bblocks((long)h->lv[0].nodes * N), kBT, 0, h->stream>>>(n, N, hh, kap, h->lv[0].a9,
                                                                              h->lv[0].m9);
  count_launches(2);
  h->lv[0].g3[1] = nu * hh;
  h->lv[0].b3[1] = hh;
  // coarse grids: Galerkin products
  for (int l = 1; l < L; ++l) {
    BLev& v = h->lv[l];
    const BLev& fv = h->lv[l - 1];
    bnd_galerkin_kernel<<<bblocks((long)v.nodes * N), kBT, 0, h->stream>>>(fv.n, N, fv.a9, v.a9);
    bnd_galerkin_kernel<<<bblocks((long)v.nodes), kBT, 0, h->stream>>>(fv.n, 1, fv.m9, v.m9);
    count_launches(2);
    line_galerkin(fv.g3, v.g3);
    line_galerkin(fv.b3, v.b3);
  }
  for (int l = 0; l < L; ++l) {
    BLev& v = h->lv[l];
    bnd_diag_kernel<<<bblocks((long)v.nodes * 32), kBT, 0, h->stream>>>(v.n, N, v.a9, v.m9, v.g3[1], v.b3[1],
                                                                         v.inva, v.isigma);
    count_launches(1);
  }
  // coarsest factors
  const size_t inv_smem = 2 * (size_t)m * m * sizeof(double);
  const size_t schur_smem = (3 * (size_t)m * m + 2 * (size_t)cl.n * cl.n) * sizeof(double);
  if (inv_smem > 200 * 1024 || schur_smem > 200 * 1024) {
    cmg_bnd_destroy(h);
    return CMG_ERR_UNSUPPORTED;
  }
  e = cudaFuncSetAttribute(bnd_coarse_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(bnd_coarse_schur_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return fin(e);
  bnd_coarse_inv_kernel<<<N, kBT, inv_smem, h->stream>>>(cl.n, N, cl.a9, h->Ainv);
  St3 g3{{cl.g3[0], cl.g3[1], cl.g3[2]}}, b3{{cl.b3[0], cl.b3[1], cl.b3[2]}};
  bnd_coarse_schur_kernel<<<1, kBT, schur_smem, h->stream>>>(cl.n, N, h->Ainv, cl.m9, g3, b3, h->Zinv);
  count_launches(2);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fin(e);
  *out = h;
  return CMG_OK;
}

void cmg_bnd_destroy(cmg_bnd* h) {
  if (!h) return;
  for (void* p : h->allocs) (void)cudaFree(p);
  if (h->hpart) (void)cudaFreeHost(h->hpart);
  delete h;
}

const char* cmg_bnd_last_error(const cmg_bnd* h) { return h ? h->err.c_str() : "null handle"; }
int cmg_bnd_num_levels(const cmg_bnd* h) { return h ? h->L : 0; }
int cmg_bnd_level_n(const cmg_bnd* h, int level) { return lev_ok(h, level) ? h->lv[level].n : -1; }

cmg_status cmg_bnd_rhs(cmg_bnd* h, const double* yd, const double* fsrc, double* fy, double* fu, double* fp) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!yd || vec_ok3(fy, fu, fp) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "null or misaligned pointer");
  // f = ((M y_d)/N broadcast over samples, 0, M f) with the finest (diagonal) mass
  const BLev& v = h->lv[0];
  const int n = v.n, N = h->N;
  const double hh = 1.0 / (n + 1);
  std::vector<double> w(v.nodes);
  for (size_t i = 0; i < v.nodes; ++i) w[i] = (i < (size_t)n ? 0.5 : 1.0) * hh * hh;
  std::vector<double> hyd(v.nodes), hf(v.nodes, 0.0), ty(v.nodes * N), tp(v.nodes * N);
  BK(cudaMemcpyAsync(hyd.data(), yd, v.nodes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (fsrc) BK(cudaMemcpyAsync(hf.data(), fsrc, v.nodes * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  BK(cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < v.nodes; ++i)
    for (int j = 0; j < N; ++j) {
      ty[i * N + j] = w[i] * hyd[i] / N;
      tp[i * N + j] = w[i] * hf[i];
    }
  BK(cudaMemcpyAsync(fy, ty.data(), ty.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  BK(cudaMemsetAsync(fu, 0, (size_t)n * sizeof(double), h->stream));
  BK(cudaMemcpyAsync(fp, tp.data(), tp.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  BK(cudaStreamSynchronize(h->stream));
  return CMG_OK;
}

cmg_status cmg_bnd_residual(cmg_bnd* h, int level, const double* y, const double* u, const double* p,
                            const double* fy, const double* fu, const double* fp, double* ry, double* ru,
                            double* rp) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!lev_ok(h, level)) return bfail(h, CMG_ERR_INVALID_ARG, "level out of range");
  if (vec_ok3(y, u, p) != CMG_OK || vec_ok3(ry, ru, rp) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  if ((fy || fu || fp) && vec_ok3(fy, fu, fp) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "partial right side");
  BK(residual(h, level, {y, u, p}, {fy, fu, fp}, {ry, ru, rp}));
  return CMG_OK;
}

cmg_status cmg_bnd_smooth(cmg_bnd* h, int level, double theta, int sweeps, double* y, double* u, double* p,
                          const double* fy, const double* fu, const double* fp) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!lev_ok(h, level)) return bfail(h, CMG_ERR_INVALID_ARG, "level out of range");
  if (vec_ok3(y, u, p) != CMG_OK || vec_ok3(fy, fu, fp) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  if (!(theta > 0.0 && theta <= 1.0) || sweeps < 0) return bfail(h, CMG_ERR_INVALID_ARG, "theta or sweeps");
  BK(smooth(h, level, theta, sweeps, {y, u, p}, {fy, fu, fp}));
  return CMG_OK;
}

cmg_status cmg_bnd_restrict(cmg_bnd* h, int level, const double* ry, const double* ru, const double* rp, double* cy,
                            double* cu, double* cp) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!lev_ok(h, level) || level == h->L - 1) return bfail(h, CMG_ERR_INVALID_ARG, "level out of range");
  if (vec_ok3(ry, ru, rp) != CMG_OK || vec_ok3(cy, cu, cp) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  BK(restrict_to(h, level, {ry, ru, rp}, {cy, cu, cp}));
  return CMG_OK;
}

cmg_status cmg_bnd_prolong_add(cmg_bnd* h, int level, const double* ey, const double* eu, const double* ep,
                               double* y, double* u, double* p) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!lev_ok(h, level) || level == h->L - 1) return bfail(h, CMG_ERR_INVALID_ARG, "level out of range");
  if (vec_ok3(ey, eu, ep) != CMG_OK || vec_ok3(y, u, p) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  BK(prolong_add(h, level, {ey, eu, ep}, {y, u, p}));
  return CMG_OK;
}

cmg_status cmg_bnd_coarse_solve(cmg_bnd* h, const double* fy, const double* fu, const double* fp, double* y,
                                double* u, double* p) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (vec_ok3(fy, fu, fp) != CMG_OK || vec_ok3(y, u, p) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  BK(coarse_solve(h, {fy, fu, fp}, {y, u, p}));
  return CMG_OK;
}

cmg_status cmg_bnd_cycle(cmg_bnd* h, double theta, int n1, int n2, int gamma, double* y, double* u, double* p,
                         const double* fy, const double* fu, const double* fp) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (vec_ok3(y, u, p) != CMG_OK || vec_ok3(fy, fu, fp) != CMG_OK) return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  if (!(theta > 0.0 && theta <= 1.0) || n1 < 0 || n2 < 0 || n1 > 64 || n2 > 64 || gamma < 1 || gamma > 2)
    return bfail(h, CMG_ERR_INVALID_ARG, "cycle options out of range");
  BK(cycle(h, 0, theta, n1, n2, gamma, {y, u, p}, {fy, fu, fp}));
  return CMG_OK;
}

cmg_status cmg_bnd_solve(cmg_bnd* h, double theta, int n1, int n2, int gamma, double tol, int maxit,
                         const double* fy, const double* fu, const double* fp, double* y, double* u, double* p,
                         cmg_stats* stats) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (vec_ok3(y, u, p) != CMG_OK || vec_ok3(fy, fu, fp) != CMG_OK || !stats)
    return bfail(h, CMG_ERR_INVALID_ARG, "bad pointer");
  if (!(theta > 0.0 && theta <= 1.0) || n1 < 0 || n2 < 0 || n1 > 64 || n2 > 64 || gamma < 1 || gamma > 2 ||
      !(tol > 0.0) || maxit < 0)
    return bfail(h, CMG_ERR_INVALID_ARG, "options out of range");
  BLev& l0 = h->lv[0];
  const Vec3<double> r = vx(l0, l0.r);
  double fn = 0.0, rho = 0.0;
  cmg_status st = paper_norm(h, {fy, fu, fp}, &fn);
  if (st != CMG_OK) return st;
  BK(residual(h, 0, {y, u, p}, {fy, fu, fp}, r));
  if ((st = paper_norm(h, cview(r), &rho)) != CMG_OK) return st;
  *stats = cmg_stats{};
  stats->relres0 = fn > 0.0 ? rho / fn : 0.0;
  int it = 0;
  while (std::isfinite(rho) && rho > tol * fn && it < maxit) {
    BK(cycle(h, 0, theta, n1, n2, gamma, {y, u, p}, {fy, fu, fp}));
    ++it;
    BK(residual(h, 0, {y, u, p}, {fy, fu, fp}, r));
    if ((st = paper_norm(h, cview(r), &rho)) != CMG_OK) return st;
  }
  stats->iters = stats->cycles = it;
  stats->relres = fn > 0.0 ? rho / fn : 0.0;
  if (!std::isfinite(rho)) return bfail(h, CMG_ERR_NONFINITE, "residual norm not finite");
  if (rho > tol * fn) return bfail(h, CMG_ERR_NOT_CONVERGED, "maxit reached");
  return CMG_OK;
}

}  // extern "C"
