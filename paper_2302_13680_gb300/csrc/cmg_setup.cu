// Coefficient setup (FP64 arithmetic).  Finest grid (and every grid in the
// nodal variant):
//   nodal field kappa_j at the (n+2)^2 grid points including the boundary
//   (the sine-mode log-Gaussian stand-in for Eq. (15): kappa = exp(amp *
//   sin(pi y) * sum_k xi_jk sin(k pi x) / k), which is separable in x and y),
//   harmonic-mean face coefficients, 1/diag(A_j) and the Schur denominators
//   sigma_i = G + sum_j d c e / a_ij^2 of Eq. (13).
// Coarse grids (averaged variant): faces averaged from the next finer grid,
// then the same 1/diag and sigma.
#include "cmg_common.cuh"

namespace cmg {

namespace {

// gx[ix][j] = sum_k xi[j][k] sin(k pi x_ix) / k, x_ix = ix h, ix = 0..n+1.
__global__ void field_x_kernel(int n, int N, int K, const double* __restrict__ xi, double* __restrict__ gx) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)(n + 2) * N) return;
  const int ix = (int)(t / N), j = (int)(t - (long)ix * N);
  const double x = (double)ix / (double)(n + 1);
  double g = 0.0;
  for (int k = 1; k <= K; ++k) g += xi[(size_t)j * K + (k - 1)] * sinpi((double)k * x) / (double)k;
  gx[t] = g;
}

// kap[iy][ix][j] = exp(amp * sin(pi y_iy) * gx[ix][j]) on the (n+2)^2 grid.
// sin(pi y) is symmetric about y = 1/2 (rows iy and n+1-iy), so each
// exponential is evaluated once for both rows (the FP64 exponential is the
// cost of this kernel on a GPU with a narrow FP64 pipe); the boundary rows
// have sin(pi y) = 0, kappa = 1.
__global__ void field_kernel(int n, int N, double amp, const double* __restrict__ gx, double* __restrict__ kap) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = (n + 1) / 2;   // rows 0 .. half; n + 1 is even
  const long total = (long)(half + 1) * (n + 2) * N;
  if (t >= total) return;
  const long node = t / N;
  const int j = (int)(t - node * N);
  const int iy = (int)(node / (n + 2)), ix = (int)(node - (long)iy * (n + 2));
  const double v = iy == 0 ? 1.0 : exp(amp * sinpi((double)iy / (double)(n + 1)) * gx[(size_t)ix * N + j]);
  kap[((size_t)iy * (n + 2) + ix) * N + j] = v;
  const int mirror = n + 1 - iy;
  if (mirror != iy) kap[((size_t)mirror * (n + 2) + ix) * N + j] = v;
}

__device__ __forceinline__ double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

// kx[iy][f][j] between grid columns f and f+1 of interior row iy (grid row iy+1);
// ky[f][ix][j] between grid rows f and f+1 of interior column ix.
__global__ void faces_kernel(int n, int N, const double* __restrict__ kap, double* __restrict__ kx64,
                             double* __restrict__ ky64, float* __restrict__ kx32, float* __restrict__ ky32) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)n * (n + 1) * N;
  if (t >= 2 * per) return;
  const size_t g = (size_t)(n + 2);
  if (t < per) {
    const long face = t / N;
    const int j = (int)(t - face * N);
    const int iy = (int)(face / (n + 1)), f = (int)(face - (long)iy * (n + 1));
    const double v = harmonic(kap[((iy + 1) * g + f) * N + j], kap[((iy + 1) * g + f + 1) * N + j]);
    kx64[t] = v;
    kx32[t] = (float)v;
  } else {
    const long tt = t - per;
    const long face = tt / N;
    const int j = (int)(tt - face * N);
    const int f = (int)(face / n), ix = (int)(face - (long)f * n);
    const double v = harmonic(kap[((size_t)f * g + ix + 1) * N + j], kap[((size_t)(f + 1) * g + ix + 1) * N + j]);
    ky64[tt] = v;
    ky32[tt] = (float)v;
  }
}

// inva[node][j] = 1 / (sum of the node's four faces); isigma[node] = 1 /
// (Schur denominator), its sum over samples reduced by one warp per node in
// a fixed order.
__global__ void diag_kernel(int n, int N, const double* __restrict__ kx, const double* __restrict__ ky,
                            double* __restrict__ inva, double* __restrict__ isigma, double dce, double G,
                            const float* __restrict__ dw = nullptr) {
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long)n * n) return;
  const int iy = (int)(warp / n), ix = (int)(warp - (long)iy * n);
  const double* kW = kx + ((size_t)iy * (n + 1) + ix) * N;
  const double* kS = ky + ((size_t)iy * n + ix) * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) {
    const double a = (kW[j] + kW[N + j]) + (kS[j] + kS[(size_t)n * N + j]);
    const double ia = 1.0 / a;
    inva[(size_t)warp * N + j] = ia;
    s += ia * ia;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) isigma[warp] = 1.0 / (G + (dw ? dce * (double)dw[warp] : dce) * s);   // d_i = d dw_i
}

// Coarse faces averaged from the next finer grid (nf = 2 nc + 1): a coarse
// face spans two fine faces in series (harmonic mean) on each of three fine
// lines across it, combined with weights 1/4, 1/2, 1/4.
__global__ void coarse_faces_kernel(int nf, int N, const double* __restrict__ kxf, const double* __restrict__ kyf,
                                    double* __restrict__ kx64, double* __restrict__ ky64, float* __restrict__ kx32,
                                    float* __restrict__ ky32) {
  const int nc = (nf - 1) / 2;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)nc * (nc + 1) * N;
  if (t >= 2 * per) return;
  const double w[3] = {0.25, 0.5, 0.25};
  double v = 0.0;
  if (t < per) {
    const long face = t / N;
    const int j = (int)(t - face * N);
    const int J = (int)(face / (nc + 1)), I = (int)(face - (long)J * (nc + 1));
    for (int k = 0; k < 3; ++k) {
      const size_t row = (size_t)(2 * J + k) * (nf + 1);
      v += w[k] * harmonic(kxf[(row + 2 * I) * N + j], kxf[(row + 2 * I + 1) * N + j]);
    }
    kx64[t] = v;
    if (kx32) kx32[t] = (float)v;
  } else {
    const long tt = t - per;
    const long face = tt / N;
    const int j = (int)(tt - face * N);
    const int J = (int)(face / nc), I = (int)(face - (long)J * nc);
    for (int k = 0; k < 3; ++k) {
      const size_t col = (size_t)(2 * I + k);
      v += w[k] * harmonic(kyf[((size_t)(2 * J) * nf + col) * N + j], kyf[((size_t)(2 * J + 1) * nf + col) * N + j]);
    }
    ky64[tt] = v;
    if (ky32) ky32[tt] = (float)v;
  }
}

// The same averaging in FP32 from the finer grid's FP32 faces: the FP32
// cycle's coarse operators, built without the FP64 pipe.
__global__ void coarse_faces32_kernel(int nf, int N, const float* __restrict__ kxf, const float* __restrict__ kyf,
                                      float* __restrict__ kx32, float* __restrict__ ky32) {
  const int nc = (nf - 1) / 2;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)nc * (nc + 1) * N;
  if (t >= 2 * per) return;
  const float w[3] = {0.25f, 0.5f, 0.25f};
  const auto hm = [](float a, float b) { return 2.0f * a * b / (a + b); };
  float v = 0.f;
  if (t < per) {
    const long face = t / N;
    const int j = (int)(t - face * N);
    const int J = (int)(face / (nc + 1)), I = (int)(face - (long)J * (nc + 1));
    for (int k = 0; k < 3; ++k) {
      const size_t row = (size_t)(2 * J + k) * (nf + 1);
      v += w[k] * hm(kxf[(row + 2 * I) * N + j], kxf[(row + 2 * I + 1) * N + j]);
    }
    kx32[t] = v;
  } else {
    const long tt = t - per;
    const long face = tt / N;
    const int j = (int)(tt - face * N);
    const int J = (int)(face / nc), I = (int)(face - (long)J * nc);
    for (int k = 0; k < 3; ++k) {
      const size_t col = (size_t)(2 * I + k);
      v += w[k] * hm(kyf[((size_t)(2 * J) * nf + col) * N + j], kyf[((size_t)(2 * J + 1) * nf + col) * N + j]);
    }
    ky32[tt] = v;
  }
}

// 1/sigma_i = 1 / (G + dce sum_j 1/a_j^2) of the FP32 operator: a_j from the
// FP32 faces and 1/a_j in FP32 as the FP32 sweeps form them, the sum over
// samples and the quotient in FP64; written in FP64 (isigma_d, read by the
// FP32 cycle's Schur scalar) and rounded to FP32 (isigma32, all-FP32 option).
__global__ void diag32_kernel(int n, int N, const float* __restrict__ kx, const float* __restrict__ ky,
                              float* __restrict__ isigma32, double* __restrict__ isigma_d, double dce, double G,
                              const float* __restrict__ dw) {
  const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long)n * n) return;
  const int iy = (int)(warp / n), ix = (int)(warp - (long)iy * n);
  const float* kW = kx + ((size_t)iy * (n + 1) + ix) * N;
  const float* kS = ky + ((size_t)iy * n + ix) * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) {
    const float ia = __frcp_rn((kW[j] + kW[N + j]) + (kS[j] + kS[(size_t)n * N + j]));
    s = fma((double)ia, (double)ia, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double is = 1.0 / (G + (dw ? dce * (double)dw[warp] : dce) * s);
    isigma_d[warp] = is;
    isigma32[warp] = (float)is;
  }
}

inline unsigned blocks_for(long threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

// a[node][j] = (kW + kE) + (kS + kN), the same expression as in the kernels
// that form it on the fly.
__global__ void diag_sum_kernel(int n, int N, const double* __restrict__ kx, const double* __restrict__ ky,
                                double* __restrict__ a) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n * n * N) return;
  const long node = t / N;
  const int j = (int)(t - node * N);
  const int iy = (int)(node / n), ix = (int)(node - (long)iy * n);
  const double* kW = kx + ((size_t)iy * (n + 1) + ix) * N;
  const double* kS = ky + ((size_t)iy * n + ix) * N;
  a[t] = (kW[j] + kW[N + j]) + (kS[j] + kS[(size_t)n * N + j]);
}

// (1/N) sum_j log kappa_j = amp sin(pi y) sum_k xbar_k sin(k pi x) / k with
// xbar_k the sample mean of xi_{jk}, at the interior nodes.
__global__ void mean_log_kappa_kernel(int n, int N, int K, double amp, const double* __restrict__ xi,
                                      double* __restrict__ out) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)n * n) return;
  const int iy = (int)(t / n), ix = (int)(t - (long)iy * n);
  const double x = (double)(ix + 1) / (double)(n + 1), y = (double)(iy + 1) / (double)(n + 1);
  double g = 0.0;
  for (int k = 1; k <= K; ++k) {
    double m = 0.0;
    for (int j = 0; j < N; ++j) m += xi[(size_t)j * K + (k - 1)];
    g += (m / N) * sinpi((double)k * x) / (double)k;
  }
  out[t] = amp * sinpi(y) * g;
}

}  // namespace

cudaError_t launch_mean_log_kappa(int n, int N, int K, double amp, const double* xi, double* out, cudaStream_t s) {
  mean_log_kappa_kernel<<<blocks_for((long)n * n, 256), 256, 0, s>>>(n, N, K, amp, xi, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_level_setup(int nf, int N, const double* kxf, const double* kyf, double* kx64,
                                      double* ky64, float* kx32, float* ky32, double* inva, double* isigma, double c,
                                      double G, double d, double e, cudaStream_t s) {
  const int nc = (nf - 1) / 2;
  coarse_faces_kernel<<<blocks_for(2L * nc * (nc + 1) * N, 256), 256, 0, s>>>(nf, N, kxf, kyf, kx64, ky64, kx32,
                                                                              ky32);
  diag_kernel<<<blocks_for((long)nc * nc * 32, 256), 256, 0, s>>>(nc, N, kx64, ky64, inva, isigma, d * c * e, G);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_level_setup(int n, int N, int K, double amp, const double* xi, double* kap, double* kx64,
                               double* ky64, float* kx32, float* ky32, double* inva, double* isigma, double c,
                               double G, double d, double e, cudaStream_t s) {
  // gx lives in the tail of kap's scratch: (n+2)*N doubles after the field.
  double* gx = kap + (size_t)(n + 2) * (n + 2) * N;
  field_x_kernel<<<blocks_for((long)(n + 2) * N, 256), 256, 0, s>>>(n, N, K, xi, gx);
  field_kernel<<<blocks_for((long)((n + 1) / 2 + 1) * (n + 2) * N, 256), 256, 0, s>>>(n, N, amp, gx, kap);
  faces_kernel<<<blocks_for(2L * n * (n + 1) * N, 256), 256, 0, s>>>(n, N, kap, kx64, ky64, kx32, ky32);
  diag_kernel<<<blocks_for((long)n * n * 32, 256), 256, 0, s>>>(n, N, kx64, ky64, inva, isigma, d * c * e, G);
  count_launches(4);
  return cudaGetLastError();
}

cudaError_t launch_diag_sum(int n, int N, const double* kx, const double* ky, double* a, cudaStream_t s) {
  diag_sum_kernel<<<blocks_for((long)n * n * N, 256), 256, 0, s>>>(n, N, kx, ky, a);
  count_launches(1);
  return cudaGetLastError();
}

// Finest grid (or a nodal grid): field and FP64 + FP32 faces only.
cudaError_t launch_field_faces(int n, int N, int K, double amp, const double* xi, double* kap, double* kx64,
                               double* ky64, float* kx32, float* ky32, cudaStream_t s) {
  double* gx = kap + (size_t)(n + 2) * (n + 2) * N;
  field_x_kernel<<<blocks_for((long)(n + 2) * N, 256), 256, 0, s>>>(n, N, K, xi, gx);
  field_kernel<<<blocks_for((long)((n + 1) / 2 + 1) * (n + 2) * N, 256), 256, 0, s>>>(n, N, amp, gx, kap);
  faces_kernel<<<blocks_for(2L * n * (n + 1) * N, 256), 256, 0, s>>>(n, N, kap, kx64, ky64, kx32, ky32);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_diag64(int n, int N, const double* kx64, const double* ky64, double* inva, double* isigma,
                          double dce, double G, cudaStream_t s, const float* dw) {
  diag_kernel<<<blocks_for((long)n * n * 32, 256), 256, 0, s>>>(n, N, kx64, ky64, inva, isigma, dce, G, dw);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_faces64(int nf, int N, const double* kxf, const double* kyf, double* kx64, double* ky64,
                                  cudaStream_t s) {
  const int nc = (nf - 1) / 2;
  coarse_faces_kernel<<<blocks_for(2L * nc * (nc + 1) * N, 256), 256, 0, s>>>(nf, N, kxf, kyf, kx64, ky64, nullptr,
                                                                              nullptr);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_faces32(int nf, int N, const float* kxf, const float* kyf, float* kx32, float* ky32,
                                  cudaStream_t s) {
  const int nc = (nf - 1) / 2;
  coarse_faces32_kernel<<<blocks_for(2L * nc * (nc + 1) * N, 256), 256, 0, s>>>(nf, N, kxf, kyf, kx32, ky32);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_diag32(int n, int N, const float* kx32, const float* ky32, float* isigma32, double* isigma_d,
                          double dce, double G, cudaStream_t s, const float* dw) {
  diag32_kernel<<<blocks_for((long)n * n * 32, 256), 256, 0, s>>>(n, N, kx32, ky32, isigma32, isigma_d, dce, G, dw);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cmg
