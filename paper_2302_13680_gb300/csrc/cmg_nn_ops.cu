// Layer kernels of the warm-start network (everything except the GEMM):
// im2col packing for 3x3 convolutions (and its transpose for weight
// gradients), the col2im gather of data gradients, ReLU / 2x2 average
// pooling / nearest upsampling and their gradients, BF16 casts and
// transposes, split-K and column reductions, the masked MSE loss, AdamW, and
// the conversions between solver grids (n x n, FP64) and the network's
// 256 x 256 BF16 images.
//
// Activations are NHWC BF16 ([B][H][W][C], C a multiple of 8 so a 16-byte
// chunk holds 8 channels of one pixel); convolution weights are
// [Cout][9 Cin] BF16 with column t*Cin + c for tap t = 3 dy + dx.
#include <cuda_bf16.h>
#include <stdint.h>

#include "cmg_internal.h"

using bf16 = __nv_bfloat16;

namespace cmg {
namespace {

constexpr int kT = 256;

inline unsigned blocks(long n) {
  long b = (n + kT - 1) / kT;
  if (b > 152L * 32) b = 152L * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

#define GRID_STRIDE(i, n) for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long)gridDim.x * blockDim.x)

// col[p][t*C + c] = X[b][y+dy-1][x+dx-1][c] (zero outside); one 16-byte chunk per thread.
__global__ void im2col_kernel(const bf16* __restrict__ X, bf16* __restrict__ col, int B, int H, int W, int C) {
  const int c8 = C / 8;
  const long total = (long)B * H * W * 9 * c8;
  GRID_STRIDE(i, total) {
    const int ch = (int)(i % c8);
    long r = i / c8;
    const int t = (int)(r % 9);
    const long p = r / 9;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W)
      v = *reinterpret_cast<const uint4*>(X + (((b * H + yy) * W + xx) * C + ch * 8));
    *reinterpret_cast<uint4*>(col + p * 9 * C + t * C + ch * 8) = v;
  }
}

// colT[t*C + c][p] (pixels contiguous), same values as im2col.
__global__ void im2col_t_kernel(const bf16* __restrict__ X, bf16* __restrict__ colT, int B, int H, int W, int C) {
  const long P = (long)B * H * W;
  const long total = P * 9 * C;
  GRID_STRIDE(i, total) {
    const long p = i % P;
    const long k = i / P;
    const int t = (int)(k / C), c = (int)(k % C);
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
    bf16 v = __float2bfloat16(0.f);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = X[((b * H + yy) * W + xx) * C + c];
    colT[k * P + p] = v;
  }
}

// dX[b][y][x][c] = sum_t dcol[(b, y-dy+1, x-dx+1)][t*C + c] over outputs inside the image.
__global__ void col2im_kernel(const float* __restrict__ dcol, bf16* __restrict__ dX, int B, int H, int W, int C) {
  const long total = (long)B * H * W * C;
  GRID_STRIDE(i, total) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yo = y - (t / 3 - 1), xo = x - (t % 3 - 1);
      if (yo >= 0 && yo < H && xo >= 0 && xo < W) s += dcol[((b * H + yo) * W + xo) * 9L * C + t * C + c];
    }
    dX[i] = __float2bfloat16_rn(s);
  }
}

// Weights of the data-gradient convolution: Wf[c][t Cout + co] =
// W[co][(8 - t) C + c] (taps turned by 180 degrees, channels exchanged), so
// that dX = conv3x3(dZ, Wf) equals col2im of dZ W.
__global__ void flip3x3_kernel(const bf16* __restrict__ W, bf16* __restrict__ Wf, int Cout, int C) {
  const long total = 9L * C * Cout;
  GRID_STRIDE(i, total) {
    const int co = (int)(i % Cout);
    const long r = i / Cout;
    const int t = (int)(r % 9), c = (int)(r / 9);
    Wf[i] = W[(long)co * 9 * C + (8 - t) * C + c];
  }
}

__global__ void transpose_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, long R, long Cc) {
  GRID_STRIDE(i, R * Cc) {
    const long r = i % R, c = i / R;
    out[c * R + r] = in[r * Cc + c];
  }
}

__global__ void relu_bwd_kernel(const bf16* __restrict__ y, const bf16* __restrict__ dy, bf16* __restrict__ dz, long n) {
  GRID_STRIDE(i, n) dz[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16(0.f);
}

__global__ void avgpool_kernel(const bf16* __restrict__ X, bf16* __restrict__ Y, int B, int H, int W, int C) {
  const int Ho = H / 2, Wo = W / 2;
  GRID_STRIDE(i, (long)B * Ho * Wo * C) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho);
    const long b = p / ((long)Wo * Ho);
    const bf16* s = X + ((b * H + 2 * y) * W + 2 * x) * C + c;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[(long)W * C]) +
                    __bfloat162float(s[(long)W * C + C]);
    Y[i] = __float2bfloat16_rn(0.25f * v);
  }
}

__global__ void avgpool_bwd_kernel(const bf16* __restrict__ dY, bf16* __restrict__ dX, int B, int H, int W, int C) {
  GRID_STRIDE(i, (long)B * H * W * C) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    dX[i] = __float2bfloat16_rn(0.25f * __bfloat162float(dY[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]));
  }
}

// Y = upsample2(X) + S (nearest neighbour, additive skip).
__global__ void upsample_add_kernel(const bf16* __restrict__ X, const bf16* __restrict__ S, bf16* __restrict__ Y,
                                    int B, int H, int W, int C) {
  GRID_STRIDE(i, (long)B * H * W * C) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    const float v = __bfloat162float(X[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]) + __bfloat162float(S[i]);
    Y[i] = __float2bfloat16_rn(v);
  }
}

// dX = sum over the 2x2 block of dY (gradient of nearest upsampling).
__global__ void upsample_bwd_kernel(const bf16* __restrict__ dY, bf16* __restrict__ dX, int B, int H, int W, int C) {
  GRID_STRIDE(i, (long)B * H * W * C) {
    const int c = (int)(i % C);
    const long p = i / C;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long b = p / ((long)W * H);
    const long W2 = 2L * W;
    const bf16* s = dY + ((b * 2 * H + 2 * y) * W2 + 2 * x) * C + c;
    const float v = __bfloat162float(s[0]) + __bfloat162float(s[C]) + __bfloat162float(s[W2 * C]) +
                    __bfloat162float(s[W2 * C + C]);
    dX[i] = __float2bfloat16_rn(v);
  }
}

__global__ void add_kernel(const bf16* __restrict__ a, const bf16* __restrict__ b, bf16* __restrict__ out, long n) {
  GRID_STRIDE(i, n) out[i] = __float2bfloat16_rn(__bfloat162float(a[i]) + __bfloat162float(b[i]));
}

// out[p][c] = a[p] * w[c] (BF16): data gradient of a 1x1 convolution to one channel.
__global__ void outer_kernel(const bf16* __restrict__ a, const float* __restrict__ w, bf16* __restrict__ out, long P,
                             int C) {
  GRID_STRIDE(i, P * C) out[i] = __float2bfloat16_rn(__bfloat162float(a[i / C]) * w[i % C]);
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, bf16* __restrict__ out, long n) {
  GRID_STRIDE(i, n) out[i] = __float2bfloat16_rn(in[i]);
}

// out[i] = sum_j part[j * n + i], fixed order.
__global__ void sum_slices_kernel(const float* __restrict__ part, int slices, float* __restrict__ out, long n) {
  GRID_STRIDE(i, n) {
    float s = 0.f;
    for (int j = 0; j < slices; ++j) s += part[(long)j * n + i];
    out[i] = s;
  }
}

// colsum[c] = sum_p in[p][c] for BF16 in [P][C]: one CTA per channel, fixed order.
__global__ void colsum_kernel(const bf16* __restrict__ in, long P, int C, float* __restrict__ out) {
  __shared__ float sh[kT / 32];
  const int c = blockIdx.x;
  float s = 0.f;
  for (long p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(in[p * C + c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kT / 32; ++w) t += sh[w];
    out[c] = t;
  }
}

// Masked MSE on [B][S][S] predictions (interior m x m region, m <= S):
// per-CTA partial sums of squared errors and the gradient 2 (pred - tgt) / count.
__global__ void mse_kernel(const float* __restrict__ pred, const float* __restrict__ tgt, int B, int S, int m,
                           bf16* __restrict__ grad, float* __restrict__ partial) {
  __shared__ float sh[kT / 32];
  const long total = (long)B * S * S;
  const float inv = 2.f / ((float)B * m * m);
  float acc = 0.f;
  GRID_STRIDE(i, total) {
    const int x = (int)(i % S), y = (int)((i / S) % S);
    float g = 0.f;
    if (x < m && y < m) {
      const float d = pred[i] - tgt[i];
      acc += d * d;
      g = inv * d;
    }
    grad[i] = __float2bfloat16_rn(g);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kT / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// AdamW on FP32 master weights; BF16 copy refreshed.
__global__ void adamw_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                             float* __restrict__ m2, bf16* __restrict__ w16, long n, float lr, float b1, float b2,
                             float eps, float wd, float bc1, float bc2) {
  GRID_STRIDE(i, n) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    float wi = w[i] * (1.f - lr * wd);
    wi -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16_rn(wi);
  }
}

// Network input [B][S][S][Cp] from two n x n FP64 fields per image (channel 0
// and 1, scaled), zero elsewhere (channels >= 2 and pixels beyond n).
__global__ void pack_input_kernel(const double* __restrict__ f0, const double* __restrict__ f1, int B, int n, int S,
                                  int Cp, float s0, float s1, bf16* __restrict__ X) {
  GRID_STRIDE(i, (long)B * S * S * Cp) {
    const int c = (int)(i % Cp);
    const long p = i / Cp;
    const int x = (int)(p % S), y = (int)((p / S) % S);
    const long b = p / ((long)S * S);
    float v = 0.f;
    if (x < n && y < n && c < 2) {
      const long node = b * (long)n * n + (long)y * n + x;
      v = c == 0 ? s0 * (float)f0[node] : s1 * (float)f1[node];
    }
    X[i] = __float2bfloat16_rn(v);
  }
}

// [B][S][S] FP32 images -> [B][n*n] FP64 (times scale), the inverse of the packing.
__global__ void unpack_output_kernel(const float* __restrict__ img, int B, int n, int S, double scale,
                                     double* __restrict__ out) {
  GRID_STRIDE(i, (long)B * n * n) {
    const int x = (int)(i % n), y = (int)((i / n) % n);
    const long b = i / ((long)n * n);
    out[i] = scale * (double)img[(b * S + y) * S + x];
  }
}

// [B][n*n] FP64 -> [B][S][S] FP32 images (times scale, zero padding).
__global__ void pack_target_kernel(const double* __restrict__ u, int B, int n, int S, double scale,
                                   float* __restrict__ img) {
  GRID_STRIDE(i, (long)B * S * S) {
    const int x = (int)(i % S), y = (int)((i / S) % S);
    const long b = i / ((long)S * S);
    img[i] = (x < n && y < n) ? (float)(scale * u[b * (long)n * n + (long)y * n + x]) : 0.f;
  }
}

}  // namespace
}  // namespace cmg

using namespace cmg;

namespace {
inline cmg_status done(int launches) {
  count_launches(launches);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CMG_OK : CMG_ERR_CUDA;
}
inline cudaStream_t st(void* s) { return static_cast<cudaStream_t>(s); }
}  // namespace

extern "C" {

cmg_status cmg_nn_im2col(const void* X, void* col, int B, int H, int W, int C, int transposed, void* stream) {
  if (!X || !col || B < 1 || H < 1 || W < 1 || C < 8 || C % 8) return CMG_ERR_INVALID_ARG;
  if (transposed)
    im2col_t_kernel<<<blocks((long)B * H * W * 9 * C), kT, 0, st(stream)>>>((const bf16*)X, (bf16*)col, B, H, W, C);
  else
    im2col_kernel<<<blocks((long)B * H * W * 9 * C / 8), kT, 0, st(stream)>>>((const bf16*)X, (bf16*)col, B, H, W, C);
  return done(1);
}

cmg_status cmg_nn_col2im(const float* dcol, void* dX, int B, int H, int W, int C, void* stream) {
  if (!dcol || !dX || B < 1 || H < 1 || W < 1 || C < 1) return CMG_ERR_INVALID_ARG;
  col2im_kernel<<<blocks((long)B * H * W * C), kT, 0, st(stream)>>>(dcol, (bf16*)dX, B, H, W, C);
  return done(1);
}

cmg_status cmg_nn_transpose(const void* in, void* out, long long R, long long Cc, void* stream) {
  if (!in || !out || R < 1 || Cc < 1) return CMG_ERR_INVALID_ARG;
  transpose_kernel<<<blocks(R * Cc), kT, 0, st(stream)>>>((const bf16*)in, (bf16*)out, R, Cc);
  return done(1);
}

cmg_status cmg_nn_flip3x3(const void* W, void* Wf, int Cout, int C, void* stream) {
  if (!W || !Wf || Cout < 1 || C < 1) return CMG_ERR_INVALID_ARG;
  flip3x3_kernel<<<blocks(9L * C * Cout), kT, 0, st(stream)>>>((const bf16*)W, (bf16*)Wf, Cout, C);
  return done(1);
}

cmg_status cmg_nn_relu_bwd(const void* y, const void* dy, void* dz, long long n, void* stream) {
  if (!y || !dy || !dz || n < 1) return CMG_ERR_INVALID_ARG;
  relu_bwd_kernel<<<blocks(n), kT, 0, st(stream)>>>((const bf16*)y, (const bf16*)dy, (bf16*)dz, n);
  return done(1);
}

cmg_status cmg_nn_avgpool(const void* X, void* Y, int B, int H, int W, int C, int backward, void* stream) {
  if (!X || !Y || B < 1 || H < 2 || W < 2 || (H | W) & 1 || C < 1) return CMG_ERR_INVALID_ARG;
  if (backward)   // X = dY [B][H/2][W/2][C], Y = dX [B][H][W][C]
    avgpool_bwd_kernel<<<blocks((long)B * H * W * C), kT, 0, st(stream)>>>((const bf16*)X, (bf16*)Y, B, H, W, C);
  else
    avgpool_kernel<<<blocks((long)B * H * W * C / 4), kT, 0, st(stream)>>>((const bf16*)X, (bf16*)Y, B, H, W, C);
  return done(1);
}

cmg_status cmg_nn_upsample_add(const void* X, const void* S, void* Y, int B, int H, int W, int C, void* stream) {
  if (!X || !S || !Y || B < 1 || H < 2 || W < 2 || (H | W) & 1 || C < 1) return CMG_ERR_INVALID_ARG;
  upsample_add_kernel<<<blocks((long)B * H * W * C), kT, 0, st(stream)>>>((const bf16*)X, (const bf16*)S, (bf16*)Y, B,
                                                                          H, W, C);
  return done(1);
}

cmg_status cmg_nn_upsample_bwd(const void* dY, void* dX, int B, int H, int W, int C, void* stream) {
  if (!dY || !dX || B < 1 || H < 1 || W < 1 || C < 1) return CMG_ERR_INVALID_ARG;
  upsample_bwd_kernel<<<blocks((long)B * H * W * C), kT, 0, st(stream)>>>((const bf16*)dY, (bf16*)dX, B, H, W, C);
  return done(1);
}

cmg_status cmg_nn_add(const void* a, const void* b, void* out, long long n, void* stream) {
  if (!a || !b || !out || n < 1) return CMG_ERR_INVALID_ARG;
  add_kernel<<<blocks(n), kT, 0, st(stream)>>>((const bf16*)a, (const bf16*)b, (bf16*)out, n);
  return done(1);
}

cmg_status cmg_nn_outer(const void* a, const float* w, void* out, long long P, int C, void* stream) {
  if (!a || !w || !out || P < 1 || C < 1) return CMG_ERR_INVALID_ARG;
  outer_kernel<<<blocks(P * C), kT, 0, st(stream)>>>((const bf16*)a, w, (bf16*)out, P, C);
  return done(1);
}

cmg_status cmg_nn_to_bf16(const float* in, void* out, long long n, void* stream) {
  if (!in || !out || n < 1) return CMG_ERR_INVALID_ARG;
  f32_to_bf16_kernel<<<blocks(n), kT, 0, st(stream)>>>(in, (bf16*)out, n);
  return done(1);
}

cmg_status cmg_nn_sum_slices(const float* part, int slices, float* out, long long n, void* stream) {
  if (!part || !out || slices < 1 || n < 1) return CMG_ERR_INVALID_ARG;
  sum_slices_kernel<<<blocks(n), kT, 0, st(stream)>>>(part, slices, out, n);
  return done(1);
}

cmg_status cmg_nn_colsum(const void* in, long long P, int C, float* out, void* stream) {
  if (!in || !out || P < 1 || C < 1) return CMG_ERR_INVALID_ARG;
  colsum_kernel<<<C, kT, 0, st(stream)>>>((const bf16*)in, P, C, out);
  return done(1);
}

cmg_status cmg_nn_mse(const float* pred, const float* tgt, int B, int S, int m, void* grad, float* partial,
                      int max_partials, int* used_partials, void* stream) {
  if (!pred || !tgt || !grad || !partial || !used_partials || B < 1 || S < 1 || m < 1 || m > S)
    return CMG_ERR_INVALID_ARG;
  const unsigned g = blocks((long)B * S * S);
  if ((int)g > max_partials) return CMG_ERR_INVALID_ARG;
  mse_kernel<<<g, kT, 0, st(stream)>>>(pred, tgt, B, S, m, (bf16*)grad, partial);
  *used_partials = (int)g;
  return done(1);
}

cmg_status cmg_nn_adamw(float* w, const float* g, float* m1, float* m2, void* w16, long long n, float lr, float b1,
                        float b2, float eps, float wd, int step, void* stream) {
  if (!w || !g || !m1 || !m2 || n < 1 || step < 1) return CMG_ERR_INVALID_ARG;
  const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
  adamw_kernel<<<blocks(n), kT, 0, st(stream)>>>(w, g, m1, m2, (bf16*)w16, n, lr, b1, b2, eps, wd, bc1, bc2);
  return done(1);
}

cmg_status cmg_nn_pack_input(const double* f0, const double* f1, int B, int n, int S, int Cp, float s0, float s1,
                             void* X, void* stream) {
  if (!f0 || !f1 || !X || B < 1 || n < 1 || S < n || Cp < 2) return CMG_ERR_INVALID_ARG;
  pack_input_kernel<<<blocks((long)B * S * S * Cp), kT, 0, st(stream)>>>(f0, f1, B, n, S, Cp, s0, s1, (bf16*)X);
  return done(1);
}

cmg_status cmg_nn_unpack_output(const float* img, int B, int n, int S, double scale, double* out, void* stream) {
  if (!img || !out || B < 1 || n < 1 || S < n) return CMG_ERR_INVALID_ARG;
  unpack_output_kernel<<<blocks((long)B * n * n), kT, 0, st(stream)>>>(img, B, n, S, scale, out);
  return done(1);
}

cmg_status cmg_nn_pack_target(const double* u, int B, int n, int S, double scale, float* img, void* stream) {
  if (!u || !img || B < 1 || n < 1 || S < n) return CMG_ERR_INVALID_ARG;
  pack_target_kernel<<<blocks((long)B * S * S), kT, 0, st(stream)>>>(u, B, n, S, scale, img);
  return done(1);
}

}  // extern "C"
