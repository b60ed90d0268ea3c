// The learned warm start's network as one handle (include/cmg.h, cmg_unet_*):
// a BF16 U-Net whose layers run on the library's own kernels (tcgen05 GEMM,
// layer kernels of cmg_nn_ops.cu), with its FP32 master weights, AdamW
// moments, activation and gradient buffers, the order of the layers in the
// forward and backward passes, and checkpoints.  The paper has no network;
// the warm start is this library's addition, and multigrid (Algorithm 1)
// always finishes the solve.
//
// Architecture (images S x S, NHWC BF16, 8 input channels of which the first
// two carry y_d and the sample mean of log kappa): four resolutions S, S/2,
// S/4, S/8 with 32, 64, 64, 64 channels; two 3x3 convolutions + ReLU per
// encoder level, 2x2 average pooling, nearest upsampling with additive
// skips, one 3x3 convolution + ReLU per decoder level, a 1x1 linear head.
// A 3x3 convolution is im2col + GEMM (weights [Cout][9 Cin], column
// t*Cin + c for tap t = 3 dy + dx); its weight gradient a split-K GEMM over
// the pixels, its data gradient a GEMM and a col2im gather.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cmg_internal.h"

using namespace cmg;

namespace {

constexpr int kCin = 8;      // input channels (one 16-byte BF16 chunk)
constexpr int kHeadC = 32;   // channels into the 1x1 head
struct ConvSpec {
  const char* name;
  int ci, co, level;
};
constexpr ConvSpec kConvs[] = {{"c0a", kCin, 32, 0}, {"c0b", 32, 32, 0}, {"c1a", 32, 64, 1}, {"c1b", 64, 64, 1},
                               {"c2a", 64, 64, 2},   {"c2b", 64, 64, 2}, {"c3a", 64, 64, 3}, {"c3b", 64, 64, 3},
                               {"d2", 64, 64, 2},    {"d1", 64, 32, 1},  {"d0", 32, 32, 0}};
constexpr int kConvCount = sizeof(kConvs) / sizeof(kConvs[0]);
constexpr int kLayers = kConvCount + 1;   // + head
enum Layer { C0A, C0B, C1A, C1B, C2A, C2B, C3A, C3B, D2, D1, D0, HEAD };

// Activations of the forward pass (the backward pass keeps a gradient
// buffer of the same shape for each): x0 is the caller's input.
enum Act { A0, S0, P1, A1, S1, P2, A2, S2, P3, A3, B3, T2, E2, T1, E1, T0, E0, kActs };
struct ActSpec {
  int level, ch;
};
constexpr ActSpec kActShape[kActs] = {{0, 32}, {0, 32}, {1, 32}, {1, 64}, {1, 64}, {2, 64}, {2, 64}, {2, 64}, {3, 64},
                                      {3, 64}, {3, 64}, {2, 64}, {2, 64}, {1, 64}, {1, 32}, {0, 32}, {0, 32}};

struct Param {
  int rows = 0, cols = 0;
  float *w = nullptr, *b = nullptr, *gw = nullptr, *gb = nullptr;
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;
  void* w16 = nullptr;
};

constexpr char kMagic[8] = {'C', 'M', 'G', 'U', 'N', 'E', 'T', '1'};
constexpr int kFormat = 1;

// Host normal draws for the initial weights: splitmix64 (Steele, Lea,
// Flood 2014) for uniform bits, Box-Muller for the normal pair.
struct HostNormal {
  uint64_t s;
  bool have = false;
  double spare = 0.0;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }   // (0, 1)
  double normal() {
    if (have) {
      have = false;
      return spare;
    }
    const double r = std::sqrt(-2.0 * std::log(uniform())), t = 6.283185307179586 * uniform();
    spare = r * std::sin(t);
    have = true;
    return r * std::cos(t);
  }
};

// loss = (sum of the CTA partials) / count, one thread, fixed order.
__global__ void loss_sum_kernel(const float* __restrict__ part, int n, double inv_count, double* __restrict__ out) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (double)part[i];
  *out = s * inv_count;
}

}  // namespace

struct cmg_unet {
  int S = 0, Bmax = 0, Bcur = 0;
  cudaStream_t stream = nullptr;
  Param prm[kLayers];
  int step = 0;
  float in_scale[2] = {1.f, 1.f};
  double out_scale = 1.0;
  int* status = nullptr;            // device: set by a tensor-core wait that ran out
  const void* x0 = nullptr;         // input of the last forward pass (caller's)
  void* act[kActs] = {};
  void* grad[kActs] = {};
  void* pool_tmp = nullptr;         // 2x2 pooling gradient before the skip sum
  float* pred = nullptr;            // [Bmax][S][S] last prediction (internal)
  void* dpred = nullptr;            // [Bmax][S][S] BF16 loss gradient
  float* mse_part = nullptr;
  int mse_cap = 0;
  // per-layer work buffers sized for the largest layer
  void *col = nullptr, *dZ = nullptr, *dZT = nullptr, *colT = nullptr, *WT = nullptr;
  float *part = nullptr, *dcol = nullptr;
  std::vector<void*> allocs;
  std::string err;
};

namespace {

cmg_status fail(cmg_unet* u, cmg_status st, const std::string& msg) {
  if (u) u->err = msg;
  return st;
}

cmg_status cuda_fail(cmg_unet* u, cudaError_t e, const char* what) {
  const cmg_status st = e == cudaErrorMemoryAllocation ? CMG_ERR_OOM : CMG_ERR_CUDA;
  (void)cudaGetLastError();
  return fail(u, st, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
cudaError_t ualloc(cmg_unet* u, T** p, size_t bytes) {
  void* q = nullptr;
  const cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  u->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

// Call into the layer-kernel ABI; a refused call is reported with its name.
#define NN(call)                                                          \
  do {                                                                    \
    const cmg_status s_ = (call);                                         \
    if (s_ != CMG_OK) return fail(u, s_, std::string("layer call: ") + #call); \
  } while (0)

long pixels(const cmg_unet* u, int B, int level) {
  const long H = u->S >> level;
  return (long)B * H * H;
}

// Pixel slice of the split-K weight gradient: the largest multiple of 8 up
// to 4096 that divides the pixel count P (P = B H^2 with H a multiple of 4,
// so 8 always divides it).
int kslice(long P) {
  for (long k = P < 4096 ? P : 4096; k >= 8; k -= 8)
    if (P % k == 0 && k % 8 == 0) return (int)k;
  return 8;
}

cmg_status conv_forward(cmg_unet* u, int layer, const void* X, void* Y, int B) {
  const ConvSpec& c = kConvs[layer];
  const int H = u->S >> c.level;
  const long P = pixels(u, B, c.level);
  const Param& p = u->prm[layer];
  // implicit GEMM (the tensor cores read X through an im2col tensor map);
  // im2col + GEMM where it does not apply (same results)
  const cmg_status st = cmg_nn_conv3x3_bf16(X, B, H, H, c.ci, p.w16, c.co, p.b, 1, Y, u->status, u->stream);
  if (st != CMG_ERR_UNSUPPORTED) return st == CMG_OK ? CMG_OK : fail(u, st, "layer call: cmg_nn_conv3x3_bf16");
  NN(cmg_nn_im2col(X, u->col, B, H, H, c.ci, 0, u->stream));
  NN(cmg_nn_gemm_bf16(u->col, 9 * c.ci, p.w16, 9 * c.ci, (int)P, c.co, 9 * c.ci, p.b, 1, nullptr, Y, c.co, u->status,
                      u->stream));
  return CMG_OK;
}

// dY: gradient of the layer's output after its ReLU; fills gw, gb and, when
// dX is given, the gradient of the input X.
cmg_status conv_backward(cmg_unet* u, int layer, const void* X, const void* Y, const void* dY, void* dX, int B) {
  const ConvSpec& c = kConvs[layer];
  const int H = u->S >> c.level;
  const long P = pixels(u, B, c.level);
  Param& p = u->prm[layer];
  NN(cmg_nn_relu_bwd(Y, dY, u->dZ, P * c.co, u->stream));
  NN(cmg_nn_colsum(u->dZ, P, c.co, p.gb, u->stream));
  NN(cmg_nn_transpose(u->dZ, u->dZT, P, c.co, u->stream));
  NN(cmg_nn_im2col(X, u->colT, B, H, H, c.ci, 1, u->stream));
  const int ks = kslice(P);
  const int nsl = (int)(P / ks);
  NN(cmg_nn_gemm_bf16_splitk(u->dZT, P, u->colT, P, c.co, 9 * c.ci, ks, nsl, u->part, 9 * c.ci, u->status,
                             u->stream));
  NN(cmg_nn_sum_slices(u->part, nsl, p.gw, (long long)c.co * 9 * c.ci, u->stream));
  if (!dX) return CMG_OK;
  // dX as a 3x3 convolution of dZ with the turned weights (implicit GEMM, no
  // patch-gradient matrix); else dZ W into patches and col2im
  NN(cmg_nn_flip3x3(p.w16, u->WT, c.co, c.ci, u->stream));
  const cmg_status st = cmg_nn_conv3x3_bf16(u->dZ, B, H, H, c.co, u->WT, c.ci, nullptr, 0, dX, u->status, u->stream);
  if (st != CMG_ERR_UNSUPPORTED) return st == CMG_OK ? CMG_OK : fail(u, st, "layer call: cmg_nn_conv3x3_bf16");
  NN(cmg_nn_transpose(p.w16, u->WT, c.co, 9 * c.ci, u->stream));
  NN(cmg_nn_gemm_bf16(u->dZ, c.co, u->WT, c.co, (int)P, 9 * c.ci, c.co, nullptr, 0, u->dcol, nullptr, 9 * c.ci,
                      u->status, u->stream));
  NN(cmg_nn_col2im(u->dcol, dX, B, H, H, c.ci, u->stream));
  return CMG_OK;
}

cmg_status check_batch(cmg_unet* u, int B) {
  if (B < 1 || B > u->Bmax) return fail(u, CMG_ERR_INVALID_ARG, "batch outside [1, the batch given at create]");
  return CMG_OK;
}

size_t param_elems(const Param& p, int which) {
  return which == CMG_UNET_B || which == CMG_UNET_GB || which == CMG_UNET_MB || which == CMG_UNET_VB
             ? (size_t)p.rows
             : (size_t)p.rows * p.cols;
}
float* param_ptr(Param& p, int which) {
  switch (which) {
    case CMG_UNET_W: return p.w;
    case CMG_UNET_B: return p.b;
    case CMG_UNET_GW: return p.gw;
    case CMG_UNET_GB: return p.gb;
    case CMG_UNET_MW: return p.mw;
    case CMG_UNET_VW: return p.vw;
    case CMG_UNET_MB: return p.mb;
    case CMG_UNET_VB: return p.vb;
    default: return nullptr;
  }
}

}  // namespace

extern "C" {

cmg_status cmg_unet_create(int S, int max_batch, unsigned long long seed, void* stream, cmg_unet** out) {
  if (!out) return CMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (S < 32 || S % 32 != 0 || S > 4096 || max_batch < 1 || max_batch > 1024) return CMG_ERR_INVALID_ARG;
  cmg_unet* u = new (std::nothrow) cmg_unet;
  if (!u) return CMG_ERR_OOM;
  u->S = S;
  u->Bmax = max_batch;
  u->stream = static_cast<cudaStream_t>(stream);
  const int B = max_batch;
  cudaError_t e = cudaSuccess;
  HostNormal rng{seed ^ 0x636D67756E6574ull};   // "cmgunet"
  std::vector<float> hw, hb;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    Param& p = u->prm[l];
    p.rows = l < kConvCount ? kConvs[l].co : 1;
    p.cols = l < kConvCount ? 9 * kConvs[l].ci : kHeadC;
    const size_t nw = (size_t)p.rows * p.cols, nb = (size_t)p.rows;
    float** fp[] = {&p.w, &p.gw, &p.mw, &p.vw};
    for (float** q : fp)
      if (e == cudaSuccess) e = ualloc(u, q, nw * sizeof(float));
    float** bp[] = {&p.b, &p.gb, &p.mb, &p.vb};
    for (float** q : bp)
      if (e == cudaSuccess) e = ualloc(u, q, nb * sizeof(float));
    if (e == cudaSuccess) e = ualloc(u, &p.w16, nw * 2);
    if (e != cudaSuccess) break;
    // He-normal initial weights for the ReLU convolutions, a small head
    const double sd = l < kConvCount ? std::sqrt(2.0 / (9.0 * kConvs[l].ci)) : 1e-2;
    hw.resize(nw);
    for (size_t i = 0; i < nw; ++i) hw[i] = (float)(sd * rng.normal());
    hb.assign(nb, 0.f);
    e = cudaMemcpy(p.w, hw.data(), nw * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p.b, hb.data(), nb * sizeof(float), cudaMemcpyHostToDevice);
    for (float* q : {p.gw, p.mw, p.vw})
      if (e == cudaSuccess) e = cudaMemset(q, 0, nw * sizeof(float));
    for (float* q : {p.gb, p.mb, p.vb})
      if (e == cudaSuccess) e = cudaMemset(q, 0, nb * sizeof(float));
  }
  // activations, their gradients and the work buffers (largest layer)
  size_t col = 0, dz = 0, colT = 0, part = 0, wt = 0, dcol = 0;
  for (int l = 0; l < kConvCount; ++l) {
    const ConvSpec& c = kConvs[l];
    const long P = pixels(u, B, c.level);
    col = std::max(col, (size_t)P * 9 * c.ci * 2);
    dz = std::max(dz, (size_t)P * c.co * 2);
    colT = std::max(colT, (size_t)P * 9 * c.ci * 2);
    part = std::max(part, (size_t)(P / kslice(P)) * c.co * 9 * c.ci * 4);
    wt = std::max(wt, (size_t)9 * c.ci * c.co * 2);
    dcol = std::max(dcol, (size_t)P * 9 * c.ci * 4);
  }
  const long P0 = pixels(u, B, 0);
  dz = std::max(dz, (size_t)P0 * kHeadC * 2);                         // head: e0 transposed
  part = std::max(part, (size_t)(P0 / kslice(P0)) * kHeadC * 4);
  size_t pool = 0;
  for (int a = 0; a < kActs && e == cudaSuccess; ++a) {
    const size_t bytes = (size_t)pixels(u, B, kActShape[a].level) * kActShape[a].ch * 2;
    pool = std::max(pool, bytes);
    e = ualloc(u, &u->act[a], bytes);
    if (e == cudaSuccess) e = ualloc(u, &u->grad[a], bytes);
  }
  u->mse_cap = 152 * 32;
  if (e == cudaSuccess) e = ualloc(u, &u->pool_tmp, pool);
  if (e == cudaSuccess) e = ualloc(u, &u->pred, (size_t)P0 * 4);
  if (e == cudaSuccess) e = ualloc(u, &u->dpred, (size_t)P0 * 2);
  if (e == cudaSuccess) e = ualloc(u, &u->mse_part, (size_t)u->mse_cap * 4);
  if (e == cudaSuccess) e = ualloc(u, &u->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(u->status, 0, sizeof(int));
  if (e == cudaSuccess) e = ualloc(u, &u->col, col);
  if (e == cudaSuccess) e = ualloc(u, &u->dZ, dz);
  if (e == cudaSuccess) e = ualloc(u, &u->dZT, dz);
  if (e == cudaSuccess) e = ualloc(u, &u->colT, colT);
  if (e == cudaSuccess) e = ualloc(u, &u->part, part);
  if (e == cudaSuccess) e = ualloc(u, &u->WT, wt);
  if (e == cudaSuccess) e = ualloc(u, &u->dcol, dcol);
  if (e != cudaSuccess) {
    const cmg_status st = e == cudaErrorMemoryAllocation ? CMG_ERR_OOM : CMG_ERR_CUDA;
    (void)cudaGetLastError();
    cmg_unet_destroy(u);
    return st;
  }
  for (int l = 0; l < kLayers; ++l) {
    const Param& p = u->prm[l];
    const cmg_status st = cmg_nn_to_bf16(p.w, p.w16, (long long)p.rows * p.cols, u->stream);
    if (st != CMG_OK) {
      cmg_unet_destroy(u);
      return st;
    }
  }
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) {
    (void)cudaGetLastError();
    cmg_unet_destroy(u);
    return CMG_ERR_CUDA;
  }
  *out = u;
  return CMG_OK;
}

void cmg_unet_destroy(cmg_unet* u) {
  if (!u) return;
  for (void* p : u->allocs) (void)cudaFree(p);
  delete u;
}

const char* cmg_unet_last_error(const cmg_unet* u) { return u ? u->err.c_str() : "null network"; }

cmg_status cmg_unet_set_scales(cmg_unet* u, float in_yd, float in_logk, double out) {
  if (!u) return CMG_ERR_INVALID_ARG;
  if (!(std::isfinite(in_yd) && std::isfinite(in_logk) && std::isfinite(out) && out != 0.0))
    return fail(u, CMG_ERR_INVALID_ARG, "scales must be finite, the output scale nonzero");
  u->in_scale[0] = in_yd;
  u->in_scale[1] = in_logk;
  u->out_scale = out;
  return CMG_OK;
}

cmg_status cmg_unet_get_scales(const cmg_unet* u, float* in_yd, float* in_logk, double* out) {
  if (!u || !in_yd || !in_logk || !out) return CMG_ERR_INVALID_ARG;
  *in_yd = u->in_scale[0];
  *in_logk = u->in_scale[1];
  *out = u->out_scale;
  return CMG_OK;
}

cmg_status cmg_unet_pack_inputs(cmg_unet* u, const double* yd, const double* mlk, int B, int n, void* X) {
  if (!u || !yd || !mlk || !X) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  if (B < 1 || n < 1 || n > u->S) return fail(u, CMG_ERR_INVALID_ARG, "batch or grid size out of range");
  NN(cmg_nn_pack_input(yd, mlk, B, n, u->S, kCin, u->in_scale[0], u->in_scale[1], X, u->stream));
  return CMG_OK;
}

cmg_status cmg_unet_pack_targets(cmg_unet* u, const double* uu, int B, int n, float* T) {
  if (!u || !uu || !T) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  if (B < 1 || n < 1 || n > u->S) return fail(u, CMG_ERR_INVALID_ARG, "batch or grid size out of range");
  NN(cmg_nn_pack_target(uu, B, n, u->S, 1.0 / u->out_scale, T, u->stream));
  return CMG_OK;
}

cmg_status cmg_unet_unpack(cmg_unet* u, const float* pred, int B, int n, double* out) {
  if (!u || !out) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  if (B < 1 || n < 1 || n > u->S) return fail(u, CMG_ERR_INVALID_ARG, "batch or grid size out of range");
  NN(cmg_nn_unpack_output(pred ? pred : u->pred, B, n, u->S, u->out_scale, out, u->stream));
  return CMG_OK;
}

cmg_status cmg_unet_forward(cmg_unet* u, const void* X, int B, float* pred) {
  if (!u || !X) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return fail(u, CMG_ERR_INVALID_ARG, "input not 16-byte aligned");
  cmg_status st = check_batch(u, B);
  if (st != CMG_OK) return st;
  const int S = u->S;
  void** a = u->act;
  u->x0 = X;
  u->Bcur = B;
  if ((st = conv_forward(u, C0A, X, a[A0], B)) != CMG_OK) return st;
  if ((st = conv_forward(u, C0B, a[A0], a[S0], B)) != CMG_OK) return st;
  NN(cmg_nn_avgpool(a[S0], a[P1], B, S, S, 32, 0, u->stream));
  if ((st = conv_forward(u, C1A, a[P1], a[A1], B)) != CMG_OK) return st;
  if ((st = conv_forward(u, C1B, a[A1], a[S1], B)) != CMG_OK) return st;
  NN(cmg_nn_avgpool(a[S1], a[P2], B, S / 2, S / 2, 64, 0, u->stream));
  if ((st = conv_forward(u, C2A, a[P2], a[A2], B)) != CMG_OK) return st;
  if ((st = conv_forward(u, C2B, a[A2], a[S2], B)) != CMG_OK) return st;
  NN(cmg_nn_avgpool(a[S2], a[P3], B, S / 4, S / 4, 64, 0, u->stream));
  if ((st = conv_forward(u, C3A, a[P3], a[A3], B)) != CMG_OK) return st;
  if ((st = conv_forward(u, C3B, a[A3], a[B3], B)) != CMG_OK) return st;
  NN(cmg_nn_upsample_add(a[B3], a[S2], a[T2], B, S / 4, S / 4, 64, u->stream));
  if ((st = conv_forward(u, D2, a[T2], a[E2], B)) != CMG_OK) return st;
  NN(cmg_nn_upsample_add(a[E2], a[S1], a[T1], B, S / 2, S / 2, 64, u->stream));
  if ((st = conv_forward(u, D1, a[T1], a[E1], B)) != CMG_OK) return st;
  NN(cmg_nn_upsample_add(a[E1], a[S0], a[T0], B, S, S, 32, u->stream));
  if ((st = conv_forward(u, D0, a[T0], a[E0], B)) != CMG_OK) return st;
  const Param& h = u->prm[HEAD];
  const long P0 = pixels(u, B, 0);
  NN(cmg_nn_gemm_bf16(a[E0], kHeadC, h.w16, kHeadC, (int)P0, 1, kHeadC, h.b, 0, u->pred, nullptr, 1, u->status,
                      u->stream));
  if (pred && pred != u->pred) {
    const cudaError_t e = cudaMemcpyAsync(pred, u->pred, (size_t)P0 * sizeof(float), cudaMemcpyDeviceToDevice,
                                          u->stream);
    if (e != cudaSuccess) return cuda_fail(u, e, "copy of the prediction");
  }
  return CMG_OK;
}

cmg_status cmg_unet_loss(cmg_unet* u, const float* target, int m, double* loss) {
  if (!u || !target || !loss) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  if (u->Bcur < 1) return fail(u, CMG_ERR_INVALID_ARG, "no forward pass yet");
  if (m < 1 || m > u->S) return fail(u, CMG_ERR_INVALID_ARG, "m outside [1, S]");
  int used = 0;
  NN(cmg_nn_mse(u->pred, target, u->Bcur, u->S, m, u->dpred, u->mse_part, u->mse_cap, &used, u->stream));
  loss_sum_kernel<<<1, 1, 0, u->stream>>>(u->mse_part, used, 1.0 / ((double)u->Bcur * m * m), loss);
  count_launches(1);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CMG_OK : cuda_fail(u, e, "loss_sum_kernel");
}

cmg_status cmg_unet_backward(cmg_unet* u, const void* dpred) {
  if (!u) return CMG_ERR_INVALID_ARG;
  if (u->Bcur < 1 || !u->x0) return fail(u, CMG_ERR_INVALID_ARG, "no forward pass yet");
  const int B = u->Bcur, S = u->S;
  void** a = u->act;
  void** g = u->grad;
  const void* dp = dpred ? dpred : u->dpred;
  const long P0 = pixels(u, B, 0);
  Param& h = u->prm[HEAD];
  // head: e0 [P0][32] times w [1][32]^T + b
  NN(cmg_nn_transpose(a[E0], u->dZT, P0, kHeadC, u->stream));
  const int ks = kslice(P0);
  const int nsl = (int)(P0 / ks);
  NN(cmg_nn_gemm_bf16_splitk(dp, P0, u->dZT, P0, 1, kHeadC, ks, nsl, u->part, kHeadC, u->status, u->stream));
  NN(cmg_nn_sum_slices(u->part, nsl, h.gw, kHeadC, u->stream));
  NN(cmg_nn_colsum(dp, P0, 1, h.gb, u->stream));
  NN(cmg_nn_outer(dp, h.w, g[E0], P0, kHeadC, u->stream));
  cmg_status st;
  if ((st = conv_backward(u, D0, a[T0], a[E0], g[E0], g[T0], B)) != CMG_OK) return st;
  NN(cmg_nn_upsample_bwd(g[T0], g[E1], B, S / 2, S / 2, 32, u->stream));
  if ((st = conv_backward(u, D1, a[T1], a[E1], g[E1], g[T1], B)) != CMG_OK) return st;
  NN(cmg_nn_upsample_bwd(g[T1], g[E2], B, S / 4, S / 4, 64, u->stream));
  if ((st = conv_backward(u, D2, a[T2], a[E2], g[E2], g[T2], B)) != CMG_OK) return st;
  NN(cmg_nn_upsample_bwd(g[T2], g[B3], B, S / 8, S / 8, 64, u->stream));
  if ((st = conv_backward(u, C3B, a[A3], a[B3], g[B3], g[A3], B)) != CMG_OK) return st;
  if ((st = conv_backward(u, C3A, a[P3], a[A3], g[A3], g[P3], B)) != CMG_OK) return st;
  // s2 feeds the pooling and the skip into t2
  NN(cmg_nn_avgpool(g[P3], u->pool_tmp, B, S / 4, S / 4, 64, 1, u->stream));
  NN(cmg_nn_add(u->pool_tmp, g[T2], g[S2], pixels(u, B, 2) * 64, u->stream));
  if ((st = conv_backward(u, C2B, a[A2], a[S2], g[S2], g[A2], B)) != CMG_OK) return st;
  if ((st = conv_backward(u, C2A, a[P2], a[A2], g[A2], g[P2], B)) != CMG_OK) return st;
  NN(cmg_nn_avgpool(g[P2], u->pool_tmp, B, S / 2, S / 2, 64, 1, u->stream));
  NN(cmg_nn_add(u->pool_tmp, g[T1], g[S1], pixels(u, B, 1) * 64, u->stream));
  if ((st = conv_backward(u, C1B, a[A1], a[S1], g[S1], g[A1], B)) != CMG_OK) return st;
  if ((st = conv_backward(u, C1A, a[P1], a[A1], g[A1], g[P1], B)) != CMG_OK) return st;
  NN(cmg_nn_avgpool(g[P1], u->pool_tmp, B, S, S, 32, 1, u->stream));
  NN(cmg_nn_add(u->pool_tmp, g[T0], g[S0], pixels(u, B, 0) * 32, u->stream));
  if ((st = conv_backward(u, C0B, a[A0], a[S0], g[S0], g[A0], B)) != CMG_OK) return st;
  return conv_backward(u, C0A, u->x0, a[A0], g[A0], nullptr, B);
}

cmg_status cmg_unet_step(cmg_unet* u, float lr, float b1, float b2, float eps, float wd) {
  if (!u) return CMG_ERR_INVALID_ARG;
  if (!(lr >= 0.f && b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps > 0.f && wd >= 0.f))
    return fail(u, CMG_ERR_INVALID_ARG, "AdamW hyper-parameters out of range");
  ++u->step;
  for (int l = 0; l < kLayers; ++l) {
    Param& p = u->prm[l];
    NN(cmg_nn_adamw(p.w, p.gw, p.mw, p.vw, p.w16, (long long)p.rows * p.cols, lr, b1, b2, eps, wd, u->step,
                    u->stream));
    NN(cmg_nn_adamw(p.b, p.gb, p.mb, p.vb, nullptr, p.rows, lr, b1, b2, eps, 0.f, u->step, u->stream));
  }
  return CMG_OK;
}

int cmg_unet_num_params(const cmg_unet* u) { return u ? kLayers : 0; }
int cmg_unet_steps_taken(const cmg_unet* u) { return u ? u->step : -1; }

cmg_status cmg_unet_param_shape(const cmg_unet* u, int layer, int* rows, int* cols) {
  if (!u || !rows || !cols || layer < 0 || layer >= kLayers) return CMG_ERR_INVALID_ARG;
  *rows = u->prm[layer].rows;
  *cols = u->prm[layer].cols;
  return CMG_OK;
}

cmg_status cmg_unet_get(cmg_unet* u, int layer, int which, float* host) {
  if (!u || !host || layer < 0 || layer >= kLayers) return fail(u, CMG_ERR_INVALID_ARG, "bad layer or pointer");
  Param& p = u->prm[layer];
  if (which == CMG_UNET_W16) {
    // the BF16 weights the kernels use, widened to FP32
    std::vector<uint16_t> tmp((size_t)p.rows * p.cols);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), p.w16, tmp.size() * 2, cudaMemcpyDeviceToHost, u->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) return cuda_fail(u, e, "read of the BF16 weights");
    for (size_t i = 0; i < tmp.size(); ++i) {
      const uint32_t bits = (uint32_t)tmp[i] << 16;
      std::memcpy(host + i, &bits, 4);
    }
    return CMG_OK;
  }
  float* src = param_ptr(p, which);
  if (!src) return fail(u, CMG_ERR_INVALID_ARG, "unknown parameter array");
  cudaError_t e = cudaMemcpyAsync(host, src, param_elems(p, which) * 4, cudaMemcpyDeviceToHost, u->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  return e == cudaSuccess ? CMG_OK : cuda_fail(u, e, "parameter read");
}

cmg_status cmg_unet_set(cmg_unet* u, int layer, int which, const float* host) {
  if (!u || !host || layer < 0 || layer >= kLayers) return fail(u, CMG_ERR_INVALID_ARG, "bad layer or pointer");
  Param& p = u->prm[layer];
  float* dst = param_ptr(p, which);
  if (!dst) return fail(u, CMG_ERR_INVALID_ARG, "unknown parameter array");
  cudaError_t e = cudaMemcpyAsync(dst, host, param_elems(p, which) * 4, cudaMemcpyHostToDevice, u->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  if (e != cudaSuccess) return cuda_fail(u, e, "parameter write");
  if (which == CMG_UNET_W) NN(cmg_nn_to_bf16(p.w, p.w16, (long long)p.rows * p.cols, u->stream));
  return CMG_OK;
}

cmg_status cmg_unet_status(cmg_unet* u, int* host) {
  if (!u || !host) return CMG_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(host, u->status, sizeof(int), cudaMemcpyDeviceToHost, u->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  return e == cudaSuccess ? CMG_OK : cuda_fail(u, e, "status read");
}

cmg_status cmg_unet_save(cmg_unet* u, const char* path) {
  if (!u || !path) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) return cuda_fail(u, cudaGetLastError(), "sync before save");
  FILE* fh = std::fopen(path, "wb");
  if (!fh) return fail(u, CMG_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
  bool ok = std::fwrite(kMagic, 1, 8, fh) == 8;
  const int32_t head[4] = {kFormat, u->S, u->step, kLayers};
  ok = ok && std::fwrite(head, 4, 4, fh) == 4;
  ok = ok && std::fwrite(u->in_scale, 4, 2, fh) == 2 && std::fwrite(&u->out_scale, 8, 1, fh) == 1;
  std::vector<float> buf;
  const int arrays[] = {CMG_UNET_W, CMG_UNET_B, CMG_UNET_MW, CMG_UNET_VW, CMG_UNET_MB, CMG_UNET_VB};
  for (int l = 0; l < kLayers && ok; ++l) {
    Param& p = u->prm[l];
    const int32_t shape[2] = {p.rows, p.cols};
    ok = std::fwrite(shape, 4, 2, fh) == 2;
    for (int w : arrays) {
      if (!ok) break;
      buf.resize(param_elems(p, w));
      if (cudaMemcpy(buf.data(), param_ptr(p, w), buf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        (void)cudaGetLastError();
        ok = false;
        break;
      }
      ok = std::fwrite(buf.data(), 4, buf.size(), fh) == buf.size();
    }
  }
  ok = (std::fclose(fh) == 0) && ok;
  return ok ? CMG_OK : fail(u, CMG_ERR_CUDA, std::string("checkpoint write failed: ") + path);
}

cmg_status cmg_unet_load(cmg_unet* u, const char* path) {
  if (!u || !path) return fail(u, CMG_ERR_INVALID_ARG, "null pointer");
  FILE* fh = std::fopen(path, "rb");
  if (!fh) return fail(u, CMG_ERR_INVALID_ARG, std::string("cannot open: ") + path);
  char magic[8];
  int32_t head[4];
  float in_scale[2];
  double out_scale;
  bool ok = std::fread(magic, 1, 8, fh) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(head, 4, 4, fh) == 4 && head[0] == kFormat && head[3] == kLayers &&
            std::fread(in_scale, 4, 2, fh) == 2 && std::fread(&out_scale, 8, 1, fh) == 1;
  if (!ok) {
    std::fclose(fh);
    return fail(u, CMG_ERR_INVALID_ARG, "not a checkpoint of this network (magic, format or layer count)");
  }
  // read everything to the host first, so a short or mismatched file leaves the network unchanged
  const int arrays[] = {CMG_UNET_W, CMG_UNET_B, CMG_UNET_MW, CMG_UNET_VW, CMG_UNET_MB, CMG_UNET_VB};
  std::vector<std::vector<float>> data;
  for (int l = 0; l < kLayers && ok; ++l) {
    Param& p = u->prm[l];
    int32_t shape[2];
    ok = std::fread(shape, 4, 2, fh) == 2 && shape[0] == p.rows && shape[1] == p.cols;
    for (int w : arrays) {
      if (!ok) break;
      data.emplace_back(param_elems(p, w));
      ok = std::fread(data.back().data(), 4, data.back().size(), fh) == data.back().size();
    }
  }
  std::fclose(fh);
  if (!ok) return fail(u, CMG_ERR_INVALID_ARG, "checkpoint truncated or layer shapes differ");
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) return cuda_fail(u, cudaGetLastError(), "sync before load");
  size_t k = 0;
  for (int l = 0; l < kLayers; ++l) {
    Param& p = u->prm[l];
    for (int w : arrays) {
      const cudaError_t e = cudaMemcpy(param_ptr(p, w), data[k].data(), data[k].size() * 4, cudaMemcpyHostToDevice);
      ++k;
      if (e != cudaSuccess) return cuda_fail(u, e, "checkpoint upload");
    }
    NN(cmg_nn_to_bf16(p.w, p.w16, (long long)p.rows * p.cols, u->stream));
  }
  u->step = head[2];
  u->in_scale[0] = in_scale[0];
  u->in_scale[1] = in_scale[1];
  u->out_scale = out_scale;
  return CMG_OK;
}

}  // extern "C"
