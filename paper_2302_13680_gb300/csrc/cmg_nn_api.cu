// C ABI of the warm-start network kernels (include/cmg.h, "learned warm
// start" section).
#include <cstdint>

#include "cmg_internal.h"

using namespace cmg;

namespace {
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

extern "C" cmg_status cmg_nn_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, int M, int N, int K,
                                       const float* bias, int relu, float* C32, void* C16, int ldc, int* status,
                                       void* stream) {
  if (!A || !B || !status || (!C32 && !C16)) return CMG_ERR_INVALID_ARG;
  if (M < 1 || N < 1 || K < 8 || K % 8 != 0 || ldc < N || lda < K || ldb < K || lda % 8 || ldb % 8)
    return CMG_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B)) return CMG_ERR_INVALID_ARG;
  const cudaError_t e = launch_gemm_bf16_tn(A, lda, B, ldb, M, N, K, bias, relu, C32, C16, ldc, status,
                                            static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_nn_conv3x3_bf16(const void* X, int B, int H, int W, int C, const void* Wt, int Cout,
                                          const float* bias, int relu, void* Y, int* status, void* stream) {
  if (!X || !Wt || !Y || !status || B < 1 || H < 1 || W < 1 || C < 1 || Cout < 1) return CMG_ERR_INVALID_ARG;
  if (!aligned16(X) || !aligned16(Wt)) return CMG_ERR_INVALID_ARG;
  const cudaError_t e = launch_conv3x3_bf16(X, B, H, W, C, Wt, Cout, bias, relu, Y, status,
                                            static_cast<cudaStream_t>(stream));
  if (e == cudaErrorNotSupported) return CMG_ERR_UNSUPPORTED;
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_nn_gemm_bf16_splitk(const void* A, long long lda, const void* B, long long ldb, int M,
                                              int N, int Kslice, int ksplit, float* partials, int ldc, int* status,
                                              void* stream) {
  if (!A || !B || !status || !partials) return CMG_ERR_INVALID_ARG;
  if (M < 1 || N < 1 || Kslice < 8 || Kslice % 8 || ksplit < 1 || ksplit > 65535 || ldc < N || lda % 8 || ldb % 8 ||
      lda < (long long)Kslice * ksplit || ldb < (long long)Kslice * ksplit)
    return CMG_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B)) return CMG_ERR_INVALID_ARG;
  const cudaError_t e = launch_gemm_bf16_tn(A, lda, B, ldb, M, N, Kslice, nullptr, 0, partials, nullptr, ldc, status,
                                            static_cast<cudaStream_t>(stream), ksplit);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  return CMG_OK;
}

extern "C" cmg_status cmg_nn_set_wait_limit(long long polls) {
  if (polls < 0) return CMG_ERR_INVALID_ARG;
  set_gemm_wait_limit(polls);
  return CMG_OK;
}
